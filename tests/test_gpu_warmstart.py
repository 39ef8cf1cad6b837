"""What the trained warm-start network gains (GPU).

The first 12 held-out sphere packs (the evaluation seed, never trained on;
every fluid fraction from 10 to 60 %) are solved to residual < 1e-6 three ways with FP32-deviation storage and the period-2
filter: from rest, from the trained network's prediction, and from the
prediction of the same network with untrained weights.  The LBM residual
alone declares convergence in every case; a run that does not converge within
60,000 steps counts 60,000.  The trained start must take fewer steps in total
than the start from rest and than the untrained network, and every
permeability where both converged must agree with the start from rest within
1e-3.
"""
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def nn():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1703_08015_gb300 import nn as nn_mod

    return nn_mod


def test_committed_weights_load(nn):
    assert os.path.exists(nn.WEIGHTS), "trained warm-start weights are missing"
    net = nn.UNet.load(nn.WEIGHTS)
    assert net.n_params > 1_000_000
    assert net.meta["a_rho"] > 0 and net.meta["a_u"] > 0


def test_trained_warm_start_gains_over_rest_and_untrained(nn):
    from paper_1703_08015_gb300 import lbm

    tau, force = 0.6, 1e-6
    nu = (tau - 0.5) / 3.0
    trained = nn.UNet.load(nn.WEIGHTS)
    untrained = nn.UNet(trained.chans, trained.cin, trained.cout, trained.wrap, seed=123)
    untrained.meta = dict(trained.meta)
    held, _ = nn.sample_geometries(12, seed=2)  # every pack, no fluid-fraction filter
    cap = 60000
    steps = {"rest": 0, "trained": 0, "untrained": 0}
    pred_err, converged = [], 0
    for m in held:
        kw = dict(tau=tau, force=force, storage=lbm.LBM_STORE_F32S, max_steps=cap, filter_period2=True)
        rest = nn.time_to_steady(m, None, **kw)
        warm = nn.time_to_steady(m, trained, **kw)
        cold = nn.time_to_steady(m, untrained, **kw)
        # a run that does not converge within the cap counts the cap
        steps["rest"] += rest["steps"] if rest["converged"] else cap
        steps["trained"] += warm["steps"] if warm["converged"] else cap
        steps["untrained"] += cold["steps"] if cold["converged"] else cap
        if rest["converged"] and warm["converged"]:
            converged += 1
            assert abs(warm["permeability"] / rest["permeability"] - 1) < 1e-3
            _, u_pred = nn.predict_fields(trained, m, force, nu)
            fl = m.astype(bool)
            d = u_pred[:, fl] - rest["u"]
            pred_err.append(np.sqrt(np.sum(d * d) / np.sum(rest["u"] ** 2)))
    assert converged >= 9, converged
    assert steps["trained"] < steps["rest"], steps
    assert steps["trained"] < steps["untrained"], steps
    assert np.median(pred_err) < 0.5, pred_err
