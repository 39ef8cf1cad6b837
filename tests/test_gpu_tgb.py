"""GPU tests of the single-copy ghost-buffer layout (TGB, Sec. 3.1, Fig. 4).

The TGB step performs the same per-node update as the two-copy (T2C) step and
only moves data differently, so after any number of steps its state must
equal the T2C state bit for bit in every storage form, and the FP64 form must
meet the 1e-12 bar against the oracle.
"""
import numpy as np
import pytest

from paper_1703_08015_gb300 import geometry as geo
from paper_1703_08015_gb300 import lbm

pytestmark = pytest.mark.gpu
TOL = 1e-12
T2C, TGB = lbm.LBM_LAYOUT_T2C, lbm.LBM_LAYOUT_TGB


def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _cases():
    m2, _ = geo.circles_2d(48, 35, seed=11, r_min=2, r_max=5, max_attempts=2000)
    m2r = geo.random_mask(64, 40, 1, fluid=0.75, seed=14)
    m3, _ = geo.sphere_pack_3d(shape=(24, 22, 18), seed=12, r_min=2, r_max=4, target_fluid=0.45)
    m3b, _ = geo.tube_tree_3d(shape=(32, 20, 19), seed=13, r_min=1.5, r_max=3.0, target_fluid=0.12)
    return [
        ("d2q9_a16_circles", m2, 9, 16, (1, 0, 0), 0.8, (1e-5, 2e-6, 0), 300, 0),
        ("d2q9_a8_random", m2r, 9, 8, (1, 1, 0), 0.7, (3e-6, 0, 0), 200, 0),
        ("d2q9_a32_circles", m2, 9, 32, (0, 0, 0), 0.9, (1e-5, 0, 0), 150, 0),
        ("d3q19_a4_spheres", m3, 19, 4, (1, 0, 0), 0.6, (1e-5, 0, 3e-6), 300, 0),
        ("d3q19_a8_tubes", m3b, 19, 8, (1, 0, 0), 0.6, (1e-5, 0, 0), 200, 0),
        ("d3q19_a4_incompressible", m3, 19, 4, (1, 0, 0), 0.7, (1e-5, 0, 0), 200, 1),
    ]


def _run(mask, lattice, a, per, tau, F, steps, model=0, layout=T2C, storage=lbm.LBM_STORE_F64,
         arith=lbm.LBM_ARITH_AUTO):
    s = lbm.Solver(mask, lattice, a, per, tau, F, model=model, storage=storage, arith=arith, layout=layout)
    try:
        s.step(steps)
        return s.export_pdfs(), s.stats()[0]
    finally:
        s.close()


def max_rel(gpu, ref, mask):
    fl = np.asarray(mask).astype(bool)
    g, r = gpu[:, fl], ref[:, fl]
    assert np.all(np.isfinite(g))
    return float(np.max(np.abs(g - r) / np.abs(r)))


@pytest.mark.parametrize("arith", [lbm.LBM_ARITH_FF, lbm.LBM_ARITH_F64], ids=["ff", "f64"])
@pytest.mark.parametrize("case", _cases(), ids=lambda c: c[0])
def test_tgb_parity_with_oracle(oracle, case, arith):
    _cuda()
    name, mask, lattice, a, per, tau, F, steps, model = case
    gpu, _ = _run(mask, lattice, a, per, tau, F, steps, model, TGB, arith=arith)
    if lattice == 9:
        mask2 = mask if mask.ndim == 3 else mask[None]
    else:
        mask2 = mask
    ref = oracle.run(lattice, mask2, per, tau, F, oracle.init(lattice, mask2, model=model), steps, model=model)
    assert max_rel(gpu.reshape(ref.shape), ref, mask2) <= TOL, name


@pytest.mark.parametrize("storage", [lbm.LBM_STORE_F64, lbm.LBM_STORE_F32, lbm.LBM_STORE_F32S, lbm.LBM_STORE_F16S],
                         ids=["f64", "f32", "f32s", "f16s"])
@pytest.mark.parametrize("case", _cases()[:5], ids=lambda c: c[0])
def test_tgb_equals_t2c_bit_for_bit(case, storage):
    _cuda()
    name, mask, lattice, a, per, tau, F, steps, model = case
    g1, s1 = _run(mask, lattice, a, per, tau, F, steps, model, T2C, storage)
    g2, s2 = _run(mask, lattice, a, per, tau, F, steps, model, TGB, storage)
    fl = np.asarray(mask if mask.ndim == 3 else mask[None]).astype(bool).reshape(-1)
    assert np.array_equal(g1.reshape(g1.shape[0], -1)[:, fl], g2.reshape(g2.shape[0], -1)[:, fl]), name
    assert s1.mass == s2.mass and list(s1.momentum) == list(s2.momentum)


def test_tgb_d2q9_circles_128_full(oracle):
    """128^2 circles, 16^2 tiles, tau 0.8, F = 1e-6, 1000 steps, every node."""
    _cuda()
    mask, params, _ = geo.workload("d2q9_circles_128")
    gpu, _ = _run(mask, 9, 16, params["periodic"], params["tau"], params["force"], params["steps"], 0, TGB)
    m = mask if mask.ndim == 3 else mask[None]
    ref = oracle.run(9, m, params["periodic"], params["tau"], params["force"], oracle.init(9, m), params["steps"])
    assert max_rel(gpu.reshape(ref.shape), ref, m) <= TOL


def test_tgb_checkpoint_batch_and_memory():
    _cuda()
    m3, _ = geo.sphere_pack_3d(shape=(24, 22, 18), seed=12, r_min=2, r_max=4, target_fluid=0.45)
    per, tau, F = (1, 0, 0), 0.6, (1e-5, 0, 0)
    # checkpoint: export at 100, import into a fresh context, continue to 250 == straight 250
    s = lbm.Solver(m3, 19, 4, per, tau, F, layout=TGB)
    try:
        s.step(100)
        snap = s.export_pdfs()
        s.step(150)
        straight = s.export_pdfs()
        with pytest.raises(lbm.LBMError):
            s.filter_period2()  # needs two copies
    finally:
        s.close()
    r = lbm.Solver(m3, 19, 4, per, tau, F, layout=TGB)
    try:
        r.import_pdfs(snap, 100)
        r.step(150)
        resumed = r.export_pdfs()
    finally:
        r.close()
    fl = m3.astype(bool)
    assert np.array_equal(straight[:, fl], resumed[:, fl])
    # a batch in the TGB layout equals the samples run one by one
    m4, _ = geo.sphere_pack_3d(shape=(16, 20, 12), seed=21, r_min=2, r_max=4, target_fluid=0.5)
    b = lbm.BatchSolver([m3, m4], 19, 4, per, tau, F, storage=lbm.LBM_STORE_F32S, layout=TGB)
    try:
        b.step(120)
        got = [b.export_pdfs(0), b.export_pdfs(1)]
    finally:
        b.close()
    for k, m in enumerate([m3, m4]):
        want, _ = _run(m, 19, 4, per, tau, F, 120, 0, T2C, lbm.LBM_STORE_F32S)
        assert np.array_equal(got[k][:, m.astype(bool)], want[:, m.astype(bool)])
    # memory: for D2Q9 with 16^2 tiles the ghost sets are far smaller than a second copy
    mask, params, _ = geo.workload("d2q9_circles_128")
    t2c = lbm.lbm_build_tilemap(lbm.make_params(9, mask.shape, 16, params["periodic"], layout=T2C), mask)[0]
    tgb = lbm.lbm_build_tilemap(lbm.make_params(9, mask.shape, 16, params["periodic"], layout=TGB), mask)[0]
    assert t2c.ghost_bytes == 0
    assert tgb.ghost_bytes == 2 * tgb.n_ftiles * (4 * 16 + 4 * 31) * 8
    assert tgb.pdf_bytes + tgb.ghost_bytes < 0.7 * 2 * t2c.pdf_bytes
