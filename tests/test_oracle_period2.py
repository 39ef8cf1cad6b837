"""The slowly damped period-2 mode of the BGK step with halfway bounce-back,
and the two-state mean that removes it (oracle only; the GPU filter is
checked against these states in tests/test_gpu_parity.py).

On a porous geometry driven by a body force, the step has an eigenmode whose
factor per step is close to -1: late in a run from rest the state flips by a
staggered velocity pattern every step, while two steps apart it barely moves.
A residual over an even number of steps cannot see the flip.  The mean of two
consecutive states cancels the mode and keeps the slowly varying part, so it
lands much closer to the steady state than either state.
"""
import numpy as np
import pytest

import oracle as O
from paper_1703_08015_gb300 import geometry as geo

TAU, F, PER = 0.6, (1e-6, 0.0, 0.0), (1, 0, 0)


@pytest.fixture(scope="module")
def pack():
    mask, _ = geo.sphere_pack_3d(20, seed=11, r_min=2.5, r_max=5.0, target_fluid=0.45)
    return mask


def _u(mask, f):
    return O.moments(19, mask, PER, F, f)[1]


def test_period2_mode_and_two_state_mean(pack):
    mask = pack
    fl = mask.astype(bool)
    norm = lambda v: float(np.sqrt(np.sum(v[:, fl] ** 2)))
    f = O.run(19, mask, PER, TAU, F, O.init(19, mask), 3000)
    f1 = O.run(19, mask, PER, TAU, F, f, 1)
    f2 = O.run(19, mask, PER, TAU, F, f1, 1)
    u0, u1, u2 = _u(mask, f), _u(mask, f1), _u(mask, f2)
    # the flip: one step apart the velocity changes far more than two steps apart
    assert norm(u1 - u0) > 1e3 * norm(u2 - u0)
    # ... and it is a staggered pattern: neighbours along x move in opposite directions
    d = (u1 - u0)[0]
    both = fl & np.roll(fl, 1, 2)
    assert np.corrcoef(d[both], np.roll(d, 1, 2)[both])[0, 1] < -0.9
    # reference steady state: mean of two states, then many more steps, repeated
    g = f
    for _ in range(3):
        g = 0.5 * (g + O.run(19, mask, PER, TAU, F, g, 1))
        g = O.run(19, mask, PER, TAU, F, g, 2000)
    ref = _u(mask, g)
    err_plain = norm(u0 - ref)
    err_mean = norm(_u(mask, 0.5 * (f + f1)) - ref)
    assert err_mean < 1e-2 * err_plain
    # the mean does not move the fixed point: the reference state is a fixed point of mean-then-step
    g2 = 0.5 * (g + O.run(19, mask, PER, TAU, F, g, 1))
    assert norm(_u(mask, g2) - ref) < 1e-9 * norm(ref)
