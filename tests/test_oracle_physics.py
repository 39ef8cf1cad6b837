"""Pins of the oracle's streaming, bounce-back, forcing and time stepping.

* streaming direction and wrap: brute force on tiny periodic boxes, and the
  gather rebuilt with numpy.roll (a library routine, not the oracle's code);
* bounce-back (Sec. 3.2 propagates only between non-solid nodes): a single
  marked value must come back to its own node in the opposite direction;
* exact invariants: total mass under bounce-back + periodic edges, and the
  uniform-force closed form u(t) = (t + 1/2) F / rho0;
* closed-form flows: plane Poiseuille (exact at tau = 1/2 + sqrt(3/16) with
  halfway walls) and the square-duct series solution, second order in h.
"""
import numpy as np
import pytest

from paper_1703_08015_gb300 import geometry as geo

MAGIC_TAU = 0.5 + np.sqrt(3.0 / 16.0)


def _rest_field(oracle, lat, mask):
    return oracle.init(lat, mask)


@pytest.mark.parametrize("lat,shape", [(9, (1, 6, 7)), (19, (5, 6, 7))])
def test_streaming_single_value(oracle, lat, shape):
    """A marked post-collision value f*_i(x0) is pulled by node x0 + c_i only."""
    L = oracle.Lattice(lat)
    mask = np.ones(shape, np.uint8)
    nz, ny, nx = shape
    x0 = np.array([2, 3, 1 if lat == 19 else 0])
    delta = 1e-3
    for i in range(L.q):
        f = _rest_field(oracle, lat, mask)
        f[i, x0[2], x0[1], x0[0]] += delta
        rho, u = oracle.moments(lat, mask, (1, 1, 1), (0, 0, 0), f)
        tgt = (x0 + L.c[i]) % np.array([nx, ny, nz])
        moved = np.abs(rho - 1.0) > 1e-9
        assert np.count_nonzero(moved) == 1 and moved[tgt[2], tgt[1], tgt[0]]
        assert rho[tgt[2], tgt[1], tgt[0]] == pytest.approx(1 + delta, rel=1e-15)
        j = u[:, tgt[2], tgt[1], tgt[0]] * rho[tgt[2], tgt[1], tgt[0]]
        assert np.allclose(j, L.c[i] * delta, atol=1e-17)


@pytest.mark.parametrize("lat,shape", [(9, (1, 5, 8)), (19, (3, 4, 5))])
def test_gather_matches_numpy_roll(oracle, lat, shape):
    """Fully periodic all-fluid box: the pulled value along c_i is np.roll(f_i, c_i)."""
    L = oracle.Lattice(lat)
    rng = np.random.default_rng(3)
    mask = np.ones(shape, np.uint8)
    f = rng.uniform(0.01, 0.2, (L.q,) + shape)
    F = (1e-4, -2e-4, 3e-4)
    pulled = np.stack([np.roll(f[i], shift=(L.c[i][2], L.c[i][1], L.c[i][0]), axis=(0, 1, 2))
                       for i in range(L.q)])
    rho_np = pulled.sum(0)
    j_np = np.einsum("ia,izyx->azyx", L.c.astype(np.float64), pulled)
    Fv = np.array(F)
    if L.d == 2:
        Fv[2] = 0.0
    u_np = (j_np + 0.5 * Fv[:, None, None, None]) / rho_np
    rho, u = oracle.moments(lat, mask, (1, 1, 1), Fv, f)
    assert np.allclose(rho, rho_np, rtol=1e-14, atol=0)
    assert np.allclose(u, u_np, rtol=1e-12, atol=1e-17)
    # a full step is the node-local collision of the pulled values
    out = oracle.step(lat, mask, (1, 1, 1), 0.7, Fv, f)
    for (z, y, x) in [(0, 0, 0), (shape[0] - 1, 2, 3), (1 % shape[0], 1, 4)]:
        ref = oracle.collide(lat, pulled[:, z, y, x], 0.7, Fv)
        assert np.array_equal(out[:, z, y, x], ref)


@pytest.mark.parametrize("lat", [9, 19])
def test_bounce_back_single_value(oracle, lat):
    """A value aimed at a solid node (or a wall beyond a non-periodic edge)
    returns to its own node in the opposite direction."""
    L = oracle.Lattice(lat)
    shape = (1, 6, 7) if lat == 9 else (5, 6, 7)
    nz, ny, nx = shape
    mask = np.ones(shape, np.uint8)
    solid = (3, 3, 2) if lat == 19 else (0, 3, 2)  # (z, y, x)
    mask[solid] = 0
    delta = 1e-3
    sx = np.array([solid[2], solid[1], solid[0]])
    for i in range(1, L.q):
        x0 = sx - L.c[i]
        f = _rest_field(oracle, lat, mask)
        f[i, x0[2], x0[1], x0[0]] += delta
        rho, u = oracle.moments(lat, mask, (1, 1, 1), (0, 0, 0), f)
        assert rho[x0[2], x0[1], x0[0]] == pytest.approx(1 + delta, rel=1e-15)
        j = u[:, x0[2], x0[1], x0[0]] * rho[x0[2], x0[1], x0[0]]
        assert np.allclose(j, -L.c[i] * delta, atol=1e-17)
        fl = mask.astype(bool)
        assert np.isnan(rho[solid])
        assert np.count_nonzero(np.abs(rho[fl] - 1.0) > 1e-9) == 1
    # walls beyond non-periodic y: a value leaving through y = ny-1 comes back
    mask = np.ones(shape, np.uint8)
    i_up = [k for k in range(L.q) if tuple(L.c[k]) == (0, 1, 0)][0]
    x0 = (0, ny - 1, 3)  # (z, y, x)
    f = _rest_field(oracle, lat, mask)
    f[i_up][x0] += delta
    rho, u = oracle.moments(lat, mask, (1, 0, 1), (0, 0, 0), f)
    assert rho[x0] == pytest.approx(1 + delta, rel=1e-15)
    assert u[1][x0] * rho[x0] == pytest.approx(-delta, rel=1e-12)


@pytest.mark.parametrize("lat", [9, 19])
def test_mass_conservation(oracle, lat):
    if lat == 9:
        mask, _ = geo.circles_2d(48, 32, seed=4, max_attempts=3000)
        per = (1, 0, 0)
    else:
        mask, _ = geo.sphere_pack_3d(shape=(24, 20, 16), seed=4, r_min=2, r_max=5, target_fluid=0.5)
        per = (1, 0, 1)
    f = oracle.init(lat, mask)
    m0 = oracle.total_mass(lat, mask, f)
    f = oracle.run(lat, mask, per, 0.6, (2e-5, 1e-5, 0.0), f, 300)
    m1 = oracle.total_mass(lat, mask, f)
    assert abs(m1 - m0) / m0 < 1e-13
    rho, u = oracle.moments(lat, mask, per, (2e-5, 1e-5, 0.0), f)
    assert np.nanmax(np.abs(u)) > 1e-5  # the force did drive a flow


@pytest.mark.parametrize("lat,shape", [(9, (1, 8, 8)), (19, (4, 4, 4))])
@pytest.mark.parametrize("model", [0, 1])
def test_uniform_force_closed_form(oracle, lat, shape, model):
    """No walls: every step adds exactly F of momentum, so u(t) = (t + 1/2) F / rho0."""
    mask = np.ones(shape, np.uint8)
    F = np.array([1e-5, -3e-6, 2e-6])
    if lat == 9:
        F[2] = 0.0
    f = oracle.init(lat, mask, model=model)
    for t in (0, 1, 7, 40):
        if t:
            f = oracle.run(lat, mask, (1, 1, 1), 0.8, F, f, t - (0 if t == 1 else prev),
                           model=model)
        prev = t
        rho, u = oracle.moments(lat, mask, (1, 1, 1), F, f, model=model)
        assert np.allclose(rho, 1.0, rtol=0, atol=1e-14)
        expect = (t + 0.5) * F
        # j is a sum of O(1) PDFs, so its rounding error is absolute (~1e-16)
        assert np.allclose(u.reshape(3, -1).T, expect, rtol=0, atol=5e-16)


def _poiseuille(oracle, H, tau, steps):
    mask = geo.channel_2d(1, H)
    F = (1e-6, 0.0, 0.0)
    f = oracle.run(9, mask, (1, 0, 0), tau, F, oracle.init(9, mask), steps, nthreads=1)
    rho, u = oracle.moments(9, mask, (1, 0, 0), F, f)
    nu = (tau - 0.5) / 3.0
    y = np.arange(H)
    exact = F[0] / (2 * nu) * (y + 0.5) * (H - 0.5 - y)
    return u[0, 0, :, 0], exact, nu


def test_poiseuille_exact_at_magic_tau(oracle):
    ux, exact, nu = _poiseuille(oracle, 32, MAGIC_TAU, 25000)
    assert np.max(np.abs(ux - exact)) / exact.max() < 1e-10
    d2 = ux[2:] - 2 * ux[1:-1] + ux[:-2]
    assert np.allclose(d2, -1e-6 / nu, rtol=1e-9)


def test_poiseuille_second_order_slip(oracle):
    errs = []
    for H in (8, 16):
        ux, exact, nu = _poiseuille(oracle, H, 0.8, 8000)
        d2 = ux[2:] - 2 * ux[1:-1] + ux[:-2]
        assert np.allclose(d2, -1e-6 / nu, rtol=1e-8)  # still exactly parabolic
        errs.append(np.max(np.abs(ux - exact)) / exact.max())
    assert 1e-5 < errs[1] < errs[0]
    assert errs[0] / errs[1] == pytest.approx(4.0, rel=0.05)


def _duct_exact(side, F, nu, nterms=401):
    b = side / 2.0
    cc = np.arange(side) - (side - 1) / 2.0
    Y, Z = np.meshgrid(cc, cc, indexing="ij")
    u = np.zeros_like(Y)
    for n in range(1, nterms, 2):
        u += ((-1) ** ((n - 1) // 2) / n ** 3
              * (1 - np.cosh(n * np.pi * Z / (2 * b)) / np.cosh(n * np.pi / 2))
              * np.cos(n * np.pi * Y / (2 * b)))
    return (16 * b * b * F / (nu * np.pi ** 3) * u).T  # -> [z, y]


def test_square_duct_series(oracle):
    """Rectangular-duct series solution (textbook), side 2b with walls halfway
    outside the last node rows: L2 error <= 1e-3 at side 16, second order."""
    errs = []
    for side in (8, 16):
        mask = geo.duct_3d(1, side)
        F = (1e-6, 0.0, 0.0)
        f = oracle.run(19, mask, (1, 0, 0), MAGIC_TAU, F, oracle.init(19, mask), 12 * side * side)
        rho, u = oracle.moments(19, mask, (1, 0, 0), F, f)
        ex = _duct_exact(side, F[0], (MAGIC_TAU - 0.5) / 3.0)
        errs.append(np.sqrt(np.sum((u[0, :, :, 0] - ex) ** 2) / np.sum(ex ** 2)))
    assert errs[1] <= 1e-3
    assert errs[0] / errs[1] > 3.5


def test_step_nodes_matches_step(oracle):
    mask, _ = geo.sphere_pack_3d(shape=(12, 10, 8), seed=9, r_min=2, r_max=3, target_fluid=0.6)
    per = (1, 0, 0)
    F = (1e-4, 0, 0)
    f = oracle.run(19, mask, per, 0.6, F, oracle.init(19, mask), 20)
    full = oracle.step(19, mask, per, 0.6, F, f)
    nodes = np.flatnonzero(mask.reshape(-1))[::7]
    part = oracle.step_nodes(19, mask, per, 0.6, F, f, nodes)
    assert np.array_equal(part, full.reshape(19, -1)[:, nodes].T)
