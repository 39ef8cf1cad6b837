"""Pins of the oracle's lattice, equilibrium (Eq. 3 / Eq. 4) and collision
(Eq. 2 + forcing) against closed-form moment identities.

The paper does not print weights or link order, so these pin them: a wrong
weight, a wrong sign in a link, a wrong coefficient in Eq. 3 (3, 4.5, 1.5) or
a wrong forcing prefactor each break one of the identities below.
"""
import numpy as np
import pytest

LATTICES = [9, 19]


@pytest.mark.parametrize("lat", LATTICES)
def test_isotropy(oracle, lat):
    L = oracle.Lattice(lat)
    c = L.c.astype(np.float64)
    w = L.w
    d = L.d
    I = np.eye(3)
    I[d:, d:] = 0.0
    assert L.q == lat
    assert np.all(L.c[0] == 0)
    assert len({tuple(v) for v in L.c}) == L.q
    assert abs(w.sum() - 1.0) < 1e-15
    assert np.allclose(np.einsum("i,ia->a", w, c), 0.0, atol=1e-16)
    assert np.allclose(np.einsum("i,ia,ib->ab", w, c, c), I / 3.0, atol=1e-15)
    assert np.allclose(np.einsum("i,ia,ib,ic->abc", w, c, c, c), 0.0, atol=1e-16)
    four = np.einsum("i,ia,ib,ic,id->abcd", w, c, c, c, c)
    iso = (np.einsum("ab,cd->abcd", I, I) + np.einsum("ac,bd->abcd", I, I)
           + np.einsum("ad,bc->abcd", I, I)) / 9.0
    assert np.allclose(four, iso, atol=1e-15)
    # opposite links
    for i in range(L.q):
        assert np.all(L.c[L.opp[i]] == -L.c[i])
        assert w[L.opp[i]] == w[i]
    assert np.all(L.c[:, d:] == 0)


@pytest.mark.parametrize("lat", LATTICES)
@pytest.mark.parametrize("model", [0, 1])
def test_equilibrium_moments(oracle, lat, model):
    L = oracle.Lattice(lat)
    rng = np.random.default_rng(5)
    c = L.c.astype(np.float64)
    for _ in range(20):
        rho = rng.uniform(0.9, 1.1)
        u = np.zeros(3)
        u[: L.d] = rng.uniform(-0.1, 0.1, L.d)
        feq = oracle.equilibrium(lat, rho, u, model=model)
        assert feq.sum() == pytest.approx(rho, rel=1e-15)
        if model == 0:  # Eq. 3 with Eq. 5: j = rho u, Pi = rho/3 I + rho u u
            j, Pi = rho * u, rho / 3.0 * np.eye(3) + rho * np.outer(u, u)
        else:           # Eq. 4 with Eq. 6: j = u, Pi = rho/3 I + u u
            j, Pi = u, rho / 3.0 * np.eye(3) + np.outer(u, u)
        Pi[L.d:, :] = 0.0
        Pi[:, L.d:] = 0.0
        assert np.allclose(c.T @ feq, j, rtol=0, atol=1e-16)
        assert np.allclose(np.einsum("i,ia,ib->ab", feq, c, c), Pi, rtol=0, atol=2e-16)


@pytest.mark.parametrize("lat", LATTICES)
@pytest.mark.parametrize("model", [0, 1])
def test_collision_moments(oracle, lat, model):
    """Collision keeps mass, adds exactly F of momentum, and relaxes the
    momentum flux: Pi* = (1-w) Pi + w Pi_eq + (1 - w/2)(u F + F u), w = 1/tau."""
    L = oracle.Lattice(lat)
    c = L.c.astype(np.float64)
    rng = np.random.default_rng(11)
    for tau in (0.55, 0.6, 0.8, 1.7):
        for _ in range(5):
            F = np.zeros(3)
            F[: L.d] = rng.uniform(-1e-3, 1e-3, L.d)
            rho0 = rng.uniform(0.95, 1.05)
            u0 = np.zeros(3)
            u0[: L.d] = rng.uniform(-0.05, 0.05, L.d)
            f = oracle.equilibrium(lat, rho0, u0, model=model) * (1 + rng.uniform(-0.02, 0.02, L.q))
            fs = oracle.collide(lat, f, tau, F, model=model)
            rho = f.sum()
            j = c.T @ f
            uh = (j + 0.5 * F) / rho if model == 0 else j + 0.5 * F
            assert fs.sum() == pytest.approx(rho, rel=1e-15)
            assert np.allclose(c.T @ fs, j + F, rtol=0, atol=5e-16)
            Pi = np.einsum("i,ia,ib->ab", f, c, c)
            Pieq = rho / 3.0 * np.eye(3) + (rho if model == 0 else 1.0) * np.outer(uh, uh)
            Pieq[L.d:, :] = 0.0
            Pieq[:, L.d:] = 0.0
            w = 1.0 / tau
            expect = (1 - w) * Pi + w * Pieq + (1 - 0.5 * w) * (np.outer(uh, F) + np.outer(F, uh))
            assert np.allclose(np.einsum("i,ia,ib->ab", fs, c, c), expect, rtol=0, atol=2e-15)


@pytest.mark.parametrize("lat", LATTICES)
def test_equilibrium_is_fixed_point(oracle, lat):
    """Without force, the equilibrium of Eq. 3 is left unchanged by collision."""
    rng = np.random.default_rng(2)
    L = oracle.Lattice(lat)
    u = np.zeros(3)
    u[: L.d] = rng.uniform(-0.05, 0.05, L.d)
    feq = oracle.equilibrium(lat, 1.02, u)
    out = oracle.collide(lat, feq, 0.7, (0.0, 0.0, 0.0))
    assert np.allclose(out, feq, rtol=1e-14, atol=0)
