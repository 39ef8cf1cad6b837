"""Pins of the FP64 reference of the warm-start network's operations."""
import numpy as np
import pytest
from scipy import ndimage

from oracle import nn_ref as R


def test_conv_matches_scipy_correlate():
    rng = np.random.default_rng(0)
    x = rng.normal(size=(1, 5, 6, 7, 1))
    w = rng.normal(size=(27, 1, 1))
    k = w[:, 0, 0].reshape(3, 3, 3)  # k[dz, dy, dx]
    ref = ndimage.correlate(x[0, :, :, :, 0], k, mode="constant", cval=0.0)
    assert np.allclose(R.conv3d(x, w)[0, :, :, :, 0], ref, rtol=1e-12, atol=1e-12)


def test_conv_adjoint_identities():
    rng = np.random.default_rng(1)
    x = rng.normal(size=(2, 4, 5, 6, 3))
    w = rng.normal(size=(27, 3, 4))
    dy = rng.normal(size=(2, 4, 5, 6, 4))
    # <conv(x), dy> = <x, conv^T(dy)> = <w, dW(x, dy)>
    lhs = np.sum(R.conv3d(x, w) * dy)
    assert np.sum(x * R.conv3d_bwd_data(dy, w)) == pytest.approx(lhs, rel=1e-12)
    dw, db = R.conv3d_bwd_weight(x, dy)
    assert np.sum(w * dw) == pytest.approx(lhs, rel=1e-12)
    assert np.allclose(db, dy.sum(axis=(0, 1, 2, 3)))


def test_conv_gradients_by_finite_differences():
    rng = np.random.default_rng(2)
    x = rng.normal(size=(1, 3, 4, 3, 2))
    w = rng.normal(size=(27, 2, 2))
    b = rng.normal(size=2)
    dy = rng.normal(size=(1, 3, 4, 3, 2))
    L = lambda w_, b_: np.sum(R.conv3d(x, w_, b_) * dy)
    dw, db = R.conv3d_bwd_weight(x, dy)
    for (t, i, o) in [(0, 0, 0), (13, 1, 0), (26, 0, 1), (5, 1, 1)]:
        e = np.zeros_like(w)
        e[t, i, o] = 1e-6
        assert (L(w + e, b) - L(w - e, b)) / 2e-6 == pytest.approx(dw[t, i, o], rel=1e-6, abs=1e-9)
    e = np.array([0.0, 1e-6])
    assert (L(w, b + e) - L(w, b - e)) / 2e-6 == pytest.approx(db[1], rel=1e-6)


def test_pool_and_upsample_adjoints():
    rng = np.random.default_rng(3)
    x = rng.normal(size=(2, 4, 6, 8, 3))
    y = rng.normal(size=(2, 2, 3, 4, 3))
    assert np.sum(R.pool2(x) * y) == pytest.approx(np.sum(x * R.pool2_bwd(y)), rel=1e-12)
    assert np.sum(R.up2(y) * x) == pytest.approx(np.sum(y * R.up2_bwd(x)), rel=1e-12)
    assert np.allclose(R.pool2(R.up2(y)), y)


def test_bf16_rounding():
    v = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 2 ** -7 + 2 ** -9, -3.14159, 0.0])
    r = R.bf16_round(v)
    assert r[0] == 1.0 and r[1] == 1.0  # tie to even
    assert r[2] == 1.0 + 2 ** -7
    assert abs(r[3] + 3.14159) < 2 ** -7 * 4


def test_periodic_conv_matches_scipy():
    rng = np.random.default_rng(4)
    x = rng.normal(size=(1, 4, 5, 6, 1))
    w = rng.normal(size=(27, 1, 1))
    k = w[:, 0, 0].reshape(3, 3, 3)
    # all axes periodic: scipy's wrap mode
    ref = ndimage.correlate(x[0, :, :, :, 0], k, mode="wrap")
    assert np.allclose(R.conv3d(x, w, wrap=7)[0, :, :, :, 0], ref, rtol=1e-12, atol=1e-12)
    # x periodic only: three copies side by side along x, zero padding, middle copy
    tiled = np.concatenate([x[0, :, :, :, 0]] * 3, axis=2)
    ref = ndimage.correlate(tiled, k, mode="constant", cval=0.0)[:, :, 6:12]
    assert np.allclose(R.conv3d(x, w, wrap=1)[0, :, :, :, 0], ref, rtol=1e-12, atol=1e-12)


def test_periodic_conv_adjoints():
    rng = np.random.default_rng(5)
    x = rng.normal(size=(2, 4, 3, 6, 3))
    w = rng.normal(size=(27, 3, 2))
    dy = rng.normal(size=(2, 4, 3, 6, 2))
    for wrap in (1, 2, 5):
        lhs = np.sum(R.conv3d(x, w, wrap=wrap) * dy)
        assert np.sum(x * R.conv3d_bwd_data(dy, w, wrap=wrap)) == pytest.approx(lhs, rel=1e-12)
        dw, _ = R.conv3d_bwd_weight(x, dy, wrap=wrap)
        assert np.sum(w * dw) == pytest.approx(lhs, rel=1e-12)


def _tiny_unet(rng, chans=(2, 3), cin=2, cout=2):
    names = []
    c = cin
    for lv, ch in enumerate(chans[:-1]):
        names += [(f"enc{lv}a", c, ch), (f"enc{lv}b", ch, ch)]
        c = ch
    names += [("mid_a", c, chans[-1]), ("mid_b", chans[-1], chans[-1])]
    c = chans[-1]
    for lv in reversed(range(len(chans) - 1)):
        names += [(f"dec{lv}a", c + chans[lv], chans[lv]), (f"dec{lv}b", chans[lv], chans[lv])]
        c = chans[lv]
    names.append(("head", c, cout))
    # positive biases keep most ReLUs active, so the finite differences see every path
    return {n: (rng.normal(0, 0.5, (27, a, b)), rng.uniform(0.2, 0.6, b)) for n, a, b in names}


def test_unet_gradients_by_finite_differences():
    rng = np.random.default_rng(6)
    chans = (2, 3)
    params = _tiny_unet(rng, chans)
    x = rng.normal(size=(1, 4, 4, 4, 2))
    dy = rng.normal(size=(1, 4, 4, 4, 2))
    y, cache = R.unet_forward(params, x, chans, wrap=1)
    grads = R.unet_backward(params, cache, dy, chans, wrap=1)

    def loss(p):
        return np.sum(R.unet_forward(p, x, chans, wrap=1)[0] * dy)

    h = 1e-6
    for name in ("enc0a", "enc0b", "mid_a", "mid_b", "dec0a", "dec0b", "head"):
        w, b = params[name]
        for idx in [(0, 0, 0), (13, w.shape[1] - 1, w.shape[2] - 1), (22, 0, w.shape[2] - 1)]:
            wp, wm = w.copy(), w.copy()
            wp[idx] += h
            wm[idx] -= h
            fd = (loss({**params, name: (wp, b)}) - loss({**params, name: (wm, b)})) / (2 * h)
            assert fd == pytest.approx(grads[name][0][idx], rel=1e-5, abs=1e-7), (name, idx)
        bp, bm = b.copy(), b.copy()
        bp[0] += h
        bm[0] -= h
        fd = (loss({**params, name: (w, bp)}) - loss({**params, name: (w, bm)})) / (2 * h)
        assert fd == pytest.approx(grads[name][1][0], rel=1e-5, abs=1e-7), name


def test_flow_symmetries_map_steady_states_to_steady_states():
    """The augmentation symmetries map a steady LBM solution (from the oracle,
    creeping flow along a periodic x axis) to the steady solution of the
    transformed geometry."""
    torch = pytest.importorskip("torch")
    import oracle as O
    from paper_1703_08015_gb300 import geometry as geo
    from paper_1703_08015_gb300.nn import augment

    mask, _ = geo.sphere_pack_3d(12, seed=3, r_min=2, r_max=3.5, target_fluid=0.55)
    per, tau, F = (1, 0, 0), 0.7, (1e-6, 0, 0)

    def steady(m):
        f = O.init(19, m)
        for _ in range(6):
            f = O.run(19, m, per, tau, F, f, 600)
            f = 0.5 * (f + O.run(19, m, per, tau, F, f, 1))  # two-state mean removes the period-2 mode
        rho, u = O.moments(19, m, per, F, f)[:2]
        t = np.stack([rho - 1, u[0], u[1], u[2]], axis=-1)
        return np.where(m[..., None] > 0, t, 0.0)

    t0 = steady(mask)
    scale = np.abs(t0).max(axis=(0, 1, 2))  # per channel
    # mirrors in y, z and the y/z swap are exact symmetries of the lattice update;
    # the x mirror holds for creeping flow (reversibility), here to ~1e-4
    for code, tol in ((1, 1e-8), (2, 1e-8), (4, 1e-8), (7, 1e-8), (8, 1e-3), (15, 1e-3)):
        x = torch.zeros((1,) + mask.shape + (2,))
        xt, tt, mt = augment(x, torch.from_numpy(t0[None]), torch.from_numpy(mask[None]), code)
        m2 = mt[0].numpy().astype(np.uint8)
        want = steady(m2)
        got = tt[0].numpy()
        assert np.all(np.max(np.abs(got - want), axis=(0, 1, 2)) < tol * scale), code
