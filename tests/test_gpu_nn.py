"""GPU tests of the warm-start network kernels against the FP64 reference in
oracle/nn_ref.py, through the C ABI of include/lbm_nn.h.  Convolutions with
cin % 16 == 0 and cout % 16 == 0 run on the tcgen05 tensor cores (a halo tile
in shared memory), the others on the mma.sync kernel; the cases below cover
both, and the tcgen05 im2col kernel (cin % 8 == 0) through lbm_nn_conv3d_tc.

Operands are BF16 values (the reference sees the same values in FP64).  The
convolutions multiply BF16 pairs exactly and add in FP32, so a result may
differ from the FP64 sum by a few FP32 roundings of the partial sums: the
tolerance is 2^-16 times sum |x||w| (the FP64 convolution of the absolute
values), far below the error of any misplaced operand.
"""
import numpy as np
import pytest

from oracle import nn_ref as R

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def nn():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1703_08015_gb300 import nn as nn_mod

    return nn_mod


def bf16_dev(a):
    return torch.from_numpy(np.asarray(a, np.float32)).cuda().to(torch.bfloat16)


def f64(t):
    return t.float().cpu().numpy().astype(np.float64)


def rand_bf16(rng, shape, scale=1.0):
    return R.bf16_round(rng.normal(0.0, scale, shape))


CONV_CASES = [
    # n, d, h, w, cin, cout, relu, wrap
    (2, 5, 6, 7, 2, 4, 0, 0),
    (1, 4, 4, 8, 16, 16, 1, 1),
    (2, 3, 5, 6, 48, 40, 0, 1),
    (1, 4, 3, 5, 32, 192, 1, 0),
    (1, 2, 4, 4, 7, 9, 0, 5),
    (1, 1, 1, 1, 16, 3, 0, 7),
    # shapes of the tcgen05 path (cin % 8 == 0, cout % 16 == 0): a partial last
    # tile of 128 voxels, cin 8 with zero padding, several channel tiles
    (2, 6, 7, 9, 16, 32, 1, 3),
    (1, 3, 4, 5, 8, 48, 1, 2),
    (1, 8, 8, 8, 64, 128, 0, 7),
]


def _conv(nn, entry):
    """The convolution entry point under test: lbm_nn_conv3d (which picks the
    kernel by shape) or lbm_nn_conv3d_tc (tcgen05 tensor cores only: the
    halo-tile kernel for cin % 16 == 0, the im2col one for cin % 8 == 0)."""
    return nn.lbm_nn_conv3d if entry == "auto" else nn.lbm_nn_conv3d_tc


def _tc_ok(cin, cout):
    return cin % 8 == 0 and cout % 16 == 0


@pytest.mark.parametrize("entry", ["auto", "tc"])
@pytest.mark.parametrize("case", CONV_CASES)
def test_conv_forward(nn, case, entry):
    n, d, h, w, cin, cout, relu, wrap = case
    if entry == "tc" and not _tc_ok(cin, cout):
        pytest.skip("shape outside the tcgen05 kernel")
    rng = np.random.default_rng(hash(case) % 2**32)
    x = rand_bf16(rng, (n, d, h, w, cin))
    wt = rand_bf16(rng, (27, cin, cout), 1.0 / np.sqrt(27 * cin))
    b = rng.normal(0, 0.1, cout).astype(np.float32)
    y = torch.empty((n, d, h, w, cout), dtype=torch.bfloat16, device="cuda")
    y32 = torch.empty((n, d, h, w, cout), dtype=torch.float32, device="cuda")
    _conv(nn, entry)(bf16_dev(x), n, d, h, w, cin, bf16_dev(wt), torch.from_numpy(b).cuda(), cout, relu, wrap, y,
                     y32)
    torch.cuda.synchronize()
    assert nn.lbm_nn_tc_timeouts() == 0
    ref = R.conv3d(x, wt, b.astype(np.float64), bool(relu), wrap)
    tol = 2.0 ** -16 * R.conv3d(np.abs(x), np.abs(wt), np.abs(b.astype(np.float64)), False, wrap) + 1e-30
    got = f64(y32)
    assert np.all(np.abs(got - ref) <= tol), np.max(np.abs(got - ref) / tol)
    # the BF16 output is the FP32 result rounded to nearest
    assert np.array_equal(f64(y), R.bf16_round(got))


@pytest.mark.parametrize("entry", ["auto", "tc"])
@pytest.mark.parametrize("case", CONV_CASES[:5] + CONV_CASES[6:])
def test_conv_backward_data_by_flipped_weights(nn, case, entry):
    n, d, h, w, cin, cout, _, wrap = case
    if entry == "tc" and not _tc_ok(cout, cin):
        pytest.skip("shape outside the tcgen05 kernel")
    rng = np.random.default_rng(7 + hash(case) % 2**31)
    dy = rand_bf16(rng, (n, d, h, w, cout))
    wt = rand_bf16(rng, (27, cin, cout), 1.0 / np.sqrt(27 * cin))
    flipped = torch.empty(27 * cin * cout, dtype=torch.bfloat16, device="cuda")
    nn.lbm_nn_weight_flip(bf16_dev(wt), cin, cout, flipped)
    dx = torch.empty((n, d, h, w, cin), dtype=torch.float32, device="cuda")
    _conv(nn, entry)(bf16_dev(dy), n, d, h, w, cout, flipped, None, cin, 0, wrap, None, dx)
    torch.cuda.synchronize()
    ref = R.conv3d_bwd_data(dy, wt, wrap)
    tol = 2.0 ** -16 * R.conv3d_bwd_data(np.abs(dy), np.abs(wt), wrap) + 1e-30
    assert np.all(np.abs(f64(dx) - ref) <= tol)
    # the flip itself is a pure permutation
    want = np.transpose(wt[::-1], (0, 2, 1)).reshape(-1)
    assert np.array_equal(f64(flipped), want)


@pytest.mark.parametrize("case", CONV_CASES[:5])
def test_conv_weight_gradient(nn, case):
    n, d, h, w, cin, cout, _, wrap = case
    rng = np.random.default_rng(11 + hash(case) % 2**31)
    x = rand_bf16(rng, (n, d, h, w, cin))
    dy = rand_bf16(rng, (n, d, h, w, cout))
    dw = torch.full((27 * cin * cout,), 0.25, dtype=torch.float32, device="cuda")  # accumulates
    db = torch.full((cout,), -0.5, dtype=torch.float32, device="cuda")
    nn.lbm_nn_conv3d_wgrad(bf16_dev(x), bf16_dev(dy), n, d, h, w, cin, cout, wrap, dw, db)
    torch.cuda.synchronize()
    ref_w, ref_b = R.conv3d_bwd_weight(x, dy, wrap)
    tol_w = 2.0 ** -16 * R.conv3d_bwd_weight(np.abs(x), np.abs(dy), wrap)[0] + 1e-6
    assert np.all(np.abs(f64(dw).reshape(27, cin, cout) - 0.25 - ref_w) <= tol_w)
    assert np.allclose(f64(db) + 0.5, ref_b, rtol=1e-5, atol=1e-4)


# shapes of the tcgen05 weight gradient: ragged rows, every periodic
# combination, channel counts off a multiple of 16 or of 8 (the input padded
# to 16), several tap groups (cin 48 .. 192), two output-
# channel tiles (cout 192 above), many voxel chunks (the last case)
WGRAD_TC_CASES = [
    (1, 3, 4, 6, 8, 16, 1),
    (2, 3, 4, 5, 16, 4, 6),
    (1, 2, 4, 4, 9, 9, 5),
    (2, 6, 7, 9, 16, 32, 3),
    (1, 5, 3, 13, 16, 16, 7),
    (2, 3, 5, 6, 48, 48, 5),
    (1, 8, 8, 8, 64, 128, 6),
    (2, 4, 6, 8, 128, 64, 1),
    (1, 4, 4, 4, 192, 16, 0),
    (4, 16, 16, 16, 16, 32, 1),
]


@pytest.mark.parametrize("case", WGRAD_TC_CASES)
def test_conv_weight_gradient_tcgen05(nn, case):
    """The weight gradient on the tensor cores (channel-major packed operands,
    one GEMM per tap) against the FP64 reference, accumulating into dw."""
    n, d, h, w, cin, cout, wrap = case
    rng = np.random.default_rng(13 + hash(case) % 2**31)
    x = rand_bf16(rng, (n, d, h, w, cin))
    dy = rand_bf16(rng, (n, d, h, w, cout))
    dw = torch.full((27 * cin * cout,), 0.25, dtype=torch.float32, device="cuda")
    db = torch.full((cout,), -0.5, dtype=torch.float32, device="cuda")
    nn.lbm_nn_conv3d_wgrad(bf16_dev(x), bf16_dev(dy), n, d, h, w, cin, cout, wrap, dw, db)
    torch.cuda.synchronize()
    assert nn.lbm_nn_tc_timeouts() == 0
    ref_w, ref_b = R.conv3d_bwd_weight(x, dy, wrap)
    tol_w = 2.0 ** -16 * R.conv3d_bwd_weight(np.abs(x), np.abs(dy), wrap)[0] + 1e-6
    err = np.abs(f64(dw).reshape(27, cin, cout) - 0.25 - ref_w)
    assert np.all(err <= tol_w), float(np.max(err / tol_w))
    assert np.allclose(f64(db) + 0.5, ref_b, rtol=1e-5, atol=1e-4)


@pytest.mark.parametrize("entry", ["auto", "tc"])
def test_large_conv_spans_many_tiles(nn, entry):
    """A 4 x 16^3 batch with 16 -> 64 channels (128 halo-tile blocks); every
    output is checked against the reference."""
    rng = np.random.default_rng(3)
    n, s, cin, cout = 4, 16, 16, 64
    x = rand_bf16(rng, (n, s, s, s, cin))
    wt = rand_bf16(rng, (27, cin, cout), 0.1)
    y32 = torch.empty((n, s, s, s, cout), dtype=torch.float32, device="cuda")
    _conv(nn, entry)(bf16_dev(x), n, s, s, s, cin, bf16_dev(wt), None, cout, 0, 1, None, y32)
    torch.cuda.synchronize()
    assert nn.lbm_nn_tc_timeouts() == 0
    ref = R.conv3d(x, wt, None, False, 1)
    tol = 2.0 ** -16 * R.conv3d(np.abs(x), np.abs(wt), None, False, 1) + 1e-30
    assert np.all(np.abs(f64(y32) - ref) <= tol)


def test_pool_upsample_concat_add(nn):
    rng = np.random.default_rng(4)
    n, d, h, w, c = 2, 4, 6, 8, 5
    # magnitudes in [0.5, 2): sums of 8 BF16 values are exact in FP32
    x = R.bf16_round(rng.uniform(0.5, 2.0, (n, d, h, w, c)) * rng.choice([-1, 1], (n, d, h, w, c)))
    xs = R.bf16_round(rng.uniform(0.5, 2.0, (n, d // 2, h // 2, w // 2, c)))
    dev = bf16_dev(x)
    small = bf16_dev(xs)
    out_s = torch.empty((n, d // 2, h // 2, w // 2, c), dtype=torch.bfloat16, device="cuda")
    out_l = torch.empty((n, d, h, w, c), dtype=torch.bfloat16, device="cuda")
    nn.lbm_nn_pool2(dev, n, d, h, w, c, out_s)
    torch.cuda.synchronize()
    assert np.array_equal(f64(out_s), R.bf16_round(R.pool2(x)))
    nn.lbm_nn_pool2_bwd(small, n, d, h, w, c, out_l)
    torch.cuda.synchronize()
    assert np.array_equal(f64(out_l), R.bf16_round(R.pool2_bwd(xs)))
    nn.lbm_nn_up2(small, n, d // 2, h // 2, w // 2, c, out_l)
    torch.cuda.synchronize()
    assert np.array_equal(f64(out_l), R.up2(xs))
    nn.lbm_nn_up2_bwd(dev, n, d // 2, h // 2, w // 2, c, out_s)
    torch.cuda.synchronize()
    assert np.array_equal(f64(out_s), R.bf16_round(R.up2_bwd(x)))
    # concat / split round trip
    vox = n * d * h * w
    b = R.bf16_round(rng.normal(size=(n, d, h, w, 3)))
    cat = torch.empty((n, d, h, w, c + 3), dtype=torch.bfloat16, device="cuda")
    nn.lbm_nn_concat(dev, c, bf16_dev(b), 3, vox, cat)
    torch.cuda.synchronize()
    assert np.array_equal(f64(cat), np.concatenate([x, b], axis=4))
    a2 = torch.empty_like(dev)
    b2 = torch.empty((n, d, h, w, 3), dtype=torch.bfloat16, device="cuda")
    nn.lbm_nn_split(cat, c, 3, vox, a2, b2)
    torch.cuda.synchronize()
    assert np.array_equal(f64(a2), x) and np.array_equal(f64(b2), b)
    # add (in place) and the ReLU mask
    s = torch.empty_like(dev)
    nn.lbm_nn_add(dev, dev, x.size, s)
    torch.cuda.synchronize()
    assert np.array_equal(f64(s), 2 * x)
    g = bf16_dev(np.ones_like(x))
    nn.lbm_nn_relu_mask(g, dev, x.size)
    torch.cuda.synchronize()
    assert np.array_equal(f64(g), (x > 0).astype(np.float64))


def test_mse_adam_and_conversions(nn):
    rng = np.random.default_rng(5)
    vox, c = 1000, 4
    pred = rng.normal(size=(vox, c)).astype(np.float32)
    tgt = rng.normal(size=(vox, c)).astype(np.float32)
    mask = (rng.uniform(size=vox) < 0.6).astype(np.uint8)
    count = int(mask.sum())
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    dpred = torch.empty((vox, c), dtype=torch.bfloat16, device="cuda")
    nn.lbm_nn_mse(torch.from_numpy(pred).cuda(), torch.from_numpy(tgt).cuda(), torch.from_numpy(mask).cuda(), vox, c,
                  count, loss, dpred)
    torch.cuda.synchronize()
    d = (pred.astype(np.float64) - tgt) * mask[:, None]
    assert loss.item() == pytest.approx(np.sum(d * d) / (count * c), rel=1e-6)
    want = R.bf16_round(2 * ((pred - tgt) * mask[:, None]).astype(np.float32) * np.float32(1.0 / (count * c)))
    assert np.allclose(f64(dpred), want, rtol=2 ** -7, atol=0)

    n = 777
    p = rng.normal(size=n).astype(np.float32)
    gr = rng.normal(size=n).astype(np.float32)
    m = rng.normal(size=n).astype(np.float32) * 0.1
    v = rng.uniform(0, 0.1, n).astype(np.float32)
    tp, tg, tm, tv = (torch.from_numpy(a.copy()).cuda() for a in (p, gr, m, v))
    pb = torch.empty(n, dtype=torch.bfloat16, device="cuda")
    lr, b1, b2, eps, t = 1e-3, 0.9, 0.999, 1e-8, 3
    nn.lbm_nn_adam(tp, tg, tm, tv, pb, n, lr, b1, b2, eps, t)
    torch.cuda.synchronize()
    # FP64 reference of the FP32 update with the FP32 values of the constants
    # (beta1 = 0.9f, 1 - beta1 in FP32, ...); tolerance a few FP32 roundings
    c1 = float(np.float32(b1))
    c1m = float(np.float32(1) - np.float32(b1))
    c2 = float(np.float32(b2))
    c2m = float(np.float32(1) - np.float32(b2))
    m_ref = c1 * m.astype(np.float64) + c1m * gr
    v_ref = c2 * v.astype(np.float64) + c2m * gr.astype(np.float64) ** 2
    u32 = 2.0 ** -24
    assert np.all(np.abs(tm.cpu().numpy() - m_ref) <= 4 * u32 * (np.abs(c1 * m) + np.abs(c1m * gr)))
    assert np.all(np.abs(tv.cpu().numpy() - v_ref) <= 4 * u32 * (np.abs(c2 * v) + c2m * gr.astype(np.float64) ** 2))
    step = lr * (m_ref / (1 - b1 ** t)) / (np.sqrt(v_ref / (1 - b2 ** t)) + eps)
    p_ref = p - step
    assert np.all(np.abs(tp.cpu().numpy() - p_ref) <= 8 * u32 * (np.abs(p) + np.abs(step)))
    assert not tg.any().item()  # gradient cleared
    assert np.array_equal(f64(pb), R.bf16_round(tp.cpu().numpy()))

    f = rng.normal(size=100).astype(np.float32)
    b16 = torch.empty(100, dtype=torch.bfloat16, device="cuda")
    back = torch.empty(100, dtype=torch.float32, device="cuda")
    nn.lbm_nn_f32_to_bf16(torch.from_numpy(f).cuda(), 100, b16)
    nn.lbm_nn_bf16_to_f32(b16, 100, back)
    torch.cuda.synchronize()
    assert np.array_equal(back.cpu().numpy().astype(np.float64), R.bf16_round(f))


def test_input_and_field_conversions(nn):
    rng = np.random.default_rng(6)
    shape = (3, 4, 5)
    vox = int(np.prod(shape))
    mask = (rng.uniform(size=shape) < 0.5).astype(np.uint8)
    x = torch.empty(shape + (2,), dtype=torch.bfloat16, device="cuda")
    nn.lbm_nn_mask_input(torch.from_numpy(mask).cuda(), vox, 2.5, x)
    rho = 1 + 1e-4 * rng.normal(size=vox)
    u = 1e-3 * rng.normal(size=3 * vox)
    rho[mask.reshape(-1) == 0] = np.nan
    t = torch.empty((vox, 4), dtype=torch.float32, device="cuda")
    nn.lbm_nn_fields_to_target(torch.from_numpy(rho).cuda(), torch.from_numpy(u).cuda(), vox, 1.0, 1e-4, 1e-3, t)
    r2 = torch.empty(vox, dtype=torch.float64, device="cuda")
    u2 = torch.empty(3 * vox, dtype=torch.float64, device="cuda")
    nn.lbm_nn_target_to_fields(t, vox, 1.0, 1e-4, 1e-3, r2, u2)
    torch.cuda.synchronize()
    xs = f64(x)
    assert np.array_equal(xs[..., 0], mask.astype(np.float64)) and np.all(xs[..., 1] == 2.5)
    fl = mask.reshape(-1) == 1
    tt = t.cpu().numpy()
    assert np.all(tt[~fl] == 0)
    assert np.allclose(r2.cpu().numpy()[fl], rho[fl], rtol=1e-9)
    uu = u2.cpu().numpy().reshape(3, vox)
    assert np.allclose(uu[:, fl], u.reshape(3, vox)[:, fl], rtol=1e-6, atol=1e-12)


def test_bad_arguments_raise(nn):
    from paper_1703_08015_gb300 import lbm

    x = torch.zeros(8, dtype=torch.bfloat16, device="cuda")
    with pytest.raises(lbm.LBMError):
        nn.lbm_nn_conv3d(x, 1, 1, 1, 1, 0, x, None, 4, 0, 0, x, None)
    with pytest.raises(lbm.LBMError):
        nn.lbm_nn_conv3d(x, 1, 1, 1, 1, 1, x, None, 4, 0, 8, x, None)
    with pytest.raises(lbm.LBMError):
        nn.lbm_nn_pool2(x, 1, 3, 2, 2, 1, x)


def _oracle_params(net):
    """The network's BF16 weights and FP32 biases as FP64 arrays per layer."""
    wb = net.pb.float().cpu().numpy().astype(np.float64)
    pf = net.p.cpu().numpy().astype(np.float64)
    out = {}
    for L in net.layers:
        out[L.name] = (wb[L.w_off:L.w_off + L.nw].reshape(27, L.cin, L.cout), pf[L.b_off:L.b_off + L.cout])
    return out


def test_unet_forward_and_gradients_match_oracle(nn):
    """A small U-Net end to end: forward output and every layer's weight and
    bias gradient against the FP64 reference network with the same BF16
    roundings of stored activations and activation gradients."""
    chans = (8, 16, 24)
    net = nn.UNet(chans, cin=2, cout=4, wrap=1, seed=3)
    # positive biases so that the ReLUs pass most values
    nb = net.p.cpu().numpy()
    for L in net.layers:
        nb[L.b_off:L.b_off + L.cout] = 0.05
    net.p.copy_(torch.from_numpy(nb))
    rng = np.random.default_rng(8)
    n, s = 2, 8
    x = rand_bf16(rng, (n, s, s, s, 2))
    dims = (n, s, s, s)
    y = net.forward(bf16_dev(x), dims, keep=True)
    dout = rand_bf16(rng, (n, s, s, s, 4), 0.01)
    net.backward(bf16_dev(dout))
    torch.cuda.synchronize()
    params = _oracle_params(net)
    y_ref, cache = R.unet_forward(params, x, chans, wrap=1, rnd=R.bf16_round)
    got = f64(y)
    assert np.linalg.norm(got - y_ref) <= 1e-3 * np.linalg.norm(y_ref)
    grads = R.unet_backward(params, cache, dout, chans, wrap=1, rnd=R.bf16_round)
    g = net.g.cpu().numpy().astype(np.float64)
    for L in net.layers:
        gw = g[L.w_off:L.w_off + L.nw].reshape(27, L.cin, L.cout)
        gb = g[L.b_off:L.b_off + L.cout]
        rw, rb = grads[L.name]
        assert np.linalg.norm(gw - rw) <= 1e-2 * np.linalg.norm(rw) + 1e-12, L.name
        assert np.linalg.norm(gb - rb) <= 1e-2 * np.linalg.norm(rb) + 1e-12, L.name


def test_training_reduces_loss(nn):
    """A few Adam steps on a fixed batch lower the masked loss."""
    net = nn.UNet((8, 16), cin=2, cout=4, wrap=1, seed=1)
    rng = np.random.default_rng(9)
    n, s = 2, 8
    masks = torch.from_numpy((rng.uniform(size=(n, s, s, s)) < 0.6).astype(np.uint8)).cuda()
    x = nn.inputs_from_masks(masks, 1e-6, net._s())
    # a learnable target: fixed values on the fluid nodes, two of them set by
    # whether the node has a solid neighbour along x
    m = masks.cpu().numpy().astype(np.float32)
    near = 1.0 - np.roll(m, 1, axis=3) * np.roll(m, -1, axis=3)
    t = np.stack([0.5 * m, -1.0 * m, 2.0 * m * near, 0.3 * m * (1 - near)], axis=4)
    tgt = torch.from_numpy(t.astype(np.float32)).cuda()
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    count = int(masks.sum().item())
    hist = []
    for it in range(60):
        y = net.forward(x, (n, s, s, s), keep=True)
        dout = torch.empty(y.shape, dtype=torch.bfloat16, device="cuda")
        nn.lbm_nn_mse(y, tgt, masks, n * s ** 3, 4, count, loss, dout, net._s())
        hist.append(loss.item())
        net.backward(dout)
        net.adam(3e-3)
    assert hist[-1] < 0.5 * hist[0]


def test_training_is_deterministic(nn):
    """Two nets from the same seed, trained on the same batches, end with the
    same bits: every gradient (weights and biases, through the tcgen05 and the
    gather weight-gradient kernels) sums its voxel chunks in a fixed order."""
    rng = np.random.default_rng(19)
    n, s = 2, 16
    masks = torch.from_numpy((rng.uniform(size=(n, s, s, s)) < 0.6).astype(np.uint8)).cuda()
    tgt = torch.from_numpy(rng.normal(size=(n, s, s, s, 4)).astype(np.float32)).cuda()
    count = int(masks.sum().item())
    states = []
    for _ in range(2):
        net = nn.UNet((16, 32), cin=2, cout=4, wrap=1, seed=3)
        x = nn.inputs_from_masks(masks, 1e-6, net._s())
        loss = torch.zeros(1, dtype=torch.float64, device="cuda")
        for it in range(4):
            y = net.forward(x, (n, s, s, s), keep=True)
            dout = torch.empty(y.shape, dtype=torch.bfloat16, device="cuda")
            nn.lbm_nn_mse(y, tgt, masks, n * s ** 3, 4, count, loss, dout, net._s())
            net.backward(dout)
            net.adam(1e-3)
        torch.cuda.synchronize()
        # FP32 master weights and biases, their BF16 copy, Adam's moments
        states.append([t.detach().contiguous().view(torch.uint8).cpu().numpy().copy()
                       for t in (net.p, net.pb, net.m, net.v)])
    for a, b in zip(*states):
        assert np.array_equal(a, b)
    assert nn.lbm_nn_tc_timeouts() == 0
