"""GPU tests of the BF16 GEMM on the 5th-generation tensor cores (tcgen05),
through the C ABI of include/lbm_nn.h, against the FP64 product of the same
BF16 values.  The tensor cores multiply BF16 pairs exactly and accumulate in
FP32, so the tolerance is 2^-16 times sum |a||b|, far below the error of any
misplaced operand (a wrong element or a swapped row group)."""
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


def _dev(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda().to(dtype)


@pytest.mark.parametrize("m,n,k", [(128, 16, 64), (256, 64, 128), (384, 128, 192), (128, 256, 64), (256, 48, 320)])
def test_gemm_bf16_tcgen05(nn, m, n, k):
    rng = np.random.default_rng(1000 * n + k)
    a = R.bf16_round(rng.normal(size=(m, k)))
    b = R.bf16_round(rng.normal(size=(n, k)))
    c = torch.full((m, n), float("nan"), dtype=torch.float32, device="cuda")
    nn.lbm_nn_gemm_bf16(_dev(a, torch.bfloat16), _dev(b, torch.bfloat16), c, m, n, k)
    torch.cuda.synchronize()
    assert nn.lbm_nn_tc_timeouts() == 0
    got = c.cpu().numpy().astype(np.float64)
    want = a @ b.T
    tol = 2.0 ** -16 * (np.abs(a) @ np.abs(b).T)
    assert np.all(np.abs(got - want) <= tol), float(np.max(np.abs(got - want) / tol))


def test_gemm_bf16_rejects_bad_shapes(nn):
    from paper_1703_08015_gb300 import lbm

    x = torch.zeros(128 * 64, dtype=torch.bfloat16, device="cuda")
    c = torch.zeros(128 * 64, dtype=torch.float32, device="cuda")
    for m, n, k in [(100, 16, 64), (128, 8, 64), (128, 24, 64), (128, 272, 64), (128, 16, 32)]:
        with pytest.raises(lbm.LBMError):
            nn.lbm_nn_gemm_bf16(x, x, c, m, n, k)


def test_conv3d_tc_rejects_shapes_outside_it(nn):
    from paper_1703_08015_gb300 import lbm

    x = torch.zeros(4 * 4 * 4 * 16, dtype=torch.bfloat16, device="cuda")
    w = torch.zeros(27 * 16 * 16, dtype=torch.bfloat16, device="cuda")
    y = torch.zeros(4 * 4 * 4 * 16, dtype=torch.float32, device="cuda")
    for cin, cout in [(7, 16), (16, 8), (12, 16)]:
        with pytest.raises(lbm.LBMError):
            nn.lbm_nn_conv3d_tc(x, 1, 4, 4, 4, cin, w, None, cout, 0, 0, None, y)


@pytest.mark.parametrize("bricks_z,cout_tile", [(1, 16), (2, 32), (3, 48), (4, 16), (4, 128), (2, 0), (0, 16)])
def test_conv_halo_launch_shapes(nn, bricks_z, cout_tile):
    """Every launch shape of the halo-tile convolution (bricks per block along
    z, output channels per block) gives the same FP32 sums, bit for bit, and
    they match the FP64 convolution: ragged bricks in x, y and z, two input
    chunks (80 = 64 + 16 channels), a partial output-channel tile, periodic x
    and z."""
    n, d, h, w, cin, cout, wrap = 1, 7, 20, 9, 80, 48, 5
    rng = np.random.default_rng(31)
    x = R.bf16_round(rng.normal(size=(n, d, h, w, cin)))
    wt = R.bf16_round(rng.normal(size=(27, cin, cout)) / np.sqrt(27 * cin))
    b = rng.normal(0, 0.1, cout).astype(np.float32)
    xd, wd, bd = _dev(x, torch.bfloat16), _dev(wt, torch.bfloat16), torch.from_numpy(b).cuda()
    y32 = torch.full((n, d, h, w, cout), float("nan"), dtype=torch.float32, device="cuda")
    base = torch.empty_like(y32)
    try:
        nn.lbm_nn_conv_tune(0, 0)
        nn.lbm_nn_conv3d_tc(xd, n, d, h, w, cin, wd, bd, cout, 0, wrap, None, base)
        nn.lbm_nn_conv_tune(bricks_z, cout_tile)
        nn.lbm_nn_conv3d_tc(xd, n, d, h, w, cin, wd, bd, cout, 0, wrap, None, y32)
        torch.cuda.synchronize()
    finally:
        nn.lbm_nn_conv_tune(0, 0)
    assert nn.lbm_nn_tc_timeouts() == 0
    assert torch.equal(y32, base)
    ref = R.conv3d(x, wt, b.astype(np.float64), False, wrap)
    tol = 2.0 ** -16 * R.conv3d(np.abs(x), np.abs(wt), np.abs(b.astype(np.float64)), False, wrap) + 1e-30
    got = y32.cpu().numpy().astype(np.float64)
    assert np.all(np.abs(got - ref) <= tol), float(np.max(np.abs(got - ref) / tol))
