"""Weight / bias gradient of one 3x3 conv layer against the float64 oracle.

dW[o][ky][kx][c] = sum_p dy[p][o] x[p + (ky-1, kx-1)][c] and db = sum_p dy:
the contraction of the training step's backward pass.  BF16 runs on the
tensor cores with BF16-rounded x and dy and FP32 accumulation, so the oracle
gets the same rounded inputs; the remaining error is FP32 accumulation only,
bounded here by a small multiple of the sum of |terms|."""
import numpy as np
import pytest
import torch

from oracle import cnn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mrs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2106_12802_gb300 as m
    m.load()
    return m


def bf16_round(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


def _case(seed, N, H, W, cin, cout):
    rng = np.random.default_rng(seed)
    x = rng.normal(size=(N, H, W, cin)).astype(np.float32)
    dy = (rng.normal(size=(N, H, W, cout)) * 0.01).astype(np.float32)
    return x, dy


def _oracle(x, dy):
    zero_w = np.zeros((dy.shape[3], 3, 3, x.shape[3]))
    _, dw, db = cnn.conv3x3_backward(x, zero_w, dy)
    _, aw, ab = cnn.conv3x3_backward(np.abs(x), zero_w, np.abs(dy))
    return dw, db, aw, ab


CASES = [(1, 1, 8, 64, 64), (2, 9, 150, 64, 64), (1, 5, 128, 12, 64), (3, 4, 37, 64, 3),
         (2, 7, 64, 64, 64), (1, 3, 300, 64, 16), (16, 128, 128, 64, 64)]


@pytest.mark.parametrize("N,H,W,cin,cout", CASES)
@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_wgrad_matches_oracle(mrs, prec, N, H, W, cin, cout):
    x, dy = _case(N * 131 + W, N, H, W, cin, cout)
    dw, db = mrs.conv3x3_wgrad(torch.from_numpy(x).cuda(), torch.from_numpy(dy).cuda(), precision=prec)
    xr, dyr = (bf16_round(x), bf16_round(dy)) if prec == "bf16" else (x.astype(np.float64), dy.astype(np.float64))
    rw, rb, aw, ab = _oracle(xr, dyr)
    ew, eb = np.abs(dw - rw), np.abs(db - rb)
    # FP32 accumulation error: far below 1e-4 of the sum of |terms| for these
    # sizes; a wrong tap, channel or pixel gives errors of order the terms
    assert (ew <= 1e-4 * aw + 1e-9).all(), (ew / (aw + 1e-30)).max()
    assert (eb <= 1e-4 * ab + 1e-9).all(), (eb / (ab + 1e-30)).max()
    assert ew.mean() <= 1e-6 * aw.mean()


def test_wgrad_bf16_equals_fp32_on_bf16_inputs(mrs):
    # on inputs already representable in BF16 the two paths compute the same
    # sums; only the FP32 accumulation order differs
    x, dy = _case(7, 2, 6, 90, 64, 64)
    x, dy = bf16_round(x).astype(np.float32), bf16_round(dy).astype(np.float32)
    xt, dyt = torch.from_numpy(x).cuda(), torch.from_numpy(dy).cuda()
    w32, b32 = mrs.conv3x3_wgrad(xt, dyt, precision="fp32")
    w16, b16 = mrs.conv3x3_wgrad(xt, dyt, precision="bf16")
    _, _, aw, ab = _oracle(x.astype(np.float64), dy.astype(np.float64))
    assert (np.abs(w32 - w16) <= 2e-4 * aw + 1e-9).all()
    assert (np.abs(b32 - b16) <= 2e-4 * ab + 1e-9).all()


def test_wgrad_is_deterministic(mrs):
    x, dy = _case(9, 4, 32, 128, 64, 64)
    xt, dyt = torch.from_numpy(x).cuda(), torch.from_numpy(dy).cuda()
    a = mrs.conv3x3_wgrad(xt, dyt, precision="bf16")
    b = mrs.conv3x3_wgrad(xt, dyt, precision="bf16")
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_wgrad_rejects_bad_arguments(mrs):
    x = torch.zeros((1, 4, 4, 65), device="cuda")
    dy = torch.zeros((1, 4, 4, 8), device="cuda")
    with pytest.raises(Exception):
        mrs.conv3x3_wgrad(x, dy, precision="bf16")
    with pytest.raises(Exception):
        mrs.conv3x3_wgrad(dy, dy, precision="fp8")
