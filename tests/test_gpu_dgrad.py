"""Input gradient of one 3x3 conv layer (the training step's transposed
convolution) against the float64 oracle, element by element, in the three
epilogues the backward pass applies: linear (the head's gradient into the
last residual stream), ReLU mask (a block's inner ReLU), residual add (the
gradient joining the skip).

BF16 runs the tensor-core kernel with the step's flipped, transposed weight
packing; the oracle gets the same BF16-rounded dy, w and aux, so what remains
is the FP32 accumulation over K = 9 cout terms, bounded by K 2^-23 sum |terms|,
and the rounding of the stored result to BF16 (half an ulp: 2^-8 relative).
FP32 runs the SIMT path on the unrounded operands with the same accumulation
bound."""
import numpy as np
import pytest

from oracle import cnn

torch = pytest.importorskip("torch")
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
    dy = (rng.normal(size=(N, H, W, cout)) * 0.01).astype(np.float32)
    w = (rng.normal(size=(cout, 3, 3, cin)) * np.sqrt(2.0 / (9 * cin))).astype(np.float32)
    # aux: a ReLU output (about half zeros) for the mask, a gradient for the skip
    relu_out = np.maximum(rng.normal(size=(N, H, W, cin)), 0).astype(np.float32)
    grad_in = (rng.normal(size=(N, H, W, cin)) * 0.01).astype(np.float32)
    return dy, w, relu_out, grad_in


def _oracle(dy, w, mode, aux):
    """float64 transposed conv of the oracle's backward pass + the epilogue,
    and sum |terms| per output element."""
    N, H, W, _ = dy.shape
    cin = w.shape[3]
    x0 = np.zeros((N, H, W, cin))
    g = cnn.conv3x3_backward(x0, w, dy)[0]
    a = cnn.conv3x3_backward(x0, np.abs(w), np.abs(dy))[0]
    if mode == "linear":
        return g, a
    if mode == "relu_mask":
        return np.where(aux > 0, g, 0.0), np.where(aux > 0, a, 0.0)
    return aux + g, a


CASES = [(1, 1, 8, 64, 64), (2, 9, 150, 64, 64), (1, 5, 130, 64, 3), (3, 4, 37, 64, 64),
         (1, 3, 300, 21, 64), (16, 16, 16, 64, 64)]


@pytest.mark.parametrize("mode", ["linear", "relu_mask", "residual"])
@pytest.mark.parametrize("N,H,W,cin,cout", CASES)
@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_dgrad_matches_oracle_elementwise(mrs, prec, mode, N, H, W, cin, cout):
    dy, w, relu_out, grad_in = _case(N * 7 + W + cout, N, H, W, cin, cout)
    aux = None if mode == "linear" else relu_out if mode == "relu_mask" else grad_in
    got = mrs.conv3x3_dgrad(torch.from_numpy(dy).cuda(), w, mode,
                            None if aux is None else torch.from_numpy(aux).cuda(),
                            precision=prec).cpu().numpy().astype(np.float64)
    if prec == "bf16":
        dq, wq = bf16_round(dy), bf16_round(w)
        aq = None if aux is None else bf16_round(aux)
    else:
        dq, wq = dy.astype(np.float64), w.astype(np.float64)
        aq = None if aux is None else aux.astype(np.float64)
    ref, terms = _oracle(dq, wq, mode, aq)
    K = 9 * cout
    bound = K * 2.0**-23 * terms + 1e-12
    if prec == "bf16":
        bound = bound + 2.0**-8 * np.abs(ref)
    else:
        bound = bound + 2.0**-23 * np.abs(ref)
    err = np.abs(got - ref)
    assert (err <= bound).all(), (err / bound).max()
    if mode == "relu_mask":
        assert not got[aq <= 0].any()      # masked entries are exactly zero
    # a wrong tap, flip or channel gives errors of the order of the terms
    assert err.mean() <= 1e-2 * terms.mean() + 1e-12


def test_dgrad_bf16_on_bf16_operands_equals_fp32(mrs):
    # on operands already representable in BF16 the two paths compute the same
    # sums; they differ by accumulation order and the BF16 result rounding
    dy, w, _, _ = _case(3, 2, 7, 90, 64, 64)
    dy, w = bf16_round(dy).astype(np.float32), bf16_round(w).astype(np.float32)
    t = torch.from_numpy(dy).cuda()
    a = mrs.conv3x3_dgrad(t, w, "linear", precision="fp32").cpu().numpy()
    b = mrs.conv3x3_dgrad(t, w, "linear", precision="bf16").cpu().numpy()
    terms = _oracle(dy.astype(np.float64), w.astype(np.float64), "linear", None)[1]
    bound = 2 * 576 * 2.0**-23 * terms + 2.0**-8 * np.abs(a) + 1e-12
    assert (np.abs(a - b) <= bound).all(), (np.abs(a - b) / bound).max()


def test_dgrad_rejects_bad_arguments(mrs):
    dy = torch.zeros((1, 4, 4, 8), device="cuda")
    w = np.zeros((8, 3, 3, 65), np.float32)
    with pytest.raises(Exception):
        mrs.conv3x3_dgrad(dy, w, "linear", precision="bf16")          # cin > 64
    w = np.zeros((8, 3, 3, 16), np.float32)
    with pytest.raises(Exception):
        mrs.conv3x3_dgrad(dy, w, "relu_mask", None, precision="bf16")  # aux missing
    with pytest.raises(Exception):
        mrs.conv3x3_dgrad(dy, w, "linear", precision="fp8")
