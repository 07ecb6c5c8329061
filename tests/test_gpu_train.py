"""GPU training step (forward with kept activations, L1-log loss, backward,
Adam) against the float64 oracle, through the C ABI.

Tolerances: the GPU step runs in FP32 (SIMT convolutions), the oracle in
float64.  Every weight and bias gradient element is compared against the
sum of |terms| of that element (sum over pixels of |dout| |x|, from the
oracle): the error is at most 2e-3 of it everywhere, 1e-4 for 99% of the
elements and 1e-5 for the median (FP32 rounding, plus ReLU masks decided
differently where a pre-activation is within rounding of zero), while a
wrong tap, channel, pixel or mask gives errors of the order of the terms.  The loss must
agree to 1e-6 relative and the Adam update to 1% of lr where the oracle
gradient is not tiny (the first Adam step is lr * g / (|g| + eps): where
|g| ~ eps its direction is ill-conditioned).  The BF16 step rounds every
activation to BF16 between layers (the precision choice itself); each of its
backward convolutions is checked element by element on its own
(test_gpu_dgrad.py, test_gpu_wgrad.py), and the whole step here by cosine
similarity to the float64 gradient."""
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


def _batch(seed, N, h, w, s):
    rng = np.random.default_rng(seed)
    lr = rng.gamma(2.0, 0.5, (N, h, w, 3)).astype(np.float32)
    hr = rng.gamma(1.0, 1.0, (N, h * s, w * s, 3)).astype(np.float32)
    hr[0, 0, 0, 0] = 250.0            # a firefly above the clip level
    alb = rng.uniform(0, 1, (N, h * s, w * s, 3)).astype(np.float32)
    nrm = rng.uniform(-1, 1, (N, h * s, w * s, 3)).astype(np.float32)
    tgt = rng.gamma(2.0, 0.5, (N, h * s, w * s, 3)).astype(np.float32)
    return lr, hr, alb, nrm, tgt


def _params(seed):
    layers = cnn.unpack(cnn.kaiming(seed))
    out = []
    for i, (w, b) in enumerate(layers):
        if 1 <= i <= 16 and i % 2 == 0:
            w = w * 0.25
        out.append((w, b + 0.02))
    return cnn.pack(out).astype(np.float32)


def _cuda(*a):
    return [torch.from_numpy(np.ascontiguousarray(t)).cuda() for t in a]


def _assert_grads_elementwise(g, rg, terms, max_r=2e-3):
    # r = |error| / sum |terms| per gradient element.  FP32 rounding alone
    # keeps r near 1e-6; a ReLU whose pre-activation lies within rounding of
    # 0 may be decided differently by the two sides, moving one pixel's
    # contribution (r up to ~1e-3 at these sizes).  A wrong tap, channel or
    # pixel gives r of order 1 / sqrt(pixels) ~ 3e-2 and more.
    r = np.abs(g.astype(np.float64) - rg) / (terms + 1e-30)
    for li, (wo, bo, ci, co) in enumerate(cnn.layer_offsets()):
        for a, b in ((wo, bo), (bo, bo + co)):
            x = r[a:b]
            q = np.quantile(x, [0.5, 0.99, 1.0])
            assert q[2] <= max_r and q[1] <= 1e-4 and q[0] <= 1e-5, (li, a, q)


@pytest.mark.parametrize("N,h,w,s", [(2, 4, 6, 4), (1, 8, 8, 2)])
def test_train_step_gradients_and_update_match_oracle(mrs, N, h, w, s):
    lr, hr, alb, nrm, tgt = _batch(1, N, h, w, s)
    p = _params(0)
    net = mrs.Net(p)
    loss = mrs.train_step(net, *_cuda(lr, hr, alb, nrm, tgt), s, lr=1e-3)
    g = mrs.get_grads(net)
    p1 = net.get_params()
    z = np.zeros(mrs.NPARAMS)
    rp, _, _, rloss, rg, terms = cnn.train_step(p.astype(np.float64), z, z, 1, 1e-3, lr, hr, alb,
                                                nrm, tgt, s, abs_terms=True)
    assert abs(loss - rloss) <= 1e-6 * rloss
    _assert_grads_elementwise(g, rg, terms)
    ok = np.abs(rg) > 1e-6
    assert np.abs((p1 - p) - (rp - p))[ok].max() <= 0.01 * 1e-3


def test_training_reduces_loss_on_a_fixed_batch(mrs):
    lr, hr, alb, nrm, tgt = _batch(2, 2, 8, 8, 4)
    net = mrs.Net(_params(1))
    t = _cuda(lr, hr, alb, nrm, tgt)
    losses = [mrs.train_step(net, *t, 4, lr=1e-3) for _ in range(40)]
    assert losses[-1] < 0.7 * losses[0], losses[::5]


def test_checkpoint_resume_is_bit_identical(mrs, tmp_path):
    lr, hr, alb, nrm, tgt = _batch(3, 1, 4, 4, 4)
    t = _cuda(lr, hr, alb, nrm, tgt)
    a = mrs.Net(_params(2))
    for _ in range(2):
        mrs.train_step(a, *t, 4, lr=1e-3)
    path = str(tmp_path / "ck.bin")
    mrs.save_checkpoint(a, path, seed=5)
    for _ in range(3):
        mrs.train_step(a, *t, 4, lr=1e-3)
    b = mrs.Net(np.zeros(mrs.NPARAMS, np.float32))
    assert mrs.load_checkpoint(b, path) == 5
    for _ in range(3):
        mrs.train_step(b, *t, 4, lr=1e-3)
    sa, sb = mrs.get_state(a), mrs.get_state(b)
    assert sa["step"] == sb["step"] == 5
    for k in ("params", "adam_m", "adam_v"):
        assert np.array_equal(sa[k], sb[k]), k


def test_bf16_train_step_gradients_close_to_oracle(mrs):
    # whole-step summary: BF16 activations / activation gradients with FP32
    # accumulation keep every layer's gradient within a few per cent of the
    # float64 gradient (each backward conv is checked element by element in
    # test_gpu_dgrad.py and test_gpu_wgrad.py)
    lr, hr, alb, nrm, tgt = _batch(4, 2, 8, 16, 4)
    p = _params(3)
    net = mrs.Net(p)
    loss = mrs.train_step(net, *_cuda(lr, hr, alb, nrm, tgt), 4, lr=1e-3, precision="bf16")
    g = mrs.get_grads(net)
    z = np.zeros(mrs.NPARAMS)
    _, _, _, rloss, rg = cnn.train_step(p.astype(np.float64), z, z, 1, 1e-3, lr, hr, alb, nrm, tgt, 4)
    assert abs(loss - rloss) <= 2e-2 * rloss
    for li, (wo, bo, ci, co) in enumerate(cnn.layer_offsets()):
        ref = rg[wo:bo]
        got = g[wo:bo].astype(np.float64)
        cos = got @ ref / (np.linalg.norm(got) * np.linalg.norm(ref) + 1e-30)
        rel = np.linalg.norm(got - ref) / (np.linalg.norm(ref) + 1e-30)
        assert cos > 0.995 and rel < 0.1, (li, cos, rel)


def test_bf16_training_reduces_loss(mrs):
    lr, hr, alb, nrm, tgt = _batch(5, 2, 8, 8, 4)
    net = mrs.Net(_params(4))
    t = _cuda(lr, hr, alb, nrm, tgt)
    losses = [mrs.train_step(net, *t, 4, lr=1e-3, precision="bf16") for _ in range(40)]
    assert losses[-1] < 0.7 * losses[0], losses[::5]


@pytest.mark.parametrize("N,h,w,s", [(2, 4, 6, 4), (1, 8, 8, 2)])
def test_robust_loss_train_step_matches_oracle(mrs, N, h, w, s):
    # the paper's l_r (beta = 0.1) through the FP32 step: loss, every layer's
    # gradient and the Adam update against the float64 oracle
    lr, hr, alb, nrm, tgt = _batch(6, N, h, w, s)
    p = _params(5)
    net = mrs.Net(p)
    loss = mrs.train_step(net, *_cuda(lr, hr, alb, nrm, tgt), s, lr=1e-3, loss="robust", beta=0.1)
    g = mrs.get_grads(net)
    p1 = net.get_params()
    z = np.zeros(mrs.NPARAMS)
    rp, _, _, rloss, rg, terms = cnn.train_step(p.astype(np.float64), z, z, 1, 1e-3, lr, hr, alb,
                                                nrm, tgt, s, loss="robust", beta=0.1,
                                                abs_terms=True)
    assert abs(loss - rloss) <= 1e-6 * rloss
    # l_r's gradient sign(e) beta / (beta + |e|)^2 also turns on a decision:
    # an output within rounding of its target takes the other sign, moving
    # that value's whole contribution (more than a ReLU mask: measured up to
    # 1.3e-2); the median and 99% bounds still single out a wrong tap,
    # channel or pixel, which moves every element of its layer
    _assert_grads_elementwise(g, rg, terms, max_r=5e-2)
    ok = np.abs(rg) > 1e-6
    assert np.abs((p1 - p) - (rp - p))[ok].max() <= 0.01 * 1e-3


def test_robust_loss_bf16_and_loss_switch(mrs):
    # l_r weights an error by beta / (beta + |e|)^2, so a forward rounding
    # error de changes the gradient of that value by 2 de / (beta + |e|)
    # relative (and near e = 0 BF16 rounding decides its sign).  The target
    # keeps every |e| in [1, 3], where BF16 forward rounding (de ~ 1e-2) moves
    # dy by ~2%, so that the comparison measures the kernels rather than the
    # loss's own sensitivity
    lr, hr, alb, nrm, _ = _batch(7, 2, 8, 8, 4)
    p = _params(6)
    y = cnn.forward(p.astype(np.float64), np.minimum(lr, 100.0), np.minimum(hr, 100.0), alb, nrm, 4)
    rng = np.random.default_rng(8)
    tgt = (y + rng.choice([-1.0, 1.0], y.shape) * rng.uniform(1.0, 3.0, y.shape)).astype(np.float32)
    net = mrs.Net(p)
    t = _cuda(lr, hr, alb, nrm, tgt)
    loss = mrs.train_step(net, *t, 4, lr=1e-3, precision="bf16", loss="robust", beta=0.1)
    g = mrs.get_grads(net)
    z = np.zeros(mrs.NPARAMS)
    _, _, _, rloss, rg = cnn.train_step(p.astype(np.float64), z, z, 1, 1e-3, lr, hr, alb, nrm, tgt, 4,
                                        loss="robust", beta=0.1)
    assert abs(loss - rloss) <= 2e-2 * rloss
    for li, (wo, bo, _, _) in enumerate(cnn.layer_offsets()):
        ref, got = rg[wo:bo], g[wo:bo].astype(np.float64)
        cos = got @ ref / (np.linalg.norm(got) * np.linalg.norm(ref) + 1e-30)
        assert cos > 0.99, (li, cos)
    # switching back to the default loss reproduces the oracle's L1-log loss
    net2 = mrs.Net(p)
    net2.set_loss("robust", 0.5)
    net2.set_loss("l1log")
    l2 = mrs.train_step(net2, *t, 4, lr=1e-3)
    r2 = cnn.train_step(p.astype(np.float64), z, z, 1, 1e-3, lr, hr, alb, nrm, tgt, 4)[3]
    assert abs(l2 - r2) <= 1e-6 * r2
    with pytest.raises(Exception):
        net2.set_loss("robust", 0.0)
