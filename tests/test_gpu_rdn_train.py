"""Training step of the method's own network (mrs_rdn_train_step: forward
with the activations kept, the loss, the backward of every step, Adam)
against the float64 oracle (oracle/rdn.py, whose backward is pinned by
finite differences), through the C ABI.

Tolerances (the GPU step runs in FP32, the oracle in float64):
* Forward: the step's I_SR equals mrs_rdn_fuse's FP32 output bit for bit
  (the same arithmetic in the same order), and the float64 forward within
  1e-5 * max(1, max |y|) as in test_gpu_rdn.py.
* Loss: |d loss| <= mean |y_gpu - y_oracle| / beta (the l_r term
  |e| / (beta + |e|) has slope at most 1 / beta) plus 1e-6 relative.
* Gradients, element by element: r = |g - g_oracle| / sum |terms| (sum over
  pixels of |dz| |x|, from the oracle), against two references.
  (1) The backward alone: the oracle's backward from the dL/dI_SR of the
  GPU's own I_SR.  FP32 rounding keeps r near 1e-6 (the activation
  gradients reaching the encoders carry the rounding of some 70 transposed
  convolutions and of the dense concatenations' sums); a ReLU whose
  pre-activation lies within rounding of 0 may be decided differently by
  the two sides, moving single pixels' terms, and the change spreads
  through the transposed convolutions below it (the 64-element bias arrays
  show it first).  Bars: median 1e-5 and 99th percentile 1e-3 per weight /
  bias array, r > 1e-3 for at most 0.1% of all elements.
  (2) End to end, against the float64 step: the robust loss's slope
  beta / (beta + |e|)^2 turns the forward's rounding (|dy| up to
  1e-5 max |y|) into a relative change of dL/dI_SR of up to
  2 |dy| / (beta + |e|): 1e-4 to 6e-3 at beta = 0.1 for outputs of 1 to 30.
  Bars: median 1e-4 per array; over all elements 99th percentile 2e-3 and
  r > 1e-2 for at most 0.1% (a 64-element bias array's 99th percentile is
  its maximum, where a single ill-conditioned element decides).
  A wrong tap, channel, part, mask or skip gives r of order 1e-2 to 1 over
  whole arrays.
* Adam update: within 1% of lr plus the FP32 spacing of the stored weight
  wherever the oracle gradient is well conditioned (|g| > 1e-6 and
  |g| > 1e-3 sum |terms|: the first step is lr * g / (|g| + eps), whose sign
  is ill-conditioned where g cancels).
"""
import numpy as np
import pytest

from oracle import cnn
from oracle import rdn as ordn

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mrs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2106_12802_gb300 as m
    m.load()
    return m


def _cuda(*a):
    return [None if t is None else torch.from_numpy(np.ascontiguousarray(t, np.float32)).cuda()
            for t in a]


def _batch(seed, N, h, w, s, c_hr=9):
    rng = np.random.default_rng(seed)
    H, W = h * s, w * s
    lr = rng.gamma(2.0, 0.5, (N, h, w, 3))
    hr = rng.gamma(1.0, 1.0, (N, H, W, 3))
    alb = rng.uniform(0, 1, (N, H, W, 3))
    nrm = rng.uniform(-1, 1, (N, H, W, 3))
    ex = rng.gamma(1.0, 0.5, (N, H, W, 9)) if c_hr == 18 else None
    tgt = rng.gamma(2.0, 0.5, (N, H, W, 3))
    tgt[0, 0, 0, 0] = 250.0            # a firefly above the clip level
    return [None if a is None else a.astype(np.float32) for a in (lr, hr, alb, nrm, ex, tgt)]


def _params(seed, s, c_hr=9):
    layers = ordn.unpack(ordn.kaiming(seed, s, c_hr, fusion_damp=0.1), s, c_hr)
    return ordn.pack([(w, b + 0.01) for w, b in layers]).astype(np.float32)


def _f64(a):
    return None if a is None else np.asarray(a, np.float64)


def _rel_errors(g, rg, terms, s, c_hr, report):
    """Per weight / bias array: (name, [median, 99th percentile, max] of
    r = |g - rg| / sum |terms|); printed as a table."""
    r = np.abs(g.astype(np.float64) - rg) / (terms + 1e-30)
    rows = []
    for name, wo, bo, k, ci, co in ordn.layer_offsets(s, c_hr):
        for a, b in ((wo, bo), (bo, bo + co)):
            rows.append((name + (".b" if a == bo else ".w"), np.quantile(r[a:b], [0.5, 0.99, 1.0])))
    q = np.array([row[1] for row in rows])
    print(f"\n{report}: max over arrays of median {q[:, 0].max():.2e}, p99 {q[:, 1].max():.2e}, "
          f"max {q[:, 2].max():.2e}; elements with r > 1e-3: {(r > 1e-3).sum()}, r > 1e-2: "
          f"{(r > 1e-2).sum()} of {r.size}")
    return rows, r


@pytest.mark.parametrize("s,N,h,w,c_hr,loss", [(2, 2, 4, 6, 9, "robust"), (4, 1, 4, 5, 9, "robust"),
                                               (8, 1, 2, 3, 9, "l1log"), (2, 1, 5, 4, 18, "robust")])
def test_rdn_train_step_matches_oracle(mrs, s, N, h, w, c_hr, loss):
    lr, hr, alb, nrm, ex, tgt = _batch(s * 10 + N, N, h, w, s, c_hr)
    p = _params(s, s, c_hr)
    net = mrs.RDN(p, s, c_hr)
    dev = _cuda(lr, hr, alb, nrm, tgt, ex)
    y = torch.empty((N, h * s, w * s, 3), device="cuda")
    v = net.train_step(*dev[:5], lr=1e-3, loss=loss, beta=0.1, extra=dev[5], out=y)
    g = net.get_grads()
    p1 = net.get_params()
    # the step's forward is the FP32 inference path, bit for bit
    ref = mrs.RDN(p, s, c_hr).fuse(*dev[:4], precision="fp32", extra=dev[5])
    assert torch.equal(y, ref)
    y = y.cpu().numpy().astype(np.float64)
    p64 = p.astype(np.float64)
    args = [_f64(a) for a in (lr, hr, alb, nrm)]
    ry, tape = ordn.forward_tape(p64, *args, s, _f64(ex))
    assert np.abs(y - ry).max() <= 1e-5 * max(1.0, np.abs(ry).max())
    tc = np.minimum(_f64(tgt), 100.0)
    rv, rdy = cnn.loss_fn(ry, tc, loss, 0.1)
    slope = 1.0 / 0.1 if loss == "robust" else 1.0
    assert abs(v - rv) <= slope * np.abs(y - ry).mean() + 1e-6 * rv, (v, rv)

    # (1) the backward alone: the oracle's backward from the dL/dI_SR of the
    # GPU's own I_SR (the robust loss's slope beta / (beta + |e|)^2 turns the
    # forward's FP32 rounding into a relative change of dy of up to
    # 2 |dy| / (beta + |e|), which this reference leaves out)
    _, gdy = cnn.loss_fn(y, tc, loss, 0.1)
    bg, bterms = ordn.backward(p64, tape, gdy, abs_terms=True)
    rows, r = _rel_errors(g, bg, bterms, s, c_hr, f"backward s={s} c_hr={c_hr} {loss}")
    for name, q in rows:
        assert q[0] <= 1e-5 and q[1] <= 1e-3, (name, q)
    # ReLU decisions taken differently where a pre-activation is within
    # rounding of 0 move single pixels' terms: few elements
    assert (r > 1e-3).mean() <= 1e-3
    # (2) end to end against the float64 step
    rg, terms = ordn.backward(p64, tape, rdy, abs_terms=True)
    rows, r = _rel_errors(g, rg, terms, s, c_hr, f"end to end s={s} c_hr={c_hr} {loss}")
    for name, q in rows:
        assert q[0] <= 1e-4, (name, q)
    assert np.quantile(r, 0.99) <= 2e-3 and (r > 1e-2).mean() <= 1e-3
    # first Adam step: p - lr g / (|g| + eps); the stored FP32 weight adds
    # its own rounding (half a spacing)
    ok = (np.abs(rg) > 1e-6) & (np.abs(rg) > 1e-3 * terms)
    assert ok.mean() > 0.3
    rp = p64 - 1e-3 * rg / (np.abs(rg) + 1e-8)
    err = np.abs(p1.astype(np.float64) - rp)
    assert (err <= 0.01 * 1e-3 + np.spacing(np.abs(p1)).astype(np.float64))[ok].all()


def test_rdn_training_reduces_loss_on_a_fixed_batch(mrs):
    # H_Rec scaled down so that the initial errors are of the order of the
    # targets (with |e| >> beta the robust loss saturates near 1 and Adam's
    # first steps move it up; the float64 oracle does the same)
    lr, hr, alb, nrm, ex, tgt = _batch(5, 2, 6, 6, 4)
    L = ordn.unpack(_params(1, 4), 4)
    L[-1] = (L[-1][0] * 0.05, L[-1][1])
    net = mrs.RDN(ordn.pack(L).astype(np.float32), 4)
    dev = _cuda(lr, hr, alb, nrm, tgt)
    losses = [net.train_step(*dev, lr=1e-4, loss="robust", beta=0.1) for _ in range(30)]
    assert losses[-1] < 0.9 * losses[0], losses[::5]
    assert all(b < a for a, b in zip(losses[::5], losses[5::5])), losses[::5]
    assert net.get_state()["step"] == 30


def test_rdn_state_resume_is_bit_identical_and_bf16_follows_training(mrs):
    lr, hr, alb, nrm, ex, tgt = _batch(6, 1, 4, 4, 4)
    dev = _cuda(lr, hr, alb, nrm, tgt)
    a = mrs.RDN(_params(2, 4), 4)
    for _ in range(2):
        a.train_step(*dev, lr=1e-3)
    st = a.get_state()
    assert st["step"] == 2 and st["adam_v"].any()
    for _ in range(3):
        a.train_step(*dev, lr=1e-3)
    b = mrs.RDN(np.zeros_like(st["params"]), 4)
    b.set_state(st)
    for _ in range(3):
        b.train_step(*dev, lr=1e-3)
    sa, sb = a.get_state(), b.get_state()
    assert sa["step"] == sb["step"] == 5
    for k in ("params", "adam_m", "adam_v"):
        assert np.array_equal(sa[k], sb[k]), k
    # the BF16 path repacks from the trained FP32 weights: identical to a
    # network created from them
    c = mrs.RDN(sa["params"], 4)
    ya = a.fuse(*dev[:4], precision="bf16")
    yc = c.fuse(*dev[:4], precision="bf16")
    assert torch.equal(ya, yc)
    assert not torch.equal(ya, mrs.RDN(_params(2, 4), 4).fuse(*dev[:4], precision="bf16"))


def test_rdn_train_step_rejects_bad_arguments(mrs):
    lr, hr, alb, nrm, ex, tgt = _batch(7, 1, 2, 2, 2)
    dev = _cuda(lr, hr, alb, nrm, tgt)
    net = mrs.RDN(_params(3, 2), 2)
    with pytest.raises(mrs.MrsError):
        net.get_grads()                                   # no step taken yet
    with pytest.raises(mrs.MrsError):
        net.train_step(*dev, precision="fp8")
    with pytest.raises(mrs.MrsError):
        net.train_step(*dev, loss=7)
    with pytest.raises(mrs.MrsError):
        net.train_step(*dev, loss="robust", beta=0.0)
    with pytest.raises(mrs.MrsError):
        net.train_step(*dev, extra=dev[0])                # extra on a 9-channel network
    with pytest.raises(mrs.MrsError):
        net.train_step(*dev, lr=-1.0)
    before = net.get_params()
    assert np.array_equal(before, _params(3, 2))          # nothing ran


@pytest.mark.parametrize("s,N,h,w,c_hr", [(2, 2, 8, 12, 9), (4, 2, 8, 8, 9), (8, 1, 4, 4, 9),
                                          (4, 2, 8, 8, 18)])
def test_rdn_bf16_train_step_close_to_oracle(mrs, s, N, h, w, c_hr):
    # tensor-core step: BF16 activations and activation gradients, FP32
    # accumulation, FP32 weight-gradient reductions and Adam.  Each backward
    # convolution kind is checked element by element on its own
    # (test_gpu_dgrad.py, test_gpu_wgrad.py, test_gpu_rdn.py for the
    # multi-chunk and view operands); the whole step here by the cosine and
    # relative L2 distance of every layer's gradient to the float64 one.  The
    # loss is L1-log, whose gradient depends on I_SR only through
    # 1 / (1 + |I_SR|): with l_r far from its targets (|e| >> beta) the
    # gradient beta / (beta + |e|)^2 is carried by the few pixels where I_SR
    # is closest to the target, and BF16's rounding of I_SR (some 0.5% of it)
    # changes those pixels' |e| entirely -- a comparison there measures the
    # precision, not the kernels.
    lr, hr, alb, nrm, ex, tgt = _batch(100 + s * 10 + N, N, h, w, s, c_hr)
    p = _params(s + 1, s, c_hr)
    net = mrs.RDN(p, s, c_hr)
    dev = _cuda(lr, hr, alb, nrm, tgt, ex)
    y = torch.empty((N, h * s, w * s, 3), device="cuda")
    v = net.train_step(*dev[:5], lr=1e-3, loss="l1log", extra=dev[5], out=y, precision="bf16")
    g = net.get_grads().astype(np.float64)
    p64 = p.astype(np.float64)
    args = [_f64(a) for a in (lr, hr, alb, nrm)]
    ry, tape = ordn.forward_tape(p64, *args, s, _f64(ex))
    tc = np.minimum(_f64(tgt), 100.0)
    rv, rdy = cnn.loss_fn(ry, tc, "l1log")
    rg = ordn.backward(p64, tape, rdy)
    yb = y.cpu().numpy().astype(np.float64)
    rel_y = np.linalg.norm(yb - ry) / np.linalg.norm(ry)
    worst = []
    for name, wo, bo, k, ci, co in ordn.layer_offsets(s, c_hr):
        ref, got = rg[wo:bo], g[wo:bo]
        cos = got @ ref / (np.linalg.norm(got) * np.linalg.norm(ref) + 1e-30)
        rel = np.linalg.norm(got - ref) / (np.linalg.norm(ref) + 1e-30)
        worst.append((cos, rel, name))
    worst.sort()
    print(f"\nbf16 s={s} c_hr={c_hr}: loss {v:.5f} vs {rv:.5f}, |y - y64| / |y64| = {rel_y:.2e}; "
          f"worst layers {[(n, round(c, 4), round(r_, 4)) for c, r_, n in worst[:4]]}")
    assert rel_y < 2e-2
    assert abs(v - rv) <= 5e-2 * rv
    for cos, rel, name in worst:
        assert cos > 0.95 and rel < 0.35, (name, cos, rel)


def test_rdn_bf16_training_reduces_loss(mrs):
    lr, hr, alb, nrm, ex, tgt = _batch(5, 2, 6, 6, 4)
    L = ordn.unpack(_params(1, 4), 4)
    L[-1] = (L[-1][0] * 0.05, L[-1][1])
    net = mrs.RDN(ordn.pack(L).astype(np.float32), 4)
    dev = _cuda(lr, hr, alb, nrm, tgt)
    losses = [net.train_step(*dev, lr=1e-4, loss="robust", beta=0.1, precision="bf16")
              for _ in range(30)]
    assert losses[-1] < 0.9 * losses[0], losses[::5]
    # the BF16 weights used by inference follow the trained FP32 weights
    c = mrs.RDN(net.get_params(), 4)
    assert torch.equal(net.fuse(*dev[:4], precision="bf16"), c.fuse(*dev[:4], precision="bf16"))


def test_rdn_bf16_recorded_steps_equal_direct_steps(mrs):
    # the first BF16 step of a shape runs its launches directly and records
    # them; later steps replay the recording on the staged batch.  Three steps
    # on one handle (two replayed, each on a different batch) equal three
    # steps that are each the first of a fresh handle, bit for bit
    batches = [_cuda(*_batch(40 + i, 2, 6, 6, 4)[:4], _batch(40 + i, 2, 6, 6, 4)[5]) for i in range(3)]
    p = _params(4, 4)
    a = mrs.RDN(p, 4)
    la = [a.train_step(*b, lr=1e-3, loss="robust", precision="bf16") for b in batches]
    st = {"params": p, "adam_m": np.zeros_like(p), "adam_v": np.zeros_like(p), "step": 0}
    lb = []
    for b in batches:
        c = mrs.RDN(st["params"], 4)
        c.set_state(st)
        lb.append(c.train_step(*b, lr=1e-3, loss="robust", precision="bf16"))
        st = c.get_state()
        c.close()
    assert la == lb
    sa = a.get_state()
    for k in ("params", "adam_m", "adam_v"):
        assert np.array_equal(sa[k], st[k]), k
