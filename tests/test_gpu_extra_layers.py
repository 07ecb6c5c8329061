"""The fusion network with the extra HRLS layers as input (Sec. 4: the HRLS
carries diffuse, specular and variance layers besides albedo and normal):
21 input channels, through mrs_fuse_extra / mrs_train_step_extra, against the
float64 oracle.

Tolerances as for the 12-channel network: FP32 within 1e-5 * max(1, max|y|)
(outputs with the variance layers reach |y| > 10, where FP32 rounding alone
exceeds 1e-5 absolute);
BF16 / FP8 as PSNR floors against float64; training gradients per layer
within 1e-4 relative (FP32) or cosine > 0.995 (BF16)."""
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


def _inputs(seed, N, h, w, s):
    rng = np.random.default_rng(seed)
    H, W = h * s, w * s
    lr = rng.gamma(2.0, 0.5, (N, h, w, 3)).astype(np.float32)
    hr = rng.gamma(1.0, 1.0, (N, H, W, 3)).astype(np.float32)
    alb = rng.uniform(0, 1, (N, H, W, 3)).astype(np.float32)
    nrm = rng.uniform(-1, 1, (N, H, W, 3)).astype(np.float32)
    # diffuse + specular split of a radiance-like image, and a variance layer
    # spanning orders of magnitude (as a low-spp render's does)
    frac = rng.uniform(0, 1, (N, H, W, 3))
    rad = rng.gamma(1.0, 1.0, (N, H, W, 3))
    var = rng.gamma(0.5, 1.0, (N, H, W, 3)) * 10.0 ** rng.uniform(-3, 1, (N, H, W, 1))
    ex = np.concatenate([rad * frac, rad * (1 - frac), var], axis=-1).astype(np.float32)
    return lr, hr, alb, nrm, ex


def _params(seed, resid_scale=0.25):
    layers = cnn.unpack(cnn.kaiming(seed, c_in=21))
    out = []
    for i, (w, b) in enumerate(layers):
        if 1 <= i <= 16 and i % 2 == 0:
            w = w * resid_scale
        out.append((w, b + 0.01 * (i % 3)))
    return cnn.pack(out).astype(np.float32)


def _cuda(*a):
    return [torch.from_numpy(np.ascontiguousarray(t)).cuda() for t in a]


def _psnr(got, ref):
    mse = np.mean((np.asarray(got, np.float64) - ref) ** 2)
    return float("inf") if mse == 0 else 10 * np.log10(np.ptp(ref) ** 2 / mse)


def test_net_reports_its_input_channels(mrs):
    assert mrs.Net(np.zeros(mrs.NPARAMS, np.float32)).input_channels == 12
    assert mrs.Net(np.zeros(mrs.NPARAMS_EXTRA, np.float32)).input_channels == 21
    assert mrs.NPARAMS_EXTRA == cnn.NPARAMS_EXTRA


@pytest.mark.parametrize("N,h,w,s", [(1, 8, 40, 4), (2, 5, 7, 2)])
def test_fuse_extra_fp32_matches_oracle(mrs, N, h, w, s):
    lr, hr, alb, nrm, ex = _inputs(1, N, h, w, s)
    p = _params(0)
    net = mrs.Net(p)
    c = _cuda(lr, hr, alb, nrm, ex)
    got = net.fuse(*c[:4], s, precision="fp32", extra=c[4]).cpu().numpy()
    ref = cnn.forward(p.astype(np.float64), lr, hr, alb, nrm, s, extra=ex)
    assert np.abs(got - ref).max() <= 1e-5 * max(1.0, np.abs(ref).max()), np.abs(got - ref).max()


@pytest.mark.parametrize("prec,min_psnr", [("bf16", 45.0), ("fp8", 28.0)])
def test_fuse_extra_low_precision_close_to_fp64(mrs, prec, min_psnr):
    N, h, w, s = 1, 16, 48, 4
    lr, hr, alb, nrm, ex = _inputs(2, N, h, w, s)
    p = _params(1)
    net = mrs.Net(p)
    c = _cuda(lr, hr, alb, nrm, ex)
    got = net.fuse(*c[:4], s, precision=prec, extra=c[4]).cpu().numpy()
    ref = cnn.forward(p.astype(np.float64), lr, hr, alb, nrm, s, extra=ex)
    assert _psnr(got, ref) >= min_psnr


def test_zero_extra_weights_reproduce_the_12_channel_net(mrs):
    # a 21-channel net whose extra-channel weights are zero computes the
    # 12-channel net: in FP32 exactly (the extra products are zero and the
    # other terms keep their order), on the tensor cores to within the FP32
    # accumulation's last bits
    lr, hr, alb, nrm, ex = _inputs(3, 1, 8, 24, 4)
    p12 = cnn.unpack(cnn.kaiming(2))
    w0 = np.zeros((64, 3, 3, 21))
    w0[..., :12] = p12[0][0]
    p21 = cnn.pack([(w0, p12[0][1])] + p12[1:]).astype(np.float32)
    c = _cuda(lr, hr, alb, nrm, ex)
    a = mrs.Net(cnn.pack(p12).astype(np.float32))
    b = mrs.Net(p21)
    for prec in ("fp32", "bf16", "fp8"):
        ya = a.fuse(*c[:4], 4, precision=prec).cpu().numpy()
        yb = b.fuse(*c[:4], 4, precision=prec, extra=c[4]).cpu().numpy()
        if prec == "fp8":
            # per-layer FP8 scales are calibrated from the first input's
            # amax, which the extra channels may raise for the input layer
            assert _psnr(yb, ya) >= 28.0
        elif prec == "bf16":
            assert np.abs(ya - yb).max() <= 1e-6 * np.abs(ya).max()
        else:
            assert np.array_equal(ya, yb)


def test_extra_argument_must_match_the_net(mrs):
    lr, hr, alb, nrm, ex = _inputs(4, 1, 4, 4, 2)
    c = _cuda(lr, hr, alb, nrm, ex)
    n12 = mrs.Net(np.zeros(mrs.NPARAMS, np.float32))
    n21 = mrs.Net(np.zeros(mrs.NPARAMS_EXTRA, np.float32))
    with pytest.raises(Exception):
        n12.fuse(*c[:4], 2, precision="fp32", extra=c[4])
    with pytest.raises(Exception):
        n21.fuse(*c[:4], 2, precision="fp32")
    with pytest.raises(Exception):
        mrs.train_step(n21, *c[:4], c[3], 2)


@pytest.mark.parametrize("loss", ["l1log", "robust"])
def test_train_step_extra_matches_oracle(mrs, loss):
    N, h, w, s = 2, 4, 6, 4
    lr, hr, alb, nrm, ex = _inputs(5, N, h, w, s)
    ex[0, 0, 0, 0] = 300.0              # a diffuse firefly above the clip level
    tgt = np.random.default_rng(6).gamma(2.0, 0.5, hr.shape).astype(np.float32)
    p = _params(3)
    net = mrs.Net(p)
    c = _cuda(lr, hr, alb, nrm, ex, tgt)
    val = mrs.train_step(net, *c[:4], c[5], s, lr=1e-3, loss=loss, extra=c[4])
    g = mrs.get_grads(net)
    p1 = net.get_params()
    z = np.zeros(cnn.NPARAMS_EXTRA)
    rp, _, _, rloss, rg = cnn.train_step(p.astype(np.float64), z, z, 1, 1e-3, lr, hr, alb, nrm, tgt,
                                         s, loss=loss, extra=ex)
    assert abs(val - rloss) <= 1e-6 * rloss
    for li, (wo, bo, ci, co) in enumerate(cnn.layer_offsets(21)):
        for a, b in ((wo, bo), (bo, bo + co)):
            ref = rg[a:b]
            err = np.linalg.norm(g[a:b] - ref) / max(np.linalg.norm(ref), 1e-30)
            assert err < 1e-4, (li, a, err)
    ok = np.abs(rg) > 1e-6
    assert np.abs((p1 - p) - (rp - p))[ok].max() <= 0.01 * 1e-3


def test_bf16_train_step_extra_close_to_oracle(mrs):
    N, h, w, s = 2, 8, 16, 4
    lr, hr, alb, nrm, ex = _inputs(7, N, h, w, s)
    tgt = np.random.default_rng(8).gamma(2.0, 0.5, hr.shape).astype(np.float32)
    p = _params(4)
    net = mrs.Net(p)
    c = _cuda(lr, hr, alb, nrm, ex, tgt)
    val = mrs.train_step(net, *c[:4], c[5], s, lr=1e-3, precision="bf16", extra=c[4])
    g = mrs.get_grads(net)
    z = np.zeros(cnn.NPARAMS_EXTRA)
    _, _, _, rloss, rg = cnn.train_step(p.astype(np.float64), z, z, 1, 1e-3, lr, hr, alb, nrm, tgt, s,
                                        extra=ex)
    assert abs(val - rloss) <= 2e-2 * rloss
    for li, (wo, bo, _, _) in enumerate(cnn.layer_offsets(21)):
        ref, got = rg[wo:bo], g[wo:bo].astype(np.float64)
        cos = got @ ref / (np.linalg.norm(got) * np.linalg.norm(ref) + 1e-30)
        rel = np.linalg.norm(got - ref) / (np.linalg.norm(ref) + 1e-30)
        assert cos > 0.995 and rel < 0.1, (li, cos, rel)


def test_rendered_layers_feed_the_network(mrs):
    # end to end on the device: an HRLS render with its extra layers goes
    # straight into the 21-channel network; the oracle fuses the same buffers
    from synth import scenes
    desc = scenes.cornell_box(sphere_subdiv=2)
    sc = mrs.Scene(desc)
    s = 4
    lo = mrs.render(sc, 8, 8, 16, 3, seed=1, counts=False)
    hi = mrs.render(sc, 32, 32, 2, 3, seed=2, counts=False, layers=True)
    ex = torch.cat([hi["diffuse"], hi["specular"], hi["variance"]], dim=-1)[None].contiguous()
    args = [lo["radiance"][None], hi["radiance"][None], hi["albedo"][None], hi["normal"][None]]
    args = [a.contiguous() for a in args]
    p = _params(5)
    net = mrs.Net(p)
    got = net.fuse(*args, s, precision="fp32", extra=ex).cpu().numpy()
    host = [a.cpu().numpy() for a in args]
    ref = cnn.forward(p.astype(np.float64), *host, s, extra=ex.cpu().numpy())
    assert np.abs(got - ref).max() <= 1e-5 * max(1.0, np.abs(ref).max()), np.abs(got - ref).max()
