"""Oracle pins for the fusion network: convolution by brute force, bilinear
upsampling by torch, special cases, finite-difference gradients, Adam."""
import numpy as np
import pytest

from oracle import cnn


def test_param_count():
    assert cnn.NPARAMS == 12 * 9 * 64 + 64 + 16 * (64 * 9 * 64 + 64) + 64 * 9 * 3 + 3
    offs = cnn.layer_offsets()
    assert len(offs) == 18 and offs[-1][1] + 3 == cnn.NPARAMS


def test_conv_equals_brute_force_loops():
    rng = np.random.default_rng(0)
    x = rng.normal(size=(2, 5, 4, 3))
    w = rng.normal(size=(2, 3, 3, 3))
    b = rng.normal(size=2)
    got = cnn.conv3x3(x, w, b)
    N, H, W, C = x.shape
    want = np.zeros((N, H, W, 2))
    for n in range(N):
        for y in range(H):
            for xx in range(W):
                for o in range(2):
                    acc = b[o]
                    for dy in range(3):
                        for dx in range(3):
                            yy, xs = y + dy - 1, xx + dx - 1
                            if 0 <= yy < H and 0 <= xs < W:
                                for c in range(C):
                                    acc += x[n, yy, xs, c] * w[o, dy, dx, c]
                    want[n, y, xx, o] = acc
    assert np.allclose(got, want, rtol=0, atol=1e-12)


@pytest.mark.parametrize("s", [2, 4])
def test_bilinear_matches_torch(s):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(s)
    x = rng.uniform(0, 3, (2, 5, 7, 3))
    got = cnn.bilinear_up(x, s)
    t = torch.nn.functional.interpolate(torch.from_numpy(x).permute(0, 3, 1, 2), scale_factor=s,
                                        mode="bilinear", align_corners=False)
    assert np.allclose(got, t.permute(0, 2, 3, 1).numpy(), rtol=0, atol=1e-12)


def _inputs(rng, N=1, h=4, w=4, s=2):
    lr = rng.uniform(0, 2, (N, h, w, 3))
    hr = rng.uniform(0, 2, (N, h * s, w * s, 3))
    alb = rng.uniform(0, 1, (N, h * s, w * s, 3))
    nrm = rng.uniform(-1, 1, (N, h * s, w * s, 3))
    return lr, hr, alb, nrm


def test_zero_weights_give_upsampled_lrhs():
    rng = np.random.default_rng(1)
    lr, hr, alb, nrm = _inputs(rng)
    y = cnn.forward(np.zeros(cnn.NPARAMS), lr, hr, alb, nrm, 2)
    assert np.array_equal(y, cnn.bilinear_up(lr, 2))


def test_identity_kernel_reproduces_input():
    rng = np.random.default_rng(2)
    x = rng.normal(size=(1, 6, 5, 4))
    w = np.zeros((4, 3, 3, 4))
    for c in range(4):
        w[c, 1, 1, c] = 1.0
    assert np.array_equal(cnn.conv3x3(x, w, np.zeros(4)), x)


def test_residual_structure_with_identity_layers():
    # conv_in = identity on the first 12 channels, every block's second conv 0,
    # conv_out reads back channels 3..5 (HRLS): y = up(LRHS) + relu(HRLS) = up + HRLS
    rng = np.random.default_rng(3)
    lr, hr, alb, nrm = _inputs(rng)
    L = [(np.zeros((co, 3, 3, ci)), np.zeros(co)) for ci, co in cnn.LAYERS]
    for c in range(12):
        L[0][0][c, 1, 1, c] = 1.0
    for k in range(3):
        L[-1][0][k, 1, 1, 3 + k] = 1.0
    y = cnn.forward(cnn.pack(L), lr, hr, alb, nrm, 2)
    assert np.allclose(y, cnn.bilinear_up(lr, 2) + hr, rtol=0, atol=1e-14)


def test_loss_gradient_matches_finite_differences():
    rng = np.random.default_rng(4)
    pred = rng.uniform(-0.5, 3, (1, 3, 3, 3))
    tgt = rng.uniform(0, 3, (1, 3, 3, 3))
    _, g = cnn.l1log_loss(pred, tgt)
    h = 1e-7
    for idx in np.ndindex(pred.shape):
        if abs(pred[idx]) < 1e-3:
            continue
        p1, p0 = pred.copy(), pred.copy()
        p1[idx] += h
        p0[idx] -= h
        fd = (cnn.l1log_loss(p1, tgt)[0] - cnn.l1log_loss(p0, tgt)[0]) / (2 * h)
        assert abs(fd - g[idx]) < 1e-7


def test_network_gradient_matches_finite_differences():
    rng = np.random.default_rng(5)
    lr, hr, alb, nrm = _inputs(rng, N=1, h=4, w=4, s=2)
    tgt = rng.uniform(0, 2, hr.shape)
    params = cnn.kaiming(0) * 0.5 + rng.normal(0, 0.01, cnn.NPARAMS)
    loss, g = cnn.loss_and_grad(params, lr, hr, alb, nrm, tgt, 2)
    h = 1e-6
    offs = cnn.layer_offsets()
    picks = []
    for li in (0, 1, 2, 9, 16, 17):
        wo, bo, ci, co = offs[li]
        picks += list(rng.integers(wo, bo, 4)) + [bo]
    for i in picks:
        p1, p0 = params.copy(), params.copy()
        p1[i] += h
        p0[i] -= h
        fd = (cnn.loss_and_grad(p1, lr, hr, alb, nrm, tgt, 2)[0]
              - cnn.loss_and_grad(p0, lr, hr, alb, nrm, tgt, 2)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1e-3, abs(g[i])) + 1e-9, (i, fd, g[i])


def test_adam_first_step_closed_form():
    # with zero moments, step 1 moves every parameter by lr * g / (|g| + eps)
    rng = np.random.default_rng(6)
    p = rng.normal(size=100)
    g = rng.normal(size=100)
    p1, m, v = cnn.adam(p, g, np.zeros(100), np.zeros(100), 1, 1e-3)
    assert np.allclose(p1, p - 1e-3 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_kaiming_statistics():
    p = cnn.unpack(cnn.kaiming(0))
    w = p[1][0]
    assert abs(w.std() - np.sqrt(2 / 576)) < 0.01 * np.sqrt(2 / 576) * 5
    assert all((b == 0).all() for _, b in p)


def test_train_step_clips_inputs_and_target():
    # with everything below the clip level, the clipped step equals the plain one;
    # scaling the inputs far above it leaves the clipped step unchanged
    rng = np.random.default_rng(7)
    lr, hr, alb, nrm = _inputs(rng, N=1, h=2, w=2, s=2)
    tgt = rng.uniform(0, 2, hr.shape)
    p = cnn.kaiming(1) * 0.3
    z = np.zeros_like(p)
    a = cnn.train_step(p, z, z, 1, 1e-3, lr, hr, alb, nrm, tgt, 2)
    loss, grad = cnn.loss_and_grad(p, lr, hr, alb, nrm, tgt, 2)
    assert a[3] == loss and np.array_equal(a[4], grad)
    big = cnn.train_step(p, z, z, 1, 1e-3, lr + 500, hr + 500, alb, nrm, tgt + 500, 2)
    ref = cnn.loss_and_grad(p, np.full_like(lr, 100.0), np.full_like(hr, 100.0), alb, nrm,
                            np.full_like(tgt, 100.0), 2)
    assert big[3] == ref[0] and np.array_equal(big[4], ref[1])


def test_slog_loss_extends_log1p():
    # for non-negative values the loss is L1 on log(1 + x); slog is odd and monotone
    rng = np.random.default_rng(8)
    a = rng.uniform(0, 5, 50)
    b = rng.uniform(0, 5, 50)
    loss, _ = cnn.l1log_loss(a, b)
    assert abs(loss - np.mean(np.abs(np.log1p(a) - np.log1p(b)))) < 1e-15
    x = np.linspace(-5, 5, 1001)
    assert np.array_equal(cnn.slog(-x), -cnn.slog(x)) and (np.diff(cnn.slog(x)) > 0).all()
    # negative predictions keep a gradient pointing back up
    _, g = cnn.l1log_loss(np.array([-0.5]), np.array([1.0]))
    assert g[0] < 0 and abs(g[0] + 1 / 1.5) < 1e-15


def test_robust_loss_closed_forms():
    # a constant error e on every value gives exactly e / (beta + e), whatever
    # the size: 1/2 at e = beta, 3/4 at e = 3 beta
    tgt = np.random.default_rng(10).uniform(0, 4, (2, 5, 7, 3))
    for e, want in ((0.1, 0.5), (0.3, 0.75), (-0.1, 0.5)):
        loss, _ = cnn.robust_loss(tgt + e, tgt, beta=0.1)
        assert abs(loss - want) < 1e-12, (e, loss)
    # bounded by 1 for huge errors, ~|e| / beta for tiny ones, 0 at e = 0
    loss, _ = cnn.robust_loss(tgt + 1e6, tgt, beta=0.1)
    assert 0.9999 < loss < 1.0
    loss, g = cnn.robust_loss(tgt + 1e-7, tgt, beta=0.1)
    assert abs(loss - 1e-6) < 1e-11
    loss, g = cnn.robust_loss(tgt, tgt, beta=0.1)
    assert loss == 0.0 and not g.any()
    # symmetric: the gradient flips sign with the error
    _, gp = cnn.robust_loss(tgt + 0.2, tgt)
    _, gm = cnn.robust_loss(tgt - 0.2, tgt)
    assert np.allclose(gp, -gm, rtol=0, atol=1e-15) and (gp > 0).all()


def test_robust_loss_gradient_matches_finite_differences():
    rng = np.random.default_rng(11)
    pred = rng.uniform(-0.5, 3, (1, 3, 3, 3))
    tgt = rng.uniform(0, 3, (1, 3, 3, 3))
    _, g = cnn.robust_loss(pred, tgt, beta=0.1)
    h = 1e-7
    for idx in np.ndindex(pred.shape):
        if abs(pred[idx] - tgt[idx]) < 1e-3:
            continue
        p1, p0 = pred.copy(), pred.copy()
        p1[idx] += h
        p0[idx] -= h
        fd = (cnn.robust_loss(p1, tgt)[0] - cnn.robust_loss(p0, tgt)[0]) / (2 * h)
        assert abs(fd - g[idx]) < 1e-7 * max(1.0, abs(g[idx]))


def test_network_gradient_robust_loss_matches_finite_differences():
    rng = np.random.default_rng(12)
    lr, hr, alb, nrm = _inputs(rng, N=1, h=4, w=4, s=2)
    tgt = rng.uniform(0, 2, hr.shape)
    params = cnn.kaiming(1) * 0.5 + rng.normal(0, 0.01, cnn.NPARAMS)
    _, g = cnn.loss_and_grad(params, lr, hr, alb, nrm, tgt, 2, loss="robust", beta=0.1)
    h = 1e-6
    offs = cnn.layer_offsets()
    for li in (0, 5, 17):
        wo, bo, _, _ = offs[li]
        for i in list(rng.integers(wo, bo, 3)) + [bo]:
            p1, p0 = params.copy(), params.copy()
            p1[i] += h
            p0[i] -= h
            fd = (cnn.loss_and_grad(p1, lr, hr, alb, nrm, tgt, 2, loss="robust")[0]
                  - cnn.loss_and_grad(p0, lr, hr, alb, nrm, tgt, 2, loss="robust")[0]) / (2 * h)
            assert abs(fd - g[i]) <= 1e-6 * max(1e-3, abs(g[i])) + 1e-9, (i, fd, g[i])


def _extra(rng, N, H, W):
    d = rng.uniform(0, 2, (N, H, W, 3))
    sp = rng.uniform(0, 1, (N, H, W, 3))
    v = rng.gamma(0.5, 2.0, (N, H, W, 3))
    return np.concatenate([d, sp, v], axis=-1)


def test_extra_input_zero_weights_reduce_to_base_network():
    # a 21-channel network whose layer-0 weights on the 9 extra channels are
    # zero is the 12-channel network: the extra layers are appended after the
    # base channels and nothing else changes
    rng = np.random.default_rng(20)
    lr, hr, alb, nrm = _inputs(rng, N=1, h=4, w=5, s=2)
    ex = _extra(rng, 1, 8, 10)
    base = cnn.kaiming(3) * 0.5
    L = cnn.unpack(base)
    w0, b0 = L[0]
    w0x = np.concatenate([w0, np.zeros(w0.shape[:3] + (cnn.C_EXTRA,))], axis=-1)
    px = cnn.pack([(w0x, b0)] + L[1:])
    assert px.size == cnn.NPARAMS_EXTRA and cnn.input_channels(px) == 21
    assert np.array_equal(cnn.forward(px, lr, hr, alb, nrm, 2, extra=ex),
                          cnn.forward(base, lr, hr, alb, nrm, 2))
    with pytest.raises(ValueError):
        cnn.forward(px, lr, hr, alb, nrm, 2)
    with pytest.raises(ValueError):
        cnn.forward(base, lr, hr, alb, nrm, 2, extra=ex)


@pytest.mark.parametrize("ch,value,want", [(12, 0.7, 0.7), (17, 0.25, 0.25),
                                           (18, np.e - 1.0, 1.0), (20, 0.0, 0.0)])
def test_extra_input_channel_order(ch, value, want):
    # a network whose first layer only passes input channel `ch` through its
    # centre tap (to feature 0, then identity to the output) sees diffuse at
    # 12-14, specular at 15-17 and log(1 + variance) at 18-20
    rng = np.random.default_rng(21)
    lr, hr, alb, nrm = _inputs(rng, N=1, h=3, w=3, s=2)
    ex = _extra(rng, 1, 6, 6)
    ex[..., ch - 12] = value
    layers = [(np.zeros((co, 3, 3, ci)), np.zeros(co)) for ci, co in cnn.layers_for(21)]
    layers[0][0][0, 1, 1, ch] = 1.0
    layers[-1][0][0, 1, 1, 0] = 1.0
    p = cnn.pack(layers)
    y = cnn.forward(p, np.zeros_like(lr), hr, alb, nrm, 2, extra=ex)
    assert np.allclose(y[..., 0], want, rtol=0, atol=1e-12), (ch, y[..., 0].max())


def test_extra_input_network_gradient_matches_finite_differences():
    rng = np.random.default_rng(22)
    lr, hr, alb, nrm = _inputs(rng, N=1, h=3, w=4, s=2)
    ex = _extra(rng, 1, 6, 8)
    tgt = rng.uniform(0, 2, hr.shape)
    params = cnn.kaiming(4, c_in=21) * 0.5 + rng.normal(0, 0.01, cnn.NPARAMS_EXTRA)
    _, g = cnn.loss_and_grad(params, lr, hr, alb, nrm, tgt, 2, extra=ex)
    h = 1e-6
    wo, bo, _, _ = cnn.layer_offsets(21)[0]
    # layer-0 weights on the extra channels (c = 12..20) and a few elsewhere
    picks = [wo + ((o * 3 + 1) * 3 + 1) * 21 + c for o, c in ((0, 12), (5, 16), (9, 20))]
    picks += [int(i) for i in rng.integers(bo, cnn.NPARAMS_EXTRA, 4)]
    for i in picks:
        p1, p0 = params.copy(), params.copy()
        p1[i] += h
        p0[i] -= h
        fd = (cnn.loss_and_grad(p1, lr, hr, alb, nrm, tgt, 2, extra=ex)[0]
              - cnn.loss_and_grad(p0, lr, hr, alb, nrm, tgt, 2, extra=ex)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1e-3, abs(g[i])) + 1e-9, (i, fd, g[i])
