"""Pins of the oracle of the method's own fusion network (Sec. 4): the
rearrangements against torch, the 1x1 conv by brute force, and closed forms
of identity-kernel networks that fix the skips and the dense concatenation."""
import numpy as np
import pytest

from oracle import cnn, rdn


def test_param_count_and_flops_by_hand():
    # H_lrhs 1,792 + H_hrls 5,248 + fuse 69,696 + 15 RDBs x 368,896
    # + 2 upsampling convs x 147,712 + H_rec 1,731 (x4, 9 HRLS channels)
    assert rdn.nparams(4) == 5_907_331
    assert rdn.nparams(2) == 5_907_331 - 147_712 - 64 * 64 * 12
    # per LR pixel: 3,456 + 16 x 10,368 + 139,264 + 15 x 737,280
    # + (1 + 4) x 294,912 + 16 x 3,456
    assert rdn.flops_per_lr_pixel(4) == 12_897_664
    names = [n for n, *_ in rdn.layers_for(8)]
    assert names[:3] == ["H_lrhs", "H_hrls", "fuse"] and names[-1] == "H_rec"
    assert len(names) == 3 + 60 + 3 + 1


@pytest.mark.parametrize("C", [1, 5])
def test_deshuffle_and_shuffle_match_torch(C):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(C)
    x = rng.normal(size=(2, 8, 6, C))
    t = torch.from_numpy(x).permute(0, 3, 1, 2)
    want = torch.nn.functional.pixel_unshuffle(t, 2).permute(0, 2, 3, 1).numpy()
    got = rdn.deshuffle(x)
    assert got.shape == (2, 4, 3, 4 * C) and np.array_equal(got, want)
    y = rng.normal(size=(2, 3, 5, 4 * C))
    ty = torch.from_numpy(y).permute(0, 3, 1, 2)
    want = torch.nn.functional.pixel_shuffle(ty, 2).permute(0, 2, 3, 1).numpy()
    assert np.array_equal(rdn.shuffle(y), want)
    assert np.array_equal(rdn.shuffle(rdn.deshuffle(x)), x)


@pytest.mark.parametrize("s", [2, 4, 8])
def test_stacked_deshuffle_index(s):
    # D stacked stride-2 deshuffles: channel k = c * s^2 + sum over steps d of
    # (2 dy_d + dx_d) * 4^(D - d) reads HR pixel (s y + sum dy_d 2^(d-1), ...)
    D = rdn.depth(s)
    rng = np.random.default_rng(s)
    x = rng.normal(size=(1, 2 * s, 3 * s, 2))
    z = x
    for _ in range(D):
        z = rdn.deshuffle(z)
    for k in range(z.shape[-1]):
        c, oy, ox = k >> (2 * D), 0, 0
        for d in range(1, D + 1):
            pair = (k >> (2 * (D - d))) & 3
            oy += (pair >> 1) << (d - 1)
            ox += (pair & 1) << (d - 1)
        assert np.array_equal(z[0, :, :, k], x[0, oy::s, ox::s, c])


def test_conv1x1_equals_brute_force():
    rng = np.random.default_rng(0)
    x = rng.normal(size=(1, 3, 2, 5))
    w = rng.normal(size=(4, 1, 1, 5))
    b = rng.normal(size=4)
    got = rdn.conv1x1(x, w, b)
    for yy in range(3):
        for xx in range(2):
            for o in range(4):
                acc = b[o] + sum(x[0, yy, xx, c] * w[o, 0, 0, c] for c in range(5))
                assert abs(got[0, yy, xx, o] - acc) <= 1e-12


def _zero_layers(s, c_hr=rdn.C_HR):
    return [(np.zeros((co, k, k, ci)), np.zeros(co)) for _, k, ci, co in rdn.layers_for(s, c_hr)]


def _inputs(rng, s, h=3, w=4):
    lr = rng.uniform(0, 2, (1, h, w, 3))
    H, W = h * s, w * s
    return (lr, rng.uniform(0, 2, (1, H, W, 3)), rng.uniform(0, 1, (1, H, W, 3)),
            rng.uniform(-1, 1, (1, H, W, 3)))


@pytest.mark.parametrize("s", [2, 4, 8])
def test_identity_network_closed_form(s):
    # identity kernels carry the LRHS RGB through H_lrhs, the fuse conv, the
    # upsampling convs (nearest-neighbour through the shuffle) and H_Rec; zero
    # RDBs are identities, each RDG doubles its input (group skip) and Eq. F_DF
    # adds F_0 once more: I_SR = (1 + 2^3) * nearest_up_s(LRHS)
    L = _zero_layers(s)
    idx = {n: i for i, (n, *_) in enumerate(rdn.layers_for(s))}
    for c in range(3):
        L[idx["H_lrhs"]][0][c, 1, 1, c] = 1.0
        L[idx["fuse"]][0][c, 0, 0, c] = 1.0
        L[idx["H_rec"]][0][c, 1, 1, c] = 1.0
        for d in range(rdn.depth(s)):
            for sub in range(4):
                L[idx[f"up{d}"]][0][4 * c + sub, 1, 1, c] = 1.0
    rng = np.random.default_rng(s)
    lr, hr, alb, nrm = _inputs(rng, s)
    y = rdn.forward(rdn.pack(L), lr, hr, alb, nrm, s)
    nn = np.repeat(np.repeat(lr, s, axis=1), s, axis=2)
    assert np.allclose(y, 9.0 * nn, rtol=1e-15, atol=0)


def test_rdb_dense_concatenation_closed_form():
    # conv1 = 2 F_in, conv2 = 3 F_1 (second block), conv3 = F_2 / 2 (third),
    # fusion = F_in + 10 F_1 + 100 F_2 + 1000 F_3 = 3621 F_in, so the block
    # returns 3622 F_in; any other concatenation order gives another factor
    def ident(cin, blocks):
        w = np.zeros((64, 3, 3, cin))
        for blk, a in blocks.items():
            for o in range(64):
                w[o, 1, 1, 64 * blk + o] = a
        return w, np.zeros(64)

    convs = [ident(64, {0: 2.0}), ident(128, {1: 3.0}), ident(192, {2: 0.5}),
             ident(256, {0: 1.0, 1: 10.0, 2: 100.0, 3: 1000.0})]
    F = np.random.default_rng(1).uniform(0, 1, (1, 3, 5, 64))
    assert np.allclose(rdn.rdb(F, convs), 3622.0 * F, rtol=1e-14, atol=0)


@pytest.mark.parametrize("s", [2, 4])
def test_fuse_selects_a_deshuffled_hr_pixel(s):
    # H_hrls copies the HRLS RGB; the fuse conv picks channel k of F_HRLS for
    # output 0; the rest is the identity network above with the H_lrhs path
    # off, so I_SR = 9 * nearest_up_s(that HR sub-pixel of the HRLS red)
    L = _zero_layers(s)
    idx = {n: i for i, (n, *_) in enumerate(rdn.layers_for(s))}
    for c in range(3):
        L[idx["H_hrls"]][0][c, 1, 1, c] = 1.0
    D = rdn.depth(s)
    k = s * s - 1                        # channel 0, last sub-pixel: offset (s-1, s-1)
    L[idx["fuse"]][0][0, 0, 0, 64 + k] = 1.0
    L[idx["H_rec"]][0][0, 1, 1, 0] = 1.0
    for d in range(D):
        for sub in range(4):
            L[idx[f"up{d}"]][0][sub, 1, 1, 0] = 1.0
    rng = np.random.default_rng(7)
    lr, hr, alb, nrm = _inputs(rng, s)
    y = rdn.forward(rdn.pack(L), lr, hr, alb, nrm, s)
    sub = hr[:, s - 1::s, s - 1::s, 0]
    want = 9.0 * np.repeat(np.repeat(sub, s, axis=1), s, axis=2)
    assert np.allclose(y[..., 0], want, rtol=1e-15, atol=0)
    assert not y[..., 1:].any()


def test_extra_hrls_layers_with_zero_weights_change_nothing():
    s = 2
    rng = np.random.default_rng(3)
    lr, hr, alb, nrm = _inputs(rng, s)
    ex = rng.uniform(0, 1, hr.shape[:3] + (9,))
    p9 = rdn.unpack(rdn.kaiming(0, s, fusion_damp=0.1), s)
    w = np.zeros((64, 3, 3, 18))
    w[..., :9] = p9[1][0]
    p18 = rdn.pack(p9[:1] + [(w, p9[1][1])] + p9[2:])
    a = rdn.forward(rdn.pack(p9), lr, hr, alb, nrm, s)
    b = rdn.forward(p18, lr, hr, alb, nrm, s, extra=ex)
    assert np.array_equal(a, b)
    # and the extra channels do reach the network when their weights are not zero
    w[..., 12] = 1.0
    c = rdn.forward(rdn.pack(p9[:1] + [(w, p9[1][1])] + p9[2:]), lr, hr, alb, nrm, s, extra=ex)
    assert not np.allclose(a, c)


def test_kaiming_network_is_finite_and_local():
    # receptive-field check: changing one LRHS pixel changes I_SR only within
    # the LR receptive field of 1 + 60 + 2 3x3 LR convs (+ the HR-side convs)
    s = 2
    rng = np.random.default_rng(4)
    lr, hr, alb, nrm = _inputs(rng, s, h=40, w=3)
    p = rdn.kaiming(1, s, fusion_damp=0.1)
    a = rdn.forward(p, lr, hr, alb, nrm, s)
    lr2 = lr.copy()
    lr2[0, 0, 0, 0] += 1.0
    b = rdn.forward(p, lr2, hr, alb, nrm, s)
    assert np.isfinite(a).all()
    rows = np.nonzero(np.abs(a - b).max(axis=(0, 2, 3)) > 0)[0]
    # LR rows 0 .. 62 at most (61 LR 3x3 convs before the upsampling conv, one
    # at LR in UP), one more HR row each for the x2 part and H_rec
    assert rows.max() <= s * 63 + 2


def _small_case(s, seed, c_hr=rdn.C_HR, h=2, w=3):
    rng = np.random.default_rng(seed)
    L = rdn.unpack(rdn.kaiming(seed, s, c_hr, fusion_damp=0.3), s, c_hr)
    # small positive biases keep most ReLUs away from their kink
    L = [(wt + rng.normal(0, 0.01, wt.shape), np.full(b.shape, 0.05)) for wt, b in L]
    p = rdn.pack(L)
    H, W = h * s, w * s
    lr = rng.gamma(2.0, 0.5, (1, h, w, 3))
    hr = rng.gamma(1.0, 1.0, (1, H, W, 3))
    alb = rng.uniform(0, 1, (1, H, W, 3))
    nrm = rng.uniform(-1, 1, (1, H, W, 3))
    extra = rng.gamma(1.0, 0.5, (1, H, W, 9)) if c_hr == rdn.C_HR_EXTRA else None
    return p, lr, hr, alb, nrm, extra, rng


@pytest.mark.parametrize("s", [2, 4])
def test_forward_tape_equals_forward(s):
    p, lr, hr, alb, nrm, ex, _ = _small_case(s, 1)
    y, _ = rdn.forward_tape(p, lr, hr, alb, nrm, s, ex)
    assert np.array_equal(y, rdn.forward(p, lr, hr, alb, nrm, s, ex))


@pytest.mark.parametrize("s,c_hr", [(2, rdn.C_HR), (4, rdn.C_HR), (8, rdn.C_HR),
                                    (2, rdn.C_HR_EXTRA)])
def test_backward_matches_finite_differences(s, c_hr):
    # L = sum(I_SR * G): dL/dI_SR = G; central differences of the float64
    # forward at weights and biases of every layer kind (H_lrhs, H_hrls, the
    # fuse conv behind the deshuffles, the four convs of a dense block in the
    # first and the last group, every upsampling conv, H_Rec)
    p, lr, hr, alb, nrm, ex, rng = _small_case(s, 7 + s, c_hr)
    y, tape = rdn.forward_tape(p, lr, hr, alb, nrm, s, ex)
    G = rng.normal(size=y.shape)
    g = rdn.backward(p, tape, G)
    assert g.shape == p.shape
    offs = rdn.layer_offsets(s, c_hr)
    nconv = rdn.N_RDG * rdn.N_RDB * rdn.N_CONV
    pick = offs[:3] + offs[3:7] + offs[3 + nconv - 4:3 + nconv] + offs[3 + nconv:]
    idx = []
    for _, wo, bo, k, ci, co in pick:
        idx += [wo + int(rng.integers(0, bo - wo)), bo + int(rng.integers(0, co))]
    eps = 1e-6
    checked = 0
    for j in idx:
        e = np.zeros_like(p)
        e[j] = eps
        fp = (rdn.forward(p + e, lr, hr, alb, nrm, s, ex) * G).sum()
        fm = (rdn.forward(p - e, lr, hr, alb, nrm, s, ex) * G).sum()
        fd = (fp - fm) / (2 * eps)
        assert abs(g[j] - fd) <= 1e-5 * max(1.0, abs(fd)), (j, g[j], fd)
        checked += fd != 0.0
    assert checked >= len(idx) // 2


def test_backward_last_layer_closed_form():
    # for L = sum(I_SR * G) the H_Rec bias gradient is the per-channel sum of
    # G, and its weight gradient the correlation of G with H_Rec's input,
    # written out with explicit loops
    s = 2
    p, lr, hr, alb, nrm, ex, rng = _small_case(s, 3)
    y, tape = rdn.forward_tape(p, lr, hr, alb, nrm, s, ex)
    G = rng.normal(size=y.shape)
    g = rdn.backward(p, tape, G)
    _, wo, bo, k, ci, co = rdn.layer_offsets(s)[-1]
    assert np.allclose(g[bo:bo + co], G.sum(axis=(0, 1, 2)), rtol=1e-12, atol=1e-12)
    U = tape["rec_in"]
    N, H, W, C = U.shape
    dw = np.zeros((co, 3, 3, ci))
    for o in range(co):
        for dy in range(3):
            for dx in range(3):
                for yy in range(H):
                    for xx in range(W):
                        sy, sx = yy + dy - 1, xx + dx - 1
                        if 0 <= sy < H and 0 <= sx < W:
                            dw[o, dy, dx] += G[0, yy, xx, o] * U[0, sy, sx]
    assert np.allclose(g[wo:bo].reshape(co, 3, 3, ci), dw, rtol=1e-10, atol=1e-12)


def test_loss_and_grad_robust_loss_by_finite_differences():
    s = 2
    p, lr, hr, alb, nrm, ex, rng = _small_case(s, 5)
    target = rng.gamma(1.0, 1.0, (1, 2 * s, 3 * s, 3))
    v, g = rdn.loss_and_grad(p, lr, hr, alb, nrm, target, s, loss="robust", beta=0.1)
    off = rdn.layer_offsets(s)
    for j in (off[0][1] + 5, off[2][2] + 1, off[-1][1] + 17):
        e = np.zeros_like(p)
        e[j] = 1e-6
        vp, _ = rdn.loss_and_grad(p + e, lr, hr, alb, nrm, target, s, loss="robust", beta=0.1)
        vm, _ = rdn.loss_and_grad(p - e, lr, hr, alb, nrm, target, s, loss="robust", beta=0.1)
        fd = (vp - vm) / 2e-6
        assert abs(g[j] - fd) <= 1e-5 * max(1e-3, abs(fd)), (j, g[j], fd)


@pytest.mark.parametrize("s", [2, 4])
def test_backward_abs_terms(s):
    # the |terms| sums that scale the training tolerances: the gradient is
    # unchanged by asking for them; every element obeys |g| <= terms (the
    # triangle inequality over its terms); where every term is non-negative
    # they are the gradient itself: H_Rec's input is a shuffle of ReLU
    # outputs (>= 0), so with dL/dI_SR = G >= 0 its weight and bias rows equal
    # the gradient
    p, lr, hr, alb, nrm, ex, rng = _small_case(s, 11)
    y, tape = rdn.forward_tape(p, lr, hr, alb, nrm, s, ex)
    G = rng.normal(size=y.shape)
    g0 = rdn.backward(p, tape, G)
    g, t = rdn.backward(p, tape, G, abs_terms=True)
    assert np.array_equal(g, g0) and t.shape == g.shape
    assert (np.abs(g) <= t * (1 + 1e-12) + 1e-300).all()
    nz = t > 0
    assert nz.mean() > 0.3
    assert (np.abs(g[nz]) < t[nz] * (1 - 1e-9)).mean() > 0.25    # mixed-sign terms
    Gp = np.abs(G)
    g, t = rdn.backward(p, tape, Gp, abs_terms=True)
    _, wo, bo, k, ci, co = rdn.layer_offsets(s)[-1]
    assert np.allclose(g[wo:bo + co], t[wo:bo + co], rtol=1e-12, atol=0)
