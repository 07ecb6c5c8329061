"""Float64 oracle of the fusion network (forward, backward, loss, Adam).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The network fuses a low-resolution/high-spp render (LRHS) with a
high-resolution/low-spp render (HRLS) and its auxiliary layers into the
high-resolution image I_SR (problem statement of Sec. 4).  Its architecture
is the all-high-resolution variant: bilinear x s upsampling of LRHS,
concatenation with HRLS RGB, albedo and normal (12 channels), a 3x3 conv to
64 channels + ReLU, 8 residual blocks x + conv(relu(conv(x))), and a 3x3 conv
to 3 channels added to the upsampled LRHS.  All kernels are 3x3 with 64
feature channels (Sec. 4, "Implement details").

Parameter layout (flat float array, NPARAMS values): for each of the 18 convs
in forward order, the weight in [Cout][3][3][Cin] order followed by the bias
[Cout].

Pins (tests/test_oracle_cnn.py): convolution equals brute-force loops on tiny
inputs; bilinear upsampling equals torch's interpolate (align_corners=False);
zero weights give out == up(LRHS) exactly; identity-kernel convs reproduce
their input; gradients equal central finite differences.
"""
from __future__ import annotations

import numpy as np

C_IN = 12
C_EXTRA = 9          # diffuse, specular, log(1 + variance) of the HRLS (Sec. 4)
C_F = 64
N_BLOCKS = 8


def layers_for(c_in=C_IN):
    return [(c_in, C_F)] + [(C_F, C_F)] * (2 * N_BLOCKS) + [(C_F, 3)]


LAYERS = layers_for(C_IN)


def layer_offsets(c_in=C_IN):
    """[(w_off, b_off, cin, cout)] into the flat parameter array."""
    offs, o = [], 0
    for cin, cout in layers_for(c_in):
        offs.append((o, o + cout * 9 * cin, cin, cout))
        o += cout * 9 * cin + cout
    return offs


def nparams(c_in=C_IN):
    return sum(co * 9 * ci + co for ci, co in layers_for(c_in))


NPARAMS = nparams(C_IN)
NPARAMS_EXTRA = nparams(C_IN + C_EXTRA)


def input_channels(params):
    """12 (base input) or 21 (with the extra HRLS layers), from the size."""
    n = len(params)
    if n == NPARAMS:
        return C_IN
    if n == NPARAMS_EXTRA:
        return C_IN + C_EXTRA
    raise ValueError(f"{n} parameters: expected {NPARAMS} or {NPARAMS_EXTRA}")


def unpack(params):
    p = np.asarray(params, dtype=np.float64)
    out = []
    for wo, bo, ci, co in layer_offsets(input_channels(p)):
        out.append((p[wo:bo].reshape(co, 3, 3, ci), p[bo:bo + co]))
    return out


def pack(layers):
    return np.concatenate([np.concatenate([w.ravel(), b.ravel()]) for w, b in layers])


def conv3x3(x, w, b):
    """NHWC 3x3 convolution, zero padding 1: out[n,y,x,o] = b[o] +
    sum_{dy,dx,c} in[n, y+dy-1, x+dx-1, c] * w[o, dy, dx, c]."""
    x = np.asarray(x, dtype=np.float64)
    N, H, W, _ = x.shape
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (0, 0)))
    out = np.broadcast_to(b, (N, H, W, w.shape[0])).copy()
    for dy in range(3):
        for dx in range(3):
            out += xp[:, dy:dy + H, dx:dx + W, :] @ w[:, dy, dx, :].T
    return out


def conv3x3_backward(x, w, dout):
    """Gradients of conv3x3 w.r.t. input, weight and bias."""
    x = np.asarray(x, dtype=np.float64)
    N, H, W, _ = x.shape
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (0, 0)))
    dxp = np.zeros_like(xp)
    dw = np.zeros_like(w)
    for dy in range(3):
        for dx in range(3):
            win = xp[:, dy:dy + H, dx:dx + W, :]
            dw[:, dy, dx, :] = np.einsum("nyxo,nyxc->oc", dout, win)
            dxp[:, dy:dy + H, dx:dx + W, :] += dout @ w[:, dy, dx, :]
    return dxp[:, 1:-1, 1:-1, :], dw, dout.sum(axis=(0, 1, 2))


def _src_index(dst, s, n_in):
    src = (dst + 0.5) / s - 0.5
    src = np.maximum(src, 0.0)
    i0 = np.floor(src).astype(np.int64)
    i0 = np.minimum(i0, n_in - 1)
    i1 = np.minimum(i0 + 1, n_in - 1)
    return i0, i1, src - i0


def bilinear_up(x, s):
    """Bilinear x s upsampling with half-pixel centres, clamped at the edges:
    src = max(0, (dst + 0.5) / s - 0.5) (align_corners=False semantics)."""
    x = np.asarray(x, dtype=np.float64)
    N, h, w, C = x.shape
    y0, y1, ly = _src_index(np.arange(h * s), s, h)
    x0, x1, lx = _src_index(np.arange(w * s), s, w)
    ly = ly[None, :, None, None]
    lx = lx[None, None, :, None]
    top = x[:, y0][:, :, x0] * (1 - lx) + x[:, y0][:, :, x1] * lx
    bot = x[:, y1][:, :, x0] * (1 - lx) + x[:, y1][:, :, x1] * lx
    return top * (1 - ly) + bot * ly


def extra_input(extra):
    """The extra HRLS layers as network input channels: extra [N,H,W,9] =
    diffuse, specular, variance as rendered -> diffuse, specular,
    log(1 + variance) (the variance spans orders of magnitude)."""
    e = np.asarray(extra, dtype=np.float64)
    return np.concatenate([e[..., :6], np.log1p(np.maximum(e[..., 6:9], 0.0))], axis=-1)


def fusion_input(lrhs, hrls, albedo, normal, s, extra=None):
    """Network input: up(LRHS), HRLS, albedo, normal (12 channels), then the
    extra layers (9 more) when given."""
    up = bilinear_up(lrhs, s)
    parts = [up, hrls, albedo, normal] + ([extra_input(extra)] if extra is not None else [])
    return np.concatenate(parts, axis=-1).astype(np.float64), up


def forward(params, lrhs, hrls, albedo, normal, s, keep=False, extra=None):
    """I_SR for batched NHWC inputs (LRHS [N,h,w,3]; the rest [N,s*h,s*w,3];
    extra [N,s*h,s*w,9] for a network with the extra-layer input)."""
    L = unpack(params)
    if (extra is not None) != (L[0][0].shape[3] == C_IN + C_EXTRA):
        raise ValueError("extra layers must be given exactly for a 21-channel network")
    x0, up = fusion_input(lrhs, hrls, albedo, normal, s, extra)
    acts = {"x0": x0}
    a = conv3x3(x0, *L[0])
    acts["pre0"] = a
    h = np.maximum(a, 0.0)
    acts["h0"] = h
    for k in range(N_BLOCKS):
        a1 = conv3x3(h, *L[1 + 2 * k])
        r = np.maximum(a1, 0.0)
        h = h + conv3x3(r, *L[2 + 2 * k])
        acts[f"a{k}"] = a1
        acts[f"r{k}"] = r
        acts[f"h{k + 1}"] = h
    y = conv3x3(h, *L[-1]) + up
    return (y, acts) if keep else y


def slog(x):
    """sign(x) * log1p(|x|): log(1 + radiance) extended oddly to negative values."""
    return np.sign(x) * np.log1p(np.abs(x))


def l1log_loss(pred, target):
    """mean |slog(pred) - slog(target)| and its gradient w.r.t. pred,
    sign(d) / (1 + |pred|) / n (subgradient 0 where d = 0).  For non-negative
    values slog is log(1 + x), the L1-on-log(1+radiance) loss."""
    pred = np.asarray(pred, dtype=np.float64)
    target = np.asarray(target, dtype=np.float64)
    d = slog(pred) - slog(target)
    n = pred.size
    loss = np.abs(d).sum() / n
    g = np.sign(d) / (1.0 + np.abs(pred)) / n
    return loss, g


def robust_loss(pred, target, beta=0.1):
    """The robust loss l_r of the method's training (Sec. 3, "Loss function"):
    mean over all pixel-channel values of |e| / (beta + |e|), e = pred - target,
    and its gradient w.r.t. pred, sign(e) * beta / (beta + |e|)^2 / n
    (subgradient 0 where e = 0).  Close to |e| / beta for small errors and
    always below 1 for large ones."""
    pred = np.asarray(pred, dtype=np.float64)
    target = np.asarray(target, dtype=np.float64)
    e = pred - target
    a = np.abs(e)
    n = pred.size
    loss = (a / (beta + a)).sum() / n
    g = np.sign(e) * beta / (beta + a) ** 2 / n
    return loss, g


LOSSES = {"l1log": 0, "robust": 1}


def loss_fn(pred, target, loss="l1log", beta=0.1):
    if loss == "l1log":
        return l1log_loss(pred, target)
    if loss == "robust":
        return robust_loss(pred, target, beta)
    raise ValueError(f"unknown loss {loss!r}")


def _abs_terms(x, dout):
    """Sums of |terms| of a layer's weight and bias gradients: for dW[o,t,c]
    sum_p |dout[p,o]| |x[p+t,c]|, for db[o] sum_p |dout[p,o]| (the scale of
    their floating-point rounding error, for tolerances)."""
    zero = np.zeros((dout.shape[3], 3, 3, x.shape[3]))
    _, aw, ab = conv3x3_backward(np.abs(x), zero, np.abs(dout))
    return aw, ab


def backward(params, acts, dy, abs_terms=False):
    """Gradient of the loss w.r.t. the flat params, given dL/dI_SR.  With
    abs_terms, also the sum of |terms| of every gradient element, in the same
    layout (see _abs_terms)."""
    L = unpack(params)
    grads = [None] * len(L)
    scale = [None] * len(L)
    h = acts[f"h{N_BLOCKS}"]
    dh, dw, db = conv3x3_backward(h, L[-1][0], dy)
    grads[-1] = (dw, db)
    if abs_terms:
        scale[-1] = _abs_terms(h, dy)
    for k in reversed(range(N_BLOCKS)):
        r = acts[f"r{k}"]
        dr, dw2, db2 = conv3x3_backward(r, L[2 + 2 * k][0], dh)
        grads[2 + 2 * k] = (dw2, db2)
        da = dr * (acts[f"a{k}"] > 0.0)
        hin = acts[f"h{k}"]
        dhin, dw1, db1 = conv3x3_backward(hin, L[1 + 2 * k][0], da)
        grads[1 + 2 * k] = (dw1, db1)
        if abs_terms:
            scale[2 + 2 * k] = _abs_terms(r, dh)
            scale[1 + 2 * k] = _abs_terms(hin, da)
        dh = dh + dhin
    da0 = dh * (acts["pre0"] > 0.0)
    _, dw0, db0 = conv3x3_backward(acts["x0"], L[0][0], da0)
    grads[0] = (dw0, db0)
    if abs_terms:
        scale[0] = _abs_terms(acts["x0"], da0)
        return pack(grads), pack(scale)
    return pack(grads)


def loss_and_grad(params, lrhs, hrls, albedo, normal, target, s, loss="l1log", beta=0.1,
                  extra=None, abs_terms=False):
    y, acts = forward(params, lrhs, hrls, albedo, normal, s, keep=True, extra=extra)
    value, dy = loss_fn(y, target, loss, beta)
    return value, backward(params, acts, dy, abs_terms)


def adam(params, grad, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One bias-corrected Adam update (Kingma & Ba 2015); step counts from 1."""
    m = beta1 * m + (1 - beta1) * grad
    v = beta2 * v + (1 - beta2) * grad * grad
    mh = m / (1 - beta1 ** step)
    vh = v / (1 - beta2 ** step)
    return params - lr * mh / (np.sqrt(vh) + eps), m, v


def train_step(params, m, v, step, lr, lrhs, hrls, albedo, normal, target, s, clip=100.0,
               loss="l1log", beta=0.1, extra=None, abs_terms=False):
    """One training step as the method's learned part runs it: radiance inputs
    and target clipped at `clip` (firefly clipping, Sec. 3.2), the loss
    ("l1log", or "robust" = l_r with factor `beta`, Sec. 3), backward,
    bias-corrected Adam at step `step` (counting from 1).  The extra layers'
    diffuse and specular radiance are clipped like the HRLS.
    Returns (new params, m, v, loss, grad), and with abs_terms also the sum of
    |terms| of every gradient element (a rounding-error scale for tests)."""
    lr_c = np.minimum(np.asarray(lrhs, np.float64), clip)
    hr_c = np.minimum(np.asarray(hrls, np.float64), clip)
    tg_c = np.minimum(np.asarray(target, np.float64), clip)
    ex_c = None
    if extra is not None:
        ex_c = np.asarray(extra, np.float64).copy()
        ex_c[..., :6] = np.minimum(ex_c[..., :6], clip)
    value, grad = loss_and_grad(params, lr_c, hr_c, albedo, normal, tg_c, s, loss, beta, ex_c,
                                abs_terms)
    scale = None
    if abs_terms:
        grad, scale = grad
    p1, m1, v1 = adam(params, grad, m, v, step, lr)
    if abs_terms:
        return p1, m1, v1, value, grad, scale
    return p1, m1, v1, value, grad


def kaiming(seed: int, c_in: int = C_IN):
    """Kaiming-normal weights (std sqrt(2 / (9 Cin))), zero biases."""
    rng = np.random.default_rng(np.random.SeedSequence([0x6B61696D, int(seed)]))
    layers = []
    for ci, co in layers_for(c_in):
        layers.append((rng.normal(0, np.sqrt(2.0 / (9 * ci)), (co, 3, 3, ci)), np.zeros(co)))
    return pack(layers)
