"""Float64 oracle of the method's own fusion network (Sec. 4, "two-encoder-one-
decoder" network of Fig. network): forward and backward passes.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Steps, in the order and notation of Sec. 4:
  F_LRHS   = H_lrhs(I_LRHS)                      3x3 conv, 3 -> 64, at LR
  F0_HRLS  = H_hrls(I_HRLS)                      3x3 conv, C_h -> 64, at HR
  F_HRLS   = DSF^D(... DSF^1(F0_HRLS))           D = log2(s) deshuffle layers, alpha = 2
  F_0      = fuse(F_LRHS || F_HRLS)              1x1 conv, 64 + 64 s^2 -> 64
  F_g      = RDB_B(... RDB_1(F_{g-1})) + F_{g-1} G = 3 residual dense groups of B = 5 blocks
  F_DF     = F_G + F_0                           (Eq. F_DF)
  I_SR     = H_Rec(UP(F_DF))                     UP: D x (3x3 conv 64 -> 256, shuffle x2);
                                                 H_Rec: 3x3 conv 64 -> 3
Every conv is followed by a ReLU except H_Rec, the last (Sec. 4, "Implement
details"); all kernels are 3x3 except the 1x1 fuse conv; 64 feature channels.

Readings (the paper does not fix these):
* I_HRLS = HRLS RGB, albedo, normal (C_h = 9); with the extra layers, diffuse,
  specular and log(1 + variance) follow (C_h = 18).
* DSF is a pure rearrangement (pixel unshuffle, no weights): (H, W, C) ->
  (H/2, W/2, 4C) with out channel 4c + 2 dy + dx = in[2y + dy, 2x + dx, c],
  the channel order of torch's pixel_unshuffle; the shuffle of UP is its
  inverse (torch's pixel_shuffle order).
* An RDB has 4 convs, all 3x3 with 64 outputs: three dense layers, each over
  the concatenation [F_in, F_1, ..., F_{c-1}] (64 c channels, in that order),
  and a local-fusion conv over [F_in, F_1, F_2, F_3] (256 channels); with the
  ReLU of every conv, RDB(F_in) = F_in + ReLU(fusion).
* Eq. F_DF adds F_0 (the text says F_LRHS; the equation is taken), and the
  equation's "RDB_1" inside the RDG chain is read as RDG_1.
* No image-level skip: I_SR is the output of H_Rec.

Parameter layout (flat): for each conv in the order above (H_lrhs, H_hrls,
fuse, then per RDG, per RDB, convs 1-4, then the D upsampling convs, H_Rec),
the weight [Cout][k][k][Cin] followed by the bias [Cout].

Backward (backward(), from forward_tape()): the same steps in reverse, for
training the network with the losses of oracle/cnn.py.

Pins (tests/test_oracle_rdn.py): deshuffle / shuffle equal torch's
pixel_unshuffle / pixel_shuffle; the 1x1 conv equals brute-force loops; an
identity-kernel network gives I_SR = (1 + 2^G) * nearest_up_s(I_LRHS) in
closed form (pins the group and global skips and the shuffle order); scaled
identity kernels in one RDB give a closed-form factor that a misordered
concatenation would change; a fuse conv that selects one deshuffled channel
reproduces that HR pixel of F0_HRLS; forward_tape() equals forward(); the
backward matches central finite differences of the float64 forward on a small
network at every scale (weights, biases of every layer kind, and the extra
layers' input), and for a linear output functional every gradient entry of
the last layer equals its closed form.
"""
from __future__ import annotations

import numpy as np

from . import cnn

C_F = 64
N_RDG = 3           # G
N_RDB = 5           # B
N_CONV = 4          # convs per RDB
C_LR = 3
C_HR = 9
C_HR_EXTRA = 18
SCALES = (2, 4, 8)


def depth(s):
    if s not in SCALES:
        raise ValueError(f"scale {s} not in {SCALES}")
    return {2: 1, 4: 2, 8: 3}[s]


def layers_for(s, c_hr=C_HR):
    """[(name, k, cin, cout)] in forward (= parameter) order."""
    L = [("H_lrhs", 3, C_LR, C_F), ("H_hrls", 3, c_hr, C_F), ("fuse", 1, C_F + C_F * s * s, C_F)]
    for g in range(N_RDG):
        for b in range(N_RDB):
            for c in range(1, N_CONV + 1):
                L.append((f"rdg{g}.rdb{b}.conv{c}", 3, C_F * c, C_F))
    for d in range(depth(s)):
        L.append((f"up{d}", 3, C_F, 4 * C_F))
    L.append(("H_rec", 3, C_F, 3))
    return L


def layer_offsets(s, c_hr=C_HR):
    """[(name, w_off, b_off, k, cin, cout)] into the flat parameter array."""
    out, o = [], 0
    for name, k, ci, co in layers_for(s, c_hr):
        out.append((name, o, o + co * k * k * ci, k, ci, co))
        o += co * k * k * ci + co
    return out


def nparams(s, c_hr=C_HR):
    return sum(co * k * k * ci + co for _, k, ci, co in layers_for(s, c_hr))


def unpack(params, s, c_hr=C_HR):
    p = np.asarray(params, dtype=np.float64)
    if p.size != nparams(s, c_hr):
        raise ValueError(f"{p.size} parameters: expected {nparams(s, c_hr)}")
    return [(p[wo:bo].reshape(co, k, k, ci), p[bo:bo + co])
            for _, wo, bo, k, ci, co in layer_offsets(s, c_hr)]


def pack(layers):
    return np.concatenate([np.concatenate([w.ravel(), b.ravel()]) for w, b in layers])


def conv1x1(x, w, b):
    """out[n,y,x,o] = b[o] + sum_c in[n,y,x,c] * w[o,0,0,c]."""
    return np.asarray(x, np.float64) @ w[:, 0, 0, :].T + b


def deshuffle(x):
    """DSF with alpha = 2: (N, H, W, C) -> (N, H/2, W/2, 4C),
    out[n, y, x, 4c + 2dy + dx] = in[n, 2y + dy, 2x + dx, c]."""
    N, H, W, C = x.shape
    t = x.reshape(N, H // 2, 2, W // 2, 2, C)          # n, y, dy, x, dx, c
    return t.transpose(0, 1, 3, 5, 2, 4).reshape(N, H // 2, W // 2, 4 * C)


def shuffle(x):
    """Inverse of deshuffle (ESPCN pixel shuffle, x2): (N, h, w, 4C) ->
    (N, 2h, 2w, C), out[n, 2y + dy, 2x + dx, c] = in[n, y, x, 4c + 2dy + dx]."""
    N, h, w, C4 = x.shape
    C = C4 // 4
    t = x.reshape(N, h, w, C, 2, 2)                     # n, y, x, c, dy, dx
    return t.transpose(0, 1, 4, 2, 5, 3).reshape(N, 2 * h, 2 * w, C)


def relu(x):
    return np.maximum(x, 0.0)


def hr_input(hrls, albedo, normal, extra=None):
    """I_HRLS as network input: RGB, albedo, normal (+ diffuse, specular,
    log(1 + variance) when the extra layers are given)."""
    parts = [hrls, albedo, normal] + ([cnn.extra_input(extra)] if extra is not None else [])
    return np.concatenate([np.asarray(a, np.float64) for a in parts], axis=-1)


def rdb(F_in, convs):
    """One residual dense block: convs = [(w, b)] x 4."""
    feats = [F_in]
    for w, b in convs[:3]:
        feats.append(relu(cnn.conv3x3(np.concatenate(feats, axis=-1), w, b)))
    return F_in + relu(cnn.conv3x3(np.concatenate(feats, axis=-1), *convs[3]))


def forward(params, lrhs, hrls, albedo, normal, s, extra=None, keep=False):
    """I_SR [N, s h, s w, 3] from LRHS [N, h, w, 3] and the HRLS buffers
    [N, s h, s w, 3] (extra [N, s h, s w, 9] for the 18-channel HRLS input)."""
    c_hr = C_HR_EXTRA if extra is not None else C_HR
    L = unpack(params, s, c_hr)
    D = depth(s)
    acts = {}
    F_lr = relu(cnn.conv3x3(np.asarray(lrhs, np.float64), *L[0]))
    F_h = relu(cnn.conv3x3(hr_input(hrls, albedo, normal, extra), *L[1]))
    acts["F_LRHS"], acts["F0_HRLS"] = F_lr, F_h
    for _ in range(D):
        F_h = deshuffle(F_h)
    F0 = relu(conv1x1(np.concatenate([F_lr, F_h], axis=-1), *L[2]))
    acts["F_0"] = F0
    F = F0
    i = 3
    for g in range(N_RDG):
        F_prev = F
        for b in range(N_RDB):
            F = rdb(F, L[i:i + N_CONV])
            i += N_CONV
        F = F + F_prev
        acts[f"F_{g + 1}"] = F
    U = F + F0
    acts["F_DF"] = U
    for d in range(D):
        U = shuffle(relu(cnn.conv3x3(U, *L[i])))
        i += 1
        acts[f"U_{d + 1}"] = U
    y = cnn.conv3x3(U, *L[i])
    return (y, acts) if keep else y


def conv1x1_backward(x, w, dout):
    """Gradients of conv1x1 w.r.t. input, weight [Cout][1][1][Cin] and bias."""
    x = np.asarray(x, np.float64)
    dw = np.einsum("nyxo,nyxc->oc", dout, x)[:, None, None, :]
    return dout @ w[:, 0, 0, :], dw, dout.sum(axis=(0, 1, 2))


def forward_tape(params, lrhs, hrls, albedo, normal, s, extra=None):
    """forward() that also records every conv's input and pre-activation, in
    forward order, for backward(): returns (I_SR, tape)."""
    c_hr = C_HR_EXTRA if extra is not None else C_HR
    L = unpack(params, s, c_hr)
    D = depth(s)
    tape = {"s": s, "c_hr": c_hr}
    x_lr = np.asarray(lrhs, np.float64)
    z = cnn.conv3x3(x_lr, *L[0])
    tape["lr"] = (x_lr, z)
    F_lr = relu(z)
    x_hr = hr_input(hrls, albedo, normal, extra)
    z = cnn.conv3x3(x_hr, *L[1])
    tape["hr"] = (x_hr, z)
    F_h = relu(z)
    for _ in range(D):
        F_h = deshuffle(F_h)
    x_f = np.concatenate([F_lr, F_h], axis=-1)
    z = conv1x1(x_f, *L[2])
    tape["fuse"] = (x_f, z)
    F0 = relu(z)
    F = F0
    i = 3
    blocks = []
    for g in range(N_RDG):
        F_prev = F
        for b in range(N_RDB):
            feats = [F]
            convs = []
            for c in range(N_CONV):
                x_c = np.concatenate(feats, axis=-1)
                z_c = cnn.conv3x3(x_c, *L[i + c])
                convs.append((x_c, z_c))
                if c < N_CONV - 1:
                    feats.append(relu(z_c))
            blocks.append(convs)
            F = F + relu(convs[-1][1])
            i += N_CONV
        F = F + F_prev
    tape["blocks"] = blocks
    U = F + F0
    ups = []
    for d in range(D):
        z = cnn.conv3x3(U, *L[i])
        ups.append((U, z))
        U = shuffle(relu(z))
        i += 1
    tape["ups"] = ups
    tape["rec_in"] = U
    return cnn.conv3x3(U, *L[i]), tape


def _abs_terms_1x1(x, dz):
    """Sums of |terms| of a 1x1 conv's weight and bias gradients."""
    ax, ad = np.abs(np.asarray(x, np.float64)), np.abs(dz)
    return np.einsum("nyxo,nyxc->oc", ad, ax)[:, None, None, :], ad.sum(axis=(0, 1, 2))


def backward(params, tape, dy, abs_terms=False):
    """Gradient of a loss w.r.t. the flat params, given dL/dI_SR: the forward
    steps of Sec. 4 in reverse (each conv's input / weight / bias gradients,
    ReLU masks from the recorded pre-activations, deshuffle and shuffle
    exchanged, the dense concatenations split back into their parts, the
    block, group and Eq. F_DF skips adding their gradients).  With abs_terms,
    also the sum of |terms| of every gradient element in the same layout
    (sum over pixels of |dz| |x| for a weight, |dz| for a bias: the scale of
    their rounding error, for tolerances)."""
    s, c_hr = tape["s"], tape["c_hr"]
    L = unpack(params, s, c_hr)
    D = depth(s)
    grads = [None] * len(L)
    terms = [None] * len(L)

    def conv_grad(i, x, dz):
        dx, dw, db = cnn.conv3x3_backward(x, L[i][0], dz)
        grads[i] = (dw, db)
        if abs_terms:
            terms[i] = cnn._abs_terms(x, dz)
        return dx

    i = len(L) - 1
    dU = conv_grad(i, tape["rec_in"], dy)
    for d in reversed(range(D)):
        i -= 1
        U_in, z = tape["ups"][d]
        dz = deshuffle(dU) * (z > 0.0)
        dU = conv_grad(i, U_in, dz)
    # U = F_G + F_0
    dF = dU
    dF0 = dU.copy()
    blocks = tape["blocks"]
    bi = len(blocks)
    for g in reversed(range(N_RDG)):
        d_skip = dF                       # F_g = chain(F_{g-1}) + F_{g-1}
        for b in reversed(range(N_RDB)):
            bi -= 1
            convs = blocks[bi]
            # RDB(F_in) = F_in + ReLU(z_4); z_c = conv_c([F_in, f_1, ..., f_{c-1}])
            d_parts = [dF] + [np.zeros_like(dF) for _ in range(N_CONV - 1)]
            dz = dF * (convs[-1][1] > 0.0)
            for c in reversed(range(N_CONV)):
                x_c, z_c = convs[c]
                if c < N_CONV - 1:
                    dz = d_parts[c + 1] * (z_c > 0.0)
                dx = conv_grad(3 + bi * N_CONV + c, x_c, dz)
                for k in range(c + 1):
                    d_parts[k] = d_parts[k] + dx[..., C_F * k:C_F * (k + 1)]
            dF = d_parts[0]
        dF = dF + d_skip
    dF0 = dF0 + dF
    x_f, z = tape["fuse"]
    dz = dF0 * (z > 0.0)
    dx_f, dw, db = conv1x1_backward(x_f, L[2][0], dz)
    grads[2] = (dw, db)
    if abs_terms:
        terms[2] = _abs_terms_1x1(x_f, dz)
    dF_lr, dF_h = dx_f[..., :C_F], dx_f[..., C_F:]
    for _ in range(D):
        dF_h = shuffle(dF_h)
    x_hr, z = tape["hr"]
    conv_grad(1, x_hr, dF_h * (z > 0.0))
    x_lr, z = tape["lr"]
    conv_grad(0, x_lr, dF_lr * (z > 0.0))
    return (pack(grads), pack(terms)) if abs_terms else pack(grads)


def loss_and_grad(params, lrhs, hrls, albedo, normal, target, s, loss="robust", beta=0.1,
                  extra=None, abs_terms=False):
    """The training loss of I_SR against `target` (cnn.loss_fn: "robust" = the
    method's l_r, or "l1log") and its gradient w.r.t. the flat params (and,
    with abs_terms, the gradient's sums of |terms|, see backward())."""
    y, tape = forward_tape(params, lrhs, hrls, albedo, normal, s, extra)
    value, dy = cnn.loss_fn(y, target, loss, beta)
    g = backward(params, tape, dy, abs_terms)
    return (value,) + g if abs_terms else (value, g)


def flops_per_lr_pixel(s, c_hr=C_HR):
    """Multiply-adds x 2 of one forward pass per LR pixel (H_hrls and H_Rec run
    at HR, the i-th upsampling conv at 4^i LR pixels)."""
    total = 0
    up = 0
    for name, k, ci, co in layers_for(s, c_hr):
        f = 2 * k * k * ci * co
        if name in ("H_hrls", "H_rec"):
            f *= s * s
        elif name.startswith("up"):
            f *= 4 ** up
            up += 1
        total += f
    return total


def kaiming(seed, s, c_hr=C_HR, fusion_damp=1.0):
    """Kaiming-normal weights (std sqrt(2 / (k^2 Cin))), zero biases; the
    RDBs' local-fusion convs scaled by fusion_damp (each RDB adds its fusion
    output to its input, so undamped random blocks grow activations
    geometrically through the 15 blocks)."""
    rng = np.random.default_rng(np.random.SeedSequence([0x72646E, int(seed), s, c_hr]))
    layers = []
    for name, k, ci, co in layers_for(s, c_hr):
        w = rng.normal(0, np.sqrt(2.0 / (k * k * ci)), (co, k, k, ci))
        if name.endswith(f"conv{N_CONV}"):
            w = w * fusion_damp
        layers.append((w, np.zeros(co)))
    return pack(layers)
