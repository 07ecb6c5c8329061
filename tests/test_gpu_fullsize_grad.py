"""Training gradients at full size, by properties that hold at any size.

The float64 oracle's backward is compared with the GPU element by element on
small images (test_gpu_train.py, test_gpu_rdn_train.py); at the training
batches themselves -- the paper's 16 x 192^2 crops at x4 for its own network,
the bench's 16 x 128^2 for the fusion network -- the oracle is too slow, so:

* the FP32 gradient g is checked against the directional derivative of the
  FP32 loss, (L(p + eps v) - L(p - eps v)) / (2 eps), along random directions
  v (each parameter moved in proportion to its magnitude).  The loss is
  reduced in float64 from FP32 values, so with eps chosen to move it by about
  1e-3 of itself the difference quotient is good to ~1e-4 relative, and the
  curvature term of a central difference is O(eps^2): the bar is 1e-2.
* the BF16 step's gradient is compared with that FP32 gradient layer by
  layer: at these sizes the rounding of the BF16 activations and gradients
  averages out over some 37k (LR) to 590k (HR) pixels per weight, and the
  worst layer measured within 1.0% (paper's network) and 0.5% (fusion
  network) relative L2 of FP32; bars 5% and 3%, cosine 0.999 (a wrong part,
  tap or view gives whole-layer errors of order 1).
Every step here has lr = 0: the loss and the gradient, weights unchanged.
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


def _batch(seed, N, crop, s):
    g = torch.Generator(device="cuda").manual_seed(seed)
    h = crop // s
    lr = torch.rand((N, h, h, 3), device="cuda", generator=g) * 2
    hr = torch.rand((N, crop, crop, 3), device="cuda", generator=g) * 2
    alb = torch.rand((N, crop, crop, 3), device="cuda", generator=g)
    nrm = torch.rand((N, crop, crop, 3), device="cuda", generator=g) * 2 - 1
    tgt = torch.rand((N, crop, crop, 3), device="cuda", generator=g) * 2
    return lr, hr, alb, nrm, tgt


def _directions(p, k, seed):
    rng = np.random.default_rng(seed)
    return [rng.normal(size=p.shape) * (np.abs(p) + 1e-3) for _ in range(k)]


def _check_directional(loss_at, p, g, dirs):
    L0 = loss_at(p)
    for v in dirs:
        gv = float(np.dot(g.astype(np.float64), v))
        eps = 1e-3 * L0 / (abs(gv) + 1e-30)
        fd = (loss_at(p + eps * v) - loss_at(p - eps * v)) / (2 * eps)
        assert abs(fd - gv) <= 1e-2 * abs(gv) + 1e-9, (fd, gv)


def _layer_compare(g16, g32, offsets, cos_min, rel_max):
    worst = []
    for name, wo, bo, co in offsets:
        a, b = g16[wo:bo].astype(np.float64), g32[wo:bo].astype(np.float64)
        cos = a @ b / (np.linalg.norm(a) * np.linalg.norm(b) + 1e-30)
        rel = np.linalg.norm(a - b) / (np.linalg.norm(b) + 1e-30)
        worst.append((cos, rel, name))
    worst.sort()
    print("\nworst layers (cos, rel L2):", [(n, round(c, 4), round(r_, 4)) for c, r_, n in worst[:3]])
    for cos, rel, name in worst:
        assert cos > cos_min and rel < rel_max, (name, cos, rel)


def test_rdn_gradients_at_the_papers_batch(mrs):
    s, N, crop = 4, 16, 192
    L = ordn.unpack(ordn.kaiming(5, s, fusion_damp=0.1), s)
    L = [(w, b + 0.01) for w, b in L]
    L[-1] = (L[-1][0] * 0.05, L[-1][1])
    p = ordn.pack(L).astype(np.float32)
    t = _batch(31, N, crop, s)

    def run(params, prec):
        net = mrs.RDN(np.asarray(params, np.float32), s)
        v = net.train_step(*t, lr=0.0, loss="l1log", precision=prec)
        g = net.get_grads()
        net.close()
        return v, g

    _, g32 = run(p, "fp32")
    _check_directional(lambda q: run(q, "fp32")[0], p.astype(np.float64), g32, _directions(p, 3, 1))
    _, g16 = run(p, "bf16")
    offs = [(n, wo, bo, co) for n, wo, bo, k, ci, co in ordn.layer_offsets(s)]
    _layer_compare(g16, g32, offs, 0.999, 0.05)


def test_fusion_network_gradients_at_the_bench_batch(mrs):
    s, N, crop = 4, 16, 128
    layers = cnn.unpack(cnn.kaiming(3))
    p = cnn.pack([(w * 0.25 if 1 <= i <= 16 and i % 2 == 0 else w, b + 0.02)
                  for i, (w, b) in enumerate(layers)]).astype(np.float32)
    t = _batch(32, N, crop, s)

    def run(params, prec):
        net = mrs.Net(np.asarray(params, np.float32))
        net.set_loss("l1log")
        v = mrs.train_step(net, *t, s, lr=0.0, precision=prec)
        g = mrs.get_grads(net)
        net.close()
        return v, g

    _, g32 = run(p, "fp32")
    _check_directional(lambda q: run(q, "fp32")[0], p.astype(np.float64), g32, _directions(p, 3, 2))
    _, g16 = run(p, "bf16")
    offs = [(f"layer{i}", wo, bo, co) for i, (wo, bo, ci, co) in enumerate(cnn.layer_offsets())]
    _layer_compare(g16, g32, offs, 0.999, 0.03)
