"""Oracle pins for the metrics (Eq. cvt_color, RelMSE, PSNR, spp_avg) and the
fallback gate."""
import os

import numpy as np

from oracle import metrics

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    return [list(map(float, l.split())) for l in open(os.path.join(GOLD, name))
            if l.strip() and not l.startswith("#")]


def test_srgb_points():
    for lin, s in _rows("srgb_points.txt"):
        assert abs(metrics.srgb(lin) - s) < 1e-8, (lin, s)


def test_srgb_continuous_at_breakpoints():
    # both branch pairs of Eq. cvt_color meet at their breakpoints
    b = 0.0031308
    assert abs(12.92 * b - (1.055 * b ** (1 / 2.4) - 0.055)) < 1e-6
    assert abs(1.055 * 1.0 ** (1 / 2.4) - 0.055 - 1.0) < 1e-15
    x = np.linspace(-0.1, 1.5, 100001)
    assert (np.diff(metrics.srgb(x)) >= 0).all()


def test_relmse_hand_computed():
    ref = np.array([[[1.0, 0, 0], [0, 0.1, 0]], [[0, 0, 2], [0.5, 0.5, 0.5]]])
    x = ref + 0.1
    want = np.mean(0.5 * 0.01 / (ref ** 2 + 0.01))
    assert abs(metrics.relmse(x, ref) - want) < 1e-15
    assert metrics.relmse(ref, ref) == 0.0
    # Gharbi-protocol constants
    assert abs(metrics.relmse(x, ref, 1.0, 1e-4) - np.mean(0.01 / (ref ** 2 + 1e-4))) < 1e-15


def test_psnr():
    ref = np.full((2, 2, 3), 0.5)
    assert metrics.psnr(ref, ref) == float("inf")
    # in sRGB, 0 vs 1 everywhere is MSE 1 -> 0 dB; above 1 clamps
    assert metrics.psnr(np.zeros((2, 2, 3)), np.full((2, 2, 3), 7.0)) == 0.0
    x = np.zeros((2, 2, 3))
    x[0, 0, 0] = 1.0
    assert abs(metrics.psnr(x, np.zeros((2, 2, 3))) - 10 * np.log10(12)) < 1e-12
    assert abs(metrics.psnr(x, np.zeros((2, 2, 3)), metrics.clamp01) - 10 * np.log10(12)) < 1e-12


def test_spp_avg_matches_table_headers():
    for s, lr, hr, col in _rows("spp_avg_table_comp_bcr.txt"):
        assert round(metrics.spp_avg(lr, hr, s)) == col


def test_box_down_and_gate():
    rng = np.random.default_rng(0)
    lr = rng.uniform(0.5, 2.0, (8, 8, 3))
    nn = np.repeat(np.repeat(lr, 4, axis=0), 4, axis=1)
    assert np.allclose(metrics.box_down(nn, 4), lr)
    use_plain, d = metrics.gate(nn, lr, 4)
    assert not use_plain and d < 1e-28
    for delta, expect in ((0.1, False), (0.3, True)):
        use_plain, d = metrics.gate(nn * (1 + delta), lr, 4)
        want = np.mean(0.5 * (delta * lr) ** 2 / (lr ** 2 + 0.01))
        assert abs(d - want) < 1e-12 and use_plain == expect


def test_clip():
    assert np.array_equal(metrics.clip(np.array([0.0, 99.0, 100.0, 1e6])), [0, 99, 100, 100])
