"""Oracle pins: Philox4x32-10 and the sin/cos used for direction sampling."""
import os

import numpy as np

GOLD = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat():
    rows = []
    for line in open(GOLD):
        if line.startswith("#") or not line.strip():
            continue
        w = [int(x, 16) for x in line.split()]
        rows.append((w[:4], w[4:6], w[6:10]))
    return rows


def test_philox_known_answers(orc):
    rows = _kat()
    assert len(rows) == 3
    for ctr, key, want in rows:
        assert list(orc.philox4x32_10(ctr, key)) == want


def test_uniforms_are_philox_top24_bits(orc):
    seed = 0x1234_5678_9ABC_DEF0
    u = orc.philox_uniforms(17, 5, 3, seed)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    w0 = orc.philox4x32_10([17, 5, 3, 0], key)
    w1 = orc.philox4x32_10([17, 5, 3, 1], key)
    want = np.concatenate([w0, w1]).astype(np.uint64) >> np.uint64(8)
    assert np.array_equal(u.astype(np.float64) * 2.0**24, want.astype(np.float64))


def test_uniformity_chi2(orc):
    # 64 bins over 2^16 draws (8 dims x 8192 (pixel, sample) pairs)
    vals = np.concatenate([orc.philox_uniforms(p, s, 0, 7) for p in range(128) for s in range(64)])
    hist = np.bincount((vals * 64).astype(int), minlength=64)
    e = len(vals) / 64
    chi2 = ((hist - e) ** 2 / e).sum()
    assert chi2 < 120.0   # 63 dof: p(chi2 > 120) ~ 1e-5
    assert vals.min() >= 0.0 and vals.max() < 1.0


def test_sincos2pi_accuracy(orc):
    u = (np.arange(1 << 16, dtype=np.float64) / (1 << 16)).astype(np.float32)
    u = np.concatenate([u, np.float32(1.0) - np.float32(2.0**-24) * np.arange(1, 100, dtype=np.float32)])
    c, s = orc.sincos2pi(u)
    ang = 2.0 * np.pi * u.astype(np.float64)
    assert np.abs(c - np.cos(ang)).max() < 5e-7
    assert np.abs(s - np.sin(ang)).max() < 5e-7
    assert np.abs(c.astype(np.float64) ** 2 + s.astype(np.float64) ** 2 - 1).max() < 2e-6
