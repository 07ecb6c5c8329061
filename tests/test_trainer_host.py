"""Host-side logic of the training-data generator (no GPU): the spp
randomisation of the method's training (Sec. 4, implementation details)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
from paper_2106_12802_gb300 import trainer  # noqa: E402


def test_random_spp_pairs_follow_the_sets_and_order():
    rng = np.random.default_rng(0)
    pairs = [trainer.random_spp_pair(rng, 256) for _ in range(4000)]
    lrs = {a for a, _ in pairs}
    hrs = {b for _, b in pairs}
    assert all(b < a < 256 for a, b in pairs)
    assert lrs == {v for v in trainer.SPP_LRHS_SET if v < 256}
    assert hrs == set(trainer.SPP_HRLS_SET)
    # with a high-spp target every LRHS value of the set occurs
    rng = np.random.default_rng(1)
    assert {trainer.random_spp_pair(rng, 8192)[0] for _ in range(8000)} == set(trainer.SPP_LRHS_SET)


def test_random_spp_pairs_are_seeded():
    a = [trainer.random_spp_pair(np.random.default_rng(5), 256) for _ in range(3)]
    b = [trainer.random_spp_pair(np.random.default_rng(5), 256) for _ in range(3)]
    assert a == b


def test_random_spp_pair_rejects_a_target_too_noisy():
    with pytest.raises(ValueError):
        trainer.random_spp_pair(np.random.default_rng(0), 2)
