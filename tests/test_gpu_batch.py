"""Batched rendering (mrs_render_batch): many jobs -- different scenes, image
sizes, sample counts, depths, sampling grids and seeds -- share waves whose
kernels run over all their jobs at once.  Every job's outputs must equal the
single render's (mrs_render_grid with the job's arguments) bit for bit, for
wave sizes that keep jobs whole, split them into sample chunks, and pack
chunks of several jobs into one wave."""
import numpy as np
import pytest

from synth import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mrs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2106_12802_gb300 as m
    m.load()
    return m


@pytest.fixture(scope="module")
def pool(mrs):
    return [mrs.Scene.seeded(11, "procedural", n_spheres=16, n_large=4),
            mrs.Scene.seeded(12, "procedural", n_spheres=8, n_large=2),
            mrs.Scene.seeded(0, "cornell", sphere_subdiv=2)]


def _jobs(pool):
    rng = np.random.default_rng(3)
    jobs = []
    for i in range(9):
        W = int(rng.choice([16, 40, 64, 96]))
        H = int(rng.choice([24, 48, 64]))
        jobs.append({"scene": pool[i % 3], "W": W, "H": H, "spp": int(rng.choice([1, 3, 4, 8])),
                     "max_depth": int(rng.choice([0, 2, 5, 8])),
                     "rr_start": None if i % 4 == 0 else 3, "seed": 100 + i,
                     "grid": 2 if i == 4 else 1})
    return jobs


@pytest.mark.parametrize("wave", [1 << 24, 40000, 3000])
def test_batch_equals_single_renders(mrs, pool, wave):
    jobs = _jobs(pool)
    ctx = mrs.RenderContext()
    ctx.set_wave(wave)
    got = mrs.render_batch(ctx, jobs)
    for j, g in zip(jobs, got):
        ref = mrs.render(j["scene"], j["W"], j["H"], j["spp"], j["max_depth"], j["rr_start"],
                         j["seed"], grid=j["grid"])
        for k in ("radiance", "albedo", "normal", "depth"):
            assert torch.equal(g[k], ref[k]), (k, j["W"], j["H"], j["spp"], wave)
    ctx.close()


def test_batch_without_aux_and_tail_settings(mrs, pool):
    # radiance only; the tail kernel from bounce 0 and no tail at all give the
    # same images
    jobs = [dict(j, aux=False) for j in _jobs(pool)[:5]]
    outs = []
    for tail in (-1, 0, 64):
        ctx = mrs.RenderContext()
        ctx.set_tail(tail)
        ctx.set_wave(20000)
        outs.append(mrs.render_batch(ctx, jobs))
        ctx.close()
    for a, b, c in zip(*outs):
        assert torch.equal(a["radiance"], b["radiance"]) and torch.equal(a["radiance"], c["radiance"])


def test_batch_rejects_bad_jobs(mrs, pool):
    ctx = mrs.RenderContext()
    good = {"scene": pool[0], "W": 8, "H": 8, "spp": 1, "max_depth": 2}
    for bad in ({"spp": 0}, {"max_depth": 40}, {"W": 0}, {"grid": 0}):
        with pytest.raises(Exception):
            mrs.render_batch(ctx, [good, dict(good, **bad)])
    from paper_2106_12802_gb300 import _lib
    with pytest.raises(Exception):          # no context, no jobs
        _lib.call("mrs_render_batch", None, None, 0, None)
    ctx.close()
