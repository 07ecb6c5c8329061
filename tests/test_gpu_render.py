"""GPU parity of the renderer (Philox, LBVH, ray casting, path tracing) against
the CPU oracle, called through the C ABI.  Integer/index outputs (random
words, Morton codes, tree topology, per-bounce ray counts) must be bit-exact;
radiance must agree within 1e-4 relative on >= 99.9% of pixels with the image
mean within 1e-5 relative (both sides evaluate the same float32 operations in
the same order, so in practice they are identical)."""

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


def assert_radiance_parity(gpu, ref):
    gpu = np.asarray(gpu, np.float64)
    ref = np.asarray(ref, np.float64)
    rel = np.abs(gpu - ref) / np.maximum(np.abs(ref), 1e-30)
    rel[(gpu == ref)] = 0.0
    px_ok = (rel.reshape(-1, 3) <= 1e-4).all(axis=1).mean()
    assert px_ok >= 0.999, px_ok
    m_ref, m_gpu = ref.mean(), gpu.mean()
    assert abs(m_gpu - m_ref) <= 1e-5 * max(abs(m_ref), 1e-30)


def test_philox_bit_exact(mrs, orc):
    rng = np.random.default_rng(0)
    tri = rng.integers(0, 2**31, (1000, 3)).astype(np.int32)
    tri[:3] = [[0, 0, 0], [2**31 - 1, 7, 3], [12345, 4095, 31]]
    seed = 0xDEADBEEF_12345678
    gpu = mrs.philox_uniforms(torch.from_numpy(tri).cuda(), seed).cpu().numpy()
    ref = np.stack([orc.philox_uniforms(int(a), int(b), int(c), seed) for a, b, c in tri])
    assert np.array_equal(gpu.view(np.uint32), ref.view(np.uint32))


@pytest.mark.parametrize("kind,n", [("rand", 1), ("rand", 2), ("rand", 3), ("rand", 1000),
                                    ("rand", 4097), ("cornell", 0), ("proc", 0)])
def test_lbvh_bit_exact(mrs, orc, kind, n):
    if kind == "rand":
        desc = scenes.random_triangles(n, n)
    elif kind == "cornell":
        desc = scenes.cornell_box()
    else:
        desc = scenes.procedural(1)
    sc = mrs.Scene(desc)
    g = sc.export_bvh()
    r = orc.lbvh(desc["V"])
    for key in ("morton", "order", "left", "right"):
        assert np.array_equal(g[key], r[key]), key
    assert np.array_equal(g["box"].view(np.uint32), r["box"].view(np.uint32))
    sc.rebuild()
    g2 = sc.export_bvh()
    assert all(np.array_equal(g[k], g2[k]) for k in g)


def test_lbvh_duplicate_codes(mrs, orc):
    desc = scenes.random_triangles(3, 50)
    desc["V"] = np.repeat(desc["V"][:1], 50, axis=0).copy()
    sc = mrs.Scene(desc)
    g = sc.export_bvh()
    r = orc.lbvh(desc["V"])
    for key in ("morton", "order", "left", "right"):
        assert np.array_equal(g[key], r[key]), key


@pytest.mark.parametrize("seed,n", [(0, 8), (1, 64), (2, 3000)])
def test_cast_equals_brute_force(mrs, orc, seed, n):
    desc = scenes.random_triangles(seed, n)
    o, d = scenes.random_rays(seed, 50000)
    sc = mrs.Scene(desc)
    prim, t = sc.cast(torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda())
    pb, tb = orc.cast(desc["V"], o, d, brute=n <= 64)
    assert np.array_equal(prim.cpu().numpy(), pb)
    assert np.array_equal(t.cpu().numpy(), tb)


def _compare_render(mrs, orc, desc, W, H, spp, D, rr=None, seed=0, wave=None, grid=1, ctx=None):
    sc = mrs.Scene(desc)
    if wave:
        sc.set_wave(wave)
    g = mrs.render(sc, W, H, spp, D, rr_start=rr, seed=seed, grid=grid, ctx=ctx)
    torch.cuda.synchronize()
    g = {k: v.cpu().numpy() for k, v in g.items()}
    r = orc.render(desc, W, H, spp, D, rr_start=rr, seed=seed, grid=grid)
    assert np.array_equal(g["counts"].astype(np.uint64), r["counts"])
    assert np.array_equal(g["shadow_counts"].astype(np.uint64), r["shadow_counts"])
    assert_radiance_parity(g["radiance"], r["radiance"])
    for k in ("albedo", "normal", "depth"):
        assert np.array_equal(g[k], r[k]), k
    return g, r


def test_render_cornell_config(mrs, orc):
    # Cornell box, 128 x 128, 32 spp, max depth 4, seed 0
    g, r = _compare_render(mrs, orc, scenes.cornell_box(), 128, 128, 32, 4)
    assert (g["radiance"] == r["radiance"]).mean() > 0.999


def test_render_ragged_multi_wave(mrs, orc):
    # 37 x 23 pixels, waves of 2 samples (851 x 2 paths), 5 spp -> ragged last wave
    _compare_render(mrs, orc, scenes.cornell_box(sphere_subdiv=2), 37, 23, 5, 3, seed=7,
                    wave=37 * 23 * 2)


def test_render_procedural_roulette(mrs, orc):
    _compare_render(mrs, orc, scenes.procedural(0), 48, 40, 4, 8, rr=3, seed=3)


def test_render_furnace_and_sky_closed_forms(mrs, orc):
    g, _ = _compare_render(mrs, orc, scenes.furnace_sphere(1.5, 0.6), 16, 16, 4, 5)
    assert np.allclose(g["radiance"], 1.5 * sum(0.6**k for k in range(6)), rtol=2e-6)
    g, _ = _compare_render(mrs, orc, scenes.sky_plane(0.6, 2.0), 16, 16, 4, 2)
    assert np.allclose(g["radiance"], 1.2, rtol=2e-6)


def test_render_degenerate_scenes(mrs, orc):
    # no triangles: every camera ray sees the environment
    desc = scenes.sky_plane(0.5, 0.7)
    empty = dict(desc, V=desc["V"][:0], tri_mat=desc["tri_mat"][:0],
                 tri_light=desc["tri_light"][:0])
    g, _ = _compare_render(mrs, orc, empty, 8, 8, 2, 3)
    assert np.allclose(g["radiance"], 0.7) and (g["depth"] == 0).all()
    one = dict(desc, V=desc["V"][:1], tri_mat=desc["tri_mat"][:1],
               tri_light=desc["tri_light"][:1])
    _compare_render(mrs, orc, one, 9, 7, 3, 2)
    # 1 x 1 image, depth 0
    _compare_render(mrs, orc, scenes.cornell_box(sphere_subdiv=1), 1, 1, 3, 0)


def test_render_sparse_grid_matches_oracle(mrs, orc):
    # nearest-neighbour LR sampling (each pixel samples only the centre
    # sub-pixel of its grid x grid block): bit-exact counts, aux and radiance
    # parity as for the ordinary render; odd grid, ragged waves, a context
    g4, _ = _compare_render(mrs, orc, scenes.cornell_box(sphere_subdiv=2), 32, 32, 16, 4, grid=4)
    _compare_render(mrs, orc, scenes.procedural(0), 40, 24, 4, 8, rr=3, seed=2, grid=4)
    _compare_render(mrs, orc, scenes.cornell_box(sphere_subdiv=2), 21, 13, 5, 3, seed=4, grid=3,
                    wave=21 * 13 * 2)
    ctx = mrs.RenderContext()
    gc, _ = _compare_render(mrs, orc, scenes.cornell_box(sphere_subdiv=2), 32, 32, 16, 4, grid=4,
                            ctx=ctx)
    assert all(np.array_equal(g4[k], gc[k]) for k in g4)
    sc = mrs.Scene(scenes.cornell_box(sphere_subdiv=1))
    for bad in (0, 65):
        with pytest.raises(Exception):
            mrs.render(sc, 8, 8, 1, 2, grid=bad)


@pytest.mark.parametrize("case", ["cornell", "procedural_ragged", "procedural_grid"])
def test_render_extra_layers_match_oracle(mrs, orc, case):
    # diffuse / specular / variance layers (Sec. 4) with the same parity bar as
    # the radiance; requesting them leaves every other output bit-identical
    desc, W, H, spp, D, rr, seed, grid, wave = {
        "cornell": (scenes.cornell_box(sphere_subdiv=2), 32, 24, 8, 4, None, 1, 1, None),
        "procedural_ragged": (scenes.procedural(0), 40, 32, 6, 8, 3, 2, 1, 40 * 32 * 4),
        "procedural_grid": (scenes.procedural(0), 24, 24, 4, 8, 3, 5, 4, None),
    }[case]
    sc = mrs.Scene(desc)
    if wave:
        sc.set_wave(wave)
    g = mrs.render(sc, W, H, spp, D, rr_start=rr, seed=seed, grid=grid, layers=True)
    plain = mrs.render(sc, W, H, spp, D, rr_start=rr, seed=seed, grid=grid)
    torch.cuda.synchronize()
    g = {k: v.cpu().numpy() for k, v in g.items()}
    plain = {k: v.cpu().numpy() for k, v in plain.items()}
    for k in plain:
        assert np.array_equal(g[k], plain[k]), k
    r = orc.render(desc, W, H, spp, D, rr_start=rr, seed=seed, grid=grid)
    assert np.array_equal(g["counts"].astype(np.uint64), r["counts"])
    for k in ("radiance", "diffuse", "specular", "variance"):
        assert_radiance_parity(g[k], r[k])
    assert (g["diffuse"] + g["specular"] <= g["radiance"] * (1 + 1e-5) + 1e-6).all()


@pytest.mark.parametrize("tail", [0, 2, 5])
def test_render_tail_kernel_bit_identical(mrs, orc, tail):
    # the late bounces in one persistent launch (every bounce >= tail) against
    # the oracle and against the wavefront-only render: same counts, same bits,
    # same traversal work; two waves (the work counter restarts per wave)
    desc = scenes.procedural(0)
    W, H, spp, D, rr, seed = 40, 24, 4, 8, 3, 5
    sc = mrs.Scene(desc)
    sc.set_wave(W * H * 2)
    sc.set_tail(64)   # > max_depth: no tail
    ref = mrs.render(sc, W, H, spp, D, rr_start=rr, seed=seed)
    ref_stats = mrs.render_stats(sc, W, H, spp, D, rr, seed)
    sc.set_tail(tail)
    g = mrs.render(sc, W, H, spp, D, rr_start=rr, seed=seed)
    stats = mrs.render_stats(sc, W, H, spp, D, rr, seed)
    ctx = mrs.RenderContext()
    ctx.set_tail(tail)
    gc = mrs.render(sc, W, H, spp, D, rr_start=rr, seed=seed, ctx=ctx, layers=True)
    torch.cuda.synchronize()
    ref = {k: v.cpu().numpy() for k, v in ref.items()}
    g = {k: v.cpu().numpy() for k, v in g.items()}
    gc = {k: v.cpu().numpy() for k, v in gc.items()}
    for k in ref:
        assert np.array_equal(g[k], ref[k]), k
        assert np.array_equal(gc[k], ref[k]), k
    for k in ("visits", "tests", "shadow_visits", "shadow_tests"):
        assert stats[k] == ref_stats[k], k
        assert ref_stats["tail_" + k] == 0
    if tail <= D:
        assert stats["tail_visits"] > 0
    r = orc.render(desc, W, H, spp, D, rr_start=rr, seed=seed)
    assert np.array_equal(g["counts"].astype(np.uint64), r["counts"])
    assert np.array_equal(g["shadow_counts"].astype(np.uint64), r["shadow_counts"])
    assert_radiance_parity(g["radiance"], r["radiance"])
    for bad in (-2, 65):
        with pytest.raises(Exception):
            sc.set_tail(bad)


def test_render_extra_layers_closed_form(mrs):
    # diffuse plane under a uniform sky: diffuse = rho * L_sky, no specular,
    # zero variance (every sample is the same value)
    sc = mrs.Scene(scenes.sky_plane(0.6, 2.0))
    g = mrs.render(sc, 16, 16, 8, 2, seed=3, layers=True)
    assert np.allclose(g["diffuse"].cpu().numpy(), 1.2, rtol=2e-6)
    assert not g["specular"].any().item() and (g["variance"] <= 1e-10).all().item()


def test_render_full_size_sampled_rows(mrs, orc):
    # the 1024 x 1024, 64 spp, depth 8 (roulette from bounce 3) configuration on
    # the 200k-triangle procedural scene, in the launch configuration the bench
    # times; the oracle recomputes a few image rows
    desc = scenes.procedural(0)
    sc = mrs.Scene(desc)
    g = mrs.render(sc, 1024, 1024, 64, 8, rr_start=3, seed=0)
    torch.cuda.synchronize()
    rows = (511, 513)
    r = orc.render(desc, 1024, 1024, 64, 8, rr_start=3, seed=0, rows=rows)
    rad = g["radiance"][rows[0]:rows[1]].cpu().numpy()
    assert_radiance_parity(rad, r["radiance"])
    assert np.array_equal(g["albedo"][rows[0]:rows[1]].cpu().numpy(), r["albedo"])
    c = g["counts"].cpu().numpy()
    assert c[0] == 1024 * 1024 * 64 and (np.diff(c) <= 0).all()


def test_invalid_render_args(mrs):
    sc = mrs.Scene(scenes.cornell_box(sphere_subdiv=1))
    with pytest.raises(mrs.MrsError):
        mrs.render(sc, 0, 8, 1, 1)
    with pytest.raises(mrs.MrsError):
        mrs.render(sc, 8, 8, 1, 33)


def test_concurrent_render_contexts_match_sequential(mrs):
    # two renders of one scene through their own contexts on two streams give
    # the same bits as the same renders one after the other
    sc = mrs.Scene(scenes.procedural(2, n_spheres=12, n_large=4))
    seq_a = mrs.render(sc, 64, 64, 8, 6, rr_start=3, seed=1)
    seq_b = mrs.render(sc, 128, 96, 2, 6, rr_start=3, seed=2)
    torch.cuda.synchronize()
    ca, cb = mrs.RenderContext(), mrs.RenderContext()
    sa, sb = torch.cuda.Stream(), torch.cuda.Stream()
    with torch.cuda.stream(sa):
        a = mrs.render(sc, 64, 64, 8, 6, rr_start=3, seed=1, ctx=ca)
    with torch.cuda.stream(sb):
        b = mrs.render(sc, 128, 96, 2, 6, rr_start=3, seed=2, ctx=cb)
    torch.cuda.synchronize()
    for k in seq_a:
        assert torch.equal(a[k], seq_a[k]), k
        assert torch.equal(b[k], seq_b[k]), k


@pytest.mark.parametrize("win,grid", [((0, 0, 64, 48), 1), ((37, 11, 50, 29), 1), ((96, 80, 32, 16), 1),
                                      ((8, 4, 40, 40), 2)])
def test_render_window_equals_crop_of_full_render(mrs, win, grid):
    # a window of the image: the same camera and per-pixel random numbers, so
    # every output (radiance, aux and extra layers) is the crop of the whole
    # render bit for bit, whatever the window's place and size
    sc = mrs.Scene(scenes.procedural(2, n_spheres=16, n_large=4))
    W, H = 128, 96
    full = mrs.render(sc, W, H, 4, 6, rr_start=3, seed=5, grid=grid, layers=True)
    part = mrs.render(sc, W, H, 4, 6, rr_start=3, seed=5, grid=grid, layers=True, window=win)
    x0, y0, w, h = win
    for k in ("radiance", "albedo", "normal", "depth", "diffuse", "specular", "variance"):
        assert torch.equal(part[k], full[k][y0:y0 + h, x0:x0 + w]), k
    assert int(part["counts"][0]) == w * h * 4


def test_render_window_rejects_outside_windows(mrs):
    sc = mrs.Scene(scenes.cornell_box(sphere_subdiv=1))
    for win in ((-1, 0, 8, 8), (0, 0, 0, 8), (60, 0, 8, 8), (0, 60, 8, 8)):
        with pytest.raises(Exception):
            mrs.render(sc, 64, 64, 1, 2, window=win)
