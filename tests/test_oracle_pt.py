"""Oracle pins for the path tracer: closed forms of light transport,
unbiasedness, error decay, and the structure of the estimator."""
import numpy as np
import pytest

from synth import scenes


@pytest.mark.parametrize("D", [1, 2, 3, 6])
def test_white_furnace_closed_form(orc, D):
    # inside a closed emissive Lambertian sphere every path returns
    # Le * sum_{k=0..D} rho^k exactly (cosine sampling: f cos / pdf = rho)
    Le, rho = 1.5, 0.6
    r = orc.render(scenes.furnace_sphere(Le, rho), 12, 10, 3, D, seed=11)
    want = Le * sum(rho**k for k in range(D + 1))
    assert np.allclose(r["radiance"], want, rtol=2e-6, atol=0)
    assert (r["counts"] == 12 * 10 * 3).all()
    assert (r["shadow_counts"] == 0).all()     # no lights to sample


def test_white_furnace_with_roulette_is_unbiased(orc):
    Le, rho, D = 1.0, 0.7, 8
    r = orc.render(scenes.furnace_sphere(Le, rho), 32, 32, 32, D, rr_start=1, seed=5)
    want = Le * sum(rho**k for k in range(D + 1))
    x = r["radiance"].reshape(-1, 3)[:, 0].astype(np.float64)
    sem = x.std(ddof=1) / np.sqrt(len(x))
    assert abs(x.mean() - want) < 4 * sem
    assert sem > 0   # roulette does add variance
    c = r["counts"].astype(np.int64)
    assert (np.diff(c) <= 0).all() and c[-1] < c[1]


@pytest.mark.parametrize("D", [1, 2, 5])
def test_diffuse_plane_under_uniform_sky(orc, D):
    # NEE of the sky and BSDF sampling have equal (cosine) pdfs, so both MIS
    # weights are 1/2 and every path returns rho * L_sky
    rho, Lsky = 0.6, 2.0
    r = orc.render(scenes.sky_plane(rho, Lsky), 16, 16, 4, D, seed=2)
    assert np.allclose(r["radiance"], rho * Lsky, rtol=2e-6, atol=0)
    assert np.allclose(r["albedo"], rho) and np.allclose(r["normal"], [0, 1, 0])


def test_depth_zero_is_emission_only(orc):
    r = orc.render(scenes.cornell_box(sphere_subdiv=1), 16, 16, 4, 0, seed=0)
    rad = r["radiance"]
    # each sample returns 0 or Le = 15 (light seen directly): pixel = 15 k / 4
    assert set(np.unique(rad)) <= {15.0 * k / 4 for k in range(5)} and (rad == 15.0).any()


def test_error_decays_as_inverse_sqrt_spp(orc):
    # furnace with Russian roulette: unbiased, finite variance, exact reference
    Le, rho, D = 1.0, 0.7, 8
    sc = scenes.furnace_sphere(Le, rho)
    ref = Le * sum(rho**k for k in range(D + 1))
    spps = [4, 16, 64, 256]
    rmse = []
    for spp in spps:
        errs = [np.mean((orc.render(sc, 16, 16, spp, D, rr_start=1, seed=s)["radiance"] - ref) ** 2)
                for s in range(3)]
        rmse.append(np.sqrt(np.mean(errs)))
    slope = np.polyfit(np.log(spps), np.log(rmse), 1)[0]
    assert -0.55 < slope < -0.45, (slope, rmse)


def test_low_res_render_is_box_average_of_high_res(orc):
    # an LR pixel jitters over its whole footprint, so in expectation it is the
    # mean of the s x s HR pixels it covers (same camera frustum)
    sc = scenes.cornell_box(sphere_subdiv=2)
    lr = orc.render(sc, 8, 8, 2048, 3, seed=3)["radiance"].astype(np.float64)
    hr = orc.render(sc, 16, 16, 512, 3, seed=4)["radiance"].astype(np.float64)
    hr_down = hr.reshape(8, 2, 8, 2, 3).mean(axis=(1, 3))
    rel = np.abs(lr - hr_down).mean() / np.abs(hr_down).mean()
    assert rel < 0.05, rel


def test_sparse_grid_render_is_nearest_neighbour_of_high_res(orc):
    # grid=2: an LR pixel samples only the centre sub-pixel (2i+1, 2j+1) of its
    # 2 x 2 block, so in expectation it equals that HR pixel (nearest-neighbour
    # downsampling, the paper's LR images); the other sub-pixels and the box
    # average are far off on this scene's edges, so a wrong offset fails
    sc = scenes.cornell_box(sphere_subdiv=2)
    lr = orc.render(sc, 8, 8, 2048, 3, seed=3, grid=2)["radiance"].astype(np.float64)
    hr = orc.render(sc, 16, 16, 512, 3, seed=4)["radiance"].astype(np.float64)

    def rel(ref):
        return np.abs(lr - ref).mean() / np.abs(ref).mean()
    good = rel(hr[1::2, 1::2])
    assert good < 0.05, good
    for oy, ox in ((0, 0), (0, 1), (1, 0)):
        assert rel(hr[oy::2, ox::2]) > 4 * good, (oy, ox)
    assert rel(hr.reshape(8, 2, 8, 2, 3).mean(axis=(1, 3))) > 4 * good
    # grid=1 is the ordinary render, bit for bit
    a = orc.render(sc, 8, 8, 4, 3, seed=9)
    b = orc.render(sc, 8, 8, 4, 3, seed=9, grid=1)
    assert all(np.array_equal(a[k], b[k]) for k in a)
    with pytest.raises(ValueError):
        orc.render(sc, 8, 8, 4, 3, grid=0)


def test_aux_buffers_on_axis_aligned_walls(orc):
    sc = scenes.cornell_box(sphere_subdiv=1)
    W = H = 32
    r = orc.render(sc, W, H, 4, 2, seed=0)
    # centre pixel sees the back wall (z = -1): white albedo, normal +z
    c = r["albedo"][H // 2, W // 2]
    assert np.array_equal(c, np.float32([0.75, 0.75, 0.75]))
    assert np.array_equal(r["normal"][H // 2, W // 2], np.float32([0, 0, 1]))
    d = r["depth"][H // 2, W // 2]
    assert 4.39 < d < 4.45     # eye at z = 3.4, wall at z = -1, near-axial ray
    # bottom-centre pixel sees the floor: normal +y
    assert np.array_equal(r["normal"][H - 1, W // 2], np.float32([0, 1, 0]))


def test_rows_and_threads_do_not_change_results(orc):
    sc = scenes.cornell_box(sphere_subdiv=1)
    full = orc.render(sc, 16, 16, 4, 3, seed=9, threads=4)
    one = orc.render(sc, 16, 16, 4, 3, seed=9, threads=1)
    part = orc.render(sc, 16, 16, 4, 3, seed=9, rows=(5, 9), threads=2)
    assert np.array_equal(full["radiance"], one["radiance"])
    assert np.array_equal(full["radiance"][5:9], part["radiance"])
    assert np.array_equal(full["counts"], one["counts"])
    strided = orc.render(sc, 16, 16, 4, 3, seed=9, rows=(1, 16, 5), threads=3)
    assert np.array_equal(full["radiance"][1::5], strided["radiance"])
    assert np.array_equal(full["depth"][1::5], strided["depth"])


def test_seed_changes_estimate(orc):
    sc = scenes.cornell_box(sphere_subdiv=1)
    a = orc.render(sc, 8, 8, 2, 3, seed=1)["radiance"]
    b = orc.render(sc, 8, 8, 2, 3, seed=2)["radiance"]
    assert not np.array_equal(a, b)


def test_procedural_scene_size_and_value_range(orc):
    sc = scenes.procedural(0)
    assert len(sc["V"]) == 200962 + 6
    assert len(sc["lights"]) == 3
    r = orc.render(sc, 32, 32, 4, 4, rr_start=3, seed=0)
    rad = r["radiance"]
    assert np.isfinite(rad).all() and (rad >= 0).all()
    assert (rad <= 10).mean() > 0.95    # linear HDR mostly in [0, 10] (Sec. 3.2)


def test_extra_layers_decompose_radiance(orc):
    # every sample's radiance goes to the layer of its first hit's lobe; the
    # Cornell box is closed and black outside (every sample hits), with
    # Lambertian walls and one GGX sphere
    r = orc.render(scenes.cornell_box(sphere_subdiv=2), 16, 16, 8, 4, seed=1)
    assert (r["specular"] > 0).any() and (r["diffuse"] > 0).any()
    assert np.allclose(r["diffuse"] + r["specular"], r["radiance"], rtol=1e-5, atol=1e-7)
    # a pixel's layers are either all-diffuse or contain the sphere's samples
    only_d = ~r["specular"].any(axis=2)
    assert np.allclose(r["diffuse"][only_d], r["radiance"][only_d], rtol=1e-5, atol=1e-7)
    # the procedural scene mixes Lambertian and GGX spheres under an environment
    # seen directly by some samples: the two layers never exceed the radiance
    p = orc.render(scenes.procedural(0), 24, 24, 4, 4, rr_start=3, seed=2)
    assert (p["specular"] > 0).any() and (p["diffuse"] > 0).any()
    assert (p["diffuse"] + p["specular"] <= p["radiance"] * (1 + 1e-5) + 1e-6).all()


def test_extra_layers_closed_forms(orc):
    # diffuse plane under a uniform sky, cosine-sampled, one scattering event:
    # every sample is rho * L_sky, so diffuse = 1.2 and the variance is 0
    r = orc.render(scenes.sky_plane(0.6, 2.0), 16, 16, 8, 2, seed=3)
    assert np.allclose(r["diffuse"], 1.2, rtol=2e-6) and not r["specular"].any()
    assert (r["variance"] <= 1e-10).all()
    # white furnace without roulette: zero-variance estimator too
    f = orc.render(scenes.furnace_sphere(1.5, 0.6), 8, 8, 16, 5, seed=4)
    assert (f["variance"] <= 1e-6 * f["radiance"] ** 2).all()
    # one sample per pixel has no sample variance
    assert not orc.render(scenes.cornell_box(sphere_subdiv=1), 8, 8, 1, 3)["variance"].any()


def test_variance_layer_matches_spread_of_independent_renders(orc):
    # the layer estimates the variance of the pixel mean: its average over
    # pixels matches the variance of the pixel values across independent
    # renders (different seeds) at the same spp
    sc = scenes.cornell_box(sphere_subdiv=2)
    runs = [orc.render(sc, 8, 8, 16, 3, seed=100 + k) for k in range(96)]
    rad = np.stack([r["radiance"] for r in runs]).astype(np.float64)
    emp = rad.var(axis=0, ddof=1)
    est = np.stack([r["variance"] for r in runs]).astype(np.float64).mean(axis=0)
    ratio = est.sum() / emp.sum()
    assert 0.85 < ratio < 1.15, ratio


# --------------------------------------------------------------------------
# area lights: next-event estimation, BSDF sampling and their MIS combination
# --------------------------------------------------------------------------

def _plane_points(cam, W, H, k=8):
    """Points where the camera rays of a k x k midpoint grid inside every
    pixel meet the plane y = 0 (the scene's pinhole model: pixel (x, y) spans
    image coordinates a = 2 (x + jx) / W - 1, b = 1 - 2 (y + jy) / H)."""
    cam = cam.astype(np.float64)
    eye, fwd, rgt, up = cam[0:3], cam[3:6], cam[6:9], cam[9:12]
    j = (np.arange(k) + 0.5) / k
    sx = (np.arange(W)[:, None] + j[None, :]).reshape(-1) / W
    sy = (np.arange(H)[:, None] + j[None, :]).reshape(-1) / H
    a = 2 * sx - 1
    b = 1 - 2 * sy
    d = fwd[None, None] + b[:, None, None] * up + a[None, :, None] * rgt   # [H k, W k, 3]
    t = -eye[1] / d[..., 1]
    return eye + d * t[..., None]


def _projected_solid_angle(x, quad):
    """Lambert's closed form for a polygon seen from points x [.., 3] on a
    surface with normal +y: the integral of cos(theta) over the solid angle
    it subtends, 1/2 |sum_i gamma_i n . unit(r_i x r_i+1)| with r_i the unit
    vectors to its vertices and gamma_i the angle between consecutive ones."""
    r = [v - x for v in quad]
    r = [v / np.linalg.norm(v, axis=-1, keepdims=True) for v in r]
    acc = 0.0
    for i in range(len(r)):
        a, b = r[i], r[(i + 1) % len(r)]
        c = np.cross(a, b)
        gam = np.arccos(np.clip(np.sum(a * b, -1), -1, 1))
        acc = acc + gam * c[..., 1] / np.linalg.norm(c, axis=-1)
    return 0.5 * np.abs(acc)


def _direct_light_closed_form(sc, rho, W, H, k=8):
    """Expected pixel radiance of a Lambertian plane under quad lights (Le_k,
    projected solid angle P_k) and an environment L_env that the lights
    block: rho / pi * (sum_k Le_k P_k + L_env (pi - sum_k P_k)), averaged
    over each pixel's footprint."""
    x = _plane_points(sc["cam"], W, H, k)
    env = sc["env"].astype(np.float64)
    E = np.zeros(x.shape[:2] + (3,)) + env * np.pi
    for p0, e1, e2, le in scenes.LIGHTS_OVER_PLANE:
        p0, e1, e2, le = (np.array(v, np.float64) for v in (p0, e1, e2, le))
        P = _projected_solid_angle(x, [p0, p0 + e1, p0 + e1 + e2, p0 + e2])
        E = E + P[..., None] * (le - env)
    L = rho / np.pi * E
    return L.reshape(H, k, W, k, 3).mean(axis=(1, 3))


def _z_scores(r, want, block=8):
    """z of the image sum and of each block sum against want, with the
    estimator's own per-pixel variance of the mean."""
    d = r["radiance"].astype(np.float64) - want
    v = r["variance"].astype(np.float64)
    H, W, _ = d.shape
    zs = [d.sum(axis=(0, 1)) / np.sqrt(v.sum(axis=(0, 1)))]
    db = d.reshape(H // block, block, W // block, block, 3).sum(axis=(1, 3))
    vb = v.reshape(H // block, block, W // block, block, 3).sum(axis=(1, 3))
    zs.append((db / np.sqrt(vb)).reshape(-1, 3))
    return np.abs(zs[0]).max(), np.abs(zs[1]).max()


@pytest.mark.parametrize("env", [0.0, 0.3])
@pytest.mark.parametrize("estimator", ["mis", "light", "bsdf"])
def test_quad_lights_over_diffuse_plane_closed_form(orc, estimator, env):
    # one scattering event on a Lambertian plane: the pixel sees the direct
    # light of two quads (different areas and colours) and of the environment
    # they block; with the environment there are 3 choices of light to pick
    rho = 0.6
    sc = scenes.lights_over_plane(scenes.LAMBERT, (rho, rho, rho), env=env)
    W = H = 32
    want = _direct_light_closed_form(sc, rho, W, H)
    r = orc.render(sc, W, H, 256, 1, seed=21, estimator=estimator)
    assert np.allclose(r["albedo"], rho) and np.allclose(r["normal"], [0, 1, 0])
    z_all, z_blk = _z_scores(r, want)
    assert z_all < 4.0 and z_blk < 4.5, (z_all, z_blk)
    rel = abs(r["radiance"].mean() - want.mean()) / want.mean()
    assert rel < 0.02, rel
    shadow = r["shadow_counts"]
    if estimator == "bsdf":
        assert shadow.sum() == 0
    else:
        assert shadow[0] > 0


@pytest.mark.parametrize("alpha", [0.15, 0.5])
def test_quad_lights_over_ggx_plane_estimators_agree(orc, alpha):
    # no closed form for a rough conductor, but light sampling alone, BSDF
    # sampling alone and their MIS combination estimate the same integral:
    # the BSDF value of the evaluator (light sampling), the weight of the
    # sampler (BSDF sampling) and both pdfs inside the MIS weights must agree
    sc = scenes.lights_over_plane(scenes.GGX, (0.9, 0.6, 0.3), alpha=alpha, env=0.3)
    W = H = 32
    rs = {e: orc.render(sc, W, H, 512, 1, seed=30 + i, estimator=e)
          for i, e in enumerate(("mis", "light", "bsdf"))}
    for a, b in (("mis", "light"), ("mis", "bsdf"), ("light", "bsdf")):
        d = rs[a]["radiance"].astype(np.float64) - rs[b]["radiance"]
        v = rs[a]["variance"].astype(np.float64) + rs[b]["variance"]
        z = np.abs(d.sum(axis=(0, 1)) / np.sqrt(v.sum(axis=(0, 1)))).max()
        db = d.reshape(4, 8, 4, 8, 3).sum(axis=(1, 3))
        vb = v.reshape(4, 8, 4, 8, 3).sum(axis=(1, 3))
        zb = np.abs(db / np.sqrt(vb)).max()
        assert z < 4.0 and zb < 4.5, (a, b, z, zb)
    # MIS is never the worse of the two techniques it combines (it need not
    # be the best: the power heuristic is near-optimal, not optimal)
    var = {e: rs[e]["variance"].sum() for e in rs}
    assert var["mis"] < max(var["light"], var["bsdf"]), var
