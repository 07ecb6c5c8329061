"""The seeded scene generator (synth/scenegen.c), shared by the CUDA library's
seeded scene build and the test side: deterministic per seed, the documented
sizes and value ranges, lights facing the scene, and icospheres equal to the
independent numpy construction in synth/scenes.py."""
import numpy as np
import pytest

from synth import scenes


def test_procedural_is_a_pure_function_of_the_seed():
    a, b = scenes.procedural(3), scenes.procedural(3)
    for k in a:
        assert np.array_equal(a[k], b[k]), k
    c = scenes.procedural(4)
    assert not np.array_equal(a["V"], c["V"])
    # the full 64-bit seed counts
    assert not np.array_equal(scenes.procedural(2**63 + 3)["V"], a["V"])


def test_procedural_sizes_and_ranges():
    d = scenes.procedural(0)
    assert len(d["V"]) == 31 * 5120 + 33 * 1280 + 2 + 6
    assert d["mats"].shape == (1 + 64 + 3, 8) and d["lights"].shape == (3, 12)
    sph = d["mats"][1:65]
    assert set(np.unique(sph[:, 0])) <= {0.0, 1.0}
    assert 0.3 < sph[:, 0].mean() < 0.7                      # about half GGX
    assert (sph[:, 1:4] >= 0.1).all() and (sph[:, 1:4] <= 0.9).all()
    assert (sph[:, 4] >= 0.05).all() and (sph[:, 4] <= 1.0).all()
    L = d["lights"]
    n = np.cross(L[:, 3:6], L[:, 6:9])
    assert (n[:, 1] < 0).all() and (np.abs(n[:, [0, 2]]) < 1e-6).all()   # facing down
    assert (L[:, 1] >= 4).all() and (L[:, 1] <= 8).all()
    assert (L[:, 9] >= 5).all() and (L[:, 9] <= 20).all()
    assert np.array_equal(d["env"], np.float32([0.5, 0.5, 0.5]))
    # spheres of radius r are centred at height r, displaced by at most 0.2 r
    assert d["V"][:, :, 1].min() >= -0.2 - 1e-6
    # light triangles carry their light index, everything else -1
    tl = d["tri_light"]
    assert sorted(set(tl[tl >= 0])) == [0, 1, 2] and (tl >= 0).sum() == 6
    # ground normal up, light triangles' normals down
    g = d["V"][0]
    assert np.cross(g[1] - g[0], g[2] - g[0])[1] > 0
    lt = d["V"][tl >= 0]
    assert (np.cross(lt[:, 1] - lt[:, 0], lt[:, 2] - lt[:, 0])[:, 1] < 0).all()


def test_procedural_size_parameters():
    d = scenes.procedural(1, n_spheres=24, n_large=8)
    assert len(d["V"]) == 8 * 5120 + 16 * 1280 + 2 + 6
    with pytest.raises(ValueError):
        scenes.procedural(1, n_spheres=4, n_large=5)


@pytest.mark.parametrize("subdiv", [0, 1, 3])
def test_cornell_spheres_equal_numpy_icospheres(subdiv):
    # the C icosphere (edge-midpoint subdivision, projected to the sphere)
    # against the numpy construction of the same definition
    d = scenes.cornell_box(sphere_subdiv=subdiv)
    v, f = scenes.icosphere(subdiv)
    nt = len(f)
    assert len(d["V"]) == 12 + 2 * nt
    for k, c in enumerate(((-0.4, 0.25, -0.3), (0.4, 0.25, 0.2))):
        want = (v[f] * 0.25 + np.array(c)).astype(np.float32)
        got = d["V"][12 + k * nt: 12 + (k + 1) * nt]
        assert np.allclose(got, want, atol=2e-7, rtol=0)
    # outward winding: normal . (centroid - centre) > 0
    got = d["V"][12:12 + nt].astype(np.float64)
    nrm = np.cross(got[:, 1] - got[:, 0], got[:, 2] - got[:, 0])
    assert (np.sum(nrm * (got.mean(axis=1) - np.array([-0.4, 0.25, -0.3])), axis=1) > 0).all()


def test_cornell_layout():
    d = scenes.cornell_box(sphere_subdiv=1)
    assert d["mats"].shape == (6, 8) and d["lights"].shape == (1, 12)
    assert np.array_equal(d["mats"][3, 5:8], np.float32([15, 15, 15]))
    L = d["lights"][0]
    assert np.cross(L[3:6], L[6:9])[1] < 0
    assert np.array_equal(d["env"], np.zeros(3, np.float32))
    assert np.allclose(d["cam"][:3], [0, 1, 3.4]) and np.allclose(d["cam"][3:6], [0, 0, -1])
    # 40 degree field of view
    assert abs(np.linalg.norm(d["cam"][9:12]) - np.tan(np.radians(20))) < 1e-7
