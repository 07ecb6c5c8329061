"""Oracle pins: Morton codes, radix-tree LBVH and ray casting."""
import numpy as np

from synth import scenes


def _ref_morton(q):
    out = 0
    for i in range(10):
        for a, sh in ((0, 2), (1, 1), (2, 0)):
            out |= ((int(q[a]) >> i) & 1) << (3 * i + sh)
    return out


def test_morton_corners(orc):
    # tiny triangles at the corners of the unit cube: centroid == vertex
    pts = np.array([[0, 0, 0], [1, 1, 1], [1, 0, 0], [0, 1, 0], [0, 0, 1], [0.5, 0.25, 0.75]],
                   dtype=np.float32)
    V = np.repeat(pts[:, None, :], 3, axis=1)
    codes = orc.morton(V)
    assert codes[0] == 0
    assert codes[1] == (1 << 30) - 1            # all 30 bits set (clamped to 1023)
    assert codes[2] == _ref_morton((1023, 0, 0))
    assert codes[3] == _ref_morton((0, 1023, 0))
    assert codes[4] == _ref_morton((0, 0, 1023))
    assert codes[5] == _ref_morton((512, 256, 768))


def _check_tree(V, t):
    n = len(V)
    order, left, right, box = t["order"], t["left"], t["right"], t["box"]
    assert sorted(order.tolist()) == list(range(n))
    keys = [(int(t["morton"][p]) << 32) | int(p) for p in order]
    assert keys == sorted(keys)
    if n == 1:
        return
    seen = np.zeros(2 * n - 1, int)
    seen[0] += 1
    for i in range(n - 1):
        seen[left[i]] += 1
        seen[right[i]] += 1
    assert (seen == 1).all()                      # every node has exactly one parent
    for i in range(n - 1):
        for c in (left[i], right[i]):
            assert (box[i, :3] <= box[c, :3]).all() and (box[i, 3:] >= box[c, 3:]).all()
    for k in range(n):
        tri = V[order[k]]
        assert np.array_equal(box[n - 1 + k, :3], tri.min(axis=0))
        assert np.array_equal(box[n - 1 + k, 3:], tri.max(axis=0))

    def leaves(node):
        if node >= n - 1:
            return [node - (n - 1)]
        return leaves(left[node]) + leaves(right[node])
    # in-order leaves are the sorted order: each internal node covers a contiguous range
    assert leaves(0) == list(range(n))


def test_radix_tree_invariants(orc):
    for n in (1, 2, 3, 7, 64, 333):
        V = scenes.random_triangles(n, n)["V"]
        _check_tree(V, orc.lbvh(V))


def test_duplicate_morton_codes(orc):
    # all centroids equal -> all codes equal; ties fall back on the prim index
    V = np.repeat(np.array([[[0, 0, 0], [1, 0, 0], [0, 1, 0]]], np.float32), 40, axis=0)
    V[::2] += 0.0
    t = orc.lbvh(V)
    assert (t["morton"] == t["morton"][0]).all()
    assert t["order"].tolist() == list(range(40))
    _check_tree(V, t)


def test_closest_hit_equals_brute_force(orc):
    for seed, n in ((0, 8), (1, 33), (2, 64)):
        V = scenes.random_triangles(seed, n)["V"]
        o, d = scenes.random_rays(seed, 20000)
        pb, tb = orc.cast(V, o, d, brute=True)
        pl, tl = orc.cast(V, o, d, brute=False)
        assert np.array_equal(pb, pl)
        assert np.array_equal(tb, tl)
        assert (pb >= 0).mean() > 0.03   # a real share of rays hits something


def test_closest_hit_on_cornell(orc):
    V = scenes.cornell_box(sphere_subdiv=1)["V"]
    o, d = scenes.random_rays(5, 20000, spread=1.0)
    o = o + np.float32([0, 1, 0])
    pb, tb = orc.cast(V, o, d, brute=True)
    pl, tl = orc.cast(V, o, d, brute=False)
    assert np.array_equal(pb, pl) and np.array_equal(tb, tl)
