"""The render tree: the radix tree (the default) and locally-ordered
clustering, in grid-wide rounds ("cluster") or inside the radix tree's
subtrees in one launch ("hcluster").  The exported trees are checked on the
host (every node but the root a child exactly once, leaf boxes the
triangles' boxes, every internal box the exact union of its children's);
closest hits and renders are the same with every tree, bit for bit, and
equal the oracle's; the clustering trees' surface-area cost and traversal
work are below the radix tree's on the procedural scene.  Sizes span the
single-block finish (2048 clusters), several grid-wide rounds, a subtree's
16 kept clusters (16, 17, 33 leaves), ties (identical triangles) and
degenerate (zero-area) triangles."""
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


def _half_area(lo, hi):
    e = np.maximum(hi - lo, 0.0)
    return e[..., 0] * e[..., 1] + e[..., 1] * e[..., 2] + e[..., 2] * e[..., 0]


def check_tree(t, V):
    """Validates the exported tree; returns its surface-area cost (internal
    node areas + leaf areas, over the root's)."""
    ns, child, box, order = t["ns"], t["child"], t["box"], t["order"]
    assert len(np.unique(order)) == ns
    if ns <= 1:
        return 0.0
    ids = child.ravel()
    assert np.array_equal(np.sort(ids), np.arange(1, 2 * ns - 1))   # root 0 is nobody's child
    bx = box.reshape(-1, 6)
    tri = np.asarray(V, np.float32).reshape(-1, 3, 3)[order]
    leaf = ids >= ns - 1
    k = ids[leaf] - (ns - 1)
    assert np.array_equal(bx[leaf, :3], tri[k].min(axis=1))
    assert np.array_equal(bx[leaf, 3:], tri[k].max(axis=1))
    c = ids[~leaf]
    assert np.array_equal(bx[~leaf, :3], box[c, :, :3].min(axis=1))
    assert np.array_equal(bx[~leaf, 3:], box[c, :, 3:].max(axis=1))
    # depth within the traversal's 128-entry stack (a far child per level);
    # every tree here is in fact at most 63 deep
    depth = np.zeros(ns - 1, np.int64)
    order_ = [0]
    for v in order_:
        for c_ in child[v]:
            if c_ < ns - 1:
                depth[c_] = depth[v] + 1
                order_.append(c_)
    assert depth.max() + 1 <= 64, depth.max()       # the stack holds 128
    node_lo, node_hi = box[:, :, :3].min(axis=1), box[:, :, 3:].max(axis=1)
    root = _half_area(node_lo[0], node_hi[0])
    return float((_half_area(node_lo, node_hi).sum() + _half_area(bx[leaf, :3], bx[leaf, 3:]).sum())
                 / root)


def _soup(seed, n, identical=False, degenerate=False):
    desc = scenes.random_triangles(seed, n)
    V = desc["V"].reshape(n, 3, 3)
    if identical:
        V[:] = V[0]
    if degenerate:
        V[::3, 2] = V[::3, 0]                 # every third triangle has zero area
        V[1::7, 1] = V[1::7, 0]
        V[1::7, 2] = V[1::7, 0]               # and some are points
    desc["V"] = V.reshape(desc["V"].shape)
    return desc


@pytest.mark.parametrize("kind", ["cluster", "hcluster"])
@pytest.mark.parametrize("n,kw", [(2, {}), (3, {}), (16, {}), (17, {}), (33, {}), (100, {}),
                                  (2047, {}), (2048, {}), (2049, {}), (5000, {}), (70000, {}),
                                  (3000, {"identical": True}), (4000, {"degenerate": True})])
def test_cluster_tree_is_valid(mrs, n, kw, kind):
    desc = _soup(n, n, **kw)
    sc = mrs.Scene(desc)
    assert sc.tree() == "lbvh"
    check_tree(sc.export_nodes(), desc["V"])
    sc.set_tree(kind)
    assert sc.tree() == kind
    check_tree(sc.export_nodes(), desc["V"])
    sc.rebuild()                        # the choice stays with the scene
    assert sc.tree() == kind
    check_tree(sc.export_nodes(), desc["V"])


@pytest.mark.parametrize("seed,n,kw", [(0, 8, {}), (2, 3000, {}), (3, 50000, {}),
                                       (4, 3000, {"identical": True}),
                                       (5, 4000, {"degenerate": True})])
def test_cast_same_with_every_tree_and_brute_force(mrs, orc, seed, n, kw):
    desc = _soup(seed, n, **kw)
    o, d = scenes.random_rays(seed, 40000)
    sc = mrs.Scene(desc)
    to, td = torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda()
    sc.set_tree("cluster")
    pc, tc = sc.cast(to, td)
    sc.set_tree("hcluster")
    ph, th = sc.cast(to, td)
    sc.set_tree("lbvh")
    assert sc.tree() == "lbvh"
    pl, tl = sc.cast(to, td)
    assert torch.equal(pc, pl) and torch.equal(tc, tl)
    assert torch.equal(ph, pl) and torch.equal(th, tl)
    pb, tb = orc.cast(desc["V"], o, d, brute=n <= 64)
    assert np.array_equal(pc.cpu().numpy(), pb)
    assert np.array_equal(tc.cpu().numpy(), tb)


def test_procedural_scene_trees(mrs, orc):
    # 200,968-triangle lit procedural scene: every tree valid, the clustering
    # ones with a lower surface-area cost and fewer node visits, renders
    # identical bit for bit and equal to the oracle's on a small image
    desc = scenes.procedural(0)
    sc = mrs.Scene(desc)
    cost, st, img = {}, {}, {}
    for kind in ("cluster", "hcluster", "lbvh"):
        sc.set_tree(kind)
        assert sc.tree() == kind
        cost[kind] = check_tree(sc.export_nodes(), desc["V"])
        st[kind] = mrs.render_stats(sc, 96, 96, 2, 8, 3, 7)
        img[kind] = mrs.render(sc, 96, 96, 2, 8, rr_start=3, seed=7)
    for kind in ("cluster", "hcluster"):
        for k in img["lbvh"]:
            assert torch.equal(img[kind][k], img["lbvh"][k]), (kind, k)
        assert cost[kind] < 0.9 * cost["lbvh"], cost
        assert st[kind]["visits"] < st["lbvh"]["visits"], st
    # the one-launch build keeps nearly the global rounds' quality
    assert cost["hcluster"] < 1.03 * cost["cluster"], cost
    r = orc.render(desc, 96, 96, 2, 8, rr_start=3, seed=7)
    rc = img["hcluster"]
    assert np.array_equal(rc["counts"].cpu().numpy().astype(np.uint64), r["counts"])
    assert np.array_equal(rc["shadow_counts"].cpu().numpy().astype(np.uint64), r["shadow_counts"])
    print("\nSAH cost:", {k: round(v, 2) for k, v in cost.items()}, "closest-hit node visits:",
          {k: v["visits"] for k, v in st.items()}, "shadow:", {k: v["shadow_visits"] for k, v in st.items()})


def test_hcluster_tree_with_overflowing_and_nan_boxes(mrs):
    # triangles a 1e20 apart make union areas overflow single precision and
    # a NaN vertex makes a NaN box: the one-launch build must still merge
    # every cluster (its pair areas are capped at FLT_MAX) into one valid
    # tree, whose closest hits equal the radix tree's (NaN triangles are
    # never hit)
    desc = _soup(11, 3000)
    V = desc["V"].reshape(3000, 3, 3)
    V[::40] *= np.float32(1e20)       # 75 of them: more than the 64 large triangles
                                      # tested outside the tree, so all are in it
    V[7::97, 1, 0] = np.nan
    desc["V"] = V.reshape(desc["V"].shape)
    o, d = scenes.random_rays(11, 20000)
    sc = mrs.Scene(desc)
    to, td = torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda()
    pl, tl = sc.cast(to, td)
    sc.set_tree("hcluster")
    assert sc.tree() == "hcluster"
    t = sc.export_nodes()
    ids = t["child"].ravel()
    assert np.array_equal(np.sort(ids), np.arange(1, 2 * t["ns"] - 1))
    ph, th = sc.cast(to, td)
    assert torch.equal(ph, pl) and torch.equal(th, tl)


def test_hcluster_node_ids_are_a_function_of_the_tree(mrs):
    # node ids come from the split positions, not from the order in which
    # warps merge: rebuilding gives the same node array bit for bit
    desc = _soup(8, 60000)
    sc = mrs.Scene(desc)
    sc.set_tree("hcluster")
    t0 = sc.export_nodes()
    for _ in range(3):
        sc.rebuild()
        t1 = sc.export_nodes()
        assert np.array_equal(t0["child"], t1["child"])
        assert np.array_equal(t0["box"], t1["box"])


def test_hcluster_tree_inside_a_capture(mrs):
    # the one-launch build reads nothing back, so a caller's stream capture
    # records it; replaying the capture rebuilds the same tree
    desc = _soup(9, 30000)
    sc = mrs.Scene(desc)
    sc.set_tree("hcluster")
    o, d = scenes.random_rays(9, 20000)
    to, td = torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda()
    p0, t0 = sc.cast(to, td)
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        sc.rebuild(stream=s)
    assert sc.tree() == "hcluster"
    g.replay()
    torch.cuda.synchronize()
    check_tree(sc.export_nodes(), desc["V"])
    p1, t1 = sc.cast(to, td)
    assert torch.equal(p0, p1) and torch.equal(t0, t1)


def test_set_tree_rejects_unknown_kind(mrs):
    from paper_2106_12802_gb300._lib import call
    sc = mrs.Scene(_soup(1, 10))
    with pytest.raises(mrs.MrsError):
        call("mrs_scene_set_tree", sc.handle, 7, None)
    assert sc.tree() == "lbvh"
