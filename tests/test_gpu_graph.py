"""A hybrid frame (LBVH rebuild, LRHS + HRLS renders, fusion, device-side gate)
captured in one CUDA graph and replayed gives bit-identical results to the
eager calls; the device-side gate agrees with the synchronous one."""
import numpy as np
import pytest

from synth import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_hybrid_frame_graph_replay_matches_eager():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2106_12802_gb300 as mrs
    from paper_2106_12802_gb300 import trainer
    sc = mrs.Scene(scenes.procedural(3, n_spheres=16, n_large=4))
    net = mrs.Net(trainer.init_params(0))
    h, H, s = 32, 128, 4
    dev = torch.device("cuda")
    lr = torch.empty((1, h, h, 3), device=dev)
    hr, alb, nrm = (torch.empty((1, H, H, 3), device=dev) for _ in range(3))
    dep = torch.empty((1, H, H), device=dev)
    fused = torch.empty((1, H, H, 3), device=dev)
    out = torch.empty((1, H, H, 3), device=dev)
    plain = torch.full((1, H, H, 3), 7.0, device=dev)
    used = torch.zeros(2, dtype=torch.int32, device=dev)
    D = torch.zeros(1, dtype=torch.float64, device=dev)

    def frame():
        sc.rebuild()
        mrs.render(sc, h, h, 16, 4, 2, 5, out={"radiance": lr[0]})
        mrs.render(sc, H, H, 2, 4, 2, 6, out={"radiance": hr[0], "albedo": alb[0],
                                              "normal": nrm[0], "depth": dep[0]})
        net.fuse(lr, hr, alb, nrm, s, precision="bf16", out=fused)
        mrs.gate_async(fused, lr, plain, s, 0.01, out=out, used=used, D=D)

    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        frame()
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    eager = {k: t.clone() for k, t in (("out", out), ("fused", fused), ("hr", hr), ("lr", lr))}
    eager_used, eager_D = used.clone(), D.clone()
    for t in (out, fused, hr, lr):
        t.zero_()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        frame()
    g.replay()
    torch.cuda.synchronize()
    for k, t in (("out", out), ("fused", fused), ("hr", hr), ("lr", lr)):
        assert torch.equal(t, eager[k]), k
    assert torch.equal(used, eager_used) and torch.equal(D, eager_D)
    # device-side decision == host-side gate
    _, used_sync, D_sync = mrs.gate(fused, lr, plain, s, 0.01)
    assert bool(used[0].item()) == used_sync and abs(D.item() - D_sync) <= 1e-12 * max(D_sync, 1e-30)
    expect = plain if used_sync else fused
    assert torch.equal(out, expect)
