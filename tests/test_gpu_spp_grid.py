"""The trend of the method's spp study (Sec. 5, Table comp_spp) on procedural
scenes: a network trained with the method's spp randomisation (Sec. 4,
implementation details) is evaluated over a grid of (LRHS spp, HRLS spp)
pairs against high-spp renders of held-out scenes.  The paper's numbers are
on its dataset and are not reproduced; its trend is: more LRHS samples and
more HRLS samples both raise PSNR and lower RelMSE, and the fused image
beats the method without the network in every cell."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def grid():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2106_12802_gb300 as mrs
    from paper_2106_12802_gb300 import trainer
    train = trainer.make_dataset(range(300, 324), size=128, s=4, spp_tgt=256, spp_random=True,
                                 examples_per_scene=2, seed=1)
    net = mrs.Net(trainer.init_params(0))
    trainer.train(net, train, 600, batch=8, crop=64, lr=1e-3, seed=0, precision="bf16",
                  loss="robust")
    del train
    g = trainer.spp_grid(net, range(400, 404), size=128, s=4, spp_tgt=1024,
                         lr_spps=(2, 8, 32, 128), hr_spps=(1, 4))
    net.close()
    for (a, b), v in sorted(g.items()):
        print(f"spp grid LRHS {a:4d} HRLS {b}: PSNR {v['psnr']:.2f} dB (upsampled LRHS "
              f"{v['up_psnr']:.2f}), RelMSE {v['relmse']:.4f}")
    return g


def test_more_lrhs_samples_help(grid):
    # the trend of Table comp_spp: along a row (fixed HRLS spp) PSNR rises
    # with the LRHS spp at every step, by more than 0.3 dB over the row
    for b in (1, 4):
        rows = [grid[(a, b)] for a in (2, 8, 32, 128) if (a, b) in grid]
        psnr = [r["psnr"] for r in rows]
        assert all(y > x for x, y in zip(psnr, psnr[1:])), (b, psnr)
        assert psnr[-1] > psnr[0] + 0.3, (b, psnr)
        assert rows[-1]["relmse"] < rows[0]["relmse"], (b, rows)


def test_more_hrls_samples_help(grid):
    for a in (8, 32, 128):
        assert grid[(a, 4)]["psnr"] > grid[(a, 1)]["psnr"], (a, grid[(a, 1)], grid[(a, 4)])


def test_network_beats_upsampling_in_every_cell(grid):
    for key, v in grid.items():
        assert v["psnr"] > v["up_psnr"], (key, v)
