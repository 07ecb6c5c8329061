"""What the trained network gains over the method without it.

The network is trained on the GPU by the library's own forward/backward
kernels on (LRHS 64 spp, HRLS 4 spp + albedo/normal, 256-spp target) triples
rendered from seeded procedural scenes, then evaluated on held-out scenes
against their 256-spp renders.  The baselines are the method without the
network (bilinear upsampling of LRHS: an untrained network with a zero head
outputs exactly that) and the HRLS input.  The paper's own ablations make the
same comparisons (Sec. 5: the HRLS input and the super-resolution baselines);
its numbers are on its dataset and are not reproduced here."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def trained():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2106_12802_gb300 as mrs
    from paper_2106_12802_gb300 import trainer
    train = trainer.make_dataset(range(100, 124), size=128, s=4)
    test = trainer.make_dataset(range(200, 204), size=128, s=4)
    net = mrs.Net(trainer.init_params(0))
    before = trainer.evaluate(net, test)
    trainer.train(net, train, 300, batch=8, crop=64, lr=1e-3, seed=0)
    return mrs, trainer, net, test, before


def test_untrained_network_is_the_upsampled_lrhs(trained):
    _, _, _, _, before = trained
    assert before["fused"] == before["upsampled_lrhs"]


def test_trained_network_beats_the_method_without_it(trained):
    _, trainer, net, test, _ = trained
    ev = trainer.evaluate(net, test)
    assert ev["fused"]["psnr"] > ev["upsampled_lrhs"]["psnr"] + 3.0, ev
    assert ev["fused"]["psnr"] > ev["hrls"]["psnr"] + 3.0, ev
    assert ev["fused"]["relmse"] < 0.5 * ev["upsampled_lrhs"]["relmse"], ev
    assert ev["fused"]["relmse"] < ev["hrls"]["relmse"], ev


@pytest.mark.parametrize("prec,max_drop", [("bf16", 0.3), ("fp8", 1.5)])
def test_low_precision_inference_keeps_the_gain(trained, prec, max_drop):
    _, trainer, net, test, _ = trained
    ev32 = trainer.evaluate(net, test, precision="fp32")
    ev = trainer.evaluate(net, test, precision=prec)
    assert ev["fused"]["psnr"] > ev32["fused"]["psnr"] - max_drop, (prec, ev, ev32)
