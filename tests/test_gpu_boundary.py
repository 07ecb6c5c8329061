"""The library's boundary calls that carry the method's own inputs and state,
through the C ABI: the seeded scene build (mrs_build_scene_seeded), the
checkpoint file (mrs_net_save / mrs_net_load) and the seeded network
(mrs_net_create_seeded)."""
import os

import numpy as np
import pytest

import oracle
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


@pytest.mark.parametrize("kind,seed,kw", [("procedural", 0, {}), ("procedural", 9, {"n_spheres": 24, "n_large": 8}),
                                          ("cornell", 0, {"sphere_subdiv": 2})])
def test_seeded_scene_equals_the_generated_arrays(mrs, kind, seed, kw):
    # the library generates the same scene the test side gets from the
    # generator: identical LBVH (codes of every centroid, leaf boxes of every
    # triangle) and an identical render, bit for bit
    desc = scenes.procedural(seed, **kw) if kind == "procedural" else scenes.cornell_box(**kw)
    a = mrs.Scene.seeded(seed, kind, **kw)
    b = mrs.Scene(desc)
    assert a.n == b.n == len(desc["V"])
    ea, eb = a.export_bvh(), b.export_bvh()
    for k in ("morton", "order", "left", "right"):
        assert np.array_equal(ea[k], eb[k]), k
    assert np.array_equal(ea["box"].view(np.uint32), eb["box"].view(np.uint32))
    ra = mrs.render(a, 48, 40, 4, 5, rr_start=3, seed=2)
    rb = mrs.render(b, 48, 40, 4, 5, rr_start=3, seed=2)
    for k in ra:
        assert torch.equal(ra[k], rb[k]), k
    # and the oracle agrees with the seeded scene's render
    ro = oracle.render(desc, 48, 40, 4, 5, rr_start=3, seed=2)
    assert np.array_equal(ra["counts"].cpu().numpy().astype(np.uint64), ro["counts"])
    assert np.allclose(ra["radiance"].cpu().numpy(), ro["radiance"], rtol=1e-4, atol=0)


def _batch(seed, N=2, h=4, w=6, s=4):
    rng = np.random.default_rng(seed)
    t = [rng.gamma(2.0, 0.5, (N, h, w, 3))] + [rng.uniform(0, 1, (N, h * s, w * s, 3)) for _ in range(4)]
    return [torch.from_numpy(a.astype(np.float32)).cuda() for a in t]


def test_checkpoint_file_round_trip_and_resume(mrs, tmp_path):
    t = _batch(1)
    a = mrs.Net(seed=3)
    a.set_loss("robust", 0.2)
    for _ in range(2):
        mrs.train_step(a, *t, 4, lr=1e-3, precision="bf16")
    path = tmp_path / "net.ckpt"
    mrs.save_checkpoint(a, path, seed=2**63 + 5)
    assert os.path.getsize(path) == 64 + 3 * 4 * mrs.NPARAMS
    assert not os.path.exists(str(path) + ".tmp")
    for _ in range(3):
        mrs.train_step(a, *t, 4, lr=1e-3, precision="bf16")
    b = mrs.Net(seed=99)                      # different weights, default loss
    assert mrs.load_checkpoint(b, path) == 2**63 + 5
    for _ in range(3):
        mrs.train_step(b, *t, 4, lr=1e-3, precision="bf16")
    sa, sb = mrs.get_state(a), mrs.get_state(b)
    assert sa["step"] == sb["step"] == 5
    for k in ("params", "adam_m", "adam_v"):       # the loss (robust, 0.2) came back too
        assert np.array_equal(sa[k], sb[k]), k


def test_checkpoint_file_errors_leave_the_net_unchanged(mrs, tmp_path):
    a = mrs.Net(seed=4)
    path = tmp_path / "ok.ckpt"
    mrs.save_checkpoint(a, path)
    raw = bytearray(path.read_bytes())
    b = mrs.Net(seed=5)
    before = b.get_params()
    cases = {
        "flipped payload byte": raw[:1000] + bytes([raw[1000] ^ 1]) + raw[1001:],
        "bad magic": b"X" + raw[1:],
        "truncated": raw[:-4],
        "trailing bytes": raw + b"\0",
        "bad version": raw[:12] + bytes([3, 0, 0, 0]) + raw[16:],
    }
    for name, data in cases.items():
        p = tmp_path / "bad.ckpt"
        p.write_bytes(bytes(data))
        with pytest.raises(mrs.MrsError) as e:
            mrs.load_checkpoint(b, p)
        assert e.value.status == -7, name        # MRS_ERR_FORMAT
        assert np.array_equal(b.get_params(), before), name
    with pytest.raises(mrs.MrsError) as e:
        mrs.load_checkpoint(b, tmp_path / "missing.ckpt")
    assert e.value.status == -8                  # MRS_ERR_IO
    # a checkpoint of the 21-channel network does not load into a 12-channel one
    c = mrs.Net(seed=1, input_channels=21)
    p21 = tmp_path / "net21.ckpt"
    mrs.save_checkpoint(c, p21)
    with pytest.raises(mrs.MrsError):
        mrs.load_checkpoint(b, p21)


def test_seeded_network_initialisation(mrs):
    from oracle import cnn
    a, b, c = mrs.Net(seed=7), mrs.Net(seed=7), mrs.Net(seed=8)
    pa = a.get_params()
    assert np.array_equal(pa, b.get_params()) and not np.array_equal(pa, c.get_params())
    for i, (wo, bo, ci, co) in enumerate(cnn.layer_offsets()):
        w, bias = pa[wo:bo].astype(np.float64), pa[bo:bo + co]
        assert not bias.any()
        if i == 17:
            assert not w.any()                    # the head starts at zero
            continue
        sd = np.sqrt(2.0 / (9 * ci)) * (0.1 if 1 <= i <= 16 and i % 2 == 0 else 1.0)
        assert abs(w.mean()) < 0.05 * sd
        assert abs(w.std() / sd - 1) < 0.05, (i, w.std() / sd)
    # the untrained network is the method without it: output = upsampled LRHS
    t = _batch(2)
    out = a.fuse(*t[:4], 4, precision="fp32").cpu().numpy()
    up = cnn.bilinear_up(t[0].cpu().numpy().astype(np.float64), 4)
    assert np.abs(out - up).max() <= 1e-6 * np.abs(up).max()
    assert mrs.Net(seed=7, input_channels=21).input_channels == 21
