"""Failure detection on the GPU without faulting it: a bounded device-side wait
that nothing completes must give up, report MRS_ERR_TIMEOUT, and leave the
context usable (a conv right after still matches)."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_device_wait_times_out_and_context_survives():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2106_12802_gb300 as mrs
    lib = mrs.load()
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.mrs_selftest_wait_timeout(2000, st) == -4      # MRS_ERR_TIMEOUT
    assert b"gave up" in lib.mrs_last_error()
    assert lib.mrs_selftest_wait_timeout(0, st) == -1         # argument check
    # the context still works
    x = torch.randn(1, 4, 40, 64, device="cuda")
    w = np.zeros((64, 3, 3, 64), np.float32)
    for c in range(64):
        w[c, 1, 1, c] = 1.0
    y = mrs.conv3x3(x, w, np.zeros(64, np.float32), precision="bf16")
    assert torch.allclose(y, x.to(torch.bfloat16).float(), atol=0, rtol=0)
