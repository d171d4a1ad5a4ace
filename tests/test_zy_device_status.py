"""Device-side failure detection (collected after the other GPU tests, before
the no-allocation test).  (1) No bounded wait inside a kernel ran out during
the session.  (2) The failure path works without a fault: a self-test kernel
waits with a small limit on a barrier that nothing completes; the wait runs
out, the kernel returns, the host reads KCS_ERR_TIMEOUT, the context stays
usable and the counter can be reset."""
import ctypes as C

import pytest
import torch

pytestmark = pytest.mark.gpu


def test_no_kernel_wait_timed_out(cuda_ok):
    import paper_1803_10045_b300 as K
    assert K.device_status() == 0


def test_forced_wait_timeout_is_reported(cuda_ok):
    import paper_1803_10045_b300 as K
    from paper_1803_10045_b300._lib import lib
    s = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.kcs_selftest_wait_timeout(1000, s) == 0
    torch.cuda.synchronize()
    n = C.c_uint(0)
    assert lib.kcs_device_status(C.byref(n)) == 4          # KCS_ERR_TIMEOUT
    assert n.value == 1
    # the context is still usable
    x = torch.arange(10, device="cuda", dtype=torch.float32)
    assert float(x.sum()) == 45.0
    assert lib.kcs_device_status_reset() == 0
    assert K.device_status() == 0
