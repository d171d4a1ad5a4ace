"""After the GPU tests of the session: no bounded wait inside a kernel ran out
(collected after the other GPU tests, before the no-allocation test)."""
import pytest

pytestmark = pytest.mark.gpu


def test_no_kernel_wait_timed_out(cuda_ok):
    import paper_1803_10045_b300 as K
    assert K.device_status() == 0
