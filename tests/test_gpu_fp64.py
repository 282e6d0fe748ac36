"""The step kernels replace IEEE division and sqrt by a hardware seed plus one
third-order series step; check those against CUDA's correctly rounded results."""
import ctypes as C

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_fast_rcp_and_sqrt_within_a_few_ulp():
    from paper_2107_06355_gb300 import _lib as L

    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    st = L.lib().pplbm_fp64_selftest(1 << 24, 12345, C.c_void_p(out.data_ptr()),
                                     C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0
    torch.cuda.synchronize()
    err_rcp, err_sqrt = out.tolist()
    ulp = 2.0**-52
    assert err_rcp <= 2 * ulp, err_rcp
    assert err_sqrt <= 2 * ulp, err_sqrt
