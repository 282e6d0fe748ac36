import os
import sys
import warnings

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# scipy's adaptive quadrature warns when asked for near-machine precision
warnings.filterwarnings("ignore", message=".*roundoff error.*")
warnings.filterwarnings("ignore", message=".*maximum number of subdivisions.*")
warnings.filterwarnings("ignore", message=".*Extremely bad integrand.*")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the compiled library")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def fixsum_host(tmp_path_factory):
    """Host build (g++) of the step kernels' fixed-point sums (csrc/fixsum.cuh) through
    tests/native/fixsum_host.cpp: fx_density(n, f, out) and fx_stencil(n, p, out)."""
    import ctypes as C
    import subprocess

    d = tmp_path_factory.mktemp("fixsum")
    so = str(d / "libfixsum_host.so")
    subprocess.run(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-o", so,
                    os.path.join(ROOT, "tests", "native", "fixsum_host.cpp")], check=True)
    lib = C.CDLL(so)
    for name in ("fx_density", "fx_stencil", "fx_j_h"):
        getattr(lib, name).argtypes = [C.c_longlong, C.c_void_p, C.c_void_p]
        getattr(lib, name).restype = None
    for name in ("fx_populations", "fx_populations_transpose"):
        getattr(lib, name).argtypes = [C.c_longlong, C.c_int, C.c_void_p, C.c_void_p]
        getattr(lib, name).restype = None
    for name in ("fx_j_h_transpose", "fx_psi_gather"):
        getattr(lib, name).argtypes = [C.c_longlong, C.c_void_p, C.c_void_p]
        getattr(lib, name).restype = None
    lib.fx_lambda.argtypes = [C.c_longlong, C.c_int, C.c_void_p, C.c_void_p]
    lib.fx_lambda.restype = None
    return lib
