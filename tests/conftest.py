import os
import sys
import warnings

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
