import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on the CPU")


def _build_library():
    """Compile libytn.so in-tree if it is missing or stale (nvcc cross-compiles
    without a GPU), so that the ABI tests run on a fresh checkout."""
    from paper_2405_12196_gb300 import build as B
    B.build()


_build_library()
