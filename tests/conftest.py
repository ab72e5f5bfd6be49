import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the CUDA library")

# the library's in-kernel bounds checks report through a device error word;
# the tests make every call wait and check it
os.environ.setdefault("BDL_DEBUG_CHECK", "1")
