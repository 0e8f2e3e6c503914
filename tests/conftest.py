import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


# Options beyond the paper's method (partition-of-unity patch weights, pointwise
# coefficients, curved elements, checkpoint/resume) run after the tests of the method
# itself, so that a stop at the first failure (-x) in them hides none of those; the
# allocation-free entry point's check (test_zz_no_alloc.py) is collected last of all.
_LATE = ("test_gpu_forward_error.py", "test_gpu_coefficients.py", "test_gpu_checkpoint.py", "test_gpu_curved.py",
         "test_gpu_weighting_pou.py", "test_zz_no_alloc.py")


def pytest_collection_modifyitems(session, config, items):
    def rank(item):
        name = item.nodeid.split("::")[0].rsplit("/", 1)[-1]
        return _LATE.index(name) + 1 if name in _LATE else 0
    items.sort(key=rank)   # stable: the order inside each group is kept
