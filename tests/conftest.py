import os
import sys

# The oracle works on many small matrices: BLAS threading only adds contention.
os.environ.setdefault("OMP_NUM_THREADS", "1")
os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
os.environ.setdefault("MKL_NUM_THREADS", "1")

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: CPU test that takes more than a few seconds")


@pytest.fixture(scope="session")
def lib():
    """The built C-ABI library (GPU tests only)."""
    from paper_1910_09142_gb300 import binding
    return binding.load()


# Run order of the GPU files: the core parity tests (parity, mixed, serving,
# susceptibility) first, then the tests of features layered on them (fused
# schedule, resume, thermal averages), then the allocation-free entry point.
# That entry point keeps a device array for the life of the process, so it
# goes last. Under -x a failure in a later group still fails the run, but it
# cannot keep an earlier group from running.
_LATE = {"test_gpu_fused.py": 1, "test_gpu_resume.py": 1, "test_gpu_thermal.py": 1, "test_zz_no_alloc.py": 2}


def pytest_collection_modifyitems(config, items):
    items.sort(key=lambda it: _LATE.get(os.path.basename(str(it.fspath)), 0))    # stable
