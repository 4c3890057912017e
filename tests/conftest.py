import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    # the autotuners' choices made on the tests' small grids go to a cache file
    # of this session, not to the user's cache that later runs start from
    if not os.environ.get("STENCIL_TUNE_CACHE"):
        import tempfile
        os.environ["STENCIL_TUNE_CACHE"] = os.path.join(tempfile.mkdtemp(prefix="stencil_tune_"),
                                                        "tune.jsonl")


@pytest.fixture(scope="session")
def oracle_mod():
    import oracle
    oracle.build()
    return oracle
