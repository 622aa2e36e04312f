import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
# mutation tests (test_oracle_mutations.py): a directory holding a copy of the oracle package with one planted
# mistake comes first, so that `import oracle` loads the copy
if os.environ.get("ISIS_ORACLE_PKG_DIR"):
    sys.path.insert(0, os.environ["ISIS_ORACLE_PKG_DIR"])


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built CUDA library")


@pytest.fixture(scope="session")
def cuda_lib():
    """Build (if stale) and load the CUDA library; skip when no GPU is visible."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1307_6748_gb300 import build, isis
    build.build()
    isis.load()
    return isis
