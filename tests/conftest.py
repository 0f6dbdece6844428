import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: a test that takes more than a few seconds (CPU oracle work at full size)")


@pytest.fixture(scope="session")
def lib():
    """The built CUDA library through its Python binding (GPU tests only)."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2010_15491_gb300 as sr3d
    return sr3d


def pytest_sessionfinish(session, exitstatus):
    """With SR3D_PARITY_REPORT=path, write every recorded parity error there (JSON)."""
    path = os.environ.get("SR3D_PARITY_REPORT")
    if not path:
        return
    from tests._problems import REPORT
    if REPORT:
        import json
        with open(path, "w") as f:
            json.dump(REPORT, f, indent=1, sort_keys=True)
