import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built extension")
    config.addinivalue_line("markers", "slow: long-running CPU test")
    config.addinivalue_line("markers", "oracle_cases(*names): oracle references computed in background "
                                       "processes (tests/oracle_jobs.py)")


def pytest_collection_finish(session):
    """Start the background oracle jobs of the selected tests before any of them runs,
    so that they overlap with the rest of the session."""
    names = []
    for item in session.items:
        m = item.get_closest_marker("oracle_cases")
        if m:
            names += [n for n in m.args if n not in names]
    if names:
        import oracle_jobs
        oracle_jobs.submit(names)


def pytest_sessionfinish(session, exitstatus):
    mod = sys.modules.get("oracle_jobs")
    if mod is not None:
        mod.shutdown()


@pytest.fixture(scope="session")
def lib():
    """The built CUDA library (GPU tests only); fails loudly when it is missing."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1604_08057_gb300 import binding
    return binding.load()
