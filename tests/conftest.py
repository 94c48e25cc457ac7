import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
HERE = os.path.dirname(os.path.abspath(__file__))
if HERE not in sys.path:
    sys.path.insert(0, HERE)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a); runs the CUDA path through the C ABI")
    config.addinivalue_line("markers", "slow: long-running (minutes) check")
    config.addinivalue_line("markers", "oracle_full(name): compares with the oracle's full B of workload `name`, "
                                       "computed in a background process from the start of the session")


def pytest_collection_finish(session):
    """Starts the oracle jobs of the selected full-size parity tests at once,
    so they run while the other tests do."""
    if session.config.option.collectonly:
        return
    names = []
    for item in session.items:
        for mark in item.iter_markers("oracle_full"):
            names.extend(mark.args)
    if names:
        import oracle_jobs
        oracle_jobs.start(sorted(set(names)))


def pytest_sessionfinish(session, exitstatus):
    mod = sys.modules.get("oracle_jobs")
    if mod is not None:
        mod.stop()
