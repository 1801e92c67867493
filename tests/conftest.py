import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def cuda_available():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def pytest_collection_modifyitems(config, items):
    if cuda_available():
        return
    skip = pytest.mark.skip(reason="no CUDA device")
    for item in items:
        if "gpu" in item.keywords:
            item.add_marker(skip)


def pytest_terminal_summary(terminalreporter):
    """Print the errors against the oracle that tests record with record_property("err:<name>", value)."""
    rows = []
    for key in ("passed", "failed"):
        for rep in terminalreporter.stats.get(key, []):
            for k, v in getattr(rep, "user_properties", []):
                if isinstance(k, str) and k.startswith("err:"):
                    rows.append((rep.nodeid.split("::")[-1], k[4:], v))
    if rows:
        terminalreporter.write_sep("-", "measured errors against the FP64 oracle")
        for test, name, v in rows:
            terminalreporter.write_line(f"{test:60s} {name:28s} {v:.3e}")
