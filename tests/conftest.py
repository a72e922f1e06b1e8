import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built libfsaconv")
    config.addinivalue_line("markers", "slow: long CPU-only oracle runs (enabled with FSA_SLOW=1)")


def pytest_collection_modifyitems(config, items):
    if os.environ.get("FSA_SLOW"):
        return
    skip = pytest.mark.skip(reason="slow oracle pin; set FSA_SLOW=1")
    for it in items:
        if "slow" in it.keywords:
            it.add_marker(skip)


def read_golden(name):
    """Rows of a golden fixture: whitespace-separated fields, '#' comments."""
    rows = []
    with open(os.path.join(ROOT, "tests", "golden", name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                rows.append(line.split())
    return rows
