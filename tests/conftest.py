import os
import sys
import types

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


# Max-norm errors recorded by the parity tests, printed once at the end of the
# run (one line per case and dtype: the largest error over the kernel
# selections and calls that test covered).  pytest loads this file as
# `conftest` while the tests import it as `tests.conftest`: the records live
# on one object in sys.modules that both copies share.
_LOG = sys.modules.setdefault("fsa_tests_parity_log", types.ModuleType("fsa_tests_parity_log"))
if not hasattr(_LOG, "records"):
    _LOG.records = {}
_PARITY = _LOG.records


def parity_record(case, dt, err_oracle, err_exact=None):
    """Record one result's error against the oracle (and against the exact
    potential, where the case has one) under (case, dt)."""
    k = (case, dt)
    o, e, cnt = _PARITY.get(k, (0.0, None, 0))
    o = max(o, float(err_oracle))
    if err_exact is not None:
        e = float(err_exact) if e is None else max(e, float(err_exact))
    _PARITY[k] = (o, e, cnt + 1)


def pytest_terminal_summary(terminalreporter):
    if not _PARITY:
        return
    terminalreporter.section("max-norm relative errors (largest over each case's results)")
    for (case, dt), (o, e, cnt) in sorted(_PARITY.items()):
        ex = f", vs exact potential {e:.2e}" if e is not None else ""
        terminalreporter.write_line(f"{case} {dt}: vs oracle {o:.2e}{ex} ({cnt} results)")
