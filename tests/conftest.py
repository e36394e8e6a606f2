import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built libbti")
    config.addinivalue_line("markers", "slow: minutes of CPU time")


def pytest_terminal_summary(terminalreporter, exitstatus, config):
    """Print every parity check's measured error beside its tolerance (tests/parity.py);
    with BTI_PARITY_JSON set, also write them to that file."""
    try:
        import parity
    except ImportError:
        return
    lines = parity.summary_lines()
    if not lines:
        return
    terminalreporter.write_sep("-", "parity errors")
    for line in lines:
        terminalreporter.write_line(line)
    path = os.environ.get("BTI_PARITY_JSON")
    if path:
        import json

        with open(path, "w") as f:
            json.dump([{"where": w, "what": what, "err": e, "tol": t} for w, what, e, t in parity.RECORDS], f, indent=1)
