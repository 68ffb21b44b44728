import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def pytest_terminal_summary(terminalreporter, exitstatus, config):
    """Print the parity numbers the GPU tests recorded (literal energy errors
    per component next to the other bars), so every run's log states them."""
    try:
        import parity
    except ImportError:
        return
    if not parity.RECORD:
        return
    tr = terminalreporter
    tr.write_sep("-", "parity against the FP64 oracle (value / bar)")
    for r in parity.RECORD:
        bar = "" if r["bar"] is None else f" / {r['bar']:.1e}"
        note = f"  [{r['note']}]" if r["note"] else ""
        tr.write_line(f"{r['case']:28s} {r['quantity']:26s} {r['value']:.3e}{bar}{note}")
