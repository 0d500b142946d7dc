import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def pytest_terminal_summary(terminalreporter):
    """Print the parity counts of the session (acceptance (a)-(c)): what was
    checked and what was excused, one line in total and one per paper-scale
    golden stage, so they stay visible under -q."""
    from tests import _parity
    line = _parity.summary()
    if not line:
        return
    terminalreporter.write_line(line)
    for r in _parity.RECORDS:
        if r["where"].startswith("c1/e2e/"):
            terminalreporter.write_line(
                f"parity {r['where']}: feasible {r['feasible']}, value-checked {r['value_checked']}, "
                f"loose {r['loose']}, mask exceptions {r.get('mask_exceptions_full_grid', r['mask_exceptions'])}"
                f" of {r.get('feasible_full_grid', r['feasible'])} feasible on the grid, decisive {r.get('decisive', 0)}, "
                f"policy-checked {r.get('policy_checked', 0)}, max rel err {r['max_rel_err']:.2e}")
