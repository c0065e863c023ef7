import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def orc():
    import oracle

    oracle.build()
    return oracle


def pytest_terminal_summary(terminalreporter, exitstatus, config):
    """The parity statistics of the session (one row per compared view): flagged depth ties, texel-ambiguous
    pixels and excluded vertices with their shares, and the gradient components that fail the stated
    1e-6 + 1e-4 |o| bound without the conditioning term (default path) with that term's largest share."""
    import json

    from tests import parity

    if not parity.LOG:
        return
    tr = terminalreporter
    tr.section("parity statistics")
    tr.write_line(f"{'comparison':<44} {'det':>3} {'ties':>9} {'texamb':>9} {'excl.V':>9} {'strict_fail':>11} "
                  f"{'of':>8} {'S share':>8} {'worst':>7}")
    for r in parity.LOG:
        if "excluded" not in r:
            continue
        tr.write_line(f"{(r['label'] + ' v' + str(r['view']))[:44]:<44} {('yes' if r['deterministic'] else 'no'):>3} "
                      f"{r['tie_share']:9.2e} {r['texamb_share']:9.2e} {r['excluded_share']:9.2e} "
                      f"{r['strict_fail']:11d} {r['components']:8d} {r['cond_share_max']:8.3f} "
                      f"{r['grad_worst']:7.3f}")
    path = os.environ.get("MER_PARITY_LOG")
    if path:
        with open(path, "w") as f:
            json.dump(parity.LOG, f, indent=1)
