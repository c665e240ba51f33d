"""Test-side access to the parity checks of the oracle package, plus a
registry of the counts each parity test saw (printed at the end of the run
by conftest.py, on green runs too)."""
from oracle.parity import *  # noqa: F401,F403

#: (test, what, checked, excluded, excluded within the loose bound,
#: excluded within the strict tolerance, failed, worst error / tolerance)
REPORTS = []


def report(name, what, tally):
    REPORTS.append((name, what, tally.checked, tally.excluded, tally.loose, tally.strict,
                    tally.failed, tally.worst))
