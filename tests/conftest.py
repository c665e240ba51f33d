import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def pytest_terminal_summary(terminalreporter, exitstatus, config):
    """Print the parity counts every parity test recorded (green runs too):
    how many rows / trials were compared with the oracle, how many were
    excluded as ill-conditioned in FP32 (and of those, how many were within
    the loose bound they are still held to, and how many within the strict
    tolerance all the same), and the worst error / tolerance."""
    try:
        import parity
    except ImportError:
        return
    if not parity.REPORTS:
        return
    tr = terminalreporter
    tr.write_sep("-", "parity against the FP64 oracle")
    tr.write_line(f"{'test':46s} {'what':6s} {'checked':>10s} {'excluded':>9s} "
                  f"{'excl %':>7s} {'in loose':>9s} {'in tol':>8s} {'failed':>6s} {'worst':>7s}")
    for name, what, checked, excluded, loose, strict, failed, worst in parity.REPORTS:
        n = checked + excluded
        pct = 100.0 * excluded / n if n else 0.0
        tr.write_line(f"{name[:46]:46s} {what:6s} {checked:10d} {excluded:9d} {pct:6.2f}% "
                      f"{loose:9d} {strict:8d} {failed:6d} {worst:7.3f}")
