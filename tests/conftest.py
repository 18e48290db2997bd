import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (runs the CUDA library)")
    config.addinivalue_line("markers", "slow: longer CPU-only oracle runs")


def pytest_terminal_summary(terminalreporter):
    """Measured error beside its bound for every parity comparison of the
    session, worst ratio per test (closest to its bound last)."""
    try:
        from tests import parity
    except Exception:
        return
    if not parity.RECORDS:
        return
    worst = {}
    for test, metric, value, bound in parity.RECORDS:
        ratio = value / bound if bound > 0 else 0.0
        if test not in worst or ratio > worst[test][0]:
            worst[test] = (ratio, metric, value, bound)
    tr = terminalreporter
    tr.section("parity: measured error / bound (worst comparison per test)")
    for test, (ratio, metric, value, bound) in sorted(worst.items(), key=lambda kv: kv[1][0]):
        tr.write_line(f"{ratio:7.3f}  {metric:18s} {value:.3e} / {bound:.0e}  {test.split('::')[-1]}")
    path = os.environ.get("DILBM_PARITY_LOG")
    if path:
        with open(path, "w") as fh:
            for rec in parity.RECORDS:
                fh.write("\t".join(str(v) for v in rec) + "\n")
