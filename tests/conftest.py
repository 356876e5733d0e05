import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (runs on a GB300)")
    config.addinivalue_line("markers", "slow: longer CPU test")


@pytest.fixture(scope="session")
def orc():
    import oracle
    oracle.lib()
    return oracle


def pytest_terminal_summary(terminalreporter, exitstatus, config):
    """One line on the force-parity comparisons of the run: how many targets
    were checked, how many were judged against the term-magnitude floor, and
    the largest errors relative to |a| alone."""
    mod = sys.modules.get("test_gpu_parity")
    log = getattr(mod, "PARITY_LOG", None) if mod else None
    if not log:
        return
    chk = sum(r["checked"] for r in log)
    flo = sum(r["floored_frac"] * r["checked"] for r in log)
    terminalreporter.write_line(
        "force parity: %d comparisons, %d targets checked, %d near ties, %.2f%% judged against 0.1 sum|a_term| "
        "(largest fraction %.2f%%); max error vs |a|: %.2e (other targets), %.2e (floored targets); "
        "max phi error %.2e" % (len(log), chk, sum(r["near_tie"] for r in log), 100.0 * flo / max(chk, 1),
                                100.0 * max(r["floored_frac"] for r in log),
                                max(r["max_err_unfloored"] for r in log), max(r["max_err_floored_vs_a"] for r in log),
                                max(r["max_err_phi"] for r in log)))
    for r in log:
        terminalreporter.write_line(
            "  %-40s checked %8d  near ties %6d  floored %5.2f%%  max err vs |a| %.2e / floored %.2e  phi %.2e"
            % (r["case"], r["checked"], r["near_tie"], 100.0 * r["floored_frac"], r["max_err_unfloored"],
               r["max_err_floored_vs_a"], r["max_err_phi"]))
