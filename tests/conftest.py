import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built CUDA library")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def pytest_collection_modifyitems(config, items):
    # gpu tests need a device; when none is present they are skipped, never silently re-routed
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except Exception:
        has_gpu = False
    if has_gpu:
        return
    skip = pytest.mark.skip(reason="no CUDA device")
    for it in items:
        if "gpu" in it.keywords:
            it.add_marker(skip)


def pytest_terminal_summary(terminalreporter, exitstatus, config):
    # pointwise errors of the parity checks, reported beside the norm-wise bar they passed
    try:
        from pointwise import RECORDS
    except Exception:
        return
    if not RECORDS:
        return
    tr = terminalreporter
    tr.section("pointwise potential errors of the parity checks (norm-wise is the asserted bar)")
    for r in RECORDS:
        tr.write_line(f"{r['case']:<48s} n={r['n']:<6d} normwise={r['normwise']:.2e} "
                      f"pointwise_rel_max={r['pointwise_rel_max']:.2e} "
                      f"pointwise_abs/max|phi|={r['pointwise_abs_over_max']:.2e}")
