import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built renderer library")
    config.addinivalue_line("markers", "slow: long-running check (minutes)")


def pytest_collection_modifyitems(config, items):
    try:
        import torch
        have_gpu = torch.cuda.is_available()
    except Exception:  # pragma: no cover - torch import failure
        have_gpu = False
    if have_gpu:
        return
    skip = pytest.mark.skip(reason="no CUDA device")
    for it in items:
        if "gpu" in it.keywords:
            it.add_marker(skip)


def pytest_terminal_summary(terminalreporter):
    """Excluded-pixel fractions of every parity comparison run in this session."""
    helpers = sys.modules.get("helpers")
    log = getattr(helpers, "EXCLUSION_LOG", None)
    if not log:
        return
    cov = sum(c for _, c, _, _ in log)
    exc = sum(e for _, _, e, _ in log)
    terminalreporter.write_line("excluded pixels: %d of %d covered (%.4f%%) over %d comparisons"
                                % (exc, cov, 100.0 * exc / max(cov, 1), len(log)))
