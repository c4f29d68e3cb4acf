"""The exclusion budget over the whole parity suite.

Each parity comparison leaves out the covered pixels whose result the FP64
oracle flags as ambiguous (ties within 1e-4 A, grazing silhouettes, SSAO
samples or occlusion tests within the FP32 error of a grid line or threshold,
toon band and outline edge decisions).  A single small scene can lose a few
pixels; over all comparisons of a session the excluded pixels must stay below
0.1 % of the covered ones.  Collected after the parity tests (file name), so
it sees their log; skipped when fewer than 20 comparisons ran.
"""
import pytest

import helpers

pytestmark = pytest.mark.gpu


def test_excluded_pixels_stay_below_a_tenth_of_a_percent():
    log = helpers.EXCLUSION_LOG
    if len(log) < 20:
        pytest.skip("only %d comparisons ran in this session" % len(log))
    cov = sum(c for _, c, _, _ in log)
    exc = sum(e for _, _, e, _ in log)
    assert cov > 100000
    assert exc <= 0.001 * cov, "%d of %d covered pixels excluded (%.4f%%)" % (exc, cov, 100.0 * exc / cov)
