"""The soft tests' candidate filter (helpers.soft_candidates) leaves the oracle's outputs unchanged."""
import numpy as np

import oracle
from paper_2501_12750_gb300 import scenes

from helpers import soft_candidates


def test_candidate_filter_gives_the_full_oracle_result():
    s = scenes.config5(n=3000, size=96)
    x64 = s.xyzr.astype(np.float64)
    sizes = []
    for v in (0, 5, 11):
        cam = s.cameras[v]
        for (x0, y0, x1, y1) in [(30, 30, 45, 41), (0, 0, 9, 95), (60, 70, 95, 95)]:
            yy, xx = np.mgrid[y0:y1 + 1, x0:x1 + 1]
            pix = np.ascontiguousarray(np.stack([xx.ravel(), yy.ravel()], 1).astype(np.int32))
            full = oracle.soft_forward(x64, cam, pix, amb_tol=1e-3)
            cand = soft_candidates(x64, cam, (x0, y0), (x1, y1))
            sizes.append(len(cand))
            sub = oracle.soft_forward(x64[cand], cam, pix, amb_tol=1e-3)
            np.testing.assert_array_equal(sub.A, full.A)
            np.testing.assert_array_equal(sub.D, full.D)
            np.testing.assert_array_equal(sub.N, full.N)
            np.testing.assert_array_equal(sub.n_used, full.n_used)
            np.testing.assert_array_equal(sub.flags, full.flags)
            gA = np.random.default_rng(v).normal(size=len(pix))
            gD = np.zeros(len(pix))
            gN = np.zeros((len(pix), 3))
            gf = oracle.soft_vjp(x64, cam, pix, gA, gD, gN)
            gs = oracle.soft_vjp(x64[cand], cam, pix, gA, gD, gN)
            np.testing.assert_allclose(gs, gf[cand], rtol=1e-12, atol=1e-18)  # per-thread summation order
            rest = np.setdiff1d(np.arange(len(x64)), cand)
            assert (gf[rest] == 0).all()
    assert np.mean(sizes) < 0.8 * len(x64)  # the filter does remove atoms
