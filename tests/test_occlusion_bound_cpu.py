"""The occlusion pass's bound on a sphere's depth keys, checked in FP64.

A deferred sphere is dropped when lb, an FP32 lower bound on the depth key of every hit it can make, is at
least (q + 1) 65536 at every pixel of its box, q = (the pixel's depth key) >> 16 from the 16-bit depth plane
(so the pixel's key is below (q + 1) 65536); the test q <= lb / 65536 - 1 is exact in FP32.  The key of a hit
at depth d is
round((z_r - zlo) S) + round((d - z_r) S) with d >= z_c - r (z_r = z_c away from the eye plane), so every hit
key is at least (z_c - r - zlo) S - 2.  The kernel forms lb from the FP32 view depth vz (|vz - z_c| <= err) as
    lb = (vz - err - 1.000002 r - zlo - 2e-7 (|vz| + |zlo|)) S,  lb -= 4e-6 |lb| + 4096.
Random spheres, views and key scales: lb stays below the FP64 minimum hit key minus the tens of keys that
the FP32 hit offset may round away."""
import numpy as np


def test_occlusion_lower_bound_is_below_every_hit_key():
    rng = np.random.default_rng(13)
    f32 = np.float32
    for _ in range(20000):
        zc = rng.uniform(5.0, 5.0e4)
        r = rng.uniform(0.5, 3.0)
        zlo = zc - rng.uniform(r, 0.9 * zc)
        span = rng.uniform(10.0, 3.0e3)
        S = f32(4294967295.0 / span)
        d = rng.uniform(50.0, 5.0e4)  # |x - eye| summed over the axes, for the view error bound
        err = f32(4e-7 * d)
        vz = f32(zc + rng.uniform(-1.0, 1.0) * float(err))
        zl = f32(zlo)
        lb = f32(f32(f32(f32(f32(vz - err) - f32(r) * f32(1.000002)) - zl) - f32(2e-7) * f32(abs(vz) + abs(zl))) * S)
        lb = f32(f32(lb - abs(lb) * f32(4e-6)) - f32(4096.0))
        true_min = (zc - r - zlo) * float(S) - 2.0 - 64.0
        assert float(lb) < true_min
        # the plane test: a pixel whose key lies just below lb's 65536-multiple passes only when truly nearer
        if not 70000.0 < true_min < 4.0e9:
            continue
        q = np.uint32(true_min - 70000.0) >> np.uint32(16)
        if float(q) <= float(f32(f32(lb * f32(1.0 / 65536.0)) - f32(1.0))):
            assert (int(q) + 1) * 65536 <= float(lb) < true_min


def test_occlusion_bound_rejects_spheres_behind_a_surface():
    """The margin costs little: a sphere 1 A behind a surface's farthest key is rejected at every key scale."""
    rng = np.random.default_rng(14)
    f32 = np.float32
    rejected = 0
    for _ in range(2000):
        zc = rng.uniform(100.0, 2000.0)
        r = 1.5
        zlo = zc - rng.uniform(20.0, 90.0)
        S = f32(4294967295.0 / 400.0)
        err = f32(4e-7 * 3 * zc)
        vz = f32(zc)
        zl = f32(zlo)
        lb = f32(f32(f32(f32(f32(vz - err) - f32(r) * f32(1.000002)) - zl) - f32(2e-7) * f32(abs(vz) + abs(zl))) * S)
        lb = f32(f32(lb - abs(lb) * f32(4e-6)) - f32(4096.0))
        key = np.uint32((zc - r - 1.0 - zlo) * float(S))   # a surface 1 A in front of the sphere's front
        q = key >> np.uint32(16)
        rejected += float(q) <= float(f32(f32(lb * f32(1.0 / 65536.0)) - f32(1.0)))
    assert rejected == 2000
