"""The occlusion pass's two FP32 bounds, checked in FP64 on random spheres, pixel rays and key scales.

Writer (k_occl_upper): at pixel ray u = (a, b, 1) (the FP32 slopes of the pixel centre) the kernel forms, from
the FP32 view centre (vx, vy, vz) (|error| <= err per component),
    w = (vx - a vz, vy - b vz),  d2 = |w|^2 - (w.u)^2 / |u|^2,  tc = vz + (w.u) / |u|^2,
    del = 2 err + 1e-6 vz,  rr = 0.999 r - 2 del,
and when d2 <= rr^2 writes U = tc - 0.99999 sqrt((rr^2 - d2) / |u|^2) + 2 del + 1e-4.  Claims: the true
distance of the centre to that ray is below 0.9995 r (the hit test meets the sphere there), and U exceeds the
ray's true entry depth by at least 5e-5 A.

Test (k_occl_test): a sphere is dropped when every bound in its box is below
    thr = vz - 2 err - 1.000002 r - 2e-6 vz - 1e-4 - 1024 / S.
Claim: thr is below the sphere's nearest possible depth zc - r by more than 256 keys (the depth-to-key rounding
of both spheres' hits is tens of keys), so a pixel whose bound is below thr ends with a key below every key
of the dropped sphere.  sqrt and 1/|u|^2 use the hardware approximations in the kernel; here they are
perturbed by up to 2^-22 relative."""
import numpy as np

f32 = np.float32


def _f(x):
    return np.asarray(x, dtype=np.float64).astype(np.float32).astype(np.float64)


def _fma(a, b, c):
    # one rounding of an exact product-sum (products of two floats are exact in FP64)
    return _f(np.asarray(a, np.float64) * np.asarray(b, np.float64) + np.asarray(c, np.float64))


def _case(rng, n):
    zc = rng.uniform(20.0, 5.0e3, n)
    r = rng.uniform(0.6, 3.0, n)
    cx = rng.uniform(-0.4, 0.4, n) * zc
    cy = rng.uniform(-0.3, 0.3, n) * zc
    dist = np.abs(cx) + np.abs(cy) + zc  # |x - eye| summed over the axes, for the view error bound
    err = _f(4e-7 * dist)
    e = rng.uniform(-1.0, 1.0, (3, n)) * err
    vx, vy, vz = _f(cx + e[0]), _f(cy + e[1]), _f(zc + e[2])
    # a pixel ray near the sphere: slopes within 1.2 angular radii of the centre direction, rounded to FP32
    ang = r / zc
    a = _f(cx / zc + rng.uniform(-1.2, 1.2, n) * ang)
    b = _f(cy / zc + rng.uniform(-1.2, 1.2, n) * ang)
    return zc, r, cx, cy, err, vx, vy, vz, a, b


def test_upper_bound_is_above_the_entry_depth_where_it_is_written():
    rng = np.random.default_rng(13)
    n = 400000
    zc, r, cx, cy, err, vx, vy, vz, a, b = _case(rng, n)
    uu = _fma(a, a, _fma(b, b, 1.0))
    inv_uu = _f(1.0 / uu * (1.0 + rng.uniform(-2.0, 2.0, n) * 2.0 ** -23))
    dl = _f(_f(2.0 * err) + _f(1e-6 * vz))
    rr = _fma(r, _f(0.999), -2.0 * dl)
    wx, wy = _fma(-a, vz, vx), _fma(-b, vz, vy)
    wu = _fma(wx, a, _f(wy * b))
    d2 = _fma(_f(-wu * wu), inv_uu, _fma(wx, wx, _f(wy * wy)))
    rr2 = _f(rr * rr)
    wr = (d2 <= rr2) & (rr > 0)
    assert wr.sum() > n // 4
    tc = _fma(wu, inv_uu, vz)
    sq = _f(np.sqrt(_f(_f(np.maximum(rr2 - d2, 0.0)) * inv_uu)) * (1.0 + rng.uniform(-2.0, 2.0, n) * 2.0 ** -23))
    U = _f(_fma(_f(-0.99999), sq, tc) + _fma(2.0, dl, _f(1e-4)))
    # FP64 truth for the exact centre and the FP32 ray direction (a, b, 1) through the eye
    C = np.stack([cx, cy, zc])
    u = np.stack([a, b, np.ones(n)])
    uun = (u * u).sum(0)
    t_c = (C * u).sum(0) / uun                  # ray parameter (= depth) of the closest point
    d2t = (C * C).sum(0) - (C * u).sum(0) ** 2 / uun
    assert np.all(np.sqrt(np.maximum(d2t[wr], 0.0)) < 0.9995 * r[wr])
    entry = t_c - np.sqrt(np.maximum(r ** 2 - d2t, 0.0) / uun)
    assert np.all(U[wr] >= entry[wr] + 5e-5)
    # and the bound is close: within 2 del + 2e-4 A plus what the 0.999 r radius gives up near the rim
    slack = U[wr] - entry[wr]
    assert np.median(slack) < 0.05


def test_threshold_is_below_every_hit_depth_by_more_than_the_key_rounding():
    rng = np.random.default_rng(14)
    n = 400000
    zc, r, cx, cy, err, vx, vy, vz, a, b = _case(rng, n)
    span = rng.uniform(5.0, 3.0e3, n)
    S = _f(4294967295.0 / span)
    invS = _f(span / 4294967295.0)
    thr = _f(_f(_f(_f(_f(vz - _f(2.0 * err)) - _f(r * _f(1.000002))) - _f(_f(2e-6) * vz)) - _f(1e-4)) - _f(1024.0 * invS))
    assert np.all(thr < zc - r - 256.0 / S)


def test_threshold_rejects_a_sphere_behind_a_surface():
    """The margins cost little: a bound 0.01 A in front of a sphere's front rejects it at every key scale."""
    rng = np.random.default_rng(15)
    n = 20000
    zc = rng.uniform(100.0, 2000.0, n)
    r = np.full(n, 1.5)
    err = _f(4e-7 * 3.0 * zc)
    vz = _f(zc)
    invS = _f(400.0 / 4294967295.0)
    thr = _f(_f(_f(_f(_f(vz - _f(2.0 * err)) - _f(r * _f(1.000002))) - _f(_f(2e-6) * vz)) - _f(1e-4)) - _f(1024.0 * invS))
    bound = _f(zc - r - 0.01)
    # the kernel compares FP32 bit patterns; for positive floats that is the float order
    assert np.all(bound.astype(np.float32).view(np.uint32) < thr.astype(np.float32).view(np.uint32))
