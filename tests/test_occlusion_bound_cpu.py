"""The occlusion pass's FP32 bounds and bound keys, checked in FP64 on random spheres, pixel rays and key scales.

Writer (k_occl_upper): at pixel ray u = (a, b, 1) (the FP32 slopes of the pixel centre) the kernel forms, from
the FP32 view centre (vx, vy, vz) (|error| <= err per component),
    w = (vx - a vz, vy - b vz),  d2 = |w|^2 - (w.u)^2 / |u|^2,  tc = vz + (w.u) / |u|^2,
    del = 2 err + 1e-6 vz,  rr = 0.999 r - 2 del,
and when d2 <= rr^2 writes U = tc - 0.99999 sqrt((rr^2 - d2) / |u|^2) + 2 del + 1e-4.  Claims: the true
distance of the centre to that ray is below 0.9995 r (the hit test meets the sphere there), and U exceeds the
ray's true entry depth by at least 5e-5 A.

Bound keys: the writer stores ceil((U - zlo) S (1 + 4e-6) + 8192) as the depth part of a key with the id of no
primitive; it must exceed the key of any hit at a depth below U.  Test (k_occl_test): a sphere is dropped when
the depth part of every key in its box is below floor(lb),
    lb = (vz - err - 1.000002 r - zlo - 2e-7 (|vz| + |zlo|)) S,  lb -= 4e-6 |lb| + 4096,
which must lie below the smallest key any of its hits can have.  sqrt and 1/|u|^2 use the hardware
approximations in the kernel; here they are perturbed by up to 2^-22 relative."""
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


def _bound_key_hi(ub, zlo, S):
    """Depth part of bound_key(ub, zlo, S) in FP32 (NaN for the background key)."""
    kf = _f(np.maximum(_f(_f(ub - zlo) * S), 0.0))
    kf = _f(_fma(kf, _f(4e-6), kf) + 8192.0)
    return np.where(kf < 4294967040.0, np.ceil(kf), np.nan)


def test_bound_key_is_above_every_key_of_a_hit_below_the_bound():
    """A hit at depth d <= ub has key round((z_r - zlo) S) + round((d - z_r) S) <= (d - zlo) S + 1 + tens of
    keys (the FP32 hit offset); the bound key's depth part must exceed that by a margin."""
    rng = np.random.default_rng(16)
    n = 400000
    zlo = _f(rng.uniform(1.0, 5.0e3, n))
    span = rng.uniform(5.0, 3.0e3, n)
    S = _f(4294966784.0 / span)
    ub = _f(zlo + rng.uniform(0.0, 1.0, n) * span)
    hi = _bound_key_hi(ub, zlo, S)
    ok = ~np.isnan(hi)
    assert ok.mean() > 0.99
    assert np.all(hi[ok] > (ub[ok] - zlo[ok]) * S[ok] + 128.0)


def test_key_lower_bound_is_below_every_hit_key():
    """lb = (vz - err - 1.000002 r - zlo - 2e-7 (|vz| + |zlo|)) S, less 4e-6 |lb| + 4096, floored: below the
    smallest key (zc - r - zlo) S - 66 any hit of the sphere can have."""
    rng = np.random.default_rng(14)
    n = 400000
    zc, r, cx, cy, err, vx, vy, vz, a, b = _case(rng, n)
    zlo = _f(zc - r - rng.uniform(0.0, 0.9, n) * (zc - r))
    span = rng.uniform(5.0, 3.0e3, n)
    S = _f(4294966784.0 / span)
    lb = _f(_f(_f(_f(_f(vz - err) - _f(r * _f(1.000002))) - zlo) - _f(_f(2e-7) * _f(np.abs(vz) + np.abs(zlo)))) * S)
    lb = _f(_f(lb - _f(np.abs(lb) * _f(4e-6))) - 4096.0)
    lbi = np.floor(np.minimum(lb, 4294967040.0))
    true_min = (zc - r - zlo.astype(np.float64)) * S - 66.0
    sel = lb > 0
    assert sel.mean() > 0.9
    assert np.all(lbi[sel] < true_min[sel])


def test_key_lower_bound_rejects_a_sphere_behind_a_surface():
    """The margins cost little: a bound key 0.01 A in front of a sphere's front lies below its lb."""
    rng = np.random.default_rng(15)
    n = 20000
    zc = rng.uniform(100.0, 2000.0, n)
    r = np.full(n, 1.5)
    err = _f(4e-7 * 3.0 * zc)
    vz = _f(zc)
    zlo = _f(zc - rng.uniform(20.0, 90.0, n))
    S = _f(4294966784.0 / 400.0)
    lb = _f(_f(_f(_f(_f(vz - err) - _f(r * _f(1.000002))) - zlo) - _f(_f(2e-7) * _f(np.abs(vz) + np.abs(zlo)))) * S)
    lb = _f(_f(lb - _f(np.abs(lb) * _f(4e-6))) - 4096.0)
    hi = _bound_key_hi(_f(zc - r - 0.01), zlo, S)
    assert np.all(hi < np.floor(lb))
