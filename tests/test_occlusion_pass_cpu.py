"""The batch occlusion pass end to end on a small crowded scene, emulated on the CPU.

A sphere blob is ray-cast exactly (FP64 entry depth per pixel centre, ties to the smaller id).  The pass is
then emulated with the kernels' FP32 formulas: the survivors in the front 35 % of the depth range write upper
bounds of their entry depth, as bound keys, at the pixels their rays certainly meet (k_occl_upper), and every
survivor whose candidate box holds only bound keys below its key bound is dropped (k_occl_test).  Claims: every
bound lies above the exact nearest depth of its pixel and every bound key above that depth's key, every key
bound below the key of its sphere's nearest depth, no dropped sphere holds any pixel of the exact image, the image of the kept spheres alone is the exact image bit for bit, and the pass
drops about half of the spheres (so the check is not vacuous)."""
import numpy as np

f32 = np.float32
W, H = 96, 64


def _scene(seed=3, n=8000):
    rng = np.random.default_rng(seed)
    # clumps of eight along random walks, as in the protein-like generator
    centres = np.cumsum(rng.normal(0.0, 0.7, (n // 8, 3)), axis=0)
    pos = (centres[:, None, :] + rng.normal(0.0, 1.0, (n // 8, 8, 3))).reshape(-1, 3)
    pos -= pos.mean(0)
    rad = rng.uniform(1.2, 1.9, len(pos))
    return pos, rad


def _camera(pos):
    ext = np.abs(pos).max()
    eye = np.array([0.0, 0.0, -2.6 * ext])
    f = H / (2.0 * np.tan(np.radians(20.0)))
    return eye, f


def _exact(pos, rad, eye, f, ids):
    """Exact nearest hit per pixel (depth along the view axis, id); ties to the smaller id."""
    depth = np.full((H, W), np.inf)
    owner = np.full((H, W), -1, np.int64)
    c = pos - eye
    ys, xs = np.mgrid[0:H, 0:W]
    a = (xs + 0.5 - W / 2) / f
    b = (H / 2 - ys - 0.5) / f
    uu = a * a + b * b + 1.0
    for i in ids:
        cu = c[i, 0] * a + c[i, 1] * b + c[i, 2]
        d2 = (c[i] ** 2).sum() - cu * cu / uu
        hit = d2 <= rad[i] ** 2
        t = np.where(hit, cu / uu - np.sqrt(np.maximum(rad[i] ** 2 - d2, 0.0) / uu), np.inf)
        better = (t < depth) | ((t == depth) & hit & (i < owner))
        depth = np.where(better, t, depth)
        owner = np.where(better, i, owner)
    return depth, owner


def _fma(a, b, c):
    return f32(np.float64(a) * np.float64(b) + np.float64(c))


def test_occlusion_pass_drops_only_spheres_that_hold_no_pixel():
    pos, rad = _scene()
    eye, f = _camera(pos)
    n = len(pos)
    depth, owner = _exact(pos, rad, eye, f, range(n))
    c = pos - eye
    # FP32 view positions with the view error bound of view_f32
    err = f32(4e-7) * f32(np.abs(c).sum(1))
    vx, vy, vz = (f32(c[:, 0]), f32(c[:, 1]), f32(c[:, 2]))
    r32 = f32(rad)
    zlo, zhi = float((c[:, 2] - rad).min()), float((c[:, 2] + rad).max())
    invS = f32((zhi - zlo) / 4294966784.0)
    zf = zlo + 0.35 * (zhi - zlo)
    fx, cx, cy, inv_f = f32(f), f32(W / 2), f32(H / 2), f32(1.0 / f)
    # k_occl_upper
    U = np.full((H, W), np.inf, dtype=np.float32)
    for i in range(n):
        if not (vz[i] - r32[i] - err[i] <= zf) or not (vz[i] > 2 * (r32[i] + err[i])):
            continue
        dl = f32(f32(2 * err[i]) + f32(1e-6) * vz[i])
        rr = _fma(r32[i], f32(0.999), -2 * dl)
        if rr <= 0:
            continue
        Rs = f32(rr * fx / vz[i])
        ux, uy = f32(cx - 0.5 + fx * vx[i] / vz[i]), f32(cy - 0.5 - fx * vy[i] / vz[i])
        rr2, dU = f32(rr * rr), _fma(2.0, dl, f32(1e-4))
        for py in range(max(int(np.ceil(uy - Rs)), 0), min(int(np.floor(uy + Rs)), H - 1) + 1):
            for px in range(max(int(np.ceil(ux - Rs)), 0), min(int(np.floor(ux + Rs)), W - 1) + 1):
                a = f32(f32(f32(px + 0.5) - cx) * inv_f)
                b = f32(f32(cy - f32(py + 0.5)) * inv_f)
                inv_uu = f32(1.0 / float(_fma(a, a, _fma(b, b, 1.0))))
                wx, wy = _fma(-a, vz[i], vx[i]), _fma(-b, vz[i], vy[i])
                wu = _fma(wx, a, f32(wy * b))
                d2 = _fma(f32(-wu * wu), inv_uu, _fma(wx, wx, f32(wy * wy)))
                if d2 <= rr2:
                    tc = _fma(wu, inv_uu, vz[i])
                    sq = f32(np.sqrt(f32(f32(rr2 - d2) * inv_uu)))
                    U[py, px] = min(U[py, px], f32(_fma(f32(-0.99999), sq, tc) + dU))
    # the writer's claim, pixel by pixel: every bound lies above the exact nearest depth there
    fin = np.isfinite(U)
    assert fin.sum() > 0.5 * (owner >= 0).sum()
    assert np.all(U[fin].astype(np.float64) >= depth[fin] + 5e-5)
    # as bound keys (depth parts): above the exact key of that depth by more than the key rounding
    S = f32(1.0) / invS
    kf = np.maximum(f32(f32(U - f32(zlo)) * S), f32(0.0))
    kf = f32(f32(kf * f32(4e-6) + kf) + f32(8192.0))
    KB = np.where(fin & (kf < 4294967040.0), np.ceil(kf.astype(np.float64)), np.inf)
    assert np.all(KB[fin] > (depth[fin] - float(f32(zlo))) * float(S) + 128.0)
    # k_occl_test, with each sphere's exact pixel box widened by a pixel for the candidate box
    dropped = []
    for i in range(n):
        if not (vz[i] > 2 * (r32[i] + err[i])):
            continue
        zl = f32(zlo)
        lb = f32(f32(f32(f32(vz[i] - err[i]) - f32(r32[i] * f32(1.000002))) - zl)
                 - f32(f32(2e-7) * f32(abs(vz[i]) + abs(zl))))
        lb = f32(f32(lb * S) - f32(abs(f32(lb * S)) * f32(4e-6))) - f32(4096.0)
        lbi = np.floor(min(float(lb), 4294967040.0))
        rp = f * rad[i] / c[i, 2] * 1.05 + 1.0
        u0, v0 = W / 2 + f * c[i, 0] / c[i, 2], H / 2 - f * c[i, 1] / c[i, 2]
        x0, x1 = max(int(np.floor(u0 - rp - 0.5)), 0), min(int(np.ceil(u0 + rp - 0.5)), W - 1)
        y0, y1 = max(int(np.floor(v0 - rp - 0.5)), 0), min(int(np.ceil(v0 + rp - 0.5)), H - 1)
        if x0 > x1 or y0 > y1:
            continue
        # the test's claim: its key bound lies below the key of the sphere's nearest depth by more than the key
        # rounding
        assert lbi < (c[i, 2] - rad[i] - float(zl)) * float(S) - 66.0
        if lb > 0 and (KB[y0:y1 + 1, x0:x1 + 1] < lbi).all():
            dropped.append(i)
    dropped = np.array(dropped)
    assert len(dropped) > 2 * n // 5, len(dropped)  # about half of the 8,000 spheres
    assert not np.isin(owner, dropped).any()
    kept = np.setdiff1d(np.arange(n), dropped)
    depth_k, owner_k = _exact(pos, rad, eye, f, kept)
    assert np.array_equal(owner_k, owner)
    assert np.array_equal(depth_k, depth)
