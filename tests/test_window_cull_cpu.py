"""The per-warp window cull of the tile walks (hard raster and soft renderer), checked in FP64.

With the reference point at the sphere's centre (dz = 0) the offset of a pixel ray's point at the reference
depth is o = k (du, -dv, 0), (du, dv) the pixel offset from the projected centre, and the centre's distance to
the ray (direction u = (a, b, 1)) is rho with rho^2 = |o|^2 - (o.u)^2 / |u|^2.  The walks drop an entry for a
rectangle of pixels when every pixel's distance d to the projected centre exceeds R |u|_max / k, relying on
rho >= |o| / |u| (so such an entry can neither be hit, R = bounding radius, nor reach the soft cutoff,
R^2 = rej2).  Random rectangles, centres and focal lengths: whenever the cull fires, every pixel of the
rectangle has rho > R.
"""
import numpy as np


def test_rho_lower_bound_and_cull_soundness():
    rng = np.random.default_rng(11)
    fired = 0
    for _ in range(400):
        W = H = 512
        f = rng.uniform(200.0, 2000.0)                 # pixels per unit slope
        cx, cy = W / 2.0, H / 2.0
        x0, y0 = rng.integers(0, W - 16), rng.integers(0, H - 2)
        px = x0 + np.arange(16) + 0.5
        py = y0 + np.arange(2) + 0.5
        PX, PY = np.meshgrid(px, py)
        a = (PX - cx) / f
        b = (cy - PY) / f
        uu = a * a + b * b + 1.0
        u0 = rng.uniform(-50.0, W + 50.0)
        v0 = rng.uniform(-50.0, H + 50.0)
        k = rng.uniform(0.01, 2.0)                       # A per pixel at the reference depth
        R = rng.uniform(0.2, 8.0)
        ox, oy = k * (PX - u0), -k * (PY - v0)
        ou = ox * a + oy * b
        rho2 = ox * ox + oy * oy - ou * ou / uu
        assert (rho2 >= (ox * ox + oy * oy) / uu * (1 - 1e-12) - 1e-12).all()
        # the rectangle test of the kernels: distance from the projected centre to the pixel-centre rectangle
        dx = max(px[0] - u0, u0 - px[-1], 0.0)
        dy = max(py[0] - v0, v0 - py[-1], 0.0)
        if np.hypot(dx, dy) > R * np.sqrt(uu.max()) / k:
            fired += 1
            assert (np.sqrt(rho2) > R).all()
    assert fired > 100


def test_entry_pixel_box_keeps_every_reachable_pixel():
    """The raster's per-entry pixel box: tile pixels whose centres lie within the reach rt of the projected
    centre along x and along y, rt = R |u|_max / k widened by 0.1 % + 0.01 px + 2e-7 of the coordinates, with
    |u|_max from the tile's extreme columns and rows.  Computed here with the kernel's FP32 roundings; every
    tile pixel whose ray passes within R of the sphere centre (FP64) must be inside the box."""
    rng = np.random.default_rng(12)
    f32 = np.float32
    checked = 0
    for _ in range(6000):
        W, H = 1920, 1080
        f = rng.uniform(200.0, 3000.0)
        cx, cy = f32(W / 2.0), f32(H / 2.0)
        inv_f = f32(1.0 / f)
        TW, TH = [(16, 16), (32, 8), (8, 8)][rng.integers(3)]
        tx0 = int(rng.integers(0, W // TW)) * TW
        ty0 = int(rng.integers(0, H // TH)) * TH
        u0 = rng.uniform(tx0 - 40.0, tx0 + TW + 40.0)
        v0 = rng.uniform(ty0 - 40.0, ty0 + TH + 40.0)
        k = rng.uniform(0.005, 2.0)
        R = rng.uniform(0.1, 6.0)
        # tile |u|^2 bound as the kernel forms it
        a = [abs(f32(f32(f32(x) + f32(0.5)) - cx) * inv_f) for x in (tx0, tx0 + TW - 1)]
        b = [abs(f32(cy - f32(f32(y) + f32(0.5))) * inv_f) for y in (ty0, ty0 + TH - 1)]
        am, bm = max(a), max(b)
        uu = f32(am * am + f32(bm * bm + f32(1.0)))
        cu, cv = f32(u0), f32(v0)
        rt = f32(f32(f32(R) * uu / np.sqrt(uu) / f32(k)) * f32(1.001) + f32(0.01) + f32(2e-7) * (abs(cu) + abs(cv)))
        lo_x = max(np.ceil(f32(cu - rt - f32(0.5))) - tx0, 0.0)
        hi_x = min(np.floor(f32(cu + rt - f32(0.5))) - tx0, TW - 1.0)
        lo_y = max(np.ceil(f32(cv - rt - f32(0.5))) - ty0, 0.0)
        hi_y = min(np.floor(f32(cv + rt - f32(0.5))) - ty0, TH - 1.0)
        # FP64 truth: the sphere centre's distance to each pixel ray of the tile
        lx, ly = np.meshgrid(np.arange(TW), np.arange(TH))
        PX, PY = tx0 + lx + 0.5, ty0 + ly + 0.5
        ra, rb = (PX - W / 2.0) / f, (H / 2.0 - PY) / f
        ruu = ra * ra + rb * rb + 1.0
        ox, oy = k * (PX - u0), -k * (PY - v0)
        ou = ox * ra + oy * rb
        rho2 = ox * ox + oy * oy - ou * ou / ruu
        reach = rho2 <= R * R
        if reach.any():
            checked += 1
            inside = (lx >= lo_x) & (lx <= hi_x) & (ly >= lo_y) & (ly <= hi_y)
            assert inside[reach].all()
    assert checked > 500
