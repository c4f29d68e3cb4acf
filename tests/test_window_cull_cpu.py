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
