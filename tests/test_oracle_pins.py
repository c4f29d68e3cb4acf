"""Pins for the CPU FP64 oracle: closed forms, invariants and independent brute force.

Each test checks the oracle against something other than itself: a value the
geometry fixes in closed form, a textbook formula it does not use, or a
property any correct renderer has.  A dropped term, a sign error or a
transposed operand in the oracle fails at least one of them.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2501_12750_gb300 import scenes


def axis_camera(D, W, H, fovy_deg=60.0, znear=0.05):
    """Eye at (0,0,D) looking down -z: view coordinates equal world coordinates shifted by D."""
    return scenes.Camera(eye=np.array([0, 0, D], np.float32), forward=np.array([0, 0, -1], np.float32),
                         right=np.array([1, 0, 0], np.float32), up=np.array([0, 1, 0], np.float32),
                         tan_half_fovy=float(np.float32(math.tan(math.radians(fovy_deg) / 2))),
                         znear=float(np.float32(znear)), width=W, height=H)


def rays(cam, pix):
    th = np.float64(np.float32(cam.tan_half_fovy))
    W, H = cam.width, cam.height
    a = (2.0 * (pix[:, 0] + 0.5) / W - 1.0) * th * (W / H)
    b = (1.0 - 2.0 * (pix[:, 1] + 0.5) / H) * th
    return np.stack([a, b, -np.ones_like(a)], axis=1)


def view_coords(cam, X):
    d = X.astype(np.float64) - cam.eye.astype(np.float64)
    return np.stack([d @ cam.right.astype(np.float64), d @ cam.up.astype(np.float64),
                     -(d @ cam.forward.astype(np.float64))], axis=-1)


def textbook_sphere(u, C, r):
    """Smaller root of |t u - C|^2 = r^2 by the quadratic formula (fine close to the eye)."""
    uu = (u * u).sum(-1)
    uc = (u * C).sum(-1)
    disc = uc * uc - uu * ((C * C).sum(-1) - r * r)
    t = (uc - np.sqrt(np.maximum(disc, 0.0))) / uu
    return np.where(disc >= 0.0, t, np.inf)


@pytest.mark.parametrize("D,r", [(10.0, 1.2), (120.0, 1.7), (450.0, 1.55), (36000.0, 1.8)])
def test_centre_pixel_depth_and_normal(D, r):
    """On-axis sphere: the centre pixel's depth is D - r and its normal faces the viewer."""
    cam = axis_camera(D, 65, 65)
    xyzr = np.array([[0, 0, 0, r]], np.float32)
    h = oracle.hits(xyzr, cam, np.array([[32, 32]], np.int32))
    assert h.id[0] == 0
    assert abs(h.depth[0] - (D - float(np.float32(r)))) < 1e-9 * D
    np.testing.assert_allclose(h.normal[0], [0, 0, 1], atol=1e-12)


@pytest.mark.parametrize("D", [30.0, 36000.0])
def test_silhouette_lattice_count_on_axis(D):
    """Covered pixel centres of an on-axis sphere are those with a^2 + b^2 < r^2 / (D^2 - r^2)."""
    r = np.float32(1.7)
    W = H = 201
    th = math.tan(math.radians(60) / 2)
    # choose the field of view so the sphere spans ~120 px
    fov = 2 * math.degrees(math.atan(th * (float(r) / math.sqrt(D * D - float(r) ** 2)) / (60 / (W / 2)) / th))
    cam = axis_camera(D, W, H, fovy_deg=fov)
    pix = oracle.all_pixels(W, H)
    u = rays(cam, pix)
    lhs = u[:, 0] ** 2 + u[:, 1] ** 2
    rhs = float(r) ** 2 / (D * D - float(r) ** 2)
    inside = lhs < rhs
    assert np.abs(lhs - rhs).min() > 1e-12 * rhs  # no pixel centre on the boundary
    h = oracle.hits(np.array([[0, 0, 0, r]], np.float32), cam, pix)
    covered = h.id == 0
    assert covered.sum() == inside.sum() > 1000
    assert np.array_equal(covered, inside)


def test_silhouette_cone_off_axis():
    """Off-axis spheres: a pixel is covered iff the angle between its ray and the centre is below asin(r/|C|)."""
    rng = np.random.default_rng(11)
    cam = axis_camera(200.0, 96, 80, fovy_deg=8.0)
    pix = oracle.all_pixels(96, 80)
    u = rays(cam, pix)
    for _ in range(5):
        c = np.array([rng.uniform(-8, 8), rng.uniform(-6, 6), rng.uniform(-20, 20)])
        r = np.float32(rng.uniform(1.5, 3.0))
        xyzr = np.array([[*c, r]], np.float32)
        C = view_coords(cam, xyzr[:, :3])[0]
        cosang = (u @ C) / (np.linalg.norm(u, axis=1) * np.linalg.norm(C))
        cos_lim = math.sqrt(1.0 - float(r) ** 2 / (C @ C))
        inside = cosang > cos_lim
        h = oracle.hits(xyzr, cam, pix)
        amb = (h.flags & oracle.ID_FLAGS) != 0
        assert inside.sum() > 20
        assert np.array_equal((h.id == 0)[~amb], inside[~amb])
        assert amb.sum() <= 1


def test_depth_matches_textbook_quadratic_and_normals():
    """Close to the eye the textbook quadratic is accurate: depths agree, normals are (P - C)/r, unit, facing."""
    s = scenes.random_tiny(3, n=30, width=64, height=48)
    cam = s.cameras[0]
    pix = oracle.all_pixels(64, 48)
    h = oracle.hits(s.xyzr, cam, pix)
    cov = h.id != oracle.NO_ID
    assert cov.sum() > 300
    u = rays(cam, pix)[cov]
    C = view_coords(cam, s.xyzr[h.id[cov], :3])
    r = s.xyzr[h.id[cov], 3].astype(np.float64)
    t = textbook_sphere(u, C, r)
    np.testing.assert_allclose(h.depth[cov], t, rtol=1e-10)
    P = h.depth[cov][:, None] * u
    np.testing.assert_allclose(h.normal[cov], (P - C) / r[:, None], atol=1e-9)
    np.testing.assert_allclose(np.linalg.norm(h.normal[cov], axis=1), 1.0, atol=1e-9)
    assert ((h.normal[cov] * -u).sum(1) >= -1e-12).all()


@pytest.mark.parametrize("seed", range(6))
def test_brute_force_tiny_scenes(seed):
    """Independent numpy brute force (textbook roots, lexicographic (depth, id) minimum) on tiny scenes."""
    s = scenes.random_tiny(100 + seed, n=25, width=40, height=32)
    cam = s.cameras[0]
    pix = oracle.all_pixels(40, 32)
    u = rays(cam, pix)
    C = view_coords(cam, s.xyzr[:, :3])
    r = s.xyzr[:, 3].astype(np.float64)
    t = textbook_sphere(u[:, None, :], C[None, :, :], r[None, :])
    t = np.where(t >= np.float32(cam.znear), t, np.inf)
    best = np.argmin(t, axis=1)
    tb = t[np.arange(len(pix)), best]
    idb = np.where(np.isfinite(tb), best, oracle.NO_ID).astype(np.uint32)
    h = oracle.hits(s.xyzr, cam, pix)
    ok = (h.flags & oracle.ID_FLAGS) == 0
    assert np.array_equal(h.id[ok], idb[ok])
    fin = ok & np.isfinite(tb)
    np.testing.assert_allclose(h.depth[fin], tb[fin], rtol=1e-10)
    assert ok.mean() > 0.99


def test_fully_occluded_sphere_never_visible():
    cam = axis_camera(50.0, 64, 64, fovy_deg=20.0)
    xyzr = np.array([[0, 0, 0, 3.0], [0.2, -0.1, -6.0, 0.8]], np.float32)  # small one in the big one's shadow
    h = oracle.hits(xyzr, cam, oracle.all_pixels(64, 64))
    assert (h.id == 0).sum() > 100
    assert not (h.id == 1).any()


def test_exact_tie_prefers_smaller_id_and_is_flagged():
    cam = axis_camera(30.0, 33, 33, fovy_deg=10.0)
    xyzr = np.array([[0.1, 0.2, 0.0, 1.0], [0.1, 0.2, 0.0, 1.0]], np.float32)
    h = oracle.hits(xyzr[::-1].copy(), cam, oracle.all_pixels(33, 33))
    cov = h.id != oracle.NO_ID
    assert (h.id[cov] == 0).all()
    assert ((h.flags[cov] & oracle.FLAG_TIE) != 0).all()


def test_near_plane_skips_entry_points_in_front_of_it():
    """A sphere cut by the near plane shows only where its entry point is at or beyond the near plane."""
    cam = axis_camera(0.35, 65, 65, fovy_deg=150.0, znear=0.05)
    r = np.float32(0.32)
    xyzr = np.array([[0, 0, 0, r]], np.float32)  # front pole at depth 0.03 < near, silhouette beyond it
    pix = oracle.all_pixels(65, 65)
    h = oracle.hits(xyzr, cam, pix)
    u = rays(cam, pix)
    C = view_coords(cam, xyzr[:, :3])[0]
    t = textbook_sphere(u, C[None, :], float(r))
    expect = np.isfinite(t) & (t >= np.float32(0.05))
    ok = (h.flags & oracle.ID_FLAGS) == 0
    assert h.id[32 * 65 + 32] == oracle.NO_ID
    assert np.array_equal((h.id == 0)[ok], expect[ok])
    assert expect.sum() > 10 and (~expect & np.isfinite(t)).sum() > 50


def test_permutation_relabels_ids_only():
    s = scenes.random_tiny(7, n=40, width=48, height=40)
    cam = s.cameras[0]
    pix = oracle.all_pixels(48, 40)
    perm = np.random.default_rng(0).permutation(40)
    h0 = oracle.hits(s.xyzr, cam, pix)
    h1 = oracle.hits(s.xyzr[perm], cam, pix)
    inv = np.argsort(perm)
    ok = ((h0.flags | h1.flags) & oracle.ID_FLAGS) == 0
    mapped = np.where(h1.id == oracle.NO_ID, oracle.NO_ID, perm[np.minimum(h1.id, 39)])
    assert np.array_equal(mapped[ok], h0.id[ok])
    np.testing.assert_array_equal(h0.depth[ok], h1.depth[ok])
    assert inv.shape == perm.shape


def test_cylinder_axis_along_view_cap_and_cutoff():
    """Bond along the view axis: near cap at depth 10 with normal +z; covered iff lateral offset <= rho_b."""
    W = H = 64  # even: no pixel ray passes exactly through the (zero-radius) atom centres
    cam = axis_camera(0.0, W, H, fovy_deg=4.0)
    xyzr = np.array([[0, 0, -10.0, 1.7], [0, 0, -11.5, 1.5]], np.float32)
    bonds = np.array([[0, 1]], np.uint32)
    pix = oracle.all_pixels(W, H)
    h = oracle.hits(xyzr, cam, pix, bonds=bonds, mode=1, ball_radius=0.0, bond_radius=0.15)
    u = rays(cam, pix)
    lateral = 10.0 * np.hypot(u[:, 0], u[:, 1])
    expect = lateral <= np.float32(0.15)
    ok = (h.flags & oracle.ID_FLAGS) == 0
    assert expect.sum() > 20
    assert np.array_equal((h.id == 2)[ok], expect[ok])
    hit = h.id == 2
    np.testing.assert_allclose(h.depth[hit], 10.0, rtol=1e-12)
    np.testing.assert_allclose(h.normal[hit], np.tile([0, 0, 1.0], (hit.sum(), 1)), atol=1e-12)
    assert (h.side[hit] == 0).all()


def test_cylinder_perpendicular_centre_line_and_colour_split():
    """Bond across the view: the centre pixel sees the side at depth D - rho_b; halves take their atom's colour."""
    W, H = 101, 31
    D = 40.0
    cam = axis_camera(D, W, H, fovy_deg=3.0)
    xyzr = np.array([[-0.75, 0, 0, 1.7], [0.75, 0, 0, 1.5]], np.float32)
    bonds = np.array([[0, 1]], np.uint32)
    pix = oracle.all_pixels(W, H)
    h = oracle.hits(xyzr, cam, pix, bonds=bonds, mode=1, ball_radius=0.0, bond_radius=0.15)
    c = 15 * W + 50
    assert h.id[c] == 2
    assert abs(h.depth[c] - (D - float(np.float32(0.15)))) < 1e-10
    np.testing.assert_allclose(h.normal[c], [0, 0, 1], atol=1e-12)
    hit = (h.id == 2) & ((h.flags & (oracle.ID_FLAGS | oracle.FLAG_SPLIT)) == 0)
    left = pix[:, 0] < 50
    right = pix[:, 0] > 50
    assert (h.side[hit & left] == 0).all() and (h.side[hit & right] == 1).all()
    assert (hit & left).sum() > 10 and (hit & right).sum() > 10
    np.testing.assert_allclose(np.linalg.norm(h.normal[h.id == 2], axis=1), 1.0, atol=1e-9)


def test_shading_closed_form_at_centre_pixel():
    """n = V = (0,0,1) at the front pole: rgb = albedo (ka + kd n.L) + ks (n.H)^32, L = (0.25,0.5,1)/|.|."""
    cam = axis_camera(60.0, 33, 33, fovy_deg=10.0)
    xyzr = np.array([[0, 0, 0, 1.52]], np.float32)
    elem = np.array([1], np.uint8)  # oxygen
    h = oracle.hits(xyzr, cam, np.array([[16, 16]], np.int32))
    rgb = oracle.shade(h, elem, scenes.PALETTE, 1, cam)[0]
    Lz = 1.0 / math.sqrt(0.25 ** 2 + 0.5 ** 2 + 1.0)
    nl = Lz
    hz = (Lz + 1.0) / math.sqrt((0.25 * Lz) ** 2 + (0.5 * Lz) ** 2 + (Lz + 1.0) ** 2)
    expect = np.minimum(scenes.PALETTE[1].astype(np.float64) * (0.2 + 0.7 * nl) + 0.3 * hz ** 32, 1.0)
    np.testing.assert_allclose(rgb, expect, rtol=1e-12)


def test_background_pixels():
    cam = axis_camera(60.0, 16, 16, fovy_deg=10.0)
    xyzr = np.array([[100.0, 0, 0, 1.0]], np.float32)  # off screen
    h = oracle.render_pixels(scenes.Scene("bg", xyzr, np.zeros(1, np.uint8), [cam], ssao=True),
                             0, oracle.all_pixels(16, 16), kernel=scenes.ssao_kernel())
    assert (h.id == oracle.NO_ID).all() and np.isinf(h.depth).all()
    np.testing.assert_array_equal(h.rgb, 1.0)
    np.testing.assert_array_equal(h.ao, 1.0)


def test_ssao_convex_surface_is_unoccluded():
    """A sphere of radius 1e5 A filling the view: samples above a convex surface are never occluded."""
    cam = axis_camera(1e5 + 20.0, 48, 40, fovy_deg=50.0)
    xyzr = np.array([[0, 0, 0, 1e5]], np.float32)
    s = scenes.Scene("wall", xyzr, np.zeros(1, np.uint8), [cam], ssao=True)
    h = oracle.render_pixels(s, 0, oracle.all_pixels(48, 40), kernel=scenes.ssao_kernel())
    assert (h.id == 0).all()
    np.testing.assert_array_equal(h.ao, 1.0)


def test_ssao_front_pole_is_unoccluded():
    """At an on-axis sphere's front pole every hemisphere sample is nearer than anything in the scene."""
    cam = axis_camera(40.0, 65, 65, fovy_deg=12.0)
    xyzr = np.array([[0, 0, 0, 1.7], [1.5, 0.5, -2.0, 1.5], [-1.2, -1.0, -1.5, 1.6]], np.float32)
    s = scenes.Scene("pole", xyzr, np.zeros(3, np.uint8), [cam], ssao=True)
    h = oracle.render_pixels(s, 0, np.array([[32, 32]], np.int32), kernel=scenes.ssao_kernel())
    assert h.id[0] == 0 and h.ao[0] == 1.0


def test_ssao_step_occlusion_closed_form():
    """A wall with a sphere standing in front: one sample direction lands on the blocker.

    The wall point P is the centre pixel of a flat-looking huge sphere (depth 50,
    normal +z, tangent T = -x, B = +y).  Kernel sample k = (-0.5, 0, 0.25) moves
    P by 2 A (0.5 T + 0.25 n) = (+1, 0, +0.5): depth 49.5, 1 A to the right.  A
    blocker sphere of radius 1 centred 1.6 A right at depth 48 covers that pixel
    in front of 49.5 - bias, so the sample is occluded with weight
    min(1, 2/|50 - z_f|) where z_f is the blocker depth there.
    """
    W = H = 101
    cam = axis_camera(0.0, W, H, fovy_deg=8.0)
    wall = 1e4
    xyzr = np.array([[0, 0, -(wall + 50.0), wall], [1.6, 0, -48.0, 1.0]], np.float32)
    s = scenes.Scene("step", xyzr, np.zeros(2, np.uint8), [cam], ssao=True)
    k = np.array([[-0.5, 0.0, 0.25]], np.float32)
    h = oracle.render_pixels(s, 0, np.array([[50, 50]], np.int32), kernel=k)
    assert h.id[0] == 0
    # independent closed form for the fetched pixel
    S = np.array([1.0, 0.0, -49.5])
    f = H / (2 * math.tan(math.radians(8.0) / 2))
    fx = math.floor(W / 2 + f * S[0] / 49.5)
    fy = math.floor(H / 2 - f * S[1] / 49.5)
    uf = rays(cam, np.array([[fx, fy]]))
    zf = textbook_sphere(uf, np.array([[float(np.float32(1.6)), 0.0, -48.0]]), 1.0)[0]
    assert zf <= 49.5 - 0.025
    w = min(1.0, 2.0 / abs(50.0 - zf))
    assert abs(h.ao[0] - (1.0 - w)) < 1e-9


# ------------------------------------------------------------------ soft --

def test_soft_single_sphere_closed_form():
    D, r = 80.0, 1.6
    cam = axis_camera(D, 65, 65, fovy_deg=10.0)
    x = np.array([[0, 0, 0, r]], np.float64)
    f = 65 / (2 * np.float64(np.float32(math.tan(math.radians(5.0)))))
    pix = oracle.all_pixels(65, 65)
    o = oracle.soft_forward(x, cam, pix)
    u = rays(cam, pix)
    C = np.array([0, 0, -D])
    # distance from C to each ray by the sine of the angle (independent of the oracle's projection form)
    cosang = (u @ C) / (np.linalg.norm(u, axis=1) * D)
    rho = D * np.sqrt(np.maximum(1 - cosang ** 2, 0))
    delta = (r - np.sqrt(rho ** 2 + 1e-12)) * f / D
    alpha = np.minimum(0.99, 1 / (1 + np.exp(-delta / 0.5)))
    alpha = np.where(delta >= -4, alpha, 0.0)
    np.testing.assert_allclose(o.A, alpha, atol=1e-9)
    c = 32 * 65 + 32
    eta = 0.05 * r
    g = math.sqrt(r * r + eta * eta) - eta
    assert abs(o.D[c] - 0.99 * (D - g)) < 1e-9
    np.testing.assert_allclose(o.N[c], [0, 0, 0.99 * g / r], atol=1e-12)


def test_soft_two_sphere_composite():
    cam = axis_camera(80.0, 33, 33, fovy_deg=6.0)
    x = np.array([[0.3, 0, -5.0, 1.2], [0, 0, 0, 1.5]], np.float64)  # id 0 is behind id 1
    pix = oracle.all_pixels(33, 33)
    o = oracle.soft_forward(x, cam, pix)
    a0 = oracle.soft_forward(x[:1], cam, pix).A
    a1 = oracle.soft_forward(x[1:], cam, pix).A
    np.testing.assert_allclose(o.A, a1 + (1 - a1) * a0, atol=1e-12)


def test_soft_sharp_limit_is_hard_mask():
    cam = axis_camera(60.0, 64, 64, fovy_deg=8.0)
    x = np.array([[0.2, 0.1, 0, 1.5]], np.float64)
    pix = oracle.all_pixels(64, 64)
    o = oracle.soft_forward(x, cam, pix, sigma=1e-3)
    h = oracle.hits(x.astype(np.float32), cam, pix)
    f = 64 / (2 * np.float64(np.float32(math.tan(math.radians(4.0)))))
    u = rays(cam, pix)
    C = view_coords(cam, x[:, :3].astype(np.float32))[0]
    cosang = (u @ C) / (np.linalg.norm(u, axis=1) * np.linalg.norm(C))
    rho = np.linalg.norm(C) * np.sqrt(1 - cosang ** 2)
    far = np.abs(1.5 - rho) * f / -C[2] > 0.01
    hard = np.where(h.id == 0, 0.99, 0.0)
    np.testing.assert_allclose(o.A[far], hard[far], atol=1e-6)


def test_soft_vjp_matches_central_differences():
    """FP64 central differences (h = 1e-4 A) of sum(gA A + gD D + gN.N) against the analytic VJP."""
    s = scenes.random_tiny(21, n=14, box=8.0, width=28, height=24, distance=25.0)
    cam = s.cameras[0]
    x = s.xyzr.astype(np.float64)
    pix = oracle.all_pixels(28, 24)
    rng = np.random.default_rng(5)
    gA, gD, gN = rng.normal(size=len(pix)), rng.normal(size=len(pix)) * 0.1, rng.normal(size=(len(pix), 3))

    def phi(xx):
        o = oracle.soft_forward(xx, cam, pix)
        return (gA * o.A).sum() + (gD * o.D).sum() + (gN * o.N).sum(), o

    grad = oracle.soft_vjp(x, cam, pix, gA, gD, gN)
    h = 1e-4
    checked = 0
    for i in range(x.shape[0]):
        for k in range(4):
            xp, xm = x.copy(), x.copy()
            xp[i, k] += h
            xm[i, k] -= h
            fp, op = phi(xp)
            fm, om = phi(xm)
            if not (np.array_equal(op.n_used, om.n_used)):
                continue  # a contributor-set or stop change inside the step: not differentiable there
            fd = (fp - fm) / (2 * h)
            assert abs(fd - grad[i, k]) <= 1e-5 * max(1.0, abs(fd)), (i, k, fd, grad[i, k])
            checked += 1
    assert checked >= 40
    assert np.abs(grad).max() > 1e-3


def test_golden_config1_fixture():
    """Regression fixture written by tests/golden/make_golden.py from the oracle alone."""
    import json
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "config1_oracle_pixels.json")
    g = json.load(open(path))
    s = scenes.config1()
    pix = np.array(g["pix"], np.int32)
    h = oracle.render_pixels(s, 0, pix)
    assert h.id.tolist() == g["id"]
    np.testing.assert_allclose(np.where(np.isfinite(h.depth), h.depth, -1.0), g["depth"], rtol=1e-12)
    np.testing.assert_allclose(h.rgb, np.array(g["rgb"]), rtol=1e-12)


# ------------------------------------------------ representations, clipping --

def test_sas_centre_depth_is_distance_minus_radius_plus_probe():
    """Solvent accessible surface: a sphere of r + probe (float32 sum), so the centre depth is D - (r + p)."""
    D, r, p = 50.0, 1.7, 1.4
    cam = axis_camera(D, 65, 65, fovy_deg=20.0)
    xyzr = np.array([[0, 0, 0, r]], np.float32)
    h = oracle.hits(xyzr, cam, np.array([[32, 32]], np.int32), mode=3, probe=p)
    R = float(np.float32(np.float32(r) + np.float32(p)))
    assert h.id[0] == 0 and abs(h.depth[0] - (D - R)) < 1e-10
    # coverage radius on screen grows accordingly: a ray at lateral offset between r and r + p hits
    u = rays(cam, oracle.all_pixels(65, 65))
    lateral = (D - 0.0) * np.hypot(u[:, 0], u[:, 1]) / np.sqrt(1 + u[:, 0] ** 2 + u[:, 1] ** 2)
    hall = oracle.hits(xyzr, cam, oracle.all_pixels(65, 65), mode=3, probe=p)
    ok = (hall.flags & oracle.ID_FLAGS) == 0
    assert np.array_equal((hall.id == 0)[ok], (lateral <= R)[ok])


def test_sticks_spheres_take_the_bond_radius():
    """Sticks: atoms are drawn with the bond radius, so the centre pixel sees depth D - rho_b; bonds stay."""
    D = 40.0
    cam = axis_camera(D, 101, 31, fovy_deg=3.0)
    xyzr = np.array([[-0.75, 0, 0, 1.7], [0.75, 0, 0, 1.5]], np.float32)
    bonds = np.array([[0, 1]], np.uint32)
    pix = oracle.all_pixels(101, 31)
    h = oracle.hits(xyzr, cam, pix, bonds=bonds, mode=2, bond_radius=0.15)
    rb = float(np.float32(0.15))
    # the pixel through atom 0's centre: ray (a, b) with a = -0.75 / D at column (a / (th * W/H) + 1) * W / 2 - 0.5
    th = np.float64(np.float32(cam.tan_half_fovy))
    col = ((-0.75 / D) / (th * 101 / 31) + 1.0) * 101 / 2 - 0.5
    k = 15 * 101 + int(round(col))
    assert h.id[k] in (0, 2)  # the sphere and the bond's cap region meet at the centre line
    assert abs(h.depth[k] - (D - rb)) < 2e-3  # off-centre by under half a pixel (< 1e-3 A laterally)
    assert set(np.unique(h.id[h.id != oracle.NO_ID]).tolist()) == {0, 1, 2}
    # no hit lies further than rho_b from the segment joining the centres
    t = h.depth[h.id != oracle.NO_ID]
    u = rays(cam, pix)[h.id != oracle.NO_ID]
    P = u * t[:, None]
    P[:, 2] += D
    x = np.clip(P[:, 0], -0.75, 0.75)
    dist = np.sqrt((P[:, 0] - x) ** 2 + P[:, 1] ** 2 + P[:, 2] ** 2)
    assert dist.max() < rb + 1e-9


def test_clip_plane_equals_removing_the_clipped_atoms():
    """Clipping n.X + d >= 0 renders exactly like the scene without the other atoms (ids mapped back)."""
    s = scenes.random_tiny(31, n=60, width=48, height=40)
    cam = s.cameras[0]
    plane = np.array([0.6, -0.8, 0.0, -1.3], np.float32)
    pix = oracle.all_pixels(48, 40)
    h = oracle.hits(s.xyzr, cam, pix, clip=plane)
    keep = s.xyzr[:, :3].astype(np.float64) @ plane[:3].astype(np.float64) + plane[3] >= 0
    assert 10 < keep.sum() < 50
    idx = np.nonzero(keep)[0]
    h2 = oracle.hits(s.xyzr[keep], cam, pix)
    m = h2.id != oracle.NO_ID
    mapped = h2.id.copy()
    mapped[m] = idx[h2.id[m]]
    assert np.array_equal(mapped, h.id)
    np.testing.assert_array_equal(h.depth, h2.depth)
    # a zero normal keeps everything
    h3 = oracle.hits(s.xyzr, cam, pix, clip=np.zeros(4, np.float32))
    h4 = oracle.hits(s.xyzr, cam, pix)
    assert np.array_equal(h3.id, h4.id)


def test_clip_plane_drops_a_bond_with_one_atom_clipped():
    cam = axis_camera(40.0, 101, 31, fovy_deg=3.0)
    xyzr = np.array([[-0.75, 0, 0, 1.7], [0.75, 0, 0, 1.5]], np.float32)
    bonds = np.array([[0, 1]], np.uint32)
    pix = oracle.all_pixels(101, 31)
    h = oracle.hits(xyzr, cam, pix, bonds=bonds, mode=1, ball_radius=0.4, clip=np.array([-1, 0, 0, 0], np.float32))
    assert set(np.unique(h.id).tolist()) == {0, oracle.NO_ID}


# ------------------------------------------------------ shading variants --

def test_flat_shading_is_the_albedo_and_matte_is_blinn_phong_without_specular():
    s = scenes.random_tiny(5, n=40, width=40, height=32)
    cam = s.cameras[0]
    h = oracle.hits(s.xyzr, cam, oracle.all_pixels(40, 32))
    cov = h.id != oracle.NO_ID
    flat = oracle.shade(h, s.elem, s.palette, 40, cam, model=1)
    np.testing.assert_array_equal(flat[cov], s.palette[s.elem[h.id[cov]]].astype(np.float64))
    matte = oracle.shade(h, s.elem, s.palette, 40, cam, model=2)
    glossy0 = oracle.shade(h, s.elem, s.palette, 40, cam, model=0, ks=0.0)
    np.testing.assert_allclose(matte[cov], glossy0[cov], rtol=0, atol=1e-15)


@pytest.mark.parametrize("levels", [2, 4, 7, 16])
def test_toon_bands_are_monotone_steps_within_one_band_of_matte(levels):
    """Toon takes at most `levels` values per albedo, is non-decreasing in n.L, and differs from matte by <= kd/(L-1)."""
    cam = axis_camera(30.0, 81, 81, fovy_deg=12.0)
    xyzr = np.array([[0, 0, 0, 2.5]], np.float32)
    elem = np.array([2], np.uint8)
    h = oracle.hits(xyzr, cam, oracle.all_pixels(81, 81))
    cov = h.id == 0
    toon = oracle.shade(h, elem, scenes.PALETTE, 1, cam, model=3, toon_levels=levels)[cov]
    matte = oracle.shade(h, elem, scenes.PALETTE, 1, cam, model=2)[cov]
    alb = scenes.PALETTE[2].astype(np.float64)
    assert len(np.unique(np.round(toon[:, 0], 12))) <= levels
    assert len(np.unique(np.round(toon[:, 0], 12))) >= min(levels, 2)
    assert np.all(np.abs(toon - matte) <= 0.7 * alb / (levels - 1) + 1e-12)
    order = np.argsort(matte[:, 0], kind="stable")
    assert np.all(np.diff(toon[order, 0]) >= -1e-15)
    # the brightest band is ka + kd (n.L = 1 reachable: the light direction lies inside the visible cap)
    assert abs(toon[:, 0].max() - min(alb[0] * 0.9, 1.0)) < 1e-12


def test_fog_limits_and_linear_ramp():
    """Fog: no change before fog_near, the background from fog_far on (density 1), linear in between."""
    cam = axis_camera(0.0, 3, 1, fovy_deg=1.0)
    pix = np.array([[1, 0]], np.int32)
    bg = (1.0, 1.0, 1.0)
    base = None
    for z, expect_w in [(10.0, 0.0), (25.0, 0.25), (40.0, 0.625), (60.0, 1.0)]:
        xyzr = np.array([[0, 0, -z - 1.0, 1.0]], np.float32)
        s = scenes.Scene("fog", xyzr, np.array([3], np.uint8), [cam], ssao=False)
        plain = oracle.render_pixels(s, 0, pix)
        fogged = oracle.render_pixels(s, 0, pix, fog_near=15.0, fog_far=55.0, fog_density=1.0)
        assert abs(plain.depth[0] - z) < 1e-9
        expect = plain.rgb_final + expect_w * (np.array(bg) - plain.rgb_final)
        np.testing.assert_allclose(fogged.rgb_final, expect, atol=1e-12)
        base = plain
    assert base is not None


def test_outline_marks_exactly_the_covered_pixels_next_to_background_or_a_deep_step():
    """Brute force over the full depth image: outline where a 4-neighbour is background or deeper than the threshold."""
    s = scenes.random_tiny(12, n=30, width=40, height=34)
    cam = s.cameras[0]
    pix = oracle.all_pixels(40, 34)
    full = oracle.hits(s.xyzr, cam, pix)
    Z = full.depth.reshape(34, 40)
    step = 1.5
    col = (1.0, 0.0, 0.5)
    pad = np.pad(Z, 1, constant_values=np.nan)
    edge = np.zeros_like(Z, bool)
    for dy, dx in [(0, -1), (0, 1), (-1, 0), (1, 0)]:
        nb = pad[1 + dy:35 + dy, 1 + dx:41 + dx]
        with np.errstate(invalid="ignore"):
            edge |= np.isinf(nb) | (np.nan_to_num(nb - Z, nan=-1.0, posinf=np.inf) > step)
    edge &= np.isfinite(Z)
    assert edge.sum() > 30 and (np.isfinite(Z) & ~edge).sum() > 30
    # a sparse subset of pixels: their neighbours are ray-cast on demand
    rng = np.random.default_rng(2)
    sub = pix[rng.choice(len(pix), 400, replace=False)]
    h = oracle.render_pixels(s, 0, sub, outline_depth=step, outline_color=col)
    e = edge[sub[:, 1], sub[:, 0]]
    ok = (h.flags & (oracle.FLAG_EDGE | oracle.FLAG_FETCH | oracle.ID_FLAGS)) == 0
    got = np.all(np.abs(h.rgb_final - np.array(col)) < 1e-15, axis=1)
    assert np.array_equal(got[ok & (h.id != oracle.NO_ID)], e[ok & (h.id != oracle.NO_ID)])
    np.testing.assert_array_equal(h.rgb_final[h.id == oracle.NO_ID], 1.0)


# ----------------------------------------------- oblique capped cylinders --

def line_sphere_t(E, d, C, r):
    """Entry parameter of E + t d into spheres (C, r) by the textbook quadratic."""
    w = E[None, None, :] - C[None, :, :]
    a = (d * d).sum(-1)[:, None]
    b = (d[:, None, :] * w).sum(-1)
    c = (w * w).sum(-1) - r[None, :] ** 2
    disc = b * b - a * c
    t = (-b - np.sqrt(np.maximum(disc, 0.0))) / a
    return np.where(disc >= 0.0, t, np.inf)


def line_capped_cylinder(E, d, Pi, Pj, rho):
    """Nearest hit of E + t d on capped cylinders Pi -> Pj of radius rho (any orthonormal frame).

    The lateral surface is the textbook quadratic |(X - Pi) - ((X - Pi).A) A|^2 = rho^2 restricted to axial
    coordinates in [0, L]; each cap is the plane through its end point with normal A, restricted to radial
    distance <= rho.  Returns (t, kind, axial): kind 1 side, 2 the cap at Pj, 3 the cap at Pi.
    """
    Av = Pj - Pi
    L = np.linalg.norm(Av, axis=1)
    A = Av / L[:, None]
    w0 = E[None, :] - Pi                                    # (B, 3)
    dA = d @ A.T                                            # (P, B)
    w0A = (w0 * A).sum(-1)[None, :]
    dd = (d * d).sum(-1)[:, None]
    dw = d @ w0.T
    ww = (w0 * w0).sum(-1)[None, :]
    qa = dd - dA * dA
    qb = dw - dA * w0A
    qc = ww - w0A * w0A - rho * rho
    disc = qb * qb - qa * qc
    with np.errstate(invalid="ignore", divide="ignore"):
        ts = (-qb - np.sqrt(np.maximum(disc, 0.0))) / qa
    ax = w0A + ts * dA
    side_ok = (disc >= 0.0) & (qa > 0.0) & (ax >= 0.0) & (ax <= L[None, :])
    best = np.where(side_ok, ts, np.inf)
    kind = np.where(side_ok, 1, 0)
    for s_end, k_end in ((L[None, :], 2), (0.0, 3)):
        with np.errstate(invalid="ignore", divide="ignore"):
            tc = (s_end - w0A) / dA
        # radial distance of the cap-plane point from the axis
        X = w0[None, :, :] + tc[:, :, None] * d[:, None, :]   # X - Pi
        rad2 = (X * X).sum(-1) - (w0A + tc * dA) ** 2
        ok = (np.abs(dA) > 1e-12) & np.isfinite(tc) & (rad2 <= rho * rho) & (tc < best)
        best = np.where(ok, tc, best)
        kind = np.where(ok, k_end, kind)
    axial = w0A + best * dA
    return best, kind, axial


def oblique_bond_scene(seed, n=24, box=5.0, W=96, H=80, distance=10.0, fovy=25.0):
    rng = np.random.default_rng(seed)
    pos = rng.uniform(0.0, box, (n, 3))
    elem = scenes.draw_elements(rng, n)
    xyzr = scenes.pack_xyzr(pos, elem)
    bonds = scenes.bonds_within(xyzr[:, :3])
    c = np.full(3, box / 2)
    cam = scenes.orbit_camera(c, distance, rng.uniform(0, 360), rng.uniform(-70, 70), W, H)
    cam = scenes.Camera(cam.eye, cam.forward, cam.right, cam.up,
                        float(np.float32(math.tan(math.radians(fovy) / 2))), cam.znear, W, H)
    return xyzr, bonds, cam


@pytest.mark.parametrize("seed,mode,ball", [(0, 1, 0.0), (1, 1, 0.0), (2, 1, 0.4), (3, 2, 0.0), (4, 1, 0.0),
                                            (5, 2, 0.0)])
def test_oblique_capped_cylinders_match_world_space_brute_force(seed, mode, ball):
    """Bonds at every angle to the view, where a cap and the side compete at the rim: the oracle's nearest
    primitive, depth, normal and half-bond side equal an independent brute force: rays from the eye,
    endpoint-relative textbook side quadratic and cap planes through the end points (the oracle works
    relative to the bond midpoint with the ray split along and across the axis).  Both use view coordinates
    with the float32 basis as passed, which is how the oracle defines them.

    mode 1 is ball-and-stick (ball radius 0 leaves the caps of free-standing cylinders visible), mode 2 is
    sticks (spheres of the bond radius at every atom)."""
    xyzr, bonds, cam = oblique_bond_scene(seed)
    assert len(bonds) >= 10
    rho = float(np.float32(0.15))
    pix = oracle.all_pixels(cam.width, cam.height)
    E = np.zeros(3)
    d = rays(cam, pix)
    X = view_coords(cam, xyzr[:, :3])
    r_sph = np.full(len(X), float(np.float32(ball if mode == 1 else 0.15)))
    ts = line_sphere_t(E, d, X, r_sph)
    tb, kind, axial = line_capped_cylinder(E, d, X[bonds[:, 0]], X[bonds[:, 1]], rho)
    zn = float(np.float32(cam.znear))
    t_all = np.concatenate([ts, tb], axis=1)
    t_all = np.where(t_all >= zn, t_all, np.inf)
    best = np.argmin(t_all, axis=1)                       # first minimum: the smaller id on exact ties
    tmin = t_all[np.arange(len(pix)), best]
    ref_id = np.where(np.isfinite(tmin), best, oracle.NO_ID).astype(np.uint32)
    h = oracle.hits(xyzr, cam, pix, bonds=bonds, mode=mode, ball_radius=ball, bond_radius=0.15)
    ok = (h.flags & oracle.ID_FLAGS) == 0
    assert ok.mean() > 0.995
    assert np.array_equal(h.id[ok], ref_id[ok])
    n_at = len(xyzr)
    on_bond = ok & (ref_id != oracle.NO_ID) & (ref_id >= n_at)
    b = ref_id[on_bond].astype(np.int64) - n_at
    rows = np.nonzero(on_bond)[0]
    k = kind[rows, b]
    assert (k == 1).sum() > 30
    if mode == 1 and ball == 0.0:
        assert (k >= 2).sum() > 10  # caps seen obliquely
    np.testing.assert_allclose(h.depth[on_bond], tmin[on_bond], rtol=1e-10)
    # normals: radial unit vector on the side, +/- axis on the caps
    Pi, Pj = X[bonds[b, 0]], X[bonds[b, 1]]
    A = (Pj - Pi) / np.linalg.norm(Pj - Pi, axis=1)[:, None]
    q = tmin[on_bond][:, None] * d[on_bond] - Pi
    radial = q - (q * A).sum(1)[:, None] * A
    n_ref = np.where((k == 1)[:, None], radial / rho, np.where((k == 2)[:, None], A, -A))
    np.testing.assert_allclose(h.normal[on_bond], n_ref, atol=1e-8)
    # the half-bond colour: atom i's half when the axial coordinate is at most half the length
    L = np.linalg.norm(Pj - Pi, axis=1)
    split_ok = (h.flags[on_bond] & oracle.FLAG_SPLIT) == 0
    side_ref = np.where(axial[rows, b] <= 0.5 * L, 0, 1)
    assert np.array_equal(h.side[on_bond][split_ok], side_ref[split_ok])


def test_ssao_tangent_frame_branch_for_normals_along_screen_up():
    """|n_y| > 0.9 takes the tangent a = (1, 0, 0): T = n x a / |n x a| = (0, n_z, -n_y), so kernel sample
    (0.5, 0, 0.25) moves the hit 2 A (0.5 T + 0.25 n) up the screen and deeper.  A blocker placed there
    occludes it; under the other tangent rule the sample lands 1 A to the left, on the unoccluded floor.

    The floor is a sphere of radius 1e4 A whose surface at the centre pixel (depth 50) has normal
    (0, 0.95, 0.3122); the blocker is a 0.5 A sphere centred 0.787 A above the centre ray at depth 49.8."""
    W = H = 101
    cam = axis_camera(0.0, W, H, fovy_deg=8.0)
    R = 1e4
    ny = 0.95
    nz = math.sqrt(1.0 - ny * ny)
    C = np.array([0.0, -ny * R, -50.0 - nz * R])
    xyzr = np.array([[C[0], C[1], C[2], R], [0.0, 0.78725, -49.8, 0.5]], np.float32)
    s = scenes.Scene("branch", xyzr, np.zeros(2, np.uint8), [cam], ssao=True)
    k = np.array([[0.5, 0.0, 0.25]], np.float32)
    h = oracle.render_pixels(s, 0, np.array([[50, 50]], np.int32), kernel=k)
    assert h.id[0] == 0
    # independent closed form: hit point and normal from the textbook quadratic on the float32 floor
    u = rays(cam, np.array([[50, 50]]))[0]
    Cf = view_coords(cam, xyzr[:1, :3])[0]
    t = textbook_sphere(u[None, :], Cf[None, :], float(np.float32(R)))[0]
    P = t * u
    n = (P - Cf) / float(np.float32(R))
    assert abs(n[0]) < 1e-12 and n[1] > 0.9
    T = np.array([0.0, n[2], -n[1]]) / math.hypot(n[1], n[2])
    S = P + 2.0 * (0.5 * T + 0.25 * n)
    f = H / (2 * float(np.float32(math.tan(math.radians(8.0) / 2))))
    fx = math.floor(W / 2 + f * S[0] / -S[2])
    fy = math.floor(H / 2 - f * S[1] / -S[2])
    assert fy < 50  # up the screen
    uf = rays(cam, np.array([[fx, fy]]))
    Cb = view_coords(cam, xyzr[1:, :3])
    zf = textbook_sphere(uf, Cb, float(np.float32(0.5)))[0]
    assert np.isfinite(zf) and zf <= -S[2] - 0.025
    w = min(1.0, 2.0 / abs(t - zf))
    assert w > 0.5
    assert abs(h.ao[0] - (1.0 - w)) < 1e-9
