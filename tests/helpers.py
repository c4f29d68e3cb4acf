"""Shared helpers for the GPU parity tests: run the CUDA path, run the oracle, compare.

Tolerances (per pixel, FP32 values, never 8-bit quantised):
  id      bit-exact, except pixels the oracle flags as ambiguous (two nearest
          depths within 1e-4 A, a silhouette / rim / near-plane decision within
          1e-6 A);
  depth   |d_gpu - d_ref| / d_ref <= 1e-5, plus the FP32 conditioning term near
          silhouettes (hit_tolerances);
  normal  max abs per component <= 1e-4, plus the same conditioning term;
  rgb     <= 1/255 per channel (no SSAO), final rgb and AO <= 2/255 with SSAO
          (excluded: pixels with an SSAO sample or occlusion test within the
          FP32 error bound of a renderer's sample position of a pixel-grid line
          or of its threshold, a fetch of a pixel whose visible surface is in
          doubt; see oracle.ssao).
Depth, normal and colour are compared where the ids match and nothing is flagged.
"""
from __future__ import annotations

import math

import numpy as np

import oracle

DEPTH_RTOL = 1e-5
NORMAL_ATOL = 1e-4
# Near a silhouette an FP32 hit is ill-conditioned: its depth and normal errors grow as 1/sqrt(sil),
# sil = (R^2 - rho^2)/(2 R^2) (measured on the GPU planes: normal error <= 1e-7 (1 + 1/sqrt(sil))).  The
# tolerances add that term with a factor of 4 to 5; away from silhouettes the plain bounds above dominate
# (at depths of tens of Angstrom or more, except within sil ~ 1e-7 of a silhouette).
DEPTH_COND = 5e-7   # A per A of radius
NORMAL_COND = 4e-7
RGB_ATOL = 1.0 / 255.0
AO_ATOL = 2.0 / 255.0
SSAO_FLAGS = oracle.FLAG_GRID | oracle.FLAG_MARGIN | oracle.FLAG_FETCH | oracle.FLAG_SILH


def gpu_render(scene, cam_index=0, ssao=None, mode=None, tile=(16, 16), splat_max=16, bonds=True, renderer=None,
               **settings):
    """Render a scene view through the C ABI; returns numpy planes.  Extra keywords go to the settings."""
    import torch

    import paper_2501_12750_gb300 as vtx
    r = renderer or vtx.Renderer()
    dev = torch.device("cuda")
    xyzr = torch.from_numpy(np.ascontiguousarray(scene.xyzr)).to(dev)
    elem = torch.from_numpy(np.ascontiguousarray(scene.elem)).to(dev)
    r.upload_atoms(xyzr, elem, scene.palette)
    m = scene.mode if mode is None else mode
    if m in (1, 2) and bonds and scene.bonds is not None and len(scene.bonds):
        r.upload_bonds(torch.from_numpy(scene.bonds.astype(np.int32)).to(dev))
    cam = scene.cameras[cam_index]
    r.set_camera(cam)
    s = vtx.default_settings(ssao_kernel=ssao, mode=m, tile_w=tile[0], tile_h=tile[1], splat_max_px=splat_max,
                             flags=vtx.FLAG_SYNC, **settings)
    out = r.render_frame(s, width=cam.width, height=cam.height)
    torch.cuda.synchronize()
    res = {k: v.cpu().numpy() for k, v in out.items()}
    res["id"] = res["id"].view(np.uint32)
    return res


def hit_tolerances(h):
    """Per-pixel depth (A) and normal tolerances of the oracle hits h (see DEPTH_COND)."""
    amp = 1.0 + 1.0 / np.sqrt(np.maximum(h.sil, 1e-30))
    rad = h.rad if h.rad is not None else np.zeros_like(h.depth)
    return DEPTH_RTOL * h.depth + DEPTH_COND * rad * amp, NORMAL_ATOL + NORMAL_COND * amp


def gather(res, pix):
    """GPU planes at the listed (px, py) pixels."""
    px, py = pix[:, 0], pix[:, 1]
    return dict(depth=res["depth"][py, px], id=res["id"][py, px], normal=res["normal"][:, py, px].T,
                rgb=res["rgb"][:, py, px].T, ao=res["ao"][py, px])


FLAG_NAMES = [("tie", oracle.FLAG_TIE), ("graze", oracle.FLAG_GRAZE), ("near", oracle.FLAG_NEAR),
              ("split", oracle.FLAG_SPLIT), ("grid", oracle.FLAG_GRID), ("margin", oracle.FLAG_MARGIN),
              ("fetch", oracle.FLAG_FETCH), ("silh", oracle.FLAG_SILH), ("band", oracle.FLAG_BAND),
              ("edge", oracle.FLAG_EDGE)]
EXCLUSION_LOG = []  # (label, covered, excluded, {flag: count}) of every comparison in this process


def compare(res, h, ssao: bool, allow_excluded=0.001, label="", colour=True):
    """Assert parity of GPU planes `res` with oracle hits `h`; returns a stats dict.

    colour=False checks ids, depths and normals only (oracle hits computed without shading).
    The fraction of covered pixels left out of the comparison (the oracle's ambiguity flags) is printed,
    returned per flag, logged in EXCLUSION_LOG and must not exceed allow_excluded (default 0.1 %).
    """
    g = gather(res, h.pix)
    amb = (h.flags & oracle.ID_FLAGS) != 0
    covered = h.id != oracle.NO_ID
    n = len(h.id)
    bad_id = (~amb) & (g["id"] != h.id)
    assert not bad_id.any(), "%s: %d id mismatches of %d pixels (first at %s: gpu %s oracle %s)" % (
        label, bad_id.sum(), n, h.pix[bad_id][:3].tolist(), g["id"][bad_id][:3], h.id[bad_id][:3])
    ok = (~amb) & covered
    if ok.any():
        dtol, ntol = hit_tolerances(h)
        derr = np.abs(g["depth"][ok].astype(np.float64) - h.depth[ok])
        rel = derr / h.depth[ok]
        assert (derr <= dtol[ok]).all(), "%s: depth err %.3g (rel %.3g)" % (label, (derr - dtol[ok]).max(), rel.max())
        nd = np.abs(g["normal"][ok].astype(np.float64) - h.normal[ok]).max(1)
        assert (nd <= ntol[ok]).all(), "%s: normal err %.3g" % (label, nd.max())
        nerr = nd.max()
    else:
        rel, nerr = np.zeros(1), 0.0
    bg = (~amb) & (~covered)
    assert np.isinf(g["depth"][bg]).all() and (g["normal"][bg] == 0).all()
    rgb_ok = (~amb) & ((h.flags & (oracle.FLAG_SPLIT | oracle.FLAG_BAND | oracle.FLAG_EDGE)) == 0)
    aoerr, cerr = 0.0, 0.0
    if colour:
        if ssao:
            rgb_ok &= (h.flags & SSAO_FLAGS) == 0
            aoerr = np.abs(g["ao"][rgb_ok] - h.ao[rgb_ok]).max() if rgb_ok.any() else 0.0
            assert aoerr <= AO_ATOL, "%s: ao err %.3g" % (label, aoerr)
            ref = h.rgb_final
            tol = AO_ATOL
        else:
            ref = h.rgb_final if h.rgb_final is not None else h.rgb
            tol = RGB_ATOL
            if h.rgb_final is not None and (h.flags & oracle.FLAG_FETCH).any():
                rgb_ok &= (h.flags & oracle.FLAG_FETCH) == 0  # outline next to an id-ambiguous neighbour
        cerr = np.abs(g["rgb"][rgb_ok] - ref[rgb_ok]).max() if rgb_ok.any() else 0.0
        assert cerr <= tol, "%s: rgb err %.3g" % (label, cerr)
        excl = amb | (~rgb_ok)
    else:
        excl = amb
    n_cov = int(covered.sum())
    n_exc = int(excl[covered].sum())
    frac = n_exc / n_cov if n_cov else 0.0
    by_flag = {name: int(((h.flags & bit) != 0)[covered].sum()) for name, bit in FLAG_NAMES}
    by_flag = {k: v for k, v in by_flag.items() if v}
    EXCLUSION_LOG.append((label, n_cov, n_exc, by_flag))
    print("EXCLUDED %-28s %7d covered %5d excluded (%.4f%%) %s" % (label, n_cov, n_exc, 100 * frac, by_flag))
    assert frac <= allow_excluded, "%s: %.3f%% of covered pixels excluded %s" % (label, 100 * frac, by_flag)
    return dict(pixels=n, covered=n_cov, excluded=n_exc, excluded_frac=frac, excluded_by_flag=by_flag,
                depth_rel=float(rel.max()), normal=float(nerr), rgb=float(cerr), ao=float(aoerr))


def sample_pixels(width, height, n, seed, windows=(), covered_mask=None):
    """n random pixels (half from covered_mask when given) plus full square windows (x, y, size)."""
    rng = np.random.default_rng(seed)
    pts = [np.stack([rng.integers(0, width, n), rng.integers(0, height, n)], 1)]
    if covered_mask is not None:
        ys, xs = np.nonzero(covered_mask)
        if len(xs):
            k = rng.integers(0, len(xs), n)
            pts.append(np.stack([xs[k], ys[k]], 1))
    for (x0, y0, s) in windows:
        yy, xx = np.mgrid[y0:min(y0 + s, height), x0:min(x0 + s, width)]
        pts.append(np.stack([xx.ravel(), yy.ravel()], 1))
    pix = np.unique(np.concatenate(pts).astype(np.int32), axis=0)
    return np.ascontiguousarray(pix)


def soft_candidates(xyzr64, cam, px_lo, px_hi, near=None):
    """Indices (ascending) of the atoms that can contribute to any pixel of the box [px_lo, px_hi] (inclusive
    (x, y) pixel indices) of a soft-edge render, by a provable bound.

    The oracle brute-forces every atom at every pixel; only atoms within -4 px of their silhouette contribute.
    For a pixel ray u = (a, b, -1) and a centre at depth z_c whose projection has slope s, the centre-to-ray
    distance is rho = |C x u| / |u| >= z_c |s - (a, b)| / |u| = z_c d / (f |u|), d the pixel distance from the
    projected centre.  delta = (r - rho) f / z_c >= -4 then needs d <= |u| (r f / z_c + 4).  Passing the oracle
    only these atoms, in their original order, changes neither its outputs nor its flags (an excluded atom
    has delta < -4 by more than a pixel)."""
    x = np.asarray(xyzr64, np.float64)
    E = cam.eye.astype(np.float64)
    Rv, Uv, Fv = (cam.right.astype(np.float64), cam.up.astype(np.float64), cam.forward.astype(np.float64))
    d = x[:, :3] - E
    zc = d @ Fv
    W, H = cam.width, cam.height
    f = H / (2.0 * float(np.float32(cam.tan_half_fovy)))
    zn = float(np.float32(cam.znear)) if near is None else near
    ok = zc > zn
    zs = np.where(ok, zc, 1.0)
    cx = W / 2.0 + f * (d @ Rv) / zs
    cy = H / 2.0 - f * (d @ Uv) / zs
    # |u| over the box: the largest slope magnitude of its corners
    ax = np.abs((np.array([px_lo[0], px_hi[0] + 1.0]) - W / 2.0) / f).max()
    ay = np.abs((np.array([px_lo[1], px_hi[1] + 1.0]) - H / 2.0) / f).max()
    umax = math.sqrt(1.0 + ax * ax + ay * ay)
    reach = umax * (x[:, 3] * f / zs + 4.0) * 1.01 + 1.0
    dx = np.maximum(np.maximum(px_lo[0] + 0.5 - cx, cx - (px_hi[0] + 0.5)), 0.0)
    dy = np.maximum(np.maximum(px_lo[1] + 0.5 - cy, cy - (px_hi[1] + 0.5)), 0.0)
    keep = ok & (dx * dx + dy * dy <= reach * reach)
    return np.nonzero(keep)[0]
