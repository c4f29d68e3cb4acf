"""Shared helpers for the GPU parity tests: run the CUDA path, run the oracle, compare.

Tolerances (per pixel, FP32 values, never 8-bit quantised):
  id      bit-exact, except pixels the oracle flags as ambiguous (two nearest
          depths within 1e-4 A, a silhouette / rim / near-plane decision within
          1e-6 A);
  depth   |d_gpu - d_ref| / d_ref <= 1e-5;
  normal  max abs per component <= 1e-4;
  rgb     <= 1/255 per channel (no SSAO), final rgb and AO <= 2/255 with SSAO
          (excluded: pixels with an SSAO sample within 1e-5 px plus the
          projection of 1e-5 A of a grid line, an occlusion test within 5e-5 A
          of its threshold, a fetch of an ambiguous pixel, or a hit within 1e-4
          (relative) of its surface's silhouette).
Depth, normal and colour are compared where the ids match and nothing is flagged.
"""
from __future__ import annotations

import numpy as np

import oracle

DEPTH_RTOL = 1e-5
NORMAL_ATOL = 1e-4
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


def gather(res, pix):
    """GPU planes at the listed (px, py) pixels."""
    px, py = pix[:, 0], pix[:, 1]
    return dict(depth=res["depth"][py, px], id=res["id"][py, px], normal=res["normal"][:, py, px].T,
                rgb=res["rgb"][:, py, px].T, ao=res["ao"][py, px])


def compare(res, h, ssao: bool, allow_excluded=0.005, label="", colour=True):
    """Assert parity of GPU planes `res` with oracle hits `h`; returns a stats dict.

    colour=False checks ids, depths and normals only (oracle hits computed without shading).
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
        rel = np.abs(g["depth"][ok].astype(np.float64) - h.depth[ok]) / h.depth[ok]
        assert rel.max() <= DEPTH_RTOL, "%s: depth rel err %.3g" % (label, rel.max())
        nerr = np.abs(g["normal"][ok].astype(np.float64) - h.normal[ok]).max()
        assert nerr <= NORMAL_ATOL, "%s: normal err %.3g" % (label, nerr)
    else:
        rel, nerr = np.zeros(1), 0.0
    bg = (~amb) & (~covered)
    assert np.isinf(g["depth"][bg]).all() and (g["normal"][bg] == 0).all()
    rgb_ok = (~amb) & ((h.flags & (oracle.FLAG_SPLIT | oracle.FLAG_BAND | oracle.FLAG_EDGE)) == 0)
    if not colour:
        return dict(pixels=n, covered=int(covered.sum()), excluded=int(amb.sum()), depth_rel=float(rel.max()),
                    normal=float(nerr))
    if ssao:
        rgb_ok &= (h.flags & SSAO_FLAGS) == 0
        aoerr = np.abs(g["ao"][rgb_ok] - h.ao[rgb_ok]).max() if rgb_ok.any() else 0.0
        assert aoerr <= AO_ATOL, "%s: ao err %.3g" % (label, aoerr)
        ref = h.rgb_final
        tol = AO_ATOL
    else:
        aoerr = 0.0
        ref = h.rgb_final if h.rgb_final is not None else h.rgb
        tol = RGB_ATOL
        if h.rgb_final is not None and (h.flags & oracle.FLAG_FETCH).any():
            rgb_ok &= (h.flags & oracle.FLAG_FETCH) == 0  # outline next to an id-ambiguous neighbour
    cerr = np.abs(g["rgb"][rgb_ok] - ref[rgb_ok]).max() if rgb_ok.any() else 0.0
    assert cerr <= tol, "%s: rgb err %.3g" % (label, cerr)
    excl = amb | (~rgb_ok)
    frac = excl[covered].mean() if covered.any() else 0.0
    by_flag = {name: int(((h.flags & bit) != 0)[covered].sum()) for name, bit in
               [("tie", oracle.FLAG_TIE), ("graze", oracle.FLAG_GRAZE), ("near", oracle.FLAG_NEAR),
                ("split", oracle.FLAG_SPLIT), ("grid", oracle.FLAG_GRID), ("margin", oracle.FLAG_MARGIN),
                ("fetch", oracle.FLAG_FETCH), ("silh", oracle.FLAG_SILH), ("band", oracle.FLAG_BAND),
                ("edge", oracle.FLAG_EDGE)]}
    assert frac <= allow_excluded, "%s: %.3f%% of covered pixels excluded %s" % (label, 100 * frac, by_flag)
    return dict(pixels=n, covered=int(covered.sum()), excluded=int(excl.sum()), depth_rel=float(rel.max()),
                normal=float(nerr), rgb=float(cerr), ao=float(aoerr))


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
