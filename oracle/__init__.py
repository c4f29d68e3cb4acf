"""CPU FP64 oracle for the meshless molecular ray-caster.

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The product renderer
never imports this package and this package never imports the renderer; the
two read the same seeded arrays from ``paper_2501_12750_gb300.scenes`` and
share nothing else.

The arithmetic lives in ``vtx_oracle.c`` (plain C, FP64, OpenMP, built with
``-ffp-contract=off``).  This module only compiles it, marshals arrays and
chains its steps: hits -> shading -> SSAO (fetching the depths the SSAO
samples need by computing those pixels too).

Parity unpinned (constants the paper does not state): the Blinn-Phong
coefficients and the SSAO kernel, radius and bias.  They are fixed by
definition here and in the renderer.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vtx_oracle.c")
_SRCS = [_SRC, os.path.join(_HERE, "ses_oracle.c")]
_SO = os.path.join(_HERE, "_vtx_oracle.so")

CFLAGS = ["-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]

FLAG_TIE, FLAG_GRAZE, FLAG_NEAR, FLAG_SPLIT = 1, 2, 4, 16
FLAG_GRID, FLAG_MARGIN, FLAG_FETCH = 32, 64, 128
FLAG_CUTOFF, FLAG_ORDER, FLAG_STOP, FLAG_CLAMP = 256, 512, 1024, 2048
FLAG_SILH = 4096    # SSAO: the pixel's hit lies within SIL_TOL (relative) of its surface's silhouette
FLAG_BAND = 8192    # toon shading: the diffuse term lies within BAND_TOL of a band boundary
FLAG_EDGE = 16384   # outline: a neighbour's depth step lies within EDGE_ABS + EDGE_REL * depth of the threshold
ID_FLAGS = FLAG_TIE | FLAG_GRAZE | FLAG_NEAR
NO_ID = 0xFFFFFFFF

TIE_TOL = 1e-4      # A: pixels whose two nearest depths differ by less are id-ambiguous
GRAZE_TOL = 1e-6    # A: distance to a silhouette/rim/near-plane decision
# SSAO ambiguity bands: test tolerances sized from the FP32 error of a renderer that computes the hit point,
# normal and sample offsets in FP32 relative to each primitive.  Near a silhouette the closest-approach
# discriminant is small and its rounding error grows as 1/sqrt(sil) (sil = (R^2 - rho^2)/(2 R^2)); measured
# on the GPU planes of the parity scenes, the sample offset stays within 9e-8 (f/d) r_ssao (1 + 1/sqrt(sil))
# px and the normal within 1e-7 (1 + 1/sqrt(sil)); the constants below keep a factor of 4 over that.
ERR_POS = 4e-7      # sample position error bound: ERR_POS * ssao radius * (1 + 1/sqrt(sil)) A
ERR_T = 2e-7        # hit depth error bound: ERR_T * R_hit * (1 + 1/sqrt(sil)) + one depth-key step
GRID_ABS = 1e-6     # px: absolute part of the grid-line band (rounding of the projected offset)
GRID_REL = 1.2e-7   # relative part
MARGIN_ABS = 2e-7   # A: absolute part of the occlusion-test margin
KEY_SPAN = 4294966784.0  # depth-key steps over a frame's depth range (32-bit keys)
SIL_TOL = 1e-7      # relative: (R^2 - rho^2)/(2 R^2) below this the FP32 normal itself is unreliable
BAND_TOL = 1e-3     # toon: |n.L * levels - boundary| (an FP32 normal is good to 1e-4 per component)
EDGE_ABS = 1e-4     # A: outline depth-step decision ...
EDGE_REL = 2e-5     # ... plus this fraction of the pixel's depth (FP32 depth keys)

SHADE_DEFAULTS = dict(ka=0.2, kd=0.7, ks=0.3, shininess=32.0,
                      light_dir=(0.25, 0.5, 1.0), background=(1.0, 1.0, 1.0))


def build(force: bool = False) -> str:
    """Compile the oracle library next to its source (gcc, no GPU needed)."""
    if force or not os.path.exists(_SO) or any(os.path.getmtime(_SO) < os.path.getmtime(f) for f in _SRCS):
        tmp = _SO + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", *CFLAGS, *_SRCS, "-o", tmp, "-lm"])
        os.replace(tmp, _SO)
    return _SO


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_SO)
        P = ctypes.c_void_p
        i64, i32, f32, f64 = ctypes.c_int64, ctypes.c_int32, ctypes.c_float, ctypes.c_double
        L.orc_hits.argtypes = [P, i64, P, i64, i32, f32, f32, f32, P, P, P, i64, f64, f64, P, P, P, P, P, P, P,
                               i32]
        L.orc_hits.restype = i32
        L.orc_shade.argtypes = [P, P, i64, P, P, P, i64, P, P, P, P, f64, f64, f64, f64, P, i32, i32, f64, P, P]
        L.orc_post.argtypes = [i64, P, P, P, P, f64, P, f64, f64, f64, P, f64, f64, P, P]
        L.orc_ses_sas.argtypes = [P, i64, f32, P, f32, P, P, P]
        L.orc_ses_k.argtypes = [f32, f32]
        L.orc_ses_k.restype = i32
        L.orc_ses_edt.argtypes = [P, P, i32, P]
        L.orc_ses_mc.argtypes = [P, P, P, f32, f32, P, i64, P, P]
        L.orc_ses_mc.restype = i64
        L.orc_ses_case_counts.argtypes = [P]
        L.orc_ssao_project.argtypes = [P, P, i64, P, P, P, P, i32, f64, f64, f64, P, P, P, P, P]
        L.orc_ssao_resolve.argtypes = [i64, i32, P, P, P, P, P, P, P, f64, f64, f64, P, P, P, P]
        L.orc_soft_forward.argtypes = [P, i64, P, f64, P, i64, f64, P, P, P, P, P, P, i32]
        L.orc_soft_vjp.argtypes = [P, i64, P, f64, P, i64, P, P, P, P, i32]
        _lib = L
    return _lib


def _p(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _cam(cam) -> np.ndarray:
    rec = cam.record() if hasattr(cam, "record") else np.asarray(cam)
    return np.array(rec).reshape(1)


def all_pixels(width: int, height: int) -> np.ndarray:
    ys, xs = np.mgrid[0:height, 0:width]
    return np.ascontiguousarray(np.stack([xs.ravel(), ys.ravel()], axis=1).astype(np.int32))


@dataclass
class Hits:
    pix: np.ndarray
    depth: np.ndarray
    id: np.ndarray
    normal: np.ndarray
    gap: np.ndarray
    flags: np.ndarray
    side: np.ndarray
    sil: np.ndarray
    rad: Optional[np.ndarray] = None  # radius of the surface hit (0 for background)
    rgb: Optional[np.ndarray] = None
    ao: Optional[np.ndarray] = None
    rgb_final: Optional[np.ndarray] = None


def hits(xyzr, cam, pix, bonds=None, mode=0, ball_radius=0.4, bond_radius=0.15, probe=1.4, clip=None,
         tie_tol=TIE_TOL, graze_tol=GRAZE_TOL, threads=0) -> Hits:
    """Nearest hit per listed pixel by brute force over all primitives (FP64).

    mode 0 van der Waals, 1 ball-and-stick, 2 sticks, 3 solvent accessible surface (r + probe);
    clip = (nx, ny, nz, d) keeps atoms with n.X + d >= 0 (a bond needs both of its atoms).
    """
    xyzr = np.ascontiguousarray(xyzr, dtype=np.float32)
    pix = np.ascontiguousarray(pix, dtype=np.int32).reshape(-1, 2)
    nb = 0 if bonds is None else int(bonds.shape[0])
    b = None if bonds is None else np.ascontiguousarray(bonds, dtype=np.uint32)
    P = pix.shape[0]
    out = Hits(pix=pix, depth=np.empty(P), id=np.empty(P, np.uint32), normal=np.empty((P, 3)),
               gap=np.empty(P), flags=np.empty(P, np.int32), side=np.empty(P, np.int32), sil=np.empty(P))
    c = _cam(cam)
    cl = None if clip is None else np.ascontiguousarray(clip, np.float32).reshape(4)
    lib().orc_hits(_p(xyzr), xyzr.shape[0], _p(b), nb, mode, ball_radius, bond_radius, probe, _p(cl), _p(c),
                   _p(pix), P,
                   tie_tol, graze_tol, _p(out.depth), _p(out.id), _p(out.normal), _p(out.gap), _p(out.flags),
                   _p(out.side), _p(out.sil), threads)
    out.rad = hit_radius(out, xyzr, xyzr.shape[0], mode=mode, ball_radius=ball_radius, bond_radius=bond_radius,
                         probe=probe)
    return out


def shade(h: Hits, elem, palette, n_atoms, cam, bonds=None, model=0, toon_levels=4, band_tol=BAND_TOL,
          **kw) -> np.ndarray:
    """Colour per hit: model 0 Blinn-Phong, 1 flat albedo, 2 matte (no specular), 3 toon bands."""
    s = dict(SHADE_DEFAULTS)
    s.update(kw)
    P = h.pix.shape[0]
    rgb = np.empty((P, 3))
    light = np.asarray(s["light_dir"], np.float32)
    bg = np.asarray(s["background"], np.float32)
    b = None if bonds is None else np.ascontiguousarray(bonds, dtype=np.uint32)
    lib().orc_shade(_p(np.ascontiguousarray(elem, np.uint8)), _p(np.ascontiguousarray(palette, np.float32)),
                    n_atoms, _p(b), _p(_cam(cam)), _p(h.pix), P, _p(h.id), _p(h.normal), _p(h.side), _p(light),
                    s["ka"], s["kd"], s["ks"], s["shininess"], _p(bg), model, toon_levels, band_tol, _p(rgb),
                    _p(h.flags))
    return rgb


def hit_radius(h: Hits, xyzr, n_atoms, mode=0, ball_radius=0.4, bond_radius=0.15, probe=1.4) -> np.ndarray:
    """Radius of the surface hit at each pixel (0 for background)."""
    rad = np.zeros(h.id.shape[0])
    cov = h.id != NO_ID
    atom = cov & (h.id.astype(np.int64) < n_atoms)
    ids = h.id[atom].astype(np.int64)
    if mode == 1:
        rad[atom] = float(np.float32(ball_radius))
    elif mode == 2:
        rad[atom] = float(np.float32(bond_radius))
    elif mode == 3:
        rad[atom] = (np.asarray(xyzr, np.float32)[ids, 3] + np.float32(probe)).astype(np.float64)
    else:
        rad[atom] = np.asarray(xyzr, np.float32)[ids, 3].astype(np.float64)
    rad[cov & ~atom] = float(np.float32(bond_radius))
    return rad


def key_step(xyzr, cam, chunk=1 << 22) -> float:
    """Depth-key step of a renderer that spreads 2^32 keys over the depth range of the primitives in front of
    the eye: (max(z + r) - max(min(z - r), near / 2)) / KEY_SPAN over every atom (a superset of any visible
    set, so the step is an upper bound)."""
    x = np.asarray(xyzr, np.float32)
    E = cam.eye.astype(np.float64)
    F = cam.forward.astype(np.float64)
    lo, hi = np.inf, 0.0
    for i0 in range(0, x.shape[0], chunk):
        c = x[i0:i0 + chunk].astype(np.float64)
        z = (c[:, :3] - E) @ F
        r = c[:, 3] + 1.5  # covers every representation's radius (probe, ball, bond)
        front = z + r > float(cam.znear)
        if front.any():
            lo = min(lo, float((z - r)[front].min()))
            hi = max(hi, float((z + r)[front].max()))
    if hi <= 0.0:
        return 0.0
    lo = max(lo, 0.5 * float(cam.znear))
    return max(hi - lo, 1.0) / KEY_SPAN


def hit_errors(h: Hits, rad: np.ndarray, step: float, radius: float = 2.0):
    """Per-pixel bounds on the SSAO sample position error (A) and the hit depth error of an FP32 renderer."""
    sil = np.maximum(h.sil, 1e-30)
    amp = 1.0 + 1.0 / np.sqrt(sil)
    err_pos = ERR_POS * radius * amp
    err_t = ERR_T * rad * amp + step
    cov = h.id != NO_ID
    return np.where(cov, err_pos, 0.0), np.where(cov, err_t, 0.0)


def ssao(h: Hits, xyzr, cam, kernel, radius=2.0, bias=0.025, bonds=None, mode=0, ball_radius=0.4,
         bond_radius=0.15, probe=1.4, clip=None, grid_abs=GRID_ABS, grid_rel=GRID_REL, margin_abs=MARGIN_ABS,
         sil_tol=SIL_TOL, depth_step=None, threads=0):
    """AO per listed pixel; flags gain GRID / MARGIN / FETCH / SILH bits.  Fetched pixels are ray-cast on demand.

    The bands flag samples whose projection or occlusion test a renderer computing the hit point in FP32
    could decide differently (see orc_ssao_project / orc_ssao_resolve); depth_step is that renderer's
    depth-key step (default: key_step() of the scene).
    """
    kernel = np.ascontiguousarray(kernel, np.float32).reshape(-1, 3)
    ns = kernel.shape[0]
    P = h.pix.shape[0]
    n_atoms = np.asarray(xyzr).shape[0]
    fetch = np.empty((P, ns, 2), np.int32)
    sdepth = np.empty((P, ns))
    c = _cam(cam)
    step = key_step(xyzr, cam) if depth_step is None else float(depth_step)
    rkw = dict(mode=mode, ball_radius=ball_radius, bond_radius=bond_radius, probe=probe)
    err_pos, err_t = hit_errors(h, hit_radius(h, xyzr, n_atoms, **rkw), step, radius)
    h.flags[(h.id != NO_ID) & (h.sil < sil_tol)] |= FLAG_SILH
    lib().orc_ssao_project(_p(c), _p(h.pix), P, _p(h.depth), _p(h.id), _p(h.normal), _p(kernel), ns, radius,
                           grid_abs, grid_rel, _p(err_pos), _p(err_t), _p(fetch), _p(sdepth), _p(h.flags))
    W = int(c["width"][0])
    lin = np.where(fetch[..., 0] >= 0, fetch[..., 1].astype(np.int64) * W + fetch[..., 0], -1)
    own = h.pix[:, 1].astype(np.int64) * W + h.pix[:, 0]
    need = np.unique(lin[lin >= 0])
    known = dict(zip(own.tolist(), range(P)))
    missing = np.array([q for q in need.tolist() if q not in known], dtype=np.int64)
    info = {}  # pixel -> (depth, id flags, gap, depth error bound)
    for q, k in known.items():
        info[q] = (h.depth[k], int(h.flags[k] & ID_FLAGS), h.gap[k], err_t[k])
    if missing.size:
        mp = np.stack([missing % W, missing // W], axis=1).astype(np.int32)
        hm = hits(xyzr, cam, mp, bonds=bonds, clip=clip, threads=threads, **rkw)
        _, et_m = hit_errors(hm, hit_radius(hm, xyzr, n_atoms, **rkw), step, radius)
        for k, q in enumerate(missing.tolist()):
            info[q] = (hm.depth[k], int(hm.flags[k] & ID_FLAGS), hm.gap[k], et_m[k])
    valid = lin >= 0
    flat = lin[valid].tolist()
    zf = np.full((P, ns), np.inf)
    famb = np.zeros((P, ns), np.int32)
    fgap = np.zeros((P, ns))
    ferr = np.zeros((P, ns))
    if flat:
        rows = np.array([info[q] for q in flat])
        zf[valid] = rows[:, 0]
        famb[valid] = rows[:, 1].astype(np.int32)
        fgap[valid] = rows[:, 2]
        ferr[valid] = rows[:, 3]
    ao = np.empty(P)
    lib().orc_ssao_resolve(P, ns, _p(h.depth), _p(h.id), _p(sdepth), _p(np.ascontiguousarray(zf)),
                           _p(np.ascontiguousarray(famb)), _p(np.ascontiguousarray(fgap)),
                           _p(np.ascontiguousarray(ferr)), radius, bias, margin_abs, _p(err_pos), _p(err_t),
                           _p(ao), _p(h.flags))
    return ao


def post(h: Hits, xyzr, cam, rgb, outline_depth=0.0, outline_color=(0.0, 0.0, 0.0), fog_near=0.0, fog_far=0.0,
         fog_density=0.0, background=SHADE_DEFAULTS["background"], rep=None, threads=0) -> np.ndarray:
    """Outline, then fog, on colours `rgb` (after shading and AO); 4-neighbour depths are ray-cast on demand."""
    rep = rep or {}
    P = h.pix.shape[0]
    out = np.ascontiguousarray(rgb, np.float64).copy()
    W, H = int(_cam(cam)["width"][0]), int(_cam(cam)["height"][0])
    nd = np.full((P, 4), np.nan)
    na = np.zeros((P, 4), np.int32)
    if outline_depth > 0.0:
        off = np.array([[-1, 0], [1, 0], [0, -1], [0, 1]], np.int64)
        q = h.pix[:, None, :].astype(np.int64) + off[None]
        inside = (q[..., 0] >= 0) & (q[..., 0] < W) & (q[..., 1] >= 0) & (q[..., 1] < H)
        lin = q[..., 1] * W + q[..., 0]
        own = dict(zip((h.pix[:, 1].astype(np.int64) * W + h.pix[:, 0]).tolist(), range(P)))
        need = np.unique(lin[inside])
        missing = np.array([v for v in need.tolist() if v not in own], np.int64)
        depth_of = {v: h.depth[k] for v, k in own.items()}
        amb_of = {v: int(h.flags[k] & ID_FLAGS) for v, k in own.items()}
        if missing.size:
            mp = np.stack([missing % W, missing // W], 1).astype(np.int32)
            hm = hits(xyzr, cam, mp, threads=threads, **rep)
            for k, v in enumerate(missing.tolist()):
                depth_of[v] = hm.depth[k]
                amb_of[v] = int(hm.flags[k] & ID_FLAGS)
        flat = lin[inside].tolist()
        nd[inside] = np.array([depth_of[v] for v in flat]) if flat else []
        na[inside] = np.array([amb_of[v] for v in flat], np.int32) if flat else []
    lib().orc_post(P, _p(h.depth), _p(h.id), _p(np.ascontiguousarray(nd)), _p(np.ascontiguousarray(na)),
                   outline_depth, _p(np.asarray(outline_color, np.float32)), fog_near, fog_far, fog_density,
                   _p(np.asarray(background, np.float32)), EDGE_ABS, EDGE_REL, _p(out), _p(h.flags))
    return out


REP_KEYS = ("mode", "ball_radius", "bond_radius", "probe", "clip")
POST_KEYS = ("outline_depth", "outline_color", "fog_near", "fog_far", "fog_density")


def render_pixels(scene, cam_index, pix, kernel=None, threads=0, **kw) -> Hits:
    """Hits, shading, (when ``kernel`` is given) SSAO, then outline and fog at the listed pixels of a scene view.

    Keyword arguments go to the step that takes them: representation (mode, ball_radius, bond_radius, probe,
    clip), shading (model, toon_levels, ka, kd, ks, shininess, light_dir, background) and post-processing
    (outline_depth, outline_color, fog_near, fog_far, fog_density).
    """
    cam = scene.cameras[cam_index]
    rep = dict(bonds=scene.bonds, mode=scene.mode)
    rep.update({k: kw.pop(k) for k in REP_KEYS if k in kw})
    pk = {k: kw.pop(k) for k in POST_KEYS if k in kw}
    h = hits(scene.xyzr, cam, pix, threads=threads, **rep)
    h.rgb = shade(h, scene.elem, scene.palette, scene.xyzr.shape[0], cam, bonds=scene.bonds, **kw)
    if kernel is not None:
        h.ao = ssao(h, scene.xyzr, cam, kernel, threads=threads, **rep)
        h.rgb_final = h.rgb * h.ao[:, None]
    else:
        h.ao = np.ones(h.pix.shape[0])
        h.rgb_final = h.rgb
    if pk:
        h.rgb_final = post(h, scene.xyzr, cam, h.rgb_final, background=kw.get("background",
                           SHADE_DEFAULTS["background"]), rep=rep, threads=threads, **pk)
    return h


# --------------------------------------------------------------- soft form --

@dataclass
class Soft:
    A: np.ndarray
    D: np.ndarray
    N: np.ndarray
    n_used: np.ndarray
    T_final: np.ndarray
    flags: np.ndarray


def soft_forward(xyzr64, cam, pix, sigma=0.5, amb_tol=1e-6, threads=0) -> Soft:
    x = np.ascontiguousarray(xyzr64, np.float64).reshape(-1, 4)
    pix = np.ascontiguousarray(pix, np.int32).reshape(-1, 2)
    P = pix.shape[0]
    o = Soft(np.empty(P), np.empty(P), np.empty((P, 3)), np.empty(P, np.int32), np.empty(P), np.empty(P, np.int32))
    lib().orc_soft_forward(_p(x), x.shape[0], _p(_cam(cam)), sigma, _p(pix), P, amb_tol, _p(o.A), _p(o.D),
                           _p(o.N), _p(o.n_used), _p(o.T_final), _p(o.flags), threads)
    return o


def soft_vjp(xyzr64, cam, pix, gA, gD, gN, sigma=0.5, threads=0) -> np.ndarray:
    """d/d(x,y,z,r) of sum(gA A + gD D + gN . N) over the listed pixels (FP64, analytic)."""
    x = np.ascontiguousarray(xyzr64, np.float64).reshape(-1, 4)
    pix = np.ascontiguousarray(pix, np.int32).reshape(-1, 2)
    P = pix.shape[0]
    grad = np.zeros((x.shape[0], 4))
    lib().orc_soft_vjp(_p(x), x.shape[0], _p(_cam(cam)), sigma, _p(pix), P,
                       _p(np.ascontiguousarray(gA, np.float64)), _p(np.ascontiguousarray(gD, np.float64)),
                       _p(np.ascontiguousarray(gN, np.float64).reshape(-1, 3)), _p(grad), threads)
    return grad


# ------------------------------------------------------------------- SES --

@dataclass
class Ses:
    origin: np.ndarray   # float32 (3,)
    h: float
    dims: np.ndarray     # int32 (nx, ny, nz)
    K: int
    sas: np.ndarray      # uint8 [nz][ny][nx]
    edt2: np.ndarray     # uint16 [nz][ny][nx], K*K + 1 = "farther than K"
    tris: np.ndarray     # float64 [T][3][3]
    edges: np.ndarray    # int64 [T][3] vertex labels: cell * 16 + edge (0..11) or cell * 16 + 12 + loop


def ses_grid(xyzr, probe=1.4, h=0.5, margin=2):
    """A grid covering every SAS sphere with `margin` spare points on each side (origin float32, dims int32)."""
    x = np.asarray(xyzr, np.float64)
    R = x[:, 3] + probe
    lo = (x[:, :3] - R[:, None]).min(0) - margin * h
    hi = (x[:, :3] + R[:, None]).max(0) + margin * h
    dims = (np.floor((hi - lo) / h).astype(np.int64) + 2).astype(np.int32)
    return lo.astype(np.float32), np.float32(h), dims


def ses(xyzr, origin, h, dims, probe=1.4, offset=None) -> Ses:
    """SAS interior, windowed squared distance transform and marching-cubes triangles (see ses_oracle.c).

    offset: grid index of this grid's first point within a larger grid of the same origin and spacing (the
    coordinates are then those of the larger grid; cell labels stay local to this one).
    """
    x = np.ascontiguousarray(xyzr, np.float32).reshape(-1, 4)
    o = np.ascontiguousarray(origin, np.float32).reshape(3)
    d = np.ascontiguousarray(dims, np.int32).reshape(3)
    off = None if offset is None else np.ascontiguousarray(offset, np.int32).reshape(3)
    n = int(d[0]) * int(d[1]) * int(d[2])
    sas = np.empty(n, np.uint8)
    lib().orc_ses_sas(_p(x), x.shape[0], probe, _p(o), float(h), _p(d), _p(off), _p(sas))
    K = int(lib().orc_ses_k(probe, float(h)))
    edt2 = np.empty(n, np.uint16)
    lib().orc_ses_edt(_p(sas), _p(d), K, _p(edt2))
    T = int(lib().orc_ses_mc(_p(edt2), _p(d), _p(o), float(h), probe, _p(off), 0, None, None))
    tris = np.empty((max(T, 1), 3, 3))
    edges = np.empty((max(T, 1), 3), np.int64)
    lib().orc_ses_mc(_p(edt2), _p(d), _p(o), float(h), probe, _p(off), T, _p(tris), _p(edges))
    shp = (int(d[2]), int(d[1]), int(d[0]))
    return Ses(o, float(h), d, K, sas.reshape(shp), edt2.reshape(shp), tris[:T], edges[:T])


def ses_case_counts() -> np.ndarray:
    c = np.empty(256, np.int32)
    lib().orc_ses_case_counts(_p(c))
    return c

