"""Seeded synthetic scenes and cameras for the meshless molecular renderer.

This module only draws inputs: atom records ``(x, y, z, r)``, element
indices, the element palette, bond pairs, camera frames and the SSAO sample
kernel. It holds none of the rendering arithmetic, so the CUDA renderer and
the CPU oracle read the same arrays and share nothing else.

The paper defines a molecule by atom positions, radii and connectivity
(Methods, "Molecular Graphics Engine") and benchmarks systems from 1e5 atoms
to a 1e8-bead whole cell (Performance evaluation, Table 1). Those datasets are
not available here, so the generators below build stand-ins with the same
sizes and a protein-like spatial structure:

* ``config1``  2,000 atoms uniform in a 40 A cube, 256x256.
* ``config2``  100,000-atom protein-like chains in a 150 A box, 1920x1080.
* ``config3``  20,000 protein-like blobs of 5,000 atoms in a 1.2 um cube
               (1e8 atoms), 3840x2160; a 5e6-atom ball-and-stick subset.
* ``config4``  a 500,000-atom system walked for 256 frames, 4 views, 1280x720.
* ``config5``  20,000 atoms, 16 views at 512x512, plus a perturbed target.

All randomness is NumPy ``default_rng(seed)`` (PCG64). Positions are drawn
in float64 and stored as float32; the float32 arrays are the contract.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

# Element order used by the element index array: C, O, N, H, S.
ELEMENTS = ("C", "O", "N", "H", "S")
ELEMENT_PROBS = np.array([0.50, 0.20, 0.15, 0.12, 0.03])
VDW_RADII = np.array([1.70, 1.52, 1.55, 1.20, 1.80], dtype=np.float32)
# Flat per-element colours (a Jmol-like palette).
PALETTE = np.array(
    [[0.56, 0.56, 0.56],
     [1.00, 0.05, 0.05],
     [0.19, 0.31, 0.97],
     [0.90, 0.90, 0.90],
     [1.00, 0.78, 0.16]], dtype=np.float32)

FOVY_DEG = 60.0
ZNEAR = 0.05
SSAO_SAMPLES = 16
SSAO_RADIUS = 2.0
SSAO_BIAS = 0.025
BALL_RADIUS = 0.4
BOND_RADIUS = 0.15
BOND_MAX = 1.9
BOND_MIN = 1e-3

CAMERA_DTYPE = np.dtype([
    ("eye", "<f4", 3), ("forward", "<f4", 3), ("right", "<f4", 3),
    ("up", "<f4", 3), ("tan_half_fovy", "<f4"), ("znear", "<f4"),
    ("width", "<i4"), ("height", "<i4")])
assert CAMERA_DTYPE.itemsize == 64


@dataclasses.dataclass
class Camera:
    """A pinhole camera: float32 eye and basis exactly as both renderers use them."""
    eye: np.ndarray
    forward: np.ndarray
    right: np.ndarray
    up: np.ndarray
    tan_half_fovy: float
    znear: float
    width: int
    height: int

    def record(self) -> np.ndarray:
        """The 64-byte camera record (one element of ``CAMERA_DTYPE``)."""
        rec = np.zeros((), dtype=CAMERA_DTYPE)
        rec["eye"] = self.eye
        rec["forward"] = self.forward
        rec["right"] = self.right
        rec["up"] = self.up
        rec["tan_half_fovy"] = np.float32(self.tan_half_fovy)
        rec["znear"] = np.float32(self.znear)
        rec["width"] = self.width
        rec["height"] = self.height
        return rec


def cameras_record(cams: List[Camera]) -> np.ndarray:
    out = np.zeros(len(cams), dtype=CAMERA_DTYPE)
    for i, c in enumerate(cams):
        out[i] = c.record()
    return out


def look_at(eye, target, width: int, height: int, fovy_deg: float = FOVY_DEG,
            world_up=(0.0, 1.0, 0.0), znear: float = ZNEAR) -> Camera:
    """Right-handed look-at frame built in float64, stored in float32."""
    eye = np.asarray(eye, dtype=np.float64)
    target = np.asarray(target, dtype=np.float64)
    fwd = target - eye
    fwd /= np.linalg.norm(fwd)
    right = np.cross(fwd, np.asarray(world_up, dtype=np.float64))
    right /= np.linalg.norm(right)
    up = np.cross(right, fwd)
    return Camera(eye=eye.astype(np.float32), forward=fwd.astype(np.float32),
                  right=right.astype(np.float32), up=up.astype(np.float32),
                  tan_half_fovy=float(np.float32(math.tan(math.radians(fovy_deg) / 2.0))),
                  znear=float(np.float32(znear)), width=int(width), height=int(height))


def orbit_camera(center, distance: float, azimuth_deg: float, elevation_deg: float,
                 width: int, height: int) -> Camera:
    """Camera on a sphere about ``center``: azimuth about +y from +z, elevation toward +y."""
    az, el = math.radians(azimuth_deg), math.radians(elevation_deg)
    c = np.asarray(center, dtype=np.float64)
    eye = c + distance * np.array([math.cos(el) * math.sin(az), math.sin(el),
                                   math.cos(el) * math.cos(az)])
    return look_at(eye, c, width, height)


def ssao_kernel(seed: int = 7, n: int = SSAO_SAMPLES) -> np.ndarray:
    """``n`` sample offsets uniform in the unit half-ball z >= 0, the j-th scaled by 0.1 + 0.9 (j/n)^2."""
    rng = np.random.default_rng(seed)
    d = rng.standard_normal((n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    d[:, 2] = np.abs(d[:, 2])
    rad = rng.uniform(0.0, 1.0, n) ** (1.0 / 3.0)
    scale = 0.1 + 0.9 * (np.arange(n) / n) ** 2
    return (d * (rad * scale)[:, None]).astype(np.float32)


def draw_elements(rng: np.random.Generator, n: int) -> np.ndarray:
    cdf = np.cumsum(ELEMENT_PROBS)
    cdf[-1] = 1.0
    return np.searchsorted(cdf, rng.uniform(0.0, 1.0, n), side="right").astype(np.uint8)


def _unit_vectors(rng, shape):
    v = rng.standard_normal(shape + (3,))
    v /= np.linalg.norm(v, axis=-1, keepdims=True)
    return v


def _ball_points(rng, shape, radius):
    return _unit_vectors(rng, shape) * (radius * rng.uniform(0.0, 1.0, shape) ** (1.0 / 3.0))[..., None]


def protein_like(rng: np.random.Generator, n: int, box: float, residues_per_chain: int = 300,
                 step: float = 3.8, atoms_per_residue: int = 8, jitter: float = 1.5) -> np.ndarray:
    """Chains of residue random walks (3.8 A steps, reflected at the box walls), 8 atoms per residue."""
    per_chain = residues_per_chain * atoms_per_residue
    n_chains = -(-n // per_chain)
    res = np.empty((n_chains, residues_per_chain, 3))
    p = rng.uniform(0.0, box, (n_chains, 3))
    res[:, 0] = p
    for k in range(1, residues_per_chain):
        p = p + step * _unit_vectors(rng, (n_chains,))
        p = np.where(p < 0.0, -p, p)
        p = np.where(p > box, 2.0 * box - p, p)
        res[:, k] = p
    atoms = res[:, :, None, :] + _ball_points(rng, (n_chains, residues_per_chain, atoms_per_residue), jitter)
    return atoms.reshape(-1, 3)[:n]


def _blob(rng, n_blobs, residues, step, ball_radius, atoms_per_residue, jitter):
    """Residue walks confined to a ball (radial reflection), centred at the origin."""
    res = np.empty((n_blobs, residues, 3))
    p = np.zeros((n_blobs, 3))
    res[:, 0] = p
    for k in range(1, residues):
        p = p + step * _unit_vectors(rng, (n_blobs,))
        rr = np.linalg.norm(p, axis=1, keepdims=True)
        over = rr > ball_radius
        p = np.where(over, p * ((2.0 * ball_radius - rr) / np.maximum(rr, 1e-30)), p)
        res[:, k] = p
    atoms = res[:, :, None, :] + _ball_points(rng, (n_blobs, residues, atoms_per_residue), jitter)
    return atoms.reshape(n_blobs, -1, 3)


def pack_xyzr(pos: np.ndarray, elem: np.ndarray) -> np.ndarray:
    out = np.empty((pos.shape[0], 4), dtype=np.float32)
    out[:, :3] = pos
    out[:, 3] = VDW_RADII[elem]
    return out


def bonds_within(pos32: np.ndarray, rmax: float = BOND_MAX, rmin: float = BOND_MIN) -> np.ndarray:
    """All pairs i < j with rmin <= |p_i - p_j| < rmax, distances in float64 from the float32 positions."""
    from scipy.spatial import cKDTree
    p = pos32.astype(np.float64)
    pairs = cKDTree(p).query_pairs(rmax, output_type="ndarray")
    if pairs.size == 0:
        return np.zeros((0, 2), dtype=np.uint32)
    pairs.sort(axis=1)
    d = np.linalg.norm(p[pairs[:, 0]] - p[pairs[:, 1]], axis=1)
    keep = (d >= rmin) & (d < rmax)
    pairs = pairs[keep]
    order = np.lexsort((pairs[:, 1], pairs[:, 0]))
    return pairs[order].astype(np.uint32)


@dataclasses.dataclass
class Scene:
    name: str
    xyzr: np.ndarray                      # (N, 4) float32: x, y, z in A and the vdW radius
    elem: np.ndarray                      # (N,) uint8 element index
    cameras: List[Camera]
    ssao: bool
    mode: int = 0                         # 0 = van der Waals spheres, 1 = ball-and-stick
    bonds: Optional[np.ndarray] = None    # (B, 2) uint32, i < j
    frames: Optional[np.ndarray] = None   # (F, N, 4) float32 trajectory
    palette: np.ndarray = dataclasses.field(default_factory=lambda: PALETTE.copy())
    extra: dict = dataclasses.field(default_factory=dict)


def config1(seed: int = 1) -> Scene:
    """2,000 atoms uniform in a 40 A cube; eye (20,20,140) looking at (20,20,20); 256x256, no SSAO."""
    rng = np.random.default_rng(seed)
    pos = rng.uniform(0.0, 40.0, (2000, 3))
    elem = draw_elements(rng, 2000)
    cam = look_at((20.0, 20.0, 140.0), (20.0, 20.0, 20.0), 256, 256)
    return Scene("config1", pack_xyzr(pos, elem), elem, [cam], ssao=False)


def box_edge(n: int) -> float:
    """Protein-like box edge that keeps 1e5 atoms per (150 A)^3."""
    return 150.0 * (n / 1e5) ** (1.0 / 3.0)


def config2(seed: int = 2, n: int = 100_000, width: int = 1920, height: int = 1080) -> Scene:
    """Protein-like 1e5 atoms in a 150 A box, viewed from 450 A (3 box edges); SSAO on."""
    rng = np.random.default_rng(seed)
    L = 150.0
    pos = protein_like(rng, n, L)
    elem = draw_elements(rng, n)
    c = np.array([L / 2] * 3)
    cam = look_at(c + np.array([0.0, 0.0, 3.0 * L]), c, width, height)
    return Scene("config2", pack_xyzr(pos, elem), elem, [cam], ssao=True)


CELL_EDGE = 12000.0


def config3(seed: int = 3, n_clusters: int = 20_000, width: int = 3840, height: int = 2160,
            chunk: int = 1000) -> Scene:
    """Whole-cell stand-in: Poisson cluster centres in a 12,000 A cube, 5,000-atom blobs each.

    Views: V1 (index 0) from 36,000 A on +z, the whole cube in view; V2 (index 1)
    600 A outside the +z face centre, looking at the cube centre.
    """
    rng = np.random.default_rng(seed)
    centres = rng.uniform(0.0, CELL_EDGE, (n_clusters, 3))
    per = 625 * 8
    xyzr = np.empty((n_clusters * per, 4), dtype=np.float32)
    elem = np.empty(n_clusters * per, dtype=np.uint8)
    for c0 in range(0, n_clusters, chunk):
        c1 = min(n_clusters, c0 + chunk)
        blob = _blob(rng, c1 - c0, 625, 3.8, 34.0, 8, 1.5)
        pos = (blob + centres[c0:c1, None, :]).reshape(-1, 3)
        e = draw_elements(rng, pos.shape[0])
        xyzr[c0 * per:c1 * per] = pack_xyzr(pos, e)
        elem[c0 * per:c1 * per] = e
    c = np.array([CELL_EDGE / 2] * 3)
    v1 = look_at(c + np.array([0.0, 0.0, 3.0 * CELL_EDGE]), c, width, height)
    v2 = look_at(np.array([CELL_EDGE / 2, CELL_EDGE / 2, CELL_EDGE + 600.0]), c, width, height)
    return Scene("config3", xyzr, elem, [v1, v2], ssao=True, extra={"centres": centres})


def config3_ball_and_stick(scene3: Optional[Scene] = None, n_clusters: int = 1000) -> Scene:
    """Ball-and-stick subset: the first ``n_clusters`` blobs, 0.4 A balls, 0.15 A bonds under 1.9 A."""
    s = scene3 if scene3 is not None else config3(n_clusters=max(n_clusters, 1))
    n = n_clusters * 625 * 8
    xyzr = np.ascontiguousarray(s.xyzr[:n])
    elem = np.ascontiguousarray(s.elem[:n])
    bonds = bonds_within(xyzr[:, :3])
    return Scene("config3_bs", xyzr, elem, list(s.cameras), ssao=True, mode=1, bonds=bonds)


def config4(seed: int = 4, walk_seed: int = 40, n: int = 500_000, n_frames: int = 256,
            width: int = 1280, height: int = 720, n_views: int = 4) -> Scene:
    """Trajectory: frame f+1 = frame f + N(0, 0.3^2) per coordinate; 4 orbit views at 90 degree steps."""
    rng = np.random.default_rng(seed)
    L = box_edge(n)
    pos0 = protein_like(rng, n, L)
    elem = draw_elements(rng, n)
    rad = VDW_RADII[elem]
    walk = np.random.default_rng(walk_seed)
    frames = np.empty((n_frames, n, 4), dtype=np.float32)
    p = pos0.copy()
    for f in range(n_frames):
        if f > 0:
            p = p + walk.normal(0.0, 0.3, p.shape)
        frames[f, :, :3] = p
        frames[f, :, 3] = rad
    c = np.array([L / 2] * 3)
    cams = [orbit_camera(c, 3.0 * L, 90.0 * k, 0.0, width, height) for k in range(n_views)]
    return Scene("config4", frames[0].copy(), elem, cams, ssao=True, frames=frames)


def config5(seed: int = 5, perturb_seed: int = 50, fd_seed: int = 51, n: int = 20_000,
            size: int = 512) -> Scene:
    """Soft-renderer scene: 16 orbit views; target = positions + N(0, 0.3^2), radii x U(0.95, 1.05)."""
    rng = np.random.default_rng(seed)
    L = box_edge(n)
    pos = protein_like(rng, n, L)
    elem = draw_elements(rng, n)
    xyzr = pack_xyzr(pos, elem)
    c = np.array([L / 2] * 3)
    cams = [orbit_camera(c, 3.0 * L, az, el, size, size)
            for az in (0.0, 90.0, 180.0, 270.0) for el in (-45.0, -15.0, 15.0, 45.0)]
    prng = np.random.default_rng(perturb_seed)
    target = xyzr.copy()
    target[:, :3] = (xyzr[:, :3].astype(np.float64) + prng.normal(0.0, 0.3, (n, 3))).astype(np.float32)
    target[:, 3] = (xyzr[:, 3].astype(np.float64) * prng.uniform(0.95, 1.05, n)).astype(np.float32)
    fd_atoms = np.random.default_rng(fd_seed).permutation(n)
    return Scene("config5", xyzr, elem, cams, ssao=False,
                 extra={"target": target, "fd_order": fd_atoms, "sigma_px": 0.5})


def random_tiny(seed: int, n: int = 40, box: float = 12.0, width: int = 48, height: int = 40,
                distance: float = 20.0) -> Scene:
    """Small random scenes for brute-force cross-checks and edge cases."""
    rng = np.random.default_rng(seed)
    pos = rng.uniform(0.0, box, (n, 3))
    elem = draw_elements(rng, n)
    c = np.array([box / 2] * 3)
    az = rng.uniform(0.0, 360.0)
    el = rng.uniform(-60.0, 60.0)
    cam = orbit_camera(c, distance, az, el, width, height)
    return Scene("tiny%d" % seed, pack_xyzr(pos, elem), elem, [cam], ssao=True)
