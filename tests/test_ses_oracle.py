"""Pins for the SES oracle (grid SAS, windowed distance transform, marching cubes) against independent references.

Each pin checks the oracle against something it does not compute itself: exact integer lattice counts, a
library Euclidean distance transform, the analytic solvent excluded surface of one and of two atoms (the
reentrant arc of a probe touching both), and combinatorial invariants of a closed oriented surface.
"""
import math

import numpy as np
import pytest

import oracle


def mesh_stats(tris, edges):
    """Area, enclosed volume (divergence theorem), Euler characteristic and edge-manifold check of a soup."""
    T = np.asarray(tris, np.float64)
    area = 0.5 * np.linalg.norm(np.cross(T[:, 1] - T[:, 0], T[:, 2] - T[:, 0]), axis=1).sum()
    vol = np.einsum("ij,ij->i", T[:, 0], np.cross(T[:, 1], T[:, 2])).sum() / 6.0
    return area, vol


def weld(edges, dims):
    """Global ids of mesh vertices: the grid edge each lies on (shared by the cells around that edge); loop
    means (labels cell * 16 + 12 + loop) stay private to their cell."""
    nx, ny, nz = (int(v) for v in dims)
    cells = edges // 16
    local = edges % 16
    e = np.where(local < 12, local, 0)
    i = cells % (nx - 1)
    j = (cells // (nx - 1)) % (ny - 1)
    k = cells // ((nx - 1) * (ny - 1))
    corner = np.array([[0, 0, 0], [1, 0, 0], [1, 1, 0], [0, 1, 0], [0, 0, 1], [1, 0, 1], [1, 1, 1], [0, 1, 1]])
    ends = np.array([[0, 1], [1, 2], [2, 3], [3, 0], [4, 5], [5, 6], [6, 7], [7, 4], [0, 4], [1, 5], [2, 6], [3, 7]])
    a = corner[ends[e, 0]]
    b = corner[ends[e, 1]]
    base = np.stack([i, j, k], -1)
    pa = base + a
    pb = base + b
    lo = np.minimum(pa, pb)
    axis = np.argmax(np.abs(pb - pa), axis=-1)
    lin = (lo[..., 2] * ny + lo[..., 1]) * nx + lo[..., 0]
    return np.where(local < 12, lin * 3 + axis, -1 - (cells * 4 + (local - 12)))


def topology(tris_edges, dims):
    ids = weld(tris_edges, dims)
    V = len(np.unique(ids))
    F = len(ids)
    und = np.sort(np.concatenate([ids[:, [0, 1]], ids[:, [1, 2]], ids[:, [2, 0]]]), axis=1)
    u, cnt = np.unique(und, axis=0, return_counts=True)
    directed = np.concatenate([ids[:, [0, 1]], ids[:, [1, 2]], ids[:, [2, 0]]])
    du, dcnt = np.unique(directed, axis=0, return_counts=True)
    return dict(V=V, E=len(u), F=F, chi=V - len(u) + F, manifold=bool((cnt == 2).all()),
                oriented=bool((dcnt == 1).all()))


def test_sas_lattice_count_is_exact_with_dyadic_values():
    """h = 0.25, origin -4.0, atom at 0 with r + p = 3.0: FP64 is exact, inside <=> i^2+j^2+k^2 < 144."""
    x = np.array([[0.0, 0.0, 0.0, 1.75]], np.float32)
    o = np.array([-4.0, -4.0, -4.0], np.float32)
    d = np.array([33, 33, 33], np.int32)
    s = oracle.ses(x, o, 0.25, d, probe=1.25)
    g = np.arange(33) - 16
    n2 = g[None, None, :] ** 2 + g[None, :, None] ** 2 + g[:, None, None] ** 2
    np.testing.assert_array_equal(s.sas, (n2 < 144).astype(np.uint8))


def test_edt_equals_library_distance_transform_within_the_window():
    ndi = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(4)
    x = np.concatenate([rng.uniform(0, 6, (12, 3)), rng.uniform(1.2, 1.9, (12, 1))], 1).astype(np.float32)
    o, h, d = oracle.ses_grid(x, probe=1.4, h=0.4)
    s = oracle.ses(x, o, h, d, probe=1.4)
    ref = ndi.distance_transform_edt(s.sas) ** 2
    ref = np.rint(ref).astype(np.int64)
    K2 = s.K * s.K
    got = s.edt2.astype(np.int64)
    near = ref <= K2
    assert near.sum() > 1000 and (~near).sum() > 0
    np.testing.assert_array_equal(got[near], ref[near])
    assert (got[~near] == K2 + 1).all()


def test_case_table_counts_and_complements():
    c = oracle.ses_case_counts()
    assert c[0] == 0 and c[255] == 0
    # one corner: a triangle; two corners on an edge: a quad (4 around its mean); a face: a quad; three
    # corners of a face: a pentagon
    assert c[1] == 1 and c[3] == 4 and c[15] == 4 and c[7] == 5
    # one inside corner or one outside corner: always one triangle
    for k in range(8):
        assert c[1 << k] == 1 and c[255 ^ (1 << k)] == 1


def _random_blob_grid(seed, n=7):
    """A closed surface from a random binary grid: EDT values 0 (outside) or K*K+1 (inside), zero border."""
    rng = np.random.default_rng(seed)
    inside = np.zeros((n, n, n), bool)
    inside[1:-1, 1:-1, 1:-1] = rng.random((n - 2, n - 2, n - 2)) < 0.5
    return inside


@pytest.mark.parametrize("seed", range(6))
def test_marching_cubes_surface_is_closed_and_consistently_oriented(seed):
    """Random inside/outside patterns (ambiguous faces included) give a closed, oriented 2-manifold."""
    inside = _random_blob_grid(seed)
    n = inside.shape[0]
    h, p = np.float32(0.5), np.float32(1.4)
    K = int(oracle.lib().orc_ses_k(p, h))
    edt2 = np.where(inside, K * K + 1, 0).astype(np.uint16)
    d = np.array([n, n, n], np.int32)
    o = np.zeros(3, np.float32)
    T = int(oracle.lib().orc_ses_mc(oracle._p(edt2), oracle._p(d), oracle._p(o), float(h), float(p), None, 0, None,
                                    None))
    tris = np.empty((T, 3, 3))
    edges = np.empty((T, 3), np.int64)
    oracle.lib().orc_ses_mc(oracle._p(edt2), oracle._p(d), oracle._p(o), float(h), float(p), None, T,
                            oracle._p(tris), oracle._p(edges))
    topo = topology(edges, d)
    assert T > 20 and topo["manifold"] and topo["oriented"]
    area, vol = mesh_stats(tris, edges)
    assert vol > 0


def _analytic_two_atom_field(P, zc, r, p):
    """dist(X, A) - p for the probe-accessible set A of atoms at (0,0,+-zc), both of radius r (exact, axisymmetric)."""
    z = P[:, 2]
    rho = np.hypot(P[:, 0], P[:, 1])
    Rp = r + p
    d1 = np.hypot(z - zc, rho)
    d2 = np.hypot(z + zc, rho)
    inside_union = (d1 < Rp) | (d2 < Rp)
    if zc < Rp:
        cusp_rho = math.sqrt(Rp * Rp - zc * zc)
        # arc of circle 1 outside disc 2 (z >= 0 side) and its mirror; beyond the arc, the cusp point
        def arc_dist(dz, c_sign):
            # radial projection of (z, rho) onto the circle of radius r + p around (c_sign * zc, 0)
            k = Rp / np.maximum(np.hypot(dz, rho), 1e-300)
            qz = c_sign * zc + dz * k
            on_arc = (c_sign * qz) >= 0  # the part of circle i outside the other disc lies on its side of z = 0
            da = np.abs(np.hypot(dz, rho) - Rp)
            dc = np.hypot(z, rho - cusp_rho)  # else the nearer arc end, the cusp ring
            return np.where(on_arc, da, dc)
        a1 = arc_dist(z - zc, 1.0)
        a2 = arc_dist(z + zc, -1.0)
        dist = np.minimum(a1, a2)
    else:
        dist = np.minimum(np.abs(d1 - Rp), np.abs(d2 - Rp))
    out = np.where(inside_union, dist, 0.0)
    return out - p


@pytest.mark.parametrize("h", [0.25, 0.15])
def test_single_atom_ses_is_its_sphere(h):
    r = 1.7
    x = np.array([[0.3, -0.2, 0.1, r]], np.float32)
    o, hh, d = oracle.ses_grid(x, probe=1.4, h=h)
    s = oracle.ses(x, o, hh, d, probe=1.4)
    c = x[0, :3].astype(np.float64)
    rr = np.linalg.norm(s.tris.reshape(-1, 3) - c, axis=1)
    # the grid distance to the nearest probe-accessible grid point overestimates by less than one cell diagonal
    assert rr.min() > r - 1e-9 and rr.max() < r + math.sqrt(3) * h
    topo = topology(s.edges, d)
    assert topo["manifold"] and topo["oriented"] and topo["chi"] == 2
    area, vol = mesh_stats(s.tris, s.edges)
    assert 4 * math.pi * r * r < area < 4 * math.pi * (r + h) ** 2
    assert 4 / 3 * math.pi * r ** 3 < vol < 4 / 3 * math.pi * (r + h) ** 3


def test_two_atoms_reentrant_surface_matches_the_analytic_ses():
    """Atoms 3.0 A apart (r 1.7, probe 1.4): every vertex within a cell diagonal of the exact SES, crevice filled."""
    r, p, zc, h = 1.7, 1.4, 1.5, 0.2
    x = np.array([[0, 0, zc, r], [0, 0, -zc, r]], np.float32)
    o, hh, d = oracle.ses_grid(x, probe=p, h=h)
    s = oracle.ses(x, o, hh, d, probe=p)
    V = s.tris.reshape(-1, 3)
    f = _analytic_two_atom_field(V, zc, r, p)
    assert np.abs(f).max() < math.sqrt(3) * h
    # the reentrant fill: in the plane z = 0 the surface lies at rho = sqrt((r+p)^2 - zc^2) - p, not at the
    # spheres' intersection circle sqrt(r^2 - zc^2)
    mid = np.abs(V[:, 2]) < 0.05
    rho = np.hypot(V[mid, 0], V[mid, 1])
    want = math.sqrt((r + p) ** 2 - zc ** 2) - p
    assert mid.sum() > 10 and np.abs(rho - want).max() < math.sqrt(3) * h
    assert want - math.sqrt(r * r - zc * zc) > 2.5 * h
    topo = topology(s.edges, d)
    assert topo["manifold"] and topo["oriented"] and topo["chi"] == 2


def test_probe_passes_between_distant_atoms():
    """Atoms 7 A apart with r + p = 3.1: two separate spheres (two components, Euler characteristic 4)."""
    x = np.array([[0, 0, 3.5, 1.7], [0, 0, -3.5, 1.7]], np.float32)
    o, h, d = oracle.ses_grid(x, probe=1.4, h=0.25)
    s = oracle.ses(x, o, h, d, probe=1.4)
    topo = topology(s.edges, d)
    assert topo["manifold"] and topo["oriented"] and topo["chi"] == 4
    V = s.tris.reshape(-1, 3)
    assert (np.abs(V[:, 2]) > 1.5).all()


def test_zero_probe_gives_the_union_of_spheres():
    """p = 0: the SES is the van der Waals surface; one atom gives its sphere (radius within one cell diagonal)."""
    r = 1.6
    x = np.array([[0.1, 0.2, -0.3, r]], np.float32)
    o, h, d = oracle.ses_grid(x, probe=0.0, h=0.2)
    s = oracle.ses(x, o, h, d, probe=0.0)
    rr = np.linalg.norm(s.tris.reshape(-1, 3) - x[0, :3].astype(np.float64), axis=1)
    assert len(s.tris) > 100 and rr.min() > r - math.sqrt(3) * h and rr.max() < r + math.sqrt(3) * h
    topo = topology(s.edges, d)
    assert topo["manifold"] and topo["oriented"] and topo["chi"] == 2
