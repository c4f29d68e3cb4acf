"""GPU parity of the solvent excluded surface (grid SAS, windowed distance transform, marching cubes).

The SAS decision, the distance transform and the marching-cubes structure (cells, loops, vertex labels and
their order) are integer or exactly-rounded FP64 decisions on both sides, so they must match bit for bit;
vertex positions are FP32 on the GPU and FP64 in the oracle.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2501_12750_gb300 import scenes

pytestmark = pytest.mark.gpu

VERTEX_ATOL = 2e-4  # A: FP32 grid coordinates (|X| <= ~200 A) and interpolation


def gpu_ses(xyzr, origin, h, dims, probe):
    import torch

    import paper_2501_12750_gb300 as vtx
    r = vtx.Renderer()
    x = torch.from_numpy(np.ascontiguousarray(xyzr, np.float32)).cuda()
    g = vtx.Renderer.ses_grid(origin, h, dims, probe)
    out = r.ses_mesh(x, g, labels=True, planes=True)
    torch.cuda.synchronize()
    return dict(tris=out["tris"].cpu().numpy().astype(np.float64), labels=out["labels"].cpu().numpy(),
                sas=out["sas"].cpu().numpy(), edt2=out["edt2"].cpu().numpy().view(np.uint16), n=out["n"])


def check_same(g, o, label):
    np.testing.assert_array_equal(g["sas"], o.sas, err_msg=label + " sas")
    np.testing.assert_array_equal(g["edt2"], o.edt2, err_msg=label + " edt2")
    assert g["n"] == len(o.tris), (label, g["n"], len(o.tris))
    np.testing.assert_array_equal(g["labels"], o.edges, err_msg=label + " labels")
    err = np.abs(g["tris"] - o.tris).max() if len(o.tris) else 0.0
    assert err <= VERTEX_ATOL, (label, err)


@pytest.mark.parametrize("case", ["one", "two", "apart", "random"])
def test_ses_small_cases_bit_exact(case):
    if case == "one":
        x = np.array([[0.3, -0.2, 0.1, 1.7]], np.float32)
    elif case == "two":
        x = np.array([[0, 0, 1.5, 1.7], [0, 0, -1.5, 1.7]], np.float32)
    elif case == "apart":
        x = np.array([[0, 0, 3.5, 1.7], [0, 0, -3.5, 1.52]], np.float32)
    else:
        rng = np.random.default_rng(9)
        x = np.concatenate([rng.uniform(0, 9, (40, 3)), rng.uniform(1.2, 1.9, (40, 1))], 1).astype(np.float32)
    for h in (0.5, 0.3):
        o, hh, d = oracle.ses_grid(x, probe=1.4, h=h)
        ref = oracle.ses(x, o, hh, d, probe=1.4)
        check_same(gpu_ses(x, o, hh, d, 1.4), ref, "%s h=%g" % (case, h))


def test_ses_probe_sizes_and_offsets():
    """Other probe radii, a non-dyadic spacing and an origin off any grid of the atoms."""
    rng = np.random.default_rng(10)
    x = np.concatenate([rng.uniform(-5, 5, (25, 3)), rng.uniform(1.0, 2.0, (25, 1))], 1).astype(np.float32)
    for p, h in [(0.0, 0.37), (0.6, 0.41), (3.0, 0.55)]:
        o, hh, d = oracle.ses_grid(x, probe=p, h=h)
        o = o + np.float32(0.0123)
        ref = oracle.ses(x, o, hh, d, probe=p)
        assert len(ref.tris) > 1000
        check_same(gpu_ses(x, o, hh, d, p), ref, "p=%g h=%g" % (p, h))


def test_ses_protein_chain_bit_exact():
    """1,200 atoms of the protein-like generator (a 150-residue chain) at 0.6 A spacing."""
    s = scenes.config2(n=1200)
    o, h, d = oracle.ses_grid(s.xyzr, probe=1.4, h=0.6)
    ref = oracle.ses(s.xyzr, o, h, d, probe=1.4)
    assert len(ref.tris) > 10000
    check_same(gpu_ses(s.xyzr, o, h, d, 1.4), ref, "chain")


def test_ses_config2_full_size_window_and_topology():
    """1e5 atoms, 0.5 A spacing on the library's fitted grid: a window against the oracle, and the whole
    surface closed, oriented and manifold."""
    import torch

    import paper_2501_12750_gb300 as vtx
    from test_ses_oracle import topology
    s = scenes.config2()
    r = vtx.Renderer()
    x = torch.from_numpy(s.xyzr).cuda()
    g = r.ses_fit_grid(x, probe=1.4, spacing=0.5)
    dims = np.array(g.dims[:], np.int32)
    origin = np.array(g.origin[:], np.float32)
    out = r.ses_mesh(x, g, labels=True, planes=True)
    torch.cuda.synchronize()
    T = out["n"]
    labels = out["labels"].cpu().numpy()
    edt_all = out["edt2"].cpu().numpy().view(np.uint16)
    sas_all = out["sas"].cpu().numpy()
    assert T > 1_000_000
    topo = topology(labels, dims)
    assert topo["manifold"] and topo["oriented"] and topo["chi"] % 2 == 0
    tris = out["tris"].cpu().numpy().astype(np.float64)
    vol = np.einsum("ij,ij->i", tris[:, 0], np.cross(tris[:, 1], tris[:, 2])).sum() / 6.0
    assert vol > 0
    # window: 28^3 points centred on a surface cell, with a margin of K + 1 points on every side
    K = int(oracle.lib().orc_ses_k(np.float32(1.4), np.float32(0.5)))
    cell = labels[T // 2, 0] // 16
    nx, ny, nz = (int(v) for v in dims)
    ci, cj, ck = cell % (nx - 1), (cell // (nx - 1)) % (ny - 1), cell // ((nx - 1) * (ny - 1))
    m = K + 1
    w = 28
    lo = np.array([ci, cj, ck]) - w // 2 - m
    lo = np.maximum(lo, 0)
    hi = np.minimum(lo + w + 2 * m, dims)
    sub_dims = (hi - lo).astype(np.int32)
    hsp = np.float32(0.5)
    # atoms that can reach the sub-grid (test-side prefilter: farther ones cannot touch a point of it)
    pmin = origin.astype(np.float64) + 0.5 * lo - 4.0
    pmax = origin.astype(np.float64) + 0.5 * (hi - 1) + 4.0
    near = np.all((s.xyzr[:, :3] >= pmin) & (s.xyzr[:, :3] <= pmax), axis=1)
    ref = oracle.ses(s.xyzr[near], origin, hsp, sub_dims, probe=1.4, offset=lo.astype(np.int32))
    sl = (slice(lo[2], hi[2]), slice(lo[1], hi[1]), slice(lo[0], hi[0]))
    np.testing.assert_array_equal(sas_all[sl], ref.sas)
    inner = (slice(m, -m),) * 3
    np.testing.assert_array_equal(edt_all[sl][inner], ref.edt2[inner])
    # triangles of the cells whose 8 corners are inner points, in the same (cell-major) order
    sdx, sdy = int(sub_dims[0]), int(sub_dims[1])
    oc = ref.edges // 16
    oi, oj, ok = oc % (sdx - 1), (oc // (sdx - 1)) % (sdy - 1), oc // ((sdx - 1) * (sdy - 1))
    keep_o = ((oi >= m) & (oi < sub_dims[0] - 1 - m) & (oj >= m) & (oj < sub_dims[1] - 1 - m) &
              (ok >= m) & (ok < sub_dims[2] - 1 - m))[:, 0]
    glob = ((ok + lo[2]) * (ny - 1) + (oj + lo[1])) * (nx - 1) + (oi + lo[0])
    want_labels = glob * 16 + ref.edges % 16
    gc = labels // 16
    gi, gj, gk = gc % (nx - 1), (gc // (nx - 1)) % (ny - 1), gc // ((nx - 1) * (ny - 1))
    keep_g = ((gi >= lo[0] + m) & (gi < hi[0] - 1 - m) & (gj >= lo[1] + m) & (gj < hi[1] - 1 - m) &
              (gk >= lo[2] + m) & (gk < hi[2] - 1 - m))[:, 0]
    assert keep_o.sum() > 100
    np.testing.assert_array_equal(labels[keep_g], want_labels[keep_o])
    err = np.abs(tris[keep_g] - ref.tris[keep_o]).max()
    assert err <= VERTEX_ATOL, err


def test_ses_capacity_and_host_outputs():
    import torch

    import paper_2501_12750_gb300 as vtx
    x = np.array([[0, 0, 1.5, 1.7], [0, 0, -1.5, 1.7]], np.float32)
    o, h, d = oracle.ses_grid(x, probe=1.4, h=0.4)
    r = vtx.Renderer()
    xd = torch.from_numpy(x).cuda()
    g = vtx.Renderer.ses_grid(o, h, d, 1.4)
    full = r.ses_mesh(xd, g)
    n = full["n"]
    small = torch.empty((10, 3, 3), dtype=torch.float32, device="cuda")
    import ctypes
    cnt = ctypes.c_int64(0)
    code = r.lib.vtx_ses_mesh(r.ctx, xd.data_ptr(), 2, ctypes.byref(g), small.data_ptr(), 10, None, None, None,
                              ctypes.byref(cnt))
    assert code == 4 and cnt.value == n  # VTX_ERR_CAPACITY with the needed count
    np.testing.assert_array_equal(small.cpu().numpy(), full["tris"][:10].cpu().numpy())
    host = torch.empty((n, 3, 3), dtype=torch.float32).pin_memory()
    code = r.lib.vtx_ses_mesh(r.ctx, xd.data_ptr(), 2, ctypes.byref(g), host.data_ptr(), n, None, None, None,
                              ctypes.byref(cnt))
    assert code == 0
    np.testing.assert_array_equal(host.numpy(), full["tris"].cpu().numpy())
    assert math.isfinite(float(host.numpy().sum()))
