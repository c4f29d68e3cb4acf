"""Atoms in page-locked host memory: streamed by the kernels over the host link, bit-exact with device memory.

This is the out-of-core form of the renderer: device memory holds only per-pixel and per-survivor state, so
the atom count is bounded by host memory (several hundred million atoms below).
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2501_12750_gb300 import scenes

from helpers import compare, sample_pixels

pytestmark = pytest.mark.gpu


def _planes(out):
    res = {k: v.cpu().numpy() for k, v in out.items()}
    res["id"] = res["id"].view(np.uint32)
    return res


def _render(r, s, xyzr, elem, settings, bonds=None, cam_index=0):
    r.upload_atoms(xyzr, elem, s.palette)
    if bonds is not None:
        r.upload_bonds(bonds)
    cam = s.cameras[cam_index]
    r.set_camera(cam)
    return _planes(r.render_frame(settings, width=cam.width, height=cam.height))


def _same(a, b, label):
    for k in a:
        assert np.array_equal(a[k], b[k], equal_nan=True), (label, k)


def test_host_resident_bit_exact_config2_with_ssao():
    import torch

    import paper_2501_12750_gb300 as vtx
    s = scenes.config2()
    st = vtx.default_settings(ssao_kernel=scenes.ssao_kernel(), flags=vtx.FLAG_SYNC)
    r = vtx.Renderer()
    dev = _render(r, s, torch.from_numpy(s.xyzr).cuda(), torch.from_numpy(s.elem).cuda(), st)
    host = _render(r, s, torch.from_numpy(s.xyzr).pin_memory(), torch.from_numpy(s.elem).pin_memory(), st)
    assert (dev["id"] != oracle.NO_ID).sum() > 50000
    _same(dev, host, "config2")


def test_host_resident_ball_and_stick_bonds_on_host():
    import torch

    import paper_2501_12750_gb300 as vtx
    s3 = scenes.config3(n_clusters=4)
    s = scenes.config3_ball_and_stick(s3, n_clusters=4)
    c = s.xyzr[:5000, :3].astype(np.float64).mean(0)
    s.cameras = [scenes.look_at(c + np.array([0.0, 0.0, 60.0]), c, 320, 240)]
    st = vtx.default_settings(ssao_kernel=scenes.ssao_kernel(), mode=vtx.MODE_BALL_AND_STICK, flags=vtx.FLAG_SYNC)
    b = torch.from_numpy(s.bonds.astype(np.int32))
    r = vtx.Renderer()
    dev = _render(r, s, torch.from_numpy(s.xyzr).cuda(), torch.from_numpy(s.elem).cuda(), st, bonds=b.cuda())
    host = _render(r, s, torch.from_numpy(s.xyzr).pin_memory(), torch.from_numpy(s.elem).pin_memory(), st,
                   bonds=b.pin_memory())
    assert ((dev["id"] >= s.xyzr.shape[0]) & (dev["id"] != oracle.NO_ID)).sum() > 500
    _same(dev, host, "ball-and-stick")


def test_host_resident_trajectory_batch():
    import torch

    import paper_2501_12750_gb300 as vtx
    s = scenes.config4(n=20000, n_frames=5, width=160, height=96)
    counts = [20000, 9000, 20000, 1, 17000]
    st = vtx.default_settings(ssao_kernel=scenes.ssao_kernel(), flags=vtx.FLAG_SYNC)
    r = vtx.Renderer()
    elem = torch.from_numpy(s.elem).cuda()
    fd = torch.from_numpy(s.frames).cuda()
    fh = torch.from_numpy(s.frames).pin_memory()
    r.upload_atoms(fd[0], elem, s.palette)
    a = _planes(r.render_batch(fd, counts, s.cameras, st))
    b = _planes(r.render_batch(fh, counts, s.cameras, st))
    g = _planes(r.render_batch(fh, counts, s.cameras, vtx.default_settings(ssao_kernel=scenes.ssao_kernel()),
                               use_graph=True))
    torch.cuda.synchronize()
    _same(a, b, "batch")
    _same(a, g, "batch graph")


def test_pageable_host_memory_is_refused():
    import paper_2501_12750_gb300 as vtx
    r = vtx.Renderer()
    x = np.zeros((64, 4), np.float32)  # ordinary (pageable) host memory, 16-byte aligned by numpy
    assert x.ctypes.data % 16 == 0
    pal = np.ascontiguousarray(scenes.PALETTE, np.float32)
    code = r.lib.vtx_upload_atoms(r.ctx, x.ctypes.data, None, pal.ctypes.data, pal.shape[0], 64)
    assert code == 1  # VTX_ERR_INVALID_ARG, before any launch
    assert b"page-locked" in r.lib.vtx_last_error(r.ctx)
    p = np.zeros((4, 2), np.uint32)
    assert r.lib.vtx_upload_bonds(r.ctx, p.ctypes.data, 4) == 1


def test_three_hundred_million_atoms_streamed_from_host():
    """3e8 atoms (60,000 whole-cell blobs, 4.8 GB) in page-locked host memory, 3840x2160 overview, no SSAO."""
    import time

    import torch

    import paper_2501_12750_gb300 as vtx
    s = scenes.config3(n_clusters=60000)
    assert s.xyzr.shape[0] == 300_000_000
    xh = torch.from_numpy(s.xyzr).pin_memory()
    eh = torch.from_numpy(s.elem).pin_memory()
    r = vtx.Renderer()
    r.upload_atoms(xh, eh, s.palette)
    cam = s.cameras[0]
    r.set_camera(cam)
    out = r.render_frame(vtx.default_settings(flags=vtx.FLAG_SYNC), width=cam.width, height=cam.height)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    r.render_frame(vtx.default_settings(), out=out)
    torch.cuda.synchronize()
    print("3e8 host-resident atoms: %.1f ms per frame" % (1e3 * (time.perf_counter() - t0)))
    res = _planes(out)
    cov = res["id"] != oracle.NO_ID
    assert cov.sum() > 200000
    pix = sample_pixels(cam.width, cam.height, 32, 5, covered_mask=cov)
    h = oracle.render_pixels(s, 0, pix)
    compare(res, h, ssao=False, label="3e8 host")


def test_output_planes_in_page_locked_host_memory():
    """vtx_render_frame writes straight into page-locked host planes: identical to device planes."""
    import torch

    import paper_2501_12750_gb300 as vtx
    s = scenes.config2(n=30000, width=640, height=360)
    st = vtx.default_settings(ssao_kernel=scenes.ssao_kernel(), outline_depth=1.0, flags=vtx.FLAG_SYNC)
    r = vtx.Renderer()
    r.upload_atoms(torch.from_numpy(s.xyzr).pin_memory(), torch.from_numpy(s.elem).pin_memory(), s.palette)
    r.set_camera(s.cameras[0])
    dev = r.render_frame(st, width=640, height=360)
    host = {k: torch.empty_like(v, device="cpu").pin_memory() for k, v in dev.items()}
    r.render_frame(st, out=host)
    torch.cuda.synchronize()
    a, b = _planes(dev), _planes(host)
    assert (a["id"] != oracle.NO_ID).sum() > 5000
    _same(a, b, "host outputs")
    # pageable output planes are refused before any launch
    bad = {k: np.zeros(tuple(v.shape), np.float32) for k, v in dev.items()}
    o = vtx.VtxOutputs(*(bad[k].ctypes.data for k in ("depth", "id", "normal", "rgb", "ao")))
    assert r.lib.vtx_render_frame(r.ctx, ctypes.byref(st), ctypes.byref(o)) == 1
