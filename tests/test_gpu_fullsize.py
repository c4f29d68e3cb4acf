"""Full-size parity on the benchmark workloads that the other GPU tests only cover at reduced size.

Each case renders at the configuration's full size in the launch configuration
bench.py uses, then compares sampled pixels (random covered pixels, random
pixels and a full window) with the FP64 oracle, which ray-casts them one by
one by brute force over every primitive.
"""
import numpy as np
import pytest

import oracle
from paper_2501_12750_gb300 import scenes

from helpers import compare, gpu_render, sample_pixels

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cell():
    return scenes.config3()


def test_config3_close_view_v2(cell):
    """1e8 atoms seen from 600 A outside the cube face: large, deeply overlapping impostors (binned path).

    Ids, depths and normals on random pixels; shading and SSAO on one window (SSAO samples fetch
    pixels ~6 px away here, each of which the oracle must ray-cast against all 1e8 atoms).
    """
    k = scenes.ssao_kernel()
    res = gpu_render(cell, cam_index=1, ssao=k)
    cov = res["id"] != oracle.NO_ID
    assert cov.mean() > 0.2
    pix = sample_pixels(3840, 2160, 60, 21, covered_mask=cov)
    h = oracle.hits(cell.xyzr, cell.cameras[1], pix)
    st = compare(res, h, ssao=False, label="config3 V2 hits", colour=False)
    assert st["covered"] > 60
    win = sample_pixels(3840, 2160, 0, 22, windows=[(1917, 1077, 6)])
    hw = oracle.render_pixels(cell, 1, win, kernel=k)
    compare(res, hw, ssao=True, label="config3 V2 window")


def test_config3_ball_and_stick_full_subset(cell):
    """5e6 atoms (0.4 A balls) and their ~2.6e7 bonds (0.15 A cylinders) from 80 A, no SSAO."""
    s = scenes.config3_ball_and_stick(cell, n_clusters=1000)
    assert 2.3e7 < s.bonds.shape[0] < 2.9e7
    # a camera 80 A in front of the first blob, which is fully inside the subset
    c = cell.extra["centres"][0]
    s.cameras = [scenes.look_at(c + np.array([0.0, 0.0, 80.0]), c, 3840, 2160)]
    res = gpu_render(s)
    ids = res["id"]
    bonds_seen = ((ids >= s.xyzr.shape[0]) & (ids != oracle.NO_ID)).sum()
    assert bonds_seen > 10000
    pix = sample_pixels(3840, 2160, 50, 23, windows=[(1910, 1070, 8)], covered_mask=ids != oracle.NO_ID)
    h = oracle.render_pixels(s, 0, pix)
    compare(res, h, ssao=False, label="ball-and-stick 5e6")


def test_config4_full_batch_sampled():
    """All 1,024 images (500k atoms x 256 frames x 4 views, 1280x720, SSAO) in one graph launch.

    Every image has ~500k survivors on ~5 % of its pixels, so the batch takes its exact occlusion pass (a
    survivor is dropped when FP32 upper bounds of the nearest depth, written by the front survivors, lie in
    front of it at every pixel of its box): three images are compared bit for bit with the per-frame renderer, which has no occlusion pass, and
    sampled pixels of the same images with the FP64 oracle."""
    import torch

    import paper_2501_12750_gb300 as vtx
    s = scenes.config4()
    k = scenes.ssao_kernel()
    r = vtx.Renderer()
    frames = torch.from_numpy(s.frames).cuda()
    r.upload_atoms(frames[0], torch.from_numpy(s.elem).cuda(), s.palette)
    F, N = s.frames.shape[0], s.frames.shape[1]
    counts = [N] * F
    out = r.render_batch(frames, counts, s.cameras, vtx.default_settings(ssao_kernel=k, flags=vtx.FLAG_SYNC))
    out = r.render_batch(frames, counts, s.cameras, vtx.default_settings(ssao_kernel=k), out=out, use_graph=True)
    torch.cuda.synchronize()
    r.sync_status()
    V = len(s.cameras)
    for f, v in [(0, 0), (128, 1), (255, 3)]:
        img = f * V + v
        res = {key: val[img].cpu().numpy() for key, val in out.items()}
        res["id"] = res["id"].view(np.uint32)
        one = vtx.Renderer()
        one.upload_atoms(frames[f], torch.from_numpy(s.elem).cuda(), s.palette)
        one.set_camera(s.cameras[v])
        single = one.render_frame(vtx.default_settings(ssao_kernel=k, flags=vtx.FLAG_SYNC), width=1280, height=720)
        for key, val in single.items():
            a = val.cpu().numpy()
            if key == "id":
                a = a.view(np.uint32)
            assert np.array_equal(a, res[key], equal_nan=True), (img, key)
        del one, single
        sc = scenes.Scene("f%d" % f, np.ascontiguousarray(s.frames[f]), s.elem, [s.cameras[v]], ssao=True)
        cov = res["id"] != oracle.NO_ID
        pix = sample_pixels(1280, 720, 150, img, windows=[(630, 350, 12)], covered_mask=cov)
        h = oracle.render_pixels(sc, 0, pix, kernel=k)
        compare(res, h, ssao=True, label="config4 img %d" % img)
