"""GPU checks of the batched trajectory renderer: bit-exact against the per-frame path, graph replay, oracle."""
import numpy as np
import pytest

import oracle
from paper_2501_12750_gb300 import scenes

from helpers import compare, sample_pixels

pytestmark = pytest.mark.gpu


def _small_traj():
    s = scenes.config4(n=20000, n_frames=6, width=160, height=96)
    counts = [20000, 15000, 20000, 7000, 20000, 1]
    return s, counts


def _np(out):
    res = {k: v.cpu().numpy() for k, v in out.items()}
    res["id"] = res["id"].view(np.uint32)
    return res


def test_batch_bit_exact_with_per_frame_and_graph():
    import torch

    import paper_2501_12750_gb300 as vtx
    s, counts = _small_traj()
    k = scenes.ssao_kernel()
    r = vtx.Renderer()
    frames = torch.from_numpy(s.frames).cuda()
    elem = torch.from_numpy(s.elem).cuda()
    r.upload_atoms(frames[0], elem, s.palette)
    st = vtx.default_settings(ssao_kernel=k, flags=vtx.FLAG_SYNC)
    out = r.render_batch(frames, counts, s.cameras, st)
    gout = r.render_batch(frames, counts, s.cameras, vtx.default_settings(ssao_kernel=k), use_graph=True)
    gout2 = r.render_batch(frames, counts, s.cameras, vtx.default_settings(ssao_kernel=k), out=gout, use_graph=True)
    torch.cuda.synchronize()
    r.sync_status()
    b = _np(out)
    g = _np(gout2)
    for key in b:
        assert np.array_equal(b[key], g[key], equal_nan=True), key
    V = len(s.cameras)
    single = r.alloc_outputs(160, 96)
    for f in range(len(counts)):
        r.upload_atoms(frames[f, :counts[f]], elem[:counts[f]], s.palette)
        for v, cam in enumerate(s.cameras):
            r.set_camera(cam)
            r.render_frame(st, out=single)
            one = _np(single)
            img = f * V + v
            for key in one:
                assert np.array_equal(one[key], b[key][img], equal_nan=True), (f, v, key)


def test_batch_images_match_oracle():
    import torch

    import paper_2501_12750_gb300 as vtx
    s, counts = _small_traj()
    k = scenes.ssao_kernel()
    r = vtx.Renderer()
    frames = torch.from_numpy(s.frames).cuda()
    r.upload_atoms(frames[0], torch.from_numpy(s.elem).cuda(), s.palette)
    out = _np(r.render_batch(frames, counts, s.cameras, vtx.default_settings(ssao_kernel=k, flags=vtx.FLAG_SYNC)))
    V = len(s.cameras)
    for f, v in [(0, 0), (3, 2), (5, 1), (4, 3)]:
        img = f * V + v
        sc = scenes.Scene("f%d" % f, np.ascontiguousarray(s.frames[f, :counts[f]]), s.elem[:counts[f]],
                          [s.cameras[v]], ssao=True)
        res = {key: out[key][img] for key in out}
        cov = res["id"] != oracle.NO_ID
        pix = sample_pixels(160, 96, 300, img, windows=[(70, 40, 16)], covered_mask=cov if cov.any() else None)
        h = oracle.render_pixels(sc, 0, pix, kernel=k)
        compare(res, h, ssao=True, label="batch img %d" % img)


@pytest.mark.parametrize("n_views", [1, 2, 3, 5])
def test_batch_view_counts_bit_exact_with_per_frame(n_views):
    """Batches of one to three views take the barrier-free multi-view cull with that many views per atom, five
    views the bulk-copy cull; every image equals the per-frame renderer's, plane for plane."""
    import torch

    import paper_2501_12750_gb300 as vtx
    s, counts = _small_traj()
    c = np.array([scenes.box_edge(20000) / 2] * 3)
    cams = [scenes.orbit_camera(c, 3.0 * scenes.box_edge(20000), 360.0 * v / n_views + 10.0, 20.0 * v - 15.0, 160, 96)
            for v in range(n_views)]
    k = scenes.ssao_kernel()
    r = vtx.Renderer()
    frames = torch.from_numpy(s.frames).cuda()
    elem = torch.from_numpy(s.elem).cuda()
    r.upload_atoms(frames[0], elem, s.palette)
    st = vtx.default_settings(ssao_kernel=k, flags=vtx.FLAG_SYNC)
    b = _np(r.render_batch(frames, counts, cams, st))
    single = r.alloc_outputs(160, 96)
    for f in (0, 3, 5):
        r.upload_atoms(frames[f, :counts[f]], elem[:counts[f]], s.palette)
        for v, cam in enumerate(cams):
            r.set_camera(cam)
            r.render_frame(st, out=single)
            one = _np(single)
            for key in one:
                assert np.array_equal(one[key], b[key][f * n_views + v], equal_nan=True), (n_views, f, v, key)
    assert (b["id"] != oracle.NO_ID).sum() > 1000


def test_batch_sas_close_clipped_bit_exact_with_per_frame():
    """SAS radii, one camera close to the system (spheres cut by the near plane and boxes wider than the
    occlusion pass writes or tests) and a clip plane through the middle: the batch, whose crowded images take
    the occlusion pass, equals the per-frame renderer image for image, plane for plane."""
    import torch

    import paper_2501_12750_gb300 as vtx
    s, counts = _small_traj()
    L = scenes.box_edge(20000)
    c = np.array([L / 2] * 3)
    cams = [scenes.orbit_camera(c, 0.6 * L, 30.0, 10.0, 160, 96),
            scenes.orbit_camera(c, 1.4 * L, 200.0, -20.0, 160, 96)]
    k = scenes.ssao_kernel()
    r = vtx.Renderer()
    frames = torch.from_numpy(s.frames).cuda()
    elem = torch.from_numpy(s.elem).cuda()
    r.upload_atoms(frames[0], elem, s.palette)
    st = vtx.default_settings(ssao_kernel=k, flags=vtx.FLAG_SYNC, mode=vtx.MODE_SAS, probe_radius=1.4,
                              clip_plane=(1.0, 0.0, 0.0, -float(c[0])))
    b = _np(r.render_batch(frames, counts, cams, st))
    single = r.alloc_outputs(160, 96)
    for f in (0, 2, 3):
        r.upload_atoms(frames[f, :counts[f]], elem[:counts[f]], s.palette)
        for v, cam in enumerate(cams):
            r.set_camera(cam)
            r.render_frame(st, out=single)
            one = _np(single)
            for key in one:
                assert np.array_equal(one[key], b[key][f * len(cams) + v], equal_nan=True), (f, v, key)
    for v in range(len(cams)):
        assert (b["id"][v] != oracle.NO_ID).sum() > 500, v
