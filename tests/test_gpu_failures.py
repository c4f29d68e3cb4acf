"""Failure detection without a GPU fault: each error path is driven by a host-side hook.

- A bounded device wait that runs out: the multi-view cull gives its first bulk-copy wait zero polls
  (its drain of the copies in flight keeps the normal limit, so no CTA exits with a copy pending); the
  status word reports VTX_ERR_TIMEOUT and the next frame, with the hook off, is correct.
- A scratch arena too small: forced capacities make the binning overflow; the kernels stop writing at the
  capacity, VTX_ERR_CAPACITY is reported once, the arena grows and the re-render is bit-identical.
- A bounds check: a host memset overwrites one depth key with an out-of-range primitive id after the tile
  ray-cast; the resolve draws that pixel as background and VTX_ERR_BOUNDS is reported.
"""
import numpy as np
import pytest

from paper_2501_12750_gb300 import scenes

pytestmark = pytest.mark.gpu

TIMEOUT, CAPACITY, BOUNDS = 5, 4, 6


def _planes(out):
    return {k: v.cpu().numpy() for k, v in out.items()}


def _same(a, b):
    for k in a:
        assert np.array_equal(a[k], b[k], equal_nan=True), k


def test_bounded_wait_timeout_is_reported_and_recovered():
    import torch

    import paper_2501_12750_gb300 as vtx
    s = scenes.config2(n=20000, width=320, height=240)
    c = s.xyzr[:, :3].astype(np.float64).mean(0)
    # six views: more than the barrier-free batch cull takes, so the bulk-copy cull (with its waits) runs
    cams = [scenes.orbit_camera(c, 150.0, az, 10.0, 320, 240) for az in (0.0, 60.0, 120.0, 180.0, 240.0, 300.0)]
    frames = torch.from_numpy(s.xyzr[None].copy()).cuda()
    r = vtx.Renderer()
    r.upload_atoms(frames[0], torch.from_numpy(s.elem).cuda(), s.palette)
    sync = vtx.default_settings(flags=vtx.FLAG_SYNC)
    ref = _planes(r.render_batch(frames, [s.xyzr.shape[0]], cams, sync))
    r.debug_hooks(first_wait_polls=0)
    with pytest.raises(vtx.VtxError) as e:
        r.render_batch(frames, [s.xyzr.shape[0]], cams, sync)
    assert e.value.code == TIMEOUT
    # asynchronous form: the call succeeds, the next synchronisation reports the timeout once
    r.render_batch(frames, [s.xyzr.shape[0]], cams, vtx.default_settings())
    with pytest.raises(vtx.VtxError) as e:
        r.sync_status()
    assert e.value.code == TIMEOUT
    r.sync_status()  # reported once
    r.debug_hooks(first_wait_polls=-1)
    _same(_planes(r.render_batch(frames, [s.xyzr.shape[0]], cams, sync)), ref)


def test_soft_path_timeout_is_reported():
    import torch

    import paper_2501_12750_gb300 as vtx
    s = scenes.config5(n=3000, size=96)
    r = vtx.Renderer()
    x = torch.from_numpy(s.xyzr).cuda()
    ref = [t.cpu().numpy() for t in r.render_soft_fwd(x, s.cameras[:4])]
    r.debug_hooks(first_wait_polls=0)
    with pytest.raises(vtx.VtxError) as e:
        r.render_soft_fwd(x, s.cameras[:4])
    assert e.value.code == TIMEOUT
    r.debug_hooks(first_wait_polls=-1)
    got = [t.cpu().numpy() for t in r.render_soft_fwd(x, s.cameras[:4])]
    for a, b in zip(got, ref):
        assert np.array_equal(a, b)


def test_forced_capacity_overflow_then_identical_rerender():
    import torch

    import paper_2501_12750_gb300 as vtx
    s = scenes.config2(n=30000, width=480, height=270)
    k = scenes.ssao_kernel()
    ref_r = vtx.Renderer()
    ref_r.upload_atoms(torch.from_numpy(s.xyzr).cuda(), torch.from_numpy(s.elem).cuda(), s.palette)
    ref_r.set_camera(s.cameras[0])
    # splat_max_px = 1 bins every primitive whose candidate box exceeds one pixel, so the records and tile
    # entries that the hook limits are needed
    ref = _planes(ref_r.render_frame(vtx.default_settings(ssao_kernel=k, splat_max_px=1, flags=vtx.FLAG_SYNC),
                                     width=480, height=270))
    r = vtx.Renderer()
    r.upload_atoms(torch.from_numpy(s.xyzr).cuda(), torch.from_numpy(s.elem).cuda(), s.palette)
    r.set_camera(s.cameras[0])
    r.debug_hooks(cap_records=64, cap_entries=256)
    out = r.render_frame(vtx.default_settings(ssao_kernel=k, splat_max_px=1), width=480, height=270)
    with pytest.raises(vtx.VtxError) as e:
        r.sync_status()
    assert e.value.code == CAPACITY
    out = r.render_frame(vtx.default_settings(ssao_kernel=k, splat_max_px=1), out=out)
    r.sync_status()  # the grown arena holds the frame
    _same(_planes(out), ref)
    assert (ref["id"] != -1).sum() > 2000


def test_corrupted_key_hits_the_bounds_check():
    import torch

    import paper_2501_12750_gb300 as vtx
    s = scenes.config1()
    r = vtx.Renderer()
    r.upload_atoms(torch.from_numpy(s.xyzr).cuda(), torch.from_numpy(s.elem).cuda(), s.palette)
    r.set_camera(s.cameras[0])
    sync = vtx.default_settings(flags=vtx.FLAG_SYNC)
    ref = _planes(r.render_frame(sync, width=256, height=256))
    r.debug_hooks(corrupt_key=True)
    out = r.render_frame(vtx.default_settings(), width=256, height=256)
    with pytest.raises(vtx.VtxError) as e:
        r.sync_status()
    assert e.value.code == BOUNDS
    got = _planes(out)
    assert got["id"][0, 0] == -1 and np.isinf(got["depth"][0, 0])  # drawn as background
    r.debug_hooks(corrupt_key=False)
    _same(_planes(r.render_frame(sync, out=out)), ref)
