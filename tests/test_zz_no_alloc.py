"""The allocation-free visibility entry point against the regular frame renderer.

Some callers cannot allocate device memory: code running inside an
allocator or memory-pool callback, plug-ins of an application that owns
every device allocation, real-time loops that must avoid cudaMalloc's
implicit synchronisation.  vtx_render_visibility_static serves them from a
fixed file-scope device array.  Here it is called through the C ABI twice in
a row, on two different scenes and image sizes (so the second call also shows
that the shared array is cleared between calls), and its ids and depths are
compared with vtx_render_frame's (ids bit-exact, depth within 1e-5 relative)
and with the FP64 oracle's (ids outside its ambiguity bands, the parity
tests' depth tolerance with its near-silhouette conditioning term).  A close-up scene exercises
the candidate boxes that whole warps share.  This file is collected last.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2501_12750_gb300 import scenes

from helpers import DEPTH_RTOL, gpu_render, hit_tolerances

pytestmark = pytest.mark.gpu


def _static_render(scene):
    import torch

    import paper_2501_12750_gb300 as vtx
    lib = vtx.load()
    cam = scene.cameras[0]
    W, H = cam.width, cam.height
    xyzr = torch.from_numpy(np.ascontiguousarray(scene.xyzr)).cuda()
    depth = torch.full((H, W), -1.0, dtype=torch.float32, device="cuda")
    ids = torch.zeros((H, W), dtype=torch.int32, device="cuda")
    c = vtx.camera_struct(cam)
    stream = torch.cuda.current_stream()
    code = lib.vtx_render_visibility_static(xyzr.data_ptr(), xyzr.shape[0], ctypes.byref(c), depth.data_ptr(),
                                            ids.data_ptr(), ctypes.c_void_p(stream.cuda_stream))
    assert code == 0
    torch.cuda.synchronize()
    return depth.cpu().numpy(), ids.cpu().numpy().view(np.uint32)


def _check(scene):
    ref = gpu_render(scene)
    depth, ids = _static_render(scene)
    assert np.array_equal(ids, ref["id"])
    cov = ids != 0xFFFFFFFF
    assert cov.sum() > 500
    rel = np.abs(depth[cov].astype(np.float64) - ref["depth"][cov]) / ref["depth"][cov]
    assert rel.max() <= DEPTH_RTOL
    assert np.isinf(depth[~cov]).all()
    # and against the FP64 oracle directly: ids outside its ambiguity bands, depths within 1e-5 relative
    cam = scene.cameras[0]
    h = oracle.hits(scene.xyzr, cam, oracle.all_pixels(cam.width, cam.height))
    ok = (h.flags & oracle.ID_FLAGS) == 0
    assert ok.mean() > 0.99
    assert np.array_equal(ids.ravel()[ok], h.id[ok])
    hit = ok & (h.id != oracle.NO_ID)
    dtol, _ = hit_tolerances(h)
    assert (np.abs(depth.ravel()[hit].astype(np.float64) - h.depth[hit]) <= dtol[hit]).all()


def test_static_visibility_matches_render_frame_twice():
    _check(scenes.config1())  # 2,000 atoms at 256x256
    s = scenes.random_tiny(31, n=300, box=20.0, width=200, height=150, distance=30.0)
    _check(s)  # a second call, other scene and size, on the same static scratch


def test_static_visibility_close_spheres_share_a_warp():
    """Spheres a few radii from the eye: candidate boxes of thousands of pixels, ray-cast by whole warps."""
    s = scenes.random_tiny(32, n=200, box=12.0, width=320, height=240, distance=9.0)
    _check(s)


def test_static_visibility_rejects_a_non_finite_camera():
    import torch

    import paper_2501_12750_gb300 as vtx
    lib = vtx.load()
    s = scenes.config1()
    xyzr = torch.from_numpy(s.xyzr).cuda()
    buf = torch.empty(256 * 256, dtype=torch.float32, device="cuda")
    c = vtx.camera_struct(s.cameras[0])
    c.eye[1] = float("nan")
    assert lib.vtx_render_visibility_static(xyzr.data_ptr(), xyzr.shape[0], ctypes.byref(c), buf.data_ptr(),
                                            buf.data_ptr(), None) == 1  # VTX_ERR_INVALID_ARG
    c = vtx.camera_struct(s.cameras[0])
    c.tan_half_fovy = float("inf")
    assert lib.vtx_render_visibility_static(xyzr.data_ptr(), xyzr.shape[0], ctypes.byref(c), buf.data_ptr(),
                                            buf.data_ptr(), None) == 1


def test_static_visibility_rejects_oversized_images():
    import torch

    import paper_2501_12750_gb300 as vtx
    lib = vtx.load()
    s = scenes.config1()
    cam = scenes.look_at((20.0, 20.0, 140.0), (20.0, 20.0, 20.0), 2048, 1024)  # 2 Mpx > 1 Mpx limit
    xyzr = torch.from_numpy(s.xyzr).cuda()
    buf = torch.empty(16, dtype=torch.float32, device="cuda")
    c = vtx.camera_struct(cam)
    code = lib.vtx_render_visibility_static(xyzr.data_ptr(), xyzr.shape[0], ctypes.byref(c), buf.data_ptr(),
                                            buf.data_ptr(), None)
    assert code == 4  # VTX_ERR_CAPACITY
