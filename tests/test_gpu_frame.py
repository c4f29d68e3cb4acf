"""GPU parity of the hard-edge frame renderer (through the C ABI) against the FP64 oracle."""
import numpy as np
import pytest

import oracle
from paper_2501_12750_gb300 import scenes

from helpers import compare, gpu_render, sample_pixels

pytestmark = pytest.mark.gpu


def test_config1_full_frame():
    """2,000 atoms, 256x256, no SSAO: every pixel against the brute-force oracle."""
    s = scenes.config1()
    res = gpu_render(s)
    h = oracle.render_pixels(s, 0, oracle.all_pixels(256, 256))
    st = compare(res, h, ssao=False, label="config1")
    assert st["covered"] > 5000


@pytest.mark.parametrize("tile,splat", [((16, 16), 16), ((32, 8), 0), ((8, 8), 0), ((16, 16), 1000000)])
def test_ragged_sizes_tiles_and_paths(tile, splat):
    """Odd image sizes (ragged last tiles), each tile shape, binned-only and splat-only paths."""
    s = scenes.config1()
    cam = s.cameras[0]
    cam = scenes.look_at((20.0, 20.0, 75.0), (20.0, 20.0, 20.0), 203, 141)
    s.cameras = [cam]
    res = gpu_render(s, tile=tile, splat_max=splat, ssao=scenes.ssao_kernel())
    h = oracle.render_pixels(s, 0, oracle.all_pixels(203, 141), kernel=scenes.ssao_kernel())
    compare(res, h, ssao=True, label="ragged %s splat %d" % (tile, splat))


@pytest.mark.parametrize("seed", range(12))
def test_random_tiny_scenes(seed):
    """Random small scenes, random orbit views, SSAO on; includes edge-of-screen primitives."""
    s = scenes.random_tiny(1000 + seed, n=60, width=72 + seed, height=50 + 2 * seed, distance=14.0 + seed)
    res = gpu_render(s, ssao=scenes.ssao_kernel())
    h = oracle.render_pixels(s, 0, oracle.all_pixels(s.cameras[0].width, s.cameras[0].height),
                             kernel=scenes.ssao_kernel())
    # 1,100-2,500 covered pixels: 0-4 of them flagged (measured at most 0.21 %)
    compare(res, h, ssao=True, allow_excluded=0.0025, label="tiny%d" % seed)


def test_near_plane_and_eye_inside():
    """Spheres cut by the near plane, one enclosing the eye, one behind it."""
    cam = scenes.look_at((0.0, 0.0, 1.0), (0.0, 0.0, 0.0), 97, 81, fovy_deg=90.0)
    # front pole of the first sphere at depth 0.03 (< near 0.05), its rim beyond the near plane;
    # the eye lies inside the second; the third is behind the eye
    xyzr = np.array([[0, 0, 0, 0.97], [0.3, 0.1, 1.0, 0.5], [0, 0, 3.0, 1.0], [-0.6, -0.3, -1.0, 0.4]],
                    np.float32)
    s = scenes.Scene("near", xyzr, np.array([0, 1, 2, 3], np.uint8), [cam], ssao=False)
    res = gpu_render(s)
    h = oracle.render_pixels(s, 0, oracle.all_pixels(97, 81))
    compare(res, h, ssao=False, label="near")


def test_empty_and_all_culled():
    s = scenes.config1()
    s.xyzr = s.xyzr[:0].copy()
    s.elem = s.elem[:0].copy()
    res = gpu_render(s)
    assert (res["id"] == oracle.NO_ID).all() and np.isinf(res["depth"]).all()
    np.testing.assert_array_equal(res["rgb"], 1.0)
    s = scenes.config1()
    s.cameras = [scenes.look_at((20.0, 20.0, 140.0), (20.0, 20.0, 300.0), 64, 64)]  # looking away
    res = gpu_render(s)
    assert (res["id"] == oracle.NO_ID).all()


def test_config2_full_size_sampled_with_ssao():
    """100,000 atoms at 1920x1080 with SSAO: random covered pixels and full windows vs the oracle."""
    s = scenes.config2()
    k = scenes.ssao_kernel()
    res = gpu_render(s, ssao=k)
    cov = res["id"] != oracle.NO_ID
    assert cov.sum() > 50000
    ys, xs = np.nonzero(cov)
    cx, cy = int(xs.mean()), int(ys.mean())
    pix = sample_pixels(1920, 1080, 1500, 7, windows=[(cx - 24, cy - 24, 48), (xs.min(), cy, 32)],
                        covered_mask=cov)
    h = oracle.render_pixels(s, 0, pix, kernel=k)
    st = compare(res, h, ssao=True, label="config2")
    assert st["covered"] > 1500


def test_config3_full_size_sampled():
    """The benchmark frame itself: 1e8 atoms, 3840x2160, SSAO, overview view V1; sampled pixels vs the oracle."""
    s = scenes.config3()
    k = scenes.ssao_kernel()
    res = gpu_render(s, ssao=k)
    cov = res["id"] != oracle.NO_ID
    assert cov.sum() > 50000
    ys, xs = np.nonzero(cov)
    j = len(xs) // 2
    pix = sample_pixels(3840, 2160, 240, 11, windows=[(xs[j] - 6, ys[j] - 6, 12)], covered_mask=cov)
    h = oracle.render_pixels(s, 0, pix, kernel=k)
    st = compare(res, h, ssao=True, label="config3 V1")
    assert st["covered"] > 150


def test_ball_and_stick_subset():
    """Ball-and-stick (0.4 A balls, 0.15 A bonds under 1.9 A) on four whole-cell blobs, close view."""
    s3 = scenes.config3(n_clusters=4)
    s = scenes.config3_ball_and_stick(s3, n_clusters=4)
    c = s.xyzr[:5000, :3].astype(np.float64).mean(0)
    cam = scenes.look_at(c + np.array([0.0, 0.0, 60.0]), c, 320, 240)
    s.cameras = [cam]
    k = scenes.ssao_kernel()
    res = gpu_render(s, ssao=k)
    assert ((res["id"] >= s.xyzr.shape[0]) & (res["id"] != oracle.NO_ID)).sum() > 500  # bonds visible
    pix = sample_pixels(320, 240, 1200, 3, windows=[(150, 110, 24)], covered_mask=res["id"] != oracle.NO_ID)
    h = oracle.render_pixels(s, 0, pix, kernel=k)
    compare(res, h, ssao=True, allow_excluded=0.0015, label="ball-and-stick")  # measured 2 of 1,799


def test_permutation_relabels_ids():
    s = scenes.random_tiny(77, n=80, width=64, height=48)
    perm = np.random.default_rng(1).permutation(80)
    r0 = gpu_render(s)
    s2 = scenes.Scene("p", s.xyzr[perm].copy(), s.elem[perm].copy(), s.cameras, ssao=False)
    r1 = gpu_render(s2)
    m = r1["id"] != oracle.NO_ID
    mapped = r1["id"].copy()
    mapped[m] = perm[r1["id"][m]]
    h = oracle.hits(s.xyzr, s.cameras[0], oracle.all_pixels(64, 48))
    ok = ((h.flags & oracle.ID_FLAGS) == 0).reshape(48, 64)
    assert np.array_equal(mapped[ok], r0["id"][ok])


def test_autotuner_choice_and_config_independence():
    """tile_w = 0 autotunes; every tile shape / splat threshold gives bit-identical planes."""
    import torch

    import paper_2501_12750_gb300 as vtx
    s = scenes.config2(n=30000, width=640, height=360)
    k = scenes.ssao_kernel()
    r = vtx.Renderer()
    r.upload_atoms(torch.from_numpy(s.xyzr).cuda(), torch.from_numpy(s.elem).cuda(), s.palette)
    r.set_camera(s.cameras[0])
    outs = {}
    auto = r.render_frame(vtx.default_settings(ssao_kernel=k, tile_w=0, tile_h=0, flags=vtx.FLAG_SYNC),
                          width=640, height=360)
    tw, th, sp = r.tuned_settings()
    assert (tw, th) in [(16, 16), (32, 8), (8, 8)] and sp in (4, 16, 64)
    outs["auto"] = {key: v.cpu().numpy() for key, v in auto.items()}
    for tile in [(16, 16), (32, 8), (8, 8)]:
        for splat in (0, 4, 64):
            o = r.render_frame(vtx.default_settings(ssao_kernel=k, tile_w=tile[0], tile_h=tile[1],
                                                    splat_max_px=splat, flags=vtx.FLAG_SYNC), width=640, height=360)
            outs[(tile, splat)] = {key: v.cpu().numpy() for key, v in o.items()}
    ref = outs["auto"]
    assert (ref["id"] != -1).sum() > 5000
    for name, o in outs.items():
        for key in ref:
            assert np.array_equal(o[key], ref[key], equal_nan=True), (name, key)
