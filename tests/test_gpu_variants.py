"""GPU parity of the representation, clipping, shading and post-processing variants against the FP64 oracle."""
import numpy as np
import pytest

import oracle
from paper_2501_12750_gb300 import scenes

from helpers import compare, gpu_render, sample_pixels

pytestmark = pytest.mark.gpu

# oracle keyword -> renderer setting
_SETTING = dict(model="shading", toon_levels="toon_levels", probe="probe_radius", clip="clip_plane",
                fog_near="fog_near", fog_far="fog_far", fog_density="fog_density", outline_depth="outline_depth",
                outline_color="outline_color")


def _both(scene, pix, kernel=None, tile=(16, 16), **kw):
    """GPU planes and oracle hits for the same variant settings (oracle keyword names)."""
    mode = kw.pop("mode", None)
    res = gpu_render(scene, ssao=kernel, mode=mode, tile=tile, **{_SETTING[k]: v for k, v in kw.items()})
    okw = dict(kw)
    if mode is not None:
        okw["mode"] = mode
    h = oracle.render_pixels(scene, 0, pix, kernel=kernel, **okw)
    return res, h


def _clear_plane(xyzr, n, d, margin=0.01):
    """Shift d until no atom centre lies within `margin` A of the plane n.X + d = 0."""
    n = np.asarray(n, np.float64) / np.linalg.norm(n)
    v = xyzr[:, :3].astype(np.float64) @ n
    while np.abs(v + d).min() < margin:
        d += 0.0037
    return np.array([n[0], n[1], n[2], d], np.float32)


def test_sas_config1_full_frame_with_ssao():
    s = scenes.config1()
    res, h = _both(s, oracle.all_pixels(256, 256), kernel=scenes.ssao_kernel(), mode=3, probe=1.4)
    st = compare(res, h, ssao=True, allow_excluded=0.0015, label="SAS")  # measured 10 of 8,798
    assert st["covered"] > 8000


def test_sas_random_tiny_probe_sizes():
    for seed, probe in [(3, 0.5), (4, 1.4), (5, 3.0)]:
        s = scenes.random_tiny(seed, n=50, width=61, height=47, distance=24.0)
        res, h = _both(s, oracle.all_pixels(61, 47), kernel=scenes.ssao_kernel(), mode=3, probe=probe)
        compare(res, h, ssao=True, allow_excluded=0.0025, label="SAS p=%g" % probe)  # at most 3 of 1,432


def test_sticks_close_view():
    """Sticks: an atom's sphere has the bond radius, so it meets its bonds' side surfaces at equal depth along
    whole pixel rows; those ties (and the SSAO samples that land on them) are excluded, hence the 4% allowance."""
    s3 = scenes.config3(n_clusters=4)
    s = scenes.config3_ball_and_stick(s3, n_clusters=4)
    c = s.xyzr[:5000, :3].astype(np.float64).mean(0)
    s.cameras = [scenes.look_at(c + np.array([0.0, 0.0, 45.0]), c, 256, 192)]
    k = scenes.ssao_kernel()
    res = gpu_render(s, ssao=k, mode=2)
    cov = res["id"] != oracle.NO_ID
    assert ((res["id"] >= s.xyzr.shape[0]) & cov).sum() > 500
    pix = sample_pixels(256, 192, 1000, 5, windows=[(120, 90, 20)], covered_mask=cov)
    h = oracle.render_pixels(s, 0, pix, kernel=k, mode=2)
    compare(res, h, ssao=True, allow_excluded=0.0025, label="sticks")  # measured 3 of 1,528


def test_clip_plane_vdw_full_frame():
    s = scenes.config1()
    plane = _clear_plane(s.xyzr, (1.0, 0.3, -0.2), -20.0)
    res, h = _both(s, oracle.all_pixels(256, 256), clip=plane)
    st = compare(res, h, ssao=False, label="clip")
    assert st["covered"] > 3000
    # nothing on the clipped side of the plane is ever the visible atom
    ids = res["id"][res["id"] != oracle.NO_ID]
    X = s.xyzr[ids, :3].astype(np.float64)
    assert (X @ plane[:3].astype(np.float64) + plane[3] >= 0).all()


def test_clip_plane_ball_and_stick_with_ssao():
    s3 = scenes.config3(n_clusters=4)
    s = scenes.config3_ball_and_stick(s3, n_clusters=4)
    c = s.xyzr[:5000, :3].astype(np.float64).mean(0)
    s.cameras = [scenes.look_at(c + np.array([0.0, 0.0, 60.0]), c, 240, 180)]
    plane = _clear_plane(s.xyzr, (0.0, 0.0, -1.0), c[2] + 2.0)
    k = scenes.ssao_kernel()
    res = gpu_render(s, ssao=k, clip_plane=plane)
    cov = res["id"] != oracle.NO_ID
    pix = sample_pixels(240, 180, 800, 9, windows=[(110, 80, 20)], covered_mask=cov)
    h = oracle.render_pixels(s, 0, pix, kernel=k, clip=plane)
    compare(res, h, ssao=True, label="clip b&s")


@pytest.mark.parametrize("model,levels", [(1, 4), (2, 4), (3, 2), (3, 4), (3, 7)])
def test_shading_models_config1(model, levels):
    s = scenes.config1()
    res, h = _both(s, oracle.all_pixels(256, 256), model=model, toon_levels=levels)
    compare(res, h, ssao=False, allow_excluded=0.0025, label="shading %d/%d" % (model, levels))  # toon band flags: at most 15 of 7,530


def test_toon_with_ssao_random_tiny():
    for seed in range(3):
        s = scenes.random_tiny(200 + seed, n=60, width=64, height=52, distance=18.0)
        res, h = _both(s, oracle.all_pixels(64, 52), kernel=scenes.ssao_kernel(), model=3, toon_levels=5)
        compare(res, h, ssao=True, allow_excluded=0.0035, label="toon tiny%d" % seed)  # at most 4 of 1,368


@pytest.mark.parametrize("density", [0.6, 1.0])
def test_fog_config1(density):
    s = scenes.config1()
    res, h = _both(s, oracle.all_pixels(256, 256), fog_near=105.0, fog_far=135.0, fog_density=density)
    compare(res, h, ssao=False, label="fog %g" % density)


def test_outline_config1_with_ssao():
    s = scenes.config1()
    res, h = _both(s, oracle.all_pixels(256, 256), kernel=scenes.ssao_kernel(), outline_depth=1.0,
                   outline_color=(0.1, 0.0, 0.3))
    st = compare(res, h, ssao=True, allow_excluded=0.0025, label="outline")  # measured 17 of 7,530
    col = np.array([0.1, 0.0, 0.3], np.float32)
    rgb = res["rgb"].transpose(1, 2, 0)
    outlined = np.all(rgb == col, axis=2)
    assert outlined.sum() > 1000 and st["covered"] - outlined.sum() > 3000


def test_all_variants_together_config2_sampled():
    """1e5 atoms at 1920x1080: SAS, clip plane, toon shading, SSAO, outline and fog in one frame."""
    s = scenes.config2()
    k = scenes.ssao_kernel()
    plane = _clear_plane(s.xyzr, (0.2, 1.0, 0.1), -80.0)
    kw = dict(mode=3, probe=1.4, clip=plane, model=3, toon_levels=4, outline_depth=2.0,
              outline_color=(0.0, 0.0, 0.0), fog_near=380.0, fog_far=470.0, fog_density=0.8)
    res = gpu_render(s, ssao=k, mode=3, **{_SETTING[key]: v for key, v in kw.items() if key != "mode"})
    cov = res["id"] != oracle.NO_ID
    assert cov.sum() > 50000
    ys, xs = np.nonzero(cov)
    cx, cy = int(xs.mean()), int(ys.mean())
    pix = sample_pixels(1920, 1080, 1200, 21, windows=[(cx - 16, cy - 16, 32), (xs.min(), cy, 24)],
                        covered_mask=cov)
    h = oracle.render_pixels(s, 0, pix, kernel=k, **kw)
    compare(res, h, ssao=True, allow_excluded=0.0025, label="config2 variants")  # 6 of 2,600


def test_batch_sas_clip_matches_per_frame():
    """The batched path takes the same representation, clip plane and post-processing bit for bit."""
    import torch

    import paper_2501_12750_gb300 as vtx
    s = scenes.config4(n=20000, n_frames=3, width=128, height=80)
    counts = [20000, 12000, 20000]
    k = scenes.ssao_kernel()
    plane = _clear_plane(s.frames[0], (0.0, 1.0, 0.0), -60.0)
    st = vtx.default_settings(ssao_kernel=k, mode=vtx.MODE_SAS, probe_radius=1.4, clip_plane=plane,
                              shading=vtx.SHADE_TOON, toon_levels=3, outline_depth=1.5, fog_near=100.0,
                              fog_far=400.0, fog_density=0.5, flags=vtx.FLAG_SYNC)
    r = vtx.Renderer()
    frames = torch.from_numpy(s.frames).cuda()
    elem = torch.from_numpy(s.elem).cuda()
    r.upload_atoms(frames[0], elem, s.palette)
    out = r.render_batch(frames, counts, s.cameras, st)
    torch.cuda.synchronize()
    b = {key: v.cpu().numpy() for key, v in out.items()}
    single = r.alloc_outputs(128, 80)
    V = len(s.cameras)
    for f in range(len(counts)):
        r.upload_atoms(frames[f, :counts[f]], elem[:counts[f]], s.palette)
        for v, cam in enumerate(s.cameras):
            r.set_camera(cam)
            r.render_frame(st, out=single)
            for key, t in single.items():
                assert np.array_equal(t.cpu().numpy(), b[key][f * V + v], equal_nan=True), (f, v, key)
