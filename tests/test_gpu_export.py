"""GPU checks of the headless RGBA8 export, up to 8K (7680 x 4320)."""
import numpy as np
import pytest

import oracle
from paper_2501_12750_gb300 import scenes

from helpers import sample_pixels

pytestmark = pytest.mark.gpu


def quantise(rgb_planes, ids, bg_alpha):
    """The export's definition on the GPU's own FP32 planes: clamp, x255 in FP32, round half to even."""
    v = np.clip(rgb_planes.astype(np.float32), np.float32(0), np.float32(1)) * np.float32(255)
    rgb = np.rint(v).astype(np.uint8)
    rgb = np.moveaxis(rgb, -3, -1)
    a = np.where(ids.view(np.uint32) == oracle.NO_ID, np.uint8(np.rint(np.float32(255) * np.float32(bg_alpha))),
                 np.uint8(255))
    return np.concatenate([rgb, a[..., None]], axis=-1)


def test_export_8k_bit_exact_alpha_and_oracle(tmp_path):
    import torch

    import paper_2501_12750_gb300 as vtx
    from paper_2501_12750_gb300.export import write_png
    from test_export_png import decode_png
    s = scenes.config2(width=7680, height=4320)
    k = scenes.ssao_kernel()
    r = vtx.Renderer()
    r.upload_atoms(torch.from_numpy(s.xyzr).cuda(), torch.from_numpy(s.elem).cuda(), s.palette)
    cam = s.cameras[0]
    r.set_camera(cam)
    out = r.render_frame(vtx.default_settings(ssao_kernel=k, flags=vtx.FLAG_SYNC), width=7680, height=4320)
    rgba = r.export_rgba8(out, background_alpha=0.25).cpu().numpy()
    planes = {key: v.cpu().numpy() for key, v in out.items()}
    assert rgba.shape == (4320, 7680, 4)
    np.testing.assert_array_equal(rgba, quantise(planes["rgb"], planes["id"], 0.25))
    cov = planes["id"].view(np.uint32) != oracle.NO_ID
    assert cov.sum() > 200000 and (rgba[..., 3][~cov] == 64).all() and (rgba[..., 3][cov] == 255).all()
    # the same bytes written straight into a page-locked host buffer
    host = torch.empty((4320, 7680, 4), dtype=torch.uint8).pin_memory()
    r.export_rgba8(out, background_alpha=0.25, rgba=host)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(host.numpy(), rgba)
    # against the oracle on sampled pixels: bytes of the FP64 colour within the float tolerance (2/255) + rounding
    pix = sample_pixels(7680, 4320, 300, 13, covered_mask=cov)
    h = oracle.render_pixels(s, 0, pix, kernel=k)
    ok = ((h.flags & (oracle.ID_FLAGS | oracle.FLAG_SPLIT | oracle.FLAG_GRID | oracle.FLAG_MARGIN |
                      oracle.FLAG_FETCH | oracle.FLAG_SILH)) == 0)
    ref = np.rint(np.clip(h.rgb_final, 0.0, 1.0) * 255.0)
    got = rgba[pix[:, 1], pix[:, 0], :3].astype(np.float64)
    assert ok.sum() > 250
    assert np.abs(got[ok] - ref[ok]).max() <= 3
    alpha_ref = np.where(h.id == oracle.NO_ID, 64, 255)
    amb = (h.flags & oracle.ID_FLAGS) != 0
    np.testing.assert_array_equal(rgba[pix[:, 1], pix[:, 0], 3][~amb], alpha_ref[~amb])
    # the PNG file decodes to the same image (a 1024 x 768 crop around the molecule)
    ys, xs = np.nonzero(cov)
    y0, x0 = max(0, int(ys.mean()) - 384), max(0, int(xs.mean()) - 512)
    crop = rgba[y0:y0 + 768, x0:x0 + 1024]
    p = tmp_path / "frame.png"
    write_png(str(p), crop)
    np.testing.assert_array_equal(decode_png(p.read_bytes()), crop)


def test_export_batch_images():
    import torch

    import paper_2501_12750_gb300 as vtx
    s = scenes.config4(n=20000, n_frames=3, width=160, height=96)
    r = vtx.Renderer()
    frames = torch.from_numpy(s.frames).cuda()
    r.upload_atoms(frames[0], torch.from_numpy(s.elem).cuda(), s.palette)
    out = r.render_batch(frames, [20000, 20000, 5000], s.cameras,
                         vtx.default_settings(ssao_kernel=scenes.ssao_kernel(), flags=vtx.FLAG_SYNC))
    rgba = r.export_rgba8(out, background_alpha=1.0).cpu().numpy()
    assert rgba.shape == (12, 96, 160, 4)
    planes = {key: v.cpu().numpy() for key, v in out.items()}
    np.testing.assert_array_equal(rgba, quantise(planes["rgb"], planes["id"], 1.0))
    assert (rgba[..., 3] == 255).all()
