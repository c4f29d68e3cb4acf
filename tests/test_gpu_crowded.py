"""Depth-crowded tiles: a near-flat sheet of atoms in front of a few far ones.

The far atoms stretch each tile's depth-key range, so the sheet's entries (depths within 0.05 A of each
other) land in one depth bucket of the tile's ordering.  The soft renderer must then finish its exact
(centre depth, id) order with its bitonic path, and the hard raster walks one crowded bucket; both must
still match the oracle.
"""
import numpy as np
import pytest

import oracle
from paper_2501_12750_gb300 import scenes

from helpers import compare, gpu_render


def sheet_scene(size=96):
    rng = np.random.default_rng(21)
    g = np.arange(20) * 1.5
    xx, yy = np.meshgrid(g, g)
    sheet = np.stack([xx.ravel(), yy.ravel(), rng.uniform(0.0, 0.05, xx.size)], 1)
    far = np.stack([rng.uniform(0.0, 28.5, 20), rng.uniform(0.0, 28.5, 20), np.full(20, -60.0)], 1)
    pos = np.concatenate([sheet, far])
    elem = scenes.draw_elements(rng, len(pos))
    c = np.array([14.25, 14.25, 0.0])
    cam = scenes.look_at(c + np.array([0.0, 0.0, 45.0]), c, size, size)
    return scenes.Scene("sheet", scenes.pack_xyzr(pos, elem), elem, [cam], ssao=False)


def max_sheet_entries_per_tile(s, dilate_px=4.0, tile=16):
    """Most sheet atoms whose (soft-dilated) projected box touches one 16x16 tile (FP64, on the CPU)."""
    cam = s.cameras[0]
    d = s.xyzr[:400, :3].astype(np.float64) - cam.eye.astype(np.float64)
    z = d @ cam.forward.astype(np.float64)
    f = cam.height / (2.0 * float(cam.tan_half_fovy))
    u = cam.width / 2 + f * (d @ cam.right.astype(np.float64)) / z
    v = cam.height / 2 - f * (d @ cam.up.astype(np.float64)) / z
    rad = f * s.xyzr[:400, 3].astype(np.float64) / z + dilate_px
    n = cam.width // tile
    best = 0
    for ty in range(n):
        for tx in range(n):
            hit = (u + rad >= tx * tile) & (u - rad <= (tx + 1) * tile) & (v + rad >= ty * tile) & \
                  (v - rad <= (ty + 1) * tile)
            best = max(best, int(hit.sum()))
    return best


def test_sheet_tiles_are_crowded():
    """The premise of the two tests below: far more sheet entries per tile than the 32 an insertion-sorted
    bucket takes, all within 0.05 A of depth against a 60 A key range."""
    assert max_sheet_entries_per_tile(sheet_scene()) > 64


@pytest.mark.gpu
def test_crowded_bucket_soft_forward_matches_oracle():
    import torch

    import paper_2501_12750_gb300 as vtx
    s = sheet_scene()
    r = vtx.Renderer()
    cov, dep, nrm = r.render_soft_fwd(torch.from_numpy(s.xyzr).cuda(), s.cameras)
    torch.cuda.synchronize()
    cov, dep, nrm = cov.cpu().numpy()[0], dep.cpu().numpy()[0], nrm.cpu().numpy()[0]
    cam = s.cameras[0]
    o = oracle.soft_forward(s.xyzr.astype(np.float64), cam, oracle.all_pixels(96, 96))
    ok = o.flags == 0
    assert ok.mean() > 0.9 and (o.A[ok] > 0.5).sum() > 500
    assert np.abs(cov.ravel()[ok] - o.A[ok]).max() <= 5e-5
    assert np.abs(dep.ravel()[ok] - o.D[ok]).max() <= 5e-5 * 45.0
    assert np.abs(nrm.reshape(3, -1).T[ok] - o.N[ok]).max() <= 5e-5


@pytest.mark.gpu
def test_crowded_bucket_hard_raster_matches_oracle():
    s = sheet_scene()
    res = gpu_render(s)
    h = oracle.render_pixels(s, 0, oracle.all_pixels(96, 96))
    st = compare(res, h, ssao=False, label="sheet")
    assert st["covered"] > 3000


def long_list_scene(n=6000, size=64):
    """n atoms in a 5 A cube seen from 35 A: every atom's soft-dilated footprint covers the central tiles."""
    rng = np.random.default_rng(23)
    pos = rng.uniform(0.0, 5.0, (n, 3))
    elem = scenes.draw_elements(rng, n)
    c = np.array([2.5, 2.5, 2.5])
    cam = scenes.look_at(c + np.array([0.0, 0.0, 35.0]), c, size, size)
    return scenes.Scene("long", scenes.pack_xyzr(pos, elem), elem, [cam], ssao=False)


def test_long_list_premise():
    """More than 4,096 soft entries in a tile: beyond what a tile orders in shared memory."""
    s = long_list_scene()
    cam = s.cameras[0]
    d = s.xyzr[:, :3].astype(np.float64) - cam.eye.astype(np.float64)
    z = d @ cam.forward.astype(np.float64)
    f = cam.height / (2.0 * float(cam.tan_half_fovy))
    u = cam.width / 2 + f * (d @ cam.right.astype(np.float64)) / z
    v = cam.height / 2 - f * (d @ cam.up.astype(np.float64)) / z
    rad = f * s.xyzr[:, 3].astype(np.float64) / z + 4.0
    hit = (u + rad >= 32) & (u - rad <= 48) & (v + rad >= 32) & (v - rad <= 48)  # tile (2, 2)
    assert hit.sum() > 4096


@pytest.mark.gpu
def test_soft_tile_lists_longer_than_shared_memory_match_oracle():
    """Tile lists of ~6,000 entries are ordered in global memory; forward and backward still match."""
    import torch

    import paper_2501_12750_gb300 as vtx
    s = long_list_scene()
    cam = s.cameras[0]
    r = vtx.Renderer()
    x = torch.from_numpy(s.xyzr).cuda()
    A, D, N = r.render_soft_fwd(x, [cam])
    pix = oracle.all_pixels(64, 64)
    x64 = s.xyzr.astype(np.float64)
    o = oracle.soft_forward(x64, cam, pix)
    ok = o.flags == 0
    assert ok.mean() > 0.9 and (o.A[ok] > 0.5).sum() > 50
    assert np.abs(A.cpu().numpy()[0].ravel()[ok] - o.A[ok]).max() <= 5e-5
    assert np.abs(D.cpu().numpy()[0].ravel()[ok] - o.D[ok]).max() <= 5e-5 * 35.0
    assert np.abs(N.cpu().numpy()[0].reshape(3, -1).T[ok] - o.N[ok]).max() <= 5e-5
    rng = np.random.default_rng(4)
    gA = np.where(ok, rng.normal(size=len(pix)), 0.0)
    gD = np.where(ok, 0.05 * rng.normal(size=len(pix)), 0.0)
    gN = np.where(ok[:, None], rng.normal(size=(len(pix), 3)), 0.0)
    ref = oracle.soft_vjp(x64, cam, pix, gA, gD, gN)
    g = r.render_soft_bwd(x, [cam], torch.from_numpy(gA.reshape(1, 64, 64).astype(np.float32)).cuda(),
                          torch.from_numpy(gD.reshape(1, 64, 64).astype(np.float32)).cuda(),
                          torch.from_numpy(gN.T.reshape(1, 3, 64, 64).astype(np.float32)).cuda())
    g = g.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(g - ref) <= 1e-4 * np.linalg.norm(ref)
    # the forward leaves the long list sorted in place; a backward reusing it skips the global sort
    r.render_soft_fwd(x, [cam])
    g2 = r.render_soft_bwd(x, [cam], torch.from_numpy(gA.reshape(1, 64, 64).astype(np.float32)).cuda(),
                           torch.from_numpy(gD.reshape(1, 64, 64).astype(np.float32)).cuda(),
                           torch.from_numpy(gN.T.reshape(1, 3, 64, 64).astype(np.float32)).cuda(), reuse_lists=True)
    g2 = g2.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(g2 - g) <= 1e-6 * np.linalg.norm(g)
