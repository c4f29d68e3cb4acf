"""GPU parity of the soft-edge renderer (forward, backward, autograd) against the FP64 oracle and FD.

Tolerances (derived from FP32 arithmetic over at most a few hundred
contributors per pixel; the paper gives none for this form):
  forward   |dA| <= 5e-5, |dN| <= 5e-5 per component, |dD| <= 5e-5 * camera distance;
  backward  relative L2 over all atoms <= 1e-4 against the oracle's analytic FP64 VJP,
            per component |dg| <= 1e-3 |g| + 1e-4 max|g| against FP64 central differences.
Pixels the oracle flags (contributor within 1e-6 px of the -4 px cutoff,
centre depths within 1e-6 A, transmittance at the stop threshold, opacity at
the 0.99 clamp) are excluded from the forward comparison and get a zero
upstream gradient in the backward comparison.
"""
import numpy as np
import pytest

import oracle
from paper_2501_12750_gb300 import scenes

pytestmark = pytest.mark.gpu

A_TOL = 5e-5
N_TOL = 5e-5
D_TOL_REL = 5e-5


def small_scene(n=2000, size=96, views=4, seed=5):
    """A reduced config-5 system viewed from 1.5 box edges (atoms a few pixels wide)."""
    s = scenes.config5(seed=seed, n=n, size=size)
    L = scenes.box_edge(n)
    c = np.array([L / 2] * 3)
    s.cameras = [scenes.orbit_camera(c, 1.5 * L, az, el, size, size)
                 for az, el in [(0, -15), (90, 15), (180, 45), (270, -45)][:views]]
    return s


def gpu_soft(s, sigma=0.5):
    import torch

    import paper_2501_12750_gb300 as vtx
    r = vtx.Renderer()
    x = torch.from_numpy(s.xyzr).cuda()
    cov, dep, nrm = r.render_soft_fwd(x, s.cameras, sigma)
    torch.cuda.synchronize()
    return r, x, cov.cpu().numpy(), dep.cpu().numpy(), nrm.cpu().numpy()


def test_soft_forward_parity():
    s = small_scene()
    _, _, cov, dep, nrm = gpu_soft(s)
    W = H = 96
    pix = oracle.all_pixels(W, H)
    D = float(np.linalg.norm(s.cameras[0].eye - s.xyzr[:, :3].mean(0)))
    for v, cam in enumerate(s.cameras):
        o = oracle.soft_forward(s.xyzr.astype(np.float64), cam, pix)
        ok = o.flags == 0
        assert ok.mean() > 0.97
        a = cov[v].ravel()
        assert np.abs(a[ok] - o.A[ok]).max() <= A_TOL
        assert np.abs(dep[v].ravel()[ok] - o.D[ok]).max() <= D_TOL_REL * D
        n = nrm[v].reshape(3, -1).T
        assert np.abs(n[ok] - o.N[ok]).max() <= N_TOL
        assert (o.A[ok] > 0.5).sum() > 500


def test_soft_backward_matches_oracle_vjp():
    import torch
    s = small_scene(n=1500, size=80, views=3, seed=9)
    r, x, cov, dep, nrm = gpu_soft(s)
    W = H = 80
    pix = oracle.all_pixels(W, H)
    rng = np.random.default_rng(3)
    V = len(s.cameras)
    gA = rng.normal(size=(V, H, W))
    gD = rng.normal(size=(V, H, W)) * 0.05
    gN = rng.normal(size=(V, 3, H, W))
    ref = np.zeros((s.xyzr.shape[0], 4))
    x64 = s.xyzr.astype(np.float64)
    for v, cam in enumerate(s.cameras):
        o = oracle.soft_forward(x64, cam, pix)
        bad = (o.flags != 0).reshape(H, W)
        gA[v][bad] = 0.0
        gD[v][bad] = 0.0
        gN[v][:, bad] = 0.0
        ref += oracle.soft_vjp(x64, cam, pix, gA[v].ravel(), gD[v].ravel(), gN[v].reshape(3, -1).T)
    g = r.render_soft_bwd(x, s.cameras, torch.from_numpy(gA.astype(np.float32)).cuda(),
                          torch.from_numpy(gD.astype(np.float32)).cuda(),
                          torch.from_numpy(gN.astype(np.float32)).cuda()).cpu().numpy().astype(np.float64)
    rel = np.linalg.norm(g - ref) / np.linalg.norm(ref)
    assert rel <= 1e-4, rel
    assert np.abs(ref).max() > 1e-2


def test_soft_autograd_matches_explicit_backward():
    import torch

    import paper_2501_12750_gb300 as vtx
    s = small_scene(n=800, size=64, views=2, seed=11)
    r = vtx.Renderer()
    x = torch.from_numpy(s.xyzr).cuda().requires_grad_(True)
    t = torch.from_numpy(s.extra["target"][:800].copy()).cuda()
    with torch.no_grad():
        At, Dt, Nt = r.render_soft_fwd(t, s.cameras)
    A, D, N = vtx.SoftRender.apply(x, r, s.cameras, 0.5)
    loss = ((A - At) ** 2).mean() + 0.1 * ((D - Dt) ** 2).mean() + ((N - Nt) ** 2).sum(1).mean()
    loss.backward()
    npx = A.numel()
    gA = 2 * (A.detach() - At) / npx
    gD = 0.2 * (D.detach() - Dt) / npx
    gN = 2 * (N.detach() - Nt) / npx
    g2 = r.render_soft_bwd(x.detach(), s.cameras, gA, gD, gN)
    torch.testing.assert_close(x.grad, g2, rtol=1e-5, atol=1e-9)
    assert float(x.grad.abs().sum()) > 0


def _footprint(cam, xyzr_row, margin_px=6.0):
    """Pixels within the atom's dilated projected box (a superset of those it can affect)."""
    W, H = cam.width, cam.height
    d = xyzr_row[:3].astype(np.float64) - cam.eye.astype(np.float64)
    z = float(d @ cam.forward.astype(np.float64))
    f = H / (2.0 * float(cam.tan_half_fovy))
    x = W / 2 + f * float(d @ cam.right.astype(np.float64)) / z
    y = H / 2 - f * float(d @ cam.up.astype(np.float64)) / z
    rad = f * float(xyzr_row[3]) / z * 1.2 + margin_px
    x0, x1 = max(0, int(x - rad)), min(W - 1, int(x + rad) + 1)
    y0, y1 = max(0, int(y - rad)), min(H - 1, int(y + rad) + 1)
    if x0 > x1 or y0 > y1:
        return np.zeros((0, 2), np.int32)
    yy, xx = np.mgrid[y0:y1 + 1, x0:x1 + 1]
    return np.stack([xx.ravel(), yy.ravel()], 1).astype(np.int32)


def test_soft_config5_fd_on_sampled_atoms():
    """Full config 5 (20,000 atoms, 16 views, 512x512) with the L2 loss against the perturbed target:
    GPU backward vs FP64 central differences (h = 1e-4 A) on sampled atoms."""
    import torch

    import paper_2501_12750_gb300 as vtx
    s = scenes.config5()
    r = vtx.Renderer()
    x = torch.from_numpy(s.xyzr).cuda()
    t = torch.from_numpy(s.extra["target"]).cuda()
    At, Dt, Nt = r.render_soft_fwd(t, s.cameras)
    A, D, N = r.render_soft_fwd(x, s.cameras)
    npx = A.numel()
    gA = (2 * (A - At) / npx).contiguous()
    gD = (0.2 * (D - Dt) / npx).contiguous()
    gN = (2 * (N - Nt) / npx).contiguous()
    g = r.render_soft_bwd(x, s.cameras, gA, gD, gN).cpu().numpy().astype(np.float64)
    gA_, gD_, gN_ = gA.cpu().numpy(), gD.cpu().numpy(), gN.cpu().numpy()
    gmax = np.abs(g).max()
    x64 = s.xyzr.astype(np.float64)
    h = 1e-4
    checked = 0
    for i in s.extra["fd_order"]:
        if checked >= 8:
            break
        fps = [(v, cam, _footprint(cam, s.xyzr[i])) for v, cam in enumerate(s.cameras)]
        fps = [(v, cam, p) for v, cam, p in fps if len(p)]
        if not fps:
            continue
        if np.abs(g[i]).max() < 1e-3 * gmax:
            continue
        fd = np.zeros(4)
        smooth = True
        for k in range(4):
            val = []
            for sgn in (+1, -1):
                xx = x64.copy()
                xx[i, k] += sgn * h
                tot = 0.0
                used = []
                for v, cam, p in fps:
                    o = oracle.soft_forward(xx, cam, p)
                    tot += (gA_[v][p[:, 1], p[:, 0]] * o.A).sum() + (gD_[v][p[:, 1], p[:, 0]] * o.D).sum()
                    tot += (gN_[v][:, p[:, 1], p[:, 0]].T * o.N).sum()
                    used.append(o.n_used)
                val.append((tot, used))
            if any(not np.array_equal(a, b) for a, b in zip(val[0][1], val[1][1])):
                smooth = False
                break
            fd[k] = (val[0][0] - val[1][0]) / (2 * h)
        if not smooth:
            continue
        err = np.abs(g[i] - fd)
        assert (err <= 1e-3 * np.abs(fd) + 1e-4 * gmax).all(), (i, g[i], fd)
        checked += 1
    assert checked >= 4
