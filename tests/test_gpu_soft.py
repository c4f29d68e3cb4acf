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

from helpers import soft_candidates

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
    """Bounding box (x0, y0, x1, y1) of the pixels an atom can affect in a view (its dilated projected disc
    plus a margin), or None when it is off screen or behind the eye."""
    W, H = cam.width, cam.height
    d = xyzr_row[:3].astype(np.float64) - cam.eye.astype(np.float64)
    z = float(d @ cam.forward.astype(np.float64))
    if z <= float(cam.znear):
        return None
    f = H / (2.0 * float(cam.tan_half_fovy))
    x = W / 2 + f * float(d @ cam.right.astype(np.float64)) / z
    y = H / 2 - f * float(d @ cam.up.astype(np.float64)) / z
    rad = 1.3 * (f * float(xyzr_row[3]) / z + 4.0) + margin_px
    x0, x1 = max(0, int(x - rad)), min(W - 1, int(x + rad) + 1)
    y0, y1 = max(0, int(y - rad)), min(H - 1, int(y + rad) + 1)
    if x0 > x1 or y0 > y1:
        return None
    return x0, y0, x1, y1


def _box_pixels(b):
    x0, y0, x1, y1 = b
    yy, xx = np.mgrid[y0:y1 + 1, x0:x1 + 1]
    return np.ascontiguousarray(np.stack([xx.ravel(), yy.ravel()], 1).astype(np.int32))


@pytest.fixture(scope="module")
def config5_run():
    """The full soft-renderer configuration (20,000 atoms, 16 views at 512x512) with the L2 loss against
    the perturbed target: GPU forward planes, the loss's upstream gradients and the GPU backward."""
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
    out = dict(s=s, r=r, x=x, A=A.cpu().numpy(), D=D.cpu().numpy(), N=N.cpu().numpy(), gA=gA.cpu().numpy(),
               gD=gD.cpu().numpy(), gN=gN.cpu().numpy(), g=g, gA_t=gA, gD_t=gD, gN_t=gN)
    return out


def test_soft_config5_forward_on_sampled_pixels(config5_run):
    """Forward parity on 4,096 random pixels of each of the 16 views of the full configuration."""
    s = config5_run["s"]
    x64 = s.xyzr.astype(np.float64)
    D0 = float(np.linalg.norm(s.cameras[0].eye - s.xyzr[:, :3].mean(0)))
    rng = np.random.default_rng(55)
    n_ok = n_cov = 0
    for v, cam in enumerate(s.cameras):
        pix = np.ascontiguousarray(np.stack([rng.integers(0, 512, 4096), rng.integers(0, 512, 4096)], 1)
                                   .astype(np.int32))
        o = oracle.soft_forward(x64, cam, pix)
        ok = o.flags == 0
        a = config5_run["A"][v][pix[:, 1], pix[:, 0]]
        d = config5_run["D"][v][pix[:, 1], pix[:, 0]]
        n = config5_run["N"][v][:, pix[:, 1], pix[:, 0]].T
        assert np.abs(a[ok] - o.A[ok]).max() <= A_TOL
        assert np.abs(d[ok] - o.D[ok]).max() <= D_TOL_REL * D0
        assert np.abs(n[ok] - o.N[ok]).max() <= N_TOL
        n_ok += int(ok.sum())
        n_cov += int((o.A[ok] > 0.5).sum())
    assert n_ok >= 0.98 * 16 * 4096
    assert n_cov > 5000


def test_soft_config5_backward_matches_oracle_vjp(config5_run):
    """The GPU backward on the full configuration against the oracle's analytic FP64 VJP over all 20,000
    atoms: the upstream gradient is the loss's, kept on 4,096 seeded pixels per view (zero elsewhere and at
    the pixels the oracle flags), so the oracle evaluates those pixels only."""
    import torch
    s, r, x = config5_run["s"], config5_run["r"], config5_run["x"]
    x64 = s.xyzr.astype(np.float64)
    rng = np.random.default_rng(56)
    V, H, W = config5_run["A"].shape
    gA = np.zeros((V, H, W))
    gD = np.zeros((V, H, W))
    gN = np.zeros((V, 3, H, W))
    ref = np.zeros((x64.shape[0], 4))
    for v, cam in enumerate(s.cameras):
        lin = np.unique(rng.integers(0, H * W, 4096))
        pix = np.ascontiguousarray(np.stack([lin % W, lin // W], 1).astype(np.int32))
        o = oracle.soft_forward(x64, cam, pix)
        keep = o.flags == 0
        pix = pix[keep]
        py, px = pix[:, 1], pix[:, 0]
        gA[v][py, px] = config5_run["gA"][v][py, px]
        gD[v][py, px] = config5_run["gD"][v][py, px]
        gN[v][:, py, px] = config5_run["gN"][v][:, py, px]
        ref += oracle.soft_vjp(x64, cam, pix, gA[v][py, px], gD[v][py, px], gN[v][:, py, px].T)
    g = r.render_soft_bwd(x, s.cameras, torch.from_numpy(gA.astype(np.float32)).cuda(),
                          torch.from_numpy(gD.astype(np.float32)).cuda(),
                          torch.from_numpy(gN.astype(np.float32)).cuda()).cpu().numpy().astype(np.float64)
    rel = np.linalg.norm(g - ref) / np.linalg.norm(ref)
    assert rel <= 1e-4, rel
    assert (np.abs(ref).max(1) > 0).sum() > 5000  # most atoms receive a gradient


def test_soft_config5_fd_on_200_sampled_atoms(config5_run):
    """Full configuration, L2 loss against the perturbed target: the GPU backward against FP64 central
    differences (h = 1e-4 A on x, y, z and r) on 200 seeded atoms with non-zero gradient.

    An atom whose +-h evaluations are not smooth is resampled and counted: a contributor count that
    changes at some pixel (the -4 px cutoff or the transmittance stop crossed), its opacity reaching the
    0.99 clamp at some pixel on one side only (the oracle rendering that atom alone, whose coverage is its
    opacity), or another candidate within 2h of its centre depth that contributes with it at some pixel
    (their order can swap).  The oracle is given, per view, only the atoms that can reach the atom's
    footprint (helpers.soft_candidates, which leaves its outputs unchanged)."""
    s = config5_run["s"]
    g = config5_run["g"]
    gA_, gD_, gN_ = config5_run["gA"], config5_run["gD"], config5_run["gN"]
    gmax = np.abs(g).max()
    x64 = s.xyzr.astype(np.float64)
    h = 1e-4
    checked, skipped, tried = 0, 0, 0
    worst = 0.0
    for i in s.extra["fd_order"]:
        if checked >= 200:
            break
        if np.abs(g[i]).max() < 1e-3 * gmax:
            continue
        tried += 1
        views = []
        smooth = True
        for v, cam in enumerate(s.cameras):
            b = _footprint(cam, s.xyzr[i])
            if b is None:
                continue
            cand = soft_candidates(x64, cam, (b[0], b[1]), (b[2], b[3]))
            if i not in cand:
                continue
            pix = _box_pixels(b)
            # a contributor whose centre depth is within 2h of the atom's can swap places with it; that
            # matters where both contribute (the pair rendered alone composites both at some pixel)
            zc = (x64[cand, :3] - cam.eye.astype(np.float64)) @ cam.forward.astype(np.float64)
            zi = float((x64[i, :3] - cam.eye.astype(np.float64)) @ cam.forward.astype(np.float64))
            for j in cand[(np.abs(zc - zi) < 2 * h) & (cand != i)]:
                pair = x64[np.sort([i, j])]
                if (oracle.soft_forward(pair, cam, pix).n_used == 2).any():
                    smooth = False
            if not smooth:
                break
            views.append((v, cam, pix, cand, int(np.nonzero(cand == i)[0][0])))
        if not smooth or not views:
            skipped += int(not smooth)
            continue
        fd = np.zeros(4)
        for k in range(4):
            val = []
            for sgn in (+1, -1):
                tot = 0.0
                used, solo = [], []
                for v, cam, pix, cand, li in views:
                    xx = x64[cand].copy()
                    xx[li, k] += sgn * h
                    o = oracle.soft_forward(xx, cam, pix)
                    py, px = pix[:, 1], pix[:, 0]
                    tot += (gA_[v][py, px] * o.A).sum() + (gD_[v][py, px] * o.D).sum()
                    tot += (gN_[v][:, py, px].T * o.N).sum()
                    used.append(o.n_used)
                    # the atom alone: its coverage is its opacity, so 0.99 marks the clamp
                    solo.append(oracle.soft_forward(xx[li:li + 1], cam, pix).A == 0.99)
                val.append((tot, used, solo))
            if any(not np.array_equal(a, b) for a, b in zip(val[0][1], val[1][1])) or \
                    any(not np.array_equal(a, b) for a, b in zip(val[0][2], val[1][2])):
                smooth = False
                break
            fd[k] = (val[0][0] - val[1][0]) / (2 * h)
        if not smooth:
            skipped += 1
            continue
        err = np.abs(g[i] - fd)
        assert (err <= 1e-3 * np.abs(fd) + 1e-4 * gmax).all(), (i, g[i], fd)
        worst = max(worst, float((err / (1e-3 * np.abs(fd) + 1e-4 * gmax)).max()))
        checked += 1
    print("soft FD: %d atoms checked, %d resampled as non-smooth, worst error / tolerance %.3f"
          % (checked, skipped, worst))
    assert checked == 200, (checked, skipped, tried)
    assert skipped <= checked  # non-smooth atoms stay a minority


def test_soft_state_and_async_paths_match_the_plain_calls(config5_run):
    """The forward's per-pixel state lets the backward skip its first walk: the gradients equal the two-walk
    backward's up to the order of the float atomics, and the asynchronous calls give the synchronous calls'
    planes bit for bit."""
    s, r, x = config5_run["s"], config5_run["r"], config5_run["x"]
    st = r.soft_state(s.cameras)
    A, D, N = r.render_soft_fwd(x, s.cameras, state=st, sync=False)
    g = r.render_soft_bwd(x, s.cameras, config5_run["gA_t"], config5_run["gD_t"], config5_run["gN_t"],
                          state=st, sync=False)
    r.sync_status()
    assert np.array_equal(A.cpu().numpy(), config5_run["A"])
    assert np.array_equal(D.cpu().numpy(), config5_run["D"])
    assert np.array_equal(N.cpu().numpy(), config5_run["N"])
    # per-sphere sums leave each warp as float atomics, whose order varies from run to run
    g = g.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(g - config5_run["g"]) <= 1e-6 * np.linalg.norm(config5_run["g"])
    r.render_soft_fwd(x, s.cameras, state=st, sync=False)
    assert r.soft_terms() > 100000


def test_soft_backward_reuses_the_forward_lists_only_when_valid(config5_run):
    """A backward call with the reuse flag takes the forward call's tile lists (no binning, no sort) and gives
    the rebuilt-list gradients up to the order of the float atomics.  It is repeated (the tile queue restarts),
    and the flag is refused, with the lists rebuilt, after another soft forward on other atoms and after a hard
    frame render on the same context."""
    import torch

    import paper_2501_12750_gb300 as vtx
    s, r, x = config5_run["s"], config5_run["r"], config5_run["x"]
    gA, gD, gN = config5_run["gA_t"], config5_run["gD_t"], config5_run["gN_t"]
    ref = config5_run["g"]

    def close(g):
        g = g.cpu().numpy().astype(np.float64)
        return np.linalg.norm(g - ref) <= 1e-6 * np.linalg.norm(ref)

    st = r.soft_state(s.cameras)
    r.render_soft_fwd(x, s.cameras, state=st, sync=False)
    assert close(r.render_soft_bwd(x, s.cameras, gA, gD, gN, state=st, sync=False, reuse_lists=True))
    assert close(r.render_soft_bwd(x, s.cameras, gA, gD, gN, state=st, sync=False, reuse_lists=True))
    r.sync_status()
    # another forward (other atoms, other pointer) in between: the lists are those of the other atoms
    other = torch.from_numpy(s.extra["target"]).cuda()
    r.render_soft_fwd(x, s.cameras, state=st, sync=False)
    r.render_soft_fwd(other, s.cameras, sync=False)
    assert close(r.render_soft_bwd(x, s.cameras, gA, gD, gN, state=st, sync=False, reuse_lists=True))
    # a hard frame on the same context in between overwrites the scratch
    r.render_soft_fwd(x, s.cameras, state=st, sync=False)
    r.upload_atoms(other, None, None)
    r.set_camera(s.cameras[0])
    r.render_frame(vtx.default_settings(), width=512, height=512)
    assert close(r.render_soft_bwd(x, s.cameras, gA, gD, gN, state=st, sync=False, reuse_lists=True))
    r.sync_status()
