"""GB300-native meshless molecular ray-caster (VTX hot path).

Thin Python binding over the C ABI in ``include/vtx.h``: every call below
marshals arguments (torch tensors for device memory and streams) and calls
the CUDA library; every step of the rendering runs in its kernels.  The
library is required: importing ``Renderer`` builds or loads ``_vtx.so`` and
raises if that fails -- there is no CPU fallback.

Names mirror the C ABI: ``upload_atoms``, ``upload_bonds``, ``set_camera``,
``render_frame``, ``render_frame_host``, ``render_batch``,
``render_soft_fwd`` / ``render_soft_bwd`` and the autograd wrapper
``SoftRender``.
"""
from __future__ import annotations

import ctypes
from typing import Dict, List, Optional, Sequence

import numpy as np

from . import scenes
from ._native import VtxCamera, VtxOutputs, VtxSesGrid, VtxSettings, load

MODE_VDW = 0
MODE_BALL_AND_STICK = 1
MODE_STICKS = 2
MODE_SAS = 3
SHADE_GLOSSY, SHADE_FLAT, SHADE_MATTE, SHADE_TOON = 0, 1, 2, 3
FLAG_SYNC = 1
FLAG_PROFILE = 2
FLAG_NO_SSAO = 4
FLAG_PROFILE_CULL = 8
FLAG_SOFT_REUSE = 16

STATUS = {0: "OK", 1: "INVALID_ARG", 2: "CUDA", 3: "OOM", 4: "CAPACITY", 5: "TIMEOUT", 6: "BOUNDS", 7: "STATE"}


class VtxError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("vtx %s: %s" % (STATUS.get(code, code), msg))
        self.code = code


def camera_struct(cam) -> VtxCamera:
    """A ``VtxCamera`` from a ``scenes.Camera`` (or a record of ``scenes.CAMERA_DTYPE``)."""
    c = VtxCamera()
    rec = cam.record() if hasattr(cam, "record") else np.asarray(cam).reshape(())
    for k in range(3):
        c.eye[k] = float(rec["eye"][k])
        c.forward[k] = float(rec["forward"][k])
        c.right[k] = float(rec["right"][k])
        c.up[k] = float(rec["up"][k])
    c.tan_half_fovy = float(rec["tan_half_fovy"])
    c.znear = float(rec["znear"])
    c.width = int(rec["width"])
    c.height = int(rec["height"])
    return c


def default_settings(ssao_kernel: Optional[np.ndarray] = None, **kw) -> VtxSettings:
    """Library defaults (Blinn-Phong 0.2/0.7/0.3/32, light (0.25,0.5,1), white background); SSAO on when a kernel is given."""
    s = VtxSettings()
    load().vtx_default_settings(ctypes.byref(s))
    if ssao_kernel is not None:
        k = np.asarray(ssao_kernel, np.float32).reshape(-1, 3)
        s.ssao_samples = k.shape[0]
        for j in range(k.shape[0]):
            for c in range(3):
                s.ssao_kernel[j][c] = float(k[j, c])
    for key, val in kw.items():
        if key in ("light_dir", "background", "outline_color", "clip_plane"):
            arr = getattr(s, key)
            for c in range(len(arr)):
                arr[c] = float(val[c])
        else:
            setattr(s, key, val)
    return s


def _ptr(t) -> Optional[int]:
    return None if t is None else t.data_ptr()


class Renderer:
    """One rendering context on one CUDA device and stream (``vtx_ctx``)."""

    def __init__(self, device: int = 0, stream=None):
        import torch
        self._torch = torch
        self.lib = load()
        self.device = device
        if stream is None:
            stream = torch.cuda.current_stream(device)
        self.stream = stream
        h = ctypes.c_void_p()
        self._check(self.lib.vtx_create(ctypes.byref(h), device, ctypes.c_void_p(stream.cuda_stream)), ctx=None)
        self.ctx = h
        self._keep = []

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.vtx_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, code: int, ctx="self"):
        if code != 0:
            c = self.ctx if ctx == "self" else None
            msg = self.lib.vtx_last_error(c).decode() if c else ""
            raise VtxError(code, msg)

    # -- scene --------------------------------------------------------------
    @staticmethod
    def _visible(t) -> bool:
        """Device tensor, or a page-locked host tensor the kernels can read over the host link."""
        return t.is_cuda or t.is_pinned()

    def upload_atoms(self, xyzr, elem=None, palette=None):
        """xyzr: float32 (N, 4), on the device or in page-locked host memory (then streamed from the host by
        every frame, so N is bounded by host memory); elem: uint8 (N,) likewise, or None; palette: (E, 3)."""
        torch = self._torch
        assert self._visible(xyzr) and xyzr.dtype == torch.float32 and xyzr.is_contiguous()
        pal = np.ascontiguousarray(scenes.PALETTE if palette is None else palette, np.float32).reshape(-1, 3)
        if elem is not None:
            assert self._visible(elem) and elem.dtype == torch.uint8 and elem.is_contiguous()
        self._keep = [xyzr, elem, pal]
        self._check(self.lib.vtx_upload_atoms(self.ctx, _ptr(xyzr), _ptr(elem), pal.ctypes.data, pal.shape[0],
                                              xyzr.shape[0]))

    def upload_bonds(self, pairs):
        """pairs: int32/uint32 (B, 2) with i < j, on the device or in page-locked host memory."""
        if pairs is None:
            self._check(self.lib.vtx_upload_bonds(self.ctx, None, 0))
            return
        assert self._visible(pairs) and pairs.is_contiguous() and pairs.element_size() == 4
        self._keep.append(pairs)
        self._check(self.lib.vtx_upload_bonds(self.ctx, _ptr(pairs), pairs.shape[0]))

    def set_camera(self, cam):
        c = camera_struct(cam)
        self._check(self.lib.vtx_set_camera(self.ctx, ctypes.byref(c)))

    # -- rendering ----------------------------------------------------------
    def alloc_outputs(self, width: int, height: int, n_images: int = 1) -> Dict[str, "object"]:
        torch = self._torch
        dev = torch.device("cuda", self.device)
        shp = (n_images, height, width) if n_images > 1 else (height, width)
        shp3 = (n_images, 3, height, width) if n_images > 1 else (3, height, width)
        return dict(depth=torch.empty(shp, dtype=torch.float32, device=dev),
                    id=torch.empty(shp, dtype=torch.int32, device=dev),
                    normal=torch.empty(shp3, dtype=torch.float32, device=dev),
                    rgb=torch.empty(shp3, dtype=torch.float32, device=dev),
                    ao=torch.empty(shp, dtype=torch.float32, device=dev))

    @staticmethod
    def _outs(o) -> VtxOutputs:
        return VtxOutputs(_ptr(o["depth"]), _ptr(o["id"]), _ptr(o["normal"]), _ptr(o["rgb"]), _ptr(o.get("ao")))

    def render_frame(self, settings: VtxSettings, out=None, width=None, height=None):
        """Render the uploaded atoms from the current camera; returns the output planes (device tensors)."""
        if out is None:
            out = self.alloc_outputs(width, height)
        o = self._outs(out)
        self._check(self.lib.vtx_render_frame(self.ctx, ctypes.byref(settings), ctypes.byref(o)))
        return out

    def export_rgba8(self, out, background_alpha: float = 0.0, rgba=None):
        """Pack the rgb and id planes of `out` (one image or a batch) into uint8 RGBA (..., H, W, 4)."""
        torch = self._torch
        rgb, ids = out["rgb"], out["id"]
        H, W = ids.shape[-2], ids.shape[-1]
        n = ids.numel() // (H * W)
        if rgba is None:
            rgba = torch.empty(tuple(ids.shape) + (4,), dtype=torch.uint8, device=ids.device)
        assert self._visible(rgba) and rgba.dtype == torch.uint8 and rgba.is_contiguous() and rgba.numel() == 4 * n * H * W
        self._check(self.lib.vtx_export_rgba8(self.ctx, _ptr(rgb), _ptr(ids), W, H, n, float(background_alpha),
                                              _ptr(rgba)))
        return rgba

    def ses_fit_grid(self, xyzr, probe: float = 1.4, spacing: float = 0.5) -> VtxSesGrid:
        """Grid covering every solvent accessible sphere of `xyzr` (device or page-locked host float32 (N, 4))."""
        g = VtxSesGrid()
        self._check(self.lib.vtx_ses_fit_grid(self.ctx, _ptr(xyzr), xyzr.shape[0], float(probe), float(spacing),
                                              ctypes.byref(g)))
        return g

    @staticmethod
    def ses_grid(origin, spacing, dims, probe=1.4) -> VtxSesGrid:
        g = VtxSesGrid()
        for d in range(3):
            g.origin[d] = float(origin[d])
            g.dims[d] = int(dims[d])
        g.spacing = float(spacing)
        g.probe = float(probe)
        return g

    def ses_mesh(self, xyzr, grid: VtxSesGrid, max_tris: Optional[int] = None, labels: bool = False,
                 planes: bool = False):
        """Solvent excluded surface on `grid` as a triangle soup (device float32 (T, 3, 3)).

        Returns a dict with "tris" and, on request, "labels" (int64 (T, 3)) and the "sas" / "edt2" planes
        (uint8 / uint16 (nz, ny, nx)).  With max_tris None the call runs twice: once to count.
        """
        torch = self._torch
        assert self._visible(xyzr) and xyzr.dtype == torch.float32 and xyzr.is_contiguous()
        dev = torch.device("cuda", self.device)
        nz, ny, nx = grid.dims[2], grid.dims[1], grid.dims[0]
        sas = torch.empty((nz, ny, nx), dtype=torch.uint8, device=dev) if planes else None
        edt = torch.empty((nz, ny, nx), dtype=torch.int16, device=dev) if planes else None
        n = ctypes.c_int64(0)
        if max_tris is None:
            code = self.lib.vtx_ses_mesh(self.ctx, _ptr(xyzr), xyzr.shape[0], ctypes.byref(grid), None, 0, None,
                                         None, None, ctypes.byref(n))
            if code not in (0, 4):
                self._check(code)
            max_tris = n.value
        tris = torch.empty((max(max_tris, 1), 3, 3), dtype=torch.float32, device=dev)
        lab = torch.empty((max(max_tris, 1), 3), dtype=torch.int64, device=dev) if labels else None
        self._check(self.lib.vtx_ses_mesh(self.ctx, _ptr(xyzr), xyzr.shape[0], ctypes.byref(grid), _ptr(tris),
                                          max_tris, _ptr(lab), _ptr(sas), _ptr(edt), ctypes.byref(n)))
        out = {"tris": tris[:n.value], "n": n.value}
        if labels:
            out["labels"] = lab[:n.value]
        if planes:
            out["sas"] = sas
            out["edt2"] = edt  # uint16 values in int16 storage
        return out

    def render_frame_host(self, xyzr_host: np.ndarray, elem_host: Optional[np.ndarray], cam, settings: VtxSettings,
                          out_host: Dict[str, np.ndarray], palette=None):
        """Host buffers in and out (copies inside the call); synchronises."""
        pal = np.ascontiguousarray(scenes.PALETTE if palette is None else palette, np.float32).reshape(-1, 3)
        c = camera_struct(cam)
        o = VtxOutputs(*(None if out_host.get(k) is None else out_host[k].ctypes.data
                         for k in ("depth", "id", "normal", "rgb", "ao")))
        ep = None if elem_host is None else elem_host.ctypes.data
        self._check(self.lib.vtx_render_frame_host(self.ctx, xyzr_host.ctypes.data, ep, pal.ctypes.data,
                                                   pal.shape[0], xyzr_host.shape[0], ctypes.byref(c),
                                                   ctypes.byref(settings), ctypes.byref(o)))
        return out_host

    def render_batch(self, frames, counts: Sequence[int], cams: List, settings: VtxSettings, out=None,
                     use_graph: bool = False):
        """frames: float32 (F, stride, 4) on the device or page-locked host; counts: atoms per frame; cams: V
        cameras of one size."""
        F, stride = frames.shape[0], frames.shape[1]
        V = len(cams)
        carr = (VtxCamera * V)(*[camera_struct(c) for c in cams])
        cnt = np.ascontiguousarray(np.asarray(counts, np.int64))
        if out is None:
            out = self.alloc_outputs(cams[0].width, cams[0].height, F * V)
        o = self._outs(out)
        self._check(self.lib.vtx_render_batch(self.ctx, _ptr(frames), stride, cnt.ctypes.data, F, carr, V,
                                              ctypes.byref(settings), ctypes.byref(o), 1 if use_graph else 0))
        return out

    def soft_state(self, cams: List):
        """A per-pixel state buffer for render_soft_fwd / render_soft_bwd (uint32 (V, H, W, 2))."""
        torch = self._torch
        return torch.empty((len(cams), cams[0].height, cams[0].width, 2), dtype=torch.int32,
                           device=torch.device("cuda", self.device))

    def render_soft_fwd(self, xyzr, cams: List, sigma_px: float = 0.5, state=None, sync: bool = True):
        """Soft-edge coverage, depth and normal planes.  state (from soft_state) receives each pixel's final
        transmittance and last contributor for a later render_soft_bwd; sync=False only enqueues (after the
        first call of a problem size)."""
        torch = self._torch
        V = len(cams)
        W, H = cams[0].width, cams[0].height
        dev = xyzr.device
        cov = torch.empty((V, H, W), dtype=torch.float32, device=dev)
        dep = torch.empty((V, H, W), dtype=torch.float32, device=dev)
        nrm = torch.empty((V, 3, H, W), dtype=torch.float32, device=dev)
        carr = (VtxCamera * V)(*[camera_struct(c) for c in cams])
        self._check(self.lib.vtx_render_soft_fwd_ex(self.ctx, _ptr(xyzr), xyzr.shape[0], carr, V, sigma_px,
                                                    FLAG_SYNC if sync else 0, _ptr(cov), _ptr(dep), _ptr(nrm),
                                                    _ptr(state)))
        return cov, dep, nrm

    def render_soft_bwd(self, xyzr, cams: List, g_cov, g_depth, g_normal, sigma_px: float = 0.5, state=None,
                        sync: bool = True, reuse_lists: bool = False):
        """d/d(x, y, z, r) of sum(g_cov cov + g_depth depth + g_normal . normal); state from the matching
        forward call (same xyzr, cams, sigma) skips the backward's front-to-back walk.  reuse_lists promises
        that xyzr's contents are those of the latest soft forward call on this renderer: its tile lists are
        then reused when nothing else has used the renderer's scratch since (else they are rebuilt)."""
        torch = self._torch
        V = len(cams)
        grad = torch.empty_like(xyzr)
        carr = (VtxCamera * V)(*[camera_struct(c) for c in cams])
        gc = None if g_cov is None else g_cov.contiguous()
        gd = None if g_depth is None else g_depth.contiguous()
        gn = None if g_normal is None else g_normal.contiguous()
        self._check(self.lib.vtx_render_soft_bwd_ex(self.ctx, _ptr(xyzr), xyzr.shape[0], carr, V, sigma_px,
                                                    (FLAG_SYNC if sync else 0) |
                                                    (FLAG_SOFT_REUSE if reuse_lists else 0),
                                                    _ptr(gc), _ptr(gd), _ptr(gn), _ptr(state), _ptr(grad)))
        return grad

    def soft_terms(self) -> int:
        """Sigmoid terms composited by the most recent soft forward call (synchronises)."""
        n = ctypes.c_uint64(0)
        self._check(self.lib.vtx_soft_terms(self.ctx, ctypes.byref(n)))
        return int(n.value)

    def tuned_settings(self):
        """(tile_w, tile_h, splat_max_px) picked by the autotuner for the last call with tile_w = 0."""
        tw, th, sp = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        self._check(self.lib.vtx_tuned_settings(self.ctx, ctypes.byref(tw), ctypes.byref(th), ctypes.byref(sp)))
        return tw.value, th.value, sp.value

    def sync_status(self):
        self._check(self.lib.vtx_sync_status(self.ctx))

    def debug_hooks(self, first_wait_polls: int = -1, cap_records: int = 0, cap_entries: int = 0,
                    corrupt_key: bool = False):
        """Failure injection for tests (vtx_debug_hooks): a short first bulk-copy wait, small arena
        capacities, a corrupted depth key.  The defaults switch the wait and key hooks off."""
        self._check(self.lib.vtx_debug_hooks(self.ctx, int(first_wait_polls), int(cap_records), int(cap_entries),
                                             1 if corrupt_key else 0))

    def stage_times(self) -> Dict[str, float]:
        """Average per-stage ms over the profiled runs since the last call (key "runs": their number)."""
        names = (ctypes.c_char_p * 8)()
        ms = (ctypes.c_float * 8)()
        n = ctypes.c_int32(8)
        runs = ctypes.c_int32(0)
        self._check(self.lib.vtx_stage_times(self.ctx, names, ms, ctypes.byref(n), ctypes.byref(runs)))
        out = {names[i].decode(): float(ms[i]) for i in range(n.value)}
        out["runs"] = runs.value
        return out


def _soft_function():
    import torch

    class SoftRender(torch.autograd.Function):
        """Differentiable soft-edge render: (xyzr) -> (coverage, depth, normal); backward in CUDA."""

        @staticmethod
        def forward(ctx, xyzr, renderer, cams, sigma_px=0.5):
            x = xyzr.detach().contiguous()
            state = renderer.soft_state(cams)
            cov, dep, nrm = renderer.render_soft_fwd(x, cams, sigma_px, state=state, sync=False)
            ctx.save_for_backward(x, state)
            ctx.renderer, ctx.cams, ctx.sigma = renderer, cams, sigma_px
            return cov, dep, nrm

        @staticmethod
        def backward(ctx, g_cov, g_dep, g_nrm):
            # saved tensors are checked against in-place changes, so x still holds the forward's contents and
            # the forward's tile lists may be reused (the library rebuilds them if another call intervened)
            x, state = ctx.saved_tensors
            grad = ctx.renderer.render_soft_bwd(x, ctx.cams, g_cov, g_dep, g_nrm, ctx.sigma, state=state,
                                                sync=False, reuse_lists=True)
            ctx.renderer.sync_status()  # a capacity overflow in either call surfaces here
            return grad, None, None, None

    return SoftRender


def __getattr__(name):
    if name == "SoftRender":
        fn = _soft_function()
        globals()["SoftRender"] = fn
        return fn
    raise AttributeError(name)
