"""Build and load the renderer's CUDA library (``_vtx.so``, C ABI of include/vtx.h).

The library is compiled in-tree with nvcc for sm_103a only.  There is no
fallback: if the library cannot be built or loaded, importing the renderer
raises, so nothing ever runs on the CPU in its place.
"""
from __future__ import annotations

import concurrent.futures as cf
import ctypes
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
SO = os.path.join(HERE, "_vtx.so")
SOURCES = ["frame.cu", "soft.cu", "api.cu", "static_vis.cu", "export.cu", "ses.cu", "peak.cu"]
HEADERS = ["vtx_device.cuh", "vtx_internal.h"]

NVCC_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-std=c++17",
              "-Xcompiler", "-fPIC", "-Xcompiler", "-O2", "-I", INCLUDE]


def nvcc() -> str:
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found: the renderer needs the CUDA toolkit to build")
    return exe


def _stale() -> bool:
    if not os.path.exists(SO):
        return True
    t = os.path.getmtime(SO)
    deps = [os.path.join(CSRC, f) for f in SOURCES + HEADERS] + [os.path.join(INCLUDE, "vtx.h")]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, extra_flags=()) -> str:
    """Compile every translation unit in parallel and link ``_vtx.so`` (no GPU needed)."""
    if not force and not _stale():
        return SO
    os.makedirs(BUILD, exist_ok=True)
    exe = nvcc()

    def compile_one(src):
        obj = os.path.join(BUILD, src.replace(".cu", ".o"))
        cmd = [exe, *NVCC_FLAGS, *extra_flags, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s%s" % (src, r.stdout, r.stderr))
        if verbose:
            print(r.stdout + r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = SO + ".%d.tmp" % os.getpid()
    cmd = [exe, "-shared", "-gencode", "arch=compute_103a,code=sm_103a", *objs, "-o", tmp]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc link failed:\n%s%s" % (r.stdout, r.stderr))
    os.replace(tmp, SO)
    return SO


# ------------------------------------------------------------- C structs --

c_float, c_int32, c_uint32, c_int64, c_void_p = (ctypes.c_float, ctypes.c_int32, ctypes.c_uint32,
                                                 ctypes.c_int64, ctypes.c_void_p)


class VtxCamera(ctypes.Structure):
    _fields_ = [("eye", c_float * 3), ("forward", c_float * 3), ("right", c_float * 3), ("up", c_float * 3),
                ("tan_half_fovy", c_float), ("znear", c_float), ("width", c_int32), ("height", c_int32)]


class VtxSettings(ctypes.Structure):
    _fields_ = [("mode", c_int32), ("ball_radius", c_float), ("bond_radius", c_float),
                ("ka", c_float), ("kd", c_float), ("ks", c_float), ("shininess", c_float),
                ("light_dir", c_float * 3), ("background", c_float * 3),
                ("ssao_samples", c_int32), ("ssao_radius", c_float), ("ssao_bias", c_float),
                ("ssao_kernel", (c_float * 3) * 64),
                ("tile_w", c_int32), ("tile_h", c_int32), ("splat_max_px", c_int32), ("flags", c_uint32),
                ("shading", c_int32), ("toon_levels", c_int32), ("probe_radius", c_float),
                ("clip_plane", c_float * 4), ("fog_near", c_float), ("fog_far", c_float), ("fog_density", c_float),
                ("outline_depth", c_float), ("outline_color", c_float * 3)]


class VtxSesGrid(ctypes.Structure):
    _fields_ = [("origin", c_float * 3), ("spacing", c_float), ("dims", c_int32 * 3), ("probe", c_float)]


class VtxOutputs(ctypes.Structure):
    _fields_ = [("depth", c_void_p), ("id", c_void_p), ("normal", c_void_p), ("rgb", c_void_p), ("ao", c_void_p)]


# Every symbol include/vtx.h declares, with its ctypes signature.
SIGNATURES = {
    "vtx_version": ([], ctypes.c_char_p),
    "vtx_default_settings": ([c_void_p], c_int32),
    "vtx_create": ([c_void_p, c_int32, c_void_p], c_int32),
    "vtx_destroy": ([c_void_p], c_int32),
    "vtx_set_stream": ([c_void_p, c_void_p], c_int32),
    "vtx_upload_atoms": ([c_void_p, c_void_p, c_void_p, c_void_p, c_int32, c_int64], c_int32),
    "vtx_upload_bonds": ([c_void_p, c_void_p, c_int64], c_int32),
    "vtx_set_camera": ([c_void_p, c_void_p], c_int32),
    "vtx_render_frame": ([c_void_p, c_void_p, c_void_p], c_int32),
    "vtx_render_frame_host": ([c_void_p, c_void_p, c_void_p, c_void_p, c_int32, c_int64, c_void_p, c_void_p,
                               c_void_p], c_int32),
    "vtx_render_batch": ([c_void_p, c_void_p, c_int64, c_void_p, c_int32, c_void_p, c_int32, c_void_p, c_void_p,
                          c_int32], c_int32),
    "vtx_render_soft_fwd": ([c_void_p, c_void_p, c_int64, c_void_p, c_int32, c_float, c_void_p, c_void_p,
                             c_void_p], c_int32),
    "vtx_render_soft_bwd": ([c_void_p, c_void_p, c_int64, c_void_p, c_int32, c_float, c_void_p, c_void_p,
                             c_void_p, c_void_p], c_int32),
    "vtx_render_soft_fwd_ex": ([c_void_p, c_void_p, c_int64, c_void_p, c_int32, c_float, c_uint32, c_void_p,
                                c_void_p, c_void_p, c_void_p], c_int32),
    "vtx_render_soft_bwd_ex": ([c_void_p, c_void_p, c_int64, c_void_p, c_int32, c_float, c_uint32, c_void_p,
                                c_void_p, c_void_p, c_void_p, c_void_p], c_int32),
    "vtx_soft_terms": ([c_void_p, c_void_p], c_int32),
    "vtx_sync_status": ([c_void_p], c_int32),
    "vtx_debug_hooks": ([c_void_p, c_int32, c_uint32, ctypes.c_uint64, c_int32], c_int32),
    "vtx_stage_times": ([c_void_p, c_void_p, c_void_p, c_void_p, c_void_p], c_int32),
    "vtx_last_error": ([c_void_p], ctypes.c_char_p),
    "vtx_ses_fit_grid": ([c_void_p, c_void_p, c_int64, c_float, c_float, c_void_p], c_int32),
    "vtx_ses_mesh": ([c_void_p, c_void_p, c_int64, c_void_p, c_void_p, c_int64, c_void_p, c_void_p, c_void_p,
                      c_void_p], c_int32),
    "vtx_export_rgba8": ([c_void_p, c_void_p, c_void_p, c_int32, c_int32, c_int32, c_float, c_void_p], c_int32),
    "vtx_render_visibility_static": ([c_void_p, c_int64, c_void_p, c_void_p, c_void_p, c_void_p], c_int32),
    "vtx_tuned_settings": ([c_void_p, c_void_p, c_void_p, c_void_p], c_int32),
    "vtx_measure_fp32_rate": ([c_int32, c_int32, c_void_p, c_void_p, c_void_p], c_int32),
}

_lib = None


def load(build_if_needed: bool = True) -> ctypes.CDLL:
    """Load ``_vtx.so`` (building it first when stale); raise if that is impossible."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_needed and _stale():
        build()
    if not os.path.exists(SO):
        raise ImportError("renderer library %s is missing; run __graft_entry__.build()" % SO)
    lib = ctypes.CDLL(SO)
    for name, (args, res) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib
