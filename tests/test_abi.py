"""CPU checks of the C ABI: the library builds for sm_103a, loads, and exports every declared symbol."""
import ctypes
import os
import re

import numpy as np

from paper_2501_12750_gb300 import _native

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "vtx.h")


def declared_symbols():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(vtx_[a-z_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for must in ["vtx_upload_atoms", "vtx_upload_bonds", "vtx_set_camera", "vtx_render_frame", "vtx_render_batch",
                 "vtx_render_soft_fwd", "vtx_render_soft_bwd"]:
        assert must in names


def test_library_exports_every_declared_symbol():
    _native.build()
    lib = ctypes.CDLL(_native.SO)
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing
    assert set(declared_symbols()) <= set(_native.SIGNATURES)


def test_struct_layouts_match_header():
    assert ctypes.sizeof(_native.VtxCamera) == 64
    # mode..flags: 3 + 4 + 3 + 3 + 3 + 64*3 + 4 scalars of 4 bytes; shading..outline_color: 2 + 1 + 4 + 3 + 1 + 3
    assert ctypes.sizeof(_native.VtxSettings) == 4 * (3 + 4 + 3 + 3 + 3 + 64 * 3 + 4 + 2 + 1 + 4 + 3 + 1 + 3)
    assert ctypes.sizeof(_native.VtxOutputs) == 5 * ctypes.sizeof(ctypes.c_void_p)


def test_host_side_argument_checks_without_gpu():
    """Calls that must fail before touching a device."""
    lib = _native.load()
    s = _native.VtxSettings()
    assert lib.vtx_default_settings(ctypes.byref(s)) == 0
    assert abs(s.ka - 0.2) < 1e-7 and s.tile_w == 16 and s.splat_max_px == 0  # 0: the adaptive default
    assert lib.vtx_default_settings(None) == 1
    assert lib.vtx_create(None, 0, None) == 1
    h = ctypes.c_void_p()
    # no CUDA device in this container: creation fails cleanly with INVALID_ARG
    code = lib.vtx_create(ctypes.byref(h), 0, None)
    assert code in (0, 1)
    if code == 0:
        lib.vtx_destroy(h)
    assert lib.vtx_version().startswith(b"vtx-gb300")


def test_camera_struct_roundtrip():
    from paper_2501_12750_gb300 import camera_struct, scenes
    cam = scenes.config1().cameras[0]
    c = camera_struct(cam)
    assert c.width == 256 and c.height == 256
    np.testing.assert_array_equal(np.array(c.eye[:], np.float32), cam.eye)
    np.testing.assert_array_equal(np.array(c.forward[:], np.float32), cam.forward)


def header_enums():
    """NAME = value pairs of the header's enums (comments removed)."""
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    out = {}
    for body in re.findall(r"enum\s*\{(.*?)\}", text, flags=re.S):
        for name, val in re.findall(r"\b(VTX_[A-Z0-9_]+)\s*=\s*(\d+)u?", body):
            out[name] = int(val)
    return out


def test_binding_constants_match_the_header():
    import paper_2501_12750_gb300 as vtx
    e = header_enums()
    pairs = {"VTX_MODE_VDW": vtx.MODE_VDW, "VTX_MODE_BALL_AND_STICK": vtx.MODE_BALL_AND_STICK,
             "VTX_MODE_STICKS": vtx.MODE_STICKS, "VTX_MODE_SAS": vtx.MODE_SAS,
             "VTX_SHADE_GLOSSY": vtx.SHADE_GLOSSY, "VTX_SHADE_FLAT": vtx.SHADE_FLAT,
             "VTX_SHADE_MATTE": vtx.SHADE_MATTE, "VTX_SHADE_TOON": vtx.SHADE_TOON,
             "VTX_FLAG_SYNC": vtx.FLAG_SYNC, "VTX_FLAG_PROFILE": vtx.FLAG_PROFILE,
             "VTX_FLAG_NO_SSAO": vtx.FLAG_NO_SSAO, "VTX_FLAG_PROFILE_CULL": vtx.FLAG_PROFILE_CULL}
    for name, val in pairs.items():
        assert e.get(name) == val, (name, e.get(name), val)
    flags = [v for k, v in e.items() if k.startswith("VTX_FLAG_")]
    assert len(flags) == len(set(flags)) and all(v & (v - 1) == 0 for v in flags)  # distinct single bits
    status = {v: k[len("VTX_ERR_"):] if k.startswith("VTX_ERR_") else "OK" for k, v in e.items()
              if k.startswith("VTX_ERR_") or k == "VTX_OK"}
    assert status == vtx.STATUS, (status, vtx.STATUS)
