"""Stage timing through vtx_stage_times: full per-stage events and the cull-only form."""
import pytest

from paper_2501_12750_gb300 import scenes

pytestmark = pytest.mark.gpu


def _renderer():
    import torch

    import paper_2501_12750_gb300 as vtx
    s = scenes.config2(n=20000, width=640, height=360)
    r = vtx.Renderer()
    r.upload_atoms(torch.from_numpy(s.xyzr).cuda(), torch.from_numpy(s.elem).cuda(), s.palette)
    r.set_camera(s.cameras[0])
    out = r.render_frame(vtx.default_settings(flags=vtx.FLAG_SYNC), width=640, height=360)
    return vtx, r, out


def test_full_profile_reports_every_stage():
    vtx, r, out = _renderer()
    for _ in range(3):
        r.render_frame(vtx.default_settings(flags=vtx.FLAG_PROFILE), out=out)
    t = r.stage_times()
    assert t["runs"] == 3
    assert all(t[k] >= 0.0 for k in ("clear", "cull", "setup", "scan", "scatter", "raster", "resolve", "shade"))
    assert t["cull"] > 0.0 and t["setup"] > 0.0
    with pytest.raises(vtx.VtxError):
        r.stage_times()  # the runs were forgotten


def test_cull_only_profile_reports_the_cull_alone():
    vtx, r, out = _renderer()
    for _ in range(4):
        r.render_frame(vtx.default_settings(flags=vtx.FLAG_PROFILE_CULL), out=out)
    t = r.stage_times()
    assert t["runs"] == 4 and t["cull"] > 0.0
    assert all(t[k] == 0.0 for k in ("clear", "setup", "scan", "scatter", "raster", "resolve", "shade"))
    # mixed runs: the cull averages over all of them, the other stages over the full runs only
    r.render_frame(vtx.default_settings(flags=vtx.FLAG_PROFILE_CULL), out=out)
    r.render_frame(vtx.default_settings(flags=vtx.FLAG_PROFILE), out=out)
    t = r.stage_times()
    assert t["runs"] == 2 and t["cull"] > 0.0 and t["setup"] > 0.0
