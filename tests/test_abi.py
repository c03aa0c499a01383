"""The C-ABI library builds, loads and exports every symbol include/hydro.h
declares; host-side planning and validation work without a GPU."""
import ctypes
import os
import re

import pytest

from paper_2007_05218_gb300 import build as hbuild
from paper_2007_05218_gb300 import hydro
from paper_2007_05218_gb300 import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for path in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if path.endswith(".h"):
            text = open(os.path.join(ROOT, "include", path)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?\w+\s*\**\s+(hydro_\w+)\s*\(", text, flags=re.M)
    return names


def test_header_declares_the_boundary_calls():
    names = set(declared_functions())
    for required in ("hydro_alloc", "hydro_fill_ghosts", "hydro_compute_dt", "hydro_step",
                     "hydro_workspace_size", "hydro_sync", "hydro_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol():
    path = hbuild.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    assert set(hydro.EXPORTED) <= set(declared_functions())


def test_binding_constants_match_the_header():
    text = open(os.path.join(ROOT, "include", "hydro.h")).read()
    defs = dict(re.findall(r"^#define (HYDRO_\w+) \(?(-?\d+)\)?", text, flags=re.M))
    mirrored = [n for n in defs if hasattr(hydro, n)]
    assert {"HYDRO_LIMITER_CS08", "HYDRO_RIEMANN_TWO_SHOCK", "HYDRO_MIXED", "HYDRO_NG"} <= set(mirrored)
    for n in mirrored:
        assert getattr(hydro, n) == int(defs[n]), n


def test_method_selection_rejects_a_null_handle():
    with pytest.raises(hydro.HydroError):
        hydro.hydro_set_method(None, hydro.HYDRO_LIMITER_CS08, hydro.HYDRO_RIEMANN_HLLC)


def test_workspace_and_layout_planning():
    pr = inputs.density_wave((20, 12, 9), noise=0.0)
    d = hydro.desc_of(pr)
    sb, wb = hydro.hydro_workspace_size([d])
    lay = hydro.hydro_box_layout([d], 0)
    assert lay.pitch == 28 and lay.pitch % 4 == 0
    assert lay.plane == 28 * 20
    assert lay.var_stride >= lay.plane * 17 and lay.var_stride % 32 == 0
    assert sb == 5 * lay.var_stride * 8
    off, nf, eb = hydro.hydro_debug_fields([d], 0)
    assert nf == 138 and eb == 8 and off % 256 == 0
    assert wb >= off + nf * lay.var_stride * 8
    # a mixed-precision box keeps FP32 fields: half the scratch bytes
    dm = hydro.desc_of(pr, hydro.HYDRO_MIXED)
    sbm, wbm = hydro.hydro_workspace_size([dm])
    offm, nfm, ebm = hydro.hydro_debug_fields([dm], 0)
    assert sbm == sb and ebm == 4 and wbm >= offm + nfm * lay.var_stride * 4
    assert wbm - offm < (wb - off) * 0.55
    # two boxes: the second starts right after the first
    d2 = hydro.desc_of(inputs.sod((32, 4, 4)))
    l2 = hydro.hydro_box_layout([d, d2], 1)
    assert l2.offset == 5 * lay.var_stride


@pytest.mark.parametrize("field,value,msg", [
    ("ng", 3, "ng must be 4"),
    ("nx", 3, "at least 4"),
    ("gamma", 1.0, "gamma"),
    ("cfl", 0.0, "cfl"),
    ("dx", -1.0, "widths"),
    ("precision", 7, "precision"),
    ("precision", -1, "precision"),
])
def test_invalid_descriptors_are_rejected(field, value, msg):
    d = hydro.desc_of(inputs.uniform(8))
    setattr(d, field, value)
    with pytest.raises(hydro.HydroError) as e:
        hydro.hydro_workspace_size([d])
    assert e.value.code == hydro.HYDRO_ERR_INVALID
    assert msg in str(e.value)


def test_unpaired_periodic_faces_are_rejected():
    d = hydro.desc_of(inputs.uniform(8))
    d.bc[0] = hydro.HYDRO_BC["outflow"]
    with pytest.raises(hydro.HydroError, match="pair"):
        hydro.hydro_workspace_size([d])


def test_empty_box_list_is_rejected():
    with pytest.raises(hydro.HydroError) as e:
        hydro.hydro_workspace_size([])
    assert e.value.code == hydro.HYDRO_ERR_INVALID


def test_alloc_checks_buffers_before_touching_the_device():
    d = hydro.desc_of(inputs.uniform(8))
    sb, wb = hydro.hydro_workspace_size([d])
    with pytest.raises(hydro.HydroError) as e:
        hydro.hydro_alloc([d], 0, sb, 0, wb)
    assert e.value.code == hydro.HYDRO_ERR_INVALID
    with pytest.raises(hydro.HydroError) as e:
        hydro.hydro_alloc([d], 256, sb - 8, 512, wb)
    assert e.value.code == hydro.HYDRO_ERR_NOMEM
    with pytest.raises(hydro.HydroError) as e:
        hydro.hydro_alloc([d], 8, sb, 512, wb)
    assert "aligned" in str(e.value)
