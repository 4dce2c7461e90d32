"""The C-ABI library builds, loads and exports every entry point that
include/*.h declares (no GPU needed: no compute call is made)."""
import ctypes
import os
import re

import pytest

from paper_1905_03917_gb300 import build, sif

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_entry_points():
    names = set()
    inc = os.path.join(ROOT, "include")
    for h in sorted(os.listdir(inc)):
        if not h.endswith(".h"):
            continue
        with open(os.path.join(inc, h)) as f:
            txt = f.read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        names |= set(re.findall(r"\b(sif3?_[a-z_0-9]+)\s*\(", txt))
    return sorted(names)


def test_library_exports_every_declared_entry_point():
    path = build.build()
    lib = ctypes.CDLL(path)
    names = declared_entry_points()
    assert len(names) >= 10
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert set(names) == set(sif.EXPORTS)


def _fields(header, start, end):
    with open(os.path.join(ROOT, "include", header)) as f:
        txt = f.read()
    body = txt[txt.index(start):]
    body = body[:body.index(end)]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = []
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl or decl.startswith("typedef"):
            decl = decl.replace("typedef struct {", "").strip()
            if not decl:
                continue
        for part in decl.split(","):
            name = re.sub(r"\[.*\]", "", part.strip().split()[-1]).lstrip("*")
            fields.append(name)
    return fields


def test_config_struct_matches_header_field_order():
    fields = _fields("sif.h", "typedef struct {\n  int dim;", "} sif_config;")
    assert fields == [f[0] for f in sif.Config._fields_]


def test_config3_struct_matches_header_field_order():
    fields = _fields("sif3d.h", "typedef struct {\n  int nx, ny, nz;", "} sif3_config;")
    assert fields == [f[0] for f in sif.Config3._fields_]


def test_invalid_3d_configuration_is_rejected_without_gpu_work():
    lib = sif.load()
    c = sif.Config3()
    c.nx = c.ny = c.nz = 2  # below the WENO5 stencil's reach
    h = ctypes.c_void_p()
    assert lib.sif3_create(ctypes.byref(c), ctypes.byref(h)) == sif.EINVAL
    assert not h.value
    assert lib.sif3_last_error(None) == b"null context"


def test_invalid_configuration_is_rejected_without_gpu_work():
    lib = sif.load()
    c = sif.Config()
    c.dim = 3
    h = ctypes.c_void_p()
    assert lib.sif_create(ctypes.byref(c), ctypes.byref(h)) == sif.EINVAL
    assert not h.value
    assert lib.sif_last_error(None) == b"null context"


def test_weno_epsilon_below_the_reciprocal_range_is_rejected():
    # the finite-volume face values take one reciprocal of a product of two
    # WENO5 denominators (each at least eps^4): eps below 1e-20 is refused
    from paper_1905_03917_gb300 import inputs
    lib = sif.load()
    cfg = dict(inputs.shock_tube_1d(64)["cfg"], weno_eps=1e-30)
    c = sif.make_config(cfg)
    h = ctypes.c_void_p()
    assert lib.sif_create(ctypes.byref(c), ctypes.byref(h)) == sif.EINVAL
    assert not h.value


@pytest.mark.parametrize("field,value", [("sigma", -1.0), ("sigma", float("nan")),
                                         ("mu", (-1e-3, 0.0)), ("mu", (0.0, float("inf"))),
                                         ("weno_char", 2)])
def test_invalid_physics_options_are_rejected_without_gpu_work(field, value):
    from paper_1905_03917_gb300 import inputs
    lib = sif.load()
    cfg = dict(inputs.shock_tube_1d(64)["cfg"])
    cfg[field] = value
    c = sif.make_config(cfg)
    h = ctypes.c_void_p()
    assert lib.sif_create(ctypes.byref(c), ctypes.byref(h)) == sif.EINVAL
    assert not h.value


def test_invalid_face_flux_options_are_rejected_without_gpu_work():
    from paper_1905_03917_gb300 import inputs
    lib = sif.load()
    cfg = dict(inputs.shock_tube_1d(64)["cfg"], flux="hllc", weno_char=1)
    c = sif.make_config(cfg)
    h = ctypes.c_void_p()
    assert lib.sif_create(ctypes.byref(c), ctypes.byref(h)) == sif.EINVAL
    assert not h.value
    c = sif.make_config(inputs.shock_tube_1d(64)["cfg"])
    c.flux = 2
    assert lib.sif_create(ctypes.byref(c), ctypes.byref(h)) == sif.EINVAL
    assert not h.value
    with pytest.raises(ValueError):
        sif.make_config(dict(inputs.shock_tube_1d(64)["cfg"], flux="roe"))
