"""The C-ABI library builds, loads and exports every entry point that
include/sif.h declares (no GPU needed: no compute call is made)."""
import ctypes
import os
import re

import pytest

from paper_1905_03917_gb300 import build, sif

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_entry_points():
    with open(os.path.join(ROOT, "include", "sif.h")) as f:
        txt = f.read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(sif_[a-z_0-9]+)\s*\(", txt)))


def test_library_exports_every_declared_entry_point():
    path = build.build()
    lib = ctypes.CDLL(path)
    names = declared_entry_points()
    assert len(names) >= 10
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert set(names) == set(sif.EXPORTS)


def test_config_struct_matches_header_field_order():
    with open(os.path.join(ROOT, "include", "sif.h")) as f:
        txt = f.read()
    body = txt[txt.index("typedef struct {\n  int dim;"):]
    body = body[:body.index("} sif_config;")]
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
    assert fields == [f[0] for f in sif.Config._fields_]


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
