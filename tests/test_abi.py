"""The C-ABI library builds, loads without a GPU, and exports every entry point
that include/*.h declares (no compute call is made here)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        for m in re.finditer(r"\b(aafwi_\w+)\s*\(", src):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2008_11778_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ("aafwi_plan_create", "aafwi_model_forward", "aafwi_born_forward",
                     "aafwi_misfit", "aafwi_adjoint_gradient", "aafwi_born_adjoint",
                     "aafwi_aa_step", "aafwi_aa_combine", "aafwi_aa_create", "aafwi_plan_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in sorted(declared_symbols()) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_2008_11778_gb300 import aafwi
    assert set(aafwi.EXPORTS) == declared_symbols()


def test_create_errors_need_no_gpu(lib):
    """Argument errors are reported with a status code and message before any
    device work (NULL arguments)."""
    lib.aafwi_plan_create.argtypes = [ctypes.c_void_p] * 5
    lib.aafwi_last_error.restype = ctypes.c_char_p
    lib.aafwi_last_error.argtypes = [ctypes.c_void_p]
    rc = lib.aafwi_plan_create(None, None, None, None, None)
    assert rc == 1
    assert b"NULL" in lib.aafwi_last_error(None)


def header_struct_fields(name):
    """Field names, in order, of `typedef struct { ... } name;` in include/aafwi.h."""
    src = open(os.path.join(ROOT, "include", "aafwi.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    m = re.search(r"typedef struct\s*\{([^{}]*)\}\s*" + name + r"\s*;", src)
    assert m, name
    fields = []
    for decl in m.group(1).split(";"):
        decl = re.sub(r"\bconst\b", "", decl).strip()
        if not decl:
            continue
        t = re.match(r"(?:long\s+long|unsigned\s+\w+|\w+)\s+(.*)$", decl, flags=re.S)
        assert t, decl
        fields += [n.replace("*", "").strip() for n in t.group(1).split(",")]
    return fields


@pytest.mark.parametrize("c_name, py_name", [("aafwi_plan_opts", "PlanOpts"), ("aafwi_plan_info", "PlanInfo"),
                                             ("aafwi_grid", "Grid"), ("aafwi_shots", "Shots"),
                                             ("aafwi_tune_entry", "TuneEntry"), ("aafwi_aa_lp_info", "AALpInfo")])
def test_binding_structs_match_the_header(c_name, py_name):
    """The ctypes mirrors of the ABI structs list the header's fields in the
    header's order (a field added on one side only would shift the rest)."""
    from paper_2008_11778_gb300 import aafwi
    py = [f[0] for f in getattr(aafwi, py_name)._fields_]
    assert py == header_struct_fields(c_name)


@pytest.mark.parametrize("field, value, words", [("lanes", 9, b"lanes"), ("steps_per_launch", 3, b"steps_per_launch"),
                                                 ("tile_z", 24, b"tile_z"), ("tile_x", 64, b"tile_x")])
def test_bad_plan_options_are_refused_before_any_device_call(lib, field, value, words):
    """Plan options out of range come back as ARG with a message naming the
    option; the checks run before the library touches the device."""
    from paper_2008_11778_gb300 import aafwi, synth
    L = aafwi.load()
    g, s, keep = aafwi._geom_structs(synth.tiny().geom, 3000.0)
    o = aafwi.PlanOpts()
    setattr(o, field, value)
    h = ctypes.c_void_p()
    rc = L.aafwi_plan_create(ctypes.byref(g), ctypes.byref(s), aafwi._np_ptr(keep[6]), ctypes.byref(o),
                             ctypes.byref(h))
    assert rc == 1 and not h.value
    assert words in L.aafwi_last_error(None)
