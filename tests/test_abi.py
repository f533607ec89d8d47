"""The C-ABI library loads and exports every symbol include/osbli.h declares (no GPU needed)."""
import ctypes
import os
import re

from paper_2007_14933_b300 import build, osbli

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(osbli_\w+)\s*\(", src))
    return names


def test_library_exports_every_declared_entry_point():
    build.build()
    lib = ctypes.CDLL(build.LIB)
    declared = _declared()
    assert "osbli_create" in declared and "osbli_rk_step" in declared
    for name in sorted(declared):
        assert hasattr(lib, name), name
    assert set(osbli.EXPORTED) <= declared


def test_params_struct_matches_header_field_order():
    src = open(os.path.join(ROOT, "include", "osbli.h")).read()
    body = src[src.index("typedef struct {"):src.index("} osbli_params;")]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = re.findall(r"\b(?:int|double)\s+([^;]+);", body)
    names = []
    for f in fields:
        for part in f.split(","):
            names.append(re.sub(r"\[.*", "", part.strip()))
    assert names == [f[0] for f in osbli.osbli_params._fields_]


def test_invalid_parameters_are_rejected_before_any_device_call():
    build.build()
    base = dict(n=(8, 8, 8), bc=[[0, 0]] * 3, h=(1, 1, 1), dt=1e-3)
    bad = [dict(base, n=(0, 8, 8)),                                  # empty
           dict(base, bc=[[0, 1], [0, 0], [0, 0]]),                  # periodic on one side
           dict(base, n=(4, 8, 8), bc=[[1, 1], [0, 0], [0, 0]]),     # too short for closures
           dict(base, scheme=7),
           dict(base, gamma=1.0),
           dict(base, dt=-1.0),
           dict(base, h=(0, 1, 1))]
    for cfg in bad:
        p = osbli.make_params(cfg)
        h = ctypes.c_void_p()
        rc = osbli.load().osbli_create(ctypes.byref(p), None, None, ctypes.byref(h))
        assert rc == osbli.OSBLI_EINVAL, cfg
        assert osbli.osbli_last_error(None)
        assert not h.value
