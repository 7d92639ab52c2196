"""The Python binding's ctypes structures and constants against include/fjofc.h (no GPU
needed): member names, order, element types and array lengths of every struct the
binding passes through the C ABI, and the numeric constants it mirrors."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fjofc.h")

SCALARS = {"int32_t": ctypes.c_int32, "int64_t": ctypes.c_int64, "uint64_t": ctypes.c_uint64,
           "double": ctypes.c_double, "float": ctypes.c_float}


def _header():
    return re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)


def _structs():
    """alias -> [(c type, name, array length or 0, is pointer)]"""
    out = {}
    for body, alias in re.findall(r"typedef struct(?:\s+\w+)?\s*\{(.*?)\}\s*(\w+)\s*;", _header(), flags=re.S):
        members = []
        for decl in body.split(";"):
            decl = " ".join(decl.split())
            if not decl:
                continue
            m = re.match(r"(.*?)(\w+)((?:\s*,\s*\w+)*)\s*(?:\[(\w+)\])?$", decl)
            ctype, first, more, count = m.group(1).strip(), m.group(2), m.group(3), m.group(4)
            names = [first] + [x.strip() for x in more.split(",") if x.strip()]
            for nm in names:
                members.append((ctype.replace("const", "").replace(" ", ""), nm, int(count) if count else 0))
        out[alias] = members
    return out


def _binding():
    from conftest import ensure_library
    fj = ensure_library()
    from paper_1502_03391_gb300 import learned
    return {"fjofc_opts": fj._Opts, "fjofc_result": fj._Result, "fjofc_init_opts": fj._InitOpts,
            "fjofc_problem": fj._Problem, "fjofc_tune_opts": fj._TuneOpts, "fjofc_tune_result": fj._TuneResult,
            "fjofc_mlp_train_opts": learned.TrainOpts}


@pytest.mark.parametrize("alias", ["fjofc_opts", "fjofc_result", "fjofc_init_opts", "fjofc_problem",
                                   "fjofc_tune_opts", "fjofc_tune_result", "fjofc_mlp_train_opts"])
def test_ctypes_struct_matches_header(alias):
    members = _structs()[alias]
    cls = _binding()[alias]
    fields = cls._fields_
    assert [f[0] for f in fields] == [m[1] for m in members], alias
    for (ctype, name, count), (_, ptype) in zip(members, fields):
        if ctype.endswith("*"):
            assert ptype is ctypes.c_void_p or issubclass(ptype, ctypes._Pointer), (alias, name)
            continue
        base = SCALARS[ctype]
        if count:
            assert issubclass(ptype, ctypes.Array) and ptype._length_ == count and ptype._type_ is base, \
                (alias, name)
        else:
            assert ptype is base, (alias, name)


def test_constants_match_header():
    defines = dict(re.findall(r"#define\s+(FJOFC_\w+)\s+(-?\d+)\b", _header()))
    fj = _binding()["fjofc_opts"].__module__
    import importlib
    mod = importlib.import_module(fj)
    for name in ("FJOFC_OK", "FJOFC_ERR_ARG", "FJOFC_ERR_CUDA", "FJOFC_ERR_NONFINITE", "FJOFC_ERR_TIMEOUT",
                 "FJOFC_ERR_NOMEM", "FJOFC_ERR_UNSUPPORTED"):
        assert getattr(mod, name) == int(defines[name]), name
    assert mod.TOL_ABS_NORMALIZED == int(defines["FJOFC_TOL_ABS_NORMALIZED"])
    assert mod.TOL_RELATIVE == int(defines["FJOFC_TOL_RELATIVE"])
    assert mod._OOS_FORMS == {"auto": int(defines["FJOFC_OOS_AUTO"]),
                              "streaming": int(defines["FJOFC_OOS_STREAMING"]),
                              "resident": int(defines["FJOFC_OOS_RESIDENT"])}
