"""The C ABI library builds for sm_103a, loads, and exports every function that
include/pp.h declares (no compute calls: these run without a GPU)."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_2606_20441_b300 import build, pp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fn.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", fn)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[\w\s\*]*?\b(pp_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_library_builds_and_loads():
    path = build.build()
    assert os.path.exists(path)
    lib = ctypes.CDLL(path)
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_exports_match_header():
    path = build.build()
    out = subprocess.check_output(["nm", "-D", "--defined-only", path]).decode()
    exported = {l.split()[-1] for l in out.splitlines() if " T " in l}
    decl = set(declared_functions())
    assert decl, "no declarations parsed"
    assert decl <= exported
    assert decl >= set(pp.EXPORTED) or set(pp.EXPORTED) <= decl


def test_binding_names_cover_header():
    decl = set(declared_functions())
    assert set(pp.EXPORTED) <= decl
    for name in decl:
        assert name in pp.EXPORTED


def test_default_options_without_gpu():
    lib = pp.load_library(build.build())
    opt = pp.pp_options()
    lib.pp_default_options(ctypes.byref(opt))
    assert opt.precision == pp.PRECISION_FP64 and opt.max_terms == 0


def test_create_rejects_bad_qubit_count():
    lib = pp.load_library(build.build())
    h = ctypes.c_void_p()
    assert lib.pp_create(None, 0, ctypes.byref(h)) == pp.PP_ERR_ARG
    assert lib.pp_create(None, 129, ctypes.byref(h)) == pp.PP_ERR_ARG
