"""The C-ABI library builds for sm_103a, loads, and exports every entry point include/gp.h declares.

No compute call is made here (no GPU in this environment); the -m gpu tests exercise the calls."""
import ctypes
import os
import re

import pytest

from paper_2411_05869_gb300 import build, gp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"^GP_API\s+[\w\s\*]+?\b(gp_\w+)\(", src, flags=re.M))
    return names


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ["gp_create", "gp_assemble", "gp_factor", "gp_loglik", "gp_predict", "gp_destroy"]:
        assert required in names
    assert names == set(gp.SYMBOLS) | (names - set(gp.SYMBOLS))


def test_library_builds_and_exports_every_symbol():
    path = build.build()
    assert os.path.exists(path)
    lib = ctypes.CDLL(path)
    for name in declared_symbols():
        assert hasattr(lib, name), name


def test_binding_declares_signatures_without_a_device():
    L = gp.load()
    for name in gp.SYMBOLS:
        assert getattr(L, name).argtypes is not None or name in ("gp_last_error",)
