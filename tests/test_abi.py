"""CPU checks of the C ABI: the library builds for sm_103a, loads, and
exports every entry point that include/fargo.h declares (no compute calls)."""
import ctypes
import os
import re

import paper_1602_02359_b300 as fb
from paper_1602_02359_b300 import build as fbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(fargo_[a-z0-9_]+)\s*\(", src))
    return names


def test_library_builds_and_exports_every_declared_symbol():
    fbuild.build()
    lib = ctypes.CDLL(fbuild.LIB)
    syms = declared_symbols()
    assert len(syms) >= 15
    for s in sorted(syms):
        assert hasattr(lib, s), s
    assert set(fb.EXPORTED) <= syms


def test_strerror_names_codes_without_a_device():
    L = fb.lib()
    assert L.fargo_strerror(-4) == b"non-finite state"
    assert L.fargo_strerror(0) == b"ok"
    assert L.fargo_strerror(5) == b"unknown error"


def test_create_without_device_reports_not_built():
    import numpy as np
    import workloads as W
    w = W.sod(ny=16)
    try:
        import torch
        if torch.cuda.is_available():
            return
    except Exception:
        pass
    try:
        fb.Fargo(w)
    except fb.FargoError as e:
        assert e.code == -8
    else:
        raise AssertionError("context created without a device")
