"""The C-ABI library builds for sm_103a, loads without a GPU and exports
every entry point include/sc.h declares; the ctypes structs match the C
layouts.  No compute call is made here."""
import ctypes
import os
import re

import pytest

from paper_2010_11540_gb300 import build, sc, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return ctypes.CDLL(build.LIB)


def declared():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            names += re.findall(r"^sc_status\s+(sc_\w+)\s*\(", txt, flags=re.M)
    return names


def test_header_declares_the_boundary():
    names = set(declared())
    for n in ("sc_create_grid", "sc_deposit", "sc_solve", "sc_kick_push", "sc_track_turns"):
        assert n in names


def test_exports_every_declared_symbol(lib):
    names = declared()
    assert len(names) >= 9
    for n in names:
        assert hasattr(lib, n), n
    assert set(sc.EXPORTS) <= set(names)


def test_struct_layouts():
    assert ctypes.sizeof(sc.Particles) == 56
    assert ctypes.sizeof(sc.Beam) == 48
    assert synth.ELEMENT_DTYPE.itemsize == 64


def test_last_error_without_gpu(lib):
    buf = ctypes.create_string_buffer(64)
    assert lib.sc_last_error(buf, 64) == 0
    assert lib.sc_last_error(None, 0) != 0
