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
    assert ctypes.sizeof(sc.GridSpec) == 40
    assert ctypes.sizeof(sc.Bunch) == 120


def test_struct_layouts_match_the_header(tmp_path):
    """sizeof / offsetof of the public structs as a C compiler sees sc.h."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "layout.c"
    src.write_text("""
#include <stddef.h>
#include <stdio.h>
#include "sc.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu %zu\\n", sizeof(sc_particles), sizeof(sc_beam), sizeof(sc_element),
         sizeof(sc_grid_spec), sizeof(sc_bunch), offsetof(sc_bunch, beam), offsetof(sc_bunch, lattice),
         offsetof(sc_element, length));
  return 0;
}
""")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()]
    assert got == [ctypes.sizeof(sc.Particles), ctypes.sizeof(sc.Beam), synth.ELEMENT_DTYPE.itemsize,
                   ctypes.sizeof(sc.GridSpec), ctypes.sizeof(sc.Bunch), sc.Bunch.beam.offset,
                   sc.Bunch.lattice.offset, synth.ELEMENT_DTYPE.fields["length"][1]]


def test_batch_argument_errors_without_gpu(lib):
    """sc_create_batch rejects bad arguments before touching the device."""
    h = ctypes.c_void_p()
    spec = (sc.GridSpec * 1)(sc.GridSpec(64, 64, -1.0, 1.0, -1.0, 1.0))
    assert lib.sc_create_batch(None, spec, 1, 0, None) == -1
    assert lib.sc_create_batch(ctypes.byref(h), spec, 0, 0, None) == -1
    assert lib.sc_create_batch(ctypes.byref(h), None, 1, 0, None) == -1
    assert lib.sc_batch_track_turns(None, None, 1, None) == -1
    assert lib.sc_destroy_batch(None) == 0


def test_last_error_without_gpu(lib):
    buf = ctypes.create_string_buffer(64)
    assert lib.sc_last_error(buf, 64) == 0
    assert lib.sc_last_error(None, 0) != 0


def test_new_entry_points_reject_null_without_gpu(lib):
    """The launch-shape, host-buffer, solve-work and charge-view calls reject a
    NULL grid or batch before touching the device."""
    i, d, v, n = ctypes.c_int(), ctypes.c_double(), ctypes.c_void_p(), ctypes.c_int64()
    assert lib.sc_set_kick_push_shape(None, 0, -1) == -1
    assert lib.sc_get_kick_push_shape(None, ctypes.byref(i), ctypes.byref(i), ctypes.byref(d)) == -1
    assert lib.sc_batch_set_kick_push_shape(None, 0, 0) == -1
    assert lib.sc_batch_get_kick_push_shape(None, ctypes.byref(i), ctypes.byref(i), ctypes.byref(d)) == -1
    assert lib.sc_track_turns_host(None, None, None, None, 0, 1, None) == -1
    assert lib.sc_batch_track_turns_host(None, None, 1, None) == -1
    assert lib.sc_get_solver_work(None, ctypes.byref(d), ctypes.byref(d)) == -1
    assert lib.sc_grid_charge_device(None, ctypes.byref(v), ctypes.byref(n)) == -1
    assert lib.sc_set_particle_count(None, 10) == -1
    assert lib.sc_tunes(None, 10, 1, None, None) == -1
    assert lib.sc_sort_particles(None, None, None) == -1
    assert lib.sc_set_charge_reduce(None, sc.REDUCE_FN(), None, 0) == -1
    assert lib.sc_moments_noalloc(None, None, None) == -1


def test_oversized_host_bunch_rejected_before_any_allocation(lib):
    """A host bunch of more particles than a grid's 64-bit charge can hold is
    refused with SC_ERR_OVERFLOW before anything is sized or copied."""
    host = sc.Particles(*(ctypes.c_void_p(8).value,) * 6, 1 << 24)
    assert lib.sc_track_turns_host(None, ctypes.byref(host), None, None, 0, 1, None) == -4


def test_host_particle_marshalling():
    """The binding's host-array view: contiguous float64 numpy arrays or CPU
    tensors of one length; anything else is refused before the library."""
    import numpy as np
    import torch
    keys = ("x", "px", "y", "py", "sigma", "psigma")
    good = {k: np.zeros(5) for k in keys}
    p = sc.host_particles(good)
    assert p.n == 5 and p.x == good["x"].ctypes.data
    t = {k: torch.zeros(5, dtype=torch.float64) for k in keys}
    assert sc.host_particles(t).n == 5
    with pytest.raises(ValueError):
        sc.host_particles(dict(good, y=np.zeros(5, dtype=np.float32)))
    with pytest.raises(ValueError):
        sc.host_particles(dict(good, y=np.zeros(6)))
    with pytest.raises(ValueError):
        sc.host_particles(dict(good, y=np.zeros(10)[::2]))
