"""Checkpoint and resume of a tracked bunch (sc_checkpoint_write /
sc_checkpoint_read, host memory, no GPU): the state comes back bit for bit
(signed zeros, subnormals, infinities and NaN payloads included) with the turn
counter; a file written for another bunch size, other beam constants or
another lattice, or one that is truncated, extended or damaged anywhere, is
refused with SC_ERR_ARG and leaves the caller's arrays untouched."""
import os

import numpy as np
import pytest

from paper_2010_11540_gb300 import build, sc, synth

KEYS = ("x", "px", "y", "py", "sigma", "psigma")
HEADER = 88  # magic, version, zero, n, turn, beam (6 float64), lattice hash


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    sc.load()


def state(n, seed):
    rng = np.random.default_rng(seed)
    bits = rng.integers(0, 2 ** 64, (6, n), dtype=np.uint64)
    st = {k: bits[i].view(np.float64).copy() for i, k in enumerate(KEYS)}
    special = np.array([0.0, -0.0, 5e-324, np.inf, -np.inf, np.nan, 1.0, -2.5e-3])
    st["x"][:special.size] = special
    st["psigma"][:3] = np.frombuffer(np.array([0x7ff8000000000123, 0xfff0000000000001, 1],
                                              dtype=np.uint64).tobytes(), dtype=np.float64)
    return st


def same_bits(a, b):
    return all(np.array_equal(a[k].view(np.uint64), b[k].view(np.uint64)) for k in KEYS)


def empty_like(st):
    return {k: np.full_like(v, 7.0) for k, v in st.items()}


@pytest.fixture
def setup(tmp_path):
    b = synth.beam(circumference=1728.0)
    lat = synth.lattice("c2")
    st = state(10007, 1)
    path = str(tmp_path / "bunch.ckpt")
    sc.checkpoint_write(path, st, 1234, b, lat)
    return path, st, b, lat


def test_round_trip_bit_for_bit(setup):
    path, st, b, lat = setup
    got = empty_like(st)
    assert sc.checkpoint_read(path, got, b, lat) == 1234
    assert same_bits(got, st)
    assert not os.path.exists(path + ".tmp")
    assert os.path.getsize(path) == HEADER + 6 * 8 * 10007 + 8


def test_overwrite_replaces(setup):
    path, st, b, lat = setup
    st2 = state(10007, 2)
    sc.checkpoint_write(path, st2, 5678, b, lat)
    got = empty_like(st)
    assert sc.checkpoint_read(path, got, b, lat) == 5678 and same_bits(got, st2)


def expect_refused(path, st, b, lat, what):
    got = empty_like(st)
    with pytest.raises(sc.ScError) as e:
        sc.checkpoint_read(path, got, b, lat)
    assert e.value.code == -1 and what in str(e.value), str(e.value)
    assert all(np.all(got[k] == 7.0) for k in KEYS)  # untouched


def test_refuses_another_bunch_beam_or_lattice(setup):
    path, st, b, lat = setup
    expect_refused(path, {k: v[:-1].copy() for k, v in st.items()}, b, lat, "particles")
    b2 = dict(b, n_lambda=b["n_lambda"] * (1 + 1e-15))
    expect_refused(path, st, b2, lat, "beam")
    lat2 = lat.copy()
    lat2["k1"][1] = np.nextafter(lat2["k1"][1], 1.0)
    expect_refused(path, st, b, lat2, "lattice")
    expect_refused(path, st, b, lat[:-1], "lattice")


def test_refuses_damaged_files(setup):
    path, st, b, lat = setup
    raw = open(path, "rb").read()
    for cut in (10, HEADER - 1, HEADER + 8 * 10007, len(raw) - 1):
        open(path, "wb").write(raw[:cut])
        expect_refused(path, st, b, lat, "checkpoint")
    open(path, "wb").write(raw + b"\0")
    expect_refused(path, st, b, lat, "trailing")
    for pos in (HEADER, HEADER + 3 * 8 * 10007 + 5, len(raw) - 3):
        bad = bytearray(raw)
        bad[pos] ^= 0x10
        open(path, "wb").write(bytes(bad))
        expect_refused(path, st, b, lat, "checksum")
    bad = bytearray(raw)
    bad[0] ^= 1
    open(path, "wb").write(bytes(bad))
    expect_refused(path, st, b, lat, "not a checkpoint")
    expect_refused(path + ".missing", st, b, lat, "cannot open")


def test_argument_errors(tmp_path):
    import ctypes
    L = sc.load()
    st = state(16, 3)
    p = sc.host_particles(st)
    bb = sc.beam(synth.beam())
    assert L.sc_checkpoint_write(None, ctypes.byref(p), 0, ctypes.byref(bb), None, 0) == -1
    assert L.sc_checkpoint_write(str(tmp_path / "a").encode(), None, 0, ctypes.byref(bb), None, 0) == -1
    assert L.sc_checkpoint_write(str(tmp_path / "a").encode(), ctypes.byref(p), 0, None, None, 0) == -1
    assert L.sc_checkpoint_write(str(tmp_path / "a").encode(), ctypes.byref(p), 0, ctypes.byref(bb), None, 3) == -1
    empty = sc.Particles(*(p.x,) * 6, 0)
    assert L.sc_checkpoint_write(str(tmp_path / "a").encode(), ctypes.byref(empty), 0, ctypes.byref(bb), None,
                                 0) == -1
    assert L.sc_checkpoint_read(str(tmp_path / "a").encode(), ctypes.byref(p), None, ctypes.byref(bb), None, 0) == -1
    # an empty lattice is a lattice too: written and read back with turn == NULL
    assert L.sc_checkpoint_write(str(tmp_path / "b").encode(), ctypes.byref(p), 9, ctypes.byref(bb), None, 0) == 0
    assert L.sc_checkpoint_read(str(tmp_path / "b").encode(), ctypes.byref(p), None, ctypes.byref(bb), None, 0) == 0
    assert L.sc_checkpoint_write(str(tmp_path / "no" / "dir").encode(), ctypes.byref(p), 0, ctypes.byref(bb), None,
                                 0) == -1


SANITIZED = r"""
#include <string>
#include <cstdio>
#include "sc_internal.cuh"
namespace sc { std::string g_msg; sc_status set_error(sc_status code, const std::string& msg) { g_msg = msg; return code; } }
#include <cstdlib>
#include <cstring>
int main() {
  const int64_t n = 1000;
  double* a = (double*)malloc(6 * n * 8);
  for (int64_t i = 0; i < 6 * n; ++i) a[i] = (double)i * 0.5;
  sc_particles p = {a, a + n, a + 2 * n, a + 3 * n, a + 4 * n, a + 5 * n, n};
  sc_beam b = {4.2, 0.97, 5e9, 1.5e-18, 100, 0.938e9};
  sc_element lat[2] = {{0, 0, 1.0, 0, 0, 0, 0, 0, 0}, {5, 0, 0, 0, 0, 0, 0, 0, 0}};
  if (sc_checkpoint_write("c.bin", &p, 7, &b, lat, 2)) return 1;
  double* c = (double*)calloc(6 * n, 8);
  sc_particles q = {c, c + n, c + 2 * n, c + 3 * n, c + 4 * n, c + 5 * n, n};
  int64_t t = 0;
  if (sc_checkpoint_read("c.bin", &q, &t, &b, lat, 2) || t != 7 || memcmp(a, c, 6 * n * 8)) return 2;
  FILE* f = fopen("c.bin", "r+b"); fseek(f, 200, SEEK_SET); fputc(0x55, f); fclose(f);
  if (sc_checkpoint_read("c.bin", &q, &t, &b, lat, 2) != SC_ERR_ARG) return 3;
  if (sc_checkpoint_read("missing.bin", &q, &t, &b, lat, 2) != SC_ERR_ARG) return 4;
  sc_particles z = {a, a, a, a, a, a, 0};
  if (sc_checkpoint_write("d.bin", &z, 0, &b, lat, 2) != SC_ERR_ARG) return 5;
  free(a); free(c);
  puts("ok");
  return 0;
}
"""


def test_checkpoint_code_under_sanitizers(tmp_path):
    """The host code of csrc/checkpoint.cu compiled by the system C++ compiler
    under AddressSanitizer, UndefinedBehaviorSanitizer and LeakSanitizer (a
    stub stands in for the library's error recorder): a write, a read, a
    damaged file, a missing file and an empty bunch, with no report."""
    import shutil
    import subprocess
    cxx = shutil.which("g++")
    cuda_inc = "/usr/local/cuda/include"
    if cxx is None or not os.path.isdir(cuda_inc):
        pytest.skip("no g++ or CUDA headers")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    csrc = os.path.join(root, "paper_2010_11540_gb300", "csrc")
    (tmp_path / "stub.cpp").write_text(SANITIZED)
    exe = tmp_path / "ck"
    r = subprocess.run([cxx, "-std=c++17", "-O1", "-g", "-fsanitize=address,undefined", "-fno-sanitize-recover=all",
                        "-I", os.path.join(root, "include"), "-I", csrc, "-I", cuda_inc,
                        "-x", "c++", os.path.join(csrc, "checkpoint.cu"), "-x", "c++", str(tmp_path / "stub.cpp"),
                        "-o", str(exe)], capture_output=True, text=True)
    if r.returncode != 0:
        pytest.skip("sanitizer build not available: " + r.stderr[-200:])
    r = subprocess.run([str(exe)], capture_output=True, text=True, cwd=tmp_path, timeout=120,
                       env=dict(os.environ, ASAN_OPTIONS="detect_leaks=1"))
    assert r.returncode == 0 and r.stdout.strip() == "ok", (r.returncode, r.stderr[-3000:])
