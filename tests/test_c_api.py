"""The C-ABI used from plain C99 (no C++, no CUDA headers): the program in
tests/c_api/ compiles with -std=c99 -pedantic -Werror against include/sc.h
and links against libsc.so (CPU); on a GPU it tracks a host-memory bunch
through sc_track_turns_host, checks the moments and the error reporting, and
its tracked state and moments are compared with the oracle's run of the same
bunch, lattice and grid."""
import math
import os
import subprocess

import numpy as np
import pytest

import oracle
from paper_2010_11540_gb300 import build, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "c_api", "track_host.c")


def compile_program(tmp_path):
    lib = build.build()
    pkg = os.path.dirname(lib)
    exe = str(tmp_path / "track_host")
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic", "-I", os.path.join(ROOT, "include"),
                    SRC, "-o", exe, "-L", pkg, "-lsc", f"-Wl,-rpath,{pkg}", "-lm"], check=True)
    return exe


def test_c_program_compiles_and_links(tmp_path):
    assert os.path.exists(compile_program(tmp_path))


def c_program_inputs():
    """The program's bunch, beam, lattice and grid, built the way it builds
    them (the same 64-bit LCG draws and double arithmetic)."""
    n = 20000
    lcg = 12345
    u = np.empty(6 * n)
    for k in range(6 * n):
        lcg = (lcg * 6364136223846793005 + 1442695040888963407) % (1 << 64)
        u[k] = (float(lcg >> 11) + 0.5) / 9007199254740992.0
    u = u.reshape(n, 6)
    parts = {"x": 4e-3 * (u[:, 0] - 0.5), "px": 4e-4 * (u[:, 1] - 0.5), "y": 4e-3 * (u[:, 2] - 0.5),
             "py": 4e-4 * (u[:, 3] - 0.5), "sigma": 20.0 * (u[:, 4] - 0.5), "psigma": 2e-3 * (u[:, 5] - 0.5)}
    gamma0 = 1.0 + 3.0 / 0.93827208816
    beam = dict(gamma0=gamma0, beta0=math.sqrt(1.0 - 1.0 / (gamma0 * gamma0)), n_lambda=5e9, r_p=1.5347e-18,
                circumference=22.0, mass_ev=0.93827208816e9)
    lat = synth.table([synth.elem(synth.QUAD, 0.5, k1=0.5), synth.elem(synth.DRIFT, 5.0), synth.elem(synth.MARK),
                       synth.elem(synth.QUAD, 0.5, k1=-0.5), synth.elem(synth.DRIFT, 5.0), synth.elem(synth.MARK)])
    return parts, beam, lat, (64, 64, -0.01, 0.01, -0.01, 0.01)


@pytest.mark.gpu
def test_c_program_tracks_on_the_gpu(tmp_path):
    exe = compile_program(tmp_path)
    out = tmp_path / "state.bin"
    r = subprocess.run([exe, str(out)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stderr
    parts, beam, lat, grid = c_program_inputs()
    n = len(parts["x"])
    raw = np.fromfile(out, dtype=np.float64)
    assert raw.size == 6 * n + 42
    got = dict(zip(("x", "px", "y", "py", "sigma", "psigma"), raw[:6 * n].reshape(6, n)))
    diag = raw[6 * n:].reshape(3, 14)
    ref = oracle.copy_state(parts)
    mom = []
    oracle.track(oracle.Geometry(*grid), ref, beam, lat, 3, diag=lambda t, s: mom.append(oracle.moments(s)))
    # three turns of the float64 form: every coordinate within 1e-10 of its rms, the moments within 1e-9
    for k in got:
        scale = np.sqrt(np.mean(ref[k] ** 2))
        assert np.max(np.abs(got[k] - ref[k])) / scale < 1e-10, k
    mom = np.array(mom)
    assert np.max(np.abs(diag - mom) / (np.abs(mom) + 1e-30)) < 1e-9
