"""The C-ABI used from plain C99 (no C++, no CUDA headers): the program in
tests/c_api/ compiles with -std=c99 -pedantic -Werror against include/sc.h
and links against libsc.so (CPU); on a GPU it tracks a host-memory bunch
through sc_track_turns_host and checks the moments and the error reporting."""
import os
import subprocess

import pytest

from paper_2010_11540_gb300 import build

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


@pytest.mark.gpu
def test_c_program_tracks_on_the_gpu(tmp_path):
    exe = compile_program(tmp_path)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stderr
