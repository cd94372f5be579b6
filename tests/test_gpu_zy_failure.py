"""Failure detection on the GPU without a fault: the tensor-core solve's
bounded waits run out (the test hook withholds the data operand's copies the
barriers expect), the kernel reports through the grid's error word, and the
context stays usable for the next grid.  (Collected after the parity tests:
each timed-out phase waits ~2 s.)"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2010_11540_gb300 import build, sc, synth
from gpu_helpers import rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    sc.load()


def test_bounded_wait_runs_out_and_reports_timeout():
    parts = synth.gaussian_bunch(50000, 5, 3e-3, 3e-3, 1e-4, 1e-4)
    grid = (64, 64, -0.01, 0.01, -0.01, 0.01)
    og = oracle.Geometry(*grid)
    Q, _ = oracle.deposit(og, parts["x"], parts["y"])
    g = sc.create_grid(*grid, precision="tf32x3")
    sc.set_solver_tiling(g, (0, 0, 0, 0))
    L = sc.load()
    assert L.sc_test_bounded_waits(g.handle, 1) == 0
    sc.grid_write_charge(g, Q, len(parts["x"]))
    sc.solve(g)
    Qr = np.zeros((64, 64), dtype=np.uint64)
    code = L.sc_grid_read(g.handle, Qr.ctypes.data, None, None, None)
    assert code == -5  # SC_ERR_TIMEOUT, no CUDA error
    buf = ctypes.create_string_buffer(256)
    L.sc_last_error(buf, 256)
    assert b"bounded wait" in buf.value
    # the error word stays set for this grid
    assert L.sc_test_bounded_waits(g.handle, 0) == 0
    assert L.sc_grid_read(g.handle, None, None, None, None) == -5
    # the context is intact: a fresh grid solves correctly
    g2 = sc.create_grid(*grid, precision="tf32x3")
    sc.grid_write_charge(g2, Q, len(parts["x"]))
    sc.solve(g2)
    _, Ex, Ey, _ = sc.grid_read(g2)
    Exo, Eyo = oracle.solve(og, Q, len(parts["x"]))
    assert rel_l2(Ex, Exo) < 1e-5 and rel_l2(Ey, Eyo) < 1e-5
