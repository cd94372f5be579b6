"""Launch shape of the fused kick/push (block size, particle traversal): it
changes only the time.  Tracked turns are bit-identical for every shape; the
shape chosen by timing at capture leaves the particles, the charge grid and the
out-of-grid counter as they were; the shape API rejects values out of range."""
import numpy as np
import pytest

from paper_2010_11540_gb300 import build, sc, synth
from gpu_helpers import KEYS, to_gpu, to_host

pytestmark = pytest.mark.gpu

N_TUNED = (1 << 18) + 4099  # above the size from which the shape is timed; ragged


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    sc.load()


def run(parts, b, grid, lat, turns, precision, shape=None, slices=None):
    g = sc.create_grid(*grid, precision=precision, slices=slices)
    if shape is not None:
        sc.set_kick_push_shape(g, *shape)
    st = to_gpu(parts)
    sc.track_turns(g, st, b, lat, turns)
    Q, _, _, n_out = sc.grid_read(g)
    return to_host(st), Q, n_out, sc.get_kick_push_shape(g)


def assert_same(a, c):
    for k in KEYS:
        assert np.array_equal(a[0][k], c[0][k]), k
    assert np.array_equal(a[1], c[1])
    assert a[2] == c[2]


@pytest.mark.parametrize("precision", ["fp64", "tf32x3"])
def test_every_shape_bit_identical(precision):
    parts, b, grid, lat = synth.workload("c2", n=N_TUNED)
    tuned = run(parts, b, grid, lat, 2, precision)
    th, tr, us = tuned[3]
    assert us > 0 and th in (384, 512, 640, 768) and tr in (0, 1)
    for shape in [(128, 0), (384, 1), (640, 0), (768, 0), (768, 1)]:
        got = run(parts, b, grid, lat, 2, precision, shape)
        assert got[3][:2] == shape and got[3][2] == 0.0  # fixed: not timed
        assert_same(got, tuned)


def test_tuned_capture_with_head_segment():
    """Elements before the first marker: the head deposits into a charge grid
    the tuner must leave cleared."""
    parts, b, grid, lat = synth.workload("c2", n=N_TUNED)
    rows = [tuple(r) for r in lat]
    k = next(i for i, r in enumerate(lat) if r["type"] == synth.MARK)
    rot = synth.table(rows[k + 1:] + rows[:k + 1])  # starts after a marker, ends with it
    assert rot[0]["type"] != synth.MARK
    tuned = run(parts, b, grid, rot, 2, "tf32x3")
    assert tuned[3][2] > 0
    fixed = run(parts, b, grid, rot, 2, "tf32x3", (768, 1))
    assert_same(fixed, tuned)


def test_sliced_grid_shapes():
    parts, b, grid, lat = synth.workload("c5", n=N_TUNED)
    sl = synth.slices("c5")
    tuned = run(parts, b, grid, lat, 1, "tf32x3", slices=sl)
    assert tuned[3][1] == 1 and tuned[3][2] > 0  # sliced grids always take chunks
    fixed = run(parts, b, grid, lat, 1, "tf32x3", (512, -1), slices=sl)
    assert fixed[3][:2] == (512, 1)
    assert_same(fixed, tuned)


def test_host_buffers_keep_the_tuned_shape():
    """The shape is chosen for the bunch's size and lattice, not for where its
    arrays live: tracking the same bunch from host buffers (through the
    library's staging copy) reuses the choice -- no second timing -- and both
    calls give the same bits."""
    parts, b, grid, lat = synth.workload("c2", n=N_TUNED)
    g = sc.create_grid(*grid, precision="tf32x3")
    st = to_gpu(parts)
    sc.track_turns(g, st, b, lat, 1)
    shape = sc.get_kick_push_shape(g)
    assert shape[2] > 0
    host = {k: np.array(parts[k], copy=True) for k in KEYS}
    sc.track_turns_host(g, host, b, lat, 1)
    assert sc.get_kick_push_shape(g) == shape
    dev = to_host(st)
    for k in KEYS:
        assert np.array_equal(host[k], dev[k]), k


def test_small_bunch_takes_default_shape():
    parts, b, grid, lat = synth.workload("c2", n=5000)
    got = run(parts, b, grid, lat, 1, "fp64")
    assert got[3] == (768, 0, 0.0)
    got = run(parts, b, grid, lat, 1, "tf32x3")
    assert got[3] == (768, 1, 0.0)


def test_shape_arguments():
    g = sc.create_grid(16, 16, -1.0, 1.0, -1.0, 1.0)
    with pytest.raises(sc.ScError):
        sc.get_kick_push_shape(g)  # nothing captured yet
    for th, tr in [(48, -1), (-32, -1), (800, -1), (1024, 0), (256, 2), (256, -2)]:
        with pytest.raises(sc.ScError):
            sc.set_kick_push_shape(g, th, tr)
    sc.set_kick_push_shape(g, 640, 0)
    g32 = sc.create_grid(64, 64, -1.0, 1.0, -1.0, 1.0, precision="tf32x3")
    sc.set_kick_push_shape(g32, 768, 1)


@pytest.mark.parametrize("precision", ["tf32x3", "bf16x3"])
def test_grids_of_one_geometry_share_the_solve_tiling(precision):
    """The split solve's tiling is timed when the first grid of a geometry is
    created on the device; later grids of that geometry take the same choice
    (a forced tiling on one grid changes only that grid), so they solve the
    same charge to the same bits -- tilings differ in FP32 summation order."""
    parts, _, grid, _ = synth.workload("c2", n=200_000)
    a = sc.create_grid(*grid, precision=precision)
    b = sc.create_grid(*grid, precision=precision)
    assert sc.get_solver_tiling(a) == sc.get_solver_tiling(b)
    forced = [1, 1, 1, 1]
    sc.set_solver_tiling(b, forced)
    assert sc.get_solver_tiling(b)[0] == forced
    c = sc.create_grid(*grid, precision=precision)
    assert sc.get_solver_tiling(c) == sc.get_solver_tiling(a)
    sc.deposit(a, to_gpu(parts))
    Q, _, _, _ = sc.grid_read(a)
    sc.grid_write_charge(c, Q, len(parts["x"]))
    sc.solve(a)
    sc.solve(c)
    Ea, Ec = sc.grid_read(a)[1:3], sc.grid_read(c)[1:3]
    assert np.array_equal(Ea[0], Ec[0]) and np.array_equal(Ea[1], Ec[1])
