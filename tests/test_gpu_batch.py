"""Batches of independent bunches (sc_batch_*): every bunch of a batch, with
its own particle count, grid and working point, ends a turn exactly where the
single-bunch turn driver (sc_track_turns, itself checked against the oracle)
puts it — bit for bit, since the fixed-point deposit makes the charge
independent of how particles are split over blocks — and, in the float64
form, within 1e-10 of the oracle."""
import numpy as np
import pytest

import oracle
from paper_2010_11540_gb300 import build, sc, synth
from gpu_helpers import KEYS, rel_state_err, to_gpu, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    sc.load()


def mixed_bunches(n_min=1e3, n_max=3e4):
    """Six bunches of uneven size on four grid classes: 64², 128² (two bunches
    share it), 256², and a 128² grid of another extent."""
    bunches = synth.c4_bunches(seed=777, n_bunches=6, n_min=n_min, n_max=n_max)
    ext = synth.grid_extent(4e-3, 3e-3)
    wide = synth.grid_extent(5e-3, 4e-3)
    grids = [(64, 64) + ext, (128, 128) + ext, (256, 256) + ext, (128, 128) + ext, (64, 64) + ext,
             (128, 128) + wide]
    return [(p, b, g, lat) for (p, b, _, lat), g in zip(bunches, grids)]


# one kernel variant per phase of the split-TF32 solve, forced on both sides of a
# bit-for-bit comparison (the tuner may pick different ones for a single grid
# and a stacked grid class; variants differ only in FP32 summation order)
FIXED_TILING = (0, 0, 0, 0)


def track_single(parts, b, grid, lat, turns, precision, diag=False):
    g = sc.create_grid(*grid, precision=precision)
    if precision in ("tf32x3", "bf16x3"):
        sc.set_solver_tiling(g, FIXED_TILING)
    st = to_gpu(parts)
    d = sc.track_turns(g, st, b, lat, turns, diag=diag)
    return to_host(st), d


@pytest.mark.parametrize("precision", ["fp64", "tf32x3", "bf16x3"])
def test_batch_equals_single_bunch_turns(precision):
    bunches = mixed_bunches()
    batch = sc.create_batch([g for _, _, g, _ in bunches], precision=precision)
    if precision in ("tf32x3", "bf16x3"):
        sc.batch_set_solver_tiling(batch, FIXED_TILING)  # the same summation order as the single grids
    states = [to_gpu(p) for p, _, _, _ in bunches]
    diag = sc.batch_track_turns(batch, states, [b for _, b, _, _ in bunches], [l for _, _, _, l in bunches], 2,
                                diag=True)
    assert diag.shape == (2, 6, 14)
    for i, (p, b, g, lat) in enumerate(bunches):
        ref, dref = track_single(p, b, g, lat, 2, precision, diag=True)
        got = to_host(states[i])
        for k in KEYS:
            assert np.array_equal(got[k], ref[k]), (i, k)
        assert np.array_equal(diag[:, i, :], dref), i
        # the bunch's grid holds its own fields (and n_out counter)
        Q, Ex, Ey, n_out = sc.batch_read(batch, i)
        assert Q.shape == (g[1], g[0]) and np.isfinite(Ex).all() and np.abs(Ex).max() > 0


def test_batch_fp64_matches_oracle():
    bunches = mixed_bunches(n_min=500, n_max=8000)
    batch = sc.create_batch([g for _, _, g, _ in bunches], precision="fp64")
    states = [to_gpu(p) for p, _, _, _ in bunches]
    sc.batch_track_turns(batch, states, [b for _, b, _, _ in bunches], [l for _, _, _, l in bunches], 1)
    for i, (p, b, g, lat) in enumerate(bunches):
        ref = oracle.copy_state(p)
        oracle.track(oracle.Geometry(*g), ref, b, lat, 1)
        err = rel_state_err(to_host(states[i]), ref)
        assert max(err.values()) < 1e-10, (i, err)


def test_batch_replay_and_rebuild():
    """A second call replays the captured turn; new particle arrays rebuild it."""
    bunches = mixed_bunches(n_min=500, n_max=5000)[:3]
    grids = [g for _, _, g, _ in bunches]
    beams = [b for _, b, _, _ in bunches]
    lats = [l for _, _, _, l in bunches]
    batch = sc.create_batch(grids)
    a = [to_gpu(p) for p, _, _, _ in bunches]
    sc.batch_track_turns(batch, a, beams, lats, 1)
    sc.batch_track_turns(batch, a, beams, lats, 1)
    c = [to_gpu(p) for p, _, _, _ in bunches]
    sc.batch_track_turns(batch, c, beams, lats, 2)
    for i in range(3):
        x, y = to_host(a[i]), to_host(c[i])
        for k in KEYS:
            assert np.array_equal(x[k], y[k])


def test_batch_with_an_empty_bunch():
    bunches = mixed_bunches(n_min=500, n_max=5000)[:3]
    empty = {k: np.zeros(0) for k in KEYS}
    p0, b0, g0, l0 = bunches[1]
    bunches[1] = (empty, b0, g0, l0)
    batch = sc.create_batch([g for _, _, g, _ in bunches])
    states = [to_gpu(p) for p, _, _, _ in bunches]
    sc.batch_track_turns(batch, states, [b for _, b, _, _ in bunches], [l for _, _, _, l in bunches], 1)
    for i in (0, 2):
        p, b, g, lat = bunches[i]
        ref, _ = track_single(p, b, g, lat, 1, "fp64")
        got = to_host(states[i])
        for k in KEYS:
            assert np.array_equal(got[k], ref[k])


def test_batch_rejects_mismatched_markers():
    bunches = mixed_bunches(n_min=500, n_max=2000)[:2]
    batch = sc.create_batch([g for _, _, g, _ in bunches])
    states = [to_gpu(p) for p, _, _, _ in bunches]
    with pytest.raises(sc.ScError) as e:
        sc.batch_track_turns(batch, states, [b for _, b, _, _ in bunches], [synth.ring_c2(), synth.fodo_c1()], 1)
    assert e.value.code == -1
    too_many = (sc.Bunch * 2)()
    import torch
    t = torch.zeros(1, dtype=torch.float64, device="cuda")
    for i in range(2):
        too_many[i] = sc.Bunch(sc.Particles(*(t.data_ptr(),) * 6, 1 << 24), sc.beam(bunches[i][1]), None, 0)
    assert sc.load().sc_batch_track_turns(batch.handle, too_many, 1, None) == -4


def test_batch_c4_full_size_sampled():
    """The full batching workload (64 bunches, 2.4e7 particles, 64²-256² grids,
    8x8 working points) in the launch configuration the benchmark times: one
    turn; the smallest, a middle and the largest bunch re-tracked alone
    (bit-exact), the smallest also against the oracle."""
    bunches = synth.c4_bunches()
    batch = sc.create_batch([g for _, _, g, _ in bunches], precision="tf32x3")
    sc.batch_set_solver_tiling(batch, FIXED_TILING)
    states = [to_gpu(p) for p, _, _, _ in bunches]
    sc.batch_track_turns(batch, states, [b for _, b, _, _ in bunches], [l for _, _, _, l in bunches], 1)
    counts = np.array([len(p["x"]) for p, _, _, _ in bunches])
    order = np.argsort(counts)
    for i in (order[0], order[len(order) // 2], order[-1]):
        p, b, g, lat = bunches[i]
        ref, _ = track_single(p, b, g, lat, 1, "tf32x3")
        got = to_host(states[i])
        for k in KEYS:
            assert np.array_equal(got[k], ref[k]), (i, k)
    # the smallest bunch against the oracle: split-precision statistics (rms difference)
    i = order[0]
    p, b, g, lat = bunches[i]
    ref = oracle.copy_state(p)
    oracle.track(oracle.Geometry(*g), ref, b, lat, 1)
    got = to_host(states[i])
    for k in KEYS:
        scale = np.sqrt(np.mean(ref[k] ** 2))
        d = got[k] - ref[k]
        assert np.sqrt(np.mean(d * d)) < 1e-5 * scale, k


def test_batch_host_buffers_equal_device_buffers():
    """sc_batch_track_turns_host (host arrays, copies inside the library) gives
    the bits of sc_batch_track_turns on device arrays; an empty bunch included."""
    bunches = mixed_bunches()
    bunches[4] = (synth.gaussian_bunch(0, 1, 1e-3, 1e-3, 1e-4, 1e-4),) + bunches[4][1:]
    grids = [g for _, _, g, _ in bunches]
    beams = [b for _, b, _, _ in bunches]
    lats = [l for _, _, _, l in bunches]
    B1 = sc.create_batch(grids, precision="tf32x3")
    sc.batch_set_solver_tiling(B1, FIXED_TILING)
    dev = [to_gpu(p) for p, _, _, _ in bunches]
    d1 = sc.batch_track_turns(B1, dev, beams, lats, 2, diag=True)
    B2 = sc.create_batch(grids, precision="tf32x3")
    sc.batch_set_solver_tiling(B2, FIXED_TILING)
    host = [{k: p[k].copy() for k in KEYS} for p, _, _, _ in bunches]
    d2 = sc.batch_track_turns_host(B2, host, beams, lats, 1, diag=True)
    d3 = sc.batch_track_turns_host(B2, host, beams, lats, 1, diag=True)  # device copies and plan reused
    for i in range(len(bunches)):
        got = to_host(dev[i])
        for k in KEYS:
            assert np.array_equal(host[i][k], got[k]), (i, k)
    assert np.array_equal(d1[0], d2[0], equal_nan=True) and np.array_equal(d1[1], d3[0], equal_nan=True)


def test_batch_kick_push_shapes_bit_identical():
    """The batched kick/push's block size and waves per launch change only the
    time: the shape timed at capture (a batch above 2^18 particles), and fixed
    shapes, track to the same bits; the tuner leaves the bunches as they were."""
    bunches = synth.c4_bunches(seed=99, n_bunches=8, n_min=2e4, n_max=1.2e5)
    assert sum(len(p["x"]) for p, _, _, _ in bunches) >= 1 << 18
    grids = [g for _, _, g, _ in bunches]
    beams = [b for _, b, _, _ in bunches]
    lats = [l for _, _, _, l in bunches]

    def run(shape):
        B = sc.create_batch(grids, precision="tf32x3")
        sc.batch_set_solver_tiling(B, FIXED_TILING)
        if shape is not None:
            sc.batch_set_kick_push_shape(B, *shape)
        st = [to_gpu(p) for p, _, _, _ in bunches]
        sc.batch_track_turns(B, st, beams, lats, 2)
        return [to_host(x) for x in st], sc.batch_get_kick_push_shape(B)

    tuned, (th, w, us) = run(None)
    assert us > 0 and th in (512, 768) and w in (1, 2, 4, 8)
    for shape in [(768, 4), (512, 1), (256, 8), (768, 2)]:
        got, sh = run(shape)
        assert sh[:2] == shape and sh[2] == 0.0
        for i in range(len(bunches)):
            for k in KEYS:
                assert np.array_equal(got[i][k], tuned[i][k]), (shape, i, k)


def test_batch_host_buffers_keep_the_tuned_shape():
    """A batch tracked from host buffers (the library's staging copies) keeps
    the kick/push shape timed for the same bunches in device buffers, and gives
    the same bits."""
    bunches = synth.c4_bunches(seed=99, n_bunches=8, n_min=2e4, n_max=1.2e5)
    grids = [g for _, _, g, _ in bunches]
    beams = [b for _, b, _, _ in bunches]
    lats = [l for _, _, _, l in bunches]
    B = sc.create_batch(grids, precision="tf32x3")
    sc.batch_set_solver_tiling(B, FIXED_TILING)
    st = [to_gpu(p) for p, _, _, _ in bunches]
    sc.batch_track_turns(B, st, beams, lats, 1)
    shape = sc.batch_get_kick_push_shape(B)
    assert shape[2] > 0
    host = [{k: np.array(p[k], copy=True) for k in KEYS} for p, _, _, _ in bunches]
    sc.batch_track_turns_host(B, host, beams, lats, 1)
    assert sc.batch_get_kick_push_shape(B) == shape
    for i, x in enumerate(st):
        got = to_host(x)
        for k in KEYS:
            assert np.array_equal(host[i][k], got[k]), (i, k)


def test_batch_shape_arguments():
    bunches = mixed_bunches()[:2]
    B = sc.create_batch([g for _, _, g, _ in bunches], precision="tf32x3")
    with pytest.raises(sc.ScError):
        sc.batch_get_kick_push_shape(B)  # nothing captured yet
    for th, w in [(48, 0), (800, 0), (-32, 0), (256, 65), (256, -1)]:
        with pytest.raises(sc.ScError):
            sc.batch_set_kick_push_shape(B, th, w)
    sc.batch_set_kick_push_shape(B, 768, 3)
    B64 = sc.create_batch([g for _, _, g, _ in bunches], precision="fp64")
    with pytest.raises(sc.ScError):
        sc.batch_set_kick_push_shape(B64, 768, 0)  # the float64 batched kernel stops at 640
    sc.batch_set_kick_push_shape(B64, 640, 0)
