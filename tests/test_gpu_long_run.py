"""Long runs and the c3 workload against the oracle, through the C-ABI.

Sec. V judges a tracking run by its beam statistics: rms emittances from the
beam moments and per-particle tunes from the one-turn phase advance.  Here
100 turns of the c2 ring (216 space-charge kicks per turn) on the c2 grid
(128x128) and on the c3 grid (256x256), 1e5 particles, are tracked by the GPU
in the float64 form and the two split-precision tensor-core forms (TF32 and
BF16 operands), and by the oracle (OpenMP on every core; bit-identical to
one thread), and compared: the rms emittances at the start of every turn and
after the last, and the rms spread of the per-particle tunes, within 1e-3
relative.  The split forms' fields differ from the oracle's by 2-6e-6
(TF32 and BF16 alike), so only these statistics (not the coordinates) are
expected to agree after many turns.  The c3 workload itself (4e6 particles on 256x256) is checked at full
size: the charge bit for bit, the fields, and one turn of the float64 form to
1e-10 per coordinate."""
import numpy as np
import pytest

import oracle
from paper_2010_11540_gb300 import build, sc, synth
from gpu_helpers import KEYS, rel_l2, rel_state_err, to_gpu, to_host

pytestmark = pytest.mark.gpu

N_LONG = 100_000
TURNS = 100
STAT_TOL = 1e-3
GRIDS = {"c2 grid 128x128": (128, 128) + synth.grid_extent(4e-3, 3e-3),
         "c3 grid 256x256": (256, 256) + synth.grid_extent(4e-3, 3e-3)}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    sc.load()
    oracle.set_threads(None)
    yield
    oracle.set_threads(1)


def emittances(m):
    """(eps_x, eps_y) from moment rows [..., 14] (Sec. V: sqrt(<uu><pp> - <up>^2))."""
    m = np.asarray(m)
    return (np.sqrt(m[..., 6] * m[..., 8] - m[..., 7] ** 2), np.sqrt(m[..., 9] * m[..., 11] - m[..., 10] ** 2))


def bare_twiss(lat, b):
    M = oracle.one_turn_matrix(lat, b)
    _, bx, ax = oracle.twiss_from_matrix(M[:2, :2])
    _, by, ay = oracle.twiss_from_matrix(M[2:, 2:])
    return bx, ax, by, ay


_reference = {}


def reference(key):
    """The oracle's 100-turn run on grid `key`: moments at the start of every
    turn and after the last, and per-particle tunes (computed once per module)."""
    if key not in _reference:
        parts, b, _, lat = synth.workload("c2", n=N_LONG)
        grid = GRIDS[key]
        tw = bare_twiss(lat, b)
        st = oracle.copy_state(parts)
        pa = oracle.PhaseAdvance(*tw)
        mom = []

        def diag(turn, s):
            mom.append(oracle.moments(s))
            pa(turn, s)

        oracle.track(oracle.Geometry(*grid), st, b, lat, TURNS, diag=diag)
        mom.append(oracle.moments(st))
        pa(TURNS, st)
        _reference[key] = dict(parts=parts, b=b, lat=lat, grid=grid, twiss=tw, moments=np.array(mom),
                               tunes=pa.tunes())
    return _reference[key]


@pytest.mark.parametrize("key", list(GRIDS))
@pytest.mark.parametrize("precision", ["fp64", "tf32x3", "bf16x3"])
def test_long_run_emittance_and_tune_spread(key, precision):
    import torch
    r = reference(key)
    g = sc.create_grid(*r["grid"], precision=precision)
    st = to_gpu(r["parts"])
    acc = torch.zeros(4 * N_LONG, dtype=torch.float64, device="cuda")
    sc.tune_setup(g, st, r["twiss"], acc)
    diag = sc.track_turns(g, st, r["b"], r["lat"], TURNS, diag=True)
    got = np.vstack([diag, oracle.moments(to_host(st))[None]])
    eg, eo = emittances(got), emittances(r["moments"])
    for a, c in zip(eg, eo):
        assert np.max(np.abs(a / c - 1)) < STAT_TOL
    # the run is not trivial: the unmatched beam's emittances change over the 100 turns
    assert max(abs(eo[0][-1] / eo[0][0] - 1), abs(eo[1][-1] / eo[1][0] - 1)) > 10 * STAT_TOL
    qx, qy = sc.tunes(acc, N_LONG, TURNS)
    rqx, rqy = r["tunes"]
    for q, rq in ((qx, rqx), (qy, rqy)):
        assert abs(np.std(q) / np.std(rq) - 1) < STAT_TOL
        assert abs(np.mean(q) - np.mean(rq)) < STAT_TOL * np.std(rq)


# ------------------------------------------------------------------ the c3 workload at full size
@pytest.fixture(scope="module")
def c3():
    return synth.workload("c3")


def test_c3_charge_and_fields_full_size(c3):
    """4e6 particles on 256x256 (512x512 padded): the charge bit for bit, the
    float64 fields within 1e-12, the split-TF32 fields within 1e-5 and the
    split-BF16 fields within 1e-5 (relative L2) of the oracle's."""
    parts, b, grid, lat = c3
    og = oracle.Geometry(*grid)
    Qo, n_out_o = oracle.deposit(og, parts["x"], parts["y"])
    Exo, Eyo = oracle.solve(og, Qo, len(parts["x"]))
    dev = to_gpu(parts)
    for precision, tol in (("fp64", 1e-12), ("tf32x3", 1e-5), ("bf16x3", 1e-5)):
        g = sc.create_grid(*grid, precision=precision)
        sc.deposit(g, dev)
        Q, _, _, n_out = sc.grid_read(g)
        assert np.array_equal(Q, Qo) and n_out == n_out_o
        sc.solve(g)
        _, Ex, Ey, _ = sc.grid_read(g)
        assert rel_l2(Ex, Exo) < tol and rel_l2(Ey, Eyo) < tol, (precision, rel_l2(Ex, Exo), rel_l2(Ey, Eyo))


def test_c3_one_turn_fp64_full_size(c3):
    """One turn of the c2 ring (216 kicks) with 4e6 particles on 256x256,
    float64 form: every coordinate within 1e-10 of the oracle (relative to
    its rms)."""
    parts, b, grid, lat = c3
    g = sc.create_grid(*grid)
    st = to_gpu(parts)
    sc.track_turns(g, st, b, lat, 1)
    got = to_host(st)
    del st
    ref = oracle.copy_state(parts)
    oracle.track(oracle.Geometry(*grid), ref, b, lat, 1)
    err = rel_state_err(got, ref)
    assert max(err.values()) < 1e-10, err
    assert all(np.all(np.isfinite(got[k])) for k in KEYS)
