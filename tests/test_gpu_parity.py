"""GPU (libsc, sm_103a) vs the FP64 CPU oracle on the same seeded inputs,
through the C-ABI.  Tolerances: charge grid bit-exact; float64 fields 1e-12
relative L2; single-step and one-turn coordinates 1e-10 relative (per
coordinate, to its rms)."""
import numpy as np
import pytest

import oracle
from paper_2010_11540_gb300 import build, sc, synth
from gpu_helpers import KEYS, rel_l2, rel_state_err, to_gpu, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    sc.load()


def grid_pair(geom_args, precision="fp64"):
    return sc.create_grid(*geom_args, precision=precision), oracle.Geometry(*geom_args)


# ------------------------------------------------------------------ deposit
@pytest.mark.parametrize("n,grid", [
    (20000, (64, 64, -0.01, 0.01, -0.01, 0.01)),     # c1 size
    (12345, (32, 16, -0.012, 0.009, -0.007, 0.008)),  # ragged count, non-square, beam past the edge
    (1, (8, 8, -1.0, 1.0, -1.0, 1.0)),
])
def test_deposit_bit_exact(n, grid):
    parts = synth.gaussian_bunch(n, 12345 + n, 3e-3, 2.5e-3, 1e-4, 1e-4)
    g, og = grid_pair(grid)
    sc.deposit(g, to_gpu(parts))
    Q, _, _, n_out = sc.grid_read(g)
    Qo, n_out_o = oracle.deposit(og, parts["x"], parts["y"])
    assert np.array_equal(Q, Qo)
    assert n_out == n_out_o


def test_deposit_bit_exact_full_size():
    """1e6 particles on 128x128 (the bench workload's grid)."""
    parts, b, grid, lat = synth.workload("c2")
    g, og = grid_pair(grid)
    sc.deposit(g, to_gpu(parts))
    Q, _, _, n_out = sc.grid_read(g)
    Qo, n_out_o = oracle.deposit(og, parts["x"], parts["y"])
    assert np.array_equal(Q, Qo) and n_out == n_out_o
    assert Q.sum() == (len(parts["x"]) - n_out) * (1 << 40)


def test_deposit_edge_cases():
    g, og = grid_pair((8, 8, 0.0, 7.0, 0.0, 7.0))
    x = np.array([7.0, -1e-12, 3.0, np.nan, 6.999999, 3.0, 3.0, 0.0])
    y = np.array([3.0, 3.0, 7.0, 1.0, 6.999999, np.inf, 0.0, 0.0])
    st = {k: np.zeros(len(x)) for k in KEYS}
    st["x"], st["y"] = x, y
    sc.deposit(g, to_gpu(st))
    # the NaN and the infinity are reported once (SC_ERR_NAN), then the count is clear
    with pytest.raises(sc.ScError, match="SC_ERR_NAN"):
        sc.grid_read(g)
    Q, _, _, n_out = sc.grid_read(g)
    Qo, n_out_o = oracle.deposit(og, x, y)
    assert np.array_equal(Q, Qo) and n_out == n_out_o == 5
    # empty deposit zeroes the grid
    sc.deposit(g, to_gpu({k: np.zeros(0) for k in KEYS}))
    assert not sc.grid_read(g)[0].any()


def test_overflow_rejected():
    import torch
    g = sc.create_grid(8, 8, 0.0, 1.0, 0.0, 1.0)
    t = torch.zeros(1, dtype=torch.float64, device="cuda")
    p = sc.Particles(*(t.data_ptr(),) * 6, 1 << 24)
    import ctypes
    code = sc.load().sc_deposit(g.handle, ctypes.byref(p))
    assert code == -4


# ------------------------------------------------------------------ solve
@pytest.mark.parametrize("grid", [(64, 64, -0.01, 0.01, -0.01, 0.01), (32, 16, -0.012, 0.009, -0.007, 0.008),
                                  (128, 128, -0.02, 0.02, -0.015, 0.015)])
def test_solve_fp64_matches_oracle(grid):
    parts = synth.gaussian_bunch(200000, 77, 4e-3, 3e-3, 1e-4, 1e-4)
    g, og = grid_pair(grid)
    Qo, _ = oracle.deposit(og, parts["x"], parts["y"])
    sc.grid_write_charge(g, Qo, len(parts["x"]))
    sc.solve(g)
    _, Ex, Ey, _ = sc.grid_read(g)
    Exo, Eyo = oracle.solve(og, Qo, len(parts["x"]))
    assert rel_l2(Ex, Exo) < 1e-12 and rel_l2(Ey, Eyo) < 1e-12


def test_solve_point_charge_corner():
    """A charge in a corner node exercises the wrap-around of the doubled grid."""
    grid = (16, 16, 0.0, 1.0, 0.0, 1.0)
    g, og = grid_pair(grid)
    Q = np.zeros((16, 16), dtype=np.int64)
    Q[0, 0] = 1 << 40
    Q[15, 15] = 3 << 40
    sc.grid_write_charge(g, Q, 4)
    sc.solve(g)
    _, Ex, Ey, _ = sc.grid_read(g)
    Exo, Eyo = oracle.solve(og, Q, 4)
    assert rel_l2(Ex, Exo) < 1e-12 and rel_l2(Ey, Eyo) < 1e-12


# ------------------------------------------------------------------ kick + push
def _one_step(parts, b, grid, elems, L, n_next=True):
    g, og = grid_pair(grid)
    st = to_gpu(parts)
    sc.deposit(g, st)
    sc.solve(g)
    sc.kick_push(g, st, b, L, elems, next_grid=g if n_next else None)
    got = to_host(st)
    Qg = sc.grid_read(g)[0]
    ref = oracle.copy_state(parts)
    Qo, _ = oracle.deposit(og, ref["x"], ref["y"])
    Ex, Ey = oracle.solve(og, Qo, len(ref["x"]))
    oracle.kick(og, ref, Ex, Ey, oracle.kick_strength(b) * L)
    oracle.push(ref, elems, b)
    return got, ref, Qg, og


@pytest.mark.parametrize("n", [20000, 4099])
def test_kick_push_c2_segments(n):
    parts, b, grid, lat = synth.workload("c2", n=n)
    b = dict(b, n_lambda=5e11)  # strong space charge so the kick is visible
    head, kicks = oracle.segments(lat)
    for L, seg in kicks[:3]:
        got, ref, Qg, og = _one_step(parts, b, grid, seg, L)
        err = rel_state_err(got, ref)
        assert max(err.values()) < 1e-10, err
        Qn, _ = oracle.deposit(og, got["x"], got["y"])
        assert np.array_equal(Qg, Qn)  # fused deposit of the pushed state


def test_kick_push_every_element_type():
    parts, b, grid, lat = synth.workload("c1", n=5000)
    b = dict(b, circumference=264.0)
    elems = synth.table([
        synth.elem(synth.DRIFT, 2.0), synth.elem(synth.QUAD, 0.7, k1=1.1), synth.elem(synth.QUAD, 0.7, k1=-0.9),
        synth.elem(synth.QUAD, 0.3, k1=0.0), synth.elem(synth.SEXT, k2l=3.0),
        synth.elem(synth.BEND, 1.5, angle=0.1), synth.elem(synth.BEND, 1.0, angle=0.0),
        synth.elem(synth.RF, volt=2e5, harmonic=9.0, lag=0.3), synth.elem(synth.MARK),
    ])
    got, ref, _, _ = _one_step(parts, b, grid, elems, 5.5)
    err = rel_state_err(got, ref)
    assert max(err.values()) < 1e-10, err


def test_kick_push_exact_bend_and_thick_sextupole():
    """The exact sector dipole (both signs, zero angle) and the thick Eq. Sym2
    sextupole, with an RF cavity between them (psigma-dependent quantities
    refreshed mid-segment), against the oracle."""
    parts, b, grid, lat = synth.workload("c1", n=5000)
    b = dict(b, circumference=264.0)
    elems = synth.table([
        synth.elem(synth.EXACT_BEND, 1.5, angle=0.1), synth.elem(synth.SEXT, 0.4, k2l=4.0),
        synth.elem(synth.RF, volt=2e5, harmonic=9.0, lag=0.3), synth.elem(synth.EXACT_BEND, 2.0, angle=-0.05),
        synth.elem(synth.EXACT_BEND, 1.0, angle=0.0), synth.elem(synth.SEXT, 0.25, k2l=-6.0),
        synth.elem(synth.DRIFT, 1.0),
    ])
    got, ref, _, _ = _one_step(parts, b, grid, elems, 5.5)
    err = rel_state_err(got, ref)
    assert max(err.values()) < 1e-10, err


# ------------------------------------------------------------------ tracking
def test_track_c1_full():
    """Config c1 in full: 2e4 particles, 64x64, 48 kicks/turn, 10 turns."""
    parts, b, grid, lat = synth.workload("c1")
    g, og = grid_pair(grid)
    st = to_gpu(parts)
    diag = sc.track_turns(g, st, b, lat, 10, diag=True)
    got = to_host(st)
    ref = oracle.copy_state(parts)
    mom = []
    oracle.track(og, ref, b, lat, 10, diag=lambda t, s: mom.append(oracle.moments(s)))
    err = rel_state_err(got, ref)
    assert max(err.values()) < 1e-10, err
    mom = np.array(mom)
    assert np.max(np.abs(diag - mom) / (np.abs(mom) + 1e-30)) < 1e-9


def test_track_graph_replay_consistent():
    """Two calls of 1 turn equal one call of 2 turns (captured graph reused)."""
    parts, b, grid, lat = synth.workload("c1", n=3000)
    g = sc.create_grid(*grid)
    a = to_gpu(parts)
    sc.track_turns(g, a, b, lat, 1)
    sc.track_turns(g, a, b, lat, 1)
    g2 = sc.create_grid(*grid)
    c = to_gpu(parts)
    sc.track_turns(g2, c, b, lat, 2)
    for k in KEYS:
        assert np.array_equal(a[k].cpu().numpy(), c[k].cpu().numpy())


def test_track_c2_one_turn_full_size():
    """The bench workload (1e6 particles, 128x128, 216 kicks) for one turn."""
    parts, b, grid, lat = synth.workload("c2")
    g, og = grid_pair(grid)
    st = to_gpu(parts)
    sc.track_turns(g, st, b, lat, 1)
    got = to_host(st)
    ref = oracle.copy_state(parts)
    oracle.track(og, ref, b, lat, 1)
    err = rel_state_err(got, ref)
    assert max(err.values()) < 1e-10, err


def test_kick_push_long_segment():
    """More elements than fit in the launch parameters (device-array path)."""
    parts, b, grid, lat = synth.workload("c1", n=3000)
    b = dict(b, circumference=264.0)
    cell = [synth.elem(synth.QUAD, 0.4, k1=0.9), synth.elem(synth.DRIFT, 1.0), synth.elem(synth.SEXT, k2l=0.5),
            synth.elem(synth.QUAD, 0.4, k1=-0.9), synth.elem(synth.DRIFT, 1.0), synth.elem(synth.BEND, 0.8, angle=0.02)]
    elems = synth.table(cell * 6)
    got, ref, _, _ = _one_step(parts, b, grid, elems, 2.0)
    err = rel_state_err(got, ref)
    assert max(err.values()) < 1e-10, err


def test_quads_large_momentum_offsets():
    """psigma up to +-0.3 drives the chromatic phase shift of the quadrupole
    past the series range into the library-trig branch."""
    parts, b, grid, lat = synth.workload("c1", n=4096)
    rng = np.random.default_rng(5)
    parts["psigma"] = rng.uniform(-0.3, 0.3, 4096)
    elems = synth.table([synth.elem(synth.QUAD, 1.0, k1=0.8), synth.elem(synth.QUAD, 1.0, k1=-1.3),
                         synth.elem(synth.QUAD, 0.5, k1=0.0), synth.elem(synth.DRIFT, 3.0)])
    got, ref, _, _ = _one_step(parts, b, grid, elems, 0.0)
    err = rel_state_err(got, ref)
    assert max(err.values()) < 1e-10, err


# ------------------------------------------------------------------ split-TF32 tensor-core solve
@pytest.mark.parametrize("n", [64, 128, 256])
def test_solve_tf32_fields_within_1e5(n):
    parts = synth.gaussian_bunch(1000000, 31 + n, 4e-3, 3e-3, 1e-4, 1e-4)
    grid = (n, n, -0.02, 0.02, -0.015, 0.015)
    g = sc.create_grid(*grid, precision="tf32x3")
    og = oracle.Geometry(*grid)
    Qo, _ = oracle.deposit(og, parts["x"], parts["y"])
    sc.grid_write_charge(g, Qo, len(parts["x"]))
    sc.solve(g)
    _, Ex, Ey, _ = sc.grid_read(g)
    Exo, Eyo = oracle.solve(og, Qo, len(parts["x"]))
    assert rel_l2(Ex, Exo) < 1e-5 and rel_l2(Ey, Eyo) < 1e-5, (rel_l2(Ex, Exo), rel_l2(Ey, Eyo))
    # a second solve on the same grid gives the same fields (no state leaks between solves)
    sc.solve(g)
    _, Ex2, Ey2, _ = sc.grid_read(g)
    assert np.array_equal(Ex, Ex2) and np.array_equal(Ey, Ey2)


# candidates per phase of the split-TF32 solve (row DFT, column DFT, inverse column DFT, inverse row DFT)
TILING_VARIANTS = (4, 5, 5, 4)


@pytest.mark.parametrize("n,nz", [(64, 1), (128, 1), (256, 1), (128, 3), (64, 5)])
def test_solve_tf32_every_tiling(n, nz):
    """Every kernel variant the tuner may pick, phase by phase, on single and
    stacked (sliced) grids: fields within 1e-5 of the oracle; variants that do
    not fit the grid are refused."""
    parts = synth.gaussian_bunch(200000, 5 + n + nz, 4e-3, 3e-3, 1e-4, 1e-4, sig_z=15.0)
    grid = (n, n, -0.02, 0.02, -0.015, 0.015)
    sl = None if nz == 1 else (nz, -60.0, 60.0)
    g = sc.create_grid(*grid, precision="tf32x3", slices=sl)
    og = oracle.Geometry(*grid)
    if sl is None:
        Qo, _ = oracle.deposit(og, parts["x"], parts["y"])
        Exo, Eyo = oracle.solve(og, Qo, len(parts["x"]))
    else:
        Qo, _ = oracle.deposit_sliced(og, oracle.Slices(*sl), parts["x"], parts["y"], parts["sigma"])
        Exo, Eyo = oracle.solve_sliced(og, Qo, len(parts["x"]))
    tuned, desc = sc.get_solver_tiling(g)
    assert all(0 <= v < c for v, c in zip(tuned, TILING_VARIANTS)) and "columns" in desc
    tried = 0
    for ph in range(4):
        for k in range(TILING_VARIANTS[ph]):
            choice = list(tuned)
            choice[ph] = k
            try:
                sc.set_solver_tiling(g, choice)
            except sc.ScError as e:
                assert e.code == -1  # does not fit this grid
                continue
            tried += 1
            sc.grid_write_charge(g, Qo, len(parts["x"]))
            sc.solve(g)
            _, Ex, Ey, _ = sc.grid_read(g)
            assert rel_l2(Ex, Exo) < 1e-5 and rel_l2(Ey, Eyo) < 1e-5, (ph, k, rel_l2(Ex, Exo))
    assert tried >= 12
    with pytest.raises(sc.ScError):
        sc.set_solver_tiling(g, [99, -1, -1, -1])


# The split-precision tolerance: the BF16 hi + lo split keeps 16 significant
# bits of each operand, but the products' 2^-16 errors are random and the
# FP32 accumulation of long sums dominates in both split forms (measured
# 4-6e-6 for BF16 and 2-5e-6 for TF32 on these grids).
BF16_FIELD_TOL = 1e-5


@pytest.mark.parametrize("n,nz", [(64, 1), (128, 1), (256, 1), (128, 3)])
def test_solve_bf16_every_tiling(n, nz):
    """The open-boundary solve with BF16 split operands (kind::f16 MMAs),
    every tiling variant phase by phase, single and stacked grids: fields
    within 1e-5 of the oracle (relative L2), as the TF32 form's on the same
    charge (the measured errors of both are printed)."""
    parts = synth.gaussian_bunch(200000, 9 + n + nz, 4e-3, 3e-3, 1e-4, 1e-4, sig_z=15.0)
    grid = (n, n, -0.02, 0.02, -0.015, 0.015)
    sl = None if nz == 1 else (nz, -60.0, 60.0)
    g = sc.create_grid(*grid, precision="bf16x3", slices=sl)
    og = oracle.Geometry(*grid)
    if sl is None:
        Qo, _ = oracle.deposit(og, parts["x"], parts["y"])
        Exo, Eyo = oracle.solve(og, Qo, len(parts["x"]))
    else:
        Qo, _ = oracle.deposit_sliced(og, oracle.Slices(*sl), parts["x"], parts["y"], parts["sigma"])
        Exo, Eyo = oracle.solve_sliced(og, Qo, len(parts["x"]))
    tuned, desc = sc.get_solver_tiling(g)
    errs = []
    for ph in range(4):
        for k in range(TILING_VARIANTS[ph]):
            choice = list(tuned)
            choice[ph] = k
            try:
                sc.set_solver_tiling(g, choice)
            except sc.ScError as e:
                assert e.code == -1
                continue
            sc.grid_write_charge(g, Qo, len(parts["x"]))
            sc.solve(g)
            _, Ex, Ey, _ = sc.grid_read(g)
            errs.append(max(rel_l2(Ex, Exo), rel_l2(Ey, Eyo)))
            assert errs[-1] < BF16_FIELD_TOL, (ph, k, errs[-1])
    g32 = sc.create_grid(*grid, precision="tf32x3", slices=sl)
    sc.grid_write_charge(g32, Qo, len(parts["x"]))
    sc.solve(g32)
    _, Ex32, Ey32, _ = sc.grid_read(g32)
    e32 = max(rel_l2(Ex32, Exo), rel_l2(Ey32, Eyo))
    print(f"bf16x3 {n}x{n}x{nz}: field rel L2 {min(errs):.3e} .. {max(errs):.3e}; tf32x3 {e32:.3e}")
    assert len(errs) >= 12 and e32 < BF16_FIELD_TOL


def test_solve_tf32_point_charges():
    """Sparse charge in the corners: the worst case for relative field error."""
    grid = (128, 128, 0.0, 1.0, 0.0, 1.0)
    g = sc.create_grid(*grid, precision="tf32x3")
    og = oracle.Geometry(*grid)
    Q = np.zeros((128, 128), dtype=np.int64)
    Q[0, 0] = 1 << 40
    Q[127, 127] = 3 << 40
    Q[64, 3] = 2 << 40
    sc.grid_write_charge(g, Q, 6)
    sc.solve(g)
    _, Ex, Ey, _ = sc.grid_read(g)
    Exo, Eyo = oracle.solve(og, Q, 6)
    assert rel_l2(Ex, Exo) < 1e-5 and rel_l2(Ey, Eyo) < 1e-5, (rel_l2(Ex, Exo), rel_l2(Ey, Eyo))


@pytest.mark.parametrize("nx,ny", [(32, 32), (512, 512), (128, 64)])
def test_tf32_unsupported_size(nx, ny):
    with pytest.raises(sc.ScError) as e:
        sc.create_grid(nx, ny, -1.0, 1.0, -1.0, 1.0, precision="tf32x3")
    assert e.value.code == -7


def test_track_tf32_statistics():
    """Split-precision form: one turn of the bench ring at 2e5 particles at the
    workload's line density: rms emittances within 1e-3 of the oracle; the rms
    over particles of each coordinate's difference within 1e-5 of that
    coordinate's rms, and no particle further off than 1e-2 of it (tail
    particles near the grid edge or in the sextupoles' nonlinear region
    amplify the 1e-6 field differences)."""
    parts, b, grid, lat = synth.workload("c2", n=200000)
    g, og = grid_pair(grid, precision="tf32x3")
    st = to_gpu(parts)
    sc.track_turns(g, st, b, lat, 1)
    got = to_host(st)
    ref = oracle.copy_state(parts)
    oracle.track(og, ref, b, lat, 1)
    eg, eo = oracle.emittances(got), oracle.emittances(ref)
    for a, c in zip(eg, eo):
        assert abs(a / c - 1) < 1e-3
    for k in KEYS:
        scale = np.sqrt(np.mean(ref[k] ** 2))
        d = got[k] - ref[k]
        assert np.sqrt(np.mean(d * d)) < 1e-5 * scale, k
        assert np.max(np.abs(d)) < 1e-2 * scale, k


def test_track_with_rf_and_head():
    """An RF cavity inside a segment changes psigma mid-push (the per-particle
    psigma-dependent quantities must follow), with elements before the first
    space-charge marker: 3 turns against the oracle."""
    parts, b, grid, lat = synth.workload("c1", n=5000)
    rows = list(lat)
    rf = synth.table([synth.elem(synth.RF, volt=4e6, harmonic=4.0, lag=0.0)])[0]
    lat2 = synth.table([tuple(rows[0]), tuple(rf)] + [tuple(r) for r in rows[1:]])
    b = dict(b, circumference=float(lat2["length"].sum()))
    g, og = grid_pair(grid)
    st = to_gpu(parts)
    sc.track_turns(g, st, b, lat2, 3)
    got = to_host(st)
    ref = oracle.copy_state(parts)
    oracle.track(og, ref, b, lat2, 3)
    err = rel_state_err(got, ref)
    assert max(err.values()) < 1e-10, err
    assert np.abs(got["psigma"] - parts["psigma"]).max() > 1e-6  # the cavity did act


def test_quad_coefficient_cache_bit_identical():
    """Tracked turns keep each particle's quadrupole matrix entries per
    quadrupole family (computed once per call and again after an RF cavity);
    the stand-alone kick/push computes them in every map.  Two turns of a
    lattice with a head segment and an RF cavity give the same bits both ways."""
    parts, b, grid, lat = synth.workload("c1", n=5000)
    rows = list(lat)
    rf = synth.table([synth.elem(synth.RF, volt=4e6, harmonic=4.0, lag=0.0)])[0]
    lat2 = synth.table([tuple(rows[0]), tuple(rf)] + [tuple(r) for r in rows[1:]])
    b = dict(b, circumference=float(lat2["length"].sum()))
    g = sc.create_grid(*grid)
    st = to_gpu(parts)
    sc.track_turns(g, st, b, lat2, 2)
    g2 = sc.create_grid(*grid)
    st2 = to_gpu(parts)
    head, kicks = oracle.segments(lat2)
    assert len(head) == 3 and len(kicks) > 1  # quad, cavity, drift
    for _ in range(2):
        sc.kick_push(g2, st2, b, 0.0, head)
        for L, seg in kicks:
            sc.deposit(g2, st2)
            sc.solve(g2)
            sc.kick_push(g2, st2, b, L, seg)
    for k in KEYS:
        assert np.array_equal(st[k].cpu().numpy(), st2[k].cpu().numpy()), k


def test_track_host_buffers_equal_device_buffers():
    """sc_track_turns_host (host numpy arrays, copies inside the library) gives
    the bits of sc_track_turns on device arrays; repeated calls reuse the
    library's device copies and captured turn."""
    parts, b, grid, lat = synth.workload("c1", n=7001)
    g = sc.create_grid(*grid)
    st = to_gpu(parts)
    d1 = sc.track_turns(g, st, b, lat, 3, diag=True)
    g2 = sc.create_grid(*grid)
    host = {k: parts[k].copy() for k in KEYS}
    d2 = sc.track_turns_host(g2, host, b, lat, 2, diag=True)
    d3 = sc.track_turns_host(g2, host, b, lat, 1, diag=True)
    got = to_host(st)
    for k in KEYS:
        assert np.array_equal(host[k], got[k]), k
    assert np.array_equal(d1[:2], d2) and np.array_equal(d1[2:], d3)
    with pytest.raises(ValueError):
        sc.track_turns_host(g2, {k: v.astype(np.float32) for k, v in host.items()}, b, lat, 1)


def test_track_without_space_charge_markers():
    parts, b, grid, lat = synth.workload("c1", n=3000)
    lat2 = lat[lat["type"] != synth.MARK]
    g = sc.create_grid(*grid)
    st = to_gpu(parts)
    sc.track_turns(g, st, b, lat2, 2)
    got = to_host(st)
    ref = oracle.copy_state(parts)
    oracle.push(ref, lat2, b)
    oracle.push(ref, lat2, b)
    err = rel_state_err(got, ref)
    assert max(err.values()) < 1e-10, err


def test_trace_accumulates_phase_times():
    parts, b, grid, lat = synth.workload("c1", n=4096)
    g = sc.create_grid(*grid)
    st = to_gpu(parts)
    sc.trace_enable(g, True)
    sc.track_turns(g, st, b, lat, 2)
    kp, sv, n = sc.trace_read(g)
    assert n == 2 * 48 and kp > 0 and sv > 0
    assert sc.trace_read(g)[2] == 0  # reading resets
    sc.trace_enable(g, False)
    a = to_host(st)
    # traced tracking gives the same state as untraced
    g2 = sc.create_grid(*grid)
    st2 = to_gpu(parts)
    sc.track_turns(g2, st2, b, lat, 2)
    c = to_host(st2)
    assert all(np.array_equal(a[k], c[k]) for k in KEYS)


# ------------------------------------------------------------------ 256x256 grids (no shared-memory tile)
def test_deposit_bit_exact_256():
    """4e6 particles on a 256x256 grid: the 512 KB int64 grid exceeds a block's
    shared memory, so the deposit accumulates straight into global memory."""
    parts = synth.gaussian_bunch(4000000, 99, 4e-3, 3e-3, 2e-4, 2e-4)
    grid = (256, 256) + synth.grid_extent(4e-3, 3e-3)
    g, og = grid_pair(grid)
    sc.deposit(g, to_gpu(parts))
    Q, _, _, n_out = sc.grid_read(g)
    Qo, n_out_o = oracle.deposit(og, parts["x"], parts["y"])
    assert np.array_equal(Q, Qo) and n_out == n_out_o


@pytest.mark.parametrize("precision", ["fp64", "tf32x3"])
def test_track_256_one_turn(precision):
    """c3-sized grid (256x256) with 5e5 particles, one turn of the c2 ring."""
    parts, b, _, lat = synth.workload("c2", n=500000)
    grid = (256, 256) + synth.grid_extent(4e-3, 3e-3)
    g, og = grid_pair(grid, precision=precision)
    st = to_gpu(parts)
    sc.track_turns(g, st, b, lat, 1)
    got = to_host(st)
    ref = oracle.copy_state(parts)
    oracle.track(og, ref, b, lat, 1)
    if precision == "fp64":
        err = rel_state_err(got, ref)
        assert max(err.values()) < 1e-10, err
    else:
        for k in KEYS:
            scale = np.sqrt(np.mean(ref[k] ** 2))
            d = got[k] - ref[k]
            assert np.sqrt(np.mean(d * d)) < 1e-5 * scale, k


def test_tunes_match_oracle_phase_advance():
    """Per-particle tunes (Sec. V: one-turn phase advance) accumulated on the GPU
    over 8 turns with space charge equal the oracle's, and without space charge
    equal the bare tune from the one-turn matrix."""
    import torch
    parts, b, grid, lat = synth.workload("c1", n=4096)
    M = oracle.one_turn_matrix(lat, b)
    mux, bx, ax = oracle.twiss_from_matrix(M[:2, :2])
    muy, by, ay = oracle.twiss_from_matrix(M[2:, 2:])
    for n_lambda in (b["n_lambda"], 0.0):
        bb = dict(b, n_lambda=n_lambda)
        g, og = grid_pair(grid)
        st = to_gpu(parts)
        acc = torch.zeros(4 * 4096, dtype=torch.float64, device="cuda")
        sc.tune_setup(g, st, (bx, ax, by, ay), acc)
        sc.track_turns(g, st, bb, lat, 8)
        qx, qy = sc.tunes(acc, 4096, 8)
        pa = oracle.PhaseAdvance(bx, ax, by, ay)
        ref = oracle.copy_state(parts)
        oracle.track(og, ref, bb, lat, 8, diag=pa)
        pa(8, ref)
        rqx, rqy = pa.tunes()
        assert np.mean(np.abs(qx - rqx) < 1e-9) > 0.999 and np.mean(np.abs(qy - rqy) < 1e-9) > 0.999
        if n_lambda == 0.0:
            # chromatic spread only: mean tune = bare tune to the psigma spread
            assert abs(np.median(qx) - mux / (2 * np.pi)) < 2e-3


# ------------------------------------------------------------------ longitudinal slices (2.5-D, batched solves)
def sliced_pair(grid, sl, precision="fp64"):
    return (sc.create_grid(*grid, precision=precision, slices=sl), oracle.Geometry(*grid), oracle.Slices(*sl))


@pytest.mark.parametrize("sorted_", [True, False])
def test_sliced_deposit_bit_exact(sorted_):
    """c5 layout: 2e6 particles in 32 slices of 128x128; sorted by sigma (tile
    path) and shuffled (mostly direct global accumulation)."""
    parts, b, grid, lat = synth.workload("c5", n=2000000)
    if not sorted_:
        perm = np.random.default_rng(1).permutation(len(parts["x"]))
        parts = {k: np.ascontiguousarray(v[perm]) for k, v in parts.items()}
    g, og, zs = sliced_pair(grid, synth.slices("c5"))
    sc.deposit(g, to_gpu(parts))
    Q, _, _, n_out = sc.grid_read(g)
    Qo, n_out_o = oracle.deposit_sliced(og, zs, parts["x"], parts["y"], parts["sigma"])
    assert Q.shape == (32, 128, 128)
    assert np.array_equal(Q, Qo) and n_out == n_out_o


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("tf32x3", 1e-5)])
def test_sliced_solve(precision, tol):
    parts, b, grid, lat = synth.workload("c5", n=1000000)
    sl = (8, -60.0, 60.0)
    g, og, zs = sliced_pair(grid, sl, precision)
    Qo, _ = oracle.deposit_sliced(og, zs, parts["x"], parts["y"], parts["sigma"])
    sc.grid_write_charge(g, Qo, len(parts["x"]))
    sc.solve(g)
    _, Ex, Ey, _ = sc.grid_read(g)
    Exo, Eyo = oracle.solve_sliced(og, Qo, len(parts["x"]))
    for k in range(8):
        assert rel_l2(Ex[k], Exo[k]) < tol and rel_l2(Ey[k], Eyo[k]) < tol, (k, rel_l2(Ex[k], Exo[k]))


@pytest.mark.parametrize("precision", ["fp64", "tf32x3"])
def test_sliced_track_one_turn(precision):
    """2e5 particles in 8 slices, one turn of the c2 ring, against the oracle."""
    parts, b, grid, lat = synth.workload("c5", n=200000)
    sl = (8, -60.0, 60.0)
    b = dict(b, n_lambda=b["n_lambda"] * 32 / 8 / 100)  # moderate space charge for a per-particle check
    g, og, zs = sliced_pair(grid, sl, precision)
    st = to_gpu(parts)
    sc.track_turns(g, st, b, lat, 1)
    got = to_host(st)
    ref = oracle.copy_state(parts)
    oracle.track(og, ref, b, lat, 1, slices=zs)
    if precision == "fp64":
        err = rel_state_err(got, ref)
        assert max(err.values()) < 1e-10, err
    else:
        for k in KEYS:
            scale = np.sqrt(np.mean(ref[k] ** 2))
            d = got[k] - ref[k]
            assert np.sqrt(np.mean(d * d)) < 1e-5 * scale, k


@pytest.mark.parametrize("precision", ["fp64", "tf32x3"])
def test_c5_full_size_sampled(precision):
    """The c5 workload at full size (1e7 particles sorted by sigma, 32 slices of
    128x128): the sliced deposit bit for bit; the solve (float64 1e-12, split
    form 1e-5); one space-charge step (kick, the segment up to the next
    location, the fused deposit into a second sliced grid) on every particle:
    its deposit bit for bit against the oracle's deposit of the pushed
    coordinates, and, in the float64 form, 20000 sampled particles against the
    oracle's kick and push (1e-10 of each coordinate's rms)."""
    parts, b, grid, lat = synth.workload("c5")
    n = len(parts["x"])
    sl = synth.slices("c5")
    g, og, zs = sliced_pair(grid, sl, precision)
    st = to_gpu(parts)
    sc.deposit(g, st)
    Q = sc.grid_read(g)[0]
    Qo, _ = oracle.deposit_sliced(og, zs, parts["x"], parts["y"], parts["sigma"])
    assert np.array_equal(Q, Qo)
    sc.solve(g)
    _, Ex, Ey, _ = sc.grid_read(g)
    Exo, Eyo = oracle.solve_sliced(og, Qo, n)
    tol = 1e-12 if precision == "fp64" else 1e-5
    assert rel_l2(Ex, Exo) < tol and rel_l2(Ey, Eyo) < tol, (rel_l2(Ex, Exo), rel_l2(Ey, Eyo))
    _, kicks = oracle.segments(lat)
    L, seg = kicks[0]
    g2 = sc.create_grid(*grid, precision=precision, slices=sl)
    sc.kick_push(g, st, b, L, seg, next_grid=g2)
    got = to_host(st)
    Q2 = sc.grid_read(g2)[0]
    Q2o, _ = oracle.deposit_sliced(og, zs, got["x"], got["y"], got["sigma"])
    assert np.array_equal(Q2, Q2o)
    if precision == "fp64":
        idx = np.sort(np.random.default_rng(5).choice(n, 20000, replace=False))
        ref = {k: np.ascontiguousarray(parts[k][idx]) for k in KEYS}
        oracle.kick_sliced(og, zs, ref, Exo, Eyo, oracle.kick_strength(b) * L)
        oracle.push(ref, seg, b)
        err = rel_state_err({k: got[k][idx] for k in KEYS}, ref)
        assert max(err.values()) < 1e-10, err


def test_sliced_deposit_edges():
    """sigma on the slice edges, outside the range, non-finite; rejected shapes."""
    grid, sl = (8, 8, 0.0, 7.0, 0.0, 7.0), (4, -2.0, 2.0)
    g, og, zs = sliced_pair(grid, sl)
    sg = np.array([-2.0, 2.0, -1.0, 0.999999999, 1.0, np.nan, -np.inf, -2.0000001, 1.9999999999])
    st = {k: np.zeros(len(sg)) for k in KEYS}
    st["x"], st["y"], st["sigma"] = np.full(len(sg), 3.25), np.full(len(sg), 2.5), sg
    sc.deposit(g, to_gpu(st))
    with pytest.raises(sc.ScError, match="SC_ERR_NAN: 2 "):  # the NaN and the infinite sigma
        sc.grid_read(g)
    Q, _, _, n_out = sc.grid_read(g)
    Qo, n_out_o = oracle.deposit_sliced(og, zs, st["x"], st["y"], sg)
    assert np.array_equal(Q, Qo) and n_out == n_out_o == 4
    assert [int(Q[k].sum()) >> 40 for k in range(4)] == [1, 1, 1, 2]
    with pytest.raises(sc.ScError):
        sc.create_grid(8, 8, 0.0, 1.0, 0.0, 1.0, slices=(0, -1.0, 1.0))
    with pytest.raises(sc.ScError):
        sc.create_grid(8, 8, 0.0, 1.0, 0.0, 1.0, slices=(4, 1.0, 1.0))
    with pytest.raises(sc.ScError):
        sc.create_grid(4096, 4096, 0.0, 1.0, 0.0, 1.0, slices=(32, -1.0, 1.0))


# ------------------------------------------------------------------ conducting pipe (Sec. IV-B)
@pytest.mark.parametrize("grid", [(129, 129, -0.02, 0.02, -0.015, 0.015), (65, 33, -0.012, 0.009, -0.007, 0.008),
                                  (17, 17, -0.01, 0.01, -0.01, 0.01)])
def test_solve_pipe_matches_oracle(grid):
    parts = synth.gaussian_bunch(300000, 17 + grid[0], 3e-3, 2.5e-3, 1e-4, 1e-4)
    parts["x"] += 1.5e-3  # off centre: the walls act unevenly
    g = sc.create_grid(*grid, precision="pipe_fp64")
    og = oracle.Geometry(*grid)
    Qo, _ = oracle.deposit(og, parts["x"], parts["y"])
    sc.grid_write_charge(g, Qo, len(parts["x"]))
    sc.solve(g)
    _, Ex, Ey, _ = sc.grid_read(g)
    phi = sc.grid_read_potential(g)
    Exo, Eyo = oracle.solve(og, Qo, len(parts["x"]), boundary="pipe")
    phio = oracle.potential_pipe(og, oracle.normalise(Qo, len(parts["x"])))[1:-1, 1:-1]
    assert rel_l2(Ex, Exo) < 1e-12 and rel_l2(Ey, Eyo) < 1e-12, (rel_l2(Ex, Exo), rel_l2(Ey, Eyo))
    assert rel_l2(phi, phio) < 1e-12
    assert not phi[0].any() and not phi[-1].any() and not phi[:, 0].any() and not phi[:, -1].any()


def test_solve_pipe_sliced():
    parts, b, _, lat = synth.workload("c5", n=400000)
    grid = (129, 129) + synth.grid_extent(4e-3, 3e-3)
    sl = (5, -60.0, 60.0)
    g = sc.create_grid(*grid, precision="pipe_fp64", slices=sl)
    og, zs = oracle.Geometry(*grid), oracle.Slices(*sl)
    Qo, _ = oracle.deposit_sliced(og, zs, parts["x"], parts["y"], parts["sigma"])
    sc.grid_write_charge(g, Qo, len(parts["x"]))
    sc.solve(g)
    _, Ex, Ey, _ = sc.grid_read(g)
    Exo, Eyo = oracle.solve_sliced(og, Qo, len(parts["x"]), boundary="pipe")
    for k in range(5):
        assert rel_l2(Ex[k], Exo[k]) < 1e-12 and rel_l2(Ey[k], Eyo[k]) < 1e-12, k


def test_track_pipe_one_turn():
    """2e5 particles, one turn of the c2 ring, fields of a conducting pipe at
    +-5 sigma on a 129 x 129 grid, against the oracle."""
    parts, b, _, lat = synth.workload("c2", n=200000)
    grid = (129, 129) + synth.grid_extent(4e-3, 3e-3)
    g = sc.create_grid(*grid, precision="pipe_fp64")
    st = to_gpu(parts)
    sc.track_turns(g, st, b, lat, 1)
    got = to_host(st)
    ref = oracle.copy_state(parts)
    oracle.track(oracle.Geometry(*grid), ref, b, lat, 1, boundary="pipe")
    err = rel_state_err(got, ref)
    assert max(err.values()) < 1e-10, err


@pytest.mark.parametrize("n", [128, 7, 1025])
def test_pipe_unsupported_size(n):
    with pytest.raises(sc.ScError) as e:
        sc.create_grid(n, 129, -1.0, 1.0, -1.0, 1.0, precision="pipe_fp64")
    assert e.value.code in (-7, -1)


# ------------------------------------------------------------------ longitudinal kick (Sec. IV)
def test_longitudinal_kick_single_step():
    """One kick (no elements) on a sliced pipe grid: transverse and longitudinal
    momentum changes against the oracle."""
    parts, _, _, _ = synth.workload("c5", n=300000)
    grid = (65, 65) + synth.grid_extent(4e-3, 3e-3)
    sl = (12, -60.0, 60.0)
    zs = oracle.Slices(*sl)
    b = synth.beam(n_lambda=1e13 / zs.dz, circumference=1728.0)
    g = sc.create_grid(*grid, precision="pipe_fp64", slices=sl)
    sc.set_longitudinal_kick(g)
    st = to_gpu(parts)
    sc.deposit(g, st)
    sc.solve(g)
    L = 8.0
    sc.kick_push(g, st, b, L, None)
    got = to_host(st)
    og = oracle.Geometry(*grid)
    ref = oracle.copy_state(parts)
    n = len(ref["x"])
    Q, _ = oracle.deposit_sliced(og, zs, ref["x"], ref["y"], ref["sigma"])
    Ex, Ey = oracle.solve_sliced(og, Q, n, boundary="pipe")
    K = oracle.kick_strength(b)
    oracle.kick_sliced(og, zs, ref, Ex, Ey, K * L)
    oracle.kick_long(og, zs, ref, oracle.potential_sliced_pipe(og, Q, n), K * b["gamma0"] * L / (2 * zs.dz))
    for k in ("px", "py", "psigma"):
        d_got, d_ref = got[k] - parts[k], ref[k] - parts[k]
        assert np.abs(d_ref).max() > 0
        assert np.abs(d_got - d_ref).max() < 1e-10 * np.abs(d_ref).max(), k


def test_longitudinal_kick_rejected_without_pipe_slices():
    g = sc.create_grid(64, 64, -1.0, 1.0, -1.0, 1.0)
    with pytest.raises(sc.ScError) as e:
        sc.set_longitudinal_kick(g)
    assert e.value.code == -7
    g2 = sc.create_grid(65, 65, -1.0, 1.0, -1.0, 1.0, precision="pipe_fp64")
    with pytest.raises(sc.ScError):
        sc.set_longitudinal_kick(g2)


def test_track_longitudinal_one_turn():
    """2e5 particles in 8 slices of 65 x 65 pipe grids, transverse and
    longitudinal kicks, one turn of the c2 ring, against the oracle."""
    parts, _, _, lat = synth.workload("c5", n=200000)
    grid = (65, 65) + synth.grid_extent(4e-3, 3e-3)
    sl = (8, -60.0, 60.0)
    zs = oracle.Slices(*sl)
    b = synth.beam(n_lambda=1e12 / zs.dz, circumference=float(lat["length"].sum()))
    g = sc.create_grid(*grid, precision="pipe_fp64", slices=sl)
    sc.set_longitudinal_kick(g)
    st = to_gpu(parts)
    sc.track_turns(g, st, b, lat, 1)
    got = to_host(st)
    ref = oracle.copy_state(parts)
    oracle.track(oracle.Geometry(*grid), ref, b, lat, 1, slices=zs, boundary="pipe", longitudinal=True)
    err = rel_state_err(got, ref)
    assert max(err.values()) < 1e-10, err
    # the longitudinal kick did act: without it psigma ends elsewhere
    ref0 = oracle.copy_state(parts)
    oracle.track(oracle.Geometry(*grid), ref0, b, lat, 1, slices=zs, boundary="pipe")
    assert np.abs(ref0["psigma"] - ref["psigma"]).max() > 1e3 * np.abs(got["psigma"] - ref["psigma"]).max()


# ------------------------------------------------------------------ Bezier gather (Sec. IV-C)
def test_bezier_kick_single_step():
    parts, b, _, _ = synth.workload("c2", n=300000)
    grid = (129, 129) + synth.grid_extent(4e-3, 3e-3)
    b = dict(b, n_lambda=5e11)
    g = sc.create_grid(*grid, precision="pipe_fp64")
    sc.set_gather(g, "bezier")
    st = to_gpu(parts)
    sc.deposit(g, st)
    sc.solve(g)
    L = 8.0
    sc.kick_push(g, st, b, L, None)
    got = to_host(st)
    og = oracle.Geometry(*grid)
    ref = oracle.copy_state(parts)
    Q, _ = oracle.deposit(og, ref["x"], ref["y"])
    phi = oracle.potential_pipe(og, oracle.normalise(Q, len(ref["x"])))[1:-1, 1:-1]
    oracle.kick_bezier(og, None, ref, phi[None], oracle.kick_strength(b) * L)
    for k in ("px", "py"):
        d_got, d_ref = got[k] - parts[k], ref[k] - parts[k]
        assert np.abs(d_ref).max() > 0
        assert np.abs(d_got - d_ref).max() < 1e-10 * np.abs(d_ref).max(), k
    assert np.array_equal(got["psigma"], parts["psigma"])


def test_bezier_needs_a_pipe_grid():
    g = sc.create_grid(64, 64, -1.0, 1.0, -1.0, 1.0)
    with pytest.raises(sc.ScError) as e:
        sc.set_gather(g, "bezier")
    assert e.value.code == -7


def test_track_bezier_longitudinal_one_turn():
    """Sliced pipe grids, Bezier gather for the transverse and the
    longitudinal kick, one turn of the c2 ring, against the oracle."""
    parts, _, _, lat = synth.workload("c5", n=150000)
    grid = (65, 65) + synth.grid_extent(4e-3, 3e-3)
    sl = (8, -60.0, 60.0)
    zs = oracle.Slices(*sl)
    b = synth.beam(n_lambda=1e12 / zs.dz, circumference=float(lat["length"].sum()))
    g = sc.create_grid(*grid, precision="pipe_fp64", slices=sl)
    sc.set_longitudinal_kick(g)
    sc.set_gather(g, "bezier")
    st = to_gpu(parts)
    sc.track_turns(g, st, b, lat, 1)
    got = to_host(st)
    ref = oracle.copy_state(parts)
    oracle.track(oracle.Geometry(*grid), ref, b, lat, 1, slices=zs, boundary="pipe", longitudinal=True,
                 gather="bezier")
    err = rel_state_err(got, ref)
    assert max(err.values()) < 1e-10, err


# ------------------------------------------------------------------ conducting pipe, split-TF32 sine GEMMs
@pytest.mark.parametrize("n,nz", [(129, 1), (65, 1), (257, 1), (129, 4)])
def test_solve_pipe_tf32_every_tiling(n, nz):
    """The pipe solve as split-TF32 sine-transform GEMMs: fields within 1e-5
    (relative L2) of the float64 oracle for every kernel variant of every phase,
    single and stacked grids; the potential too."""
    parts = synth.gaussian_bunch(200000, 3 + n + nz, 4e-3, 3e-3, 1e-4, 1e-4, sig_z=15.0)
    parts["x"] += 1e-3
    grid = (n, n, -0.02, 0.02, -0.015, 0.015)
    sl = None if nz == 1 else (nz, -60.0, 60.0)
    g = sc.create_grid(*grid, precision="pipe_tf32x3", slices=sl)
    og = oracle.Geometry(*grid)
    N = len(parts["x"])
    if sl is None:
        Qo, _ = oracle.deposit(og, parts["x"], parts["y"])
        Exo, Eyo = oracle.solve(og, Qo, N, boundary="pipe")
        phio = oracle.potential_pipe(og, oracle.normalise(Qo, N))[1:-1, 1:-1]
    else:
        Qo, _ = oracle.deposit_sliced(og, oracle.Slices(*sl), parts["x"], parts["y"], parts["sigma"])
        Exo, Eyo = oracle.solve_sliced(og, Qo, N, boundary="pipe")
        phio = oracle.potential_sliced_pipe(og, Qo, N)
    tuned, desc = sc.get_solver_tiling(g)
    assert "sine" in desc
    tried = 0
    for ph in range(4):
        for k in range(TILING_VARIANTS[ph]):
            choice = list(tuned)
            choice[ph] = k
            try:
                sc.set_solver_tiling(g, choice)
            except sc.ScError as e:
                assert e.code == -1
                continue
            tried += 1
            sc.grid_write_charge(g, Qo, N)
            sc.solve(g)
            _, Ex, Ey, _ = sc.grid_read(g)
            assert rel_l2(Ex, Exo) < 1e-5 and rel_l2(Ey, Eyo) < 1e-5, (ph, k, rel_l2(Ex, Exo), rel_l2(Ey, Eyo))
    assert tried >= 12
    phi = sc.grid_read_potential(g)
    assert rel_l2(phi, phio) < 1e-5


def test_track_pipe_tf32_statistics():
    """One c2 turn with the split-TF32 pipe solve: rms coordinate differences
    from the float64 oracle within 1e-5 of each coordinate's rms."""
    parts, b, _, lat = synth.workload("c2", n=200000)
    grid = (129, 129) + synth.grid_extent(4e-3, 3e-3)
    g = sc.create_grid(*grid, precision="pipe_tf32x3")
    st = to_gpu(parts)
    sc.track_turns(g, st, b, lat, 1)
    got = to_host(st)
    ref = oracle.copy_state(parts)
    oracle.track(oracle.Geometry(*grid), ref, b, lat, 1, boundary="pipe")
    for k in KEYS:
        scale = np.sqrt(np.mean(ref[k] ** 2))
        d = got[k] - ref[k]
        assert np.sqrt(np.mean(d * d)) < 1e-5 * scale, k


def test_pipe_tf32_limits():
    with pytest.raises(sc.ScError) as e:
        sc.create_grid(129, 65, -1.0, 1.0, -1.0, 1.0, precision="pipe_tf32x3")
    assert e.value.code == -7
    g = sc.create_grid(33, 33, -1.0, 1.0, -1.0, 1.0, precision="pipe_tf32x3")
    with pytest.raises(sc.ScError):
        sc.set_longitudinal_kick(g)  # not sliced
    sc.set_gather(g, "bezier")


@pytest.mark.parametrize("gather", ["bilinear", "bezier"])
def test_track_pipe_tf32_longitudinal_statistics(gather):
    """The paper's 2.5-D model in the split form: sliced pipe grids, the
    longitudinal kick and the chosen gather from the float32 potential, one
    turn against the float64 oracle: rms coordinate differences within 1e-5 of
    each coordinate's rms."""
    parts, _, _, lat = synth.workload("c5", n=150000)
    grid = (65, 65) + synth.grid_extent(4e-3, 3e-3)
    sl = (8, -60.0, 60.0)
    zs = oracle.Slices(*sl)
    b = synth.beam(n_lambda=1e12 / zs.dz, circumference=float(lat["length"].sum()))
    g = sc.create_grid(*grid, precision="pipe_tf32x3", slices=sl)
    sc.set_longitudinal_kick(g)
    sc.set_gather(g, gather)
    st = to_gpu(parts)
    sc.track_turns(g, st, b, lat, 1)
    got = to_host(st)
    ref = oracle.copy_state(parts)
    oracle.track(oracle.Geometry(*grid), ref, b, lat, 1, slices=zs, boundary="pipe", longitudinal=True,
                 gather=gather)
    ref0 = oracle.copy_state(parts)
    oracle.track(oracle.Geometry(*grid), ref0, b, lat, 1, slices=zs, boundary="pipe", gather=gather)
    for k in KEYS:
        scale = np.sqrt(np.mean(ref[k] ** 2))
        d = got[k] - ref[k]
        assert np.sqrt(np.mean(d * d)) < 1e-5 * scale, k
    # the longitudinal kick's effect is resolved far above the split form's error
    d_lon = ref["psigma"] - ref0["psigma"]
    d_err = got["psigma"] - ref["psigma"]
    assert np.sqrt(np.mean(d_lon ** 2)) > 100 * np.sqrt(np.mean(d_err ** 2))


def test_solver_work_counts():
    """sc_get_solver_work: the FFT-equivalent count of the zero-padded 256²
    transform pair is exact; the split-TF32 GEMMs' count covers the four DFT
    phases (about 1.3e8 real flops, three split products), stacked grids
    scale it; the float64 forms report no tensor work."""
    ext = (-1.0, 1.0, -1.0, 1.0)
    g64 = sc.create_grid(128, 128, *ext)
    t, f = sc.solver_work(g64)
    assert t == 0.0 and f == 2 * 5 * 256 * 256 * 16
    g32 = sc.create_grid(128, 128, *ext, precision="tf32x3")
    t32, f32 = sc.solver_work(g32)
    assert f32 == f and 3 * 1.2e8 < t32 < 3 * 2.5e8
    gs = sc.create_grid(128, 128, *ext, precision="tf32x3", slices=(4, -1.0, 1.0))
    ts, fs = sc.solver_work(gs)
    assert fs == 4 * f and abs(ts / t32 - 4) < 0.5


@pytest.mark.parametrize("precision", ["fp64", "tf32x3"])
def test_sharded_bunch_through_the_charge_view(precision):
    """A bunch split in two shards, each deposited on its own grid, the grids
    summed in place through their device views (the cross-rank integer
    all-reduce, done here between two grids of one GPU) and normalised by the
    whole count: every shard grid then holds the whole bunch's charge and
    fields bit for bit, and one kick/push of each shard gives the bits of the
    unsharded kick/push."""
    import torch

    parts, b, grid, lat = synth.workload("c2", n=300001)
    n, split = len(parts["x"]), 123457
    _, kicks = oracle.segments(lat)
    L, seg = kicks[0]

    def make():
        g = sc.create_grid(*grid, precision=precision)
        if precision == "tf32x3":
            sc.set_solver_tiling(g, (0, 0, 0, 0))  # one summation order for every grid
        return g

    g_all = make()
    st_all = to_gpu(parts)
    sc.deposit(g_all, st_all)
    sc.solve(g_all)
    Q_all, Ex_all, Ey_all, _ = sc.grid_read(g_all)
    shards = [{k: v[:split].copy() for k, v in parts.items()}, {k: v[split:].copy() for k, v in parts.items()}]
    gs = [make(), make()]
    sts = [to_gpu(s) for s in shards]
    for g, st in zip(gs, sts):
        sc.deposit(g, st)
    torch.cuda.synchronize()
    views = [sc.charge_tensor(g) for g in gs]
    assert views[0].numel() == 128 * 128 and views[0].dtype == torch.int64
    total = views[0] + views[1]
    for v in views:
        v.copy_(total)
    torch.cuda.synchronize()
    for g in gs:
        sc.set_particle_count(g, n)
        sc.solve(g)
        Q, Ex, Ey, _ = sc.grid_read(g)
        assert np.array_equal(Q, Q_all) and np.array_equal(Ex, Ex_all) and np.array_equal(Ey, Ey_all)
    sc.kick_push(g_all, st_all, b, L, seg)
    for g, st in zip(gs, sts):
        sc.kick_push(g, st, b, L, seg)
    got_all = to_host(st_all)
    got = [to_host(st) for st in sts]
    for k in KEYS:
        assert np.array_equal(np.concatenate([got[0][k], got[1][k]]), got_all[k]), k
    with pytest.raises(sc.ScError):
        sc.set_particle_count(gs[0], -1)


def test_moments_off_centre_bunch():
    """Per-turn moments of a bunch whose centre sits 1e4 rms sizes off the axis
    in x and y (50 rms in px, py): computed in two passes (the means, then the
    moments of the offsets from them), they equal the oracle's within 1e-12 of
    each moment's scale (a one-pass E[x^2] - E[x]^2 would lose 8 digits here);
    so do those of the allocation-free entry point."""
    import torch
    parts, b, grid, lat = synth.workload("c1", n=20000)
    shift = {"x": 1e4, "y": 1e4, "px": 50.0, "py": 50.0}
    off = {k: np.ascontiguousarray(v + shift.get(k, 0.0) * np.std(v)) for k, v in parts.items()}
    ref = oracle.moments(off)
    # scale of each moment: |mean| for the means, sqrt(<aa><bb>) for <ab>
    pairs = [(6, 6), (6, 8), (8, 8), (9, 9), (9, 11), (11, 11), (12, 12), (13, 13)]
    scale = np.concatenate([np.abs(ref[:6]), [np.sqrt(ref[a] * ref[c]) for a, c in pairs]])
    g = sc.create_grid(*grid)
    # a marker and a drift: the moments are taken at the start of the turn (the
    # ring's quadrupoles would throw a bunch 20 m off axis out of the paraxial range)
    short = synth.table([synth.elem(synth.MARK), synth.elem(synth.DRIFT, 1.0)])
    got = sc.track_turns(g, to_gpu(off), dict(b, n_lambda=0.0), short, 1, diag=True)[0]
    assert np.all(np.abs(got - ref) <= 1e-12 * scale), (got - ref) / scale
    out = torch.full((14,), np.nan, dtype=torch.float64, device="cuda")
    sc.moments_noalloc(to_gpu(off), out)
    got2 = out.cpu().numpy()
    assert np.all(np.abs(got2 - ref) <= 1e-12 * scale), (got2 - ref) / scale


def test_nonfinite_state_reported_by_tracking():
    """A particle whose px is NaN drifts to a NaN position, which the next
    deposit finds: sc_track_turns with diagnostics (a synchronous call)
    returns SC_ERR_NAN; the other particles are tracked as without it."""
    parts, b, grid, lat = synth.workload("c1", n=2000)
    bad = oracle.copy_state(parts)
    bad["px"][7] = np.nan
    g = sc.create_grid(*grid)
    st = to_gpu(bad)
    with pytest.raises(sc.ScError, match="SC_ERR_NAN"):
        sc.track_turns(g, st, b, lat, 1, diag=True)
    got = to_host(st)
    assert np.isnan(got["x"][7]) and np.all(np.isfinite(np.delete(got["x"], 7)))


# ------------------------------------------------------------------ cell ordering and warp-combined deposits
def test_sorted_bunch_deposit_bit_exact():
    """sc_sort_particles orders the c2 bunch by cell (stable, outside last) and
    reports the permutation; the deposit of the ordered bunch -- whose warps
    combine the weights of neighbouring particles in one cell -- equals the
    oracle's deposit of the original bunch bit for bit."""
    import torch
    parts, b, grid, lat = synth.workload("c2")
    g, og = grid_pair(grid)
    st = to_gpu(parts)
    perm = torch.empty(len(parts["x"]), dtype=torch.int32, device="cuda")
    sc.sort_particles(g, st, perm)
    got = to_host(st)
    pm = perm.cpu().numpy()
    assert np.array_equal(np.sort(pm), np.arange(len(pm)))
    for k in KEYS:
        assert np.array_equal(got[k], parts[k][pm]), k
    cell = oracle.deposit_cells(og, got["x"], got["y"])
    key = np.where(cell < 0, grid[0] * grid[1], cell)
    assert np.all(np.diff(key) >= 0)
    same = np.diff(key) == 0
    assert np.all(np.diff(pm)[same] > 0)  # stable
    sc.deposit(g, st)
    Q, _, _, n_out = sc.grid_read(g)
    Qo, n_out_o = oracle.deposit(og, parts["x"], parts["y"])
    assert np.array_equal(Q, Qo) and n_out == n_out_o


@pytest.mark.parametrize("n,grid,centre", [
    (12345, (256, 256) + synth.grid_extent(4e-3, 3e-3), (0.0, 0.0)),     # window of the 256x256 grid
    (200003, (256, 256) + synth.grid_extent(4e-3, 3e-3), (0.012, -0.009)),  # beam mostly outside the window
    (4099, (64, 32, -0.01, 0.01, -0.01, 0.01), (0.0, 0.0)),
])
@pytest.mark.parametrize("ordered", [False, True])
def test_deposit_windows_and_runs_bit_exact(n, grid, centre, ordered):
    """Grids beyond the 200 KB tile deposit through a centred window of it plus
    global atomics for the rest; ordered or not, ragged counts, beams off the
    window: the charge is the oracle's bit for bit."""
    parts = synth.gaussian_bunch(n, 777 + n, 4e-3, 3e-3, 2e-4, 2e-4)
    parts["x"] += centre[0]
    parts["y"] += centre[1]
    g, og = grid_pair(grid)
    st = to_gpu(parts)
    if ordered:
        sc.sort_particles(g, st)
    sc.deposit(g, st)
    Q, _, _, n_out = sc.grid_read(g)
    Qo, n_out_o = oracle.deposit(og, parts["x"], parts["y"])
    assert np.array_equal(Q, Qo) and n_out == n_out_o


@pytest.mark.parametrize("precision", ["fp64", "tf32x3"])
def test_sorted_bunch_tracks_like_unsorted(precision):
    """A turn of the ordered bunch gives, particle by particle (through the
    permutation), the same bits as a turn of the original order: the charge is
    an integer sum and every particle's arithmetic is its own."""
    import torch
    parts, b, grid, lat = synth.workload("c2", n=200000)
    g = sc.create_grid(*grid, precision=precision)
    a = to_gpu(parts)
    sc.track_turns(g, a, b, lat, 1)
    ref = to_host(a)
    c = to_gpu(parts)
    perm = torch.empty(len(parts["x"]), dtype=torch.int32, device="cuda")
    sc.sort_particles(g, c, perm)
    sc.track_turns(g, c, b, lat, 1)
    got = to_host(c)
    pm = perm.cpu().numpy()
    for k in KEYS:
        assert np.array_equal(got[k], ref[k][pm]), k


@pytest.mark.parametrize("precision", ["fp64", "tf32x3"])
def test_sharded_turn_through_the_reduce_hook(precision):
    """The charge reduction of a sharded bunch inside the captured turn
    (sc_set_charge_reduce), on one GPU with two identical shards: the callback
    stands in for the all-reduce by doubling the grid's charge (the other rank
    holds the same particles) and the solve normalises by both shards'
    count, so the fields -- and, in the float64 form, every particle after two
    turns -- are those of the unsharded bunch.  The callback runs once per
    space-charge location, while the turn is captured."""
    import torch
    parts, b, grid, lat = synth.workload("c2", n=100000)
    n = len(parts["x"])
    g0 = sc.create_grid(*grid, precision=precision)
    a = to_gpu(parts)
    sc.track_turns(g0, a, b, lat, 2)
    ref = to_host(a)
    g1 = sc.create_grid(*grid, precision=precision)
    if precision != "fp64":  # the same GEMM tiling (summation order) on both grids
        sc.set_solver_tiling(g1, sc.get_solver_tiling(g0)[0])
    calls = []

    def reduce(q, stream):
        calls.append(q.numel())
        with torch.cuda.stream(stream):
            q.mul_(2)

    sc.set_charge_reduce(g1, reduce, 2 * n)
    c = to_gpu(parts)
    sc.track_turns(g1, c, b, lat, 2)
    got = to_host(c)
    assert calls == [grid[0] * grid[1]] * 216
    if precision == "fp64":
        for k in KEYS:
            assert np.array_equal(got[k], ref[k]), k
    else:
        for k in KEYS:
            scale = np.sqrt(np.mean(ref[k] ** 2))
            d = got[k] - ref[k]
            assert np.sqrt(np.mean(d * d)) < 1e-5 * scale, k
    # switched off: the local count normalises again (the same turn as the unsharded grid)
    sc.set_charge_reduce(g1, None, 0)
    e = to_gpu(parts)
    sc.track_turns(g1, e, b, lat, 1)
    f = to_gpu(parts)
    sc.track_turns(g0, f, b, lat, 1)
    assert all(np.array_equal(to_host(e)[k], to_host(f)[k]) for k in KEYS)
