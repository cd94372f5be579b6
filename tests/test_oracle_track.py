"""Host-logic pins of the oracle's PIC loop (Sec. I loop, Sec. V kick
spacing): segment lengths, the wrap-around kick length, and that with zero
line density tracking reduces to the bare push."""
import numpy as np

import oracle
from paper_2010_11540_gb300 import synth


def test_segments_c1():
    lat = synth.fodo_c1()
    head, kicks = oracle.segments(lat)
    assert len(head) == 2 and len(kicks) == 48
    assert all(abs(L - 5.5) < 1e-12 for L, _ in kicks)
    assert abs(sum(L for L, _ in kicks) - 264.0) < 1e-9


def test_segments_c2():
    lat = synth.ring_c2()
    head, kicks = oracle.segments(lat)
    assert len(head) == 0 and len(kicks) == 216
    assert all(abs(L - 8.0) < 1e-12 for L, _ in kicks)


def test_zero_intensity_is_bare_push():
    parts, b, grid, lat = synth.workload("c1", n=2000)
    b = dict(b, n_lambda=0.0)
    g = oracle.Geometry(*grid)
    a = oracle.copy_state(parts)
    oracle.track(g, a, b, lat, 2)
    c = oracle.copy_state(parts)
    oracle.push(c, lat, b)
    oracle.push(c, lat, b)
    for k in a:
        assert np.array_equal(a[k], c[k])


def test_deterministic():
    parts, b, grid, lat = synth.workload("c1", n=3000)
    g = oracle.Geometry(*grid)
    a, c = oracle.copy_state(parts), oracle.copy_state(parts)
    oracle.track(g, a, b, lat, 1)
    oracle.track(g, c, b, lat, 1)
    assert all(np.array_equal(a[k], c[k]) for k in a)


def test_threads_bit_identical():
    """The OpenMP oracle (particle loops split over threads, each thread's
    deposit into its own grid, the integer grids added afterwards) gives the
    same bits as one thread: deposit, fields and three kicks of tracking, on
    plain and sliced grids."""
    parts, b, grid, lat = synth.workload("c2", n=20011)
    g = oracle.Geometry(*grid)
    zs = oracle.Slices(4, -10.0, 10.0)
    out = []
    for n in (1, 4):
        assert oracle.set_threads(n) == n or oracle.lib().orc_max_threads() == 1
        st = oracle.copy_state(parts)
        oracle.track(g, st, b, lat, 1, max_kicks=3)
        Q, n_out = oracle.deposit(g, st["x"], st["y"])
        Qs, n_out_s = oracle.deposit_sliced(g, zs, st["x"], st["y"], st["sigma"])
        out.append((st, Q, n_out, Qs, n_out_s, oracle.solve(g, Q, len(st["x"]))))
    oracle.set_threads(1)
    (a, Qa, na, Qsa, nsa, Ea), (c, Qc, nc, Qsc, nsc, Ec) = out
    assert all(np.array_equal(a[k], c[k]) for k in a)
    assert np.array_equal(Qa, Qc) and na == nc and np.array_equal(Qsa, Qsc) and nsa == nsc
    assert np.array_equal(Ea[0], Ec[0]) and np.array_equal(Ea[1], Ec[1])
