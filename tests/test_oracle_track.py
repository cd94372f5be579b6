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
