"""Pins of the synthetic rings' linear optics (Sec. III-B quadrupole and
Sec. III-A drift, linearised on the reference orbit) against the textbook
thick-lens transfer matrices: the c2 cell's gradients (stored in synth.py,
matched by oracle/match_ring.py through the oracle's own one-turn matrix)
give the bare tunes (22.40, 20.75) the workload names, every c4 working
point gives its scan tunes, and the c1 FODO cell its phase advance; the
oracle's numerically linearised one-turn matrix agrees with the product of
the textbook matrices."""
import numpy as np
import pytest

import oracle
from paper_2010_11540_gb300 import synth


def drift(L):
    return np.array([[1.0, L], [0.0, 1.0]])


def quad(k1, L):
    """Thick quadrupole on momentum: cos/sin where k1 > 0 focuses, cosh/sinh where it defocuses."""
    if k1 > 0:
        w = np.sqrt(k1)
        return np.array([[np.cos(w * L), np.sin(w * L) / w], [-w * np.sin(w * L), np.cos(w * L)]])
    w = np.sqrt(-k1)
    return np.array([[np.cosh(w * L), np.sinh(w * L) / w], [w * np.sinh(w * L), np.cosh(w * L)]])


def cell_matrices(elems):
    """(Mx, My) of an element list at psigma = 0 (markers and thin sextupoles on
    the reference orbit act as identities)."""
    Mx, My = np.eye(2), np.eye(2)
    for e in elems:
        t, L, k1 = e[0], e[2], e[3]
        if t == synth.DRIFT:
            mx = my = drift(L)
        elif t == synth.QUAD:
            mx, my = quad(k1, L), quad(-k1, L)
        else:
            continue
        Mx, My = mx @ Mx, my @ My
    return Mx, My


def tunes(elems, n_cells):
    Mx, My = cell_matrices(elems)
    return tuple(n_cells * np.arccos(0.5 * np.trace(M)) / (2 * np.pi) for M in (Mx, My))


def test_c2_ring_bare_tunes():
    qx, qy = tunes(synth.ring_c2_cell(), 72)
    assert qx == pytest.approx(22.40, abs=1e-9) and qy == pytest.approx(20.75, abs=1e-9)


def test_c4_working_points():
    pts = synth.C4_WORKING_POINTS
    assert len(pts) == 64
    steps = np.linspace(-0.1, 0.1, 8)
    for n, (k1f, k1d) in enumerate(pts):
        qx, qy = tunes(synth.ring_c2_cell(k1f=k1f, k1d=k1d), 72)
        assert qx == pytest.approx(22.40 + steps[n // 8], abs=1e-8), n
        assert qy == pytest.approx(20.75 + steps[n % 8], abs=1e-8), n


def test_c1_cell_phase_advance():
    """The c1 FODO cell (QF 0.5 m k1 = 0.5, 5 m drifts): thick-lens phase
    advance; the thin-lens estimate sin(mu/2) = L_cell / (4 f) is close."""
    cell = [tuple(r) for r in synth.fodo_c1()[:6]]
    Mx, My = cell_matrices(cell)
    mu = np.arccos(0.5 * np.trace(Mx))
    f = 1.0 / (0.5 * 0.5)
    assert mu == pytest.approx(2 * np.arcsin(11.0 / (4 * f)), rel=0.05)
    assert np.arccos(0.5 * np.trace(My)) == pytest.approx(mu, rel=0.02)


def test_oracle_one_turn_matrix_is_the_textbook_product():
    b = synth.beam(circumference=24.0)
    cell = synth.ring_c2_cell()
    M = oracle.one_turn_matrix(synth.table(cell), b)
    Mx, My = cell_matrices(cell)
    assert np.max(np.abs(M[:2, :2] - Mx)) < 1e-7 and np.max(np.abs(M[2:, 2:] - My)) < 1e-7
    assert np.max(np.abs(M[:2, 2:])) < 1e-12 and np.max(np.abs(M[2:, :2])) < 1e-12
