"""Pins of the oracle's CIC deposit (Sec. IV-A, charge-assignment equation)
against facts the paper and arithmetic fix: exact charge conservation,
node/centre special cases, the paper's product weights, linearity,
permutation invariance and the exact first moment of linear weights."""
import numpy as np
import pytest

import oracle
from paper_2010_11540_gb300 import synth

UNIT = 1 << 40


def geom(n=16, m=12):
    return oracle.Geometry(n, m, -1.0, 2.0, -0.5, 0.7)


def test_charge_conservation_exact():
    g = geom()
    x, y = synth.uniform_points(5000, 1, -1.3, 2.3)
    Q, n_out = oracle.deposit(g, x, y)
    inside = ((x >= g.xmin) & (x < g.xmax) & (y >= g.ymin) & (y < g.ymax)).sum()
    assert n_out == len(x) - inside
    assert int(Q.sum()) == (len(x) - n_out) * UNIT


@pytest.mark.parametrize("i,j", [(0, 0), (3, 5), (14, 10)])
def test_particle_on_node(i, j):
    g = oracle.Geometry(16, 12, 0.0, 15.0, 0.0, 11.0)  # h = 1: nodes at integers
    Q, _ = oracle.deposit(g, np.array([float(i)]), np.array([float(j)]))
    assert Q[j, i] == UNIT and Q.sum() == UNIT


def test_particle_at_cell_centre():
    g = oracle.Geometry(8, 8, 0.0, 7.0, 0.0, 7.0)
    Q, _ = oracle.deposit(g, np.array([2.5]), np.array([4.5]))
    for (jj, ii) in [(4, 2), (4, 3), (5, 2), (5, 3)]:
        assert Q[jj, ii] == UNIT // 4
    assert Q.sum() == UNIT


def test_paper_weights():
    """Q/2^40 equals (x_{i+1}-x)(y_{j+1}-y)/(dx dy) etc. to the 2^-20 resolution."""
    g = geom()
    xs, ys = synth.uniform_points(300, 7, -0.99, 1.99)
    xs = xs[(ys > g.ymin) & (ys < g.ymax)]
    ys = ys[(ys > g.ymin) & (ys < g.ymax)]
    nodes_x, nodes_y = g.node_x, g.node_y
    for x, y in zip(xs, ys):
        i = np.searchsorted(nodes_x, x, side="right") - 1
        j = np.searchsorted(nodes_y, y, side="right") - 1
        dx = nodes_x[i + 1] - nodes_x[i]
        dy = nodes_y[j + 1] - nodes_y[j]
        want = np.zeros((g.ny, g.nx))
        want[j, i] = (nodes_x[i + 1] - x) * (nodes_y[j + 1] - y) / (dx * dy)
        want[j, i + 1] = (x - nodes_x[i]) * (nodes_y[j + 1] - y) / (dx * dy)
        want[j + 1, i] = (nodes_x[i + 1] - x) * (y - nodes_y[j]) / (dx * dy)
        want[j + 1, i + 1] = (x - nodes_x[i]) * (y - nodes_y[j]) / (dx * dy)
        Q, _ = oracle.deposit(g, np.array([x]), np.array([y]))
        assert np.max(np.abs(Q / UNIT - want)) < 2.0 ** -19


def test_outside_and_nan_counted():
    g = oracle.Geometry(8, 8, 0.0, 7.0, 0.0, 7.0)
    x = np.array([7.0, -1e-12, 3.0, np.nan, 6.999999, 3.0, 3.0])
    y = np.array([3.0, 3.0, 7.0, 1.0, 6.999999, np.inf, 0.0])
    Q, n_out = oracle.deposit(g, x, y)
    assert n_out == 5
    assert Q.sum() == 2 * UNIT
    assert Q[6, 6] + Q[6, 7] + Q[7, 6] + Q[7, 7] == UNIT


def test_linearity_and_permutation():
    g = geom()
    x, y = synth.uniform_points(4000, 3, -1.0, 1.9)
    Qa, _ = oracle.deposit(g, x[:1500], y[:1500])
    Qb, _ = oracle.deposit(g, x[1500:], y[1500:])
    Q, _ = oracle.deposit(g, x, y)
    assert np.array_equal(Qa + Qb, Q)
    perm = np.random.default_rng(0).permutation(len(x))
    Qp, _ = oracle.deposit(g, np.ascontiguousarray(x[perm]), np.ascontiguousarray(y[perm]))
    assert np.array_equal(Qp, Q)


def test_first_moment():
    """Linear (CIC) weights reproduce the particle position exactly:
    sum_nodes w x_node = x, up to the 2^-20 rounding of each fraction."""
    g = geom()
    x, y = synth.uniform_points(2000, 11, -0.9, 1.9)
    keep = (y > g.ymin) & (y < g.ymax)
    x, y = np.ascontiguousarray(x[keep]), np.ascontiguousarray(y[keep])
    Q, _ = oracle.deposit(g, x, y)
    mx = (Q.sum(axis=0) / UNIT * g.node_x).sum()
    my = (Q.sum(axis=1) / UNIT * g.node_y).sum()
    tol = len(x) * 2.0 ** -21 * max(g.hx, g.hy) * 1.01
    assert abs(mx - x.sum()) < tol and abs(my - y.sum()) < tol


def test_deposit_cells_follow_the_deposit():
    """deposit_cells names the cell each particle's four weights go to: a
    single particle's deposit lands on that cell's four nodes; outside and
    non-finite particles get -1."""
    g = oracle.Geometry(8, 6, -1.0, 1.0, -0.5, 0.7)
    rng = np.random.default_rng(5)
    x = rng.uniform(-1.2, 1.2, 300)
    y = rng.uniform(-0.7, 0.9, 300)
    x[:3] = [np.nan, 1.0, -1.0]
    cells = oracle.deposit_cells(g, x, y)
    assert cells[0] == -1 and cells[1] == -1
    for p in range(300):
        Q, n_out = oracle.deposit(g, x[p:p + 1], y[p:p + 1])
        if cells[p] < 0:
            assert n_out == 1 and not Q.any()
        else:
            j, i = divmod(int(cells[p]), g.nx)
            nz = np.argwhere(Q.reshape(g.ny, g.nx) > 0)
            assert set(map(tuple, nz)) <= {(j, i), (j, i + 1), (j + 1, i), (j + 1, i + 1)}
            assert Q[j, i] > 0 or Q[j, i + 1] > 0 or Q[j + 1, i] > 0 or Q[j + 1, i + 1] > 0
