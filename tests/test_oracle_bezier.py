"""Pins of the oracle's Bezier gather (Sec. IV-C; control points u_{i-1..i+2},
parameter over their span): a linear potential is reproduced exactly (value
and gradient); a quadratic one is smoothed by the closed-form Bernstein amount
3 t (1 - t) h^2; a constant gives no field; a round Gaussian beam in a wide
pipe gets its closed-form field, and across it the closed-form smoothing bias
of the surface; the kick is antisymmetric for a symmetric beam."""
import numpy as np
import pytest

import oracle
from paper_2010_11540_gb300 import synth

G = oracle.Geometry(33, 17, -0.4, 0.4, -0.2, 0.2)


def node_field(f):
    x, y = np.meshgrid(G.node_x, G.node_y)
    return f(x, y)


@pytest.mark.parametrize("i,j,fx,fy", [(1, 1, 0.0, 0.0), (5, 7, 0.3, 0.8), (29, 13, 0.999, 0.01), (16, 8, 0.5, 0.5)])
def test_linear_potential_is_reproduced(i, j, fx, fy):
    a, b, c = 2.5, -1.25, 0.75
    phi = node_field(lambda x, y: a * x + b * y + c)
    u, gx, gy = oracle.bezier_point(G, phi, i, j, fx, fy)
    x = G.xmin + (i + fx) * G.hx
    y = G.ymin + (j + fy) * G.hy
    assert abs(u - (a * x + b * y + c)) < 1e-14
    assert abs(gx - a) < 1e-13 and abs(gy - b) < 1e-13


@pytest.mark.parametrize("i,fx", [(3, 0.0), (10, 0.25), (20, 0.9)])
def test_quadratic_is_smoothed_by_the_bernstein_amount(i, fx):
    phi = node_field(lambda x, y: x * x + 0 * y)
    u, gx, gy = oracle.bezier_point(G, phi, i, 6, fx, 0.4)
    x = G.xmin + (i + fx) * G.hx
    t = (1 + fx) / 3
    assert abs(u - (x * x + 3 * t * (1 - t) * G.hx ** 2)) < 1e-14
    assert abs(gx - (2 * x + G.hx * (1 - 2 * t))) < 1e-13
    assert abs(gy) < 1e-14


def test_constant_gives_no_field():
    phi = node_field(lambda x, y: 0 * x + 3.0)
    u, gx, gy = oracle.bezier_point(G, phi, 12, 5, 0.37, 0.61)
    assert abs(u - 3.0) < 1e-14 and abs(gx) < 1e-13 and abs(gy) < 1e-13


def test_round_gaussian_in_a_wide_pipe():
    g = oracle.Geometry(257, 257, -20.0, 20.0, -20.0, 20.0)
    x, y = np.meshgrid(g.node_x, g.node_y)
    q = np.exp(-(x ** 2 + y ** 2) / 2)
    q /= q.sum()
    Q = np.round(q * oracle.Q_UNIT * 1000).astype(np.uint64)
    phi = oracle.potential_pipe(g, oracle.normalise(Q, 1000))[1:-1, 1:-1]
    r = np.linspace(1.0, 2.5, 7)
    st = {k: np.zeros(len(r)) for k in ("x", "px", "y", "py", "sigma", "psigma")}
    st["x"] = r.copy()
    oracle.kick_bezier(g, None, st, phi[None], 1.0)
    Er = (1 - np.exp(-r ** 2 / 2)) / r
    np.testing.assert_allclose(st["px"], Er, rtol=2e-2)


@pytest.mark.parametrize("fy", [0.0, 0.25, 0.5])
def test_bezier_smoothing_bias_closed_form(fy):
    """Across the beam axis the Bezier gradient carries the smoothing bias of
    its cubic.  With control values f(n), n = 0..3, of a quadratic f(s) =
    s^2 (s the node index from j-1, t = s/3), the Bernstein sum is
    E[N^2] = s^2 + 3 t (1 - t) for N ~ Binomial(3, t), so its s-derivative is
    2 s + (1 - 2t): the surface's y-derivative exceeds the true one by
    u_yy h (1 - 2t) / 2.  For a round Gaussian beam (unit rms, unit charge)
    u_yy = -E_r / r on the axis, so a particle at (r, fy hy) gets
    py = E_y(r, fy hy) + (hy / 2) (1 - 2t) E_r(r) / r, t = (1 + fy)/3 -- the
    node line (fy = 0) has the largest bias, hy E_r / (6 r); mid-cell (fy =
    1/2, t = 1/2) there is none.  Holds to O(h^2) (the 5-point potential,
    quartic terms): 2% here, where the bias itself is 2-3% of px."""
    g = oracle.Geometry(257, 257, -20.0, 20.0, -20.0, 20.0)
    x, y = np.meshgrid(g.node_x, g.node_y)
    q = np.exp(-(x ** 2 + y ** 2) / 2)
    q /= q.sum()
    Q = np.round(q * oracle.Q_UNIT * 1000).astype(np.uint64)
    phi = oracle.potential_pipe(g, oracle.normalise(Q, 1000))[1:-1, 1:-1]
    r = np.linspace(1.0, 2.5, 7)
    yv = fy * g.hy
    st = {k: np.zeros(len(r)) for k in ("x", "px", "y", "py", "sigma", "psigma")}
    st["x"] = r.copy()
    st["y"][:] = yv
    oracle.kick_bezier(g, None, st, phi[None], 1.0)
    Er = (1 - np.exp(-r ** 2 / 2)) / r
    rr = np.hypot(r, yv)
    Ey = (1 - np.exp(-rr ** 2 / 2)) / rr * yv / rr
    t = (1 + fy) / 3
    bias = 0.5 * g.hy * (1 - 2 * t) * Er / r
    np.testing.assert_allclose(st["py"], Ey + bias, rtol=2e-2)
    if fy < 0.5:  # the bias is resolved: well beyond the tolerance
        assert np.all(bias > 0.1 * np.abs(st["py"]))


def test_symmetric_beam_gets_antisymmetric_kicks():
    g = oracle.Geometry(65, 65, -0.02, 0.02, -0.02, 0.02)
    parts = synth.gaussian_bunch(100000, 3, 3e-3, 3e-3, 1e-4, 1e-4)
    xs = np.concatenate([parts["x"], -parts["x"]])
    ys = np.concatenate([parts["y"], parts["y"]])
    Q, _ = oracle.deposit(g, xs, ys)
    Q = Q + Q[:, ::-1]  # exactly mirror-symmetric in x
    phi = oracle.potential_pipe(g, oracle.normalise(Q, 2 * len(xs)))[1:-1, 1:-1]
    probe = np.array([0.001, 0.004, 0.009])
    a = {k: np.zeros(3) for k in ("x", "px", "y", "py", "sigma", "psigma")}
    b = {k: np.zeros(3) for k in ("x", "px", "y", "py", "sigma", "psigma")}
    a["x"], b["x"] = probe.copy(), -probe
    a["y"][:] = b["y"][:] = 0.0013
    oracle.kick_bezier(g, None, a, phi[None], 1.0)
    oracle.kick_bezier(g, None, b, phi[None], 1.0)
    np.testing.assert_allclose(a["px"], -b["px"], rtol=1e-10)
    np.testing.assert_allclose(a["py"], b["py"], rtol=1e-10)
    assert np.all(a["px"] > 0)
