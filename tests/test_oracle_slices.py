"""Pins of the oracle's longitudinal slicing (the line density lambda(z) of
Sec. IV as a histogram of sigma, each bin with its own transverse grid):
the slices' charges add up bit for bit to the unsliced deposit, the slices'
fields add up to the unsliced field (linearity of the solve), particles
outside the slice range are counted out, and bin edges follow floor()."""
import numpy as np

import oracle
from paper_2010_11540_gb300 import synth


def bunch(n=20000, seed=5):
    return synth.gaussian_bunch(n, seed, 3e-3, 2e-3, 1e-4, 1e-4, sig_z=10.0)


def geom():
    return oracle.Geometry(32, 32, -0.015, 0.015, -0.01, 0.01)


def test_slices_sum_to_unsliced_charge():
    p = bunch()
    g = geom()
    zs = oracle.Slices(8, -41.0, 41.0)  # covers the 4-sigma truncated bunch
    Qs, out_s = oracle.deposit_sliced(g, zs, p["x"], p["y"], p["sigma"])
    Q, out = oracle.deposit(g, p["x"], p["y"])
    assert np.array_equal(Qs.sum(axis=0), Q) and out_s == out
    assert (Qs.reshape(8, -1).sum(axis=1) > 0).all()


def test_outside_slices_counted():
    p = bunch()
    g = geom()
    zs = oracle.Slices(4, -5.0, 5.0)
    Qs, out_s = oracle.deposit_sliced(g, zs, p["x"], p["y"], p["sigma"])
    _, out_t = oracle.deposit(g, p["x"], p["y"])
    inside_z = ((p["sigma"] >= -5.0) & (p["sigma"] < 5.0))
    assert out_s >= len(p["x"]) - inside_z.sum()
    assert int(Qs.sum()) == (len(p["x"]) - out_s) * (1 << 40)


def test_bin_edges():
    g = oracle.Geometry(8, 8, 0.0, 7.0, 0.0, 7.0)
    zs = oracle.Slices(4, 0.0, 4.0)
    x = np.full(5, 3.5)
    y = np.full(5, 3.5)
    sg = np.array([0.0, 1.0, 2.999999, 4.0, -1e-12])
    Qs, out = oracle.deposit_sliced(g, zs, x, y, sg)
    per = Qs.reshape(4, -1).sum(axis=1) >> 40
    assert list(per) == [1, 1, 1, 0] and out == 2


def test_slice_fields_add_up_to_the_unsliced_field():
    p = bunch()
    g = geom()
    zs = oracle.Slices(6, -41.0, 41.0)
    Qs, _ = oracle.deposit_sliced(g, zs, p["x"], p["y"], p["sigma"])
    Exs, Eys = oracle.solve_sliced(g, Qs, len(p["x"]))
    Q, _ = oracle.deposit(g, p["x"], p["y"])
    Ex, Ey = oracle.solve(g, Q, len(p["x"]))
    assert np.max(np.abs(Exs.sum(axis=0) - Ex)) < 1e-12 * np.max(np.abs(Ex))
    assert np.max(np.abs(Eys.sum(axis=0) - Ey)) < 1e-12 * np.max(np.abs(Ey))


def test_one_slice_bunch_kick_equals_unsliced():
    """All particles in one slice of width dz, n_lambda = N/dz there: the sliced
    kick is the unsliced kick with line density N/dz."""
    p = synth.gaussian_bunch(5000, 6, 3e-3, 2e-3, 1e-4, 1e-4, z_half=0.4)
    g = geom()
    zs = oracle.Slices(3, -1.5, 1.5)  # bunch inside the middle slice [-0.5, 0.5)
    Qs, _ = oracle.deposit_sliced(g, zs, p["x"], p["y"], p["sigma"])
    Exs, Eys = oracle.solve_sliced(g, Qs, len(p["x"]))
    a, c = oracle.copy_state(p), oracle.copy_state(p)
    oracle.kick_sliced(g, zs, a, Exs, Eys, 1e-6)
    Q, _ = oracle.deposit(g, p["x"], p["y"])
    Ex, Ey = oracle.solve(g, Q, len(p["x"]))
    oracle.kick(g, c, Ex, Ey, 1e-6)
    assert np.allclose(a["px"], c["px"], rtol=0, atol=1e-18) and np.allclose(a["py"], c["py"], rtol=0, atol=1e-18)
