"""Pins of the oracle's open-boundary field solve (Hockney convolution with
G = -ln r, centred-difference E) against the direct pairwise sum, numerical
quadrature of the self term, and textbook closed forms: the linear interior
field of a uniform round beam (KV), the field of a round Gaussian beam, the
centre gradient of an elliptical Gaussian, the 1/r far field and the mirror
symmetry of E."""
import numpy as np
import pytest
from scipy import integrate

import oracle
from paper_2010_11540_gb300 import synth


@pytest.mark.parametrize("hx,hy", [(1.0, 1.0), (0.3, 0.7), (2e-4, 1e-4)])
def test_green_self_is_cell_average(hx, hy):
    f = lambda y, x: -0.5 * np.log(x * x + y * y)
    v, _ = integrate.dblquad(f, 0, hx / 2, 0, hy / 2, epsabs=1e-13, epsrel=1e-12)
    assert oracle.green_self(hx, hy) == pytest.approx(v / (hx * hy / 4), rel=1e-9, abs=1e-12)


@pytest.mark.parametrize("nx,ny", [(8, 8), (12, 7), (16, 16)])
def test_fft_equals_direct_sum(nx, ny):
    g = oracle.Geometry(nx, ny, -1.0, 1.3, -0.4, 0.9)
    q = np.random.default_rng(nx * ny).random((ny, nx))
    q[0, :] = 0.0  # leave some zero rows/columns
    a = oracle.potential_fft(g, q)
    b = oracle.potential_direct(g, q)
    assert a.shape == (ny + 2, nx + 2)
    assert np.max(np.abs(a - b)) < 1e-12 * np.max(np.abs(b))


def _radial(g, Ex, Ey, x0=0.0, y0=0.0):
    X, Y = np.meshgrid(g.node_x - x0, g.node_y - y0)
    r = np.hypot(X, Y)
    with np.errstate(invalid="ignore", divide="ignore"):
        Er = (Ex * X + Ey * Y) / r
    return r, Er


@pytest.mark.parametrize("n", [64, 128])
def test_kv_round_beam_linear_interior_field(n):
    """Uniform disc of radius a (unit total line charge): E_r = r / a^2 inside,
    1/r outside (normalised lambda/(2 pi eps0) = 1)."""
    a = 1.0
    g = oracle.Geometry(n, n, -2.0, 2.0, -2.0, 2.0)
    x, y = synth.uniform_disk(400000, 5, a)
    Q, n_out = oracle.deposit(g, x, y)
    assert n_out == 0
    Ex, Ey = oracle.solve(g, Q, len(x))
    r, Er = _radial(g, Ex, Ey)
    inner = (r > 0.2) & (r < 0.8)
    outer = (r > 1.2) & (r < 1.9)
    err_in = np.sqrt(np.mean((Er[inner] - r[inner] / a**2) ** 2)) / (0.8 / a**2)
    err_out = np.sqrt(np.mean((Er[outer] - 1.0 / r[outer]) ** 2)) / (1 / 1.2)
    assert err_in < 0.02 and err_out < 0.01


def test_round_gaussian_field():
    """E_r = (1 - exp(-r^2 / 2 s^2)) / r for a round Gaussian beam."""
    s = 1.0
    g = oracle.Geometry(128, 128, -5.0, 5.0, -5.0, 5.0)
    parts = synth.gaussian_bunch(1000000, 9, s, s, 1.0, 1.0, trunc=5.0)
    Q, n_out = oracle.deposit(g, parts["x"], parts["y"])
    Ex, Ey = oracle.solve(g, Q, len(parts["x"]))
    r, Er = _radial(g, Ex, Ey)
    ring = (r > 0.5) & (r < 3.5)
    want = (1 - np.exp(-r[ring] ** 2 / (2 * s * s))) / r[ring]
    err = np.sqrt(np.mean((Er[ring] - want) ** 2)) / np.max(want)
    assert err < 0.01


def test_elliptical_gaussian_centre_gradient():
    """Near the centre of an elliptical Gaussian, Ex = x / (sx (sx + sy)),
    Ey = y / (sy (sx + sy))."""
    sx, sy = 1.0, 0.6
    g = oracle.Geometry(128, 128, -5 * sx, 5 * sx, -5 * sy, 5 * sy)
    parts = synth.gaussian_bunch(2000000, 4, sx, sy, 1.0, 1.0, trunc=5.0)
    Q, _ = oracle.deposit(g, parts["x"], parts["y"])
    Ex, Ey = oracle.solve(g, Q, len(parts["x"]))
    X, Y = np.meshgrid(g.node_x, g.node_y)
    m = (np.abs(X) < 0.25 * sx) & (np.abs(Y) < 0.25 * sy)
    kx = np.sum(Ex[m] * X[m]) / np.sum(X[m] ** 2)
    ky = np.sum(Ey[m] * Y[m]) / np.sum(Y[m] ** 2)
    assert kx == pytest.approx(1 / (sx * (sx + sy)), rel=0.03)
    assert ky == pytest.approx(1 / (sy * (sx + sy)), rel=0.03)


def test_point_charge_far_field():
    """A unit charge on one node: E -> (r - r0)/|r - r0|^2 away from it, with
    the centred difference's O(h^2 / r^2) error."""
    g = oracle.Geometry(32, 32, 0.0, 31.0, 0.0, 31.0)
    Q = np.zeros((32, 32), dtype=np.int64)
    Q[10, 12] = 1 << 40
    Ex, Ey = oracle.solve(g, Q, 1)
    X, Y = np.meshgrid(g.node_x - 12.0, g.node_y - 10.0)
    r2 = X * X + Y * Y
    far = r2 > 64
    with np.errstate(divide="ignore", invalid="ignore"):
        ex, ey = X / r2, Y / r2
    rel = np.hypot(Ex - ex, Ey - ey)[far] / np.sqrt(1 / r2[far])
    assert np.max(rel) < 0.01


def test_mirror_symmetry():
    """q symmetric under x -> -x gives Ex odd and Ey even."""
    g = oracle.Geometry(24, 20, -1.0, 1.0, -0.7, 0.9)
    rng = np.random.default_rng(2)
    q = rng.random((20, 24))
    q = q + q[:, ::-1]
    phi = oracle.potential_fft(g, q)
    Ex, Ey = oracle.fields(g, phi)
    assert np.max(np.abs(Ex + Ex[:, ::-1])) < 1e-12 * np.max(np.abs(Ex))
    assert np.max(np.abs(Ey - Ey[:, ::-1])) < 1e-12 * np.max(np.abs(Ey))


def test_solve_linear_in_charge():
    g = oracle.Geometry(16, 16, -1.0, 1.0, -1.0, 1.0)
    rng = np.random.default_rng(8)
    Q1 = rng.integers(0, 1 << 40, (16, 16))
    Q2 = rng.integers(0, 1 << 40, (16, 16))
    a = oracle.solve(g, Q1, 7)[0] + oracle.solve(g, Q2, 7)[0]
    b = oracle.solve(g, Q1 + Q2, 7)[0]
    assert np.max(np.abs(a - b)) < 1e-12 * np.max(np.abs(b))
