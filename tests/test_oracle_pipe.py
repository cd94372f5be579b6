"""Pins of the oracle's conducting-pipe (Dirichlet) solve, Sec. IV-B: the
5-point stencil of the result reproduces the right-hand side on every interior
node, the walls hold phi = 0, tiny grids equal a dense direct solve of the
discrete system, the lowest sine mode is an exact eigenvector, the field is
normal to the walls, and a small beam far from the walls sees the free-space
field."""
import numpy as np
import pytest

import oracle


def lap5(phi_ext, g):
    """5-point Laplacian on the interior nodes of phi given on i = -1..nx."""
    p = phi_ext[1:-1, 1:-1]  # nodes 0..n-1
    c = p[1:-1, 1:-1]
    return ((p[1:-1, 2:] - 2 * c + p[1:-1, :-2]) / g.hx ** 2 + (p[2:, 1:-1] - 2 * c + p[:-2, 1:-1]) / g.hy ** 2)


@pytest.mark.parametrize("nx,ny", [(9, 9), (17, 33), (129, 65)])
def test_stencil_reproduces_rhs_and_walls_are_zero(nx, ny):
    rng = np.random.default_rng(nx + ny)
    g = oracle.Geometry(nx, ny, -0.01, 0.013, -0.007, 0.009)
    q = rng.random((ny, nx))
    phi = oracle.potential_pipe(g, q)
    rhs = -2 * np.pi * q[1:-1, 1:-1] / (g.hx * g.hy)
    np.testing.assert_allclose(lap5(phi, g), rhs, rtol=1e-10, atol=1e-10 * np.abs(rhs).max())
    walls = phi[1:-1, 1:-1]
    assert not walls[0].any() and not walls[-1].any() and not walls[:, 0].any() and not walls[:, -1].any()
    # odd extension beyond the walls
    np.testing.assert_array_equal(phi[:, 0], -phi[:, 2])
    np.testing.assert_array_equal(phi[0, :], -phi[2, :])


def test_tiny_grid_equals_dense_direct_solve():
    """The discrete system assembled as a dense matrix and solved directly."""
    g = oracle.Geometry(6, 7, 0.0, 1.0, 0.0, 1.3)
    mx, my = g.nx - 2, g.ny - 2
    rng = np.random.default_rng(3)
    q = rng.random((g.ny, g.nx))
    N = mx * my
    A = np.zeros((N, N))
    idx = lambda i, j: j * mx + i  # noqa: E731
    for j in range(my):
        for i in range(mx):
            r = idx(i, j)
            A[r, r] = -2 / g.hx ** 2 - 2 / g.hy ** 2
            if i > 0:
                A[r, idx(i - 1, j)] = 1 / g.hx ** 2
            if i < mx - 1:
                A[r, idx(i + 1, j)] = 1 / g.hx ** 2
            if j > 0:
                A[r, idx(i, j - 1)] = 1 / g.hy ** 2
            if j < my - 1:
                A[r, idx(i, j + 1)] = 1 / g.hy ** 2
    b = (-2 * np.pi * q[1:-1, 1:-1] / (g.hx * g.hy)).ravel()
    want = np.linalg.solve(A, b).reshape(my, mx)
    got = oracle.potential_pipe(g, q)[2:-2, 2:-2]
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-12 * np.abs(want).max())


def test_lowest_mode_is_an_exact_eigenvector():
    """q = sin(pi i/(m+1)) sin(pi j/(m+1)): phi = -2 pi q/(hx hy) / lambda_11 with
    lambda_11 = -4 (sin^2(pi/2(mx+1))/hx^2 + sin^2(pi/2(my+1))/hy^2)."""
    g = oracle.Geometry(33, 17, 0.0, 0.1, 0.0, 0.05)
    i = np.arange(g.nx)
    j = np.arange(g.ny)
    q = np.outer(np.sin(np.pi * j / (g.ny - 1)), np.sin(np.pi * i / (g.nx - 1)))
    lam = -4 * (np.sin(np.pi / (2 * (g.nx - 1))) ** 2 / g.hx ** 2 + np.sin(np.pi / (2 * (g.ny - 1))) ** 2 / g.hy ** 2)
    want = -2 * np.pi * q / (g.hx * g.hy) / lam
    got = oracle.potential_pipe(g, q)[1:-1, 1:-1]
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-13 * np.abs(want).max())


def test_field_is_normal_to_the_walls():
    rng = np.random.default_rng(11)
    g = oracle.Geometry(33, 33, -1.0, 1.0, -1.0, 1.0)
    q = np.zeros((33, 33))
    q[10:20, 12:22] = rng.random((10, 10))
    Ex, Ey = oracle.fields(g, oracle.potential_pipe(g, q))
    assert np.abs(Ex[0]).max() == 0 and np.abs(Ex[-1]).max() == 0  # horizontal walls: no tangential Ex
    assert np.abs(Ey[:, 0]).max() == 0 and np.abs(Ey[:, -1]).max() == 0
    assert np.abs(Ey[0]).max() > 0 and np.abs(Ex[:, 0]).max() > 0  # normal components do not vanish


def test_small_beam_far_from_the_walls_sees_the_free_space_field():
    """A round Gaussian beam of rms 1 in a 40 x 40 pipe: the walls' image field
    near the beam is far below its own field, so the pipe solve agrees with the
    open solve to their different discretisations (5-point Laplacian vs sampled
    -ln r, both O(h^2), h = 0.156) and with the closed form (1 - e^{-r^2/2})/r."""
    g = oracle.Geometry(257, 257, -20.0, 20.0, -20.0, 20.0)
    x, y = np.meshgrid(g.node_x, g.node_y)
    q = np.exp(-(x ** 2 + y ** 2) / 2)
    q /= q.sum()
    Q = np.round(q * oracle.Q_UNIT * 1000).astype(np.uint64)
    Exp, Eyp = oracle.solve(g, Q, 1000, boundary="pipe")
    Exo, Eyo = oracle.solve(g, Q, 1000)
    r = np.hypot(x, y)
    core = r <= 2.0
    scale = np.abs(Exo[core]).max()
    assert np.abs(Exp[core] - Exo[core]).max() < 5e-3 * scale
    # and the field of the open solve at r = 1..2 is the round Gaussian's (1 - e^{-r^2/2})/r
    ring = (r > 1.0) & (r < 2.0) & (np.abs(y) < 1e-9)
    want = (1 - np.exp(-x[ring] ** 2 / 2)) / x[ring]
    np.testing.assert_allclose(Exp[ring], want, rtol=2e-2)
