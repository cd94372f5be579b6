"""Pins of the oracle's single-particle maps (Sec. III) against the
Hamiltonians they come from: each map must equal a fine RK4 integration of
Hamilton's equations of its Hamiltonian (Eq. H: exact form for the drift,
H_approx for the quadrupole and the linear dipole), with the vector field
taken by complex-step differentiation of H itself, and each map must be
symplectic (M^T J M = J for its 6-D Jacobian)."""
import numpy as np
import pytest

import oracle
from paper_2010_11540_gb300 import synth

B = synth.beam(circumference=100.0)
G0, B0 = B["gamma0"], B["beta0"]


def h_drift(z):
    x, px, y, py, sg, ps = z
    return ps - np.sqrt(1 + 2 * ps + B0**2 * ps**2 - px**2 - py**2)


def h_quad(k1):
    def H(z):
        x, px, y, py, sg, ps = z
        return (px**2 + py**2) / 2 + ps**2 / (2 * G0**2) - (px**2 + py**2) / 2 * ps + k1 / 2 * (x**2 - y**2)
    return H


def h_bend(h):
    def H(z):
        x, px, y, py, sg, ps = z
        return (px**2 + py**2) / 2 + ps**2 / (2 * G0**2) - h * x * ps + h * h * x * x / 2
    return H


def vector_field(H, z):
    """dz/ds = J grad H, gradient by complex step."""
    grad = np.zeros(6)
    for k in range(6):
        zc = z.astype(complex)
        zc[k] += 1e-30j
        grad[k] = H(zc).imag / 1e-30
    # (x,px),(y,py),(sg,ps) conjugate pairs: dq/ds = dH/dp, dp/ds = -dH/dq
    return np.array([grad[1], -grad[0], grad[3], -grad[2], grad[5], -grad[4]])


def rk4(H, z, L, n=2000):
    h = L / n
    for _ in range(n):
        k1 = vector_field(H, z)
        k2 = vector_field(H, z + 0.5 * h * k1)
        k3 = vector_field(H, z + 0.5 * h * k2)
        k4 = vector_field(H, z + h * k3)
        z = z + h / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
    return z


def apply(elems, z):
    st = {k: np.array([v]) for k, v in zip(("x", "px", "y", "py", "sigma", "psigma"), z)}
    oracle.push(st, synth.table(elems), B)
    return np.array([st[k][0] for k in ("x", "px", "y", "py", "sigma", "psigma")])


Z0 = np.array([2e-3, -3e-4, -1.5e-3, 2e-4, 0.3, 2.5e-3])


@pytest.mark.parametrize("case", ["drift", "qf", "qd", "bend"])
def test_map_equals_hamiltonian_flow(case):
    L = 1.3
    if case == "drift":
        e, H = synth.elem(synth.DRIFT, L), h_drift
    elif case == "qf":
        e, H = synth.elem(synth.QUAD, L, k1=0.8), h_quad(0.8)
    elif case == "qd":
        e, H = synth.elem(synth.QUAD, L, k1=-0.6), h_quad(-0.6)
    else:
        e, H = synth.elem(synth.BEND, L, angle=0.2), h_bend(0.2 / L)
    got = apply([e], Z0)
    want = rk4(H, Z0.copy(), L)
    scale = np.array([1e-3, 1e-4, 1e-3, 1e-4, 1e-3, 1e-3])
    assert np.max(np.abs(got - want) / scale) < 1e-9


def jacobian(elems, z, eps=1e-6):
    M = np.zeros((6, 6))
    for c in range(6):
        dz = np.zeros(6)
        dz[c] = eps
        M[:, c] = (apply(elems, z + dz) - apply(elems, z - dz)) / (2 * eps)
    return M


J = np.zeros((6, 6))
for _k in range(3):
    J[2 * _k, 2 * _k + 1] = 1.0
    J[2 * _k + 1, 2 * _k] = -1.0


@pytest.mark.parametrize("e", [
    synth.elem(synth.DRIFT, 2.0),
    synth.elem(synth.QUAD, 0.7, k1=1.1),
    synth.elem(synth.QUAD, 0.7, k1=-0.9),
    synth.elem(synth.QUAD, 0.7, k1=0.0),
    synth.elem(synth.SEXT, k2l=3.0),
    synth.elem(synth.BEND, 1.5, angle=0.1),
    synth.elem(synth.RF, volt=2e5, harmonic=9.0, lag=0.3),
])
def test_symplectic(e):
    M = jacobian([e], Z0)
    assert np.max(np.abs(M.T @ J @ M - J)) < 1e-7
    assert abs(np.linalg.det(M) - 1.0) < 1e-7


def test_quad_tends_to_h0_drift():
    a = apply([synth.elem(synth.QUAD, 1.0, k1=1e-13)], Z0)
    b = apply([synth.elem(synth.QUAD, 1.0, k1=0.0)], Z0)
    assert np.max(np.abs(a - b)) < 1e-12


def test_sextupole_kick_values():
    """Thin kick of V = k2 (x^3 - 3 x y^2)/6: dpx = -k2l/2 (x^2-y^2), dpy = k2l x y."""
    z = apply([synth.elem(synth.SEXT, k2l=2.0)], Z0)
    x, y = Z0[0], Z0[2]
    assert z[1] - Z0[1] == pytest.approx(-(x * x - y * y), rel=1e-12)
    assert z[3] - Z0[3] == pytest.approx(2.0 * x * y, rel=1e-12)


def test_bare_tune_trace_vs_tracked_phase_advance():
    """Tune from cos mu = Tr(M)/2 equals the tracked mean phase advance of a
    small-amplitude particle (Sec. V tune definition)."""
    lat = synth.fodo_c1()
    b = synth.beam(circumference=264.0)
    M = oracle.one_turn_matrix(lat, b)
    mux, bx, ax = oracle.twiss_from_matrix(M[:2, :2])
    muy, by, ay = oracle.twiss_from_matrix(M[2:, 2:])
    st = {k: np.zeros(3) for k in ("x", "px", "y", "py", "sigma", "psigma")}
    st["x"][:] = [1e-6, 2e-6, -1e-6]
    st["y"][:] = [1e-6, -3e-6, 2e-6]
    pa = oracle.PhaseAdvance(bx, ax, by, ay)
    for t in range(60):
        pa(t, st)
        oracle.push(st, lat, b)
    qx, qy = pa.tunes()
    assert np.allclose(qx, mux / (2 * np.pi), atol=1e-9)
    assert np.allclose(qy, muy / (2 * np.pi), atol=1e-9)


def test_rms_size_gives_beta():
    """Sec. V: for a matched Gaussian, sigma(s)^2 / eps = beta(s), with beta
    propagated from the start by the transfer matrix."""
    lat = synth.fodo_c1()
    b = synth.beam(circumference=264.0)
    M = oracle.one_turn_matrix(lat, b)
    _, bx, ax = oracle.twiss_from_matrix(M[:2, :2])
    eps = 4e-7
    n = 200000
    rng = np.random.default_rng(3)
    u, v = rng.standard_normal(n), rng.standard_normal(n)
    x = np.sqrt(eps * bx) * u
    px = np.sqrt(eps / bx) * (v - ax * u)
    st = {"x": x, "px": px, "y": np.zeros(n), "py": np.zeros(n), "sigma": np.zeros(n), "psigma": np.zeros(n)}
    part = lat[:2]  # QF + drift
    oracle.push(st, part, b)
    Mp = oracle.one_turn_matrix(part, b)[:2, :2]
    g0 = (1 + ax * ax) / bx
    b1 = Mp[0, 0] ** 2 * bx - 2 * Mp[0, 0] * Mp[0, 1] * ax + Mp[0, 1] ** 2 * g0
    eps_meas = oracle.emittances(st)[0]
    assert np.var(st["x"]) / eps_meas == pytest.approx(b1, rel=0.01)  # sampling error ~ 1/sqrt(n)
    assert eps_meas == pytest.approx(eps, rel=0.01)


# ------------------------------------------------------------------ exact sector dipole, thick sextupole
def h_exact_bend(h):
    """Exact sector-dipole Hamiltonian in curvilinear coordinates: the uniform
    field's A_s with (1+hx) A_s = -B0 (x + h x^2/2):
    H = ps - (1 + h x) sqrt((1+delta)^2 - px^2 - py^2) + h x + h^2 x^2 / 2."""
    def H(z):
        x, px, y, py, sg, ps = z
        return ps - (1 + h * x) * np.sqrt(1 + 2 * ps + B0**2 * ps**2 - px**2 - py**2) + h * x + h * h * x * x / 2
    return H


def h_sext(k2):
    def H(z):
        x, px, y, py, sg, ps = z
        return ((px**2 + py**2) / 2 * (1 - ps) + ps**2 / (2 * G0**2) + k2 / 6 * (x**3 - 3 * x * y**2))
    return H


@pytest.mark.parametrize("angle,L", [(0.2, 1.3), (-0.35, 2.0), (0.05, 0.5)])
def test_exact_bend_equals_hamiltonian_flow(angle, L):
    got = apply([synth.elem(synth.EXACT_BEND, L, angle=angle)], Z0)
    want = rk4(h_exact_bend(angle / L), Z0.copy(), L)
    scale = np.array([1e-3, 1e-4, 1e-3, 1e-4, 1e-3, 1e-3])
    assert np.max(np.abs(got - want) / scale) < 1e-9


def test_exact_bend_linearises_to_the_linear_bend():
    """The Jacobian of the exact map at the reference orbit is the linear
    sector-dipole matrix (H_approx is the exact H to second order)."""
    e_exact = synth.elem(synth.EXACT_BEND, 1.5, angle=0.12)
    e_lin = synth.elem(synth.BEND, 1.5, angle=0.12)
    z = np.zeros(6)
    assert np.max(np.abs(jacobian([e_exact], z, 1e-7) - jacobian([e_lin], z, 1e-7))) < 1e-7
    # and zero angle is the exact drift
    a = apply([synth.elem(synth.EXACT_BEND, 1.5, angle=0.0)], Z0)
    b = apply([synth.elem(synth.DRIFT, 1.5)], Z0)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("e", [synth.elem(synth.EXACT_BEND, 1.5, angle=0.1),
                               synth.elem(synth.SEXT, 0.4, k2l=4.0)])
def test_symplectic_new_elements(e):
    M = jacobian([e], Z0)
    assert np.max(np.abs(M.T @ J @ M - J)) < 1e-7


def test_thick_sextupole_is_the_papers_split():
    """Eq. Sym2 with a, b, c of the paper (SABA2): zero strength is the H0
    flow; against the exact flow of H0 + V its error is second order in the
    step and quadratic in the strength (O(eps^2 tau^2 + eps tau^4): the
    linear-in-strength part of a plain second-order split cancels); a very
    short element is the thin kick."""
    L = 0.6
    zero = apply([synth.elem(synth.SEXT, L, k2l=0.0)], Z0)
    h0 = apply([synth.elem(synth.QUAD, L, k1=0.0)], Z0)
    assert np.max(np.abs(zero - h0)) < 1e-15
    z = np.array([8e-3, -6e-4, -5e-3, 4e-4, 0.3, 2.5e-3])

    def err(k2l, pieces):
        exact = rk4(h_sext(k2l / L), z.copy(), L, n=4000)
        got = apply([synth.elem(synth.SEXT, L / pieces, k2l=k2l / pieces)] * pieces, z)
        return np.abs(got - exact).max()

    e30, e30h, e3 = err(30.0, 1), err(30.0, 2), err(3.0, 1)
    assert 3.5 < e30 / e30h < 4.5, (e30, e30h)  # second order in the step
    assert e30 / e3 > 50, (e30, e3)  # quadratic in the strength
    thin = apply([synth.elem(synth.SEXT, 1e-7, k2l=30.0)], z)
    kick = apply([synth.elem(synth.SEXT, 0.0, k2l=30.0)], z)
    assert np.max(np.abs(thin - kick)) < 1e-9


def test_synchrotron_tune_of_a_small_oscillation():
    """RF cavity and drift together against small-oscillation theory: a ring of
    one drift of length C (no bends, so the slip factor is 1/gamma0^2: the
    exact drift advances sigma by C psigma / gamma0^2 to first order) and one
    thin cavity (psigma kick V/(beta0^2 E0) sin(-2 pi h sigma / C), the
    linearised restoring strength k = V/(beta0^2 E0) 2 pi h / C) has the
    one-turn matrix [[1, C/g^2], [-k, 1 - k C/g^2]], so
    cos(2 pi Q_s) = 1 - k C / (2 gamma0^2) -- for small Q_s the textbook
    Q_s^2 = h V eta / (2 pi beta0^2 E0).  The tracked small-amplitude
    particle's period (from its interpolated zero crossings of sigma) must
    give that tune: a wrong sign of the kick, a missing beta0^2 or gamma0^2,
    or a wrong 2 pi h / C fails it."""
    C, V, h = 100.0, 2e6, 20.0
    b = synth.beam(circumference=C)
    g0, b0 = b["gamma0"], b["beta0"]
    k = V / (b0 * b0 * g0 * b["mass_ev"]) * 2 * np.pi * h / C
    qs = np.arccos(1 - k * C / (2 * g0 * g0)) / (2 * np.pi)
    assert 0.005 < qs < 0.02
    ring = synth.table([synth.elem(synth.DRIFT, C), synth.elem(synth.RF, volt=V, harmonic=h, lag=0.0)])
    st = {key: np.zeros(1) for key in ("x", "px", "y", "py", "sigma", "psigma")}
    st["sigma"][0] = 1e-3
    sg = np.empty(4000)
    for t in range(sg.size):
        sg[t] = st["sigma"][0]
        oracle.push(st, ring, b)
    assert np.max(np.abs(sg)) < 1.01e-3  # a stable, small oscillation
    i = np.nonzero(np.sign(sg[:-1]) != np.sign(sg[1:]))[0]
    z = i + sg[i] / (sg[i] - sg[i + 1])  # interpolated zero crossings (turns)
    period = 2 * (z[-1] - z[0]) / (len(z) - 1)
    assert 1 / period == pytest.approx(qs, rel=1e-5)
