"""Physics pins of the oracle's kick normalisation (Sec. IV kick equation and
Eq. pot2) and of the whole PIC loop: the paper's printed tune spread (Sec. V,
Eq. tuneshift), and the small-amplitude space-charge tune shift measured by
tracking a matched Gaussian beam through the FODO ring against the
Laslett/Gaussian sum  dQ = -(1/4pi) sum_k beta_k K L_k / (sig_x (sig_x + sig_y))."""
import os

import numpy as np
import pytest

import oracle
from paper_2010_11540_gb300 import synth

HERE = os.path.dirname(os.path.abspath(__file__))


def golden(name):
    out = {}
    for line in open(os.path.join(HERE, "golden", name)):
        line = line.strip()
        if line and not line.startswith("#"):
            k, v = line.split()
            out[k] = float(v)
    return out


def test_paper_tune_spread_formula():
    g = golden("tune_spread_jparc.txt")
    gamma0, beta0 = synth.kinematics(g["kinetic_ev"])
    dnu = -g["n_ppb"] * g["harmonic"] * g["r_p_paper"] / (
        4 * np.pi * beta0**2 * gamma0**3 * g["eps_1sigma"] * g["bunch_factor"])
    assert round(dnu, 2) == g["delta_nu_printed"]
    # The same number from the oracle's kick strength K: for a round beam with
    # sigma^2 = beta eps, dQ = -K C / (8 pi eps) with N_lambda = N h / (C B_f).
    C = 1567.5
    b = dict(gamma0=gamma0, beta0=beta0, r_p=g["r_p_paper"],
             n_lambda=g["n_ppb"] * g["harmonic"] / (C * g["bunch_factor"]))
    dq = -oracle.kick_strength(b) * C / (8 * np.pi * g["eps_1sigma"])
    assert dq == pytest.approx(dnu, rel=1e-12)


@pytest.mark.slow
def test_tracked_small_amplitude_tune_shift():
    lat = synth.fodo_c1()
    C = float(lat["length"].sum())
    b = synth.beam(circumference=C, n_lambda=1.7e10)
    M = oracle.one_turn_matrix(lat, b)
    mux, bx, ax = oracle.twiss_from_matrix(M[:2, :2])
    muy, by, ay = oracle.twiss_from_matrix(M[2:, 2:])
    eps = 4e-7
    n = 50000
    rng = np.random.default_rng(21)
    u = rng.standard_normal((4, n))
    st = {"x": np.sqrt(eps * bx) * u[0], "px": np.sqrt(eps / bx) * (u[1] - ax * u[0]),
          "y": np.sqrt(eps * by) * u[2], "py": np.sqrt(eps / by) * (u[3] - ay * u[2]),
          "sigma": np.zeros(n), "psigma": np.zeros(n)}
    # probes on a 0.2-sigma invariant circle: small enough for the linear
    # (centre-gradient) shift to within ~1%, large enough to sit above the PIC
    # field noise of 5e4 macroparticles
    npb = 64
    ph = np.arange(npb) * 2 * np.pi / npb
    a = 0.2
    st["x"][:npb] = a * np.sqrt(eps * bx) * np.cos(ph)
    st["px"][:npb] = -a * np.sqrt(eps / bx) * (np.sin(ph) + ax * np.cos(ph))
    st["y"][:npb] = a * np.sqrt(eps * by) * np.cos(ph + 1)
    st["py"][:npb] = -a * np.sqrt(eps / by) * (np.sin(ph + 1) + ay * np.cos(ph + 1))
    # fine grid (h ~ 0.1 sigma) so that the CIC smoothing of deposit + gather,
    # which widens the beam by ~h^2/3 in variance, stays below 1%
    sig = 6 * np.sqrt(eps * max(bx, by))
    g = oracle.Geometry(128, 128, -sig, sig, -sig, sig)

    # expected shift: lumped kicks at the markers, Twiss propagated from s = 0
    head, kicks = oracle.segments(lat)
    K = oracle.kick_strength(b)
    seg_elems = [head] + [e for _, e in kicks]
    Mcum = np.eye(4)
    want = np.zeros(2)
    Mcum = oracle.one_turn_matrix(head, b) if len(head) else np.eye(4)
    for k, (L, seg) in enumerate(kicks):
        bxk = _beta_at(Mcum[:2, :2], bx, ax)
        byk = _beta_at(Mcum[2:, 2:], by, ay)
        sx, sy = np.sqrt(eps * bxk), np.sqrt(eps * byk)
        want[0] -= bxk * K * L / (sx * (sx + sy)) / (4 * np.pi)
        want[1] -= byk * K * L / (sy * (sx + sy)) / (4 * np.pi)
        if len(seg):
            Mcum = oracle.one_turn_matrix(seg, b) @ Mcum

    pa = oracle.PhaseAdvance(bx, ax, by, ay)

    def diag(t, s):
        pa(t, {k: v[:npb] for k, v in s.items()})

    oracle.track(g, st, b, lat, 20, diag=diag)
    pa(20, {k: v[:npb] for k, v in st.items()})
    qx, qy = pa.tunes()
    dqx = np.mean(qx) - mux / (2 * np.pi)
    dqy = np.mean(qy) - muy / (2 * np.pi)
    assert want[0] < -0.01
    assert dqx == pytest.approx(want[0], rel=0.05)
    assert dqy == pytest.approx(want[1], rel=0.05)


def _beta_at(M2, b0, a0):
    g0 = (1 + a0 * a0) / b0
    return M2[0, 0] ** 2 * b0 - 2 * M2[0, 0] * M2[0, 1] * a0 + M2[0, 1] ** 2 * g0
