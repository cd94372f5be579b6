"""Pins of the oracle's longitudinal space-charge kick (Sec. IV,
dps = -(e/(m gamma0^2 beta0^2 c^2)) u dlambda/dz L), taken per slice as the
centred z-difference of the slices' pipe potentials: for a bunch whose
transverse shape is the same in every slice it equals the paper's form
(one transverse potential u times the derivative of the line-density
histogram); the total longitudinal momentum it gives is zero (the self-field
does no net work on the bunch: the pipe's Green matrix is symmetric); the head
gains energy and the tail loses it; a flat line density gives no kick away
from the ends."""
import numpy as np

import oracle
from paper_2010_11540_gb300 import synth

GRID = (65, 65) + synth.grid_extent(4e-3, 3e-3)


def setup(nz=16, n=200000, seed=5):
    parts = synth.gaussian_bunch(n, seed, 4e-3, 3e-3, 2e-4, 2e-4, sig_z=15.0)
    zs = oracle.Slices(nz, -60.0, 60.0)
    b = synth.beam(n_lambda=1e13 / zs.dz, circumference=1728.0)
    return parts, zs, b


def long_kick(g, zs, st, b, L=8.0):
    n = len(st["x"])
    Q, _ = oracle.deposit_sliced(g, zs, st["x"], st["y"], st["sigma"])
    phi = oracle.potential_sliced_pipe(g, Q, n)
    klz = oracle.kick_strength(b) * b["gamma0"] * L / (2 * zs.dz)
    out = oracle.copy_state(st)
    oracle.kick_long(g, zs, out, phi, klz)
    return out["psigma"] - st["psigma"]


def test_total_longitudinal_momentum_is_zero():
    parts, zs, b = setup()
    g = oracle.Geometry(*GRID)
    d = long_kick(g, zs, parts, b)
    assert np.abs(d).sum() > 0
    assert abs(d.sum()) < 1e-4 * np.abs(d).sum()


def test_head_gains_and_tail_loses_energy():
    parts, zs, b = setup()
    g = oracle.Geometry(*GRID)
    d = long_kick(g, zs, parts, b)
    s = parts["sigma"]
    assert d[s > 15.0].mean() > 0 and d[s < -15.0].mean() < 0
    # antisymmetric in z to the statistics of the sample
    assert abs(d[s > 15.0].mean() + d[s < -15.0].mean()) < 0.1 * d[s > 15.0].mean()


def replicated(weights, base, zs):
    """The same transverse set `base` placed w_k times at the centre of slice k."""
    out = {k: [] for k in base}
    for k, w in enumerate(weights):
        for _ in range(w):
            for key in base:
                v = base[key].copy()
                if key == "sigma":
                    v[:] = zs.zmin + (k + 0.5) * zs.dz
                out[key].append(v)
    return {k: np.concatenate(v) for k, v in out.items()}


def test_flat_line_density_gives_no_kick_away_from_the_ends():
    base = synth.gaussian_bunch(3000, 9, 4e-3, 3e-3, 2e-4, 2e-4)
    zs = oracle.Slices(8, -60.0, 60.0)
    b = synth.beam(n_lambda=1e13 / zs.dz, circumference=1728.0)
    st = replicated([1] * 8, base, zs)
    g = oracle.Geometry(*GRID)
    d = long_kick(g, zs, st, b)
    k = np.floor((st["sigma"] - zs.zmin) / zs.dz).astype(int)
    interior = (k > 0) & (k < 7)
    assert np.all(d[interior] == 0.0)
    assert np.all(d[k == 7] > 0) and np.all(d[k == 0] < 0)  # the ends are pushed apart


def test_separable_bunch_equals_the_papers_form():
    """w_k copies of one transverse set in slice k: the per-slice form equals
    -(2 r_p / (beta0^2 gamma0^2)) u(x, y) lambda'(z) L with u the pipe potential
    of the normalised transverse distribution (one solve) and lambda'(z) the
    centred difference of the line-density histogram lambda_k = N_ppb n_k / (N dz),
    n_k = w_k n_base macroparticles in slice k."""
    base = synth.gaussian_bunch(2000, 21, 4e-3, 3e-3, 2e-4, 2e-4)
    zs = oracle.Slices(7, -60.0, 60.0)
    w = [1, 2, 4, 6, 3, 2, 1]
    n_ppb = 1e13
    b = synth.beam(n_lambda=n_ppb / zs.dz, circumference=1728.0)
    st = replicated(w, base, zs)
    N = len(st["x"])
    g = oracle.Geometry(*GRID)
    L = 8.0
    d = long_kick(g, zs, st, b, L)
    # the paper's form: one transverse solve of the projected distribution, the histogram's derivative
    Qb, _ = oracle.deposit(g, base["x"], base["y"])
    u = oracle.potential_pipe(g, oracle.normalise(Qb, len(base["x"])))[1:-1, 1:-1]
    lam = n_ppb * np.array(w, dtype=float) * len(base["x"]) / (N * zs.dz)
    lam_ext = np.r_[0.0, lam, 0.0]
    dlam = (lam_ext[2:] - lam_ext[:-2]) / (2 * zs.dz)
    coef = 2 * b["r_p"] / (b["beta0"] ** 2 * b["gamma0"] ** 2)
    k = np.floor((st["sigma"] - zs.zmin) / zs.dz).astype(int)
    xi = (st["x"] - g.xmin) * g.inv_hx
    eta = (st["y"] - g.ymin) * g.inv_hy
    i, j = np.floor(xi).astype(int), np.floor(eta).astype(int)
    fx, fy = xi - i, eta - j
    ok = (i >= 0) & (i < g.nx - 1) & (j >= 0) & (j < g.ny - 1)
    ii, jj = np.clip(i, 0, g.nx - 2), np.clip(j, 0, g.ny - 2)
    up = ((1 - fx) * (1 - fy) * u[jj, ii] + fx * (1 - fy) * u[jj, ii + 1] + (1 - fx) * fy * u[jj + 1, ii]
          + fx * fy * u[jj + 1, ii + 1])
    want = np.where(ok, -coef * up * dlam[k] * L, 0.0)
    scale = np.abs(want).max()
    assert scale > 0
    np.testing.assert_allclose(d, want, rtol=0, atol=1e-9 * scale)  # FFT rounding of each slice solve
