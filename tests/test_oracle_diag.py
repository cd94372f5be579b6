"""Pin of the oracle's beam moments (Sec. V: rms sizes and emittances from
the second moments of the distribution) against numpy's own mean and
covariance routines, in the documented layout -- the means of (x, px, y, py,
sigma, psigma), then the central <xx>, <x px>, <px px>, <yy>, <y py>,
<py py>, <sigma sigma>, <psigma psigma> -- including a bunch far off the axis
(1e4 rms sizes), where a one-pass E[x^2] - E[x]^2 would lose every digit."""
import numpy as np
import pytest

import oracle

KEYS = ("x", "px", "y", "py", "sigma", "psigma")
PAIRS = [("x", "x"), ("x", "px"), ("px", "px"), ("y", "y"), ("y", "py"), ("py", "py"), ("sigma", "sigma"),
         ("psigma", "psigma")]


def bunch(n, offset, seed):
    rng = np.random.default_rng(seed)
    cov = np.array([[4e-6, 3e-8], [3e-8, 4e-8]])  # correlated x-px (and y-py)
    xs = rng.multivariate_normal([0, 0], cov, n)
    ys = rng.multivariate_normal([0, 0], 0.5 * cov, n)
    st = {"x": xs[:, 0] + offset * 2e-3, "px": xs[:, 1] + offset * 2e-4, "y": ys[:, 0] - offset * 1.4e-3,
          "py": ys[:, 1], "sigma": rng.uniform(-10, 10, n) + offset * 5.8, "psigma": rng.normal(0, 1e-3, n)}
    return {k: np.ascontiguousarray(v) for k, v in st.items()}


@pytest.mark.parametrize("offset", [0.0, 1e4])
def test_moments_equal_numpy_mean_and_covariance(offset):
    st = bunch(20011, offset, 3)
    m = oracle.moments(st)
    for c, k in enumerate(KEYS):  # sums in another order: agreement to rounding of the terms' size
        assert m[c] == pytest.approx(np.mean(st[k]), abs=1e-13 * np.sqrt(np.mean(st[k] ** 2)))
    for c, (a, b) in enumerate(PAIRS):
        want = np.cov(st[a], st[b], bias=True)[0, 1]
        assert m[6 + c] == pytest.approx(want, rel=1e-9), (a, b)


def test_emittance_of_a_known_covariance():
    """eps = sqrt(det) of the (x, px) covariance: for a large Gaussian sample
    with a chosen covariance the sample determinant, from numpy, is matched."""
    st = bunch(200003, 0.0, 4)
    ex, ey = oracle.emittances(st)
    cx = np.cov(st["x"], st["px"], bias=True)
    cy = np.cov(st["y"], st["py"], bias=True)
    assert ex == pytest.approx(np.sqrt(np.linalg.det(cx)), rel=1e-10)
    assert ey == pytest.approx(np.sqrt(np.linalg.det(cy)), rel=1e-10)
    # and the population value it estimates (sqrt(4e-6 * 4e-8 - 9e-16) = 3.87e-7)
    assert ex == pytest.approx(np.sqrt(4e-6 * 4e-8 - 9e-16), rel=1e-2)
