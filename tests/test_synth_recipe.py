"""The seeded synthetic inputs follow the stated recipe (the workloads the
bench and the parity tests run): 4-D Gaussian bunches truncated at 4 sigma
(rms of a normal truncated at 4 sigma: 0.99946 sigma), sigma uniform over
+-10 m or (c5) Gaussian with sigma_z = 15 m cut at 4 sigma_z and sorted,
psigma Gaussian with rms 1e-3, grids over +-5 sigma, the c2 ring's 216
space-charge locations over 1728 m, 3 GeV protons, 1e11 protons per 20 m;
the c4 batch's 64 bunches with log-uniform counts in [1e4, 2e6] and their
grid classes.  Same seed, same bits."""
import math

import numpy as np
import pytest

from paper_2010_11540_gb300 import synth

TRUNC4 = math.sqrt(1 - 2 * 4 * math.exp(-8) / math.sqrt(2 * math.pi) / math.erf(4 / math.sqrt(2)))


def test_truncated_normal_factor():
    stats = pytest.importorskip("scipy.stats")
    assert TRUNC4 == pytest.approx(stats.truncnorm(-4, 4).std(), rel=1e-12)


def test_c2_bunch_beam_grid_ring():
    n = 400_000
    p, b, grid, lat = synth.workload("c2", n=n)
    tol = 4 / math.sqrt(2 * n)  # 4 standard errors of an rms estimate
    for k, s in (("x", 4e-3), ("y", 3e-3), ("px", 2e-4), ("py", 2e-4)):
        assert np.std(p[k]) == pytest.approx(TRUNC4 * s, rel=tol), k
        assert np.max(np.abs(p[k])) <= 4 * s
    assert np.min(p["sigma"]) >= -10.0 and np.max(p["sigma"]) <= 10.0
    assert np.std(p["sigma"]) == pytest.approx(20 / math.sqrt(12), rel=tol)
    assert np.std(p["psigma"]) == pytest.approx(1e-3, rel=tol)
    assert grid == (128, 128, -0.02, 0.02, -0.015, 0.015)
    assert b["n_lambda"] == pytest.approx(1e11 / 20) and b["gamma0"] == pytest.approx(1 + 3e9 / 938.27208816e6)
    assert b["circumference"] == pytest.approx(1728.0)
    assert int((lat["type"] == synth.MARK).sum()) == 216


def test_c5_longitudinal_recipe():
    n = 400_000
    p, b, grid, lat = synth.workload("c5", n=n)
    assert np.all(np.diff(p["sigma"]) >= 0)  # sorted by sigma
    assert np.max(np.abs(p["sigma"])) <= 60.0
    assert np.std(p["sigma"]) == pytest.approx(15.0 * TRUNC4, rel=4 / math.sqrt(2 * n))
    assert synth.slices("c5") == (32, -60.0, 60.0)
    assert b["n_lambda"] == pytest.approx(1e13 / (120.0 / 32))


def test_c4_batch_structure():
    bunches = synth.c4_bunches(scale=1e-3)
    assert len(bunches) == 64
    for parts, b, grid, lat in bunches:
        n = len(parts["x"])
        assert 10 <= n <= 2000
        assert grid[0] == grid[1] and grid[0] in (64, 128, 256) and grid[2:] == (-0.02, 0.02, -0.015, 0.015)
        assert int((lat["type"] == synth.MARK).sum()) == 216
    # the grid class follows the unscaled count (scaled counts are 1/1000 of it)
    for parts, _, grid, _ in bunches:
        n_full = 1000 * len(parts["x"])
        if abs(n_full - 1e5) > 1000 and abs(n_full - 5e5) > 1000:
            assert grid[0] == synth.c4_grid_size(n_full)


def test_same_seed_same_bits():
    a = synth.workload("c1", n=5000)[0]
    c = synth.workload("c1", n=5000)[0]
    d = synth.workload("c1", n=5000, seed=12346)[0]
    assert all(np.array_equal(a[k], c[k]) for k in a)
    assert not np.array_equal(a["x"], d["x"])


def test_ring_and_beam_json_round_trip():
    """The rings and beams as plain text: every preset comes back bit for bit."""
    for name in ("c1", "c2", "c5"):
        _, b, _, lat = synth.workload(name, n=10)
        b2, lat2 = synth.config_from_json(synth.config_to_json(b, lat))
        assert b2 == b
        assert lat2.dtype == lat.dtype and lat2.tobytes() == lat.tobytes()
    with pytest.raises(ValueError):
        synth.config_from_json('{"beam": {}, "lattice": [{"type": "quad", "k3": 1.0}]}')
