"""The allocation-free moments entry point (sc_moments_noalloc), for callers
that cannot allocate device memory while they run: called through the C-ABI
twice in a row, it must give the same moments as sc_track_turns' per-turn
diagnostics (the existing entry point) on the same state.  Collected last on
purpose, and independent of the other tests' state."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2010_11540_gb300 import build, sc, synth
from gpu_helpers import to_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    sc.load()


def test_noalloc_moments_match_track_diagnostics_twice():
    import torch

    parts, b, grid, lat = synth.workload("c1", n=20000)
    # existing entry point: moments at the start of the first turn
    g = sc.create_grid(*grid)
    ref = sc.track_turns(g, to_gpu(parts), b, lat, 1, diag=True)[0]
    st = to_gpu(parts)
    for _ in range(2):  # two calls in a row share the static scratch
        out = torch.full((14,), np.nan, dtype=torch.float64, device="cuda")
        sc.moments_noalloc(st, out)
        got = out.cpu().numpy()
        assert np.all(np.abs(got - ref) <= 1e-12 * np.abs(ref) + 1e-300), (got, ref)
    # and both agree with the oracle's moments
    assert np.max(np.abs(got - oracle.moments(parts)) / np.abs(oracle.moments(parts))) < 1e-9


def test_noalloc_moments_allocate_nothing():
    """After the first call (which looks up the scratch array), further calls
    leave the device's free memory unchanged: no allocation on any path."""
    import torch

    parts, _, _, _ = synth.workload("c1", n=20000)
    st = to_gpu(parts)
    out = torch.zeros(14, dtype=torch.float64, device="cuda")
    sc.moments_noalloc(st, out)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(8):
        sc.moments_noalloc(st, out)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


def test_noalloc_moments_rejects_bad_sizes():
    import torch

    t = torch.zeros(1, dtype=torch.float64, device="cuda")
    out = torch.zeros(14, dtype=torch.float64, device="cuda")
    L = sc.load()
    too_many = sc.Particles(*(t.data_ptr(),) * 6, 1 << 24)
    assert L.sc_moments_noalloc(ctypes.byref(too_many), out.data_ptr(), None) == -4
    empty = sc.Particles(*(t.data_ptr(),) * 6, 0)
    assert L.sc_moments_noalloc(ctypes.byref(empty), out.data_ptr(), None) == -1
    one = sc.Particles(*(t.data_ptr(),) * 6, 1)
    assert L.sc_moments_noalloc(ctypes.byref(one), None, None) == -1
