"""Thin Python binding of libsc's C-ABI (include/sc.h): argument marshalling only.

Every step of the space-charge path runs in libsc's CUDA kernels; this module
converts torch tensors / numpy arrays into the C structs and raises on error
codes.  There is no CPU fallback: if libsc.so is missing or no GPU is present
the calls fail loudly.

Names follow the C-ABI: create_grid, deposit, solve, kick_push, track_turns,
grid_read, grid_write_charge.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import synth

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libsc.so")

SC_OK = 0
ERRORS = {-1: "SC_ERR_ARG", -2: "SC_ERR_CUDA", -3: "SC_ERR_OOM", -4: "SC_ERR_OVERFLOW",
          -5: "SC_ERR_TIMEOUT", -6: "SC_ERR_NAN", -7: "SC_ERR_UNSUPPORTED"}
PRECISION = {"fp64": 0, "tf32x3": 1, "pipe_fp64": 2, "pipe_tf32x3": 3, "bf16x3": 4}
EXPORTS = ("sc_create_grid", "sc_create_grid_sliced", "sc_destroy_grid", "sc_deposit", "sc_solve", "sc_kick_push", "sc_track_turns",
           "sc_grid_read", "sc_grid_write_charge", "sc_tune_setup", "sc_trace_enable", "sc_trace_read",
           "sc_moments_noalloc", "sc_create_batch", "sc_destroy_batch", "sc_batch_track_turns", "sc_batch_read",
           "sc_batch_trace_enable", "sc_batch_trace_read", "sc_get_solver_tiling", "sc_set_solver_tiling",
           "sc_batch_set_solver_tiling", "sc_batch_get_solver_tiling", "sc_tunes", "sc_grid_read_potential",
           "sc_set_longitudinal_kick", "sc_set_gather", "sc_test_bounded_waits", "sc_set_kick_push_shape",
           "sc_get_kick_push_shape", "sc_track_turns_host", "sc_batch_track_turns_host", "sc_batch_set_kick_push_shape",
           "sc_batch_get_kick_push_shape", "sc_get_solver_work", "sc_grid_charge_device",
           "sc_set_particle_count", "sc_sort_particles", "sc_set_charge_reduce", "sc_checkpoint_write",
           "sc_checkpoint_read", "sc_last_error")


class ScError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class Particles(ctypes.Structure):
    _fields_ = [("x", ctypes.c_void_p), ("px", ctypes.c_void_p), ("y", ctypes.c_void_p),
                ("py", ctypes.c_void_p), ("sigma", ctypes.c_void_p), ("psigma", ctypes.c_void_p),
                ("n", ctypes.c_int64)]


class Beam(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in ("gamma0", "beta0", "n_lambda", "r_p", "circumference", "mass_ev")]


class GridSpec(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int)] + [
        (k, ctypes.c_double) for k in ("xmin", "xmax", "ymin", "ymax")]


class Bunch(ctypes.Structure):
    _fields_ = [("particles", Particles), ("beam", Beam), ("lattice", ctypes.c_void_p), ("n_elems", ctypes.c_int)]


# int (*)(uint64_t* charge, int64_t cells, void* stream, void* user)
REDUCE_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p)

_lib = None


def load():
    """Load libsc.so (built by paper_2010_11540_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libsc.so not built ({LIB_PATH}); run paper_2010_11540_gb300.build.build()")
    L = ctypes.CDLL(LIB_PATH)
    vp, i64, dp = ctypes.c_void_p, ctypes.c_int64, ctypes.POINTER(ctypes.c_double)
    L.sc_create_grid.argtypes = [ctypes.POINTER(vp), ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                 ctypes.c_double, ctypes.c_double, ctypes.c_int, vp]
    L.sc_create_grid_sliced.argtypes = [ctypes.POINTER(vp), ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                        ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                        ctypes.c_double, ctypes.c_double, ctypes.c_int, vp]
    L.sc_destroy_grid.argtypes = [vp]
    L.sc_deposit.argtypes = [vp, ctypes.POINTER(Particles)]
    L.sc_solve.argtypes = [vp]
    L.sc_kick_push.argtypes = [vp, ctypes.POINTER(Particles), ctypes.POINTER(Beam), ctypes.c_double, vp,
                               ctypes.c_int, vp]
    L.sc_track_turns.argtypes = [vp, ctypes.POINTER(Particles), ctypes.POINTER(Beam), vp, ctypes.c_int,
                                 ctypes.c_int, dp]
    L.sc_grid_read.argtypes = [vp, vp, vp, vp, ctypes.POINTER(i64)]
    L.sc_grid_write_charge.argtypes = [vp, vp, i64]
    L.sc_tune_setup.argtypes = [vp, ctypes.POINTER(Particles), dp, vp]
    L.sc_trace_enable.argtypes = [vp, ctypes.c_int]
    L.sc_trace_read.argtypes = [vp, dp, dp, ctypes.POINTER(i64)]
    L.sc_moments_noalloc.argtypes = [ctypes.POINTER(Particles), vp, vp]
    L.sc_create_batch.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(GridSpec), ctypes.c_int, ctypes.c_int, vp]
    L.sc_destroy_batch.argtypes = [vp]
    L.sc_batch_track_turns.argtypes = [vp, ctypes.POINTER(Bunch), ctypes.c_int, dp]
    L.sc_batch_read.argtypes = [vp, ctypes.c_int, vp, vp, vp, ctypes.POINTER(i64)]
    L.sc_batch_trace_enable.argtypes = [vp, ctypes.c_int]
    L.sc_batch_trace_read.argtypes = [vp, dp, dp, ctypes.POINTER(i64)]
    L.sc_get_solver_tiling.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.c_char_p, ctypes.c_size_t]
    L.sc_set_solver_tiling.argtypes = [vp, ctypes.POINTER(ctypes.c_int)]
    L.sc_batch_set_solver_tiling.argtypes = [vp, ctypes.POINTER(ctypes.c_int)]
    L.sc_batch_get_solver_tiling.argtypes = [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.c_char_p,
                                             ctypes.c_size_t]
    L.sc_tunes.argtypes = [vp, i64, ctypes.c_int, vp, vp]
    L.sc_sort_particles.argtypes = [vp, ctypes.POINTER(Particles), vp]
    L.sc_set_charge_reduce.argtypes = [vp, REDUCE_FN, vp, i64]
    L.sc_grid_read_potential.argtypes = [vp, vp]
    L.sc_set_longitudinal_kick.argtypes = [vp, ctypes.c_int]
    L.sc_set_gather.argtypes = [vp, ctypes.c_int]
    L.sc_test_bounded_waits.argtypes = [vp, ctypes.c_int]
    L.sc_set_kick_push_shape.argtypes = [vp, ctypes.c_int, ctypes.c_int]
    L.sc_get_solver_work.argtypes = [vp, dp, dp]
    L.sc_grid_charge_device.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(i64)]
    L.sc_set_particle_count.argtypes = [vp, i64]
    L.sc_track_turns_host.argtypes = [vp, ctypes.POINTER(Particles), ctypes.POINTER(Beam), vp, ctypes.c_int,
                                      ctypes.c_int, dp]
    L.sc_batch_track_turns_host.argtypes = [vp, ctypes.POINTER(Bunch), ctypes.c_int, dp]
    L.sc_batch_set_kick_push_shape.argtypes = [vp, ctypes.c_int, ctypes.c_int]
    L.sc_batch_get_kick_push_shape.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int), dp]
    L.sc_get_kick_push_shape.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int), dp]
    L.sc_checkpoint_write.argtypes = [ctypes.c_char_p, ctypes.POINTER(Particles), i64, ctypes.POINTER(Beam), vp,
                                      ctypes.c_int]
    L.sc_checkpoint_read.argtypes = [ctypes.c_char_p, ctypes.POINTER(Particles), ctypes.POINTER(i64),
                                     ctypes.POINTER(Beam), vp, ctypes.c_int]
    L.sc_last_error.argtypes = [ctypes.c_char_p, ctypes.c_size_t]
    for name in EXPORTS:
        getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def _check(code):
    if code != SC_OK:
        buf = ctypes.create_string_buffer(1024)
        load().sc_last_error(buf, 1024)
        raise ScError(code, buf.value.decode(errors="replace"))


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


class Grid:
    """An sc_grid: nx x ny nodes over [xmin, xmax] x [ymin, ymax] with its solver."""

    def __init__(self, nx, ny, xmin, xmax, ymin, ymax, precision="fp64", stream=None, slices=None):
        """slices = (n_slices, zmin, zmax) for a longitudinally sliced grid."""
        self.nx, self.ny = int(nx), int(ny)
        self.extent = (float(xmin), float(xmax), float(ymin), float(ymax))
        self.precision = precision
        self.nz = 1 if slices is None else int(slices[0])
        h = ctypes.c_void_p()
        if slices is None:
            _check(load().sc_create_grid(ctypes.byref(h), self.nx, self.ny, *self.extent, PRECISION[precision],
                                         _stream_handle(stream)))
        else:
            _check(load().sc_create_grid_sliced(ctypes.byref(h), self.nx, self.ny, *self.extent, self.nz,
                                                float(slices[1]), float(slices[2]), PRECISION[precision],
                                                _stream_handle(stream)))
        self._h = h

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().sc_destroy_grid(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def create_grid(nx, ny, xmin, xmax, ymin, ymax, precision="fp64", stream=None, slices=None) -> Grid:
    return Grid(nx, ny, xmin, xmax, ymin, ymax, precision, stream, slices)


def particles(state) -> Particles:
    """sc_particles from a dict of six CUDA float64 contiguous tensors of equal length."""
    keys = ("x", "px", "y", "py", "sigma", "psigma")
    ts = [state[k] for k in keys]
    n = int(ts[0].numel())
    for t in ts:
        if not (t.is_cuda and t.dtype.is_floating_point and t.element_size() == 8 and t.is_contiguous()):
            raise ValueError("particle arrays must be contiguous CUDA float64 tensors")
        if t.numel() != n:
            raise ValueError("particle arrays differ in length")
    return Particles(*(t.data_ptr() for t in ts), n)


def beam(b: dict) -> Beam:
    return Beam(*(float(b[k]) for k in ("gamma0", "beta0", "n_lambda", "r_p", "circumference", "mass_ev")))


def _elements(elems):
    if elems is None or len(elems) == 0:
        return None, 0, None
    arr = np.ascontiguousarray(elems, dtype=synth.ELEMENT_DTYPE)
    return arr.ctypes.data, len(arr), arr


def deposit(grid: Grid, state):
    p = particles(state)
    _check(load().sc_deposit(grid.handle, ctypes.byref(p)))


def sort_particles(grid: Grid, state, perm=None):
    """Reorder the bunch (CUDA float64 tensors) in place by its cell on `grid`
    (sc_sort_particles); perm: optional CUDA int32 tensor of n receiving the
    old index of each new position."""
    p = particles(state)
    _check(load().sc_sort_particles(grid.handle, ctypes.byref(p), perm.data_ptr() if perm is not None else None))


def solve(grid: Grid):
    _check(load().sc_solve(grid.handle))


def kick_push(grid: Grid, state, b: dict, L_sc: float, elems=None, next_grid: Grid | None = None):
    p = particles(state)
    bb = beam(b)
    ptr, n, keep = _elements(elems)
    _check(load().sc_kick_push(grid.handle, ctypes.byref(p), ctypes.byref(bb), float(L_sc), ptr, n,
                               next_grid.handle if next_grid is not None else None))


def track_turns(grid: Grid, state, b: dict, lattice, n_turns: int, diag: bool = False):
    p = particles(state)
    bb = beam(b)
    ptr, n, keep = _elements(lattice)
    out = np.zeros((n_turns, 14)) if diag else None
    _check(load().sc_track_turns(grid.handle, ctypes.byref(p), ctypes.byref(bb), ptr, n, int(n_turns),
                                 out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if diag else None))
    return out


def grid_read(grid: Grid):
    """-> (Q uint64, Ex, Ey, n_out); arrays [ny, nx], or [n_slices, ny, nx] for sliced grids"""
    shape = (grid.ny, grid.nx) if grid.nz == 1 else (grid.nz, grid.ny, grid.nx)
    Q = np.zeros(shape, dtype=np.uint64)
    Ex = np.zeros(shape)
    Ey = np.zeros(shape)
    n_out = ctypes.c_int64(0)
    _check(load().sc_grid_read(grid.handle, Q.ctypes.data, Ex.ctypes.data, Ey.ctypes.data, ctypes.byref(n_out)))
    return Q, Ex, Ey, int(n_out.value)


def set_longitudinal_kick(grid: Grid, enable: bool = True):
    """Longitudinal space-charge kick on a sliced conducting-pipe grid."""
    _check(load().sc_set_longitudinal_kick(grid.handle, 1 if enable else 0))


GATHER = {"bilinear": 0, "bezier": 1}


def set_gather(grid: Grid, mode: str):
    """Field gather of the kick: "bilinear" node fields, or "bezier" (Sec. IV-C, pipe grids)."""
    _check(load().sc_set_gather(grid.handle, GATHER[mode]))


def grid_read_potential(grid: Grid):
    """-> phi [ny, nx] (or [n_slices, ny, nx]) of a conducting-pipe grid."""
    shape = (grid.ny, grid.nx) if grid.nz == 1 else (grid.nz, grid.ny, grid.nx)
    phi = np.zeros(shape)
    _check(load().sc_grid_read_potential(grid.handle, phi.ctypes.data))
    return phi


def tune_setup(grid: Grid, state, twiss, acc):
    """Arm per-particle tune accumulation (sc_tune_setup); acc: CUDA float64
    tensor of 4 n elements (None disarms).  twiss = (beta_x, alpha_x, beta_y, alpha_y)."""
    p = particles(state)
    tw = (ctypes.c_double * 4)(*[float(v) for v in twiss])
    _check(load().sc_tune_setup(grid.handle, ctypes.byref(p), tw, acc.data_ptr() if acc is not None else None))


def tunes(acc, n, turns, stream=None):
    """Fractional tunes (qx, qy) per particle from a tune accumulator after
    `turns` turns (sc_tunes on the device), as host arrays."""
    import torch
    q = torch.empty(2 * n, dtype=torch.float64, device=acc.device)
    _check(load().sc_tunes(acc.data_ptr(), n, int(turns), q.data_ptr(), _stream_handle(stream)))
    if stream is not None:
        stream.synchronize()
    q = q.cpu().numpy()
    return q[:n], q[n:]


def trace_enable(grid: Grid, enable: bool = True):
    _check(load().sc_trace_enable(grid.handle, 1 if enable else 0))


def trace_read(grid: Grid):
    """-> (kick_push_ms, solve_ms, n_kicks) accumulated since the last read."""
    a, c, n = ctypes.c_double(0), ctypes.c_double(0), ctypes.c_int64(0)
    _check(load().sc_trace_read(grid.handle, ctypes.byref(a), ctypes.byref(c), ctypes.byref(n)))
    return a.value, c.value, int(n.value)


def get_solver_tiling(grid: Grid):
    """-> ([variant index per phase], description) of a split-TF32 grid."""
    c = (ctypes.c_int * 4)()
    buf = ctypes.create_string_buffer(1024)
    _check(load().sc_get_solver_tiling(grid.handle, c, buf, 1024))
    return list(c), buf.value.decode()


def set_solver_tiling(grid: Grid, choice):
    """Force the split-TF32 solve's kernel variant per phase (-1 keeps one)."""
    _check(load().sc_set_solver_tiling(grid.handle, (ctypes.c_int * 4)(*[int(v) for v in choice])))


class _DeviceArray:
    """A raw device buffer described through __cuda_array_interface__ (no copy)."""

    def __init__(self, ptr, n, typestr):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": typestr, "data": (ptr, False), "version": 2,
                                         "strides": None}


def charge_tensor(grid: Grid):
    """The grid's uint64 charge as a CUDA int64 tensor sharing its memory
    ([nstack * ny * nx], sc_grid_charge_device): sum it across ranks in place
    (e.g. torch.distributed.all_reduce) between the deposit and the solve."""
    import torch
    q, cells = ctypes.c_void_p(), ctypes.c_int64(0)
    _check(load().sc_grid_charge_device(grid.handle, ctypes.byref(q), ctypes.byref(cells)))
    return torch.as_tensor(_DeviceArray(q.value, int(cells.value), "<i8"), device="cuda")


def set_charge_reduce(grid: Grid, reduce, total_particles: int):
    """Sharded bunch inside track_turns (sc_set_charge_reduce): reduce(charge,
    stream) gets the grid's charge as a CUDA int64 tensor and the grid's stream
    (a torch.cuda.ExternalStream) while a turn is captured, and must enqueue
    on that stream an in-place sum of the tensor over the ranks; None switches
    it off.  The callback object is kept on the grid."""
    if reduce is None:
        grid._reduce_cb = None
        _check(load().sc_set_charge_reduce(grid.handle, REDUCE_FN(), None, 0))
        return
    import torch
    q = charge_tensor(grid)

    def cb(ptr, cells, stream, user):
        try:
            reduce(q, torch.cuda.ExternalStream(stream))
            return 0
        except Exception:  # noqa: BLE001 -- a failure becomes the capture's error code
            import traceback
            traceback.print_exc()
            return 1

    grid._reduce_cb = REDUCE_FN(cb)
    _check(load().sc_set_charge_reduce(grid.handle, grid._reduce_cb, None, int(total_particles)))


def set_particle_count(grid: Grid, n: int):
    """The count that normalises the next solve (the whole bunch's, after a cross-rank sum)."""
    _check(load().sc_set_particle_count(grid.handle, int(n)))


def solver_work(grid: Grid):
    """-> (tensor-core flops, FFT-equivalent flops) of one solve on the grid."""
    t, f = ctypes.c_double(0), ctypes.c_double(0)
    _check(load().sc_get_solver_work(grid.handle, ctypes.byref(t), ctypes.byref(f)))
    return t.value, f.value


def set_kick_push_shape(grid: Grid, threads: int = 0, traversal: int = -1):
    """Fix the kick/push block size (0: chosen at capture) and traversal
    (-1: chosen, 0: grid stride, 1: contiguous chunks) of tracked turns."""
    _check(load().sc_set_kick_push_shape(grid.handle, int(threads), int(traversal)))


def get_kick_push_shape(grid: Grid):
    """-> (threads, traversal, trial_us) of the grid's captured turn (trial_us:
    the timed trial of the chosen shape, 0 when the shape was not timed)."""
    t, v, us = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_double(0)
    _check(load().sc_get_kick_push_shape(grid.handle, ctypes.byref(t), ctypes.byref(v), ctypes.byref(us)))
    return int(t.value), int(v.value), us.value


def moments_noalloc(state, out, stream=None):
    """Beam moments into the 14-element CUDA float64 tensor `out`, through the
    entry point that allocates no device memory (sc_moments_noalloc)."""
    p = particles(state)
    _check(load().sc_moments_noalloc(ctypes.byref(p), out.data_ptr(), _stream_handle(stream)))
    return out


def grid_write_charge(grid: Grid, Q, n_particles: int):
    Q = np.ascontiguousarray(Q, dtype=np.uint64)
    assert Q.size == grid.nz * grid.ny * grid.nx
    _check(load().sc_grid_write_charge(grid.handle, Q.ctypes.data, int(n_particles)))


def host_particles(state) -> Particles:
    """sc_particles from a dict of six host float64 arrays of equal length:
    contiguous writable numpy arrays or CPU torch tensors (pinned memory copies
    fastest)."""
    keys = ("x", "px", "y", "py", "sigma", "psigma")
    ptrs, n = [], None
    for k in keys:
        a = state[k]
        if isinstance(a, np.ndarray):
            if a.dtype != np.float64 or not a.flags.c_contiguous or not a.flags.writeable:
                raise ValueError("host particle arrays must be contiguous writable float64")
            ptrs.append(a.ctypes.data)
            m = a.size
        else:
            if a.is_cuda or a.element_size() != 8 or not a.dtype.is_floating_point or not a.is_contiguous():
                raise ValueError("host particle tensors must be contiguous CPU float64")
            ptrs.append(a.data_ptr())
            m = a.numel()
        if n is not None and m != n:
            raise ValueError("particle arrays differ in length")
        n = m
    return Particles(*ptrs, n)


def track_turns_host(grid: Grid, host_state, b: dict, lattice, n_turns: int, diag: bool = False):
    """sc_track_turns_host: track a bunch held in host memory (the library
    copies it to its own device buffers and back); host_state is updated in
    place.  diag -> [n_turns, 14] moments as in track_turns."""
    p = host_particles(host_state)
    bb = beam(b)
    ptr, n, keep = _elements(lattice)
    out = np.zeros((n_turns, 14)) if diag else None
    _check(load().sc_track_turns_host(grid.handle, ctypes.byref(p), ctypes.byref(bb), ptr, n, int(n_turns),
                                      out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if diag else None))
    return out


def checkpoint_write(path, host_state, turn: int, b: dict, lattice):
    """sc_checkpoint_write: the bunch's six host arrays, the turn counter, the
    beam constants and a hash of the lattice into the file `path`."""
    p = host_particles(host_state)
    bb = beam(b)
    ptr, n, keep = _elements(lattice)
    _check(load().sc_checkpoint_write(os.fsencode(path), ctypes.byref(p), int(turn), ctypes.byref(bb), ptr, n))


def checkpoint_read(path, host_state, b: dict, lattice) -> int:
    """sc_checkpoint_read: fill the six host arrays from `path` after checking
    that it was written for this bunch size, beam and lattice; -> the turn counter."""
    p = host_particles(host_state)
    bb = beam(b)
    ptr, n, keep = _elements(lattice)
    t = ctypes.c_int64(0)
    _check(load().sc_checkpoint_read(os.fsencode(path), ctypes.byref(p), ctypes.byref(t), ctypes.byref(bb), ptr, n))
    return int(t.value)


# ---------------------------------------------------------------- batches of bunches
class Batch:
    """An sc_batch: one grid per bunch, grids = [(nx, ny, xmin, xmax, ymin, ymax), ...]."""

    def __init__(self, grids, precision="fp64", stream=None):
        self.grids = [tuple(g) for g in grids]
        arr = (GridSpec * len(self.grids))(*[GridSpec(int(g[0]), int(g[1]), *map(float, g[2:])) for g in self.grids])
        h = ctypes.c_void_p()
        _check(load().sc_create_batch(ctypes.byref(h), arr, len(self.grids), PRECISION[precision],
                                      _stream_handle(stream)))
        self._h = h
        self.precision = precision

    @property
    def handle(self):
        return self._h

    def __len__(self):
        return len(self.grids)

    def __del__(self):
        try:
            if self._h:
                load().sc_destroy_batch(self._h)
                self._h = None
        except Exception:
            pass


def create_batch(grids, precision="fp64", stream=None) -> Batch:
    return Batch(grids, precision, stream)


def batch_track_turns(batch: Batch, states, beams, lattices, n_turns: int, diag: bool = False):
    """Track every bunch n_turns turns (sc_batch_track_turns); states, beams and
    lattices are per-bunch lists.  diag -> [n_turns, n_bunches, 14]."""
    nb = len(batch)
    if not (len(states) == len(beams) == len(lattices) == nb):
        raise ValueError("one state, beam and lattice per bunch")
    keep = []
    arr = (Bunch * nb)()
    for b in range(nb):
        ptr, n, k = _elements(lattices[b])
        keep.append(k)
        arr[b] = Bunch(particles(states[b]), beam(beams[b]), ptr, n)
    out = np.zeros((n_turns, nb, 14)) if diag else None
    _check(load().sc_batch_track_turns(batch.handle, arr, int(n_turns),
                                       out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if diag else None))
    return out


def batch_track_turns_host(batch: Batch, host_states, beams, lattices, n_turns: int, diag: bool = False):
    """sc_batch_track_turns_host: bunches held in host memory (numpy arrays or
    CPU torch tensors, updated in place); diag -> [n_turns, n_bunches, 14]."""
    nb = len(batch)
    if not (len(host_states) == len(beams) == len(lattices) == nb):
        raise ValueError("one state, beam and lattice per bunch")
    keep = []
    arr = (Bunch * nb)()
    for b in range(nb):
        ptr, n, k = _elements(lattices[b])
        keep.append(k)
        arr[b] = Bunch(host_particles(host_states[b]), beam(beams[b]), ptr, n)
    out = np.zeros((n_turns, nb, 14)) if diag else None
    _check(load().sc_batch_track_turns_host(batch.handle, arr, int(n_turns),
                                            out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if diag else None))
    return out


def batch_set_kick_push_shape(batch: Batch, threads: int = 0, waves: int = 0):
    """Fix the batched kick/push block size and waves per launch (0: chosen at capture)."""
    _check(load().sc_batch_set_kick_push_shape(batch.handle, int(threads), int(waves)))


def batch_get_kick_push_shape(batch: Batch):
    """-> (threads, waves, trial_us) of the batch's captured turn."""
    t, w, us = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_double(0)
    _check(load().sc_batch_get_kick_push_shape(batch.handle, ctypes.byref(t), ctypes.byref(w), ctypes.byref(us)))
    return int(t.value), int(w.value), us.value


def batch_read(batch: Batch, b: int):
    """-> (Q uint64 [ny, nx], Ex, Ey, n_out) of bunch b's grid."""
    nx, ny = batch.grids[b][0], batch.grids[b][1]
    Q = np.zeros((ny, nx), dtype=np.uint64)
    Ex = np.zeros((ny, nx))
    Ey = np.zeros((ny, nx))
    n_out = ctypes.c_int64(0)
    _check(load().sc_batch_read(batch.handle, int(b), Q.ctypes.data, Ex.ctypes.data, Ey.ctypes.data,
                                ctypes.byref(n_out)))
    return Q, Ex, Ey, int(n_out.value)


def batch_get_solver_tiling(batch: Batch, b: int):
    """-> ([variant index per phase], description) of bunch b's grid class."""
    c = (ctypes.c_int * 4)()
    buf = ctypes.create_string_buffer(1024)
    _check(load().sc_batch_get_solver_tiling(batch.handle, int(b), c, buf, 1024))
    return list(c), buf.value.decode()


def batch_set_solver_tiling(batch: Batch, choice):
    _check(load().sc_batch_set_solver_tiling(batch.handle, (ctypes.c_int * 4)(*[int(v) for v in choice])))


def batch_trace_enable(batch: Batch, enable: bool = True):
    _check(load().sc_batch_trace_enable(batch.handle, 1 if enable else 0))


def batch_trace_read(batch: Batch):
    """-> (kick_push_ms, solve_ms, n_kicks) accumulated since the last read."""
    a, c, n = ctypes.c_double(0), ctypes.c_double(0), ctypes.c_int64(0)
    _check(load().sc_batch_trace_read(batch.handle, ctypes.byref(a), ctypes.byref(c), ctypes.byref(n)))
    return a.value, c.value, int(n.value)
