"""FP64 CPU oracle of the 2-D PIC space-charge step (arXiv:2010.11540).

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and the
cpu_baseline / reference legs of bench.py, never by the product package.  It
shares no code with the CUDA path; the seeded inputs come from
paper_2010_11540_gb300.synth, which the caller passes in as plain arrays.

The particle loops are plain C (sc_oracle.c, built with -ffp-contract=off
and OpenMP: set_threads(n) splits them over n threads, bit-identically to one
thread); the open-boundary convolution uses a library FFT (pocketfft, through
scipy.fft with one worker per thread when scipy is present, else numpy.fft)
as the primitive of Hockney's zero-padded method (Sec. I reference
[Hockney]); the tracking loop follows the PIC loop of Sec. I (deposit ->
Poisson -> kick/push) with the kick of Sec. IV.

Every function is pinned by tests/test_oracle_*.py against something other
than itself (closed forms, invariants, brute force on tiny inputs, values the
paper prints).  The long-run statistics (100-turn emittances and tune spreads
of an unmatched beam) have no closed form: track(), which produces them, is
pinned step by step (one-turn pins, the small-amplitude tune shift, the maps'
symplecticity, thread bit-identity), not over 100 turns.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sc_oracle.c")
_LIB = os.path.join(_HERE, "libsc_oracle.so")

ONE_FX = 1 << 20  # fixed-point unit per axis
Q_UNIT = float(1 << 40)  # one particle's total deposited charge

DRIFT, QUAD, SEXT, BEND, RF, MARK, EXACT_BEND = 0, 1, 2, 3, 4, 5, 6


def build(force=False):
    """Compile the C oracle (gcc, -O2 -ffp-contract=off, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared",
                               "-std=c11", "-D_DEFAULT_SOURCE", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Beam(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in
                ("gamma0", "beta0", "n_lambda", "r_p", "circumference", "mass_ev")]


_lib = None
_dp = ctypes.POINTER(ctypes.c_double)
_lp = ctypes.POINTER(ctypes.c_uint64)


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        L.orc_deposit.restype = ctypes.c_uint64
        L.orc_deposit.argtypes = [ctypes.c_int64, _dp, _dp, ctypes.c_int, ctypes.c_int,
                                  ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double, _lp]
        L.orc_deposit_sliced.restype = ctypes.c_uint64
        L.orc_deposit_sliced.argtypes = [ctypes.c_int64, _dp, _dp, _dp, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                         ctypes.c_int, ctypes.c_double, ctypes.c_double, _lp]
        L.orc_kick_sliced.restype = None
        L.orc_kick_sliced.argtypes = [ctypes.c_int64, _dp, _dp, _dp, _dp, _dp, ctypes.c_int, ctypes.c_int,
                                      ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_int, ctypes.c_double, ctypes.c_double, _dp, _dp, ctypes.c_double]
        L.orc_kick_long.restype = None
        L.orc_kick_long.argtypes = [ctypes.c_int64, _dp, _dp, _dp, _dp, ctypes.c_int, ctypes.c_int,
                                    ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                    ctypes.c_int, ctypes.c_double, ctypes.c_double, _dp, ctypes.c_double]
        L.orc_kick_bezier.restype = None
        L.orc_kick_bezier.argtypes = [ctypes.c_int64, _dp, _dp, _dp, _dp, _dp, _dp, ctypes.c_int, ctypes.c_int,
                                      ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_double,
                                      ctypes.c_double, _dp, ctypes.c_double, ctypes.c_double]
        L.orc_bezier_point.restype = None
        L.orc_bezier_point.argtypes = [_dp, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, _dp]
        L.orc_green_self.restype = ctypes.c_double
        L.orc_green_self.argtypes = [ctypes.c_double, ctypes.c_double]
        L.orc_green_cyclic.restype = None
        L.orc_green_cyclic.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, _dp]
        L.orc_potential_direct.restype = None
        L.orc_potential_direct.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                           _dp, _dp]
        L.orc_fields.restype = None
        L.orc_fields.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, _dp, _dp, _dp]
        L.orc_kick.restype = None
        L.orc_kick.argtypes = [ctypes.c_int64, _dp, _dp, _dp, _dp, ctypes.c_int, ctypes.c_int,
                               ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                               _dp, _dp, ctypes.c_double]
        L.orc_push.restype = None
        L.orc_push.argtypes = [ctypes.c_int64, _dp, _dp, _dp, _dp, _dp, _dp, ctypes.c_void_p, ctypes.c_int,
                               ctypes.POINTER(_Beam)]
        L.orc_moments.restype = None
        L.orc_moments.argtypes = [ctypes.c_int64, _dp, _dp, _dp, _dp, _dp, _dp, _dp]
        L.orc_set_threads.restype = ctypes.c_int
        L.orc_set_threads.argtypes = [ctypes.c_int]
        L.orc_max_threads.restype = ctypes.c_int
        L.orc_max_threads.argtypes = []
        _lib = L
    return _lib


_threads = 1


def set_threads(n=None):
    """Threads of the particle loops and FFT workers (None: every core);
    returns the count in use.  Results are bit-identical for any count."""
    global _threads
    L = lib()
    _threads = int(L.orc_set_threads(int(L.orc_max_threads() if n is None else n)))
    return _threads


def threads():
    return _threads


try:  # the library FFT of the convolution: pocketfft through scipy (threaded) or numpy
    import scipy.fft as _sfft

    def _rfft2(a):
        return _sfft.rfft2(a, workers=_threads)

    def _irfft2(a, s):
        return _sfft.irfft2(a, s=s, workers=_threads)
except ImportError:  # pragma: no cover
    def _rfft2(a):
        return np.fft.rfft2(a)

    def _irfft2(a, s):
        return np.fft.irfft2(a, s=s)


def _d(a):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_dp)


def _beam(b):
    return _Beam(*(float(b[k]) for k in ("gamma0", "beta0", "n_lambda", "r_p", "circumference", "mass_ev")))


# ---------------------------------------------------------------------------
# Grid geometry (nodes x_i = xmin + i*hx, i = 0..nx-1)
# ---------------------------------------------------------------------------
class Geometry:
    def __init__(self, nx, ny, xmin, xmax, ymin, ymax):
        self.nx, self.ny = int(nx), int(ny)
        self.xmin, self.xmax, self.ymin, self.ymax = map(float, (xmin, xmax, ymin, ymax))
        self.hx = (self.xmax - self.xmin) / (self.nx - 1)
        self.hy = (self.ymax - self.ymin) / (self.ny - 1)
        self.inv_hx = 1.0 / self.hx
        self.inv_hy = 1.0 / self.hy

    @property
    def node_x(self):
        return self.xmin + np.arange(self.nx) * self.hx

    @property
    def node_y(self):
        return self.ymin + np.arange(self.ny) * self.hy


class Slices:
    """Longitudinal slicing: nz bins of sigma over [zmin, zmax) (the line density
    lambda(z) of Sec. IV as a histogram of sigma), each bin with its own grid."""

    def __init__(self, nz, zmin, zmax):
        self.nz, self.zmin, self.zmax = int(nz), float(zmin), float(zmax)
        self.dz = (self.zmax - self.zmin) / self.nz
        self.inv_dz = 1.0 / self.dz


def deposit_sliced(g: Geometry, zs: Slices, x, y, sg):
    """CIC deposit per slice -> (Q uint64 [nz, ny, nx], n_out)."""
    Q = np.zeros((zs.nz, g.ny, g.nx), dtype=np.uint64)
    n_out = lib().orc_deposit_sliced(len(x), _d(x), _d(y), _d(sg), g.nx, g.ny, g.xmin, g.ymin, g.inv_hx, g.inv_hy,
                                     zs.nz, zs.zmin, zs.inv_dz, Q.ctypes.data_as(_lp))
    return Q, int(n_out)


def kick_sliced(g: Geometry, zs: Slices, st, Ex, Ey, kl):
    lib().orc_kick_sliced(len(st["x"]), _d(st["x"]), _d(st["y"]), _d(st["sigma"]), _d(st["px"]), _d(st["py"]),
                          g.nx, g.ny, g.xmin, g.ymin, g.inv_hx, g.inv_hy, zs.nz, zs.zmin, zs.inv_dz,
                          _d(np.ascontiguousarray(Ex)), _d(np.ascontiguousarray(Ey)), kl)


def potential_sliced_pipe(g: Geometry, Q, n_total):
    """Node potentials [nz, ny, nx] of every slice in the conducting pipe
    (each slice's charge normalised by the total count)."""
    return np.stack([potential_pipe(g, normalise(Q[k], n_total))[1:-1, 1:-1] for k in range(Q.shape[0])])


def kick_long(g: Geometry, zs: Slices, st, phi, klz):
    """Longitudinal kick of Sec. IV on sliced potentials (see orc_kick_long);
    klz = K gamma0 L / (2 dz)."""
    lib().orc_kick_long(len(st["x"]), _d(st["x"]), _d(st["y"]), _d(st["sigma"]), _d(st["psigma"]), g.nx, g.ny,
                        g.xmin, g.ymin, g.inv_hx, g.inv_hy, zs.nz, zs.zmin, zs.inv_dz,
                        _d(np.ascontiguousarray(phi, dtype=np.float64)), klz)


def bezier_point(g: Geometry, phi, i, j, fx, fy):
    """(u, du/dx, du/dy) of the Bezier surface (Sec. IV-C) of node potentials
    phi [ny, nx] in cell (i, j) at fractions (fx, fy)."""
    out = np.zeros(3)
    lib().orc_bezier_point(_d(np.ascontiguousarray(phi, dtype=np.float64)), g.nx, g.ny, g.hx, g.hy, int(i), int(j),
                           float(fx), float(fy), _d(out))
    return out


def kick_bezier(g: Geometry, zs, st, phi, kl, klz=0.0):
    """Space-charge kick from the Bezier surface of the node potentials
    (Sec. IV-C), phi [nz, ny, nx] (nz = 1 unsliced); with klz the longitudinal
    kick from the same surfaces."""
    nz, zmin, inv_dz = (1, 0.0, 0.0) if zs is None else (zs.nz, zs.zmin, zs.inv_dz)
    lib().orc_kick_bezier(len(st["x"]), _d(st["x"]), _d(st["y"]), _d(st["sigma"]), _d(st["px"]), _d(st["py"]),
                          _d(st["psigma"]), g.nx, g.ny, g.xmin, g.ymin, g.inv_hx, g.inv_hy, g.hx, g.hy, nz, zmin,
                          inv_dz, _d(np.ascontiguousarray(phi, dtype=np.float64)), kl, klz)


def solve_sliced(g: Geometry, Q, n_total, method="fft", boundary="open"):
    """Per-slice fields (Ex, Ey) [nz, ny, nx], each slice's charge normalised by
    the total macroparticle count."""
    out = [solve(g, Q[k], n_total, method, boundary) for k in range(Q.shape[0])]
    return np.stack([e[0] for e in out]), np.stack([e[1] for e in out])


def deposit(g: Geometry, x, y):
    """CIC deposit (Sec. IV-A) -> (Q uint64 [ny, nx], n_out)."""
    Q = np.zeros((g.ny, g.nx), dtype=np.uint64)
    n_out = lib().orc_deposit(len(x), _d(x), _d(y), g.nx, g.ny, g.xmin, g.ymin, g.inv_hx, g.inv_hy,
                              Q.ctypes.data_as(_lp))
    return Q, int(n_out)


def deposit_cells(g: Geometry, x, y):
    """Cell index j*nx + i of each particle by the deposit's rule (Sec. IV-A:
    xi = (x - xmin) / hx, inside iff 0 <= xi < nx-1, likewise eta), -1 outside."""
    xi = (np.asarray(x, dtype=np.float64) - g.xmin) * g.inv_hx
    eta = (np.asarray(y, dtype=np.float64) - g.ymin) * g.inv_hy
    with np.errstate(invalid="ignore"):
        inside = (xi >= 0.0) & (xi < g.nx - 1) & (eta >= 0.0) & (eta < g.ny - 1)
    cell = np.full(len(xi), -1, dtype=np.int64)
    cell[inside] = np.floor(eta[inside]).astype(np.int64) * g.nx + np.floor(xi[inside]).astype(np.int64)
    return cell


def green_self(hx, hy):
    return lib().orc_green_self(hx, hy)


def green_cyclic(g: Geometry):
    G = np.zeros((2 * g.ny, 2 * g.nx))
    lib().orc_green_cyclic(g.nx, g.ny, g.hx, g.hy, _d(G))
    return G


def normalise(Q, n_total):
    """q = Q 2^-40 / N_mp: each macroparticle carries 1/N_mp of the line charge."""
    return Q.astype(np.float64) / Q_UNIT / float(n_total)


def potential_direct(g: Geometry, q):
    """phi on nodes i=-1..nx, j=-1..ny by direct pairwise sum (small grids only)."""
    q = np.ascontiguousarray(q, dtype=np.float64)
    phi = np.zeros((g.ny + 2, g.nx + 2))
    lib().orc_potential_direct(g.nx, g.ny, g.hx, g.hy, _d(q), _d(phi))
    return phi


_green_spectra = {}


def green_spectrum(g: Geometry):
    """rfft2 of green_cyclic(g), kept per geometry (it depends on nx, ny, hx, hy only)."""
    key = (g.nx, g.ny, g.hx, g.hy)
    if key not in _green_spectra:
        if len(_green_spectra) > 16:
            _green_spectra.clear()
        _green_spectra[key] = _rfft2(green_cyclic(g))
    return _green_spectra[key]


def potential_fft(g: Geometry, q):
    """phi on nodes i=-1..nx, j=-1..ny: Hockney's method, q zero-padded to the
    doubled grid and cyclically convolved with G by FFT (pocketfft, float64)."""
    Mx, My = 2 * g.nx, 2 * g.ny
    qp = np.zeros((My, Mx))
    qp[: g.ny, : g.nx] = q
    phi = _irfft2(_rfft2(qp) * green_spectrum(g), s=(My, Mx))
    iy = np.r_[My - 1, np.arange(0, g.ny + 1)]
    ix = np.r_[Mx - 1, np.arange(0, g.nx + 1)]
    return np.ascontiguousarray(phi[np.ix_(iy, ix)])


def fields(g: Geometry, phi_ext):
    """E = -grad phi at the nodes by centred differences -> (Ex, Ey) [ny, nx]."""
    phi_ext = np.ascontiguousarray(phi_ext, dtype=np.float64)
    Ex = np.zeros((g.ny, g.nx))
    Ey = np.zeros((g.ny, g.nx))
    lib().orc_fields(g.nx, g.ny, g.hx, g.hy, _d(phi_ext), _d(Ex), _d(Ey))
    return Ex, Ey


def potential_pipe(g: Geometry, q):
    """Potential inside a rectangular conducting pipe whose walls are the
    grid's outer nodes (Sec. IV-B: Eqs. poisson2D, boundary, disc, extension,
    solution), on nodes i = -1..nx, j = -1..ny.

    The 5-point discretisation (Eq. disc) holds on the m_x x m_y interior
    nodes (m = n - 2), with phi = 0 on the walls (Eq. boundary).  Its right-hand
    side is the density of the normalised line charge with the sign and 2 pi
    of the free-space Green function -ln r that the open solve uses
    (lap(-ln r) = -2 pi delta): f = -2 pi q / (hx hy).  The paper's steps:
    F = odd extension of f to period 2(m+1) along both axes (Eq. extension);
    2-D DFT of F (numpy FFT, the library step); division by
    -4 (sin^2(p pi / 2(m+1)) / hx^2 + sin^2(q pi / 2(m+1)) / hy^2), indices
    p, q = 0 .. 2m+1 (the paper prints 1..N: a garble; the p = q = 0 term of an
    odd extension is 0 and stays 0); inverse 2-D DFT; V at the interior nodes
    is phi.  The ring of nodes just outside the walls takes the odd extension
    (phi(-1) = -phi(1)), so centred differences give the field at the walls."""
    mx, my = g.nx - 2, g.ny - 2
    f = -2.0 * np.pi * np.asarray(q, dtype=np.float64)[1:-1, 1:-1] / (g.hx * g.hy)

    def odd(a, axis):
        z = np.zeros_like(np.take(a, [0], axis=axis))
        return np.concatenate([z, a, z, -np.flip(a, axis=axis)], axis=axis)

    F = odd(odd(f, 1), 0)  # [2(my+1), 2(mx+1)]
    P = 2 * (mx + 1)
    Qn = 2 * (my + 1)
    sp = np.sin(np.arange(P) * np.pi / P) ** 2 / g.hx ** 2
    sq = np.sin(np.arange(Qn) * np.pi / Qn) ** 2 / g.hy ** 2
    den = -4.0 * (sq[:, None] + sp[None, :])
    Fh = np.fft.fft2(F)
    Vh = np.zeros_like(Fh)
    nz = den != 0.0
    Vh[nz] = Fh[nz] / den[nz]
    V = np.fft.ifft2(Vh).real
    phi = np.zeros((g.ny + 2, g.nx + 2))
    phi[2:-2, 2:-2] = V[1:my + 1, 1:mx + 1]
    # odd extension across the walls (rows/columns 1 and n hold the walls, 0 and n+1 the ring)
    phi[:, 0] = -phi[:, 2]
    phi[:, -1] = -phi[:, -3]
    phi[0, :] = -phi[2, :]
    phi[-1, :] = -phi[-3, :]
    return phi


def solve(g: Geometry, Q, n_total, method="fft", boundary="open"):
    """Charge grid -> node fields (Ex, Ey), normalised per unit line charge.
    boundary "open": free space (Hockney); "pipe": conducting rectangular pipe
    on the grid's outer nodes (Sec. IV-B)."""
    q = normalise(Q, n_total)
    if boundary == "pipe":
        return fields(g, potential_pipe(g, q))
    phi = potential_fft(g, q) if method == "fft" else potential_direct(g, q)
    return fields(g, phi)


def kick_strength(b):
    """K = 2 r_p N_lambda / (beta0^2 gamma0^3) (Sec. IV kick eq. and Eq. pot2)."""
    return 2.0 * b["r_p"] * b["n_lambda"] / (b["beta0"] ** 2 * b["gamma0"] ** 3)


def kick(g: Geometry, st, Ex, Ey, kl):
    lib().orc_kick(len(st["x"]), _d(st["x"]), _d(st["y"]), _d(st["px"]), _d(st["py"]), g.nx, g.ny,
                   g.xmin, g.ymin, g.inv_hx, g.inv_hy, _d(np.ascontiguousarray(Ex)),
                   _d(np.ascontiguousarray(Ey)), kl)


def push(st, elems, b):
    elems = np.ascontiguousarray(elems)
    if len(elems) == 0:
        return
    bb = _beam(b)
    lib().orc_push(len(st["x"]), _d(st["x"]), _d(st["px"]), _d(st["y"]), _d(st["py"]), _d(st["sigma"]),
                   _d(st["psigma"]), elems.ctypes.data, len(elems), ctypes.byref(bb))


def moments(st):
    out = np.zeros(14)
    lib().orc_moments(len(st["x"]), _d(st["x"]), _d(st["px"]), _d(st["y"]), _d(st["py"]), _d(st["sigma"]),
                      _d(st["psigma"]), _d(out))
    return out


def emittances(st):
    """rms emittances eps_u = sqrt(<uu><pp> - <up>^2) (Sec. V)."""
    m = moments(st)
    ex = np.sqrt(m[6] * m[8] - m[7] ** 2)
    ey = np.sqrt(m[9] * m[11] - m[10] ** 2)
    return ex, ey


def copy_state(st):
    return {k: np.array(v, dtype=np.float64, copy=True) for k, v in st.items()}


# ---------------------------------------------------------------------------
# Lattice: space-charge locations and the segments between them (Sec. V:
# kicks at chosen locations, L = distance since the previous location).
# ---------------------------------------------------------------------------
def segments(lattice):
    """-> (head, kicks): head = elements before the first marker; kicks = list of
    (L_since_previous_marker, elements_after_this_marker_up_to_the_next)."""
    lat = np.asarray(lattice)
    marks = [i for i in range(len(lat)) if int(lat["type"][i]) == MARK]
    s = np.concatenate([[0.0], np.cumsum(lat["length"])])
    circ = float(s[-1])
    if not marks:
        return lat, []
    head = lat[: marks[0]]
    kicks = []
    for k, m in enumerate(marks):
        end = marks[k + 1] if k + 1 < len(marks) else len(lat)
        prev = s[marks[k - 1]] if k > 0 else s[marks[-1]] - circ
        kicks.append((float(s[m] - prev), lat[m + 1:end]))
    return head, kicks


def track(g: Geometry, st, b, lattice, n_turns, method="fft", diag=None, max_kicks=None, slices=None,
          boundary="open", longitudinal=False, gather="bilinear"):
    """Track `st` (modified in place) for n_turns with the PIC loop of Sec. I.
    Each space-charge location: deposit -> solve -> kick (L since the previous
    location) -> push to the next location.  Returns the number of kicks done.
    `diag(turn, st)` is called at the start of every turn.  With `slices`
    (a Slices), every slice has its own grid and b["n_lambda"] is the line
    density of a slice that held the whole bunch (N / dz).  boundary "pipe":
    the conducting-pipe solve of Sec. IV-B on the grid's outer nodes.
    longitudinal (sliced pipe grids): also the longitudinal kick of Sec. IV,
    after the transverse one, from the same positions.  gather "bezier" (pipe
    grids): kicks from the Bezier surface of the potential (Sec. IV-C)."""
    if longitudinal and (slices is None or boundary != "pipe"):
        raise ValueError("the longitudinal kick needs sliced grids in a conducting pipe")
    if gather == "bezier" and boundary != "pipe":
        raise ValueError("the Bezier gather needs the potential of a conducting pipe")
    head, kicks = segments(lattice)
    K = kick_strength(b)
    n = len(st["x"])
    done = 0
    for t in range(n_turns):
        if diag is not None:
            diag(t, st)
        push(st, head, b)
        for L, seg in kicks:
            if max_kicks is not None and done >= max_kicks:
                return done
            if gather == "bezier":
                if slices is None:
                    Q, _ = deposit(g, st["x"], st["y"])
                    phi = potential_pipe(g, normalise(Q, n))[1:-1, 1:-1][None]
                else:
                    Q, _ = deposit_sliced(g, slices, st["x"], st["y"], st["sigma"])
                    phi = potential_sliced_pipe(g, Q, n)
                klz = K * b["gamma0"] * L / (2.0 * slices.dz) if longitudinal else 0.0
                kick_bezier(g, slices, st, phi, K * L, klz)
            elif slices is None:
                Q, _ = deposit(g, st["x"], st["y"])
                Ex, Ey = solve(g, Q, n, method, boundary)
                kick(g, st, Ex, Ey, K * L)
            else:
                Q, _ = deposit_sliced(g, slices, st["x"], st["y"], st["sigma"])
                Ex, Ey = solve_sliced(g, Q, n, method, boundary)
                if longitudinal:
                    phi = potential_sliced_pipe(g, Q, n)
                    klz = K * b["gamma0"] * L / (2.0 * slices.dz)
                kick_sliced(g, slices, st, Ex, Ey, K * L)
                if longitudinal:
                    kick_long(g, slices, st, phi, klz)
            push(st, seg, b)
            done += 1
    return done


# ---------------------------------------------------------------------------
# Linear optics diagnostics (Sec. V: beta from rms size, tunes from the
# one-turn phase advance).
# ---------------------------------------------------------------------------
def one_turn_matrix(lattice, b, eps=1e-8, ps=0.0):
    """4x4 transverse one-turn matrix at the given psigma by central differences
    of the push (space charge off)."""
    M = np.zeros((4, 4))
    keys = ("x", "px", "y", "py")
    for c in range(4):
        st = {k: np.zeros(2) for k in ("x", "px", "y", "py", "sigma", "psigma")}
        st["psigma"][:] = ps
        st[keys[c]][0] = eps
        st[keys[c]][1] = -eps
        push(st, np.asarray(lattice), b)
        for r in range(4):
            M[r, c] = (st[keys[r]][0] - st[keys[r]][1]) / (2 * eps)
    return M


def twiss_from_matrix(M2):
    """(mu, beta, alpha) of a 2x2 periodic matrix: cos mu = Tr/2."""
    cmu = 0.5 * (M2[0, 0] + M2[1, 1])
    smu = np.sign(M2[0, 1]) * np.sqrt(1.0 - cmu * cmu)
    mu = np.arctan2(smu, cmu)
    beta = M2[0, 1] / smu
    alpha = (M2[0, 0] - M2[1, 1]) / (2.0 * smu)
    return mu % (2 * np.pi), beta, alpha


def bare_tunes(lattice, b):
    M = one_turn_matrix(lattice, b)
    qx = twiss_from_matrix(M[:2, :2])[0] / (2 * np.pi)
    qy = twiss_from_matrix(M[2:, 2:])[0] / (2 * np.pi)
    return qx, qy


class PhaseAdvance:
    """Per-particle tunes as the mean one-turn phase advance (Sec. V), in
    normalised coordinates of the bare one-turn Twiss at the observation point.
    Returns fractional tunes in [0, 1)."""

    def __init__(self, beta_x, alpha_x, beta_y, alpha_y):
        self.t = (beta_x, alpha_x, beta_y, alpha_y)
        self.prev = None
        self.acc = None
        self.turns = 0

    def _angles(self, st):
        bx, ax, by, ay = self.t
        X, PX = st["x"] / np.sqrt(bx), (ax * st["x"] + bx * st["px"]) / np.sqrt(bx)
        Y, PY = st["y"] / np.sqrt(by), (ay * st["y"] + by * st["py"]) / np.sqrt(by)
        return np.arctan2(-PX, X), np.arctan2(-PY, Y)

    def __call__(self, turn, st):
        ang = self._angles(st)
        if self.prev is not None:
            d = [np.mod(a - p, 2 * np.pi) for a, p in zip(ang, self.prev)]
            self.acc = d if self.acc is None else [s + x for s, x in zip(self.acc, d)]
            self.turns += 1
        self.prev = ang

    def tunes(self):
        return [a / (2 * np.pi * self.turns) for a in self.acc]
