"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the CPU oracle.

This module draws random numbers and lays out plain data (particle arrays,
element tables, grid extents, beam constants).  It holds none of the
space-charge method's arithmetic: no deposition, no field, no transfer map.

Workloads stand in for the paper's J-PARC Main Ring runs (Sec. V, Table II:
2e5 macroparticles, ~100x100 grids, ~1 m between space-charge locations),
whose lattice is not available; they are synthetic FODO rings.

Element table layout (one 64-byte record per element, the C-ABI `sc_element`):
    type:int32, pad:int32, length, k1, k2l, angle, volt, harmonic, lag (float64)
Element type codes are part of the C-ABI (include/sc.h):
    0 drift (exact, Sec. III-A), 1 thick quadrupole (Sec. III-B),
    2 thin sextupole (Sec. III-C, single-kick limit), 3 sector dipole (Sec. III-A),
    4 thin RF cavity (Sec. V), 5 space-charge location marker (Sec. IV, kick eq.).
"""
from __future__ import annotations

import numpy as np

# ---- element table -------------------------------------------------------
DRIFT, QUAD, SEXT, BEND, RF, MARK, EXACT_BEND = 0, 1, 2, 3, 4, 5, 6

ELEMENT_DTYPE = np.dtype(
    [
        ("type", "<i4"),
        ("pad", "<i4"),
        ("length", "<f8"),
        ("k1", "<f8"),
        ("k2l", "<f8"),
        ("angle", "<f8"),
        ("volt", "<f8"),
        ("harmonic", "<f8"),
        ("lag", "<f8"),
    ],
    align=True,
)
assert ELEMENT_DTYPE.itemsize == 64

# ---- physical constants (CODATA 2018) ------------------------------------
PROTON_MASS_EV = 938.27208816e6
CLASSICAL_PROTON_RADIUS = 2.8179403262e-15 / 1836.15267343  # m: r_e / (m_p/m_e)
# The paper prints r_p ~ 1.547e-18 m next to its tune-spread formula (Sec. V);
# the CODATA value above is used everywhere except the test that reproduces
# the paper's printed -0.45.
PAPER_PROTON_RADIUS = 1.547e-18


def elem(type_, length=0.0, k1=0.0, k2l=0.0, angle=0.0, volt=0.0, harmonic=0.0, lag=0.0):
    """One element record as a tuple in ELEMENT_DTYPE order."""
    return (type_, 0, length, k1, k2l, angle, volt, harmonic, lag)


def table(elems) -> np.ndarray:
    return np.array(list(elems), dtype=ELEMENT_DTYPE)


def kinematics(kinetic_ev: float, mass_ev: float = PROTON_MASS_EV):
    """gamma0, beta0 of the reference particle from its kinetic energy."""
    gamma0 = 1.0 + kinetic_ev / mass_ev
    beta0 = float(np.sqrt(1.0 - 1.0 / (gamma0 * gamma0)))
    return gamma0, beta0


def beam(kinetic_ev=3.0e9, n_lambda=5.0e9, circumference=0.0, r_p=CLASSICAL_PROTON_RADIUS):
    """Beam constants as a plain dict (the C-ABI `sc_beam` fields)."""
    g, b = kinematics(kinetic_ev)
    return dict(gamma0=g, beta0=b, n_lambda=n_lambda, r_p=r_p,
                circumference=circumference, mass_ev=PROTON_MASS_EV)


# ---- particles -----------------------------------------------------------
def _truncated_normal(rng, n, sigma, cut):
    out = rng.standard_normal(n)
    bad = np.abs(out) > cut
    while bad.any():
        out[bad] = rng.standard_normal(int(bad.sum()))
        bad = np.abs(out) > cut
    return out * sigma


def gaussian_bunch(n, seed, sig_x, sig_y, sig_px, sig_py, sig_psigma=1e-3,
                   z_half=10.0, trunc=4.0, sig_z=None, z_trunc=4.0):
    """6-D particle arrays (x, px, y, py, sigma, psigma), float64, C-contiguous.

    Transverse: independent Gaussians, each truncated at `trunc` sigma (redraw).
    Longitudinal: sigma uniform on [-z_half, z_half], or Gaussian with rms
    `sig_z` truncated at `z_trunc` sigma when `sig_z` is given.
    Momentum: psigma Gaussian with rms `sig_psigma` (psigma equals dp/p to
    first order, Sec. III).
    Random numbers: numpy Philox counter-based generator keyed by `seed`.
    """
    rng = np.random.Generator(np.random.Philox(key=int(seed)))
    x = _truncated_normal(rng, n, sig_x, trunc)
    px = _truncated_normal(rng, n, sig_px, trunc)
    y = _truncated_normal(rng, n, sig_y, trunc)
    py = _truncated_normal(rng, n, sig_py, trunc)
    if sig_z is None:
        sg = rng.uniform(-z_half, z_half, n)
    else:
        sg = _truncated_normal(rng, n, sig_z, z_trunc)
    ps = rng.standard_normal(n) * sig_psigma
    return {k: np.ascontiguousarray(v, dtype=np.float64)
            for k, v in zip(("x", "px", "y", "py", "sigma", "psigma"), (x, px, y, py, sg, ps))}


def uniform_disk(n, seed, radius, cx=0.0, cy=0.0):
    """Round uniform (KV-like transverse projection) beam of given radius."""
    rng = np.random.Generator(np.random.Philox(key=int(seed)))
    r = radius * np.sqrt(rng.uniform(0.0, 1.0, n))
    t = rng.uniform(0.0, 2.0 * np.pi, n)
    return cx + r * np.cos(t), cy + r * np.sin(t)


def uniform_points(n, seed, lo, hi):
    rng = np.random.Generator(np.random.Philox(key=int(seed)))
    return rng.uniform(lo, hi, n), rng.uniform(lo, hi, n)


# ---- lattices --------------------------------------------------------------
def fodo_c1():
    """24 identical FODO cells: QF(0.5 m, k1=+0.5) D(5) QD(0.5 m, k1=-0.5) D(5),
    a space-charge location after each drift (48 per turn, 5.5 m apart)."""
    cell = [elem(QUAD, 0.5, k1=0.5), elem(DRIFT, 5.0), elem(MARK),
            elem(QUAD, 0.5, k1=-0.5), elem(DRIFT, 5.0), elem(MARK)]
    return table(cell * 24)


# Quadrupole gradients of the 72-cell ring, matched to bare tunes
# (22.40, 20.75) at psigma = 0 by oracle/match_ring.py (Newton on the
# one-turn matrix trace).
C2_K1F = 0.14154544140329006
C2_K1D = -0.13573619989395166
C2_K2L = 0.5 * 0.2  # k2 = 0.5 m^-3 over 0.2 m


def ring_c2_cell(k1f=C2_K1F, k1d=C2_K1D, k2l=C2_K2L):
    """One 24 m cell: three 8 m segments, each opened by a space-charge location.
    QF at [0,1] m, QD at [12,13] m, thin SF/SD next to them."""
    return [
        elem(MARK), elem(QUAD, 1.0, k1=k1f), elem(DRIFT, 1.0), elem(SEXT, k2l=+k2l), elem(DRIFT, 6.0),
        elem(MARK), elem(DRIFT, 4.0), elem(QUAD, 1.0, k1=k1d), elem(DRIFT, 1.0), elem(SEXT, k2l=-k2l),
        elem(DRIFT, 2.0),
        elem(MARK), elem(DRIFT, 8.0),
    ]


def ring_c2(k1f=C2_K1F, k1d=C2_K1D, k2l=C2_K2L, n_cells=72):
    """72-cell ring (3-fold symmetric: 3 x 24 identical cells), 216 SC locations."""
    return table(ring_c2_cell(k1f, k1d, k2l) * n_cells)


# ---- workload presets ------------------------------------------------------
def grid_extent(sig_x, sig_y, n_sigma=5.0):
    return (-n_sigma * sig_x, n_sigma * sig_x, -n_sigma * sig_y, n_sigma * sig_y)


CONFIGS = {
    # 2e4 particles, 64x64, 24-cell FODO, 48 kicks/turn, 10 turns
    "c1": dict(n=20000, sig_x=2e-3, sig_y=2e-3, sig_px=2e-4, sig_py=2e-4, grid=64,
               lattice="c1", n_lambda=1e11 / 20.0, turns=10),
    # 1e6 particles, 128x128, 72-cell ring, 216 kicks/turn
    "c2": dict(n=1000000, sig_x=4e-3, sig_y=3e-3, sig_px=2e-4, sig_py=2e-4, grid=128,
               lattice="c2", n_lambda=1e11 / 20.0, turns=1000),
    # 4e6 particles, 256x256, same ring
    "c3": dict(n=4000000, sig_x=4e-3, sig_y=3e-3, sig_px=2e-4, sig_py=2e-4, grid=256,
               lattice="c2", n_lambda=1e11 / 20.0, turns=100),
    # 1e7 particles, Gaussian bunch (sigma_z = 15 m, cut at 4 sigma_z) in 32
    # slices of its own 128x128 grid over +-4 sigma_z; n_ppb protons per bunch
    # (scan 0.5e13 .. 2e13); sorted by sigma (the layout the sliced deposit prefers)
    "c5": dict(n=10000000, sig_x=4e-3, sig_y=3e-3, sig_px=2e-4, sig_py=2e-4, grid=128,
               lattice="c2", sig_z=15.0, n_slices=32, n_ppb=1.0e13, turns=500),
}


# c4: 8 x 8 working points (Qx, Qy) = (22.40, 20.75) + (dqx, dqy), dqx and dqy
# in 8 equal steps over [-0.1, 0.1] (row-major: dqx outer), as (k1F, k1D) of
# the c2 ring; matched on the bare one-turn trace by `python -m oracle.match_ring --scan`.
C4_WORKING_POINTS = [
    (0.14111251691365673, -0.13528782290733868),  # (22.3000, 20.6500)
    (0.1411244595147973, -0.1354025965324823),  # (22.3000, 20.6786)
    (0.14113638556241373, -0.1355172960540812),  # (22.3000, 20.7071)
    (0.14114829501187626, -0.13563192078266814),  # (22.3000, 20.7357)
    (0.14116018781875456, -0.1357464700292751),  # (22.3000, 20.7643)
    (0.14117206393881762, -0.13586094310543687),  # (22.3000, 20.7929)
    (0.14118392332803284, -0.13597533932319486),  # (22.3000, 20.8214)
    (0.14119576594256567, -0.13608965799510062),  # (22.3000, 20.8500)
    (0.1412246072383412, -0.13530145143623215),  # (22.3286, 20.6500)
    (0.14123650067254964, -0.13541617589794486),  # (22.3286, 20.6786)
    (0.1412483776302314, -0.13553082633304672),  # (22.3286, 20.7071)
    (0.14126023806689691, -0.1356454020522107),  # (22.3286, 20.7357)
    (0.14127208193825505, -0.13575990236660795),  # (22.3286, 20.7643)
    (0.1412839092002132, -0.1358743265879119),  # (22.3286, 20.7929)
    (0.14129571980887634, -0.13598867402830156),  # (22.3286, 20.8214)
    (0.1413075137205467, -0.1361029440004653),  # (22.3286, 20.8500)
    (0.1413365793575812, -0.13531505592871587),  # (22.3571, 20.6500)
    (0.14134842372146947, -0.1354297313236655),  # (22.3571, 20.6786)
    (0.14136025168560162, -0.1355443327687113),  # (22.3571, 20.7071)
    (0.1413720632056282, -0.13565885957466622),  # (22.3571, 20.7357)
    (0.14138385823739755, -0.13577331105284113),  # (22.3571, 20.7643)
    (0.1413956367369555, -0.13588768651504796),  # (22.3571, 20.7929)
    (0.1414073986605448, -0.13600198527360352),  # (22.3571, 20.8214)
    (0.14141914396460453, -0.13611620664133303),  # (22.3571, 20.8500)
    (0.14144843261138837, -0.13532863634556808),  # (22.3857, 20.6500)
    (0.14146022800164954, -0.13544326277050348),  # (22.3857, 20.6786)
    (0.1414720070686985, -0.1355578153220152),  # (22.3857, 20.7071)
    (0.14148376976832597, -0.13567229331105674),  # (22.3857, 20.7357)
    (0.14149551605651997, -0.13578669604907845),  # (22.3857, 20.7643)
    (0.141507245889465, -0.1359010228480311),  # (22.3857, 20.7929)
    (0.1415189592235416, -0.13601527302036948),  # (22.3857, 20.8214)
    (0.14153065601532586, -0.13612944587905576),  # (22.3857, 20.8500)
    (0.1415601663405168, -0.13534219264777203),  # (22.4143, 20.6500)
    (0.1415719128539242, -0.13545677019952196),  # (22.4143, 20.6786)
    (0.14158364312043706, -0.13557127395410212),  # (22.4143, 20.7071)
    (0.14159535709598642, -0.13568570322260667),  # (22.4143, 20.7357)
    (0.14160705473670002, -0.13580005731662576),  # (22.4143, 20.7643)
    (0.1416187359989011, -0.13591433554824886),  # (22.4143, 20.7929)
    (0.14163040083910816, -0.13602853723006872),  # (22.4143, 20.8214)
    (0.1416420492140344, -0.1361426616751851),  # (22.4143, 20.8500)
    (0.1416717798864663, -0.1353557247965145),  # (22.4429, 20.6500)
    (0.14168347761987302, -0.13547025357198722),  # (22.4429, 20.6786)
    (0.14169515918247674, -0.1355847086263183),  # (22.4429, 20.7071)
    (0.14170682453034938, -0.1356990892707426),  # (22.4429, 20.7357)
    (0.14171847361975815, -0.13581339481698998),  # (22.4429, 20.7643)
    (0.14173010640716543, -0.13592762457728902),  # (22.4429, 20.7929)
    (0.14174172284922773, -0.13604177786437063),  # (22.4429, 20.8214)
    (0.1417533229027955, -0.1361558539914719),  # (22.4429, 20.8500)
    (0.14178327259148568, -0.13536923275318566),  # (22.4714, 20.6500)
    (0.1417949216418237, -0.13548371284936822),  # (22.4714, 20.6786)
    (0.14180655459722488, -0.13559811930021182),  # (22.4714, 20.7071)
    (0.1418181714139017, -0.13571245141709198),  # (22.4714, 20.7357)
    (0.14182977204826155, -0.13582670851187859),  # (22.4714, 20.7643)
    (0.1418413564569056, -0.13594088989693928),  # (22.4714, 20.7929)
    (0.14185292459662857, -0.13605499488514347),  # (22.4714, 20.8214)
    (0.1418644764244185, -0.13616902278986537),  # (22.4714, 20.8500)
    (0.14189464379857594, -0.13538271647937763),  # (22.5000, 20.6500)
    (0.14190624426285564, -0.13549714799333532),  # (22.5000, 20.6786)
    (0.14191782870783945, -0.13561150593753157),  # (22.5000, 20.7071)
    (0.14192939708988075, -0.13572578962348272),  # (22.5000, 20.7357)
    (0.14194094936552676, -0.1358399983631987),  # (22.5000, 20.7643)
    (0.1419524854915179, -0.13595413146918653),  # (22.5000, 20.7929)
    (0.14196400542478743, -0.1360681882544539),  # (22.5000, 20.8214)
    (0.1419755091224605, -0.1361821680325128),  # (22.5000, 20.8500)
]


def lattice(name):
    return {"c1": fodo_c1, "c2": ring_c2}[name]()


def c4_grid_size(n):
    """Grid nodes per axis for a bunch of n macroparticles."""
    return 64 if n < 100000 else (128 if n < 500000 else 256)


def c4_bunches(seed=12345, n_bunches=64, n_min=1e4, n_max=2e6, scale=1.0):
    """Batching workload: n_bunches independent bunches, counts log-uniform in
    [n_min, n_max] (times `scale`), bunch b seeded with seed + b and tracked at
    working point b of C4_WORKING_POINTS (cyclic); each with the c2 distribution,
    line density and grid extent, and a grid of c4_grid_size(count) nodes.
    -> list of (particles, beam dict, grid, lattice table)."""
    rng = np.random.Generator(np.random.Philox(key=seed))
    counts = np.exp(rng.uniform(np.log(n_min), np.log(n_max), n_bunches))
    c = CONFIGS["c2"]
    out = []
    for b in range(n_bunches):
        n = max(1, int(round(counts[b] * scale)))
        parts = gaussian_bunch(n, seed + b, c["sig_x"], c["sig_y"], c["sig_px"], c["sig_py"])
        k1f, k1d = C4_WORKING_POINTS[b % len(C4_WORKING_POINTS)]
        lat = ring_c2(k1f=k1f, k1d=k1d)
        bm = beam(n_lambda=c["n_lambda"], circumference=float(lat["length"].sum()))
        g = c4_grid_size(int(round(counts[b])))
        out.append((parts, bm, (g, g) + grid_extent(c["sig_x"], c["sig_y"]), lat))
    return out


def sort_by_sigma(parts):
    order = np.argsort(parts["sigma"], kind="stable")
    return {k: np.ascontiguousarray(v[order]) for k, v in parts.items()}


def slices(name):
    """(n_slices, zmin, zmax) of a sliced workload."""
    c = CONFIGS[name]
    return c["n_slices"], -4.0 * c["sig_z"], 4.0 * c["sig_z"]


def workload(name, seed=12345, n=None):
    """(particles, beam dict, grid (nx, ny, xmin, xmax, ymin, ymax), lattice table).
    For sliced workloads n_lambda is n_ppb / dz (a slice holding the whole bunch)."""
    c = CONFIGS[name]
    n = c["n"] if n is None else n
    parts = gaussian_bunch(n, seed, c["sig_x"], c["sig_y"], c["sig_px"], c["sig_py"], sig_z=c.get("sig_z"))
    if "n_slices" in c:
        parts = sort_by_sigma(parts)
    lat = lattice(c["lattice"])
    circ = float(lat["length"].sum())
    if "n_slices" in c:
        nz, z0, z1 = slices(name)
        n_lambda = c["n_ppb"] / ((z1 - z0) / nz)
    else:
        n_lambda = c["n_lambda"]
    b = beam(n_lambda=n_lambda, circumference=circ)
    g = c["grid"]
    grid = (g, g) + grid_extent(c["sig_x"], c["sig_y"])
    return parts, b, grid, lat


# ---- plain-text description of a ring and its beam -------------------------
TYPE_NAMES = {DRIFT: "drift", QUAD: "quad", SEXT: "sext", BEND: "bend", RF: "rf", MARK: "mark",
              EXACT_BEND: "exact_bend"}
FIELDS = ("length", "k1", "k2l", "angle", "volt", "harmonic", "lag")


def config_to_json(b: dict, lattice) -> str:
    """A beam dict and an element table as JSON: {"beam": {...}, "lattice":
    [{"type": "quad", "length": 1.0, "k1": 0.14, ...}, ...]} (fields that are
    zero are left out; float64 values written with all their digits)."""
    import json
    elems = []
    for r in np.asarray(lattice, dtype=ELEMENT_DTYPE):
        e = {"type": TYPE_NAMES[int(r["type"])]}
        e.update({f: float(r[f]) for f in FIELDS if float(r[f]) != 0.0})
        elems.append(e)
    return json.dumps({"beam": {k: float(v) for k, v in b.items()}, "lattice": elems}, indent=1)


def config_from_json(text: str):
    """-> (beam dict, element table) from config_to_json's format."""
    import json
    d = json.loads(text)
    codes = {v: k for k, v in TYPE_NAMES.items()}
    rows = []
    for e in d["lattice"]:
        unknown = set(e) - set(FIELDS) - {"type"}
        if unknown or e.get("type") not in codes:
            raise ValueError(f"bad element {e}")
        rows.append(elem(codes[e["type"]], **{f: float(e[f]) for f in FIELDS if f in e}))
    return {k: float(v) for k, v in d["beam"].items()}, table(rows)
