/*
 * sc.h -- C-ABI of libsc, the GB300 (sm_103a) 2-D particle-in-cell
 * space-charge step for proton-ring tracking (arXiv:2010.11540).
 *
 * The calls follow the paper's PIC loop (Sec. I: assign charge to the grid,
 * solve Poisson's equation, move particles in the field) with the space-charge
 * kick of Sec. IV and the single-particle maps of Sec. III.
 *
 * Conventions
 *  - Every call returns sc_status: SC_OK (0) or a negative error code.  No
 *    C++ exception crosses this boundary.  sc_last_error() returns a text for
 *    the most recent failure of the calling thread.
 *  - Device pointers are plain CUDA device addresses on the current device.
 *    Particle arrays are owned by the caller; libsc never frees them.  Grids
 *    own their device buffers (charge, fields, Green's-function spectra,
 *    scratch, captured graphs) and release them in sc_destroy_grid().
 *  - All work on a grid is enqueued on the CUDA stream given to
 *    sc_create_grid() (NULL: a stream the grid creates, which orders with
 *    the legacy default stream; graph capture needs a non-legacy stream) and
 *    is asynchronous, except the calls documented as synchronous
 *    (sc_grid_read, sc_grid_write_charge, the *_host tracking calls,
 *    sc_track_turns when diag != NULL, and the first call that captures a
 *    turn, which times the candidate launch shapes).  Errors raised inside
 *    kernels surface at the next synchronous call of that grid:
 *    SC_ERR_TIMEOUT when a tensor-core solve gave up on a bounded wait (the
 *    grid then refuses further solves, sc_solve and sc_track_turns return
 *    SC_ERR_TIMEOUT; destroy it and create a new one), else SC_ERR_NAN for
 *    non-finite particle coordinates: sc_grid_read reports those sc_deposit
 *    met (x or y, or sigma on a sliced grid, NaN or infinite; such particles
 *    are outside the grid: no charge, no kick; the count is cleared by the
 *    call that reports it, whose outputs are still written), and tracking
 *    with diagnostics reports a turn whose moments are not finite (the fused
 *    deposits of a tracked turn do not test every particle: that costs the
 *    FP64-bound push a few percent).
 *  - Particle state is SoA float64: x [m], px = Px/p0, y [m], py = Py/p0,
 *    sigma = s - c beta0 t [m], psigma (Sec. III, Eq. H).
 */
#ifndef SC_H
#define SC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int sc_status;

#define SC_OK 0
#define SC_ERR_ARG (-1)         /* bad argument (null, size, geometry)        */
#define SC_ERR_CUDA (-2)        /* a CUDA runtime call failed                 */
#define SC_ERR_OOM (-3)         /* device allocation failed                   */
#define SC_ERR_OVERFLOW (-4)    /* more particles than the 64-bit charge grid can hold */
#define SC_ERR_TIMEOUT (-5)     /* a bounded device wait ran out              */
#define SC_ERR_NAN (-6)         /* deposits met particles whose position is not finite */
#define SC_ERR_UNSUPPORTED (-7) /* grid size / precision not supported        */

/* Poisson-solve arithmetic (sc_create_grid `precision`). */
#define SC_SOLVE_FP64 0   /* float64 FFT convolution (the plain form)           */
#define SC_SOLVE_TF32X3 1 /* DFT as tcgen05 GEMMs, 3-term split TF32, FP32 acc. */
/* Conducting rectangular pipe (Sec. IV-B, Dirichlet walls on the grid's outer
 * nodes), float64 sine transforms by FFT; nx - 1, ny - 1 powers of two in
 * 8..512.  The potential is kept (sc_grid_read_potential). */
#define SC_SOLVE_PIPE_FP64 2
/* The same conducting pipe with the sine transforms as dense GEMMs on the
 * tensor cores (3-term split TF32, FP32 accumulate; tiling tuned as for
 * SC_SOLVE_TF32X3), float32 fields; nx = ny in 10..258. */
#define SC_SOLVE_PIPE_TF32X3 3
/* The open-boundary solve of SC_SOLVE_TF32X3 with BF16 operands instead:
 * tcgen05 kind::f16 MMAs on bf16 hi/lo splits (8 significant bits each, ~16
 * together), FP32 accumulate, float32 fields; half the operand bytes of the
 * TF32 form, and fields about 1e-5 (relative L2) from the float64 solution
 * rather than 1e-7.  nx = ny in {64, 128, 256}. */
#define SC_SOLVE_BF16X3 4

/* Element types (sc_element.type). */
#define SC_DRIFT 0 /* exact drift, Sec. III-A                                  */
#define SC_QUAD 1  /* thick quadrupole with chromatic factor, Sec. III-B       */
#define SC_SEXT 2  /* sextupole, Sec. III-C: thin kick, or Eq. Sym2 if thick  */
#define SC_BEND 3  /* linear sector dipole from H_approx, Sec. III             */
#define SC_RF 4    /* thin RF cavity                                           */
#define SC_MARK 5  /* space-charge location (kick point), Sec. V               */
#define SC_EXACT_BEND 6 /* exact sector dipole (uniform field, Sec. III-A)  */

/* Largest macroparticle count per call: each particle deposits exactly 2^40
 * fixed-point units into an unsigned 64-bit grid, which holds fewer than 2^24
 * particles' worth even if all of them land in one cell (or one slice). */
#define SC_MAX_PARTICLES_PER_GRID ((1LL << 24) - 1)

typedef struct sc_grid sc_grid; /* opaque */

/* Caller-owned particle arrays (device pointers, n float64 each). */
typedef struct {
  double *x, *px, *y, *py, *sigma, *psigma;
  int64_t n;
} sc_particles;

/* Reference-particle and beam constants.
 * gamma0, beta0: reference Lorentz factors; n_lambda: line density [protons/m]
 * used by the transverse kick; r_p: classical proton radius [m];
 * circumference [m] and mass_ev (m c^2 [eV]) are used by SC_RF only. */
typedef struct {
  double gamma0, beta0, n_lambda, r_p, circumference, mass_ev;
} sc_beam;

/* One lattice element, 64 bytes.
 * length [m] (0 for thin elements); k1 [m^-2] (SC_QUAD; >0 focuses x);
 * k2l [m^-2] integrated sextupole strength (SC_SEXT: length 0 is one thin
 * kick, length > 0 the split exp(H0 aL) exp(V bL) exp(H0 cL) exp(V bL)
 * exp(H0 aL) of Eq. Sym2 with k2 = k2l/length); angle [rad] (SC_BEND: linear
 * map of H_approx; SC_EXACT_BEND: exact uniform-field sector dipole);
 * volt [V], harmonic, lag [rad] (SC_RF: dpsigma = volt/(beta0^2 E0) *
 * sin(lag - 2 pi harmonic sigma / circumference)). */
typedef struct {
  int32_t type;
  int32_t pad;
  double length, k1, k2l, angle, volt, harmonic, lag;
} sc_element;

/* Create a transverse grid of nx x ny nodes at x_i = xmin + i hx,
 * hx = (xmax - xmin)/(nx - 1) (same for y) -- the mesh of the charge
 * assignment of Sec. IV-A -- with the Poisson solver of Sec. IV in the given
 * precision: the open boundary (Hockney's zero-padded convolution, cited in
 * Sec. I) or, for the SC_SOLVE_PIPE_* forms, the conducting rectangular pipe
 * of Sec. IV-B.  Builds the Green's-function spectra (or sine-transform
 * matrices) on the device (synchronous on `stream`); the grid owns them and
 * every other device buffer it uses (released by sc_destroy_grid).
 * nx, ny: powers of two in 8..512 for SC_SOLVE_FP64; nx = ny in {64, 128, 256}
 * for SC_SOLVE_TF32X3 and SC_SOLVE_BF16X3; nx - 1, ny - 1 powers of two in 8..512 for
 * SC_SOLVE_PIPE_FP64; nx = ny in 10..258 for SC_SOLVE_PIPE_TF32X3.  Errors: SC_ERR_ARG, SC_ERR_UNSUPPORTED,
 * SC_ERR_OOM, SC_ERR_CUDA.  *out is set only on success. */
sc_status sc_create_grid(sc_grid **out, int nx, int ny, double xmin, double xmax, double ymin,
                         double ymax, int precision, void *stream);

/* Longitudinally sliced grid (2.5-D): the line density lambda(z) of Sec. IV
 * as a histogram of sigma with n_slices bins over [zmin, zmax), each bin with
 * its own nx x ny transverse grid of the given extent.  A particle belongs to
 * slice k = floor((sigma - zmin) * (1 / dz)), dz = (zmax - zmin) / n_slices; particles outside
 * [zmin, zmax) are outside the grid.  Every call then works on all slices:
 * deposits fill each particle's slice, one solve call solves every slice
 * (batched launches), the kick gathers from the particle's slice.  Each
 * slice's charge is normalised by the total particle count N, so sc_beam's
 * n_lambda is the line density of a slice holding the whole bunch (N_ppb / dz).
 * Deposits are fastest with particles sorted by sigma.  Charge and field
 * arrays of sc_grid_read / sc_grid_write_charge then hold n_slices grids,
 * slice-major.  1 <= n_slices <= 1024 and nx*ny*n_slices <= 2^28, else
 * SC_ERR_ARG; other arguments and errors as sc_create_grid. */
sc_status sc_create_grid_sliced(sc_grid **out, int nx, int ny, double xmin, double xmax, double ymin,
                                double ymax, int n_slices, double zmin, double zmax, int precision,
                                void *stream);

/* Release a grid and everything it owns (synchronises its stream). NULL ok. */
sc_status sc_destroy_grid(sc_grid *g);

/* CIC charge deposition, Sec. IV-A: zero the grid's uint64 charge Q, then add
 * each particle's four fixed-point weights (2^-20 per axis, 2^40 per
 * particle).  Particles outside [xmin, xmax) x [ymin, ymax) (and non-finite
 * ones) deposit nothing and are counted (sc_grid_read's n_out).
 * Errors: SC_ERR_ARG, SC_ERR_OVERFLOW (n > SC_MAX_PARTICLES_PER_GRID). */
sc_status sc_deposit(sc_grid *g, const sc_particles *p);

/* Reorder a bunch by its cell on grid g (an option; the paper has no
 * counterpart): the six arrays of p are permuted in place, all by the same
 * permutation -- particles sorted by cell index (slice, then row j, then
 * column i), those outside the grid last, equal cells in their old order
 * (stable) -- and, when perm != NULL (device, caller-owned, p->n int32), perm[k]
 * receives the old index of the particle now at k.  Physics results do not
 * depend on the order (particles are independent and the charge is an
 * integer sum).  sc_deposit on this grid of the bunch it last ordered (same
 * x array and count) runs faster: each warp combines the weights of
 * neighbouring particles in the same cell before its atomic adds, which only
 * pays on an ordered bunch.  Per-particle arrays the caller keeps elsewhere (e.g. tune
 * accumulators) are not permuted; sc_track_turns rebuilds its own at every
 * call.  The grid keeps a scratch buffer for the sort (20 bytes per particle
 * plus the radix sort's storage, grown on demand: the call then synchronises
 * and allocates); asynchronous on the grid's stream otherwise.
 * Errors: SC_ERR_ARG, SC_ERR_OVERFLOW, SC_ERR_OOM, SC_ERR_CUDA. */
sc_status sc_sort_particles(sc_grid *g, const sc_particles *p, int32_t *perm);

/* Open-boundary Poisson solve (Sec. IV, Eq. poisson3D, free-space part):
 * phi = G * q with G = -ln r, q = Q 2^-40 / N (N = particle count of the last
 * deposit), and node fields E = -grad phi by centred differences; stored as
 * interleaved (Ex, Ey) float64 per node, in units of 1/m per unit line charge. */
sc_status sc_solve(sc_grid *g);

/* Fused space-charge step for one location (Sec. IV kick, Sec. III maps):
 * for every particle, gather E of grid g bilinearly at (x, y), kick
 * px += K L_sc Ex, py += K L_sc Ey with K = 2 r_p n_lambda / (beta0^2 gamma0^3)
 * (no kick when L_sc == 0 or the particle is outside g), push through
 * elems[0..n_elems) (host array, copied at the call), and, when next != NULL,
 * deposit the new positions into `next` as sc_deposit does (next may be g).
 * Errors: SC_ERR_ARG, SC_ERR_OVERFLOW. */
sc_status sc_kick_push(sc_grid *g, const sc_particles *p, const sc_beam *b, double L_sc,
                       const sc_element *elems, int n_elems, sc_grid *next);

/* The PIC loop of Sec. I over whole turns (Sec. V: space-charge kicks at
 * chosen locations of the ring, each with the path length since the previous
 * one).  Track n_turns turns of the ring `lattice` (host array of n_elems elements;
 * SC_MARK entries are the space-charge locations, the kick length being the
 * path length since the previous marker, cyclically).  Each marker runs
 * deposit -> solve -> kick, then the elements up to the next marker are
 * pushed; elements before the first marker are pushed without a kick.  One
 * turn is captured once as a CUDA graph and replayed (re-captured when any
 * argument changes).  The grid keeps per-particle working arrays for the run
 * (cell/fraction cache of the last deposit, psigma-dependent quantities, and
 * the 2x2 matrix entries of each distinct thick quadrupole, up to 8, as long
 * as psigma is unchanged; 60 + 48 per quadrupole bytes per particle),
 * recomputed at the start of every call.  When diag != NULL
 * (host, n_turns x 14 doubles) the beam moments at the start of every turn
 * are written there: means of (x, px, y, py, sigma, psigma), then central
 * <xx>, <x px>, <px px>, <yy>, <y py>, <py py>, <sigma sigma>,
 * <psigma psigma>; the call is then synchronous.
 * Errors: SC_ERR_ARG, SC_ERR_OVERFLOW, SC_ERR_CUDA. */
sc_status sc_track_turns(sc_grid *g, const sc_particles *p, const sc_beam *b,
                         const sc_element *lattice, int n_elems, int n_turns, double *diag);

/* sc_track_turns on a bunch held in HOST memory: host->x .. host->psigma are
 * host arrays of host->n doubles (page-locked memory copies fastest), read at
 * the call and overwritten with the tracked state before it returns.  The
 * grid owns device copies (grown on demand, reused across calls, so the
 * captured turn is reused too); the copies run on the grid's stream around
 * the turns and the call is synchronous.  Errors: as sc_track_turns, and
 * SC_ERR_OOM when the device copies cannot be allocated. */
sc_status sc_track_turns_host(sc_grid *g, const sc_particles *host, const sc_beam *b,
                              const sc_element *lattice, int n_elems, int n_turns, double *diag);

/* Synchronous copy-out of a grid's state into host arrays (each may be NULL):
 * Q (n_slices*ny*nx uint64, row-major [k][j][i]), Ex and Ey (same layout,
 * float64), and n_out = particles found outside the grid by deposits since
 * the grid was created.  Errors: SC_ERR_ARG; after the copies, SC_ERR_TIMEOUT
 * or SC_ERR_NAN as described under Conventions. */
sc_status sc_grid_read(sc_grid *g, uint64_t *Q, double *Ex, double *Ey, int64_t *n_out);

/* Synchronous upload of a charge grid Q (host, n_slices*ny*nx uint64) and the
 * particle count N used to normalise it, e.g. to solve a given charge. */
sc_status sc_grid_write_charge(sc_grid *g, const uint64_t *Q, int64_t n_particles);

/* Device view of the charge grid, for a reduction across ranks of a bunch
 * whose particles are sharded (the Sec. IV-A charge is a sum over particles):
 * *Q receives the device pointer of the grid's uint64 charge ([nstack][ny][nx],
 * owned by the grid, valid until sc_destroy_grid) and *cells its element
 * count.  Each rank deposits its share with sc_deposit (or a fused
 * sc_kick_push deposit), the ranks sum their grids in place on the grid's
 * stream (an integer sum all-reduce; uint64 sums wrap modulo 2^64, so an int64
 * reduction gives the same bits), sc_set_particle_count gives the bunch's
 * total count, and sc_solve then yields on every rank the fields of the whole
 * bunch, bit for bit those of one GPU.  Errors: SC_ERR_ARG. */
sc_status sc_grid_charge_device(sc_grid *g, uint64_t **Q, int64_t *cells);

/* The sharded bunch inside sc_track_turns (no counterpart in the paper; the
 * charge of Sec. IV-A is a sum over particles, so ranks holding parts of one
 * bunch add their grids).  fn is a caller function that enqueues, on the CUDA
 * stream it is given, an in-place sum of `cells` uint64 charge values at the
 * device pointer `charge` over every rank of the bunch (e.g. an NCCL uint64
 * sum all-reduce; uint64 sums wrap modulo 2^64, so an int64 reduction gives
 * the same bits) and returns 0 (non-zero: the capture fails with
 * SC_ERR_CUDA).  sc_track_turns calls it while it captures a turn, once per
 * space-charge location, between that location's deposit and its solve, so
 * the reduction is part of the replayed turn graph; every rank must track the
 * same lattice for the same turns.  The solve then normalises by
 * total_particles (the whole bunch) instead of the local count; fields and
 * kicks on every rank equal those of the whole bunch on one GPU, bit for bit.
 * Per-turn moments and tunes stay per rank (local particles).  The launch-
 * shape trials of a first capture do not call fn.  fn == NULL switches the
 * reduction off.  Synchronises the grid's stream; the next sc_track_turns
 * re-captures.  Errors: SC_ERR_ARG (NULL grid; fn with total_particles < 1). */
typedef int (*sc_charge_reduce_fn)(uint64_t *charge, int64_t cells, void *stream, void *user);
sc_status sc_set_charge_reduce(sc_grid *g, sc_charge_reduce_fn fn, void *user, int64_t total_particles);

/* The particle count N that normalises the next sc_solve (q = Q 2^-40 / N);
 * every deposit sets it to the count it deposited.  Errors: SC_ERR_ARG (NULL
 * grid, negative count). */
sc_status sc_set_particle_count(sc_grid *g, int64_t n_particles);

/* Longitudinal space-charge kick, Sec. IV (dps = -(e/(m gamma0^2 beta0^2
 * c^2)) u dlambda/dz L), on a sliced pipe grid (SC_SOLVE_PIPE_FP64, or
 * SC_SOLVE_PIPE_TF32X3 with the float32 potential): every kick on
 * this grid then also applies dps = -(K gamma0) L (Phi_{k+1} - Phi_{k-1}) /
 * (2 dz) at the particle's (x, y), Phi_k the potential of slice k (0 beyond
 * the first and last slice), K the transverse kick strength.  For a bunch
 * whose transverse shape is the same in every slice this is the paper's
 * u dlambda/dz.  Errors: SC_ERR_UNSUPPORTED (not a sliced pipe grid). */
sc_status sc_set_longitudinal_kick(sc_grid *g, int enable);

/* Field gather of the kick (sc_set_gather).  BILINEAR: the node fields
 * interpolated with the CIC weights (Sec. IV-A).  BEZIER: E = -grad of the
 * Bezier surface of the potential over the 4 x 4 nodes i-1..i+2, j-1..j+2
 * (Sec. IV-C), the cubic's parameter running over those nodes,
 * t = (x - x_{i-1}) / (3 hx); nodes beyond the walls take the odd extension;
 * on a sliced grid with the longitudinal kick the neighbouring slices'
 * potentials come from the same surfaces.  BEZIER needs a pipe grid
 * (SC_SOLVE_PIPE_FP64; SC_SOLVE_PIPE_TF32X3 evaluates the surface of its
 * float32 potential in float32), SC_ERR_UNSUPPORTED otherwise. */
#define SC_GATHER_BILINEAR 0
#define SC_GATHER_BEZIER 1
sc_status sc_set_gather(sc_grid *g, int mode);

/* Synchronous copy-out of a pipe grid's potential (n_slices*ny*nx float64,
 * row-major, 0 on the walls): normalised like the fields (per unit line
 * charge, -ln r normalisation), i.e. phi solves lap phi = -2 pi q / (hx hy).
 * Errors: SC_ERR_ARG (NULL), SC_ERR_UNSUPPORTED (not a pipe grid),
 * SC_ERR_CUDA. */
sc_status sc_grid_read_potential(sc_grid *g, double *phi);

/* Per-particle tunes, Sec. V (the betatron tune of a particle is its one-turn
 * phase advance).  Arms grid g: every turn sc_track_turns then runs ends with
 * the phase advance of each particle of p in the normalised coordinates of the
 * bare Twiss functions at the turn start, twiss = {beta_x, alpha_x, beta_y,
 * alpha_y} (host array), accumulated in acc (device, caller-owned, 4 n
 * doubles: phases x, phases y, summed advances x, summed advances y, each
 * advance taken mod 2 pi).  This call records the initial phases and zeroes the
 * sums (asynchronous, on the grid's stream).  After T tracked turns, the
 * fractional tunes are sums / (2 pi T).  acc == NULL disarms.
 * Errors: SC_ERR_ARG. */
sc_status sc_tune_setup(sc_grid *g, const sc_particles *p, const double *twiss, double *acc);

/* Per-phase tracing.  When enabled, the next turn sc_track_turns captures
 * records CUDA events around every solve and every kick/push launch (on the
 * grid's stream); sc_track_turns then waits after each turn and accumulates
 * the elapsed times (this serialises the kernels of a turn: a profiling mode,
 * not the fast path).  Enabling or disabling re-captures the turn. */
sc_status sc_trace_enable(sc_grid *g, int enable);

/* Totals accumulated since the last read (then reset): kick/push launch time
 * and solve time in ms, and the number of kicks they cover. */
sc_status sc_trace_read(sc_grid *g, double *kick_push_ms, double *solve_ms, int64_t *n_kicks);

/* Tiling of the split-TF32 solve (SC_SOLVE_TF32X3).  Each of its four GEMM
 * phases (row DFT, column DFT, inverse column DFT, inverse row DFT) has a few
 * kernel variants (tile width, split-K cluster size, pipeline depth); the
 * fastest for the grid (and its stacked slices) is chosen by timing them all
 * when the first grid of its geometry (size, stack depth, operand type) is
 * created on a device; later grids of that geometry in the process take the
 * same choice, so they give the same bits.  sc_get_solver_tiling reads the four variant
 * indices and, if desc != NULL, describes them in desc (n bytes, always
 * NUL-terminated); sc_set_solver_tiling forces them (an entry of -1 keeps
 * that phase's variant), e.g. to compare grids bit for bit.  Variants differ
 * only in the summation order of the FP32 accumulation.  Errors:
 * SC_ERR_UNSUPPORTED (not a split-TF32 grid), SC_ERR_ARG (index out of range
 * or a variant that does not fit the grid). */
sc_status sc_get_solver_tiling(sc_grid *g, int *choice, char *desc, size_t n);
sc_status sc_set_solver_tiling(sc_grid *g, const int *choice);

/* Launch shape of sc_track_turns' fused kick/push (Sec. IV-A, IV-B): block
 * size (threads, a multiple of 32 up to 768) and particle traversal (0: all blocks sweep a common window,
 * grid stride; 1: each block takes one contiguous chunk; sliced grids always
 * use chunks).  Every shape gives bit-identical results.  Left free (threads
 * 0, traversal -1: the default), the shape is chosen when a turn is captured
 * for a bunch of 2^18 particles or more: each candidate runs the turn's first
 * 16 space-charge steps (solve, then kick/push with its deposit), captured as
 * a graph, on a scratch copy of the bunch, and the fastest is kept (the
 * particles, the charge grid and the out-of-grid counter are left as they
 * were); smaller bunches take the largest block and the field type's default
 * traversal.  A re-capture for the same particles, beam, lattice and options
 * (tracing or diagnostics switched) reuses the choice.
 * sc_set_kick_push_shape fixes either part (the next sc_track_turns
 * re-captures); sc_get_kick_push_shape reads the shape of the captured turn
 * and, in trial_us, the timed trial of the chosen shape (0 when not timed).
 * Errors: SC_ERR_ARG (NULL grid, a value out of range, or no captured turn). */
sc_status sc_set_kick_push_shape(sc_grid *g, int threads, int traversal);
sc_status sc_get_kick_push_shape(sc_grid *g, int *threads, int *traversal, double *trial_us);

/* Work of one sc_solve on this grid (all stacked grids), for rooflines:
 * tensor_flops = the split-TF32 DFT GEMMs' 2 M N K per phase times the three
 * split products (0 for the float64 forms); fft_flops = the FFT-equivalent
 * count 2 x 5 N log2 N of a forward and an inverse complex 2-D transform of
 * N points (the zero-padded 2nx x 2ny grid, or the pipe's odd extension
 * 2(nx-1) x 2(ny-1)) per stacked grid.  Errors: SC_ERR_ARG (NULL grid). */
sc_status sc_get_solver_work(sc_grid *g, double *tensor_flops, double *fft_flops);

/* Failure-detection test hook (no counterpart in the paper).  The tensor-core
 * solve's waits on its copy and MMA barriers are bounded (~2 s of SM clock);
 * when one runs out the kernel records an error word, lets its issued work
 * drain, frees its tensor memory and returns, and sc_grid_read reports
 * SC_ERR_TIMEOUT (the word stays set for this grid).  While enabled, the
 * split-TF32 solve announces its data-operand copies to the pipeline barriers
 * without issuing them, so those waits run out (≈ 2 s per phase); no copy,
 * MMA or memory access is left in flight and the context stays usable.
 * Errors: SC_ERR_UNSUPPORTED (no split-TF32 solve). */
sc_status sc_test_bounded_waits(sc_grid *g, int enable);

/* ---- Batches of independent bunches --------------------------------------
 * Many bunches (working points of a tune scan, bunches of a train, intensity
 * scans), each with its own particles, beam, lattice and transverse grid,
 * tracked together: per space-charge location one batched solve per grid
 * class (bunches whose grids have the same nodes and extent share the solver
 * constants and are solved by one set of launches, one stacked grid each) and
 * ONE kick/push/deposit launch for all bunches, whose blocks are split over
 * the bunches in proportion to their particle counts.  A whole turn of all
 * bunches is captured as one CUDA graph.  The physics per bunch is exactly
 * sc_track_turns on a grid of that bunch's own: each bunch's charge is
 * normalised by its own particle count and kicked with its own N_lambda. */
typedef struct {
  int nx, ny; /* as sc_create_grid */
  double xmin, xmax, ymin, ymax;
} sc_grid_spec;

typedef struct {
  sc_particles particles;     /* caller-owned device arrays of this bunch */
  sc_beam beam;
  const sc_element *lattice;  /* host array, as sc_track_turns */
  int n_elems;
} sc_bunch;

typedef struct sc_batch sc_batch; /* opaque */

/* Create a batch of n_bunches grids (grids[b] is bunch b's) with the solver
 * of the given precision on `stream` (NULL: a stream of its own).  Grids must
 * meet sc_create_grid's rules; 1 <= n_bunches <= 4096.  Errors as
 * sc_create_grid.  *out is set only on success. */
sc_status sc_create_batch(sc_batch **out, const sc_grid_spec *grids, int n_bunches, int precision,
                          void *stream);

/* Release a batch (synchronises its stream).  NULL ok. */
sc_status sc_destroy_batch(sc_batch *B);

/* Track bunches[0 .. n_bunches-1] (the batch's count) n_turns turns, as
 * sc_track_turns does for each bunch alone.  Every lattice must hold the same
 * number of SC_MARK elements and either all or none start with one; the
 * elements between markers may differ (different working points).  The
 * captured turn is kept while the bunches (pointers, counts, beams, lattices)
 * stay the same.  diag: NULL, or host [n_turns][n_bunches][14] receiving each
 * bunch's moments at the start of every turn (layout of sc_track_turns).
 * Errors: SC_ERR_ARG (NULL, mismatched markers), SC_ERR_OVERFLOW (a bunch over
 * SC_MAX_PARTICLES_PER_GRID), SC_ERR_CUDA, SC_ERR_OOM. */
sc_status sc_batch_track_turns(sc_batch *B, const sc_bunch *bunches, int n_turns, double *diag);

/* sc_batch_track_turns on bunches held in HOST memory (each bunch's
 * particles.x .. psigma host arrays, read at the call and overwritten with
 * the tracked state), with device copies owned by the batch as in
 * sc_track_turns_host.  Synchronous.  Errors: as sc_batch_track_turns, and
 * SC_ERR_OOM. */
sc_status sc_batch_track_turns_host(sc_batch *B, const sc_bunch *bunches, int n_turns, double *diag);

/* Synchronous copy-out of bunch b's grid state, as sc_grid_read. */
sc_status sc_batch_read(sc_batch *B, int b, uint64_t *Q, double *Ex, double *Ey, int64_t *n_out);

/* Tracing of batched turns, as sc_trace_enable / sc_trace_read (kick/push
 * time is the batched launch covering every bunch; solve time covers every
 * grid class). */
sc_status sc_batch_trace_enable(sc_batch *B, int enable);
/* Launch shape of the batched kick/push: block size (a multiple of 32 up to
 * 768 for split-TF32 batches, 640 for float64 fields) and the number of waves
 * of resident blocks each launch's bunch chunks are cut into (more waves
 * balance bunches of uneven size, fewer flush fewer deposit tiles).  Every
 * shape gives bit-identical results.  Left free (0), the shape is chosen when
 * a turn is captured for batches of 2^18 particles or more, by timing the
 * candidates (512 or the largest block; 1, 2, 4 or 8 waves) over the turn's
 * first 16 space-charge steps on scratch copies of the bunches (the bunches,
 * charge grids and out-of-grid counters are left as they were); else 4 waves
 * of the largest block.  sc_batch_set_kick_push_shape fixes either part (the
 * next turn re-captures); sc_batch_get_kick_push_shape reads the captured
 * turn's shape and the timed trial (0 when not timed).  Errors: SC_ERR_ARG
 * (NULL batch, value out of range, or no captured turn). */
sc_status sc_batch_set_kick_push_shape(sc_batch *B, int threads, int waves);
sc_status sc_batch_get_kick_push_shape(sc_batch *B, int *threads, int *waves, double *trial_us);

/* sc_get_solver_tiling of bunch b's grid class; sc_set_solver_tiling for
 * every grid class of the batch (split-TF32 batches). */
sc_status sc_batch_get_solver_tiling(sc_batch *B, int b, int *choice, char *desc, size_t n);
sc_status sc_batch_set_solver_tiling(sc_batch *B, const int *choice);
sc_status sc_batch_trace_read(sc_batch *B, double *kick_push_ms, double *solve_ms, int64_t *n_kicks);

/* Per-particle tunes of Sec. V (the mean one-turn phase advance): the
 * fractional tunes from a tune accumulator (sc_tune_setup) after n_turns
 * tracked turns: q (device, caller-owned, 2 n doubles) receives acc's summed
 * advances / (2 pi n_turns), x for particles 0..n-1, then y.  Asynchronous on
 * `stream` (NULL: the legacy default stream); acc and q are device pointers.
 * Errors: SC_ERR_ARG (NULL pointer, n < 0, n_turns < 1), SC_ERR_CUDA. */
sc_status sc_tunes(const double *acc, int64_t n, int n_turns, double *q, void *stream);

/* Largest particle count sc_moments_noalloc accepts (its partial sums are
 * reduced in float64 by a fixed 304-block grid; counts are bounded like a
 * grid's). */
#define SC_MOMENTS_NOALLOC_MAX_N SC_MAX_PARTICLES_PER_GRID

/* Beam moments that allocate nothing: the paper has no counterpart; this
 * entry point exists for callers that cannot allocate device memory while
 * they run (an arena that owns the whole device, an allocator that must not be
 * re-entered, a real-time loop where cudaMalloc/cudaFree may synchronise).
 * Writes 14 doubles to the device pointer `out` on `stream` (asynchronous):
 * means of (x, px, y, py, sigma, psigma), then the central moments <xx>,
 * <x px>, <px px>, <yy>, <y py>, <py py>, <sigma sigma>, <psigma psigma>
 * (two passes: the means, then the moments of the offsets from them) — the
 * same numbers as sc_track_turns' per-turn diagnostics.  Scratch: a
 * file-scope device array of 304 x 14 doubles (34 KB), held by every GPU that
 * loads the library until the process exits.  The first call on a device
 * looks up that array's address (make it before any stream capture), and so
 * does the first call after the device's context was reset (cudaDeviceReset);
 * calls that overlap on the GPU share the array and race.  Calls no
 * cudaMalloc, cudaFree or other allocating routine.
 * Errors: SC_ERR_ARG (NULL, n <= 0), SC_ERR_OVERFLOW (n > SC_MOMENTS_NOALLOC_MAX_N),
 * SC_ERR_CUDA. */
sc_status sc_moments_noalloc(const sc_particles *p, double *out, void *stream);

/* Checkpoint and resume of a tracked bunch (host memory; the paper has no
 * counterpart, but its runs reach ~5e5 turns).  sc_checkpoint_write stores
 * the bunch's six HOST arrays (host->x .. host->psigma, host->n > 0 doubles
 * each, e.g. after sc_track_turns_host or a copy from the device) bit for bit
 * together with the caller's turn counter, the beam constants and a 64-bit
 * hash of the lattice (element count and records) in the file `path`,
 * replacing it in one step (written to path".tmp", then renamed), with a
 * checksum of the contents.  sc_checkpoint_read checks the file (format,
 * particle count = host->n, the same beam constants bit for bit, the same
 * lattice, the checksum) before it fills the host arrays and *turn (turn may
 * be NULL); on any mismatch it returns SC_ERR_ARG and leaves the arrays
 * untouched.  Tracking is deterministic, so resuming from a checkpoint gives
 * the bits of the uninterrupted run.  Synchronous host I/O, no GPU work.
 * Errors: SC_ERR_ARG (NULL or empty bunch, bad element list, I/O failure,
 * mismatch or damage, with the reason in sc_last_error). */
sc_status sc_checkpoint_write(const char *path, const sc_particles *host, int64_t turn, const sc_beam *b,
                              const sc_element *lattice, int n_elems);
sc_status sc_checkpoint_read(const char *path, const sc_particles *host, int64_t *turn, const sc_beam *b,
                             const sc_element *lattice, int n_elems);

/* Text of the last error on the calling thread (always NUL-terminated). */
sc_status sc_last_error(char *buf, size_t n);

#ifdef __cplusplus
}
#endif

#endif /* SC_H */
