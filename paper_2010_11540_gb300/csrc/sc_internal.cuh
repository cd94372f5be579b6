// Internal declarations shared by the libsc translation units (CUDA path only).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <utility>
#include <vector>

#include "sc.h"

namespace sc {

// Solve forms whose fields are float32 (tensor-core split-precision GEMMs).
inline bool split_solve(int precision) {
  return precision == SC_SOLVE_TF32X3 || precision == SC_SOLVE_PIPE_TF32X3 || precision == SC_SOLVE_BF16X3;
}

// ---------------------------------------------------------------------------
// Error reporting (thread-local last error, status codes of sc.h)
// ---------------------------------------------------------------------------
sc_status set_error(sc_status code, const std::string& msg);
sc_status cuda_error(cudaError_t e, const char* what);

#define SC_CUDA(call)                                    \
  do {                                                   \
    cudaError_t _e = (call);                             \
    if (_e != cudaSuccess) return sc::cuda_error(_e, #call); \
  } while (0)

// ---------------------------------------------------------------------------
// Programmatic dependent launch: kernels of a turn are launched so that the
// next one may start its prologue while the previous one finishes; each kernel
// calls pdl_wait() before touching anything the previous kernels wrote, and
// pdl_allow() once its dependents may be scheduled.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_allow() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// ---------------------------------------------------------------------------
// Grid geometry as the kernels see it.  Nodes x_i = xmin + i*hx.
// ---------------------------------------------------------------------------
struct GridGeom {
  int nx, ny;
  double xmin, ymin, inv_hx, inv_hy;
  double xlast, ylast;  // (double)(nx-1), (double)(ny-1): exclusive upper bounds of xi, eta
  // longitudinal slices (nz == 1: none): slice k = floor((sigma - zmin) * inv_dz), 0 <= k < nz;
  // cell indices then carry the slice offset k * nx * ny
  int nz;
  double zmin, inv_dz;
  // deposit tile window: nodes [wx0, wx0 + wnx) x [wy0, wy0 + wny) of one
  // slice, held in a block's shared memory (the whole slice when it fits in
  // kTileBytes, else the centred window that does)
  int wx0, wy0, wnx, wny;
};

// Shared memory of a block's deposit tile (uint64 per node of its window).
constexpr int kTileBytes = 200 * 1024;

// Element compiled for the kernels: the user's sc_element plus per-element
// constants precomputed on the host in float64 (see compile_elements).
struct DevElem {
  int type;
  int flags;
  double p[9];
};

// Segments up to this many elements travel inside the launch parameters.
constexpr int KP_INLINE = 12;

// Kick/push/deposit launch parameters, passed by value (constant bank).
struct KPParams {
  double *x, *px, *y, *py, *sg, *ps;
  int64_t n;
  // gather + kick
  GridGeom gk;
  const double2* E;  // (Ex, Ey) per node of the kick grid
  double kl;         // K * L_sc
  int do_kick;
  // Cell cache: the deposit of the previous step located every particle on
  // the same grid at the same position; the gather reuses it.  cell = j*nx+i
  // or -1 (outside), frac = (fx, fy).  NULL: locate again.
  int* cell;
  double2* frac;   // float64 fractions (float64 fields)
  int2* fix;       // fixed-point fractions (ax, ay) of the deposit (float32 fields)
  // float32 fields: E32 holds (Ex, Ey) as float2 and the gather runs in float32
  int field32;
  const float2* E32;
  // deposit
  int do_deposit;
  GridGeom gd;
  unsigned long long* Q;      // uint64 charge of the deposit grid
  unsigned long long* n_out;  // running count of particles outside the deposit grid
  unsigned long long* n_nan;  // running count of those with a non-finite x, y (or sigma on sliced grids)
  // beam constants
  double beta0_sq, inv_gamma0_sq;
  const DevElem* el;  // device array of the segment's compiled elements, or NULL: use inl
  int n_elem;
  int has_quad;       // the segment holds an SC_QUAD
  int has_xe;         // the segment holds a thick SC_SEXT or an SC_EXACT_BEND
  // Per-particle ps-dependent quantities, 5 arrays of n: (1+delta)^2,
  // 1 + beta0^2 ps, sqrt(1-ps), 1/sqrt(1-ps), 1/(4(1-ps)).  psc_mode 0: none
  // (computed in registers), 1: read (rewritten after an RF cavity), 2: compute and write.
  double* psc;
  int psc_mode;
  // Per-particle coefficients of the lattice's quadrupole families (they
  // depend on ps alone), qfam_n x 6 arrays of n: written with psc (psc_mode 2,
  // and after an RF cavity), read by the quadrupoles tagged with a family while
  // ps is unchanged.  NULL: every quadrupole computes its own.
  double* qcache;
  const DevElem* qfam;  // the families' compiled elements (device)
  int qfam_n;
  // psc arrays the segment does not read (psc_mode 1): bit 0 sqrt(1-ps) and
  // 1/sqrt(1-ps) (only quadrupoles computing their own matrix entries use
  // them), bit 1 1/(4(1-ps)) (only thick quadrupoles)
  int psc_skip;
  // psigma traffic of the segment (psc_mode 1): bit 0 psigma is not changed
  // (no RF cavity, no longitudinal kick: not stored), bit 1 not read either
  // (drifts and thin sextupoles only: not loaded)
  int ps_mode;
  // Longitudinal kick (sliced pipe grids, float64 form): psigma -= klz *
  // (Phi_{k+1} - Phi_{k-1}) at the particle, phi the slices' node potentials
  // of the kick grid, klz = K gamma0 L / (2 dz).
  int lon;
  const double* phi;
  const float* phi32;  // the split form's float32 potential (lon / Bezier with float32 fields)
  double klz;
  // Bezier gather (pipe grids, float64 form): E = -grad of the Bezier surface
  // of phi (Sec. IV-C) instead of bilinear node fields; with lon the
  // neighbouring slices' potentials come from the same surfaces.
  int bezier;
  // particle traversal of the blocks: -1 default, 0 grid stride, 1 contiguous chunks
  int traversal;
  DevElem inl[KP_INLINE];
};

// Host: compile n user elements into out (float64 constants per element).
void compile_elements(const sc_element* in, int n, const sc_beam* b, DevElem* out);
// Host: the distinct (thick, non-zero) quadrupoles of compiled elements, up to
// max, copied into fam; returns their count.
constexpr int KP_QFAM_MAX = 8;
int quad_families(const DevElem* el, int n, DevElem* fam, int max);
// Host: tag each quadrupole of el equal to a family with its index.
void tag_quad_families(DevElem* el, int n, const DevElem* fam, int nf);
// Host: KPParams::psc_skip for a segment of n user elements whose
// quadrupoles are tagged against the nf families fam.
int psc_skip_mask(const sc_element* host, int n, const sc_beam* b, const DevElem* fam, int nf);
// Host: KPParams::ps_mode for a segment of n user elements (lon: the launch's longitudinal kick).
int ps_mode_mask(const sc_element* host, int n, bool lon);

// Solve scratch and spectra for the float64 FFT form.
struct Fft64Plan {
  int M;                 // 2 * n (padded length), per axis: Mx, My
  double2* twx;          // Mx/2 twiddles exp(-2 pi i t / Mx)
  double2* twy;          // My/2 twiddles
  double2* F1;           // row transforms  [ny][nx+1]
  double2* Hx;           // column results for Ex [ny][nx+1]
  double2* Hy;           // column results for Ey [ny][nx+1]
  double* Sx;            // imaginary part of the Ex kernel spectrum [My][nx+1]
  double* Sy;            // imaginary part of the Ey kernel spectrum [My][nx+1]
};

// Solve scratch for the conducting-pipe form (solve_pipe64.cu).
struct PipePlan {
  double2* twx;      // (nx-1) twiddles exp(-2 pi i t / 2(nx-1))
  double2* twy;      // (ny-1) twiddles
  double* inv_lam;   // [ny][nx]: 1 / lambda_pq at (q, p), interior indices
  double* T1;        // [nstack][ny][nx] row sine transforms
  double* T2;        // [nstack][ny][nx] after the column transforms
  double* phi;       // [nstack][ny][nx] potential (0 on the walls)
};

struct Tf32Plan;  // tensor-core DFT-GEMM form (solve_tf32.cu)

struct TrackPlan;  // captured turn graph (api.cu)

// Host<->device copies spread over a few streams (forked from and joined back
// to the caller's stream), so that several copy engines share a large transfer.
struct CopyJob {
  void* dst;
  const void* src;
  size_t bytes;
};
struct CopyStreams {
  static constexpr int kStreams = 4;
  cudaStream_t s[kStreams] = {};
  cudaEvent_t fork = nullptr, join[kStreams] = {};
};
sc_status copy_spread(CopyStreams** cs, cudaStream_t s, cudaMemcpyKind kind, const std::vector<CopyJob>& jobs);
void copy_streams_destroy(CopyStreams* cs);

}  // namespace sc

struct sc_grid {
  int nx, ny, nz, precision;   // nz: longitudinal slices, each with its own nx x ny grid
  // Transverse grids stored back to back and solved by one batched solve: nz
  // for a sliced grid, the bunch count for the grid class of a batch.
  int nstack;
  // Per stacked grid normalisation of the charge (2^-40 / N of that grid),
  // device float64 (FP64 form) or float32 (split form) array of nstack, or
  // NULL: every stacked grid is normalised by n_particles.
  void* stack_scale;
  double zmin, zmax;
  double xmin, xmax, ymin, ymax, hx, hy;
  sc::GridGeom geom;
  cudaStream_t stream;
  bool own_stream;
  int device;
  unsigned long long* Q;      // [nstack][ny][nx] uint64 charge (2^40 per particle)
  double2* E;                 // [nstack][ny][nx] (Ex, Ey); float32 pairs in the first half when field32
  int field32;                // the solve writes float32 fields (SC_SOLVE_TF32X3)
  unsigned long long* n_out;  // device counter (one per stacked grid in a batch class)
  unsigned long long* n_nan;  // device counter of non-finite particles seen by deposits (n_out + nstack)
  int poisoned;               // a tensor-core solve gave up on a bounded wait: no further solves
  int64_t n_particles;        // particle count of the last deposit (normalises Q)
  sc::Fft64Plan fft;
  sc::PipePlan pipe;
  sc::Tf32Plan* tf32;
  sc::TrackPlan* track;
  int trace;                   // record per-phase events in captured turns
  double* tune_acc;            // per-particle phase accumulators (caller-owned, 4 n) or NULL
  double tune_twiss[4];        // bare beta_x, alpha_x, beta_y, alpha_y at the turn start
  double trace_kp_ms, trace_solve_ms;
  int64_t trace_kicks;
  int lon;                     // longitudinal kick on (sliced pipe grids)
  int gather;                  // SC_GATHER_BILINEAR or SC_GATHER_BEZIER (pipe grids)
  int kp_blocks, dep_blocks;   // persistent grid sizes for this grid's tile size
  int kp_blocks_plain;         // kick/push without a deposit
  int kp_threads_set, kp_trav_set;  // kick/push shape forced by the caller (0 / -1: tuned)
  // last tuned kick/push shape and what it was timed on (particles, beam, lattice, options),
  // reused by re-captures that differ only in tracing or diagnostics
  std::vector<unsigned char> kp_tuned_key;
  int kp_tuned_threads, kp_tuned_trav;
  double kp_tuned_us;
  sc::DevElem* el_stage;       // device copy of sc_kick_push's last long segment
  int el_stage_cap;
  double* host_stage;          // device copy of sc_track_turns_host's particles [6][cap]
  int64_t host_stage_cap;
  sc::CopyStreams* copies;     // streams the host copies are spread over (created on first use)
  void* sort_scratch;          // sc_sort_particles' keys, indices, gather buffer and sort storage
  size_t sort_cap;
  const double* sorted_x;      // the bunch (x array, count) this grid last ordered by cell
  int64_t sorted_n;
  // charge reduction across the ranks of a sharded bunch (sc_set_charge_reduce)
  sc_charge_reduce_fn reduce_fn;
  void* reduce_user;
  int64_t reduce_total;        // particles of the whole bunch (normalises the solve)
};

namespace sc {

// deposit.cu
sc_status launch_deposit(sc_grid* g, const sc_particles* p);
// reorder the particles by their cell on g (stable); perm_out (device, n, or NULL) gets the old indices
sc_status sort_particles(sc_grid* g, const sc_particles* p, int32_t* perm_out);
// kick_push.cu
// blocks: dep->kp_blocks when depositing into dep, else the kick grid's kp_blocks_plain.
// threads: block size (0: the variant's largest); blocks as above.
sc_status launch_kick_push(const KPParams& P, const sc_grid* dep, int blocks, cudaStream_t s, int threads = 0);
int kick_push_max_threads(bool f32);
// resident blocks on the device at the given block size (smallest over the
// variants of this field type; smem_bytes: the deposit tile when tile)
int kick_push_blocks_at(int smem_bytes, bool tile, bool f32, int threads);
// Batched form: descs[bunch] per bunch, blocks[b] = (bunch, chunk, chunks of that bunch, 0) per block;
// deposits of grids whose tile window has at most tile_cells nodes go through the shared-memory tile.
// threads: block size (0: the field type's largest, kick_push_batched_threads)
sc_status launch_kick_push_batched(const KPParams* descs, const int4* blocks, int n_blocks, int tile_cells, bool f32,
                                   bool cache, bool xe, cudaStream_t s, int threads = 0);
int kick_push_batched_threads(bool f32);
// resident blocks on the device at this block size (0: the largest)
int kick_push_batched_resident(int smem_bytes, bool f32, bool cache, int threads = 0);
// shared memory of a grid's deposit tile; the tile window of an nx x ny grid
int tile_bytes(const sc_grid* g);
void tile_window(int nx, int ny, int* wx0, int* wy0, int* wnx, int* wny);
int deposit_blocks_for(int smem_bytes);
int kick_push_blocks_for(int smem_bytes, bool tile);
// solve_fft64.cu
sc_status fft64_create(sc_grid* g);
void fft64_destroy(sc_grid* g);
// zero_q: also clear the charge grid once it has been read (for the next deposit)
sc_status fft64_solve(sc_grid* g, bool zero_q);
// solve_pipe64.cu
sc_status pipe_create(sc_grid* g);
void pipe_destroy(sc_grid* g);
sc_status pipe_solve(sc_grid* g, bool zero_q);
// solve_tf32.cu
double tf32_tensor_flops(const sc_grid* g);  // tensor-core flops of one solve (all stacked grids)
sc_status tf32_create(sc_grid* g);
void tf32_destroy(sc_grid* g);
sc_status tf32_solve(sc_grid* g, bool zero_q);
int tf32_error(sc_grid* g);  // 1 when a tensor-core solve gave up on a bounded wait
// kernel variant per phase (4 entries) chosen by the tuner, with a description
sc_status tf32_get_tiling(const sc_grid* g, int* choice, std::string* desc);
sc_status tf32_set_tiling(sc_grid* g, const int* choice);  // -1 entries keep the current variant
sc_status tf32_read_potential(const sc_grid* g, double* out);  // pipe grids of the split form
const float* tf32_potential(const sc_grid* g);                 // device potential of a split-form pipe grid
sc_status tf32_test_bounded_waits(sc_grid* g, int enable);     // failure-detection test hook
// diag.cu
// out = *base_ptr + stride * (*turn) receives the 14 moments; bumps *turn
sc_status launch_moments(const sc_particles* p, double* partial, int n_blocks, double* const* base_ptr, int* turn,
                         int stride, cudaStream_t s);
int moments_blocks();
sc_status launch_phase_advance(const sc_particles* p, const double* twiss, double* acc, int accumulate,
                               cudaStream_t s);

// api.cu helpers shared with batch.cu
sc_status check_particles(const sc_particles* p);
sc_status check_beam(const sc_beam* b);
sc_status check_elements(const sc_element* e, int n);
double kick_strength(const sc_beam* b);
KPParams base_params(const sc_particles* p, const sc_beam* b);
void set_kick(KPParams& P, const sc_grid* g, double kl, double gamma0);
void set_deposit(KPParams& P, sc_grid* d);
void set_elements(KPParams& P, const sc_element* host, int n, const sc_beam* b, const DevElem* dev);
sc_status solve_dispatch(sc_grid* g, bool zero_q);
// After a synchronisation: SC_ERR_TIMEOUT (and the grid refuses further solves)
// when a tensor-core solve gave up on a bounded wait, else SC_ERR_NAN (and the
// count is cleared) when deposits met particles with a non-finite position.
sc_status check_grid_errors(sc_grid* g);
// Grid construction shared by sc_create_grid_sliced and batches: nstack stacked
// grids; n_slices > 1 slices them by sigma (then nstack == n_slices).
sc_status create_grid(sc_grid** out, int nx, int ny, double xmin, double xmax, double ymin, double ymax,
                      int n_slices, double zmin, double zmax, int nstack, int precision, void* stream);

// Build the cyclic difference-kernel fields Dx, Dy on the doubled grid, float64
// host arrays [My][Mx] (used by both solve forms).
void build_field_kernels(const sc_grid* g, double* Dx, double* Dy);

}  // namespace sc
