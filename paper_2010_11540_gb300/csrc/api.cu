// C-ABI of libsc (include/sc.h): grid lifecycle, the PIC-loop calls of
// Sec. I (deposit, solve, kick + push) and the turn driver that captures one
// turn of the ring as a CUDA graph and replays it: the per-particle plan
// arrays (cell cache, psigma quantities, quadrupole matrix entries), the
// kick/push launch shape timed on a scratch copy of the bunch, and the
// host-buffer entry point with its device copies.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "sc_internal.cuh"

namespace sc {

namespace {
thread_local std::string g_last_error;
}

sc_status set_error(sc_status code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

sc_status cuda_error(cudaError_t e, const char* what) {
  char buf[512];
  std::snprintf(buf, sizeof buf, "%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
  if (e == cudaErrorMemoryAllocation) return set_error(SC_ERR_OOM, buf);
  return set_error(SC_ERR_CUDA, buf);
}

// Captured turn of a ring for one (grid, particles, beam, lattice) set.
struct TrackPlan {
  std::vector<unsigned char> key;
  DevElem* d_elems = nullptr;  // compiled lattice (segments longer than KP_INLINE read it)
  int* cell = nullptr;         // cell cache [n]
  double2* frac = nullptr;     // float64 fraction cache [n] (float64 fields)
  int2* fix = nullptr;         // fixed-point fraction cache [n] (float32 fields)
  double* psc = nullptr;       // per-particle ps-dependent quantities [5][n]
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  bool has_head = false;
  bool diag = false;
  int n_kicks = 0;
  KPParams prologue{};        // deposit at the first marker (lattices that start with one)
  double* partial = nullptr;  // moments partial sums
  double** d_base = nullptr;  // device cell holding the diag output pointer
  int* d_turn = nullptr;      // device turn counter
  double* d_diag = nullptr;   // [cap][14]
  int diag_cap = 0;
  std::vector<cudaEvent_t> ev;  // tracing: per kick (solve start, kick/push start, kick/push end)
  int kp_threads = 0;           // kick/push block size (0: the variant's largest)
  int kp_trav = -1;             // kick/push traversal (-1: the variant's default, 0 grid stride, 1 chunks)
  int kp_blocks_dep = 0;        // resident grid sizes at kp_threads: with the deposit tile
  int kp_blocks_plain = 0;      //   and without a deposit
  double kp_trial_us = 0.0;     // timed trial of the chosen shape (0: not timed)
  std::vector<DevElem> qfam;    // quadrupole families with cached per-particle coefficients
  DevElem* d_qfam = nullptr;    // their device copy
  double* qcache = nullptr;     // [qfam][6][n]
};

namespace {

void destroy_plan(TrackPlan* t) {
  if (!t) return;
  if (t->exec) cudaGraphExecDestroy(t->exec);
  if (t->graph) cudaGraphDestroy(t->graph);
  cudaFree(t->d_elems);
  cudaFree(t->cell);
  cudaFree(t->frac);
  cudaFree(t->fix);
  cudaFree(t->psc);
  cudaFree(t->partial);
  cudaFree(t->d_base);
  cudaFree(t->d_turn);
  cudaFree(t->d_diag);
  cudaFree(t->d_qfam);
  cudaFree(t->qcache);
  for (cudaEvent_t e : t->ev) cudaEventDestroy(e);
  delete t;
}

}  // namespace

namespace {

// Bunches from this size up have their kick/push launch shape timed at plan build.
constexpr int64_t kShapeTuneMinParticles = int64_t(1) << 18;

// Launch shape of a captured turn's kick/push: block size and particle
// traversal.  Every shape gives bit-identical results (the charge is an
// integer sum, the particles are independent), so the choice changes only the
// time.  Each candidate (of the parts the caller left free) is captured as a
// graph of the turn's first kShapeTuneKicks space-charge steps (solve, then
// kick/push with its deposit, as in the turn itself) on a scratch copy of the
// particles and timed: one untimed launch, then the best of three.  The charge
// grid and the out-of-grid counters are put back afterwards; the fields and
// the psc, cell and fraction caches the trials overwrite are rebuilt by every
// call before they are read.
constexpr int kShapeTuneKicks = 16;

template <class Head, class Mark, class Launch, class Blocks>
sc_status tune_shape(sc_grid* g, TrackPlan* T, const sc_particles* p, Head&& head_params, Mark&& mark_params,
                     Launch&& launch, Blocks&& set_blocks) {
  const int64_t n = p->n;
  // the charge grid and its counters (out-of-grid per stacked grid, then the non-finite count)
  const size_t qbytes = (size_t)g->nx * g->ny * g->nstack * 8, obytes = 8 * (size_t)(g->nstack + 1);
  const int kicks = T->n_kicks < kShapeTuneKicks ? T->n_kicks : kShapeTuneKicks;
  double* scratch = nullptr;
  unsigned char* saved = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  sc_status st = SC_OK;
  auto cu = [&st](cudaError_t e, const char* what) {
    if (!st && e != cudaSuccess) st = cuda_error(e, what);
    return st == SC_OK;
  };
  // no room for the scratch copy: keep the default shape rather than fail the call
  if (cudaMalloc(&scratch, (size_t)n * 6 * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&saved, qbytes + obytes) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(scratch);
    return SC_OK;
  }
  cu(cudaEventCreate(&e0), "cudaEventCreate");
  cu(cudaEventCreate(&e1), "cudaEventCreate");
  sc_particles q = {scratch, scratch + n, scratch + 2 * n, scratch + 3 * n, scratch + 4 * n, scratch + 5 * n, n};
  const double* src[6] = {p->x, p->px, p->y, p->py, p->sigma, p->psigma};
  double* dst[6] = {q.x, q.px, q.y, q.py, q.sigma, q.psigma};
  cu(cudaMemcpyAsync(saved, g->Q, qbytes, cudaMemcpyDeviceToDevice, g->stream), "cudaMemcpyAsync");
  cu(cudaMemcpyAsync(saved + qbytes, g->n_out, obytes, cudaMemcpyDeviceToDevice, g->stream), "cudaMemcpyAsync");
  // Before every timed trial: the scratch bunch as the caller's, its psc cache,
  // and its charge (and cell cache) at the first marker when the lattice opens
  // with one (otherwise the trial opens with the head segment's deposit into a
  // cleared grid).  Every trial then runs the same first steps of the turn (a
  // bunch tracked again and again through a part of the ring would not stay
  // the workload: its optics need not be stable).
  auto reset = [&]() {
    for (int a = 0; a < 6 && st == SC_OK; ++a)
      cu(cudaMemcpyAsync(dst[a], src[a], (size_t)n * 8, cudaMemcpyDeviceToDevice, g->stream), "cudaMemcpyAsync");
    if (st == SC_OK && cu(cudaMemsetAsync(g->Q, 0, qbytes, g->stream), "cudaMemsetAsync")) {
      KPParams pro = T->prologue;
      pro.x = q.x, pro.px = q.px, pro.y = q.y, pro.py = q.py, pro.sg = q.sigma, pro.ps = q.psigma;
      st = launch(pro, !T->has_head);
    }
  };
  auto capture = [&](cudaGraphExec_t* exec) -> sc_status {
    SC_CUDA(cudaStreamBeginCapture(g->stream, cudaStreamCaptureModeThreadLocal));
    sc_status r = SC_OK;
    if (T->has_head) r = launch(head_params(&q), true);
    for (int k = 0; !r && k < kicks; ++k) {
      r = solve_dispatch(g, true);
      bool dep = false;
      if (!r) r = launch(mark_params(&q, (size_t)k, dep), dep);
    }
    cudaGraph_t graph = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(g->stream, &graph);
    if (!r && ce != cudaSuccess) r = cuda_error(ce, "cudaStreamEndCapture(shape trial)");
    if (!r) {
      const cudaError_t ie = cudaGraphInstantiate(exec, graph, 0);
      if (ie != cudaSuccess) r = cuda_error(ie, "cudaGraphInstantiate(shape trial)");
    }
    if (graph) cudaGraphDestroy(graph);
    return r;
  };
  const int th_set = g->kp_threads_set, tr_set = g->nz > 1 ? -1 : g->kp_trav_set;
  const int f32_max = kick_push_max_threads(g->field32);
  int best_th = T->kp_threads, best_tr = T->kp_trav;
  float best = 0.f;
  for (int th : {384, 512, 640, 768}) {
    if (th > f32_max || (th_set > 0 && th != th_set)) continue;
    for (int tr = 0; tr < 2 && st == SC_OK; ++tr) {
      if (g->nz > 1 ? tr != 0 : (tr_set >= 0 && tr != tr_set)) continue;
      T->kp_threads = th;
      T->kp_trav = g->nz > 1 ? -1 : tr;
      set_blocks();
      cudaGraphExec_t exec = nullptr;
      st = capture(&exec);
      float t_min = 0.f;
      for (int r = 0; r < 4 && st == SC_OK; ++r) {
        reset();
        cu(cudaEventRecord(e0, g->stream), "cudaEventRecord");
        cu(cudaGraphLaunch(exec, g->stream), "cudaGraphLaunch(shape trial)");
        cu(cudaEventRecord(e1, g->stream), "cudaEventRecord");
        cu(cudaEventSynchronize(e1), "shape trial");
        float ms = 0.f;
        cu(cudaEventElapsedTime(&ms, e0, e1), "cudaEventElapsedTime");
        if (r > 0 && (t_min == 0.f || ms < t_min)) t_min = ms;
      }
      if (exec) cudaGraphExecDestroy(exec);
      if (st == SC_OK && (best == 0.f || t_min < best)) {
        best = t_min;
        best_th = th;
        best_tr = T->kp_trav;
      }
    }
  }
  T->kp_threads = best_th;
  T->kp_trav = best_tr;
  T->kp_trial_us = 1e3 * (double)best;
  set_blocks();
  // the charge grid and the counters as the caller left them
  if (saved) {
    cu(cudaMemcpyAsync(g->Q, saved, qbytes, cudaMemcpyDeviceToDevice, g->stream), "cudaMemcpyAsync");
    cu(cudaMemcpyAsync(g->n_out, saved + qbytes, obytes, cudaMemcpyDeviceToDevice, g->stream), "cudaMemcpyAsync");
  }
  cu(cudaStreamSynchronize(g->stream), "shape trial");
  cudaFree(scratch);
  cudaFree(saved);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  return st;
}

}  // namespace

sc_status copy_spread(CopyStreams** csp, cudaStream_t s, cudaMemcpyKind kind, const std::vector<CopyJob>& jobs) {
  if (!*csp) {
    CopyStreams* cs = new (std::nothrow) CopyStreams();
    if (!cs) return set_error(SC_ERR_OOM, "host allocation failed");
    cudaError_t e = cudaEventCreateWithFlags(&cs->fork, cudaEventDisableTiming);
    for (int k = 0; k < CopyStreams::kStreams && e == cudaSuccess; ++k) {
      e = cudaStreamCreateWithFlags(&cs->s[k], cudaStreamNonBlocking);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&cs->join[k], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
      copy_streams_destroy(cs);
      return cuda_error(e, "copy streams");
    }
    *csp = cs;
  }
  CopyStreams* cs = *csp;
  constexpr size_t kChunk = size_t(8) << 20;
  SC_CUDA(cudaEventRecord(cs->fork, s));
  for (int k = 0; k < CopyStreams::kStreams; ++k) SC_CUDA(cudaStreamWaitEvent(cs->s[k], cs->fork, 0));
  int next = 0;
  for (const CopyJob& j : jobs)
    for (size_t o = 0; o < j.bytes; o += kChunk) {
      const size_t b = j.bytes - o < kChunk ? j.bytes - o : kChunk;
      SC_CUDA(cudaMemcpyAsync((char*)j.dst + o, (const char*)j.src + o, b, kind, cs->s[next]));
      next = (next + 1) % CopyStreams::kStreams;
    }
  for (int k = 0; k < CopyStreams::kStreams; ++k) {
    SC_CUDA(cudaEventRecord(cs->join[k], cs->s[k]));
    SC_CUDA(cudaStreamWaitEvent(s, cs->join[k], 0));
  }
  return SC_OK;
}

void copy_streams_destroy(CopyStreams* cs) {
  if (!cs) return;
  for (int k = 0; k < CopyStreams::kStreams; ++k) {
    if (cs->s[k]) {
      cudaStreamSynchronize(cs->s[k]);
      cudaStreamDestroy(cs->s[k]);
    }
    if (cs->join[k]) cudaEventDestroy(cs->join[k]);
  }
  if (cs->fork) cudaEventDestroy(cs->fork);
  delete cs;
}

sc_status check_particles(const sc_particles* p) {
  if (!p) return set_error(SC_ERR_ARG, "particles is NULL");
  if (p->n < 0) return set_error(SC_ERR_ARG, "negative particle count");
  if (p->n > 0 && (!p->x || !p->px || !p->y || !p->py || !p->sigma || !p->psigma))
    return set_error(SC_ERR_ARG, "particle array pointer is NULL");
  if (p->n > SC_MAX_PARTICLES_PER_GRID)
    return set_error(SC_ERR_OVERFLOW, "2^24 or more particles on one grid could overflow the 64-bit charge");
  return SC_OK;
}

sc_status check_beam(const sc_beam* b) {
  if (!b) return set_error(SC_ERR_ARG, "beam is NULL");
  if (!(b->gamma0 >= 1.0) || !(b->beta0 > 0.0 && b->beta0 < 1.0) || !std::isfinite(b->n_lambda) ||
      !std::isfinite(b->r_p))
    return set_error(SC_ERR_ARG, "beam constants out of range (gamma0 >= 1, 0 < beta0 < 1, finite n_lambda, r_p)");
  return SC_OK;
}

sc_status check_elements(const sc_element* e, int n) {
  if (n < 0 || (n > 0 && !e)) return set_error(SC_ERR_ARG, "bad element list");
  for (int k = 0; k < n; ++k) {
    if (e[k].type < SC_DRIFT || e[k].type > SC_EXACT_BEND) return set_error(SC_ERR_ARG, "unknown element type");
    if (!std::isfinite(e[k].length) || e[k].length < 0.0) return set_error(SC_ERR_ARG, "bad element length");
  }
  return SC_OK;
}

static bool any_quad(const sc_element* e, int n) {
  for (int k = 0; k < n; ++k)
    if (e[k].type == SC_QUAD) return true;
  return false;
}

// thick sextupoles and exact dipoles need the extended kernels
static bool any_xe(const sc_element* e, int n) {
  for (int k = 0; k < n; ++k)
    if (e[k].type == SC_EXACT_BEND || (e[k].type == SC_SEXT && e[k].length > 0.0)) return true;
  return false;
}

// K = 2 r_p N_lambda / (beta0^2 gamma0^3): the transverse kick of Sec. IV per
// unit length and unit normalised field.
double kick_strength(const sc_beam* b) {
  return 2.0 * b->r_p * b->n_lambda / (b->beta0 * b->beta0 * b->gamma0 * b->gamma0 * b->gamma0);
}

KPParams base_params(const sc_particles* p, const sc_beam* b) {
  KPParams P;
  std::memset(&P, 0, sizeof P);
  P.x = p->x;
  P.px = p->px;
  P.y = p->y;
  P.py = p->py;
  P.sg = p->sigma;
  P.ps = p->psigma;
  P.n = p->n;
  P.beta0_sq = b->beta0 * b->beta0;
  P.inv_gamma0_sq = 1.0 / (b->gamma0 * b->gamma0);
  P.traversal = -1;
  return P;
}

void set_kick(KPParams& P, const sc_grid* g, double kl, double gamma0) {
  P.do_kick = (kl != 0.0);
  P.gk = g->geom;
  P.E = g->E;
  P.E32 = (const float2*)g->E;
  P.field32 = g->field32;
  P.kl = kl;
  if (g->lon || g->gather == SC_GATHER_BEZIER) {
    P.phi = g->pipe.phi;         // float64 form
    P.phi32 = tf32_potential(g);  // split form
  }
  if (g->lon) {  // K gamma0 L / (2 dz)
    P.lon = 1;
    P.klz = kl * gamma0 / (2.0 * (g->zmax - g->zmin) / (double)g->nz);
  }
  if (g->gather == SC_GATHER_BEZIER) P.bezier = 1;
}

// The cell cache a deposit writes follows the deposit grid's field precision.
void set_deposit(KPParams& P, sc_grid* d) {
  P.field32 = d->field32;
  P.do_deposit = 1;
  P.gd = d->geom;
  P.Q = d->Q;
  P.n_out = d->n_out;
  P.n_nan = d->n_nan;
}

// Elements of a segment: inline in the launch parameters when they fit,
// else the device array `dev` (compiled already) at the same offset.
void set_elements(KPParams& P, const sc_element* host, int n, const sc_beam* b, const DevElem* dev) {
  P.n_elem = n;
  P.has_quad = any_quad(host, n);
  P.has_xe = any_xe(host, n);
  if (n <= KP_INLINE) {
    compile_elements(host, n, b, P.inl);
    P.el = nullptr;
  } else {
    P.el = dev;
  }
}

sc_status check_grid_errors(sc_grid* g) {
  if (tf32_error(g)) {
    g->poisoned = 1;
    return set_error(SC_ERR_TIMEOUT, "tensor-core solve gave up on a bounded wait; the grid takes no more solves");
  }
  unsigned long long v = 0;
  SC_CUDA(cudaMemcpy(&v, g->n_nan, 8, cudaMemcpyDeviceToHost));
  if (v) {
    SC_CUDA(cudaMemset(g->n_nan, 0, 8));
    return set_error(SC_ERR_NAN, std::to_string(v) + " particle(s) with a non-finite position reached a deposit");
  }
  return SC_OK;
}

sc_status solve_dispatch(sc_grid* g, bool zero_q) {
  if (g->poisoned) return set_error(SC_ERR_TIMEOUT, "a tensor-core solve on this grid gave up on a bounded wait");
  if (split_solve(g->precision)) return tf32_solve(g, zero_q);
  if (g->precision == SC_SOLVE_PIPE_FP64) return pipe_solve(g, zero_q);
  return fft64_solve(g, zero_q);
}

sc_status create_grid(sc_grid** out, int nx, int ny, double xmin, double xmax, double ymin, double ymax,
                      int n_slices, double zmin, double zmax, int nstack, int precision, void* stream) {
  if (!out) return set_error(SC_ERR_ARG, "out is NULL");
  if (n_slices < 1 || n_slices > 1024) return set_error(SC_ERR_ARG, "n_slices must be in 1..1024");
  if (n_slices > 1 && (!(zmax > zmin) || !std::isfinite(zmin) || !std::isfinite(zmax)))
    return set_error(SC_ERR_ARG, "slice range must be finite with zmax > zmin");
  if (nstack < 1 || (n_slices > 1 && nstack != n_slices)) return set_error(SC_ERR_ARG, "bad stacked grid count");
  if (nx < 2 || ny < 2 || nx > 4096 || ny > 4096) return set_error(SC_ERR_ARG, "grid needs 2..4096 nodes per axis");
  if ((int64_t)nx * ny * nstack > (1LL << 28))  // cell indices stay 32-bit
    return set_error(SC_ERR_ARG, "more than 2^28 nodes over all slices");
  if (!(xmax > xmin) || !(ymax > ymin) || !std::isfinite(xmin) || !std::isfinite(xmax) || !std::isfinite(ymin) ||
      !std::isfinite(ymax))
    return set_error(SC_ERR_ARG, "grid extent must be finite with xmax > xmin, ymax > ymin");
  if (precision != SC_SOLVE_FP64 && precision != SC_SOLVE_TF32X3 && precision != SC_SOLVE_PIPE_FP64 &&
      precision != SC_SOLVE_PIPE_TF32X3 && precision != SC_SOLVE_BF16X3)
    return set_error(SC_ERR_UNSUPPORTED, "unknown solve precision");
  sc_grid* g = new (std::nothrow) sc_grid();
  if (!g) return set_error(SC_ERR_OOM, "host allocation failed");
  g->kp_trav_set = -1;
  g->nx = nx;
  g->ny = ny;
  g->nz = n_slices;
  g->nstack = nstack;
  g->zmin = zmin;
  g->zmax = zmax;
  g->precision = precision;
  g->field32 = split_solve(precision);
  g->xmin = xmin;
  g->xmax = xmax;
  g->ymin = ymin;
  g->ymax = ymax;
  g->hx = (xmax - xmin) / (nx - 1);
  g->hy = (ymax - ymin) / (ny - 1);
  g->geom.nx = nx;
  g->geom.ny = ny;
  g->geom.xmin = xmin;
  g->geom.ymin = ymin;
  g->geom.inv_hx = 1.0 / g->hx;
  g->geom.inv_hy = 1.0 / g->hy;
  g->geom.xlast = (double)(nx - 1);
  g->geom.ylast = (double)(ny - 1);
  g->geom.nz = n_slices;
  g->geom.zmin = zmin;
  g->geom.inv_dz = n_slices > 1 ? 1.0 / ((zmax - zmin) / (double)n_slices) : 0.0;  // 1 / dz
  tile_window(nx, ny, &g->geom.wx0, &g->geom.wy0, &g->geom.wnx, &g->geom.wny);
  sc_status st = SC_OK;
  cudaError_t e = cudaGetDevice(&g->device);
  if (e != cudaSuccess) {
    st = cuda_error(e, "cudaGetDevice");
    delete g;
    return st;
  }
  if (stream) {
    g->stream = (cudaStream_t)stream;
  } else {
    // Graph capture needs a non-legacy stream; this one still orders with the legacy default stream.
    e = cudaStreamCreate(&g->stream);
    if (e != cudaSuccess) {
      st = cuda_error(e, "cudaStreamCreate");
      delete g;
      return st;
    }
    g->own_stream = true;
  }
  const size_t cells = (size_t)nx * ny * nstack;  // all stacked grids
  if ((e = cudaMalloc(&g->Q, cells * 8)) != cudaSuccess || (e = cudaMalloc(&g->E, cells * sizeof(double2))) != cudaSuccess ||
      (e = cudaMalloc(&g->n_out, 8 * (size_t)(nstack + 1))) != cudaSuccess) {
    st = cuda_error(e, "cudaMalloc(grid)");
    sc_destroy_grid(g);
    return st;
  }
  cudaMemsetAsync(g->Q, 0, cells * 8, g->stream);
  cudaMemsetAsync(g->E, 0, cells * sizeof(double2), g->stream);
  g->n_nan = g->n_out + nstack;
  cudaMemsetAsync(g->n_out, 0, 8 * (size_t)(nstack + 1), g->stream);
  g->dep_blocks = deposit_blocks_for(tile_bytes(g));
  g->kp_blocks = kick_push_blocks_for(tile_bytes(g), true);
  g->kp_blocks_plain = kick_push_blocks_for(0, false);
  st = split_solve(precision)                                                ? tf32_create(g)
       : (precision == SC_SOLVE_PIPE_FP64)                                    ? pipe_create(g)
                                                                              : fft64_create(g);
  if (st == SC_OK) {
    e = cudaStreamSynchronize(g->stream);
    if (e != cudaSuccess) st = cuda_error(e, "sc_create_grid");
  }
  if (st != SC_OK) {
    sc_destroy_grid(g);
    return st;
  }
  *out = g;
  return SC_OK;
}

}  // namespace sc

using namespace sc;

extern "C" {

sc_status sc_last_error(char* buf, size_t n) {
  if (!buf || n == 0) return SC_ERR_ARG;
  std::snprintf(buf, n, "%s", g_last_error.c_str());
  return SC_OK;
}

sc_status sc_create_grid(sc_grid** out, int nx, int ny, double xmin, double xmax, double ymin, double ymax,
                         int precision, void* stream) {
  return sc_create_grid_sliced(out, nx, ny, xmin, xmax, ymin, ymax, 1, 0.0, 0.0, precision, stream);
}

sc_status sc_create_grid_sliced(sc_grid** out, int nx, int ny, double xmin, double xmax, double ymin, double ymax,
                                int n_slices, double zmin, double zmax, int precision, void* stream) {
  return create_grid(out, nx, ny, xmin, xmax, ymin, ymax, n_slices, zmin, zmax, n_slices < 1 ? 1 : n_slices,
                     precision, stream);
}

sc_status sc_destroy_grid(sc_grid* g) {
  if (!g) return SC_OK;
  if (g->stream) cudaStreamSynchronize(g->stream);
  destroy_plan(g->track);
  if (split_solve(g->precision))
    tf32_destroy(g);
  else if (g->precision == SC_SOLVE_PIPE_FP64)
    pipe_destroy(g);
  else
    fft64_destroy(g);
  cudaFree(g->Q);
  cudaFree(g->E);
  cudaFree(g->host_stage);
  copy_streams_destroy(g->copies);
  cudaFree(g->n_out);
  cudaFree(g->stack_scale);
  cudaFree(g->el_stage);
  cudaFree(g->sort_scratch);
  if (g->own_stream) cudaStreamDestroy(g->stream);
  delete g;
  return SC_OK;
}

sc_status sc_deposit(sc_grid* g, const sc_particles* p) {
  if (!g) return set_error(SC_ERR_ARG, "grid is NULL");
  sc_status st = check_particles(p);
  if (st) return st;
  SC_CUDA(cudaMemsetAsync(g->Q, 0, (size_t)g->nx * g->ny * g->nstack * 8, g->stream));
  g->n_particles = p->n;
  if (p->n == 0) return SC_OK;
  return launch_deposit(g, p);
}

sc_status sc_sort_particles(sc_grid* g, const sc_particles* p, int32_t* perm) {
  if (!g) return set_error(SC_ERR_ARG, "grid is NULL");
  sc_status st = check_particles(p);
  if (st) return st;
  if (p->n == 0) return SC_OK;
  return sort_particles(g, p, perm);
}

sc_status sc_solve(sc_grid* g) {
  if (!g) return set_error(SC_ERR_ARG, "grid is NULL");
  return solve_dispatch(g, false);
}

sc_status sc_kick_push(sc_grid* g, const sc_particles* p, const sc_beam* b, double L_sc, const sc_element* elems,
                       int n_elems, sc_grid* next) {
  if (!g) return set_error(SC_ERR_ARG, "grid is NULL");
  if (!std::isfinite(L_sc)) return set_error(SC_ERR_ARG, "L_sc must be finite");
  sc_status st;
  if ((st = check_beam(b)) || (st = check_particles(p)) || (st = check_elements(elems, n_elems))) return st;
  if (next) {
    SC_CUDA(cudaMemsetAsync(next->Q, 0, (size_t)next->nx * next->ny * next->nstack * 8, g->stream));
    next->n_particles = p->n;
  }
  if (p->n == 0) return SC_OK;
  KPParams P = base_params(p, b);
  set_kick(P, g, kick_strength(b) * L_sc, b->gamma0);
  if (next) set_deposit(P, next);
  if (n_elems > KP_INLINE) {
    // long segment: compiled copy in device memory (synchronous upload)
    std::vector<DevElem> dev(n_elems);
    compile_elements(elems, n_elems, b, dev.data());
    SC_CUDA(cudaStreamSynchronize(g->stream));
    if (n_elems > g->el_stage_cap) {
      cudaFree(g->el_stage);
      g->el_stage = nullptr;
      g->el_stage_cap = 0;
      SC_CUDA(cudaMalloc(&g->el_stage, (size_t)n_elems * sizeof(DevElem)));
      g->el_stage_cap = n_elems;
    }
    SC_CUDA(cudaMemcpy(g->el_stage, dev.data(), (size_t)n_elems * sizeof(DevElem), cudaMemcpyHostToDevice));
  }
  set_elements(P, elems, n_elems, b, g->el_stage);
  return launch_kick_push(P, next, next ? next->kp_blocks : g->kp_blocks_plain, g->stream);
}

sc_status sc_grid_read(sc_grid* g, uint64_t* Q, double* Ex, double* Ey, int64_t* n_out) {
  if (!g) return set_error(SC_ERR_ARG, "grid is NULL");
  SC_CUDA(cudaStreamSynchronize(g->stream));
  const size_t cells = (size_t)g->nx * g->ny * g->nstack;
  if (Q) SC_CUDA(cudaMemcpy(Q, g->Q, cells * 8, cudaMemcpyDeviceToHost));
  if ((Ex || Ey) && g->field32) {
    std::vector<float2> E(cells);
    SC_CUDA(cudaMemcpy(E.data(), g->E, cells * sizeof(float2), cudaMemcpyDeviceToHost));
    for (size_t c = 0; c < cells; ++c) {
      if (Ex) Ex[c] = E[c].x;
      if (Ey) Ey[c] = E[c].y;
    }
  } else if (Ex || Ey) {
    std::vector<double2> E(cells);
    SC_CUDA(cudaMemcpy(E.data(), g->E, cells * sizeof(double2), cudaMemcpyDeviceToHost));
    for (size_t c = 0; c < cells; ++c) {
      if (Ex) Ex[c] = E[c].x;
      if (Ey) Ey[c] = E[c].y;
    }
  }
  if (n_out) {
    unsigned long long v = 0;
    SC_CUDA(cudaMemcpy(&v, g->n_out, 8, cudaMemcpyDeviceToHost));
    *n_out = (int64_t)v;
  }
  return check_grid_errors(g);
}

sc_status sc_set_longitudinal_kick(sc_grid* g, int enable) {
  if (!g) return set_error(SC_ERR_ARG, "grid is NULL");
  const bool pipe = g->precision == SC_SOLVE_PIPE_FP64 || g->precision == SC_SOLVE_PIPE_TF32X3;
  if (enable && (!pipe || g->nz < 2))
    return set_error(SC_ERR_UNSUPPORTED, "the longitudinal kick needs a sliced pipe grid");
  SC_CUDA(cudaStreamSynchronize(g->stream));
  g->lon = enable ? 1 : 0;
  return SC_OK;
}

sc_status sc_set_gather(sc_grid* g, int mode) {
  if (!g) return set_error(SC_ERR_ARG, "grid is NULL");
  if (mode != SC_GATHER_BILINEAR && mode != SC_GATHER_BEZIER) return set_error(SC_ERR_ARG, "unknown gather mode");
  if (mode == SC_GATHER_BEZIER && g->precision != SC_SOLVE_PIPE_FP64 && g->precision != SC_SOLVE_PIPE_TF32X3)
    return set_error(SC_ERR_UNSUPPORTED, "the Bezier gather needs the potential of a pipe grid");
  SC_CUDA(cudaStreamSynchronize(g->stream));
  g->gather = mode;
  return SC_OK;
}

sc_status sc_grid_read_potential(sc_grid* g, double* phi) {
  if (!g || !phi) return set_error(SC_ERR_ARG, "grid or phi is NULL");
  if (g->precision == SC_SOLVE_PIPE_TF32X3) {
    SC_CUDA(cudaStreamSynchronize(g->stream));
    return tf32_read_potential(g, phi);
  }
  if (g->precision != SC_SOLVE_PIPE_FP64) return set_error(SC_ERR_UNSUPPORTED, "only pipe grids keep the potential");
  SC_CUDA(cudaStreamSynchronize(g->stream));
  SC_CUDA(cudaMemcpy(phi, g->pipe.phi, (size_t)g->nx * g->ny * g->nstack * sizeof(double), cudaMemcpyDeviceToHost));
  return SC_OK;
}

sc_status sc_tune_setup(sc_grid* g, const sc_particles* p, const double* twiss, double* acc) {
  if (!g) return set_error(SC_ERR_ARG, "grid is NULL");
  if (!acc) {
    g->tune_acc = nullptr;
    return SC_OK;
  }
  sc_status st = check_particles(p);
  if (st) return st;
  if (!twiss || !(twiss[0] > 0.0) || !(twiss[2] > 0.0) || !std::isfinite(twiss[1]) || !std::isfinite(twiss[3]))
    return set_error(SC_ERR_ARG, "twiss needs beta_x > 0, alpha_x, beta_y > 0, alpha_y");
  for (int k = 0; k < 4; ++k) g->tune_twiss[k] = twiss[k];
  g->tune_acc = acc;
  if (p->n == 0) return SC_OK;
  SC_CUDA(cudaMemsetAsync(acc + 2 * p->n, 0, (size_t)p->n * 2 * sizeof(double), g->stream));
  return launch_phase_advance(p, g->tune_twiss, acc, 0, g->stream);
}

sc_status sc_get_solver_tiling(sc_grid* g, int* choice, char* desc, size_t n) {
  if (!g) return set_error(SC_ERR_ARG, "grid is NULL");
  std::string d;
  sc_status st = tf32_get_tiling(g, choice, desc ? &d : nullptr);
  if (st) return st;
  if (desc && n > 0) {
    std::strncpy(desc, d.c_str(), n - 1);
    desc[n - 1] = '\0';
  }
  return SC_OK;
}

sc_status sc_set_solver_tiling(sc_grid* g, const int* choice) {
  if (!g || !choice) return set_error(SC_ERR_ARG, "grid or choice is NULL");
  SC_CUDA(cudaStreamSynchronize(g->stream));
  if (g->track) {  // captured turns hold the old launches
    destroy_plan(g->track);
    g->track = nullptr;
  }
  return tf32_set_tiling(g, choice);
}

sc_status sc_test_bounded_waits(sc_grid* g, int enable) {
  if (!g) return set_error(SC_ERR_ARG, "grid is NULL");
  SC_CUDA(cudaStreamSynchronize(g->stream));
  if (g->track) {  // captured turns hold the old launch arguments
    destroy_plan(g->track);
    g->track = nullptr;
  }
  return tf32_test_bounded_waits(g, enable);
}

sc_status sc_trace_enable(sc_grid* g, int enable) {
  if (!g) return set_error(SC_ERR_ARG, "grid is NULL");
  g->trace = enable ? 1 : 0;
  g->trace_kp_ms = g->trace_solve_ms = 0.0;
  g->trace_kicks = 0;
  return SC_OK;
}

sc_status sc_trace_read(sc_grid* g, double* kick_push_ms, double* solve_ms, int64_t* n_kicks) {
  if (!g) return set_error(SC_ERR_ARG, "grid is NULL");
  if (kick_push_ms) *kick_push_ms = g->trace_kp_ms;
  if (solve_ms) *solve_ms = g->trace_solve_ms;
  if (n_kicks) *n_kicks = g->trace_kicks;
  g->trace_kp_ms = g->trace_solve_ms = 0.0;
  g->trace_kicks = 0;
  return SC_OK;
}

sc_status sc_grid_charge_device(sc_grid* g, uint64_t** Q, int64_t* cells) {
  if (!g || !Q) return set_error(SC_ERR_ARG, "grid or Q is NULL");
  *Q = (uint64_t*)g->Q;
  if (cells) *cells = (int64_t)g->nx * g->ny * g->nstack;
  return SC_OK;
}

sc_status sc_set_charge_reduce(sc_grid* g, sc_charge_reduce_fn fn, void* user, int64_t total_particles) {
  if (!g) return set_error(SC_ERR_ARG, "grid is NULL");
  if (fn && (total_particles < 1 || total_particles > ((int64_t)1 << 62)))
    return set_error(SC_ERR_ARG, "total_particles must be positive");
  SC_CUDA(cudaStreamSynchronize(g->stream));
  g->reduce_fn = fn;
  g->reduce_user = fn ? user : nullptr;
  g->reduce_total = fn ? total_particles : 0;
  return SC_OK;
}

sc_status sc_set_particle_count(sc_grid* g, int64_t n_particles) {
  if (!g) return set_error(SC_ERR_ARG, "grid is NULL");
  if (n_particles < 0) return set_error(SC_ERR_ARG, "negative particle count");
  g->n_particles = n_particles;
  return SC_OK;
}

sc_status sc_track_turns_host(sc_grid* g, const sc_particles* host, const sc_beam* b, const sc_element* lattice,
                              int n_elems, int n_turns, double* diag) {
  // every argument is checked before the device copies are sized
  sc_status st;
  if ((st = check_particles(host))) return st;
  if (!g) return set_error(SC_ERR_ARG, "grid is NULL");
  if ((st = check_beam(b)) || (st = check_elements(lattice, n_elems))) return st;
  if (n_turns < 0) return set_error(SC_ERR_ARG, "negative turn count");
  const int64_t n = host->n;
  if (n_turns == 0 || n == 0) return SC_OK;
  if (n > g->host_stage_cap) {
    SC_CUDA(cudaStreamSynchronize(g->stream));
    cudaFree(g->host_stage);
    g->host_stage = nullptr;
    g->host_stage_cap = 0;
    SC_CUDA(cudaMalloc(&g->host_stage, (size_t)n * 6 * sizeof(double)));
    g->host_stage_cap = n;
  }
  const size_t cap = (size_t)g->host_stage_cap;
  double* src[6] = {host->x, host->px, host->y, host->py, host->sigma, host->psigma};
  sc_particles dev = {g->host_stage, g->host_stage + cap, g->host_stage + 2 * cap, g->host_stage + 3 * cap,
                      g->host_stage + 4 * cap, g->host_stage + 5 * cap, n};
  double* dst[6] = {dev.x, dev.px, dev.y, dev.py, dev.sigma, dev.psigma};
  std::vector<CopyJob> in(6), out(6);
  for (int a = 0; a < 6; ++a) {
    in[a] = CopyJob{dst[a], src[a], (size_t)n * 8};
    out[a] = CopyJob{src[a], dst[a], (size_t)n * 8};
  }
  if ((st = copy_spread(&g->copies, g->stream, cudaMemcpyHostToDevice, in))) return st;
  if ((st = sc_track_turns(g, &dev, b, lattice, n_elems, n_turns, diag))) return st;
  if ((st = copy_spread(&g->copies, g->stream, cudaMemcpyDeviceToHost, out))) return st;
  SC_CUDA(cudaStreamSynchronize(g->stream));
  return check_grid_errors(g);
}

sc_status sc_get_solver_work(sc_grid* g, double* tensor_flops, double* fft_flops) {
  if (!g) return set_error(SC_ERR_ARG, "grid is NULL");
  const bool pipe = g->precision == SC_SOLVE_PIPE_FP64 || g->precision == SC_SOLVE_PIPE_TF32X3;
  // transform lengths: the zero-padded 2nx x 2ny grid (open), the odd extension 2(nx-1) x 2(ny-1) (pipe)
  const double lx = pipe ? 2.0 * (g->nx - 1) : 2.0 * g->nx, ly = pipe ? 2.0 * (g->ny - 1) : 2.0 * g->ny;
  const double n = lx * ly;
  if (fft_flops) *fft_flops = 2.0 * 5.0 * n * std::log2(n) * g->nstack;
  if (tensor_flops) *tensor_flops = g->tf32 ? tf32_tensor_flops(g) : 0.0;
  return SC_OK;
}

sc_status sc_set_kick_push_shape(sc_grid* g, int threads, int traversal) {
  if (!g) return set_error(SC_ERR_ARG, "grid is NULL");
  const int max = kick_push_max_threads(g->field32);
  if (threads < 0 || threads % 32 != 0 || threads > max)
    return set_error(SC_ERR_ARG, "kick/push block size must be 0 or a multiple of 32 up to the variant's maximum");
  if (traversal < -1 || traversal > 1) return set_error(SC_ERR_ARG, "traversal must be -1, 0 or 1");
  g->kp_threads_set = threads;
  g->kp_trav_set = traversal;
  return SC_OK;
}

sc_status sc_get_kick_push_shape(sc_grid* g, int* threads, int* traversal, double* trial_us) {
  if (!g) return set_error(SC_ERR_ARG, "grid is NULL");
  const TrackPlan* T = g->track;
  if (!T || !T->exec) return set_error(SC_ERR_ARG, "no captured turn on this grid");
  if (threads) *threads = T->kp_threads > 0 ? T->kp_threads : kick_push_max_threads(g->field32);
  if (traversal) *traversal = g->nz > 1 ? 1 : T->kp_trav >= 0 ? T->kp_trav : (g->field32 ? 1 : 0);
  if (trial_us) *trial_us = T->kp_trial_us;
  return SC_OK;
}

sc_status sc_grid_write_charge(sc_grid* g, const uint64_t* Q, int64_t n_particles) {
  if (!g || !Q) return set_error(SC_ERR_ARG, "grid or Q is NULL");
  if (n_particles < 0) return set_error(SC_ERR_ARG, "negative particle count");
  SC_CUDA(cudaStreamSynchronize(g->stream));
  SC_CUDA(cudaMemcpy(g->Q, Q, (size_t)g->nx * g->ny * g->nstack * 8, cudaMemcpyHostToDevice));
  g->n_particles = n_particles;
  return SC_OK;
}

sc_status sc_track_turns(sc_grid* g, const sc_particles* p, const sc_beam* b, const sc_element* lattice, int n_elems,
                         int n_turns, double* diag) {
  if (!g) return set_error(SC_ERR_ARG, "grid is NULL");
  if (n_turns < 0) return set_error(SC_ERR_ARG, "negative turn count");
  sc_status st;
  if ((st = check_beam(b)) || (st = check_particles(p)) || (st = check_elements(lattice, n_elems))) return st;
  if (n_turns == 0 || p->n == 0) return SC_OK;

  // ---- key of the captured plan ------------------------------------------------
  std::vector<unsigned char> key;
  auto put = [&key](const void* v, size_t n) {
    const unsigned char* c = (const unsigned char*)v;
    key.insert(key.end(), c, c + n);
  };
  // what the kick/push shape depends on: the particle count, beam, lattice and
  // settings, not where the particles live (the host-buffer call tracks from
  // the library's own staging copy and keeps the shape chosen for the caller's)
  put(&p->n, sizeof p->n);
  put(b, sizeof *b);
  put(&n_elems, sizeof n_elems);
  if (n_elems) put(lattice, (size_t)n_elems * sizeof(sc_element));
  put(&g->lon, sizeof g->lon);
  put(&g->gather, sizeof g->gather);
  put(&g->kp_threads_set, sizeof g->kp_threads_set);
  put(&g->kp_trav_set, sizeof g->kp_trav_set);
  const std::vector<unsigned char> shape_key = key;
  put(p, sizeof *p);
  put(&g->reduce_fn, sizeof g->reduce_fn);
  put(&g->reduce_user, sizeof g->reduce_user);
  put(&g->reduce_total, sizeof g->reduce_total);
  // the solve's normalisation: the whole bunch when its particles are sharded over ranks
  const int64_t n_norm = g->reduce_fn ? g->reduce_total : p->n;
  const int want_diag = diag != nullptr;
  put(&want_diag, sizeof want_diag);
  put(&g->trace, sizeof g->trace);
  put(&g->tune_acc, sizeof g->tune_acc);
  put(g->tune_twiss, sizeof g->tune_twiss);

  TrackPlan* T = g->track;
  if (!T || T->key != key) {
    destroy_plan(T);
    g->track = nullptr;
    T = new (std::nothrow) TrackPlan();
    if (!T) return set_error(SC_ERR_OOM, "host allocation failed");
    T->diag = want_diag;
    g->track = T;
    // ---- segments: head (before the first marker) and one per marker -----------
    std::vector<int> marks;
    std::vector<double> s(n_elems + 1, 0.0);
    for (int k = 0; k < n_elems; ++k) {
      s[k + 1] = s[k] + lattice[k].length;
      if (lattice[k].type == SC_MARK) marks.push_back(k);
    }
    const double circ = s[n_elems];
    T->n_kicks = (int)marks.size();
    T->has_head = marks.empty() ? true : marks[0] > 0;
    std::vector<DevElem> dev(n_elems > 0 ? n_elems : 1);
    compile_elements(lattice, n_elems, b, dev.data());
    // Quadrupole families whose per-particle coefficients the turn keeps: ps
    // changes only in RF cavities (after which they are recomputed); with the
    // longitudinal kick it changes at every kick, and each map computes its own.
    if (!g->lon) {
      T->qfam.resize(KP_QFAM_MAX);
      T->qfam.resize(quad_families(dev.data(), n_elems, T->qfam.data(), KP_QFAM_MAX));
      tag_quad_families(dev.data(), n_elems, T->qfam.data(), (int)T->qfam.size());
    }
    if (!T->qfam.empty()) {
      SC_CUDA(cudaMalloc(&T->qcache, T->qfam.size() * 6 * (size_t)p->n * sizeof(double)));
      SC_CUDA(cudaMalloc(&T->d_qfam, T->qfam.size() * sizeof(DevElem)));
      SC_CUDA(cudaMemcpy(T->d_qfam, T->qfam.data(), T->qfam.size() * sizeof(DevElem), cudaMemcpyHostToDevice));
    }
    auto with_qcache = [T](KPParams& P) {
      if (T->qfam.empty()) return;
      P.qcache = T->qcache;
      P.qfam = T->d_qfam;
      P.qfam_n = (int)T->qfam.size();
      if (!P.el) tag_quad_families(P.inl, P.n_elem, T->qfam.data(), P.qfam_n);
    };
    SC_CUDA(cudaMalloc(&T->d_elems, dev.size() * sizeof(DevElem)));
    SC_CUDA(cudaMemcpy(T->d_elems, dev.data(), dev.size() * sizeof(DevElem), cudaMemcpyHostToDevice));
    if (!marks.empty()) {
      SC_CUDA(cudaMalloc(&T->cell, (size_t)p->n * sizeof(int)));
      if (g->field32)
        SC_CUDA(cudaMalloc(&T->fix, (size_t)p->n * sizeof(int2)));
      else
        SC_CUDA(cudaMalloc(&T->frac, (size_t)p->n * sizeof(double2)));
    }
    SC_CUDA(cudaMalloc(&T->psc, (size_t)p->n * 5 * sizeof(double)));
    if (g->trace) {
      T->ev.resize(3 * marks.size());
      for (auto& e : T->ev) SC_CUDA(cudaEventCreate(&e));
    }
    if (want_diag) {
      SC_CUDA(cudaMalloc(&T->partial, (size_t)moments_blocks() * 14 * sizeof(double)));
      SC_CUDA(cudaMalloc(&T->d_base, sizeof(double*)));
      SC_CUDA(cudaMalloc(&T->d_turn, sizeof(int)));
    }
    g->n_particles = n_norm;
    const double K = kick_strength(b);
    // prologue of every call: the ps-dependent quantities of each particle, and
    // for lattices that open with a marker the charge (and cell cache) there
    T->prologue = base_params(p, b);
    T->prologue.psc = T->psc;
    T->prologue.psc_mode = 2;
    T->prologue.field32 = g->field32;  // every launch of the plan takes the grid's kernel family (and block size)
    with_qcache(T->prologue);
    if (!T->has_head && T->n_kicks > 0) {
      set_deposit(T->prologue, g);
      T->prologue.cell = T->cell;
      T->prologue.frac = T->frac;
      T->prologue.fix = T->fix;
    }
    // ---- kick/push launches of one turn, for particles q ------------------------
    const int nh = marks.empty() ? n_elems : marks[0];
    auto head_params = [&](const sc_particles* q) {
      KPParams P = base_params(q, b);
      P.psc = T->psc;
      P.psc_mode = 1;
      set_elements(P, lattice, nh, b, T->d_elems);
      with_qcache(P);
      P.psc_skip = psc_skip_mask(lattice, nh, b, T->qfam.data(), (int)T->qfam.size());
      P.ps_mode = ps_mode_mask(lattice, nh, false);
      if (!marks.empty()) {
        // the turn's last solve cleared the charge (and the prologue did before the first turn)
        set_deposit(P, g);
        P.cell = T->cell;
        P.frac = T->frac;
        P.fix = T->fix;
      }
      return P;
    };
    // marker k: kick, the segment up to the next marker, and (dep) the next deposit
    auto mark_params = [&](const sc_particles* q, size_t k, bool& dep) {
      const int m = marks[k];
      const int end = (k + 1 < marks.size()) ? marks[k + 1] : n_elems;
      const double prev = (k > 0) ? s[marks[k - 1]] : s[marks.back()] - circ;
      KPParams P = base_params(q, b);
      P.psc = T->psc;
      P.psc_mode = 1;
      set_kick(P, g, K * (s[m] - prev), b->gamma0);
      set_elements(P, lattice + m + 1, end - m - 1, b, T->d_elems + m + 1);
      with_qcache(P);
      P.psc_skip = psc_skip_mask(lattice + m + 1, end - m - 1, b, T->qfam.data(), (int)T->qfam.size());
      P.ps_mode = ps_mode_mask(lattice + m + 1, end - m - 1, P.lon != 0);
      // the cell cache is valid at every marker: the previous launch deposited on this grid
      P.cell = T->cell;
      P.frac = T->frac;
      P.fix = T->fix;
      dep = (k + 1 < marks.size()) || !T->has_head;
      if (dep) set_deposit(P, g);
      return P;
    };
    auto launch = [&](KPParams P, bool dep) {
      P.field32 = g->field32;
      P.traversal = T->kp_trav;
      return launch_kick_push(P, dep ? g : nullptr, dep ? T->kp_blocks_dep : T->kp_blocks_plain, g->stream,
                              T->kp_threads);
    };
    // ---- launch shape (block size, traversal) ----------------------------------
    T->kp_threads = g->kp_threads_set;
    T->kp_trav = g->nz > 1 ? -1 : g->kp_trav_set;  // sliced grids always use chunks
    auto set_blocks = [&] {
      const int th = T->kp_threads > 0 ? T->kp_threads : kick_push_max_threads(g->field32);
      T->kp_blocks_dep = kick_push_blocks_at(tile_bytes(g), true, g->field32, th);
      T->kp_blocks_plain = kick_push_blocks_at(0, false, g->field32, th);
    };
    set_blocks();
    const bool free_shape = T->kp_threads == 0 || (T->kp_trav < 0 && g->nz == 1);
    if (T->n_kicks > 0 && p->n >= kShapeTuneMinParticles && free_shape) {
      if (g->kp_tuned_key == shape_key) {
        T->kp_threads = g->kp_tuned_threads;
        T->kp_trav = g->kp_tuned_trav;
        T->kp_trial_us = g->kp_tuned_us;
        set_blocks();
      } else {
        sc_status tst = tune_shape(g, T, p, head_params, mark_params, launch, set_blocks);
        if (tst) {
          destroy_plan(T);
          g->track = nullptr;
          return tst;
        }
        g->kp_tuned_key = shape_key;
        g->kp_tuned_threads = T->kp_threads;
        g->kp_tuned_trav = T->kp_trav;
        g->kp_tuned_us = T->kp_trial_us;
      }
    }
    // ---- capture one turn ------------------------------------------------------
    SC_CUDA(cudaStreamBeginCapture(g->stream, cudaStreamCaptureModeThreadLocal));
    sc_status cst = SC_OK;
    if (want_diag) cst = launch_moments(p, T->partial, moments_blocks(), T->d_base, T->d_turn, 14, g->stream);
    if (!cst && T->has_head) cst = launch(head_params(p), !marks.empty());
    for (size_t k = 0; !cst && k < marks.size(); ++k) {
      if (g->trace && cudaEventRecordWithFlags(T->ev[3 * k], g->stream, cudaEventRecordExternal) != cudaSuccess) cst = set_error(SC_ERR_CUDA, "event");
      // a sharded bunch: the ranks' charges summed in place (the callback enqueues the reduction)
      if (!cst && g->reduce_fn &&
          g->reduce_fn((uint64_t*)g->Q, (int64_t)g->nx * g->ny * g->nstack, (void*)g->stream, g->reduce_user) != 0)
        cst = set_error(SC_ERR_CUDA, "the charge reduction callback failed");
      // the solve clears the charge after reading it, ready for this marker's deposit
      if (!cst) cst = solve_dispatch(g, true);
      if (cst) break;
      if (g->trace && cudaEventRecordWithFlags(T->ev[3 * k + 1], g->stream, cudaEventRecordExternal) != cudaSuccess) {
        cst = set_error(SC_ERR_CUDA, "event");
        break;
      }
      bool dep = false;
      const KPParams P = mark_params(p, k, dep);
      cst = launch(P, dep);
      if (!cst && g->trace && cudaEventRecordWithFlags(T->ev[3 * k + 2], g->stream, cudaEventRecordExternal) != cudaSuccess)
        cst = set_error(SC_ERR_CUDA, "event");
    }
    // per-particle phase advance over the turn (state at the end of the turn = start of the next)
    if (!cst && g->tune_acc) cst = launch_phase_advance(p, g->tune_twiss, g->tune_acc, 1, g->stream);
    cudaGraph_t graph = nullptr;
    cudaError_t ce = cudaStreamEndCapture(g->stream, &graph);
    if (cst) {
      if (graph) cudaGraphDestroy(graph);
      destroy_plan(T);
      g->track = nullptr;
      return cst;
    }
    if (ce != cudaSuccess) {
      destroy_plan(T);
      g->track = nullptr;
      return cuda_error(ce, "cudaStreamEndCapture");
    }
    T->graph = graph;
    ce = cudaGraphInstantiate(&T->exec, graph, 0);
    if (ce != cudaSuccess) {
      destroy_plan(T);
      g->track = nullptr;
      return cuda_error(ce, "cudaGraphInstantiate");
    }
    T->key = key;  // complete: a plan left half-built by an error is rebuilt by the next call
  }

  // ---- run -------------------------------------------------------------------------
  if (T->diag) {
    if (n_turns > T->diag_cap) {
      SC_CUDA(cudaStreamSynchronize(g->stream));
      cudaFree(T->d_diag);
      T->d_diag = nullptr;
      SC_CUDA(cudaMalloc(&T->d_diag, (size_t)n_turns * 14 * sizeof(double)));
      T->diag_cap = n_turns;
    }
    SC_CUDA(cudaMemcpyAsync(T->d_base, &T->d_diag, sizeof(double*), cudaMemcpyHostToDevice, g->stream));
    SC_CUDA(cudaMemsetAsync(T->d_turn, 0, sizeof(int), g->stream));
  }
  g->n_particles = n_norm;
  {
    KPParams P = T->prologue;
    P.traversal = T->kp_trav;
    if (!T->has_head && T->n_kicks > 0) {
      // charge at the first space-charge location of the first turn
      SC_CUDA(cudaMemsetAsync(g->Q, 0, (size_t)g->nx * g->ny * g->nstack * 8, g->stream));
      if ((st = launch_kick_push(P, g, T->kp_blocks_dep, g->stream, T->kp_threads))) return st;
    } else {
      if ((st = launch_kick_push(P, nullptr, T->kp_blocks_plain, g->stream, T->kp_threads))) return st;
    }
  }
  for (int t = 0; t < n_turns; ++t) {
    SC_CUDA(cudaGraphLaunch(T->exec, g->stream));
    if (!T->ev.empty()) {
      SC_CUDA(cudaStreamSynchronize(g->stream));
      for (size_t k = 0; 3 * k + 2 < T->ev.size(); ++k) {
        float a = 0.f, c = 0.f;
        SC_CUDA(cudaEventElapsedTime(&a, T->ev[3 * k], T->ev[3 * k + 1]));
        SC_CUDA(cudaEventElapsedTime(&c, T->ev[3 * k + 1], T->ev[3 * k + 2]));
        g->trace_solve_ms += a;
        g->trace_kp_ms += c;
        g->trace_kicks += 1;
      }
    }
  }
  if (T->diag) {
    SC_CUDA(cudaMemcpyAsync(diag, T->d_diag, (size_t)n_turns * 14 * sizeof(double), cudaMemcpyDeviceToHost,
                            g->stream));
    SC_CUDA(cudaStreamSynchronize(g->stream));
    if ((st = check_grid_errors(g))) return st;
    // a non-finite coordinate of any particle makes the moments of its turn non-finite
    for (int k = 0; k < n_turns * 14; ++k)
      if (!std::isfinite(diag[k]))
        return set_error(SC_ERR_NAN, "non-finite particle coordinates: the moments of turn " +
                                         std::to_string(k / 14) + " are not finite");
    return SC_OK;
  }
  return SC_OK;
}

}  // extern "C"
