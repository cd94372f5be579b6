// Batches of independent bunches: each bunch has its own particles, beam,
// lattice (working point) and transverse grid; per space-charge location the
// bunches' grids are solved class by class (grids with the same nodes and
// extent are stacked and solved by one set of launches) and ONE kick/push/
// deposit launch serves every bunch.  The per-bunch physics is that of
// sc_track_turns (Sec. I PIC loop, Sec. IV kick, Sec. III maps).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "sc_internal.cuh"

namespace sc {
namespace {

// Waves of resident blocks a batched launch is cut into by default: more
// waves balance bunches of uneven size better, fewer flush fewer deposit
// tiles.  Batches of kShapeTuneMin particles or more time the candidates
// (waves x block size) at capture instead.
constexpr int kWaves = 4;
constexpr int64_t kShapeTuneMin = int64_t(1) << 18;
constexpr int kShapeTuneKicks = 16;

struct BatchPlan {
  std::vector<unsigned char> key;
  int n_bunches = 0;
  bool has_head = false, diag = false;
  int n_kicks = 0;
  // per bunch
  std::vector<DevElem*> d_elems;
  std::vector<int*> cell;
  std::vector<double2*> frac;
  std::vector<int2*> fix;
  std::vector<double*> psc;
  // quadrupole families with cached per-particle coefficients (batch grids are
  // not sliced: ps changes only in RF cavities)
  std::vector<std::vector<DevElem>> qfam;
  std::vector<DevElem*> d_qfam;
  std::vector<double*> qcache;  // [qfam][6][n]
  // launch descriptors: [launch][bunch]; launch 0 = prologue, 1 = head (if any), then one per marker
  KPParams* d_descs = nullptr;
  int n_launches = 0;
  std::vector<char> launch_cache;  // CACHE flag per launch
  std::vector<char> launch_xe;     // extended-element kernels per launch (any bunch's segment needs them)
  int4* d_blocks = nullptr;
  int n_blocks = 0;
  int tile_cells = 0;
  int kp_threads = 0;     // batched kick/push block size (0: the field type's largest)
  int kp_waves = kWaves;  // waves of resident blocks per launch
  double trial_us = 0.0;  // timed trial of the chosen shape (0: not timed)
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  double* partial = nullptr;
  double** d_base = nullptr;  // [bunch]
  int* d_turn = nullptr;      // [bunch]
  double* d_diag = nullptr;
  int diag_cap = 0;
  std::vector<cudaEvent_t> ev;
};

void destroy_batch_plan(BatchPlan* t) {
  if (!t) return;
  if (t->exec) cudaGraphExecDestroy(t->exec);
  if (t->graph) cudaGraphDestroy(t->graph);
  for (auto* p : t->d_elems) cudaFree(p);
  for (auto* p : t->cell) cudaFree(p);
  for (auto* p : t->frac) cudaFree(p);
  for (auto* p : t->fix) cudaFree(p);
  for (auto* p : t->psc) cudaFree(p);
  for (auto* p : t->d_qfam) cudaFree(p);
  for (auto* p : t->qcache) cudaFree(p);
  cudaFree(t->d_descs);
  cudaFree(t->d_blocks);
  cudaFree(t->partial);
  cudaFree(t->d_base);
  cudaFree(t->d_turn);
  cudaFree(t->d_diag);
  for (cudaEvent_t e : t->ev) cudaEventDestroy(e);
  delete t;
}

}  // namespace
}  // namespace sc

struct sc_batch {
  int n_bunches = 0, precision = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::vector<sc_grid*> cls;   // grid classes (stacked grids)
  // classes after the first solve on side streams forked from the batch's
  // stream inside the captured turn (independent solves overlap)
  std::vector<cudaStream_t> side;
  cudaEvent_t fork_ev = nullptr;
  std::vector<cudaEvent_t> join_ev;
  std::vector<int> cls_of;     // bunch -> class
  std::vector<int> idx;        // bunch -> stacked grid within its class
  sc::BatchPlan* plan = nullptr;
  int trace = 0;
  double trace_kp_ms = 0.0, trace_solve_ms = 0.0;
  int64_t trace_kicks = 0;
  int kp_threads_set = 0, kp_waves_set = 0;  // batched kick/push shape fixed by the caller (0: tuned)
  // last tuned shape and what it was timed on, reused by re-captures that
  // differ only in tracing or diagnostics
  std::vector<unsigned char> tuned_key;
  int tuned_threads = 0, tuned_waves = 0;
  double tuned_us = 0.0;
  double* host_stage = nullptr;  // device copies for sc_batch_track_turns_host: bunch after bunch, [6][n_b] each
  int64_t host_stage_cap = 0;    // particles
  sc::CopyStreams* copies = nullptr;
};

using namespace sc;

namespace {

bool same_spec(const sc_grid_spec& a, const sc_grid_spec& b) {
  return a.nx == b.nx && a.ny == b.ny && a.xmin == b.xmin && a.xmax == b.xmax && a.ymin == b.ymin && a.ymax == b.ymax;
}

size_t cells_of(const sc_grid* g) { return (size_t)g->nx * g->ny; }

// Bunch b's view of its class grid: fields, charge and out-of-grid counter of
// its own stacked grid.
void bunch_kick(const sc_batch* B, int b, KPParams& P, double kl) {
  const sc_grid* g = B->cls[B->cls_of[b]];
  set_kick(P, g, kl, 1.0);  // batch grids are not sliced: no longitudinal kick
  const size_t off = (size_t)B->idx[b] * cells_of(g);
  P.E = g->E + off;
  P.E32 = (const float2*)g->E + off;
}

void bunch_deposit(const sc_batch* B, int b, KPParams& P) {
  sc_grid* g = B->cls[B->cls_of[b]];
  set_deposit(P, g);
  P.Q = g->Q + (size_t)B->idx[b] * cells_of(g);
  P.n_out = g->n_out + B->idx[b];
}

// Blocks of one batched launch: the smallest chunk for which the bunches'
// chunks fit `waves` waves of resident blocks; bunch by bunch, chunk by chunk.
std::vector<int4> partition(const std::vector<int64_t>& n, int resident, int waves) {
  const int target = waves * (resident > 0 ? resident : 1);
  int64_t total = 0;
  for (int64_t v : n) total += v;
  auto count = [&](int64_t chunk) {
    int64_t c = 0;
    for (int64_t v : n) c += (v + chunk - 1) / chunk;
    return c;
  };
  int64_t lo = 1, hi = std::max<int64_t>(1, total);
  while (lo < hi) {
    const int64_t mid = lo + (hi - lo) / 2;
    if (count(mid) <= target)
      hi = mid;
    else
      lo = mid + 1;
  }
  std::vector<int4> blocks;
  for (size_t b = 0; b < n.size(); ++b) {
    const int k = (int)((n[b] + lo - 1) / lo);
    for (int c = 0; c < k; ++c) blocks.push_back(make_int4((int)b, c, k, 0));
  }
  return blocks;
}

// Launch shape of the batched kick/push: block size and the waves of resident
// blocks each launch is cut into.  Every shape gives bit-identical results
// (integer charge, independent particles).  Each candidate (of the parts the
// caller left free) is captured as a graph of the turn's first
// kShapeTuneKicks space-charge steps (every class's solve, then the batched
// kick/push) on scratch copies of the bunches and timed: one untimed launch,
// then the best of three.  The classes' charge grids and out-of-grid counters
// are put back afterwards; the fields and per-particle caches the trials
// overwrite are rebuilt by every call before they are read.
template <class Capture, class Blocks>
sc_status tune_batch_shape(sc_batch* B, BatchPlan* T, const sc_bunch* bunches, const std::vector<int64_t>& counts,
                           const std::vector<KPParams>& descs, Capture&& capture, Blocks&& set_blocks) {
  const int nb = B->n_bunches;
  const bool f32 = split_solve(B->precision);
  cudaStream_t S = B->stream;
  const int kicks = T->n_kicks < kShapeTuneKicks ? T->n_kicks : kShapeTuneKicks;
  int64_t total = 0;
  for (int64_t v : counts) total += v;
  // candidates
  std::vector<int> ths, ws;
  const int th_max = kick_push_batched_threads(f32);
  for (int th : {512, th_max})
    if ((B->kp_threads_set == 0 || th == B->kp_threads_set) &&
        std::find(ths.begin(), ths.end(), th) == ths.end())
      ths.push_back(th);
  if (ths.empty()) ths.push_back(B->kp_threads_set);
  for (int w : {1, 2, 4, 8})
    if (B->kp_waves_set == 0 || w == B->kp_waves_set) ws.push_back(w);
  if (ws.empty()) ws.push_back(B->kp_waves_set);
  size_t max_blocks = 0;
  for (int th : ths) {
    T->kp_threads = th;
    for (int w : ws) {
      std::vector<int4> bl;
      set_blocks(w, bl);
      max_blocks = std::max(max_blocks, bl.size());
    }
  }
  size_t saved_bytes = 0;
  for (sc_grid* g : B->cls) saved_bytes += cells_of(g) * g->nstack * 8 + 8 * (size_t)(g->nstack + 1);
  double* scratch = nullptr;
  KPParams* d_sdescs = nullptr;
  int4* d_blk = nullptr;
  unsigned char* saved = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  sc_status st = SC_OK;
  auto cu = [&st](cudaError_t e, const char* what) {
    if (!st && e != cudaSuccess) st = cuda_error(e, what);
    return st == SC_OK;
  };
  // no room for the scratch copies: keep the default shape rather than fail the call
  if (cudaMalloc(&scratch, (size_t)(total > 0 ? total : 1) * 6 * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&d_sdescs, descs.size() * sizeof(KPParams)) != cudaSuccess ||
      cudaMalloc(&d_blk, (max_blocks > 0 ? max_blocks : 1) * sizeof(int4)) != cudaSuccess ||
      cudaMalloc(&saved, saved_bytes) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(scratch);
    cudaFree(d_sdescs);
    cudaFree(d_blk);
    T->kp_threads = B->kp_threads_set;
    T->kp_waves = B->kp_waves_set > 0 ? B->kp_waves_set : kWaves;
    return SC_OK;
  }
  cu(cudaEventCreate(&e0), "cudaEventCreate");
  cu(cudaEventCreate(&e1), "cudaEventCreate");
  // scratch copies of the bunches (refreshed before every trial) and descriptors that point at them
  std::vector<KPParams> sd = descs;
  auto copy_bunches = [&]() {
    size_t o = 0;
    for (int b = 0; b < nb && st == SC_OK; ++b) {
      const sc_particles& h = bunches[b].particles;
      const size_t n = (size_t)h.n;
      double* base = scratch + 6 * o;
      const double* src[6] = {h.x, h.px, h.y, h.py, h.sigma, h.psigma};
      for (int a = 0; a < 6 && n > 0; ++a)
        cu(cudaMemcpyAsync(base + a * n, src[a], n * 8, cudaMemcpyDeviceToDevice, S), "cudaMemcpyAsync");
      o += n;
    }
  };
  size_t off = 0;
  for (int b = 0; b < nb && st == SC_OK; ++b) {
    const size_t n = (size_t)bunches[b].particles.n;
    double* base = scratch + 6 * off;
    for (int L = 0; L < T->n_launches; ++L) {
      KPParams& P = sd[(size_t)L * nb + b];
      P.x = base, P.px = base + n, P.y = base + 2 * n, P.py = base + 3 * n, P.sg = base + 4 * n,
      P.ps = base + 5 * n;
    }
    off += n;
  }
  cu(cudaMemcpyAsync(d_sdescs, sd.data(), sd.size() * sizeof(KPParams), cudaMemcpyHostToDevice, S),
     "cudaMemcpyAsync");
  auto grids = [&](bool save) {
    size_t o = 0;
    for (sc_grid* g : B->cls) {
      const size_t qb = cells_of(g) * g->nstack * 8, ob = 8 * (size_t)(g->nstack + 1);
      if (save) {
        cu(cudaMemcpyAsync(saved + o, g->Q, qb, cudaMemcpyDeviceToDevice, S), "cudaMemcpyAsync");
        cu(cudaMemcpyAsync(saved + o + qb, g->n_out, ob, cudaMemcpyDeviceToDevice, S), "cudaMemcpyAsync");
      } else {
        cu(cudaMemcpyAsync(g->Q, saved + o, qb, cudaMemcpyDeviceToDevice, S), "cudaMemcpyAsync");
        cu(cudaMemcpyAsync(g->n_out, saved + o + qb, ob, cudaMemcpyDeviceToDevice, S), "cudaMemcpyAsync");
      }
      o += qb + ob;
    }
  };
  auto clear_q = [&] {
    for (sc_grid* g : B->cls) cu(cudaMemsetAsync(g->Q, 0, cells_of(g) * g->nstack * 8, S), "cudaMemsetAsync");
  };
  if (st == SC_OK) grids(true);
  int best_th = ths[0], best_w = ws[0];
  float best = 0.f;
  for (int th : ths) {
    for (int w : ws) {
      if (st != SC_OK) break;
      T->kp_threads = th;
      std::vector<int4> bl;
      set_blocks(w, bl);
      if (bl.empty()) continue;
      cu(cudaMemcpyAsync(d_blk, bl.data(), bl.size() * sizeof(int4), cudaMemcpyHostToDevice, S), "cudaMemcpyAsync");
      cudaGraph_t graph = nullptr;
      cudaGraphExec_t exec = nullptr;
      if (st == SC_OK) st = capture(d_sdescs, d_blk, (int)bl.size(), kicks, false, &graph);
      if (st == SC_OK) cu(cudaGraphInstantiate(&exec, graph, 0), "cudaGraphInstantiate(shape trial)");
      if (graph) cudaGraphDestroy(graph);
      float t_min = 0.f;
      for (int r = 0; r < 4 && st == SC_OK; ++r) {
        // every trial from the bunches as the caller's: their psc and quadrupole caches, and
        // their charge at the first marker when the lattices open with one (else the trial
        // opens with the head's deposit into cleared grids)
        copy_bunches();
        clear_q();
        if (st == SC_OK)
          st = launch_kick_push_batched(d_sdescs, d_blk, (int)bl.size(), T->tile_cells, f32, T->launch_cache[0] != 0,
                                        T->launch_xe[0] != 0, S, th);
        cu(cudaEventRecord(e0, S), "cudaEventRecord");
        cu(cudaGraphLaunch(exec, S), "cudaGraphLaunch(shape trial)");
        cu(cudaEventRecord(e1, S), "cudaEventRecord");
        cu(cudaEventSynchronize(e1), "shape trial");
        float ms = 0.f;
        cu(cudaEventElapsedTime(&ms, e0, e1), "cudaEventElapsedTime");
        if (r > 0 && (t_min == 0.f || ms < t_min)) t_min = ms;
      }
      if (exec) cudaGraphExecDestroy(exec);
      if (st == SC_OK && (best == 0.f || t_min < best)) {
        best = t_min;
        best_th = th;
        best_w = w;
      }
    }
  }
  T->kp_threads = best_th;
  T->kp_waves = best_w;
  T->trial_us = 1e3 * (double)best;
  if (saved) grids(false);
  cu(cudaStreamSynchronize(S), "shape trial");
  cudaFree(scratch);
  cudaFree(d_sdescs);
  cudaFree(d_blk);
  cudaFree(saved);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  return st;
}

}  // namespace

extern "C" {

sc_status sc_create_batch(sc_batch** out, const sc_grid_spec* grids, int n_bunches, int precision, void* stream) {
  if (!out || !grids) return set_error(SC_ERR_ARG, "out or grids is NULL");
  if (n_bunches < 1 || n_bunches > 4096) return set_error(SC_ERR_ARG, "n_bunches must be in 1..4096");
  sc_batch* B = new (std::nothrow) sc_batch();
  if (!B) return set_error(SC_ERR_OOM, "host allocation failed");
  B->n_bunches = n_bunches;
  B->precision = precision;
  if (stream) {
    B->stream = (cudaStream_t)stream;
  } else {
    cudaError_t e = cudaStreamCreate(&B->stream);
    if (e != cudaSuccess) {
      delete B;
      return cuda_error(e, "cudaStreamCreate");
    }
    B->own_stream = true;
  }
  std::vector<sc_grid_spec> spec;  // per class
  std::vector<int> count;
  B->cls_of.resize(n_bunches);
  B->idx.resize(n_bunches);
  for (int b = 0; b < n_bunches; ++b) {
    int c = 0;
    while (c < (int)spec.size() && !same_spec(spec[c], grids[b])) ++c;
    if (c == (int)spec.size()) {
      spec.push_back(grids[b]);
      count.push_back(0);
    }
    B->cls_of[b] = c;
    B->idx[b] = count[c]++;
  }
  for (size_t c = 0; c < spec.size(); ++c) {
    const sc_grid_spec& s = spec[c];
    sc_grid* g = nullptr;
    sc_status st = create_grid(&g, s.nx, s.ny, s.xmin, s.xmax, s.ymin, s.ymax, 1, 0.0, 0.0, count[c], precision,
                               B->stream);
    if (st == SC_OK) {
      const bool f32 = split_solve(precision);
      const size_t bytes = (size_t)count[c] * (f32 ? sizeof(float) : sizeof(double));
      cudaError_t e = cudaMalloc(&g->stack_scale, bytes);
      if (e != cudaSuccess) {
        sc_destroy_grid(g);
        st = cuda_error(e, "cudaMalloc(stack_scale)");
      }
    }
    if (st != SC_OK) {
      sc_destroy_batch(B);
      return st;
    }
    B->cls.push_back(g);
  }
  if (B->cls.size() > 1) {
    cudaError_t e = cudaEventCreateWithFlags(&B->fork_ev, cudaEventDisableTiming);
    for (size_t c = 1; c < B->cls.size() && e == cudaSuccess; ++c) {
      cudaStream_t st = nullptr;
      cudaEvent_t ev = nullptr;
      e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
      if (e == cudaSuccess) B->side.push_back(st);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
      if (e == cudaSuccess) B->join_ev.push_back(ev);
    }
    if (e != cudaSuccess) {
      sc_destroy_batch(B);
      return cuda_error(e, "side streams of a batch");
    }
  }
  *out = B;
  return SC_OK;
}

sc_status sc_destroy_batch(sc_batch* B) {
  if (!B) return SC_OK;
  if (B->stream) cudaStreamSynchronize(B->stream);
  destroy_batch_plan(B->plan);
  for (sc_grid* g : B->cls) sc_destroy_grid(g);
  for (cudaStream_t st : B->side) cudaStreamDestroy(st);
  for (cudaEvent_t ev : B->join_ev) cudaEventDestroy(ev);
  if (B->fork_ev) cudaEventDestroy(B->fork_ev);
  cudaFree(B->host_stage);
  copy_streams_destroy(B->copies);
  if (B->own_stream) cudaStreamDestroy(B->stream);
  delete B;
  return SC_OK;
}

sc_status sc_batch_set_kick_push_shape(sc_batch* B, int threads, int waves) {
  if (!B) return set_error(SC_ERR_ARG, "batch is NULL");
  const bool f32 = split_solve(B->precision);
  if (threads < 0 || threads % 32 != 0 || threads > kick_push_batched_threads(f32))
    return set_error(SC_ERR_ARG, "batched kick/push block size must be 0 or a multiple of 32 up to the maximum");
  if (waves < 0 || waves > 64) return set_error(SC_ERR_ARG, "waves must be in 0..64");
  B->kp_threads_set = threads;
  B->kp_waves_set = waves;
  return SC_OK;
}

sc_status sc_batch_get_kick_push_shape(sc_batch* B, int* threads, int* waves, double* trial_us) {
  if (!B) return set_error(SC_ERR_ARG, "batch is NULL");
  const BatchPlan* T = B->plan;
  if (!T || !T->exec) return set_error(SC_ERR_ARG, "no captured turn on this batch");
  const bool f32 = split_solve(B->precision);
  if (threads) *threads = T->kp_threads > 0 ? T->kp_threads : kick_push_batched_threads(f32);
  if (waves) *waves = T->kp_waves;
  if (trial_us) *trial_us = T->trial_us;
  return SC_OK;
}

sc_status sc_batch_track_turns_host(sc_batch* B, const sc_bunch* bunches, int n_turns, double* diag) {
  if (!B || !bunches) return set_error(SC_ERR_ARG, "batch or bunches is NULL");
  if (n_turns < 0) return set_error(SC_ERR_ARG, "negative turn count");
  const int nb = B->n_bunches;
  sc_status st;
  int64_t total = 0;
  for (int b = 0; b < nb; ++b) {
    if ((st = check_particles(&bunches[b].particles))) return st;
    total += bunches[b].particles.n;
  }
  if (n_turns == 0) return SC_OK;
  if (total > B->host_stage_cap) {
    SC_CUDA(cudaStreamSynchronize(B->stream));
    cudaFree(B->host_stage);
    B->host_stage = nullptr;
    B->host_stage_cap = 0;
    SC_CUDA(cudaMalloc(&B->host_stage, (size_t)(total > 0 ? total : 1) * 6 * sizeof(double)));
    B->host_stage_cap = total;
  }
  std::vector<sc_bunch> dev(bunches, bunches + nb);
  std::vector<CopyJob> in, out;
  size_t off = 0;
  for (int b = 0; b < nb; ++b) {
    const sc_particles& h = bunches[b].particles;
    const size_t n = (size_t)h.n;
    sc_particles& d = dev[b].particles;
    double* base = B->host_stage + 6 * off;
    d.x = base, d.px = base + n, d.y = base + 2 * n, d.py = base + 3 * n, d.sigma = base + 4 * n,
    d.psigma = base + 5 * n;
    double* host[6] = {h.x, h.px, h.y, h.py, h.sigma, h.psigma};
    for (int a = 0; a < 6 && n > 0; ++a) {
      in.push_back(CopyJob{base + a * n, host[a], n * 8});
      out.push_back(CopyJob{host[a], base + a * n, n * 8});
    }
    off += n;
  }
  if ((st = copy_spread(&B->copies, B->stream, cudaMemcpyHostToDevice, in))) return st;
  if ((st = sc_batch_track_turns(B, dev.data(), n_turns, diag))) return st;
  if ((st = copy_spread(&B->copies, B->stream, cudaMemcpyDeviceToHost, out))) return st;
  SC_CUDA(cudaStreamSynchronize(B->stream));
  return SC_OK;
}

sc_status sc_batch_track_turns(sc_batch* B, const sc_bunch* bunches, int n_turns, double* diag) {
  if (!B || !bunches) return set_error(SC_ERR_ARG, "batch or bunches is NULL");
  if (n_turns < 0) return set_error(SC_ERR_ARG, "negative turn count");
  const int nb = B->n_bunches;
  sc_status st;
  // markers of every lattice
  std::vector<std::vector<int>> marks(nb);
  for (int b = 0; b < nb; ++b) {
    const sc_bunch& u = bunches[b];
    if ((st = check_beam(&u.beam)) || (st = check_particles(&u.particles)) ||
        (st = check_elements(u.lattice, u.n_elems)))
      return st;
    for (int k = 0; k < u.n_elems; ++k)
      if (u.lattice[k].type == SC_MARK) marks[b].push_back(k);
    const bool head = marks[b].empty() || marks[b][0] > 0;
    const bool head0 = marks[0].empty() || marks[0][0] > 0;
    if (marks[b].size() != marks[0].size() || head != head0)
      return set_error(SC_ERR_ARG, "every lattice of a batch needs the same SC markers (count, and one at the start or none)");
  }
  if (n_turns == 0) return SC_OK;

  // ---- key of the captured plan ------------------------------------------------
  std::vector<unsigned char> key;
  auto put = [&key](const void* v, size_t n) {
    const unsigned char* c = (const unsigned char*)v;
    key.insert(key.end(), c, c + n);
  };
  // what the kick/push shape depends on: the bunches' counts, beams and lattices
  // and the settings, not where the particles live (the host-buffer call tracks
  // from the library's own staging copies and keeps the shape chosen for the caller's)
  for (int b = 0; b < nb; ++b) {
    put(&bunches[b].particles.n, sizeof(int64_t));
    put(&bunches[b].beam, sizeof(sc_beam));
    put(&bunches[b].n_elems, sizeof(int));
    if (bunches[b].n_elems) put(bunches[b].lattice, (size_t)bunches[b].n_elems * sizeof(sc_element));
  }
  put(&B->kp_threads_set, sizeof B->kp_threads_set);
  put(&B->kp_waves_set, sizeof B->kp_waves_set);
  const std::vector<unsigned char> shape_key = key;
  for (int b = 0; b < nb; ++b) put(&bunches[b].particles, sizeof(sc_particles));
  const int want_diag = diag != nullptr;
  put(&want_diag, sizeof want_diag);
  put(&B->trace, sizeof B->trace);

  const bool f32 = split_solve(B->precision);
  BatchPlan* T = B->plan;
  if (!T || T->key != key) {
    destroy_batch_plan(T);
    B->plan = nullptr;
    T = new (std::nothrow) BatchPlan();
    if (!T) return set_error(SC_ERR_OOM, "host allocation failed");
    B->plan = T;
    T->diag = want_diag;
    T->n_bunches = nb;
    const int n_marks = (int)marks[0].size();
    T->n_kicks = n_marks;
    T->has_head = marks[0].empty() || marks[0][0] > 0;
    T->d_elems.assign(nb, nullptr);
    T->cell.assign(nb, nullptr);
    T->frac.assign(nb, nullptr);
    T->fix.assign(nb, nullptr);
    T->psc.assign(nb, nullptr);
    T->qfam.assign(nb, {});
    T->d_qfam.assign(nb, nullptr);
    T->qcache.assign(nb, nullptr);
    std::vector<int64_t> counts(nb);
    for (int b = 0; b < nb; ++b) {
      const sc_bunch& u = bunches[b];
      const int64_t n = u.particles.n;
      counts[b] = n;
      std::vector<DevElem> dev(u.n_elems > 0 ? u.n_elems : 1);
      compile_elements(u.lattice, u.n_elems, &u.beam, dev.data());
      std::vector<DevElem>& fam = T->qfam[b];
      fam.resize(KP_QFAM_MAX);
      fam.resize(quad_families(dev.data(), u.n_elems, fam.data(), KP_QFAM_MAX));
      tag_quad_families(dev.data(), u.n_elems, fam.data(), (int)fam.size());
      if (!fam.empty() && n > 0) {
        SC_CUDA(cudaMalloc(&T->qcache[b], fam.size() * 6 * (size_t)n * sizeof(double)));
        SC_CUDA(cudaMalloc(&T->d_qfam[b], fam.size() * sizeof(DevElem)));
        SC_CUDA(cudaMemcpy(T->d_qfam[b], fam.data(), fam.size() * sizeof(DevElem), cudaMemcpyHostToDevice));
      }
      SC_CUDA(cudaMalloc(&T->d_elems[b], dev.size() * sizeof(DevElem)));
      SC_CUDA(cudaMemcpy(T->d_elems[b], dev.data(), dev.size() * sizeof(DevElem), cudaMemcpyHostToDevice));
      const size_t m = (size_t)(n > 0 ? n : 1);
      if (n_marks > 0) {
        SC_CUDA(cudaMalloc(&T->cell[b], m * sizeof(int)));
        if (f32)
          SC_CUDA(cudaMalloc(&T->fix[b], m * sizeof(int2)));
        else
          SC_CUDA(cudaMalloc(&T->frac[b], m * sizeof(double2)));
      }
      SC_CUDA(cudaMalloc(&T->psc[b], m * 5 * sizeof(double)));
    }
    // per-bunch charge normalisation 2^-40 / N_b, class by class
    for (size_t c = 0; c < B->cls.size(); ++c) {
      sc_grid* g = B->cls[c];
      std::vector<double> sd(g->nstack, 0.0);
      for (int b = 0; b < nb; ++b)
        if (B->cls_of[b] == (int)c) sd[B->idx[b]] = 1.0 / 1099511627776.0 / (double)(counts[b] > 0 ? counts[b] : 1);
      if (f32) {
        std::vector<float> sf(sd.begin(), sd.end());
        SC_CUDA(cudaMemcpy(g->stack_scale, sf.data(), sf.size() * sizeof(float), cudaMemcpyHostToDevice));
      } else {
        SC_CUDA(cudaMemcpy(g->stack_scale, sd.data(), sd.size() * sizeof(double), cudaMemcpyHostToDevice));
      }
    }
    // blocks of the batched launch: the shared-memory tile holds the largest class grid that fits
    // whole (bunches on larger grids add straight to the global grid), or, when none fits, the
    // largest tile window: every block allocates the tile, and the shared memory it takes is L1
    // cache the field gathers of every bunch lose (measured on c4: a 200 KB window for its
    // 256^2 bunches made the launch 7% slower than 128 KB tiles and global atomics for them)
    int whole = 0, window = 0;
    for (sc_grid* g : B->cls) {
      if (g->geom.wnx == g->nx && g->geom.wny == g->ny) whole = std::max(whole, g->nx * g->ny);
      window = std::max(window, g->geom.wnx * g->geom.wny);
    }
    T->tile_cells = whole > 0 ? whole : window;
    // ---- descriptors: prologue, head, one per marker ------------------------------
    T->n_launches = 1 + (T->has_head ? 1 : 0) + n_marks;
    std::vector<KPParams> descs((size_t)T->n_launches * nb);
    T->launch_cache.assign(T->n_launches, 0);
    T->launch_xe.assign(T->n_launches, 0);
    for (int b = 0; b < nb; ++b) {
      const sc_bunch& u = bunches[b];
      const sc_particles* p = &u.particles;
      const sc_beam* bm = &u.beam;
      const std::vector<int>& mk = marks[b];
      std::vector<double> s(u.n_elems + 1, 0.0);
      for (int k = 0; k < u.n_elems; ++k) s[k + 1] = s[k] + u.lattice[k].length;
      const double circ = s[u.n_elems];
      const double K = kick_strength(bm);
      auto with_qcache = [&](KPParams& P) {
        if (!T->qcache[b]) return;
        P.qcache = T->qcache[b];
        P.qfam = T->d_qfam[b];
        P.qfam_n = (int)T->qfam[b].size();
        if (!P.el) tag_quad_families(P.inl, P.n_elem, T->qfam[b].data(), P.qfam_n);
      };
      int L = 0;
      // prologue: the ps-dependent quantities, and the first deposit for lattices opening with a marker
      KPParams& P0 = descs[(size_t)L * nb + b];
      P0 = base_params(p, bm);
      P0.psc = T->psc[b];
      P0.psc_mode = 2;
      with_qcache(P0);
      if (!T->has_head && n_marks > 0) {
        bunch_deposit(B, b, P0);
        P0.cell = T->cell[b];
        P0.frac = T->frac[b];
        P0.fix = T->fix[b];
      }
      T->launch_cache[L] = P0.cell != nullptr;
      ++L;
      if (T->has_head) {
        KPParams& P = descs[(size_t)L * nb + b];
        P = base_params(p, bm);
        P.psc = T->psc[b];
        P.psc_mode = 1;
        const int nh = mk.empty() ? u.n_elems : mk[0];
        set_elements(P, u.lattice, nh, bm, T->d_elems[b]);
        with_qcache(P);
        P.psc_skip = psc_skip_mask(u.lattice, nh, bm, T->qfam[b].data(), (int)T->qfam[b].size());
        P.ps_mode = ps_mode_mask(u.lattice, nh, false);
        if (!mk.empty()) {
          bunch_deposit(B, b, P);
          P.cell = T->cell[b];
          P.frac = T->frac[b];
          P.fix = T->fix[b];
        }
        T->launch_cache[L] = P.cell != nullptr;
        ++L;
      }
      for (int k = 0; k < n_marks; ++k, ++L) {
        const int m = mk[k];
        const int end = (k + 1 < n_marks) ? mk[k + 1] : u.n_elems;
        const double prev = (k > 0) ? s[mk[k - 1]] : s[mk.back()] - circ;
        KPParams& P = descs[(size_t)L * nb + b];
        P = base_params(p, bm);
        P.psc = T->psc[b];
        P.psc_mode = 1;
        bunch_kick(B, b, P, K * (s[m] - prev));
        set_elements(P, u.lattice + m + 1, end - m - 1, bm, T->d_elems[b] + m + 1);
        with_qcache(P);
        P.psc_skip = psc_skip_mask(u.lattice + m + 1, end - m - 1, bm, T->qfam[b].data(), (int)T->qfam[b].size());
        P.ps_mode = ps_mode_mask(u.lattice + m + 1, end - m - 1, P.lon != 0);
        P.cell = T->cell[b];
        P.frac = T->frac[b];
        P.fix = T->fix[b];
        if ((k + 1 < n_marks) || !T->has_head) bunch_deposit(B, b, P);
        T->launch_cache[L] = 1;
      }
    }
    for (int L = 0; L < T->n_launches; ++L)
      for (int b = 0; b < nb; ++b)
        if (descs[(size_t)L * nb + b].has_xe || descs[(size_t)L * nb + b].bezier) T->launch_xe[L] = 1;
    SC_CUDA(cudaMalloc(&T->d_descs, descs.size() * sizeof(KPParams)));
    SC_CUDA(cudaMemcpy(T->d_descs, descs.data(), descs.size() * sizeof(KPParams), cudaMemcpyHostToDevice));
    if (B->trace) {
      T->ev.resize(3 * (size_t)n_marks);
      for (auto& e : T->ev) SC_CUDA(cudaEventCreate(&e));
    }
    if (want_diag) {
      SC_CUDA(cudaMalloc(&T->partial, (size_t)moments_blocks() * 14 * sizeof(double)));
      SC_CUDA(cudaMalloc(&T->d_base, (size_t)nb * sizeof(double*)));
      SC_CUDA(cudaMalloc(&T->d_turn, (size_t)nb * sizeof(int)));
    }
    for (sc_grid* g : B->cls) g->n_particles = 1;  // normalisation comes from stack_scale

    // ---- the turn (or its first `kicks` space-charge steps) as a graph -----------
    cudaStream_t S = B->stream;
    auto capture = [&](const KPParams* d_descs, const int4* d_blocks, int n_blocks, int kicks, bool full,
                       cudaGraph_t* graph) -> sc_status {
      SC_CUDA(cudaStreamBeginCapture(S, cudaStreamCaptureModeThreadLocal));
      sc_status cst = SC_OK;
      const bool diag_on = full && want_diag, trace_on = full && B->trace;
      for (int b = 0; !cst && diag_on && b < nb; ++b)
        if (bunches[b].particles.n > 0)
          cst = launch_moments(&bunches[b].particles, T->partial, moments_blocks(), T->d_base + b, T->d_turn + b,
                               14 * nb, S);
      int L = 1;
      const bool any = n_blocks > 0;  // some bunch holds particles
      if (T->has_head) {
        if (!cst && any)
          cst = launch_kick_push_batched(d_descs + (size_t)L * nb, d_blocks, n_blocks, T->tile_cells, f32,
                                         T->launch_cache[L] != 0, T->launch_xe[L] != 0, S, T->kp_threads);
        ++L;
      }
      for (int k = 0; !cst && k < kicks; ++k, ++L) {
        if (trace_on && cudaEventRecordWithFlags(T->ev[3 * k], S, cudaEventRecordExternal) != cudaSuccess)
          cst = set_error(SC_ERR_CUDA, "event");
        // every class: solve, then clear the charge for this marker's deposit; classes after the
        // first on their side streams (forked after the previous kick/push, joined before the next)
        if (!cst && B->cls.size() > 1 && cudaEventRecord(B->fork_ev, S) != cudaSuccess)
          cst = set_error(SC_ERR_CUDA, "fork event");
        for (size_t c = 1; !cst && c < B->cls.size(); ++c) {
          sc_grid* g = B->cls[c];
          if (cudaStreamWaitEvent(B->side[c - 1], B->fork_ev, 0) != cudaSuccess) {
            cst = set_error(SC_ERR_CUDA, "fork wait");
            break;
          }
          g->stream = B->side[c - 1];
          cst = solve_dispatch(g, true);
          g->stream = S;
          if (!cst && cudaEventRecord(B->join_ev[c - 1], B->side[c - 1]) != cudaSuccess)
            cst = set_error(SC_ERR_CUDA, "join event");
        }
        if (!cst) cst = solve_dispatch(B->cls[0], true);
        for (size_t c = 1; !cst && c < B->cls.size(); ++c)
          if (cudaStreamWaitEvent(S, B->join_ev[c - 1], 0) != cudaSuccess) cst = set_error(SC_ERR_CUDA, "join wait");
        if (!cst && trace_on && cudaEventRecordWithFlags(T->ev[3 * k + 1], S, cudaEventRecordExternal) != cudaSuccess)
          cst = set_error(SC_ERR_CUDA, "event");
        if (!cst && any)
          cst = launch_kick_push_batched(d_descs + (size_t)L * nb, d_blocks, n_blocks, T->tile_cells, f32,
                                         T->launch_cache[L] != 0, T->launch_xe[L] != 0, S, T->kp_threads);
        if (!cst && trace_on && cudaEventRecordWithFlags(T->ev[3 * k + 2], S, cudaEventRecordExternal) != cudaSuccess)
          cst = set_error(SC_ERR_CUDA, "event");
      }
      cudaGraph_t gr = nullptr;
      const cudaError_t ce = cudaStreamEndCapture(S, &gr);
      if (!cst && ce != cudaSuccess) cst = cuda_error(ce, "cudaStreamEndCapture");
      if (cst) {
        if (gr) cudaGraphDestroy(gr);
        return cst;
      }
      *graph = gr;
      return SC_OK;
    };
    auto set_blocks = [&](int waves, std::vector<int4>& blocks) {
      blocks = partition(counts, kick_push_batched_resident(T->tile_cells * 8, f32, true, T->kp_threads), waves);
    };
    auto fail = [&](sc_status e) {
      destroy_batch_plan(T);
      B->plan = nullptr;
      return e;
    };
    // ---- launch shape of the batched kick/push (block size, waves) -----------------
    int64_t total = 0;
    for (int64_t v : counts) total += v;
    T->kp_threads = B->kp_threads_set;
    T->kp_waves = B->kp_waves_set > 0 ? B->kp_waves_set : kWaves;
    const bool free_shape = B->kp_threads_set == 0 || B->kp_waves_set == 0;
    if (n_marks > 0 && total >= kShapeTuneMin && free_shape) {
      if (B->tuned_key == shape_key) {
        T->kp_threads = B->tuned_threads;
        T->kp_waves = B->tuned_waves;
        T->trial_us = B->tuned_us;
      } else {
        const sc_status tst = tune_batch_shape(B, T, bunches, counts, descs, capture, set_blocks);
        if (tst) return fail(tst);
        B->tuned_key = shape_key;
        B->tuned_threads = T->kp_threads;
        B->tuned_waves = T->kp_waves;
        B->tuned_us = T->trial_us;
      }
    }
    {
      std::vector<int4> blocks;
      set_blocks(T->kp_waves, blocks);
      T->n_blocks = (int)blocks.size();
      if (T->n_blocks > 0) {
        cudaError_t e = cudaMalloc(&T->d_blocks, blocks.size() * sizeof(int4));
        if (e == cudaSuccess)
          e = cudaMemcpy(T->d_blocks, blocks.data(), blocks.size() * sizeof(int4), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return fail(cuda_error(e, "block table"));
      }
    }
    // ---- capture one turn of every bunch -----------------------------------------
    cudaGraph_t graph = nullptr;
    if ((st = capture(T->d_descs, T->d_blocks, T->n_blocks, n_marks, true, &graph))) return fail(st);
    T->graph = graph;
    const cudaError_t ce = cudaGraphInstantiate(&T->exec, graph, 0);
    if (ce != cudaSuccess) return fail(cuda_error(ce, "cudaGraphInstantiate"));
    T->key = key;  // complete: a plan left half-built by an error is rebuilt by the next call
  }

  // ---- run -------------------------------------------------------------------------
  cudaStream_t S = B->stream;
  if (T->diag) {
    if (n_turns > T->diag_cap) {
      SC_CUDA(cudaStreamSynchronize(S));
      cudaFree(T->d_diag);
      T->d_diag = nullptr;
      SC_CUDA(cudaMalloc(&T->d_diag, (size_t)n_turns * nb * 14 * sizeof(double)));
      T->diag_cap = n_turns;
    }
    std::vector<double*> base(nb);
    for (int b = 0; b < nb; ++b) base[b] = T->d_diag + (size_t)14 * b;
    SC_CUDA(cudaMemcpy(T->d_base, base.data(), nb * sizeof(double*), cudaMemcpyHostToDevice));
    SC_CUDA(cudaMemsetAsync(T->d_turn, 0, nb * sizeof(int), S));
    SC_CUDA(cudaMemsetAsync(T->d_diag, 0, (size_t)n_turns * nb * 14 * sizeof(double), S));
  }
  if (T->n_blocks > 0) {
    if (!T->has_head && T->n_kicks > 0)
      for (sc_grid* g : B->cls) SC_CUDA(cudaMemsetAsync(g->Q, 0, cells_of(g) * g->nstack * 8, S));
    if ((st = launch_kick_push_batched(T->d_descs, T->d_blocks, T->n_blocks, T->tile_cells, f32,
                                       T->launch_cache[0] != 0, T->launch_xe[0] != 0, S, T->kp_threads)))
      return st;
  }
  for (int t = 0; t < n_turns; ++t) {
    SC_CUDA(cudaGraphLaunch(T->exec, S));
    if (!T->ev.empty()) {
      SC_CUDA(cudaStreamSynchronize(S));
      for (size_t k = 0; 3 * k + 2 < T->ev.size(); ++k) {
        float a = 0.f, c = 0.f;
        SC_CUDA(cudaEventElapsedTime(&a, T->ev[3 * k], T->ev[3 * k + 1]));
        SC_CUDA(cudaEventElapsedTime(&c, T->ev[3 * k + 1], T->ev[3 * k + 2]));
        B->trace_solve_ms += a;
        B->trace_kp_ms += c;
        B->trace_kicks += 1;
      }
    }
  }
  if (T->diag) {
    SC_CUDA(cudaMemcpyAsync(diag, T->d_diag, (size_t)n_turns * nb * 14 * sizeof(double), cudaMemcpyDeviceToHost, S));
    SC_CUDA(cudaStreamSynchronize(S));
    // a non-finite coordinate of any particle makes its bunch's moments of that turn non-finite
    for (size_t k = 0; k < (size_t)n_turns * nb * 14; ++k)
      if (!std::isfinite(diag[k]))
        return set_error(SC_ERR_NAN, "non-finite particle coordinates in bunch " + std::to_string((k / 14) % nb));
  }
  return SC_OK;
}

sc_status sc_batch_read(sc_batch* B, int b, uint64_t* Q, double* Ex, double* Ey, int64_t* n_out) {
  if (!B) return set_error(SC_ERR_ARG, "batch is NULL");
  if (b < 0 || b >= B->n_bunches) return set_error(SC_ERR_ARG, "bunch index out of range");
  SC_CUDA(cudaStreamSynchronize(B->stream));
  sc_grid* g = B->cls[B->cls_of[b]];
  const size_t cells = cells_of(g), off = (size_t)B->idx[b] * cells;
  if (Q) SC_CUDA(cudaMemcpy(Q, g->Q + off, cells * 8, cudaMemcpyDeviceToHost));
  if ((Ex || Ey) && g->field32) {
    std::vector<float2> E(cells);
    SC_CUDA(cudaMemcpy(E.data(), (const float2*)g->E + off, cells * sizeof(float2), cudaMemcpyDeviceToHost));
    for (size_t c = 0; c < cells; ++c) {
      if (Ex) Ex[c] = E[c].x;
      if (Ey) Ey[c] = E[c].y;
    }
  } else if (Ex || Ey) {
    std::vector<double2> E(cells);
    SC_CUDA(cudaMemcpy(E.data(), g->E + off, cells * sizeof(double2), cudaMemcpyDeviceToHost));
    for (size_t c = 0; c < cells; ++c) {
      if (Ex) Ex[c] = E[c].x;
      if (Ey) Ey[c] = E[c].y;
    }
  }
  if (n_out) {
    unsigned long long v = 0;
    SC_CUDA(cudaMemcpy(&v, g->n_out + B->idx[b], 8, cudaMemcpyDeviceToHost));
    *n_out = (int64_t)v;
  }
  sc_status first = SC_OK;
  for (sc_grid* c : B->cls) {
    const sc_status st = check_grid_errors(c);
    if (st && (!first || st == SC_ERR_TIMEOUT)) first = st;
  }
  return first;
}

sc_status sc_batch_get_solver_tiling(sc_batch* B, int b, int* choice, char* desc, size_t n) {
  if (!B) return set_error(SC_ERR_ARG, "batch is NULL");
  if (b < 0 || b >= B->n_bunches) return set_error(SC_ERR_ARG, "bunch index out of range");
  return sc_get_solver_tiling(B->cls[B->cls_of[b]], choice, desc, n);
}

sc_status sc_batch_set_solver_tiling(sc_batch* B, const int* choice) {
  if (!B || !choice) return set_error(SC_ERR_ARG, "batch or choice is NULL");
  SC_CUDA(cudaStreamSynchronize(B->stream));
  destroy_batch_plan(B->plan);  // captured turns hold the old launches
  B->plan = nullptr;
  for (sc_grid* g : B->cls) {
    sc_status st = sc_set_solver_tiling(g, choice);
    if (st) return st;
  }
  return SC_OK;
}

sc_status sc_batch_trace_enable(sc_batch* B, int enable) {
  if (!B) return set_error(SC_ERR_ARG, "batch is NULL");
  B->trace = enable ? 1 : 0;
  B->trace_kp_ms = B->trace_solve_ms = 0.0;
  B->trace_kicks = 0;
  return SC_OK;
}

sc_status sc_batch_trace_read(sc_batch* B, double* kick_push_ms, double* solve_ms, int64_t* n_kicks) {
  if (!B) return set_error(SC_ERR_ARG, "batch is NULL");
  if (kick_push_ms) *kick_push_ms = B->trace_kp_ms;
  if (solve_ms) *solve_ms = B->trace_solve_ms;
  if (n_kicks) *n_kicks = B->trace_kicks;
  B->trace_kp_ms = B->trace_solve_ms = 0.0;
  B->trace_kicks = 0;
  return SC_OK;
}

}  // extern "C"
