// Beam moments for the per-turn diagnostics (Sec. V: rms sizes -> beta,
// emittances), in two passes over the particles as the definition reads: the
// means first, then the central second moments of the particles' offsets from
// them (no E[x^2] - E[x]^2 cancellation for a bunch far off the axis).  A fixed
// grid reduces the float64 sums in the same order every time (deterministic).
#include <atomic>
#include <cuda.h>

#include "sc_internal.cuh"

namespace sc {

namespace {

constexpr int kMomThreads = 256;
constexpr int kMomBlocks = 304;  // fixed: 2 per SM on a 152-SM GB300
constexpr int kNM = 14;          // 6 means + 8 central second moments

// Block-wide sums of v[0..C) into partial[blockIdx.x * kNM + off + c].
template <int C>
__device__ __forceinline__ void block_sums(double (&v)[C], double* __restrict__ partial, int off) {
  __shared__ double red[kMomThreads / 32][C];
#pragma unroll
  for (int c = 0; c < C; ++c) {
    double w = v[c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5][c] = w;
  }
  __syncthreads();
  if (threadIdx.x < C) {
    double w = 0.0;
    for (int k = 0; k < kMomThreads / 32; ++k) w += red[k][threadIdx.x];
    partial[(size_t)blockIdx.x * kNM + off + threadIdx.x] = w;
  }
}

// The six means from the first pass's block sums, in a fixed order (every
// caller gets the same bits).
__device__ __forceinline__ void means_of(const double* __restrict__ partial, int n_blocks, int64_t n, double (&m)[6]) {
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    double v = 0.0;
    for (int b = 0; b < n_blocks; ++b) v += partial[(size_t)b * kNM + c];
    m[c] = v / (double)n;
  }
}

// Pass 1: per-block sums of x, px, y, py, sigma, psigma -> partial[b][0..6).
__global__ void __launch_bounds__(kMomThreads) moments_sums(const double* __restrict__ x, const double* __restrict__ px,
                                                            const double* __restrict__ y, const double* __restrict__ py,
                                                            const double* __restrict__ sg,
                                                            const double* __restrict__ ps, int64_t n,
                                                            double* __restrict__ partial) {
  double s[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += stride) {
    s[0] += x[p];
    s[1] += px[p];
    s[2] += y[p];
    s[3] += py[p];
    s[4] += sg[p];
    s[5] += ps[p];
  }
  block_sums<6>(s, partial, 0);
}

// Pass 2: per-block sums of the products of the offsets from the means
// (xx, x px, px px, yy, y py, py py, sigma sigma, psigma psigma) -> partial[b][6..14).
// Every block derives the means from pass 1's sums itself.
__global__ void __launch_bounds__(kMomThreads) moments_central(const double* __restrict__ x,
                                                               const double* __restrict__ px,
                                                               const double* __restrict__ y,
                                                               const double* __restrict__ py,
                                                               const double* __restrict__ sg,
                                                               const double* __restrict__ ps, int64_t n,
                                                               double* __restrict__ partial) {
  __shared__ double mean_s[6];
  if (threadIdx.x == 0) {
    double m[6];
    means_of(partial, gridDim.x, n, m);
#pragma unroll
    for (int c = 0; c < 6; ++c) mean_s[c] = m[c];
  }
  __syncthreads();
  const double m0 = mean_s[0], m1 = mean_s[1], m2 = mean_s[2], m3 = mean_s[3], m4 = mean_s[4], m5 = mean_s[5];
  double s[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += stride) {
    const double a = x[p] - m0, b = px[p] - m1, c = y[p] - m2, d = py[p] - m3, e = sg[p] - m4, f = ps[p] - m5;
    s[0] += a * a;
    s[1] += a * b;
    s[2] += b * b;
    s[3] += c * c;
    s[4] += c * d;
    s[5] += d * d;
    s[6] += e * e;
    s[7] += f * f;
  }
  block_sums<8>(s, partial, 6);
}

// The 14 moments from both passes' block sums into out.
__device__ __forceinline__ void moments_store(const double* __restrict__ partial, int n_blocks, int64_t n,
                                              double* out) {
  __shared__ double tot[kNM];
  if (threadIdx.x < kNM - 6) {
    double v = 0.0;
    for (int b = 0; b < n_blocks; ++b) v += partial[(size_t)b * kNM + 6 + threadIdx.x];
    tot[6 + threadIdx.x] = v / (double)n;
  }
  if (threadIdx.x == 31) {
    double m[6];
    means_of(partial, n_blocks, n, m);
    for (int c = 0; c < 6; ++c) tot[c] = m[c];
  }
  __syncthreads();
  if (threadIdx.x < kNM) out[threadIdx.x] = tot[threadIdx.x];
}

// out = base_ptr[0] + stride * (*turn) receives the 14 moments; bumps *turn.
__global__ void moments_final(const double* __restrict__ partial, int n_blocks, int64_t n, double* const* base_ptr,
                              int* turn, int stride) {
  double* out = *base_ptr + (size_t)stride * (*turn);
  moments_store(partial, n_blocks, n, out);
  __syncthreads();
  if (threadIdx.x == 0) *turn += 1;
}

}  // namespace

int moments_blocks() { return kMomBlocks; }

// Per-particle betatron phase, Sec. V (tunes as the one-turn phase advance):
// in normalised coordinates of the bare Twiss (beta, alpha) at the turn start,
// U = u / sqrt(beta), PU = (alpha u + beta pu) / sqrt(beta), the phase is
// atan2(-PU, U).  acc (4 arrays of n): previous phase x, previous phase y,
// accumulated advance x, accumulated advance y; each call adds
// (phase - previous) mod 2 pi when `accumulate`, and stores the phase.
__global__ void phase_advance(const double* __restrict__ x, const double* __restrict__ px,
                              const double* __restrict__ y, const double* __restrict__ py, int64_t n, double bx,
                              double ax, double by, double ay, double* acc, int accumulate) {
  const double rbx = rsqrt(bx), rby = rsqrt(by);
  const double two_pi = 6.283185307179586;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    const double tx = atan2(-(ax * x[p] + bx * px[p]) * rbx, x[p] * rbx);
    const double ty = atan2(-(ay * y[p] + by * py[p]) * rby, y[p] * rby);
    if (accumulate) {
      double dx = fmod(tx - acc[p], two_pi), dy = fmod(ty - acc[n + p], two_pi);
      if (dx < 0.0) dx += two_pi;
      if (dy < 0.0) dy += two_pi;
      acc[2 * n + p] += dx;
      acc[3 * n + p] += dy;
    }
    acc[p] = tx;
    acc[n + p] = ty;
  }
}

sc_status launch_phase_advance(const sc_particles* p, const double* twiss, double* acc, int accumulate,
                               cudaStream_t s) {
  phase_advance<<<kMomBlocks, kMomThreads, 0, s>>>(p->x, p->px, p->y, p->py, p->n, twiss[0], twiss[1], twiss[2],
                                                   twiss[3], acc, accumulate);
  SC_CUDA(cudaGetLastError());
  return SC_OK;
}

// Fractional tunes from the accumulated advances: q[p] = acc[2n + p] / (2 pi T)
// (x), q[n + p] = acc[3n + p] / (2 pi T) (y).
__global__ void tunes_from_advances(const double* __restrict__ acc, int64_t n, double inv_two_pi_turns,
                                    double* __restrict__ q) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < 2 * n; p += (int64_t)gridDim.x * blockDim.x)
    q[p] = acc[2 * n + p] * inv_two_pi_turns;
}

sc_status launch_moments(const sc_particles* p, double* partial, int n_blocks, double* const* base_ptr, int* turn,
                         int stride, cudaStream_t s) {
  moments_sums<<<n_blocks, kMomThreads, 0, s>>>(p->x, p->px, p->y, p->py, p->sigma, p->psigma, p->n, partial);
  moments_central<<<n_blocks, kMomThreads, 0, s>>>(p->x, p->px, p->y, p->py, p->sigma, p->psigma, p->n, partial);
  moments_final<<<1, 32, 0, s>>>(partial, n_blocks, p->n, base_ptr, turn, stride);
  SC_CUDA(cudaGetLastError());
  return SC_OK;
}

}  // namespace sc

// ---------------------------------------------------------------------------
// Beam moments without any device allocation.
//
// For callers that cannot allocate device memory while they run: code inside
// a memory pool or arena that owns all of the device's memory, code running in
// a process whose allocator must not be re-entered (callbacks, signal-driven
// monitors), or a real-time loop where cudaMalloc/cudaFree (which can
// synchronise the device) are not allowed.  The block partial sums live in a
// file-scope device array instead of a caller- or library-allocated buffer.
//
// Every GPU that loads the library's device code holds the array (34 KB) until
// the process exits.  The first call on a device (and the first after the
// device's context was reset) looks up its device address
// (cudaGetSymbolAddress) with that device current; make that first call
// before any stream capture.  Every call writes all kMomBlocks partial rows of
// both passes before they are read, so nothing needs clearing between calls;
// calls that overlap on the GPU (different streams, or different host threads
// on the same device) share the array and race.
// ---------------------------------------------------------------------------
namespace sc {
namespace {

constexpr int kMaxDevices = 64;
static __device__ __align__(256) double g_noalloc_partial[kMomBlocks * kNM];

__global__ void moments_final_to(const double* __restrict__ partial, int n_blocks, int64_t n, double* out) {
  moments_store(partial, n_blocks, n, out);
}

// Per device ordinal: the address of g_noalloc_partial and the id of the
// context it was looked up in (a context created after cudaDeviceReset loads
// the module again, possibly elsewhere, and has a new id).
struct NoallocSlot {
  std::atomic<unsigned long long> ctx_id{0};
  std::atomic<double*> addr{nullptr};
};
NoallocSlot g_noalloc[kMaxDevices];

using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);

// Id of the current context (0 when it cannot be read: the address is then looked up every call).
unsigned long long current_context_id() {
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  static std::atomic<int> looked{0};
  if (!looked.load()) {
    cudaDriverEntryPointQueryResult q;
    void* f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = (CtxGetCurrentFn)f;
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = (CtxGetIdFn)f;
    looked.store(1);
  }
  CUcontext c = nullptr;
  unsigned long long id = 0;
  if (!get_current || !get_id || get_current(&c) != CUDA_SUCCESS || !c || get_id(c, &id) != CUDA_SUCCESS) return 0;
  return id;
}

// Device address of g_noalloc_partial in the current device's current context.
sc_status noalloc_scratch(double** out) {
  int dev = 0;
  SC_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return set_error(SC_ERR_UNSUPPORTED, "device ordinal beyond 63");
  NoallocSlot& slot = g_noalloc[dev];
  double* a = slot.addr.load();
  const unsigned long long id = current_context_id();  // 0 before the runtime made a context current
  if (!a || id == 0 || slot.ctx_id.load() != id) {
    // the lookup makes the device's primary context current; the id is read again after it
    SC_CUDA(cudaGetSymbolAddress((void**)&a, g_noalloc_partial));
    slot.addr.store(a);
    slot.ctx_id.store(current_context_id());
  }
  *out = a;
  return SC_OK;
}

}  // namespace
}  // namespace sc

extern "C" sc_status sc_moments_noalloc(const sc_particles* p, double* out, void* stream) {
  using namespace sc;
  if (!p || !out) return set_error(SC_ERR_ARG, "particles or out is NULL");
  if (p->n <= 0) return set_error(SC_ERR_ARG, "sc_moments_noalloc needs at least one particle");
  if (p->n > SC_MOMENTS_NOALLOC_MAX_N)
    return set_error(SC_ERR_OVERFLOW, "sc_moments_noalloc: more than SC_MOMENTS_NOALLOC_MAX_N particles");
  if (!p->x || !p->px || !p->y || !p->py || !p->sigma || !p->psigma)
    return set_error(SC_ERR_ARG, "particle array pointer is NULL");
  double* scratch = nullptr;
  sc_status st = noalloc_scratch(&scratch);
  if (st) return st;
  cudaStream_t s = (cudaStream_t)stream;
  moments_sums<<<kMomBlocks, kMomThreads, 0, s>>>(p->x, p->px, p->y, p->py, p->sigma, p->psigma, p->n, scratch);
  moments_central<<<kMomBlocks, kMomThreads, 0, s>>>(p->x, p->px, p->y, p->py, p->sigma, p->psigma, p->n, scratch);
  moments_final_to<<<1, 32, 0, s>>>(scratch, kMomBlocks, p->n, out);
  SC_CUDA(cudaGetLastError());
  return SC_OK;
}

extern "C" sc_status sc_tunes(const double* acc, int64_t n, int n_turns, double* q, void* stream) {
  using namespace sc;
  if (!acc || !q) return set_error(SC_ERR_ARG, "acc or q is NULL");
  if (n < 0 || n_turns <= 0) return set_error(SC_ERR_ARG, "sc_tunes needs n >= 0 and n_turns > 0");
  if (n == 0) return SC_OK;
  const double two_pi = 6.283185307179586;
  tunes_from_advances<<<kMomBlocks, kMomThreads, 0, (cudaStream_t)stream>>>(acc, n, 1.0 / (two_pi * n_turns), q);
  SC_CUDA(cudaGetLastError());
  return SC_OK;
}
