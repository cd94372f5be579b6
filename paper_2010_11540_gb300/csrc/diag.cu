// Beam moments for the per-turn diagnostics (Sec. V: rms sizes -> beta,
// emittances).  Two launches with a fixed grid so that the float64 sums are
// reduced in the same order every time (deterministic).
#include <atomic>

#include "sc_internal.cuh"

namespace sc {

namespace {

constexpr int kMomThreads = 256;
constexpr int kMomBlocks = 304;  // fixed: 2 per SM on a 152-SM GB300
constexpr int kNM = 14;

__global__ void __launch_bounds__(kMomThreads) moments_partial(const double* __restrict__ x,
                                                                const double* __restrict__ px,
                                                                const double* __restrict__ y,
                                                                const double* __restrict__ py,
                                                                const double* __restrict__ sg,
                                                                const double* __restrict__ ps, int64_t n,
                                                                double* __restrict__ partial) {
  double s[kNM];
#pragma unroll
  for (int c = 0; c < kNM; ++c) s[c] = 0.0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += stride) {
    const double a = x[p], b = px[p], c = y[p], d = py[p], e = sg[p], f = ps[p];
    s[0] += a; s[1] += b; s[2] += c; s[3] += d; s[4] += e; s[5] += f;
    s[6] += a * a; s[7] += a * b; s[8] += b * b;
    s[9] += c * c; s[10] += c * d; s[11] += d * d;
    s[12] += e * e; s[13] += f * f;
  }
  __shared__ double red[kMomThreads / 32][kNM];
#pragma unroll
  for (int c = 0; c < kNM; ++c) {
    double v = s[c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5][c] = v;
  }
  __syncthreads();
  if (threadIdx.x < kNM) {
    double v = 0.0;
    for (int w = 0; w < kMomThreads / 32; ++w) v += red[w][threadIdx.x];
    partial[(size_t)blockIdx.x * kNM + threadIdx.x] = v;
  }
}

// out = base_ptr[0] + stride * (*turn): means, then central second moments; bumps *turn.
__global__ void moments_final(const double* __restrict__ partial, int n_blocks, int64_t n, double* const* base_ptr,
                              int* turn, int stride) {
  __shared__ double tot[kNM];
  if (threadIdx.x < kNM) {
    double v = 0.0;
    for (int b = 0; b < n_blocks; ++b) v += partial[(size_t)b * kNM + threadIdx.x];
    tot[threadIdx.x] = v / (double)n;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double* out = *base_ptr + (size_t)stride * (*turn);
    const double* m = tot;
    for (int c = 0; c < 6; ++c) out[c] = m[c];
    out[6] = m[6] - m[0] * m[0];
    out[7] = m[7] - m[0] * m[1];
    out[8] = m[8] - m[1] * m[1];
    out[9] = m[9] - m[2] * m[2];
    out[10] = m[10] - m[2] * m[3];
    out[11] = m[11] - m[3] * m[3];
    out[12] = m[12] - m[4] * m[4];
    out[13] = m[13] - m[5] * m[5];
    *turn += 1;
  }
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

sc_status launch_moments(const sc_particles* p, double* partial, int n_blocks, double* const* base_ptr, int* turn,
                         int stride, cudaStream_t s) {
  moments_partial<<<n_blocks, kMomThreads, 0, s>>>(p->x, p->px, p->y, p->py, p->sigma, p->psigma, p->n, partial);
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
// the process exits.  The first call on a device looks up its device
// address (cudaGetSymbolAddress) with that device current; make that first
// call before any stream capture.  Every call writes all kMomBlocks partial
// rows before they are read, so nothing needs clearing between calls; calls
// that overlap on the GPU (different streams, or different host threads on the
// same device) share the array and race.
// ---------------------------------------------------------------------------
namespace sc {
namespace {

constexpr int kMaxDevices = 64;
static __device__ __align__(256) double g_noalloc_partial[kMomBlocks * kNM];

__global__ void moments_final_to(const double* __restrict__ partial, int n_blocks, int64_t n, double* out) {
  __shared__ double tot[kNM];
  if (threadIdx.x < kNM) {
    double v = 0.0;
    for (int b = 0; b < n_blocks; ++b) v += partial[(size_t)b * kNM + threadIdx.x];
    tot[threadIdx.x] = v / (double)n;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const double* m = tot;
    for (int c = 0; c < 6; ++c) out[c] = m[c];
    out[6] = m[6] - m[0] * m[0];
    out[7] = m[7] - m[0] * m[1];
    out[8] = m[8] - m[1] * m[1];
    out[9] = m[9] - m[2] * m[2];
    out[10] = m[10] - m[2] * m[3];
    out[11] = m[11] - m[3] * m[3];
    out[12] = m[12] - m[4] * m[4];
    out[13] = m[13] - m[5] * m[5];
  }
}

std::atomic<double*> g_noalloc_addr[kMaxDevices];

// Device address of g_noalloc_partial on the current device (looked up once).
sc_status noalloc_scratch(double** out) {
  int dev = 0;
  SC_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return set_error(SC_ERR_UNSUPPORTED, "device ordinal beyond 63");
  double* a = g_noalloc_addr[dev].load();
  if (!a) {
    SC_CUDA(cudaGetSymbolAddress((void**)&a, g_noalloc_partial));
    g_noalloc_addr[dev].store(a);
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
  moments_partial<<<kMomBlocks, kMomThreads, 0, s>>>(p->x, p->px, p->y, p->py, p->sigma, p->psigma, p->n, scratch);
  moments_final_to<<<1, 32, 0, s>>>(scratch, kMomBlocks, p->n, out);
  SC_CUDA(cudaGetLastError());
  return SC_OK;
}
