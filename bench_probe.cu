// Machine probes for bench.py's roofline denominators (not part of libsc):
// the throughput of shared-memory 64-bit atomic adds (the unit of work of the
// CIC deposit, Sec. IV-A) and of FP64 fused multiply-adds (the FP64 pipe that
// bounds the transfer-map push, Sec. III), measured on the device in use.
// The kernels touch only their own shared memory / registers and one output
// word per block.  Built into libsc_probe.so beside bench.py.
#include <cuda_runtime.h>

namespace {

constexpr int kProbeThreads = 1024;
constexpr int kTable = 4096;  // 32 KB of u64 counters per block

// Each warp's 32 lanes add to 32 consecutive words (the fewest shared-memory
// wavefronts a 64-bit atomic can take), four independent adds per iteration.
__global__ void __launch_bounds__(kProbeThreads) probe_atomics_kernel(int iters, unsigned long long* sink) {
  __shared__ unsigned long long tab[kTable];
  for (int i = threadIdx.x; i < kTable; i += blockDim.x) tab[i] = 0ull;
  __syncthreads();
  const unsigned a = threadIdx.x;
  for (int it = 0; it < iters; ++it) {
    atomicAdd(&tab[a], 1ull);
    atomicAdd(&tab[a + 1024], 1ull);
    atomicAdd(&tab[a + 2048], 1ull);
    atomicAdd(&tab[a + 3072], 1ull);
  }
  __syncthreads();
  if (threadIdx.x == 0) sink[blockIdx.x] = tab[0] + tab[kTable - 1];
}

// Random cells of a 128 KB table (the deposit tile of a 128 x 128 grid):
// each thread walks its own linear congruential sequence of word indices.
constexpr int kRandTable = 16384;
__global__ void __launch_bounds__(kProbeThreads) probe_atomics_random_kernel(int iters, unsigned long long* sink) {
  extern __shared__ unsigned long long rtab[];
  for (int i = threadIdx.x; i < kRandTable; i += blockDim.x) rtab[i] = 0ull;
  __syncthreads();
  unsigned h = 2654435761u * (threadIdx.x + 1) + 97u * blockIdx.x;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      h = h * 1664525u + 1013904223u;
      atomicAdd(&rtab[h >> 18], 1ull);  // top 14 bits: 0 .. 16383
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) sink[blockIdx.x] = rtab[0] + rtab[kRandTable - 1];
}

// CH independent FMA chains per thread (enough to hide the pipe latency).
template <int CH>
__global__ void __launch_bounds__(256) probe_fp64_kernel(int iters, double* sink) {
  double x[CH];
#pragma unroll
  for (int k = 0; k < CH; ++k) x[k] = 1e-3 * (threadIdx.x + k);
  const double b = 0.999999, c = 1e-7 * (1 + blockIdx.x);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < CH; ++k) x[k] = fma(x[k], b, c);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < CH; ++k) s += x[k];
  if (s == 12345.678) sink[blockIdx.x] = s;  // never true: keeps the chains alive
}

template <class F>
int time_launches(F launch, cudaStream_t s, float* ms) {
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return -2;
  launch();  // warm-up
  cudaEventRecord(e0, s);
  for (int r = 0; r < 5; ++r) launch();
  cudaEventRecord(e1, s);
  cudaError_t e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
  if (e == cudaSuccess) e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return -2;
  *ms /= 5.f;
  return 0;
}

}  // namespace

// Throughput of conflict-free shared u64 atomics (each warp on 32 consecutive
// words), of shared u64 atomics on random words of a 128 KB table, and of FP64
// FMA instructions, per second on the current device, each timed over five
// launches on `stream` (synchronous).  Outputs may be NULL (not all).
// Returns 0, -1 (nothing asked) or -2 (a CUDA call failed).
extern "C" int scb_probe_peaks(double* shared_atomics_per_s, double* random_atomics_per_s, double* fp64_inst_per_s,
                               void* stream) {
  if (!shared_atomics_per_s && !random_atomics_per_s && !fp64_inst_per_s) return -1;
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return -2;
  const int blocks = 2 * sms;
  unsigned long long* sink = nullptr;
  if (cudaMalloc(&sink, (size_t)blocks * 8 * sizeof(unsigned long long)) != cudaSuccess) return -2;
  int st = 0;
  if (shared_atomics_per_s) {
    const int iters = 4096;
    float ms = 0.f;
    st = time_launches([&] { probe_atomics_kernel<<<blocks, kProbeThreads, 0, s>>>(iters, sink); }, s, &ms);
    if (!st) *shared_atomics_per_s = (double)blocks * kProbeThreads * iters * 4 / (ms * 1e-3);
  }
  if (!st && random_atomics_per_s) {
    const int iters = 1024;
    float ms = 0.f;
    if (cudaFuncSetAttribute(probe_atomics_random_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kRandTable * 8) != cudaSuccess)
      st = -2;
    if (!st)
      st = time_launches(
        [&] { probe_atomics_random_kernel<<<sms, kProbeThreads, kRandTable * 8, s>>>(iters, sink); }, s, &ms);
    if (!st) *random_atomics_per_s = (double)sms * kProbeThreads * iters * 4 / (ms * 1e-3);
  }
  if (!st && fp64_inst_per_s) {
    // best of two shapes: 8 chains x 8 blocks of 256 per SM, 16 chains x 4 blocks
    const int iters = 8192, threads = 256;
    float ms8 = 0.f, ms16 = 0.f;
    st = time_launches([&] { probe_fp64_kernel<8><<<8 * sms, threads, 0, s>>>(iters, (double*)sink); }, s, &ms8);
    if (!st)
      st = time_launches([&] { probe_fp64_kernel<16><<<4 * sms, threads, 0, s>>>(iters, (double*)sink); }, s,
                         &ms16);
    if (!st) {
      const double r8 = (double)8 * sms * threads * iters * 8 / (ms8 * 1e-3);
      const double r16 = (double)4 * sms * threads * iters * 16 / (ms16 * 1e-3);
      *fp64_inst_per_s = r8 > r16 ? r8 : r16;
    }
  }
  cudaFree(sink);
  return st;
}
