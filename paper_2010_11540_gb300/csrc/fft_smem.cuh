// Radix-2 Stockham FFT in shared memory, float64, shared by the float64
// solves (open boundary and conducting pipe).
#pragma once

#include "sc_internal.cuh"

namespace sc {

// Radix-2 Stockham FFT of length M in shared memory, blockDim.x == M/2.
// tw[t] = exp(-2 pi i t / M), t < M/2; INV uses the conjugate.  Returns the
// buffer that holds the result (a or b).  Caller synchronises before.
template <bool INV>
__device__ double2* fft_smem(double2* a, double2* b, int M, const double2* __restrict__ tw) {
  const int half = M >> 1;
  const int j = threadIdx.x;
  for (int Ns = 1; Ns < M; Ns <<= 1) {
    const int k = j & (Ns - 1);
    const double2 v0 = a[j], v1 = a[j + half];
    double2 w = __ldg(tw + k * (half / Ns));
    if (INV) w.y = -w.y;
    const double tx = v1.x * w.x - v1.y * w.y;
    const double ty = v1.x * w.y + v1.y * w.x;
    const int idx = ((j - k) << 1) + k;
    b[idx] = make_double2(v0.x + tx, v0.y + ty);
    b[idx + Ns] = make_double2(v0.x - tx, v0.y - ty);
    __syncthreads();
    double2* t = a;
    a = b;
    b = t;
  }
  return a;
}

}  // namespace sc
