// Cloud-in-cell helpers for the deposit and the field gather (Sec. IV-A).
#pragma once

#include "sc_internal.cuh"

namespace sc {

// Cell and fractions of a particle: xi = (x - xmin) * inv_hx rounded twice
// (no fused multiply-add, so every platform takes the same integer decision),
// i = floor(xi), fx = xi - i (exact).  Inside iff 0 <= xi < nx-1 and
// 0 <= eta < ny-1; non-finite coordinates are outside.  The range test is
// done on the integer floor (0 <= i <= nx-2 is the same condition for finite
// xi; out-of-range values saturate), and finiteness on the exponent bits, so
// that only the subtract, multiply, floor-convert, back-convert and subtract
// of each axis use the FP64 pipe.  Returns the cell index j*nx+i or -1.
__device__ __forceinline__ int locate(const GridGeom& g, double x, double y, double& fx, double& fy) {
  const bool finite = ((__double2hiint(x) & 0x7ff00000) != 0x7ff00000) &&
                      ((__double2hiint(y) & 0x7ff00000) != 0x7ff00000);
  const double xi = __dmul_rn(__dsub_rn(x, g.xmin), g.inv_hx);
  const double eta = __dmul_rn(__dsub_rn(y, g.ymin), g.inv_hy);
  const int i = __double2int_rd(xi);
  const int j = __double2int_rd(eta);
  fx = __dsub_rn(xi, (double)i);
  fy = __dsub_rn(eta, (double)j);
  const bool inside = finite && (unsigned)i < (unsigned)(g.nx - 1) && (unsigned)j < (unsigned)(g.ny - 1);
  return inside ? j * g.nx + i : -1;
}

// The four CIC weights in 2^-20 fixed point per axis: a = rint(f 2^20)
// (round half to even), b = 2^20 - a; the products sum to exactly 2^40.
// dst is either a shared-memory tile or the global grid (same [j][i] layout).
// Returns the fixed-point fractions (ax, ay).
__device__ __forceinline__ int2 deposit4(unsigned long long* dst, int nx, int cell, double fx, double fy) {
  const long long ax = __double2ll_rn(__dmul_rn(fx, 1048576.0));
  const long long ay = __double2ll_rn(__dmul_rn(fy, 1048576.0));
  const long long bx = 1048576LL - ax, by = 1048576LL - ay;
  unsigned long long* q = dst + cell;
  atomicAdd(q, (unsigned long long)(bx * by));
  atomicAdd(q + 1, (unsigned long long)(ax * by));
  atomicAdd(q + nx, (unsigned long long)(bx * ay));
  atomicAdd(q + nx + 1, (unsigned long long)(ax * ay));
  return make_int2((int)ax, (int)ay);
}

// Zero a shared-memory tile of `cells` int64 bins (whole block).
__device__ __forceinline__ void tile_zero(unsigned long long* tile, int cells) {
  for (int c = threadIdx.x; c < cells; c += blockDim.x) tile[c] = 0ull;
}

// Add the non-zero bins of a block's tile into the global grid (whole block;
// caller synchronises before).  This is the only cross-block reduction of the
// deposit.
__device__ __forceinline__ void tile_flush(const unsigned long long* tile, unsigned long long* Q, int cells) {
  for (int c = threadIdx.x; c < cells; c += blockDim.x) {
    const unsigned long long v = tile[c];
    if (v) atomicAdd(Q + c, v);
  }
}

// Block-wide sum of per-thread out-of-grid counts into a global counter.
__device__ __forceinline__ void count_out(unsigned int out, unsigned long long* n_out) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) out += __shfl_xor_sync(0xffffffffu, out, o);
  if ((threadIdx.x & 31) == 0 && out) atomicAdd(n_out, (unsigned long long)out);
}

}  // namespace sc
