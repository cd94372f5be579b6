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
// With longitudinal slices the particle's slice k = floor((sg - zmin) *
// inv_dz) (same two roundings, 0 <= k < nz) selects the grid and the cell index
// is k*nx*ny + j*nx + i.
__device__ __forceinline__ int locate(const GridGeom& g, double x, double y, double sg, double& fx, double& fy) {
  bool finite = ((__double2hiint(x) & 0x7ff00000) != 0x7ff00000) &&
                ((__double2hiint(y) & 0x7ff00000) != 0x7ff00000);
  const double xi = __dmul_rn(__dsub_rn(x, g.xmin), g.inv_hx);
  const double eta = __dmul_rn(__dsub_rn(y, g.ymin), g.inv_hy);
  const int i = __double2int_rd(xi);
  const int j = __double2int_rd(eta);
  fx = __dsub_rn(xi, (double)i);
  fy = __dsub_rn(eta, (double)j);
  int k = 0;
  if (g.nz > 1) {
    finite = finite && ((__double2hiint(sg) & 0x7ff00000) != 0x7ff00000);
    k = __double2int_rd(__dmul_rn(__dsub_rn(sg, g.zmin), g.inv_dz));
    finite = finite && (unsigned)k < (unsigned)g.nz;
  }
  const bool inside = finite && (unsigned)i < (unsigned)(g.nx - 1) && (unsigned)j < (unsigned)(g.ny - 1);
  return inside ? (k * g.ny + j) * g.nx + i : -1;
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

// Deposit into a block's shared tile when the cell's slice is the tile's,
// else straight into the global grid.  The tile takes the slice of the first
// particle that reaches this (tile_k, shared, starts at -1).  Returns the
// fixed-point fractions.
__device__ __forceinline__ int2 deposit_tiled(unsigned long long* tile, int* tile_k, unsigned long long* Q,
                                              const GridGeom& g, int cell, double fx, double fy) {
  const int cells = g.nx * g.ny;
  const int k = cell / cells;
  int tk = *(volatile int*)tile_k;
  if (tk < 0) {
    const int prev = atomicCAS(tile_k, -1, k);
    tk = prev < 0 ? k : prev;
  }
  return (tk == k) ? deposit4(tile, g.nx, cell - k * cells, fx, fy) : deposit4(Q, g.nx, cell, fx, fy);
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
