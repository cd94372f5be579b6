// Cloud-in-cell helpers for the deposit and the field gather (Sec. IV-A).
#pragma once

#include "fixpt.h"
#include "sc_internal.cuh"

namespace sc {

// Cell, CIC weights and fractions of a particle: xi = (x - xmin) * inv_hx
// rounded twice (no fused multiply-add, so every platform takes the same
// integer decision), i = floor(xi), fixed-point weight a = rint((xi - i) 2^20)
// (ties to even) and, for FRAC, the float64 fraction fx = xi - i (exact); the
// same for eta.  Inside iff 0 <= xi < nx-1 and 0 <= eta < ny-1; non-finite
// coordinates are outside.  Only the subtract and multiply of each axis run on
// the FP64 pipe: floor, fraction and rounding are decoded from the bits of xi
// with integer instructions (cic_split, exact).  Returns the cell index
// j*nx+i or -1.  With longitudinal slices the particle's slice k =
// floor((sg - zmin) * inv_dz) (same two roundings, 0 <= k < nz) selects the
// grid and the cell index is k*nx*ny + j*nx + i.
template <bool FRAC>
__device__ __forceinline__ int locate(const GridGeom& g, double x, double y, double sg, int2& a, double& fx,
                                      double& fy, int& i, int& j, int& k) {
  const double xi = __dmul_rn(__dsub_rn(x, g.xmin), g.inv_hx);
  const double eta = __dmul_rn(__dsub_rn(y, g.ymin), g.inv_hy);
  i = 0;
  j = 0;
  k = 0;
  bool in = cic_split(xi, g.nx - 1, i, a.x, FRAC ? &fx : nullptr);
  in = cic_split(eta, g.ny - 1, j, a.y, FRAC ? &fy : nullptr) && in;
  if (g.nz > 1) in = floor_index(__dmul_rn(__dsub_rn(sg, g.zmin), g.inv_dz), g.nz, k) && in;
  return in ? (k * g.ny + j) * g.nx + i : -1;
}

template <bool FRAC>
__device__ __forceinline__ int locate(const GridGeom& g, double x, double y, double sg, int2& a, double& fx,
                                      double& fy, int& k) {
  int i, j;
  return locate<FRAC>(g, x, y, sg, a, fx, fy, i, j, k);
}

template <bool FRAC>
__device__ __forceinline__ int locate(const GridGeom& g, double x, double y, double sg, int2& a, double& fx,
                                      double& fy) {
  int k;
  return locate<FRAC>(g, x, y, sg, a, fx, fy, k);
}

// The four CIC weights in 2^-20 fixed point per axis: a (from locate), b =
// 2^20 - a; the products sum to exactly 2^40 (32 x 32 -> 64-bit multiplies).
// dst is either a shared-memory tile or the global grid (same [j][i] layout,
// row length nx).
__device__ __forceinline__ void deposit4(unsigned long long* dst, int nx, int cell, int2 a) {
  const unsigned ax = (unsigned)a.x, ay = (unsigned)a.y;
  const unsigned bx = 1048576u - ax, by = 1048576u - ay;
  unsigned long long* q = dst + cell;
  atomicAdd(q, (unsigned long long)bx * by);
  atomicAdd(q + 1, (unsigned long long)ax * by);
  atomicAdd(q + nx, (unsigned long long)bx * ay);
  atomicAdd(q + nx + 1, (unsigned long long)ax * ay);
}

// Deposit target of a particle in cell (i, j) of slice k (`cell` its global
// index, -1 outside): the block's tile when it holds slice k (the tile takes
// the slice of the first particle that asks, tile_k starting at -1) and the
// tile's window holds the cell's four nodes -- key = the cell's lower-left
// node in the tile -- else the global grid -- key = kGlobalKey | cell.  -1:
// nothing to deposit.
constexpr int kGlobalKey = 1 << 29;

// The tile holds the whole grid of an unsliced deposit: every cell's four
// nodes are in it at their own index (the common case, no key needed).
__device__ __forceinline__ bool tile_is_grid(const GridGeom& g) {
  return g.nz == 1 && g.wnx == g.nx && g.wny == g.ny;
}
__device__ __forceinline__ int deposit_key(bool use_tile, int* tile_k, const GridGeom& g, int cell, int i, int j,
                                           int k) {
  if (cell < 0) return -1;
  if (use_tile) {
    int tk = *(volatile int*)tile_k;
    if (tk < 0) {
      const int prev = atomicCAS(tile_k, -1, k);
      tk = prev < 0 ? k : prev;
    }
    const int li = i - g.wx0, lj = j - g.wy0;
    if (tk == k && (unsigned)li < (unsigned)(g.wnx - 1) && (unsigned)lj < (unsigned)(g.wny - 1))
      return lj * g.wnx + li;
  }
  return kGlobalKey | cell;
}

// The four CIC adds of one particle at its target key (deposit_key; -1: none).
__device__ __forceinline__ void deposit_at(int key, int2 a, unsigned long long* tile, int wnx, unsigned long long* Q,
                                           int nx) {
  if (key < 0) return;
  if (key & kGlobalKey)
    deposit4(Q, nx, key & (kGlobalKey - 1), a);
  else
    deposit4(tile, wnx, key, a);
}

// One warp's CIC deposits (Sec. IV-A), the lanes of `mask` calling together,
// each with its target key (deposit_key) and fixed-point weights a.  Lanes
// next to each other with the same key form a run (a bunch ordered by cell
// puts a warp's particles in one or two runs); a run's four node sums are
// formed in registers -- over the run, sum bx by = n 2^40 - 2^20 (Sax + Say)
// + Saxay, sum ax by = 2^20 Sax - Saxay, sum bx ay = 2^20 Say - Saxay, sum
// ax ay = Saxay, exact in 64-bit integers -- and its first lane issues the
// four atomic adds.  Integer sums do not depend on their order, so the grid
// gets the same bits as with one atomic per weight.  When no two neighbouring
// lanes share a key each lane adds its own.  (For particles in random order
// the test itself costs more than it saves: callers use deposit_at there.)
__device__ __forceinline__ void deposit_warp(unsigned mask, int key, int2 a, unsigned long long* tile, int wnx,
                                             unsigned long long* Q, int nx) {
  const int lane = threadIdx.x & 31;
  const int prev = __shfl_up_sync(mask, key, 1);
  const bool head = lane == 0 || !((mask >> (lane - 1)) & 1u) || prev != key;
  const unsigned heads = __ballot_sync(mask, head);
  if (heads == mask) {
    deposit_at(key, a, tile, wnx, Q, nx);
    return;
  }
  // suffix sums over each run by doubling: after the step of offset d, a lane
  // holds the sums of its run's lanes [lane, lane + 2d)
  unsigned sx = (unsigned)a.x, sy = (unsigned)a.y;
  unsigned long long sxy = (unsigned long long)sx * sy;
  const int rid = __popc(heads & ((2u << lane) - 1u));  // runs that start at or below this lane
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const unsigned ox = __shfl_down_sync(mask, sx, d);
    const unsigned oy = __shfl_down_sync(mask, sy, d);
    const unsigned long long oxy = __shfl_down_sync(mask, sxy, d);
    const int src = lane + d;
    if (src < 32 && ((mask >> src) & 1u) && __popc(heads & ((2u << src) - 1u)) == rid) {
      sx += ox;
      sy += oy;
      sxy += oxy;
    }
  }
  if (head && key >= 0) {
    // run length: the lanes of the mask from this one up to the next run's head
    const unsigned above = heads & ~((2u << lane) - 1u);
    const unsigned span = above ? ((1u << (__ffs(above) - 1)) - 1u) : 0xffffffffu;
    const unsigned long long n = (unsigned long long)__popc(mask & span & ~((1u << lane) - 1u));
    const unsigned long long one = 1048576ull;
    const unsigned long long w11 = sxy, w10 = one * sx - sxy, w01 = one * sy - sxy;
    const unsigned long long w00 = (n << 40) - one * ((unsigned long long)sx + sy) + sxy;
    const bool global = key & kGlobalKey;
    const int stride = global ? nx : wnx;
    unsigned long long* q = global ? Q + (key & (kGlobalKey - 1)) : tile + key;
    atomicAdd(q, w00);
    atomicAdd(q + 1, w10);
    atomicAdd(q + stride, w01);
    atomicAdd(q + stride + 1, w11);
  }
}

// Cubic Bernstein weights b_m(t) and their derivatives (R = double for the
// float64 form, float for the split form whose potential is float32).
template <typename R>
__device__ __forceinline__ void bernstein3(R t, R (&b)[4], R (&db)[4]) {
  const R u = R(1) - t, uu = u * u, tt = t * t, tu = t * u;
  b[0] = uu * u;
  b[1] = R(3) * tu * u;
  b[2] = R(3) * tu * t;
  b[3] = tt * t;
  db[0] = R(-3) * uu;
  db[1] = fma(R(3), uu, R(-6) * tu);
  db[2] = fma(R(6), tu, R(-3) * tt);
  db[3] = R(3) * tt;
}

// Potential of node (i, j) of one grid, i in -1..nx, j in -1..ny: beyond the
// walls the odd extension (u_{-1} = -u_1, u_n = -u_{n-2}).
template <typename R>
__device__ __forceinline__ R phi_node(const R* __restrict__ phi, int nx, int ny, int i, int j) {
  R sgn = R(1);
  if (i < 0) { i = -i; sgn = -sgn; }
  if (i > nx - 1) { i = 2 * (nx - 1) - i; sgn = -sgn; }
  if (j < 0) { j = -j; sgn = -sgn; }
  if (j > ny - 1) { j = 2 * (ny - 1) - j; sgn = -sgn; }
  return sgn * __ldg(phi + (size_t)j * nx + i);
}

// Bezier surface (Sec. IV-C) of grid phi in cell (i, j) at fractions (fx, fy):
// value u and the derivatives with respect to the cell fractions' span
// parameters (d/dx = gx / (3 hx), d/dy = gy / (3 hy)).
template <typename R, bool VALUE, bool GRAD>
__device__ __forceinline__ void bezier_eval(const R* __restrict__ phi, int nx, int ny, int i, int j, R fx, R fy,
                                            R& u, R& gx, R& gy) {
  R bx[4], dbx[4], by[4], dby[4];
  bernstein3<R>((R(1) + fx) * (R(1) / R(3)), bx, dbx);
  bernstein3<R>((R(1) + fy) * (R(1) / R(3)), by, dby);
  u = gx = gy = R(0);
#pragma unroll
  for (int n = 0; n < 4; ++n) {
    R rv = R(0), rx = R(0);
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const R c = phi_node<R>(phi, nx, ny, i + m - 1, j + n - 1);
      rv = fma(c, bx[m], rv);
      if (GRAD) rx = fma(c, dbx[m], rx);
    }
    if (VALUE) u = fma(rv, by[n], u);
    if (GRAD) {
      gx = fma(rx, by[n], gx);
      gy = fma(rv, dby[n], gy);
    }
  }
}

// Zero a shared-memory tile of `cells` int64 bins (whole block).
__device__ __forceinline__ void tile_zero(unsigned long long* tile, int cells) {
  for (int c = threadIdx.x; c < cells; c += blockDim.x) tile[c] = 0ull;
}

// Add the non-zero bins of a block's tile into the global grid Q (one
// slice; whole block; caller synchronises before): bin (li, lj) of the window
// is node (wx0 + li, wy0 + lj).  This is the only cross-block reduction of
// the deposit.
__device__ __forceinline__ void tile_flush(const unsigned long long* tile, unsigned long long* Q, const GridGeom& g) {
  const int cells = g.wnx * g.wny;
  if (g.wnx == g.nx && g.wny == g.ny) {  // the tile is the whole slice: same indices
    for (int c = threadIdx.x; c < cells; c += blockDim.x) {
      const unsigned long long v = tile[c];
      if (v) atomicAdd(Q + c, v);
    }
    return;
  }
  // a window: walk its bins with a running (row, column), no division per bin
  int lj = threadIdx.x / g.wnx, li = threadIdx.x - lj * g.wnx;
  const int step_j = blockDim.x / g.wnx, step_i = blockDim.x - step_j * g.wnx;
  for (int c = threadIdx.x; c < cells; c += blockDim.x) {
    const unsigned long long v = tile[c];
    if (v) atomicAdd(Q + (size_t)(g.wy0 + lj) * g.nx + g.wx0 + li, v);
    lj += step_j;
    li += step_i;
    if (li >= g.wnx) {
      li -= g.wnx;
      ++lj;
    }
  }
}

// A non-finite coordinate (NaN or infinity), tested on the bits: no FP64 instruction.
__device__ __forceinline__ bool nonfinite(double v) {
  return ((unsigned long long)__double_as_longlong(v) & 0x7ff0000000000000ull) == 0x7ff0000000000000ull;
}

// 1 for a particle whose position (or, on a sliced grid, its sigma) is not
// finite: bit tests only, for particles the deposit found outside grid g; the
// caller sums them in a register like the out-of-grid count (count_out).
__device__ __forceinline__ unsigned int nonfinite_state(const GridGeom& g, double x, double y, double sg) {
  return (unsigned int)(nonfinite(x) | nonfinite(y) | (g.nz > 1 && nonfinite(sg)));
}

// Block-wide sum of per-thread out-of-grid counts into a global counter.
__device__ __forceinline__ void count_out(unsigned int out, unsigned long long* n_out) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) out += __shfl_xor_sync(0xffffffffu, out, o);
  if ((threadIdx.x & 31) == 0 && out && n_out) atomicAdd(n_out, (unsigned long long)out);
}

}  // namespace sc
