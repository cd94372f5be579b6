// Fused space-charge step for one location: field gather + kick (Sec. IV kick
// equation; bilinear node fields, or the Bezier surface of the potential, plus
// the longitudinal kick on sliced pipe grids), push through the segment's
// elements (Sec. III), and CIC deposit of the new positions (Sec. IV-A) into
// a per-block shared-memory uint64 tile (the grid, or its centred window)
// flushed once per block.  One thread per
// particle, persistent grid over SoA float64 state; one launch serves one grid
// (kick_push_kernel) or every bunch of a batch (kick_push_batched).
#include <cmath>
#include <cstring>
#include <vector>

#include "cic.cuh"
#include "maps.cuh"

namespace sc {

namespace {

// Block sizes are multiples of 4 warps so that the four SM sub-partitions,
// each with its own FP64 unit, carry the same number of warps.  Largest block
// per variant (measured on the c2 workload): 768 threads (80 registers) for
// the single-grid kernels (bounding the float32-field kernel at 1024 threads,
// 64 registers, spilled and ran 1% slower; the float64-field kernel gained 3%
// over 640 threads with 96 registers); the batched float64-field kernel,
// whose per-bunch descriptor costs registers, keeps 640 (96 registers).
template <bool F32>
constexpr int kp_max_threads() {
  return 768;
}
template <bool F32>
constexpr int kpb_max_threads() {
  return F32 ? 768 : 640;
}

// Kick from the Bezier surface of the potential (Sec. IV-C): E = -grad u, and
// with the longitudinal kick the neighbouring slices' u from the same
// surfaces.  Not inlined: its registers stay out of the bilinear path.
__device__ __noinline__ void bezier_kick(State& s, const KPParams& P, int cell, double fx, double fy) {
  const int nxk = P.gk.nx, nyk = P.gk.ny, cells = nxk * nyk;
  const int k = cell / cells, rem = cell - k * cells, j = rem / nxk, i = rem - j * nxk;
  const double* ph = P.phi + (size_t)k * cells;
  double u, gx, gy;
  bezier_eval<double, false, true>(ph, nxk, nyk, i, j, fx, fy, u, gx, gy);
  s.px = fma(-P.kl * (1.0 / 3.0) * P.gk.inv_hx, gx, s.px);
  s.py = fma(-P.kl * (1.0 / 3.0) * P.gk.inv_hy, gy, s.py);
  if (P.lon) {
    double up = 0.0, dn = 0.0, a, b;
    if (k + 1 < P.gk.nz) bezier_eval<double, true, false>(ph + cells, nxk, nyk, i, j, fx, fy, up, a, b);
    if (k > 0) bezier_eval<double, true, false>(ph - cells, nxk, nyk, i, j, fx, fy, dn, a, b);
    s.ps = fma(-P.klz, up - dn, s.ps);
  }
}

// The same from the split form's float32 potential, in float32 arithmetic
// (its fields carry float32 accuracy); the momentum updates in float64.
__device__ __noinline__ void bezier_kick32(State& s, const KPParams& P, int cell, float fx, float fy) {
  const int nxk = P.gk.nx, nyk = P.gk.ny, cells = nxk * nyk;
  const int k = cell / cells, rem = cell - k * cells, j = rem / nxk, i = rem - j * nxk;
  const float* ph = P.phi32 + (size_t)k * cells;
  float u, gx, gy;
  bezier_eval<float, false, true>(ph, nxk, nyk, i, j, fx, fy, u, gx, gy);
  s.px = fma(-P.kl * (1.0 / 3.0) * P.gk.inv_hx, (double)gx, s.px);
  s.py = fma(-P.kl * (1.0 / 3.0) * P.gk.inv_hy, (double)gy, s.py);
  if (P.lon) {
    float up = 0.f, dn = 0.f, a, b;
    if (k + 1 < P.gk.nz) bezier_eval<float, true, false>(ph + cells, nxk, nyk, i, j, fx, fy, up, a, b);
    if (k > 0) bezier_eval<float, true, false>(ph - cells, nxk, nyk, i, j, fx, fy, dn, a, b);
    s.ps = fma(-P.klz, (double)(up - dn), s.ps);
  }
}

// The particle's coefficients of every quadrupole family, from its current ps
// (k), into the cache.  Not inlined: it runs once per call and after RF cavities.
__device__ __noinline__ void store_quad_cache(const KPParams& P, const PsConst& k, int64_t p) {
  const size_t n = (size_t)P.n;
  for (int f = 0; f < P.qfam_n; ++f) {
    const QuadCoef q = quad_coef(P.qfam[f], k);
    double* c = P.qcache + (size_t)f * 6 * n + p;
    c[0] = q.cx;
    c[n] = q.sxa;
    c[2 * n] = q.sxb;
    c[3 * n] = q.cy;
    c[4 * n] = q.sya;
    c[5 * n] = q.syb;
  }
}

// One block's share of a space-charge location: particles p_begin, p_begin +
// p_step, ... below p_end.  use_tile: deposit into the block's shared-memory
// tile (zeroed by the caller), flushed at the end; CACHE: the cell cache of
// the previous deposit is valid for the gather and is refreshed by this
// deposit; F32: float32 fields and gather (the split-precision solve's fields
// carry float32 accuracy; the fractions are then the deposit's own fixed-point
// weights), else float64 fields and fractions.
template <bool CACHE, bool F32, bool XE>
__device__ __forceinline__ void kick_push_range(const KPParams& P, bool use_tile, unsigned long long* tile,
                                                int* tile_k, int64_t p_begin, int64_t p_end, int64_t p_step) {
  const int cells = P.gd.nx * P.gd.ny;
  const int psc_mode = P.psc ? P.psc_mode : 0;
  const size_t n = (size_t)P.n;
  unsigned int out = 0;
  for (int64_t p = p_begin + threadIdx.x; p < p_end; p += p_step) {
    State s{P.x[p], P.px[p], P.y[p], P.py[p], P.sg[p], (P.ps_mode & 2) ? 0.0 : P.ps[p]};
    if (P.do_kick) {
      int cell;
      if (F32) {
        float fx, fy;
        if (CACHE) {
          cell = P.cell[p];
          const int2 a = P.fix[p];
          fx = (float)a.x * (1.0f / 1048576.0f);
          fy = (float)a.y * (1.0f / 1048576.0f);
        } else {
          double dx, dy;
          int2 a;
          cell = locate<false>(P.gk, s.x, s.y, s.sg, a, dx, dy);
          fx = (float)a.x * (1.0f / 1048576.0f);
          fy = (float)a.y * (1.0f / 1048576.0f);
        }
        if (XE && cell >= 0 && P.bezier) {
          bezier_kick32(s, P, cell, fx, fy);
        } else if (cell >= 0) {
          const float2* e = P.E32 + cell;
          const float2 e00 = __ldg(e), e10 = __ldg(e + 1);
          const float2 e01 = __ldg(e + P.gk.nx), e11 = __ldg(e + P.gk.nx + 1);
          const float ax = fmaf(fx, e10.x - e00.x, e00.x), bx = fmaf(fx, e11.x - e01.x, e01.x);
          const float ay = fmaf(fx, e10.y - e00.y, e00.y), by = fmaf(fx, e11.y - e01.y, e01.y);
          s.px = fma(P.kl, f32_widen(fmaf(fy, bx - ax, ax)), s.px);
          s.py = fma(P.kl, f32_widen(fmaf(fy, by - ay, ay)), s.py);
          if (P.lon) {
            // longitudinal kick from the float32 potentials of the neighbouring slices
            const int cells = P.gk.nx * P.gk.ny, k = cell / cells, nxk = P.gk.nx;
            float up = 0.f, dn = 0.f;
            if (k + 1 < P.gk.nz) {
              const float* f = P.phi32 + cell + cells;
              const float a0 = fmaf(fx, __ldg(f + 1) - __ldg(f), __ldg(f));
              const float a1 = fmaf(fx, __ldg(f + nxk + 1) - __ldg(f + nxk), __ldg(f + nxk));
              up = fmaf(fy, a1 - a0, a0);
            }
            if (k > 0) {
              const float* f = P.phi32 + cell - cells;
              const float a0 = fmaf(fx, __ldg(f + 1) - __ldg(f), __ldg(f));
              const float a1 = fmaf(fx, __ldg(f + nxk + 1) - __ldg(f + nxk), __ldg(f + nxk));
              dn = fmaf(fy, a1 - a0, a0);
            }
            s.ps = fma(-P.klz, (double)(up - dn), s.ps);
          }
        }
      } else {
        double fx, fy;
        if (CACHE) {
          cell = P.cell[p];
          const double2 f = P.frac[p];
          fx = f.x;
          fy = f.y;
        } else {
          int2 a;
          cell = locate<true>(P.gk, s.x, s.y, s.sg, a, fx, fy);
        }
        if (XE && cell >= 0 && P.bezier) {
          bezier_kick(s, P, cell, fx, fy);
        } else if (cell >= 0) {
          const double2* e = P.E + cell;
          const double2 e00 = __ldg(e), e10 = __ldg(e + 1);
          const double2 e01 = __ldg(e + P.gk.nx), e11 = __ldg(e + P.gk.nx + 1);
          // bilinear interpolation with the gather weights (1-fx)(1-fy), fx(1-fy), (1-fx)fy, fx fy
          const double ax = fma(fx, e10.x - e00.x, e00.x), bx = fma(fx, e11.x - e01.x, e01.x);
          const double ay = fma(fx, e10.y - e00.y, e00.y), by = fma(fx, e11.y - e01.y, e01.y);
          s.px = fma(P.kl, fma(fy, bx - ax, ax), s.px);
          s.py = fma(P.kl, fma(fy, by - ay, ay), s.py);
          if (P.lon) {
            // longitudinal kick: centred z-difference of the neighbouring slices' potentials
            const int cells = P.gk.nx * P.gk.ny, k = cell / cells, nxk = P.gk.nx;
            double up = 0.0, dn = 0.0;
            if (k + 1 < P.gk.nz) {
              const double* f = P.phi + cell + cells;
              const double a0 = fma(fx, __ldg(f + 1) - __ldg(f), __ldg(f));
              const double a1 = fma(fx, __ldg(f + nxk + 1) - __ldg(f + nxk), __ldg(f + nxk));
              up = fma(fy, a1 - a0, a0);
            }
            if (k > 0) {
              const double* f = P.phi + cell - cells;
              const double a0 = fma(fx, __ldg(f + 1) - __ldg(f), __ldg(f));
              const double a1 = fma(fx, __ldg(f + nxk + 1) - __ldg(f + nxk), __ldg(f + nxk));
              dn = fma(fy, a1 - a0, a0);
            }
            s.ps = fma(-P.klz, up - dn, s.ps);
          }
        }
      }
    }
    PsConst k;
    // the longitudinal kick changed psigma: its dependent quantities are recomputed and stored
    const bool fresh = psc_mode == 2 || (psc_mode == 1 && P.lon);
    if (psc_mode == 1 && !fresh) {
      k.opd2 = P.psc[p];
      k.opb = P.psc[n + p];
      k.s1 = (P.psc_skip & 1) ? 0.0 : P.psc[2 * n + p];
      k.r = (P.psc_skip & 1) ? 0.0 : P.psc[3 * n + p];
      k.qi = (P.psc_skip & 2) ? 0.0 : P.psc[4 * n + p];
    } else {
      ps_const(k, s.ps, P.beta0_sq, fresh || P.has_quad != 0);
    }
    const bool quads = psc_mode != 0 || P.has_quad != 0;
    // the quadrupole coefficient cache holds this particle's values unless ps changed in this launch
    const double* qc = (P.qcache && psc_mode == 1 && !fresh) ? P.qcache + p : nullptr;
    const bool changed = P.el ? push_elements<XE>(s, k, P.el, P.n_elem, P.beta0_sq, P.inv_gamma0_sq, quads, qc, n)
                              : push_elements<XE>(s, k, P.inl, P.n_elem, P.beta0_sq, P.inv_gamma0_sq, quads, qc, n);
    if (fresh || (psc_mode == 1 && changed)) {
      P.psc[p] = k.opd2;
      P.psc[n + p] = k.opb;
      P.psc[2 * n + p] = k.s1;
      P.psc[3 * n + p] = k.r;
      P.psc[4 * n + p] = k.qi;
      if (P.qcache) store_quad_cache(P, k, p);
    }
    if (P.do_deposit) {
      double fx = 0.0, fy = 0.0;
      int2 a = make_int2(0, 0);
      int i, j, kz;
      const int cell = locate<!F32>(P.gd, s.x, s.y, s.sg, a, fx, fy, i, j, kz);
      if (cell < 0) {
        ++out;
        a = make_int2(0, 0);
      }
      if (use_tile && tile_is_grid(P.gd)) {
        if (cell >= 0) deposit4(tile, P.gd.nx, cell, a);
      } else {
        deposit_at(deposit_key(use_tile, tile_k, P.gd, cell, i, j, kz), a, tile, P.gd.wnx, P.Q, P.gd.nx);
      }
      if (CACHE) {
        P.cell[p] = cell;
        if (F32)
          P.fix[p] = a;
        else
          P.frac[p] = make_double2(fx, fy);
      }
    }
    P.x[p] = s.x;
    P.px[p] = s.px;
    P.y[p] = s.y;
    P.py[p] = s.py;
    P.sg[p] = s.sg;
    if (!(P.ps_mode & 1)) P.ps[p] = s.ps;
  }
  pdl_allow();
  if (P.do_deposit) {
    count_out(out, P.n_out);
    if (use_tile) {
      __syncthreads();
      if (*tile_k >= 0) tile_flush(tile, P.Q + (size_t)*tile_k * cells, P.gd);
    }
  }
}

// One grid, one location.  TILE: the launch deposits (through the block's tile);
// XE: thick sextupoles, exact dipoles or the Bezier gather may occur.
template <bool TILE, bool CACHE, bool F32, bool XE>
__global__ void __launch_bounds__(kp_max_threads<F32>()) kick_push_kernel(const __grid_constant__ KPParams P) {
  extern __shared__ unsigned long long tile[];
  __shared__ int tile_k;  // slice held by the tile (-1: not yet claimed)
  if (TILE) {
    tile_zero(tile, P.gd.wnx * P.gd.wny);
    if (threadIdx.x == 0) tile_k = P.gd.nz > 1 ? -1 : 0;
  }
  pdl_wait();  // fields, charge grid and particles of the previous kernels
  if (TILE) __syncthreads();
  // Traversal: each block one contiguous, equal chunk, or all blocks sweeping a
  // common window (grid stride); consecutive threads take consecutive particles
  // either way.  Default (measured on the c2 workload): chunks for the
  // float32-field variant (every SM finishes together), grid stride for the
  // float64-field variant (whose plan arrays take more of L2); the launch-shape
  // tuner may choose (P.traversal).  Sliced grids always use chunks, so that a
  // block's particles (sorted by sigma) stay in the slice its tile holds.
  const bool chunked = P.gd.nz > 1 || (P.traversal < 0 ? F32 : P.traversal == 1);
  const int64_t chunk = chunked ? (P.n + gridDim.x - 1) / gridDim.x : 0;
  const int64_t p_begin = chunked ? (int64_t)blockIdx.x * chunk : (int64_t)blockIdx.x * blockDim.x;
  const int64_t p_end = chunked ? min(P.n, (int64_t)(blockIdx.x + 1) * chunk) : P.n;
  const int64_t p_step = chunked ? (int64_t)blockDim.x : (int64_t)gridDim.x * blockDim.x;
  kick_push_range<CACHE, F32, XE>(P, TILE, tile, &tile_k, p_begin, p_end, p_step);
}

// Many bunches, one location each, one launch.  Block b works for bunch
// blocks[b].x (its descriptor descs[bunch], copied to shared memory) on the
// contiguous chunk blocks[b].y of blocks[b].z equal chunks of that bunch.
// The bunch's deposit uses the tile when its grid's tile window fits tile_cells.
template <bool CACHE, bool F32, bool XE>
__global__ void __launch_bounds__(kpb_max_threads<F32>())
    kick_push_batched(const KPParams* __restrict__ descs, const int4* __restrict__ blocks, int tile_cells) {
  extern __shared__ unsigned long long tile[];
  __shared__ int tile_k;
  __shared__ KPParams sP;
  const int4 bt = blocks[blockIdx.x];
  {
    // the descriptor is plain data: copy it as 8-byte words
    const unsigned long long* src = (const unsigned long long*)(descs + bt.x);
    unsigned long long* dst = (unsigned long long*)&sP;
    for (int w = threadIdx.x; w < (int)(sizeof(KPParams) / 8); w += blockDim.x) dst[w] = src[w];
  }
  __syncthreads();
  const bool use_tile = sP.do_deposit && sP.gd.wnx * sP.gd.wny <= tile_cells;
  if (use_tile) {
    tile_zero(tile, sP.gd.wnx * sP.gd.wny);
    if (threadIdx.x == 0) tile_k = sP.gd.nz > 1 ? -1 : 0;
  }
  pdl_wait();
  __syncthreads();
  const int64_t chunk = (sP.n + bt.z - 1) / bt.z;
  const int64_t p_begin = (int64_t)bt.y * chunk;
  const int64_t p_end = min(sP.n, p_begin + chunk);
  kick_push_range<CACHE, F32, XE>(sP, use_tile, tile, &tile_k, p_begin, p_end, blockDim.x);
}

using KPKernel = void (*)(KPParams);
using KPBatched = void (*)(const KPParams*, const int4*, int);

// kick_push_kernel<TILE, CACHE, F32, XE> indexed by the four flags
KPKernel kp_kernel(bool tile, bool cache, bool f32, bool xe) {
  static const KPKernel k[16] = {
      kick_push_kernel<false, false, false, false>, kick_push_kernel<false, false, false, true>,
      kick_push_kernel<false, false, true, false>,  kick_push_kernel<false, false, true, true>,
      kick_push_kernel<false, true, false, false>,  kick_push_kernel<false, true, false, true>,
      kick_push_kernel<false, true, true, false>,   kick_push_kernel<false, true, true, true>,
      kick_push_kernel<true, false, false, false>,  kick_push_kernel<true, false, false, true>,
      kick_push_kernel<true, false, true, false>,   kick_push_kernel<true, false, true, true>,
      kick_push_kernel<true, true, false, false>,   kick_push_kernel<true, true, false, true>,
      kick_push_kernel<true, true, true, false>,    kick_push_kernel<true, true, true, true>};
  return k[(tile ? 8 : 0) + (cache ? 4 : 0) + (f32 ? 2 : 0) + (xe ? 1 : 0)];
}

KPBatched kp_batched(bool cache, bool f32, bool xe) {
  static const KPBatched k[8] = {kick_push_batched<false, false, false>, kick_push_batched<false, false, true>,
                                 kick_push_batched<false, true, false>,  kick_push_batched<false, true, true>,
                                 kick_push_batched<true, false, false>,  kick_push_batched<true, false, true>,
                                 kick_push_batched<true, true, false>,   kick_push_batched<true, true, true>};
  return k[(cache ? 4 : 0) + (f32 ? 2 : 0) + (xe ? 1 : 0)];
}

// Resident blocks per SM of the smallest-occupancy variant for this tile size.
int min_blocks(int smem, bool tile) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int best = 1 << 30;
  for (int v = 0; v < 8; ++v) {
    const bool cache = v & 4, f32 = v & 2, xe = v & 1;
    const KPKernel k = kp_kernel(tile, cache, f32, xe);
    if (tile) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, kTileBytes);
    int per = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k, f32 ? kp_max_threads<true>() : kp_max_threads<false>(),
                                                  tile ? smem : 0);
    best = per < best ? per : best;
  }
  return sms * (best < 1 ? 1 : best);
}

}  // namespace

int kick_push_blocks_for(int smem_bytes, bool tile) {
  // all variants share the shared memory size; size the grid on the largest register count
  return min_blocks(smem_bytes, tile);
}

int kick_push_max_threads(bool f32) { return f32 ? kp_max_threads<true>() : kp_max_threads<false>(); }

int kick_push_blocks_at(int smem_bytes, bool tile, bool f32, int threads) {
  // the smallest occupancy over the gather variants (cell cache, XE) of this field type
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int best = 1 << 30;
  for (int v = 0; v < 4; ++v) {
    const KPKernel k = kp_kernel(tile, v & 2, f32, v & 1);
    if (tile) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, kTileBytes);
    int per = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k, threads, tile ? smem_bytes : 0);
    best = per < best ? per : best;
  }
  return sms * (best < 1 ? 1 : best);
}

sc_status launch_kick_push(const KPParams& P, const sc_grid* dep, int blocks, cudaStream_t s, int threads) {
  const bool tile = P.do_deposit && dep;
  const bool cache = P.cell != nullptr;
  const bool f32 = P.field32 != 0;
  const bool xe = P.has_xe != 0 || P.bezier != 0;
  // default: the variant's largest block (measured: the extra warps outweigh a partly empty last round)
  if (threads <= 0) threads = kick_push_max_threads(f32);
  const int64_t need = (P.n + threads - 1) / threads;
  if (need < blocks) blocks = (int)(need > 0 ? need : 1);
  const int smem = tile ? tile_bytes(dep) : 0;
  SC_CUDA(launch_pdl(kp_kernel(tile, cache, f32, xe), dim3(blocks), dim3(threads), (size_t)smem, s, P));
  return SC_OK;
}

int kick_push_batched_threads(bool f32) { return f32 ? kpb_max_threads<true>() : kpb_max_threads<false>(); }

int kick_push_batched_resident(int smem_bytes, bool f32, bool cache, int threads) {
  if (threads <= 0) threads = kick_push_batched_threads(f32);
  int dev = 0, sms = 0, per = 1 << 30;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  for (int v = 0; v < 8; ++v) {
    const KPBatched k = kp_batched(v & 4, v & 2, v & 1);
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, kTileBytes);
  }
  for (int xe = 0; xe < 2; ++xe) {
    int p = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p, kp_batched(cache, f32, xe), threads, smem_bytes);
    per = p < per ? p : per;
  }
  return sms * (per < 1 ? 1 : per);
}

sc_status launch_kick_push_batched(const KPParams* descs, const int4* blocks, int n_blocks, int tile_cells, bool f32,
                                   bool cache, bool xe, cudaStream_t s, int threads) {
  // (the shared-memory limit was raised by kick_push_batched_resident, called before any launch)
  if (threads <= 0) threads = kick_push_batched_threads(f32);
  SC_CUDA(launch_pdl(kp_batched(cache, f32, xe), dim3(n_blocks), dim3(threads), (size_t)tile_cells * 8, s, descs,
                     blocks, tile_cells));
  return SC_OK;
}

// Per-element constants in float64 on the host (libm), in the layouts that
// maps.cuh documents for each element type.
void compile_elements(const sc_element* in, int n, const sc_beam* b, DevElem* out) {
  const double beta0_sq = b->beta0 * b->beta0;
  const double e0 = b->gamma0 * b->mass_ev;
  for (int i = 0; i < n; ++i) {
    const sc_element& e = in[i];
    DevElem& d = out[i];
    d = DevElem{};
    d.type = e.type;
    switch (e.type) {
      case SC_DRIFT:
        d.p[0] = e.length;
        break;
      case SC_QUAD: {
        d.p[0] = e.length;
        if (e.k1 == 0.0) {
          d.flags = QF_ZERO;
          break;
        }
        const double sqk = std::sqrt(std::fabs(e.k1));
        const double th0 = sqk * e.length;
        d.flags = e.k1 > 0.0 ? QF_FOCUS_X : QF_FOCUS_Y;
        d.p[0] = 0.25 * e.length;
        d.p[1] = e.length / (b->gamma0 * b->gamma0);
        d.p[2] = std::cos(th0);
        d.p[3] = std::sin(th0);
        d.p[4] = std::cosh(th0);
        d.p[5] = std::sinh(th0);
        d.p[6] = sqk;
        d.p[7] = 1.0 / sqk;
        d.p[8] = e.length * e.k1;
        break;
      }
      case SC_SEXT:
        if (e.length > 0.0) {  // Eq. Sym2: kicks of k2 b L = k2l/2 between H0 flows of a L, c L, a L
          d.flags = 1;
          d.p[0] = 0.25 * e.k2l;
          d.p[1] = 0.5 * e.k2l;
          d.p[2] = 0.5 * (1.0 - 1.0 / std::sqrt(3.0)) * e.length;
          d.p[3] = e.length / std::sqrt(3.0);
        } else {
          d.p[0] = 0.5 * e.k2l;
          d.p[1] = e.k2l;
        }
        break;
      case SC_EXACT_BEND: {
        d.p[0] = e.length;
        if (e.angle == 0.0 || e.length == 0.0) {
          d.flags = 1;  // exact drift
          break;
        }
        d.p[1] = e.angle;
        d.p[2] = std::cos(e.angle);
        d.p[3] = std::sin(e.angle);
        d.p[4] = e.length / e.angle;  // rho
        d.p[5] = e.angle / e.length;  // 1 / rho
        break;
      }
      case SC_BEND: {
        d.p[0] = e.length;
        if (e.angle == 0.0 || e.length == 0.0) {
          d.flags = 1;
          break;
        }
        const double h = e.angle / e.length, C = std::cos(e.angle), S = std::sin(e.angle);
        d.p[1] = C;
        d.p[2] = S;
        d.p[3] = S / h;
        d.p[4] = (1.0 - C) / h;
        d.p[5] = h * S;
        d.p[6] = e.length - S / h;
        break;
      }
      case SC_RF:
        d.p[0] = (e0 > 0.0) ? e.volt / (beta0_sq * e0) : 0.0;
        d.p[1] = (b->circumference > 0.0) ? 2.0 * M_PI * e.harmonic / b->circumference : 0.0;
        d.p[2] = e.lag;
        break;
      default:
        break;
    }
  }
}

int quad_families(const DevElem* el, int n, DevElem* fam, int max) {
  int nf = 0;
  for (int i = 0; i < n; ++i) {
    const DevElem& e = el[i];
    if (e.type != SC_QUAD || (e.flags & QF_KIND) == QF_ZERO) continue;
    bool seen = false;
    for (int f = 0; f < nf && !seen; ++f)
      seen = (fam[f].flags & QF_KIND) == (e.flags & QF_KIND) && std::memcmp(fam[f].p, e.p, sizeof e.p) == 0;
    if (!seen && nf < max) {
      fam[nf] = e;
      fam[nf].flags = e.flags & QF_KIND;
      ++nf;
    }
  }
  return nf;
}

int psc_skip_mask(const sc_element* host, int n, const sc_beam* b, const DevElem* fam, int nf) {
  std::vector<DevElem> d(n > 0 ? n : 1);
  compile_elements(host, n, b, d.data());
  tag_quad_families(d.data(), n, fam, nf);
  bool thick = false, own = false;
  for (int i = 0; i < n; ++i)
    if (d[i].type == SC_QUAD && (d[i].flags & QF_KIND) != QF_ZERO) {
      thick = true;
      own = own || (d[i].flags >> QF_FAM_SHIFT) == 0;
    }
  return (own ? 0 : 1) | (thick ? 0 : 2);
}

int ps_mode_mask(const sc_element* host, int n, bool lon) {
  bool reads = lon, writes = lon;
  for (int i = 0; i < n; ++i) {
    const sc_element& e = host[i];
    if (e.type == SC_QUAD || e.type == SC_BEND || e.type == SC_RF || (e.type == SC_SEXT && e.length > 0.0))
      reads = true;
    if (e.type == SC_RF) writes = true;
  }
  return (writes ? 0 : 1) | (reads || writes ? 0 : 2);
}

void tag_quad_families(DevElem* el, int n, const DevElem* fam, int nf) {
  for (int i = 0; i < n; ++i) {
    DevElem& e = el[i];
    if (e.type != SC_QUAD) continue;
    e.flags &= QF_KIND;
    for (int f = 0; f < nf; ++f)
      if (fam[f].flags == e.flags && std::memcmp(fam[f].p, e.p, sizeof e.p) == 0) {
        e.flags |= (f + 1) << QF_FAM_SHIFT;
        break;
      }
  }
}

}  // namespace sc
