// Fused space-charge step for one location: bilinear field gather + kick
// (Sec. IV kick equation), push through the segment's elements (Sec. III),
// and CIC deposit of the new positions (Sec. IV-A) into a per-block
// shared-memory int64 tile flushed once per block.  One thread per particle,
// persistent grid-stride loop over SoA float64 state.
#include <cmath>

#include "cic.cuh"
#include "maps.cuh"

namespace sc {

namespace {

constexpr int kKPThreads = 512;

// TILE: deposit into a shared-memory tile (grid fits); CACHE: the cell cache
// P.cell / P.frac is valid for the gather and is refreshed by the deposit.
template <bool TILE, bool CACHE>
__global__ void __launch_bounds__(kKPThreads) kick_push_kernel(const __grid_constant__ KPParams P) {
  extern __shared__ unsigned long long tile[];
  const int cells = P.gd.nx * P.gd.ny;
  if (TILE) tile_zero(tile, cells);
  pdl_wait();  // fields, charge grid and particles of the previous kernels
  if (TILE) __syncthreads();
  unsigned long long* dst = TILE ? tile : P.Q;
  unsigned int out = 0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < P.n; p += stride) {
    State s{P.x[p], P.px[p], P.y[p], P.py[p], P.sg[p], P.ps[p]};
    if (P.do_kick) {
      double fx, fy;
      int cell;
      if (CACHE) {
        cell = P.cell[p];
        const double2 f = P.frac[p];
        fx = f.x;
        fy = f.y;
      } else {
        cell = locate(P.gk, s.x, s.y, fx, fy);
      }
      if (cell >= 0) {
        const double2* e = P.E + cell;
        const double2 e00 = __ldg(e), e10 = __ldg(e + 1);
        const double2 e01 = __ldg(e + P.gk.nx), e11 = __ldg(e + P.gk.nx + 1);
        // bilinear interpolation with the gather weights (1-fx)(1-fy), fx(1-fy), (1-fx)fy, fx fy
        const double ax = fma(fx, e10.x - e00.x, e00.x), bx = fma(fx, e11.x - e01.x, e01.x);
        const double ay = fma(fx, e10.y - e00.y, e00.y), by = fma(fx, e11.y - e01.y, e01.y);
        s.px = fma(P.kl, fma(fy, bx - ax, ax), s.px);
        s.py = fma(P.kl, fma(fy, by - ay, ay), s.py);
      }
    }
    if (P.el)
      push_elements(s, P.el, P.n_elem, P.beta0_sq, P.inv_gamma0_sq, P.has_quad != 0);
    else
      push_elements(s, P.inl, P.n_elem, P.beta0_sq, P.inv_gamma0_sq, P.has_quad != 0);
    if (P.do_deposit) {
      double fx, fy;
      const int cell = locate(P.gd, s.x, s.y, fx, fy);
      if (cell >= 0)
        deposit4(dst, P.gd.nx, cell, fx, fy);
      else
        ++out;
      if (CACHE) {
        P.cell[p] = cell;
        P.frac[p] = make_double2(fx, fy);
      }
    }
    P.x[p] = s.x;
    P.px[p] = s.px;
    P.y[p] = s.y;
    P.py[p] = s.py;
    P.sg[p] = s.sg;
    P.ps[p] = s.ps;
  }
  pdl_allow();
  if (P.do_deposit) {
    count_out(out, P.n_out);
    if (TILE) {
      __syncthreads();
      tile_flush(tile, P.Q, cells);
    }
  }
}

template <bool TILE, bool CACHE>
int blocks_for(int smem) {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (TILE) cudaFuncSetAttribute(kick_push_kernel<TILE, CACHE>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kick_push_kernel<TILE, CACHE>, kKPThreads, smem);
  return sms * (per < 1 ? 1 : per);
}

}  // namespace

int kick_push_blocks_for(int smem_bytes, bool tile) {
  // the cached and uncached variants have the same shared memory; size on the larger register count
  if (tile) {
    const int a = blocks_for<true, false>(smem_bytes), b = blocks_for<true, true>(smem_bytes);
    return a < b ? a : b;
  }
  const int a = blocks_for<false, false>(0), b = blocks_for<false, true>(0);
  return a < b ? a : b;
}

sc_status launch_kick_push(const KPParams& P, const sc_grid* dep, int blocks, cudaStream_t s) {
  const bool tile = P.do_deposit && dep && deposit_uses_tile(dep);
  const bool cache = P.cell != nullptr;
  const int64_t need = (P.n + kKPThreads - 1) / kKPThreads;
  if (need < blocks) blocks = (int)(need > 0 ? need : 1);
  const int smem = tile ? dep->nx * dep->ny * 8 : 0;
  auto k = tile ? (cache ? kick_push_kernel<true, true> : kick_push_kernel<true, false>)
                : (cache ? kick_push_kernel<false, true> : kick_push_kernel<false, false>);
  SC_CUDA(launch_pdl(k, dim3(blocks), dim3(kKPThreads), (size_t)smem, s, P));
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
        d.p[1] = th0;
        d.p[2] = std::cos(th0);
        d.p[3] = std::sin(th0);
        d.p[4] = std::cosh(th0);
        d.p[5] = std::sinh(th0);
        d.p[6] = sqk;
        d.p[7] = 1.0 / sqk;
        d.p[8] = e.k1;
        break;
      }
      case SC_SEXT:
        d.p[0] = 0.5 * e.k2l;
        d.p[1] = e.k2l;
        break;
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

}  // namespace sc
