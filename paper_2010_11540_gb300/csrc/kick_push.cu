// Fused space-charge step for one location: bilinear field gather + kick
// (Sec. IV kick equation), push through the segment's elements (Sec. III),
// and CIC deposit of the new positions (Sec. IV-A) into a per-block
// shared-memory int64 tile flushed once per block.  One thread per particle,
// persistent grid-stride loop over SoA float64 state.
#include "cic.cuh"
#include "maps.cuh"

namespace sc {

namespace {

constexpr int kKPThreads = 512;

template <bool TILE>
__global__ void __launch_bounds__(kKPThreads) kick_push_kernel(const KPParams P) {
  extern __shared__ unsigned long long tile[];
  const int cells = P.gd.nx * P.gd.ny;
  if (TILE) {
    tile_zero(tile, cells);
    __syncthreads();
  }
  unsigned long long* dst = TILE ? tile : P.Q;
  const BeamK bk{P.beta0_sq, P.inv_gamma0_sq, P.rf_scale, P.two_pi_over_c};
  unsigned int out = 0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < P.n; p += stride) {
    State s{P.x[p], P.px[p], P.y[p], P.py[p], P.sg[p], P.ps[p]};
    if (P.do_kick) {
      Cell c;
      if (locate(P.gk, s.x, s.y, c)) {
        const double2* e = P.E + (size_t)c.j * P.gk.nx + c.i;
        const double2 e00 = __ldg(e), e10 = __ldg(e + 1);
        const double2 e01 = __ldg(e + P.gk.nx), e11 = __ldg(e + P.gk.nx + 1);
        const double gx = 1.0 - c.fx, gy = 1.0 - c.fy;
        const double w00 = gx * gy, w10 = c.fx * gy, w01 = gx * c.fy, w11 = c.fx * c.fy;
        const double ex = w00 * e00.x + w10 * e10.x + w01 * e01.x + w11 * e11.x;
        const double ey = w00 * e00.y + w10 * e10.y + w01 * e01.y + w11 * e11.y;
        s.px = fma(P.kl, ex, s.px);
        s.py = fma(P.kl, ey, s.py);
      }
    }
    push_elements(s, P.el, P.n_elem, bk);
    if (P.do_deposit) {
      Cell c;
      if (locate(P.gd, s.x, s.y, c))
        deposit4(dst, P.gd.nx, c);
      else
        ++out;
    }
    P.x[p] = s.x;
    P.px[p] = s.px;
    P.y[p] = s.y;
    P.py[p] = s.py;
    P.sg[p] = s.sg;
    P.ps[p] = s.ps;
  }
  if (P.do_deposit) {
    count_out(out, P.n_out);
    if (TILE) {
      __syncthreads();
      tile_flush(tile, P.Q, cells);
    }
  }
}

}  // namespace

int kick_push_blocks_for(int smem_bytes, bool tile) {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (tile) {
    cudaFuncSetAttribute(kick_push_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kick_push_kernel<true>, kKPThreads, smem_bytes);
  } else {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kick_push_kernel<false>, kKPThreads, 0);
  }
  if (per < 1) per = 1;
  return sms * per;
}

// dep: the deposit grid (NULL when P.do_deposit == 0).
sc_status launch_kick_push(const KPParams& P, const sc_grid* dep, int blocks, cudaStream_t s) {
  const bool tile = P.do_deposit && dep && deposit_uses_tile(dep);
  const int64_t need = (P.n + kKPThreads - 1) / kKPThreads;
  if (need < blocks) blocks = (int)(need > 0 ? need : 1);
  if (tile)
    kick_push_kernel<true><<<blocks, kKPThreads, dep->nx * dep->ny * 8, s>>>(P);
  else
    kick_push_kernel<false><<<blocks, kKPThreads, 0, s>>>(P);
  SC_CUDA(cudaGetLastError());
  return SC_OK;
}

}  // namespace sc
