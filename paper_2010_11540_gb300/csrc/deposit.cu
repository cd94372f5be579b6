// Stand-alone CIC charge deposition (Sec. IV-A): per-block shared-memory
// uint64 tile, flushed once per block into the global grid.
#include "cic.cuh"

namespace sc {

namespace {

// 1024 threads: the shared-memory atomics of random cells are latency-bound
// (bank conflicts), more warps per SM hide more of it (measured).
constexpr int kDepThreads = 1024;

template <bool TILE>
__global__ void __launch_bounds__(kDepThreads) deposit_kernel(const double* __restrict__ x,
                                                               const double* __restrict__ y,
                                                               const double* __restrict__ sg, int64_t n,
                                                               GridGeom g, unsigned long long* Q,
                                                               unsigned long long* n_out) {
  extern __shared__ unsigned long long tile[];
  __shared__ int tile_k;
  const int cells = g.nx * g.ny;
  if (TILE) {
    tile_zero(tile, cells);
    if (threadIdx.x == 0) tile_k = g.nz > 1 ? -1 : 0;
    __syncthreads();
  }
  unsigned int out = 0;
  // one contiguous chunk per block (a sigma-sorted bunch keeps a block in one slice)
  const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const int64_t p_end = min(n, (int64_t)(blockIdx.x + 1) * chunk);
  const bool sliced = g.nz > 1;
  // the next particle's coordinates are loaded before this one's atomics
  int64_t p = (int64_t)blockIdx.x * chunk + threadIdx.x;
  double xn = 0.0, yn = 0.0, sn = 0.0;
  if (p < p_end) {
    xn = __ldg(x + p);
    yn = __ldg(y + p);
    if (sliced) sn = __ldg(sg + p);
  }
  for (; p < p_end; p += blockDim.x) {
    const double xc = xn, yc = yn, sc_ = sn;
    const int64_t q = p + blockDim.x;
    if (q < p_end) {
      xn = __ldg(x + q);
      yn = __ldg(y + q);
      if (sliced) sn = __ldg(sg + q);
    }
    double fx, fy;
    int2 a;
    int k;
    const int cell = locate<false>(g, xc, yc, sc_, a, fx, fy, k);
    if (cell < 0)
      ++out;
    else if (TILE)
      deposit_tiled(tile, &tile_k, Q, g, cell, k, a);
    else
      deposit4(Q, g.nx, cell, a);
  }
  count_out(out, n_out);
  if (TILE) {
    __syncthreads();
    if (tile_k >= 0) tile_flush(tile, Q + (size_t)tile_k * cells, cells);
  }
}

}  // namespace

bool deposit_uses_tile(const sc_grid* g) { return (size_t)g->nx * g->ny * 8 <= 200 * 1024; }

sc_status launch_deposit(sc_grid* g, const sc_particles* p) {
  const bool tile = deposit_uses_tile(g);
  const int smem = tile ? g->nx * g->ny * 8 : 0;
  int blocks = g->dep_blocks;
  const int64_t need = (p->n + kDepThreads - 1) / kDepThreads;
  if (need < blocks) blocks = (int)(need > 0 ? need : 1);
  if (tile)
    deposit_kernel<true><<<blocks, kDepThreads, smem, g->stream>>>(p->x, p->y, p->sigma, p->n, g->geom, g->Q, g->n_out);
  else
    deposit_kernel<false><<<blocks, kDepThreads, 0, g->stream>>>(p->x, p->y, p->sigma, p->n, g->geom, g->Q, g->n_out);
  SC_CUDA(cudaGetLastError());
  return SC_OK;
}

int deposit_blocks_for(int smem_bytes, bool tile) {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (tile) {
    cudaFuncSetAttribute(deposit_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, deposit_kernel<true>, kDepThreads, smem_bytes);
  } else {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, deposit_kernel<false>, kDepThreads, 0);
  }
  if (per < 1) per = 1;
  return sms * per;
}

}  // namespace sc
