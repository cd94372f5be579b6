// Stand-alone CIC charge deposition (Sec. IV-A): per-block shared-memory
// uint64 tile (the whole grid, or a centred window of it for grids beyond the
// tile's 200 KB), flushed once per block into the global grid.  For a bunch
// the grid itself ordered by cell (sc_sort_particles) each warp combines the
// weights of neighbouring lanes in the same cell before the atomic adds
// (deposit_warp); otherwise every particle adds its own four weights.
#include <algorithm>

#include "cic.cuh"

namespace sc {

namespace {

// 1024 threads: the shared-memory atomics of random cells are latency-bound
// (bank conflicts), more warps per SM hide more of it (measured).
constexpr int kDepThreads = 1024;

template <bool AGG>
__global__ void __launch_bounds__(kDepThreads) deposit_kernel(const double* __restrict__ x,
                                                               const double* __restrict__ y,
                                                               const double* __restrict__ sg, int64_t n,
                                                               GridGeom g, unsigned long long* Q,
                                                               unsigned long long* n_out,
                                                               unsigned long long* n_nan) {
  extern __shared__ unsigned long long tile[];
  __shared__ int tile_k;
  const int cells = g.nx * g.ny;
  tile_zero(tile, g.wnx * g.wny);
  if (threadIdx.x == 0) tile_k = g.nz > 1 ? -1 : 0;
  __syncthreads();
  unsigned int out = 0, bad = 0;  // particles outside the grid; of those, non-finite ones
  // one contiguous chunk per block (a sigma-sorted bunch keeps a block in one slice)
  const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const int64_t p_end = min(n, (int64_t)(blockIdx.x + 1) * chunk);
  const bool sliced = g.nz > 1;
  int64_t p = (int64_t)blockIdx.x * chunk + threadIdx.x;
  // the next particle's coordinates are loaded before this one's deposit (hides their latency)
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
    int i, j, k;
    const int cell = locate<false>(g, xc, yc, sc_, a, fx, fy, i, j, k);
    if (cell < 0) {
      ++out;
      bad += nonfinite_state(g, xc, yc, sc_);
    }
    if (AGG) {  // an ordered bunch: the warp combines equal cells
      deposit_warp(__activemask(), deposit_key(true, &tile_k, g, cell, i, j, k), a, tile, g.wnx, Q, g.nx);
    } else if (tile_is_grid(g)) {
      if (cell >= 0) deposit4(tile, g.nx, cell, a);
    } else {
      deposit_at(deposit_key(true, &tile_k, g, cell, i, j, k), a, tile, g.wnx, Q, g.nx);
    }
  }
  count_out(out, n_out);
  count_out(bad, n_nan);
  __syncthreads();
  if (tile_k >= 0) tile_flush(tile, Q + (size_t)tile_k * cells, g);
}

}  // namespace

int tile_bytes(const sc_grid* g) { return g->geom.wnx * g->geom.wny * 8; }

void tile_window(int nx, int ny, int* wx0, int* wy0, int* wnx, int* wny) {
  // A grid whose uint64 bins fit kTileBytes is held whole.  A larger one gets
  // the centred window of about equal sides of 128 KB (128 x 128 of a 256 x 256
  // grid spanning +-5 sigma: +-2.5 sigma, 97.5% of a Gaussian beam; the rest
  // goes straight to the global grid).  Not larger: shared memory is taken from
  // the L1 cache the field gathers use (measured on c3, 4e6 particles on
  // 256 x 256: a 160 x 160 window of 200 KB made the fused kick/push 5% slower
  // than 128 x 128, with the same stand-alone deposit time).
  constexpr int kWindowCells = 16384;
  int w = nx, h = ny;
  if ((long long)nx * ny * 8 > kTileBytes) {
    w = nx < 128 ? nx : 128;
    h = ny < kWindowCells / w ? ny : kWindowCells / w;
    w = nx < kWindowCells / h ? nx : kWindowCells / h;
  }
  *wnx = w;
  *wny = h;
  *wx0 = (nx - w) / 2;
  *wy0 = (ny - h) / 2;
}

sc_status launch_deposit(sc_grid* g, const sc_particles* p) {
  int blocks = g->dep_blocks;
  const int64_t need = (p->n + kDepThreads - 1) / kDepThreads;
  if (need < blocks) blocks = (int)(need > 0 ? need : 1);
  // the bunch this grid last ordered by cell: combine equal cells within warps
  const bool agg = p->x == g->sorted_x && p->n == g->sorted_n;
  (agg ? deposit_kernel<true> : deposit_kernel<false>)<<<blocks, kDepThreads, tile_bytes(g), g->stream>>>(
      p->x, p->y, p->sigma, p->n, g->geom, g->Q, g->n_out, g->n_nan);
  SC_CUDA(cudaGetLastError());
  return SC_OK;
}

int deposit_blocks_for(int smem_bytes) {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaFuncSetAttribute(deposit_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTileBytes);
  cudaFuncSetAttribute(deposit_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTileBytes);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, deposit_kernel<false>, kDepThreads, smem_bytes);
  if (per < 1) per = 1;
  return sms * per;
}

}  // namespace sc

// ---------------------------------------------------------------------------
// Cell ordering of a bunch (opt-in): the deposit's warps combine the weights
// of neighbouring particles in the same cell, so a bunch ordered by cell sends
// a warp's 32 particles to one or two cells' four nodes.
// ---------------------------------------------------------------------------

#include <cub/device/device_radix_sort.cuh>

namespace sc {

namespace {

// Sort key of each particle: its cell on grid g (slice included), or the
// total cell count (sorted last) when it is outside; value = its index.
__global__ void cell_keys(const double* __restrict__ x, const double* __restrict__ y, const double* __restrict__ sg,
                          int64_t n, GridGeom g, int* __restrict__ keys, int* __restrict__ idx) {
  const int outside = g.nx * g.ny * g.nz;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    double fx, fy;
    int2 a;
    const int cell = locate<false>(g, x[p], y[p], g.nz > 1 ? sg[p] : 0.0, a, fx, fy);
    keys[p] = cell < 0 ? outside : cell;
    idx[p] = (int)p;
  }
}

__global__ void gather_by(const double* __restrict__ src, const int* __restrict__ perm, int64_t n,
                          double* __restrict__ dst) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x)
    dst[p] = src[perm[p]];
}

__global__ void copy_perm(const int* __restrict__ perm, int64_t n, int32_t* __restrict__ out) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x)
    out[p] = perm[p];
}

}  // namespace

sc_status sort_particles(sc_grid* g, const sc_particles* p, int32_t* perm_out) {
  const int64_t n = p->n;
  const int outside = g->nx * g->ny * g->nz;
  int end_bit = 1;
  while (end_bit < 31 && (1LL << end_bit) <= outside) ++end_bit;
  size_t temp = 0;
  SC_CUDA(cub::DeviceRadixSort::SortPairs(nullptr, temp, (const int*)nullptr, (int*)nullptr, (const int*)nullptr,
                                          (int*)nullptr, (int)n, 0, end_bit, g->stream));
  // scratch: keys and indices twice (sort input / output), one float64 array, the sort's temporary storage
  const size_t need = (size_t)n * (4 * sizeof(int) + sizeof(double)) + temp + 256;
  if (need > g->sort_cap) {
    SC_CUDA(cudaStreamSynchronize(g->stream));
    cudaFree(g->sort_scratch);
    g->sort_scratch = nullptr;
    g->sort_cap = 0;
    SC_CUDA(cudaMalloc(&g->sort_scratch, need));
    g->sort_cap = need;
  }
  unsigned char* base = (unsigned char*)g->sort_scratch;
  double* tmp = (double*)base;
  int* keys_in = (int*)(tmp + n);
  int* keys_out = keys_in + n;
  int* idx_in = keys_out + n;
  int* idx_out = idx_in + n;
  void* cub_temp = (void*)(((uintptr_t)(idx_out + n) + 255) & ~(uintptr_t)255);
  int dev = 0, sms = 0;
  SC_CUDA(cudaGetDevice(&dev));
  SC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int blocks = (int)std::min<int64_t>((n + 255) / 256, (int64_t)sms * 8);
  cell_keys<<<blocks, 256, 0, g->stream>>>(p->x, p->y, p->sigma, n, g->geom, keys_in, idx_in);
  SC_CUDA(cudaGetLastError());
  SC_CUDA(cub::DeviceRadixSort::SortPairs(cub_temp, temp, keys_in, keys_out, idx_in, idx_out, (int)n, 0, end_bit,
                                          g->stream));
  double* arr[6] = {p->x, p->px, p->y, p->py, p->sigma, p->psigma};
  for (double* a : arr) {
    gather_by<<<blocks, 256, 0, g->stream>>>(a, idx_out, n, tmp);
    SC_CUDA(cudaGetLastError());
    SC_CUDA(cudaMemcpyAsync(a, tmp, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, g->stream));
  }
  if (perm_out) {
    copy_perm<<<blocks, 256, 0, g->stream>>>(idx_out, n, perm_out);
    SC_CUDA(cudaGetLastError());
  }
  g->sorted_x = p->x;
  g->sorted_n = n;
  return SC_OK;
}

}  // namespace sc
