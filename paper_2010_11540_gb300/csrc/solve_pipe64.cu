// Poisson solve inside a conducting rectangular pipe (Sec. IV-B), float64.
//
// The walls are the grid's outer nodes (phi = 0 there, Eq. boundary); the
// 5-point discretisation (Eq. disc) holds on the mx x my interior nodes
// (mx = nx - 2).  Following the paper, each direction is transformed through
// the odd extension of the data to period P = 2(m+1) (Eq. extension) and a
// length-P DFT: the DFT of an odd sequence is -2i times its sine transform,
// so one complex FFT per row or column gives the DST-I coefficients.  In the
// sine basis the discrete Laplacian is diagonal with eigenvalues
//   lambda_pq = -4 (sin^2(p pi / P_x) / hx^2 + sin^2(q pi / P_y) / hy^2),
// and the inverse transforms are the same sine transforms up to 2/(m+1) per
// axis.  The right-hand side is -2 pi q / (hx hy) (q the normalised charge at
// the nodes), the normalisation of the free-space kernel -ln r of the open
// solve.  Fields at the nodes are centred differences of phi, across the walls
// by the odd extension (phi(-1) = -phi(1)).
//
// Kernels (one FFT direction per block, Stockham radix-2 in shared memory):
//   pipe_rows     : interior charge row j          -> T1[j][p] = -2 a_p
//   pipe_columns  : T1[:, p] -> sine transform over j, / lambda, inverse over q
//                                                   -> T2[j][p]
//   pipe_rows_inv : T2[j, :] -> inverse over p      -> phi[j][i]
//   pipe_fields   : phi -> (Ex, Ey) at every node.
#include <cmath>
#include <vector>

#include "fft_smem.cuh"

namespace sc {

namespace {

// blockDim.x = nx - 1 = P/2; block (j - 1, stacked grid)
__global__ void pipe_rows(const unsigned long long* __restrict__ Q, int nx, int ny, double scale,
                          const double* __restrict__ stack_scale, double fac, double* __restrict__ T1,
                          const double2* __restrict__ tw) {
  extern __shared__ double2 sm[];
  const int P = 2 * (nx - 1), t = threadIdx.x, j = blockIdx.x + 1;
  const size_t so = (size_t)blockIdx.y * nx * ny;
  double2 *a = sm, *b = sm + P;
  pdl_wait();
  const double s = fac * (stack_scale ? stack_scale[blockIdx.y] : scale);
  const unsigned long long* q = Q + so + (size_t)j * nx;
  // V[l] = f_l (l = 1..nx-2), V[0] = V[nx-1] = 0, V[P - l] = -f_l
  a[t] = make_double2(t == 0 ? 0.0 : (double)q[t] * s, 0.0);
  a[t + nx - 1] = make_double2(t == 0 ? 0.0 : -(double)q[nx - 1 - t] * s, 0.0);
  __syncthreads();
  const double2* r = fft_smem<false>(a, b, P, tw);
  pdl_allow();
  if (t >= 1) T1[so + (size_t)j * nx + t] = r[t].y;
}

// blockDim.x = ny - 1; block (p - 1, stacked grid)
__global__ void pipe_columns(const double* __restrict__ T1, int nx, int ny, const double* __restrict__ inv_lam,
                             double* __restrict__ T2, const double2* __restrict__ tw, unsigned long long* Qzero) {
  extern __shared__ double2 sm[];
  const int P = 2 * (ny - 1), t = threadIdx.x, p = blockIdx.x + 1;
  const size_t so = (size_t)blockIdx.y * nx * ny;
  double2 *A = sm, *B = sm + P, *C = sm + 2 * P;
  pdl_wait();
  if (Qzero) {  // the row transform has read every stacked grid's charge: clear it for the next deposit
    const int64_t total = (int64_t)gridDim.y * nx * ny;
    for (int64_t c = ((int64_t)blockIdx.y * gridDim.x + blockIdx.x) * blockDim.x + t; c < total;
         c += (int64_t)gridDim.x * gridDim.y * blockDim.x)
      Qzero[c] = 0ull;
  }
  A[t] = make_double2(t == 0 ? 0.0 : T1[so + (size_t)t * nx + p], 0.0);
  A[t + ny - 1] = make_double2(t == 0 ? 0.0 : -T1[so + (size_t)(ny - 1 - t) * nx + p], 0.0);
  __syncthreads();
  double2* R = fft_smem<false>(A, B, P, tw);  // R[q].y = 4 x (2-D sine transform of f)
  double2* freebuf = (R == A) ? B : A;
  // W_q = R[q].y / lambda_pq, odd extension over q
  {
    const double w = t == 0 ? 0.0 : R[t].y * inv_lam[(size_t)t * nx + p];
    const int qm = ny - 1 - t;
    const double wm = t == 0 ? 0.0 : R[qm].y * inv_lam[(size_t)qm * nx + p];
    C[t] = make_double2(w, 0.0);
    C[t + ny - 1] = make_double2(-wm, 0.0);
  }
  __syncthreads();
  const double2* r = fft_smem<false>(C, freebuf, P, tw);
  pdl_allow();
  if (t >= 1) T2[so + (size_t)t * nx + p] = r[t].y;
}

// blockDim.x = nx - 1; block (j - 1, stacked grid)
__global__ void pipe_rows_inv(const double* __restrict__ T2, int nx, int ny, double norm, double* __restrict__ phi,
                              const double2* __restrict__ tw) {
  extern __shared__ double2 sm[];
  const int P = 2 * (nx - 1), t = threadIdx.x, j = blockIdx.x + 1;
  const size_t so = (size_t)blockIdx.y * nx * ny;
  double2 *a = sm, *b = sm + P;
  pdl_wait();
  const double* row = T2 + so + (size_t)j * nx;
  a[t] = make_double2(t == 0 ? 0.0 : row[t], 0.0);
  a[t + nx - 1] = make_double2(t == 0 ? 0.0 : -row[nx - 1 - t], 0.0);
  __syncthreads();
  const double2* r = fft_smem<false>(a, b, P, tw);
  pdl_allow();
  double* out = phi + so + (size_t)j * nx;
  if (t >= 1) out[t] = r[t].y * norm;  // walls (i = 0, nx-1; rows 0, ny-1) stay 0
}

// One thread per node of every stacked grid.
__global__ void pipe_fields(const double* __restrict__ phi, int nx, int ny, int nstack, double inv2hx,
                            double inv2hy, double2* __restrict__ E) {
  pdl_wait();
  const int64_t total = (int64_t)nstack * nx * ny;
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < total; c += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(c % nx), j = (int)((c / nx) % ny);
    const double* p = phi + (c - (int64_t)j * nx - i);  // this grid's row 0
    const double* row = p + (size_t)j * nx;
    // odd extension across the walls: phi(-1) = -phi(1), phi(n) = -phi(n-2)
    const double xr = (i + 1 < nx) ? row[i + 1] : -row[nx - 2];
    const double xl = (i > 0) ? row[i - 1] : -row[1];
    const double yu = (j + 1 < ny) ? p[(size_t)(j + 1) * nx + i] : -p[(size_t)(ny - 2) * nx + i];
    const double yd = (j > 0) ? p[(size_t)(j - 1) * nx + i] : -p[(size_t)nx + i];
    E[c] = make_double2(-(xr - xl) * inv2hx, -(yu - yd) * inv2hy);
  }
}

std::vector<double2> twiddles_p(int M) {
  std::vector<double2> t(M / 2);
  for (int k = 0; k < M / 2; ++k) {
    const double ang = -2.0 * M_PI * (double)k / (double)M;
    t[k] = make_double2(std::cos(ang), std::sin(ang));
  }
  return t;
}

bool pow2p(int v) { return v > 0 && (v & (v - 1)) == 0; }

}  // namespace

sc_status pipe_create(sc_grid* g) {
  const int nx = g->nx, ny = g->ny;
  if (!pow2p(nx - 1) || !pow2p(ny - 1) || nx - 1 < 8 || ny - 1 < 8 || nx - 1 > 512 || ny - 1 > 512)
    return set_error(SC_ERR_UNSUPPORTED, "pipe solve needs nx - 1, ny - 1 powers of two in [8, 512]");
  PipePlan& f = g->pipe;
  const int Px = 2 * (nx - 1), Py = 2 * (ny - 1);
  const auto twx = twiddles_p(Px), twy = twiddles_p(Py);
  // 1 / lambda_pq for q = 1..ny-2 (rows), p = 1..nx-2 (columns)
  std::vector<double> il((size_t)nx * ny, 0.0);
  for (int q = 1; q <= ny - 2; ++q)
    for (int p = 1; p <= nx - 2; ++p) {
      const double sp = std::sin(M_PI * p / Px), sq = std::sin(M_PI * q / Py);
      il[(size_t)q * nx + p] = 1.0 / (-4.0 * (sp * sp / (g->hx * g->hx) + sq * sq / (g->hy * g->hy)));
    }
  const size_t cells = (size_t)g->nstack * nx * ny;
  if (cudaMalloc(&f.twx, twx.size() * sizeof(double2)) != cudaSuccess ||
      cudaMalloc(&f.twy, twy.size() * sizeof(double2)) != cudaSuccess ||
      cudaMalloc(&f.inv_lam, il.size() * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&f.T1, cells * sizeof(double)) != cudaSuccess || cudaMalloc(&f.T2, cells * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&f.phi, cells * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return set_error(SC_ERR_OOM, "pipe_create: cudaMalloc failed");
  }
  SC_CUDA(cudaMemcpyAsync(f.twx, twx.data(), twx.size() * sizeof(double2), cudaMemcpyHostToDevice, g->stream));
  SC_CUDA(cudaMemcpyAsync(f.twy, twy.data(), twy.size() * sizeof(double2), cudaMemcpyHostToDevice, g->stream));
  SC_CUDA(cudaMemcpyAsync(f.inv_lam, il.data(), il.size() * sizeof(double), cudaMemcpyHostToDevice, g->stream));
  SC_CUDA(cudaMemsetAsync(f.phi, 0, cells * sizeof(double), g->stream));
  SC_CUDA(cudaMemsetAsync(f.T1, 0, cells * sizeof(double), g->stream));
  SC_CUDA(cudaMemsetAsync(f.T2, 0, cells * sizeof(double), g->stream));
  SC_CUDA(cudaStreamSynchronize(g->stream));
  const int smax = 3 * 1024 * (int)sizeof(double2);
  SC_CUDA(cudaFuncSetAttribute(pipe_columns, cudaFuncAttributeMaxDynamicSharedMemorySize, smax));
  return SC_OK;
}

void pipe_destroy(sc_grid* g) {
  PipePlan& f = g->pipe;
  cudaFree(f.twx);
  cudaFree(f.twy);
  cudaFree(f.inv_lam);
  cudaFree(f.T1);
  cudaFree(f.T2);
  cudaFree(f.phi);
  f = PipePlan{};
}

sc_status pipe_solve(sc_grid* g, bool zero_q) {
  const int nx = g->nx, ny = g->ny;
  PipePlan& f = g->pipe;
  const double scale = 1.0 / 1099511627776.0 / (double)(g->n_particles > 0 ? g->n_particles : 1);
  const double fac = -2.0 * M_PI / (g->hx * g->hy);
  const unsigned nz = (unsigned)g->nstack;
  const double norm = 1.0 / (4.0 * (double)(nx - 1) * (double)(ny - 1));
  SC_CUDA(launch_pdl(pipe_rows, dim3(ny - 2, nz), dim3(nx - 1), 2 * 2 * (nx - 1) * sizeof(double2), g->stream,
                     (const unsigned long long*)g->Q, nx, ny, scale, (const double*)g->stack_scale, fac, f.T1,
                     (const double2*)f.twx));
  SC_CUDA(launch_pdl(pipe_columns, dim3(nx - 2, nz), dim3(ny - 1), 3 * 2 * (ny - 1) * sizeof(double2), g->stream,
                     (const double*)f.T1, nx, ny, (const double*)f.inv_lam, f.T2, (const double2*)f.twy,
                     zero_q ? g->Q : (unsigned long long*)nullptr));
  SC_CUDA(launch_pdl(pipe_rows_inv, dim3(ny - 2, nz), dim3(nx - 1), 2 * 2 * (nx - 1) * sizeof(double2), g->stream,
                     (const double*)f.T2, nx, ny, norm, f.phi, (const double2*)f.twx));
  int dev = 0, sms = 0;
  SC_CUDA(cudaGetDevice(&dev));
  SC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int64_t total = (int64_t)nz * nx * ny;
  const int blocks = (int)std::min<int64_t>((total + 255) / 256, (int64_t)sms * 8);
  SC_CUDA(launch_pdl(pipe_fields, dim3(blocks), dim3(256), 0, g->stream, (const double*)f.phi, nx, ny, (int)nz,
                     0.5 / g->hx, 0.5 / g->hy, g->E));
  return SC_OK;
}

}  // namespace sc
