// Open-boundary Poisson solve in float64 by FFT convolution (the plain form).
//
// Hockney's method (cited in Sec. I): the charge q (nx x ny) is zero-padded
// to the doubled grid (Mx = 2nx, My = 2ny) and convolved cyclically with the
// free-space kernel.  Instead of the potential, the convolution kernels are
// the centred differences of G = -ln r,
//   Dx(d) = -(G(d + ex) - G(d - ex)) / (2 hx),   Dy likewise,
// so one convolution gives E = -grad phi at the nodes directly (the same
// numbers as differencing phi, without the cancellation).  Dx is odd in x and
// even in y, so its spectrum is i*Sx with Sx real; likewise Dy.
//
// Three kernels, each one FFT direction per block in shared memory
// (Stockham radix-2, float64):
//   rows_fwd  : q row j (real, zero-padded)        -> F1[j][p], p = 0..nx
//   columns   : F1[:, p] -> F(p, k) -> i Sx F, i Sy F -> inverse over k, keep j < ny
//   rows_inv  : Hermitian half rows -> Ex, Ey at the nx x ny nodes.
#include <complex>
#include <vector>

#include "fft_smem.cuh"

namespace sc {

namespace {

__global__ void fft64_rows_fwd(const unsigned long long* __restrict__ Q, int nx, double scale,
                               const double* __restrict__ stack_scale,
                               double2* __restrict__ F1, const double2* __restrict__ twx) {
  extern __shared__ double2 sm[];
  const int Mx = 2 * nx, j = blockIdx.x, t = threadIdx.x;
  // slice blockIdx.y: its charge grid and its row transforms
  Q += (size_t)blockIdx.y * gridDim.x * nx;
  F1 += (size_t)blockIdx.y * gridDim.x * (nx + 1);
  double2 *a = sm, *b = sm + Mx;
  pdl_wait();
  if (stack_scale) scale = stack_scale[blockIdx.y];  // per stacked grid (bunches of a batch)
  a[t] = make_double2((double)Q[(size_t)j * nx + t] * scale, 0.0);
  a[t + nx] = make_double2(0.0, 0.0);
  __syncthreads();
  const double2* r = fft_smem<false>(a, b, Mx, twx);
  pdl_allow();
  for (int p = t; p <= nx; p += nx) F1[(size_t)j * (nx + 1) + p] = r[p];
}

__global__ void fft64_columns(const double2* __restrict__ F1, int nx, int ny, const double* __restrict__ Sx,
                              const double* __restrict__ Sy, double2* __restrict__ Hx, double2* __restrict__ Hy,
                              const double2* __restrict__ twy, unsigned long long* Qzero) {
  extern __shared__ double2 sm[];
  const int My = 2 * ny, p = blockIdx.x, t = threadIdx.x;
  double2 *A = sm, *B = sm + My, *C = sm + 2 * My, *D = sm + 3 * My;
  const size_t so = (size_t)blockIdx.y * ny * (nx + 1);  // slice blockIdx.y
  F1 += so;
  Hx += so;
  Hy += so;
  pdl_wait();
  if (Qzero) {  // the row transform has read every slice's charge: clear it for the next deposit
    const int64_t total = (int64_t)gridDim.y * nx * ny;
    for (int64_t c = ((int64_t)blockIdx.y * gridDim.x + blockIdx.x) * blockDim.x + t; c < total;
         c += (int64_t)gridDim.x * gridDim.y * blockDim.x)
      Qzero[c] = 0ull;
  }
  A[t] = F1[(size_t)t * (nx + 1) + p];
  A[t + ny] = make_double2(0.0, 0.0);
  __syncthreads();
  double2* R = fft_smem<false>(A, B, My, twy);
  double2* freebuf = (R == A) ? B : A;
  for (int k = t; k < My; k += ny) {
    const double2 f = R[k];
    const double sx = Sx[(size_t)k * (nx + 1) + p], sy = Sy[(size_t)k * (nx + 1) + p];
    C[k] = make_double2(-sx * f.y, sx * f.x);
    D[k] = make_double2(-sy * f.y, sy * f.x);
  }
  __syncthreads();
  const double2* rx = fft_smem<true>(C, freebuf, My, twy);
  const double2* ry = fft_smem<true>(D, R, My, twy);
  pdl_allow();
  Hx[(size_t)t * (nx + 1) + p] = rx[t];
  Hy[(size_t)t * (nx + 1) + p] = ry[t];
}

__global__ void fft64_rows_inv(const double2* __restrict__ Hx, const double2* __restrict__ Hy, int nx,
                               double inv_norm, double2* __restrict__ E, const double2* __restrict__ twx) {
  extern __shared__ double2 sm[];
  const int Mx = 2 * nx, j = blockIdx.x, t = threadIdx.x;
  double2 *A = sm, *B = sm + Mx, *C = sm + 2 * Mx, *D = sm + 3 * Mx;
  const size_t so = (size_t)blockIdx.y * gridDim.x * (nx + 1);  // slice blockIdx.y
  E += (size_t)blockIdx.y * gridDim.x * nx;
  const double2* hx = Hx + so + (size_t)j * (nx + 1);
  const double2* hy = Hy + so + (size_t)j * (nx + 1);
  pdl_wait();
  // p = t (<= nx) straight from the half spectrum; p = t + nx from Hermitian symmetry
  A[t] = hx[t];
  C[t] = hy[t];
  {
    const int pp = t + nx;
    if (pp == nx) {
      A[pp] = hx[nx];
      C[pp] = hy[nx];
    } else {
      const double2 vx = hx[Mx - pp], vy = hy[Mx - pp];
      A[pp] = make_double2(vx.x, -vx.y);
      C[pp] = make_double2(vy.x, -vy.y);
    }
  }
  __syncthreads();
  const double2* rx = fft_smem<true>(A, B, Mx, twx);
  const double2* ry = fft_smem<true>(C, D, Mx, twx);
  pdl_allow();
  E[(size_t)j * nx + t] = make_double2(rx[t].x * inv_norm, ry[t].x * inv_norm);
}

// Iterative radix-2 FFT on the host (used once per grid for the kernel spectra).
void host_fft(std::complex<double>* a, int n, int stride) {
  for (int i = 1, j = 0; i < n; ++i) {
    int bit = n >> 1;
    for (; j & bit; bit >>= 1) j ^= bit;
    j ^= bit;
    if (i < j) std::swap(a[(size_t)i * stride], a[(size_t)j * stride]);
  }
  for (int len = 2; len <= n; len <<= 1) {
    const double ang = -2.0 * M_PI / len;
    for (int i = 0; i < n; i += len)
      for (int k = 0; k < len / 2; ++k) {
        const std::complex<double> w(std::cos(ang * k), std::sin(ang * k));
        std::complex<double>& u = a[(size_t)(i + k) * stride];
        std::complex<double>& v = a[(size_t)(i + k + len / 2) * stride];
        const std::complex<double> t = v * w;
        v = u - t;
        u = u + t;
      }
  }
}

void host_fft2(std::vector<std::complex<double>>& a, int Mx, int My) {
  for (int b = 0; b < My; ++b) host_fft(a.data() + (size_t)b * Mx, Mx, 1);
  for (int c = 0; c < Mx; ++c) host_fft(a.data() + c, My, Mx);
}

std::vector<double2> twiddles(int M) {
  std::vector<double2> t(M / 2);
  for (int k = 0; k < M / 2; ++k) {
    const double ang = -2.0 * M_PI * (double)k / (double)M;
    t[k] = make_double2(std::cos(ang), std::sin(ang));
  }
  return t;
}

bool pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

}  // namespace

// Cyclic free-space Green's function on the doubled grid and its centred
// differences.  G(dx, dy) = -1/2 ln(dx^2 + dy^2); the node's own cell uses the
// cell average of -ln r,  G0 = -(ab(ln(a^2+b^2) - 3) + a^2 atan(b/a) +
// b^2 atan(a/b)) / (2ab), a = hx/2, b = hy/2.  Index c of an axis of length
// M = 2n holds offset c for c <= n and c - M above.
void build_field_kernels(const sc_grid* g, double* Dx, double* Dy) {
  const int nx = g->nx, ny = g->ny, Mx = 2 * nx, My = 2 * ny;
  const double hx = g->hx, hy = g->hy;
  std::vector<double> G((size_t)Mx * My);
  const double a = 0.5 * hx, b = 0.5 * hy;
  const double g0 = -(a * b * (std::log(a * a + b * b) - 3.0) + a * a * std::atan(b / a) + b * b * std::atan(a / b)) /
                    (2.0 * a * b);
  for (int r = 0; r < My; ++r) {
    const int dj = r <= ny ? r : r - My;
    for (int c = 0; c < Mx; ++c) {
      const int di = c <= nx ? c : c - Mx;
      const double dx = di * hx, dy = dj * hy;
      G[(size_t)r * Mx + c] = (di == 0 && dj == 0) ? g0 : -0.5 * std::log(dx * dx + dy * dy);
    }
  }
  for (int r = 0; r < My; ++r)
    for (int c = 0; c < Mx; ++c) {
      const int cp = (c + 1) % Mx, cm = (c + Mx - 1) % Mx;
      const int rp = (r + 1) % My, rm = (r + My - 1) % My;
      Dx[(size_t)r * Mx + c] = -(G[(size_t)r * Mx + cp] - G[(size_t)r * Mx + cm]) / (2.0 * hx);
      Dy[(size_t)r * Mx + c] = -(G[(size_t)rp * Mx + c] - G[(size_t)rm * Mx + c]) / (2.0 * hy);
    }
}

sc_status fft64_create(sc_grid* g) {
  const int nx = g->nx, ny = g->ny, Mx = 2 * nx, My = 2 * ny;
  if (!pow2(nx) || !pow2(ny) || nx < 8 || ny < 8 || nx > 512 || ny > 512)
    return set_error(SC_ERR_UNSUPPORTED, "float64 FFT solve needs power-of-two nx, ny in [8, 512]");
  Fft64Plan& f = g->fft;
  f.M = Mx;
  std::vector<double> Dx((size_t)Mx * My), Dy((size_t)Mx * My);
  build_field_kernels(g, Dx.data(), Dy.data());
  std::vector<std::complex<double>> cx((size_t)Mx * My), cy((size_t)Mx * My);
  for (size_t i = 0; i < cx.size(); ++i) {
    cx[i] = Dx[i];
    cy[i] = Dy[i];
  }
  host_fft2(cx, Mx, My);
  host_fft2(cy, Mx, My);
  std::vector<double> Sx((size_t)My * (nx + 1)), Sy((size_t)My * (nx + 1));
  for (int k = 0; k < My; ++k)
    for (int p = 0; p <= nx; ++p) {
      Sx[(size_t)k * (nx + 1) + p] = cx[(size_t)k * Mx + p].imag();
      Sy[(size_t)k * (nx + 1) + p] = cy[(size_t)k * Mx + p].imag();
    }
  const auto twx = twiddles(Mx), twy = twiddles(My);
  const size_t half = (size_t)g->nstack * ny * (nx + 1) * sizeof(double2);  // one set per stacked grid
  if (cudaMalloc(&f.twx, twx.size() * sizeof(double2)) != cudaSuccess ||
      cudaMalloc(&f.twy, twy.size() * sizeof(double2)) != cudaSuccess || cudaMalloc(&f.F1, half) != cudaSuccess ||
      cudaMalloc(&f.Hx, half) != cudaSuccess || cudaMalloc(&f.Hy, half) != cudaSuccess ||
      cudaMalloc(&f.Sx, Sx.size() * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&f.Sy, Sy.size() * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return set_error(SC_ERR_OOM, "fft64_create: cudaMalloc failed");
  }
  SC_CUDA(cudaMemcpyAsync(f.twx, twx.data(), twx.size() * sizeof(double2), cudaMemcpyHostToDevice, g->stream));
  SC_CUDA(cudaMemcpyAsync(f.twy, twy.data(), twy.size() * sizeof(double2), cudaMemcpyHostToDevice, g->stream));
  SC_CUDA(cudaMemcpyAsync(f.Sx, Sx.data(), Sx.size() * sizeof(double), cudaMemcpyHostToDevice, g->stream));
  SC_CUDA(cudaMemcpyAsync(f.Sy, Sy.data(), Sy.size() * sizeof(double), cudaMemcpyHostToDevice, g->stream));
  SC_CUDA(cudaStreamSynchronize(g->stream));
  const int smax = 4 * 1024 * (int)sizeof(double2);
  SC_CUDA(cudaFuncSetAttribute(fft64_columns, cudaFuncAttributeMaxDynamicSharedMemorySize, smax));
  SC_CUDA(cudaFuncSetAttribute(fft64_rows_inv, cudaFuncAttributeMaxDynamicSharedMemorySize, smax));
  SC_CUDA(cudaFuncSetAttribute(fft64_rows_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, smax));
  return SC_OK;
}

void fft64_destroy(sc_grid* g) {
  Fft64Plan& f = g->fft;
  cudaFree(f.twx);
  cudaFree(f.twy);
  cudaFree(f.F1);
  cudaFree(f.Hx);
  cudaFree(f.Hy);
  cudaFree(f.Sx);
  cudaFree(f.Sy);
  f = Fft64Plan{};
}

sc_status fft64_solve(sc_grid* g, bool zero_q) {
  const int nx = g->nx, ny = g->ny, Mx = 2 * nx, My = 2 * ny;
  Fft64Plan& f = g->fft;
  const double scale = 1.0 / 1099511627776.0 / (double)(g->n_particles > 0 ? g->n_particles : 1);
  const unsigned nz = (unsigned)g->nstack;
  SC_CUDA(launch_pdl(fft64_rows_fwd, dim3(ny, nz), dim3(nx), 2 * Mx * sizeof(double2), g->stream,
                     (const unsigned long long*)g->Q, nx, scale, (const double*)g->stack_scale, f.F1,
                     (const double2*)f.twx));
  SC_CUDA(launch_pdl(fft64_columns, dim3(nx + 1, nz), dim3(ny), 4 * My * sizeof(double2), g->stream,
                     (const double2*)f.F1, nx, ny, (const double*)f.Sx, (const double*)f.Sy, f.Hx, f.Hy,
                     (const double2*)f.twy, zero_q ? g->Q : (unsigned long long*)nullptr));
  SC_CUDA(launch_pdl(fft64_rows_inv, dim3(ny, nz), dim3(nx), 4 * Mx * sizeof(double2), g->stream, (const double2*)f.Hx,
                     (const double2*)f.Hy, nx, 1.0 / ((double)Mx * (double)My), g->E, (const double2*)f.twx));
  return SC_OK;
}

}  // namespace sc
