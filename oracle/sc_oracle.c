/*
 * sc_oracle.c -- plain, slow, obviously-correct FP64 CPU reference of the
 * 2-D particle-in-cell space-charge step (Kurimoto, "Particle Tracking with
 * Space Charge Effects using GPU", arXiv:2010.11540).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library.  It shares
 * no code, header, table or helper with the CUDA path.  Build with
 * -ffp-contract=off so that every product and sum below is rounded exactly as
 * written (no fused multiply-add).
 *
 * Threads (orc_set_threads, default 1): with OpenMP the particle loops of the
 * deposit, kicks and push are split over threads.  Each particle's arithmetic
 * is the same whatever the split, and the deposit's integer sums do not depend
 * on their order (each thread fills its own zeroed grid over a contiguous
 * range of particles, and the grids are added afterwards), so the results are
 * bit-identical to one thread.  Moments stay sequential (floating-point sums
 * in particle order).
 *
 * Contents, each following the passage cited at the function:
 *   orc_deposit        Sec. IV-A, CIC charge-assignment equation (4 weights),
 *                      in 2^-20 fixed point per axis, uint64 accumulation;
 *                      optionally into one of nz longitudinal slices by sigma
 *                      (the line density lambda(z) of Sec. IV as a histogram
 *                      of sigma, each bin with its own transverse grid).
 *   orc_green_self     cell-averaged -ln r (self term of the open-boundary
 *                      Green's function; the paper is silent on it).
 *   orc_green_cyclic   Hockney's zero-padded free-space Green's function
 *                      G = -ln r laid out on the doubled (2nx x 2ny) grid.
 *   orc_potential_direct  direct pairwise sum phi = sum G q (definition).
 *   orc_fields         E = -grad phi by centred differences (Sec. IV-C, the
 *                      field equation, with bilinear gather in place of the
 *                      Bezier surface).
 *   orc_kick           Sec. IV, transverse kick equation, bilinear gather.
 *   orc_push           Sec. III: exact drift (III-A), thick chromatic
 *                      quadrupole (III-B), thin sextupole (III-C, V of the
 *                      H0+V split), linear sector dipole (H_approx with
 *                      curvature), thin RF kick (Sec. V mentions RF cavities).
 *   orc_moments        Sec. V: rms sizes / emittances from beam moments.
 *
 * Parity pins live in tests/test_oracle_*.py.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
  int32_t type, pad;
  double length, k1, k2l, angle, volt, harmonic, lag;
} orc_elem;

typedef struct {
  double gamma0, beta0, n_lambda, r_p, circumference, mass_ev;
} orc_beam;

enum { ORC_DRIFT = 0, ORC_QUAD = 1, ORC_SEXT = 2, ORC_BEND = 3, ORC_RF = 4, ORC_MARK = 5, ORC_EXACT_BEND = 6 };

static const double ORC_ONE_FX = 1048576.0; /* 2^20 */

/* Threads of the particle loops (1 without OpenMP). */
static int orc_threads = 1;

int orc_set_threads(int n) {
#ifdef _OPENMP
  orc_threads = n < 1 ? 1 : n;
#else
  (void)n;
  orc_threads = 1;
#endif
  return orc_threads;
}

int orc_max_threads(void) {
#ifdef _OPENMP
  return omp_get_num_procs();
#else
  return 1;
#endif
}

/* ---------------------------------------------------------------------
 * Charge deposition, Sec. IV-A (CIC equation).  Grid nodes are
 * x_i = xmin + i*hx, i = 0..nx-1 (same for y); inv_hx = 1/hx is passed in.
 * A particle with xi = (x - xmin)*inv_hx, eta = (y - ymin)*inv_hy lies in
 * cell (i, j) = (floor xi, floor eta) with fractions fx = xi - i, fy = eta - j.
 * It is inside iff 0 <= xi < nx-1 and 0 <= eta < ny-1; outside particles
 * deposit nothing and are counted (return value).
 * The paper's weights (x_{i+1}-x)(y_{j+1}-y)/(dx dy), ... are taken at 2^-20
 * resolution per axis: ax = rint(fx*2^20), bx = 2^20 - ax, and Q (uint64,
 * Q[j*nx + i]) gets bx*by, ax*by, bx*ay, ax*ay at (i,j), (i+1,j), (i,j+1),
 * (i+1,j+1).  Each particle adds exactly 2^40.  Q is accumulated, not zeroed.
 * ------------------------------------------------------------------- */
/* Slice of a particle: zeta = (sg - zmin)*inv_dz (two roundings), slice
 * k = floor(zeta), valid iff 0 <= zeta < nz.  nz == 1 means no slicing
 * (every particle is in slice 0). */
static int orc_slice(double sg, int nz, double zmin, double inv_dz) {
  if (nz <= 1) return 0;
  double zeta = (sg - zmin) * inv_dz;
  if (!(zeta >= 0.0 && zeta < (double)nz)) return -1;
  return (int)floor(zeta);
}

static uint64_t orc_deposit_range(int64_t p0, int64_t p1, const double *x, const double *y, const double *sg,
                                  int nx, int ny, double xmin, double ymin, double inv_hx, double inv_hy, int nz,
                                  double zmin, double inv_dz, uint64_t *Q) {
  uint64_t n_out = 0;
  for (int64_t p = p0; p < p1; ++p) {
    int k = orc_slice(sg ? sg[p] : 0.0, nz, zmin, inv_dz);
    double xi = (x[p] - xmin) * inv_hx;
    double eta = (y[p] - ymin) * inv_hy;
    if (k < 0 || !(xi >= 0.0 && xi < (double)(nx - 1) && eta >= 0.0 && eta < (double)(ny - 1))) {
      ++n_out;
      continue;
    }
    double fi = floor(xi), fj = floor(eta);
    int i = (int)fi, j = (int)fj;
    double fx = xi - fi, fy = eta - fj;
    uint64_t ax = (uint64_t)llrint(fx * ORC_ONE_FX);
    uint64_t ay = (uint64_t)llrint(fy * ORC_ONE_FX);
    uint64_t bx = (uint64_t)ORC_ONE_FX - ax;
    uint64_t by = (uint64_t)ORC_ONE_FX - ay;
    uint64_t *q = Q + (int64_t)k * nx * ny;
    q[(int64_t)j * nx + i] += bx * by;
    q[(int64_t)j * nx + i + 1] += ax * by;
    q[(int64_t)(j + 1) * nx + i] += bx * ay;
    q[(int64_t)(j + 1) * nx + i + 1] += ax * ay;
  }
  return n_out;
}

uint64_t orc_deposit_sliced(int64_t n, const double *x, const double *y, const double *sg, int nx, int ny,
                            double xmin, double ymin, double inv_hx, double inv_hy, int nz, double zmin,
                            double inv_dz, uint64_t *Q) {
  int nt = orc_threads;
  if (n < 4096) nt = 1;
  uint64_t *priv = 0;
  size_t cells = (size_t)nx * ny * nz;
  if (nt > 1) priv = (uint64_t *)calloc((size_t)(nt - 1) * cells, sizeof(uint64_t));
  if (!priv) return orc_deposit_range(0, n, x, y, sg, nx, ny, xmin, ymin, inv_hx, inv_hy, nz, zmin, inv_dz, Q);
  uint64_t n_out = 0;
#pragma omp parallel for num_threads(nt) schedule(static, 1) reduction(+ : n_out)
  for (int t = 0; t < nt; ++t) {
    /* thread t: particles [n t / nt, n (t+1) / nt) into Q (t = 0) or its own zeroed grid */
    uint64_t *dst = t == 0 ? Q : priv + (size_t)(t - 1) * cells;
    n_out += orc_deposit_range(n * t / nt, n * (t + 1) / nt, x, y, sg, nx, ny, xmin, ymin, inv_hx, inv_hy, nz, zmin,
                               inv_dz, dst);
  }
  for (int t = 1; t < nt; ++t)
    for (size_t c = 0; c < cells; ++c) Q[c] += priv[(size_t)(t - 1) * cells + c];
  free(priv);
  return n_out;
}

uint64_t orc_deposit(int64_t n, const double *x, const double *y, int nx, int ny, double xmin, double ymin,
                     double inv_hx, double inv_hy, uint64_t *Q) {
  return orc_deposit_sliced(n, x, y, 0, nx, ny, xmin, ymin, inv_hx, inv_hy, 1, 0.0, 0.0, Q);
}

/* ---------------------------------------------------------------------
 * Open-boundary Green's function of the 2-D Poisson equation (Sec. IV,
 * Eq. poisson3D with u -> the free-space part; Hockney's method cited in
 * Sec. I).  With potential normalised so that a unit line charge gives
 * phi = -ln r, G(dx, dy) = -1/2 ln(dx^2 + dy^2).
 * Self term G(0,0): mean of -ln r over the hx x hy cell centred on the node,
 *   = -(1/(2ab)) * I(a,b), a = hx/2, b = hy/2,
 *   I(a,b) = int_0^a int_0^b ln(x^2+y^2) dy dx
 *          = ab(ln(a^2+b^2) - 3) + a^2 atan(b/a) + b^2 atan(a/b).
 * ------------------------------------------------------------------- */
double orc_green_self(double hx, double hy) {
  double a = 0.5 * hx, b = 0.5 * hy;
  double I = a * b * (log(a * a + b * b) - 3.0) + a * a * atan(b / a) + b * b * atan(a / b);
  return -I / (2.0 * a * b);
}

static double orc_green_at(int di, int dj, double hx, double hy) {
  if (di == 0 && dj == 0) return orc_green_self(hx, hy);
  double dx = di * hx, dy = dj * hy;
  return -0.5 * log(dx * dx + dy * dy);
}

/* G on the doubled grid, cyclic: index a in [0, 2nx) holds offset a for
 * a <= nx and a - 2nx for a > nx (index nx holds offset nx, which equals
 * offset -nx by symmetry); the same for b.  Layout Gc[b*(2nx) + a]. */
void orc_green_cyclic(int nx, int ny, double hx, double hy, double *Gc) {
  int Mx = 2 * nx, My = 2 * ny;
  for (int b = 0; b < My; ++b) {
    int dj = (b <= ny) ? b : b - My;
    for (int a = 0; a < Mx; ++a) {
      int di = (a <= nx) ? a : a - Mx;
      Gc[(int64_t)b * Mx + a] = orc_green_at(di, dj, hx, hy);
    }
  }
}

/* Direct pairwise sum (the definition of the open-boundary convolution):
 * phi(i, j) = sum_{k,l} G((i-k)hx, (j-l)hy) q[l*nx + k] for the extended node
 * range i = -1..nx, j = -1..ny; output phi_ext[(j+1)*(nx+2) + (i+1)]. */
void orc_potential_direct(int nx, int ny, double hx, double hy, const double *q, double *phi_ext) {
  int ex = nx + 2;
  for (int j = -1; j <= ny; ++j)
    for (int i = -1; i <= nx; ++i) {
      double s = 0.0;
      for (int l = 0; l < ny; ++l)
        for (int k = 0; k < nx; ++k) {
          double ql = q[(int64_t)l * nx + k];
          if (ql != 0.0) s += orc_green_at(i - k, j - l, hx, hy) * ql;
        }
      phi_ext[(int64_t)(j + 1) * ex + (i + 1)] = s;
    }
}

/* E = -grad phi at the nx x ny nodes by centred differences, using the
 * potential on the surrounding ring of nodes (i = -1, nx; j = -1, ny), which
 * the open-boundary solution defines.  Ex[j*nx+i], Ey[j*nx+i]. */
void orc_fields(int nx, int ny, double hx, double hy, const double *phi_ext, double *Ex, double *Ey) {
  int ex = nx + 2;
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      double pxp = phi_ext[(int64_t)(j + 1) * ex + (i + 2)];
      double pxm = phi_ext[(int64_t)(j + 1) * ex + (i + 0)];
      double pyp = phi_ext[(int64_t)(j + 2) * ex + (i + 1)];
      double pym = phi_ext[(int64_t)(j + 0) * ex + (i + 1)];
      Ex[(int64_t)j * nx + i] = -(pxp - pxm) / (2.0 * hx);
      Ey[(int64_t)j * nx + i] = -(pyp - pym) / (2.0 * hy);
    }
}

/* ---------------------------------------------------------------------
 * Space-charge kick, Sec. IV (transverse kick equation), optionally per
 * longitudinal slice (E arrays then hold nz grids):
 *   dp = -(e lambda / (m gamma0^3 beta0^2 c^2)) grad u * L,
 * with u normalised per unit line charge.  In the normalisation above this
 * is dpx = K * L * Ex, dpy = K * L * Ey, K = 2 r_p N_lambda / (beta0^2 gamma0^3),
 * and kl = K * L is passed in.  E at the particle is the bilinear
 * interpolation of the node fields with the same cell and fractions as the
 * deposit (float64 fractions).  Particles outside the grid get no kick.
 * ------------------------------------------------------------------- */
void orc_kick_sliced(int64_t n, const double *x, const double *y, const double *sg, double *px, double *py,
                     int nx, int ny, double xmin, double ymin, double inv_hx, double inv_hy, int nz, double zmin,
                     double inv_dz, const double *Ex, const double *Ey, double kl) {
#pragma omp parallel for num_threads(orc_threads) schedule(static)
  for (int64_t p = 0; p < n; ++p) {
    int k = orc_slice(sg ? sg[p] : 0.0, nz, zmin, inv_dz);
    double xi = (x[p] - xmin) * inv_hx;
    double eta = (y[p] - ymin) * inv_hy;
    if (k < 0 || !(xi >= 0.0 && xi < (double)(nx - 1) && eta >= 0.0 && eta < (double)(ny - 1))) continue;
    double fi = floor(xi), fj = floor(eta);
    int i = (int)fi, j = (int)fj;
    double fx = xi - fi, fy = eta - fj;
    double w00 = (1.0 - fx) * (1.0 - fy), w10 = fx * (1.0 - fy);
    double w01 = (1.0 - fx) * fy, w11 = fx * fy;
    int64_t c = (int64_t)k * nx * ny + (int64_t)j * nx + i;
    double ex = w00 * Ex[c] + w10 * Ex[c + 1] + w01 * Ex[c + nx] + w11 * Ex[c + nx + 1];
    double ey = w00 * Ey[c] + w10 * Ey[c + 1] + w01 * Ey[c + nx] + w11 * Ey[c + nx + 1];
    px[p] += kl * ex;
    py[p] += kl * ey;
  }
}

/* ---------------------------------------------------------------------
 * Longitudinal space-charge kick, Sec. IV (longitudinal kick equation):
 *   dps = -(e / (m gamma0^2 beta0^2 c^2)) u dlambda/dz L.
 * In the normalisation of the transverse kick, lambda(z) u(x, y) is
 * N_lambda Phi_k(x, y), Phi_k the potential of slice k (its charge n_k/N
 * of a slice holding the whole bunch, -ln r normalisation), so
 *   dps = -(K gamma0) L dPhi/dz,   K gamma0 = 2 r_p N_lambda / (beta0^2 gamma0^2).
 * dPhi/dz is the centred difference of the neighbouring slices at the
 * particle's (x, y): (Phi_{k+1} - Phi_{k-1}) / (2 dz), Phi = 0 beyond the
 * first and the last slice (no charge there).  For a bunch whose transverse
 * shape does not change along z (the paper's assumption) Phi_k = lambda_k u and
 * this is the paper's u dlambda/dz.  Phi at the particle: bilinear, with the
 * cell and float64 fractions of the transverse kick.  klz = K gamma0 L / (2 dz).
 * phi holds nz grids [k][j][i] of node potentials.
 * ------------------------------------------------------------------- */
void orc_kick_long(int64_t n, const double *x, const double *y, const double *sg, double *ps, int nx, int ny,
                   double xmin, double ymin, double inv_hx, double inv_hy, int nz, double zmin, double inv_dz,
                   const double *phi, double klz) {
  int64_t cells = (int64_t)nx * ny;
#pragma omp parallel for num_threads(orc_threads) schedule(static)
  for (int64_t p = 0; p < n; ++p) {
    int k = orc_slice(sg[p], nz, zmin, inv_dz);
    double xi = (x[p] - xmin) * inv_hx;
    double eta = (y[p] - ymin) * inv_hy;
    if (k < 0 || !(xi >= 0.0 && xi < (double)(nx - 1) && eta >= 0.0 && eta < (double)(ny - 1))) continue;
    double fi = floor(xi), fj = floor(eta);
    int i = (int)fi, j = (int)fj;
    double fx = xi - fi, fy = eta - fj;
    double w00 = (1.0 - fx) * (1.0 - fy), w10 = fx * (1.0 - fy);
    double w01 = (1.0 - fx) * fy, w11 = fx * fy;
    int64_t c = (int64_t)j * nx + i;
    double up = 0.0, dn = 0.0;
    if (k + 1 < nz) {
      const double *f = phi + (int64_t)(k + 1) * cells + c;
      up = w00 * f[0] + w10 * f[1] + w01 * f[nx] + w11 * f[nx + 1];
    }
    if (k > 0) {
      const double *f = phi + (int64_t)(k - 1) * cells + c;
      dn = w00 * f[0] + w10 * f[1] + w01 * f[nx] + w11 * f[nx + 1];
    }
    ps[p] -= klz * (up - dn);
  }
}

/* ---------------------------------------------------------------------
 * Bezier gather of the potential, Sec. IV-C:
 *   u(x, y) = sum_{m,n=0..3} u_{i+m-1, j+n-1} B_m(tx) B_n(ty),
 *   B_m(t) = 3!/(m!(3-m)!) t^m (1-t)^(3-m),   E = -grad u.
 * Reading: the cubic's four control points are the nodes i-1 .. i+2, so its
 * parameter runs over them, tx = (x - x_{i-1}) / (3 hx) = (1 + fx)/3 (the
 * printed (x - x_i)/hx over one cell would triple every gradient: a linear
 * potential's printed dU/dx is 3 times its slope).  Linear potentials are then
 * reproduced exactly; for u = x^2 the surface is x^2 + 3 tx (1 - tx) hx^2 (the
 * Bernstein smoothing).  Nodes beyond the walls take the odd extension of the
 * pipe potential (u_{-1} = -u_1, u_{n} = -u_{n-2}).  Cell, fractions and
 * validity as orc_kick_sliced.
 * The kick: px += kl Ex, py += kl Ey; with klz != 0 also the longitudinal kick
 * of orc_kick_long with the neighbouring slices' u taken from the same
 * surface.  phi: nz grids [k][j][i] of node potentials.
 * ------------------------------------------------------------------- */
static double orc_phi_at(const double *phi, int nx, int ny, int i, int j) {
  double sgn = 1.0;
  if (i < 0) { i = -i; sgn = -sgn; }
  if (i > nx - 1) { i = 2 * (nx - 1) - i; sgn = -sgn; }
  if (j < 0) { j = -j; sgn = -sgn; }
  if (j > ny - 1) { j = 2 * (ny - 1) - j; sgn = -sgn; }
  return sgn * phi[(int64_t)j * nx + i];
}

static void orc_bernstein3(double t, double *b, double *db) {
  double u = 1.0 - t;
  b[0] = u * u * u;
  b[1] = 3.0 * t * u * u;
  b[2] = 3.0 * t * t * u;
  b[3] = t * t * t;
  db[0] = -3.0 * u * u;
  db[1] = 3.0 * u * u - 6.0 * t * u;
  db[2] = 6.0 * t * u - 3.0 * t * t;
  db[3] = 3.0 * t * t;
}

/* Value and gradient of the Bezier surface of grid `phi` in cell (i, j) at fractions (fx, fy). */
static void orc_bezier_eval(const double *phi, int nx, int ny, int i, int j, double fx, double fy, double hx,
                            double hy, double *u, double *dudx, double *dudy) {
  double bx[4], dbx[4], by[4], dby[4];
  orc_bernstein3((1.0 + fx) / 3.0, bx, dbx);
  orc_bernstein3((1.0 + fy) / 3.0, by, dby);
  double v = 0.0, gx = 0.0, gy = 0.0;
  for (int n = 0; n < 4; ++n)
    for (int m = 0; m < 4; ++m) {
      double c = orc_phi_at(phi, nx, ny, i + m - 1, j + n - 1);
      v += c * bx[m] * by[n];
      gx += c * dbx[m] * by[n];
      gy += c * bx[m] * dby[n];
    }
  *u = v;
  *dudx = gx / (3.0 * hx);
  *dudy = gy / (3.0 * hy);
}

void orc_bezier_point(const double *phi, int nx, int ny, double hx, double hy, int i, int j, double fx, double fy,
                      double *out3) {
  orc_bezier_eval(phi, nx, ny, i, j, fx, fy, hx, hy, &out3[0], &out3[1], &out3[2]);
}

void orc_kick_bezier(int64_t n, const double *x, const double *y, const double *sg, double *px, double *py,
                     double *ps, int nx, int ny, double xmin, double ymin, double inv_hx, double inv_hy, double hx,
                     double hy, int nz, double zmin, double inv_dz, const double *phi, double kl, double klz) {
  int64_t cells = (int64_t)nx * ny;
#pragma omp parallel for num_threads(orc_threads) schedule(static)
  for (int64_t p = 0; p < n; ++p) {
    int k = orc_slice(sg ? sg[p] : 0.0, nz, zmin, inv_dz);
    double xi = (x[p] - xmin) * inv_hx;
    double eta = (y[p] - ymin) * inv_hy;
    if (k < 0 || !(xi >= 0.0 && xi < (double)(nx - 1) && eta >= 0.0 && eta < (double)(ny - 1))) continue;
    double fi = floor(xi), fj = floor(eta);
    int i = (int)fi, j = (int)fj;
    double fx = xi - fi, fy = eta - fj;
    double u, gx, gy;
    orc_bezier_eval(phi + (int64_t)k * cells, nx, ny, i, j, fx, fy, hx, hy, &u, &gx, &gy);
    px[p] += kl * -gx;
    py[p] += kl * -gy;
    if (klz != 0.0) {
      double up = 0.0, dn = 0.0, a, b;
      if (k + 1 < nz) orc_bezier_eval(phi + (int64_t)(k + 1) * cells, nx, ny, i, j, fx, fy, hx, hy, &up, &a, &b);
      if (k > 0) orc_bezier_eval(phi + (int64_t)(k - 1) * cells, nx, ny, i, j, fx, fy, hx, hy, &dn, &a, &b);
      ps[p] -= klz * (up - dn);
    }
  }
}

void orc_kick(int64_t n, const double *x, const double *y, double *px, double *py, int nx, int ny, double xmin,
              double ymin, double inv_hx, double inv_hy, const double *Ex, const double *Ey, double kl) {
  orc_kick_sliced(n, x, y, 0, px, py, nx, ny, xmin, ymin, inv_hx, inv_hy, 1, 0.0, 0.0, Ex, Ey, kl);
}

/* ---------------------------------------------------------------------
 * Single-particle maps, Sec. III.  State (x, px, y, py, sg, ps) with
 * px = Px/p0, sg = s - c beta0 t, ps = p_sigma.
 * ------------------------------------------------------------------- */

/* Exact drift (Sec. III-A: field-free motion solved without approximation).
 * With (1+delta)^2 = 1 + 2 ps + beta0^2 ps^2 (Eq. BEND2) and
 * pz = sqrt((1+delta)^2 - px^2 - py^2):
 *   x += L px/pz,  y += L py/pz,  sg += L (1 - (1 + beta0^2 ps)/pz). */
static void orc_drift(double *s, double L, double beta0) {
  double px = s[1], py = s[3], ps = s[5];
  double opd2 = 1.0 + 2.0 * ps + beta0 * beta0 * ps * ps;
  double pz = sqrt(opd2 - px * px - py * py);
  s[0] += L * px / pz;
  s[2] += L * py / pz;
  s[4] += L * (1.0 - (1.0 + beta0 * beta0 * ps) / pz);
}

/* Flow of H0 = (px^2+py^2)/2 (1-ps) + ps^2/(2 gamma0^2) over L (the k1 -> 0
 * limit of the quadrupole below). */
static void orc_h0_drift(double *s, double L, double gamma0) {
  double px = s[1], py = s[3], ps = s[5];
  s[0] += px * (1.0 - ps) * L;
  s[2] += py * (1.0 - ps) * L;
  s[4] += ps * L / (gamma0 * gamma0) - 0.5 * (px * px + py * py) * L;
}

/* One transverse plane of the thick quadrupole (Sec. III-B), focusing
 * (foc = 1: cos/sin) or defocusing (foc = 0: cosh/sinh), with
 * w = sqrt(|k1| (1 - ps)), a = sqrt((1-ps)/|k1|), b = sqrt(|k1|/(1-ps)):
 *   focusing:   u = u0 cos wL + a pu0 sin wL,  pu = pu0 cos wL - b u0 sin wL
 *   defocusing: u = u0 cosh wL + a pu0 sinh wL, pu = pu0 cosh wL + b u0 sinh wL
 * Returns I = int_0^L pu(s)^2 ds in closed form (used by the sg equation). */
static double orc_quad_plane(double *u, double *pu, double absk1, double ps, double L, int foc) {
  double w = sqrt(absk1 * (1.0 - ps));
  double a = sqrt((1.0 - ps) / absk1);
  double b = sqrt(absk1 / (1.0 - ps));
  double u0 = *u, p0 = *pu, I;
  if (foc) {
    double c = cos(w * L), s = sin(w * L);
    *u = u0 * c + a * p0 * s;
    *pu = p0 * c - b * u0 * s;
    /* pu(s) = p0 cos(ws) - b u0 sin(ws) */
    double icc = 0.5 * L + s * c / (2.0 * w);  /* int cos^2 */
    double iss = 0.5 * L - s * c / (2.0 * w);  /* int sin^2 */
    double isc = s * s / (2.0 * w);            /* int sin cos */
    I = p0 * p0 * icc - 2.0 * p0 * b * u0 * isc + b * b * u0 * u0 * iss;
  } else {
    double c = cosh(w * L), s = sinh(w * L);
    *u = u0 * c + a * p0 * s;
    *pu = p0 * c + b * u0 * s;
    /* pu(s) = p0 cosh(ws) + b u0 sinh(ws) */
    double icc = 0.5 * L + s * c / (2.0 * w);   /* int cosh^2 */
    double iss = -0.5 * L + s * c / (2.0 * w);  /* int sinh^2 */
    double isc = s * s / (2.0 * w);             /* int sinh cosh */
    I = p0 * p0 * icc + 2.0 * p0 * b * u0 * isc + b * b * u0 * u0 * iss;
  }
  return I;
}

/* Thick quadrupole, Sec. III-B: x/y maps as printed (k1 > 0 focuses x;
 * k1 < 0 swaps the planes), and
 *   sg(L) = sg(0) + ps L / gamma0^2 - 1/2 int_0^L (px^2 + py^2) ds. */
static void orc_quad(double *s, double L, double k1, double gamma0) {
  if (k1 == 0.0) { orc_h0_drift(s, L, gamma0); return; }
  double ps = s[5], absk1 = fabs(k1);
  double Ix = orc_quad_plane(&s[0], &s[1], absk1, ps, L, k1 > 0.0);
  double Iy = orc_quad_plane(&s[2], &s[3], absk1, ps, L, k1 < 0.0);
  s[4] += ps * L / (gamma0 * gamma0) - 0.5 * (Ix + Iy);
}

/* Thin sextupole: the V = k2 (x^3 - 3 x y^2)/6 step of Eq. Sym2 taken as
 * one kick of integrated strength k2l:
 *   px -= k2l/2 (x^2 - y^2),  py += k2l x y. */
static void orc_sext(double *s, double k2l) {
  double x = s[0], y = s[2];
  s[1] -= 0.5 * k2l * (x * x - y * y);
  s[3] += k2l * x * y;
}

/* Thick sextupole, Sec. III-C: H_approx = H0 + V with
 * H0 = (px^2+py^2)/2 (1-ps) + ps^2/(2 gamma0^2) and V = k2 (x^3 - 3 x y^2)/6,
 * k2 = k2l / L, integrated by the symplectic split of Eq. Sym2,
 *   exp(H0 a L) exp(V b L) exp(H0 c L) exp(V b L) exp(H0 a L),
 * a = (1 - 1/sqrt 3)/2, b = 1/2, c = 1/sqrt 3 (the V steps are kicks of
 * integrated strength k2 b L = k2l/2). */
static void orc_thick_sext(double *s, double L, double k2l, double gamma0) {
  const double a = 0.5 * (1.0 - 1.0 / sqrt(3.0)), c = 1.0 / sqrt(3.0);
  orc_h0_drift(s, a * L, gamma0);
  orc_sext(s, 0.5 * k2l);
  orc_h0_drift(s, c * L, gamma0);
  orc_sext(s, 0.5 * k2l);
  orc_h0_drift(s, a * L, gamma0);
}

/* Exact sector dipole (Sec. III-A: uniform field solved without H_approx,
 * Eqs. BEND1, BEND2 and the transformation to (x, sg) at the exit face, with
 * the printed sqrt(x~ + z~) read as sqrt(x~^2 + z~^2)).  Worked out in the
 * bending plane: the particle circles with radius rho P, P^2 = (1+delta)^2 -
 * py^2, about C = (rho + x0 - rho pz0, rho px0) (rho = L/angle, origin at the
 * reference orbit's centre); the exit face is the ray at `angle`.  With
 * pz0 = sqrt(P^2 - px0^2), C = cos(angle), S = sin(angle):
 *   px = px0 C + (pz0 - 1 - x0/rho) S,         pz = sqrt(P^2 - px^2),
 *   x  = (x0 + rho (1 - pz0)) C + rho px0 S + rho (pz - 1),
 *   alpha = angle + asin(px0/P) - asin(px/P)   (turn of the momentum),
 *   y += py rho alpha,  sg += L - (1 + beta0^2 ps) rho alpha,  py, ps const.
 * Zero angle: the exact drift. */
static void orc_exact_bend(double *s, double L, double angle, double beta0) {
  if (angle == 0.0) { orc_drift(s, L, beta0); return; }
  double rho = L / angle, C = cos(angle), S = sin(angle);
  double x0 = s[0], px0 = s[1], py = s[3], ps = s[5];
  double P2 = 1.0 + 2.0 * ps + beta0 * beta0 * ps * ps - py * py;
  double pz0 = sqrt(P2 - px0 * px0);
  double px = px0 * C + (pz0 - 1.0 - x0 / rho) * S;
  double pz = sqrt(P2 - px * px);
  double P = sqrt(P2);
  double alpha = angle + asin(px0 / P) - asin(px / P);
  s[0] = (x0 + rho * (1.0 - pz0)) * C + rho * px0 * S + rho * (pz - 1.0);
  s[1] = px;
  s[2] += py * rho * alpha;
  s[4] += L - (1.0 + beta0 * beta0 * ps) * rho * alpha;
}

/* Linear sector dipole from H_approx with curvature h = angle/L and the
 * bending field's h^2 x^2/2 term (Sec. III, Eq. H):
 *   H = (px^2+py^2)/2 + ps^2/(2 gamma0^2) - h x ps + h^2 x^2 / 2.
 * With C = cos(hL), S = sin(hL):
 *   x  = x0 C + px0 S/h + ps (1-C)/h
 *   px = -x0 h S + px0 C + ps S
 *   y  = y0 + py0 L,  py = py0
 *   sg = sg0 + ps L/gamma0^2 - (x0 S + px0 (1-C)/h + ps (L - S/h)). */
static void orc_bend(double *s, double L, double angle, double gamma0) {
  if (angle == 0.0) { orc_h0_drift(s, L, gamma0); return; }
  double h = angle / L, C = cos(angle), S = sin(angle);
  double x0 = s[0], px0 = s[1], ps = s[5];
  s[0] = x0 * C + px0 * S / h + ps * (1.0 - C) / h;
  s[1] = -x0 * h * S + px0 * C + ps * S;
  s[2] += s[3] * L;
  s[4] += ps * L / (gamma0 * gamma0) - (x0 * S + px0 * (1.0 - C) / h + ps * (L - S / h));
}

/* Thin RF cavity: energy gain e V sin(lag - 2 pi h sg / C) per passage,
 * ps += (V / (beta0^2 E0)) sin(lag - 2 pi h sg / C), E0 = gamma0 m c^2 [eV]. */
static void orc_rf(double *s, const orc_elem *e, const orc_beam *bm) {
  double e0 = bm->gamma0 * bm->mass_ev;
  double phase = e->lag - 2.0 * M_PI * e->harmonic * s[4] / bm->circumference;
  s[5] += e->volt / (bm->beta0 * bm->beta0 * e0) * sin(phase);
}

/* Push every particle through elements[0..n_elems) in order. */
void orc_push(int64_t n, double *x, double *px, double *y, double *py, double *sg, double *ps,
              const orc_elem *el, int n_elems, const orc_beam *bm) {
#pragma omp parallel for num_threads(orc_threads) schedule(static)
  for (int64_t p = 0; p < n; ++p) {
    double s[6] = {x[p], px[p], y[p], py[p], sg[p], ps[p]};
    for (int k = 0; k < n_elems; ++k) {
      const orc_elem *e = &el[k];
      switch (e->type) {
        case ORC_DRIFT: orc_drift(s, e->length, bm->beta0); break;
        case ORC_QUAD: orc_quad(s, e->length, e->k1, bm->gamma0); break;
        case ORC_SEXT:
          if (e->length > 0.0)
            orc_thick_sext(s, e->length, e->k2l, bm->gamma0);
          else
            orc_sext(s, e->k2l);
          break;
        case ORC_EXACT_BEND: orc_exact_bend(s, e->length, e->angle, bm->beta0); break;
        case ORC_BEND: orc_bend(s, e->length, e->angle, bm->gamma0); break;
        case ORC_RF: orc_rf(s, e, bm); break;
        default: break; /* markers: no-op */
      }
    }
    x[p] = s[0]; px[p] = s[1]; y[p] = s[2]; py[p] = s[3]; sg[p] = s[4]; ps[p] = s[5];
  }
}

/* Beam moments for Sec. V diagnostics: out[0..6) = means of
 * (x, px, y, py, sg, ps); out[6..) = central second moments
 * <xx>, <x px>, <px px>, <yy>, <y py>, <py py>, <sg sg>, <ps ps>. */
void orc_moments(int64_t n, const double *x, const double *px, const double *y, const double *py,
                 const double *sg, const double *ps, double *out) {
  const double *a[6] = {x, px, y, py, sg, ps};
  double m[6] = {0, 0, 0, 0, 0, 0};
  for (int c = 0; c < 6; ++c) {
    double t = 0.0;
    for (int64_t p = 0; p < n; ++p) t += a[c][p];
    m[c] = t / (double)n;
    out[c] = m[c];
  }
  double s[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int64_t p = 0; p < n; ++p) {
    double dx = x[p] - m[0], dpx = px[p] - m[1], dy = y[p] - m[2], dpy = py[p] - m[3];
    double ds = sg[p] - m[4], dps = ps[p] - m[5];
    s[0] += dx * dx; s[1] += dx * dpx; s[2] += dpx * dpx;
    s[3] += dy * dy; s[4] += dy * dpy; s[5] += dpy * dpy;
    s[6] += ds * ds; s[7] += dps * dps;
  }
  for (int c = 0; c < 8; ++c) out[6 + c] = s[c] / (double)n;
}
