"""The oracle's C code under AddressSanitizer, UndefinedBehaviorSanitizer
(with float-to-int overflow checks) and LeakSanitizer: every exported
function on a small grid, with particles on and off the grid, at its last
node, NaN, infinite, huge and signed-zero coordinates, large momentum
offsets and every element type -- no out-of-bounds access, no undefined
behaviour, no leak.  Host only; skipped where the sanitizer runtimes are
missing."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

HARNESS = r"""
#include "sc_oracle.c"
#include <stdio.h>
static unsigned long long lcg = 1;
static double u01(void) { lcg = lcg * 6364136223846793005ull + 1442695040888963407ull; return ((lcg >> 11) + 0.5) / 9007199254740992.0; }
int main(void) {
  const int nx = 16, ny = 12, nz = 4; const int64_t n = 3000;
  const double xmin = -0.01, xmax = 0.01, ymin = -0.008, ymax = 0.008, zmin = -5, zmax = 5;
  const double hx = (xmax - xmin) / (nx - 1), hy = (ymax - ymin) / (ny - 1), dz = (zmax - zmin) / nz;
  double *x = malloc(n * 8), *px = malloc(n * 8), *y = malloc(n * 8), *py = malloc(n * 8), *sg = malloc(n * 8), *ps = malloc(n * 8);
  for (int64_t p = 0; p < n; ++p) {
    x[p] = 0.024 * (u01() - 0.5); y[p] = 0.02 * (u01() - 0.5); sg[p] = 12 * (u01() - 0.5);
    px[p] = 4e-4 * (u01() - 0.5); py[p] = 4e-4 * (u01() - 0.5); ps[p] = 2e-3 * (u01() - 0.5);
  }
  double sp[] = {NAN, INFINITY, -INFINITY, -0.0, 0.0, 1e300, -1e300, xmax, xmin, 5e-324};
  for (int k = 0; k < 10; ++k) { x[k] = sp[k]; y[20 + k] = sp[k]; sg[40 + k] = sp[k]; }
  x[60] = xmax; y[60] = ymax; x[61] = xmin; y[61] = ymin; ps[70] = 0.3; ps[71] = -0.3;
  uint64_t *Q = calloc((size_t)nx * ny * nz, 8);
  uint64_t out = orc_deposit_sliced(n, x, y, sg, nx, ny, xmin, ymin, 1 / hx, 1 / hy, nz, zmin, 1 / dz, Q);
  out += orc_deposit(n, x, y, nx, ny, xmin, ymin, 1 / hx, 1 / hy, Q);
  double *Gc = malloc((size_t)4 * nx * ny * 8); orc_green_cyclic(nx, ny, hx, hy, Gc);
  double *q = calloc((size_t)nx * ny, 8); for (int c = 0; c < nx * ny; ++c) q[c] = (double)Q[c] * 1e-12;
  double *phe = malloc((size_t)(nx + 2) * (ny + 2) * 8); orc_potential_direct(nx, ny, hx, hy, q, phe);
  double *Ex = malloc((size_t)nx * ny * nz * 8), *Ey = malloc((size_t)nx * ny * nz * 8), *phi = malloc((size_t)nx * ny * nz * 8);
  for (int k = 0; k < nz; ++k) orc_fields(nx, ny, hx, hy, phe, Ex + k * nx * ny, Ey + k * nx * ny);
  for (int c = 0; c < nx * ny * nz; ++c) phi[c] = u01();
  orc_kick_sliced(n, x, y, sg, px, py, nx, ny, xmin, ymin, 1 / hx, 1 / hy, nz, zmin, 1 / dz, Ex, Ey, 1e-3);
  orc_kick(n, x, y, px, py, nx, ny, xmin, ymin, 1 / hx, 1 / hy, Ex, Ey, 1e-3);
  orc_kick_long(n, x, y, sg, ps, nx, ny, xmin, ymin, 1 / hx, 1 / hy, nz, zmin, 1 / dz, phi, 1e-6);
  orc_kick_bezier(n, x, y, sg, px, py, ps, nx, ny, xmin, ymin, 1 / hx, 1 / hy, hx, hy, nz, zmin, 1 / dz, phi, 1e-3, 1e-6);
  double o3[3];
  for (int i = 0; i < nx - 1; ++i) for (int j = 0; j < ny - 1; ++j) orc_bezier_point(phi, nx, ny, hx, hy, i, j, 0.5, 0.25, o3);
  orc_elem el[] = {{ORC_DRIFT, 0, 2.0, 0, 0, 0, 0, 0, 0}, {ORC_QUAD, 0, 0.5, 0.8, 0, 0, 0, 0, 0},
                   {ORC_QUAD, 0, 0.5, -0.7, 0, 0, 0, 0, 0}, {ORC_QUAD, 0, 0.5, 0.0, 0, 0, 0, 0, 0},
                   {ORC_SEXT, 0, 0, 0, 1.0, 0, 0, 0, 0}, {ORC_SEXT, 0, 0.3, 0, 1.0, 0, 0, 0, 0},
                   {ORC_BEND, 0, 2.0, 0, 0, 0.1, 0, 0, 0}, {ORC_BEND, 0, 0, 0, 0, 0, 0, 0, 0},
                   {ORC_EXACT_BEND, 0, 2.0, 0, 0, 0.1, 0, 0, 0}, {ORC_EXACT_BEND, 0, 1.0, 0, 0, 0, 0, 0, 0},
                   {ORC_RF, 0, 0, 0, 0, 0, 2e5, 9, 0.3}, {ORC_MARK, 0, 0, 0, 0, 0, 0, 0, 0}};
  orc_beam bm = {4.197, 0.9712, 5e9, 1.5347e-18, 100.0, 0.938e9};
  orc_push(n, x, px, y, py, sg, ps, el, 12, &bm);
  double m[14]; orc_moments(n, x, px, y, py, sg, ps, m);
  printf("ok %llu\n", (unsigned long long)out);
  free(x); free(px); free(y); free(py); free(sg); free(ps); free(Q); free(Gc); free(q); free(phe); free(Ex); free(Ey); free(phi);
  return 0;
}
"""


def test_oracle_c_under_sanitizers(tmp_path):
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no gcc")
    src = tmp_path / "h.c"
    src.write_text(HARNESS)
    exe = tmp_path / "h"
    flags = ["-std=gnu99", "-O1", "-g", "-fsanitize=address,undefined,float-cast-overflow",
             "-fno-sanitize-recover=all", "-fno-omit-frame-pointer", "-ffp-contract=off"]
    r = subprocess.run([gcc, *flags, "-I", os.path.join(ROOT, "oracle"), str(src), "-o", str(exe), "-lm"],
                       capture_output=True, text=True)
    if r.returncode != 0:
        pytest.skip("sanitizer runtimes not available: " + r.stderr[-200:])
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=1:abort_on_error=0", UBSAN_OPTIONS="print_stacktrace=1")
    r = subprocess.run([str(exe)], capture_output=True, text=True, env=env, timeout=300)
    assert r.returncode == 0 and r.stdout.startswith("ok"), r.stderr[-3000:]
