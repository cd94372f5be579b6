/* The C-ABI from plain C99: a bunch in host memory tracked for three turns of
 * a FODO cell with two space-charge locations (sc_track_turns_host), the
 * moments read back, argument errors reported through sc_last_error.
 * Prints "ok" and exits 0 on success.  With a file name argument it also
 * writes the tracked state (x, px, y, py, sigma, psigma: n doubles each) and
 * the three turns' moments (3 x 14 doubles) there, for a comparison with the
 * oracle. */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include "sc.h"

static uint64_t lcg = 12345u;
static double uniform(void) { /* deterministic, (0, 1) */
  lcg = lcg * 6364136223846793005ull + 1442695040888963407ull;
  return ((double)(lcg >> 11) + 0.5) / 9007199254740992.0;
}

static int fail(const char *what) {
  char buf[512];
  sc_last_error(buf, sizeof buf);
  fprintf(stderr, "%s: %s\n", what, buf);
  return 1;
}

int main(int argc, char **argv) {
  const int64_t n = 20000;
  double *a = malloc((size_t)n * 6 * sizeof(double));
  if (!a) return 1;
  sc_particles p = {a, a + n, a + 2 * n, a + 3 * n, a + 4 * n, a + 5 * n, n};
  for (int64_t i = 0; i < n; ++i) {
    p.x[i] = 4e-3 * (uniform() - 0.5);
    p.px[i] = 4e-4 * (uniform() - 0.5);
    p.y[i] = 4e-3 * (uniform() - 0.5);
    p.py[i] = 4e-4 * (uniform() - 0.5);
    p.sigma[i] = 20.0 * (uniform() - 0.5);
    p.psigma[i] = 2e-3 * (uniform() - 0.5);
  }
  const double gamma0 = 1.0 + 3.0 / 0.93827208816, beta0 = sqrt(1.0 - 1.0 / (gamma0 * gamma0));
  sc_beam b = {gamma0, beta0, 5e9, 1.5347e-18, 22.0, 0.93827208816e9};
  sc_element lat[6] = {
      {SC_QUAD, 0, 0.5, 0.5, 0, 0, 0, 0, 0}, {SC_DRIFT, 0, 5.0, 0, 0, 0, 0, 0, 0}, {SC_MARK, 0, 0, 0, 0, 0, 0, 0, 0},
      {SC_QUAD, 0, 0.5, -0.5, 0, 0, 0, 0, 0}, {SC_DRIFT, 0, 5.0, 0, 0, 0, 0, 0, 0}, {SC_MARK, 0, 0, 0, 0, 0, 0, 0, 0}};

  sc_grid *bad = NULL;
  if (sc_create_grid(&bad, 1, 64, -0.01, 0.01, -0.01, 0.01, SC_SOLVE_FP64, NULL) != SC_ERR_ARG || bad) {
    fprintf(stderr, "a 1-node grid was accepted\n");
    return 1;
  }
  char msg[256];
  if (sc_last_error(msg, sizeof msg) != SC_OK || msg[0] == 0) return 1;

  sc_grid *g = NULL;
  if (sc_create_grid(&g, 64, 64, -0.01, 0.01, -0.01, 0.01, SC_SOLVE_FP64, NULL) != SC_OK) return fail("create");
  double diag[3 * 14];
  if (sc_track_turns_host(g, &p, &b, lat, 6, 3, diag) != SC_OK) return fail("track");
  for (int t = 0; t < 3; ++t) {
    const double *d = diag + 14 * t;
    for (int k = 0; k < 14; ++k)
      if (!isfinite(d[k])) return fail("moments not finite");
    /* rms size of order the 1.15 mm of the uniform +-2 mm start, in every turn */
    if (!(d[6] > 1e-7 && d[6] < 1e-4 && d[9] > 1e-7 && d[9] < 1e-4)) {
      fprintf(stderr, "turn %d: <xx> = %g, <yy> = %g\n", t, d[6], d[9]);
      return 1;
    }
  }
  for (int64_t i = 0; i < n; ++i)
    if (!isfinite(p.x[i]) || !isfinite(p.px[i]) || !isfinite(p.y[i]) || !isfinite(p.psigma[i]))
      return fail("state not finite");
  if (sc_destroy_grid(g) != SC_OK) return fail("destroy");
  if (argc > 1) {
    FILE *fp = fopen(argv[1], "wb");
    if (!fp || fwrite(a, sizeof(double), (size_t)n * 6, fp) != (size_t)n * 6 ||
        fwrite(diag, sizeof(double), 3 * 14, fp) != 3 * 14 || fclose(fp) != 0)
      return fail("writing the state");
  }
  free(a);
  printf("ok\n");
  return 0;
}
