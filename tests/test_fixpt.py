"""The deposit's integer-domain split of a grid coordinate (csrc/fixpt.h):
cell index, fixed-point CIC weight and fraction decoded from the IEEE-754
bits must equal the float64 formulas floor(xi), rint((xi - floor xi) 2^20)
(ties to even) and xi - floor(xi), bit for bit, for every input -- random
coordinates, random bit patterns, exact ties of the weight rounding, integer
boundaries, signed zeros, subnormals, infinities and NaNs.  Host compile of the
header with the system C++ compiler; no GPU."""
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2010_11540_gb300", "csrc")

HARNESS = r"""
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <vector>
#include "fixpt.h"
int main(int argc, char** argv) {
  const int limit = atoi(argv[2]);
  FILE* fp = fopen(argv[1], "rb");
  std::vector<double> v;
  double d;
  while (fread(&d, 8, 1, fp) == 1) v.push_back(d);
  fclose(fp);
  long bad = 0, inside = 0;
  for (double xi : v) {
    int i = -1, a = -1, k = -1;
    double f = -1.0;
    const bool got = sc::cic_split(xi, limit, i, a, &f);
    const bool gotk = sc::floor_index(xi, limit, k);
    const bool ref = std::isfinite(xi) && xi >= 0.0 && xi < (double)limit;
    if (got != ref || gotk != ref) { ++bad; if (bad < 5) printf("valid %.17g\n", xi); continue; }
    if (!ref) continue;
    ++inside;
    const double fl = std::floor(xi);
    const double fx = xi - fl;
    const long long ra = std::llrint(fx * 1048576.0);
    if (i != (int)fl || k != (int)fl || a != ra || f != fx) {
      ++bad;
      if (bad < 5) printf("mismatch %.17g: i %d/%d k %d a %d/%lld f %.17g/%.17g\n", xi, i, (int)fl, k, a, ra, f, fx);
    }
  }
  printf("%ld %ld\n", bad, inside);
  return 0;
}
"""


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    d = tmp_path_factory.mktemp("fixpt")
    src = d / "h.cpp"
    src.write_text(HARNESS)
    exe = d / "h"
    subprocess.run([cxx, "-std=c++17", "-O2", "-ffp-contract=off", "-I", CSRC, str(src), "-o", str(exe)],
                   check=True)
    return exe, d


def run(harness, values, limit):
    exe, d = harness
    f = d / "in.bin"
    np.ascontiguousarray(values, dtype=np.float64).tofile(f)
    out = subprocess.run([str(exe), str(f), str(limit)], check=True, capture_output=True, text=True).stdout
    bad, inside = map(int, out.split()[-2:])
    return bad, inside, out


@pytest.mark.parametrize("limit", [127, 255, 4095, 1])
def test_random_coordinates(harness, limit):
    rng = np.random.default_rng(limit)
    v = np.concatenate([rng.uniform(-2.0, limit + 2.0, 400000),
                        rng.uniform(0, 1, 100000) * 2.0 ** rng.integers(-70, 3, 100000)])
    bad, inside, out = run(harness, v, limit)
    assert bad == 0, out
    assert inside > 100000


def test_random_bit_patterns(harness):
    rng = np.random.default_rng(7)
    bits = rng.integers(0, 2 ** 63, 500000, dtype=np.int64).astype(np.uint64)
    bits[::2] |= np.uint64(1) << np.uint64(63)
    # bias the exponents towards the interesting range
    e = rng.integers(1023 - 70, 1023 + 14, 250000).astype(np.uint64)
    bits[1::2] = (bits[1::2] & np.uint64((1 << 52) - 1)) | (e << np.uint64(52))
    bad, inside, out = run(harness, bits.view(np.float64), 127)
    assert bad == 0, out
    assert inside > 100000


def test_exact_ties_and_boundaries(harness):
    """xi = i + (k + 1/2) 2^-20 (exact ties: even k stays, odd k rounds up), the
    neighbours of integers and of the limit, signed zeros, subnormals, specials."""
    i = np.arange(0, 127, dtype=np.float64)
    k = np.array([0, 1, 2, 3, 524287, 524288, 1048574, 1048575], dtype=np.float64)
    ties = (i[:, None] + (k[None, :] + 0.5) / 2.0 ** 20).ravel()
    near = np.concatenate([np.nextafter(i, -np.inf), i, np.nextafter(i, np.inf), np.nextafter(ties, np.inf),
                           np.nextafter(ties, -np.inf)])
    special = np.array([0.0, -0.0, 5e-324, -5e-324, 2.2250738585072014e-308, 1e-300, -1e-300, 127.0,
                        np.nextafter(127.0, 0.0), np.inf, -np.inf, np.nan, 2.0 ** 30, 2.0 ** 29 + 0.5,
                        0.5 / 2 ** 20, 1.5 / 2 ** 20, 2.0 ** -21, 2.0 ** -61, 2.0 ** -59])
    bad, inside, out = run(harness, np.concatenate([ties, near, special]), 127)
    assert bad == 0, out


WIDEN = r"""
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include "fixpt.h"
int main() {
  unsigned long long bad = 0, checked = 0;
  uint32_t u = 0;
  do {
    float f;
    memcpy(&f, &u, 4);
    const double w = sc::f32_widen(f);
    uint64_t wb, rb;
    memcpy(&wb, &w, 8);
    const double r = (double)f;
    memcpy(&rb, &r, 8);
    const uint32_t mag = u & 0x7fffffffu;
    bool ok;
    if (mag > 0x7f800000u)            // NaN: a NaN of the same sign (quieting may differ)
      ok = std::isnan(w) && ((wb >> 63) == (u >> 31));
    else if (mag != 0 && mag < 0x00800000u)  // subnormal: zero of the same sign
      ok = wb == ((uint64_t)(u >> 31) << 63);
    else                              // zero, normal, infinity: the conversion's bits
      ok = wb == rb;
    if (!ok && ++bad < 5) printf("mismatch %08x\n", (unsigned)u);
    ++checked;
  } while (++u != 0);
  printf("%llu %llu\n", bad, checked);
  return 0;
}
"""


def test_f32_widen_every_float(tmp_path):
    """f32_widen (the split form's float32 field values widened to float64 on
    the integer pipe) against the compiler's float -> double conversion for
    all 2^32 bit patterns: the same bits for zero, normal and infinite values,
    a NaN for a NaN, signed zero for the (never used) subnormals."""
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    src = tmp_path / "w.cpp"
    src.write_text(WIDEN)
    exe = tmp_path / "w"
    subprocess.run([cxx, "-std=c++17", "-O2", "-I", CSRC, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    bad, checked = map(int, out.split()[-2:])
    assert bad == 0 and checked == 2 ** 32, out
