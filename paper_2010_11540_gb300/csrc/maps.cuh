// Single-particle transfer maps of Sec. III in float64, one particle per
// thread.  State: (x, px, y, py, sg, ps) with px = Px/p0, sg = s - c beta0 t.
#pragma once

#include "sc_internal.cuh"

namespace sc {

struct State {
  double x, px, y, py, sg, ps;
};

struct BeamK {
  double beta0_sq, inv_gamma0_sq, rf_scale, two_pi_over_c;
};

// Exact field-free drift (Sec. III-A, uniform field solved without the
// approximate Hamiltonian).  (1+delta)^2 = 1 + 2 ps + beta0^2 ps^2 (Eq. BEND2),
// 1/pz = ((1+delta)^2 - px^2 - py^2)^(-1/2):
//   x += L px/pz, y += L py/pz, sg += L (1 - (1 + beta0^2 ps)/pz).
__device__ __forceinline__ void map_drift(State& s, double L, const BeamK& b) {
  const double opd2 = fma(b.beta0_sq * s.ps, s.ps, fma(2.0, s.ps, 1.0));
  const double rpz = rsqrt(opd2 - s.px * s.px - s.py * s.py);
  const double Lr = L * rpz;
  s.x = fma(Lr, s.px, s.x);
  s.y = fma(Lr, s.py, s.y);
  s.sg += L - Lr * fma(b.beta0_sq, s.ps, 1.0);
}

// Flow of H0 (k1 -> 0 limit of the quadrupole): straight line with the
// chromatic factor (1 - ps).
__device__ __forceinline__ void map_h0(State& s, double L, const BeamK& b) {
  const double f = (1.0 - s.ps) * L;
  s.x = fma(f, s.px, s.x);
  s.y = fma(f, s.py, s.y);
  s.sg += s.ps * L * b.inv_gamma0_sq - 0.5 * L * (s.px * s.px + s.py * s.py);
}

// One plane of the thick quadrupole (Sec. III-B), w = sqrt(|k1|(1-ps)),
// a = sqrt((1-ps)/|k1|) = (1-ps)/w, bq = sqrt(|k1|/(1-ps)) = w/(1-ps).
// Focusing: u' = u c + a pu s, pu' = pu c - bq u s (c, s = cos, sin wL);
// defocusing: cosh/sinh and + sign.  Returns int_0^L pu(s)^2 ds.
template <bool FOC>
__device__ __forceinline__ double quad_plane(double& u, double& pu, double w, double a, double bq, double L) {
  double c, s;
  if (FOC) {
    sincos(w * L, &s, &c);
  } else {
    s = sinh(w * L);
    c = cosh(w * L);
  }
  const double u0 = u, p0 = pu;
  const double sc2w = s * c / (2.0 * w);
  const double s2w = s * s / (2.0 * w);
  if (FOC) {
    u = fma(u0, c, a * p0 * s);
    pu = fma(p0, c, -bq * u0 * s);
    const double icc = 0.5 * L + sc2w, iss = 0.5 * L - sc2w;
    return p0 * p0 * icc - 2.0 * p0 * bq * u0 * s2w + bq * bq * u0 * u0 * iss;
  } else {
    u = fma(u0, c, a * p0 * s);
    pu = fma(p0, c, bq * u0 * s);
    const double icc = 0.5 * L + sc2w, iss = -0.5 * L + sc2w;
    return p0 * p0 * icc + 2.0 * p0 * bq * u0 * s2w + bq * bq * u0 * u0 * iss;
  }
}

// Thick quadrupole: planes as above (k1 > 0 focuses x), and
// sg += ps L / gamma0^2 - 1/2 (int px^2 + int py^2).
__device__ __forceinline__ void map_quad(State& s, double L, double k1, const BeamK& b) {
  if (k1 == 0.0) {
    map_h0(s, L, b);
    return;
  }
  const double ak = fabs(k1);
  const double opm = 1.0 - s.ps;
  const double w = sqrt(ak * opm);
  const double a = opm / w;
  const double bq = w / opm;
  double Ix, Iy;
  if (k1 > 0.0) {
    Ix = quad_plane<true>(s.x, s.px, w, a, bq, L);
    Iy = quad_plane<false>(s.y, s.py, w, a, bq, L);
  } else {
    Ix = quad_plane<false>(s.x, s.px, w, a, bq, L);
    Iy = quad_plane<true>(s.y, s.py, w, a, bq, L);
  }
  s.sg += s.ps * L * b.inv_gamma0_sq - 0.5 * (Ix + Iy);
}

// Thin sextupole (V-step of Eq. Sym2): px -= k2l/2 (x^2 - y^2), py += k2l x y.
__device__ __forceinline__ void map_sext(State& s, double k2l) {
  s.px -= 0.5 * k2l * (s.x - s.y) * (s.x + s.y);
  s.py = fma(k2l * s.x, s.y, s.py);
}

// Linear sector dipole from H_approx with curvature h = angle/L (Sec. III,
// Eq. H including the bending field's h^2 x^2/2).
__device__ __forceinline__ void map_bend(State& s, double L, double angle, const BeamK& b) {
  if (angle == 0.0) {
    map_h0(s, L, b);
    return;
  }
  const double h = angle / L;
  double S, C;
  sincos(angle, &S, &C);
  const double x0 = s.x, px0 = s.px, ps = s.ps;
  s.x = x0 * C + px0 * S / h + ps * (1.0 - C) / h;
  s.px = -x0 * h * S + px0 * C + ps * S;
  s.y = fma(s.py, L, s.y);
  s.sg += ps * L * b.inv_gamma0_sq - (x0 * S + px0 * (1.0 - C) / h + ps * (L - S / h));
}

// Thin RF cavity: ps += volt / (beta0^2 E0) sin(lag - 2 pi h sg / C).
__device__ __forceinline__ void map_rf(State& s, double volt, double harmonic, double lag, const BeamK& b) {
  s.ps += volt * b.rf_scale * sin(lag - b.two_pi_over_c * harmonic * s.sg);
}

__device__ __forceinline__ void push_elements(State& s, const sc_element* __restrict__ el, int n_elem,
                                              const BeamK& b) {
#pragma unroll 1
  for (int k = 0; k < n_elem; ++k) {
    const int type = __ldg(&el[k].type);
    const double L = __ldg(&el[k].length);
    switch (type) {
      case SC_DRIFT: map_drift(s, L, b); break;
      case SC_QUAD: map_quad(s, L, __ldg(&el[k].k1), b); break;
      case SC_SEXT: map_sext(s, __ldg(&el[k].k2l)); break;
      case SC_BEND: map_bend(s, L, __ldg(&el[k].angle), b); break;
      case SC_RF: map_rf(s, __ldg(&el[k].volt), __ldg(&el[k].harmonic), __ldg(&el[k].lag), b); break;
      default: break;
    }
  }
}

}  // namespace sc
