// Single-particle transfer maps of Sec. III in float64, one particle per
// thread, arranged to spend few instructions on the FP64 pipe (the GB300's
// scarcest unit: every FP64 add, multiply, fma, compare, floor and
// conversion takes one of its two issue slots per SM clock).
//
// State: (x, px, y, py, sg, ps) with px = Px/p0, sg = s - c beta0 t.
// Per-particle quantities that depend on ps alone (the chromatic factors of
// PsConst, the thick quadrupoles' matrix entries QuadCoef) are computed once
// per call of a tracked turn and kept per particle (ps changes only in RF
// cavities, after which they are refreshed).
#pragma once

#include "sc_internal.cuh"

namespace sc {

// Quadrupole flags: the kind (QF_KIND bits) and, from bit QF_FAM_SHIFT, 1 +
// the index of the quadrupole's family in the per-particle coefficient cache
// (0: the map computes its own coefficients).
enum : int { QF_ZERO = 0, QF_FOCUS_X = 1, QF_FOCUS_Y = 2, QF_KIND = 3, QF_FAM_SHIFT = 4 };

// Largest chromatic phase shift |Delta| = |theta0 (sqrt(1-ps) - 1)| handled by
// the angle-addition series: with terms up to Delta^5 (sin) and Delta^4 (cos),
// the truncation is below 2e-18 for |Delta| <= 2^-8; beyond it the library
// sin/cos/sinh/cosh are used.
constexpr double kMaxDelta = 0.00390625;

struct State {
  double x, px, y, py, sg, ps;
};

// (The quadrupole's chromatic factor 1 - ps is formed where a map needs it:
// the cached quadrupole map does not.)
struct PsConst {
  double opd2;  // (1+delta)^2 = 1 + 2 ps + beta0^2 ps^2        (Eq. BEND2)
  double opb;   // 1 + beta0^2 ps = (1+delta) d(delta)/d(ps)
  double s1;    // sqrt(1 - ps)
  double r;     // 1/sqrt(1 - ps)
  double qi;    // 1/(4 (1 - ps))
};

__device__ __forceinline__ void ps_const(PsConst& k, double ps, double beta0_sq, bool quads) {
  k.opd2 = fma(beta0_sq * ps, ps, fma(2.0, ps, 1.0));
  k.opb = fma(beta0_sq, ps, 1.0);
  if (quads) {
    const double opm = 1.0 - ps;
    k.r = rsqrt(opm);
    k.s1 = opm * k.r;
    k.qi = 0.25 * k.r * k.r;
  } else {
    k.r = k.s1 = k.qi = 0.0;
  }
}

// Exact drift (Sec. III-A): with pz = sqrt((1+delta)^2 - px^2 - py^2),
// x += L px/pz, y += L py/pz, sg += L (1 - (1 + beta0^2 ps)/pz).
// e.p[0] = L.
__device__ __forceinline__ void map_drift(State& s, const DevElem& e, const PsConst& k) {
  const double L = e.p[0];
  const double rpz = rsqrt(fma(-s.py, s.py, fma(-s.px, s.px, k.opd2)));
  const double Lr = L * rpz;
  s.x = fma(Lr, s.px, s.x);
  s.y = fma(Lr, s.py, s.y);
  s.sg += fma(-Lr, k.opb, L);
}

// Thick quadrupole (Sec. III-B) for H_approx with K1 = k1:
//   w = sqrt(|k1| (1-ps)), a = sqrt((1-ps)/|k1|) = s1/sqk, bq = sqrt(|k1|/(1-ps)) = sqk r
//   focusing plane:   u = u0 cos wL + a pu0 sin wL,  pu = pu0 cos wL - bq u0 sin wL
//   defocusing plane: u = u0 cosh wL + a pu0 sinh wL, pu = pu0 cosh wL + bq u0 sinh wL
// wL = theta0 s1 = theta0 + Delta, theta0 = sqk L; cos/sin/cosh/sinh of
// theta0 come from the host, those of the small Delta from their Taylor
// series, combined by the addition theorems.
// sg: d sg/ds = ps/gamma0^2 - (px^2+py^2)/2.  Each plane conserves
// h_u = ((1-ps) pu^2 + k_u u^2)/2 (k_x = k1, k_y = -k1) and
// d(u pu)/ds = (1-ps) pu^2 - k_u u^2, so
//   int_0^L pu^2 ds = (h_u L + [u pu]_0^L / 2) / (1-ps),
// which gives sg += ps L/gamma0^2 - (L S2 + D) / (4 (1-ps)) with
// S2 = (1-ps)(px0^2+py0^2) + k1 (x0^2 - y0^2), D = [x px + y py]_0^L, i.e.
//   sg += ps L/gamma0^2 - (L/4)(px0^2+py0^2) - (L k1 (x0^2-y0^2) + D) / (4 (1-ps)).
// e.p = {L/4, L/gamma0^2, cos theta0, sin theta0, cosh theta0, sinh theta0, sqk, 1/sqk, L k1}
// (theta0 = sqk L = sqk (4 e.p[0]), the host's product bit for bit: the
// record keeps nine words, the size the kernels copy per element), e.flags =
// QF_* (plus the family bits); a zero-gradient quadrupole (QF_ZERO) has e.p[0] = L.
//
// The entries of the two planes' 2x2 matrices depend on ps alone (QuadCoef:
// u = cu u0 + sua pu0, pu = cu pu0 + sub u0), so a turn's tracking keeps them
// per particle and quadrupole family (computed where psc is, read by the map).
struct QuadCoef {
  double cx, sxa, sxb, cy, sya, syb;
};

__device__ __forceinline__ QuadCoef quad_coef(const DevElem& e, const PsConst& k) {
  const double th0 = e.p[6] * (4.0 * e.p[0]);
  const double delta = fma(th0, k.s1, -th0);
  double c, sn, ch, sh;
  if (fabs(delta) <= kMaxDelta) {
    const double d2 = delta * delta;
    const double sd = fma(delta, fma(d2, 1.0 / 120.0, -1.0 / 6.0) * d2, delta);   // sin(delta)
    const double cm = fma(d2, 1.0 / 24.0, -0.5) * d2;                             // cos(delta) - 1
    const double shd = fma(delta, fma(d2, 1.0 / 120.0, 1.0 / 6.0) * d2, delta);   // sinh(delta)
    const double chm = fma(d2, 1.0 / 24.0, 0.5) * d2;                             // cosh(delta) - 1
    const double c0 = e.p[2], s0 = e.p[3], ch0 = e.p[4], sh0 = e.p[5];
    c = fma(-s0, sd, fma(c0, cm, c0));
    sn = fma(c0, sd, fma(s0, cm, s0));
    ch = fma(sh0, shd, fma(ch0, chm, ch0));
    sh = fma(ch0, shd, fma(sh0, chm, sh0));
  } else {
    const double th = th0 * k.s1;
    sincos(th, &sn, &c);
    ch = cosh(th);
    sh = sinh(th);
  }
  const double a = k.s1 * e.p[7];
  const double bq = e.p[6] * k.r;
  // focusing plane on trig (c, sn), defocusing on hyperbolic (ch, sh)
  if ((e.flags & QF_KIND) == QF_FOCUS_X) return QuadCoef{c, a * sn, -bq * sn, ch, a * sh, bq * sh};
  return QuadCoef{ch, a * sh, bq * sh, c, a * sn, -bq * sn};
}

__device__ __forceinline__ void quad_apply(State& s, const DevElem& e, const QuadCoef& q, const PsConst& k) {
  const double x0 = s.x, px0 = s.px, y0 = s.y, py0 = s.py;
  const double xy = fma(x0, x0, -y0 * y0);
  const double pp = fma(px0, px0, py0 * py0);
  s.x = fma(q.cx, x0, q.sxa * px0);
  s.px = fma(q.cx, px0, q.sxb * x0);
  s.y = fma(q.cy, y0, q.sya * py0);
  s.py = fma(q.cy, py0, q.syb * y0);
  // L k1 (x0^2 - y0^2) + D, D = x px + y py - x0 px0 - y0 py0
  const double u = fma(e.p[8], xy, fma(-y0, py0, fma(-x0, px0, fma(s.x, s.px, s.y * s.py))));
  s.sg = fma(-u, k.qi, fma(-e.p[0], pp, fma(s.ps, e.p[1], s.sg)));
}

__device__ __forceinline__ void map_quad(State& s, const DevElem& e, const PsConst& k, double inv_gamma0_sq) {
  if ((e.flags & QF_KIND) == QF_ZERO) {  // flow of H0: straight line with the chromatic factor
    const double L = e.p[0];
    const double f = (1.0 - s.ps) * L;
    const double pp = fma(s.px, s.px, s.py * s.py);
    s.x = fma(f, s.px, s.x);
    s.y = fma(f, s.py, s.y);
    s.sg = fma(-0.5 * L, pp, fma(s.ps, L * inv_gamma0_sq, s.sg));
    return;
  }
  quad_apply(s, e, quad_coef(e, k), k);
}

// The map with the particle's cached coefficients: qc points at its entry of
// the family's six arrays of n (cx, sxa, sxb, cy, sya, syb).
__device__ __forceinline__ void map_quad_cached(State& s, const DevElem& e, const double* __restrict__ qc, size_t n,
                                                const PsConst& k) {
  const QuadCoef q{qc[0], qc[n], qc[2 * n], qc[3 * n], qc[4 * n], qc[5 * n]};
  quad_apply(s, e, q, k);
}

// Flow of H0 = (px^2+py^2)/2 (1-ps) + ps^2/(2 gamma0^2) over l.
__device__ __forceinline__ void h0_flow(State& s, const PsConst& k, double l, double inv_gamma0_sq) {
  const double f = (1.0 - s.ps) * l;
  const double pp = fma(s.px, s.px, s.py * s.py);
  s.x = fma(f, s.px, s.x);
  s.y = fma(f, s.py, s.y);
  s.sg = fma(-0.5 * l, pp, fma(s.ps, l * inv_gamma0_sq, s.sg));
}

// Sextupole (Sec. III-C).  Thin: the V step of Eq. Sym2 as one kick,
// px -= k2l/2 (x^2 - y^2), py += k2l x y; e.p = {k2l/2, k2l}.  Thick
// (e.flags = 1): Eq. Sym2, H0 flows of a L, c L, a L around two kicks of
// integrated strength k2l/2; e.p = {k2l/4, k2l/2, a L, c L}.
__device__ __forceinline__ void sext_kick(State& s, double half, double full) {
  s.px = fma(-half, (s.x - s.y) * (s.x + s.y), s.px);
  s.py = fma(full * s.x, s.y, s.py);
}

// (Thick elements and the exact dipole are not inlined: their registers stay
// out of the hot kernels' allocation.)
__device__ __noinline__ void map_sext_thick(State& s, const DevElem& e, const PsConst& k, double inv_gamma0_sq) {
  h0_flow(s, k, e.p[2], inv_gamma0_sq);
  sext_kick(s, e.p[0], e.p[1]);
  h0_flow(s, k, e.p[3], inv_gamma0_sq);
  sext_kick(s, e.p[0], e.p[1]);
  h0_flow(s, k, e.p[2], inv_gamma0_sq);
}

__device__ __forceinline__ void map_sext(State& s, const DevElem& e, const PsConst& k, double inv_gamma0_sq) {
  if (e.flags != 1)
    sext_kick(s, e.p[0], e.p[1]);
  else
    map_sext_thick(s, e, k, inv_gamma0_sq);
}

// Exact sector dipole (Sec. III-A, uniform field without H_approx): the
// particle's circle in the bending plane carried to the exit face.  With
// P^2 = (1+delta)^2 - py^2, pz0 = sqrt(P^2 - px0^2), C = cos(angle), S = sin(angle):
//   px = px0 C + (pz0 - 1 - x0/rho) S,  pz = sqrt(P^2 - px^2),
//   x = (x0 + rho (1 - pz0)) C + rho px0 S + rho (pz - 1),
//   alpha = angle + asin(px0/P) - asin(px/P),
//   y += py rho alpha,  sg += L - (1 + beta0^2 ps) rho alpha.
// e.p = {L, angle, C, S, rho, 1/rho}; zero angle (e.flags = 1): the exact drift.
__device__ __noinline__ void map_exact_bend(State& s, const DevElem& e, const PsConst& k) {
  if (e.flags == 1) {
    map_drift(s, e, k);
    return;
  }
  const double L = e.p[0], angle = e.p[1], C = e.p[2], S = e.p[3], rho = e.p[4], h = e.p[5];
  const double x0 = s.x, px0 = s.px;
  const double P2 = fma(-s.py, s.py, k.opd2);
  const double pz0 = sqrt(fma(-px0, px0, P2));
  const double px = fma(px0, C, (pz0 - 1.0 - x0 * h) * S);
  const double pz = sqrt(fma(-px, px, P2));
  const double rP = rsqrt(P2);
  const double alpha = angle + (asin(px0 * rP) - asin(px * rP));
  s.x = fma(x0 + rho * (1.0 - pz0), C, fma(rho * px0, S, rho * (pz - 1.0)));
  s.px = px;
  s.y = fma(s.py * rho, alpha, s.y);
  s.sg += fma(-k.opb * rho, alpha, L);
}

// Linear sector dipole from H_approx with curvature h (Sec. III, Eq. H plus
// the bending field's h^2 x^2 / 2):
//   x = C x0 + (S/h) px0 + ((1-C)/h) ps,  px = -hS x0 + C px0 + S ps,
//   y += L py, sg += ps L/gamma0^2 - (S x0 + ((1-C)/h) px0 + (L - S/h) ps).
// e.p = {L, C, S, S/h, (1-C)/h, h S, L - S/h}; angle 0: e.flags = 1 (H0 flow).
__device__ __forceinline__ void map_bend(State& s, const DevElem& e, const PsConst& k, double inv_gamma0_sq) {
  const double L = e.p[0];
  if (e.flags == 1) {
    const double f = (1.0 - s.ps) * L;
    const double pp = fma(s.px, s.px, s.py * s.py);
    s.x = fma(f, s.px, s.x);
    s.y = fma(f, s.py, s.y);
    s.sg = fma(-0.5 * L, pp, fma(s.ps, L * inv_gamma0_sq, s.sg));
    return;
  }
  const double C = e.p[1], S = e.p[2], Soh = e.p[3], Cm = e.p[4], hS = e.p[5], LS = e.p[6];
  const double x0 = s.x, px0 = s.px, ps = s.ps;
  s.x = fma(C, x0, fma(Soh, px0, Cm * ps));
  s.px = fma(-hS, x0, fma(C, px0, S * ps));
  s.y = fma(L, s.py, s.y);
  s.sg = fma(ps, L * inv_gamma0_sq, s.sg) - fma(S, x0, fma(Cm, px0, LS * ps));
}

// Thin RF cavity: ps += V/(beta0^2 E0) sin(lag - 2 pi h sg / C).
// e.p = {V/(beta0^2 E0), 2 pi h / C, lag}.
__device__ __forceinline__ void map_rf(State& s, const DevElem& e) {
  s.ps = fma(e.p[0], sin(fma(-e.p[1], s.sg, e.p[2])), s.ps);
}

// Push through n_elem elements with the ps-dependent quantities k (valid on
// entry).  quads: refresh k's square roots after an RF cavity.  Returns true
// when an RF cavity changed ps (k then holds the new values).  qc: the
// particle's entry in the quadrupole coefficient cache (arrays of n), valid
// until an RF cavity; NULL: none.  XE: the segment may hold thick sextupoles
// or exact dipoles (their code is compiled only into the kernels that need
// it, keeping the common kernels' registers).
template <bool XE>
__device__ __forceinline__ bool push_elements(State& s, PsConst& k, const DevElem* __restrict__ el, int n_elem,
                                              double beta0_sq, double inv_gamma0_sq, bool quads,
                                              const double* __restrict__ qc, size_t n) {
  bool changed = false;
#pragma unroll 1
  for (int i = 0; i < n_elem; ++i) {
    const DevElem e = el[i];
    switch (e.type) {
      case SC_DRIFT: map_drift(s, e, k); break;
      case SC_QUAD: {
        const int fam = e.flags >> QF_FAM_SHIFT;
        if (qc && fam && !changed)
          map_quad_cached(s, e, qc + (size_t)(fam - 1) * 6 * n, n, k);
        else
          map_quad(s, e, k, inv_gamma0_sq);
        break;
      }
      case SC_SEXT:
        if (XE)
          map_sext(s, e, k, inv_gamma0_sq);
        else
          sext_kick(s, e.p[0], e.p[1]);
        break;
      case SC_BEND: map_bend(s, e, k, inv_gamma0_sq); break;
      case SC_EXACT_BEND:
        if (XE) map_exact_bend(s, e, k);
        break;
      case SC_RF:
        map_rf(s, e);
        ps_const(k, s.ps, beta0_sq, quads);
        changed = true;
        break;
      default: break;
    }
  }
  return changed;
}

}  // namespace sc
