// The More-Thuente line search the paper uses for Step III (Section 2.1,
// Eq. linesearch; Section 2.4 parameters; method of J. J. More and
// D. J. Thuente, ACM TOMS 20(3), 1994), as device functions:
//  * sufficient decrease  phi(a) <= phi(0) + ftol a phi'(0),
//    curvature            |phi'(a)| <= gtol |phi'(0)|;
//  * stage 1 works on psi(a) = phi(a) - phi(0) - ftol a phi'(0) until a trial
//    has psi <= 0 and phi' >= min(ftol, gtol) phi'(0);
//  * trial selection by the four cases of cubic / quadratic / secant
//    interpolation, the interval update rules, extrapolation into
//    [a_t + 1.1 (a_t - a_l), a_t + 4 (a_t - a_l)] while unbracketed, and
//    bisection when a bracketed interval fails to shrink by 0.66 in two trials.
//
// The quotients and the square root of the interpolation formulas use the
// Newton-refined FP64 operations (div_nr, sqrt_nr): the search runs in one
// thread, where each IEEE divide or sqrt is a ~650-cycle serial chain.
#pragma once

#include "linesearch.cuh"
#include "newton.cuh"

namespace cpg {
namespace mtdev {
struct Pt {
  double a, f, g;
};

// Local minimiser of the cubic with values/derivatives (a, fa, da), (b, fb, db).
__device__ inline bool cubic_min(double a, double fa, double da, double b, double fb, double db, double* x) {
  const double d1 = da + db - div_nr(3.0 * (fa - fb), a - b);
  const double disc = d1 * d1 - da * db;
  if (!(disc >= 0.0)) return false;
  const double d2 = copysign(sqrt_nr(disc), b - a);
  const double den = db - da + 2.0 * d2;
  if (den == 0.0) return false;
  *x = b - div_nr((b - a) * (db + d2 - d1), den);
  return true;
}

// Minimiser of the quadratic matching fa, da at a and fb at b.
__device__ inline bool quad_min(double a, double fa, double da, double b, double fb, double* x) {
  const double h = b - a;
  const double den = 2.0 * (fb - fa - da * h);
  if (den == 0.0) return false;
  *x = a - div_nr(da * h * h, den);
  return true;
}

// Minimiser of the quadratic matching derivatives da at a and db at b.
__device__ inline bool secant_min(double a, double da, double b, double db, double* x) {
  if (db == da) return false;
  *x = b - div_nr(db * (b - a), db - da);
  return true;
}

// Case analysis for the next trial and the interval update.
__device__ inline double next_trial(Pt& lo, Pt& hi, const Pt& t, int& brackt, double xlo, double xhi) {
  double nxt;
  if (t.f > lo.f) {                              // case 1
    double c, q;
    bool hc = cubic_min(lo.a, lo.f, lo.g, t.a, t.f, t.g, &c);
    bool hq = quad_min(lo.a, lo.f, lo.g, t.a, t.f, &q);
    if (!hc && hq) { c = q; hc = true; }
    if (!hq && hc) { q = c; hq = true; }
    if (!hc)
      nxt = lo.a + 0.5 * (t.a - lo.a);
    else
      nxt = fabs(c - lo.a) < fabs(q - lo.a) ? c : c + 0.5 * (q - c);
    brackt = 1;
  } else if (t.g * lo.g < 0.0) {                 // case 2
    double c, s;
    bool hc = cubic_min(lo.a, lo.f, lo.g, t.a, t.f, t.g, &c);
    bool hs = secant_min(lo.a, lo.g, t.a, t.g, &s);
    if (!hc && hs) { c = s; hc = true; }
    if (!hs && hc) { s = c; hs = true; }
    if (!hc)
      nxt = lo.a + 0.5 * (t.a - lo.a);
    else
      nxt = fabs(c - t.a) >= fabs(s - t.a) ? c : s;
    brackt = 1;
  } else if (fabs(t.g) <= fabs(lo.g)) {          // case 3
    double c, s;
    const double fwd = t.a - lo.a;
    if (!cubic_min(lo.a, lo.f, lo.g, t.a, t.f, t.g, &c) || (c - t.a) * fwd <= 0.0)
      c = t.a > lo.a ? xhi : xlo;
    if (!secant_min(lo.a, lo.g, t.a, t.g, &s)) s = c;
    if (brackt) {
      nxt = fabs(c - t.a) < fabs(s - t.a) ? c : s;
      const double lim = t.a + 0.66 * (hi.a - t.a);
      nxt = t.a > lo.a ? fmin(lim, nxt) : fmax(lim, nxt);
    } else {
      nxt = fabs(c - t.a) > fabs(s - t.a) ? c : s;
      nxt = fmin(xhi, fmax(xlo, nxt));
    }
  } else {                                       // case 4
    if (brackt) {
      double c;
      nxt = cubic_min(t.a, t.f, t.g, hi.a, hi.f, hi.g, &c) ? c : t.a + 0.5 * (hi.a - t.a);
    } else {
      nxt = t.a > lo.a ? xhi : xlo;
    }
  }
  if (t.f > lo.f) {
    hi = t;
  } else {
    if (t.g * (lo.a - t.a) < 0.0) hi = lo;
    lo = t;
  }
  return nxt;
}


__device__ inline void mt_advance(MTState* st, const double* fval, const double* gval) {
  MTState s = *st;
  if (s.done) return;
  const double f = *fval, g = *gval;
  s.stp_eval = s.stp;
  s.f = f;
  s.g = g;
  s.nfev += 1;
  const double stp = s.stp;
  const double ftest = s.f0 + stp * s.ftol * s.g0;
  int info = 0;
  if (s.brackt && (stp <= s.imin || stp >= s.imax)) info = 6;
  if (s.brackt && s.imax - s.imin <= s.xtol * s.imax) info = 2;
  if (stp == s.stpmax && f <= ftest && g <= s.ftol * s.g0) info = 5;
  if (stp == s.stpmin && (f > ftest || g >= s.ftol * s.g0)) info = 4;
  if (s.nfev >= s.maxfev) info = 3;
  if (f <= ftest && fabs(g) <= s.gtol * (-s.g0)) info = 1;
  if (!isfinite(f) || !isfinite(g)) info = 7;
  if (info) {
    s.info = info;
    s.done = 1;
    *st = s;
    return;
  }
  if (s.stage == 1 && f <= ftest && g >= fmin(s.ftol, s.gtol) * s.g0) s.stage = 2;
  Pt lo{s.lo_a, s.lo_f, s.lo_g}, hi{s.hi_a, s.hi_f, s.hi_g}, t{stp, f, g};
  const double xlo = stp + 1.1 * (stp - lo.a);
  const double xhi = stp + 4.0 * (stp - lo.a);
  double nxt;
  if (s.stage == 1 && f <= lo.f && f > ftest) {
    // auxiliary function psi
    const double c = s.ftol * s.g0;
    Pt lm{lo.a, lo.f - s.f0 - lo.a * c, lo.g - c};
    Pt hm{hi.a, hi.f - s.f0 - hi.a * c, hi.g - c};
    Pt tm{t.a, t.f - s.f0 - t.a * c, t.g - c};
    nxt = next_trial(lm, hm, tm, s.brackt, xlo, xhi);
    lo = Pt{lm.a, lm.f + s.f0 + lm.a * c, lm.g + c};
    hi = Pt{hm.a, hm.f + s.f0 + hm.a * c, hm.g + c};
  } else {
    nxt = next_trial(lo, hi, t, s.brackt, xlo, xhi);
  }
  if (s.brackt) {
    if (fabs(hi.a - lo.a) >= 0.66 * s.width1) nxt = lo.a + 0.5 * (hi.a - lo.a);
    s.width1 = s.width;
    s.width = fabs(hi.a - lo.a);
    s.imin = fmin(lo.a, hi.a);
    s.imax = fmax(lo.a, hi.a);
  } else {
    s.imin = xlo;
    s.imax = xhi;
  }
  nxt = fmin(fmax(nxt, s.stpmin), s.stpmax);
  if (s.brackt && (nxt <= s.imin || nxt >= s.imax || s.imax - s.imin <= s.xtol * s.imax))
    nxt = lo.a;
  s.stp = nxt;
  s.lo_a = lo.a; s.lo_f = lo.f; s.lo_g = lo.g;
  s.hi_a = hi.a; s.hi_f = hi.f; s.hi_g = hi.g;
  *st = s;
}


}  // namespace mtdev
}  // namespace cpg
