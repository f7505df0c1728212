// The More-Thuente line search of Step III (Section 2.1, Eq. linesearch;
// parameters of Section 2.4; J. J. More and D. J. Thuente, "Line search
// algorithms with guaranteed sufficient decrease", ACM TOMS 20(3), 1994),
// as device functions that advance a search by one evaluated trial.
//
// Written from the method's definitions:
//  * the search ends when a trial meets the sufficient-decrease condition
//    phi(a) <= phi(0) + ftol a phi'(0) and the curvature condition
//    |phi'(a)| <= gtol |phi'(0)|, or when it cannot go on (interval below
//    xtol, maxfev trials, a bound reached, no progress possible);
//  * while no trial has had psi(a) <= 0 and phi'(a) >= min(ftol, gtol)
//    phi'(0), a trial above the sufficient-decrease line that is no higher
//    than the best point is handled on psi(a) = phi(a) - phi(0) - ftol a
//    phi'(0) instead of phi;
//  * the next trial comes from the four cases of the trial-value selection
//    (new value higher; slopes of opposite sign; slope flattening; slope
//    steepening), built from the local minimiser of the Hermite cubic, the
//    minimiser of the quadratic through two values and one slope, and the
//    zero of the secant of the two slopes;
//  * the interval of uncertainty follows the updating rules U1-U3; while
//    it is open, trials extrapolate into [a_t + 1.1 (a_t - a_l),
//    a_t + 4 (a_t - a_l)]; a bracket that has not shrunk to 0.66 of its width
//    two trials earlier is bisected; a trial outside the bracket, or a
//    bracket below xtol, sends the search back to its best point.
//
// Quotients and square roots use the Newton-refined FP64 operations
// (div_nr, sqrt_nr): the search runs in one thread, where each IEEE divide or
// square root is a serial chain of about 650 cycles.
#pragma once

#include "linesearch.cuh"
#include "newton.cuh"

namespace cpg {
namespace mtdev {

// A point of the search: step, value and slope (of phi, or of psi).
struct Pt {
  double a, f, g;
};

// Interpolants between two points p and q, in the local coordinate
// s = (x - p.a) / h with h = q.a - p.a.  hp = h p.g and hq = h q.g are the
// slopes per unit s.

// Local minimiser of the cubic with the values and slopes of p and q:
// c(s) = p.f + hp s + c2 s^2 + c3 s^3 with c2 = 3 df - 2 hp - hq,
// c3 = hp + hq - 2 df.  c'(s) = 0 at s = (-c2 +- sqrt(D)) / (3 c3),
// D = c2^2 - 3 c3 hp; the minimiser is the root where c'' = 2 sqrt(D) > 0.
// Both forms of that root, (sqrt(D) - c2) / (3 c3) and -hp / (c2 + sqrt(D)),
// are used where they add quantities of one sign: the second for c2 >= 0,
// the first for c2 < 0.  False when the cubic has no local minimiser (D < 0,
// or a parabola that opens downwards).
__device__ inline bool hermite_cubic_argmin(const Pt& p, const Pt& q, double* x) {
  const double h = q.a - p.a;
  const double df = q.f - p.f;
  const double hp = h * p.g, hq = h * q.g;
  const double c2 = 3.0 * df - 2.0 * hp - hq;
  const double c3 = hp + hq - 2.0 * df;
  const double D = c2 * c2 - 3.0 * c3 * hp;
  if (!(D >= 0.0)) return false;
  const double sq = sqrt_nr(D);
  double s;
  if (c2 >= 0.0 && c2 + sq != 0.0) {
    s = -div_nr(hp, c2 + sq);
  } else if (c3 != 0.0) {
    s = div_nr(sq - c2, 3.0 * c3);
  } else {
    return false;
  }
  *x = p.a + s * h;
  return true;
}

// Stationary point of the quadratic with p's value and slope and q's value:
// v(s) = p.f + hp s + (df - hp) s^2.
__device__ inline bool value_quadratic_argmin(const Pt& p, const Pt& q, double* x) {
  const double h = q.a - p.a;
  const double curv = (q.f - p.f) - h * p.g;
  if (curv == 0.0) return false;
  *x = p.a - div_nr(h * p.g * h, 2.0 * curv);
  return true;
}

// Zero of the straight line through the slopes of p and q (the minimiser of
// the quadratic with those two slopes): s = p.g / (p.g - q.g).
__device__ inline bool slope_secant_zero(const Pt& p, const Pt& q, double* x) {
  const double dg = p.g - q.g;
  if (dg == 0.0) return false;
  *x = p.a + (q.a - p.a) * div_nr(p.g, dg);
  return true;
}

// A search from phi(0) = f0 and phi'(0) = g0 < 0 (done at once, info -1,
// when g0 is not negative): first trial stp0 clamped to [stpmin, stpmax],
// no bracket yet, first stage.
__device__ inline void mt_init(MTState& s, double f0, double g0, const cp_ls_opts& o) {
  s.ftol = o.ftol;
  s.gtol = o.gtol;
  s.xtol = o.xtol;
  s.stpmin = o.stpmin;
  s.stpmax = o.stpmax;
  s.maxfev = o.maxfev;
  s.f0 = f0;
  s.g0 = g0;
  s.nfev = 0;
  s.info = 0;
  s.done = 0;
  s.brackt = 0;
  s.stage = 1;
  s.lo_a = 0.0; s.lo_f = f0; s.lo_g = g0;
  s.hi_a = 0.0; s.hi_f = f0; s.hi_g = g0;
  s.width = o.stpmax - o.stpmin;
  s.width1 = 2.0 * s.width;
  s.stp = fmin(fmax(o.stp0, o.stpmin), o.stpmax);
  s.imin = 0.0;
  s.imax = s.stp + 4.0 * s.stp;
  s.stp_eval = s.stp;
  s.f = f0;
  s.g = g0;
  if (!(g0 < 0.0)) {
    s.info = -1;
    s.done = 1;
    s.stp_eval = 0.0;
  }
}

enum TrialCase { kHigher = 1, kSlopesCross = 2, kFlattening = 3, kSteepening = 4 };

__device__ inline int classify(const Pt& l, const Pt& t) {
  if (t.f > l.f) return kHigher;
  if (t.g * l.g < 0.0) return kSlopesCross;
  return fabs(t.g) <= fabs(l.g) ? kFlattening : kSteepening;
}

// Trial-value selection.  l: best point so far, u: other end of the
// interval, t: newest trial; [bmin, bmax]: the extrapolation range while the
// interval is open.  An interpolant without a minimiser is replaced by the
// other one of its case; with neither, the midpoint of l and t is taken.
__device__ inline double select_trial(const Pt& l, const Pt& u, const Pt& t, int& brackt, double bmin,
                                      double bmax) {
  const int c = classify(l, t);
  const double dir_bound = t.a > l.a ? bmax : bmin;   // bound in the direction of the step
  if (c == kHigher || c == kSlopesCross) {
    double xc, xo;
    bool hc = hermite_cubic_argmin(l, t, &xc);
    bool ho = c == kHigher ? value_quadratic_argmin(l, t, &xo) : slope_secant_zero(l, t, &xo);
    brackt = 1;
    if (!hc && !ho) return l.a + 0.5 * (t.a - l.a);
    if (!hc) xc = xo;
    if (!ho) xo = xc;
    if (c == kHigher)                       // the cubic step if nearer a_l
      return fabs(xc - l.a) < fabs(xo - l.a) ? xc : xc + 0.5 * (xo - xc);
    return fabs(xc - t.a) >= fabs(xo - t.a) ? xc : xo;   // the farther from a_t
  }
  if (c == kFlattening) {
    double xc, xs;
    // the cubic step counts only if it lies beyond a_t in the step's direction
    if (!hermite_cubic_argmin(l, t, &xc) || !((xc - t.a) * (t.a - l.a) > 0.0)) xc = dir_bound;
    if (!slope_secant_zero(l, t, &xs)) xs = xc;
    if (brackt) {
      const double nearer = fabs(xc - t.a) < fabs(xs - t.a) ? xc : xs;
      const double cap = t.a + 0.66 * (u.a - t.a);
      return t.a > l.a ? fmin(cap, nearer) : fmax(cap, nearer);
    }
    const double farther = fabs(xc - t.a) > fabs(xs - t.a) ? xc : xs;
    return fmin(bmax, fmax(bmin, farther));
  }
  // kSteepening
  if (!brackt) return dir_bound;
  double xc;
  return hermite_cubic_argmin(t, u, &xc) ? xc : t.a + 0.5 * (u.a - t.a);
}

// Updating rules of the interval: U1 a higher trial becomes the other end;
// otherwise the trial becomes the best point, and the old best point becomes
// the other end when the trial's slope points back towards it (U3), else
// the other end stays (U2).
__device__ inline void update_interval(Pt& l, Pt& u, const Pt& t) {
  if (t.f > l.f) {
    u = t;
  } else if (t.g * (l.a - t.a) < 0.0) {
    u = l;
    l = t;
  } else {
    l = t;
  }
}

// Take in phi and phi' at the step st->stp, decide whether the search ends
// (st->info, st->done) and otherwise choose the next step.
__device__ inline void mt_advance(MTState* st, const double* fval, const double* gval) {
  MTState s = *st;
  if (s.done) return;
  const double f = *fval, g = *gval;
  const double a = s.stp;
  s.stp_eval = a;
  s.f = f;
  s.g = g;
  s.nfev += 1;
  const double line = s.f0 + a * s.ftol * s.g0;        // sufficient-decrease line at a
  const bool decrease = f <= line;
  // exit codes, highest priority first
  int info = 0;
  if (!isfinite(f) || !isfinite(g)) info = 7;
  else if (decrease && fabs(g) <= s.gtol * (-s.g0)) info = 1;
  else if (s.nfev >= s.maxfev) info = 3;
  else if (a == s.stpmin && (!decrease || g >= s.ftol * s.g0)) info = 4;
  else if (a == s.stpmax && decrease && g <= s.ftol * s.g0) info = 5;
  else if (s.brackt && s.imax - s.imin <= s.xtol * s.imax) info = 2;
  else if (s.brackt && (a <= s.imin || a >= s.imax)) info = 6;
  if (info) {
    s.info = info;
    s.done = 1;
    *st = s;
    return;
  }
  if (s.stage == 1 && decrease && g >= fmin(s.ftol, s.gtol) * s.g0) s.stage = 2;
  Pt l{s.lo_a, s.lo_f, s.lo_g}, u{s.hi_a, s.hi_f, s.hi_g};
  const Pt t{a, f, g};
  const double bmin = a + 1.1 * (a - l.a);
  const double bmax = a + 4.0 * (a - l.a);
  double next;
  if (s.stage == 1 && f <= l.f && !decrease) {
    // first stage: the same selection on psi, whose value at x is
    // phi(x) - phi(0) - x ftol phi'(0) and whose slope is phi'(x) - ftol phi'(0)
    const double k = s.ftol * s.g0;
    Pt lp{l.a, l.f - s.f0 - l.a * k, l.g - k};
    Pt up{u.a, u.f - s.f0 - u.a * k, u.g - k};
    const Pt tp{t.a, t.f - s.f0 - t.a * k, t.g - k};
    next = select_trial(lp, up, tp, s.brackt, bmin, bmax);
    update_interval(lp, up, tp);
    l = Pt{lp.a, lp.f + s.f0 + lp.a * k, lp.g + k};
    u = Pt{up.a, up.f + s.f0 + up.a * k, up.g + k};
  } else {
    next = select_trial(l, u, t, s.brackt, bmin, bmax);
    update_interval(l, u, t);
  }
  if (s.brackt) {
    const double w = fabs(u.a - l.a);
    if (w >= 0.66 * s.width1) next = l.a + 0.5 * (u.a - l.a);   // too slow: bisect
    s.width1 = s.width;
    s.width = w;
    s.imin = fmin(l.a, u.a);
    s.imax = fmax(l.a, u.a);
  } else {
    s.imin = bmin;
    s.imax = bmax;
  }
  next = fmin(fmax(next, s.stpmin), s.stpmax);
  // no progress possible: return to the best point
  if (s.brackt && (next <= s.imin || next >= s.imax || s.imax - s.imin <= s.xtol * s.imax)) next = l.a;
  s.stp = next;
  s.lo_a = l.a; s.lo_f = l.f; s.lo_g = l.g;
  s.hi_a = u.a; s.hi_f = u.f; s.hi_g = u.g;
  *st = s;
}

}  // namespace mtdev
}  // namespace cpg
