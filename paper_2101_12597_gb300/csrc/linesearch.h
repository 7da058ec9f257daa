// Line search of one ETDM step (Eq. 25-29) as a resumable state machine: it
// asks for the energy and directional derivative at one step length at a
// time, so a minimizer can evaluate many systems' trial points together.
//
// Rules (the paper names the conditions, not the bracketing): alpha = 1 first;
// accept on strong Wolfe (Eq. 25-26) or on approximate Wolfe (Eq. 27) with the
// energy condition Eq. 28, constants Eq. 29; otherwise bracket by doubling or
// cubic extrapolation (the cubic's minimum taken when it lies in [1.1, 4]
// times the current step, else twice the step), then zoom with the cubic
// through the bracket ends (kept inside the middle 80 % of the bracket, else
// the midpoint); at most 20 trials; if none is accepted, the best point seen
// (the bracket's low end) is evaluated once more and taken, unless it is the
// start point.
#pragma once

#include <math.h>

namespace etdm {

constexpr double kC1 = 1e-4, kC2 = 0.9, kDel = 0.1, kSig = 0.9, kEpsE = 1e-6;
constexpr int kMaxTrials = 20;

inline bool cubic_min(double a, double fa, double da, double b, double fb, double db,
                      double *out) {
  if (a == b) return false;
  double d1 = da + db - 3.0 * (fa - fb) / (a - b);
  double disc = d1 * d1 - da * db;
  if (disc < 0.0) return false;
  double d2 = copysign(sqrt(disc), b - a);
  double den = db - da + 2.0 * d2;
  if (den == 0.0) return false;
  *out = b - (b - a) * (db + d2 - d1) / den;
  return true;
}

inline bool wolfe_ok(double alpha, double E, double d, double E0, double d0) {
  bool strong = (E <= E0 + kC1 * alpha * d0) && (fabs(d) <= kC2 * fabs(d0));
  bool approx = ((2.0 * kDel - 1.0) * d0 >= d) && (d >= kSig * d0) && (E <= E0 + kEpsE * fabs(E0));
  return strong || approx;
}

struct LsPoint {
  double a, E, d;  // step length, energy, directional derivative g . p
};

class LineSearch {
 public:
  // a new search from E0 with slope d0 (< 0) along the direction
  void start(double E0, double d0) {
    E0_ = E0;
    d0_ = d0;
    prev_ = LsPoint{0.0, E0, d0};
    trials_ = 0;
    bracket_ = false;
    accepted_ = false;
    phase_ = kBracket;
    alpha_ = 1.0;
  }
  bool done() const { return phase_ == kDone; }
  double alpha() const { return alpha_; }  // the step length to evaluate next
  bool accepted() const { return accepted_; }
  const LsPoint &result() const { return cur_; }  // valid once done() and accepted()
  int trials() const { return trials_; }

  // the energy and slope at alpha()
  void feed(double E, double d) {
    const LsPoint cur{alpha_, E, d};
    if (phase_ == kFinal) {  // the best point, evaluated again (not a trial)
      cur_ = cur;
      accepted_ = true;
      phase_ = kDone;
      return;
    }
    ++trials_;
    if (wolfe_ok(cur.a, cur.E, cur.d, E0_, d0_)) {
      cur_ = cur;
      accepted_ = true;
      phase_ = kDone;
      return;
    }
    if (phase_ == kBracket) {
      if (cur.E > E0_ + kC1 * cur.a * d0_ || (trials_ > 1 && cur.E >= prev_.E)) {
        lo_ = prev_;
        hi_ = cur;
        bracket_ = true;
        zoom();
        return;
      }
      if (cur.d >= 0.0) {
        lo_ = cur;
        hi_ = prev_;
        bracket_ = true;
        zoom();
        return;
      }
      double nxt;
      if (!cubic_min(prev_.a, prev_.E, prev_.d, cur.a, cur.E, cur.d, &nxt) ||
          !(1.1 * cur.a <= nxt && nxt <= 4.0 * cur.a))
        nxt = 2.0 * cur.a;
      prev_ = cur;
      alpha_ = nxt;
      if (trials_ >= kMaxTrials) finish();
      return;
    }
    // zoom
    if (cur.E > E0_ + kC1 * cur.a * d0_ || cur.E >= lo_.E) {
      hi_ = cur;
    } else {
      if (cur.d * (hi_.a - lo_.a) >= 0.0) hi_ = lo_;
      lo_ = cur;
    }
    zoom();
  }

 private:
  enum { kBracket, kZoom, kFinal, kDone };

  void zoom() {
    if (trials_ >= kMaxTrials) {
      finish();
      return;
    }
    phase_ = kZoom;
    const double w = fabs(hi_.a - lo_.a), left = fmin(lo_.a, hi_.a), right = fmax(lo_.a, hi_.a);
    double aj;
    if (!cubic_min(lo_.a, lo_.E, lo_.d, hi_.a, hi_.E, hi_.d, &aj) ||
        !(left + 0.1 * w <= aj && aj <= right - 0.1 * w))
      aj = 0.5 * (lo_.a + hi_.a);
    alpha_ = aj;
  }

  // no acceptable point within the trial limit: the best point seen
  void finish() {
    const LsPoint best = bracket_ ? lo_ : prev_;
    if (best.a != 0.0) {
      phase_ = kFinal;
      alpha_ = best.a;
    } else {
      phase_ = kDone;
    }
  }

  double E0_ = 0.0, d0_ = 0.0, alpha_ = 1.0;
  LsPoint prev_{}, lo_{}, hi_{}, cur_{};
  int trials_ = 0, phase_ = kDone;
  bool bracket_ = false, accepted_ = false;
};

}  // namespace etdm
