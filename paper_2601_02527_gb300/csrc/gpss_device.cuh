// Device-side arithmetic of the augmented state-space filter.
//
// Notation follows the paper (arXiv 2601.02527): for one SHO term with
// angular frequency omega0 and quality Q (Appendix B), write
//   a    = omega0 / (2Q)             (decay rate of the impulse response)
//   beta = omega0^2 (1 - 1/(4 Q^2))  (squared oscillation frequency, eta^2 omega0^2)
//   w2   = omega0^2 = beta + a^2
//   Qc   = 2 omega0^3 sigma^2 / Q    (driving-noise density, Eq. sho_Qc_Pinf)
// Matern-3/2 is the same oscillator at Q = 1/2 (beta = 0).
//
// Everything per step follows from the impulse response f(t) = Phi_12(t),
// f'' + 2a f' + w2 f = 0, f(0) = 0, f'(0) = 1:
//   Phi(t)   = [[f' + 2a f, f], [-w2 f, f']]                      (Eq. sho_phi)
//   Phibar_x = [f + 2a F1, F1],  F1 = int_0^t f                   (Eq. sho_phibar)
//   Q(t)     = Qc [[I_ff, f^2/2], [f^2/2, I_pp]]                   (Eq. Q)
//   Q~12     = Qc [F1^2/2, f F1 - I_ff]                           (Eq. analytic_Qaug12)
//   Q~22     = Qc I_FF                                            (Eq. analytic_Qaug22)
// with I_ff = int f^2, I_pp = int f'^2, I_FF = int F1^2 over [0, t].  These
// six scalars (Disc below) are computed once per term per step.
//
// FP32 evaluation: the closed forms cancel catastrophically for small
// omega0 t (the z-noise I_FF ~ t^5/20 is a difference of O(1) terms).  For
// w2 t^2 <= XT2 (omega0 t <= 1.2) the six scalars come from their Taylor series in t, whose
// coefficients follow from the recurrence of f (the chunk kernels read an
// economised form of them from per-row tables); above it from closed forms
// rewritten through the identities
//   w2 F1  = 1 - f' - 2a f
//   4a I_pp = 1 - f'^2 - w2 f^2
//   w2 I_ff = I_pp - f f' - a f^2
//   w2^2 I_FF = t + I_pp + 4a^2 I_ff - 2f - 4a F1 + 2a f^2
// (integrals of the oscillator equation multiplied by f', f and of F1^2),
// which stay accurate once the exponential has decayed.
//
// Overdamped oscillator (Q < 1/2, beta < 0; the cosh/sinh transition of
// Appendix B): f = e^{-a t} sinh(b t)/b, b = sqrt(-beta), decays with the two
// rates l1 = w2/(a + b) (slow) and a + b (fast).  The Taylor branch then
// covers (a + b) t <= 1.2 (its convergence is set by the fast rate) and the
// identities above need the slow mode to have decayed (l1 t >= 1.2: below
// that they cancel like (a + b)^4 / w2^2).  In between, the step is halved
// into the Taylor range and the integrals doubled back with the semigroup
// identities of the augmented model, Phi~(2t) = Phi~(t)^2 and Q~(2t) =
// Phi~(t) Q~(t) Phi~(t)^T + Q~(t), written on the six scalars
// (disc_double_integrals), with f and f' evaluated directly from the two
// decaying modes at every level.
#pragma once

#include <cuda_runtime.h>
#include <math.h>

#include <atomic>
#include <stdint.h>

#define GPSS_HD __host__ __device__ __forceinline__
#define GPSS_HDNI static __host__ __device__ __noinline__
#define GPSS_D __device__ __forceinline__

namespace gpss {

// Kernels launched by this library in the process (counted on the host at
// each launch; launches replayed from a captured CUDA graph are not counted).
inline std::atomic<long long> g_launches{0};
#define GPSS_COUNT_LAUNCH() (::gpss::g_launches.fetch_add(1, std::memory_order_relaxed))

// ---------------------------------------------------------------------------
// Compile-time shape of the augmented state.
//   NT terms (state (x_t, xdot_t) each), NS instrument slots,
//   LAYOUT 0: one integral state z_j per slot integrating H x = sum_t x_t,
//   LAYOUT 1: one z_{t,j} per term and slot integrating x_t.
// ---------------------------------------------------------------------------
template <int NT_, int NS_, int LAYOUT_>
struct Shape {
  static constexpr int NT = NT_;
  static constexpr int NS = NS_;
  static constexpr int LAYOUT = (NT_ == 1) ? 0 : LAYOUT_;
  static constexpr int NZPER = (LAYOUT == 0) ? 1 : NT;
  static constexpr int NZ = NS * NZPER;
  static constexpr int D = 2 * NT + NZ;
  static constexpr int NP = D * (D + 1) / 2;  // packed upper triangle
  static GPSS_HD constexpr int zslot(int zi) {
    return LAYOUT == 0 ? zi - 2 * NT : (zi - 2 * NT) / NT;
  }
  static GPSS_HD constexpr bool zint(int zi, int t) {
    return LAYOUT == 0 ? true : ((zi - 2 * NT) % NT) == t;
  }
  static GPSS_HD constexpr int pk(int i, int j) {
    return i <= j ? i * D - i * (i - 1) / 2 + (j - i) : j * D - j * (j - 1) / 2 + (i - j);
  }
};

// ---------------------------------------------------------------------------
// Forward-mode dual number with two tangents, (d/da, d/dbeta).  Used only to
// differentiate the per-step discretisation in the reverse-time gradient.
// ---------------------------------------------------------------------------
template <class F>
struct Dual2 {
  F v, da, db;
};

template <class F> GPSS_HD Dual2<F> mk(F v, F da, F db) { return Dual2<F>{v, da, db}; }
template <class F> GPSS_HD Dual2<F> operator+(Dual2<F> x, Dual2<F> y) { return mk(x.v + y.v, x.da + y.da, x.db + y.db); }
template <class F> GPSS_HD Dual2<F> operator-(Dual2<F> x, Dual2<F> y) { return mk(x.v - y.v, x.da - y.da, x.db - y.db); }
template <class F> GPSS_HD Dual2<F> operator-(Dual2<F> x) { return mk(-x.v, -x.da, -x.db); }
template <class F> GPSS_HD Dual2<F> operator*(Dual2<F> x, Dual2<F> y) {
  return mk(x.v * y.v, x.da * y.v + x.v * y.da, x.db * y.v + x.v * y.db);
}
template <class F> GPSS_HD Dual2<F> operator/(Dual2<F> x, Dual2<F> y) {
  F iy = F(1) / y.v;
  F q = x.v * iy;
  return mk(q, (x.da - q * y.da) * iy, (x.db - q * y.db) * iy);
}
template <class F> GPSS_HD Dual2<F> operator+(Dual2<F> x, F c) { return mk(x.v + c, x.da, x.db); }
template <class F> GPSS_HD Dual2<F> operator+(F c, Dual2<F> x) { return mk(x.v + c, x.da, x.db); }
template <class F> GPSS_HD Dual2<F> operator-(Dual2<F> x, F c) { return mk(x.v - c, x.da, x.db); }
template <class F> GPSS_HD Dual2<F> operator-(F c, Dual2<F> x) { return mk(c - x.v, -x.da, -x.db); }
template <class F> GPSS_HD Dual2<F> operator*(Dual2<F> x, F c) { return mk(x.v * c, x.da * c, x.db * c); }
template <class F> GPSS_HD Dual2<F> operator*(F c, Dual2<F> x) { return mk(x.v * c, x.da * c, x.db * c); }
template <class F> GPSS_HD Dual2<F> operator/(Dual2<F> x, F c) { F ic = F(1) / c; return mk(x.v * ic, x.da * ic, x.db * ic); }

template <class F> struct Real { using type = F; };
template <class F> struct Real<Dual2<F>> { using type = F; };

// constant of type T
template <class T> struct Cst { static GPSS_HD T of(T v) { return v; } };
template <class F> struct Cst<Dual2<F>> { static GPSS_HD Dual2<F> of(F v) { return mk(v, F(0), F(0)); } };
template <class T, class F> GPSS_HD T cst(F v) { return Cst<T>::of(v); }

GPSS_HD float val(float x) { return x; }
GPSS_HD double val(double x) { return x; }
template <class F> GPSS_HD F val(Dual2<F> x) { return x.v; }

GPSS_HD float gexp(float x) { return expf(x); }
GPSS_HD double gexp(double x) { return exp(x); }
template <class F> GPSS_HD Dual2<F> gexp(Dual2<F> x) {
  F e = gexp(x.v);
  return mk(e, e * x.da, e * x.db);
}
GPSS_HD float gsqrt(float x) { return sqrtf(x); }
GPSS_HD double gsqrt(double x) { return sqrt(x); }
template <class F> GPSS_HD Dual2<F> gsqrt(Dual2<F> x) {
  F r = gsqrt(x.v), h = F(0.5) / r;
  return mk(r, h * x.da, h * x.db);
}

// S(beta, t) = sin(sqrt(beta) t) / sqrt(beta)  (= t at beta = 0),
// C(beta, t) = cos(sqrt(beta) t), for beta >= 0 (the overdamped case is
// evaluated by disc_overdamped).
GPSS_HD void sinc_pair(float beta, float t, float &S, float &C) {
  float b = sqrtf(beta);
  float tau = b * t;
  float s, c;
  sincosf(tau, &s, &c);
  C = c;
  S = (tau < 1e-3f) ? t * (1.0f - tau * tau * (1.0f / 6.0f)) : s / b;
}
GPSS_HD void sinc_pair(double beta, double t, double &S, double &C) {
  double b = sqrt(beta);
  double tau = b * t;
  double s, c;
  sincos(tau, &s, &c);
  C = c;
  S = (tau < 1e-6) ? t * (1.0 - tau * tau * (1.0 / 6.0)) : s / b;
}
// Dual version: dC/dbeta = -t S / 2; dS/dbeta = (t C - S) / (2 beta), which
// for small beta t^2 is evaluated from its series
// t^3 (-1/6 + beta t^2/60 - beta^2 t^4/1680 + beta^3 t^6/90720 - ...).
template <class F>
GPSS_HD void sinc_pair(Dual2<F> beta, F t, Dual2<F> &S, Dual2<F> &C) {
  F s, c;
  sinc_pair(beta.v, t, s, c);
  F x = beta.v * t * t;
  F dS;
  if (x < F(0.5)) {
    dS = t * t * t *
         (F(-1.0 / 6.0) + x * (F(1.0 / 60.0) + x * (F(-1.0 / 1680.0) + x * (F(1.0 / 90720.0) +
                                                                         x * F(-1.0 / 7983360.0)))));
  } else {
    dS = (t * c - s) / (F(2) * beta.v);
  }
  F dC = -t * s * F(0.5);
  S = mk(s, dS * beta.da, dS * beta.db);
  C = mk(c, dC * beta.da, dC * beta.db);
}

template <class T>
struct Disc {
  T f, fp, F1, Iff, Ipp, IFF;
};

template <class F> struct TaylorOrder;
// Degree and range of the Taylor branch: FP32 degree 16 for omega0 t <= 1.2
// and FP64 degree 20 for omega0 t <= 1 keep the truncation below the
// rounding of the closed forms that take over above (FP32: <= ~4e-6 relative
// from omega0 t = 1.2 on; below it their cancellation grows like (omega0 t)^-4).
template <> struct TaylorOrder<float> { static constexpr int N = 16; static constexpr float XT2 = 1.44f; };
template <> struct TaylorOrder<double> { static constexpr int N = 20; static constexpr double XT2 = 1.0; };

// Taylor branch: f(s) = sum_{n>=1} c_n s^n with c_1 = 1, c_2 = -a,
// c_{n+2} = -(2a (n+1) c_{n+1} + w2 c_n) / ((n+2)(n+1)); p_n = c_n t^n.
//   I_ff = t   sum p_n p_m / (n+m+1)
//   I_pp = 1/t sum n m p_n p_m / (n+m-1)
//   I_FF = t^3 sum p_n p_m / ((n+1)(m+1)(n+m+3))
// (double sums over n + m <= N + 1).
template <class T, class F>
GPSS_HD Disc<T> disc_taylor(F t, T a, T w2) {
  constexpr int N = TaylorOrder<F>::N;
  T p[N + 1];
  p[1] = cst<T>(t);
  p[2] = -a * (t * t);
  const F t2 = t * t;
#pragma unroll
  for (int n = 1; n + 2 <= N; ++n) {
    const F inv = F(1) / F((n + 2) * (n + 1));
    p[n + 2] = -(a * (F(2 * (n + 1)) * t) * p[n + 1] + w2 * t2 * p[n]) * inv;
  }
  Disc<T> d;
  T f = p[1], fp = p[1], F1 = p[1] * F(0.5);
#pragma unroll
  for (int n = 2; n <= N; ++n) {
    f = f + p[n];
    fp = fp + p[n] * F(n);
    F1 = F1 + p[n] * (F(1) / F(n + 1));
  }
  T sff = p[1] * p[1] * (F(1) / F(3));
  T spp = p[1] * p[1];
  T sFF = p[1] * p[1] * (F(1) / F(4 * 5));
#pragma unroll
  for (int n = 1; n <= N; ++n) {
#pragma unroll
    for (int m = n; m <= N; ++m) {
      if (n + m > N + 1 || (n == 1 && m == 1)) continue;
      const F mult = (n == m) ? F(1) : F(2);
      const T pp = p[n] * p[m];
      sff = sff + pp * (mult / F(n + m + 1));
      spp = spp + pp * (mult * F(n * m) / F(n + m - 1));
      sFF = sFF + pp * (mult / F((n + 1) * (m + 1) * (n + m + 3)));
    }
  }
  const F it = F(1) / t;
  d.f = f;
  d.fp = fp * it;
  d.F1 = F1 * t;
  d.Iff = sff * t;
  d.Ipp = spp * it;
  d.IFF = sFF * (t * t2);
  return d;
}

// Closed-form branch from f and f' through the integral identities of the
// header comment.
template <class T, class F>
GPSS_HD Disc<T> disc_from_ffp(F t, T a, T w2, T f, T fp) {
  Disc<T> d;
  d.f = f;
  d.fp = fp;
  const T rw2 = cst<T>(F(1)) / w2;
  d.F1 = (F(1) - d.fp - F(2) * a * d.f) * rw2;
  d.Ipp = (F(1) - d.fp * d.fp - w2 * d.f * d.f) / (F(4) * a);
  d.Iff = (d.Ipp - d.f * d.fp - a * d.f * d.f) * rw2;
  d.IFF = (cst<T>(t) + d.Ipp + F(4) * a * a * d.Iff - F(2) * d.f - F(4) * a * d.F1 +
           F(2) * a * d.f * d.f) *
          rw2 * rw2;
  return d;
}

template <class T, class F>
GPSS_HD Disc<T> disc_closed(F t, T a, T beta, T w2) {
  T E = gexp(-a * t);
  T S, C;
  sinc_pair(beta, t, S, C);
  return disc_from_ffp<T, F>(t, a, w2, E * S, E * (C - a * S));
}

// The integrals at 2t from the six scalars at t (Phi~(2t) = Phi~(t)^2,
// Q~(2t) = Phi~(t) Q~(t) Phi~(t)^T + Q~(t) on the blocks of one term; p =
// Phi_00, (p0, F1) = Phibar).  f and f' at 2t are left to the caller: formed
// by the same squaring their relative error would double with every step.
template <class T, class F>
GPSS_HD void disc_double_integrals(Disc<T> &d, T a, T w2) {
  const T f = d.f, fp = d.fp, F1 = d.F1, Iff = d.Iff, Ipp = d.Ipp;
  const T ff = f * f, f3 = ff * f;
  const T p = fp + F(2) * a * f;
  const T p0 = f + F(2) * a * F1;
  d.F1 = F1 * (F(1) + p) + ff;
  d.Iff = Iff * (F(1) + p * p) + p * f3 + ff * Ipp;
  d.Ipp = Ipp * (F(1) + fp * fp) + w2 * w2 * ff * Iff - w2 * fp * f3;
  d.IFF = F(2) * d.IFF + p0 * p0 * Iff + p0 * F1 * ff + F1 * F1 * Ipp + p0 * F1 * F1 +
          F(2) * F1 * (f * F1 - Iff);
}

// Number of halvings that bring a step t into the Taylor range r2 h^2 <= XT2
// (h = t / 2^k exactly; at most 64).
template <class F>
GPSS_HD int halvings(F t, F r2, F xt2, F &h) {
  int k = 0;
  h = t;
  while (r2 * h * h > xt2 && k < 64) {
    h *= F(0.5);
    ++k;
  }
  return k;
}

// e^{-a t} (sinh(b t)/b, cosh(b t)) for b t < 1/2 by their series in
// x = (b t)^2 = -beta t^2 (truncation below 1e-17 of each).
template <class T, class F>
GPSS_HD void sinhc_pair(T x, F t, T &S, T &C) {
  S = (F(1) + x * (F(1.0 / 6) + x * (F(1.0 / 120) + x * (F(1.0 / 5040) + x * (F(1.0 / 362880) +
        x * (F(1.0 / 39916800) + x * F(1.0 / 6227020800.0))))))) * t;
  C = F(1) + x * (F(0.5) + x * (F(1.0 / 24) + x * (F(1.0 / 720) + x * (F(1.0 / 40320) +
        x * (F(1.0 / 3628800) + x * (F(1.0 / 479001600) + x * F(1.0 / 87178291200.0)))))));
}

// f = e^{-a t} sinh(b t)/b and f' of the overdamped oscillator (b =
// sqrt(-beta)) without cancellation: the series below b t = 1/2, else the two
// decaying modes, f = (e^{-l1 t} - e^{-l2 t}) / (2b), f' = (l2 e^{-l2 t} -
// l1 e^{-l1 t}) / (2b), l2 = a + b, l1 = w2 / l2 (= a - b).
template <class T, class F>
GPSS_HD void od_f_fp(F t, T a, T beta, T b, T w2, T &f, T &fp) {
  if (val(b) * t < F(0.5)) {
    T S, C;
    sinhc_pair<T, F>(-beta * (t * t), t, S, C);
    const T E = gexp(-a * t);
    f = E * S;
    fp = E * (C - a * S);
  } else {
    const T l2 = a + b, l1 = w2 / l2;
    const T e1 = gexp(-l1 * t), e2 = gexp(-l2 * t);
    const T r = cst<T>(F(0.5)) / b;
    f = (e1 - e2) * r;
    fp = (l2 * e2 - l1 * e1) * r;
  }
}

// Overdamped step above the Taylor range (beta < 0).  While the slow mode
// has not decayed (l1 t < sqrt(XT2)) the step is halved into the Taylor
// range and the integrals doubled back, with f and f' evaluated directly at
// every level; after that the identities from f and f'.
template <class T, class F>
GPSS_HD Disc<T> disc_overdamped(F t, T a, T beta, T w2, F r2) {
  const F xt2 = TaylorOrder<F>::XT2;
  const F l1 = val(w2) / sqrt(r2);
  const T b = gsqrt(-beta);
  if (l1 * t * l1 * t < xt2) {
    F h;
    const int k = halvings<F>(t, r2, xt2, h);
    Disc<T> d = disc_taylor<T, F>(h, a, w2);
    for (int i = 0; i < k; ++i) {
      disc_double_integrals<T, F>(d, a, w2);
      h *= F(2);
      od_f_fp<T, F>(h, a, beta, b, w2, d.f, d.fp);
    }
    return d;
  }
  T f, fp;
  od_f_fp<T, F>(t, a, beta, b, w2, f, fp);
  return disc_from_ffp<T, F>(t, a, w2, f, fp);
}

// Square of the fastest rate of the impulse response: w2 (beta >= 0) or
// (a + b)^2 (beta < 0); the Taylor branch serves r2 t^2 <= XT2.
template <class F>
GPSS_HD F rate2(F a, F beta) {
  if (beta >= F(0)) return beta + a * a;
  const F r = a + sqrt(-beta);
  return r * r;
}

// All six per-term scalars for a step of length t >= 0.  OD = false drops
// the overdamped branches (for hyperparameter rows without a Q < 1/2 term).
template <class T, class F, bool OD = true>
GPSS_HD Disc<T> discretize(F t, T a, T beta) {
  T w2 = beta + a * a;
  if (t == F(0)) {
    Disc<T> d;
    d.f = cst<T>(F(0));
    d.fp = cst<T>(F(1));
    d.F1 = d.f;
    d.Iff = d.f;
    d.Ipp = d.f;
    d.IFF = d.f;
    return d;
  }
  if constexpr (!OD) {
    if (val(w2) * t * t <= TaylorOrder<F>::XT2) return disc_taylor<T, F>(t, a, w2);
  } else {
    const F r2 = rate2<F>(val(a), val(beta));
    if (r2 * t * t <= TaylorOrder<F>::XT2) return disc_taylor<T, F>(t, a, w2);
    if (val(beta) < F(0)) return disc_overdamped<T, F>(t, a, beta, w2, r2);
  }
  return disc_closed<T, F>(t, a, beta, w2);
}

// Per-term constants from natural parameters, with the reciprocals and the
// oscillation frequency the closed-form branch needs precomputed:
// b = sqrt(|beta|), rb = 1/b (0 when b = 0), rw2 = 1/w2, r4a = 1/(4a),
// r2 = rate2(a, beta) (the Taylor branch's bound).
template <class F>
struct TermC {
  F a, beta, w2, qc, var;
  F b, rb, rw2, r4a, r2;
};

template <class F>
GPSS_HD void finish_termc(TermC<F> &c) {
  c.b = sqrt(fabs(c.beta));
  c.rb = c.b > F(0) ? F(1) / c.b : F(0);
  c.rw2 = F(1) / c.w2;
  c.r4a = F(1) / (F(4) * c.a);
  c.r2 = rate2<F>(c.a, c.beta);
}

// Closed-form branch with the per-term constants precomputed (no division,
// no square root per step).  S = sin(b t)/b, C = cos(b t) as in sinc_pair.
template <class T, class F>
GPSS_HD Disc<T> disc_closed_ffp(F t, T a, T w2, T rw2, T r4a, T f, T fp) {
  Disc<T> d;
  d.f = f;
  d.fp = fp;
  const T a2 = a * F(2);
  d.F1 = (F(1) - d.fp - a2 * d.f) * rw2;
  const T ff = d.f * d.f;
  d.Ipp = (F(1) - d.fp * d.fp - w2 * ff) * r4a;
  d.Iff = (d.Ipp - d.f * d.fp - a * ff) * rw2;
  d.IFF = (cst<T>(t) + d.Ipp + a2 * a2 * d.Iff - F(2) * d.f - a2 * F(2) * d.F1 + a2 * ff) *
          (rw2 * rw2);
  return d;
}

template <class T, class F>
GPSS_HD Disc<T> disc_closed_k(F t, T a, T w2, T rw2, T r4a, T S, T C) {
  const T E = gexp(-a * t);
  return disc_closed_ffp<T, F>(t, a, w2, rw2, r4a, E * S, E * (C - a * S));
}

GPSS_HD void sinc_pair_k(float t, float b, float rb, float &S, float &C) {
  const float tau = b * t;
  float s, c;
  sincosf(tau, &s, &c);
  C = c;
  S = (tau < 1e-3f) ? t * (1.0f - tau * tau * (1.0f / 6.0f)) : s * rb;
}

// ---------------------------------------------------------------------------
// Step-scalar tables.  The Taylor coefficients of the six per-term scalars
// depend only on (a, beta), so the polynomials are built once per
// hyperparameter row and evaluated per step by Horner's rule.  Each scalar is
// t^p0 * g(t), p0 = 1, 0, 2, 3, 1, 5 for f, f', F1, I_ff, I_pp, I_FF, with
// Taylor coefficients
//   g^f_k   = c_{k+1},                  g^f'_k  = (k+1) c_{k+1},
//   g^F1_k  = c_{k+1} / (k+2),
//   g^Iff_k = sum_{n+m=k+2} c_n c_m / (k+3),
//   g^Ipp_k = sum_{n+m=k+2} n m c_n c_m / (k+1),
//   g^IFF_k = sum_{n+m=k+2} c_n c_m / ((n+1)(m+1)) / (k+5),
// where f(s) = sum_{n>=1} c_n s^n (c_1 = 1, c_2 = -a,
// c_{n+2} = -(2a (n+1) c_{n+1} + w2 c_n) / ((n+2)(n+1))).
//
// The table holds the Chebyshev economisation of these series on the range
// the table serves, [0, T] with r2 T^2 = XT2 (1% margin): TAB_NTAY Taylor
// terms (truncation ~1e-13 there), then each power u^n (u = t/T) from the
// top down to TAB_NC is traded for the lower powers of the shifted Chebyshev
// polynomial T*_n(u) = T_n(2u - 1), whose leading coefficient is 2^(2n-1)
// and whose size on [0, 1] is 1.  Each step adds at most |d_n| / 2^(2n-1)
// to the maximum error, d_n the current coefficient of u^n.  With ten
// coefficients the error stays below 1e-8 of each value series' size and
// below 1e-6 of each (a, beta) tangent's (those enter only the gradient) for
// omega0 t <= 1.2 at every damping the SHO and Matern-3/2 terms allow; the
// worst case is critical damping.  The map is linear with T held fixed, so
// the tangent series are economised like the values.
//
// Unrolling of the Horner loops over the table's records (sm_103a: three)
#ifndef GPSS_HORNER_UNROLL
#define GPSS_HORNER_UNROLL _Pragma("unroll 3")
#endif

// Table layout per (row, term): for k = 0..NC-1 one record of TAB_W floats:
// [6 values, 2 pad, 6 d/da, 6 d/dbeta] (five float4: the values are read as
// two, the twelve tangents as three).
// ---------------------------------------------------------------------------
constexpr int TAB_NC = 10;
constexpr int TAB_NTAY = 22;
constexpr int TAB_W = 20;
constexpr int TAB_TERM = TAB_NC * TAB_W;

// Taylor coefficients g[j][k], k < TAB_NTAY, of the six series.
template <class T>
GPSS_HD void taylor_coeffs(T a, T beta, T (&g)[6][TAB_NTAY]) {
  constexpr int NCF = TAB_NTAY + 2;
  T c[NCF + 1];
  const T w2 = beta + a * a;
  c[0] = a * 0.0;
  c[1] = c[0] + 1.0;
  c[2] = -a;
  for (int n = 1; n + 2 <= NCF; ++n)
    c[n + 2] = -(a * (2.0 * (n + 1)) * c[n + 1] + w2 * c[n]) / (double)((n + 2) * (n + 1));
  for (int k = 0; k < TAB_NTAY; ++k) {
    g[0][k] = c[k + 1];
    g[1][k] = c[k + 1] * (double)(k + 1);
    g[2][k] = c[k + 1] / (double)(k + 2);
    T s1 = c[0], s2 = c[0], s3 = c[0];
    for (int n = 1; n <= k + 1; ++n) {
      const int m = k + 2 - n;
      const T pp = c[n] * c[m];
      s1 = s1 + pp;
      s2 = s2 + pp * (double)(n * m);
      s3 = s3 + pp / (double)((n + 1) * (m + 1));
    }
    g[3][k] = s1 / (double)(k + 3);
    g[4][k] = s2 / (double)(k + 1);
    g[5][k] = s3 / (double)(k + 5);
  }
}

// The division-free form the table kernel uses.  c[0..NCF] (NCF = TAB_NTAY
// + 2) receives f's Taylor coefficients by the recurrence, with rcp[i] = 1/i;
// then coefficient k of the six series follows from c, e_n = c_n / (n+1)
// and p_n = n c_n (same definitions as taylor_coeffs).
constexpr int TAB_NCF = TAB_NTAY + 2;

template <class T>
GPSS_HD void taylor_c(T a, T beta, const double *rcp, T *c) {
  const T w2 = beta + a * a;
  c[0] = a * 0.0;
  c[1] = c[0] + 1.0;
  c[2] = -a;
  for (int n = 1; n + 2 <= TAB_NCF; ++n)
    c[n + 2] = -(a * (2.0 * (n + 1)) * c[n + 1] + w2 * c[n]) * (rcp[n + 2] * rcp[n + 1]);
}

template <class T>
GPSS_HD void taylor_coeff_pre(const T *c, const T *e, const T *p, const double *rcp, int k,
                              T (&g)[6]) {
  T s1 = c[0], s2 = c[0], s3 = c[0];
  for (int n = 1; n <= k + 1; ++n) {
    const int m = k + 2 - n;
    s1 = s1 + c[n] * c[m];
    s2 = s2 + p[n] * p[m];
    s3 = s3 + e[n] * e[m];
  }
  g[0] = c[k + 1];
  g[1] = c[k + 1] * (double)(k + 1);
  g[2] = c[k + 1] * rcp[k + 2];
  g[3] = s1 * rcp[k + 3];
  g[4] = s2 * rcp[k + 1];
  g[5] = s3 * rcp[k + 5];
}

// Range of the table: t in [0, T], T = 1.01 sqrt(XT2 / r2), r2 = rate2(a, beta).
GPSS_HD double table_range(double r2) {
  return 1.01 * sqrt((double)TaylorOrder<float>::XT2 / r2);
}

// The economisation as a fixed linear map in u = t / T: coefficient k < NC of
// the economised polynomial is sum_n m[k][n] d_n, d_n the Taylor
// coefficients of u^n.  Built by applying the reductions (top power first)
// to the unit vectors.  Monomial coefficients of T*_n: s_{n,0} = (-1)^n and
// s_{n,j+1} = -4 (n+j)(n-j) / ((2j+1)(2j+2)) s_{n,j} (integers).
struct EconMap {
  double m[TAB_NC][TAB_NTAY];
  double rcp[2 * TAB_NTAY + 8];  // 1/i (rcp[0] unused)
};

GPSS_HD void econ_map(EconMap &E) {
  E.rcp[0] = 0.0;
  for (int i = 1; i < 2 * TAB_NTAY + 8; ++i) E.rcp[i] = 1.0 / (double)i;
  for (int col = 0; col < TAB_NTAY; ++col) {
    double d[TAB_NTAY];
    for (int k = 0; k < TAB_NTAY; ++k) d[k] = (k == col) ? 1.0 : 0.0;
    for (int n = TAB_NTAY - 1; n >= TAB_NC; --n) {
      if (d[n] == 0.0) continue;
      const double lead = ldexp(1.0, 2 * n - 1);
      double sn = (n & 1) ? -1.0 : 1.0;
      for (int k = 0; k < n; ++k) {
        d[k] -= d[n] * (sn / lead);
        sn *= -4.0 * (double)(n + k) * (double)(n - k) / ((double)(2 * k + 1) * (double)(2 * k + 2));
      }
      d[n] = 0.0;
    }
    for (int k = 0; k < TAB_NC; ++k) E.m[k][col] = d[k];
  }
}

// Table coefficient k (in t) from the Taylor coefficients g[j][n] (all n):
// e_k = sum_n m[k][n] T^(n-k) g_n.
template <class T>
GPSS_HD T econ_apply(const double (*m)[TAB_NTAY], int k, double rng, const T *g, int stride) {
  T acc = g[0] * 0.0;
  double p = 1.0;  // T^(n-k)
  for (int n = k; n < TAB_NTAY; ++n) {
    acc = acc + g[(size_t)n * stride] * (m[k][n] * p);
    p *= rng;
  }
  return acc;
}
template <class T>
GPSS_HD T econ_apply(const EconMap &E, int k, double rng, const T *g, int stride) {
  return econ_apply<T>(E.m, k, rng, g, stride);
}

// ---------------------------------------------------------------------------
// Double-float numbers for the table generation: the unevaluated sum hi + lo
// of two floats (about 48 significant bits), built on the error-free
// transformations TwoSum (Knuth) and TwoProduct by fused multiply-add
// (Dekker's product with an FMA), with the accurate addition of the
// double-double literature (both parts' errors carried).  They run on the
// FP32 pipe, which on this GPU is many times wider than the FP64 one.
// ---------------------------------------------------------------------------
struct DF {
  float hi, lo;
};
GPSS_HD DF df_of(double x) {
  const float h = (float)x;
  return DF{h, (float)(x - (double)h)};
}
GPSS_HD double df_val(DF x) { return (double)x.hi + (double)x.lo; }
GPSS_HD DF df_fast(float a, float b) {  // |a| >= |b| or a == 0
  const float s = a + b;
  return DF{s, b - (s - a)};
}
GPSS_HD DF df_two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return DF{s, (a - (s - bb)) + (b - bb)};
}
GPSS_HD DF operator+(DF x, DF y) {
  DF s = df_two_sum(x.hi, y.hi);
  const DF t = df_two_sum(x.lo, y.lo);
  s.lo += t.hi;
  s = df_fast(s.hi, s.lo);
  s.lo += t.lo;
  return df_fast(s.hi, s.lo);
}
GPSS_HD DF operator-(DF x) { return DF{-x.hi, -x.lo}; }
GPSS_HD DF operator-(DF x, DF y) { return x + (-y); }
GPSS_HD DF operator*(DF x, DF y) {
  const float p = x.hi * y.hi;
  float e = fmaf(x.hi, y.hi, -p);
  e = fmaf(x.hi, y.lo, fmaf(x.lo, y.hi, e));
  return df_fast(p, e);
}
GPSS_HD Dual2<DF> mkdf(DF v, DF da, DF db) { return Dual2<DF>{v, da, db}; }
GPSS_HD Dual2<DF> operator*(Dual2<DF> x, DF c) { return mkdf(x.v * c, x.da * c, x.db * c); }

// Table coefficients with the scale of the table's range T taken out, in
// double-float (the form the table kernel computes; FP64 inputs, FP32 pipe).
// With c~_n = c_n T^n the oscillator recurrence reads
//   c~_{n+2} = -(2 a T (n+1) c~_{n+1} + w2 T^2 c~_n) / ((n+2)(n+1)),
// c~_0 = 0, c~_1 = T, c~_2 = -a T^2, and every coefficient stays of order one
// however large or small omega0 is (omega0 T is about 1.2).  Coefficient n of
// series j times T^(n + q_j) (q = 1 for f, f', F1; 2 for I_ff, I_pp, I_FF)
// then follows from the c~ alone, and the economisation, linear with T fixed,
// maps these to the table's coefficients times T^(k + q_j).
// taylor_c_scaled: the recurrence into c (NCF + 1 entries).
GPSS_HD void taylor_c_scaled(Dual2<DF> aT, Dual2<DF> w2T2, const DF *rcp, Dual2<DF> *c,
                             DF T) {
  const DF z = df_of(0.0);
  c[0] = mkdf(z, z, z);
  c[1] = mkdf(T, z, z);
  c[2] = -(aT * T);
  for (int n = 1; n + 2 <= TAB_NCF; ++n) {
    const DF two_n1 = df_of(2.0 * (n + 1));
    c[n + 2] = -((aT * two_n1) * c[n + 1] + w2T2 * c[n]) * (rcp[n + 2] * rcp[n + 1]);
  }
}

// Coefficient k of the six scaled series from c~ (e_n = c~_n / (n+1) and
// p_n = n c~_n precomputed), as taylor_coeff_pre with the T factors out.
GPSS_HD void taylor_coeff_scaled(const Dual2<DF> *c, const Dual2<DF> *e, const Dual2<DF> *p,
                                 const DF *rcp, int k, Dual2<DF> (&g)[6]) {
  const DF z = df_of(0.0);
  Dual2<DF> s1 = mkdf(z, z, z), s2 = s1, s3 = s1;
  for (int n = 1; n <= k + 1; ++n) {
    const int m = k + 2 - n;
    s1 = s1 + c[n] * c[m];
    s2 = s2 + p[n] * p[m];
    s3 = s3 + e[n] * e[m];
  }
  g[0] = c[k + 1];
  g[1] = c[k + 1] * df_of((double)(k + 1));
  g[2] = c[k + 1] * rcp[k + 2];
  g[3] = s1 * rcp[k + 3];
  g[4] = s2 * rcp[k + 1];
  g[5] = s3 * rcp[k + 5];
}

// Economised coefficient k of one scaled series: sum_n m[k][n] g~_n.
GPSS_HD Dual2<DF> econ_apply_scaled(const DF (*m)[TAB_NTAY], int k, const Dual2<DF> *g) {
  const DF z = df_of(0.0);
  Dual2<DF> acc = mkdf(z, z, z);
  for (int n = k; n < TAB_NTAY; ++n) acc = acc + g[n] * m[k][n];
  return acc;
}

// Power of T that scales series j's coefficients (beyond T^k).
GPSS_HD int table_q(int j) { return j < 3 ? 1 : 2; }

// One term's table by the double-float path, sequentially (the table kernel
// computes the same quantities, one coefficient per lane): values and (a,
// beta) tangents of e[j][k] = table coefficient k of series j, in t.
GPSS_HD void table_coeffs_df(const EconMap &E, double a, double beta, double (&v)[6][TAB_NC],
                             double (&da)[6][TAB_NC], double (&db)[6][TAB_NC]) {
  DF rcp[2 * TAB_NTAY + 8];
  for (int i = 0; i < 2 * TAB_NTAY + 8; ++i) rcp[i] = df_of(E.rcp[i]);
  const double T = table_range(rate2<double>(a, beta));
  const DF one = df_of(1.0), zero = df_of(0.0);
  const Dual2<DF> ad = mkdf(df_of(a), one, zero), bd = mkdf(df_of(beta), zero, one);
  const Dual2<DF> w2 = bd + ad * ad;
  Dual2<DF> c[TAB_NCF + 1], e[TAB_NCF + 1], p[TAB_NCF + 1], g[6][TAB_NTAY];
  taylor_c_scaled(ad * df_of(T), w2 * df_of(T * T), rcp, c, df_of(T));
  for (int n = 0; n <= TAB_NCF; ++n) {
    e[n] = c[n] * rcp[n + 1];
    p[n] = c[n] * df_of((double)n);
  }
  for (int k = 0; k < TAB_NTAY; ++k) {
    Dual2<DF> h[6];
    taylor_coeff_scaled(c, e, p, rcp, k, h);
    for (int j = 0; j < 6; ++j) g[j][k] = h[j];
  }
  DF m[TAB_NC][TAB_NTAY];
  for (int k = 0; k < TAB_NC; ++k)
    for (int n = 0; n < TAB_NTAY; ++n) m[k][n] = df_of(E.m[k][n]);
  for (int j = 0; j < 6; ++j)
    for (int k = 0; k < TAB_NC; ++k) {
      const Dual2<DF> r = econ_apply_scaled(m, k, g[j]);
      const double sc = pow(T, -(double)(k + table_q(j)));
      v[j][k] = df_val(r.v) * sc;
      da[j][k] = df_val(r.da) * sc;
      db[j][k] = df_val(r.db) * sc;
    }
}

// Economised table coefficients e[j][k], k < TAB_NC, on [0, T] (FP64).
template <class T>
GPSS_HD void table_coeffs(const EconMap &E, T a, T beta, T (&e)[6][TAB_NC]) {
  T g[6][TAB_NTAY];
  taylor_coeffs<T>(a, beta, g);
  const double rng = table_range(rate2<double>(val(a), val(beta)));
  for (int j = 0; j < 6; ++j)
    for (int k = 0; k < TAB_NC; ++k) e[j][k] = econ_apply<T>(E, k, rng, g[j], 1);
}

// Six Taylor-branch scalars from a table in shared memory (broadcast reads).
GPSS_HD Disc<float> disc_tab(float t, const float4 *__restrict__ tab) {
  float acc[6];
  {
    const float4 q0 = tab[(TAB_NC - 1) * (TAB_W / 4)], q1 = tab[(TAB_NC - 1) * (TAB_W / 4) + 1];
    acc[0] = q0.x; acc[1] = q0.y; acc[2] = q0.z; acc[3] = q0.w; acc[4] = q1.x; acc[5] = q1.y;
  }
GPSS_HORNER_UNROLL
  for (int k = TAB_NC - 2; k >= 0; --k) {
    const float4 q0 = tab[k * (TAB_W / 4)], q1 = tab[k * (TAB_W / 4) + 1];
    acc[0] = fmaf(acc[0], t, q0.x);
    acc[1] = fmaf(acc[1], t, q0.y);
    acc[2] = fmaf(acc[2], t, q0.z);
    acc[3] = fmaf(acc[3], t, q0.w);
    acc[4] = fmaf(acc[4], t, q1.x);
    acc[5] = fmaf(acc[5], t, q1.y);
  }
  const float t2 = t * t, t3 = t2 * t;
  Disc<float> d;
  d.f = acc[0] * t;
  d.fp = acc[1];
  d.F1 = acc[2] * t2;
  d.Iff = acc[3] * t3;
  d.Ipp = acc[4] * t;
  d.IFF = acc[5] * (t3 * t2);
  return d;
}

GPSS_HD Disc<Dual2<float>> disc_tab_dual(float t, const float4 *__restrict__ tab) {
  float v[6], da[6], db[6];
  {
    const float4 *r = tab + (TAB_NC - 1) * (TAB_W / 4);
    const float4 q0 = r[0], q1 = r[1], q2 = r[2], q3 = r[3], q4 = r[4];
    v[0] = q0.x; v[1] = q0.y; v[2] = q0.z; v[3] = q0.w; v[4] = q1.x; v[5] = q1.y;
    da[0] = q2.x; da[1] = q2.y; da[2] = q2.z; da[3] = q2.w; da[4] = q3.x; da[5] = q3.y;
    db[0] = q3.z; db[1] = q3.w; db[2] = q4.x; db[3] = q4.y; db[4] = q4.z; db[5] = q4.w;
  }
GPSS_HORNER_UNROLL
  for (int k = TAB_NC - 2; k >= 0; --k) {
    const float4 *r = tab + k * (TAB_W / 4);
    const float4 q0 = r[0], q1 = r[1], q2 = r[2], q3 = r[3], q4 = r[4];
    v[0] = fmaf(v[0], t, q0.x); v[1] = fmaf(v[1], t, q0.y); v[2] = fmaf(v[2], t, q0.z);
    v[3] = fmaf(v[3], t, q0.w); v[4] = fmaf(v[4], t, q1.x); v[5] = fmaf(v[5], t, q1.y);
    da[0] = fmaf(da[0], t, q2.x); da[1] = fmaf(da[1], t, q2.y); da[2] = fmaf(da[2], t, q2.z);
    da[3] = fmaf(da[3], t, q2.w); da[4] = fmaf(da[4], t, q3.x); da[5] = fmaf(da[5], t, q3.y);
    db[0] = fmaf(db[0], t, q3.z); db[1] = fmaf(db[1], t, q3.w); db[2] = fmaf(db[2], t, q4.x);
    db[3] = fmaf(db[3], t, q4.y); db[4] = fmaf(db[4], t, q4.z); db[5] = fmaf(db[5], t, q4.w);
  }
  const float t2 = t * t, t3 = t2 * t;
  const float sc[6] = {t, 1.f, t2, t3, t, t3 * t2};
  Disc<Dual2<float>> d;
  Dual2<float> *o[6] = {&d.f, &d.fp, &d.F1, &d.Iff, &d.Ipp, &d.IFF};
#pragma unroll
  for (int i = 0; i < 6; ++i) *o[i] = mk(v[i] * sc[i], da[i] * sc[i], db[i] * sc[i]);
  return d;
}

// Overdamped step above the table's range (beta < 0), FP32 values or (a,
// beta) duals (T = Dual2<float>: the forward-mode arithmetic differentiates
// the same steps), as disc_overdamped with the Taylor branch read from the
// table.  The dual version is kept out of line (it serves only the
// gradient's tangents; inlined, its registers would spill in the reverse walk).
GPSS_HD void tab_eval(float h, const float4 *tab, Disc<float> &d) { d = disc_tab(h, tab); }
GPSS_HD void tab_eval(float h, const float4 *tab, Disc<Dual2<float>> &d) { d = disc_tab_dual(h, tab); }

template <class T>
GPSS_HD Disc<T> disc_od_tab_t(float t, const TermC<float> &c, T a, T beta, T b, T w2,
                              const float4 *tab) {
  const float xt2 = TaylorOrder<float>::XT2;
  const float l1t = c.w2 * t / sqrtf(c.r2);
  if (l1t * l1t < xt2) {
    float h;
    const int k = halvings<float>(t, c.r2, xt2, h);
    Disc<T> d;
    tab_eval(h, tab, d);
    for (int i = 0; i < k; ++i) {
      disc_double_integrals<T, float>(d, a, w2);
      h *= 2.f;
      od_f_fp<T, float>(h, a, beta, b, w2, d.f, d.fp);
    }
    return d;
  }
  T f, fp;
  od_f_fp<T, float>(t, a, beta, b, w2, f, fp);
  return disc_from_ffp<T, float>(t, a, w2, f, fp);
}

GPSS_HDNI Disc<Dual2<float>> disc_od_tab_dual(float t, const TermC<float> &c, const float4 *tab) {
  // b = sqrt(-beta): db/dbeta = -1/(2b); w2 = beta + a^2
  return disc_od_tab_t<Dual2<float>>(t, c, mk(c.a, 1.f, 0.f), mk(c.beta, 0.f, 1.f),
                                     mk(c.b, 0.f, -0.5f * c.rb), mk(c.w2, 2.f * c.a, 1.f), tab);
}

// Discretisation with the Taylor branch read from a table.  OD = false
// drops the overdamped branches (rows without a Q < 1/2 term).
template <bool OD = true>
GPSS_HD Disc<float> discretize_tab(float t, const TermC<float> &c, const float4 *tab) {
  if (t == 0.f) {
    Disc<float> d;
    d.f = 0.f;
    d.fp = 1.f;
    d.F1 = d.Iff = d.Ipp = d.IFF = 0.f;
    return d;
  }
  if constexpr (!OD) {
    if (c.w2 * t * t <= TaylorOrder<float>::XT2) return disc_tab(t, tab);
    float S, C;
    sinc_pair_k(t, c.b, c.rb, S, C);
    return disc_closed_k<float, float>(t, c.a, c.w2, c.rw2, c.r4a, S, C);
  }
  constexpr float xt2 = TaylorOrder<float>::XT2;
  float h = t;
  int k = 0;
  bool in_tab = c.r2 * t * t <= xt2;
  if (!in_tab && c.beta < 0.f) {
    // overdamped with the slow mode not yet decayed: halve into the table's
    // range, double the integrals back (f, f' direct at every level)
    const float l1t = c.w2 * t * rsqrtf(c.r2);
    if (l1t * l1t < xt2) {
      k = halvings<float>(t, c.r2, xt2, h);
      in_tab = true;
    }
  }
  if (in_tab) {
    Disc<float> d = disc_tab(h, tab);
    for (int i = 0; i < k; ++i) {
      disc_double_integrals<float, float>(d, c.a, c.w2);
      h *= 2.f;
      od_f_fp<float, float>(h, c.a, c.beta, c.b, c.w2, d.f, d.fp);
    }
    return d;
  }
  float f, fp;
  if (c.beta < 0.f) {
    od_f_fp<float, float>(t, c.a, c.beta, c.b, c.w2, f, fp);
  } else {
    float S, C;
    sinc_pair_k(t, c.b, c.rb, S, C);
    const float E = gexp(-c.a * t);
    f = E * S;
    fp = E * (C - c.a * S);
  }
  return disc_closed_ffp<float, float>(t, c.a, c.w2, c.rw2, c.r4a, f, fp);
}

// Same with forward-mode derivatives in (a, beta).
template <bool OD = true>
GPSS_HD Disc<Dual2<float>> discretize_tab_dual(float t, const TermC<float> &c, const float4 *tab) {
  if (t == 0.f) {
    Disc<Dual2<float>> d;
    d.f = mk(0.f, 0.f, 0.f);
    d.fp = mk(1.f, 0.f, 0.f);
    d.F1 = d.Iff = d.Ipp = d.IFF = d.f;
    return d;
  }
  if constexpr (!OD) {
    if (c.w2 * t * t <= TaylorOrder<float>::XT2) return disc_tab_dual(t, tab);
  } else {
    if (c.r2 * t * t <= TaylorOrder<float>::XT2) return disc_tab_dual(t, tab);
    if (c.beta < 0.f) return disc_od_tab_dual(t, c, tab);
  }
  float s, co;
  sinc_pair_k(t, c.b, c.rb, s, co);
  // dS/dbeta = (t C - S) / (2 beta) (series for small beta t^2); dC/dbeta = -t S / 2
  const float x = c.beta * t * t;
  float dS;
  if (x < 0.5f)
    dS = t * t * t *
         (-1.f / 6.f + x * (1.f / 60.f + x * (-1.f / 1680.f + x * (1.f / 90720.f + x * (-1.f / 7983360.f)))));
  else
    dS = (t * co - s) * (0.5f * c.rb * c.rb);
  const float dC = -0.5f * t * s;
  // w2 = beta + a^2 ; rw2 = 1/w2 ; r4a = 1/(4a)
  const Dual2<float> a = mk(c.a, 1.f, 0.f);
  const Dual2<float> w2 = mk(c.w2, 2.f * c.a, 1.f);
  const Dual2<float> rw2 = mk(c.rw2, -2.f * c.a * c.rw2 * c.rw2, -c.rw2 * c.rw2);
  const Dual2<float> r4a = mk(c.r4a, -4.f * c.r4a * c.r4a, 0.f);
  return disc_closed_k<Dual2<float>, float>(t, a, w2, rw2, r4a, mk(s, 0.f, dS), mk(co, 0.f, dC));
}


// (a, beta) tangents of the six scalars given their values d (FP32).
// Order of da, db: f, f', F1, I_ff, I_pp, I_FF.
//
// Table branch: Horner on the tangent columns of the table.
GPSS_HD void disc_tab_tangents(float t, const float4 *__restrict__ tab, float (&da)[6],
                               float (&db)[6]) {
  {
    const float4 *r = tab + (TAB_NC - 1) * (TAB_W / 4);
    const float4 q2 = r[2], q3 = r[3], q4 = r[4];
    da[0] = q2.x; da[1] = q2.y; da[2] = q2.z; da[3] = q2.w; da[4] = q3.x; da[5] = q3.y;
    db[0] = q3.z; db[1] = q3.w; db[2] = q4.x; db[3] = q4.y; db[4] = q4.z; db[5] = q4.w;
  }
GPSS_HORNER_UNROLL
  for (int k = TAB_NC - 2; k >= 0; --k) {
    const float4 *r = tab + k * (TAB_W / 4);
    const float4 q2 = r[2], q3 = r[3], q4 = r[4];
    da[0] = fmaf(da[0], t, q2.x); da[1] = fmaf(da[1], t, q2.y); da[2] = fmaf(da[2], t, q2.z);
    da[3] = fmaf(da[3], t, q2.w); da[4] = fmaf(da[4], t, q3.x); da[5] = fmaf(da[5], t, q3.y);
    db[0] = fmaf(db[0], t, q3.z); db[1] = fmaf(db[1], t, q3.w); db[2] = fmaf(db[2], t, q4.x);
    db[3] = fmaf(db[3], t, q4.y); db[4] = fmaf(db[4], t, q4.z); db[5] = fmaf(db[5], t, q4.w);
  }
  const float t2 = t * t, t3 = t2 * t;
  const float sc[6] = {t, 1.f, t2, t3, t, t3 * t2};
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    da[i] *= sc[i];
    db[i] *= sc[i];
  }
}

// Closed-form branch: the derivatives of the closed forms written through
// the values themselves.  With E = exp(-a t), S = sin(b t)/b, C = cos(b t):
// E S = f and E C = f' + a f, so df/da = -t f, df'/da = -t f' - f,
// G := df/dbeta = E dS/dbeta = (t (f' + a f) - f) / (2 beta) (series in
// beta t^2 below 1/2, where that difference cancels), df'/dbeta = -t f/2 - a G,
// and F1, I_pp, I_ff, I_FF follow by differentiating their identities
// (w2 = beta + a^2, dw2/da = 2a, dw2/dbeta = 1).
GPSS_HD void disc_closed_tangents(float t, const TermC<float> &c, const Disc<float> &d,
                                  float (&da)[6], float (&db)[6]) {
  const float a = c.a, w2 = c.w2, rw2 = c.rw2, r4a = c.r4a;
  const float f = d.f, fp = d.fp, F1 = d.F1, Iff = d.Iff, Ipp = d.Ipp, IFF = d.IFF;
  const float tf = t * f, ff = f * f;
  // d/da
  const float fa = -tf;
  const float fpa = -t * fp - f;
  const float F1a = (t * (fp + 2.f * a * f) - f - 2.f * a * F1) * rw2;
  const float Ippa = r4a * (2.f * fp * (t * fp + f) - 2.f * a * ff + 2.f * w2 * t * ff) - 4.f * r4a * Ipp;
  const float Iffa = (Ippa + 2.f * tf * fp + 2.f * a * t * ff - 2.f * a * Iff) * rw2;
  const float IFFa = (Ippa + 8.f * a * Iff + 4.f * a * a * Iffa + 2.f * tf - 4.f * F1 - 4.f * a * F1a +
                      2.f * ff - 4.f * a * t * ff) * (rw2 * rw2) - 4.f * a * IFF * rw2;
  // d/dbeta
  const float x = c.beta * t * t;
  float G;
  if (x < 0.5f)
    G = gexp(-a * t) * t * t * t *
        (-1.f / 6.f + x * (1.f / 60.f + x * (-1.f / 1680.f + x * (1.f / 90720.f + x * (-1.f / 7983360.f)))));
  else
    G = (t * (fp + a * f) - f) * (0.5f * c.rb * c.rb);
  const float fpb = -0.5f * tf - a * G;
  const float F1b = (0.5f * tf - a * G - F1) * rw2;
  const float Ippb = r4a * (-2.f * fp * fpb - ff - 2.f * w2 * f * G);
  const float Iffb = (Ippb - G * fp - f * fpb - 2.f * a * f * G - Iff) * rw2;
  const float IFFb = (Ippb + 4.f * a * a * Iffb - 2.f * G - 4.f * a * F1b + 4.f * a * f * G) *
                         (rw2 * rw2) - 2.f * IFF * rw2;
  da[0] = fa; da[1] = fpa; da[2] = F1a; da[3] = Iffa; da[4] = Ippa; da[5] = IFFa;
  db[0] = G; db[1] = fpb; db[2] = F1b; db[3] = Iffb; db[4] = Ippb; db[5] = IFFb;
}

// Tangents for a step of length t, either branch (same branch rule as
// discretize_tab).
template <bool OD = true>
GPSS_HD void disc_tangents(float t, const TermC<float> &c, const float4 *tab, const Disc<float> &d,
                           float (&da)[6], float (&db)[6]) {
  if (t == 0.f) {
#pragma unroll
    for (int i = 0; i < 6; ++i) da[i] = db[i] = 0.f;
    return;
  }
  if constexpr (!OD) {
    if (c.w2 * t * t <= TaylorOrder<float>::XT2)
      disc_tab_tangents(t, tab, da, db);
    else
      disc_closed_tangents(t, c, d, da, db);
    return;
  }
  if (c.r2 * t * t <= TaylorOrder<float>::XT2) {
    disc_tab_tangents(t, tab, da, db);
  } else if (c.beta < 0.f) {
    const Disc<Dual2<float>> e = disc_od_tab_dual(t, c, tab);
    const Dual2<float> v[6] = {e.f, e.fp, e.F1, e.Iff, e.Ipp, e.IFF};
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      da[i] = v[i].da;
      db[i] = v[i].db;
    }
  } else {
    disc_closed_tangents(t, c, d, da, db);
  }
}

// Blocks of Phi~ and Q~ for one term (see header comment).
template <class F>
struct Blocks {
  F p00, p01, p10, p11, pb0, pb1, q00, q01, q11, qz0, qz1, qzz;
};

template <class F>
GPSS_HD Blocks<F> make_blocks(const Disc<F> &d, const TermC<F> &c) {
  Blocks<F> B;
  B.p00 = d.fp + F(2) * c.a * d.f;
  B.p01 = d.f;
  B.p10 = -c.w2 * d.f;
  B.p11 = d.fp;
  B.pb0 = d.f + F(2) * c.a * d.F1;
  B.pb1 = d.F1;
  B.q00 = c.qc * d.Iff;
  B.q01 = c.qc * d.f * d.f * F(0.5);
  B.q11 = c.qc * d.Ipp;
  B.qz0 = c.qc * d.F1 * d.F1 * F(0.5);
  B.qz1 = c.qc * (d.f * d.F1 - d.Iff);
  B.qzz = c.qc * d.IFF;
  return B;
}

// out = Phi~ v
template <class S, class F>
GPSS_HD void apply_phi(const Blocks<F> *B, const F *v, F *out) {
#pragma unroll
  for (int t = 0; t < S::NT; ++t) {
    out[2 * t] = B[t].p00 * v[2 * t] + B[t].p01 * v[2 * t + 1];
    out[2 * t + 1] = B[t].p10 * v[2 * t] + B[t].p11 * v[2 * t + 1];
  }
#pragma unroll
  for (int zi = 2 * S::NT; zi < S::D; ++zi) {
    F acc = v[zi];
#pragma unroll
    for (int t = 0; t < S::NT; ++t)
      if (S::zint(zi, t)) acc = acc + B[t].pb0 * v[2 * t] + B[t].pb1 * v[2 * t + 1];
    out[zi] = acc;
  }
}

// out = Phi~^T v
template <class S, class F>
GPSS_HD void apply_phi_t(const Blocks<F> *B, const F *v, F *out) {
#pragma unroll
  for (int t = 0; t < S::NT; ++t) {
    F a0 = B[t].p00 * v[2 * t] + B[t].p10 * v[2 * t + 1];
    F a1 = B[t].p01 * v[2 * t] + B[t].p11 * v[2 * t + 1];
#pragma unroll
    for (int zi = 2 * S::NT; zi < S::D; ++zi)
      if (S::zint(zi, t)) {
        a0 = a0 + B[t].pb0 * v[zi];
        a1 = a1 + B[t].pb1 * v[zi];
      }
    out[2 * t] = a0;
    out[2 * t + 1] = a1;
  }
#pragma unroll
  for (int zi = 2 * S::NT; zi < S::D; ++zi) out[zi] = v[zi];
}

// P <- P + Q~ (packed)
template <class S, class F>
GPSS_HD void add_q(const Blocks<F> *B, F *P) {
#pragma unroll
  for (int t = 0; t < S::NT; ++t) {
    P[S::pk(2 * t, 2 * t)] += B[t].q00;
    P[S::pk(2 * t, 2 * t + 1)] += B[t].q01;
    P[S::pk(2 * t + 1, 2 * t + 1)] += B[t].q11;
#pragma unroll
    for (int zi = 2 * S::NT; zi < S::D; ++zi)
      if (S::zint(zi, t)) {
        P[S::pk(2 * t, zi)] += B[t].qz0;
        P[S::pk(2 * t + 1, zi)] += B[t].qz1;
      }
  }
#pragma unroll
  for (int zi = 2 * S::NT; zi < S::D; ++zi)
#pragma unroll
    for (int zj = zi; zj < S::D; ++zj) {
      F acc = F(0);
#pragma unroll
      for (int t = 0; t < S::NT; ++t)
        if (S::zint(zi, t) && S::zint(zj, t)) acc += B[t].qzz;
      P[S::pk(zi, zj)] += acc;
    }
}

// P <- Phi~ P Phi~^T + Q~ on packed storage, in place, one term at a time.
// Phi~ is the product of commuting factors Phi_t, each the identity except
// on term t's pair a = (2t, 2t+1), which it maps by its 2x2 block, and on the
// integral states z of that term, which gain pb0 x_a0 + pb1 x_a1.  The
// congruence P <- Phi_t P Phi_t^T changes only the rows and columns of a and
// of the z: with W = P Phi_t^T (columns j in a and z),
//   W[k][a_r] = A[r][0] P[k][a0] + A[r][1] P[k][a1],
//   W[k][z]   = P[k][z] + pb0 P[k][a0] + pb1 P[k][a1],
// the new entries are W[k][j] for k outside a and z, and, for i, j in a and
// z, Phi_t[i,:] W[:, j] (a row of Phi_t has two or three nonzeros).
template <class S, class F>
GPSS_HD void predict_cov(const Blocks<F> *B, F *P) {
  constexpr int D = S::D;
#pragma unroll
  for (int t = 0; t < S::NT; ++t) {
    const int a0 = 2 * t, a1 = 2 * t + 1;
    const F p00 = B[t].p00, p01 = B[t].p01, p10 = B[t].p10, p11 = B[t].p11;
    const F pb0 = B[t].pb0, pb1 = B[t].pb1;
    // W = P Phi_t^T at the changed columns, every row
    F W[D][D];  // only columns a0, a1 and term t's z are formed
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const F x0 = P[S::pk(k, a0)], x1 = P[S::pk(k, a1)];
      W[k][a0] = p00 * x0 + p01 * x1;
      W[k][a1] = p10 * x0 + p11 * x1;
#pragma unroll
      for (int z = 2 * S::NT; z < D; ++z)
        if (S::zint(z, t)) W[k][z] = P[S::pk(k, z)] + pb0 * x0 + pb1 * x1;
    }
    // rows outside the changed set keep W; the changed block is Phi_t W
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const bool kc = (k == a0 || k == a1 || (k >= 2 * S::NT && S::zint(k, t)));
      if (kc) continue;
      P[S::pk(k, a0)] = W[k][a0];
      P[S::pk(k, a1)] = W[k][a1];
#pragma unroll
      for (int z = 2 * S::NT; z < D; ++z)
        if (S::zint(z, t)) P[S::pk(k, z)] = W[k][z];
    }
    auto row = [&](int i, int j) -> F {  // (Phi_t W)[i][j], i and j changed
      if (i == a0) return p00 * W[a0][j] + p01 * W[a1][j];
      if (i == a1) return p10 * W[a0][j] + p11 * W[a1][j];
      return W[i][j] + pb0 * W[a0][j] + pb1 * W[a1][j];
    };
    P[S::pk(a0, a0)] = row(a0, a0);
    P[S::pk(a0, a1)] = row(a0, a1);
    P[S::pk(a1, a1)] = row(a1, a1);
#pragma unroll
    for (int z = 2 * S::NT; z < D; ++z) {
      if (!S::zint(z, t)) continue;
      P[S::pk(a0, z)] = row(a0, z);
      P[S::pk(a1, z)] = row(a1, z);
#pragma unroll
      for (int z2 = 2 * S::NT; z2 <= z; ++z2)
        if (S::zint(z2, t)) P[S::pk(z2, z)] = row(z2, z);
    }
  }
  add_q<S>(B, P);
}

// Reset of slot j (Eq. integrated_kalman_update with R_j of Section 3.2.3).
template <class S, class F>
GPSS_HD void reset_slot(int j, F *m, F *P) {
#pragma unroll
  for (int zi = 2 * S::NT; zi < S::D; ++zi) {
    const bool hit = (S::zslot(zi) == j);
    m[zi] = hit ? F(0) : m[zi];
#pragma unroll
    for (int i = 0; i < S::D; ++i) P[S::pk(i, zi)] = hit ? F(0) : P[S::pk(i, zi)];
  }
}

// An instantaneous measurement (Section 2) observes the latent with h = H =
// (1 0 1 0 ... 0): u = P h, hu = h.u, hm = h.m.
template <class S, class F>
GPSS_HD void obs_latent(const F *m, const F *P, F *u, F &hu, F &hm) {
#pragma unroll
  for (int i = 0; i < S::D; ++i) {
    F acc = F(0);
#pragma unroll
    for (int t = 0; t < S::NT; ++t) acc += P[S::pk(i, 2 * t)];
    u[i] = acc;
  }
  F a1 = F(0), a2 = F(0);
#pragma unroll
  for (int t = 0; t < S::NT; ++t) {
    a1 += u[2 * t];
    a2 += m[2 * t];
  }
  hu = a1;
  hm = a2;
}

// Tag bit of an instantaneous measurement in a model whose shape has
// integral states (exposure averages and instants in one model): the event
// observes the latent instead of a slot's integral state.
constexpr uint8_t TAG_INSTANT = 0x10;

// Shared pieces of the measurement update with H~ = w * sum_{z in slot j} e_z
// (Eq. H_aug; w = 1/delta):  u = P H~^T, S = H~ u + r, hm = H~ m.  Shapes
// without integral states (NS = 0) observe the latent instead.
template <class S, class F>
GPSS_HD void obs_project(int j, F w, const F *m, const F *P, F *u, F &hu, F &hm) {
  if constexpr (S::NS == 0) {
    // no integral states: every measurement is instantaneous (w unused)
    obs_latent<S>(m, P, u, hu, hm);
    return;
  }
#pragma unroll
  for (int i = 0; i < S::D; ++i) {
    F acc = F(0);
#pragma unroll
    for (int zi = 2 * S::NT; zi < S::D; ++zi) acc += (S::zslot(zi) == j) ? P[S::pk(i, zi)] : F(0);
    u[i] = acc * w;
  }
  F a1 = F(0), a2 = F(0);
#pragma unroll
  for (int zi = 2 * S::NT; zi < S::D; ++zi) {
    const bool hit = (S::zslot(zi) == j);
    a1 += hit ? u[zi] : F(0);
    a2 += hit ? m[zi] : F(0);
  }
  hu = a1 * w;
  hm = a2 * w;
}

// The update's projections for a measurement event given its tag: with MIX
// (a model mixing instants with exposure averages), an event tagged
// TAG_INSTANT observes the latent; otherwise slot (tag >> 1) & 7.
template <class S, class F, bool MIX>
GPSS_HD void obs_project_tag(uint8_t tag, F w, const F *m, const F *P, F *u, F &hu, F &hm) {
  if constexpr (MIX && S::NS > 0) {
    if (tag & TAG_INSTANT) {
      obs_latent<S>(m, P, u, hu, hm);
      return;
    }
  }
  obs_project<S>((tag >> 1) & 7, w, m, P, u, hu, hm);
}

// Load per-term constants and s^2 from a row of natural parameters.
template <int NT, class F>
GPSS_HD void load_terms(const float *th, const int *kinds, TermC<F> *tc, F &s2) {
  int j = 0;
#pragma unroll
  for (int t = 0; t < NT; ++t) {
    F sig, w0, q;
    if (kinds[t] == 1) {
      sig = F(th[j]);
      w0 = F(th[j + 1]);
      q = F(th[j + 2]);
      j += 3;
    } else {
      sig = F(th[j]);
      w0 = F(1.7320508075688772) / F(th[j + 1]);
      q = F(0.5);
      j += 2;
    }
    tc[t].var = sig * sig;
    tc[t].a = w0 / (F(2) * q);
    tc[t].w2 = w0 * w0;
    tc[t].beta = (q == F(0.5)) ? F(0) : w0 * w0 * (F(1) - F(1) / (F(4) * q * q));
    tc[t].qc = F(2) * w0 * w0 * w0 * sig * sig / q;
    finish_termc(tc[t]);
  }
  F s = F(th[j]);
  s2 = s * s;
}

// True when some term of the row is an overdamped oscillator (beta < 0);
// rows without one run the kernels' specialisation without those branches.
template <int NT, class F>
GPSS_HD bool any_overdamped(const TermC<F> *tc) {
  bool od = false;
#pragma unroll
  for (int t = 0; t < NT; ++t) od |= tc[t].beta < F(0);
  return od;
}

// P0 = blkdiag(P_inf, I) (Section 3.2.3); m0 = 0.
template <class S, class F>
GPSS_HD void init_state(const TermC<F> *tc, F *m, F *P) {
#pragma unroll
  for (int i = 0; i < S::D; ++i) m[i] = F(0);
#pragma unroll
  for (int i = 0; i < S::NP; ++i) P[i] = F(0);
#pragma unroll
  for (int t = 0; t < S::NT; ++t) {
    P[S::pk(2 * t, 2 * t)] = tc[t].var;
    P[S::pk(2 * t + 1, 2 * t + 1)] = tc[t].var * tc[t].w2;
  }
#pragma unroll
  for (int zi = 2 * S::NT; zi < S::D; ++zi) P[S::pk(zi, zi)] = F(1);
}

// Dense solve with partial pivoting: B <- A^{-1} B (A destroyed); returns
// log|det A|.  Row swaps are done with selects so that every index stays a
// compile-time constant (register arrays).
template <int D, int R, class F>
GPSS_HD F solve_inplace(F (&A)[D][D], F (&B)[D][R]) {
  F logdet = F(0);
#pragma unroll
  for (int k = 0; k < D; ++k) {
    // pivot row among k..D-1
    int piv = k;
    F best = fabs(A[k][k]);
#pragma unroll
    for (int r = k + 1; r < D; ++r) {
      F v = fabs(A[r][k]);
      if (v > best) {
        best = v;
        piv = r;
      }
    }
#pragma unroll
    for (int r = k + 1; r < D; ++r) {
      const bool sw = (piv == r);
#pragma unroll
      for (int c = 0; c < D; ++c) {
        F x = A[k][c], y = A[r][c];
        A[k][c] = sw ? y : x;
        A[r][c] = sw ? x : y;
      }
#pragma unroll
      for (int c = 0; c < R; ++c) {
        F x = B[k][c], y = B[r][c];
        B[k][c] = sw ? y : x;
        B[r][c] = sw ? x : y;
      }
    }
    const F pivv = A[k][k];
    logdet += log(fabs(pivv));
    const F ip = F(1) / pivv;
    // scale the pivot row of [A | B], then eliminate column k from every other row
#pragma unroll
    for (int c = k + 1; c < D; ++c) A[k][c] *= ip;
#pragma unroll
    for (int c = 0; c < R; ++c) B[k][c] *= ip;
#pragma unroll
    for (int r = 0; r < D; ++r) {
      if (r == k) continue;
      const F fct = A[r][k];
#pragma unroll
      for (int c = k + 1; c < D; ++c) A[r][c] -= fct * A[k][c];
#pragma unroll
      for (int c = 0; c < R; ++c) B[r][c] -= fct * B[k][c];
    }
  }
  return logdet;
}

}  // namespace gpss
