/*
 * gpss_oracle.c -- plain FP64 reference for the log-likelihood of a Gaussian
 * process observed through integrated, possibly overlapping exposures, computed
 * by the sequential Kalman filter over the augmented state-space model of
 * Section 3 of the paper (arXiv 2601.02527).
 *
 * TEST INFRASTRUCTURE.  Only the test-suite, the smoke check and the CPU
 * baseline of the benchmark load this library.  It shares no code with the
 * CUDA path, and the CUDA path never calls it.
 *
 * What it computes, in the paper's order:
 *   - model matrices from natural parameters (Appendix B, C.1; products of
 *     two SHO terms as the Kronecker model of Appendix C.2);
 *   - discretisation by the Van Loan matrix exponential (Eq. Q_from_vanloan)
 *     with exact semigroup doubling for long steps;
 *   - the integrated Kalman filter with resets (Eqs. integrated_kalman_pred,
 *     integrated_kalman_update) and one integral state per slot (Section
 *     3.2.3), and the prediction-error log-likelihood (Eq. loglikelihood);
 *   - gradients by the complex-step method: the filter is compiled a second
 *     time over double complex, theta_i is perturbed by i*h, and
 *     d loglik / d theta_i = Im(loglik) / h, exact up to rounding.
 *   - the integrated RTS smoother (Eqs. rts, integrated_rts) and prediction
 *     at arbitrary times (Algorithm 1).
 * Events arrive already sorted and labelled (start / end / instantaneous
 * measurement, slot) by the Python side of the oracle.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define MAXT 4
#define TWO_PI 6.283185307179586476925286766559
#define MAXD 12

typedef struct {
  int n_terms;
  int kind[MAXT]; /* 1 = SHO, 2 = Matern-3/2, 3 = product of two SHOs */
  int toff[MAXT]; /* first state index of each term */
  int tdim[MAXT]; /* its state dimension: 2, or 4 for a product */
  int nx;         /* latent (non-integral) state dimension, sum of tdim */
  int layout;     /* 0: one z per slot; 1: one z per term per slot */
  int n_slots;
  int dim;    /* augmented state dimension */
  int n_zper; /* integral states per slot */
  int closed; /* 1: the filter's timing mode (Appendix B closed forms where they apply) */
} model_t;

static int zindex(const model_t *M, int slot, int t) {
  if (M->layout == 0) return M->nx + slot;
  return M->nx + slot * M->n_terms + t;
}

/* Observation vector of a measurement event (Eq. H_aug): an exposure end
 * (kind 1) reads its slot's integral state(s) times 1/delta; an
 * instantaneous measurement (kind 2, Section 2: t_start = t_end) reads the
 * latent f = H x = sum_t x_t directly. */
static void obs_vector(const model_t *M, int kind, int slot, double invd, double *h) {
  for (int i = 0; i < M->dim; ++i) h[i] = 0.0;
  if (kind == 2) {
    for (int t = 0; t < M->n_terms; ++t) h[M->toff[t]] = 1.0;
  } else {
    for (int t = 0; t < M->n_zper; ++t) h[zindex(M, slot, t)] = invd;
  }
}

/* spec: n_terms, layout (bit 8: closed-form timing mode), n_slots, kinds. */
static int parse_spec(const int32_t *spec, model_t *M) {
  M->n_terms = spec[0];
  M->layout = spec[1] & 0xff;
  M->closed = (spec[1] >> 8) & 1;
  if (spec[1] & ~0x1ff) return 1;
  M->n_slots = spec[2];
  if (M->n_terms < 1 || M->n_terms > MAXT || M->n_slots < 0) return 1;
  if (M->layout != 0 && M->layout != 1) return 1;
  M->nx = 0;
  for (int t = 0; t < M->n_terms; ++t) {
    M->kind[t] = spec[3 + t];
    if (M->kind[t] < 1 || M->kind[t] > 3) return 1;
    M->toff[t] = M->nx;
    M->tdim[t] = M->kind[t] == 3 ? 4 : 2;
    M->nx += M->tdim[t];
  }
  M->n_zper = M->layout == 0 ? 1 : M->n_terms;
  M->dim = M->nx + M->n_slots * M->n_zper;
  if (M->dim > MAXD) return 1;
  return 0;
}

static int n_params(const model_t *M) {
  int n = 1;
  for (int t = 0; t < M->n_terms; ++t) n += (M->kind[t] == 1) ? 3 : (M->kind[t] == 2 ? 2 : 5);
  return n;
}

/* ---- real instantiation ---- */
#define SCALAR double
#define SFX(name) name##_r
#define S_SQRT sqrt
#define S_LOG log
#define S_ABS fabs
#define S_RE(x) (x)
#define S_EXP exp
#define S_SIN sin
#define S_COS cos
#include "oracle_body.h"
#undef SCALAR
#undef SFX
#undef S_SQRT
#undef S_LOG
#undef S_ABS
#undef S_RE
#undef S_EXP
#undef S_SIN
#undef S_COS

/* ---- complex instantiation (complex-step derivatives) ---- */
#define SCALAR double complex
#define SFX(name) name##_c
#define S_SQRT csqrt
#define S_LOG clog
#define S_ABS cabs
#define S_RE(x) creal(x)
#define S_EXP cexp
#define S_SIN csin
#define S_COS ccos
#include "oracle_body.h"
#undef SCALAR
#undef SFX
#undef S_SQRT
#undef S_LOG
#undef S_ABS
#undef S_RE
#undef S_EXP
#undef S_SIN
#undef S_COS

int gpss_oracle_dim(const int32_t *spec) {
  model_t M;
  if (parse_spec(spec, &M)) return -1;
  return M.dim;
}

/* Phi~, Q~ and P0 (row-major dim x dim) for one step dt of the augmented model
 * (Van Loan, or the closed forms in the timing mode where they apply). */
int gpss_oracle_discretize(const int32_t *spec, const double *theta, double dt, double *Phi,
                           double *Q, double *P0) {
  model_t M;
  if (parse_spec(spec, &M)) return 1;
  double w0[2 * MAXT], q[2 * MAXT], var[MAXT], s2;
  double F[MAXD * MAXD], LQL[MAXD * MAXD];
  term_params_r(&M, theta, w0, q, var, &s2);
  build_F_r(&M, w0, q, var, F, LQL);
  if (!M.closed || discretize_closed_r(&M, w0, q, var, dt, Phi, Q))
    discretize_r(&M, F, LQL, dt, Phi, Q);
  if (P0) initial_cov_r(&M, w0, var, P0);
  return 0;
}

/* Log-likelihood of one series (and, if grad != NULL, its gradient with
 * respect to the natural parameters by the complex-step method).
 * Per event k (time-sorted): t_ev, kind (0 start, 1 end, 2 instantaneous
 * measurement), slot, and for measurement
 * events y, r0 = yerr^2 and 1/delta.  dumpP (n_ev * dim * dim) receives the
 * filtered covariance after each event and dumpS (n_end) the innovation
 * variances; both may be NULL.  Returns 0 on success. */
int gpss_oracle_loglik(const int32_t *spec, int64_t n_ev, const double *t_ev,
                       const int32_t *kind, const int32_t *slot, const double *y_ev,
                       const double *r0_ev, const double *invd_ev, const double *theta,
                       double *loglik, double *grad, double *dumpP, double *dumpS) {
  model_t M;
  if (parse_spec(spec, &M)) return 1;
  double ll;
  int rc = filter_r(&M, theta, n_ev, t_ev, kind, slot, y_ev, r0_ev, invd_ev, &ll, dumpP, dumpS);
  if (rc) return rc;
  *loglik = ll;
  if (grad) {
    const int np = n_params(&M);
    double complex thc[16];
    double complex *tc = malloc(sizeof(double complex) * (size_t)(n_ev > 0 ? n_ev : 1));
    double complex *ic = malloc(sizeof(double complex) * (size_t)(n_ev > 0 ? n_ev : 1));
    if (!tc || !ic) {
      free(tc);
      free(ic);
      return 4;
    }
    for (int64_t k = 0; k < n_ev; ++k) {
      tc[k] = t_ev[k];
      ic[k] = invd_ev[k];
    }
    for (int i = 0; i < np && !rc; ++i) {
      for (int j = 0; j < np; ++j) thc[j] = theta[j];
      double hstep = 1e-20 * (fabs(theta[i]) > 1.0 ? fabs(theta[i]) : 1.0);
      thc[i] = theta[i] + I * hstep;
      double complex llc;
      rc = filter_c(&M, thc, n_ev, tc, kind, slot, y_ev, r0_ev, ic, &llc, NULL, NULL);
      if (!rc) grad[i] = cimag(llc) / hstep;
    }
    free(tc);
    free(ic);
  }
  return rc;
}

/* Gradient of one series' log-likelihood with respect to its exposure
 * windows, by the complex-step method on the event times: for measurement
 * n (events ev_start[n], ev_end[n] of the sorted sequence), t_start or t_end
 * is moved by i*h, which moves that event's time (and so the gaps on both
 * sides of it; the event order is kept) and 1/delta of the measurement's end
 * event, 1/(t_end - t_start).  The first event's time is the initial time
 * (the prior is stationary), so it moves with it.  d_ts[n], d_te[n] =
 * Im(loglik) / h.  One complex filter pass per window edge: O(N^2) work, for
 * test-sized series. */
int gpss_oracle_exposure_grad(const int32_t *spec, int64_t n_ev, const double *t_ev,
                              const int32_t *kind, const int32_t *slot, const double *y_ev,
                              const double *r0_ev, const double *invd_ev, const double *theta,
                              int64_t n_meas, const int64_t *ev_start, const int64_t *ev_end,
                              double *d_ts, double *d_te) {
  model_t M;
  if (parse_spec(spec, &M)) return 1;
  const int np = n_params(&M);
  double complex thc[16];
  for (int j = 0; j < np; ++j) thc[j] = theta[j];
  double complex *tc = malloc(sizeof(double complex) * (size_t)(n_ev > 0 ? n_ev : 1));
  double complex *ic = malloc(sizeof(double complex) * (size_t)(n_ev > 0 ? n_ev : 1));
  if (!tc || !ic) {
    free(tc);
    free(ic);
    return 4;
  }
  int rc = 0;
  for (int64_t n = 0; n < n_meas && !rc; ++n) {
    const int64_t ks = ev_start[n], ke = ev_end[n];
    if (ks == ke) {
      /* instantaneous measurement (one event): moving its time moves both
       * "edges"; each column holds half of d loglik / d t */
      for (int64_t k = 0; k < n_ev; ++k) {
        tc[k] = t_ev[k];
        ic[k] = invd_ev[k];
      }
      const double hstep = 1e-20 * (fabs(t_ev[ke]) > 1.0 ? fabs(t_ev[ke]) : 1.0);
      tc[ke] += I * hstep;
      double complex llc;
      rc = filter_c(&M, thc, n_ev, tc, kind, slot, y_ev, r0_ev, ic, &llc, NULL, NULL);
      if (!rc) d_ts[n] = d_te[n] = 0.5 * cimag(llc) / hstep;
      continue;
    }
    const double delta = 1.0 / invd_ev[ke];
    for (int edge = 0; edge < 2 && !rc; ++edge) {
      for (int64_t k = 0; k < n_ev; ++k) {
        tc[k] = t_ev[k];
        ic[k] = invd_ev[k];
      }
      const int64_t ke_or_ks = edge ? ke : ks;
      const double hstep = 1e-20 * (fabs(t_ev[ke_or_ks]) > 1.0 ? fabs(t_ev[ke_or_ks]) : 1.0);
      tc[ke_or_ks] += I * hstep;
      ic[ke] = 1.0 / (delta + (edge ? 1.0 : -1.0) * I * hstep);
      double complex llc;
      rc = filter_c(&M, thc, n_ev, tc, kind, slot, y_ev, r0_ev, ic, &llc, NULL, NULL);
      if (!rc) (edge ? d_te : d_ts)[n] = cimag(llc) / hstep;
    }
  }
  free(tc);
  free(ic);
  return rc;
}

/* ---- integrated RTS smoother (real arithmetic only) ---- */

/* Solve S G^T = X for the smoother gain (S symmetric positive semidefinite,
 * n x n; X n x n; both row-major, overwritten; G^T returned in X).  A reset
 * followed by a zero gap leaves an exactly zero row and column in S (that
 * integral state is known to be zero); those indices are left out and the
 * rest is solved exactly by Gauss-Jordan with partial pivoting, which is the
 * Moore-Penrose solution for this structure.  Returns 0, or 1 if the
 * remaining matrix is singular. */
static int gain_solve(int n, double *S, double *X) {
  int keep[MAXD], nk = 0;
  for (int i = 0; i < n; ++i)
    if (S[i * n + i] > 0.0) keep[nk++] = i;
  double A[MAXD * MAXD], B[MAXD * MAXD];
  for (int r = 0; r < nk; ++r)
    for (int c = 0; c < nk; ++c) A[r * nk + c] = S[keep[r] * n + keep[c]];
  for (int r = 0; r < nk; ++r)
    for (int j = 0; j < n; ++j) B[r * n + j] = X[keep[r] * n + j];
  for (int c = 0; c < nk; ++c) {
    int p = c;
    for (int r = c + 1; r < nk; ++r)
      if (fabs(A[r * nk + c]) > fabs(A[p * nk + c])) p = r;
    if (A[p * nk + c] == 0.0) return 1;
    if (p != c) {
      for (int j = 0; j < nk; ++j) {
        const double t = A[c * nk + j];
        A[c * nk + j] = A[p * nk + j];
        A[p * nk + j] = t;
      }
      for (int j = 0; j < n; ++j) {
        const double t = B[c * n + j];
        B[c * n + j] = B[p * n + j];
        B[p * n + j] = t;
      }
    }
    const double inv = 1.0 / A[c * nk + c];
    for (int j = 0; j < nk; ++j) A[c * nk + j] *= inv;
    for (int j = 0; j < n; ++j) B[c * n + j] *= inv;
    for (int r = 0; r < nk; ++r) {
      if (r == c || A[r * nk + c] == 0.0) continue;
      const double f = A[r * nk + c];
      for (int j = 0; j < nk; ++j) A[r * nk + j] -= f * A[c * nk + j];
      for (int j = 0; j < n; ++j) B[r * n + j] -= f * B[c * n + j];
    }
  }
  for (int i = 0; i < n * n; ++i) X[i] = 0.0;
  for (int r = 0; r < nk; ++r)
    for (int j = 0; j < n; ++j) X[keep[r] * n + j] = B[r * n + j];
  return 0;
}

/* Conditioned mean and variance of every measurement's exposure average
 * given all the series' data: the filter of gpss_oracle_loglik keeping the
 * predicted (m-, P-) and filtered (m, P) state of every event, then the RTS
 * recursion backwards from the last event (smoothed = filtered there):
 *   end state k:   G = P_k A_k^T (P-_{k+1})^-1, smoothed m^_k, P^_k from the
 *                  filtered (m_k, P_k)                        (Eq. rts);
 *   start state k: G = P-_k (A_k R_k)^T (P-_{k+1})^-1, from the pre-reset
 *                  (m-_k, P-_k)                    (Eq. integrated_rts);
 *   m^_k = base + G (m^_{k+1} - m-_{k+1}),
 *   P^_k = base + G (P^_{k+1} - P-_{k+1}) G^T,
 * with A_k the transition from event k to k+1.  At each end event (output
 * in event order) mean = H m^, var = H P^ H^T, H = e_z / delta (the latent
 * sum for an instantaneous measurement).  P-_{k+1}
 * is inverted as in gain_solve.  Returns 0, or 5 if it is singular beyond
 * zeroed integral states. */
static int smooth_all(const model_t *Mp, int64_t n_ev, const double *t_ev, const int32_t *kind,
                      const int32_t *slot, const double *y_ev, const double *r0_ev,
                      const double *invd_ev, const double *theta, double *mp, double *Pp,
                      double *mf, double *Pf, double *msa, double *Psa, double *mean_ev,
                      double *var_ev) {
  const model_t M = *Mp;
  const int D = M.dim, DD = D * D;
  double w0[2 * MAXT], q[2 * MAXT], var[MAXT], s2;
  double F[MAXD * MAXD], LQL[MAXD * MAXD], Phi[MAXD * MAXD], Qd[MAXD * MAXD];
  term_params_r(&M, theta, w0, q, var, &s2);
  build_F_r(&M, w0, q, var, F, LQL);
  int rc = 0;
  /* forward: predicted and filtered states (Joseph-form update as in the filter) */
  double m[MAXD], P[MAXD * MAXD], T[MAXD * MAXD], A[MAXD * MAXD], h[MAXD], u[MAXD], K[MAXD];
  initial_cov_r(&M, w0, var, P);
  for (int i = 0; i < D; ++i) m[i] = 0;
  double tprev = n_ev > 0 ? t_ev[0] : 0.0;
  for (int64_t k = 0; k < n_ev && !rc; ++k) {
    const double dt = t_ev[k] - tprev;
    tprev = t_ev[k];
    if (dt < 0) {
      rc = 2;
      break;
    }
    discretize_r(&M, F, LQL, dt, Phi, Qd);
    double mt[MAXD];
    for (int i = 0; i < D; ++i) {
      double acc = 0;
      for (int j = 0; j < D; ++j) acc += Phi[i * D + j] * m[j];
      mt[i] = acc;
    }
    memcpy(m, mt, sizeof(double) * D);
    matmul_r(D, Phi, P, T);
    for (int i = 0; i < D; ++i)
      for (int j = 0; j <= i; ++j) {
        double acc = 0;
        for (int kk = 0; kk < D; ++kk) acc += T[i * D + kk] * Phi[j * D + kk];
        P[i * D + j] = acc + 0.5 * (Qd[i * D + j] + Qd[j * D + i]);
        P[j * D + i] = P[i * D + j];
      }
    memcpy(mp + k * D, m, sizeof(double) * D);
    memcpy(Pp + k * DD, P, sizeof(double) * DD);
    const int sj = slot[k];
    if (kind[k] == 0) {
      for (int t = 0; t < M.n_zper; ++t) {
        const int z = zindex(&M, sj, t);
        m[z] = 0;
        for (int i = 0; i < D; ++i) P[z * D + i] = P[i * D + z] = 0;
      }
    } else {
      obs_vector(&M, kind[k], sj, invd_ev[k], h);
      const double r = r0_ev[k] + s2;
      double Sv = r, hm = 0;
      for (int i = 0; i < D; ++i) {
        double acc = 0;
        for (int j = 0; j < D; ++j) acc += P[i * D + j] * h[j];
        u[i] = acc;
        Sv += h[i] * acc;
        hm += h[i] * m[i];
      }
      const double v = y_ev[k] - hm;
      for (int i = 0; i < D; ++i) {
        K[i] = u[i] / Sv;
        m[i] += K[i] * v;
      }
      for (int i = 0; i < D; ++i)
        for (int j = 0; j < D; ++j) A[i * D + j] = (i == j ? 1.0 : 0.0) - K[i] * h[j];
      matmul_r(D, A, P, T);
      for (int i = 0; i < D; ++i)
        for (int j = 0; j <= i; ++j) {
          double acc = 0;
          for (int kk = 0; kk < D; ++kk) acc += T[i * D + kk] * A[j * D + kk];
          P[i * D + j] = acc + K[i] * r * K[j];
          P[j * D + i] = P[i * D + j];
        }
    }
    memcpy(mf + k * D, m, sizeof(double) * D);
    memcpy(Pf + k * DD, P, sizeof(double) * DD);
  }
  /* backward: smoothed (m^, P^), starting from the last (end) event */
  double ms[MAXD], Ps[MAXD * MAXD];
  if (!rc && n_ev > 0) {
    memcpy(ms, mf + (n_ev - 1) * D, sizeof(double) * D);
    memcpy(Ps, Pf + (n_ev - 1) * DD, sizeof(double) * DD);
  }
  for (int64_t k = n_ev - 1; k >= 0 && !rc; --k) {
    if (k < n_ev - 1) {
      /* transition from event k to k+1 (with the reset at a start state) */
      discretize_r(&M, F, LQL, t_ev[k + 1] - t_ev[k], Phi, Qd);
      const double *bm, *bP;
      double AR[MAXD * MAXD];
      memcpy(AR, Phi, sizeof(double) * DD);
      if (kind[k] == 0) {
        for (int t = 0; t < M.n_zper; ++t) {
          const int z = zindex(&M, slot[k], t);
          for (int i = 0; i < D; ++i) AR[i * D + z] = 0; /* Phi R: column z zeroed */
        }
        bm = mp + k * D;
        bP = Pp + k * DD;
      } else {
        bm = mf + k * D;
        bP = Pf + k * DD;
      }
      /* G = bP AR^T (P-_{k+1})^-1  <=>  P-_{k+1} G^T = AR bP */
      double S[MAXD * MAXD], X[MAXD * MAXD];
      memcpy(S, Pp + (k + 1) * DD, sizeof(double) * DD);
      matmul_r(D, AR, bP, X);
      if (gain_solve(D, S, X)) {
        rc = 5;
        break;
      }
      double G[MAXD * MAXD], dm[MAXD], dP[MAXD * MAXD], GT[MAXD * MAXD];
      for (int i = 0; i < D; ++i)
        for (int j = 0; j < D; ++j) G[i * D + j] = X[j * D + i];
      for (int i = 0; i < D; ++i) dm[i] = ms[i] - mp[(k + 1) * D + i];
      for (int i = 0; i < DD; ++i) dP[i] = Ps[i] - Pp[(k + 1) * DD + i];
      double nm[MAXD];
      for (int i = 0; i < D; ++i) {
        double acc = bm[i];
        for (int j = 0; j < D; ++j) acc += G[i * D + j] * dm[j];
        nm[i] = acc;
      }
      matmul_r(D, G, dP, T);
      for (int i = 0; i < D; ++i)
        for (int j = 0; j < D; ++j) GT[i * D + j] = G[j * D + i];
      matmul_r(D, T, GT, X);
      for (int i = 0; i < DD; ++i) Ps[i] = bP[i] + X[i];
      for (int i = 0; i < D; ++i)
        for (int j = 0; j < i; ++j) Ps[i * D + j] = Ps[j * D + i] = 0.5 * (Ps[i * D + j] + Ps[j * D + i]);
      memcpy(ms, nm, sizeof(double) * D);
    }
    memcpy(msa + k * D, ms, sizeof(double) * D);
    memcpy(Psa + k * DD, Ps, sizeof(double) * DD);
    if (!mean_ev) continue;
    if (kind[k] != 0) {
      obs_vector(&M, kind[k], slot[k], invd_ev[k], h);
      double mu = 0, va = 0;
      for (int i = 0; i < D; ++i) {
        mu += h[i] * ms[i];
        for (int j = 0; j < D; ++j) va += h[i] * Ps[i * D + j] * h[j];
      }
      mean_ev[k] = mu;
      var_ev[k] = va;
    } else {
      mean_ev[k] = var_ev[k] = 0.0;
    }
  }
  return rc;
}

/* Per-event state arrays of the smoother: predicted, filtered, smoothed
 * (at start states the smoothed state is the pre-reset one). */
typedef struct {
  double *mp, *Pp, *mf, *Pf, *ms, *Ps;
} states_t;

static int states_alloc(states_t *S, int64_t n_ev, int D) {
  const size_t n = (size_t)(n_ev > 0 ? n_ev : 1);
  S->mp = malloc(sizeof(double) * n * D);
  S->mf = malloc(sizeof(double) * n * D);
  S->ms = malloc(sizeof(double) * n * D);
  S->Pp = malloc(sizeof(double) * n * D * D);
  S->Pf = malloc(sizeof(double) * n * D * D);
  S->Ps = malloc(sizeof(double) * n * D * D);
  return (S->mp && S->mf && S->ms && S->Pp && S->Pf && S->Ps) ? 0 : 4;
}

static void states_free(states_t *S) {
  free(S->mp);
  free(S->mf);
  free(S->ms);
  free(S->Pp);
  free(S->Pf);
  free(S->Ps);
}

int gpss_oracle_condition(const int32_t *spec, int64_t n_ev, const double *t_ev,
                          const int32_t *kind, const int32_t *slot, const double *y_ev,
                          const double *r0_ev, const double *invd_ev, const double *theta,
                          double *mean_ev, double *var_ev) {
  model_t M;
  if (parse_spec(spec, &M)) return 1;
  states_t S;
  int rc = states_alloc(&S, n_ev, M.dim);
  if (!rc)
    rc = smooth_all(&M, n_ev, t_ev, kind, slot, y_ev, r0_ev, invd_ev, theta, S.mp, S.Pp, S.mf,
                    S.Pf, S.ms, S.Ps, mean_ev, var_ev);
  states_free(&S);
  return rc;
}

/* Prediction of the latent f(t*) = sum_t x_t(t*) (mean and variance, given
 * all of the series' data) at test times t_star[0..n_star) by Algorithm 1,
 * on the augmented model:
 *   retrodiction (t* <= first event time): the stationary latent block,
 *     x* ~ N(0, Pinf); G = Pinf Phi^T Pinf^-1 with Phi = Phi(t_1 - t*) (the
 *     latent prior is stationary, so the predicted covariance at t_1 is
 *     Pinf), smoothed from the first event's pre-reset smoothed latent state;
 *   interpolation (t_{k-1} < t* <= t_k): predict from the filtered state
 *     after event k-1 over t* - t_{k-1}, then one RTS step from event k's
 *     smoothed state, G = P* A^T (P-_k)^-1 with A = Phi~(t_k - t*) and
 *     P-_k = A P* A^T + Q~(t_k - t*);
 *   extrapolation (t* > last event time): predict from the last filtered
 *     (= smoothed) state.
 * Smoothed covariances carry G (.) G^T.  Returns 0, 5 as the smoother. */
int gpss_oracle_predict(const int32_t *spec, int64_t n_ev, const double *t_ev, const int32_t *kind,
                        const int32_t *slot, const double *y_ev, const double *r0_ev,
                        const double *invd_ev, const double *theta, int64_t n_star,
                        const double *t_star, double *mean_out, double *var_out) {
  model_t M;
  if (parse_spec(spec, &M)) return 1;
  const int D = M.dim, DD = D * D, NX = M.nx;
  states_t S;
  int rc = states_alloc(&S, n_ev, D);
  if (!rc)
    rc = smooth_all(&M, n_ev, t_ev, kind, slot, y_ev, r0_ev, invd_ev, theta, S.mp, S.Pp, S.mf,
                    S.Pf, S.ms, S.Ps, NULL, NULL);
  double w0[2 * MAXT], q[2 * MAXT], var[MAXT], s2;
  double F[MAXD * MAXD], LQL[MAXD * MAXD], A[MAXD * MAXD], Qd[MAXD * MAXD], P0[MAXD * MAXD];
  term_params_r(&M, theta, w0, q, var, &s2);
  build_F_r(&M, w0, q, var, F, LQL);
  initial_cov_r(&M, w0, var, P0);
  for (int64_t j = 0; j < n_star && !rc; ++j) {
    const double ts = t_star[j];
    double mh[MAXD], Ph[MAXD * MAXD];
    /* first event with t_k >= t* */
    int64_t lo = 0, hi = n_ev;
    while (lo < hi) {
      const int64_t mid = (lo + hi) / 2;
      if (t_ev[mid] < ts)
        lo = mid + 1;
      else
        hi = mid;
    }
    const int64_t k = lo;
    if (k == n_ev) {
      /* extrapolation */
      discretize_r(&M, F, LQL, ts - t_ev[n_ev - 1], A, Qd);
      const double *m = S.mf + (n_ev - 1) * D, *P = S.Pf + (n_ev - 1) * DD;
      double T[MAXD * MAXD];
      for (int i = 0; i < D; ++i) {
        double acc = 0;
        for (int c = 0; c < D; ++c) acc += A[i * D + c] * m[c];
        mh[i] = acc;
      }
      matmul_r(D, A, P, T);
      for (int i = 0; i < D; ++i)
        for (int c = 0; c < D; ++c) {
          double acc = Qd[i * D + c];
          for (int e = 0; e < D; ++e) acc += T[i * D + e] * A[c * D + e];
          Ph[i * D + c] = acc;
        }
    } else if (k == 0) {
      /* retrodiction on the latent block (indices < NX) */
      discretize_r(&M, F, LQL, t_ev[0] - ts, A, Qd);
      double Ax[MAXD * MAXD], X[MAXD * MAXD], Sx[MAXD * MAXD], G[MAXD * MAXD];
      for (int i = 0; i < NX; ++i)
        for (int c = 0; c < NX; ++c) {
          Ax[i * NX + c] = A[i * D + c];
          Sx[i * NX + c] = P0[i * D + c];
        }
      /* G = P0 Ax^T P0^-1  <=>  P0 G^T = Ax P0 */
      for (int i = 0; i < NX; ++i)
        for (int c = 0; c < NX; ++c) {
          double acc = 0;
          for (int e = 0; e < NX; ++e) acc += Ax[i * NX + e] * P0[e * D + c];
          X[i * NX + c] = acc;
        }
      if (gain_solve(NX, Sx, X)) {
        rc = 5;
        break;
      }
      for (int i = 0; i < NX; ++i)
        for (int c = 0; c < NX; ++c) G[i * NX + c] = X[c * NX + i];
      const double *m1 = S.ms, *P1 = S.Ps;
      for (int i = 0; i < D; ++i) mh[i] = 0;
      for (int i = 0; i < DD; ++i) Ph[i] = 0;
      for (int i = 0; i < NX; ++i) {
        double acc = 0;
        for (int c = 0; c < NX; ++c) acc += G[i * NX + c] * m1[c];
        mh[i] = acc;
      }
      for (int i = 0; i < NX; ++i)
        for (int c = 0; c < NX; ++c) {
          double acc = P0[i * D + c];
          for (int e = 0; e < NX; ++e)
            for (int f = 0; f < NX; ++f)
              acc += G[i * NX + e] * (P1[e * D + f] - P0[e * D + f]) * G[c * NX + f];
          Ph[i * D + c] = acc;
        }
    } else {
      /* interpolation: filtered after k-1, predicted to t*, smoothed from k */
      double ms_[MAXD], Ps_[MAXD * MAXD], T[MAXD * MAXD], B[MAXD * MAXD], Qb[MAXD * MAXD];
      discretize_r(&M, F, LQL, ts - t_ev[k - 1], A, Qd);
      const double *m = S.mf + (k - 1) * D, *P = S.Pf + (k - 1) * DD;
      for (int i = 0; i < D; ++i) {
        double acc = 0;
        for (int c = 0; c < D; ++c) acc += A[i * D + c] * m[c];
        ms_[i] = acc;
      }
      matmul_r(D, A, P, T);
      for (int i = 0; i < D; ++i)
        for (int c = 0; c < D; ++c) {
          double acc = Qd[i * D + c];
          for (int e = 0; e < D; ++e) acc += T[i * D + e] * A[c * D + e];
          Ps_[i * D + c] = acc;
        }
      discretize_r(&M, F, LQL, t_ev[k] - ts, B, Qb);
      double Pn[MAXD * MAXD], mn[MAXD], X[MAXD * MAXD], G[MAXD * MAXD];
      matmul_r(D, B, Ps_, T);
      for (int i = 0; i < D; ++i) {
        double acc = 0;
        for (int c = 0; c < D; ++c) acc += B[i * D + c] * ms_[c];
        mn[i] = acc;
        for (int c = 0; c < D; ++c) {
          double a2 = Qb[i * D + c];
          for (int e = 0; e < D; ++e) a2 += T[i * D + e] * B[c * D + e];
          Pn[i * D + c] = a2;
        }
      }
      memcpy(X, T, sizeof(double) * DD); /* B P* = (P* B^T)^T */
      if (gain_solve(D, Pn, X)) {
        rc = 5;
        break;
      }
      for (int i = 0; i < D; ++i)
        for (int c = 0; c < D; ++c) G[i * D + c] = X[c * D + i];
      const double *m1 = S.ms + k * D, *P1 = S.Ps + k * DD;
      double mp1[MAXD], Pp1[MAXD * MAXD];
      memcpy(mp1, mn, sizeof(mn));
      /* P-_k recomputed from t* (equal to the filter's by the semigroup) */
      for (int i = 0; i < DD; ++i) Pp1[i] = Pn[i];
      /* restore Pn: gain_solve overwrote it */
      matmul_r(D, B, Ps_, T);
      for (int i = 0; i < D; ++i)
        for (int c = 0; c < D; ++c) {
          double a2 = Qb[i * D + c];
          for (int e = 0; e < D; ++e) a2 += T[i * D + e] * B[c * D + e];
          Pp1[i * D + c] = a2;
        }
      for (int i = 0; i < D; ++i) {
        double acc = ms_[i];
        for (int c = 0; c < D; ++c) acc += G[i * D + c] * (m1[c] - mp1[c]);
        mh[i] = acc;
      }
      for (int i = 0; i < D; ++i)
        for (int c = 0; c < D; ++c) {
          double acc = Ps_[i * D + c];
          for (int e = 0; e < D; ++e)
            for (int f = 0; f < D; ++f)
              acc += G[i * D + e] * (P1[e * D + f] - Pp1[e * D + f]) * G[c * D + f];
          Ph[i * D + c] = acc;
        }
    }
    double mu = 0, va = 0;
    for (int t = 0; t < M.n_terms; ++t) {
      mu += mh[M.toff[t]];
      for (int u = 0; u < M.n_terms; ++u) va += Ph[M.toff[t] * D + M.toff[u]];
    }
    mean_out[j] = mu;
    var_out[j] = va;
  }
  states_free(&S);
  return rc;
}
