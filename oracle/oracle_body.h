/*
 * Scalar-generic body of the FP64 oracle (see gpss_oracle.c).  Included twice:
 * once with SCALAR = double and once with SCALAR = double complex, so that the
 * complex-step derivative runs the very same arithmetic as the plain value.
 *
 * TEST INFRASTRUCTURE ONLY: never linked into, or called by, the product path.
 */

/* Per-term kernel constants from natural parameters.
 * SHO (Appendix B, Eqs. sho_kernel, sho_Qc_Pinf): (sigma, omega0, Q),
 *   Q_c = 2 omega0^3 sigma^2 / Q, P_inf = sigma^2 diag(1, omega0^2).
 * Matern-3/2 is the critically damped SHO: Q = 1/2, omega0 = sqrt(3)/ell
 * (Eq. sho_kernel, Q = 1/2 case).
 * Product of two SHOs (Appendix C.2): (sigma, omega_a, Q_a, omega_b, Q_b),
 *   k = sigma^2 k_a k_b with unit-variance factors; factor b's (omega, Q)
 *   are stored at index MAXT + t of w0 and q.
 * Last parameter: white-noise sd s. */
static void SFX(term_params)(const model_t *M, const SCALAR *th, SCALAR *w0, SCALAR *q,
                             SCALAR *var, SCALAR *s2) {
  int j = 0;
  for (int t = 0; t < M->n_terms; ++t) {
    SCALAR sig;
    if (M->kind[t] == 1) {
      sig = th[j];
      w0[t] = th[j + 1];
      q[t] = th[j + 2];
      j += 3;
    } else if (M->kind[t] == 2) {
      sig = th[j];
      w0[t] = S_SQRT(3.0) / th[j + 1];
      q[t] = 0.5;
      j += 2;
    } else {
      sig = th[j];
      w0[t] = th[j + 1];
      q[t] = th[j + 2];
      w0[MAXT + t] = th[j + 3];
      q[MAXT + t] = th[j + 4];
      j += 5;
    }
    var[t] = sig * sig;
  }
  *s2 = th[j] * th[j];
}

/* Augmented feedback matrix F~ (Eq. augmented_sde, generalised to several
 * integral states in Section 3.2.3) and L~ Q_c L~^T.
 * State order: (x_t, xdot_t) for every term t, then the integral states.
 * Layout 0: one z_j per slot j, dz_j/dt = H x = sum_t x_t (Appendix C.1).
 * Layout 1: one z_{t,j} per term and slot, dz_{t,j}/dt = x_t. */
static void SFX(build_F)(const model_t *M, const SCALAR *w0, const SCALAR *q, const SCALAR *var,
                         SCALAR *F, SCALAR *LQL) {
  const int D = M->dim;
  for (int i = 0; i < D * D; ++i) {
    F[i] = 0;
    LQL[i] = 0;
  }
  for (int t = 0; t < M->n_terms; ++t) {
    const int i = M->toff[t];
    if (M->kind[t] != 3) {
      F[i * D + i + 1] = 1.0;
      F[(i + 1) * D + i] = -w0[t] * w0[t];
      F[(i + 1) * D + i + 1] = -w0[t] / q[t];
      LQL[(i + 1) * D + i + 1] = 2.0 * w0[t] * w0[t] * w0[t] * var[t] / q[t];
      continue;
    }
    /* product (Appendix C.2): F = F_a (x) I + I (x) F_b and
     * L Q_c L^T = (L Q_c L^T)_a (x) P_inf,b + P_inf,a (x) (L Q_c L^T)_b,
     * factor a of unit variance, factor b of variance sigma^2; index of
     * (row of a, row of b) = 2 r_a + r_b. */
    const SCALAR wa = w0[t], qa = q[t], wb = w0[MAXT + t], qb = q[MAXT + t];
    const SCALAR Fa[4] = {0.0, 1.0, -wa * wa, -wa / qa}, Fb[4] = {0.0, 1.0, -wb * wb, -wb / qb};
    const SCALAR Pa[2] = {1.0, wa * wa}, Pb[2] = {var[t], var[t] * wb * wb};
    const SCALAR La = 2.0 * wa * wa * wa / qa, Lb = 2.0 * wb * wb * wb * var[t] / qb;
    for (int ra = 0; ra < 2; ++ra)
      for (int rb = 0; rb < 2; ++rb)
        for (int ca = 0; ca < 2; ++ca)
          for (int cb = 0; cb < 2; ++cb) {
            const int r = i + 2 * ra + rb, c = i + 2 * ca + cb;
            F[r * D + c] = (rb == cb ? Fa[2 * ra + ca] : 0.0) + (ra == ca ? Fb[2 * rb + cb] : 0.0);
          }
    for (int ra = 0; ra < 2; ++ra)
      for (int rb = 0; rb < 2; ++rb) {
        const int r = i + 2 * ra + rb;
        LQL[r * D + r] = (ra == 1 ? La : 0.0) * Pb[rb] + Pa[ra] * (rb == 1 ? Lb : 0.0);
      }
  }
  for (int j = 0; j < M->n_slots; ++j) {
    for (int t = 0; t < M->n_terms; ++t) {
      int zi = zindex(M, j, t);
      F[zi * D + M->toff[t]] = 1.0;
    }
  }
}

static void SFX(matmul)(int n, const SCALAR *A, const SCALAR *B, SCALAR *C) {
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      SCALAR acc = 0;
      for (int k = 0; k < n; ++k) acc += A[i * n + k] * B[k * n + j];
      C[i * n + j] = acc;
    }
}

/* Matrix exponential by scaling and squaring of a truncated Taylor series:
 * exp(A) = (exp(A / 2^r))^(2^r) with ||A / 2^r||_1 <= 1/2 and 24 Taylor terms
 * (truncation below 1e-30).  A library-free restatement of the textbook
 * method; adequate because every argument here has a small norm. */
static void SFX(expm)(int n, const SCALAR *A, SCALAR *E) {
  SCALAR X[4 * MAXD * MAXD], T[4 * MAXD * MAXD], U[4 * MAXD * MAXD];
  double nrm = 0;
  for (int j = 0; j < n; ++j) {
    double c = 0;
    for (int i = 0; i < n; ++i) c += S_ABS(A[i * n + j]);
    if (c > nrm) nrm = c;
  }
  int r = 0;
  while (nrm > 0.5 && r < 200) {
    nrm *= 0.5;
    ++r;
  }
  double sc = ldexp(1.0, -r);
  for (int i = 0; i < n * n; ++i) X[i] = A[i] * sc;
  for (int i = 0; i < n * n; ++i) {
    E[i] = (i % (n + 1) == 0) ? 1.0 : 0.0;
    T[i] = E[i];
  }
  for (int k = 1; k <= 24; ++k) {
    SFX(matmul)(n, T, X, U);
    for (int i = 0; i < n * n; ++i) {
      T[i] = U[i] / (double)k;
      E[i] += T[i];
    }
  }
  for (int s = 0; s < r; ++s) {
    SFX(matmul)(n, E, E, U);
    memcpy(E, U, sizeof(SCALAR) * n * n);
  }
}

/* Transition Phi~(dt) and process noise Q~(dt) of the augmented model.
 * Van Loan (Eq. Q_from_vanloan): with C = [[-F~, L~QcL~^T], [0, F~^T]] dt,
 * exp(C) = [[F2, G2], [0, F3]], Phi~ = F3^T and Q~ = F3^T G2.
 * The exponential of C grows like exp(|F| dt), which the paper notes is
 * unusable for long gaps (Section 2.2.2, Section 3.2).  So Van Loan is applied
 * to h = dt / 2^s with ||F~|| h <= 1/2 and the result is doubled s times with
 * the exact semigroup identities of Eq. sde_sol:
 *   Phi~(2h) = Phi~(h)^2,  Q~(2h) = Phi~(h) Q~(h) Phi~(h)^T + Q~(h). */
static void SFX(discretize)(const model_t *M, const SCALAR *F, const SCALAR *LQL, SCALAR dt,
                            SCALAR *Phi, SCALAR *Q) {
  const int D = M->dim, D2 = 2 * M->dim;
  for (int i = 0; i < D * D; ++i) {
    Phi[i] = (i % (D + 1) == 0) ? 1.0 : 0.0;
    Q[i] = 0;
  }
  if (dt == 0.0) return;
  double nrm = 0;
  for (int j = 0; j < D; ++j) {
    double c = 0;
    for (int i = 0; i < D; ++i) c += S_ABS(F[i * D + j]);
    if (c > nrm) nrm = c;
  }
  int s = 0;
  SCALAR h = dt;
  while (nrm * S_ABS(h) > 0.5 && s < 400) {
    h *= 0.5;
    ++s;
  }
  SCALAR C[4 * MAXD * MAXD], E[4 * MAXD * MAXD], T[MAXD * MAXD], U[MAXD * MAXD];
  for (int i = 0; i < D2 * D2; ++i) C[i] = 0;
  for (int i = 0; i < D; ++i)
    for (int j = 0; j < D; ++j) {
      C[i * D2 + j] = -F[i * D + j] * h;
      C[i * D2 + D + j] = LQL[i * D + j] * h;
      C[(D + i) * D2 + D + j] = F[j * D + i] * h;
    }
  SFX(expm)(D2, C, E);
  for (int i = 0; i < D; ++i)
    for (int j = 0; j < D; ++j) Phi[i * D + j] = E[(D + j) * D2 + D + i]; /* F3^T */
  for (int i = 0; i < D; ++i)
    for (int j = 0; j < D; ++j) {
      SCALAR acc = 0;
      for (int k = 0; k < D; ++k) acc += E[(D + k) * D2 + D + i] * E[k * D2 + D + j];
      Q[i * D + j] = acc; /* F3^T G2 */
    }
  for (int i = 0; i < D; ++i)
    for (int j = 0; j < i; ++j) {
      SCALAR a = 0.5 * (Q[i * D + j] + Q[j * D + i]);
      Q[i * D + j] = a;
      Q[j * D + i] = a;
    }
  for (int it = 0; it < s; ++it) {
    /* Q <- Phi Q Phi^T + Q */
    SFX(matmul)(D, Phi, Q, T);
    for (int i = 0; i < D; ++i)
      for (int j = 0; j <= i; ++j) {
        SCALAR acc = 0;
        for (int k = 0; k < D; ++k) acc += T[i * D + k] * Phi[j * D + k];
        U[i * D + j] = acc + Q[i * D + j];
        U[j * D + i] = U[i * D + j];
      }
    memcpy(Q, U, sizeof(SCALAR) * D * D);
    SFX(matmul)(D, Phi, Phi, T);
    memcpy(Phi, T, sizeof(SCALAR) * D * D);
  }
}

/* Timing mode of the CPU baseline: Phi~ and Q~ of a model whose terms are
 * all SHOs with Q >= 1/2 (Matern-3/2 included) in closed form.  Underdamped
 * terms (Q > 1/2) take the closed forms printed in Appendix B, per term: Phi (Eq. sho_phi), Q (Eq. sho_Q), the first row of
 * Phibar = int_0^dt Phi (Eq. sho_phibar), Q~12 (Eq. analytic_Qaug12) and
 * Q~22 (Eq. analytic_Qaug22).  The terms are independent, so an integral
 * state z gets Phibar's row and Q~12 of every term it integrates, and two
 * integral states share Q~22 of every term both integrate (each integrates
 * the same function over the same step).  sigma^2 e^{-w0 dt/Q} (e^{w0 dt/Q}
 * - 1 - ...) of Eq. sho_Q is written (1 - e^{-w0 dt/Q}) - e^{-w0 dt/Q}(...)
 * so that long steps do not overflow.  A critically damped term (Matern-3/2,
 * or an SHO with Q = 1/2) takes Phi of Eq. sho_phi (Q = 1/2), Q = P_inf -
 * Phi P_inf Phi^T (Eq. Q), and Phibar, Q~12, Q~22 from their defining
 * integrals (Eqs. phiaug, Q_aug: Q~12_i = Q_c int_0^dt (Phi(s) L)_i G(s) ds,
 * Q~22 = Q_c int_0^dt G(s)^2 ds, G(s) = int_0^s Phi_01) worked out for
 * Phi(s) L = e^{-w s} (s, 1 - w s); with x = w dt and E = e^{-x}:
 *   Phibar = ((2 - (2 + x) E) / w, (1 - (1 + x) E) / w^2),
 *   Q~12 = sigma^2 (2 (x^2 E^2 + 2 x E^2 - 2 (x + 1) E + 1 + E^2) / w,
 *                   -2 x^2 E^2 + 4 x E - 2 x E^2 - 1 + E^2),
 *   Q~22 = sigma^2 (4 x - 11 + 8 (x + 2) E - (2 x^2 + 6 x + 5) E^2) / w^2.
 * Returns 0, or 1 when a term is overdamped or a product (the caller then
 * uses Van Loan). */
static int SFX(discretize_closed)(const model_t *M, const SCALAR *w0v, const SCALAR *qv,
                                  const SCALAR *var, SCALAR dt, SCALAR *Phi, SCALAR *Q) {
  const int D = M->dim;
  for (int t = 0; t < M->n_terms; ++t)
    if (M->kind[t] == 3 || !(S_RE(qv[t]) >= 0.5)) return 1;
  for (int i = 0; i < D * D; ++i) {
    Phi[i] = (i % (D + 1) == 0) ? 1.0 : 0.0;
    Q[i] = 0;
  }
  if (dt == 0.0) return 0;
  SCALAR pb[MAXT][2], q12[MAXT][2], q22[MAXT];
  for (int t = 0; t < M->n_terms; ++t) {
    const int i = M->toff[t];
    const SCALAR w0 = w0v[t], q = qv[t], v = var[t];
    if (S_RE(q) == 0.5) {
      /* critically damped */
      const SCALAR x = w0 * dt, E = S_EXP(-x), E2 = E * E;
      Phi[i * D + i] = E * (1.0 + x);
      Phi[i * D + i + 1] = E * dt;
      Phi[(i + 1) * D + i] = -E * w0 * w0 * dt;
      Phi[(i + 1) * D + i + 1] = E * (1.0 - x);
      Q[i * D + i] = v * (1.0 - (x * x + (x + 1.0) * (x + 1.0)) * E2);
      Q[i * D + i + 1] = Q[(i + 1) * D + i] = v * 2.0 * x * x * w0 * E2;
      Q[(i + 1) * D + i + 1] = v * w0 * w0 * (1.0 - (x * x + (x - 1.0) * (x - 1.0)) * E2);
      pb[t][0] = (2.0 - (2.0 + x) * E) / w0;
      pb[t][1] = (1.0 - (1.0 + x) * E) / (w0 * w0);
      q12[t][0] = v * 2.0 * (x * x * E2 + 2.0 * x * E2 - 2.0 * (x + 1.0) * E + 1.0 + E2) / w0;
      q12[t][1] = v * (-2.0 * x * x * E2 + 4.0 * x * E - 2.0 * x * E2 - 1.0 + E2);
      q22[t] = v * (4.0 * x - 11.0 + 8.0 * (x + 2.0) * E - (2.0 * x * x + 6.0 * x + 5.0) * E2) /
               (w0 * w0);
      continue;
    }
    const SCALAR eta = S_SQRT(1.0 - 1.0 / (4.0 * q * q));
    const SCALAR tau = eta * w0 * dt, A = 1.0 / (2.0 * eta * q);
    const SCALAR e1 = S_EXP(-w0 * dt / (2.0 * q)), e2 = e1 * e1;
    const SCALAR sn = S_SIN(tau), cs = S_COS(tau), s2t = S_SIN(2.0 * tau), c2t = S_COS(2.0 * tau);
    const SCALAR ss = sn * sn;
    /* Eq. sho_phi, Q > 1/2 */
    Phi[i * D + i] = e1 * (cs + A * sn);
    Phi[i * D + i + 1] = e1 * sn / (eta * w0);
    Phi[(i + 1) * D + i] = -e1 * w0 * sn / eta;
    Phi[(i + 1) * D + i + 1] = e1 * (cs - A * sn);
    /* Eq. sho_Q */
    const SCALAR k2 = 1.0 / (2.0 * eta * eta * q * q);
    Q[i * D + i] = v * ((1.0 - e2) - e2 * (A * s2t + k2 * ss));
    Q[i * D + i + 1] = Q[(i + 1) * D + i] = v * e2 * w0 / (eta * eta * q) * ss;
    Q[(i + 1) * D + i + 1] = v * w0 * w0 * ((1.0 - e2) + e2 * (A * s2t - k2 * ss));
    /* Eq. sho_phibar, first row: e^{a t}/(a^2 + b^2) (Ic + A Is, B Is) from 0 to dt */
    const SCALAR a = -w0 / (2.0 * q), b = eta * w0, B = 1.0 / (eta * w0);
    const SCALAR n1 = S_EXP(a * dt) / (a * a + b * b), n0 = 1.0 / (a * a + b * b);
    const SCALAR Is1 = a * sn - b * cs, Ic1 = a * cs + b * sn; /* at t = dt (b dt = tau) */
    const SCALAR Is0 = -b, Ic0 = a;                            /* at t = 0 */
    pb[t][0] = n1 * (Ic1 + A * Is1) - n0 * (Ic0 + A * Is0);
    pb[t][1] = n1 * (B * Is1) - n0 * (B * Is0);
    /* Eq. analytic_Qaug12 */
    const SCALAR r = e1 * (cs + A * sn) - 1.0;
    q12[t][0] = v / (q * w0) * r * r;
    q12[t][1] = v * (A * e1 * (4.0 * sn - e1 * s2t) - 2.0 * A * A * e2 * ss + e2 - 1.0);
    /* Eq. analytic_Qaug22 */
    q22[t] = v / (4.0 * q * q * w0 * w0) *
             (8.0 * q * w0 * dt + 4.0 * q * q - 12.0 + A * A * e2 * (c2t - 16.0 * q * q * q * q) +
              16.0 * e1 * (cs + (1.0 - 2.0 * q * q) * A * sn) +
              e2 * ((1.0 - 3.0 * A * A) / A * s2t - 3.0 * c2t));
  }
  for (int z = M->nx; z < D; ++z) {
    const int zs = z - M->nx;
    for (int t = 0; t < M->n_terms; ++t) {
      if (M->layout == 1 && zs % M->n_terms != t) continue; /* z_{t,j} integrates x_t only */
      const int i = M->toff[t];
      Phi[z * D + i] = pb[t][0];
      Phi[z * D + i + 1] = pb[t][1];
      Q[i * D + z] = Q[z * D + i] = q12[t][0];
      Q[(i + 1) * D + z] = Q[z * D + i + 1] = q12[t][1];
    }
    for (int z2 = M->nx; z2 < D; ++z2) {
      const int zs2 = z2 - M->nx;
      SCALAR acc = 0;
      for (int t = 0; t < M->n_terms; ++t) {
        if (M->layout == 1 && (zs % M->n_terms != t || zs2 % M->n_terms != t)) continue;
        acc += q22[t];
      }
      Q[z * D + z2] = acc;
    }
  }
  return 0;
}

/* Initial covariance P0 = blkdiag(P_inf, I) (Section 3.2.3, final paragraph). */
static void SFX(initial_cov)(const model_t *M, const SCALAR *w0, const SCALAR *var, SCALAR *P) {
  const int D = M->dim;
  for (int i = 0; i < D * D; ++i) P[i] = 0;
  for (int t = 0; t < M->n_terms; ++t) {
    const int i = M->toff[t];
    if (M->kind[t] != 3) {
      P[i * D + i] = var[t];
      P[(i + 1) * D + i + 1] = var[t] * w0[t] * w0[t];
      continue;
    }
    /* P_inf = P_inf,a (x) P_inf,b (Appendix C.2) */
    const SCALAR Pa[2] = {1.0, w0[t] * w0[t]}, Pb[2] = {var[t], var[t] * w0[MAXT + t] * w0[MAXT + t]};
    for (int ra = 0; ra < 2; ++ra)
      for (int rb = 0; rb < 2; ++rb) P[(i + 2 * ra + rb) * D + i + 2 * ra + rb] = Pa[ra] * Pb[rb];
  }
  for (int i = M->nx; i < D; ++i) P[i * D + i] = 1.0;
}

/* Sequential integrated Kalman filter and log-likelihood.
 * Predict with Phi~, Q~ (Eq. integrated_kalman_pred); at an exposure start
 * apply the reset R_j of that exposure's slot (Eq. integrated_kalman_update,
 * Section 3.2.3); at an exposure end update with H~ = e_z / delta
 * (Eqs. H_aug, kalman_update) and add the term of Eq. loglikelihood.
 * The covariance update uses the Joseph form, which is algebraically equal
 * to P - K S K^T.  Summation is Neumaier-compensated. */
static int SFX(filter)(const model_t *M, const SCALAR *th, int64_t n_ev, const SCALAR *t_ev,
                       const int32_t *kind, const int32_t *slot, const double *y_ev,
                       const double *r0_ev, const SCALAR *invd_ev, SCALAR *ll_out, double *dumpP,
                       double *dumpS) {
  const int D = M->dim;
  SCALAR w0[2 * MAXT], q[2 * MAXT], var[MAXT], s2;
  SCALAR F[MAXD * MAXD], LQL[MAXD * MAXD], Phi[MAXD * MAXD], Qd[MAXD * MAXD];
  SCALAR P[MAXD * MAXD], T[MAXD * MAXD], A[MAXD * MAXD];
  SCALAR m[MAXD], mt[MAXD], h[MAXD], u[MAXD], K[MAXD];
  SFX(term_params)(M, th, w0, q, var, &s2);
  SFX(build_F)(M, w0, q, var, F, LQL);
  SFX(initial_cov)(M, w0, var, P);
  for (int i = 0; i < D; ++i) m[i] = 0;
  SCALAR sum = 0, comp = 0;
  SCALAR tprev = n_ev > 0 ? t_ev[0] : 0.0;
  int64_t n_end = 0;
  for (int64_t k = 0; k < n_ev; ++k) {
    SCALAR dt = t_ev[k] - tprev;
    tprev = t_ev[k];
    if (S_RE(dt) < 0) return 2;
    if (!M->closed || SFX(discretize_closed)(M, w0, q, var, dt, Phi, Qd))
      SFX(discretize)(M, F, LQL, dt, Phi, Qd);
    for (int i = 0; i < D; ++i) {
      SCALAR acc = 0;
      for (int j = 0; j < D; ++j) acc += Phi[i * D + j] * m[j];
      mt[i] = acc;
    }
    memcpy(m, mt, sizeof(SCALAR) * D);
    SFX(matmul)(D, Phi, P, T);
    for (int i = 0; i < D; ++i)
      for (int j = 0; j <= i; ++j) {
        SCALAR acc = 0;
        for (int kk = 0; kk < D; ++kk) acc += T[i * D + kk] * Phi[j * D + kk];
        P[i * D + j] = acc + 0.5 * (Qd[i * D + j] + Qd[j * D + i]);
        P[j * D + i] = P[i * D + j];
      }
    const int sj = slot[k];
    if (kind[k] != 2 && (sj < 0 || sj >= M->n_slots)) return 3;
    if (kind[k] == 0) {
      /* exposure start: zero this slot's integral state(s) */
      for (int t = 0; t < M->n_zper; ++t) {
        int z = zindex(M, sj, t);
        m[z] = 0;
        for (int i = 0; i < D; ++i) {
          P[z * D + i] = 0;
          P[i * D + z] = 0;
        }
      }
    } else {
      for (int i = 0; i < D; ++i) h[i] = 0;
      if (kind[k] == 2)
        for (int t = 0; t < M->n_terms; ++t) h[M->toff[t]] = 1.0; /* instantaneous: f = H x */
      else
        for (int t = 0; t < M->n_zper; ++t) h[zindex(M, sj, t)] = invd_ev[k];
      SCALAR Sv = r0_ev[k] + s2, hm = 0;
      for (int i = 0; i < D; ++i) {
        SCALAR acc = 0;
        for (int j = 0; j < D; ++j) acc += P[i * D + j] * h[j];
        u[i] = acc;
        Sv += h[i] * acc;
        hm += h[i] * m[i];
      }
      SCALAR v = y_ev[k] - hm;
      SCALAR r = r0_ev[k] + s2;
      for (int i = 0; i < D; ++i) {
        K[i] = u[i] / Sv;
        m[i] += K[i] * v;
      }
      /* Joseph form: (I - K h^T) P (I - K h^T)^T + K r K^T */
      for (int i = 0; i < D; ++i)
        for (int j = 0; j < D; ++j) A[i * D + j] = (i == j ? 1.0 : 0.0) - K[i] * h[j];
      SFX(matmul)(D, A, P, T);
      for (int i = 0; i < D; ++i)
        for (int j = 0; j <= i; ++j) {
          SCALAR acc = 0;
          for (int kk = 0; kk < D; ++kk) acc += T[i * D + kk] * A[j * D + kk];
          P[i * D + j] = acc + K[i] * r * K[j];
          P[j * D + i] = P[i * D + j];
        }
      SCALAR term = -0.5 * (S_LOG(TWO_PI * Sv) + v * v / Sv);
      SCALAR tt = sum + term;
      if (S_ABS(sum) >= S_ABS(term))
        comp += (sum - tt) + term;
      else
        comp += (term - tt) + sum;
      sum = tt;
      if (dumpS) dumpS[n_end] = S_RE(Sv);
      ++n_end;
    }
    if (dumpP)
      for (int i = 0; i < D * D; ++i) dumpP[k * D * D + i] = S_RE(P[i]);
  }
  *ll_out = sum + comp;
  return 0;
}
