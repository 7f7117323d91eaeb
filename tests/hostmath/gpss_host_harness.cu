// Host build of the CUDA path's device arithmetic, for CPU tests: the same
// header functions the kernels inline, called from ordinary host code.
// Compiled by tests/test_host_math.py with nvcc into a shared library.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "gpss_kernels.cuh"
#include "gpss_prod.cuh"

using namespace gpss;

namespace {

void build_table(float a, float beta, float *tab) {
  EconMap E;
  econ_map(E);
  Dual2<double> g[6][TAB_NC];
  table_coeffs<Dual2<double>>(E, mk((double)a, 1.0, 0.0), mk((double)beta, 0.0, 1.0), g);
  for (int k = 0; k < TAB_NC; ++k) {
    float *r = tab + k * TAB_W;
    for (int j = 0; j < TAB_W; ++j) r[j] = 0.f;
    for (int j = 0; j < 6; ++j) {
      r[j] = (float)g[j][k].v;
      r[8 + j] = (float)g[j][k].da;
      r[14 + j] = (float)g[j][k].db;
    }
  }
}

TermC<float> termc(float a, float beta) {
  TermC<float> c;
  c.a = a;
  c.beta = beta;
  c.w2 = beta + a * a;
  c.qc = 1.f;
  c.var = 1.f;
  finish_termc(c);
  return c;
}

template <class S>
void combine_s(const float *Ei, const float *Ej, float *out) {
  constexpr int NF = Elem<S>::NF;
  float a[NF], b[NF], o[NF];
  std::memcpy(a, Ei, sizeof a);
  std::memcpy(b, Ej, sizeof b);
  combine<S>(EView{a, 1}, EView{b, 1}, EView{o, 1});
  std::memcpy(out, o, sizeof o);
}

template <class S>
double chunk_ll_s(const float *m, const float *P, const float *eta, const float *J, double gam,
                  double ld, double ne) {
  return chunk_loglik<S>(m, P, eta, J, gam, ld, ne);
}

template <class S>
void adj_s(const float *m, const float *P, const float *eta, const float *J, float *lam,
           float *Lam) {
  boundary_adjoint<S>(m, P, eta, J, lam, Lam);
}

template <int D>
float solve_d(const float *A, const float *B, float *X, int R) {
  float a[D][D], b[D][8];
  for (int i = 0; i < D; ++i) {
    for (int j = 0; j < D; ++j) a[i][j] = A[i * D + j];
    for (int j = 0; j < 8; ++j) b[i][j] = j < R ? B[i * R + j] : 0.f;
  }
  const float ld = solve_inplace<D, 8, float>(a, b);
  for (int i = 0; i < D; ++i)
    for (int j = 0; j < R; ++j) X[i * R + j] = b[i][j];
  return ld;
}

// Observation of a measurement event and its conditioned (mean, variance)
// from full symmetric P and Lam (row-major D x D), for shape ids
// 3 = (2 terms, no slot: instantaneous), 4 = (2 terms, 2 slots), 1 = (2 terms,
// 1 slot, layout 1).  out4 = (hu, hm, cond mean, cond var); u receives P h.
template <class S>
void observe_s(int j, float w, const float *m, const float *Pf, const float *lam,
               const float *Lf, float *u, float *out4) {
  constexpr int D = S::D;
  float P[S::NP], L[S::NP];
  for (int i = 0; i < D; ++i)
    for (int k = i; k < D; ++k) {
      P[S::pk(i, k)] = Pf[i * D + k];
      L[S::pk(i, k)] = Lf[i * D + k];
    }
  float hu, hm;
  obs_project<S>(j, w, m, P, u, hu, hm);
  const float2 c = conditioned<S>(j, w, m, P, lam, L);
  out4[0] = hu;
  out4[1] = hm;
  out4[2] = c.x;
  out4[3] = c.y;
}
// The product term's transition and noise (row-major 4 x 4) for a step dt
// and parameters (sigma, omega_a, Q_a, omega_b, Q_b), built as the kernels
// build them: Phi_a (x) Phi_b and Eq. product_Q from the two factors' 2 x 2
// blocks (osc2), in FP64 (prec 64) or FP32 (prec 32).
template <class F>
void prod_disc_t(double dt, const double *th, double *Phi, double *Q) {
  const F var = F(th[0]) * F(th[0]);
  const Osc2<F> A = osc2<F, F>(F(dt), F(th[1]), F(th[2]), F(1));
  const Osc2<F> B = osc2<F, F>(F(dt), F(th[3]), F(th[4]), var);
  const F Pa[2] = {F(1), F(th[1]) * F(th[1])}, Pb[2] = {var, var * F(th[3]) * F(th[3])};
  for (int ra = 0; ra < 2; ++ra)
    for (int rb = 0; rb < 2; ++rb)
      for (int ca = 0; ca < 2; ++ca)
        for (int cb = 0; cb < 2; ++cb) {
          const int r = 2 * ra + rb, c = 2 * ca + cb;
          Phi[4 * r + c] = (double)(A.p[ra][ca] * B.p[rb][cb]);
          Q[4 * r + c] = (double)((ra == ca ? Pa[ra] * B.q[rb][cb] : F(0)) +
                                  (rb == cb ? A.q[ra][ca] * Pb[rb] : F(0)) -
                                  A.q[ra][ca] * B.q[rb][cb]);
        }
}
}  // namespace

namespace {

// Element of events [k_begin, k_end) of one series, as the chunk kernels
// form it but in FP64 with the on-the-fly discretisation: chunks of
// chunk_len events from k_begin, each run by elem_event from an unknown
// incoming state (from the prior for the series' first chunk), then combined
// in time order with their log-normalisers.  dt, tag: the series' events;
// meas3: (y, r0, w) per measurement in event order; theta: one row.
// out: NF + 1 doubles (fields of Elem, then c).
template <class S>
void span_elem_s(const double *dt, const uint8_t *tag, const double *meas3, const float *theta,
                 const int *kinds, int64_t k_begin, int64_t k_end, int chunk_len, double *out) {
  constexpr int D = S::D, NF = Elem<S>::NF, NC = NF + 1;
  TermC<double> tc[S::NT];
  double s2;
  load_terms<S::NT, double>(theta, kinds, tc, s2);
  int64_t mi = 0;
  for (int64_t k = 0; k < k_begin; ++k) mi += tag[k] & 1;
  double acc[NC], cur[NC], tmp[NC];
  bool have = false;
  for (int64_t c0 = k_begin; c0 < k_end; c0 += chunk_len) {
    const int64_t c1 = std::min<int64_t>(k_end, c0 + chunk_len);
    double A[D][D], b[D], C[S::NP], eta[D], J[S::NP];
    const bool first = c0 == 0;
    if (first) {
      init_state<S>(tc, b, C);
    } else {
      for (int i = 0; i < D; ++i) b[i] = 0.0;
      for (int i = 0; i < S::NP; ++i) C[i] = 0.0;
    }
    for (int i = 0; i < D; ++i) {
      eta[i] = 0.0;
      for (int j = 0; j < D; ++j) A[i][j] = (!first && i == j) ? 1.0 : 0.0;
    }
    for (int i = 0; i < S::NP; ++i) J[i] = 0.0;
    double gam = 0.0, ld = 0.0;
    int n_end = 0;
    bool bad = false;
    for (int64_t k = c0; k < c1; ++k) {
      Blocks<double> B[S::NT];
      for (int t = 0; t < S::NT; ++t)
        B[t] = make_blocks(discretize<double, double, true>(dt[k], tc[t].a, tc[t].beta), tc[t]);
      double y = 0.0, r0 = 0.0, w = 0.0;
      if (tag[k] & 1) {
        y = meas3[3 * mi];
        r0 = meas3[3 * mi + 1];
        w = meas3[3 * mi + 2];
        ++mi;
      }
      elem_event<S, double>(B, tag[k], y, r0, w, s2, A, b, C, eta, J, gam, ld, n_end, bad);
    }
    using L = Elem<S>;
    for (int i = 0; i < D; ++i) {
      for (int j = 0; j < D; ++j) cur[L::A + i * D + j] = A[i][j];
      cur[L::B + i] = b[i];
      cur[L::ETA + i] = eta[i];
    }
    for (int i = 0; i < S::NP; ++i) {
      cur[L::C + i] = C[i];
      cur[L::J + i] = J[i];
    }
    cur[NF] = -0.5 * (ld + gam + n_end * LOG_2PI);
    if (!have) {
      std::memcpy(acc, cur, sizeof acc);
      have = true;
    } else {
      combine<S, double, true>(EViewT<double>{acc, 1}, EViewT<double>{cur, 1},
                               EViewT<double>{tmp, 1});
      std::memcpy(acc, tmp, sizeof acc);
    }
  }
  std::memcpy(out, acc, sizeof acc);
}

// The log-likelihood of a series from its spans' elements (n_spans x NC,
// time order), folded as the device does.
template <class S>
double span_fold_s(const double *elems, int n_spans) {
  constexpr int NC = Elem<S>::NF + 1;
  double acc[NC], tmp[NC];
  std::memcpy(acc, elems, sizeof acc);
  for (int sp = 1; sp < n_spans; ++sp) {
    double nxt[NC];
    std::memcpy(nxt, elems + (size_t)sp * NC, sizeof nxt);
    combine<S, double, true>(EViewT<double>{acc, 1}, EViewT<double>{nxt, 1},
                             EViewT<double>{tmp, 1});
    std::memcpy(acc, tmp, sizeof acc);
  }
  return acc[NC - 1];
}

}  // namespace

extern "C" {

// out6 = (f, f', F1, I_ff, I_pp, I_FF); mode 0: table path (FP32),
// 1: on-the-fly series / closed forms (FP32), 2: same in FP64.
void hh_discretize(int mode, double t, double a, double beta, double *out6) {
  if (mode == 2) {
    Disc<double> d = discretize<double, double>(t, a, beta);
    double v[6] = {d.f, d.fp, d.F1, d.Iff, d.Ipp, d.IFF};
    std::memcpy(out6, v, sizeof v);
    return;
  }
  Disc<float> d;
  if (mode == 0) {
    float tab[TAB_TERM];
    build_table((float)a, (float)beta, tab);
    d = discretize_tab((float)t, termc((float)a, (float)beta), reinterpret_cast<const float4 *>(tab));
  } else {
    d = discretize<float, float>((float)t, (float)a, (float)beta);
  }
  const float v[6] = {d.f, d.fp, d.F1, d.Iff, d.Ipp, d.IFF};
  for (int i = 0; i < 6; ++i) out6[i] = v[i];
}

// out18 = values, d/da, d/dbeta of the six scalars (table path, FP32 duals)
void hh_discretize_dual(double t, double a, double beta, double *out18) {
  float tab[TAB_TERM];
  build_table((float)a, (float)beta, tab);
  Disc<Dual2<float>> d = discretize_tab_dual((float)t, termc((float)a, (float)beta),
                                             reinterpret_cast<const float4 *>(tab));
  const Dual2<float> v[6] = {d.f, d.fp, d.F1, d.Iff, d.Ipp, d.IFF};
  for (int i = 0; i < 6; ++i) {
    out18[i] = v[i].v;
    out18[6 + i] = v[i].da;
    out18[12 + i] = v[i].db;
  }
}

// out18 = values (table path, FP32) and their (a, beta) tangents from the
// values (disc_tangents: table columns or the closed-form identities)
void hh_discretize_tangents(double t, double a, double beta, double *out18) {
  float tab[TAB_TERM];
  build_table((float)a, (float)beta, tab);
  const TermC<float> c = termc((float)a, (float)beta);
  const float4 *tb = reinterpret_cast<const float4 *>(tab);
  const Disc<float> d = discretize_tab((float)t, c, tb);
  float da[6], db[6];
  disc_tangents((float)t, c, tb, d, da, db);
  const float v[6] = {d.f, d.fp, d.F1, d.Iff, d.Ipp, d.IFF};
  for (int i = 0; i < 6; ++i) {
    out18[i] = v[i];
    out18[6 + i] = da[i];
    out18[12 + i] = db[i];
  }
}

// Economised table polynomials (FP64) against the TAB_NTAY-term Taylor
// series they replace, on 401 points of the table's range [0, T]: the worst
// error of any of the 18 series (6 values, d/da, d/dbeta) relative to that
// series' largest magnitude on the range; which = 0: the six values,
// 1: the twelve (a, beta) tangents.
double hh_table_check(double a, double beta, int which) {
  EconMap E;
  econ_map(E);
  Dual2<double> g[6][TAB_NTAY], e[6][TAB_NC];
  taylor_coeffs<Dual2<double>>(mk(a, 1.0, 0.0), mk(beta, 0.0, 1.0), g);
  table_coeffs<Dual2<double>>(E, mk(a, 1.0, 0.0), mk(beta, 0.0, 1.0), e);
  const double T = table_range(rate2<double>(a, beta));
  double worst = 0.0;
  for (int j = 0; j < 6; ++j)
    for (int q = which ? 1 : 0; q < (which ? 3 : 1); ++q) {
      auto comp = [q](const Dual2<double> &x) { return q == 0 ? x.v : (q == 1 ? x.da : x.db); };
      double mx = 0.0, err = 0.0;
      for (int i = 0; i <= 400; ++i) {
        const double t = T * i / 400.0;
        double r = 0.0, h = 0.0;
        for (int k = TAB_NTAY - 1; k >= 0; --k) r = r * t + comp(g[j][k]);
        for (int k = TAB_NC - 1; k >= 0; --k) h = h * t + comp(e[j][k]);
        mx = std::fmax(mx, std::fabs(r));
        err = std::fmax(err, std::fabs(h - r));
      }
      if (mx > 0.0) worst = std::fmax(worst, err / mx);
    }
  return worst;
}

float hh_solve(int D, const float *A, const float *B, float *X, int R) {
  switch (D) {
    case 3: return solve_d<3>(A, B, X, R);
    case 5: return solve_d<5>(A, B, X, R);
    case 6: return solve_d<6>(A, B, X, R);
    case 7: return solve_d<7>(A, B, X, R);
  }
  return 0.f;
}

// shape ids: 0 = (1 term, 1 slot), 1 = (2 terms, 1 slot, layout 1), 2 = (2 terms, 3 slots)
int hh_dim(int shape) {
  return shape == 0 ? Shape<1, 1, 0>::D : shape == 1 ? Shape<2, 1, 1>::D : Shape<2, 3, 0>::D;
}
void hh_combine(int shape, const float *Ei, const float *Ej, float *out) {
  if (shape == 0) combine_s<Shape<1, 1, 0>>(Ei, Ej, out);
  else if (shape == 1) combine_s<Shape<2, 1, 1>>(Ei, Ej, out);
  else combine_s<Shape<2, 3, 0>>(Ei, Ej, out);
}
double hh_chunk_loglik(int shape, const float *m, const float *P, const float *eta,
                       const float *J, double gam, double ld, double ne) {
  if (shape == 0) return chunk_ll_s<Shape<1, 1, 0>>(m, P, eta, J, gam, ld, ne);
  if (shape == 1) return chunk_ll_s<Shape<2, 1, 1>>(m, P, eta, J, gam, ld, ne);
  return chunk_ll_s<Shape<2, 3, 0>>(m, P, eta, J, gam, ld, ne);
}
void hh_boundary_adjoint(int shape, const float *m, const float *P, const float *eta,
                         const float *J, float *lam, float *Lam) {
  if (shape == 0) adj_s<Shape<1, 1, 0>>(m, P, eta, J, lam, Lam);
  else if (shape == 1) adj_s<Shape<2, 1, 1>>(m, P, eta, J, lam, Lam);
  else adj_s<Shape<2, 3, 0>>(m, P, eta, J, lam, Lam);
}

int hh_obs_dim(int shape) {
  return shape == 3 ? Shape<2, 0, 0>::D : shape == 4 ? Shape<2, 2, 0>::D : Shape<2, 1, 1>::D;
}
void hh_observe(int shape, int j, float w, const float *m, const float *Pf, const float *lam,
                const float *Lf, float *u, float *out4) {
  if (shape == 3) observe_s<Shape<2, 0, 0>>(j, w, m, Pf, lam, Lf, u, out4);
  else if (shape == 4) observe_s<Shape<2, 2, 0>>(j, w, m, Pf, lam, Lf, u, out4);
  else observe_s<Shape<2, 1, 1>>(j, w, m, Pf, lam, Lf, u, out4);
}

void hh_prod_disc(int prec, double dt, const double *th, double *Phi, double *Q) {
  if (prec == 64)
    prod_disc_t<double>(dt, th, Phi, Q);
  else
    prod_disc_t<float>(dt, th, Phi, Q);
}

// coefficient k of the six Taylor series: the division-free per-lane form
// the table kernel runs vs the full generator
double hh_taylor_k_check(double a, double beta) {
  using DD = Dual2<double>;
  DD g[6][TAB_NTAY];
  taylor_coeffs<DD>(mk(a, 1.0, 0.0), mk(beta, 0.0, 1.0), g);
  EconMap E;
  econ_map(E);
  DD c[TAB_NCF + 1], e[TAB_NCF + 1], p[TAB_NCF + 1];
  taylor_c<DD>(mk(a, 1.0, 0.0), mk(beta, 0.0, 1.0), E.rcp, c);
  for (int n = 0; n <= TAB_NCF; ++n) {
    e[n] = c[n] * E.rcp[n + 1];
    p[n] = c[n] * (double)n;
  }
  // error of every coefficient relative to the largest coefficient of the
  // same series and component (cancelling sums can leave exact zeros)
  double worst = 0.0, mx[6][3] = {};
  for (int k = 0; k < TAB_NTAY; ++k)
    for (int j = 0; j < 6; ++j) {
      mx[j][0] = std::fmax(mx[j][0], std::fabs(g[j][k].v));
      mx[j][1] = std::fmax(mx[j][1], std::fabs(g[j][k].da));
      mx[j][2] = std::fmax(mx[j][2], std::fabs(g[j][k].db));
    }
  for (int k = 0; k < TAB_NTAY; ++k) {
    DD h[6];
    taylor_coeff_pre<DD>(c, e, p, E.rcp, k, h);
    for (int j = 0; j < 6; ++j) {
      const double d[3] = {h[j].v - g[j][k].v, h[j].da - g[j][k].da, h[j].db - g[j][k].db};
      for (int q = 0; q < 3; ++q)
        if (mx[j][q] > 0.0) worst = std::fmax(worst, std::fabs(d[q]) / mx[j][q]);
    }
  }
  return worst;
}

// The double-float table path the table kernel runs against the FP64 one:
// the largest difference of a coefficient, relative to the largest
// coefficient of the same series and component (values, d/da, d/dbeta).
double hh_table_df_check(double a, double beta) {
  EconMap E;
  econ_map(E);
  Dual2<double> g[6][TAB_NC];
  table_coeffs<Dual2<double>>(E, mk(a, 1.0, 0.0), mk(beta, 0.0, 1.0), g);
  static double v[6][TAB_NC], da[6][TAB_NC], db[6][TAB_NC];
  table_coeffs_df(E, a, beta, v, da, db);
  double worst = 0.0;
  for (int j = 0; j < 6; ++j) {
    double mx[3] = {0.0, 0.0, 0.0};
    for (int k = 0; k < TAB_NC; ++k) {
      mx[0] = std::fmax(mx[0], std::fabs(g[j][k].v));
      mx[1] = std::fmax(mx[1], std::fabs(g[j][k].da));
      mx[2] = std::fmax(mx[2], std::fabs(g[j][k].db));
    }
    for (int k = 0; k < TAB_NC; ++k) {
      const double d[3] = {v[j][k] - g[j][k].v, da[j][k] - g[j][k].da, db[j][k] - g[j][k].db};
      for (int q = 0; q < 3; ++q)
        if (mx[q] > 0.0) worst = std::fmax(worst, std::fabs(d[q]) / mx[q]);
    }
  }
  return worst;
}

// span shape ids: 0 = (1 term, 1 slot), 1 = (1 term, 3 slots), 2 = (2 terms,
// 3 slots), 3 = (2 terms, 1 slot, layout 1)
int hh_span_nc(int shape) {
  switch (shape) {
    case 0: return Elem<Shape<1, 1, 0>>::NF + 1;
    case 1: return Elem<Shape<1, 3, 0>>::NF + 1;
    case 2: return Elem<Shape<2, 3, 0>>::NF + 1;
  }
  return Elem<Shape<2, 1, 1>>::NF + 1;
}
void hh_span_element(int shape, const double *dt, const uint8_t *tag, const double *meas3,
                     const float *theta, const int *kinds, int64_t k_begin, int64_t k_end,
                     int chunk_len, double *out) {
  switch (shape) {
    case 0: span_elem_s<Shape<1, 1, 0>>(dt, tag, meas3, theta, kinds, k_begin, k_end, chunk_len, out); break;
    case 1: span_elem_s<Shape<1, 3, 0>>(dt, tag, meas3, theta, kinds, k_begin, k_end, chunk_len, out); break;
    case 2: span_elem_s<Shape<2, 3, 0>>(dt, tag, meas3, theta, kinds, k_begin, k_end, chunk_len, out); break;
    default: span_elem_s<Shape<2, 1, 1>>(dt, tag, meas3, theta, kinds, k_begin, k_end, chunk_len, out);
  }
}
double hh_span_fold(int shape, const double *elems, int n_spans) {
  switch (shape) {
    case 0: return span_fold_s<Shape<1, 1, 0>>(elems, n_spans);
    case 1: return span_fold_s<Shape<1, 3, 0>>(elems, n_spans);
    case 2: return span_fold_s<Shape<2, 3, 0>>(elems, n_spans);
  }
  return span_fold_s<Shape<2, 1, 1>>(elems, n_spans);
}

// Covariance prediction in FP64: P (packed upper triangle of the shape's
// state) <- Phi~ P Phi~^T + Q~ with the blocks of each term given as 12
// doubles (p00 p01 p10 p11 pb0 pb1 q00 q01 q11 qz0 qz1 qzz).  Shape ids: 0 =
// (1 term, 1 slot), 1 = (1 term, 3 slots), 2 = (2 terms, 1 slot, layout 1),
// 3 = (2 terms, 3 slots), 4 = (2 terms, 2 slots), 5 = (2 terms, no slot).
void hh_predict_cov(int shape, const double *blocks, double *P) {
  auto run = [&](auto tag) {
    using S = decltype(tag);
    Blocks<double> B[S::NT];
    for (int t = 0; t < S::NT; ++t) {
      const double *b = blocks + 12 * t;
      B[t] = Blocks<double>{b[0], b[1], b[2], b[3], b[4], b[5], b[6], b[7], b[8], b[9], b[10], b[11]};
    }
    predict_cov<S, double>(B, P);
  };
  switch (shape) {
    case 0: run(Shape<1, 1, 0>{}); break;
    case 1: run(Shape<1, 3, 0>{}); break;
    case 2: run(Shape<2, 1, 1>{}); break;
    case 3: run(Shape<2, 3, 0>{}); break;
    case 4: run(Shape<2, 2, 0>{}); break;
    case 5: run(Shape<2, 0, 0>{}); break;
  }
}

}  // extern "C"
