// Product kernels (Appendix C.2) on instantaneous measurements.
//
// A product of two SHO terms, k = sigma^2 k_a k_b with unit-variance factors
// (parameters sigma, omega_a, Q_a, omega_b, Q_b), is the state-space model
// with F = F_a (x) I + I (x) F_b, P_inf = P_inf,a (x) P_inf,b and observation
// H = H_a (x) H_b = e_0; its transition is Phi_a (x) Phi_b and its process
// noise Q = P_inf,a (x) Q_b + Q_a (x) P_inf,b - Q_a (x) Q_b (Eq. product_Q),
// all from the two factors' per-step scalars (f, f', I_ff, I_pp; see
// gpss_device.cuh).  Optionally a second, plain SHO / Matern-3/2 term is
// added (state 4 + 2).  The state dimension grows as the product of the
// factors' (Section C.2), so the covariance is kept dense: the FP32
// log-likelihood runs in parallel in time (k_elem_prod forms dense chunk
// elements, the dimension-generic combination of a same-size shape does the
// rest), the plain sequential filter (one thread per series) serves FP64 and
// schedule 3, and the hyperparameter gradient comes from forward-mode tangents:
// per chunk and parameter against the combination's boundary adjoints
// (k_prod_grad_chunk, the chunked schedule), or per series and parameter
// (k_prod_grad, schedule 3).
#pragma once

#include <type_traits>

#include "gpss_kernels.cuh"

namespace gpss {

// The 2 x 2 transition and process noise of one oscillator factor of
// variance var from its six per-step scalars (Eqs. sho_phi, Q).  T is F, or
// Dual2<F> carrying one parameter tangent in .da (forward-mode gradient).
template <class T>
struct Osc2 {
  T p[2][2], q[2][2];
};

template <class T, class F>
GPSS_HD Osc2<T> osc2(F dt, T w0, T Q, T var) {
  const T a = w0 / (F(2) * Q);
  const T beta = (val(Q) == F(0.5)) ? cst<T>(F(0))
                                    : w0 * w0 * (F(1) - cst<T>(F(1)) / (F(4) * Q * Q));
  const Disc<T> d = discretize<T, F, true>(dt, a, beta);
  const T qc = F(2) * w0 * w0 * w0 * var / Q;
  Osc2<T> o;
  o.p[0][0] = d.fp + F(2) * a * d.f;
  o.p[0][1] = d.f;
  o.p[1][0] = -(w0 * w0 * d.f);
  o.p[1][1] = d.fp;
  o.q[0][0] = qc * d.Iff;
  o.q[0][1] = o.q[1][0] = qc * d.f * d.f * F(0.5);
  o.q[1][1] = qc * d.Ipp;
  return o;
}

// One thread per (parameter set, series).  Parameter row: (sigma, omega_a,
// Q_a, omega_b, Q_b) of the product, then (sigma, omega0, Q) or (sigma, ell)
// of the plain term when SUM, then the white-noise sd.
template <bool SUM, class F>
__global__ void __launch_bounds__(128) k_plain_prod(DevModel M, const float *__restrict__ theta,
                                                    int n_out, int per_series,
                                                    double *__restrict__ ll_out,
                                                    int *__restrict__ err) {
  constexpr int D = SUM ? 6 : 4;
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n_out) return;
  const int s = per_series ? v : v % M.n_series;
  const int row = per_series ? v : v / M.n_series;
  const float *th = theta + (size_t)row * M.n_params;
  const F sig = th[0], wa = th[1], qa = th[2], wb = th[3], qb = th[4];
  const F var = sig * sig;
  const F Pa[2] = {F(1), wa * wa}, Pb[2] = {var, var * wb * wb};
  F sc = F(0), wc = F(1), qcq = F(0.5);
  int j = 5;
  if constexpr (SUM) {
    sc = th[5];
    if (M.kinds[1] == 1) {
      wc = th[6];
      qcq = th[7];
      j = 8;
    } else {
      wc = F(1.7320508075688772) / F(th[6]);
      j = 7;
    }
  }
  const F s2 = F(th[j]) * F(th[j]);
  // P0 = blkdiag(P_inf,a (x) P_inf,b, P_inf,c); m0 = 0
  F m[D], P[D][D];
#pragma unroll
  for (int i = 0; i < D; ++i) {
    m[i] = F(0);
#pragma unroll
    for (int c = 0; c < D; ++c) P[i][c] = F(0);
  }
#pragma unroll
  for (int ra = 0; ra < 2; ++ra)
#pragma unroll
    for (int rb = 0; rb < 2; ++rb) P[2 * ra + rb][2 * ra + rb] = Pa[ra] * Pb[rb];
  if constexpr (SUM) {
    P[4][4] = sc * sc;
    P[5][5] = sc * sc * wc * wc;
  }
  double sum_logS = 0.0, sum_q = 0.0;
  int64_t n_end = 0;
  bool bad = false;
  int64_t mi = M.meas_off[s];
  const int64_t e1 = M.ev_off[s + 1];
  for (int64_t k = M.ev_off[s]; k < e1; ++k) {
    const F dt = load_dt<F>(M, k);
    F y, r0, w;
    load_meas<F>(M, mi, y, r0, w);
    ++mi;
    const Osc2<F> A = osc2<F, F>(dt, wa, qa, F(1));
    const Osc2<F> B = osc2<F, F>(dt, wb, qb, var);
    // Phi (block-diagonal: the product's Kronecker block, then the plain term)
    F Phi[D][D], Qd[D][D];
#pragma unroll
    for (int r = 0; r < D; ++r)
#pragma unroll
      for (int c = 0; c < D; ++c) Phi[r][c] = Qd[r][c] = F(0);
#pragma unroll
    for (int ra = 0; ra < 2; ++ra)
#pragma unroll
      for (int rb = 0; rb < 2; ++rb)
#pragma unroll
        for (int ca = 0; ca < 2; ++ca)
#pragma unroll
          for (int cb = 0; cb < 2; ++cb) {
            const int r = 2 * ra + rb, c = 2 * ca + cb;
            Phi[r][c] = A.p[ra][ca] * B.p[rb][cb];
            // Eq. product_Q: P_inf,a (x) Q_b + Q_a (x) P_inf,b - Q_a (x) Q_b
            Qd[r][c] = (ra == ca ? Pa[ra] * B.q[rb][cb] : F(0)) +
                       (rb == cb ? A.q[ra][ca] * Pb[rb] : F(0)) - A.q[ra][ca] * B.q[rb][cb];
          }
    if constexpr (SUM) {
      const Osc2<F> C = osc2<F, F>(dt, wc, qcq, sc * sc);
#pragma unroll
      for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          Phi[4 + r][4 + c] = C.p[r][c];
          Qd[4 + r][4 + c] = C.q[r][c];
        }
    }
    // predict: m <- Phi m, P <- Phi P Phi^T + Q
    F mt[D], T[D][D];
#pragma unroll
    for (int r = 0; r < D; ++r) {
      F acc = F(0);
#pragma unroll
      for (int c = 0; c < D; ++c) acc += Phi[r][c] * m[c];
      mt[r] = acc;
#pragma unroll
      for (int c = 0; c < D; ++c) {
        F a2 = F(0);
#pragma unroll
        for (int e = 0; e < D; ++e) a2 += Phi[r][e] * P[e][c];
        T[r][c] = a2;
      }
    }
#pragma unroll
    for (int r = 0; r < D; ++r) {
      m[r] = mt[r];
#pragma unroll
      for (int c = r; c < D; ++c) {
        F a2 = Qd[r][c];
#pragma unroll
        for (int e = 0; e < D; ++e) a2 += T[r][e] * Phi[c][e];
        P[r][c] = a2;
        P[c][r] = a2;
      }
    }
    // update with h = e_0 (+ e_4): the latent f(t) of the product (and term)
    F u[D], hu = F(0), hm = m[0] + (SUM ? m[4] : F(0));
#pragma unroll
    for (int r = 0; r < D; ++r) u[r] = P[r][0] + (SUM ? P[r][4] : F(0));
    hu = u[0] + (SUM ? u[4] : F(0));
    const F Sv = hu + r0 + s2;
    const F vv = y - hm;
    bad |= !(Sv > F(0));
    const F iS = F(1) / Sv;
#pragma unroll
    for (int r = 0; r < D; ++r) {
      m[r] += u[r] * vv * iS;
#pragma unroll
      for (int c = 0; c < D; ++c) P[r][c] -= u[r] * u[c] * iS;
    }
    sum_logS += glog(Sv);
    sum_q += (double)(vv * vv / Sv);
    ++n_end;
  }
  const double ll = -0.5 * ((double)n_end * LOG_2PI + sum_logS + sum_q);
  bad |= !isfinite(ll);
  ll_out[v] = ll;
  if (bad) flag_error(err, v, 7);
}

// Forward-mode gradient of the product filter: the filter runs in
// Dual2<float> with d/d theta_i in .da, and d loglik / d theta_i accumulates
// -1/2 sum (dS/S + 2 v dv / S - v^2 dS / S^2) in FP64.
template <class T>
GPSS_D T seed(float v, bool on);
template <>
GPSS_D Dual2<float> seed<Dual2<float>>(float v, bool on) { return mk(v, on ? 1.f : 0.f, 0.f); }

// The product model's parameters as duals, parameter ip seeded (row layout as
// for k_plain_prod).
template <bool SUM>
struct ProdPar {
  using T = Dual2<float>;
  T wa, qa, wb, qb, var, sc, wc, qcq, s2;
};

template <bool SUM>
GPSS_D ProdPar<SUM> prod_par(const DevModel &M, const float *th, int ip) {
  using F = float;
  using T = Dual2<F>;
  auto par = [&](int i) { return seed<T>(th[i], i == ip); };
  ProdPar<SUM> p;
  const T sig = par(0);
  p.wa = par(1);
  p.qa = par(2);
  p.wb = par(3);
  p.qb = par(4);
  p.var = sig * sig;
  p.sc = cst<T>(F(0));
  p.wc = cst<T>(F(1));
  p.qcq = cst<T>(F(0.5));
  int j = 5;
  if constexpr (SUM) {
    p.sc = par(5);
    if (M.kinds[1] == 1) {
      p.wc = par(6);
      p.qcq = par(7);
      j = 8;
    } else {
      p.wc = cst<T>(F(1.7320508075688772)) / par(6);
      j = 7;
    }
  }
  const T sw = par(j);
  p.s2 = sw * sw;
  return p;
}

// Stationary prior of the product state (P_inf,a (x) P_inf,b; the plain term's
// block when SUM), zero mean.
template <bool SUM>
GPSS_D void prod_prior(const ProdPar<SUM> &p, Dual2<float> (*m), Dual2<float> (*P)[SUM ? 6 : 4]) {
  using F = float;
  using T = Dual2<F>;
  constexpr int D = SUM ? 6 : 4;
  const T one = cst<T>(F(1));
  const T Pa[2] = {one, p.wa * p.wa}, Pb[2] = {p.var, p.var * p.wb * p.wb};
#pragma unroll
  for (int i = 0; i < D; ++i) {
    m[i] = cst<T>(F(0));
#pragma unroll
    for (int c = 0; c < D; ++c) P[i][c] = cst<T>(F(0));
  }
#pragma unroll
  for (int ra = 0; ra < 2; ++ra)
#pragma unroll
    for (int rb = 0; rb < 2; ++rb) P[2 * ra + rb][2 * ra + rb] = Pa[ra] * Pb[rb];
  if constexpr (SUM) {
    P[4][4] = p.sc * p.sc;
    P[5][5] = p.sc * p.sc * p.wc * p.wc;
  }
}

// One event (instantaneous measurement y with variance r0) of the dual
// product filter on the dense (m, P); adds log S + v^2/S and its tangent.
template <bool SUM>
GPSS_D void prod_event(const ProdPar<SUM> &p, float dt, float y, float r0, Dual2<float> *m,
                       Dual2<float> (*P)[SUM ? 6 : 4], double &sum_ll, double &sum_d, bool &bad) {
  using F = float;
  using T = Dual2<F>;
  constexpr int D = SUM ? 6 : 4;
  const T one = cst<T>(F(1));
  const T Pa[2] = {one, p.wa * p.wa}, Pb[2] = {p.var, p.var * p.wb * p.wb};
  const Osc2<T> A = osc2<T, F>(dt, p.wa, p.qa, one);
  const Osc2<T> B = osc2<T, F>(dt, p.wb, p.qb, p.var);
  T Phi[D][D], Qd[D][D];
#pragma unroll
  for (int r = 0; r < D; ++r)
#pragma unroll
    for (int c = 0; c < D; ++c) Phi[r][c] = Qd[r][c] = cst<T>(F(0));
#pragma unroll
  for (int ra = 0; ra < 2; ++ra)
#pragma unroll
    for (int rb = 0; rb < 2; ++rb)
#pragma unroll
      for (int ca = 0; ca < 2; ++ca)
#pragma unroll
        for (int cb = 0; cb < 2; ++cb) {
          const int r = 2 * ra + rb, c = 2 * ca + cb;
          Phi[r][c] = A.p[ra][ca] * B.p[rb][cb];
          T q = -(A.q[ra][ca] * B.q[rb][cb]);  // Eq. product_Q
          if (ra == ca) q = q + Pa[ra] * B.q[rb][cb];
          if (rb == cb) q = q + A.q[ra][ca] * Pb[rb];
          Qd[r][c] = q;
        }
  if constexpr (SUM) {
    const Osc2<T> C = osc2<T, F>(dt, p.wc, p.qcq, p.sc * p.sc);
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        Phi[4 + r][4 + c] = C.p[r][c];
        Qd[4 + r][4 + c] = C.q[r][c];
      }
  }
  T mt[D], Tm[D][D];
#pragma unroll
  for (int r = 0; r < D; ++r) {
    T acc = cst<T>(F(0));
#pragma unroll
    for (int c = 0; c < D; ++c) acc = acc + Phi[r][c] * m[c];
    mt[r] = acc;
#pragma unroll
    for (int c = 0; c < D; ++c) {
      T a2 = cst<T>(F(0));
#pragma unroll
      for (int e = 0; e < D; ++e) a2 = a2 + Phi[r][e] * P[e][c];
      Tm[r][c] = a2;
    }
  }
#pragma unroll
  for (int r = 0; r < D; ++r) {
    m[r] = mt[r];
#pragma unroll
    for (int c = r; c < D; ++c) {
      T a2 = Qd[r][c];
#pragma unroll
      for (int e = 0; e < D; ++e) a2 = a2 + Tm[r][e] * Phi[c][e];
      P[r][c] = a2;
      P[c][r] = a2;
    }
  }
  T u[D];
#pragma unroll
  for (int r = 0; r < D; ++r) u[r] = SUM ? P[r][0] + P[r][4] : P[r][0];
  const T hu = SUM ? u[0] + u[4] : u[0];
  const T hm = SUM ? m[0] + m[4] : m[0];
  const T Sv = hu + p.s2 + r0;
  const T vv = y - hm;
  bad |= !(Sv.v > F(0));
  const T iS = one / Sv;
#pragma unroll
  for (int r = 0; r < D; ++r) {
    m[r] = m[r] + u[r] * vv * iS;
#pragma unroll
    for (int c = 0; c < D; ++c) P[r][c] = P[r][c] - u[r] * u[c] * iS;
  }
  const double S = Sv.v, dS = Sv.da, e = vv.v, de = vv.da;
  sum_ll += log(S) + e * e / S;
  sum_d += dS / S + 2.0 * e * de / S - e * e * dS / (S * S);
}

// One thread per (output row, parameter i) over the whole series (the plain
// schedule); the i = 0 thread also writes the log-likelihood.
template <bool SUM>
__global__ void __launch_bounds__(64) k_prod_grad(DevModel M, const float *__restrict__ theta,
                                                  int n_out, int per_series,
                                                  double *__restrict__ ll_out,
                                                  float *__restrict__ grad_out,
                                                  int *__restrict__ err) {
  using F = float;
  using T = Dual2<F>;
  constexpr int D = SUM ? 6 : 4;
  const int np = M.n_params;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= (int64_t)n_out * np) return;
  const int v = (int)(tid / np), ip = (int)(tid % np);
  const int s = per_series ? v : v % M.n_series;
  const int row = per_series ? v : v / M.n_series;
  const ProdPar<SUM> p = prod_par<SUM>(M, theta + (size_t)row * np, ip);
  T m[D], P[D][D];
  prod_prior<SUM>(p, m, P);
  double sum_ll = 0.0, sum_d = 0.0;
  int64_t n_end = 0;
  bool bad = false;
  int64_t mi = M.meas_off[s];
  const int64_t e1 = M.ev_off[s + 1];
  for (int64_t k = M.ev_off[s]; k < e1; ++k) {
    F y, r0, w;
    load_meas<F>(M, mi, y, r0, w);
    ++mi;
    prod_event<SUM>(p, load_dt<F>(M, k), y, r0, m, P, sum_ll, sum_d, bad);
    ++n_end;
  }
  const double ll = -0.5 * ((double)n_end * LOG_2PI + sum_ll);
  const double g = -0.5 * sum_d;
  bad |= !isfinite(ll) || !isfinite(g);
  grad_out[(size_t)v * np + ip] = (float)g;
  if (ip == 0) ll_out[v] = ll;
  if (bad) flag_error(err, v, 7);
}

// Chunked gradient of a product model: one thread per (chunk, parameter i).
// With the chunk's incoming filtered state s_in (from the parallel-in-time
// combination) held fixed, the log-likelihood splits as 𝓛 = sum_c 𝓛_c(s_in,c,
// theta), and by the chain rule over chunks
//   d𝓛/dtheta_i = sum_c [ d𝓛_c/dtheta_i + lam_c . dm_end,c/dtheta_i
//                         + sum_jk Lam_c[j,k] dP_end,c[j,k]/dtheta_i ],
// the derivatives taken through chunk c's own steps only, (lam_c, Lam_c) the
// adjoint of all later data's log-likelihood with respect to chunk c's end
// state (the combination's boundary adjoint; full-matrix convention).  The
// thread runs its chunk's filter in Dual2 from s_in (zero tangent; the prior,
// with its tangent, for a series' first chunk) and writes its part of
// d𝓛/dtheta_i; the per-series sums add the parts in chunk order.
template <bool SUM, class ES>
__global__ void __launch_bounds__(64) k_prod_grad_chunk(DevModel M, const float *__restrict__ theta,
                                                        int n_vch, int per_series,
                                                        const void *__restrict__ state_end, int se64,
                                                        const float *__restrict__ adj_end,
                                                        float *__restrict__ gpart,
                                                        int *__restrict__ err) {
  using F = float;
  using T = Dual2<F>;
  constexpr int D = SUM ? 6 : 4;
  static_assert(ES::D == D, "combination shape of the product's state size");
  const int np = M.n_params;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= (int64_t)n_vch * np) return;
  // the threads of one chunk are adjacent and read the same events
  const int vc = (int)(tid / np), ip = (int)(tid % np);
  const int c = vc % M.n_chunks, set = vc / M.n_chunks;
  const int s = M.ch_series[c];
  const int row = per_series ? s : set;
  const int orow = per_series ? s : set * M.n_series + s;
  const uint8_t flags = M.ch_flags[c];
  const ProdPar<SUM> p = prod_par<SUM>(M, theta + (size_t)row * np, ip);
  T m[D], P[D][D];
  if (flags & 1) {
    prod_prior<SUM>(p, m, P);
  } else {
    F mf[D], Pf[ES::NP];
    load_state_f<ES>(state_end, se64, n_vch, vc - 1, mf, Pf);
#pragma unroll
    for (int i = 0; i < D; ++i) {
      m[i] = cst<T>(mf[i]);
#pragma unroll
      for (int j = 0; j < D; ++j) P[i][j] = cst<T>(Pf[ES::pk(i, j)]);
    }
  }
  double sum_ll = 0.0, sum_d = 0.0;
  bool bad = false;
  int64_t mi = M.ch_meas0[c];
  const int64_t k0 = M.ch_ev0[c], k1 = k0 + M.ch_len[c];
  for (int64_t k = k0; k < k1; ++k) {
    F y, r0, w;
    load_meas<F>(M, mi, y, r0, w);
    ++mi;
    prod_event<SUM>(p, load_dt<F>(M, k), y, r0, m, P, sum_ll, sum_d, bad);
  }
  double g = -0.5 * sum_d;
  if (!(flags & 2)) {
    F lam[D], Lam[ES::NP];
    load_rec<ES>(adj_end, n_vch, vc, lam, Lam);
#pragma unroll
    for (int i = 0; i < D; ++i) {
      g += (double)lam[i] * (double)m[i].da;
#pragma unroll
      for (int j = i; j < D; ++j)
        g += (i == j ? 1.0 : 2.0) * (double)Lam[ES::pk(i, j)] * (double)P[i][j].da;
    }
  }
  bad |= !isfinite(g);
  gpart[(size_t)ip * n_vch + vc] = (float)g;
  if (bad) flag_error(err, orow, 7);
}

template <bool SUM>
cudaError_t launch_prod_grad(const DevModel &M, const float *theta, int n_out, int per_series,
                             double *ll, float *grad, int *err, cudaStream_t st) {
  if (n_out <= 0) return cudaSuccess;
  const int bs = 64;
  const int64_t nt = (int64_t)n_out * M.n_params;
  k_prod_grad<SUM><<<(unsigned)((nt + bs - 1) / bs), bs, 0, st>>>(M, theta, n_out, per_series, ll,
                                                                 grad, err);
  GPSS_COUNT_LAUNCH();
  return cudaGetLastError();
}

template <bool SUM, class ES>
cudaError_t launch_prod_grad_chunk(const DevModel &M, const float *theta, int n_vch, int per_series,
                                   const void *state_end, int se64, const float *adj_end,
                                   float *gpart, int *err, cudaStream_t st) {
  if (n_vch <= 0) return cudaSuccess;
  const int bs = 64;
  const int64_t nt = (int64_t)n_vch * M.n_params;
  k_prod_grad_chunk<SUM, ES><<<(unsigned)((nt + bs - 1) / bs), bs, 0, st>>>(
      M, theta, n_vch, per_series, state_end, se64, adj_end, gpart, err);
  GPSS_COUNT_LAUNCH();
  return cudaGetLastError();
}

template <bool SUM, class F>
cudaError_t launch_plain_prod(const DevModel &M, const float *theta, int n_out, int per_series,
                              double *ll, int *err, cudaStream_t st) {
  if (n_out <= 0) return cudaSuccess;
  const int bs = 128;
  k_plain_prod<SUM, F><<<(n_out + bs - 1) / bs, bs, 0, st>>>(M, theta, n_out, per_series, ll, err);
  GPSS_COUNT_LAUNCH();
  return cudaGetLastError();
}

// Chunk elements of a product model (the parallel-in-time log-likelihood,
// Section 3.2.5 with the SG21 elements): as k_elem, with the dense
// Kronecker-structured transition and noise of the product (and the plain
// term).  The combination, the chunk log-likelihoods and the per-series sums
// depend on the state dimension only, so the kernels of a shape with the
// same dimension (ES) serve them.
template <bool SUM, class ES>
__global__ void __launch_bounds__(128) k_elem_prod(DevModel M, const float *__restrict__ theta,
                                                   int n_vch, int per_series,
                                                   float *__restrict__ ef, double *__restrict__ ed,
                                                   int *__restrict__ err, int c_begin,
                                                   int c_count) {
  using F = float;
  constexpr int D = SUM ? 6 : 4;
  static_assert(ES::D == D, "element shape of the product state");
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= (n_vch / M.n_chunks) * c_count) return;
  const int set = l / c_count;
  const int c = c_begin + l % c_count;
  const int vc = set * M.n_chunks + c;
  const int s = M.ch_series[c];
  const int row = per_series ? s : set;
  const int orow = per_series ? s : set * M.n_series + s;
  const float *th = theta + (size_t)row * M.n_params;
  const F sig = th[0], wa = th[1], qa = th[2], wb = th[3], qb = th[4];
  const F var = sig * sig;
  const F Pa[2] = {F(1), wa * wa}, Pb[2] = {var, var * wb * wb};
  F sc = F(0), wc = F(1), qcq = F(0.5);
  int j = 5;
  if constexpr (SUM) {
    sc = th[5];
    if (M.kinds[1] == 1) {
      wc = th[6];
      qcq = th[7];
      j = 8;
    } else {
      wc = F(1.7320508075688772) / F(th[6]);
      j = 7;
    }
  }
  const F s2 = F(th[j]) * F(th[j]);
  const bool first = M.ch_flags[c] & 1;
  // element: A (D x D), b, C (full here, packed on store), eta, J (full)
  F A[D][D], b[D], C[D][D], eta[D], J[D][D];
#pragma unroll
  for (int i = 0; i < D; ++i) {
    b[i] = F(0);
    eta[i] = F(0);
#pragma unroll
    for (int k = 0; k < D; ++k) {
      A[i][k] = (!first && i == k) ? F(1) : F(0);
      C[i][k] = F(0);
      J[i][k] = F(0);
    }
  }
  if (first) {  // the series' first chunk starts from the prior
#pragma unroll
    for (int ra = 0; ra < 2; ++ra)
#pragma unroll
      for (int rb = 0; rb < 2; ++rb) C[2 * ra + rb][2 * ra + rb] = Pa[ra] * Pb[rb];
    if constexpr (SUM) {
      C[4][4] = sc * sc;
      C[5][5] = sc * sc * wc * wc;
    }
  }
  double gam = 0.0, ld = 0.0;
  int n_end = 0;
  bool bad = false;
  const int64_t e0 = M.ch_ev0[c];
  const int len = M.ch_len[c];
  int64_t mi = M.ch_meas0[c];
  for (int kk = 0; kk < len; ++kk) {
    const F dt = __ldg(M.dt + e0 + kk);
    const float4 q = __ldg(M.meas + mi);
    ++mi;
    const Osc2<F> Ao = osc2<F, F>(dt, wa, qa, F(1));
    const Osc2<F> Bo = osc2<F, F>(dt, wb, qb, var);
    F Phi[D][D], Qd[D][D];
#pragma unroll
    for (int r = 0; r < D; ++r)
#pragma unroll
      for (int cc = 0; cc < D; ++cc) Phi[r][cc] = Qd[r][cc] = F(0);
#pragma unroll
    for (int ra = 0; ra < 2; ++ra)
#pragma unroll
      for (int rb = 0; rb < 2; ++rb)
#pragma unroll
        for (int ca = 0; ca < 2; ++ca)
#pragma unroll
          for (int cb = 0; cb < 2; ++cb) {
            const int r = 2 * ra + rb, cc = 2 * ca + cb;
            Phi[r][cc] = Ao.p[ra][ca] * Bo.p[rb][cb];
            Qd[r][cc] = (ra == ca ? Pa[ra] * Bo.q[rb][cb] : F(0)) +
                        (rb == cb ? Ao.q[ra][ca] * Pb[rb] : F(0)) - Ao.q[ra][ca] * Bo.q[rb][cb];
          }
    if constexpr (SUM) {
      const Osc2<F> Co = osc2<F, F>(dt, wc, qcq, sc * sc);
#pragma unroll
      for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int cc = 0; cc < 2; ++cc) {
          Phi[4 + r][4 + cc] = Co.p[r][cc];
          Qd[4 + r][4 + cc] = Co.q[r][cc];
        }
    }
    // A <- Phi A, b <- Phi b, C <- Phi C Phi^T + Q
    F T1[D][D], T2[D][D], bt[D];
#pragma unroll
    for (int r = 0; r < D; ++r) {
      F acc = F(0);
#pragma unroll
      for (int e = 0; e < D; ++e) acc += Phi[r][e] * b[e];
      bt[r] = acc;
#pragma unroll
      for (int cc = 0; cc < D; ++cc) {
        F a1 = F(0), a2 = F(0);
#pragma unroll
        for (int e = 0; e < D; ++e) {
          a1 += Phi[r][e] * A[e][cc];
          a2 += Phi[r][e] * C[e][cc];
        }
        T1[r][cc] = a1;
        T2[r][cc] = a2;
      }
    }
#pragma unroll
    for (int r = 0; r < D; ++r) {
      b[r] = bt[r];
#pragma unroll
      for (int cc = 0; cc < D; ++cc) A[r][cc] = T1[r][cc];
#pragma unroll
      for (int cc = r; cc < D; ++cc) {
        F a2 = Qd[r][cc];
#pragma unroll
        for (int e = 0; e < D; ++e) a2 += T2[r][e] * Phi[cc][e];
        C[r][cc] = a2;
        C[cc][r] = a2;
      }
    }
    // update with h = e_0 (+ e_4): the latent of the product (and term)
    const F y = q.x, r0 = q.y;
    F u[D], g[D];
#pragma unroll
    for (int r = 0; r < D; ++r) {
      u[r] = C[r][0] + (SUM ? C[r][4] : F(0));
      g[r] = A[0][r] + (SUM ? A[4][r] : F(0));  // h^T A
    }
    const F hu = u[0] + (SUM ? u[4] : F(0));
    const F hb = b[0] + (SUM ? b[4] : F(0));
    const F Sv = hu + r0 + s2;
    const F cc = y - hb;
    bad |= !(Sv > F(0));
    const F iS = F(1) / Sv;
    const F ci = cc * iS;
#pragma unroll
    for (int r = 0; r < D; ++r) {
      eta[r] += g[r] * ci;
#pragma unroll
      for (int k = 0; k < D; ++k) J[r][k] += g[r] * g[k] * iS;
    }
    gam += (double)(cc * ci);
    ld += glog(Sv);
    ++n_end;
#pragma unroll
    for (int r = 0; r < D; ++r) {
      const F Kr = u[r] * iS;
#pragma unroll
      for (int k = 0; k < D; ++k) A[r][k] -= Kr * g[k];
      b[r] += Kr * cc;
#pragma unroll
      for (int k = 0; k < D; ++k) C[r][k] -= u[r] * u[k] * iS;
    }
  }
  F Cp[ES::NP], Jp[ES::NP];
#pragma unroll
  for (int r = 0; r < D; ++r)
#pragma unroll
    for (int k = r; k < D; ++k) {
      Cp[ES::pk(r, k)] = C[r][k];
      Jp[ES::pk(r, k)] = J[r][k];
    }
  store_elem<ES>(ef, n_vch, vc, A, b, Cp, eta, Jp);
  ed[vc] = gam;
  ed[(size_t)n_vch + vc] = ld;
  ed[(size_t)2 * n_vch + vc] = (double)n_end;
  if (bad) flag_error(err, orow, 7);
}

template <bool SUM, class ES>
cudaError_t launch_elem_prod(const DevModel &M, const float *theta, int n_vch, int per_series,
                             float *ef, double *ed, int *err, const float *, float *, int, float *,
                             int c_begin, int c_count, cudaStream_t st) {
  if (n_vch <= 0 || c_count <= 0) return cudaSuccess;
  if (c_begin < 0 || c_begin + c_count > M.n_chunks) return cudaErrorInvalidValue;
  const int bs = 128;
  const int64_t nt = (int64_t)(n_vch / M.n_chunks) * c_count;
  k_elem_prod<SUM, ES><<<(unsigned)((nt + bs - 1) / bs), bs, 0, st>>>(
      M, theta, n_vch, per_series, ef, ed, err, c_begin, c_count);
  GPSS_COUNT_LAUNCH();
  return cudaGetLastError();
}

// A product model has no step-scalar tables (its factors are discretised on
// the fly).
inline cudaError_t no_tables(const float *, int, int, int, int, float *, cudaStream_t) {
  return cudaSuccess;
}

// Operation table of a product model: the plain filters, the forward-mode
// gradient, and the chunked log-likelihood (dense product elements, then the
// combination and chunk log-likelihoods of the shape ES of the same state
// dimension; its FP64 combination is filled by make_ops_c64 like the others).
template <bool SUM>
OpTable make_prod_ops() {
  using ES = typename std::conditional<SUM, Shape<3, 0, 0>, Shape<2, 0, 0>>::type;
  OpTable o{};
  o.D = ES::D;
  o.NP = ES::NP;
  o.NF = ElemLayout<ES>::NF;
  o.ND = ElemLayout<ES>::ND;
  o.NT = 1;  // tables unused; keeps the table scratch small
  o.plain32 = &launch_plain_prod<SUM, float>;
  o.plain64 = &launch_plain_prod<SUM, double>;
  o.prod_grad = &launch_prod_grad<SUM>;
  o.prod_grad_chunk = &launch_prod_grad_chunk<SUM, ES>;
  o.tables = &no_tables;
  o.elem = &launch_elem_prod<SUM, ES>;
  o.comb32 = make_combine<ES, float>();
  o.span_element = &launch_span_element<ES>;
  o.span_scratch = &span_scratch_count<ES>;
  o.span_fold = &launch_span_fold<ES>;
  return o;
}

}  // namespace gpss
