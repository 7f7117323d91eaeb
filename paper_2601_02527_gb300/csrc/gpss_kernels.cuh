// Kernels of the integrated-measurement GP log-likelihood (arXiv 2601.02527).
//
// Event stream (built on the host, Section 3.2): per series 2N events in time
// order (N for a series of instantaneous measurements, which observe the
// latent and need no integral state); per event a gap dt (FP32, formed in
// FP64) and a tag byte (bit 0: measurement, bits 1-3: slot); per measurement,
// in event order, a float4 (y, yerr^2, 1/delta, 0).
//
// Schedules
//  * k_plain  -- one thread per series runs the whole sequential filter
//                (Eqs. integrated_kalman_pred/update, loglikelihood).  The FP64
//                instantiation is the plain FP64 GPU baseline.
//  * chunked parallel-in-time (Section 3.2.5, with the associative elements of
//    Sarkka & Garcia-Fernandez 2021):
//      k_elem     one thread per chunk of events; runs the filter from an
//                 unknown incoming state x, keeping the mean as M x + b, the
//                 covariance C, the information (eta, J) about x and the
//                 scalars gamma = sum c^2/S, sum log S.  That is the chunk's
//                 5-tuple element; the first chunk of a series starts from
//                 the prior instead (M = 0), like Eq. parallel_ikf_first.
//      k_scan_seq combines elements across the chunks of a series: the
//                 filtered state entering each chunk, each chunk's marginal
//                 log-likelihood in closed form, and for the gradient the
//                 information about each chunk's end state from all later
//                 data, turned into the adjoint of that state.
//      k_grad     one thread per chunk, segments of ck events from last to
//                 first: the segment's starting state from the partial
//                 element k_elem saved there and the chunk's incoming state,
//                 a forward replay of the segment, then a sweep back in time
//                 accumulating d loglik / d theta.
#pragma once

#include "gpss_device.cuh"
#include "gpss_scan.cuh"

namespace gpss {

constexpr double LOG_2PI = 1.8378770664093454836;

struct DevModel {
  int n_series;
  int n_params;
  int n_terms;
  int kinds[4];
  const int64_t *ev_off;    // [n_series+1]
  const int64_t *meas_off;  // [n_series+1]
  int64_t n_events;         // all series
  const float *dt;          // [n_events]
  const uint8_t *tag;       // [n_events]
  const float4 *meas;       // [n_meas] (y, yerr^2, 1/delta, 0)
  const double *dt64;       // FP64 copies (plain FP64 path only; may be null)
  const double *meas64;     // [3 * n_meas]
  // chunk plan
  int n_chunks;              // physical chunks (one theta set)
  const int64_t *ch_ev0;     // first event of chunk
  const int64_t *ch_meas0;   // first measurement (end event) index of chunk
  const int32_t *ch_len;     // events in chunk
  const int32_t *ch_series;  // series of chunk
  const uint8_t *ch_flags;   // bit0 first chunk of its series, bit1 last
  const int32_t *ch_first;   // [n_series+1] first chunk of each series
  // step-scalar cache layout: warp w of chunks (32 consecutive chunks, one
  // series) owns lane-steps [w_doff[w], w_doff[w+1]) of each theta set's
  // dcache_steps; the record of step k is DcW<NT>::G float4 groups x 32 lanes
  const int64_t *w_doff;
  int64_t dcache_steps;
  // the event stream re-laid out for the chunk kernels, in the lane-step
  // order of the step-scalar cache: step k of the chunk on lane l of warp w
  // at w_doff[w] + 32 k + l; record (dt, y, yerr^2, 1/delta) (zeros but dt
  // at an exposure start) and its tag byte.  A warp's loads of one step are
  // one 512-byte and one 32-byte contiguous access.
  const float4 *ilv;
  const uint8_t *ilv_tag;
  // nonzero: instantaneous measurements (TAG_INSTANT) among exposure averages;
  // every row then runs the kernels' general bodies, which read that bit
  int mixed;
};

// Lane-step index of step k of chunk c.
GPSS_D int64_t lane_step(const DevModel &M, int c, int k) {
  return M.w_doff[c >> 5] + (int64_t)k * 32 + (c & 31);
}

// Test times of a prediction call, grouped by the event that closes their
// interval: points [off[e], off[e+1]) lie in (t_{e-1}, t_e] of event e's
// series (or before its first event); points [xoff[s], xoff[s+1]) lie after
// series s's last event.  d = (t* - t_prev, t_next - t*) (FP32 of FP64
// differences; t* - t_last for the latter), idx = the point's index in the
// caller's order; out [rows * n_star * 2].  off == nullptr: no prediction.
struct PredPlan {
  const int *off = nullptr, *xoff = nullptr, *idx = nullptr;
  const float2 *d = nullptr;
  float *out = nullptr;
  int64_t n_star = 0;
};

// Step-scalar cache record: the 6 NT scalars of a step (term-major, in Disc
// order) padded to whole float4 groups, one float4 per lane per group.
template <int NT>
struct DcW {
  static constexpr int G = (6 * NT + 3) / 4;
  static constexpr int W = 4 * G;
};

// This chunk's column of the step-scalar cache (null when there is none):
// group v of step k at [k * 32 G + 32 v] (float4 units).
template <int NT>
GPSS_D float4 *dcache_col(const DevModel &M, float *dcache, int vc) {
  if (!dcache) return nullptr;
  const int c = vc % M.n_chunks, set = vc / M.n_chunks;
  return reinterpret_cast<float4 *>(dcache) +
         ((size_t)set * M.dcache_steps + M.w_doff[c >> 5]) * DcW<NT>::G + (c & 31);
}

// Load / store one step's cached scalars (W floats) for this lane.
template <int NT>
GPSS_D void dcache_load(const float4 *rec, float (&x)[DcW<NT>::W]) {
#pragma unroll
  for (int v = 0; v < DcW<NT>::G; ++v) {
    const float4 q = __ldg(rec + 32 * v);
    x[4 * v] = q.x;
    x[4 * v + 1] = q.y;
    x[4 * v + 2] = q.z;
    x[4 * v + 3] = q.w;
  }
}

template <int NT>
GPSS_D Disc<float> dcache_term(const float (&x)[DcW<NT>::W], int t) {
  return Disc<float>{x[6 * t], x[6 * t + 1], x[6 * t + 2], x[6 * t + 3], x[6 * t + 4], x[6 * t + 5]};
}

// log of an innovation variance: computed at the filter's precision, summed in FP64
GPSS_HD double glog(float x) { return (double)logf(x); }
GPSS_HD double glog(double x) { return log(x); }

template <class F> GPSS_D F load_dt(const DevModel &M, int64_t k);
template <> GPSS_D float load_dt<float>(const DevModel &M, int64_t k) { return __ldg(M.dt + k); }
template <> GPSS_D double load_dt<double>(const DevModel &M, int64_t k) { return __ldg(M.dt64 + k); }

template <class F> GPSS_D void load_meas(const DevModel &M, int64_t i, F &y, F &r0, F &w);
template <> GPSS_D void load_meas<float>(const DevModel &M, int64_t i, float &y, float &r0, float &w) {
  const float4 q = __ldg(M.meas + i);
  y = q.x;
  r0 = q.y;
  w = q.z;
}
template <> GPSS_D void load_meas<double>(const DevModel &M, int64_t i, double &y, double &r0, double &w) {
  y = __ldg(M.meas64 + 3 * i);
  r0 = __ldg(M.meas64 + 3 * i + 1);
  w = __ldg(M.meas64 + 3 * i + 2);
}

// Compile-time tag selecting a kernel body with (true) or without (false) the
// overdamped-oscillator branches of the discretisation; the kernels test the
// row's terms once and run the matching body.
template <bool V>
struct OdTag {
  static constexpr bool value = V;
};

// One event of the sequential filter on (m, P); returns true for an end
// event, with S and v of its innovation.
// Per-step scalars of term t: from the warp's Taylor table when one is given
// (FP32 chunk kernels), else from the on-the-fly series (per-series kernels).
template <class F, bool OD>
GPSS_D Disc<F> disc_step(F dt, const TermC<F> &c, const float4 *tab) {
  if constexpr (sizeof(F) == sizeof(float)) {
    if (tab) return discretize_tab<OD>(dt, c, tab);
  }
  return discretize<F, F, OD>(dt, c.a, c.beta);
}

// One event of the sequential filter on (m, P) given its gap, tag and (for an
// exposure end) its measurement record; returns true for an end event, with
// S and v of its innovation.
template <class S, class F, bool MIX = false>
GPSS_D bool filter_blocks(const Blocks<F> *B, uint8_t tag, F y, F r0, F w, F s2, F *m, F *P,
                          F &Sv, F &v);

template <class S, class F, bool OD = true>
GPSS_D bool filter_step(F dt, uint8_t tag, F y, F r0, F w, const TermC<F> *tc, F s2, F *m, F *P,
                        F &Sv, F &v, const float4 *tab) {
  Blocks<F> B[S::NT];
#pragma unroll
  for (int t = 0; t < S::NT; ++t)
    B[t] = make_blocks(disc_step<F, OD>(dt, tc[t], tab ? tab + t * (TAB_TERM / 4) : nullptr), tc[t]);
  return filter_blocks<S, F, OD>(B, tag, y, r0, w, s2, m, P, Sv, v);
}

// The filter step given the step's blocks.  MIX: the tag may mark an
// instantaneous measurement among exposure averages.
template <class S, class F, bool MIX>
GPSS_D bool filter_blocks(const Blocks<F> *B, uint8_t tag, F y, F r0, F w, F s2, F *m, F *P,
                          F &Sv, F &v) {
  F mt[S::D];
  apply_phi<S>(B, m, mt);
#pragma unroll
  for (int i = 0; i < S::D; ++i) m[i] = mt[i];
  predict_cov<S>(B, P);
  const int j = (tag >> 1) & 7;
  if (!(tag & 1)) {
    reset_slot<S>(j, m, P);
    return false;
  }
  F u[S::D], hu, hm;
  obs_project_tag<S, F, MIX>(tag, w, m, P, u, hu, hm);
  Sv = hu + r0 + s2;
  v = y - hm;
  const F iS = F(1) / Sv;
  const F kv = v * iS;
#pragma unroll
  for (int i = 0; i < S::D; ++i) m[i] += u[i] * kv;
#pragma unroll
  for (int i = 0; i < S::D; ++i)
#pragma unroll
    for (int jj = i; jj < S::D; ++jj) P[S::pk(i, jj)] -= u[i] * u[jj] * iS;
  return true;
}

// Same, loading the event's data itself (per-series kernels).
template <class S, class F, bool OD = true>
GPSS_D bool filter_event(const DevModel &M, int64_t k, int64_t &mi, const TermC<F> *tc, F s2, F *m,
                         F *P, F &Sv, F &v, const float4 *tab = nullptr) {
  const F dt = load_dt<F>(M, k);
  const uint8_t tag = __ldg(M.tag + k);
  F y = F(0), r0 = F(0), w = F(0);
  if (tag & 1) {
    load_meas<F>(M, mi, y, r0, w);
    ++mi;
  }
  return filter_step<S, F, OD>(dt, tag, y, r0, w, tc, s2, m, P, Sv, v, tab);
}

// Event reader for the FP32 chunk kernels over the lane-step records: the
// next step's record and tag are loaded one step ahead of their use, so
// their latency overlaps the arithmetic of the current event.  The lanes of
// a warp read consecutive records (coalesced).
struct EventReader {
  const float4 *rec;
  const uint8_t *tg;
  int64_t idx;
  int k, kend;
  float4 r_n;
  uint8_t tag_n;
  // steps [k0, k1) of chunk c
  GPSS_D void start(const DevModel &M, int c, int k0, int k1) {
    rec = M.ilv;
    tg = M.ilv_tag;
    idx = lane_step(M, c, k0);
    k = k0;
    kend = k1;
    if (k < kend) {
      r_n = __ldg(rec + idx);
      tag_n = __ldg(tg + idx);
    }
  }
  // current event's gap, tag and measurement record (y, yerr^2, 1/delta, 0);
  // prefetches the following one
  GPSS_D void next(float &d, uint8_t &t, float4 &q) {
    d = r_n.x;
    t = tag_n;
    q = make_float4(r_n.y, r_n.z, r_n.w, 0.f);
    ++k;
    idx += 32;
    if (k < kend) {
      r_n = __ldg(rec + idx);
      tag_n = __ldg(tg + idx);
    }
  }
};

// Lay the event stream out in lane-step order (one warp per chunk, 128-thread
// blocks, after every change of the chunk plan or of the event stream):
// chunks [c_begin, c_begin + c_count).
__global__ void __launch_bounds__(128) k_interleave(DevModel M, int c_begin, int c_count,
                                                    float4 *__restrict__ ilv,
                                                    uint8_t *__restrict__ ilv_tag);

GPSS_D void flag_error(int *err, int row, int code) {
  if (err) atomicMax(err + row, code);
}

// Asynchronous 16-byte global -> shared copy through L2 (cp.async.cg,
// sm_80 and later), committed as groups; wait_group<N> returns once at most
// N of this thread's groups are still in flight, and the thread then sees
// its own copies.  Both addresses 16-byte aligned.
GPSS_D void cp_async16(float4 *sdst, const float4 *gsrc) {
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 800
  const unsigned a = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(a), "l"(gsrc) : "memory");
#else
  *sdst = *gsrc;
#endif
}
GPSS_D void cp_async_commit() {
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 800
  asm volatile("cp.async.commit_group;\n" ::: "memory");
#endif
}
template <int N>
GPSS_D void cp_async_wait() {
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 800
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
#endif
}

// ---------------------------------------------------------------------------
// Step-scalar tables, one warp per (hyperparameter row, term), with (a, beta)
// tangents, in double-float arithmetic on the FP32 pipe (table_coeffs_df is
// the same computation written sequentially).  Lane 0 runs the scaled
// recurrence of f's Taylor coefficients c~_n = c_n T^n; lanes form c~_n/(n+1)
// and n c~_n; lane k sums the products giving coefficient k of the six
// series; all lanes then share the outputs of the economisation map, each
// scaled back by T^-(k+q) in FP64 and rounded once to FP32.
// ---------------------------------------------------------------------------
constexpr int TABLE_WARPS = 4;

template <int NT>
__global__ void __launch_bounds__(32 * TABLE_WARPS) k_tables(const float *__restrict__ theta,
                                                            int n_rows, int n_params, int kind0,
                                                            int kind1, float *__restrict__ tab,
                                                            EconMap E) {
  using DD = Dual2<DF>;
  constexpr int NCF = TAB_NCF;  // c_0 .. c_NCF
  __shared__ DD sc[TABLE_WARPS][NCF + 1], se[TABLE_WARPS][NCF + 1], sf[TABLE_WARPS][NCF + 1];
  __shared__ DD sg[TABLE_WARPS][6][TAB_NTAY];
  // the economisation map and reciprocals in shared memory: the lanes index
  // them with different k, which the parameter (constant) bank would serialise
  __shared__ DF sm_m[TAB_NC][TAB_NTAY];
  __shared__ DF sm_rcp[2 * TAB_NTAY + 8];
  for (int i = threadIdx.x; i < TAB_NC * TAB_NTAY; i += blockDim.x)
    sm_m[i / TAB_NTAY][i % TAB_NTAY] = df_of(E.m[i / TAB_NTAY][i % TAB_NTAY]);
  for (int i = threadIdx.x; i < 2 * TAB_NTAY + 8; i += blockDim.x) sm_rcp[i] = df_of(E.rcp[i]);
  __syncthreads();
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rt = blockIdx.x * TABLE_WARPS + w;
  if (rt >= n_rows * NT) return;  // whole warps leave together
  const int row = rt / NT, t = rt % NT;
  const int kinds[4] = {kind0, kind1, 0, 0};
  TermC<double> tc[NT];
  double s2;
  load_terms<NT, double>(theta + (size_t)row * n_params, kinds, tc, s2);
  const double T = table_range(tc[t].r2);
  const DF one = df_of(1.0), zero = df_of(0.0);
  const DD a = mkdf(df_of(tc[t].a), one, zero), beta = mkdf(df_of(tc[t].beta), zero, one);
  const DD w2 = beta + a * a;
  if (lane == 0) taylor_c_scaled(a * df_of(T), w2 * df_of(T * T), sm_rcp, &sc[w][0], df_of(T));
  __syncwarp();
  for (int n = lane; n <= NCF; n += 32) {
    const DD c = sc[w][n];
    se[w][n] = c * sm_rcp[n + 1];
    sf[w][n] = c * df_of((double)n);
  }
  __syncwarp();
  if (lane < TAB_NTAY) {
    DD g[6];
    taylor_coeff_scaled(&sc[w][0], &se[w][0], &sf[w][0], sm_rcp, lane, g);
#pragma unroll
    for (int j = 0; j < 6; ++j) sg[w][j][lane] = g[j];
  }
  __syncwarp();
  float *base = tab + (size_t)rt * TAB_NC * TAB_W;
  for (int o = lane; o < 6 * TAB_NC; o += 32) {
    const int j = o / TAB_NC, k = o % TAB_NC;
    const DD e = econ_apply_scaled(sm_m, k, &sg[w][j][0]);
    double sT = 1.0;
    const double iT = 1.0 / T;
    for (int i = 0; i < k + table_q(j); ++i) sT *= iT;
    float *r = base + (size_t)k * TAB_W;
    r[j] = (float)(df_val(e.v) * sT);
    r[8 + j] = (float)(df_val(e.da) * sT);
    r[14 + j] = (float)(df_val(e.db) * sT);
  }
  for (int o = lane; o < TAB_NC * 2; o += 32) {
    // the pads: columns 6, 7 of each record
    float *r = base + (size_t)(o >> 1) * TAB_W;
    r[6 + (o & 1)] = 0.f;
  }
}

// Copy the table of hyperparameter row `row` (all NT terms) into this warp's
// shared-memory slot.  Every lane of a warp works on the same row (the chunk
// plan gives each series a multiple of 32 chunks).
template <int NT>
GPSS_D const float4 *stage_table(const float *__restrict__ tab, int row, float4 *slot) {
  const float4 *src = reinterpret_cast<const float4 *>(tab + (size_t)row * NT * TAB_TERM);
  const int lane = threadIdx.x & 31;
  for (int i = lane; i < NT * TAB_TERM / 4; i += 32) slot[i] = __ldg(src + i);
  __syncwarp();
  return slot;
}

// ---------------------------------------------------------------------------
// Plain per-series filter (loglik only).
// ---------------------------------------------------------------------------
template <class S, class F>
__global__ void __launch_bounds__(128) k_plain(DevModel M, const float *__restrict__ theta, int n_out,
                                               int per_series, double *__restrict__ ll_out,
                                               int *__restrict__ err) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n_out) return;
  const int s = per_series ? v : v % M.n_series;
  const int row = per_series ? v : v / M.n_series;
  TermC<F> tc[S::NT];
  F s2;
  load_terms<S::NT, F>(theta + (size_t)row * M.n_params, M.kinds, tc, s2);
  auto body = [&](auto od_tag) {
    constexpr bool OD = decltype(od_tag)::value;
    F m[S::D], P[S::NP];
    init_state<S>(tc, m, P);
    double sum_logS = 0.0, sum_q = 0.0;
    int64_t n_end = 0;
    bool bad = false;
    int64_t mi = M.meas_off[s];
    const int64_t e1 = M.ev_off[s + 1];
    for (int64_t k = M.ev_off[s]; k < e1; ++k) {
      F Sv, vv;
      if (filter_event<S, F, OD>(M, k, mi, tc, s2, m, P, Sv, vv)) {
        bad |= !(Sv > F(0));
        sum_logS += glog(Sv);
        sum_q += (double)(vv * vv / Sv);
        ++n_end;
      }
    }
    const double ll = -0.5 * ((double)n_end * LOG_2PI + sum_logS + sum_q);
    bad |= !isfinite(ll);
    ll_out[v] = ll;
    if (bad) flag_error(err, v, 7);
  };
  if (any_overdamped<S::NT>(tc) || M.mixed)
    body(OdTag<true>{});
  else
    body(OdTag<false>{});
}

// ---------------------------------------------------------------------------
// Chunk elements.
// Layout of the float part (field-major, stride n_vch):
//   A (D*D row-major) | b (D) | C (NP) | eta (D) | J (NP)
// double part (stride n_vch): gamma | sum log S | n_end
// ---------------------------------------------------------------------------
template <class S>
struct ElemLayout : Elem<S> {
  static constexpr int ND = 3;
};

template <class S>
GPSS_D void store_elem(float *dst, int n_vch, int vc, const float (&A)[S::D][S::D], const float *b,
                       const float *C, const float *eta, const float *J) {
  using L = ElemLayout<S>;
  constexpr int D = S::D;
#pragma unroll
  for (int i = 0; i < D; ++i) {
#pragma unroll
    for (int j = 0; j < D; ++j) dst[(size_t)(L::A + i * D + j) * n_vch + vc] = A[i][j];
    dst[(size_t)(L::B + i) * n_vch + vc] = b[i];
    dst[(size_t)(L::ETA + i) * n_vch + vc] = eta[i];
  }
#pragma unroll
  for (int i = 0; i < S::NP; ++i) {
    dst[(size_t)(L::C + i) * n_vch + vc] = C[i];
    dst[(size_t)(L::J + i) * n_vch + vc] = J[i];
  }
}

// resident 128-thread blocks per SM the register budget of k_elem is sized for
#ifndef GPSS_ELEM_MIN_BLOCKS
#define GPSS_ELEM_MIN_BLOCKS 3
#endif
constexpr int ELEM_MIN_BLOCKS = GPSS_ELEM_MIN_BLOCKS;

// One event of a chunk element: the filter run from an unknown incoming state
// x, with mean A x + b, covariance C, information (eta, J) about x from the
// chunk's measurements so far, gamma = sum c^2/S and sum log S (the element
// of Sarkka & Garcia-Fernandez 2021 for a stretch of events, Section 3.2.5).
// Predict with the step's blocks (A <- Phi~ A, b <- Phi~ b, C <- Phi~ C
// Phi~^T + Q~), then reset the slot at an exposure start or update with the
// measurement (y, r0, w) at an end.
template <class S, class F, bool MIX = false>
GPSS_HD void elem_event(const Blocks<F> *B, uint8_t tag, F y, F r0, F w, F s2,
                        F (&A)[S::D][S::D], F *b, F *C, F *eta, F *J, double &gam, double &ld,
                        int &n_end, bool &bad) {
  constexpr int D = S::D;
#pragma unroll
  for (int col = 0; col < D; ++col) {
    F v[D], o[D];
#pragma unroll
    for (int i = 0; i < D; ++i) v[i] = A[i][col];
    apply_phi<S>(B, v, o);
#pragma unroll
    for (int i = 0; i < D; ++i) A[i][col] = o[i];
  }
  {
    F o[D];
    apply_phi<S>(B, b, o);
#pragma unroll
    for (int i = 0; i < D; ++i) b[i] = o[i];
  }
  predict_cov<S>(B, C);
  const int j = (tag >> 1) & 7;
  if (!(tag & 1)) {
    reset_slot<S>(j, b, C);
#pragma unroll
    for (int zi = 2 * S::NT; zi < D; ++zi) {
      const bool hit = (S::zslot(zi) == j);
#pragma unroll
      for (int col = 0; col < D; ++col) A[zi][col] = hit ? F(0) : A[zi][col];
    }
    return;
  }
  F u[D], hu, hb;
  obs_project_tag<S, F, MIX>(tag, w, b, C, u, hu, hb);
  const F Sv = hu + r0 + s2;
  const F cc = y - hb;
  // an instantaneous measurement reads the latent (always in shapes without
  // integral states; by its tag in a mixed model)
  const bool inst = S::NS == 0 || (MIX && (tag & TAG_INSTANT));
  F g[D];  // h^T A
#pragma unroll
  for (int col = 0; col < D; ++col) {
    F acc = F(0), lat = F(0);
#pragma unroll
    for (int t = 0; t < S::NT; ++t) lat += A[2 * t][col];
#pragma unroll
    for (int zi = 2 * S::NT; zi < D; ++zi) acc += (S::zslot(zi) == j) ? A[zi][col] : F(0);
    g[col] = inst ? lat : acc * w;
  }
  bad |= !(Sv > F(0));
  const F iS = F(1) / Sv;
  const F ci = cc * iS;
#pragma unroll
  for (int i = 0; i < D; ++i) {
    eta[i] += g[i] * ci;
#pragma unroll
    for (int jj = i; jj < D; ++jj) J[S::pk(i, jj)] += g[i] * g[jj] * iS;
  }
  gam += (double)(cc * ci);
  ld += glog(Sv);
  ++n_end;
#pragma unroll
  for (int i = 0; i < D; ++i) {
    const F Ki = u[i] * iS;
#pragma unroll
    for (int col = 0; col < D; ++col) A[i][col] -= Ki * g[col];
    b[i] += Ki * cc;
#pragma unroll
    for (int jj = i; jj < D; ++jj) C[S::pk(i, jj)] -= u[i] * u[jj] * iS;
  }
}

// With pck set, the partial element of the chunk's first events is also saved
// at the start of every gradient segment but the first (segments of ck
// events, aligned to the chunk's end): record j at pck + j (NF + 1) n_vch,
// fields as above plus the number of measurements before that point.  With
// dcache set, every step's six scalars per term go to the step-scalar cache
// (for the gradient's forward replay).
template <class S, bool OD>
__global__ void __launch_bounds__(128, ELEM_MIN_BLOCKS) k_elem(DevModel M, const float *__restrict__ theta, int n_vch,
                                              int per_series, float *__restrict__ ef,
                                              double *__restrict__ ed, int *__restrict__ err,
                                              const float *__restrict__ tabs,
                                              float *__restrict__ pck, int ck,
                                              float *__restrict__ dcache, int c_begin,
                                              int c_count) {
  using F = float;
  constexpr int D = S::D;
  using L = ElemLayout<S>;
  extern __shared__ float4 smem_tab[];
  // chunks [c_begin, c_begin + c_count) of every parameter set (a multiple of
  // 32 chunks per series keeps each warp in one series)
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= (n_vch / M.n_chunks) * c_count) return;
  const int set = l / c_count;
  const int c = c_begin + l % c_count;
  const int vc = set * M.n_chunks + c;
  const int s = M.ch_series[c];
  const int row = per_series ? s : set;
  const int orow = per_series ? s : set * M.n_series + s;
  TermC<F> tc[S::NT];
  F s2;
  load_terms<S::NT, F>(theta + (size_t)row * M.n_params, M.kinds, tc, s2);
  // rows with an overdamped term (and every row of a mixed model) run in the
  // OD = true launch, the others in the OD = false one (whole warps: a warp's
  // chunks share one row)
  if ((any_overdamped<S::NT>(tc) || M.mixed) != OD) return;
  const float4 *tab =
      stage_table<S::NT>(tabs, row, smem_tab + (threadIdx.x >> 5) * (S::NT * TAB_TERM / 4));
  const bool first = M.ch_flags[c] & 1;
  F A[D][D], b[D], C[S::NP], eta[D], J[S::NP];
  if (first) {
    init_state<S>(tc, b, C);
  } else {
#pragma unroll
    for (int i = 0; i < D; ++i) b[i] = F(0);
#pragma unroll
    for (int i = 0; i < S::NP; ++i) C[i] = F(0);
  }
#pragma unroll
  for (int i = 0; i < D; ++i) {
    eta[i] = F(0);
#pragma unroll
    for (int j = 0; j < D; ++j) A[i][j] = (!first && i == j) ? F(1) : F(0);
  }
#pragma unroll
  for (int i = 0; i < S::NP; ++i) J[i] = F(0);
  double gam = 0.0, ld = 0.0;
  int n_end = 0;
  bool bad = false;
  const int len = M.ch_len[c];
  float4 *dc = dcache_col<S::NT>(M, dcache, vc);
  EventReader rd;
  rd.start(M, c, 0, len);
  // gradient segments end at len - j ck (the first one is the short one);
  // at each later segment's start the partial element is saved
  const int f0 = len - ((len - 1) / ck) * ck;
  int next_ck = pck ? f0 : len;
  for (int kk = 0; kk < len; ++kk) {
    if (kk == next_ck) {
      float *dst = pck + (size_t)((kk - f0) / ck) * (L::NF + 1) * n_vch;
      store_elem<S>(dst, n_vch, vc, A, b, C, eta, J);
      dst[(size_t)L::NF * n_vch + vc] = __int_as_float(n_end);
      next_ck += ck;
    }
    F dt;
    uint8_t tag;
    float4 q;
    rd.next(dt, tag, q);
    Blocks<F> B[S::NT];
    {
      constexpr int W = DcW<S::NT>::W;
      float x[W];
#pragma unroll
      for (int t = 0; t < S::NT; ++t) {
        const Disc<F> d = discretize_tab<OD>(dt, tc[t], tab + t * (TAB_TERM / 4));
        x[6 * t] = d.f;
        x[6 * t + 1] = d.fp;
        x[6 * t + 2] = d.F1;
        x[6 * t + 3] = d.Iff;
        x[6 * t + 4] = d.Ipp;
        x[6 * t + 5] = d.IFF;
        B[t] = make_blocks(d, tc[t]);
      }
#pragma unroll
      for (int i = 6 * S::NT; i < W; ++i) x[i] = 0.f;
      if (dc) {
        float4 *r = dc + (size_t)kk * (32 * DcW<S::NT>::G);
#pragma unroll
        for (int v = 0; v < DcW<S::NT>::G; ++v)
          r[32 * v] = make_float4(x[4 * v], x[4 * v + 1], x[4 * v + 2], x[4 * v + 3]);
      }
    }
    elem_event<S, F, OD>(B, tag, q.x, q.y, q.z, s2, A, b, C, eta, J, gam, ld, n_end, bad);
  }
  store_elem<S>(ef, n_vch, vc, A, b, C, eta, J);
  ed[vc] = gam;
  ed[(size_t)n_vch + vc] = ld;
  ed[(size_t)2 * n_vch + vc] = (double)n_end;
  if (bad) flag_error(err, orow, 7);
}

// ---------------------------------------------------------------------------
// Cross-chunk combination, one thread per (virtual) series, sequential over
// its chunks.  With the incoming filtered state N(m, P) and a chunk element
// (A, b, C, eta, J, gamma, sum log S):
//   X = I + P J
//   chunk loglik = -1/2 [sum log 2 pi S + log det X + gamma - 2 eta^T m
//                        + m^T J m - u^T X^{-1} P u],      u = eta - J m
//   outgoing m'  = A X^{-1} (m + P eta) + b,  P' = A X^{-1} P A^T + C.
// Backward, the information (eta_n, J_n) about a chunk's end state from all
// later data folds in as
//   eta <- A^T (I + J_n C)^{-1} (eta_n - J_n b) + eta,  J <- A^T (I + J_n C)^{-1} J_n A + J,
// and the adjoint of the log-likelihood of later data w.r.t. the filtered
// end state (m, P) is  lambda = (I + J P)^{-1} (eta - J m),
// Lambda = (lambda lambda^T - (I + J P)^{-1} J) / 2.
// State / adjoint records: (vector D | packed NP), stride n_vch.
// ---------------------------------------------------------------------------
// Marginal log-likelihood of a chunk's data given N(m, P) for the state
// entering it, from the chunk's information (eta, J), gamma = sum c^2/S and
// sum log S over its n_end measurements; arithmetic of T.
template <class S, class T = float>
GPSS_HD double chunk_loglik(const T *m, const T *P, const T *eta, const T *J, double gam,
                            double ld, double ne) {
  constexpr int D = S::D;
  T X[D][D], R[D][D];
  T u[D];
#pragma unroll
  for (int i = 0; i < D; ++i) {
    T jm = T(0);
#pragma unroll
    for (int k = 0; k < D; ++k) jm += J[S::pk(i, k)] * m[k];
    u[i] = eta[i] - jm;
#pragma unroll
    for (int j = 0; j < D; ++j) {
      T acc = (i == j) ? T(1) : T(0);
#pragma unroll
      for (int k = 0; k < D; ++k) acc += P[S::pk(i, k)] * J[S::pk(k, j)];
      X[i][j] = acc;
      R[i][j] = P[S::pk(i, j)];
    }
  }
  const T logdet = solve_inplace<D, D, T>(X, R);  // R = (I + P J)^{-1} P
  T etam = T(0), mJm = T(0), uWu = T(0);
#pragma unroll
  for (int i = 0; i < D; ++i) {
    etam += eta[i] * m[i];
    T jm = T(0), wu = T(0);
#pragma unroll
    for (int k = 0; k < D; ++k) {
      jm += J[S::pk(i, k)] * m[k];
      wu += R[i][k] * u[k];
    }
    mJm += m[i] * jm;
    uWu += u[i] * wu;
  }
  const double quad = gam + (double)(T(-2) * etam + mJm - uWu);
  return -0.5 * (ld + ne * LOG_2PI + (double)logdet + quad);
}

// Adjoint of the log-likelihood of all later data with respect to the
// filtered state (m, P), given their information (eta, J) about it:
// lambda = (I + J P)^{-1} (eta - J m), Lambda = (lambda lambda^T - (I + J P)^{-1} J) / 2.
template <class S, class T = float>
GPSS_HD void boundary_adjoint(const T *m, const T *P, const T *eta, const T *J, float *lam,
                              float *Lam) {
  constexpr int D = S::D;
  T X[D][D], R[D][D + 1];
#pragma unroll
  for (int i = 0; i < D; ++i) {
    T jm = T(0);
#pragma unroll
    for (int k = 0; k < D; ++k) jm += J[S::pk(i, k)] * m[k];
    R[i][D] = eta[i] - jm;
#pragma unroll
    for (int j = 0; j < D; ++j) {
      T acc = (i == j) ? T(1) : T(0);
#pragma unroll
      for (int k = 0; k < D; ++k) acc += J[S::pk(i, k)] * P[S::pk(k, j)];
      X[i][j] = acc;
      R[i][j] = J[S::pk(i, j)];
    }
  }
  solve_inplace<D, D + 1, T>(X, R);
#pragma unroll
  for (int i = 0; i < D; ++i) lam[i] = (float)R[i][D];
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int j = i; j < D; ++j)
      Lam[S::pk(i, j)] = (float)(T(0.5) * (R[i][D] * R[j][D] - T(0.5) * (R[i][j] + R[j][i])));
}

template <class S>
GPSS_D void load_elem(const float *ef, int n_vch, int vc, float (&A)[S::D][S::D], float *b, float *C,
                      float *eta, float *J) {
  load_elem_t<S, float, float>(ef, (size_t)n_vch, (size_t)vc, A, b, C, eta, J);
}

// State / adjoint records (vector D | packed NP), stride n_vch, stored as U
// and held as T.
template <class S, class U, class T>
GPSS_D void store_rec(U *dst, int n_vch, int vc, const T *v, const T *P) {
#pragma unroll
  for (int i = 0; i < S::D; ++i) dst[(size_t)i * n_vch + vc] = (U)v[i];
#pragma unroll
  for (int i = 0; i < S::NP; ++i) dst[(size_t)(S::D + i) * n_vch + vc] = (U)P[i];
}

template <class S, class U, class T>
GPSS_D void load_rec(const U *src, int n_vch, int vc, T *v, T *P) {
#pragma unroll
  for (int i = 0; i < S::D; ++i) v[i] = (T)src[(size_t)i * n_vch + vc];
#pragma unroll
  for (int i = 0; i < S::NP; ++i) P[i] = (T)src[(size_t)(S::D + i) * n_vch + vc];
}

// A filtered-state record that is FP32 or FP64 (the combination's
// precision), read as FP32.
template <class S>
GPSS_D void load_state_f(const void *src, int se64, int n_vch, int vc, float *v, float *P) {
  if (se64)
    load_rec<S>(static_cast<const double *>(src), n_vch, vc, v, P);
  else
    load_rec<S>(static_cast<const float *>(src), n_vch, vc, v, P);
}

// Sequential schedule of the cross-chunk combination: one thread per
// (virtual) series folds its chunks in time order, in the arithmetic of T.
// Writes the filtered state at the end of every chunk (state_end, records of
// T), the series log-likelihood, and for the gradient the adjoint of each
// chunk's end state (adj_end, FP32).
template <class S, class T>
__global__ void __launch_bounds__(64) k_scan_seq(DevModel M, int n_out, int per_series,
                                                 const float *__restrict__ ef,
                                                 const double *__restrict__ ed, int n_vch,
                                                 T *__restrict__ state_end,
                                                 float *__restrict__ adj_end,
                                                 double *__restrict__ ll_out, int want_grad,
                                                 int *__restrict__ err) {
  constexpr int D = S::D;
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n_out) return;
  const int s = per_series ? v : v % M.n_series;
  const int set = per_series ? 0 : v / M.n_series;
  const int c0 = M.ch_first[s], c1 = M.ch_first[s + 1];
  const int base = set * M.n_chunks;
  T m[D], P[S::NP];
  double ll = 0.0;
  for (int c = c0; c < c1; ++c) {
    const int vc = base + c;
    T A[D][D], b[D], C[S::NP], eta[D], J[S::NP];
    load_elem_t<S, T, float>(ef, (size_t)n_vch, (size_t)vc, A, b, C, eta, J);
    const double gam = ed[vc], ld = ed[(size_t)n_vch + vc], ne = ed[(size_t)2 * n_vch + vc];
    if (c == c0) {
      ll += -0.5 * (ld + gam + ne * LOG_2PI);
#pragma unroll
      for (int i = 0; i < D; ++i) m[i] = b[i];
#pragma unroll
      for (int i = 0; i < S::NP; ++i) P[i] = C[i];
    } else {
      ll += chunk_loglik<S, T>(m, P, eta, J, gam, ld, ne);
      state_through<S, T>(A, b, C, eta, J, m, P);
    }
    if (want_grad) store_rec<S>(state_end, n_vch, vc, m, P);
  }
  if (ll_out) ll_out[v] = ll;
  if (!isfinite(ll)) flag_error(err, v, 7);
  if (!want_grad) return;
  // backward information and end-of-chunk adjoints
  T ie[D], iJ[S::NP];
#pragma unroll
  for (int i = 0; i < D; ++i) ie[i] = T(0);
#pragma unroll
  for (int i = 0; i < S::NP; ++i) iJ[i] = T(0);
  for (int c = c1 - 1; c >= c0; --c) {
    const int vc = base + c;
    float lam[D], Lam[S::NP];
    if (c == c1 - 1) {
#pragma unroll
      for (int i = 0; i < D; ++i) lam[i] = 0.f;
#pragma unroll
      for (int i = 0; i < S::NP; ++i) Lam[i] = 0.f;
    } else {
      T mb[D], Pb[S::NP];
      load_rec<S>(state_end, n_vch, vc, mb, Pb);
      boundary_adjoint<S, T>(mb, Pb, ie, iJ, lam, Lam);
    }
    store_rec<S>(adj_end, n_vch, vc, lam, Lam);
    if (c == c0) break;
    // fold chunk c into the backward information
    T A[D][D], b[D], C[S::NP], eta[D], J[S::NP];
    load_elem_t<S, T, float>(ef, (size_t)n_vch, (size_t)vc, A, b, C, eta, J);
    info_through<S, T>(A, b, C, eta, J, ie, iJ);
  }
}

// Tree schedule, last step: per chunk, its log-likelihood contribution
// (closed form given the state entering it) and, for the gradient, the
// adjoint of its end state from the information of the following chunks.
//   state_end  (b, C) of the inclusive prefix scan   (filtered end state)
//   info_incl  (eta, J) of the inclusive suffix scan (information about the
//              state entering the chunk from it and all later chunks)
// Both are records of T (the combination's arithmetic), which is also the
// arithmetic of the closed-form chunk log-likelihood and of the adjoint.
template <class S, class T>
__global__ void __launch_bounds__(128) k_finish(DevModel M, int n_vch, int per_series,
                                                const float *__restrict__ ef,
                                                const double *__restrict__ ed,
                                                const T *__restrict__ state_end,
                                                const T *__restrict__ info_incl,
                                                float *__restrict__ adj_end,
                                                double *__restrict__ ll_part,
                                                int *__restrict__ err) {
  constexpr int D = S::D;
  using L = ElemLayout<S>;
  const int vc = blockIdx.x * blockDim.x + threadIdx.x;
  if (vc >= n_vch) return;
  const int c = vc % M.n_chunks;
  const int set = vc / M.n_chunks;
  const int s = M.ch_series[c];
  const int orow = per_series ? s : set * M.n_series + s;
  const uint8_t flags = M.ch_flags[c];
  const double gam = ed[vc], ld = ed[(size_t)n_vch + vc], ne = ed[(size_t)2 * n_vch + vc];
  double ll;
  if (flags & 1) {
    ll = -0.5 * (ld + gam + ne * LOG_2PI);
  } else {
    T m[D], P[S::NP], eta[D], J[S::NP];
    load_rec<S>(state_end, n_vch, vc - 1, m, P);
#pragma unroll
    for (int i = 0; i < D; ++i) eta[i] = T(ef[(size_t)(L::ETA + i) * n_vch + vc]);
#pragma unroll
    for (int i = 0; i < S::NP; ++i) J[i] = T(ef[(size_t)(L::J + i) * n_vch + vc]);
    ll = chunk_loglik<S, T>(m, P, eta, J, gam, ld, ne);
  }
  ll_part[vc] = ll;
  if (!isfinite(ll)) flag_error(err, orow, 7);
  if (!adj_end) return;
  float lam[D], Lam[S::NP];
  if (flags & 2) {
#pragma unroll
    for (int i = 0; i < D; ++i) lam[i] = 0.f;
#pragma unroll
    for (int i = 0; i < S::NP; ++i) Lam[i] = 0.f;
  } else {
    T mb[D], Pb[S::NP], ie[D], iJ[S::NP];
    load_rec<S>(state_end, n_vch, vc, mb, Pb);
    load_rec<S>(info_incl, n_vch, vc + 1, ie, iJ);
    boundary_adjoint<S, T>(mb, Pb, ie, iJ, lam, Lam);
  }
  store_rec<S>(adj_end, n_vch, vc, lam, Lam);
}

// ---------------------------------------------------------------------------
// Reverse-time gradient, one thread per chunk.
// ---------------------------------------------------------------------------
constexpr int GRAD_BS = 64;
// resident blocks per SM the register budget of k_grad is sized for
#ifndef GPSS_GRAD_MIN_BLOCKS
#define GPSS_GRAD_MIN_BLOCKS 6
#endif
constexpr int GRAD_MIN_BLOCKS = GPSS_GRAD_MIN_BLOCKS;
// cp.async stages of the backward walk's staging (replay record and cached
// step scalars): the step GRAD_STAGES - 1 ahead is in flight
#ifndef GPSS_GRAD_STAGES
#define GPSS_GRAD_STAGES 2
#endif
constexpr int GRAD_STAGES = GPSS_GRAD_STAGES;
template <int NT>
struct TermGrad {
  float a[NT], beta[NT], w2[NT], qc[NT], var[NT];
  float s2;
};

// Latent f(t*) = sum_t x_t(t*) at a test time between two events, given all
// the data: (m, P) is the filtered state after the earlier event, d1 = t* -
// t_prev, d2 = t_next - t*, and (lp, Lp) the adjoint of the later data's
// log-likelihood with respect to the predicted state of the next event.  The
// state at t* is predicted over d1 (m*, P*); its adjoint is that of the next
// event pulled back over d2, lambda* = Phi2^T lp, Lambda* = Phi2^T Lp Phi2;
// the smoothed state is m* + P* lambda*, P* - P* (lambda* lambda*^T -
// 2 Lambda*) P*.  With h_x selecting the latent components and u = P* h_x,
// v = Phi2 u:  mean = h_x.m* + v.lp,  var = h_x.u + 2 v^T Lp v - (v.lp)^2.
// Retrodiction: (m, P) the prior and d1 = 0; extrapolation: zero adjoint.
template <class S, bool OD = true>
GPSS_D float2 predict_point(float d1, float d2, const TermC<float> *tc, const float4 *tab,
                            const float *m, const float *P, const float *lp, const float *Lp) {
  constexpr int D = S::D;
  Blocks<float> B1[S::NT], B2[S::NT];
#pragma unroll
  for (int t = 0; t < S::NT; ++t) {
    B1[t] = make_blocks(discretize_tab<OD>(d1, tc[t], tab + t * (TAB_TERM / 4)), tc[t]);
    B2[t] = make_blocks(discretize_tab<OD>(d2, tc[t], tab + t * (TAB_TERM / 4)), tc[t]);
  }
  float ms[D], Ps[S::NP];
  apply_phi<S>(B1, m, ms);
#pragma unroll
  for (int i = 0; i < S::NP; ++i) Ps[i] = P[i];
  predict_cov<S>(B1, Ps);
  float u[D], hm = 0.f;
#pragma unroll
  for (int i = 0; i < D; ++i) {
    float acc = 0.f;
#pragma unroll
    for (int t = 0; t < S::NT; ++t) acc += Ps[S::pk(i, 2 * t)];
    u[i] = acc;
  }
  float hu = 0.f;
#pragma unroll
  for (int t = 0; t < S::NT; ++t) {
    hm += ms[2 * t];
    hu += u[2 * t];
  }
  float v[D];
  apply_phi<S>(B2, u, v);
  float vl = 0.f, vLv = 0.f;
#pragma unroll
  for (int i = 0; i < D; ++i) {
    vl += v[i] * lp[i];
    float acc = 0.f;
#pragma unroll
    for (int k = 0; k < D; ++k) acc += Lp[S::pk(i, k)] * v[k];
    vLv += v[i] * acc;
  }
  return make_float2(hm + vl, hu + 2.f * vLv - vl * vl);
}

// Conditioned mean and variance of an exposure average from the filtered
// state (m, P) just after its end event (slot j, w = 1/delta) and the
// adjoint (lam, Lam) of the log-likelihood of all later data with respect
// to that state: the smoothed state is m + P lam and P - P (lam lam^T -
// 2 Lam) P (the Gaussian conditioning identities behind the RTS smoother),
// so with h = w e_j and u = P h:  mean = h.m + u.lam,
// var = h.u + u^T (2 Lam) u - (u.lam)^2.
template <class S>
GPSS_HD float2 conditioned_latent(const float *m, const float *P, const float *lam,
                                  const float *Lam) {
  constexpr int D = S::D;
  {
    // instantaneous measurement: h selects the latent components
    float u[D], hm = 0.f;
#pragma unroll
    for (int i = 0; i < D; ++i) {
      float acc = 0.f;
#pragma unroll
      for (int t = 0; t < S::NT; ++t) acc += P[S::pk(i, 2 * t)];
      u[i] = acc;
    }
    float ul = 0.f, hu = 0.f, uLu = 0.f;
#pragma unroll
    for (int t = 0; t < S::NT; ++t) {
      hm += m[2 * t];
      hu += u[2 * t];
    }
#pragma unroll
    for (int i = 0; i < D; ++i) {
      ul += u[i] * lam[i];
      float acc = 0.f;
#pragma unroll
      for (int k = 0; k < D; ++k) acc += Lam[S::pk(i, k)] * u[k];
      uLu += u[i] * acc;
    }
    return make_float2(hm + ul, hu + 2.f * uLu - ul * ul);
  }
}

template <class S>
GPSS_HD float2 conditioned(int j, float w, const float *m, const float *P, const float *lam,
                           const float *Lam) {
  constexpr int D = S::D;
  if constexpr (S::NS == 0) return conditioned_latent<S>(m, P, lam, Lam);
  float u[D], hm = 0.f;
#pragma unroll
  for (int i = 0; i < D; ++i) {
    float acc = 0.f;
#pragma unroll
    for (int z = 2 * S::NT; z < D; ++z)
      if (S::zslot(z) == j) acc += P[S::pk(i, z)];
    u[i] = w * acc;
    if (i >= 2 * S::NT && S::zslot(i) == j) hm += m[i];
  }
  float ul = 0.f, hu = 0.f, uLu = 0.f;
#pragma unroll
  for (int i = 0; i < D; ++i) {
    ul += u[i] * lam[i];
    if (i >= 2 * S::NT && S::zslot(i) == j) hu += u[i];
    float acc = 0.f;
#pragma unroll
    for (int k = 0; k < D; ++k) acc += Lam[S::pk(i, k)] * u[k];
    uLu += u[i] * acc;
  }
  return make_float2(w * hm + ul, w * hu + 2.f * uLu - ul * ul);
}

// The same for a measurement event given its tag (MIX: instants among
// exposure averages, marked TAG_INSTANT).
template <class S, bool MIX>
GPSS_HD float2 conditioned_tag(uint8_t tag, float w, const float *m, const float *P,
                               const float *lam, const float *Lam) {
  if constexpr (MIX && S::NS > 0) {
    if (tag & TAG_INSTANT) return conditioned_latent<S>(m, P, lam, Lam);
  }
  return conditioned<S>((tag >> 1) & 7, w, m, P, lam, Lam);
}

// Reverse of one event.  (m, P): filtered state before the event; dv: the
// step's six scalars per term.  (lam, Lam): adjoint of the filtered state
// after the event (full-matrix gradient convention, stored packed); on
// return, adjoint of (m, P).
// With want_exp, also g_dt = d loglik / d (this step's gap) and, at an end
// event, g_w = d loglik / d (1/delta of its measurement).
// hook(lam, Lam) runs once the update (or reset) is reversed, with the
// adjoint of the predicted state of this event.
struct NoHook {
  GPSS_D void operator()(const float *, const float *) const {}
};

// Value i of a staged replay record (m first, then packed P) in shared
// memory: float4 group g of this thread's slot at sb[g bs].
struct StagedRec {
  const float4 *sb;
  int bs, off;
  GPSS_D float operator[](int i) const {
    const int k = i + off;
    return reinterpret_cast<const float *>(sb + (size_t)(k >> 2) * bs)[k & 3];
  }
};

//
// m and P are read through operator[] (register arrays, or the staged replay
// record in shared memory, which the walk then reads where it needs them
// instead of holding them in registers across the event).
template <class S, bool OD = true, class Hook = NoHook, class V = const float *>
GPSS_D void reverse_event(float dt, uint8_t tag, float4 q, const TermC<float> *tc, float s2,
                          const V &m, const V &P, float *lam, float *Lam,
                          TermGrad<S::NT> &gr, const float4 *tab, const Disc<float> *dv,
                          bool want_exp, float &g_dt, float &g_w, const Hook &hook = Hook()) {
  using F = float;
  constexpr int D = S::D;
  const int j = (tag >> 1) & 7;
  g_dt = F(0);
  g_w = F(0);
  Blocks<F> B[S::NT];
#pragma unroll
  for (int t = 0; t < S::NT; ++t) B[t] = make_blocks(dv[t], tc[t]);
  // recompute the prediction
  F mp[D], Pp[S::NP];
  {
    F mv[D];
#pragma unroll
    for (int i = 0; i < D; ++i) mv[i] = m[i];
    apply_phi<S>(B, mv, mp);
  }
#pragma unroll
  for (int i = 0; i < S::NP; ++i) Pp[i] = P[i];
  predict_cov<S>(B, Pp);
  if (tag & 1) {
    const F y = q.x, r0 = q.y, w = q.z;
    // an instantaneous measurement reads the latent (always in shapes without
    // integral states; by its tag in a mixed model, whose rows run OD bodies)
    const bool inst = S::NS == 0 || (OD && (tag & TAG_INSTANT));
    F u[D], hu, hm;
    obs_project_tag<S, F, OD>(tag, w, mp, Pp, u, hu, hm);
    const F Sv = hu + r0 + s2;
    const F v = y - hm;
    const F iS = F(1) / Sv;
    F lu = F(0), uLu = F(0), Lu[D];
#pragma unroll
    for (int i = 0; i < D; ++i) {
      F acc = F(0);
#pragma unroll
      for (int kk = 0; kk < D; ++kk) acc += Lam[S::pk(i, kk)] * u[kk];
      Lu[i] = acc;
      lu += lam[i] * u[i];
    }
#pragma unroll
    for (int i = 0; i < D; ++i) uLu += u[i] * Lu[i];
    F ub[D];
#pragma unroll
    for (int i = 0; i < D; ++i) ub[i] = (F(-2) * Lu[i] + lam[i] * v) * iS;
    const F Sb = uLu * iS * iS - lu * v * iS * iS - F(0.5) * (iS - v * v * iS * iS);
    const F vb = lu * iS - v * iS;
    F h[D];
#pragma unroll
    for (int i = 0; i < D; ++i) {
      const F hl = (i < 2 * S::NT && i % 2 == 0) ? F(1) : F(0);  // the latent
      const F hz = (i >= 2 * S::NT && S::zslot(i) == j) ? w : F(0);
      h[i] = inst ? hl : hz;
    }
    if (S::NS > 0 && want_exp && !inst) {
      // h = w e (e selects the slot's integral states): d/dh = Pp ub + 2 Sb u - vb mp
      F gw = F(0);
#pragma unroll
      for (int i = 2 * S::NT; i < D; ++i) {
        if (S::zslot(i) != j) continue;
        F acc = F(2) * Sb * u[i] - vb * mp[i];
#pragma unroll
        for (int kk = 0; kk < D; ++kk) acc += Pp[S::pk(i, kk)] * ub[kk];
        gw += acc;
      }
      g_w = gw;
    }
#pragma unroll
    for (int i = 0; i < D; ++i) {
      lam[i] -= h[i] * vb;
#pragma unroll
      for (int kk = i; kk < D; ++kk)
        Lam[S::pk(i, kk)] += F(0.5) * (ub[i] * h[kk] + h[i] * ub[kk]) + Sb * h[i] * h[kk];
    }
    gr.s2 += Sb;
  } else {
    reset_slot<S>(j, lam, Lam);
  }
  hook(lam, Lam);
  // reverse of the prediction: (lam, Lam) are now adjoints of (m-, P-).
  // d/dPhi~ = lam m^T + 2 Lam Phi~ P and d/dQ~ = Lam.  With T2 = Lam Phi~ the
  // middle term is T2 P and the adjoint of P is Phi~^T T2, so Phi~ P need not
  // be kept from the prediction; P is read again here.
  F T2[D][D];  // row i = (Phi~^T Lam[i,:])^T
#pragma unroll
  for (int i = 0; i < D; ++i) {
    F row[D], o[D];
#pragma unroll
    for (int kk = 0; kk < D; ++kk) row[kk] = Lam[S::pk(i, kk)];
    apply_phi_t<S>(B, row, o);
#pragma unroll
    for (int kk = 0; kk < D; ++kk) T2[i][kk] = o[kk];
  }
  // adjoints of the six step scalars per term, (f, f', F1, I_ff, I_pp, I_FF)
  F bX[S::NT][6];
#pragma unroll
  for (int t = 0; t < S::NT; ++t) {
    const int i0 = 2 * t, i1 = 2 * t + 1;
    // structured adjoints of Phi_t: LG = (lam m^T + 2 T2 P) at rows and
    // columns (i0, i1)
    F LG[2][2];
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
      for (int cc = 0; cc < 2; ++cc) {
        F acc = F(0);
#pragma unroll
        for (int kk = 0; kk < D; ++kk) acc += T2[i0 + r][kk] * P[S::pk(kk, i0 + cc)];
        LG[r][cc] = lam[i0 + r] * m[i0 + cc] + F(2) * acc;
      }
    // z rows integrating this term: their summed rows of lam m^T + 2 T2 P at
    // columns (i0, i1), and the Q blocks' adjoints
    F pb0 = F(0), pb1 = F(0);
    F q_z0 = F(0), q_z1 = F(0), q_zz = F(0);
#pragma unroll
    for (int zi = 2 * S::NT; zi < D; ++zi) {
      if (!S::zint(zi, t)) continue;
      F a0 = F(0), a1 = F(0);
#pragma unroll
      for (int kk = 0; kk < D; ++kk) {
        a0 += T2[zi][kk] * P[S::pk(kk, i0)];
        a1 += T2[zi][kk] * P[S::pk(kk, i1)];
      }
      pb0 += lam[zi] * m[i0] + F(2) * a0;
      pb1 += lam[zi] * m[i1] + F(2) * a1;
      q_z0 += F(2) * Lam[S::pk(i0, zi)];
      q_z1 += F(2) * Lam[S::pk(i1, zi)];
#pragma unroll
      for (int zj = 2 * S::NT; zj < D; ++zj)
        if (S::zint(zj, t)) q_zz += Lam[S::pk(zi, zj)];
    }
    const F q00 = Lam[S::pk(i0, i0)], q01 = F(2) * Lam[S::pk(i0, i1)], q11 = Lam[S::pk(i1, i1)];
    // blocks -> (f, f', F1, I_ff, I_pp, I_FF) adjoints and explicit (a, w2, Qc)
    const TermC<F> &c = tc[t];
    const F f = dv[t].f, F1 = dv[t].F1, Iff = dv[t].Iff, Ipp = dv[t].Ipp, IFF = dv[t].IFF;
    F bf = F(0), bfp = F(0), bF1 = F(0), bIff = F(0), bIpp = F(0), bIFF = F(0);
    // p00 = fp + 2a f ; p01 = f ; p10 = -w2 f ; p11 = fp
    bfp += LG[0][0] + LG[1][1];
    bf += F(2) * c.a * LG[0][0] + LG[0][1] - c.w2 * LG[1][0];
    gr.a[t] += F(2) * f * LG[0][0];
    gr.w2[t] += -f * LG[1][0];
    // pb0 = f + 2a F1 ; pb1 = F1
    bf += pb0;
    bF1 += F(2) * c.a * pb0 + pb1;
    gr.a[t] += F(2) * F1 * pb0;
    // Q blocks
    bIff += c.qc * q00 - c.qc * q_z1;
    bf += c.qc * f * q01 + c.qc * F1 * q_z1;
    bIpp += c.qc * q11;
    bF1 += c.qc * F1 * q_z0 + c.qc * f * q_z1;
    bIFF += c.qc * q_zz;
    gr.qc[t] += Iff * q00 + F(0.5) * f * f * q01 + Ipp * q11 + F(0.5) * F1 * F1 * q_z0 +
                (f * F1 - Iff) * q_z1 + IFF * q_zz;
    bX[t][0] = bf;
    bX[t][1] = bfp;
    bX[t][2] = bF1;
    bX[t][3] = bIff;
    bX[t][4] = bIpp;
    bX[t][5] = bIFF;
  }
  // lam <- Phi~^T lam ; Lam <- Phi~^T T2 = Phi~^T Lam Phi~
  {
    F o[D];
    apply_phi_t<S>(B, lam, o);
#pragma unroll
    for (int i = 0; i < D; ++i) lam[i] = o[i];
  }
#pragma unroll
  for (int cc = 0; cc < D; ++cc) {
    F col[D], o[D];
#pragma unroll
    for (int i = 0; i < D; ++i) col[i] = T2[i][cc];
    apply_phi_t<S>(B, col, o);
#pragma unroll
    for (int i = 0; i <= cc; ++i) Lam[S::pk(i, cc)] = o[i];
  }
  // through the discretisation: (a, beta) tangents of the six scalars
#pragma unroll
  for (int t = 0; t < S::NT; ++t) {
    const TermC<F> &c = tc[t];
    F da[6], db[6];
    disc_tangents<OD>(dt, c, tab + t * (TAB_TERM / 4), dv[t], da, db);
    gr.a[t] += bX[t][0] * da[0] + bX[t][1] * da[1] + bX[t][2] * da[2] + bX[t][3] * da[3] +
               bX[t][4] * da[4] + bX[t][5] * da[5];
    gr.beta[t] += bX[t][0] * db[0] + bX[t][1] * db[1] + bX[t][2] * db[2] + bX[t][3] * db[3] +
                  bX[t][4] * db[4] + bX[t][5] * db[5];
    if (want_exp) {
      // d/dt of the six scalars: f', f'' = -2a f' - w2 f, f, f^2, f'^2, F1^2
      const F f = dv[t].f, fp = dv[t].fp, F1 = dv[t].F1;
      g_dt += bX[t][0] * fp + bX[t][1] * (F(-2) * c.a * fp - c.w2 * f) + bX[t][2] * f +
              bX[t][3] * f * f + bX[t][4] * fp * fp + bX[t][5] * F1 * F1;
    }
  }
}

// Filtered state after the first events of a chunk, from the state entering
// the chunk, N(m_in, P_in), and the partial element (A, b, C, eta, J) of
// those events (the same combination as between chunks):
//   X = I + P_in J,  m = A X^{-1} (m_in + P_in eta) + b,  P = A X^{-1} P_in A^T + C.
template <class S>
GPSS_HD void apply_partial(const float *src, int n_vch, int vc, const float *m_in,
                           const float *P_in, float *m, float *P) {
  using L = ElemLayout<S>;
  constexpr int D = S::D;
  float J[S::NP], X[D][D], R[D][D + 1];
#pragma unroll
  for (int i = 0; i < S::NP; ++i) J[i] = src[(size_t)(L::J + i) * n_vch + vc];
#pragma unroll
  for (int i = 0; i < D; ++i) {
    float pe = 0.f;
#pragma unroll
    for (int k = 0; k < D; ++k) pe += P_in[S::pk(i, k)] * src[(size_t)(L::ETA + k) * n_vch + vc];
    R[i][D] = m_in[i] + pe;
#pragma unroll
    for (int j = 0; j < D; ++j) {
      float acc = (i == j) ? 1.f : 0.f;
#pragma unroll
      for (int k = 0; k < D; ++k) acc += P_in[S::pk(i, k)] * J[S::pk(k, j)];
      X[i][j] = acc;
      R[i][j] = P_in[S::pk(i, j)];
    }
  }
  solve_inplace<D, D + 1, float>(X, R);  // R = X^{-1} [P_in | m_in + P_in eta]
  float T[D][D + 1];
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int j = 0; j <= D; ++j) {
      float acc = 0.f;
#pragma unroll
      for (int k = 0; k < D; ++k) acc += src[(size_t)(L::A + i * D + k) * n_vch + vc] * R[k][j];
      T[i][j] = acc;
    }
#pragma unroll
  for (int i = 0; i < D; ++i) {
    m[i] = T[i][D] + src[(size_t)(L::B + i) * n_vch + vc];
#pragma unroll
    for (int j = i; j < D; ++j) {
      float acc = src[(size_t)(L::C + S::pk(i, j)) * n_vch + vc];
#pragma unroll
      for (int k = 0; k < D; ++k) acc += T[i][k] * src[(size_t)(L::A + j * D + k) * n_vch + vc];
      P[S::pk(i, j)] = acc;
    }
  }
}

// Segments of ck events aligned to the chunk's end (the first may be
// shorter).  Walking the segments from last to first: the filtered state at
// the segment's start comes from the partial element saved there by k_elem,
// the segment is replayed forward into this thread's column of rbuf (global,
// coalesced across the warp; slot k holds (m, P) before the segment's k-th
// event), then walked backwards in time.  With gdt set, the walk also
// writes, per event k of theta set r, gdt[r n_events + k] = d loglik / d
// (gap before k) and, at an end event, gwe[...] = w^2 d loglik / d w
// (w = 1/delta of its measurement; dw/dt_start = w^2 = -dw/dt_end).
template <class S>
__global__ void __launch_bounds__(GRAD_BS, GRAD_MIN_BLOCKS) k_grad(DevModel M, const float *__restrict__ theta, int n_vch,
                                             int per_series, const void *__restrict__ state_end,
                                             int se64, const float *__restrict__ adj_end,
                                             const float *__restrict__ pck, float *__restrict__ gpart,
                                             int *__restrict__ err,
                                             const float *__restrict__ tabs,
                                             float *__restrict__ rbuf,
                                             const float *__restrict__ dcache, int ck,
                                             float *__restrict__ gdt, float *__restrict__ gwe,
                                             float2 *__restrict__ cond, PredPlan pp) {
  using F = float;
  constexpr int D = S::D;
  constexpr int SD = D + S::NP;
  constexpr int NF = ElemLayout<S>::NF;
  constexpr int NDC = DcW<S::NT>::W;  // cached scalars per step (padded)
  constexpr int NDG = DcW<S::NT>::G;  // ... in float4 groups
  constexpr int SG = (SD + 3) / 4;    // replay slot: (m, P) in float4 groups
  extern __shared__ float sm[];
  const int vc = blockIdx.x * blockDim.x + threadIdx.x;
  if (vc >= n_vch) return;
  const int c = vc % M.n_chunks;
  const int set = vc / M.n_chunks;
  const int s = M.ch_series[c];
  const int row = per_series ? s : set;
  const int orow = per_series ? s : set * M.n_series + s;
  TermC<F> tc[S::NT];
  F s2;
  load_terms<S::NT, F>(theta + (size_t)row * M.n_params, M.kinds, tc, s2);
  // shared memory: the warps' tables, then GRAD_STAGES staging buffers per
  // thread for the backward walk, stg[(buf (SG + NDG) + group) bs + thread]
  float4 *tab_slots = reinterpret_cast<float4 *>(sm);
  const int bs = blockDim.x;
  float4 *stg = tab_slots + (bs / 32) * (S::NT * TAB_TERM / 4) + threadIdx.x;
  const float4 *tab = stage_table<S::NT>(tabs, row, tab_slots + (threadIdx.x >> 5) * (S::NT * TAB_TERM / 4));
  // EX: conditioned outputs, predictions or exposure gradients requested
  auto body = [&](auto od_tag, auto ex_tag) {
    constexpr bool OD = decltype(od_tag)::value;
    constexpr bool EX = decltype(ex_tag)::value;
    const uint8_t flags = M.ch_flags[c];
    const bool first = flags & 1, last = flags & 2;
    F m[D], P[S::NP];
    const int64_t e0 = M.ch_ev0[c];
    const int len = M.ch_len[c];
    const int nseg = (len + ck - 1) / ck;
    const int f0 = len - (nseg - 1) * ck;
    F lam[D], Lam[S::NP];
    if (last) {
  #pragma unroll
      for (int i = 0; i < D; ++i) lam[i] = F(0);
  #pragma unroll
      for (int i = 0; i < S::NP; ++i) Lam[i] = F(0);
    } else {
      load_rec<S>(adj_end, n_vch, vc, lam, Lam);
    }
    TermGrad<S::NT> gr;
  #pragma unroll
    for (int t = 0; t < S::NT; ++t) gr.a[t] = gr.beta[t] = gr.w2[t] = gr.qc[t] = gr.var[t] = F(0);
    gr.s2 = F(0);
    // per-event exposure adjoints of this chunk (theta set `set`)
    const int64_t eo = (int64_t)set * M.n_events + e0;
    float4 *my = reinterpret_cast<float4 *>(rbuf) + vc;  // group v of slot k at (k SG + v) n_vch
    const size_t rs = (size_t)n_vch;
    const float4 *dc = dcache_col<S::NT>(M, const_cast<float *>(dcache), vc);
    bool bad = false;
    for (int seg = nseg - 1; seg >= 0; --seg) {
      const int k0 = seg == 0 ? 0 : f0 + (seg - 1) * ck;
      const int k1 = seg == 0 ? f0 : k0 + ck;
      if (seg == 0) {
        if (first)
          init_state<S>(tc, m, P);
        else
          load_state_f<S>(state_end, se64, n_vch, vc - 1, m, P);
      } else {
        F mi[D], Pi[S::NP];
        if (first) {
          // the first chunk's element already starts from the prior (A = 0)
  #pragma unroll
          for (int i = 0; i < D; ++i) mi[i] = F(0);
  #pragma unroll
          for (int i = 0; i < S::NP; ++i) Pi[i] = F(0);
        } else {
          load_state_f<S>(state_end, se64, n_vch, vc - 1, mi, Pi);
        }
        const float *src = pck + (size_t)(seg - 1) * (NF + 1) * n_vch;
        apply_partial<S>(src, n_vch, vc, mi, Pi, m, P);
      }
      // forward replay of the segment (step scalars from the cache, the next
      // step's loaded one ahead, or recomputed)
      EventReader rd;
      rd.start(M, c, k0, k1);
      const float4 *dcr = dc ? dc + (size_t)k0 * (32 * NDG) : nullptr;
      float nx[NDC];
      if (dcr) dcache_load<S::NT>(dcr, nx);
      for (int kk = k0; kk < k1; ++kk) {
        const int slot = kk - k0;
        {
          float r[4 * SG];
  #pragma unroll
          for (int i = 0; i < D; ++i) r[i] = m[i];
  #pragma unroll
          for (int i = 0; i < S::NP; ++i) r[D + i] = P[i];
  #pragma unroll
          for (int i = SD; i < 4 * SG; ++i) r[i] = 0.f;
  #pragma unroll
          for (int v = 0; v < SG; ++v)
            my[(size_t)(slot * SG + v) * rs] = make_float4(r[4 * v], r[4 * v + 1], r[4 * v + 2], r[4 * v + 3]);
        }
        F dt, Sv, vv;
        uint8_t tag;
        float4 q;
        rd.next(dt, tag, q);
        Blocks<F> B[S::NT];
        if (dcr) {
  #pragma unroll
          for (int t = 0; t < S::NT; ++t) B[t] = make_blocks(dcache_term<S::NT>(nx, t), tc[t]);
          dcr += 32 * NDG;
          if (kk + 1 < k1) dcache_load<S::NT>(dcr, nx);
        } else {
  #pragma unroll
          for (int t = 0; t < S::NT; ++t)
            B[t] = make_blocks(discretize_tab<OD>(dt, tc[t], tab + t * (TAB_TERM / 4)), tc[t]);
        }
        if (filter_blocks<S, F, OD>(B, tag, q.x, q.y, q.z, s2, m, P, Sv, vv)) bad |= !(Sv > F(0));
      }
      // conditioned mean and variance of the chunk's last event, if it ends an
      // exposure: the chunk's end state and its boundary adjoint
      if (EX && cond && seg == nseg - 1 && (__ldg(M.ilv_tag + lane_step(M, c, k1 - 1)) & 1)) {
        const int64_t il = lane_step(M, c, k1 - 1);
        const uint8_t tl = __ldg(M.ilv_tag + il);
        const float4 rl = __ldg(M.ilv + il);
        F mb[D], Pb[S::NP];
        load_state_f<S>(state_end, se64, n_vch, vc, mb, Pb);
        cond[eo + k1 - 1] = conditioned_tag<S, OD>(tl, rl.w, mb, Pb, lam, Lam);
      }
      // test times after the series' last event: predicted from its filtered
      // state (which all the data already conditions)
      if (EX && pp.off && last && seg == nseg - 1) {
        F mb[D], Pb[S::NP], z[D], Z[S::NP];
        load_state_f<S>(state_end, se64, n_vch, vc, mb, Pb);
  #pragma unroll
        for (int i = 0; i < D; ++i) z[i] = F(0);
  #pragma unroll
        for (int i = 0; i < S::NP; ++i) Z[i] = F(0);
        for (int jj = pp.xoff[s]; jj < pp.xoff[s + 1]; ++jj) {
          const float2 r = predict_point<S, OD>(pp.d[jj].x, 0.f, tc, tab, mb, Pb, z, Z);
          float *o = pp.out + ((int64_t)set * pp.n_star + pp.idx[jj]) * 2;
          o[0] = r.x;
          o[1] = r.y;
        }
      }
      // backward walk.  The earlier step's replayed state and cached scalars
      // are staged into shared memory by cp.async while the current step is
      // processed; its lane-step record and tag are loaded one ahead.
      auto stage = [&](int buf, int slot, int kk) {
        float4 *dst = stg + (size_t)buf * (SG + NDG) * bs;
  #pragma unroll
        for (int v = 0; v < SG; ++v) cp_async16(dst + v * bs, my + (size_t)(slot * SG + v) * rs);
        if (dc) {
          const float4 *src = dc + (size_t)kk * (32 * NDG);
  #pragma unroll
          for (int v = 0; v < NDG; ++v) cp_async16(dst + (SG + v) * bs, src + 32 * v);
        }
        cp_async_commit();
      };
      int k2 = k1 - 1;
      int64_t li = lane_step(M, c, k2);
      float4 r_n = __ldg(M.ilv + li);
      uint8_t tag_n = __ldg(M.ilv_tag + li);
      // GRAD_STAGES - 1 steps are staged ahead (empty groups past the
      // segment's start keep the group count uniform)
#pragma unroll
      for (int p = 0; p < GRAD_STAGES - 1; ++p) {
        if (k2 - p >= k0)
          stage(p, k2 - p - k0, k2 - p);
        else
          cp_async_commit();
      }
      for (int it = 0; k2 >= k0; --k2, ++it) {
        const int buf = it % GRAD_STAGES;
        const F dt = r_n.x;
        const uint8_t tag = tag_n;
        const float4 q = make_float4(r_n.y, r_n.z, r_n.w, 0.f);
        if (k2 > k0) {
          li -= 32;
          r_n = __ldg(M.ilv + li);
          tag_n = __ldg(M.ilv_tag + li);
        }
        {
          const int ka = k2 - (GRAD_STAGES - 1);
          if (ka >= k0)
            stage((it + GRAD_STAGES - 1) % GRAD_STAGES, ka - k0, ka);
          else
            cp_async_commit();
          cp_async_wait<GRAD_STAGES - 1>();
        }
        const float4 *sb = stg + (size_t)buf * (SG + NDG) * bs;
        // the extra outputs read (m, P) as arrays; so does the lean body of a
        // shape without integral states, whose smaller state fits in registers
        // (reading it from shared memory there measured slower)
        constexpr bool ARR = EX || S::NS == 0;
        if constexpr (ARR) {
          float r[4 * SG];
  #pragma unroll
          for (int v = 0; v < SG; ++v) {
            const float4 g4 = sb[v * bs];
            r[4 * v] = g4.x;
            r[4 * v + 1] = g4.y;
            r[4 * v + 2] = g4.z;
            r[4 * v + 3] = g4.w;
          }
  #pragma unroll
          for (int i = 0; i < D; ++i) m[i] = r[i];
  #pragma unroll
          for (int i = 0; i < S::NP; ++i) P[i] = r[D + i];
        }
        Disc<F> dv[S::NT];
        if (dc) {
  #pragma unroll
          for (int v = 0; v < NDG; ++v) {
            const float4 g4 = sb[(SG + v) * bs];
            nx[4 * v] = g4.x;
            nx[4 * v + 1] = g4.y;
            nx[4 * v + 2] = g4.z;
            nx[4 * v + 3] = g4.w;
          }
  #pragma unroll
          for (int t = 0; t < S::NT; ++t) dv[t] = dcache_term<S::NT>(nx, t);
        } else {
  #pragma unroll
          for (int t = 0; t < S::NT; ++t) dv[t] = discretize_tab<OD>(dt, tc[t], tab + t * (TAB_TERM / 4));
        }
        F g_dt, g_w;
        // test times in (t_{k2-1}, t_{k2}] (before the data for the series'
        // first event): predicted from (m, P), smoothed from this event's adjoint
        auto hook = [&](const float *lp, const float *Lp) {
          if (!EX || !pp.off) return;
          const int64_t e = e0 + k2;
          for (int jj = pp.off[e]; jj < pp.off[e + 1]; ++jj) {
            const float2 d = pp.d[jj];
            const float2 r = predict_point<S, OD>(d.x, d.y, tc, tab, m, P, lp, Lp);
            float *o = pp.out + ((int64_t)set * pp.n_star + pp.idx[jj]) * 2;
            o[0] = r.x;
            o[1] = r.y;
          }
        };
        if constexpr (ARR)
          reverse_event<S, OD, decltype(hook), const float *>(dt, tag, q, tc, s2, m, P, lam, Lam, gr, tab,
                                                              dv, gdt != nullptr, g_dt, g_w, hook);
        else
          reverse_event<S, OD, NoHook, StagedRec>(dt, tag, q, tc, s2, StagedRec{sb, bs, 0},
                                                  StagedRec{sb, bs, D}, lam, Lam, gr, tab, dv, false,
                                                  g_dt, g_w);
        if (EX && gdt) {
          gdt[eo + k2] = g_dt;
          if (tag & 1) gwe[eo + k2] = q.z * q.z * g_w;
        }
        // (m, P) is the filtered state after event k2 - 1 and (lam, Lam) now its
        // adjoint: the conditioned values of that event's measurement
        if (EX && cond && k2 > 0) {
          const int64_t lp = lane_step(M, c, k2 - 1);
          const uint8_t tp = k2 > k0 ? tag_n : __ldg(M.ilv_tag + lp);
          if (tp & 1) {
            const float wp = k2 > k0 ? r_n.w : __ldg(M.ilv + lp).w;
            cond[eo + k2 - 1] = conditioned_tag<S, OD>(tp, wp, m, P, lam, Lam);
          }
        }
      }
    }
    if (first) {
      // P0 = blkdiag(var diag(1, w2), I)
  #pragma unroll
      for (int t = 0; t < S::NT; ++t) {
        gr.var[t] += Lam[S::pk(2 * t, 2 * t)] + tc[t].w2 * Lam[S::pk(2 * t + 1, 2 * t + 1)];
        gr.w2[t] += tc[t].var * Lam[S::pk(2 * t + 1, 2 * t + 1)];
      }
    }
    // chain to natural parameters
    const float *th = theta + (size_t)row * M.n_params;
    float *g = gpart + vc;
    const size_t gs = (size_t)n_vch;
    int p = 0;
  #pragma unroll
    for (int t = 0; t < S::NT; ++t) {
      const F ga = gr.a[t] + F(2) * tc[t].a * gr.w2[t];
      const F gb = gr.beta[t] + gr.w2[t];
      if (M.kinds[t] == 1) {
        const F sig = th[p], w0 = th[p + 1], q = th[p + 2];
        const F dsig = gr.qc[t] * F(4) * w0 * w0 * w0 * sig / q + gr.var[t] * F(2) * sig;
        const F dw0 = ga / (F(2) * q) + gb * F(2) * w0 * (F(1) - F(1) / (F(4) * q * q)) +
                      gr.qc[t] * F(6) * w0 * w0 * sig * sig / q;
        const F dq = -ga * w0 / (F(2) * q * q) + gb * w0 * w0 / (F(2) * q * q * q) -
                     gr.qc[t] * F(2) * w0 * w0 * w0 * sig * sig / (q * q);
        g[p * gs] = dsig;
        g[(p + 1) * gs] = dw0;
        g[(p + 2) * gs] = dq;
        p += 3;
      } else {
        const F sig = th[p], ell = th[p + 1];
        const F w0 = F(1.7320508075688772) / ell;
        const F dsig = gr.qc[t] * F(8) * w0 * w0 * w0 * sig + gr.var[t] * F(2) * sig;
        // a = w0, w2 = w0^2 (through ga), qc = 4 w0^3 sig^2 ; beta = 0 along this family
        const F dw0 = gr.a[t] + F(2) * w0 * gr.w2[t] + gr.qc[t] * F(12) * w0 * w0 * sig * sig;
        g[p * gs] = dsig;
        g[(p + 1) * gs] = dw0 * (-w0 / ell);
        p += 2;
      }
    }
    g[p * gs] = gr.s2 * F(2) * th[p];
    if (bad) flag_error(err, orow, 7);
  };
  // rows with an overdamped term, and every row of a mixed model, take the
  // general body; the others the lean one unless extra outputs are requested
  if (any_overdamped<S::NT>(tc) || M.mixed)
    body(OdTag<true>{}, OdTag<true>{});
  else if (cond || pp.off || gdt)
    body(OdTag<false>{}, OdTag<true>{});
  else
    body(OdTag<false>{}, OdTag<false>{});
}

// Ordered per-series sums over chunks (deterministic): log-likelihood parts
// and gradient parts (field-major, stride n_vch), FP64 accumulation.
__global__ void k_series_sum(int n_out, int per_series, int n_series, int n_chunks,
                             const int32_t *__restrict__ ch_first,
                             const double *__restrict__ ll_part, int n_vch,
                             const float *__restrict__ gpart, int n_params,
                             double *__restrict__ ll_out, float *__restrict__ grad_out);

// Exposure-window gradient per measurement (input order) from the per-event
// adjoints of k_grad: d/dt_start = gt(start) + gwe(end), d/dt_end = gt(end) -
// gwe(end), where gt(k) = gdt(k) - gdt(k+1) (the event's time ends the gap
// before it and starts the one after it; a series' first event sets the
// initial time, so its own gap is always zero).  out[(row N + n) 2 + {0,1}].
__global__ void k_exposure_grad(int n_rows, int n_series, const int64_t *__restrict__ ev_off,
                                const int64_t *__restrict__ meas_off,
                                const int2 *__restrict__ mev, int64_t n_meas, int64_t n_events,
                                const float *__restrict__ gdt, const float *__restrict__ gwe,
                                float *__restrict__ out);

// Per measurement (input order): the conditioned (mean, variance) k_grad
// wrote at its end event.  out[(row N + n) 2 + {0,1}].
__global__ void k_gather_cond(int n_rows, int n_series, const int64_t *__restrict__ ev_off,
                              const int64_t *__restrict__ meas_off, const int2 *__restrict__ mev,
                              int64_t n_meas, int64_t n_events, const float2 *__restrict__ cond,
                              float *__restrict__ out);

// Dense Phi~(dt_k), Q~(dt_k) for a list of gaps (one thread per gap).
template <class S>
__global__ void k_disc(const float *__restrict__ theta, const float *__restrict__ tabs, int kinds0,
                       int kinds1, const float *__restrict__ dt, int n, float *__restrict__ phi,
                       float *__restrict__ q) {
  constexpr int D = S::D;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  int kk[4] = {kinds0, kinds1, 0, 0};
  TermC<float> tc[S::NT];
  float s2;
  load_terms<S::NT, float>(theta, kk, tc, s2);
  const float4 *tab = reinterpret_cast<const float4 *>(tabs);
  Blocks<float> B[S::NT];
#pragma unroll
  for (int t = 0; t < S::NT; ++t)
    B[t] = make_blocks(discretize_tab(dt[k], tc[t], tab + t * (TAB_TERM / 4)), tc[t]);
  float P[S::NP];
#pragma unroll
  for (int i = 0; i < S::NP; ++i) P[i] = 0.f;
  add_q<S>(B, P);
  float *ph = phi + (size_t)k * D * D, *qq = q + (size_t)k * D * D;
#pragma unroll
  for (int c = 0; c < D; ++c) {
    float e[D], o[D];
#pragma unroll
    for (int i = 0; i < D; ++i) e[i] = (i == c) ? 1.f : 0.f;
    apply_phi<S>(B, e, o);
#pragma unroll
    for (int i = 0; i < D; ++i) {
      ph[i * D + c] = o[i];
      qq[i * D + c] = P[S::pk(i, c)];
    }
  }
}

// ---------------------------------------------------------------------------
// A series split in time (Section 3.2.5 across devices): the chunks
// [c_begin, c_end) of every row combined into one element with its
// log-normaliser c (Elem fields, then c; NC = NF + 1 values, FP64).  Each
// level reduces tiles of SPAN_T items by a tree of combinations in shared
// memory; the first level reads the chunk elements, later ones the tile
// totals ([row][item][field]).  Folding the spans' elements in time order
// gives the series' log-likelihood in c (the first span starts from the
// prior, A = 0).
// ---------------------------------------------------------------------------
constexpr int SPAN_T = 64;

template <class S>
constexpr size_t span_smem_bytes() {
  return (size_t)SPAN_T * (Elem<S>::NF + 1) * sizeof(double);
}

template <class S, bool FROM_CHUNKS>
__global__ void __launch_bounds__(SPAN_T) k_span_reduce(const float *__restrict__ ef,
                                                        const double *__restrict__ ed,
                                                        int n_vch, int n_chunks, int c_begin,
                                                        const double *__restrict__ src, int n,
                                                        double *__restrict__ dst,
                                                        int n_out_tiles) {
  constexpr int NF = Elem<S>::NF, NC = NF + 1;
  extern __shared__ __align__(16) unsigned char sm_raw[];
  double *sm = reinterpret_cast<double *>(sm_raw);
  const int tile = blockIdx.x, row = blockIdx.y, tid = threadIdx.x;
  const int i0 = tile * SPAN_T;
  const int len = min(SPAN_T, n - i0);
  EViewT<double> mine{sm + tid, SPAN_T};
  if (tid < len) {
    const int i = i0 + tid;
    if (FROM_CHUNKS) {
      const size_t vc = (size_t)row * n_chunks + c_begin + i;
      for (int f = 0; f < NF; ++f) mine[f] = (double)ef[(size_t)f * n_vch + vc];
      const double gam = ed[vc], ld = ed[(size_t)n_vch + vc], ne = ed[(size_t)2 * n_vch + vc];
      mine[NF] = -0.5 * (ld + gam + ne * LOG_2PI);
    } else {
      for (int f = 0; f < NC; ++f) mine[f] = src[((size_t)row * n + i) * NC + f];
    }
  }
  __syncthreads();
  for (int s = 1; s < SPAN_T; s <<= 1) {
    if ((tid % (2 * s)) == 0 && tid + s < len)
      combine<S, double, true>(mine, EViewT<double>{sm + tid + s, SPAN_T}, mine);
    __syncthreads();
  }
  if (tid == 0)
    for (int f = 0; f < NC; ++f) dst[((size_t)row * n_out_tiles + tile) * NC + f] = mine[f];
}

// Fold the spans' elements [span][row][NC] in time order, one thread per
// row; the log-normaliser of the whole is the series' log-likelihood.
template <class S>
__global__ void k_span_fold(const double *__restrict__ elems, int n_spans, int n_rows,
                            double *__restrict__ ll_out) {
  constexpr int NC = Elem<S>::NF + 1;
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= n_rows) return;
  double acc[NC], nxt[NC], out[NC];
  for (int f = 0; f < NC; ++f) acc[f] = elems[(size_t)row * NC + f];
  for (int sp = 1; sp < n_spans; ++sp) {
    for (int f = 0; f < NC; ++f) nxt[f] = elems[((size_t)sp * n_rows + row) * NC + f];
    combine<S, double, true>(EViewT<double>{acc, 1}, EViewT<double>{nxt, 1},
                             EViewT<double>{out, 1});
    for (int f = 0; f < NC; ++f) acc[f] = out[f];
  }
  ll_out[row] = acc[NC - 1];
}

// Element of chunks [c_begin, c_end) of each of n_rows rows (the chunk
// elements already in ef / ed) -> elem_out [n_rows][NC].  scratch: at least
// span_scratch_count(c_end - c_begin, n_rows) doubles.
template <class S>
size_t span_scratch_count(int n, int n_rows) {
  size_t tot = 0;
  while (n > 1) {
    n = (n + SPAN_T - 1) / SPAN_T;
    tot += (size_t)n * n_rows * (Elem<S>::NF + 1);
  }
  return tot + 1;
}

template <class S>
cudaError_t launch_span_element(const float *ef, const double *ed, int n_vch, int n_chunks,
                                int c_begin, int c_end, int n_rows, double *scratch,
                                double *elem_out, cudaStream_t st) {
  constexpr int NC = Elem<S>::NF + 1;
  const size_t smem = span_smem_bytes<S>();
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_span_reduce<S, true>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_span_reduce<S, false>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  int n = c_end - c_begin;
  if (n <= 0 || n_rows <= 0) return cudaErrorInvalidValue;
  const double *src = nullptr;
  double *buf = scratch;
  bool first = true;
  do {
    const int nt = (n + SPAN_T - 1) / SPAN_T;
    double *dst = nt == 1 ? elem_out : buf;
    if (first)
      k_span_reduce<S, true><<<dim3(nt, n_rows), SPAN_T, smem, st>>>(
          ef, ed, n_vch, n_chunks, c_begin, nullptr, n, dst, nt);
    else
      k_span_reduce<S, false><<<dim3(nt, n_rows), SPAN_T, smem, st>>>(
          nullptr, nullptr, 0, 0, 0, src, n, dst, nt);
    GPSS_COUNT_LAUNCH();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    src = dst;
    buf += (size_t)nt * n_rows * NC;
    n = nt;
    first = false;
  } while (n > 1);
  return cudaSuccess;
}

template <class S>
cudaError_t launch_span_fold(const double *elems, int n_spans, int n_rows, double *ll,
                             cudaStream_t st) {
  if (n_spans <= 0 || n_rows <= 0) return cudaErrorInvalidValue;
  k_span_fold<S><<<(n_rows + 63) / 64, 64, 0, st>>>(elems, n_spans, n_rows, ll);
  GPSS_COUNT_LAUNCH();
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Host launchers, one table per compiled shape.
// ---------------------------------------------------------------------------
// Cross-chunk combination in one arithmetic (FP32 or FP64): the sequential
// fold per series, the warp-level scans with the scan or fold of warp totals
// and the per-chunk join, and the chunk log-likelihoods with the boundary
// adjoints.  Buffers other than the chunk elements (FP32) and the adjoints
// (FP32) hold elem_bytes per value.
struct CombineOps {
  int elem_bytes;
  cudaError_t (*scan)(const DevModel &, int, int, const float *, const double *, int, void *,
                      float *, double *, int, int *, cudaStream_t);
  cudaError_t (*warp_combine)(const DevModel &, const float *, int, void *, void *, void *,
                              void *, void *, void *, void *, void *, int, int, int, int,
                              cudaStream_t);
  size_t (*warp_scratch)(int);  // values of the scan of warp totals
  cudaError_t (*finish)(const DevModel &, int, int, const float *, const double *, const void *,
                        const void *, float *, double *, int *, cudaStream_t);
};

struct OpTable {
  int D, NP, NF, ND;
  cudaError_t (*plain32)(const DevModel &, const float *, int, int, double *, int *, cudaStream_t);
  cudaError_t (*plain64)(const DevModel &, const float *, int, int, double *, int *, cudaStream_t);
  cudaError_t (*elem)(const DevModel &, const float *, int, int, float *, double *, int *,
                      const float *, float *, int, float *, int, int, cudaStream_t);
  cudaError_t (*grad)(const DevModel &, const float *, int, int, const void *, int,
                      const float *, const float *, float *, int *, const float *, float *,
                      const float *, int, float *, float *, float2 *, const PredPlan &,
                      cudaStream_t);
  cudaError_t (*tables)(const float *, int, int, int, int, float *, cudaStream_t);
  CombineOps comb32, comb64;  // the combination in FP32 / FP64
  int NT;
  cudaError_t (*disc)(const float *, const float *, int, int, const float *, int, float *, float *,
                      cudaStream_t);
  // product models: log-likelihood and hyperparameter gradient (else null)
  cudaError_t (*prod_grad)(const DevModel &, const float *, int, int, double *, float *, int *,
                           cudaStream_t);
  // product models, chunked schedule: gradient parts per (chunk, parameter)
  // from the combination's incoming states and boundary adjoints (else null)
  cudaError_t (*prod_grad_chunk)(const DevModel &, const float *, int, int, const void *, int,
                                 const float *, float *, int *, cudaStream_t);
  // a series split in time: element of a chunk range, fold of span elements
  cudaError_t (*span_element)(const float *, const double *, int, int, int, int, int, double *,
                              double *, cudaStream_t);
  size_t (*span_scratch)(int, int);
  cudaError_t (*span_fold)(const double *, int, int, double *, cudaStream_t);
};


template <class S, class F>
cudaError_t launch_plain(const DevModel &M, const float *theta, int n_out, int per_series,
                         double *ll, int *err, cudaStream_t st) {
  if (n_out <= 0) return cudaSuccess;
  const int bs = 128;
  k_plain<S, F><<<(n_out + bs - 1) / bs, bs, 0, st>>>(M, theta, n_out, per_series, ll, err);
  GPSS_COUNT_LAUNCH();
  return cudaGetLastError();
}

template <class S>
cudaError_t launch_elem(const DevModel &M, const float *theta, int n_vch, int per_series,
                        float *ef, double *ed, int *err, const float *tabs, float *pck, int ck,
                        float *dcache, int c_begin, int c_count, cudaStream_t st) {
  if (n_vch <= 0 || c_count <= 0) return cudaSuccess;
  if (c_begin < 0 || c_begin + c_count > M.n_chunks) return cudaErrorInvalidValue;
  if (pck && (ck < 2 || ck > 64 || (ck & 1))) return cudaErrorInvalidValue;
  const int bs = 128;
  const size_t smem = (size_t)(bs / 32) * S::NT * TAB_TERM * sizeof(float);
  // two launches: rows without an overdamped term (the lean body), then rows
  // with one; each skips the other's rows
  const int64_t nt = (int64_t)(n_vch / M.n_chunks) * c_count;
  const int nb = (int)((nt + bs - 1) / bs);
  k_elem<S, false><<<nb, bs, smem, st>>>(M, theta, n_vch, per_series, ef, ed, err, tabs, pck,
                                         pck ? ck : 1, dcache, c_begin, c_count);
  GPSS_COUNT_LAUNCH();
  k_elem<S, true><<<nb, bs, smem, st>>>(M, theta, n_vch, per_series, ef, ed, err, tabs, pck,
                                        pck ? ck : 1, dcache, c_begin, c_count);
  GPSS_COUNT_LAUNCH();
  return cudaGetLastError();
}

template <class S>
cudaError_t launch_tables(const float *theta, int n_rows, int n_params, int k0, int k1,
                          float *tab, cudaStream_t st) {
  const int n = n_rows * S::NT;
  if (n <= 0) return cudaSuccess;
  static const EconMap E = [] {
    EconMap e;
    econ_map(e);
    return e;
  }();
  k_tables<S::NT><<<(n + TABLE_WARPS - 1) / TABLE_WARPS, 32 * TABLE_WARPS, 0, st>>>(
      theta, n_rows, n_params, k0, k1, tab, E);
  GPSS_COUNT_LAUNCH();
  return cudaGetLastError();
}

template <class S, class T>
cudaError_t launch_scan(const DevModel &M, int n_out, int per_series, const float *ef,
                        const double *ed, int n_vch, void *state_end, float *adj_end, double *ll,
                        int want_grad, int *err, cudaStream_t st) {
  if (n_out <= 0) return cudaSuccess;
  const int bs = 64;
  k_scan_seq<S, T><<<(n_out + bs - 1) / bs, bs, 0, st>>>(M, n_out, per_series, ef, ed, n_vch,
                                                        static_cast<T *>(state_end), adj_end, ll,
                                                        want_grad, err);
  GPSS_COUNT_LAUNCH();
  return cudaGetLastError();
}

// Warp-level combination (k_warp_scan, scan of warp totals, k_join): writes
// state_end (and info_incl when want_info), records of T.  Buffers of T:
// pre_local, suf_local [NF * n_vch]; wtot, wpre, wsuf [NF * n_vch/32];
// scratch [warp_scratch values].
template <class S, class T>
cudaError_t launch_warp_combine(const DevModel &M, const float *ef, int n_vch, void *pre_local_v,
                                void *suf_local_v, void *wtot_v, void *wpre_v, void *wsuf_v,
                                void *scratch_v, void *state_end_v, void *info_incl_v,
                                int want_info, int fold, int n_out, int per_series,
                                cudaStream_t st) {
  if (n_vch <= 0) return cudaSuccess;
  T *pre_local = static_cast<T *>(pre_local_v), *suf_local = static_cast<T *>(suf_local_v);
  T *wtot = static_cast<T *>(wtot_v), *wpre = static_cast<T *>(wpre_v),
    *wsuf = static_cast<T *>(wsuf_v), *scratch = static_cast<T *>(scratch_v);
  T *state_end = static_cast<T *>(state_end_v), *info_incl = static_cast<T *>(info_incl_v);
  const int n_w = n_vch / 32;
  const size_t smem = warp_scan_smem_bytes<S, T>(2);
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_warp_scan<S, T>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  k_warp_scan<S, T><<<(n_vch + 63) / 64, 64, smem, st>>>(ef, n_vch, pre_local, suf_local, wtot,
                                                         want_info);
  GPSS_COUNT_LAUNCH();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (fold) {
    // few warps per series: sequential fold of the warp totals per series
    k_warp_fold<S, T><<<(n_out + 63) / 64, 64, 0, st>>>(n_out, per_series, M.n_series,
                                                        M.n_chunks, M.ch_first, wtot, n_w, wpre,
                                                        wsuf, want_info);
    GPSS_COUNT_LAUNCH();
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  } else {
    e = scan_elems<S, T>(wtot, n_w, wpre, 0, 0, 0, scratch, st);
    if (e != cudaSuccess) return e;
    if (want_info) {
      e = scan_elems<S, T>(wtot, n_w, wsuf, 3, 1, 1, scratch, st);
      if (e != cudaSuccess) return e;
    }
  }
  k_join<S, T><<<(n_vch + 127) / 128, 128, 0, st>>>(n_vch, M.n_chunks, M.ch_flags, pre_local,
                                                    suf_local, wpre, wsuf, state_end,
                                                    want_info ? info_incl : nullptr);
  GPSS_COUNT_LAUNCH();
  return cudaGetLastError();
}

template <class S>
size_t warp_scratch_count(int n_vch) {
  return scan_scratch_count<S>(n_vch / 32);
}

template <class S, class T>
cudaError_t launch_finish(const DevModel &M, int n_vch, int per_series, const float *ef,
                          const double *ed, const void *state_end, const void *info_incl,
                          float *adj_end, double *ll_part, int *err, cudaStream_t st) {
  if (n_vch <= 0) return cudaSuccess;
  k_finish<S, T><<<(n_vch + 127) / 128, 128, 0, st>>>(
      M, n_vch, per_series, ef, ed, static_cast<const T *>(state_end),
      static_cast<const T *>(info_incl), adj_end, ll_part, err);
  GPSS_COUNT_LAUNCH();
  return cudaGetLastError();
}

template <class S, class T>
CombineOps make_combine() {
  CombineOps c;
  c.elem_bytes = (int)sizeof(T);
  c.scan = &launch_scan<S, T>;
  c.warp_combine = &launch_warp_combine<S, T>;
  c.warp_scratch = &warp_scratch_count<S>;
  c.finish = &launch_finish<S, T>;
  return c;
}

// ck: events per recomputation segment (even, 2..64), the value k_elem saved
// the partial elements pck with ([(max_len-1)/ck] * (NF+1) * n_vch floats).
// Scratch: rbuf [ck * 4 ceil(SD/4) * n_vch] floats.  dcache: the step-scalar
// cache k_elem filled, or null (the replay then recomputes the scalars).
// gdt, gwe: per-event exposure adjoints [rows * n_events] (see k_grad), or
// null when the exposure gradient is not wanted; cond: per-event conditioned
// (mean, variance) of end events [rows * n_events], or null.
template <class S>
cudaError_t launch_grad(const DevModel &M, const float *theta, int n_vch, int per_series,
                        const void *state_end, int se64, const float *adj_end, const float *pck,
                        float *gpart, int *err, const float *tabs, float *rbuf,
                        const float *dcache, int ck, float *gdt, float *gwe, float2 *cond,
                        const PredPlan &pp, cudaStream_t st) {
  if (n_vch <= 0) return cudaSuccess;
  if (ck < 2 || ck > 64 || (ck & 1)) return cudaErrorInvalidValue;
  const int SG = (S::D + S::NP + 3) / 4, NDG = DcW<S::NT>::G;
  const size_t smem = (size_t)(GRAD_BS / 32) * S::NT * TAB_TERM * sizeof(float) +
                      (size_t)GRAD_STAGES * (SG + NDG) * GRAD_BS * sizeof(float4);
  k_grad<S><<<(n_vch + GRAD_BS - 1) / GRAD_BS, GRAD_BS, smem, st>>>(
      M, theta, n_vch, per_series, state_end, se64, adj_end, pck, gpart, err, tabs, rbuf, dcache,
      ck, gdt, gwe, cond, pp);
  GPSS_COUNT_LAUNCH();
  return cudaGetLastError();
}

template <class S>
cudaError_t launch_disc(const float *theta, const float *tabs, int k0, int k1, const float *dt,
                        int n, float *phi, float *q, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_disc<S><<<(n + 127) / 128, 128, 0, st>>>(theta, tabs, k0, k1, dt, n, phi, q);
  GPSS_COUNT_LAUNCH();
  return cudaGetLastError();
}

// The operation table of a shape; the FP64 combination (comb64) is filled
// by make_ops_c64, compiled in its own translation unit.
template <class S>
OpTable make_ops() {
  OpTable o{};
  o.D = S::D;
  o.NP = S::NP;
  o.NF = ElemLayout<S>::NF;
  o.ND = ElemLayout<S>::ND;
  o.plain32 = &launch_plain<S, float>;
  o.plain64 = &launch_plain<S, double>;
  o.elem = &launch_elem<S>;
  o.grad = &launch_grad<S>;
  o.disc = &launch_disc<S>;
  o.comb32 = make_combine<S, float>();
  o.tables = &launch_tables<S>;
  o.NT = S::NT;
  o.prod_grad = nullptr;
  o.span_element = &launch_span_element<S>;
  o.span_scratch = &span_scratch_count<S>;
  o.span_fold = &launch_span_fold<S>;
  return o;
}

}  // namespace gpss
