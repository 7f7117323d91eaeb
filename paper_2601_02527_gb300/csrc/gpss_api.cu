// Host side of the libgpss C ABI: event building (Section 3.2 of arXiv
// 2601.02527), validation, chunk planning, device buffers and dispatch.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <numeric>
#include <thread>
#include <tuple>
#include <vector>

#include "gpss.h"
#include "gpss_kernels.cuh"

namespace gpss {
OpTable ops_1_1_0();
OpTable ops_1_2_0();
OpTable ops_1_3_0();
OpTable ops_2_1_0();
OpTable ops_2_2_0();
OpTable ops_2_3_0();
OpTable ops_2_1_1();
OpTable ops_1_0_0();
OpTable ops_2_0_0();
OpTable ops_prod1();
OpTable ops_prod2();
CombineOps comb64_1_0_0();
CombineOps comb64_1_1_0();
CombineOps comb64_1_2_0();
CombineOps comb64_1_3_0();
CombineOps comb64_2_0_0();
CombineOps comb64_3_0_0();
CombineOps comb64_2_1_0();
CombineOps comb64_2_2_0();
CombineOps comb64_2_1_1();
CombineOps comb64_2_3_0();

__global__ void k_series_sum(int n_out, int per_series, int n_series, int n_chunks,
                             const int32_t *__restrict__ ch_first,
                             const double *__restrict__ ll_part, int n_vch,
                             const float *__restrict__ gpart, int n_params,
                             double *__restrict__ ll_out, float *__restrict__ grad_out) {
  // one warp per output row; lanes stride over the row's chunks and a fixed
  // shuffle tree combines them (the same order on every call)
  const int v = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (v >= n_out) return;
  const int s = per_series ? v : v % n_series;
  const int base = per_series ? 0 : (v / n_series) * n_chunks;
  const int c0 = ch_first[s], c1 = ch_first[s + 1];
  if (ll_part) {
    double acc = 0.0;
    for (int c = c0 + lane; c < c1; c += 32) acc += ll_part[base + c];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) ll_out[v] = acc;
  }
  if (gpart) {
    for (int p = 0; p < n_params; ++p) {
      double acc = 0.0;
      const float *g = gpart + (size_t)p * n_vch + base;
      for (int c = c0 + lane; c < c1; c += 32) acc += (double)g[c];
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
      if (lane == 0) grad_out[(size_t)v * n_params + p] = (float)acc;
    }
  }
}

__global__ void k_exposure_grad(int n_rows, int n_series, const int64_t *__restrict__ ev_off,
                                const int64_t *__restrict__ meas_off,
                                const int2 *__restrict__ mev, int64_t n_meas, int64_t n_events,
                                const float *__restrict__ gdt, const float *__restrict__ gwe,
                                float *__restrict__ out) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)n_rows * n_meas) return;
  const int64_t row = idx / n_meas, n = idx % n_meas;
  // series of measurement n: last s with meas_off[s] <= n
  int lo = 0, hi = n_series - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (meas_off[mid] <= n)
      lo = mid;
    else
      hi = mid - 1;
  }
  const int64_t kb = ev_off[lo], kend = ev_off[lo + 1];
  const float *g = gdt + row * n_events;
  const int2 p = mev[n];
  const int64_t ks = kb + p.x, ke = kb + p.y;
  auto gt = [&](int64_t k) {
    return (k == kb ? 0.f : g[k]) - (k + 1 < kend ? g[k + 1] : 0.f);
  };
  if (p.x == p.y) {
    // instantaneous measurement: moving its time moves both "edges"; each
    // column holds half of d loglik / d t
    out[2 * idx] = out[2 * idx + 1] = 0.5f * gt(ks);
    return;
  }
  const float wpart = gwe[row * n_events + ke];
  out[2 * idx] = gt(ks) + wpart;
  out[2 * idx + 1] = gt(ke) - wpart;
}

// FP32 FMA throughput probe: eight independent FMA chains per thread, iters
// steps each (2 FLOP per FMA).  The result is stored only when it equals a
// value the chains never reach, which keeps the compiler from removing them.
__global__ void __launch_bounds__(256) k_fma_peak(float *__restrict__ sink, int iters, float b,
                                                  float c) {
  float a0 = threadIdx.x * 1e-7f, a1 = a0 + 1e-7f, a2 = a0 + 2e-7f, a3 = a0 + 3e-7f;
  float a4 = a0 + 4e-7f, a5 = a0 + 5e-7f, a6 = a0 + 6e-7f, a7 = a0 + 7e-7f;
#pragma unroll 4
  for (int i = 0; i < iters; ++i) {
    a0 = fmaf(a0, b, c);
    a1 = fmaf(a1, b, c);
    a2 = fmaf(a2, b, c);
    a3 = fmaf(a3, b, c);
    a4 = fmaf(a4, b, c);
    a5 = fmaf(a5, b, c);
    a6 = fmaf(a6, b, c);
    a7 = fmaf(a7, b, c);
  }
  const float r = ((a0 + a1) + (a2 + a3)) + ((a4 + a5) + (a6 + a7));
  if (r == -12345.0f) sink[blockIdx.x] = r;
}

// One warp per chunk, so that a series group's share (a quarter of the chunks
// or less) still fills the GPU.  A tile of 32 x ILV_RUN steps: lane j takes
// the run of steps [j ILV_RUN, (j + 1) ILV_RUN) of the tile, counts its end
// events, and an exclusive warp scan of the counts gives the run's first
// measurement; each lane then writes its run's lane-step records.
constexpr int ILV_RUN = 8;

__global__ void __launch_bounds__(128) k_interleave(DevModel M, int c_begin, int c_count,
                                                    float4 *__restrict__ ilv,
                                                    uint8_t *__restrict__ ilv_tag) {
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= c_count) return;  // whole warps
  const int c = c_begin + (int)w;
  const int64_t e0 = M.ch_ev0[c];
  const int len = M.ch_len[c];
  int64_t mi = M.ch_meas0[c];
  const int64_t idx0 = lane_step(M, c, 0);
  for (int k0 = 0; k0 < len; k0 += 32 * ILV_RUN) {  // len is the same on every lane
    const int ks = k0 + lane * ILV_RUN;
    uint8_t t[ILV_RUN];
    float dt[ILV_RUN];
    int cnt = 0;
#pragma unroll
    for (int u = 0; u < ILV_RUN; ++u) {
      const bool in = ks + u < len;
      t[u] = in ? M.tag[e0 + ks + u] : 0;
      dt[u] = in ? M.dt[e0 + ks + u] : 0.f;
      cnt += t[u] & 1;
    }
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += v;
    }
    int64_t mu = mi + (incl - cnt);
    mi += __shfl_sync(0xffffffffu, incl, 31);
#pragma unroll
    for (int u = 0; u < ILV_RUN; ++u) {
      if (ks + u < len) {
        const float4 q = (t[u] & 1) ? M.meas[mu] : make_float4(0.f, 0.f, 0.f, 0.f);
        mu += t[u] & 1;
        const int64_t o = idx0 + (int64_t)32 * (ks + u);
        ilv[o] = make_float4(dt[u], q.x, q.y, q.z);
        ilv_tag[o] = t[u];
      }
    }
  }
}

// Measurement records (y, r0, w) -> the float4 layout the chunk kernels read.
__global__ void k_pack_meas(const float *__restrict__ in3, float4 *__restrict__ out, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  out[i] = make_float4(in3[3 * i], in3[3 * i + 1], in3[3 * i + 2], 0.f);
}

__global__ void k_gather_cond(int n_rows, int n_series, const int64_t *__restrict__ ev_off,
                              const int64_t *__restrict__ meas_off, const int2 *__restrict__ mev,
                              int64_t n_meas, int64_t n_events, const float2 *__restrict__ cond,
                              float *__restrict__ out) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)n_rows * n_meas) return;
  const int64_t row = idx / n_meas, n = idx % n_meas;
  int lo = 0, hi = n_series - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (meas_off[mid] <= n)
      lo = mid;
    else
      hi = mid - 1;
  }
  const float2 v = cond[row * n_events + ev_off[lo] + mev[n].y];
  out[2 * idx] = v.x;
  out[2 * idx + 1] = v.y;
}
}  // namespace gpss

using gpss::OpTable;

namespace {

constexpr int kMaxSlots = 3;
constexpr int kDefaultChunk = 256;
// arithmetic of the cross-chunk combination when the options leave it open
constexpr int kDefaultCombPrec = 32;
// largest step-scalar cache a gradient call allocates (bytes)
constexpr size_t kDcacheMax = (size_t)8 << 30;

template <class T>
struct DevBuf {
  T *p = nullptr;
  size_t n = 0;
};

struct GraphKey {
  int kind;
  const void *theta;
  int n_sets, per_series;
  const void *out1, *out2;
  cudaStream_t stream;
  bool operator<(const GraphKey &o) const {
    return std::tie(kind, theta, n_sets, per_series, out1, out2, stream) <
           std::tie(o.kind, o.theta, o.n_sets, o.per_series, o.out1, o.out2, o.stream);
  }
};

}  // namespace

struct gp_ss_model {
  int device = 0;
  int n_series = 0, n_terms = 0, kinds[4] = {0, 0, 0, 0}, layout = 0, n_slots = 1;
  bool product = false;  // a product term (instantaneous measurements only)
  bool mixed = false;    // instantaneous measurements among exposure averages
  int n_params = 0, precision = 32, schedule = 0;
  int64_t n_meas = 0, n_events = 0;
  OpTable ops{};
  // host copies
  std::vector<int64_t> ev_off, meas_off;
  std::vector<uint8_t> tag;
  float *h_dt = nullptr;  // host copies of the event stream (pinned when possible)
  uint8_t *h_tag = nullptr;
  float4 *h_meas = nullptr;
  float *h_meas3 = nullptr;  // pinned (y, r0, w) per measurement: the host-buffer call sends these
  bool pinned = false;
  // device event stream
  int64_t *d_ev_off = nullptr, *d_meas_off = nullptr;
  float *d_dt = nullptr;
  uint8_t *d_tag = nullptr;
  float4 *d_meas = nullptr;
  double *d_dt64 = nullptr, *d_meas64 = nullptr;
  int2 *d_mev = nullptr;  // per measurement (input order): its start and end event in the series
  std::vector<double> tev;  // event times (FP64, sorted per series) for predictions
  // chunk plan
  int chunk_len = 0, n_chunks = 0, max_chunk = 0, max_chunks_per_series = 0;
  int combine = 0;  // cross-chunk combination: 0 auto, 1 sequential per series, 2 tree
  int ckpt_interval = 32;  // events per recomputation segment of the gradient
  int step_cache = 0;      // 0 auto, 1 never keep the gradient's step scalars
  int comb_prec = 32;      // arithmetic of the cross-chunk combination: 32 or 64
  int64_t *d_ch_ev0 = nullptr, *d_ch_meas0 = nullptr;
  int32_t *d_ch_len = nullptr, *d_ch_series = nullptr, *d_ch_first = nullptr;
  std::vector<int32_t> ch_first;  // host copy: first chunk of each series
  uint8_t *d_ch_flags = nullptr;
  // step-scalar cache of the gradient: per warp of chunks, 32 x (its longest
  // chunk) lane-steps; d_w_doff[w] = lane-steps before warp w, [n_w] = total
  int64_t *d_w_doff = nullptr;
  int64_t dcache_steps = 0;
  // the event stream in lane-step order (k_interleave), for the chunk plan
  float4 *d_ilv = nullptr;
  uint8_t *d_ilv_tag = nullptr;
  // per-call scratch comes from this model's stream-ordered pool, which keeps
  // freed memory reserved (no unmapping and re-mapping at every synchronise)
  cudaMemPool_t pool = nullptr;
  // device error flags of the last call
  mutable std::mutex mu;
  mutable int *d_err = nullptr;
  mutable int err_cap = 0;
  mutable int last_n_out = 0;
  mutable std::map<GraphKey, cudaGraphExec_t> graphs;
  // optional per-phase timing (event pairs around kernels of direct calls)
  mutable bool timing = false;
  mutable std::vector<std::tuple<int, cudaEvent_t, cudaEvent_t>> timings;
};

namespace {

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

bool pick_ops(int n_terms, int n_slots, int layout, OpTable *o) {
  if (n_slots == 0) {  // instantaneous measurements only
    if (n_terms == 1) {
      *o = gpss::ops_1_0_0();
      o->comb64 = gpss::comb64_1_0_0();
    } else if (n_terms == 2) {
      *o = gpss::ops_2_0_0();
      o->comb64 = gpss::comb64_2_0_0();
    } else {
      return false;
    }
    return true;
  }
  if (n_terms == 1) {
    if (n_slots == 1) {
      *o = gpss::ops_1_1_0();
      o->comb64 = gpss::comb64_1_1_0();
    } else if (n_slots == 2) {
      *o = gpss::ops_1_2_0();
      o->comb64 = gpss::comb64_1_2_0();
    } else if (n_slots == 3) {
      *o = gpss::ops_1_3_0();
      o->comb64 = gpss::comb64_1_3_0();
    } else {
      return false;
    }
    return true;
  }
  if (n_terms == 2 && layout == 0) {
    if (n_slots == 1) {
      *o = gpss::ops_2_1_0();
      o->comb64 = gpss::comb64_2_1_0();
    } else if (n_slots == 2) {
      *o = gpss::ops_2_2_0();
      o->comb64 = gpss::comb64_2_2_0();
    } else if (n_slots == 3) {
      *o = gpss::ops_2_3_0();
      o->comb64 = gpss::comb64_2_3_0();
    } else {
      return false;
    }
    return true;
  }
  if (n_terms == 2 && layout == 1 && n_slots == 1) {
    *o = gpss::ops_2_1_1();
    o->comb64 = gpss::comb64_2_1_1();
    return true;
  }
  return false;
}

// Allocate *dst and copy n elements of src into it.  On failure *dst is
// null and nothing stays allocated.
template <class T>
gp_ss_status dev_upload(T **dst, const T *src, size_t n) {
  *dst = nullptr;
  if (n == 0) n = 1;
  T *p = nullptr;
  if (cudaMalloc((void **)&p, n * sizeof(T)) != cudaSuccess) return GP_SS_ENOMEM;
  if (src && cudaMemcpy(p, src, n * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaFree(p);
    return GP_SS_ECUDA;
  }
  *dst = p;
  return GP_SS_OK;
}

void free_model_buffers(gp_ss_model *m) {
  void *dev[] = {m->d_ev_off, m->d_meas_off, m->d_dt, m->d_tag, m->d_meas, m->d_dt64, m->d_meas64,
                 m->d_mev,
                 m->d_ch_ev0, m->d_ch_meas0, m->d_ch_len, m->d_ch_series, m->d_ch_first,
                 m->d_ch_flags, m->d_w_doff, m->d_err, m->d_ilv, m->d_ilv_tag};
  for (void *p : dev)
    if (p) cudaFree(p);
  if (m->pool) {
    cudaMemPoolDestroy(m->pool);
    m->pool = nullptr;
  }
  if (m->h_meas3) cudaFreeHost(m->h_meas3);
  m->h_meas3 = nullptr;
  void *hst[] = {m->h_dt, m->h_tag, m->h_meas};
  for (void *p : hst)
    if (p) {
      if (m->pinned)
        cudaFreeHost(p);
      else
        std::free(p);
    }
  for (auto &kv : m->graphs) cudaGraphExecDestroy(kv.second);
  for (auto &t : m->timings) {
    cudaEventDestroy(std::get<1>(t));
    cudaEventDestroy(std::get<2>(t));
  }
}

// Per-series event build.  Two events per exposure, time-ordered with every
// end before any start at equal times (a reset must not wipe an integral
// before it is read), then by measurement index; slot = instrument label or
// greedy lowest free slot in start order (footnote of Section 3.2.3).
struct SeriesOut {
  gp_ss_status st = GP_SS_OK;
  int n_slots = 1;
};

// Per measurement: 0 = exposure (t_end > t_start), 1 = instantaneous
// (t_end == t_start, Section 2), -1 = invalid input.
inline int meas_kind(double ts, double te, float y, float yerr) {
  const double d = te - ts;
  if (!std::isfinite(d) || !std::isfinite(ts) || !std::isfinite(y) || !std::isfinite(yerr) ||
      d < 0)
    return -1;
  return d == 0 ? 1 : 0;
}

// Events of series [a, b) at event offset e0: two per exposure (start, end),
// one per instantaneous measurement (a measurement event observing the
// latent; a model holds one kind only, checked by the caller).
void build_series_mixed(int64_t a, int64_t b, int64_t e0, const double *ts, const double *te,
                        const float *y, const float *yerr, const int32_t *inst, float *dt,
                        uint8_t *tag, float4 *meas, double *dt64, double *meas64, int2 *mev,
                        double *tev, SeriesOut *out);

void build_series(int64_t a, int64_t b, int64_t e0, const double *ts, const double *te,
                  const float *y, const float *yerr, const int32_t *inst, float *dt, uint8_t *tag,
                  float4 *meas, double *dt64, double *meas64, int2 *mev, double *tev,
                  SeriesOut *out, bool mixed = false) {
  const int64_t n = b - a;
  if (n == 0) {  // an empty series asks for no integral state
    out->n_slots = 0;
    return;
  }
  if (mixed) {
    build_series_mixed(a, b, e0, ts, te, y, yerr, inst, dt, tag, meas, dt64, meas64, mev, tev,
                       out);
    return;
  }
  std::vector<int> slot(n);
  int n_slots = 1;
  int64_t n_inst = 0;
  for (int64_t i = 0; i < n; ++i) {
    const int kd = meas_kind(ts[a + i], te[a + i], y[a + i], yerr[a + i]);
    if (kd < 0) {
      out->st = GP_SS_EINVAL;
      return;
    }
    n_inst += kd;
  }
  if (n_inst > 0) {
    // instantaneous series: one measurement event each, in time order (ties
    // by input order; simultaneous updates commute)
    out->n_slots = 0;
    std::vector<int64_t> ord(n);
    std::iota(ord.begin(), ord.end(), 0);
    std::stable_sort(ord.begin(), ord.end(),
                     [&](int64_t p, int64_t q) { return ts[a + p] < ts[a + q]; });
    double tprev = n > 0 ? ts[a + ord[0]] : 0.0;
    for (int64_t k = 0; k < n; ++k) {
      const int64_t i = ord[k];
      const double gap = ts[a + i] - tprev;
      tprev = ts[a + i];
      dt[e0 + k] = (float)gap;
      if (dt64) dt64[e0 + k] = gap;
      tev[e0 + k] = ts[a + i];
      tag[e0 + k] = 1;
      mev[a + i] = make_int2((int)k, (int)k);
      const double r0 = (double)yerr[a + i] * (double)yerr[a + i];
      meas[a + k] = make_float4(y[a + i], (float)r0, 1.0f, 0.0f);
      if (meas64) {
        meas64[3 * (a + k)] = (double)y[a + i];
        meas64[3 * (a + k) + 1] = r0;
        meas64[3 * (a + k) + 2] = 1.0;
      }
    }
    return;
  }
  std::vector<int64_t> order(n);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(),
                   [&](int64_t p, int64_t q) { return ts[a + p] < ts[a + q]; });
  if (inst) {
    std::vector<double> last_end;
    for (int64_t r = 0; r < n; ++r) {
      const int64_t i = order[r];
      const int s = inst[a + i];
      if (s < 0 || s >= 8) {
        out->st = s < 0 ? GP_SS_EINVAL : GP_SS_EUNSUPPORTED;
        return;
      }
      if ((int)last_end.size() <= s) last_end.resize(s + 1, -INFINITY);
      if (last_end[s] > ts[a + i]) {
        out->st = GP_SS_ESELFOVERLAP;
        return;
      }
      last_end[s] = te[a + i];
      slot[i] = s;
      n_slots = std::max(n_slots, s + 1);
    }
  } else {
    std::vector<double> last_end;
    for (int64_t r = 0; r < n; ++r) {
      const int64_t i = order[r];
      int s = 0;
      while (s < (int)last_end.size() && last_end[s] > ts[a + i]) ++s;
      if (s == (int)last_end.size()) last_end.push_back(0);
      last_end[s] = te[a + i];
      slot[i] = s;
      n_slots = std::max(n_slots, s + 1);
    }
  }
  out->n_slots = n_slots;
  // events: key (time, kind with end = 0 first, measurement)
  struct Ev {
    double t;
    int kind;  // 0 end, 1 start
    int64_t i;
  };
  std::vector<Ev> ev(2 * n);
  for (int64_t i = 0; i < n; ++i) {
    ev[2 * i] = {ts[a + i], 1, i};
    ev[2 * i + 1] = {te[a + i], 0, i};
  }
  std::sort(ev.begin(), ev.end(), [](const Ev &p, const Ev &q) {
    if (p.t != q.t) return p.t < q.t;
    if (p.kind != q.kind) return p.kind < q.kind;
    return p.i < q.i;
  });
  int64_t mi = a;
  double tprev = n > 0 ? ev[0].t : 0.0;
  for (int64_t k = 0; k < 2 * n; ++k) {
    const double gap = ev[k].t - tprev;
    tprev = ev[k].t;
    dt[e0 + k] = (float)gap;
    if (dt64) dt64[e0 + k] = gap;
    tev[e0 + k] = ev[k].t;
    const int64_t i = ev[k].i;
    const bool is_end = ev[k].kind == 0;
    tag[e0 + k] = (uint8_t)((is_end ? 1 : 0) | (slot[i] << 1));
    // where this measurement's window edges sit in the series' events
    if (is_end)
      mev[a + i].y = (int)k;
    else
      mev[a + i].x = (int)k;
    if (is_end) {
      const double delta = te[a + i] - ts[a + i];
      const double w = 1.0 / delta;
      const double r0 = (double)yerr[a + i] * (double)yerr[a + i];
      meas[mi] = make_float4(y[a + i], (float)r0, (float)w, 0.0f);
      if (meas64) {
        meas64[3 * mi] = (double)y[a + i];
        meas64[3 * mi + 1] = r0;
        meas64[3 * mi + 2] = w;
      }
      ++mi;
    }
  }
}

// A series of a model that mixes instantaneous measurements with exposure
// averages: two events per exposure (reset at the start, read at the end,
// slots as in build_series), one per instant (tagged TAG_INSTANT: it
// observes the latent, Section 2).  Order: time, then exposure ends, then
// instants, then starts (every read before a reset at the same time), then
// measurement index.
void build_series_mixed(int64_t a, int64_t b, int64_t e0, const double *ts, const double *te,
                        const float *y, const float *yerr, const int32_t *inst, float *dt,
                        uint8_t *tag, float4 *meas, double *dt64, double *meas64, int2 *mev,
                        double *tev, SeriesOut *out) {
  const int64_t n = b - a;
  std::vector<int> slot(n, 0), kind(n);
  for (int64_t i = 0; i < n; ++i) {
    kind[i] = meas_kind(ts[a + i], te[a + i], y[a + i], yerr[a + i]);
    if (kind[i] < 0) {
      out->st = GP_SS_EINVAL;
      return;
    }
  }
  std::vector<int64_t> order(n);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(),
                   [&](int64_t p, int64_t q) { return ts[a + p] < ts[a + q]; });
  int n_slots = 0;
  std::vector<double> last_end;
  for (int64_t r = 0; r < n; ++r) {
    const int64_t i = order[r];
    if (kind[i] == 1) continue;  // instants take no slot
    int s = 0;
    if (inst) {
      s = inst[a + i];
      if (s < 0 || s >= 8) {
        out->st = s < 0 ? GP_SS_EINVAL : GP_SS_EUNSUPPORTED;
        return;
      }
      if ((int)last_end.size() <= s) last_end.resize(s + 1, -INFINITY);
      if (last_end[s] > ts[a + i]) {
        out->st = GP_SS_ESELFOVERLAP;
        return;
      }
    } else {
      while (s < (int)last_end.size() && last_end[s] > ts[a + i]) ++s;
      if (s == (int)last_end.size()) last_end.push_back(0);
    }
    last_end[s] = te[a + i];
    slot[i] = s;
    n_slots = std::max(n_slots, s + 1);
  }
  out->n_slots = n_slots;
  struct Ev {
    double t;
    int kind;  // 0 exposure end, 1 instant, 2 exposure start
    int64_t i;
  };
  std::vector<Ev> ev;
  ev.reserve(2 * n);
  for (int64_t i = 0; i < n; ++i) {
    if (kind[i] == 1) {
      ev.push_back({ts[a + i], 1, i});
    } else {
      ev.push_back({ts[a + i], 2, i});
      ev.push_back({te[a + i], 0, i});
    }
  }
  std::sort(ev.begin(), ev.end(), [](const Ev &p, const Ev &q) {
    if (p.t != q.t) return p.t < q.t;
    if (p.kind != q.kind) return p.kind < q.kind;
    return p.i < q.i;
  });
  int64_t mi = a;
  double tprev = ev.empty() ? 0.0 : ev[0].t;
  for (size_t k = 0; k < ev.size(); ++k) {
    const double gap = ev[k].t - tprev;
    tprev = ev[k].t;
    dt[e0 + k] = (float)gap;
    if (dt64) dt64[e0 + k] = gap;
    tev[e0 + k] = ev[k].t;
    const int64_t i = ev[k].i;
    if (ev[k].kind == 2) {
      tag[e0 + k] = (uint8_t)(slot[i] << 1);
      mev[a + i].x = (int)k;
      continue;
    }
    const bool instant = ev[k].kind == 1;
    tag[e0 + k] = instant ? (uint8_t)(1 | gpss::TAG_INSTANT) : (uint8_t)(1 | (slot[i] << 1));
    if (instant)
      mev[a + i] = make_int2((int)k, (int)k);
    else
      mev[a + i].y = (int)k;
    const double w = instant ? 1.0 : 1.0 / (te[a + i] - ts[a + i]);
    const double r0 = (double)yerr[a + i] * (double)yerr[a + i];
    meas[mi] = make_float4(y[a + i], (float)r0, (float)w, 0.0f);
    if (meas64) {
      meas64[3 * mi] = (double)y[a + i];
      meas64[3 * mi + 1] = r0;
      meas64[3 * mi + 2] = w;
    }
    ++mi;
  }
}

gpss::DevModel dev_view(const gp_ss_model *m);

// Re-lay the event stream of chunks [c0, c0 + cn) in the plan's lane-step
// order (after a new plan, or after the event stream was re-sent).
cudaError_t interleave_events(const gp_ss_model *m, int c0, int cn, cudaStream_t st) {
  if (cn <= 0 || !m->d_ilv) return cudaSuccess;
  const int64_t threads = (int64_t)cn * 32;  // one warp per chunk
  gpss::k_interleave<<<(unsigned)((threads + 127) / 128), 128, 0, st>>>(dev_view(m), c0, cn,
                                                                       m->d_ilv, m->d_ilv_tag);
  GPSS_COUNT_LAUNCH();
  return cudaGetLastError();
}

gp_ss_status make_plan(gp_ss_model *m, int chunk_len) {
  const int n = m->n_series;
  int L = chunk_len;
  if (m->schedule == 1 || m->schedule == 3 || L <= 0) {
    if (m->schedule == 1 || m->schedule == 3) {
      // one warp per series: 32 chunks of about K/32 events each
      int64_t mx = 1;
      for (int s = 0; s < n; ++s) mx = std::max<int64_t>(mx, m->ev_off[s + 1] - m->ev_off[s]);
      if (mx > (int64_t)1 << 35) return GP_SS_EUNSUPPORTED;
      L = (int)std::max<int64_t>(1, (mx + 31) / 32);
    } else {
      L = kDefaultChunk;
    }
  }
  std::vector<int64_t> ev0, meas0;
  std::vector<int32_t> len, ser, first(n + 1);
  std::vector<uint8_t> flags;
  int max_len = 0;
  for (int s = 0; s < n; ++s) {
    first[s] = (int32_t)len.size();
    const int64_t a = m->ev_off[s], K = m->ev_off[s + 1] - a;
    // a multiple of 32 chunks per series: every warp of the chunk kernels then
    // works on one series (one hyperparameter row), which lets it share the
    // row's Taylor table; chunk lengths are balanced within the series
    const int64_t nch = 32 * std::max<int64_t>(1, (K + 32 * (int64_t)L - 1) / (32 * (int64_t)L));
    // boundaries at even event offsets: in a series whose events alternate
    // start / end, every lane of a warp then meets the same kind of event at
    // the same step (no divergence between the reset and update paths)
    int64_t e = a, mi = m->meas_off[s];
    for (int64_t c = 0; c < nch; ++c) {
      const int64_t hi = (c == nch - 1) ? K : std::min<int64_t>(K, 2 * (((c + 1) * K) / (2 * nch)));
      const int64_t l = std::max<int64_t>(0, a + hi - e);
      ev0.push_back(e);
      meas0.push_back(mi);
      len.push_back((int32_t)l);
      ser.push_back(s);
      flags.push_back((uint8_t)((c == 0 ? 1 : 0) | (c == nch - 1 ? 2 : 0)));
      for (int64_t k = e; k < e + l; ++k) mi += m->tag[k] & 1;
      e += l;
      max_len = std::max<int>(max_len, (int)l);
    }
  }
  first[n] = (int32_t)len.size();
  if (len.size() > (size_t)INT32_MAX / 4) return GP_SS_EUNSUPPORTED;
  // every warp of 32 chunks lies in one series (32 | chunks per series)
  const size_t n_w = len.size() / 32;
  std::vector<int64_t> doff(n_w + 1, 0);
  for (size_t w = 0; w < n_w; ++w) {
    int ml = 0;
    for (int l = 0; l < 32; ++l) ml = std::max(ml, len[w * 32 + l]);
    doff[w + 1] = doff[w] + 32 * (int64_t)ml;
  }
  // upload the new plan into fresh buffers first: the model keeps its old
  // plan, untouched, unless every upload succeeds
  int64_t *n_ev0 = nullptr, *n_meas0 = nullptr, *n_doff = nullptr;
  int32_t *n_len = nullptr, *n_ser = nullptr, *n_first = nullptr;
  uint8_t *n_flags = nullptr;
  gp_ss_status st = GP_SS_OK;
  if (!st) st = dev_upload(&n_ev0, ev0.data(), ev0.size());
  if (!st) st = dev_upload(&n_meas0, meas0.data(), meas0.size());
  if (!st) st = dev_upload(&n_len, len.data(), len.size());
  if (!st) st = dev_upload(&n_ser, ser.data(), ser.size());
  if (!st) st = dev_upload(&n_first, first.data(), first.size());
  if (!st) st = dev_upload(&n_flags, flags.data(), flags.size());
  if (!st) st = dev_upload(&n_doff, doff.data(), doff.size());
  // the event stream in this plan's lane-step order
  float4 *n_ilv = nullptr;
  uint8_t *n_ilv_tag = nullptr;
  if (!st) st = dev_upload<float4>(&n_ilv, nullptr, (size_t)doff[n_w]);
  if (!st) st = dev_upload<uint8_t>(&n_ilv_tag, nullptr, (size_t)doff[n_w]);
  if (st) {
    void *fresh[] = {n_ev0, n_meas0, n_len, n_ser, n_first, n_flags, n_doff, n_ilv, n_ilv_tag};
    for (void *p : fresh)
      if (p) cudaFree(p);
    return st;
  }
  // kernels queued earlier may still read the old plan
  if (cudaDeviceSynchronize() != cudaSuccess) {
    void *fresh[] = {n_ev0, n_meas0, n_len, n_ser, n_first, n_flags, n_doff, n_ilv, n_ilv_tag};
    for (void *p : fresh) cudaFree(p);
    return GP_SS_ECUDA;
  }
  void *old[] = {m->d_ch_ev0, m->d_ch_meas0, m->d_ch_len, m->d_ch_series, m->d_ch_first,
                 m->d_ch_flags, m->d_w_doff, m->d_ilv, m->d_ilv_tag};
  for (void *p : old)
    if (p) cudaFree(p);
  m->d_ilv = n_ilv;
  m->d_ilv_tag = n_ilv_tag;
  m->d_ch_ev0 = n_ev0;
  m->d_ch_meas0 = n_meas0;
  m->d_ch_len = n_len;
  m->d_ch_series = n_ser;
  m->d_ch_first = n_first;
  m->d_ch_flags = n_flags;
  m->d_w_doff = n_doff;
  m->ch_first = first;
  m->dcache_steps = doff[n_w];
  m->chunk_len = L;
  m->n_chunks = (int)len.size();
  m->max_chunk = max_len;
  m->max_chunks_per_series = 0;
  for (int s = 0; s < n; ++s)
    m->max_chunks_per_series = std::max(m->max_chunks_per_series, first[s + 1] - first[s]);
  if (interleave_events(m, 0, m->n_chunks, nullptr) != cudaSuccess ||
      cudaDeviceSynchronize() != cudaSuccess)
    return GP_SS_ECUDA;
  for (auto &kv : m->graphs) cudaGraphExecDestroy(kv.second);
  m->graphs.clear();
  return GP_SS_OK;
}

gpss::DevModel dev_view(const gp_ss_model *m) {
  gpss::DevModel d;
  d.n_series = m->n_series;
  d.n_params = m->n_params;
  d.n_terms = m->n_terms;
  for (int i = 0; i < 4; ++i) d.kinds[i] = m->kinds[i];
  d.ev_off = m->d_ev_off;
  d.meas_off = m->d_meas_off;
  d.dt = m->d_dt;
  d.tag = m->d_tag;
  d.meas = m->d_meas;
  d.dt64 = m->d_dt64;
  d.meas64 = m->d_meas64;
  d.n_chunks = m->n_chunks;
  d.ch_ev0 = m->d_ch_ev0;
  d.ch_meas0 = m->d_ch_meas0;
  d.ch_len = m->d_ch_len;
  d.ch_series = m->d_ch_series;
  d.ch_flags = m->d_ch_flags;
  d.ch_first = m->d_ch_first;
  d.n_events = m->n_events;
  d.w_doff = m->d_w_doff;
  d.dcache_steps = m->dcache_steps;
  d.ilv = m->d_ilv;
  d.ilv_tag = m->d_ilv_tag;
  d.mixed = m->mixed ? 1 : 0;
  return d;
}

#define GPSS_CK(call)                         \
  do {                                        \
    cudaError_t e_ = (call);                  \
    if (e_ != cudaSuccess) return GP_SS_ECUDA; \
  } while (0)

gp_ss_status prepare_err(const gp_ss_model *m, int n_out, cudaStream_t st) {
  std::lock_guard<std::mutex> lk(m->mu);
  if (m->err_cap < n_out) {
    if (m->d_err) cudaFree(m->d_err);
    m->d_err = nullptr;
    if (cudaMalloc((void **)&m->d_err, std::max(n_out, 1) * sizeof(int)) != cudaSuccess) {
      m->err_cap = 0;
      return GP_SS_ENOMEM;
    }
    m->err_cap = n_out;
  }
  m->last_n_out = n_out;
  GPSS_CK(cudaMemsetAsync(m->d_err, 0, std::max(n_out, 1) * sizeof(int), st));
  return GP_SS_OK;
}

// Records an event pair around one kernel phase when timing is on and the
// stream is not being captured.
struct PhaseTimer {
  const gp_ss_model *m;
  cudaStream_t st;
  int phase;
  cudaEvent_t a = nullptr, b = nullptr;
  PhaseTimer(const gp_ss_model *m_, cudaStream_t st_, int phase_) : m(m_), st(st_), phase(phase_) {
    if (!m->timing) return;
    cudaStreamCaptureStatus cs;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return;
    if (cudaEventCreate(&a) || cudaEventCreate(&b)) {
      a = b = nullptr;
      return;
    }
    cudaEventRecord(a, st);
  }
  ~PhaseTimer() {
    if (!a) return;
    cudaEventRecord(b, st);
    std::lock_guard<std::mutex> lk(m->mu);
    m->timings.emplace_back(phase, a, b);
  }
};

// Scratch from the model's pool; the default pool while the stream is
// being captured into a graph (graph allocations have their own pool) or
// when the model has no pool.
// On failure *p is null.
cudaError_t scratch_alloc(const gp_ss_model *m, void **p, size_t bytes, cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaError_t e;
  if (m->pool && cudaStreamIsCapturing(st, &cs) == cudaSuccess &&
      cs == cudaStreamCaptureStatusNone)
    e = cudaMallocFromPoolAsync(p, bytes, m->pool, st);
  else
    e = cudaMallocAsync(p, bytes, st);
  if (e != cudaSuccess) *p = nullptr;
  return e;
}

gp_ss_status check_call(const gp_ss_model *m, const float *theta, int n_sets, int per_series,
                        const void *out) {
  if (!m || !theta || !out || n_sets <= 0) return GP_SS_EINVAL;
  if (per_series && n_sets != m->n_series) return GP_SS_EINVAL;
  return GP_SS_OK;
}

// Series groups whose event streams arrive separately: the element pass of
// group g (chunks [c0[g], c0[g+1])) waits for event ready[g] and first lays
// the group's new events out in lane-step order.
struct ElemSlices {
  int n;
  const int *c0;
  const cudaEvent_t *ready;
};

// Enqueue the log-likelihood (and optionally gradient) computation.
gp_ss_status enqueue(const gp_ss_model *m, const float *theta, int n_sets, int per_series,
                     double *ll, float *grad, cudaStream_t st, float *dexp = nullptr,
                     float *cond_out = nullptr, const gpss::PredPlan *pred = nullptr,
                     const ElemSlices *slices = nullptr) {
  const int n_out = per_series ? m->n_series : n_sets * m->n_series;
  gp_ss_status s0 = prepare_err(m, n_out, st);
  if (s0) return s0;
  const gpss::DevModel dm = dev_view(m);
  const OpTable &o = m->ops;
  if (m->product) {
    // product kernels: the plain filters (FP64, schedule 3), or the chunked
    // log-likelihood below; the hyperparameter gradient by forward-mode
    // tangents (FP32), per series (schedule 3) or per chunk
    if (dexp || cond_out || pred) return GP_SS_EUNSUPPORTED;
    if (grad) {
      if (m->precision == 64) return GP_SS_EUNSUPPORTED;
      // the plain schedule: one thread per series and parameter over the
      // whole series; otherwise the chunked path below
      if (m->schedule == 3 || !o.prod_grad_chunk) {
        PhaseTimer pt(m, st, 2);
        GPSS_CK(o.prod_grad(dm, theta, n_out, per_series, ll, grad, m->d_err, st));
        return GP_SS_OK;
      }
    }
    if (m->precision == 64 && !m->d_dt64) return GP_SS_EINVAL;
    if (m->precision == 64 || m->schedule == 3) {
      PhaseTimer pt(m, st, 4);
      GPSS_CK((m->precision == 64 ? o.plain64 : o.plain32)(dm, theta, n_out, per_series, ll,
                                                           m->d_err, st));
      return GP_SS_OK;
    }
    // else the chunked log-likelihood below (product elements, shared combination)
  }
  if (m->precision == 64) {
    if (grad) return GP_SS_EUNSUPPORTED;
    if (!m->d_dt64) return GP_SS_EINVAL;
    PhaseTimer pt(m, st, 4);
    GPSS_CK(o.plain64(dm, theta, n_out, per_series, ll, m->d_err, st));
    return GP_SS_OK;
  }
  if (m->schedule == 3 && !grad) {
    // one thread per series, the whole sequential filter in registers
    PhaseTimer pt(m, st, 4);
    GPSS_CK(o.plain32(dm, theta, n_out, per_series, ll, m->d_err, st));
    return GP_SS_OK;
  }
  const int64_t n_vch64 = (int64_t)(per_series ? 1 : n_sets) * m->n_chunks;
  if (n_vch64 > INT32_MAX / 8) return GP_SS_EUNSUPPORTED;
  const int n_vch = (int)n_vch64;
  const int SD = o.D + o.NP;
  // the cross-chunk combination's arithmetic (its state, information and
  // partial-combination buffers hold eb bytes per value)
  const gpss::CombineOps &cb = m->comb_prec == 64 ? o.comb64 : o.comb32;
  const size_t eb = (size_t)cb.elem_bytes;
  // cross-chunk combination: warp-level scans plus a scan of warp totals
  // (default), or the sequential fold with one thread per series
  bool tree = m->combine != 1;
  std::vector<void *> bufs;
  auto grab = [&](void **p, size_t bytes) -> bool {
    if (scratch_alloc(m, p, std::max<size_t>(bytes, 16), st) != cudaSuccess) {
      *p = nullptr;
      return false;
    }
    bufs.push_back(*p);
    return true;
  };
  float *ef = nullptr, *adj = nullptr, *ckpt = nullptr, *gpart = nullptr, *tabs = nullptr;
  void *state_end = nullptr, *info = nullptr, *scratch = nullptr;
  double *ed = nullptr, *ll_part = nullptr;
  gp_ss_status res = GP_SS_OK;
  do {
    // for the gradient, k_elem also saves the partial element at the start of
    // every recomputation segment but a chunk's first
    const int ck = m->ckpt_interval;
    const int n_pck = std::max((m->max_chunk - 1) / ck, 1);
    if (!grab((void **)&ef, (size_t)o.NF * n_vch * sizeof(float)) ||
        !grab((void **)&ed, (size_t)o.ND * n_vch * sizeof(double)) ||
        !grab((void **)&tabs, (size_t)n_sets * o.NT * gpss::TAB_TERM * sizeof(float)) ||
        (grad && !m->product &&
         !grab((void **)&ckpt, (size_t)n_pck * (o.NF + 1) * n_vch * sizeof(float)))) {
      res = GP_SS_ENOMEM;
      break;
    }
    // the element pass keeps every step's scalars for the gradient's replay
    // while that takes at most kDcacheMax bytes (else the replay recomputes them)
    float *dcache = nullptr;
    if (grad && !m->product) {
      const size_t dbytes = (size_t)(n_vch / m->n_chunks) * (size_t)m->dcache_steps *
                            (4 * ((6 * o.NT + 3) / 4)) * sizeof(float);
      if (m->step_cache == 0 && dbytes <= kDcacheMax && !grab((void **)&dcache, dbytes)) {
        res = GP_SS_ENOMEM;
        break;
      }
    }
    {
      PhaseTimer pt(m, st, 0);
      if (o.tables(theta, n_sets, m->n_params, m->kinds[0], m->kinds[1], tabs, st)) {
        res = GP_SS_ECUDA;
        break;
      }
      // whole model, or series groups as their event streams arrive
      const int ng = slices ? slices->n : 1;
      for (int g = 0; g < ng && !res; ++g) {
        const int c0 = slices ? slices->c0[g] : 0;
        const int cn = slices ? slices->c0[g + 1] - c0 : m->n_chunks;
        if (slices && cudaStreamWaitEvent(st, slices->ready[g], 0) != cudaSuccess) res = GP_SS_ECUDA;
        // a re-sent group's events are laid out for the chunk kernels here,
        // on the compute stream, while the copy stream sends the next group
        if (!res && slices && interleave_events(m, c0, cn, st) != cudaSuccess) res = GP_SS_ECUDA;
        if (!res && o.elem(dm, theta, n_vch, per_series, ef, ed, m->d_err, tabs,
                           grad ? ckpt : nullptr, ck, dcache, c0, cn, st))
          res = GP_SS_ECUDA;
      }
      if (res) break;
    }
    if ((grad || tree) && !grab(&state_end, (size_t)SD * n_vch * eb)) {
      res = GP_SS_ENOMEM;
      break;
    }
    if (grad && !grab((void **)&adj, (size_t)SD * n_vch * sizeof(float))) {
      res = GP_SS_ENOMEM;
      break;
    }
    // warp-level combination buffers
    void *pre_local = nullptr, *suf_local = nullptr, *wtot = nullptr, *wpre = nullptr,
         *wsuf = nullptr;
    const int n_w = n_vch / 32;
    if (tree && (!grab((void **)&ll_part, (size_t)n_vch * sizeof(double)) ||
                 !grab(&pre_local, (size_t)o.NF * n_vch * eb) ||
                 !grab(&wtot, (size_t)o.NF * n_w * eb) || !grab(&wpre, (size_t)o.NF * n_w * eb) ||
                 !grab(&scratch, cb.warp_scratch(n_vch) * eb) ||
                 (grad && (!grab(&info, (size_t)SD * n_vch * eb) ||
                           !grab(&suf_local, (size_t)o.NF * n_vch * eb) ||
                           !grab(&wsuf, (size_t)o.NF * n_w * eb))))) {
      res = GP_SS_ENOMEM;
      break;
    }
    {
      PhaseTimer pt(m, st, 1);
      cudaError_t e;
      if (!tree) {
        e = cb.scan(dm, n_out, per_series, ef, ed, n_vch, state_end, adj, ll, grad ? 1 : 0,
                    m->d_err, st);
      } else {
        // few warps per series: fold warp totals sequentially; else scan them
        const int fold = m->max_chunks_per_series <= 16 * 32 ? 1 : 0;
        e = cb.warp_combine(dm, ef, n_vch, pre_local, suf_local, wtot, wpre, wsuf, scratch,
                            state_end, info, grad ? 1 : 0, fold, n_out, per_series, st);
        if (e == cudaSuccess)
          e = cb.finish(dm, n_vch, per_series, ef, ed, state_end, info, adj, ll_part, m->d_err,
                        st);
      }
      if (e != cudaSuccess) {
        res = GP_SS_ECUDA;
        break;
      }
    }
    if (grad) {
      float *rbuf = nullptr, *gdt = nullptr, *gwe = nullptr;
      float2 *cond = nullptr;
      const int exp_rows = per_series ? 1 : n_sets;
      if ((dexp && (!grab((void **)&gdt, (size_t)exp_rows * m->n_events * sizeof(float)) ||
                    !grab((void **)&gwe, (size_t)exp_rows * m->n_events * sizeof(float)))) ||
          (cond_out && !grab((void **)&cond, (size_t)exp_rows * m->n_events * sizeof(float2)))) {
        res = GP_SS_ENOMEM;
        break;
      }
      if ((!m->product &&
           !grab((void **)&rbuf, (size_t)ck * (4 * ((SD + 3) / 4)) * n_vch * sizeof(float))) ||
          !grab((void **)&gpart, (size_t)m->n_params * n_vch * sizeof(float))) {
        res = GP_SS_ENOMEM;
        break;
      }
      PhaseTimer pt(m, st, 2);
      if (m->product) {
        // chunked forward-mode tangents against the boundary adjoints
        if (o.prod_grad_chunk(dm, theta, n_vch, per_series, state_end, eb == 8 ? 1 : 0, adj, gpart,
                              m->d_err, st))
          res = GP_SS_ECUDA;
        if (res) break;
      } else {
        const gpss::PredPlan none;
        if (o.grad(dm, theta, n_vch, per_series, state_end, eb == 8 ? 1 : 0, adj, ckpt, gpart,
                   m->d_err, tabs, rbuf, dcache, ck, gdt, gwe, cond, pred ? *pred : none, st)) {
          res = GP_SS_ECUDA;
          break;
        }
        if (cond_out && m->n_meas > 0) {
          const int64_t nt = (int64_t)exp_rows * m->n_meas;
          gpss::k_gather_cond<<<(unsigned)((nt + 255) / 256), 256, 0, st>>>(
              exp_rows, m->n_series, m->d_ev_off, m->d_meas_off, m->d_mev, m->n_meas, m->n_events,
              cond, cond_out);
          GPSS_COUNT_LAUNCH();
          if (cudaGetLastError() != cudaSuccess) {
            res = GP_SS_ECUDA;
            break;
          }
        }
        if (dexp && m->n_meas > 0) {
          const int64_t nt = (int64_t)exp_rows * m->n_meas;
          gpss::k_exposure_grad<<<(unsigned)((nt + 255) / 256), 256, 0, st>>>(
              exp_rows, m->n_series, m->d_ev_off, m->d_meas_off, m->d_mev, m->n_meas, m->n_events,
              gdt, gwe, dexp);
          GPSS_COUNT_LAUNCH();
          if (cudaGetLastError() != cudaSuccess) {
            res = GP_SS_ECUDA;
            break;
          }
        }
      }
    }
    if (tree || grad) {
      PhaseTimer pt(m, st, 3);
      gpss::k_series_sum<<<(n_out * 32 + 127) / 128, 128, 0, st>>>(
          n_out, per_series, m->n_series, m->n_chunks, m->d_ch_first, tree ? ll_part : nullptr,
          n_vch, grad ? gpart : nullptr, m->n_params, ll, grad);
      GPSS_COUNT_LAUNCH();
      if (cudaGetLastError() != cudaSuccess) res = GP_SS_ECUDA;
    }
  } while (0);
  for (void *p : bufs) cudaFreeAsync(p, st);
  return res;
}

gp_ss_status run_graph(const gp_ss_model *m, int kind, const float *theta, int n_sets,
                       int per_series, double *ll, float *grad, cudaStream_t st) {
  GraphKey key{kind, theta, n_sets, per_series, ll, grad, st};
  cudaGraphExec_t exec = nullptr;
  {
    std::lock_guard<std::mutex> lk(m->mu);
    auto it = m->graphs.find(key);
    if (it != m->graphs.end()) exec = it->second;
  }
  if (!exec) {
    cudaStream_t cap;
    GPSS_CK(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    // make sure the error buffer exists outside the capture
    gp_ss_status s0 = prepare_err(m, per_series ? m->n_series : n_sets * m->n_series, st);
    if (s0) {
      cudaStreamDestroy(cap);
      return s0;
    }
    GPSS_CK(cudaStreamSynchronize(st));
    cudaGraph_t g;
    if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      cudaStreamDestroy(cap);
      return GP_SS_ECUDA;
    }
    gp_ss_status r = enqueue(m, theta, n_sets, per_series, ll, grad, cap);
    cudaError_t ce = cudaStreamEndCapture(cap, &g);
    cudaStreamDestroy(cap);
    if (r) return r;
    if (ce != cudaSuccess) return GP_SS_ECUDA;
    ce = cudaGraphInstantiate(&exec, g, 0);
    cudaGraphDestroy(g);
    if (ce != cudaSuccess) return GP_SS_ECUDA;
    std::lock_guard<std::mutex> lk(m->mu);
    m->graphs[key] = exec;
  }
  GPSS_CK(cudaGraphLaunch(exec, st));
  return GP_SS_OK;
}

}  // namespace

extern "C" {

const char *gp_ss_status_string(gp_ss_status s) {
  switch (s) {
    case GP_SS_OK: return "ok";
    case GP_SS_EINVAL: return "invalid argument";
    case GP_SS_EUNSORTED: return "series offsets not sorted";
    case GP_SS_ESELFOVERLAP: return "an instrument's exposures overlap each other";
    case GP_SS_EUNSUPPORTED: return "unsupported model shape or parameter regime";
    case GP_SS_ENOMEM: return "out of memory";
    case GP_SS_ECUDA: return "CUDA runtime error";
    case GP_SS_ENUMERIC: return "non-positive or non-finite innovation variance";
    case GP_SS_ETIMEOUT: return "bounded device wait timed out";
    case GP_SS_ETOOBIG: return "problem needs more than the fixed scratch of gp_ss_loglik_noalloc";
  }
  return "unknown status";
}

gp_ss_status gp_ss_build_model(const gp_ss_kernel_spec *spec, int n_series,
                               const int64_t *series_offsets, const double *t_start,
                               const double *t_end, const float *y, const float *yerr,
                               const int32_t *instrument, const gp_ss_options *opts,
                               gp_ss_model **out) {
  if (!out) return GP_SS_EINVAL;
  *out = nullptr;
  if (!spec || !spec->terms || n_series < 1 || !series_offsets) return GP_SS_EINVAL;
  if (spec->n_terms < 1 || spec->n_terms > 2) return GP_SS_EUNSUPPORTED;
  if (spec->integral_layout != 0 && spec->integral_layout != 1) return GP_SS_EINVAL;
  for (int t = 0; t < spec->n_terms; ++t)
    if (spec->terms[t] != GP_SS_TERM_SHO && spec->terms[t] != GP_SS_TERM_MATERN32 &&
        spec->terms[t] != GP_SS_TERM_SHO_PRODUCT)
      return GP_SS_EINVAL;
  // a product term is compiled as the first term, with at most one plain term
  for (int t = 1; t < spec->n_terms; ++t)
    if (spec->terms[t] == GP_SS_TERM_SHO_PRODUCT) return GP_SS_EUNSUPPORTED;
  gp_ss_options o{};
  o.precision = 32;
  if (opts) o = *opts;
  if (o.precision == 0) o.precision = 32;
  if (o.precision != 32 && o.precision != 64) return GP_SS_EINVAL;
  if (o.threads_per_series > 1) return GP_SS_EUNSUPPORTED;
  if (o.chunk_combine < 0 || o.chunk_combine > 2) return GP_SS_EINVAL;
  if (o.ckpt_interval != 0 && o.ckpt_interval != 8 && o.ckpt_interval != 16 &&
      o.ckpt_interval != 32 && o.ckpt_interval != 64)
    return GP_SS_EINVAL;
  if (o.step_cache != 0 && o.step_cache != 1) return GP_SS_EINVAL;
  if (o.combine_precision != 0 && o.combine_precision != 32 && o.combine_precision != 64)
    return GP_SS_EINVAL;
  if (o.schedule < 0 || o.schedule > 3 || o.chunk_combine < 0 || o.chunk_combine > 2)
    return GP_SS_EINVAL;
  if (series_offsets[0] != 0) return GP_SS_EINVAL;
  for (int s = 0; s < n_series; ++s)
    if (series_offsets[s + 1] < series_offsets[s]) return GP_SS_EUNSORTED;
  const int64_t N = series_offsets[n_series];
  if (N > 0 && (!t_start || !t_end || !y || !yerr)) return GP_SS_EINVAL;
  if (2 * N > (int64_t)INT32_MAX * 4) return GP_SS_EUNSUPPORTED;

  gp_ss_model *m = new (std::nothrow) gp_ss_model();
  if (!m) return GP_SS_ENOMEM;
  cudaGetDevice(&m->device);
  m->n_series = n_series;
  m->n_terms = spec->n_terms;
  m->layout = spec->n_terms == 1 ? 0 : spec->integral_layout;
  m->precision = o.precision;
  m->schedule = o.schedule;
  m->combine = o.chunk_combine;
  m->ckpt_interval = o.ckpt_interval == 0 ? 32 : o.ckpt_interval;
  m->step_cache = o.step_cache;
  m->comb_prec = o.combine_precision == 0 ? kDefaultCombPrec : o.combine_precision;
  m->n_params = 1;
  for (int t = 0; t < spec->n_terms; ++t) {
    m->kinds[t] = spec->terms[t];
    m->n_params += spec->terms[t] == GP_SS_TERM_SHO ? 3
                   : spec->terms[t] == GP_SS_TERM_MATERN32 ? 2 : 5;
  }
  m->product = spec->terms[0] == GP_SS_TERM_SHO_PRODUCT;
  m->n_meas = N;
  m->ev_off.resize(n_series + 1);
  m->meas_off.resize(n_series + 1);
  // events per series: two per exposure, one per instantaneous measurement.
  // A model of instants only has no integral states; one that mixes instants
  // with exposure averages marks its instants' events (TAG_INSTANT)
  int64_t n_inst = 0, n_bad = 0;
  for (int64_t i = 0; i < N; ++i) {
    const int kd = meas_kind(t_start[i], t_end[i], y[i], yerr[i]);
    n_bad += kd < 0;
    n_inst += kd > 0;
  }
  if (n_bad) {
    delete m;
    return GP_SS_EINVAL;
  }
  if (m->product && n_inst < N) {
    // a product kernel on exposure averages: not compiled
    delete m;
    return GP_SS_EUNSUPPORTED;
  }
  m->mixed = n_inst > 0 && n_inst < N;
  m->ev_off[0] = 0;
  for (int s = 0; s < n_series; ++s) {
    m->meas_off[s] = series_offsets[s];
    int64_t ne = 0;
    for (int64_t i = series_offsets[s]; i < series_offsets[s + 1]; ++i)
      ne += (t_end[i] == t_start[i]) ? 1 : 2;
    m->ev_off[s + 1] = m->ev_off[s] + ne;
  }
  m->meas_off[n_series] = series_offsets[n_series];
  m->n_events = m->ev_off[n_series];
  // one record past the last measurement: the chunk kernels prefetch the
  // next measurement record before they know whether another one follows
  const size_t nE = std::max<int64_t>(m->n_events, 1), nM = (size_t)N + 1;
  // host copies: pinned for fast re-upload when a device is present, plain
  // otherwise (validation then still runs and reports before any device work)
  m->pinned = cudaMallocHost((void **)&m->h_dt, nE * sizeof(float)) == cudaSuccess &&
              cudaMallocHost((void **)&m->h_tag, nE) == cudaSuccess &&
              cudaMallocHost((void **)&m->h_meas, nM * sizeof(float4)) == cudaSuccess;
  if (!m->pinned) {
    if (m->h_dt) cudaFreeHost(m->h_dt);
    if (m->h_tag) cudaFreeHost(m->h_tag);
    m->h_dt = nullptr;
    m->h_tag = nullptr;
    m->h_meas = nullptr;
    cudaGetLastError();
    m->h_dt = (float *)std::malloc(nE * sizeof(float));
    m->h_tag = (uint8_t *)std::malloc(nE);
    m->h_meas = (float4 *)std::malloc(nM * sizeof(float4));
    if (!m->h_dt || !m->h_tag || !m->h_meas) {
      free_model_buffers(m);
      delete m;
      return GP_SS_ENOMEM;
    }
  }
  m->h_meas[N] = make_float4(0.f, 0.f, 0.f, 0.f);
  std::vector<int2> mev(std::max<int64_t>(N, 1));
  m->tev.assign(nE, 0.0);
  std::vector<double> dt64, meas64;
  if (o.precision == 64) {
    dt64.resize(nE);
    meas64.resize(3 * nM);
  }
  // build series in parallel on host threads
  std::vector<SeriesOut> so(n_series);
  unsigned nthr = std::max(1u, std::min(std::thread::hardware_concurrency(), 64u));
  nthr = std::min<unsigned>(nthr, (unsigned)n_series);
  {
    std::vector<std::thread> pool;
    for (unsigned w = 0; w < nthr; ++w)
      pool.emplace_back([&, w]() {
        for (int s = (int)w; s < n_series; s += (int)nthr)
          build_series(series_offsets[s], series_offsets[s + 1], m->ev_off[s], t_start, t_end,
                       y, yerr, instrument, m->h_dt, m->h_tag, m->h_meas,
                       dt64.empty() ? nullptr : dt64.data(),
                       meas64.empty() ? nullptr : meas64.data(), mev.data(), m->tev.data(),
                       &so[s], m->mixed);
      });
    for (auto &t : pool) t.join();
  }
  int n_slots = (n_inst > 0 && !m->mixed) ? 0 : 1;
  for (int s = 0; s < n_series; ++s) {
    if (so[s].st != GP_SS_OK) {
      gp_ss_status st = so[s].st;
      free_model_buffers(m);
      delete m;
      return st;
    }
    n_slots = std::max(n_slots, so[s].n_slots);
  }
  m->n_slots = n_slots;
  if (m->product) {
    m->ops = m->n_terms == 1 ? gpss::ops_prod1() : gpss::ops_prod2();
    m->ops.comb64 = m->n_terms == 1 ? gpss::comb64_2_0_0() : gpss::comb64_3_0_0();
  } else if (n_slots > kMaxSlots || !pick_ops(m->n_terms, n_slots, m->layout, &m->ops)) {
    free_model_buffers(m);
    delete m;
    return GP_SS_EUNSUPPORTED;
  }
  m->tag.assign(m->h_tag, m->h_tag + m->n_events);
  gp_ss_status st = GP_SS_OK;
  if (!st) st = dev_upload(&m->d_ev_off, m->ev_off.data(), m->ev_off.size());
  if (!st) st = dev_upload(&m->d_meas_off, m->meas_off.data(), m->meas_off.size());
  if (!st) st = dev_upload(&m->d_dt, m->h_dt, nE);
  if (!st) st = dev_upload(&m->d_tag, m->h_tag, nE);
  if (!st) st = dev_upload(&m->d_meas, m->h_meas, nM);
  // the 12-byte records the host-buffer call sends (pinned hosts only)
  if (!st && m->pinned && cudaMallocHost((void **)&m->h_meas3, (size_t)nM * 3 * sizeof(float)) ==
                              cudaSuccess) {
    for (int64_t i = 0; i < N; ++i) {
      m->h_meas3[3 * i] = m->h_meas[i].x;
      m->h_meas3[3 * i + 1] = m->h_meas[i].y;
      m->h_meas3[3 * i + 2] = m->h_meas[i].z;
    }
  } else {
    m->h_meas3 = nullptr;
    cudaGetLastError();
  }
  if (!st) st = dev_upload(&m->d_mev, mev.data(), mev.size());
  if (!st && o.precision == 64) {
    st = dev_upload(&m->d_dt64, dt64.data(), nE);
    if (!st) st = dev_upload(&m->d_meas64, meas64.data(), 3 * nM);
  }
  if (!st) st = make_plan(m, o.chunk_len);
  if (!st) {
    cudaMemPoolProps pp = {};
    pp.allocType = cudaMemAllocationTypePinned;
    pp.handleTypes = cudaMemHandleTypeNone;
    pp.location.type = cudaMemLocationTypeDevice;
    pp.location.id = m->device;
    if (cudaMemPoolCreate(&m->pool, &pp) == cudaSuccess) {
      uint64_t keep = UINT64_MAX;
      cudaMemPoolSetAttribute(m->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    } else {
      m->pool = nullptr;
      cudaGetLastError();
    }
  }
  if (st) {
    free_model_buffers(m);
    delete m;
    return st;
  }
  *out = m;
  return GP_SS_OK;
}

gp_ss_status gp_ss_set_chunk_len(gp_ss_model *m, int chunk_len) {
  if (!m || chunk_len < 0) return GP_SS_EINVAL;
  DeviceGuard g(m->device);
  std::lock_guard<std::mutex> lk(m->mu);
  if (cudaDeviceSynchronize() != cudaSuccess) return GP_SS_ECUDA;
  return make_plan(m, chunk_len);
}

gp_ss_status gp_ss_discretize(const gp_ss_kernel_spec *spec, int n_slots, const float *theta,
                              const float *dt, int n, float *phi_out, float *q_out,
                              void *cuda_stream) {
  if (!spec || !spec->terms || !theta || !dt || !phi_out || !q_out || n < 0) return GP_SS_EINVAL;
  if (spec->n_terms < 1 || spec->n_terms > 2 || n_slots < 1) return GP_SS_EUNSUPPORTED;
  for (int t = 0; t < spec->n_terms; ++t)
    if (spec->terms[t] != GP_SS_TERM_SHO && spec->terms[t] != GP_SS_TERM_MATERN32 &&
        spec->terms[t] != GP_SS_TERM_SHO_PRODUCT)
      return GP_SS_EINVAL;
  // a product term is compiled as the first term, with at most one plain term
  for (int t = 1; t < spec->n_terms; ++t)
    if (spec->terms[t] == GP_SS_TERM_SHO_PRODUCT) return GP_SS_EUNSUPPORTED;
  OpTable o;
  const int layout = spec->n_terms == 1 ? 0 : spec->integral_layout;
  if (!pick_ops(spec->n_terms, n_slots, layout, &o)) return GP_SS_EUNSUPPORTED;
  const int k1 = spec->n_terms > 1 ? spec->terms[1] : 0;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  int np = 1;
  for (int t = 0; t < spec->n_terms; ++t) np += spec->terms[t] == GP_SS_TERM_SHO ? 3 : 2;
  float *tabs = nullptr;
  if (cudaMallocAsync((void **)&tabs, (size_t)o.NT * gpss::TAB_TERM * sizeof(float), st))
    return GP_SS_ENOMEM;
  cudaError_t e = o.tables(theta, 1, np, spec->terms[0], k1, tabs, st);
  if (e == cudaSuccess) e = o.disc(theta, tabs, spec->terms[0], k1, dt, n, phi_out, q_out, st);
  cudaFreeAsync(tabs, st);
  return e == cudaSuccess ? GP_SS_OK : GP_SS_ECUDA;
}

gp_ss_status gp_ss_model_info(const gp_ss_model *m, int *n_series, int64_t *n_meas,
                              int64_t *n_events, int *n_params, int *state_dim, int *n_slots,
                              int *n_chunks) {
  if (!m) return GP_SS_EINVAL;
  if (n_series) *n_series = m->n_series;
  if (n_meas) *n_meas = m->n_meas;
  if (n_events) *n_events = m->n_events;
  if (n_params) *n_params = m->n_params;
  if (state_dim) *state_dim = m->ops.D;
  if (n_slots) *n_slots = m->n_slots;
  if (n_chunks) *n_chunks = m->n_chunks;
  return GP_SS_OK;
}

gp_ss_status gp_ss_loglik(const gp_ss_model *m, const float *theta, int n_sets,
                          int theta_per_series, double *loglik_out, void *cuda_stream) {
  gp_ss_status s = check_call(m, theta, n_sets, theta_per_series, loglik_out);
  if (s) return s;
  DeviceGuard g(m->device);
  return enqueue(m, theta, n_sets, theta_per_series, loglik_out, nullptr,
                 (cudaStream_t)cuda_stream);
}

gp_ss_status gp_ss_loglik_grad(const gp_ss_model *m, const float *theta, int n_sets,
                               int theta_per_series, double *loglik_out, float *grad_out,
                               float *dlogl_dexposure, void *cuda_stream) {
  gp_ss_status s = check_call(m, theta, n_sets, theta_per_series, loglik_out);
  if (s) return s;
  if (!grad_out) return GP_SS_EINVAL;
  if (dlogl_dexposure && m->precision == 64) return GP_SS_EUNSUPPORTED;
  DeviceGuard g(m->device);
  return enqueue(m, theta, n_sets, theta_per_series, loglik_out, grad_out,
                 (cudaStream_t)cuda_stream, dlogl_dexposure);
}

gp_ss_status gp_ss_condition(const gp_ss_model *m, const float *theta, int n_sets,
                             int theta_per_series, double *loglik_out, float *cond_out,
                             void *cuda_stream) {
  gp_ss_status s = check_call(m, theta, n_sets, theta_per_series, loglik_out);
  if (s) return s;
  if (!cond_out) return GP_SS_EINVAL;
  if (m->precision == 64) return GP_SS_EUNSUPPORTED;
  DeviceGuard g(m->device);
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const int n_out = theta_per_series ? m->n_series : n_sets * m->n_series;
  float *grad = nullptr;
  if (scratch_alloc(m, (void **)&grad, (size_t)n_out * m->n_params * sizeof(float), st))
    return GP_SS_ENOMEM;
  s = enqueue(m, theta, n_sets, theta_per_series, loglik_out, grad, st, nullptr, cond_out);
  cudaFreeAsync(grad, st);
  return s;
}

gp_ss_status gp_ss_predict(const gp_ss_model *m, const float *theta, int n_sets,
                           int theta_per_series, const double *t_star,
                           const int64_t *star_offsets, double *loglik_out, float *pred_out,
                           void *cuda_stream) {
  gp_ss_status s = check_call(m, theta, n_sets, theta_per_series, loglik_out);
  if (s) return s;
  if (!t_star || !star_offsets || !pred_out) return GP_SS_EINVAL;
  if (m->precision == 64) return GP_SS_EUNSUPPORTED;
  const int ns = m->n_series;
  if (star_offsets[0] != 0) return GP_SS_EINVAL;
  for (int i = 0; i < ns; ++i)
    if (star_offsets[i + 1] < star_offsets[i]) return GP_SS_EUNSORTED;
  const int64_t M = star_offsets[ns];
  if (M > INT32_MAX / 2) return GP_SS_EUNSUPPORTED;
  for (int64_t j = 0; j < M; ++j)
    if (!std::isfinite(t_star[j])) return GP_SS_EINVAL;
  DeviceGuard g(m->device);
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const int n_out = theta_per_series ? m->n_series : n_sets * m->n_series;
  if (M == 0) return gp_ss_loglik(m, theta, n_sets, theta_per_series, loglik_out, cuda_stream);
  // each test time's interval: the first event at or after it (or none: after
  // the series); gaps formed in FP64 and rounded once
  std::vector<int64_t> key(M);  // event index, or n_events + series for "after"
  std::vector<float2> dd(M);
  std::vector<int> cnt(m->n_events + ns + 1, 0);
  for (int i = 0; i < ns; ++i) {
    const int64_t e0 = m->ev_off[i], e1 = m->ev_off[i + 1];
    const double *t = m->tev.data();
    for (int64_t j = star_offsets[i]; j < star_offsets[i + 1]; ++j) {
      const double ts = t_star[j];
      const int64_t k = std::lower_bound(t + e0, t + e1, ts) - t;
      if (e1 == e0) {
        key[j] = m->n_events + i;  // empty series: the prior (no data)
        dd[j] = make_float2(0.f, 0.f);
      } else if (k == e1) {
        key[j] = m->n_events + i;
        dd[j] = make_float2((float)(ts - t[e1 - 1]), 0.f);
      } else if (k == e0) {
        key[j] = k;
        dd[j] = make_float2(0.f, (float)(t[k] - ts));
      } else {
        key[j] = k;
        dd[j] = make_float2((float)(ts - t[k - 1]), (float)(t[k] - ts));
      }
      ++cnt[key[j]];
    }
  }
  // counting sort by key: interior points by event, then "after" points by series
  std::vector<int> off(m->n_events + ns + 1, 0);
  for (int64_t k = 0; k < m->n_events + ns; ++k) off[k + 1] = off[k] + cnt[k];
  std::vector<int> pos(off.begin(), off.end() - 1), idx(M);
  std::vector<float2> dsort(M);
  for (int64_t j = 0; j < M; ++j) {
    const int p = pos[key[j]]++;
    idx[p] = (int)j;
    dsort[p] = dd[j];
  }
  gp_ss_status res = GP_SS_OK;
  int *d_off = nullptr, *d_idx = nullptr;
  float2 *d_d = nullptr;
  float *grad = nullptr;
  const size_t noff = off.size();
  if (scratch_alloc(m, (void **)&d_off, noff * sizeof(int), st) ||
      scratch_alloc(m, (void **)&d_idx, M * sizeof(int), st) ||
      scratch_alloc(m, (void **)&d_d, M * sizeof(float2), st) ||
      scratch_alloc(m, (void **)&grad, (size_t)n_out * m->n_params * sizeof(float), st))
    res = GP_SS_ENOMEM;
  if (!res && (cudaMemcpyAsync(d_off, off.data(), noff * sizeof(int), cudaMemcpyHostToDevice, st) ||
               cudaMemcpyAsync(d_idx, idx.data(), M * sizeof(int), cudaMemcpyHostToDevice, st) ||
               cudaMemcpyAsync(d_d, dsort.data(), M * sizeof(float2), cudaMemcpyHostToDevice, st)))
    res = GP_SS_ECUDA;
  // points of empty series: the prior, which no kernel visits
  if (!res) {
    bool any_empty = false;
    for (int i = 0; i < ns; ++i) any_empty |= (m->ev_off[i] == m->ev_off[i + 1] &&
                                               star_offsets[i + 1] > star_offsets[i]);
    if (any_empty) res = GP_SS_EUNSUPPORTED;
  }
  if (!res) {
    gpss::PredPlan pp;
    pp.off = d_off;
    pp.xoff = d_off + m->n_events;
    pp.idx = d_idx;
    pp.d = d_d;
    pp.out = pred_out;
    pp.n_star = M;
    res = enqueue(m, theta, n_sets, theta_per_series, loglik_out, grad, st, nullptr, nullptr, &pp);
  }
  // the host vectors must outlive the copies
  if (cudaStreamSynchronize(st) != cudaSuccess && !res) res = GP_SS_ECUDA;
  for (void *p : {(void *)d_off, (void *)d_idx, (void *)d_d, (void *)grad})
    if (p) cudaFreeAsync(p, st);
  return res;
}

gp_ss_status gp_ss_loglik_batched(const gp_ss_model *m, const float *theta, int n_sets,
                                  int theta_per_series, double *loglik_out, void *cuda_stream) {
  gp_ss_status s = check_call(m, theta, n_sets, theta_per_series, loglik_out);
  if (s) return s;
  DeviceGuard g(m->device);
  return run_graph(m, 0, theta, n_sets, theta_per_series, loglik_out, nullptr,
                   (cudaStream_t)cuda_stream);
}

gp_ss_status gp_ss_loglik_grad_batched(const gp_ss_model *m, const float *theta, int n_sets,
                                       int theta_per_series, double *loglik_out,
                                       float *grad_out, void *cuda_stream) {
  gp_ss_status s = check_call(m, theta, n_sets, theta_per_series, loglik_out);
  if (s) return s;
  if (!grad_out) return GP_SS_EINVAL;
  DeviceGuard g(m->device);
  return run_graph(m, 1, theta, n_sets, theta_per_series, loglik_out, grad_out,
                   (cudaStream_t)cuda_stream);
}

gp_ss_status gp_ss_loglik_grad_host(const gp_ss_model *m, const float *theta_host, int n_sets,
                                    int theta_per_series, double *loglik_host, float *grad_host,
                                    int reupload_events, void *cuda_stream) {
  gp_ss_status s = check_call(m, theta_host, n_sets, theta_per_series, loglik_host);
  if (s) return s;
  if (!grad_host) return GP_SS_EINVAL;
  DeviceGuard g(m->device);
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const int n_out = theta_per_series ? m->n_series : n_sets * m->n_series;
  float *d_theta = nullptr, *d_grad = nullptr;
  double *d_ll = nullptr;
  const size_t nth = (size_t)n_sets * m->n_params;
  if (scratch_alloc(m, (void **)&d_theta, nth * sizeof(float), st) != cudaSuccess ||
      scratch_alloc(m, (void **)&d_ll, (size_t)n_out * sizeof(double), st) != cudaSuccess ||
      scratch_alloc(m, (void **)&d_grad, (size_t)n_out * m->n_params * sizeof(float), st) !=
          cudaSuccess) {
    // give back whichever of the three was taken
    void *taken[] = {d_theta, d_ll, d_grad};
    for (void *p : taken)
      if (p) cudaFreeAsync(p, st);
    return GP_SS_ENOMEM;
  }
  gp_ss_status res = GP_SS_OK;
  // A re-sent event stream goes up in series groups on a second stream, and
  // each group's element pass starts as soon as its events are in (the copy
  // of the rest overlaps it).  The copy stream first waits for earlier work
  // on st, which may still read the device copy.  Four groups (c4 element
  // phase with the upload: 1.84 ms with four, 1.90 ms with two; 0.80 ms
  // without the upload, 1.18 ms for the upload alone).
  constexpr int kGroups = 4;
  cudaStream_t cs = nullptr;
  cudaEvent_t start_ev = nullptr, ready[kGroups] = {};
  int c0[kGroups + 1] = {};
  ElemSlices slices{0, c0, ready};
  const bool pipe = reupload_events && !m->product && m->precision == 32 && m->n_series >= 2 &&
                    m->ch_first.size() == (size_t)m->n_series + 1 && m->h_meas3;
  float *d_meas3 = nullptr;
  if (pipe) {
    std::vector<int> sb{0};
    for (int g = 1; g < kGroups; ++g) {
      const int64_t target = m->ev_off[m->n_series] * g / kGroups;
      const int sp = (int)(std::lower_bound(m->ev_off.begin(), m->ev_off.end(), target) -
                           m->ev_off.begin());
      if (sp > sb.back() && sp < m->n_series) sb.push_back(sp);
    }
    sb.push_back(m->n_series);
    slices.n = (int)sb.size() - 1;
    // measurement records go up as 12-byte (y, r0, w) and are widened to the
    // kernels' float4 on the device (a quarter fewer bytes than the float4s)
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) ||
        cudaEventCreateWithFlags(&start_ev, cudaEventDisableTiming) ||
        cudaEventRecord(start_ev, st) || cudaStreamWaitEvent(cs, start_ev, 0) ||
        scratch_alloc(m, (void **)&d_meas3, (size_t)std::max<int64_t>(m->n_meas, 1) * 3 *
                                                sizeof(float), cs))
      res = GP_SS_ECUDA;
    for (int g = 0; g < slices.n && !res; ++g) {
      const int64_t e0 = m->ev_off[sb[g]], e1 = m->ev_off[sb[g + 1]];
      const int64_t q0 = m->meas_off[sb[g]], q1 = m->meas_off[sb[g + 1]];
      c0[g] = m->ch_first[sb[g]];
      if (cudaEventCreateWithFlags(&ready[g], cudaEventDisableTiming) ||
          cudaMemcpyAsync(d_meas3 + 3 * q0, m->h_meas3 + 3 * q0, (size_t)(q1 - q0) * 3 * sizeof(float),
                          cudaMemcpyHostToDevice, cs) ||
          cudaMemcpyAsync(m->d_dt + e0, m->h_dt + e0, (size_t)(e1 - e0) * sizeof(float),
                          cudaMemcpyHostToDevice, cs) ||
          cudaMemcpyAsync(m->d_tag + e0, m->h_tag + e0, (size_t)(e1 - e0),
                          cudaMemcpyHostToDevice, cs)) {
        res = GP_SS_ECUDA;
        break;
      }
      if (q1 > q0) {
        gpss::k_pack_meas<<<(unsigned)((q1 - q0 + 255) / 256), 256, 0, cs>>>(
            d_meas3 + 3 * q0, m->d_meas + q0, q1 - q0);
        GPSS_COUNT_LAUNCH();
      }

      if (cudaGetLastError() != cudaSuccess || cudaEventRecord(ready[g], cs)) res = GP_SS_ECUDA;
    }
    if (d_meas3) cudaFreeAsync(d_meas3, cs);
    c0[slices.n] = m->ch_first[m->n_series];
  } else if (reupload_events) {
    if (cudaMemcpyAsync(m->d_dt, m->h_dt, (size_t)m->n_events * sizeof(float),
                        cudaMemcpyHostToDevice, st) ||
        cudaMemcpyAsync(m->d_tag, m->h_tag, (size_t)m->n_events, cudaMemcpyHostToDevice, st) ||
        cudaMemcpyAsync(m->d_meas, m->h_meas, (size_t)m->n_meas * sizeof(float4),
                        cudaMemcpyHostToDevice, st) ||
        interleave_events(m, 0, m->n_chunks, st))
      res = GP_SS_ECUDA;
  }
  if (!res && cudaMemcpyAsync(d_theta, theta_host, nth * sizeof(float), cudaMemcpyHostToDevice, st))
    res = GP_SS_ECUDA;
  if (!res)
    res = enqueue(m, d_theta, n_sets, theta_per_series, d_ll, d_grad, st, nullptr, nullptr,
                  nullptr, pipe ? &slices : nullptr);
  if (!res && (cudaMemcpyAsync(loglik_host, d_ll, (size_t)n_out * sizeof(double),
                               cudaMemcpyDeviceToHost, st) ||
               cudaMemcpyAsync(grad_host, d_grad, (size_t)n_out * m->n_params * sizeof(float),
                               cudaMemcpyDeviceToHost, st)))
    res = GP_SS_ECUDA;
  cudaFreeAsync(d_theta, st);
  cudaFreeAsync(d_ll, st);
  cudaFreeAsync(d_grad, st);
  if (cudaStreamSynchronize(st) != cudaSuccess && !res) res = GP_SS_ECUDA;
  if (cs) {
    if (cudaStreamSynchronize(cs) != cudaSuccess && !res) res = GP_SS_ECUDA;
    cudaStreamDestroy(cs);
  }
  if (start_ev) cudaEventDestroy(start_ev);
  for (cudaEvent_t e : ready)
    if (e) cudaEventDestroy(e);
  return res;
}

gp_ss_status gp_ss_span_element(const gp_ss_model *m, const float *theta, int n_sets,
                                int theta_per_series, int c_begin, int c_end, double *elem_out,
                                void *cuda_stream) {
  gp_ss_status s = check_call(m, theta, n_sets, theta_per_series, elem_out);
  if (s) return s;
  if (m->n_series != 1 || m->precision != 32) return GP_SS_EUNSUPPORTED;
  if (c_begin < 0 || c_end > m->n_chunks || c_begin >= c_end) return GP_SS_EINVAL;
  DeviceGuard g(m->device);
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const OpTable &o = m->ops;
  const int rows = theta_per_series ? 1 : n_sets;
  const int64_t n_vch64 = (int64_t)rows * m->n_chunks;
  if (n_vch64 > INT32_MAX / 8) return GP_SS_EUNSUPPORTED;
  const int n_vch = (int)n_vch64;
  if ((s = prepare_err(m, rows, st))) return s;
  const gpss::DevModel dm = dev_view(m);
  float *ef = nullptr, *tabs = nullptr;
  double *ed = nullptr, *scratch = nullptr;
  gp_ss_status res = GP_SS_OK;
  if (scratch_alloc(m, (void **)&ef, (size_t)o.NF * n_vch * sizeof(float), st) ||
      scratch_alloc(m, (void **)&ed, (size_t)o.ND * n_vch * sizeof(double), st) ||
      scratch_alloc(m, (void **)&tabs, (size_t)n_sets * o.NT * gpss::TAB_TERM * sizeof(float),
                    st) ||
      scratch_alloc(m, (void **)&scratch, o.span_scratch(c_end - c_begin, rows) * sizeof(double),
                    st)) {
    res = GP_SS_ENOMEM;
  } else if (o.tables(theta, n_sets, m->n_params, m->kinds[0], m->kinds[1], tabs, st) ||
             o.elem(dm, theta, n_vch, theta_per_series, ef, ed, m->d_err, tabs, nullptr, 0,
                    nullptr, c_begin, c_end - c_begin, st) ||
             o.span_element(ef, ed, n_vch, m->n_chunks, c_begin, c_end, rows, scratch, elem_out,
                            st)) {
    res = GP_SS_ECUDA;
  }
  void *bufs[] = {ef, ed, tabs, scratch};
  for (void *p : bufs)
    if (p) cudaFreeAsync(p, st);
  return res;
}

gp_ss_status gp_ss_span_loglik(const gp_ss_model *m, const double *span_elems, int n_spans,
                               int n_rows, double *loglik_out, void *cuda_stream) {
  if (!m || !span_elems || !loglik_out || n_spans < 1 || n_rows < 1) return GP_SS_EINVAL;
  if (m->n_series != 1 || m->precision != 32) return GP_SS_EUNSUPPORTED;
  DeviceGuard g(m->device);
  if (m->ops.span_fold(span_elems, n_spans, n_rows, loglik_out, (cudaStream_t)cuda_stream))
    return GP_SS_ECUDA;
  return GP_SS_OK;
}

gp_ss_status gp_ss_build_events(int64_t n, const double *t_start, const double *t_end,
                                const float *y, const float *yerr, const int32_t *instrument,
                                int64_t *n_events, double *dt_out, uint8_t *tag_out,
                                double *meas_out, int *n_slots) {
  if (n < 0 || !n_events || !n_slots || (n > 0 && (!t_start || !t_end || !y || !yerr ||
                                                  !dt_out || !tag_out || !meas_out)))
    return GP_SS_EINVAL;
  if (n == 0) {
    *n_events = 0;
    *n_slots = 0;
    return GP_SS_OK;
  }
  int64_t n_inst = 0;
  for (int64_t i = 0; i < n; ++i) {
    const int kd = meas_kind(t_start[i], t_end[i], y[i], yerr[i]);
    if (kd < 0) return GP_SS_EINVAL;
    n_inst += kd;
  }
  const bool mixed = n_inst != 0 && n_inst != n;
  const int64_t ne = n_inst == n ? n : 2 * n - n_inst;
  std::vector<float> dt(ne);
  std::vector<uint8_t> tag(ne);
  std::vector<float4> meas(n + 1);
  std::vector<double> dt64(ne), meas64(3 * n), tev(ne);
  std::vector<int2> mev(n);
  SeriesOut so;
  build_series(0, n, 0, t_start, t_end, y, yerr, instrument, dt.data(), tag.data(), meas.data(),
               dt64.data(), meas64.data(), mev.data(), tev.data(), &so, mixed);
  if (so.st) return so.st;
  if (mixed) so.n_slots = std::max(so.n_slots, 1);
  if (so.n_slots > kMaxSlots) return GP_SS_EUNSUPPORTED;
  *n_events = ne;
  *n_slots = so.n_slots;
  std::memcpy(dt_out, dt64.data(), ne * sizeof(double));
  std::memcpy(tag_out, tag.data(), ne);
  std::memcpy(meas_out, meas64.data(), 3 * n * sizeof(double));
  return GP_SS_OK;
}

gp_ss_status gp_ss_last_error_series(const gp_ss_model *m, int64_t *first_bad_series,
                                     gp_ss_status *code) {
  if (!m || !first_bad_series || !code) return GP_SS_EINVAL;
  DeviceGuard g(m->device);
  std::lock_guard<std::mutex> lk(m->mu);
  *first_bad_series = -1;
  *code = GP_SS_OK;
  const int n = m->last_n_out;
  if (n <= 0 || !m->d_err) return GP_SS_OK;
  std::vector<int> h(n);
  if (cudaMemcpy(h.data(), m->d_err, n * sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    return GP_SS_ECUDA;
  for (int i = 0; i < n; ++i)
    if (h[i]) {
      *first_bad_series = i;
      *code = (gp_ss_status)h[i];
      break;
    }
  return GP_SS_OK;
}

gp_ss_status gp_ss_measure_fp32_peak(double *tflops, int *n_sms, void *cuda_stream) {
  if (!tflops || !n_sms) return GP_SS_EINVAL;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return GP_SS_ECUDA;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  float *sink = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  const int blocks = sms * 8, threads = 256, iters = 1 << 16;
  gp_ss_status res = GP_SS_OK;
  if (cudaMalloc((void **)&sink, (size_t)blocks * sizeof(float)) != cudaSuccess)
    return GP_SS_ENOMEM;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    res = GP_SS_ECUDA;
  } else {
    float best = 1e30f;
    for (int r = 0; r < 6 && !res; ++r) {
      cudaEventRecord(e0, st);
      gpss::k_fma_peak<<<blocks, threads, 0, st>>>(sink, iters, 0.999999f, 1e-7f);
      GPSS_COUNT_LAUNCH();
      cudaEventRecord(e1, st);
      float ms = 0.f;
      if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
          cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
        res = GP_SS_ECUDA;
      else if (r > 0)
        best = std::min(best, ms);  // the first launch warms up
    }
    if (!res) *tflops = 2.0 * 8.0 * iters * (double)blocks * threads / (best * 1e-3) / 1e12;
    *n_sms = sms;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(sink);
  return res;
}

gp_ss_status gp_ss_launch_count(int64_t *out) {
  if (!out) return GP_SS_EINVAL;
  *out = (int64_t)gpss::g_launches.load(std::memory_order_relaxed);
  return GP_SS_OK;
}

gp_ss_status gp_ss_autotune(gp_ss_model *m, const float *theta, int n_sets,
                            int theta_per_series, int want_grad, int reps, gp_ss_tuning *best,
                            void *cuda_stream) {
  gp_ss_status s = check_call(m, theta, n_sets, theta_per_series, best);
  if (s) return s;
  if (m->precision != 32 || reps < 1 || reps > 100) return GP_SS_EINVAL;
  if (m->product) return GP_SS_EUNSUPPORTED;  // product models are not tuned
  DeviceGuard g(m->device);
  cudaStream_t st = (cudaStream_t)cuda_stream;
  if (cudaDeviceSynchronize() != cudaSuccess) return GP_SS_ECUDA;
  const int n_out = theta_per_series ? m->n_series : n_sets * m->n_series;
  double *ll = nullptr;
  float *gr = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaMalloc((void **)&ll, (size_t)n_out * sizeof(double)) ||
      (want_grad && cudaMalloc((void **)&gr, (size_t)n_out * m->n_params * sizeof(float))) ||
      cudaEventCreate(&e0) || cudaEventCreate(&e1)) {
    if (ll) cudaFree(ll);
    if (gr) cudaFree(gr);
    if (e0) cudaEventDestroy(e0);
    return GP_SS_ENOMEM;
  }
  // candidates: (schedule, chunk length, combination, segment length)
  struct Cand {
    int schedule, L, combine, ck;
  };
  std::vector<Cand> cands;
  // chunk lengths: besides the work per thread, the length sets how many
  // waves of blocks a launch takes, so lengths between the round ones let the
  // last wave come out fuller
  const int Ls[] = {64, 128, 160, 192, 224, 256, 288, 320, 384, 448, 512, 1024};
  if (want_grad) {
    for (int ck : {32, 64}) {
      cands.push_back({1, 0, 2, ck});
      for (int L : Ls)
        if (L >= 128 && L <= 512) cands.push_back({2, L, 2, ck});
    }
    cands.push_back({2, 256, 2, 16});
    cands.push_back({2, 256, 1, 32});
  } else {
    cands.push_back({3, 0, 2, 32});
    for (int cb : {2, 1}) {
      cands.push_back({1, 0, cb, 32});
      for (int L : Ls) cands.push_back({2, L, cb, 32});
    }
  }
  const Cand saved{m->schedule, m->chunk_len, m->combine, m->ckpt_interval};
  Cand win = saved;
  double win_ms = 1e300;
  int tried = 0;
  gp_ss_status res = GP_SS_OK;
  for (const Cand &c : cands) {
    m->schedule = c.schedule;
    m->combine = c.combine;
    m->ckpt_interval = c.ck;
    if ((res = make_plan(m, c.schedule == 2 ? c.L : 0))) break;
    std::vector<float> t;
    for (int r = 0; r <= reps && !res; ++r) {
      cudaEventRecord(e0, st);
      res = enqueue(m, theta, n_sets, theta_per_series, ll, gr, st);
      cudaEventRecord(e1, st);
      if (cudaEventSynchronize(e1) != cudaSuccess) res = GP_SS_ECUDA;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (r > 0) t.push_back(ms);  // the first run warms up
    }
    if (res) break;
    std::sort(t.begin(), t.end());
    const double med = t[t.size() / 2];
    ++tried;
    if (med < win_ms) {
      win_ms = med;
      win = c;
    }
  }
  // apply the winner (or restore the old settings on failure)
  const Cand &use = res ? saved : win;
  m->schedule = use.schedule;
  m->combine = use.combine;
  m->ckpt_interval = use.ck;
  gp_ss_status r2 = make_plan(m, use.schedule == 2 ? use.L : (res ? saved.L : 0));
  if (!res) res = r2;
  if (!res && best) {
    best->schedule = win.schedule;
    best->chunk_len = m->chunk_len;
    best->chunk_combine = win.combine;
    best->ckpt_interval = win.ck;
    best->threads_per_series = m->max_chunks_per_series;
    best->ms = win_ms;
    best->n_tried = tried;
  }
  cudaFree(ll);
  if (gr) cudaFree(gr);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return res;
}

gp_ss_status gp_ss_set_timing(gp_ss_model *m, int enable) {
  if (!m) return GP_SS_EINVAL;
  std::lock_guard<std::mutex> lk(m->mu);
  m->timing = enable != 0;
  return GP_SS_OK;
}

gp_ss_status gp_ss_get_timing(gp_ss_model *m, double *ms, int64_t *launches) {
  if (!m || !ms || !launches) return GP_SS_EINVAL;
  DeviceGuard g(m->device);
  std::vector<std::tuple<int, cudaEvent_t, cudaEvent_t>> tv;
  {
    std::lock_guard<std::mutex> lk(m->mu);
    tv.swap(m->timings);
  }
  for (int i = 0; i < 5; ++i) {
    ms[i] = 0.0;
    launches[i] = 0;
  }
  gp_ss_status res = GP_SS_OK;
  for (auto &t : tv) {
    float e = 0.f;
    if (cudaEventSynchronize(std::get<2>(t)) != cudaSuccess ||
        cudaEventElapsedTime(&e, std::get<1>(t), std::get<2>(t)) != cudaSuccess)
      res = GP_SS_ECUDA;
    ms[std::get<0>(t)] += e;
    launches[std::get<0>(t)] += 1;
    cudaEventDestroy(std::get<1>(t));
    cudaEventDestroy(std::get<2>(t));
  }
  return res;
}

void gp_ss_free_model(gp_ss_model *m) {
  if (!m) return;
  {
    DeviceGuard g(m->device);
    cudaDeviceSynchronize();
    free_model_buffers(m);
  }
  delete m;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Log-likelihood without any device allocation.
//
// gp_ss_loglik takes its chunk-element scratch from the stream-ordered
// allocator on every call.  Some callers cannot allocate device memory at
// call time: a host application that has handed all device memory to its own
// pool, code that must not risk the device-wide synchronisation or the
// latency of an allocation inside a latency-critical loop, or a process whose
// allocator is disabled or capped.  For them, gp_ss_loglik_noalloc runs the
// same element pass and sequential per-series combination out of one fixed
// scratch array compiled into this library.
// ---------------------------------------------------------------------------
namespace {

constexpr size_t kNoAllocScratchBytes = (size_t)16 << 20;  // 16 MiB per GPU
constexpr int kNoAllocMaxDevices = 64;

// One copy exists on every GPU that loads the library, for the life of the
// process.  Host code must not use this name as a pointer; it takes the
// device address with cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_noalloc_mu;
void *g_noalloc_ptr[kNoAllocMaxDevices] = {nullptr};

// Device address of the scratch array on `dev`, looked up once per device
// with that device current.
gp_ss_status noalloc_scratch(int dev, void **out) {
  if (dev < 0 || dev >= kNoAllocMaxDevices) return GP_SS_EUNSUPPORTED;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return GP_SS_ECUDA;
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return GP_SS_OK;
}

}  // namespace

extern "C" gp_ss_status gp_ss_loglik_noalloc(const gp_ss_model *m, const float *theta,
                                             int n_sets, int theta_per_series,
                                             double *loglik_out, void *cuda_stream) {
  gp_ss_status s = check_call(m, theta, n_sets, theta_per_series, loglik_out);
  if (s) return s;
  if (m->precision != 32 || m->product) return GP_SS_EUNSUPPORTED;
  const int n_out = theta_per_series ? m->n_series : n_sets * m->n_series;
  const int64_t n_vch64 = (int64_t)(theta_per_series ? 1 : n_sets) * m->n_chunks;
  const OpTable &o = m->ops;
  // Taylor tables of the hyperparameter rows, element floats (field-major),
  // then the three FP64 sums per chunk
  const size_t t_bytes =
      ((size_t)n_sets * o.NT * gpss::TAB_TERM * sizeof(float) + 255) & ~(size_t)255;
  const size_t f_bytes = ((size_t)o.NF * (size_t)n_vch64 * sizeof(float) + 255) & ~(size_t)255;
  const size_t need = t_bytes + f_bytes + (size_t)o.ND * (size_t)n_vch64 * sizeof(double);
  if (n_vch64 > INT32_MAX / 8 || need > kNoAllocScratchBytes) return GP_SS_ETOOBIG;
  DeviceGuard g(m->device);
  void *base = nullptr;
  s = noalloc_scratch(m->device, &base);
  if (s) return s;
  float *tabs = (float *)base;
  float *ef = (float *)((unsigned char *)base + t_bytes);
  double *ed = (double *)((unsigned char *)base + t_bytes + f_bytes);
  const int n_vch = (int)n_vch64;
  const gpss::DevModel dm = dev_view(m);
  cudaStream_t st = (cudaStream_t)cuda_stream;
  // every field the combination reads is written by the element pass first,
  // so nothing in the shared array needs clearing between calls
  if (o.tables(theta, n_sets, m->n_params, m->kinds[0], m->kinds[1], tabs, st) != cudaSuccess ||
      o.elem(dm, theta, n_vch, theta_per_series, ef, ed, nullptr, tabs, nullptr, 0, nullptr, 0,
             m->n_chunks, st) !=
          cudaSuccess)
    return GP_SS_ECUDA;
  const gpss::CombineOps &cb = m->comb_prec == 64 ? o.comb64 : o.comb32;
  if (cb.scan(dm, n_out, theta_per_series, ef, ed, n_vch, nullptr, nullptr, loglik_out, 0,
              nullptr, st) != cudaSuccess)
    return GP_SS_ECUDA;
  return GP_SS_OK;
}
