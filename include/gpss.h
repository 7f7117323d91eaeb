/*
 * gpss.h -- C ABI of libgpss: the log-likelihood (and its gradient) of a
 * Gaussian process observed through integrated, possibly overlapping
 * exposures, computed on the GPU by a Kalman filter over the augmented
 * state-space model of Rubenzahl, Hattori et al., "Scalable Gaussian
 * Processes for Integrated and Overlapping Measurements via Augmented
 * State-Space Models" (arXiv 2601.02527).
 *
 * The model (Section 3.2 of the paper): measurement n averages the latent
 * process f = H x over its exposure [t_start[n], t_end[n]],
 *     y_n = (1/delta_n) * int_{t_start}^{t_end} f(t) dt + eps_n,
 *     delta_n = t_end - t_start,  eps_n ~ N(0, yerr_n^2 + s^2),
 * where x is the state of a sum of stochastically driven damped harmonic
 * oscillator (SHO) and Matern-3/2 terms (Appendix B, Appendix C.1) and s is a
 * white-noise standard deviation.  The state is augmented with one integral
 * state per instrument slot (Section 3.2.3), reset at each exposure start and
 * read at each exposure end.  The returned value is the log marginal
 * likelihood of Eq. loglikelihood.
 *
 * Conventions
 *  - Every call returns a gp_ss_status; no C++ exception crosses the ABI.
 *  - "host" pointers are ordinary CPU memory; "device" pointers are CUDA
 *    device memory of the device that was current when the model was built.
 *  - Compute calls are asynchronous on the caller's stream (a cudaStream_t
 *    passed as void*, NULL = legacy default stream).  Numeric failures found
 *    on the device (a non-positive or non-finite innovation variance) are
 *    reported by gp_ss_last_error_series() after the stream has synchronised.
 *  - Scratch memory is taken from the stream-ordered allocator
 *    (cudaMallocAsync) on the caller's stream and released before the call
 *    returns, so calls on different streams may share one model.
 *  - Hyperparameters are natural parameters, one row of n_params floats per
 *    set: per term (sigma, omega0, Q) for GP_SS_TERM_SHO (any Q > 0: the
 *    overdamped oscillator Q < 1/2 of Appendix B included), (sigma, ell)
 *    for GP_SS_TERM_MATERN32 or (sigma, omega_a, Q_a, omega_b, Q_b) for
 *    GP_SS_TERM_SHO_PRODUCT, in the order of the kernel spec, then the
 *    white-noise sd s.  n_params = 3*#SHO + 2*#Matern + 5*#product + 1.
 *    Non-finite or non-positive hyperparameters surface as GP_SS_ENUMERIC
 *    (gp_ss_last_error_series).
 *  - A measurement with t_end == t_start is instantaneous: it observes the
 *    latent f(t) itself (Section 2), as one event.  A model of instantaneous
 *    measurements only has no integral states; one that mixes them with
 *    exposure averages keeps the exposures' integral states and orders
 *    simultaneous events exposure ends, then instants, then starts.
 *    (Product kernels: instantaneous measurements only.)
 */
#ifndef GPSS_H
#define GPSS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gp_ss_model gp_ss_model; /* opaque; immutable after build */

typedef enum {
  GP_SS_OK = 0,
  GP_SS_EINVAL = 1,        /* bad argument: negative or non-finite exposure length, NULL pointer, ... */
  GP_SS_EUNSORTED = 2,     /* series offsets not non-decreasing */
  GP_SS_ESELFOVERLAP = 3,  /* one instrument's exposures overlap each other */
  GP_SS_EUNSUPPORTED = 4,  /* model shape not compiled (too many terms/slots) */
  GP_SS_ENOMEM = 5,        /* device or host allocation failed */
  GP_SS_ECUDA = 6,         /* a CUDA runtime call failed */
  GP_SS_ENUMERIC = 7,      /* S <= 0 or non-finite value met on the device */
  GP_SS_ETIMEOUT = 8,      /* a bounded device wait gave up */
  GP_SS_ETOOBIG = 9        /* problem exceeds the fixed scratch of gp_ss_loglik_noalloc */
} gp_ss_status;

typedef enum {
  GP_SS_TERM_SHO = 1,      /* (sigma, omega0, Q): Appendix B, Eq. sho_kernel */
  GP_SS_TERM_MATERN32 = 2, /* (sigma, ell) == SHO with Q = 1/2, omega0 = sqrt(3)/ell */
  GP_SS_TERM_SHO_PRODUCT = 3 /* (sigma, omega_a, Q_a, omega_b, Q_b): sigma^2 k_a k_b, two
                                unit-variance SHO factors (Appendix C.2, Kronecker state of
                                dimension 4).  First term only, at most one plain term after
                                it, instantaneous measurements only; gp_ss_loglik (FP32
                                parallel in time, or the plain per-series filter: FP64 and
                                schedule 3) and gp_ss_loglik_grad (hyperparameter gradient
                                by forward-mode tangents in FP32: per chunk and parameter
                                against the combination's boundary adjoints, or per series
                                and parameter under schedule 3); other calls return
                                GP_SS_EUNSUPPORTED. */
} gp_ss_term;

typedef struct {
  int n_terms;          /* 1..2 */
  const int *terms;     /* host [n_terms] gp_ss_term values */
  int integral_layout;  /* 0: one integral state per slot integrating H x (Section 3.2.3);
                           1: one integral state per term and slot; the measurement reads
                              their sum.  Both give the same likelihood. */
} gp_ss_kernel_spec;

typedef struct {
  int precision;          /* 32 (default): FP32 filter with FP64 log-det/likelihood sums;
                             64: plain FP64 per-series filter (log-likelihood only) */
  int schedule;           /* 0 auto (chunked, default chunk length);
                             1 one warp per series: 32 chunks per series;
                             2 chunked parallel-in-time with chunk_len events per chunk;
                             3 one thread per series running the whole filter (the
                               log-likelihood; gradient calls use one warp per series) */
  int threads_per_series; /* reserved, must be 0 or 1 */
  int chunk_len;          /* events per chunk of the parallel-in-time schedule, 0 = auto */
  int ckpt_interval;      /* events per recomputation segment of the gradient: 8, 16, 32
                             or 64 (0 = 32); the reverse sweep replays each segment from
                             its starting state before walking it backwards */
  int debug_checks;       /* nonzero: extra host-side validation */
  int chunk_combine;      /* combination of chunk elements across a series: 0 auto (= 2),
                             1 sequential fold per series (one thread per series),
                             2 parallel scan (Section 3.2.5): each warp's 32 chunks in
                               shared memory, then a tree scan of the warp totals */
  int step_cache;         /* gradient calls: 0 auto -- the element pass keeps every step's
                             per-term scalars (f, f', F1, I_ff, I_pp, I_FF) in device
                             memory for the reverse sweep while they take at most 8 GiB
                             (24 bytes per event and term per theta set), else the sweep
                             recomputes them; 1 always recompute */
  int combine_precision;  /* arithmetic of the combination of chunk elements across a series
                             (every level of the scan of Section 3.2.5, the closed-form chunk
                             log-likelihoods and the adjoints at chunk ends): 0 auto (= 32),
                             64 FP64, 32 FP32.  The chunk elements themselves are always
                             FP32; the log-likelihood sums are always FP64. */
} gp_ss_options;

/* Build a model from exposures (Section 3.2: two events per exposure, reset
 * at the start, measurement at the end; Section 3.2.3: one integral state per
 * instrument slot).
 *   spec            host, kernel structure
 *   n_series        number of independent series (>= 1)
 *   series_offsets  host int64 [n_series+1], non-decreasing, offsets[0] = 0;
 *                   series i owns measurements [offsets[i], offsets[i+1])
 *   t_start, t_end  host f64 [N] exposure windows (t_end > t_start, finite)
 *   y, yerr         host f32 [N] exposure-averaged values and their sd
 *   instrument      host i32 [N] slot label per measurement (>= 0, one label
 *                   must not overlap itself: t_end <= next t_start), or NULL
 *                   for greedy assignment (lowest free slot in start order)
 *   opts            host, may be NULL for defaults
 *   out             receives the model; the caller frees it with gp_ss_free_model
 * Events are ordered by time with every exposure end before any start at
 * the same time, and time gaps are formed in FP64 before rounding to FP32.
 * Inputs are copied; the model owns its device buffers.  Returns EINVAL,
 * EUNSORTED, ESELFOVERLAP, EUNSUPPORTED (more than 3 slots, or a shape with
 * augmented dimension above 7), ENOMEM or ECUDA on failure. */
gp_ss_status gp_ss_build_model(const gp_ss_kernel_spec *spec, int n_series,
                               const int64_t *series_offsets, const double *t_start,
                               const double *t_end, const float *y, const float *yerr,
                               const int32_t *instrument, const gp_ss_options *opts,
                               gp_ss_model **out);

/* Log-likelihood (Eq. loglikelihood) for n_sets hyperparameter vectors.
 *   theta             device f32 [n_sets * n_params], natural parameters
 *   theta_per_series  1: n_sets == n_series, set i applies to series i;
 *                     0: every set applies to every series
 *   loglik_out        device f64 [n_series] (per-series mode) or
 *                     [n_sets * n_series] (set-major) in the other mode */
gp_ss_status gp_ss_loglik(const gp_ss_model *model, const float *theta, int n_sets,
                          int theta_per_series, double *loglik_out, void *cuda_stream);

/* Log-likelihood and its gradient with respect to the natural parameters,
 * by a reverse-time adjoint of the filter (the paper states the likelihood
 * only; Section 2.4 notes it feeds gradient-based optimisation).
 *   grad_out   device f32 [n_out * n_params], same row order as loglik_out
 *   dlogl_dexposure  NULL, or device f32 [rows * N * 2]: the gradient with respect
 *              to every exposure window, (d/d t_start, d/d t_end) of measurement n (in
 *              the build's measurement order) at [(row * N + n) * 2 + {0, 1}];
 *              rows = 1 when theta_per_series (each series' own theta), else n_sets.
 *              The event order is held fixed (windows that touch stay ordered end
 *              before start).  FP32 models only (GP_SS_EUNSUPPORTED otherwise). */
gp_ss_status gp_ss_loglik_grad(const gp_ss_model *model, const float *theta, int n_sets,
                               int theta_per_series, double *loglik_out, float *grad_out,
                               float *dlogl_dexposure, void *cuda_stream);

/* Conditioned mean and variance of every measurement's exposure average
 * given all of its series' data (the integrated RTS smoother of Section
 * 3.2, Eqs. rts and integrated_rts: the smoothed state at each exposure end
 * projected through H~ = e_z / delta), with the log-likelihood.  Computed by
 * the gradient pipeline: the smoothed state is the filtered state corrected
 * by the adjoint of the log-likelihood of all later data.
 *   loglik_out  as gp_ss_loglik
 *   cond_out    device f32 [rows * N * 2]: (mean, variance) of measurement n
 *               (build order) at [(row * N + n) * 2 + {0, 1}]; rows = 1 when
 *               theta_per_series, else n_sets.  The variance is that of the
 *               noise-free exposure average (white noise and yerr excluded).
 *   FP32 models only (GP_SS_EUNSUPPORTED otherwise). */
gp_ss_status gp_ss_condition(const gp_ss_model *model, const float *theta, int n_sets,
                             int theta_per_series, double *loglik_out, float *cond_out,
                             void *cuda_stream);

/* Prediction of the latent f(t*) = sum of the terms' x(t*) at arbitrary test
 * times, mean and variance given all of the series' data (Section 2.5,
 * Algorithm 1 on the augmented model: retrodiction before the data,
 * interpolation between events -- inside exposures too --, extrapolation
 * after), with the log-likelihood.  Computed by the gradient pipeline: at
 * each event the walk predicts every test time of the interval before it
 * from the filtered state and corrects it by the event's adjoint.
 *   t_star        host f64 [M], test times of series i at
 *                 [star_offsets[i], star_offsets[i+1]), any order
 *   star_offsets  host int64 [n_series + 1], non-decreasing, [0] = 0
 *   loglik_out    as gp_ss_loglik
 *   pred_out      device f32 [rows * M * 2]: (mean, variance) of test time j at
 *                 [(row * M + j) * 2 + {0, 1}]; rows as gp_ss_condition
 *   Test times of a series without measurements: GP_SS_EUNSUPPORTED.  The
 *   call synchronises the stream (the test-time plan is built on the host).
 *   FP32 models only. */
gp_ss_status gp_ss_predict(const gp_ss_model *model, const float *theta, int n_sets,
                           int theta_per_series, const double *t_star,
                           const int64_t *star_offsets, double *loglik_out, float *pred_out,
                           void *cuda_stream);

/* Same computations replayed from a CUDA graph captured on first use for
 * this (model, pointers, n_sets, mode); a later call with other pointers
 * re-captures.  The first call must not itself be made during a capture. */
gp_ss_status gp_ss_loglik_batched(const gp_ss_model *model, const float *theta, int n_sets,
                                  int theta_per_series, double *loglik_out, void *cuda_stream);
gp_ss_status gp_ss_loglik_grad_batched(const gp_ss_model *model, const float *theta,
                                       int n_sets, int theta_per_series, double *loglik_out,
                                       float *grad_out, void *cuda_stream);

/* Host-buffer variant of gp_ss_loglik_grad for end-to-end use: copies theta
 * (host f32) to the device, optionally re-uploads the model's event stream
 * from its pinned host copy (reupload_events != 0), computes, and copies the
 * results back into host buffers before returning (synchronous).  The
 * re-upload goes in series groups on an internal copy stream (it first waits
 * for the work already queued on cuda_stream), each group's element pass
 * starting once its events are in; it rewrites the model's device copy, so
 * it must not run concurrently with other calls on the same model. */
gp_ss_status gp_ss_loglik_grad_host(const gp_ss_model *model, const float *theta_host,
                                    int n_sets, int theta_per_series, double *loglik_host,
                                    float *grad_host, int reupload_events, void *cuda_stream);

/* The per-step discretisation on its own: for n gaps dt (device f32 [n]) and
 * one parameter row theta (device f32 [n_params]), write the augmented
 * transition Phi~(dt) (Eq. phiaug with the block layout of Section 3.2.3) and
 * process noise Q~(dt) (Eq. Q_aug) as dense row-major d x d matrices,
 * d = 2*n_terms + n_slots*(layout ? n_terms : 1), into phi_out and q_out
 * (device f32 [n * d * d] each).  Same arithmetic as inside the filters. */
gp_ss_status gp_ss_discretize(const gp_ss_kernel_spec *spec, int n_slots, const float *theta,
                              const float *dt, int n, float *phi_out, float *q_out,
                              void *cuda_stream);

/* Log-likelihood without device allocation.  (Not part of the paper's method:
 * a deployment variant of gp_ss_loglik.)
 * gp_ss_loglik takes scratch memory from the stream-ordered allocator on every
 * call.  Callers that cannot allocate device memory at call time -- a host
 * application that gives all device memory to its own pool, a latency-critical
 * loop that must not pay for or synchronise on an allocation, a process whose
 * allocator is disabled or capped -- can call this instead.  It computes the
 * same log-likelihood (FP32 models only; element pass plus sequential
 * per-series combination in the model's combination_precision) with its
 * scratch in one array of 16 MiB compiled
 * into the library: every GPU that loads libgpss holds that array until the
 * process exits.  It calls no allocation routine of CUDA or of any library.
 *   - Arguments and result as gp_ss_loglik; theta and loglik_out are
 *     caller-owned device buffers.
 *   - Scratch needed: 800*n_terms*n_sets bytes of step-scalar tables and
 *     NF*n_chunks*4 bytes (each rounded up to 256) + 24*n_chunks bytes,
 *     NF = 2d^2 + 3d (d = augmented dimension; 90 at d = 6), n_chunks the
 *     model's chunk count times n_sets when theta_per_series = 0.
 *     A call that needs more than 16 MiB returns GP_SS_ETOOBIG and launches
 *     nothing.
 *   - The first call on a device looks up the array's device address with
 *     that device current; make that first call before any stream capture.
 *   - All calls share the one array and it keeps the last call's contents
 *     (every value is written before it is read, so nothing needs clearing).
 *     Calls whose work overlaps on the GPU -- on different streams, or from
 *     different threads without ordering -- race on the array: serialise them.
 *   - Device-side numeric failures are not recorded for
 *     gp_ss_last_error_series; check loglik_out for non-finite values. */
gp_ss_status gp_ss_loglik_noalloc(const gp_ss_model *model, const float *theta, int n_sets,
                                  int theta_per_series, double *loglik_out, void *cuda_stream);

/* Model facts: any output pointer may be NULL. */
gp_ss_status gp_ss_model_info(const gp_ss_model *model, int *n_series, int64_t *n_meas,
                              int64_t *n_events, int *n_params, int *state_dim,
                              int *n_slots, int *n_chunks);

/* Re-plan the parallel-in-time chunks (events per chunk); 0 = auto. */
gp_ss_status gp_ss_set_chunk_len(gp_ss_model *model, int chunk_len);

/* After the stream of the last compute call has synchronised: the first
 * series (output row) with a device-side failure and its code, or -1/GP_SS_OK. */
gp_ss_status gp_ss_last_error_series(const gp_ss_model *model, int64_t *first_bad_series,
                                     gp_ss_status *code);

/* Per-phase device timing, for profiling.  With enable != 0, later direct
 * compute calls (not graph replays, not calls made during a stream capture)
 * record a CUDA event pair on the caller's stream around each kernel phase.
 * gp_ss_get_timing waits for the recorded events, writes the accumulated
 * milliseconds and launch counts per phase into ms[5] / launches[5]
 * (0 chunk elements, 1 cross-chunk combination, 2 reverse-time gradient,
 * 3 result conversion, 4 plain per-series filter) and clears the record. */
gp_ss_status gp_ss_set_timing(gp_ss_model *model, int enable);
gp_ss_status gp_ss_get_timing(gp_ss_model *model, double *ms, int64_t *launches);

/* Autotuner (no counterpart in the paper): times candidate schedules on this
 * model with the caller's theta and keeps the fastest.  Candidates: one
 * thread per series (log-likelihood only), one warp per series, and chunked
 * parallel-in-time with chunk lengths 64..1024 (which sets the threads per
 * series), each with the warp-level or the sequential cross-chunk
 * combination, and for gradient calls segment lengths 16, 32 and 64.  Each
 * candidate runs once to warm up, then reps times (1..100) timed with CUDA
 * events on the stream; the median decides.
 *   The model's plan changes: no other call may use the model meanwhile; the
 *   call synchronises the device.  theta as gp_ss_loglik; want_grad selects
 *   loglik+grad (1) or loglik (0) timing; best (host) receives the choice. */
typedef struct {
  int schedule;           /* 1, 2 or 3 as gp_ss_options.schedule */
  int chunk_len;          /* events per chunk of the chosen plan */
  int chunk_combine;      /* 1 sequential, 2 warp-level + scan of warp totals */
  int ckpt_interval;      /* gradient segment length */
  int threads_per_series; /* chunks (threads) given to the longest series */
  int n_tried;            /* candidates timed */
  double ms;              /* median time per call of the choice */
} gp_ss_tuning;

gp_ss_status gp_ss_autotune(gp_ss_model *model, const float *theta, int n_sets,
                            int theta_per_series, int want_grad, int reps, gp_ss_tuning *best,
                            void *cuda_stream);

/* Kernels this library has launched in the calling process, all models and
 * devices together (no counterpart in the paper; an accounting aid).  Counted
 * on the host at every launch, so kernels replayed from a captured CUDA graph
 * (the _batched calls after their first capture) are not included.
 *   out  host int64, written.  GP_SS_EINVAL if NULL. */
gp_ss_status gp_ss_launch_count(int64_t *out);

/* A single long series split in time across devices (Section 3.2.5: the
 * associative combination of the elements of Sarkka & Garcia-Fernandez 2021,
 * applied to contiguous ranges of the model's chunks).  Every device builds
 * the same one-series model; device r calls gp_ss_span_element on its chunk
 * range, the spans' elements are exchanged (an all-gather of a few hundred
 * bytes per span and row), and gp_ss_span_loglik folds them in time order.
 *
 * gp_ss_span_element: the element of chunks [c_begin, c_end) of a model with
 * one series (FP32 models only), for every row (theta_per_series = 1: one
 * set, one row; 0: n_sets rows), combined in FP64:
 *   elem_out  device f64 [rows * (NF + 1)], per row the fields A (d x d,
 *             row-major), b (d), C (d(d+1)/2, packed upper triangle), eta (d),
 *             J (packed), then the log-normaliser c; NF = 2d^2 + 3d.  The data
 *             of the range have likelihood exp(c + eta^T x - x^T J x / 2)
 *             given the state x entering it, which then leaves it as
 *             N(A x + b, C); the range starting at chunk 0 has A = 0 and c its
 *             own log-likelihood.
 * Returns EUNSUPPORTED for models with more than one series, EINVAL for an
 * empty or out-of-range chunk range.  Numeric failures as gp_ss_loglik. */
gp_ss_status gp_ss_span_element(const gp_ss_model *model, const float *theta, int n_sets,
                                int theta_per_series, int c_begin, int c_end, double *elem_out,
                                void *cuda_stream);

/* gp_ss_span_loglik: the series' log-likelihood per row from the elements of
 * n_spans consecutive chunk ranges covering the series in time order, the
 * first starting at chunk 0.
 *   span_elems  device f64 [n_spans * n_rows * (NF + 1)], span-major
 *   loglik_out  device f64 [n_rows] */
gp_ss_status gp_ss_span_loglik(const gp_ss_model *model, const double *span_elems, int n_spans,
                               int n_rows, double *loglik_out, void *cuda_stream);

/* Host-only event build of one series, as gp_ss_build_model builds each
 * series (no CUDA call; for host-side checks and tools).
 *   n                       measurements; inputs as gp_ss_build_model
 *   n_events                host, receives 2n (exposures) or n (instantaneous)
 *   dt_out                  host f64 [2n], gaps between consecutive events
 *   tag_out                 host u8 [2n], bit 0 measurement event, bits 1-3 slot
 *   meas_out                host f64 [3n], (y, yerr^2, 1/delta) of each
 *                           measurement in the order its event comes
 *                           (1/delta = 1 for an instantaneous measurement)
 *   n_slots                 host, receives the number of integral-state slots
 * Returns EINVAL, ESELFOVERLAP or EUNSUPPORTED as gp_ss_build_model. */
gp_ss_status gp_ss_build_events(int64_t n, const double *t_start, const double *t_end,
                                const float *y, const float *yerr, const int32_t *instrument,
                                int64_t *n_events, double *dt_out, uint8_t *tag_out,
                                double *meas_out, int *n_slots);

/* FP32 FMA throughput of the current device (no counterpart in the paper; a
 * measurement aid for the roofline of the FP32-bound kernels): a kernel of
 * independent FMA chains on 8 blocks of 256 threads per SM, timed with CUDA
 * events on the stream, best of five launches after one warm-up.
 *   tflops  host, receives 2 x FMAs / second / 1e12
 *   n_sms   host, receives the device's multiprocessor count
 * Synchronises the stream.  Allocates (and frees) a few bytes of device
 * memory. */
gp_ss_status gp_ss_measure_fp32_peak(double *tflops, int *n_sms, void *cuda_stream);

void gp_ss_free_model(gp_ss_model *model);
const char *gp_ss_status_string(gp_ss_status status);

#ifdef __cplusplus
}
#endif

#endif /* GPSS_H */
