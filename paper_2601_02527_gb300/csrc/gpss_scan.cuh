// Parallel-in-time combination of chunk elements (Section 3.2.5 of
// arXiv 2601.02527; operator of Sarkka & Garcia-Fernandez 2021).
//
// An element E = (A, b, C, eta, J) describes one stretch of events: given the
// state x entering it, the filtered state leaving it is N(A x + b, C), and
// the stretch's data carry information (eta, J) about x.  Combining E_i
// (earlier) with E_j (later), with X = I + C_i J_j:
//   Y = X^{-1} A_i,  W = X^{-1} C_i,  w = X^{-1} (b_i + C_i eta_j)
//   A = A_j Y,  b = A_j w + b_j,  C = A_j W A_j^T + C_j,
//   eta = Y^T (eta_j - J_j b_i) + eta_i,  J = Y^T J_j A_i + J_i,
// which is the SG21 operator written with one factorisation of X (the
// (I + J_j C_i)^{-1} there equals X^{-T}).  The identity element is
// (I, 0, 0, 0, 0).  The first chunk of every series has A = 0 and
// eta = J = 0, so one unsegmented scan over all chunks of all series restarts
// at every series boundary in both directions.
//
// Scan structure (no inter-block waiting): for n elements and tiles of T,
//   1. k_tile_reduce   one block per tile folds its T elements (tree);
//   2. the tile totals are scanned recursively by the same three steps;
//   3. k_tile_scan     one block per tile: Blelloch exclusive scan in shared
//                      memory, then prefix-of-tile o exclusive o own element.
// rev = 1 runs the mirrored scan (suffixes), whose operator is the same
// combine with its arguments in time order.
#pragma once

#include "gpss_device.cuh"

namespace gpss {

template <class S>
struct Elem {
  static constexpr int D = S::D;
  static constexpr int NP = S::NP;
  static constexpr int A = 0;
  static constexpr int B = D * D;
  static constexpr int C = B + D;
  static constexpr int ETA = C + NP;
  static constexpr int J = ETA + D;
  static constexpr int NF = J + NP;
};

// Element accessor over a strided field-major buffer of T (float, or double
// for the FP64 combination of chunk elements).
template <class T>
struct EViewT {
  T *p;
  int stride;
  GPSS_HD T &operator[](int f) const { return p[(size_t)f * stride]; }
};
using EView = EViewT<float>;

template <class S, class T>
GPSS_HD void set_identity(EViewT<T> e) {
  using L = Elem<S>;
#pragma unroll
  for (int f = 0; f < L::NF; ++f) e[f] = T(0);
#pragma unroll
  for (int i = 0; i < S::D; ++i) e[L::A + i * S::D + i] = T(1);
}

template <class S, class T>
GPSS_HD void copy_elem(EViewT<T> dst, EViewT<T> src) {
#pragma unroll 8
  for (int f = 0; f < Elem<S>::NF; ++f) dst[f] = src[f];
}

// out <- Ei o Ej (Ei earlier), in the arithmetic of T.  out may alias Ej (the
// operands are read into registers field by field before out is written, see
// ordering below).
//
// With WITH_C, field NF of each element is its log-normaliser c: the data of
// the stretch have likelihood exp(c + eta^T x - x^T J x / 2) as a function of
// the state x entering it (c = -(sum log S + gamma + n log 2 pi) / 2 for a
// chunk).  Integrating x' ~ N(A_i x + b_i, C_i) against the later stretch's
// likelihood gives
//   c = c_i + c_j - log det X / 2 + eta_j^T b_i - b_i^T J_j b_i / 2
//       + u^T X^{-1} C_i u / 2,   u = eta_j - J_j b_i,
// so for a series that starts from the prior (A = 0) the combination of all
// its stretches carries the series' log-likelihood in c.
template <class S, class T, bool WITH_C = false>
GPSS_HD void combine(EViewT<T> Ei, EViewT<T> Ej, EViewT<T> out) {
  using L = Elem<S>;
  constexpr int D = S::D;
  // X = I + C_i J_j ; right-hand sides [A_i | C_i | b_i + C_i eta_j]
  T X[D][D], R[D][2 * D + 1];
#pragma unroll
  for (int r = 0; r < D; ++r) {
    T ce = T(0);
#pragma unroll
    for (int k = 0; k < D; ++k) ce += Ei[L::C + S::pk(r, k)] * Ej[L::ETA + k];
    R[r][2 * D] = Ei[L::B + r] + ce;
#pragma unroll
    for (int c = 0; c < D; ++c) {
      T acc = (r == c) ? T(1) : T(0);
#pragma unroll
      for (int k = 0; k < D; ++k) acc += Ei[L::C + S::pk(r, k)] * Ej[L::J + S::pk(k, c)];
      X[r][c] = acc;
      R[r][c] = Ei[L::A + r * D + c];
      R[r][D + c] = Ei[L::C + S::pk(r, c)];
    }
  }
  const T logdet_x = solve_inplace<D, 2 * D + 1, T>(X, R);
  // R = [Y | W | w].  New (eta, J) first: they need b_i, A_i, J_j, eta_j.
  T u[D], eta_n[D];
  T c_n = T(0);
#pragma unroll
  for (int r = 0; r < D; ++r) {
    T jb = T(0);
#pragma unroll
    for (int k = 0; k < D; ++k) jb += Ej[L::J + S::pk(r, k)] * Ei[L::B + k];
    u[r] = Ej[L::ETA + r] - jb;
  }
  if constexpr (WITH_C) {
    T q = T(0);
#pragma unroll
    for (int r = 0; r < D; ++r) {
      const T bi = Ei[L::B + r];
      T wu = T(0), jb = T(0);
#pragma unroll
      for (int k = 0; k < D; ++k) {
        wu += R[r][D + k] * u[k];
        jb += Ej[L::J + S::pk(r, k)] * Ei[L::B + k];
      }
      q += Ej[L::ETA + r] * bi - T(0.5) * bi * jb + T(0.5) * u[r] * wu;
    }
    c_n = Ei[L::NF] + Ej[L::NF] - T(0.5) * logdet_x + q;
  }
#pragma unroll
  for (int r = 0; r < D; ++r) {
    T acc = Ei[L::ETA + r];
#pragma unroll
    for (int k = 0; k < D; ++k) acc += R[k][r] * u[k];
    eta_n[r] = acc;
  }
  // T = J_j A_i ; J = Y^T T + J_i
  T TT[D][D];
#pragma unroll
  for (int r = 0; r < D; ++r)
#pragma unroll
    for (int c = 0; c < D; ++c) {
      T acc = T(0);
#pragma unroll
      for (int k = 0; k < D; ++k) acc += Ej[L::J + S::pk(r, k)] * Ei[L::A + k * D + c];
      TT[r][c] = acc;
    }
  T J_n[S::NP];
#pragma unroll
  for (int r = 0; r < D; ++r)
#pragma unroll
    for (int c = r; c < D; ++c) {
      T a1 = T(0), a2 = T(0);
#pragma unroll
      for (int k = 0; k < D; ++k) {
        a1 += R[k][r] * TT[k][c];
        a2 += R[k][c] * TT[k][r];
      }
      J_n[S::pk(r, c)] = Ei[L::J + S::pk(r, c)] + T(0.5) * (a1 + a2);
    }
  // (A, b, C) with A_j
  T Aj[D][D];
#pragma unroll
  for (int r = 0; r < D; ++r)
#pragma unroll
    for (int c = 0; c < D; ++c) Aj[r][c] = Ej[L::A + r * D + c];
  T b_n[D], A_n[D][D], AW[D][D];
#pragma unroll
  for (int r = 0; r < D; ++r) {
    T acc = Ej[L::B + r];
#pragma unroll
    for (int k = 0; k < D; ++k) acc += Aj[r][k] * R[k][2 * D];
    b_n[r] = acc;
#pragma unroll
    for (int c = 0; c < D; ++c) {
      T a1 = T(0), a2 = T(0);
#pragma unroll
      for (int k = 0; k < D; ++k) {
        a1 += Aj[r][k] * R[k][c];
        a2 += Aj[r][k] * R[k][D + c];
      }
      A_n[r][c] = a1;
      AW[r][c] = a2;
    }
  }
  T C_n[S::NP];
#pragma unroll
  for (int r = 0; r < D; ++r)
#pragma unroll
    for (int c = r; c < D; ++c) {
      T a1 = T(0), a2 = T(0);
#pragma unroll
      for (int k = 0; k < D; ++k) {
        a1 += AW[r][k] * Aj[c][k];
        a2 += AW[c][k] * Aj[r][k];
      }
      C_n[S::pk(r, c)] = Ej[L::C + S::pk(r, c)] + T(0.5) * (a1 + a2);
    }
  // write
#pragma unroll
  for (int r = 0; r < D; ++r) {
#pragma unroll
    for (int c = 0; c < D; ++c) out[L::A + r * D + c] = A_n[r][c];
    out[L::B + r] = b_n[r];
    out[L::ETA + r] = eta_n[r];
  }
#pragma unroll
  for (int i = 0; i < S::NP; ++i) {
    out[L::C + i] = C_n[i];
    out[L::J + i] = J_n[i];
  }
  if constexpr (WITH_C) out[L::NF] = c_n;
}

// Logical index i of a scan of n items -> physical position.
GPSS_HD int phys(int i, int n, int rev) { return rev ? n - 1 - i : i; }

// Combine in time order: with rev_op = 0 the logical order is time order;
// with rev_op = 1 the logical predecessor is later in time.
template <class S, class T>
GPSS_HD void combine_logical(EViewT<T> left, EViewT<T> right, EViewT<T> out, int rev_op) {
  if (rev_op)
    combine<S, T>(right, left, out);
  else
    combine<S, T>(left, right, out);
}

// Element fields of entry idx of a field-major buffer (stride = entries),
// converted to T.
template <class S, class T, class U>
GPSS_HD void load_elem_t(const U *src, size_t stride, size_t idx, T (&A)[S::D][S::D], T *b, T *C,
                         T *eta, T *J) {
  using L = Elem<S>;
  constexpr int D = S::D;
#pragma unroll
  for (int i = 0; i < D; ++i) {
#pragma unroll
    for (int j = 0; j < D; ++j) A[i][j] = T(src[(L::A + i * D + j) * stride + idx]);
    b[i] = T(src[(L::B + i) * stride + idx]);
    eta[i] = T(src[(L::ETA + i) * stride + idx]);
  }
#pragma unroll
  for (int i = 0; i < S::NP; ++i) {
    C[i] = T(src[(L::C + i) * stride + idx]);
    J[i] = T(src[(L::J + i) * stride + idx]);
  }
}

// Filtered state through an element: given the state N(m, P) entering it,
//   m <- A (I + P J)^{-1} (m + P eta) + b,  P <- A (I + P J)^{-1} P A^T + C
// (the combination of a state, an element with A = 0, with the element).
template <class S, class T>
GPSS_HD void state_through(const T (&A)[S::D][S::D], const T *b, const T *C, const T *eta,
                           const T *J, T *m, T *P) {
  constexpr int D = S::D;
  T X[D][D], R[D][D + 1];
#pragma unroll
  for (int i = 0; i < D; ++i) {
    T pe = T(0);
#pragma unroll
    for (int k = 0; k < D; ++k) pe += P[S::pk(i, k)] * eta[k];
    R[i][D] = m[i] + pe;
#pragma unroll
    for (int j = 0; j < D; ++j) {
      T acc = (i == j) ? T(1) : T(0);
#pragma unroll
      for (int k = 0; k < D; ++k) acc += P[S::pk(i, k)] * J[S::pk(k, j)];
      X[i][j] = acc;
      R[i][j] = P[S::pk(i, j)];
    }
  }
  solve_inplace<D, D + 1, T>(X, R);
  T TT[D][D];
#pragma unroll
  for (int i = 0; i < D; ++i) {
    T acc = b[i];
#pragma unroll
    for (int k = 0; k < D; ++k) acc += A[i][k] * R[k][D];
    m[i] = acc;
#pragma unroll
    for (int j = 0; j < D; ++j) {
      T a2 = T(0);
#pragma unroll
      for (int k = 0; k < D; ++k) a2 += A[i][k] * R[k][j];
      TT[i][j] = a2;
    }
  }
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int j = i; j < D; ++j) {
      T acc = C[S::pk(i, j)];
#pragma unroll
      for (int k = 0; k < D; ++k) acc += TT[i][k] * A[j][k];
      P[S::pk(i, j)] = acc;
    }
}

// Information about an element's end state (ie, iJ) carried back to the
// state entering it, plus the element's own information:
//   ie <- A^T (I + iJ C)^{-1} (ie - iJ b) + eta,  iJ <- A^T (I + iJ C)^{-1} iJ A + J.
template <class S, class T>
GPSS_HD void info_through(const T (&A)[S::D][S::D], const T *b, const T *C, const T *eta,
                          const T *J, T *ie, T *iJ) {
  constexpr int D = S::D;
  T X[D][D], R[D][D + 1];
#pragma unroll
  for (int i = 0; i < D; ++i) {
    T jb = T(0);
#pragma unroll
    for (int k = 0; k < D; ++k) jb += iJ[S::pk(i, k)] * b[k];
    R[i][D] = ie[i] - jb;
#pragma unroll
    for (int j = 0; j < D; ++j) {
      T acc = (i == j) ? T(1) : T(0), ja = T(0);
#pragma unroll
      for (int k = 0; k < D; ++k) {
        acc += iJ[S::pk(i, k)] * C[S::pk(k, j)];
        ja += iJ[S::pk(i, k)] * A[k][j];
      }
      X[i][j] = acc;
      R[i][j] = ja;
    }
  }
  solve_inplace<D, D + 1, T>(X, R);
#pragma unroll
  for (int i = 0; i < D; ++i) {
    T acc = eta[i];
#pragma unroll
    for (int k = 0; k < D; ++k) acc += A[k][i] * R[k][D];
    ie[i] = acc;
  }
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int j = i; j < D; ++j) {
      T a1 = T(0), a2 = T(0);
#pragma unroll
      for (int k = 0; k < D; ++k) {
        a1 += A[k][i] * R[k][j];
        a2 += A[k][j] * R[k][i];
      }
      iJ[S::pk(i, j)] = J[S::pk(i, j)] + T(0.5) * (a1 + a2);
    }
}

// Shared memory of the tile kernels: three regions of TL elements
// (working tree, own element, one temporary per thread).
template <class S, int TL, class T>
constexpr size_t tile_smem_bytes() {
  return (size_t)3 * TL * Elem<S>::NF * sizeof(T);
}

template <class S, int TL, class T>
__global__ void __launch_bounds__(TL) k_tile_reduce(const T *__restrict__ src, int n,
                                                    T *__restrict__ dst, int n_tiles,
                                                    int rev_index, int rev_op) {
  using L = Elem<S>;
  extern __shared__ __align__(16) unsigned char sm_raw[];
  T *sm = reinterpret_cast<T *>(sm_raw);
  const int tile = blockIdx.x, tid = threadIdx.x;
  const int i0 = tile * TL;
  const int len = min(TL, n - i0);
  EViewT<T> mine{sm + tid, TL};
  if (tid < len) {
    const T *s = src + phys(i0 + tid, n, rev_index);
    for (int f = 0; f < L::NF; ++f) mine[f] = s[(size_t)f * n];
  }
  __syncthreads();
  for (int s = 1; s < TL; s <<= 1) {
    if ((tid % (2 * s)) == 0 && tid + s < len) {
      EViewT<T> right{sm + tid + s, TL};
      combine_logical<S, T>(mine, right, mine, rev_op);
    }
    __syncthreads();
  }
  if (tid == 0) {
    EViewT<T> out{dst + tile, n_tiles};
    copy_elem<S, T>(out, mine);
  }
}

// Inclusive scan of one tile (logical order) preceded by the inclusive scan
// of earlier tiles, pre[tile - 1] (full elements, logical order, stride
// n_pre; may be null).  Output mode 0: full elements to dst (logical order,
// stride n); mode 3: full elements at the physical position.
template <class S, int TL, class T>
__global__ void __launch_bounds__(TL) k_tile_scan(const T *__restrict__ src, int n,
                                                  const T *__restrict__ pre, int n_pre,
                                                  T *__restrict__ dst, int mode, int rev_index,
                                                  int rev_op) {
  using L = Elem<S>;
  extern __shared__ __align__(16) unsigned char sm_raw[];
  T *sm = reinterpret_cast<T *>(sm_raw);
  const int tile = blockIdx.x, tid = threadIdx.x;
  const int i0 = tile * TL;
  const int len = min(TL, n - i0);
  EViewT<T> mine{sm + tid, TL};
  EViewT<T> own{sm + (size_t)TL * L::NF + tid, TL};
  EViewT<T> tmp{sm + (size_t)2 * TL * L::NF + tid, TL};
  if (tid < len) {
    const T *s = src + phys(i0 + tid, n, rev_index);
    for (int f = 0; f < L::NF; ++f) {
      const T v = s[(size_t)f * n];
      mine[f] = v;
      own[f] = v;
    }
  } else {
    set_identity<S, T>(mine);
    set_identity<S, T>(own);
  }
  __syncthreads();
  // Blelloch up-sweep
  for (int s = 1; s < TL; s <<= 1) {
    const int r = (tid + 1) * 2 * s - 1;
    if (r < TL) {
      EViewT<T> a{sm + r - s, TL}, b{sm + r, TL};
      combine_logical<S, T>(a, b, b, rev_op);
    }
    __syncthreads();
  }
  if (tid == 0) set_identity<S, T>(EViewT<T>{sm + TL - 1, TL});
  __syncthreads();
  // down-sweep: exclusive prefixes
  for (int s = TL / 2; s >= 1; s >>= 1) {
    const int r = (tid + 1) * 2 * s - 1;
    if (r < TL) {
      EViewT<T> a{sm + r - s, TL}, b{sm + r, TL};
      copy_elem<S, T>(tmp, a);  // left subtree total
      copy_elem<S, T>(a, b);    // left child gets the parent's prefix
      combine_logical<S, T>(b, tmp, b, rev_op);
    }
    __syncthreads();
  }
  if (tid >= len) return;
  combine_logical<S, T>(mine, own, own, rev_op);  // inclusive within the tile
  if (pre && tile > 0) {
    for (int f = 0; f < L::NF; ++f) tmp[f] = pre[(size_t)f * n_pre + tile - 1];
    combine_logical<S, T>(tmp, own, own, rev_op);
  }
  const int i = i0 + tid;
  EViewT<T> out{dst + (mode == 3 ? phys(i, n, rev_index) : i), n};
  copy_elem<S, T>(out, own);
}

constexpr int SCAN_T = 64;

// Scratch entries of T needed by scan_elems for n elements.
template <class S>
size_t scan_scratch_count(int n) {
  size_t tot = 0;
  while (n > SCAN_T) {
    n = (n + SCAN_T - 1) / SCAN_T;
    tot += (size_t)2 * Elem<S>::NF * n;
  }
  return tot + 1;
}

// Inclusive scan of n elements (field-major, stride n) -> full elements (mode
// 0: logical order; mode 3: physical order).  Recursion depth is log_T(n).
template <class S, class T>
cudaError_t scan_elems(const T *src, int n, T *dst, int mode, int rev_index, int rev_op,
                       T *scratch, cudaStream_t st) {
  constexpr int TL = SCAN_T;
  const size_t smem = tile_smem_bytes<S, TL, T>();
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_tile_scan<S, TL, T>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_tile_reduce<S, TL, T>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  if (n <= 0) return cudaSuccess;
  if (n <= TL) {
    k_tile_scan<S, TL, T><<<1, TL, smem, st>>>(src, n, nullptr, 0, dst, mode, rev_index, rev_op);
    GPSS_COUNT_LAUNCH();
    return cudaGetLastError();
  }
  const int nt = (n + TL - 1) / TL;
  T *agg = scratch, *aggscan = scratch + (size_t)Elem<S>::NF * nt;
  k_tile_reduce<S, TL, T><<<nt, TL, smem, st>>>(src, n, agg, nt, rev_index, rev_op);
  GPSS_COUNT_LAUNCH();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = scan_elems<S, T>(agg, nt, aggscan, 0, 0, rev_op, aggscan + (size_t)Elem<S>::NF * nt, st);
  if (e != cudaSuccess) return e;
  k_tile_scan<S, TL, T><<<nt, TL, smem, st>>>(src, n, aggscan, nt, dst, mode, rev_index, rev_op);
  GPSS_COUNT_LAUNCH();
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Warp-level combination.  The chunk plan gives every series a multiple of 32
// chunks, so each warp holds 32 consecutive chunks of one series.  Each warp
// scans its 32 elements in shared memory (Kogge-Stone, five steps, warp
// synchronous): inclusive prefixes (forward) and, for the gradient, inclusive
// suffixes (backward), plus the warp's total.  The warp totals -- 32x fewer
// than chunks -- are then scanned by scan_elems (or folded per series), and
// k_join combines the two levels per chunk.  T is the arithmetic of every
// combination (the chunk elements themselves are FP32).
// ---------------------------------------------------------------------------
template <class S, class T>
constexpr size_t warp_scan_smem_bytes(int warps) {
  return (size_t)warps * 2 * 32 * Elem<S>::NF * sizeof(T);
}

template <class S, class T>
__global__ void __launch_bounds__(64) k_warp_scan(const float *__restrict__ ef, int n_vch,
                                                  T *__restrict__ pre_local,
                                                  T *__restrict__ suf_local,
                                                  T *__restrict__ wtot, int want_suffix) {
  using L = Elem<S>;
  extern __shared__ __align__(16) unsigned char sm_raw[];
  T *sm = reinterpret_cast<T *>(sm_raw);
  const int lane = threadIdx.x & 31;
  const int vc = blockIdx.x * blockDim.x + threadIdx.x;
  const int n_w = n_vch >> 5;
  const int w = vc >> 5;
  if (w >= n_w) return;  // whole warps only (n_vch is a multiple of 32)
  T *bufA = sm + (size_t)(threadIdx.x >> 5) * 2 * 32 * L::NF;
  T *bufB = bufA + 32 * L::NF;
  for (int dir = 0; dir < (want_suffix ? 2 : 1); ++dir) {
    for (int f = 0; f < L::NF; ++f) bufA[f * 32 + lane] = T(ef[(size_t)f * n_vch + vc]);
    __syncwarp();
    T *src = bufA, *dst = bufB;
    for (int s = 1; s < 32; s <<= 1) {
      const bool act = dir == 0 ? lane >= s : lane + s < 32;
      if (act) {
        if (dir == 0)
          combine<S, T>(EViewT<T>{src + lane - s, 32}, EViewT<T>{src + lane, 32},
                        EViewT<T>{dst + lane, 32});
        else
          combine<S, T>(EViewT<T>{src + lane, 32}, EViewT<T>{src + lane + s, 32},
                        EViewT<T>{dst + lane, 32});
      } else {
        copy_elem<S, T>(EViewT<T>{dst + lane, 32}, EViewT<T>{src + lane, 32});
      }
      __syncwarp();
      T *t = src;
      src = dst;
      dst = t;
    }
    T *out = dir == 0 ? pre_local : suf_local;
    for (int f = 0; f < L::NF; ++f) out[(size_t)f * n_vch + vc] = src[f * 32 + lane];
    if (dir == 0 && lane == 31)
      for (int f = 0; f < L::NF; ++f) wtot[(size_t)f * n_w + w] = src[f * 32 + 31];
    __syncwarp();
  }
}

// Per chunk: filtered end state = (state entering the warp) o (warp-local
// inclusive prefix); information about the state entering the chunk from it
// and all later chunks of its series = (warp-local inclusive suffix) folded
// with the information from later warps.  wpre / wsuf: inclusive scans of
// the warp totals forward / backward (full elements, stride n_w).
// Records (vector D | packed NP) of T, stride n_vch.
template <class S, class T>
__global__ void __launch_bounds__(128) k_join(int n_vch, int n_chunks,
                                              const uint8_t *__restrict__ ch_flags,
                                              const T *__restrict__ pre_local,
                                              const T *__restrict__ suf_local,
                                              const T *__restrict__ wpre,
                                              const T *__restrict__ wsuf,
                                              T *__restrict__ state_end,
                                              T *__restrict__ info_incl) {
  using L = Elem<S>;
  constexpr int D = S::D;
  const int vc = blockIdx.x * blockDim.x + threadIdx.x;
  if (vc >= n_vch) return;
  const int n_w = n_vch >> 5;
  const int w = vc >> 5, lane = vc & 31;
  const int c0 = (vc - lane) % n_chunks;  // first chunk of this warp
  const bool first_warp = ch_flags[c0] & 1;
  // element of the warp-local prefix
  T A[D][D], b[D], C[S::NP], eta[D], J[S::NP];
  load_elem_t<S, T, T>(pre_local, n_vch, vc, A, b, C, eta, J);
  T m[D], P[S::NP];
  if (first_warp) {
#pragma unroll
    for (int i = 0; i < D; ++i) m[i] = b[i];
#pragma unroll
    for (int i = 0; i < S::NP; ++i) P[i] = C[i];
  } else {
    // state entering the warp: (b, C) of the inclusive warp prefix of w - 1
#pragma unroll
    for (int i = 0; i < D; ++i) m[i] = wpre[(size_t)(L::B + i) * n_w + w - 1];
#pragma unroll
    for (int i = 0; i < S::NP; ++i) P[i] = wpre[(size_t)(L::C + i) * n_w + w - 1];
    state_through<S, T>(A, b, C, eta, J, m, P);
  }
#pragma unroll
  for (int i = 0; i < D; ++i) state_end[(size_t)i * n_vch + vc] = m[i];
#pragma unroll
  for (int i = 0; i < S::NP; ++i) state_end[(size_t)(D + i) * n_vch + vc] = P[i];
  if (!info_incl) return;
  // backward: warp-local inclusive suffix folded with the information from
  // later warps (zero past the end of the series)
  load_elem_t<S, T, T>(suf_local, n_vch, vc, A, b, C, eta, J);
  T ie[D], iJ[S::NP];
  if (w + 1 < n_w) {
#pragma unroll
    for (int i = 0; i < D; ++i) ie[i] = wsuf[(size_t)(L::ETA + i) * n_w + w + 1];
#pragma unroll
    for (int i = 0; i < S::NP; ++i) iJ[i] = wsuf[(size_t)(L::J + i) * n_w + w + 1];
  } else {
#pragma unroll
    for (int i = 0; i < D; ++i) ie[i] = T(0);
#pragma unroll
    for (int i = 0; i < S::NP; ++i) iJ[i] = T(0);
  }
  info_through<S, T>(A, b, C, eta, J, ie, iJ);
#pragma unroll
  for (int i = 0; i < D; ++i) info_incl[(size_t)i * n_vch + vc] = ie[i];
#pragma unroll
  for (int i = 0; i < S::NP; ++i) info_incl[(size_t)(D + i) * n_vch + vc] = iJ[i];
}

// Sequential alternative to the scan of warp totals when every series spans
// only a few warps: one thread per (virtual) series folds its warp totals in
// time order.  Writes, in the field positions k_join reads, the filtered
// state at the end of each warp ((b, C) of wpre) and the information about
// the state entering each warp from it and all later warps of the series
// ((eta, J) of wsuf).
template <class S, class T>
__global__ void __launch_bounds__(64) k_warp_fold(int n_out, int per_series, int n_series,
                                                  int n_chunks,
                                                  const int32_t *__restrict__ ch_first,
                                                  const T *__restrict__ wtot, int n_w,
                                                  T *__restrict__ wpre, T *__restrict__ wsuf,
                                                  int want_info) {
  using L = Elem<S>;
  constexpr int D = S::D;
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n_out) return;
  const int s = per_series ? v : v % n_series;
  const int base = per_series ? 0 : (v / n_series) * n_chunks;
  const int w0 = (base + ch_first[s]) >> 5, w1 = (base + ch_first[s + 1]) >> 5;
  T m[D], P[S::NP];
  for (int w = w0; w < w1; ++w) {
    T A[D][D], b[D], C[S::NP], eta[D], J[S::NP];
    load_elem_t<S, T, T>(wtot, n_w, w, A, b, C, eta, J);
    if (w == w0) {
#pragma unroll
      for (int i = 0; i < D; ++i) m[i] = b[i];
#pragma unroll
      for (int i = 0; i < S::NP; ++i) P[i] = C[i];
    } else {
      state_through<S, T>(A, b, C, eta, J, m, P);
    }
#pragma unroll
    for (int i = 0; i < D; ++i) wpre[(size_t)(L::B + i) * n_w + w] = m[i];
#pragma unroll
    for (int i = 0; i < S::NP; ++i) wpre[(size_t)(L::C + i) * n_w + w] = P[i];
  }
  if (!want_info) return;
  T ie[D], iJ[S::NP];
#pragma unroll
  for (int i = 0; i < D; ++i) ie[i] = T(0);
#pragma unroll
  for (int i = 0; i < S::NP; ++i) iJ[i] = T(0);
  for (int w = w1 - 1; w >= w0; --w) {
    T A[D][D], b[D], C[S::NP], eta[D], J[S::NP];
    load_elem_t<S, T, T>(wtot, n_w, w, A, b, C, eta, J);
    info_through<S, T>(A, b, C, eta, J, ie, iJ);
#pragma unroll
    for (int i = 0; i < D; ++i) wsuf[(size_t)(L::ETA + i) * n_w + w] = ie[i];
#pragma unroll
    for (int i = 0; i < S::NP; ++i) wsuf[(size_t)(L::J + i) * n_w + w] = iJ[i];
  }
}

}  // namespace gpss
