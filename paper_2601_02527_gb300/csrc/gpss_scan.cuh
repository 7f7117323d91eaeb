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

// Element accessor over a strided field-major buffer.
struct EView {
  float *p;
  int stride;
  GPSS_HD float &operator[](int f) const { return p[(size_t)f * stride]; }
};

template <class S>
GPSS_HD void set_identity(EView e) {
  using L = Elem<S>;
#pragma unroll
  for (int f = 0; f < L::NF; ++f) e[f] = 0.f;
#pragma unroll
  for (int i = 0; i < S::D; ++i) e[L::A + i * S::D + i] = 1.f;
}

template <class S>
GPSS_HD void copy_elem(EView dst, EView src) {
#pragma unroll 8
  for (int f = 0; f < Elem<S>::NF; ++f) dst[f] = src[f];
}

// out <- Ei o Ej (Ei earlier).  out may alias Ej (the operands are read into
// registers field by field before out is written, see ordering below).
template <class S>
GPSS_HD void combine(EView Ei, EView Ej, EView out) {
  using L = Elem<S>;
  constexpr int D = S::D;
  // X = I + C_i J_j ; right-hand sides [A_i | C_i | b_i + C_i eta_j]
  float X[D][D], R[D][2 * D + 1];
#pragma unroll
  for (int r = 0; r < D; ++r) {
    float ce = 0.f;
#pragma unroll
    for (int k = 0; k < D; ++k) ce += Ei[L::C + S::pk(r, k)] * Ej[L::ETA + k];
    R[r][2 * D] = Ei[L::B + r] + ce;
#pragma unroll
    for (int c = 0; c < D; ++c) {
      float acc = (r == c) ? 1.f : 0.f;
#pragma unroll
      for (int k = 0; k < D; ++k) acc += Ei[L::C + S::pk(r, k)] * Ej[L::J + S::pk(k, c)];
      X[r][c] = acc;
      R[r][c] = Ei[L::A + r * D + c];
      R[r][D + c] = Ei[L::C + S::pk(r, c)];
    }
  }
  solve_inplace<D, 2 * D + 1, float>(X, R);
  // R = [Y | W | w].  New (eta, J) first: they need b_i, A_i, J_j, eta_j.
  float u[D], eta_n[D];
#pragma unroll
  for (int r = 0; r < D; ++r) {
    float jb = 0.f;
#pragma unroll
    for (int k = 0; k < D; ++k) jb += Ej[L::J + S::pk(r, k)] * Ei[L::B + k];
    u[r] = Ej[L::ETA + r] - jb;
  }
#pragma unroll
  for (int r = 0; r < D; ++r) {
    float acc = Ei[L::ETA + r];
#pragma unroll
    for (int k = 0; k < D; ++k) acc += R[k][r] * u[k];
    eta_n[r] = acc;
  }
  // T = J_j A_i ; J = Y^T T + J_i
  float T[D][D];
#pragma unroll
  for (int r = 0; r < D; ++r)
#pragma unroll
    for (int c = 0; c < D; ++c) {
      float acc = 0.f;
#pragma unroll
      for (int k = 0; k < D; ++k) acc += Ej[L::J + S::pk(r, k)] * Ei[L::A + k * D + c];
      T[r][c] = acc;
    }
  float J_n[S::NP];
#pragma unroll
  for (int r = 0; r < D; ++r)
#pragma unroll
    for (int c = r; c < D; ++c) {
      float a1 = 0.f, a2 = 0.f;
#pragma unroll
      for (int k = 0; k < D; ++k) {
        a1 += R[k][r] * T[k][c];
        a2 += R[k][c] * T[k][r];
      }
      J_n[S::pk(r, c)] = Ei[L::J + S::pk(r, c)] + 0.5f * (a1 + a2);
    }
  // (A, b, C) with A_j
  float Aj[D][D];
#pragma unroll
  for (int r = 0; r < D; ++r)
#pragma unroll
    for (int c = 0; c < D; ++c) Aj[r][c] = Ej[L::A + r * D + c];
  float b_n[D], A_n[D][D], AW[D][D];
#pragma unroll
  for (int r = 0; r < D; ++r) {
    float acc = Ej[L::B + r];
#pragma unroll
    for (int k = 0; k < D; ++k) acc += Aj[r][k] * R[k][2 * D];
    b_n[r] = acc;
#pragma unroll
    for (int c = 0; c < D; ++c) {
      float a1 = 0.f, a2 = 0.f;
#pragma unroll
      for (int k = 0; k < D; ++k) {
        a1 += Aj[r][k] * R[k][c];
        a2 += Aj[r][k] * R[k][D + c];
      }
      A_n[r][c] = a1;
      AW[r][c] = a2;
    }
  }
  float C_n[S::NP];
#pragma unroll
  for (int r = 0; r < D; ++r)
#pragma unroll
    for (int c = r; c < D; ++c) {
      float a1 = 0.f, a2 = 0.f;
#pragma unroll
      for (int k = 0; k < D; ++k) {
        a1 += AW[r][k] * Aj[c][k];
        a2 += AW[c][k] * Aj[r][k];
      }
      C_n[S::pk(r, c)] = Ej[L::C + S::pk(r, c)] + 0.5f * (a1 + a2);
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
}

// Logical index i of a scan of n items -> physical position.
GPSS_HD int phys(int i, int n, int rev) { return rev ? n - 1 - i : i; }

// Combine in time order: with rev_op = 0 the logical order is time order;
// with rev_op = 1 the logical predecessor is later in time.
template <class S>
GPSS_HD void combine_logical(EView left, EView right, EView out, int rev_op) {
  if (rev_op)
    combine<S>(right, left, out);
  else
    combine<S>(left, right, out);
}

// Shared memory of the tile kernels: three regions of T elements
// (working tree, own element, one temporary per thread).
template <class S, int T>
constexpr size_t tile_smem_bytes() {
  return (size_t)3 * T * Elem<S>::NF * sizeof(float);
}

template <class S, int T>
__global__ void __launch_bounds__(T) k_tile_reduce(const float *__restrict__ src, int n,
                                                   float *__restrict__ dst, int n_tiles,
                                                   int rev_index, int rev_op) {
  using L = Elem<S>;
  extern __shared__ float sm[];
  const int tile = blockIdx.x, tid = threadIdx.x;
  const int i0 = tile * T;
  const int len = min(T, n - i0);
  EView mine{sm + tid, T};
  if (tid < len) {
    const float *s = src + phys(i0 + tid, n, rev_index);
    for (int f = 0; f < L::NF; ++f) mine[f] = s[(size_t)f * n];
  }
  __syncthreads();
  for (int s = 1; s < T; s <<= 1) {
    if ((tid % (2 * s)) == 0 && tid + s < len) {
      EView right{sm + tid + s, T};
      combine_logical<S>(mine, right, mine, rev_op);
    }
    __syncthreads();
  }
  if (tid == 0) {
    EView out{dst + tile, n_tiles};
    copy_elem<S>(out, mine);
  }
}

// Inclusive scan of one tile (logical order) preceded by the inclusive scan
// of earlier tiles, pre[tile - 1] (full elements, logical order, stride
// n_pre; may be null).  Output mode 0: full elements to dst (logical order,
// stride n); mode 3: full elements at the physical position; mode 1: (b, C)
// as state records at the physical position (stride n); mode 2: (eta, J) as
// information records.
template <class S, int T>
__global__ void __launch_bounds__(T) k_tile_scan(const float *__restrict__ src, int n,
                                                 const float *__restrict__ pre, int n_pre,
                                                 float *__restrict__ dst, int mode, int rev_index,
                                                 int rev_op) {
  using L = Elem<S>;
  constexpr int D = S::D;
  extern __shared__ float sm[];
  const int tile = blockIdx.x, tid = threadIdx.x;
  const int i0 = tile * T;
  const int len = min(T, n - i0);
  EView mine{sm + tid, T};
  EView own{sm + (size_t)T * L::NF + tid, T};
  EView tmp{sm + (size_t)2 * T * L::NF + tid, T};
  if (tid < len) {
    const float *s = src + phys(i0 + tid, n, rev_index);
    for (int f = 0; f < L::NF; ++f) {
      const float v = s[(size_t)f * n];
      mine[f] = v;
      own[f] = v;
    }
  } else {
    set_identity<S>(mine);
    set_identity<S>(own);
  }
  __syncthreads();
  // Blelloch up-sweep
  for (int s = 1; s < T; s <<= 1) {
    const int r = (tid + 1) * 2 * s - 1;
    if (r < T) {
      EView a{sm + r - s, T}, b{sm + r, T};
      combine_logical<S>(a, b, b, rev_op);
    }
    __syncthreads();
  }
  if (tid == 0) set_identity<S>(EView{sm + T - 1, T});
  __syncthreads();
  // down-sweep: exclusive prefixes
  for (int s = T / 2; s >= 1; s >>= 1) {
    const int r = (tid + 1) * 2 * s - 1;
    if (r < T) {
      EView a{sm + r - s, T}, b{sm + r, T};
      copy_elem<S>(tmp, a);  // left subtree total
      copy_elem<S>(a, b);    // left child gets the parent's prefix
      combine_logical<S>(b, tmp, b, rev_op);
    }
    __syncthreads();
  }
  if (tid >= len) return;
  combine_logical<S>(mine, own, own, rev_op);  // inclusive within the tile
  if (pre && tile > 0) {
    for (int f = 0; f < L::NF; ++f) tmp[f] = pre[(size_t)f * n_pre + tile - 1];
    combine_logical<S>(tmp, own, own, rev_op);
  }
  const int i = i0 + tid;
  if (mode == 0) {
    EView out{dst + i, n};
    copy_elem<S>(out, own);
  } else if (mode == 3) {
    EView out{dst + phys(i, n, rev_index), n};
    copy_elem<S>(out, own);
  } else if (mode == 1) {
    const int p = phys(i, n, rev_index);
#pragma unroll
    for (int k = 0; k < D; ++k) dst[(size_t)k * n + p] = own[L::B + k];
#pragma unroll
    for (int k = 0; k < S::NP; ++k) dst[(size_t)(D + k) * n + p] = own[L::C + k];
  } else {
    const int p = phys(i, n, rev_index);
#pragma unroll
    for (int k = 0; k < D; ++k) dst[(size_t)k * n + p] = own[L::ETA + k];
#pragma unroll
    for (int k = 0; k < S::NP; ++k) dst[(size_t)(D + k) * n + p] = own[L::J + k];
  }
}

constexpr int SCAN_T = 64;

// Scratch floats needed by scan_elems for n elements.
template <class S>
size_t scan_scratch_floats(int n) {
  size_t tot = 0;
  while (n > SCAN_T) {
    n = (n + SCAN_T - 1) / SCAN_T;
    tot += (size_t)2 * Elem<S>::NF * n;
  }
  return tot + 1;
}

// Inclusive scan of n elements (field-major, stride n) -> records (mode 1/2)
// or full elements (mode 0).  Recursion depth is log_T(n).
template <class S>
cudaError_t scan_elems(const float *src, int n, float *dst, int mode, int rev_index, int rev_op,
                       float *scratch, cudaStream_t st) {
  constexpr int T = SCAN_T;
  const size_t smem = tile_smem_bytes<S, T>();
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_tile_scan<S, T>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_tile_reduce<S, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  if (n <= 0) return cudaSuccess;
  if (n <= T) {
    k_tile_scan<S, T><<<1, T, smem, st>>>(src, n, nullptr, 0, dst, mode, rev_index, rev_op);
    GPSS_COUNT_LAUNCH();
    return cudaGetLastError();
  }
  const int nt = (n + T - 1) / T;
  float *agg = scratch, *aggscan = scratch + (size_t)Elem<S>::NF * nt;
  k_tile_reduce<S, T><<<nt, T, smem, st>>>(src, n, agg, nt, rev_index, rev_op);
  GPSS_COUNT_LAUNCH();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = scan_elems<S>(agg, nt, aggscan, 0, 0, rev_op, aggscan + (size_t)Elem<S>::NF * nt, st);
  if (e != cudaSuccess) return e;
  k_tile_scan<S, T><<<nt, T, smem, st>>>(src, n, aggscan, nt, dst, mode, rev_index, rev_op);
  GPSS_COUNT_LAUNCH();
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Warp-level combination.  The chunk plan gives every series a multiple of 32
// chunks, so each warp holds 32 consecutive chunks of one series.  Each warp
// scans its 32 elements in shared memory (Kogge-Stone, five steps, warp
// synchronous): inclusive prefixes (forward) and, for the gradient, inclusive
// suffixes (backward), plus the warp's total.  The warp totals -- 32x fewer
// than chunks -- are then scanned by scan_elems, and k_join combines the
// two levels per chunk.
// ---------------------------------------------------------------------------
template <class S>
constexpr size_t warp_scan_smem_bytes(int warps) {
  return (size_t)warps * 2 * 32 * Elem<S>::NF * sizeof(float);
}

template <class S>
__global__ void __launch_bounds__(64) k_warp_scan(const float *__restrict__ ef, int n_vch,
                                                  float *__restrict__ pre_local,
                                                  float *__restrict__ suf_local,
                                                  float *__restrict__ wtot, int want_suffix) {
  using L = Elem<S>;
  extern __shared__ float sm[];
  const int lane = threadIdx.x & 31;
  const int vc = blockIdx.x * blockDim.x + threadIdx.x;
  const int n_w = n_vch >> 5;
  const int w = vc >> 5;
  if (w >= n_w) return;  // whole warps only (n_vch is a multiple of 32)
  float *bufA = sm + (size_t)(threadIdx.x >> 5) * 2 * 32 * L::NF;
  float *bufB = bufA + 32 * L::NF;
  for (int dir = 0; dir < (want_suffix ? 2 : 1); ++dir) {
    for (int f = 0; f < L::NF; ++f) bufA[f * 32 + lane] = ef[(size_t)f * n_vch + vc];
    __syncwarp();
    float *src = bufA, *dst = bufB;
    for (int s = 1; s < 32; s <<= 1) {
      const bool act = dir == 0 ? lane >= s : lane + s < 32;
      if (act) {
        if (dir == 0)
          combine<S>(EView{src + lane - s, 32}, EView{src + lane, 32}, EView{dst + lane, 32});
        else
          combine<S>(EView{src + lane, 32}, EView{src + lane + s, 32}, EView{dst + lane, 32});
      } else {
        copy_elem<S>(EView{dst + lane, 32}, EView{src + lane, 32});
      }
      __syncwarp();
      float *t = src;
      src = dst;
      dst = t;
    }
    float *out = dir == 0 ? pre_local : suf_local;
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
template <class S>
__global__ void __launch_bounds__(128) k_join(int n_vch, int n_chunks,
                                              const uint8_t *__restrict__ ch_flags,
                                              const float *__restrict__ pre_local,
                                              const float *__restrict__ suf_local,
                                              const float *__restrict__ wpre,
                                              const float *__restrict__ wsuf,
                                              float *__restrict__ state_end,
                                              float *__restrict__ info_incl) {
  using L = Elem<S>;
  constexpr int D = S::D;
  const int vc = blockIdx.x * blockDim.x + threadIdx.x;
  if (vc >= n_vch) return;
  const int n_w = n_vch >> 5;
  const int w = vc >> 5, lane = vc & 31;
  const int c0 = (vc - lane) % n_chunks;  // first chunk of this warp
  const bool first_warp = ch_flags[c0] & 1;
  // element of the warp-local prefix
  float A[D][D], b[D], C[S::NP], eta[D], J[S::NP];
#pragma unroll
  for (int i = 0; i < D; ++i) {
#pragma unroll
    for (int j = 0; j < D; ++j) A[i][j] = pre_local[(size_t)(L::A + i * D + j) * n_vch + vc];
    b[i] = pre_local[(size_t)(L::B + i) * n_vch + vc];
    eta[i] = pre_local[(size_t)(L::ETA + i) * n_vch + vc];
  }
#pragma unroll
  for (int i = 0; i < S::NP; ++i) {
    C[i] = pre_local[(size_t)(L::C + i) * n_vch + vc];
    J[i] = pre_local[(size_t)(L::J + i) * n_vch + vc];
  }
  float m[D], P[S::NP];
  if (first_warp) {
#pragma unroll
    for (int i = 0; i < D; ++i) m[i] = b[i];
#pragma unroll
    for (int i = 0; i < S::NP; ++i) P[i] = C[i];
  } else {
    // state entering the warp: (b, C) of the inclusive warp prefix of w - 1
    float mi[D], Pi[S::NP];
#pragma unroll
    for (int i = 0; i < D; ++i) mi[i] = wpre[(size_t)(L::B + i) * n_w + w - 1];
#pragma unroll
    for (int i = 0; i < S::NP; ++i) Pi[i] = wpre[(size_t)(L::C + i) * n_w + w - 1];
    // m = A (I + Pi J)^{-1} (mi + Pi eta) + b ; P = A (I + Pi J)^{-1} Pi A^T + C
    float X[D][D], R[D][D + 1];
#pragma unroll
    for (int i = 0; i < D; ++i) {
      float pe = 0.f;
#pragma unroll
      for (int k = 0; k < D; ++k) pe += Pi[S::pk(i, k)] * eta[k];
      R[i][D] = mi[i] + pe;
#pragma unroll
      for (int j = 0; j < D; ++j) {
        float acc = (i == j) ? 1.f : 0.f;
#pragma unroll
        for (int k = 0; k < D; ++k) acc += Pi[S::pk(i, k)] * J[S::pk(k, j)];
        X[i][j] = acc;
        R[i][j] = Pi[S::pk(i, j)];
      }
    }
    solve_inplace<D, D + 1, float>(X, R);
    float T[D][D];
#pragma unroll
    for (int i = 0; i < D; ++i) {
      float acc = b[i];
#pragma unroll
      for (int k = 0; k < D; ++k) acc += A[i][k] * R[k][D];
      m[i] = acc;
#pragma unroll
      for (int j = 0; j < D; ++j) {
        float a2 = 0.f;
#pragma unroll
        for (int k = 0; k < D; ++k) a2 += A[i][k] * R[k][j];
        T[i][j] = a2;
      }
    }
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
      for (int j = i; j < D; ++j) {
        float acc = C[S::pk(i, j)];
#pragma unroll
        for (int k = 0; k < D; ++k) acc += T[i][k] * A[j][k];
        P[S::pk(i, j)] = acc;
      }
  }
#pragma unroll
  for (int i = 0; i < D; ++i) state_end[(size_t)i * n_vch + vc] = m[i];
#pragma unroll
  for (int i = 0; i < S::NP; ++i) state_end[(size_t)(D + i) * n_vch + vc] = P[i];
  if (!info_incl) return;
  // backward: warp-local inclusive suffix folded with the information from
  // later warps (zero past the end of the series)
#pragma unroll
  for (int i = 0; i < D; ++i) {
#pragma unroll
    for (int j = 0; j < D; ++j) A[i][j] = suf_local[(size_t)(L::A + i * D + j) * n_vch + vc];
    b[i] = suf_local[(size_t)(L::B + i) * n_vch + vc];
    eta[i] = suf_local[(size_t)(L::ETA + i) * n_vch + vc];
  }
#pragma unroll
  for (int i = 0; i < S::NP; ++i) {
    C[i] = suf_local[(size_t)(L::C + i) * n_vch + vc];
    J[i] = suf_local[(size_t)(L::J + i) * n_vch + vc];
  }
  float ie[D], iJ[S::NP];
  if (w + 1 < n_w) {
#pragma unroll
    for (int i = 0; i < D; ++i) ie[i] = wsuf[(size_t)(L::ETA + i) * n_w + w + 1];
#pragma unroll
    for (int i = 0; i < S::NP; ++i) iJ[i] = wsuf[(size_t)(L::J + i) * n_w + w + 1];
  } else {
#pragma unroll
    for (int i = 0; i < D; ++i) ie[i] = 0.f;
#pragma unroll
    for (int i = 0; i < S::NP; ++i) iJ[i] = 0.f;
  }
  // eta' = A^T (I + iJ C)^{-1} (ie - iJ b) + eta ; J' = A^T (I + iJ C)^{-1} iJ A + J
  float X[D][D], R[D][D + 1];
#pragma unroll
  for (int i = 0; i < D; ++i) {
    float jb = 0.f;
#pragma unroll
    for (int k = 0; k < D; ++k) jb += iJ[S::pk(i, k)] * b[k];
    R[i][D] = ie[i] - jb;
#pragma unroll
    for (int j = 0; j < D; ++j) {
      float acc = (i == j) ? 1.f : 0.f, ja = 0.f;
#pragma unroll
      for (int k = 0; k < D; ++k) {
        acc += iJ[S::pk(i, k)] * C[S::pk(k, j)];
        ja += iJ[S::pk(i, k)] * A[k][j];
      }
      X[i][j] = acc;
      R[i][j] = ja;
    }
  }
  solve_inplace<D, D + 1, float>(X, R);
#pragma unroll
  for (int i = 0; i < D; ++i) {
    float acc = eta[i];
#pragma unroll
    for (int k = 0; k < D; ++k) acc += A[k][i] * R[k][D];
    info_incl[(size_t)i * n_vch + vc] = acc;
  }
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int j = i; j < D; ++j) {
      float a1 = 0.f, a2 = 0.f;
#pragma unroll
      for (int k = 0; k < D; ++k) {
        a1 += A[k][i] * R[k][j];
        a2 += A[k][j] * R[k][i];
      }
      info_incl[(size_t)(D + S::pk(i, j)) * n_vch + vc] = J[S::pk(i, j)] + 0.5f * (a1 + a2);
    }
}

// Sequential alternative to the scan of warp totals when every series spans
// only a few warps: one thread per (virtual) series folds its warp totals in
// time order.  Writes, in the field positions k_join reads, the filtered
// state at the end of each warp ((b, C) of wpre) and the information about
// the state entering each warp from it and all later warps of the series
// ((eta, J) of wsuf).
template <class S>
__global__ void __launch_bounds__(64) k_warp_fold(int n_out, int per_series, int n_series,
                                                  int n_chunks,
                                                  const int32_t *__restrict__ ch_first,
                                                  const float *__restrict__ wtot, int n_w,
                                                  float *__restrict__ wpre,
                                                  float *__restrict__ wsuf, int want_info) {
  using L = Elem<S>;
  constexpr int D = S::D;
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n_out) return;
  const int s = per_series ? v : v % n_series;
  const int base = per_series ? 0 : (v / n_series) * n_chunks;
  const int w0 = (base + ch_first[s]) >> 5, w1 = (base + ch_first[s + 1]) >> 5;
  float m[D], P[S::NP];
  for (int w = w0; w < w1; ++w) {
    float A[D][D], b[D], C[S::NP], eta[D], J[S::NP];
#pragma unroll
    for (int i = 0; i < D; ++i) {
#pragma unroll
      for (int j = 0; j < D; ++j) A[i][j] = wtot[(size_t)(L::A + i * D + j) * n_w + w];
      b[i] = wtot[(size_t)(L::B + i) * n_w + w];
      eta[i] = wtot[(size_t)(L::ETA + i) * n_w + w];
    }
#pragma unroll
    for (int i = 0; i < S::NP; ++i) {
      C[i] = wtot[(size_t)(L::C + i) * n_w + w];
      J[i] = wtot[(size_t)(L::J + i) * n_w + w];
    }
    if (w == w0) {
#pragma unroll
      for (int i = 0; i < D; ++i) m[i] = b[i];
#pragma unroll
      for (int i = 0; i < S::NP; ++i) P[i] = C[i];
    } else {
      float X[D][D], R[D][D + 1];
#pragma unroll
      for (int i = 0; i < D; ++i) {
        float pe = 0.f;
#pragma unroll
        for (int k = 0; k < D; ++k) pe += P[S::pk(i, k)] * eta[k];
        R[i][D] = m[i] + pe;
#pragma unroll
        for (int j = 0; j < D; ++j) {
          float acc = (i == j) ? 1.f : 0.f;
#pragma unroll
          for (int k = 0; k < D; ++k) acc += P[S::pk(i, k)] * J[S::pk(k, j)];
          X[i][j] = acc;
          R[i][j] = P[S::pk(i, j)];
        }
      }
      solve_inplace<D, D + 1, float>(X, R);
      float T[D][D];
#pragma unroll
      for (int i = 0; i < D; ++i) {
        float acc = b[i];
#pragma unroll
        for (int k = 0; k < D; ++k) acc += A[i][k] * R[k][D];
        m[i] = acc;
#pragma unroll
        for (int j = 0; j < D; ++j) {
          float a2 = 0.f;
#pragma unroll
          for (int k = 0; k < D; ++k) a2 += A[i][k] * R[k][j];
          T[i][j] = a2;
        }
      }
#pragma unroll
      for (int i = 0; i < D; ++i)
#pragma unroll
        for (int j = i; j < D; ++j) {
          float acc = C[S::pk(i, j)];
#pragma unroll
          for (int k = 0; k < D; ++k) acc += T[i][k] * A[j][k];
          P[S::pk(i, j)] = acc;
        }
    }
#pragma unroll
    for (int i = 0; i < D; ++i) wpre[(size_t)(L::B + i) * n_w + w] = m[i];
#pragma unroll
    for (int i = 0; i < S::NP; ++i) wpre[(size_t)(L::C + i) * n_w + w] = P[i];
  }
  if (!want_info) return;
  float ie[D], iJ[S::NP];
#pragma unroll
  for (int i = 0; i < D; ++i) ie[i] = 0.f;
#pragma unroll
  for (int i = 0; i < S::NP; ++i) iJ[i] = 0.f;
  for (int w = w1 - 1; w >= w0; --w) {
    float A[D][D], b[D], C[S::NP], eta[D], J[S::NP];
#pragma unroll
    for (int i = 0; i < D; ++i) {
#pragma unroll
      for (int j = 0; j < D; ++j) A[i][j] = wtot[(size_t)(L::A + i * D + j) * n_w + w];
      b[i] = wtot[(size_t)(L::B + i) * n_w + w];
      eta[i] = wtot[(size_t)(L::ETA + i) * n_w + w];
    }
#pragma unroll
    for (int i = 0; i < S::NP; ++i) {
      C[i] = wtot[(size_t)(L::C + i) * n_w + w];
      J[i] = wtot[(size_t)(L::J + i) * n_w + w];
    }
    float X[D][D], R[D][D + 1];
#pragma unroll
    for (int i = 0; i < D; ++i) {
      float jb = 0.f;
#pragma unroll
      for (int k = 0; k < D; ++k) jb += iJ[S::pk(i, k)] * b[k];
      R[i][D] = ie[i] - jb;
#pragma unroll
      for (int j = 0; j < D; ++j) {
        float acc = (i == j) ? 1.f : 0.f, ja = 0.f;
#pragma unroll
        for (int k = 0; k < D; ++k) {
          acc += iJ[S::pk(i, k)] * C[S::pk(k, j)];
          ja += iJ[S::pk(i, k)] * A[k][j];
        }
        X[i][j] = acc;
        R[i][j] = ja;
      }
    }
    solve_inplace<D, D + 1, float>(X, R);
    float ne[D], nJ[S::NP];
#pragma unroll
    for (int i = 0; i < D; ++i) {
      float acc = eta[i];
#pragma unroll
      for (int k = 0; k < D; ++k) acc += A[k][i] * R[k][D];
      ne[i] = acc;
    }
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
      for (int j = i; j < D; ++j) {
        float a1 = 0.f, a2 = 0.f;
#pragma unroll
        for (int k = 0; k < D; ++k) {
          a1 += A[k][i] * R[k][j];
          a2 += A[k][j] * R[k][i];
        }
        nJ[S::pk(i, j)] = J[S::pk(i, j)] + 0.5f * (a1 + a2);
      }
#pragma unroll
    for (int i = 0; i < D; ++i) {
      ie[i] = ne[i];
      wsuf[(size_t)(L::ETA + i) * n_w + w] = ne[i];
    }
#pragma unroll
    for (int i = 0; i < S::NP; ++i) {
      iJ[i] = nJ[i];
      wsuf[(size_t)(L::J + i) * n_w + w] = nJ[i];
    }
  }
}

}  // namespace gpss
