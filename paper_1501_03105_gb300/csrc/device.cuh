// Device-side building blocks shared by the kernels of libpirmcut:
// deterministic block reductions (fixed shuffle trees, no float atomics),
// the "last block finishes the reduction" pattern, and the device-resident
// PCG state.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "internal.h"

namespace pirmcut {

constexpr int kThreads = 256;       // block size of the streaming kernels
constexpr int kMaxBlocks = 152 * 8; // cap on grid size (152 SMs x 8 resident blocks)

// Device-resident state of one PCG solve.  Written only by the last block of
// a kernel (or by the host before a solve); read by every block of the next.
struct PcgState {
  double rz;        // (r, z) of the current iterate
  double rr;        // ||r||^2
  double bb;        // ||b||^2
  double pq;        // (p, L~ p)
  double alpha, beta;
  double tol2;      // pcg_tol^2
  double xmin, xmax;
  int iters;        // iterations done in this solve
  int maxit;
  int stop_req;     // set when the recurrence has converged / hit the cap / broke down
  int stopped;      // set by the first kernel of the iteration after stop_req
  int status;       // PIRMCUT_OK or PIRMCUT_ENUMERIC
  int pad;
  unsigned int counter[4];  // last-block counters (one per reduction site)
  // FP64 path: ||r||^2 of the stopping test is summed in FP32 from
  // |r_v| 2^rr_shift unless rr_fp64 (a diagonal outside [2^-80, 2^80])
  int rr_shift;
  int rr_fp64;
};

// Geometry of the DIA storage (upper diagonals only; L~ is symmetric).
struct DiaDesc {
  int64_t nt;
  int64_t off[kMaxDiag];
};

// Tree sums into the first lane of a warp or of a G-lane group (G divides
// 32), in a fixed order.
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

template <int G>
__device__ __forceinline__ double group_sum(double v, unsigned mask) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v += __shfl_down_sync(mask, v, o, G);
  return v;
}

// acc - sum of g[e] p[col[e]] over e = e, e + S, ... < e1, added in that
// order; the column indices and gathers of four entries are issued before
// their FMAs, so that each thread keeps several loads in flight (CSR rows are
// short and their gathers dependent on the index loads).
__device__ __forceinline__ double row_dot_neg(const double* __restrict__ g,
                                              const int32_t* __restrict__ col,
                                              const double* __restrict__ p, int64_t e, int64_t e1,
                                              int S, double acc) {
  for (; e + 3 * S < e1; e += 4 * S) {
    const int32_t c0 = col[e], c1 = col[e + S], c2 = col[e + 2 * S], c3 = col[e + 3 * S];
    const double g0 = g[e], g1 = g[e + S], g2 = g[e + 2 * S], g3 = g[e + 3 * S];
    const double p0 = p[c0], p1 = p[c1], p2 = p[c2], p3 = p[c3];
    acc = fma(-g0, p0, acc);
    acc = fma(-g1, p1, acc);
    acc = fma(-g2, p2, acc);
    acc = fma(-g3, p3, acc);
  }
  for (; e < e1; e += S) acc = fma(-g[e], p[col[e]], acc);
  return acc;
}

// Sum NV doubles over the block; the result is valid in thread 0.
// Fixed tree: the sum is bit-identical from run to run.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV]) {
  __shared__ double sm[32 * NV];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < NV; ++j) v[j] = warp_sum(v[j]);
  if (lane == 0) {
#pragma unroll
    for (int j = 0; j < NV; ++j) sm[wid * NV + j] = v[j];
  }
  __syncthreads();
  if (wid == 0) {
    const int nw = blockDim.x >> 5;
#pragma unroll
    for (int j = 0; j < NV; ++j) v[j] = warp_sum(lane < nw ? sm[lane * NV + j] : 0.0);
  }
  __syncthreads();
}

// Each block contributes v (NV doubles); the last block to arrive sums the
// per-block partials in block order and returns true in all of its threads,
// with the totals in tot (valid in thread 0).  partials holds NV * gridDim.x
// doubles.  No thread ever waits on another block.
template <int NV>
__device__ __forceinline__ bool grid_sum(double (&v)[NV], double* partials,
                                         unsigned int* counter, double (&tot)[NV]) {
  __shared__ unsigned int s_last;
  block_sum<NV>(v);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int j = 0; j < NV; ++j) partials[j * gridDim.x + blockIdx.x] = v[j];
    __threadfence();
    const unsigned int prev = atomicAdd(counter, 1u);
    s_last = (prev == gridDim.x - 1) ? 1u : 0u;
  }
  __syncthreads();
  if (!s_last) return false;
  __threadfence();
  double acc[NV];
#pragma unroll
  for (int j = 0; j < NV; ++j) acc[j] = 0.0;
  for (unsigned int b = threadIdx.x; b < gridDim.x; b += blockDim.x) {
#pragma unroll
    for (int j = 0; j < NV; ++j) acc[j] += __ldcg(partials + j * gridDim.x + b);
  }
  block_sum<NV>(acc);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int j = 0; j < NV; ++j) tot[j] = acc[j];
    *counter = 0u;
  }
  return true;
}

// Conductance of an edge with capacity c and voltage difference d
// (Eq. define-reweight-vector with Eq. reweighted-laplacian).
// form 0: c / sqrt(d^2 + eps^2); form 1: c^2 / sqrt((c d)^2 + eps^2).
__device__ __forceinline__ double conductance(double c, double d, double eps2, int form) {
  if (form == PIRMCUT_REWEIGHT_PAPER) {
    const double cd = c * d;
    return c * c * rsqrt(fma(cd, cd, eps2));
  }
  return c * rsqrt(fma(d, d, eps2));
}

// FP32 value of a double by truncation of its significand, built with
// integer instructions (GB300 runs FP64 <-> FP32 conversions on its narrow
// FP64 pipe); relative error below 2^-23, magnitudes below the FP32 normal
// range give a signed zero, above it (and NaN) an infinity.
__device__ __forceinline__ float f32_trunc(double v) {
  const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(v));
  const unsigned hi = unsigned(b >> 32), lo = unsigned(b);
  const int e = int((hi >> 20) & 0x7FFu) - 896;
  const unsigned m = __funnelshift_r(lo, hi, 29) & 0x7FFFFFu;
  const unsigned sgn = hi & 0x80000000u;
  if (e <= 0) return __uint_as_float(sgn);
  if (e >= 255) return __uint_as_float(sgn | 0x7f800000u);
  return __uint_as_float(sgn | (unsigned(e) << 23) | m);
}

// Compile-time dispatch of the DIA width K (1..8) and the CSR group size G.
#define PIRMCUT_DISPATCH_K(KVAR, CALL) \
  switch (KVAR) {                      \
    case 1: { constexpr int KK = 1; CALL; } break; \
    case 2: { constexpr int KK = 2; CALL; } break; \
    case 3: { constexpr int KK = 3; CALL; } break; \
    case 4: { constexpr int KK = 4; CALL; } break; \
    case 5: { constexpr int KK = 5; CALL; } break; \
    case 6: { constexpr int KK = 6; CALL; } break; \
    case 7: { constexpr int KK = 7; CALL; } break; \
    default: { constexpr int KK = 8; CALL; } break; \
  }

#define PIRMCUT_DISPATCH_G(GVAR, CALL) \
  switch (GVAR) {                      \
    case 1: { constexpr int GG = 1; CALL; } break; \
    case 2: { constexpr int GG = 2; CALL; } break; \
    case 4: { constexpr int GG = 4; CALL; } break; \
    case 8: { constexpr int GG = 8; CALL; } break; \
    case 16: { constexpr int GG = 16; CALL; } break; \
    default: { constexpr int GG = 32; CALL; } break; \
  }

// Lane mask of the G-thread group that owns a row (G divides 32).
template <int G>
__device__ __forceinline__ unsigned group_mask() {
  return (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << ((threadIdx.x & 31) / G * G));
}

inline int grid_for(int64_t n, int threads = kThreads) {
  int64_t b = (n + threads - 1) / threads;
  if (b > kMaxBlocks) b = kMaxBlocks;
  if (b < 1) b = 1;
  return int(b);
}

}  // namespace pirmcut
