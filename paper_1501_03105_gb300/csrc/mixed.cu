// Mixed-precision IRLS step: FP32 conjugate gradients on the Jacobi-scaled
// system inside an FP64 iterative-refinement loop.
//
// Step 1 (reweighting) and the assembly of L~, b and the diagonal D run in FP64
// as in the FP64 path.  Step 2 solves L~ v = b (Eq. reduced-laplacian-system)
// to the same FP64 criterion as the FP64 path, ||b - L~ x||_2 <= tol ||b||_2
// with the residual computed in FP64, by refinement:
//
//   repeat:  r = b - L~ x                       (FP64, FP64 conductances)
//            stop when ||r|| <= tol ||b||
//            solve A^ d^ = D^-1/2 r roughly      (FP32 CG from d^ = 0)
//            x += D^-1/2 d^                      (FP64)
//
// with A^ = D^-1/2 L~ D^-1/2 (unit diagonal, off-diagonal -g_uv/sqrt(d_u d_v)).
// CG on A^ is Jacobi-preconditioned CG on L~ in exact arithmetic (Section 3.1's
// solver); the scaling removes the diagonal and its inverse from the inner
// loop, so an inner iteration touches the scaled conductances and four FP32
// vectors only (48 bytes per row of a 2-D grid instead of 60), a working set
// small enough to stay in GB300's L2 for million-row systems.
//
// Inner products are accumulated per thread in float-float (error-free product
// by FMA and error-free sum: the compensated dot product of Ogita, Rump and
// Oishi, 2005), reduced across the block in float-float and across blocks in
// FP64, so they carry about twice FP32 precision without using the FP64 pipe
// per row.  Each IRLS step is one CUDA graph: a WHILE node for the refinement
// loop whose body holds the FP64 residual, a nested WHILE node for the FP32 CG
// (three kernels per iteration), and the FP64 update of x.  Both loops have
// device-side caps, so both end.
#include <cuda_runtime.h>

#include <cmath>
#include <cstddef>

#include "ctx.h"

// Minimum resident blocks per SM requested for the FP32 inner kernels
// (register cap = 65536 / (256 * this)); chosen by measurement.
#ifndef PIRMCUT_INNER_MINB
#define PIRMCUT_INNER_MINB 1
#endif
// Unroll factor of the vectorised SpMV's row loop (more loads in flight).
#ifndef PIRMCUT_SPMV_UNROLL
#define PIRMCUT_SPMV_UNROLL 1
#endif
// Two-kernel CG iteration on vectorised DIA grids (1) or the three-kernel one (0).
#ifndef PIRMCUT_FUSED_INNER
#define PIRMCUT_FUSED_INNER 1
#endif
// Minimum resident blocks per SM for the fused SpMV (caps its registers at
// 48); measured on grid2048: 3 -> 33.3 us, 4 -> 31.0, 5 -> 30.2-30.6, 6 -> 32.8
// (spills), unbounded (84 registers) -> 40.8.
#ifndef PIRMCUT_FUSED_MINB
#define PIRMCUT_FUSED_MINB 5
#endif
// Threads per block of the fused SpMV.
#ifndef PIRMCUT_FUSED_THREADS
#define PIRMCUT_FUSED_THREADS 256
#endif
// 1: loads and stores of data that one inner iteration touches once (the
// conductances, the correction d, q in update32_r) carry evict-first cache
// hints, leaving L2 to the vectors the next kernel reads again (q, r, p).
// Measured on grid2048: mixed step 88.3 -> 85.3 ms.
#ifndef PIRMCUT_STREAM_HINTS
#define PIRMCUT_STREAM_HINTS 1
#endif


namespace pirmcut {

namespace {

constexpr int kSpmvUnroll = PIRMCUT_SPMV_UNROLL;

__device__ __forceinline__ int64_t gtid() { return int64_t(blockIdx.x) * blockDim.x + threadIdx.x; }
__device__ __forceinline__ int64_t gstride() { return int64_t(gridDim.x) * blockDim.x; }

// ---------------------------------------------------------------------------
// float-float arithmetic
// ---------------------------------------------------------------------------

struct FF {
  float hi, lo;
};

// acc += a * b with the product's and the sum's rounding errors kept in lo.
// __fmul_rn / __fadd_rn keep the compiler from fusing the error-free steps.
__device__ __forceinline__ void ff_fma(FF& acc, float a, float b) {
  const float p = __fmul_rn(a, b);
  const float pe = fmaf(a, b, -p);  // exact: a*b = p + pe
  const float s = __fadd_rn(acc.hi, p);
  const float bb = __fsub_rn(s, acc.hi);
  const float e = __fadd_rn(__fsub_rn(acc.hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));  // hi + p = s + e
  acc.hi = s;
  acc.lo = __fadd_rn(acc.lo, __fadd_rn(e, pe));
}

__device__ __forceinline__ double ff_value(const FF& a) { return double(a.hi) + double(a.lo); }

// a + b for float-float values (error-free sum of the high parts, renormalised).
__device__ __forceinline__ FF ff_add(FF a, FF b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float bb = __fsub_rn(s, a.hi);
  const float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
  const float lo = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  const float hi = __fadd_rn(s, lo);
  return FF{hi, __fsub_rn(lo, __fsub_rn(hi, s))};
}

// Sum NV float-float values over the grid: warps and the block reduce in
// float-float (FP32 pipe), one double per block goes to the partials, and the
// last block to arrive adds the partials in block order in FP64 (the GB300
// FP64 pipe is 1/64 of FP32, so per-thread FP64 work is kept out of the FP32
// kernels).  Fixed order: bit-identical from run to run.
template <int NV>
__device__ __forceinline__ bool grid_sum_ff(FF (&v)[NV], double* partials, unsigned int* counter,
                                            double (&tot)[NV]) {
  __shared__ float sh[32 * NV], sl[32 * NV];
  __shared__ unsigned int s_last;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int j = 0; j < NV; ++j) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      FF other{__shfl_down_sync(0xffffffffu, v[j].hi, o), __shfl_down_sync(0xffffffffu, v[j].lo, o)};
      v[j] = ff_add(v[j], other);
    }
    if (lane == 0) {
      sh[wid * NV + j] = v[j].hi;
      sl[wid * NV + j] = v[j].lo;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int j = 0; j < NV; ++j) {
      FF acc{sh[j], sl[j]};
      for (int w = 1; w < nw; ++w) acc = ff_add(acc, FF{sh[w * NV + j], sl[w * NV + j]});
      partials[j * gridDim.x + blockIdx.x] = ff_value(acc);
    }
    __threadfence();
    s_last = (atomicAdd(counter, 1u) == gridDim.x - 1) ? 1u : 0u;
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

__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }
// streaming (evict-first) variants when PIRMCUT_STREAM_HINTS is on
__device__ __forceinline__ float4 ld4s(const float* p) {
#if PIRMCUT_STREAM_HINTS
  return __ldcs(reinterpret_cast<const float4*>(p));
#else
  return ld4(p);
#endif
}
__device__ __forceinline__ void st4s(float* p, float4 v) {
#if PIRMCUT_STREAM_HINTS
  __stcs(reinterpret_cast<float4*>(p), v);
#else
  *reinterpret_cast<float4*>(p) = v;
#endif
}
__device__ __forceinline__ void st4(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }

// ---------------------------------------------------------------------------
// assembly: FP64 diagonal, b, D^-1/2, ||b||^2, loop state
// ---------------------------------------------------------------------------

struct MAssemble {
  const double* cs;
  const double* ct;
  const double* x;
  const double* eps_list;
  const StepCounters* C;
  int form;
  int initial;
  double tol2, eta2;
  int max_outer, inner_maxit;
  double* diag64;
  double* b64;
  double* s64;
  float* s32;
  double* partials;
  PcgState* S;
  OuterState* O;
};

__device__ __forceinline__ void massemble_row(const MAssemble& a, int64_t i, double sum, double gs,
                                              double& bb) {
  a.diag64[i] = sum;
  a.b64[i] = gs;
  // the scaling only shapes the inner system (the FP64 residual decides
  // convergence), so an FP32 reciprocal square root serves; the same value
  // scales the matrix, the right-hand side and the correction
  const float si = rsqrtf(float(sum));
  a.s64[i] = double(si);
  a.s32[i] = si;
  bb = fma(gs, gs, bb);
}

__device__ __forceinline__ void massemble_finish(const MAssemble& a, double bb) {
  double v[1] = {bb}, tot[1];
  if (grid_sum<1>(v, a.partials, &a.S->counter[0], tot) && threadIdx.x == 0) {
    OuterState* O = a.O;
    O->bb = tot[0];
    O->rr64 = 0.0;
    O->tol2 = a.tol2;
    O->eta2 = a.eta2;
    O->outer_iters = 0;
    O->max_outer = a.max_outer;
    O->inner_maxit = a.inner_maxit;
    O->total_inner = 0;
    O->outer_stop = 0;
    O->status = isfinite(tot[0]) ? PIRMCUT_OK : PIRMCUT_ENUMERIC;
    PcgState* S = a.S;
    S->iters = 0;
    S->stop_req = 1;
    S->stopped = 1;
    S->status = PIRMCUT_OK;
  }
}

template <int K>
__global__ void __launch_bounds__(kThreads)
k_massemble_dia(DiaDesc d, const double* __restrict__ g, MAssemble a) {
  const int64_t nt = d.nt;
  const double eps = a.initial ? 0.0 : a.eps_list[a.C->eps_idx];
  const double eps2 = eps * eps;
  double bb = 0.0;
  for (int64_t i = gtid(); i < nt; i += gstride()) {
    const double xi = a.x[i];
    double gs = a.cs[i], gt = a.ct[i];
    if (!a.initial) {
      gs = conductance(gs, 1.0 - xi, eps2, a.form);
      gt = conductance(gt, xi, eps2, a.form);
    }
    double sum = gs + gt;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int64_t o = d.off[k];
      if (i + o < nt) sum += g[k * nt + i];
      if (i >= o) sum += g[k * nt + i - o];
    }
    massemble_row(a, i, sum, gs, bb);
  }
  massemble_finish(a, bb);
}

// CSR row kernels: blocks [0, light_blocks) take the rows with at most
// heavy_deg entries, G threads per row; each later block takes one heavy row
// (a power-law hub) with all of its threads.
template <int G>
__global__ void __launch_bounds__(kThreads)
k_massemble_csr(int64_t nt, const int64_t* __restrict__ rp, const double* __restrict__ g,
                MAssemble a, int64_t heavy_deg, const int32_t* __restrict__ heavy,
                int light_blocks) {
  const double eps = a.initial ? 0.0 : a.eps_list[a.C->eps_idx];
  const double eps2 = eps * eps;
  double bb = 0.0;
  if (int(blockIdx.x) >= light_blocks) {
    const int64_t i = heavy[blockIdx.x - light_blocks];
    double v[1] = {0.0};
    for (int64_t e = rp[i] + threadIdx.x; e < rp[i + 1]; e += blockDim.x) v[0] += g[e];
    block_sum<1>(v);
    if (threadIdx.x == 0) {
      const double xi = a.x[i];
      double gs = a.cs[i], gt = a.ct[i];
      if (!a.initial) {
        gs = conductance(gs, 1.0 - xi, eps2, a.form);
        gt = conductance(gt, xi, eps2, a.form);
      }
      massemble_row(a, i, v[0] + gs + gt, gs, bb);
    }
    massemble_finish(a, bb);
    return;
  }
  const int lane = threadIdx.x % G;
  const unsigned mask = group_mask<G>();
  const int64_t ng = int64_t(light_blocks) * blockDim.x / G;
  for (int64_t i = gtid() / G; i < nt; i += ng) {
    if (rp[i + 1] - rp[i] > heavy_deg) continue;  // the group agrees: same row
    double sum = 0.0;
    for (int64_t e = rp[i] + lane; e < rp[i + 1]; e += G) sum += g[e];
    sum = group_sum<G>(sum, mask);
    if (lane == 0) {
      const double xi = a.x[i];
      double gs = a.cs[i], gt = a.ct[i];
      if (!a.initial) {
        gs = conductance(gs, 1.0 - xi, eps2, a.form);
        gt = conductance(gt, xi, eps2, a.form);
      }
      massemble_row(a, i, sum + gs + gt, gs, bb);
    }
  }
  massemble_finish(a, bb);
}

// scaled conductances g_uv d_u^-1/2 d_v^-1/2 in FP32 (g truncated to FP32
// with integer instructions; the scaled system only shapes the inner solve)
template <int K>
__global__ void __launch_bounds__(kThreads)
k_mscale_dia(DiaDesc d, const double* __restrict__ g, const float* __restrict__ s32,
             float* __restrict__ g32) {
  const int64_t nt = d.nt;
  for (int64_t i = gtid(); i < nt; i += gstride()) {
    const float si = s32[i];
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int64_t j = i + d.off[k];
      g32[k * nt + i] = j < nt ? f32_trunc(g[k * nt + i]) * si * s32[j] : 0.0f;
    }
  }
}

// (the product of the two scale factors is formed first, so both directions of
// an edge get the same bits)
template <int G>
__global__ void __launch_bounds__(kThreads)
k_mscale_csr(int64_t nt, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
             const double* __restrict__ g, const float* __restrict__ s32, float* __restrict__ g32,
             int64_t heavy_deg, const int32_t* __restrict__ heavy, int light_blocks) {
  if (int(blockIdx.x) >= light_blocks) {
    const int64_t i = heavy[blockIdx.x - light_blocks];
    const float si = s32[i];
    for (int64_t e = rp[i] + threadIdx.x; e < rp[i + 1]; e += blockDim.x)
      g32[e] = f32_trunc(g[e]) * (si * s32[col[e]]);
    return;
  }
  const int lane = threadIdx.x % G;
  const int64_t ng = int64_t(light_blocks) * blockDim.x / G;
  for (int64_t i = gtid() / G; i < nt; i += ng) {
    if (rp[i + 1] - rp[i] > heavy_deg) continue;  // the group agrees: same row
    const float si = s32[i];
    for (int64_t e = rp[i] + lane; e < rp[i + 1]; e += G) g32[e] = f32_trunc(g[e]) * (si * s32[col[e]]);
  }
}

// ---------------------------------------------------------------------------
// refinement loop head: FP64 residual, convergence test, inner set-up
// ---------------------------------------------------------------------------

struct Resid {
  const double* diag64;
  const double* b64;
  const double* x;
  const float* s32;
  float* r32;
  float* p32;
  float* d32;
  double* partials;
  PcgState* S;
  OuterState* O;
  cudaGraphConditionalHandle h_out, h_in;
  int use_cond;
};

// r = b - L~x in FP64; the scaled FP32 residual D^-1/2 r starts the inner CG.
// ||r||^2 (for the FP64 stopping test) and ||D^-1/2 r||^2 are accumulated from
// the FP32 values (truncated from FP64 with integer instructions) in
// float-float: relative error below 3e-7 in norms used only for stopping
// decisions.
__device__ __forceinline__ void resid_row(const Resid& a, int64_t i, double ax, FF& rr, FF& ss) {
  const float r = f32_trunc(a.b64[i] - ax);  // within 2^-23: an inner right-hand side
  const float rs = a.s32[i] * r;
  a.r32[i] = rs;
  a.p32[i] = rs;
  a.d32[i] = 0.0f;
  ff_fma(rr, r, r);
  ff_fma(ss, rs, rs);
}

__device__ __forceinline__ void resid_finish(const Resid& a, FF rr, FF ss) {
  FF v[2] = {rr, ss};
  double tot[2];
  if (grid_sum_ff<2>(v, a.partials, &a.O->counter[0], tot) && threadIdx.x == 0) {
    OuterState* O = a.O;
    PcgState* S = a.S;
    O->total_inner += S->iters;
    const double rr64 = tot[0];
    O->rr64 = rr64;
    int status = O->status;
    if (S->status != PIRMCUT_OK) status = S->status;
    if (!isfinite(rr64) || !isfinite(tot[1])) status = PIRMCUT_ENUMERIC;
    const bool stop = status != PIRMCUT_OK || rr64 <= O->tol2 * O->bb || O->bb == 0.0 ||
                      O->outer_iters >= O->max_outer || !(tot[1] > 0.0);
    if (stop) {
      O->outer_stop = 1;
      O->status = status;
      S->iters = O->total_inner;
      S->rr = rr64;
      S->bb = O->bb;
      S->status = status;
      S->stop_req = 1;
      S->stopped = 1;
    } else {
      O->outer_iters += 1;
      // inner target: reduce by inner_tol, or just below what the FP64 test needs
      const double need = 0.01 * O->tol2 * O->bb / rr64;
      S->tol2 = need > O->eta2 ? need : O->eta2;
      S->bb = tot[1];
      S->rz = tot[1];
      S->rr = tot[1];
      S->iters = 0;
      S->maxit = O->inner_maxit;
      S->stop_req = 0;
      S->stopped = 0;
      S->status = PIRMCUT_OK;
      S->alpha = 0.0;
      S->beta = 0.0;
    }
    if (a.use_cond) {
      cudaGraphSetConditional(a.h_out, stop ? 0u : 1u);
      cudaGraphSetConditional(a.h_in, stop ? 0u : 1u);
    }
  }
}

template <int K>
__global__ void __launch_bounds__(kThreads)
k_resid_dia(DiaDesc d, const double* __restrict__ g, Resid a) {
  if (a.O->outer_stop) return;
  const int64_t nt = d.nt;
  const double* __restrict__ x = a.x;
  FF rr{0.f, 0.f}, ss{0.f, 0.f};
  for (int64_t i = gtid(); i < nt; i += gstride()) {
    double ax = a.diag64[i] * x[i];
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int64_t o = d.off[k];
      if (i + o < nt) ax = fma(-g[k * nt + i], x[i + o], ax);
      if (i >= o) ax = fma(-g[k * nt + i - o], x[i - o], ax);
    }
    resid_row(a, i, ax, rr, ss);
  }
  resid_finish(a, rr, ss);
}

template <int G>
__global__ void __launch_bounds__(kThreads)
k_resid_csr(int64_t nt, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
            const double* __restrict__ g, Resid a, int64_t heavy_deg,
            const int32_t* __restrict__ heavy, int light_blocks) {
  if (a.O->outer_stop) return;
  FF rr{0.f, 0.f}, ss{0.f, 0.f};
  if (int(blockIdx.x) >= light_blocks) {
    const int64_t i = heavy[blockIdx.x - light_blocks];
    double v[1] = {0.0};
    for (int64_t e = rp[i] + threadIdx.x; e < rp[i + 1]; e += blockDim.x)
      v[0] = fma(-g[e], a.x[col[e]], v[0]);
    block_sum<1>(v);
    if (threadIdx.x == 0) resid_row(a, i, fma(a.diag64[i], a.x[i], v[0]), rr, ss);
    resid_finish(a, rr, ss);
    return;
  }
  const int lane = threadIdx.x % G;
  const unsigned mask = group_mask<G>();
  const int64_t ng = int64_t(light_blocks) * blockDim.x / G;
  for (int64_t i = gtid() / G; i < nt; i += ng) {
    if (rp[i + 1] - rp[i] > heavy_deg) continue;  // the group agrees: same row
    double acc = 0.0;
    for (int64_t e = rp[i] + lane; e < rp[i + 1]; e += G) acc = fma(-g[e], a.x[col[e]], acc);
    acc = group_sum<G>(acc, mask);
    if (lane == 0) resid_row(a, i, fma(a.diag64[i], a.x[i], acc), rr, ss);
  }
  resid_finish(a, rr, ss);
}

// ---------------------------------------------------------------------------
// FP32 inner CG on the scaled system: the three-kernel recurrence of the FP64
// path with z = r (unit diagonal).  (p, q) and ||r||^2 are computed directly
// from the vectors each iteration.  (Forming ||r'||^2 from dot products with q
// in the SpMV pass saves a reduction but drifts and diverges once an FP32
// inner solve works near its precision floor, as the late, ill-conditioned
// IRLS systems make it do.)
// ---------------------------------------------------------------------------

__device__ __forceinline__ void spmv32_finish(FF pq, double* partials, PcgState* S) {
  FF v[1] = {pq};
  double tot[1];
  if (grid_sum_ff<1>(v, partials, &S->counter[1], tot) && threadIdx.x == 0) {
    const double al = S->rz / tot[0];
    S->pq = tot[0];
    if (!(tot[0] > 0.0) || !isfinite(al)) {
      S->alpha = 0.0;
      S->status = PIRMCUT_ENUMERIC;
      S->stop_req = 1;
    } else {
      S->alpha = al;
    }
  }
}

template <int K>
__global__ void __launch_bounds__(kThreads)
k_spmv32_dia(DiaDesc d, const float* __restrict__ g, const float* __restrict__ p,
             float* __restrict__ q, double* partials, PcgState* S) {
  if (S->stop_req) {
    if (blockIdx.x == 0 && threadIdx.x == 0) S->stopped = 1;
    return;
  }
  const int64_t nt = d.nt;
  FF pq{0.f, 0.f};
  for (int64_t i = gtid(); i < nt; i += gstride()) {
    const float pi = p[i];
    float acc = pi;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int64_t o = d.off[k];
      if (i + o < nt) acc = fmaf(-g[k * nt + i], p[i + o], acc);
      if (i >= o) acc = fmaf(-g[k * nt + i - o], p[i - o], acc);
    }
    q[i] = acc;
    ff_fma(pq, pi, acc);
  }
  spmv32_finish(pq, partials, S);
}

// Four consecutive rows per thread with 16-byte loads; for n~ % 4 == 0 and DIA
// offsets that are 1 or multiples of 4 (grids whose widths are multiples of 4).
// For offset 1 the neighbours of rows i..i+3 come from the same float4 plus one
// scalar at each end.
template <int K>
__global__ void __launch_bounds__(kThreads, PIRMCUT_INNER_MINB)
k_spmv32v_dia(DiaDesc d, const float* __restrict__ g, const float* __restrict__ p,
              float* __restrict__ q, double* partials, PcgState* S) {
  if (S->stop_req) {
    if (blockIdx.x == 0 && threadIdx.x == 0) S->stopped = 1;
    return;
  }
  const int64_t nt = d.nt, n4 = nt >> 2;
  FF pq{0.f, 0.f};
#pragma unroll kSpmvUnroll
  for (int64_t t = gtid(); t < n4; t += gstride()) {
    const int64_t i0 = t << 2;
    const float4 p4 = ld4(p + i0);
    float a0 = p4.x, a1 = p4.y, a2 = p4.z, a3 = p4.w;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int64_t o = d.off[k];
      const float* gk = g + k * nt;
      const float4 gu = ld4(gk + i0);  // edges (i, i+o) of rows i0..i0+3; 0 past the end
      if (o == 1) {
        const float pn = (i0 + 4 < nt) ? p[i0 + 4] : 0.f;
        const float gl = (i0 >= 1) ? gk[i0 - 1] : 0.f;
        const float pl = (i0 >= 1) ? p[i0 - 1] : 0.f;
        a0 = fmaf(-gu.x, p4.y, a0);
        a1 = fmaf(-gu.y, p4.z, a1);
        a2 = fmaf(-gu.z, p4.w, a2);
        a3 = fmaf(-gu.w, pn, a3);
        a0 = fmaf(-gl, pl, a0);
        a1 = fmaf(-gu.x, p4.x, a1);
        a2 = fmaf(-gu.y, p4.y, a2);
        a3 = fmaf(-gu.z, p4.z, a3);
      } else {
        if (i0 + o < nt) {
          const float4 pu = ld4(p + i0 + o);
          a0 = fmaf(-gu.x, pu.x, a0);
          a1 = fmaf(-gu.y, pu.y, a1);
          a2 = fmaf(-gu.z, pu.z, a2);
          a3 = fmaf(-gu.w, pu.w, a3);
        }
        if (i0 >= o) {
          const float4 gl = ld4(gk + i0 - o);
          const float4 pl = ld4(p + i0 - o);
          a0 = fmaf(-gl.x, pl.x, a0);
          a1 = fmaf(-gl.y, pl.y, a1);
          a2 = fmaf(-gl.z, pl.z, a2);
          a3 = fmaf(-gl.w, pl.w, a3);
        }
      }
    }
    st4(q + i0, make_float4(a0, a1, a2, a3));
    ff_fma(pq, p4.x, a0);
    ff_fma(pq, p4.y, a1);
    ff_fma(pq, p4.z, a2);
    ff_fma(pq, p4.w, a3);
  }
  spmv32_finish(pq, partials, S);
}

// The vectorised SpMV with the previous iteration's vector updates folded in
// (two kernels per CG iteration instead of three): with beta and the pending
// alpha of the previous iteration,
//   p_new = r + beta p_old     (own rows, and recomputed for the neighbours)
//   d    += alpha p_old        (the update the previous iteration left pending)
//   q     = A^ p_new,  (p_new, q)
// p_old and p_new are two buffers used in turn.  Every value is formed by the
// same FMAs as in the three-kernel recurrence, so the iterates are identical.
// The update of d left pending by the last iteration is applied by k_xupdate.
template <int K>
__global__ void __launch_bounds__(PIRMCUT_FUSED_THREADS, PIRMCUT_FUSED_MINB)
k_spmv32v_fused_dia(DiaDesc d, const float* __restrict__ g, const float* __restrict__ r,
                    const float* __restrict__ pold, float* __restrict__ pnew, float* __restrict__ dv,
                    float* __restrict__ q, double* partials, PcgState* S) {
  if (S->stop_req) {
    if (blockIdx.x == 0 && threadIdx.x == 0) S->stopped = 1;
    return;
  }
  const float alpha = float(S->alpha), beta = float(S->beta);
  const int64_t nt = d.nt, n4 = nt >> 2;
  FF pq{0.f, 0.f};
  for (int64_t t = gtid(); t < n4; t += gstride()) {
    const int64_t i0 = t << 2;
    const float4 po = ld4(pold + i0), r4 = ld4(r + i0), d4 = ld4s(dv + i0);
    const float4 p4 = make_float4(fmaf(beta, po.x, r4.x), fmaf(beta, po.y, r4.y),
                                  fmaf(beta, po.z, r4.z), fmaf(beta, po.w, r4.w));
    st4(pnew + i0, p4);
    st4s(dv + i0, make_float4(fmaf(alpha, po.x, d4.x), fmaf(alpha, po.y, d4.y),
                              fmaf(alpha, po.z, d4.z), fmaf(alpha, po.w, d4.w)));
    float a0 = p4.x, a1 = p4.y, a2 = p4.z, a3 = p4.w;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int64_t o = d.off[k];
      const float* gk = g + k * nt;
      const float4 gu = ld4s(gk + i0);
      if (o == 1) {
        const float pn = (i0 + 4 < nt) ? fmaf(beta, pold[i0 + 4], r[i0 + 4]) : 0.f;
        const float gl = (i0 >= 1) ? gk[i0 - 1] : 0.f;
        const float pl = (i0 >= 1) ? fmaf(beta, pold[i0 - 1], r[i0 - 1]) : 0.f;
        a0 = fmaf(-gu.x, p4.y, a0);
        a1 = fmaf(-gu.y, p4.z, a1);
        a2 = fmaf(-gu.z, p4.w, a2);
        a3 = fmaf(-gu.w, pn, a3);
        a0 = fmaf(-gl, pl, a0);
        a1 = fmaf(-gu.x, p4.x, a1);
        a2 = fmaf(-gu.y, p4.y, a2);
        a3 = fmaf(-gu.z, p4.z, a3);
      } else {
        if (i0 + o < nt) {
          const float4 ou = ld4(pold + i0 + o), ru = ld4(r + i0 + o);
          a0 = fmaf(-gu.x, fmaf(beta, ou.x, ru.x), a0);
          a1 = fmaf(-gu.y, fmaf(beta, ou.y, ru.y), a1);
          a2 = fmaf(-gu.z, fmaf(beta, ou.z, ru.z), a2);
          a3 = fmaf(-gu.w, fmaf(beta, ou.w, ru.w), a3);
        }
        if (i0 >= o) {
          const float4 gl = ld4s(gk + i0 - o);
          const float4 ol = ld4(pold + i0 - o), rl = ld4(r + i0 - o);
          a0 = fmaf(-gl.x, fmaf(beta, ol.x, rl.x), a0);
          a1 = fmaf(-gl.y, fmaf(beta, ol.y, rl.y), a1);
          a2 = fmaf(-gl.z, fmaf(beta, ol.z, rl.z), a2);
          a3 = fmaf(-gl.w, fmaf(beta, ol.w, rl.w), a3);
        }
      }
    }
    st4(q + i0, make_float4(a0, a1, a2, a3));
    ff_fma(pq, p4.x, a0);
    ff_fma(pq, p4.y, a1);
    ff_fma(pq, p4.z, a2);
    ff_fma(pq, p4.w, a3);
  }
  spmv32_finish(pq, partials, S);
}

template <int G>
__global__ void __launch_bounds__(kThreads)
k_spmv32_csr(int64_t nt, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
             const float* __restrict__ g, const float* __restrict__ p, float* __restrict__ q,
             double* partials, PcgState* S, int64_t heavy_deg, const int32_t* __restrict__ heavy,
             int light_blocks) {
  if (S->stop_req) {
    if (blockIdx.x == 0 && threadIdx.x == 0) S->stopped = 1;
    return;
  }
  FF pq{0.f, 0.f};
  if (int(blockIdx.x) >= light_blocks) {
    const int64_t i = heavy[blockIdx.x - light_blocks];
    float acc = 0.f;
    for (int64_t e = rp[i] + threadIdx.x; e < rp[i + 1]; e += blockDim.x)
      acc = fmaf(-g[e], p[col[e]], acc);
    double v[1] = {double(acc)};
    block_sum<1>(v);
    if (threadIdx.x == 0) {
      const float pi = p[i];
      const float qi = float(v[0]) + pi;
      q[i] = qi;
      ff_fma(pq, pi, qi);
    }
    spmv32_finish(pq, partials, S);
    return;
  }
  const int lane = threadIdx.x % G;
  const unsigned mask = group_mask<G>();
  const int64_t ng = int64_t(light_blocks) * blockDim.x / G;
  for (int64_t i = gtid() / G; i < nt; i += ng) {
    if (rp[i + 1] - rp[i] > heavy_deg) continue;  // the group agrees: same row
    float acc = 0.f;
    for (int64_t e = rp[i] + lane; e < rp[i + 1]; e += G) acc = fmaf(-g[e], p[col[e]], acc);
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) acc += __shfl_down_sync(mask, acc, o, G);
    if (lane == 0) {
      const float pi = p[i];
      acc += pi;
      q[i] = acc;
      ff_fma(pq, pi, acc);
    }
  }
  spmv32_finish(pq, partials, S);
}

__device__ __forceinline__ void update32_finish(FF rr, double* partials, PcgState* S,
                                                cudaGraphConditionalHandle h, int end_loop) {
  FF v[1] = {rr};
  double tot[1];
  if (grid_sum_ff<1>(v, partials, &S->counter[2], tot) && threadIdx.x == 0) {
    const int it = S->iters + 1;
    S->iters = it;
    const double beta = tot[0] / S->rz;
    S->beta = beta;
    S->rz = tot[0];
    S->rr = tot[0];
    int stop = (tot[0] <= S->tol2 * S->bb) || it >= S->maxit;
    if (!isfinite(tot[0]) || !isfinite(beta)) {
      stop = 1;
      S->status = PIRMCUT_ENUMERIC;
      S->beta = 0.0;
    }
    S->stop_req = stop;
    if (end_loop && stop) cudaGraphSetConditional(h, 0u);
  }
}

// r -= alpha q; ||r||^2 -> beta and the stop test.  vec selects the float4
// loop (n~ % 4 == 0).  end_loop: this kernel ends the WHILE loop when it
// requests the stop (fused recurrence; otherwise k_update32_xp does).
__global__ void __launch_bounds__(kThreads, 8)
k_update32_r(int64_t nt, int vec, const float* __restrict__ q, float* __restrict__ r,
             double* partials, PcgState* S, cudaGraphConditionalHandle h, int end_loop) {
  if (S->stop_req) {
    // an earlier kernel of this loop body stopped the recurrence
    if (end_loop && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(h, 0u);
    return;
  }
  const float alpha = float(S->alpha);
  FF rr{0.f, 0.f};
  if (vec) {
    for (int64_t t = gtid(); t < (nt >> 2); t += gstride()) {
      const int64_t i0 = t << 2;
      const float4 q4 = ld4s(q + i0), r4 = ld4(r + i0);
      const float4 rn = make_float4(fmaf(-alpha, q4.x, r4.x), fmaf(-alpha, q4.y, r4.y),
                                    fmaf(-alpha, q4.z, r4.z), fmaf(-alpha, q4.w, r4.w));
      st4(r + i0, rn);
      ff_fma(rr, rn.x, rn.x);
      ff_fma(rr, rn.y, rn.y);
      ff_fma(rr, rn.z, rn.z);
      ff_fma(rr, rn.w, rn.w);
    }
  } else {
    for (int64_t i = gtid(); i < nt; i += gstride()) {
      const float ri = fmaf(-alpha, q[i], r[i]);
      r[i] = ri;
      ff_fma(rr, ri, ri);
    }
  }
  update32_finish(rr, partials, S, h, end_loop);
}

// d += alpha p; p = r + beta p.  Ends the inner loop once a stop was requested.
__global__ void __launch_bounds__(kThreads, PIRMCUT_INNER_MINB)
k_update32_xp(int64_t nt, int vec, float* __restrict__ d, float* __restrict__ p,
              const float* __restrict__ r, PcgState* S, cudaGraphConditionalHandle h, int use_cond) {
  if (!S->stopped) {
    const float alpha = float(S->alpha), beta = float(S->beta);
    if (vec) {
      for (int64_t t = gtid(); t < (nt >> 2); t += gstride()) {
        const int64_t i0 = t << 2;
        const float4 p4 = ld4(p + i0), d4 = ld4(d + i0), r4 = ld4(r + i0);
        st4(d + i0, make_float4(fmaf(alpha, p4.x, d4.x), fmaf(alpha, p4.y, d4.y),
                                fmaf(alpha, p4.z, d4.z), fmaf(alpha, p4.w, d4.w)));
        st4(p + i0, make_float4(fmaf(beta, p4.x, r4.x), fmaf(beta, p4.y, r4.y),
                                fmaf(beta, p4.z, r4.z), fmaf(beta, p4.w, r4.w)));
      }
    } else {
      for (int64_t i = gtid(); i < nt; i += gstride()) {
        const float pi = p[i];
        d[i] = fmaf(alpha, pi, d[i]);
        p[i] = fmaf(beta, pi, r[i]);
      }
    }
  }
  if (use_cond && blockIdx.x == 0 && threadIdx.x == 0 && S->stop_req) cudaGraphSetConditional(h, 0u);
}

// x += D^-1/2 d^ (FP64), skipped once the refinement loop has stopped.  With
// the fused recurrence the last iteration's d += alpha p is still pending:
// p_last is pa after an even number of iterations, pb after an odd one.
__global__ void __launch_bounds__(kThreads)
k_xupdate(int64_t nt, double* __restrict__ x, const float* __restrict__ d,
          const double* __restrict__ s64, const OuterState* O, const PcgState* S,
          const float* __restrict__ pa, const float* __restrict__ pb, int fused) {
  if (O->outer_stop) return;
  if (fused) {
    const float alpha = float(S->alpha);
    const float* __restrict__ p = (S->iters & 1) ? pb : pa;
    for (int64_t i = gtid(); i < nt; i += gstride())
      x[i] = fma(s64[i], double(fmaf(alpha, p[i], d[i])), x[i]);
    return;
  }
  for (int64_t i = gtid(); i < nt; i += gstride()) x[i] = fma(s64[i], double(d[i]), x[i]);
}

// ---------------------------------------------------------------------------
// enqueue helpers
// ---------------------------------------------------------------------------

// float4 kernels apply when n~ % 4 == 0 (and, for the DIA SpMV, every offset
// is 1 or a multiple of 4)
bool vector_rows(const Ctx& c) { return (c.nt & 3) == 0; }
bool vector_dia(const Ctx& c) {
  if (c.format != PIRMCUT_FORMAT_DIA || !vector_rows(c)) return false;
  for (int k = 0; k < c.K; ++k)
    if (c.dd.off[k] != 1 && (c.dd.off[k] & 3)) return false;
  return true;
}

int enqueue_massemble(Ctx& c, cudaStream_t st, bool initial) {
  const int grid = row_grid(c);
  MAssemble a;
  a.cs = c.cs;
  a.ct = c.ct;
  a.x = c.x;
  a.eps_list = c.eps_list;
  a.C = c.C;
  a.form = c.opt.reweight_form;
  a.initial = initial ? 1 : 0;
  a.tol2 = c.opt.pcg_tol * c.opt.pcg_tol;
  a.eta2 = c.opt.inner_tol * c.opt.inner_tol;
  a.max_outer = 64;
  a.inner_maxit = c.opt.pcg_max_iter < 2000 ? c.opt.pcg_max_iter : 2000;
  a.diag64 = c.diag;
  a.b64 = c.b64;
  a.s64 = c.s64;
  a.s32 = c.s32;
  a.partials = c.partials;
  a.S = c.S;
  a.O = c.O;
  if (c.format == PIRMCUT_FORMAT_DIA) {
    PIRMCUT_DISPATCH_K(c.K, (k_massemble_dia<KK><<<grid, kThreads, 0, st>>>(c.dd, c.gdia, a)));
    PIRMCUT_DISPATCH_K(c.K, (k_mscale_dia<KK><<<grid, kThreads, 0, st>>>(c.dd, c.gdia, c.s32, c.g32)));
  } else {
    PIRMCUT_DISPATCH_G(c.group, (k_massemble_csr<GG><<<grid + c.n_heavy, kThreads, 0, st>>>(
                                    c.nt, c.rp, c.gval, a, c.heavy_deg, c.heavy, grid)));
    PIRMCUT_DISPATCH_G(c.group, (k_mscale_csr<GG><<<grid + c.n_heavy, kThreads, 0, st>>>(
                                    c.nt, c.rp, c.col, c.gval, c.s32, c.g32, c.heavy_deg, c.heavy,
                                    grid)));
  }
  return 2;
}

int enqueue_resid(Ctx& c, cudaStream_t st, cudaGraphConditionalHandle ho,
                  cudaGraphConditionalHandle hi, int use_cond) {
  const int grid = row_grid(c);
  Resid a;
  a.diag64 = c.diag;
  a.b64 = c.b64;
  a.x = c.x;
  a.s32 = c.s32;
  a.r32 = c.r32;
  a.p32 = c.p32;
  a.d32 = c.d32;
  a.partials = c.partials;
  a.S = c.S;
  a.O = c.O;
  a.h_out = ho;
  a.h_in = hi;
  a.use_cond = use_cond;
  if (c.format == PIRMCUT_FORMAT_DIA) {
    PIRMCUT_DISPATCH_K(c.K, (k_resid_dia<KK><<<grid, kThreads, 0, st>>>(c.dd, c.gdia, a)));
  } else {
    PIRMCUT_DISPATCH_G(c.group, (k_resid_csr<GG><<<grid + c.n_heavy, kThreads, 0, st>>>(
                                    c.nt, c.rp, c.col, c.gval, a, c.heavy_deg, c.heavy, grid)));
  }
  return 1;
}

int enqueue_spmv32(Ctx& c, cudaStream_t st) {
  if (vector_dia(c)) {
    PIRMCUT_DISPATCH_K(c.K, (k_spmv32v_dia<KK><<<grid_for(c.nt / 4), kThreads, 0, st>>>(
                                c.dd, c.g32, c.p32, c.q32, c.partials, c.S)));
  } else if (c.format == PIRMCUT_FORMAT_DIA) {
    PIRMCUT_DISPATCH_K(c.K, (k_spmv32_dia<KK><<<row_grid(c), kThreads, 0, st>>>(
                                c.dd, c.g32, c.p32, c.q32, c.partials, c.S)));
  } else {
    PIRMCUT_DISPATCH_G(c.group, (k_spmv32_csr<GG><<<row_grid(c) + c.n_heavy, kThreads, 0, st>>>(
                                    c.nt, c.rp, c.col, c.g32, c.p32, c.q32, c.partials, c.S,
                                    c.heavy_deg, c.heavy, row_grid(c))));
  }
  return 1;
}

// One launch of the fused SpMV: p_old = (odd ? pb : pa), p_new the other.
int enqueue_fused_spmv32(Ctx& c, cudaStream_t st, bool odd, cudaEvent_t e0 = nullptr,
                         cudaEvent_t e1 = nullptr) {
  if (e0) cudaEventRecord(e0, st);
  const float* pold = odd ? c.p32b : c.p32;
  float* pnew = odd ? c.p32 : c.p32b;
  PIRMCUT_DISPATCH_K(c.K, (k_spmv32v_fused_dia<KK><<<c.fused_grid, PIRMCUT_FUSED_THREADS, 0, st>>>(
                              c.dd, c.g32, c.r32, pold, pnew, c.d32, c.q32, c.partials, c.S)));
  if (e1) cudaEventRecord(e1, st);
  return 1;
}

// The kernels of CG iterations.  Three-kernel recurrence: one iteration
// (spmv, update_r, update_xp).  Fused recurrence (vectorised DIA): two
// iterations (spmv_fused(pa -> pb), update_r, spmv_fused(pb -> pa), update_r),
// so that the body of a graph loop leaves p in its starting buffer; a stop
// requested by the first update_r turns the second pair into no-ops.
// ev, when given, holds one event pair per SpMV launch (two with the fused
// recurrence).
int enqueue_inner_iteration(Ctx& c, cudaStream_t st, cudaGraphConditionalHandle h, int use_cond,
                            cudaEvent_t* ev = nullptr) {
  const int vec = vector_rows(c) ? 1 : 0;
  const int g = vec ? grid_for(c.nt / 4) : grid_for(c.nt);
  if (c.fused_inner) {
    for (int half = 0; half < 2; ++half) {
      enqueue_fused_spmv32(c, st, half == 1, ev ? ev[2 * half] : nullptr,
                           ev ? ev[2 * half + 1] : nullptr);
      k_update32_r<<<g, kThreads, 0, st>>>(c.nt, vec, c.q32, c.r32, c.partials, c.S, h, use_cond);
    }
    return 4;
  }
  if (ev) cudaEventRecord(ev[0], st);
  enqueue_spmv32(c, st);
  if (ev) cudaEventRecord(ev[1], st);
  k_update32_r<<<g, kThreads, 0, st>>>(c.nt, vec, c.q32, c.r32, c.partials, c.S, h, 0);
  k_update32_xp<<<g, kThreads, 0, st>>>(c.nt, vec, c.d32, c.p32, c.r32, c.S, h, use_cond);
  return 3;
}

int enqueue_xupdate(Ctx& c, cudaStream_t st) {
  k_xupdate<<<grid_for(c.nt), kThreads, 0, st>>>(c.nt, c.x, c.d32, c.s64, c.O, c.S, c.p32, c.p32b,
                                                 c.fused_inner ? 1 : 0);
  return 1;
}

// Add a WHILE node after the current capture frontier of st; returns its body graph.
cudaError_t add_while(cudaStream_t st, cudaGraphConditionalHandle h, cudaGraphNode_t* node,
                      cudaGraph_t* body) {
  cudaStreamCaptureStatus cst;
  cudaGraph_t graph = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t ndeps = 0;
  cudaError_t e = cudaStreamGetCaptureInfo(st, &cst, nullptr, &graph, &deps, nullptr, &ndeps);
  if (e != cudaSuccess) return e;
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  e = cudaGraphAddNode(node, graph, deps, nullptr, ndeps, &cp);
  if (e != cudaSuccess) return e;
  *body = cp.conditional.phGraph_out[0];
  return cudaSuccess;
}

}  // namespace

cudaError_t mixed_alloc(Ctx& c) {
  if (c.O) return cudaSuccess;
  const size_t nt = size_t(c.nt);
  const size_t ng = c.format == PIRMCUT_FORMAT_DIA ? size_t(c.K) * nt
                                                    : (c.hg.nnz ? size_t(c.hg.nnz) : 1);
  cudaError_t e = cudaSuccess;
  auto A = [&](void** p, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(p, bytes ? bytes : 1);
  };
  A((void**)&c.g32, sizeof(float) * ng);
  A((void**)&c.s64, sizeof(double) * nt);
  A((void**)&c.s32, sizeof(float) * nt);
  A((void**)&c.r32, sizeof(float) * nt);
  A((void**)&c.p32, sizeof(float) * nt);
  c.fused_inner = PIRMCUT_FUSED_INNER && vector_dia(c);
  if (c.fused_inner) A((void**)&c.p32b, sizeof(float) * nt);
  A((void**)&c.q32, sizeof(float) * nt);
  A((void**)&c.d32, sizeof(float) * nt);
  A((void**)&c.b64, sizeof(double) * nt);
  A((void**)&c.O, sizeof(OuterState));
  if (e == cudaSuccess) e = cudaMemset(c.O, 0, sizeof(OuterState));
  if (e == cudaSuccess && c.fused_inner) {
    // one wave of resident blocks (grid-stride loop over the rest)
    int dev = 0, sms = 0, per_sm = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) {
      PIRMCUT_DISPATCH_K(c.K, (e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                                   &per_sm, k_spmv32v_fused_dia<KK>, PIRMCUT_FUSED_THREADS, 0)));
    }
    if (e == cudaSuccess) {
      const int want = grid_for(c.nt / 4, PIRMCUT_FUSED_THREADS);
      const int wave = (per_sm > 0 ? per_sm : 1) * (sms > 0 ? sms : 1);
      c.fused_grid = want < wave ? want : wave;
    }
  }
  if (e != cudaSuccess) mixed_free(c);
  return e;
}

void mixed_free(Ctx& c) {
  void* ps[] = {c.g32, c.s64, c.s32, c.r32, c.p32, c.p32b, c.q32, c.d32, c.b64, c.O};
  for (void* p : ps)
    if (p) cudaFree(p);
  c.g32 = c.s32 = c.r32 = c.p32 = c.p32b = c.q32 = c.d32 = nullptr;
  c.s64 = c.b64 = nullptr;
  c.O = nullptr;
}

// reweight -> assemble (FP64 diagonal, D^-1/2, scaled FP32 conductances) -> [x = 0] ->
// WHILE_out{ resid64 -> WHILE_in{ spmv32, update32_r, update32_xp } -> x += D^-1/2 d } -> step_end
cudaError_t build_step_graph_mixed(Ctx& c, bool initial, cudaGraphExec_t* out, int* nodes) {
  cudaStream_t st = c.cap_stream;
  int n_nodes = 0;
  cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  cudaGraph_t graph = nullptr;
  cudaStreamCaptureStatus cst;
  cudaGraphConditionalHandle ho{}, hi{};
  cudaGraphNode_t out_node{}, in_node{};
  cudaGraph_t out_body = nullptr, in_body = nullptr;
  cudaStream_t bs = nullptr, is = nullptr;
  e = cudaStreamGetCaptureInfo(st, &cst, nullptr, &graph, nullptr, nullptr, nullptr);
  if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&ho, graph, 1, cudaGraphCondAssignDefault);
  if (e == cudaSuccess) {
    const bool mlp = mlp_active(c, initial);
    e = enqueue_stats_pre(c, st);
    if (mlp) n_nodes += enqueue_mlp_pre(c, st);
    n_nodes += enqueue_reweight(c, st, initial);
    if (mlp) n_nodes += enqueue_mlp_post(c, st);
    n_nodes += enqueue_massemble(c, st, initial);
    if (mlp) n_nodes += enqueue_mlp_start_mixed(c, st);
    if (initial || !c.opt.warm_start) cudaMemsetAsync(c.x, 0, sizeof(double) * c.nt, st);
    if (e == cudaSuccess) e = add_while(st, ho, &out_node, &out_body);
  }
  if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&hi, out_body, 0, cudaGraphCondAssignDefault);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&bs, cudaStreamNonBlocking);
  if (e == cudaSuccess)
    e = cudaStreamBeginCaptureToGraph(bs, out_body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    enqueue_resid(c, bs, ho, hi, 1);
    e = add_while(bs, hi, &in_node, &in_body);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&is, cudaStreamNonBlocking);
    if (e == cudaSuccess)
      e = cudaStreamBeginCaptureToGraph(is, in_body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      enqueue_inner_iteration(c, is, hi, 1);
      cudaGraph_t g2 = nullptr;
      e = cudaStreamEndCapture(is, &g2);
    }
    if (e == cudaSuccess)
      e = cudaStreamUpdateCaptureDependencies(bs, &in_node, nullptr, 1, cudaStreamSetCaptureDependencies);
    if (e == cudaSuccess) enqueue_xupdate(c, bs);
    cudaGraph_t g1 = nullptr;
    cudaError_t e1 = cudaStreamEndCapture(bs, &g1);
    if (e == cudaSuccess) e = e1;
  }
  if (is) cudaStreamDestroy(is);
  if (bs) cudaStreamDestroy(bs);
  if (e == cudaSuccess)
    e = cudaStreamUpdateCaptureDependencies(st, &out_node, nullptr, 1, cudaStreamSetCaptureDependencies);
  if (e == cudaSuccess && mlp_active(c, initial)) n_nodes += enqueue_mlp_train(c, st);
  if (e == cudaSuccess) n_nodes += enqueue_step_end(c, st, initial, c.O);
  cudaGraph_t captured = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(st, &captured);
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess) e = cudaGraphInstantiate(out, captured, 0);
  if (captured) cudaGraphDestroy(captured);
  *nodes = n_nodes;
  return e;
}

cudaError_t launch_spmv32_once(Ctx& c) {
  if (c.fused_inner) enqueue_fused_spmv32(c, c.stream, false);
  else enqueue_spmv32(c, c.stream);
  c.launches += 1;
  return cudaGetLastError();
}

// Host-driven launches of the same mixed step (for profilers).
cudaError_t run_step_stream_mixed(Ctx& c, bool initial, int* flag_host, int64_t* kernels) {
  cudaStream_t st = c.stream;
  cudaGraphConditionalHandle none{};
  const bool mlp = mlp_active(c, initial);
  const cudaError_t ep = enqueue_stats_pre(c, st);
  int64_t k = mlp ? enqueue_mlp_pre(c, st) : 0;
  k += enqueue_reweight(c, st, initial);
  if (mlp) k += enqueue_mlp_post(c, st);
  k += enqueue_massemble(c, st, initial);
  if (mlp) k += enqueue_mlp_start_mixed(c, st);
  if (initial || !c.opt.warm_start) cudaMemsetAsync(c.x, 0, sizeof(double) * c.nt, st);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = ep;
  const size_t off_o = offsetof(OuterState, outer_stop);
  const size_t off_s = offsetof(PcgState, iters);
  PcgProgress* prog = reinterpret_cast<PcgProgress*>(flag_host);
  const int per_call = c.fused_inner ? 2 : 1;  // SpMV launches per enqueue_inner_iteration
  cudaEvent_t* ev = c.opt.time_spmv ? spmv_events(c, 8 * per_call) : nullptr;
  for (int outer = 0; e == cudaSuccess && outer < 70; ++outer) {
    k += enqueue_resid(c, st, none, none, 0);
    e = cudaMemcpyAsync(flag_host, reinterpret_cast<char*>(c.O) + off_o, sizeof(int),
                        cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess || *flag_host) break;
    int iters_before = 0;  // the residual kernel restarted the inner count
    for (int guard = 0; e == cudaSuccess; ++guard) {
      for (int j = 0; j < 8; ++j)
        k += enqueue_inner_iteration(c, st, none, 0, ev ? ev + 2 * per_call * j : nullptr);
      e = cudaMemcpyAsync(prog, reinterpret_cast<char*>(c.S) + off_s, sizeof(PcgProgress),
                          cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) break;
      if (ev) spmv_events_collect(c, 8 * per_call, prog->iters - iters_before);
      iters_before = prog->iters;
      if (prog->stop_req) break;
      if (guard > 2000 / 8 + 2) break;
    }
    k += enqueue_xupdate(c, st);
  }
  if (e == cudaSuccess) {
    if (mlp) k += enqueue_mlp_train(c, st);
    k += enqueue_step_end(c, st, initial, c.O);
    e = cudaGetLastError();
  }
  *kernels = k;
  return e;
}

}  // namespace pirmcut
