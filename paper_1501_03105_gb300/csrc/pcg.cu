// FP64 kernels of one IRLS step on the GPU and the CUDA graph that runs it.
//
// A step is (Section 2.1, Steps 1-2; Section 3.1):
//   reweight   g_e from x^(l-1) for every stored edge  (Eq. define-reweight-vector)
//   assemble   terminal conductances, b_v = g(s,v), the Jacobi diagonal D,
//              r = b - L~ x (Eq. reduced-laplacian-system with x_s = 1,
//              x_t = 0), then the Jacobi-scaled start x^ = D^1/2 x,
//              r^ = D^-1/2 r, p = r^, (r^, r^), ||r||^2, ||b||^2
//   scale      g^_uv = g_uv d_u^-1/2 d_v^-1/2: the matrix A^ = D^-1/2 L~ D^-1/2
//              with unit diagonal
//   PCG loop   a CUDA-graph WHILE node whose body is three kernels:
//                spmv      q = A^ p, (p, q) -> alpha
//                update_r  r^ -= alpha q, (r^, r^), ||D^1/2 r^||^2 -> beta, stop?
//                update_xp x^ += alpha p, p = r^ + beta p; clears the loop
//                          condition once stop is requested
//   step_end   x = D^-1/2 x^, range of x, per-step record.
// CG on A^ from x^ is Jacobi-preconditioned CG on L~ from x (the iterates are
// the same in exact arithmetic; z = D^-1 r becomes r^ itself), with two FP64
// operations per row fewer per iteration -- GB300 issues FP64 at 1/64 of its
// FP32 rate, and these kernels are bound by that pipe.  The stopping test is
// the unpreconditioned ||r|| / ||b|| <= tol with ||r||^2 = sum_v d_v r^_v^2,
// summed in FP32 from integer-built FP32 copies of r^ and d^1/2 (relative
// error below 1e-6: it decides only when to stop).
// Every reduction is a fixed-order tree over fixed per-thread row sets, so
// results are bit-identical from run to run.  Scalars (alpha, beta, the stop
// flag) live in device memory; the host never synchronises inside a solve.
#include <cuda_runtime.h>

#include <cmath>
#include <cstddef>

#include "ctx.h"

// Resident blocks per SM the FP64 PCG-iteration kernels are launched with
// (the grid is capped at 152 times this): fewer, longer-running blocks spend
// less of GB300's FP64 pipe on the per-block reduction trees, more keep more
// loads in flight.  On the 2048x2048 grid (x^(0) + 50 steps) 4, 5, 6, 7 and 8
// blocks gave 151, 141, 137-138, 146 and 148 ms.
#ifndef PIRMCUT_FP64_BLOCKS_PER_SM
#define PIRMCUT_FP64_BLOCKS_PER_SM 6
#endif

namespace pirmcut {

namespace {

constexpr int kFp64MaxBlocks = 152 * PIRMCUT_FP64_BLOCKS_PER_SM;

// Grid of the SpMV: the cap above on DIA (bound by the FP64 pipe); on CSR,
// whose gathers are latency-bound, every resident block.
inline int spmv_grid(const Ctx& c) {
  const int rg = row_grid(c);
  const int cap = c.format == PIRMCUT_FORMAT_DIA ? kFp64MaxBlocks : kMaxBlocks;
  return rg < cap ? rg : cap;
}

__device__ __forceinline__ int64_t gtid() {
  return int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
}
__device__ __forceinline__ int64_t gstride() { return int64_t(gridDim.x) * blockDim.x; }

// ---------------------------------------------------------------------------
// reweighting (Step 1)
// ---------------------------------------------------------------------------

template <int K>
__global__ void __launch_bounds__(kThreads)
k_reweight_dia(DiaDesc d, const double* __restrict__ c, const double* __restrict__ x,
               const double* __restrict__ eps_list, const StepCounters* __restrict__ C,
               int form, double* __restrict__ g) {
  const int64_t nt = d.nt;
  const double eps = eps_list[C->eps_idx];
  const double eps2 = eps * eps;
  for (int64_t i = gtid(); i < nt; i += gstride()) {
    const double xi = x[i];
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int64_t j = i + d.off[k];
      double gg = 0.0;
      if (j < nt) gg = conductance(c[k * nt + i], xi - x[j], eps2, form);
      g[k * nt + i] = gg;
    }
  }
}

// CSR row kernels: blocks [0, light_blocks) take the rows with at most
// heavy_deg entries, G threads per row; each later block takes one of the
// heavy rows (a power-law hub) with all of its threads.
template <int G>
__global__ void __launch_bounds__(kThreads)
k_reweight_csr(int64_t nt, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
               const double* __restrict__ c, const double* __restrict__ x,
               const double* __restrict__ eps_list, const StepCounters* __restrict__ C,
               int form, double* __restrict__ g, int64_t heavy_deg,
               const int32_t* __restrict__ heavy, int light_blocks) {
  const double eps = eps_list[C->eps_idx];
  const double eps2 = eps * eps;
  if (int(blockIdx.x) >= light_blocks) {
    const int64_t i = heavy[blockIdx.x - light_blocks];
    const double xi = x[i];
    for (int64_t e = rp[i] + threadIdx.x; e < rp[i + 1]; e += blockDim.x)
      g[e] = conductance(c[e], xi - x[col[e]], eps2, form);
    return;
  }
  const int lane = threadIdx.x % G;
  const int64_t ng = int64_t(light_blocks) * blockDim.x / G;
  for (int64_t i = gtid() / G; i < nt; i += ng) {
    if (rp[i + 1] - rp[i] > heavy_deg) continue;  // the group agrees: same row
    const double xi = x[i];
    for (int64_t e = rp[i] + lane; e < rp[i + 1]; e += G)
      g[e] = conductance(c[e], xi - x[col[e]], eps2, form);
  }
}

// ---------------------------------------------------------------------------
// assembly of L~, b and the Jacobi preconditioner; initial residual
// ---------------------------------------------------------------------------

struct AssembleArgs {
  const double* cs;
  const double* ct;
  const double* x;   // start vector of the PCG
  const double* xw;  // reweighting point x^(l-1) of the terminal conductances (the start x)
  const double* eps_list;
  const StepCounters* C;
  int form;
  int initial;     // W^(0) = C: conductances are the capacities
  int zero_start;  // PCG starts from v = 0 (residual = b)
  double tol2;
  int maxit;
  double* diag;
  double* rsd;     // d^-1/2
  float* sq32;     // d^1/2 in FP32
  double* xs;      // scaled start D^1/2 x
  double* r;       // scaled residual D^-1/2 r
  double* p;
  double* partials;
  PcgState* S;
  cudaGraphConditionalHandle h;
  int use_cond;    // 1 inside the step graph (set the WHILE condition), 0 for stream launches
};

// Range of d^1/2 for which the FP32 norm of the stopping test is used: with
// |r| 2^rr_shift near 2^20, every FP32 value it forms (r^ 2^rr_shift, d^1/2
// and their product) stays inside the FP32 normal range.
constexpr double kSqrtDiagLo = 0x1p-40, kSqrtDiagHi = 0x1p40;

// |v| 2^sh as a float, built from v's bit pattern with integer instructions
// only (GB300 runs FP64 <-> FP32 conversions on its narrow FP64 pipe).  The
// significand is truncated to 24 bits (relative error below 2^-23);
// magnitudes below the FP32 normal range give 0, above it (and NaN) +inf.
__device__ __forceinline__ float abs_f32_scaled(double v, int sh) {
  const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(v));
  const unsigned hi = unsigned(b >> 32), lo = unsigned(b);
  const int e = int((hi >> 20) & 0x7FFu) - 896 + sh;  // FP32 biased exponent (1023 - 127 = 896)
  const unsigned m = __funnelshift_r(lo, hi, 29) & 0x7FFFFFu;
  if (e <= 0) return 0.0f;
  if (e >= 255) return __int_as_float(0x7f800000);
  return __uint_as_float((unsigned(e) << 23) | m);
}

// Assembly of one row after its diagonal d and residual r are known: the
// scaled quantities, and the row's terms of (r^, r^), ||r||^2, ||b||^2.
__device__ __forceinline__ void assemble_store(const AssembleArgs& a, int64_t i, double d,
                                               double ri, double xi, double bi, double& rz,
                                               double& rr, double& bb, double& nbad) {
  const double si = rsqrt(d);
  const double qi = d * si;
  const double rh = si * ri;
  a.diag[i] = d;
  a.rsd[i] = si;
  a.sq32[i] = abs_f32_scaled(qi, 0);
  a.xs[i] = a.zero_start ? 0.0 : xi * qi;
  a.r[i] = rh;
  a.p[i] = rh;
  rz = fma(rh, rh, rz);
  rr = fma(ri, ri, rr);
  bb = fma(bi, bi, bb);
  if (!(qi >= kSqrtDiagLo && qi <= kSqrtDiagHi)) nbad += 1.0;
}

__device__ __forceinline__ void assemble_finish(const AssembleArgs& a, double rz, double rr,
                                                double bb, double nbad) {
  double v[4] = {rz, rr, bb, nbad}, tot[4];
  if (grid_sum<4>(v, a.partials, &a.S->counter[0], tot) && threadIdx.x == 0) {
    PcgState* S = a.S;
    S->rz = tot[0];
    S->rr = tot[1];
    S->bb = tot[2];
    S->tol2 = a.tol2;
    S->maxit = a.maxit;
    S->iters = 0;
    S->stopped = 0;
    S->status = PIRMCUT_OK;
    S->alpha = 0.0;
    S->beta = 0.0;
    // FP32 stopping norm: scale |r| to about 2^20 at the start
    S->rr_fp64 = tot[3] > 0.0 ? 1 : 0;
    int sh = 0;
    if (tot[1] > 0.0 && isfinite(tot[1])) sh = 20 - ilogb(tot[1]) / 2;
    S->rr_shift = sh < -200 ? -200 : (sh > 200 ? 200 : sh);
    int stop = (tot[1] <= a.tol2 * tot[2]) || a.maxit <= 0 || tot[2] == 0.0;
    if (!isfinite(tot[0]) || !isfinite(tot[1]) || !isfinite(tot[2])) {
      stop = 1;
      S->status = PIRMCUT_ENUMERIC;
    }
    S->stop_req = stop;
    if (a.use_cond) cudaGraphSetConditional(a.h, stop ? 0u : 1u);
  }
}

template <int K>
__global__ void __launch_bounds__(kThreads, 4)
k_assemble_dia(DiaDesc d, const double* __restrict__ g, AssembleArgs a) {
  const int64_t nt = d.nt;
  const double eps = a.initial ? 0.0 : a.eps_list[a.C->eps_idx];
  const double eps2 = eps * eps;
  const double* __restrict__ x = a.x;
  double rz = 0.0, rr = 0.0, bb = 0.0, nbad = 0.0;
  for (int64_t i = gtid(); i < nt; i += gstride()) {
    const double xi = x[i];
    double gs = a.cs[i], gt = a.ct[i];
    if (!a.initial) {
      const double wi = a.xw[i];
      gs = conductance(gs, 1.0 - wi, eps2, a.form);
      gt = conductance(gt, wi, eps2, a.form);
    }
    double sum = gs + gt, ax = 0.0;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int64_t o = d.off[k];
      if (i + o < nt) {
        const double gg = g[k * nt + i];
        sum += gg;
        ax = fma(gg, x[i + o], ax);
      }
      if (i >= o) {
        const double gg = g[k * nt + i - o];
        sum += gg;
        ax = fma(gg, x[i - o], ax);
      }
    }
    const double ri = a.zero_start ? gs : gs - fma(sum, xi, -ax);
    assemble_store(a, i, sum, ri, xi, gs, rz, rr, bb, nbad);
  }
  assemble_finish(a, rz, rr, bb, nbad);
}

// Step 1 and the assembly in one pass (options.fuse_reweight, FP64 DIA
// steps): row i forms the conductances of its upper edges and stores them, as
// k_reweight_dia does, and forms those of its lower edges again (their own
// rows store them) from the same operands in the same order -- the same
// values bit for bit -- then assembles the row as k_assemble_dia does.  Each
// edge's conductance is formed twice (more FP64 work) for one pass fewer
// over the conductances.
template <int K>
__global__ void __launch_bounds__(kThreads, 4)
k_reweight_assemble_dia(DiaDesc d, const double* __restrict__ cap, double* __restrict__ g,
                        AssembleArgs a) {
  const int64_t nt = d.nt;
  const double eps = a.eps_list[a.C->eps_idx];
  const double eps2 = eps * eps;
  const double* __restrict__ x = a.x;
  double rz = 0.0, rr = 0.0, bb = 0.0, nbad = 0.0;
  for (int64_t i = gtid(); i < nt; i += gstride()) {
    const double xi = x[i];
    const double wi = a.xw[i];
    const double gs = conductance(a.cs[i], 1.0 - wi, eps2, a.form);
    const double gt = conductance(a.ct[i], wi, eps2, a.form);
    double sum = gs + gt, ax = 0.0;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int64_t o = d.off[k];
      double gu = 0.0;
      if (i + o < nt) {
        const double xj = x[i + o];
        gu = conductance(cap[k * nt + i], xi - xj, eps2, a.form);
        sum += gu;
        ax = fma(gu, xj, ax);
      }
      g[k * nt + i] = gu;
      if (i >= o) {
        const double xj = x[i - o];
        const double gl = conductance(cap[k * nt + i - o], xj - xi, eps2, a.form);
        sum += gl;
        ax = fma(gl, xj, ax);
      }
    }
    const double ri = a.zero_start ? gs : gs - fma(sum, xi, -ax);
    assemble_store(a, i, sum, ri, xi, gs, rz, rr, bb, nbad);
  }
  assemble_finish(a, rz, rr, bb, nbad);
}

template <int G>
__global__ void __launch_bounds__(kThreads, 4)
k_assemble_csr(int64_t nt, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
               const double* __restrict__ g, AssembleArgs a, int64_t heavy_deg,
               const int32_t* __restrict__ heavy, int light_blocks) {
  const double eps = a.initial ? 0.0 : a.eps_list[a.C->eps_idx];
  const double eps2 = eps * eps;
  const double* __restrict__ x = a.x;
  double rz = 0.0, rr = 0.0, bb = 0.0, nbad = 0.0;
  if (int(blockIdx.x) >= light_blocks) {
    const int64_t i = heavy[blockIdx.x - light_blocks];
    double v[2] = {0.0, 0.0};  // sum of g, (g, x) over the row
    for (int64_t e = rp[i] + threadIdx.x; e < rp[i + 1]; e += blockDim.x) {
      const double gg = g[e];
      v[0] += gg;
      v[1] = fma(gg, x[col[e]], v[1]);
    }
    block_sum<2>(v);
    if (threadIdx.x == 0) {
      const double xi = x[i];
      double gs = a.cs[i], gt = a.ct[i];
      if (!a.initial) {
        const double wi = a.xw[i];
        gs = conductance(gs, 1.0 - wi, eps2, a.form);
        gt = conductance(gt, wi, eps2, a.form);
      }
      const double sum = v[0] + (gs + gt);
      const double ri = a.zero_start ? gs : gs - fma(sum, xi, -v[1]);
      assemble_store(a, i, sum, ri, xi, gs, rz, rr, bb, nbad);
    }
    assemble_finish(a, rz, rr, bb, nbad);
    return;
  }
  const int lane = threadIdx.x % G;
  const unsigned mask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << ((threadIdx.x & 31) / G * G));
  const int64_t ng = int64_t(light_blocks) * blockDim.x / G;
  for (int64_t i = gtid() / G; i < nt; i += ng) {
    if (rp[i + 1] - rp[i] > heavy_deg) continue;  // the group agrees: same row
    double sum = 0.0, ax = 0.0;
    for (int64_t e = rp[i] + lane; e < rp[i + 1]; e += G) {
      const double gg = g[e];
      sum += gg;
      ax = fma(gg, x[col[e]], ax);
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
      sum += __shfl_down_sync(mask, sum, o, G);
      ax += __shfl_down_sync(mask, ax, o, G);
    }
    if (lane == 0) {
      const double xi = x[i];
      double gs = a.cs[i], gt = a.ct[i];
      if (!a.initial) {
        const double wi = a.xw[i];
        gs = conductance(gs, 1.0 - wi, eps2, a.form);
        gt = conductance(gt, wi, eps2, a.form);
      }
      sum += gs + gt;
      const double ri = a.zero_start ? gs : gs - fma(sum, xi, -ax);
      assemble_store(a, i, sum, ri, xi, gs, rz, rr, bb, nbad);
    }
  }
  assemble_finish(a, rz, rr, bb, nbad);
}

// g^_uv = g_uv (d_u^-1/2 d_v^-1/2): the off-diagonal of A^.  The product of
// the two scale factors is formed first, so both directions of an edge get
// the same bits (A^ stays exactly symmetric).
template <int K>
__global__ void __launch_bounds__(kThreads)
k_scale_dia(DiaDesc d, const double* __restrict__ g, const double* __restrict__ rsd,
            double* __restrict__ gh) {
  const int64_t nt = d.nt;
  for (int64_t i = gtid(); i < nt; i += gstride()) {
    const double si = rsd[i];
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int64_t j = i + d.off[k];
      gh[k * nt + i] = j < nt ? g[k * nt + i] * (si * rsd[j]) : 0.0;
    }
  }
}

template <int G>
__global__ void __launch_bounds__(kThreads)
k_scale_csr(int64_t nt, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
            const double* __restrict__ g, const double* __restrict__ rsd,
            double* __restrict__ gh, int64_t heavy_deg, const int32_t* __restrict__ heavy,
            int light_blocks) {
  if (int(blockIdx.x) >= light_blocks) {
    const int64_t i = heavy[blockIdx.x - light_blocks];
    const double si = rsd[i];
    for (int64_t e = rp[i] + threadIdx.x; e < rp[i + 1]; e += blockDim.x) gh[e] = g[e] * (si * rsd[col[e]]);
    return;
  }
  const int lane = threadIdx.x % G;
  const int64_t ng = int64_t(light_blocks) * blockDim.x / G;
  for (int64_t i = gtid() / G; i < nt; i += ng) {
    if (rp[i + 1] - rp[i] > heavy_deg) continue;  // the group agrees: same row
    const double si = rsd[i];
    for (int64_t e = rp[i] + lane; e < rp[i + 1]; e += G) gh[e] = g[e] * (si * rsd[col[e]]);
  }
}

// ---------------------------------------------------------------------------
// PCG iteration
// ---------------------------------------------------------------------------

__device__ __forceinline__ void spmv_finish(double pq, double* partials, PcgState* S) {
  double v[1] = {pq}, tot[1];
  if (grid_sum<1>(v, partials, &S->counter[1], tot) && threadIdx.x == 0) {
    const double a = S->rz / tot[0];
    S->pq = tot[0];
    if (!(tot[0] > 0.0) || !isfinite(a)) {
      S->alpha = 0.0;
      S->status = PIRMCUT_ENUMERIC;
      S->stop_req = 1;
    } else {
      S->alpha = a;
    }
  }
}

// q = A^ p with A^ = I - (scaled conductances), and (p, q)
template <int K>
__global__ void __launch_bounds__(kThreads)
k_spmv_dia(DiaDesc d, const double* __restrict__ g, const double* __restrict__ p,
           double* __restrict__ q, double* partials, PcgState* S) {
  if (S->stop_req) {
    if (blockIdx.x == 0 && threadIdx.x == 0) S->stopped = 1;
    return;
  }
  const int64_t nt = d.nt;
  double pq = 0.0;
  for (int64_t i = gtid(); i < nt; i += gstride()) {
    const double pi = p[i];
    double acc = pi;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int64_t o = d.off[k];
      if (i + o < nt) acc = fma(-g[k * nt + i], p[i + o], acc);
      if (i >= o) acc = fma(-g[k * nt + i - o], p[i - o], acc);
    }
    q[i] = acc;
    pq = fma(pi, acc, pq);
  }
  spmv_finish(pq, partials, S);
}

template <int G>
__global__ void __launch_bounds__(kThreads)
k_spmv_csr(int64_t nt, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
           const double* __restrict__ g, const double* __restrict__ p, double* __restrict__ q,
           double* partials, PcgState* S, int64_t heavy_deg, const int32_t* __restrict__ heavy,
           int light_blocks) {
  if (S->stop_req) {
    if (blockIdx.x == 0 && threadIdx.x == 0) S->stopped = 1;
    return;
  }
  double pq = 0.0;
  if (int(blockIdx.x) >= light_blocks) {
    const int64_t i = heavy[blockIdx.x - light_blocks];
    double v[1] = {0.0};
    for (int64_t e = rp[i] + threadIdx.x; e < rp[i + 1]; e += blockDim.x)
      v[0] = fma(-g[e], p[col[e]], v[0]);
    block_sum<1>(v);
    if (threadIdx.x == 0) {
      const double pi = p[i];
      const double acc = v[0] + pi;
      q[i] = acc;
      pq = pi * acc;
    }
    spmv_finish(pq, partials, S);
    return;
  }
  const int lane = threadIdx.x % G;
  const unsigned mask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << ((threadIdx.x & 31) / G * G));
  const int64_t ng = int64_t(light_blocks) * blockDim.x / G;
  for (int64_t i = gtid() / G; i < nt; i += ng) {
    if (rp[i + 1] - rp[i] > heavy_deg) continue;  // the group agrees: same row
    double acc = 0.0;
    acc = row_dot_neg(g, col, p, rp[i] + lane, rp[i + 1], G, acc);
    acc = group_sum<G>(acc, mask);
    if (lane == 0) {
      const double pi = p[i];
      acc += pi;
      q[i] = acc;
      pq = fma(pi, acc, pq);
    }
  }
  spmv_finish(pq, partials, S);
}

// grid_sum<2> for an FP64 sum a and an FP32 sum b: within a block b takes an
// FP32 tree (its FP64 adds would be a third of the residual update's FP64
// work), the last block adds the block partials of both in FP64.
__device__ __forceinline__ bool grid_sum_df(double a, float b, double* partials,
                                            unsigned int* counter, double (&tot)[2]) {
  __shared__ double sa[32];
  __shared__ float sb[32];
  __shared__ unsigned int s_last;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  a = warp_sum(a);
  b = warp_sum_f(b);
  if (lane == 0) {
    sa[wid] = a;
    sb[wid] = b;
  }
  __syncthreads();
  if (wid == 0) {
    const int nw = blockDim.x >> 5;
    a = warp_sum(lane < nw ? sa[lane] : 0.0);
    b = warp_sum_f(lane < nw ? sb[lane] : 0.0f);
  }
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = a;
    partials[gridDim.x + blockIdx.x] = double(b);
    __threadfence();
    s_last = (atomicAdd(counter, 1u) == gridDim.x - 1) ? 1u : 0u;
  }
  __syncthreads();
  if (!s_last) return false;
  __threadfence();
  double acc[2] = {0.0, 0.0};
  for (unsigned int k = threadIdx.x; k < gridDim.x; k += blockDim.x) {
    acc[0] += __ldcg(partials + k);
    acc[1] += __ldcg(partials + gridDim.x + k);
  }
  block_sum<2>(acc);
  if (threadIdx.x == 0) {
    tot[0] = acc[0];
    tot[1] = acc[1];
    *counter = 0u;
  }
  return true;
}

// r^ -= alpha q; (r^, r^) and ||r||^2 = sum_v d_v r^_v^2 -> beta, stop.  The
// norm is summed in FP32 from |r^_v| 2^rr_shift and d_v^1/2 (both built with
// integer instructions), in FP64 when a diagonal lies outside the FP32-safe
// range.
__global__ void __launch_bounds__(kThreads)
k_update_r(int64_t nt, const double* __restrict__ q, const float* __restrict__ sq32,
           const double* __restrict__ diag, double* __restrict__ r, double* partials,
           PcgState* S) {
  if (S->stop_req) return;
  const double alpha = S->alpha;
  const int sh = S->rr_shift;
  const bool fp64_norm = S->rr_fp64 != 0;
  double rz = 0.0, rr = 0.0;
  if (fp64_norm) {
    for (int64_t i = gtid(); i < nt; i += gstride()) {
      const double ri = fma(-alpha, q[i], r[i]);
      r[i] = ri;
      rz = fma(ri, ri, rz);
      rr = fma(diag[i] * ri, ri, rr);
    }
  }
  float rr32 = 0.0f;
  if (!fp64_norm) {
    for (int64_t i = gtid(); i < nt; i += gstride()) {
      const double ri = fma(-alpha, q[i], r[i]);
      r[i] = ri;
      rz = fma(ri, ri, rz);
      const float ui = sq32[i] * abs_f32_scaled(ri, sh);
      rr32 = fmaf(ui, ui, rr32);
    }
  }
  double tot[2];
  bool last;
  if (fp64_norm) {
    double v[2] = {rz, rr};
    last = grid_sum<2>(v, partials, &S->counter[2], tot);
  } else {
    last = grid_sum_df(rz, rr32, partials, &S->counter[2], tot);
  }
  if (last && threadIdx.x == 0) {
    const int it = S->iters + 1;
    S->iters = it;
    const double beta = tot[0] / S->rz;
    const double rrt = fp64_norm ? tot[1] : ldexp(tot[1], -2 * sh);
    S->beta = beta;
    S->rz = tot[0];
    S->rr = rrt;
    int stop = (rrt <= S->tol2 * S->bb) || it >= S->maxit;
    if (!isfinite(rrt) || !isfinite(beta)) {
      stop = 1;
      S->status = PIRMCUT_ENUMERIC;
      S->beta = 0.0;
    }
    S->stop_req = stop;
  }
}

// x^ += alpha p; p = r^ + beta p.  Ends the loop once a stop was requested
// in this or an earlier kernel.
__global__ void __launch_bounds__(kThreads)
k_update_xp(int64_t nt, double* __restrict__ x, double* __restrict__ p,
            const double* __restrict__ z, PcgState* S, cudaGraphConditionalHandle h,
            int use_cond) {
  if (!S->stopped) {
    const double alpha = S->alpha, beta = S->beta;
    for (int64_t i = gtid(); i < nt; i += gstride()) {
      const double pi = p[i];
      x[i] = fma(alpha, pi, x[i]);
      p[i] = fma(beta, pi, z[i]);
    }
  }
  if (use_cond && blockIdx.x == 0 && threadIdx.x == 0 && S->stop_req) cudaGraphSetConditional(h, 0u);
}

// ---------------------------------------------------------------------------
// end of a step: range of x, record
// ---------------------------------------------------------------------------

__device__ __forceinline__ double warp_min(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_down_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  return v;
}

// xs, when given, is the scaled iterate of the FP64 path: x = rsd * xs.
__global__ void __launch_bounds__(kThreads)
k_step_end(int64_t nt, double* __restrict__ x, const double* __restrict__ xs,
           const double* __restrict__ rsd, PcgState* S, StepCounters* C, StepRec* recs,
           const double* __restrict__ eps_list, int consumes_eps, double* partials,
           const OuterState* O) {
  __shared__ double smn[32], smx[32];
  __shared__ unsigned int s_last;
  const bool zero = S->bb == 0.0;  // b = 0: the solution of L~ v = b is v = 0
  double mn = INFINITY, mx = -INFINITY;
  for (int64_t i = gtid(); i < nt; i += gstride()) {
    double xi;
    if (zero) {
      xi = 0.0;
      x[i] = 0.0;
    } else if (xs) {
      xi = rsd[i] * xs[i];
      x[i] = xi;
    } else {
      xi = x[i];
    }
    mn = fmin(mn, xi);
    mx = fmax(mx, xi);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  mn = warp_min(mn);
  mx = warp_max(mx);
  if (lane == 0) {
    smn[wid] = mn;
    smx[wid] = mx;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
      mn = fmin(mn, smn[w]);
      mx = fmax(mx, smx[w]);
    }
    partials[blockIdx.x] = mn;
    partials[gridDim.x + blockIdx.x] = mx;
    __threadfence();
    s_last = (atomicAdd(&S->counter[3], 1u) == gridDim.x - 1) ? 1u : 0u;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  mn = INFINITY;
  mx = -INFINITY;
  for (unsigned int b = threadIdx.x; b < gridDim.x; b += blockDim.x) {
    mn = fmin(mn, __ldcg(partials + b));
    mx = fmax(mx, __ldcg(partials + gridDim.x + b));
  }
  mn = warp_min(mn);
  mx = warp_max(mx);
  __syncthreads();
  if (lane == 0) {
    smn[wid] = mn;
    smx[wid] = mx;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
    mn = fmin(mn, smn[w]);
    mx = fmax(mx, smx[w]);
  }
  S->counter[3] = 0u;
  S->xmin = mn;
  S->xmax = mx;
  StepRec rec;
  rec.step = C->step;
  rec.iters = S->iters;
  rec.eps = consumes_eps ? eps_list[C->eps_idx] : 0.0;
  rec.rr = S->rr;
  rec.bb = S->bb;
  rec.xmin = mn;
  rec.xmax = mx;
  rec.cut = NAN;
  rec.status = S->status;
  rec.refine = O ? O->outer_iters : 0;
  rec.obj = NAN;
  rec.flow = NAN;
  recs[C->rec_idx] = rec;
  C->rec_idx += 1;
  C->step += 1;
  if (consumes_eps) C->eps_idx += 1;
}

// ---------------------------------------------------------------------------
// per-step objective and flow value (options.step_stats)
// ---------------------------------------------------------------------------

// Term of edge e in S_eps (Eq. l1-min-smooth-version): weighted-l1 form
// c sqrt(d^2 + eps^2), the paper's form sqrt((c d)^2 + eps^2); edges of zero
// capacity are not told apart from absent ones in the packed storage and
// count 0 in both forms.
__device__ __forceinline__ double edge_objective(double c, double d, double eps2, int form) {
  if (form == PIRMCUT_REWEIGHT_PAPER) {
    const double cd = c * d;
    return c > 0.0 ? sqrt(fma(cd, cd, eps2)) : 0.0;
  }
  return c * sqrt(fma(d, d, eps2));
}

struct StatsArgs {
  const double* cs;
  const double* ct;
  const double* x;   // x^(l), after the step
  const double* xw;  // x^(l-1): the point the step's conductances came from
  const double* eps_list;
  const StepCounters* C;
  StepRec* recs;
  double* partials;
  unsigned int* counter;
  double c_st;       // the direct s-t edge (d = 1)
  int form;
  int initial;       // x^(0): g = c and eps = 0
};

// the terminal edges of row i: objective and flow terms (x_s = 1, x_t = 0)
__device__ __forceinline__ void stats_terminals(const StatsArgs& a, int64_t i, double xi,
                                                double eps2, double& obj, double& flow) {
  const double cs = a.cs[i], ct = a.ct[i];
  double gs = cs, gt = ct;
  if (!a.initial) {
    const double wi = a.xw[i];
    gs = conductance(cs, 1.0 - wi, eps2, a.form);
    gt = conductance(ct, wi, eps2, a.form);
  }
  const double ds = 1.0 - xi;
  obj += edge_objective(cs, ds, eps2, a.form) + edge_objective(ct, xi, eps2, a.form);
  flow = fma(gs * ds, ds, flow);
  flow = fma(gt * xi, xi, flow);
}

__device__ __forceinline__ double stats_eps2(const StatsArgs& a) {
  const double eps = a.initial ? 0.0 : a.eps_list[a.C->eps_idx - 1];  // the step end advanced it
  return eps * eps;
}

__device__ __forceinline__ void stats_finish(const StatsArgs& a, double obj, double flow) {
  double v[2] = {obj, flow}, tot[2];
  if (grid_sum<2>(v, a.partials, a.counter, tot) && threadIdx.x == 0) {
    const double eps2 = stats_eps2(a);
    double o = tot[0], f = tot[1];
    if (a.c_st > 0.0) {
      o += edge_objective(a.c_st, 1.0, eps2, a.form);
      f += a.initial ? a.c_st : conductance(a.c_st, 1.0, eps2, a.form);
    }
    StepRec& r = a.recs[a.C->rec_idx - 1];
    r.obj = o;
    r.flow = f;
  }
}

// each undirected edge once: DIA rows own their upper diagonals
template <int K>
__global__ void __launch_bounds__(kThreads)
k_step_stats_dia(DiaDesc d, const double* __restrict__ c, const double* __restrict__ g,
                 StatsArgs a) {
  const int64_t nt = d.nt;
  const double eps2 = stats_eps2(a);
  double obj = 0.0, flow = 0.0;
  for (int64_t i = gtid(); i < nt; i += gstride()) {
    const double xi = a.x[i];
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int64_t j = i + d.off[k];
      if (j < nt) {
        const double dd = xi - a.x[j];
        obj += edge_objective(c[k * nt + i], dd, eps2, a.form);
        flow = fma(g[k * nt + i] * dd, dd, flow);
      }
    }
    stats_terminals(a, i, xi, eps2, obj, flow);
  }
  stats_finish(a, obj, flow);
}

// each undirected edge once: the entry (i, j) with j > i.  Blocks
// [0, light_blocks) take the rows with at most heavy_deg entries, G threads
// per row; each later block takes one heavy row (a hub) with all its threads.
template <int G>
__global__ void __launch_bounds__(kThreads)
k_step_stats_csr(int64_t nt, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                 const double* __restrict__ c, const double* __restrict__ g, StatsArgs a,
                 int64_t heavy_deg, const int32_t* __restrict__ heavy, int light_blocks) {
  const double eps2 = stats_eps2(a);
  double obj = 0.0, flow = 0.0;
  if (int(blockIdx.x) >= light_blocks) {
    const int64_t i = heavy[blockIdx.x - light_blocks];
    const double xi = a.x[i];
    double v[2] = {0.0, 0.0};
    for (int64_t e = rp[i] + threadIdx.x; e < rp[i + 1]; e += blockDim.x) {
      const int32_t j = col[e];
      if (j > i) {
        const double dd = xi - a.x[j];
        v[0] += edge_objective(c[e], dd, eps2, a.form);
        v[1] = fma(g[e] * dd, dd, v[1]);
      }
    }
    block_sum<2>(v);
    if (threadIdx.x == 0) {
      obj = v[0];
      flow = v[1];
      stats_terminals(a, i, xi, eps2, obj, flow);
    }
    stats_finish(a, obj, flow);
    return;
  }
  const int lane = threadIdx.x % G;
  const unsigned mask = group_mask<G>();
  const int64_t ng = int64_t(light_blocks) * blockDim.x / G;
  for (int64_t i = gtid() / G; i < nt; i += ng) {
    if (rp[i + 1] - rp[i] > heavy_deg) continue;  // the group agrees: same row
    const double xi = a.x[i];
    double o = 0.0, f = 0.0;
    for (int64_t e = rp[i] + lane; e < rp[i + 1]; e += G) {
      const int32_t j = col[e];
      if (j > i) {
        const double dd = xi - a.x[j];
        o += edge_objective(c[e], dd, eps2, a.form);
        f = fma(g[e] * dd, dd, f);
      }
    }
    o = group_sum<G>(o, mask);
    f = group_sum<G>(f, mask);
    if (lane == 0) {
      obj += o;
      flow += f;
      stats_terminals(a, i, xi, eps2, obj, flow);
    }
  }
  stats_finish(a, obj, flow);
}

// ---------------------------------------------------------------------------
// learned start of the FP64 path, in the Jacobi-scaled space
// ---------------------------------------------------------------------------
// After the assembly and the scaling at x^(l-1): d^ = D^1/2 d, w = A^ d^ and
// the exact minimiser of the CG energy along d^ (the same as along d in the
// unscaled space: d^T r^ = d^T r, d^T A^ d^ = d^T L~ d),
//   alpha = (d^, r^) / (d^, w),
// then x^ += alpha d^, r^ -= alpha w, p = r^, and the CG state from there.
// No conductance is computed again: the assembly's diagonal and the scaled
// matrix serve.  alpha = 0 when the start already meets the tolerance, or
// when the curvature is not positive and finite.

// d^ = D^1/2 d = d * (diag * diag^-1/2), in place
__global__ void __launch_bounds__(kThreads)
k_ls_prep(int64_t nt, double* __restrict__ dir, const double* __restrict__ diag,
          const double* __restrict__ rsd) {
  for (int64_t i = gtid(); i < nt; i += gstride()) dir[i] *= diag[i] * rsd[i];
}

__device__ __forceinline__ void ls_scaled_finish(double dr, double dw, double* partials,
                                                 const PcgState* S, MlpState* M) {
  double v[2] = {dr, dw}, tot[2];
  if (grid_sum<2>(v, partials, &M->counter, tot) && threadIdx.x == 0) {
    const double a = tot[1] > 0.0 ? tot[0] / tot[1] : 0.0;
    const bool ok = !S->stop_req && S->bb > 0.0 && isfinite(a) && a != 0.0;
    M->alpha = ok ? a : 0.0;
    M->energy_change = ok ? -tot[0] * a : 0.0;
    M->res_plain = S->rr;  // ||b - L~ x^(l-1)||^2 from the assembly
  }
}

// w = A^ d^ into w, (d^, r^) and (d^, w)
template <int K>
__global__ void __launch_bounds__(kThreads)
k_ls_scaled_dia(DiaDesc d, const double* __restrict__ gh, const double* __restrict__ dh,
                const double* __restrict__ rh, double* __restrict__ w, double* partials,
                const PcgState* S, MlpState* M) {
  const int64_t nt = d.nt;
  double dr = 0.0, dw = 0.0;
  for (int64_t i = gtid(); i < nt; i += gstride()) {
    const double di = dh[i];
    double acc = di;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int64_t o = d.off[k];
      if (i + o < nt) acc = fma(-gh[k * nt + i], dh[i + o], acc);
      if (i >= o) acc = fma(-gh[k * nt + i - o], dh[i - o], acc);
    }
    w[i] = acc;
    dr = fma(di, rh[i], dr);
    dw = fma(di, acc, dw);
  }
  ls_scaled_finish(dr, dw, partials, S, M);
}

template <int G>
__global__ void __launch_bounds__(kThreads)
k_ls_scaled_csr(int64_t nt, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                const double* __restrict__ gh, const double* __restrict__ dh,
                const double* __restrict__ rh, double* __restrict__ w, double* partials,
                const PcgState* S, MlpState* M, int64_t heavy_deg,
                const int32_t* __restrict__ heavy, int light_blocks) {
  double dr = 0.0, dw = 0.0;
  if (int(blockIdx.x) >= light_blocks) {
    const int64_t i = heavy[blockIdx.x - light_blocks];
    double v[1] = {0.0};
    for (int64_t e = rp[i] + threadIdx.x; e < rp[i + 1]; e += blockDim.x)
      v[0] = fma(-gh[e], dh[col[e]], v[0]);
    block_sum<1>(v);
    if (threadIdx.x == 0) {
      const double di = dh[i], acc = v[0] + di;
      w[i] = acc;
      dr = di * rh[i];
      dw = di * acc;
    }
    ls_scaled_finish(dr, dw, partials, S, M);
    return;
  }
  const int lane = threadIdx.x % G;
  const unsigned mask = group_mask<G>();
  const int64_t ng = int64_t(light_blocks) * blockDim.x / G;
  for (int64_t i = gtid() / G; i < nt; i += ng) {
    if (rp[i + 1] - rp[i] > heavy_deg) continue;  // the group agrees: same row
    double acc = row_dot_neg(gh, col, dh, rp[i] + lane, rp[i + 1], G, 0.0);
    acc = group_sum<G>(acc, mask);
    if (lane == 0) {
      const double di = dh[i];
      acc += di;
      w[i] = acc;
      dr = fma(di, rh[i], dr);
      dw = fma(di, acc, dw);
    }
  }
  ls_scaled_finish(dr, dw, partials, S, M);
}

// x^ += alpha d^; r^ -= alpha w; p = r^; the CG state from the moved start
// (the same sums and stopping test as the assembly).  Counts the step in M.
__global__ void __launch_bounds__(kThreads)
k_ls_commit(int64_t nt, const double* __restrict__ dh, const double* __restrict__ w,
            const float* __restrict__ sq32, const double* __restrict__ diag,
            double* __restrict__ xs, double* __restrict__ rh, double* __restrict__ p,
            double* partials, PcgState* S, MlpState* M, cudaGraphConditionalHandle h,
            int use_cond) {
  const double a = M->alpha;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    M->steps += 1;
    M->used += a != 0.0 ? 1 : 0;
    M->sum_alpha += a;
  }
  if (a == 0.0) return;  // the start, its residual and the CG state stand
  const int sh = S->rr_shift;
  const bool fp64_norm = S->rr_fp64 != 0;
  double rz = 0.0, rr = 0.0;
  float rr32 = 0.0f;
  for (int64_t i = gtid(); i < nt; i += gstride()) {
    xs[i] = fma(a, dh[i], xs[i]);
    const double ri = fma(-a, w[i], rh[i]);
    rh[i] = ri;
    p[i] = ri;
    rz = fma(ri, ri, rz);
    if (fp64_norm) {
      rr = fma(diag[i] * ri, ri, rr);
    } else {
      const float ui = sq32[i] * abs_f32_scaled(ri, sh);
      rr32 = fmaf(ui, ui, rr32);
    }
  }
  double tot[2];
  bool last;
  if (fp64_norm) {
    double v[2] = {rz, rr};
    last = grid_sum<2>(v, partials, &S->counter[0], tot);
  } else {
    last = grid_sum_df(rz, rr32, partials, &S->counter[0], tot);
  }
  if (last && threadIdx.x == 0) {
    const double rrt = fp64_norm ? tot[1] : ldexp(tot[1], -2 * sh);
    S->rz = tot[0];
    S->rr = rrt;
    int stop = (rrt <= S->tol2 * S->bb) || S->maxit <= 0;
    if (!isfinite(tot[0]) || !isfinite(rrt)) {
      stop = 1;
      S->status = PIRMCUT_ENUMERIC;
    }
    S->stop_req = stop;
    if (use_cond) cudaGraphSetConditional(h, stop ? 0u : 1u);
  }
}

// ---------------------------------------------------------------------------
// x in the caller's numbering <-> reduced x
// ---------------------------------------------------------------------------

__global__ void k_scatter_x(int64_t nt, int32_t s, int32_t t, const double* __restrict__ xr,
                            double* __restrict__ xf) {
  const int64_t a = s < t ? s : t, b = s < t ? t : s;
  for (int64_t i = gtid(); i < nt; i += gstride()) {
    int64_t v = i;
    if (v >= a) ++v;
    if (v >= b) ++v;
    xf[v] = xr[i];
  }
  if (gtid() == 0) {
    xf[s] = 1.0;
    xf[t] = 0.0;
  }
}

__global__ void k_gather_x(int64_t nt, int32_t s, int32_t t, const double* __restrict__ xf,
                           double* __restrict__ xr) {
  const int64_t a = s < t ? s : t, b = s < t ? t : s;
  for (int64_t i = gtid(); i < nt; i += gstride()) {
    int64_t v = i;
    if (v >= a) ++v;
    if (v >= b) ++v;
    xr[i] = xf[v];
  }
}

// ---------------------------------------------------------------------------
// launch helpers (templates dispatched on the DIA width / CSR group size)
// ---------------------------------------------------------------------------


}  // namespace

cudaError_t launch_scatter_x(Ctx& c, double* xfull) {
  k_scatter_x<<<grid_for(c.nt), kThreads, 0, c.stream>>>(c.nt, c.hg.s, c.hg.t, c.x, xfull);
  c.launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_gather_x(Ctx& c, const double* xfull) {
  k_gather_x<<<grid_for(c.nt), kThreads, 0, c.stream>>>(c.nt, c.hg.s, c.hg.t, xfull, c.x);
  c.launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_spmv_once(Ctx& c) {
  const int grid = spmv_grid(c);
  if (c.format == PIRMCUT_FORMAT_DIA) {
    PIRMCUT_DISPATCH_K(c.K, (k_spmv_dia<KK><<<grid, kThreads, 0, c.stream>>>(
                                c.dd, c.ghat, c.p, c.q, c.partials, c.S)));
  } else {
    PIRMCUT_DISPATCH_G(c.group, (k_spmv_csr<GG><<<grid + c.n_heavy, kThreads, 0, c.stream>>>(
                                    c.nt, c.rp, c.col, c.ghat, c.p, c.q, c.partials, c.S,
                                    c.heavy_deg, c.heavy, grid)));
  }
  c.launches += 1;
  return cudaGetLastError();
}

namespace {

}  // namespace

// Step 1 (reweighting) into the FP64 conductance array; for x^(0) the
// capacities are copied instead (W^(0) = C).  Returns the kernels enqueued.
int enqueue_reweight(Ctx& c, cudaStream_t st, bool initial) {
  const int grid = row_grid(c);
  double* g = c.format == PIRMCUT_FORMAT_DIA ? c.gdia : c.gval;
  const double* cap = c.format == PIRMCUT_FORMAT_DIA ? c.cdia : c.cval;
  const size_t gbytes = sizeof(double) * (c.format == PIRMCUT_FORMAT_DIA
                                              ? size_t(c.K) * c.nt
                                              : size_t(c.hg.nnz));
  if (initial) {
    cudaMemcpyAsync(g, cap, gbytes, cudaMemcpyDeviceToDevice, st);
    return 0;
  }
  if (c.format == PIRMCUT_FORMAT_DIA) {
    PIRMCUT_DISPATCH_K(c.K, (k_reweight_dia<KK><<<grid, kThreads, 0, st>>>(
                                c.dd, c.cdia, c.x, c.eps_list, c.C, c.opt.reweight_form, c.gdia)));
  } else {
    PIRMCUT_DISPATCH_G(c.group, (k_reweight_csr<GG><<<grid + c.n_heavy, kThreads, 0, st>>>(
                                    c.nt, c.rp, c.col, c.cval, c.x, c.eps_list, c.C,
                                    c.opt.reweight_form, c.gval, c.heavy_deg, c.heavy, grid)));
  }
  return 1;
}

// Epilogue of a step: x from the scaled iterate (FP64 path), range of x and
// the step record; with options.step_stats, the objective and flow value.
int enqueue_step_end(Ctx& c, cudaStream_t st, bool initial, const OuterState* O) {
  const bool scaled = c.opt.precision == PIRMCUT_PREC_FP64;
  k_step_end<<<grid_for(c.nt), kThreads, 0, st>>>(c.nt, c.x, scaled ? c.xs : nullptr,
                                                  scaled ? c.rsd : nullptr, c.S, c.C, c.recs,
                                                  c.eps_list, initial ? 0 : 1, c.partials, O);
  if (!c.opt.step_stats) return 1;
  StatsArgs a;
  a.cs = c.cs;
  a.ct = c.ct;
  a.x = c.x;
  a.xw = c.xstats;
  a.eps_list = c.eps_list;
  a.C = c.C;
  a.recs = c.recs;
  a.partials = c.partials;
  // the step end's last-block counter, released by that block before this launch
  a.counter = reinterpret_cast<unsigned int*>(reinterpret_cast<char*>(c.S) +
                                              offsetof(PcgState, counter) + 3 * sizeof(unsigned int));
  a.c_st = c.hg.c_st;
  a.form = c.opt.reweight_form;
  a.initial = initial ? 1 : 0;
  if (c.format == PIRMCUT_FORMAT_DIA) {
    PIRMCUT_DISPATCH_K(c.K, (k_step_stats_dia<KK><<<grid_for(c.nt), kThreads, 0, st>>>(
                                c.dd, c.cdia, c.gdia, a)));
  } else {
    const int grid = row_grid(c);
    PIRMCUT_DISPATCH_G(c.group, (k_step_stats_csr<GG><<<grid + c.n_heavy, kThreads, 0, st>>>(
                                    c.nt, c.rp, c.col, c.cval, c.gval, a, c.heavy_deg, c.heavy,
                                    grid)));
  }
  return 2;
}

cudaError_t enqueue_stats_pre(Ctx& c, cudaStream_t st) {
  if (!c.opt.step_stats) return cudaSuccess;
  return cudaMemcpyAsync(c.xstats, c.x, sizeof(double) * size_t(c.nt), cudaMemcpyDeviceToDevice, st);
}

namespace {

// Kernels of a step before the PCG loop:
//   [keep x^(l-1), g^(l-1)] -> [c -> g | reweight] -> [features, learned start]
//   -> assemble -> scale.
int enqueue_prologue(Ctx& c, cudaStream_t st, bool initial, cudaGraphConditionalHandle h,
                     int use_cond, cudaError_t* err) {
  const int grid = row_grid(c);
  const bool zero_start = initial || !c.opt.warm_start;
  const bool mlp = mlp_active(c, initial);
  double* g = c.format == PIRMCUT_FORMAT_DIA ? c.gdia : c.gval;
  *err = enqueue_stats_pre(c, st);
  int kernels = mlp ? enqueue_mlp_pre(c, st) : 0;
  // the learned start reads this step's conductances before the assembly
  const bool fused = !initial && !mlp && c.opt.fuse_reweight && c.format == PIRMCUT_FORMAT_DIA;
  if (!fused) kernels += enqueue_reweight(c, st, initial);
  if (mlp) kernels += enqueue_mlp_post(c, st);
  AssembleArgs a;
  a.cs = c.cs;
  a.ct = c.ct;
  a.x = c.x;
  a.xw = c.x;
  a.eps_list = c.eps_list;
  a.C = c.C;
  a.form = c.opt.reweight_form;
  a.initial = initial ? 1 : 0;
  a.zero_start = zero_start ? 1 : 0;
  a.tol2 = c.opt.pcg_tol * c.opt.pcg_tol;
  a.maxit = c.opt.pcg_max_iter;
  a.diag = c.diag;
  a.rsd = c.rsd;
  a.sq32 = c.sq32;
  a.xs = c.xs;
  a.r = c.r;
  a.p = c.p;
  a.partials = c.partials;
  a.S = c.S;
  a.h = h;
  a.use_cond = use_cond;
  if (c.format == PIRMCUT_FORMAT_DIA) {
    if (fused) {
      PIRMCUT_DISPATCH_K(c.K, (k_reweight_assemble_dia<KK><<<grid, kThreads, 0, st>>>(c.dd, c.cdia, g, a)));
    } else {
      PIRMCUT_DISPATCH_K(c.K, (k_assemble_dia<KK><<<grid, kThreads, 0, st>>>(c.dd, g, a)));
    }
    PIRMCUT_DISPATCH_K(c.K, (k_scale_dia<KK><<<grid, kThreads, 0, st>>>(c.dd, g, c.rsd, c.ghat)));
  } else {
    PIRMCUT_DISPATCH_G(c.group, (k_assemble_csr<GG><<<grid + c.n_heavy, kThreads, 0, st>>>(
                                    c.nt, c.rp, c.col, g, a, c.heavy_deg, c.heavy, grid)));
    PIRMCUT_DISPATCH_G(c.group, (k_scale_csr<GG><<<grid + c.n_heavy, kThreads, 0, st>>>(
                                    c.nt, c.rp, c.col, g, c.rsd, c.ghat, c.heavy_deg, c.heavy, grid)));
  }
  kernels += 2;
  if (mlp && (c.mlp_mode & PIRMCUT_MLP_PREDICT)) {
    // the learned start, in the scaled space of this step's system
    MlpState* M = c.mlp.state;
    k_ls_prep<<<grid_for(c.nt), kThreads, 0, st>>>(c.nt, c.mlp.dir, c.diag, c.rsd);
    if (c.format == PIRMCUT_FORMAT_DIA) {
      PIRMCUT_DISPATCH_K(c.K, (k_ls_scaled_dia<KK><<<grid, kThreads, 0, st>>>(
                                  c.dd, c.ghat, c.mlp.dir, c.r, c.q, c.partials, c.S, M)));
    } else {
      PIRMCUT_DISPATCH_G(c.group, (k_ls_scaled_csr<GG><<<grid + c.n_heavy, kThreads, 0, st>>>(
                                      c.nt, c.rp, c.col, c.ghat, c.mlp.dir, c.r, c.q, c.partials,
                                      c.S, M, c.heavy_deg, c.heavy, grid)));
    }
    k_ls_commit<<<grid_for(c.nt), kThreads, 0, st>>>(c.nt, c.mlp.dir, c.q, c.sq32, c.diag, c.xs,
                                                      c.r, c.p, c.partials, c.S, M, h, use_cond);
    kernels += 3;
  }
  return kernels;
}

// One PCG iteration: spmv -> update_r -> update_xp (events, when given,
// bracket the spmv launch).
int enqueue_iteration(Ctx& c, cudaStream_t st, cudaGraphConditionalHandle h, int use_cond,
                      cudaEvent_t e0 = nullptr, cudaEvent_t e1 = nullptr) {
  const int vg = grid_for(c.nt);
  const int grid = spmv_grid(c);
  const int vgrid = vg < kFp64MaxBlocks ? vg : kFp64MaxBlocks;
  if (e0) cudaEventRecord(e0, st);
  if (c.format == PIRMCUT_FORMAT_DIA) {
    PIRMCUT_DISPATCH_K(c.K, (k_spmv_dia<KK><<<grid, kThreads, 0, st>>>(
                                c.dd, c.ghat, c.p, c.q, c.partials, c.S)));
  } else {
    PIRMCUT_DISPATCH_G(c.group, (k_spmv_csr<GG><<<grid + c.n_heavy, kThreads, 0, st>>>(
                                    c.nt, c.rp, c.col, c.ghat, c.p, c.q, c.partials, c.S,
                                    c.heavy_deg, c.heavy, grid)));
  }
  if (e1) cudaEventRecord(e1, st);
  k_update_r<<<vgrid, kThreads, 0, st>>>(c.nt, c.q, c.sq32, c.diag, c.r, c.partials, c.S);
  k_update_xp<<<vgrid, kThreads, 0, st>>>(c.nt, c.xs, c.p, c.r, c.S, h, use_cond);
  return 3;
}

}  // namespace

// Build the graph of one IRLS step (initial = x^(0) with W^(0) = C):
//   prologue -> WHILE{spmv, update_r, update_xp} -> step_end
cudaError_t build_step_graph(Ctx& c, bool initial, cudaGraphExec_t* out, int* nodes) {
  cudaError_t e;
  cudaStream_t st = c.cap_stream;
  int n_nodes = 0;
  if ((e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) return e;
  cudaGraph_t graph = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t ndeps = 0;
  cudaStreamCaptureStatus cst;
  cudaGraphConditionalHandle h{};
  cudaGraphNode_t cond_node{};
  e = cudaStreamGetCaptureInfo(st, &cst, nullptr, &graph, nullptr, nullptr, nullptr);
  if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&h, graph, 1, cudaGraphCondAssignDefault);
  if (e != cudaSuccess) {
    cudaGraph_t dummy = nullptr;
    cudaStreamEndCapture(st, &dummy);
    if (dummy) cudaGraphDestroy(dummy);
    return e;
  }
  cudaError_t ep = cudaSuccess;
  n_nodes += enqueue_prologue(c, st, initial, h, 1, &ep);
  // WHILE node holding one PCG iteration
  e = ep != cudaSuccess ? ep : cudaStreamGetCaptureInfo(st, &cst, nullptr, &graph, &deps, nullptr, &ndeps);
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  if (e == cudaSuccess) e = cudaGraphAddNode(&cond_node, graph, deps, nullptr, ndeps, &cp);
  if (e == cudaSuccess) {
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    cudaStream_t bs;
    e = cudaStreamCreateWithFlags(&bs, cudaStreamNonBlocking);
    if (e == cudaSuccess) {
      e = cudaStreamBeginCaptureToGraph(bs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        enqueue_iteration(c, bs, h, 1);
        cudaGraph_t bg = nullptr;
        e = cudaStreamEndCapture(bs, &bg);
      }
      cudaStreamDestroy(bs);
    }
  }
  if (e == cudaSuccess)
    e = cudaStreamUpdateCaptureDependencies(st, &cond_node, nullptr, 1, cudaStreamSetCaptureDependencies);
  // the step end writes x = D^-1/2 x^, which the learned start trains on
  if (e == cudaSuccess) n_nodes += enqueue_step_end(c, st, initial, nullptr);
  if (e == cudaSuccess && mlp_active(c, initial)) n_nodes += enqueue_mlp_train(c, st);
  cudaGraph_t captured = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(st, &captured);
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess) e = cudaGraphInstantiate(out, captured, 0);
  if (captured) cudaGraphDestroy(captured);
  *nodes = n_nodes;
  return e;
}

// The same step launched kernel by kernel on the context's stream (no graph):
// PCG iterations go in chunks of 8, the stop flag is read back between chunks.
// Kernels queued after the stop are no-ops (they test the flag first).
cudaError_t run_step_stream(Ctx& c, bool initial, int* stop_flag_host, int64_t* kernels) {
  cudaStream_t st = c.stream;
  cudaGraphConditionalHandle none{};
  cudaError_t ep = cudaSuccess;
  int64_t k = enqueue_prologue(c, st, initial, none, 0, &ep);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = ep;
  static_assert(offsetof(PcgState, maxit) == offsetof(PcgState, iters) + sizeof(int) &&
                    offsetof(PcgState, stop_req) == offsetof(PcgState, iters) + 2 * sizeof(int),
                "iters, maxit, stop_req are read back together");
  const size_t off = offsetof(PcgState, iters);
  PcgProgress* prog = reinterpret_cast<PcgProgress*>(stop_flag_host);
  cudaEvent_t* ev = c.opt.time_spmv ? spmv_events(c, 8) : nullptr;
  int iters_before = 0;
  for (int guard = 0; e == cudaSuccess; ++guard) {
    for (int j = 0; j < 8; ++j)
      k += enqueue_iteration(c, st, none, 0, ev ? ev[2 * j] : nullptr, ev ? ev[2 * j + 1] : nullptr);
    e = cudaMemcpyAsync(prog, reinterpret_cast<char*>(c.S) + off, sizeof(PcgProgress),
                        cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) break;
    if (ev) spmv_events_collect(c, 8, prog->iters - iters_before);
    iters_before = prog->iters;
    if (prog->stop_req) break;
    if (guard > c.opt.pcg_max_iter / 8 + 2) break;  // the device caps iterations; belt and braces
  }
  if (e == cudaSuccess) {
    k += enqueue_step_end(c, st, initial, nullptr);
    if (mlp_active(c, initial)) k += enqueue_mlp_train(c, st);
    e = cudaGetLastError();
  }
  *kernels = k;
  return e;
}

}  // namespace pirmcut
