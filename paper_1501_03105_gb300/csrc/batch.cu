// Batched IRLS solves: many independent s-t min-cut instances advanced by the
// same kernel launches (Section 6 motivates sequences and batches of related
// FlowImprove problems).
//
// The instances' reduced graphs are concatenated into one block-diagonal
// CSR (global row offsets, instance-local column ids).  Rows are cut into
// tiles that never straddle two instances, in three tiers by degree: range
// tiles cover consecutive rows, a group of G threads per row; rows above a
// middle threshold are listed in medium tiles, a warp per row (so one long
// row no longer holds up the short rows of its warp); a row above the hub
// threshold (a power-law hub) gets a tile of its own, processed by a whole
// block.  Range tiles skip the rows of the other two tiers.  Every kernel runs
// one block per tile.  Each instance keeps its own PCG scalars: a tile's block
// writes its partial sums, and the last tile of an instance to finish (an
// atomic ticket per instance) adds that instance's partials in tile order and
// updates its alpha / beta / stop flag -- deterministic, and no block waits on
// another.  Instances that have converged skip their tiles; the WHILE node of
// the step graph runs until no instance is active.  The number of threads per
// row and the tile height are chosen by timing the SpMV on the batch
// (pirmcut_batch_create's autotuner).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "ctx.h"
#include "pirmcut.h"

namespace pirmcut {

namespace {

constexpr int kBT = 256;  // threads per block (one block per tile)

// Tile kinds: consecutive rows [r0, r1); one hub row r0 for the whole block;
// entries [r0, r1) of the medium-row list, a warp per row.
constexpr int32_t kRangeTile = 0, kHubTile = 1, kMediumTile = 2;
constexpr int kMediumRowsPerTile = 64;  // 8 rows per warp
constexpr int kHubDeg = 512;            // rows with more entries: a block each

struct Tile {
  int32_t inst;
  int32_t kind;
  int64_t r0, r1;
};

struct BInst {
  int64_t base;   // first global row
  int64_t nt;
  int32_t t0, t1; // tile range
};

struct BArgs {
  const Tile* tiles;
  const BInst* insts;
  const int64_t* rp;    // global offsets into col/val
  const int32_t* col;   // instance-local ids
  int64_t mid_deg;      // rows with more entries go to medium or hub tiles
  int64_t heavy_deg;    // rows with more entries go to hub tiles
  const int64_t* med;   // medium rows (global ids), grouped by tile
  PcgState* S;          // per instance
  double* partials;     // NV * ntiles
  int ntiles;
  int* active;
  // the CG iterations' work list (rebuilt at the head of every iteration):
  // the active instances in order and the prefix sums of their tile counts
  const int* act_inst;  // [count]
  const int* act_pref;  // [count + 1]; act_pref[n_act] = active tiles
  const int* n_act;     // number of active instances
  int* work_next;       // [3] next work item of the three iteration kernels
  const int* order;     // instances, heaviest row first (the work list's order)
};

// Next item of a kernel's work list for this block (every thread gets it):
// blocks take items as they free up, so that long tiles (hub rows) do not
// hold up a fixed share of the list.
__device__ __forceinline__ int next_item(int* counter) {
  __shared__ int s_item;
  __syncthreads();  // every thread has read the previous item
  if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
  __syncthreads();
  return s_item;
}

// Tile of virtual index v of the work list (v < act_pref[n_act]).
__device__ __forceinline__ int work_tile(const BArgs& a, int n, int v) {
  int lo = 0, hi = n;  // act_pref[lo] <= v < act_pref[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (__ldg(a.act_pref + mid) <= v) lo = mid;
    else hi = mid;
  }
  return a.insts[a.act_inst[lo]].t0 + (v - a.act_pref[lo]);
}

__device__ __forceinline__ int64_t deg_of(const BArgs& a, int64_t r) { return a.rp[r + 1] - a.rp[r]; }

// Per-tile partials -> per-instance totals.  Returns true in every thread of
// the block that finished the instance; totals valid in thread 0.
template <int NV>
__device__ __forceinline__ bool inst_sum(const BArgs& a, const Tile& tl, int tile, double (&v)[NV],
                                         int site, double (&tot)[NV]) {
  __shared__ unsigned int s_last;
  block_sum<NV>(v);
  const BInst in = a.insts[tl.inst];
  if (threadIdx.x == 0) {
#pragma unroll
    for (int j = 0; j < NV; ++j) a.partials[j * a.ntiles + tile] = v[j];
    __threadfence();
    const unsigned int prev = atomicAdd(&a.S[tl.inst].counter[site], 1u);
    s_last = (prev == unsigned(in.t1 - in.t0 - 1)) ? 1u : 0u;
  }
  __syncthreads();
  if (!s_last) return false;
  __threadfence();
  double acc[NV];
#pragma unroll
  for (int j = 0; j < NV; ++j) acc[j] = 0.0;
  for (int t = in.t0 + int(threadIdx.x); t < in.t1; t += blockDim.x) {
#pragma unroll
    for (int j = 0; j < NV; ++j) acc[j] += __ldcg(a.partials + j * a.ntiles + t);
  }
  block_sum<NV>(acc);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int j = 0; j < NV; ++j) tot[j] = acc[j];
    a.S[tl.inst].counter[site] = 0u;
  }
  return true;
}

// sum of a row's partial products over its G-thread group (result in lane 0)
template <int G>
__device__ __forceinline__ double group_reduce(double v, unsigned mask) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v += __shfl_down_sync(mask, v, o, G);
  return v;
}

// sum of v over the block, result in thread 0 (heavy tiles)
__device__ __forceinline__ double block_total(double v) {
  double a[1] = {v};
  block_sum<1>(a);
  return a[0];
}

// ---------------------------------------------------------------------------
// reweighting
// ---------------------------------------------------------------------------

template <int G>
__global__ void __launch_bounds__(kBT)
kb_reweight(BArgs a, const double* __restrict__ c, const double* __restrict__ x,
            const double* __restrict__ eps_list, const StepCounters* __restrict__ C, int form,
            double* __restrict__ g) {
  const Tile tl = a.tiles[blockIdx.x];
  const int64_t base = a.insts[tl.inst].base;
  const double eps = eps_list[C->eps_idx];
  const double eps2 = eps * eps;
  if (tl.kind == kHubTile) {
    const int64_t r = tl.r0;
    const double xr = x[r];
    for (int64_t e = a.rp[r] + threadIdx.x; e < a.rp[r + 1]; e += kBT)
      g[e] = conductance(c[e], xr - x[base + a.col[e]], eps2, form);
    return;
  }
  if (tl.kind == kMediumTile) {
    const int lane = threadIdx.x & 31;
    for (int64_t m = tl.r0 + threadIdx.x / 32; m < tl.r1; m += kBT / 32) {
      const int64_t r = a.med[m];
      const double xr = x[r];
      for (int64_t e = a.rp[r] + lane; e < a.rp[r + 1]; e += 32)
        g[e] = conductance(c[e], xr - x[base + a.col[e]], eps2, form);
    }
    return;
  }
  const int lane = threadIdx.x % G;
  for (int64_t r = tl.r0 + threadIdx.x / G; r < tl.r1; r += kBT / G) {
    if (deg_of(a, r) > a.mid_deg) continue;
    const double xr = x[r];
    for (int64_t e = a.rp[r] + lane; e < a.rp[r + 1]; e += G)
      g[e] = conductance(c[e], xr - x[base + a.col[e]], eps2, form);
  }
}

// ---------------------------------------------------------------------------
// assembly + initial residual
// ---------------------------------------------------------------------------

struct BAssemble {
  const double* cs;
  const double* ct;
  const double* x;
  const double* eps_list;
  const StepCounters* C;
  int form, initial, zero_start;
  double tol2;
  int maxit;
  double* diag;
  double* dinv;
  double* r;
  double* p;
};

__device__ __forceinline__ void bassemble_row(const BAssemble& b, int64_t r, double sum, double ax,
                                              double eps2, double& rz, double& rr, double& bb) {
  const double xr = b.x[r];
  double gs = b.cs[r], gt = b.ct[r];
  if (!b.initial) {
    gs = conductance(gs, 1.0 - xr, eps2, b.form);
    gt = conductance(gt, xr, eps2, b.form);
  }
  sum += gs + gt;
  const double di = 1.0 / sum;
  const double ri = b.zero_start ? gs : gs - fma(sum, xr, -ax);
  const double zi = di * ri;
  b.diag[r] = sum;
  b.dinv[r] = di;
  b.r[r] = ri;
  b.p[r] = zi;
  rz = fma(ri, zi, rz);
  rr = fma(ri, ri, rr);
  bb = fma(gs, gs, bb);
}

template <int G>
__global__ void __launch_bounds__(kBT)
kb_assemble(BArgs a, const double* __restrict__ g, BAssemble b) {
  const Tile tl = a.tiles[blockIdx.x];
  const int64_t base = a.insts[tl.inst].base;
  const double eps = b.initial ? 0.0 : b.eps_list[b.C->eps_idx];
  const double eps2 = eps * eps;
  double rz = 0.0, rr = 0.0, bb = 0.0;
  if (tl.kind == kHubTile) {
    const int64_t r = tl.r0;
    double sum = 0.0, ax = 0.0;
    for (int64_t e = a.rp[r] + threadIdx.x; e < a.rp[r + 1]; e += kBT) {
      sum += g[e];
      ax = fma(g[e], b.x[base + a.col[e]], ax);
    }
    sum = block_total(sum);
    ax = block_total(ax);
    if (threadIdx.x == 0) bassemble_row(b, r, sum, ax, eps2, rz, rr, bb);
  } else if (tl.kind == kMediumTile) {
    const int lane = threadIdx.x & 31;
    for (int64_t m = tl.r0 + threadIdx.x / 32; m < tl.r1; m += kBT / 32) {
      const int64_t r = a.med[m];
      double sum = 0.0, ax = 0.0;
      for (int64_t e = a.rp[r] + lane; e < a.rp[r + 1]; e += 32) {
        sum += g[e];
        ax = fma(g[e], b.x[base + a.col[e]], ax);
      }
      sum = group_reduce<32>(sum, 0xffffffffu);
      ax = group_reduce<32>(ax, 0xffffffffu);
      if (lane == 0) bassemble_row(b, r, sum, ax, eps2, rz, rr, bb);
    }
  } else {
    const int lane = threadIdx.x % G;
    const unsigned mask = group_mask<G>();
    for (int64_t r = tl.r0 + threadIdx.x / G; r < tl.r1; r += kBT / G) {
      if (deg_of(a, r) > a.mid_deg) continue;
      double sum = 0.0, ax = 0.0;
      for (int64_t e = a.rp[r] + lane; e < a.rp[r + 1]; e += G) {
        sum += g[e];
        ax = fma(g[e], b.x[base + a.col[e]], ax);
      }
      sum = group_reduce<G>(sum, mask);
      ax = group_reduce<G>(ax, mask);
      if (lane == 0) bassemble_row(b, r, sum, ax, eps2, rz, rr, bb);
    }
  }
  double v[3] = {rz, rr, bb}, tot[3];
  if (inst_sum<3>(a, tl, int(blockIdx.x), v, 0, tot) && threadIdx.x == 0) {
    PcgState* S = &a.S[tl.inst];
    S->rz = tot[0];
    S->rr = tot[1];
    S->bb = tot[2];
    S->tol2 = b.tol2;
    S->maxit = b.maxit;
    S->iters = 0;
    S->stopped = 0;
    S->status = PIRMCUT_OK;
    S->alpha = 0.0;
    S->beta = 0.0;
    int stop = (tot[1] <= b.tol2 * tot[2]) || b.maxit <= 0 || tot[2] == 0.0;
    if (!isfinite(tot[0]) || !isfinite(tot[1]) || !isfinite(tot[2])) {
      stop = 1;
      S->status = PIRMCUT_ENUMERIC;
    }
    S->stop_req = stop;
    if (!stop) atomicAdd(a.active, 1);
  }
}

// ---------------------------------------------------------------------------
// PCG iteration
// ---------------------------------------------------------------------------

// Work list of a CG iteration: the instances that have not stopped, in
// order, with the prefix sums of their tile counts (one block, fixed order).
// Instances that stopped cost the iteration's kernels nothing.
__global__ void __launch_bounds__(kBT)
kb_worklist(BArgs a, int count, int* act_inst, int* act_pref, int* n_act) {
  __shared__ int s_cnt[kBT], s_tiles[kBT];
  const int per = (count + kBT - 1) / kBT;  // consecutive list positions per thread
  const int i0 = threadIdx.x * per, i1 = min(count, i0 + per);
  int cnt = 0, tiles = 0;
  for (int k = i0; k < i1; ++k) {
    const int i = a.order[k];
    if (!a.S[i].stop_req) {
      ++cnt;
      tiles += a.insts[i].t1 - a.insts[i].t0;
    }
  }
  s_cnt[threadIdx.x] = cnt;
  s_tiles[threadIdx.x] = tiles;
  __syncthreads();
  if (threadIdx.x == 0) {  // exclusive scan in place, in thread order
    int c = 0, t = 0;
    for (int k = 0; k < kBT; ++k) {
      const int ck = s_cnt[k], tk = s_tiles[k];
      s_cnt[k] = c;
      s_tiles[k] = t;
      c += ck;
      t += tk;
    }
    *n_act = c;
    act_pref[c] = t;
    a.work_next[0] = 0;
    a.work_next[1] = 0;
    a.work_next[2] = 0;
  }
  __syncthreads();
  int j = s_cnt[threadIdx.x], t = s_tiles[threadIdx.x];
  for (int k = i0; k < i1; ++k) {
    const int i = a.order[k];
    if (!a.S[i].stop_req) {
      act_inst[j] = i;
      act_pref[j] = t;
      ++j;
      t += a.insts[i].t1 - a.insts[i].t0;
    }
  }
}

// The CG iteration kernels run a fixed grid; each block walks the work list.
template <int G>
__global__ void __launch_bounds__(kBT)
kb_spmv(BArgs a, const double* __restrict__ g, const double* __restrict__ diag,
        const double* __restrict__ p, double* __restrict__ q) {
  const int n = *a.n_act;
  const int work = a.act_pref[n];
  for (int v = next_item(a.work_next); v < work; v = next_item(a.work_next)) {
    const int tile = work_tile(a, n, v);
    const Tile tl = a.tiles[tile];
    PcgState* S = &a.S[tl.inst];
    const int64_t base = a.insts[tl.inst].base;
    double pq = 0.0;
    if (tl.kind == kHubTile) {
      const int64_t r = tl.r0;
      double acc = 0.0;
      for (int64_t e = a.rp[r] + threadIdx.x; e < a.rp[r + 1]; e += kBT)
        acc = fma(-g[e], p[base + a.col[e]], acc);
      acc = block_total(acc);
      if (threadIdx.x == 0) {
        acc = fma(diag[r], p[r], acc);
        q[r] = acc;
        pq = p[r] * acc;
      }
    } else if (tl.kind == kMediumTile) {
      const int lane = threadIdx.x & 31;
      for (int64_t m = tl.r0 + threadIdx.x / 32; m < tl.r1; m += kBT / 32) {
        const int64_t r = a.med[m];
        double acc = 0.0;
        acc = row_dot_neg(g, a.col, p + base, a.rp[r] + lane, a.rp[r + 1], 32, acc);
        acc = group_reduce<32>(acc, 0xffffffffu);
        if (lane == 0) {
          const double pr = p[r];
          acc = fma(diag[r], pr, acc);
          q[r] = acc;
          pq = fma(pr, acc, pq);
        }
      }
    } else {
      const int lane = threadIdx.x % G;
      const unsigned mask = group_mask<G>();
      for (int64_t r = tl.r0 + threadIdx.x / G; r < tl.r1; r += kBT / G) {
        if (deg_of(a, r) > a.mid_deg) continue;
        double acc = 0.0;
        acc = row_dot_neg(g, a.col, p + base, a.rp[r] + lane, a.rp[r + 1], G, acc);
        acc = group_reduce<G>(acc, mask);
        if (lane == 0) {
          const double pr = p[r];
          acc = fma(diag[r], pr, acc);
          q[r] = acc;
          pq = fma(pr, acc, pq);
        }
      }
    }
    double vv[1] = {pq}, tot[1];
    if (inst_sum<1>(a, tl, tile, vv, 1, tot) && threadIdx.x == 0) {
      const double al = S->rz / tot[0];
      S->pq = tot[0];
      if (!(tot[0] > 0.0) || !isfinite(al)) {
        S->alpha = 0.0;
        S->status = PIRMCUT_ENUMERIC;
        S->stop_req = 1;
        atomicSub(a.active, 1);
      } else {
        S->alpha = al;
      }
    }
  }
}

// elementwise kernels visit the full row range of range tiles (medium and
// hub rows included) and only post a zero partial for the other tiles
__global__ void __launch_bounds__(kBT)
kb_update_r(BArgs a, double* __restrict__ qz, const double* __restrict__ dinv,
            double* __restrict__ r) {
  const int n = *a.n_act;
  const int work = a.act_pref[n];
  for (int v = next_item(a.work_next + 1); v < work; v = next_item(a.work_next + 1)) {
    const int tile = work_tile(a, n, v);
    const Tile tl = a.tiles[tile];
    PcgState* S = &a.S[tl.inst];
    if (S->stop_req) continue;  // broke down in this iteration's SpMV (the instance agrees)
    const double alpha = S->alpha;
    double rz = 0.0, rr = 0.0;
    if (tl.kind == kRangeTile) {
      for (int64_t i = tl.r0 + threadIdx.x; i < tl.r1; i += kBT) {
        const double ri = fma(-alpha, qz[i], r[i]);
        const double zi = dinv[i] * ri;
        r[i] = ri;
        qz[i] = zi;
        rz = fma(ri, zi, rz);
        rr = fma(ri, ri, rr);
      }
    }
    double vv[2] = {rz, rr}, tot[2];
    if (inst_sum<2>(a, tl, tile, vv, 2, tot) && threadIdx.x == 0) {
      const int it = S->iters + 1;
      S->iters = it;
      const double beta = tot[0] / S->rz;
      S->beta = beta;
      S->rz = tot[0];
      S->rr = tot[1];
      int stop = (tot[1] <= S->tol2 * S->bb) || it >= S->maxit;
      if (!isfinite(tot[1]) || !isfinite(beta)) {
        stop = 1;
        S->status = PIRMCUT_ENUMERIC;
        S->beta = 0.0;
      }
      S->stop_req = stop;
      if (stop) atomicSub(a.active, 1);
    }
  }
}

// x += alpha p, p = z + beta p for the instances of this iteration's list
// (an instance that stopped in this iteration's residual update still takes
// its last step); ends the loop once no instance is active.
__global__ void __launch_bounds__(kBT)
kb_update_xp(BArgs a, double* __restrict__ x, double* __restrict__ p, const double* __restrict__ z,
             cudaGraphConditionalHandle h, int use_cond) {
  const int n = *a.n_act;
  const int work = a.act_pref[n];
  for (int v = next_item(a.work_next + 2); v < work; v = next_item(a.work_next + 2)) {
    const Tile tl = a.tiles[work_tile(a, n, v)];
    if (tl.kind != kRangeTile) continue;
    const PcgState* S = &a.S[tl.inst];
    const double alpha = S->alpha, beta = S->beta;
    for (int64_t i = tl.r0 + threadIdx.x; i < tl.r1; i += kBT) {
      const double pi = p[i];
      x[i] = fma(alpha, pi, x[i]);
      p[i] = fma(beta, pi, z[i]);
    }
  }
  if (use_cond && blockIdx.x == 0 && threadIdx.x == 0 && *a.active == 0) cudaGraphSetConditional(h, 0u);
}

// per-instance step record (x range, iterations, residual)
__global__ void __launch_bounds__(kBT)
kb_step_end(BArgs a, const double* __restrict__ x, StepRec* recs, int rec_cap,
            const StepCounters* C, const double* eps_list, int consumes_eps) {
  const Tile tl = a.tiles[blockIdx.x];
  double mn = INFINITY, mx = -INFINITY;
  if (tl.kind == kRangeTile) {
    for (int64_t i = tl.r0 + threadIdx.x; i < tl.r1; i += kBT) {
      mn = fmin(mn, x[i]);
      mx = fmax(mx, x[i]);
    }
  }
  // block min / max, then the instance's last tile takes them over its tiles
  __shared__ double smn[kBT / 32], smx[kBT / 32];
  __shared__ unsigned int s_last;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    mn = fmin(mn, __shfl_down_sync(0xffffffffu, mn, o));
    mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, o));
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    smn[wid] = mn;
    smx[wid] = mx;
  }
  __syncthreads();
  const BInst in = a.insts[tl.inst];
  if (threadIdx.x == 0) {
    for (int w = 1; w < kBT / 32; ++w) {
      mn = fmin(mn, smn[w]);
      mx = fmax(mx, smx[w]);
    }
    a.partials[blockIdx.x] = mn;
    a.partials[a.ntiles + blockIdx.x] = mx;
    __threadfence();
    s_last = (atomicAdd(&a.S[tl.inst].counter[3], 1u) == unsigned(in.t1 - in.t0 - 1)) ? 1u : 0u;
  }
  __syncthreads();
  if (!s_last || threadIdx.x != 0) return;
  __threadfence();
  mn = INFINITY;
  mx = -INFINITY;
  for (int t = in.t0; t < in.t1; ++t) {
    mn = fmin(mn, __ldcg(a.partials + t));
    mx = fmax(mx, __ldcg(a.partials + a.ntiles + t));
  }
  PcgState* S = &a.S[tl.inst];
  S->counter[3] = 0u;
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
  rec.refine = 0;
  rec.obj = NAN;
  rec.flow = NAN;
  recs[size_t(tl.inst) * rec_cap + C->rec_idx] = rec;
}

__global__ void kb_advance(StepCounters* C, int consumes_eps) {
  C->rec_idx += 1;
  C->step += 1;
  if (consumes_eps) C->eps_idx += 1;
}

// b = 0 instances: the solution of L~ v = 0 is v = 0
__global__ void __launch_bounds__(kBT) kb_zero_if_b0(BArgs a, double* __restrict__ x) {
  const Tile tl = a.tiles[blockIdx.x];
  if (tl.kind != kRangeTile || a.S[tl.inst].bb != 0.0) return;
  for (int64_t i = tl.r0 + threadIdx.x; i < tl.r1; i += kBT) x[i] = 0.0;
}

__global__ void kb_scatter_x(int64_t nt, int64_t base, int32_t s, int32_t t, const double* __restrict__ xr,
                             double* __restrict__ xf) {
  const int64_t a = s < t ? s : t, b = s < t ? t : s;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < nt; i += int64_t(gridDim.x) * blockDim.x) {
    int64_t v = i;
    if (v >= a) ++v;
    if (v >= b) ++v;
    xf[v] = xr[base + i];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    xf[s] = 1.0;
    xf[t] = 0.0;
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

struct Batch {
  int count = 0;
  pirmcut_options opt{};
  std::string err;
  cudaStream_t stream = nullptr;
  cudaStream_t cap_stream = nullptr;
  std::vector<HostGraph> hg;
  std::vector<BInst> h_insts;
  std::vector<Tile> h_tiles;
  int64_t N = 0, M = 0;
  int G = 8;
  int tile_rows = 1024;
  int64_t mid_deg = 512;    // rows above: a warp each (medium tiles)
  int64_t heavy_deg = 512;  // rows above: a block each (hub tiles)
  std::vector<int64_t> h_med;
  // device
  int64_t* rp = nullptr;
  int32_t* col = nullptr;
  double *cval = nullptr, *gval = nullptr, *cs = nullptr, *ct = nullptr;
  double *x = nullptr, *r = nullptr, *p = nullptr, *q = nullptr, *diag = nullptr, *dinv = nullptr;
  Tile* tiles = nullptr;
  int64_t* med = nullptr;
  BInst* insts = nullptr;
  int* act_inst = nullptr;   // CG work list: active instances, prefix of their tiles, count
  int* act_pref = nullptr;
  int* n_act = nullptr;
  int* work_next = nullptr;  // [3]
  int* order = nullptr;      // instances by descending largest row degree
  int work_grid = 608;       // blocks of the CG iteration kernels (SMs x resident blocks)
  PcgState* S = nullptr;
  double* partials = nullptr;
  int* active = nullptr;
  StepCounters* C = nullptr;
  StepCounters* h_ctr = nullptr;  // pinned; followed by one int, the active-instance count read back in stream mode
  double* eps_list = nullptr;
  int eps_cap = 0;
  StepRec* recs = nullptr;
  StepRec* h_recs = nullptr;
  int rec_cap = 0;
  double* xfull = nullptr;
  int64_t xfull_cap = 0;
  cudaGraphExec_t g_init = nullptr, g_step = nullptr;
  int64_t launches = 0;
  bool x_set = false;
  Ctx view;  // sweep-cut view of one instance
  std::vector<cudaEvent_t> events;
};

namespace {

BArgs make_args(Batch& b) {
  BArgs a;
  a.tiles = b.tiles;
  a.insts = b.insts;
  a.rp = b.rp;
  a.col = b.col;
  a.mid_deg = b.mid_deg;
  a.heavy_deg = b.heavy_deg;
  a.med = b.med;
  a.S = b.S;
  a.partials = b.partials;
  a.ntiles = int(b.h_tiles.size());
  a.active = b.active;
  a.act_inst = b.act_inst;
  a.act_pref = b.act_pref;
  a.n_act = b.n_act;
  a.work_next = b.work_next;
  a.order = b.order;
  return a;
}

// Blocks of the CG iteration kernels: every block resident at once, never
// more than there are tiles.
int work_grid(const Batch& b) {
  const int nt = int(b.h_tiles.size());
  return nt < b.work_grid ? nt : b.work_grid;
}

void enqueue_worklist(Batch& b, cudaStream_t st) {
  kb_worklist<<<1, kBT, 0, st>>>(make_args(b), b.count, b.act_inst, b.act_pref, b.n_act);
}

void build_tiles(Batch& b) {
  // per instance: hub tiles first (the longest work items), then medium
  // tiles, then consecutive-row tiles
  b.h_tiles.clear();
  b.h_med.clear();
  for (int i = 0; i < b.count; ++i) {
    BInst& in = b.h_insts[i];
    const HostGraph& g = b.hg[i];
    in.t0 = int32_t(b.h_tiles.size());
    const int64_t m0 = int64_t(b.h_med.size());
    for (int64_t r = 0; r < g.nt; ++r) {
      const int64_t deg = g.rp[r + 1] - g.rp[r];
      if (deg > b.heavy_deg)
        b.h_tiles.push_back(Tile{i, kHubTile, in.base + r, in.base + r + 1});
      else if (deg > b.mid_deg)
        b.h_med.push_back(in.base + r);
    }
    const int64_t m1 = int64_t(b.h_med.size());
    for (int64_t m = m0; m < m1; m += kMediumRowsPerTile)
      b.h_tiles.push_back(Tile{i, kMediumTile, m, std::min<int64_t>(m1, m + kMediumRowsPerTile)});
    for (int64_t r0 = 0; r0 < g.nt; r0 += b.tile_rows) {
      const int64_t r1 = std::min<int64_t>(g.nt, r0 + b.tile_rows);
      b.h_tiles.push_back(Tile{i, kRangeTile, in.base + r0, in.base + r1});
    }
    in.t1 = int32_t(b.h_tiles.size());
  }
}

cudaError_t upload_tiles(Batch& b) {
  if (b.tiles) cudaFree(b.tiles);
  if (b.partials) cudaFree(b.partials);
  if (b.med) cudaFree(b.med);
  b.tiles = nullptr;
  b.partials = nullptr;
  b.med = nullptr;
  cudaError_t e = cudaMalloc(&b.tiles, sizeof(Tile) * b.h_tiles.size());
  if (e == cudaSuccess) e = cudaMalloc(&b.med, sizeof(int64_t) * std::max<size_t>(1, b.h_med.size()));
  if (e == cudaSuccess && !b.h_med.empty())
    e = cudaMemcpy(b.med, b.h_med.data(), sizeof(int64_t) * b.h_med.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&b.partials, sizeof(double) * 4 * b.h_tiles.size());
  if (e == cudaSuccess)
    e = cudaMemcpy(b.tiles, b.h_tiles.data(), sizeof(Tile) * b.h_tiles.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(b.insts, b.h_insts.data(), sizeof(BInst) * b.count, cudaMemcpyHostToDevice);
  return e;
}

void enqueue_spmv(Batch& b, cudaStream_t st, const double* g) {
  BArgs a = make_args(b);
  const int wg = work_grid(b);
  PIRMCUT_DISPATCH_G(b.G, (kb_spmv<GG><<<wg, kBT, 0, st>>>(a, g, b.diag, b.p, b.q)));
}

int enqueue_bstep(Batch& b, cudaStream_t st, bool initial, cudaGraphConditionalHandle h,
                  int use_cond, int part) {
  // part 0: prologue, 1: one PCG iteration, 2: epilogue
  BArgs a = make_args(b);
  const int nt = int(b.h_tiles.size());
  int k = 0;
  if (part == 0) {
    if (initial) {
      cudaMemcpyAsync(b.gval, b.cval, sizeof(double) * b.M, cudaMemcpyDeviceToDevice, st);
    } else {
      PIRMCUT_DISPATCH_G(b.G, (kb_reweight<GG><<<nt, kBT, 0, st>>>(a, b.cval, b.x, b.eps_list, b.C,
                                                                  b.opt.reweight_form, b.gval)));
      ++k;
    }
    cudaMemsetAsync(b.active, 0, sizeof(int), st);
    BAssemble as;
    as.cs = b.cs;
    as.ct = b.ct;
    as.x = b.x;
    as.eps_list = b.eps_list;
    as.C = b.C;
    as.form = b.opt.reweight_form;
    as.initial = initial ? 1 : 0;
    as.zero_start = (initial || !b.opt.warm_start) ? 1 : 0;
    as.tol2 = b.opt.pcg_tol * b.opt.pcg_tol;
    as.maxit = b.opt.pcg_max_iter;
    as.diag = b.diag;
    as.dinv = b.dinv;
    as.r = b.r;
    as.p = b.p;
    PIRMCUT_DISPATCH_G(b.G, (kb_assemble<GG><<<nt, kBT, 0, st>>>(a, b.gval, as)));
    ++k;
    if (as.zero_start) cudaMemsetAsync(b.x, 0, sizeof(double) * b.N, st);
  } else if (part == 1) {
    const int wg = work_grid(b);
    enqueue_worklist(b, st);
    enqueue_spmv(b, st, b.gval);
    kb_update_r<<<wg, kBT, 0, st>>>(a, b.q, b.dinv, b.r);
    kb_update_xp<<<wg, kBT, 0, st>>>(a, b.x, b.p, b.q, h, use_cond);
    k += 4;
  } else {
    kb_zero_if_b0<<<nt, kBT, 0, st>>>(a, b.x);
    kb_step_end<<<nt, kBT, 0, st>>>(a, b.x, b.recs, b.rec_cap, b.C, b.eps_list, initial ? 0 : 1);
    kb_advance<<<1, 1, 0, st>>>(b.C, initial ? 0 : 1);
    k += 3;
  }
  return k;
}

cudaError_t build_bgraph(Batch& b, bool initial, cudaGraphExec_t* out) {
  cudaStream_t st = b.cap_stream;
  cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  cudaGraph_t graph = nullptr;
  cudaStreamCaptureStatus cst;
  cudaGraphConditionalHandle h{};
  cudaGraphNode_t node{};
  const cudaGraphNode_t* deps = nullptr;
  size_t ndeps = 0;
  e = cudaStreamGetCaptureInfo(st, &cst, nullptr, &graph, nullptr, nullptr, nullptr);
  if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&h, graph, 1, cudaGraphCondAssignDefault);
  if (e == cudaSuccess) {
    enqueue_bstep(b, st, initial, h, 1, 0);
    e = cudaStreamGetCaptureInfo(st, &cst, nullptr, &graph, &deps, nullptr, &ndeps);
  }
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  if (e == cudaSuccess) e = cudaGraphAddNode(&node, graph, deps, nullptr, ndeps, &cp);
  if (e == cudaSuccess) {
    cudaStream_t bs = nullptr;
    e = cudaStreamCreateWithFlags(&bs, cudaStreamNonBlocking);
    if (e == cudaSuccess)
      e = cudaStreamBeginCaptureToGraph(bs, cp.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                        cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      enqueue_bstep(b, bs, initial, h, 1, 1);
      cudaGraph_t bg = nullptr;
      e = cudaStreamEndCapture(bs, &bg);
    }
    if (bs) cudaStreamDestroy(bs);
  }
  if (e == cudaSuccess)
    e = cudaStreamUpdateCaptureDependencies(st, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
  if (e == cudaSuccess) enqueue_bstep(b, st, initial, h, 1, 2);
  cudaGraph_t captured = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(st, &captured);
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess) e = cudaGraphInstantiate(out, captured, 0);
  if (captured) cudaGraphDestroy(captured);
  return e;
}

void free_batch(Batch& b) {
  void* ps[] = {b.rp, b.col, b.cval, b.gval, b.cs, b.ct, b.x, b.r, b.p, b.q, b.diag, b.dinv,
                b.tiles, b.med, b.insts, b.S, b.partials, b.active, b.C, b.eps_list, b.recs, b.xfull,
                b.act_inst, b.act_pref, b.n_act, b.work_next, b.order};
  for (void* p : ps)
    if (p) cudaFree(p);
  sweep_free(b.view);
  if (b.view.heavy) cudaFree(b.view.heavy);
  if (b.g_init) cudaGraphExecDestroy(b.g_init);
  if (b.g_step) cudaGraphExecDestroy(b.g_step);
  if (b.cap_stream) cudaStreamDestroy(b.cap_stream);
  if (b.h_ctr) cudaFreeHost(b.h_ctr);
  if (b.h_recs) cudaFreeHost(b.h_recs);
  for (cudaEvent_t ev : b.events) cudaEventDestroy(ev);
}

// Autotuner: time the batched SpMV (capacities as conductances) for each
// (threads per row, tile height, medium-row threshold) candidate and keep the
// fastest.  A medium threshold equal to the hub threshold disables that tier.
// A value fixed in the options replaces its list of candidates.  The timing
// runs with every instance active, but most PCG iterations of a step run with
// few instances left, where each tile costs a block launch that finds nothing
// to do; so a taller tile height (fewer tiles) is kept unless a shorter one
// is more than 10 % faster.
cudaError_t autotune(Batch& b) {
  std::vector<int> Gs = {1, 2, 4, 8, 16, 32}, Ts = {512, 2048};
  std::vector<int64_t> Ms = {16, 32, 64, b.heavy_deg};
  if (b.opt.batch_threads_per_row) Gs = {b.opt.batch_threads_per_row};
  if (b.opt.batch_tile_rows) Ts = {b.opt.batch_tile_rows};
  if (b.opt.batch_medium_deg) Ms = {int64_t(b.opt.batch_medium_deg)};
  cudaError_t e = cudaMemcpy(b.gval, b.cval, sizeof(double) * b.M, cudaMemcpyDeviceToDevice);
  if (e == cudaSuccess) e = cudaMemset(b.p, 0, sizeof(double) * b.N);
  if (e == cudaSuccess) e = cudaMemset(b.diag, 0, sizeof(double) * b.N);
  if (e != cudaSuccess) return e;
  // keep every instance "active" for timing
  std::vector<PcgState> st(b.count);
  std::memset(st.data(), 0, sizeof(PcgState) * b.count);
  for (auto& s : st) s.rz = 1.0;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  int bestG = b.G, bestT = b.tile_rows;
  int64_t bestM = b.heavy_deg;
  const int nM = int(Ms.size());
  for (int tm = 0; tm < int(Ts.size()) * nM; ++tm) {
    const int T = Ts[tm / nM];
    const int64_t M = Ms[tm % nM];
    b.tile_rows = T;
    b.mid_deg = M;
    build_tiles(b);
    if ((e = upload_tiles(b)) != cudaSuccess) break;
    for (int G : Gs) {
      b.G = G;
      float tot = 0.f;
      for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
        e = cudaMemcpy(b.S, st.data(), sizeof(PcgState) * b.count, cudaMemcpyHostToDevice);
        enqueue_worklist(b, b.stream);
        cudaEventRecord(e0, b.stream);
        enqueue_spmv(b, b.stream, b.gval);
        cudaEventRecord(e1, b.stream);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0) tot += ms;  // first launch warms up
        b.launches += 1;
      }
      if (e == cudaSuccess) e = cudaGetLastError();
      if (e != cudaSuccess) break;
      const bool taller = T > bestT, shorter = T < bestT;
      if ((taller && tot < best * 1.1f) || (shorter && tot < best * 0.9f) ||
          (!taller && !shorter && tot < best)) {
        best = tot;
        bestG = G;
        bestT = T;
        bestM = M;
      }
    }
    if (e != cudaSuccess) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return e;
  b.G = bestG;
  b.tile_rows = bestT;
  b.mid_deg = bestM;
  build_tiles(b);
  e = upload_tiles(b);
  if (e == cudaSuccess) e = cudaMemset(b.S, 0, sizeof(PcgState) * b.count);
  return e;
}

}  // namespace

}  // namespace pirmcut

struct pirmcut_batch {
  pirmcut::Batch b;
};

namespace {

thread_local std::string g_batch_err;

pirmcut_status bfail(pirmcut_batch* h, pirmcut_status st, const std::string& m) {
  if (h) h->b.err = m;
  else g_batch_err = m;
  pirmcut::set_global_error(m);
  return st;
}

#define BCK(h, call, where)                                                                        \
  do {                                                                                             \
    cudaError_t e_ = (call);                                                                       \
    if (e_ != cudaSuccess)                                                                         \
      return bfail(h, e_ == cudaErrorMemoryAllocation ? PIRMCUT_ENOMEM : PIRMCUT_ECUDA,            \
                   std::string(where) + ": " + cudaGetErrorString(e_));                           \
  } while (0)

}  // namespace

extern "C" {

pirmcut_status pirmcut_batch_create(int count, const int64_t* n, const int64_t* const* row_ptr,
                                    const int32_t* const* col, const double* const* c,
                                    const int32_t* s, const int32_t* t, const pirmcut_options* opt,
                                    void* stream, pirmcut_batch** out) {
  using namespace pirmcut;
  if (!out) return bfail(nullptr, PIRMCUT_EINVAL, "out must not be NULL");
  *out = nullptr;
  if (count < 1 || !n || !row_ptr || !col || !c || !s || !t)
    return bfail(nullptr, PIRMCUT_EINVAL, "count must be >= 1 and every array non-NULL");
  pirmcut_options o;
  pirmcut_default_options(&o);
  if (opt) o = *opt;
  if (o.precision != PIRMCUT_PREC_FP64)
    return bfail(nullptr, PIRMCUT_EINVAL, "batches run the FP64 solver");
  if (!(o.pcg_tol > 0.0) || o.pcg_max_iter < 0)
    return bfail(nullptr, PIRMCUT_EINVAL, "bad pcg_tol or pcg_max_iter");
  {
    const int g = o.batch_threads_per_row, tr = o.batch_tile_rows, md = o.batch_medium_deg;
    if (!(g == 0 || g == 1 || g == 2 || g == 4 || g == 8 || g == 16 || g == 32) ||
        !(tr == 0 || (tr >= 64 && tr <= 65536)) || md < 0 || md > kHubDeg)
      return bfail(nullptr, PIRMCUT_EINVAL,
                   "batch_threads_per_row must be 0, 1, 2, 4, 8, 16 or 32, batch_tile_rows 0 or "
                   "64..65536, batch_medium_deg 0..512");
  }
  pirmcut_batch* h = new (std::nothrow) pirmcut_batch();
  if (!h) return bfail(nullptr, PIRMCUT_ENOMEM, "out of host memory");
  Batch& b = h->b;
  b.count = count;
  b.opt = o;
  b.stream = reinterpret_cast<cudaStream_t>(stream);
  b.hg.resize(count);
  b.h_insts.resize(count);
  for (int i = 0; i < count; ++i) {
    std::string msg;
    pirmcut_status ps = reduce_graph(n[i], row_ptr[i], col[i], c[i], s[i], t[i], PIRMCUT_FORMAT_CSR,
                                     &b.hg[i], &msg);
    if (ps != PIRMCUT_OK) {
      delete h;
      return bfail(nullptr, ps, "instance " + std::to_string(i) + ": " + msg);
    }
    b.h_insts[i].base = b.N;
    b.h_insts[i].nt = b.hg[i].nt;
    b.N += b.hg[i].nt;
    b.M += int64_t(b.hg[i].col.size());
  }
  // concatenate: global row offsets, local columns
  std::vector<int64_t> rp(b.N + 1);
  std::vector<int32_t> cl(b.M);
  std::vector<double> cv(b.M), csv(b.N), ctv(b.N);
  int64_t off = 0;
  for (int i = 0; i < count; ++i) {
    const HostGraph& g = b.hg[i];
    const int64_t base = b.h_insts[i].base;
    for (int64_t r = 0; r < g.nt; ++r) rp[base + r] = off + g.rp[r];
    std::copy(g.col.begin(), g.col.end(), cl.begin() + off);
    std::copy(g.cval.begin(), g.cval.end(), cv.begin() + off);
    std::copy(g.cs.begin(), g.cs.end(), csv.begin() + base);
    std::copy(g.ct.begin(), g.ct.end(), ctv.begin() + base);
    off += int64_t(g.col.size());
  }
  rp[b.N] = off;
  auto bail = [&](cudaError_t e, const char* w) {
    free_batch(b);
    delete h;
    return bfail(nullptr, e == cudaErrorMemoryAllocation ? PIRMCUT_ENOMEM : PIRMCUT_ECUDA,
                 std::string(w) + ": " + cudaGetErrorString(e));
  };
  cudaError_t e = cudaStreamCreateWithFlags(&b.cap_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) return bail(e, "cudaStreamCreate");
  auto A = [&](void** p, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(p, bytes ? bytes : 8);
  };
  A((void**)&b.rp, sizeof(int64_t) * (b.N + 1));
  A((void**)&b.col, sizeof(int32_t) * b.M);
  A((void**)&b.cval, sizeof(double) * b.M);
  A((void**)&b.gval, sizeof(double) * b.M);
  for (double** v : {&b.cs, &b.ct, &b.x, &b.r, &b.p, &b.q, &b.diag, &b.dinv}) A((void**)v, sizeof(double) * b.N);
  A((void**)&b.insts, sizeof(BInst) * count);
  A((void**)&b.act_inst, sizeof(int) * count);
  A((void**)&b.act_pref, sizeof(int) * (count + 1));
  A((void**)&b.n_act, sizeof(int));
  A((void**)&b.work_next, sizeof(int) * 3);
  A((void**)&b.order, sizeof(int) * count);
  A((void**)&b.S, sizeof(PcgState) * count);
  A((void**)&b.active, sizeof(int));
  A((void**)&b.C, sizeof(StepCounters));
  if (e != cudaSuccess) return bail(e, "cudaMalloc");
  e = cudaMemcpy(b.rp, rp.data(), sizeof(int64_t) * (b.N + 1), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(b.col, cl.data(), sizeof(int32_t) * b.M, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(b.cval, cv.data(), sizeof(double) * b.M, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(b.cs, csv.data(), sizeof(double) * b.N, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(b.ct, ctv.data(), sizeof(double) * b.N, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(b.S, 0, sizeof(PcgState) * count);
  if (e == cudaSuccess) e = cudaMemset(b.C, 0, sizeof(StepCounters));
  if (e == cudaSuccess)
    e = cudaHostAlloc((void**)&b.h_ctr, sizeof(StepCounters) + sizeof(int), cudaHostAllocDefault);
  if (e != cudaSuccess) return bail(e, "upload");
  // the work list's instance order: largest row degree first, then larger
  // instances first (longest work items early)
  {
    std::vector<int> ord(count);
    std::vector<int64_t> maxdeg(count, 0);
    for (int i = 0; i < count; ++i) {
      ord[i] = i;
      const HostGraph& g = b.hg[i];
      for (int64_t r = 0; r < g.nt; ++r) maxdeg[i] = std::max(maxdeg[i], g.rp[r + 1] - g.rp[r]);
    }
    std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) {
      return maxdeg[x] != maxdeg[y] ? maxdeg[x] > maxdeg[y] : b.hg[x].nt > b.hg[y].nt;
    });
    e = cudaMemcpy(b.order, ord.data(), sizeof(int) * count, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return bail(e, "upload");
  }
  // hub rows: more entries than 32 threads can cover in 16 passes
  b.heavy_deg = kHubDeg;
  {
    int dev = 0, sms = 152, per_sm = 4;
    if (cudaGetDevice(&dev) == cudaSuccess)
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kb_update_r, kBT, 0);
    b.work_grid = std::max(1, sms) * std::max(1, std::min(per_sm, 8));
  }
  e = autotune(b);
  if (e != cudaSuccess) return bail(e, "autotune");
  *out = h;
  return PIRMCUT_OK;
}

pirmcut_status pirmcut_batch_solve(pirmcut_batch* h, int T, const double* eps, pirmcut_step_info* infos) {
  using namespace pirmcut;
  if (!h) return bfail(nullptr, PIRMCUT_EINVAL, "batch is NULL");
  Batch& b = h->b;
  if (T < 0 || (T > 0 && !eps)) return bfail(h, PIRMCUT_EINVAL, "bad T or eps");
  for (int l = 0; l < T; ++l)
    if (!(eps[l] > 0.0) || !std::isfinite(eps[l])) return bfail(h, PIRMCUT_EINVAL, "every eps must be > 0");
  if (b.eps_cap < T || b.rec_cap < T + 1) {
    if (b.eps_list) cudaFree(b.eps_list);
    if (b.recs) cudaFree(b.recs);
    if (b.h_recs) cudaFreeHost(b.h_recs);
    b.eps_list = nullptr;
    b.recs = nullptr;
    b.h_recs = nullptr;
    int cap = 64;
    while (cap < T + 1) cap *= 2;
    BCK(h, cudaMalloc(&b.eps_list, sizeof(double) * cap), "cudaMalloc");
    BCK(h, cudaMalloc(&b.recs, sizeof(StepRec) * cap * b.count), "cudaMalloc");
    BCK(h, cudaHostAlloc((void**)&b.h_recs, sizeof(StepRec) * cap * b.count, cudaHostAllocDefault), "cudaHostAlloc");
    b.eps_cap = cap;
    b.rec_cap = cap;
    if (b.g_init) cudaGraphExecDestroy(b.g_init);
    if (b.g_step) cudaGraphExecDestroy(b.g_step);
    b.g_init = b.g_step = nullptr;
  }
  const bool graphs = b.opt.graph_launch != 0;
  if (graphs && !b.g_init) BCK(h, build_bgraph(b, true, &b.g_init), "building the batch x0 graph");
  if (graphs && !b.g_step) BCK(h, build_bgraph(b, false, &b.g_step), "building the batch step graph");
  if (T > 0) BCK(h, cudaMemcpyAsync(b.eps_list, eps, sizeof(double) * T, cudaMemcpyHostToDevice, b.stream), "eps");
  std::memset(b.h_ctr, 0, sizeof(StepCounters));
  BCK(h, cudaMemcpyAsync(b.C, b.h_ctr, sizeof(StepCounters), cudaMemcpyHostToDevice, b.stream), "counters");
  while (b.events.size() < size_t(T) + 2) {
    cudaEvent_t ev;
    BCK(h, cudaEventCreate(&ev), "cudaEventCreate");
    b.events.push_back(ev);
  }
  BCK(h, cudaEventRecord(b.events[0], b.stream), "event");
  int64_t stream_kernels = 0;
  for (int k = 0; k <= T; ++k) {
    if (graphs) {
      BCK(h, cudaGraphLaunch(k == 0 ? b.g_init : b.g_step, b.stream), "graph launch");
    } else {
      // the same kernels from the host: PCG iterations in chunks of 8, the
      // number of active instances read back between chunks; iterations queued
      // after the last instance stopped are no-ops (the kernels test the flags)
      cudaGraphConditionalHandle none{};
      int* h_active = reinterpret_cast<int*>(b.h_ctr + 1);
      stream_kernels += enqueue_bstep(b, b.stream, k == 0, none, 0, 0);
      for (int guard = 0;; ++guard) {
        for (int j = 0; j < 8; ++j) stream_kernels += enqueue_bstep(b, b.stream, k == 0, none, 0, 1);
        BCK(h, cudaMemcpyAsync(h_active, b.active, sizeof(int), cudaMemcpyDeviceToHost, b.stream), "active");
        BCK(h, cudaStreamSynchronize(b.stream), "batch step");
        if (*h_active == 0 || guard > b.opt.pcg_max_iter / 8 + 2) break;
      }
      stream_kernels += enqueue_bstep(b, b.stream, k == 0, none, 0, 2);
      BCK(h, cudaGetLastError(), "batch step launch");
    }
    BCK(h, cudaEventRecord(b.events[k + 1], b.stream), "event");
  }
  b.launches += stream_kernels;
  BCK(h, cudaMemcpyAsync(b.h_recs, b.recs, sizeof(StepRec) * b.rec_cap * b.count, cudaMemcpyDeviceToHost, b.stream), "records");
  BCK(h, cudaStreamSynchronize(b.stream), "batch solve");
  b.x_set = true;
  pirmcut_status worst = PIRMCUT_OK;
  for (int k = 0; k <= T; ++k) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, b.events[k], b.events[k + 1]);
    int64_t it_total = 0;
    for (int i = 0; i < b.count; ++i) {
      const StepRec& r = b.h_recs[size_t(i) * b.rec_cap + k];
      pirmcut_step_info info;
      info.step = r.step;
      info.pcg_iters = r.iters;
      info.eps = r.eps;
      info.rel_residual = r.bb > 0.0 ? std::sqrt(r.rr / r.bb) : 0.0;
      info.x_min = r.xmin;
      info.x_max = r.xmax;
      info.cut_value = r.cut;
      info.ms = ms;
      int st = r.status;
      if (st == PIRMCUT_OK && r.bb > 0.0 && !(r.rr <= b.opt.pcg_tol * b.opt.pcg_tol * r.bb)) st = PIRMCUT_ENOCONV;
      info.status = st;
      info.refinements = 0;
      info.objective = r.obj;
      info.flow_value = r.flow;
      if (infos) infos[size_t(i) * (T + 1) + k] = info;
      it_total = std::max<int64_t>(it_total, r.iters);
      if (st == PIRMCUT_ENUMERIC) worst = PIRMCUT_ENUMERIC;
      else if (st == PIRMCUT_ENOCONV && worst == PIRMCUT_OK) worst = PIRMCUT_ENOCONV;
    }
    if (graphs) b.launches += 8 + 4 * (it_total + 1);
  }
  if (worst != PIRMCUT_OK) return bfail(h, worst, "an instance did not converge or broke down");
  return PIRMCUT_OK;
}

// One instance's view as a CSR context for the sweep cut.
static pirmcut_status batch_view(pirmcut_batch* h, int index) {
  using namespace pirmcut;
  Batch& b = h->b;
  const BInst& in = b.h_insts[index];
  const HostGraph& g = b.hg[index];
  Ctx& v = b.view;
  v.nt = in.nt;
  v.format = PIRMCUT_FORMAT_CSR;
  v.group = b.G;
  v.rp = b.rp + in.base;
  v.col = b.col;
  v.cval = b.cval;
  v.cs = b.cs + in.base;
  v.ct = b.ct + in.base;
  v.x = b.x + in.base;
  v.C = b.C;
  v.recs = b.recs;
  v.stream = b.stream;
  v.hg.sum_cs = g.sum_cs;
  v.hg.c_st = g.c_st;
  v.hg.s = g.s;
  v.hg.t = g.t;
  v.hg.n = g.n;
  return PIRMCUT_OK;
}

pirmcut_status pirmcut_batch_cut(pirmcut_batch* h, int index, uint8_t* side, double* value, double* tau) {
  using namespace pirmcut;
  if (!h) return bfail(nullptr, PIRMCUT_EINVAL, "batch is NULL");
  Batch& b = h->b;
  if (index < 0 || index >= b.count) return bfail(h, PIRMCUT_EINVAL, "index out of range");
  if (!b.x_set) return bfail(h, PIRMCUT_EINVAL, "solve first");
  batch_view(h, index);
  Ctx& v = b.view;
  // the sweep scratch is sized for the largest instance
  int64_t mx = 0;
  for (const BInst& in : b.h_insts) mx = std::max(mx, in.nt);
  if (v.sw.cap < mx) {
    const int64_t keep = v.nt;
    v.nt = mx;
    BCK(h, sweep_alloc(v), "sweep buffers");
    v.nt = keep;
  }
  BCK(h, set_heavy_rows(v, b.hg[index].rp.data()), "sweep rows");  // this instance's hubs
  int kernels = 0;
  BCK(h, enqueue_sweep(v, b.stream, false, &kernels), "sweep");
  b.launches += kernels;
  double res[4];
  BCK(h, cudaMemcpyAsync(res, v.sw.result, sizeof(res), cudaMemcpyDeviceToHost, b.stream), "result");
  BCK(h, cudaStreamSynchronize(b.stream), "cut");
  if (side) {
    std::vector<uint8_t> sr(size_t(v.nt));
    BCK(h, cudaMemcpy(sr.data(), v.sw.side_red, size_t(v.nt), cudaMemcpyDeviceToHost), "side");
    const HostGraph& g = b.hg[index];
    for (int64_t i = 0; i < v.nt; ++i) side[original_index(i, g.s, g.t)] = sr[i];
    side[g.s] = 1;
    side[g.t] = 0;
  }
  if (value) *value = res[1];
  if (tau) *tau = res[2];
  return PIRMCUT_OK;
}

pirmcut_status pirmcut_batch_get_x(pirmcut_batch* h, int index, double* x) {
  using namespace pirmcut;
  if (!h) return bfail(nullptr, PIRMCUT_EINVAL, "batch is NULL");
  Batch& b = h->b;
  if (index < 0 || index >= b.count || !x) return bfail(h, PIRMCUT_EINVAL, "bad index or x");
  if (!b.x_set) return bfail(h, PIRMCUT_EINVAL, "solve first");
  const BInst& in = b.h_insts[index];
  const HostGraph& g = b.hg[index];
  if (b.xfull_cap < g.n) {
    if (b.xfull) cudaFree(b.xfull);
    b.xfull = nullptr;
    BCK(h, cudaMalloc(&b.xfull, sizeof(double) * g.n), "cudaMalloc");
    b.xfull_cap = g.n;
  }
  kb_scatter_x<<<grid_for(in.nt), 256, 0, b.stream>>>(in.nt, in.base, g.s, g.t, b.x, b.xfull);
  BCK(h, cudaGetLastError(), "scatter");
  BCK(h, cudaMemcpyAsync(x, b.xfull, sizeof(double) * g.n, cudaMemcpyDeviceToHost, b.stream), "get_x");
  BCK(h, cudaStreamSynchronize(b.stream), "get_x");
  return PIRMCUT_OK;
}

pirmcut_status pirmcut_batch_info(const pirmcut_batch* h, int64_t* total_rows, int64_t* total_nnz,
                                  int* threads_per_row, int* tile_rows, int* tiles,
                                  int64_t* medium_deg) {
  if (!h) return PIRMCUT_EINVAL;
  const pirmcut::Batch& b = h->b;
  if (total_rows) *total_rows = b.N;
  if (total_nnz) *total_nnz = b.M;
  if (threads_per_row) *threads_per_row = b.G;
  if (tile_rows) *tile_rows = b.tile_rows;
  if (tiles) *tiles = int(b.h_tiles.size());
  if (medium_deg) *medium_deg = b.mid_deg;
  return PIRMCUT_OK;
}

int64_t pirmcut_batch_kernel_launches(const pirmcut_batch* h) { return h ? h->b.launches : 0; }

void pirmcut_batch_destroy(pirmcut_batch* h) {
  if (!h) return;
  if (h->b.stream) cudaStreamSynchronize(h->b.stream);
  pirmcut::free_batch(h->b);
  delete h;
}

}  // extern "C"
