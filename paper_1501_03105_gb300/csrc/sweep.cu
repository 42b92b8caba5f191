// Sweep cut over x (Section 3.3; Algorithm 1, step 6) on the GPU.
//
//  1. keys: x mapped to 64-bit integers whose ascending order is x descending
//     (-0 folded into +0); payload = reduced vertex index.
//  2. stable LSD radix sort, 8 passes of 8 bits (per-tile histograms,
//     per-digit scans, stable tile-local ranking with warp match masks and a
//     shared-memory staging so that every digit's run is written coalesced).
//     Stability keeps equal x in ascending vertex order.
//  3. rank[v] = sweep position of v.
//  4. delta_v = c(v,t) - c(s,v) + sum over non-terminal neighbours u of
//     c(u,v) * (+1 if v comes before u, -1 otherwise): the change of the cut
//     when v moves from the sink side to the source side.
//  5. cut(k) = cut(0) + sum_{i<k} delta_(i) by a deterministic tiled FP64 scan;
//     argmin over k = 0, k = n~ and every k with x_(k) > x_(k+1) (1-based),
//     least value first, then least k.
//  6. side, threshold, and the exact FP64 cut value of the chosen side.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <utility>
#include <vector>

#include "ctx.h"

namespace pirmcut {

namespace {

constexpr int RS_THREADS = 256;
constexpr int RS_ITEMS = 8;
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;   // keys per sort tile
constexpr int SC_ITEMS = 8;
constexpr int SC_TILE = kThreads * SC_ITEMS;     // positions per scan tile

__device__ __forceinline__ int64_t gtid() { return int64_t(blockIdx.x) * blockDim.x + threadIdx.x; }
__device__ __forceinline__ int64_t gstride() { return int64_t(gridDim.x) * blockDim.x; }

__device__ __forceinline__ uint64_t desc_key(double x) {
  x = x + 0.0;  // -0.0 -> +0.0 so that equal values get equal keys
  uint64_t b = (uint64_t)__double_as_longlong(x);
  b = (b & 0x8000000000000000ull) ? ~b : (b | 0x8000000000000000ull);  // ascending in x
  return ~b;                                                             // descending in x
}

// exclusive scan of one uint32 per thread over a block of 256 threads
__device__ __forceinline__ uint32_t block_excl_scan_u32(uint32_t v, uint32_t* total) {
  __shared__ uint32_t sw[8];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) sw[wid] = inc;
  __syncthreads();
  uint32_t woff = 0, tot = 0;
  for (int w = 0; w < 8; ++w) {
    if (w < wid) woff += sw[w];
    tot += sw[w];
  }
  __syncthreads();
  if (total) *total = tot;
  return woff + inc - v;
}

// exclusive scan of one double per thread over the block (fixed order)
__device__ __forceinline__ double block_excl_scan_f64(double v, double* total) {
  __shared__ double sw[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  double inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const double t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) sw[wid] = inc;
  __syncthreads();
  double woff = 0.0, tot = 0.0;
  for (int w = 0; w < nw; ++w) {
    if (w < wid) woff += sw[w];
    tot += sw[w];
  }
  __syncthreads();
  if (total) *total = tot;
  return woff + (inc - v);
}

__global__ void k_sweep_init(int64_t nt, const double* __restrict__ x, uint64_t* __restrict__ keys,
                             uint32_t* __restrict__ vals) {
  for (int64_t i = gtid(); i < nt; i += gstride()) {
    keys[i] = desc_key(x[i]);
    vals[i] = (uint32_t)i;
  }
}

__global__ void __launch_bounds__(RS_THREADS)
k_radix_hist(const uint64_t* __restrict__ keys, int64_t n, int shift, uint32_t* __restrict__ hist,
             int nblocks) {
  __shared__ uint32_t h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = int64_t(blockIdx.x) * RS_TILE;
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int j = 0; j < RS_ITEMS; ++j) {
    const int64_t i = base + j * RS_THREADS + threadIdx.x;
    const bool valid = i < n;
    const uint32_t d = valid ? (uint32_t(keys[i] >> shift) & 255u) : 256u;
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    if (valid && lane == __ffs(peers) - 1) atomicAdd(&h[d], (uint32_t)__popc(peers));
  }
  __syncthreads();
  hist[threadIdx.x * nblocks + blockIdx.x] = h[threadIdx.x];
}

// block d: exclusive scan of hist[d * nblocks .. +nblocks) in place; total -> tot[d]
__global__ void __launch_bounds__(1024)
k_radix_scan(uint32_t* __restrict__ hist, int nblocks, uint32_t* __restrict__ tot) {
  __shared__ uint32_t sw[32];
  uint32_t* h = hist + size_t(blockIdx.x) * nblocks;
  const int per = (nblocks + 1023) / 1024;
  const int lo = threadIdx.x * per;
  const int hi = min(nblocks, lo + per);
  uint32_t s = 0;
  for (int b = lo; b < hi; ++b) s += h[b];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t inc = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) sw[wid] = inc;
  __syncthreads();
  uint32_t woff = 0, all = 0;
  for (int w = 0; w < 32; ++w) {
    if (w < wid) woff += sw[w];
    all += sw[w];
  }
  uint32_t run = woff + inc - s;
  for (int b = lo; b < hi; ++b) {
    const uint32_t c = h[b];
    h[b] = run;
    run += c;
  }
  if (threadIdx.x == 0) tot[blockIdx.x] = all;
}

__global__ void __launch_bounds__(RS_THREADS)
k_radix_scatter(const uint64_t* __restrict__ kin, const uint32_t* __restrict__ vin,
                uint64_t* __restrict__ kout, uint32_t* __restrict__ vout, int64_t n, int shift,
                const uint32_t* __restrict__ hist, const uint32_t* __restrict__ tot, int nblocks) {
  __shared__ uint32_t s_base[256];
  __shared__ uint32_t s_warp[8][256];
  __shared__ uint32_t s_run[256];
  __shared__ uint32_t s_start[256];
  __shared__ uint64_t s_keys[RS_TILE];
  __shared__ uint32_t s_vals[RS_TILE];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t base = int64_t(blockIdx.x) * RS_TILE;
  {
    const uint32_t dig_off = block_excl_scan_u32(tot[tid], nullptr);
    s_base[tid] = dig_off + hist[size_t(tid) * nblocks + blockIdx.x];
  }
  s_run[tid] = 0;
#pragma unroll
  for (int w = 0; w < 8; ++w) s_warp[w][tid] = 0;
  uint64_t k[RS_ITEMS];
  uint32_t v[RS_ITEMS], d[RS_ITEMS], lr[RS_ITEMS];
#pragma unroll
  for (int j = 0; j < RS_ITEMS; ++j) {
    const int64_t i = base + j * RS_THREADS + tid;
    const bool valid = i < n;
    k[j] = valid ? kin[i] : 0ull;
    v[j] = valid ? vin[i] : 0u;
    d[j] = valid ? (uint32_t(k[j] >> shift) & 255u) : 256u;
  }
  __syncthreads();
  // stable ranking: round j holds the tile's keys j*256 .. j*256+255 in order
#pragma unroll
  for (int j = 0; j < RS_ITEMS; ++j) {
    const uint32_t dj = d[j];
    const unsigned peers = __match_any_sync(0xffffffffu, dj);
    const uint32_t below = __popc(peers & ((1u << lane) - 1u));
    if (dj < 256u && lane == __ffs(peers) - 1) s_warp[warp][dj] = __popc(peers);
    __syncthreads();
    uint32_t run = s_run[tid];
#pragma unroll
    for (int w = 0; w < 8; ++w) {
      const uint32_t cnt = s_warp[w][tid];
      s_warp[w][tid] = run;
      run += cnt;
    }
    s_run[tid] = run;
    __syncthreads();
    lr[j] = (dj < 256u) ? s_warp[warp][dj] + below : 0u;
    __syncthreads();
#pragma unroll
    for (int w = 0; w < 8; ++w) s_warp[w][tid] = 0;
    __syncthreads();
  }
  s_start[tid] = block_excl_scan_u32(s_run[tid], nullptr);
  __syncthreads();
#pragma unroll
  for (int j = 0; j < RS_ITEMS; ++j) {
    if (d[j] < 256u) {
      const uint32_t pos = s_start[d[j]] + lr[j];
      s_keys[pos] = k[j];
      s_vals[pos] = v[j];
    }
  }
  __syncthreads();
  const int64_t rem = n - base;
  const int64_t valid = rem < RS_TILE ? rem : RS_TILE;
#pragma unroll
  for (int j = 0; j < RS_ITEMS; ++j) {
    const int p = j * RS_THREADS + tid;
    if (p < valid) {
      const uint64_t key = s_keys[p];
      const uint32_t dd = uint32_t(key >> shift) & 255u;
      const uint32_t dst = s_base[dd] + (uint32_t(p) - s_start[dd]);
      kout[dst] = key;
      vout[dst] = s_vals[p];
    }
  }
}

__global__ void k_rank(int64_t nt, const uint32_t* __restrict__ order, int32_t* __restrict__ rank) {
  for (int64_t k = gtid(); k < nt; k += gstride()) rank[order[k]] = (int32_t)k;
}

template <int K>
__global__ void __launch_bounds__(kThreads)
k_delta_dia(DiaDesc d, const double* __restrict__ c, const double* __restrict__ cs,
            const double* __restrict__ ct, const int32_t* __restrict__ rank,
            double* __restrict__ delta) {
  const int64_t nt = d.nt;
  for (int64_t i = gtid(); i < nt; i += gstride()) {
    const int32_t ri = rank[i];
    double acc = ct[i] - cs[i];
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int64_t o = d.off[k];
      if (i + o < nt) {
        const double w = c[k * nt + i];
        acc += (ri < rank[i + o]) ? w : -w;
      }
      if (i >= o) {
        const double w = c[k * nt + i - o];
        acc += (ri < rank[i - o]) ? w : -w;
      }
    }
    delta[i] = acc;
  }
}

template <int G>
__global__ void __launch_bounds__(kThreads)
k_delta_csr(int64_t nt, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
            const double* __restrict__ c, const double* __restrict__ cs,
            const double* __restrict__ ct, const int32_t* __restrict__ rank,
            double* __restrict__ delta, int64_t heavy_deg, const int32_t* __restrict__ heavy,
            int light_blocks) {
  if (int(blockIdx.x) >= light_blocks) {  // one heavy row per block
    const int64_t i = heavy[blockIdx.x - light_blocks];
    const int32_t ri = rank[i];
    double acc = 0.0;
    for (int64_t e = rp[i] + threadIdx.x; e < rp[i + 1]; e += blockDim.x) {
      const double w = c[e];
      acc += (ri < rank[col[e]]) ? w : -w;
    }
    double v[1] = {acc};
    block_sum<1>(v);
    if (threadIdx.x == 0) delta[i] = (ct[i] - cs[i]) + v[0];
    return;
  }
  const int lane = threadIdx.x % G;
  const unsigned mask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << ((threadIdx.x & 31) / G * G));
  const int64_t ng = int64_t(light_blocks) * blockDim.x / G;
  for (int64_t i = gtid() / G; i < nt; i += ng) {
    if (rp[i + 1] - rp[i] > heavy_deg) continue;  // the group agrees: same row
    const int32_t ri = rank[i];
    double acc = 0.0;
    for (int64_t e = rp[i] + lane; e < rp[i + 1]; e += G) {
      const double w = c[e];
      acc += (ri < rank[col[e]]) ? w : -w;
    }
    acc = group_sum<G>(acc, mask);
    if (lane == 0) delta[i] = (ct[i] - cs[i]) + acc;
  }
}

// per scan tile: sum of delta in sweep order
__global__ void __launch_bounds__(kThreads)
k_tile_sum(int64_t nt, const uint32_t* __restrict__ order, const double* __restrict__ delta,
           double* __restrict__ blk) {
  const int64_t base = int64_t(blockIdx.x) * SC_TILE + int64_t(threadIdx.x) * SC_ITEMS;
  double s = 0.0;
#pragma unroll
  for (int j = 0; j < SC_ITEMS; ++j) {
    const int64_t k = base + j;
    if (k < nt) s += delta[order[k]];
  }
  double v[1] = {s};
  block_sum<1>(v);
  if (threadIdx.x == 0) blk[blockIdx.x] = v[0];
}

// exclusive scan of the tile sums (one block)
__global__ void __launch_bounds__(1024) k_tile_scan(int ntiles, double* __restrict__ blk) {
  const int per = (ntiles + 1023) / 1024;
  const int lo = threadIdx.x * per, hi = min(ntiles, lo + per);
  double s = 0.0;
  for (int b = lo; b < hi; ++b) s += blk[b];
  double run = block_excl_scan_f64(s, nullptr);
  for (int b = lo; b < hi; ++b) {
    const double c = blk[b];
    blk[b] = run;
    run += c;
  }
}

struct ArgMin {
  double v;
  int64_t k;
};
__device__ __forceinline__ ArgMin amin(ArgMin a, ArgMin b) {
  if (b.v < a.v || (b.v == a.v && b.k < a.k)) return b;
  return a;
}

// per tile: cut(k+1) for the tile's positions k, eligible ones only; the last
// tile to finish reduces the tile minima (with k = 0 as the first candidate).
__global__ void __launch_bounds__(kThreads)
k_tile_argmin(int64_t nt, const uint32_t* __restrict__ order, const double* __restrict__ delta,
              const double* __restrict__ x, const double* __restrict__ blk, double cut0,
              double* __restrict__ bv, int64_t* __restrict__ bk, unsigned int* counter,
              double* __restrict__ result) {
  __shared__ double sv[32];
  __shared__ int64_t sk[32];
  __shared__ unsigned int s_last;
  const int64_t base = int64_t(blockIdx.x) * SC_TILE + int64_t(threadIdx.x) * SC_ITEMS;
  double dl[SC_ITEMS];
  double s = 0.0;
#pragma unroll
  for (int j = 0; j < SC_ITEMS; ++j) {
    const int64_t k = base + j;
    dl[j] = (k < nt) ? delta[order[k]] : 0.0;
    s += dl[j];
  }
  double run = cut0 + blk[blockIdx.x] + block_excl_scan_f64(s, nullptr);
  ArgMin best{INFINITY, INT64_MAX};
#pragma unroll
  for (int j = 0; j < SC_ITEMS; ++j) {
    const int64_t k = base + j;
    run += dl[j];
    if (k < nt) {
      // prefix of length k+1 ends between positions k and k+1
      const bool elig = (k + 1 == nt) || (x[order[k]] > x[order[k + 1]]);
      if (elig) best = amin(best, ArgMin{run, k + 1});
    }
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    ArgMin other{__shfl_down_sync(0xffffffffu, best.v, o),
                 (int64_t)__shfl_down_sync(0xffffffffu, (long long)best.k, o)};
    best = amin(best, other);
  }
  if (lane == 0) {
    sv[wid] = best.v;
    sk[wid] = best.k;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) best = amin(best, ArgMin{sv[w], sk[w]});
    bv[blockIdx.x] = best.v;
    bk[blockIdx.x] = best.k;
    __threadfence();
    s_last = (atomicAdd(counter, 1u) == gridDim.x - 1) ? 1u : 0u;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  // the last tile's block reduces the tile minima (amin is associative and
  // breaks ties by k, so the result does not depend on the order)
  ArgMin all{INFINITY, INT64_MAX};
  if (threadIdx.x == 0) all = ArgMin{cut0, 0};
  for (unsigned int b = threadIdx.x; b < gridDim.x; b += blockDim.x)
    all = amin(all, ArgMin{__ldcg(bv + b), __ldcg(bk + b)});
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    ArgMin other{__shfl_down_sync(0xffffffffu, all.v, o),
                 (int64_t)__shfl_down_sync(0xffffffffu, (long long)all.k, o)};
    all = amin(all, other);
  }
  if (lane == 0) {
    sv[wid] = all.v;
    sk[wid] = all.k;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  for (int w = 1; w < (int)(blockDim.x >> 5); ++w) all = amin(all, ArgMin{sv[w], sk[w]});
  *counter = 0u;
  result[0] = all.v;
  result[3] = (double)all.k;
  const double hi = all.k == 0 ? 1.0 : x[order[all.k - 1]];
  const double lo = all.k == nt ? 0.0 : x[order[all.k]];
  result[2] = 0.5 * (hi + lo);
}

__global__ void k_side(int64_t nt, const uint32_t* __restrict__ order, const double* __restrict__ result,
                       uint8_t* __restrict__ side) {
  const int64_t ks = (int64_t)result[3];
  for (int64_t k = gtid(); k < nt; k += gstride()) side[order[k]] = k < ks ? 1 : 0;
}

struct CutArgs {
  const double* cs;
  const double* ct;
  const uint8_t* side;
  double c_st;
  double* partials;
  unsigned int* counter;
  double* result;
  const StepCounters* C;
  StepRec* recs;
  int record;
};

__device__ __forceinline__ void cut_finish(const CutArgs& a, double acc) {
  double v[1] = {acc}, tot[1];
  if (grid_sum<1>(v, a.partials, a.counter, tot) && threadIdx.x == 0) {
    const double val = a.c_st + tot[0];
    a.result[1] = val;
    if (a.record && a.C->rec_idx > 0) a.recs[a.C->rec_idx - 1].cut = val;
  }
}

template <int K>
__global__ void __launch_bounds__(kThreads)
k_cut_dia(DiaDesc d, const double* __restrict__ c, CutArgs a) {
  const int64_t nt = d.nt;
  double acc = 0.0;
  for (int64_t i = gtid(); i < nt; i += gstride()) {
    const uint8_t si = a.side[i];
    double t = si ? a.ct[i] : a.cs[i];
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int64_t j = i + d.off[k];
      if (j < nt && a.side[j] != si) t += c[k * nt + i];
    }
    acc += t;
  }
  cut_finish(a, acc);
}

template <int G>
__global__ void __launch_bounds__(kThreads)
k_cut_csr(int64_t nt, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
          const double* __restrict__ c, CutArgs a, int64_t heavy_deg,
          const int32_t* __restrict__ heavy, int light_blocks) {
  double acc = 0.0;
  if (int(blockIdx.x) >= light_blocks) {  // one heavy row per block
    const int64_t i = heavy[blockIdx.x - light_blocks];
    const uint8_t si = a.side[i];
    for (int64_t e = rp[i] + threadIdx.x; e < rp[i + 1]; e += blockDim.x) {
      const int32_t j = col[e];
      if (j > i && a.side[j] != si) acc += c[e];
    }
    if (threadIdx.x == 0) acc += si ? a.ct[i] : a.cs[i];
  } else {
    const int lane = threadIdx.x % G;
    const unsigned mask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << ((threadIdx.x & 31) / G * G));
    const int64_t ng = int64_t(light_blocks) * blockDim.x / G;
    for (int64_t i = gtid() / G; i < nt; i += ng) {
      if (rp[i + 1] - rp[i] > heavy_deg) continue;
      const uint8_t si = a.side[i];
      double t = 0.0;
      for (int64_t e = rp[i] + lane; e < rp[i + 1]; e += G) {
        const int32_t j = col[e];
        if (j > i && a.side[j] != si) t += c[e];
      }
      t = group_sum<G>(t, mask);
      if (lane == 0) acc += t + (si ? a.ct[i] : a.cs[i]);
    }
  }
  cut_finish(a, acc);
}

__global__ void k_side_full(int64_t nt, int32_t s, int32_t t, const uint8_t* __restrict__ sr,
                            uint8_t* __restrict__ sf) {
  const int64_t a = s < t ? s : t, b = s < t ? t : s;
  for (int64_t i = gtid(); i < nt; i += gstride()) {
    int64_t v = i;
    if (v >= a) ++v;
    if (v >= b) ++v;
    sf[v] = sr[i];
  }
  if (gtid() == 0) {
    sf[s] = 1;
    sf[t] = 0;
  }
}

#define SW_DISPATCH_K(KVAR, CALL) \
  switch (KVAR) {                 \
    case 1: { constexpr int KK = 1; CALL; } break; \
    case 2: { constexpr int KK = 2; CALL; } break; \
    case 3: { constexpr int KK = 3; CALL; } break; \
    case 4: { constexpr int KK = 4; CALL; } break; \
    case 5: { constexpr int KK = 5; CALL; } break; \
    case 6: { constexpr int KK = 6; CALL; } break; \
    case 7: { constexpr int KK = 7; CALL; } break; \
    default: { constexpr int KK = 8; CALL; } break; \
  }
#define SW_DISPATCH_G(GVAR, CALL) \
  switch (GVAR) {                 \
    case 1: { constexpr int GG = 1; CALL; } break; \
    case 2: { constexpr int GG = 2; CALL; } break; \
    case 4: { constexpr int GG = 4; CALL; } break; \
    case 8: { constexpr int GG = 8; CALL; } break; \
    case 16: { constexpr int GG = 16; CALL; } break; \
    default: { constexpr int GG = 32; CALL; } break; \
  }

}  // namespace

cudaError_t sweep_alloc(Ctx& c) {
  SweepBuf& b = c.sw;
  if (b.cap == c.nt) return cudaSuccess;
  sweep_free(c);
  const int64_t nt = c.nt;
  b.nblocks_sort = int((nt + RS_TILE - 1) / RS_TILE);
  b.ntiles = int((nt + SC_TILE - 1) / SC_TILE);
  cudaError_t e = cudaSuccess;
  auto A = [&](void** p, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(p, bytes);
  };
  A((void**)&b.keys[0], sizeof(uint64_t) * nt);
  A((void**)&b.keys[1], sizeof(uint64_t) * nt);
  A((void**)&b.vals[0], sizeof(uint32_t) * nt);
  A((void**)&b.vals[1], sizeof(uint32_t) * nt);
  A((void**)&b.hist, sizeof(uint32_t) * 256 * size_t(b.nblocks_sort));
  A((void**)&b.digit_tot, sizeof(uint32_t) * 256);
  A((void**)&b.rank, sizeof(int32_t) * nt);
  A((void**)&b.delta, sizeof(double) * nt);
  A((void**)&b.blk, sizeof(double) * ((size_t(b.ntiles) + kMaxBlocks) * 2 + kHeavyRowsMax));
  A((void**)&b.blk_k, sizeof(int64_t) * (size_t(b.ntiles) + 1));
  A((void**)&b.side_red, nt);
  A((void**)&b.result, sizeof(double) * 4 + sizeof(unsigned int) * 8);
  if (e == cudaSuccess) e = cudaMemset(b.result, 0, sizeof(double) * 4 + sizeof(unsigned int) * 8);
  if (e != cudaSuccess) {
    sweep_free(c);
    return e;
  }
  b.cap = nt;
  return e;
}

// Rows with more than max(512, 16 x mean) entries, at most kHeavyRowsMax of
// them (the longest), listed in ascending order.
cudaError_t set_heavy_rows(Ctx& c, const int64_t* rp) {
  const int64_t nt = c.nt;
  const int64_t mean = nt ? (rp[nt] - rp[0]) / nt : 0;
  int64_t thr = std::max<int64_t>(512, 16 * mean);
  std::vector<std::pair<int64_t, int32_t>> rows;  // (degree, row)
  for (int64_t i = 0; i < nt; ++i) {
    const int64_t d = rp[i + 1] - rp[i];
    if (d > thr) rows.push_back({d, int32_t(i)});
  }
  if (int64_t(rows.size()) > kHeavyRowsMax) {
    std::nth_element(rows.begin(), rows.begin() + kHeavyRowsMax, rows.end(),
                     [](const std::pair<int64_t, int32_t>& x, const std::pair<int64_t, int32_t>& y) {
                       return x.first > y.first;
                     });
    thr = rows[kHeavyRowsMax].first;  // heavy: strictly longer than the first one left out
    std::vector<std::pair<int64_t, int32_t>> keep;
    for (const auto& r : rows)
      if (r.first > thr) keep.push_back(r);
    rows.swap(keep);
  }
  std::vector<int32_t> ids;
  for (const auto& r : rows) ids.push_back(r.second);
  std::sort(ids.begin(), ids.end());
  if (!c.heavy) {
    cudaError_t e = cudaMalloc((void**)&c.heavy, sizeof(int32_t) * kHeavyRowsMax);
    if (e != cudaSuccess) return e;
  }
  c.n_heavy = int(ids.size());
  c.heavy_deg = thr;
  if (ids.empty()) return cudaSuccess;
  return cudaMemcpy(c.heavy, ids.data(), sizeof(int32_t) * ids.size(), cudaMemcpyHostToDevice);
}

void sweep_free(Ctx& c) {
  SweepBuf& b = c.sw;
  void* ps[] = {b.keys[0], b.keys[1], b.vals[0], b.vals[1], b.hist, b.digit_tot, b.rank,
                b.delta, b.blk, b.blk_k, b.side_red, b.result};
  for (void* p : ps)
    if (p) cudaFree(p);
  b = SweepBuf();
}

// Enqueue the whole sweep on st; writes result[0..3] = {prefix value, exact
// value, tau, k}, the reduced side vector, and (when record) the cut of the
// last step record.  Tile counts follow c.nt; the scratch may be larger.
cudaError_t enqueue_sweep(Ctx& c, cudaStream_t st, bool record, int* nodes) {
  SweepBuf& b = c.sw;
  const int64_t nt = c.nt;
  const int nblocks_sort = int((nt + RS_TILE - 1) / RS_TILE);
  const int ntiles = int((nt + SC_TILE - 1) / SC_TILE);
  int n_nodes = 0;
  unsigned int* counters = reinterpret_cast<unsigned int*>(b.result + 4);
  k_sweep_init<<<grid_for(nt), kThreads, 0, st>>>(nt, c.x, b.keys[0], b.vals[0]);
  ++n_nodes;
  int cur = 0;
  for (int pass = 0; pass < 8; ++pass) {
    const int shift = 8 * pass;
    k_radix_hist<<<nblocks_sort, RS_THREADS, 0, st>>>(b.keys[cur], nt, shift, b.hist, nblocks_sort);
    k_radix_scan<<<256, 1024, 0, st>>>(b.hist, nblocks_sort, b.digit_tot);
    k_radix_scatter<<<nblocks_sort, RS_THREADS, 0, st>>>(b.keys[cur], b.vals[cur], b.keys[cur ^ 1],
                                                         b.vals[cur ^ 1], nt, shift, b.hist,
                                                         b.digit_tot, nblocks_sort);
    n_nodes += 3;
    cur ^= 1;
  }
  const uint32_t* order = b.vals[cur];
  k_rank<<<grid_for(nt), kThreads, 0, st>>>(nt, order, b.rank);
  ++n_nodes;
  const int rgrid = grid_for(c.format == PIRMCUT_FORMAT_DIA ? nt : nt * c.group);
  if (c.format == PIRMCUT_FORMAT_DIA) {
    SW_DISPATCH_K(c.K, (k_delta_dia<KK><<<rgrid, kThreads, 0, st>>>(c.dd, c.cdia, c.cs, c.ct, b.rank, b.delta)));
  } else {
    SW_DISPATCH_G(c.group, (k_delta_csr<GG><<<rgrid + c.n_heavy, kThreads, 0, st>>>(
                                c.nt, c.rp, c.col, c.cval, c.cs, c.ct, b.rank, b.delta, c.heavy_deg,
                                c.heavy, rgrid)));
  }
  ++n_nodes;
  k_tile_sum<<<ntiles, kThreads, 0, st>>>(nt, order, b.delta, b.blk);
  k_tile_scan<<<1, 1024, 0, st>>>(ntiles, b.blk);
  k_tile_argmin<<<ntiles, kThreads, 0, st>>>(nt, order, b.delta, c.x, b.blk, c.hg.sum_cs,
                                             b.blk + ntiles, b.blk_k, counters + 0, b.result);
  k_side<<<grid_for(nt), kThreads, 0, st>>>(nt, order, b.result, b.side_red);
  n_nodes += 4;
  CutArgs a;
  a.cs = c.cs;
  a.ct = c.ct;
  a.side = b.side_red;
  a.c_st = c.hg.c_st;
  a.partials = b.blk + ntiles;
  a.counter = counters + 1;
  a.result = b.result;
  a.C = c.C;
  a.recs = c.recs;
  a.record = record ? 1 : 0;
  if (c.format == PIRMCUT_FORMAT_DIA) {
    SW_DISPATCH_K(c.K, (k_cut_dia<KK><<<rgrid, kThreads, 0, st>>>(c.dd, c.cdia, a)));
  } else {
    SW_DISPATCH_G(c.group, (k_cut_csr<GG><<<rgrid + c.n_heavy, kThreads, 0, st>>>(
                                c.nt, c.rp, c.col, c.cval, a, c.heavy_deg, c.heavy, rgrid)));
  }
  ++n_nodes;
  if (nodes) *nodes = n_nodes;
  return cudaGetLastError();
}

// Exact FP64 cut value of a given reduced side vector (s on the source side,
// t on the sink side) into result[1]; uses the sweep's scratch.
cudaError_t enqueue_cut_value(Ctx& c, cudaStream_t st, const uint8_t* side_red) {
  SweepBuf& b = c.sw;
  const int ntiles = int((c.nt + SC_TILE - 1) / SC_TILE);
  unsigned int* counters = reinterpret_cast<unsigned int*>(b.result + 4);
  CutArgs a;
  a.cs = c.cs;
  a.ct = c.ct;
  a.side = side_red;
  a.c_st = c.hg.c_st;
  a.partials = b.blk + ntiles;
  a.counter = counters + 1;
  a.result = b.result;
  a.C = c.C;
  a.recs = c.recs;
  a.record = 0;
  const int rgrid = grid_for(c.format == PIRMCUT_FORMAT_DIA ? c.nt : c.nt * c.group);
  if (c.format == PIRMCUT_FORMAT_DIA) {
    SW_DISPATCH_K(c.K, (k_cut_dia<KK><<<rgrid, kThreads, 0, st>>>(c.dd, c.cdia, a)));
  } else {
    SW_DISPATCH_G(c.group, (k_cut_csr<GG><<<rgrid + c.n_heavy, kThreads, 0, st>>>(
                                c.nt, c.rp, c.col, c.cval, a, c.heavy_deg, c.heavy, rgrid)));
  }
  return cudaGetLastError();
}

// The sweep as a CUDA graph (records the cut of the last step record).
cudaError_t build_cut_graph(Ctx& c, cudaGraphExec_t* out, int* nodes) {
  cudaStream_t st = c.cap_stream;
  cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  enqueue_sweep(c, st, true, nodes);
  cudaGraph_t g = nullptr;
  e = cudaStreamEndCapture(st, &g);
  if (e == cudaSuccess) e = cudaGraphInstantiate(out, g, 0);
  if (g) cudaGraphDestroy(g);
  return e;
}

cudaError_t launch_side_full(Ctx& c, uint8_t* side_full) {
  k_side_full<<<grid_for(c.nt), kThreads, 0, c.stream>>>(c.nt, c.hg.s, c.hg.t, c.sw.side_red, side_full);
  c.launches += 1;
  return cudaGetLastError();
}

}  // namespace pirmcut
