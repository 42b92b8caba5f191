// Reduction of the input graph on the GPU (the work of graph_host.cpp for
// inputs whose rows are already in order): validation, removal of the
// terminals with their edges folded into c(s, v), c(v, t) and c(s, t), the
// symmetry check, the storage choice and the DIA/CSR packing of L~'s fixed
// structure (Section 2, Section 3.1).  It takes the inputs whose every row
// lists strictly increasing columns (no parallel entries) and in which every
// non-terminal has a positive terminal capacity (so that solvability,
// Prop. nonsingular, needs no search); anything else -- and every input
// error, so that the message names the offending row -- goes to the host
// reduction instead.  For the inputs it takes, every stored value is copied,
// never summed, except the cut value of S = {s}, which is summed in the same
// fixed order as on the host: the two paths produce identical problems.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "ctx.h"

namespace pirmcut {

namespace {

constexpr unsigned kFlagRowPtr = 1u << 0;   // row_ptr not monotone or past nnz
constexpr unsigned kFlagInput = 1u << 1;    // a column, a self-loop or a capacity is invalid
constexpr unsigned kFlagOrder = 1u << 2;    // a row's columns do not strictly increase
constexpr unsigned kFlagAsym = 1u << 3;     // the two directions of an edge differ
constexpr unsigned kFlagSeed = 1u << 4;     // a non-terminal without terminal capacity
constexpr int kOffSlots = kMaxDiag + 2;     // per-block offset set (one more than allowed)
constexpr int kScanTile = 4096;             // rows per scan tile (1024 threads x 4)
constexpr int kSumChunks = 256;             // fixed chunking of the c(s, v) sum

__device__ __forceinline__ int64_t gtid() { return int64_t(blockIdx.x) * blockDim.x + threadIdx.x; }
__device__ __forceinline__ int64_t gstride() { return int64_t(gridDim.x) * blockDim.x; }
__device__ __forceinline__ int64_t red(int64_t v, int32_t s, int32_t t) { return v - (v > s) - (v > t); }

// Per non-terminal input row: bounds of the row, validity of its entries,
// strict order of its columns, the count of its non-terminal entries and its
// terminal capacities (one entry each at most, by the order).  The rows of s
// and t, which can hold an entry per vertex, are k_terminal_rows' work.
__global__ void __launch_bounds__(kThreads)
k_rows(int64_t n, int64_t nnz, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
       const double* __restrict__ c, int32_t s, int32_t t, int64_t* __restrict__ cnt,
       double* __restrict__ cs, double* __restrict__ ct, unsigned int* flags) {
  for (int64_t v = gtid(); v < n; v += gstride()) {
    if (v == s || v == t) continue;
    const int64_t b = rp[v], e = rp[v + 1];
    if (b < 0 || e < b || e > nnz) {
      atomicOr(flags, kFlagRowPtr);
      continue;
    }
    unsigned f = 0;
    int64_t m = 0, prev = -1;
    double a = 0.0, z = 0.0;
    for (int64_t k = b; k < e; ++k) {
      const int32_t u = col[k];
      const double w = c[k];
      if (u < 0 || u >= n || u == v || !isfinite(w) || w < 0.0) {
        f |= kFlagInput;
        break;
      }
      if (u <= prev) f |= kFlagOrder;
      prev = u;
      if (u == s) a = w;
      else if (u == t) z = w;
      else ++m;
    }
    if (f) atomicOr(flags, f);
    const int64_t i = red(v, s, t);
    cnt[i] = m;
    cs[i] = a;
    ct[i] = z;
  }
}

// Exclusive scan of cnt[0, nt) into rp[0, nt] (rp[0] = 0): tile sums, one
// block over the tile sums, then each tile writes its running sums.
__global__ void __launch_bounds__(1024)
k_scan_tiles(const int64_t* __restrict__ cnt, int64_t nt, int64_t* __restrict__ tile_sum) {
  __shared__ int64_t sw[32];
  const int64_t base = int64_t(blockIdx.x) * kScanTile;
  int64_t acc = 0;
  for (int j = 0; j < 4; ++j) {
    const int64_t i = base + int64_t(j) * 1024 + threadIdx.x;
    if (i < nt) acc += cnt[i];
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t tot = 0;
    for (int w = 0; w < 32; ++w) tot += sw[w];
    tile_sum[blockIdx.x] = tot;
  }
}

__global__ void __launch_bounds__(1024) k_scan_sums(int64_t* __restrict__ tile_sum, int ntiles) {
  __shared__ int64_t sw[32];
  const int per = (ntiles + 1023) / 1024;
  const int lo = threadIdx.x * per, hi = min(ntiles, lo + per);
  int64_t s = 0;
  for (int b = lo; b < hi; ++b) s += tile_sum[b];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int64_t inc = s;
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t x = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += x;
  }
  if (lane == 31) sw[wid] = inc;
  __syncthreads();
  int64_t woff = 0;
  for (int w = 0; w < wid; ++w) woff += sw[w];
  int64_t run = woff + inc - s;
  for (int b = lo; b < hi; ++b) {
    const int64_t x = tile_sum[b];
    tile_sum[b] = run;
    run += x;
  }
}

__global__ void __launch_bounds__(1024)
k_scan_apply(const int64_t* __restrict__ cnt, int64_t nt, const int64_t* __restrict__ tile_off,
             int64_t* __restrict__ rp) {
  __shared__ int64_t sw[32];
  const int64_t base = int64_t(blockIdx.x) * kScanTile + int64_t(threadIdx.x) * 4;
  int64_t v[4];
  int64_t s = 0;
  for (int j = 0; j < 4; ++j) {
    v[j] = (base + j < nt) ? cnt[base + j] : 0;
    s += v[j];
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int64_t inc = s;
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t x = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += x;
  }
  if (lane == 31) sw[wid] = inc;
  __syncthreads();
  int64_t woff = 0;
  for (int w = 0; w < wid; ++w) woff += sw[w];
  int64_t run = tile_off[blockIdx.x] + woff + inc - s;
  for (int j = 0; j < 4; ++j) {
    run += v[j];
    if (base + j < nt) rp[base + j + 1] = run;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) rp[0] = 0;
}

// The reduced CSR: non-terminal entries of every non-terminal row, in order.
__global__ void __launch_bounds__(kThreads)
k_fill(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
       const double* __restrict__ c, int32_t s, int32_t t, const int64_t* __restrict__ rrp,
       int32_t* __restrict__ rc, double* __restrict__ rv) {
  for (int64_t v = gtid(); v < n; v += gstride()) {
    if (v == s || v == t) continue;
    int64_t o = rrp[red(v, s, t)];
    for (int64_t k = rp[v]; k < rp[v + 1]; ++k) {
      const int32_t u = col[k];
      if (u == s || u == t) continue;
      rc[o] = int32_t(red(u, s, t));
      rv[o] = c[k];
      ++o;
    }
  }
}

// Rows s and t, one entry per thread: their bounds, the validity and strict
// order of their entries (as k_rows checks the other rows), then c(s, v) as
// seen from s, c(v, t) as seen from t, and c(s, t) from both sides (one entry
// per column, by the order).
__global__ void __launch_bounds__(kThreads)
k_terminal_rows(int64_t n, int64_t nnz, const int64_t* __restrict__ rp,
                const int32_t* __restrict__ col, const double* __restrict__ c, int32_t s,
                int32_t t, double* __restrict__ cs_from_s, double* __restrict__ ct_from_t,
                double* __restrict__ cst /* [2] */, unsigned int* flags) {
  const int64_t bs = rp[s], es = rp[s + 1], bt = rp[t], et = rp[t + 1];
  if (bs < 0 || es < bs || es > nnz || bt < 0 || et < bt || et > nnz) {
    if (gtid() == 0) atomicOr(flags, kFlagRowPtr);
    return;
  }
  const int64_t ls = es - bs, total = ls + (et - bt);
  for (int64_t q = gtid(); q < total; q += gstride()) {
    const bool from_s = q < ls;
    const int64_t k = from_s ? bs + q : bt + (q - ls);
    const int64_t row = from_s ? s : t, first = from_s ? bs : bt;
    const int32_t u = col[k];
    const double w = c[k];
    if (u < 0 || u >= n || u == row || !isfinite(w) || w < 0.0) {
      atomicOr(flags, kFlagInput);
      continue;
    }
    if (k > first && col[k - 1] >= u) atomicOr(flags, kFlagOrder);
    if (from_s) {
      if (u == t) cst[0] = c[k];
      else cs_from_s[red(u, s, t)] = c[k];
    } else {
      if (u == s) cst[1] = c[k];
      else ct_from_t[red(u, s, t)] = c[k];
    }
  }
}

// Per reduced row: terminal capacities equal from both sides, every entry's
// mirror present with the same capacity, a positive terminal capacity.
__global__ void __launch_bounds__(kThreads)
k_check(int64_t nt, const int64_t* __restrict__ rrp, const int32_t* __restrict__ rc,
        const double* __restrict__ rv, const double* __restrict__ cs, const double* __restrict__ ct,
        const double* __restrict__ cs_from_s, const double* __restrict__ ct_from_t,
        unsigned int* flags) {
  for (int64_t i = gtid(); i < nt; i += gstride()) {
    unsigned f = 0;
    if (cs[i] != cs_from_s[i] || ct[i] != ct_from_t[i]) f |= kFlagAsym;
    if (!(cs[i] > 0.0 || ct[i] > 0.0)) f |= kFlagSeed;
    for (int64_t k = rrp[i]; k < rrp[i + 1] && !(f & kFlagAsym); ++k) {
      const int64_t j = rc[k];
      int64_t lo = rrp[j], hi = rrp[j + 1];
      while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (rc[mid] < i) lo = mid + 1;
        else hi = mid;
      }
      if (lo == rrp[j + 1] || rc[lo] != i || rv[lo] != rv[k]) f |= kFlagAsym;
    }
    if (f) atomicOr(flags, f);
  }
}

// The distinct positive offsets rc - i of each block's rows (at most
// kOffSlots; a full set means "more than kMaxDiag").
__global__ void __launch_bounds__(kThreads)
k_offsets(int64_t nt, const int64_t* __restrict__ rrp, const int32_t* __restrict__ rc,
          unsigned long long* __restrict__ blk_off) {
  __shared__ unsigned long long so[kOffSlots];
  if (threadIdx.x < kOffSlots) so[threadIdx.x] = 0ull;
  __syncthreads();
  for (int64_t i = gtid(); i < nt; i += gstride()) {
    for (int64_t k = rrp[i]; k < rrp[i + 1]; ++k) {
      const int64_t o = int64_t(rc[k]) - i;
      if (o <= 0) continue;
      const unsigned long long uo = (unsigned long long)o;
      for (int slot = 0; slot < kOffSlots; ++slot) {
        const unsigned long long cur = *((volatile unsigned long long*)&so[slot]);
        if (cur == uo) break;
        if (cur == 0ull) {
          const unsigned long long old = atomicCAS(&so[slot], 0ull, uo);
          if (old == 0ull || old == uo) break;
        }
      }
    }
  }
  __syncthreads();
  if (threadIdx.x < kOffSlots) blk_off[size_t(blockIdx.x) * kOffSlots + threadIdx.x] = so[threadIdx.x];
}

struct Offsets {
  int64_t off[kMaxDiag];
};

__global__ void __launch_bounds__(kThreads)
k_pack_dia(int64_t nt, int K, Offsets os, const int64_t* __restrict__ rrp,
           const int32_t* __restrict__ rc, const double* __restrict__ rv, double* __restrict__ cdia) {
  for (int64_t i = gtid(); i < nt; i += gstride()) {
    for (int64_t k = rrp[i]; k < rrp[i + 1]; ++k) {
      const int64_t o = int64_t(rc[k]) - i;
      if (o <= 0) continue;
      int f = 0;
      while (f < K - 1 && os.off[f] != o) ++f;
      cdia[size_t(f) * nt + i] = rv[k];
    }
  }
}

// sum of cs in the order the host reduction uses: kSumChunks fixed chunks, a
// warp per chunk (one block each, spread over the SMs) whose lane j runs over
// the elements a + j, a + j + 32, ...; the lane sums in lane order; then
// k_sum_parts adds the chunk sums in order.
__global__ void __launch_bounds__(32)
k_sum_chunks(const double* __restrict__ v, int64_t n, double* __restrict__ part) {
  const int lane = threadIdx.x, ch = blockIdx.x;
  const int64_t a = n * ch / kSumChunks, b = n * (ch + 1) / kSumChunks;
  double acc = 0.0;
  for (int64_t i = a + lane; i < b; i += 32) acc += v[i];
  double s = 0.0;
  for (int j = 0; j < 32; ++j) s += __shfl_sync(0xffffffffu, acc, j);
  if (lane == 0) part[ch] = s;
}

__global__ void k_sum_parts(const double* __restrict__ part, double* __restrict__ out) {
  if (threadIdx.x != 0) return;
  double s = 0.0;
  for (int k = 0; k < kSumChunks; ++k) s += part[k];
  *out = s;
}

template <class T>
cudaError_t dmalloc(T** p, size_t count) {
  return cudaMalloc((void**)p, sizeof(T) * (count ? count : 1));
}

}  // namespace

void DeviceGraph::release() {
  void* ps[] = {in_rp, in_col, cs, ct, cdia, rp, col, cval};
  for (void* p : ps)
    if (p) cudaFree(p);
  *this = DeviceGraph();
}

// float -> double, exact
__global__ void k_widen(int64_t n, const float* __restrict__ in, double* __restrict__ out) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += int64_t(gridDim.x) * blockDim.x)
    out[i] = double(in[i]);
}

// Returns PIRMCUT_OK with *taken = true when the GPU built the problem (the
// arrays in *dg, the scalars in *g), PIRMCUT_OK with *taken = false when the
// host must do it, or a CUDA error status.  rp_dev / col_dev: when non-null,
// the input structure already on the device (kept from an earlier call).
pirmcut_status reduce_graph_device(int64_t n, const int64_t* row_ptr, const int32_t* col,
                                   const void* c, int c_fp32, int32_t s, int32_t t, int format_req,
                                   int mem_kind, void* stream, const int64_t* rp_dev,
                                   const int32_t* col_dev, HostGraph* g, DeviceGraph* dg,
                                   bool* taken, std::string* err) {
  *taken = false;
  *dg = DeviceGraph();
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (n < 3 || n >= (int64_t(1) << 31) || s < 0 || t < 0 || s >= n || t >= n || s == t)
    return PIRMCUT_OK;  // the host reports it
  const int64_t nt = n - 2;
  // temporaries
  int64_t* d_cnt = nullptr;
  int64_t* d_tile = nullptr;
  double* d_c = nullptr;
  float* d_c32 = nullptr;     // float capacities uploaded from the host
  double* d_cs_s = nullptr;
  double* d_ct_t = nullptr;
  double* d_small = nullptr;  // [cst_s, cst_t, sum, -, kSumChunks chunk sums]
  unsigned int* d_flags = nullptr;
  unsigned long long* d_off = nullptr;
  cudaError_t e = cudaSuccess;
  pirmcut_status ret = PIRMCUT_OK;
  DeviceGraph out;
  auto cleanup = [&]() {
    void* ps[] = {d_cnt, d_tile, d_c, d_c32, d_cs_s, d_ct_t, d_small, d_flags, d_off};
    for (void* p : ps)
      if (p) cudaFree(p);
  };
  auto drop = [&]() {  // free what this call allocated (never the caller's structure)
    cleanup();
    if (rp_dev) {
      out.in_rp = nullptr;
      out.in_col = nullptr;
    }
    out.release();
  };
  auto cuda_error = [&](cudaError_t ce, const char* where) {
    *err = std::string(where) + ": " + cudaGetErrorString(ce);
    drop();
    return ce == cudaErrorMemoryAllocation ? PIRMCUT_ENOMEM : PIRMCUT_ECUDA;
  };
  auto give_up = [&]() {
    drop();
    return PIRMCUT_OK;
  };
  const cudaMemcpyKind h2d = mem_kind == PIRMCUT_MEM_DEVICE ? cudaMemcpyDeviceToDevice
                                                            : cudaMemcpyHostToDevice;
  // ---- the input structure and capacities on the device
  int64_t nnz = 0;
  if (rp_dev) {
    out.in_rp = const_cast<int64_t*>(rp_dev);
    out.in_col = const_cast<int32_t*>(col_dev);
    if ((e = cudaMemcpy(&nnz, rp_dev + n, sizeof(int64_t), cudaMemcpyDeviceToHost)) != cudaSuccess)
      return cuda_error(e, "reading row_ptr");
  } else {
    if (mem_kind == PIRMCUT_MEM_DEVICE) {
      int64_t ends[2];
      if ((e = cudaMemcpy(&ends[0], row_ptr, sizeof(int64_t), cudaMemcpyDeviceToHost)) != cudaSuccess ||
          (e = cudaMemcpy(&ends[1], row_ptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost)) != cudaSuccess)
        return cuda_error(e, "reading row_ptr");
      if (ends[0] != 0) return give_up();
      nnz = ends[1];
    } else {
      if (row_ptr[0] != 0) return give_up();
      nnz = row_ptr[n];
    }
    if (nnz < 0 || nnz >= (int64_t(1) << 40) || (nnz > 0 && (!col || !c))) return give_up();
    if ((e = dmalloc(&out.in_rp, size_t(n) + 1)) != cudaSuccess) return cuda_error(e, "cudaMalloc");
    if ((e = dmalloc(&out.in_col, size_t(nnz))) != cudaSuccess) return cuda_error(e, "cudaMalloc");
    if ((e = cudaMemcpyAsync(out.in_rp, row_ptr, sizeof(int64_t) * (size_t(n) + 1), h2d, st)) != cudaSuccess ||
        (nnz && (e = cudaMemcpyAsync(out.in_col, col, sizeof(int32_t) * size_t(nnz), h2d, st)) != cudaSuccess))
      return cuda_error(e, "uploading the graph");
  }
  if (nnz > 0 && !c) return give_up();
  const double* dc = static_cast<const double*>(c);
  if (c_fp32) {
    // float capacities: uploaded as they are (half the bytes of doubles)
    // and widened exactly on the GPU
    const float* src = static_cast<const float*>(c);
    if (mem_kind != PIRMCUT_MEM_DEVICE) {
      if ((e = dmalloc(&d_c32, size_t(nnz))) != cudaSuccess) return cuda_error(e, "cudaMalloc");
      if (nnz && (e = cudaMemcpyAsync(d_c32, c, sizeof(float) * size_t(nnz), h2d, st)) != cudaSuccess)
        return cuda_error(e, "uploading the capacities");
      src = d_c32;
    }
    if ((e = dmalloc(&d_c, size_t(nnz))) != cudaSuccess) return cuda_error(e, "cudaMalloc");
    if (nnz) k_widen<<<grid_for(nnz), kThreads, 0, st>>>(nnz, src, d_c);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_error(e, "widening the capacities");
    dc = d_c;
  } else if (mem_kind != PIRMCUT_MEM_DEVICE) {
    if ((e = dmalloc(&d_c, size_t(nnz))) != cudaSuccess) return cuda_error(e, "cudaMalloc");
    if (nnz && (e = cudaMemcpyAsync(d_c, c, sizeof(double) * size_t(nnz), h2d, st)) != cudaSuccess)
      return cuda_error(e, "uploading the capacities");
    dc = d_c;
  }
  // ---- per-row pass
  if ((e = dmalloc(&d_cnt, size_t(nt))) != cudaSuccess || (e = dmalloc(&out.cs, size_t(nt))) != cudaSuccess ||
      (e = dmalloc(&out.ct, size_t(nt))) != cudaSuccess || (e = dmalloc(&d_cs_s, size_t(nt))) != cudaSuccess ||
      (e = dmalloc(&d_ct_t, size_t(nt))) != cudaSuccess || (e = dmalloc(&d_small, 4 + kSumChunks)) != cudaSuccess ||
      (e = dmalloc(&d_flags, 1)) != cudaSuccess)
    return cuda_error(e, "cudaMalloc");
  cudaMemsetAsync(d_flags, 0, sizeof(unsigned int), st);
  cudaMemsetAsync(d_small, 0, 4 * sizeof(double), st);
  cudaMemsetAsync(d_cs_s, 0, sizeof(double) * size_t(nt), st);
  cudaMemsetAsync(d_ct_t, 0, sizeof(double) * size_t(nt), st);
  k_rows<<<grid_for(n), kThreads, 0, st>>>(n, nnz, out.in_rp, out.in_col, dc, s, t, d_cnt, out.cs,
                                           out.ct, d_flags);
  unsigned int flags = 0;
  if ((e = cudaGetLastError()) != cudaSuccess ||
      (e = cudaMemcpyAsync(&flags, d_flags, sizeof(flags), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
      (e = cudaStreamSynchronize(st)) != cudaSuccess)
    return cuda_error(e, "checking the graph");
  if (flags) return give_up();
  // ---- reduced CSR
  const int ntiles = int((nt + kScanTile - 1) / kScanTile);
  if ((e = dmalloc(&d_tile, size_t(ntiles))) != cudaSuccess || (e = dmalloc(&out.rp, size_t(nt) + 1)) != cudaSuccess)
    return cuda_error(e, "cudaMalloc");
  if (ntiles > 0) {
    k_scan_tiles<<<ntiles, 1024, 0, st>>>(d_cnt, nt, d_tile);
    k_scan_sums<<<1, 1024, 0, st>>>(d_tile, ntiles);
    k_scan_apply<<<ntiles, 1024, 0, st>>>(d_cnt, nt, d_tile, out.rp);
  }
  int64_t mnt = 0;
  if ((e = cudaGetLastError()) != cudaSuccess ||
      (e = cudaMemcpyAsync(&mnt, out.rp + nt, sizeof(int64_t), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
      (e = cudaStreamSynchronize(st)) != cudaSuccess)
    return cuda_error(e, "building the reduced graph");
  if ((e = dmalloc(&out.col, size_t(mnt))) != cudaSuccess || (e = dmalloc(&out.cval, size_t(mnt))) != cudaSuccess)
    return cuda_error(e, "cudaMalloc");
  k_fill<<<grid_for(n), kThreads, 0, st>>>(n, out.in_rp, out.in_col, dc, s, t, out.rp, out.col, out.cval);
  k_terminal_rows<<<grid_for(nt), kThreads, 0, st>>>(n, nnz, out.in_rp, out.in_col, dc, s, t, d_cs_s,
                                                      d_ct_t, d_small, d_flags);
  k_check<<<grid_for(nt), kThreads, 0, st>>>(nt, out.rp, out.col, out.cval, out.cs, out.ct, d_cs_s,
                                             d_ct_t, d_flags);
  k_sum_chunks<<<kSumChunks, 32, 0, st>>>(out.cs, nt, d_small + 4);
  k_sum_parts<<<1, 32, 0, st>>>(d_small + 4, d_small + 2);
  double small[4] = {0, 0, 0, 0};
  if ((e = cudaGetLastError()) != cudaSuccess ||
      (e = cudaMemcpyAsync(&flags, d_flags, sizeof(flags), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
      (e = cudaMemcpyAsync(small, d_small, sizeof(small), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
      (e = cudaStreamSynchronize(st)) != cudaSuccess)
    return cuda_error(e, "checking the graph");
  if (flags || small[0] != small[1]) return give_up();
  // ---- storage choice (the host reduction's rule)
  int K = 0;
  int64_t offs[kMaxDiag];
  bool dia_ok = format_req != PIRMCUT_FORMAT_CSR;
  if (dia_ok) {
    const int nb = grid_for(nt);
    if ((e = dmalloc(&d_off, size_t(nb) * kOffSlots)) != cudaSuccess) return cuda_error(e, "cudaMalloc");
    k_offsets<<<nb, kThreads, 0, st>>>(nt, out.rp, out.col, d_off);
    std::vector<unsigned long long> ho(size_t(nb) * kOffSlots);
    if ((e = cudaGetLastError()) != cudaSuccess ||
        (e = cudaMemcpyAsync(ho.data(), d_off, sizeof(unsigned long long) * ho.size(), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
      return cuda_error(e, "reading the offsets");
    for (size_t q = 0; q < ho.size() && dia_ok; ++q) {
      const int64_t o = int64_t(ho[q]);
      if (o == 0) continue;
      int f = 0;
      while (f < K && offs[f] != o) ++f;
      if (f == K) {
        if (K == kMaxDiag) dia_ok = false;
        else offs[K++] = o;
      }
    }
    if (dia_ok && K > 0) {
      for (int a = 1; a < K; ++a)  // ascending; K <= kMaxDiag
        for (int b = a; b > 0 && offs[b - 1] > offs[b]; --b) std::swap(offs[b - 1], offs[b]);
      dia_ok = double(mnt / 2) / (double(K) * double(nt)) >= 0.5;
    }
    if (K == 0) dia_ok = false;
  }
  if (format_req == PIRMCUT_FORMAT_DIA && !dia_ok) {
    *err = "DIA storage requested but the graph has more than 8 offsets or sparse diagonals";
    drop();
    return PIRMCUT_EINVAL;
  }
  // ---- the problem
  HostGraph& hg = *g;
  hg = HostGraph();
  hg.n = n;
  hg.nt = nt;
  hg.s = s;
  hg.t = t;
  hg.n_edges = mnt / 2;
  hg.nnz = mnt;
  hg.c_st = small[0];
  hg.sum_cs = small[2] + small[0];
  if (dia_ok) {
    hg.format = PIRMCUT_FORMAT_DIA;
    hg.K = K;
    Offsets os{};
    for (int k = 0; k < K; ++k) os.off[k] = hg.off[k] = offs[k];
    if ((e = dmalloc(&out.cdia, size_t(K) * size_t(nt))) != cudaSuccess) return cuda_error(e, "cudaMalloc");
    cudaMemsetAsync(out.cdia, 0, sizeof(double) * size_t(K) * size_t(nt), st);
    k_pack_dia<<<grid_for(nt), kThreads, 0, st>>>(nt, K, os, out.rp, out.col, out.cval, out.cdia);
    if ((e = cudaGetLastError()) != cudaSuccess || (e = cudaStreamSynchronize(st)) != cudaSuccess)
      return cuda_error(e, "packing the diagonals");
    cudaFree(out.rp);
    cudaFree(out.col);
    cudaFree(out.cval);
    out.rp = nullptr;
    out.col = nullptr;
    out.cval = nullptr;
  } else {
    hg.format = PIRMCUT_FORMAT_CSR;
    const double avg = nt ? double(mnt) / double(nt) : 0.0;
    int grp = 1;
    while (grp < 32 && grp < avg) grp *= 2;
    hg.group = grp;
  }
  cleanup();
  if (rp_dev) {
    out.in_rp = nullptr;  // owned by the caller
    out.in_col = nullptr;
  }
  *dg = out;
  *taken = true;
  return ret;
}

}  // namespace pirmcut
