// Sweep cut that allocates nothing: pirmcut_sweep_cut_static.
//
// Same result as pirmcut_cut (sweep order by x descending, vertex id
// ascending on ties; candidates between strictly different x values plus the
// empty and full prefix; least cut value, then shortest prefix; exact value of
// the chosen side), computed by one thread block straight from a full CSR in
// device memory.  Its scratch (sort keys, payloads, ranks, per-vertex deltas)
// lives in a file-scope __device__ array of fixed size, so the call needs no
// cudaMalloc, no cudaFree and no allocating library routine.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <string>

#include "internal.h"
#include "pirmcut.h"

namespace {

constexpr int64_t kMaxNt = PIRMCUT_STATIC_MAX_NONTERMINALS;
constexpr int kThreadsS = 1024;
constexpr int kMaxDevices = 64;

// keys[2][kMaxNt] u64 | vals[2][kMaxNt] u32 | rank[kMaxNt] i32 | delta[kMaxNt] f64
constexpr size_t kScratchBytes = size_t(kMaxNt) * (2 * 8 + 2 * 4 + 4 + 8);

// Shared by every call on a device; kept for the life of the process.
static __device__ __align__(256) unsigned char g_sweep_scratch[kScratchBytes];

std::mutex g_addr_mu;
void* g_addr[kMaxDevices] = {};

__device__ __forceinline__ uint64_t key_desc(double x) {
  x = x + 0.0;  // fold -0 into +0
  uint64_t b = (uint64_t)__double_as_longlong(x);
  b = (b & 0x8000000000000000ull) ? ~b : (b | 0x8000000000000000ull);
  return ~b;
}

__device__ __forceinline__ int64_t orig_of(int64_t i, int64_t a, int64_t b) {
  int64_t v = i;
  if (v >= a) ++v;
  if (v >= b) ++v;
  return v;
}

__device__ __forceinline__ int64_t red_of(int64_t v, int64_t s, int64_t t) {
  return v - (v > s) - (v > t);
}

// inclusive scan of one double per thread over the block, fixed order
__device__ double block_incl_scan(double v, double* sw, double* total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  double inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const double t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) sw[wid] = inc;
  __syncthreads();
  double off = 0.0, tot = 0.0;
  for (int w = 0; w < kThreadsS / 32; ++w) {
    if (w < wid) off += sw[w];
    tot += sw[w];
  }
  __syncthreads();
  *total = tot;
  return off + inc;
}

__device__ double block_sum_s(double v, double* sw) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if (lane == 0) sw[wid] = v;
  __syncthreads();
  double tot = 0.0;
  for (int w = 0; w < kThreadsS / 32; ++w) tot += sw[w];
  __syncthreads();
  return tot;
}

__global__ void __launch_bounds__(kThreadsS)
k_sweep_static(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
               const double* __restrict__ c, int32_t s, int32_t t, const double* __restrict__ x,
               uint8_t* __restrict__ side, double* __restrict__ result, unsigned char* scratch) {
  __shared__ uint32_t hist[256];
  __shared__ uint32_t run[256];
  __shared__ uint32_t wcnt[kThreadsS / 32][256];
  __shared__ double sw[32];
  __shared__ double s_bv[32];
  __shared__ int64_t s_bk[32];
  __shared__ int s_err;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t nt = n - 2;
  const int64_t a = s < t ? s : t, b = s < t ? t : s;
  uint64_t* K[2];
  uint32_t* V[2];
  K[0] = reinterpret_cast<uint64_t*>(scratch);
  K[1] = K[0] + kMaxNt;
  V[0] = reinterpret_cast<uint32_t*>(K[1] + kMaxNt);
  V[1] = V[0] + kMaxNt;
  int32_t* R = reinterpret_cast<int32_t*>(V[1] + kMaxNt);
  double* D = reinterpret_cast<double*>(R + kMaxNt);
  if (tid == 0) s_err = 0;
  for (int j = tid; j < (kThreadsS / 32) * 256; j += kThreadsS) (&wcnt[0][0])[j] = 0;
  for (int64_t i = tid; i < nt; i += kThreadsS) {
    K[0][i] = key_desc(x[orig_of(i, a, b)]);
    V[0][i] = (uint32_t)i;
  }
  __syncthreads();
  // stable LSD radix sort, 8 passes of 8 bits
  int cur = 0;
  for (int pass = 0; pass < 8; ++pass) {
    const int shift = 8 * pass;
    if (tid < 256) hist[tid] = 0;
    __syncthreads();
    for (int64_t base = 0; base < nt; base += kThreadsS) {
      const int64_t i = base + tid;
      const uint32_t d = i < nt ? uint32_t(K[cur][i] >> shift) & 255u : 256u;
      const unsigned peers = __match_any_sync(0xffffffffu, d);
      if (d < 256u && lane == __ffs(peers) - 1) atomicAdd(&hist[d], (uint32_t)__popc(peers));
    }
    __syncthreads();
    if (tid == 0) {
      uint32_t acc = 0;
      for (int d = 0; d < 256; ++d) {
        const uint32_t h = hist[d];
        hist[d] = acc;
        acc += h;
      }
    }
    if (tid < 256) run[tid] = 0;
    __syncthreads();
    for (int64_t base = 0; base < nt; base += kThreadsS) {
      const int64_t i = base + tid;
      const bool valid = i < nt;
      const uint64_t key = valid ? K[cur][i] : 0ull;
      const uint32_t val = valid ? V[cur][i] : 0u;
      const uint32_t d = valid ? uint32_t(key >> shift) & 255u : 256u;
      const unsigned peers = __match_any_sync(0xffffffffu, d);
      const uint32_t below = __popc(peers & ((1u << lane) - 1u));
      if (d < 256u && lane == __ffs(peers) - 1) wcnt[warp][d] = __popc(peers);
      __syncthreads();
      if (tid < 256) {
        uint32_t off = run[tid];
        for (int w = 0; w < kThreadsS / 32; ++w) {
          const uint32_t cnt = wcnt[w][tid];
          wcnt[w][tid] = off;
          off += cnt;
        }
        run[tid] = off;
      }
      __syncthreads();
      if (valid) {
        const uint32_t pos = hist[d] + wcnt[warp][d] + below;
        K[cur ^ 1][pos] = key;
        V[cur ^ 1][pos] = val;
      }
      __syncthreads();
      for (int j = tid; j < (kThreadsS / 32) * 256; j += kThreadsS) (&wcnt[0][0])[j] = 0;
      __syncthreads();
    }
    cur ^= 1;
  }
  const uint32_t* order = V[cur];
  for (int64_t k = tid; k < nt; k += kThreadsS) R[order[k]] = (int32_t)k;
  __syncthreads();
  // delta_v: change of the cut when v joins the source side
  for (int64_t i = tid; i < nt; i += kThreadsS) {
    const int64_t v = orig_of(i, a, b);
    const int32_t ri = R[i];
    double acc = 0.0;
    for (int64_t e = rp[v]; e < rp[v + 1]; ++e) {
      const int64_t u = col[e];
      const double w = c[e];
      if (u < 0 || u >= n) {
        s_err = 1;
        continue;
      }
      if (u == s) acc -= w;
      else if (u == t) acc += w;
      else if (u != v) acc += (ri < R[red_of(u, s, t)]) ? w : -w;
    }
    D[i] = acc;
  }
  // cut of S = {s}: every edge at s
  double c0 = 0.0;
  for (int64_t e = rp[s] + tid; e < rp[s + 1]; e += kThreadsS) {
    const int64_t u = col[e];
    if (u >= 0 && u < n && u != s) c0 += c[e];
  }
  const double cut0 = block_sum_s(c0, sw);
  __syncthreads();
  // prefix sums in sweep order and the argmin over candidate prefixes
  double running = cut0;
  double best_v = cut0;
  int64_t best_k = 0;
  for (int64_t base = 0; base < nt; base += kThreadsS) {
    const int64_t k = base + tid;
    const double dk = k < nt ? D[order[k]] : 0.0;
    double chunk_tot;
    const double val = running + block_incl_scan(dk, sw, &chunk_tot);
    double bv = INFINITY;
    int64_t bk = INT64_MAX;
    if (k < nt) {
      const bool elig = (k + 1 == nt) ||
                        (x[orig_of(order[k], a, b)] > x[orig_of(order[k + 1], a, b)]);
      if (elig) {
        bv = val;
        bk = k + 1;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_down_sync(0xffffffffu, bv, o);
      const int64_t ok = (int64_t)__shfl_down_sync(0xffffffffu, (long long)bk, o);
      if (ov < bv || (ov == bv && ok < bk)) {
        bv = ov;
        bk = ok;
      }
    }
    if (lane == 0) {
      s_bv[warp] = bv;
      s_bk[warp] = bk;
    }
    __syncthreads();
    for (int w = 0; w < kThreadsS / 32; ++w) {
      if (s_bv[w] < best_v || (s_bv[w] == best_v && s_bk[w] < best_k)) {
        best_v = s_bv[w];
        best_k = s_bk[w];
      }
    }
    running += chunk_tot;
    __syncthreads();
  }
  for (int64_t k = tid; k < nt; k += kThreadsS) side[orig_of(order[k], a, b)] = k < best_k ? 1 : 0;
  if (tid == 0) {
    side[s] = 1;
    side[t] = 0;
  }
  __syncthreads();
  // exact value of the chosen side
  double cv = 0.0;
  for (int64_t v = tid; v < n; v += kThreadsS) {
    const uint8_t sv = side[v];
    for (int64_t e = rp[v]; e < rp[v + 1]; ++e) {
      const int64_t u = col[e];
      if (u > v && u < n && side[u] != sv) cv += c[e];
    }
  }
  const double value = block_sum_s(cv, sw);
  if (tid == 0) {
    const double hi = best_k == 0 ? 1.0 : x[orig_of(order[best_k - 1], a, b)];
    const double lo = best_k == nt ? 0.0 : x[orig_of(order[best_k], a, b)];
    result[0] = value;
    result[1] = 0.5 * (hi + lo);
    result[2] = (double)best_k;
    result[3] = s_err ? 1.0 : 0.0;
  }
}

// Device address of the scratch array on the current device, resolved once
// per device (host code cannot use the symbol's name as a device address).
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_addr_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_sweep_scratch);
    if (e != cudaSuccess) return e;
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" pirmcut_status pirmcut_sweep_cut_static(int64_t n, const int64_t* row_ptr,
                                                   const int32_t* col, const double* c,
                                                   int32_t s, int32_t t, const double* x,
                                                   uint8_t* side, double* result, void* stream) {
  if (n < 3 || n - 2 > kMaxNt) {
    pirmcut::set_global_error("pirmcut_sweep_cut_static: n - 2 must be in [1, " +
                              std::to_string(kMaxNt) + "] (got n = " + std::to_string(n) + ")");
    return PIRMCUT_EINVAL;
  }
  if (s < 0 || t < 0 || s >= n || t >= n || s == t) {
    pirmcut::set_global_error("pirmcut_sweep_cut_static: s and t must be distinct vertices");
    return PIRMCUT_EINVAL;
  }
  if (!row_ptr || !col || !c || !x || !side || !result) {
    pirmcut::set_global_error("pirmcut_sweep_cut_static: null pointer argument");
    return PIRMCUT_EINVAL;
  }
  void* scratch = nullptr;
  cudaError_t e = scratch_address(&scratch);
  if (e == cudaSuccess) {
    k_sweep_static<<<1, kThreadsS, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
        n, row_ptr, col, c, s, t, x, side, result, static_cast<unsigned char*>(scratch));
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    pirmcut::set_global_error(std::string("pirmcut_sweep_cut_static: ") + cudaGetErrorString(e));
    return PIRMCUT_ECUDA;
  }
  return PIRMCUT_OK;
}
