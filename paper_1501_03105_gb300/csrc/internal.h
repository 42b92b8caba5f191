// Internal declarations shared by the translation units of libpirmcut.
#pragma once

#include <sched.h>

#include <algorithm>
#include <cstdint>
#include <memory>
#include <string>
#include <thread>
#include <vector>

#include "pirmcut.h"

namespace pirmcut {

constexpr int kMaxDiag = 8;  // most upper diagonals the DIA storage accepts

// Allocator whose value-less construction leaves the element uninitialised,
// so that large host buffers are not zero-filled by one thread before a
// parallel pass writes every element anyway.
template <class T>
struct NoInitAllocator : std::allocator<T> {
  template <class U>
  struct rebind {
    using other = NoInitAllocator<U>;
  };
  NoInitAllocator() = default;
  template <class U>
  NoInitAllocator(const NoInitAllocator<U>&) noexcept {}
  template <class U>
  void construct(U* p) noexcept {
    ::new (static_cast<void*>(p)) U;
  }
  template <class U, class... A>
  void construct(U* p, A&&... a) {
    ::new (static_cast<void*>(p)) U(std::forward<A>(a)...);
  }
};
template <class T>
using hvec = std::vector<T, NoInitAllocator<T>>;

// Cores this process may run on (its CPU affinity mask; hardware_concurrency
// counts every CPU of the machine, which oversubscribes a restricted process).
inline int host_threads() {
  static const int n = [] {
    cpu_set_t set;
    CPU_ZERO(&set);
    int k = 0;
    if (sched_getaffinity(0, sizeof(set), &set) == 0) k = CPU_COUNT(&set);
    if (k <= 0) k = int(std::thread::hardware_concurrency());
    return k > 0 ? k : 1;
  }();
  return n;
}

// Run fn(lo, hi) over [0, n) split across the host's cores (at least
// min_per_thread items per thread).
template <class F>
void parallel_for(int64_t n, F fn, int64_t min_per_thread = 32768) {
  int64_t nth = std::max<int64_t>(1, std::min<int64_t>(host_threads(), 64));
  nth = std::min<int64_t>(nth, std::max<int64_t>(1, n / min_per_thread));
  std::vector<std::thread> th;
  for (int64_t k = 0; k < nth; ++k) {
    const int64_t lo = n * k / nth, hi = n * (k + 1) / nth;
    if (k + 1 == nth) fn(lo, hi);
    else th.emplace_back([=] { fn(lo, hi); });
  }
  for (auto& x : th) x.join();
}

// Smallest i in [0, n) with pred(i), or n: a parallel search over fixed
// chunks (the answer does not depend on the thread count).
template <class P>
int64_t parallel_find_first(int64_t n, P pred) {
  constexpr int kChunks = 256;
  int64_t first[kChunks];
  parallel_for(kChunks, [&](int64_t lo, int64_t hi) {
    for (int64_t ch = lo; ch < hi; ++ch) {
      const int64_t a = n * ch / kChunks, b = n * (ch + 1) / kChunks;
      int64_t f = n;
      for (int64_t i = a; i < b; ++i)
        if (pred(i)) {
          f = i;
          break;
        }
      first[ch] = f;
    }
  }, 1);
  for (int ch = 0; ch < kChunks; ++ch)
    if (first[ch] < n) return first[ch];
  return n;
}

// out[0] = 0, out[i + 1] = out[i] + in[i] for i < n (inclusive running sum of
// in, shifted): chunk sums in parallel, then each chunk fills its range.
template <class T>
void parallel_scan_shifted(const T* in, int64_t n, T* out) {
  constexpr int kChunks = 256;
  T part[kChunks + 1];
  parallel_for(kChunks, [&](int64_t lo, int64_t hi) {
    for (int64_t ch = lo; ch < hi; ++ch) {
      const int64_t a = n * ch / kChunks, b = n * (ch + 1) / kChunks;
      T acc = 0;
      for (int64_t i = a; i < b; ++i) acc += in[i];
      part[ch + 1] = acc;
    }
  }, 1);
  part[0] = 0;
  for (int ch = 0; ch < kChunks; ++ch) part[ch + 1] += part[ch];
  out[0] = 0;
  parallel_for(kChunks, [&](int64_t lo, int64_t hi) {
    for (int64_t ch = lo; ch < hi; ++ch) {
      const int64_t a = n * ch / kChunks, b = n * (ch + 1) / kChunks;
      T acc = part[ch];
      for (int64_t i = a; i < b; ++i) {
        acc += in[i];
        out[i + 1] = acc;
      }
    }
  }, 1);
}

// Sum of v[0, n) in a fixed order, independent of the thread count (and the
// order the device reduction of the input uses): 256 chunks; in a chunk
// [a, b), 32 running sums over the elements a + j, a + j + 32, ... (j < 32),
// added in order of j; then the chunk sums in order.
inline double chunked_sum(const double* v, int64_t n) {
  constexpr int kChunks = 256, kLanes = 32;
  double part[kChunks];
  parallel_for(kChunks, [&](int64_t lo, int64_t hi) {
    for (int64_t ch = lo; ch < hi; ++ch) {
      const int64_t a = n * ch / kChunks, b = n * (ch + 1) / kChunks;
      double lane[kLanes] = {0.0};
      for (int64_t base = a; base < b; base += kLanes) {
        const int m = int(std::min<int64_t>(kLanes, b - base));
        for (int j = 0; j < m; ++j) lane[j] += v[base + j];
      }
      double acc = 0.0;
      for (int j = 0; j < kLanes; ++j) acc += lane[j];
      part[ch] = acc;
    }
  }, 1);
  double s = 0.0;
  for (int ch = 0; ch < kChunks; ++ch) s += part[ch];
  return s;
}

// dst[0, n) = v in parallel
template <class T>
void parallel_fill(T* dst, int64_t n, T v) {
  parallel_for(n, [=](int64_t lo, int64_t hi) { std::fill(dst + lo, dst + hi, v); }, 1 << 20);
}

// dst[0, n) = src[0, n) in parallel
template <class T>
void parallel_copy(T* dst, const T* src, int64_t n) {
  parallel_for(n, [=](int64_t lo, int64_t hi) { std::copy(src + lo, src + hi, dst + lo); }, 1 << 20);
}

// The reduced problem built once per instance on the host: the non-terminal
// graph G~ (Section 2), the terminal capacities folded per vertex, and the
// packed storage of L~'s structure (Section 3.1: the structure never changes).
struct HostGraph {
  int64_t n = 0;        // vertices including s and t
  int64_t nt = 0;       // non-terminals n~
  int32_t s = 0, t = 0;
  int64_t n_edges = 0;  // e~: undirected non-terminal edges
  int format = PIRMCUT_FORMAT_CSR;
  // DIA: capacity of edge (i, i + off[k]) at cdia[k * nt + i]; 0 where absent.
  int K = 0;
  int64_t off[kMaxDiag] = {0};
  hvec<double> cdia;
  // CSR of G~ (both directions stored, rows sorted, parallel entries merged).
  hvec<int64_t> rp;
  hvec<int32_t> col;
  hvec<double> cval;
  int group = 1;        // threads per row for the CSR kernels
  // Terminal capacities c(s, v), c(v, t) per non-terminal and c(s, t).
  hvec<double> cs, ct;
  double c_st = 0.0;
  double sum_cs = 0.0;  // sum_v c(s, v) + c(s, t): the cut value of S = {s}
  int64_t nnz = 0;      // stored entries of G~'s CSR (both directions)
};

// The reduced problem built on the GPU (device arrays, owned): the input
// structure kept for later capacity updates, the terminal capacities, and
// either the DIA capacities or the reduced CSR.
struct DeviceGraph {
  int64_t* in_rp = nullptr;
  int32_t* in_col = nullptr;
  double* cs = nullptr;
  double* ct = nullptr;
  double* cdia = nullptr;
  int64_t* rp = nullptr;
  int32_t* col = nullptr;
  double* cval = nullptr;
  void release();  // cudaFree of every non-null array
};

// Validate the full CSR and build the reduced problem.  Returns PIRMCUT_OK or
// an error status with a message in *err.  format_req is PIRMCUT_FORMAT_*.
pirmcut_status reduce_graph(int64_t n, const int64_t* row_ptr, const int32_t* col,
                            const double* c, int32_t s, int32_t t, int format_req,
                            HostGraph* out, std::string* err);

// The same reduction on the GPU for inputs whose rows list strictly increasing
// columns and whose non-terminals all have a terminal capacity; *taken says
// whether it built the problem (otherwise the host reduction must run).
// c is double[nnz], or float[nnz] when c_fp32 (widened exactly on the GPU).
// mem_kind says where row_ptr, col and c live; rp_dev / col_dev, when non-null,
// are an input structure already on the device (owned by the caller).
pirmcut_status reduce_graph_device(int64_t n, const int64_t* row_ptr, const int32_t* col,
                                   const void* c, int c_fp32, int32_t s, int32_t t, int format_req,
                                   int mem_kind, void* stream, const int64_t* rp_dev,
                                   const int32_t* col_dev, HostGraph* g, DeviceGraph* dg,
                                   bool* taken, std::string* err);

// Record the message returned by pirmcut_last_error(NULL) for calls that have
// no context.
void set_global_error(const std::string& msg);

// Reduced index of original vertex v (v not a terminal) and its inverse.
inline int64_t reduced_index(int64_t v, int32_t s, int32_t t) {
  return v - (v > s) - (v > t);
}
inline int64_t original_index(int64_t i, int32_t s, int32_t t) {
  const int64_t a = s < t ? s : t, b = s < t ? t : s;
  int64_t v = i;
  if (v >= a) ++v;
  if (v >= b) ++v;
  return v;
}

}  // namespace pirmcut
