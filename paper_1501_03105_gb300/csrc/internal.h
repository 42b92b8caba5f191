// Internal declarations shared by the translation units of libpirmcut.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "pirmcut.h"

namespace pirmcut {

constexpr int kMaxDiag = 8;  // most upper diagonals the DIA storage accepts

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
  std::vector<double> cdia;
  // CSR of G~ (both directions stored, rows sorted, parallel entries merged).
  std::vector<int64_t> rp;
  std::vector<int32_t> col;
  std::vector<double> cval;
  int group = 1;        // threads per row for the CSR kernels
  // Terminal capacities c(s, v), c(v, t) per non-terminal and c(s, t).
  std::vector<double> cs, ct;
  double c_st = 0.0;
  double sum_cs = 0.0;  // sum_v c(s, v) + c(s, t): the cut value of S = {s}
};

// Validate the full CSR and build the reduced problem.  Returns PIRMCUT_OK or
// an error status with a message in *err.  format_req is PIRMCUT_FORMAT_*.
pirmcut_status reduce_graph(int64_t n, const int64_t* row_ptr, const int32_t* col,
                            const double* c, int32_t s, int32_t t, int format_req,
                            HostGraph* out, std::string* err);

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
