// Host-side reduction of the input graph: validation, removal of the
// terminals (the non-terminal graph G~ and the terminal edges of Section 2),
// the solvability check of Prop. (nonsingular), and the packing of L~'s
// fixed structure (Section 3.1) into DIA or CSR storage.  Runs once per
// instance inside pirmcut_create / pirmcut_update_weights.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <thread>
#include <utility>

#include "internal.h"

namespace pirmcut {

namespace {

struct Entry {
  int32_t col;
  double c;
};


// Stable sort of a row's entries by column: insertion sort for the short rows
// of meshes and sparse graphs (no allocation), std::stable_sort otherwise.
void sort_row(std::vector<Entry>& buf) {
  bool sorted = true;
  for (size_t k = 1; k < buf.size() && sorted; ++k) sorted = buf[k - 1].col <= buf[k].col;
  if (sorted) return;
  if (buf.size() <= 32) {
    for (size_t k = 1; k < buf.size(); ++k) {
      const Entry e = buf[k];
      size_t j = k;
      while (j > 0 && buf[j - 1].col > e.col) {
        buf[j] = buf[j - 1];
        --j;
      }
      buf[j] = e;
    }
    return;
  }
  std::stable_sort(buf.begin(), buf.end(), [](const Entry& a, const Entry& b) { return a.col < b.col; });
}

}  // namespace

pirmcut_status reduce_graph(int64_t n, const int64_t* row_ptr, const int32_t* col,
                            const double* c, int32_t s, int32_t t, int format_req,
                            HostGraph* out, std::string* err) {
  if (n < 3 || n >= (int64_t(1) << 31)) {
    *err = "n must be in [3, 2^31)";
    return PIRMCUT_EINVAL;
  }
  if (s < 0 || t < 0 || s >= n || t >= n || s == t) {
    *err = "s and t must be distinct vertices";
    return PIRMCUT_EINVAL;
  }
  if (!row_ptr || row_ptr[0] != 0) {
    *err = "row_ptr[0] must be 0";
    return PIRMCUT_EINVAL;
  }
  if (parallel_find_first(n, [&](int64_t v) { return row_ptr[v + 1] < row_ptr[v]; }) < n) {
    *err = "row_ptr must be non-decreasing";
    return PIRMCUT_EINVAL;
  }
  const int64_t nnz = row_ptr[n];
  if (nnz > 0 && (!col || !c)) {
    *err = "col and c must be non-null";
    return PIRMCUT_EINVAL;
  }
  HostGraph& g = *out;
  g = HostGraph();
  g.n = n;
  g.nt = n - 2;
  g.s = s;
  g.t = t;
  const int64_t nt = g.nt;

  // ---- per-row pass: validate entries, fold terminal edges, merge parallel
  // entries of the non-terminal rows (sorted by reduced column).
  hvec<int64_t> cnt(nt + 1);
  hvec<double> cs(nt), ct(nt), cs_from_s(nt), ct_from_t(nt);
  cnt[0] = 0;
  parallel_fill(cs_from_s.data(), nt, 0.0);
  parallel_fill(ct_from_t.data(), nt, 0.0);
  double cst_s = 0.0, cst_t = 0.0;
  // pass 1 (parallel): validate, count merged non-terminal entries per row.
  // row_bad: 0 = valid and its non-terminal columns strictly increase (copied
  // as they are), 4 = valid but unsorted or with parallel entries (sorted and
  // merged), 1-3 = an error.
  hvec<uint8_t> row_bad(n);
  parallel_for(n, [&](int64_t lo, int64_t hi) {
    std::vector<Entry> buf;
    for (int64_t v = lo; v < hi; ++v) {
      const int64_t b = row_ptr[v], e = row_ptr[v + 1];
      uint8_t code = 0;
      int64_t m = 0, prev = -1;
      for (int64_t k = b; k < e; ++k) {
        const int32_t u = col[k];
        const double w = c[k];
        if (u < 0 || u >= n) { code = 1; break; }
        if (u == v) { code = 2; break; }
        if (!std::isfinite(w) || w < 0.0) { code = 3; break; }
        if (u == s || u == t) continue;
        const int64_t r = reduced_index(u, s, t);
        if (r <= prev) code = 4;
        prev = r;
        ++m;
      }
      row_bad[v] = code;
      if ((code != 0 && code != 4) || v == s || v == t) continue;
      if (code == 0) {
        cnt[reduced_index(v, s, t) + 1] = m;
        continue;
      }
      buf.clear();
      for (int64_t k = b; k < e; ++k) {
        const int32_t u = col[k];
        if (u == s || u == t) continue;
        buf.push_back({(int32_t)reduced_index(u, s, t), c[k]});
      }
      sort_row(buf);
      int64_t merged = 0;
      for (size_t k = 0; k < buf.size(); ++k)
        if (k == 0 || buf[k].col != buf[k - 1].col) ++merged;
      cnt[reduced_index(v, s, t) + 1] = merged;
    }
  });
  {
    const int64_t v = parallel_find_first(n, [&](int64_t i) { return row_bad[i] >= 1 && row_bad[i] <= 3; });
    if (v < n) {
      if (row_bad[v] == 1) *err = "column index out of range in row " + std::to_string(v);
      else if (row_bad[v] == 2) *err = "self-loop at vertex " + std::to_string(v);
      else *err = "capacity not finite or negative in row " + std::to_string(v);
      return PIRMCUT_EINVAL;
    }
  }
  hvec<int64_t> rp(nt + 1);
  parallel_scan_shifted(cnt.data() + 1, nt, rp.data());
  const int64_t mnt = rp[nt];
  hvec<int32_t> rc(mnt);
  hvec<double> rv(mnt);
  // pass 2 (parallel): fill merged rows and the terminal capacities
  parallel_for(n, [&](int64_t lo, int64_t hi) {
    std::vector<Entry> buf;
    for (int64_t v = lo; v < hi; ++v) {
      if (v == s || v == t) continue;
      const int64_t i = reduced_index(v, s, t);
      double a = 0.0, z = 0.0;
      if (row_bad[v] == 0) {
        int64_t o = rp[i];
        for (int64_t k = row_ptr[v]; k < row_ptr[v + 1]; ++k) {
          const int32_t u = col[k];
          if (u == s) a += c[k];
          else if (u == t) z += c[k];
          else {
            rc[o] = (int32_t)reduced_index(u, s, t);
            rv[o] = c[k];
            ++o;
          }
        }
        cs[i] = a;
        ct[i] = z;
        continue;
      }
      buf.clear();
      for (int64_t k = row_ptr[v]; k < row_ptr[v + 1]; ++k) {
        const int32_t u = col[k];
        if (u == s) a += c[k];
        else if (u == t) z += c[k];
        else buf.push_back({(int32_t)reduced_index(u, s, t), c[k]});
      }
      cs[i] = a;
      ct[i] = z;
      sort_row(buf);
      int64_t o = rp[i];
      for (size_t k = 0; k < buf.size(); ++k) {
        if (k > 0 && buf[k].col == buf[k - 1].col) {
          rv[o - 1] += buf[k].c;
        } else {
          rc[o] = buf[k].col;
          rv[o] = buf[k].c;
          ++o;
        }
      }
    }
  });
  // terminal rows: c(s, v) and c(v, t) as seen from s and t.  A row whose
  // columns strictly increase has no parallel entries: filled in parallel;
  // otherwise the entries are summed in row order.
  auto fold_terminal_row = [&](int32_t term, int32_t other, hvec<double>& dst, double& c_other) {
    const int64_t b = row_ptr[term], e = row_ptr[term + 1];
    constexpr int kChunks = 64;
    uint8_t chunk_ok[kChunks];
    parallel_for(kChunks, [&](int64_t lo, int64_t hi) {
      for (int64_t ch = lo; ch < hi; ++ch) {
        const int64_t k0 = b + (e - b) * ch / kChunks, k1 = b + (e - b) * (ch + 1) / kChunks;
        uint8_t ok = 1;
        for (int64_t k = (k0 > b ? k0 : b + 1); k < k1 && ok; ++k) ok = col[k - 1] < col[k];
        chunk_ok[ch] = ok;
      }
    }, 1);
    bool strict = true;
    for (int ch = 0; ch < kChunks; ++ch) strict = strict && chunk_ok[ch];
    if (strict) {
      parallel_for(e - b, [&](int64_t lo, int64_t hi) {
        for (int64_t k = b + lo; k < b + hi; ++k)
          if (col[k] != other) dst[reduced_index(col[k], s, t)] = c[k];
      });
      for (int64_t k = b; k < e; ++k)
        if (col[k] == other) c_other += c[k];
      return;
    }
    for (int64_t k = b; k < e; ++k) {
      const int32_t u = col[k];
      if (u == other) c_other += c[k];
      else dst[reduced_index(u, s, t)] += c[k];
    }
  };
  fold_terminal_row(s, t, cs_from_s, cst_s);
  fold_terminal_row(t, s, ct_from_t, cst_t);
  // ---- symmetry: every pair carries the same total capacity in both rows
  if (cst_s != cst_t) {
    *err = "CSR is not symmetric (s-t edge)";
    return PIRMCUT_EINVAL;
  }
  hvec<uint8_t> asym(nt);
  parallel_for(nt, [&](int64_t lo, int64_t hi) {
    for (int64_t i = lo; i < hi; ++i)
      asym[i] = (cs[i] != cs_from_s[i] || ct[i] != ct_from_t[i]) ? 1 : 0;
  });
  {
    const int64_t i = parallel_find_first(nt, [&](int64_t k) { return asym[k] != 0; });
    if (i < nt) {
      *err = "CSR is not symmetric (terminal edge of vertex " +
             std::to_string(original_index(i, s, t)) + ")";
      return PIRMCUT_EINVAL;
    }
  }
  parallel_for(nt, [&](int64_t lo, int64_t hi) {
    for (int64_t i = lo; i < hi; ++i) {
      asym[i] = 0;
      for (int64_t k = rp[i]; k < rp[i + 1]; ++k) {
        const int64_t j = rc[k];
        const int32_t* b = rc.data() + rp[j];
        const int32_t* e = rc.data() + rp[j + 1];
        const int32_t* f = std::lower_bound(b, e, (int32_t)i);
        if (f == e || *f != i || rv[rp[j] + (f - b)] != rv[k]) {
          asym[i] = 1;
          break;
        }
      }
    }
  });
  {
    const int64_t i = parallel_find_first(nt, [&](int64_t k) { return asym[k] != 0; });
    if (i < nt) {
      *err = "CSR is not symmetric (row " + std::to_string(original_index(i, s, t)) + ")";
      return PIRMCUT_EINVAL;
    }
  }
  // ---- solvability (Prop. nonsingular): every non-terminal reaches a vertex
  // with a positive terminal capacity through positive-capacity edges.
  {
    hvec<uint8_t> seen(nt);
    parallel_for(nt, [&](int64_t lo, int64_t hi) {
      for (int64_t i = lo; i < hi; ++i) seen[i] = (cs[i] > 0.0 || ct[i] > 0.0) ? 1 : 0;
    });
    // a depth-first search from the seeds that have an unseen neighbour
    // (on meshes where every vertex has a terminal edge there is none)
    hvec<uint8_t> frontier(nt);
    parallel_for(nt, [&](int64_t lo, int64_t hi) {
      for (int64_t i = lo; i < hi; ++i) {
        frontier[i] = 0;
        if (!seen[i]) continue;
        for (int64_t k = rp[i]; k < rp[i + 1]; ++k)
          if (!seen[rc[k]] && rv[k] > 0.0) {
            frontier[i] = 1;
            break;
          }
      }
    });
    std::vector<int64_t> stack;
    if (parallel_find_first(nt, [&](int64_t k) { return frontier[k] != 0; }) < nt)
      for (int64_t i = 0; i < nt; ++i)
        if (frontier[i]) stack.push_back(i);
    while (!stack.empty()) {
      const int64_t i = stack.back();
      stack.pop_back();
      for (int64_t k = rp[i]; k < rp[i + 1]; ++k) {
        const int64_t j = rc[k];
        if (!seen[j] && rv[k] > 0.0) {
          seen[j] = 1;
          stack.push_back(j);
        }
      }
    }
    const int64_t i = parallel_find_first(nt, [&](int64_t k) { return seen[k] == 0; });
    if (i < nt) {
      *err = "disconnected: vertex " + std::to_string(original_index(i, s, t)) +
             " reaches neither s nor t through positive capacity";
      return PIRMCUT_EDISCONNECTED;
    }
  }
  g.n_edges = mnt / 2;
  g.nnz = mnt;
  g.c_st = cst_s;
  const double sc = chunked_sum(cs.data(), nt);
  g.sum_cs = sc + cst_s;
  g.cs = std::move(cs);
  g.ct = std::move(ct);

  // ---- storage choice: DIA when the upper entries use few distinct offsets
  // and fill most of those diagonals, else CSR.
  int K = 0;
  int64_t offs[kMaxDiag + 1];
  bool dia_ok = true;
  {
    // each chunk collects up to kMaxDiag + 1 distinct positive offsets
    constexpr int kChunks = 64;
    int64_t chunk_offs[kChunks][kMaxDiag + 1];
    int chunk_k[kChunks] = {0};
    parallel_for(kChunks, [&](int64_t lo, int64_t hi) {
      for (int64_t ch = lo; ch < hi; ++ch) {
        int kk = 0;
        const int64_t r0 = nt * ch / kChunks, r1 = nt * (ch + 1) / kChunks;
        for (int64_t i = r0; i < r1 && kk <= kMaxDiag; ++i) {
          for (int64_t k = rp[i]; k < rp[i + 1] && kk <= kMaxDiag; ++k) {
            const int64_t o = int64_t(rc[k]) - i;
            if (o <= 0) continue;
            int f = 0;
            while (f < kk && chunk_offs[ch][f] != o) ++f;
            if (f == kk) chunk_offs[ch][kk++] = o;
          }
        }
        chunk_k[ch] = kk;
      }
    }, /*min_per_thread=*/1);
    for (int ch = 0; ch < kChunks && dia_ok; ++ch) {
      for (int j = 0; j < chunk_k[ch] && dia_ok; ++j) {
        const int64_t o = chunk_offs[ch][j];
        int f = 0;
        while (f < K && offs[f] != o) ++f;
        if (f == K) {
          if (K == kMaxDiag) dia_ok = false;
          else offs[K++] = o;
        }
      }
    }
  }
  if (dia_ok && K > 0) {
    for (int a = 1; a < K; ++a)  // ascending; K <= kMaxDiag
      for (int b = a; b > 0 && offs[b - 1] > offs[b]; --b) std::swap(offs[b - 1], offs[b]);
    const double fill = double(g.n_edges) / (double(K) * double(nt));
    dia_ok = fill >= 0.5;
  }
  if (K == 0) dia_ok = false;
  if (format_req == PIRMCUT_FORMAT_DIA && !dia_ok) {
    *err = "DIA storage requested but the graph has more than 8 offsets or sparse diagonals";
    return PIRMCUT_EINVAL;
  }
  const bool use_dia = (format_req == PIRMCUT_FORMAT_DIA) ||
                       (format_req == PIRMCUT_FORMAT_AUTO && dia_ok);
  if (use_dia) {
    g.format = PIRMCUT_FORMAT_DIA;
    g.K = K;
    for (int k = 0; k < K; ++k) g.off[k] = offs[k];
    g.cdia.resize(size_t(K) * nt);
    parallel_fill(g.cdia.data(), int64_t(K) * nt, 0.0);
    parallel_for(nt, [&](int64_t lo, int64_t hi) {
      for (int64_t i = lo; i < hi; ++i) {
        for (int64_t k = rp[i]; k < rp[i + 1]; ++k) {
          const int64_t o = int64_t(rc[k]) - i;
          if (o <= 0) continue;
          int f = 0;
          while (g.off[f] != o) ++f;
          g.cdia[size_t(f) * nt + i] = rv[k];
        }
      }
    });
  } else {
    g.format = PIRMCUT_FORMAT_CSR;
    g.rp = std::move(rp);
    g.col = std::move(rc);
    g.cval = std::move(rv);
    const double avg = nt ? double(mnt) / double(nt) : 0.0;
    int grp = 1;
    while (grp < 32 && grp < avg) grp *= 2;
    g.group = grp;
  }
  return PIRMCUT_OK;
}

}  // namespace pirmcut
