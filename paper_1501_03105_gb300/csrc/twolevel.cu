// Two-level rounding (Section 3.3): 1-D K-means on x (centres started at 0.1
// and 0.9) gives gamma0 = c0 + 0.05 and gamma1 = c1 - 0.05; vertices with
// x <= gamma0 join t (S0), x >= gamma1 join s (S1), the rest (Sc) stay.  The
// coarse graph G_c keeps the Sc-Sc edges and contracts S1 into s_c and S0 into
// t_c (edge weights summed: the paper's four cases), and an s_c-t_c min cut of
// G_c induces the returned cut of G.
//
// On the GPU: the K-means passes (deterministic grid reductions over x), the
// S0/S1/Sc labels and the exact FP64 value of the final cut.  On the host (as
// the paper does on its root process): the contraction over the edges that
// touch Sc or join S1 to S0, and an exact max-flow on G_c (Dinic's algorithm:
// BFS levels, blocking flows by an iterative depth-first search).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "ctx.h"

namespace pirmcut {

namespace {

__global__ void __launch_bounds__(kThreads)
k_kmeans(int64_t nt, const double* __restrict__ x, double c0, double c1, double* partials,
         unsigned int* counter, double* out) {
  double s0 = 0.0, n0 = 0.0, s1 = 0.0, n1 = 0.0;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < nt;
       i += int64_t(gridDim.x) * blockDim.x) {
    const double v = x[i];
    if (fabs(v - c1) < fabs(v - c0)) {
      s1 += v;
      n1 += 1.0;
    } else {
      s0 += v;
      n0 += 1.0;
    }
  }
  double acc[4] = {s0, n0, s1, n1}, tot[4];
  if (grid_sum<4>(acc, partials, counter, tot) && threadIdx.x == 0) {
    for (int j = 0; j < 4; ++j) out[j] = tot[j];
  }
}

__global__ void k_labels(int64_t nt, const double* __restrict__ x, double g0, double g1,
                         uint8_t* __restrict__ lab) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < nt;
       i += int64_t(gridDim.x) * blockDim.x) {
    const double v = x[i];
    uint8_t l = 2;
    if (v <= g0) l = 0;
    if (v >= g1) l = 1;
    lab[i] = l;
  }
}

// Dinic's max-flow on an undirected graph (each edge two arcs of capacity c).
struct Dinic {
  struct Arc {
    int to;
    double cap;
  };
  int n;
  std::vector<Arc> arcs;
  std::vector<int> head, next_arc;
  std::vector<int> level, it;
  double tiny = 0.0;

  explicit Dinic(int nv) : n(nv), head(nv, -1), level(nv), it(nv) {}

  void add(int u, int v, double c) {
    arcs.push_back({v, c});
    next_arc.push_back(head[u]);
    head[u] = int(arcs.size()) - 1;
    arcs.push_back({u, c});
    next_arc.push_back(head[v]);
    head[v] = int(arcs.size()) - 1;
  }

  bool bfs(int s, int t) {
    std::fill(level.begin(), level.end(), -1);
    std::vector<int> q;
    q.reserve(n);
    q.push_back(s);
    level[s] = 0;
    for (size_t k = 0; k < q.size(); ++k) {
      const int u = q[k];
      for (int a = head[u]; a >= 0; a = next_arc[a])
        if (arcs[a].cap > tiny && level[arcs[a].to] < 0) {
          level[arcs[a].to] = level[u] + 1;
          q.push_back(arcs[a].to);
        }
    }
    return level[t] >= 0;
  }

  // one augmenting path along increasing levels (iterative DFS with current-arc pointers)
  double augment(int s, int t) {
    std::vector<int> path;  // arcs
    int u = s;
    while (true) {
      if (u == t) {
        double f = INFINITY;
        for (int a : path) f = std::min(f, arcs[a].cap);
        for (int a : path) {
          arcs[a].cap -= f;
          arcs[a ^ 1].cap += f;
        }
        return f;
      }
      int& a = it[u];
      while (a >= 0 && !(arcs[a].cap > tiny && level[arcs[a].to] == level[u] + 1)) a = next_arc[a];
      if (a >= 0) {
        path.push_back(a);
        u = arcs[a].to;
      } else {
        level[u] = -1;  // dead end
        if (path.empty()) return 0.0;
        const int back = path.back();
        path.pop_back();
        u = arcs[back ^ 1].to;
        it[u] = next_arc[it[u]];
      }
    }
  }

  double maxflow(int s, int t) {
    double cmax = 0.0;
    for (const Arc& a : arcs) cmax = std::max(cmax, a.cap);
    tiny = 1e-12 * cmax;
    double flow = 0.0;
    while (bfs(s, t)) {
      for (int v = 0; v < n; ++v) it[v] = head[v];
      for (double f; (f = augment(s, t)) > 0.0;) flow += f;
    }
    return flow;
  }

  // vertices reachable from s in the residual graph
  std::vector<uint8_t> source_side(int s) {
    std::vector<uint8_t> seen(n, 0);
    std::vector<int> q{s};
    seen[s] = 1;
    for (size_t k = 0; k < q.size(); ++k)
      for (int a = head[q[k]]; a >= 0; a = next_arc[a])
        if (arcs[a].cap > tiny && !seen[arcs[a].to]) {
          seen[arcs[a].to] = 1;
          q.push_back(arcs[a].to);
        }
    return seen;
  }
};

}  // namespace

}  // namespace pirmcut

extern "C" pirmcut_status pirmcut_cut_two_level(pirmcut_ctx* h, uint8_t* side, double* value,
                                                double* gamma, int64_t* coarse_vertices,
                                                int mem_kind) {
  using namespace pirmcut;
  if (!h) {
    set_global_error("ctx is NULL");
    return PIRMCUT_EINVAL;
  }
  Ctx& c = h->c;
  auto fail = [&](pirmcut_status st, const std::string& m) {
    c.err = m;
    return st;
  };
  auto cuda = [&](cudaError_t e, const char* w) {
    return fail(e == cudaErrorMemoryAllocation ? PIRMCUT_ENOMEM : PIRMCUT_ECUDA,
                std::string(w) + ": " + cudaGetErrorString(e));
  };
  if (!c.x_set) return fail(PIRMCUT_EINVAL, "x is not set");
  if (mem_kind != PIRMCUT_MEM_HOST && mem_kind != PIRMCUT_MEM_DEVICE)
    return fail(PIRMCUT_EINVAL, "unknown mem_kind");
  cudaError_t e = sweep_alloc(c);
  if (e != cudaSuccess) return cuda(e, "sweep buffers");
  // the contraction reads the reduced graph on the host: a problem built on
  // the device is copied back once
  if (c.device_reduced && c.hg.cs.empty() && c.nt > 0) {
    HostGraph& hg = c.hg;
    const size_t nt = size_t(c.nt);
    hg.cs.resize(nt);
    hg.ct.resize(nt);
    e = cudaMemcpyAsync(hg.cs.data(), c.cs, sizeof(double) * nt, cudaMemcpyDeviceToHost, c.stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hg.ct.data(), c.ct, sizeof(double) * nt, cudaMemcpyDeviceToHost, c.stream);
    if (c.format == PIRMCUT_FORMAT_DIA) {
      hg.cdia.resize(size_t(c.K) * nt);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(hg.cdia.data(), c.cdia, sizeof(double) * hg.cdia.size(), cudaMemcpyDeviceToHost, c.stream);
    } else {
      hg.rp.resize(nt + 1);
      hg.col.resize(size_t(hg.nnz));
      hg.cval.resize(size_t(hg.nnz));
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(hg.rp.data(), c.rp, sizeof(int64_t) * (nt + 1), cudaMemcpyDeviceToHost, c.stream);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(hg.col.data(), c.col, sizeof(int32_t) * hg.col.size(), cudaMemcpyDeviceToHost, c.stream);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(hg.cval.data(), c.cval, sizeof(double) * hg.cval.size(), cudaMemcpyDeviceToHost, c.stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
    if (e != cudaSuccess) {
      hg.cs.clear();
      return cuda(e, "reading the reduced graph");
    }
  }
  const HostGraph& g = c.hg;
  const int64_t nt = c.nt;
  // --- K-means on x (s and t included: x_s = 1, x_t = 0)
  double* out = c.sw.blk;           // 4 doubles (the sweep scratch holds >= 2 * kMaxBlocks)
  double* partials = c.partials;    // 4 * kMaxBlocks, as grid_sum<4> needs
  unsigned int* counter = reinterpret_cast<unsigned int*>(c.sw.result + 4) + 2;
  double c0 = 0.1, c1 = 0.9;
  for (int iter = 0; iter < 100; ++iter) {
    k_kmeans<<<grid_for(nt), kThreads, 0, c.stream>>>(nt, c.x, c0, c1, partials, counter, out);
    c.launches += 1;
    double tot[4];
    if ((e = cudaMemcpyAsync(tot, out, sizeof(tot), cudaMemcpyDeviceToHost, c.stream)) != cudaSuccess ||
        (e = cudaStreamSynchronize(c.stream)) != cudaSuccess)
      return cuda(e, "k-means");
    for (double v : {1.0, 0.0}) {  // the terminals
      if (std::fabs(v - c1) < std::fabs(v - c0)) {
        tot[2] += v;
        tot[3] += 1.0;
      } else {
        tot[0] += v;
        tot[1] += 1.0;
      }
    }
    const double nc0 = tot[1] > 0.0 ? tot[0] / tot[1] : c0;
    const double nc1 = tot[3] > 0.0 ? tot[2] / tot[3] : c1;
    const bool same = nc0 == c0 && nc1 == c1;
    c0 = nc0;
    c1 = nc1;
    if (same) break;
  }
  const double g0 = c0 + 0.05, g1 = c1 - 0.05;
  // --- labels
  uint8_t* lab_d = c.sw.side_red;  // reused: labels first, then the final side
  k_labels<<<grid_for(nt), kThreads, 0, c.stream>>>(nt, c.x, g0, g1, lab_d);
  c.launches += 1;
  std::vector<uint8_t> lab(static_cast<size_t>(nt));
  if ((e = cudaMemcpyAsync(lab.data(), lab_d, size_t(nt), cudaMemcpyDeviceToHost, c.stream)) != cudaSuccess ||
      (e = cudaStreamSynchronize(c.stream)) != cudaSuccess)
    return cuda(e, "labels");
  // --- contraction (host): Sc vertices keep their order
  std::vector<int64_t> cid(static_cast<size_t>(nt), -1);
  int64_t nsc = 0;
  for (int64_t i = 0; i < nt; ++i)
    if (lab[i] == 2) cid[i] = nsc++;
  if (nsc + 2 > (int64_t(1) << 31) - 1) return fail(PIRMCUT_EINVAL, "coarse graph too large");
  const int sC = int(nsc), tC = int(nsc + 1);
  std::vector<double> ws(static_cast<size_t>(nsc), 0.0), wt(static_cast<size_t>(nsc), 0.0);
  double wst = g.c_st;
  std::vector<std::pair<std::pair<int, int>, double>> inner;
  auto edge = [&](int64_t i, int64_t j, double w) {
    const int li = lab[i], lj = lab[j];
    if (li == 2 && lj == 2) inner.push_back({{int(cid[i]), int(cid[j])}, w});
    else if (li == 2) (lj == 1 ? ws : wt)[cid[i]] += w;
    else if (lj == 2) (li == 1 ? ws : wt)[cid[j]] += w;
    else if (li != lj) wst += w;
  };
  if (c.format == PIRMCUT_FORMAT_DIA) {
    for (int k = 0; k < g.K; ++k)
      for (int64_t i = 0; i + g.off[k] < nt; ++i) {
        const double w = g.cdia[size_t(k) * nt + i];
        if (w != 0.0) edge(i, i + g.off[k], w);
      }
  } else {
    for (int64_t i = 0; i < nt; ++i)
      for (int64_t e2 = g.rp[i]; e2 < g.rp[i + 1]; ++e2)
        if (g.col[e2] > i) edge(i, g.col[e2], g.cval[e2]);
  }
  for (int64_t i = 0; i < nt; ++i) {  // terminal edges: s in S1, t in S0
    const int li = lab[i];
    if (li == 2) {
      ws[cid[i]] += g.cs[i];
      wt[cid[i]] += g.ct[i];
    } else if (li == 0) {
      wst += g.cs[i];
    } else {
      wst += g.ct[i];
    }
  }
  Dinic mf(int(nsc + 2));
  for (const auto& ed : inner) mf.add(ed.first.first, ed.first.second, ed.second);
  for (int64_t u = 0; u < nsc; ++u) {
    if (ws[u] > 0.0) mf.add(int(u), sC, ws[u]);
    if (wt[u] > 0.0) mf.add(int(u), tC, wt[u]);
  }
  if (wst > 0.0) mf.add(sC, tC, wst);
  mf.maxflow(sC, tC);
  const std::vector<uint8_t> cside = mf.source_side(sC);
  // --- induced side, exact value on the GPU
  std::vector<uint8_t> sred(static_cast<size_t>(nt));
  for (int64_t i = 0; i < nt; ++i) sred[i] = lab[i] == 1 || (lab[i] == 2 && cside[cid[i]]);
  if ((e = cudaMemcpyAsync(lab_d, sred.data(), size_t(nt), cudaMemcpyHostToDevice, c.stream)) != cudaSuccess)
    return cuda(e, "side");
  if ((e = enqueue_cut_value(c, c.stream, lab_d)) != cudaSuccess) return cuda(e, "cut value");
  c.launches += 1;
  if (side && mem_kind == PIRMCUT_MEM_DEVICE) {
    if ((e = launch_side_full(c, side)) != cudaSuccess) return cuda(e, "side");
  }
  double res[4];
  if ((e = cudaMemcpyAsync(res, c.sw.result, sizeof(res), cudaMemcpyDeviceToHost, c.stream)) != cudaSuccess ||
      (e = cudaStreamSynchronize(c.stream)) != cudaSuccess)
    return cuda(e, "result");
  if (side && mem_kind == PIRMCUT_MEM_HOST) {
    for (int64_t i = 0; i < nt; ++i) side[original_index(i, g.s, g.t)] = sred[i];
    side[g.s] = 1;
    side[g.t] = 0;
  }
  if (value) *value = res[1];
  if (gamma) {
    gamma[0] = g0;
    gamma[1] = g1;
  }
  if (coarse_vertices) *coarse_vertices = nsc + 2;
  return PIRMCUT_OK;
}
