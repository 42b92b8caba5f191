// extern "C" entry points of libpirmcut (declared in include/pirmcut.h).
#include <cuda_runtime.h>

#include <cmath>
#include <cstddef>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "ctx.h"
#include "pirmcut.h"


namespace {

thread_local std::string g_create_error;

using pirmcut::Ctx;

pirmcut_status fail(pirmcut_ctx* h, pirmcut_status st, const std::string& msg) {
  if (h) h->c.err = msg;
  else g_create_error = msg;
  return st;
}

pirmcut_status cuda_fail(pirmcut_ctx* h, cudaError_t e, const char* where) {
  return fail(h, e == cudaErrorMemoryAllocation ? PIRMCUT_ENOMEM : PIRMCUT_ECUDA,
              std::string(where) + ": " + cudaGetErrorString(e));
}

#define CK(h, call, where)                          \
  do {                                              \
    cudaError_t e_ = (call);                        \
    if (e_ != cudaSuccess) return cuda_fail(h, e_, where); \
  } while (0)

template <class T>
cudaError_t dalloc(T** p, size_t count) {
  if (count == 0) count = 1;
  return cudaMalloc((void**)p, sizeof(T) * count);
}

void free_device(Ctx& c) {
  void* ps[] = {c.cdia, c.gdia, c.rp, c.col, c.cval, c.gval, c.cs, c.ct, c.x, c.r, c.p,
                c.q, c.diag, c.rsd, c.sq32, c.xs, c.ghat, c.xstats, c.heavy, c.partials, c.S, c.C,
                c.eps_list,
                c.recs, c.xfull, c.side_full, c.d_in_rp, c.d_in_col};
  for (void* p : ps)
    if (p) cudaFree(p);
  pirmcut::sweep_free(c);
  pirmcut::mixed_free(c);
  pirmcut::mlp_free(c);
  if (c.g_init) cudaGraphExecDestroy(c.g_init);
  if (c.g_step) cudaGraphExecDestroy(c.g_step);
  if (c.g_cut) cudaGraphExecDestroy(c.g_cut);
  if (c.cap_stream) cudaStreamDestroy(c.cap_stream);
  for (cudaEvent_t ev : c.spmv_ev) cudaEventDestroy(ev);
  c.spmv_ev.clear();
  if (c.h_recs) cudaFreeHost(c.h_recs);
}

pirmcut_status check_options(const pirmcut_options& o, std::string* msg) {
  if (o.reweight_form != PIRMCUT_REWEIGHT_WEIGHTED_L1 && o.reweight_form != PIRMCUT_REWEIGHT_PAPER) {
    *msg = "unknown reweight_form";
    return PIRMCUT_EINVAL;
  }
  if (o.precision != PIRMCUT_PREC_FP64 && o.precision != PIRMCUT_PREC_MIXED) {
    *msg = "unknown precision";
    return PIRMCUT_EINVAL;
  }
  if (o.precision == PIRMCUT_PREC_MIXED && (!(o.inner_tol > 0.0) || !(o.inner_tol < 1.0))) {
    *msg = "inner_tol must be in (0, 1)";
    return PIRMCUT_EINVAL;
  }
  if (!(o.pcg_tol > 0.0) || !std::isfinite(o.pcg_tol)) {
    *msg = "pcg_tol must be finite and > 0";
    return PIRMCUT_EINVAL;
  }
  if (o.pcg_max_iter < 0 || o.pcg_max_iter > 100000000) {
    *msg = "pcg_max_iter must be in [0, 1e8]";
    return PIRMCUT_EINVAL;
  }
  if (o.graph_launch != 0 && o.graph_launch != 1) {
    *msg = "graph_launch must be 0 or 1";
    return PIRMCUT_EINVAL;
  }
  if (o.format < PIRMCUT_FORMAT_AUTO || o.format > PIRMCUT_FORMAT_CSR) {
    *msg = "unknown format";
    return PIRMCUT_EINVAL;
  }
  if (o.capacity_fp32 != 0 && o.capacity_fp32 != 1) {
    *msg = "capacity_fp32 must be 0 or 1";
    return PIRMCUT_EINVAL;
  }
  if (o.step_stats != 0 && o.step_stats != 1) {
    *msg = "step_stats must be 0 or 1";
    return PIRMCUT_EINVAL;
  }
  return PIRMCUT_OK;
}

// copy a caller buffer (host or device) into a host vector
template <class T>
cudaError_t to_host(pirmcut::hvec<T>& dst, const T* src, size_t count, int mem_kind) {
  dst.resize(count);
  if (count == 0) return cudaSuccess;
  if (mem_kind == PIRMCUT_MEM_DEVICE)
    return cudaMemcpy(dst.data(), src, sizeof(T) * count, cudaMemcpyDeviceToHost);
  pirmcut::parallel_copy(dst.data(), src, int64_t(count));
  return cudaSuccess;
}

// The capacities as doubles on the host for the host reduction: read in
// place (host doubles), copied (device doubles), or widened exactly from
// floats (options.capacity_fp32), in parallel.
cudaError_t host_capacities(pirmcut::hvec<double>& buf, const void* c, int fp32, size_t nnz,
                            int mem_kind, const double** out) {
  if (!fp32) {
    if (mem_kind != PIRMCUT_MEM_DEVICE) {
      *out = static_cast<const double*>(c);
      return cudaSuccess;
    }
    cudaError_t e = to_host(buf, static_cast<const double*>(c), nnz, mem_kind);
    *out = buf.data();
    return e;
  }
  pirmcut::hvec<float> f;
  const float* src = static_cast<const float*>(c);
  if (mem_kind == PIRMCUT_MEM_DEVICE) {
    cudaError_t e = to_host(f, src, nnz, mem_kind);
    if (e != cudaSuccess) return e;
    src = f.data();
  }
  buf.resize(nnz);
  double* dst = buf.data();
  pirmcut::parallel_for(int64_t(nnz), [=](int64_t lo, int64_t hi) {
    for (int64_t k = lo; k < hi; ++k) dst[k] = double(src[k]);
  }, 1 << 20);
  *out = buf.data();
  return cudaSuccess;
}

pirmcut_status upload_problem(pirmcut_ctx* h) {
  Ctx& c = h->c;
  const pirmcut::HostGraph& g = c.hg;
  cudaStream_t st = c.stream;
  // the conductances start as the capacities (W^(0) = C): a defined g^(l-1)
  // for the first step even when x is set by the caller
  if (c.device_reduced) {  // built in place on the device
    if (c.format == PIRMCUT_FORMAT_DIA)
      CK(h, cudaMemcpyAsync(c.gdia, c.cdia, sizeof(double) * size_t(c.K) * size_t(c.nt), cudaMemcpyDeviceToDevice, st), "upload");
    else
      CK(h, cudaMemcpyAsync(c.gval, c.cval, sizeof(double) * size_t(g.nnz), cudaMemcpyDeviceToDevice, st), "upload");
    CK(h, cudaStreamSynchronize(st), "upload");
    return PIRMCUT_OK;
  }
  if (c.format == PIRMCUT_FORMAT_DIA) {
    CK(h, cudaMemcpyAsync(c.cdia, g.cdia.data(), sizeof(double) * g.cdia.size(), cudaMemcpyHostToDevice, st), "upload");
    CK(h, cudaMemcpyAsync(c.gdia, c.cdia, sizeof(double) * g.cdia.size(), cudaMemcpyDeviceToDevice, st), "upload");
  } else {
    CK(h, cudaMemcpyAsync(c.rp, g.rp.data(), sizeof(int64_t) * g.rp.size(), cudaMemcpyHostToDevice, st), "upload");
    CK(h, cudaMemcpyAsync(c.col, g.col.data(), sizeof(int32_t) * g.col.size(), cudaMemcpyHostToDevice, st), "upload");
    CK(h, cudaMemcpyAsync(c.cval, g.cval.data(), sizeof(double) * g.cval.size(), cudaMemcpyHostToDevice, st), "upload");
    CK(h, cudaMemcpyAsync(c.gval, c.cval, sizeof(double) * g.cval.size(), cudaMemcpyDeviceToDevice, st), "upload");
  }
  CK(h, cudaMemcpyAsync(c.cs, g.cs.data(), sizeof(double) * g.cs.size(), cudaMemcpyHostToDevice, st), "upload");
  CK(h, cudaMemcpyAsync(c.ct, g.ct.data(), sizeof(double) * g.ct.size(), cudaMemcpyHostToDevice, st), "upload");
  CK(h, cudaStreamSynchronize(st), "upload");
  return PIRMCUT_OK;
}

pirmcut_status ensure_capacity(pirmcut_ctx* h, int steps) {
  Ctx& c = h->c;
  if (c.eps_cap < steps) {
    if (c.eps_list) cudaFree(c.eps_list);
    c.eps_list = nullptr;
    c.eps_cap = 0;
    int cap = 64;
    while (cap < steps) cap *= 2;
    CK(h, dalloc(&c.eps_list, cap), "eps buffer");
    c.eps_cap = cap;
    // graphs bake the eps pointer: rebuild
    if (c.g_init) { cudaGraphExecDestroy(c.g_init); c.g_init = nullptr; }
    if (c.g_step) { cudaGraphExecDestroy(c.g_step); c.g_step = nullptr; }
  }
  if (c.rec_cap < steps + 1) {
    if (c.recs) cudaFree(c.recs);
    c.recs = nullptr;
    c.rec_cap = 0;
    int cap = 64;
    while (cap < steps + 1) cap *= 2;
    CK(h, dalloc(&c.recs, cap), "record buffer");
    c.rec_cap = cap;
    if (c.h_recs) cudaFreeHost(c.h_recs);
    c.h_recs = nullptr;
    CK(h, cudaHostAlloc((void**)&c.h_recs, sizeof(pirmcut::StepRec) * cap, cudaHostAllocDefault), "record buffer");
    c.h_rec_cap = cap;
    if (c.g_init) { cudaGraphExecDestroy(c.g_init); c.g_init = nullptr; }
    if (c.g_step) { cudaGraphExecDestroy(c.g_step); c.g_step = nullptr; }
    if (c.g_cut) { cudaGraphExecDestroy(c.g_cut); c.g_cut = nullptr; }
  }
  return PIRMCUT_OK;
}

pirmcut_status ensure_graphs(pirmcut_ctx* h, bool need_cut) {
  Ctx& c = h->c;
  const bool mixed = c.opt.precision == PIRMCUT_PREC_MIXED;
  if (!c.g_init)
    CK(h, mixed ? pirmcut::build_step_graph_mixed(c, true, &c.g_init, &c.nodes_init)
                : pirmcut::build_step_graph(c, true, &c.g_init, &c.nodes_init), "building the x0 graph");
  if (!c.g_step)
    CK(h, mixed ? pirmcut::build_step_graph_mixed(c, false, &c.g_step, &c.nodes_step)
                : pirmcut::build_step_graph(c, false, &c.g_step, &c.nodes_step), "building the step graph");
  if (need_cut) {
    CK(h, pirmcut::sweep_alloc(c), "sweep buffers");
    if (!c.g_cut) CK(h, pirmcut::build_cut_graph(c, &c.g_cut, &c.nodes_cut), "building the sweep graph");
  }
  return PIRMCUT_OK;
}

cudaEvent_t event_at(pirmcut_ctx* h, size_t i) {
  while (h->events.size() <= i) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    h->events.push_back(e);
  }
  return h->events[i];
}

void fill_info(const Ctx& c, const pirmcut::StepRec& r, float ms, pirmcut_step_info* info) {
  info->step = r.step;
  info->pcg_iters = r.iters;
  info->eps = r.eps;
  info->rel_residual = r.bb > 0.0 ? std::sqrt(r.rr / r.bb) : 0.0;
  info->x_min = r.xmin;
  info->x_max = r.xmax;
  info->cut_value = r.cut;
  info->ms = ms;
  int st = r.status;
  if (st == PIRMCUT_OK && r.bb > 0.0 && !(r.rr <= c.opt.pcg_tol * c.opt.pcg_tol * r.bb))
    st = PIRMCUT_ENOCONV;
  info->status = st;
  info->refinements = r.refine;
  info->objective = r.obj;
  info->flow_value = r.flow;
}

// Run x^(0) (when with_initial) and the eps steps already in eps_list[0..T).
pirmcut_status run_steps(pirmcut_ctx* h, bool with_initial, int T, int first_step,
                         pirmcut_step_info* infos) {
  Ctx& c = h->c;
  const int nrec = T + (with_initial ? 1 : 0);
  if (nrec == 0) return PIRMCUT_OK;
  const bool graphs = c.opt.graph_launch != 0;
  pirmcut_status ps = graphs ? ensure_graphs(h, c.opt.track_cut != 0) : PIRMCUT_OK;
  if (ps == PIRMCUT_OK && !graphs && c.opt.track_cut) {
    CK(h, pirmcut::sweep_alloc(c), "sweep buffers");
    if (!c.g_cut) CK(h, pirmcut::build_cut_graph(c, &c.g_cut, &c.nodes_cut), "building the sweep graph");
  }
  if (ps != PIRMCUT_OK) return ps;
  h->h_ctr->eps_idx = 0;
  h->h_ctr->rec_idx = 0;
  h->h_ctr->step = first_step;
  h->h_ctr->pad = 0;
  CK(h, cudaMemcpyAsync(c.C, h->h_ctr, sizeof(pirmcut::StepCounters), cudaMemcpyHostToDevice, c.stream), "counters");
  cudaEvent_t e0 = event_at(h, 0);
  if (!e0) return fail(h, PIRMCUT_ECUDA, "cudaEventCreate failed");
  CK(h, cudaEventRecord(e0, c.stream), "event");
  for (int k = 0; k < nrec; ++k) {
    const bool init = with_initial && k == 0;
    if (graphs) {
      CK(h, cudaGraphLaunch(init ? c.g_init : c.g_step, c.stream), "graph launch");
      c.launches += init ? c.nodes_init : c.nodes_step;
    } else {
      int64_t kernels = 0;
      if (c.opt.precision == PIRMCUT_PREC_MIXED) {
        CK(h, pirmcut::run_step_stream_mixed(c, init, h->h_stop, &kernels), "step launch");
      } else {
        CK(h, pirmcut::run_step_stream(c, init, h->h_stop, &kernels), "step launch");
      }
      c.launches += kernels;
    }
    if (c.opt.track_cut) {
      CK(h, cudaGraphLaunch(c.g_cut, c.stream), "graph launch");
      c.launches += c.nodes_cut;
    }
    cudaEvent_t ek = event_at(h, size_t(k) + 1);
    if (!ek) return fail(h, PIRMCUT_ECUDA, "cudaEventCreate failed");
    CK(h, cudaEventRecord(ek, c.stream), "event");
  }
  CK(h, cudaMemcpyAsync(c.h_recs, c.recs, sizeof(pirmcut::StepRec) * nrec, cudaMemcpyDeviceToHost, c.stream), "records");
  CK(h, cudaStreamSynchronize(c.stream), "solve");
  pirmcut_status worst = PIRMCUT_OK;
  for (int k = 0; k < nrec; ++k) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, h->events[k], h->events[k + 1]);
    pirmcut_step_info info;
    fill_info(c, c.h_recs[k], ms, &info);
    if (graphs) {
      // kernels inside the graphs' loops: three per CG iteration, two with the
      // fused recurrence (whose loop body holds two iterations, so a solve with
      // an odd count also runs one pair of no-op kernels), plus the residual
      // and the x update per refinement
      if (c.fused_inner && c.opt.precision == PIRMCUT_PREC_MIXED)
        c.launches += 2LL * info.pcg_iters + 3LL * info.refinements;
      else
        c.launches += 3LL * info.pcg_iters + 2LL * info.refinements;
    }
    if (infos) infos[k] = info;
    if (info.status == PIRMCUT_ENUMERIC) worst = PIRMCUT_ENUMERIC;
    else if (info.status == PIRMCUT_ENOCONV && worst == PIRMCUT_OK) worst = PIRMCUT_ENOCONV;
  }
  c.x_set = true;
  if (worst == PIRMCUT_ENUMERIC) return fail(h, worst, "NaN/Inf or loss of positive definiteness in PCG");
  if (worst == PIRMCUT_ENOCONV) return fail(h, worst, "PCG reached pcg_max_iter");
  return PIRMCUT_OK;
}

// Everything after the reduction: device arrays, staging, the upload (or
// adoption of arrays the device reduction built), the step buffers.
pirmcut_status finish_create(pirmcut_ctx* h, const pirmcut_options& o, void* stream,
                             pirmcut::DeviceGraph* dg, pirmcut_ctx** out) {
  Ctx& cx = h->c;
  cudaError_t e = cudaSuccess;
  if (dg) {  // the problem arrays were built on the device: adopt them (freed with cx)
    cx.cdia = dg->cdia;
    cx.rp = dg->rp;
    cx.col = dg->col;
    cx.cval = dg->cval;
    cx.cs = dg->cs;
    cx.ct = dg->ct;
    cx.d_in_rp = dg->in_rp;
    cx.d_in_col = dg->in_col;
    *dg = pirmcut::DeviceGraph();
    cx.device_reduced = true;
  }
  cx.opt = o;
  cx.nt = cx.hg.nt;
  cx.format = cx.hg.format;
  cx.K = cx.hg.K;
  cx.dd.nt = cx.nt;
  for (int k = 0; k < pirmcut::kMaxDiag; ++k) cx.dd.off[k] = cx.hg.off[k];
  cx.group = cx.hg.group;
  cx.stream = reinterpret_cast<cudaStream_t>(stream);
  auto bail = [&](cudaError_t err, const char* where) {
    std::string m = std::string(where) + ": " + cudaGetErrorString(err);
    free_device(cx);
    if (h->h_ctr) cudaFreeHost(h->h_ctr);
    delete h;
    return fail(nullptr, err == cudaErrorMemoryAllocation ? PIRMCUT_ENOMEM : PIRMCUT_ECUDA, m);
  };
  if ((e = cudaGetDevice(&cx.device)) != cudaSuccess) return bail(e, "cudaGetDevice");
  if ((e = cudaStreamCreateWithFlags(&cx.cap_stream, cudaStreamNonBlocking)) != cudaSuccess)
    return bail(e, "cudaStreamCreate");
  const size_t nt = size_t(cx.nt);
  const size_t m = size_t(cx.hg.nnz);
  if (!cx.device_reduced) {
    if (cx.format == PIRMCUT_FORMAT_DIA) {
      if ((e = dalloc(&cx.cdia, size_t(cx.K) * nt)) != cudaSuccess) return bail(e, "cudaMalloc");
    } else {
      if ((e = dalloc(&cx.rp, nt + 1)) != cudaSuccess) return bail(e, "cudaMalloc");
      if ((e = dalloc(&cx.col, m)) != cudaSuccess) return bail(e, "cudaMalloc");
      if ((e = dalloc(&cx.cval, m)) != cudaSuccess) return bail(e, "cudaMalloc");
    }
    if ((e = dalloc(&cx.cs, nt)) != cudaSuccess) return bail(e, "cudaMalloc");
    if ((e = dalloc(&cx.ct, nt)) != cudaSuccess) return bail(e, "cudaMalloc");
  }
  if (cx.format == PIRMCUT_FORMAT_DIA) {
    if ((e = dalloc(&cx.gdia, size_t(cx.K) * nt)) != cudaSuccess) return bail(e, "cudaMalloc");
  } else {
    if ((e = dalloc(&cx.gval, m)) != cudaSuccess) return bail(e, "cudaMalloc");
  }
  double** vecs[] = {&cx.x, &cx.r, &cx.p, &cx.q, &cx.diag};
  for (double** v : vecs)
    if ((e = dalloc(v, nt)) != cudaSuccess) return bail(e, "cudaMalloc");
  if (o.step_stats && (e = dalloc(&cx.xstats, nt)) != cudaSuccess) return bail(e, "cudaMalloc");
  if (o.precision == PIRMCUT_PREC_FP64) {
    if ((e = dalloc(&cx.rsd, nt)) != cudaSuccess) return bail(e, "cudaMalloc");
    if ((e = dalloc(&cx.xs, nt)) != cudaSuccess) return bail(e, "cudaMalloc");
    if ((e = dalloc(&cx.sq32, nt)) != cudaSuccess) return bail(e, "cudaMalloc");
    if ((e = dalloc(&cx.ghat, cx.format == PIRMCUT_FORMAT_DIA ? size_t(cx.K) * nt : size_t(m))) != cudaSuccess)
      return bail(e, "cudaMalloc");
  }
  if ((e = dalloc(&cx.partials, 4 * size_t(pirmcut::kMaxBlocks + pirmcut::kHeavyRowsMax))) != cudaSuccess)
    return bail(e, "cudaMalloc");
  if ((e = dalloc(&cx.S, 1)) != cudaSuccess) return bail(e, "cudaMalloc");
  if ((e = dalloc(&cx.C, 1)) != cudaSuccess) return bail(e, "cudaMalloc");
  if ((e = cudaMemset(cx.S, 0, sizeof(pirmcut::PcgState))) != cudaSuccess) return bail(e, "cudaMemset");
  if (o.precision == PIRMCUT_PREC_MIXED && (e = pirmcut::mixed_alloc(cx)) != cudaSuccess)
    return bail(e, "cudaMalloc");
  if ((e = cudaMemset(cx.C, 0, sizeof(pirmcut::StepCounters))) != cudaSuccess) return bail(e, "cudaMemset");
  if ((e = cudaHostAlloc((void**)&h->h_ctr, sizeof(pirmcut::StepCounters) + 10 * sizeof(double),
                         cudaHostAllocDefault)) != cudaSuccess)
    return bail(e, "cudaHostAlloc");
  h->h_eps = reinterpret_cast<double*>(h->h_ctr + 1);
  h->h_result = h->h_eps + 2;
  h->h_stop = reinterpret_cast<int*>(h->h_eps + 7);
  pirmcut_status ps = upload_problem(h);
  if (ps != PIRMCUT_OK) {
    std::string m = cx.err;
    free_device(cx);
    cudaFreeHost(h->h_ctr);
    delete h;
    return fail(nullptr, ps, m);
  }
  ps = ensure_capacity(h, 1);
  if (ps == PIRMCUT_OK && cx.format == PIRMCUT_FORMAT_CSR) {
    // rows far longer than the mean get a block each in the per-row kernels
    if (!cx.hg.rp.empty()) {
      e = pirmcut::set_heavy_rows(cx, cx.hg.rp.data());
    } else {
      pirmcut::hvec<int64_t> hrp(nt + 1);  // problem built on the device: its row pointers
      e = cudaMemcpy(hrp.data(), cx.rp, sizeof(int64_t) * (nt + 1), cudaMemcpyDeviceToHost);
      if (e == cudaSuccess) e = pirmcut::set_heavy_rows(cx, hrp.data());
    }
    if (e != cudaSuccess) {
      cx.err = std::string("heavy rows: ") + cudaGetErrorString(e);
      ps = PIRMCUT_ECUDA;
    }
  }
  if (ps != PIRMCUT_OK) {
    std::string m = cx.err;
    free_device(cx);
    cudaFreeHost(h->h_ctr);
    delete h;
    return fail(nullptr, ps, m);
  }
  *out = h;
  return PIRMCUT_OK;
}

pirmcut_status create_from_device(int64_t n, const pirmcut_options& o, void* stream,
                                  pirmcut::HostGraph&& g, pirmcut::DeviceGraph& dg, pirmcut_ctx** out) {
  (void)n;
  pirmcut_ctx* h = new (std::nothrow) pirmcut_ctx();
  if (!h) {
    dg.release();
    return fail(nullptr, PIRMCUT_ENOMEM, "out of host memory");
  }
  h->c.hg = std::move(g);
  return finish_create(h, o, stream, &dg, out);
}

}  // namespace

namespace pirmcut {
void set_global_error(const std::string& msg) { g_create_error = msg; }

cudaEvent_t* spmv_events(Ctx& c, int pairs) {
  while (c.spmv_ev.size() < size_t(2 * pairs)) {
    cudaEvent_t ev;
    if (cudaEventCreate(&ev) != cudaSuccess) return nullptr;
    c.spmv_ev.push_back(ev);
  }
  return c.spmv_ev.data();
}

void spmv_events_collect(Ctx& c, int pairs, int executed) {
  if (executed > pairs) executed = pairs;
  for (int j = 0; j < executed; ++j) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, c.spmv_ev[2 * j], c.spmv_ev[2 * j + 1]) == cudaSuccess) {
      c.spmv_ms += ms;
      c.spmv_count += 1;
    }
  }
}
}  // namespace pirmcut

extern "C" {

void pirmcut_default_options(pirmcut_options* opt) {
  if (!opt) return;
  opt->reweight_form = PIRMCUT_REWEIGHT_WEIGHTED_L1;
  opt->precision = PIRMCUT_PREC_FP64;
  opt->pcg_tol = 1e-10;
  opt->pcg_max_iter = 20000;
  opt->warm_start = 1;
  opt->format = PIRMCUT_FORMAT_AUTO;
  opt->track_cut = 0;
  opt->graph_launch = 1;
  opt->inner_tol = 1e-5;
  opt->time_spmv = 0;
  opt->reduce_on_host = 0;
  opt->batch_threads_per_row = 0;
  opt->batch_tile_rows = 0;
  opt->batch_medium_deg = 0;
  opt->step_stats = 0;
  opt->capacity_fp32 = 0;
  opt->fuse_reweight = 0;
}

pirmcut_status pirmcut_create(int64_t n, const int64_t* row_ptr, const int32_t* col,
                              const void* c, int32_t s, int32_t t,
                              const pirmcut_options* opt, int mem_kind, void* stream,
                              pirmcut_ctx** out) {
  if (!out) return fail(nullptr, PIRMCUT_EINVAL, "out must not be NULL");
  *out = nullptr;
  if (mem_kind != PIRMCUT_MEM_HOST && mem_kind != PIRMCUT_MEM_DEVICE)
    return fail(nullptr, PIRMCUT_EINVAL, "unknown mem_kind");
  if (n < 3 || n >= (int64_t(1) << 31)) return fail(nullptr, PIRMCUT_EINVAL, "n must be in [3, 2^31)");
  if (!row_ptr) return fail(nullptr, PIRMCUT_EINVAL, "row_ptr must not be NULL");
  pirmcut_options o;
  pirmcut_default_options(&o);
  if (opt) o = *opt;
  std::string msg;
  if (check_options(o, &msg) != PIRMCUT_OK) return fail(nullptr, PIRMCUT_EINVAL, msg);

  // the GPU builds the problem when the input allows (rows in order, every
  // non-terminal with a terminal capacity); otherwise, and for every input
  // error, the host does
  pirmcut::DeviceGraph dg;
  pirmcut::HostGraph dhg;
  bool taken = false;
  if (!o.reduce_on_host) {
    // a failed device attempt (no device, no memory, an unusable storage
    // request) leaves the problem and its diagnosis to the host reduction
    pirmcut_status dps = pirmcut::reduce_graph_device(n, row_ptr, col, c, o.capacity_fp32, s, t,
                                                      o.format, mem_kind,
                                                      stream, nullptr, nullptr, &dhg, &dg, &taken, &msg);
    if (dps != PIRMCUT_OK) {
      taken = false;
      cudaGetLastError();
    }
  }
  if (taken) return create_from_device(n, o, stream, std::move(dhg), dg, out);

  // host reduction: the structure is kept (pirmcut_update_weights re-reduces
  // it); host capacities are read in place, device ones through a host copy
  pirmcut::hvec<int64_t> rp;
  pirmcut::hvec<int32_t> cl;
  pirmcut::hvec<double> cv;
  cudaError_t e = to_host(rp, row_ptr, size_t(n) + 1, mem_kind);
  if (e != cudaSuccess) return fail(nullptr, PIRMCUT_ECUDA, std::string("reading row_ptr: ") + cudaGetErrorString(e));
  const int64_t nnz = rp[n];
  if (nnz < 0 || rp[0] != 0) return fail(nullptr, PIRMCUT_EINVAL, "bad row_ptr");
  if (nnz > 0 && (!col || !c)) return fail(nullptr, PIRMCUT_EINVAL, "col and c must not be NULL");
  e = to_host(cl, col, size_t(nnz), mem_kind);
  const double* cin = static_cast<const double*>(c);
  if (e == cudaSuccess) e = host_capacities(cv, c, o.capacity_fp32, size_t(nnz), mem_kind, &cin);
  if (e != cudaSuccess) return fail(nullptr, PIRMCUT_ECUDA, std::string("reading the graph: ") + cudaGetErrorString(e));

  pirmcut_ctx* h = new (std::nothrow) pirmcut_ctx();
  if (!h) return fail(nullptr, PIRMCUT_ENOMEM, "out of host memory");
  Ctx& cx = h->c;
  pirmcut_status ps = pirmcut::reduce_graph(n, rp.data(), cl.data(), cin, s, t, o.format, &cx.hg, &msg);
  if (ps != PIRMCUT_OK) {
    delete h;
    return fail(nullptr, ps, msg);
  }
  cx.in_rp = std::move(rp);
  cx.in_col = std::move(cl);
  return finish_create(h, o, stream, nullptr, out);
}

pirmcut_status pirmcut_initial(pirmcut_ctx* h, pirmcut_step_info* info) {
  if (!h) return fail(nullptr, PIRMCUT_EINVAL, "ctx is NULL");
  pirmcut_step_info tmp;
  pirmcut_status st = run_steps(h, true, 0, 0, info ? info : &tmp);
  if (st == PIRMCUT_OK || st == PIRMCUT_ENOCONV) h->next_step = 1;
  return st;
}

pirmcut_status pirmcut_irls_step(pirmcut_ctx* h, double eps, pirmcut_step_info* info) {
  if (!h) return fail(nullptr, PIRMCUT_EINVAL, "ctx is NULL");
  Ctx& c = h->c;
  if (!c.x_set) return fail(h, PIRMCUT_EINVAL, "x is not set: call pirmcut_initial or pirmcut_set_x first");
  if (!(eps > 0.0) || !std::isfinite(eps)) return fail(h, PIRMCUT_EINVAL, "eps must be finite and > 0");
  *h->h_eps = eps;
  CK(h, cudaMemcpyAsync(c.eps_list, h->h_eps, sizeof(double), cudaMemcpyHostToDevice, c.stream), "eps");
  pirmcut_step_info tmp;
  pirmcut_status st = run_steps(h, false, 1, h->next_step, info ? info : &tmp);
  if (st == PIRMCUT_OK || st == PIRMCUT_ENOCONV) h->next_step += 1;
  return st;
}

pirmcut_status pirmcut_solve(pirmcut_ctx* h, int T, const double* eps, pirmcut_step_info* infos) {
  if (!h) return fail(nullptr, PIRMCUT_EINVAL, "ctx is NULL");
  Ctx& c = h->c;
  if (T < 0) return fail(h, PIRMCUT_EINVAL, "T must be >= 0");
  if (T > 0 && !eps) return fail(h, PIRMCUT_EINVAL, "eps must not be NULL");
  for (int l = 0; l < T; ++l)
    if (!(eps[l] > 0.0) || !std::isfinite(eps[l])) return fail(h, PIRMCUT_EINVAL, "every eps must be finite and > 0");
  pirmcut_status ps = ensure_capacity(h, T);
  if (ps != PIRMCUT_OK) return ps;
  if (T > 0) CK(h, cudaMemcpyAsync(c.eps_list, eps, sizeof(double) * T, cudaMemcpyHostToDevice, c.stream), "eps");
  std::vector<pirmcut_step_info> tmp;
  if (!infos) {
    tmp.resize(size_t(T) + 1);
    infos = tmp.data();
  }
  pirmcut_status st = run_steps(h, true, T, 0, infos);
  if (st == PIRMCUT_OK || st == PIRMCUT_ENOCONV) h->next_step = T + 1;
  return st;
}

pirmcut_status pirmcut_cut(pirmcut_ctx* h, uint8_t* side, double* value, double* tau, int mem_kind) {
  if (!h) return fail(nullptr, PIRMCUT_EINVAL, "ctx is NULL");
  Ctx& c = h->c;
  if (!c.x_set) return fail(h, PIRMCUT_EINVAL, "x is not set");
  if (mem_kind != PIRMCUT_MEM_HOST && mem_kind != PIRMCUT_MEM_DEVICE)
    return fail(h, PIRMCUT_EINVAL, "unknown mem_kind");
  pirmcut_status ps = ensure_graphs(h, true);
  if (ps != PIRMCUT_OK) return ps;
  CK(h, cudaGraphLaunch(c.g_cut, c.stream), "graph launch");
  c.launches += c.nodes_cut;
  if (side) {
    if (mem_kind == PIRMCUT_MEM_DEVICE) {
      CK(h, pirmcut::launch_side_full(c, side), "side");
    } else {
      if (!c.side_full) CK(h, dalloc(&c.side_full, size_t(c.hg.n)), "cudaMalloc");
      CK(h, pirmcut::launch_side_full(c, c.side_full), "side");
      CK(h, cudaMemcpyAsync(side, c.side_full, size_t(c.hg.n), cudaMemcpyDeviceToHost, c.stream), "side");
    }
  }
  CK(h, cudaMemcpyAsync(h->h_result, c.sw.result, 4 * sizeof(double), cudaMemcpyDeviceToHost, c.stream), "result");
  CK(h, cudaStreamSynchronize(c.stream), "cut");
  if (value) *value = h->h_result[1];
  if (tau) *tau = h->h_result[2];
  return PIRMCUT_OK;
}

pirmcut_status pirmcut_get_x(pirmcut_ctx* h, double* x, int mem_kind) {
  if (!h) return fail(nullptr, PIRMCUT_EINVAL, "ctx is NULL");
  Ctx& c = h->c;
  if (!c.x_set) return fail(h, PIRMCUT_EINVAL, "x is not set");
  if (!x) return fail(h, PIRMCUT_EINVAL, "x must not be NULL");
  if (mem_kind == PIRMCUT_MEM_DEVICE) {
    CK(h, pirmcut::launch_scatter_x(c, x), "get_x");
  } else if (mem_kind == PIRMCUT_MEM_HOST) {
    if (!c.xfull) CK(h, dalloc(&c.xfull, size_t(c.hg.n)), "cudaMalloc");
    CK(h, pirmcut::launch_scatter_x(c, c.xfull), "get_x");
    CK(h, cudaMemcpyAsync(x, c.xfull, sizeof(double) * c.hg.n, cudaMemcpyDeviceToHost, c.stream), "get_x");
  } else {
    return fail(h, PIRMCUT_EINVAL, "unknown mem_kind");
  }
  CK(h, cudaStreamSynchronize(c.stream), "get_x");
  return PIRMCUT_OK;
}

pirmcut_status pirmcut_set_x(pirmcut_ctx* h, const double* x, int mem_kind) {
  if (!h) return fail(nullptr, PIRMCUT_EINVAL, "ctx is NULL");
  Ctx& c = h->c;
  if (!x) return fail(h, PIRMCUT_EINVAL, "x must not be NULL");
  if (mem_kind == PIRMCUT_MEM_DEVICE) {
    CK(h, pirmcut::launch_gather_x(c, x), "set_x");
  } else if (mem_kind == PIRMCUT_MEM_HOST) {
    if (!c.xfull) CK(h, dalloc(&c.xfull, size_t(c.hg.n)), "cudaMalloc");
    CK(h, cudaMemcpyAsync(c.xfull, x, sizeof(double) * c.hg.n, cudaMemcpyHostToDevice, c.stream), "set_x");
    CK(h, pirmcut::launch_gather_x(c, c.xfull), "set_x");
  } else {
    return fail(h, PIRMCUT_EINVAL, "unknown mem_kind");
  }
  CK(h, cudaStreamSynchronize(c.stream), "set_x");
  c.x_set = true;
  return PIRMCUT_OK;
}

namespace {
// After new capacities: the sweep graph bakes c(s,t) and cut(0), and with
// options.step_stats the step graphs bake c(s,t) into the statistics kernel's
// arguments; drop the graphs that hold a stale value (they are rebuilt on
// the next use).
void drop_graphs_baking_cst(Ctx& c, double old_cst) {
  if (c.g_cut) {
    cudaGraphExecDestroy(c.g_cut);
    c.g_cut = nullptr;
  }
  if (c.opt.step_stats && !(c.hg.c_st == old_cst)) {
    if (c.g_init) {
      cudaGraphExecDestroy(c.g_init);
      c.g_init = nullptr;
    }
    if (c.g_step) {
      cudaGraphExecDestroy(c.g_step);
      c.g_step = nullptr;
    }
  }
}
}  // namespace

pirmcut_status pirmcut_update_weights(pirmcut_ctx* h, const void* cnew, int mem_kind) {
  if (!h) return fail(nullptr, PIRMCUT_EINVAL, "ctx is NULL");
  Ctx& c = h->c;
  if (mem_kind != PIRMCUT_MEM_HOST && mem_kind != PIRMCUT_MEM_DEVICE)
    return fail(h, PIRMCUT_EINVAL, "unknown mem_kind");
  if (c.device_reduced) {
    // the structure is on the device: rebuild there; an input the device
    // reduction does not take goes through the host for its message or result
    pirmcut::DeviceGraph dg;
    pirmcut::HostGraph ng;
    bool taken = false;
    std::string msg;
    pirmcut_status dps = pirmcut::reduce_graph_device(c.hg.n, nullptr, nullptr, cnew,
                                                      c.opt.capacity_fp32, c.hg.s, c.hg.t,
                                                      c.format, mem_kind, c.stream, c.d_in_rp,
                                                      c.d_in_col, &ng, &dg, &taken, &msg);
    if (dps != PIRMCUT_OK) return fail(h, dps, msg);
    if (taken) {
      bool same = ng.format == c.format && ng.nt == c.nt && ng.K == c.K && ng.nnz == c.hg.nnz;
      for (int k = 0; same && k < c.K; ++k) same = ng.off[k] == c.hg.off[k];
      if (!same) {
        dg.release();
        return fail(h, PIRMCUT_EINVAL, "the new capacities change the stored structure");
      }
      // copy into the context's arrays: captured graphs hold their addresses
      cudaError_t ce = cudaSuccess;
      if (c.format == PIRMCUT_FORMAT_DIA)
        ce = cudaMemcpyAsync(c.cdia, dg.cdia, sizeof(double) * size_t(c.K) * size_t(c.nt),
                             cudaMemcpyDeviceToDevice, c.stream);
      else
        ce = cudaMemcpyAsync(c.cval, dg.cval, sizeof(double) * size_t(c.hg.nnz),
                             cudaMemcpyDeviceToDevice, c.stream);
      if (ce == cudaSuccess)
        ce = cudaMemcpyAsync(c.cs, dg.cs, sizeof(double) * size_t(c.nt), cudaMemcpyDeviceToDevice, c.stream);
      if (ce == cudaSuccess)
        ce = cudaMemcpyAsync(c.ct, dg.ct, sizeof(double) * size_t(c.nt), cudaMemcpyDeviceToDevice, c.stream);
      if (ce == cudaSuccess) ce = cudaStreamSynchronize(c.stream);
      dg.release();
      if (ce != cudaSuccess) return cuda_fail(h, ce, "updating the capacities");
      const double old_cst = c.hg.c_st;
      c.hg = std::move(ng);
      drop_graphs_baking_cst(c, old_cst);
      return PIRMCUT_OK;
    }
    // host reduction of the device-resident structure
    CK(h, to_host(c.in_rp, static_cast<const int64_t*>(c.d_in_rp), size_t(c.hg.n) + 1, PIRMCUT_MEM_DEVICE), "reading the structure");
    CK(h, to_host(c.in_col, static_cast<const int32_t*>(c.d_in_col), size_t(c.in_rp.back()), PIRMCUT_MEM_DEVICE), "reading the structure");
  }
  const int64_t nnz = c.in_rp.back();
  if (nnz > 0 && !cnew) return fail(h, PIRMCUT_EINVAL, "c must not be NULL");
  pirmcut::hvec<double> cv;
  const double* cin = static_cast<const double*>(cnew);
  CK(h, host_capacities(cv, cnew, c.opt.capacity_fp32, size_t(nnz), mem_kind, &cin), "reading c");
  pirmcut::HostGraph ng;
  std::string msg;
  pirmcut_status ps = pirmcut::reduce_graph(c.hg.n, c.in_rp.data(), c.in_col.data(), cin,
                                            c.hg.s, c.hg.t, c.format, &ng, &msg);
  if (ps != PIRMCUT_OK) return fail(h, ps, msg);
  bool same = ng.format == c.format && ng.nt == c.nt && ng.K == c.K && ng.nnz == c.hg.nnz;
  for (int k = 0; same && k < c.K; ++k) same = ng.off[k] == c.hg.off[k];
  if (!same) return fail(h, PIRMCUT_EINVAL, "the new capacities change the stored structure");
  const double old_cst = c.hg.c_st;
  c.hg = std::move(ng);
  if (c.format == PIRMCUT_FORMAT_CSR) {
    CK(h, cudaMemcpyAsync(c.cval, c.hg.cval.data(), sizeof(double) * c.hg.cval.size(), cudaMemcpyHostToDevice, c.stream), "upload");
  } else {
    CK(h, cudaMemcpyAsync(c.cdia, c.hg.cdia.data(), sizeof(double) * c.hg.cdia.size(), cudaMemcpyHostToDevice, c.stream), "upload");
  }
  CK(h, cudaMemcpyAsync(c.cs, c.hg.cs.data(), sizeof(double) * c.nt, cudaMemcpyHostToDevice, c.stream), "upload");
  CK(h, cudaMemcpyAsync(c.ct, c.hg.ct.data(), sizeof(double) * c.nt, cudaMemcpyHostToDevice, c.stream), "upload");
  CK(h, cudaStreamSynchronize(c.stream), "upload");
  drop_graphs_baking_cst(c, old_cst);
  return PIRMCUT_OK;
}

pirmcut_status pirmcut_problem_size(const pirmcut_ctx* h, int64_t* n_nonterminal, int64_t* n_edges,
                                    int* format) {
  if (!h) return PIRMCUT_EINVAL;
  if (n_nonterminal) *n_nonterminal = h->c.nt;
  if (n_edges) *n_edges = h->c.hg.n_edges;
  if (format) *format = h->c.format;
  return PIRMCUT_OK;
}

int64_t pirmcut_kernel_launches(const pirmcut_ctx* h) { return h ? h->c.launches : 0; }

pirmcut_status pirmcut_time_spmv(pirmcut_ctx* h, int reps, double* avg_ms, double* bytes,
                                 double* flops) {
  if (!h) return fail(nullptr, PIRMCUT_EINVAL, "ctx is NULL");
  Ctx& c = h->c;
  if (!c.x_set || h->next_step == 0) return fail(h, PIRMCUT_EINVAL, "no step has run yet");
  if (reps < 1 || !avg_ms) return fail(h, PIRMCUT_EINVAL, "reps must be >= 1 and avg_ms non-NULL");
  const double nt = double(c.nt);
  const double nnz = c.format == PIRMCUT_FORMAT_DIA ? 2.0 * double(c.hg.n_edges)
                                                     : double(c.hg.nnz);
  const bool mx = c.opt.precision == PIRMCUT_PREC_MIXED;
  const double V = mx ? 4.0 : 8.0;
  // vectors read/written once per row: p and q (both systems are scaled to
  // unit diagonal; the fused FP32 kernel also reads r and d and writes the
  // new p and d)
  const double nvec = mx && c.fused_inner ? 6.0 : 2.0;
  if (bytes) {
    *bytes = c.format == PIRMCUT_FORMAT_DIA ? nt * (V * c.K + V * nvec)
                                            : nnz * (V + 4.0) + nt * (V * nvec + 8.0);
  }
  // one FMA per stored off-diagonal entry, the unit diagonal's add and the
  // (p, q) FMA per row
  if (flops) *flops = 2.0 * nnz + 3.0 * nt;
  // the solve left stop_req set: clear it so the kernel runs, restore after
  const size_t off_stop = offsetof(pirmcut::PcgState, stop_req);
  int one = 1, zero = 0;
  CK(h, cudaMemcpyAsync(reinterpret_cast<char*>(c.S) + off_stop, &zero, sizeof(int), cudaMemcpyHostToDevice, c.stream), "time");
  cudaEvent_t a = event_at(h, 0), b = event_at(h, 1);
  if (!a || !b) return fail(h, PIRMCUT_ECUDA, "cudaEventCreate failed");
  const bool m = c.opt.precision == PIRMCUT_PREC_MIXED;
  CK(h, m ? pirmcut::launch_spmv32_once(c) : pirmcut::launch_spmv_once(c), "spmv");  // warm-up
  // every timed launch starts from a cold L2: a 256 MB buffer (about twice
  // the L2) is written between launches, outside the timed interval
  const size_t flush_bytes = size_t(256) << 20;
  struct DeviceBuffer {
    void* p = nullptr;
    ~DeviceBuffer() {
      if (p) cudaFree(p);
    }
  } flush;
  CK(h, cudaMalloc(&flush.p, flush_bytes), "L2 flush buffer");
  double total = 0.0;
  for (int k = 0; k < reps; ++k) {
    CK(h, cudaMemsetAsync(flush.p, k & 0xff, flush_bytes, c.stream), "L2 flush");
    CK(h, cudaEventRecord(a, c.stream), "event");
    CK(h, m ? pirmcut::launch_spmv32_once(c) : pirmcut::launch_spmv_once(c), "spmv");
    CK(h, cudaEventRecord(b, c.stream), "event");
    CK(h, cudaEventSynchronize(b), "event");
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    total += ms;
  }
  CK(h, cudaMemcpyAsync(reinterpret_cast<char*>(c.S) + off_stop, &one, sizeof(int), cudaMemcpyHostToDevice, c.stream), "time");
  CK(h, cudaStreamSynchronize(c.stream), "time");
  *avg_ms = total / reps;
  return PIRMCUT_OK;
}

pirmcut_status pirmcut_mlp_enable(pirmcut_ctx* h, int mode, uint64_t seed) {
  if (!h) return fail(nullptr, PIRMCUT_EINVAL, "null context");
  Ctx& c = h->c;
  if (mode & ~(PIRMCUT_MLP_PREDICT | PIRMCUT_MLP_TRAIN))
    return fail(h, PIRMCUT_EINVAL, "mode must be 0 or an OR of PIRMCUT_MLP_PREDICT and PIRMCUT_MLP_TRAIN");
  if (mode && !c.mlp.master) {
    CK(h, pirmcut::mlp_alloc(c), "model buffers");
    CK(h, pirmcut::mlp_init(c, seed), "model initialisation");
  }
  if (mode != c.mlp_mode) {
    // the step graphs bake the hooks in: rebuild
    if (c.g_step) { cudaGraphExecDestroy(c.g_step); c.g_step = nullptr; }
    c.mlp_mode = mode;
  }
  return PIRMCUT_OK;
}

pirmcut_status pirmcut_mlp_configure(pirmcut_ctx* h, int iters_per_step, float learning_rate) {
  if (!h) return fail(nullptr, PIRMCUT_EINVAL, "null context");
  Ctx& c = h->c;
  if (iters_per_step < 0 || iters_per_step > 1024)
    return fail(h, PIRMCUT_EINVAL, "iters_per_step must be in [0, 1024]");
  if (!(learning_rate > 0.0f) || !std::isfinite(learning_rate))
    return fail(h, PIRMCUT_EINVAL, "learning_rate must be positive and finite");
  if (iters_per_step != c.mlp.iters_per_step || learning_rate != c.mlp.lr) {
    if (c.g_step) { cudaGraphExecDestroy(c.g_step); c.g_step = nullptr; }
  }
  c.mlp.iters_per_step = iters_per_step;
  c.mlp.lr = learning_rate;
  return PIRMCUT_OK;
}

namespace {
// ETIMEOUT when a bounded wait of the tensor-core network expired (the
// outputs past that point are not written).
pirmcut_status tensor_status(pirmcut_ctx* h) {
  pirmcut::MlpState m;
  cudaError_t e = pirmcut::mlp_get_state(h->c, &m);
  if (e != cudaSuccess) return cuda_fail(h, e, "reading the model state");
  if (m.tc_error) return fail(h, PIRMCUT_ETIMEOUT, "a tensor-core wait of the network expired");
  return PIRMCUT_OK;
}
}  // namespace

pirmcut_status pirmcut_mlp_predict(pirmcut_ctx* h, const float* features, int64_t count,
                                   float* delta, int mem_kind) {
  if (!h) return fail(nullptr, PIRMCUT_EINVAL, "null context");
  Ctx& c = h->c;
  if (!c.mlp.master) return fail(h, PIRMCUT_EINVAL, "no model: call pirmcut_mlp_enable first");
  if (count < 0) return fail(h, PIRMCUT_EINVAL, "count must be >= 0");
  if (count == 0) return PIRMCUT_OK;
  if (!features || !delta) return fail(h, PIRMCUT_EINVAL, "null feature or output buffer");
  if (mem_kind != PIRMCUT_MEM_HOST && mem_kind != PIRMCUT_MEM_DEVICE)
    return fail(h, PIRMCUT_EINVAL, "mem_kind must be PIRMCUT_MEM_HOST or PIRMCUT_MEM_DEVICE");
  const size_t fb = sizeof(float) * pirmcut::kMlpFeatures * size_t(count);
  const size_t db = sizeof(float) * size_t(count);
  if (mem_kind == PIRMCUT_MEM_DEVICE) {
    CK(h, pirmcut::mlp_predict_delta(c, features, count, delta), "inference");
    CK(h, cudaStreamSynchronize(c.stream), "inference");
    return tensor_status(h);
  }
  float* df = nullptr;
  float* dd = nullptr;
  cudaError_t e = cudaMalloc((void**)&df, fb);
  if (e == cudaSuccess) e = cudaMalloc((void**)&dd, db);
  if (e == cudaSuccess) e = cudaMemcpyAsync(df, features, fb, cudaMemcpyHostToDevice, c.stream);
  if (e == cudaSuccess) e = pirmcut::mlp_predict_delta(c, df, count, dd);
  if (e == cudaSuccess) e = cudaMemcpyAsync(delta, dd, db, cudaMemcpyDeviceToHost, c.stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
  if (df) cudaFree(df);
  if (dd) cudaFree(dd);
  if (e != cudaSuccess) return cuda_fail(h, e, "inference");
  return tensor_status(h);
}

pirmcut_status pirmcut_mlp_time_predict(pirmcut_ctx* h, const float* features, int64_t count,
                                        float* delta, int reps, double* avg_ms) {
  if (!h) return fail(nullptr, PIRMCUT_EINVAL, "null context");
  Ctx& c = h->c;
  if (!c.mlp.master) return fail(h, PIRMCUT_EINVAL, "no model: call pirmcut_mlp_enable first");
  if (count < 1 || reps < 1 || !features || !delta || !avg_ms)
    return fail(h, PIRMCUT_EINVAL, "count and reps must be >= 1 and every pointer non-NULL");
  CK(h, pirmcut::mlp_time_predict(c, features, count, delta, reps, avg_ms), "timed inference");
  return tensor_status(h);
}

pirmcut_status pirmcut_mlp_weights(pirmcut_ctx* h, float* w, int direction) {
  if (!h) return fail(nullptr, PIRMCUT_EINVAL, "null context");
  Ctx& c = h->c;
  if (!c.mlp.master) return fail(h, PIRMCUT_EINVAL, "no model: call pirmcut_mlp_enable first");
  if (!w) return fail(h, PIRMCUT_EINVAL, "null weight buffer");
  if (direction == 0) {
    CK(h, pirmcut::mlp_get_weights(c, w), "reading the weights");
  } else if (direction == 1) {
    CK(h, pirmcut::mlp_set_weights(c, w), "loading the weights");
  } else {
    return fail(h, PIRMCUT_EINVAL, "direction must be 0 (read) or 1 (load)");
  }
  return PIRMCUT_OK;
}

pirmcut_status pirmcut_mlp_stats(pirmcut_ctx* h, pirmcut_mlp_info* info) {
  if (!h) return fail(nullptr, PIRMCUT_EINVAL, "null context");
  Ctx& c = h->c;
  if (!info) return fail(h, PIRMCUT_EINVAL, "null info");
  if (!c.mlp.master) return fail(h, PIRMCUT_EINVAL, "no model: call pirmcut_mlp_enable first");
  pirmcut::MlpState m;
  CK(h, pirmcut::mlp_get_state(c, &m), "reading the model state");
  info->steps = m.steps;
  info->used = m.used;
  info->train_steps = m.train_steps;
  info->loss = m.loss;
  info->alpha = m.alpha;
  info->energy_change = m.energy_change;
  info->res_plain = std::sqrt(m.res_plain);
  info->mean_alpha = m.steps ? m.sum_alpha / m.steps : 0.0;
  info->tensor_timeouts = m.tc_error;
  return PIRMCUT_OK;
}

pirmcut_status pirmcut_mlp_features(pirmcut_ctx* h, float* f) {
  if (!h) return fail(nullptr, PIRMCUT_EINVAL, "null context");
  Ctx& c = h->c;
  if (!f) return fail(h, PIRMCUT_EINVAL, "null feature buffer");
  if (!c.mlp.master) return fail(h, PIRMCUT_EINVAL, "no model: call pirmcut_mlp_enable first");
  CK(h, pirmcut::mlp_get_features(c, f), "reading the features");
  return PIRMCUT_OK;
}

pirmcut_status pirmcut_spmv_timing(pirmcut_ctx* h, double* total_ms, int64_t* launches, int reset) {
  if (!h) return fail(nullptr, PIRMCUT_EINVAL, "null context");
  if (total_ms) *total_ms = h->c.spmv_ms;
  if (launches) *launches = h->c.spmv_count;
  if (reset) {
    h->c.spmv_ms = 0.0;
    h->c.spmv_count = 0;
  }
  return PIRMCUT_OK;
}

const char* pirmcut_last_error(const pirmcut_ctx* h) {
  return h ? h->c.err.c_str() : g_create_error.c_str();
}

void pirmcut_destroy(pirmcut_ctx* h) {
  if (!h) return;
  if (h->c.stream) cudaStreamSynchronize(h->c.stream);
  free_device(h->c);
  for (cudaEvent_t e : h->events) cudaEventDestroy(e);
  if (h->h_ctr) cudaFreeHost(h->h_ctr);
  delete h;
}

}  // extern "C"
