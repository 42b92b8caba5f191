// The solver context behind the opaque pirmcut_ctx handle.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "device.cuh"
#include "internal.h"

namespace pirmcut {

// Per-step record written on the device by the last kernel of a step.
struct StepRec {
  int step;
  int iters;
  double eps;
  double rr, bb;
  double xmin, xmax;
  double cut;
  int status;
  int pad;
};

// Counters that sequence the steps of one solve on the device.
struct StepCounters {
  int eps_idx;  // next entry of eps_list a reweighting step consumes
  int rec_idx;  // next StepRec slot
  int step;     // IRLS index l of the next record
  int pad;
};

// Scratch of the sweep cut (allocated on first use).
struct SweepBuf {
  int64_t cap = 0;            // n~ the buffers were sized for
  uint64_t* keys[2] = {nullptr, nullptr};
  uint32_t* vals[2] = {nullptr, nullptr};
  uint32_t* hist = nullptr;   // 256 * nblocks (scanned in place)
  uint32_t* digit_tot = nullptr;  // 256
  int32_t* rank = nullptr;
  double* delta = nullptr;    // per vertex, then gathered in sweep order
  double* blk = nullptr;      // per-tile partial sums / argmin partials
  int64_t* blk_k = nullptr;
  uint8_t* side_red = nullptr;
  double* result = nullptr;   // [value_prefix, value_exact, tau, k]
  int nblocks_sort = 0;
  int ntiles = 0;
};

struct Ctx {
  // problem
  HostGraph hg;               // reduced problem (host copy kept for update_weights)
  std::vector<int64_t> in_rp; // original CSR structure (for update_weights)
  std::vector<int32_t> in_col;
  int64_t nt = 0;
  int format = PIRMCUT_FORMAT_CSR;
  int K = 0;
  DiaDesc dd{};
  int group = 1;
  pirmcut_options opt{};
  std::string err;
  int device = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t cap_stream = nullptr;  // private stream used only for graph capture

  // device problem data
  double* cdia = nullptr;  // K * nt (DIA)
  double* gdia = nullptr;
  int64_t* rp = nullptr;   // CSR
  int32_t* col = nullptr;
  double* cval = nullptr;
  double* gval = nullptr;
  double* cs = nullptr;
  double* ct = nullptr;

  // PCG vectors (FP64)
  double* x = nullptr;
  double* r = nullptr;
  double* p = nullptr;
  double* q = nullptr;
  double* diag = nullptr;
  double* dinv = nullptr;
  double* partials = nullptr;   // 4 * kMaxBlocks
  PcgState* S = nullptr;
  StepCounters* C = nullptr;
  double* eps_list = nullptr;   // capacity eps_cap
  int eps_cap = 0;
  StepRec* recs = nullptr;      // capacity rec_cap
  int rec_cap = 0;
  double* xfull = nullptr;      // n, staging for get/set_x with device buffers
  uint8_t* side_full = nullptr; // n

  // host staging (pinned)
  StepRec* h_recs = nullptr;
  int h_rec_cap = 0;

  // graphs
  cudaGraphExec_t g_init = nullptr;
  cudaGraphExec_t g_step = nullptr;
  cudaGraphExec_t g_cut = nullptr;
  int nodes_init = 0, nodes_step = 0, nodes_cut = 0;

  SweepBuf sw;

  bool x_set = false;
  int64_t launches = 0;
};

// pcg.cu
cudaError_t build_step_graph(Ctx& c, bool initial, cudaGraphExec_t* out, int* nodes);
cudaError_t run_step_stream(Ctx& c, bool initial, int* stop_flag_host, int64_t* kernels);
cudaError_t launch_scatter_x(Ctx& c, double* xfull);           // reduced x -> full n
cudaError_t launch_gather_x(Ctx& c, const double* xfull);      // full n -> reduced x
cudaError_t launch_spmv_once(Ctx& c);                          // one standalone SpMV launch
// sweep.cu
cudaError_t sweep_alloc(Ctx& c);
cudaError_t build_cut_graph(Ctx& c, cudaGraphExec_t* out, int* nodes);
cudaError_t launch_side_full(Ctx& c, uint8_t* side_full);
void sweep_free(Ctx& c);

}  // namespace pirmcut
