// The solver context behind the opaque pirmcut_ctx handle.
#pragma once

#include <climits>
#include <cstdint>
#include <string>
#include <vector>

#include <cuda_bf16.h>
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
  int refine;   // FP64 refinement cycles (mixed precision), 0 otherwise
  double obj;   // S_eps(x^(l)) and x^T L(g^(l)) x with options.step_stats, else NaN
  double flow;
};

// State of the FP64 iterative-refinement loop around the FP32 inner PCG.
struct OuterState {
  double rr64;      // ||b - L~ x||^2 in FP64 at the last loop head
  double bb;        // ||b||^2
  double tol2;      // pcg_tol^2
  double eta2;      // inner_tol^2
  int outer_iters;  // refinement cycles run in this solve
  int max_outer;
  int total_inner;  // FP32 PCG iterations summed over cycles
  int outer_stop;
  int status;
  int inner_maxit;
  unsigned int counter[2];
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
// Most CSR rows that get a block of their own in the per-row kernels.
constexpr int kHeavyRowsMax = 1024;

// Learned warm start (per-node MLP, 6 -> 64 -> 64 -> 1).
constexpr int kMlpFeatures = 6;
constexpr int kMlpParams = 64 * kMlpFeatures + 64 + 64 * 64 + 64 + 64 + 1;

struct MlpState {
  double alpha;          // step length along the learned direction, last step
  double energy_change;  // E(x^(l-1) + alpha d) - E(x^(l-1)) <= 0, last step
  double res_plain;      // ||b - L~ x^(l-1)||^2, last step
  double sum_alpha;      // sum of alpha over steps
  float loss;            // mean squared error of the last minibatch
  int sel;               // 1 when the last step started from the candidate
  int steps;             // steps that evaluated a candidate
  int used;              // steps that started from it
  int train_steps;       // Adam steps taken
  unsigned int counter;  // last-block counter of the residual reductions
  unsigned int adam_ticket;  // last-block counter of the Adam step
  int tc_error;          // 1 once a tensor-core wait of the network expired
};

struct MlpBuf {
  float* master = nullptr;       // FP32 weights (kMlpParams)
  __nv_bfloat16* w16 = nullptr;  // BF16 copy read by the inference/gradient kernels
  float* m = nullptr;            // Adam moments
  float* v = nullptr;
  float* grad_part = nullptr;    // per-block gradient sums
  float* loss_part = nullptr;
  float* feat = nullptr;         // nt x kMlpFeatures
  double* dir = nullptr;         // learned direction d (FP64)
  double* xprev = nullptr;       // x^(l-1): reweighting point and training baseline
  double* gprev = nullptr;       // g^(l-1)
  MlpState* state = nullptr;
  uint64_t seed = 0;
  int iters_per_step = 8;        // Adam steps after each IRLS step
  float lr = 1e-3f;              // Adam learning rate
};

struct Ctx {
  // problem
  HostGraph hg;               // reduced problem (host copy kept for update_weights)
  hvec<int64_t> in_rp;        // original CSR structure (for update_weights), host reduction
  hvec<int32_t> in_col;
  int64_t* d_in_rp = nullptr; // the same on the device, device reduction
  int32_t* d_in_col = nullptr;
  bool device_reduced = false;  // the problem was built on the GPU (hg holds scalars only)
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
  double* partials = nullptr;   // 4 * (kMaxBlocks + kHeavyRowsMax)
  // CSR rows far longer than the mean (more than max(512, 16 x mean) entries,
  // at most kHeavyRowsMax of them, ascending): the per-row PCG and sweep
  // kernels give each a block of its own, appended to their grids
  int32_t* heavy = nullptr;
  int n_heavy = 0;
  int64_t heavy_deg = INT64_MAX;  // rows with more entries than this are heavy
  // FP64 path: CG on the Jacobi-scaled system D^-1/2 L~ D^-1/2 (unit
  // diagonal), allocated for precision FP64 only
  double* rsd = nullptr;        // d_v^-1/2
  float* sq32 = nullptr;        // d_v^1/2 in FP32 (norm of the stopping test)
  double* xs = nullptr;         // scaled iterate D^1/2 x
  double* ghat = nullptr;       // scaled conductances g_uv d_u^-1/2 d_v^-1/2 (DIA K*nt or CSR nnz)
  double* xstats = nullptr;     // x at the start of a step (options.step_stats)
  PcgState* S = nullptr;
  // mixed precision: FP32 CG on the Jacobi-scaled system D^-1/2 L~ D^-1/2
  // (unit diagonal) inside FP64 iterative refinement
  float* g32 = nullptr;         // scaled conductances g_uv / sqrt(d_u d_v) (DIA K*nt or CSR nnz)
  double* s64 = nullptr;        // d_v^-1/2
  float* s32 = nullptr;
  float* r32 = nullptr;         // scaled inner residual
  float* p32 = nullptr;
  float* p32b = nullptr;        // second direction buffer of the fused recurrence
  float* q32 = nullptr;
  float* d32 = nullptr;         // scaled correction
  double* b64 = nullptr;        // right-hand side (FP64)
  OuterState* O = nullptr;
  bool fused_inner = false;     // two-kernel inner CG iteration (vectorised DIA)
  int fused_grid = 1;
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
  MlpBuf mlp;
  int mlp_mode = 0;             // PIRMCUT_MLP_* bits

  bool x_set = false;
  int64_t launches = 0;

  // live SpMV timing in stream-launch mode (options.time_spmv)
  std::vector<cudaEvent_t> spmv_ev;  // 2 per SpMV launch of a chunk
  double spmv_ms = 0.0;
  int64_t spmv_count = 0;
};

// Events for timing `pairs` SpMV launches (created on first use); nullptr on failure.
cudaEvent_t* spmv_events(Ctx& c, int pairs);
// Add the first `executed` of `pairs` bracketed launches to the totals.
void spmv_events_collect(Ctx& c, int pairs, int executed);

// pcg.cu
inline int row_grid(const Ctx& c) {
  const int64_t threads = c.format == PIRMCUT_FORMAT_DIA ? c.nt : c.nt * c.group;
  return grid_for(threads);
}
int enqueue_reweight(Ctx& c, cudaStream_t st, bool initial);
// offsets of the PCG counters the stream-launch loops read back
struct PcgProgress {
  int iters, maxit, stop_req;
};
int enqueue_step_end(Ctx& c, cudaStream_t st, bool initial, const OuterState* O);
// options.step_stats: keep x^(l-1) at the start of a step (a copy, no kernel)
cudaError_t enqueue_stats_pre(Ctx& c, cudaStream_t st);
cudaError_t build_step_graph(Ctx& c, bool initial, cudaGraphExec_t* out, int* nodes);
cudaError_t run_step_stream(Ctx& c, bool initial, int* stop_flag_host, int64_t* kernels);
cudaError_t launch_scatter_x(Ctx& c, double* xfull);           // reduced x -> full n
cudaError_t launch_gather_x(Ctx& c, const double* xfull);      // full n -> reduced x
cudaError_t launch_spmv_once(Ctx& c);                          // one standalone SpMV launch
// mixed.cu
cudaError_t mixed_alloc(Ctx& c);
void mixed_free(Ctx& c);
cudaError_t build_step_graph_mixed(Ctx& c, bool initial, cudaGraphExec_t* out, int* nodes);
cudaError_t run_step_stream_mixed(Ctx& c, bool initial, int* flag_host, int64_t* kernels);
cudaError_t launch_spmv32_once(Ctx& c);
// mlp.cu
bool mlp_active(const Ctx& c, bool initial);          // the step runs the MLP hooks
cudaError_t mlp_alloc(Ctx& c);
void mlp_free(Ctx& c);
cudaError_t mlp_init(Ctx& c, uint64_t seed);
cudaError_t mlp_get_weights(Ctx& c, float* host);
cudaError_t mlp_set_weights(Ctx& c, const float* host);
cudaError_t mlp_get_state(Ctx& c, MlpState* host);
cudaError_t mlp_get_features(Ctx& c, float* host);
cudaError_t mlp_predict_delta(Ctx& c, const float* feat, int64_t count, float* delta);
cudaError_t mlp_time_predict(Ctx& c, const float* feat, int64_t count, float* delta, int reps,
                             double* avg_ms);
int enqueue_mlp_pre(Ctx& c, cudaStream_t st);    // before the reweighting
int enqueue_mlp_post(Ctx& c, cudaStream_t st);   // after it: features and the learned direction
int enqueue_mlp_start_mixed(Ctx& c, cudaStream_t st);  // mixed path, after its assembly
int enqueue_mlp_train(Ctx& c, cudaStream_t st);  // after the solve
// sweep.cu
cudaError_t sweep_alloc(Ctx& c);
cudaError_t enqueue_sweep(Ctx& c, cudaStream_t st, bool record, int* nodes);
cudaError_t enqueue_cut_value(Ctx& c, cudaStream_t st, const uint8_t* side_red);
cudaError_t build_cut_graph(Ctx& c, cudaGraphExec_t* out, int* nodes);
cudaError_t launch_side_full(Ctx& c, uint8_t* side_full);
// The heavy rows of a CSR problem from its host row pointers (global entry
// offsets for a batch instance's view).
cudaError_t set_heavy_rows(Ctx& c, const int64_t* host_rp);
void sweep_free(Ctx& c);

}  // namespace pirmcut

// The opaque handle of include/pirmcut.h.
struct pirmcut_ctx {
  pirmcut::Ctx c;
  // pinned host staging for small transfers
  pirmcut::StepCounters* h_ctr = nullptr;
  double* h_eps = nullptr;
  double* h_result = nullptr;  // 4
  int* h_stop = nullptr;       // PCG stop flag read back in stream-launch mode
  std::vector<cudaEvent_t> events;
  int next_step = 0;           // IRLS index of the next step record
};
