/*
 * pirmcut.h -- C ABI of libpirmcut, a GB300 (sm_103a) implementation of the
 * IRLS hot path of PIRMCut (Zhu & Gleich, "A Parallel Min-Cut Algorithm using
 * Iteratively Reweighted Least Squares", arXiv:1501.03105).
 *
 * Problem (Section 2): an undirected graph G = (V, E) with capacities
 * c(e) >= 0 and two terminals s != t; find S with s in S, t not in S that
 * minimises cut(S, S-bar) = sum of c over edges with exactly one end in S.
 *
 * Method (Section 2.1, Algorithm 1): x^(0) solves the weighted least squares
 * problem (Eq. constrained-wls) with W^(0) = C; then for l = 1..T each edge
 * is reweighted from x^(l-1) (Eq. define-reweight-vector) and the reduced
 * Laplacian system  L~ v = b  (Eq. reduced-laplacian-system: x_s = 1 and
 * x_t = 0 held as Dirichlet values) is solved by Jacobi-preconditioned
 * conjugate gradients (Section 3.1), warm-started from v^(l-1).  Finally a
 * sweep cut over x (Section 3.3) rounds x to a cut.
 *
 * Conventions for every entry point:
 *  - Vertices are 0..n-1 in the caller's numbering; s and t are ordinary
 *    vertex ids.  Vectors of length n (x, side) use that numbering.
 *  - mem_kind is PIRMCUT_MEM_HOST for host pointers (pageable or pinned) and
 *    PIRMCUT_MEM_DEVICE for device pointers on the context's device.
 *  - All GPU work of a context is ordered on the CUDA stream given at
 *    creation (NULL = the legacy default stream).  Entry points that return
 *    host scalars or fill host buffers synchronise that stream before they
 *    return.
 *  - The library copies every input; the caller keeps ownership of all
 *    buffers it passes and of the outputs it receives.
 *  - Errors are returned as pirmcut_status codes; nothing aborts.  The text
 *    of the last error of a context is available from pirmcut_last_error().
 *  - A context is not thread-safe: serialise calls on one context.
 */
#ifndef PIRMCUT_H
#define PIRMCUT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pirmcut_ctx pirmcut_ctx; /* opaque, owned by the library */

typedef enum {
  PIRMCUT_OK = 0,
  PIRMCUT_EINVAL = 1,        /* invalid argument or malformed graph */
  PIRMCUT_EDISCONNECTED = 2, /* a non-terminal component reaches neither s nor t
                                through positive capacity: L~ would be singular
                                (Prop. nonsingular) */
  PIRMCUT_ENOMEM = 3,        /* host or device allocation failed */
  PIRMCUT_ECUDA = 4,         /* a CUDA runtime call failed */
  PIRMCUT_ENOCONV = 5,       /* PCG hit pcg_max_iter; the iterate is kept and usable */
  PIRMCUT_ETIMEOUT = 6,      /* a bounded device-side wait gave up */
  PIRMCUT_ENUMERIC = 7       /* NaN/Inf or a non-positive curvature p^T L~ p met */
} pirmcut_status;

enum { PIRMCUT_MEM_HOST = 0, PIRMCUT_MEM_DEVICE = 1 };

/* Reweighting form.  WEIGHTED_L1: g_e = c_e / sqrt(d_e^2 + eps^2), d = x_u - x_v.
 * PAPER: the literal Eq. (define-reweight-vector) + Eq. (reweighted-laplacian),
 * w_e = sqrt((c_e d_e)^2 + eps^2) and g_e = c_e^2 / w_e. */
enum { PIRMCUT_REWEIGHT_WEIGHTED_L1 = 0, PIRMCUT_REWEIGHT_PAPER = 1 };

/* Arithmetic of the PCG.  FP64: every vector, matrix value and reduction in
 * FP64.  MIXED: FP32 matrix values and vectors in the inner PCG with
 * compensated (twice-working-precision) inner products, and FP64 outer
 * residuals with iterative refinement of an FP64 iterate. */
enum { PIRMCUT_PREC_FP64 = 0, PIRMCUT_PREC_MIXED = 1 };

/* Storage of L~.  DIA: symmetric diagonal storage, used when the non-terminal
 * graph in the given numbering has few distinct index offsets (grids).  CSR:
 * general rows.  AUTO picks DIA when it applies. */
enum { PIRMCUT_FORMAT_AUTO = 0, PIRMCUT_FORMAT_DIA = 1, PIRMCUT_FORMAT_CSR = 2 };

typedef struct {
  int reweight_form;   /* PIRMCUT_REWEIGHT_*                                   */
  int precision;       /* PIRMCUT_PREC_*                                       */
  double pcg_tol;      /* stop when ||b - L~ v||_2 <= pcg_tol * ||b||_2        */
  int pcg_max_iter;    /* PCG iteration cap per linear system                  */
  int warm_start;      /* 1: start PCG of step l from v^(l-1); 0: from zero    */
  int format;          /* PIRMCUT_FORMAT_*                                     */
  int track_cut;       /* 1: run a sweep cut after every IRLS step and record
                          its value in pirmcut_step_info.cut_value             */
  int graph_launch;    /* 1: each step is one CUDA graph whose PCG loop is a
                          device-side WHILE node (no host sync inside a solve);
                          0: the same kernels launched one by one from the host,
                          PCG iterations in chunks of 8 with the stop flag (for
                          batches: the number of active instances) read back
                          between chunks (for profilers that cannot see into
                          conditional graph nodes); the results are identical */
  double inner_tol;    /* MIXED only: each FP32 inner solve reduces its residual
                          by this factor (or just enough for the FP64 test)   */
  int time_spmv;       /* 1 (with graph_launch 0): bracket every PCG
                          matrix-vector launch with CUDA events on the
                          context's stream; pirmcut_spmv_timing reports them  */
  int reduce_on_host;  /* 0: validate and pack the input on the GPU when every
                          row lists strictly increasing columns and every
                          non-terminal has a terminal capacity (else, and for
                          every input error, on the host); 1: always on the
                          host.  Both give the same problem.                  */
  int batch_threads_per_row; /* batches: threads per short row (1, 2, 4, 8, 16
                          or 32), rows per consecutive-row tile (64 to 65536),
                          and the warp-row threshold (1 to 512; 512 turns the
                          warp tier off); 0 = chosen by the autotuner          */
  int batch_tile_rows;
  int batch_medium_deg;
  int step_stats;      /* 1: every step also records its objective and flow
                          value in pirmcut_step_info (one more pass over the
                          edges per step); batches leave them NaN             */
  int capacity_fp32;   /* 0: the capacities c passed to pirmcut_create and
                          pirmcut_update_weights are double[nnz]; 1: they are
                          float[nnz] (half the bytes to copy in), widened
                          exactly to FP64 by the library: the problem is the
                          same as for the doubles of equal value.  Batches
                          take doubles.                                      */
  int fuse_reweight;   /* 1: FP64 steps on DIA storage form the conductances
                          (Eq. define-reweight-vector) inside the assembly
                          pass instead of a pass of their own, each edge's
                          twice (once per endpoint row): the same values and
                          results bit for bit, more FP64 work, one pass fewer.
                          Ignored on CSR, in mixed precision and while the
                          learned start predicts (it reads the conductances
                          first).  0 (default): separate passes.             */
} pirmcut_options;

typedef struct {
  int step;            /* l (0 for x^(0))                                      */
  int pcg_iters;       /* PCG iterations spent on this step's system           */
  double eps;          /* smoothing parameter used (0 for step 0)             */
  double rel_residual; /* final ||r||_2 / ||b||_2 of the PCG recurrence        */
  double x_min, x_max; /* range of x over the non-terminals                   */
  double cut_value;    /* sweep-cut value after the step if track_cut, else NaN */
  double ms;           /* GPU time of the step in milliseconds                */
  int status;          /* pirmcut_status of the step                          */
  int refinements;     /* MIXED: FP64 refinement cycles (FP64 residuals that
                          started an inner solve); 0 for FP64                 */
  double objective;    /* with options.step_stats: the smoothed objective
                          S_eps(x^(l)) of the reweighting form (Eq.
                          l1-min-smooth-version; eps = 0 for step 0), over the
                          edges of positive capacity; else NaN               */
  double flow_value;   /* with options.step_stats: x^T L(g^(l)) x, the value of
                          the electrical flow of the step's system (Prop.
                          wls-equal-electrical-flow); else NaN               */
} pirmcut_step_info;

/* Fill *opt with the defaults: WEIGHTED_L1, FP64, pcg_tol 1e-10,
 * pcg_max_iter 20000, warm_start 1, FORMAT_AUTO, track_cut 0, graph_launch 1,
 * inner_tol 1e-5, time_spmv 0, reduce_on_host 0, batch_* 0, step_stats 0,
 * capacity_fp32 0.  With MIXED,
 * pcg_iters counts FP32 inner iterations, at most
 * min(pcg_max_iter, 2000) per refinement cycle and 64 cycles per system. */
void pirmcut_default_options(pirmcut_options* opt);

/*
 * Build a solver context for one s-t min-cut instance (Section 2; the
 * non-terminal graph and terminal edges of Algorithm 1, step 1).
 *
 * n        number of vertices (>= 3 and < 2^31), terminals included.
 * row_ptr  int64[n+1], CSR row offsets, row_ptr[0] = 0, non-decreasing.
 * col      int32[row_ptr[n]], neighbour ids in [0, n).
 * c        double[row_ptr[n]] (float[row_ptr[n]] with opt->capacity_fp32),
 *          capacities, finite and >= 0.
 *          The CSR must be symmetric: each undirected edge {u, v} appears in
 *          row u and in row v with the same total capacity.  Parallel entries
 *          of one pair are summed; self-loops are rejected.
 * s, t     source and sink, s != t.
 * opt      options (NULL = defaults).
 * mem_kind where row_ptr/col/c live.  Device input is first copied to the
 *          host: the reduction and packing of the graph run on the host once.
 * stream   cudaStream_t (as void*) on which all work of the context runs.
 * out      receives the context on success, NULL on failure.
 *
 * The terminal edges are folded into two per-vertex capacity vectors
 * (c(s,v), c(v,t)) plus the constant c(s,t); the non-terminal graph's
 * structure is packed once and reused by every step (Section 3.1: the nonzero
 * structure of L~ never changes).  The context starts with x^(0) unset.
 * Errors: EINVAL (malformed input), EDISCONNECTED, ENOMEM, ECUDA.
 */
pirmcut_status pirmcut_create(int64_t n, const int64_t* row_ptr, const int32_t* col,
                              const void* c, int32_t s, int32_t t,
                              const pirmcut_options* opt, int mem_kind, void* stream,
                              pirmcut_ctx** out);

/*
 * Compute x^(0): the WLS solution with W^(0) = C (Section 2.1, Algorithm 1
 * step 2), i.e. conductances g = c, solved by Jacobi-PCG from zero.
 * info may be NULL.  Returns OK, ENOCONV (cap reached, iterate kept),
 * ENUMERIC or ECUDA.
 */
pirmcut_status pirmcut_initial(pirmcut_ctx* ctx, pirmcut_step_info* info);

/*
 * One IRLS iteration (Section 2.1, Steps 1-2; Algorithm 1 step 4): reweight
 * every edge from the current x with smoothing parameter eps > 0, assemble
 * L~ and b (x_s = 1, x_t = 0 as Dirichlet values) together with the Jacobi
 * diagonal, and solve L~ v = b by PCG warm-started from the current x
 * (Section 3.1).  The current x (from pirmcut_initial, a previous step or
 * pirmcut_set_x) is replaced by the new iterate.  info may be NULL.
 * Errors: EINVAL (eps <= 0 or x unset), ENOCONV, ENUMERIC, ECUDA.
 */
pirmcut_status pirmcut_irls_step(pirmcut_ctx* ctx, double eps, pirmcut_step_info* info);

/*
 * Algorithm 1 steps 2-4 on one GPU: x^(0), then T IRLS steps with
 * eps[0..T-1].  infos (may be NULL) receives T+1 records (x^(0) first).
 * Returns the worst status met (ENOCONV if any system hit the cap).
 */
pirmcut_status pirmcut_solve(pirmcut_ctx* ctx, int T, const double* eps,
                             pirmcut_step_info* infos);

/*
 * Sweep cut over the current x (Section 3.3; Algorithm 1 step 6).
 * Non-terminals are ordered by x descending (vertex id ascending on ties);
 * the prefixes that end between two strictly different x values, together
 * with the empty and the full prefix, are the candidate source sides (s
 * always in, t always out); the candidate of least cut value wins (the
 * shorter prefix on exact ties of the evaluated values).
 *
 * side   uint8[n] (may be NULL): 1 for the source side, 0 for the sink side.
 * value  (may be NULL) the exact FP64 cut value of the returned side.
 * tau    (may be NULL) the threshold (x_(k) + x_(k+1))/2 between the last
 *        vertex taken and the first one left (x_(0) = 1, x_(n~+1) = 0).
 * Errors: EINVAL (x unset), ECUDA.
 */
pirmcut_status pirmcut_cut(pirmcut_ctx* ctx, uint8_t* side, double* value, double* tau,
                           int mem_kind);

/* Copy the current x (double[n], x_s = 1, x_t = 0) out.  EINVAL if x unset. */
pirmcut_status pirmcut_get_x(pirmcut_ctx* ctx, double* x, int mem_kind);

/* Set the current x from double[n] (entries at s and t are ignored): a warm
 * start, a resume from a saved iterate, or a teacher-forced step. */
pirmcut_status pirmcut_set_x(pirmcut_ctx* ctx, const double* x, int mem_kind);

/*
 * Replace the capacities of the instance while keeping its structure (a
 * sequence of related problems, Section 6): c is double[nnz] (float[nnz]
 * with options.capacity_fp32) in the CSR layout given to pirmcut_create.
 * The current x is kept as a warm start.
 * Errors: EINVAL (non-finite, negative or asymmetric c), EDISCONNECTED, ECUDA.
 */
pirmcut_status pirmcut_update_weights(pirmcut_ctx* ctx, const void* c, int mem_kind);

/* Sizes of the reduced problem: n~ (non-terminals), e~ (non-terminal
 * undirected edges), and the storage format chosen (PIRMCUT_FORMAT_DIA/CSR). */
pirmcut_status pirmcut_problem_size(const pirmcut_ctx* ctx, int64_t* n_nonterminal,
                                    int64_t* n_edges, int* format);

/* Number of kernel launches the context has issued so far (graph launches
 * count each kernel node they run). */
int64_t pirmcut_kernel_launches(const pirmcut_ctx* ctx);

/*
 * Diagnostics for roofline reports: time the PCG matrix-vector kernel
 * (q = L~ p with the fused (p, q) reduction, Section 3.1; for MIXED contexts
 * the FP32 inner one, which on DIA grids whose width is a multiple of 4 also
 * forms the new search direction and applies the previous d update) on the
 * current matrix and search direction, `reps` launches bracketed one by one
 * with CUDA events on the context's stream, each after a 256 MB write that
 * evicts L2 (outside the timed interval; the buffer is allocated for the call).
 * Needs a completed step (EINVAL otherwise); leaves x untouched (the FP32
 * scratch vectors are overwritten).  avg_ms receives the mean launch time; bytes and flops
 * (either may be NULL) the algorithmic bytes moved and floating-point
 * operations of one launch (every stored value, matrix index and vector entry
 * read or written once; an FMA counts 2).
 */
pirmcut_status pirmcut_time_spmv(pirmcut_ctx* ctx, int reps, double* avg_ms, double* bytes,
                                 double* flops);

/*
 * The matrix-vector launches timed during solves run with time_spmv = 1 and
 * graph_launch = 0: their summed CUDA-event time in milliseconds and their
 * count, since creation or the last reset (reset != 0 clears the totals after
 * reading).  Launches that found the stop test already met (and skipped their
 * work) are not counted; the algorithmic bytes of one launch are those that
 * pirmcut_time_spmv reports.  Errors: EINVAL (NULL ctx).
 */
pirmcut_status pirmcut_spmv_timing(pirmcut_ctx* ctx, double* total_ms, int64_t* launches, int reset);

/*
 * Two-level rounding (Section 3.3) of the current x: 1-D K-means on x with
 * centres started at 0.1 and 0.9 (each value to the nearer centre, the lower
 * on a tie; centres = means; until the assignment is stable; s and t included
 * with x_s = 1, x_t = 0) gives gamma0 = c0 + 0.05 and gamma1 = c1 - 0.05.
 * Vertices with x <= gamma0 are contracted into t, x >= gamma1 into s; the
 * coarse graph keeps every edge between the remaining vertices and sums the
 * rest per the paper's four cases; its s-t min cut (exact max-flow, host side)
 * induces the returned cut of G.
 *
 * side   uint8[n] (may be NULL) in mem_kind memory: 1 on the source side.
 * value  (may be NULL) exact FP64 cut value of the returned side.
 * gamma  (may be NULL) double[2] = {gamma0, gamma1}.
 * coarse_vertices (may be NULL) number of vertices of the coarse graph.
 * Errors: EINVAL (x unset), ENOMEM, ECUDA.
 */
pirmcut_status pirmcut_cut_two_level(pirmcut_ctx* ctx, uint8_t* side, double* value, double* gamma,
                                     int64_t* coarse_vertices, int mem_kind);

/*
 * Learned warm start.  The paper starts the PCG of step l from x^(l-1)
 * (Section 3.1) and aims at sequences of related problems (Section 6).  With
 * PIRMCUT_MLP_PREDICT on, each IRLS step after x^(0) (with warm_start = 1)
 * starts instead from x^(l-1) + alpha * d, where d is a per-node direction
 * predicted by an MLP (6 features -> 64 -> 64 -> 1, ReLU; BF16 weights;
 * inference on the tensor cores with BF16 operands -- the features enter as
 * a BF16 head and tail, about 2^-17 relative -- and FP32 accumulation) and
 * alpha comes from an exact line search (FP64) on the
 * quadratic energy E(v) = v^T L~ v - 2 b^T v = ||v - v*||^2_{L~} - const:
 *   alpha = d^T r / d^T L~ d,  r = b - L~ x^(l-1)   (alpha = 0 if d^T L~ d <= 0).
 * E is the error norm that CG minimises, so the learned start is never
 * worse than x^(l-1) in that norm: the plain warm start is the fallback and
 * the yardstick.  The conductances always come from x^(l-1), so the solved system
 * is unchanged and every result keeps the solver's tolerance.
 * The features of node v, all of step l:
 *   f0 x^(l-1)_v;
 *   f1, f2 mean and standard deviation of the neighbours' x^(l-1), weighted by
 *          the new conductances, s and t included (x_s = 1, x_t = 0);
 *   f3 mean of log(g^(l)/g^(l-1)) over v's non-terminal edges with both
 *      conductances positive (0 if none), / 8; g^(l-1) are the conductances
 *      of the last step this context ran (the capacities after creation);
 *   f4 log of the weighted degree of v in L~ (its diagonal entry), / 8;
 *   f5 log(eps_l) / 8.
 * With PIRMCUT_MLP_TRAIN on, each such step ends with 8 Adam steps (by
 * default; learning rate 1e-3) on minibatches of 2048 nodes drawn by a
 * counter-based hash (SplitMix64), fitting d to x^(l) - x^(l-1) (mean squared
 * error).  Everything runs on the GPU inside the step; results are
 * reproducible.
 *
 * Weight layout (PIRMCUT_MLP_PARAMS floats, row-major, out x in):
 *   W1[64][6] b1[64] W2[64][64] b2[64] w3[64] b3.
 *
 * pirmcut_mlp_enable: mode = 0 or an OR of the two flags.  The first call
 *   with mode != 0 allocates the model and its buffers (two doubles and six
 *   floats per non-terminal plus one copy of the conductances) and
 *   initialises it from seed: Glorot-uniform W1, W2, zero biases and output
 *   layer, so an untrained model proposes d = 0 (alpha = 0).  Later calls
 *   change the mode only (weights and statistics are kept, e.g. across
 *   pirmcut_update_weights).  The step graphs are rebuilt on the next solve.
 *   Errors: EINVAL (mode), ENOMEM, ECUDA.
 * pirmcut_mlp_configure: iters_per_step Adam steps (0..1024, default 8) with
 *   learning rate learning_rate (> 0, default 1e-3) after each step when
 *   training.  Errors: EINVAL.
 * pirmcut_mlp_predict: the model's output d for count feature rows
 *   (float[count * 6], row-major) into float[count]; both arrays in mem_kind
 *   memory.  Errors: EINVAL (no model, sizes), ENOMEM, ECUDA, ETIMEOUT (a
 *   bounded wait on the tensor cores expired).
 * pirmcut_mlp_weights: direction 0 copies the FP32 master weights to w
 *   (host, PIRMCUT_MLP_PARAMS floats); direction 1 loads them from w and
 *   resets the optimizer state.  Errors: EINVAL (no model, NULL w), ECUDA.
 * pirmcut_mlp_stats: steps that ran the line search, steps that moved
 *   (alpha != 0), Adam steps taken, the last minibatch loss; for the last
 *   step alpha, the energy change E(start) - E(x^(l-1)) (<= 0) and
 *   ||b - L~ x^(l-1)||_2; the mean of alpha over steps.
 * pirmcut_mlp_features: the features of the last step, float[n~ * 6] in host
 *   memory, in reduced numbering (the caller's order with s and t removed).
 */
#define PIRMCUT_MLP_PREDICT 1
#define PIRMCUT_MLP_TRAIN 2
#define PIRMCUT_MLP_FEATURES 6
#define PIRMCUT_MLP_PARAMS 4673
typedef struct {
  int steps;
  int used;
  int train_steps;
  float loss;
  double alpha;
  double energy_change;
  double res_plain;
  double mean_alpha;
  int tensor_timeouts; /* 1 once a bounded wait of the tensor-core network
                          expired (its outputs past that point were not
                          written; the line search then uses what it finds) */
} pirmcut_mlp_info;
pirmcut_status pirmcut_mlp_enable(pirmcut_ctx* ctx, int mode, uint64_t seed);
pirmcut_status pirmcut_mlp_configure(pirmcut_ctx* ctx, int iters_per_step, float learning_rate);
pirmcut_status pirmcut_mlp_predict(pirmcut_ctx* ctx, const float* features, int64_t count,
                                   float* delta, int mem_kind);
pirmcut_status pirmcut_mlp_weights(pirmcut_ctx* ctx, float* w, int direction);
pirmcut_status pirmcut_mlp_stats(pirmcut_ctx* ctx, pirmcut_mlp_info* info);
/* Diagnostics for roofline reports: reps launches of the inference kernel of
 * pirmcut_mlp_predict on count feature rows (device memory, as there),
 * back to back between CUDA events on the context's stream after one
 * untimed launch; avg_ms receives the mean time per launch.  Errors:
 * EINVAL, ECUDA, ETIMEOUT. */
pirmcut_status pirmcut_mlp_time_predict(pirmcut_ctx* ctx, const float* features, int64_t count,
                                        float* delta, int reps, double* avg_ms);
pirmcut_status pirmcut_mlp_features(pirmcut_ctx* ctx, float* f);

/*
 * Sweep cut that allocates no memory.  The paper has no counterpart: this
 * entry point exists for callers that cannot call cudaMalloc -- code that runs
 * while a stream is being captured into a CUDA graph (an allocation there
 * would break or invalidate the capture), host frameworks that own all device
 * memory through their own pool and forbid allocations from libraries, and
 * real-time loops that must never block in the allocator.
 *
 * It returns what pirmcut_cut returns for the same graph and x (same sweep
 * order, candidates and tie rules; FP64 throughout), computed by a single
 * thread block directly from a full CSR in device memory, without a context.
 * Its scratch is one fixed array in the library's device memory of
 * 36 * PIRMCUT_STATIC_MAX_NONTERMINALS bytes (about 2.4 MB), which every GPU
 * that loads the library holds until the process exits.
 *
 * n, row_ptr, col, c, s, t  the graph exactly as for pirmcut_create, but every
 *          array in device memory; it must already be valid (the library
 *          reads it as is: out-of-range column ids are skipped and reported
 *          in result[3], nothing else is checked).  n - 2 must not exceed
 *          PIRMCUT_STATIC_MAX_NONTERMINALS, otherwise EINVAL.
 * x        double[n] in device memory, the voltages to round.
 * side     uint8[n] in device memory, receives 1 on the source side, 0 else.
 * result   double[4] in device memory: {cut value, tau, chosen prefix length
 *          k, 1 if an out-of-range column id was met else 0}.
 * stream   cudaStream_t (as void*) the kernel is queued on; the call returns
 *          without waiting for it.
 *
 * The first call on a device looks up the scratch array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture begins.  All calls on a device share the one
 * array, so calls that may overlap on the GPU (other streams, other host
 * threads) race and must be serialised by the caller.  No part of the array
 * needs to start cleared: every entry a call reads it has written first.
 * Errors: EINVAL (sizes, terminals, null pointers; see pirmcut_last_error(NULL)),
 * ECUDA (lookup or launch failed).
 */
#define PIRMCUT_STATIC_MAX_NONTERMINALS 65536
pirmcut_status pirmcut_sweep_cut_static(int64_t n, const int64_t* row_ptr, const int32_t* col,
                                        const double* c, int32_t s, int32_t t, const double* x,
                                        uint8_t* side, double* result, void* stream);

/*
 * Batches of independent instances (Section 6: sequences and batches of
 * related FlowImprove problems).  All instances of a batch are solved together:
 * every kernel launch covers all of them, each instance keeps its own PCG
 * scalars and stopping test, and one CUDA graph per IRLS step runs until every
 * instance has converged.  FP64 solver, CSR storage; options as for
 * pirmcut_create (precision must be FP64).
 *
 * pirmcut_batch_create: count instances; n[i], row_ptr[i], col[i], c[i],
 * s[i], t[i] describe instance i exactly as the arguments of pirmcut_create
 * (host memory).  Rows are processed in three tiers by degree: short rows by
 * groups of threads per row in consecutive-row tiles, longer rows a warp each,
 * hub rows (more than 512 entries) a block each.  At creation an autotuner
 * times the batched SpMV for several (threads per row, tile height, warp-row
 * threshold) choices and keeps the fastest.
 * Errors: EINVAL (with the failing instance in the message), EDISCONNECTED,
 * ENOMEM, ECUDA.
 */
typedef struct pirmcut_batch pirmcut_batch;
pirmcut_status pirmcut_batch_create(int count, const int64_t* n, const int64_t* const* row_ptr,
                                    const int32_t* const* col, const double* const* c,
                                    const int32_t* s, const int32_t* t, const pirmcut_options* opt,
                                    void* stream, pirmcut_batch** out);
/* x^(0) and T IRLS steps for every instance (Algorithm 1 steps 2-4).  infos
 * (may be NULL) receives count * (T+1) records, instance-major; their ms field
 * is the step's time for the whole batch. */
pirmcut_status pirmcut_batch_solve(pirmcut_batch* b, int T, const double* eps,
                                   pirmcut_step_info* infos);
/* Sweep cut of instance index (host outputs; side is uint8[n_index] or NULL). */
pirmcut_status pirmcut_batch_cut(pirmcut_batch* b, int index, uint8_t* side, double* value,
                                 double* tau);
/* x of instance index, double[n_index] in host memory (x_s = 1, x_t = 0). */
pirmcut_status pirmcut_batch_get_x(pirmcut_batch* b, int index, double* x);
/* Totals and the autotuner's choice: threads per short row, rows per
 * consecutive-row tile, the number of tiles, and medium_deg (rows with more
 * entries, up to the hub threshold, are processed a warp each; equal to the
 * hub threshold when that tier is off).  Any output pointer may be NULL. */
pirmcut_status pirmcut_batch_info(const pirmcut_batch* b, int64_t* total_rows, int64_t* total_nnz,
                                  int* threads_per_row, int* tile_rows, int* tiles,
                                  int64_t* medium_deg);
/* Kernels the batch has launched so far (creation's autotuner included; the
 * kernels of a graph launch are counted by its structure).  0 for NULL. */
int64_t pirmcut_batch_kernel_launches(const pirmcut_batch* b);
/* Free every host and device resource of the batch (after its stream's work
 * has finished).  NULL is ignored. */
void pirmcut_batch_destroy(pirmcut_batch* b);

/* Text of the last error of ctx (or of the last failed create when ctx is NULL). */
const char* pirmcut_last_error(const pirmcut_ctx* ctx);

/* Free every host and device resource of ctx.  NULL is ignored. */
void pirmcut_destroy(pirmcut_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* PIRMCUT_H */
