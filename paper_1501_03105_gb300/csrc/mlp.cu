// Learned warm start for the linear solve of each IRLS step.
//
// The paper starts the PCG of step l from v^(l-1) (Section 3.1) and targets
// sequences of closely related problems (Section 6).  Here a small per-node
// MLP (6 -> 64 -> 64 -> 1, ReLU, BF16 weights, FP32 accumulation) predicts
// the change x^(l) - x^(l-1) from local features of step l:
//   f0  x^(l-1)_v
//   f1  mean of the neighbours' voltages weighted by the new conductances,
//       terminals included (x_s = 1, x_t = 0): one Jacobi sweep of the new system
//   f2  weighted standard deviation of those voltages
//   f3  mean over the incident non-terminal edges of log(g^(l) / g^(l-1)), / 8
//   f4  log of the weighted degree (the diagonal of L~), / 8
//   f5  log(eps_l) / 8
// The start is x^(l-1) + alpha * delta with alpha from an exact line search
// on the quadratic energy E(v) = v^T L~ v - 2 b^T v = ||v - v*||_{L~}^2 - const
// (FP64): alpha = delta^T r / delta^T L~ delta with r = b - L~ x^(l-1).  E is
// the error norm CG minimises, so the learned start is never worse than the
// plain warm start (alpha = 0 is always available): x^(l-1) is both the
// fallback and the yardstick.  The reweighting point stays x^(l-1) (in xprev).
// Inference runs on the tcgen05 tensor cores (BF16 operands, FP32
// accumulation in tensor memory; mlp_tc.cuh), the features in FP32 on DIA
// grids (a memory-bound pass) and FP64 on CSR rows.
// Training runs on the trajectory the solver itself produces: after a step,
// minibatches of nodes drawn by a counter-based hash go through hand-written
// forward/backward kernels written as block-level GEMMs over each block's
// samples; each block sums its samples' gradients in a fixed order, blocks
// are summed in block order, and one Adam step updates the FP32 master
// weights and their BF16 copy.  Runs are bit-reproducible.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>

#include "ctx.h"
#include "mlp_tc.cuh"

namespace pirmcut {

namespace {

constexpr int H = 64;
constexpr int NF = kMlpFeatures;
constexpr int OFF_W1 = 0;                 // [H][NF]
constexpr int OFF_B1 = OFF_W1 + H * NF;   // [H]
constexpr int OFF_W2 = OFF_B1 + H;        // [H][H]
constexpr int OFF_B2 = OFF_W2 + H * H;    // [H]
constexpr int OFF_W3 = OFF_B2 + H;        // [H]
constexpr int OFF_B3 = OFF_W3 + H;        // [1]
constexpr int NPARAM = OFF_B3 + 1;
static_assert(NPARAM == kMlpParams, "parameter layout");
constexpr int TRAIN_BLOCKS = 32;
constexpr int SAMPLES_PER_BLOCK = 64;

// SplitMix64 finaliser (Steele, Lea, Flood 2014): a counter-based generator.
__device__ __forceinline__ uint64_t splitmix64(uint64_t z) {
  z += 0x9e3779b97f4a7c15ull;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ float uniform01(uint64_t h) {
  return float(h >> 40) * (1.0f / 16777216.0f);
}

// Glorot-uniform hidden weights, zero biases, zero output layer (so that an
// untrained model predicts no change and the candidate is never chosen).
__global__ void k_mlp_init(float* master, __nv_bfloat16* w16, float* m, float* v, uint64_t seed) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < NPARAM; i += gridDim.x * blockDim.x) {
    float a = 0.0f;
    if (i < OFF_B1) a = sqrtf(6.0f / float(NF + H));
    else if (i >= OFF_W2 && i < OFF_B2) a = sqrtf(6.0f / float(H + H));
    const float w = a * (2.0f * uniform01(splitmix64(seed * 0x100000001b3ull + uint64_t(i))) - 1.0f);
    master[i] = w;
    w16[i] = __float2bfloat16(w);
    m[i] = 0.0f;
    v[i] = 0.0f;
  }
}

// after the host wrote master: BF16 copy, fresh Adam moments
__global__ void k_mlp_refresh(const float* master, __nv_bfloat16* w16, float* m, float* v, MlpState* M) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < NPARAM; i += gridDim.x * blockDim.x) {
    w16[i] = __float2bfloat16(master[i]);
    m[i] = 0.0f;
    v[i] = 0.0f;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) M->train_steps = 0;
}

__device__ __forceinline__ void finish_features(float* __restrict__ f, int64_t i, double xi,
                                                double wsum, double wx, double wxx, float lr,
                                                int nlr, double gs, double gt, double eps) {
  wsum += gs + gt;
  wx += gs;  // x_s = 1; x_t = 0 adds nothing
  wxx += gs;
  const double mean = wx / wsum;
  const double var = fmax(wxx / wsum - mean * mean, 0.0);
  float* o = f + i * NF;
  o[0] = float(xi);
  o[1] = float(mean);
  o[2] = sqrtf(float(var));
  o[3] = nlr ? lr / float(nlr) * 0.125f : 0.0f;
  o[4] = logf(float(wsum)) * 0.125f;
  o[5] = logf(float(eps)) * 0.125f;
}

__device__ __forceinline__ void edge_feature(double w, double w0, double xj, double& wsum,
                                             double& wx, double& wxx, float& lr, int& nlr) {
  wsum += w;
  wx = fma(w, xj, wx);
  wxx = fma(w * xj, xj, wxx);
  if (w > 0.0 && w0 > 0.0) {
    lr += logf(float(w) / float(w0));
    ++nlr;
  }
}

__global__ void __launch_bounds__(kThreads)
k_features_csr(int64_t nt, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
               const double* __restrict__ g, const double* __restrict__ gprev,
               const double* __restrict__ cs, const double* __restrict__ ct,
               const double* __restrict__ x, const double* __restrict__ eps_list,
               const StepCounters* __restrict__ C, int form, float* __restrict__ f,
               int64_t heavy_deg, const int32_t* __restrict__ heavy, int light_blocks) {
  const double eps = eps_list[C->eps_idx];
  const double eps2 = eps * eps;
  if (int(blockIdx.x) >= light_blocks) {  // one heavy row (a hub) for the whole block
    const int64_t i = heavy[blockIdx.x - light_blocks];
    double wsum = 0.0, wx = 0.0, wxx = 0.0;
    float lr = 0.0f;
    int nlr = 0;
    for (int64_t e = rp[i] + threadIdx.x; e < rp[i + 1]; e += blockDim.x)
      edge_feature(g[e], gprev[e], x[col[e]], wsum, wx, wxx, lr, nlr);
    double v[5] = {wsum, wx, wxx, double(lr), double(nlr)};
    block_sum<5>(v);
    if (threadIdx.x == 0) {
      const double xi = x[i];
      const double gs = conductance(cs[i], 1.0 - xi, eps2, form);
      const double gt = conductance(ct[i], xi, eps2, form);
      finish_features(f, i, xi, v[0], v[1], v[2], float(v[3]), int(v[4]), gs, gt, eps);
    }
    return;
  }
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < nt;
       i += int64_t(light_blocks) * blockDim.x) {
    if (rp[i + 1] - rp[i] > heavy_deg) continue;
    const double xi = x[i];
    double wsum = 0.0, wx = 0.0, wxx = 0.0;
    float lr = 0.0f;
    int nlr = 0;
    for (int64_t e = rp[i]; e < rp[i + 1]; ++e)
      edge_feature(g[e], gprev[e], x[col[e]], wsum, wx, wxx, lr, nlr);
    const double gs = conductance(cs[i], 1.0 - xi, eps2, form);
    const double gt = conductance(ct[i], xi, eps2, form);
    finish_features(f, i, xi, wsum, wx, wxx, lr, nlr, gs, gt, eps);
  }
}


// Conductance in FP32 (a feature input only): the two reweighting forms.
__device__ __forceinline__ float conductance32(float c, float d, float eps2, int form) {
  if (form == PIRMCUT_REWEIGHT_PAPER) {
    const float cd = c * d;
    return c * c * rsqrtf(fmaf(cd, cd, eps2));
  }
  return c * rsqrtf(fmaf(d, d, eps2));
}

// The six features of DIA row i (< nt) in FP32: neighbour differences
// x_u - x_i are formed in FP64 and then truncated, the weighted mean and
// variance of the neighbours' voltages are taken about x_i in two passes
// (no cancellation), logarithms in FP32.
template <int K>
__device__ __forceinline__ void features_dia32(const DiaDesc& d, const double* __restrict__ g,
                                               const double* __restrict__ gprev,
                                               const double* __restrict__ cs,
                                               const double* __restrict__ ct,
                                               const double* __restrict__ x, float eps2f,
                                               float log_eps8, int form, int64_t i, float (&f)[NF]) {
  const int64_t nt = d.nt;
  const double xi = x[i];
  float w[2 * K + 2], dx[2 * K + 2];
  float lr = 0.f;
  int nlr = 0;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const int64_t o = d.off[k];
    w[2 * k] = 0.f;
    dx[2 * k] = 0.f;
    w[2 * k + 1] = 0.f;
    dx[2 * k + 1] = 0.f;
    if (i + o < nt) {
      const float wu = f32_trunc(g[k * nt + i]), wp = f32_trunc(gprev[k * nt + i]);
      w[2 * k] = wu;
      dx[2 * k] = f32_trunc(x[i + o] - xi);
      if (wu > 0.f && wp > 0.f) {
        lr += __log2f(wu) - __log2f(wp);
        ++nlr;
      }
    }
    if (i >= o) {
      const float wu = f32_trunc(g[k * nt + i - o]), wp = f32_trunc(gprev[k * nt + i - o]);
      w[2 * k + 1] = wu;
      dx[2 * k + 1] = f32_trunc(x[i - o] - xi);
      if (wu > 0.f && wp > 0.f) {
        lr += __log2f(wu) - __log2f(wp);
        ++nlr;
      }
    }
  }
  // terminals: x_s = 1, x_t = 0, conductances of step l from x^(l-1)
  const float ds = f32_trunc(1.0 - xi), dt = -f32_trunc(xi);
  w[2 * K] = conductance32(f32_trunc(cs[i]), ds, eps2f, form);
  dx[2 * K] = ds;
  w[2 * K + 1] = conductance32(f32_trunc(ct[i]), dt, eps2f, form);
  dx[2 * K + 1] = dt;
  float wsum = 0.f, wd = 0.f;
#pragma unroll
  for (int k = 0; k < 2 * K + 2; ++k) {
    wsum += w[k];
    wd = fmaf(w[k], dx[k], wd);
  }
  const float inv = 1.0f / wsum;
  const float m = wd * inv;
  float var = 0.f;
#pragma unroll
  for (int k = 0; k < 2 * K + 2; ++k) {
    const float e = dx[k] - m;
    var = fmaf(w[k] * e, e, var);
  }
  const float x32 = f32_trunc(xi);
  f[0] = x32;
  f[1] = x32 + m;
  f[2] = sqrtf(var * inv);
  f[3] = nlr ? lr * (0.69314718f * 0.125f) / float(nlr) : 0.f;
  f[4] = logf(wsum) * 0.125f;
  f[5] = log_eps8;
}

// ---- Inference on the tcgen05 tensor cores (mlp_tc.cuh: BF16 operands,
// FP32 accumulation in tensor memory): one CTA of 128 threads walks 128-row
// tiles, one thread per row.  Five CTAs share an SM (64 TMEM columns each).
// A wait that expires sets M->tc_error.

// The features of a DIA grid in FP32 (features_dia32), one row per thread:
// a memory-bound pass; the network then reads them (k_mlp_predict_t5).
template <int K>
__global__ void __launch_bounds__(kThreads)
k_features_dia32(DiaDesc d, const double* __restrict__ g, const double* __restrict__ gprev,
                 const double* __restrict__ cs, const double* __restrict__ ct,
                 const double* __restrict__ x, const double* __restrict__ eps_list,
                 const StepCounters* __restrict__ C, int form, float* __restrict__ feat) {
  const int64_t nt = d.nt;
  const double eps = eps_list[C->eps_idx];
  const float eps2f = float(eps) * float(eps);
  const float log_eps8 = logf(float(eps)) * 0.125f;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < nt;
       i += int64_t(gridDim.x) * blockDim.x) {
    float f[NF];
    features_dia32<K>(d, g, gprev, cs, ct, x, eps2f, log_eps8, form, i, f);
#pragma unroll
    for (int k = 0; k < NF; ++k) feat[i * NF + k] = f[k];
  }
}

// The network on stored feature rows (CSR problems, and the inference entry
// point): delta -> dir (FP64) or out32 (FP32).
template <bool kF32>
__global__ void __launch_bounds__(128, 5)
k_mlp_predict_t5(int64_t nt, const float* __restrict__ f, const __nv_bfloat16* __restrict__ w16,
                 double* __restrict__ dir, float* __restrict__ out32, MlpState* M) {
  __shared__ tc5::Smem S;
  tc5::setup(S, w16);
  uint32_t phase = 0;
  bool ok = true;
  const int64_t tiles = (nt + tc5::kRows - 1) / tc5::kRows;
  // the next tile's features are loaded while this one runs
  auto load = [&](int64_t t, float (&v)[NF]) {
    const int64_t i = t * tc5::kRows + threadIdx.x;
#pragma unroll
    for (int k = 0; k < NF; ++k) v[k] = 0.f;
    if (t < tiles && i < nt) {
#pragma unroll
      for (int k = 0; k < NF; ++k) v[k] = __ldcs(f + i * NF + k);
    }
  };
  float nxt[NF];
  load(blockIdx.x, nxt);
  for (int64_t t = blockIdx.x; t < tiles && ok; t += gridDim.x) {
    const int64_t i = t * tc5::kRows + threadIdx.x;
    float in[NF];
#pragma unroll
    for (int k = 0; k < NF; ++k) in[k] = nxt[k];
    load(t + gridDim.x, nxt);
    float out = 0.f;
    ok = tc5::tile(S, in, phase, out);
    if (ok && i < nt) {
      if (kF32) out32[i] = out;
      else dir[i] = double(out);
    }
  }
  if (!ok) {
    tc5::wait_phase(tc5::smem_u32(&S.mbar), phase);
    if (threadIdx.x == 0) atomicExch(&M->tc_error, 1);
  }
  tc5::teardown(S);
}

// Resident CTAs per SM of the tcgen05 kernels: five (registers bound them;
// 5 x 64 TMEM columns of the SM's 512; shared memory would allow six).
constexpr int kT5PerSm = 5;
static_assert(kT5PerSm * tc5::kTmemCols <= 512, "tensor memory of an SM");
constexpr size_t kT5Pad = 0;

// CTAs of the tcgen05 kernels: kT5PerSm per SM, never more than there are tiles.
inline int mlp_t5_grid(int64_t rows) {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0, v = 152;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0)
      sms = v;
    else
      sms = 152;
  }
  const int64_t tiles = (rows + tc5::kRows - 1) / tc5::kRows;
  const int64_t cap = int64_t(sms) * kT5PerSm;
  return int(tiles < 1 ? 1 : (tiles < cap ? tiles : cap));
}


// Line search of the mixed path along the learned direction d from
// x = x^(l-1), after the assembly (its FP64 diagonal and b = g(s, .)): with
// r = b - L~ x, the last block forms alpha = (d, r) / (d, L~ d) (0 when the
// denominator is not positive and finite) and the energy change
// -(d, r)^2 / (d, L~ d).  No conductance is computed again.
__device__ __forceinline__ void linesearch_finish(double dr, double dad, double rr, double* partials,
                                                  MlpState* M) {
  double v[3] = {dr, dad, rr}, tot[3];
  if (grid_sum<3>(v, partials, &M->counter, tot) && threadIdx.x == 0) {
    const double a = tot[1] > 0.0 ? tot[0] / tot[1] : 0.0;
    const bool ok = isfinite(a) && a != 0.0;
    M->alpha = ok ? a : 0.0;
    M->energy_change = ok ? -tot[0] * a : 0.0;
    M->res_plain = tot[2];
  }
}

template <int K>
__global__ void __launch_bounds__(kThreads)
k_linesearch_dia(DiaDesc d, const double* __restrict__ g, const double* __restrict__ diag,
                 const double* __restrict__ b, const double* __restrict__ x,
                 const double* __restrict__ dir, double* partials, MlpState* M) {
  const int64_t nt = d.nt;
  double dr = 0.0, dad = 0.0, rr = 0.0;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < nt;
       i += int64_t(gridDim.x) * blockDim.x) {
    const double xi = x[i], di = dir[i], dg = diag[i];
    double ax = 0.0, ad = 0.0;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int64_t o = d.off[k];
      if (i + o < nt) {
        const double w = g[k * nt + i];
        ax = fma(w, x[i + o], ax);
        ad = fma(w, dir[i + o], ad);
      }
      if (i >= o) {
        const double w = g[k * nt + i - o];
        ax = fma(w, x[i - o], ax);
        ad = fma(w, dir[i - o], ad);
      }
    }
    const double r = b[i] - fma(dg, xi, -ax);
    dr = fma(di, r, dr);
    dad = fma(di, fma(dg, di, -ad), dad);
    rr = fma(r, r, rr);
  }
  linesearch_finish(dr, dad, rr, partials, M);
}

__global__ void __launch_bounds__(kThreads)
k_linesearch_csr(int64_t nt, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                 const double* __restrict__ g, const double* __restrict__ diag,
                 const double* __restrict__ b, const double* __restrict__ x,
                 const double* __restrict__ dir, double* partials, MlpState* M,
                 int64_t heavy_deg, const int32_t* __restrict__ heavy, int light_blocks) {
  double dr = 0.0, dad = 0.0, rr = 0.0;
  if (int(blockIdx.x) >= light_blocks) {  // one heavy row (a hub) for the whole block
    const int64_t i = heavy[blockIdx.x - light_blocks];
    double v[2] = {0.0, 0.0};  // (g, x), (g, d) over the row
    for (int64_t e = rp[i] + threadIdx.x; e < rp[i + 1]; e += blockDim.x) {
      const double w = g[e];
      v[0] = fma(w, x[col[e]], v[0]);
      v[1] = fma(w, dir[col[e]], v[1]);
    }
    block_sum<2>(v);
    if (threadIdx.x == 0) {
      const double xi = x[i], di = dir[i], dg = diag[i];
      const double r = b[i] - fma(dg, xi, -v[0]);
      dr = di * r;
      dad = di * fma(dg, di, -v[1]);
      rr = r * r;
    }
    linesearch_finish(dr, dad, rr, partials, M);
    return;
  }
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < nt;
       i += int64_t(light_blocks) * blockDim.x) {
    if (rp[i + 1] - rp[i] > heavy_deg) continue;
    const double xi = x[i], di = dir[i], dg = diag[i];
    double ax = 0.0, ad = 0.0;
    for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
      const double w = g[e];
      ax = fma(w, x[col[e]], ax);
      ad = fma(w, dir[col[e]], ad);
    }
    const double r = b[i] - fma(dg, xi, -ax);
    dr = fma(di, r, dr);
    dad = fma(di, fma(dg, di, -ad), dad);
    rr = fma(r, r, rr);
  }
  linesearch_finish(dr, dad, rr, partials, M);
}

// x += alpha * d
__global__ void __launch_bounds__(kThreads)
k_mlp_commit(int64_t nt, MlpState* M, const double* __restrict__ dir, double* __restrict__ x) {
  const double a = M->alpha;
  if (a != 0.0) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < nt;
         i += int64_t(gridDim.x) * blockDim.x)
      x[i] = fma(a, dir[i], x[i]);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    M->steps += 1;
    M->used += a != 0.0 ? 1 : 0;
    M->sum_alpha += a;
  }
}

// One minibatch as block-level GEMMs.  Block b takes the SAMPLES_PER_BLOCK
// (64) nodes drawn for it and runs the forward and backward pass of its
// samples together, FP32 arithmetic on the BF16 weights:
//   Z1 = F W1^T + b1,  H1 = relu(Z1)                      [64 x 64]
//   Z2 = H1 W2^T + b2, out = relu(Z2) w3 + b3             [64 x 64], [64]
//   dZ2 = (2 (out - target) / batch) w3^T . [Z2 > 0]
//   dW2 = dZ2^T H1,  dH1 = dZ2 W2,  dZ1 = dH1 . [Z1 > 0],  dW1 = dZ1^T F
// Each of the 256 threads owns a 4 x 4 tile of every 64 x 64 product; the
// sums over the samples of a block run in a fixed order, and grad_part[b]
// receives the block's gradient (summed over blocks in block order by the
// Adam step), so that training is reproducible.
constexpr int GB_THREADS = 256;
constexpr int LD = H + 1;  // padded row stride of the 64 x 64 tiles in shared memory
constexpr size_t GRAD_SMEM =
    sizeof(float) * (size_t(H) * LD * 3 + H * NF + 3 * H + 1 + SAMPLES_PER_BLOCK * (NF + 2) +
                     GB_THREADS);

__global__ void __launch_bounds__(GB_THREADS)
k_mlp_grad(int64_t nt, const float* __restrict__ f, const double* __restrict__ x,
           const double* __restrict__ xprev, const __nv_bfloat16* __restrict__ w16,
           const MlpState* __restrict__ M, uint64_t seed, float* __restrict__ grad_part,
           float* __restrict__ loss_part) {
  extern __shared__ float sm[];
  float* W2s = sm;                          // [j][k], stride LD
  float* Z1 = W2s + H * LD;                 // [s][k]: Z1, later dZ1
  float* D2 = Z1 + H * LD;                  // [s][j]: dZ2
  float* W1s = D2 + H * LD;                 // [k][m]
  float* b1s = W1s + H * NF;
  float* b2s = b1s + H;
  float* w3s = b2s + H;
  float* b3s = w3s + H;                     // [1]
  float* Fs = b3s + 1;                      // [s][m]
  float* tgt = Fs + SAMPLES_PER_BLOCK * NF; // [s]
  float* dout = tgt + SAMPLES_PER_BLOCK;    // [s]
  float* red = dout + SAMPLES_PER_BLOCK;    // [GB_THREADS] per-thread partials
  const int t = threadIdx.x;
  for (int i = t; i < H * H; i += GB_THREADS) W2s[(i / H) * LD + i % H] = __bfloat162float(w16[OFF_W2 + i]);
  for (int i = t; i < H * NF; i += GB_THREADS) W1s[i] = __bfloat162float(w16[OFF_W1 + i]);
  if (t < H) {
    b1s[t] = __bfloat162float(w16[OFF_B1 + t]);
    b2s[t] = __bfloat162float(w16[OFF_B2 + t]);
    w3s[t] = __bfloat162float(w16[OFF_W3 + t]);
  }
  if (t == 0) b3s[0] = __bfloat162float(w16[OFF_B3]);
  const uint64_t stream = splitmix64(seed ^ (uint64_t(M->train_steps) << 20));
  if (t < SAMPLES_PER_BLOCK) {
    const uint64_t hsh = splitmix64(stream + uint64_t(blockIdx.x) * SAMPLES_PER_BLOCK + uint64_t(t));
    const int64_t node = int64_t(hsh % uint64_t(nt));
#pragma unroll
    for (int m = 0; m < NF; ++m) Fs[t * NF + m] = f[node * NF + m];
    tgt[t] = float(x[node] - xprev[node]);
  }
  __syncthreads();
  // Z1 (16 entries per thread)
  for (int i = t; i < SAMPLES_PER_BLOCK * H; i += GB_THREADS) {
    const int s = i / H, k = i % H;
    float z = b1s[k];
#pragma unroll
    for (int m = 0; m < NF; ++m) z = fmaf(W1s[k * NF + m], Fs[s * NF + m], z);
    Z1[s * LD + k] = z;
  }
  __syncthreads();
  // Z2 tile (samples 4 ts .. 4 ts + 3, units 4 tj .. 4 tj + 3); a half-warp
  // shares ts, so the output's reduction over j stays inside it
  const int ts = t >> 4, tj = t & 15;
  float z2[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b2 = 0; b2 < 4; ++b2) z2[a][b2] = b2s[4 * tj + b2];
  for (int k = 0; k < H; ++k) {
    float hv[4], wv[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) hv[a] = fmaxf(Z1[(4 * ts + a) * LD + k], 0.f);
#pragma unroll
    for (int b2 = 0; b2 < 4; ++b2) wv[b2] = W2s[(4 * tj + b2) * LD + k];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b2 = 0; b2 < 4; ++b2) z2[a][b2] = fmaf(hv[a], wv[b2], z2[a][b2]);
  }
  float po[4];
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    po[a] = 0.f;
#pragma unroll
    for (int b2 = 0; b2 < 4; ++b2) po[a] = fmaf(fmaxf(z2[a][b2], 0.f), w3s[4 * tj + b2], po[a]);
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) po[a] += __shfl_xor_sync(0xffffffffu, po[a], o, 16);
  }
  const float inv_batch = 1.0f / float(TRAIN_BLOCKS * SAMPLES_PER_BLOCK);
  float sse = 0.f;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int s = 4 * ts + a;
    const float err = po[a] + b3s[0] - tgt[s];
    const float dz = 2.0f * err * inv_batch;
    if (tj == 0) {
      dout[s] = dz;
      sse = fmaf(err, err, sse);
    }
#pragma unroll
    for (int b2 = 0; b2 < 4; ++b2)
      D2[s * LD + 4 * tj + b2] = z2[a][b2] > 0.f ? dz * w3s[4 * tj + b2] : 0.f;
  }
  // g(w3) partials: sum over this thread's samples
  float gw3[4];
#pragma unroll
  for (int b2 = 0; b2 < 4; ++b2) {
    gw3[b2] = 0.f;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const float dzs = 2.0f * (po[a] + b3s[0] - tgt[4 * ts + a]) * inv_batch;
      gw3[b2] = fmaf(dzs, fmaxf(z2[a][b2], 0.f), gw3[b2]);
    }
  }
  __syncthreads();
  float* gout = grad_part + size_t(blockIdx.x) * NPARAM;
  // g(w3)[j] = sum over ts of the partials (fixed order through shared memory)
#pragma unroll
  for (int b2 = 0; b2 < 4; ++b2) {
    red[t] = gw3[b2];
    __syncthreads();
    if (t < 16) {
      float acc = 0.f;
      for (int q = 0; q < 16; ++q) acc += red[q * 16 + t];
      gout[OFF_W3 + 4 * t + b2] = acc;
    }
    __syncthreads();
  }
  // dW2 = dZ2^T H1: tile (units 4 tj, inputs 4 ts); g(b2); g(b3)
  {
    const int tk = ts;
    float acc[4][4] = {};
    for (int s = 0; s < SAMPLES_PER_BLOCK; ++s) {
      float dv[4], hv[4];
#pragma unroll
      for (int b2 = 0; b2 < 4; ++b2) dv[b2] = D2[s * LD + 4 * tj + b2];
#pragma unroll
      for (int c = 0; c < 4; ++c) hv[c] = fmaxf(Z1[s * LD + 4 * tk + c], 0.f);
#pragma unroll
      for (int b2 = 0; b2 < 4; ++b2)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[b2][c] = fmaf(dv[b2], hv[c], acc[b2][c]);
    }
#pragma unroll
    for (int b2 = 0; b2 < 4; ++b2)
#pragma unroll
      for (int c = 0; c < 4; ++c) gout[OFF_W2 + (4 * tj + b2) * H + 4 * tk + c] = acc[b2][c];
    if (t < H) {
      float gb = 0.f;
      for (int s = 0; s < SAMPLES_PER_BLOCK; ++s) gb += D2[s * LD + t];
      gout[OFF_B2 + t] = gb;
    }
    if (t == 0) {
      float gb = 0.f;
      for (int s = 0; s < SAMPLES_PER_BLOCK; ++s) gb += dout[s];
      gout[OFF_B3] = gb;
    }
  }
  // dH1 = dZ2 W2: tile (samples 4 ts, inputs 4 tj); dZ1 = dH1 . [Z1 > 0] in place
  {
    float acc[4][4] = {};
    for (int j = 0; j < H; ++j) {
      float dv[4], wv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) dv[a] = D2[(4 * ts + a) * LD + j];
#pragma unroll
      for (int c = 0; c < 4; ++c) wv[c] = W2s[j * LD + 4 * tj + c];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[a][c] = fmaf(dv[a], wv[c], acc[a][c]);
    }
    __syncthreads();  // every thread is done reading Z1 as H1
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        float* zp = Z1 + (4 * ts + a) * LD + 4 * tj + c;
        *zp = *zp > 0.f ? acc[a][c] : 0.f;
      }
  }
  __syncthreads();
  // dW1 = dZ1^T F, g(b1)
  for (int i = t; i < H * NF; i += GB_THREADS) {
    const int k = i / NF, m = i % NF;
    float acc = 0.f;
    for (int s = 0; s < SAMPLES_PER_BLOCK; ++s) acc = fmaf(Z1[s * LD + k], Fs[s * NF + m], acc);
    gout[OFF_W1 + i] = acc;
  }
  if (t < H) {
    float gb = 0.f;
    for (int s = 0; s < SAMPLES_PER_BLOCK; ++s) gb += Z1[s * LD + t];
    gout[OFF_B1 + t] = gb;
  }
  // the block's squared error (threads tj == 0 hold four samples each)
  red[t] = sse;
  __syncthreads();
  if (t == 0) {
    float acc = 0.f;
    for (int q = 0; q < GB_THREADS; q += 16) acc += red[q];
    loss_part[blockIdx.x] = acc;
  }
}

// Block gradients summed in block order; one Adam step (Kingma & Ba) on the
// FP32 master weights, BF16 copy refreshed.  Every block reads the step
// count; the last block to finish (a ticket, no waiting) records the loss
// and advances the count.
constexpr int ADAM_THREADS = 256;
constexpr int ADAM_BLOCKS = (NPARAM + ADAM_THREADS - 1) / ADAM_THREADS;

__global__ void __launch_bounds__(ADAM_THREADS)
k_mlp_adam(const float* __restrict__ grad_part, const float* __restrict__ loss_part,
           float* master, __nv_bfloat16* w16, float* m, float* v, MlpState* M, float lr) {
  __shared__ unsigned int s_last;
  const int step = M->train_steps + 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.0f - powf(b1, float(step)), c2 = 1.0f - powf(b2, float(step));
  const int i = blockIdx.x * ADAM_THREADS + threadIdx.x;
  if (i < NPARAM) {
    float gsum = 0.0f;
    for (int b = 0; b < TRAIN_BLOCKS; ++b) gsum += grad_part[size_t(b) * NPARAM + i];
    const float mi = b1 * m[i] + (1.0f - b1) * gsum;
    const float vi = b2 * v[i] + (1.0f - b2) * gsum * gsum;
    m[i] = mi;
    v[i] = vi;
    const float w = master[i] - lr * (mi / c1) / (sqrtf(vi / c2) + 1e-8f);
    master[i] = w;
    w16[i] = __float2bfloat16(w);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    s_last = (atomicAdd(&M->adam_ticket, 1u) == gridDim.x - 1) ? 1u : 0u;
  }
  __syncthreads();
  if (s_last && threadIdx.x == 0) {
    float s = 0.0f;
    for (int b = 0; b < TRAIN_BLOCKS; ++b) s += loss_part[b];
    M->loss = s * (1.0f / float(TRAIN_BLOCKS * SAMPLES_PER_BLOCK));
    M->train_steps = step;
    M->adam_ticket = 0u;
  }
}

}  // namespace

bool mlp_active(const Ctx& c, bool initial) {
  return !initial && c.opt.warm_start && c.mlp_mode != 0 && c.mlp.master != nullptr;
}

cudaError_t mlp_alloc(Ctx& c) {
  if (c.mlp.master) return cudaSuccess;
  MlpBuf& b = c.mlp;
  const size_t ng = c.format == PIRMCUT_FORMAT_DIA ? size_t(c.K) * c.nt : size_t(c.hg.nnz);
  cudaError_t e = cudaSuccess;
  auto A = [&](void** p, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(p, bytes ? bytes : 16);
  };
  A((void**)&b.master, sizeof(float) * NPARAM);
  A((void**)&b.w16, sizeof(__nv_bfloat16) * NPARAM);
  A((void**)&b.m, sizeof(float) * NPARAM);
  A((void**)&b.v, sizeof(float) * NPARAM);
  A((void**)&b.grad_part, sizeof(float) * NPARAM * TRAIN_BLOCKS);
  A((void**)&b.loss_part, sizeof(float) * TRAIN_BLOCKS);
  A((void**)&b.feat, sizeof(float) * NF * size_t(c.nt));
  A((void**)&b.dir, sizeof(double) * size_t(c.nt));
  A((void**)&b.xprev, sizeof(double) * size_t(c.nt));
  A((void**)&b.gprev, sizeof(double) * ng);
  A((void**)&b.state, sizeof(MlpState));
  if (e == cudaSuccess) e = cudaMemsetAsync(b.state, 0, sizeof(MlpState), c.stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(b.feat, 0, sizeof(float) * NF * size_t(c.nt), c.stream);
  // the gradient kernel's tiles take more than the default 48 KB of shared memory
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, int(GRAD_SMEM));
  if (e != cudaSuccess) mlp_free(c);
  return e;
}

void mlp_free(Ctx& c) {
  MlpBuf& b = c.mlp;
  void* ps[] = {b.master, b.w16, b.m, b.v, b.grad_part, b.loss_part, b.feat, b.dir,
                b.xprev, b.gprev, b.state};
  for (void* p : ps)
    if (p) cudaFree(p);
  b = MlpBuf();
}

cudaError_t mlp_init(Ctx& c, uint64_t seed) {
  c.mlp.seed = seed;
  k_mlp_init<<<(NPARAM + 255) / 256, 256, 0, c.stream>>>(c.mlp.master, c.mlp.w16, c.mlp.m,
                                                         c.mlp.v, seed);
  c.launches += 1;
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemsetAsync(c.mlp.state, 0, sizeof(MlpState), c.stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
  return e;
}

cudaError_t mlp_get_weights(Ctx& c, float* host) {
  cudaError_t e = cudaMemcpyAsync(host, c.mlp.master, sizeof(float) * NPARAM,
                                  cudaMemcpyDeviceToHost, c.stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
  return e;
}

cudaError_t mlp_set_weights(Ctx& c, const float* host) {
  cudaError_t e = cudaMemcpyAsync(c.mlp.master, host, sizeof(float) * NPARAM,
                                  cudaMemcpyHostToDevice, c.stream);
  if (e == cudaSuccess) {
    k_mlp_refresh<<<(NPARAM + 255) / 256, 256, 0, c.stream>>>(c.mlp.master, c.mlp.w16, c.mlp.m,
                                                              c.mlp.v, c.mlp.state);
    c.launches += 1;
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
  return e;
}

cudaError_t mlp_get_state(Ctx& c, MlpState* host) {
  cudaError_t e = cudaMemcpyAsync(host, c.mlp.state, sizeof(MlpState), cudaMemcpyDeviceToHost, c.stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
  return e;
}

cudaError_t mlp_get_features(Ctx& c, float* host) {
  cudaError_t e = cudaMemcpyAsync(host, c.mlp.feat, sizeof(float) * NF * size_t(c.nt),
                                  cudaMemcpyDeviceToHost, c.stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
  return e;
}

// Before the reweighting of a step: keep x^(l-1) and g^(l-1).
int enqueue_mlp_pre(Ctx& c, cudaStream_t st) {
  const size_t ng = c.format == PIRMCUT_FORMAT_DIA ? size_t(c.K) * c.nt : size_t(c.hg.nnz);
  cudaMemcpyAsync(c.mlp.xprev, c.x, sizeof(double) * size_t(c.nt), cudaMemcpyDeviceToDevice, st);
  if (ng)
    cudaMemcpyAsync(c.mlp.gprev, c.format == PIRMCUT_FORMAT_DIA ? c.gdia : c.gval,
                    sizeof(double) * ng, cudaMemcpyDeviceToDevice, st);
  return 0;
}

// After the reweighting: features; with prediction on, the learned
// direction, the line search along it and the move x += alpha d.
// Returns the kernels enqueued.
int enqueue_mlp_post(Ctx& c, cudaStream_t st) {
  MlpBuf& b = c.mlp;
  const int grid = grid_for(c.nt);
  const int form = c.opt.reweight_form;
  const bool predict = (c.mlp_mode & PIRMCUT_MLP_PREDICT) != 0;
  if (c.format == PIRMCUT_FORMAT_DIA) {
    PIRMCUT_DISPATCH_K(c.K, (k_features_dia32<KK><<<grid, kThreads, 0, st>>>(
                                c.dd, c.gdia, b.gprev, c.cs, c.ct, c.x, c.eps_list, c.C, form,
                                b.feat)));
  } else {
    k_features_csr<<<grid + c.n_heavy, kThreads, 0, st>>>(c.nt, c.rp, c.col, c.gval, b.gprev, c.cs,
                                                          c.ct, c.x, c.eps_list, c.C, form, b.feat,
                                                          c.heavy_deg, c.heavy, grid);
  }
  if (!predict) return 1;
  k_mlp_predict_t5<false><<<mlp_t5_grid(c.nt), 128, kT5Pad, st>>>(c.nt, b.feat, b.w16, b.dir,
                                                                   nullptr, b.state);
  return 2;
}

// The learned start of the mixed path, after its assembly: the FP64 line
// search on the assembled system and x += alpha d (the refinement loop then
// forms the residual at the moved start).
int enqueue_mlp_start_mixed(Ctx& c, cudaStream_t st) {
  if (!(c.mlp_mode & PIRMCUT_MLP_PREDICT)) return 0;
  MlpBuf& b = c.mlp;
  const int grid = grid_for(c.nt);
  if (c.format == PIRMCUT_FORMAT_DIA) {
    PIRMCUT_DISPATCH_K(c.K, (k_linesearch_dia<KK><<<grid, kThreads, 0, st>>>(
                                c.dd, c.gdia, c.diag, c.b64, c.x, b.dir, c.partials, b.state)));
  } else {
    k_linesearch_csr<<<grid + c.n_heavy, kThreads, 0, st>>>(c.nt, c.rp, c.col, c.gval, c.diag,
                                                            c.b64, c.x, b.dir, c.partials, b.state,
                                                            c.heavy_deg, c.heavy, grid);
  }
  k_mlp_commit<<<grid, kThreads, 0, st>>>(c.nt, b.state, b.dir, c.x);
  return 2;
}

// After the solve of a step, with training on: iters_per_step Adam steps on
// minibatches of (features, x^(l) - x^(l-1)).
int enqueue_mlp_train(Ctx& c, cudaStream_t st) {
  if (!(c.mlp_mode & PIRMCUT_MLP_TRAIN)) return 0;
  MlpBuf& b = c.mlp;
  for (int it = 0; it < b.iters_per_step; ++it) {
    k_mlp_grad<<<TRAIN_BLOCKS, GB_THREADS, GRAD_SMEM, st>>>(
        c.nt, b.feat, c.x, b.xprev, b.w16, b.state, b.seed, b.grad_part, b.loss_part);
    k_mlp_adam<<<ADAM_BLOCKS, ADAM_THREADS, 0, st>>>(b.grad_part, b.loss_part, b.master, b.w16,
                                                     b.m, b.v, b.state, b.lr);
  }
  return 2 * b.iters_per_step;
}

// reps launches of the inference kernel back to back between CUDA events on
// the context's stream; mean milliseconds per launch.
cudaError_t mlp_time_predict(Ctx& c, const float* feat, int64_t count, float* delta, int reps,
                             double* avg_ms) {
  cudaEvent_t e0, e1;
  cudaError_t e = cudaEventCreate(&e0);
  if (e != cudaSuccess) return e;
  if ((e = cudaEventCreate(&e1)) != cudaSuccess) {
    cudaEventDestroy(e0);
    return e;
  }
  k_mlp_predict_t5<true><<<mlp_t5_grid(count), 128, kT5Pad, c.stream>>>(count, feat, c.mlp.w16,
                                                                         nullptr, delta, c.mlp.state);
  e = cudaEventRecord(e0, c.stream);
  for (int k = 0; k < reps && e == cudaSuccess; ++k) {
    k_mlp_predict_t5<true><<<mlp_t5_grid(count), 128, kT5Pad, c.stream>>>(
        count, feat, c.mlp.w16, nullptr, delta, c.mlp.state);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1, c.stream);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  *avg_ms = reps > 0 ? double(ms) / reps : 0.0;
  c.launches += reps + 1;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return e;
}

// Inference on caller-supplied features (count x kMlpFeatures, device) -> delta (device).
cudaError_t mlp_predict_delta(Ctx& c, const float* feat, int64_t count, float* delta) {
  k_mlp_predict_t5<true><<<mlp_t5_grid(count), 128, kT5Pad, c.stream>>>(count, feat, c.mlp.w16, nullptr,
                                                                     delta, c.mlp.state);
  c.launches += 1;
  return cudaGetLastError();
}

}  // namespace pirmcut
