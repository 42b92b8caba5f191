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
// Training runs on the trajectory the solver itself produces: after a step,
// minibatches of nodes drawn by a counter-based hash go through hand-written
// forward/backward kernels; each block accumulates its samples' gradients in
// a fixed order, blocks are summed in block order, and one Adam step updates
// the FP32 master weights and their BF16 copy.  Runs are bit-reproducible.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>

#include "ctx.h"

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
constexpr int TRAIN_THREADS = 128;
constexpr int TRAIN_BLOCKS = 32;
constexpr int SAMPLES_PER_BLOCK = 64;
constexpr size_t TRAIN_SMEM = sizeof(float) * (2 * NPARAM + NF + 4 * H + 2);

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

template <int K>
__global__ void __launch_bounds__(kThreads)
k_features_dia(DiaDesc d, const double* __restrict__ g, const double* __restrict__ gprev,
               const double* __restrict__ cs, const double* __restrict__ ct,
               const double* __restrict__ x, const double* __restrict__ eps_list,
               const StepCounters* __restrict__ C, int form, float* __restrict__ f) {
  const int64_t nt = d.nt;
  const double eps = eps_list[C->eps_idx];
  const double eps2 = eps * eps;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < nt;
       i += int64_t(gridDim.x) * blockDim.x) {
    const double xi = x[i];
    double wsum = 0.0, wx = 0.0, wxx = 0.0;
    float lr = 0.0f;
    int nlr = 0;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int64_t o = d.off[k];
      if (i + o < nt) edge_feature(g[k * nt + i], gprev[k * nt + i], x[i + o], wsum, wx, wxx, lr, nlr);
      if (i >= o) edge_feature(g[k * nt + i - o], gprev[k * nt + i - o], x[i - o], wsum, wx, wxx, lr, nlr);
    }
    const double gs = conductance(cs[i], 1.0 - xi, eps2, form);
    const double gt = conductance(ct[i], xi, eps2, form);
    finish_features(f, i, xi, wsum, wx, wxx, lr, nlr, gs, gt, eps);
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

// delta = MLP(f), one node per thread.  The BF16 weights are
// widened to FP32 in shared memory with W2 transposed, so that the 64 layer-2
// accumulators of a thread take one hidden unit k at a time from consecutive
// (vectorisable, broadcast) shared-memory words; FP32 accumulation.
// delta -> dir (FP64, the search direction) or out32 (FP32, inference API)
template <bool kF32>
__global__ void __launch_bounds__(kThreads)
k_mlp_predict(int64_t nt, const float* __restrict__ f, const __nv_bfloat16* __restrict__ w16,
              double* __restrict__ dir, float* __restrict__ out32) {
  extern __shared__ __align__(16) float sw[];
  for (int i = threadIdx.x; i < NPARAM; i += blockDim.x) {
    int dst = i;
    if (i >= OFF_W2 && i < OFF_B2) {
      const int j = (i - OFF_W2) / H, k = (i - OFF_W2) % H;
      dst = OFF_W2 + k * H + j;
    }
    sw[dst] = __bfloat162float(w16[i]);
  }
  __syncthreads();
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < nt;
       i += int64_t(gridDim.x) * blockDim.x) {
    float in[NF];
#pragma unroll
    for (int k = 0; k < NF; ++k) in[k] = f[i * NF + k];
    float z[H];
#pragma unroll
    for (int j = 0; j < H; ++j) z[j] = sw[OFF_B2 + j];
#pragma unroll 1
    for (int k = 0; k < H; ++k) {
      float h = sw[OFF_B1 + k];
#pragma unroll
      for (int m = 0; m < NF; ++m) h = fmaf(sw[OFF_W1 + k * NF + m], in[m], h);
      h = fmaxf(h, 0.0f);
      const float* w2t = sw + OFF_W2 + k * H;
#pragma unroll
      for (int j = 0; j < H; ++j) z[j] = fmaf(w2t[j], h, z[j]);
    }
    float out = sw[OFF_B3];
#pragma unroll
    for (int j = 0; j < H; ++j) out = fmaf(sw[OFF_W3 + j], fmaxf(z[j], 0.0f), out);
    if (kF32) out32[i] = out;
    else dir[i] = double(out);
  }
}

// Line search along the learned direction d from x = x^(l-1): with
// r = b - L~ x, the last block forms alpha = (d, r) / (d, L~ d) (0 when the
// denominator is not positive and finite) and the energy change
// -(d, r)^2 / (d, L~ d).
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
k_linesearch_dia(DiaDesc d, const double* __restrict__ g, const double* __restrict__ cs,
                 const double* __restrict__ ct, const double* __restrict__ x,
                 const double* __restrict__ dir, const double* __restrict__ eps_list,
                 const StepCounters* __restrict__ C, int form, double* partials, MlpState* M) {
  const int64_t nt = d.nt;
  const double eps = eps_list[C->eps_idx];
  const double eps2 = eps * eps;
  double dr = 0.0, dad = 0.0, rr = 0.0;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < nt;
       i += int64_t(gridDim.x) * blockDim.x) {
    const double xi = x[i], di = dir[i];
    const double gs = conductance(cs[i], 1.0 - xi, eps2, form);
    const double gt = conductance(ct[i], xi, eps2, form);
    double sum = gs + gt, ax = 0.0, ad = 0.0;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int64_t o = d.off[k];
      if (i + o < nt) {
        const double w = g[k * nt + i];
        sum += w;
        ax = fma(w, x[i + o], ax);
        ad = fma(w, dir[i + o], ad);
      }
      if (i >= o) {
        const double w = g[k * nt + i - o];
        sum += w;
        ax = fma(w, x[i - o], ax);
        ad = fma(w, dir[i - o], ad);
      }
    }
    const double r = gs - fma(sum, xi, -ax);
    dr = fma(di, r, dr);
    dad = fma(di, fma(sum, di, -ad), dad);
    rr = fma(r, r, rr);
  }
  linesearch_finish(dr, dad, rr, partials, M);
}

__global__ void __launch_bounds__(kThreads)
k_linesearch_csr(int64_t nt, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                 const double* __restrict__ g, const double* __restrict__ cs,
                 const double* __restrict__ ct, const double* __restrict__ x,
                 const double* __restrict__ dir, const double* __restrict__ eps_list,
                 const StepCounters* __restrict__ C, int form, double* partials, MlpState* M,
                 int64_t heavy_deg, const int32_t* __restrict__ heavy, int light_blocks) {
  const double eps = eps_list[C->eps_idx];
  const double eps2 = eps * eps;
  double dr = 0.0, dad = 0.0, rr = 0.0;
  if (int(blockIdx.x) >= light_blocks) {  // one heavy row (a hub) for the whole block
    const int64_t i = heavy[blockIdx.x - light_blocks];
    double v[3] = {0.0, 0.0, 0.0};  // sum of g, (g, x), (g, d) over the row
    for (int64_t e = rp[i] + threadIdx.x; e < rp[i + 1]; e += blockDim.x) {
      const double w = g[e];
      v[0] += w;
      v[1] = fma(w, x[col[e]], v[1]);
      v[2] = fma(w, dir[col[e]], v[2]);
    }
    block_sum<3>(v);
    if (threadIdx.x == 0) {
      const double xi = x[i], di = dir[i];
      const double gs = conductance(cs[i], 1.0 - xi, eps2, form);
      const double gt = conductance(ct[i], xi, eps2, form);
      const double sum = v[0] + (gs + gt);
      const double r = gs - fma(sum, xi, -v[1]);
      dr = di * r;
      dad = di * fma(sum, di, -v[2]);
      rr = r * r;
    }
    linesearch_finish(dr, dad, rr, partials, M);
    return;
  }
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < nt;
       i += int64_t(light_blocks) * blockDim.x) {
    if (rp[i + 1] - rp[i] > heavy_deg) continue;
    const double xi = x[i], di = dir[i];
    const double gs = conductance(cs[i], 1.0 - xi, eps2, form);
    const double gt = conductance(ct[i], xi, eps2, form);
    double sum = gs + gt, ax = 0.0, ad = 0.0;
    for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
      const double w = g[e];
      sum += w;
      ax = fma(w, x[col[e]], ax);
      ad = fma(w, dir[col[e]], ad);
    }
    const double r = gs - fma(sum, xi, -ax);
    dr = fma(di, r, dr);
    dad = fma(di, fma(sum, di, -ad), dad);
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

// One minibatch: each block takes SAMPLES_PER_BLOCK sampled nodes in turn
// and accumulates their gradients in shared memory (every parameter has one
// owning thread); the block's sums go to grad_part[block].
__global__ void __launch_bounds__(TRAIN_THREADS)
k_mlp_grad(int64_t nt, const float* __restrict__ f, const double* __restrict__ x,
           const double* __restrict__ xprev, const __nv_bfloat16* __restrict__ w16,
           const MlpState* __restrict__ M, uint64_t seed, float* __restrict__ grad_part,
           float* __restrict__ loss_part) {
  extern __shared__ float sm[];
  float* sw = sm;             // NPARAM weights
  float* sg = sw + NPARAM;    // NPARAM gradient sums
  float* in = sg + NPARAM;    // NF
  float* z1 = in + NF;        // H pre-activations, layer 1
  float* z2 = z1 + H;         // H pre-activations, layer 2
  float* dz2 = z2 + H;        // H
  float* dz1 = dz2 + H;       // H
  float* red = dz1 + H;       // [output error]
  const int t = threadIdx.x;
  for (int i = t; i < NPARAM; i += blockDim.x) {
    sw[i] = __bfloat162float(w16[i]);
    sg[i] = 0.0f;
  }
  const uint64_t stream = splitmix64(seed ^ (uint64_t(M->train_steps) << 20));
  const float inv_batch = 1.0f / float(TRAIN_BLOCKS * SAMPLES_PER_BLOCK);
  float sse = 0.0f;
  __syncthreads();
  for (int smp = 0; smp < SAMPLES_PER_BLOCK; ++smp) {
    const uint64_t h = splitmix64(stream + uint64_t(blockIdx.x) * SAMPLES_PER_BLOCK + uint64_t(smp));
    const int64_t node = int64_t(h % uint64_t(nt));
    if (t < NF) in[t] = f[node * NF + t];
    __syncthreads();
    if (t < H) {
      float z = sw[OFF_B1 + t];
#pragma unroll
      for (int k = 0; k < NF; ++k) z = fmaf(sw[OFF_W1 + t * NF + k], in[k], z);
      z1[t] = z;
    }
    __syncthreads();
    if (t < H) {
      float z = sw[OFF_B2 + t];
      for (int k = 0; k < H; ++k) z = fmaf(sw[OFF_W2 + t * H + k], fmaxf(z1[k], 0.0f), z);
      z2[t] = z;
    }
    __syncthreads();
    if (t == 0) {
      float out = sw[OFF_B3];
      for (int j = 0; j < H; ++j) out = fmaf(sw[OFF_W3 + j], fmaxf(z2[j], 0.0f), out);
      const float err = out - float(x[node] - xprev[node]);
      red[0] = err;
      sse = fmaf(err, err, sse);
    }
    __syncthreads();
    const float dout = 2.0f * red[0] * inv_batch;  // d(mean squared error)/d(out)
    if (t < H) {
      sg[OFF_W3 + t] += dout * fmaxf(z2[t], 0.0f);
      dz2[t] = z2[t] > 0.0f ? dout * sw[OFF_W3 + t] : 0.0f;
    }
    if (t == 0) sg[OFF_B3] += dout;
    __syncthreads();
    if (t < H) {
      float a = 0.0f;
      for (int k = 0; k < H; ++k) a = fmaf(sw[OFF_W2 + k * H + t], dz2[k], a);
      dz1[t] = z1[t] > 0.0f ? a : 0.0f;
      sg[OFF_B2 + t] += dz2[t];
    }
    __syncthreads();
    for (int idx = t; idx < H * H; idx += TRAIN_THREADS)
      sg[OFF_W2 + idx] += dz2[idx / H] * fmaxf(z1[idx % H], 0.0f);
    for (int idx = t; idx < H * NF; idx += TRAIN_THREADS)
      sg[OFF_W1 + idx] += dz1[idx / NF] * in[idx % NF];
    if (t < H) sg[OFF_B1 + t] += dz1[t];
    __syncthreads();
  }
  for (int i = t; i < NPARAM; i += blockDim.x) grad_part[size_t(blockIdx.x) * NPARAM + i] = sg[i];
  if (t == 0) loss_part[blockIdx.x] = sse;
}

// Block gradients summed in block order; one Adam step (Kingma & Ba) on the
// FP32 master weights, BF16 copy refreshed.  One block, so the step counter
// is read before and written after every update.
__global__ void __launch_bounds__(1024)
k_mlp_adam(const float* __restrict__ grad_part, const float* __restrict__ loss_part,
           float* master, __nv_bfloat16* w16, float* m, float* v, MlpState* M, float lr) {
  const int step = M->train_steps + 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.0f - powf(b1, float(step)), c2 = 1.0f - powf(b2, float(step));
  for (int i = threadIdx.x; i < NPARAM; i += blockDim.x) {
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
    float s = 0.0f;
    for (int b = 0; b < TRAIN_BLOCKS; ++b) s += loss_part[b];
    M->loss = s * (1.0f / float(TRAIN_BLOCKS * SAMPLES_PER_BLOCK));
    M->train_steps = step;
  }
}

}  // namespace

bool mlp_active(const Ctx& c, bool initial) {
  return !initial && c.opt.warm_start && c.mlp_mode != 0 && c.mlp.master != nullptr;
}

const double* reweight_point(const Ctx& c, bool initial) {
  return mlp_active(c, initial) ? c.mlp.xprev : c.x;
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
  if (c.format == PIRMCUT_FORMAT_DIA) {
    PIRMCUT_DISPATCH_K(c.K, (k_features_dia<KK><<<grid, kThreads, 0, st>>>(
                                c.dd, c.gdia, b.gprev, c.cs, c.ct, c.x, c.eps_list, c.C, form, b.feat)));
  } else {
    k_features_csr<<<grid + c.n_heavy, kThreads, 0, st>>>(c.nt, c.rp, c.col, c.gval, b.gprev, c.cs,
                                                          c.ct, c.x, c.eps_list, c.C, form, b.feat,
                                                          c.heavy_deg, c.heavy, grid);
  }
  if (!(c.mlp_mode & PIRMCUT_MLP_PREDICT)) return 1;
  k_mlp_predict<false><<<grid, kThreads, sizeof(float) * NPARAM, st>>>(c.nt, b.feat, b.w16, b.dir,
                                                                       nullptr);
  if (c.format == PIRMCUT_FORMAT_DIA) {
    PIRMCUT_DISPATCH_K(c.K, (k_linesearch_dia<KK><<<grid, kThreads, 0, st>>>(
                                c.dd, c.gdia, c.cs, c.ct, c.x, b.dir, c.eps_list, c.C, form,
                                c.partials, b.state)));
  } else {
    k_linesearch_csr<<<grid + c.n_heavy, kThreads, 0, st>>>(c.nt, c.rp, c.col, c.gval, c.cs, c.ct,
                                                            c.x, b.dir, c.eps_list, c.C, form,
                                                            c.partials, b.state, c.heavy_deg,
                                                            c.heavy, grid);
  }
  k_mlp_commit<<<grid, kThreads, 0, st>>>(c.nt, b.state, b.dir, c.x);
  return 4;
}

// After the solve of a step, with training on: iters_per_step Adam steps on
// minibatches of (features, x^(l) - x^(l-1)).
int enqueue_mlp_train(Ctx& c, cudaStream_t st) {
  if (!(c.mlp_mode & PIRMCUT_MLP_TRAIN)) return 0;
  MlpBuf& b = c.mlp;
  for (int it = 0; it < b.iters_per_step; ++it) {
    k_mlp_grad<<<TRAIN_BLOCKS, TRAIN_THREADS, TRAIN_SMEM, st>>>(
        c.nt, b.feat, c.x, b.xprev, b.w16, b.state, b.seed, b.grad_part, b.loss_part);
    k_mlp_adam<<<1, 1024, 0, st>>>(b.grad_part, b.loss_part, b.master, b.w16, b.m, b.v, b.state,
                                    b.lr);
  }
  return 2 * b.iters_per_step;
}

// Inference on caller-supplied features (count x kMlpFeatures, device) -> delta (device).
cudaError_t mlp_predict_delta(Ctx& c, const float* feat, int64_t count, float* delta) {
  k_mlp_predict<true><<<grid_for(count), kThreads, sizeof(float) * NPARAM, c.stream>>>(
      count, feat, c.mlp.w16, nullptr, delta);
  c.launches += 1;
  return cudaGetLastError();
}

}  // namespace pirmcut
