// The learned warm start's network on GB300's fifth-generation tensor cores
// (tcgen05): 128 rows per tile, one thread per row, accumulators in tensor
// memory (TMEM).
//
//   layer 1  D1[128 x 64] = A1[128 x 16] B1^T: the K slot of a row holds the
//            six features as BF16 heads (K 0-5), a constant 1 that meets b1
//            (K 6), the six BF16 tails f - BF16(f) (K 8-13), zeros; so a
//            feature enters with about 2^-17 relative precision and
//            differences such as f1 - f0 keep their digits;
//   layer 2  D2[128 x 64] = A2[128 x 80] B2^T: ReLU(D1) rounded to BF16
//            (K 0-63), a constant 1 that meets b2 (K 64), zeros; D2 takes the
//            tensor-memory columns of D1, which every thread has read out
//            before the barrier that precedes the MMA;
//   layer 3  out = b3 + sum_j w3[j] ReLU(D2[:, j]) in FP32 on the CUDA cores.
//
// Operands live in shared memory in the K-major layout without swizzling
// that the MMA reads: 8-row x 16-byte core matrices, core matrices adjacent
// along K 128 bytes apart (the leading-byte offset), 8-row groups one K row
// (K x 2 bytes x 8) apart (the stride-byte offset).  One thread of the CTA
// issues the MMAs; completion reaches an mbarrier through tcgen05.commit;
// every wait on it is bounded (on expiry the CTA records an error, stops
// and still frees its tensor memory).
#pragma once

#include <cuda_bf16.h>
#include <cstdint>

namespace pirmcut {
namespace tc5 {

constexpr int kRows = 128;        // rows of a tile: the MMA's M, TMEM lanes
constexpr int kLBO = 128;         // bytes between core matrices along K
constexpr int kSboA1 = 2 * kLBO;  // K = 16: two core matrices per 8-row group
constexpr int kSboA2 = 10 * kLBO; // K = 80
constexpr int kTmemCols = 64;     // D1, then D2 in the same columns (D1 is read out first)
constexpr uint32_t kMaxPolls = 1u << 22;  // bound on the polls of one mbarrier wait

struct __align__(1024) Smem {
  uint8_t a1[kRows * 32];   // [128 rows x K 16] BF16
  uint8_t a2[kRows * 160];  // [128 rows x K 80]
  uint8_t b1[64 * 32];      // [64 units x K 16]
  uint8_t b2[64 * 160];     // [64 units x K 80]
  __align__(16) float w3[64];
  float b3;
  uint32_t tmem_base;
  unsigned long long mbar;
  int timed_out;
};

// byte offset of the 16-byte K chunk kc of a row in a core-matrix tile
__device__ __forceinline__ uint32_t cm_off(int row, int kc, int sbo) {
  return uint32_t((row >> 3) * sbo + kc * kLBO + (row & 7) * 16);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor: start address, leading-byte offset (K
// direction), stride-byte offset (M/N direction), the descriptor version of
// this generation (bits 46-47 = 1), no base offset, no swizzling.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t sbo) {
  return uint64_t((saddr >> 4) & 0x3FFFu) | (uint64_t((kLBO >> 4) & 0x3FFFu) << 16) |
         (uint64_t((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: D FP32 (bits 4-5 = 1), A and B BF16
// (bits 7-9 and 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 in bits
// 17-22, M >> 4 in bits 24-28.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(64 >> 3) << 17) |
                            (uint32_t(kRows >> 4) << 24);

__device__ __forceinline__ void mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
      :
      : "r"(d_tmem), "l"(a), "l"(b), "r"(kIdesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
               :
               : "r"(mbar)
               : "memory");
}

__device__ __forceinline__ bool try_wait(uint32_t mbar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(done)
      : "r"(mbar), "r"(parity)
      : "memory");
  return done != 0;
}

// bounded wait for the phase with the given parity; false on expiry
__device__ __forceinline__ bool wait_phase(uint32_t mbar, uint32_t parity) {
  for (uint32_t k = 0; k < kMaxPolls; ++k)
    if (try_wait(mbar, parity)) return true;
  return false;
}

__device__ __forceinline__ void fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// generic-proxy shared-memory writes made visible to the tensor core
__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// 32 consecutive FP32 columns of this thread's TMEM lane
__device__ __forceinline__ void ld32(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
        "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]),
        "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]),
        "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr)
      : "memory");
}
__device__ __forceinline__ void ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ void st16(uint8_t* base, uint32_t off, uint32_t a, uint32_t b, uint32_t c,
                                     uint32_t d) {
  *reinterpret_cast<uint4*>(base + off) = make_uint4(a, b, c, d);
}

__device__ __forceinline__ uint32_t bf(const __nv_bfloat16* p) {
  return uint32_t(__bfloat16_as_ushort(*p));
}
// two adjacent BF16 values (the first at an even index, so 4-byte aligned)
__device__ __forceinline__ uint32_t bf2(const __nv_bfloat16* p) {
  return __ldg(reinterpret_cast<const unsigned int*>(p));
}

// two FP32 values rounded to BF16 and packed, lo in the low half
__device__ __forceinline__ uint32_t pk(float lo, float hi) {
  uint32_t r;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
  return r;
}
__device__ __forceinline__ uint32_t pk_relu(float lo, float hi) {
  uint32_t r;
  asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
  return r;
}
__device__ __forceinline__ float lo_of(uint32_t v) { return __uint_as_float(v << 16); }
__device__ __forceinline__ float hi_of(uint32_t v) { return __uint_as_float(v & 0xffff0000u); }

// Parameter offsets of the flat weight vector (out x in, row-major):
// W1[64][6] b1[64] W2[64][64] b2[64] w3[64] b3.
constexpr int kW1 = 0, kB1 = 384, kW2 = 448, kB2 = 4544, kW3 = 4608, kB3 = 4672;

// Stage the weights and the constant parts of A2; allocate the tensor
// memory; initialise the mbarrier.  All threads of the CTA (128) take part.
__device__ __forceinline__ void setup(Smem& S, const __nv_bfloat16* __restrict__ w16) {
  const int tid = threadIdx.x;
  for (int idx = tid; idx < 64 * 2; idx += blockDim.x) {  // B1: 64 units x 2 K chunks
    const int n = idx >> 1, kc = idx & 1;
    const __nv_bfloat16* w = w16 + kW1 + n * 6;
    const uint32_t last = kc == 0 ? bf(w16 + kB1 + n) : 0u;  // (b1[n], 0) or (0, 0)
    st16(S.b1, cm_off(n, kc, kSboA1), bf2(w), bf2(w + 2), bf2(w + 4), last);
  }
  for (int idx = tid; idx < 64 * 10; idx += blockDim.x) {  // B2: 64 units x 10 K chunks
    const int n = idx / 10, kc = idx % 10;
    uint4 q = make_uint4(0u, 0u, 0u, 0u);
    if (kc < 8)  // eight weights W2[n][8kc ..]: 16 bytes at a 16-byte boundary
      q = __ldg(reinterpret_cast<const uint4*>(w16 + kW2 + n * 64 + kc * 8));
    else if (kc == 8)
      q.x = bf(w16 + kB2 + n);  // (b2[n], 0)
    st16(S.b2, cm_off(n, kc, kSboA2), q.x, q.y, q.z, q.w);
  }
  for (int idx = tid; idx < kRows * 2; idx += blockDim.x) {  // A2 K chunks 8 (1, 0 ...), 9 (0)
    const int r = idx >> 1, kc = 8 + (idx & 1);
    st16(S.a2, cm_off(r, kc, kSboA2), kc == 8 ? pk(1.0f, 0.0f) : 0u, 0u, 0u, 0u);
  }
  if (tid < 64) S.w3[tid] = __bfloat162float(w16[kW3 + tid]);
  if (tid == 0) {
    S.b3 = __bfloat162float(w16[kB3]);
    S.timed_out = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&S.mbar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (tid < 32) {  // warp 0 owns the tensor memory
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 ::"r"(smem_u32(&S.tmem_base)), "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_async_smem();
  fence_before();
  __syncthreads();
  fence_after();
}

__device__ __forceinline__ void teardown(Smem& S) {
  fence_before();
  __syncthreads();
  fence_after();
  if (threadIdx.x < 32)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;"
                 ::"r"(S.tmem_base), "r"(kTmemCols)
                 : "memory");
}

// One tile: thread r supplies the features f of row r of the tile (any
// values for rows past the end) and gets that row's output.  phase is the
// parity of the mbarrier's next phase (two phases per tile).  Returns false
// on an expired wait (the same in every thread; the CTA must then stop).
__device__ __forceinline__ bool tile(Smem& S, const float (&f)[6], uint32_t& phase, float& out) {
  const int r = threadIdx.x;
  const uint32_t mbar = smem_u32(&S.mbar);
  // A1: heads (f0..f5, 1, 0) and tails (f - BF16(f), 0, 0)
  const uint32_t h0 = pk(f[0], f[1]), h1 = pk(f[2], f[3]), h2 = pk(f[4], f[5]);
  st16(S.a1, cm_off(r, 0, kSboA1), h0, h1, h2, pk(1.0f, 0.0f));
  st16(S.a1, cm_off(r, 1, kSboA1), pk(f[0] - lo_of(h0), f[1] - hi_of(h0)),
       pk(f[2] - lo_of(h1), f[3] - hi_of(h1)), pk(f[4] - lo_of(h2), f[5] - hi_of(h2)), 0u);
  fence_async_smem();
  fence_before();
  __syncthreads();
  const uint32_t tbase = S.tmem_base;
  if (r == 0) {
    fence_after();
    mma(tbase, sdesc(smem_u32(S.a1), kSboA1), sdesc(smem_u32(S.b1), kSboA1), 0u);
    commit(mbar);
  }
  bool ok = wait_phase(mbar, phase);
  if (__syncthreads_or(!ok)) return false;
  phase ^= 1u;
  fence_after();
  // D1 -> ReLU -> BF16 -> A2 (K chunks 0-7); warp w reads TMEM lanes 32w..32w+31
  const uint32_t lane_addr = tbase + (uint32_t(r & ~31) << 16);
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    uint32_t v[32];
    ld32(lane_addr + 32u * h, v);
    ld_wait();
#pragma unroll
    for (int q = 0; q < 4; ++q)
      st16(S.a2, cm_off(r, 4 * h + q, kSboA2),
           pk_relu(__uint_as_float(v[8 * q + 0]), __uint_as_float(v[8 * q + 1])),
           pk_relu(__uint_as_float(v[8 * q + 2]), __uint_as_float(v[8 * q + 3])),
           pk_relu(__uint_as_float(v[8 * q + 4]), __uint_as_float(v[8 * q + 5])),
           pk_relu(__uint_as_float(v[8 * q + 6]), __uint_as_float(v[8 * q + 7])));
  }
  fence_async_smem();
  fence_before();
  __syncthreads();
  if (r == 0) {
    fence_after();
    const uint32_t a2 = smem_u32(S.a2), b2 = smem_u32(S.b2);
#pragma unroll
    for (int j = 0; j < 5; ++j)  // K chunks of 16: 64 hidden units, then b2
      mma(tbase, sdesc(a2 + 256u * j, kSboA2), sdesc(b2 + 256u * j, kSboA2), j > 0 ? 1u : 0u);
    commit(mbar);
  }
  ok = wait_phase(mbar, phase);
  if (__syncthreads_or(!ok)) return false;
  phase ^= 1u;
  fence_after();
  float acc = S.b3;
  const float4* w3 = reinterpret_cast<const float4*>(S.w3);
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    uint32_t v[32];
    ld32(lane_addr + 32u * h, v);
    ld_wait();
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const float4 w = w3[8 * h + j];  // one 16-byte broadcast load for four weights
      acc = fmaf(fmaxf(__uint_as_float(v[4 * j + 0]), 0.f), w.x, acc);
      acc = fmaf(fmaxf(__uint_as_float(v[4 * j + 1]), 0.f), w.y, acc);
      acc = fmaf(fmaxf(__uint_as_float(v[4 * j + 2]), 0.f), w.z, acc);
      acc = fmaf(fmaxf(__uint_as_float(v[4 * j + 3]), 0.f), w.w, acc);
    }
  }
  out = acc;
  return true;
}

}  // namespace tc5
}  // namespace pirmcut
