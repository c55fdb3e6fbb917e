// Coarse-level block operator on the 5th-generation tensor cores (tcgen05, sm_100 family).
//
// For a coarse box B the block step is a dense product D (b x M) = A_B (b x Wp) X_win (Wp x M):
// the box's b rows (dense b x b blocks over its neighbour slots, stored row by row) times the
// window of the M-column block vector.  One CTA (4 warps) per box at a time:
//   * the K dimension (window positions) is cut into chunks of kTcK = 64; for each chunk the
//     threads load the box rows and the gathered window rows of X, split every FP32 value into a
//     TF32 head (low 13 mantissa bits cleared) and the TF32 head of the exact remainder (the
//     3 x TF32 scheme keeps near-FP32 accuracy), and store the four operand tiles in shared
//     memory in the tensor cores' canonical K-major layout (8-row x 16-byte core matrices,
//     no swizzle);
//   * one thread issues, per 8-wide K step, the three products head*head, head*tail, tail*head
//     (tcgen05.mma kind::tf32, M = 128, N = M columns) into a TMEM accumulator, then commits
//     them to the chunk's mbarrier; the threads meanwhile fill the other stage;
//   * after the last chunk, warp 0 reads rows 0..31 of the accumulator (tcgen05.ld, one row per
//     lane) and applies the epilogue (Chebyshev step or product) to the box's b rows.
// Accumulator rows b..127 come from operand rows the tile does not hold (whatever the shared
// memory after the tile contains, always inside the CTA's allocation); a row of D depends only
// on its own row of A, so they are never read.  Every mbarrier wait is bounded; on expiry the
// kernel raises *err, waits (bounded) for its issued products and frees its TMEM.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "kernels_mrhs.cuh"

namespace r3mg {

constexpr int kTcK = 64;                         // K elements per chunk
constexpr int kTcRows = 32;                      // operand rows held for A (b <= 32)
constexpr int kTcChunks16 = kTcK / 4;            // 16-byte core-matrix columns per chunk
constexpr uint32_t kTcCoreBytes = 128;           // 8 rows x 16 bytes
constexpr uint32_t kTcSBO_A = kTcChunks16 * kTcCoreBytes;   // between 8-row groups of a tile
constexpr uint32_t kTcTileA = (kTcRows / 8) * kTcSBO_A;     // 8 KB

template <int M>
struct TcLayout {   // byte offsets of one stage (two stages), tiles 1024-byte aligned
  static constexpr uint32_t kTileB = (M / 8) * kTcSBO_A;
  static constexpr uint32_t kStage = 2 * kTcTileA + 2 * kTileB;
  __host__ __device__ static constexpr uint32_t ahi(int s) { return s * kStage; }
  __host__ __device__ static constexpr uint32_t alo(int s) { return s * kStage + kTcTileA; }
  __host__ __device__ static constexpr uint32_t bhi(int s) { return s * kStage + 2 * kTcTileA; }
  __host__ __device__ static constexpr uint32_t blo(int s) { return s * kStage + 2 * kTcTileA + kTileB; }
  // the M = 128 products read 16 row groups from each A tile: the allocation covers them
  static constexpr uint32_t kTotal = kStage + kTcTileA + 16 * kTcSBO_A;
};

__device__ __forceinline__ uint64_t tc_smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;   // descriptor version of the sm_100 family; base offset 0, no swizzle
  return d;
}

// instruction descriptor of kind::tf32: FP32 accumulator, TF32 A and B, both K-major
__host__ __device__ constexpr uint32_t tc_idesc_tf32(int m, int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t tmem_d, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ uint32_t tf32_head(float x) { return __float_as_uint(x) & 0xffffe000u; }

// one FP32 value -> (TF32 head, TF32 head of the exact remainder)
__device__ __forceinline__ void tc_split(float x, float& hi, float& lo) {
  const float h = __uint_as_float(tf32_head(x));
  hi = h;
  lo = __uint_as_float(tf32_head(x - h));
}

template <int M, class Ep>
__global__ void __launch_bounds__(128) k_mr_coarse_tc(LevelView<float> L, const float* __restrict__ xin, Ep ep,
                                                      int* __restrict__ err, long long wait_limit) {
  static_assert(M == 16, "kind::tf32 with M = 128 takes N in multiples of 16");
  using Lay = TcLayout<M>;
  extern __shared__ __align__(1024) unsigned char tsm_raw[];
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ uint32_t tmem_base;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int b = L.b;
  const uint32_t sbase = smem_u32(tsm_raw);
  if (warp == 0) {   // 32 TMEM columns hold the 128 x M FP32 accumulator
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 32;\n" ::"r"(smem_u32(&tmem_base))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = tmem_base;
  constexpr uint32_t idesc = tc_idesc_tf32(128, M);
  uint32_t commits[2] = {0u, 0u};   // products committed on each stage's barrier (thread 0 issues)
  uint32_t waited[2] = {0u, 0u};    // completions observed on each stage's barrier
  bool alive = true;
  for (int64_t B = blockIdx.x; B < L.nbox && alive; B += gridDim.x) {
    const int64_t e0 = L.nbr_ptr[B];
    const int nn = (int)(L.nbr_ptr[B + 1] - e0);
    const int W = nn * b, Wp = (W + 3) & ~3;
    const int64_t kbase = L.row_ptr[B * b];   // the box's rows: equal length Wp, consecutive
    const int nchunk = (Wp + kTcK - 1) / kTcK;
    for (int c = 0; c < nchunk; ++c) {
      const int s = c & 1;
      // the stage is free once the products issued from it two chunks ago have completed
      if (commits[s] > waited[s]) {
        const bool ok = mbar_wait_bounded(&bar[s], (waited[s] & 1u), err, wait_limit);
        if (__syncthreads_or(!ok)) { alive = false; break; }
        ++waited[s];
      }
      const int k0 = c * kTcK;
      // A: b rows x 16 columns of 16 bytes; eight consecutive threads take eight rows of one
      // column (distinct bank groups), four of them cover 64 contiguous bytes of each row
      for (int it = tid; it < ((b + 7) >> 3) * 128; it += blockDim.x) {
        const int q = (it >> 7) * 8 + (it & 7), kc = (it >> 3) & 15;
        if (q >= b) continue;
        const int k = k0 + 4 * kc;
        float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
        if (k < Wp) a = __ldcs(reinterpret_cast<const float4*>(L.vals + kbase + (int64_t)q * Wp + k));
        float4 h, l;
        tc_split(a.x, h.x, l.x); tc_split(a.y, h.y, l.y); tc_split(a.z, h.z, l.z); tc_split(a.w, h.w, l.w);
        const uint32_t off = (uint32_t)((q >> 3) * kTcSBO_A + kc * kTcCoreBytes + (q & 7) * 16);
        *reinterpret_cast<float4*>(tsm_raw + Lay::ahi(s) + off) = h;
        *reinterpret_cast<float4*>(tsm_raw + Lay::alo(s) + off) = l;
      }
      // B = X_win^T: M rows (columns of X) x 64 window positions; window position w is level
      // row nbr[e0 + w / b] * b + w % b.  Sixteen consecutive threads read one gathered row of X.
      for (int it = tid; it < kTcK * M; it += blockDim.x) {
        const int n = it % M, kk = it / M;
        const int w = k0 + kk;
        float xv = 0.f;
        if (w < W) xv = __ldg(xin + (L.nbr[e0 + w / b] * b + w % b) * M + n);
        float h, l;
        tc_split(xv, h, l);
        const uint32_t off = (uint32_t)((n >> 3) * kTcSBO_A + (kk >> 2) * kTcCoreBytes + (n & 7) * 16 + (kk & 3) * 4);
        *reinterpret_cast<float*>(tsm_raw + Lay::bhi(s) + off) = h;
        *reinterpret_cast<float*>(tsm_raw + Lay::blo(s) + off) = l;
      }
      // the tiles were written by the generic proxy; the tensor cores read them by the async proxy
      asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
      __syncthreads();
      if (tid == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
#pragma unroll
        for (int ks = 0; ks < kTcK / 8; ++ks) {   // 8-wide K steps: two core-matrix columns
          const uint32_t ko = ks * 2 * kTcCoreBytes;
          const uint64_t ah = tc_smem_desc(sbase + Lay::ahi(s) + ko, kTcCoreBytes, kTcSBO_A);
          const uint64_t al = tc_smem_desc(sbase + Lay::alo(s) + ko, kTcCoreBytes, kTcSBO_A);
          const uint64_t bh = tc_smem_desc(sbase + Lay::bhi(s) + ko, kTcCoreBytes, kTcSBO_A);
          const uint64_t bl = tc_smem_desc(sbase + Lay::blo(s) + ko, kTcCoreBytes, kTcSBO_A);
          const uint32_t acc0 = (c > 0 || ks > 0) ? 1u : 0u;
          tc_mma(tmem, al, bh, idesc, acc0);   // small terms first
          tc_mma(tmem, ah, bl, idesc, 1u);
          tc_mma(tmem, ah, bh, idesc, 1u);
        }
        tc_commit(&bar[s]);
      }
      ++commits[s];
    }
    if (!alive) break;
    // every product of the box has completed once both stages' last commits have
    for (int st = 0; st < 2 && alive; ++st) {
      const int s = ((nchunk - 1) & 1) ^ st;
      if (commits[s] > waited[s]) {
        const bool ok = mbar_wait_bounded(&bar[s], (waited[s] & 1u), err, wait_limit);
        if (__syncthreads_or(!ok)) { alive = false; break; }
        ++waited[s];
      }
    }
    if (!alive) break;
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (warp == 0) {
      uint32_t v[16];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
            "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
          : "r"(tmem));
      asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
      if (nchunk == 0)
#pragma unroll
        for (int j = 0; j < 16; ++j) v[j] = 0u;   // an empty window: nothing was accumulated
      if (lane < b) {   // lane i holds row i of the box: its 16 columns as four 16-byte slices
        double unused[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
        for (int c0 = 0; c0 < M; c0 += 4) {
          Slice<float> sl;
#pragma unroll
          for (int j = 0; j < 4; ++j) sl.v[j] = __uint_as_float(v[c0 + j]);
          ep.post(B * b + lane, c0, sl, unused);
        }
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();   // the accumulator is overwritten by the next box's first product
  }
  if (!alive) {
    // leave only after every product this CTA issued has completed (bounded), so TMEM is idle
    if (tid == 0)
      for (int s = 0; s < 2; ++s)
        while (commits[s] > waited[s]) {
          if (!mbar_wait_bounded(&bar[s], (waited[s] & 1u), nullptr, kWaitCycles)) break;
          ++waited[s];
        }
    __syncthreads();
  }
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 32;\n" ::"r"(tmem) : "memory");
}

}  // namespace r3mg
