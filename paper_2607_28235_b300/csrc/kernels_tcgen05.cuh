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

namespace r3mg {

// ---------------------------------------------------------------------------------------------
// Warp-specialised form (block form 6).  The same product D (b x 16) = A_B X_win per box, with
//   * the A operand in TMEM: the M = 128 products read it from tensor memory, not from shared
//     memory, so a product no longer pays a 4 KB shared-memory read for 27 real rows;
//   * both operands fetched by the copy engine, kT2Stages chunks ahead: per chunk of 64 window
//     positions, one cp.async.bulk per box row (its 64 entries) and one per run of consecutive
//     window rows of X (the window is a list of b-row segments of the level), completion on the
//     stage's mbarrier;
//   * one CTA per SM, six warps: warp 1 issues the copies; warp 0 splits the staged A chunk into
//     TF32 head and tail and writes both into a TMEM stage (tcgen05.st, lane q = box row q);
//     warps 2-3 split and transpose the staged X chunk into the K-major head/tail tiles; warp 5
//     (one thread) issues the 3 x 8 products of the chunk and commits them; warp 4 reads the
//     finished accumulator (tcgen05.ld) and applies the epilogue.  Accumulators are double-
//     buffered across boxes, A stages and B tiles across chunks.
// Hand-offs are mbarriers; every wait is bounded and also gives up when another warp has raised
// the CTA's abort flag, so an expiry anywhere stops every warp; before the CTA frees its TMEM and
// exits, the producer waits (bounded) for the copies it issued and the issuer for its products.
constexpr int kT2K = 64;         // window positions per chunk
constexpr int kT2Stages = 6;     // staged chunks in flight
constexpr int kT2Warps = 6;
constexpr uint32_t kT2AStage = (uint32_t)kTcRows * kT2K * 4;     // 8 KB: 32 rows x 64 floats
constexpr uint32_t kT2XStage = (uint32_t)kT2K * 16 * 4;          // 4 KB: 64 window rows x 16 floats
constexpr uint32_t kT2Stage = kT2AStage + kT2XStage;
constexpr uint32_t kT2BTile = 2 * kTcSBO_A;                      // 4 KB: 16 rows (N) x 64 (K)
constexpr uint32_t kT2BOff = kT2Stages * kT2Stage;               // B tiles: [slot][hi, lo]
constexpr uint32_t kT2Smem = kT2BOff + 2 * 2 * kT2BTile;         // 88 KB
// the launch asks for more, so that no two CTAs share an SM (each allocates all 512 TMEM columns)
constexpr uint32_t kT2SmemLaunch = 120 * 1024;
// TMEM columns: accumulators 0..31 (two of 16), A stages from 128 (two of hi 64 + lo 64)
constexpr uint32_t kT2ACol = 128;

struct T2Bars {   // mbarriers and the abort flag (static shared memory)
  uint64_t full[kT2Stages], empty[kT2Stages], ready[2], tfree[2], dfull[2], dempty[2];
  int abort;
  uint32_t tmem;
};

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}

// bounded wait that also gives up when the CTA's abort flag is raised; on expiry it raises both
__device__ __forceinline__ bool t2_wait(uint64_t* bar, uint32_t parity, volatile int* abort, int* err,
                                        long long limit) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (*abort) return false;
    if (clock64() - t0 > limit) {
      *abort = 1;
      if (err) atomicExch(err, 1);
      return false;
    }
  }
  return true;
}

__device__ __forceinline__ void tc_mma_ta(uint32_t tmem_d, uint32_t tmem_a, uint64_t bd, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}\n" ::"r"(tmem_d),
      "r"(tmem_a), "l"(bd), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
      "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};\n" ::"r"(taddr),
      "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]), "r"(v[9]),
      "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15]), "r"(v[16]), "r"(v[17]), "r"(v[18]),
      "r"(v[19]), "r"(v[20]), "r"(v[21]), "r"(v[22]), "r"(v[23]), "r"(v[24]), "r"(v[25]), "r"(v[26]), "r"(v[27]),
      "r"(v[28]), "r"(v[29]), "r"(v[30]), "r"(v[31])
      : "memory");
}

// per-box geometry shared by every role
struct T2Box {
  int64_t e0, kbase;
  int nn, W, Wp, nchunk;
};
__device__ __forceinline__ T2Box t2_box(const LevelView<float>& L, int64_t B) {
  T2Box x;
  x.e0 = L.nbr_ptr[B];
  x.nn = (int)(L.nbr_ptr[B + 1] - x.e0);
  x.W = x.nn * L.b;
  x.Wp = (x.W + 3) & ~3;
  x.kbase = L.row_ptr[B * L.b];
  x.nchunk = (x.Wp + kT2K - 1) / kT2K;
  return x;
}

template <class Ep>
__global__ void __launch_bounds__(kT2Warps * 32, 1) k_mr_coarse_tc2(LevelView<float> L, const float* __restrict__ xin,
                                                                   Ep ep, int* __restrict__ err, long long wait_limit) {
  constexpr int M = 16;
  extern __shared__ __align__(1024) unsigned char t2sm[];
  __shared__ T2Bars S;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int b = L.b;
  const uint32_t sbase = smem_u32(t2sm);
  volatile int* abort = &S.abort;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;\n" ::"r"(smem_u32(&S.tmem))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  if (tid == 0) {
    for (int s = 0; s < kT2Stages; ++s) { mbar_init(&S.full[s], 1); mbar_init(&S.empty[s], 3); }
    for (int t = 0; t < 2; ++t) {
      mbar_init(&S.ready[t], 3); mbar_init(&S.tfree[t], 1); mbar_init(&S.dfull[t], 1); mbar_init(&S.dempty[t], 1);
    }
    S.abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = S.tmem;

  if (warp == 1) {
    // ---------------- producer: bulk copies of A row chunks and X window runs
    int64_t g = 0;   // chunk counter of this CTA
    bool ok = true;
    for (int64_t B = blockIdx.x; B < L.nbox && ok; B += gridDim.x) {
      const T2Box bx = t2_box(L, B);
      for (int c = 0; c < bx.nchunk; ++c, ++g) {
        const int s = (int)(g % kT2Stages);
        if (g >= kT2Stages) {
          ok = t2_wait(&S.empty[s], (uint32_t)(((g / kT2Stages) - 1) & 1), abort, err, wait_limit);
          if (!ok) break;
        }
        const int k0 = c * kT2K;
        const uint32_t abytes = (uint32_t)(min(kT2K, bx.Wp - k0) * 4);
        const int xend = min(k0 + kT2K, bx.W);
        const uint32_t xbytes = xend > k0 ? (uint32_t)((xend - k0) * 64) : 0u;
        unsigned char* st = t2sm + (size_t)s * kT2Stage;
        if (lane == 0) mbar_expect_tx(&S.full[s], (uint32_t)b * abytes + xbytes);
        __syncwarp();
        if (lane < b) bulk_g2s(st + (size_t)lane * kT2K * 4, L.vals + bx.kbase + (int64_t)lane * bx.Wp + k0, abytes, &S.full[s]);
        // X: each run of consecutive window rows (one neighbour slot) in one copy
        for (int w = k0 + lane; w < xend; w += 32) {
          const int o = w % b;
          if (w == k0 || o == 0) {
            const int len = min(b - o, xend - w);
            const int64_t row = L.nbr[bx.e0 + w / b] * b + o;
            bulk_g2s(st + kT2AStage + (size_t)(w - k0) * 64, xin + row * M, (uint32_t)len * 64u, &S.full[s]);
          }
        }
      }
    }
    // drain: the copies of the last kT2Stages issued chunks land before the CTA may exit
    if (lane == 0)
      for (int64_t j = g > kT2Stages ? g - kT2Stages : 0; j < g; ++j)
        mbar_wait_bounded(&S.full[j % kT2Stages], (uint32_t)((j / kT2Stages) & 1), nullptr, wait_limit);
  } else if (warp == 0) {
    // ---------------- A converter: staged rows -> TF32 head / tail -> TMEM stage (lane q = row q)
    int64_t g = 0;
    bool ok = true;
    for (int64_t B = blockIdx.x; B < L.nbox && ok; B += gridDim.x) {
      const T2Box bx = t2_box(L, B);
      for (int c = 0; c < bx.nchunk; ++c, ++g) {
        const int s = (int)(g % kT2Stages), t = (int)(g & 1);
        ok = t2_wait(&S.full[s], (uint32_t)((g / kT2Stages) & 1), abort, err, wait_limit);
        if (ok && g >= 2) ok = t2_wait(&S.tfree[t], (uint32_t)(((g >> 1) - 1) & 1), abort, err, wait_limit);
        if (!ok) break;
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        const int valid = min(kT2K, bx.Wp - c * kT2K);   // entries of this chunk in the row
        const float* arow = reinterpret_cast<const float*>(t2sm + (size_t)s * kT2Stage) + lane * kT2K;
#pragma unroll
        for (int h = 0; h < 2; ++h) {   // two halves of 32 columns
          uint32_t hi[32], lo[32];
#pragma unroll
          for (int j4 = 0; j4 < 8; ++j4) {
            const int k = h * 32 + 4 * j4;
            float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
            if (lane < b && k < valid) a = *reinterpret_cast<const float4*>(arow + k);
            const float av[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              float fh, fl;
              tc_split(av[e], fh, fl);
              hi[4 * j4 + e] = __float_as_uint(fh);
              lo[4 * j4 + e] = __float_as_uint(fl);
            }
          }
          tmem_st32(tmem + kT2ACol + (uint32_t)t * 128u + (uint32_t)h * 32u, hi);
          tmem_st32(tmem + kT2ACol + (uint32_t)t * 128u + 64u + (uint32_t)h * 32u, lo);
        }
        asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
        __syncwarp();
        if (lane == 0) { mbar_arrive(&S.empty[s]); mbar_arrive(&S.ready[t]); }
      }
    }
  } else if (warp == 2 || warp == 3) {
    // ---------------- B builders: staged X rows -> TF32 head / tail, K-major core matrices
    const int bt = tid - 64;   // 0..63
    int64_t g = 0;
    bool ok = true;
    for (int64_t B = blockIdx.x; B < L.nbox && ok; B += gridDim.x) {
      const T2Box bx = t2_box(L, B);
      for (int c = 0; c < bx.nchunk; ++c, ++g) {
        const int s = (int)(g % kT2Stages), t = (int)(g & 1);
        ok = t2_wait(&S.full[s], (uint32_t)((g / kT2Stages) & 1), abort, err, wait_limit);
        if (ok && g >= 2) ok = t2_wait(&S.tfree[t], (uint32_t)(((g >> 1) - 1) & 1), abort, err, wait_limit);
        if (!ok) break;
        const int k0 = c * kT2K;
        const int xvalid = max(0, min(kT2K, bx.W - k0));
        const float* xs = reinterpret_cast<const float*>(t2sm + (size_t)s * kT2Stage + kT2AStage);
        unsigned char* bh = t2sm + kT2BOff + (size_t)t * 2 * kT2BTile;
        unsigned char* bl = bh + kT2BTile;
        for (int it = bt; it < kT2K * M; it += 64) {
          const int n = it % M, kk = it / M;
          const float v = kk < xvalid ? xs[kk * M + n] : 0.f;
          float fh, fl;
          tc_split(v, fh, fl);
          const uint32_t off = (uint32_t)((n >> 3) * kTcSBO_A + (kk >> 2) * kTcCoreBytes + (n & 7) * 16 + (kk & 3) * 4);
          *reinterpret_cast<float*>(bh + off) = fh;
          *reinterpret_cast<float*>(bl + off) = fl;
        }
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        __syncwarp();
        if (lane == 0) { mbar_arrive(&S.empty[s]); mbar_arrive(&S.ready[t]); }
      }
    }
  } else if (warp == 5) {
    // ---------------- MMA issuer (one thread)
    if (lane == 0) {
      constexpr uint32_t idesc = tc_idesc_tf32(128, M);
      int64_t g = 0, j = 0;
      bool ok = true;
      int64_t commits = 0;
      for (int64_t B = blockIdx.x; B < L.nbox && ok; B += gridDim.x, ++j) {
        const T2Box bx = t2_box(L, B);
        const int db = (int)(j & 1);
        if (j >= 2) {
          ok = t2_wait(&S.dempty[db], (uint32_t)(((j >> 1) - 1) & 1), abort, err, wait_limit);
          if (!ok) break;
        }
        for (int c = 0; c < bx.nchunk; ++c, ++g) {
          const int t = (int)(g & 1);
          ok = t2_wait(&S.ready[t], (uint32_t)((g >> 1) & 1), abort, err, wait_limit);
          if (!ok) break;
          asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
          const uint32_t bh = sbase + kT2BOff + (uint32_t)t * 2u * kT2BTile, bl = bh + kT2BTile;
          const uint32_t ah = tmem + kT2ACol + (uint32_t)t * 128u, al = ah + 64u;
          const uint32_t d = tmem + (uint32_t)db * 16u;
#pragma unroll
          for (int ks = 0; ks < kT2K / 8; ++ks) {
            const uint32_t ko = (uint32_t)ks * 2u * kTcCoreBytes;
            const uint64_t dh = tc_smem_desc(bh + ko, kTcCoreBytes, kTcSBO_A);
            const uint64_t dl = tc_smem_desc(bl + ko, kTcCoreBytes, kTcSBO_A);
            const uint32_t acc0 = (c > 0 || ks > 0) ? 1u : 0u;
            tc_mma_ta(d, al + (uint32_t)ks * 8u, dh, idesc, acc0);   // small terms first
            tc_mma_ta(d, ah + (uint32_t)ks * 8u, dl, idesc, 1u);
            tc_mma_ta(d, ah + (uint32_t)ks * 8u, dh, idesc, 1u);
          }
          tc_commit(&S.tfree[t]);
          ++commits;
          if (c + 1 == bx.nchunk) tc_commit(&S.dfull[db]);
        }
      }
      // drain: every product issued has completed before TMEM is freed
      if (commits > 0) {
        const int64_t gl = g - 1;   // the last committed chunk
        mbar_wait_bounded(&S.tfree[gl & 1], (uint32_t)((gl >> 1) & 1), nullptr, wait_limit);
      }
    }
  } else {
    // ---------------- epilogue (warp 4: TMEM lanes 0..31 = box rows)
    int64_t j = 0;
    for (int64_t B = blockIdx.x; B < L.nbox; B += gridDim.x, ++j) {
      const int db = (int)(j & 1);   // every box holds its diagonal block: at least one chunk, one commit
      if (!t2_wait(&S.dfull[db], (uint32_t)((j >> 1) & 1), abort, err, wait_limit)) break;
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      uint32_t v[16];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
            "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
          : "r"(tmem + (uint32_t)db * 16u));
      asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(&S.dempty[db]);
      if (lane < b) {
        double unused[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
        for (int c0 = 0; c0 < M; c0 += 4) {
          Slice<float> sl;
#pragma unroll
          for (int e = 0; e < 4; ++e) sl.v[e] = __uint_as_float(v[c0 + e]);
          ep.post(B * b + lane, c0, sl, unused);
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;\n" ::"r"(tmem) : "memory");
}

}  // namespace r3mg
