// Symmetric block form of a coarse level step (FP32 V-cycle).
//
// A Galerkin level A_l = P^T A_{l-1} P is symmetric, so only the blocks (B, B') with B' >= B are
// stored ("upper" rows: the diagonal block followed by the upper neighbours' blocks).  One pass
// over a stored block serves both products it takes part in:
//   y_B  += A_BB' x_B'             (row-wise, reduced across the CTA)
//   t_BB' = A_BB'^T x_B            (column-wise, one b-vector per off-diagonal upper pair)
// k_sym_block streams every stored block once (half the bytes of the full operator), one CTA
// per box with one thread per 4 columns; k_sym_finish adds to each row the transposed
// contributions of its lower neighbours, in increasing box order, and applies the fused
// Chebyshev-Jacobi update.  Both passes are deterministic.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "kernels_level.cuh"
#include "kernels_level_tma.cuh"

namespace r3mg {

struct SymView {
  int64_t nbox = 0;
  int b = 0;
  const float* vals = nullptr;     // upper rows: row (B, q') at up_base[B] + q' * up_len[B]
  const int64_t* up_base = nullptr;
  const int32_t* up_len = nullptr; // padded upper row length of box B (multiple of 4)
  const int64_t* nbr_ptr = nullptr;
  const int64_t* nbr = nullptr;
  const int32_t* dslot = nullptr;  // slot of the diagonal block in box B's neighbour list
  const int64_t* tp_off = nullptr; // first transposed-pair vector of box B
  const int64_t* low_ptr = nullptr;// per box: range of lower pairs (transposed vectors to add)
  const int64_t* low_pair = nullptr;
  int win_max = 0;                 // largest upper window (padded)
  int stage_max = 0;               // largest upper slice of one box, b x up_len floats
};

constexpr int kSymMaxB = 32;
constexpr int kSymThreads = 128;
static_assert(kSymMaxB == 32, "the halving exchange maps lane q to row q of up to 32 rows");

template <bool SMEM>
__device__ __forceinline__ float4 sym_ld(const float* p) {
  if constexpr (SMEM) return *reinterpret_cast<const float4*>(p);
  else return __ldcs(reinterpret_cast<const float4*>(p));   // read once: stream past the caches
}

// One box of the symmetric product, the upper slice at `base` (row stride Wp, global or shared
// memory) and the upper x window in `swin`: row partials reduced into ybuf, column sums of the
// off-diagonal upper blocks into tbuf.  Shared by the streamed and the staged kernels, so both give
// the same bits.
template <bool SMEM, int WAVE = 8, int NT = kSymThreads>
__device__ __forceinline__ void sym_box(const SymView& V, int64_t B, int W, int Wp, const float* swin,
                                        const float* base, float* __restrict__ ybuf, float* __restrict__ tbuf,
                                        float (&ysum)[NT / 32][32]) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, NW = NT / 32;
  const int b = V.b;
  float yp[kSymMaxB];
#pragma unroll
  for (int q = 0; q < kSymMaxB; ++q) yp[q] = 0.f;
  const int64_t tp = V.tp_off[B];
  for (int c4 = tid; 4 * c4 < Wp; c4 += NT) {
    const float4 xw = *reinterpret_cast<const float4*>(swin + 4 * c4);
    float4 t = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int q0r = 0; q0r < kSymMaxB; q0r += WAVE) {
      if (q0r >= b) break;
      float4 a[WAVE];
#pragma unroll
      for (int j = 0; j < WAVE; ++j)
        a[j] = (q0r + j < b) ? sym_ld<SMEM>(base + (int64_t)(q0r + j) * Wp + 4 * c4)
                             : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int j = 0; j < WAVE; ++j) {
        const int q = q0r + j;
        yp[q] += a[j].x * xw.x + a[j].y * xw.y + a[j].z * xw.z + a[j].w * xw.w;
        const float xq = (q < b) ? swin[q] : 0.f;   // x_B: the diagonal slot opens the window
        t.x += a[j].x * xq; t.y += a[j].y * xq; t.z += a[j].z * xq; t.w += a[j].w * xq;
      }
    }
    const float tv[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = 4 * c4 + j;
      if (c >= b && c < W) {   // an off-diagonal upper block: keep A_BB'^T x_B
        const int sI = c / b;
        tbuf[(tp + sI - 1) * b + (c - sI * b)] = tv[j];
      }
    }
  }
  // halving exchange: at each step a lane keeps the half of its values its lane bit selects
  // and adds the partner's copy of that half; lane q ends with the warp's sum of row q
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) {
    const bool hi = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < o; ++i) {
      const float send = hi ? yp[i] : yp[i + o];
      const float keep = hi ? yp[i + o] : yp[i];
      yp[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
  ysum[warp][lane] = yp[0];
  __syncthreads();
  if (tid < b) {
    float y = 0.f;
    for (int w = 0; w < NW; ++w) y += ysum[w][tid];
    ybuf[B * b + tid] = y;
  }
}

// One CTA (NT = 128 threads, or 96: an interior box of a 27-row level has 95 four-column groups,
// so 96 threads leave none idle and let more CTAs reside) per box.  The box's upper window (x over
// the diagonal and upper neighbour slots) is staged in shared memory; each thread owns 4
// consecutive columns of the box's upper rows (one 16-byte load per row, coalesced along the
// row), walks all b rows in waves of WAVE loads in flight (8, or 4 for fewer registers and more
// resident CTAs), and keeps
//   * the row partials y_q += A[q, cols] . x_win[cols] for every row q (registers), and
//   * the column sums t_cols = sum_q A[q, cols] x_B[q] (A_BB'^T x_B for its upper slots).
// The row partials are reduced across each warp by a halving exchange (31 shuffles leave lane q
// with row q's warp sum) and across the 4 warps in a fixed order, so the result is deterministic.
template <int WAVE, int NT = kSymThreads>
__global__ void __launch_bounds__(NT, (WAVE == 4 ? 8 : 6) * kSymThreads / NT) k_sym_block(SymView V,
                                                          const float* __restrict__ xin,
                                                          float* __restrict__ ybuf, float* __restrict__ tbuf) {
  extern __shared__ __align__(16) float swin[];
  __shared__ float ysum[NT / 32][32];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, NW = NT / 32;
  const int b = V.b;
  for (int64_t B = blockIdx.x; B < V.nbox; B += gridDim.x) {
    const int64_t q0 = V.nbr_ptr[B];
    const int nn = (int)(V.nbr_ptr[B + 1] - q0), d = V.dslot[B], nup = nn - d;
    const int W = nup * b, Wp = V.up_len[B];
    for (int sI = warp; sI < nup; sI += NW) {
      const int64_t src = V.nbr[q0 + d + sI] * b;
      for (int t = lane; t < b; t += 32) cp_async_elem(swin + sI * b + t, xin + src + t);
    }
    for (int t = W + tid; t < Wp; t += NT) swin[t] = 0.f;
    cp_async_wait_all();
    __syncthreads();
    sym_box<false, WAVE, NT>(V, B, W, Wp, swin, V.vals + V.up_base[B], ybuf, tbuf, ysum);
    __syncthreads();   // the window and ysum are free for the next box
  }
}

// Staged symmetric block step.  A box's upper slice (b x up_len floats) is one contiguous run of
// the upper values, so one CTA per box requests all of it at once with a single bulk copy
// (cp.async.bulk into shared memory, completion on an mbarrier) while its threads gather the x
// window; with several CTAs resident per SM, whole boxes are in flight instead of eight rows per
// thread.  A box whose slice exceeds the shared-memory stage (`cap_floats`) reads its slice
// from global memory as k_sym_block does.  The arithmetic of a box is sym_box's, so both kernels
// give the same bits.  The mbarrier wait is bounded; on expiry the CTA raises *err, waits
// (bounded) for its copy and returns.
__global__ void __launch_bounds__(kSymThreads) k_sym_block_staged(SymView V, const float* __restrict__ xin,
                                                                 float* __restrict__ ybuf, float* __restrict__ tbuf,
                                                                 int cap_floats, int* __restrict__ err,
                                                                 long long wait_limit, int withhold_first) {
  extern __shared__ __align__(128) float sstage[];   // stage (cap_floats) | window (win_max)
  __shared__ float ysum[kSymThreads / 32][32];
  __shared__ __align__(8) uint64_t bar;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, NW = kSymThreads / 32;
  const int b = V.b;
  const int64_t B = blockIdx.x;
  const int Wp = V.up_len[B];
  const bool staged = (int64_t)b * Wp <= (int64_t)cap_floats;
  const bool withheld = withhold_first && B == 0 && staged;   // test of the expiry path
  if (tid == 0 && staged) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    if (!withheld) {
      const uint32_t bytes = (uint32_t)(sizeof(float) * (size_t)b * Wp);
      mbar_expect_tx(&bar, bytes);
      bulk_g2s(sstage, V.vals + V.up_base[B], bytes, &bar);
    }
  }
  float* swin = sstage + cap_floats;
  const int64_t q0 = V.nbr_ptr[B];
  const int nn = (int)(V.nbr_ptr[B + 1] - q0), d = V.dslot[B], nup = nn - d;
  const int W = nup * b;
  for (int sI = warp; sI < nup; sI += NW) {
    const int64_t src = V.nbr[q0 + d + sI] * b;
    for (int t = lane; t < b; t += 32) cp_async_elem(swin + sI * b + t, xin + src + t);
  }
  for (int t = W + tid; t < Wp; t += kSymThreads) swin[t] = 0.f;
  cp_async_wait_all();
  __syncthreads();   // the window is complete and the mbarrier initialised
  if (staged) {
    const bool got = mbar_wait_bounded(&bar, 0u, err, wait_limit);
    if (__syncthreads_or(!got)) {
      if (tid == 0 && !withheld) mbar_wait_bounded(&bar, 0u, nullptr, wait_limit);   // the copy lands first
      __syncthreads();
      return;
    }
    sym_box<true>(V, B, W, Wp, swin, sstage, ybuf, tbuf, ysum);
  } else {
    sym_box<false>(V, B, W, Wp, swin, V.vals + V.up_base[B], ybuf, tbuf, ysum);
  }
}

// Chebyshev step on the completed product: y = ybuf + sum over lower pairs of t.
struct SymCheb {
  float* x; float* r; const float* d; float* dnext; const float* dinv; float a, c;
  const double* A = nullptr; const double* C = nullptr; const int32_t* rprob = nullptr;   // batched coefficients
  __device__ void operator()(int64_t i, float y) const {
    float aa = a, cc = c;
    if (rprob) { const int p = rprob[i]; aa = (float)A[p]; cc = (float)C[p]; }
    const float di = d[i];
    x[i] += di;
    const float rn = r[i] - y;
    r[i] = rn;
    dnext[i] = aa * di + cc * dinv[i] * rn;
  }
};

__global__ void k_sym_finish(SymView V, const float* __restrict__ ybuf, const float* __restrict__ tbuf, SymCheb ep) {
  const int64_t n = V.nbox * V.b;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t B = i / V.b;
    const int q = (int)(i - B * V.b);
    float y = ybuf[i];
    const int64_t k0 = V.low_ptr[B], k1 = V.low_ptr[B + 1];
    int64_t k = k0;
    // four independent loads in flight, added in increasing pair order (deterministic)
    for (; k + 4 <= k1; k += 4) {
      const float t0 = tbuf[V.low_pair[k] * V.b + q], t1 = tbuf[V.low_pair[k + 1] * V.b + q];
      const float t2 = tbuf[V.low_pair[k + 2] * V.b + q], t3 = tbuf[V.low_pair[k + 3] * V.b + q];
      y += t0; y += t1; y += t2; y += t3;
    }
    for (; k < k1; ++k) y += tbuf[V.low_pair[k] * V.b + q];
    ep(i, y);
  }
}

// upper rows from the full FP32 block rows: row (B, q') keeps its slots from the diagonal on
__global__ void k_sym_gather(SymView V, const int64_t* __restrict__ row_ptr, const float* __restrict__ full,
                             float* __restrict__ up) {
  const int64_t nrows = V.nbox * V.b;
  for (int64_t i = blockIdx.x; i < nrows; i += gridDim.x) {
    const int64_t B = i / V.b;
    const int q = (int)(i - B * V.b);
    const int d = V.dslot[B];
    const int nup = (int)(V.nbr_ptr[B + 1] - V.nbr_ptr[B]) - d;
    const int len = V.up_len[B];
    float* dst = up + V.up_base[B] + (int64_t)q * len;
    const float* src = full + row_ptr[i] + (int64_t)d * V.b;
    for (int t = threadIdx.x; t < len; t += blockDim.x) dst[t] = (t < nup * V.b) ? src[t] : 0.f;
  }
}

}  // namespace r3mg
