// Symmetric block form of a coarse level step (FP32 V-cycle).
//
// A Galerkin level A_l = P^T A_{l-1} P is symmetric, so only the blocks (B, B') with B' >= B are
// stored ("upper" rows: the diagonal block followed by the upper neighbours' blocks).  One pass
// over a stored block serves both products it takes part in:
//   y_B  += A_BB' x_B'             (row-wise, reduced across the CTA)
//   t_BB' = A_BB'^T x_B            (column-wise, one b-vector per off-diagonal upper pair)
// k_sym_block streams every stored block once (half the bytes of the full operator) with one
// thread per 4 columns and all b rows in flight; k_sym_finish adds to each row the transposed
// contributions of its lower neighbours, in increasing box order, and applies the fused
// Chebyshev-Jacobi update.  Both passes are deterministic.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "kernels_level.cuh"

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
};

constexpr int kSymMaxB = 32;

// One warp per box (8 boxes per CTA, no CTA-wide barrier).  A pass gives each lane two 16-byte
// column chunks of the box's upper rows and walks all b rows: the row partials of y stay in
// the lane's registers (reduced across the warp at the end), the transposed sums t of the
// lane's columns are complete after the pass and are written at once.
__global__ void __launch_bounds__(256) k_sym_block(SymView V, const float* __restrict__ xin, float* __restrict__ ybuf,
                                                   float* __restrict__ tbuf) {
  extern __shared__ __align__(16) float swin_all[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float* swin = swin_all + warp * V.win_max;
  const int b = V.b;
  for (int64_t B = (int64_t)blockIdx.x * 8 + warp; B < V.nbox; B += (int64_t)gridDim.x * 8) {
    const int64_t q0 = V.nbr_ptr[B];
    const int nn = (int)(V.nbr_ptr[B + 1] - q0), d = V.dslot[B], nup = nn - d;
    const int W = nup * b, Wp = V.up_len[B];
    for (int sI = 0; sI < nup; ++sI) {
      const int64_t src = V.nbr[q0 + d + sI] * b;
      for (int t = lane; t < b; t += 32) cp_async_elem(swin + sI * b + t, xin + src + t);
    }
    for (int t = W + lane; t < Wp; t += 32) swin[t] = 0.f;
    cp_async_wait_all();
    __syncwarp();
    float yacc[kSymMaxB];
#pragma unroll
    for (int q = 0; q < kSymMaxB; ++q) yacc[q] = 0.f;
    const float* base = V.vals + V.up_base[B];
    const int nch = Wp >> 2;
    for (int p0 = 0; p0 < nch; p0 += 64) {
      const int c0 = p0 + lane, c1 = p0 + 32 + lane;
      const bool v0 = c0 < nch, v1 = c1 < nch;
      const float4 x0 = v0 ? *reinterpret_cast<const float4*>(swin + 4 * c0) : make_float4(0.f, 0.f, 0.f, 0.f);
      const float4 x1 = v1 ? *reinterpret_cast<const float4*>(swin + 4 * c1) : make_float4(0.f, 0.f, 0.f, 0.f);
      float4 t0 = make_float4(0.f, 0.f, 0.f, 0.f), t1 = t0;
#pragma unroll
      for (int q = 0; q < kSymMaxB; ++q) {
        if (q < b) {
          const float* row = base + (int64_t)q * Wp;
          const float4 a0 = v0 ? __ldcs(reinterpret_cast<const float4*>(row + 4 * c0)) : make_float4(0.f, 0.f, 0.f, 0.f);
          const float4 a1 = v1 ? __ldcs(reinterpret_cast<const float4*>(row + 4 * c1)) : make_float4(0.f, 0.f, 0.f, 0.f);
          yacc[q] += a0.x * x0.x + a0.y * x0.y + a0.z * x0.z + a0.w * x0.w + a1.x * x1.x + a1.y * x1.y + a1.z * x1.z +
                     a1.w * x1.w;
          const float xq = swin[q];   // x_B: the diagonal slot is the window's first segment
          t0.x += a0.x * xq; t0.y += a0.y * xq; t0.z += a0.z * xq; t0.w += a0.w * xq;
          t1.x += a1.x * xq; t1.y += a1.y * xq; t1.z += a1.z * xq; t1.w += a1.w * xq;
        }
      }
      const float tv[8] = {t0.x, t0.y, t0.z, t0.w, t1.x, t1.y, t1.z, t1.w};
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int c = 4 * (j < 4 ? c0 : c1) + (j & 3);
        if (c >= b && c < W) {   // off-diagonal upper block: keep A_BB'^T x_B
          const int sI = c / b;
          tbuf[(V.tp_off[B] + sI - 1) * b + (c - sI * b)] = tv[j];
        }
      }
    }
    // y_B: reduce the lanes' row partials (fixed butterfly order)
#pragma unroll
    for (int q = 0; q < kSymMaxB; ++q) {
      if (q < b) {
        float v = yacc[q];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) ybuf[B * b + q] = v;
      }
    }
    __syncwarp();
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
    for (int64_t k = V.low_ptr[B]; k < V.low_ptr[B + 1]; ++k) y += tbuf[V.low_pair[k] * V.b + q];
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
