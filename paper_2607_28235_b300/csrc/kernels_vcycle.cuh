// V-cycle transfer kernels (Section 4): restriction b_{l+1} = P^T r_l fused with the
// initialisation of the next level's smoother, prolongation d_l = P (x_{l+1} + d_{l+1}),
// and the coarsest-level solve with the explicit inverse of the Cholesky-factored A_{L-1}.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace r3mg {

// Next-level initialisation after restriction: r = b, x = 0, d = c0 * dinv * b (first
// Chebyshev update of the zero initial guess).  On the coarsest level only r = b is written.
template <typename T>
struct NextInit {
  T* r; T* x; T* d; const T* dinv; T c0;
  __device__ void operator()(int64_t i, T bi) const {
    r[i] = bi;
    if (x) { x[i] = T(0); d[i] = c0 * dinv[i] * bi; }
  }
};

// The transfer kernels' bodies are device functions so that the persistent batched solve runs
// the same code; `rprob`/`act` (both null in the plain kernels) skip the rows of problems that
// have stopped.
__device__ __forceinline__ bool skip_row(const int32_t* rprob, const int* act, int64_t row) {
  return act != nullptr && !act[rprob[row]];
}

// Fine -> level 1: b1[B*b + q] = sum_{i in B} P0[i][q] r[i].  One CTA per box.
template <typename T, class NX>
__device__ __forceinline__ void restrict_fine_body(const T* __restrict__ P0, const T* __restrict__ r,
                                                   const int64_t* __restrict__ box_row, int64_t nbox, int b, NX nx,
                                                   const int32_t* rprob1, const int* act) {
  __shared__ T part[256];
  const int per = blockDim.x / b;   // row lanes per coefficient (b <= 256)
  const int q = threadIdx.x % b, j = threadIdx.x / b;
  for (int64_t B = blockIdx.x; B < nbox; B += gridDim.x) {
    if (skip_row(rprob1, act, B * b)) continue;   // uniform across the CTA
    T s = T(0);
    if (j < per) {
      // unrolled so that several rows' loads are in flight at once (the sum keeps its order)
#pragma unroll 4
      for (int64_t i = box_row[B] + j; i < box_row[B + 1]; i += per) s += P0[i * b + q] * r[i];
    }
    part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x < b) {
      T t = T(0);
      for (int k = 0; k < per; ++k) t += part[k * b + threadIdx.x];
      nx(B * b + threadIdx.x, t);
    }
    __syncthreads();
  }
}

template <typename T, class NX>
__global__ void __launch_bounds__(256) k_restrict_fine(const T* __restrict__ P0, const T* __restrict__ r,
                                                       const int64_t* __restrict__ box_row, int64_t nbox, int b,
                                                       NX nx) {
  restrict_fine_body<T, NX>(P0, r, box_row, nbox, b, nx, nullptr, nullptr);
}

// Level l -> l+1 (l >= 1): b_{l+1}[B][q] = sum_{children c} sum_{q'} Pt[c][q'][q] r_l[c][q'].
template <typename T, class NX>
__device__ __forceinline__ void restrict_coarse_body(const T* __restrict__ Pt, const T* __restrict__ r,
                                                     int64_t nparent, int b, int fan, NX nx, int64_t t0, int64_t ts,
                                                     const int32_t* rprob1, const int* act) {
  const int64_t tot = nparent * b;
  for (int64_t t = t0; t < tot; t += ts) {
    if (skip_row(rprob1, act, t)) continue;
    const int64_t B = t / b;
    const int q = (int)(t - B * b);
    T s = T(0);
    for (int64_t c = B * fan; c < (B + 1) * fan; ++c)
      for (int qp = 0; qp < b; ++qp) s += Pt[(c * b + qp) * b + q] * r[c * b + qp];
    nx(t, s);
  }
}

template <typename T, class NX>
__global__ void k_restrict_coarse(const T* __restrict__ Pt, const T* __restrict__ r, int64_t nparent, int b, int fan,
                                  NX nx) {
  restrict_coarse_body<T, NX>(Pt, r, nparent, b, fan, nx, blockIdx.x * (int64_t)blockDim.x + threadIdx.x,
                              (int64_t)gridDim.x * blockDim.x, nullptr, nullptr);
}

// The same restriction with one CTA per parent box: the threads take the (child, q) pairs, each
// summing its child's b products, and threads q < b add the fan partials in child order.  Every
// output's fan * b products then run on fan threads instead of one (the single-hierarchy V-cycle;
// the batched loops keep the thread-per-output body above, which their persistent kernel shares).
// Dynamic shared memory: fan * b values of T.
template <typename T, class NX>
__global__ void __launch_bounds__(256) k_restrict_coarse_box(const T* __restrict__ Pt, const T* __restrict__ r,
                                                           int64_t nparent, int b, int fan, NX nx) {
  extern __shared__ __align__(16) unsigned char rc_raw[];
  T* part = reinterpret_cast<T*>(rc_raw);
  for (int64_t B = blockIdx.x; B < nparent; B += gridDim.x) {
    for (int it = threadIdx.x; it < fan * b; it += blockDim.x) {
      const int ci = it / b, q = it - ci * b;
      const int64_t c = B * fan + ci;
      T s = T(0);
      for (int qp = 0; qp < b; ++qp) s += Pt[(c * b + qp) * b + q] * r[c * b + qp];
      part[it] = s;
    }
    __syncthreads();
    if (threadIdx.x < b) {
      T t = T(0);
      for (int ci = 0; ci < fan; ++ci) t += part[ci * b + threadIdx.x];
      nx(B * b + threadIdx.x, t);
    }
    __syncthreads();
  }
}

// Level 1 -> fine: d0[k] = sum_q P0[k][q] (x1 + d1)[box(k)*b + q]   (d1 may be null).
template <typename T>
__device__ __forceinline__ void prolong_fine_body(const T* __restrict__ P0, const int32_t* __restrict__ box_of,
                                                  const T* __restrict__ x1, const T* __restrict__ d1, int64_t n, int b,
                                                  T* __restrict__ d0, int64_t k0, int64_t ks, const int32_t* rprob,
                                                  const int* act) {
  for (int64_t k = k0; k < n; k += ks) {
    if (skip_row(rprob, act, k)) continue;
    const int64_t B = box_of[k];
    T s = T(0);
#pragma unroll 4
    for (int q = 0; q < b; ++q) {
      const T e = x1[B * b + q] + (d1 ? d1[B * b + q] : T(0));
      s += P0[k * b + q] * e;
    }
    d0[k] = s;
  }
}

template <typename T>
__global__ void k_prolong_fine(const T* __restrict__ P0, const int32_t* __restrict__ box_of, const T* __restrict__ x1,
                               const T* __restrict__ d1, int64_t n, int b, T* __restrict__ d0) {
  prolong_fine_body<T>(P0, box_of, x1, d1, n, b, d0, blockIdx.x * (int64_t)blockDim.x + threadIdx.x,
                       (int64_t)gridDim.x * blockDim.x, nullptr, nullptr);
}

// The same prolongation with each warp's 32 rows of P0 (32 x b contiguous values) first copied
// to shared memory by coalesced loads, so that a row's b values are not gathered at a stride of
// b values across the warp; each row's sum keeps its order.  The single-hierarchy V-cycle; the
// batched loops keep the body above.  Dynamic shared memory: 32 x b values of T per warp.
template <typename T>
__global__ void k_prolong_fine_staged(const T* __restrict__ P0, const int32_t* __restrict__ box_of,
                                      const T* __restrict__ x1, const T* __restrict__ d1, int64_t n, int b,
                                      T* __restrict__ d0) {
  extern __shared__ __align__(16) unsigned char pf_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, NW = blockDim.x >> 5;
  T* wp = reinterpret_cast<T*>(pf_raw) + (int64_t)warp * 32 * b;
  for (int64_t base = ((int64_t)blockIdx.x * NW + warp) * 32; base < n; base += (int64_t)gridDim.x * NW * 32) {
    const int rows = (int)(n - base < 32 ? n - base : 32);
    const T* src = P0 + base * b;
    for (int t = lane; t < rows * b; t += 32) wp[t] = src[t];
    __syncwarp();
    if (lane < rows) {
      const int64_t k = base + lane;
      const int64_t B = box_of[k];
      T s = T(0);
#pragma unroll 4
      for (int q = 0; q < b; ++q) {
        const T e = x1[B * b + q] + (d1 ? d1[B * b + q] : T(0));
        s += wp[lane * b + q] * e;
      }
      d0[k] = s;
    }
    __syncwarp();
  }
}

// Level l+1 -> l: d_l[c][q'] = sum_q Pt[c][q'][q] (x + d)_{l+1}[parent(c)][q].
template <typename T>
__device__ __forceinline__ void prolong_coarse_body(const T* __restrict__ Pt, const T* __restrict__ x1,
                                                    const T* __restrict__ d1, int64_t nchild, int b, int fan,
                                                    T* __restrict__ d0, int64_t t0, int64_t ts, const int32_t* rprob,
                                                    const int* act) {
  for (int64_t t = t0; t < nchild * b; t += ts) {
    if (skip_row(rprob, act, t)) continue;
    const int64_t c = t / b;
    const int qp = (int)(t - c * b);
    const int64_t B = c / fan;
    T s = T(0);
    for (int q = 0; q < b; ++q) s += Pt[(c * b + qp) * b + q] * (x1[B * b + q] + (d1 ? d1[B * b + q] : T(0)));
    d0[t] = s;
  }
}

template <typename T>
__global__ void k_prolong_coarse(const T* __restrict__ Pt, const T* __restrict__ x1, const T* __restrict__ d1,
                                 int64_t nchild, int b, int fan, T* __restrict__ d0) {
  prolong_coarse_body<T>(Pt, x1, d1, nchild, b, fan, d0, blockIdx.x * (int64_t)blockDim.x + threadIdx.x,
                         (int64_t)gridDim.x * blockDim.x, nullptr, nullptr);
}

// Coarsest solve x = A_c^{-1} r with the symmetric inverse formed from the Cholesky factor.
// One warp per row, 16-byte loads along the row.
template <typename T>
__global__ void __launch_bounds__(256) k_dense_gemv(const T* __restrict__ M, int64_t ld, const T* __restrict__ r,
                                                    int64_t nc, T* __restrict__ x) {
  const int lane = threadIdx.x & 31;
  const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t row = w; row < nc; row += nw) {
    const T* a = M + row * ld;
    T s = T(0);
    for (int64_t k = lane; k < nc; k += 32) s += a[k] * r[k];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) x[row] = s;
  }
}

}  // namespace r3mg
