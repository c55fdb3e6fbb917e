// Batched solves: many independent problems, each with its own R-tree hierarchy, concatenated
// level by level into one block-diagonal hierarchy.  A V-cycle step of every problem is one
// launch; what differs per problem (Chebyshev coefficients, CG scalars, coarsest factor) is
// looked up through a per-row problem id.  Dots are segmented per problem and reduced in a
// fixed order, so results do not depend on the other problems of the batch.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "kernels_level.cuh"

namespace r3mg {

// Chebyshev step with per-problem coefficients: a = A[prob(i)], c = C[prob(i)] (tables of the step).
template <typename T>
struct TEpChebB {
  T* x; T* r; const T* d; T* dnext; const T* dinv; const double* A; const double* C; const int32_t* rprob;
  static constexpr bool kDot = false;
  static constexpr int kStage = 4;
  __device__ const T* src(int j) const { return j == 0 ? x : j == 1 ? r : j == 2 ? d : dinv; }
  __device__ bool stage(int) const { return true; }
  __device__ void post(int64_t i, int lr, T y_r, T* const* aux, double&) const {
    const int p = rprob[i];
    const T di = aux[2][lr];
    x[i] = aux[0][lr] + di;
    const T rn = aux[1][lr] - y_r;
    r[i] = rn;
    dnext[i] = (T)A[p] * di + (T)C[p] * aux[3][lr] * rn;
  }
};

// Next-level initialisation after restriction with the per-problem first Chebyshev factor.
template <typename T>
struct NextInitB {
  T* r; T* x; T* d; const T* dinv; const double* c0; const int32_t* rprob;
  __device__ void operator()(int64_t i, T bi) const {
    r[i] = bi;
    if (x) { x[i] = T(0); d[i] = (T)c0[rprob[i]] * dinv[i] * bi; }
  }
};

// Block-diagonal coarsest solve: row r of problem p uses its own dense inverse (rows of stopped
// problems skipped when `act` is given).
template <typename T>
__device__ __forceinline__ void block_gemv_body(const T* __restrict__ M, const int64_t* __restrict__ moff,
                                                const int64_t* __restrict__ mld, const int64_t* __restrict__ cof,
                                                const int32_t* __restrict__ rprob, const T* __restrict__ r,
                                                int64_t nrows, T* __restrict__ x, const int* act) {
  const int lane = threadIdx.x & 31;
  const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t row = w; row < nrows; row += nw) {
    const int p = rprob[row];
    if (act && !act[p]) continue;   // uniform across the warp (one row per warp)
    const int64_t c0 = cof[p], nc = cof[p + 1] - c0, ld = mld[p];
    const T* a = M + moff[p] + (row - c0) * ld;
    T s = T(0);
    for (int64_t k = lane; k < nc; k += 32) s += a[k] * r[c0 + k];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) x[row] = s;
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_block_gemv(const T* __restrict__ M, const int64_t* __restrict__ moff,
                                                    const int64_t* __restrict__ mld, const int64_t* __restrict__ cof,
                                                    const int32_t* __restrict__ rprob, const T* __restrict__ r,
                                                    int64_t nrows, T* __restrict__ x) {
  block_gemv_body<T>(M, moff, mld, cof, rprob, r, nrows, x, nullptr);
}

// Segmented dot products: segment s covers rows [sb[s], se[s]) of one problem.
template <typename T>
__global__ void k_seg_dot(const T* __restrict__ x, const T* __restrict__ y, const int64_t* __restrict__ sb,
                          const int64_t* __restrict__ se, int nseg, double* __restrict__ part) {
  __shared__ double red[32];
  for (int s = blockIdx.x; s < nseg; s += gridDim.x) {
    double acc = 0.0;
    for (int64_t k = sb[s] + threadIdx.x; k < se[s]; k += blockDim.x)
      acc += (double)x[k] * (double)(y ? y[k] : x[k]);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[k];
      part[s] = t;
    }
    __syncthreads();
  }
}

// out[p] = sum of the partials of problem p's segments [soff[p], soff[p+1]), in order.
__global__ void k_seg_reduce(const double* __restrict__ part, const int* __restrict__ soff, int np,
                             double* __restrict__ out) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < np; p += gridDim.x * blockDim.x) {
    double t = 0.0;
    for (int s = soff[p]; s < soff[p + 1]; ++s) t += part[s];
    out[p] = t;
  }
}

// Batched CG scalars and state, one entry per problem.
struct BatchScal {
  double *pq, *pr, *zq, *rz, *rzn, *rr, *bb, *alpha, *beta;
  int *active, *its, *any, *err;
};

enum BFin : int { BF_ALPHA_PCG = 0, BF_ALPHA_FCG, BF_BETA_PCG, BF_BETA_FCG };

__global__ void k_bscal(BatchScal S, int np, int mode) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < np; p += gridDim.x * blockDim.x) {
    if (mode == BF_ALPHA_PCG || mode == BF_ALPHA_FCG) {
      const double num = (mode == BF_ALPHA_PCG) ? S.rz[p] : S.pr[p];
      const double pq = S.pq[p];
      if (!S.active[p]) { S.alpha[p] = 0.0; continue; }
      if (!(pq > 0.0) || !isfinite(num)) { S.alpha[p] = 0.0; S.active[p] = 0; atomicExch(S.err, 1); continue; }
      S.alpha[p] = num / pq;
    } else if (mode == BF_BETA_PCG) {
      S.beta[p] = S.rzn[p] / S.rz[p];
      S.rz[p] = S.rzn[p];
    } else {
      S.beta[p] = S.zq[p] / S.pq[p];
    }
  }
}

// After an x update: count it, stop problems whose ||r|| <= rtol ||b|| or that reached maxit,
// and publish whether any problem is still running (the graph's loop condition).
__global__ void k_bconverge(BatchScal S, int np, double rtol2, int maxit) {
  __shared__ int any;
  if (threadIdx.x == 0) any = 0;
  __syncthreads();
  for (int p = threadIdx.x; p < np; p += blockDim.x) {
    if (S.active[p]) {
      S.its[p] += 1;
      if (S.rr[p] <= rtol2 * S.bb[p] || S.its[p] >= maxit) S.active[p] = 0;
    }
    if (S.active[p]) atomicOr(&any, 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) *S.any = any;
}

__global__ void k_set_condition(cudaGraphConditionalHandle hdl, const int* __restrict__ flag) {
  if (threadIdx.x == 0 && blockIdx.x == 0) cudaGraphSetConditional(hdl, *flag ? 1u : 0u);
}

template <typename T>
__global__ void k_bvc_init(const double* __restrict__ r, int64_t n, T* vr, T* vx, T* vd, const T* __restrict__ dinv,
                           const double* __restrict__ c0, const int32_t* __restrict__ rprob) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    const T rt = (T)r[k];
    vr[k] = rt;
    vx[k] = T(0);
    vd[k] = (T)c0[rprob[k]] * dinv[k] * rt;
  }
}

// x += alpha_p p;  r -= alpha_p q;  V-cycle entry from the new r.
template <typename T>
__global__ void k_bcg_update(double* __restrict__ x, double* __restrict__ r, const double* __restrict__ p,
                             const double* __restrict__ q, const double* __restrict__ alpha,
                             const int32_t* __restrict__ rprob, int64_t n, T* vr, T* vx, T* vd,
                             const T* __restrict__ dinv, const double* __restrict__ c0) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    const int pp = rprob[k];
    const double a = alpha[pp];
    x[k] += a * p[k];
    const double rk = r[k] - a * q[k];
    r[k] = rk;
    const T rt = (T)rk;
    vr[k] = rt;
    vx[k] = T(0);
    vd[k] = (T)c0[pp] * dinv[k] * rt;
  }
}

template <typename T>
__global__ void k_bvc_final(const T* __restrict__ vx, const T* __restrict__ vd, double* __restrict__ z, int64_t n) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    z[k] = (double)vx[k] + (double)vd[k];
}

// PCG: p = z + beta_p p.  FCG: p = z - beta_p p.
__global__ void k_bp_update(double* __restrict__ p, const double* __restrict__ z, const double* __restrict__ beta,
                            const int32_t* __restrict__ rprob, int64_t n, int fcg) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    const double b = beta[rprob[k]];
    p[k] = fcg ? z[k] - b * p[k] : z[k] + b * p[k];
  }
}

// Lanczos helpers with per-row scalars: y += s_p x ;  y = x + s_p y
__global__ void k_baxpy(const double* __restrict__ s, const int32_t* __restrict__ rprob, const double* __restrict__ x,
                        double* __restrict__ y, int64_t n) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    y[k] += s[rprob[k]] * x[k];
}

__global__ void k_bxpay(const double* __restrict__ x, const double* __restrict__ s, const int32_t* __restrict__ rprob,
                        double* __restrict__ y, int64_t n) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    y[k] = x[k] + s[rprob[k]] * y[k];
}

__global__ void k_jacobi(const double* __restrict__ dinv, const double* __restrict__ x, double* __restrict__ y,
                         int64_t n) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    y[k] = dinv[k] * x[k];
}

}  // namespace r3mg
