// Krylov vector kernels: permutation to and from tree order, the CG / flexible-CG updates
// (FP64 vectors and scalars), V-cycle entry/exit conversions, deterministic reductions.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace r3mg {

enum Scal : int {
  S_PQ = 0, S_RR, S_RZ, S_RZNEW, S_ZQ, S_PR, S_ALPHA, S_BETA, S_BB, S_TMP,
  S_NA, S_NB,        // counts of recorded alphas / betas (condition estimate)
  S_THR,             // block solves: per-column stop threshold on ||r||^2
  S_COUNT = 16
};
// CG coefficients kept per solve for the condition estimate (the Lanczos tridiagonal of the
// iteration, Section 6's "condition number estimated by PCG"): the first kHist alphas and betas.
constexpr int kHist = 1024;
// single-vector scalar array: S_COUNT slots, then the alpha history, then the beta history
constexpr int kScalTotal = S_COUNT + 2 * kHist;
enum Fin : int { FIN_NONE = 0, FIN_ALPHA_PCG, FIN_ALPHA_FCG, FIN_BETA_PCG, FIN_BETA_FCG };

constexpr int kVecBlocks = 148 * 4;   // grid of the vector kernels (4 CTAs per SM)
constexpr int kVecThreads = 256;

template <typename S, typename D>
__global__ void k_gather_perm(const S* __restrict__ src, const int64_t* __restrict__ perm, D* __restrict__ dst, int64_t n) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    dst[k] = (D)src[perm ? perm[k] : k];   // null perm: identity (coarse-level numbering)
}

template <typename S, typename D>
__global__ void k_scatter_perm(const S* __restrict__ src, const int64_t* __restrict__ perm, D* __restrict__ dst, int64_t n) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    dst[perm ? perm[k] : k] = (D)src[k];
}

__device__ __forceinline__ void store_partial(double v, double* part) {
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) red[w] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += red[k];
    part[blockIdx.x] = s;
  }
}

// r = b - y, partial ||r||^2, and (optionally) ||b||^2 into part2.
__global__ void k_residual(const double* __restrict__ b, const double* __restrict__ y, double* __restrict__ r,
                           int64_t n, double* part, double* part2) {
  double s = 0.0, s2 = 0.0;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    const double v = b[k] - y[k];
    r[k] = v;
    s += v * v;
    s2 += b[k] * b[k];
  }
  store_partial(s, part);
  if (part2) { __syncthreads(); store_partial(s2, part2); }
}

// V-cycle entry on level 0: vr = r, vx = 0, vd = c0 dinv r (first Chebyshev update).
template <typename T>
__device__ __forceinline__ void vc_init_row(int64_t k, double rk, T* vr, T* vx, T* vd, const T* dinv, T c0) {
  const T rt = (T)rk;
  vr[k] = rt;
  vx[k] = T(0);
  vd[k] = c0 * dinv[k] * rt;
}

template <typename T>
__global__ void k_vc_init(const double* __restrict__ r, int64_t n, T* vr, T* vx, T* vd, const T* __restrict__ dinv, T c0) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    vc_init_row(k, r[k], vr, vx, vd, dinv, c0);
}

// x += alpha p; r -= alpha q; partial ||r||^2; V-cycle entry from the new r.
template <typename T>
__global__ void k_cg_update(double* __restrict__ x, double* __restrict__ r, const double* __restrict__ p,
                            const double* __restrict__ q, const double* __restrict__ scal, int64_t n, double* part,
                            T* vr, T* vx, T* vd, const T* __restrict__ dinv, T c0) {
  const double alpha = scal[S_ALPHA];
  double s = 0.0;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    x[k] += alpha * p[k];
    const double rk = r[k] - alpha * q[k];
    r[k] = rk;
    s += rk * rk;
    vc_init_row(k, rk, vr, vx, vd, dinv, c0);
  }
  store_partial(s, part);
}

// z = vx + vd (final Chebyshev update of level 0); partial z . w.
template <typename T>
__global__ void k_vc_final_dot(const T* __restrict__ vx, const T* __restrict__ vd, double* __restrict__ z,
                               const double* __restrict__ w, int64_t n, double* part) {
  double s = 0.0;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    const double zk = (double)vx[k] + (double)vd[k];
    z[k] = zk;
    if (w) s += zk * w[k];
  }
  if (part) store_partial(s, part);
}

// PCG: p = z + beta p.  FCG: p = z - beta p and partial p . r (next alpha's numerator).
__global__ void k_p_update(double* __restrict__ p, const double* __restrict__ z, const double* __restrict__ r,
                           const double* __restrict__ scal, int64_t n, int fcg, double* part) {
  const double beta = scal[S_BETA];
  double s = 0.0;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    const double pk = fcg ? z[k] - beta * p[k] : z[k] + beta * p[k];
    p[k] = pk;
    s += pk * r[k];
  }
  if (part) store_partial(s, part);
}

// Deterministic single-CTA sum of `m` partials into scal[slot], then the scalar finish step.
__global__ void k_reduce(const double* __restrict__ part, int m, double* scal, int slot, int fin, int* status) {
  __shared__ double red[32];
  double s = 0.0;
  for (int k = threadIdx.x; k < m; k += blockDim.x) s += part[k];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[k];
    scal[slot] = t;
    // alpha and beta of every iteration also go to the history (the flexible-CG beta with its
    // sign flipped: with a fixed SPD preconditioner it is minus the PCG beta)
    if (fin == FIN_ALPHA_PCG || fin == FIN_ALPHA_FCG) {
      const double num = (fin == FIN_ALPHA_PCG) ? scal[S_RZ] : scal[S_PR];
      if (!(t > 0.0) || !isfinite(num)) { if (status) atomicExch(status, 1); scal[S_ALPHA] = 0.0; }
      else {
        const double a = num / t;
        scal[S_ALPHA] = a;
        const int ia = (int)scal[S_NA];
        if (ia < kHist) scal[S_COUNT + ia] = a;
        scal[S_NA] = (double)(ia + 1);
      }
    } else if (fin == FIN_BETA_PCG || fin == FIN_BETA_FCG) {
      const double be = (fin == FIN_BETA_PCG) ? t / scal[S_RZ] : t / scal[S_PQ];
      scal[S_BETA] = be;
      if (fin == FIN_BETA_PCG) scal[S_RZ] = t;
      const int ib = (int)scal[S_NB];
      if (ib < kHist) scal[S_COUNT + kHist + ib] = (fin == FIN_BETA_PCG) ? be : -be;
      scal[S_NB] = (double)(ib + 1);
    }
  }
}

// *flag = 1 if any entry of x is nonzero (a zero initial guess lets the solver skip A x0).
__global__ void k_any_nonzero(const double* __restrict__ x, int64_t n, int* __restrict__ flag) {
  bool any = false;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    any = any || (x[k] != 0.0);
  if (__any_sync(0xffffffffu, any) && (threadIdx.x & 31) == 0) atomicOr(flag, 1);
}

// y = dinv * x (Jacobi) for the Lanczos estimate; partial x . y.
__global__ void k_jacobi_dot(const double* __restrict__ dinv, const double* __restrict__ x, double* __restrict__ y,
                             int64_t n, double* part) {
  double s = 0.0;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    const double v = dinv[k] * x[k];
    y[k] = v;
    s += v * x[k];
  }
  store_partial(s, part);
}

// y = x + a * y
__global__ void k_xpay(const double* __restrict__ x, double a, double* __restrict__ y, int64_t n) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    y[k] = x[k] + a * y[k];
}

// y += a * x
__global__ void k_axpy(double a, const double* __restrict__ x, double* __restrict__ y, int64_t n) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    y[k] += a * x[k];
}

// Loop state of the single-problem solve graph: lp[0] = threshold on ||r||^2, lp[1] = iteration budget.
__global__ void k_loop_init(double* __restrict__ lp, int* __restrict__ its, int* __restrict__ status,
                            double thr2, int budget) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    lp[0] = thr2;
    lp[1] = (double)budget;
    *its = 0;
    *status = 0;
  }
}

// Device-side stop test after the x/r update of one iteration: count it, then continue the loop
// (and run this iteration's V-cycle and direction update) only while ||r||^2 > the threshold,
// the budget is not spent and no breakdown was flagged.
__global__ void k_converge1(const double* __restrict__ scal, const double* __restrict__ lp, int* __restrict__ its,
                            const int* __restrict__ status, cudaGraphConditionalHandle loop,
                            cudaGraphConditionalHandle rest) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    const int k = *its + 1;
    *its = k;
    const double rr = scal[S_RR];
    const bool go = isfinite(rr) && rr > lp[0] && (double)k < lp[1] && *status == 0;
    cudaGraphSetConditional(loop, go ? 1u : 0u);
    cudaGraphSetConditional(rest, go ? 1u : 0u);
  }
}

// Sampled outer product on the stored pattern of A (the adjoint's matrix gradient):
// out[k] = alpha * lam[i] * u[col[k]] for every entry k of row i, in the caller's CSR order.
// One warp per row; the row's values are read once, u is gathered from L2.
__global__ void k_sampled_outer(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                const double* __restrict__ lam, const double* __restrict__ u, double alpha,
                                double* __restrict__ out, int64_t n) {
  const int lane = threadIdx.x & 31;
  const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = w; i < n; i += nw) {
    const double li = alpha * lam[i];
    for (int64_t k = rowptr[i] + lane; k < rowptr[i + 1]; k += 32) out[k] = li * u[col[k]];
  }
}

}  // namespace r3mg
