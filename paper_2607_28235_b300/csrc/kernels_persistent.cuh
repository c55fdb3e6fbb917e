// Persistent batched solve: every problem of a batched hierarchy advances through the whole
// FCG / PCG iteration inside ONE cooperative launch.  The CTAs (all co-resident) walk the
// phases of an iteration -- each Chebyshev step of each level, the transfers, the coarsest
// block solve, the per-problem dots and scalars, the CG product and update, the stop test --
// with a bounded grid barrier between phases, and skip the work of problems that have
// stopped.  The phase bodies are the same device code the per-step kernels run, in the same
// order of rounding, so every problem's iterates equal those of the graph-of-kernels loop.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "kernels_batch.cuh"
#include "kernels_krylov.cuh"
#include "kernels_level.cuh"
#include "kernels_vcycle.cuh"

namespace r3mg {

constexpr int kPMaxLevels = 8;
constexpr int kPThreads = 256;

// Bounded grid barrier of a cooperative launch: arrival counter and generation word in global
// memory.  A wait that runs past `limit` clock64 cycles raises *err and returns false (the
// kernel then leaves; a barrier never waits on a CTA that is not resident, since a cooperative
// launch places every CTA at once).  `skip` withholds this CTA's arrival (test of the expiry
// path).
struct GridBar {
  unsigned* count;
  unsigned* gen;
  int* err;
  long long limit;
  int withhold;   // 1: CTA 0 does not arrive at the first barrier (expiry-path test)
};

__device__ __forceinline__ bool grid_barrier(const GridBar& gb, bool skip_arrive) {
  __shared__ int ok_s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    volatile unsigned* genp = gb.gen;
    const unsigned g = *genp;                     // the generation this barrier waits to leave
    __threadfence();                              // the CTA's writes before its arrival
    if (!skip_arrive) {
      if (atomicAdd(gb.count, 1u) == gridDim.x - 1) {
        *gb.count = 0u;                           // last arrival: reset, then release
        __threadfence();
        atomicAdd(gb.gen, 1u);
      }
    }
    const long long t0 = clock64();
    while (*genp == g) {
      if (clock64() - t0 > gb.limit) { atomicExch(gb.err, 1); ok = 0; break; }
    }
    __threadfence();                              // acquire: the other CTAs' writes
    ok_s = ok;
  }
  __syncthreads();
  return ok_s != 0;
}

// Everything one persistent batched solve reads and writes.  Level vectors and values are in
// the V-cycle precision T; the Krylov vectors and scalars are FP64.
template <typename T>
struct PBatchArgs {
  int L, np, fcg, b, fan, maxit;
  int64_t n;                                   // fine rows (all problems)
  double rtol2;
  LevelView<T> lv[kPMaxLevels];
  int G[kPMaxLevels];                          // lanes per row of each level's step
  T* x[kPMaxLevels];
  T* r[kPMaxLevels];
  T* d[kPMaxLevels][2];
  const T* dinv[kPMaxLevels];
  const T* P[kPMaxLevels];                     // transfer from level l+1 to level l
  const int32_t* rprob[kPMaxLevels];
  const double *preA[kPMaxLevels], *preC[kPMaxLevels], *postA[kPMaxLevels], *postC[kPMaxLevels];
  const double* c0[kPMaxLevels];
  int npre[kPMaxLevels], npost[kPMaxLevels];
  const int32_t* box_of_tree;                  // fine row -> level-1 box
  // coarsest block solve
  const T* Ainv;
  const int64_t *moff, *mld, *cof;
  // fine FP64 product of the CG iteration
  LevelView<double> f64;
  int G64;
  double *cx, *cr, *cp, *cq, *cz;
  BatchScal S;
  const int64_t *sb, *se;                      // fine-level dot segments
  const int* soff;
  int nseg;
  double* seg_part;
  int* any_count;                              // per iteration: problems still running
  GridBar bar;
};

// a level step or product on the boxes of the running problems
template <typename T, int G, bool FINE, class Ep>
__device__ void p_level(const LevelView<T>& L, const T* xin, const Ep& ep, const int32_t* rprob, const int* active,
                        unsigned char* smem) {
  const LevelSmem lay(sizeof(T), L.win_max, L.max_box_rows);
  double acc = 0.0;
  for (int64_t B = blockIdx.x; B < L.nbox; B += gridDim.x) {
    const int64_t r0 = FINE ? L.box_row[B] : B * L.b;
    if (!active[rprob[r0]]) continue;          // uniform across the CTA
    level_stage<T, FINE, Ep>(L, xin, ep, lay, B, smem);
    cp_async_wait_all();
    __syncthreads();
    level_compute<T, G, FINE, Ep, (sizeof(T) == 4 ? 4 : 2), false>(L, ep, lay, B, smem, acc);
    __syncthreads();
  }
}

template <typename T, bool FINE, class Ep>
__device__ void p_level_g(int G, const LevelView<T>& L, const T* xin, const Ep& ep, const int32_t* rprob,
                          const int* active, unsigned char* smem) {
  switch (G) {
    case 4: p_level<T, 4, FINE, Ep>(L, xin, ep, rprob, active, smem); break;
    case 8: p_level<T, 8, FINE, Ep>(L, xin, ep, rprob, active, smem); break;
    case 16: p_level<T, 16, FINE, Ep>(L, xin, ep, rprob, active, smem); break;
    default: p_level<T, 32, FINE, Ep>(L, xin, ep, rprob, active, smem); break;
  }
}

// Per-problem dot of the fine FP64 vectors x . y (y null: x . x) into out[p] for every running
// problem: segment partials (the segments of k_seg_dot), a barrier, each problem's partials summed
// in order (k_seg_reduce's order), then the scalar finish `fin` of k_bscal (beta), or none (-1).
template <typename T>
__device__ bool p_dot(const PBatchArgs<T>& A, const double* x, const double* y, double* out, int fin) {
  __shared__ double red[32];
  const int* act = A.S.active;
  for (int s = blockIdx.x; s < A.nseg; s += gridDim.x) {
    if (!act[A.rprob[0][A.sb[s]]]) continue;     // uniform across the CTA
    double acc = 0.0;
    for (int64_t k = A.sb[s] + threadIdx.x; k < A.se[s]; k += blockDim.x) acc += x[k] * (y ? y[k] : x[k]);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[k];
      A.seg_part[s] = t;
    }
    __syncthreads();
  }
  if (!grid_barrier(A.bar, false)) return false;
  const BatchScal& S = A.S;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < A.np; p += gridDim.x * blockDim.x) {
    if (!act[p]) continue;
    double t = 0.0;
    for (int s = A.soff[p]; s < A.soff[p + 1]; ++s) t += A.seg_part[s];
    out[p] = t;
    if (fin == BF_BETA_PCG) {
      S.beta[p] = S.rzn[p] / S.rz[p];
      S.rz[p] = S.rzn[p];
    } else if (fin == BF_BETA_FCG) {
      S.beta[p] = S.zq[p] / S.pq[p];
    }
  }
  return grid_barrier(A.bar, false);
}

template <typename T>
__global__ void __launch_bounds__(kPThreads) k_batch_persistent(PBatchArgs<T> A) {
  extern __shared__ __align__(16) unsigned char psmem[];
  const int* act = A.S.active;
  const int64_t gt = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, gs = (int64_t)gridDim.x * blockDim.x;
  const int L = A.L;
  auto sync = [&](bool first = false) {
    return grid_barrier(A.bar, first && A.bar.withhold && blockIdx.x == 0);
  };
  bool first = true;
  for (int it = 0; it < A.maxit; ++it) {
    // ---------------- V-cycle (the per-step kernels' order: pre steps, restriction, coarsest,
    // prolongation, post steps), entered with level 0's x = 0, r = r_k, d = c0 D^-1 r_k
    int cur[kPMaxLevels];
    for (int l = 0; l < L; ++l) cur[l] = 0;
    for (int l = 0; l + 1 < L; ++l) {
      for (int st = 0; st < A.npre[l]; ++st) {
        T* d = A.d[l][cur[l]];
        T* dn = A.d[l][cur[l] ^ 1];
        TEpChebB<T> ep{A.x[l], A.r[l], d, dn, A.dinv[l], A.preA[l] + (int64_t)st * A.np, A.preC[l] + (int64_t)st * A.np,
                       A.rprob[l]};
        if (l == 0) p_level_g<T, true>(A.G[l], A.lv[l], d, ep, A.rprob[l], act, psmem);
        else p_level_g<T, false>(A.G[l], A.lv[l], d, ep, A.rprob[l], act, psmem);
        cur[l] ^= 1;
        if (!sync(first)) return;
        first = false;
      }
      const bool coarsest = (l + 2 == L);
      NextInitB<T> nx{A.r[l + 1], coarsest ? nullptr : A.x[l + 1], coarsest ? nullptr : A.d[l + 1][0], A.dinv[l + 1],
                      A.c0[l + 1], A.rprob[l + 1]};
      const int64_t nbox1 = A.lv[l + 1].nrows / A.b;
      if (l == 0) restrict_fine_body<T>(A.P[0], A.r[0], A.lv[0].box_row, nbox1, A.b, nx, A.rprob[1], act);
      else restrict_coarse_body<T>(A.P[l], A.r[l], nbox1, A.b, A.fan, nx, gt, gs, A.rprob[l + 1], act);
      if (!sync()) return;
    }
    {
      const int lc = L - 1;
      block_gemv_body<T>(A.Ainv, A.moff, A.mld, A.cof, A.rprob[lc], A.r[lc], A.lv[lc].nrows, A.x[lc], act);
      if (!sync()) return;
    }
    for (int l = L - 2; l >= 0; --l) {
      const bool coarsest = (l + 2 == L);
      const T* x1 = A.x[l + 1];
      const T* d1 = coarsest ? nullptr : A.d[l + 1][cur[l + 1]];
      T* d = A.d[l][cur[l]];
      if (l == 0) prolong_fine_body<T>(A.P[0], A.box_of_tree, x1, d1, A.n, A.b, d, gt, gs, A.rprob[0], act);
      else prolong_coarse_body<T>(A.P[l], x1, d1, A.lv[l].nrows / A.b, A.b, A.fan, d, gt, gs, A.rprob[l], act);
      if (!sync()) return;
      for (int st = 0; st < A.npost[l]; ++st) {
        T* dd = A.d[l][cur[l]];
        T* dn = A.d[l][cur[l] ^ 1];
        TEpChebB<T> ep{A.x[l], A.r[l], dd, dn, A.dinv[l], A.postA[l] + (int64_t)st * A.np,
                       A.postC[l] + (int64_t)st * A.np, A.rprob[l]};
        if (l == 0) p_level_g<T, true>(A.G[l], A.lv[l], dd, ep, A.rprob[l], act, psmem);
        else p_level_g<T, false>(A.G[l], A.lv[l], dd, ep, A.rprob[l], act, psmem);
        cur[l] ^= 1;
        if (!sync()) return;
      }
    }
    // ---------------- z = x0 + d0; beta; new direction; A p; alpha; update; ||r||; stop test
    const T* vx = A.x[0];
    const T* vd = A.d[0][cur[0]];
    for (int64_t k = gt; k < A.n; k += gs)
      if (act[A.rprob[0][k]]) A.cz[k] = (double)vx[k] + (double)vd[k];
    if (!sync()) return;
    if (A.fcg) { if (!p_dot(A, A.cz, A.cq, A.S.zq, BF_BETA_FCG)) return; }
    else { if (!p_dot(A, A.cz, A.cr, A.S.rzn, BF_BETA_PCG)) return; }
    for (int64_t k = gt; k < A.n; k += gs) {
      const int p = A.rprob[0][k];
      if (!act[p]) continue;
      const double bt = A.S.beta[p];
      A.cp[k] = A.fcg ? A.cz[k] - bt * A.cp[k] : A.cz[k] + bt * A.cp[k];
    }
    if (!sync()) return;
    {
      TEpApplyDot<double> ep{A.cq, nullptr};
      p_level_g<double, true>(A.G64, A.f64, A.cp, ep, A.rprob[0], act, psmem);
      if (!sync()) return;
    }
    if (!p_dot(A, A.cp, A.cq, A.S.pq, -1)) return;
    if (A.fcg) { if (!p_dot(A, A.cp, A.cr, A.S.pr, -1)) return; }
    // alpha of every running problem (breakdown deactivates the problem and raises err)
    for (int p = (int)gt; p < A.np; p += (int)gs) {
      const BatchScal& S = A.S;
      if (!S.active[p]) { S.alpha[p] = 0.0; continue; }
      const double num = A.fcg ? S.pr[p] : S.rz[p];
      const double pq = S.pq[p];
      if (!(pq > 0.0) || !isfinite(num)) { S.alpha[p] = 0.0; S.active[p] = 0; atomicExch(S.err, 1); continue; }
      S.alpha[p] = num / pq;
    }
    if (!sync()) return;
    for (int64_t k = gt; k < A.n; k += gs) {
      const int pp = A.rprob[0][k];
      if (!act[pp]) continue;
      const double a = A.S.alpha[pp];
      A.cx[k] += a * A.cp[k];
      const double rk = A.cr[k] - a * A.cq[k];
      A.cr[k] = rk;
      const T rt = (T)rk;
      A.r[0][k] = rt;
      A.x[0][k] = T(0);
      A.d[0][0][k] = (T)A.c0[0][pp] * A.dinv[0][k] * rt;
    }
    if (!sync()) return;
    if (!p_dot(A, A.cr, nullptr, A.S.rr, -1)) return;
    for (int p = (int)gt; p < A.np; p += (int)gs) {
      const BatchScal& S = A.S;
      if (S.active[p]) {
        S.its[p] += 1;
        if (S.rr[p] <= A.rtol2 * S.bb[p] || S.its[p] >= A.maxit) S.active[p] = 0;
      }
      if (S.active[p]) atomicAdd(&A.any_count[it], 1);
    }
    if (!sync()) return;
    if (*(volatile int*)&A.any_count[it] == 0) return;
  }
}

}  // namespace r3mg
