// Coarsest level: blocked right-looking Cholesky A = L L^T, blocked inverse of L, and the
// symmetric inverse A^{-1} = L^{-T} L^{-1}, all on 32 x 32 FP64 tiles.  Every tile product
// runs on the FP64 tensor-core path (mma.sync m8n8k4 f64; B300's FP64 tensor rate is close
// to its FP64 FMA rate, measured 0.99 vs 1.13 TFLOP/s).  Matrices are row-major with
// leading dimension ncp (a multiple of 32); padding rows/columns hold the identity.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace r3mg {

constexpr int kTile = 32;
constexpr int kTS = 33;   // shared-memory row stride (doubles)

// C (32x32, per-warp fragments) += As . Bs^T with As[m][k], Bs[n][k] in shared memory.
// 8 warps: warp w owns rows 8*(w>>1)..+8, columns 16*(w&1)..+16 as two 8x8 accumulators.
__device__ __forceinline__ void tile_mma_nt(const double* As, const double* Bs, double (&c)[2][2]) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = 8 * (warp >> 1), n0 = 16 * (warp & 1);
  const int gr = lane >> 2, gc = lane & 3;
#pragma unroll
  for (int k0 = 0; k0 < kTile; k0 += 4) {
    const double a = As[(m0 + gr) * kTS + k0 + gc];
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      const double b = Bs[(n0 + 8 * t + gr) * kTS + k0 + gc];
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
                   : "+d"(c[t][0]), "+d"(c[t][1])
                   : "d"(a), "d"(b));
    }
  }
}

// Element (row, col) of the warp's accumulator c[t][u] inside the 32x32 tile.
__device__ __forceinline__ void frag_pos(int t, int u, int& row, int& col) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  row = 8 * (warp >> 1) + (lane >> 2);
  col = 16 * (warp & 1) + 8 * t + 2 * (lane & 3) + u;
}

// load a tile (bi, bj) of M into S; transposed if tr
__device__ __forceinline__ void load_tile(const double* M, int64_t ld, int bi, int bj, double* S, bool tr) {
  for (int t = threadIdx.x; t < kTile * kTile; t += blockDim.x) {
    const int r = t / kTile, c = t % kTile;
    const double v = M[(int64_t)(bi * kTile + r) * ld + bj * kTile + c];
    if (tr) S[c * kTS + r] = v; else S[r * kTS + c] = v;
  }
}

// Factor the diagonal tile k in place and store its triangular inverse in Dinv (32x32 at k).
__global__ void __launch_bounds__(256) k_potrf_diag(double* A, int64_t ld, int k, double* Linv, int* status) {
  __shared__ double S[kTile * kTS];
  __shared__ double X[kTile * kTS];
  __shared__ int bad;
  load_tile(A, ld, k, k, S, false);
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  for (int j = 0; j < kTile; ++j) {
    if (threadIdx.x == 0) {
      const double piv = S[j * kTS + j];
      if (!(piv > 0.0) || !isfinite(piv)) bad = 1;
      S[j * kTS + j] = sqrt(fmax(piv, 1e-300));
    }
    __syncthreads();
    for (int i = j + 1 + threadIdx.x; i < kTile; i += blockDim.x) S[i * kTS + j] /= S[j * kTS + j];
    __syncthreads();
    for (int t = threadIdx.x; t < kTile * kTile; t += blockDim.x) {
      const int i = t / kTile, c = t % kTile;
      if (c > j && i >= c) S[i * kTS + c] -= S[i * kTS + j] * S[c * kTS + j];
    }
    __syncthreads();
  }
  // inverse of the lower factor: column c solves L y = e_c by forward substitution
  if (threadIdx.x < kTile) {
    const int c = threadIdx.x;
    for (int i = 0; i < kTile; ++i) {
      double v = (i == c) ? 1.0 : 0.0;
      if (i >= c)
        for (int m = c; m < i; ++m) v -= S[i * kTS + m] * X[m * kTS + c];
      X[i * kTS + c] = (i >= c) ? v / S[i * kTS + i] : 0.0;
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < kTile * kTile; t += blockDim.x) {
    const int r = t / kTile, c = t % kTile;
    A[(int64_t)(k * kTile + r) * ld + k * kTile + c] = (c <= r) ? S[r * kTS + c] : 0.0;
    Linv[(int64_t)(k * kTile + r) * ld + k * kTile + c] = X[r * kTS + c];
  }
  if (threadIdx.x == 0 && bad) atomicExch(status, 1);
}

// Panel: L_ik = A_ik L_kk^{-T} for i = k+1+blockIdx.x.
__global__ void __launch_bounds__(256) k_trsm_panel(double* A, int64_t ld, int k, const double* Linv) {
  __shared__ double As[kTile * kTS];
  __shared__ double Bs[kTile * kTS];
  const int i = k + 1 + blockIdx.x;
  load_tile(A, ld, i, k, As, false);
  load_tile(Linv, ld, k, k, Bs, false);   // Bs[n][k'] = Linv_kk[n][k'] -> C = A_ik Linv_kk^T
  __syncthreads();
  double c[2][2] = {{0, 0}, {0, 0}};
  tile_mma_nt(As, Bs, c);
  for (int t = 0; t < 2; ++t)
    for (int u = 0; u < 2; ++u) {
      int r, col; frag_pos(t, u, r, col);
      A[(int64_t)(i * kTile + r) * ld + k * kTile + col] = c[t][u];
    }
}

// Trailing update A_ij -= L_ik L_jk^T for k < j <= i < nb (lower triangle of tiles).
__global__ void __launch_bounds__(256) k_syrk_update(double* A, int64_t ld, int k, int nb) {
  __shared__ double As[kTile * kTS];
  __shared__ double Bs[kTile * kTS];
  const int m = nb - k - 1;   // remaining tiles
  // blockIdx.x -> (ii, jj) with 0 <= jj <= ii < m
  int ii = (int)((sqrt(8.0 * blockIdx.x + 1.0) - 1.0) / 2.0);
  while ((ii + 1) * (ii + 2) / 2 <= (int)blockIdx.x) ++ii;
  while (ii * (ii + 1) / 2 > (int)blockIdx.x) --ii;
  const int jj = blockIdx.x - ii * (ii + 1) / 2;
  if (ii >= m) return;
  const int i = k + 1 + ii, j = k + 1 + jj;
  load_tile(A, ld, i, k, As, false);
  load_tile(A, ld, j, k, Bs, false);
  __syncthreads();
  double c[2][2] = {{0, 0}, {0, 0}};
  tile_mma_nt(As, Bs, c);
  for (int t = 0; t < 2; ++t)
    for (int u = 0; u < 2; ++u) {
      int r, col; frag_pos(t, u, r, col);
      A[(int64_t)(i * kTile + r) * ld + j * kTile + col] -= c[t][u];
    }
}

// Inverse of L, tile diagonal t: Linv_ij = -Linv_ii sum_{m=j}^{i-1} L_im Linv_mj, i = j + t.
__global__ void __launch_bounds__(256) k_trtri_step(const double* L, double* Linv, int64_t ld, int t, int nb) {
  __shared__ double As[kTile * kTS];
  __shared__ double Bs[kTile * kTS];
  const int j = blockIdx.x, i = j + t;
  if (i >= nb) return;
  double c[2][2] = {{0, 0}, {0, 0}};
  for (int m = j; m < i; ++m) {
    __syncthreads();
    load_tile(L, ld, i, m, As, false);
    load_tile(Linv, ld, m, j, Bs, true);     // Bs[n][k'] = Linv_mj[k'][n]
    __syncthreads();
    tile_mma_nt(As, Bs, c);
  }
  __syncthreads();
  // S -> Bs transposed: Bs[n][k'] = S[k'][n]
  for (int tt = 0; tt < 2; ++tt)
    for (int u = 0; u < 2; ++u) {
      int r, col; frag_pos(tt, u, r, col);
      Bs[col * kTS + r] = c[tt][u];
    }
  load_tile(Linv, ld, i, i, As, false);
  __syncthreads();
  double c2[2][2] = {{0, 0}, {0, 0}};
  tile_mma_nt(As, Bs, c2);
  for (int tt = 0; tt < 2; ++tt)
    for (int u = 0; u < 2; ++u) {
      int r, col; frag_pos(tt, u, r, col);
      Linv[(int64_t)(i * kTile + r) * ld + j * kTile + col] = -c2[tt][u];
    }
}

// Ainv_ij = sum_{m >= i} Linv_mi^T Linv_mj for j <= i; mirrored to (j, i).
__global__ void __launch_bounds__(256) k_lauum(const double* Linv, double* Ainv, int64_t ld, int nb) {
  __shared__ double As[kTile * kTS];
  __shared__ double Bs[kTile * kTS];
  int ii = (int)((sqrt(8.0 * blockIdx.x + 1.0) - 1.0) / 2.0);
  while ((ii + 1) * (ii + 2) / 2 <= (int)blockIdx.x) ++ii;
  while (ii * (ii + 1) / 2 > (int)blockIdx.x) --ii;
  const int jj = blockIdx.x - ii * (ii + 1) / 2;
  if (ii >= nb) return;
  double c[2][2] = {{0, 0}, {0, 0}};
  for (int m = ii; m < nb; ++m) {
    __syncthreads();
    load_tile(Linv, ld, m, ii, As, true);   // As[r][k'] = Linv_mi[k'][r]
    load_tile(Linv, ld, m, jj, Bs, true);   // Bs[n][k'] = Linv_mj[k'][n]
    __syncthreads();
    tile_mma_nt(As, Bs, c);
  }
  for (int t = 0; t < 2; ++t)
    for (int u = 0; u < 2; ++u) {
      int r, col; frag_pos(t, u, r, col);
      if (ii == jj && r < col) continue;   // diagonal tile: mirror the lower half only (deterministic)
      Ainv[(int64_t)(ii * kTile + r) * ld + jj * kTile + col] = c[t][u];
      Ainv[(int64_t)(jj * kTile + col) * ld + ii * kTile + r] = c[t][u];
    }
}


// ---------------------------------------------------------------- triangular solves
// The coarsest solve by forward and back substitution with the Cholesky factor (L y = r,
// L^T x = y), the textbook alternative to the explicit inverse.  A substitution is a chain of
// dependent 32-row blocks, so it runs in ONE CTA (1024 threads) with the solution vector in
// shared memory (n * sizeof(T) bytes of dynamic shared memory): per block, the warps form the
// rows' dot products with the solved part (coalesced along rows of L), then warp 0 solves the
// 32 x 32 diagonal block.  L: row-major, leading dimension ld, lower triangle.

template <typename T>
__device__ __forceinline__ T warp_allsum(T v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename T>
__global__ void __launch_bounds__(1024) k_trsv_lower(const T* __restrict__ L, int64_t ld, const T* __restrict__ r,
                                                     int n, T* __restrict__ y) {
  extern __shared__ __align__(16) unsigned char trsv_smem[];
  T* ys = reinterpret_cast<T*>(trsv_smem);
  __shared__ T blk[32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, NW = blockDim.x >> 5;
  for (int k0 = 0; k0 < n; k0 += 32) {
    const int nb = min(32, n - k0);
    for (int i = warp; i < nb; i += NW) {          // s_i = r_i - L[i, 0:k0] y[0:k0]
      const T* Lr = L + (int64_t)(k0 + i) * ld;
      T s = T(0);
      for (int j = lane; j < k0; j += 32) s += Lr[j] * ys[j];
      s = warp_allsum(s);
      if (lane == 0) blk[i] = r[k0 + i] - s;
    }
    __syncthreads();
    if (warp == 0) {                               // the diagonal block, column by column
      T v = lane < nb ? blk[lane] : T(0);
      for (int i = 0; i < nb; ++i) {
        const T yi = __shfl_sync(0xffffffffu, v, i) / L[(int64_t)(k0 + i) * ld + k0 + i];
        if (lane == i) v = yi;
        else if (lane > i && lane < nb) v -= L[(int64_t)(k0 + lane) * ld + k0 + i] * yi;
      }
      if (lane < nb) ys[k0 + lane] = v;
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) y[i] = ys[i];
}

template <typename T>
__global__ void __launch_bounds__(1024) k_trsv_lower_t(const T* __restrict__ L, int64_t ld, const T* __restrict__ y,
                                                       int n, T* __restrict__ x) {
  extern __shared__ __align__(16) unsigned char trsv_smem[];
  T* xs = reinterpret_cast<T*>(trsv_smem);
  __shared__ T part[32][33];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, NW = blockDim.x >> 5;
  const int nblk = (n + 31) / 32;
  for (int kb = nblk - 1; kb >= 0; --kb) {
    const int k0 = kb * 32, nb = min(32, n - k0), k1 = k0 + nb;
    // t_c = y_c - sum_{j >= k1} L[j, c] x_j for the block's columns c = k0 + lane:
    // rows j split over the warps, each warp reads 32 consecutive entries of a row
    T s = T(0);
    if (lane < nb)
      for (int j = k1 + warp; j < n; j += NW) s += L[(int64_t)j * ld + k0 + lane] * xs[j];
    if (warp < 32) part[warp][lane] = s;
    __syncthreads();
    if (warp == 0) {
      T t = T(0);
      for (int w = 0; w < min(NW, 32); ++w) t += part[w][lane];
      T v = lane < nb ? y[k0 + lane] - t : T(0);
      for (int i = nb - 1; i >= 0; --i) {       // the diagonal block, bottom row first
        const T xi = __shfl_sync(0xffffffffu, v, i) / L[(int64_t)(k0 + i) * ld + k0 + i];
        if (lane == i) v = xi;
        else if (lane < i) v -= L[(int64_t)(k0 + i) * ld + k0 + lane] * xi;
      }
      if (lane < nb) xs[k0 + lane] = v;
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) x[i] = xs[i];
}

}  // namespace r3mg
