// Several right-hand sides on one hierarchy (block vectors).  Every level vector holds M
// columns row-interleaved: row i keeps its M values contiguous (i*M + c), so one matrix entry,
// read once from HBM, multiplies M gathered values that sit in one or two 32-byte sectors.
// The level operators, the transfers P / P^T, the coarsest solve and the CG updates below are
// the single-vector kernels' arithmetic (Sections 3-4, Chebyshev-Jacobi smoothing, PCG/FCG)
// applied column by column; only the data layout and the thread mapping differ.
#pragma once
#include <algorithm>
#include <cstdint>
#include <cuda_runtime.h>

#include "kernels_level.cuh"
#include "kernels_level_tma.cuh"
#include "kernels_krylov.cuh"

namespace r3mg {

// 16-byte column slice of one row: 4 floats or 2 doubles
template <typename T>
struct Slice {
  static constexpr int V = 16 / (int)sizeof(T);
  T v[V];
  __device__ __forceinline__ void ldg(const T* p) {   // read-only path (gathered operands)
    if constexpr (sizeof(T) == 4) {
      const float4 a = __ldg(reinterpret_cast<const float4*>(p));
      v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    } else {
      const double2 a = __ldg(reinterpret_cast<const double2*>(p));
      v[0] = a.x; v[1] = a.y;
    }
  }
  __device__ __forceinline__ void ld(const T* p) {
    if constexpr (sizeof(T) == 4) {
      const float4 a = *reinterpret_cast<const float4*>(p);
      v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    } else {
      const double2 a = *reinterpret_cast<const double2*>(p);
      v[0] = a.x; v[1] = a.y;
    }
  }
  __device__ __forceinline__ void st(T* p) const {
    if constexpr (sizeof(T) == 4) *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
    else *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
  }
};

// ---------------------------------------------------------------- level operators
// Epilogues get the row, the first column of the lane's slice, the slice of (A X)_row and the
// lane's per-column dot partials.

template <typename T, int M>
struct MEpApply {   // Y = A X, and per-column partials of W . Y when W is given
  T* y; const T* w;
  static constexpr bool kDot = true;
  __device__ void post(int64_t row, int c0, const Slice<T>& a, double (&dacc)[Slice<T>::V]) const {
    a.st(y + row * M + c0);
    if (w) {
      Slice<T> ws;
      ws.ld(w + row * M + c0);
#pragma unroll
      for (int v = 0; v < Slice<T>::V; ++v) dacc[v] += (double)ws.v[v] * (double)a.v[v];
    }
  }
  __device__ void post1(int64_t row, int col, T a, double& dacc) const {
    y[row * M + col] = a;
    if (w) dacc += (double)w[row * M + col] * (double)a;
  }
};

// One Chebyshev-Jacobi step per column (the input block is the current update D):
// X += D;  R -= A D;  D' = a D + c dinv R.
template <typename T, int M>
struct MEpCheb {
  T* x; T* r; const T* d; T* dnext; const T* dinv; T a, c;
  static constexpr bool kDot = false;
  __device__ void post(int64_t row, int c0, const Slice<T>& ad, double (&)[Slice<T>::V]) const {
    const int64_t o = row * M + c0;
    Slice<T> xs, rs, ds;
    xs.ld(x + o); rs.ld(r + o); ds.ld(d + o);
    const T di = dinv[row];
#pragma unroll
    for (int v = 0; v < Slice<T>::V; ++v) {
      xs.v[v] += ds.v[v];
      rs.v[v] -= ad.v[v];
      ds.v[v] = a * ds.v[v] + c * di * rs.v[v];
    }
    xs.st(x + o); rs.st(r + o); ds.st(dnext + o);
  }
  __device__ void post1(int64_t row, int col, T ad, double&) const {
    const int64_t o = row * M + col;
    const T di = d[o];
    x[o] += di;
    const T rn = r[o] - ad;
    r[o] = rn;
    dnext[o] = a * di + c * dinv[row] * rn;
  }
};

// Level operator on M columns.  One CTA per box (grid-stride).  The box's window map (window
// position -> row of the level, the same windows the single-vector kernel stages) is built in
// shared memory; each row is taken by CL*S lanes: CL lanes cover the M columns with 16-byte
// slices, S lanes split the row's entries in groups of four.  Entry values and indices are
// read once per lane group (the CL lanes of a slot read the same address), the gathered rows
// of X come through the read-only L1 path.
template <typename T, int M, int S, bool FINE, class Ep>
__global__ void __launch_bounds__(256) k_mr_level(LevelView<T> L, const T* __restrict__ xin, Ep ep,
                                                  double* __restrict__ part) {
  constexpr int V = Slice<T>::V, CL = M / V, LPR = CL * S, RPW = 32 / LPR;
  static_assert(M % V == 0 && 32 % LPR == 0, "lane layout");
  extern __shared__ __align__(16) int32_t smap[];
  __shared__ double red[8][M];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, NW = blockDim.x >> 5;
  const int cl = lane % CL, s = (lane / CL) % S, rw = lane / LPR;
  double dacc[V];
#pragma unroll
  for (int v = 0; v < V; ++v) dacc[v] = 0.0;
  for (int64_t B = blockIdx.x; B < L.nbox; B += gridDim.x) {
    const int64_t e0 = L.nbr_ptr[B];
    const int nn = (int)(L.nbr_ptr[B + 1] - e0);
    int W;
    int64_t r0, r1;
    if constexpr (FINE) {
      W = L.win_size[B];
      for (int q = warp; q < nn; q += NW) {
        const int wo = L.win_off[e0 + q];
        const int64_t src = L.slot_src[e0 + q];
        const int len = (q + 1 < nn ? L.win_off[e0 + q + 1] : W) - wo;
        for (int t = lane; t < len; t += 32) smap[wo + t] = (int32_t)(src + t);
      }
      r0 = L.box_row[B]; r1 = L.box_row[B + 1];
    } else {
      const int b = L.b;
      W = nn * b;
      for (int t = threadIdx.x; t < W; t += blockDim.x) smap[t] = (int32_t)(L.nbr[e0 + t / b] * b + t % b);
      r0 = B * b; r1 = r0 + b;
    }
    // padding entries (zero values) point at row 0
    for (int t = W + threadIdx.x; t < ((W + 3) & ~3); t += blockDim.x) smap[t] = 0;
    __syncthreads();
    // warp-uniform trip count: the slot shuffles below see the whole warp
    for (int64_t base = r0 + (int64_t)warp * RPW; base < r1; base += (int64_t)NW * RPW) {
      const int64_t row = base + rw;
      const bool ok = row < r1;
      int64_t k0 = 0, k1 = 0;
      if (ok) { k0 = L.row_ptr[row]; k1 = L.row_ptr[row + 1]; }
      Slice<T> acc;
#pragma unroll
      for (int v = 0; v < V; ++v) acc.v[v] = T(0);
      for (int64_t k = k0 + 4 * s; k < k1; k += 4 * S) {
        T a[4];
        int ii[4];
        Vec4<T>::load(L.vals + k, a);
        if constexpr (FINE) load_idx4(L.idx + k, ii);
        else { const int t = (int)(k - k0); ii[0] = t; ii[1] = t + 1; ii[2] = t + 2; ii[3] = t + 3; }
        Slice<T> xv[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) xv[e].ldg(xin + (int64_t)smap[ii[e]] * M + cl * V);
#pragma unroll
        for (int e = 0; e < 4; ++e)
#pragma unroll
          for (int v = 0; v < V; ++v) acc.v[v] += a[e] * xv[e].v[v];
      }
#pragma unroll
      for (int o = CL; o < LPR; o <<= 1)
#pragma unroll
        for (int v = 0; v < V; ++v) acc.v[v] += __shfl_xor_sync(0xffffffffu, acc.v[v], o);
      if (ok && s == 0) ep.post(row, cl * V, acc, dacc);
    }
    __syncthreads();
  }
  if constexpr (Ep::kDot) {
    if (part != nullptr) {
      // fold the lanes of equal column slice, then the warps in a fixed order
#pragma unroll
      for (int o = CL; o < 32; o <<= 1)
#pragma unroll
        for (int v = 0; v < V; ++v) dacc[v] += __shfl_xor_sync(0xffffffffu, dacc[v], o);
      if (lane < CL)
#pragma unroll
        for (int v = 0; v < V; ++v) red[warp][lane * V + v] = dacc[v];
      __syncthreads();
      if (threadIdx.x < M) {
        double t = 0.0;
        for (int w = 0; w < NW; ++w) t += red[w][threadIdx.x];
        part[(int64_t)blockIdx.x * M + threadIdx.x] = t;
      }
    }
  }
}

// Coarse-level operator on M columns with the box's window staged in shared memory.  Every
// row of a box multiplies the same window (its neighbour boxes' rows, nn*b of them), so the
// window's M columns are copied once per box (cp.async, 16-byte pieces) and each staged slice
// feeds R rows held by one lane.  Lanes: ceil(b/R) row groups x CL column slices; the 8 warps
// split the window's entries in groups of four and meet in shared memory for the sum.
template <typename T, int M, int R, class Ep>
__global__ void __launch_bounds__(256) k_mr_coarse(LevelView<T> L, const T* __restrict__ xin, Ep ep,
                                                   double* __restrict__ part) {
  constexpr int V = Slice<T>::V, CL = M / V;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* xs = reinterpret_cast<T*>(smem_raw);                       // [Wpad][M]
  const int b = L.b;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, NW = blockDim.x >> 5;
  const int cl = lane % CL, rg = lane / CL;
  const int ngroups = (b + R - 1) / R;
  T* red = xs;                         // [NW][b][M] partial sums, over the window once it is consumed
  double dacc = 0.0;
  for (int64_t B = blockIdx.x; B < L.nbox; B += gridDim.x) {
    const int64_t e0 = L.nbr_ptr[B];
    const int nn = (int)(L.nbr_ptr[B + 1] - e0);
    const int W = nn * b, Wp = (W + 3) & ~3;
    // stage the window: row w of the window is level row nbr[e0 + w / b] * b + w % b
    constexpr int PPR = M * (int)sizeof(T) / 16;                // 16-byte pieces per row
    for (int t = threadIdx.x; t < W * PPR; t += blockDim.x) {
      const int w = t / PPR, pc = t % PPR;
      const int64_t src = (L.nbr[e0 + w / b] * b + w % b) * M + pc * (16 / (int)sizeof(T));
      const unsigned d = (unsigned)__cvta_generic_to_shared(xs + (size_t)w * M + pc * (16 / (int)sizeof(T)));
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(xin + src));
    }
    for (int t = W * M + threadIdx.x; t < Wp * M; t += blockDim.x) xs[t] = T(0);
    cp_async_wait_all();
    __syncthreads();
    const int64_t r0 = B * b;
    const int64_t kbase = L.row_ptr[r0];                          // rows of a box: equal length Wp
    T acc[R][V];
#pragma unroll
    for (int i = 0; i < R; ++i)
#pragma unroll
      for (int v = 0; v < V; ++v) acc[i][v] = T(0);
    if (rg < ngroups) {
      for (int g = warp; g * 4 < Wp; g += NW) {
        const int w0 = g * 4;
        Slice<T> xv[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const T* p = xs + (size_t)(w0 + e) * M + cl * V;
          if constexpr (sizeof(T) == 4) {
            const float4 a = *reinterpret_cast<const float4*>(p);
            xv[e].v[0] = a.x; xv[e].v[1] = a.y; xv[e].v[2] = a.z; xv[e].v[3] = a.w;
          } else {
            const double2 a = *reinterpret_cast<const double2*>(p);
            xv[e].v[0] = a.x; xv[e].v[1] = a.y;
          }
        }
#pragma unroll
        for (int i = 0; i < R; ++i) {
          const int row = rg * R + i;
          if (row < b) {
            T a[4];
            Vec4<T>::load(L.vals + kbase + (int64_t)row * Wp + w0, a);
#pragma unroll
            for (int e = 0; e < 4; ++e)
#pragma unroll
              for (int v = 0; v < V; ++v) acc[i][v] += a[e] * xv[e].v[v];
          }
        }
      }
    }
    __syncthreads();   // window reads done: the partial-sum area may follow
    if (rg < ngroups) {
#pragma unroll
      for (int i = 0; i < R; ++i) {
        const int row = rg * R + i;
        if (row < b)
#pragma unroll
          for (int v = 0; v < V; ++v) red[((size_t)warp * b + row) * M + cl * V + v] = acc[i][v];
      }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < b * M; t += blockDim.x) {
      T s = T(0);
      for (int w = 0; w < NW; ++w) s += red[(size_t)w * b * M + t];
      ep.post1(r0 + t / M, t % M, s, dacc);
    }
    __syncthreads();
  }
  if constexpr (Ep::kDot) {
    if (part != nullptr) {
      // thread t always finishes elements of column t % M (blockDim is a multiple of M)
      __shared__ double redd[8][M];
      for (int o = M; o < 32; o <<= 1) dacc += __shfl_xor_sync(0xffffffffu, dacc, o);
      if (lane < M) redd[warp][lane] = dacc;
      __syncthreads();
      if (threadIdx.x < M) {
        double t = 0.0;
        for (int w = 0; w < NW; ++w) t += redd[w][threadIdx.x];
        part[(int64_t)blockIdx.x * M + threadIdx.x] = t;
      }
    }
  }
}

template <typename T, int M>
inline size_t mr_coarse_smem(const LevelView<T>& L) {   // staged window, later the per-warp partial sums
  return sizeof(T) * M * std::max<size_t>((size_t)L.win_max, 8 * (size_t)L.b);
}

// Coarse-level operator on M columns, streamed: persistent CTAs walk their boxes in chunks of
// RC rows; the copy engine brings each chunk's block rows (contiguous, RC * Wp values) into one
// of two shared-memory buffers (cp.async.bulk, mbarrier completion) while the previous chunk is
// computed, and the box's window of X is staged once per box (16-byte cp.async).  Every operand
// of the inner loop then comes from shared memory.  Every mbarrier wait is bounded: on expiry
// the kernel raises *err, waits (bounded) for its copies still in flight, and all threads leave.
struct MrStreamLayout {
  size_t xs = 0, vals0 = 0, vals1 = 0, red = 0, bar = 0, total = 0;
  int RC = 0;
  __host__ __device__ MrStreamLayout() {}
  __host__ __device__ MrStreamLayout(int win_max, int b, int M, int es, int rc) {
    RC = rc;
    auto up = [](size_t v) { return (v + 127) & ~(size_t)127; };
    xs = 0;
    vals0 = up((size_t)win_max * M * es);
    vals1 = vals0 + up((size_t)rc * win_max * es);
    red = vals1 + up((size_t)rc * win_max * es);
    bar = red + up((size_t)8 * rc * M * es);
    total = bar + 16;
  }
};

template <typename T, int M, int R, class Ep>
__global__ void __launch_bounds__(256) k_mr_coarse_stream(LevelView<T> L, const T* __restrict__ xin, Ep ep,
                                                          double* __restrict__ part, MrStreamLayout lay,
                                                          int* __restrict__ err) {
  constexpr int V = Slice<T>::V, CL = M / V;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* xs = reinterpret_cast<T*>(smem_raw + lay.xs);
  T* red = reinterpret_cast<T*>(smem_raw + lay.red);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw + lay.bar);
  const int b = L.b, RC = lay.RC;
  const int nch = (b + RC - 1) / RC;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, NW = blockDim.x >> 5;
  const int cl = lane % CL, rg = lane / CL;
  const int ngroups = (RC + R - 1) / R;
  double dacc = 0.0;
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();
  // item k of this CTA: box blockIdx.x + (k / nch) * gridDim.x, chunk k % nch
  const int64_t nitems = L.nbox > blockIdx.x ? ((L.nbox - 1 - blockIdx.x) / gridDim.x + 1) * nch : 0;
  auto issue = [&](int64_t k) {   // thread 0: bulk copy of item k's block rows into buffer k & 1
    const int64_t B = blockIdx.x + (k / nch) * (int64_t)gridDim.x;
    const int ch = (int)(k % nch);
    const int64_t e0 = L.nbr_ptr[B];
    const int Wp = ((int)(L.nbr_ptr[B + 1] - e0) * b + 3) & ~3;
    const int q0 = ch * RC, q1 = min(b, q0 + RC);
    const uint32_t bytes = (uint32_t)((int64_t)(q1 - q0) * Wp * (int64_t)sizeof(T));
    T* dst = reinterpret_cast<T*>(smem_raw + ((k & 1) ? lay.vals1 : lay.vals0));
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    mbar_expect_tx(&bar[k & 1], bytes);
    bulk_g2s(dst, L.vals + L.row_ptr[B * b + q0], bytes, &bar[k & 1]);
  };
  if (tid == 0 && nitems > 0) issue(0);
  for (int64_t k = 0; k < nitems; ++k) {
    const int64_t B = blockIdx.x + (k / nch) * (int64_t)gridDim.x;
    const int ch = (int)(k % nch);
    const int64_t e0 = L.nbr_ptr[B];
    const int nn = (int)(L.nbr_ptr[B + 1] - e0);
    const int W = nn * b, Wp = (W + 3) & ~3;
    if (ch == 0) {
      // the box's window of X: row w of the window is level row nbr[e0 + w / b] * b + w % b
      constexpr int PPR = M * (int)sizeof(T) / 16;
      for (int t = tid; t < W * PPR; t += blockDim.x) {
        const int w = t / PPR, pc = t % PPR;
        const int64_t src = (L.nbr[e0 + w / b] * b + w % b) * M + pc * (16 / (int)sizeof(T));
        const unsigned d = (unsigned)__cvta_generic_to_shared(xs + (size_t)w * M + pc * (16 / (int)sizeof(T)));
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(xin + src));
      }
      for (int t = W * M + tid; t < Wp * M; t += blockDim.x) xs[t] = T(0);
      cp_async_wait_all();
    }
    // the next item's block rows go into the other buffer (its last reader finished at the
    // barrier that ended the previous item)
    if (tid == 0 && k + 1 < nitems) issue(k + 1);
    const bool alive = mbar_wait_bounded(&bar[k & 1], (uint32_t)((k >> 1) & 1), err);
    if (__syncthreads_or(!alive)) {
      // leave only after the copies still in flight have landed (bounded as well): this item's,
      // whose wait ran out, and the one issued for the next item
      if (tid == 0) {
        mbar_wait_bounded(&bar[k & 1], (uint32_t)((k >> 1) & 1), nullptr);
        if (k + 1 < nitems) mbar_wait_bounded(&bar[(k + 1) & 1], (uint32_t)(((k + 1) >> 1) & 1), nullptr);
      }
      return;
    }
    const T* vb = reinterpret_cast<const T*>(smem_raw + ((k & 1) ? lay.vals1 : lay.vals0));
    const int q0 = ch * RC, nr = min(b, q0 + RC) - q0;
    T acc[R][V];
#pragma unroll
    for (int i = 0; i < R; ++i)
#pragma unroll
      for (int v = 0; v < V; ++v) acc[i][v] = T(0);
    if (rg < ngroups) {
      for (int g = warp; g * 4 < Wp; g += NW) {
        const int w0 = g * 4;
        Slice<T> xv[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const T* p = xs + (size_t)(w0 + e) * M + cl * V;
          if constexpr (sizeof(T) == 4) {
            const float4 a = *reinterpret_cast<const float4*>(p);
            xv[e].v[0] = a.x; xv[e].v[1] = a.y; xv[e].v[2] = a.z; xv[e].v[3] = a.w;
          } else {
            const double2 a = *reinterpret_cast<const double2*>(p);
            xv[e].v[0] = a.x; xv[e].v[1] = a.y;
          }
        }
#pragma unroll
        for (int i = 0; i < R; ++i) {
          const int row = rg * R + i;
          if (row < nr) {
            T a[4];
            if constexpr (sizeof(T) == 4) {
              const float4 t4 = *reinterpret_cast<const float4*>(vb + (size_t)row * Wp + w0);
              a[0] = t4.x; a[1] = t4.y; a[2] = t4.z; a[3] = t4.w;
            } else {
              const double2 t0 = *reinterpret_cast<const double2*>(vb + (size_t)row * Wp + w0);
              const double2 t1 = *reinterpret_cast<const double2*>(vb + (size_t)row * Wp + w0 + 2);
              a[0] = t0.x; a[1] = t0.y; a[2] = t1.x; a[3] = t1.y;
            }
#pragma unroll
            for (int e = 0; e < 4; ++e)
#pragma unroll
              for (int v = 0; v < V; ++v) acc[i][v] += a[e] * xv[e].v[v];
          }
        }
      }
#pragma unroll
      for (int i = 0; i < R; ++i) {
        const int row = rg * R + i;
        if (row < nr)
#pragma unroll
          for (int v = 0; v < V; ++v) red[((size_t)warp * RC + row) * M + cl * V + v] = acc[i][v];
      }
    }
    __syncthreads();
    const int64_t r0 = B * b + q0;
    for (int t = tid; t < nr * M; t += blockDim.x) {
      const int row = t / M, col = t % M;
      T s = T(0);
      for (int w = 0; w < NW; ++w) s += red[((size_t)w * RC + row) * M + col];
      ep.post1(r0 + row, col, s, dacc);
    }
    __syncthreads();   // red, xs (at a box change) and this item's buffer are free again
  }
  if constexpr (Ep::kDot) {
    if (part != nullptr) {
      __shared__ double redd[8][M];
      for (int o = M; o < 32; o <<= 1) dacc += __shfl_xor_sync(0xffffffffu, dacc, o);
      if (lane < M) redd[warp][lane] = dacc;
      __syncthreads();
      if (tid < M) {
        double t = 0.0;
        for (int w = 0; w < NW; ++w) t += redd[w][tid];
        part[(int64_t)blockIdx.x * M + tid] = t;
      }
    }
  }
}

// Coarse-level FP32 operator on M = 8 or 16 columns on the tensor cores.  A box's rows times its
// window is a dense product D (b x M) = A_B (b x Wp) X_win (Wp x M); it is cut into 16 x 8 tiles
// of mma.sync m16n8k8 (TF32 inputs, FP32 accumulation), one tile per warp over the whole
// window.  Near-FP32 accuracy is kept by splitting each operand into a TF32 head and tail by
// mantissa truncation (hi = x with the low 13 mantissa bits cleared, lo = the same truncation
// of the exact remainder x - hi) and accumulating hi*hi + hi*lo + lo*hi: the tail truncation
// and the dropped lo*lo term cost at most 3 * 2^-20 relative per product (about 22 bits where
// FP32 rounding keeps 24; plain TF32 would keep 11).  The sum over k is taken in
// a permuted order (any order of k gives the same product): for two consecutive MMA steps a
// lane of quad position t holds the window positions 4t .. 4t+3 of its rows, so it reads them
// as one 16-byte load; the window rows of X come through the read-only path by the
// shared-memory window map.  Products only (no dot partials): the Chebyshev step or a plain
// product.
__device__ __forceinline__ uint32_t tf32_trunc(float x) { return __float_as_uint(x) & 0xffffe000u; }

__device__ __forceinline__ void mma_tf32(float (&c)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// head/tail split of four values, then one split MMA step: fragment element j of the step
__device__ __forceinline__ void split3_mma(float (&c)[4], const float (&a)[4], const float (&b)[2]) {
  uint32_t ah[4], al[4], bh[2], bl[2];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    ah[j] = tf32_trunc(a[j]);
    al[j] = tf32_trunc(a[j] - __uint_as_float(ah[j]));
  }
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    bh[j] = tf32_trunc(b[j]);
    bl[j] = tf32_trunc(b[j] - __uint_as_float(bh[j]));
  }
  mma_tf32(c, al, bh);
  mma_tf32(c, ah, bl);
  mma_tf32(c, ah, bh);
}

template <int M, class Ep>
__global__ void __launch_bounds__(128) k_mr_coarse_mma(LevelView<float> L, const float* __restrict__ xin, Ep ep) {
  static_assert(M % 8 == 0, "n tiles of 8 columns");
  constexpr int NT = M / 8;
  extern __shared__ __align__(16) int32_t smap[];
  const int b = L.b;
  const int MT = (b + 15) / 16;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, NW = blockDim.x >> 5;
  const int gid = lane >> 2, tig = lane & 3;
  double unused = 0.0;
  for (int64_t B = blockIdx.x; B < L.nbox; B += gridDim.x) {
    const int64_t e0 = L.nbr_ptr[B];
    const int nn = (int)(L.nbr_ptr[B + 1] - e0);
    const int W = nn * b, Wp = (W + 3) & ~3, W16 = (W + 15) & ~15;
    for (int t = threadIdx.x; t < W; t += blockDim.x) smap[t] = (int32_t)(L.nbr[e0 + t / b] * b + t % b);
    for (int t = W + threadIdx.x; t < W16; t += blockDim.x) smap[t] = 0;   // zero A entries meet row 0
    __syncthreads();
    const int64_t kbase = L.row_ptr[B * b];                                 // box rows: equal length Wp
    for (int tile = warp; tile < MT * NT; tile += NW) {
      const int mt = tile / NT, nt = tile % NT;
      const int ra = mt * 16 + gid, rb = ra + 8;
      const bool va = ra < b, vb = rb < b;
      const float* Aa = L.vals + kbase + (int64_t)(va ? ra : 0) * Wp;
      const float* Ab = L.vals + kbase + (int64_t)(vb ? rb : 0) * Wp;
      const int n = nt * 8 + gid;
      float c[4] = {0.f, 0.f, 0.f, 0.f};
      // one pass = 16 window positions = two MMA steps; U passes of loads in flight
      constexpr int U = 2;
      for (int k0 = 0; k0 < W16; k0 += 16 * U) {
        float4 xa[U], xb[U];
        float y[U][4];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int p = k0 + 16 * u + 4 * tig;          // this lane's 4 window positions
          const bool in = p < W16;
          const bool inA = in && p < Wp;                // Wp is a multiple of 4: the 4 are all in or all out
          xa[u] = (inA && va) ? __ldg(reinterpret_cast<const float4*>(Aa + p)) : make_float4(0.f, 0.f, 0.f, 0.f);
          xb[u] = (inA && vb) ? __ldg(reinterpret_cast<const float4*>(Ab + p)) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
          for (int e = 0; e < 4; ++e) y[u][e] = in ? __ldg(xin + (int64_t)smap[p + e] * M + n) : 0.f;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
          // step 0: fragment k = t <- position 4t, k = t+4 <- 4t+1; step 1: 4t+2 and 4t+3
          const float a0[4] = {xa[u].x, xb[u].x, xa[u].y, xb[u].y};
          const float b0[2] = {y[u][0], y[u][1]};
          split3_mma(c, a0, b0);
          const float a1[4] = {xa[u].z, xb[u].z, xa[u].w, xb[u].w};
          const float b1[2] = {y[u][2], y[u][3]};
          split3_mma(c, a1, b1);
        }
      }
      const int col = nt * 8 + 2 * tig;
      if (va) { ep.post1(B * b + ra, col, c[0], unused); ep.post1(B * b + ra, col + 1, c[1], unused); }
      if (vb) { ep.post1(B * b + rb, col, c[2], unused); ep.post1(B * b + rb, col + 1, c[3], unused); }
    }
    __syncthreads();
  }
}

// Fine-level block operator on global column indices: the level rows taken in one flat sweep
// (no per-box window map, no barriers), each stored entry carrying the level row of its column
// (built once from the windowed layout by k_mr_build_gidx).  Lane layout as in k_mr_level.
template <typename T, int M, int S, class Ep>
__global__ void __launch_bounds__(256) k_mr_rows(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ gidx,
                                                 const T* __restrict__ vals, int64_t nrows, const T* __restrict__ xin,
                                                 Ep ep, double* __restrict__ part) {
  constexpr int V = Slice<T>::V, CL = M / V, LPR = CL * S, RPW = 32 / LPR;
  static_assert(M % V == 0 && 32 % LPR == 0, "lane layout");
  __shared__ double red[8][M];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, NW = blockDim.x >> 5;
  const int cl = lane % CL, s = (lane / CL) % S, rw = lane / LPR;
  double dacc[V];
#pragma unroll
  for (int v = 0; v < V; ++v) dacc[v] = 0.0;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwt = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t base = gw * RPW; base < nrows; base += nwt * RPW) {   // warp-uniform trip count
    const int64_t row = base + rw;
    const bool ok = row < nrows;
    int64_t k0 = 0, k1 = 0;
    if (ok) { k0 = row_ptr[row]; k1 = row_ptr[row + 1]; }
    Slice<T> acc;
#pragma unroll
    for (int v = 0; v < V; ++v) acc.v[v] = T(0);
    for (int64_t k = k0 + 4 * s; k < k1; k += 4 * S) {
      T a[4];
      Vec4<T>::load(vals + k, a);
      const int4 g = __ldcs(reinterpret_cast<const int4*>(gidx + k));
      Slice<T> xv[4];
      xv[0].ldg(xin + (int64_t)g.x * M + cl * V);
      xv[1].ldg(xin + (int64_t)g.y * M + cl * V);
      xv[2].ldg(xin + (int64_t)g.z * M + cl * V);
      xv[3].ldg(xin + (int64_t)g.w * M + cl * V);
#pragma unroll
      for (int e = 0; e < 4; ++e)
#pragma unroll
        for (int v = 0; v < V; ++v) acc.v[v] += a[e] * xv[e].v[v];
    }
#pragma unroll
    for (int o = CL; o < LPR; o <<= 1)
#pragma unroll
      for (int v = 0; v < V; ++v) acc.v[v] += __shfl_xor_sync(0xffffffffu, acc.v[v], o);
    if (ok && s == 0) ep.post(row, cl * V, acc, dacc);
  }
  if constexpr (Ep::kDot) {
    if (part != nullptr) {
#pragma unroll
      for (int o = CL; o < 32; o <<= 1)
#pragma unroll
        for (int v = 0; v < V; ++v) dacc[v] += __shfl_xor_sync(0xffffffffu, dacc[v], o);
      if (lane < CL)
#pragma unroll
        for (int v = 0; v < V; ++v) red[warp][lane * V + v] = dacc[v];
      __syncthreads();
      if (threadIdx.x < M) {
        double t = 0.0;
        for (int w = 0; w < NW; ++w) t += red[w][threadIdx.x];
        part[(int64_t)blockIdx.x * M + threadIdx.x] = t;
      }
    }
  }
}

// ---- grouped fine level.  Rows of one box whose stored column lists are identical (with Q_p
// elements: the degrees of freedom interior to one cell, or to one face, or to one edge) form a
// group of R rows.  A group stores its column list once and its values entry-major (entry k of
// its row r at k*R + r), so each gathered slice of X serves R rows instead of one.  Groups of
// one size R in {1, 2, 4, 8} are launched together; larger sets of equal rows are split.

// N consecutive values (N * sizeof(T) a multiple of 16 bytes, or one 8- or 4-byte value run;
// the group layout aligns them), read once (streaming)
template <int N>
__device__ __forceinline__ void load_run(const float* p, float (&w)[N]) {
  if constexpr (N >= 4) {
#pragma unroll
    for (int q = 0; q < N / 4; ++q) {
      const float4 a = __ldcs(reinterpret_cast<const float4*>(p) + q);
      w[4 * q] = a.x; w[4 * q + 1] = a.y; w[4 * q + 2] = a.z; w[4 * q + 3] = a.w;
    }
  } else if constexpr (N == 2) {
    const float2 a = __ldcs(reinterpret_cast<const float2*>(p));
    w[0] = a.x; w[1] = a.y;
  } else {
    w[0] = __ldcs(p);
  }
}
template <int N>
__device__ __forceinline__ void load_run(const double* p, double (&w)[N]) {
  if constexpr (N >= 2) {
#pragma unroll
    for (int q = 0; q < N / 2; ++q) {
      const double2 a = __ldcs(reinterpret_cast<const double2*>(p) + q);
      w[2 * q] = a.x; w[2 * q + 1] = a.y;
    }
  } else {
    w[0] = __ldcs(p);
  }
}
// E consecutive column indices (E = 2 or 4; group entry lists start on multiples of 4)
template <int E>
__device__ __forceinline__ void load_cols(const int32_t* p, int (&c)[E]) {
  if constexpr (E == 4) {
    const int4 a = __ldcs(reinterpret_cast<const int4*>(p));
    c[0] = a.x; c[1] = a.y; c[2] = a.z; c[3] = a.w;
  } else {
    const int2 a = __ldcs(reinterpret_cast<const int2*>(p));
    c[0] = a.x; c[1] = a.y;
  }
}

// Entry slots per group for R rows and CL lanes per row slice: fewer slots as R grows, so that
// the slot reduction (R x V values per lane and level) stays small next to the R x V FMAs per entry.
__host__ __device__ constexpr int mr_group_slots(int R, int CL) {
  const int want = R == 1 ? 8 : (R == 8 ? 2 : 4);
  return want * CL <= 32 ? want : 32 / CL;
}

// Entries per slot step: four for groups of one or two rows, two for larger groups (the R
// accumulators and the step's R x E values share the registers).
__host__ __device__ constexpr int mr_group_step(int R) { return R <= 2 ? 4 : 2; }

// Level operator on M columns over the groups of one size R: CL lanes cover the M columns with
// 16-byte slices, S slots split the group's entries E at a time; each step reads the E column
// indices and R x E values once per slot and E slices of X per lane (all in flight together),
// and multiplies them into R accumulators.  After the slot reduction, slot s finishes the
// group's rows r = s, s + S, ... through the epilogue.
template <typename T, int M, int R, class Ep>
__global__ void __launch_bounds__(256) k_mr_grouped(int64_t ng, const int64_t* __restrict__ geoff,
                                                    const int64_t* __restrict__ gvoff, const int32_t* __restrict__ grows,
                                                    const int32_t* __restrict__ gcol, const T* __restrict__ gvals,
                                                    const T* __restrict__ xin, Ep ep, double* __restrict__ part) {
  constexpr int V = Slice<T>::V, CL = M / V, S = mr_group_slots(R, CL), LPR = CL * S, GPW = 32 / LPR;
  constexpr int E = mr_group_step(R);
  static_assert(M % V == 0 && 32 % LPR == 0, "lane layout");
  __shared__ double red[8][M];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, NW = blockDim.x >> 5;
  const int cl = lane % CL, s = (lane / CL) % S, gw = lane / LPR;
  double dacc[V];
#pragma unroll
  for (int v = 0; v < V; ++v) dacc[v] = 0.0;
  const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwt = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t base = wid * GPW; base < ng; base += nwt * GPW) {   // warp-uniform trip count
    const int64_t g = base + gw;
    const bool ok = g < ng;
    int64_t e0 = 0, e1 = 0, v0 = 0;
    if (ok) { e0 = geoff[g]; e1 = geoff[g + 1]; v0 = gvoff[g]; }
    T acc[R][V];
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
      for (int v = 0; v < V; ++v) acc[r][v] = T(0);
    // group entry counts are multiples of 4, so a step never runs past the group's end
    for (int64_t e = e0 + (int64_t)E * s; e < e1; e += (int64_t)E * S) {
      int c[E];
      load_cols<E>(gcol + e, c);
      T w[R * E];
      load_run<R * E>(gvals + v0 + (e - e0) * R, w);
      Slice<T> xs[E];
#pragma unroll
      for (int q = 0; q < E; ++q) xs[q].ldg(xin + (int64_t)c[q] * M + cl * V);
#pragma unroll
      for (int q = 0; q < E; ++q)
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
          for (int v = 0; v < V; ++v) acc[r][v] += w[q * R + r] * xs[q].v[v];
    }
#pragma unroll
    for (int o = CL; o < LPR; o <<= 1)
#pragma unroll
      for (int r = 0; r < R; ++r)
#pragma unroll
        for (int v = 0; v < V; ++v) acc[r][v] += __shfl_xor_sync(0xffffffffu, acc[r][v], o);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if (ok && r % S == s) {
        Slice<T> out;
#pragma unroll
        for (int v = 0; v < V; ++v) out.v[v] = acc[r][v];
        ep.post(grows[g * R + r], cl * V, out, dacc);
      }
    }
  }
  if constexpr (Ep::kDot) {
    if (part != nullptr) {
#pragma unroll
      for (int o = CL; o < 32; o <<= 1)
#pragma unroll
        for (int v = 0; v < V; ++v) dacc[v] += __shfl_xor_sync(0xffffffffu, dacc[v], o);
      if (lane < CL)
#pragma unroll
        for (int v = 0; v < V; ++v) red[warp][lane * V + v] = dacc[v];
      __syncthreads();
      if (threadIdx.x < M) {
        double t = 0.0;
        for (int w = 0; w < NW; ++w) t += red[w][threadIdx.x];
        part[(int64_t)blockIdx.x * M + threadIdx.x] = t;
      }
    }
  }
}

// The grouped layout's column lists and values, gathered from the per-row layout: one warp per
// group; entry k of the group's row r is entry k of that row (equal lists, equal padding).
// gcol_out may be null (values only, for the second precision).
template <typename T>
__global__ void __launch_bounds__(256) k_mr_group_gather(int R, int64_t ng, const int64_t* __restrict__ geoff,
                                                         const int64_t* __restrict__ gvoff,
                                                         const int32_t* __restrict__ grows,
                                                         const int64_t* __restrict__ row_ptr,
                                                         const int32_t* __restrict__ gidx, const T* __restrict__ vals,
                                                         int32_t* __restrict__ gcol_out, T* __restrict__ gvals_out) {
  const int lane = threadIdx.x & 31;
  const int64_t nwt = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; g < ng; g += nwt) {
    const int64_t e0 = geoff[g], K = geoff[g + 1] - e0, v0 = gvoff[g];
    for (int r = 0; r < R; ++r) {
      const int64_t k0 = row_ptr[grows[g * R + r]];
      for (int64_t k = lane; k < K; k += 32) {
        if (r == 0 && gcol_out) gcol_out[e0 + k] = gidx[k0 + k];
        gvals_out[v0 + k * R + r] = vals[k0 + k];
      }
    }
  }
}

// Global column of every stored fine-level entry: the window map of its box applied to its
// 16-bit window index (padding entries keep window position 0, a valid row with value 0).
template <typename T>
__global__ void __launch_bounds__(256) k_mr_build_gidx(LevelView<T> L, int32_t* __restrict__ gidx) {
  extern __shared__ __align__(16) int32_t smap[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, NW = blockDim.x >> 5;
  for (int64_t B = blockIdx.x; B < L.nbox; B += gridDim.x) {
    const int64_t e0 = L.nbr_ptr[B];
    const int nn = (int)(L.nbr_ptr[B + 1] - e0);
    const int W = L.win_size[B];
    for (int q = warp; q < nn; q += NW) {
      const int wo = L.win_off[e0 + q];
      const int64_t src = L.slot_src[e0 + q];
      const int len = (q + 1 < nn ? L.win_off[e0 + q + 1] : W) - wo;
      for (int t = lane; t < len; t += 32) smap[wo + t] = (int32_t)(src + t);
    }
    __syncthreads();
    const int64_t k0 = L.row_ptr[L.box_row[B]], k1 = L.row_ptr[L.box_row[B + 1]];
    for (int64_t k = k0 + threadIdx.x; k < k1; k += blockDim.x) gidx[k] = smap[L.idx[k]];
    __syncthreads();
  }
}

// ---------------------------------------------------------------- transfers
// Next-level initialisation after restriction, per column: R = B, X = 0, D = c0 dinv B.
template <typename T, int M>
struct MNextInit {
  T* r; T* x; T* d; const T* dinv; T c0;
  __device__ void operator()(int64_t i, int c, T bi) const {
    r[i * M + c] = bi;
    if (x) { x[i * M + c] = T(0); d[i * M + c] = c0 * dinv[i] * bi; }
  }
};

// Fine -> level 1: B1[(B*b+q), c] = sum_{i in B} P0[i][q] R[i, c].  One CTA per box.
template <typename T, int M, class NX>
__global__ void __launch_bounds__(256) k_mr_restrict_fine(const T* __restrict__ P0, const T* __restrict__ r,
                                                          const int64_t* __restrict__ box_row, int64_t nbox, int b,
                                                          NX nx) {
  for (int64_t B = blockIdx.x; B < nbox; B += gridDim.x) {
    const int64_t i0 = box_row[B], i1 = box_row[B + 1];
    for (int t = threadIdx.x; t < b * M; t += blockDim.x) {
      const int q = t / M, c = t % M;
      T s = T(0);
      for (int64_t i = i0; i < i1; ++i) s += P0[i * b + q] * r[i * M + c];
      nx(B * b + q, c, s);
    }
  }
}

// Level l -> l+1: B[(P,q), c] = sum_{children ch} sum_{q'} Pt[ch][q'][q] R[(ch,q'), c].
template <typename T, int M, class NX>
__global__ void k_mr_restrict_coarse(const T* __restrict__ Pt, const T* __restrict__ r, int64_t nparent, int b,
                                     int fan, NX nx) {
  const int64_t tot = nparent * b * M;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot; t += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(t % M);
    const int64_t bq = t / M;
    const int64_t B = bq / b;
    const int q = (int)(bq - B * b);
    T s = T(0);
    for (int64_t ch = B * fan; ch < (B + 1) * fan; ++ch)
      for (int qp = 0; qp < b; ++qp) s += Pt[(ch * b + qp) * b + q] * r[(ch * b + qp) * M + c];
    nx(bq, c, s);
  }
}

// Level 1 -> fine: D0[k, c] = sum_q P0[k][q] (X1 + D1)[(box(k)*b+q), c]   (D1 may be null).
template <typename T, int M>
__global__ void k_mr_prolong_fine(const T* __restrict__ P0, const int32_t* __restrict__ box_of,
                                  const T* __restrict__ x1, const T* __restrict__ d1, int64_t n, int b,
                                  T* __restrict__ d0) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n * M; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = t / M;
    const int c = (int)(t - k * M);
    const int64_t B = box_of[k];
    T s = T(0);
    for (int q = 0; q < b; ++q) {
      const int64_t o = (B * b + q) * M + c;
      s += P0[k * b + q] * (x1[o] + (d1 ? d1[o] : T(0)));
    }
    d0[t] = s;
  }
}

// Level l+1 -> l: D[(ch,q'), c] = sum_q Pt[ch][q'][q] (X + D)_{l+1}[(parent(ch), q), c].
template <typename T, int M>
__global__ void k_mr_prolong_coarse(const T* __restrict__ Pt, const T* __restrict__ x1, const T* __restrict__ d1,
                                    int64_t nchild, int b, int fan, T* __restrict__ d0) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nchild * b * M;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(t % M);
    const int64_t cq = t / M;
    const int64_t ch = cq / b;
    const int64_t B = ch / fan;
    T s = T(0);
    for (int q = 0; q < b; ++q) {
      const int64_t o = (B * b + q) * M + c;
      s += Pt[cq * b + q] * (x1[o] + (d1 ? d1[o] : T(0)));
    }
    d0[t] = s;
  }
}

// Coarsest solve X = A_c^{-1} R on M columns: one warp per row of the inverse, lanes split as
// in k_mr_level (CL column slices x S entry slots); the inverse is read once for all columns.
template <typename T, int M>
__global__ void __launch_bounds__(256) k_mr_dense(const T* __restrict__ Ainv, int64_t ld, const T* __restrict__ r,
                                                  int64_t nc, T* __restrict__ x) {
  constexpr int V = Slice<T>::V, CL = M / V, S = 32 / CL;
  const int lane = threadIdx.x & 31, cl = lane % CL, s = lane / CL;
  const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t row = w; row < nc; row += nw) {
    const T* a = Ainv + row * ld;
    Slice<T> acc;
#pragma unroll
    for (int v = 0; v < V; ++v) acc.v[v] = T(0);
    for (int64_t k = s; k < nc; k += S) {
      const T ak = a[k];
      Slice<T> xv;
      xv.ldg(r + k * M + cl * V);
#pragma unroll
      for (int v = 0; v < V; ++v) acc.v[v] += ak * xv.v[v];
    }
#pragma unroll
    for (int o = CL; o < 32; o <<= 1)
#pragma unroll
      for (int v = 0; v < V; ++v) acc.v[v] += __shfl_xor_sync(0xffffffffu, acc.v[v], o);
    if (s == 0) acc.st(x + row * M + cl * V);
  }
}

// ---------------------------------------------------------------- CG on M columns (FP64)
// Per-column scalars live in mscal[slot * M + c] (slots as in Scal).  The element loops below
// stride by a multiple of M, so every thread stays on one column c = threadIdx.x % M.

// Per-CTA, per-column partial sums: part[blockIdx.x * M + c].  blockDim = 256.
template <int M>
__device__ __forceinline__ void store_partial_m(double v, double* part) {
  __shared__ double red[8][M];
  for (int o = M; o < 32; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l < M) red[w][l] = v;
  __syncthreads();
  if (threadIdx.x < M) {
    double s = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += red[k][threadIdx.x];
    part[(int64_t)blockIdx.x * M + threadIdx.x] = s;
  }
}

// Caller-order column blocks (m vectors of length n, each contiguous) <-> tree-order,
// row-interleaved blocks of M >= m columns (the extra columns are zero).  perm == nullptr:
// identity (coarse levels keep their own numbering).
__global__ void k_mr_gather(const double* __restrict__ src, const int64_t* __restrict__ perm, int64_t n, int m,
                            int M, double* __restrict__ dst) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n * M; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / M;
    const int c = (int)(t - i * M);
    dst[t] = c < m ? src[(int64_t)c * n + (perm ? perm[i] : i)] : 0.0;
  }
}

__global__ void k_mr_scatter(const double* __restrict__ src, const int64_t* __restrict__ perm, int64_t n, int m,
                             int M, double* __restrict__ dst) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n * M; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / M;
    const int c = (int)(t - i * M);
    if (c < m) dst[(int64_t)c * n + (perm ? perm[i] : i)] = src[t];
  }
}

// R = B - Y with per-column partials of ||R||^2 and (optionally) ||B||^2.
template <int M>
__global__ void __launch_bounds__(256) k_mr_residual(const double* __restrict__ b, const double* __restrict__ y,
                                                     double* __restrict__ r, int64_t nm, double* part, double* part2) {
  double s = 0.0, s2 = 0.0;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nm; k += (int64_t)gridDim.x * blockDim.x) {
    const double v = b[k] - y[k];
    r[k] = v;
    s += v * v;
    s2 += b[k] * b[k];
  }
  store_partial_m<M>(s, part);
  if (part2) { __syncthreads(); store_partial_m<M>(s2, part2); }
}

// V-cycle entry on level 0 from the FP64 residual: VR = R, VX = 0, VD = c0 dinv R.
template <typename T, int M>
__global__ void k_mr_vc_init(const double* __restrict__ r, int64_t nm, T* vr, T* vx, T* vd,
                             const T* __restrict__ dinv, T c0) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nm; k += (int64_t)gridDim.x * blockDim.x) {
    const T rt = (T)r[k];
    vr[k] = rt;
    vx[k] = T(0);
    vd[k] = c0 * dinv[k / M] * rt;
  }
}

// X += alpha_c P; R -= alpha_c Q; per-column ||R||^2; V-cycle entry from the new R.
template <typename T, int M>
__global__ void __launch_bounds__(256) k_mr_cg_update(double* __restrict__ x, double* __restrict__ r,
                                                      const double* __restrict__ p, const double* __restrict__ q,
                                                      const double* __restrict__ mscal, int64_t nm, double* part,
                                                      T* vr, T* vx, T* vd, const T* __restrict__ dinv, T c0) {
  const double alpha = mscal[S_ALPHA * M + threadIdx.x % M];
  double s = 0.0;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nm; k += (int64_t)gridDim.x * blockDim.x) {
    x[k] += alpha * p[k];
    const double rk = r[k] - alpha * q[k];
    r[k] = rk;
    s += rk * rk;
    const T rt = (T)rk;
    vr[k] = rt;
    vx[k] = T(0);
    vd[k] = c0 * dinv[k / M] * rt;
  }
  store_partial_m<M>(s, part);
}

// Z = VX + VD (level 0's last update), per-column partials of Z . W.
template <typename T, int M>
__global__ void __launch_bounds__(256) k_mr_vc_final_dot(const T* __restrict__ vx, const T* __restrict__ vd,
                                                         double* __restrict__ z, const double* __restrict__ w,
                                                         int64_t nm, double* part) {
  double s = 0.0;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nm; k += (int64_t)gridDim.x * blockDim.x) {
    const double zk = (double)vx[k] + (double)vd[k];
    z[k] = zk;
    s += zk * w[k];
  }
  store_partial_m<M>(s, part);
}

// PCG: P = Z + beta_c P.  FCG: P = Z - beta_c P and per-column partials of P . R.
template <int M>
__global__ void __launch_bounds__(256) k_mr_p_update(double* __restrict__ p, const double* __restrict__ z,
                                                     const double* __restrict__ r, const double* __restrict__ mscal,
                                                     int64_t nm, int fcg, double* part) {
  const double beta = mscal[S_BETA * M + threadIdx.x % M];
  double s = 0.0;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nm; k += (int64_t)gridDim.x * blockDim.x) {
    const double pk = fcg ? z[k] - beta * p[k] : z[k] + beta * p[k];
    p[k] = pk;
    s += pk * r[k];
  }
  if (part) store_partial_m<M>(s, part);
}

// Per-column deterministic sums of `nb` CTA partials into mscal[slot][c], then the scalar
// finish of each active column (inactive columns take alpha = beta = 0 and stay put).
// blockDim = 32 * M: warp c sums column c.
template <int M>
__global__ void k_mr_reduce(const double* __restrict__ part, int nb, double* mscal, int slot, int fin,
                            const int* __restrict__ active, int* status) {
  const int c = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (c >= M) return;
  double s = 0.0;
  for (int k = l; k < nb; k += 32) s += part[(int64_t)k * M + c];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (l != 0) return;
  mscal[slot * M + c] = s;
  const bool act = active == nullptr || active[c] != 0;
  // per-column coefficient history after the S_COUNT x M slots: column c owns 2 x kHist
  // doubles (alphas, then betas; flexible-CG betas sign-flipped to their PCG equivalent)
  double* hist = mscal + S_COUNT * M + (int64_t)c * 2 * kHist;
  if (fin == FIN_ALPHA_PCG || fin == FIN_ALPHA_FCG) {
    const double num = (fin == FIN_ALPHA_PCG) ? mscal[S_RZ * M + c] : mscal[S_PR * M + c];
    if (!act) mscal[S_ALPHA * M + c] = 0.0;
    else if (!(s > 0.0) || !isfinite(num)) { if (status) atomicExch(status, 1); mscal[S_ALPHA * M + c] = 0.0; }
    else {
      const double a = num / s;
      mscal[S_ALPHA * M + c] = a;
      const int ia = (int)mscal[S_NA * M + c];
      if (ia < kHist) hist[ia] = a;
      mscal[S_NA * M + c] = (double)(ia + 1);
    }
  } else if (fin == FIN_BETA_PCG || fin == FIN_BETA_FCG) {
    const double be = act ? s / mscal[(fin == FIN_BETA_PCG ? S_RZ : S_PQ) * M + c] : 0.0;
    mscal[S_BETA * M + c] = be;
    if (act) {
      if (fin == FIN_BETA_PCG) mscal[S_RZ * M + c] = s;
      const int ib = (int)mscal[S_NB * M + c];
      if (ib < kHist) hist[kHist + ib] = (fin == FIN_BETA_PCG) ? be : -be;
      mscal[S_NB * M + c] = (double)(ib + 1);
    }
  }
}

// Restart of the active columns' coefficient histories (a restarted column begins a new
// Lanczos sequence).  One warp.
template <int M>
__global__ void k_mr_hist_reset(double* mscal, const int* __restrict__ active) {
  const int c = threadIdx.x;
  if (c < M && active[c]) { mscal[S_NA * M + c] = 0.0; mscal[S_NB * M + c] = 0.0; }
}

// Device-side stop test after the X/R update: count the update of every active column, retire
// columns with ||r_c||^2 <= their threshold or a spent budget, continue while any is active.
// mscal[S_THR][c] = the column's threshold on ||r_c||^2, lp[1] = iteration budget per column.  One warp.  Inside the loop graph
// (in_graph = 1) the decision sets the loop's conditions, else it goes to *go_out.
template <int M>
__global__ void k_mr_converge(const double* __restrict__ mscal, const double* __restrict__ lp, int* __restrict__ its,
                              int* __restrict__ active, int* __restrict__ status, cudaGraphConditionalHandle loop,
                              cudaGraphConditionalHandle rest, int in_graph, int* __restrict__ go_out) {
  const int c = threadIdx.x;
  bool go = false;
  if (c < M && active[c]) {
    const int k = its[c] + 1;
    its[c] = k;
    const double rr = mscal[S_RR * M + c];
    if (!isfinite(rr)) atomicExch(status, 1);
    const bool done = !(rr > mscal[S_THR * M + c]) || (double)k >= lp[1];
    if (done) active[c] = 0;
    go = !done;
  }
  const unsigned any = __ballot_sync(0xffffffffu, go);
  if (c == 0) {
    const bool g = any != 0u && *status == 0;
    if (in_graph) {
      cudaGraphSetConditional(loop, g ? 1u : 0u);
      cudaGraphSetConditional(rest, g ? 1u : 0u);
    } else {
      *go_out = g ? 1 : 0;
    }
  }
}

}  // namespace r3mg
