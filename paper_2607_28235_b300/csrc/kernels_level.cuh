// Level operator kernels: windowed sparse / block-dense row products with fused epilogues.
//
// One CTA handles one box at a time (grid-stride over boxes).  The box's window -- the
// concatenation of the input vector over its neighbour boxes (fine level: the points of the
// level-1 neighbour boxes; coarse level l: the b coefficients of each neighbour box) -- is
// staged once in shared memory, so the matrix stream carries 16-bit window indices on the
// fine level and no index at all on coarse levels (dense b x b blocks stored row by row).
// Rows of the box are spread over groups of G lanes; each lane loads 4 consecutive entries
// per step with 16-byte vector loads; the G partial sums are combined by warp shuffles and
// the rows' sums (FP64: up to 8 partials per row) are parked in shared memory, and one thread
// per row then applies the epilogue (plain product, Chebyshev-Jacobi step, residual...).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace r3mg {

template <typename T>
struct LevelView {
  int64_t nrows = 0, nbox = 0;
  int b = 0;                          // coarse block size; 0 on the fine level
  const int64_t* box_row = nullptr;   // fine: nbox+1 row offsets of the boxes
  const int64_t* nbr_ptr = nullptr;   // nbox+1
  const int64_t* nbr = nullptr;       // neighbour boxes
  const int32_t* win_off = nullptr;   // fine: per (box, slot) window offset
  const int64_t* slot_src = nullptr;  // fine: per (box, slot) first row of the neighbour box
  const int32_t* win_size = nullptr;  // fine: per box window length
  const int64_t* row_ptr = nullptr;   // nrows+1 entry offsets, multiples of 4
  const uint16_t* idx = nullptr;      // fine: window index per entry
  const T* vals = nullptr;
  const T* dinv = nullptr;
  int max_slots = 0;                  // largest neighbour count
  int win_max = 0;                    // largest window (padded to 4)
  int max_box_rows = 0;               // rows of the largest box (own-row staging)
  const int32_t* row_order = nullptr; // fine: per box, local rows longest first (balances the groups)
  int keep = 0;                       // values fit half of L2: cached loads, so the next step of
                                      // the same level finds them there (else streaming loads)
};

template <typename T>
struct Vec4;
template <>
struct Vec4<float> {
  static __device__ __forceinline__ void load(const float* p, float (&v)[4]) {   // streamed (read once)
    const float4 a = __ldcs(reinterpret_cast<const float4*>(p));
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
  }
  static __device__ __forceinline__ void load(const float* p, float (&v)[4], int keep) {
    const float4 a = keep ? __ldg(reinterpret_cast<const float4*>(p)) : __ldcs(reinterpret_cast<const float4*>(p));
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
  }
};
template <>
struct Vec4<double> {
  static __device__ __forceinline__ void load(const double* p, double (&v)[4]) {   // streamed (read once)
    const double2* q = reinterpret_cast<const double2*>(p);
    const double2 a = __ldcs(q), c = __ldcs(q + 1);
    v[0] = a.x; v[1] = a.y; v[2] = c.x; v[3] = c.y;
  }
  static __device__ __forceinline__ void load(const double* p, double (&v)[4], int keep) {
    const double2* q = reinterpret_cast<const double2*>(p);
    const double2 a = keep ? __ldg(q) : __ldcs(q);
    const double2 c = keep ? __ldg(q + 1) : __ldcs(q + 1);
    v[0] = a.x; v[1] = a.y; v[2] = c.x; v[3] = c.y;
  }
};

__device__ __forceinline__ void load_idx4(const uint16_t* p, int (&i)[4]) {
  uint2 a = __ldcs(reinterpret_cast<const uint2*>(p));
  i[0] = a.x & 0xffff; i[1] = a.x >> 16; i[2] = a.y & 0xffff; i[3] = a.y >> 16;
}

// asynchronous 4- or 8-byte global -> shared copy (cp.async.ca), completed by cp_async_wait_all
template <typename T>
__device__ __forceinline__ void cp_async_elem(T* dst, const T* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(d), "l"(src), "n"(sizeof(T)));
}

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }
// L2 prefetch of a contiguous range by the copy engine (no registers, no shared memory);
// start and size are rounded to the 16-byte granularity the instruction requires
__device__ __forceinline__ void bulk_prefetch_l2(const void* base, int64_t begin_byte, int64_t end_byte) {
  const int64_t a = begin_byte & ~(int64_t)15;
  const int64_t z = (end_byte + 15) & ~(int64_t)15;
  if (z > a)
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"((const char*)base + a), "r"((uint32_t)(z - a))
                 : "memory");
}

__device__ __forceinline__ void cp_async_commit_group() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_group1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }

template <int G, typename T>
__device__ __forceinline__ T group_sum(T v) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o, G);
  return v;
}

// Block-wide sum of one double per thread; result valid in thread 0.  blockDim % 32 == 0.
__device__ __forceinline__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += red[k];
  return s;
}

// ---------------------------------------------------------------- epilogues
// Each gets (row, y = (A x)_row) from one thread (the register kernels: a thread per row once the
// box's rows are summed; the TMA form: the group leader); `acc` is a per-thread partial sum
// folded into one value per CTA written to `part[blockIdx.x]` when the epilogue wants it.

// Epilogues.  Each names up to kAuxMax own-row vectors (src(j), staged when stage(j)); the
// kernels copy them into shared memory with the window, and post() finishes a row from the
// staged values: aux[j][lr] is vector j at local row lr of the box (or item).
constexpr int kAuxMax = 4;

template <typename T>
struct TEpApplyDot {     // y = A x, and partial += w . y when w is given
  T* y; const T* w;
  static constexpr bool kDot = true;
  static constexpr int kStage = 1;
  __device__ const T* src(int) const { return w; }
  __device__ bool stage(int) const { return w != nullptr; }
  __device__ void post(int64_t r, int lr, T y_r, T* const* aux, double& acc) const {
    y[r] = y_r;
    if (w) acc += (double)aux[0][lr] * (double)y_r;
  }
};

// One Chebyshev-Jacobi step (Saad, Algorithm 12.1, D^{-1}-preconditioned), with the input
// window being the current update d:  x += d;  r -= A d;  d' = a d + c D^{-1} r.
template <typename T>
struct TEpCheb {
  T* x; T* r; const T* d; T* dnext; const T* dinv; T a, c;
  static constexpr bool kDot = false;
  static constexpr int kStage = 4;
  __device__ const T* src(int j) const { return j == 0 ? x : j == 1 ? r : j == 2 ? d : dinv; }
  __device__ bool stage(int) const { return true; }
  __device__ void post(int64_t i, int lr, T y_r, T* const* aux, double&) const {
    const T di = aux[2][lr];
    x[i] = aux[0][lr] + di;
    const T rn = aux[1][lr] - y_r;
    r[i] = rn;
    dnext[i] = a * di + c * aux[3][lr] * rn;
  }
};

// FP64 rows park up to kParkLanes partial sums each, kParkStride apart (an odd stride of
// doubles, so the epilogue pass's reads, one row per thread, meet at most 2-way bank conflicts)
constexpr int kParkLanes = 8;
constexpr int kParkStride = 9;

// Shared-memory carve-up of one stage of the register kernels (byte offsets): the window,
// the epilogue's own-row vectors, the box's row offsets (absolute entry positions, int64),
// (fine level) its row order, so that no row waits on a dependent global load for its bounds,
// and the rows' parked (partial) sums, which the epilogue pass reads.
struct LevelSmem {
  size_t aux = 0, rp = 0, ord = 0, ys = 0, total = 0;
  static __host__ __device__ size_t up16(size_t v) { return (v + 15) & ~(size_t)15; }
  __host__ __device__ LevelSmem(size_t elem, int win_max, int max_box_rows) {
    aux = up16(elem * (size_t)win_max);
    rp = aux + up16(elem * (size_t)kAuxMax * max_box_rows);
    ord = rp + up16(sizeof(int64_t) * ((size_t)max_box_rows + 1));
    ys = ord + up16(sizeof(int32_t) * (size_t)max_box_rows);
    total = ys + up16(elem * (size_t)(elem == 8 ? kParkStride : 1) * max_box_rows);
  }
};

// One chunk of a row: U steps of 4 consecutive entries per lane (values, and the fine level's
// packed 16-bit window indices; coarse rows index the window by position).
template <typename T, int U, bool FINE>
struct Chunk {
  T v[U][4];
  uint2 q[U];   // fine: packed indices; coarse: q[u].x = window position of the step's first entry
  int nv;       // steps that start before the row's end (a prefix of the U steps)
  __device__ __forceinline__ void load(const T* vals, const uint16_t* idx, int64_t k, int64_t k0, int64_t k1, int G,
                                      int keep) {
    nv = 0;
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t kk = k + (int64_t)u * 4 * G;
      if (kk < k1) {
        ++nv;
        if constexpr (FINE) Vec4<T>::load(vals + kk, v[u]);   // the fine level never fits L2
        else Vec4<T>::load(vals + kk, v[u], keep);
        if constexpr (FINE) q[u] = __ldcs(reinterpret_cast<const uint2*>(idx + kk));
        else q[u] = make_uint2((unsigned)(kk - k0), 0u);
      } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) v[u][j] = T(0);
        q[u] = make_uint2(0u, 0u);
      }
    }
  }
  // FP64: one fused multiply-add chain, one FP64-pipe instruction per stored entry (the FP64
  // pipe, not HBM and not the chain's latency, bounds the FP64 form; a product tree adds a
  // multiply and an add per four entries, a second chain an add per row), and steps wholly past
  // the row's end are skipped rather than multiplied by zeros.  FP32: a short product tree per
  // step, alternating two accumulators (shorter dependent chains).
  __device__ __forceinline__ void consume(const T* win, T (&acc)[2]) const {
#pragma unroll
    for (int u = 0; u < U; ++u) {
      int ii[4];
      if constexpr (FINE) { ii[0] = q[u].x & 0xffff; ii[1] = q[u].x >> 16; ii[2] = q[u].y & 0xffff; ii[3] = q[u].y >> 16; }
      else { const int t = (int)q[u].x; ii[0] = t; ii[1] = t + 1; ii[2] = t + 2; ii[3] = t + 3; }
      T& a = acc[sizeof(T) == 8 ? 0 : (u & 1)];
      if constexpr (sizeof(T) == 8) {
        if (u >= nv) break;
#pragma unroll
        for (int j = 0; j < 4; ++j) a = fma_rn(v[u][j], win[ii[j]], a);
      } else {
        a += v[u][0] * win[ii[0]] + v[u][1] * win[ii[1]] + v[u][2] * win[ii[2]] + v[u][3] * win[ii[3]];
      }
    }
  }
};

// ---- one box of a level step, as device functions shared by the level kernels and the
// persistent batched solve.  A box is staged (window, own-row vectors, row bounds) into one
// shared-memory stage, then its rows are computed from it.
template <typename T, bool FINE>
__device__ __forceinline__ void level_box_rows(const LevelView<T>& L, int64_t B, int64_t& r0, int64_t& r1) {
  if constexpr (FINE) { r0 = L.box_row[B]; r1 = L.box_row[B + 1]; }
  else { r0 = B * L.b; r1 = r0 + L.b; }
}

// the box's matrix slice is contiguous: one thread asks the copy engine to pull it into L2
template <typename T, bool FINE>
__device__ __forceinline__ void level_prefetch(const LevelView<T>& L, int64_t B) {
  if (threadIdx.x == 0) {
    int64_t r0, r1;
    level_box_rows<T, FINE>(L, B, r0, r1);
    const int64_t k0 = L.row_ptr[r0], k1 = L.row_ptr[r1];
    bulk_prefetch_l2(L.vals, k0 * (int64_t)sizeof(T), k1 * (int64_t)sizeof(T));
    if constexpr (FINE) bulk_prefetch_l2(L.idx, k0 * 2, k1 * 2);
  }
}

// window staging: one warp per neighbour slot, asynchronous global->shared copies (cp.async)
// so every element of the window is in flight at once; then the epilogue's own-row vectors and
// the rows' bounds, so no row waits on a dependent global load.  Completed by cp_async_wait_*.
template <typename T, bool FINE, class Ep>
__device__ __forceinline__ void level_stage(const LevelView<T>& L, const T* __restrict__ xin, const Ep& ep,
                                            const LevelSmem& lay, int64_t B, unsigned char* base) {
  const int NW = blockDim.x >> 5, warp = threadIdx.x >> 5, wl = threadIdx.x & 31;
  T* win = reinterpret_cast<T*>(base);
  const int64_t e0 = L.nbr_ptr[B];
  const int nn = (int)(L.nbr_ptr[B + 1] - e0);
  int W;
  if constexpr (FINE) {
    W = L.win_size[B];
    for (int s = warp; s < nn; s += NW) {
      const int wo = L.win_off[e0 + s];
      const int64_t src = L.slot_src[e0 + s];
      const int len = (s + 1 < nn ? L.win_off[e0 + s + 1] : W) - wo;
      for (int t = wl; t < len; t += 32) cp_async_elem(win + wo + t, xin + src + t);
    }
  } else {
    const int b = L.b;
    W = nn * b;
    for (int s = warp; s < nn; s += NW) {
      const int64_t src = L.nbr[e0 + s] * b;
      for (int t = wl; t < b; t += 32) cp_async_elem(win + s * b + t, xin + src + t);
    }
  }
  const int Wp = (W + 3) & ~3;
  for (int k = W + threadIdx.x; k < Wp; k += blockDim.x) win[k] = T(0);
  int64_t r0, r1;
  level_box_rows<T, FINE>(L, B, r0, r1);
  T* aux = reinterpret_cast<T*>(base + lay.aux);
  const int nr = (int)(r1 - r0);
  for (int j = 0; j < Ep::kStage; ++j) {
    if (!ep.stage(j)) continue;
    const T* sp = ep.src(j);
    for (int t = threadIdx.x; t < nr; t += blockDim.x) cp_async_elem(aux + j * L.max_box_rows + t, sp + r0 + t);
  }
  int64_t* rp = reinterpret_cast<int64_t*>(base + lay.rp);
  for (int t = threadIdx.x; t <= nr; t += blockDim.x) cp_async_elem(rp + t, L.row_ptr + r0 + t);
  if (FINE && L.row_order) {
    int32_t* od = reinterpret_cast<int32_t*>(base + lay.ord);
    for (int t = threadIdx.x; t < nr; t += blockDim.x) cp_async_elem(od + t, L.row_order + r0 + t);
  }
}

// The rows of a staged box: groups of G lanes per row, U steps of 4 entries per lane in flight;
// SP: software-pipelined row loop (the next chunk -- of the same row, or the group's next row --
// is loaded into registers before the current chunk is consumed, so loads stay in flight through
// the arithmetic and the group reduction).  Every thread of the CTA calls it (the epilogue
// pass follows a CTA barrier).
template <typename T, int G, bool FINE, class Ep, int U, bool SP>
__device__ __forceinline__ void level_compute(const LevelView<T>& L, const Ep& ep, const LevelSmem& lay, int64_t B,
                                              unsigned char* base, double& acc) {
  const int NG = blockDim.x / G;
  const int g = threadIdx.x / G, lane = threadIdx.x % G;
  const T* win = reinterpret_cast<const T*>(base);
  int64_t r0, r1;
  level_box_rows<T, FINE>(L, B, r0, r1);
  const int nr = (int)(r1 - r0);
  T* auxp[kAuxMax];
  for (int j = 0; j < kAuxMax; ++j) auxp[j] = reinterpret_cast<T*>(base + lay.aux) + j * L.max_box_rows;
  const int64_t* rp = reinterpret_cast<const int64_t*>(base + lay.rp);
  const int32_t* od = reinterpret_cast<const int32_t*>(base + lay.ord);
  // A group folds its lanes' sums down to kPL partials and parks them in shared memory; after
  // the rows, one thread per row adds its partials and applies the epilogue, so the epilogue's
  // loads and stores are coalesced over consecutive rows.  FP64 stops the shuffle tree at
  // kParkLanes partials: every FP64 instruction costs the FP64 pipe a whole warp's slot however
  // few of its lanes are active, so a tree level costs G slots per row and a serial add one,
  // and the epilogue's FP64 arithmetic runs on full warps instead of one lane per group.
  constexpr int kPL = sizeof(T) == 8 ? (G < kParkLanes ? G : kParkLanes) : 1;
  constexpr int kStride = sizeof(T) == 8 ? kParkStride : 1;
  T* ys = reinterpret_cast<T*>(base + lay.ys);
  auto finish = [&](int lr, T s) {
#pragma unroll
    for (int o = G / 2; o >= kPL; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o, G);
    if (lr >= 0 && lane < kPL) ys[lr * kStride + lane] = s;
  };
  // local row of this group at row-loop iteration `it` (-1 past the box's end); rows are
  // taken longest first on the fine level (host-built order) so the groups finish together
  auto row_at = [&](int it) -> int {
    const int i = it * NG + g;
    if (i >= nr) return -1;
    return (FINE && L.row_order) ? od[i] : i;
  };
  // warp-uniform trip count: every lane of a warp runs the same iterations so the
  // group shuffles always see the full warp; rows past the box end are masked.
  const int g_first = (threadIdx.x >> 5) * (32 / G);
  const int nit = (nr > g_first) ? (nr - g_first + NG - 1) / NG : 0;
  if constexpr (!SP) {
    for (int it = 0; it < nit; ++it) {
      const int lr = row_at(it);
      int64_t k0 = 0, k1 = 0;
      if (lr >= 0) { k0 = rp[lr]; k1 = rp[lr + 1]; }
      T a[2] = {T(0), T(0)};
      // U steps of 4 entries per lane are loaded before any is consumed: more bytes in flight
      for (int64_t k = k0 + 4 * lane; k < k1; k += 4 * G * U) {
        Chunk<T, U, FINE> c;
        c.load(L.vals, L.idx, k, k0, k1, G, L.keep);
        c.consume(win, a);
      }
      finish(lr, sizeof(T) == 8 ? a[0] : a[0] + a[1]);   // FP64: one chain
    }
  } else {
    int lr = row_at(0);
    int64_t k0 = 0, k1 = 0;
    if (lr >= 0) { k0 = rp[lr]; k1 = rp[lr + 1]; }
    int64_t k = k0 + 4 * lane;
    Chunk<T, U, FINE> cur;
    if (nit > 0) cur.load(L.vals, L.idx, k, k0, k1, G, L.keep);
    for (int it = 0; it < nit; ++it) {
      T a[2] = {T(0), T(0)};
      const int lr_now = lr;
      while (true) {
        // the next chunk: further along this row, or the first of the group's next row
        const bool same = k + 4 * G * U < k1;
        int64_t nk, nk0 = k0, nk1 = k1;
        int nlr = lr;
        if (same) {
          nk = k + 4 * G * U;
        } else {
          nlr = (it + 1 < nit) ? row_at(it + 1) : -1;
          nk0 = 0; nk1 = 0;
          if (nlr >= 0) { nk0 = rp[nlr]; nk1 = rp[nlr + 1]; }
          nk = nk0 + 4 * lane;
        }
        Chunk<T, U, FINE> nxt;
        nxt.load(L.vals, L.idx, nk, nk0, nk1, G, L.keep);   // loads nothing past the row's end
        cur.consume(win, a);
        cur = nxt;
        k = nk;
        if (!same) { lr = nlr; k0 = nk0; k1 = nk1; break; }
      }
      finish(lr_now, sizeof(T) == 8 ? a[0] : a[0] + a[1]);   // FP64: one chain
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < nr; t += blockDim.x) {
    T y = ys[t * kStride];
#pragma unroll
    for (int j = 1; j < kPL; ++j) y += ys[t * kStride + j];
    ep.post(r0 + t, t, y, auxp, acc);
  }
}

// PIPE: persistent CTAs with two stages (the next box staged while the current one computes).
// PF: an L2 bulk prefetch of each box's matrix slice.  SP: software-pipelined row loop.
template <typename T, int G, bool FINE, class Ep, int U, bool PIPE, bool PF, bool SP>
__global__ void __launch_bounds__(256, 4) level_kernel(LevelView<T> L, const T* __restrict__ xin, Ep ep,
                                                    double* __restrict__ part) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[8];
  const LevelSmem lay(sizeof(T), L.win_max, L.max_box_rows);
  double acc = 0.0;
  unsigned char* base0 = smem_raw;
  if constexpr (!PIPE) {
    for (int64_t B = blockIdx.x; B < L.nbox; B += gridDim.x) {
      if (PF) level_prefetch<T, FINE>(L, B);
      level_stage<T, FINE, Ep>(L, xin, ep, lay, B, base0);
      cp_async_wait_all();
      __syncthreads();
      level_compute<T, G, FINE, Ep, U, SP>(L, ep, lay, B, base0, acc);
      __syncthreads();
    }
  } else {
    // persistent CTAs: the next box's window is staged while the current box computes
    unsigned char* base1 = smem_raw + lay.total;
    int64_t B = blockIdx.x;
    if (B < L.nbox) { if (PF) level_prefetch<T, FINE>(L, B); level_stage<T, FINE, Ep>(L, xin, ep, lay, B, base0); }
    cp_async_commit_group();
    for (int k = 0; B < L.nbox; B += gridDim.x, ++k) {
      const int64_t nxt = B + gridDim.x;
      if (nxt < L.nbox) {
        if (PF) level_prefetch<T, FINE>(L, nxt);
        level_stage<T, FINE, Ep>(L, xin, ep, lay, nxt, (k & 1) ? base0 : base1);
      }
      cp_async_commit_group();
      cp_async_wait_group1();
      __syncthreads();
      level_compute<T, G, FINE, Ep, U, SP>(L, ep, lay, B, (k & 1) ? base1 : base0, acc);
      __syncthreads();
    }
  }
  if constexpr (Ep::kDot) {
    if (part != nullptr) {   // a product without a dot passes no partial buffer
      const double t = block_sum(acc, red);
      if (threadIdx.x == 0) part[blockIdx.x] = t;
    }
  }
}

template <typename T>
inline size_t level_smem_bytes(const LevelView<T>& L) {   // one stage: window, own-row vectors, row bounds
  return LevelSmem(sizeof(T), L.win_max, L.max_box_rows).total;
}

}  // namespace r3mg
