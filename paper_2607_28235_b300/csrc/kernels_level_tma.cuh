// Persistent, TMA-streamed level operator kernel (sm_100+ bulk async copies).
//
// The work of a level is a list of items (a box, or a run of rows of one box when the box's
// matrix slice exceeds one stage).  Each CTA walks its items in order with a two-stage
// pipeline: while the 8 warps compute item k from shared memory, one elected thread has
// already issued the bulk copies (cp.async.bulk, completion on an mbarrier) of item k+1's
// contiguous matrix slice (values, and 16-bit window indices on the fine level), and every
// thread has issued cp.async copies of item k+1's window (the input vector over the box's
// neighbour boxes) and of the item's own-row vector entries the epilogue needs.  The HBM
// stream therefore never waits on register-held loads: the copy engine keeps a whole item
// (tens of KB per SM) in flight.  Every mbarrier wait is bounded (about one second of
// clock64 cycles by default); on expiry the kernel raises an error flag, waits (bounded again)
// for the bulk copies it still has in flight and for its cp.async copies, and returns.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "kernels_level.cuh"

namespace r3mg {

constexpr int kAux = kAuxMax;                 // own-row vectors an epilogue may stage
constexpr long long kWaitCycles = 2000000000LL;  // bounded mbarrier wait (~1 s at 2 GHz)

// Per-item descriptor, built on the host and bulk-copied to shared memory two items ahead:
//   int64 e0, e1        matrix entry range of the item (multiples of 4)
//   int64 rb            first row
//   int32 nr, nn        rows, window segments
//   int32 W, pad        window length
//   nn x {int64 src; int32 wo; int32 len}   window segments: xin[src .. src+len) -> win[wo ..]
//   (nr + 1) x int32    row offsets relative to e0
// padded to a multiple of 16 bytes.
struct ItemDesc {
  int64_t e0, e1, rb;
  int32_t nr, nn, W, pad;
};
struct SegDesc {
  int64_t src;
  int32_t wo, len;
};

template <typename T>
struct TmaView {
  LevelView<T> L;
  const unsigned char* desc = nullptr;  // descriptor blob
  const int64_t* desc_off = nullptr;    // nitems + 1 byte offsets (multiples of 16)
  int64_t nitems = 0;
  int stage_entries = 0;                // matrix entries per stage buffer (multiple of 8)
  int max_item_rows = 0;                // rows per item at most
  int desc_max = 0;                     // largest descriptor in bytes (multiple of 16)
  int* err = nullptr;                   // set to 1 when a bounded wait expires
  long long wait_cycles = kWaitCycles;  // limit of every mbarrier wait
  int withhold_first = 0;               // test of the expiry path: CTA 0 announces its first
                                        // descriptor copy but never issues it, so that wait runs out
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// bounded wait: true on completion, false (and err raised when err is given) after `limit` cycles
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, int* err,
                                                  long long limit = kWaitCycles) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > limit) {
      if (err) atomicExch(err, 1);
      return false;
    }
  }
  return true;
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

template <typename T, bool FINE>
struct TmaLayout {  // shared-memory carve-up (byte offsets), shared by host and device
  size_t dsc[3], vals[2], idx[2], win[2], aux[2], total;
  __host__ __device__ TmaLayout(int SE, int win_max, int rmax, int dmax) {
    size_t o = 128;  // five mbarriers + padding
    for (int s = 0; s < 3; ++s) { dsc[s] = o; o += (size_t)dmax; o = (o + 127) & ~(size_t)127; }
    for (int s = 0; s < 2; ++s) { vals[s] = o; o += (size_t)SE * sizeof(T); o = (o + 127) & ~(size_t)127; }
    for (int s = 0; s < 2; ++s) {
      idx[s] = o;
      if (FINE) { o += (size_t)SE * 2 + 32; o = (o + 127) & ~(size_t)127; }
    }
    for (int s = 0; s < 2; ++s) { win[s] = o; o += (size_t)win_max * sizeof(T); o = (o + 127) & ~(size_t)127; }
    for (int s = 0; s < 2; ++s) { aux[s] = o; o += (size_t)kAux * rmax * sizeof(T); o = (o + 127) & ~(size_t)127; }
    total = o;
  }
};

template <typename T, int G, bool FINE, class Ep>
__global__ void __launch_bounds__(1024, 1) level_kernel_tma(TmaView<T> V, const T* __restrict__ xin, Ep ep,
                                                           double* __restrict__ part) {
  extern __shared__ __align__(128) unsigned char tsm[];
  __shared__ double red[32];
  const LevelView<T>& L = V.L;
  const TmaLayout<T, FINE> lay(V.stage_entries, L.win_max, V.max_item_rows, V.desc_max);
  uint64_t* bar = reinterpret_cast<uint64_t*>(tsm);        // [0..1] matrix stages
  uint64_t* dbar = bar + 2;                                 // [0..2] descriptor ring
  const int tid = threadIdx.x, warp = tid >> 5, wl = tid & 31;
  const int NT = blockDim.x, NW = NT >> 5;   // 256, 512 or 1024 threads
  const int NG = NT / G;
  const int g = tid / G, lane = tid % G;
  if (tid == 0) {
    for (int j = 0; j < 5; ++j) mbar_init(&bar[j], 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();
  // thread 0 tracks the barriers (0-1 stages, 2-4 descriptor ring) with a phase in flight and
  // the parity of that phase, so that an expired wait can drain every copy it issued
  uint32_t pend = 0, par = 0;
  auto issued = [&](int j) { pend |= 1u << j; };
  auto completed = [&](int j) { pend &= ~(1u << j); par ^= 1u << j; };
  auto drain = [&]() {   // after an expired wait: no CTA leaves with a copy into its shared memory in flight
    if (tid == 0)
      for (int j = 0; j < 5; ++j)
        if ((pend >> j) & 1u) mbar_wait_bounded(&bar[j], (par >> j) & 1u, nullptr, kWaitCycles);
    cp_async_wait_all();
  };

  bool withheld = false;
  auto fetch_desc = [&](int64_t it, int j) {   // thread 0 only
    const int64_t o = V.desc_off[it];
    const uint32_t bytes = (uint32_t)(V.desc_off[it + 1] - o);
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    mbar_expect_tx(&dbar[j], bytes);
    issued(2 + j);
    if (V.withhold_first && blockIdx.x == 0 && !withheld) { withheld = true; return; }
    bulk_g2s(tsm + lay.dsc[j], V.desc + o, bytes, &dbar[j]);
  };

  // item copies: matrix slice by the copy engine, window and own-row vectors by cp.async
  auto issue = [&](const unsigned char* dsc, int st) {
    const ItemDesc* hd = reinterpret_cast<const ItemDesc*>(dsc);
    const int64_t e0 = hd->e0, e1 = hd->e1, rb = hd->rb;
    const int nr = hd->nr, nn = hd->nn, W = hd->W;
    if (tid == 0) {
      asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
      const uint32_t bv = (uint32_t)((e1 - e0) * (int64_t)sizeof(T));
      uint32_t bi = 0;
      int64_t ia = 0;
      if (FINE) {
        ia = e0 & ~(int64_t)7;                              // 16-byte aligned start of the index run
        bi = (uint32_t)((((e1 - ia) * 2) + 15) & ~(int64_t)15);
      }
      mbar_expect_tx(&bar[st], bv + bi);
      issued(st);
      bulk_g2s(tsm + lay.vals[st], L.vals + e0, bv, &bar[st]);
      if (FINE) bulk_g2s(tsm + lay.idx[st], L.idx + ia, bi, &bar[st]);
    }
    T* win = reinterpret_cast<T*>(tsm + lay.win[st]);
    const SegDesc* seg = reinterpret_cast<const SegDesc*>(dsc + sizeof(ItemDesc));
    for (int sI = warp; sI < nn; sI += NW) {
      const SegDesc sd = seg[sI];
      for (int t = wl; t < sd.len; t += 32) cp_async_elem(win + sd.wo + t, xin + sd.src + t);
    }
    // block rows are padded to a multiple of 4 entries with value 0: a zero window tail keeps
    // the padded products finite
    const int Wp = (W + 3) & ~3;
    for (int t = W + tid; t < Wp; t += NT) win[t] = T(0);
    T* aux = reinterpret_cast<T*>(tsm + lay.aux[st]);
    for (int j = 0; j < Ep::kStage; ++j) {
      if (!ep.stage(j)) continue;
      const T* sp = ep.src(j);
      for (int t = tid; t < nr; t += NT) cp_async_elem(aux + j * V.max_item_rows + t, sp + rb + t);
    }
    cp_async_commit();
  };

  double acc = 0.0;
  const int64_t it0 = blockIdx.x, G0 = gridDim.x;
  bool alive = true;
  if (it0 < V.nitems) {
    if (tid == 0) {
      fetch_desc(it0, 0);
      if (it0 + G0 < V.nitems) fetch_desc(it0 + G0, 1);
    }
    alive = mbar_wait_bounded(&dbar[0], 0, V.err, V.wait_cycles);
    if (__syncthreads_or(!alive)) { drain(); return; }
    completed(2);
    issue(tsm + lay.dsc[0], 0);
  } else {
    cp_async_commit();
  }
  int k = 0;
  for (int64_t it = it0; it < V.nitems; it += G0, ++k) {
    const int st = k & 1;
    const int64_t nxt = it + G0, nxt2 = it + 2 * G0;
    if (tid == 0 && nxt2 < V.nitems) fetch_desc(nxt2, (k + 2) % 3);
    if (nxt < V.nitems) {
      const int j = (k + 1) % 3;
      alive = mbar_wait_bounded(&dbar[j], (uint32_t)(((k + 1) / 3) & 1), V.err, V.wait_cycles);
      if (__syncthreads_or(!alive)) { drain(); return; }
      completed(2 + j);
      issue(tsm + lay.dsc[j], st ^ 1);
    } else {
      cp_async_commit();
    }
    cp_async_wait_1();
    alive = mbar_wait_bounded(&bar[st], (uint32_t)((k >> 1) & 1), V.err, V.wait_cycles);
    if (__syncthreads_or(!alive)) { drain(); return; }   // error flag raised; nothing is consumed
    completed(st);
    const unsigned char* dsc = tsm + lay.dsc[k % 3];
    const ItemDesc* hd = reinterpret_cast<const ItemDesc*>(dsc);
    const int64_t e0 = hd->e0, rb = hd->rb;
    const int nr = hd->nr;
    const int32_t* roff = reinterpret_cast<const int32_t*>(dsc + sizeof(ItemDesc) + sizeof(SegDesc) * hd->nn);
    const T* vb = reinterpret_cast<const T*>(tsm + lay.vals[st]);
    const uint16_t* ib = reinterpret_cast<const uint16_t*>(tsm + lay.idx[st]) + (FINE ? (e0 & 7) : 0);
    const T* win = reinterpret_cast<const T*>(tsm + lay.win[st]);
    T* auxp[kAux];
    for (int j = 0; j < kAux; ++j) auxp[j] = reinterpret_cast<T*>(tsm + lay.aux[st]) + j * V.max_item_rows;
    const int g_first = warp * (32 / G);
    for (int base = 0; base + g_first < nr; base += NG) {
      const int lr = base + g;
      const bool ok = lr < nr;
      int k0 = 0, k1 = 0;
      if (ok) { k0 = roff[lr]; k1 = roff[lr + 1]; }
      T s = T(0);   // FP64: one fused multiply-add per stored entry (see the register kernel)
      for (int kk = k0 + 4 * lane; kk < k1; kk += 4 * G) {
        T v[4];
        if constexpr (sizeof(T) == 4) {
          const float4 a = *reinterpret_cast<const float4*>(vb + kk);
          v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
        } else {
          const double2 a = *reinterpret_cast<const double2*>(vb + kk);
          const double2 c = *reinterpret_cast<const double2*>(vb + kk + 2);
          v[0] = a.x; v[1] = a.y; v[2] = c.x; v[3] = c.y;
        }
        int wi[4];
        if constexpr (FINE) {
          const uint2 q = *reinterpret_cast<const uint2*>(ib + kk);
          wi[0] = q.x & 0xffff; wi[1] = q.x >> 16; wi[2] = q.y & 0xffff; wi[3] = q.y >> 16;
        } else {
          // coarse rows: dense blocks laid out over the window in slot order
          const int t = kk - k0;
          wi[0] = t; wi[1] = t + 1; wi[2] = t + 2; wi[3] = t + 3;
        }
        if constexpr (sizeof(T) == 8) {
#pragma unroll
          for (int j = 0; j < 4; ++j) s = fma_rn(v[j], win[wi[j]], s);
        } else {
          s += v[0] * win[wi[0]] + v[1] * win[wi[1]] + v[2] * win[wi[2]] + v[3] * win[wi[3]];
        }
      }
      s = group_sum<G>(s);
      if (ok && lane == 0) ep.post(rb + lr, lr, s, auxp, acc);
    }
    __syncthreads();
  }
  if constexpr (Ep::kDot) {
    if (part != nullptr) {   // a product without a dot passes no partial buffer
      const double t = block_sum(acc, red);
      if (threadIdx.x == 0) part[blockIdx.x] = t;
    }
  }
}

}  // namespace r3mg
