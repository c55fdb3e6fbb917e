// Device characterisation for the FP64 roofline: sustained FP64 FMA and FP64 tensor-core
// (mma.sync m8n8k4) rates of the current GPU.  The FP64 level kernels do one FMA per 8-10
// bytes of matrix stream; on a part whose FP64 rate is low next to its memory bandwidth they
// are bound by the FP64 pipe, and this measurement is the denominator of that bound.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "../../include/r3mg.h"

namespace {

constexpr int kChains = 8;   // independent FMA chains per thread (hides the pipe latency)

__global__ void __launch_bounds__(256) k_probe_fma(double* out, int iters, double m, double c) {
  double a[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) a[j] = 1e-3 * (threadIdx.x + j);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < kChains; ++j) a[j] = fma(a[j], m, c);
  }
  double s = 0.0;
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += a[j];
  if (s == 12345.678) out[blockIdx.x] = s;   // never true for the probe's inputs; keeps the chains live
}

__global__ void __launch_bounds__(256) k_probe_dmma(double* out, int iters, double m) {
  double c[kChains / 2][2];
#pragma unroll
  for (int j = 0; j < kChains / 2; ++j) { c[j][0] = 1e-3 * threadIdx.x; c[j][1] = 1e-3 * j; }
  const double a = m * (1 + (threadIdx.x & 3)), b = m;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < kChains / 2; ++j)
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
                   : "+d"(c[j][0]), "+d"(c[j][1])
                   : "d"(a), "d"(b));
  }
  double s = 0.0;
#pragma unroll
  for (int j = 0; j < kChains / 2; ++j) s += c[j][0] + c[j][1];
  if (s == 12345.678) out[blockIdx.x] = s;
}

}  // namespace

extern "C" r3mg_status r3mg_measure_fp64_rates(double* fma_tflops, double* mma_tflops, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return R3MG_E_CUDA;
  const int grid = nsm * 8, threads = 256;
  double* out = nullptr;
  if (cudaMalloc(&out, sizeof(double) * grid) != cudaSuccess) return R3MG_E_OOM;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  r3mg_status st = R3MG_OK;
  auto time_ms = [&](auto launch) -> float {
    launch();   // warm-up
    cudaEventRecord(e0, s);
    launch();
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    return ms;
  };
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) st = R3MG_E_CUDA;
  if (st == R3MG_OK) {
    const int it_fma = 1 << 14, it_mma = 1 << 13;
    const float t_fma = time_ms([&] { k_probe_fma<<<grid, threads, 0, s>>>(out, it_fma, 0.9999999, 1e-9); });
    const float t_mma = time_ms([&] { k_probe_dmma<<<grid, threads, 0, s>>>(out, it_mma, 0.5); });
    if (cudaGetLastError() != cudaSuccess || !(t_fma > 0.f) || !(t_mma > 0.f)) st = R3MG_E_CUDA;
    else {
      const double fma_flop = 2.0 * kChains * (double)it_fma * grid * threads;
      const double warps = (double)grid * threads / 32.0;
      const double mma_flop = 512.0 * (kChains / 2) * (double)it_mma * warps;   // 2 x 8 x 8 x 4 per warp-level mma
      if (fma_tflops) *fma_tflops = fma_flop / (t_fma * 1e-3) / 1e12;
      if (mma_tflops) *mma_tflops = mma_flop / (t_mma * 1e-3) / 1e12;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(out);
  return st;
}

// ---------------------------------------------------------------- bounded-wait self-test
// One CTA waits on an mbarrier phase whose arrival announces 16 bytes that no copy ever
// delivers, so every wait must run out after `limit` clock64 cycles; the kernel records the
// expiry, invalidates the barrier and returns (nothing is in flight).
namespace {

__global__ void k_wait_selftest(long long limit, int* flag) {
  __shared__ __align__(8) uint64_t bar;
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(&bar);
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(a) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], 16;\n" ::"r"(a) : "memory");
  __syncthreads();
  bool done = false;
  const long long t0 = clock64();
  while (!done && clock64() - t0 <= limit) {
    uint32_t ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(ok) : "r"(a) : "memory");
    done = ok != 0;
  }
  if (!done) atomicExch(flag, 1);
  __syncthreads();
  if (threadIdx.x == 0) asm volatile("mbarrier.inval.shared::cta.b64 [%0];\n" ::"r"(a) : "memory");
}

}  // namespace

extern "C" r3mg_status r3mg_wait_selftest(long long limit_cycles, int* expired_out, void* stream) {
  if (limit_cycles < 1 || limit_cycles > 4000000000LL) return R3MG_E_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  int* flag = nullptr;
  if (cudaMalloc(&flag, sizeof(int)) != cudaSuccess) return R3MG_E_OOM;
  int host = 0;
  r3mg_status st = R3MG_OK;
  if (cudaMemsetAsync(flag, 0, sizeof(int), s) != cudaSuccess) st = R3MG_E_CUDA;
  if (st == R3MG_OK) {
    k_wait_selftest<<<1, 32, 0, s>>>(limit_cycles, flag);
    if (cudaGetLastError() != cudaSuccess || cudaMemcpyAsync(&host, flag, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      st = R3MG_E_CUDA;
  }
  cudaFree(flag);
  if (expired_out) *expired_out = host;
  if (st != R3MG_OK) return st;
  return host ? R3MG_E_TIMEOUT : R3MG_OK;
}
