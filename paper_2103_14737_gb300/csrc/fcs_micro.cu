// fcs_micro.cu - throughput microbenchmarks of the units the hit path uses,
// the denominators of its roofline: Philox4x32-10 blocks, 32x32->64-bit
// integer multiplies (Philox's rounds), 3-input XORs, FP32 FMAs, the MUFU
// sine (the hit's sincos), 32-bit shared-memory loads (the staged tables),
// and float reductions into global memory (the deposit) at random addresses.  Each
// kernel runs independent chains in every thread of a full grid and folds its
// results into one word per thread, so no work can be optimised away.
#include <cstdio>

#include "fcs_internal.cuh"

namespace fcs {
namespace {

constexpr int kMbThreads = 256;

__global__ void __launch_bounds__(kMbThreads) k_mb_philox(uint32_t* out, int iters, uint32_t k0, uint32_t k1) {
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t acc = 0;
  for (int i = 0; i < iters; ++i) {
    const uint4 x = philox4x32_10(make_uint4((uint32_t)i, tid, 7u, 11u), k0, k1);
    acc ^= x.x ^ x.y ^ x.z ^ x.w;
  }
  out[tid] = acc;
}

// 8 independent chains of 32x32->64 multiplies per thread (2 per step each).
__global__ void __launch_bounds__(kMbThreads) k_mb_mulwide(uint32_t* out, int iters, uint32_t seed) {
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t a[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) a[j] = tid * 2654435761u + j + seed;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const uint64_t p = (uint64_t)a[j] * 0xD2511F53u;
      a[j] = (uint32_t)(p >> 32) ^ (uint32_t)p;
    }
  }
  uint32_t acc = 0;
#pragma unroll
  for (int j = 0; j < 8; ++j) acc ^= a[j];
  out[tid] = acc;
}

// 8 independent chains of 3-input XORs (LOP3) with adds to defeat folding.
__global__ void __launch_bounds__(kMbThreads) k_mb_lop3(uint32_t* out, int iters, uint32_t seed) {
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t a[8], b = tid ^ seed;
#pragma unroll
  for (int j = 0; j < 8; ++j) a[j] = tid + j * 977u;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] = (a[j] ^ (a[(j + 1) & 7] >> 3) ^ b) + 0x9E3779B9u;
  }
  uint32_t acc = 0;
#pragma unroll
  for (int j = 0; j < 8; ++j) acc ^= a[j];
  out[tid] = acc;
}

// 8 independent FP32 FMA chains.
__global__ void __launch_bounds__(kMbThreads) k_mb_ffma(float* out, int iters, float seed) {
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  float a[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) a[j] = seed + (float)(tid & 1023) * 1e-3f + (float)j;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] = fmaf(a[j], 0.999999f, 1e-7f);
  }
  float acc = 0.0f;
#pragma unroll
  for (int j = 0; j < 8; ++j) acc += a[j];
  out[tid] = acc;
}

// 8 independent chains of the hardware sine (__sinf).
__global__ void __launch_bounds__(kMbThreads) k_mb_mufu(float* out, int iters, float seed) {
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  float a[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) a[j] = seed + (float)(tid & 255) * 1e-3f + (float)j * 0.1f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] = __sinf(a[j]);
  }
  float acc = 0.0f;
#pragma unroll
  for (int j = 0; j < 8; ++j) acc += a[j];
  out[tid] = acc;
}

// 8 independent 128-bit shared-memory loads per thread and iteration (the
// hit kernel reads its staged tables with vector loads), lanes on distinct
// 16-byte slots, folded by XOR; the rate is counted in 32-bit words.
__global__ void __launch_bounds__(kMbThreads) k_mb_lds(uint32_t* out, int iters, uint32_t seed) {
  __shared__ uint4 s[1024];
  for (int i = threadIdx.x; i < 1024; i += blockDim.x)
    s[i] = make_uint4((uint32_t)i * 2654435761u ^ seed, (uint32_t)i, seed, (uint32_t)i * 7u);
  __syncthreads();
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  uint4 acc = make_uint4(tid, 0u, 0u, 0u);
  for (int i = 0; i < iters; ++i) {
    const uint32_t base = ((uint32_t)i * 256u + (acc.x & 1u)) & 767u;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const uint4 v = s[base + j * 32 + (threadIdx.x & 31)];
      acc.x ^= v.x;
      acc.y ^= v.y;
      acc.z ^= v.z;
      acc.w ^= v.w;
    }
  }
  out[tid] = acc.x ^ acc.y ^ acc.z ^ acc.w;
}

// Float reductions at pseudo-random addresses of an n-float array.
__global__ void __launch_bounds__(kMbThreads) k_mb_red(float* arr, int64_t n, int iters, uint32_t seed) {
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t s = tid * 2654435761u ^ seed;
  for (int i = 0; i < iters; ++i) {
    s = s * 1664525u + 1013904223u;  // LCG address stream
    const uint64_t idx = ((uint64_t)s * (uint64_t)n) >> 32;
    atomicAdd(arr + idx, 1.0f);
  }
}

// FP64 reductions at pseudo-random addresses of an n-double array (the
// accumulation rows' atomics).
__global__ void __launch_bounds__(kMbThreads) k_mb_red64(double* arr, int64_t n, int iters, uint32_t seed) {
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t s = tid * 2654435761u ^ seed;
  for (int i = 0; i < iters; ++i) {
    s = s * 1664525u + 1013904223u;  // LCG address stream
    const uint64_t idx = ((uint64_t)s * (uint64_t)n) >> 32;
    atomicAdd(arr + idx, 1.0);
  }
}

}  // namespace
}  // namespace fcs

using namespace fcs;

extern "C" int fcs_microbench(int32_t kind, int64_t size, int32_t iters, double* rate, cudaStream_t s) {
  if (!rate || iters < 1) return FCS_E_ARG;
  *rate = 0.0;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return FCS_E_CUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return FCS_E_CUDA;
  const int blocks = sms * (2048 / kMbThreads) * 4;  // four full waves of 256-thread blocks
  const int64_t threads = (int64_t)blocks * kMbThreads;
  void* buf = nullptr;
  const bool red = kind == FCS_MB_RED || kind == FCS_MB_RED64;
  const int64_t arr_n = red ? size : 0;
  if (arr_n < 0 || (red && arr_n < 1)) return FCS_E_ARG;
  const size_t elem = kind == FCS_MB_RED64 ? 8 : 4;
  // per-thread outputs (4 bytes), then the reduction array (8-byte aligned)
  const size_t arr_off = ((size_t)threads * 4 + 255) / 256 * 256;
  if (cudaMalloc(&buf, arr_off + (size_t)arr_n * elem) != cudaSuccess) return FCS_E_OOM;
  void* arr = (unsigned char*)buf + arr_off;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  auto launch = [&](int it) {
    switch (kind) {
      case FCS_MB_PHILOX: k_mb_philox<<<blocks, kMbThreads, 0, s>>>((uint32_t*)buf, it, 0x1234u, 0x5678u); break;
      case FCS_MB_MULWIDE: k_mb_mulwide<<<blocks, kMbThreads, 0, s>>>((uint32_t*)buf, it, 3u); break;
      case FCS_MB_LOP3: k_mb_lop3<<<blocks, kMbThreads, 0, s>>>((uint32_t*)buf, it, 5u); break;
      case FCS_MB_FFMA: k_mb_ffma<<<blocks, kMbThreads, 0, s>>>((float*)buf, it, 0.5f); break;
      case FCS_MB_RED: k_mb_red<<<blocks, kMbThreads, 0, s>>>((float*)arr, arr_n, it, 9u); break;
      case FCS_MB_RED64: k_mb_red64<<<blocks, kMbThreads, 0, s>>>((double*)arr, arr_n, it, 9u); break;
      case FCS_MB_MUFU: k_mb_mufu<<<blocks, kMbThreads, 0, s>>>((float*)buf, it, 0.3f); break;
      case FCS_MB_LDS: k_mb_lds<<<blocks, kMbThreads, 0, s>>>((uint32_t*)buf, it, 13u); break;
      default: break;
    }
  };
  int rc = FCS_OK;
  if (kind < FCS_MB_PHILOX || kind > FCS_MB_RED64) rc = FCS_E_ARG;
  float ms = 0.0f;
  if (rc == FCS_OK) {
    if (red) cudaMemsetAsync(arr, 0, (size_t)arr_n * elem, s);
    launch(iters);  // warm-up
    cudaEventRecord(e0, s);
    launch(iters);
    cudaEventRecord(e1, s);
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess ||
        cudaGetLastError() != cudaSuccess)
      rc = FCS_E_CUDA;
  }
  if (rc == FCS_OK && ms > 0.0f) {
    // operations per thread per iteration of each kernel
    const double per = (kind == FCS_MB_PHILOX || red) ? 1.0 : (kind == FCS_MB_LDS) ? 32.0 : 8.0;
    *rate = (double)threads * iters * per / (ms * 1e-3);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(buf);
  return rc;
}
