// Issue-rate microbenchmarks of this GPU (pic_measure_alu_peaks): the
// denominators of the collision kernel's roofline. Each kernel runs
// independent dependency chains of one instruction kind in every thread of
// a full grid (blocks = SMs x resident blocks), so the rate it reaches is
// the issue rate of that pipe, not a latency. The inline PTX pins each
// operation to one instruction (mad.lo.u32 -> IMAD, lop3.b32 -> LOP3,
// fma.rn.f32 -> FFMA, fma.rn.f64 -> DFMA); a predicated store of the chains'
// result that never fires keeps them alive.
#include <cuda_runtime.h>
#include <stdint.h>

#include "pic_internal.cuh"

namespace pic {
namespace {

constexpr int kPeakThreads = 256;
constexpr int kChains = 8;
constexpr int kUnroll = 16;

__global__ void __launch_bounds__(kPeakThreads) k_peak_imad(uint32_t* sink, int iters, uint32_t seed) {
  uint32_t a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) a[c] = seed + threadIdx.x * (c + 1) + blockIdx.x;
  const uint32_t m = seed | 1u, d = seed ^ 0x5bd1e995u;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
      for (int c = 0; c < kChains; ++c) asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(a[c]) : "r"(m), "r"(d));
    }
  }
  uint32_t s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s ^= a[c];
  if (s == 0x12345678u) sink[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kPeakThreads) k_peak_lop3(uint32_t* sink, int iters, uint32_t seed) {
  uint32_t a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) a[c] = seed + threadIdx.x * (c + 3) + blockIdx.x;
  const uint32_t b = seed * 0x9E3779B9u, d = seed ^ 0xBB67AE85u;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
      for (int c = 0; c < kChains; ++c)
        asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(a[c]) : "r"(b), "r"(d));  // a ^ b ^ d
    }
  }
  uint32_t s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += a[c];
  if (s == 0x12345678u) sink[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kPeakThreads) k_peak_ffma(uint32_t* sink, int iters, uint32_t seed) {
  float a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) a[c] = (float)(seed & 255u) * 1e-3f + (float)(threadIdx.x * (c + 1)) * 1e-6f;
  const float m = 0.999999f, d = 1e-7f * (float)(seed & 7u);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
      for (int c = 0; c < kChains; ++c) asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(a[c]) : "f"(m), "f"(d));
    }
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += a[c];
  if (s == 1234.5f) sink[blockIdx.x] = 1u;
}

__global__ void __launch_bounds__(kPeakThreads) k_peak_dfma(uint32_t* sink, int iters, uint32_t seed) {
  double a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) a[c] = (double)(seed & 255u) * 1e-3 + (double)(threadIdx.x * (c + 1)) * 1e-6;
  const double m = 0.999999, d = 1e-7 * (double)(seed & 7u);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
      for (int c = 0; c < kChains; ++c) asm volatile("fma.rn.f64 %0, %0, %1, %2;" : "+d"(a[c]) : "d"(m), "d"(d));
    }
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += a[c];
  if (s == 1234.5) sink[blockIdx.x] = 1u;
}

// Philox4x32-10 blocks as the collision kernel forms them (round keys in the
// kernel parameters, 32 x 32 -> 64 products); two independent blocks per
// thread per iteration
struct PhiloxPeakArgs {
  uint32_t rk[2][10];
  uint32_t* sink;
  int iters;
};

__global__ void __launch_bounds__(kPeakThreads) k_peak_philox(PhiloxPeakArgs a) {
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t acc = 0;
  for (int i = 0; i < a.iters; ++i) {
    const U4 x = philox_rk<true>((uint32_t)i, t, 0u, acc & 1u, a.rk);
    const U4 y = philox_rk<true>((uint32_t)i, t, 1u, acc & 1u, a.rk);
    acc += x.x ^ x.y ^ x.z ^ x.w ^ y.x ^ y.y ^ y.z ^ y.w;
  }
  if (acc == 0x12345678u) a.sink[blockIdx.x] = acc;
}

}  // namespace
}  // namespace pic

using namespace pic;

extern "C" pic_status pic_measure_alu_peaks(void* cuda_stream, double out[5]) {
  if (!out) return PIC_EINVAL;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                cudaSuccess) {
    cudaGetLastError();
    return PIC_ECUDA;
  }
  uint32_t* sink = nullptr;
  if (cudaMallocAsync((void**)&sink, 4096 * sizeof(uint32_t), st) != cudaSuccess) {
    cudaGetLastError();
    return PIC_ENOMEM;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t err = cudaEventCreate(&e0);
  if (err == cudaSuccess) err = cudaEventCreate(&e1);
  // 8 blocks of 256 threads per SM (2048 threads: full occupancy at <= 32
  // registers, enough warps to cover every pipe's latency)
  const int blocks = sms * 8;
  const double threads = (double)blocks * kPeakThreads;
  auto timed = [&](auto launch, double ops_per_thread) -> double {
    launch();  // warm-up (clocks up, code loaded)
    if (err == cudaSuccess) err = cudaEventRecord(e0, st);
    launch();
    if (err == cudaSuccess) err = cudaEventRecord(e1, st);
    if (err == cudaSuccess) err = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
    if (err == cudaSuccess) err = cudaGetLastError();
    return (err == cudaSuccess && ms > 0.f) ? threads * ops_per_thread / (ms * 1e-3) : 0.0;
  };
  const int it32 = 4096, it64 = 128, itp = 1024;
  const double per32 = (double)it32 * kUnroll * kChains, per64 = (double)it64 * kUnroll * kChains;
  out[0] = timed([&] { k_peak_imad<<<blocks, kPeakThreads, 0, st>>>(sink, it32, 0x1234567u); }, per32);
  out[1] = timed([&] { k_peak_lop3<<<blocks, kPeakThreads, 0, st>>>(sink, it32, 0x1234567u); }, per32);
  out[2] = timed([&] { k_peak_ffma<<<blocks, kPeakThreads, 0, st>>>(sink, it32, 0x1234567u); }, per32);
  out[3] = timed([&] { k_peak_dfma<<<blocks, kPeakThreads, 0, st>>>(sink, it64, 0x1234567u); }, per64);
  PhiloxPeakArgs pa;
  for (int r = 0; r < 10; ++r) {
    pa.rk[0][r] = 0x12345678u + (uint32_t)r * 0x9E3779B9u;
    pa.rk[1][r] = 0x9abcdef0u + (uint32_t)r * 0xBB67AE85u;
  }
  pa.sink = sink;
  pa.iters = itp;
  out[4] = timed([&] { k_peak_philox<<<blocks, kPeakThreads, 0, st>>>(pa); }, 2.0 * itp);
  cudaFreeAsync(sink, st);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (err != cudaSuccess) {
    cudaGetLastError();
    return PIC_ECUDA;
  }
  return cudaStreamSynchronize(st) == cudaSuccess ? PIC_OK : PIC_ECUDA;
}

extern "C" pic_status pic_measure_link(void* host, uint64_t bytes, void* cuda_stream, double out[2]) {
  if (!host || bytes == 0 || !out) return PIC_EINVAL;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, host) != cudaSuccess) {
    cudaGetLastError();
    return PIC_EINVAL;
  }
  if (at.type != cudaMemoryTypeHost) return PIC_EINVAL;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  void* dev = nullptr;
  if (cudaMallocAsync(&dev, (size_t)bytes, st) != cudaSuccess) {
    cudaGetLastError();
    return PIC_ENOMEM;
  }
  cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
  cudaError_t err = cudaSuccess;
  for (int i = 0; i < 3 && err == cudaSuccess; ++i) err = cudaEventCreate(&ev[i]);
  const int reps = 3;
  // warm-up, one copy each way
  if (err == cudaSuccess) err = cudaMemcpyAsync(dev, host, (size_t)bytes, cudaMemcpyHostToDevice, st);
  if (err == cudaSuccess) err = cudaMemcpyAsync(host, dev, (size_t)bytes, cudaMemcpyDeviceToHost, st);
  if (err == cudaSuccess) err = cudaEventRecord(ev[0], st);
  for (int r = 0; r < reps && err == cudaSuccess; ++r)
    err = cudaMemcpyAsync(dev, host, (size_t)bytes, cudaMemcpyHostToDevice, st);
  if (err == cudaSuccess) err = cudaEventRecord(ev[1], st);
  for (int r = 0; r < reps && err == cudaSuccess; ++r)
    err = cudaMemcpyAsync(host, dev, (size_t)bytes, cudaMemcpyDeviceToHost, st);
  if (err == cudaSuccess) err = cudaEventRecord(ev[2], st);
  if (err == cudaSuccess) err = cudaEventSynchronize(ev[2]);
  float ms[2] = {0.f, 0.f};
  if (err == cudaSuccess) err = cudaEventElapsedTime(&ms[0], ev[0], ev[1]);
  if (err == cudaSuccess) err = cudaEventElapsedTime(&ms[1], ev[1], ev[2]);
  for (int i = 0; i < 2; ++i) out[i] = (err == cudaSuccess && ms[i] > 0.f) ? reps * (double)bytes / (ms[i] * 1e-3) : 0.0;
  cudaFreeAsync(dev, st);
  for (int i = 0; i < 3; ++i)
    if (ev[i]) cudaEventDestroy(ev[i]);
  if (err != cudaSuccess) {
    cudaGetLastError();
    return PIC_ECUDA;
  }
  return cudaStreamSynchronize(st) == cudaSuccess ? PIC_OK : PIC_ECUDA;
}
