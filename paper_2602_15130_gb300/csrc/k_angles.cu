// Scattering-angle CDF errors (Sec. 4.4) from the recorded histograms.
//
// The collision kernels put every recorded collision into bin
// floor(u PIC_ANGLE_BINS) of u = F^M(alpha) for alpha in {chi, eps}. Here a
// bin b with count c and C samples in the bins before it stands for c
// samples at its centre m_b = (b + 1/2) / PIC_ANGLE_BINS with empirical
// CDF values (C + k)/N, k = 1..c, so its share of sum_r e_r^2 is the
// closed form
//     c a^2 + a c (c + 1)/N + c (c + 1)(2c + 1)/(6 N^2),   a = C/N - m_b,
// and its largest |e| is max(|a + 1/N|, |a + c/N|). Three launches: chunk
// totals, per-chunk prefix + closed forms, one block for the totals; every
// sum runs in a fixed order.
#include <math.h>

#include "pic_internal.cuh"

namespace pic {
namespace {

constexpr int kAT = 256;
constexpr int kChunk = PIC_ANGLE_BINS / kAngleBlocks;
constexpr int kPer = kChunk / kAT;
static_assert(kChunk % kAT == 0, "chunk must split evenly over the block");

__device__ unsigned long long block_sum_u64(unsigned long long v, unsigned long long* sh) {
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  unsigned long long t = 0;
  for (int i = 0; i < kAT / 32; ++i) t += sh[i];
  return t;
}

__device__ unsigned long long block_max_u64(unsigned long long v, unsigned long long* sh) {
  for (int off = 16; off > 0; off >>= 1) {
    const unsigned long long o = __shfl_xor_sync(0xffffffffu, v, off);
    v = o > v ? o : v;
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  unsigned long long t = 0;
  for (int i = 0; i < kAT / 32; ++i) t = sh[i] > t ? sh[i] : t;
  return t;
}

// exclusive prefix of one u64 per thread in thread order
__device__ unsigned long long block_exclusive_u64(unsigned long long v, unsigned long long* sh) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  unsigned long long inc = v;
  for (int off = 1; off < 32; off <<= 1) {
    const unsigned long long o = __shfl_up_sync(0xffffffffu, inc, off);
    if (lane >= off) inc += o;
  }
  __syncthreads();
  if (lane == 31) sh[w] = inc;
  __syncthreads();
  unsigned long long base = 0;
  for (int i = 0; i < w; ++i) base += sh[i];
  return base + inc - v;
}

__device__ void block_sum_max_f64(double& s, double& m, double* sh) {
  for (int off = 16; off > 0; off >>= 1) {
    s += __shfl_xor_sync(0xffffffffu, s, off);
    m = fmax(m, __shfl_xor_sync(0xffffffffu, m, off));
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) {
    sh[w] = s;
    sh[kAT / 32 + w] = m;
  }
  __syncthreads();
  s = 0.0;
  m = 0.0;
  for (int i = 0; i < kAT / 32; ++i) {
    s += sh[i];
    m = fmax(m, sh[kAT / 32 + i]);
  }
}

// 1: totals and maxima of every chunk (block = (angle, chunk))
__global__ void __launch_bounds__(kAT) k_ang_chunks(const unsigned long long* __restrict__ hist,
                                                     unsigned long long* __restrict__ bsum) {
  __shared__ unsigned long long sh[kAT / 32];
  const int a = blockIdx.x / kAngleBlocks, ch = blockIdx.x % kAngleBlocks;
  const unsigned long long* h = hist + (size_t)a * PIC_ANGLE_BINS + (size_t)ch * kChunk;
  unsigned long long s = 0, m = 0;
  for (int i = threadIdx.x; i < kChunk; i += kAT) {
    const unsigned long long c = h[i];
    s += c;
    m = c > m ? c : m;
  }
  s = block_sum_u64(s, sh);
  m = block_max_u64(m, sh);
  if (threadIdx.x == 0) {
    bsum[blockIdx.x] = s;
    bsum[2 * kAngleBlocks + blockIdx.x] = m;
  }
}

// 2: prefix counts and the closed-form shares of one chunk
__global__ void __launch_bounds__(kAT) k_ang_errors(const unsigned long long* __restrict__ hist,
                                                     const unsigned long long* __restrict__ bsum,
                                                     double* __restrict__ part) {
  __shared__ unsigned long long sh[kAT / 32];
  __shared__ double shd[kAT / 16];
  const int a = blockIdx.x / kAngleBlocks, ch = blockIdx.x % kAngleBlocks;
  const unsigned long long* bs = bsum + (size_t)a * kAngleBlocks;
  unsigned long long off = 0, tot = 0;
  for (int i = threadIdx.x; i < kAngleBlocks; i += kAT) {
    tot += bs[i];
    if (i < ch) off += bs[i];
  }
  off = block_sum_u64(off, sh);
  tot = block_sum_u64(tot, sh);
  if (tot == 0) {
    if (threadIdx.x == 0) {
      part[2 * blockIdx.x] = 0.0;
      part[2 * blockIdx.x + 1] = 0.0;
    }
    return;
  }
  const double N = (double)tot, invN = 1.0 / N;
  const int b0 = threadIdx.x * kPer;
  const unsigned long long* h = hist + (size_t)a * PIC_ANGLE_BINS + (size_t)ch * kChunk + b0;
  unsigned long long cnt[kPer];
  unsigned long long ls = 0;
#pragma unroll
  for (int k = 0; k < kPer; ++k) {
    cnt[k] = h[k];
    ls += cnt[k];
  }
  unsigned long long C = off + block_exclusive_u64(ls, sh);
  double S = 0.0, M = 0.0;
  const double binw = 1.0 / (double)PIC_ANGLE_BINS;
#pragma unroll
  for (int k = 0; k < kPer; ++k) {
    const unsigned long long c = cnt[k];
    if (c) {
      const double m = ((double)(ch * kChunk + b0 + k) + 0.5) * binw;
      const double av = (double)C * invN - m;
      const double cd = (double)c;
      S += cd * av * av + av * cd * (cd + 1.0) * invN + cd * (cd + 1.0) * (2.0 * cd + 1.0) * invN * invN / 6.0;
      M = fmax(M, fmax(fabs(av + invN), fabs(av + cd * invN)));
      C += c;
    }
  }
  block_sum_max_f64(S, M, shd);
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = S;
    part[2 * blockIdx.x + 1] = M;
  }
}

// 3: one block; out[4 a + 0..3] = eps_2, eps_inf, N, largest bin count
__global__ void __launch_bounds__(kAT) k_ang_final(const double* __restrict__ part,
                                                    const unsigned long long* __restrict__ bsum,
                                                    double* __restrict__ out) {
  __shared__ unsigned long long sh[kAT / 32];
  __shared__ double shd[kAT / 16];
  for (int a = 0; a < 2; ++a) {
    double S = 0.0, M = 0.0;
    unsigned long long tot = 0, mb = 0;
    for (int i = threadIdx.x; i < kAngleBlocks; i += kAT) {
      const int b = a * kAngleBlocks + i;
      S += part[2 * b];
      M = fmax(M, part[2 * b + 1]);
      tot += bsum[b];
      const unsigned long long x = bsum[2 * kAngleBlocks + b];
      mb = x > mb ? x : mb;
    }
    block_sum_max_f64(S, M, shd);
    tot = block_sum_u64(tot, sh);
    mb = block_max_u64(mb, sh);
    if (threadIdx.x == 0) {
      out[4 * a + 0] = tot ? sqrt(S / (double)tot) : 0.0;
      out[4 * a + 1] = M;
      out[4 * a + 2] = (double)tot;
      out[4 * a + 3] = (double)mb;
    }
    __syncthreads();
  }
}

}  // namespace

cudaError_t launch_angle_stats(pic_ctx* c, pic_angle_stats* out) {
  k_ang_chunks<<<2 * kAngleBlocks, kAT, 0, c->stream>>>(c->ang_hist, c->ang_bsum);
  k_ang_errors<<<2 * kAngleBlocks, kAT, 0, c->stream>>>(c->ang_hist, c->ang_bsum, c->ang_part);
  k_ang_final<<<1, kAT, 0, c->stream>>>(c->ang_part, c->ang_bsum, c->ang_out);
  c->launches += 3;
  cudaError_t e = cudaGetLastError();
  double h[8];
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, c->ang_out, sizeof(h), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return e;
  out->eps2_chi = h[0];
  out->epsinf_chi = h[1];
  out->n_coll = (int64_t)h[2];
  out->max_bin[0] = (int64_t)h[3];
  out->eps2_eps = h[4];
  out->epsinf_eps = h[5];
  out->max_bin[1] = (int64_t)h[7];
  return cudaSuccess;
}

}  // namespace pic
