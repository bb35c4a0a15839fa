// Device helpers shared by the precision-form kernels (single domain and
// batched): FP32 time terms, 24-bit uniforms, double-float arithmetic, the
// FP32 inverse-CDF evaluation and the FP32 hard-sphere moment.
#pragma once

#include "pic_internal.cuh"

namespace pic {

// ---------------------------------------------------------------- helpers --
struct TimeTermsF {
  float ct, cos2ct, sin2ct, em_amp;
};

__host__ __device__ inline TimeTermsF to_float(const TimeTerms& t) {
  TimeTermsF f;
  f.ct = (float)t.ct;
  f.cos2ct = (float)t.cos2ct;
  f.sin2ct = (float)t.sin2ct;
  f.em_amp = (float)t.em_amp;
  return f;
}

__device__ __forceinline__ TimeTermsF to_float_dev(const TimeTerms& t) { return to_float(t); }

// top 24 bits of a Philox word as an FP32 uniform in (0, 1): exact
__device__ __forceinline__ float unif24(uint32_t w) { return ((float)(w >> 8) + 0.5f) * 0x1p-24f; }

// double-float: hi + lo with |lo| <= ulp(hi)/2
struct DF {
  float hi, lo;
};
__device__ __forceinline__ DF two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  const float e = (a - (s - bb)) + (b - bb);
  return DF{s, e};
}
__device__ __forceinline__ DF df_add(DF a, DF b) {
  DF s = two_sum(a.hi, b.hi);
  const float lo = s.lo + a.lo + b.lo;
  const float hi = s.hi + lo;
  return DF{hi, lo - (hi - s.hi)};
}
__device__ __forceinline__ DF df_add_f(DF a, float b) {
  DF s = two_sum(a.hi, b);
  const float lo = s.lo + a.lo;
  const float hi = s.hi + lo;
  return DF{hi, lo - (hi - s.hi)};
}
// a += x y exactly up to the double-float rounding (TwoProd by fma)
__device__ __forceinline__ DF df_fma(DF a, float x, float y) {
  const float p = x * y;
  const float e = fmaf(x, y, -p);
  DF s = two_sum(a.hi, p);
  const float lo = s.lo + a.lo + e;
  const float hi = s.hi + lo;
  return DF{hi, lo - (hi - s.hi)};
}
__device__ __forceinline__ DF df_shfl_xor(DF a, int off) {
  return DF{__shfl_xor_sync(0xffffffffu, a.hi, off), __shfl_xor_sync(0xffffffffu, a.lo, off)};
}
__device__ __forceinline__ double df_to_double(DF a) { return (double)a.hi + (double)a.lo; }

// sin(2 pi (x^M - c t)) in FP32: G^{-1} from the Hermite table, one Newton
// correction, sine updated to first order.
__device__ __forceinline__ float xm_sin_f(const ParamsF& P, const TimeTermsF& tt, float xi) {
  const float T = xi - tt.ct - P.fx_a2pi * tt.cos2ct;
  const float fl = floorf(T);
  const float t = (T - fl) * (float)P.ginv_M;
  int k = (int)t;
  k = k >= P.ginv_M ? P.ginv_M - 1 : k;
  const float u = t - (float)k, u2 = u * u, u3 = u2 * u, h = 1.f / (float)P.ginv_M;
  const float2 q0 = __ldg(reinterpret_cast<const float2*>(P.ginv_f) + k);
  const float2 q1 = __ldg(reinterpret_cast<const float2*>(P.ginv_f) + k + 1);
  const float y = fl + (2.f * u3 - 3.f * u2 + 1.f) * q0.x + (u3 - 2.f * u2 + u) * h * q0.y +
                  (3.f * u2 - 2.f * u3) * q1.x + (u3 - u2) * h * q1.y;
  float s, c;
  sincospif(2.f * y, &s, &c);
  const float dy = (y - P.fx_a2pi * c - T) / (1.f + P.fx_amp * s);
  return s - 6.283185307f * c * dy;
}

// y = x^M - c t in FP32 (G^{-1} from the Hermite table, one Newton step):
// the isolated-collision drift moves by y(t_{n+1}) - y(t_n) + c dt.
__device__ __forceinline__ float xm_y_f(const ParamsF& P, const TimeTermsF& tt, float xi) {
  const float T = xi - tt.ct - P.fx_a2pi * tt.cos2ct;
  const float fl = floorf(T);
  const float t = (T - fl) * (float)P.ginv_M;
  int k = (int)t;
  k = k >= P.ginv_M ? P.ginv_M - 1 : k;
  const float u = t - (float)k, u2 = u * u, u3 = u2 * u, h = 1.f / (float)P.ginv_M;
  const float2 q0 = __ldg(reinterpret_cast<const float2*>(P.ginv_f) + k);
  const float2 q1 = __ldg(reinterpret_cast<const float2*>(P.ginv_f) + k + 1);
  const float y = fl + (2.f * u3 - 3.f * u2 + 1.f) * q0.x + (u3 - 2.f * u2 + u) * h * q0.y +
                  (3.f * u2 - 2.f * u3) * q1.x + (u3 - u2) * h * q1.y;
  float s, c;
  sincospif(2.f * y, &s, &c);
  return y - (y - P.fx_a2pi * c - T) / (1.f + P.fx_amp * s);
}

// 32 x 32 bit-matrix transpose across a warp: lane r holds row r on entry
// and column r on return (bit c of row r becomes bit r of column c). Five
// exchange stages swap the off-diagonal blocks of size 16, 8, 4, 2, 1.
__device__ __forceinline__ uint32_t warp_transpose32(uint32_t x, int lane) {
  uint32_t m = 0x0000FFFFu;
#pragma unroll
  for (int j = 16; j != 0; j >>= 1, m ^= m << j) {
    const uint32_t y = __shfl_xor_sync(0xffffffffu, x, j);
    x = (lane & j) ? ((x & ~m) | ((y & ~m) >> j)) : ((x & m) | ((y & m) << j));
  }
  return x;
}

// FP32 form of record_angles (Sec. 4.4)
__device__ __forceinline__ void record_angles_f(unsigned long long* hist, bool aniso, float g, float gx, float gy,
                                                float gz) {
  const float cz = fminf(1.f, fmaxf(-1.f, gz / g));
  const float u = 0.5f * (1.f - cz);
  const float uc = aniso ? u * (13.f + u * (96.f + u * (-160.f + 80.f * u))) * (1.f / 29.f) : u;
  float e = atan2f(gy, gx);
  if (e < 0.f) e += 6.283185307f;
  const int bc = min(PIC_ANGLE_BINS - 1, max(0, (int)(uc * (float)PIC_ANGLE_BINS)));
  const int be = min(PIC_ANGLE_BINS - 1, max(0, (int)(e * (0.1591549431f * (float)PIC_ANGLE_BINS))));
  atomicAdd(hist + bc, 1ull);
  atomicAdd(hist + PIC_ANGLE_BINS + be, 1ull);
}

__device__ __forceinline__ float hs_R_f(const ParamsF& P, float a) {
  const float a2 = a * a;
  if (a < 0.1f) {
    float acc = P.R_series[4];
#pragma unroll
    for (int j = 3; j >= 0; --j) acc = fmaf(acc, a2, P.R_series[j]);
    return acc;
  }
  const float ia = 1.f / a, ia2 = ia * ia;
  return 0.7978845608f * (1.f + ia2) * __expf(-0.5f * a2) + (a + 2.f * ia - ia2 * ia) * erff(a * 0.7071067812f);
}

// cell index -> (i, j, k), by shifts when n is a power of two
__device__ __forceinline__ void cell_ijk(const ParamsF& P, int c, int* ci) {
  if (P.log2n >= 0) {
    const int m = P.n - 1;
    ci[0] = c & m;
    ci[1] = (c >> P.log2n) & m;
    ci[2] = c >> (2 * P.log2n);
  } else {
    ci[0] = c % P.n;
    ci[1] = (c / P.n) % P.n;
    ci[2] = c / P.nn;
  }
}

}  // namespace pic
