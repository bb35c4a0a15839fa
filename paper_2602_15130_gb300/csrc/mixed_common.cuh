// Device helpers shared by the precision-form kernels (single domain and
// batched): FP32 time terms, 24-bit uniforms, double-float arithmetic, the
// FP32 inverse-CDF evaluation and the FP32 hard-sphere moment.
#pragma once

#include "pic_internal.cuh"

namespace pic {

// ---------------------------------------------------------------- helpers --
struct TimeTermsF {
  float ct, cos2ct, sin2ct, em_amp;
  // PIC_DIST_PAPER: the per-axis terms of TimeTerms in FP32
  float fA[3], fs[3], fdA[3], fds[3], fcs[3], fsn[3], vh[3], dvh[3];
};

__host__ __device__ inline TimeTermsF to_float(const TimeTerms& t) {
  TimeTermsF f;
  f.ct = (float)t.ct;
  f.cos2ct = (float)t.cos2ct;
  f.sin2ct = (float)t.sin2ct;
  f.em_amp = (float)t.em_amp;
  for (int d = 0; d < 3; ++d) {
    // the phase enters only through sin/cos(2 pi (x - s)): reduce it mod 1
    f.fA[d] = (float)t.fA[d];
    f.fs[d] = (float)(t.fs[d] - floor(t.fs[d]));
    f.fdA[d] = (float)t.fdA[d];
    f.fds[d] = (float)t.fds[d];
    f.fcs[d] = (float)t.fcs[d];
    f.fsn[d] = (float)t.fsn[d];
    f.vh[d] = (float)t.vh[d];
    f.dvh[d] = (float)t.dvh[d];
  }
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

// sin(2 pi (x^M - c t)) in FP32 by cubic Hermite interpolation of the
// tabulated s(T) = sin(2 pi G^{-1}(T)) (knots behind the G^{-1} knots, exact
// slopes): the argument T = xi - c t - A/(2 pi) cos(2 pi c t) is that of
// xm_solve, and s has period 1 in T.
__device__ __forceinline__ float xm_sin_f(const ParamsF& P, const TimeTermsF& tt, float xi) {
  const float T = xi - tt.ct - P.fx_a2pi * tt.cos2ct;
  const float t = (T - floorf(T)) * (float)P.ginv_M;
  int k = (int)t;
  k = k >= P.ginv_M ? P.ginv_M - 1 : k;
  const float u = t - (float)k, u2 = u * u, u3 = u2 * u, h = 1.f / (float)P.ginv_M;
  const float2* st = reinterpret_cast<const float2*>(P.ginv_f) + (P.ginv_M + 1);
  const float2 q0 = __ldg(st + k), q1 = __ldg(st + k + 1);
  return (2.f * u3 - 3.f * u2 + 1.f) * q0.x + (u3 - 2.f * u2 + u) * h * q0.y + (3.f * u2 - 2.f * u3) * q1.x +
         (u3 - u2) * h * q1.y;
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

// PIC_DIST_PAPER in FP32: sin and cos of 2 pi y, y = x_d^M - s_d, for the
// drift's xdot^M. G(y) = y - A/(2 pi) cos(2 pi y) = T (the FP64 xm_solve_gen
// equation) by Newton from y = T inside the bracket |y - T| <= |A|/(2 pi);
// the iteration stops once a step is below 2^-22 (FP32 resolution of y).
__device__ __forceinline__ void xm_sc_gen_f(const TimeTermsF& tt, int d, float xi, float* sy, float* cy) {
  const float A = tt.fA[d], a2p = A * 0.15915494309f;
  const float T = xi - tt.fs[d] - a2p * tt.fcs[d];
  const float r = fabsf(a2p);
  float lo = T - r, hi = T + r, y = T, s, c;
  for (int it = 0; it < 12; ++it) {
    sincospif(2.f * y, &s, &c);
    const float G = y - a2p * c - T;
    if (G == 0.f) break;
    if (G < 0.f) lo = y; else hi = y;
    float yn = y - G / (1.f + A * s);
    if (!(yn > lo && yn < hi)) yn = 0.5f * (lo + hi);
    const bool done = fabsf(yn - y) <= 0x1p-22f;
    y = yn;
    if (done) break;
  }
  sincospif(2.f * y, sy, cy);
}
__device__ __forceinline__ float xm_dot_gen_f(const TimeTermsF& tt, int d, float sy, float cy) {
  const float A = tt.fA[d];
  return (A * tt.fds[d] * (sy + tt.fsn[d]) - tt.fdA[d] * 0.15915494309f * (tt.fcs[d] - cy)) / (1.f + A * sy);
}

// Odd-power source of Eq. vel_change_3 in FP32 (the closed forms of
// odd_source): Gaussian f_v or the paper's f_v with scales vh.
__device__ __forceinline__ void odd_source_f(const ParamsF& P, const float* vh, float vx, float vy, float vz, int c,
                                             float* out) {
  const float pref = P.src_pref_n * (float)(c - 1);
  const float s0 = P.sigma_n[0], s1 = P.sigma_n[1], s2 = P.sigma_n[2];
  if (P.dist == PIC_DIST_CONFIG) {
    const float mx = P.vmean[0] - vx, my = P.vmean[1] - vy, mz = P.vmean[2] - vz;
    const float m2 = mx * mx + my * my + mz * mz, q2 = P.vsig * P.vsig;
    const float k = pref * (s0 + s1 * (m2 + 5.f * q2) + s2 * (m2 * m2 + 14.f * q2 * m2 + 35.f * q2 * q2));
    out[0] = k * mx; out[1] = k * my; out[2] = k * mz;
    return;
  }
  const float v[3] = {vx, vy, vz};
  const float a2[3] = {vh[0] * vh[0], vh[1] * vh[1], vh[2] * vh[2]};
  const float vh2 = a2[0] + a2[1] + a2[2], vp2 = vx * vx + vy * vy + vz * vz;
  const float cross = a2[0] * vx * vx + a2[1] * vy * vy + a2[2] * vz * vz;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const float others = a2[(i + 1) % 3] * a2[(i + 2) % 3];
    const float f1 = -0.5f * (3.f * vh2 + 6.f * a2[i] + 2.f * vp2);
    const float f2 = -0.25f * (15.f * vh2 * vh2 + 36.f * a2[i] * a2[i] + 24.f * vp2 * a2[i] + 4.f * vp2 * vp2 +
                               24.f * a2[i] * vh2 + 12.f * vp2 * vh2 + 24.f * cross - 12.f * others);
    out[i] = pref * (-s0 + s1 * f1 + s2 * f2) * v[i];
  }
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
  // cubic Hermite interpolation of the tabulated R (interpolation error
  // below 1e-10); beyond the table erf(a/sqrt 2) = 1 and e^{-a^2/2} = 0 to
  // FP32 precision, which leaves a + 2/a - 1/a^3
  if (a >= kRTabAmax) {
    const float ia = 1.f / a;
    return a + 2.f * ia - ia * ia * ia;
  }
  const float2* rt = reinterpret_cast<const float2*>(P.ginv_f + 4 * (P.ginv_M + 1));
  const float t = a * ((float)kRTabM / kRTabAmax);
  int k = (int)t;
  k = k >= kRTabM ? kRTabM - 1 : k;
  const float u = t - (float)k, u2 = u * u, u3 = u2 * u, h = kRTabAmax / (float)kRTabM;
  const float2 q0 = __ldg(rt + k), q1 = __ldg(rt + k + 1);
  return (2.f * u3 - 3.f * u2 + 1.f) * q0.x + (u3 - 2.f * u2 + u) * h * q0.y + (3.f * u2 - 2.f * u3) * q1.x +
         (u3 - u2) * h * q1.y;
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

// ----------------------------------------------------- sort gather + CIC --
struct Gather32Args {
  int n;
  int64_t ncell;
  const int32_t *start, *perm;
  const float* in[9];   // o0..2, v0..2, m0..2
  float* out[9];
  const uint32_t* pid_in;
  uint32_t* pid_out;
  int32_t* cell_out;
  double* corner;       // [8][ncell]
  int big_lo;             // cells above this count go to the block sort
  const uint32_t* spid;   // optional: pids in arrival order (slot s + e holds perm[s + e]'s pid)
  // optional: the source as 48-byte records (o0 o1 o2 v0 | v1 v2 m0 m1 |
  // m2 cell pid -) instead of in[] and pid_in: a random source read as
  // records touches two 32-byte sectors a particle instead of nine
  const float4* rec = nullptr;
  // records binned by cell (rec holds [ncell][bin_cap] records, a cell's
  // arrival e at its slot e): each cell reads its own contiguous span, and
  // perm is not used
  int64_t bin_cap = 0;
};

// particle src of the gather's source: o0..o2, v0..v2, m0..m2 (kRec: record
// src of rb, the records or the cell's bin)
template <bool kRec>
__device__ __forceinline__ void gather_load32(const Gather32Args& a, const float4* rb, int32_t src, float* d) {
  if constexpr (kRec) {
    const float4 r0 = __ldg(rb + 3 * (int64_t)src), r1 = __ldg(rb + 3 * (int64_t)src + 1),
                 r2 = __ldg(rb + 3 * (int64_t)src + 2);
    d[0] = r0.x; d[1] = r0.y; d[2] = r0.z; d[3] = r0.w;
    d[4] = r1.x; d[5] = r1.y; d[6] = r1.z; d[7] = r1.w;
    d[8] = r2.x;
  } else {
#pragma unroll
    for (int q = 0; q < 9; ++q) d[q] = a.in[q][src];
  }
}
template <bool kRec>
__device__ __forceinline__ uint32_t gather_pid32(const Gather32Args& a, const float4* rb, int32_t src) {
  if constexpr (kRec) return __float_as_uint(__ldg(rb + 3 * (int64_t)src + 2).z);
  else return a.pid_in[src];
}

// CIC corner weights of one particle (offsets in cell units) in 64-bit fixed
// point: integer sums are exact in any order, so a cell's corner partials do
// not depend on the order its particles are visited in. The conversion
// rounds with FP32 arithmetic only (64-bit float-to-integer conversions run
// on the slow FP64 pipe): adding 1.5 2^23 rounds w 2^22 to an integer held
// in the low mantissa bits, an FMA recovers the remainder exactly, and the
// remainder is rounded the same way to lo_bits more bits. Resolution 2^-40
// (error <= 2^-41 per weight) below 2^23 particles per cell, 2^-30 above, so
// a corner sum never leaves int64.
struct CicFixed {
  float lo_scale;  // 2^lo_bits
  int lo_bits;     // 18 or 8
  double inv;      // 2^-(22 + lo_bits)
};
__device__ __forceinline__ CicFixed cic_fixed_for(int32_t cnt) {
  return cnt < (1 << 23) ? CicFixed{262144.f, 18, 1.0 / 1099511627776.0} : CicFixed{256.f, 8, 1.0 / 1073741824.0};
}
__device__ __forceinline__ long long to_fixed(float w, const CicFixed& f) {
  constexpr float M = 12582912.f;  // 1.5 2^23
  const float hs = fmaf(w, 4194304.f, M);
  const int hi = __float_as_int(hs) - 0x4B400000;
  const float rem = fmaf(w, 4194304.f, -(hs - M));
  const int lo = __float_as_int(fmaf(rem, f.lo_scale, M)) - 0x4B400000;
  return ((long long)hi << f.lo_bits) + lo;
}

__device__ __forceinline__ void cic_add_fixed(long long* acc, float ox, float oy, float oz, const CicFixed& f) {
  const float wx[2] = {1.f - ox, ox}, wy[2] = {1.f - oy, oy}, wz[2] = {1.f - oz, oz};
#pragma unroll
  for (int c = 0; c < 2; ++c)
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const float wyz = wy[b] * wz[c];
#pragma unroll
      for (int q = 0; q < 2; ++q) acc[q + 2 * b + 4 * c] += to_fixed(wx[q] * wyz, f);
    }
}

__device__ __forceinline__ long long shfl_xor_ll(long long v, int off) {
  return (long long)__shfl_xor_sync(0xffffffffu, (unsigned long long)v, off);
}

// warp sum of 8 fixed-point corner partials: each xor level halves the
// values a lane keeps; lane l then holds corner 4 [l & 16] + 2 [l & 8] + [l & 4]
__device__ __forceinline__ void store_corners_fixed(const long long* acc, int lane, double* corner, int64_t ncell,
                                                    int64_t cell, double inv) {
  const bool u16 = lane & 16, u8 = lane & 8, u4 = lane & 4;
  long long a4[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) a4[i] = (u16 ? acc[4 + i] : acc[i]) + shfl_xor_ll(u16 ? acc[i] : acc[4 + i], 16);
  long long a2[2];
#pragma unroll
  for (int i = 0; i < 2; ++i) a2[i] = (u8 ? a4[2 + i] : a4[i]) + shfl_xor_ll(u8 ? a4[i] : a4[2 + i], 8);
  long long a1 = (u4 ? a2[1] : a2[0]) + shfl_xor_ll(u4 ? a2[0] : a2[1], 4);
  a1 += shfl_xor_ll(a1, 2);
  a1 += shfl_xor_ll(a1, 1);
  if ((lane & 3) == 0) {
    const int c = (u16 ? 4 : 0) + (u8 ? 2 : 0) + (u4 ? 1 : 0);
    corner[(int64_t)c * ncell + cell] = (double)a1 * inv;
  }
}

// C chunks of 32 arrival slots of one cell (C * 32 >= cnt) held in
// registers: each particle's in-cell rank counted against every pid of the
// cell, then the particle copied to slot s + rank and its CIC weights
// added. Up to two chunks load the particle data with the pids (one memory
// round trip); wider cells load it after the count, to bound the registers.
template <int C, bool kRec>
__device__ __forceinline__ void gather_chunks32(const Gather32Args& a, const float4* rb, bool binned, int64_t cell,
                                                int32_t s, int32_t cnt, int lane, const CicFixed& fx,
                                                long long* acc) {
  constexpr bool kPre = C <= 2;
  int32_t src[C];
  uint32_t p[C];
  float d[kPre ? C : 1][9];
#pragma unroll
  for (int k = 0; k < C; ++k) {
    const int32_t e = 32 * k + lane;
    src[k] = 0;
    p[k] = 0xFFFFFFFFu;
    if (e < cnt) {
      src[k] = binned ? e : a.perm[s + e];
      if (a.spid) p[k] = a.spid[s + e];
    }
  }
#pragma unroll
  for (int k = 0; k < C; ++k)
    if (32 * k + lane < cnt) {
      if (!a.spid) p[k] = gather_pid32<kRec>(a, rb, src[k]);
      if constexpr (kPre) gather_load32<kRec>(a, rb, src[k], d[k]);
    }
  int r[C];
#pragma unroll
  for (int k = 0; k < C; ++k) r[k] = 0;
  if (C == 1) {
    for (int l = 0; l < cnt; ++l) r[0] += __shfl_sync(0xffffffffu, p[0], l) < p[0] ? 1 : 0;
  } else {
    // unused slots hold pid 0xFFFFFFFF, above every particle's
    for (int l = 0; l < 32; ++l) {
      uint32_t x[C];
#pragma unroll
      for (int j = 0; j < C; ++j) x[j] = __shfl_sync(0xffffffffu, p[j], l);
#pragma unroll
      for (int k = 0; k < C; ++k)
#pragma unroll
        for (int j = 0; j < C; ++j) r[k] += x[j] < p[k] ? 1 : 0;
    }
  }
#pragma unroll
  for (int k = 0; k < C; ++k)
    if (32 * k + lane < cnt) {
      const int32_t dst = s + r[k];
      float* dk = d[kPre ? k : 0];
      if constexpr (!kPre) gather_load32<kRec>(a, rb, src[k], dk);
#pragma unroll
      for (int q = 0; q < 9; ++q) a.out[q][dst] = dk[q];
      a.pid_out[dst] = p[k];
      a.cell_out[dst] = (int32_t)cell;
      cic_add_fixed(acc, dk[0], dk[1], dk[2], fx);
    }
}

// One cell of the sort gather (a warp): the cell's particles in ascending
// pid order (their in-cell rank by pid), copied to the destination arrays,
// and the cell's eight CIC corner partials. Cells of big_lo < count <=
// kMaxBlockSort are left to the block sort. Cells of up to 32 kRegChunks
// particles take the register path, larger ones the chunked pairwise count.
template <int kRegChunks = 4, bool kRec = false>
__device__ __forceinline__ void gather_cell32(const Gather32Args& a, int64_t cell, int lane) {
  const int32_t s = a.start[cell];
  const int32_t cnt = a.start[cell + 1] - s;
  if (cnt > a.big_lo && cnt <= kMaxBlockSort) return;  // k_sort_big32
  const CicFixed fx = cic_fixed_for(cnt);
  long long acc[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) acc[q] = 0;
  // the source of arrival e: records at perm[s + e], or slot e of the cell's bin
  const float4* rb = a.rec;
  bool binned = false;
  if constexpr (kRec) {
    if (a.bin_cap > 0) {
      binned = true;
      rb += 3 * cell * a.bin_cap;
    }
  }
  const int32_t nch = (cnt + 31) >> 5;  // warp-uniform
  if (nch <= 1) {
    gather_chunks32<1, kRec>(a, rb, binned, cell, s, cnt, lane, fx, acc);
  } else if (nch == 2) {
    gather_chunks32<2, kRec>(a, rb, binned, cell, s, cnt, lane, fx, acc);
  } else if (kRegChunks >= 3 && nch == 3) {
    if constexpr (kRegChunks >= 3) gather_chunks32<3, kRec>(a, rb, binned, cell, s, cnt, lane, fx, acc);
  } else if (kRegChunks >= 4 && nch == 4) {
    if constexpr (kRegChunks >= 4) gather_chunks32<4, kRec>(a, rb, binned, cell, s, cnt, lane, fx, acc);
  } else {
    for (int32_t e0 = 0; e0 < cnt; e0 += 32) {
      const int32_t e = e0 + lane;
      int32_t src = 0;
      uint32_t mp = 0xFFFFFFFFu;
      if (e < cnt) {
        src = binned ? e : a.perm[s + e];
        mp = gather_pid32<kRec>(a, rb, src);  // spid is pid_out: rewritten by earlier chunks
      }
      int32_t r = 0;
      for (int32_t f0 = 0; f0 < cnt; f0 += 32) {
        uint32_t other = mp;
        if (f0 != e0) {
          const int32_t f = f0 + lane;
          other = f < cnt ? gather_pid32<kRec>(a, rb, binned ? f : a.perm[s + f]) : 0xFFFFFFFFu;
        }
        const int lim = min(32, cnt - f0);
        for (int l = 0; l < lim; ++l) r += __shfl_sync(0xffffffffu, other, l) < mp ? 1 : 0;
      }
      if (e < cnt) {
        const int32_t dst = s + r;
        float d[9];
        gather_load32<kRec>(a, rb, src, d);
#pragma unroll
        for (int q = 0; q < 9; ++q) a.out[q][dst] = d[q];
        a.pid_out[dst] = mp;
        a.cell_out[dst] = (int32_t)cell;
        cic_add_fixed(acc, d[0], d[1], d[2], fx);
      }
    }
  }
  store_corners_fixed(acc, lane, a.corner, a.ncell, cell, fx.inv);
}

}  // namespace pic
