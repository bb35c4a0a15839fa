// Internal definitions of the GB300 PIC + DSMC library: launch parameters,
// device helpers and the context. Not part of the C ABI.
#pragma once

#include <cuda_runtime.h>
#include <climits>
#include <functional>
#include <stdint.h>

#include "../../include/pic.h"

namespace pic {

constexpr double kPi = 3.14159265358979323846;
constexpr double kTwoPi = 2.0 * 3.14159265358979323846;
constexpr int kSeriesTerms = 10;
// FP32 table of the hard-sphere moment R(a) on [0, kRTabAmax]: kRTabM
// intervals of cubic Hermite knots (R, dR/da), stored after the two G^{-1}
// tables of the precision form
constexpr int kRTabM = 512;
// steps of the per-step history (pic_get_step_history)
constexpr int kHistSteps = 4096;
constexpr float kRTabAmax = 8.f;

// ---------------------------------------------------------------------------
// Everything a kernel needs to know about the problem, passed by value.
// ---------------------------------------------------------------------------
struct Params {
  int n;              // cells per axis
  int K;              // outcomes per collision call
  int64_t ncell;      // n^3
  int64_t np;         // N_p
  double dt, qm_eff, q_eff, eps0, nphys;
  double sigma0, gmax;
  double fx_amp, fx_speed, fx_amp_over_2pi;
  double vmean[3], vsig, inv_vsig;
  double phi_amp, phi_T, phi_shift[3];
  uint32_t key0, key1;   // Philox key = seed
  // derived (host-computed, see derive_params)
  double h, dV, w;
  double sg_max;         // (sigma g)_max = sigma0 g_max
  double pmax;           // P_coll,max = (sigma g)_max w dt / dV
  double rho_scale;      // q w / h^3
  double src_pref;       // w dt sigma0 / (2 dV): multiplies (c - 1) s R(a) m
  double R_series[kSeriesTerms];  // sqrt(2/pi) c_j, small-a series of R(a)
  // G^{-1} on T in [0,1], G(y) = y - A/(2 pi) cos(2 pi y): M+1 knots of
  // (y_k, dy/dT at k) for cubic Hermite interpolation (device arrays)
  const double* ginv;
  const float* ginv_f;
  int ginv_M;
  int verify;                      // PIC_VERIFY_* bits
  unsigned long long* ang_hist;    // [2][PIC_ANGLE_BINS] when recording angles
  double E_app[3];                 // uniform applied field in the push (adjoint parameter; 0 otherwise)
  int dist;                        // PIC_DIST_*
  int n_sigma;                     // 0: hard sphere; 1..3: odd-power sigma(g)
  double sigma_n[3];               // sigma_k (zero beyond n_sigma)
  double src_pref_n;               // w dt / (2 dV): multiplies (c - 1) sum_k sigma_k f_k
  double vbar, t_ref;              // PIC_DIST_PAPER
};


// FP32 copy of the parameters the precision-form kernels use, converted
// once on the host (FP64 arithmetic in a kernel would run on the slow
// FP64 pipe).
struct ParamsF {
  int n, nn, K;
  int log2n;                  // log2(n) when n is a power of two, else -1
  int64_t np, ncell;
  uint32_t key0, key1;
  uint32_t rk[2][10];          // Philox round keys: key + r (Weyl constants), r = 0..9
  float h, dt_qm, dtn;        // dt q/m, dt n (drift in cell units)
  float fx_amp, fx_a2pi, fx_Ac;
  float vmean[3], vsig, inv_vsig;
  float src_pref, pmax, gmax, gmax2;
  float phi_shift[3];
  const float* ginv_f;
  int ginv_M;
  int verify;                      // PIC_VERIFY_* bits
  float nf, cdt;                   // n, and c dt of the manufactured drift
  unsigned long long* ang_hist;    // [2][PIC_ANGLE_BINS] when recording angles
  int dist, n_sigma;               // PIC_DIST_*, odd-power cross section terms (0: hard sphere)
  float sigma_n[3], sgmax, src_pref_n, dt;
};

// Decision log of the collision kernels (pic_set_decision_log): records of
// 8 int32 (c0, cell, outcome, slot, p, q, result, kind). mode 0 is off.
struct DLog {
  int32_t* buf;
  unsigned long long* n;
  long long cap;
  int mode;
};

__device__ __forceinline__ void dlog_put(const DLog& L, uint32_t c0, uint32_t cell, uint32_t o, int slot, int p,
                                         int q, int result, int kind) {
  const unsigned long long i = atomicAdd(L.n, 1ull);
  if ((long long)i < L.cap) {
    int4* e = reinterpret_cast<int4*>(L.buf + 8 * (size_t)i);
    e[0] = make_int4((int)c0, (int)cell, (int)o, slot);
    e[1] = make_int4(p, q, result, kind);
  }
}

// Per-replicate data of a batch (device copy).
struct BatchRep {
  ParamsF f;
  int64_t poff, coff;  // first particle, first cell/node
  int Kc, G, nchunks;
};
constexpr int kBatchTile = 256;
// a batched replicate's Poisson solve runs on a team of blocks: one per
// kTeamNodes nodes, at most kTeamMax
constexpr int kTeamNodes = 16384;
constexpr int kTeamMax = 32;
__host__ __device__ inline int cg_team_size(int m) {
  const int T = m / kTeamNodes;
  return T < 1 ? 1 : (T > kTeamMax ? kTeamMax : T);
}


// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11). Round: two 32x32 -> 64 products with
// the published multipliers, key bumped by the published Weyl constants.
// ---------------------------------------------------------------------------
struct U4 {
  uint32_t x, y, z, w;
};

// kWide: each product as one 32 x 32 -> 64 multiply (the same bits; see
// philox_rk for when each form is used).
template <bool kWide = false>
__device__ __forceinline__ U4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                     uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    uint32_t hi0, lo0, hi1, lo1;
    if (kWide) {
      const unsigned long long p0 = (unsigned long long)c0 * 0xD2511F53ull;
      const unsigned long long p1 = (unsigned long long)c2 * 0xCD9E8D57ull;
      hi0 = (uint32_t)(p0 >> 32); lo0 = (uint32_t)p0;
      hi1 = (uint32_t)(p1 >> 32); lo1 = (uint32_t)p1;
    } else {
      hi0 = __umulhi(0xD2511F53u, c0); lo0 = 0xD2511F53u * c0;
      hi1 = __umulhi(0xCD9E8D57u, c2); lo1 = 0xCD9E8D57u * c2;
    }
    const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return U4{c0, c1, c2, c3};
}

// The same generator with its ten round keys given (key0 + r 0x9E3779B9,
// key1 + r 0xBB67AE85): where they sit in the kernel parameters, each round
// takes them as constant operands instead of bumping the key in registers.
// kWide forms each product as one 32 x 32 -> 64 multiply instead of separate
// high and low halves: the same bits; measured faster in the collision
// kernel (1.90 -> 1.87 ms per launch at 128^3) and slower in the kick (1.52
// -> 1.56 ms), so each kernel takes the form that suits it.
template <bool kWide = false>
__device__ __forceinline__ U4 philox_rk(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                        const uint32_t (&rk)[2][10]) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    uint32_t hi0, lo0, hi1, lo1;
    if (kWide) {
      const unsigned long long p0 = (unsigned long long)c0 * 0xD2511F53ull;
      const unsigned long long p1 = (unsigned long long)c2 * 0xCD9E8D57ull;
      hi0 = (uint32_t)(p0 >> 32); lo0 = (uint32_t)p0;
      hi1 = (uint32_t)(p1 >> 32); lo1 = (uint32_t)p1;
    } else {
      hi0 = __umulhi(0xD2511F53u, c0); lo0 = 0xD2511F53u * c0;
      hi1 = __umulhi(0xCD9E8D57u, c2); lo1 = 0xCD9E8D57u * c2;
    }
    const uint32_t n0 = hi1 ^ c1 ^ rk[0][r], n2 = hi0 ^ c3 ^ rk[1][r];
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
  }
  return U4{c0, c1, c2, c3};
}

// (2m + 1) 2^-53 with m the top 52 bits of (hi, lo): exact, inside (0, 1).
__device__ __forceinline__ double unif52(uint32_t hi, uint32_t lo) {
  const unsigned long long m = ((unsigned long long)hi << 20) | (unsigned long long)(lo >> 12);
  return __ull2double_rn(2ull * m + 1ull) * 0x1p-53;
}
// (2 w + 1) 2^-33: exact, inside (0, 1).
__device__ __forceinline__ double unif32(uint32_t w) {
  return __ull2double_rn(2ull * (unsigned long long)w + 1ull) * 0x1p-33;
}
// floor(U c) with U = w 2^-32: a 0-based uniform index below c.
__device__ __forceinline__ uint32_t draw_index(uint32_t w, uint32_t c) { return __umulhi(w, c); }

// Sampling stream of one particle: counter (pid_lo, pid_hi, 0, 0xFFFFFF00|j).
__device__ __forceinline__ U4 sample_block(const Params& P, uint64_t pid, uint32_t j) {
  return philox((uint32_t)pid, (uint32_t)(pid >> 32), 0u, 0xFFFFFF00u | j, P.key0, P.key1);
}

// ---------------------------------------------------------------------------
// Manufactured solution.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int cell_coord(double x, int n) {
  int i = (int)floor(x * (double)n);
  return i < 0 ? 0 : (i > n - 1 ? n - 1 : i);
}

// Time-only terms of the manufactured solution at one time t (host-computed
// once per launch): c t, cos(2 pi c t), sin(2 pi c t) and the amplitude
// 2 pi phibar e^{t/(2T)} of grad phi^M.
struct TimeTerms {
  double t, ct, cos2ct, sin2ct, em_amp;
  // PIC_DIST_PAPER: per axis A_d, s_d of f_{x_d} = 1 + A_d sin(2 pi (x - s_d)),
  // their time derivatives, cos and sin of 2 pi s_d, and vh_d, vh_d'
  double fA[3], fs[3], fdA[3], fds[3], fcs[3], fsn[3];
  double vh[3], dvh[3];
};

// G^{-1}(T) by cubic Hermite interpolation of the knot table (T any real:
// G^{-1}(T + 1) = G^{-1}(T) + 1).
__device__ __forceinline__ double ginv_eval(const Params& P, double T) {
  const double fl = floor(T);
  const double t = (T - fl) * (double)P.ginv_M;
  int k = (int)t;
  k = k >= P.ginv_M ? P.ginv_M - 1 : k;
  const double u = t - (double)k, u2 = u * u, u3 = u2 * u, h = 1.0 / (double)P.ginv_M;
  const double* q = P.ginv + 2 * k;
  return fl + (2.0 * u3 - 3.0 * u2 + 1.0) * q[0] + (u3 - 2.0 * u2 + u) * h * q[1] + (3.0 * u2 - 2.0 * u3) * q[2] +
         (u3 - u2) * h * q[3];
}

// x^M(t) with F_x(x^M, t) = xi for f_x = 1 + A sin(2 pi (x - c t)). With
// y = x - c t the equation is G(y) = y - A/(2 pi) cos(2 pi y) = T, T = xi -
// c t - A/(2 pi) cos(2 pi c t): time only shifts T, so one table of G^{-1}
// serves every t. Newton polishes the interpolated start (G' = 1 + A sin
// >= 1 - |A|, |G''/(2 G')| < 1.35 for |A| = 0.3); once a correction is at
// most 2^-27 the next one would be below half an ulp of y = O(1), so the
// loop stops and updates sin(2 pi y) to first order. The Hermite start is
// within ~1e-11, so one iteration is the rule.
// Returns x^M and sin(2 pi (x^M - c t)) (for xdot^M).
__device__ __forceinline__ double xm_solve(const Params& P, const TimeTerms& tt, double xi, double* s_out) {
  const double T = xi - tt.ct - P.fx_amp_over_2pi * tt.cos2ct;
  double y = ginv_eval(P, T);
  for (int it = 0; it < 12; ++it) {
    double s, c;
    sincospi(2.0 * y, &s, &c);
    const double dy = (y - P.fx_amp_over_2pi * c - T) / (1.0 + P.fx_amp * s);
    y -= dy;
    if (fabs(dy) <= 0x1p-27) {
      *s_out = s - kTwoPi * c * dy;
      return y + tt.ct;
    }
  }
  *s_out = sinpi(2.0 * y);
  return y + tt.ct;
}

// xdot^M = A c [sin(2 pi (x^M - c t)) + sin(2 pi c t)] / (1 + A sin(2 pi (x^M - c t)))
__device__ __forceinline__ double xm_dot(const Params& P, const TimeTerms& tt, double s) {
  return P.fx_amp * P.fx_speed * (s + tt.sin2ct) / (1.0 + P.fx_amp * s);
}

// PIC_DIST_PAPER: x_d^M(t) solves F_{x_d}(x, t) = xi for f_{x_d} = 1 + A
// sin(2 pi (x - s)), A and s varying in time. With y = x - s the equation
// is G(y) = y - A/(2 pi) cos(2 pi y) = T, T = xi - s - A/(2 pi) cos(2 pi s)
// (G' = 1 + A sin >= 1 - |A| > 0, root within |A|/(2 pi) of T): Newton from
// y = T, kept inside a bracket that every step narrows (bisection where a
// step leaves it). Returns x^M = y + s, with sin and cos of 2 pi y.
__device__ __forceinline__ double xm_solve_gen(const TimeTerms& tt, int d, double xi, double* sy, double* cy) {
  const double A = tt.fA[d], a2p = A / kTwoPi;
  const double T = xi - tt.fs[d] - a2p * tt.fcs[d];
  const double r = fabs(a2p);
  double lo = T - r, hi = T + r, y = T;
  for (int it = 0; it < 64; ++it) {
    double s, c;
    sincospi(2.0 * y, &s, &c);
    const double G = y - a2p * c - T;
    if (G == 0.0) break;
    if (G < 0.0) lo = y; else hi = y;
    double yn = y - G / (1.0 + A * s);
    if (!(yn > lo && yn < hi)) yn = 0.5 * (lo + hi);
    const bool done = fabs(yn - y) <= 0x1p-52;
    y = yn;
    if (done) break;
  }
  sincospi(2.0 * y, sy, cy);
  return y + tt.fs[d];
}

// xdot^M = -(1/f) int_0^{x^M} d/dt f = [A s' (sin 2 pi y + sin 2 pi s) -
// A'/(2 pi) (cos 2 pi s - cos 2 pi y)] / (1 + A sin 2 pi y), y = x^M - s.
__device__ __forceinline__ double xm_dot_gen(const TimeTerms& tt, int d, double sy, double cy) {
  const double A = tt.fA[d];
  return (A * tt.fds[d] * (sy + tt.fsn[d]) - tt.fdA[d] / kTwoPi * (tt.fcs[d] - cy)) / (1.0 + A * sy);
}

// PIC_DIST_PAPER: tau(xi) with G(tau) = (1 + erf tau)/2 - tau e^{-tau^2}/sqrt pi
// = xi, the quantile of the standardised f_v (v^M = vh(t) tau). G is odd
// about 1/2, so |tau| solves P(|tau|) = |2 xi - 1| with P(t) = erf t -
// (2/sqrt pi) t e^{-t^2}; below P = 1/2 by Newton on P^{1/3} (P ~ 4 t^3 /
// (3 sqrt pi) near 0, summed as its alternating series there), above it by
// Newton on log Q, Q = 1 - P = erfc t + (2/sqrt pi) t e^{-t^2} = 2 min(xi,
// 1 - xi) (exact), each inside a bracket with bisection as the fallback.
__device__ __forceinline__ double tau_P(double t) {
  const double two_sqpi = 1.1283791670955126;  // 2/sqrt(pi)
  if (t < 0.5) {
    // (2/sqrt pi) sum_{k>=1} (-1)^{k+1} 2k/(2k+1) t^{2k+1}/k!
    const double t2 = t * t;
    double term = t, acc = 0.0;
    for (int k = 1; k <= 24; ++k) {
      term *= t2 / (double)k;   // t^{2k+1}/k!
      const double c = (2.0 * k) / (2.0 * k + 1.0) * term;
      acc += (k & 1) ? c : -c;
    }
    return two_sqpi * acc;
  }
  return erf(t) - two_sqpi * t * exp(-t * t);
}
__device__ __forceinline__ double tau_inv(double xi) {
  const double two_sqpi = 1.1283791670955126, four_sqpi = 2.2567583341910252;
  const bool neg = xi < 0.5;
  const double q = neg ? 2.0 * xi : 2.0 * (1.0 - xi);   // Q(|tau|), exact
  double t;
  if (q >= 0.5) {
    const double r = 1.0 - q;                           // P(|tau|), exact
    if (r <= 0.0) return 0.0;
    const double r3 = cbrt(r);
    double lo = 0.0, hi = 1.2;
    t = cbrt(0.75 * 1.7724538509055160 * r);            // P ~ 4 t^3/(3 sqrt pi)
    if (!(t > lo && t < hi)) t = 0.5 * (lo + hi);
    for (int it = 0; it < 80; ++it) {
      const double P = tau_P(t);
      const double h = cbrt(P) - r3;
      if (h == 0.0) break;
      if (h < 0.0) lo = t; else hi = t;
      const double dP = four_sqpi * t * t * exp(-t * t);
      double tn = t - h * 3.0 * cbrt(P) * cbrt(P) / dP;
      if (!(tn > lo && tn < hi)) tn = 0.5 * (lo + hi);
      const bool done = fabs(tn - t) <= 0x1p-53 * t;
      t = tn;
      if (done) break;
    }
  } else {
    const double lq = log(q);
    double lo = 0.8, hi = 7.0;
    t = sqrt(-log(q * 0.88622692545275801));            // Q ~ (2/sqrt pi) t e^{-t^2}
    if (!(t > lo && t < hi)) t = 0.5 * (lo + hi);
    for (int it = 0; it < 80; ++it) {
      const double e = exp(-t * t);
      const double Q = erfc(t) + two_sqpi * t * e;
      const double h = log(Q) - lq;                     // decreasing in t
      if (h == 0.0) break;
      if (h > 0.0) lo = t; else hi = t;
      const double dlogQ = -four_sqpi * t * t * e / Q;
      double tn = t - h / dlogQ;
      if (!(tn > lo && tn < hi)) tn = 0.5 * (lo + hi);
      const bool done = fabs(tn - t) <= 0x1p-53 * t;
      t = tn;
      if (done) break;
    }
  }
  return neg ? -t : t;
}

// <Delta v^M> of Eq. vel_change_3 for sigma(g) = sum_k sigma_k g^{2k-1}
// (k < 3): src_pref_n (c - 1) sum_k sigma_k f_k with f_k = E[g^{2k} (v_q -
// v_p)] (Eq. fn) in closed form. Gaussian f_v (mean mu, width s), M = mu - v:
// f_0 = M, f_1 = (|M|^2 + 5 s^2) M, f_2 = (|M|^4 + 14 s^2 |M|^2 + 35 s^4) M.
// The paper's f_v (scales vh at the call's time): the f_0, f_1, f_2 of
// Sec. 3.3.
__device__ __forceinline__ void odd_source(const Params& P, const double* vh, double vx, double vy, double vz,
                                           int c, double* out) {
  const double pref = P.src_pref_n * (double)(c - 1);
  const double s0 = P.sigma_n[0], s1 = P.sigma_n[1], s2 = P.sigma_n[2];
  if (P.dist == PIC_DIST_CONFIG) {
    const double mx = P.vmean[0] - vx, my = P.vmean[1] - vy, mz = P.vmean[2] - vz;
    const double m2 = mx * mx + my * my + mz * mz, q2 = P.vsig * P.vsig;
    const double k = pref * (s0 + s1 * (m2 + 5.0 * q2) + s2 * (m2 * m2 + 14.0 * q2 * m2 + 35.0 * q2 * q2));
    out[0] = k * mx; out[1] = k * my; out[2] = k * mz;
    return;
  }
  const double v[3] = {vx, vy, vz};
  const double a2[3] = {vh[0] * vh[0], vh[1] * vh[1], vh[2] * vh[2]};
  const double vh2 = a2[0] + a2[1] + a2[2], vp2 = vx * vx + vy * vy + vz * vz;
  const double cross = a2[0] * vx * vx + a2[1] * vy * vy + a2[2] * vz * vz;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const double others = a2[(i + 1) % 3] * a2[(i + 2) % 3];
    const double f1 = -0.5 * (3.0 * vh2 + 6.0 * a2[i] + 2.0 * vp2);
    const double f2 = -0.25 * (15.0 * vh2 * vh2 + 36.0 * a2[i] * a2[i] + 24.0 * vp2 * a2[i] + 4.0 * vp2 * vp2 +
                               24.0 * a2[i] * vh2 + 12.0 * vp2 * vh2 + 24.0 * cross - 12.0 * others);
    out[i] = pref * (-s0 + s1 * f1 + s2 * f2) * v[i];
  }
}

// sigma(g) g = sigma_0 + sigma_1 g^2 + sigma_2 g^4 (zero coefficients beyond
// n_sigma), summed in ascending order without contraction.
__device__ __forceinline__ double sigma_g(const Params& P, double g2) {
  return __dadd_rn(__dadd_rn(P.sigma_n[0], __dmul_rn(P.sigma_n[1], g2)), __dmul_rn(P.sigma_n[2], __dmul_rn(g2, g2)));
}

// E^M = -grad phi^M at x (time terms in tt).
__device__ __forceinline__ void e_manufactured(const Params& P, const TimeTerms& tt, double x, double y, double z,
                                               double* ex, double* ey, double* ez) {
  double s0, c0, s1, c1, s2, c2;
  sincospi(2.0 * (x - P.phi_shift[0]), &s0, &c0);
  sincospi(2.0 * (y - P.phi_shift[1]), &s1, &c1);
  sincospi(2.0 * (z - P.phi_shift[2]), &s2, &c2);
  *ex = -tt.em_amp * c0 * s1 * s2;
  *ey = -tt.em_amp * s0 * c1 * s2;
  *ez = -tt.em_amp * s0 * s1 * c2;
}

// R(a): E_{X ~ N(m, s^2 I)} |X| X = s R(|m|/s) m (hard spheres, Gaussian f_v).
__device__ __forceinline__ double hs_R(const Params& P, double a) {
  const double a2 = a * a;
  if (a < 0.1) {
    double acc = P.R_series[kSeriesTerms - 1];
#pragma unroll
    for (int j = kSeriesTerms - 2; j >= 0; --j) acc = fma(acc, a2, P.R_series[j]);
    return acc;
  }
  const double ia = 1.0 / a, ia2 = ia * ia;
  const double sq2pi = 0.79788456080286535588;  // sqrt(2/pi)
  return sq2pi * (1.0 + ia2) * exp(-0.5 * a2) + (a + 2.0 * ia - ia2 * ia) * erf(a * 0.70710678118654752440);
}

// <Delta v^M> of Eq. vel_change_1c for a particle of velocity v in a cell of c.
__device__ __forceinline__ void hs_source(const Params& P, double vx, double vy, double vz, int c,
                                          double* sx, double* sy, double* sz) {
  const double mx = P.vmean[0] - vx, my = P.vmean[1] - vy, mz = P.vmean[2] - vz;
  const double a = sqrt(mx * mx + my * my + mz * mz) * P.inv_vsig;
  const double f = P.src_pref * (double)(c - 1) * P.vsig * hs_R(P, a);
  *sx = f * mx;
  *sy = f * my;
  *sz = f * mz;
}

// Cells above kBigCell particles are ranked by a block-level bitonic sort
// in shared memory (up to kMaxBlockSort particles); smaller and larger ones
// by the warp's pairwise count.
// blocks of the angle-histogram reduction (PIC_ANGLE_BINS / kAngleBlocks
// bins each)
constexpr int kAngleBlocks = 1024;

constexpr int kBigCell = 256;
constexpr int kMaxBlockSort = 16384;

// The block sort is launched only when the mean occupancy is high enough for
// big cells to be common; otherwise the warp pass takes every cell.
inline int big_cell_threshold(int64_t ncell, int64_t np) {
  return (ncell > 0 && np >= 128 * ncell) ? kBigCell : INT_MAX;
}

// Ascending bitonic sort of n (a power of two) (key, val) pairs in shared
// memory by the whole block; returns after a __syncthreads.
__device__ __forceinline__ void block_bitonic_sort(uint32_t* key, int32_t* val, int n) {
  for (int k = 2; k <= n; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int ixj = i ^ j;
        if (ixj > i) {
          const bool up = (i & k) == 0;
          const uint32_t a = key[i], b = key[ixj];
          if ((a > b) == up) {
            key[i] = b;
            key[ixj] = a;
            const int32_t t = val[i];
            val[i] = val[ixj];
            val[ixj] = t;
          }
        }
      }
      __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Manufactured anisotropic scattering (Sec. 5.1): with u = sin^2(chi/2) the
// CDF of chi is F(u) = (13 u + 96 u^2 - 160 u^3 + 80 u^4)/29; u(xi) is the
// root of the quartic F(u) = xi in [0, 1] by its closed form (a resolvent
// cube root, then two square roots).
// ---------------------------------------------------------------------------
__device__ __forceinline__ double aniso_u(double xi) {
  const double r = sqrt(298924665.0 + 55680.0 * xi * (376377.0 + 2320.0 * xi * (-429.0 + 290.0 * xi)));
  const double a = cbrt(81909.0 - 83520.0 * xi + r) / 83.20335292207616;  // 40 3^{2/3}
  const double b = 0.2 + a + (161.0 - 290.0 * xi) / (600.0 * a);
  const double sb = sqrt(b);
  const double u = 0.5 * (1.0 - sb + sqrt(0.6 - b + 29.0 / (40.0 * sb)));
  return u < 0.0 ? 0.0 : (u > 1.0 ? 1.0 : u);
}
__device__ __forceinline__ float aniso_u_f(float xi) {
  const float r = sqrtf(298924665.f + 55680.f * xi * (376377.f + 2320.f * xi * (-429.f + 290.f * xi)));
  const float a = cbrtf(81909.f - 83520.f * xi + r) / 83.2033529f;
  const float b = 0.2f + a + (161.f - 290.f * xi) / (600.f * a);
  const float sb = sqrtf(b);
  const float u = 0.5f * (1.f - sb + sqrtf(fmaxf(0.f, 0.6f - b + 29.f / (40.f * sb))));
  return fminf(fmaxf(u, 0.f), 1.f);
}
__host__ __device__ __forceinline__ double aniso_F(double u) {
  return u * (13.0 + u * (96.0 + u * (-160.0 + 80.0 * u))) / 29.0;
}

// One recorded collision (Sec. 4.4): u_chi = F^M(chi) with cos chi =
// g'_z / g (g the pre-collision speed), u_eps = eps / (2 pi) with eps =
// atan2(g'_y, g'_x) in [0, 2 pi); each goes into its bin of PIC_ANGLE_BINS.
__device__ __forceinline__ int angle_bin(double u) {
  int b = (int)(u * (double)PIC_ANGLE_BINS);
  return b < 0 ? 0 : (b >= PIC_ANGLE_BINS ? PIC_ANGLE_BINS - 1 : b);
}
__device__ __forceinline__ void record_angles(unsigned long long* hist, bool aniso, double g, double gx, double gy,
                                              double gz) {
  double cz = gz / g;
  cz = cz > 1.0 ? 1.0 : (cz < -1.0 ? -1.0 : cz);
  const double u = 0.5 * (1.0 - cz);
  const double uc = aniso ? aniso_F(u) : u;
  double e = atan2(gy, gx);
  if (e < 0.0) e += kTwoPi;
  atomicAdd(hist + angle_bin(uc), 1ull);
  atomicAdd(hist + PIC_ANGLE_BINS + angle_bin(e / kTwoPi), 1ull);
}

// Slot of one particle in its cell's count: lanes of a warp with the same
// key share one atomic (particles arrive sorted by cell, so a warp covers
// one or two cells); the ranks inside a cell are a permutation of
// 0..count-1 in any order (the in-cell pid sort fixes the final order).
__device__ __forceinline__ int32_t cell_slot(int32_t* count, int32_t key) {
  const unsigned act = __activemask();
  const unsigned peers = __match_any_sync(act, key);
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(peers) - 1;
  int32_t base = 0;
  if (lane == leader) base = atomicAdd(count + key, __popc(peers));
  base = __shfl_sync(act, base, leader);
  return base + __popc(peers & ((1u << lane) - 1u));
}

__device__ __forceinline__ double wrap_unit(double x) {
  double y = x - floor(x);
  return y >= 1.0 ? 0.0 : y;
}

}  // namespace pic

// ---------------------------------------------------------------------------
// Context (host side). Device arrays are structure-of-arrays, sorted by
// (cell, pid); two copies of every per-particle array for the sort.
// ---------------------------------------------------------------------------
namespace pic {
struct AdjointBuffers;
}

struct pic_ctx {
  pic_config cfg;
  pic::Params P;
  cudaStream_t stream;
  int device, num_sms;
  pic_allocator alloc;
  bool have_alloc;

  bool mixed;       // precision form (PIC_MIXED)

  // particles, buffer [b][component]
  double* x[2][3];
  double* v[2][3];
  double* vm[2][3];  // v^M (constant for the Gaussian f_v)
  uint32_t* pid[2];
  int cur;

  int32_t* key;     // cell of each particle (current order)
  int32_t* rank;    // arrival rank inside its cell (atomic, unordered)
  int32_t* perm;    // sorted slot -> source index (before the in-cell sort)
  int32_t* count;   // [ncell]
  int32_t* start;   // [ncell + 1]
  int32_t* scan_blocks;  // scan scratch
  int64_t scan_nblocks;

  double* dv[3];    // collision term per particle (sorted order)
  double* lor[3];   // dt q/m (E_p - E^M_p) of the last kick without drift
  bool lor_valid;   // lor matches the current order, positions and field
  bool rec_state;   // the next sort reads the state from records in the staging area
  // A state load's records binned by cell as well ([ncell][bin_cap]
  // records; allocated at the first load that reads the caller's arrays
  // in place, when they fit): the sort then reads each cell's records as
  // one span, and skips its scatter, unless a cell outgrew its bin.
  float4* bins;
  int64_t bin_cap;  // 0: no bins
  int* bin_over;    // device flag: some cell held more than bin_cap particles
  bool bin_tried;   // the bins' allocation was attempted
  bool bin_state;   // the next sort reads the records from the bins
  int64_t binned_loads;  // state loads sorted from the bins (pic_stats)
  bool inv_valid;   // perm holds the inverse of the current sort permutation
  // auxiliary stream (created at first use, higher priority) and its fork
  // and join events: the inverse permutation overlaps the state store
  cudaStream_t aux;
  cudaEvent_t aux_fork, aux_join;
  // multigrid-preconditioned CG of the precision form (0 levels: plain CG)
  int mg_nlev, mg_nlev_grid;
  float *mg_z, *mg_z2;  // the preconditioned residual and a second buffer
  float* mg_work;       // the coarse levels' iterate, second buffer and rhs, level after level
  double* dvm[3];   // source term when requested separately

  // precision form: int32 cell + FP32 offset, FP32 v and v^M, FP32 mesh
  int32_t* cell32[2];
  float* off[2][3];
  float* vf[2][3];
  float* vmf[2][3];
  float* dvf[3];
  float* dvmf[3];
  float* lorf[3];
  float4* Ef4;      // (Ex, Ey, Ez, 0) per node: one 16-byte load per node in the gather
  float* phif;
  float* bf;
  float* cgf_r;
  float* cgf_p;
  float* cgf_q;
  float* overlay32;

  // mesh
  double* corner;   // [8][ncell] per-cell CIC partials
  double* rho;      // [ncell]
  double* b;        // [ncell]
  double* rhs_part; // per-block partial sums of b
  int64_t rhs_blocks;
  double* phi;      // [ncell]
  double* E[3];     // [ncell] each
  double* cg_r;
  double* cg_p[2];
  double* cg_q;
  double* cg_red;   // reduction slots
  unsigned int* cg_bar;  // grid barrier words
  int* cg_info;     // [0] iterations, [1] status (0 ok, 1 noconv, 2 timeout)
  double* cg_res;   // relative residual
  int cg_grid, cg_block;
  bool stall_next_cg;  // failure injection: the next CG launch has one block leave before its first barrier

  // G^{-1} knot tables (FP64 and FP32)
  double* ginv;
  float* ginv_f;

  // collisions
  double* overlay;  // per-lane working velocities
  int dsmc_grid, dsmc_block, dsmc_G, dsmc_Kc, bm_words;
  int64_t dsmc_groups;
  size_t dsmc_smem;
  pic::AdjointBuffers* adj;      // pathwise-adjoint working set, allocated on first use
  unsigned long long* counters;  // n_cand, n_coll, n_gmax, n_tie, n_floor_tie
  unsigned long long* dsmc_queue;  // next cell group of the FP32 collision kernel (zeroed per launch)
  // decision log of the collision calls (pic_set_decision_log)
  // per-step record since pic_reset_stats: [kHistSteps][4] (CG iterations,
  // candidates, collisions, g > g_max); hist_row is the current step's row
  // while pic_step enqueues it, else nullptr
  long long* step_hist;
  long long* hist_row;
  int64_t hist_base;
  int32_t* dlog;                 // [dlog_cap][8]
  unsigned long long* dlog_n;    // records produced
  int64_t dlog_cap;
  int dlog_mode;
  // recorded scattering angles (PIC_VERIFY_ANGLES): histograms of F^M(chi)
  // and eps/(2 pi), and the scratch of their CDF-error reduction
  unsigned long long* ang_hist;  // [2][PIC_ANGLE_BINS]
  unsigned long long* ang_bsum;  // [2][kAngleBlocks] counts, then [2][kAngleBlocks] maxima
  double* ang_part;              // [2][kAngleBlocks][2] (sum of e^2, max |e|)
  double* ang_out;               // [8]
  int* flags;       // sticky: [0] bits 1 capacity, 2 no convergence, 4 timeout; [1] max CG iterations

  // error norms
  double* err_part; // per-block partials
  int err_blocks;
  double* err_out;  // 14 doubles

  // boundary staging
  double* stage;    // 6 N_p doubles
  int32_t* stage_i; // N_p ints

  // host state
  double t0;
  int64_t step;
  bool sampled;
  int64_t launches;
  int cg_iters_last, cg_iters_max;
  double cg_res_last;
  pic_status pending;  // sticky status from asynchronous checks

  // batch of independent replicates (0 = single domain). Arrays above hold
  // all replicates back to back: particles at poff[r], cells and nodes at
  // coff[r] (padded to a multiple of 256).
  int nrep;
  pic::BatchRep* reps_dev;       // [nrep] per-replicate parameters
  pic::BatchRep* reps_host;
  pic::Params* prm_dev;          // [nrep] FP64 parameters
  pic::Params* prm_host;
  uint16_t* rep_of_cell;         // [ncell total] replicate of each cell/node, 0xFFFF = padding
  int64_t* poff_dev;             // [nrep + 1]
  int2* dsmc_items;              // (replicate, first local cell) per warp work item
  int64_t n_items;
  int* cg_order;                 // replicates by decreasing size
  int* cg_iters_rep;             // [nrep]
  double* cg_res_rep;            // [nrep]
  pic::TimeTerms* tt_dev;        // [nrep][3]: t_n, t_{n+1/2}, t_{n+1}, then the step (int64)
  pic::TimeTerms* tt_host;       // pinned mirror
  int kick_block;                // autotuned block size of the batched kick (per-phase launches)
  int tune_step;
  float tune_ms[8];
  // persistent batched step (one launch per step): work items of the chosen
  // candidate (block size, tile shapes), items per (replicate, phase), queue
  // head and completion counters, the persistent grid per block size
  int4* step_items;
  int4* step_items_host;
  int64_t step_items_cap;
  int n_step_items;
  int* step_need;                // [nrep][kStepPhases]
  int* step_sync;                // [0] queue head, then [nrep][kStepPhases] completed items
  int step_stall_item;           // the item a stall injection leaves uncounted
  int step_cand;                 // candidate the items were built for
  int step_grid[2];              // persistent grid for 128- and 256-thread blocks (0: unavailable)
  int64_t overlay_warps;         // warps the collision overlay is sized for (batches)
  unsigned* cg_team_bar;         // [nrep] team barrier counters of the batched solves
  double* cg_team_red;           // [nrep][2][kTeamMax] part totals
  int2* cg_parts;                // (replicate, part) items of the per-phase batched solve, CG order
  int n_cg_parts;
  int* cg_head;                  // its queue head
  cudaGraphExec_t graph[2];      // steady-state step, by buffer parity
  int64_t graph_launches;        // kernels per captured step
  int64_t graph_replays;
  bool use_graphs;

  // profiling: pairs of events recorded on the stream, resolved lazily
  bool profiling;
  cudaEvent_t* ev_pool;
  int* ev_class;
  int ev_cap, ev_used;
  double prof_ms[PIC_NUM_KERNEL_CLASSES];
  int64_t prof_launches[PIC_NUM_KERNEL_CLASSES];
};

namespace pic {
enum KernelClass {
  KC_SAMPLE = 0, KC_SORT = 1, KC_GATHER = 2, KC_RHS = 3, KC_CG = 4,
  KC_DSMC = 5, KC_KICK = 6, KC_ERR = 7, KC_OTHER = 8
};

// Kernel-launching helpers (each returns cudaGetLastError()).
cudaError_t launch_sample(pic_ctx* c, double t0);
cudaError_t launch_load_state(pic_ctx* c, const double* x, const double* v, double t);
cudaError_t launch_store_state(pic_ctx* c, double* xv_dev);
cudaError_t launch_keys(pic_ctx* c);
cudaError_t launch_sort(pic_ctx* c);            // scan + scatter + in-cell sort + gather + CIC
cudaError_t launch_rhs(pic_ctx* c, double t);
cudaError_t launch_cg(pic_ctx* c);             // CG + zero-mean + E
// the FP64 CG on caller buffers: solves -Lap_h x = b - mean(b) (warm start
// from x, mean removed from x) and writes E = -grad_h x
cudaError_t launch_cg_on(pic_ctx* c, double* b, double* x, const double* rhs_part, int rhs_blocks, double* E0,
                         double* E1, double* E2);
using StepHook = std::function<cudaError_t(int)>;
cudaError_t step_fp64(pic_ctx* c, int64_t n, const StepHook* hook);
cudaError_t launch_dsmc(pic_ctx* c, uint32_t c0, bool separate_source, double t_src);
// kick at time tE; drift to th if drift. Reuses / refreshes c->lor.
cudaError_t launch_kick(pic_ctx* c, double tE, bool with_collisions, bool drift, double th, double tn1);
cudaError_t launch_errors(pic_ctx* c, double t);
TimeTerms time_terms(const Params& P, double t);
ParamsF params_f(const Params& P);

// batched kernels (k_batch.cu)
cudaError_t launch_batch_sample(pic_ctx* c, const double* xv);
cudaError_t launch_batch_rhs(pic_ctx* c, int slot);
cudaError_t launch_batch_cg(pic_ctx* c);
cudaError_t launch_batch_dsmc(pic_ctx* c, int phase);
cudaError_t launch_batch_kick(pic_ctx* c, bool with_collisions, bool drift);
cudaError_t launch_batch_errors(pic_ctx* c, int rep, double t);
cudaError_t launch_batch_store_state(pic_ctx* c, int rep, double* xv);
cudaError_t launch_store_field(pic_ctx* c, double* rho, double* phi, double* E);
cudaError_t launch_store_sort(pic_ctx* c, int32_t* cell_of_pid, int32_t* perm);
cudaError_t launch_store_dv(pic_ctx* c, double* dv, double* dvm);
cudaError_t launch_scan(pic_ctx* c);           // scan of counts into start
cudaError_t launch_scan_scatter(pic_ctx* c);   // scan of counts + scatter into perm
cudaError_t launch_err_final(pic_ctx* c, int nblocks);
// precision form
// held >= 0: the buffer of a state the context holds, whose v^M (tau) the
// load keeps instead of recomputing them, read from its sorted arrays at
// the inverse of its sort permutation (formed here when perm does not hold
// it); to_records: write the state into the staging area as 48-byte records
// with their cell keys and ranks (sort_and_field then skips the keys), for
// a state load whose caller arrays are used in place
cudaError_t launch_sample32(pic_ctx* c, double t0, const double* x, const double* v, int held = -1,
                           bool to_records = false);
cudaError_t ensure_aux_stream(pic_ctx* c);    // the auxiliary stream and its events
// the multigrid levels of an n^3 mesh (n a power of two >= 16, else 0) and
// the floats their coarse levels need
int mg_levels(int n, int* nlev_grid, size_t* work_floats);
cudaError_t launch_keys32(pic_ctx* c);
cudaError_t launch_gather32(pic_ctx* c);
cudaError_t launch_dsmc32(pic_ctx* c, uint32_t c0, bool separate_source, double t_src);
cudaError_t launch_kick32(pic_ctx* c, double tE, bool with_collisions, bool drift, double th, double tn1);
// angle CDF errors of the recorded collisions into out (synchronises)
cudaError_t launch_angle_stats(pic_ctx* c, pic_angle_stats* out);
// device memory through the context's allocator; adjoint buffers (k_adjoint.cu)
void* ctx_alloc(pic_ctx* c, size_t bytes);
void dev_free_ctx(pic_ctx* c, void* p);
// persistent batched step (k_batch.cu)
constexpr int kStepPhases = 9;
int step_candidates();
int step_block_of(int cand);
int step_tile_of(int cand);
const void* step_kernel_ptr(int block);
size_t step_smem(const pic_ctx* c, int block);
cudaError_t build_step_items(pic_ctx* c, int cand);
cudaError_t launch_batch_step(pic_ctx* c, bool coll, bool stall);
void ctx_free(pic_ctx* c, void* p);
void adjoint_free(pic_ctx* c);
cudaError_t launch_cg32(pic_ctx* c);
cudaError_t launch_errors32(pic_ctx* c, double t);
cudaError_t launch_store_state32(pic_ctx* c, double* xv_dev, int32_t* cell_of_pid);
cudaError_t launch_store_state32_by_pid(pic_ctx* c, double* x, double* v);
cudaError_t launch_store_field32(pic_ctx* c, double* phi, double* E);
cudaError_t launch_store_dv32(pic_ctx* c, double* dv, double* dvm);

// Profiling brackets (no-ops unless profiling is on).
void prof_begin(pic_ctx* c);
void prof_end(pic_ctx* c, int kclass);
}  // namespace pic
