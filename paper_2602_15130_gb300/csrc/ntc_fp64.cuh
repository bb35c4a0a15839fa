// Algorithm 1 for one (cell, outcome) lane in FP64, shared by the K-averaged
// collision kernel and its pathwise adjoint. The lane's working velocities
// live in a private overlay ov, valid where the lane's bitmap bm has the
// particle's bit; untouched particles are read from v. A recorder receives
// every accepted isotropic-or-anisotropic pair (in-cell indices, the
// pre-collision velocities, the scattering direction n and g) before the
// update; the forward kernel passes one that does nothing.
#pragma once

#include "pic_internal.cuh"

namespace pic {

struct NoRecord {
  __device__ __forceinline__ void operator()(uint32_t, uint32_t, const double*, const double*, const double*,
                                             double) const {}
};

struct LaneCounts {
  unsigned long long cand, coll, gmax, tie;
};

__device__ __forceinline__ void load_vel(int p, const uint32_t* bm, const double* ov, const double* v0,
                                         const double* v1, const double* v2, double* o) {
  if ((bm[p >> 5] >> (p & 31)) & 1u) {
    o[0] = ov[3 * p]; o[1] = ov[3 * p + 1]; o[2] = ov[3 * p + 2];
  } else {
    o[0] = v0[p]; o[1] = v1[p]; o[2] = v2[p];
  }
}

// kVerify: the verification switches of Sec. 5.4 (injected Errors 1 and 2,
// manufactured anisotropy, angle recording) are compiled in.
// lg: decision log (mode 0 off); every decision is logged only in the
// kVerify instantiation, flagged near ties in both.
template <bool kVerify, class Rec>
__device__ void ntc_outcome(const Params& P, uint32_t c0, uint32_t cell, uint32_t o, int c,
                            const double* v0, const double* v1, const double* v2, uint32_t* bm,
                            double* ov, LaneCounts& cnt, Rec& rec, const DLog lg = DLog{nullptr, nullptr, 0, 0}) {
  // the chi stream (c0, cell, slot, (o << 8) | 1): word 0 of slot 0 is the
  // N_pairs uniform, word (s + 1) mod 4 of slot (s + 1) / 4 the chi of
  // candidate s
  U4 bchi = philox(c0, cell, 0u, (o << 8) | 1u, P.key0, P.key1);
  long long chi_group = 0;
  const double base = __dmul_rn(__dmul_rn((double)((long long)c * (long long)(c - 1)), P.pmax), 0.5);
  const long long npairs = (long long)floor(__dadd_rn(base, unif32(bchi.x)));
  const bool log_all = kVerify && lg.mode == PIC_DLOG_ALL;
  if (log_all) dlog_put(lg, c0, cell, o, -1, -1, -1, (int)npairs, PIC_DLOG_NPAIRS);
  // candidate s: block (c0, cell, s, o << 8) = (p, q, accept, epsilon);
  // its chi block is formed when an accepted candidate needs it
  for (long long s = 0; s < npairs; ++s) {
    const U4 b0 = philox(c0, cell, (uint32_t)s, o << 8, P.key0, P.key1);
    const uint32_t p = draw_index(b0.x, (uint32_t)c);
    // q uniform over the other c - 1 particles: the distribution of
    // drawing again until q != p
    uint32_t q = draw_index(b0.y, (uint32_t)(c - 1));
    q += q >= p ? 1u : 0u;
    double vp[3], vq[3];
    load_vel((int)p, bm, ov, v0, v1, v2, vp);
    load_vel((int)q, bm, ov, v0, v1, v2, vq);
    const double dx = __dsub_rn(vp[0], vq[0]), dy = __dsub_rn(vp[1], vq[1]), dz = __dsub_rn(vp[2], vq[2]);
    const double g2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
    const double g = __dsqrt_rn(g2);
    // sigma(g) g / (sigma g)_max: hard sphere, or the odd-power sigma of Eq. sigma_ms
    const double ratio = P.n_sigma == 0 ? __ddiv_rn(__dmul_rn(P.sigma0, g), P.sg_max)
                                        : __ddiv_rn(sigma_g(P, g2), P.sg_max);
    const double U = unif32(b0.z);
    ++cnt.cand;
    if (g > P.gmax) ++cnt.gmax;
    const bool tie = fabs(U - ratio) < 1e-12;
    if (tie) ++cnt.tie;
    if (log_all || (tie && lg.mode != PIC_DLOG_OFF))
      dlog_put(lg, c0, cell, o, (int)s, (int)p, (int)q, U < ratio ? 1 : 0, tie ? PIC_DLOG_TIE : 0);
    if (U < ratio) {
      const long long js = s + 1;
      if ((js >> 2) != chi_group) {
        chi_group = js >> 2;
        bchi = philox(c0, cell, (uint32_t)chi_group, (o << 8) | 1u, P.key0, P.key1);
      }
      const uint32_t wchi = (js & 3) == 0 ? bchi.x : (js & 3) == 1 ? bchi.y : (js & 3) == 2 ? bchi.z : bchi.w;
      if (kVerify && (P.verify & PIC_VERIFY_ERROR2)) {
        // injected Error 2: swap with probability 1/2 (coin = chi draw)
        const bool swap = unif32(wchi) < 0.5;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          ov[3 * p + d] = swap ? vq[d] : vp[d];
          ov[3 * q + d] = swap ? vp[d] : vq[d];
        }
      } else {
        const double eps = __dmul_rn(kTwoPi, unif32(b0.w));
        double se, ce;
        sincos(eps, &se, &ce);
        double uchi = unif32(wchi);
        if (kVerify && (P.verify & PIC_VERIFY_ANISO)) uchi = aniso_u(uchi);
        const double cchi = __dsub_rn(1.0, __dmul_rn(2.0, uchi));
        const double schi = __dsqrt_rn(__dsub_rn(1.0, __dmul_rn(cchi, cchi)));
        const double nv[3] = {__dmul_rn(ce, schi), __dmul_rn(se, schi), cchi};
        rec(p, q, vp, vq, nv, g);
        const bool err1 = kVerify && (P.verify & PIC_VERIFY_ERROR1);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          const double gp = __dmul_rn(g, nv[d]);
          // Eq. v_cm; injected Error 1 flips the sign of v_q
          const double cm = __dmul_rn(err1 ? __dsub_rn(vp[d], vq[d]) : __dadd_rn(vp[d], vq[d]), 0.5);
          ov[3 * p + d] = __dadd_rn(cm, __dmul_rn(gp, 0.5));
          ov[3 * q + d] = __dsub_rn(cm, __dmul_rn(gp, 0.5));
        }
      }
      if (kVerify && P.ang_hist)
        record_angles(P.ang_hist, (P.verify & PIC_VERIFY_ANISO) != 0, g, __dsub_rn(ov[3 * p], ov[3 * q]),
                      __dsub_rn(ov[3 * p + 1], ov[3 * q + 1]), __dsub_rn(ov[3 * p + 2], ov[3 * q + 2]));
      bm[p >> 5] |= 1u << (p & 31);
      bm[q >> 5] |= 1u << (q & 31);
      ++cnt.coll;
    }
  }
}

}  // namespace pic
