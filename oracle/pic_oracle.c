/*
 * Plain FP64 CPU oracle of the manufactured-solution PIC + DSMC time step of
 * Freno, McDoniel, Moore and Matula, "Code-Verification Techniques for
 * Particle-in-Cell Simulations with Direct Simulation Monte Carlo Collisions".
 *
 * TEST INFRASTRUCTURE. Only the tests, the smoke check and the CPU-baseline
 * leg of the benchmark may load this library. It shares no code, header,
 * table or constant generator with the CUDA path, and it never calls it.
 *
 * Everything is written for a reader checking it against the paper: plain
 * loops, array-of-structures layouts ([particle][component]), FP64
 * throughout, no blocking, no fusion, no reordering beyond what the paper
 * states. It must be compiled with -ffp-contract=off so that x86 and Arm
 * builds give the same bits. Loops over independent cells or particles
 * may run on several host threads (OpenMP, orc_set_threads; one thread by
 * default): each iteration writes only its own cell's or particle's
 * results, so the bits do not depend on the thread count.
 *
 * Workloads, on the periodic unit cube [0,1)^3 with n^3 cells of size
 * h = 1/n and node i at x = i h:
 *  dist = 0 (the paper's Sec. 3 machinery applied to a simpler distribution)
 *   f_x(x,t) = N prod_d (1 + A sin(2 pi (x_d - c t)))                 (Eq. fx)
 *   f_v(v,t) = prod_d Normal(v_d; mu_d, s^2), constant in time         (Eq. fv)
 *  dist = 1 (the paper's own problem of Sec. 5.2, lengths in units of L,
 *  times in units of T = t_ref):
 *   f_x(x,t) = N prod_d (1 + A_d(t) sin(2 pi (x_d - s_d(t)))) with
 *     A = (e^{t/T}/5, 1/5, -e^{t/T}/6), s = (0, 3 e^{t/T}/20, -e^{t/T}/15)
 *   f_v(v,t) = prod_d (2/sqrt pi) v_d^2 / vh_d^3 e^{-v_d^2/vh_d^2}     (Eq. fv)
 *     vh = vbar (1 + sin(pi t/(2T))/5, 1 + cos(pi t/T)/5, 1 + sin(3 pi t/(2T))/5)
 *  both:
 *   phi^M(x,t) = phibar e^{t/(2T)} prod_d sin(2 pi (x_d - s_d))        (Sec. 5.2)
 *   cross section: n_sigma = 0 hard sphere sigma(g) = sigma0; n_sigma > 0
 *   sigma(g) = sum_{k<n_sigma} sigma_k g^{2k-1} (Eq. sigma_ms) with its
 *   exact source (Eqs. vel_change_3, fn); isotropic scattering (Eq. chi_iso)
 *
 * Every function is pinned to something other than itself, in
 * tests/test_oracle_pins.py, test_oracle_verification_pins.py and
 * test_oracle_paper_pins.py; none is left unpinned:
 *  - orc_philox, orc_u52, orc_u32, orc_index: published known-answer
 *    vectors; uniform and index conventions.
 *  - orc_sample_xi: uniformity, distinct draws.
 *  - orc_fxd, orc_Fxd, orc_xM, orc_xMdot, orc_fx_terms, orc_fx, orc_Fx,
 *    orc_xM_d, orc_xMdot_d: printed forms, quadrature of f_x, inversion to
 *    1e-14, central differences in t.
 *  - orc_Phi, orc_Phi_inv, orc_vM, orc_vhat, orc_fv_paper, orc_Fv_paper,
 *    orc_vM_t, orc_vMdot: scipy ndtri, printed forms, inversion, central
 *    differences, sampled moments.
 *  - orc_phiM, orc_EM, orc_lap_phiM, orc_rhoM: finite differences, integral.
 *  - orc_hs_R, orc_hs_source: series against the closed form, Monte Carlo
 *    vector, expected NTC change.
 *  - orc_fn, orc_odd_source: printed formulas, Gauss-Hermite quadrature.
 *  - orc_sigma_g, orc_sg_max, orc_pmax: dense scan, Table 1 column.
 *  - orc_cell_of, orc_sort, orc_deposit, orc_gather, orc_rhs: brute force,
 *    total charge, affine fields, the right-hand side rebuilt term by term
 *    from closed forms.
 *  - orc_neg_lap, orc_cg, orc_efield, orc_field: Fourier eigenvalues, FFT
 *    solve, closed forms, uncoupled phi^M.
 *  - orc_ntc_cell, orc_dsmc_avg, orc_aniso_F, orc_aniso_u: momentum and
 *    energy, relative speed, isotropy, brute-force expectation, variance
 *    falling as 1/K and growing as dt (Eq. var), Errors 1 and 2,
 *    anisotropic CDF and its inverse.
 *  - orc_step, orc_source_all, orc_wrap: observed second order, zero-mean
 *    collision error, sign of the source, wrap convention.
 *  - orc_errors, orc_objective and the angle metric of oracle.py:
 *    hand-computed values, KS bound, field energy plus velocity error.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846

typedef struct {
  int64_t n;            /* cells per axis                                 */
  int64_t np;           /* computational particles N_p                   */
  int64_t K;            /* N_avg, outcomes per collision call; 0 = off    */
  int64_t cg_maxit;
  uint64_t seed;
  int64_t couple_qm_zero;  /* q/m = 0: field does not push particles      */
  int64_t couple_q_zero;   /* q = 0: particles do not source the field    */
  double dt, qm, q, eps0, nphys;
  double sigma0, gmax;
  double fx_amp, fx_speed;
  double vmean[3];
  double vsig;
  double phi_amp, phi_T;
  double phi_shift[3];
  double cg_tol;
  int64_t verify;  /* verification switches, bit flags (Sec. 5.4):
                    *   1  isolated-collision mode: the drift moves x by the
                    *      exact manufactured increment x^M(t_{n+1}) - x^M(t_n)
                    *      in place of dt xdot^M(t_{n+1/2}) (v^M is constant,
                    *      so the kicks' vdot^M terms are zero either way)
                    *   2  injected Error 1: v_cm = (v_p - v_q)/2
                    *   4  injected Error 2: velocities swapped with
                    *      probability 1/2, else left unchanged
                    *   8  record (chi, eps) of every collision (Sec. 4.4)
                    *  16  manufactured anisotropic scattering (Sec. 5.1):
                    *      p_chi = (29/2 + 12 cos chi - 20 cos^3 chi)
                    *      sin chi / 29 in place of sin chi / 2           */
  double E_app[3];   /* uniform applied field added to E_p in the push      */
  int64_t dist;      /* 0: travelling-wave f_x and Gaussian f_v; 1: Sec. 5.2 */
  int64_t n_sigma;   /* 0: hard sphere sigma0; 1..3: odd-power sigma_k      */
  double sigma_n[3]; /* sigma_k of Eq. sigma_ms (k < n_sigma)               */
  double vbar;       /* dist 1: vbar of vh_d(t)                             */
  double t_ref;      /* dist 1: T of A_d(t), s_d(t), vh_d(t)                */
} orc_cfg;

#define ORC_ISOLATE 1
#define ORC_ERROR1 2
#define ORC_ERROR2 4
#define ORC_ANGLES 8
#define ORC_ANISO 16

/* ------------------------------------------------------------------------
 * Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
 * easy as 1, 2, 3", SC'11): ten rounds of two 32x32->64 multiplies with the
 * published multipliers, key bumped by the published Weyl constants between
 * rounds. Pinned by the published known-answer vectors.
 * ---------------------------------------------------------------------- */
void orc_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; round++) {
    if (round > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    uint64_t prod0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
    uint64_t prod1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
    uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static void philox4(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                    uint64_t seed, uint32_t out[4]) {
  uint32_t ctr[4] = {c0, c1, c2, c3};
  uint32_t key[2] = {(uint32_t)(seed & 0xFFFFFFFFu), (uint32_t)(seed >> 32)};
  orc_philox(ctr, key, out);
}

/* Uniforms used by the method's draws. Both are odd multiples of a power of
 * two, hence exactly representable and strictly inside (0, 1).           */
double orc_u52(uint32_t hi, uint32_t lo) {
  uint64_t m = ((uint64_t)hi << 20) | (uint64_t)(lo >> 12); /* 52 bits */
  return (double)(2 * m + 1) * 0x1p-53;
}
double orc_u32(uint32_t w) { return (double)(2 * (uint64_t)w + 1) * 0x1p-33; }
/* floor(U * c) with U = w / 2^32: Algorithm 1's "floor(rand * N) + 1", 0-based */
uint32_t orc_index(uint32_t w, uint32_t c) {
  return (uint32_t)(((uint64_t)w * (uint64_t)c) >> 32);
}

/* ------------------------------------------------------------------------
 * Manufactured distribution, Sec. 3.1 / 3.2.
 * ---------------------------------------------------------------------- */

/* f_{x_d}(x,t) = 1 + A sin(2 pi (x - c t)), unit integral over [0,1).    */
double orc_fxd(const orc_cfg* cf, double x, double t) {
  return 1.0 + cf->fx_amp * sin(2.0 * ORC_PI * (x - cf->fx_speed * t));
}

/* Amplitude A_d(t) and phase s_d(t) of the paper's f_{x_d} = 1 + A_d
 * sin(2 pi (x - s_d)) on the unit cube (Sec. 5.2), with their time
 * derivatives. dist = 0 reads A_d = A, s_d = c t.                         */
void orc_fx_terms(const orc_cfg* cf, int d, double t, double out[4]) {
  if (cf->dist == 0) {
    out[0] = cf->fx_amp; out[1] = cf->fx_speed * t;
    out[2] = 0.0;        out[3] = cf->fx_speed;
    return;
  }
  double T = cf->t_ref, e = exp(t / T);
  if (d == 0)      { out[0] = e / 5.0;  out[1] = 0.0; }
  else if (d == 1) { out[0] = 1.0 / 5.0; out[1] = 3.0 * e / 20.0; }
  else             { out[0] = -e / 6.0; out[1] = -e / 15.0; }
  /* d/dt e^{t/T} = e^{t/T} / T; the constant amplitude has derivative 0 */
  out[2] = (d == 1) ? 0.0 : out[0] / T;
  out[3] = out[1] / T;
}

/* f_{x_d}(x,t) of either form (unit integral over [0,1)).                */
double orc_fx(const orc_cfg* cf, int d, double x, double t) {
  if (cf->dist == 0) return orc_fxd(cf, x, t);
  double a[4];
  orc_fx_terms(cf, d, t, a);
  return 1.0 + a[0] * sin(2.0 * ORC_PI * (x - a[1]));
}

/* F_{x_d}(x,t) = int_0^x f_{x_d}(x',t) dx' in closed form (Sec. 3.1).   */
double orc_Fxd(const orc_cfg* cf, double x, double t) {
  double A = cf->fx_amp, c = cf->fx_speed;
  return x + A / (2.0 * ORC_PI) *
                 (cos(2.0 * ORC_PI * (0.0 - c * t)) - cos(2.0 * ORC_PI * (x - c * t)));
}

/* F_{x_d}(x,t) of either form: x + A_d/(2 pi) [cos(2 pi (0 - s_d)) -
 * cos(2 pi (x - s_d))].                                                   */
double orc_Fx(const orc_cfg* cf, int d, double x, double t) {
  if (cf->dist == 0) return orc_Fxd(cf, x, t);
  double a[4];
  orc_fx_terms(cf, d, t, a);
  return x + a[0] / (2.0 * ORC_PI) *
                 (cos(2.0 * ORC_PI * (0.0 - a[1])) - cos(2.0 * ORC_PI * (x - a[1])));
}

/* x_d^M(t) solves F_{x_d}(x^M, t) = xi on [0,1] (Eq. mms_sol), bisection. */
double orc_xM_d(const orc_cfg* cf, int d, double xi, double t) {
  double lo = 0.0, hi = 1.0;
  for (int it = 0; it < 200; it++) {
    double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    if (orc_Fx(cf, d, mid, t) < xi) lo = mid; else hi = mid;
  }
  double rl = fabs(orc_Fx(cf, d, lo, t) - xi), rh = fabs(orc_Fx(cf, d, hi, t) - xi);
  return rl <= rh ? lo : hi;
}

/* x^M(t) solves F_x(x^M, t) = xi on [0,1] (Eq. mms_sol). F is increasing,
 * so plain bisection to the last representable bracket.                  */
double orc_xM(const orc_cfg* cf, double xi, double t) {
  double lo = 0.0, hi = 1.0;
  for (int it = 0; it < 200; it++) {
    double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    if (orc_Fxd(cf, mid, t) < xi) lo = mid; else hi = mid;
  }
  /* return the bracket end with the smaller residual */
  double rl = fabs(orc_Fxd(cf, lo, t) - xi), rh = fabs(orc_Fxd(cf, hi, t) - xi);
  return rl <= rh ? lo : hi;
}

/* xdot^M = -(1/f_x(x^M,t)) int_0^{x^M} d/dt f_x(x',t) dx' (Sec. 3.2). With
 * d/dt f = -2 pi A c cos(2 pi (x - c t)), the integral is
 * -A c [sin(2 pi (x^M - c t)) - sin(2 pi (0 - c t))].                      */
double orc_xMdot(const orc_cfg* cf, double xM, double t) {
  double A = cf->fx_amp, c = cf->fx_speed;
  double integral = -A * c * (sin(2.0 * ORC_PI * (xM - c * t)) -
                              sin(2.0 * ORC_PI * (0.0 - c * t)));
  return -integral / orc_fxd(cf, xM, t);
}

/* xdot_d^M of either form (Sec. 3.2): with d/dt f = A' sin(2 pi (x - s))
 * - 2 pi A s' cos(2 pi (x - s)), the integral from 0 to x^M is
 * A'/(2 pi) [cos(2 pi (0 - s)) - cos(2 pi (x^M - s))]
 * - A s' [sin(2 pi (x^M - s)) - sin(2 pi (0 - s))].                        */
double orc_xMdot_d(const orc_cfg* cf, int d, double xM, double t) {
  if (cf->dist == 0) return orc_xMdot(cf, xM, t);
  double a[4];
  orc_fx_terms(cf, d, t, a);
  double A = a[0], s = a[1], dA = a[2], ds = a[3];
  double integral = dA / (2.0 * ORC_PI) * (cos(2.0 * ORC_PI * (0.0 - s)) - cos(2.0 * ORC_PI * (xM - s))) -
                    A * ds * (sin(2.0 * ORC_PI * (xM - s)) - sin(2.0 * ORC_PI * (0.0 - s)));
  return -integral / orc_fx(cf, d, xM, t);
}

/* Standard normal CDF Phi(z) = erfc(-z/sqrt 2)/2.                        */
static double orc_Phi(double z) { return 0.5 * erfc(-z / sqrt(2.0)); }

/* v^M solves F_v(v^M) = xi for the Gaussian f_v (Eq. mms_sol); f_v does not
 * depend on t, so v^M is constant and vdot^M = 0. Bisection on Phi in the
 * lower tail; for xi > 1/2 the symmetry Phi^{-1}(xi) = -Phi^{-1}(1 - xi)
 * (1 - xi is exact there) keeps the upper tail well conditioned.          */
static double orc_Phi_inv(double xi) {
  if (xi > 0.5) return -orc_Phi_inv(1.0 - xi);
  double lo = -40.0, hi = 0.0;
  for (int it = 0; it < 400; it++) {
    double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    if (orc_Phi(mid) < xi) lo = mid; else hi = mid;
  }
  return 0.5 * (lo + hi);
}
double orc_vM(const orc_cfg* cf, int d, double xi) {
  return cf->vmean[d] + cf->vsig * orc_Phi_inv(xi);
}

/* The paper's velocity scales vh_d(t) (Sec. 5.2) and their derivatives.  */
void orc_vhat(const orc_cfg* cf, double t, double vh[3], double dvh[3]) {
  double T = cf->t_ref, vb = cf->vbar;
  vh[0] = vb * (1.0 + sin(ORC_PI * t / (2.0 * T)) / 5.0);
  vh[1] = vb * (1.0 + cos(ORC_PI * t / T) / 5.0);
  vh[2] = vb * (1.0 + sin(3.0 * ORC_PI * t / (2.0 * T)) / 5.0);
  dvh[0] = vb * (ORC_PI / (2.0 * T)) * cos(ORC_PI * t / (2.0 * T)) / 5.0;
  dvh[1] = -vb * (ORC_PI / T) * sin(ORC_PI * t / T) / 5.0;
  dvh[2] = vb * (3.0 * ORC_PI / (2.0 * T)) * cos(3.0 * ORC_PI * t / (2.0 * T)) / 5.0;
}

/* The paper's f_{v_d}(v,t) = (2/sqrt pi) v^2/vh^3 e^{-v^2/vh^2} (Eq. fv)
 * and its CDF F_{v_d}(v,t) = (1 + erf(v/vh))/2 - (v/vh) e^{-v^2/vh^2}/sqrt pi
 * (the antiderivative, zero at -infinity).                                */
double orc_fv_paper(const orc_cfg* cf, int d, double v, double t) {
  double vh[3], dvh[3];
  orc_vhat(cf, t, vh, dvh);
  double z = v / vh[d];
  return 2.0 / sqrt(ORC_PI) * z * z / vh[d] * exp(-z * z);
}
double orc_Fv_paper(const orc_cfg* cf, int d, double v, double t) {
  double vh[3], dvh[3];
  orc_vhat(cf, t, vh, dvh);
  double z = v / vh[d];
  return 0.5 * (1.0 + erf(z)) - z * exp(-z * z) / sqrt(ORC_PI);
}

/* v_d^M(t) solves F_{v_d}(v^M, t) = xi (Eq. mms_sol). Gaussian form: the
 * constant orc_vM. Paper form: bisection on F_v at time t; f_v is even in
 * v, so for xi > 1/2 the root is minus the root for 1 - xi (exact there). */
double orc_vM_t(const orc_cfg* cf, int d, double xi, double t) {
  if (cf->dist == 0) return orc_vM(cf, d, xi);
  if (xi > 0.5) return -orc_vM_t(cf, d, 1.0 - xi, t);
  double vh[3], dvh[3];
  orc_vhat(cf, t, vh, dvh);
  double lo = -40.0 * vh[d], hi = 0.0;
  for (int it = 0; it < 400; it++) {
    double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    if (orc_Fv_paper(cf, d, mid, t) < xi) lo = mid; else hi = mid;
  }
  return 0.5 * (lo + hi);
}

/* vdot_d^M = -(1/f_v(v^M,t)) int_{-inf}^{v^M} d/dt f_v dv' (Sec. 3.2). The
 * integral is d/dt F_v(v^M,t) = f_v(v^M,t) (-v^M vh'/vh) by the chain rule
 * on F_v(v,t) = G(v/vh(t)). Zero for the Gaussian form.                  */
double orc_vMdot(const orc_cfg* cf, int d, double vM, double t) {
  if (cf->dist == 0) return 0.0;
  double vh[3], dvh[3];
  orc_vhat(cf, t, vh, dvh);
  double integral = orc_fv_paper(cf, d, vM, t) * (-vM * dvh[d] / vh[d]);
  return -integral / orc_fv_paper(cf, d, vM, t);
}

/* phi^M and its derivatives (Sec. 5.2 form on the unit cube).            */
double orc_phiM(const orc_cfg* cf, const double x[3], double t) {
  double val = cf->phi_amp * exp(t / (2.0 * cf->phi_T));
  for (int d = 0; d < 3; d++) val *= sin(2.0 * ORC_PI * (x[d] - cf->phi_shift[d]));
  return val;
}
/* E^M = -grad phi^M (Eq. potential).                                     */
void orc_EM(const orc_cfg* cf, const double x[3], double t, double E[3]) {
  double amp = cf->phi_amp * exp(t / (2.0 * cf->phi_T));
  double s[3], c[3];
  for (int d = 0; d < 3; d++) {
    s[d] = sin(2.0 * ORC_PI * (x[d] - cf->phi_shift[d]));
    c[d] = cos(2.0 * ORC_PI * (x[d] - cf->phi_shift[d]));
  }
  E[0] = -amp * 2.0 * ORC_PI * c[0] * s[1] * s[2];
  E[1] = -amp * 2.0 * ORC_PI * s[0] * c[1] * s[2];
  E[2] = -amp * 2.0 * ORC_PI * s[0] * s[1] * c[2];
}
/* Laplacian of phi^M: each factor contributes -(2 pi)^2.                 */
double orc_lap_phiM(const orc_cfg* cf, const double x[3], double t) {
  return -3.0 * (2.0 * ORC_PI) * (2.0 * ORC_PI) * orc_phiM(cf, x, t);
}
/* rho^M = q f_x (Sec. 3.4).                                              */
double orc_rhoM(const orc_cfg* cf, double q, const double x[3], double t) {
  double f = cf->nphys;
  for (int d = 0; d < 3; d++) f *= orc_fx(cf, d, x[d], t);
  return q * f;
}

/* ------------------------------------------------------------------------
 * Expected velocity change for hard spheres, Eq. vel_change_1c with
 * sigma(g) = sigma0 and a Gaussian f_v. The paper's closed form needs odd
 * powers of g; for sigma = sigma0 the integral is instead
 *   E_{v_q ~ N(mu, s^2 I)} [ |v_q - v_p| (v_q - v_p) ] = s R(a) m,
 *   m = mu - v_p,  a = |m| / s,
 *   R(a) = sqrt(2/pi) (1 + 1/a^2) e^{-a^2/2} + (a + 2/a - 1/a^3) erf(a/sqrt 2)
 * (Stein's lemma on E|X| of a noncentral 3D normal). For a < 0.1 the same
 * function is summed as its even power series R = sqrt(2/pi) sum_j c_j a^{2j}
 * to avoid the cancellation of the 1/a terms.
 * ---------------------------------------------------------------------- */
double orc_hs_R(double a) {
  if (a < 0.1) {
    /* c_j = d_j + d_{j+1} + e_{j-1} + 2 e_j - e_{j+1} with the Taylor
     * coefficients d_k of e^{-a^2/2} and e_k of sqrt(pi/2) erf(a/sqrt 2).  */
    double d[12], e[12];
    double fact = 1.0, pow2 = 1.0;
    for (int k = 0; k < 12; k++) {
      if (k > 0) { fact *= (double)k; pow2 *= 2.0; }
      double sgn = (k % 2 == 0) ? 1.0 : -1.0;
      d[k] = sgn / (pow2 * fact);
      e[k] = sgn / (pow2 * fact * (double)(2 * k + 1));
    }
    double sum = 0.0, a2 = a * a, ap = 1.0;
    for (int j = 0; j < 10; j++) {
      double cj = d[j] + d[j + 1] + (j > 0 ? e[j - 1] : 0.0) + 2.0 * e[j] - e[j + 1];
      sum += cj * ap;
      ap *= a2;
    }
    return sqrt(2.0 / ORC_PI) * sum;
  }
  double a2 = a * a;
  return sqrt(2.0 / ORC_PI) * (1.0 + 1.0 / a2) * exp(-0.5 * a2) +
         (a + 2.0 / a - 1.0 / (a2 * a)) * erf(a / sqrt(2.0));
}

/* <Delta v_p^M>_coll = w dt (c - 1) sigma0 / (2 dV) * E[|v_q - v_p|(v_q - v_p)]
 * (Eq. vel_change_1c), c = particles in p's cell.                          */
void orc_hs_source(const orc_cfg* cf, const double vp[3], int64_t ccell, double out[3]) {
  double h = 1.0 / (double)cf->n;
  double dV = h * h * h;
  double w = cf->nphys / (double)cf->np;
  double pref = w * cf->dt * (double)(ccell - 1) * cf->sigma0 / (2.0 * dV);
  double m[3], a2 = 0.0;
  for (int d = 0; d < 3; d++) {
    m[d] = cf->vmean[d] - vp[d];
    a2 += m[d] * m[d];
  }
  double a = sqrt(a2) / cf->vsig;
  double R = orc_hs_R(a);
  for (int d = 0; d < 3; d++) out[d] = pref * cf->vsig * R * m[d];
}

/* ------------------------------------------------------------------------
 * Manufactured cross section sigma(g) = sum_k sigma_k g^{2k-1} (Eq.
 * sigma_ms), so sigma(g) g = sum_k sigma_k g^{2k}, and its source (Eq.
 * vel_change_3): <Delta v_p^M> = w dt (c - 1)/(2 dV) sum_k sigma_k f_k with
 * f_k = E_{v_q ~ f_v}[ g^{2k} (v_q - v_p) ] (Eq. fn).
 *
 * f_k is evaluated from its definition by expanding the polynomial: with
 * X = v_q - v_p, |X|^{2k} X_i = sum_{a+b+c=k} k!/(a! b! c!) X_1^{2a} X_2^{2b}
 * X_3^{2c} X_i, the components of v_q are independent, and
 * E[X_j^m] = sum_l C(m,l) E[V_j^l] (-v_pj)^{m-l} with the raw moments of
 * f_{v_j}: Gaussian E[V^l] = sum_{r even} C(l,r) mu^{l-r} s^r (r-1)!!;
 * paper form E[V^l] = vh^l (l+1)!!/2^{l/2} for even l, 0 for odd l.
 * ---------------------------------------------------------------------- */
static double binom(int n, int k) {
  double r = 1.0;
  for (int i = 1; i <= k; i++) r = r * (double)(n - k + i) / (double)i;
  return r;
}
static double dfact(int m) { /* m!! for m >= -1 */
  double r = 1.0;
  for (int i = m; i > 1; i -= 2) r *= (double)i;
  return r;
}
/* raw moment E[V_d^l] of f_{v_d} at time t                                */
static double vmoment(const orc_cfg* cf, int d, int l, double t) {
  if (cf->dist == 0) {
    double mu = cf->vmean[d], sg = cf->vsig, acc = 0.0;
    for (int r = 0; r <= l; r += 2) acc += binom(l, r) * pow(mu, l - r) * pow(sg, r) * dfact(r - 1);
    return acc;
  }
  if (l % 2) return 0.0;
  double vh[3], dvh[3];
  orc_vhat(cf, t, vh, dvh);
  return pow(vh[d], l) * dfact(l + 1) / pow(2.0, l / 2);
}
/* E[X_d^m], X_d = V_d - v_pd                                              */
static double xmoment(const orc_cfg* cf, int d, int m, double vpd, double t) {
  double acc = 0.0;
  for (int l = 0; l <= m; l++) acc += binom(m, l) * vmoment(cf, d, l, t) * pow(-vpd, m - l);
  return acc;
}
/* f_k (Eq. fn) at v_p and time t                                          */
void orc_fn(const orc_cfg* cf, int k, const double vp[3], double t, double out[3]) {
  for (int i = 0; i < 3; i++) {
    double acc = 0.0;
    for (int a = 0; a <= k; a++)
      for (int b = 0; a + b <= k; b++) {
        int c = k - a - b;
        int e[3] = {2 * a, 2 * b, 2 * c};
        e[i] += 1;
        double coef = binom(k, a) * binom(k - a, b);   /* k!/(a! b! c!) */
        acc += coef * xmoment(cf, 0, e[0], vp[0], t) * xmoment(cf, 1, e[1], vp[1], t) *
               xmoment(cf, 2, e[2], vp[2], t);
      }
    out[i] = acc;
  }
}

/* sigma(g) g = sum_{k < n_sigma} sigma_k (g^2)^k, summed in ascending k.  */
double orc_sigma_g(const orc_cfg* cf, double g2) {
  double sum = 0.0, g2k = 1.0;
  for (int k = 0; k < cf->n_sigma; k++) {
    sum += cf->sigma_n[k] * g2k;
    g2k *= g2;
  }
  return sum;
}

/* (sigma g)_max over g in [0, g_max] (Sec. 5.2): hard sphere sigma0 g_max;
 * odd power: the largest of the polynomial in u = g^2 at u = 0, at
 * u = g_max^2 and at its interior stationary point.                       */
double orc_sg_max(const orc_cfg* cf) {
  if (cf->n_sigma == 0) return cf->sigma0 * cf->gmax;
  double u1 = cf->gmax * cf->gmax;
  double best = orc_sigma_g(cf, 0.0), e = orc_sigma_g(cf, u1);
  if (e > best) best = e;
  if (cf->n_sigma == 3 && cf->sigma_n[2] != 0.0) {
    double us = -cf->sigma_n[1] / (2.0 * cf->sigma_n[2]);
    if (us > 0.0 && us < u1) {
      double m = orc_sigma_g(cf, us);
      if (m > best) best = m;
    }
  }
  return best;
}

/* <Delta v_p^M>_coll of Eq. vel_change_3 for the odd-power sigma.        */
void orc_odd_source(const orc_cfg* cf, const double vp[3], int64_t ccell, double t, double out[3]) {
  double h = 1.0 / (double)cf->n;
  double dV = h * h * h;
  double w = cf->nphys / (double)cf->np;
  double pref = w * cf->dt * (double)(ccell - 1) / (2.0 * dV);
  out[0] = out[1] = out[2] = 0.0;
  for (int k = 0; k < cf->n_sigma; k++) {
    double f[3];
    orc_fn(cf, k, vp, t, f);
    for (int d = 0; d < 3; d++) out[d] += cf->sigma_n[k] * f[d];
  }
  for (int d = 0; d < 3; d++) out[d] *= pref;
}

/* ------------------------------------------------------------------------
 * State
 * ---------------------------------------------------------------------- */
typedef struct {
  orc_cfg c;
  double t0;
  int64_t step;
  double* xi;   /* [np][6]: xi_x, xi_y, xi_z, xi_u, xi_v, xi_w */
  double* x;    /* [np][3] */
  double* v;    /* [np][3] */
  double* rho;  /* [n^3]   */
  double* phi;  /* [n^3]   */
  double* E;    /* [n^3][3] */
  int32_t* cell;  /* [np]  */
  int32_t* count; /* [n^3] */
  int32_t* start; /* [n^3 + 1] */
  int32_t* perm;  /* [np]: pids sorted by (cell, pid) */
  int64_t n_cand, n_coll, n_gmax, n_tie;
  int64_t cg_iters;
  double cg_res;
  double* ang;          /* [n_ang][2]: (chi, eps) of recorded collisions  */
  int64_t n_ang, cap_ang;
  int32_t* plog;        /* [n_plog][8] pair-list records, when logging     */
  int64_t n_plog, cap_plog;
  int plog_on;
} orc_state;

static int64_t ncell(const orc_cfg* c) { return c->n * c->n * c->n; }

/* Sampling of xi (Sec. 3.2): per particle, three Philox blocks with counter
 * (pid_lo, pid_hi, 0, 0xFFFFFF00 | j), each giving two 52-bit uniforms.    */
void orc_sample_xi(const orc_cfg* cf, int64_t pid, double xi[6]) {
  for (int j = 0; j < 3; j++) {
    uint32_t o[4];
    philox4((uint32_t)(pid & 0xFFFFFFFF), (uint32_t)((uint64_t)pid >> 32), 0u,
            0xFFFFFF00u | (uint32_t)j, cf->seed, o);
    xi[2 * j + 0] = orc_u52(o[0], o[1]);
    xi[2 * j + 1] = orc_u52(o[2], o[3]);
  }
}

orc_state* orc_create(const orc_cfg* cf) {
  orc_state* s = (orc_state*)calloc(1, sizeof(orc_state));
  if (!s) return NULL;
  s->c = *cf;
  int64_t np = cf->np, nc = ncell(cf);
  s->xi = (double*)calloc((size_t)(6 * np + 1), sizeof(double));
  s->x = (double*)calloc((size_t)(3 * np + 1), sizeof(double));
  s->v = (double*)calloc((size_t)(3 * np + 1), sizeof(double));
  s->rho = (double*)calloc((size_t)nc, sizeof(double));
  s->phi = (double*)calloc((size_t)nc, sizeof(double));
  s->E = (double*)calloc((size_t)(3 * nc), sizeof(double));
  s->cell = (int32_t*)calloc((size_t)(np + 1), sizeof(int32_t));
  s->count = (int32_t*)calloc((size_t)nc, sizeof(int32_t));
  s->start = (int32_t*)calloc((size_t)(nc + 1), sizeof(int32_t));
  s->perm = (int32_t*)calloc((size_t)(np + 1), sizeof(int32_t));
  if (!s->xi || !s->x || !s->v || !s->rho || !s->phi || !s->E || !s->cell ||
      !s->count || !s->start || !s->perm)
    return NULL;
  for (int64_t p = 0; p < np; p++) orc_sample_xi(cf, p, s->xi + 6 * p);
  return s;
}

void orc_destroy(orc_state* s) {
  if (!s) return;
  free(s->xi); free(s->x); free(s->v); free(s->rho); free(s->phi); free(s->E);
  free(s->cell); free(s->count); free(s->start); free(s->perm);
  free(s->ang);
  free(s->plog);
  free(s);
}

static double time_at(const orc_state* s, double steps) {
  return s->t0 + steps * s->c.dt;
}

/* ------------------------------------------------------------------------
 * Cells and the (cell, pid) order. Cell i_d = floor(x_d n), clamped to
 * [0, n-1]; linear index x-fastest. A stable counting sort of the pids in
 * increasing order gives ascending pid inside each cell.
 * ---------------------------------------------------------------------- */
int32_t orc_cell_of(const orc_cfg* cf, const double x[3]) {
  int64_t n = cf->n, i[3];
  for (int d = 0; d < 3; d++) {
    double f = floor(x[d] * (double)n);
    int64_t k = (int64_t)f;
    if (k < 0) k = 0;
    if (k > n - 1) k = n - 1;
    i[d] = k;
  }
  return (int32_t)(i[0] + n * (i[1] + n * i[2]));
}

void orc_sort(orc_state* s) {
  const orc_cfg* cf = &s->c;
  int64_t np = cf->np, nc = ncell(cf);
  for (int64_t k = 0; k < nc; k++) s->count[k] = 0;
  for (int64_t p = 0; p < np; p++) {
    s->cell[p] = orc_cell_of(cf, s->x + 3 * p);
    s->count[s->cell[p]]++;
  }
  s->start[0] = 0;
  for (int64_t k = 0; k < nc; k++) s->start[k + 1] = s->start[k] + s->count[k];
  int32_t* fill = (int32_t*)calloc((size_t)nc, sizeof(int32_t));
  for (int64_t p = 0; p < np; p++) {
    int32_t k = s->cell[p];
    s->perm[s->start[k] + fill[k]] = (int32_t)p;
    fill[k]++;
  }
  free(fill);
}

/* ------------------------------------------------------------------------
 * Cloud-in-cell deposit (Sec. 2): rho_node = (q w / h^3) sum_p S(x_p - X),
 * S the product of 1D hats 1 - |x - X|/h over the 8 nodes around x_p.
 * ---------------------------------------------------------------------- */
static int64_t node_index(int64_t n, int64_t i, int64_t j, int64_t k) {
  i = ((i % n) + n) % n;
  j = ((j % n) + n) % n;
  k = ((k % n) + n) % n;
  return i + n * (j + n * k);
}

/* hat weights of the two nodes below/above x along one axis              */
static void hat_weights(double xd, int64_t n, int64_t* i0, double w[2]) {
  double u = xd * (double)n; /* position in units of h */
  int64_t i = (int64_t)floor(u);
  if (i < 0) i = 0;
  if (i > n - 1) i = n - 1;
  *i0 = i;
  w[0] = 1.0 - fabs(u - (double)i);
  w[1] = 1.0 - fabs(u - (double)(i + 1));
}

void orc_deposit(orc_state* s) {
  const orc_cfg* cf = &s->c;
  int64_t n = cf->n, nc = ncell(cf);
  double h = 1.0 / (double)n;
  double q = cf->couple_q_zero ? 0.0 : cf->q;
  double w = cf->nphys / (double)cf->np;
  double scale = q * w / (h * h * h);
  for (int64_t k = 0; k < nc; k++) s->rho[k] = 0.0;
  for (int64_t p = 0; p < cf->np; p++) {
    int64_t i0[3];
    double wt[3][2];
    for (int d = 0; d < 3; d++) hat_weights(s->x[3 * p + d], n, &i0[d], wt[d]);
    for (int c = 0; c < 2; c++)
      for (int b = 0; b < 2; b++)
        for (int a = 0; a < 2; a++)
          s->rho[node_index(n, i0[0] + a, i0[1] + b, i0[2] + c)] +=
              scale * wt[0][a] * wt[1][b] * wt[2][c];
  }
}

/* Field gather with the same hats (Sec. 2, "interpolated onto the particles"). */
void orc_gather(const orc_cfg* cf, const double* E, const double x[3], double Ep[3]) {
  int64_t n = cf->n, i0[3];
  double wt[3][2];
  for (int d = 0; d < 3; d++) hat_weights(x[d], n, &i0[d], wt[d]);
  Ep[0] = Ep[1] = Ep[2] = 0.0;
  for (int c = 0; c < 2; c++)
    for (int b = 0; b < 2; b++)
      for (int a = 0; a < 2; a++) {
        int64_t node = node_index(n, i0[0] + a, i0[1] + b, i0[2] + c);
        double ww = wt[0][a] * wt[1][b] * wt[2][c];
        for (int d = 0; d < 3; d++) Ep[d] += ww * E[3 * node + d];
      }
}

/* ------------------------------------------------------------------------
 * Poisson with the manufactured source (Eq. poisson_mms), periodic:
 *   -Lap_h phi = b,  b = rho/eps0 - Lap phi^M - rho^M/eps0, minus its mean,
 * Lap_h the 7-point Laplacian at nodes; zero-mean phi (Sec. 2).
 * ---------------------------------------------------------------------- */
void orc_rhs(const orc_state* s, double t, double* b) {
  const orc_cfg* cf = &s->c;
  int64_t n = cf->n, nc = ncell(cf);
  double h = 1.0 / (double)n;
  double q = cf->couple_q_zero ? 0.0 : cf->q;
  double mean = 0.0;
  for (int64_t k = 0; k < n; k++)
    for (int64_t j = 0; j < n; j++)
      for (int64_t i = 0; i < n; i++) {
        int64_t id = i + n * (j + n * k);
        double X[3] = {(double)i * h, (double)j * h, (double)k * h};
        b[id] = s->rho[id] / cf->eps0 - orc_lap_phiM(cf, X, t) -
                orc_rhoM(cf, q, X, t) / cf->eps0;
        mean += b[id];
      }
  mean /= (double)nc;
  for (int64_t id = 0; id < nc; id++) b[id] -= mean;
}

/* y = -Lap_h x with periodic wrap                                        */
void orc_neg_lap(int64_t n, const double* xv, double* y) {
  double inv_h2 = (double)n * (double)n;
  for (int64_t k = 0; k < n; k++)
    for (int64_t j = 0; j < n; j++)
      for (int64_t i = 0; i < n; i++) {
        double sum = xv[node_index(n, i + 1, j, k)] + xv[node_index(n, i - 1, j, k)] +
                     xv[node_index(n, i, j + 1, k)] + xv[node_index(n, i, j - 1, k)] +
                     xv[node_index(n, i, j, k + 1)] + xv[node_index(n, i, j, k - 1)];
        y[i + n * (j + n * k)] = (6.0 * xv[i + n * (j + n * k)] - sum) * inv_h2;
      }
}

static double dot(int64_t m, const double* a, const double* b) {
  double s = 0.0;
  for (int64_t i = 0; i < m; i++) s += a[i] * b[i];
  return s;
}

/* Textbook conjugate gradients (Hestenes-Stiefel) from the warm start in
 * phi, stopping at ||r|| <= tol ||b||; the result is projected to zero mean.
 * Returns the iteration count, or -1 if maxit was reached.               */
int64_t orc_cg(int64_t n, const double* b, double* phi, double tol, int64_t maxit,
               double* res_out) {
  int64_t m = n * n * n;
  double* r = (double*)malloc((size_t)m * sizeof(double));
  double* p = (double*)malloc((size_t)m * sizeof(double));
  double* Ap = (double*)malloc((size_t)m * sizeof(double));
  orc_neg_lap(n, phi, Ap);
  for (int64_t i = 0; i < m; i++) r[i] = b[i] - Ap[i];
  for (int64_t i = 0; i < m; i++) p[i] = r[i];
  double bb = dot(m, b, b), rr = dot(m, r, r);
  int64_t it = 0, status = 0;
  if (bb == 0.0) {
    for (int64_t i = 0; i < m; i++) phi[i] = 0.0;
    rr = 0.0;
  } else {
    while (!(sqrt(rr) <= tol * sqrt(bb))) {
      if (it >= maxit) { status = -1; break; }
      orc_neg_lap(n, p, Ap);
      double alpha = rr / dot(m, p, Ap);
      for (int64_t i = 0; i < m; i++) phi[i] += alpha * p[i];
      for (int64_t i = 0; i < m; i++) r[i] -= alpha * Ap[i];
      double rr_new = dot(m, r, r);
      it++;
      if (sqrt(rr_new) <= tol * sqrt(bb)) { rr = rr_new; break; }
      double beta = rr_new / rr;
      for (int64_t i = 0; i < m; i++) p[i] = r[i] + beta * p[i];
      rr = rr_new;
    }
  }
  double mean = 0.0;
  for (int64_t i = 0; i < m; i++) mean += phi[i];
  mean /= (double)m;
  for (int64_t i = 0; i < m; i++) phi[i] -= mean;
  if (res_out) *res_out = bb > 0.0 ? sqrt(rr) / sqrt(bb) : 0.0;
  free(r); free(p); free(Ap);
  return status < 0 ? -1 : it;
}

/* E = -grad phi by second-order central differences at nodes (Sec. 4.1). */
void orc_efield(int64_t n, const double* phi, double* E) {
  double h = 1.0 / (double)n;
  for (int64_t k = 0; k < n; k++)
    for (int64_t j = 0; j < n; j++)
      for (int64_t i = 0; i < n; i++) {
        int64_t id = i + n * (j + n * k);
        E[3 * id + 0] = -(phi[node_index(n, i + 1, j, k)] - phi[node_index(n, i - 1, j, k)]) / (2.0 * h);
        E[3 * id + 1] = -(phi[node_index(n, i, j + 1, k)] - phi[node_index(n, i, j - 1, k)]) / (2.0 * h);
        E[3 * id + 2] = -(phi[node_index(n, i, j, k + 1)] - phi[node_index(n, i, j, k - 1)]) / (2.0 * h);
      }
}

int64_t orc_field(orc_state* s, double t) {
  const orc_cfg* cf = &s->c;
  int64_t nc = ncell(cf);
  double* b = (double*)malloc((size_t)nc * sizeof(double));
  orc_deposit(s);
  orc_rhs(s, t, b);
  double res = 0.0;
  int64_t it = orc_cg(cf->n, b, s->phi, cf->cg_tol, cf->cg_maxit, &res);
  s->cg_iters = it;
  s->cg_res = res;
  orc_efield(cf->n, s->phi, s->E);
  free(b);
  return it;
}

/* ------------------------------------------------------------------------
 * Algorithm 1 (no-time-counter, binary elastic, same species and weight),
 * run K times from the same pre-collision velocities and averaged
 * (Eq. avg_outcome). Draws for call counter c0 = 2 step + phase, cell k,
 * outcome o:
 *   N_pairs : Philox(c0, k, 0, o<<8 | 1), word 0   -> U32
 *   pair s  : Philox(c0, k, s, o<<8 | 0)  = (p, q, accept, epsilon)
 *             Philox(c0, k, (s+1)/4, o<<8 | 1), word (s+1) mod 4 = chi
 * (the o<<8 | 1 stream's words in order: the N_pairs uniform, then one chi
 * per candidate)
 * p = floor(U c) over the c particles; q = floor(U (c-1)) over the other
 * c - 1, counted past p (q' >= p gives q' + 1). That is the distribution of
 * Algorithm 1's second draw repeated until it differs from the first:
 * uniform over the particles other than p.
 * ---------------------------------------------------------------------- */
typedef struct {
  double* a;  /* [n][2] (chi, eps) */
  int64_t n, cap;
} orc_angles;

/* Pair list of Algorithm 1: one record of 8 int32 per N_pairs draw and
 * per candidate pair, in the order the oracle draws them:
 *   (c0, cell, outcome, slot, p, q, result, kind)
 * slot = -1, p = q = -1, result = N_pairs, kind = 4 for the N_pairs draw;
 * slot = s, the in-cell indices p, q, result = 1 accepted / 0 rejected,
 * kind = 1 where |U - sigma g/(sigma g)_max| < 1e-12 (a near tie), else 0,
 * for candidate s.                                                        */
typedef struct {
  int32_t* r;
  int64_t n, cap;
} orc_pairlog;

typedef struct {
  int64_t n_cand, n_coll, n_gmax, n_tie;
  orc_angles* rec;  /* NULL: angles not recorded */
  orc_pairlog* log; /* NULL: pair list not recorded */
} orc_dsmc_stats;

static void log_pair(orc_pairlog* lg, uint32_t c0, uint32_t cell, uint32_t o, int64_t slot, int64_t p,
                     int64_t q, int64_t result, int32_t kind) {
  if (!lg) return;
  if (lg->n == lg->cap) {
    int64_t cap = lg->cap ? 2 * lg->cap : 1024;
    int32_t* r = (int32_t*)realloc(lg->r, (size_t)(8 * cap) * sizeof(int32_t));
    if (!r) return;
    lg->r = r;
    lg->cap = cap;
  }
  int32_t* e = lg->r + 8 * lg->n;
  e[0] = (int32_t)c0; e[1] = (int32_t)cell; e[2] = (int32_t)o; e[3] = (int32_t)slot;
  e[4] = (int32_t)p; e[5] = (int32_t)q; e[6] = (int32_t)result; e[7] = kind;
  lg->n++;
}

/* Manufactured anisotropy (Sec. 5.1): with u = sin^2(chi/2) the CDF of chi
 * is F(u) = (13 u + 96 u^2 - 160 u^3 + 80 u^4)/29, increasing on [0, 1]
 * (p_chi > 0). chi = F^{-1}(xi) by bisection on u to the last bit; the
 * isotropic kernel is F(u) = u.                                            */
double orc_aniso_F(double u) {
  return (13.0 * u + 96.0 * u * u - 160.0 * u * u * u + 80.0 * u * u * u * u) / 29.0;
}

double orc_aniso_u(double xi) {
  double lo = 0.0, hi = 1.0;
  for (int it = 0; it < 200; it++) {
    double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    if (orc_aniso_F(mid) < xi) lo = mid;
    else hi = mid;
  }
  return 0.5 * (lo + hi);
}

/* Sec. 4.4, Eq. angle_recovery: chi = acos(g'_z / g) with the PRE-collision
 * relative speed g, eps = atan2(g'_y, g'_x) taken into [0, 2 pi).          */
static void record_angles(orc_angles* r, double g, const double gp[3]) {
  if (r->n == r->cap) {
    r->cap = r->cap ? 2 * r->cap : 1024;
    r->a = (double*)realloc(r->a, (size_t)(2 * r->cap) * sizeof(double));
  }
  double cz = gp[2] / g;
  if (cz > 1.0) cz = 1.0;
  if (cz < -1.0) cz = -1.0;
  double eps = atan2(gp[1], gp[0]);
  if (eps < 0.0) eps += 2.0 * ORC_PI;
  r->a[2 * r->n] = acos(cz);
  r->a[2 * r->n + 1] = eps;
  r->n++;
}

/* P_coll,max = (sigma g)_max w dt / dV (Algorithm 1; Eq. p_coll at g where
 * sigma g peaks). For hard spheres (sigma g)_max = sigma0 g_max.          */
double orc_pmax(const orc_cfg* cf) {
  double h = 1.0 / (double)cf->n;
  double dV = h * h * h;
  double w = cf->nphys / (double)cf->np;
  double sg_max = orc_sg_max(cf);
  return sg_max * w * cf->dt / dV;
}

static void ntc_one_outcome(const orc_cfg* cf, uint32_t c0, uint32_t cellk, uint32_t o,
                            int64_t c, double* vloc /* [c][3], updated in place */,
                            orc_dsmc_stats* st) {
  double sg_max = orc_sg_max(cf);                     /* (sigma g)_max              */
  double Pmax = orc_pmax(cf);
  uint32_t u[4];
  philox4(c0, cellk, 0u, (o << 8) | 1u, cf->seed, u);
  double npairs_real = ((double)(c * (c - 1)) * Pmax) * 0.5 + orc_u32(u[0]);
  int64_t npairs = (int64_t)floor(npairs_real);       /* Algorithm 1: NTC pair count */
  log_pair(st->log, c0, cellk, o, -1, -1, -1, npairs, 4);
  for (int64_t sl = 0; sl < npairs; sl++) {
    uint32_t b0[4], bchi[4];
    philox4(c0, cellk, (uint32_t)sl, (o << 8) | 0u, cf->seed, b0);
    philox4(c0, cellk, (uint32_t)((sl + 1) / 4), (o << 8) | 1u, cf->seed, bchi);
    uint32_t p = orc_index(b0[0], (uint32_t)c);
    uint32_t q = orc_index(b0[1], (uint32_t)(c - 1)); /* one of the others */
    if (q >= p) q++;
    uint32_t wchi = bchi[(sl + 1) % 4];
    st->n_cand++;
    double* vp = vloc + 3 * p;
    double* vq = vloc + 3 * q;
    double dx = vp[0] - vq[0], dy = vp[1] - vq[1], dz = vp[2] - vq[2];
    double g2 = dx * dx + dy * dy + dz * dz;
    double g = sqrt(g2);
    /* sigma(g) g / (sigma g)_max                                         */
    double ratio = cf->n_sigma == 0 ? (cf->sigma0 * g) / sg_max : orc_sigma_g(cf, g2) / sg_max;
    double U = orc_u32(b0[2]);
    if (g > cf->gmax) st->n_gmax++;
    if (fabs(U - ratio) < 1e-12) st->n_tie++;
    log_pair(st->log, c0, cellk, o, sl, p, q, U < ratio, fabs(U - ratio) < 1e-12 ? 1 : 0);
    if (U < ratio) {
      if (cf->verify & ORC_ERROR2) {
        /* injected Error 2 (Sec. 5.4): swap with probability beta = 1/2,
         * the coin being the candidate's chi word                        */
        if (orc_u32(wchi) < 0.5) {
          for (int d = 0; d < 3; d++) {
            double tmp = vp[d];
            vp[d] = vq[d];
            vq[d] = tmp;
          }
        }
      } else {
        double eps = 2.0 * ORC_PI * orc_u32(b0[3]);     /* epsilon = 2 pi U        */
        /* chi = F^{-1}(U) (Eq. chi): cos chi = 1 - 2U isotropic, 1 - 2u(U) anisotropic */
        double uchi = (cf->verify & ORC_ANISO) ? orc_aniso_u(orc_u32(wchi)) : orc_u32(wchi);
        double cchi = 1.0 - 2.0 * uchi;
        double schi = sqrt(1.0 - cchi * cchi);
        double n[3] = {cos(eps) * schi, sin(eps) * schi, cchi}; /* Eq. n (lab frame) */
        double gp[3], vcm[3];
        for (int d = 0; d < 3; d++) {
          gp[d] = g * n[d];
          /* Eq. v_cm; injected Error 1 flips the sign of v_q             */
          vcm[d] = (cf->verify & ORC_ERROR1) ? (vp[d] - vq[d]) / 2.0 : (vp[d] + vq[d]) / 2.0;
        }
        for (int d = 0; d < 3; d++) {
          vp[d] = vcm[d] + gp[d] / 2.0;
          vq[d] = vcm[d] - gp[d] / 2.0;
        }
      }
      if (st->rec) {
        double gpost[3] = {vp[0] - vq[0], vp[1] - vq[1], vp[2] - vq[2]};
        record_angles(st->rec, g, gpost);
      }
      st->n_coll++;
    }
  }
}

/* <Delta v_p>_coll for every particle (pid-indexed dv[np][3]) from the
 * cells in s->perm/start/count and the velocities v.                     */
void orc_dsmc_avg(orc_state* s, const double* v, uint32_t c0, double* dv) {
  const orc_cfg* cf = &s->c;
  int64_t nc = ncell(cf);
  orc_angles rec = {s->ang, s->n_ang, s->cap_ang};
  orc_pairlog lg = {s->plog, s->n_plog, s->cap_plog};
  orc_dsmc_stats st = {0, 0, 0, 0, (cf->verify & ORC_ANGLES) ? &rec : NULL, s->plog_on ? &lg : NULL};
  for (int64_t p = 0; p < 3 * cf->np; p++) dv[p] = 0.0;
  if (cf->K <= 0) return;
  /* Cells are independent (each writes only its own particles' dv), so
   * threads may take different cells; the recorded angles and the pair
   * log keep the serial cell order, so they run on one thread. The counters
   * are integers: their sum does not depend on the order.                 */
  int serial = st.rec != NULL || st.log != NULL;
  (void)serial;
#pragma omp parallel if (!serial)
  {
  orc_dsmc_stats lst = {0, 0, 0, 0, st.rec, st.log};
  double* v0 = NULL;
  double* vloc = NULL;
  double* acc = NULL;
  int64_t cap = 0;
#pragma omp for schedule(dynamic, 16)
  for (int64_t k = 0; k < nc; k++) {
    int64_t c = s->count[k];
    if (c < 2) continue;
    if (c > cap) {
      cap = c;
      v0 = (double*)realloc(v0, (size_t)(3 * c) * sizeof(double));
      vloc = (double*)realloc(vloc, (size_t)(3 * c) * sizeof(double));
      acc = (double*)realloc(acc, (size_t)(3 * c) * sizeof(double));
    }
    for (int64_t j = 0; j < c; j++) {
      int32_t pid = s->perm[s->start[k] + j];
      for (int d = 0; d < 3; d++) {
        v0[3 * j + d] = v[3 * pid + d];
        acc[3 * j + d] = 0.0;
      }
    }
    for (int64_t o = 0; o < cf->K; o++) {
      memcpy(vloc, v0, (size_t)(3 * c) * sizeof(double));
      ntc_one_outcome(cf, c0, (uint32_t)k, (uint32_t)o, c, vloc, &lst);
      for (int64_t j = 0; j < 3 * c; j++) acc[j] += vloc[j] - v0[j];
    }
    for (int64_t j = 0; j < c; j++) {
      int32_t pid = s->perm[s->start[k] + j];
      for (int d = 0; d < 3; d++) dv[3 * pid + d] = acc[3 * j + d] / (double)cf->K;
    }
  }
  free(v0); free(vloc); free(acc);
#pragma omp critical
  {
    st.n_cand += lst.n_cand;
    st.n_coll += lst.n_coll;
    st.n_gmax += lst.n_gmax;
    st.n_tie += lst.n_tie;
  }
  }
  s->plog = lg.r;
  s->n_plog = lg.n;
  s->cap_plog = lg.cap;
  s->ang = rec.a;
  s->n_ang = rec.n;
  s->cap_ang = rec.cap;
  s->n_cand += st.n_cand;
  s->n_coll += st.n_coll;
  s->n_gmax += st.n_gmax;
  s->n_tie += st.n_tie;
}

/* Analytic source for every particle, using its cell's count and f_v at
 * the call's time t.                                                     */
void orc_source_all(orc_state* s, const double* v, double t, double* dvM) {
  const orc_cfg* cf = &s->c;
#pragma omp parallel for schedule(static)
  for (int64_t p = 0; p < cf->np; p++) {
    if (cf->K <= 0) {
      dvM[3 * p] = dvM[3 * p + 1] = dvM[3 * p + 2] = 0.0;
      continue;
    }
    if (cf->n_sigma == 0)
      orc_hs_source(cf, v + 3 * p, s->count[s->cell[p]], dvM + 3 * p);
    else
      orc_odd_source(cf, v + 3 * p, s->count[s->cell[p]], t, dvM + 3 * p);
  }
}

/* ------------------------------------------------------------------------
 * Initialisation and the velocity-Verlet step (Eq. velocity_verlet).
 * ---------------------------------------------------------------------- */
void orc_sample(orc_state* s, double t0) {
  const orc_cfg* cf = &s->c;
  s->t0 = t0;
  s->step = 0;
  s->n_ang = 0;
#pragma omp parallel for schedule(static)
  for (int64_t p = 0; p < cf->np; p++) {
    for (int d = 0; d < 3; d++) {
      s->x[3 * p + d] = orc_xM_d(cf, d, s->xi[6 * p + d], t0);
      s->v[3 * p + d] = orc_vM_t(cf, d, s->xi[6 * p + 3 + d], t0);
    }
  }
  for (int64_t i = 0; i < ncell(cf); i++) s->phi[i] = 0.0;
  orc_sort(s);
  orc_field(s, t0);
}

void orc_set_state(orc_state* s, const double* x, const double* v, double t0, int64_t step) {
  const orc_cfg* cf = &s->c;
  s->t0 = t0;
  s->step = step;
  memcpy(s->x, x, (size_t)(3 * cf->np) * sizeof(double));
  memcpy(s->v, v, (size_t)(3 * cf->np) * sizeof(double));
  orc_sort(s);
  orc_field(s, time_at(s, (double)step));
}

double orc_wrap(double x) {
  double y = x - floor(x);
  if (y >= 1.0) y = 0.0;
  return y;
}

/* the Lorentz term dt q/m (E_p - E_p^M) for every particle at time t     */
static void lorentz_term(orc_state* s, double t, double* out) {
  const orc_cfg* cf = &s->c;
  double qm = cf->couple_qm_zero ? 0.0 : cf->qm;
#pragma omp parallel for schedule(static)
  for (int64_t p = 0; p < cf->np; p++) {
    double Ep[3], EMp[3];
    orc_gather(cf, s->E, s->x + 3 * p, Ep);
    orc_EM(cf, s->x + 3 * p, t, EMp);
    for (int d = 0; d < 3; d++) out[3 * p + d] = cf->dt * qm * (Ep[d] + cf->E_app[d] - EMp[d]);
  }
}

void orc_step(orc_state* s, int64_t nsteps) {
  const orc_cfg* cf = &s->c;
  int64_t np = cf->np;
  double* L = (double*)malloc((size_t)(3 * np + 1) * sizeof(double));
  double* dv = (double*)malloc((size_t)(3 * np + 1) * sizeof(double));
  double* dvM = (double*)malloc((size_t)(3 * np + 1) * sizeof(double));
  double* vh = (double*)malloc((size_t)(3 * np + 1) * sizeof(double));
  for (int64_t it = 0; it < nsteps; it++) {
    int64_t n = s->step;
    double tn = time_at(s, (double)n);
    double th = time_at(s, (double)n + 0.5);
    double tn1 = time_at(s, (double)(n + 1));
    /* v^{n+1/2}: Lorentz term, collision call A at (x^n, v^n)             */
    lorentz_term(s, tn, L);
    orc_dsmc_avg(s, s->v, (uint32_t)(2 * n + 0), dv);
    orc_source_all(s, s->v, tn, dvM);
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < np; p++)
      for (int d = 0; d < 3; d++) {
        int64_t j = 3 * p + d;
        /* vdot^M is zero for the constant Gaussian f_v */
        double vdotM = cf->dist == 0 ? 0.0 : orc_vMdot(cf, d, orc_vM_t(cf, d, s->xi[6 * p + 3 + d], tn), tn);
        vh[j] = s->v[j] + 0.5 * (L[j] + dv[j] - dvM[j] + cf->dt * vdotM);
      }
    /* x^{n+1} = x^n + dt (v + xdot^M - v^M)^{n+1/2}, wrapped; in the
     * isolated-collision mode dt xdot^M(t_{n+1/2}) becomes the exact
     * increment x^M(t_{n+1}) - x^M(t_n) (Sec. 5.4)                       */
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < np; p++) {
      for (int d = 0; d < 3; d++) {
        double vm = orc_vM_t(cf, d, s->xi[6 * p + 3 + d], th);
        if (cf->verify & ORC_ISOLATE) {
          double dxm = orc_xM(cf, s->xi[6 * p + d], tn1) - orc_xM(cf, s->xi[6 * p + d], tn);
          s->x[3 * p + d] = orc_wrap(s->x[3 * p + d] + (cf->dt * (vh[3 * p + d] - vm) + dxm));
        } else {
          double xm = orc_xM_d(cf, d, s->xi[6 * p + d], th);
          double xmd = orc_xMdot_d(cf, d, xm, th);
          s->x[3 * p + d] = orc_wrap(s->x[3 * p + d] + cf->dt * (vh[3 * p + d] + xmd - vm));
        }
      }
    }
    /* field at t^{n+1} from x^{n+1}                                       */
    orc_sort(s);
    orc_field(s, tn1);
    /* v^{n+1}: Lorentz term at x^{n+1}, collision call B at (x^{n+1}, v^{n+1/2}) */
    lorentz_term(s, tn1, L);
    orc_dsmc_avg(s, vh, (uint32_t)(2 * n + 1), dv);
    orc_source_all(s, vh, th, dvM);
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < np; p++)
      for (int d = 0; d < 3; d++) {
        int64_t j = 3 * p + d;
        /* vdot^M is zero for the constant Gaussian f_v */
        double vdotM = cf->dist == 0 ? 0.0 : orc_vMdot(cf, d, orc_vM_t(cf, d, s->xi[6 * p + 3 + d], tn1), tn1);
        s->v[j] = vh[j] + 0.5 * (L[j] + dv[j] - dvM[j] + cf->dt * vdotM);
      }
    s->step = n + 1;
  }
  free(L); free(dv); free(dvM); free(vh);
}

/* One K-averaged collision call on the current state (cells of x, v); the
 * phase selects the counter 2 step + phase; the source uses f_v at the
 * state's time.                                                          */
void orc_collide_avg(orc_state* s, int64_t phase, double* dv, double* dvM) {
  orc_dsmc_avg(s, s->v, (uint32_t)(2 * s->step + phase), dv);
  orc_source_all(s, s->v, time_at(s, (double)s->step), dvM);
}

/* ------------------------------------------------------------------------
 * Error norms at t = t0 + step dt (Sec. 4.3): eps_2 = sqrt(mean e^2) and
 * eps_inf = max |e| for x, y, z (minimum-image), u, v, w, and phi at nodes.
 * out[0..6] = eps_2, out[7..13] = eps_inf.
 * ---------------------------------------------------------------------- */
void orc_errors(const orc_state* s, double out[14]) {
  const orc_cfg* cf = &s->c;
  double t = time_at(s, (double)s->step);
  double s2[7] = {0}, mx[7] = {0};
  for (int64_t p = 0; p < cf->np; p++) {
    for (int d = 0; d < 3; d++) {
      double e = s->x[3 * p + d] - orc_xM_d(cf, d, s->xi[6 * p + d], t);
      e -= floor(e + 0.5);
      s2[d] += e * e;
      if (fabs(e) > mx[d]) mx[d] = fabs(e);
      double ev = s->v[3 * p + d] - orc_vM_t(cf, d, s->xi[6 * p + 3 + d], t);
      s2[3 + d] += ev * ev;
      if (fabs(ev) > mx[3 + d]) mx[3 + d] = fabs(ev);
    }
  }
  int64_t n = cf->n;
  double h = 1.0 / (double)n;
  for (int64_t k = 0; k < n; k++)
    for (int64_t j = 0; j < n; j++)
      for (int64_t i = 0; i < n; i++) {
        double X[3] = {(double)i * h, (double)j * h, (double)k * h};
        double e = s->phi[i + n * (j + n * k)] - orc_phiM(cf, X, t);
        s2[6] += e * e;
        if (fabs(e) > mx[6]) mx[6] = fabs(e);
      }
  for (int a = 0; a < 6; a++) out[a] = sqrt(s2[a] / (double)cf->np);
  out[6] = sqrt(s2[6] / (double)(n * n * n));
  for (int a = 0; a < 7; a++) out[7 + a] = mx[a];
}

/* Objective of the pathwise-gradient study: out[1] = field energy
 * (eps0/2) h^3 sum_nodes |E|^2, out[2] = mean-square velocity error
 * (1/N_p) sum_p |v_p - v_p^M|^2, out[0] = their sum.                      */
void orc_objective(const orc_state* s, double out[3]) {
  const orc_cfg* cf = &s->c;
  double h = 1.0 / (double)cf->n, ef = 0.0, ev = 0.0;
  double t = time_at(s, (double)s->step);
  for (int64_t i = 0; i < 3 * ncell(cf); i++) ef += s->E[i] * s->E[i];
  for (int64_t p = 0; p < cf->np; p++)
    for (int d = 0; d < 3; d++) {
      double e = s->v[3 * p + d] - orc_vM_t(cf, d, s->xi[6 * p + 3 + d], t);
      ev += e * e;
    }
  out[1] = 0.5 * cf->eps0 * h * h * h * ef;
  out[2] = ev / (double)cf->np;
  out[0] = out[1] + out[2];
}

/* ------------------------------------------------------------------------
 * Accessors for the Python wrapper.
 * ---------------------------------------------------------------------- */
void orc_get_state(const orc_state* s, double* x, double* v) {
  memcpy(x, s->x, (size_t)(3 * s->c.np) * sizeof(double));
  memcpy(v, s->v, (size_t)(3 * s->c.np) * sizeof(double));
}
void orc_get_xi(const orc_state* s, double* xi) {
  memcpy(xi, s->xi, (size_t)(6 * s->c.np) * sizeof(double));
}
void orc_get_field(const orc_state* s, double* rho, double* phi, double* E) {
  int64_t nc = ncell(&s->c);
  if (rho) memcpy(rho, s->rho, (size_t)nc * sizeof(double));
  if (phi) memcpy(phi, s->phi, (size_t)nc * sizeof(double));
  if (E) memcpy(E, s->E, (size_t)(3 * nc) * sizeof(double));
}
void orc_get_sort(const orc_state* s, int32_t* cell, int32_t* count, int32_t* start,
                  int32_t* perm) {
  int64_t nc = ncell(&s->c);
  if (cell) memcpy(cell, s->cell, (size_t)s->c.np * sizeof(int32_t));
  if (count) memcpy(count, s->count, (size_t)nc * sizeof(int32_t));
  if (start) memcpy(start, s->start, (size_t)(nc + 1) * sizeof(int32_t));
  if (perm) memcpy(perm, s->perm, (size_t)s->c.np * sizeof(int32_t));
}
void orc_get_stats(const orc_state* s, int64_t out[6], double* cg_res) {
  out[0] = s->n_cand; out[1] = s->n_coll; out[2] = s->n_gmax; out[3] = s->n_tie;
  out[4] = s->cg_iters; out[5] = s->step;
  if (cg_res) *cg_res = s->cg_res;
}
void orc_reset_stats(orc_state* s) {
  s->n_cand = s->n_coll = s->n_gmax = s->n_tie = 0;
  s->n_ang = 0;
}
void orc_set_phi(orc_state* s, const double* phi) {
  memcpy(s->phi, phi, (size_t)ncell(&s->c) * sizeof(double));
}
/* Single-cell NTC outcome for brute-force tests: velocities [c][3] updated
 * in place, returns the number of collisions.                            */
int64_t orc_ntc_cell(const orc_cfg* cf, uint32_t c0, uint32_t cellk, uint32_t o, int64_t c,
                     double* v) {
  orc_dsmc_stats st = {0, 0, 0, 0, NULL, NULL};
  ntc_one_outcome(cf, c0, cellk, o, c, v, &st);
  return st.n_coll;
}

/* Host threads for the loops over independent cells and particles (1 =
 * serial; without OpenMP the oracle is always serial). Every other loop
 * (the sort, the deposit's scatter, the mesh sums and CG) runs serially,
 * and so does the collision loop while angles or the pair list are
 * recorded: results are the same bits for any thread count. Returns the
 * thread count in effect.                                                 */
int orc_set_threads(int n) {
#ifdef _OPENMP
  if (n >= 1) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

/* Pair-list logging of the collision calls (orc_pairlog records): on != 0
 * starts (and clears) the log, 0 stops it. orc_pair_log copies up to cap
 * records into out[cap][8], returns how many the log holds, and clears it;
 * orc_pair_log_peek does the same without clearing.                       */
void orc_set_pair_log(orc_state* s, int on) {
  s->plog_on = on != 0;
  s->n_plog = 0;
}

int64_t orc_pair_log_peek(const orc_state* s, int32_t* out, int64_t cap) {
  int64_t n = s->n_plog;
  if (out && cap > 0 && n > 0) memcpy(out, s->plog, (size_t)(8 * (n < cap ? n : cap)) * sizeof(int32_t));
  return n;
}

int64_t orc_pair_log(orc_state* s, int32_t* out, int64_t cap) {
  int64_t n = orc_pair_log_peek(s, out, cap);
  s->n_plog = 0;
  return n;
}

/* Recorded (chi, eps) pairs of every collision since sampling or the last
 * orc_reset_stats, in the order the oracle ran them.                      */
int64_t orc_angle_count(const orc_state* s) { return s->n_ang; }

void orc_get_angles(const orc_state* s, double* out) {
  if (s->n_ang) memcpy(out, s->ang, (size_t)(2 * s->n_ang) * sizeof(double));
}
