// Pathwise adjoint of the FP64 step (not in the paper): gradient of
//   J = (eps0/2) h^3 sum_nodes |E|^2 + (1/N_p) sum_p |v_p - v_p^M|^2   at t_N
// with respect to a uniform applied field E_app (added to E_p in the push)
// and the initial velocities, through gather, push, CIC deposit, the
// Poisson solve and the K-averaged collisions with their candidate pairs,
// accept decisions and scattering directions frozen at the sampled values.
//
// One step (Eq. velocity_verlet) in the notation of the reverse sweep:
//   L^n     = dt q/m (E(x^n) + E_app - E^M(x^n))
//   v^{n+h} = v^n + (L^n + C_A(v^n)) / 2                 C = <dv> - <dv^M>
//   x^{n+1} = x^n + dt (v^{n+h} + xdot^M - v^M)           (wrapped)
//   E^{n+1} = -grad_h P (-Lap_h)^+ P (rho(x^{n+1}) / eps0 - ...)
//   v^{n+1} = v^{n+h} + (L^{n+1} + C_B(v^{n+h})) / 2
// L^n enters the closing kick of step n-1 and the opening kick of step n, so
// its adjoint is lam_v^n / 2 + lam_{v^{n+h}} / 2 (the second part is carried).
//
// Checkpoints every few steps hold x, v (pid order), phi and E, so each
// segment is recomputed bit-identically; its per-step states are stored in
// pid order and the segment is swept in reverse. Every sum runs in a fixed
// order: the gradient is deterministic.
#include <math.h>

#include "ntc_fp64.cuh"
#include "pic_internal.cuh"

namespace pic {

struct AdjointBuffers {
  int seg = 0, ncp = 0, max_rec = 0;
  size_t np3 = 0, nc = 0, mu_len = 0, rec_len = 0;
  double *lam_x = nullptr, *lam_v = nullptr, *carry = nullptr, *G = nullptr, *lamL = nullptr;
  double *tx = nullptr, *tv = nullptr, *tvh = nullptr, *tE = nullptr;
  double* ck = nullptr;
  double *corner24 = nullptr, *lamE = nullptr, *badj = nullptr, *mu = nullptr, *Etmp = nullptr, *seedE = nullptr;
  double *part = nullptr, *acc = nullptr;
  double *mu_ov = nullptr, *rec = nullptr;
};

namespace {

constexpr int kT = 256;
constexpr int kAdjMaxRec = 64;  // accepted pairs one outcome may record
inline int nblk(int64_t n) { return (int)((n + kT - 1) / kT < 1 ? 1 : (n + kT - 1) / kT); }

template <class F>
void each_buffer(AdjointBuffers& B, F f) {
  const size_t np3 = B.np3, nc = B.nc;
  f(&B.lam_x, np3); f(&B.lam_v, np3); f(&B.carry, np3); f(&B.G, np3); f(&B.lamL, np3);
  f(&B.tx, (size_t)(B.seg + 1) * np3); f(&B.tv, (size_t)B.seg * np3); f(&B.tvh, (size_t)B.seg * np3);
  f(&B.tE, (size_t)B.seg * 3 * nc);
  f(&B.ck, (size_t)B.ncp * (2 * np3 + 4 * nc));
  f(&B.corner24, 24 * nc); f(&B.lamE, 3 * nc); f(&B.badj, nc); f(&B.mu, nc); f(&B.Etmp, 3 * nc);
  f(&B.seedE, 3 * nc);
  f(&B.part, (size_t)3 * (nblk((int64_t)(np3 > nc ? np3 : nc)) + 8));
  f(&B.acc, 16);
  f(&B.mu_ov, B.mu_len);
  f(&B.rec, B.rec_len);
}

// fixed-shape block sum; the result is valid in thread 0
__device__ double block_sum_d(double v, double* sh) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += sh[i];
  __syncthreads();
  return t;
}

__device__ __forceinline__ void vM_of(const Params& P, uint64_t p, double* vm) {
  const U4 b1 = sample_block(P, p, 1), b2 = sample_block(P, p, 2);
  vm[0] = P.vmean[0] + P.vsig * normcdfinv(unif52(b1.z, b1.w));
  vm[1] = P.vmean[1] + P.vsig * normcdfinv(unif52(b2.x, b2.y));
  vm[2] = P.vmean[2] + P.vsig * normcdfinv(unif52(b2.z, b2.w));
}

// sorted buffers -> pid-ordered AoS
__global__ void __launch_bounds__(kT) k_adj_store(int64_t np, const double* x0, const double* x1, const double* x2,
                                                   const double* v0, const double* v1, const double* v2,
                                                   const uint32_t* pid, double* X, double* V) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= np) return;
  const int64_t p = pid[j];
  if (X) { X[3 * p] = x0[j]; X[3 * p + 1] = x1[j]; X[3 * p + 2] = x2[j]; }
  if (V) { V[3 * p] = v0[j]; V[3 * p + 1] = v1[j]; V[3 * p + 2] = v2[j]; }
}

// pid-ordered AoS -> the current buffers (slot = pid), with v^M of each pid
__global__ void __launch_bounds__(kT) k_adj_load(Params P, const double* X, const double* V, double* x0, double* x1,
                                                  double* x2, double* v0, double* v1, double* v2, double* m0,
                                                  double* m1, double* m2, uint32_t* pid) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P.np) return;
  double vm[3];
  vM_of(P, (uint64_t)i, vm);
  m0[i] = vm[0]; m1[i] = vm[1]; m2[i] = vm[2];
  x0[i] = X[3 * i]; x1[i] = X[3 * i + 1]; x2[i] = X[3 * i + 2];
  v0[i] = V[3 * i]; v1[i] = V[3 * i + 1]; v2[i] = V[3 * i + 2];
  pid[i] = (uint32_t)i;
}

// lam_v = (2/N_p)(v - v^M), lam_x = carry = 0; block partials of |v - v^M|^2
__global__ void __launch_bounds__(kT) k_adj_seed(Params P, const double* V, double* lam_v, double* lam_x,
                                                  double* carry, double* part) {
  __shared__ double sh[32];
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double e2 = 0.0;
  if (i < P.np) {
    double vm[3];
    vM_of(P, (uint64_t)i, vm);
    for (int d = 0; d < 3; ++d) {
      const double e = V[3 * i + d] - vm[d];
      e2 += e * e;
      if (lam_v) {
        lam_v[3 * i + d] = 2.0 / (double)P.np * e;
        lam_x[3 * i + d] = 0.0;
        carry[3 * i + d] = 0.0;
      }
    }
  }
  const double t = block_sum_d(e2, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

__global__ void __launch_bounds__(kT) k_adj_energy(int64_t m, const double* E0, const double* E1, const double* E2,
                                                    double* part) {
  __shared__ double sh[32];
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double e = 0.0;
  if (i < m) e = E0[i] * E0[i] + E1[i] * E1[i] + E2[i] * E2[i];
  const double t = block_sum_d(e, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// out[k] (+)= scale * sum_b part[b * ncomp + k], one block, fixed order
__global__ void __launch_bounds__(kT) k_adj_final(const double* part, int nb, int ncomp, double* out, double scale,
                                                   int accumulate) {
  __shared__ double sh[32];
  for (int k = 0; k < ncomp; ++k) {
    double s = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) s += part[(size_t)b * ncomp + k];
    const double t = block_sum_d(s, sh);
    if (threadIdx.x == 0) out[k] = (accumulate ? out[k] : 0.0) + scale * t;
  }
}

// trilinear weights of x in its cell and their derivatives (cell units n)
struct Tri {
  int ii[2], jj[2], kk[2];
  double w[3][2];   // w[axis][0] = 1 - f, w[axis][1] = f
};
__device__ __forceinline__ Tri tri(const Params& P, double x, double y, double z) {
  const int n = P.n;
  Tri t;
  const double X[3] = {x, y, z};
  int c[3];
  for (int d = 0; d < 3; ++d) {
    c[d] = cell_coord(X[d], n);
    const double f = X[d] * (double)n - (double)c[d];
    t.w[d][0] = 1.0 - f;
    t.w[d][1] = f;
  }
  t.ii[0] = c[0]; t.ii[1] = c[0] + 1 == n ? 0 : c[0] + 1;
  t.jj[0] = c[1]; t.jj[1] = c[1] + 1 == n ? 0 : c[1] + 1;
  t.kk[0] = c[2]; t.kk[1] = c[2] + 1 == n ? 0 : c[2] + 1;
  return t;
}

// gradient of the trilinear interpolation of a nodal field f at the point
__device__ __forceinline__ void interp_grad(const Params& P, const Tri& t, const double* f, double* g) {
  const int n = P.n;
  const double dn = (double)n;
  g[0] = g[1] = g[2] = 0.0;
#pragma unroll
  for (int c = 0; c < 2; ++c)
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
      for (int a = 0; a < 2; ++a) {
        const double v = f[t.ii[a] + (int64_t)n * (t.jj[b] + (int64_t)n * t.kk[c])];
        const double sa = a ? dn : -dn, sb = b ? dn : -dn, sc = c ? dn : -dn;
        g[0] += sa * t.w[1][b] * t.w[2][c] * v;
        g[1] += t.w[0][a] * sb * t.w[2][c] * v;
        g[2] += t.w[0][a] * t.w[1][b] * sc * v;
      }
}

// closing kick of step n, reversed at t_{n+1}: lam_L = lam_v / 2 + carry;
// lam_x += dt q/m (dE/dx - dE^M/dx)^T lam_L; lamL (sorted) = dt q/m lam_L;
// block partials of dt q/m lam_L for dJ/dE_app
struct CloseArgs {
  Params P;
  TimeTerms tt;
  const double *x0, *x1, *x2;
  const uint32_t* pid;
  const double *E0, *E1, *E2;
  const double *lam_v, *carry;
  double *lam_x, *lamL, *part;
  double scale;
};
__global__ void __launch_bounds__(kT) k_adj_close(CloseArgs a) {
  __shared__ double sh[32];
  const Params& P = a.P;
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double lL[3] = {0.0, 0.0, 0.0};
  if (j < P.np) {
    const int64_t p = a.pid[j];
    for (int d = 0; d < 3; ++d) lL[d] = a.scale * (0.5 * a.lam_v[3 * p + d] + a.carry[3 * p + d]);
    const double x = a.x0[j], y = a.x1[j], z = a.x2[j];
    const Tri t = tri(P, x, y, z);
    double gE[3][3];
    interp_grad(P, t, a.E0, gE[0]);
    interp_grad(P, t, a.E1, gE[1]);
    interp_grad(P, t, a.E2, gE[2]);
    double s0, c0, s1, c1, s2, c2;
    sincospi(2.0 * (x - P.phi_shift[0]), &s0, &c0);
    sincospi(2.0 * (y - P.phi_shift[1]), &s1, &c1);
    sincospi(2.0 * (z - P.phi_shift[2]), &s2, &c2);
    const double A = kTwoPi * a.tt.em_amp;
    // dE^M_d / dx_k (symmetric): E^M = -grad phi^M
    const double H[3][3] = {{A * s0 * s1 * s2, -A * c0 * c1 * s2, -A * c0 * s1 * c2},
                            {-A * c0 * c1 * s2, A * s0 * s1 * s2, -A * s0 * c1 * c2},
                            {-A * c0 * s1 * c2, -A * s0 * c1 * c2, A * s0 * s1 * s2}};
    for (int k = 0; k < 3; ++k) {
      double g = 0.0;
      for (int d = 0; d < 3; ++d) g += lL[d] * (gE[d][k] - H[d][k]);
      a.lam_x[3 * p + k] += g;
    }
    for (int d = 0; d < 3; ++d) a.lamL[3 * j + d] = lL[d];
  }
  for (int d = 0; d < 3; ++d) {
    const double t = block_sum_d(lL[d], sh);
    if (threadIdx.x == 0) a.part[3 * blockIdx.x + d] = t;
  }
}

// per cell (sorted slots): corner partials of the CIC weights times lamL,
// 3 components x 8 corners, summed in slot order with a fixed warp tree
__global__ void __launch_bounds__(kT) k_adj_scatter(Params P, const int32_t* start, const double* x0,
                                                     const double* x1, const double* x2, const double* lamL,
                                                     double* corner24) {
  const int lane = threadIdx.x & 31;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t cell = gw; cell < P.ncell; cell += nw) {
    const int32_t s = start[cell], cnt = start[cell + 1] - s;
    double acc[24];
#pragma unroll
    for (int q = 0; q < 24; ++q) acc[q] = 0.0;
    for (int e = lane; e < cnt; e += 32) {
      const int64_t j = s + e;
      const Tri t = tri(P, x0[j], x1[j], x2[j]);
      const double l[3] = {lamL[3 * j], lamL[3 * j + 1], lamL[3 * j + 2]};
#pragma unroll
      for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
          for (int q = 0; q < 2; ++q) {
            const double w = t.w[0][q] * t.w[1][b] * t.w[2][c];
#pragma unroll
            for (int d = 0; d < 3; ++d) acc[8 * d + q + 2 * b + 4 * c] += w * l[d];
          }
    }
#pragma unroll
    for (int q = 0; q < 24; ++q) {
      double v = acc[q];
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
      if (lane == 0) corner24[(int64_t)q * P.ncell + cell] = v;
    }
  }
}

// node sums of the corner partials (+ the objective's eps0 h^3 E at t_N)
__global__ void __launch_bounds__(kT) k_adj_nodes(Params P, const double* corner24, const double* seedE,
                                                   double seed_scale, double* lamE) {
  const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= P.ncell) return;
  const int n = P.n;
  const int i = (int)(id % n), j = (int)((id / n) % n), k = (int)(id / ((int64_t)n * n));
  for (int d = 0; d < 3; ++d) {
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int b = 0; b < 2; ++b)
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const int ii = i - q < 0 ? n - 1 : i - q, jj = j - b < 0 ? n - 1 : j - b, kk = k - c < 0 ? n - 1 : k - c;
          s += corner24[(int64_t)(8 * d + q + 2 * b + 4 * c) * P.ncell + ii + (int64_t)n * (jj + (int64_t)n * kk)];
        }
    if (seedE) s += seed_scale * seedE[(int64_t)d * P.ncell + id];
    lamE[(int64_t)d * P.ncell + id] = s;
  }
}

// adjoint of E = -grad_h phi (central differences): lam_phi(j) =
// sum_d (lam_E_d(j + e_d) - lam_E_d(j - e_d)) / (2h); block partials for the mean
__global__ void __launch_bounds__(kT) k_adj_div(Params P, const double* lamE, double* badj, double* part) {
  __shared__ double sh[32];
  const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double v = 0.0;
  if (id < P.ncell) {
    const int n = P.n;
    const int64_t nn = (int64_t)n * n;
    const int i = (int)(id % n), j = (int)((id / n) % n), k = (int)(id / nn);
    const int64_t xp = i == n - 1 ? id - (n - 1) : id + 1, xm = i == 0 ? id + (n - 1) : id - 1;
    const int64_t yp = j == n - 1 ? id - (int64_t)(n - 1) * n : id + n, ym = j == 0 ? id + (int64_t)(n - 1) * n : id - n;
    const int64_t zp = k == n - 1 ? id - (n - 1) * nn : id + nn, zm = k == 0 ? id + (n - 1) * nn : id - nn;
    const double inv2h = 0.5 * (double)n;
    const double* E0 = lamE;
    const double* E1 = lamE + P.ncell;
    const double* E2 = lamE + 2 * P.ncell;
    v = inv2h * ((E0[xp] - E0[xm]) + (E1[yp] - E1[ym]) + (E2[zp] - E2[zm]));
    badj[id] = v;
  }
  const double t = block_sum_d(v, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// lam_x += (q w / (h^3 eps0)) grad (trilinear interpolation of mu) at x
__global__ void __launch_bounds__(kT) k_adj_depgrad(Params P, const double* x0, const double* x1, const double* x2,
                                                     const uint32_t* pid, const double* mu, double scale,
                                                     double* lam_x) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= P.np) return;
  const int64_t p = pid[j];
  const Tri t = tri(P, x0[j], x1[j], x2[j]);
  double g[3];
  interp_grad(P, t, mu, g);
  for (int d = 0; d < 3; ++d) lam_x[3 * p + d] += scale * g[d];
}

// lam_{v^{n+h}} = lam_v^{n+1} + G_B / 2 + dt lam_x^{n+1}
__global__ void __launch_bounds__(kT) k_adj_vh(int64_t np3, double* lam_v, const double* G, const double* lam_x,
                                                double dt) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= np3) return;
  lam_v[i] = lam_v[i] + 0.5 * G[i] + dt * lam_x[i];
}

// carry = lam_{v^{n+h}} / 2 (the opening kick's share of lam_L^n);
// lam_v^n = lam_{v^{n+h}} + G_A / 2
__global__ void __launch_bounds__(kT) k_adj_open(int64_t np3, double* lam_v, const double* G, double* carry) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= np3) return;
  carry[i] = 0.5 * lam_v[i];
  lam_v[i] = lam_v[i] + 0.5 * G[i];
}

// block partials of scale * carry (dJ/dE_app from L^0)
__global__ void __launch_bounds__(kT) k_adj_sum3(int64_t np, const double* v, double scale, double* part) {
  __shared__ double sh[32];
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (int d = 0; d < 3; ++d) {
    const double t = block_sum_d(i < np ? scale * v[3 * i + d] : 0.0, sh);
    if (threadIdx.x == 0) part[3 * blockIdx.x + d] = t;
  }
}

// ------------------------------------------------------------------------
// Collisions: G = (dC/dv)^T lam for C = <dv> - <dv^M> with frozen pairs.
// Each (cell, outcome) lane replays Algorithm 1 (same draws, same in-place
// updates) recording its accepted pairs, then sweeps them in reverse on a
// private adjoint overlay mu (mu = lam on the particles it touched). For a
// pair with pre-collision v_p, v_q, g = |v_p - v_q|, g^ = (v_p - v_q)/g and
// direction n, the post-collision adjoints mu_p', mu_q' give
//   mu_p = s + d g^,  mu_q = s - d g^,  s = (mu_p' + mu_q')/2,
//   d = n . (mu_p' - mu_q') / 2.
// The K outcomes average in ascending order; the analytic source adds
//   -(d<dv^M>/dv)^T lam = pref (c-1) [s_v R(a) lam + (R'(a)/a)(m.lam) m/s_v]
// with m = mu_v - v, a = |m|/s_v (R'(a)/a by its series below a = 0.3).
// ------------------------------------------------------------------------
struct ListRec {
  double* r;
  int cap, n;
  bool overflow;
  __device__ __forceinline__ void operator()(uint32_t p, uint32_t q, const double* vp, const double* vq,
                                             const double* nv, double g) {
    if (n >= cap) {
      overflow = true;
      return;
    }
    double* e = r + (size_t)n * 12;
    e[0] = (double)p; e[1] = (double)q;
    e[2] = vp[0]; e[3] = vp[1]; e[4] = vp[2];
    e[5] = vq[0]; e[6] = vq[1]; e[7] = vq[2];
    e[8] = nv[0]; e[9] = nv[1]; e[10] = nv[2];
    e[11] = g;
    ++n;
  }
};

__device__ __forceinline__ double hs_Rp_over_a(const Params& P, double a) {
  if (a < 0.3) {
    double acc = 2.0 * (kSeriesTerms - 1) * P.R_series[kSeriesTerms - 1];
    for (int j = kSeriesTerms - 2; j >= 1; --j) acc = fma(acc, a * a, 2.0 * j * P.R_series[j]);
    return acc;
  }
  const double ia = 1.0 / a, ia2 = ia * ia;
  const double sq2pi = 0.79788456080286535588;
  const double rp = sq2pi * exp(-0.5 * a * a) * (ia - 3.0 * ia2 * ia) +
                    (1.0 - 2.0 * ia2 + 3.0 * ia2 * ia2) * erf(a * 0.70710678118654752440);
  return rp * ia;
}

struct DsmcAdjArgs {
  Params P;
  const double *v0, *v1, *v2;
  const uint32_t* pid;
  const int32_t* start;
  uint32_t c0;
  const double* lam;
  double* G;
  double *ov, *mu, *rec;
  int max_ppc, bm_words, Gc, Kc, nchunks, max_rec;
  int64_t ngroups;
  int* flags;
};

constexpr int kAdjDsmcThreads = 128;

__global__ void __launch_bounds__(kAdjDsmcThreads) k_dsmc_adj(DsmcAdjArgs a) {
  extern __shared__ uint32_t smem[];
  const Params& P = a.P;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int wpb = blockDim.x >> 5;
  const int64_t gwarp = (int64_t)blockIdx.x * wpb + wib;
  const int64_t nwarps = (int64_t)gridDim.x * wpb;
  uint32_t* wbm = smem + (size_t)wib * 32 * a.bm_words;
  uint32_t* bm = wbm + (size_t)lane * a.bm_words;
  double* ov = a.ov + ((size_t)gwarp * 32 + lane) * a.max_ppc * 3;
  double* wmu = a.mu + (size_t)gwarp * 32 * a.max_ppc * 3;
  double* mu = wmu + (size_t)lane * a.max_ppc * 3;
  double* rec = a.rec + ((size_t)gwarp * 32 + lane) * a.max_rec * 12;
  for (int i = 0; i < a.bm_words; ++i) bm[i] = 0u;
  __syncwarp();
  LaneCounts cnt = {0, 0, 0, 0};
  for (int64_t grp = gwarp; grp < a.ngroups; grp += nwarps) {
    const int64_t cell0 = grp * a.Gc;
    const int ncl = (int)min((int64_t)a.Gc, P.ncell - cell0);
    const int mycl = lane / a.Kc;
    const bool lane_cell = mycl < ncl;
    int32_t s = 0, c = 0;
    if (lane_cell) {
      s = a.start[cell0 + mycl];
      c = a.start[cell0 + mycl + 1] - s;
    }
    const int32_t gs = a.start[cell0], ge = a.start[cell0 + ncl];
    for (int ch = 0; ch < a.nchunks; ++ch) {
      const int o = ch * a.Kc + lane % a.Kc;
      bool run = lane_cell && o < P.K && c >= 2;
      if (run && c > a.max_ppc) {
        atomicOr(a.flags, 1);
        run = false;
      }
      if (run) {
        ListRec R{rec, a.max_rec, 0, false};
        ntc_outcome<false>(P, a.c0, (uint32_t)(cell0 + mycl), (uint32_t)o, c, a.v0 + s, a.v1 + s, a.v2 + s, bm, ov,
                           cnt, R);
        if (R.overflow) atomicOr(a.flags, 1);
        for (int w = 0; w < (c + 31) / 32; ++w) {
          uint32_t bits = bm[w];
          while (bits) {
            const int i = 32 * w + __ffs(bits) - 1;
            bits &= bits - 1u;
            const double* l = a.lam + 3 * (size_t)a.pid[s + i];
            mu[3 * i] = l[0]; mu[3 * i + 1] = l[1]; mu[3 * i + 2] = l[2];
          }
        }
        for (int r = R.n - 1; r >= 0; --r) {
          const double* e = rec + (size_t)r * 12;
          const int p = (int)e[0], q = (int)e[1];
          const double ig = 1.0 / e[11];
          const double gh[3] = {(e[2] - e[5]) * ig, (e[3] - e[6]) * ig, (e[4] - e[7]) * ig};
          double sg[3], dd = 0.0;
          for (int d = 0; d < 3; ++d) {
            sg[d] = 0.5 * (mu[3 * p + d] + mu[3 * q + d]);
            dd += e[8 + d] * (mu[3 * p + d] - mu[3 * q + d]);
          }
          dd *= 0.5;
          for (int d = 0; d < 3; ++d) {
            mu[3 * p + d] = sg[d] + dd * gh[d];
            mu[3 * q + d] = sg[d] - dd * gh[d];
          }
        }
      }
      __syncwarp();
      const bool last = ch == a.nchunks - 1;
      for (int32_t j = gs + lane; j < ge; j += 32) {
        int cl = 0;
        while (cl + 1 < ncl && a.start[cell0 + cl + 1] <= j) ++cl;
        const int32_t cs = a.start[cell0 + cl];
        const int cc = a.start[cell0 + cl + 1] - cs;
        const int jj = j - cs;
        const size_t pj = a.pid[j];
        const double l0 = a.lam[3 * pj], l1 = a.lam[3 * pj + 1], l2 = a.lam[3 * pj + 2];
        double acc0 = 0.0, acc1 = 0.0, acc2 = 0.0;
        if (ch > 0) { acc0 = a.G[3 * pj]; acc1 = a.G[3 * pj + 1]; acc2 = a.G[3 * pj + 2]; }
        if (cc >= 2 && cc <= a.max_ppc) {
          for (int k = 0; k < a.Kc; ++k) {
            if (ch * a.Kc + k >= P.K) break;
            const int L = cl * a.Kc + k;
            if ((wbm[(size_t)L * a.bm_words + (jj >> 5)] >> (jj & 31)) & 1u) {
              const double* M = wmu + ((size_t)L * a.max_ppc + jj) * 3;
              acc0 += M[0] - l0;
              acc1 += M[1] - l1;
              acc2 += M[2] - l2;
            }
          }
        }
        if (!last) {
          a.G[3 * pj] = acc0; a.G[3 * pj + 1] = acc1; a.G[3 * pj + 2] = acc2;
        } else {
          const double K = (double)P.K;
          const double m[3] = {P.vmean[0] - a.v0[j], P.vmean[1] - a.v1[j], P.vmean[2] - a.v2[j]};
          const double am = sqrt(m[0] * m[0] + m[1] * m[1] + m[2] * m[2]) * P.inv_vsig;
          const double pc = P.src_pref * (double)(cc - 1);
          const double f1 = pc * P.vsig * hs_R(P, am);
          const double f2 = pc * hs_Rp_over_a(P, am) * P.inv_vsig * (m[0] * l0 + m[1] * l1 + m[2] * l2);
          a.G[3 * pj] = acc0 / K + f1 * l0 + f2 * m[0];
          a.G[3 * pj + 1] = acc1 / K + f1 * l1 + f2 * m[1];
          a.G[3 * pj + 2] = acc2 / K + f1 * l2 + f2 * m[2];
        }
      }
      __syncwarp();
      if (run)
        for (int i = 0; i < (c + 31) / 32; ++i) bm[i] = 0u;
      __syncwarp();
    }
  }
}

}  // namespace

void adjoint_free(pic_ctx* c) {
  if (!c->adj) return;
  each_buffer(*c->adj, [&](double** p, size_t) {
    ctx_free(c, *p);
    *p = nullptr;
  });
  delete c->adj;
  c->adj = nullptr;
}

}  // namespace pic

using namespace pic;

namespace {

pic_status cuda_err(cudaError_t e) {
  if (e == cudaSuccess) return PIC_OK;
  cudaGetLastError();
  return e == cudaErrorMemoryAllocation ? PIC_ENOMEM : PIC_ECUDA;
}

#define AK(expr)                                              \
  do {                                                        \
    cudaError_t e_ = (expr);                                  \
    if (e_ != cudaSuccess) return cuda_err(e_);               \
  } while (0)
#define AS(expr)                                              \
  do {                                                        \
    pic_status s_ = (expr);                                   \
    if (s_ != PIC_OK) return s_;                              \
  } while (0)

double tval(const pic_ctx* c, double steps) { return c->t0 + steps * c->cfg.dt; }

pic_status ensure_buffers(pic_ctx* c, int seg, int ncp) {
  AdjointBuffers* B = c->adj;
  const size_t np3 = 3 * (size_t)c->P.np, nc = (size_t)c->P.ncell;
  const size_t lanes = (size_t)c->dsmc_grid * (c->dsmc_block / 32) * 32;
  if (B && B->seg >= seg && B->ncp >= ncp && B->np3 == np3) return PIC_OK;
  adjoint_free(c);
  B = new (std::nothrow) AdjointBuffers();
  if (!B) return PIC_ENOMEM;
  B->seg = seg;
  B->ncp = ncp;
  B->np3 = np3;
  B->nc = nc;
  B->max_rec = kAdjMaxRec;
  B->mu_len = lanes * (size_t)c->cfg.max_ppc * 3;
  B->rec_len = lanes * (size_t)kAdjMaxRec * 12;
  c->adj = B;
  bool ok = true;
  each_buffer(*B, [&](double** p, size_t len) {
    if (!ok) return;
    *p = (double*)ctx_alloc(c, (len ? len : 1) * sizeof(double));
    if (!*p) ok = false;
  });
  if (!ok) {
    adjoint_free(c);
    return PIC_ENOMEM;
  }
  return PIC_OK;
}

cudaError_t store_xv(pic_ctx* c, double* X, double* V) {
  const int b = c->cur;
  k_adj_store<<<nblk(c->P.np), kT, 0, c->stream>>>(c->P.np, c->x[b][0], c->x[b][1], c->x[b][2], c->v[b][0],
                                                   c->v[b][1], c->v[b][2], c->pid[b], X, V);
  c->launches++;
  return cudaGetLastError();
}

// pid-ordered (X, V) into the context, sorted by (cell, pid)
cudaError_t load_sorted(pic_ctx* c, const double* X, const double* V) {
  const int b = c->cur;
  k_adj_load<<<nblk(c->P.np), kT, 0, c->stream>>>(c->P, X, V, c->x[b][0], c->x[b][1], c->x[b][2], c->v[b][0],
                                                  c->v[b][1], c->v[b][2], c->vm[b][0], c->vm[b][1], c->vm[b][2],
                                                  c->pid[b]);
  c->launches++;
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemsetAsync(c->count, 0, (size_t)c->P.ncell * 4, c->stream);
  if (e == cudaSuccess) e = launch_keys(c);
  if (e == cudaSuccess) e = launch_sort(c);
  return e;
}

cudaError_t collide_adjoint(pic_ctx* c, uint32_t c0, const double* lam, double* G) {
  AdjointBuffers& B = *c->adj;
  if (c->cfg.K <= 0) return cudaMemsetAsync(G, 0, B.np3 * sizeof(double), c->stream);
  DsmcAdjArgs a;
  a.P = c->P;
  const int b = c->cur;
  a.v0 = c->v[b][0]; a.v1 = c->v[b][1]; a.v2 = c->v[b][2];
  a.pid = c->pid[b];
  a.start = c->start;
  a.c0 = c0;
  a.lam = lam;
  a.G = G;
  a.ov = c->overlay;
  a.mu = B.mu_ov;
  a.rec = B.rec;
  a.max_ppc = c->cfg.max_ppc;
  a.bm_words = c->bm_words;
  a.Gc = c->dsmc_G;
  a.Kc = c->dsmc_Kc;
  a.nchunks = (c->P.K + c->dsmc_Kc - 1) / c->dsmc_Kc;
  a.max_rec = B.max_rec;
  a.ngroups = c->dsmc_groups;
  a.flags = c->flags;
  if (c->dsmc_smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute((const void*)k_dsmc_adj, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)c->dsmc_smem);
    if (e != cudaSuccess) return e;
  }
  k_dsmc_adj<<<c->dsmc_grid, kAdjDsmcThreads, c->dsmc_smem, c->stream>>>(a);
  c->launches++;
  return cudaGetLastError();
}

// reverse of the closing kick of step n and of the field solve at t_{n+1};
// the context holds x^{n+1} sorted, E at t_{n+1} is E_nodes
cudaError_t close_adjoint(pic_ctx* c, int64_t n1, const double* E_nodes, bool final_step) {
  AdjointBuffers& B = *c->adj;
  const Params& P = c->P;
  const int b = c->cur;
  const int nbp = nblk(P.np), nbc = nblk(P.ncell);
  CloseArgs a;
  a.P = P;
  a.tt = time_terms(P, tval(c, (double)n1));
  a.x0 = c->x[b][0]; a.x1 = c->x[b][1]; a.x2 = c->x[b][2];
  a.pid = c->pid[b];
  a.E0 = E_nodes; a.E1 = E_nodes + P.ncell; a.E2 = E_nodes + 2 * P.ncell;
  a.lam_v = B.lam_v;
  a.carry = B.carry;
  a.lam_x = B.lam_x;
  a.lamL = B.lamL;
  a.part = B.part;
  a.scale = P.dt * P.qm_eff;
  k_adj_close<<<nbp, kT, 0, c->stream>>>(a);
  k_adj_final<<<1, kT, 0, c->stream>>>(B.part, nbp, 3, B.acc, 1.0, 1);
  // lam_E at t_{n+1}: scatter of dt q/m lam_L (+ eps0 h^3 E^N at the end)
  const int64_t sc_need = (P.ncell * 32 + kT - 1) / kT, sc_cap = 16 * (int64_t)c->num_sms;
  k_adj_scatter<<<(int)(sc_need < sc_cap ? sc_need : sc_cap), kT, 0, c->stream>>>(P, c->start, a.x0, a.x1, a.x2,
                                                                                   B.lamL, B.corner24);
  k_adj_nodes<<<nbc, kT, 0, c->stream>>>(P, B.corner24, final_step ? B.seedE : nullptr, P.eps0 * P.dV, B.lamE);
  k_adj_div<<<nbc, kT, 0, c->stream>>>(P, B.lamE, B.badj, B.part);
  c->launches += 5;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // mu = P (-Lap_h)^+ P lam_phi, then the deposit's share of lam_x
  e = launch_cg_on(c, B.badj, B.mu, B.part, nbc, B.Etmp, B.Etmp + P.ncell, B.Etmp + 2 * P.ncell);
  if (e != cudaSuccess) return e;
  k_adj_depgrad<<<nbp, kT, 0, c->stream>>>(P, a.x0, a.x1, a.x2, a.pid, B.mu, P.rho_scale / P.eps0, B.lam_x);
  c->launches++;
  return cudaGetLastError();
}

}  // namespace

extern "C" pic_status pic_adjoint_gradient(pic_ctx* c, int32_t nsteps, int32_t every, const double E_app[3],
                                           const double* v0, double J[3], double dJ_dEapp[3], double* dJ_dv0) {
  if (!c || nsteps < 0 || every < 1 || !J) return PIC_EINVAL;
  if (c->mixed || c->nrep > 0) return PIC_EINVAL;
  if (c->cfg.verify & (PIC_VERIFY_ERROR1 | PIC_VERIFY_ERROR2)) return PIC_EINVAL;
  if (c->cfg.dist != PIC_DIST_CONFIG || c->cfg.n_sigma != 0) return PIC_EINVAL;
  const bool grad = dJ_dEapp || dJ_dv0;
  const int seg = grad ? (nsteps < every ? (nsteps > 0 ? nsteps : 1) : every) : 1;
  const int ncp = grad ? (nsteps + every - 1) / every : 0;
  AS(ensure_buffers(c, seg, ncp > 0 ? ncp : 1));
  AdjointBuffers& B = *c->adj;
  const Params& P = c->P;
  const size_t np3 = B.np3, nc = B.nc;
  for (int d = 0; d < 3; ++d) c->P.E_app[d] = E_app ? E_app[d] : 0.0;
  struct Reset {
    pic_ctx* c;
    ~Reset() {
      for (int d = 0; d < 3; ++d) c->P.E_app[d] = 0.0;
    }
  } reset{c};
  // initial state: x^M(0), and v^M(0) or the given velocities
  AS(pic_sample_mms(c, 0.0));
  if (v0) {
    AK(store_xv(c, B.tx, nullptr));
    AK(cudaMemcpyAsync(B.tv, v0, np3 * sizeof(double), cudaMemcpyDefault, c->stream));
    AK(load_sorted(c, B.tx, B.tv));
    AK(launch_rhs(c, c->t0));
    AK(launch_cg(c));
    c->lor_valid = false;
  }
  c->step = 0;
  // forward with checkpoints (x, v, phi, E)
  const size_t ckn = 2 * np3 + 4 * nc;
  for (int64_t n = 0; n < nsteps; ++n) {
    if (grad && n % every == 0) {
      double* ck = B.ck + (size_t)(n / every) * ckn;
      AK(store_xv(c, ck, ck + np3));
      AK(cudaMemcpyAsync(ck + 2 * np3, c->phi, nc * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
      for (int d = 0; d < 3; ++d)
        AK(cudaMemcpyAsync(ck + 2 * np3 + (1 + d) * nc, c->E[d], nc * sizeof(double), cudaMemcpyDeviceToDevice,
                           c->stream));
    }
    AK(step_fp64(c, n, nullptr));
    c->step = n + 1;
  }
  // objective
  AK(store_xv(c, nullptr, B.tv));
  const int nbp = nblk(P.np), nbc = nblk(P.ncell);
  k_adj_seed<<<nbp, kT, 0, c->stream>>>(P, B.tv, grad ? B.lam_v : nullptr, B.lam_x, B.carry, B.part);
  k_adj_final<<<1, kT, 0, c->stream>>>(B.part, nbp, 1, B.acc + 8, 1.0 / (double)P.np, 0);
  k_adj_energy<<<nbc, kT, 0, c->stream>>>(P.ncell, c->E[0], c->E[1], c->E[2], B.part);
  k_adj_final<<<1, kT, 0, c->stream>>>(B.part, nbc, 1, B.acc + 9, 0.5 * P.eps0 * P.dV, 0);
  c->launches += 4;
  AK(cudaGetLastError());
  double obj[2];
  AK(cudaMemcpyAsync(obj, B.acc + 8, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  AK(cudaStreamSynchronize(c->stream));
  J[0] = obj[0] + obj[1];
  J[1] = obj[1];
  J[2] = obj[0];
  pic_status st = PIC_OK;
  if (!grad) return st;
  // reverse sweep
  for (int d = 0; d < 3; ++d)
    AK(cudaMemcpyAsync(B.seedE + d * nc, c->E[d], nc * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
  AK(cudaMemsetAsync(B.acc, 0, 8 * sizeof(double), c->stream));
  AK(cudaMemsetAsync(B.mu, 0, nc * sizeof(double), c->stream));
  for (int k = ncp - 1; k >= 0; --k) {
    const int64_t s0 = (int64_t)k * every, s1 = s0 + every < nsteps ? s0 + every : nsteps;
    double* ck = B.ck + (size_t)k * ckn;
    AK(load_sorted(c, ck, ck + np3));
    AK(cudaMemcpyAsync(c->phi, ck + 2 * np3, nc * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    for (int d = 0; d < 3; ++d)
      AK(cudaMemcpyAsync(c->E[d], ck + 2 * np3 + (1 + d) * nc, nc * sizeof(double), cudaMemcpyDeviceToDevice,
                         c->stream));
    c->lor_valid = false;
    for (int64_t n = s0; n < s1; ++n) {
      const int64_t r = n - s0;
      StepHook hook = [&](int where) -> cudaError_t {
        if (where == 0) return store_xv(c, B.tx + r * np3, B.tv + r * np3);
        if (where == 1) return store_xv(c, B.tx + (r + 1) * np3, B.tvh + r * np3);
        cudaError_t e = cudaSuccess;
        for (int d = 0; d < 3 && e == cudaSuccess; ++d)
          e = cudaMemcpyAsync(B.tE + (r * 3 + d) * nc, c->E[d], nc * sizeof(double), cudaMemcpyDeviceToDevice,
                              c->stream);
        return e;
      };
      AK(step_fp64(c, n, &hook));
      c->step = n + 1;
    }
    for (int64_t n = s1 - 1; n >= s0; --n) {
      const int64_t r = n - s0;
      // closing kick of step n and the field at t_{n+1}
      AK(load_sorted(c, B.tx + (r + 1) * np3, B.tvh + r * np3));
      AK(collide_adjoint(c, (uint32_t)(2 * n + 1), B.lam_v, B.G));
      AK(close_adjoint(c, n + 1, B.tE + r * 3 * nc, n + 1 == nsteps));
      k_adj_vh<<<nblk((int64_t)np3), kT, 0, c->stream>>>((int64_t)np3, B.lam_v, B.G, B.lam_x, P.dt);
      c->launches++;
      AK(cudaGetLastError());
      // opening kick of step n at (x^n, v^n)
      AK(load_sorted(c, B.tx + r * np3, B.tv + r * np3));
      AK(collide_adjoint(c, (uint32_t)(2 * n), B.lam_v, B.G));
      k_adj_open<<<nblk((int64_t)np3), kT, 0, c->stream>>>((int64_t)np3, B.lam_v, B.G, B.carry);
      c->launches++;
      AK(cudaGetLastError());
    }
  }
  // L^0 has only the opening kick of step 0
  k_adj_sum3<<<nbp, kT, 0, c->stream>>>(P.np, B.carry, P.dt * P.qm_eff, B.part);
  k_adj_final<<<1, kT, 0, c->stream>>>(B.part, nbp, 3, B.acc, 1.0, 1);
  c->launches += 2;
  AK(cudaGetLastError());
  if (dJ_dEapp) AK(cudaMemcpyAsync(dJ_dEapp, B.acc, 3 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  if (dJ_dv0) AK(cudaMemcpyAsync(dJ_dv0, B.lam_v, np3 * sizeof(double), cudaMemcpyDefault, c->stream));
  AK(cudaStreamSynchronize(c->stream));
  c->sampled = false;  // the context's state is the restored first segment
  int flags[2] = {0, 0};
  AK(cudaMemcpyAsync(flags, c->flags, sizeof(flags), cudaMemcpyDeviceToHost, c->stream));
  AK(cudaMemsetAsync(c->flags, 0, sizeof(flags), c->stream));
  AK(cudaStreamSynchronize(c->stream));
  if (flags[0] & 4) st = PIC_ETIMEOUT;
  else if (flags[0] & 1) st = PIC_ECAPACITY;
  else if (flags[0] & 2) st = PIC_ENOCONV;
  return st;
}
