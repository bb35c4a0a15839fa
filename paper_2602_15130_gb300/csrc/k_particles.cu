// Particle-parallel kernels: manufactured sampling (Sec. 3.2), state
// load/store, K-averaged NTC collisions (Algorithm 1, Eq. avg_outcome) with
// the hard-sphere source (Eq. vel_change_1c) or the odd-power one (Eqs.
// vel_change_3, fn), the velocity-Verlet kick and drift (Eq.
// velocity_verlet with the sources of Eq. eom_mms, for the travelling-wave
// and the paper's manufactured problem) and the error norms of Sec. 4.3.
#include "pic_internal.cuh"
#include "ntc_fp64.cuh"

namespace pic {
namespace {

constexpr int kThreads = 256;

inline int blocks_for(int64_t n, int t = kThreads) {
  int64_t b = (n + t - 1) / t;
  return (int)(b < 1 ? 1 : b);
}

// --------------------------------------------------------------------------
// Sampling: xi from the particle's Philox stream, x = x^M(t0), v = v^M.
// Written in pid order into the current buffer.
// --------------------------------------------------------------------------
struct SampleArgs {
  Params P;
  TimeTerms tt;
  double *x0, *x1, *x2, *v0, *v1, *v2, *vm0, *vm1, *vm2;
  uint32_t* pid;
};

__global__ void __launch_bounds__(kThreads) k_sample(SampleArgs a) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.P.np) return;
  const Params& P = a.P;
  const U4 b0 = sample_block(P, (uint64_t)i, 0), b1 = sample_block(P, (uint64_t)i, 1),
           b2 = sample_block(P, (uint64_t)i, 2);
  const double xi[6] = {unif52(b0.x, b0.y), unif52(b0.z, b0.w), unif52(b1.x, b1.y),
                        unif52(b1.z, b1.w), unif52(b2.x, b2.y), unif52(b2.z, b2.w)};
  double s;
  if (P.dist == PIC_DIST_PAPER) {
    // x^M(t0) per axis; v^M(t0) = vh(t0) tau(xi), tau kept in the v^M arrays
    double c;
    a.x0[i] = wrap_unit(xm_solve_gen(a.tt, 0, xi[0], &s, &c));
    a.x1[i] = wrap_unit(xm_solve_gen(a.tt, 1, xi[1], &s, &c));
    a.x2[i] = wrap_unit(xm_solve_gen(a.tt, 2, xi[2], &s, &c));
    const double t0 = tau_inv(xi[3]), t1 = tau_inv(xi[4]), t2 = tau_inv(xi[5]);
    a.v0[i] = t0 * a.tt.vh[0]; a.v1[i] = t1 * a.tt.vh[1]; a.v2[i] = t2 * a.tt.vh[2];
    a.vm0[i] = t0; a.vm1[i] = t1; a.vm2[i] = t2;
    a.pid[i] = (uint32_t)i;
    return;
  }
  const double X0 = xm_solve(P, a.tt, xi[0], &s);
  const double X1 = xm_solve(P, a.tt, xi[1], &s);
  const double X2 = xm_solve(P, a.tt, xi[2], &s);
  const double V0 = P.vmean[0] + P.vsig * normcdfinv(xi[3]);
  const double V1 = P.vmean[1] + P.vsig * normcdfinv(xi[4]);
  const double V2 = P.vmean[2] + P.vsig * normcdfinv(xi[5]);
  a.x0[i] = wrap_unit(X0); a.x1[i] = wrap_unit(X1); a.x2[i] = wrap_unit(X2);
  a.v0[i] = V0; a.v1[i] = V1; a.v2[i] = V2;
  a.vm0[i] = V0; a.vm1[i] = V1; a.vm2[i] = V2;
  a.pid[i] = (uint32_t)i;
}

// Load a caller state (x and v, each [N_p][3] in pid order) into SoA.
struct LoadArgs {
  Params P;
  TimeTerms tt;
  const double *xs, *vs;  // device memory or mapped pinned host memory
  double *x0, *x1, *x2, *v0, *v1, *v2, *vm0, *vm1, *vm2;
  uint32_t* pid;
};

__global__ void __launch_bounds__(kThreads) k_load_state(LoadArgs a) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.P.np) return;
  const Params& P = a.P;
  const U4 b0 = sample_block(P, (uint64_t)i, 0), b1 = sample_block(P, (uint64_t)i, 1),
           b2 = sample_block(P, (uint64_t)i, 2);
  const double xi[6] = {unif52(b0.x, b0.y), unif52(b0.z, b0.w), unif52(b1.x, b1.y),
                        unif52(b1.z, b1.w), unif52(b2.x, b2.y), unif52(b2.z, b2.w)};
  if (P.dist == PIC_DIST_PAPER) {
    a.vm0[i] = tau_inv(xi[3]); a.vm1[i] = tau_inv(xi[4]); a.vm2[i] = tau_inv(xi[5]);
  } else {
    a.vm0[i] = P.vmean[0] + P.vsig * normcdfinv(xi[3]);
    a.vm1[i] = P.vmean[1] + P.vsig * normcdfinv(xi[4]);
    a.vm2[i] = P.vmean[2] + P.vsig * normcdfinv(xi[5]);
  }
  const double* xs = a.xs;
  const double* vs = a.vs;
  a.x0[i] = xs[3 * i]; a.x1[i] = xs[3 * i + 1]; a.x2[i] = xs[3 * i + 2];
  a.v0[i] = vs[3 * i]; a.v1[i] = vs[3 * i + 1]; a.v2[i] = vs[3 * i + 2];
  a.pid[i] = (uint32_t)i;
}

struct StoreArgs {
  int64_t np;
  const double *x0, *x1, *x2, *v0, *v1, *v2;
  const uint32_t* pid;
  double* xv;
};

__global__ void __launch_bounds__(kThreads) k_store_state(StoreArgs a) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= a.np) return;
  const int64_t p = a.pid[j];
  a.xv[3 * p] = a.x0[j]; a.xv[3 * p + 1] = a.x1[j]; a.xv[3 * p + 2] = a.x2[j];
  double* vs = a.xv + 3 * a.np;
  vs[3 * p] = a.v0[j]; vs[3 * p + 1] = a.v1[j]; vs[3 * p + 2] = a.v2[j];
}

struct StoreDvArgs {
  int64_t np;
  const double *d0, *d1, *d2, *m0, *m1, *m2;
  const uint32_t* pid;
  double *dv, *dvm;
};

__global__ void __launch_bounds__(kThreads) k_store_dv(StoreDvArgs a) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= a.np) return;
  const int64_t p = a.pid[j];
  a.dv[3 * p] = a.d0[j]; a.dv[3 * p + 1] = a.d1[j]; a.dv[3 * p + 2] = a.d2[j];
  a.dvm[3 * p] = a.m0[j]; a.dvm[3 * p + 1] = a.m1[j]; a.dvm[3 * p + 2] = a.m2[j];
}

// --------------------------------------------------------------------------
// K-averaged NTC collisions. One warp serves a group of G consecutive cells;
// lane l runs outcome (chunk Kc + l % Kc) of cell (l / Kc) of the group,
// sequentially over its candidate pairs with in-place updates (Algorithm 1).
// The lane's working velocities live in a private overlay slot in global
// memory (L1-resident in practice), valid where the lane's bitmap in shared
// memory has the particle's bit; untouched particles are read from v.
// After __syncwarp the warp sums each particle's per-outcome changes in
// ascending outcome order and divides by K.
// --------------------------------------------------------------------------
struct DsmcArgs {
  Params P;
  const double *v0, *v1, *v2;
  const int32_t* start;
  uint32_t c0;
  double *dv0, *dv1, *dv2;  // out: <dv> - <dv^M>, or <dv> when m0 != nullptr
  double *m0, *m1, *m2;     // out (optional): <dv^M>
  double* overlay;
  int max_ppc, bm_words, G, Kc, nchunks;
  int64_t ngroups;
  unsigned long long* counters;
  int* flags;
  double vh[3];             // PIC_DIST_PAPER: f_v scales at the call's time
  DLog lg;                  // decision log (mode 0: off)
  long long* hist;          // per-step history row: [1] candidates, [2] collisions, [3] g > g_max
};

constexpr int kDsmcThreads = 128;

template <bool kVerify>
__global__ void __launch_bounds__(kDsmcThreads) k_dsmc(DsmcArgs a) {
  extern __shared__ uint32_t smem[];
  const Params& P = a.P;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int wpb = blockDim.x >> 5;
  const int64_t gwarp = (int64_t)blockIdx.x * wpb + wib;
  const int64_t nwarps = (int64_t)gridDim.x * wpb;
  uint32_t* wbm = smem + (size_t)wib * 32 * a.bm_words;     // warp's 32 bitmaps
  uint32_t* bm = wbm + (size_t)lane * a.bm_words;            // this lane's
  double* wov = a.overlay + (size_t)gwarp * 32 * a.max_ppc * 3;
  double* ov = wov + (size_t)lane * a.max_ppc * 3;
  for (int i = 0; i < a.bm_words; ++i) bm[i] = 0u;
  __syncwarp();
  LaneCounts cnt = {0, 0, 0, 0};
  const bool separate = a.m0 != nullptr;

  for (int64_t grp = gwarp; grp < a.ngroups; grp += nwarps) {
    const int64_t cell0 = grp * a.G;
    const int ncl = (int)min((int64_t)a.G, P.ncell - cell0);  // cells in this group
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
      if (run)
      {
        NoRecord none;
        ntc_outcome<kVerify>(P, a.c0, (uint32_t)(cell0 + mycl), (uint32_t)o, c, a.v0 + s, a.v1 + s, a.v2 + s,
                             bm, ov, cnt, none, a.lg);
      }
      __syncwarp();
      // sum this chunk's changes per particle in ascending outcome order
      const bool last = ch == a.nchunks - 1;
      for (int32_t j = gs + lane; j < ge; j += 32) {
        int cl = 0;
        while (cl + 1 < ncl && a.start[cell0 + cl + 1] <= j) ++cl;
        const int32_t cs = a.start[cell0 + cl];
        const int cc = a.start[cell0 + cl + 1] - cs;
        const int jj = j - cs;
        double acc0 = 0.0, acc1 = 0.0, acc2 = 0.0;
        if (ch > 0) { acc0 = a.dv0[j]; acc1 = a.dv1[j]; acc2 = a.dv2[j]; }
        if (cc >= 2 && cc <= a.max_ppc) {
          const double w0 = a.v0[j], w1 = a.v1[j], w2 = a.v2[j];
          for (int k = 0; k < a.Kc; ++k) {
            if (ch * a.Kc + k >= P.K) break;
            const int L = cl * a.Kc + k;
            if ((wbm[(size_t)L * a.bm_words + (jj >> 5)] >> (jj & 31)) & 1u) {
              const double* W = wov + ((size_t)L * a.max_ppc + jj) * 3;
              acc0 = __dadd_rn(acc0, __dsub_rn(W[0], w0));
              acc1 = __dadd_rn(acc1, __dsub_rn(W[1], w1));
              acc2 = __dadd_rn(acc2, __dsub_rn(W[2], w2));
            }
          }
        }
        if (!last) {
          a.dv0[j] = acc0; a.dv1[j] = acc1; a.dv2[j] = acc2;
        } else {
          const double K = (double)P.K;
          const double m0 = acc0 != 0.0 ? acc0 / K : 0.0, m1 = acc1 != 0.0 ? acc1 / K : 0.0,
                       m2 = acc2 != 0.0 ? acc2 / K : 0.0;
          double s0, s1, s2;
          if (P.n_sigma == 0) {
            hs_source(P, a.v0[j], a.v1[j], a.v2[j], cc, &s0, &s1, &s2);
          } else {
            double so[3];
            odd_source(P, a.vh, a.v0[j], a.v1[j], a.v2[j], cc, so);
            s0 = so[0]; s1 = so[1]; s2 = so[2];
          }
          if (separate) {
            a.dv0[j] = m0; a.dv1[j] = m1; a.dv2[j] = m2;
            a.m0[j] = s0; a.m1[j] = s1; a.m2[j] = s2;
          } else {
            a.dv0[j] = m0 - s0; a.dv1[j] = m1 - s1; a.dv2[j] = m2 - s2;
          }
        }
      }
      __syncwarp();
      if (run)
        for (int i = 0; i < (c + 31) / 32; ++i) bm[i] = 0u;
      __syncwarp();
    }
  }
  // warp totals, one atomic per counter per warp
  for (int off = 16; off > 0; off >>= 1) {
    cnt.cand += __shfl_down_sync(0xffffffffu, cnt.cand, off);
    cnt.coll += __shfl_down_sync(0xffffffffu, cnt.coll, off);
    cnt.gmax += __shfl_down_sync(0xffffffffu, cnt.gmax, off);
    cnt.tie += __shfl_down_sync(0xffffffffu, cnt.tie, off);
  }
  if (lane == 0) {
    if (cnt.cand) atomicAdd(a.counters + 0, cnt.cand);
    if (cnt.coll) atomicAdd(a.counters + 1, cnt.coll);
    if (cnt.gmax) atomicAdd(a.counters + 2, cnt.gmax);
    if (cnt.tie) atomicAdd(a.counters + 3, cnt.tie);
    if (a.hist) {
      if (cnt.cand) atomicAdd((unsigned long long*)a.hist + 1, cnt.cand);
      if (cnt.coll) atomicAdd((unsigned long long*)a.hist + 2, cnt.coll);
      if (cnt.gmax) atomicAdd((unsigned long long*)a.hist + 3, cnt.gmax);
    }
  }
}

// --------------------------------------------------------------------------
// Kick (and optionally drift) in sorted order:
//   v += 1/2 (dt q/m (E_p - E^M_p) + dv + dt vdot^M) (vdot^M = 0 for the
//   Gaussian f_v, vh'(t) tau for the paper's f_v),
//   x += dt (v + xdot^M - v^M) at t_half (drift), wrapped; new cell key.
// --------------------------------------------------------------------------
struct KickArgs {
  Params P;
  double *x0, *x1, *x2, *v0, *v1, *v2;
  const double *vm0, *vm1, *vm2;
  const uint32_t* pid;
  const double *dv0, *dv1, *dv2;
  const double *E0, *E1, *E2;
  double *L0, *L1, *L2;  // Lorentz term dt q/m (E_p - E^M_p)
  int lor_mode;          // 0: compute, 1: compute and store, 2: load
  TimeTerms tE, th;
  TimeTerms t0, t1;      // t_n, t_{n+1} for the isolated-collision drift
  int drift;
  int32_t *key, *rank, *count;
};

__device__ __forceinline__ void gather_E(const Params& P, const double* E0, const double* E1, const double* E2,
                                         double x, double y, double z, double* e) {
  const int n = P.n;
  const double un = x * (double)n, vn = y * (double)n, wn = z * (double)n;
  const int i = cell_coord(x, n), j = cell_coord(y, n), k = cell_coord(z, n);
  const double fx = un - (double)i, fy = vn - (double)j, fz = wn - (double)k;
  const int i1 = i + 1 == n ? 0 : i + 1, j1 = j + 1 == n ? 0 : j + 1, k1 = k + 1 == n ? 0 : k + 1;
  const double wx[2] = {1.0 - fx, fx}, wy[2] = {1.0 - fy, fy}, wz[2] = {1.0 - fz, fz};
  const int ii[2] = {i, i1}, jj[2] = {j, j1}, kk[2] = {k, k1};
  double a0 = 0.0, a1 = 0.0, a2 = 0.0;
#pragma unroll
  for (int c = 0; c < 2; ++c)
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
      for (int a = 0; a < 2; ++a) {
        const int64_t node = ii[a] + (int64_t)n * (jj[b] + (int64_t)n * kk[c]);
        const double ww = wx[a] * wy[b] * wz[c];
        a0 += ww * __ldg(E0 + node);
        a1 += ww * __ldg(E1 + node);
        a2 += ww * __ldg(E2 + node);
      }
  e[0] = a0; e[1] = a1; e[2] = a2;
}

__global__ void __launch_bounds__(kThreads) k_kick(KickArgs a) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const Params& P = a.P;
  if (j >= P.np) return;
  double x[3] = {a.x0[j], a.x1[j], a.x2[j]};
  double v[3] = {a.v0[j], a.v1[j], a.v2[j]};
  double L[3];
  if (a.lor_mode == 2) {
    L[0] = a.L0[j]; L[1] = a.L1[j]; L[2] = a.L2[j];
  } else {
    double Ep[3], EM[3];
    gather_E(P, a.E0, a.E1, a.E2, x[0], x[1], x[2], Ep);
    e_manufactured(P, a.tE, x[0], x[1], x[2], &EM[0], &EM[1], &EM[2]);
#pragma unroll
    for (int d = 0; d < 3; ++d) L[d] = P.dt * P.qm_eff * (Ep[d] + P.E_app[d] - EM[d]);
    if (a.lor_mode == 1) {
      a.L0[j] = L[0]; a.L1[j] = L[1]; a.L2[j] = L[2];
    }
  }
  double dv[3] = {0.0, 0.0, 0.0};
  if (a.dv0) { dv[0] = a.dv0[j]; dv[1] = a.dv1[j]; dv[2] = a.dv2[j]; }
  const bool paper = P.dist == PIC_DIST_PAPER;
  double vm[3] = {0.0, 0.0, 0.0};
  if (a.drift || paper) { vm[0] = a.vm0[j]; vm[1] = a.vm1[j]; vm[2] = a.vm2[j]; }
  if (paper) {
    // v^M arrays hold tau: vdot^M(t) = vh'(t) tau (Eq. velocity_verlet)
#pragma unroll
    for (int d = 0; d < 3; ++d) v[d] = v[d] + 0.5 * ((L[d] + dv[d]) + P.dt * (vm[d] * a.tE.dvh[d]));
  } else {
#pragma unroll
    for (int d = 0; d < 3; ++d) v[d] = v[d] + 0.5 * (L[d] + dv[d]);
  }
  a.v0[j] = v[0]; a.v1[j] = v[1]; a.v2[j] = v[2];
  if (!a.drift) return;
  const uint64_t p = a.pid[j];
  const U4 b0 = sample_block(P, p, 0), b1 = sample_block(P, p, 1);
  const double xi[3] = {unif52(b0.x, b0.y), unif52(b0.z, b0.w), unif52(b1.x, b1.y)};
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    double s;
    if (paper) {
      double c;
      xm_solve_gen(a.th, d, xi[d], &s, &c);
      const double xd = xm_dot_gen(a.th, d, s, c);
      x[d] = wrap_unit(x[d] + P.dt * (v[d] + xd - vm[d] * a.th.vh[d]));
    } else if (P.verify & PIC_VERIFY_ISOLATE) {
      // exact manufactured increment x^M(t_{n+1}) - x^M(t_n) (Sec. 5.4)
      const double dxm = xm_solve(P, a.t1, xi[d], &s) - xm_solve(P, a.t0, xi[d], &s);
      x[d] = wrap_unit(x[d] + (P.dt * (v[d] - vm[d]) + dxm));
    } else {
      xm_solve(P, a.th, xi[d], &s);
      const double xd = xm_dot(P, a.th, s);
      x[d] = wrap_unit(x[d] + P.dt * (v[d] + xd - vm[d]));
    }
  }
  a.x0[j] = x[0]; a.x1[j] = x[1]; a.x2[j] = x[2];
  const int n = P.n;
  const int32_t k = cell_coord(x[0], n) + n * (cell_coord(x[1], n) + n * cell_coord(x[2], n));
  a.key[j] = k;
  a.rank[j] = cell_slot(a.count, k);
}

// --------------------------------------------------------------------------
// Error norms (Sec. 4.3): per-block partial sums of squares and maxima of
// e = alpha - alpha^M for x, y, z (minimum image), u, v, w; then phi over
// nodes; a single block combines the partials in fixed order.
// --------------------------------------------------------------------------
struct ErrArgs {
  Params P;
  TimeTerms tt;
  const double *x0, *x1, *x2, *v0, *v1, *v2, *vm0, *vm1, *vm2;
  const uint32_t* pid;
  const double* phi;
  double* part;  // [blocks][14]: 7 sums then 7 maxima
  int pblocks;   // blocks over particles; the rest cover nodes
  double* out;
};

__device__ __forceinline__ void block_reduce_14(double* vals, double* sh) {
  // vals[0..6] summed, vals[7..13] max-reduced; result in thread 0
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < 14; ++q) {
    double x = vals[q];
    for (int off = 16; off > 0; off >>= 1) {
      const double y = __shfl_down_sync(0xffffffffu, x, off);
      x = q < 7 ? x + y : fmax(x, y);
    }
    if (lane == 0) sh[w * 14 + q] = x;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int q = 0; q < 14; ++q) {
      double x = sh[q];
      for (int ww = 1; ww < (int)(blockDim.x >> 5); ++ww) x = q < 7 ? x + sh[ww * 14 + q] : fmax(x, sh[ww * 14 + q]);
      vals[q] = x;
    }
  }
}

__global__ void __launch_bounds__(kThreads) k_err_partial(ErrArgs a) {
  __shared__ double sh[(kThreads / 32) * 14];
  const Params& P = a.P;
  double vals[14];
#pragma unroll
  for (int q = 0; q < 14; ++q) vals[q] = 0.0;
  if ((int)blockIdx.x < a.pblocks) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < P.np) {
      const uint64_t p = a.pid[j];
      const U4 b0 = sample_block(P, p, 0), b1 = sample_block(P, p, 1);
      const double xi[3] = {unif52(b0.x, b0.y), unif52(b0.z, b0.w), unif52(b1.x, b1.y)};
      const double xs[3] = {a.x0[j], a.x1[j], a.x2[j]};
      const double vs[3] = {a.v0[j], a.v1[j], a.v2[j]};
      const double vms[3] = {a.vm0[j], a.vm1[j], a.vm2[j]};
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        double s, c;
        const bool paper = P.dist == PIC_DIST_PAPER;
        const double xm = paper ? xm_solve_gen(a.tt, d, xi[d], &s, &c) : xm_solve(P, a.tt, xi[d], &s);
        double e = xs[d] - xm;
        e -= floor(e + 0.5);
        vals[d] = e * e;
        vals[7 + d] = fabs(e);
        const double ev = vs[d] - (paper ? vms[d] * a.tt.vh[d] : vms[d]);
        vals[3 + d] = ev * ev;
        vals[10 + d] = fabs(ev);
      }
    }
  } else {
    const int64_t id = (int64_t)(blockIdx.x - a.pblocks) * blockDim.x + threadIdx.x;
    if (id < P.ncell) {
      const int n = P.n;
      const int i = (int)(id % n), jj = (int)((id / n) % n), k = (int)(id / ((int64_t)n * n));
      const double X = i * P.h, Y = jj * P.h, Z = k * P.h;
      double s0, s1, s2;
      s0 = sinpi(2.0 * (X - P.phi_shift[0]));
      s1 = sinpi(2.0 * (Y - P.phi_shift[1]));
      s2 = sinpi(2.0 * (Z - P.phi_shift[2]));
      const double phiM = a.tt.em_amp / kTwoPi * s0 * s1 * s2;
      const double e = a.phi[id] - phiM;
      vals[6] = e * e;
      vals[13] = fabs(e);
    }
  }
  block_reduce_14(vals, sh);
  if (threadIdx.x == 0)
    for (int q = 0; q < 14; ++q) a.part[(size_t)blockIdx.x * 14 + q] = vals[q];
}

constexpr int kFinalThreads = 512;

// one block: each thread sums a fixed strided subset, then a fixed tree
__global__ void __launch_bounds__(kFinalThreads) k_err_final(ErrArgs a, int nblocks) {
  __shared__ double sh[kFinalThreads];
  for (int q = 0; q < 14; ++q) {
    double x = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
      const double y = a.part[(size_t)b * 14 + q];
      x = q < 7 ? x + y : fmax(x, y);
    }
    sh[threadIdx.x] = x;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
      if ((int)threadIdx.x < w) sh[threadIdx.x] = q < 7 ? sh[threadIdx.x] + sh[threadIdx.x + w]
                                                       : fmax(sh[threadIdx.x], sh[threadIdx.x + w]);
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      double r = sh[0];
      if (q < 6) r = sqrt(r / (double)a.P.np);
      else if (q == 6) r = sqrt(r / (double)a.P.ncell);
      a.out[q] = r;
    }
    __syncthreads();
  }
}

}  // namespace

// ---------------------------------------------------------------------------
cudaError_t launch_sample(pic_ctx* c, double t0) {
  SampleArgs a;
  a.P = c->P;
  a.tt = time_terms(c->P, t0);
  const int b = c->cur;
  a.x0 = c->x[b][0]; a.x1 = c->x[b][1]; a.x2 = c->x[b][2];
  a.v0 = c->v[b][0]; a.v1 = c->v[b][1]; a.v2 = c->v[b][2];
  a.vm0 = c->vm[b][0]; a.vm1 = c->vm[b][1]; a.vm2 = c->vm[b][2];
  a.pid = c->pid[b];
  prof_begin(c);
  k_sample<<<blocks_for(c->P.np), kThreads, 0, c->stream>>>(a);
  prof_end(c, KC_SAMPLE);
  c->launches++;
  return cudaGetLastError();
}

cudaError_t launch_load_state(pic_ctx* c, const double* x, const double* v, double t) {
  LoadArgs a;
  a.P = c->P;
  a.tt = time_terms(c->P, t);
  a.xs = x;
  a.vs = v;
  const int b = c->cur;
  a.x0 = c->x[b][0]; a.x1 = c->x[b][1]; a.x2 = c->x[b][2];
  a.v0 = c->v[b][0]; a.v1 = c->v[b][1]; a.v2 = c->v[b][2];
  a.vm0 = c->vm[b][0]; a.vm1 = c->vm[b][1]; a.vm2 = c->vm[b][2];
  a.pid = c->pid[b];
  prof_begin(c);
  k_load_state<<<blocks_for(c->P.np), kThreads, 0, c->stream>>>(a);
  prof_end(c, KC_OTHER);
  c->launches++;
  return cudaGetLastError();
}

cudaError_t launch_store_state(pic_ctx* c, double* xv) {
  StoreArgs a;
  a.np = c->P.np;
  const int b = c->cur;
  a.x0 = c->x[b][0]; a.x1 = c->x[b][1]; a.x2 = c->x[b][2];
  a.v0 = c->v[b][0]; a.v1 = c->v[b][1]; a.v2 = c->v[b][2];
  a.pid = c->pid[b];
  a.xv = xv;
  prof_begin(c);
  k_store_state<<<blocks_for(c->P.np), kThreads, 0, c->stream>>>(a);
  prof_end(c, KC_OTHER);
  c->launches++;
  return cudaGetLastError();
}

cudaError_t launch_store_dv(pic_ctx* c, double* dv, double* dvm) {
  StoreDvArgs a;
  a.np = c->P.np;
  a.d0 = c->dv[0]; a.d1 = c->dv[1]; a.d2 = c->dv[2];
  a.m0 = c->dvm[0]; a.m1 = c->dvm[1]; a.m2 = c->dvm[2];
  a.pid = c->pid[c->cur];
  a.dv = dv;
  a.dvm = dvm;
  prof_begin(c);
  k_store_dv<<<blocks_for(c->P.np), kThreads, 0, c->stream>>>(a);
  prof_end(c, KC_OTHER);
  c->launches++;
  return cudaGetLastError();
}

cudaError_t launch_dsmc(pic_ctx* c, uint32_t c0, bool separate, double t_src) {
  DsmcArgs a;
  a.P = c->P;
  const TimeTerms ts = time_terms(c->P, t_src);
  for (int d = 0; d < 3; ++d) a.vh[d] = ts.vh[d];
  const int b = c->cur;
  a.v0 = c->v[b][0]; a.v1 = c->v[b][1]; a.v2 = c->v[b][2];
  a.start = c->start;
  a.c0 = c0;
  a.dv0 = c->dv[0]; a.dv1 = c->dv[1]; a.dv2 = c->dv[2];
  if (separate) { a.m0 = c->dvm[0]; a.m1 = c->dvm[1]; a.m2 = c->dvm[2]; }
  else { a.m0 = a.m1 = a.m2 = nullptr; }
  a.overlay = c->overlay;
  a.max_ppc = c->cfg.max_ppc;
  a.bm_words = c->bm_words;
  a.G = c->dsmc_G;
  a.Kc = c->dsmc_Kc;
  a.nchunks = (c->P.K + c->dsmc_Kc - 1) / c->dsmc_Kc;
  a.ngroups = c->dsmc_groups;
  a.counters = c->counters;
  a.flags = c->flags;
  a.lg = DLog{c->dlog, c->dlog_n, (long long)c->dlog_cap, c->dlog ? c->dlog_mode : 0};
  a.hist = c->hist_row;
  prof_begin(c);
  if (c->P.verify || a.lg.mode == PIC_DLOG_ALL)
    k_dsmc<true><<<c->dsmc_grid, kDsmcThreads, c->dsmc_smem, c->stream>>>(a);
  else
    k_dsmc<false><<<c->dsmc_grid, kDsmcThreads, c->dsmc_smem, c->stream>>>(a);
  prof_end(c, KC_DSMC);
  c->launches++;
  return cudaGetLastError();
}

int dsmc_threads() { return kDsmcThreads; }
const void* dsmc_kernel_ptr(bool verify) {
  return verify ? (const void*)k_dsmc<true> : (const void*)k_dsmc<false>;
}

cudaError_t launch_kick(pic_ctx* c, double tE, bool with_coll, bool drift, double th, double tn1) {
  KickArgs a;
  a.P = c->P;
  const int b = c->cur;
  a.x0 = c->x[b][0]; a.x1 = c->x[b][1]; a.x2 = c->x[b][2];
  a.v0 = c->v[b][0]; a.v1 = c->v[b][1]; a.v2 = c->v[b][2];
  a.vm0 = c->vm[b][0]; a.vm1 = c->vm[b][1]; a.vm2 = c->vm[b][2];
  a.pid = c->pid[b];
  if (with_coll) { a.dv0 = c->dv[0]; a.dv1 = c->dv[1]; a.dv2 = c->dv[2]; }
  else { a.dv0 = a.dv1 = a.dv2 = nullptr; }
  a.E0 = c->E[0]; a.E1 = c->E[1]; a.E2 = c->E[2];
  a.L0 = c->lor[0]; a.L1 = c->lor[1]; a.L2 = c->lor[2];
  // the kick without drift closes a step at the time level where the next
  // step's first kick starts: keep its Lorentz term for that kick
  a.lor_mode = drift ? (c->lor_valid ? 2 : 0) : 1;
  a.tE = time_terms(c->P, tE);
  a.th = time_terms(c->P, th);
  a.t0 = time_terms(c->P, tE);
  a.t1 = time_terms(c->P, tn1);
  a.drift = drift ? 1 : 0;
  a.key = c->key;
  a.rank = c->rank;
  a.count = c->count;
  prof_begin(c);
  k_kick<<<blocks_for(c->P.np), kThreads, 0, c->stream>>>(a);
  prof_end(c, KC_KICK);
  c->launches++;
  c->lor_valid = !drift;
  return cudaGetLastError();
}

cudaError_t launch_errors(pic_ctx* c, double t) {
  ErrArgs a;
  a.P = c->P;
  a.tt = time_terms(c->P, t);
  const int b = c->cur;
  a.x0 = c->x[b][0]; a.x1 = c->x[b][1]; a.x2 = c->x[b][2];
  a.v0 = c->v[b][0]; a.v1 = c->v[b][1]; a.v2 = c->v[b][2];
  a.vm0 = c->vm[b][0]; a.vm1 = c->vm[b][1]; a.vm2 = c->vm[b][2];
  a.pid = c->pid[b];
  a.phi = c->phi;
  a.part = c->err_part;
  a.pblocks = blocks_for(c->P.np);
  a.out = c->err_out;
  const int nb = a.pblocks + blocks_for(c->P.ncell);
  prof_begin(c);
  k_err_partial<<<nb, kThreads, 0, c->stream>>>(a);
  k_err_final<<<1, kFinalThreads, 0, c->stream>>>(a, nb);
  prof_end(c, KC_ERR);
  c->launches += 2;
  return cudaGetLastError();
}

int err_blocks_needed(int64_t np, int64_t ncell) { return blocks_for(np) + blocks_for(ncell); }

cudaError_t launch_err_final(pic_ctx* c, int nb) {
  ErrArgs a;
  a.P = c->P;
  a.part = c->err_part;
  a.out = c->err_out;
  k_err_final<<<1, kFinalThreads, 0, c->stream>>>(a, nb);
  c->launches++;
  return cudaGetLastError();
}

}  // namespace pic

namespace pic {
TimeTerms time_terms(const Params& P, double t) {
  TimeTerms tt;
  tt.t = t;
  tt.ct = P.fx_speed * t;
  tt.cos2ct = cos(kTwoPi * tt.ct);
  tt.sin2ct = sin(kTwoPi * tt.ct);
  tt.em_amp = kTwoPi * P.phi_amp * exp(t / (2.0 * P.phi_T));
  for (int d = 0; d < 3; ++d) {
    tt.fA[d] = tt.fs[d] = tt.fdA[d] = tt.fds[d] = tt.fsn[d] = 0.0;
    tt.fcs[d] = 1.0;
    tt.vh[d] = tt.dvh[d] = 0.0;
  }
  if (P.dist == PIC_DIST_PAPER) {
    // Sec. 5.2 on the unit cube, T = t_ref
    const double T = P.t_ref, e = exp(t / T), vb = P.vbar;
    tt.fA[0] = e / 5.0;  tt.fs[0] = 0.0;
    tt.fA[1] = 1.0 / 5.0; tt.fs[1] = 3.0 * e / 20.0;
    tt.fA[2] = -e / 6.0; tt.fs[2] = -e / 15.0;
    for (int d = 0; d < 3; ++d) {
      tt.fdA[d] = d == 1 ? 0.0 : tt.fA[d] / T;
      tt.fds[d] = tt.fs[d] / T;
      tt.fcs[d] = cos(kTwoPi * tt.fs[d]);
      tt.fsn[d] = sin(kTwoPi * tt.fs[d]);
    }
    tt.vh[0] = vb * (1.0 + sin(kPi * t / (2.0 * T)) / 5.0);
    tt.vh[1] = vb * (1.0 + cos(kPi * t / T) / 5.0);
    tt.vh[2] = vb * (1.0 + sin(3.0 * kPi * t / (2.0 * T)) / 5.0);
    tt.dvh[0] = vb * (kPi / (2.0 * T)) * cos(kPi * t / (2.0 * T)) / 5.0;
    tt.dvh[1] = -vb * (kPi / T) * sin(kPi * t / T) / 5.0;
    tt.dvh[2] = vb * (3.0 * kPi / (2.0 * T)) * cos(3.0 * kPi * t / (2.0 * T)) / 5.0;
  }
  return tt;
}
}  // namespace pic
