// Batched precision form: many independent replicates (their own mesh edge,
// particle count, K, dt, cross section and Philox seed) advanced together.
// All replicates live back to back in the context's arrays: particles of
// replicate r at [poff_r, poff_{r+1}), its cells and nodes at coff_r + local
// index (each replicate's range padded to a multiple of 256 so that no tile
// straddles two replicates). The cell sort, gather and CIC kernels of the
// single-domain form work on the global indices unchanged; the kernels here
// are the ones where per-replicate parameters enter.
//
//  - sampling: binary search of the particle's replicate;
//  - RHS: the node's replicate from rep_of_cell, FP64 manufactured terms;
//  - CG: one block per replicate (largest first), block-level phases only
//    (no grid-wide barriers), double-float inner products;
//  - DSMC: a static list of (replicate, cell group) work items so warps of
//    one launch serve replicates of different K and cell size;
//  - kick/drift: per particle, the replicate of its cell.
// Philox counters use the replicate's seed, local cell index and local pid,
// so replicate r of a batch draws the same pairs as a single-domain run of
// the same configuration.
#include "mixed_common.cuh"

namespace pic {
namespace {

constexpr int kThreads = 256;

inline int blocks_for(int64_t n, int t = kThreads) {
  int64_t b = (n + t - 1) / t;
  return (int)(b < 1 ? 1 : b);
}

__device__ __forceinline__ int find_rep(const int64_t* poff, int R, int64_t i) {
  int lo = 0, hi = R;  // poff[lo] <= i < poff[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (poff[mid] <= i) lo = mid; else hi = mid;
  }
  return lo;
}

// ---------------------------------------------------------------- sample --
struct BSampleArgs {
  const Params* prm;
  const BatchRep* reps;
  const TimeTerms* tt;  // [R][3], slot 0 = t0
  const int64_t* poff;
  int R;
  int64_t np;
  const double* xv;     // optional caller state (global particle order)
  int32_t* cell;
  float *o0, *o1, *o2, *v0, *v1, *v2, *m0, *m1, *m2;
  uint32_t* pid;
};

__global__ void __launch_bounds__(kThreads) kb_sample(BSampleArgs a) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.np) return;
  const int r = find_rep(a.poff, a.R, i);
  const Params& P = a.prm[r];
  const int64_t loc = i - a.poff[r];
  const U4 b0 = sample_block(P, (uint64_t)loc, 0), b1 = sample_block(P, (uint64_t)loc, 1),
           b2 = sample_block(P, (uint64_t)loc, 2);
  const double xi[6] = {unif52(b0.x, b0.y), unif52(b0.z, b0.w), unif52(b1.x, b1.y),
                        unif52(b1.z, b1.w), unif52(b2.x, b2.y), unif52(b2.z, b2.w)};
  double x[3], v[3], vm[3];
  for (int d = 0; d < 3; ++d) {
    double s;
    vm[d] = P.vmean[d] + P.vsig * normcdfinv(xi[3 + d]);
    if (a.xv) {
      x[d] = a.xv[3 * i + d];
      v[d] = a.xv[3 * a.np + 3 * i + d];
    } else {
      x[d] = wrap_unit(xm_solve(P, a.tt[3 * r], xi[d], &s));
      v[d] = vm[d];
    }
  }
  const int n = P.n;
  int ci[3];
  float off[3];
  for (int d = 0; d < 3; ++d) {
    ci[d] = cell_coord(x[d], n);
    const float o = (float)(x[d] * (double)n - (double)ci[d]);
    off[d] = o >= 1.f ? 0x1.fffffep-1f : (o < 0.f ? 0.f : o);
  }
  a.cell[i] = (int32_t)(a.reps[r].coff + ci[0] + n * (ci[1] + n * ci[2]));
  a.o0[i] = off[0]; a.o1[i] = off[1]; a.o2[i] = off[2];
  a.v0[i] = (float)v[0]; a.v1[i] = (float)v[1]; a.v2[i] = (float)v[2];
  a.m0[i] = (float)vm[0]; a.m1[i] = (float)vm[1]; a.m2[i] = (float)vm[2];
  a.pid[i] = (uint32_t)loc;
}

// ------------------------------------------------------------------- RHS --
struct BRhsArgs {
  const Params* prm;
  const BatchRep* reps;
  const TimeTerms* tt;
  int slot;
  const uint16_t* rep_of_cell;
  int64_t ncell;
  const double* corner;
  double* rho;
  float* b32;
};

__global__ void __launch_bounds__(kThreads) kb_rhs(BRhsArgs a) {
  const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= a.ncell) return;
  const uint16_t r = a.rep_of_cell[id];
  if (r == 0xFFFFu) {
    a.rho[id] = 0.0;
    a.b32[id] = 0.f;
    return;
  }
  const Params& P = a.prm[r];
  const TimeTerms& tt = a.tt[3 * r + a.slot];
  const int64_t base = a.reps[r].coff;
  const int n = P.n;
  const int loc = (int)(id - base);
  const int i = loc % n, j = (loc / n) % n, k = loc / (n * n);
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < 2; ++c)
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int ii = i - q < 0 ? n - 1 : i - q, jj = j - b < 0 ? n - 1 : j - b, kk = k - c < 0 ? n - 1 : k - c;
        s += a.corner[(int64_t)(q + 2 * b + 4 * c) * a.ncell + base + ii + (int64_t)n * (jj + (int64_t)n * kk)];
      }
  const double rho = P.rho_scale * s;
  const double X = i * P.h, Y = j * P.h, Z = k * P.h;
  const double phiM = tt.em_amp / kTwoPi * sinpi(2.0 * (X - P.phi_shift[0])) * sinpi(2.0 * (Y - P.phi_shift[1])) *
                      sinpi(2.0 * (Z - P.phi_shift[2]));
  const double lap_phiM = -3.0 * kTwoPi * kTwoPi * phiM;
  const double rhoM = P.q_eff * P.nphys * (1.0 + P.fx_amp * sinpi(2.0 * (X - tt.ct))) *
                      (1.0 + P.fx_amp * sinpi(2.0 * (Y - tt.ct))) * (1.0 + P.fx_amp * sinpi(2.0 * (Z - tt.ct)));
  a.rho[id] = rho;
  a.b32[id] = (float)(rho / P.eps0 - lap_phiM - rhoM / P.eps0);
}

// -------------------------------------------------------------------- CG --
// One block per replicate; phases separated by __syncthreads only.
constexpr int kCgThreads = 1024;

struct BCgArgs {
  const BatchRep* reps;
  const int* order;
  int R;
  float *b, *x, *r, *p, *q;
  float4* E4;  // (Ex, Ey, Ez, 0) per node
  double tol;
  int maxit;
  int* iters;
  double* res;
  int* flags;
};

// FP64 total of a double-float partial; valid in thread 0 only
__device__ __forceinline__ double block_df_total0(DF v, double* sh) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v = df_add(v, df_shfl_xor(v, off));
  __syncthreads();
  if (lane == 0) sh[w] = df_to_double(v);
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < nw; ++i) t += sh[i];
  return t;
}

// Thread 0 keeps the FP64 scalars (rr, bb, the stopping threshold) and
// broadcasts FP32 coefficients and the stop decision through shared memory.
__global__ void __launch_bounds__(kCgThreads) kb_cg(BCgArgs a) {
  __shared__ double sh[40];
  __shared__ float fsc[2];  // [0] broadcast coefficient (mean, alpha), [1] beta
  __shared__ int stop;
  for (int ri = blockIdx.x; ri < a.R; ri += gridDim.x) {
    const int rep = a.order[ri];
    const BatchRep& B = a.reps[rep];
    const int n = B.f.n, nn = n * n, m = nn * n;
    float* b = a.b + B.coff;
    float* x = a.x + B.coff;
    float* r = a.r + B.coff;
    float* p = a.p + B.coff;
    float* q = a.q + B.coff;
    const float inv_h2 = (float)n * (float)n, inv_2h = 0.5f * (float)n;
    auto nbr = [&](int id, int* o) {
      const int i = id % n, j = (id / n) % n, k = id / nn;
      o[0] = i == n - 1 ? id - (n - 1) : id + 1;
      o[1] = i == 0 ? id + (n - 1) : id - 1;
      o[2] = j == n - 1 ? id - (n - 1) * n : id + n;
      o[3] = j == 0 ? id + (n - 1) * n : id - n;
      o[4] = k == n - 1 ? id - (n - 1) * nn : id + nn;
      o[5] = k == 0 ? id + (n - 1) * nn : id - nn;
    };
    // zero-mean b
    DF acc{0.f, 0.f};
    for (int id = threadIdx.x; id < m; id += blockDim.x) acc = df_add_f(acc, b[id]);
    {
      const double t = block_df_total0(acc, sh);
      if (threadIdx.x == 0) fsc[0] = (float)(t / (double)m);
      __syncthreads();
    }
    const float mean_b = fsc[0];
    DF rr_l{0.f, 0.f}, bb_l{0.f, 0.f};
    for (int id = threadIdx.x; id < m; id += blockDim.x) {
      int o[6];
      nbr(id, o);
      const float bv = b[id] - mean_b;
      b[id] = bv;
      const float rv = bv - (6.f * x[id] - (x[o[0]] + x[o[1]] + x[o[2]] + x[o[3]] + x[o[4]] + x[o[5]])) * inv_h2;
      r[id] = rv;
      rr_l = df_fma(rr_l, rv, rv);
      bb_l = df_fma(bb_l, bv, bv);
    }
    double rr = block_df_total0(rr_l, sh);  // thread 0
    const double bb = block_df_total0(bb_l, sh);
    const double thresh = a.tol * sqrt(bb);
    int it = 0, status = 0;
    while (true) {
      if (threadIdx.x == 0) stop = (bb == 0.0 || sqrt(rr) <= thresh) ? 1 : (it >= a.maxit ? 2 : 0);
      __syncthreads();
      if (stop == 1) break;
      if (stop == 2) { status = 1; break; }
      const float beta = fsc[1];
      for (int id = threadIdx.x; id < m; id += blockDim.x) p[id] = it == 0 ? r[id] : fmaf(beta, p[id], r[id]);
      __syncthreads();
      DF pq_l{0.f, 0.f};
      for (int id = threadIdx.x; id < m; id += blockDim.x) {
        int o[6];
        nbr(id, o);
        const float pc = p[id];
        const float qv = (6.f * pc - (p[o[0]] + p[o[1]] + p[o[2]] + p[o[3]] + p[o[4]] + p[o[5]])) * inv_h2;
        q[id] = qv;
        pq_l = df_fma(pq_l, pc, qv);
      }
      {
        const double pq = block_df_total0(pq_l, sh);
        if (threadIdx.x == 0) fsc[0] = (float)(rr / pq);
        __syncthreads();
      }
      const float alpha = fsc[0];
      DF rn_l{0.f, 0.f};
      for (int id = threadIdx.x; id < m; id += blockDim.x) {
        x[id] = fmaf(alpha, p[id], x[id]);
        const float rv = fmaf(-alpha, q[id], r[id]);
        r[id] = rv;
        rn_l = df_fma(rn_l, rv, rv);
      }
      const double rr_new = block_df_total0(rn_l, sh);
      ++it;
      if (threadIdx.x == 0) {
        fsc[1] = (float)(rr_new / rr);
        rr = rr_new;
      }
    }
    DF xs{0.f, 0.f};
    for (int id = threadIdx.x; id < m; id += blockDim.x) xs = df_add_f(xs, x[id]);
    {
      const double t = block_df_total0(xs, sh);
      if (threadIdx.x == 0) fsc[0] = (float)(t / (double)m);
      __syncthreads();
    }
    const float mean_x = fsc[0];
    for (int id = threadIdx.x; id < m; id += blockDim.x) x[id] -= mean_x;
    __syncthreads();
    for (int id = threadIdx.x; id < m; id += blockDim.x) {
      int o[6];
      nbr(id, o);
      a.E4[B.coff + id] = make_float4(-(x[o[0]] - x[o[1]]) * inv_2h, -(x[o[2]] - x[o[3]]) * inv_2h,
                                      -(x[o[4]] - x[o[5]]) * inv_2h, 0.f);
    }
    if (threadIdx.x == 0) {
      a.iters[rep] = it;
      a.res[rep] = bb > 0.0 ? sqrt(rr) / sqrt(bb) : 0.0;
      if (status) atomicOr(a.flags, 2);
      atomicMax(a.flags + 1, it);
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------ DSMC --
struct BDsmcArgs {
  const BatchRep* reps;
  const float *v0, *v1, *v2;
  const int32_t* start;
  const int64_t* step;  // device-side step counter (graph replays change no argument)
  int phase;
  const int2* items;
  int64_t n_items;
  float *dv0, *dv1, *dv2;
  float* overlay;
  int max_ppc, bm_words;
  unsigned long long* counters;
  int* flags;
};

// overlay copy where this outcome touched the particle, else the cell's
// velocity (a branch here: selecting the addresses, which helps the
// single-domain kernel, measured 502 -> 532 ms per batched step)
__device__ __forceinline__ void load_vel_b(int p, const uint32_t* bm, const float* ov, const float* v0,
                                           const float* v1, const float* v2, float* o) {
  if ((bm[p >> 5] >> (p & 31)) & 1u) {
    o[0] = ov[3 * p]; o[1] = ov[3 * p + 1]; o[2] = ov[3 * p + 2];
  } else {
    o[0] = v0[p]; o[1] = v1[p]; o[2] = v2[p];
  }
}

struct CountsB {
  unsigned long long cand, coll, gmax, tie, ftie;
};

// Algorithm 1 for one (cell, outcome), as in the single-domain FP32 kernel.
__device__ void ntc_outcome_b(const ParamsF& P, uint32_t c0, uint32_t cell, uint32_t o, int c, const float* v0,
                              const float* v1, const float* v2, uint32_t* bm, float* ov, CountsB& cnt) {
  const U4 u = philox<true>(c0, cell, 0xFFFFFFFFu, o << 8, P.key0, P.key1);
  const float base = (float)(((long long)c * (long long)(c - 1)) >> 1) * P.pmax;
  const float S = base + unif24(u.x);
  const int npairs = (int)floorf(S);
  // flagged FP32 decisions: the bounds of the single-domain kernel
  if (fabsf(S - rintf(S)) <= fmaf(base + S, 0x1p-22f, 0x1p-24f)) ++cnt.ftie;
  // candidate s: block (c0, cell, s, o << 8) = (p, q, accept, epsilon);
  // chi is word s mod 4 of block (c0, cell, s / 4, (o << 8) | 1)
  U4 bchi{0u, 0u, 0u, 0u};
  for (int s = 0; s < npairs; ++s) {
    const U4 b0 = philox<true>(c0, cell, (uint32_t)s, o << 8, P.key0, P.key1);
    if ((s & 3) == 0) bchi = philox<true>(c0, cell, (uint32_t)(s >> 2), (o << 8) | 1u, P.key0, P.key1);
    const uint32_t wchi = (s & 3) == 0 ? bchi.x : (s & 3) == 1 ? bchi.y : (s & 3) == 2 ? bchi.z : bchi.w;
    const uint32_t p = draw_index(b0.x, (uint32_t)c);
    // q uniform over the other c - 1 particles
    uint32_t q = draw_index(b0.y, (uint32_t)(c - 1));
    q += q >= p ? 1u : 0u;
    float vp[3], vq[3];
    load_vel_b((int)p, bm, ov, v0, v1, v2, vp);
    load_vel_b((int)q, bm, ov, v0, v1, v2, vq);
    const float dx = vp[0] - vq[0], dy = vp[1] - vq[1], dz = vp[2] - vq[2];
    const float g2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    const float ug = unif24(b0.z) * P.gmax;
    const float ug2 = ug * ug;
    ++cnt.cand;
    if (g2 > P.gmax2) ++cnt.gmax;
    const float dg = (P.gmax + ug) * 0x1p-19f;
    if (fabsf(ug2 - g2) <= dg * fmaf(2.f, ug, dg)) ++cnt.tie;
    if (ug2 < g2) {
      float se, ce;
      sincospif(2.f * unif24(b0.w), &se, &ce);
      const float cchi = 1.f - 2.f * unif24(wchi);
      const float schi = sqrtf(fmaxf(0.f, 1.f - cchi * cchi));
      const float g = sqrtf(g2);
      const float nv[3] = {ce * schi, se * schi, cchi};
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const float cm = 0.5f * (vp[d] + vq[d]);
        const float hg = 0.5f * g * nv[d];
        ov[3 * p + d] = cm + hg;
        ov[3 * q + d] = cm - hg;
      }
      bm[p >> 5] |= 1u << (p & 31);
      bm[q >> 5] |= 1u << (q & 31);
      ++cnt.coll;
    }
  }
}

constexpr int kDsmcThreads = 128;

__global__ void __launch_bounds__(kDsmcThreads, 7) kb_dsmc(BDsmcArgs a) {
  extern __shared__ uint32_t smem[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int wpb = blockDim.x >> 5;
  const int64_t gwarp = (int64_t)blockIdx.x * wpb + wib;
  const int64_t nwarps = (int64_t)gridDim.x * wpb;
  uint32_t* bm = smem + ((size_t)wib * 32 + lane) * a.bm_words;
  float* wov = a.overlay + (size_t)gwarp * 32 * a.max_ppc * 3;
  float* ov = wov + (size_t)lane * a.max_ppc * 3;
  for (int i = 0; i < a.bm_words; ++i) bm[i] = 0u;
  __syncwarp();
  CountsB cnt = {0, 0, 0, 0, 0};
  const uint32_t c0 = (uint32_t)(2 * (*a.step) + a.phase);
  for (int64_t it = gwarp; it < a.n_items; it += nwarps) {
    const int2 item = a.items[it];
    const BatchRep& B = a.reps[item.x];
    const ParamsF& P = B.f;
    const int Kc = B.Kc, G = B.G, nchunks = B.nchunks;
    const int32_t* start = a.start + B.coff;  // local cell index -> global start
    const int cell0 = item.y;
    const int ncl = min(G, (int)P.ncell - cell0);
    const int mycl = lane / Kc;
    const bool lane_cell = mycl < ncl;
    int32_t s = 0, c = 0;
    if (lane_cell) {
      s = start[cell0 + mycl];
      c = start[cell0 + mycl + 1] - s;
    }
    const float invK = 1.f / (float)P.K;
    for (int ch = 0; ch < nchunks; ++ch) {
      const int o = ch * Kc + lane % Kc;
      bool run = lane_cell && o < P.K && c >= 2;
      if (run && c > a.max_ppc) {
        atomicOr(a.flags, 1);
        run = false;
      }
      if (run)
        ntc_outcome_b(P, c0, (uint32_t)(cell0 + mycl), (uint32_t)o, c, a.v0 + s, a.v1 + s, a.v2 + s, bm, ov,
                      cnt);
      __syncwarp();
      const bool last = ch == nchunks - 1;
      // one transpose per 32-particle word serves every cell of the group
      // (lane l holds outcome l % Kc of cell l / Kc; lanes without
      // collisions hold zero words), as in the single-domain kernel
      const int wmax = (int)__reduce_max_sync(0xffffffffu, (unsigned)((c + 31) / 32));
      const uint32_t kseg = Kc == 32 ? 0xffffffffu : ((1u << Kc) - 1u);
      for (int w = 0; w < wmax; ++w) {
        const uint32_t tw = warp_transpose32(w < a.bm_words ? bm[w] : 0u, lane);
        const int jj = 32 * w + lane;
        for (int cl = 0; cl < ncl; ++cl) {
          const int32_t cs = __shfl_sync(0xffffffffu, s, cl * Kc);
          const int cc = __shfl_sync(0xffffffffu, c, cl * Kc);
          if (jj >= cc) continue;
          uint32_t mine = tw & (kseg << (cl * Kc));
          const int32_t j = cs + jj;
          const float w0 = a.v0[j], w1 = a.v1[j], w2 = a.v2[j];
          float acc0 = 0.f, acc1 = 0.f, acc2 = 0.f;
          if (ch > 0) { acc0 = a.dv0[j]; acc1 = a.dv1[j]; acc2 = a.dv2[j]; }
          while (mine) {
            const int L = __ffs(mine) - 1;
            mine &= mine - 1u;
            const float* W = wov + ((size_t)L * a.max_ppc + jj) * 3;
            acc0 += W[0] - w0;
            acc1 += W[1] - w1;
            acc2 += W[2] - w2;
          }
          if (!last) {
            a.dv0[j] = acc0; a.dv1[j] = acc1; a.dv2[j] = acc2;
          } else {
            const float mx = P.vmean[0] - w0, my = P.vmean[1] - w1, mz = P.vmean[2] - w2;
            const float am = sqrtf(fmaf(mx, mx, fmaf(my, my, mz * mz))) * P.inv_vsig;
            const float f = P.src_pref * (float)(cc - 1) * P.vsig * hs_R_f(P, am);
            a.dv0[j] = fmaf(acc0, invK, -f * mx);
            a.dv1[j] = fmaf(acc1, invK, -f * my);
            a.dv2[j] = fmaf(acc2, invK, -f * mz);
          }
        }
      }
      __syncwarp();
      if (run)
        for (int i = 0; i < (c + 31) / 32; ++i) bm[i] = 0u;
      __syncwarp();
    }
  }
  for (int off = 16; off > 0; off >>= 1) {
    cnt.cand += __shfl_down_sync(0xffffffffu, cnt.cand, off);
    cnt.coll += __shfl_down_sync(0xffffffffu, cnt.coll, off);
    cnt.gmax += __shfl_down_sync(0xffffffffu, cnt.gmax, off);
    cnt.tie += __shfl_down_sync(0xffffffffu, cnt.tie, off);
    cnt.ftie += __shfl_down_sync(0xffffffffu, cnt.ftie, off);
  }
  if (lane == 0) {
    if (cnt.cand) atomicAdd(a.counters + 0, cnt.cand);
    if (cnt.coll) atomicAdd(a.counters + 1, cnt.coll);
    if (cnt.gmax) atomicAdd(a.counters + 2, cnt.gmax);
    if (cnt.tie) atomicAdd(a.counters + 3, cnt.tie);
    if (cnt.ftie) atomicAdd(a.counters + 4, cnt.ftie);
  }
}

// ------------------------------------------------------------ kick/drift --
struct BKickArgs {
  const BatchRep* reps;
  const TimeTerms* tt;  // [R][3]
  int slotE, slotH;     // time slot of the field/E^M and of the drift midpoint
  const uint16_t* rep_of_cell;
  int64_t np;
  int32_t* cell;
  float *o0, *o1, *o2, *v0, *v1, *v2;
  const float *m0, *m1, *m2;
  const uint32_t* pid;
  const float *dv0, *dv1, *dv2;
  const float4* E4;
  float *L0, *L1, *L2;
  int lor_mode;
  int drift;
  int32_t *key, *rank, *count;
};

__global__ void __launch_bounds__(512) kb_kick(BKickArgs a) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= a.np) return;
  const int cg = a.cell[j];
  float o[3] = {a.o0[j], a.o1[j], a.o2[j]};
  float v[3] = {a.v0[j], a.v1[j], a.v2[j]};
  const int r = a.rep_of_cell[cg];
  const BatchRep& B = a.reps[r];
  const ParamsF& P = B.f;
  // replicates without collisions have no DSMC work items: no collision term
  float dv[3] = {0.f, 0.f, 0.f};
  if (a.dv0 && P.K > 0) { dv[0] = a.dv0[j]; dv[1] = a.dv1[j]; dv[2] = a.dv2[j]; }
  const int n = P.n, nn = P.nn;
  const int64_t base = B.coff;
  int ci[3];
  cell_ijk(P, (int)(cg - base), ci);
  float L[3];
  if (a.lor_mode == 2) {
    L[0] = a.L0[j]; L[1] = a.L1[j]; L[2] = a.L2[j];
  } else {
    const int i1 = ci[0] + 1 == n ? 0 : ci[0] + 1, j1 = ci[1] + 1 == n ? 0 : ci[1] + 1,
              k1 = ci[2] + 1 == n ? 0 : ci[2] + 1;
    const int ii[2] = {ci[0], i1}, jj[2] = {ci[1] * n, j1 * n}, kk[2] = {ci[2] * nn, k1 * nn};
    const float wx[2] = {1.f - o[0], o[0]}, wy[2] = {1.f - o[1], o[1]}, wz[2] = {1.f - o[2], o[2]};
    float e0 = 0.f, e1 = 0.f, e2 = 0.f;
#pragma unroll
    for (int cc = 0; cc < 2; ++cc)
#pragma unroll
      for (int b = 0; b < 2; ++b)
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const int64_t node = base + ii[q] + jj[b] + kk[cc];
          const float w = wx[q] * wy[b] * wz[cc];
          const float4 en = __ldg(a.E4 + node);
          e0 = fmaf(w, en.x, e0);
          e1 = fmaf(w, en.y, e1);
          e2 = fmaf(w, en.z, e2);
        }
    const TimeTerms& tE = a.tt[3 * r + a.slotE];
    float s0, c0, s1, c1, s2, c2;
    sincospif(2.f * (((float)ci[0] + o[0]) * P.h - P.phi_shift[0]), &s0, &c0);
    sincospif(2.f * (((float)ci[1] + o[1]) * P.h - P.phi_shift[1]), &s1, &c1);
    sincospif(2.f * (((float)ci[2] + o[2]) * P.h - P.phi_shift[2]), &s2, &c2);
    const float amp = (float)tE.em_amp, k = P.dt_qm;
    L[0] = k * (e0 + amp * c0 * s1 * s2);
    L[1] = k * (e1 + amp * s0 * c1 * s2);
    L[2] = k * (e2 + amp * s0 * s1 * c2);
    if (a.lor_mode == 1) {
      a.L0[j] = L[0]; a.L1[j] = L[1]; a.L2[j] = L[2];
    }
  }
#pragma unroll
  for (int d = 0; d < 3; ++d) v[d] = fmaf(0.5f, L[d] + dv[d], v[d]);
  a.v0[j] = v[0]; a.v1[j] = v[1]; a.v2[j] = v[2];
  if (!a.drift) return;
  const uint32_t p = a.pid[j];
  const float vm[3] = {a.m0[j], a.m1[j], a.m2[j]};
  const TimeTermsF th = to_float_dev(a.tt[3 * r + a.slotH]);
  const U4 b0 = philox(p, 0u, 0u, 0xFFFFFF00u, P.key0, P.key1);
  const U4 b1 = philox(p, 0u, 0u, 0xFFFFFF01u, P.key0, P.key1);
  const float xi[3] = {unif24(b0.x), unif24(b0.z), unif24(b1.x)};
  float* op[3] = {a.o0, a.o1, a.o2};
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const float s = xm_sin_f(P, th, xi[d]);
    const float xd = P.fx_Ac * (s + th.sin2ct) / (1.f + P.fx_amp * s);
    float on = fmaf(P.dtn, v[d] + xd - vm[d], o[d]);
    const float fl = floorf(on);
    on -= fl;
    int shift = (int)fl;
    if (on >= 1.f) { on = 0.f; shift += 1; }
    int cd = (ci[d] + shift) % n;
    ci[d] = cd < 0 ? cd + n : cd;
    op[d][j] = on;
  }
  const int32_t k = (int32_t)(base + ci[0] + n * (ci[1] + n * ci[2]));
  a.key[j] = k;
  a.rank[j] = cell_slot(a.count, k);
}

}  // namespace

// ============================================================== launches ==
cudaError_t launch_batch_sample(pic_ctx* c, const double* xv) {
  BSampleArgs a;
  a.prm = c->prm_dev;
  a.reps = c->reps_dev;
  a.tt = c->tt_dev;
  a.poff = c->poff_dev;
  a.R = c->nrep;
  a.np = c->P.np;
  a.xv = xv;
  const int b = c->cur;
  a.cell = c->cell32[b];
  a.o0 = c->off[b][0]; a.o1 = c->off[b][1]; a.o2 = c->off[b][2];
  a.v0 = c->vf[b][0]; a.v1 = c->vf[b][1]; a.v2 = c->vf[b][2];
  a.m0 = c->vmf[b][0]; a.m1 = c->vmf[b][1]; a.m2 = c->vmf[b][2];
  a.pid = c->pid[b];
  prof_begin(c);
  kb_sample<<<blocks_for(a.np), kThreads, 0, c->stream>>>(a);
  prof_end(c, xv ? KC_OTHER : KC_SAMPLE);
  c->launches++;
  return cudaGetLastError();
}

cudaError_t launch_batch_rhs(pic_ctx* c, int slot) {
  BRhsArgs a;
  a.prm = c->prm_dev;
  a.reps = c->reps_dev;
  a.tt = c->tt_dev;
  a.slot = slot;
  a.rep_of_cell = c->rep_of_cell;
  a.ncell = c->P.ncell;
  a.corner = c->corner;
  a.rho = c->rho;
  a.b32 = c->bf;
  prof_begin(c);
  kb_rhs<<<blocks_for(a.ncell), kThreads, 0, c->stream>>>(a);
  prof_end(c, KC_RHS);
  c->launches++;
  return cudaGetLastError();
}

cudaError_t launch_batch_cg(pic_ctx* c) {
  BCgArgs a;
  a.reps = c->reps_dev;
  a.order = c->cg_order;
  a.R = c->nrep;
  a.b = c->bf;
  a.x = c->phif;
  a.r = c->cgf_r;
  a.p = c->cgf_p;
  a.q = c->cgf_q;
  a.E4 = c->Ef4;
  a.tol = c->cfg.cg_tol;
  a.maxit = c->cfg.cg_maxit;
  a.iters = c->cg_iters_rep;
  a.res = c->cg_res_rep;
  a.flags = c->flags;
  int grid = c->nrep < 4 * c->num_sms ? c->nrep : 4 * c->num_sms;
  prof_begin(c);
  kb_cg<<<grid, kCgThreads, 0, c->stream>>>(a);
  prof_end(c, KC_CG);
  c->launches++;
  return cudaGetLastError();
}

int batch_dsmc_threads() { return kDsmcThreads; }
const void* batch_dsmc_kernel_ptr() { return (const void*)kb_dsmc; }

cudaError_t launch_batch_dsmc(pic_ctx* c, int phase) {
  BDsmcArgs a;
  a.reps = c->reps_dev;
  const int b = c->cur;
  a.v0 = c->vf[b][0]; a.v1 = c->vf[b][1]; a.v2 = c->vf[b][2];
  a.start = c->start;
  a.step = reinterpret_cast<const int64_t*>(c->tt_dev + 3 * c->nrep);
  a.phase = phase;
  a.items = c->dsmc_items;
  a.n_items = c->n_items;
  a.dv0 = c->dvf[0]; a.dv1 = c->dvf[1]; a.dv2 = c->dvf[2];
  a.overlay = c->overlay32;
  a.max_ppc = c->cfg.max_ppc;
  a.bm_words = c->bm_words;
  a.counters = c->counters;
  a.flags = c->flags;
  prof_begin(c);
  kb_dsmc<<<c->dsmc_grid, kDsmcThreads, c->dsmc_smem, c->stream>>>(a);
  prof_end(c, KC_DSMC);
  c->launches++;
  return cudaGetLastError();
}

cudaError_t launch_batch_kick(pic_ctx* c, bool with_coll, bool drift) {
  BKickArgs a;
  a.reps = c->reps_dev;
  a.tt = c->tt_dev;
  a.slotE = drift ? 0 : 2;
  a.slotH = 1;
  a.rep_of_cell = c->rep_of_cell;
  a.np = c->P.np;
  const int b = c->cur;
  a.cell = c->cell32[b];
  a.o0 = c->off[b][0]; a.o1 = c->off[b][1]; a.o2 = c->off[b][2];
  a.v0 = c->vf[b][0]; a.v1 = c->vf[b][1]; a.v2 = c->vf[b][2];
  a.m0 = c->vmf[b][0]; a.m1 = c->vmf[b][1]; a.m2 = c->vmf[b][2];
  a.pid = c->pid[b];
  if (with_coll) { a.dv0 = c->dvf[0]; a.dv1 = c->dvf[1]; a.dv2 = c->dvf[2]; }
  else { a.dv0 = a.dv1 = a.dv2 = nullptr; }
  a.E4 = c->Ef4;
  a.L0 = c->lorf[0]; a.L1 = c->lorf[1]; a.L2 = c->lorf[2];
  a.lor_mode = drift ? (c->lor_valid ? 2 : 0) : 1;
  a.drift = drift ? 1 : 0;
  a.key = c->key;
  a.rank = c->rank;
  a.count = c->count;
  const int t = c->kick_block > 0 ? c->kick_block : kThreads;
  prof_begin(c);
  kb_kick<<<blocks_for(a.np, t), t, 0, c->stream>>>(a);
  prof_end(c, KC_KICK);
  c->launches++;
  c->lor_valid = !drift;
  return cudaGetLastError();
}

}  // namespace pic
