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
//  - CG: a team of blocks per replicate (one per 16,384 nodes, at most 32)
//    meeting at bounded per-replicate barriers, double-float inner products;
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

// RHS of Eq. poisson_mms at node id (global index) of its replicate
__device__ __forceinline__ void rhs_node(const BRhsArgs& a, int64_t id) {
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

__global__ void __launch_bounds__(kThreads) kb_rhs(BRhsArgs a) {
  const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (id < a.ncell) rhs_node(a, id);
}

// -------------------------------------------------------------------- CG --
// The solve's node loops are done by kCgWidth threads of each block in
// every kernel that runs it (the per-phase CG launch and the persistent
// step), so it gives the same bits whatever block size the step was tuned
// to.
constexpr int kCgWidth = 128;
constexpr int kCgThreads = kCgWidth;

struct BCgArgs {
  const BatchRep* reps;
  const int* order;
  int R;
  unsigned* team_bar;     // [R] arrival counters, zero at launch
  double* team_red;       // [R][2][kTeamMax] part totals
  const int2* parts;      // (replicate, part) items of the per-phase solve
  int n_parts;
  int* head;              // their queue head, zero at launch
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

// A replicate's solve is split over a team of T blocks (cg_team_size: one
// per kTeamNodes nodes, at most kTeamMax), part k owning a contiguous node
// range. The team meets at bounded barriers on a per-replicate arrival
// counter (the k-th barrier passes once the counter reaches k T), and its
// inner products are the parts' block totals summed by every part in part
// order, so the iterates do not depend on which block runs which part or
// on the block size. Thread 0 of each part keeps the FP64 scalars.
constexpr long long kTeamWaitCycles = 4000000000LL;  // about 2 s of SM clock

__device__ bool team_barrier(const BCgArgs& a, int rep, int T, int* ok_sh) {
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    if (T > 1) {
      unsigned* bar = a.team_bar + rep;
      __threadfence();
      const unsigned arrived = atomicAdd(bar, 1u) + 1u;
      const unsigned target = (arrived + (unsigned)T - 1u) / (unsigned)T * (unsigned)T;
      const long long t0 = clock64();
      while (*(volatile unsigned*)bar < target) {
        if (clock64() - t0 > kTeamWaitCycles || (((volatile int*)a.flags)[0] & 4)) {
          ok = 0;
          atomicOr(a.flags, 4);
          break;
        }
        __nanosleep(64);
      }
      __threadfence();
    }
    *ok_sh = ok;
  }
  __syncthreads();
  return *ok_sh != 0;
}

// the team total of one double-float partial per thread: valid in thread 0
__device__ __forceinline__ double team_total(const BCgArgs& a, int rep, int part, int T, int slot, DF v, double* sh,
                                             int* ok_sh, bool* ok) {
  const double bt = block_df_total0(v, sh);
  double* red = a.team_red + ((size_t)rep * 2 + slot) * kTeamMax;
  if (threadIdx.x == 0) red[part] = bt;
  if (!team_barrier(a, rep, T, ok_sh)) {
    *ok = false;
    return 0.0;
  }
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int k = 0; k < T; ++k) t += ((volatile double*)red)[k];
  return t;
}

// part `part` of replicate rep's solve by one block (any size up to 1024;
// kCgWidth threads do the node loops, the others only join the barriers
// and contribute zero partials); sh, fsc, stop and ok_sh are the block's
// shared scratch
__device__ void cg_part(const BCgArgs& a, int rep, int part, double* sh, float* fsc, int& stop, int* ok_sh) {
  const BatchRep& B = a.reps[rep];
  const int n = B.f.n, nn = n * n, m = nn * n;
  const int T = cg_team_size(m);
  const int chunk = (m + T - 1) / T;
  const int lo = part * chunk, hi = min(m, lo + chunk);
  const int t0 = threadIdx.x < kCgWidth ? lo + (int)threadIdx.x : INT_MAX;
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
  bool ok = true;
  int slot = 0;
  // zero-mean b
  DF acc{0.f, 0.f};
  for (int id = t0; id < hi; id += kCgWidth) acc = df_add_f(acc, b[id]);
  {
    const double t = team_total(a, rep, part, T, slot, acc, sh, ok_sh, &ok);
    if (!ok) return;
    slot ^= 1;
    if (threadIdx.x == 0) fsc[0] = (float)(t / (double)m);
    __syncthreads();
  }
  const float mean_b = fsc[0];
  DF rr_l{0.f, 0.f}, bb_l{0.f, 0.f};
  for (int id = t0; id < hi; id += kCgWidth) {
    int o[6];
    nbr(id, o);
    const float bv = b[id] - mean_b;
    b[id] = bv;
    const float rv = bv - (6.f * x[id] - (x[o[0]] + x[o[1]] + x[o[2]] + x[o[3]] + x[o[4]] + x[o[5]])) * inv_h2;
    r[id] = rv;
    rr_l = df_fma(rr_l, rv, rv);
    bb_l = df_fma(bb_l, bv, bv);
  }
  double rr = team_total(a, rep, part, T, slot, rr_l, sh, ok_sh, &ok);  // thread 0
  if (!ok) return;
  slot ^= 1;
  const double bb = team_total(a, rep, part, T, slot, bb_l, sh, ok_sh, &ok);
  if (!ok) return;
  slot ^= 1;
  const double thresh = a.tol * sqrt(bb);
  int it = 0, status = 0;
  while (true) {
    if (threadIdx.x == 0) stop = (bb == 0.0 || sqrt(rr) <= thresh) ? 1 : (it >= a.maxit ? 2 : 0);
    __syncthreads();
    if (stop == 1) break;
    if (stop == 2) { status = 1; break; }
    const float beta = fsc[1];
    for (int id = t0; id < hi; id += kCgWidth) p[id] = it == 0 ? r[id] : fmaf(beta, p[id], r[id]);
    if (!team_barrier(a, rep, T, ok_sh)) return;  // the stencil reads the other parts' p
    DF pq_l{0.f, 0.f};
    for (int id = t0; id < hi; id += kCgWidth) {
      int o[6];
      nbr(id, o);
      const float pc = p[id];
      const float qv = (6.f * pc - (p[o[0]] + p[o[1]] + p[o[2]] + p[o[3]] + p[o[4]] + p[o[5]])) * inv_h2;
      q[id] = qv;
      pq_l = df_fma(pq_l, pc, qv);
    }
    {
      const double pq = team_total(a, rep, part, T, slot, pq_l, sh, ok_sh, &ok);
      if (!ok) return;
      slot ^= 1;
      if (threadIdx.x == 0) fsc[0] = (float)(rr / pq);
      __syncthreads();
    }
    const float alpha = fsc[0];
    DF rn_l{0.f, 0.f};
    for (int id = t0; id < hi; id += kCgWidth) {
      x[id] = fmaf(alpha, p[id], x[id]);
      const float rv = fmaf(-alpha, q[id], r[id]);
      r[id] = rv;
      rn_l = df_fma(rn_l, rv, rv);
    }
    const double rr_new = team_total(a, rep, part, T, slot, rn_l, sh, ok_sh, &ok);
    if (!ok) return;
    slot ^= 1;
    ++it;
    if (threadIdx.x == 0) {
      fsc[1] = (float)(rr_new / rr);
      rr = rr_new;
    }
  }
  DF xs{0.f, 0.f};
  for (int id = t0; id < hi; id += kCgWidth) xs = df_add_f(xs, x[id]);
  {
    const double t = team_total(a, rep, part, T, slot, xs, sh, ok_sh, &ok);
    if (!ok) return;
    slot ^= 1;
    if (threadIdx.x == 0) fsc[0] = (float)(t / (double)m);
    __syncthreads();
  }
  const float mean_x = fsc[0];
  for (int id = t0; id < hi; id += kCgWidth) x[id] -= mean_x;
  if (!team_barrier(a, rep, T, ok_sh)) return;  // E reads the other parts' x
  for (int id = t0; id < hi; id += kCgWidth) {
    int o[6];
    nbr(id, o);
    a.E4[B.coff + id] = make_float4(-(x[o[0]] - x[o[1]]) * inv_2h, -(x[o[2]] - x[o[3]]) * inv_2h,
                                    -(x[o[4]] - x[o[5]]) * inv_2h, 0.f);
  }
  if (threadIdx.x == 0 && part == 0) {
    a.iters[rep] = it;
    a.res[rep] = bb > 0.0 ? sqrt(rr) / sqrt(bb) : 0.0;
    if (status) atomicOr(a.flags, 2);
    atomicMax(a.flags + 1, it);
  }
  __syncthreads();
}

// the per-phase solve of every replicate: blocks take (replicate, part)
// items in order from a queue (a team's parts are consecutive, so every
// part a block waits for at a team barrier is taken by a running block)
__global__ void __launch_bounds__(kCgThreads) kb_cg(BCgArgs a) {
  __shared__ double sh[40];
  __shared__ float fsc[2];  // [0] broadcast coefficient (mean, alpha), [1] beta
  __shared__ int stop, item, ok_sh;
  while (true) {
    if (threadIdx.x == 0) item = atomicAdd(a.head, 1);
    __syncthreads();
    const int it = item;
    __syncthreads();
    if (it >= a.n_parts) break;
    const int2 pr = a.parts[it];
    cg_part(a, pr.x, pr.y, sh, fsc, stop, &ok_sh);
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
  // the chi stream: word 0 of slot 0 is the N_pairs uniform, word (s + 1)
  // mod 4 of slot (s + 1) / 4 the chi of candidate s
  U4 bchi = philox<true>(c0, cell, 0u, (o << 8) | 1u, P.key0, P.key1);
  const float base = (float)(((long long)c * (long long)(c - 1)) >> 1) * P.pmax;
  const float S = base + unif24(bchi.x);
  const int npairs = (int)floorf(S);
  // flagged FP32 decisions: the bounds of the single-domain kernel
  if (fabsf(S - rintf(S)) <= fmaf(base + S, 0x1p-22f, 0x1p-24f)) ++cnt.ftie;
  // candidate s: block (c0, cell, s, o << 8) = (p, q, accept, epsilon)
  for (int s = 0; s < npairs; ++s) {
    const U4 b0 = philox<true>(c0, cell, (uint32_t)s, o << 8, P.key0, P.key1);
    const int js = s + 1;
    if ((js & 3) == 0) bchi = philox<true>(c0, cell, (uint32_t)(js >> 2), (o << 8) | 1u, P.key0, P.key1);
    const uint32_t wchi = (js & 3) == 0 ? bchi.x : (js & 3) == 1 ? bchi.y : (js & 3) == 2 ? bchi.z : bchi.w;
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

// One DSMC work item (a group of G cells of replicate item.x from local
// cell item.y) by one warp: Algorithm 1 per (cell, outcome) lane and the
// per-particle averages, as in the single-domain kernel
__device__ void dsmc_group(const BDsmcArgs& a, int2 item, uint32_t c0, int lane, uint32_t* bm, float* wov,
                           float* ov, CountsB& cnt) {
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

__device__ __forceinline__ void dsmc_counts_out(const BDsmcArgs& a, CountsB& cnt, int lane) {
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
  for (int64_t it = gwarp; it < a.n_items; it += nwarps) dsmc_group(a, a.items[it], c0, lane, bm, wov, ov, cnt);
  dsmc_counts_out(a, cnt, lane);
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

// kick (and drift) of particle j in sorted order
__device__ void kick_particle(const BKickArgs& a, int64_t j) {
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

__global__ void __launch_bounds__(512) kb_kick(BKickArgs a) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j < a.np) kick_particle(a, j);
}

// ------------------------------------------------------ persistent step --
// One launch per batched step. The step's work is a queue of items, each a
// (phase, replicate, tile) triple: phase-major, replicates in the order of
// their work (largest first), tiles in index order. A block takes the next
// item from the queue head, waits until the replicate's earlier phases it
// depends on are complete (per-replicate completion counters; the wait is
// bounded and sets the timeout flag when it runs out), does the tile, and
// counts it complete. Every item a block waits for was taken earlier by a
// running block, so the waits end without any assumption about how many
// blocks are resident. Replicates do not share particles, cells or nodes,
// so a replicate's later phases overlap other replicates' earlier ones.
enum BPhase {
  BP_DSMC_A = 0, BP_KICK_DRIFT, BP_SCAN, BP_SCATTER, BP_GATHER, BP_RHS, BP_CG, BP_DSMC_B, BP_KICK_CLOSE, BP_N
};
static_assert(BP_N == kStepPhases, "phase count");

struct BStepArgs {
  BDsmcArgs dA, dB;         // collision calls A (sorted state of step n) and B (after the sort)
  BKickArgs kd, kc;         // drift kick (old buffer) and closing kick (new buffer)
  Gather32Args g;
  BRhsArgs rh;
  BCgArgs cg;
  const BatchRep* reps;
  const int64_t* poff;      // [R + 1] first particle of each replicate
  int64_t ncell_total;
  const int32_t *key, *rank;
  int32_t *count, *start, *perm;
  uint32_t* spid;           // pids in arrival order for the gather (the gather's pid output)
  const int4* items;        // (phase | rep << 8, lo, hi, 0)
  int n_items;
  int* head;                // queue head, zero at launch
  int* done;                // [R][BP_N] completed items, zero at launch
  const int* need;          // [R][BP_N] items per (replicate, phase)
  int* flags;               // [0] bit 4: a bounded wait ran out
  int skip_item;            // failure injection: this item is never counted complete (-1: none)
  int bm_words, max_ppc;
  float* overlay;
};

constexpr long long kStepWaitCycles = 4000000000LL;  // about 2 s of SM clock

// thread 0: wait until every item of (rep, phase) is complete
__device__ __forceinline__ bool wait_phase(const BStepArgs& a, int rep, int phase) {
  const int target = a.need[rep * BP_N + phase];
  const volatile int* d = a.done + rep * BP_N + phase;
  if (*d >= target) return true;
  const long long t0 = clock64();
  while (*d < target) {
    if (clock64() - t0 > kStepWaitCycles) return false;
    if (((volatile int*)a.flags)[0] & 4) return false;  // another wait ran out
    __nanosleep(256);
  }
  return true;
}

// block-level exclusive scan of the replicate's cell counts into the global
// start offsets (its first particle + local prefix), the padding cells
// pointing at the replicate's end; the next replicate's first start, which
// the gather of this replicate's last cell reads, is written too
__device__ void scan_rep(const BStepArgs& a, int rep, int* sh) {
  const BatchRep& B = a.reps[rep];
  const int64_t c0 = B.coff;
  const int64_t c1 = rep + 1 < a.cg.R ? a.reps[rep + 1].coff : a.ncell_total;
  const int nt = blockDim.x, t = threadIdx.x;
  int64_t carry = a.poff[rep];
  for (int64_t base = c0; base < c1; base += nt) {
    const int64_t i = base + t;
    const int v = i < c1 ? a.count[i] : 0;
    // inclusive warp scan, then across the block's warps
    int x = v;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, off);
      if ((t & 31) >= off) x += y;
    }
    if ((t & 31) == 31) sh[t >> 5] = x;
    __syncthreads();
    if (t < 32) {
      int w = t < (nt >> 5) ? sh[t] : 0;
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, w, off);
        if (t >= off) w += y;
      }
      sh[32 + t] = w;  // inclusive over warps
    }
    __syncthreads();
    const int wex = (t >> 5) ? sh[32 + (t >> 5) - 1] : 0;
    if (i < c1) a.start[i] = (int32_t)(carry + wex + x - v);
    const int tot = sh[32 + (nt >> 5) - 1];
    __syncthreads();
    carry += tot;
  }
  if (t == 0) a.start[c1] = (int32_t)a.poff[rep + 1];
}

// resident blocks per SM the register budget is bounded for: about 80
// registers a thread (the collision phase's need), 24 warps per SM
template <int kT>
__global__ void __launch_bounds__(kT, 768 / kT) kb_step(BStepArgs a) {
  extern __shared__ uint32_t smem[];
  __shared__ int item_sh, ok_sh;
  __shared__ double cg_sh[40];
  __shared__ float cg_fsc[2];
  __shared__ int cg_stop, cg_ok;
  __shared__ int scan_sh[64];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, wpb = kT / 32;
  const int64_t gwarp = (int64_t)blockIdx.x * wpb + wib;
  uint32_t* bm = smem + ((size_t)wib * 32 + lane) * a.bm_words;
  float* wov = a.overlay + (size_t)gwarp * 32 * a.max_ppc * 3;
  float* ov = wov + (size_t)lane * a.max_ppc * 3;
  for (int i = 0; i < a.bm_words; ++i) bm[i] = 0u;
  __syncwarp();
  const uint32_t c0A = (uint32_t)(2 * (*a.dA.step)), c0B = c0A + 1u;
  while (true) {
    if (threadIdx.x == 0) {
      const int it = atomicAdd(a.head, 1);
      item_sh = it;
      int ok = 1;
      if (it < a.n_items && !(((volatile int*)a.flags)[0] & 4)) {
        const int4 e = a.items[it];
        const int ph = e.x & 0xFF, rep = e.x >> 8;
        // the phases this one reads the results of
        switch (ph) {
          case BP_KICK_DRIFT: ok = wait_phase(a, rep, BP_DSMC_A); break;
          case BP_SCAN: ok = wait_phase(a, rep, BP_KICK_DRIFT); break;
          case BP_SCATTER: ok = wait_phase(a, rep, BP_SCAN); break;
          case BP_GATHER: ok = wait_phase(a, rep, BP_SCATTER); break;
          case BP_RHS: ok = wait_phase(a, rep, BP_GATHER); break;
          case BP_CG: ok = wait_phase(a, rep, BP_RHS); break;
          case BP_DSMC_B: ok = wait_phase(a, rep, BP_GATHER); break;
          case BP_KICK_CLOSE: ok = wait_phase(a, rep, BP_CG) && wait_phase(a, rep, BP_DSMC_B); break;
          default: break;
        }
        if (!ok) atomicOr(a.flags, 4);
        __threadfence();
      } else if (it < a.n_items) {
        ok = 0;  // a wait ran out: drain the queue without work
      }
      ok_sh = ok;
    }
    __syncthreads();
    const int it = item_sh;
    if (it >= a.n_items) break;
    const int4 e = a.items[it];
    const int ph = e.x & 0xFF, rep = e.x >> 8;
    if (ok_sh) {
      switch (ph) {
        case BP_DSMC_A:
        case BP_DSMC_B: {
          const BDsmcArgs& d = ph == BP_DSMC_A ? a.dA : a.dB;
          // the item's counts leave with the item: no counters stay live
          // across the other phases
          CountsB cnt = {0, 0, 0, 0, 0};
          for (int gi = e.y + wib; gi < e.z; gi += wpb)
            dsmc_group(d, d.items[gi], ph == BP_DSMC_A ? c0A : c0B, lane, bm, wov, ov, cnt);
          dsmc_counts_out(d, cnt, lane);
          break;
        }
        case BP_KICK_DRIFT:
        case BP_KICK_CLOSE: {
          const BKickArgs& k = ph == BP_KICK_DRIFT ? a.kd : a.kc;
          const int64_t p0 = a.poff[rep] + e.y, p1 = a.poff[rep] + e.z;
          for (int64_t j = p0 + threadIdx.x; j < p1; j += kT) kick_particle(k, j);
          break;
        }
        case BP_SCAN: scan_rep(a, rep, scan_sh); break;
        case BP_SCATTER: {
          const int64_t p0 = a.poff[rep] + e.y, p1 = a.poff[rep] + e.z;
          for (int64_t j = p0 + threadIdx.x; j < p1; j += kT) {
            const int32_t slot = a.start[a.key[j]] + a.rank[j];
            a.perm[slot] = (int32_t)j;
            a.spid[slot] = a.g.pid_in[j];
          }
          break;
        }
        case BP_GATHER: {
          const int64_t cbase = a.reps[rep].coff;
          for (int64_t cl = e.y + wib; cl < e.z; cl += wpb) gather_cell32<2>(a.g, cbase + cl, lane);
          break;
        }
        case BP_RHS: {
          const int64_t cbase = a.reps[rep].coff;
          for (int64_t id = e.y + threadIdx.x; id < e.z; id += kT) rhs_node(a.rh, cbase + id);
          break;
        }
        case BP_CG: cg_part(a.cg, rep, e.y, cg_sh, cg_fsc, cg_stop, &cg_ok); break;
        default: break;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0 && it != a.skip_item) {
      __threadfence();
      atomicAdd(a.done + rep * BP_N + ph, 1);
    }
  }
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
  a.team_bar = c->cg_team_bar;
  a.team_red = c->cg_team_red;
  a.parts = c->cg_parts;
  a.n_parts = c->n_cg_parts;
  a.head = c->cg_head;
  cudaError_t e = cudaMemsetAsync(c->cg_team_bar, 0, sizeof(unsigned) * c->nrep, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->cg_head, 0, sizeof(int), c->stream);
  if (e != cudaSuccess) return e;
  // the queue needs at least kTeamMax running blocks; more fill the SMs
  int grid = c->n_cg_parts < 8 * c->num_sms ? c->n_cg_parts : 8 * c->num_sms;
  if (grid < 1) grid = 1;
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


// ------------------------------------------------ persistent step: host --
// Tile shapes of the step's work items (tile configuration t) and the
// block sizes the autotuner tries: every (block, tile) pair is timed on one
// step, and the fastest is captured in the graphs.
const int kStepBlocks[2] = {128, 256};
constexpr int kStepTiles = 2;
struct StepTiles {
  int dsmc_groups_per_warp, kick_particles, gather_cells_per_warp, rhs_nodes;
};
const StepTiles kTiles[kStepTiles] = {{2, 4096, 4, 4096}, {8, 16384, 16, 16384}};

int step_candidates() { return 2 * kStepTiles; }
int step_block_of(int cand) { return kStepBlocks[cand / kStepTiles]; }
int step_tile_of(int cand) { return cand % kStepTiles; }

const void* step_kernel_ptr(int block) {
  return block == 128 ? (const void*)kb_step<128> : (const void*)kb_step<256>;
}

size_t step_smem(const pic_ctx* c, int block) { return (size_t)(block / 32) * 32 * c->bm_words * 4; }

// the work items of one step for candidate cand (phase-major, replicates in
// CG order, tiles in index order) and the items per (replicate, phase)
cudaError_t build_step_items(pic_ctx* c, int cand) {
  const int wpb = step_block_of(cand) / 32;
  const StepTiles& T = kTiles[step_tile_of(cand)];
  const int R = c->nrep;
  int* order = (int*)malloc(sizeof(int) * R);
  int64_t* ditem0 = (int64_t*)malloc(sizeof(int64_t) * (R + 1));
  int* need = (int*)calloc((size_t)R * BP_N, sizeof(int));
  if (!order || !ditem0 || !need) {
    free(order); free(ditem0); free(need);
    return cudaErrorMemoryAllocation;
  }
  cudaError_t e = cudaMemcpy(order, c->cg_order, sizeof(int) * R, cudaMemcpyDeviceToHost);
  // first DSMC work item of each replicate (the static list is in replicate order)
  int64_t k = 0;
  for (int r = 0; r < R; ++r) {
    ditem0[r] = k;
    const BatchRep& B = c->reps_host[r];
    if (B.f.K > 0) k += (B.f.ncell + B.G - 1) / B.G;
  }
  ditem0[R] = k;
  // count, then fill
  int64_t n = 0;
  for (int pass = 0; pass < 2 && e == cudaSuccess; ++pass) {
    int4* out = pass == 1 ? c->step_items_host : nullptr;
    n = 0;
    auto add = [&](int ph, int r, int64_t lo, int64_t hi) {
      if (out) out[n] = make_int4(ph | (r << 8), (int)lo, (int)hi, 0);
      ++n;
      if (!out) ++need[r * BP_N + ph];
    };
    for (int ph = 0; ph < BP_N; ++ph)
      for (int oi = 0; oi < R; ++oi) {
        const int r = order[oi];
        const BatchRep& B = c->reps_host[r];
        const int64_t np = c->prm_host[r].np, nc = B.f.ncell;
        switch (ph) {
          case BP_DSMC_A:
          case BP_DSMC_B: {
            const int64_t per = (int64_t)T.dsmc_groups_per_warp * wpb;
            for (int64_t g = ditem0[r]; g < ditem0[r + 1]; g += per)
              add(ph, r, g, g + per < ditem0[r + 1] ? g + per : ditem0[r + 1]);
            break;
          }
          case BP_KICK_DRIFT:
          case BP_KICK_CLOSE:
          case BP_SCATTER:
            for (int64_t j = 0; j < np; j += T.kick_particles)
              add(ph, r, j, j + T.kick_particles < np ? j + T.kick_particles : np);
            break;
          case BP_GATHER: {
            const int64_t per = (int64_t)T.gather_cells_per_warp * wpb;
            for (int64_t i = 0; i < nc; i += per) add(ph, r, i, i + per < nc ? i + per : nc);
            break;
          }
          case BP_RHS:
            for (int64_t i = 0; i < nc; i += T.rhs_nodes) add(ph, r, i, i + T.rhs_nodes < nc ? i + T.rhs_nodes : nc);
            break;
          case BP_CG: {
            const int T = cg_team_size((int)nc);  // the solve's team: consecutive items
            for (int k = 0; k < T; ++k) add(ph, r, k, T);
            break;
          }
          default:
            add(ph, r, 0, 1);  // scan: one item per replicate
        }
      }
    if (pass == 0) {
      if (n > c->step_items_cap) {
        free(c->step_items_host);
        c->step_items_host = (int4*)malloc(sizeof(int4) * n);
        dev_free_ctx(c, c->step_items);
        c->step_items = (int4*)ctx_alloc(c, sizeof(int4) * n);
        c->step_items_cap = (c->step_items_host && c->step_items) ? n : 0;
        if (!c->step_items_cap) e = cudaErrorMemoryAllocation;
      }
    }
  }
  if (e == cudaSuccess) e = cudaMemcpy(c->step_items, c->step_items_host, sizeof(int4) * n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(c->step_need, need, sizeof(int) * R * BP_N, cudaMemcpyHostToDevice);
  // the first drift-kick item of the first replicate in CG order: the one a
  // stall injection leaves uncounted
  int64_t skip = 0;
  for (int ph = 0; ph < BP_KICK_DRIFT; ++ph)
    for (int r = 0; r < R; ++r) skip += need[r * BP_N + ph];
  c->step_stall_item = (int)skip;
  c->n_step_items = (int)n;
  c->step_cand = cand;
  free(order); free(ditem0); free(need);
  return e;
}

cudaError_t launch_batch_step(pic_ctx* c, bool coll, bool stall) {
  BStepArgs a;
  const int b = c->cur, o = 1 - c->cur;
  const int block = step_block_of(c->step_cand);
  // collisions: call A on the sorted state of step n, call B on the new order
  for (int ph = 0; ph < 2; ++ph) {
    BDsmcArgs& d = ph == 0 ? a.dA : a.dB;
    const int bb = ph == 0 ? b : o;
    d.reps = c->reps_dev;
    d.v0 = c->vf[bb][0]; d.v1 = c->vf[bb][1]; d.v2 = c->vf[bb][2];
    d.start = c->start;
    d.step = reinterpret_cast<const int64_t*>(c->tt_dev + 3 * c->nrep);
    d.phase = ph;
    d.items = c->dsmc_items;
    d.n_items = c->n_items;
    d.dv0 = c->dvf[0]; d.dv1 = c->dvf[1]; d.dv2 = c->dvf[2];
    d.overlay = c->overlay32;
    d.max_ppc = c->cfg.max_ppc;
    d.bm_words = c->bm_words;
    d.counters = c->counters;
    d.flags = c->flags;
  }
  for (int ph = 0; ph < 2; ++ph) {
    BKickArgs& k = ph == 0 ? a.kd : a.kc;
    const int bb = ph == 0 ? b : o;
    k.reps = c->reps_dev;
    k.tt = c->tt_dev;
    k.slotE = ph == 0 ? 0 : 2;
    k.slotH = 1;
    k.rep_of_cell = c->rep_of_cell;
    k.np = c->P.np;
    k.cell = c->cell32[bb];
    k.o0 = c->off[bb][0]; k.o1 = c->off[bb][1]; k.o2 = c->off[bb][2];
    k.v0 = c->vf[bb][0]; k.v1 = c->vf[bb][1]; k.v2 = c->vf[bb][2];
    k.m0 = c->vmf[bb][0]; k.m1 = c->vmf[bb][1]; k.m2 = c->vmf[bb][2];
    k.pid = c->pid[bb];
    if (coll) { k.dv0 = c->dvf[0]; k.dv1 = c->dvf[1]; k.dv2 = c->dvf[2]; }
    else { k.dv0 = k.dv1 = k.dv2 = nullptr; }
    k.E4 = c->Ef4;
    k.L0 = c->lorf[0]; k.L1 = c->lorf[1]; k.L2 = c->lorf[2];
    k.lor_mode = ph == 0 ? (c->lor_valid ? 2 : 0) : 1;
    k.drift = ph == 0 ? 1 : 0;
    k.key = c->key;
    k.rank = c->rank;
    k.count = c->count;
  }
  Gather32Args& g = a.g;
  g.n = c->P.n;
  g.ncell = c->P.ncell;
  g.start = c->start;
  g.perm = c->perm;
  for (int d = 0; d < 3; ++d) {
    g.in[d] = c->off[b][d]; g.in[3 + d] = c->vf[b][d]; g.in[6 + d] = c->vmf[b][d];
    g.out[d] = c->off[o][d]; g.out[3 + d] = c->vf[o][d]; g.out[6 + d] = c->vmf[o][d];
  }
  g.pid_in = c->pid[b];
  g.pid_out = c->pid[o];
  g.cell_out = c->cell32[o];
  g.corner = c->corner;
  g.big_lo = INT_MAX;  // every cell by its warp (no block sort inside the step)
  g.spid = c->pid[o];  // written in arrival order by the scatter phase
  a.rh.prm = c->prm_dev;
  a.rh.reps = c->reps_dev;
  a.rh.tt = c->tt_dev;
  a.rh.slot = 2;
  a.rh.rep_of_cell = c->rep_of_cell;
  a.rh.ncell = c->P.ncell;
  a.rh.corner = c->corner;
  a.rh.rho = c->rho;
  a.rh.b32 = c->bf;
  a.cg.reps = c->reps_dev;
  a.cg.order = c->cg_order;
  a.cg.R = c->nrep;
  a.cg.b = c->bf;
  a.cg.x = c->phif;
  a.cg.r = c->cgf_r;
  a.cg.p = c->cgf_p;
  a.cg.q = c->cgf_q;
  a.cg.E4 = c->Ef4;
  a.cg.tol = c->cfg.cg_tol;
  a.cg.maxit = c->cfg.cg_maxit;
  a.cg.iters = c->cg_iters_rep;
  a.cg.res = c->cg_res_rep;
  a.cg.flags = c->flags;
  a.cg.team_bar = c->cg_team_bar;
  a.cg.team_red = c->cg_team_red;
  a.cg.parts = nullptr;
  a.cg.n_parts = 0;
  a.cg.head = nullptr;
  a.reps = c->reps_dev;
  a.poff = c->poff_dev;
  a.ncell_total = c->P.ncell;
  a.key = c->key;
  a.rank = c->rank;
  a.count = c->count;
  a.start = c->start;
  a.perm = c->perm;
  a.spid = c->pid[o];
  a.items = c->step_items;
  a.n_items = c->n_step_items;
  a.head = c->step_sync;
  a.done = c->step_sync + 1;
  a.need = c->step_need;
  a.flags = c->flags;
  a.skip_item = stall ? c->step_stall_item : -1;
  a.bm_words = c->bm_words;
  a.max_ppc = c->cfg.max_ppc;
  a.overlay = c->overlay32;
  cudaError_t e = cudaMemsetAsync(c->step_sync, 0, sizeof(int) * (1 + (size_t)c->nrep * BP_N), c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->count, 0, (size_t)c->P.ncell * 4, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->cg_team_bar, 0, sizeof(unsigned) * c->nrep, c->stream);
  if (e != cudaSuccess) return e;
  const size_t smem = step_smem(c, block);
  prof_begin(c);
  if (block == 128)
    kb_step<128><<<c->step_grid[0], 128, smem, c->stream>>>(a);
  else
    kb_step<256><<<c->step_grid[1], 256, smem, c->stream>>>(a);
  prof_end(c, KC_OTHER);
  c->launches++;
  c->cur = o;
  c->lor_valid = true;
  return cudaGetLastError();
}
}  // namespace pic
