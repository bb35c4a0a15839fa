// Precision form (PIC_MIXED) of the step. Particle state per particle:
// int32 cell, FP32 offset inside the cell in cell units [0,1)^3, FP32
// velocity, FP32 v^M and the pid; velocities, field gather, manufactured
// terms and scattering are FP32. Kept FP64-accurate: the per-cell charge
// sums, the CG inner products and residual, and the error norms. On this
// GPU the FP64 pipe runs at 1/74 of the FP32 FMA rate, so the charge sums
// are exact 64-bit fixed point and the CG's inner products are formed in
// double-float arithmetic (an unevaluated sum hi + lo of two floats,
// error-free TwoSum / TwoProd of Knuth and Dekker, relative error about
// 2^-44) on the FP32 pipe, within and across blocks; the CG's scalar
// recurrences and the error norms are true FP64.
#include "mixed_common.cuh"

namespace pic {
namespace {

constexpr int kThreads = 256;

inline int blocks_for(int64_t n, int t = kThreads) {
  int64_t b = (n + t - 1) / t;
  return (int)(b < 1 ? 1 : b);
}

// --------------------------------------------------------------- sampling --
struct Sample32Args {
  Params P;
  TimeTerms tt;
  int64_t row0, row_end;  // the particles (pids) this launch takes
  const double *xs, *vs;  // optional caller state (pid order, [N][3] each; device or mapped host)
  // optional v^M (tau for the paper's f_v) to keep: a context's sorted
  // arrays, read for pid i at vslot[i] (the inverse sort permutation)
  const int32_t* vslot;
  const float *vin0, *vin1, *vin2;
  // optional: the state as 48-byte records in pid order (o0 o1 o2 v0 | v1 v2
  // m0 m1 | m2 cell pid -) with its cell keys and in-cell arrival ranks,
  // instead of the structure-of-arrays buffers (a state load followed by
  // the sort: its gather reads the records at random)
  float4* rec = nullptr;
  int32_t *key = nullptr, *rank = nullptr, *count = nullptr;
  // optional, with rec: the records also binned by cell ([ncell][bin_cap],
  // arrival rank r at slot r); a rank at or above bin_cap sets *bin_over
  float4* bins = nullptr;
  int64_t bin_cap = 0;
  int* bin_over = nullptr;
  int32_t* cell;
  float *o0, *o1, *o2, *v0, *v1, *v2, *m0, *m1, *m2;
  uint32_t* pid;
};

// A caller's state ([N][3] rows, in place in pinned host memory over
// NVLink-C2C or in device memory) is read by the block in contiguous spans
// into shared memory (16-byte loads where the rows allow), so each byte
// crosses the link once; a thread's three components are then three
// shared-memory reads.
__global__ void __launch_bounds__(kThreads) k_sample32(Sample32Args a) {
  __shared__ __align__(16) double sxs[3 * kThreads], svs[3 * kThreads];
  const int64_t base = a.row0 + (int64_t)blockIdx.x * kThreads;
  const int64_t i = base + threadIdx.x;
  const Params& P = a.P;
  if (a.xs) {
    const int64_t rows = a.row_end - base < kThreads ? a.row_end - base : kThreads;
    const double* gx = a.xs + 3 * base;
    const double* gv = a.vs + 3 * base;
    if (rows == kThreads && ((reinterpret_cast<uintptr_t>(gx) | reinterpret_cast<uintptr_t>(gv)) & 15) == 0) {
      for (int k = threadIdx.x; k < 3 * kThreads / 2; k += kThreads) {
        reinterpret_cast<double2*>(sxs)[k] = reinterpret_cast<const double2*>(gx)[k];
        reinterpret_cast<double2*>(svs)[k] = reinterpret_cast<const double2*>(gv)[k];
      }
    } else {
      for (int64_t k = threadIdx.x; k < 3 * rows; k += kThreads) {
        sxs[k] = gx[k];
        svs[k] = gv[k];
      }
    }
    __syncthreads();
  }
  if (i >= a.row_end) return;
  double xi[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  const bool given_vm = a.vslot != nullptr;
  const int32_t vj = given_vm ? a.vslot[i] : 0;
  if (!a.xs || !given_vm) {
    const U4 b0 = sample_block(P, (uint64_t)i, 0), b1 = sample_block(P, (uint64_t)i, 1),
             b2 = sample_block(P, (uint64_t)i, 2);
    xi[0] = unif52(b0.x, b0.y); xi[1] = unif52(b0.z, b0.w); xi[2] = unif52(b1.x, b1.y);
    xi[3] = unif52(b1.z, b1.w); xi[4] = unif52(b2.x, b2.y); xi[5] = unif52(b2.z, b2.w);
  }
  const float* vin[3] = {a.vin0, a.vin1, a.vin2};
  double x[3], v[3], vm[3];
  const bool paper = P.dist == PIC_DIST_PAPER;
  for (int d = 0; d < 3; ++d) {
    double s, cc;
    // the paper's f_v: the v^M array holds tau, v^M(t) = vh(t) tau; a state
    // loaded into a context that already holds one keeps its v^M values
    if (given_vm)
      vm[d] = (double)vin[d][vj];
    else
      vm[d] = paper ? tau_inv(xi[3 + d]) : P.vmean[d] + P.vsig * normcdfinv(xi[3 + d]);
    if (a.xs) {
      x[d] = sxs[3 * threadIdx.x + d];
      v[d] = svs[3 * threadIdx.x + d];
    } else if (paper) {
      x[d] = wrap_unit(xm_solve_gen(a.tt, d, xi[d], &s, &cc));
      v[d] = vm[d] * a.tt.vh[d];
    } else {
      x[d] = wrap_unit(xm_solve(P, a.tt, xi[d], &s));
      v[d] = vm[d];
    }
  }
  const int n = P.n;
  int ci[3];
  float off[3];
  for (int d = 0; d < 3; ++d) {
    ci[d] = cell_coord(x[d], n);
    float o = (float)(x[d] * (double)n - (double)ci[d]);
    off[d] = o >= 1.f ? 0x1.fffffep-1f : (o < 0.f ? 0.f : o);
  }
  const int32_t cell = ci[0] + n * (ci[1] + n * ci[2]);
  if (a.rec) {
    const float4 r0 = make_float4(off[0], off[1], off[2], (float)v[0]);
    const float4 r1 = make_float4((float)v[1], (float)v[2], (float)vm[0], (float)vm[1]);
    const float4 r2 = make_float4((float)vm[2], __int_as_float(cell), __uint_as_float((uint32_t)i), 0.f);
    float4* r = a.rec + 3 * i;
    r[0] = r0; r[1] = r1; r[2] = r2;
    a.key[i] = cell;
    const int32_t rk = cell_slot(a.count, cell);
    a.rank[i] = rk;
    if (a.bins) {
      // random 48-byte stores into HBM, while the load itself waits on the
      // host link
      if (rk < a.bin_cap) {
        float4* q = a.bins + 3 * ((int64_t)cell * a.bin_cap + rk);
        q[0] = r0; q[1] = r1; q[2] = r2;
      } else {
        *a.bin_over = 1;
      }
    }
    return;
  }
  a.cell[i] = cell;
  a.o0[i] = off[0]; a.o1[i] = off[1]; a.o2[i] = off[2];
  a.v0[i] = (float)v[0]; a.v1[i] = (float)v[1]; a.v2[i] = (float)v[2];
  a.m0[i] = (float)vm[0]; a.m1[i] = (float)vm[1]; a.m2[i] = (float)vm[2];
  a.pid[i] = (uint32_t)i;
}

struct Keys32Args {
  int64_t np;
  const int32_t* cell;
  int32_t *key, *rank, *count;
};

__global__ void __launch_bounds__(kThreads) k_keys32(Keys32Args a) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= a.np) return;
  const int32_t k = a.cell[j];
  a.key[j] = k;
  a.rank[j] = cell_slot(a.count, k);
}

struct Store32Args {
  int64_t np;
  int n;
  double h;
  int64_t cell_base;  // subtracted from the stored cell (batches)
  const int32_t* cell;
  const float *o0, *o1, *o2, *v0, *v1, *v2;
  const uint32_t* pid;
  double* xv;
  int32_t* cell_of_pid;
};

__global__ void __launch_bounds__(kThreads) k_store_state32(Store32Args a) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= a.np) return;
  const int64_t p = a.pid[j];
  const int n = a.n, c = (int)(a.cell[j] - a.cell_base);
  if (a.cell_of_pid) a.cell_of_pid[p] = c;
  if (!a.xv) return;
  const int ci = c % n, cj = (c / n) % n, ck = c / (n * n);
  a.xv[3 * p] = ((double)ci + (double)a.o0[j]) * a.h;
  a.xv[3 * p + 1] = ((double)cj + (double)a.o1[j]) * a.h;
  a.xv[3 * p + 2] = ((double)ck + (double)a.o2[j]) * a.h;
  double* vs = a.xv + 3 * a.np;
  vs[3 * p] = a.v0[j]; vs[3 * p + 1] = a.v1[j]; vs[3 * p + 2] = a.v2[j];
}

// Inverse of the sort permutation: the slot of every pid, in passes over
// windows of kInvWindow pids. Each pass streams every pid and writes only
// the slots of its window, so its random 4-byte stores land in a span L2
// holds (64 MB) and reach HBM as whole sectors; one pass over all pids
// scattered its stores over the whole array.
constexpr int64_t kInvWindow = int64_t(1) << 24;

struct InvPerm32Args {
  int64_t np;
  const uint32_t* pid;
  int32_t* slot;
  int64_t lo, hi;  // the pass's window of pids
};

// One thread per pid: the fastest pass on its own.
__global__ void __launch_bounds__(kThreads) k_inv_perm32(InvPerm32Args a) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= a.np) return;
  const int64_t p = (int64_t)__ldcs(a.pid + j);
  if (p >= a.lo && p < a.hi) a.slot[p] = (int32_t)j;
}

// Grid-stride, four independent loads a thread in flight, for a small grid
// that leaves the SMs to a kernel running beside it.
__global__ void __launch_bounds__(kThreads) k_inv_perm32_gs(InvPerm32Args a) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t j0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j0 < a.np; j0 += 4 * stride) {
    int64_t p[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int64_t j = j0 + u * stride;
      p[u] = j < a.np ? (int64_t)__ldcs(a.pid + j) : -1;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (p[u] >= a.lo && p[u] < a.hi) a.slot[p[u]] = (int32_t)(j0 + u * stride);
  }
}

// The state in pid order for a destination the kernel writes in place
// (device memory, or pinned host memory reached over NVLink-C2C): each
// thread gathers one pid through the inverse permutation, the block's rows
// go through shared memory, and the stores cover contiguous spans. Same
// arithmetic as k_store_state32. Rows row0 .. row_end - 1.
struct StoreByPid32Args {
  int64_t row0, row_end;
  int n;
  double h;
  const int32_t *slot, *cell;
  const float *o0, *o1, *o2, *v0, *v1, *v2;
  double *x, *v;
};

__global__ void __launch_bounds__(kThreads) k_store_state32_by_pid(StoreByPid32Args a) {
  __shared__ __align__(16) double sx[3 * kThreads], sv[3 * kThreads];
  const int64_t base = a.row0 + (int64_t)blockIdx.x * kThreads;
  const int t = threadIdx.x;
  if (base + t < a.row_end) {
    const int64_t j = a.slot[base + t];
    const int n = a.n, c = a.cell[j];
    const int ci = c % n, cj = (c / n) % n, ck = c / (n * n);
    sx[3 * t] = ((double)ci + (double)a.o0[j]) * a.h;
    sx[3 * t + 1] = ((double)cj + (double)a.o1[j]) * a.h;
    sx[3 * t + 2] = ((double)ck + (double)a.o2[j]) * a.h;
    sv[3 * t] = a.v0[j]; sv[3 * t + 1] = a.v1[j]; sv[3 * t + 2] = a.v2[j];
  }
  __syncthreads();
  const int64_t rows = a.row_end - base < kThreads ? a.row_end - base : kThreads;
  double* gx = a.x + 3 * base;
  double* gv = a.v + 3 * base;
  if (rows == kThreads && ((reinterpret_cast<uintptr_t>(gx) | reinterpret_cast<uintptr_t>(gv)) & 15) == 0) {
    for (int k = t; k < 3 * kThreads / 2; k += kThreads) {
      reinterpret_cast<double2*>(gx)[k] = reinterpret_cast<const double2*>(sx)[k];
      reinterpret_cast<double2*>(gv)[k] = reinterpret_cast<const double2*>(sv)[k];
    }
  } else {
    for (int64_t k = t; k < 3 * rows; k += kThreads) {
      gx[k] = sx[k];
      gv[k] = sv[k];
    }
  }
}

constexpr int kGatherThreads = 128;

template <bool kRec>
__global__ void __launch_bounds__(kGatherThreads) k_sort_gather32(Gather32Args a) {
  const int lane = threadIdx.x & 31;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t cell = gw; cell < a.ncell; cell += nw) gather_cell32<4, kRec>(a, cell, lane);
}

// Cells of kBigCell < count <= kMaxBlockSort particles: one block per cell,
// shared-memory bitonic sort by pid, double-float CIC partials reduced in a
// fixed block order.
constexpr int kBigThreads = 512;

__global__ void __launch_bounds__(kBigThreads) k_sort_big32(Gather32Args a) {
  extern __shared__ uint32_t shm[];
  uint32_t* key = shm;
  int32_t* val = reinterpret_cast<int32_t*>(shm + kMaxBlockSort);
  __shared__ long long red[kBigThreads / 32][8];
  for (int64_t cell = blockIdx.x; cell < a.ncell; cell += gridDim.x) {
    const int32_t s = a.start[cell];
    const int32_t cnt = a.start[cell + 1] - s;
    if (cnt <= a.big_lo || cnt > kMaxBlockSort) continue;  // uniform per block
    int np2 = 1;
    while (np2 < cnt) np2 <<= 1;
    for (int e = threadIdx.x; e < np2; e += blockDim.x) {
      if (e < cnt) {
        // never binned: a binned load holds no cell above its bin, which
        // is at most kBigCell
        const int32_t src = a.perm[s + e];
        key[e] = a.rec ? gather_pid32<true>(a, a.rec, src) : gather_pid32<false>(a, a.rec, src);
        val[e] = src;
      } else {
        key[e] = 0xFFFFFFFFu;
        val[e] = -1;
      }
    }
    __syncthreads();
    block_bitonic_sort(key, val, np2);
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
      const int32_t src = val[e], dst = s + e;
      float d[9];
      if (a.rec) gather_load32<true>(a, a.rec, src, d);
      else gather_load32<false>(a, a.rec, src, d);
#pragma unroll
      for (int q = 0; q < 9; ++q) a.out[q][dst] = d[q];
      a.pid_out[dst] = key[e];
      a.cell_out[dst] = (int32_t)cell;
    }
    __syncthreads();
    long long acc[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) acc[q] = 0;
    const CicFixed fx = cic_fixed_for(cnt);
    for (int e = threadIdx.x; e < cnt; e += blockDim.x)
      cic_add_fixed(acc, a.out[0][s + e], a.out[1][s + e], a.out[2][s + e], fx);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) acc[q] += shfl_xor_ll(acc[q], off);
      if (lane == 0) red[w][q] = acc[q];
    }
    __syncthreads();
    if (threadIdx.x < 8) {
      long long t = 0;
      for (int ww = 0; ww < (int)(blockDim.x >> 5); ++ww) t += red[ww][threadIdx.x];
      a.corner[(int64_t)threadIdx.x * a.ncell + cell] = (double)t * fx.inv;
    }
    __syncthreads();
  }
}

// ----------------------------------------------------------- collisions --
struct Dsmc32Args {
  ParamsF P;
  const float *v0, *v1, *v2;
  const int32_t* start;
  uint32_t c0;
  float *dv0, *dv1, *dv2;  // out: v + (<dv> - <dv^M>)/2, or <dv> when m0 != nullptr
  float *m0, *m1, *m2;     // out (optional): <dv^M>
  float* overlay;
  int max_ppc, bm_words, G, Kc, nchunks;
  int64_t ngroups;
  unsigned long long* counters;
  unsigned long long* queue;  // next cell group to take (zero at launch)
  int chunk;                  // cell groups a warp takes from the queue at a time
  int* flags;
  float vh[3];             // PIC_DIST_PAPER: f_v scales at the call's time
  DLog lg;                 // decision log (mode 0: off)
  long long* hist;         // per-step history row: [1] candidates, [2] collisions, [3] g > g_max
};

struct Counts32 {
  unsigned long long cand, coll, gmax, tie, ftie;
};

// The working velocities of a (cell, outcome) lane: the cell's velocities,
// except for the particles this outcome has changed (their bits are set in
// the lane's bitmap). The first kList changed particles keep their working
// velocity in a list in shared memory (entry k of lane l at list[32 k + l]:
// x, y, z and the in-cell index as w), any further ones in the lane's
// particle-indexed overlay in global memory; at these collision rates an
// outcome changes a few particles, so the overlay is almost never touched.
constexpr int kList = 4;

// position k < t of particle p in a lane's list, or -1
__device__ __forceinline__ int wl_find(const float4* wl, int t, int p) {
  int k = -1;
#pragma unroll
  for (int i = 0; i < kList; ++i)
    if (i < t && __float_as_int(wl[32 * i].w) == p) k = i;
  return k;
}

__device__ __forceinline__ void vel_get(int p, const uint32_t* bm, const float4* wl, int t, const float* ov,
                                        const float* v0, const float* v1, const float* v2, float* o) {
  if ((bm[p >> 5] >> (p & 31)) & 1u) {
    const int k = wl_find(wl, t, p);
    if (k >= 0) {
      const float4 e = wl[32 * k];
      o[0] = e.x; o[1] = e.y; o[2] = e.z;
    } else {
      o[0] = ov[3 * p]; o[1] = ov[3 * p + 1]; o[2] = ov[3 * p + 2];
    }
  } else {
    o[0] = v0[p]; o[1] = v1[p]; o[2] = v2[p];
  }
}

__device__ __forceinline__ void vel_put(int p, const float* v, uint32_t* bm, float4* wl, int& t, float* ov) {
  const uint32_t bit = 1u << (p & 31);
  if (bm[p >> 5] & bit) {
    const int k = wl_find(wl, t, p);
    if (k >= 0) {
      wl[32 * k] = make_float4(v[0], v[1], v[2], __int_as_float(p));
      return;
    }
  } else {
    bm[p >> 5] |= bit;
    if (t < kList) {
      wl[32 * t] = make_float4(v[0], v[1], v[2], __int_as_float(p));
      ++t;
      return;
    }
  }
  ov[3 * p] = v[0]; ov[3 * p + 1] = v[1]; ov[3 * p + 2] = v[2];
}

// Decisions the FP32 arithmetic may take differently from an FP64
// evaluation of the same draws are counted and, with a decision log, logged:
//  - N_pairs = floor(S), S = base + U: base carries 2^-23 relative error
//    (P_coll,max rounded to FP32, one product), the 24-bit uniform is within
//    2^-25 of the 32-bit one, and the sum rounds by 2^-24 S; S within twice
//    that bound of an integer is flagged;
//  - accept: the 24-bit uniform times g_max is within 2^-25 g_max of the
//    32-bit one's, and g carries the rounding of the FP32 velocities (a few
//    ulp per collision they took part in); |U g_max - g| <= 2^-19 (g_max +
//    U g_max) is flagged (tested on the squares: |(U g_max)^2 - g^2| <=
//    dg (2 U g_max + dg) holds whenever |U g_max - g| <= dg). For the
//    odd-power cross section the same margin is 2^-17 of the compared
//    values.
// Every decision is logged only in the kVerify instantiation.
template <bool kVerify>
__device__ void ntc_outcome_f(const ParamsF& P, uint32_t c0, uint32_t cell, uint32_t o, int c, const float* v0,
                              const float* v1, const float* v2, uint32_t* bm, float4* wl, int& t, float* ov,
                              Counts32& cnt, const DLog& lg) {
  // the chi stream (c0, cell, slot, (o << 8) | 1): word 0 of slot 0 is the
  // N_pairs uniform, word (s + 1) mod 4 of slot (s + 1) / 4 the chi of
  // candidate s
  U4 bchi = philox_rk<true>(c0, cell, 0u, (o << 8) | 1u, P.rk);
  const float base = (float)(((long long)c * (long long)(c - 1)) >> 1) * P.pmax;
  const float S = base + unif24(bchi.x);
  const int npairs = (int)floorf(S);
  const bool ftie = fabsf(S - rintf(S)) <= fmaf(base + S, 0x1p-22f, 0x1p-24f);
  if (ftie) ++cnt.ftie;
  const bool log_all = kVerify && lg.mode == PIC_DLOG_ALL;
  if (log_all || (ftie && lg.mode != PIC_DLOG_OFF))
    dlog_put(lg, c0, cell, o, -1, -1, -1, npairs, PIC_DLOG_NPAIRS | (ftie ? PIC_DLOG_FLOOR : 0));
  const float gmax = P.gmax;
  // candidate s: block (c0, cell, s, o << 8) = (p, q, accept, epsilon). The
  // next candidate's block is formed while this one's velocities load: the
  // draws depend on no velocity.
  U4 bnext{0u, 0u, 0u, 0u};
  if (npairs > 0) bnext = philox_rk<true>(c0, cell, 0u, o << 8, P.rk);
  for (int s = 0; s < npairs; ++s) {
    const U4 b0 = bnext;
    const uint32_t p = draw_index(b0.x, (uint32_t)c);
    // q uniform over the other c - 1 particles: the distribution of
    // drawing again until q != p
    uint32_t q = draw_index(b0.y, (uint32_t)(c - 1));
    q += q >= p ? 1u : 0u;
    float vp[3], vq[3];
    vel_get((int)p, bm, wl, t, ov, v0, v1, v2, vp);
    vel_get((int)q, bm, wl, t, ov, v0, v1, v2, vq);
    const int js = s + 1;
    if ((js & 3) == 0) bchi = philox_rk<true>(c0, cell, (uint32_t)(js >> 2), (o << 8) | 1u, P.rk);
    if (s + 1 < npairs) bnext = philox_rk<true>(c0, cell, (uint32_t)(s + 1), o << 8, P.rk);
    const uint32_t wchi = (js & 3) == 0 ? bchi.x : (js & 3) == 1 ? bchi.y : (js & 3) == 2 ? bchi.z : bchi.w;
    const float dx = vp[0] - vq[0], dy = vp[1] - vq[1], dz = vp[2] - vq[2];
    const float g2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    // accept if U < sigma g / (sigma g)_max: hard spheres g / g_max, i.e.
    // (U g_max)^2 < g^2; odd-power sigma U (sigma g)_max < sum_k sigma_k g^2k
    float lhs, rhs, tol;
    if (P.n_sigma == 0) {
      const float ug = unif24(b0.z) * gmax;
      lhs = ug * ug;
      rhs = g2;
      const float dg = (gmax + ug) * 0x1p-19f;
      tol = dg * fmaf(2.f, ug, dg);
    } else {
      lhs = unif24(b0.z) * P.sgmax;
      rhs = fmaf(fmaf(P.sigma_n[2], g2, P.sigma_n[1]), g2, P.sigma_n[0]);
      tol = (P.sgmax + fabsf(rhs)) * 0x1p-17f;
    }
    ++cnt.cand;
    if (g2 > P.gmax2) ++cnt.gmax;
    const bool tie = fabsf(lhs - rhs) <= tol;
    if (tie) ++cnt.tie;
    if (log_all || (tie && lg.mode != PIC_DLOG_OFF))
      dlog_put(lg, c0, cell, o, s, (int)p, (int)q, lhs < rhs ? 1 : 0, tie ? PIC_DLOG_TIE : 0);
    if (lhs < rhs) {
      const float g = sqrtf(g2);
      float np_[3], nq_[3];
      if (kVerify && (P.verify & PIC_VERIFY_ERROR2)) {
        // injected Error 2: swap with probability 1/2 (coin = chi draw)
        const bool swap = unif24(wchi) < 0.5f;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          np_[d] = swap ? vq[d] : vp[d];
          nq_[d] = swap ? vp[d] : vq[d];
        }
      } else {
        float se, ce;
        sincospif(2.f * unif24(b0.w), &se, &ce);
        float uchi = unif24(wchi);
        if (kVerify && (P.verify & PIC_VERIFY_ANISO)) uchi = aniso_u_f(uchi);
        const float cchi = 1.f - 2.f * uchi;
        const float schi = sqrtf(fmaxf(0.f, 1.f - cchi * cchi));
        const float nv[3] = {ce * schi, se * schi, cchi};
        const bool err1 = kVerify && (P.verify & PIC_VERIFY_ERROR1);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          // Eq. v_cm; injected Error 1 flips the sign of v_q
          const float cm = 0.5f * (err1 ? vp[d] - vq[d] : vp[d] + vq[d]);
          const float hg = 0.5f * g * nv[d];
          np_[d] = cm + hg;
          nq_[d] = cm - hg;
        }
      }
      if (kVerify && P.ang_hist)
        record_angles_f(P.ang_hist, (P.verify & PIC_VERIFY_ANISO) != 0, g, np_[0] - nq_[0], np_[1] - nq_[1],
                        np_[2] - nq_[2]);
      vel_put((int)p, np_, bm, wl, t, ov);
      vel_put((int)q, nq_, bm, wl, t, ov);
      ++cnt.coll;
    }
  }
}

constexpr int kDsmcThreads = 128;
// cell groups a warp takes from the launch's queue at a time, at most: a
// cell's work varies with its particle count, and a static split left the
// SMs idle through the last warps' tails. Launches with few groups per
// warp take fewer at a time, so that every resident warp gets work.
constexpr int kDsmcChunk = 8;

// shared memory of one warp, in 32-bit words: bitmaps, lists, list lengths
__host__ __device__ constexpr size_t dsmc32_smem_words(int bm_words) {
  return (size_t)32 * bm_words + (size_t)kList * 32 * 4 + 32;
}

template <bool kVerify>
__global__ void __launch_bounds__(kDsmcThreads, 6) k_dsmc32(Dsmc32Args a) {
  extern __shared__ uint32_t smem[];
  const ParamsF& P = a.P;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int wpb = blockDim.x >> 5;
  const int64_t gwarp = (int64_t)blockIdx.x * wpb + wib;
  // per warp: the lanes' bitmaps [32][bm_words], their lists [kList][32]
  // and list lengths [32]
  uint32_t* wbm = smem + (size_t)wib * dsmc32_smem_words(a.bm_words);
  uint32_t* bm = wbm + (size_t)lane * a.bm_words;
  float4* wlist = reinterpret_cast<float4*>(wbm + 32 * a.bm_words);
  float4* wl = wlist + lane;
  int* wlen = reinterpret_cast<int*>(wlist + 32 * kList);
  float* wov = a.overlay + (size_t)gwarp * 32 * a.max_ppc * 3;
  float* ov = wov + (size_t)lane * a.max_ppc * 3;
  for (int i = 0; i < a.bm_words; ++i) bm[i] = 0u;
  __syncwarp();
  Counts32 cnt = {0, 0, 0, 0, 0};
  const bool separate = a.m0 != nullptr;
  const float invK = 1.f / (float)P.K;
  const float mu0 = P.vmean[0], mu1 = P.vmean[1], mu2 = P.vmean[2];
  const float vs = P.vsig, ivs = P.inv_vsig, pref = P.src_pref;

  int64_t gbase = 0;
  int gk = a.chunk;
  for (;;) {
    if (gk == a.chunk) {
      unsigned long long q = 0;
      if (lane == 0) q = atomicAdd(a.queue, (unsigned long long)a.chunk);
      gbase = (int64_t)__shfl_sync(0xffffffffu, q, 0);
      gk = 0;
    }
    const int64_t grp = gbase + gk++;
    if (grp >= a.ngroups) break;  // warp-uniform
    const int64_t cell0 = grp * a.G;
    const int ncl = (int)min((int64_t)a.G, P.ncell - cell0);
    const int mycl = lane / a.Kc;
    const bool lane_cell = mycl < ncl;
    int32_t s = 0, c = 0;
    if (lane_cell) {
      s = a.start[cell0 + mycl];
      c = a.start[cell0 + mycl + 1] - s;
    }
    for (int ch = 0; ch < a.nchunks; ++ch) {
      const int o = ch * a.Kc + lane % a.Kc;
      bool run = lane_cell && o < P.K && c >= 2;
      if (run && c > a.max_ppc) {
        atomicOr(a.flags, 1);
        run = false;
      }
      int t = 0;
      if (run)
        ntc_outcome_f<kVerify>(P, a.c0, (uint32_t)(cell0 + mycl), (uint32_t)o, c, a.v0 + s, a.v1 + s, a.v2 + s,
                               bm, wl, t, ov, cnt, a.lg);
      wlen[lane] = t;
      __syncwarp();
      // per 32-particle word: one transpose of the lanes' bitmap words across
      // the warp serves every cell of the group, since lane l holds outcome
      // l % Kc of cell l / Kc: lane b receives, in the Kc-bit segment of cell
      // cl, the outcomes that touched particle 32 w + b of that cell; their
      // changes are then added in ascending outcome order
      const bool last = ch == a.nchunks - 1;
      const int wmax = (int)__reduce_max_sync(0xffffffffu, (unsigned)((c + 31) / 32));
      const uint32_t kseg = a.Kc == 32 ? 0xffffffffu : ((1u << a.Kc) - 1u);
      for (int w = 0; w < wmax; ++w) {
        // lanes without collisions in this word (no cell, outcome beyond K,
        // cell outside 2..max_ppc) hold zero words
        const uint32_t tw = warp_transpose32(w < a.bm_words ? bm[w] : 0u, lane);
        const int jj = 32 * w + lane;
        for (int cl = 0; cl < ncl; ++cl) {
          const int32_t cs = __shfl_sync(0xffffffffu, s, cl * a.Kc);
          const int cc = __shfl_sync(0xffffffffu, c, cl * a.Kc);
          if (jj >= cc) continue;
          uint32_t mine = tw & (kseg << (cl * a.Kc));
          const int32_t j = cs + jj;
          const float w0 = a.v0[j], w1 = a.v1[j], w2 = a.v2[j];
          float acc0 = 0.f, acc1 = 0.f, acc2 = 0.f;
          if (ch > 0) { acc0 = a.dv0[j]; acc1 = a.dv1[j]; acc2 = a.dv2[j]; }
          while (mine) {
            const int L = __ffs(mine) - 1;
            mine &= mine - 1u;
            // lane L's working velocity of particle jj: its list, else its overlay
            const int k = wl_find(wlist + L, wlen[L], jj);
            float W0, W1, W2;
            if (k >= 0) {
              const float4 e = wlist[32 * k + L];
              W0 = e.x; W1 = e.y; W2 = e.z;
            } else {
              const float* W = wov + ((size_t)L * a.max_ppc + jj) * 3;
              W0 = W[0]; W1 = W[1]; W2 = W[2];
            }
            acc0 += W0 - w0;
            acc1 += W1 - w1;
            acc2 += W2 - w2;
          }
          if (!last) {
            a.dv0[j] = acc0; a.dv1[j] = acc1; a.dv2[j] = acc2;
          } else {
            // analytic <Delta v^M> (hard spheres: f m with m = mu - v)
            float sm[3];
            if (P.n_sigma == 0) {
              const float mx = mu0 - w0, my = mu1 - w1, mz = mu2 - w2;
              const float am = sqrtf(fmaf(mx, mx, fmaf(my, my, mz * mz))) * ivs;
              const float f = pref * (float)(cc - 1) * vs * hs_R_f(P, am);
              sm[0] = f * mx; sm[1] = f * my; sm[2] = f * mz;
            } else {
              odd_source_f(P, a.vh, w0, w1, w2, cc, sm);
            }
            if (separate) {
              a.dv0[j] = acc0 * invK; a.dv1[j] = acc1 * invK; a.dv2[j] = acc2 * invK;
              a.m0[j] = sm[0]; a.m1[j] = sm[1]; a.m2[j] = sm[2];
            } else {
              // inside a step: the velocity with this call's half kick of
              // Eq. velocity_verlet applied, v + (<dv> - <dv^M>)/2, so that
              // the kick that follows reads one array instead of two
              a.dv0[j] = fmaf(0.5f, fmaf(acc0, invK, -sm[0]), w0);
              a.dv1[j] = fmaf(0.5f, fmaf(acc1, invK, -sm[1]), w1);
              a.dv2[j] = fmaf(0.5f, fmaf(acc2, invK, -sm[2]), w2);
            }
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
    if (a.hist) {
      if (cnt.cand) atomicAdd((unsigned long long*)a.hist + 1, cnt.cand);
      if (cnt.coll) atomicAdd((unsigned long long*)a.hist + 2, cnt.coll);
      if (cnt.gmax) atomicAdd((unsigned long long*)a.hist + 3, cnt.gmax);
    }
  }
}

// ------------------------------------------------------------ kick/drift --
// The Lorentz term dt q/m (E + E^M) of Eq. velocity_verlet at a particle of
// cell ci with offsets o: E trilinear from the cell's eight corner nodes
// (corner q + 2 b + 4 c at i + q, j + b, k + c), the manufactured field
// analytic. Every kernel that forms the term calls this one function, so a
// stored term and a recomputed one agree bit for bit.
__device__ __forceinline__ void lorentz32(const ParamsF& P, const TimeTermsF& tE, const int* ci, const float* o,
                                          const float4* corner, float* L) {
  const float wx[2] = {1.f - o[0], o[0]}, wy[2] = {1.f - o[1], o[1]}, wz[2] = {1.f - o[2], o[2]};
  float e0 = 0.f, e1 = 0.f, e2 = 0.f;
#pragma unroll
  for (int cc = 0; cc < 2; ++cc)
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const float w = wx[q] * wy[b] * wz[cc];
        const float4 en = corner[q + 2 * b + 4 * cc];
        e0 = fmaf(w, en.x, e0);
        e1 = fmaf(w, en.y, e1);
        e2 = fmaf(w, en.z, e2);
      }
  float s0, c0, s1, c1, s2, c2;
  sincospif(2.f * (((float)ci[0] + o[0]) * P.h - P.phi_shift[0]), &s0, &c0);
  sincospif(2.f * (((float)ci[1] + o[1]) * P.h - P.phi_shift[1]), &s1, &c1);
  sincospif(2.f * (((float)ci[2] + o[2]) * P.h - P.phi_shift[2]), &s2, &c2);
  const float amp = tE.em_amp, k = P.dt_qm;
  L[0] = k * (e0 + amp * c0 * s1 * s2);
  L[1] = k * (e1 + amp * s0 * c1 * s2);
  L[2] = k * (e2 + amp * s0 * s1 * c2);
}

// node index of corner q + 2 b + 4 c of cell ci (periodic)
__device__ __forceinline__ int corner_node(const ParamsF& P, const int* ci, int corner) {
  const int n = P.n;
  const int q = corner & 1, b = (corner >> 1) & 1, cc = corner >> 2;
  const int i = ci[0] + q == n ? 0 : ci[0] + q;
  const int j = ci[1] + b == n ? 0 : ci[1] + b;
  const int k = ci[2] + cc == n ? 0 : ci[2] + cc;
  return i + n * j + P.nn * k;
}

struct Kick32Args {
  ParamsF P;
  const int32_t* cell;
  float *o0, *o1, *o2, *v0, *v1, *v2;
  const float *m0, *m1, *m2;
  const uint32_t* pid;
  const float *dv0, *dv1, *dv2;  // v + (<dv> - <dv^M>)/2 from the collision call, or nullptr: read v
  const float4* E4;
  float *L0, *L1, *L2;
  int lor_mode;  // 0: compute, 1: compute and store, 2: load
  TimeTermsF tE, th;
  TimeTermsF t0, t1;  // t_n, t_{n+1} for the isolated-collision drift
  int drift;
  int32_t *key, *rank, *count;
};

// kMode 0: the plain step; 1: the isolated-collision drift of Sec. 5.4;
// 2: the paper's problem (per-axis x^M solve, vdot^M). Kept apart so that
// the plain kernel keeps its register budget.
constexpr int kKickThreads = 128;  // measured against 256 and 512

template <int kMode>
__global__ void __launch_bounds__(kKickThreads) k_kick32(Kick32Args a) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const ParamsF& P = a.P;
  if (j >= P.np) return;
  const int n = P.n;
  // every independent load first (memory-level parallelism), then the
  // dependent field gather
  const int c = a.cell[j];
  float o[3] = {a.o0[j], a.o1[j], a.o2[j]};
  // with collisions the velocity arrives with the collision half kick
  // applied (the collision kernel's output), else it is read as it is
  float v[3];
  if (a.dv0) { v[0] = a.dv0[j]; v[1] = a.dv1[j]; v[2] = a.dv2[j]; }
  else { v[0] = a.v0[j]; v[1] = a.v1[j]; v[2] = a.v2[j]; }
  const float dv[3] = {0.f, 0.f, 0.f};
  float vm[3] = {0.f, 0.f, 0.f};
  uint32_t p = 0;
  constexpr bool paper = kMode == 2, kIsolate = kMode == 1;
  if (a.drift || paper) { vm[0] = a.m0[j]; vm[1] = a.m1[j]; vm[2] = a.m2[j]; }
  if (a.drift) p = a.pid[j];
  int ci[3];
  cell_ijk(P, c, ci);
  float L[3];
  if (a.lor_mode == 2) {
    L[0] = a.L0[j]; L[1] = a.L1[j]; L[2] = a.L2[j];
  } else {
    float4 corner[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) corner[q] = __ldg(a.E4 + corner_node(P, ci, q));
    lorentz32(P, a.tE, ci, o, corner, L);
    if (a.lor_mode == 1) {
      a.L0[j] = L[0]; a.L1[j] = L[1]; a.L2[j] = L[2];
    }
  }
  if (paper) {
    // v^M arrays hold tau: vdot^M(t) = vh'(t) tau (Eq. velocity_verlet)
#pragma unroll
    for (int d = 0; d < 3; ++d) v[d] = fmaf(0.5f, (L[d] + dv[d]) + P.dt * (vm[d] * a.tE.dvh[d]), v[d]);
  } else {
#pragma unroll
    for (int d = 0; d < 3; ++d) v[d] = fmaf(0.5f, L[d] + dv[d], v[d]);
  }
  a.v0[j] = v[0]; a.v1[j] = v[1]; a.v2[j] = v[2];
  if (!a.drift) return;
  const U4 b0 = philox_rk(p, 0u, 0u, 0xFFFFFF00u, P.rk);
  const U4 b1 = philox_rk(p, 0u, 0u, 0xFFFFFF01u, P.rk);
  const float xi[3] = {unif24(b0.x), unif24(b0.z), unif24(b1.x)};
  float* op[3] = {a.o0, a.o1, a.o2};
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    float on;
    if (paper) {
      float sy, cy;
      xm_sc_gen_f(a.th, d, xi[d], &sy, &cy);
      on = fmaf(P.dtn, v[d] + xm_dot_gen_f(a.th, d, sy, cy) - vm[d] * a.th.vh[d], o[d]);
    } else if (kIsolate) {
      // exact manufactured increment y(t_{n+1}) - y(t_n) + c dt (Sec. 5.4)
      const float dy = xm_y_f(P, a.t1, xi[d]) - xm_y_f(P, a.t0, xi[d]);
      on = fmaf(P.dtn, v[d] - vm[d], o[d]) + P.nf * (dy + P.cdt);
    } else {
      const float s = xm_sin_f(P, a.th, xi[d]);
      const float xd = P.fx_Ac * (s + a.th.sin2ct) / (1.f + P.fx_amp * s);
      on = fmaf(P.dtn, v[d] + xd - vm[d], o[d]);
    }
    const float fl = floorf(on);
    on -= fl;
    int shift = (int)fl;
    if (on >= 1.f) { on = 0.f; shift += 1; }
    // periodic wrap: a mask when n is a power of two (exact for negative
    // shifts in two's complement), else a remainder
    int cd = P.log2n >= 0 ? (ci[d] + shift) & (n - 1) : (ci[d] + shift) % n;
    ci[d] = cd < 0 ? cd + n : cd;
    op[d][j] = on;
  }
  const int32_t k = ci[0] + n * (ci[1] + n * ci[2]);
  a.key[j] = k;
  a.rank[j] = cell_slot(a.count, k);
}

// The closing half kick of a step (Eq. velocity_verlet, second half) by
// cells: one warp per cell of the sorted order loads the cell's eight
// corner values of E once into shared memory, then its lanes take the
// cell's particles. The per-particle arithmetic is k_kick32's (lorentz32),
// and the term is stored for the next step's first half kick.
constexpr int kCloseThreads = 128;

struct Close32Args {
  ParamsF P;
  int64_t ncell;
  const int32_t* start;
  const float *o0, *o1, *o2;
  float *v0, *v1, *v2;
  const float *dv0, *dv1, *dv2;  // v + (<dv> - <dv^M>)/2 from the collision call, or nullptr: read v
  const float *m0, *m1, *m2;     // PIC_DIST_PAPER: tau
  const float4* E4;
  float *L0, *L1, *L2;
  TimeTermsF tE;
};

template <bool kPaper>
__global__ void __launch_bounds__(kCloseThreads) k_close32(Close32Args a) {
  __shared__ float4 sE[kCloseThreads / 32][8];
  const ParamsF& P = a.P;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t cell = gw; cell < a.ncell; cell += nw) {
    const int32_t s = a.start[cell], e = a.start[cell + 1];
    int ci[3];
    cell_ijk(P, (int)cell, ci);
    __syncwarp();  // the previous cell's corners are no longer read
    if (lane < 8) sE[wib][lane] = __ldg(a.E4 + corner_node(P, ci, lane));
    __syncwarp();
    for (int32_t j = s + lane; j < e; j += 32) {
      const float o[3] = {a.o0[j], a.o1[j], a.o2[j]};
      float v[3];
      if (a.dv0) { v[0] = a.dv0[j]; v[1] = a.dv1[j]; v[2] = a.dv2[j]; }
      else { v[0] = a.v0[j]; v[1] = a.v1[j]; v[2] = a.v2[j]; }
      float L[3];
      lorentz32(P, a.tE, ci, o, sE[wib], L);
      a.L0[j] = L[0]; a.L1[j] = L[1]; a.L2[j] = L[2];
      if (kPaper) {
        const float vm[3] = {a.m0[j], a.m1[j], a.m2[j]};
#pragma unroll
        for (int d = 0; d < 3; ++d) v[d] = fmaf(0.5f, (L[d] + 0.f) + P.dt * (vm[d] * a.tE.dvh[d]), v[d]);
      } else {
#pragma unroll
        for (int d = 0; d < 3; ++d) v[d] = fmaf(0.5f, L[d] + 0.f, v[d]);
      }
      a.v0[j] = v[0]; a.v1[j] = v[1]; a.v2[j] = v[2];
    }
  }
}

// ---------------------------------------------------------------- CG32 --
struct Cg32Args {
  int n;
  int log2n;  // log2(n) when n is a power of two, else -1
  int64_t ncell;
  float inv_h2, inv_2h;
  float *b, *x, *r, *p, *q;
  const double* rhs_part;
  int rhs_blocks;
  double* red;
  unsigned int* bar;
  int* info;
  int* flags;
  double* res;
  double tol;
  int maxit;
  float4* E4;  // (Ex, Ey, Ez, 0) per node
  int skip_block = -1;  // failure injection: this block leaves before its first barrier
  long long* hist = nullptr;  // per-step history row: [0] iterations
};

constexpr long long kBarrierCycles = 4000000000LL;

__device__ __forceinline__ bool grid_barrier32(unsigned int* bar, int* info, int* flags) {
  // monotonic arrival counter (zero at launch): the k-th barrier of the
  // launch is passed once the counter reaches k gridDim.x; the wait is
  // bounded, after which the timeout flag is set and every block returns
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned int arrived = atomicAdd(bar, 1u) + 1u;
    const unsigned int target = (arrived + gridDim.x - 1u) / gridDim.x * gridDim.x;
    ok = 1;
    const long long t0 = clock64();
    while (*(volatile unsigned int*)bar < target) {
      if (clock64() - t0 > kBarrierCycles) {
        atomicOr(info + 2, 1);
        atomicOr(flags, 4);
        ok = 0;
        break;
      }
    }
    __threadfence();
    if (ok && *((volatile int*)(info + 2))) ok = 0;
  }
  __syncthreads();
  return ok != 0;
}

// Block and grid totals of double-float partials, in double-float
// arithmetic throughout: each warp sums by shuffles, then warp 0 sums the
// warps' (or the blocks') values the same way, in a fixed order. A serial
// chain of FP64 adds on one thread costs several microseconds per
// iteration on this part's narrow FP64 pipe; FP32 pairs cost a few hundred
// cycles. Results are valid in thread 0.
__device__ __forceinline__ DF warp_total_df(DF v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v = df_add(v, df_shfl_xor(v, off));
  return v;
}

// two block totals at once (sh holds at least 32 float4)
__device__ __forceinline__ void block_total_df2(DF u, DF v, float4* sh, DF* tu, DF* tv) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  u = warp_total_df(u);
  v = warp_total_df(v);
  __syncthreads();  // sh is free
  if (lane == 0) sh[w] = make_float4(u.hi, u.lo, v.hi, v.lo);
  __syncthreads();
  if (w == 0) {
    const float4 e = lane < nw ? sh[lane] : make_float4(0.f, 0.f, 0.f, 0.f);
    const DF a = warp_total_df(DF{e.x, e.y}), b = warp_total_df(DF{e.z, e.w});
    if (lane == 0) {
      *tu = a;
      *tv = b;
    }
  }
}

// a partial published by another block before a grid barrier, read at L2
__device__ __forceinline__ DF ld_partial(const float2* p) {
  float hi, lo;
  asm volatile("ld.relaxed.gpu.global.v2.f32 {%0, %1}, [%2];" : "=f"(hi), "=f"(lo) : "l"(p) : "memory");
  return DF{hi, lo};
}

// totals of two arrays of m block partials, by warp 0
__device__ __forceinline__ void grid_total_df2(const float2* pa, const float2* pb, int m, DF* ta, DF* tb) {
  if (threadIdx.x < 32) {
    DF a{0.f, 0.f}, b{0.f, 0.f};
    for (int i = threadIdx.x; i < m; i += 32) {
      a = df_add(a, ld_partial(pa + i));
      b = df_add(b, ld_partial(pb + i));
    }
    a = warp_total_df(a);
    b = warp_total_df(b);
    if (threadIdx.x == 0) {
      *ta = a;
      *tb = b;
    }
  }
}

// total of FP64 partials (another kernel's), in every thread
__device__ __forceinline__ double grid_total32(const double* part, int m, double* sh) {
  const int lane = threadIdx.x & 31;
  __syncthreads();
  if (threadIdx.x < 32) {
    double s = 0.0;
    for (int i = lane; i < m; i += 32) s += ((volatile const double*)part)[i];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (lane == 0) sh[0] = s;
  }
  __syncthreads();
  return sh[0];
}

struct Nbr {
  int xp, xm, yp, ym, zp, zm;
};
// log2n >= 0: n = 2^log2n, the coordinates by shifts and masks instead of
// integer divisions (the same neighbours)
__device__ __forceinline__ Nbr neighbours(int id, int n, int nn, int log2n) {
  int i, j, k;
  if (log2n >= 0) {
    i = id & (n - 1);
    j = (id >> log2n) & (n - 1);
    k = id >> (2 * log2n);
  } else {
    i = id % n;
    j = (id / n) % n;
    k = id / nn;
  }
  Nbr b;
  b.xp = i == n - 1 ? id - (n - 1) : id + 1;
  b.xm = i == 0 ? id + (n - 1) : id - 1;
  b.yp = j == n - 1 ? id - (n - 1) * n : id + n;
  b.ym = j == 0 ? id + (n - 1) * n : id - n;
  b.zp = k == n - 1 ? id - (n - 1) * nn : id + nn;
  b.zm = k == 0 ? id + (n - 1) * nn : id - nn;
  return b;
}

// FP32 vectors and stencil; inner products and the residual in double-float
// (per thread, across a block and across blocks), the scalar recurrences in
// FP64 on thread 0 of each block. Chronopoulos-Gear form of CG: with
// w = A r and s = A p carried by recurrence, (r, r) and (r, w) come from one
// reduction, so an iteration needs two grid barriers (r complete before
// the stencil; the partial sums published) instead of three. The iterates
// are those of standard CG in exact arithmetic. b's storage holds w once
// the initial residual has been formed.
constexpr int kCgThreads = 1024;

__global__ void __launch_bounds__(kCgThreads) k_cg32(Cg32Args a) {
  __shared__ double sh[1];
  __shared__ float4 sh4[32];
  __shared__ float fscal[2];  // alpha, beta formed once per block by thread 0
  __shared__ int stop;
  // the others then wait for an arrival that never comes, until the bound
  if ((int)blockIdx.x == a.skip_block) return;
  const int n = a.n, nn = a.n * a.n;
  const int m = (int)a.ncell;
  const int stride = gridDim.x * blockDim.x;
  const int t0 = blockIdx.x * blockDim.x + threadIdx.x;
  const int G = gridDim.x;
  int ph = 0;
  // block partials, double-buffered: slot q holds 2 G double-float values
  auto slot = [&](int q) { return reinterpret_cast<float2*>(a.red) + (size_t)q * 2 * G; };
  auto publish = [&](int q, DF u, DF v) {
    if (threadIdx.x == 0) {
      slot(q)[blockIdx.x] = make_float2(u.hi, u.lo);
      slot(q)[G + blockIdx.x] = make_float2(v.hi, v.lo);
    }
  };
  float* const w = a.b;  // reused after the initial residual
  float* const s = a.q;

  const float mean_b = (float)(grid_total32(a.rhs_part, a.rhs_blocks, sh) / (double)m);
  DF rr_loc{0.f, 0.f}, bb_loc{0.f, 0.f};
  for (int id = t0; id < m; id += stride) {
    const Nbr q = neighbours(id, n, nn, a.log2n);
    const float bv = a.b[id] - mean_b;
    const float* x = a.x;
    const float nb = x[q.xp] + x[q.xm] + x[q.yp] + x[q.ym] + x[q.zp] + x[q.zm];
    const float rv = bv - (6.f * x[id] - nb) * a.inv_h2;
    a.r[id] = rv;
    rr_loc = df_fma(rr_loc, rv, rv);
    bb_loc = df_fma(bb_loc, bv, bv);
  }
  {
    DF u, v;
    block_total_df2(rr_loc, bb_loc, sh4, &u, &v);
    publish(ph, u, v);
  }
  if (!grid_barrier32(a.bar, a.info, a.flags)) return;
  // the scalars below are meaningful in thread 0 only
  double gamma = 0.0, bb = 0.0;
  {
    DF u, v;
    grid_total_df2(slot(ph), slot(ph) + G, G, &u, &v);
    gamma = df_to_double(u);
    bb = df_to_double(v);
  }
  ph ^= 1;
  const double thresh = a.tol * sqrt(bb), thresh2 = thresh * thresh;
  int it = 0, status = 0;
  double alpha = 0.0;
  // w = A r and delta = (r, w) for the first step
  {
    DF rw_loc{0.f, 0.f};
    for (int id = t0; id < m; id += stride) {
      const Nbr q = neighbours(id, n, nn, a.log2n);
      const float* r = a.r;
      const float rc = r[id];
      const float wv = (6.f * rc - (r[q.xp] + r[q.xm] + r[q.yp] + r[q.ym] + r[q.zp] + r[q.zm])) * a.inv_h2;
      w[id] = wv;
      rw_loc = df_fma(rw_loc, rc, wv);
    }
    DF u, v;
    block_total_df2(rw_loc, DF{0.f, 0.f}, sh4, &u, &v);
    publish(ph, u, v);
  }
  if (!grid_barrier32(a.bar, a.info, a.flags)) return;
  double delta = 0.0;
  {
    DF u, v;
    grid_total_df2(slot(ph), slot(ph) + G, G, &u, &v);
    delta = df_to_double(u);
  }
  ph ^= 1;
  double beta = 0.0;
  while (true) {
    if (threadIdx.x == 0) {
      stop = (bb == 0.0 || gamma <= thresh2) ? 1 : (it >= a.maxit ? 2 : 0);
      if (!stop) {
        const double den = it == 0 ? delta : delta - beta * gamma / alpha;
        alpha = gamma / den;
        fscal[0] = (float)alpha;
        fscal[1] = (float)beta;
      }
    }
    __syncthreads();
    if (stop == 1) break;
    if (stop == 2) { status = 1; break; }
    const float al = fscal[0], be = fscal[1];
    for (int id = t0; id < m; id += stride) {
      const float rv = a.r[id], wv = w[id];
      const float pn = it == 0 ? rv : fmaf(be, a.p[id], rv);
      const float sn = it == 0 ? wv : fmaf(be, s[id], wv);
      a.p[id] = pn;
      s[id] = sn;
      a.x[id] = fmaf(al, pn, a.x[id]);
      a.r[id] = fmaf(-al, sn, rv);
    }
    if (!grid_barrier32(a.bar, a.info, a.flags)) return;
    DF rr_l{0.f, 0.f}, rw_l{0.f, 0.f};
    for (int id = t0; id < m; id += stride) {
      const Nbr q = neighbours(id, n, nn, a.log2n);
      const float* r = a.r;
      const float rc = r[id];
      const float wv = (6.f * rc - (r[q.xp] + r[q.xm] + r[q.yp] + r[q.ym] + r[q.zp] + r[q.zm])) * a.inv_h2;
      w[id] = wv;
      rr_l = df_fma(rr_l, rc, rc);
      rw_l = df_fma(rw_l, rc, wv);
    }
    {
      DF u, v;
      block_total_df2(rr_l, rw_l, sh4, &u, &v);
      publish(ph, u, v);
    }
    if (!grid_barrier32(a.bar, a.info, a.flags)) return;
    {
      DF u, v;
      grid_total_df2(slot(ph), slot(ph) + G, G, &u, &v);
      if (threadIdx.x == 0) {
        const double gamma_new = df_to_double(u);
        delta = df_to_double(v);
        beta = gamma_new / gamma;
        gamma = gamma_new;
      }
    }
    ph ^= 1;
    ++it;
  }
  DF xs{0.f, 0.f};
  for (int id = t0; id < m; id += stride) xs = df_add_f(xs, a.x[id]);
  {
    DF u, v;
    block_total_df2(xs, DF{0.f, 0.f}, sh4, &u, &v);
    publish(ph, u, v);
  }
  if (!grid_barrier32(a.bar, a.info, a.flags)) return;
  {
    DF u, v;
    grid_total_df2(slot(ph), slot(ph) + G, G, &u, &v);
    if (threadIdx.x == 0) fscal[0] = (float)(df_to_double(u) / (double)m);
  }
  __syncthreads();
  const float mean_x = fscal[0];
  ph ^= 1;
  for (int id = t0; id < m; id += stride) a.x[id] -= mean_x;
  if (!grid_barrier32(a.bar, a.info, a.flags)) return;
  for (int id = t0; id < m; id += stride) {
    const Nbr q = neighbours(id, n, nn, a.log2n);
    const float* x = a.x;
    a.E4[id] = make_float4(-(x[q.xp] - x[q.xm]) * a.inv_2h, -(x[q.yp] - x[q.ym]) * a.inv_2h,
                           -(x[q.zp] - x[q.zm]) * a.inv_2h, 0.f);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    a.info[0] = it;
    a.info[1] = status;
    if (a.hist) a.hist[0] = it;
    a.res[0] = bb > 0.0 ? sqrt(gamma) / sqrt(bb) : 0.0;
    if (status) atomicOr(a.flags, 2);
    atomicMax(a.flags + 1, it);
  }
}

// ------------------------------------------- multigrid-preconditioned CG --
// The precision form's Poisson solve on meshes of 2^k >= 16 nodes per edge:
// CG preconditioned by one multigrid V-cycle (the same discrete system
// -Delta_h phi = b and the same stopping rule ||r|| <= tol ||b|| as the
// plain CG above, in far fewer iterations). Levels halve the edge down to
// 4; each level takes two damped-Jacobi sweeps (omega = 6/7) before and
// after its coarse correction, full-weighting restriction (per axis 1/4,
// 1/2, 1/4) and trilinear prolongation, so the V-cycle is a symmetric
// positive operator on zero-mean vectors, as CG needs. The coarsest level
// takes Jacobi sweeps from zero and is projected to zero mean. Levels above
// kMgLocalNodes nodes run on the whole grid between grid barriers; the
// smaller ones on block 0 alone between block barriers.
constexpr int kMgMaxLevels = 12;
constexpr int kMgLocalNodes = 4096;
constexpr int kMgCoarseSweeps = 16;
constexpr float kMgOmega = 6.f / 7.f;

struct Mg32Level {
  int n, log2n;
  float inv_h2;      // 1 / h_l^2
  float *ua, *ub;    // the level's iterate and a second buffer
  float* f;          // its right-hand side (level 0: the CG residual)
};

struct MgCg32Args {
  Cg32Args cg;       // the fine level's vectors, barrier words and outputs
  float *z, *z2;     // the preconditioned residual and a second buffer
  int nlev, nlev_grid;
  Mg32Level lev[kMgMaxLevels];
};

__device__ __forceinline__ float lap32(const float* u, int id, int n, int log2n, float inv_h2) {
  const Nbr q = neighbours(id, n, n * n, log2n);
  return (6.f * u[id] - (u[q.xp] + u[q.xm] + u[q.yp] + u[q.ym] + u[q.zp] + u[q.zm])) * inv_h2;
}

// full weighting at coarse node I of the fine field r (edge n = 2 nc)
__device__ __forceinline__ float restrict_fw(const float* r, int I, int log2nc, int log2n) {
  const int mc = (1 << log2nc) - 1, m = (1 << log2n) - 1;
  const int ci = I & mc, cj = (I >> log2nc) & mc, ck = I >> (2 * log2nc);
  float acc = 0.f;
#pragma unroll
  for (int c = -1; c <= 1; ++c) {
    const int kk = (2 * ck + c) & m;
    const float wz = c == 0 ? 0.5f : 0.25f;
#pragma unroll
    for (int b = -1; b <= 1; ++b) {
      const int jj = (2 * cj + b) & m;
      const float wyz = (b == 0 ? 0.5f : 0.25f) * wz;
      const int row = (jj << log2n) + (kk << (2 * log2n));
#pragma unroll
      for (int a = -1; a <= 1; ++a) acc = fmaf((a == 0 ? 0.5f : 0.25f) * wyz, r[((2 * ci + a) & m) + row], acc);
    }
  }
  return acc;
}

// trilinear prolongation at fine node id of the coarse field e (edge nc):
// the eight surrounding coarse values (repeated where a fine coordinate is
// even) with weight 1/8 each
__device__ __forceinline__ float prolong_tl(const float* e, int id, int log2n, int log2nc) {
  const int m = (1 << log2n) - 1, mc = (1 << log2nc) - 1;
  const int i = id & m, j = (id >> log2n) & m, k = id >> (2 * log2n);
  const int i0 = i >> 1, i1 = (i0 + (i & 1)) & mc;
  const int j0 = j >> 1, j1 = (j0 + (j & 1)) & mc;
  const int k0 = k >> 1, k1 = (k0 + (k & 1)) & mc;
  const int r00 = (j0 << log2nc) + (k0 << (2 * log2nc)), r10 = (j1 << log2nc) + (k0 << (2 * log2nc));
  const int r01 = (j0 << log2nc) + (k1 << (2 * log2nc)), r11 = (j1 << log2nc) + (k1 << (2 * log2nc));
  const float s = ((e[i0 + r00] + e[i1 + r00]) + (e[i0 + r10] + e[i1 + r10])) +
                  ((e[i0 + r01] + e[i1 + r01]) + (e[i0 + r11] + e[i1 + r11]));
  return 0.125f * s;
}

// node range and barrier of a V-cycle stage: the whole grid or block 0
template <bool kGrid>
struct MgSync {
  const Cg32Args* cg;
  __device__ int first() const { return kGrid ? (int)(blockIdx.x * blockDim.x + threadIdx.x) : (int)threadIdx.x; }
  __device__ int stride() const { return kGrid ? (int)(gridDim.x * blockDim.x) : (int)blockDim.x; }
  __device__ bool sync() const {
    if (kGrid) return grid_barrier32(cg->bar, cg->info, cg->flags);
    __syncthreads();
    return true;
  }
};

// level l's descent: two Jacobi sweeps from zero (the first, u = c f, is
// done by the caller at level 0), the residual, and its restriction to
// level l + 1. On entry L.f is complete; on exit C.f is.
template <bool kGrid>
__device__ bool mg_down(const MgSync<kGrid>& S, const Mg32Level& L, const Mg32Level& C, bool first_done) {
  const int m = 1 << (3 * L.log2n);
  const float cw = kMgOmega / (6.f * L.inv_h2);
  if (!first_done) {
    for (int id = S.first(); id < m; id += S.stride()) L.ub[id] = cw * L.f[id];
    if (!S.sync()) return false;
  }
  for (int id = S.first(); id < m; id += S.stride())
    L.ua[id] = fmaf(cw, L.f[id] - lap32(L.ub, id, L.n, L.log2n, L.inv_h2), L.ub[id]);
  if (!S.sync()) return false;
  for (int id = S.first(); id < m; id += S.stride()) L.ub[id] = L.f[id] - lap32(L.ua, id, L.n, L.log2n, L.inv_h2);
  if (!S.sync()) return false;
  const int mc = 1 << (3 * C.log2n);
  for (int I = S.first(); I < mc; I += S.stride()) C.f[I] = restrict_fw(L.ub, I, C.log2n, L.log2n);
  return S.sync();
}

// level l's ascent: the coarse correction added, then two Jacobi sweeps;
// the result is in L.ua. The last sweep is left to the caller at level 0.
template <bool kGrid>
__device__ bool mg_up(const MgSync<kGrid>& S, const Mg32Level& L, const Mg32Level& C, bool last_by_caller) {
  const int m = 1 << (3 * L.log2n);
  const float cw = kMgOmega / (6.f * L.inv_h2);
  for (int id = S.first(); id < m; id += S.stride()) L.ua[id] += prolong_tl(C.ua, id, L.log2n, C.log2n);
  if (!S.sync()) return false;
  for (int id = S.first(); id < m; id += S.stride())
    L.ub[id] = fmaf(cw, L.f[id] - lap32(L.ua, id, L.n, L.log2n, L.inv_h2), L.ua[id]);
  if (!S.sync()) return false;
  if (last_by_caller) return true;
  for (int id = S.first(); id < m; id += S.stride())
    L.ua[id] = fmaf(cw, L.f[id] - lap32(L.ub, id, L.n, L.log2n, L.inv_h2), L.ub[id]);
  return S.sync();
}

// the coarsest level by one block: Jacobi sweeps from zero, then the mean
// removed (the periodic operator's null space); the result in L.ua
__device__ void mg_coarsest(const Mg32Level& L, float* sh) {
  const int m = 1 << (3 * L.log2n);
  const float cw = kMgOmega / (6.f * L.inv_h2);
  for (int id = threadIdx.x; id < m; id += blockDim.x) L.ua[id] = cw * L.f[id];
  __syncthreads();
  for (int s = 1; s < kMgCoarseSweeps; ++s) {
    const float* src = (s & 1) ? L.ua : L.ub;
    float* dst = (s & 1) ? L.ub : L.ua;
    for (int id = threadIdx.x; id < m; id += blockDim.x)
      dst[id] = fmaf(cw, L.f[id] - lap32(src, id, L.n, L.log2n, L.inv_h2), src[id]);
    __syncthreads();
  }
  // kMgCoarseSweeps is even: the last sweep wrote ub
  if (threadIdx.x == 0) {
    float s = 0.f;
    for (int id = 0; id < m; ++id) s += L.ub[id];
    sh[0] = s / (float)m;
  }
  __syncthreads();
  for (int id = threadIdx.x; id < m; id += blockDim.x) L.ua[id] = L.ub[id] - sh[0];
  __syncthreads();
}

// z = M r for levels from l0 down (their right-hand side f[l0] complete on
// entry; at l0 = 0 the first sweep has been done by the caller); the
// levels from nlev_grid on are done by block 0. At level 0 the last sweep
// is left to the caller.
__device__ bool mg_vcycle(const MgCg32Args& a, float* sh) {
  const MgSync<true> G{&a.cg};
  const MgSync<false> B{&a.cg};
  for (int l = 0; l + 1 < a.nlev_grid; ++l)
    if (!mg_down(G, a.lev[l], a.lev[l + 1], l == 0)) return false;
  // the local levels on block 0: descent, coarsest, ascent
  if (blockIdx.x == 0) {
    const int lg = a.nlev_grid - 1;
    for (int l = lg; l + 1 < a.nlev; ++l) mg_down(B, a.lev[l], a.lev[l + 1], l == 0);
    mg_coarsest(a.lev[a.nlev - 1], sh);
    for (int l = a.nlev - 2; l >= lg; --l) mg_up(B, a.lev[l], a.lev[l + 1], l == 0);
  }
  if (!G.sync()) return false;
  for (int l = a.nlev_grid - 2; l >= 0; --l)
    if (!mg_up(G, a.lev[l], a.lev[l + 1], l == 0)) return false;
  return true;
}

__global__ void __launch_bounds__(kCgThreads) k_mgcg32(MgCg32Args a) {
  __shared__ double shd[1];
  __shared__ float4 sh4[32];
  __shared__ float sh[2];
  __shared__ float fscal[2];
  __shared__ int stop;
  const Cg32Args& c = a.cg;
  if ((int)blockIdx.x == c.skip_block) return;
  const int n = c.n, nn = n * n;
  const int m = (int)c.ncell;
  const int stride = gridDim.x * blockDim.x;
  const int t0 = blockIdx.x * blockDim.x + threadIdx.x;
  const int G = gridDim.x;
  int ph = 0;
  auto slot = [&](int q) { return reinterpret_cast<float2*>(c.red) + (size_t)q * 2 * G; };
  auto publish = [&](int q, DF u, DF v) {
    if (threadIdx.x == 0) {
      slot(q)[blockIdx.x] = make_float2(u.hi, u.lo);
      slot(q)[G + blockIdx.x] = make_float2(v.hi, v.lo);
    }
  };
  const Mg32Level& L0 = a.lev[0];
  const float cw0 = kMgOmega / (6.f * L0.inv_h2);
  float* const z = a.z;

  // r = (b - mean b) - A x; the first sweep of the V-cycle, z2 = c r, in the
  // same pass needs r at this node only
  const float mean_b = (float)(grid_total32(c.rhs_part, c.rhs_blocks, shd) / (double)m);
  DF bb_loc{0.f, 0.f};
  for (int id = t0; id < m; id += stride) {
    const float bv = c.b[id] - mean_b;
    const float rv = bv - lap32(c.x, id, n, c.log2n, c.inv_h2);
    c.r[id] = rv;
    a.z2[id] = cw0 * rv;
    bb_loc = df_fma(bb_loc, bv, bv);
  }
  {
    DF u, v;
    block_total_df2(bb_loc, DF{0.f, 0.f}, sh4, &u, &v);
    publish(ph, u, v);
  }
  if (!grid_barrier32(c.bar, c.info, c.flags)) return;
  double bb = 0.0;
  {
    DF u, v;
    grid_total_df2(slot(ph), slot(ph) + G, G, &u, &v);
    bb = df_to_double(u);
  }
  ph ^= 1;
  const double thresh = c.tol * sqrt(bb), thresh2 = thresh * thresh;
  double gamma = 0.0, rr = 0.0, alpha = 0.0;
  int it = 0, status = 0;
  bool first = true;
  while (true) {
    // z = M r (its first sweep is done), then the last sweep with (r, z)
    // and (r, r)
    if (!mg_vcycle(a, sh)) return;
    DF rz_l{0.f, 0.f}, rr_l{0.f, 0.f};
    for (int id = t0; id < m; id += stride) {
      const float zv = fmaf(cw0, c.r[id] - lap32(a.z2, id, n, c.log2n, L0.inv_h2), a.z2[id]);
      z[id] = zv;
      const float rv = c.r[id];
      rz_l = df_fma(rz_l, rv, zv);
      rr_l = df_fma(rr_l, rv, rv);
    }
    {
      DF u, v;
      block_total_df2(rz_l, rr_l, sh4, &u, &v);
      publish(ph, u, v);
    }
    if (!grid_barrier32(c.bar, c.info, c.flags)) return;
    {
      DF u, v;
      grid_total_df2(slot(ph), slot(ph) + G, G, &u, &v);
      if (threadIdx.x == 0) {
        const double g_new = df_to_double(u);
        rr = df_to_double(v);
        fscal[1] = first ? 0.f : (float)(g_new / gamma);
        gamma = g_new;
        stop = (bb == 0.0 || rr <= thresh2) ? 1 : (it >= c.maxit ? 2 : 0);
      }
    }
    ph ^= 1;
    __syncthreads();
    if (stop == 1) break;
    if (stop == 2) { status = 1; break; }
    // p = z + beta p
    const float be = fscal[1];
    for (int id = t0; id < m; id += stride) c.p[id] = first ? z[id] : fmaf(be, c.p[id], z[id]);
    first = false;
    if (!grid_barrier32(c.bar, c.info, c.flags)) return;
    // q = A p and (p, q)
    DF pq_l{0.f, 0.f};
    for (int id = t0; id < m; id += stride) {
      const float qv = lap32(c.p, id, n, c.log2n, c.inv_h2);
      c.q[id] = qv;
      pq_l = df_fma(pq_l, c.p[id], qv);
    }
    {
      DF u, v;
      block_total_df2(pq_l, DF{0.f, 0.f}, sh4, &u, &v);
      publish(ph, u, v);
    }
    if (!grid_barrier32(c.bar, c.info, c.flags)) return;
    {
      DF u, v;
      grid_total_df2(slot(ph), slot(ph) + G, G, &u, &v);
      if (threadIdx.x == 0) {
        alpha = gamma / df_to_double(u);
        fscal[0] = (float)alpha;
      }
    }
    ph ^= 1;
    __syncthreads();
    // x += alpha p, r -= alpha q, and the next V-cycle's first sweep
    const float al = fscal[0];
    for (int id = t0; id < m; id += stride) {
      c.x[id] = fmaf(al, c.p[id], c.x[id]);
      const float rv = fmaf(-al, c.q[id], c.r[id]);
      c.r[id] = rv;
      a.z2[id] = cw0 * rv;
    }
    ++it;
    if (!grid_barrier32(c.bar, c.info, c.flags)) return;
  }
  // zero-mean potential and E, as in k_cg32
  DF xs{0.f, 0.f};
  for (int id = t0; id < m; id += stride) xs = df_add_f(xs, c.x[id]);
  {
    DF u, v;
    block_total_df2(xs, DF{0.f, 0.f}, sh4, &u, &v);
    publish(ph, u, v);
  }
  if (!grid_barrier32(c.bar, c.info, c.flags)) return;
  {
    DF u, v;
    grid_total_df2(slot(ph), slot(ph) + G, G, &u, &v);
    if (threadIdx.x == 0) fscal[0] = (float)(df_to_double(u) / (double)m);
  }
  __syncthreads();
  const float mean_x = fscal[0];
  for (int id = t0; id < m; id += stride) c.x[id] -= mean_x;
  if (!grid_barrier32(c.bar, c.info, c.flags)) return;
  for (int id = t0; id < m; id += stride) {
    const Nbr q = neighbours(id, n, nn, c.log2n);
    const float* x = c.x;
    c.E4[id] = make_float4(-(x[q.xp] - x[q.xm]) * c.inv_2h, -(x[q.yp] - x[q.ym]) * c.inv_2h,
                           -(x[q.zp] - x[q.zm]) * c.inv_2h, 0.f);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    c.info[0] = it;
    c.info[1] = status;
    if (c.hist) c.hist[0] = it;
    c.res[0] = bb > 0.0 ? sqrt(rr) / sqrt(bb) : 0.0;
    if (status) atomicOr(c.flags, 2);
    atomicMax(c.flags + 1, it);
  }
}

// --------------------------------------------------------- error norms --
struct Err32Args {
  Params P;
  TimeTerms tt;
  int64_t cell_base;  // subtracted from the stored cell (batches)
  const int32_t* cell;
  const float *o0, *o1, *o2, *v0, *v1, *v2;
  const uint32_t* pid;
  const float* phi;
  double* part;
  int pblocks;
};

__global__ void __launch_bounds__(kThreads) k_err_partial32(Err32Args a) {
  __shared__ double sh[(kThreads / 32) * 14];
  const Params& P = a.P;
  double vals[14];
#pragma unroll
  for (int q = 0; q < 14; ++q) vals[q] = 0.0;
  if ((int)blockIdx.x < a.pblocks) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < P.np) {
      const uint64_t p = a.pid[j];
      const U4 b0 = sample_block(P, p, 0), b1 = sample_block(P, p, 1), b2 = sample_block(P, p, 2);
      const double xi[6] = {unif52(b0.x, b0.y), unif52(b0.z, b0.w), unif52(b1.x, b1.y),
                            unif52(b1.z, b1.w), unif52(b2.x, b2.y), unif52(b2.z, b2.w)};
      const int n = P.n, c = (int)(a.cell[j] - a.cell_base);
      const int ci[3] = {c % n, (c / n) % n, c / (n * n)};
      const float os[3] = {a.o0[j], a.o1[j], a.o2[j]};
      const float vs[3] = {a.v0[j], a.v1[j], a.v2[j]};
      const bool paper = P.dist == PIC_DIST_PAPER;
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        double s, cc;
        const double xm = paper ? xm_solve_gen(a.tt, d, xi[d], &s, &cc) : xm_solve(P, a.tt, xi[d], &s);
        double e = ((double)ci[d] + (double)os[d]) * P.h - xm;
        e -= floor(e + 0.5);
        vals[d] = e * e;
        vals[7 + d] = fabs(e);
        const double vmd = paper ? tau_inv(xi[3 + d]) * a.tt.vh[d] : P.vmean[d] + P.vsig * normcdfinv(xi[3 + d]);
        const double ev = (double)vs[d] - vmd;
        vals[3 + d] = ev * ev;
        vals[10 + d] = fabs(ev);
      }
    }
  } else {
    const int64_t id = (int64_t)(blockIdx.x - a.pblocks) * blockDim.x + threadIdx.x;
    if (id < P.ncell) {
      const int n = P.n;
      const int i = (int)(id % n), jj = (int)((id / n) % n), k = (int)(id / ((int64_t)n * n));
      const double phiM = a.tt.em_amp / kTwoPi * sinpi(2.0 * (i * P.h - P.phi_shift[0])) *
                          sinpi(2.0 * (jj * P.h - P.phi_shift[1])) * sinpi(2.0 * (k * P.h - P.phi_shift[2]));
      const double e = (double)a.phi[id] - phiM;
      vals[6] = e * e;
      vals[13] = fabs(e);
    }
  }
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
  if (threadIdx.x < 14) {
    const int q = threadIdx.x;
    double x = sh[q];
    for (int ww = 1; ww < (int)(blockDim.x >> 5); ++ww) x = q < 7 ? x + sh[ww * 14 + q] : fmax(x, sh[ww * 14 + q]);
    a.part[(size_t)blockIdx.x * 14 + q] = x;
  }
}

struct StoreField32Args {
  int64_t ncell;
  const float* phi;
  const float4* E4;
  double *ophi, *oE;
};

__global__ void __launch_bounds__(kThreads) k_store_field32(StoreField32Args a) {
  const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= a.ncell) return;
  if (a.ophi) a.ophi[id] = a.phi[id];
  if (a.oE) {
    const float4 e = a.E4[id];
    a.oE[3 * id] = e.x;
    a.oE[3 * id + 1] = e.y;
    a.oE[3 * id + 2] = e.z;
  }
}

struct StoreDv32Args {
  int64_t np;
  const float *d0, *d1, *d2, *m0, *m1, *m2;
  const uint32_t* pid;
  double *dv, *dvm;
};

__global__ void __launch_bounds__(kThreads) k_store_dv32(StoreDv32Args a) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= a.np) return;
  const int64_t p = a.pid[j];
  a.dv[3 * p] = a.d0[j]; a.dv[3 * p + 1] = a.d1[j]; a.dv[3 * p + 2] = a.d2[j];
  a.dvm[3 * p] = a.m0[j]; a.dvm[3 * p + 1] = a.m1[j]; a.dvm[3 * p + 2] = a.m2[j];
}

}  // namespace

// ============================================================== launches ==
// The inverse of a sort permutation (slot[pid[j]] = j) by windows of
// kInvWindow pids, each window's pass on the context's auxiliary stream
// (higher priority) ahead of consume(lo, hi), which the caller launches on
// the context's stream for the rows (pids) lo .. hi - 1 of a load or store
// that waits on the host link: window r's pass runs beside the consumer of
// window r - 1. Only the first pass is not hidden; it takes a grid of one
// thread per pid, the later ones two blocks per SM, so that they do not
// hold the SMs the consumer needs (full-grid passes there took every SM a
// consumer block freed, and the two kernels took turns).
template <class Consume>
cudaError_t inverse_by_windows(pic_ctx* c, const uint32_t* pid, Consume consume) {
  cudaError_t e = ensure_aux_stream(c);
  if (e != cudaSuccess) return e;
  InvPerm32Args ia;
  ia.np = c->P.np;
  ia.pid = pid;
  ia.slot = c->perm;
  // the auxiliary stream starts after the work already on the context's
  e = cudaEventRecord(c->aux_fork, c->stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(c->aux, c->aux_fork, 0);
  for (int64_t lo = 0; lo < ia.np && e == cudaSuccess; lo += kInvWindow) {
    ia.lo = lo;
    ia.hi = lo + kInvWindow < ia.np ? lo + kInvWindow : ia.np;
    if (lo == 0)
      k_inv_perm32<<<blocks_for(ia.np), kThreads, 0, c->aux>>>(ia);
    else
      k_inv_perm32_gs<<<2 * c->num_sms, kThreads, 0, c->aux>>>(ia);
    c->launches++;
    // the wait takes the record made just before it, so one event serves
    // every window
    e = cudaEventRecord(c->aux_join, c->aux);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c->stream, c->aux_join, 0);
    if (e == cudaSuccess) consume(ia.lo, ia.hi);
  }
  return e == cudaSuccess ? cudaGetLastError() : e;
}

cudaError_t launch_sample32(pic_ctx* c, double t0, const double* x, const double* v, int held, bool to_records) {
  Sample32Args a;
  a.P = c->P;
  a.tt = time_terms(c->P, t0);
  a.row0 = 0;
  a.row_end = c->P.np;
  a.xs = x;
  a.vs = v;
  a.vslot = held >= 0 ? c->perm : nullptr;
  a.vin0 = held >= 0 ? c->vmf[held][0] : nullptr;
  a.vin1 = held >= 0 ? c->vmf[held][1] : nullptr;
  a.vin2 = held >= 0 ? c->vmf[held][2] : nullptr;
  const int b = c->cur;
  a.cell = c->cell32[b];
  a.o0 = c->off[b][0]; a.o1 = c->off[b][1]; a.o2 = c->off[b][2];
  a.v0 = c->vf[b][0]; a.v1 = c->vf[b][1]; a.v2 = c->vf[b][2];
  a.m0 = c->vmf[b][0]; a.m1 = c->vmf[b][1]; a.m2 = c->vmf[b][2];
  a.pid = c->pid[b];
  if (to_records) {
    a.rec = reinterpret_cast<float4*>(c->stage);
    a.key = c->key;
    a.rank = c->rank;
    a.count = c->count;
    if (c->bins) {
      a.bins = c->bins;
      a.bin_cap = c->bin_cap;
      a.bin_over = c->bin_over;
    }
  }
  if (held < 0 || c->inv_valid) {
    prof_begin(c);
    k_sample32<<<blocks_for(c->P.np), kThreads, 0, c->stream>>>(a);
    prof_end(c, x ? KC_OTHER : KC_SAMPLE);
    c->launches++;
    return cudaGetLastError();
  }
  // v^M read through the inverse of the held state's permutation, formed
  // by windows ahead of the load of the same rows (pids)
  prof_begin(c);
  const cudaError_t e = inverse_by_windows(c, c->pid[held], [&](int64_t lo, int64_t hi) {
    a.row0 = lo;
    a.row_end = hi;
    k_sample32<<<blocks_for(hi - lo), kThreads, 0, c->stream>>>(a);
    c->launches++;
  });
  prof_end(c, KC_OTHER);
  // perm now holds the inverse of the held state's order, which the sort
  // that follows replaces
  return e;
}

cudaError_t launch_keys32(pic_ctx* c) {
  Keys32Args a;
  a.np = c->P.np;
  a.cell = c->cell32[c->cur];
  a.key = c->key;
  a.rank = c->rank;
  a.count = c->count;
  prof_begin(c);
  k_keys32<<<blocks_for(a.np), kThreads, 0, c->stream>>>(a);
  prof_end(c, KC_SORT);
  c->launches++;
  return cudaGetLastError();
}

cudaError_t launch_gather32(pic_ctx* c) {
  Gather32Args g;
  g.n = c->P.n;
  g.ncell = c->P.ncell;
  g.start = c->start;
  g.perm = c->perm;
  const int b = c->cur, o = 1 - c->cur;
  for (int d = 0; d < 3; ++d) {
    g.in[d] = c->off[b][d]; g.in[3 + d] = c->vf[b][d]; g.in[6 + d] = c->vmf[b][d];
    g.out[d] = c->off[o][d]; g.out[3 + d] = c->vf[o][d]; g.out[6 + d] = c->vmf[o][d];
  }
  g.pid_in = c->pid[b];
  g.pid_out = c->pid[o];
  g.cell_out = c->cell32[o];
  g.corner = c->corner;
  g.big_lo = big_cell_threshold(g.ncell, c->P.np);
  g.spid = c->pid[o];  // written in arrival order by the scatter
  if (c->rec_state) {
    g.rec = c->bin_state ? c->bins : reinterpret_cast<const float4*>(c->stage);
    g.bin_cap = c->bin_state ? c->bin_cap : 0;
    g.spid = nullptr;  // the pids come with the records
  }
  // one warp per cell: blocks of consecutive cells, handed to the SMs as
  // they free up (measured faster than resident warps walking the cells
  // with a grid stride)
  int64_t blocks = (c->P.ncell * 32 + kGatherThreads - 1) / kGatherThreads;
  if (blocks > INT_MAX) blocks = INT_MAX;  // the grid-stride loop takes the rest
  prof_begin(c);
  if (g.rec)
    k_sort_gather32<true><<<(int)blocks, kGatherThreads, 0, c->stream>>>(g);
  else
    k_sort_gather32<false><<<(int)blocks, kGatherThreads, 0, c->stream>>>(g);
  if (g.big_lo < INT_MAX) {
    k_sort_big32<<<2 * c->num_sms, kBigThreads, (size_t)kMaxBlockSort * 8, c->stream>>>(g);
    c->launches++;
  }
  prof_end(c, KC_GATHER);
  c->launches++;
  c->cur = o;
  c->rec_state = false;
  c->bin_state = false;
  return cudaGetLastError();
}

const void* sort_big32_kernel_ptr() { return (const void*)k_sort_big32; }
int dsmc32_threads() { return kDsmcThreads; }
size_t dsmc32_smem_bytes(int bm_words) { return (size_t)(kDsmcThreads / 32) * dsmc32_smem_words(bm_words) * 4; }
const void* dsmc32_kernel_ptr(bool verify) {
  return verify ? (const void*)k_dsmc32<true> : (const void*)k_dsmc32<false>;
}
int cg32_threads() { return kCgThreads; }
const void* cg32_kernel_ptr() { return (const void*)k_cg32; }

cudaError_t launch_dsmc32(pic_ctx* c, uint32_t c0, bool separate, double t_src) {
  Dsmc32Args a;
  a.P = params_f(c->P);
  const TimeTermsF ts = to_float(time_terms(c->P, t_src));
  for (int d = 0; d < 3; ++d) a.vh[d] = ts.vh[d];
  const int b = c->cur;
  a.v0 = c->vf[b][0]; a.v1 = c->vf[b][1]; a.v2 = c->vf[b][2];
  a.start = c->start;
  a.c0 = c0;
  a.dv0 = c->dvf[0]; a.dv1 = c->dvf[1]; a.dv2 = c->dvf[2];
  if (separate) { a.m0 = c->dvmf[0]; a.m1 = c->dvmf[1]; a.m2 = c->dvmf[2]; }
  else { a.m0 = a.m1 = a.m2 = nullptr; }
  a.overlay = c->overlay32;
  a.max_ppc = c->cfg.max_ppc;
  a.bm_words = c->bm_words;
  a.G = c->dsmc_G;
  a.Kc = c->dsmc_Kc;
  a.nchunks = (c->P.K + c->dsmc_Kc - 1) / c->dsmc_Kc;
  a.ngroups = c->dsmc_groups;
  {
    // groups per take: kDsmcChunk while every resident warp gets at least
    // four takes, fewer (down to one) on launches with few groups per warp
    const int64_t warps = (int64_t)c->dsmc_grid * (kDsmcThreads / 32);
    const int64_t ch = a.ngroups / (4 * warps);
    a.chunk = (int)(ch < 1 ? 1 : (ch > kDsmcChunk ? kDsmcChunk : ch));
  }
  a.counters = c->counters;
  a.queue = c->dsmc_queue;
  a.flags = c->flags;
  a.lg = DLog{c->dlog, c->dlog_n, (long long)c->dlog_cap, c->dlog ? c->dlog_mode : 0};
  a.hist = c->hist_row;
  prof_begin(c);
  const cudaError_t eq = cudaMemsetAsync(c->dsmc_queue, 0, 8, c->stream);
  if (eq != cudaSuccess) return eq;
  if (c->P.verify || a.lg.mode == PIC_DLOG_ALL)
    k_dsmc32<true><<<c->dsmc_grid, kDsmcThreads, c->dsmc_smem, c->stream>>>(a);
  else
    k_dsmc32<false><<<c->dsmc_grid, kDsmcThreads, c->dsmc_smem, c->stream>>>(a);
  prof_end(c, KC_DSMC);
  c->launches++;
  return cudaGetLastError();
}

cudaError_t launch_kick32(pic_ctx* c, double tE, bool with_coll, bool drift, double th, double tn1) {
  Kick32Args a;
  a.P = params_f(c->P);
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
  a.tE = to_float(time_terms(c->P, tE));
  a.th = to_float(time_terms(c->P, th));
  a.t0 = to_float(time_terms(c->P, tE));
  a.t1 = to_float(time_terms(c->P, tn1));
  a.drift = drift ? 1 : 0;
  a.key = c->key;
  a.rank = c->rank;
  a.count = c->count;
  prof_begin(c);
  if (!drift) {
    // the closing half kick: by cells
    Close32Args k;
    k.P = a.P;
    k.ncell = c->P.ncell;
    k.start = c->start;
    k.o0 = a.o0; k.o1 = a.o1; k.o2 = a.o2;
    k.v0 = a.v0; k.v1 = a.v1; k.v2 = a.v2;
    k.dv0 = a.dv0; k.dv1 = a.dv1; k.dv2 = a.dv2;
    k.m0 = a.m0; k.m1 = a.m1; k.m2 = a.m2;
    k.E4 = a.E4;
    k.L0 = a.L0; k.L1 = a.L1; k.L2 = a.L2;
    k.tE = a.tE;
    int64_t blocks = (c->P.ncell * 32 + kCloseThreads - 1) / kCloseThreads;
    if (blocks > INT_MAX) blocks = INT_MAX;
    if (c->P.dist == PIC_DIST_PAPER)
      k_close32<true><<<(int)blocks, kCloseThreads, 0, c->stream>>>(k);
    else
      k_close32<false><<<(int)blocks, kCloseThreads, 0, c->stream>>>(k);
  } else if (c->P.dist == PIC_DIST_PAPER)
    k_kick32<2><<<blocks_for(c->P.np, kKickThreads), kKickThreads, 0, c->stream>>>(a);
  else if (c->P.verify & PIC_VERIFY_ISOLATE)
    k_kick32<1><<<blocks_for(c->P.np, kKickThreads), kKickThreads, 0, c->stream>>>(a);
  else
    k_kick32<0><<<blocks_for(c->P.np, kKickThreads), kKickThreads, 0, c->stream>>>(a);
  prof_end(c, KC_KICK);
  c->launches++;
  c->lor_valid = !drift;
  return cudaGetLastError();
}

int mg_levels(int n, int* nlev_grid, size_t* work_floats) {
  *nlev_grid = 0;
  *work_floats = 0;
  if (n < 16 || (n & (n - 1)) != 0) return 0;
  int nlev = 0, first_local = -1;
  for (int e = n; e >= 4; e >>= 1, ++nlev) {
    if (first_local < 0 && (int64_t)e * e * e <= kMgLocalNodes) first_local = nlev;
    if (nlev > 0) *work_floats += 3 * (size_t)e * e * e;
  }
  if (nlev > kMgMaxLevels) return 0;
  *nlev_grid = first_local + 1;
  return nlev;
}

cudaError_t launch_cg32(pic_ctx* c) {
  Cg32Args a;
  a.n = c->P.n;
  a.log2n = (c->P.n & (c->P.n - 1)) == 0 ? __builtin_ctz((unsigned)c->P.n) : -1;
  a.ncell = c->P.ncell;
  a.inv_h2 = (float)((double)c->P.n * (double)c->P.n);
  a.inv_2h = (float)(0.5 * (double)c->P.n);
  a.b = c->bf;
  a.x = c->phif;
  a.r = c->cgf_r;
  a.p = c->cgf_p;
  a.q = c->cgf_q;
  a.rhs_part = c->rhs_part;
  a.rhs_blocks = (int)c->rhs_blocks;
  a.red = c->cg_red;
  a.bar = c->cg_bar;
  a.info = c->cg_info;
  a.flags = c->flags;
  a.res = c->cg_res;
  a.tol = c->cfg.cg_tol;
  a.maxit = c->cfg.cg_maxit;
  a.E4 = c->Ef4;
  a.skip_block = c->stall_next_cg ? c->cg_grid - 1 : -1;
  a.hist = c->hist_row;
  c->stall_next_cg = false;
  cudaError_t e = cudaMemsetAsync(c->cg_bar, 0, 2 * sizeof(unsigned int), c->stream);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(c->cg_info, 0, 3 * sizeof(int), c->stream);
  if (e != cudaSuccess) return e;
  prof_begin(c);
  if (c->mg_nlev > 0) {
    MgCg32Args m;
    m.cg = a;
    m.z = c->mg_z;
    m.z2 = c->mg_z2;
    m.nlev = c->mg_nlev;
    m.nlev_grid = c->mg_nlev_grid;
    float* w = c->mg_work;
    for (int l = 0; l < m.nlev; ++l) {
      Mg32Level& L = m.lev[l];
      L.n = c->P.n >> l;
      L.log2n = a.log2n - l;
      L.inv_h2 = (float)((double)L.n * (double)L.n);
      if (l == 0) {
        L.ua = c->mg_z;
        L.ub = c->mg_z2;
        L.f = c->cgf_r;
      } else {
        const size_t nl = (size_t)L.n * L.n * L.n;
        L.ua = w;
        L.ub = w + nl;
        L.f = w + 2 * nl;
        w += 3 * nl;
      }
    }
    for (int l = m.nlev; l < kMgMaxLevels; ++l) m.lev[l] = Mg32Level{0, 0, 0.f, nullptr, nullptr, nullptr};
    void* args[] = {&m};
    e = cudaLaunchCooperativeKernel((const void*)k_mgcg32, dim3(c->cg_grid), dim3(kCgThreads), args, 0, c->stream);
  } else {
    void* args[] = {&a};
    e = cudaLaunchCooperativeKernel((const void*)k_cg32, dim3(c->cg_grid), dim3(kCgThreads), args, 0, c->stream);
  }
  prof_end(c, KC_CG);
  c->launches++;
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

cudaError_t launch_errors32(pic_ctx* c, double t) {
  Err32Args a;
  a.P = c->P;
  a.tt = time_terms(c->P, t);
  a.cell_base = 0;
  const int b = c->cur;
  a.cell = c->cell32[b];
  a.o0 = c->off[b][0]; a.o1 = c->off[b][1]; a.o2 = c->off[b][2];
  a.v0 = c->vf[b][0]; a.v1 = c->vf[b][1]; a.v2 = c->vf[b][2];
  a.pid = c->pid[b];
  a.phi = c->phif;
  a.part = c->err_part;
  a.pblocks = blocks_for(c->P.np);
  const int nb = a.pblocks + blocks_for(c->P.ncell);
  prof_begin(c);
  k_err_partial32<<<nb, kThreads, 0, c->stream>>>(a);
  prof_end(c, KC_ERR);
  c->launches++;
  return cudaGetLastError();
}

cudaError_t launch_store_state32(pic_ctx* c, double* xv, int32_t* cell_of_pid) {
  Store32Args a;
  a.np = c->P.np;
  a.n = c->P.n;
  a.h = c->P.h;
  a.cell_base = 0;
  const int b = c->cur;
  a.cell = c->cell32[b];
  a.o0 = c->off[b][0]; a.o1 = c->off[b][1]; a.o2 = c->off[b][2];
  a.v0 = c->vf[b][0]; a.v1 = c->vf[b][1]; a.v2 = c->vf[b][2];
  a.pid = c->pid[b];
  a.xv = xv;
  a.cell_of_pid = cell_of_pid;
  prof_begin(c);
  k_store_state32<<<blocks_for(c->P.np), kThreads, 0, c->stream>>>(a);
  prof_end(c, KC_OTHER);
  c->launches++;
  return cudaGetLastError();
}

// x, v [N_p][3] in pid order written in place (device or mapped pinned host
// memory, 8-byte aligned); the inverse permutation goes into the sort's
// free permutation buffer

// Into arrays in pid order used in place; without a valid inverse the
// store goes by windows of the inverse.
cudaError_t launch_store_state32_by_pid(pic_ctx* c, double* x, double* v) {
  const int b = c->cur;
  StoreByPid32Args a;
  a.row0 = 0;
  a.row_end = c->P.np;
  a.n = c->P.n;
  a.h = c->P.h;
  a.slot = c->perm;
  a.cell = c->cell32[b];
  a.o0 = c->off[b][0]; a.o1 = c->off[b][1]; a.o2 = c->off[b][2];
  a.v0 = c->vf[b][0]; a.v1 = c->vf[b][1]; a.v2 = c->vf[b][2];
  a.x = x;
  a.v = v;
  prof_begin(c);
  cudaError_t e;
  if (c->inv_valid) {
    k_store_state32_by_pid<<<blocks_for(a.row_end), kThreads, 0, c->stream>>>(a);
    c->launches++;
    e = cudaGetLastError();
  } else {
    e = inverse_by_windows(c, c->pid[b], [&](int64_t lo, int64_t hi) {
      a.row0 = lo;
      a.row_end = hi;
      k_store_state32_by_pid<<<blocks_for(hi - lo), kThreads, 0, c->stream>>>(a);
      c->launches++;
    });
    c->inv_valid = e == cudaSuccess;
  }
  prof_end(c, KC_OTHER);
  return e;
}

// replicate rep of a batch: the single-domain kernels on its sub-ranges
cudaError_t launch_batch_errors(pic_ctx* c, int rep, double t) {
  const Params& P = c->prm_host[rep];
  const BatchRep& B = c->reps_host[rep];
  Err32Args a;
  a.P = P;
  a.tt = time_terms(P, t);
  a.cell_base = B.coff;
  const int b = c->cur;
  a.cell = c->cell32[b] + B.poff;
  a.o0 = c->off[b][0] + B.poff; a.o1 = c->off[b][1] + B.poff; a.o2 = c->off[b][2] + B.poff;
  a.v0 = c->vf[b][0] + B.poff; a.v1 = c->vf[b][1] + B.poff; a.v2 = c->vf[b][2] + B.poff;
  a.pid = c->pid[b] + B.poff;
  a.phi = c->phif + B.coff;
  a.part = c->err_part;
  a.pblocks = blocks_for(P.np);
  const int nb = a.pblocks + blocks_for(P.ncell);
  prof_begin(c);
  k_err_partial32<<<nb, kThreads, 0, c->stream>>>(a);
  prof_end(c, KC_ERR);
  c->launches++;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // final reduction with this replicate's counts
  const Params saved = c->P;
  c->P = P;
  e = launch_err_final(c, nb);
  c->P = saved;
  return e;
}

cudaError_t launch_batch_store_state(pic_ctx* c, int rep, double* xv) {
  const Params& P = c->prm_host[rep];
  const BatchRep& B = c->reps_host[rep];
  Store32Args a;
  a.np = P.np;
  a.n = P.n;
  a.h = P.h;
  a.cell_base = B.coff;
  const int b = c->cur;
  a.cell = c->cell32[b] + B.poff;
  a.o0 = c->off[b][0] + B.poff; a.o1 = c->off[b][1] + B.poff; a.o2 = c->off[b][2] + B.poff;
  a.v0 = c->vf[b][0] + B.poff; a.v1 = c->vf[b][1] + B.poff; a.v2 = c->vf[b][2] + B.poff;
  a.pid = c->pid[b] + B.poff;
  a.xv = xv;
  a.cell_of_pid = nullptr;
  prof_begin(c);
  k_store_state32<<<blocks_for(a.np), kThreads, 0, c->stream>>>(a);
  prof_end(c, KC_OTHER);
  c->launches++;
  return cudaGetLastError();
}

cudaError_t launch_store_field32(pic_ctx* c, double* phi, double* E) {
  StoreField32Args a;
  a.ncell = c->P.ncell;
  a.phi = c->phif;
  a.E4 = c->Ef4;
  a.ophi = phi;
  a.oE = E;
  prof_begin(c);
  k_store_field32<<<blocks_for(a.ncell), kThreads, 0, c->stream>>>(a);
  prof_end(c, KC_OTHER);
  c->launches++;
  return cudaGetLastError();
}

cudaError_t launch_store_dv32(pic_ctx* c, double* dv, double* dvm) {
  StoreDv32Args a;
  a.np = c->P.np;
  a.d0 = c->dvf[0]; a.d1 = c->dvf[1]; a.d2 = c->dvf[2];
  a.m0 = c->dvmf[0]; a.m1 = c->dvmf[1]; a.m2 = c->dvmf[2];
  a.pid = c->pid[c->cur];
  a.dv = dv;
  a.dvm = dvm;
  prof_begin(c);
  k_store_dv32<<<blocks_for(c->P.np), kThreads, 0, c->stream>>>(a);
  prof_end(c, KC_OTHER);
  c->launches++;
  return cudaGetLastError();
}

}  // namespace pic

namespace pic {
ParamsF params_f(const Params& P) {
  ParamsF f;
  f.n = P.n;
  f.nn = P.n * P.n;
  f.log2n = -1;
  for (int b = 0; b < 31; ++b)
    if ((1 << b) == P.n) f.log2n = b;
  f.K = P.K;
  f.np = P.np;
  f.ncell = P.ncell;
  f.key0 = P.key0;
  f.key1 = P.key1;
  for (int r = 0; r < 10; ++r) {
    f.rk[0][r] = P.key0 + (uint32_t)r * 0x9E3779B9u;
    f.rk[1][r] = P.key1 + (uint32_t)r * 0xBB67AE85u;
  }
  f.h = (float)P.h;
  f.dt_qm = (float)(P.dt * P.qm_eff);
  f.dtn = (float)(P.dt * (double)P.n);
  f.fx_amp = (float)P.fx_amp;
  f.fx_a2pi = (float)P.fx_amp_over_2pi;
  f.fx_Ac = (float)(P.fx_amp * P.fx_speed);
  for (int d = 0; d < 3; ++d) {
    f.vmean[d] = (float)P.vmean[d];
    f.phi_shift[d] = (float)P.phi_shift[d];
  }
  f.vsig = (float)P.vsig;
  f.inv_vsig = (float)P.inv_vsig;
  f.src_pref = (float)P.src_pref;
  f.pmax = (float)P.pmax;
  f.gmax = (float)P.gmax;
  f.gmax2 = (float)(P.gmax * P.gmax);
  f.ginv_f = P.ginv_f;
  f.ginv_M = P.ginv_M;
  f.verify = P.verify;
  f.nf = (float)P.n;
  f.cdt = (float)(P.fx_speed * P.dt);
  f.ang_hist = P.ang_hist;
  f.dist = P.dist;
  f.n_sigma = P.n_sigma;
  for (int k = 0; k < 3; ++k) f.sigma_n[k] = (float)P.sigma_n[k];
  f.sgmax = (float)P.sg_max;
  f.src_pref_n = (float)P.src_pref_n;
  f.dt = (float)P.dt;
  return f;
}
}  // namespace pic
