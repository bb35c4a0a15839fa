// Counting sort of the particles by (cell, pid) and the cloud-in-cell charge
// partials of every cell (Sec. 2).
//
//  keys    : cell of every particle and an arrival rank from one atomic per
//            particle (the rank order is arbitrary);
//  scan    : exclusive scan of the per-cell counts into start[];
//  scatter : perm[start[cell] + rank] = source index;
//  gather  : one warp per cell ranks the cell's entries by pid (ascending
//            pid is the canonical in-cell order), moves every per-particle
//            array into the other buffer at its final slot, then sums the 8
//            corner CIC weights of the cell's particles in that order with a
//            fixed-shape warp reduction (deterministic, no floating-point
//            atomics).
#include "pic_internal.cuh"

namespace pic {
namespace {

constexpr int kThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kThreads * kScanItems;

inline int blocks_for(int64_t n, int t = kThreads) {
  int64_t b = (n + t - 1) / t;
  return (int)(b < 1 ? 1 : b);
}

struct KeysArgs {
  int64_t np;
  int n;
  const double *x0, *x1, *x2;
  int32_t *key, *rank, *count;
};

__global__ void __launch_bounds__(kThreads) k_keys(KeysArgs a) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= a.np) return;
  const int n = a.n;
  const int32_t k = cell_coord(a.x0[j], n) + n * (cell_coord(a.x1[j], n) + n * cell_coord(a.x2[j], n));
  a.key[j] = k;
  a.rank[j] = cell_slot(a.count, k);
}

// block-wide exclusive scan of one int per thread; returns the block total
__device__ __forceinline__ int32_t block_exclusive_scan(int32_t v, int32_t* total, int32_t* sh) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int32_t incl = v;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const int32_t y = __shfl_up_sync(0xffffffffu, incl, off);
    if (lane >= off) incl += y;
  }
  if (lane == 31) sh[w] = incl;
  __syncthreads();
  if (w == 0) {
    int32_t s = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const int32_t y = __shfl_up_sync(0xffffffffu, s, off);
      if (lane >= off) s += y;
    }
    sh[32 + lane] = s;  // inclusive warp prefix
  }
  __syncthreads();
  const int32_t warp_off = w > 0 ? sh[32 + w - 1] : 0;
  *total = sh[32 + (blockDim.x >> 5) - 1];
  __syncthreads();
  return warp_off + incl - v;
}

__global__ void __launch_bounds__(kThreads) k_scan_reduce(const int32_t* count, int64_t m, int32_t* bsum) {
  __shared__ int32_t sh[64];
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  int32_t s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    const int64_t id = base + (int64_t)threadIdx.x * kScanItems + i;
    if (id < m) s += count[id];
  }
  int32_t total;
  block_exclusive_scan(s, &total, sh);
  if (threadIdx.x == 0) bsum[blockIdx.x] = total;
}

__global__ void __launch_bounds__(1024) k_scan_blocks(int32_t* bsum, int64_t nb) {
  __shared__ int32_t sh[64];
  int32_t carry = 0;
  for (int64_t base = 0; base < nb; base += blockDim.x) {
    const int64_t id = base + threadIdx.x;
    const int32_t v = id < nb ? bsum[id] : 0;
    int32_t total;
    const int32_t ex = block_exclusive_scan(v, &total, sh);
    if (id < nb) bsum[id] = carry + ex;
    carry += total;
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kThreads) k_scan_final(const int32_t* count, int64_t m, const int32_t* boff,
                                                         int32_t* start) {
  __shared__ int32_t sh[64];
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  int32_t vals[kScanItems];
  int32_t s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    const int64_t id = base + (int64_t)threadIdx.x * kScanItems + i;
    vals[i] = id < m ? count[id] : 0;
    s += vals[i];
  }
  int32_t total;
  int32_t run = block_exclusive_scan(s, &total, sh) + boff[blockIdx.x];
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    const int64_t id = base + (int64_t)threadIdx.x * kScanItems + i;
    if (id < m) start[id] = run;
    run += vals[i];
    if (id == m - 1) start[m] = run;
  }
}

struct ScatterArgs {
  int64_t np;
  const int32_t *key, *rank, *start;
  int32_t* perm;
  const uint32_t* pid;  // each particle's pid, also written to its arrival slot (nullptr: pid = j)
  uint32_t* spid;       // optional
};

__global__ void __launch_bounds__(kThreads) k_scatter(ScatterArgs a) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= a.np) return;
  const int32_t slot = a.start[a.key[j]] + a.rank[j];
  a.perm[slot] = (int32_t)j;
  if (a.spid) a.spid[slot] = a.pid ? a.pid[j] : (uint32_t)j;
}

struct GatherArgs {
  int n;
  int64_t ncell;
  const int32_t *start, *perm;
  const double* in[9];    // x0..2, v0..2, vm0..2
  double* out[9];
  const uint32_t* pid_in;
  uint32_t* pid_out;
  double* corner;         // [8][ncell]
  int big_lo;             // cells above this count go to the block sort
};

__device__ __forceinline__ void move_particle(const GatherArgs& a, int32_t src, int32_t dst) {
#pragma unroll
  for (int q = 0; q < 9; ++q) a.out[q][dst] = a.in[q][src];
  a.pid_out[dst] = a.pid_in[src];
}

// add the 8 corner weights of the moved particle in output slot j
__device__ __forceinline__ void add_cic(const GatherArgs& a, int32_t j, int ci, int cj, int ck, double* acc) {
  const double n = (double)a.n;
  const double fx = a.out[0][j] * n - (double)ci;
  const double fy = a.out[1][j] * n - (double)cj;
  const double fz = a.out[2][j] * n - (double)ck;
  const double wx[2] = {1.0 - fx, fx}, wy[2] = {1.0 - fy, fy}, wz[2] = {1.0 - fz, fz};
#pragma unroll
  for (int c = 0; c < 2; ++c)
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
      for (int q = 0; q < 2; ++q) acc[q + 2 * b + 4 * c] += wx[q] * wy[b] * wz[c];
}

constexpr int kGatherThreads = 256;

__global__ void __launch_bounds__(kGatherThreads) k_sort_gather(GatherArgs a) {
  const int lane = threadIdx.x & 31;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int n = a.n;
  for (int64_t cell = gw; cell < a.ncell; cell += nw) {
    const int32_t s = a.start[cell];
    const int32_t cnt = a.start[cell + 1] - s;
    if (cnt > a.big_lo && cnt <= kMaxBlockSort) continue;  // k_sort_big
    const int ci = (int)(cell % n), cj = (int)((cell / n) % n), ck = (int)(cell / ((int64_t)n * n));
    double acc[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) acc[q] = 0.0;
    if (cnt <= 32) {
      int32_t src = 0;
      uint32_t mp = 0xFFFFFFFFu;
      if (lane < cnt) {
        src = a.perm[s + lane];
        mp = a.pid_in[src];
      }
      int r = 0;
      for (int l = 0; l < cnt; ++l) {
        const uint32_t o = __shfl_sync(0xffffffffu, mp, l);
        r += o < mp ? 1 : 0;
      }
      if (lane < cnt) move_particle(a, src, s + r);
    } else {
      for (int32_t e0 = 0; e0 < cnt; e0 += 32) {
        const int32_t e = e0 + lane;
        int32_t src = 0;
        uint32_t mp = 0xFFFFFFFFu;
        if (e < cnt) {
          src = a.perm[s + e];
          mp = a.pid_in[src];
        }
        int32_t r = 0;
        for (int32_t f0 = 0; f0 < cnt; f0 += 32) {
          const uint32_t other = (f0 + lane < cnt) ? a.pid_in[a.perm[s + f0 + lane]] : 0xFFFFFFFFu;
          const int lim = min(32, cnt - f0);
          for (int l = 0; l < lim; ++l) {
            const uint32_t o = __shfl_sync(0xffffffffu, other, l);
            r += o < mp ? 1 : 0;
          }
        }
        if (e < cnt) move_particle(a, src, s + r);
      }
    }
    // CIC partials in sorted (ascending pid) order: lane l takes slots l,
    // l + 32, ... of the moved particles, so the sums do not depend on the
    // arrival order of the atomic ranks
    __syncwarp();
    for (int32_t e = lane; e < cnt; e += 32) add_cic(a, s + e, ci, cj, ck, acc);
    // fixed-shape transpose reduction of the 8 corner sums across the warp:
    // each xor level halves the values a lane keeps (4 + 2 + 1 adds), two
    // more levels finish the sum; lane l then holds corner
    // 4 [l & 16] + 2 [l & 8] + [l & 4]
    const bool u16 = lane & 16, u8 = lane & 8, u4 = lane & 4;
    double a4[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const double send = u16 ? acc[i] : acc[4 + i];
      a4[i] = (u16 ? acc[4 + i] : acc[i]) + __shfl_xor_sync(0xffffffffu, send, 16);
    }
    double a2[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const double send = u8 ? a4[i] : a4[2 + i];
      a2[i] = (u8 ? a4[2 + i] : a4[i]) + __shfl_xor_sync(0xffffffffu, send, 8);
    }
    double a1 = (u4 ? a2[1] : a2[0]) + __shfl_xor_sync(0xffffffffu, u4 ? a2[0] : a2[1], 4);
    a1 += __shfl_xor_sync(0xffffffffu, a1, 2);
    a1 += __shfl_xor_sync(0xffffffffu, a1, 1);
    if ((lane & 3) == 0) {
      const int corner = (u16 ? 4 : 0) + (u8 ? 2 : 0) + (u4 ? 1 : 0);
      a.corner[(int64_t)corner * a.ncell + cell] = a1;
    }
  }
}

// Cells of kBigCell < count <= kMaxBlockSort particles: one block per cell,
// (pid, source) pairs sorted in shared memory, particles moved in pid order,
// CIC corner partials summed with a fixed-shape block reduction.
constexpr int kBigThreads = 512;

__global__ void __launch_bounds__(kBigThreads) k_sort_big(GatherArgs a) {
  extern __shared__ uint32_t shm[];
  uint32_t* key = shm;
  int32_t* val = reinterpret_cast<int32_t*>(shm + kMaxBlockSort);
  __shared__ double red[kBigThreads / 32][8];
  const int n = a.n;
  for (int64_t cell = blockIdx.x; cell < a.ncell; cell += gridDim.x) {
    const int32_t s = a.start[cell];
    const int32_t cnt = a.start[cell + 1] - s;
    if (cnt <= a.big_lo || cnt > kMaxBlockSort) continue;  // uniform per block
    int np2 = 1;
    while (np2 < cnt) np2 <<= 1;
    for (int e = threadIdx.x; e < np2; e += blockDim.x) {
      if (e < cnt) {
        const int32_t src = a.perm[s + e];
        key[e] = a.pid_in[src];
        val[e] = src;
      } else {
        key[e] = 0xFFFFFFFFu;
        val[e] = -1;
      }
    }
    __syncthreads();
    block_bitonic_sort(key, val, np2);
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) move_particle(a, val[e], s + e);
    __syncthreads();
    const int ci = (int)(cell % n), cj = (int)((cell / n) % n), ck = (int)(cell / ((int64_t)n * n));
    double acc[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) acc[q] = 0.0;
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) add_cic(a, s + e, ci, cj, ck, acc);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], off);
      if (lane == 0) red[w][q] = acc[q];
    }
    __syncthreads();
    if (threadIdx.x < 8) {
      double t = 0.0;
      for (int ww = 0; ww < (int)(blockDim.x >> 5); ++ww) t += red[ww][threadIdx.x];
      a.corner[(int64_t)threadIdx.x * a.ncell + cell] = t;
    }
    __syncthreads();
  }
}

}  // namespace

size_t big_sort_smem() { return (size_t)kMaxBlockSort * 8; }
const void* sort_big_kernel_ptr() { return (const void*)k_sort_big; }

cudaError_t launch_keys(pic_ctx* c) {
  KeysArgs a;
  a.np = c->P.np;
  a.n = c->P.n;
  const int b = c->cur;
  a.x0 = c->x[b][0]; a.x1 = c->x[b][1]; a.x2 = c->x[b][2];
  a.key = c->key;
  a.rank = c->rank;
  a.count = c->count;
  prof_begin(c);
  k_keys<<<blocks_for(a.np), kThreads, 0, c->stream>>>(a);
  prof_end(c, KC_SORT);
  c->launches++;
  return cudaGetLastError();
}

int64_t scan_blocks_needed(int64_t ncell) { return (ncell + kScanTile - 1) / kScanTile; }

// the three scan launches (no profiling region of their own)
void enqueue_scan(pic_ctx* c) {
  c->inv_valid = false;  // a new sorted order follows
  const int64_t m = c->P.ncell;
  const int64_t nb = scan_blocks_needed(m);
  k_scan_reduce<<<(int)nb, kThreads, 0, c->stream>>>(c->count, m, c->scan_blocks);
  k_scan_blocks<<<1, 1024, 0, c->stream>>>(c->scan_blocks, nb);
  k_scan_final<<<(int)nb, kThreads, 0, c->stream>>>(c->count, m, c->scan_blocks, c->start);
  c->launches += 3;
}

cudaError_t launch_scan(pic_ctx* c) {
  prof_begin(c);
  enqueue_scan(c);
  prof_end(c, KC_SORT);
  return cudaGetLastError();
}

cudaError_t launch_scan_scatter(pic_ctx* c) {
  prof_begin(c);
  enqueue_scan(c);  // perm becomes the sort's permutation
  ScatterArgs s;
  s.np = c->P.np;
  s.key = c->key;
  s.rank = c->rank;
  s.start = c->start;
  s.perm = c->perm;
  // the precision form's gather reads each cell's pids in arrival order
  // from the output pid array (coalesced) instead of through perm; a state
  // loaded as records carries its pids in the records, which the gather
  // reads anyway, so the scatter writes only perm
  s.pid = c->mixed ? c->pid[c->cur] : nullptr;
  s.spid = c->mixed && !c->rec_state ? c->pid[1 - c->cur] : nullptr;
  k_scatter<<<blocks_for(s.np), kThreads, 0, c->stream>>>(s);
  prof_end(c, KC_SORT);
  c->launches++;
  return cudaGetLastError();
}

cudaError_t launch_sort(pic_ctx* c) {
  c->inv_valid = false;
  const int64_t m = c->P.ncell;
  cudaError_t e = launch_scan_scatter(c);
  if (e != cudaSuccess) return e;

  GatherArgs g;
  g.n = c->P.n;
  g.ncell = m;
  g.start = c->start;
  g.perm = c->perm;
  const int b = c->cur, o = 1 - c->cur;
  for (int d = 0; d < 3; ++d) {
    g.in[d] = c->x[b][d]; g.in[3 + d] = c->v[b][d]; g.in[6 + d] = c->vm[b][d];
    g.out[d] = c->x[o][d]; g.out[3 + d] = c->v[o][d]; g.out[6 + d] = c->vm[o][d];
  }
  g.pid_in = c->pid[b];
  g.pid_out = c->pid[o];
  g.corner = c->corner;
  g.big_lo = big_cell_threshold(m, c->P.np);
  const int64_t warps = m;
  // one warp per cell, blocks handed out as SMs free up
  int64_t blocks = (warps * 32 + kGatherThreads - 1) / kGatherThreads;
  if (blocks > INT_MAX) blocks = INT_MAX;  // the grid-stride loop takes the rest
  prof_begin(c);
  k_sort_gather<<<(int)blocks, kGatherThreads, 0, c->stream>>>(g);
  if (g.big_lo < INT_MAX) {
    k_sort_big<<<2 * c->num_sms, kBigThreads, big_sort_smem(), c->stream>>>(g);
    c->launches++;
  }
  prof_end(c, KC_GATHER);
  c->launches++;
  c->cur = o;
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
struct StoreSortArgs {
  int64_t np;
  int n;
  const double *x0, *x1, *x2;
  const uint32_t* pid;
  int32_t *cell_of_pid, *perm;
};

__global__ void __launch_bounds__(kThreads) k_store_sort(StoreSortArgs a) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= a.np) return;
  const int n = a.n;
  const uint32_t p = a.pid[j];
  if (a.cell_of_pid)
    a.cell_of_pid[p] = cell_coord(a.x0[j], n) + n * (cell_coord(a.x1[j], n) + n * cell_coord(a.x2[j], n));
  if (a.perm) a.perm[j] = (int32_t)p;
}

cudaError_t launch_store_sort(pic_ctx* c, int32_t* cell_of_pid, int32_t* perm) {
  StoreSortArgs a;
  a.np = c->P.np;
  a.n = c->P.n;
  const int b = c->cur;
  a.x0 = c->x[b][0]; a.x1 = c->x[b][1]; a.x2 = c->x[b][2];
  a.pid = c->pid[b];
  a.cell_of_pid = cell_of_pid;
  a.perm = perm;
  prof_begin(c);
  k_store_sort<<<blocks_for(a.np), kThreads, 0, c->stream>>>(a);
  prof_end(c, KC_OTHER);
  c->launches++;
  return cudaGetLastError();
}

}  // namespace pic
