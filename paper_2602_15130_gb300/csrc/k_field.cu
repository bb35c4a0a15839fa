// Field solve of Eq. poisson_mms on the periodic node mesh:
//   rhs : rho at nodes from the per-cell CIC partials, b = rho/eps0 -
//         Lap phi^M - rho^M/eps0 and per-block partial sums of b;
//   cg  : one cooperative persistent kernel: b -= mean(b), conjugate
//         gradients on -Lap_h phi = b (7-point, warm start, three grid
//         barriers per iteration: p update, q = A p with p.q, x/r update
//         with r.r), zero-mean projection and E = -grad_h phi by central
//         differences.
// All reductions are per-block partials combined in a fixed order, so a
// solve is deterministic for a given grid. Grid barriers are bounded: a
// wait that exceeds ~2 s of SM clock sets a timeout flag and the kernel
// returns.
#include "pic_internal.cuh"

namespace pic {
namespace {

constexpr int kThreads = 256;
constexpr long long kBarrierCycles = 4000000000LL;

inline int blocks_for(int64_t n, int t = kThreads) {
  int64_t b = (n + t - 1) / t;
  return (int)(b < 1 ? 1 : b);
}

// fixed-shape block sum (sh holds at least 33 doubles); thread 0 adds the
// warp totals and the result is broadcast to every thread
__device__ __forceinline__ double block_sum(double v, double* sh) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < nw; ++i) t += sh[i];
    sh[32] = t;
  }
  __syncthreads();
  return sh[32];
}

struct RhsArgs {
  Params P;
  TimeTerms tt;
  const double* corner;
  double *rho, *b, *part;
  float* b32;  // precision form: b in FP32 (b may then be null)
};

__global__ void __launch_bounds__(kThreads) k_rhs(RhsArgs a) {
  __shared__ double sh[40];
  const Params& P = a.P;
  const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double bv = 0.0;
  if (id < P.ncell) {
    const int n = P.n;
    const int i = (int)(id % n), j = (int)((id / n) % n), k = (int)(id / ((int64_t)n * n));
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int b = 0; b < 2; ++b)
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const int ii = i - q < 0 ? n - 1 : i - q, jj = j - b < 0 ? n - 1 : j - b, kk = k - c < 0 ? n - 1 : k - c;
          s += a.corner[(int64_t)(q + 2 * b + 4 * c) * P.ncell + ii + (int64_t)n * (jj + (int64_t)n * kk)];
        }
    const double rho = P.rho_scale * s;
    const double X = i * P.h, Y = j * P.h, Z = k * P.h;
    const double ct = a.tt.ct;
    const double phiM = a.tt.em_amp / kTwoPi * sinpi(2.0 * (X - P.phi_shift[0])) *
                        sinpi(2.0 * (Y - P.phi_shift[1])) * sinpi(2.0 * (Z - P.phi_shift[2]));
    const double lap_phiM = -3.0 * kTwoPi * kTwoPi * phiM;
    const double rhoM =
        P.dist == PIC_DIST_PAPER
            ? P.q_eff * P.nphys * (1.0 + a.tt.fA[0] * sinpi(2.0 * (X - a.tt.fs[0]))) *
                  (1.0 + a.tt.fA[1] * sinpi(2.0 * (Y - a.tt.fs[1]))) * (1.0 + a.tt.fA[2] * sinpi(2.0 * (Z - a.tt.fs[2])))
            : P.q_eff * P.nphys * (1.0 + P.fx_amp * sinpi(2.0 * (X - ct))) * (1.0 + P.fx_amp * sinpi(2.0 * (Y - ct))) *
                  (1.0 + P.fx_amp * sinpi(2.0 * (Z - ct)));
    bv = rho / P.eps0 - lap_phiM - rhoM / P.eps0;
    a.rho[id] = rho;
    if (a.b) a.b[id] = bv;
    if (a.b32) a.b32[id] = (float)bv;
  }
  const double tot = block_sum(bv, sh);
  if (threadIdx.x == 0) a.part[blockIdx.x] = tot;
}

// Precision form: the same RHS with the manufactured terms in FP32 (the
// FP64 pipe is slow on this part); the corner sums, rho and the block
// partial of the mean stay FP64.
struct Rhs32Consts {
  float h, two_pi_over, lap_scale;   // h, phi^M amplitude / (2 pi) * e^{t/2T}, -3 (2 pi)^2
  float shift[3], ct, fx_amp;
  float rhoM_scale, inv_eps0;         // q N, 1/eps0
  int paper;                          // PIC_DIST_PAPER: per-axis amplitude fA and phase fs
  float fA[3], fs[3];
};

__global__ void __launch_bounds__(kThreads) k_rhs32(RhsArgs a, Rhs32Consts k) {
  __shared__ double sh[40];
  const Params& P = a.P;
  const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double bsum = 0.0;
  if (id < P.ncell) {
    const int n = P.n;
    const int i = (int)(id % n), j = (int)((id / n) % n), kk0 = (int)(id / ((int64_t)n * n));
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int b = 0; b < 2; ++b)
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const int ii = i - q < 0 ? n - 1 : i - q, jj = j - b < 0 ? n - 1 : j - b, kk = kk0 - c < 0 ? n - 1 : kk0 - c;
          s += a.corner[(int64_t)(q + 2 * b + 4 * c) * P.ncell + ii + (int64_t)n * (jj + (int64_t)n * kk)];
        }
    const double rho = P.rho_scale * s;
    const float X = (float)i * k.h, Y = (float)j * k.h, Z = (float)kk0 * k.h;
    const float phiM = k.two_pi_over * sinpif(2.f * (X - k.shift[0])) * sinpif(2.f * (Y - k.shift[1])) *
                       sinpif(2.f * (Z - k.shift[2]));
    const float rhoM =
        k.paper ? k.rhoM_scale * (1.f + k.fA[0] * sinpif(2.f * (X - k.fs[0]))) *
                      (1.f + k.fA[1] * sinpif(2.f * (Y - k.fs[1]))) * (1.f + k.fA[2] * sinpif(2.f * (Z - k.fs[2])))
                : k.rhoM_scale * (1.f + k.fx_amp * sinpif(2.f * (X - k.ct))) *
                      (1.f + k.fx_amp * sinpif(2.f * (Y - k.ct))) * (1.f + k.fx_amp * sinpif(2.f * (Z - k.ct)));
    const float bv = (float)(rho * (double)k.inv_eps0) - k.lap_scale * phiM - rhoM * k.inv_eps0;
    a.rho[id] = rho;
    a.b32[id] = bv;
    bsum = (double)bv;
  }
  const double tot = block_sum(bsum, sh);
  if (threadIdx.x == 0) a.part[blockIdx.x] = tot;
}

struct CgArgs {
  int n;
  int64_t ncell;
  double inv_h2, two_h;
  double *b, *x, *r, *p0, *p1, *q;
  const double* rhs_part;
  int rhs_blocks;
  double* red;  // [4][gridDim.x]
  unsigned int* bar;
  int* info;    // [0] iterations [1] status (1 = no convergence) [2] timeout
  int* flags;   // sticky context flags
  double* res;
  int skip_block = -1;  // failure injection: this block leaves before its first barrier
  double tol;
  int maxit;
  double *E0, *E1, *E2;
  long long* hist = nullptr;  // per-step history row: [0] iterations
};

// Grid barrier for a cooperative grid, bounded in time.
__device__ __forceinline__ bool grid_barrier(unsigned int* bar, int* info, int* flags) {
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

// total of gridDim.x partials in fixed order, in every thread
__device__ __forceinline__ double grid_total(const double* part, int m, double* sh) {
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

// the six periodic neighbours of node id = i + n (j + n k), 32-bit indices
// (n^3 < 2^31): x+, x-, y+, y-, z+, z-
struct Nbr {
  int xp, xm, yp, ym, zp, zm;
};
__device__ __forceinline__ Nbr neighbours(int id, int n, int nn) {
  const int i = id % n, j = (id / n) % n, k = id / nn;
  Nbr b;
  b.xp = i == n - 1 ? id - (n - 1) : id + 1;
  b.xm = i == 0 ? id + (n - 1) : id - 1;
  b.yp = j == n - 1 ? id - (n - 1) * n : id + n;
  b.ym = j == 0 ? id + (n - 1) * n : id - n;
  b.zp = k == n - 1 ? id - (n - 1) * nn : id + nn;
  b.zm = k == 0 ? id + (n - 1) * nn : id - nn;
  return b;
}

// One block per SM of 1024 threads keeps the grid barriers and the
// per-block partial sums short.
constexpr int kCgThreads = 1024;

__global__ void __launch_bounds__(kCgThreads) k_cg(CgArgs a) {
  __shared__ double sh[40];
  __shared__ double scal[2];  // scalars formed once per block by thread 0
  __shared__ int stop;
  const int n = a.n, nn = a.n * a.n;
  const int m = (int)a.ncell;
  const int stride = gridDim.x * blockDim.x;
  const int t0 = blockIdx.x * blockDim.x + threadIdx.x;
  const int G = gridDim.x;
  int ph = 0;  // alternating reduction slots
  auto slot = [&](int q) { return a.red + (size_t)q * 2 * G; };
  // the others then wait for an arrival that never comes, until the bound
  if ((int)blockIdx.x == a.skip_block) return;

  // phase 0: zero-mean b, r = b - A x, ||r||^2 and ||b||^2
  const double mean_b = grid_total(a.rhs_part, a.rhs_blocks, sh) / (double)m;
  double rr_loc = 0.0, bb_loc = 0.0;
  for (int id = t0; id < m; id += stride) {
    const Nbr q = neighbours(id, n, nn);
    const double bv = a.b[id] - mean_b;
    a.b[id] = bv;
    const double* x = a.x;
    const double nb = x[q.xp] + x[q.xm] + x[q.yp] + x[q.ym] + x[q.zp] + x[q.zm];
    const double Ax = (6.0 * x[id] - nb) * a.inv_h2;
    const double rv = bv - Ax;
    a.r[id] = rv;
    rr_loc += rv * rv;
    bb_loc += bv * bv;
  }
  {
    const double s1 = block_sum(rr_loc, sh);
    if (threadIdx.x == 0) slot(ph)[blockIdx.x] = s1;
    const double s2 = block_sum(bb_loc, sh);
    if (threadIdx.x == 0) slot(ph)[G + blockIdx.x] = s2;
  }
  if (!grid_barrier(a.bar, a.info, a.flags)) return;
  double rr = grid_total(slot(ph), G, sh);
  const double bb = grid_total(slot(ph) + G, G, sh);
  ph ^= 1;
  double beta = 0.0;
  int it = 0, status = 0;
  double* p = a.p0;
  const double thresh = a.tol * sqrt(bb);
  while (true) {
    if (threadIdx.x == 0) stop = (bb == 0.0 || sqrt(rr) <= thresh) ? 1 : (it >= a.maxit ? 2 : 0);
    __syncthreads();
    if (stop == 1) break;
    if (stop == 2) { status = 1; break; }
    // p = r + beta p
    if (it == 0) {
      for (int id = t0; id < m; id += stride) p[id] = a.r[id];
    } else {
      for (int id = t0; id < m; id += stride) p[id] = a.r[id] + beta * p[id];
    }
    if (!grid_barrier(a.bar, a.info, a.flags)) return;
    // q = A p, p.q
    double pq_loc = 0.0;
    for (int id = t0; id < m; id += stride) {
      const Nbr q = neighbours(id, n, nn);
      const double nb = p[q.xp] + p[q.xm] + p[q.yp] + p[q.ym] + p[q.zp] + p[q.zm];
      const double pc = p[id];
      const double qv = (6.0 * pc - nb) * a.inv_h2;
      a.q[id] = qv;
      pq_loc += pc * qv;
    }
    {
      const double s = block_sum(pq_loc, sh);
      if (threadIdx.x == 0) slot(ph)[blockIdx.x] = s;
    }
    if (!grid_barrier(a.bar, a.info, a.flags)) return;
    const double pq = grid_total(slot(ph), G, sh);
    ph ^= 1;
    if (threadIdx.x == 0) scal[0] = rr / pq;
    __syncthreads();
    const double alpha = scal[0];
    double rn_loc = 0.0;
    for (int id = t0; id < m; id += stride) {
      a.x[id] += alpha * p[id];
      const double rv = a.r[id] - alpha * a.q[id];
      a.r[id] = rv;
      rn_loc += rv * rv;
    }
    {
      const double s = block_sum(rn_loc, sh);
      if (threadIdx.x == 0) slot(ph)[blockIdx.x] = s;
    }
    if (!grid_barrier(a.bar, a.info, a.flags)) return;
    const double rr_new = grid_total(slot(ph), G, sh);
    ph ^= 1;
    ++it;
    if (threadIdx.x == 0) scal[1] = rr_new / rr;
    __syncthreads();
    beta = scal[1];
    rr = rr_new;
  }
  // zero-mean projection
  double xs = 0.0;
  for (int id = t0; id < m; id += stride) xs += a.x[id];
  {
    const double s = block_sum(xs, sh);
    if (threadIdx.x == 0) slot(ph)[blockIdx.x] = s;
  }
  if (!grid_barrier(a.bar, a.info, a.flags)) return;
  const double mean_x = grid_total(slot(ph), G, sh) / (double)m;
  ph ^= 1;
  for (int id = t0; id < m; id += stride) a.x[id] -= mean_x;
  if (!grid_barrier(a.bar, a.info, a.flags)) return;
  // E = -grad_h phi, second-order central differences
  for (int id = t0; id < m; id += stride) {
    const Nbr q = neighbours(id, n, nn);
    const double* x = a.x;
    a.E0[id] = -(x[q.xp] - x[q.xm]) / a.two_h;
    a.E1[id] = -(x[q.yp] - x[q.ym]) / a.two_h;
    a.E2[id] = -(x[q.zp] - x[q.zm]) / a.two_h;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    a.info[0] = it;
    a.info[1] = status;
    if (a.hist) a.hist[0] = it;
    a.res[0] = bb > 0.0 ? sqrt(rr) / sqrt(bb) : 0.0;
    if (status) atomicOr(a.flags, 2);
    atomicMax(a.flags + 1, it);
  }
}

struct StoreFieldArgs {
  int64_t ncell;
  const double *rho, *phi, *E0, *E1, *E2;
  double *orho, *ophi, *oE;
};

__global__ void __launch_bounds__(kThreads) k_store_field(StoreFieldArgs a) {
  const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= a.ncell) return;
  if (a.orho) a.orho[id] = a.rho[id];
  if (a.ophi) a.ophi[id] = a.phi[id];
  if (a.oE) {
    a.oE[3 * id] = a.E0[id];
    a.oE[3 * id + 1] = a.E1[id];
    a.oE[3 * id + 2] = a.E2[id];
  }
}

}  // namespace

int rhs_blocks_needed(int64_t ncell) { return blocks_for(ncell); }

cudaError_t launch_rhs(pic_ctx* c, double t) {
  RhsArgs a;
  a.P = c->P;
  a.tt = time_terms(c->P, t);
  a.corner = c->corner;
  a.rho = c->rho;
  a.b = c->mixed ? nullptr : c->b;
  a.b32 = c->mixed ? c->bf : nullptr;
  a.part = c->rhs_part;
  prof_begin(c);
  if (c->mixed) {
    Rhs32Consts k;
    k.h = (float)c->P.h;
    k.two_pi_over = (float)(a.tt.em_amp / kTwoPi);
    k.lap_scale = (float)(-3.0 * kTwoPi * kTwoPi);
    for (int d = 0; d < 3; ++d) k.shift[d] = (float)c->P.phi_shift[d];
    k.ct = (float)(a.tt.ct - floor(a.tt.ct));
    k.fx_amp = (float)c->P.fx_amp;
    k.rhoM_scale = (float)(c->P.q_eff * c->P.nphys);
    k.inv_eps0 = (float)(1.0 / c->P.eps0);
    k.paper = c->P.dist == PIC_DIST_PAPER;
    for (int d = 0; d < 3; ++d) {
      k.fA[d] = (float)a.tt.fA[d];
      k.fs[d] = (float)(a.tt.fs[d] - floor(a.tt.fs[d]));
    }
    k_rhs32<<<(int)c->rhs_blocks, kThreads, 0, c->stream>>>(a, k);
  } else {
    k_rhs<<<(int)c->rhs_blocks, kThreads, 0, c->stream>>>(a);
  }
  prof_end(c, KC_RHS);
  c->launches++;
  return cudaGetLastError();
}

int cg_threads() { return kCgThreads; }
const void* cg_kernel_ptr() { return (const void*)k_cg; }

cudaError_t launch_cg_on(pic_ctx* c, double* b, double* x, const double* rhs_part, int rhs_blocks, double* E0,
                         double* E1, double* E2) {
  CgArgs a;
  a.n = c->P.n;
  a.ncell = c->P.ncell;
  a.inv_h2 = (double)c->P.n * (double)c->P.n;
  a.two_h = 2.0 * c->P.h;
  a.b = b;
  a.x = x;
  a.r = c->cg_r;
  a.p0 = c->cg_p[0];
  a.p1 = c->cg_p[1];
  a.q = c->cg_q;
  a.rhs_part = rhs_part;
  a.rhs_blocks = rhs_blocks;
  a.red = c->cg_red;
  a.bar = c->cg_bar;
  a.info = c->cg_info;
  a.flags = c->flags;
  a.res = c->cg_res;
  a.tol = c->cfg.cg_tol;
  a.maxit = c->cfg.cg_maxit;
  a.E0 = E0;
  a.E1 = E1;
  a.E2 = E2;
  a.skip_block = c->stall_next_cg ? c->cg_grid - 1 : -1;
  a.hist = c->hist_row;
  c->stall_next_cg = false;
  cudaError_t e = cudaMemsetAsync(c->cg_bar, 0, 2 * sizeof(unsigned int), c->stream);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(c->cg_info, 0, 3 * sizeof(int), c->stream);
  if (e != cudaSuccess) return e;
  void* args[] = {&a};
  prof_begin(c);
  e = cudaLaunchCooperativeKernel((const void*)k_cg, dim3(c->cg_grid), dim3(kCgThreads), args, 0, c->stream);
  prof_end(c, KC_CG);
  c->launches++;
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

cudaError_t launch_cg(pic_ctx* c) {
  return launch_cg_on(c, c->b, c->phi, c->rhs_part, (int)c->rhs_blocks, c->E[0], c->E[1], c->E[2]);
}

cudaError_t launch_store_field(pic_ctx* c, double* rho, double* phi, double* E) {
  StoreFieldArgs a;
  a.ncell = c->P.ncell;
  a.rho = c->rho;
  a.phi = c->phi;
  a.E0 = c->E[0];
  a.E1 = c->E[1];
  a.E2 = c->E[2];
  a.orho = rho;
  a.ophi = phi;
  a.oE = E;
  prof_begin(c);
  k_store_field<<<blocks_for(a.ncell), kThreads, 0, c->stream>>>(a);
  prof_end(c, KC_OTHER);
  c->launches++;
  return cudaGetLastError();
}

}  // namespace pic

// ---------------------------------------------------------------------------
// Allocation-free Poisson solve (pic_poisson_solve_noalloc).
//
// Some callers cannot allocate device memory at solve time: code running
// under a memory budget fixed at start-up, or a host framework that forbids
// cudaMalloc/cudaFree on its hot path because they synchronise the device.
// For them the CG scratch lives in this one fixed array in the library's own
// device memory: every GPU that loads the library holds it until the process
// exits. Host code must not use the array's name as a device address; it
// looks the address up once per device with cudaGetSymbolAddress.
// ---------------------------------------------------------------------------
#include <mutex>

namespace pic {
namespace {

constexpr int64_t kNoallocMaxNodes = 48 * 48 * 48;   // largest mesh: 48^3 nodes
constexpr int kNoallocMaxGrid = 4096;                  // cooperative blocks
constexpr int64_t kNoallocPartBlocks = (kNoallocMaxNodes + kThreads - 1) / kThreads;
// layout in doubles: b copy, r, p0, p1, q [5 N]; partial sums of b; CG
// reduction slots [4 grid]; 16 words of barrier / status / residual
constexpr int64_t kNoallocDoubles = 5 * kNoallocMaxNodes + kNoallocPartBlocks + 4 * kNoallocMaxGrid + 16;

static __device__ __align__(256) double g_noalloc_scratch[kNoallocDoubles];

std::mutex g_noalloc_mutex;
double* g_noalloc_ptr[64] = {nullptr};

// copy b into the scratch and write per-block partial sums for its mean
__global__ void __launch_bounds__(kThreads) k_noalloc_prep(const double* b, double* bcopy, double* part, int64_t m) {
  __shared__ double sh[40];
  const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double v = 0.0;
  if (id < m) {
    v = b[id];
    bcopy[id] = v;
  }
  const double tot = block_sum(v, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

}  // namespace
}  // namespace pic

extern "C" pic_status pic_poisson_solve_noalloc(int32_t n, const double* b, double* phi, double* E, double tol,
                                                int32_t maxit, void* cuda_stream, int32_t* iters, double* rel_res) {
  using namespace pic;
  if (n < 2 || b == nullptr || phi == nullptr || E == nullptr || !(tol > 0.0) || maxit < 1) return PIC_EINVAL;
  const int64_t m = (int64_t)n * n * n;
  if (m > kNoallocMaxNodes) return PIC_EINVAL;  // beyond the fixed scratch: n <= 48
  cudaStream_t stream = (cudaStream_t)cuda_stream;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return PIC_ECUDA;
  }
  // b, phi and E must be device memory of the current device
  const void* ptrs[3] = {b, phi, E};
  for (const void* p : ptrs) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
      cudaGetLastError();
      return PIC_EINVAL;
    }
    if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) return PIC_EINVAL;
    // device memory of another GPU would be read across the link, or fault
    // without peer access: only the current device's memory is accepted
    if (at.type == cudaMemoryTypeDevice && at.device != dev) return PIC_EINVAL;
  }
  // one-time set-up per device: the scratch array's device address
  double* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) {
        cudaGetLastError();
        return PIC_ECUDA;
      }
      g_noalloc_ptr[dev] = (double*)p;
    }
    base = g_noalloc_ptr[dev];
  }
  int sms = 0, occ = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_cg, kThreads, 0) != cudaSuccess || occ < 1) {
    cudaGetLastError();
    return PIC_ECUDA;
  }
  int64_t grid = (m + kThreads - 1) / kThreads;
  if (grid > (int64_t)occ * sms) grid = (int64_t)occ * sms;
  if (grid > kNoallocMaxGrid) grid = kNoallocMaxGrid;
  const int part_blocks = (int)((m + kThreads - 1) / kThreads);

  double* bcopy = base;
  double* part = base + 5 * kNoallocMaxNodes;
  double* red = part + kNoallocPartBlocks;
  int* words = (int*)(red + 4 * kNoallocMaxGrid);   // [0,1] barrier, [2..4] info, [5,6] flags
  double* res = (double*)(words + 8);

  CgArgs a;
  a.n = n;
  a.ncell = m;
  a.inv_h2 = (double)n * (double)n;
  a.two_h = 2.0 * (1.0 / (double)n);
  a.b = bcopy;
  a.x = phi;
  a.r = base + kNoallocMaxNodes;
  a.p0 = base + 2 * kNoallocMaxNodes;
  a.p1 = base + 3 * kNoallocMaxNodes;
  a.q = base + 4 * kNoallocMaxNodes;
  a.rhs_part = part;
  a.rhs_blocks = part_blocks;
  a.red = red;
  a.bar = (unsigned int*)words;
  a.info = words + 2;
  a.flags = words + 5;
  a.res = res;
  a.tol = tol;
  a.maxit = maxit;
  a.E0 = E;
  a.E1 = E + m;
  a.E2 = E + 2 * m;
  // the array keeps the last call's contents: clear the barrier and status words
  cudaError_t e = cudaMemsetAsync(words, 0, 8 * sizeof(int), stream);
  if (e == cudaSuccess) {
    k_noalloc_prep<<<part_blocks, kThreads, 0, stream>>>(b, bcopy, part, m);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    void* args[] = {&a};
    e = cudaLaunchCooperativeKernel((const void*)k_cg, dim3((unsigned)grid), dim3(kThreads), args, 0, stream);
  }
  int info[5] = {0, 0, 0, 0, 0};
  double r = 0.0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(info, words + 2, 5 * sizeof(int), cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&r, res, sizeof(double), cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return PIC_ECUDA;
  }
  if (iters) *iters = info[0];
  if (rel_res) *rel_res = r;
  if (info[2]) return PIC_ETIMEOUT;
  if (info[1]) return PIC_ENOCONV;
  return PIC_OK;
}
