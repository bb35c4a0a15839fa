// Host runtime and C ABI (include/pic.h): configuration checks, derived
// constants, device buffers, the step schedule of Eq. velocity_verlet and
// the boundary: caller arrays in device or pinned host memory are read and
// written by the kernels in place, pageable ones are staged through a copy.
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <new>

#include "pic_internal.cuh"

namespace pic {
int dsmc_threads();
const void* dsmc_kernel_ptr(bool verify);
int cg_threads();
const void* cg_kernel_ptr();
int64_t scan_blocks_needed(int64_t ncell);
int rhs_blocks_needed(int64_t ncell);
int err_blocks_needed(int64_t np, int64_t ncell);
int dsmc32_threads();
size_t dsmc32_smem_bytes(int bm_words);
const void* dsmc32_kernel_ptr(bool verify);
int batch_dsmc_threads();
const void* batch_dsmc_kernel_ptr();
const void* sort_big_kernel_ptr();
const void* sort_big32_kernel_ptr();

// the big-cell sorts keep kMaxBlockSort (pid, source) pairs in shared memory
cudaError_t allow_big_sort_smem() {
  const int bytes = kMaxBlockSort * 8;
  cudaError_t e = cudaFuncSetAttribute(sort_big_kernel_ptr(), cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(sort_big32_kernel_ptr(), cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  return e;
}
int cg32_threads();
const void* cg32_kernel_ptr();

// Resolve recorded event pairs into per-class totals (synchronises).
void prof_flush(pic_ctx* c) {
  if (c->ev_used == 0) return;
  cudaEventSynchronize(c->ev_pool[2 * (c->ev_used - 1) + 1]);
  for (int i = 0; i < c->ev_used; ++i) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, c->ev_pool[2 * i], c->ev_pool[2 * i + 1]) == cudaSuccess) {
      c->prof_ms[c->ev_class[i]] += ms;
      c->prof_launches[c->ev_class[i]] += 1;
    }
  }
  c->ev_used = 0;
  cudaGetLastError();
}

static bool prof_slot(pic_ctx* c) {
  if (c->ev_used < c->ev_cap) return true;
  if (c->ev_cap >= 1 << 16) {
    prof_flush(c);
    return true;
  }
  const int cap = c->ev_cap ? 2 * c->ev_cap : 256;
  cudaEvent_t* pool = (cudaEvent_t*)realloc(c->ev_pool, sizeof(cudaEvent_t) * 2 * cap);
  if (!pool) return false;
  c->ev_pool = pool;
  int* cls = (int*)realloc(c->ev_class, sizeof(int) * cap);
  if (!cls) return false;
  c->ev_class = cls;
  for (int i = 2 * c->ev_cap; i < 2 * cap; ++i)
    if (cudaEventCreate(&c->ev_pool[i]) != cudaSuccess) {
      for (int j = 2 * c->ev_cap; j < i; ++j) cudaEventDestroy(c->ev_pool[j]);
      cudaGetLastError();
      return false;
    }
  c->ev_cap = cap;
  return true;
}

void prof_begin(pic_ctx* c) {
  if (!c->profiling || !prof_slot(c)) return;
  cudaEventRecord(c->ev_pool[2 * c->ev_used], c->stream);
}
void prof_end(pic_ctx* c, int kclass) {
  if (!c->profiling || c->ev_used >= c->ev_cap) return;
  cudaEventRecord(c->ev_pool[2 * c->ev_used + 1], c->stream);
  c->ev_class[c->ev_used] = kclass;
  c->ev_used++;
}
}  // namespace pic

using namespace pic;

namespace {

constexpr int kGinvM = 1024;

// Knots of G^{-1}, G(y) = y - a cos(2 pi y), a = A/(2 pi), at T_k = k/M:
// y_k by Newton in FP64 (converged to |dy| < 1e-16) and the slope
// dy/dT = 1/G'(y_k) = 1/(1 + A sin(2 pi y_k)).
void ginv_table(double A, double* out) {
  const double a = A / (2.0 * kPi);
  for (int k = 0; k <= kGinvM; ++k) {
    const double T = (double)k / kGinvM;
    double y = T;
    for (int it = 0; it < 100; ++it) {
      const double dy = (y - a * cos(2.0 * kPi * y) - T) / (1.0 + A * sin(2.0 * kPi * y));
      y -= dy;
      if (fabs(dy) < 1e-16) break;
    }
    out[2 * k] = y;
    out[2 * k + 1] = 1.0 / (1.0 + A * sin(2.0 * kPi * y));
  }
}

void series_coefficients(double* out);

// R(a) and R'(a) in FP64: the even series sqrt(2/pi) sum_j c_j a^{2j} below
// a = 1/2, the closed form above (see hs_R).
void hs_R_host(double a, const double* ser, double* R, double* dR) {
  if (a < 0.5) {
    double r = 0.0, d = 0.0;
    for (int j = kSeriesTerms - 1; j >= 0; --j) r = r * a * a + ser[j];
    for (int j = kSeriesTerms - 1; j >= 1; --j) d = d * a * a + 2.0 * j * ser[j];
    *R = r;
    *dR = d * a;
    return;
  }
  const double s = sqrt(2.0 / kPi), e = exp(-0.5 * a * a), f = erf(a / sqrt(2.0));
  *R = s * (1.0 + 1.0 / (a * a)) * e + (a + 2.0 / a - 1.0 / (a * a * a)) * f;
  *dR = s * e * (1.0 / a - 3.0 / (a * a * a)) + (1.0 - 2.0 / (a * a) + 3.0 / (a * a * a * a)) * f;
}

// FP32 tables of the precision form: the knots of G^{-1} (y_k, dy/dT) and
// behind them those of s(T) = sin(2 pi G^{-1}(T)), the one quantity the
// drift's xdot^M needs, with its exact slope ds/dT = 2 pi cos(2 pi y_k)
// dy/dT (cubic Hermite interpolation error of s below 1e-10 at M = 1024).
void ginv_table_f(const double* tab, float* tabf) {
  for (int k = 0; k < 2 * (kGinvM + 1); ++k) tabf[k] = (float)tab[k];
  float* st = tabf + 2 * (kGinvM + 1);
  for (int k = 0; k <= kGinvM; ++k) {
    const double y = tab[2 * k], dy = tab[2 * k + 1];
    st[2 * k] = (float)sin(2.0 * kPi * y);
    st[2 * k + 1] = (float)(2.0 * kPi * cos(2.0 * kPi * y) * dy);
  }
  // then the knots (R, dR/da) of the hard-sphere moment on [0, kRTabAmax]
  double ser[kSeriesTerms];
  series_coefficients(ser);
  float* rt = tabf + 4 * (kGinvM + 1);
  for (int k = 0; k <= kRTabM; ++k) {
    double R, dR;
    hs_R_host((double)k * (double)kRTabAmax / kRTabM, ser, &R, &dR);
    rt[2 * k] = (float)R;
    rt[2 * k + 1] = (float)dR;
  }
}

// R(a) small-argument series: R = sqrt(2/pi) sum_j c_j a^{2j},
// c_j = d_j + d_{j+1} + e_{j-1} + 2 e_j - e_{j+1}, with d_k the Taylor
// coefficients of e^{-a^2/2} and e_k those of sqrt(pi/2) erf(a/sqrt 2).
void series_coefficients(double* out) {
  double d[kSeriesTerms + 2], e[kSeriesTerms + 2];
  double fact = 1.0, pw = 1.0;
  for (int k = 0; k < kSeriesTerms + 2; ++k) {
    if (k > 0) { fact *= k; pw *= 2.0; }
    const double sg = (k & 1) ? -1.0 : 1.0;
    d[k] = sg / (pw * fact);
    e[k] = sg / (pw * fact * (2.0 * k + 1.0));
  }
  const double s = sqrt(2.0 / kPi);
  for (int j = 0; j < kSeriesTerms; ++j)
    out[j] = s * (d[j] + d[j + 1] + (j > 0 ? e[j - 1] : 0.0) + 2.0 * e[j] - e[j + 1]);
}

// (sigma g)_max over g in [0, g_max] (Sec. 5.2). Odd-power sigma: sigma(g)
// g = sum_k sigma_k u^k with u = g^2 is a polynomial of degree < 3 in u, so
// its maximum is at u = 0, u = g_max^2 or the stationary point.
double poly_sg(const pic_config& c, double u) {
  double sum = 0.0, uk = 1.0;
  for (int k = 0; k < c.n_sigma; ++k) {
    sum += c.sigma_n[k] * uk;
    uk *= u;
  }
  return sum;
}
double sg_max_of(const pic_config& c) {
  if (c.n_sigma == 0) return c.sigma0 * c.g_max;
  const double u1 = c.g_max * c.g_max;
  double best = poly_sg(c, 0.0);
  const double e = poly_sg(c, u1);
  if (e > best) best = e;
  if (c.n_sigma == 3 && c.sigma_n[2] != 0.0) {
    const double us = -c.sigma_n[1] / (2.0 * c.sigma_n[2]);
    if (us > 0.0 && us < u1) {
      const double m = poly_sg(c, us);
      if (m > best) best = m;
    }
  }
  return best;
}
// smallest sigma(g) g on [0, g_max] (the same candidates)
double sg_min_of(const pic_config& c) {
  const double u1 = c.g_max * c.g_max;
  double lo = poly_sg(c, 0.0);
  const double e = poly_sg(c, u1);
  if (e < lo) lo = e;
  if (c.n_sigma == 3 && c.sigma_n[2] != 0.0) {
    const double us = -c.sigma_n[1] / (2.0 * c.sigma_n[2]);
    if (us > 0.0 && us < u1) {
      const double m = poly_sg(c, us);
      if (m < lo) lo = m;
    }
  }
  return lo;
}

void derive_params(const pic_config& c, Params& P) {
  memset(&P, 0, sizeof(P));
  P.n = c.n;
  P.K = c.K;
  P.ncell = (int64_t)c.n * c.n * c.n;
  P.np = c.n_particles;
  P.dt = c.dt;
  P.qm_eff = c.couple_qm_zero ? 0.0 : c.qm;
  P.q_eff = c.couple_q_zero ? 0.0 : c.q;
  P.eps0 = c.eps0;
  P.nphys = c.n_phys;
  P.sigma0 = c.sigma0;
  P.gmax = c.g_max;
  P.fx_amp = c.fx_amp;
  P.fx_speed = c.fx_speed;
  P.fx_amp_over_2pi = c.fx_amp / (2.0 * kPi);
  for (int d = 0; d < 3; ++d) {
    P.vmean[d] = c.v_mean[d];
    P.phi_shift[d] = c.phi_shift[d];
  }
  P.vsig = c.v_sigma;
  P.inv_vsig = 1.0 / c.v_sigma;
  P.phi_amp = c.phi_amp;
  P.phi_T = c.phi_T;
  P.key0 = (uint32_t)(c.seed & 0xFFFFFFFFull);
  P.key1 = (uint32_t)(c.seed >> 32);
  P.h = 1.0 / (double)c.n;
  P.dV = P.h * P.h * P.h;
  P.w = c.n_phys / (double)c.n_particles;
  P.sg_max = sg_max_of(c);
  P.pmax = P.sg_max * P.w * c.dt / P.dV;
  P.dist = c.dist;
  P.n_sigma = c.n_sigma;
  for (int k = 0; k < 3; ++k) P.sigma_n[k] = k < c.n_sigma ? c.sigma_n[k] : 0.0;
  P.src_pref_n = P.w * c.dt / (2.0 * P.dV);
  P.vbar = c.v_bar;
  P.t_ref = c.t_ref;
  P.rho_scale = P.q_eff * P.w / P.dV;
  P.src_pref = P.w * c.dt * c.sigma0 / (2.0 * P.dV);
  series_coefficients(P.R_series);
  P.verify = c.verify;
  P.ang_hist = nullptr;
}

pic_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return PIC_OK;
  if (e == cudaErrorMemoryAllocation) return PIC_ENOMEM;
  return PIC_ECUDA;
}

void* dev_alloc(pic_ctx* c, size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (c->have_alloc) return c->alloc.alloc(c->alloc.user, (uint64_t)bytes);
  void* p = nullptr;
  if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return p;
}

void dev_free(pic_ctx* c, void* p) {
  if (!p) return;
  if (c->have_alloc) c->alloc.free(c->alloc.user, p);
  else cudaFree(p);
}

#define CK(expr)                                   \
  do {                                             \
    cudaError_t e_ = (expr);                       \
    if (e_ != cudaSuccess) return cuda_status(e_); \
  } while (0)

// Every device array of the context, in one list for allocation and release.
template <class F>
void for_each_buffer(pic_ctx* c, F f) {
  const size_t np = (size_t)c->P.np, nc = (size_t)c->P.ncell;
  const size_t warps = c->overlay_warps > 0 ? (size_t)c->overlay_warps : (size_t)c->dsmc_grid * (c->dsmc_block / 32);
  const size_t lanes = warps * 32 * (size_t)c->cfg.max_ppc * 3;
  if (!c->mixed) {
    for (int b = 0; b < 2; ++b)
      for (int d = 0; d < 3; ++d) {
        f((void**)&c->x[b][d], np * 8);
        f((void**)&c->v[b][d], np * 8);
        f((void**)&c->vm[b][d], np * 8);
      }
    for (int d = 0; d < 3; ++d) {
      f((void**)&c->lor[d], np * 8);
      f((void**)&c->dv[d], np * 8);
      f((void**)&c->dvm[d], np * 8);
      f((void**)&c->E[d], nc * 8);
    }
    f((void**)&c->b, nc * 8);
    f((void**)&c->phi, nc * 8);
    f((void**)&c->cg_r, nc * 8);
    f((void**)&c->cg_p[0], nc * 8);
    f((void**)&c->cg_p[1], nc * 8);
    f((void**)&c->cg_q, nc * 8);
    f((void**)&c->overlay, lanes * 8);
  } else {
    for (int b = 0; b < 2; ++b) {
      f((void**)&c->cell32[b], np * 4);
      for (int d = 0; d < 3; ++d) {
        f((void**)&c->off[b][d], np * 4);
        f((void**)&c->vf[b][d], np * 4);
        f((void**)&c->vmf[b][d], np * 4);
      }
    }
    for (int d = 0; d < 3; ++d) {
      f((void**)&c->lorf[d], np * 4);
      f((void**)&c->dvf[d], np * 4);
      if (c->nrep == 0) f((void**)&c->dvmf[d], np * 4);  // pic_collide_avg only
    }
    f((void**)&c->Ef4, nc * 16);
    f((void**)&c->bf, nc * 4);
    f((void**)&c->phif, nc * 4);
    f((void**)&c->cgf_r, nc * 4);
    f((void**)&c->cgf_p, nc * 4);
    f((void**)&c->cgf_q, nc * 4);
    if (c->mg_nlev > 0) {
      int ng = 0;
      size_t wf = 0;
      mg_levels(c->P.n, &ng, &wf);
      f((void**)&c->mg_z, nc * 4);
      f((void**)&c->mg_z2, nc * 4);
      f((void**)&c->mg_work, wf * 4);
    }
    f((void**)&c->overlay32, lanes * 4);
  }
  for (int b = 0; b < 2; ++b) f((void**)&c->pid[b], np * 4);
  f((void**)&c->key, np * 4);
  f((void**)&c->rank, np * 4);
  f((void**)&c->perm, np * 4);
  f((void**)&c->count, nc * 4);
  f((void**)&c->start, (nc + 1) * 4);
  f((void**)&c->scan_blocks, (size_t)c->scan_nblocks * 4 + 16);
  f((void**)&c->corner, 8 * nc * 8);
  f((void**)&c->rho, nc * 8);
  f((void**)&c->rhs_part, (size_t)c->rhs_blocks * 8);
  f((void**)&c->cg_red, (size_t)4 * c->cg_grid * 8);
  f((void**)&c->cg_bar, 64);
  f((void**)&c->cg_info, 64);
  f((void**)&c->cg_res, 64);
  f((void**)&c->counters, 8 * 8);
  f((void**)&c->dsmc_queue, 64);
  f((void**)&c->step_hist, (size_t)kHistSteps * 4 * 8);
  f((void**)&c->flags, 64);
  f((void**)&c->err_part, (size_t)c->err_blocks * 14 * 8);
  f((void**)&c->err_out, 14 * 8);
  f((void**)&c->ginv, (size_t)(kGinvM + 1) * 2 * 8);
  f((void**)&c->ginv_f, (size_t)(kGinvM + 1) * 4 * 4 + (size_t)(kRTabM + 1) * 2 * 4);
  if (c->nrep == 0 && (c->cfg.verify & PIC_VERIFY_ANGLES)) {
    f((void**)&c->ang_hist, (size_t)2 * PIC_ANGLE_BINS * 8);
    f((void**)&c->ang_bsum, (size_t)4 * kAngleBlocks * 8);
    f((void**)&c->ang_part, (size_t)4 * kAngleBlocks * 8);
    f((void**)&c->ang_out, 8 * 8);
  }
  // host-boundary staging: the largest replicate of a batch, else everything
  size_t stage_np = np;
  if (c->nrep > 0 && c->prm_host) {  // (null only when a failed create is released)
    stage_np = 1;
    for (int r = 0; r < c->nrep; ++r)
      stage_np = (size_t)c->prm_host[r].np > stage_np ? (size_t)c->prm_host[r].np : stage_np;
  }
  f((void**)&c->stage, 6 * stage_np * 8);
  f((void**)&c->stage_i, (stage_np + 1) * 4);
}

// The address at which a kernel may use a caller array in place: device
// memory of the context's GPU, or pinned (registered) host memory mapped
// into the device address space, which kernels reach over NVLink-C2C
// without a staging copy. nullptr: pageable or other memory, staged through
// a copy.
template <class T>
T* in_place(const pic_ctx* c, T* p) {
  if (((uintptr_t)p & 7) != 0) return nullptr;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, (const void*)p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (at.type == cudaMemoryTypeDevice && at.device == c->device) return p;
  if (at.type == cudaMemoryTypeHost && at.devicePointer) return (T*)at.devicePointer;
  return nullptr;
}

// Read and clear the sticky device flags of the work enqueued so far
// (synchronises the stream).
pic_status check_pending(pic_ctx* c) {
  int info[3] = {0, 0, 0};
  int flags[2] = {0, 0};
  double res = 0.0;
  CK(cudaMemcpyAsync(info, c->cg_info, sizeof(info), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(flags, c->flags, sizeof(flags), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(&res, c->cg_res, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemsetAsync(c->flags, 0, sizeof(flags), c->stream));
  CK(cudaStreamSynchronize(c->stream));
  c->cg_iters_last = info[0];
  if (flags[1] > c->cg_iters_max) c->cg_iters_max = flags[1];
  c->cg_res_last = res;
  if (flags[0] & 4) return PIC_ETIMEOUT;
  if (flags[0] & 1) return PIC_ECAPACITY;
  if (flags[0] & 2) return PIC_ENOCONV;
  return PIC_OK;
}

// sort by (cell, pid) from the current positions and solve the field at t
// keys_done: the state load wrote the keys, ranks and counts itself
// Bins for a state load's records, by cell: a capacity of four times the
// mean particles per cell (a multiple of 32), if that is at most kBigCell
// (larger cells take the block sort, which reads through perm), the bins
// hold at most eight times the records (a sparse state on a fine mesh
// would mostly bin nothing) and take at most a quarter of the free device
// memory. Tried once per context; without bins the loads take the scatter
// and a random gather.
void ensure_bins(pic_ctx* c) {
  if (c->bin_tried) return;
  c->bin_tried = true;
  if (c->P.ncell <= 0 || c->P.np <= 0) return;
  const int64_t mean = (c->P.np + c->P.ncell - 1) / c->P.ncell;
  int64_t cap = (4 * mean + 31) / 32 * 32;
  if (cap > kBigCell) return;
  const size_t bytes = (size_t)c->P.ncell * (size_t)cap * 48;
  if (bytes > (size_t)8 * 48 * (size_t)c->P.np) return;
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  if (bytes > free_b / 4) return;
  c->bins = (float4*)dev_alloc(c, bytes);
  c->bin_over = (int*)dev_alloc(c, sizeof(int));
  if (!c->bins || !c->bin_over) {
    dev_free(c, c->bins);
    dev_free(c, c->bin_over);
    c->bins = nullptr;
    c->bin_over = nullptr;
    return;
  }
  c->bin_cap = cap;
}

pic_status sort_and_field(pic_ctx* c, double t, bool keys_done = false) {
  c->lor_valid = false;
  if (!keys_done) CK(cudaMemsetAsync(c->count, 0, (size_t)c->P.ncell * 4, c->stream));
  if (c->mixed) {
    if (!keys_done) CK(launch_keys32(c));
    // records binned by cell need no permutation: the gather reads each
    // cell's bin
    if (c->bin_state) CK(launch_scan(c));
    else CK(launch_scan_scatter(c));
    CK(launch_gather32(c));
    CK(launch_rhs(c, t));
    CK(launch_cg32(c));
  } else {
    CK(launch_keys(c));
    CK(launch_sort(c));
    CK(launch_rhs(c, t));
    CK(launch_cg(c));
  }
  return PIC_OK;
}

double time_at(const pic_ctx* c, double steps) { return c->t0 + steps * c->cfg.dt; }

// The precision form's state in pid order (sampled, or a caller's rows used
// in place, keeping the v^M of a held state buffer) written by the sampling
// kernel as records in the staging area and into the per-cell bins, then
// sorted with its field: from the bins, or, when a cell outgrew its bin
// (or there are no bins), by the scatter and a random gather of the
// records. *binned: the sort read the bins.
pic_status records_then_sort(pic_ctx* c, double t, const double* xs, const double* vs, int held, bool* binned) {
  ensure_bins(c);
  CK(cudaMemsetAsync(c->count, 0, (size_t)c->P.ncell * 4, c->stream));
  if (c->bins) CK(cudaMemsetAsync(c->bin_over, 0, sizeof(int), c->stream));
  CK(launch_sample32(c, t, xs, vs, held, true));
  *binned = false;
  if (c->bins) {
    int over = 1;
    CK(cudaMemcpyAsync(&over, c->bin_over, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    *binned = over == 0;
  }
  c->rec_state = true;
  c->bin_state = *binned;
  pic_status s = sort_and_field(c, t, true);
  if (s != PIC_OK) {
    c->rec_state = false;
    c->bin_state = false;
  }
  return s;
}

// Per-replicate time terms of step n (t_n, t_{n+1/2}, t_{n+1}) and the step
// number into the pinned mirror (every replicate has its own dt); the copy
// to the device is enqueued by batch_enqueue_times (and captured in graphs).
pic_status batch_time_terms(pic_ctx* c, int64_t n) {
  CK(cudaStreamSynchronize(c->stream));  // the pinned mirror may still feed a copy
  for (int r = 0; r < c->nrep; ++r) {
    const double dt = c->prm_host[r].dt;
    c->tt_host[3 * r + 0] = time_terms(c->prm_host[r], c->t0 + (double)n * dt);
    c->tt_host[3 * r + 1] = time_terms(c->prm_host[r], c->t0 + ((double)n + 0.5) * dt);
    c->tt_host[3 * r + 2] = time_terms(c->prm_host[r], c->t0 + (double)(n + 1) * dt);
  }
  memset((void*)(c->tt_host + 3 * c->nrep), 0, sizeof(TimeTerms));
  *reinterpret_cast<int64_t*>(c->tt_host + 3 * c->nrep) = n;
  return PIC_OK;
}

cudaError_t batch_enqueue_times(pic_ctx* c) {
  return cudaMemcpyAsync(c->tt_dev, c->tt_host, sizeof(TimeTerms) * (3 * c->nrep + 1), cudaMemcpyHostToDevice,
                         c->stream);
}

// One step of every replicate, enqueued without host synchronisation (so it
// can be captured into a graph).
cudaError_t batch_enqueue_step(pic_ctx* c, bool coll) {
  cudaError_t e = batch_enqueue_times(c);
  if (e == cudaSuccess && coll) e = launch_batch_dsmc(c, 0);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->count, 0, (size_t)c->P.ncell * 4, c->stream);
  if (e == cudaSuccess) e = launch_batch_kick(c, coll, true);
  if (e == cudaSuccess) e = launch_scan_scatter(c);
  if (e == cudaSuccess) e = launch_gather32(c);
  if (e == cudaSuccess) e = launch_batch_rhs(c, 2);
  if (e == cudaSuccess) e = launch_batch_cg(c);
  if (e == cudaSuccess && coll) e = launch_batch_dsmc(c, 1);
  if (e == cudaSuccess) e = launch_batch_kick(c, coll, false);
  return e;
}

// the two timing events of one tuning step, released on every return
struct EventPair {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  ~EventPair() {
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  }
};

// per-step work of the persistent batched step: the time terms, then its
// one launch (and two memsets)
cudaError_t batch_enqueue_persistent(pic_ctx* c, bool coll, bool stall) {
  cudaError_t e = batch_enqueue_times(c);
  if (e == cudaSuccess) e = launch_batch_step(c, coll, stall);
  return e;
}

// One batched step: one launch of the persistent step kernel. The first
// steps time every candidate (block size, tile shapes) of it, one step each
// (the result does not depend on the candidate); later steady-state steps
// replay a captured graph per buffer parity. With profiling on, the step
// runs as one launch per phase, so that each phase is timed.
pic_status batch_step(pic_ctx* c, int64_t n, bool coll) {
  pic_status s = batch_time_terms(c, n);
  if (s != PIC_OK) return s;
  const bool stall = c->stall_next_cg;
  c->stall_next_cg = false;
  if (c->profiling) {
    CK(batch_enqueue_step(c, coll));
    return PIC_OK;
  }
  const int ncand = step_candidates();
  while (c->tune_step < ncand && c->step_grid[step_block_of(c->tune_step) == 128 ? 0 : 1] == 0)
    c->tune_ms[c->tune_step++] = 1e30f;  // a block size whose shared memory does not fit
  if (c->tune_step < ncand && !stall) {
    const int cand = c->tune_step;
    if (c->step_cand != cand) CK(build_step_items(c, cand));
    EventPair ev;
    CK(cudaEventCreate(&ev.e0));
    CK(cudaEventCreate(&ev.e1));
    CK(cudaEventRecord(ev.e0, c->stream));
    CK(batch_enqueue_persistent(c, coll, false));
    CK(cudaEventRecord(ev.e1, c->stream));
    CK(cudaEventSynchronize(ev.e1));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, ev.e0, ev.e1));
    c->tune_ms[cand] = ms;
    if (++c->tune_step == ncand) {
      int best = 0;
      for (int k = 1; k < ncand; ++k)
        if (c->tune_ms[k] < c->tune_ms[best]) best = k;
      CK(build_step_items(c, best));
    }
    return PIC_OK;
  }
  if (stall || !c->use_graphs || !c->lor_valid) {
    CK(batch_enqueue_persistent(c, coll, stall));
    return PIC_OK;
  }
  const int parity = c->cur;
  if (!c->graph[parity]) {
    const int64_t l0 = c->launches;
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = batch_enqueue_persistent(c, coll, false);
    cudaError_t e2 = cudaStreamEndCapture(c->stream, &g);
    if (e != cudaSuccess || e2 != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      return PIC_ECUDA;
    }
    c->graph_launches = c->launches - l0;
    c->launches = l0;
    e = cudaGraphInstantiate(&c->graph[parity], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      cudaGetLastError();
      c->graph[parity] = nullptr;
      return PIC_ECUDA;
    }
    // the capture advanced the host state (buffer parity, Lorentz flag) as a
    // step would; restore it, then replay
    c->cur = parity;
  }
  CK(cudaGraphLaunch(c->graph[parity], c->stream));
  c->graph_replays++;
  c->cur = 1 - parity;
  c->lor_valid = true;
  c->launches += c->graph_launches;
  return PIC_OK;
}

}  // namespace

namespace pic {

void* ctx_alloc(pic_ctx* c, size_t bytes) { return dev_alloc(c, bytes); }
void dev_free_ctx(pic_ctx* c, void* p) { dev_free(c, p); }
void ctx_free(pic_ctx* c, void* p) { dev_free(c, p); }

// The context's auxiliary stream (non-blocking, the device's highest
// priority, so that its short kernels start as soon as SMs free up) and its
// fork and join events, created at first use.
cudaError_t ensure_aux_stream(pic_ctx* c) {
  if (c->aux) return cudaSuccess;
  int lo = 0, hi = 0;
  cudaError_t e = cudaDeviceGetStreamPriorityRange(&lo, &hi);
  cudaStream_t s = nullptr;
  cudaEvent_t f = nullptr, j = nullptr;
  if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&s, cudaStreamNonBlocking, hi);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&f, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&j, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    if (j) cudaEventDestroy(j);
    if (f) cudaEventDestroy(f);
    if (s) cudaStreamDestroy(s);
    return e;
  }
  c->aux = s;
  c->aux_fork = f;
  c->aux_join = j;
  return cudaSuccess;
}

// One FP64 step of Eq. velocity_verlet. hook(where), if given, runs at
// 0: the start (x^n, v^n in the current buffers), 1: after the drift and the
// sort (x^{n+1}, v^{n+1/2}), 2: after the field solve (E^{n+1}).
cudaError_t step_fp64(pic_ctx* c, int64_t n, const StepHook* hook) {
  const bool coll = c->cfg.K > 0;
  const double tn = time_at(c, (double)n), th = time_at(c, (double)n + 0.5), tn1 = time_at(c, (double)(n + 1));
  cudaError_t e;
  if (hook && (e = (*hook)(0)) != cudaSuccess) return e;
  // v^{n+1/2} and x^{n+1}: collision call A at (x^n, v^n)
  if (coll && (e = launch_dsmc(c, (uint32_t)(2 * n), false, tn)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(c->count, 0, (size_t)c->P.ncell * 4, c->stream)) != cudaSuccess) return e;
  if ((e = launch_kick(c, tn, coll, true, th, tn1)) != cudaSuccess) return e;
  // cells of x^{n+1}, field at t^{n+1}
  if ((e = launch_sort(c)) != cudaSuccess) return e;
  if (hook && (e = (*hook)(1)) != cudaSuccess) return e;
  if ((e = launch_rhs(c, tn1)) != cudaSuccess) return e;
  if ((e = launch_cg(c)) != cudaSuccess) return e;
  if (hook && (e = (*hook)(2)) != cudaSuccess) return e;
  // v^{n+1}: collision call B at (x^{n+1}, v^{n+1/2})
  if (coll && (e = launch_dsmc(c, (uint32_t)(2 * n + 1), false, th)) != cudaSuccess) return e;
  return launch_kick(c, tn1, coll, false, 0.0, 0.0);
}

}  // namespace pic

extern "C" {

pic_status pic_config_default(pic_config* cfg) {
  if (!cfg) return PIC_EINVAL;
  memset(cfg, 0, sizeof(*cfg));
  cfg->n = 8;
  cfg->K = 16;
  cfg->n_particles = 4096;
  cfg->dt = 0.01;
  cfg->qm = cfg->q = cfg->eps0 = cfg->n_phys = 1.0;
  const double ppc = 4096.0 / 512.0, mean_g = 4.0 / sqrt(kPi);
  cfg->sigma0 = 0.1 * ppc / ((ppc - 1.0) * mean_g * cfg->dt);
  cfg->g_max = 10.0 * sqrt(3.0);
  cfg->fx_amp = 0.3;
  cfg->fx_speed = 0.1;
  cfg->v_mean[0] = cfg->v_mean[1] = cfg->v_mean[2] = 0.2;
  cfg->v_sigma = 1.0;
  cfg->phi_amp = 0.1;
  cfg->phi_T = 1.0;
  cfg->phi_shift[0] = 1.0 / 7.0;
  cfg->phi_shift[1] = 1.0 / 5.0;
  cfg->phi_shift[2] = 1.0 / 3.0;
  cfg->precision = PIC_FP64;
  cfg->max_ppc = 512;
  cfg->seed = 0;
  cfg->cg_tol = 1e-10;
  cfg->cg_maxit = 20000;
  return PIC_OK;
}

pic_status pic_validate_config(const pic_config* c) {
  if (!c) return PIC_EINVAL;
  if (c->n < 2 || c->n > 1024) return PIC_EINVAL;
  if (c->n_particles < 1 || c->n_particles > 2147483647LL) return PIC_EINVAL;
  if (c->K < 0 || c->K > (1 << 20)) return PIC_EINVAL;
  if (!(c->dt > 0.0) || !isfinite(c->dt)) return PIC_EINVAL;
  if (!isfinite(c->qm) || !isfinite(c->q) || !(c->eps0 > 0.0) || !(c->n_phys > 0.0)) return PIC_EINVAL;
  if (c->K > 0 && (!(c->sigma0 >= 0.0) || !(c->g_max > 0.0))) return PIC_EINVAL;
  if (!(fabs(c->fx_amp) < 1.0) || !isfinite(c->fx_speed)) return PIC_EINVAL;
  if (!(c->v_sigma > 0.0)) return PIC_EINVAL;
  for (int d = 0; d < 3; ++d)
    if (!isfinite(c->v_mean[d]) || !isfinite(c->phi_shift[d])) return PIC_EINVAL;
  if (!isfinite(c->phi_amp) || !(c->phi_T > 0.0)) return PIC_EINVAL;
  if (c->precision != PIC_FP64 && c->precision != PIC_MIXED) return PIC_EINVAL;
  if (c->max_ppc < 0 || c->max_ppc > 65536) return PIC_EINVAL;
  if (!(c->cg_tol > 0.0) || c->cg_maxit < 1) return PIC_EINVAL;
  if (c->verify & ~31) return PIC_EINVAL;
  if ((c->verify & PIC_VERIFY_ERROR1) && (c->verify & PIC_VERIFY_ERROR2)) return PIC_EINVAL;
  // the paper's problem and the odd-power cross section (single contexts)
  if (c->dist != PIC_DIST_CONFIG && c->dist != PIC_DIST_PAPER) return PIC_EINVAL;
  if (c->n_sigma < 0 || c->n_sigma > 3) return PIC_EINVAL;
  if (c->dist == PIC_DIST_PAPER) {
    if (!(c->v_bar > 0.0) || !isfinite(c->v_bar) || !(c->t_ref > 0.0) || !isfinite(c->t_ref)) return PIC_EINVAL;
    if (c->verify & PIC_VERIFY_ISOLATE) return PIC_EINVAL;
    if (c->K > 0 && c->n_sigma == 0) return PIC_EINVAL;  // no closed-form hard-sphere source for this f_v
  }
  if (c->n_sigma > 0) {
    for (int k = 0; k < c->n_sigma; ++k)
      if (!isfinite(c->sigma_n[k])) return PIC_EINVAL;
    if (c->K > 0 && (!(sg_max_of(*c) > 0.0) || !(sg_min_of(*c) >= 0.0))) return PIC_EINVAL;
  }
  const int64_t ncell = (int64_t)c->n * c->n * c->n;
  if (ncell > 2147483647LL) return PIC_EINVAL;
  return PIC_OK;
}

pic_status pic_derived(const pic_config* cfg, double out[5]) {
  if (!cfg || !out) return PIC_EINVAL;
  pic_status s = pic_validate_config(cfg);
  if (s != PIC_OK) return s;
  Params P;
  derive_params(*cfg, P);
  out[0] = P.w;
  out[1] = P.dV;
  out[2] = P.pmax;
  out[3] = (double)P.np / (double)P.ncell;
  out[4] = P.pmax > 0.0 ? 1.0 / P.pmax : INFINITY;
  return PIC_OK;
}

void pic_destroy(pic_ctx* c) {
  if (!c) return;
  adjoint_free(c);
  dev_free(c, c->dlog);
  dev_free(c, c->dlog_n);
  dev_free(c, c->bins);
  dev_free(c, c->bin_over);
  if (c->aux) {
    cudaStreamSynchronize(c->aux);
    cudaEventDestroy(c->aux_fork);
    cudaEventDestroy(c->aux_join);
    cudaStreamDestroy(c->aux);
  }
  for_each_buffer(c, [&](void** p, size_t) {
    dev_free(c, *p);
    *p = nullptr;
  });
  void* batch_dev[] = {c->reps_dev, c->prm_dev, c->rep_of_cell, c->poff_dev, c->dsmc_items, c->cg_order,
                       c->cg_iters_rep, c->cg_res_rep, c->tt_dev, c->step_items, c->step_need, c->step_sync,
                       c->cg_team_bar, c->cg_team_red, c->cg_parts, c->cg_head};
  free(c->step_items_host);
  for (void* p : batch_dev) dev_free(c, p);
  if (c->tt_host) cudaFreeHost(c->tt_host);
  for (int k = 0; k < 2; ++k)
    if (c->graph[k]) cudaGraphExecDestroy(c->graph[k]);
  free(c->reps_host);
  free(c->prm_host);
  for (int i = 0; i < 2 * c->ev_cap; ++i) cudaEventDestroy(c->ev_pool[i]);
  free(c->ev_pool);
  free(c->ev_class);
  delete c;
}

pic_status pic_create(const pic_config* cfg, void* stream, const pic_allocator* alloc, pic_ctx** out) {
  if (!out) return PIC_EINVAL;
  *out = nullptr;
  pic_status s = pic_validate_config(cfg);
  if (s != PIC_OK) return s;
  if (alloc && (!alloc->alloc || !alloc->free)) return PIC_EINVAL;
  pic_ctx* c = new (std::nothrow) pic_ctx();
  if (!c) return PIC_ENOMEM;
  memset((void*)c, 0, sizeof(*c));
  c->cfg = *cfg;
  if (c->cfg.max_ppc == 0) c->cfg.max_ppc = 512;
  c->cfg.max_ppc = (c->cfg.max_ppc + 31) / 32 * 32;
  c->stream = (cudaStream_t)stream;
  c->mixed = c->cfg.precision == PIC_MIXED;
  if (alloc) {
    c->alloc = *alloc;
    c->have_alloc = true;
  }
  derive_params(c->cfg, c->P);
  cudaError_t e = cudaGetDevice(&c->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
  int coop = 0;
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, c->device);
  if (e == cudaSuccess) e = allow_big_sort_smem();
  if (e != cudaSuccess || !coop) {
    cudaGetLastError();
    delete c;
    return PIC_ECUDA;
  }
  // launch geometry
  c->scan_nblocks = scan_blocks_needed(c->P.ncell);
  c->rhs_blocks = rhs_blocks_needed(c->P.ncell);
  c->err_blocks = err_blocks_needed(c->P.np, c->P.ncell);
  int occ = 0;
  const void* cg_fn = c->mixed ? cg32_kernel_ptr() : cg_kernel_ptr();
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, cg_fn, cg_threads(), 0);
  if (e != cudaSuccess || occ < 1) {
    cudaGetLastError();
    delete c;
    return PIC_ECUDA;
  }
  c->cg_block = cg_threads();
  int64_t cg_need = (c->P.ncell + c->cg_block - 1) / c->cg_block;
  c->cg_grid = (int)(cg_need < (int64_t)occ * c->num_sms ? cg_need : (int64_t)occ * c->num_sms);
  if (c->cg_grid < 1) c->cg_grid = 1;
  // the precision form's Poisson solve: CG preconditioned by a multigrid
  // V-cycle on meshes of 2^k >= 16 nodes per edge, plain CG otherwise
  if (c->mixed) {
    size_t wf = 0;
    c->mg_nlev = mg_levels(c->P.n, &c->mg_nlev_grid, &wf);
  }
  // collisions: lanes = (cell in group, outcome); bitmaps in shared memory
  const int K = c->cfg.K > 0 ? c->cfg.K : 1;
  c->dsmc_Kc = K < 32 ? K : 32;
  c->dsmc_G = K < 32 ? 32 / K : 1;
  c->dsmc_groups = (c->P.ncell + c->dsmc_G - 1) / c->dsmc_G;
  c->bm_words = c->cfg.max_ppc / 32;
  c->dsmc_block = c->mixed ? dsmc32_threads() : dsmc_threads();
  const void* dsmc_fn = c->mixed ? dsmc32_kernel_ptr(c->P.verify != 0) : dsmc_kernel_ptr(c->P.verify != 0);
  c->dsmc_smem = c->mixed ? dsmc32_smem_bytes(c->bm_words) : (size_t)(c->dsmc_block / 32) * 32 * c->bm_words * 4;
  if (c->dsmc_smem > 48 * 1024) {
    e = cudaFuncSetAttribute(dsmc_fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c->dsmc_smem);
    if (e != cudaSuccess) {
      cudaGetLastError();
      delete c;
      return PIC_EINVAL;
    }
  }
  int docc = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&docc, dsmc_fn, c->dsmc_block, c->dsmc_smem);
  if (e != cudaSuccess || docc < 1) {
    cudaGetLastError();
    delete c;
    return PIC_ECUDA;
  }
  const int64_t wpb = c->dsmc_block / 32;
  int64_t dgrid = (c->dsmc_groups + wpb - 1) / wpb;
  if (dgrid > (int64_t)docc * c->num_sms) dgrid = (int64_t)docc * c->num_sms;
  c->dsmc_grid = (int)(dgrid < 1 ? 1 : dgrid);
  if (c->cfg.K == 0) c->dsmc_grid = 1;

  bool ok = true;
  for_each_buffer(c, [&](void** p, size_t bytes) {
    if (!ok) return;
    *p = dev_alloc(c, bytes);
    if (!*p) ok = false;
  });
  if (!ok) {
    pic_destroy(c);
    return PIC_ENOMEM;
  }
  {
    double* tab = (double*)malloc((size_t)(kGinvM + 1) * 2 * 8);
    float* tabf = (float*)malloc((size_t)(kGinvM + 1) * 4 * 4 + (size_t)(kRTabM + 1) * 2 * 4);
    if (!tab || !tabf) {
      free(tab);
      free(tabf);
      pic_destroy(c);
      return PIC_ENOMEM;
    }
    ginv_table(c->cfg.fx_amp, tab);
    ginv_table_f(tab, tabf);
    e = cudaMemcpy(c->ginv, tab, (size_t)(kGinvM + 1) * 2 * 8, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(c->ginv_f, tabf, (size_t)(kGinvM + 1) * 4 * 4 + (size_t)(kRTabM + 1) * 2 * 4,
                                         cudaMemcpyHostToDevice);
    free(tab);
    free(tabf);
    c->P.ginv = c->ginv;
    c->P.ginv_f = c->ginv_f;
    c->P.ginv_M = kGinvM;
    c->P.ang_hist = c->ang_hist;
  }
  if (e == cudaSuccess && c->ang_hist)
    e = cudaMemsetAsync(c->ang_hist, 0, (size_t)2 * PIC_ANGLE_BINS * 8, c->stream);
  if (e == cudaSuccess)
    e = c->mixed ? cudaMemsetAsync(c->phif, 0, (size_t)c->P.ncell * 4, c->stream)
                 : cudaMemsetAsync(c->phi, 0, (size_t)c->P.ncell * 8, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->counters, 0, 64, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->flags, 0, 64, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->cg_info, 0, 64, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->cg_res, 0, 64, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    pic_destroy(c);
    return cuda_status(e);
  }
  c->cur = 0;
  *out = c;
  return PIC_OK;
}

}  // extern "C"
namespace {
// a new state starts a new per-step history
cudaError_t restart_history(pic_ctx* c) {
  c->hist_base = c->step;
  return cudaMemsetAsync(c->step_hist, 0, (size_t)kHistSteps * 4 * 8, c->stream);
}
pic_status step_loop(pic_ctx* c, int32_t nsteps);
}  // namespace
extern "C" {

pic_status pic_sample_mms(pic_ctx* c, double t0) {
  if (!c || !isfinite(t0)) return PIC_EINVAL;
  c->t0 = t0;
  c->step = 0;
  c->cur = 0;
  CK(restart_history(c));
  if (c->nrep > 0) {
    c->lor_valid = false;
    CK(cudaMemsetAsync(c->phif, 0, (size_t)c->P.ncell * 4, c->stream));
    pic_status s = batch_time_terms(c, 0);
    if (s != PIC_OK) return s;
    CK(batch_enqueue_times(c));
    CK(launch_batch_sample(c, nullptr));
    CK(cudaMemsetAsync(c->count, 0, (size_t)c->P.ncell * 4, c->stream));
    CK(launch_keys32(c));
    CK(launch_scan_scatter(c));
    CK(launch_gather32(c));
    CK(launch_batch_rhs(c, 0));
    CK(launch_batch_cg(c));
    c->sampled = true;
    return check_pending(c);
  }
  if (c->ang_hist) CK(cudaMemsetAsync(c->ang_hist, 0, (size_t)2 * PIC_ANGLE_BINS * 8, c->stream));
  if (c->mixed) {
    // the sampled state is in pid order, which the first sort would read
    // at random: through the records and the bins, as a state load
    CK(cudaMemsetAsync(c->phif, 0, (size_t)c->P.ncell * 4, c->stream));
    bool binned = false;
    pic_status s = records_then_sort(c, t0, nullptr, nullptr, -1, &binned);
    if (s != PIC_OK) return s;
    c->sampled = true;
    return check_pending(c);
  } else {
    CK(cudaMemsetAsync(c->phi, 0, (size_t)c->P.ncell * 8, c->stream));
    CK(launch_sample(c, t0));
  }
  pic_status s = sort_and_field(c, t0);
  if (s != PIC_OK) return s;
  c->sampled = true;
  return check_pending(c);
}

pic_status pic_set_state(pic_ctx* c, const double* x, const double* v, double t0, int64_t step) {
  if (!c || !x || !v || !isfinite(t0) || step < 0) return PIC_EINVAL;
  if (c->nrep > 0) return PIC_EINVAL;  // batches: use the pic_batch_* calls
  // the load kernels read device and pinned host arrays in place
  const size_t bytes = (size_t)c->P.np * 3 * 8;
  const double* xs = in_place(c, x);
  const double* vs = in_place(c, v);
  if (!xs) {
    CK(cudaMemcpyAsync(c->stage, x, bytes, cudaMemcpyDefault, c->stream));
    xs = c->stage;
  }
  if (!vs) {
    CK(cudaMemcpyAsync(c->stage + 3 * c->P.np, v, bytes, cudaMemcpyDefault, c->stream));
    vs = c->stage + 3 * c->P.np;
  }
  c->t0 = t0;
  c->step = step;
  CK(restart_history(c));
  if (c->mixed) {
    // v^M is a per-particle constant (tau for the paper's f_v): a context that
    // already holds a state keeps its values, read through the inverse sort
    // permutation by the load, instead of re-deriving them from xi in FP64.
    // Caller arrays used in place leave the staging area free: the load then
    // writes the state there as records, which the sort's random gather
    // reads in two sectors a particle instead of nine.
    const bool records = xs != c->stage && vs != c->stage + 3 * c->P.np;
    if (records) {
      bool binned = false;
      pic_status s = records_then_sort(c, time_at(c, (double)step), xs, vs, c->sampled ? c->cur : -1, &binned);
      if (s != PIC_OK) return s;
      if (binned) c->binned_loads++;
      c->sampled = true;
      return check_pending(c);
    }
    if (c->sampled) {
      const int src = c->cur;
      c->cur = 1 - src;
      CK(launch_sample32(c, time_at(c, (double)step), xs, vs, src));
    } else {
      c->cur = 0;
      CK(launch_sample32(c, time_at(c, (double)step), xs, vs));
    }
  } else {
    c->cur = 0;
    CK(launch_load_state(c, xs, vs, time_at(c, (double)step)));
  }
  pic_status s = sort_and_field(c, time_at(c, (double)step));
  if (s != PIC_OK) return s;
  c->sampled = true;
  return check_pending(c);
}

pic_status pic_step(pic_ctx* c, int32_t nsteps) {
  const pic_status s = step_loop(c, nsteps);
  if (c) c->hist_row = nullptr;  // also on an early return: no later launch writes the history
  return s;
}

}  // extern "C"
namespace {
pic_status step_loop(pic_ctx* c, int32_t nsteps) {
  if (!c || nsteps < 0) return PIC_EINVAL;
  if (!c->sampled) return PIC_ESTATE;
  const bool coll = c->cfg.K > 0;
  for (int32_t it = 0; it < nsteps; ++it) {
    const int64_t n = c->step;
    const double tn = time_at(c, (double)n), th = time_at(c, (double)n + 0.5), tn1 = time_at(c, (double)(n + 1));
    const int64_t row = n - c->hist_base;
    c->hist_row = (c->nrep == 0 && row >= 0 && row < kHistSteps) ? c->step_hist + 4 * row : nullptr;
    if (c->nrep > 0) {
      pic_status s = batch_step(c, n, coll);
      if (s != PIC_OK) return s;
    } else if (c->mixed) {
      if (coll) CK(launch_dsmc32(c, (uint32_t)(2 * n), false, tn));
      CK(cudaMemsetAsync(c->count, 0, (size_t)c->P.ncell * 4, c->stream));
      CK(launch_kick32(c, tn, coll, true, th, tn1));
      CK(launch_scan_scatter(c));
      CK(launch_gather32(c));
      CK(launch_rhs(c, tn1));
      CK(launch_cg32(c));
      if (coll) CK(launch_dsmc32(c, (uint32_t)(2 * n + 1), false, th));
      CK(launch_kick32(c, tn1, coll, false, 0.0, 0.0));
    } else {
      CK(step_fp64(c, n, nullptr));
    }
    c->step = n + 1;
  }
  c->hist_row = nullptr;
  return nsteps > 0 ? check_pending(c) : PIC_OK;
}
}  // namespace
extern "C" {

pic_status pic_collide_avg(pic_ctx* c, int32_t phase, double* dv, double* dvM) {
  if (!c || !dv || !dvM || (phase != 0 && phase != 1)) return PIC_EINVAL;
  if (c->nrep > 0) return PIC_EINVAL;  // batches: use the pic_batch_* calls
  if (!c->sampled) return PIC_ESTATE;
  const size_t bytes = (size_t)c->P.np * 3 * 8;
  if (c->mixed) {
    if (c->cfg.K > 0) {
      CK(launch_dsmc32(c, (uint32_t)(2 * c->step + phase), true, time_at(c, (double)c->step)));
    } else {
      for (int d = 0; d < 3; ++d) {
        CK(cudaMemsetAsync(c->dvf[d], 0, (size_t)c->P.np * 4, c->stream));
        CK(cudaMemsetAsync(c->dvmf[d], 0, (size_t)c->P.np * 4, c->stream));
      }
    }
    CK(launch_store_dv32(c, c->stage, c->stage + 3 * c->P.np));
  } else {
    if (c->cfg.K > 0) {
      CK(launch_dsmc(c, (uint32_t)(2 * c->step + phase), true, time_at(c, (double)c->step)));
    } else {
      for (int d = 0; d < 3; ++d) {
        CK(cudaMemsetAsync(c->dv[d], 0, (size_t)c->P.np * 8, c->stream));
        CK(cudaMemsetAsync(c->dvm[d], 0, (size_t)c->P.np * 8, c->stream));
      }
    }
    CK(launch_store_dv(c, c->stage, c->stage + 3 * c->P.np));
  }
  CK(cudaMemcpyAsync(dv, c->stage, bytes, cudaMemcpyDefault, c->stream));
  CK(cudaMemcpyAsync(dvM, c->stage + 3 * c->P.np, bytes, cudaMemcpyDefault, c->stream));
  return check_pending(c);
}

pic_status pic_mms_error(pic_ctx* c, pic_errors* out) {
  if (!c || !out) return PIC_EINVAL;
  if (c->nrep > 0) return PIC_EINVAL;  // batches: use the pic_batch_* calls
  if (!c->sampled) return PIC_ESTATE;
  if (c->mixed) {
    CK(launch_errors32(c, time_at(c, (double)c->step)));
    CK(launch_err_final(c, c->err_blocks));
  } else {
    CK(launch_errors(c, time_at(c, (double)c->step)));
  }
  double h[14];
  CK(cudaMemcpyAsync(h, c->err_out, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  for (int q = 0; q < 7; ++q) {
    out->eps2[q] = h[q];
    out->epsinf[q] = h[7 + q];
  }
  return check_pending(c);
}

pic_status pic_get_state(pic_ctx* c, double* x, double* v) {
  if (!c || !x || !v) return PIC_EINVAL;
  if (c->nrep > 0) return PIC_EINVAL;  // batches: use the pic_batch_* calls
  if (!c->sampled) return PIC_ESTATE;
  const size_t bytes = (size_t)c->P.np * 3 * 8;
  if (c->mixed) {
    // device and pinned host destinations are written in place, in pid order
    double* xd = in_place(c, x);
    double* vd = in_place(c, v);
    if (xd && vd) {
      CK(launch_store_state32_by_pid(c, xd, vd));
      CK(cudaStreamSynchronize(c->stream));
      return PIC_OK;
    }
    CK(launch_store_state32(c, c->stage, nullptr));
  } else {
    CK(launch_store_state(c, c->stage));
  }
  CK(cudaMemcpyAsync(x, c->stage, bytes, cudaMemcpyDefault, c->stream));
  CK(cudaMemcpyAsync(v, c->stage + 3 * c->P.np, bytes, cudaMemcpyDefault, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return PIC_OK;
}

pic_status pic_inject_barrier_stall(pic_ctx* c) {
  if (!c || (c->nrep == 0 && c->cg_grid < 2)) return PIC_EINVAL;
  c->stall_next_cg = true;
  return PIC_OK;
}

pic_status pic_get_field(pic_ctx* c, double* rho, double* phi, double* E) {
  if (!c) return PIC_EINVAL;
  if (c->nrep > 0) return PIC_EINVAL;  // batches: use the pic_batch_* calls
  if (!c->sampled) return PIC_ESTATE;
  const size_t nc = (size_t)c->P.ncell;
  double* sphi = c->stage;
  double* sE = c->stage + nc;
  const bool fits = 4 * nc <= 6 * (size_t)c->P.np;
  if (rho) CK(cudaMemcpyAsync(rho, c->rho, nc * 8, cudaMemcpyDefault, c->stream));
  if (fits) {
    if (c->mixed) CK(launch_store_field32(c, phi ? sphi : nullptr, E ? sE : nullptr));
    else CK(launch_store_field(c, nullptr, phi ? sphi : nullptr, E ? sE : nullptr));
    if (phi) CK(cudaMemcpyAsync(phi, sphi, nc * 8, cudaMemcpyDefault, c->stream));
    if (E) CK(cudaMemcpyAsync(E, sE, 3 * nc * 8, cudaMemcpyDefault, c->stream));
  } else if (phi || E) {
    // fewer particles than nodes: stage through host memory
    const size_t esz = c->mixed ? 4 : 8;
    // the precision form's field is interleaved (Ex, Ey, Ez, 0) per node
    unsigned char* comp = (unsigned char*)malloc(nc * (c->mixed ? 16 : esz));
    double* tmp = (double*)malloc(3 * nc * 8);
    if (!comp || !tmp) { free(comp); free(tmp); return PIC_ENOMEM; }
    const void* srcs[4] = {c->mixed ? (const void*)c->phif : (const void*)c->phi,
                           c->mixed ? (const void*)c->Ef4 : (const void*)c->E[0],
                           c->mixed ? nullptr : (const void*)c->E[1],
                           c->mixed ? nullptr : (const void*)c->E[2]};
    cudaError_t e = cudaSuccess;
    for (int q = 0; q < 4 && e == cudaSuccess; ++q) {
      if ((q == 0 && !phi) || (q > 0 && !E) || !srcs[q]) continue;
      const bool e4 = c->mixed && q == 1;  // all three components at once
      e = cudaMemcpyAsync(comp, srcs[q], nc * (e4 ? 16 : esz), cudaMemcpyDeviceToHost, c->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
      if (e != cudaSuccess) break;
      for (size_t i = 0; i < nc; ++i) {
        if (e4) {
          for (int d = 0; d < 3; ++d) tmp[3 * i + d] = (double)((const float*)comp)[4 * i + d];
          continue;
        }
        const double val = c->mixed ? (double)((const float*)comp)[i] : ((const double*)comp)[i];
        if (q == 0) tmp[i] = val;
        else tmp[3 * i + (q - 1)] = val;
      }
      if (q == 0) e = cudaMemcpy(phi, tmp, nc * 8, cudaMemcpyDefault);
    }
    if (e == cudaSuccess && E) e = cudaMemcpy(E, tmp, 3 * nc * 8, cudaMemcpyDefault);
    free(comp);
    free(tmp);
    if (e != cudaSuccess) return cuda_status(e);
  }
  CK(cudaStreamSynchronize(c->stream));
  return PIC_OK;
}

pic_status pic_get_sort(pic_ctx* c, int32_t* cell_of_pid, int32_t* count, int32_t* start, int32_t* perm) {
  if (!c) return PIC_EINVAL;
  if (c->nrep > 0) return PIC_EINVAL;  // batches: use the pic_batch_* calls
  if (!c->sampled) return PIC_ESTATE;
  const size_t np = (size_t)c->P.np, nc = (size_t)c->P.ncell;
  int32_t* scell = (int32_t*)c->stage;            // fits: 6 np doubles = 12 np ints
  int32_t* sperm = (int32_t*)c->stage + np;
  if (c->mixed) {
    if (cell_of_pid) CK(launch_store_state32(c, nullptr, scell));
    if (perm) CK(cudaMemcpyAsync(sperm, c->pid[c->cur], np * 4, cudaMemcpyDeviceToDevice, c->stream));
  } else {
    CK(launch_store_sort(c, cell_of_pid ? scell : nullptr, perm ? sperm : nullptr));
  }
  if (cell_of_pid) CK(cudaMemcpyAsync(cell_of_pid, scell, np * 4, cudaMemcpyDefault, c->stream));
  if (perm) CK(cudaMemcpyAsync(perm, sperm, np * 4, cudaMemcpyDefault, c->stream));
  if (count) CK(cudaMemcpyAsync(count, c->count, nc * 4, cudaMemcpyDefault, c->stream));
  if (start) CK(cudaMemcpyAsync(start, c->start, (nc + 1) * 4, cudaMemcpyDefault, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return PIC_OK;
}

pic_status pic_get_stats(pic_ctx* c, pic_stats* out) {
  if (!c || !out) return PIC_EINVAL;
  unsigned long long h[5] = {0, 0, 0, 0, 0};
  CK(cudaMemcpyAsync(h, c->counters, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  pic_status s = c->sampled ? check_pending(c) : PIC_OK;
  memset(out, 0, sizeof(*out));
  out->n_cand = (int64_t)h[0];
  out->n_coll = (int64_t)h[1];
  out->n_gmax_exceed = (int64_t)h[2];
  out->n_near_ties = (int64_t)h[3];
  out->n_floor_ties = (int64_t)h[4];
  out->kernel_launches = c->launches;
  out->step = c->step;
  out->t = time_at(c, (double)c->step);
  out->cg_iters_last = c->cg_iters_last;
  out->cg_iters_max = c->cg_iters_max;
  out->cg_res_last = c->cg_res_last;
  out->graph_replays = c->graph_replays;
  out->binned_loads = c->binned_loads;
  if (c->nrep > 0 && c->tune_step >= step_candidates()) {
    out->tuned_block = step_block_of(c->step_cand);
    out->tuned_tile = step_tile_of(c->step_cand);
  }
  return s;
}

pic_status pic_reset_stats(pic_ctx* c) {
  if (!c) return PIC_EINVAL;
  CK(cudaMemsetAsync(c->counters, 0, 64, c->stream));
  CK(cudaMemsetAsync(c->step_hist, 0, (size_t)kHistSteps * 4 * 8, c->stream));
  c->hist_base = c->step;
  CK(cudaMemsetAsync(c->flags, 0, 64, c->stream));
  if (c->ang_hist) CK(cudaMemsetAsync(c->ang_hist, 0, (size_t)2 * PIC_ANGLE_BINS * 8, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  c->launches = 0;
  c->cg_iters_max = 0;
  c->binned_loads = 0;
  return PIC_OK;
}

pic_status pic_get_step_history(pic_ctx* c, int64_t* out, int64_t cap, int64_t* n) {
  if (!c || !n || cap < 0 || (cap > 0 && !out)) return PIC_EINVAL;
  if (c->nrep > 0) return PIC_EINVAL;
  int64_t k = c->step - c->hist_base;
  if (k < 0) k = 0;
  if (k > kHistSteps) k = kHistSteps;
  if (k > cap) k = cap;
  if (k > 0) {
    CK(cudaMemcpyAsync(out, c->step_hist, (size_t)k * 32, cudaMemcpyDefault, c->stream));
    CK(cudaStreamSynchronize(c->stream));
  }
  *n = k;
  return PIC_OK;
}

pic_status pic_set_decision_log(pic_ctx* c, int32_t mode, int64_t capacity) {
  if (!c || c->nrep > 0) return PIC_EINVAL;
  if (mode != PIC_DLOG_OFF && mode != PIC_DLOG_FLAGGED && mode != PIC_DLOG_ALL) return PIC_EINVAL;
  if (mode != PIC_DLOG_OFF && (capacity < 1 || capacity > INT32_MAX)) return PIC_EINVAL;
  CK(cudaStreamSynchronize(c->stream));  // no kernel of an earlier call still writes the old buffer
  if (mode == PIC_DLOG_OFF || capacity != c->dlog_cap) {
    dev_free(c, c->dlog);
    dev_free(c, c->dlog_n);
    c->dlog = nullptr;
    c->dlog_n = nullptr;
    c->dlog_cap = 0;
  }
  c->dlog_mode = mode;
  if (mode == PIC_DLOG_OFF) return PIC_OK;
  if (!c->dlog) {
    c->dlog = (int32_t*)dev_alloc(c, (size_t)capacity * 32);
    c->dlog_n = (unsigned long long*)dev_alloc(c, 64);
    if (!c->dlog || !c->dlog_n) {
      dev_free(c, c->dlog);
      dev_free(c, c->dlog_n);
      c->dlog = nullptr;
      c->dlog_n = nullptr;
      c->dlog_mode = PIC_DLOG_OFF;
      return PIC_ENOMEM;
    }
    c->dlog_cap = capacity;
  }
  CK(cudaMemsetAsync(c->dlog_n, 0, 8, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return PIC_OK;
}

pic_status pic_get_decision_log(pic_ctx* c, int32_t* out, int64_t cap, int64_t* n_total) {
  if (!c || !n_total || cap < 0 || (cap > 0 && !out)) return PIC_EINVAL;
  if (c->nrep > 0) return PIC_EINVAL;
  *n_total = 0;
  if (!c->dlog) return PIC_OK;
  unsigned long long n = 0;
  CK(cudaMemcpyAsync(&n, c->dlog_n, 8, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  int64_t k = (int64_t)n;
  if (k > c->dlog_cap) k = c->dlog_cap;
  if (k > cap) k = cap;
  if (k > 0) CK(cudaMemcpyAsync(out, c->dlog, (size_t)k * 32, cudaMemcpyDefault, c->stream));
  CK(cudaMemsetAsync(c->dlog_n, 0, 8, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  *n_total = (int64_t)n;
  return PIC_OK;
}

pic_status pic_get_angle_stats(pic_ctx* c, pic_angle_stats* out) {
  if (!c || !out) return PIC_EINVAL;
  if (!c->ang_hist) return PIC_ESTATE;
  CK(launch_angle_stats(c, out));
  return PIC_OK;
}

pic_status pic_set_profiling(pic_ctx* c, int32_t on) {
  if (!c) return PIC_EINVAL;
  prof_flush(c);
  c->profiling = on != 0;
  memset(c->prof_ms, 0, sizeof(c->prof_ms));
  memset(c->prof_launches, 0, sizeof(c->prof_launches));
  return PIC_OK;
}

pic_status pic_get_kernel_times(pic_ctx* c, pic_kernel_times* out) {
  if (!c || !out) return PIC_EINVAL;
  prof_flush(c);
  for (int k = 0; k < PIC_NUM_KERNEL_CLASSES; ++k) {
    out->ms[k] = c->prof_ms[k];
    out->launches[k] = c->prof_launches[k];
  }
  return PIC_OK;
}

pic_status pic_create_batch(const pic_config* cfgs, int32_t nrep, void* stream, const pic_allocator* alloc,
                            pic_ctx** out) {
  if (!out) return PIC_EINVAL;
  *out = nullptr;
  if (!cfgs || nrep < 1 || nrep > 65534) return PIC_EINVAL;
  if (alloc && (!alloc->alloc || !alloc->free)) return PIC_EINVAL;
  const pic_config& c0 = cfgs[0];
  int64_t np_tot = 0, nc_tot = 0, items = 0;
  int max_ppc = c0.max_ppc ? c0.max_ppc : 512;
  for (int r = 0; r < nrep; ++r) {
    const pic_config& c = cfgs[r];
    if (pic_validate_config(&c) != PIC_OK || c.precision != PIC_MIXED || c.verify != 0) return PIC_EINVAL;
    if (c.dist != PIC_DIST_CONFIG || c.n_sigma != 0) return PIC_EINVAL;  // single contexts only
    // everything but n, n_particles, K, dt, sigma0 and seed is shared
    if (c.qm != c0.qm || c.q != c0.q || c.eps0 != c0.eps0 || c.n_phys != c0.n_phys || c.g_max != c0.g_max ||
        c.fx_amp != c0.fx_amp || c.fx_speed != c0.fx_speed || c.v_sigma != c0.v_sigma || c.phi_amp != c0.phi_amp ||
        c.phi_T != c0.phi_T || c.couple_qm_zero != c0.couple_qm_zero || c.couple_q_zero != c0.couple_q_zero ||
        c.cg_tol != c0.cg_tol || c.cg_maxit != c0.cg_maxit || (c.max_ppc ? c.max_ppc : 512) != max_ppc)
      return PIC_EINVAL;
    for (int d = 0; d < 3; ++d)
      if (c.v_mean[d] != c0.v_mean[d] || c.phi_shift[d] != c0.phi_shift[d]) return PIC_EINVAL;
    np_tot += c.n_particles;
    const int64_t nc = (int64_t)c.n * c.n * c.n;
    nc_tot += (nc + kBatchTile - 1) / kBatchTile * kBatchTile;
    if (c.K > 0) {
      const int G = c.K < 32 ? 32 / c.K : 1;
      items += (nc + G - 1) / G;
    }
  }
  if (np_tot > 2147483647LL || nc_tot > 2147483647LL) return PIC_EINVAL;
  pic_ctx* c = new (std::nothrow) pic_ctx();
  if (!c) return PIC_ENOMEM;
  memset((void*)c, 0, sizeof(*c));
  c->cfg = c0;
  c->cfg.max_ppc = (max_ppc + 31) / 32 * 32;
  c->cfg.n_particles = np_tot;
  c->stream = (cudaStream_t)stream;
  c->mixed = true;
  c->nrep = nrep;
  if (alloc) {
    c->alloc = *alloc;
    c->have_alloc = true;
  }
  derive_params(c->cfg, c->P);
  c->P.np = np_tot;
  c->P.ncell = nc_tot;
  int kmax = 1;
  for (int r = 0; r < nrep; ++r) kmax = cfgs[r].K > kmax ? cfgs[r].K : kmax;
  c->cfg.K = kmax;
  c->P.K = kmax;
  cudaError_t e = cudaGetDevice(&c->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
  if (e == cudaSuccess) e = allow_big_sort_smem();
  if (e != cudaSuccess) {
    cudaGetLastError();
    delete c;
    return PIC_ECUDA;
  }
  c->scan_nblocks = scan_blocks_needed(nc_tot);
  c->rhs_blocks = 1;
  int64_t eb = 1;
  for (int r = 0; r < nrep; ++r) {
    const int64_t b = err_blocks_needed(cfgs[r].n_particles, (int64_t)cfgs[r].n * cfgs[r].n * cfgs[r].n);
    eb = b > eb ? b : eb;
  }
  c->err_blocks = (int)eb;
  c->cg_grid = 1;
  c->bm_words = c->cfg.max_ppc / 32;
  c->dsmc_block = batch_dsmc_threads();
  c->dsmc_smem = (size_t)(c->dsmc_block / 32) * 32 * c->bm_words * 4;
  if (c->dsmc_smem > 48 * 1024) {
    e = cudaFuncSetAttribute(batch_dsmc_kernel_ptr(), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c->dsmc_smem);
    if (e != cudaSuccess) {
      cudaGetLastError();
      delete c;
      return PIC_EINVAL;
    }
  }
  int docc = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&docc, batch_dsmc_kernel_ptr(), c->dsmc_block, c->dsmc_smem);
  if (e != cudaSuccess || docc < 1) {
    cudaGetLastError();
    delete c;
    return PIC_ECUDA;
  }
  const int64_t wpb = c->dsmc_block / 32;
  int64_t dgrid = (items + wpb - 1) / wpb;
  if (dgrid > (int64_t)docc * c->num_sms) dgrid = (int64_t)docc * c->num_sms;
  c->dsmc_grid = (int)(dgrid < 1 ? 1 : dgrid);
  c->n_items = items;
  // persistent step: one block per resident slot for each block size it
  // may run with (0 where its shared memory does not fit)
  c->overlay_warps = (int64_t)c->dsmc_grid * wpb;
  for (int k = 0; k < 2; ++k) {
    const int blk = k == 0 ? 128 : 256;
    const size_t sm = step_smem(c, blk);
    int occ = 0;
    if (sm > 48 * 1024 &&
        cudaFuncSetAttribute(step_kernel_ptr(blk), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess)
      occ = 0;
    else if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, step_kernel_ptr(blk), blk, sm) != cudaSuccess)
      occ = 0;
    cudaGetLastError();
    c->step_grid[k] = occ * c->num_sms;
    const int64_t w = (int64_t)c->step_grid[k] * (blk / 32);
    if (w > c->overlay_warps) c->overlay_warps = w;
  }
  if (c->step_grid[0] == 0 && c->step_grid[1] == 0) {
    delete c;
    return PIC_EINVAL;
  }

  // host tables
  c->reps_host = (BatchRep*)calloc((size_t)nrep, sizeof(BatchRep));
  c->prm_host = (Params*)calloc((size_t)nrep, sizeof(Params));
  uint16_t* roc = (uint16_t*)malloc((size_t)nc_tot * sizeof(uint16_t));
  int64_t* poff = (int64_t*)malloc((size_t)(nrep + 1) * sizeof(int64_t));
  int2* it_h = (int2*)malloc((size_t)(items > 0 ? items : 1) * sizeof(int2));
  int* order = (int*)malloc((size_t)nrep * sizeof(int));
  bool ok = c->reps_host && c->prm_host && roc && poff && it_h && order;
  if (ok) {
    int64_t p = 0, cc = 0, k = 0;
    for (int r = 0; r < nrep; ++r) {
      Params P;
      derive_params(cfgs[r], P);
      c->prm_host[r] = P;
      BatchRep& B = c->reps_host[r];
      B.poff = p;
      B.coff = cc;
      const int K = cfgs[r].K > 0 ? cfgs[r].K : 1;
      B.Kc = K < 32 ? K : 32;
      B.G = K < 32 ? 32 / K : 1;
      B.nchunks = (cfgs[r].K + B.Kc - 1) / B.Kc;
      poff[r] = p;
      const int64_t nc = (int64_t)cfgs[r].n * cfgs[r].n * cfgs[r].n;
      const int64_t ncp = (nc + kBatchTile - 1) / kBatchTile * kBatchTile;
      for (int64_t i = 0; i < ncp; ++i) roc[cc + i] = i < nc ? (uint16_t)r : (uint16_t)0xFFFF;
      if (cfgs[r].K > 0)
        for (int64_t g = 0; g < nc; g += B.G) it_h[k++] = make_int2(r, (int)g);
      p += cfgs[r].n_particles;
      cc += ncp;
      order[r] = r;
    }
    poff[nrep] = p;
    // CG work: largest replicates first
    for (int i = 1; i < nrep; ++i)
      for (int j = i; j > 0 && cfgs[order[j]].n > cfgs[order[j - 1]].n; --j) {
        const int t = order[j];
        order[j] = order[j - 1];
        order[j - 1] = t;
      }
  }
  for_each_buffer(c, [&](void** pp, size_t bytes) {
    if (!ok) return;
    *pp = dev_alloc(c, bytes);
    if (!*pp) ok = false;
  });
  auto grab = [&](void** pp, size_t bytes) {
    if (!ok) return;
    *pp = dev_alloc(c, bytes);
    if (!*pp) ok = false;
  };
  grab((void**)&c->reps_dev, sizeof(BatchRep) * nrep);
  grab((void**)&c->prm_dev, sizeof(Params) * nrep);
  grab((void**)&c->rep_of_cell, sizeof(uint16_t) * nc_tot);
  grab((void**)&c->poff_dev, sizeof(int64_t) * (nrep + 1));
  grab((void**)&c->dsmc_items, sizeof(int2) * (items > 0 ? items : 1));
  grab((void**)&c->cg_order, sizeof(int) * nrep);
  grab((void**)&c->cg_iters_rep, sizeof(int) * nrep);
  grab((void**)&c->cg_res_rep, sizeof(double) * nrep);
  grab((void**)&c->tt_dev, sizeof(TimeTerms) * (3 * nrep + 1));
  int n_parts = 0;
  for (int r = 0; r < nrep; ++r) n_parts += cg_team_size(cfgs[r].n * cfgs[r].n * cfgs[r].n);
  c->n_cg_parts = n_parts;
  grab((void**)&c->cg_team_bar, sizeof(unsigned) * nrep);
  grab((void**)&c->cg_team_red, sizeof(double) * (size_t)nrep * 2 * kTeamMax);
  grab((void**)&c->cg_parts, sizeof(int2) * n_parts);
  grab((void**)&c->cg_head, 64);
  grab((void**)&c->step_need, sizeof(int) * (size_t)nrep * kStepPhases);
  grab((void**)&c->step_sync, sizeof(int) * (1 + (size_t)nrep * kStepPhases));
  if (ok && cudaMallocHost((void**)&c->tt_host, sizeof(TimeTerms) * (3 * nrep + 1)) != cudaSuccess) {
    cudaGetLastError();
    c->tt_host = nullptr;
    ok = false;
  }
  if (!ok) {
    free(roc); free(poff); free(it_h); free(order);
    pic_destroy(c);
    return PIC_ENOMEM;
  }
  // G^{-1} tables (shared manufactured distribution), then per-replicate copies
  {
    double* tab = (double*)malloc((size_t)(kGinvM + 1) * 2 * 8);
    float* tabf = (float*)malloc((size_t)(kGinvM + 1) * 4 * 4 + (size_t)(kRTabM + 1) * 2 * 4);
    if (tab && tabf) {
      ginv_table(c0.fx_amp, tab);
      ginv_table_f(tab, tabf);
      e = cudaMemcpy(c->ginv, tab, (size_t)(kGinvM + 1) * 2 * 8, cudaMemcpyHostToDevice);
      if (e == cudaSuccess) e = cudaMemcpy(c->ginv_f, tabf, (size_t)(kGinvM + 1) * 4 * 4 + (size_t)(kRTabM + 1) * 2 * 4,
                                         cudaMemcpyHostToDevice);
    } else {
      e = cudaErrorMemoryAllocation;
    }
    free(tab);
    free(tabf);
  }
  c->P.ginv = c->ginv;
  c->P.ginv_f = c->ginv_f;
  c->P.ginv_M = kGinvM;
  for (int r = 0; r < nrep; ++r) {
    c->prm_host[r].ginv = c->ginv;
    c->prm_host[r].ginv_f = c->ginv_f;
    c->prm_host[r].ginv_M = kGinvM;
    c->reps_host[r].f = params_f(c->prm_host[r]);
  }
  if (e == cudaSuccess) e = cudaMemcpy(c->reps_dev, c->reps_host, sizeof(BatchRep) * nrep, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(c->prm_dev, c->prm_host, sizeof(Params) * nrep, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(c->rep_of_cell, roc, sizeof(uint16_t) * nc_tot, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(c->poff_dev, poff, sizeof(int64_t) * (nrep + 1), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && items > 0) e = cudaMemcpy(c->dsmc_items, it_h, sizeof(int2) * items, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(c->cg_order, order, sizeof(int) * nrep, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    // the per-phase solve's (replicate, part) queue, largest replicates first
    int2* parts = (int2*)malloc(sizeof(int2) * (size_t)c->n_cg_parts);
    if (!parts) {
      e = cudaErrorMemoryAllocation;
    } else {
      int k = 0;
      for (int i = 0; i < nrep; ++i) {
        const int r = order[i];
        const int T = cg_team_size(cfgs[r].n * cfgs[r].n * cfgs[r].n);
        for (int t = 0; t < T; ++t) parts[k++] = make_int2(r, t);
      }
      e = cudaMemcpy(c->cg_parts, parts, sizeof(int2) * (size_t)c->n_cg_parts, cudaMemcpyHostToDevice);
      free(parts);
    }
  }
  free(roc); free(poff); free(it_h); free(order);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->counters, 0, 64, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->flags, 0, 64, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->cg_info, 0, 64, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    pic_destroy(c);
    return cuda_status(e);
  }
  // the step's work items for the first candidate the autotuner tries (a
  // block size that fits)
  e = build_step_items(c, c->step_grid[0] > 0 ? 0 : step_candidates() / 2);
  if (e != cudaSuccess) {
    cudaGetLastError();
    pic_destroy(c);
    return cuda_status(e);
  }
  // graphs cannot capture the legacy default stream
  c->use_graphs = c->stream != nullptr;
  *out = c;
  return PIC_OK;
}

pic_status pic_batch_mms_error(pic_ctx* c, pic_errors* out) {
  if (!c || !out || c->nrep < 1) return PIC_EINVAL;
  if (!c->sampled) return PIC_ESTATE;
  for (int r = 0; r < c->nrep; ++r) {
    const double t = c->t0 + (double)c->step * c->prm_host[r].dt;
    CK(launch_batch_errors(c, r, t));
    double h[14];
    CK(cudaMemcpyAsync(h, c->err_out, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    for (int q = 0; q < 7; ++q) {
      out[r].eps2[q] = h[q];
      out[r].epsinf[q] = h[7 + q];
    }
  }
  return check_pending(c);
}

pic_status pic_batch_get_state(pic_ctx* c, int32_t rep, double* x, double* v) {
  if (!c || !x || !v || c->nrep < 1 || rep < 0 || rep >= c->nrep) return PIC_EINVAL;
  if (!c->sampled) return PIC_ESTATE;
  const size_t bytes = (size_t)c->prm_host[rep].np * 3 * 8;
  CK(launch_batch_store_state(c, rep, c->stage));
  CK(cudaMemcpyAsync(x, c->stage, bytes, cudaMemcpyDefault, c->stream));
  CK(cudaMemcpyAsync(v, c->stage + 3 * c->prm_host[rep].np, bytes, cudaMemcpyDefault, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return PIC_OK;
}

pic_status pic_batch_info(pic_ctx* c, int32_t* nrep, int64_t* n_particles, int32_t* cg_iters) {
  if (!c) return PIC_EINVAL;
  if (nrep) *nrep = c->nrep;
  if (n_particles) *n_particles = c->P.np;
  if (cg_iters && c->nrep > 0) {
    CK(cudaMemcpyAsync(cg_iters, c->cg_iters_rep, sizeof(int) * c->nrep, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
  }
  return PIC_OK;
}

const char* pic_status_string(pic_status s) {
  switch (s) {
    case PIC_OK: return "ok";
    case PIC_EINVAL: return "invalid argument or configuration";
    case PIC_ENOMEM: return "allocation failed";
    case PIC_ECUDA: return "CUDA error";
    case PIC_ENOCONV: return "Poisson CG did not reach its tolerance within cg_maxit";
    case PIC_ETIMEOUT: return "a bounded device-side wait timed out";
    case PIC_ESTATE: return "call out of order (sample or set the state first)";
    case PIC_ECAPACITY: return "a cell held more particles than max_ppc";
  }
  return "unknown status";
}

}  // extern "C"
