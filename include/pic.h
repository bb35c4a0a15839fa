/*
 * pic.h - C ABI of the GB300 manufactured-solution PIC + DSMC time step.
 *
 * The method is the one of Freno, McDoniel, Moore and Matula, "Code-
 * Verification Techniques for Particle-in-Cell Simulations with Direct
 * Simulation Monte Carlo Collisions": a 3D periodic electrostatic
 * particle-in-cell step (cloud-in-cell deposit, Poisson solve, gather,
 * velocity-Verlet push; Sec. 2 and Eq. velocity_verlet) with binary elastic
 * no-time-counter collisions (Algorithm 1) averaged over K independent
 * outcomes (Eq. avg_outcome), driven by manufactured solutions obtained by
 * inverse-CDF queries (Eq. mms_sol, Eq. eom_mms, Eq. poisson_mms).
 *
 * Conventions shared by every entry point:
 *  - All work is enqueued on the CUDA stream given to pic_create, in call
 *    order. Every call that returns a device-side status or host data
 *    (pic_sample_mms, pic_set_state, pic_step, pic_collide_avg,
 *    pic_mms_error, pic_get_*) synchronises that stream before returning.
 *  - Particle arrays crossing the boundary are indexed by particle id (pid,
 *    0 .. N_p-1) and laid out [N_p][3] (component fastest), FP64. Mesh
 *    arrays are [n^3] with x fastest (node (i,j,k) at index i + n (j + n k),
 *    position (i h, j h, k h), h = 1/n), vector fields [n^3][3].
 *  - Pointers marked "host or device" may point to host memory (pageable or
 *    pinned) or device memory of the context's GPU, 8-byte aligned for FP64
 *    arrays. Device memory and pinned (registered) host memory may be read
 *    or written by the kernels in place, the latter over NVLink-C2C;
 *    pageable memory is staged through a copy (cudaMemcpyDefault). Either
 *    way the array must hold the stated number of elements. The caller owns
 *    every pointer it passes; the library never keeps one after the call
 *    returns.
 *  - No call throws. Every call returns a pic_status; a failed call leaves
 *    the context usable unless it returns PIC_ESTATE or PIC_ECUDA.
 *  - The context owns all device buffers. pic_destroy(NULL) is a no-op.
 *  - One context is used by one host thread at a time.
 */
#ifndef PIC_GB300_PIC_H
#define PIC_GB300_PIC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pic_ctx pic_ctx;

typedef enum {
  PIC_OK = 0,
  PIC_EINVAL = 1,     /* invalid argument or configuration                 */
  PIC_ENOMEM = 2,     /* device or host allocation failed                  */
  PIC_ECUDA = 3,      /* a CUDA runtime call or kernel launch failed       */
  PIC_ENOCONV = 4,    /* the Poisson CG hit cg_maxit before cg_tol         */
  PIC_ETIMEOUT = 5,   /* a bounded device-side wait gave up                */
  PIC_ESTATE = 6,     /* call out of order (e.g. pic_step before sampling) */
  PIC_ECAPACITY = 7   /* a cell held more particles than max_ppc           */
} pic_status;

enum { PIC_FP64 = 0, PIC_MIXED = 1 };

/* Verification switches of pic_config.verify (bit flags, Sec. 5.4 and 5.1):
 *  PIC_VERIFY_ISOLATE  isolated-collision mode: the drift moves x by the
 *                      exact manufactured increment x^M(t_{n+1}) - x^M(t_n)
 *                      instead of dt xdot^M(t_{n+1/2}); with q/m = 0
 *                      (couple_qm_zero) the particle error is then the
 *                      collision error alone. v^M does not depend on t, so
 *                      the kicks' vdot^M terms are zero in both modes.
 *  PIC_VERIFY_ERROR1   injected coding error 1: v_cm = (v_p - v_q)/2.
 *  PIC_VERIFY_ERROR2   injected coding error 2: an accepted pair swaps its
 *                      velocities with probability 1/2 (the coin is the
 *                      chi draw, U < 1/2) or keeps them. Exclusive with 1.
 *  PIC_VERIFY_ANGLES   record the scattering angles of every collision for
 *                      pic_get_angle_stats (Sec. 4.4).
 *  PIC_VERIFY_ANISO    manufactured anisotropic scattering (Sec. 5.1):
 *                      p_chi = (29/2 + 12 cos chi - 20 cos^3 chi) sin chi
 *                      / 29, drawn by the closed-form quartic inverse; its
 *                      mean cos chi is 0, so the hard-sphere source term
 *                      is unchanged.
 * Only single contexts accept them (pic_create_batch rejects any bit). */
enum {
  PIC_VERIFY_ISOLATE = 1,
  PIC_VERIFY_ERROR1 = 2,
  PIC_VERIFY_ERROR2 = 4,
  PIC_VERIFY_ANGLES = 8,
  PIC_VERIFY_ANISO = 16
};

/* Manufactured-distribution forms of pic_config.dist:
 *  PIC_DIST_CONFIG  f_{x_d} = 1 + fx_amp sin(2 pi (x - fx_speed t)) and a
 *                   Gaussian f_v (mean v_mean, width v_sigma), constant in t.
 *  PIC_DIST_PAPER   the paper's own problem of Sec. 5.2 on the unit cube
 *                   (lengths in units of the box edge L, times in units of
 *                   t_ref = T): f_{x_d} = 1 + A_d(t) sin(2 pi (x - s_d(t)))
 *                   with A = (e^{t/T}/5, 1/5, -e^{t/T}/6) and
 *                   s = (0, 3 e^{t/T}/20, -e^{t/T}/15); the non-Maxwellian
 *                   f_{v_d} = (2/sqrt pi) v^2/vh_d^3 e^{-v^2/vh_d^2} of Eq. fv
 *                   with vh = v_bar (1 + sin(pi t/(2T))/5, 1 + cos(pi t/T)/5,
 *                   1 + sin(3 pi t/(2T))/5). v^M(t) = vh(t) tau(xi) and
 *                   vdot^M = vh'(t) tau(xi) enter the kicks (Eq.
 *                   velocity_verlet). Single contexts of either precision
 *                   (pic_create_batch and pic_adjoint_gradient reject it);
 *                   collisions need the odd-power cross section (n_sigma >=
 *                   1), whose source is closed-form for this f_v (Eq. fn);
 *                   the isolated-collision switch is not available. */
enum { PIC_DIST_CONFIG = 0, PIC_DIST_PAPER = 1 };

/* Bins per angle of the recorded-angle histograms. */
#define PIC_ANGLE_BINS 4194304

/* Problem statement (unit cube [0,1)^3, periodic). Field meanings:
 *  n             cells = nodes per axis (2 .. 1024); cell (i,j,k) spans
 *                [i h,(i+1) h) x ...; node (i,j,k) sits at (i h, j h, k h).
 *  n_particles   N_p computational particles (1 .. 2^31-1), equal weight
 *                w = n_phys / N_p (Sec. 3.3).
 *  K             N_avg, outcomes averaged per collision call (Eq.
 *                avg_outcome), 0 .. 2^20; 0 switches collisions off.
 *  dt            time step of Eq. velocity_verlet; t_n = t0 + n dt.
 *  qm, q, eps0   charge-to-mass ratio, charge and permittivity (Eqs.
 *                eom_full, poisson); n_phys = N, physical particles in the box.
 *  sigma0, g_max hard-sphere cross section sigma(g) = sigma0 and the g_max
 *                of (sigma g)_max = sigma0 g_max (Algorithm 1, Sec. 5.2).
 *  fx_amp, fx_speed  manufactured density f_{x_d}(x,t) = 1 + fx_amp
 *                sin(2 pi (x - fx_speed t)) per axis (Eq. fx); |fx_amp| < 1.
 *  v_mean, v_sigma   manufactured Gaussian velocity density per axis (Eq. fv
 *                replaced by a Gaussian of common width v_sigma > 0).
 *  phi_amp, phi_T, phi_shift  manufactured potential phi^M = phi_amp
 *                e^{t/(2 phi_T)} prod_d sin(2 pi (x_d - phi_shift_d))
 *                (Sec. 5.2 form).
 *  couple_qm_zero  nonzero: q/m = 0 in the push (field does not act).
 *  couple_q_zero   nonzero: q = 0 in the deposit and in rho^M (Sec. 5.3).
 *  precision     PIC_FP64: every step in FP64. PIC_MIXED (the precision
 *                form): positions as int32 cell + FP32 offset, FP32
 *                velocities, gather, manufactured terms and scattering, FP32
 *                field and CG vectors; per-cell charge sums, CG inner
 *                products and residual, and the error norms FP64-accurate.
 *  max_ppc       most particles one cell may hold during collisions (working
 *                set of the collision kernel), 0 .. 65536, rounded up to a
 *                multiple of 32; 0 selects 512. The collision kernel keeps
 *                16 max_ppc bytes of bitmaps in shared memory per block, so
 *                pic_create accepts at most 14,528 on a GB300 (227 KB).
 *  seed          Philox4x32-10 key (low word, high word).
 *  cg_tol, cg_maxit  CG stops at ||r||_2 <= cg_tol ||b||_2 or cg_maxit.
 *                The precision form's FP32 vectors limit the attainable
 *                accuracy to about 1e-6 relative, so use 1e-6 there: a
 *                smaller cg_tol costs iterations without adding accuracy
 *                and can end at cg_maxit with PIC_ENOCONV.
 *  verify        PIC_VERIFY_* bit flags (0: the method as stated).
 *  dist          PIC_DIST_* (0: the fields fx_*, v_mean, v_sigma above).
 *  n_sigma       0: hard spheres (sigma0). 1..3: the manufactured cross
 *                section sigma(g) = sum_{k<n_sigma} sigma_n[k] g^{2k-1} of
 *                Eq. sigma_ms with the source of Eqs. vel_change_3 and fn;
 *                (sigma g)_max is its maximum over [0, g_max] (Sec. 5.2),
 *                and sigma(g) g must be >= 0 there. Single contexts (batches
 *                and the adjoint reject it).
 *  v_bar, t_ref  PIC_DIST_PAPER: vbar and T of the manufactured solution. */
typedef struct {
  int32_t n;
  int32_t K;
  int64_t n_particles;
  double dt;
  double qm, q, eps0, n_phys;
  double sigma0, g_max;
  double fx_amp, fx_speed;
  double v_mean[3];
  double v_sigma;
  double phi_amp, phi_T;
  double phi_shift[3];
  int32_t couple_qm_zero, couple_q_zero;
  int32_t precision;
  int32_t max_ppc;
  uint64_t seed;
  double cg_tol;
  int32_t cg_maxit;
  int32_t verify;
  int32_t dist;
  int32_t n_sigma;
  double sigma_n[3];
  double v_bar, t_ref;
} pic_config;

/* Error norms of Sec. 4.3 at the context's current time: index 0..5 =
 * x, y, z (minimum-image), u, v, w over particles; index 6 = phi over nodes. */
typedef struct {
  double eps2[7];
  double epsinf[7];
} pic_errors;

/* Counters accumulated since pic_create or pic_reset_stats. */
typedef struct {
  int64_t n_cand;         /* candidate pairs drawn (Algorithm 1 loop)       */
  int64_t n_coll;         /* accepted collisions                            */
  int64_t n_gmax_exceed;  /* candidates with g > g_max (ratio above 1)      */
  int64_t n_near_ties;    /* accept decisions within the tie bound: FP64
                             |U - sigma g/(sigma g)_max| < 1e-12; precision
                             form |U g_max - g| <= 2^-19 (g_max + U g_max)
                             (hard spheres) or |U (sigma g)_max - sigma g|
                             <= 2^-17 ((sigma g)_max + sigma g), the bound of
                             its FP32 uniforms and velocities (flagged)     */
  int64_t kernel_launches;/* kernels this library launched                  */
  int64_t step;           /* steps taken since sampling                     */
  double t;               /* current time t0 + step dt                      */
  int32_t cg_iters_last;  /* iterations of the last Poisson solve           */
  int32_t cg_iters_max;
  double cg_res_last;     /* last relative residual ||r|| / ||b||           */
  int64_t graph_replays;  /* batched steps replayed from a captured CUDA graph */
  int32_t tuned_block;    /* batches: block size of the persistent step the
                             autotuner chose (0: not tuned yet)            */
  int32_t tuned_tile;     /* batches: its tile-shape configuration (0, 1)   */
  int64_t n_floor_ties;   /* precision form: N_pairs draws whose FP32 sum lay
                             within its rounding bound of an integer, so that
                             its floor may differ from the FP64 one (flagged) */
  int64_t binned_loads;   /* precision form: pic_set_state calls whose sort
                             read the loaded records binned by cell (arrays
                             used in place, every cell within its bin)      */
} pic_stats;

/* Scattering-angle CDF errors of Sec. 4.4 over every collision recorded
 * since sampling or pic_reset_stats (PIC_VERIFY_ANGLES): for alpha in
 * {chi, eps}, e_r = F_emp(alpha_r) - F^M(alpha_r), eps_2 = sqrt(mean e^2),
 * eps_inf = max |e|. chi = acos(g'_z / g) with the pre-collision g and
 * eps = atan2(g'_y, g'_x) in [0, 2 pi) (Eq. angle_recovery); F^M is the
 * isotropic or the manufactured anisotropic CDF (Eqs. Fp_chi, Fp_eps).
 * The device keeps u = F^M(alpha) in PIC_ANGLE_BINS equal bins and puts each
 * sample at its bin's centre with its rank inside the bin, so each e_r is
 * within 1/(2 PIC_ANGLE_BINS) of the exact value of a sample that fell in
 * that bin; max_bin is the largest bin count (ties inside a bin can move
 * the exact empirical CDF by up to max_bin / n_coll). */
typedef struct {
  int64_t n_coll;         /* recorded collisions N_coll                      */
  int64_t max_bin[2];     /* largest bin count, chi and eps                  */
  double eps2_chi, epsinf_chi;
  double eps2_eps, epsinf_eps;
} pic_angle_stats;

/* Optional device allocator (e.g. a framework's caching allocator). Both
 * callbacks are called on the creating thread; alloc returns NULL on
 * failure. NULL selects cudaMalloc / cudaFree. */
typedef struct {
  void* (*alloc)(void* user, uint64_t bytes);
  void (*free)(void* user, void* ptr);
  void* user;
} pic_allocator;

/* Per-kernel timing gathered with CUDA events on the context stream while
 * profiling is on (pic_set_profiling). Index = kernel class:
 * 0 sample, 1 sort (keys/scan/scatter), 2 sort gather + deposit,
 * 3 rhs, 4 cg + E, 5 dsmc, 6 kick/drift, 7 error norms, 8 copies/other. */
#define PIC_NUM_KERNEL_CLASSES 9
typedef struct {
  double ms[PIC_NUM_KERNEL_CLASSES];
  int64_t launches[PIC_NUM_KERNEL_CLASSES];
} pic_kernel_times;

/* Fill *cfg with the defaults (the smallest manufactured workload: n = 8,
 * N_p = 4096, dt = 0.01, K = 16 ...). Host only, no CUDA. */
pic_status pic_config_default(pic_config* cfg);

/* Check a configuration without touching the GPU. Host only, no CUDA.
 * Returns PIC_OK or PIC_EINVAL. */
pic_status pic_validate_config(const pic_config* cfg);

/* Derived constants of a configuration (host only, no CUDA):
 * out[0] = w = n_phys/N_p, out[1] = dV = h^3, out[2] = P_coll,max =
 * (sigma g)_max w dt / dV (Algorithm 1, Eq. p_coll), out[3] = N_p^cell mean,
 * out[4] = the sufficient bound 1/P_coll,max of Eq. navg_ineq. */
pic_status pic_derived(const pic_config* cfg, double out[5]);

/* Create a context on the current CUDA device: validates cfg, allocates
 * all device buffers (via alloc, or cudaMalloc when alloc is NULL) and
 * binds the stream (a cudaStream_t; NULL = legacy default stream).
 * *out is set to NULL on failure: PIC_EINVAL also when max_ppc needs more
 * shared memory than the device gives a block, PIC_ENOMEM when a buffer
 * cannot be allocated. */
pic_status pic_create(const pic_config* cfg, void* cuda_stream, const pic_allocator* alloc,
                      pic_ctx** out);

/* Sec. 3.2: draw xi_{x_i}, xi_{v_i} for every pid from Philox4x32-10
 * (counter (pid_lo, pid_hi, 0, 0xFFFFFF00 | j), j = 0..2, two 52-bit
 * uniforms per block), set x = x^M(t0), v = v^M(t0) by inverse-CDF queries
 * (Eq. mms_sol), sort by (cell, pid), deposit, solve Eq. poisson_mms and
 * compute E at t0. Resets the step counter to 0. */
pic_status pic_sample_mms(pic_ctx* ctx, double t0);

/* Advance nsteps >= 0 steps of Eq. velocity_verlet with the manufactured
 * sources of Eq. eom_mms: per step, K-averaged collision call A at
 * (x^n, v^n) and call B at (x^{n+1}, v^{n+1/2}), each with the full dt in
 * P_coll and applied with weight 1/2; the field is re-solved at t^{n+1}.
 * Synchronises the stream once at the end and returns the first device-
 * side failure of the steps: PIC_ENOCONV if a Poisson solve missed cg_tol
 * (the steps still complete), PIC_ECAPACITY if a cell exceeded max_ppc
 * (its collisions were skipped), PIC_ETIMEOUT if a bounded device wait gave
 * up (the field is then invalid). */
pic_status pic_step(pic_ctx* ctx, int32_t nsteps);

/* One K-averaged collision call (Eq. avg_outcome, Algorithm 1) on the
 * current state: counter word 2 step + phase (phase 0 or 1). The draws of
 * cell k, outcome o come from Philox4x32-10 with counter (2 step + phase,
 * k, slot, (o << 8) | b): the words of stream b = 1 in slot order are the
 * N_pairs uniform, then one chi per candidate (candidate s: word (s + 1)
 * mod 4 of slot (s + 1) / 4); candidate s takes stream b = 0 at slot s,
 * (p, q, accept, epsilon). Writes
 * <Delta v_p>_coll to dv and the analytic <Delta v_p^M>_coll to dvM (Eq.
 * vel_change_1c for hard spheres with the Gaussian f_v, Eqs. vel_change_3
 * and fn for the odd-power cross section, f_v at the context's current
 * time), both [N_p][3], pid indexed, host or device. Does not change the
 * state. */
pic_status pic_collide_avg(pic_ctx* ctx, int32_t phase, double* dv, double* dvM);

/* Error norms of Sec. 4.3 at the current time into *out (host). */
pic_status pic_mms_error(pic_ctx* ctx, pic_errors* out);

/* Copy the particle state out: x, v [N_p][3], pid indexed, host or device.
 * Pinned host and device arrays of the context's GPU are written in place
 * by the kernels (other memory through a staging copy). */
pic_status pic_get_state(pic_ctx* ctx, double* x, double* v);

/* Replace the particle state (x in [0,1)^3, v; [N_p][3], pid indexed, host
 * or device), set the time to t0 + step dt, re-sort and re-solve the field
 * (the CG starts from the potential the context holds). v^M of a particle
 * depends only on its pid and the distribution, so a context that already
 * holds a state keeps those values rather than deriving them again.
 * Pinned host and device arrays of the context's GPU are read in place.
 * Memory: in the precision form, the first such load (or pic_sample_mms)
 * allocates per-cell bins of the loaded records, ncell x (four times the
 * mean particles per cell, rounded up to 32) x 48 bytes (about four times
 * the particle state), when they hold at most eight times the loaded
 * records and take at most a quarter of the free device memory; they stay
 * with the context (released by pic_destroy). Without
 * them, or when a cell holds more particles than its bin, the load sorts
 * the same state by a scatter and a random gather. */
pic_status pic_set_state(pic_ctx* ctx, const double* x, const double* v, double t0,
                         int64_t step);

/* Failure injection for tests, made on the host and caught by a bounded
 * device wait. Single contexts: the next Poisson solve (of pic_sample_mms,
 * pic_set_state or pic_step) launches one block that leaves before its
 * first grid barrier, so the other blocks wait for an arrival that never
 * comes. Batches: the next pic_step's persistent launch leaves one work
 * item (the first drift-kick tile of a replicate) uncounted, so the items
 * that depend on it wait for a completion that never comes. Either bounded
 * wait (4e9 SM cycles, about 2 s) ends the launch. That call returns
 * PIC_ETIMEOUT, and the field and the state it moves are invalid. The
 * context stays usable: the next pic_sample_mms or pic_set_state starts
 * clean. PIC_EINVAL for a single-context solve of one block (nothing would
 * wait). */
pic_status pic_inject_barrier_stall(pic_ctx* ctx);

/* Copy mesh quantities out (any pointer may be NULL): rho [n^3] (the CIC
 * charge density of Sec. 2), phi [n^3], E [n^3][3]; host or device. */
pic_status pic_get_field(pic_ctx* ctx, double* rho, double* phi, double* E);

/* Copy the sort out (any pointer may be NULL): cell of every pid [N_p],
 * count [n^3], start [n^3 + 1], perm [N_p] = pids in (cell, pid) order;
 * int32, host or device. */
pic_status pic_get_sort(pic_ctx* ctx, int32_t* cell_of_pid, int32_t* count, int32_t* start,
                        int32_t* perm);

pic_status pic_get_stats(pic_ctx* ctx, pic_stats* out);
/* Zero the counters of pic_stats and the recorded scattering angles. */
pic_status pic_reset_stats(pic_ctx* ctx);

/* Per-step record of the steps taken since the last pic_reset_stats,
 * pic_sample_mms or pic_set_state (the first 4096 of them), written by the
 * kernels themselves, so reading it afterwards does not perturb the timing
 * of the steps: out[i][0] = CG iterations of step i's Poisson solve,
 * out[i][1] = candidate pairs, out[i][2] = accepted collisions, out[i][3] =
 * candidates with g > g_max, the last three summed over both collision
 * calls of the step. out is int64 [cap][4], host or device; *n = the steps
 * written (min(steps recorded, cap)). PIC_EINVAL for a batch. */
pic_status pic_get_step_history(pic_ctx* ctx, int64_t* out, int64_t cap, int64_t* n);

/* Decision log of the collision calls (a verification hook for Algorithm 1;
 * the paper has no counterpart). While on, the collision kernels append one
 * record of 8 int32 per logged decision:
 *   (c0, cell, outcome, slot, p, q, result, kind)
 * c0 = 2 step + phase (Philox counter word 0 of the call), the linear cell
 * index, the outcome k < K, and
 *  - for the N_pairs draw of a (cell, outcome): slot = -1, p = q = -1,
 *    result = N_pairs, kind has PIC_DLOG_NPAIRS;
 *  - for candidate pair s: slot = s, the in-cell indices p and q (0-based,
 *    ascending-pid order of the cell), result = 1 accepted / 0 rejected.
 * kind also carries PIC_DLOG_TIE for an accept decision inside the tie bound
 * of pic_stats.n_near_ties and PIC_DLOG_FLOOR for an N_pairs draw inside the
 * bound of pic_stats.n_floor_ties: the decisions on which the precision
 * form may differ from an FP64 evaluation of the same draws.
 *  mode      PIC_DLOG_OFF (0, the default), PIC_DLOG_FLAGGED (only records
 *            with PIC_DLOG_TIE or PIC_DLOG_FLOOR) or PIC_DLOG_ALL (every
 *            N_pairs draw and candidate pair; slower kernels, for small
 *            problems).
 *  capacity  records kept, 1 .. 2^31-1; the buffer (32 capacity bytes)
 *            comes from the context's allocator. Records beyond it are
 *            counted but dropped.
 * Setting the mode clears the log. Records are appended in no particular
 * order (sort them by (c0, cell, outcome, slot)). PIC_EINVAL for a batch. */
enum { PIC_DLOG_OFF = 0, PIC_DLOG_FLAGGED = 1, PIC_DLOG_ALL = 2 };
enum { PIC_DLOG_TIE = 1, PIC_DLOG_FLOOR = 2, PIC_DLOG_NPAIRS = 4 };
pic_status pic_set_decision_log(pic_ctx* ctx, int32_t mode, int64_t capacity);

/* Copy the logged records into out [cap][8] (host or device; NULL with cap
 * 0 to query), set *n_total to the number of records produced since the
 * log was last cleared (it may exceed the capacity and cap: the first
 * min(n_total, capacity, cap) records are written), and clear the log. */
pic_status pic_get_decision_log(pic_ctx* ctx, int32_t* out, int64_t cap, int64_t* n_total);

/* Pathwise gradient (an extension of the method; the paper has no adjoint):
 * runs nsteps FP64 steps from x^M(0) and the velocities v0 with a uniform
 * applied field E_app in the push, L = dt q/m (E_p + E_app - E^M_p), and
 * returns at t_N
 *   J[1] = (eps0/2) h^3 sum_nodes |E|^2,  J[2] = (1/N_p) sum_p |v_p - v_p^M|^2,
 *   J[0] = J[1] + J[2];
 * when dJ_dEapp or dJ_dv0 is non-NULL, also the gradient of J[0] by a
 * hand-written adjoint of gather, push, CIC deposit, the Poisson solve and
 * the K-averaged collisions with candidate pairs, accept decisions and
 * scattering directions frozen at their sampled values (a pathwise
 * derivative). Checkpoints (x, v, phi, E) every `every` steps; each segment
 * is recomputed bit-identically and swept in reverse, so the result does not
 * depend on `every`. Arguments: ctx an FP64 single context (PIC_EINVAL for
 * the precision form, a batch, or the injected-error switches); E_app 3
 * doubles, host (NULL = 0); v0 [N_p][3] in pid order, host or device (NULL =
 * v^M(0)); J 3 doubles, host; dJ_dEapp 3 doubles, host, or NULL; dJ_dv0
 * [N_p][3], host or device, or NULL. The working set (about 24 N_p bytes x
 * (3 every + 2 ceil(nsteps/every) + 6), plus collision overlays) comes from
 * the context's allocator on first use and is kept. With a gradient the
 * context's particle state afterwards is unspecified (pic_step returns
 * PIC_ESTATE until pic_sample_mms or pic_set_state); without one it holds
 * t_N. PIC_ECAPACITY if an outcome recorded more than 64 accepted pairs. */
pic_status pic_adjoint_gradient(pic_ctx* ctx, int32_t nsteps, int32_t every, const double E_app[3],
                                const double* v0, double J[3], double dJ_dEapp[3], double* dJ_dv0);

/* Angle CDF errors (pic_angle_stats) of the recorded collisions; computed by
 * kernels on the context stream, then synchronised. PIC_ESTATE when the
 * context was created without PIC_VERIFY_ANGLES. */
pic_status pic_get_angle_stats(pic_ctx* ctx, pic_angle_stats* out);

/* Per-kernel CUDA-event timing on the context stream (off by default).
 * Turning it on or off clears the accumulated times. */
pic_status pic_set_profiling(pic_ctx* ctx, int32_t on);
pic_status pic_get_kernel_times(pic_ctx* ctx, pic_kernel_times* out);

/* ---- Batched form: independent replicates advanced together ----------
 * pic_create_batch builds one context holding nrep independent replicates
 * (the refinement-study use of the method: many runs of uneven mesh edge,
 * particle count and N_avg). pic_step advances them with one persistent
 * launch per step: a queue of (phase, replicate, tile) work items that
 * blocks take in order, each waiting (bounded) until the earlier phases of
 * its replicate are complete; the first steps time the launch for each
 * block size and tile shape (pic_stats.tuned_block, tuned_tile), and steady
 * steps replay it from a captured CUDA graph when the context has a
 * non-default stream. cfgs[r] gives replicate r; all must use
 * PIC_MIXED and share every field except n, n_particles, K, dt, sigma0
 * and seed (PIC_EINVAL otherwise); 1 <= nrep <= 65534. Replicate r draws
 * from its own Philox key, local pids and local cell indices, so it
 * reproduces a single-domain PIC_MIXED run of cfgs[r] (up to the reduction
 * order of its Poisson solve). pic_sample_mms and pic_step act on every
 * replicate; replicate r's time is t0 + step * cfgs[r].dt. The
 * single-domain calls pic_collide_avg, pic_mms_error, pic_get_state,
 * pic_set_state, pic_get_field and pic_get_sort return PIC_EINVAL on a
 * batch; use the pic_batch_* calls below. */
pic_status pic_create_batch(const pic_config* cfgs, int32_t nrep, void* cuda_stream,
                            const pic_allocator* alloc, pic_ctx** out);

/* Error norms of Sec. 4.3 for every replicate: out[nrep] (host). */
pic_status pic_batch_mms_error(pic_ctx* ctx, pic_errors* out);

/* State of replicate rep: x, v [n_particles_rep][3], pid indexed, host or device. */
pic_status pic_batch_get_state(pic_ctx* ctx, int32_t rep, double* x, double* v);

/* Number of replicates, total particles, and (optional, host int[nrep]) the
 * CG iterations of every replicate's last Poisson solve. */
pic_status pic_batch_info(pic_ctx* ctx, int32_t* nrep, int64_t* n_particles, int32_t* cg_iters);

void pic_destroy(pic_ctx* ctx);
const char* pic_status_string(pic_status s);

/* Issue rates of the current GPU, measured by short kernels on cuda_stream
 * (NULL = legacy default stream; about 30 ms in all, synchronised), for
 * the roofline of the compute-bound collision kernel (no counterpart in the
 * paper). Every thread of a full grid (8 blocks of 256 threads per SM) runs
 * independent chains of one instruction; out[i] is operations per second
 * over the whole GPU at the clocks it ran at:
 *  out[0] INT32 multiply-add (mad.lo.u32)   out[1] 3-input logic (lop3.b32)
 *  out[2] FP32 FMA (fma.rn.f32)             out[3] FP64 FMA (fma.rn.f64)
 *  out[4] Philox4x32-10 blocks (the collision kernel's generator, round
 *         keys as kernel parameters).
 * PIC_ENOMEM if its 16 KB scratch cannot be allocated, PIC_ECUDA on a CUDA
 * error. */
pic_status pic_measure_alu_peaks(void* cuda_stream, double out[5]);

/* Rate of the host link each way, measured by DMA copies (cudaMemcpyAsync)
 * between a caller's pinned host buffer and a device buffer of the same
 * size on cuda_stream (NULL = legacy default stream; synchronised): one
 * copy each way to warm up, then three host-to-device copies and three
 * device-to-host copies, timed with events. It is the ceiling of
 * pic_set_state and pic_get_state with pinned arrays used in place (no
 * counterpart in the paper).
 *  host   pinned (page-locked) host memory of at least `bytes` bytes; its
 *         content is copied to the device and back, so it is unchanged.
 *  bytes  > 0; the call allocates that much device memory for its duration.
 *  out    out[0] host-to-device, out[1] device-to-host, bytes per second.
 * PIC_EINVAL for a null or non-pinned host pointer or bytes == 0,
 * PIC_ENOMEM if the device buffer cannot be allocated, PIC_ECUDA on a CUDA
 * error. */
pic_status pic_measure_link(void* host, uint64_t bytes, void* cuda_stream, double out[2]);

/* Poisson solve that allocates nothing. The paper has no counterpart: this
 * entry point exists for callers that cannot allocate device memory when
 * they solve (a memory budget fixed at start-up, or a host framework that
 * bans cudaMalloc/cudaFree on its hot path because they synchronise the
 * device). It solves -Lap_h phi = b - mean(b) on the periodic n^3 node mesh
 * (7-point Laplacian, h = 1/n) by the same conjugate-gradient kernel the
 * contexts use, projects phi to zero mean and writes E = -grad_h phi.
 *  n        2 .. 48 (n^3 <= 110,592 nodes); larger meshes return
 *           PIC_EINVAL, nothing is launched.
 *  b        [n^3] right-hand side, device memory, read only.
 *  phi      [n^3] device memory: in, the warm start; out, the solution.
 *  E        [3][n^3] device memory, component-major (E_x, then E_y, E_z).
 *  tol, maxit  stop at ||r||_2 <= tol ||b - mean b||_2 or after maxit
 *           iterations (then PIC_ENOCONV, phi holds the last iterate).
 *  cuda_stream  stream to run on (NULL = legacy default stream); the call
 *           synchronises it before returning.
 *  iters, rel_res  optional host outputs: iterations and ||r|| / ||b||.
 * Its scratch (569,792 doubles: 4.56 MB = 4.35 MiB) is one fixed array
 * inside the library, held on every GPU that loads the library until the
 * process exits. The first call
 * on a device looks up that array's device address (cudaGetSymbolAddress)
 * with the device current. Every call shares the array: calls whose work overlaps on the GPU (two
 * streams, two host threads) race and give wrong results. Host pointers and
 * device memory of another GPU return PIC_EINVAL. Calls no allocating
 * routine. */
pic_status pic_poisson_solve_noalloc(int32_t n, const double* b, double* phi, double* E, double tol,
                                     int32_t maxit, void* cuda_stream, int32_t* iters, double* rel_res);

#ifdef __cplusplus
}
#endif
#endif /* PIC_GB300_PIC_H */
