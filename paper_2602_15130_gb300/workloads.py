"""Synthetic manufactured-solution workloads (parameter recipes only).

The benchmark and study workloads (all recipes except ``paper_*``) are the
periodic unit cube [0,1)^3 with the separable
manufactured position density prod_d (1 + 0.3 sin(2 pi (x_d - 0.1 t))),
Gaussian velocities (mean 0.2, sigma 1 per axis), q/m = q = eps0 = 1, one
physical particle in the box (w = 1/N_p, mean charge density 1), the
manufactured potential phi^M = 0.1 e^{t/2} prod_d sin(2 pi (x_d - s_d)) with
s = (1/7, 1/5, 1/3) (the form of the paper's Sec. 5.2 on the unit cube) and
hard-sphere collisions with isotropic scattering.

The hard-sphere cross section sigma0 is chosen so that a particle undergoes
``coll_per_call`` expected collisions per collision call at the recipe's own
particles per cell and time step: with the mean relative speed of two
Gaussian samples <g> = 4 s / sqrt(pi), Eq. p_coll gives
(c - 1) sigma0 <g> w dt / dV = coll_per_call.

The ``paper_*`` recipes are the paper's own problem of Sec. 5.2 (per-axis
f_x with time-varying amplitude and phase, the non-Maxwellian f_v with
vh(t), the odd-power cross section) expressed in box units; see
``paper_units``.

Nothing here performs any step of the method; these are inputs.
"""
from __future__ import annotations

import math

G_MAX = 10.0 * math.sqrt(3.0)  # g_max = 10 sqrt(3) vbar with vbar = sigma_v = 1


def hard_sphere_sigma0(ppc: float, dt: float, coll_per_call: float = 0.1, v_sigma: float = 1.0) -> float:
    mean_g = 4.0 * v_sigma / math.sqrt(math.pi)
    # w / dV = (1/N_p) / (1/n^3) = 1 / ppc
    return coll_per_call * ppc / ((ppc - 1.0) * mean_g * dt)


def base(n: int, n_particles: int, dt: float, K: int, sigma0: float, seed: int = 0, **kw) -> dict:
    p = dict(
        n=n, n_particles=n_particles, dt=dt, K=K, sigma0=sigma0, g_max=G_MAX, seed=seed,
        qm=1.0, q=1.0, eps0=1.0, n_phys=1.0,
        fx_amp=0.3, fx_speed=0.1, v_mean=(0.2, 0.2, 0.2), v_sigma=1.0,
        phi_amp=0.1, phi_T=1.0, phi_shift=(1.0 / 7.0, 1.0 / 5.0, 1.0 / 3.0),
        couple_qm_zero=0, couple_q_zero=0, cg_tol=1e-10, cg_maxit=20000,
    )
    p.update(kw)
    return p


def smallest(**kw) -> dict:
    """8^3 cells, 4,096 particles, dt = 0.01, 10 steps, K = 16, seed 0,
    about 0.1 collisions per particle per step."""
    n, npart, dt = 8, 4096, 0.01
    p = base(n, npart, dt, 16, hard_sphere_sigma0(npart / n ** 3, dt), steps=10)
    p.update(kw)
    return p


REFINE_PPC = 32
REFINE_DT0 = 0.02
REFINE_T_END = 0.5


def refinement_level(level: int, collisions: bool = True, **kw) -> dict:
    """Refinement sweep level l = 0..4: n = 8 * 2^l, 32 particles per cell,
    dt = 0.02 / 2^l, 0.5 time units, K = 16 (or 0 with collisions off).
    sigma0 is fixed from level 0 (it is physics, not discretisation)."""
    n = 8 * 2 ** level
    dt = REFINE_DT0 / 2 ** level
    sigma0 = hard_sphere_sigma0(REFINE_PPC, REFINE_DT0)
    p = base(n, REFINE_PPC * n ** 3, dt, 16 if collisions else 0, sigma0,
             steps=int(round(REFINE_T_END / dt)))
    p.update(kw)
    return p


# Table 1 of the paper: five discretizations with T/dt = n = 8, 12, 16, 20,
# 24, N_p = 10240 (n/8)^7 and N_avg = 32 (n/8)^5 (collisional, Eq.
# refinements with s = 7, r = 5) or N_p = 10240 (n/8)^5 (collisionless,
# s = 5), and 1/P_coll,max = 108.28 at the first level.
TABLE1_N = (8, 12, 16, 20, 24)
TABLE1_INV_PMAX_L1 = 108.28
TABLE1_T = 0.1   # T = L / (10 vbar) with L = 1 and vbar = sigma_v = 1 (Sec. 5.2)


def table1_sigma0(g_max: float = G_MAX) -> float:
    """Hard-sphere sigma0 giving Table 1's P_coll,max at its first level
    (P_max = sigma0 g_max w dt / dV with w = 1/10240, dt = T/8, dV = 8^-3);
    P_max then follows Table 1 at every level (P_max ~ h^5)."""
    n, npart = TABLE1_N[0], 10240
    dt = TABLE1_T / n
    return (1.0 / TABLE1_INV_PMAX_L1) * (1.0 / n ** 3) / (g_max * (1.0 / npart) * dt)


def table1_level(level: int, collisions: bool = True, **kw) -> dict:
    """Level l = 0..4 of Table 1 on the unit cube: n = 8 + 4 l cells per
    axis, dt = T/n, n steps to T = 0.1; collisional: N_p = 10240 (n/8)^7,
    K = 32 (n/8)^5; collisionless: N_p = 10240 (n/8)^5, K = 0. max_ppc
    covers the densest cell ((1 + 0.3)^3 times the mean) with margin."""
    n = TABLE1_N[level]
    r = n / 8
    npart = int(round(10240 * r ** (7 if collisions else 5)))
    K = int(round(32 * r ** 5)) if collisions else 0
    dt = TABLE1_T / n
    ppc = npart / n ** 3
    max_ppc = int(math.ceil((ppc * 1.3 ** 3 * 1.15 + 64) / 32.0)) * 32
    p = base(n, npart, dt, K, table1_sigma0(), steps=n, max_ppc=max_ppc)
    p.update(kw)
    return p


# ---------------------------------------------------------------------------
# The paper's own problem (Sec. 5.2) in box units: lengths in units of
# L = 1.5 m, times in units of T = L / (10 vbar) = 1.5e-7 s, potentials in
# units of phibar = 1e10 V. Then vbar = 0.1, g_max = 10 sqrt(3) vbar = sqrt 3,
# phi^M = e^{t/2} prod_d sin(2 pi (x_d - s_d)), a run to t = T ends at t = 1,
# and with n_phys = 1 and eps0 = 1:
#   q/m   -> (q/m) phibar T^2 / L^2          (q = e, m = 3e8 m_e)
#   q     -> q N / (eps0 phibar L)           (N = 1e20 physical particles)
#   sigma(g) g -> sigma(g) g N T / L^3       (Eq. p_coll is unit-free)
# The cross section is sigma(g) = sigmabar [a0 vbar/g + a1 g/vbar + a2
# (g/vbar)^3] (Eq. sigma_ms with N_sigma = 3, sigmabar = 1 A^2): the paper
# shows its sigma_n only in a figure, so the reading here is a0 = 1 and a
# peak of sigma(g) g at g^2 = 150 vbar^2 inside [0, g_max], scaled so that
# (sigma g)_max gives Table 1's 1/P_coll,max = 108.28 at the first level
# ((sigma g)_max = 3.3247e-13 m^3/s).
E_CHARGE = 1.602176634e-19
M_ELECTRON = 9.1093837015e-31
EPS0_SI = 8.8541878128e-12
PAPER_L, PAPER_VBAR, PAPER_PHIBAR, PAPER_N = 1.5, 1.0e6, 1.0e10, 1.0e20
PAPER_T = PAPER_L / (10.0 * PAPER_VBAR)
PAPER_SIGMABAR = 1.0e-20
PAPER_SG_PEAK_U = 150.0


def paper_units() -> dict:
    """Box-unit constants of the paper's problem (see above)."""
    qm_si = E_CHARGE / (3.0e8 * M_ELECTRON)
    vbar = PAPER_VBAR * PAPER_T / PAPER_L
    return dict(qm=qm_si * PAPER_PHIBAR * PAPER_T ** 2 / PAPER_L ** 2,
                q=E_CHARGE * PAPER_N / (EPS0_SI * PAPER_PHIBAR * PAPER_L),
                v_bar=vbar, g_max=10.0 * math.sqrt(3.0) * vbar,
                sg_scale=PAPER_SIGMABAR * PAPER_VBAR * PAPER_N * PAPER_T / PAPER_L ** 3)


def paper_sigma_n() -> tuple[float, float, float]:
    """sigma_0..2 in box units: sigma g = C (a0 + a1 u + a2 u^2), u = (g/vbar)^2,
    C = sigmabar vbar N T / L^3, a0 = 1, the peak at u = 150 equal to the
    (sigma g)_max of Table 1's first level."""
    u = paper_units()
    n0, np0 = TABLE1_N[0], 10240
    sg_max = (1.0 / TABLE1_INV_PMAX_L1) * (1.0 / n0 ** 3) / ((1.0 / np0) * (1.0 / n0))
    M = sg_max / u["sg_scale"]                 # peak in units of sigmabar vbar
    a0 = 1.0
    a2 = -(M - a0) / PAPER_SG_PEAK_U ** 2
    a1 = -2.0 * a2 * PAPER_SG_PEAK_U
    C, vb = u["sg_scale"], u["v_bar"]
    return (C * a0, C * a1 / vb ** 2, C * a2 / vb ** 4)


def paper_problem(n: int, n_particles: int, dt: float, K: int, seed: int = 0, **kw) -> dict:
    """The paper's Sec. 5.2 problem in box units (FP64 form)."""
    u = paper_units()
    p = dict(
        n=n, n_particles=n_particles, dt=dt, K=K, seed=seed, dist=1, v_bar=u["v_bar"], t_ref=1.0,
        qm=u["qm"], q=u["q"], eps0=1.0, n_phys=1.0, sigma0=0.0, g_max=u["g_max"],
        n_sigma=3 if K > 0 else 0, sigma_n=paper_sigma_n() if K > 0 else (0.0, 0.0, 0.0),
        phi_amp=1.0, phi_T=1.0, phi_shift=(1.0 / 7.0, 1.0 / 5.0, 1.0 / 3.0),
        couple_qm_zero=0, couple_q_zero=0, cg_tol=1e-10, cg_maxit=20000, precision=0,
    )
    ppc = n_particles / n ** 3
    # densest cell: prod_d (1 + |A_d(T)|) = (1 + e/5)(1 + 1/5)(1 + e/6) times the mean
    p["max_ppc"] = int(math.ceil((ppc * 2.7 * 1.15 + 64) / 32.0)) * 32
    p.update(kw)
    return p


def paper_table1_level(level: int, collisions: bool = True, **kw) -> dict:
    """Level l = 0..4 of Table 1 for the paper's own problem: n = 8 + 4 l,
    dt = T/n, n steps to t = T; N_p = 10240 (n/8)^7 and N_avg = 32 (n/8)^5
    collisional, N_p = 10240 (n/8)^5 collisionless."""
    n = TABLE1_N[level]
    r = n / 8
    npart = int(round(10240 * r ** (7 if collisions else 5)))
    K = int(round(32 * r ** 5)) if collisions else 0
    p = paper_problem(n, npart, 1.0 / n, K, steps=n)
    p.update(kw)
    return p


def paper_small(**kw) -> dict:
    """A small case of the paper's problem for parity tests: 8^3 cells,
    4,096 particles, dt = T/16, K = 8."""
    p = paper_problem(8, 4096, 1.0 / 16, 8, steps=4, cg_tol=1e-13)
    p.update(kw)
    return p


PRECISION_CG_TOL = 1e-6


# Expected collisions per particle per call of the precision-form study.
# The collisional MMS error is zero-mean but not damped: it grows as a
# random walk whose variance per step scales with the collision rate over K,
# and once a velocity's relative speed to its cell-mates passes g_max, NTC
# under-collides it while the analytic source keeps growing (the runaway of
# the fixed-ppc sweep). Measured at 128^3, 64 per cell, K = 32, dt = 0.005
# over 200 steps: 0.1 per call passes g_max at step 9 and is non-finite at
# step 20; 0.05 runs away near step 50; 0.025 near step 110 (FP32) and 140
# (FP64); 0.011 stays finite to step 200 with no relative speed above g_max.
PRECISION_COLL_PER_CALL = 0.01


def precision_form(**kw) -> dict:
    """128^3 cells, 64 particles per cell (134,217,728), K = 32, dt = 0.005,
    200 steps, FP32 particle state (int32 cell + FP32 offset); sigma0 gives
    0.01 expected collisions per particle per call (PRECISION_COLL_PER_CALL:
    the largest round rate whose 200-step run stays finite); CG to a
    relative residual of 1e-6 (FP32 vectors)."""
    n, ppc, dt = 128, 64, 0.005
    p = base(n, ppc * n ** 3, dt, 32, hard_sphere_sigma0(ppc, dt, PRECISION_COLL_PER_CALL), steps=200,
             precision=1, cg_tol=PRECISION_CG_TOL)
    p.update(kw)
    return p


DIFF_COLL_PER_CALL = 0.005


def differentiation(**kw) -> dict:
    """Pathwise-gradient study: 64^3 cells, 64 particles per cell
    (16,777,216), 200 steps of dt = 0.005, K = 8, FP64, applied field
    E_app = (0.1, 0.1, 0.1), checkpoints every 20 steps. sigma0 gives 0.005
    expected collisions per particle per call: at 0.02 and above, K = 8
    leaves a collision error that grows until velocities pass g_max and run
    away within the 200 steps (the saturated-NTC runaway of the fixed-ppc
    sweep). CG is capped at 2000 iterations so a diverging run stops."""
    n, ppc, dt = 64, 64, 0.005
    p = base(n, ppc * n ** 3, dt, 8, hard_sphere_sigma0(ppc, dt, DIFF_COLL_PER_CALL), steps=200,
             E_app=(0.1, 0.1, 0.1), checkpoint_every=20, cg_maxit=2000)
    p.update(kw)
    return p


def mixed(p: dict) -> dict:
    """The same workload in the precision form."""
    q = dict(p)
    q["precision"] = 1
    q["cg_tol"] = max(p.get("cg_tol", 1e-10), PRECISION_CG_TOL)
    return q


def scaled(p: dict, n: int) -> dict:
    """Same particles per cell, K and dt on an n^3 mesh (used for bounded
    samples of a large workload)."""
    q = dict(p)
    ppc = p["n_particles"] / p["n"] ** 3
    q["n"] = n
    q["n_particles"] = int(round(ppc * n ** 3))
    return q


def batched(n_rep: int = 256, seed: int = 42, dt: float = 0.005, steps: int = 100) -> list[dict]:
    """Batched refinement study: n_rep independent replicates; mesh edge
    uniform on {8, 16, 32, 64}, particles per cell uniform in [8, 64], K
    uniform in [4, 64] (drawn from a host generator seeded with ``seed``),
    replicate r with Philox seed 1000 + r; same manufactured distribution,
    precision form, dt = 0.005, sigma0 from the 0.1-collision rule at each
    replicate's particles per cell."""
    import numpy as np

    g = np.random.default_rng(seed)
    out = []
    for r in range(n_rep):
        n = int(g.choice([8, 16, 32, 64]))
        ppc = int(g.integers(8, 65))
        K = int(g.integers(4, 65))
        p = base(n, ppc * n ** 3, dt, K, hard_sphere_sigma0(ppc, dt), seed=1000 + r, steps=steps, precision=1,
                 cg_tol=PRECISION_CG_TOL)
        out.append(p)
    return out
