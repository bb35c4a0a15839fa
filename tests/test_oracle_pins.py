"""Pins of the FP64 CPU oracle against what the paper and mathematics fix.

Each test checks the oracle against something other than itself: published
known-answer vectors, a table the paper prints, closed forms, library special
cases (scipy ndtri, numpy FFT, scipy quadrature), invariants (conservation,
normalisation) and brute force on tiny inputs.
"""
import math
from pathlib import Path

import numpy as np
import pytest
from scipy import integrate, special, stats

import inputs
from oracle import oracle as O
from paper_2602_15130_gb300 import workloads as W

GOLDEN = Path(__file__).parent / "golden"


def cfg(**kw):
    return O.make_cfg(W.smallest(**kw))


# --------------------------------------------------------------- Philox ----
def test_philox_known_answers():
    rows = [l.split() for l in (GOLDEN / "philox4x32_10_kat.txt").read_text().splitlines()
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        assert O.philox(v[0:4], v[4:6]) == v[6:10]


def test_uniform_conventions():
    L = O.lib()
    assert L.orc_u52(0, 0) == 2.0 ** -53
    assert L.orc_u52(0xFFFFFFFF, 0xFFFFFFFF) == 1.0 - 2.0 ** -53
    assert L.orc_u32(0) == 2.0 ** -33
    assert L.orc_u32(0xFFFFFFFF) == 1.0 - 2.0 ** -33
    g = np.random.default_rng(5)
    for w, c in zip(g.integers(0, 2 ** 32, 2000), g.integers(1, 5000, 2000)):
        assert L.orc_index(int(w), int(c)) == (int(w) * int(c)) >> 32
        assert 0 <= L.orc_index(int(w), int(c)) < c


def test_sampling_xi_uniform_and_distinct():
    c = cfg()
    xi = np.array([O.sample_xi(c, p) for p in range(4000)])
    assert np.all((xi > 0) & (xi < 1))
    for j in range(6):
        assert stats.kstest(xi[:, j], "uniform").pvalue > 1e-4
    # the six streams of one particle are not copies of one another
    assert np.abs(np.corrcoef(xi.T) - np.eye(6)).max() < 0.1


# ------------------------------------------------- manufactured solution ----
@pytest.mark.parametrize("t", [0.0, 0.37, 2.5])
def test_Fx_is_integral_of_fx(t):
    c = cfg()
    for x in [0.0, 0.1, 0.33, 0.5, 0.77, 1.0]:
        q, _ = integrate.quad(lambda s: O.fxd(c, s, t), 0.0, x, epsabs=1e-15, epsrel=1e-13)
        assert abs(O.Fxd(c, x, t) - q) < 1e-13
    assert abs(O.Fxd(c, 1.0, t) - 1.0) < 1e-15


def test_xM_inverts_F_and_has_right_mean():
    c = cfg()
    g = np.random.default_rng(1)
    for xi in g.random(200):
        for t in (0.0, 0.31, 1.7):
            x = O.xM(c, xi, t)
            assert 0.0 <= x <= 1.0
            assert abs(O.Fxd(c, x, t) - xi) < 4e-16
    # E[x^M] over uniform xi equals int_0^1 x f_x dx (midpoint rule in xi)
    N = 4000
    t = 0.42
    xs = np.array([O.xM(c, (i + 0.5) / N, t) for i in range(N)])
    mean_ref, _ = integrate.quad(lambda s: s * O.fxd(c, s, t), 0, 1, epsabs=1e-14)
    assert abs(xs.mean() - mean_ref) < 1e-6


def test_xMdot_matches_finite_difference():
    c = cfg()
    d = 1e-5
    for xi in [0.05, 0.3, 0.5, 0.81, 0.99]:
        for t in [0.0, 0.2, 1.3]:
            fd = (O.xM(c, xi, t + d) - O.xM(c, xi, t - d)) / (2 * d)
            assert abs(O.xMdot(c, O.xM(c, xi, t), t) - fd) < 1e-8


def test_vM_is_normal_quantile():
    c = cfg()
    g = np.random.default_rng(2)
    xis = np.concatenate([g.random(300), [1e-15, 1e-9, 0.5, 1 - 1e-9, 1 - 2 ** -52]])
    for d in range(3):
        for xi in xis:
            ref = c.vmean[d] + c.vsig * special.ndtri(xi)
            assert abs(O.vM(c, d, xi) - ref) < 2e-14 * max(1.0, abs(ref))


def test_phiM_field_and_laplacian_by_finite_differences():
    c = cfg()
    g = np.random.default_rng(3)
    d = 1e-5
    for _ in range(20):
        x = g.random(3)
        t = g.random()
        E = O.EM(c, x, t)
        lap = 0.0
        for k in range(3):
            e = np.zeros(3); e[k] = d
            fd = (O.phiM(c, x + e, t) - O.phiM(c, x - e, t)) / (2 * d)
            assert abs(E[k] + fd) < 1e-9
            dd = 1e-3
            e = np.zeros(3); e[k] = dd
            lap += (O.phiM(c, x + e, t) - 2 * O.phiM(c, x, t) + O.phiM(c, x - e, t)) / dd ** 2
        assert abs(O.lap_phiM(c, x, t) - lap) < 1e-4 * max(1.0, abs(lap))


def test_rhoM_integrates_to_total_charge():
    c = cfg()
    t = 0.6
    # separable: the integral is q N times the product of 1D integrals
    one_d = integrate.quad(lambda s: O.fxd(c, s, t), 0, 1)[0]
    assert abs(one_d - 1.0) < 1e-13
    pts, wts = np.polynomial.legendre.leggauss(24)
    pts = 0.5 * (pts + 1.0); wts = 0.5 * wts
    tot = 0.0
    for i, xi in enumerate(pts):
        for j, yj in enumerate(pts):
            for k, zk in enumerate(pts):
                tot += wts[i] * wts[j] * wts[k] * O.rhoM(c, 2.0, [xi, yj, zk], t)
    assert abs(tot - 2.0) < 1e-12


# ------------------------------------------------- hard-sphere source -----
def _quad_E_absX_Xpar(a):
    """E[|X| X_par] for X ~ N((a,0,0), I) by 2D quadrature (cylindrical)."""
    def f(rho, x):
        return math.sqrt(x * x + rho * rho) * x * math.exp(-0.5 * (x - a) ** 2) / math.sqrt(2 * math.pi) \
            * rho * math.exp(-0.5 * rho * rho)
    val, err = integrate.dblquad(f, a - 13, a + 13, 0, 13, epsabs=1e-13, epsrel=1e-12)
    return val


@pytest.mark.parametrize("a", [0.02, 0.0999, 0.1001, 0.35, 1.0, 2.7, 7.5])
def test_hs_R_against_quadrature(a):
    # E[|X| X] = s R(a) m; with s = 1, |m| = a the parallel component is R(a) a
    assert abs(O.hs_R(a) * a - _quad_E_absX_Xpar(a)) < 1e-10


def test_hs_R_small_a_limit_and_continuity():
    # R(0) = (8/3) sqrt(2/pi): E[|X|X] ~ (4/3) m s E|Z|, E|Z| = 2 sqrt(2/pi)
    assert abs(O.hs_R(0.0) - 8.0 / 3.0 * math.sqrt(2 / math.pi)) < 1e-15
    assert abs(O.hs_R(0.1 - 1e-12) - O.hs_R(0.1 + 1e-12)) < 1e-13


def test_hs_source_monte_carlo_vector():
    """E[|v_q - v_p|(v_q - v_p)] by Monte Carlo, anisotropic offset, s != 1."""
    c = O.make_cfg(W.smallest(v_sigma=1.7, v_mean=(0.2, -0.4, 1.1)))
    vp = np.array([0.9, 0.1, -0.3])
    g = np.random.default_rng(11)
    vq = np.array(c.vmean[:])[None, :] + 1.7 * g.standard_normal((2_000_000, 3))
    X = vq - vp
    samp = np.linalg.norm(X, axis=1)[:, None] * X
    mc, se = samp.mean(0), samp.std(0) / math.sqrt(len(samp))
    ccell = 9
    pref = (1.0 / c.np) * c.dt * (ccell - 1) * c.sigma0 / (2.0 * (1.0 / c.n) ** 3)
    src = O.hs_source(c, vp, ccell)
    assert np.all(np.abs(src / pref - mc) < 5 * se)


def test_source_equals_expected_ntc_change():
    """<Delta v^M> equals the outcome- and sample-average of Algorithm 1's
    Delta v_p for a particle whose cell partners are drawn from f_v
    (Eq. vel_change_1a), checked statistically with 512 cells x K outcomes."""
    p = W.smallest(K=3000, dt=0.005)
    n, ppc = p["n"], 6
    p["n_particles"] = n ** 3 * ppc
    o = O.Oracle(p)
    h = 1.0 / n
    g = np.random.default_rng(21)
    ijk = np.stack(np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij"), -1).reshape(-1, 3)
    x = np.repeat((ijk[:, [2, 1, 0]] + 0.5) * h, ppc, axis=0)
    v = 0.2 + g.standard_normal((n ** 3 * ppc, 3))
    vp = np.array([1.2, -0.6, 0.4])
    first = np.arange(0, n ** 3 * ppc, ppc)
    v[first] = vp
    o.set_state(x, v)
    dv, dvM = o.collide_avg(0)
    est = dv[first]
    mean, se = est.mean(0), est.std(0) / math.sqrt(len(first))
    src = O.hs_source(o.cfg, vp, ppc)
    assert np.allclose(dvM[first], src, rtol=0, atol=1e-15)
    # the first-order (no repeated-collision) expectation is exact to O(P^2)
    assert O.pmax(o.cfg) < 0.08
    assert np.all(np.abs(mean - src) < 4.5 * se + 0.02 * np.abs(src))


# ------------------------------------------------------- P_max, Table 1 ---
def test_pmax_against_paper_table1():
    rows = [list(map(float, l.split())) for l in (GOLDEN / "paper_table1_discretizations.txt").read_text().splitlines()
            if l.strip() and not l.startswith("#")]
    implied = []
    for lvl, steps, nax, ncell, navg, inv_p, np_coll, np_free in rows:
        assert nax ** 3 == ncell
        c = O.make_cfg(dict(n=int(nax), n_particles=int(np_coll), K=int(navg), dt=1.0 / steps,
                            sigma0=1.0, g_max=1.0, n_phys=1e20))
        # with (sigma g)_max = 1 in units of the box, P_max = w dt / dV
        implied.append(1.0 / (inv_p * O.pmax(c)))
    implied = np.array(implied)
    assert np.all(np.abs(implied / implied[0] - 1) < 2e-4)


def test_refinement_schedule_matches_table1():
    rows = [list(map(float, l.split())) for l in (GOLDEN / "paper_table1_discretizations.txt").read_text().splitlines()
            if l.strip() and not l.startswith("#")]
    for lvl, steps, nax, ncell, navg, inv_p, np_coll, np_free in rows:
        f = nax / 8.0
        # Eq. refinements with s = 7, r = 5 (collisional) and s = 5 (collisionless)
        assert round(10240 * f ** 7) == np_coll
        assert round(10240 * f ** 5) == np_free
        assert round(32 * f ** 5) == navg


# ----------------------------------------------------------- sort / CIC ---
def test_sort_is_cell_then_pid():
    p = W.smallest(n_particles=3000)
    o = O.Oracle(p)
    x, v = inputs.particles(3000, seed=4, clustered_cells=40, n=8)
    o.set_state(x, v)
    cell, count, start, perm = o.sort()
    ref_cell = np.clip(np.floor(x * 8).astype(int), 0, 7)
    ref_cell = ref_cell[:, 0] + 8 * (ref_cell[:, 1] + 8 * ref_cell[:, 2])
    assert np.array_equal(cell, ref_cell)
    assert np.array_equal(perm, np.lexsort((np.arange(3000), ref_cell)))
    assert np.array_equal(count, np.bincount(ref_cell, minlength=512))
    assert np.array_equal(start[1:], np.cumsum(count))


def _brute_cic(x, n, scale):
    h = 1.0 / n
    nodes = np.stack(np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij"), -1).reshape(-1, 3)[:, [2, 1, 0]] * h
    d = x[:, None, :] - nodes[None, :, :]
    d -= np.round(d)
    S = np.prod(np.maximum(0.0, 1.0 - np.abs(d) / h), axis=2)
    return scale * S.sum(0)


def test_deposit_brute_force_and_total_charge():
    n, npart = 4, 300
    p = W.smallest(n=n, n_particles=npart)
    o = O.Oracle(p)
    x, v = inputs.particles(npart, seed=6)
    o.set_state(x, v)
    rho, phi, E = o.field()
    scale = 1.0 * (1.0 / npart) / (1.0 / n) ** 3
    assert np.allclose(rho, _brute_cic(x, n, scale), rtol=0, atol=1e-13)
    assert abs(rho.sum() * (1.0 / n) ** 3 - 1.0) < 1e-13


def test_gather_reproduces_nodes_and_affine_fields():
    c = cfg()
    n = c.n
    g = np.random.default_rng(8)
    E = g.standard_normal((n ** 3, 3))
    h = 1.0 / n
    for idx in [0, 5, 77, 511]:
        i, j, k = idx % n, (idx // n) % n, idx // n ** 2
        assert np.allclose(O.gather(c, E, [i * h, j * h, k * h]), E[idx], atol=1e-15)
    # an affine field on the nodes of one interior cell is reproduced inside it
    A = g.standard_normal((3, 3)); b = g.standard_normal(3)
    E2 = np.zeros((n ** 3, 3))
    for k in range(n):
        for j in range(n):
            for i in range(n):
                E2[i + n * (j + n * k)] = b + A @ np.array([i, j, k]) * h
    for _ in range(20):
        xx = (np.array([2, 3, 4]) + g.random(3)) * h
        assert np.allclose(O.gather(c, E2, xx), b + A @ xx, atol=1e-13)


# ------------------------------------------------------------ Poisson -----
def test_neg_laplacian_eigenvalues():
    n = 8
    h = 1.0 / n
    ii = np.arange(n ** 3)
    X = np.stack([ii % n, (ii // n) % n, ii // n ** 2], 1) * h
    for k in [(1, 0, 0), (1, 2, 3), (4, 4, 1)]:
        u = np.sin(2 * np.pi * (k[0] * X[:, 0] + 0.1)) * np.cos(2 * np.pi * k[1] * X[:, 1]) * \
            np.cos(2 * np.pi * (k[2] * X[:, 2] - 0.3))
        lam = sum(4 / h ** 2 * np.sin(np.pi * kk * h) ** 2 for kk in k)
        assert np.allclose(O.neg_lap(n, u), lam * u, atol=1e-10 * lam)


@pytest.mark.parametrize("n", [4, 8, 16])
def test_cg_matches_fft_solve(n):
    b = inputs.mesh_vector(n, seed=n)
    phi, it, res = O.cg(n, b, np.zeros(n ** 3), 1e-14, 5000)
    assert it > 0 and res <= 1e-14
    bh = np.fft.fftn(b.reshape(n, n, n))
    k = np.fft.fftfreq(n) * n
    h = 1.0 / n
    lam = sum(np.meshgrid(*(4 / h ** 2 * np.sin(np.pi * k * h) ** 2,) * 3, indexing="ij"))
    lam[0, 0, 0] = 1.0
    ph = bh / lam
    ph[0, 0, 0] = 0.0
    ref = np.real(np.fft.ifftn(ph)).reshape(-1)
    assert np.allclose(phi, ref, rtol=0, atol=1e-12 * np.abs(ref).max())
    assert abs(phi.mean()) < 1e-15 * np.abs(ref).max() * n ** 3


def test_efield_central_difference_closed_form():
    n = 16
    h = 1.0 / n
    ii = np.arange(n ** 3)
    X = np.stack([ii % n, (ii // n) % n, ii // n ** 2], 1) * h
    phi = np.sin(2 * np.pi * 3 * X[:, 0]) + np.cos(2 * np.pi * 2 * X[:, 2])
    E = O.efield(n, phi)
    assert np.allclose(E[:, 0], -np.cos(2 * np.pi * 3 * X[:, 0]) * np.sin(2 * np.pi * 3 * h) / h, atol=1e-12)
    assert np.allclose(E[:, 1], 0.0, atol=1e-12)
    assert np.allclose(E[:, 2], np.sin(2 * np.pi * 2 * X[:, 2]) * np.sin(2 * np.pi * 2 * h) / h, atol=1e-12)


@pytest.mark.parametrize("n", [4, 8, 16])
def test_uncoupled_potential_closed_form(n):
    """q = 0: -Lap_h phi = -Lap phi^M = 12 pi^2 phi^M at the nodes, a discrete
    eigenvector with eigenvalue 12 sin^2(pi h)/h^2, so the discrete solution
    is phi^M (pi h)^2 / sin^2(pi h)."""
    p = W.smallest(n=n, n_particles=64, couple_q_zero=1, cg_tol=1e-14)
    o = O.Oracle(p)
    o.sample(0.25)
    rho, phi, E = o.field()
    assert np.all(rho == 0.0)
    h = 1.0 / n
    ii = np.arange(n ** 3)
    X = np.stack([ii % n, (ii // n) % n, ii // n ** 2], 1) * h
    phiM = np.array([O.phiM(o.cfg, X[i], 0.25) for i in range(n ** 3)])
    exact = phiM * (np.pi * h) ** 2 / np.sin(np.pi * h) ** 2
    assert np.allclose(phi, exact, rtol=0, atol=1e-12 * np.abs(exact).max())
    err = o.errors()
    assert abs(err[13] - np.abs(exact - phiM).max()) < 1e-13


# --------------------------------------------------------------- NTC ------
def _cell_velocities(c, seed):
    return 0.2 + np.random.default_rng(seed).standard_normal((c, 3))


@pytest.mark.parametrize("dist", [0, 1])
def test_rhs_terms_signs_and_scales(dist):
    """Eq. poisson_mms: b = rho/eps0 - Lap phi^M - rho^M/eps0 with the mean
    removed, rebuilt from independent pieces: the deposited rho (pinned
    above), Lap phi^M = -12 pi^2 phi^M for the product of sines, and rho^M =
    q N f_x from the printed densities; q, eps0 and N away from 1 so that a
    dropped, sign-flipped or misscaled term fails."""
    import ctypes

    q, eps0, N, t = 2.0, 1.5, 1.3, 0.37
    if dist == 0:
        p = W.smallest(n=6, n_particles=6 ** 3 * 20, K=0, q=q, eps0=eps0, n_phys=N)
    else:
        p = W.paper_small(n=6, n_particles=6 ** 3 * 20, K=0, n_sigma=0, q=q, eps0=eps0, n_phys=N)
    o = O.Oracle(p)
    o.sample(t)
    rho, _, _ = o.field()
    n = p["n"]
    b = np.zeros(n ** 3)
    O.lib().orc_rhs(o.h, t, b.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    k, j, i = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    X = np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1) / n
    amp = p["phi_amp"] * math.exp(t / (2 * p["phi_T"]))
    phiM = amp * np.prod(np.sin(2 * math.pi * (X - np.array(p["phi_shift"]))), axis=1)
    if dist == 0:
        fx = np.prod(1 + p["fx_amp"] * np.sin(2 * math.pi * (X - p["fx_speed"] * t)), axis=1)
    else:
        e = math.exp(t / p["t_ref"])
        fx = ((1 + e / 5 * np.sin(2 * math.pi * X[:, 0])) * (1 + 0.2 * np.sin(2 * math.pi * (X[:, 1] - 3 * e / 20)))
              * (1 - e / 6 * np.sin(2 * math.pi * (X[:, 2] + e / 15))))
    ref = rho / eps0 + 12 * math.pi ** 2 * phiM - q * N * fx / eps0
    ref -= ref.mean()
    assert np.abs(b - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("c", [2, 3, 7, 40])
def test_ntc_conserves_momentum_and_energy(c):
    cf = O.make_cfg(W.smallest(dt=0.5))  # large P_max: many collisions per outcome
    for o_ in range(30):
        v0 = _cell_velocities(c, 100 + o_)
        v1, ncoll = O.ntc_cell(cf, 7, 3, o_, v0)
        assert np.allclose(v1.sum(0), v0.sum(0), rtol=0, atol=1e-13 * c)
        assert abs((v1 ** 2).sum() - (v0 ** 2).sum()) < 1e-12 * (v0 ** 2).sum()
        if ncoll == 0:
            assert np.array_equal(v0, v1)


def test_ntc_pair_keeps_relative_speed_and_scatters_isotropically():
    """c = 2: every accepted pair keeps g and rotates g onto a direction n
    uniform on the sphere (Eqs. n, chi_iso). Recover chi, epsilon as in
    Eq. angle_recovery and test their CDFs."""
    cf = O.make_cfg(W.smallest(dt=0.09))  # P_max just below 1: at most one pair
    assert O.pmax(cf) < 1.0
    v0 = np.array([[0.3, -1.0, 0.5], [1.4, 0.2, -0.9]])
    g0 = v0[0] - v0[1]
    cos_chi, eps = [], []
    for o_ in range(8000):
        v1, ncoll = O.ntc_cell(cf, 1, 9, o_, v0)
        if ncoll == 1:
            gp = v1[0] - v1[1]
            assert abs(np.linalg.norm(gp) - np.linalg.norm(g0)) < 1e-14
            cos_chi.append(gp[2] / np.linalg.norm(g0))
            eps.append(np.arctan2(gp[1], gp[0]) % (2 * np.pi))
    assert len(cos_chi) > 200
    assert stats.kstest(np.array(cos_chi), stats.uniform(-1, 2).cdf).pvalue > 1e-4
    assert stats.kstest(np.array(eps), stats.uniform(0, 2 * np.pi).cdf).pvalue > 1e-4


def test_ntc_expectation_brute_force():
    """E_K[Delta v_p] for fixed velocities is sum_{q != p} P_coll(g_pq)
    (v_q - v_p)/2 to first order in P (Eqs. delta_vp, p_coll; Algorithm 1)."""
    c = 6
    p = W.smallest(dt=0.002)
    cf = O.make_cfg(p)
    v0 = _cell_velocities(c, 77)
    K = 60000
    acc = np.zeros((K, c, 3))
    for o_ in range(K):
        v1, _ = O.ntc_cell(cf, 3, 5, o_, v0)
        acc[o_] = v1 - v0
    mean, se = acc.mean(0), acc.std(0) / math.sqrt(K)
    w_dt_dV = (1.0 / cf.np) * cf.dt / (1.0 / cf.n) ** 3
    ref = np.zeros((c, 3))
    for i in range(c):
        for j in range(c):
            if i != j:
                g = np.linalg.norm(v0[i] - v0[j])
                ref[i] += cf.sigma0 * g * w_dt_dV * (v0[j] - v0[i]) / 2
    assert np.all(np.abs(mean - ref) < 4.5 * se + 1e-3 * np.abs(ref).max())


def _repeated_calls(K, dt, sigma0, M, c=48):
    """<Delta v> of M K-averaged calls on one fixed cell state (48 particles
    in one cell of a 2^3 mesh), each call with its own Philox counter."""
    g = np.random.default_rng(5)
    x = g.random((c, 3)) * 0.5
    v = 0.2 + g.standard_normal((c, 3))
    o = O.Oracle(W.smallest(n=2, n_particles=c, K=K, dt=dt, sigma0=sigma0))
    out = np.empty((M, c, 3))
    for s in range(M):
        o.set_state(x, v, 0.0, s)
        out[s], _ = o.collide_avg(0)
    return out


def test_algorithmic_variance_falls_as_one_over_K_and_grows_with_dt():
    """Eq. var, algorithmic term: for a fixed velocity set the K outcomes of
    Eq. avg_outcome are independent, so Var[<Delta v>] = C_alg dt / N_avg
    exactly in K, and linear in dt while collisions per particle are rare.
    Shared outcome streams, a wrong 1/K, or dt missing from (or squared in)
    P_coll,max fail it. Here about 2% (dt ratio) and 1.5% (K ratio) are
    sampling spread, and O(lambda) of the dt ratio is the memory loss of a
    particle that collides twice."""
    var = lambda a: a.var(axis=0, ddof=1).mean()
    v1 = var(_repeated_calls(1, 0.01, 0.5, 2000))
    for K in (4, 16):
        r = K * var(_repeated_calls(K, 0.01, 0.5, 2000)) / v1
        assert 0.92 < r < 1.08, (K, r)
    r = var(_repeated_calls(4, 0.01, 0.2, 4000)) / var(_repeated_calls(4, 0.005, 0.2, 4000))
    assert 1.88 < r < 2.08, r


def test_collisions_off_is_exactly_zero():
    p = W.smallest(K=0)
    o = O.Oracle(p)
    o.sample()
    dv, dvM = o.collide_avg(0)
    assert np.all(dv == 0) and np.all(dvM == 0)


# -------------------------------------------------------------- norms -----
def test_error_norms_hand_computed():
    p = W.smallest(n=4, n_particles=3)
    o = O.Oracle(p)
    o.sample(0.0)
    x, v = o.state()
    xi = o.xi()
    dx = np.array([[0.01, -0.02, 0.0], [0.0, 0.0, 0.03], [-0.5 + 1e-9, 0.0, 0.0]])
    dv = np.array([[1.0, 0.0, 0.0], [0.0, -2.0, 0.0], [0.0, 0.0, 0.5]])
    x2 = (x + dx) % 1.0
    o.set_state(x2, v + dv)
    e = o.errors()
    # minimum-image position errors; the third particle sits half a box away
    ex = np.array([0.01, 0.0, 0.5 - 1e-9])
    assert abs(e[0] - np.sqrt((ex ** 2).mean())) < 1e-12
    assert abs(e[7] - 0.5 + 1e-9) < 1e-12
    assert abs(e[3] - np.sqrt(1.0 / 3.0)) < 1e-14 and e[10] == 1.0
    assert abs(e[4] - np.sqrt(4.0 / 3.0)) < 1e-14 and e[11] == 2.0


def test_wrap_convention():
    assert O.wrap(-1e-18) == 0.0
    assert O.wrap(1.25) == 0.25
    assert O.wrap(-0.25) == 0.75
    assert O.wrap(0.0) == 0.0


# ---------------------------------------------- rates of the paper --------
def test_uncoupled_collisionless_push_is_second_order():
    """q/m = 0, q = 0, no collisions: the particle error comes from the
    velocity-Verlet truncation only and falls as dt^2 (Eq. velocity_verlet,
    Sec. 5.3 uncoupled case)."""
    errs = []
    for dt in (0.1, 0.05, 0.025):
        p = W.smallest(n=4, n_particles=400, K=0, dt=dt, couple_qm_zero=1, couple_q_zero=1)
        o = O.Oracle(p)
        o.sample(0.0)
        o.step(int(round(2.0 / dt)))
        errs.append(o.errors()[7])  # eps_inf of x
    r1, r2 = np.log2(errs[0] / errs[1]), np.log2(errs[1] / errs[2])
    assert 1.8 < r1 < 2.2 and 1.8 < r2 < 2.2, (errs, r1, r2)


def test_collision_error_has_zero_mean():
    """The expected collision error <Delta v> - <Delta v^M> is zero by
    construction (Sec. 4.2.2): averaged over all particles of a sampled
    state it is within a few standard errors of 0."""
    p = W.smallest(n=8, n_particles=8 * 8 * 8 * 30, K=64)
    o = O.Oracle(p)
    o.sample(0.0)
    dv, dvM = o.collide_avg(0)
    e = dv - dvM
    # particles of one cell are correlated: use cell-level means
    cell, count, start, perm = o.sort()
    cm = np.array([e[perm[start[k]:start[k + 1]]].mean(0) for k in range(512) if count[k] > 1])
    mean, se = cm.mean(0), cm.std(0) / math.sqrt(len(cm))
    assert np.all(np.abs(mean) < 4.5 * se)
    assert np.abs(dvM).mean() > 10 * se.max()


def test_one_way_coupled_collisionless_is_second_order():
    """q = 0 (the field does not see the particles), q/m = 1: particles are
    pushed by E - E^M with E the discrete manufactured field, whose error is
    O(h^2); refining h and dt together gives second order (Sec. 5.3)."""
    errs = []
    for n in (8, 16, 32):
        dt = 0.4 / n
        p = W.smallest(n=n, n_particles=300, K=0, dt=dt, couple_q_zero=1)
        o = O.Oracle(p)
        o.sample(0.0)
        o.step(int(round(0.6 / dt)))
        errs.append(o.errors()[10])  # eps_inf of u
    r1, r2 = np.log2(errs[0] / errs[1]), np.log2(errs[1] / errs[2])
    assert 1.7 < r1 < 2.3 and 1.7 < r2 < 2.3, (errs, r1, r2)


def test_step_collision_term_carries_source_with_right_sign():
    """Uncoupled collisional step: the velocity error e_v after one step is
    1/2 (e_coll^A + e_coll^B); with the source subtracted it is uncorrelated
    with the source itself, while dropping the source (or adding it) would
    give a correlation near +1 (or +2) of sum <dv^M>^2 (Eq. velocity_verlet)."""
    p = W.smallest(n=8, n_particles=8 ** 3 * 24, K=64, dt=0.02, couple_qm_zero=1, couple_q_zero=1)
    o = O.Oracle(p)
    o.sample(0.0)
    _, dvM = o.collide_avg(0)
    x0, v0 = o.state()
    o.step(1)
    x1, v1 = o.state()
    e = v1 - v0  # v^M is constant, so this is the error increment
    s = (dvM * dvM).sum()
    corr = (e * dvM).sum() / s
    assert abs(corr) < 0.25, corr
