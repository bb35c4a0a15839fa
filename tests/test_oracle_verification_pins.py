"""Pins of the oracle's verification switches (Sec. 5.4) and of the
scattering-angle CDF metrics (Sec. 4.4).

Each switch is checked against what it must do by construction: the
isolated-collision drift reproduces the manufactured positions exactly when
nothing else acts; Error 1 shifts every post-collision velocity by -v_q and
changes the expected outcome; Error 2 conserves momentum and energy and keeps
the expected outcome, and only the manufactured anisotropy lets the angle
metric see it; the angle metric is the one-sample Kolmogorov-Smirnov
statistic up to 1/N.
"""
import math

import numpy as np
import pytest
from scipy import stats

import inputs
from oracle import oracle as O
from paper_2602_15130_gb300 import workloads as W


def _cell_velocities(c, seed):
    return 0.2 + np.random.default_rng(seed).standard_normal((c, 3))


def _min_image(d):
    return d - np.floor(d + 0.5)


# ------------------------------------------------------ isolated collisions --
def test_isolated_mode_collisionless_reproduces_manufactured_solution():
    """q/m = 0, K = 0, isolated drift: x^n = x^M(t_n) up to rounding and v
    never changes, whereas the plain drift carries the O(dt^2) midpoint-rule
    error of the manufactured velocity."""
    base = W.smallest(K=0, couple_qm_zero=1)
    o = O.Oracle(dict(base, verify=O.ISOLATE))
    o.sample()
    o.step(10)
    e = o.errors()
    assert e[7:10].max() < 1e-13        # eps_inf of x, y, z
    assert e[10:13].max() == 0.0        # velocities untouched
    plain = O.Oracle(base)
    plain.sample()
    plain.step(10)
    assert plain.errors()[7:10].max() > 1e-10


def test_isolated_mode_position_error_is_dt_times_velocity_error():
    """With collisions and q/m = 0, one isolated step moves x - x^M by
    exactly dt (v^{n+1/2} - v^M), v^{n+1/2} = v^M + (<dv> - <dv^M>)/2 from
    the step's first collision call."""
    p = dict(W.smallest(couple_qm_zero=1), verify=O.ISOLATE)
    o = O.Oracle(p)
    o.sample()
    x0, v0 = o.state()
    dvA, dvMA = o.collide_avg(0)
    vh = v0 + 0.5 * (dvA - dvMA)
    o.step(1)
    x1, _ = o.state()
    cf = O.make_cfg(p)
    xi = o.xi()
    t1 = p["dt"]
    xm1 = np.array([[O.xM(cf, xi[i, d], t1) for d in range(3)] for i in range(p["n_particles"])])
    err = _min_image(x1 - xm1)
    want = p["dt"] * (vh - v0)
    assert np.abs(want).max() > 1e-6    # collisions did move something
    assert np.abs(err - want).max() < 1e-14


# ----------------------------------------------------------------- Error 1 --
def test_error1_shifts_post_collision_velocities_by_minus_vq():
    """v_cm = (v_p - v_q)/2 instead of (v_p + v_q)/2 moves both post-collision
    velocities by -v_q, with the same draws."""
    ok = O.make_cfg(W.smallest(dt=0.09))
    bad = O.make_cfg(dict(W.smallest(dt=0.09), verify=O.ERROR1))
    v0 = np.array([[0.3, -1.0, 0.5], [1.4, 0.2, -0.9]])
    seen = 0
    for o_ in range(3000):
        v_ok, n_ok = O.ntc_cell(ok, 1, 9, o_, v0)
        v_bad, n_bad = O.ntc_cell(bad, 1, 9, o_, v0)
        assert n_ok == n_bad
        if n_ok == 1:
            d = v_bad - v_ok
            assert np.allclose(d[0], d[1], atol=1e-15)
            assert np.allclose(d[0], -v0[0], atol=1e-15) or np.allclose(d[0], -v0[1], atol=1e-15)
            seen += 1
        else:
            assert np.array_equal(v_bad, v_ok)
    assert seen > 50


def test_error1_changes_expected_outcome():
    """With Error 1 the pair {i, j} moves v_i by -(v_i + v_j)/2 as p and by
    (v_j - 3 v_i)/2 as q, on average -v_i: E_K[dv_i] = sum_j P_coll(g_ij)
    (-v_i) to first order, not sum_j P_coll(g_ij) (v_j - v_i)/2."""
    c = 6
    p = dict(W.smallest(dt=0.002), verify=O.ERROR1)
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
    right = np.zeros((c, 3))
    for i in range(c):
        for j in range(c):
            if i != j:
                P = cf.sigma0 * np.linalg.norm(v0[i] - v0[j]) * w_dt_dV
                ref[i] += P * (-v0[i])
                right[i] += P * (v0[j] - v0[i]) / 2
    assert np.all(np.abs(mean - ref) < 4.5 * se + 1e-3 * np.abs(ref).max())
    assert np.abs(mean - right).max() > 10 * se.max()


# ----------------------------------------------------------------- Error 2 --
@pytest.mark.parametrize("c", [2, 5, 40])
def test_error2_conserves_momentum_and_energy(c):
    cf = O.make_cfg(dict(W.smallest(dt=0.5), verify=O.ERROR2))
    for o_ in range(30):
        v0 = _cell_velocities(c, 300 + o_)
        v1, ncoll = O.ntc_cell(cf, 7, 3, o_, v0)
        assert np.allclose(v1.sum(0), v0.sum(0), rtol=0, atol=1e-13 * c)
        assert abs((v1 ** 2).sum() - (v0 ** 2).sum()) < 1e-12 * (v0 ** 2).sum()
        # a swap only permutes the rows
        assert np.array_equal(np.sort(v1, axis=0), np.sort(v0, axis=0))


def test_error2_keeps_expected_outcome():
    """beta = 1/2: E[dv_p] = (v_q - v_p)/2 per collision, the same as Eq. J2."""
    c = 6
    p = dict(W.smallest(dt=0.002), verify=O.ERROR2)
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


# ------------------------------------------------------------ angle metric --
def test_angle_metric_hand_computed():
    F = lambda a: np.asarray(a)  # noqa: E731
    assert O.angle_cdf_errors(np.array([0.25, 0.75]), F) == (0.25, 0.25)
    # ties: theta(0) = 1, so both samples see F_emp = 1
    e2, einf = O.angle_cdf_errors(np.array([0.5, 0.5]), F)
    assert e2 == 0.5 and einf == 0.5
    e2, einf = O.angle_cdf_errors(np.array([0.1, 0.2, 0.9]), F)
    e = np.array([1 / 3 - 0.1, 2 / 3 - 0.2, 1.0 - 0.9])
    assert abs(e2 - math.sqrt(np.mean(e * e))) < 1e-15 and abs(einf - e.max()) < 1e-15


@pytest.mark.parametrize("N", [10, 137, 5000])
def test_angle_metric_is_ks_statistic_within_one_over_n(N):
    """max_r |i/N - F(x_(i))| lies in [D - 1/N, D] for the one-sample KS
    statistic D = max_i max(i/N - F, F - (i-1)/N)."""
    u = inputs.rng(500 + N).random(N)
    _, einf = O.angle_cdf_errors(u, lambda a: np.asarray(a))
    D = stats.kstest(u, "uniform").statistic
    assert D - 1.0 / N - 1e-15 <= einf <= D + 1e-15


def _run_with_angles(verify, steps=3):
    p = dict(W.smallest(), verify=O.ANGLES | verify)
    o = O.Oracle(p)
    o.sample()
    o.step(steps)
    ang = o.angles()
    assert len(ang) == o.stats()["n_coll"]
    return ang


def test_recorded_angles_follow_isotropic_cdfs():
    """Reference algorithm and Error 1: both angle errors are O(N^-1/2) (the
    KS statistic of N samples is about 0.87/sqrt(N) and below 1.63/sqrt(N)
    with probability 0.99)."""
    for verify in (0, O.ERROR1):
        ang = _run_with_angles(verify)
        N = len(ang)
        assert N > 5000
        for a, F in ((ang[:, 0], O.F_chi_iso), (ang[:, 1], O.F_eps)):
            e2, einf = O.angle_cdf_errors(a, F)
            assert 0.2 < einf * math.sqrt(N) < 2.0
            assert e2 < einf


def test_error2_angles_isotropic_kernel_cannot_tell():
    """Error 2 leaves g' = +-g. For Gaussian velocities the direction of g is
    already uniform on the sphere, so with the isotropic kernel the recovered
    lab-frame angles follow the isotropic CDFs and the metric stays
    O(N^-1/2): the coding error is invisible here."""
    ang = _run_with_angles(O.ERROR2)
    N = len(ang)
    assert N > 5000
    _, einf = O.angle_cdf_errors(ang[:, 0], O.F_chi_iso)
    assert einf * math.sqrt(N) < 2.0


def _run_aniso(verify, steps=3):
    return _run_with_angles(O.ANISO | verify, steps)


def test_aniso_cdf_and_inverse():
    """u = sin^2(chi/2): F(u) is the integral of p_chi, increasing, F(0) = 0,
    F(1) = 1; its inverse is exact to rounding; the mean of cos chi is zero
    (Eq. int_np vanishes, so Eq. J2 and the hard-sphere source still hold);
    and the paper's closed-form quartic root agrees with the bisection."""
    L = O.lib()
    from scipy import integrate
    p = lambda c: (29 / 2 + 12 * np.cos(c) - 20 * np.cos(c) ** 3) * np.sin(c) / 29  # noqa: E731
    for chi in (0.0, 0.3, 1.2, 2.0, np.pi):
        val, _ = integrate.quad(p, 0, chi, epsabs=1e-14)
        assert abs(L.orc_aniso_F(math.sin(chi / 2) ** 2) - val) < 1e-12
        assert abs(float(O.F_chi_aniso(chi)) - val) < 1e-12
    m1, _ = integrate.quad(lambda c: p(c) * np.cos(c), 0, np.pi, epsabs=1e-14)
    assert abs(m1) < 1e-13
    for xi in np.linspace(0, 1, 101):
        u = L.orc_aniso_u(xi)
        assert 0.0 <= u <= 1.0 and abs(L.orc_aniso_F(u) - xi) < 2e-15
        # closed form of Sec. 5.1 (a, b of the quartic's resolvent)
        a = (81909 - 83520 * xi + math.sqrt(298924665 + 55680 * xi * (376377 + 2320 * xi * (-429 + 290 * xi))))
        a = a ** (1 / 3) / (40 * 3 ** (2 / 3))
        b = 0.2 + a + (161 - 290 * xi) / (600 * a)
        uc = 0.5 * (1 - math.sqrt(b) + math.sqrt(0.6 - b + 29 / (40 * math.sqrt(b))))
        assert abs(uc - u) < 1e-13


def test_aniso_pairs_conserve_and_keep_expected_outcome():
    cf = O.make_cfg(dict(W.smallest(dt=0.5), verify=O.ANISO))
    for o_ in range(20):
        v0 = _cell_velocities(7, 900 + o_)
        v1, _ = O.ntc_cell(cf, 7, 3, o_, v0)
        assert np.allclose(v1.sum(0), v0.sum(0), rtol=0, atol=1e-12)
        assert abs((v1 ** 2).sum() - (v0 ** 2).sum()) < 1e-12 * (v0 ** 2).sum()
    c = 6
    cf = O.make_cfg(dict(W.smallest(dt=0.002), verify=O.ANISO))
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
                ref[i] += cf.sigma0 * np.linalg.norm(v0[i] - v0[j]) * w_dt_dV * (v0[j] - v0[i]) / 2
    assert np.all(np.abs(mean - ref) < 4.5 * se + 1e-3 * np.abs(ref).max())


def test_aniso_angles_converge_and_error2_does_not():
    """Manufactured anisotropy: the reference algorithm's chi follows
    F_chi_aniso at O(N^-1/2); with Error 2 the recovered chi is isotropic,
    so eps_inf stalls near max |F_aniso - F_iso| = 2/58 (at chi = pi/2)."""
    ang = _run_aniso(0)
    N = len(ang)
    assert N > 5000
    _, einf = O.angle_cdf_errors(ang[:, 0], O.F_chi_aniso)
    assert einf * math.sqrt(N) < 2.0
    _, einf_iso = O.angle_cdf_errors(ang[:, 0], O.F_chi_iso)
    assert einf_iso > 0.02
    ang2 = _run_aniso(O.ERROR2)
    _, einf2 = O.angle_cdf_errors(ang2[:, 0], O.F_chi_aniso)
    assert 0.025 < einf2 < 0.045
    _, e_eps = O.angle_cdf_errors(ang2[:, 1], O.F_eps)
    assert e_eps * math.sqrt(len(ang2)) < 2.0


# --------------------------------------------------------------- objective --
def test_objective_is_field_energy_plus_velocity_error():
    """J_field = (eps0/2) h^3 sum |E|^2 over the nodes and J_vel = sum of the
    squared eps_2 of u, v, w (Sec. 4.3 norms), after a few steps with an
    applied field."""
    p = dict(W.smallest(), E_app=(0.1, -0.2, 0.05))
    o = O.Oracle(p)
    o.sample()
    o.step(3)
    J = o.objective()
    _, _, E = o.field()
    h = 1.0 / p["n"]
    assert abs(J[1] - 0.5 * h ** 3 * (E ** 2).sum()) <= 1e-14 * J[1]
    e = o.errors()
    assert abs(J[2] - (e[3:6] ** 2).sum()) <= 1e-12 * J[2]
    assert J[0] == J[1] + J[2]


def test_applied_field_enters_the_push():
    """With q/m = 1 a uniform E_app changes every velocity after one step
    by dt E_app (two half kicks); the shifted drift moves x by dt^2 E_app/2,
    which changes the gathered fields at second order only."""
    base = W.smallest(K=0, couple_q_zero=1)
    a, b = O.Oracle(base), O.Oracle(dict(base, E_app=(0.3, 0.0, -0.1)))
    for o in (a, b):
        o.sample()
        o.step(1)
    _, va = a.state()
    _, vb = b.state()
    shift = np.array([0.3, 0.0, -0.1]) * base["dt"]
    assert np.abs(vb - va - shift).max() < 1e-6 < np.abs(shift).max()
