"""Pins of the oracle's paper-form problem (Sec. 5.2) and odd-power cross
section (Eqs. sigma_ms, vel_change_3, fn) against what the paper and the
mathematics fix, independently of the oracle's own arithmetic:

- f_0, f_1, f_2 for the paper's f_v as printed in Sec. 3.3 (the oracle
  computes them by exact moment expansion, a different route);
- f_k for both velocity densities by tensor-product Gauss-Hermite
  quadrature from numpy (exact for these polynomial integrands);
- the CDF round trips F(F^{-1}(xi)) = xi, the densities integrating to 1
  and to their CDFs (scipy quadrature), the paper's printed f_x, f_v and
  vh(t), and central differences in t for xdot^M and vdot^M;
- the scale-family property v^M(xi, t) / vh(t) = const in t;
- sample moments of the paper's f_v within 4 sigma / sqrt(N);
- (sigma g)_max against a dense brute-force scan, and the Maxwell-molecule
  special case sigma = sigma_0 / g (every candidate accepted);
- the manufactured anisotropy's constants (1/2, 12/29) as the solution of
  the least-squares problem of Sec. 5.1, and the oracle's CDF as the
  integral of that ansatz.
"""
import math

import numpy as np
import pytest
from scipy import integrate

import inputs
from oracle import oracle as O

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")

T_REF = 1.0
VBAR = 0.1


def paper_cfg(**kw):
    p = dict(n=4, n_particles=64, K=0, dt=0.01, dist=O.DIST_PAPER, v_bar=VBAR, t_ref=T_REF)
    p.update(kw)
    return O.make_cfg(p)


def gauss_cfg(**kw):
    p = dict(n=4, n_particles=64, K=0, dt=0.01, v_mean=(0.2, -0.1, 0.35), v_sigma=0.8)
    p.update(kw)
    return O.make_cfg(p)


# ---------------------------------------------------------------- f_x ------
@pytest.mark.parametrize("t", [0.0, 0.37, 1.0])
def test_paper_fx_matches_the_printed_forms(t):
    c = paper_cfg()
    e = math.exp(t / T_REF)
    for x in np.linspace(0.0, 1.0, 17):
        fx = 1 + e / 5 * math.sin(2 * math.pi * x)
        fy = 1 + 1 / 5 * math.sin(2 * math.pi * (x - 3 * e / 20))
        fz = 1 - e / 6 * math.sin(2 * math.pi * (x + e / 15))
        for d, want in enumerate((fx, fy, fz)):
            assert abs(O.fx(c, d, x, t) - want) <= 1e-15 * 4


@pytest.mark.parametrize("t", [0.0, 0.5, 1.0])
def test_paper_Fx_is_the_integral_and_inverts(t):
    c = paper_cfg()
    for d in range(3):
        assert abs(integrate.quad(lambda x: O.fx(c, d, x, t), 0.0, 1.0, epsabs=1e-14)[0] - 1.0) < 1e-13
        for x in (0.1, 0.45, 0.8):
            q = integrate.quad(lambda y: O.fx(c, d, y, t), 0.0, x, epsabs=1e-14)[0]
            assert abs(O.Fx(c, d, x, t) - q) < 1e-13
        for xi in inputs.rng(11).uniform(0, 1, 50):
            xm = O.xM_d(c, d, xi, t)
            assert 0.0 <= xm <= 1.0 and abs(O.Fx(c, d, xm, t) - xi) < 1e-14


def test_paper_xdot_matches_central_differences():
    c = paper_cfg()
    dl = 1e-5
    for d in range(3):
        for xi in inputs.rng(12).uniform(0.02, 0.98, 20):
            for t in (0.1, 0.6):
                fd = (O.xM_d(c, d, xi, t + dl) - O.xM_d(c, d, xi, t - dl)) / (2 * dl)
                assert abs(O.xMdot_d(c, d, O.xM_d(c, d, xi, t), t) - fd) < 1e-8


def test_config_form_axes_agree_with_the_single_axis_functions():
    c = O.make_cfg(dict(n=4, n_particles=64, K=0, dt=0.01))
    for d in range(3):
        for xi in (0.1, 0.5, 0.93):
            assert O.xM_d(c, d, xi, 0.3) == O.xM(c, xi, 0.3)
            xm = O.xM(c, xi, 0.3)
            assert O.xMdot_d(c, d, xm, 0.3) == O.xMdot(c, xm, 0.3)
            assert O.vM_t(c, d, xi, 0.7) == O.vM(c, d, xi)
            assert O.vMdot(c, d, 0.3, 0.7) == 0.0


# ---------------------------------------------------------------- f_v ------
@pytest.mark.parametrize("t", [0.0, 0.25, 0.8])
def test_paper_vhat_and_fv_match_the_printed_forms(t):
    c = paper_cfg()
    vh, dvh = O.vhat(c, t)
    want = VBAR * np.array([1 + math.sin(math.pi * t / (2 * T_REF)) / 5, 1 + math.cos(math.pi * t / T_REF) / 5,
                            1 + math.sin(3 * math.pi * t / (2 * T_REF)) / 5])
    assert np.allclose(vh, want, rtol=1e-15, atol=0)
    dl = 1e-6
    fd = (O.vhat(c, t + dl)[0] - O.vhat(c, t - dl)[0]) / (2 * dl)
    assert np.allclose(dvh, fd, rtol=1e-8, atol=1e-12)
    for d in range(3):
        for v in (-0.3, -0.05, 0.0, 0.02, 0.17):
            z = v / vh[d]
            assert abs(O.fv_paper(c, d, v, t) - 2 / math.sqrt(math.pi) * v * v / vh[d] ** 3 * math.exp(-z * z)) \
                <= 1e-14 * (1 + O.fv_paper(c, d, v, t))
        assert abs(integrate.quad(lambda v: O.fv_paper(c, d, v, t), -np.inf, np.inf)[0] - 1.0) < 1e-12
        for v in (-0.2, -0.01, 0.0, 0.04, 0.3):
            q = integrate.quad(lambda u: O.fv_paper(c, d, u, t), -np.inf, v, epsabs=1e-15)[0]
            assert abs(O.Fv_paper(c, d, v, t) - q) < 1e-12


def test_paper_vM_inverts_and_is_a_scale_family():
    c = paper_cfg()
    xis = np.concatenate([inputs.rng(13).uniform(0, 1, 60), [1e-9, 0.25, 0.5 - 1e-6, 0.5 + 1e-6, 1 - 1e-9]])
    for d in range(3):
        for xi in xis:
            v0 = O.vM_t(c, d, xi, 0.0)
            assert abs(O.Fv_paper(c, d, v0, 0.0) - xi) < 1e-14
            vh0 = O.vhat(c, 0.0)[0][d]
            for t in (0.3, 0.9):
                vt = O.vM_t(c, d, xi, t)
                assert abs(O.Fv_paper(c, d, vt, t) - xi) < 1e-14
                assert abs(vt / O.vhat(c, t)[0][d] - v0 / vh0) <= 1e-12 * max(1.0, abs(v0 / vh0))


def test_paper_vdot_matches_central_differences():
    c = paper_cfg()
    dl = 1e-5
    for d in range(3):
        for xi in inputs.rng(14).uniform(0.01, 0.99, 20):
            for t in (0.15, 0.7):
                fd = (O.vM_t(c, d, xi, t + dl) - O.vM_t(c, d, xi, t - dl)) / (2 * dl)
                assert abs(O.vMdot(c, d, O.vM_t(c, d, xi, t), t) - fd) < 1e-8


def test_paper_sampled_velocity_moments():
    N = 20000
    p = dict(n=4, n_particles=N, K=0, dt=0.01, dist=O.DIST_PAPER, v_bar=VBAR, t_ref=T_REF)
    o = O.Oracle(p)
    o.sample(0.0)
    _, v = o.state()
    vh = O.vhat(o.cfg, 0.0)[0]
    for d in range(3):
        z = v[:, d] / vh[d]
        # E z = 0, E z^2 = 3/2, Var z^2 = E z^4 - 9/4 = 15/4 - 9/4 = 3/2
        assert abs(z.mean()) < 4 * math.sqrt(1.5 / N)
        assert abs((z * z).mean() - 1.5) < 4 * math.sqrt(1.5 / N)


# ---------------------------------------------------------------- f_n ------
def paper_f_printed(k, vp, vh):
    """f_0, f_1, f_2 as printed in Sec. 3.3 for the paper's f_v."""
    vh2 = float(np.sum(vh ** 2))
    vp2 = float(np.sum(vp ** 2))
    out = np.zeros(3)
    for i in range(3):
        if k == 0:
            out[i] = -vp[i]
        elif k == 1:
            out[i] = -0.5 * (3 * vh2 + 6 * vh[i] ** 2 + 2 * vp2) * vp[i]
        else:
            others = np.prod([vh[j] ** 2 for j in range(3) if j != i])
            out[i] = -0.25 * (15 * vh2 ** 2 + 36 * vh[i] ** 4 + 24 * vp2 * vh[i] ** 2 + 4 * vp2 ** 2
                              + 24 * vh[i] ** 2 * vh2 + 12 * vp2 * vh2
                              + 24 * float(np.sum(vh ** 2 * vp ** 2)) - 12 * others) * vp[i]
    return out


@pytest.mark.parametrize("k", [0, 1, 2])
def test_paper_fn_matches_the_printed_formulas(k):
    c = paper_cfg()
    r = inputs.rng(20 + k)
    for _ in range(20):
        t = float(r.uniform(0, 1))
        vp = r.normal(0, 0.15, 3)
        vh = O.vhat(c, t)[0]
        want = paper_f_printed(k, vp, vh)
        got = O.fn(c, k, vp, t)
        assert np.allclose(got, want, rtol=1e-12, atol=1e-16 * VBAR ** (2 * k + 1))


def _gh_expect(nodes_weights, fun):
    z, w = nodes_weights
    acc = 0.0
    for a in range(len(z)):
        for b in range(len(z)):
            for c in range(len(z)):
                acc = acc + w[a][0] * w[b][1] * w[c][2] * fun(np.array([z[a][0], z[b][1], z[c][2]]))
    return acc


@pytest.mark.parametrize("form", ["gauss", "paper"])
@pytest.mark.parametrize("k", [0, 1, 2])
def test_fn_matches_gauss_hermite_quadrature(form, k):
    x, w = np.polynomial.hermite.hermgauss(8)   # weight e^{-x^2}, exact to degree 15
    r = inputs.rng(30 + k)
    c = gauss_cfg() if form == "gauss" else paper_cfg()
    t = 0.42
    if form == "gauss":
        mu, s = np.array(c.vmean[:]), c.vsig
        nodes = [[mu[d] + math.sqrt(2) * s * xx for d in range(3)] for xx in x]
        wts = [[ww / math.sqrt(math.pi)] * 3 for ww in w]
    else:
        vh = O.vhat(c, t)[0]
        nodes = [[vh[d] * xx for d in range(3)] for xx in x]
        wts = [[ww * 2 / math.sqrt(math.pi) * xx * xx] * 3 for xx, ww in zip(x, w)]
    for _ in range(5):
        vp = r.normal(0, 0.3, 3)
        want = _gh_expect((nodes, wts), lambda V: float(np.sum((V - vp) ** 2)) ** k * (V - vp))
        assert np.allclose(O.fn(c, k, vp, t), want, rtol=1e-11, atol=1e-14)


def test_odd_source_combines_fn_with_the_prefactor():
    c = paper_cfg(n=8, n_particles=5000, K=4, dt=0.02, n_sigma=3, sigma_n=(0.7, 0.3, -0.002))
    vp = np.array([0.05, -0.12, 0.02])
    t, cc = 0.3, 11
    w, dV = 1.0 / 5000, (1 / 8) ** 3
    want = w * 0.02 * (cc - 1) / (2 * dV) * sum(s * O.fn(c, k, vp, t) for k, s in enumerate((0.7, 0.3, -0.002)))
    assert np.allclose(O.odd_source(c, vp, cc, t), want, rtol=1e-14, atol=0)


# ------------------------------------------------------------ sigma g ------
@pytest.mark.parametrize("sig", [(1.0, 0.0, 0.0), (0.0, 2.0, 0.0), (1.0, 0.43, -1.4e-3), (2.0, 0.1, 1e-4),
                                 (0.5, -0.001, 0.0)])
def test_sg_max_against_a_dense_scan(sig):
    n_sigma = 3 if sig[2] else (2 if sig[1] else 1)
    c = O.make_cfg(dict(n=4, n_particles=64, K=1, dt=0.01, n_sigma=n_sigma, sigma_n=sig, g_max=17.3))
    g = np.linspace(0.0, 17.3, 200001)
    sg = sum(s * g ** (2 * k) for k, s in enumerate(sig[:n_sigma]))
    assert np.allclose([O.sigma_g(c, x * x) for x in (0.0, 1.3, 9.0)],
                       [sum(s * x ** (2 * k) for k, s in enumerate(sig[:n_sigma])) for x in (0.0, 1.3, 9.0)],
                       rtol=1e-14)
    m = O.sg_max(c)
    assert m >= sg.max() * (1 - 1e-15) and m <= sg.max() * (1 + 1e-8)


def test_maxwell_molecules_accept_every_candidate():
    """n_sigma = 1: sigma(g) g = sigma_0 is constant, so the acceptance ratio
    sigma g / (sigma g)_max is 1 and every candidate collides."""
    p = dict(n=2, n_particles=400, K=8, dt=0.05, n_sigma=1, sigma_n=(30.0, 0.0, 0.0), cg_tol=1e-12)
    o = O.Oracle(p)
    o.sample(0.0)
    o.collide_avg(0)
    st = o.stats()
    assert st["n_cand"] > 100 and st["n_coll"] == st["n_cand"]
    # ratio g^2 / g_max^2 for sigma = sigma_1 g: acceptance well below 1
    q = dict(p, sigma_n=(0.0, 5.0, 0.0), n_sigma=2)
    o = O.Oracle(q)
    o.sample(0.0)
    o.collide_avg(0)
    st = o.stats()
    assert 0 < st["n_coll"] < 0.2 * st["n_cand"]


# ------------------------------------------------- manufactured anisotropy --
def _p_chi(chi, c0, c1):
    """The ansatz of Eq. pchi_ms with the two constraints imposed."""
    c = np.cos(chi)
    return (c0 + c1 * c - 1.5 * (2 * c0 - 1) * c * c - 5 * c1 / 3 * c ** 3) * np.sin(chi)


def test_anisotropy_constants_minimise_the_distance_to_the_soft_sphere_target():
    """Sec. 5.1: with the variable-soft-sphere target p_bar = 2 cos^3(chi/2)
    sin(chi/2) (alpha = 2, Eq. pbar) the least-squares problem of Eq.
    anisotropy_opt is linear in (C0, C1); its solution is the printed (1/2,
    12/29), and the oracle's CDF of the manufactured anisotropy is the
    integral of the ansatz with these constants."""
    pbar = lambda x: 2 * np.cos(x / 2) ** 3 * np.sin(x / 2)
    # p = a0(chi) + C0 a1(chi) + C1 a2(chi)
    c = lambda x: np.cos(x)
    a0 = lambda x: 1.5 * c(x) ** 2 * np.sin(x)
    a1 = lambda x: (1 - 3 * c(x) ** 2) * np.sin(x)
    a2 = lambda x: (c(x) - 5 / 3 * c(x) ** 3) * np.sin(x)
    q = lambda f: integrate.quad(f, 0, np.pi, epsabs=1e-14, epsrel=1e-13)[0]
    M = np.array([[q(lambda x: a1(x) * a1(x)), q(lambda x: a1(x) * a2(x))],
                  [q(lambda x: a2(x) * a1(x)), q(lambda x: a2(x) * a2(x))]])
    rhs = np.array([q(lambda x: (pbar(x) - a0(x)) * a1(x)), q(lambda x: (pbar(x) - a0(x)) * a2(x))])
    c0, c1 = np.linalg.solve(M, rhs)
    assert abs(c0 - 0.5) < 1e-10 and abs(c1 - 12 / 29) < 1e-10, (c0, c1)
    # constraints hold for any constants: unit mass and zero mean cos chi
    for cc0, cc1 in ((0.5, 12 / 29), (0.3, -0.2), (0.9, 1.1)):
        assert abs(q(lambda x: _p_chi(x, cc0, cc1)) - 1.0) < 1e-12
        assert abs(q(lambda x: _p_chi(x, cc0, cc1) * np.cos(x))) < 1e-12
    # the oracle's F(u), u = sin^2(chi/2), is the CDF of the optimal ansatz
    for chi in (0.2, 0.9, 1.7, 2.5, 3.1):
        F = integrate.quad(lambda x: _p_chi(x, 0.5, 12 / 29), 0, chi, epsabs=1e-14)[0]
        assert abs(O.lib().orc_aniso_F(np.sin(chi / 2) ** 2) - F) < 1e-12, chi


# ------------------------------------------------------ norms and push -----
def _paper(**kw):
    from paper_2602_15130_gb300 import workloads as W

    return W.paper_small(**kw)


@pytest.mark.parametrize("t0", [0.0, 0.3])
def test_paper_error_norms_hand_computed(t0):
    """Sec. 4.3 norms on the paper's problem: known offsets from the
    manufactured state at the context time (v^M(t0) = tau vh(t0))."""
    p = _paper(n=4, n_particles=3, K=0)
    o = O.Oracle(p)
    o.sample(t0)
    x, v = o.state()
    dx = np.array([[0.01, -0.02, 0.0], [0.0, 0.0, 0.03], [-0.5 + 1e-9, 0.0, 0.0]])
    dv = np.array([[0.1, 0.0, 0.0], [0.0, -0.2, 0.0], [0.0, 0.0, 0.05]])
    o.set_state((x + dx) % 1.0, v + dv, t0, 0)
    e = o.errors()
    assert abs(e[0] - np.sqrt((np.array([0.01, 0.0, 0.5 - 1e-9]) ** 2).mean())) < 1e-12
    assert abs(e[1] - np.sqrt((np.array([0.02, 0.0, 0.0]) ** 2).mean())) < 1e-12
    assert abs(e[7] - (0.5 - 1e-9)) < 1e-12
    assert abs(e[3] - np.sqrt(0.01 / 3.0)) < 1e-13 and abs(e[10] - 0.1) < 1e-13
    assert abs(e[4] - np.sqrt(0.04 / 3.0)) < 1e-13 and abs(e[11] - 0.2) < 1e-13
    assert abs(e[5] - np.sqrt(0.0025 / 3.0)) < 1e-13 and abs(e[12] - 0.05) < 1e-13


def test_paper_uncoupled_push_is_second_order():
    """q/m = 0, q = 0, no collisions on the paper's problem: the exact
    solution is x^M(t), v^M(t) = tau vh(t), and Eq. velocity_verlet with the
    sources of Eq. eom_mms (vdot^M in both half kicks, the general xdot^M in
    the drift) leaves errors that fall as dt^2. A dropped or sign-flipped
    vdot^M term leaves an O(1) velocity error and fails it."""
    ex, ev = [], []
    for m in (8, 16, 32):
        p = _paper(n=4, n_particles=200, K=0, n_sigma=0, dt=1.0 / m, couple_qm_zero=1, couple_q_zero=1)
        o = O.Oracle(p)
        o.sample(0.0)
        o.step(m)
        e = o.errors()
        ex.append(e[7])
        ev.append(max(e[10], e[11], e[12]))
    for errs in (ex, ev):
        r1, r2 = np.log2(errs[0] / errs[1]), np.log2(errs[1] / errs[2])
        assert 1.8 < r1 < 2.2 and 1.8 < r2 < 2.2, (errs, r1, r2)


@pytest.mark.parametrize("t", [0.0, 0.37])
def test_paper_rhoM_is_the_printed_density_and_integrates_to_qN(t):
    """rho^M = q f_x (Eq. poisson_mms) with the paper's printed per-axis f_x
    at random points, and its integral over the box is q N (scipy)."""
    q, N = 2.5, 3.0
    c = paper_cfg(n_phys=N)
    e = math.exp(t / T_REF)
    for x in inputs.rng(3).random((25, 3)):
        want = q * N * ((1 + e / 5 * math.sin(2 * math.pi * x[0]))
                        * (1 + 1 / 5 * math.sin(2 * math.pi * (x[1] - 3 * e / 20)))
                        * (1 - e / 6 * math.sin(2 * math.pi * (x[2] + e / 15))))
        assert abs(O.rhoM(c, q, x, t) - want) <= 1e-14 * abs(want)
    total, _ = integrate.tplquad(lambda z, y, x: O.rhoM(c, q, np.array([x, y, z]), t), 0, 1, 0, 1, 0, 1,
                                 epsabs=1e-9, epsrel=1e-9)
    assert abs(total - q * N) < 1e-7
