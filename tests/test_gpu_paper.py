"""The paper's own manufactured problem (Sec. 5.2: per-axis f_x with
time-varying amplitude and phase, the non-Maxwellian f_v of Eq. fv with
vh(t), and the vdot^M terms it brings into Eq. velocity_verlet) and the
odd-power cross section (Eq. sigma_ms, source of Eqs. vel_change_3 and fn)
on the GPU, through the C ABI, against the FP64 oracle: positions and
velocities within 1e-10, candidate and collision counts equal, error norms
within 1e-10; then the observed convergence of the paper's problem on the
first levels of Table 1 (Sec. 5.3), where Sec. 4 predicts second order.
"""
import numpy as np
import pytest

import pairlists
from oracle import oracle as O
from paper_2602_15130_gb300 import Pic, workloads
from paper_2602_15130_gb300 import _lib
from paper_2602_15130_gb300 import convergence as C

pytestmark = pytest.mark.gpu

TOL = 1e-10
ANG, ANI, E2 = _lib.PIC_VERIFY_ANGLES, _lib.PIC_VERIFY_ANISO, _lib.PIC_VERIFY_ERROR2


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch

    import __graft_entry__ as g

    g.build()
    assert torch.cuda.is_available()
    yield


def dpos(a, b):
    d = np.abs(a - b)
    return np.minimum(d, 1.0 - d)


CASES = {
    "paper": workloads.paper_small(),
    "paper_collisionless": workloads.paper_small(K=0, n_sigma=0),
    "paper_aniso_error2": workloads.paper_small(verify=ANI | E2 | ANG),
    "gauss_odd_sigma": dict(workloads.smallest(cg_tol=1e-13, steps=4), n_sigma=3, sigma_n=(1.0, 0.25, -0.0005)),
    "gauss_maxwell": dict(workloads.smallest(cg_tol=1e-13, steps=4), n_sigma=1, sigma_n=(6.0, 0.0, 0.0)),
}


@pytest.mark.parametrize("name", list(CASES))
def test_sample_matches_oracle(name):
    p = CASES[name]
    g, o = Pic(p), O.Oracle(p)
    for t0 in (0.0, 0.3):
        g.sample_mms(t0)
        o.sample(t0)
        x, v = g.get_state()
        xo, vo = o.state()
        assert dpos(x, xo).max() <= 1e-12
        assert np.abs(v - vo).max() <= 1e-12 * max(1.0, np.abs(vo).max())
        eg, eo = g.mms_error()["array"], o.errors()
        assert np.all(np.abs(eg - eo) <= TOL * np.abs(eo).max())


@pytest.mark.parametrize("name", list(CASES))
def test_steps_match_oracle(name):
    p = CASES[name]
    g, o = Pic(p), O.Oracle(p)
    g.sample_mms(0.0)
    o.sample(0.0)
    g.step(4)
    o.step(4)
    x, v = g.get_state()
    xo, vo = o.state()
    assert dpos(x, xo).max() <= TOL
    assert np.abs(v - vo).max() <= TOL * max(1.0, np.abs(vo).max())
    sg, so = g.stats(), o.stats()
    assert sg["n_coll"] == so["n_coll"] and sg["n_cand"] == so["n_cand"]
    if p["K"] > 0:
        assert so["n_coll"] > 0
    eg, eo = g.mms_error()["array"], o.errors()
    assert np.all(np.abs(eg - eo) <= TOL * np.abs(eo).max())


@pytest.mark.parametrize("name", ["paper", "gauss_odd_sigma", "gauss_maxwell"])
def test_collision_call_matches_oracle(name):
    """One K-averaged call on a stepped state: <dv> and the analytic source
    <dv^M> (the f_k closed forms against the oracle's moment expansion)."""
    p = CASES[name]
    g, o = Pic(p), O.Oracle(p)
    g.sample_mms(0.0)
    o.sample(0.0)
    g.step(1)
    o.step(1)
    g.set_decision_log(2, 1 << 20)
    o.set_pair_log(True)
    dv, dvm = g.collide_avg(1)
    dvo, dvmo = o.collide_avg(1)
    lg, lo = pairlists.canonical(g.decision_log()), pairlists.canonical(o.pair_log())
    assert len(lo) > 0 and lg.shape == lo.shape and np.array_equal(lg, lo)
    assert np.abs(dv - dvo).max() <= TOL * max(1e-3, np.abs(dvo).max())
    assert np.abs(dvm - dvmo).max() <= TOL * np.abs(dvmo).max()
    assert np.abs(dvmo).max() > 0.0


def test_maxwell_molecules_accept_every_candidate():
    g = Pic(CASES["gauss_maxwell"])
    g.sample_mms(0.0)
    g.step(2)
    st = g.stats()
    assert st["n_cand"] > 1000 and st["n_coll"] == st["n_cand"]


@pytest.mark.parametrize("name", ["paper", "gauss_odd_sigma"])
def test_precision_form_tracks_oracle(name):
    """Precision form (FP32 state, per-axis x^M solve and f_k source in
    FP32): sampled within FP32 rounding of the oracle; then, with the oracle
    started from the precision form's own state, every particle that no
    flagged FP32 decision (nor an FP32 position across a cell face) can
    have reached agrees after 4 steps, and the error norms within 3%."""
    p = workloads.mixed(CASES[name])
    g, o = Pic(p), O.Oracle(dict(p, cg_tol=1e-12))
    g.sample_mms(0.0)
    o.sample(0.0)
    x, v = g.get_state()
    xo, vo = o.state()
    assert dpos(x, xo).max() <= 1e-6 and np.abs(v - vo).max() <= 1e-6 * np.abs(vo).max()
    o.set_state(x, v, 0.0, 0)
    for a, b in zip(g.get_sort(), o.sort()):
        assert np.array_equal(a, b)
    g.set_decision_log(1, 1 << 16)
    reached = pairlists.step_tracking_flags(g, o, 4)
    x, v = g.get_state()
    xo, vo = o.state()
    far = (dpos(x, xo) > 1e-5).any(axis=1) | (np.abs(v - vo) > 1e-4 * np.abs(vo).max()).any(axis=1)
    assert not (far & ~reached).any(), (np.flatnonzero(far & ~reached)[:10], reached.mean())
    assert reached.mean() <= 0.05, reached.mean()
    eg, eo = g.mms_error()["array"], o.errors()
    assert np.all(np.abs(eg - eo) <= 0.03 * eo + 1e-7), (eg, eo)


def test_precision_form_keeps_the_error_floor():
    """On the paper's problem (Table 1 levels 0-2) the precision form's
    error norms equal the FP64 form's within 3%: FP32 does not raise the
    error floor."""
    r32 = C.run_study("paper-collisional", [0, 1, 2], "mixed", ["coupled"], log=lambda s: None)
    r64 = C.run_study("paper-collisional", [0, 1, 2], "fp64", ["coupled"], log=lambda s: None)
    for key in ("x_eps2", "v_eps2", "phi_eps2"):
        e32 = r32["variants"]["coupled"]["rates"][key]["errors"]
        e64 = r64["variants"]["coupled"]["rates"][key]["errors"]
        assert all(abs(a - b) <= 0.03 * b for a, b in zip(e32, e64)), (key, e32, e64)


def test_paper_problem_rejected_by_other_forms():
    with pytest.raises(_lib.PicError) as ei:
        Pic(dict(workloads.paper_small(), n_sigma=0))
    assert ei.value.status == _lib.PIC_EINVAL
    g = Pic(workloads.paper_small())
    with pytest.raises(_lib.PicError) as ei:
        g.adjoint_gradient(2, 1, (0.1, 0.1, 0.1))
    assert ei.value.status == _lib.PIC_EINVAL


def _rates(res, variant, key):
    return res["variants"][variant]["rates"][key]["pairwise"]


# eps_2 carries the predicted rates; eps_inf, a maximum over particles, is
# checked through the full studies (python -m paper_2602_15130_gb300.convergence)
def test_paper_problem_collisionless_second_order():
    res = C.run_study("paper-collisionless", [0, 1, 2], "fp64", ["coupled"], log=lambda s: None)
    for key in ("x_eps2", "v_eps2", "phi_eps2"):
        r = _rates(res, "coupled", key)
        assert all(1.6 <= q <= 2.5 for q in r), (key, r)


def test_paper_problem_collisional_second_order():
    """Collision error accumulates between the worst case 2 and the random
    walk 2.5 (Sec. 4.2)."""
    res = C.run_study("paper-collisional", [0, 1, 2], "fp64", ["uncoupled", "coupled"], log=lambda s: None)
    for v in ("uncoupled", "coupled"):
        for key in ("x_eps2", "v_eps2"):
            r = _rates(res, v, key)
            assert all(1.6 <= q <= 2.9 for q in r), (v, key, r)
