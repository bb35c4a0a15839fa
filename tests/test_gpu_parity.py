"""CUDA path vs the FP64 CPU oracle, element by element, through the C ABI.

Bars: cell indices, sort permutations, counts and pair decisions bit-exact
(collision counts equal); FP64 positions, velocities, charge, potential and
field within 1e-10 relative (to the array's magnitude); near-tie accept
decisions (|U - ratio| < 1e-12) are the only allowed differences and are
counted.
"""
import numpy as np
import pytest

import inputs
import pairlists
from oracle import oracle as O
from paper_2602_15130_gb300 import Pic, workloads

pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch

    import __graft_entry__ as g

    g.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    yield


def close(a, b, tol=TOL, scale=None):
    a, b = np.asarray(a), np.asarray(b)
    s = scale if scale is not None else max(1.0, np.abs(b).max() if b.size else 1.0)
    err = np.abs(a - b).max() / s if a.size else 0.0
    return err <= tol, err


def pos_close(a, b, tol=TOL):
    d = np.abs(np.asarray(a) - np.asarray(b))
    d = np.minimum(d, 1.0 - d)
    return d.max() <= tol, d.max()


def pair(p, **kw):
    q = dict(p)
    q.update(kw)
    return Pic(q), O.Oracle(q)


CASES = {
    "smallest": workloads.smallest(cg_tol=1e-13),
    "ragged": workloads.smallest(n=12, n_particles=12 ** 3 * 9 + 37, cg_tol=1e-13),
    "n2": workloads.smallest(n=2, n_particles=300, cg_tol=1e-13),
    "k40": workloads.smallest(n=6, n_particles=6 ** 3 * 12 + 5, K=40, cg_tol=1e-13),
    "k5": workloads.smallest(n=8, n_particles=4096, K=5, cg_tol=1e-13),
}


@pytest.mark.parametrize("name", list(CASES))
def test_sampling_matches_oracle(name):
    p = CASES[name]
    g, o = pair(p)
    g.sample_mms(0.3)
    o.sample(0.3)
    x, v = g.get_state()
    xo, vo = o.state()
    ok, e = pos_close(x, xo)
    assert ok, e
    ok, e = close(v, vo)
    assert ok, e


@pytest.mark.parametrize("name", list(CASES))
def test_sort_bit_exact(name):
    p = CASES[name]
    g, o = pair(p)
    g.sample_mms(0.0)
    o.sample(0.0)
    for a, b in zip(g.get_sort(), o.sort()):
        assert np.array_equal(a, b)


def test_sort_crowded_cells_and_empty_cells():
    p = workloads.smallest(n=8, n_particles=3000, cg_tol=1e-13)
    g, o = pair(p)
    x, v = inputs.particles(3000, seed=3, clustered_cells=5, n=8)  # ~600 per cell, most cells empty
    g.set_state(x, v)
    o.set_state(x, v)
    for a, b in zip(g.get_sort(), o.sort()):
        assert np.array_equal(a, b)
    rho, phi, E = g.get_field()
    ro, po, Eo = o.field()
    assert close(rho, ro)[0] and close(phi, po)[0] and close(E, Eo)[0]


@pytest.mark.parametrize("npart,clustered", [(4 * 4 * 4 * 260, 0), (20000, 1), (26000, 3)])
def test_sort_big_cells(npart, clustered):
    """Mean occupancy >= 128 switches on the block sort for cells of 257 to
    16384 particles; smaller and larger cells stay on the warp pass."""
    p = workloads.smallest(n=4, n_particles=npart, cg_tol=1e-13)
    g, o = pair(p)
    x, v = inputs.particles(npart, seed=11 + clustered, clustered_cells=clustered, n=4)
    g.set_state(x, v)
    o.set_state(x, v)
    srt = o.sort()
    counts = srt[1]
    if clustered == 0:
        assert ((counts > 256) & (counts <= 16384)).any() and (counts <= 256).any()
    else:
        assert (counts > 16384).any() or ((counts > 256) & (counts <= 16384)).any()
    for a, b in zip(g.get_sort(), srt):
        assert np.array_equal(a, b)
    xg, vg = g.get_state()
    xo, vo = o.state()
    assert pos_close(xg, xo)[0] and close(vg, vo)[0]
    rho, phi, E = g.get_field()
    ro, po, Eo = o.field()
    assert close(rho, ro, scale=np.abs(ro).max())[0] and close(phi, po, scale=np.abs(po).max())[0]


@pytest.mark.parametrize("name", list(CASES))
def test_field_matches_oracle(name):
    p = CASES[name]
    g, o = pair(p)
    g.sample_mms(0.1)
    o.sample(0.1)
    rho, phi, E = g.get_field()
    ro, po, Eo = o.field()
    for a, b in ((rho, ro), (phi, po), (E, Eo)):
        ok, e = close(a, b, scale=max(np.abs(b).max(), 1e-300))
        assert ok, e


@pytest.mark.parametrize("name", ["smallest", "ragged", "k40", "k5"])
@pytest.mark.parametrize("phase", [0, 1])
def test_collisions_match_oracle(name, phase):
    p = CASES[name]
    g, o = pair(p)
    g.sample_mms(0.0)
    o.sample(0.0)
    g.reset_stats()
    o.reset_stats()
    dv, dvm = g.collide_avg(phase)
    dvo, dvmo = o.collide_avg(phase)
    sg, so = g.stats(), o.stats()
    assert sg["n_cand"] == so["n_cand"] and sg["n_cand"] > 0
    assert sg["n_near_ties"] == so["n_near_ties"] == 0
    assert sg["n_coll"] == so["n_coll"] and sg["n_coll"] > 0
    ok, e = close(dv, dvo, scale=1.0)
    assert ok, e
    ok, e = close(dvm, dvmo, scale=1.0)
    assert ok, e


@pytest.mark.parametrize("name", ["smallest", "ragged", "k40", "k5", "n2"])
@pytest.mark.parametrize("phase", [0, 1])
def test_pair_lists_bit_exact(name, phase):
    """Algorithm 1's pair list of one K-averaged call, record by record:
    N_pairs of every (cell, outcome), then (p, q, accepted) of every
    candidate slot, equal to the oracle's (near ties: none here)."""
    p = CASES[name]
    g, o = pair(p)
    g.sample_mms(0.0)
    o.sample(0.0)
    g.set_decision_log(2, 1 << 20)
    o.set_pair_log(True)
    g.collide_avg(phase)
    o.collide_avg(phase)
    lg, lo = pairlists.canonical(g.decision_log()), pairlists.canonical(o.pair_log())
    assert len(lo) > 0 and (lo[:, 3] >= 0).any()
    assert lg.shape == lo.shape and np.array_equal(lg, lo)


def test_pair_lists_bit_exact_over_steps_and_crowded_cells():
    """The same over two whole steps (both calls of each, counter word
    2 step + phase) from a state with about 300 particles in each of ten
    cells and a large dt (long in-place chains of collisions). A third step
    is not taken: this state runs away (velocities of 1e13 by then), and
    after that the last-bit differences of the field solve decide cells."""
    p = workloads.smallest(n=8, n_particles=3000, K=12, dt=0.05, cg_tol=1e-12)
    g, o = pair(p)
    x, v = inputs.particles(3000, seed=9, clustered_cells=10, n=8)
    g.set_state(x, v)
    o.set_state(x, v)
    g.set_decision_log(2, 1 << 23)
    o.set_pair_log(True)
    g.step(2)
    o.step(2)
    lg, lo = pairlists.canonical(g.decision_log()), pairlists.canonical(o.pair_log())
    assert sorted(set(lo[:, 0])) == list(range(4))
    assert (lo[lo[:, 3] >= 0, 6] == 1).sum() > 1000
    assert lg.shape == lo.shape and np.array_equal(lg, lo)


def test_collisions_crowded_cells_large_dt():
    # ~300 particles in each of 10 cells, P_max large: long in-place chains
    p = workloads.smallest(n=8, n_particles=3000, K=24, dt=0.05, cg_tol=1e-12)
    g, o = pair(p)
    x, v = inputs.particles(3000, seed=9, clustered_cells=10, n=8)
    g.set_state(x, v)
    o.set_state(x, v)
    dv, dvm = g.collide_avg(0)
    dvo, dvmo = o.collide_avg(0)
    st = g.stats()
    assert st["n_coll"] == o.stats()["n_coll"] > 1000
    assert close(dv, dvo, scale=1.0)[0] and close(dvm, dvmo, scale=1.0)[0]


def test_capacity_error_is_reported():
    p = workloads.smallest(n=4, n_particles=800, max_ppc=64, cg_tol=1e-12)
    g = Pic(p)
    x, v = inputs.particles(800, seed=1, clustered_cells=2, n=4)
    g.set_state(x, v)
    from paper_2602_15130_gb300._lib import PIC_ECAPACITY, PicError
    with pytest.raises(PicError) as ei:
        g.collide_avg(0)
    assert ei.value.status == PIC_ECAPACITY


@pytest.mark.parametrize("name", ["smallest", "ragged", "k40", "n2"])
def test_whole_steps_match_oracle(name):
    p = CASES[name]
    g, o = pair(p)
    g.sample_mms(0.0)
    o.sample(0.0)
    nsteps = 10 if name == "smallest" else 4
    g.step(nsteps)
    o.step(nsteps)
    x, v = g.get_state()
    xo, vo = o.state()
    ok, e = pos_close(x, xo)
    assert ok, e
    ok, e = close(v, vo)
    assert ok, e
    sg, so = g.stats(), o.stats()
    assert sg["n_coll"] == so["n_coll"] and sg["n_cand"] == so["n_cand"]
    assert sg["n_near_ties"] == 0
    rho, phi, E = g.get_field()
    ro, po, Eo = o.field()
    assert close(phi, po, scale=np.abs(po).max())[0]
    eg = g.mms_error()["array"]
    eo = o.errors()
    ok, e = close(eg, eo, scale=np.abs(eo).max())
    assert ok, (e, eg, eo)


@pytest.mark.parametrize("flags", [dict(K=0), dict(couple_qm_zero=1), dict(couple_q_zero=1),
                                   dict(couple_qm_zero=1, couple_q_zero=1, K=0)])
def test_coupling_modes_match_oracle(flags):
    p = workloads.smallest(n=8, n_particles=2000, cg_tol=1e-13, **flags)
    g, o = pair(p)
    g.sample_mms(0.0)
    o.sample(0.0)
    g.step(3)
    o.step(3)
    x, v = g.get_state()
    xo, vo = o.state()
    assert pos_close(x, xo)[0] and close(v, vo)[0]
    assert close(g.mms_error()["array"], o.errors(), scale=np.abs(o.errors()).max())[0]


def test_set_state_from_device_tensors_and_host_arrays_agree():
    import torch

    p = CASES["smallest"]
    x, v = inputs.particles(p["n_particles"], seed=12)
    g1 = Pic(p)
    g1.set_state(x, v, t0=0.0, step=2)
    g2 = Pic(p)
    g2.set_state(torch.tensor(x, device="cuda"), torch.tensor(v, device="cuda"), t0=0.0, step=2)
    xo = torch.zeros((p["n_particles"], 3), dtype=torch.float64, device="cuda")
    vo = torch.zeros_like(xo)
    g2.get_state((xo, vo))
    assert np.array_equal(xo.cpu().numpy(), x) and np.array_equal(vo.cpu().numpy(), v)
    g1.step(2)
    g2.step(2)
    a, b = g1.get_state(), g2.get_state()
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_single_particle_and_determinism():
    p = workloads.smallest(n=4, n_particles=1, cg_tol=1e-13)
    g, o = pair(p)
    g.sample_mms(0.0)
    o.sample(0.0)
    g.step(3)
    o.step(3)
    assert pos_close(g.get_state()[0], o.state()[0])[0]
    # two runs of the same configuration are bit-identical
    p = CASES["ragged"]
    a, b = Pic(p), Pic(p)
    for s in (a, b):
        s.sample_mms(0.0)
        s.step(3)
    xa, va = a.get_state()
    xb, vb = b.get_state()
    assert np.array_equal(xa, xb) and np.array_equal(va, vb)


def test_step_before_sampling_is_a_state_error():
    from paper_2602_15130_gb300._lib import PIC_ESTATE, PicError

    g = Pic(CASES["smallest"])
    with pytest.raises(PicError) as ei:
        g.step(1)
    assert ei.value.status == PIC_ESTATE


def test_cg_iteration_cap_reports_no_convergence():
    from paper_2602_15130_gb300._lib import PIC_ENOCONV

    p = workloads.smallest(cg_maxit=1, cg_tol=1e-14)
    g = Pic(p)
    assert g.sample_mms(0.0, allow=(PIC_ENOCONV,)) == PIC_ENOCONV
    assert g.step(1, allow=(PIC_ENOCONV,)) == PIC_ENOCONV
    assert g.stats()["cg_iters_last"] == 1
