"""Pathwise adjoint (pic_adjoint_gradient) on the GPU.

J = (eps0/2) h^3 sum |E|^2 + (1/N_p) sum |v - v^M|^2 at t_N, gradient with
respect to a uniform applied field E_app and the initial velocities, with
collision pairs, accept decisions and scattering directions frozen. Checked
against central finite differences (h = 1e-6, FP64) of the library's own
forward, against finite differences of the FP64 oracle (an independent
forward), for invariance under the checkpoint interval (bit-identical: the
segments are recomputed exactly), and through torch.autograd.
"""
import numpy as np
import pytest

import inputs
from oracle import oracle as O
from paper_2602_15130_gb300 import Pic, PicObjective, workloads
from paper_2602_15130_gb300 import _lib

pytestmark = pytest.mark.gpu

E0 = (0.1, 0.1, 0.1)
FD_H = 1e-6


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch

    import __graft_entry__ as g

    g.build()
    assert torch.cuda.is_available()
    yield


def case(K, n=8, npart=4096, **kw):
    return workloads.smallest(n=n, n_particles=npart, K=K, cg_tol=1e-13, **kw)


def fd_eapp(sim, nsteps, d, v0=None):
    e_p, e_m = list(E0), list(E0)
    e_p[d] += FD_H
    e_m[d] -= FD_H
    jp = sim.adjoint_gradient(nsteps, 5, e_p, v0, grad=False)["J"]
    jm = sim.adjoint_gradient(nsteps, 5, e_m, v0, grad=False)["J"]
    return (jp - jm) / (2 * FD_H)


@pytest.mark.parametrize("K", [0, 8])
def test_eapp_gradient_matches_central_differences(K):
    sim = Pic(case(K))
    nsteps = 10
    r = sim.adjoint_gradient(nsteps, 4, E0)
    g = r["dJ_dEapp"]
    assert np.abs(g).max() > 1e-6
    for d in range(3):
        fd = fd_eapp(sim, nsteps, d)
        assert abs(g[d] - fd) <= 2e-5 * abs(fd) + 1e-8, (d, g[d], fd)


@pytest.mark.parametrize("K", [0, 8])
def test_v0_gradient_matches_directional_differences(K):
    p = case(K)
    sim = Pic(p)
    nsteps = 8
    o = O.Oracle(p)
    o.sample()
    _, vM0 = o.state()
    r = sim.adjoint_gradient(nsteps, 3, E0, vM0)
    delta = inputs.rng(5).standard_normal(vM0.shape)
    delta /= np.linalg.norm(delta)
    jp = sim.adjoint_gradient(nsteps, 3, E0, vM0 + FD_H * delta, grad=False)["J"]
    jm = sim.adjoint_gradient(nsteps, 3, E0, vM0 - FD_H * delta, grad=False)["J"]
    fd = (jp - jm) / (2 * FD_H)
    ad = float((r["dJ_dv0"] * delta).sum())
    assert abs(ad - fd) <= 2e-5 * abs(fd) + 1e-8, (ad, fd)
    # the default v0 is v^M(0): same objective as passing it explicitly
    r0 = sim.adjoint_gradient(nsteps, 3, E0, None)
    assert abs(r0["J"] - r["J"]) <= 1e-13 * abs(r["J"])


def test_gradient_does_not_depend_on_checkpoint_interval():
    sim = Pic(case(8))
    ref = sim.adjoint_gradient(12, 12, E0)
    for every in (1, 5, 7):
        r = sim.adjoint_gradient(12, every, E0)
        assert r["J"] == ref["J"]
        assert np.array_equal(r["dJ_dEapp"], ref["dJ_dEapp"])
        assert np.array_equal(r["dJ_dv0"], ref["dJ_dv0"])


def test_objective_and_gradient_against_oracle_differences():
    """The oracle's FP64 forward (an independent code) gives the same J, and
    its central differences give the same dJ/dE_app."""
    p = case(4, n=4, npart=300)
    nsteps = 4
    sim = Pic(p)
    r = sim.adjoint_gradient(nsteps, 2, E0)

    def J_oracle(e):
        o = O.Oracle(dict(p, E_app=tuple(e)))
        o.sample()
        o.step(nsteps)
        return o.objective()

    jo = J_oracle(E0)
    assert abs(r["J"] - jo[0]) <= 1e-10 * jo[0]
    assert abs(r["J_field"] - jo[1]) <= 1e-10 * jo[1] and abs(r["J_vel"] - jo[2]) <= 1e-10 * max(jo[2], 1e-30)
    for d in range(3):
        e_p, e_m = list(E0), list(E0)
        e_p[d] += FD_H
        e_m[d] -= FD_H
        fd = (J_oracle(e_p)[0] - J_oracle(e_m)[0]) / (2 * FD_H)
        assert abs(r["dJ_dEapp"][d] - fd) <= 2e-5 * abs(fd) + 1e-8, (d, r["dJ_dEapp"][d], fd)


def test_autograd_function_returns_the_adjoint():
    import torch

    p = case(8)
    sim = Pic(p)
    o = O.Oracle(p)
    o.sample()
    _, vM0 = o.state()
    E = torch.tensor(E0, dtype=torch.float64, requires_grad=True)
    v = torch.tensor(vM0, dtype=torch.float64, device="cuda", requires_grad=True)
    J = PicObjective.apply(E, v, sim, 6, 3)
    (2.0 * J).backward()
    r = sim.adjoint_gradient(6, 3, E0, vM0)
    assert abs(J.item() - r["J"]) <= 1e-14 * r["J"]
    assert np.allclose(E.grad.numpy(), 2.0 * r["dJ_dEapp"], rtol=0, atol=0)
    assert np.allclose(v.grad.cpu().numpy(), 2.0 * r["dJ_dv0"], rtol=0, atol=0)


def test_adjoint_rejects_other_forms():
    g = Pic(workloads.mixed(case(8)))
    with pytest.raises(_lib.PicError) as ei:
        g.adjoint_gradient(2, 1, E0)
    assert ei.value.status == _lib.PIC_EINVAL
    g = Pic(case(8, verify=_lib.PIC_VERIFY_ERROR1))
    with pytest.raises(_lib.PicError) as ei:
        g.adjoint_gradient(2, 1, E0)
    assert ei.value.status == _lib.PIC_EINVAL
