"""pic_poisson_solve_noalloc: the Poisson solve for callers that cannot
allocate device memory while they run (a memory budget fixed at start-up,
or a framework that forbids cudaMalloc/cudaFree on its hot path). Its
scratch is a fixed array inside the library, so this test checks that two
calls in a row, through the C ABI, give the same potential and field as the
context path (pic_set_state + pic_get_field) within the tolerance of the
other GPU tests."""
import ctypes

import numpy as np
import pytest

import inputs
from oracle import oracle as O
from paper_2602_15130_gb300 import Pic, _lib, workloads

pytestmark = pytest.mark.gpu

TOL = 1e-10


def _rhs(p, rho, t):
    """b = rho/eps0 - Lap phi^M - rho^M/eps0 at the nodes (Eq. poisson_mms)."""
    cfg = O.make_cfg(p)
    n = p["n"]
    h = 1.0 / n
    q = 0.0 if p.get("couple_q_zero") else p["q"]
    b = np.empty(n ** 3)
    for k in range(n):
        for j in range(n):
            for i in range(n):
                X = [i * h, j * h, k * h]
                b[i + n * (j + n * k)] = rho[i + n * (j + n * k)] / p["eps0"] - O.lap_phiM(cfg, X, t) - \
                    O.rhoM(cfg, q, X, t) / p["eps0"]
    return b


def _context_field(p, seed, t0):
    x, v = inputs.particles(p["n_particles"], seed=seed)
    sim = Pic(p)
    sim.set_state(x, v, t0=t0, step=0)
    rho, phi, E = sim.get_field()
    sim.close()
    return rho, phi, E


def test_noalloc_solve_matches_context_path_twice():
    import torch

    import __graft_entry__ as g

    g.build()
    L = _lib.load()
    p = workloads.smallest(n=16, n_particles=16 ** 3 * 8, cg_tol=1e-13)
    n, m = p["n"], p["n"] ** 3
    stream = torch.cuda.current_stream()
    for call, (seed, t0) in enumerate([(5, 0.0), (6, 0.37)]):
        rho, phi_ref, E_ref = _context_field(p, seed, t0)
        b = torch.tensor(_rhs(p, rho, t0), device="cuda")
        phi = torch.zeros(m, dtype=torch.float64, device="cuda")
        E = torch.full((3, m), float("nan"), dtype=torch.float64, device="cuda")
        iters = ctypes.c_int32(-1)
        res = ctypes.c_double(-1.0)
        st = L.pic_poisson_solve_noalloc(n, b.data_ptr(), phi.data_ptr(), E.data_ptr(), 1e-13, 20000,
                                         ctypes.c_void_p(stream.cuda_stream), ctypes.byref(iters),
                                         ctypes.byref(res))
        assert st == _lib.PIC_OK, (call, _lib.STATUS.get(st))
        assert iters.value > 0 and 0.0 <= res.value <= 1e-13
        got_phi = phi.cpu().numpy()
        got_E = E.cpu().numpy().T  # [3][n^3] -> [n^3][3]
        assert np.abs(got_phi - phi_ref).max() <= TOL * np.abs(phi_ref).max(), call
        assert np.abs(got_E - E_ref).max() <= TOL * np.abs(E_ref).max(), call


def test_noalloc_rejects_oversize_and_host_pointers():
    import torch

    L = _lib.load()
    big = 49
    t = torch.zeros(big ** 3, dtype=torch.float64, device="cuda")
    E = torch.zeros(3 * big ** 3, dtype=torch.float64, device="cuda")
    assert L.pic_poisson_solve_noalloc(big, t.data_ptr(), t.data_ptr(), E.data_ptr(), 1e-10, 100, None,
                                       None, None) == _lib.PIC_EINVAL
    hb = np.zeros(8 ** 3)
    d = torch.zeros(8 ** 3, dtype=torch.float64, device="cuda")
    dE = torch.zeros(3 * 8 ** 3, dtype=torch.float64, device="cuda")
    assert L.pic_poisson_solve_noalloc(8, hb.ctypes.data, d.data_ptr(), dE.data_ptr(), 1e-10, 100, None,
                                       None, None) == _lib.PIC_EINVAL


def _solve(L, n, b, phi, E, tol, maxit):
    import torch

    iters = ctypes.c_int32(-1)
    res = ctypes.c_double(-1.0)
    st = L.pic_poisson_solve_noalloc(n, b.data_ptr(), phi.data_ptr(), E.data_ptr(), tol, maxit,
                                     ctypes.c_void_p(torch.cuda.current_stream().cuda_stream),
                                     ctypes.byref(iters), ctypes.byref(res))
    return st, iters.value, res.value


def test_noalloc_maxit_and_warm_start():
    """maxit = 1 stops after one iteration with PIC_ENOCONV and phi holding
    that iterate; a solve warm-started from the converged phi (the documented
    use of phi as input) takes no iteration and returns the same phi and E."""
    import torch

    L = _lib.load()
    p = workloads.smallest(n=12, n_particles=12 ** 3 * 8, cg_tol=1e-13)
    n, m = p["n"], p["n"] ** 3
    rho, phi_ref, E_ref = _context_field(p, 9, 0.2)
    b = torch.tensor(_rhs(p, rho, 0.2), device="cuda")
    phi = torch.zeros(m, dtype=torch.float64, device="cuda")
    E = torch.zeros((3, m), dtype=torch.float64, device="cuda")
    st, it, res = _solve(L, n, b, phi, E, 1e-13, 1)
    assert st == _lib.PIC_ENOCONV and it == 1 and res > 1e-13, (st, it, res)
    assert np.abs(phi.cpu().numpy()).max() > 0.0  # the first iterate was written
    st, it, res = _solve(L, n, b, phi, E, 1e-13, 20000)
    assert st == _lib.PIC_OK and it > 1 and res <= 1e-13
    phi1, E1 = phi.cpu().numpy().copy(), E.cpu().numpy().copy()
    assert np.abs(phi1 - phi_ref).max() <= TOL * np.abs(phi_ref).max()
    # the true residual of the 1e-13 solution is far below 1e-10: no iteration
    st, it, res = _solve(L, n, b, phi, E, 1e-10, 20000)
    assert st == _lib.PIC_OK and it == 0 and res <= 1e-10, (st, it, res)
    assert np.abs(phi.cpu().numpy() - phi1).max() <= 1e-14 * np.abs(phi1).max()
    assert np.abs(E.cpu().numpy() - E1).max() <= 1e-13 * np.abs(E1).max()


def test_noalloc_rejects_another_devices_memory():
    import torch

    if torch.cuda.device_count() < 2:
        pytest.skip("one visible GPU: no memory of another device to pass")
    L = _lib.load()
    n, m = 8, 8 ** 3
    with torch.cuda.device(1):
        b1 = torch.zeros(m, dtype=torch.float64, device="cuda:1")
    phi = torch.zeros(m, dtype=torch.float64, device="cuda:0")
    E = torch.zeros(3 * m, dtype=torch.float64, device="cuda:0")
    torch.cuda.set_device(0)
    assert L.pic_poisson_solve_noalloc(n, b1.data_ptr(), phi.data_ptr(), E.data_ptr(), 1e-10, 100, None,
                                       None, None) == _lib.PIC_EINVAL
