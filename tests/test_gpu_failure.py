"""Failure detection without a GPU fault: the persistent CG kernels' grid
barriers and the persistent batched step's phase waits are bounded (4e9 SM
cycles, about 2 s). A host-side injection makes a wait run out (one block
leaves before its first barrier, or one work item is never counted
complete, so what the others wait for never comes); the call returns
PIC_ETIMEOUT, and after a new sampling the context steps bit for bit like a
fresh one."""
import time

import numpy as np
import pytest

from paper_2602_15130_gb300 import Batch, Pic, _lib, workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch

    import __graft_entry__ as g

    g.build()
    assert torch.cuda.is_available()
    yield


@pytest.mark.parametrize("form", ["fp64", "mixed"])
def test_bounded_barrier_wait_runs_out_and_the_context_recovers(form):
    p = workloads.smallest(n=16, n_particles=16 ** 3 * 8)  # a 4-block CG grid
    if form == "mixed":
        p = workloads.mixed(p)
    ref = Pic(p)
    ref.sample_mms(0.0)
    ref.step(2)
    xr, vr = ref.get_state()
    g = Pic(p)
    g.sample_mms(0.0)
    g.inject_barrier_stall()
    t0 = time.time()
    assert g.step(1, allow=(_lib.PIC_ETIMEOUT,)) == _lib.PIC_ETIMEOUT
    assert time.time() - t0 < 60
    g.sample_mms(0.0)
    g.step(2)
    x, v = g.get_state()
    assert np.array_equal(x, xr) and np.array_equal(v, vr)


def test_injection_needs_a_grid_barrier():
    small = Pic(workloads.smallest())  # 8^3 nodes: a one-block CG grid
    with pytest.raises(_lib.PicError) as ei:
        small.inject_barrier_stall()
    assert ei.value.status == _lib.PIC_EINVAL


def test_batched_step_bounded_wait_runs_out_and_the_batch_recovers():
    """The persistent batched step: one work item left uncounted makes the
    items that depend on it wait out their bound; the step returns
    PIC_ETIMEOUT, and after a new sampling the batch steps bit for bit like
    a fresh one (through its tuning steps and graph replays)."""
    import torch

    cf = [workloads.mixed(workloads.smallest(n=n, n_particles=n ** 3 * 8, K=k, seed=s))
          for n, k, s in ((8, 16, 1), (12, 8, 2), (16, 32, 3))]
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        ref = Batch(cf, stream=stream)
        ref.sample_mms(0.0)
        ref.step(7)
        xr, vr = ref.get_state(2)
        b = Batch(cf, stream=stream)
        b.sample_mms(0.0)
        b.step(2)
        b.inject_barrier_stall()
        t0 = time.time()
        assert b.step(1, allow=(_lib.PIC_ETIMEOUT,)) == _lib.PIC_ETIMEOUT
        assert time.time() - t0 < 60
        b.sample_mms(0.0)
        b.step(7)
        x, v = b.get_state(2)
    assert np.array_equal(x, xr) and np.array_equal(v, vr)
