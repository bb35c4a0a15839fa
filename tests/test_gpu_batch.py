"""Batched form: replicates advanced together against single-domain runs of
the same configurations (and, for a small replicate, the FP64 oracle).

Sampling is identical (same FP64 inverse-CDF path per particle); after
steps a replicate matches its single-domain run within the precision form's
stated error (the batched Poisson solve sums in a different order), its
error norms within 3%."""
import ctypes

import numpy as np
import pytest

from oracle import oracle as O
from paper_2602_15130_gb300 import Batch, Pic, _lib, make_config, workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch

    import __graft_entry__ as g

    g.build()
    assert torch.cuda.is_available()
    yield


def configs():
    return [
        workloads.mixed(workloads.smallest(n=8, n_particles=8 ** 3 * 9 + 11, K=5, seed=3, dt=0.008)),
        workloads.mixed(workloads.smallest(n=12, n_particles=12 ** 3 * 20, K=16, seed=4, dt=0.01)),
        workloads.mixed(workloads.smallest(n=16, n_particles=16 ** 3 * 12 + 1, K=40, seed=5, dt=0.006)),
        workloads.mixed(workloads.smallest(n=4, n_particles=200, K=0, seed=6)),
    ]


def dpos(a, b):
    d = np.abs(a - b)
    return np.minimum(d, 1.0 - d)


def test_batch_sampling_is_identical_to_single_runs():
    cf = configs()
    b = Batch(cf)
    b.sample_mms(0.1)
    for r, p in enumerate(cf):
        s = Pic(p)
        s.sample_mms(0.1)
        xb, vb = b.get_state(r)
        xs, vs = s.get_state()
        assert np.array_equal(xb, xs) and np.array_equal(vb, vs), r


def test_batch_steps_track_single_runs_and_oracle():
    cf = configs()
    b = Batch(cf)
    b.sample_mms(0.0)
    b.step(5)
    eb = b.mms_error()
    for r, p in enumerate(cf):
        s = Pic(p)
        s.sample_mms(0.0)
        s.step(5)
        xb, vb = b.get_state(r)
        xs, vs = s.get_state()
        far_x = (dpos(xb, xs) > 1e-5).any(axis=1).mean()
        far_v = (np.abs(vb - vs) > 1e-4).any(axis=1).mean()
        assert far_x <= 0.01 and far_v <= 0.02, (r, far_x, far_v)
        es = s.mms_error()["array"]
        assert np.all(np.abs(eb[r] - es) <= 0.03 * es + 1e-7), (r, eb[r], es)
    # the smallest replicate against the FP64 oracle
    o = O.Oracle(dict(cf[0], cg_tol=1e-12))
    o.sample(0.0)
    o.step(5)
    eo = o.errors()
    assert np.all(np.abs(eb[0] - eo) <= 0.03 * eo + 1e-7), (eb[0], eo)
    assert all(i > 0 for i in b.cg_iters())


def test_batch_rejects_mixed_distributions_and_fp64():
    L = _lib.load()
    cf = configs()[:2]
    bad = [dict(cf[0]), dict(cf[1], fx_amp=0.2)]
    arr = (_lib.PicConfig * 2)(*[make_config(p) for p in bad])
    out = ctypes.c_void_p()
    assert L.pic_create_batch(arr, 2, None, None, ctypes.byref(out)) == _lib.PIC_EINVAL
    fp64 = [dict(cf[0], precision=0), cf[1]]
    arr = (_lib.PicConfig * 2)(*[make_config(p) for p in fp64])
    assert L.pic_create_batch(arr, 2, None, None, ctypes.byref(out)) == _lib.PIC_EINVAL


def test_batched_workload_recipe_small():
    cf = workloads.batched(n_rep=12, seed=7)
    cf = [dict(p, n=min(p["n"], 16), n_particles=min(p["n"], 16) ** 3 * (p["n_particles"] // p["n"] ** 3)) for p in cf]
    b = Batch(cf)
    b.sample_mms(0.0)
    b.step(2)
    e = b.mms_error()
    assert np.all(np.isfinite(e)) and e.shape == (12, 14)
    st = b.stats()
    assert st["n_coll"] > 0 and st["n_near_ties"] >= 0


def test_graph_replayed_steps_are_bit_identical_and_tuned():
    """After the autotuning steps a batch on a real stream replays captured
    graphs; its state must equal a batch on the legacy stream (no graphs)."""
    import torch

    cf = configs()[:3]
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        a = Batch(cf, stream=stream)
        a.sample_mms(0.0)
        a.step(8)
        sa = a.stats()
    b = Batch(cf, stream=0)
    b.sample_mms(0.0)
    b.step(8)
    assert sa["graph_replays"] >= 4 and b.stats()["graph_replays"] == 0
    assert sa["tuned_block"] in (128, 256) and sa["tuned_tile"] in (0, 1)
    for r in range(3):
        xa, va = a.get_state(r)
        xb, vb = b.get_state(r)
        assert np.array_equal(xa, xb) and np.array_equal(va, vb), r
