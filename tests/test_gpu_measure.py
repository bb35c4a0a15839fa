"""The library's measurement calls, which the benchmark's rooflines divide
by (no counterpart in the paper): the ALU issue rates of the GPU, and the
rate of the host link each way between a pinned host buffer and the device."""
import ctypes

import numpy as np
import pytest

from paper_2602_15130_gb300 import _lib, measure_alu_peaks, measure_link

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch

    import __graft_entry__ as g

    g.build()
    assert torch.cuda.is_available()
    yield


def test_alu_peaks_positive_with_the_fp64_pipe_far_below_fp32():
    pk = measure_alu_peaks()
    assert set(pk) == {"imad", "lop3", "ffma", "dfma", "philox_blocks"}
    assert all(v > 0 for v in pk.values()), pk
    assert pk["dfma"] < pk["ffma"] / 8, pk


def test_link_rate_leaves_the_buffer_unchanged_and_rejects_bad_buffers():
    import torch

    h = torch.arange(1 << 22, dtype=torch.int64).pin_memory()  # 32 MiB
    want = h.clone()
    r = measure_link(h)
    assert r["bytes"] == 32 << 20
    assert r["h2d"] > 1e9 and r["d2h"] > 1e9, r
    assert torch.equal(h, want)
    L = _lib.load()
    out = (ctypes.c_double * 2)()
    pageable = np.zeros(1024)
    assert L.pic_measure_link(ctypes.c_void_p(pageable.ctypes.data), 8192, None, out) == _lib.PIC_EINVAL
    assert L.pic_measure_link(ctypes.c_void_p(h.data_ptr()), 0, None, out) == _lib.PIC_EINVAL
    assert L.pic_measure_link(None, 8192, None, out) == _lib.PIC_EINVAL
