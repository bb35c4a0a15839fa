"""The oracle's threaded loops (over independent cells and particles) give
the same bits as its serial run: positions, velocities, field and every
counter after whole steps with collisions, in both distribution forms."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2602_15130_gb300 import workloads


@pytest.mark.parametrize("p", [workloads.smallest(K=8), dict(workloads.paper_small(), K=4)],
                         ids=["config", "paper"])
def test_threads_give_the_serial_bits(p):
    out = []
    try:
        for th in (1, 3):
            O.set_threads(th)
            o = O.Oracle(p)
            o.sample(0.0)
            o.step(2)
            x, v = o.state()
            rho, phi, E = o.field()
            st = o.stats()
            out.append((x, v, phi, E, st["n_cand"], st["n_coll"]))
            o.close()
    finally:
        O.set_threads(1)
    for a, b in zip(out[0], out[1]):
        assert np.array_equal(a, b)
    assert out[0][5] > 0
