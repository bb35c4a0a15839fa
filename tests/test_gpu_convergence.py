"""Observed convergence on the first three levels of Table 1 (Sec. 5.3,
s = 7, r = 5 collisional, s = 5 collisionless), through the C ABI: the rates
the error analysis of Sec. 4 predicts, and the verdicts of Sec. 5.4 on the
injected coding errors. Levels 0-2 (n = 8, 12, 16) run in seconds; the full
five-level study is ``python -m paper_2602_15130_gb300.convergence``."""
import pytest

from paper_2602_15130_gb300 import convergence as C

pytestmark = pytest.mark.gpu

LEVELS = [0, 1, 2]


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch

    import __graft_entry__ as g

    g.build()
    assert torch.cuda.is_available()
    yield


def _rates(res, variant, key):
    return res["variants"][variant]["rates"][key]["pairwise"]


def test_collisionless_second_order():
    res = C.run_study("table1-collisionless", LEVELS, "fp64", ["coupled"], log=lambda s: None)
    for key in ("x_eps2", "v_eps2", "phi_eps2"):
        r = _rates(res, "coupled", key)
        assert all(1.7 <= p <= 2.3 for p in r), (key, r)


def test_isolated_collisions_converge_and_injected_errors():
    res = C.run_study("table1-collisional", LEVELS, "mixed", ["isolated", "isolated_error1", "isolated_error2"],
                      log=lambda s: None)
    # reference and Error 2: eps_2 between the worst case 2 and the random walk 2.5
    for v in ("isolated", "isolated_error2"):
        for key in ("x_eps2", "v_eps2"):
            r = _rates(res, v, key)
            assert all(2.0 <= p <= 2.8 for p in r), (v, key, r)
    # Error 1 changes the expected outcome: no convergence
    for key in ("x_eps2", "v_eps2"):
        assert _rates(res, "isolated_error1", key)[-1] < 0.5
    # the angle metric converges for the reference and Error 1, and stalls
    # near max |F_aniso - F_iso| for Error 2
    for v in ("isolated", "isolated_error1"):
        e = res["variants"][v]["rates"]["angle_epsinf_chi"]["errors"]
        assert e[-1] < e[0] / 10
    e = res["variants"]["isolated_error2"]["rates"]["angle_epsinf_chi"]["errors"]
    assert all(0.025 < x < 0.045 for x in e), e
