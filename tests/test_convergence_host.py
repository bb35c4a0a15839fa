"""Host logic of the refinement studies (no GPU): the Table 1 schedule
recipe against the paper's printed table, and the rate fit against exact
power laws."""
import math
from pathlib import Path

import pytest

from paper_2602_15130_gb300 import convergence as C
from paper_2602_15130_gb300 import derived, workloads as W

GOLDEN = Path(__file__).parent / "golden"


def _table1():
    return [list(map(float, l.split())) for l in (GOLDEN / "paper_table1_discretizations.txt").read_text().splitlines()
            if l.strip() and not l.startswith("#")]


def test_table1_recipe_reproduces_the_paper_table():
    for lvl, steps, nax, ncell, navg, inv_p, np_coll, np_free in _table1():
        l = int(lvl) - 1
        p = W.table1_level(l, collisions=True)
        q = W.table1_level(l, collisions=False)
        assert p["n"] == nax and p["steps"] == steps and abs(p["dt"] * steps - W.TABLE1_T) < 1e-15
        assert p["n_particles"] == np_coll and p["K"] == navg
        assert q["n_particles"] == np_free and q["K"] == 0
        # 1/P_coll,max of the table, to its printed rounding
        assert abs(1.0 / derived(p)["pmax"] / inv_p - 1.0) < 2e-4
        # the densest cell of (1 + 0.3)^3 times the mean fits max_ppc
        assert p["max_ppc"] >= 1.3 ** 3 * np_coll / ncell + 64 and p["max_ppc"] % 32 == 0


@pytest.mark.parametrize("p", [1.0, 2.0, 2.5])
def test_rate_fit_recovers_power_laws(p):
    h = [1 / 8, 1 / 12, 1 / 16, 1 / 20, 1 / 24]
    e = [3.0 * x ** p for x in h]
    r = C.observed_rates(h, e)
    assert all(abs(x - p) < 1e-12 for x in r["pairwise"])
    assert abs(r["fit"] - p) < 1e-12


def test_group_errors():
    rec = {"eps2": dict(x=3.0, y=4.0, z=0.0, u=1.0, v=1.0, w=1.0, phi=0.5),
           "epsinf": dict(x=1.0, y=5.0, z=2.0, u=0.1, v=0.3, w=0.2, phi=0.25)}
    assert C.group_error(rec, "epsinf", "x") == 5.0
    assert C.group_error(rec, "epsinf", "v") == 0.3
    assert abs(C.group_error(rec, "eps2", "x") - math.sqrt(25.0 / 3)) < 1e-15
    assert C.group_error(rec, "eps2", "phi") == 0.5


def test_study_tables_are_consistent():
    for table in (C.TABLE1_COLLISIONAL, C.TABLE1_COLLISIONLESS, C.PAPER_COLLISIONAL, C.PAPER_COLLISIONLESS,
                  C.REFINE):
        for name, (over, pred) in table.items():
            assert set(pred) <= {"x", "v", "phi", "x2", "v2"}
            assert set(over) <= {"verify", "couple_qm_zero", "couple_q_zero", "K"}
    # the isolated-collision variants switch the field off the particles
    for name, (over, _) in C.TABLE1_COLLISIONAL.items():
        if name.startswith("isolated"):
            assert over["couple_qm_zero"] == 1 and over["verify"] & C.ISO


def test_paper_table1_schedule():
    for lvl, steps, nax, ncell, navg, inv_p, np_coll, np_free in _table1():
        l = int(lvl) - 1
        p = W.paper_table1_level(l, collisions=True)
        q = W.paper_table1_level(l, collisions=False)
        assert p["n"] == nax and p["steps"] == steps and abs(p["dt"] * steps - 1.0) < 1e-15
        assert p["n_particles"] == np_coll and p["K"] == navg and q["n_particles"] == np_free and q["K"] == 0
        assert abs(1.0 / derived(p)["pmax"] / inv_p - 1.0) < 2e-4
        assert p["dist"] == 1 and p["n_sigma"] == 3 and q["n_sigma"] == 0


def test_batched_study_replicates_match_the_committed_list():
    """The batched study's replicate draws (mesh edge on {8, 16, 32, 64},
    particles per cell in [8, 64], K in [4, 64], host generator seed 42)
    equal the committed list, and each follows its stated recipe."""
    rows = [l.split() for l in (GOLDEN / "batched_replicates.txt").read_text().splitlines()
            if l.strip() and not l.startswith("#")]
    reps = W.batched()
    assert len(rows) == len(reps) == 256
    for r, (row, p) in enumerate(zip(rows, reps)):
        assert [int(x) for x in row[:5]] == [r, p["n"], p["n_particles"], p["K"], p["seed"]]
        assert float(row[5]) == p["sigma0"]
        ppc = p["n_particles"] // p["n"] ** 3
        assert p["n"] in (8, 16, 32, 64) and 8 <= ppc <= 64 and p["n_particles"] == ppc * p["n"] ** 3
        assert 4 <= p["K"] <= 64 and p["seed"] == 1000 + r
    assert len({p["n"] for p in reps}) == 4


def test_a_level_that_outgrows_max_ppc_runs_again_with_twice_the_capacity(monkeypatch):
    """run_one: a cell over max_ppc makes the steps return PIC_ECAPACITY;
    the level starts over with max_ppc doubled, and the record names the
    capacity it ran with. Other errors still stop the study."""
    from paper_2602_15130_gb300 import _lib

    made = []

    class FakePic:
        def __init__(self, p):
            self.p = p
            made.append(p["max_ppc"])

        def sample_mms(self, t0):
            pass

        def set_profiling(self, on):
            pass

        def step(self, n, allow=()):
            if self.p["max_ppc"] < 1000:
                raise _lib.PicError(_lib.PIC_ECAPACITY, "pic_step")
            return _lib.PIC_OK

        def kernel_times(self):
            return {"dsmc": {"ms": 1.0, "launches": 2}}

        def mms_error(self):
            e = {k: 1.0 for k in ("x", "y", "z", "u", "v", "w", "phi")}
            return {"eps2": e, "epsinf": e}

        def stats(self):
            return {"n_coll": 0, "n_cand": 0, "cg_iters_max": 1, "n_gmax_exceed": 0}

        def close(self):
            pass

    monkeypatch.setattr(C, "Pic", FakePic)
    rec = C.run_one(dict(W.paper_table1_level(1), max_ppc=384), "mixed")
    assert made == [384, 768, 1536] and rec["max_ppc"] == 1536 and rec["status"] == "PIC_OK"

    class Failing(FakePic):
        def step(self, n, allow=()):
            raise _lib.PicError(_lib.PIC_ETIMEOUT, "pic_step")

    monkeypatch.setattr(C, "Pic", Failing)
    with pytest.raises(_lib.PicError):
        C.run_one(W.paper_table1_level(1), "mixed")
