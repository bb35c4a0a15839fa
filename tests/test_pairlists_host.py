"""The oracle's pair log of Algorithm 1 and the rules that compare pair
lists (CPU only).

The log must say what the oracle did: its candidate and accepted counts are
the oracle's n_cand and n_coll, every candidate has p != q below the cell
count, every (cell, outcome) with c >= 2 draws N_pairs once, and N_pairs is
the floor of C(c, 2) P_coll,max + U within one of its expectation. The
comparison rules accept a difference only after a flagged decision: a
planted accept flip or N_pairs change fails them unless the record carries
its flag.
"""
import numpy as np
import pytest

import pairlists
from oracle import oracle as O
from paper_2602_15130_gb300 import workloads


@pytest.fixture(scope="module")
def logged():
    p = workloads.smallest()
    o = O.Oracle(p)
    o.sample(0.0)
    o.reset_stats()
    o.set_pair_log(True)
    o.collide_avg(0)
    log = o.pair_log()
    _, count, _, _ = o.sort()
    return p, o, log, count


def test_pair_log_matches_the_counts(logged):
    p, o, log, count = logged
    st = o.stats()
    cand = log[log[:, 3] >= 0]
    assert len(cand) == st["n_cand"] > 0
    assert cand[:, 6].sum() == st["n_coll"] > 0
    assert ((cand[:, 7] & pairlists.TIE) != 0).sum() == st["n_near_ties"]
    c = count[cand[:, 1]]
    assert (cand[:, 4] != cand[:, 5]).all()
    assert (cand[:, 4] >= 0).all() and (cand[:, 4] < c).all() and (cand[:, 5] < c).all()


def test_pair_log_draws_n_pairs_once_per_cell_and_outcome(logged):
    p, o, log, count = logged
    head = log[log[:, 3] == -1]
    cells = np.flatnonzero(count >= 2)
    assert len(head) == len(cells) * p["K"]
    assert set(map(tuple, head[:, 1:3])) == {(int(c), k) for c in cells for k in range(p["K"])}
    assert (head[:, 7] == pairlists.NPAIRS).all()
    pm = O.pmax(O.make_cfg(p))
    mean = count[head[:, 1]].astype(float) * (count[head[:, 1]] - 1) / 2.0 * pm
    assert (head[:, 6] >= np.floor(mean)).all() and (head[:, 6] <= np.floor(mean) + 1).all()
    # slots of each (cell, outcome) run 0 .. N_pairs - 1
    for (c0, cell, k), grp in pairlists._groups(pairlists.canonical(log)).items():
        assert np.array_equal(grp[1:, 3], np.arange(grp[0, 6]))


def test_identical_lists_compare_clean(logged):
    _, _, log, _ = logged
    flagged, n = pairlists.compare_flagged(log.copy(), log)
    assert flagged == set() and n == 0


def test_an_unflagged_accept_flip_is_caught_and_a_flagged_one_allowed(logged):
    _, _, log, _ = logged
    cand = np.flatnonzero(log[:, 3] >= 0)
    i = cand[len(cand) // 2]
    bad = log.copy()
    bad[i, 6] ^= 1
    with pytest.raises(AssertionError):
        pairlists.compare_flagged(bad, log)
    bad[i, 7] |= pairlists.TIE
    flagged, n = pairlists.compare_flagged(bad, log)
    assert flagged == {(int(log[i, 0]), int(log[i, 1]))} and n == 1


def test_an_unflagged_n_pairs_change_is_caught_and_a_flagged_one_allowed(logged):
    _, _, log, _ = logged
    can = pairlists.canonical(log)
    groups = pairlists._groups(can)
    key = next(k for k, g in groups.items() if g[0, 6] >= 2)
    grp = groups[key]
    shorter = np.concatenate([grp[:1], grp[1:-1]])  # one candidate fewer
    shorter = shorter.copy()
    shorter[0, 6] -= 1
    rest = [g for k, g in groups.items() if k != key]
    bad = np.concatenate(rest + [shorter])
    with pytest.raises(AssertionError):
        pairlists.compare_flagged(bad, log)
    bad[-len(shorter), 7] |= pairlists.FLOOR
    flagged, n = pairlists.compare_flagged(bad, log)
    assert flagged == {key[:2]} and n == 1


def test_a_changed_index_draw_is_caught_even_after_a_flag(logged):
    _, _, log, _ = logged
    cand = np.flatnonzero(log[:, 3] >= 1)
    i = cand[0]
    bad = log.copy()
    bad[i - 1 if log[i - 1, 3] >= 0 else i, 7] |= pairlists.TIE
    bad[i, 5] = (bad[i, 5] + 1) % 8 if bad[i, 5] + 1 != bad[i, 4] else (bad[i, 5] + 2) % 8
    with pytest.raises(AssertionError):
        pairlists.compare_flagged(bad, log)


def test_pair_draws_are_uniform_over_ordered_pairs():
    """Algorithm 1 draws p uniformly over the cell and q uniformly over the
    others (the distribution of redrawing q until it differs from p): over
    every candidate of many outcomes in one cell of six particles the 30
    ordered pairs are equally frequent (chi-square at the 0.1% level) and
    no candidate has p = q."""
    import inputs
    from scipy import stats

    p = workloads.smallest(n=2, n_particles=6, K=400, dt=0.5)
    o = O.Oracle(p)
    x, v = inputs.particles(6, seed=4, clustered_cells=1, n=2)
    o.set_state(x, v)
    o.set_pair_log(True)
    o.collide_avg(0)
    cand = o.pair_log()
    cand = cand[cand[:, 3] >= 0]
    assert (cand[:, 4] != cand[:, 5]).all()
    counts = np.zeros((6, 6))
    np.add.at(counts, (cand[:, 4], cand[:, 5]), 1)
    off = counts[~np.eye(6, dtype=bool)]
    assert off.sum() == len(cand) > 3000
    assert stats.chisquare(off).pvalue > 1e-3
