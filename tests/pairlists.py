"""Pair lists of Algorithm 1 from the library's decision log and the
oracle's pair log, and the rules that compare them.

A record is 8 int32: (c0, cell, outcome, slot, p, q, result, kind); slot -1
is the N_pairs draw of a (cell, outcome) with result = N_pairs, a candidate
record carries the in-cell indices p, q and result 1 (accepted) or 0.
kind bit 1 marks an accept decision inside the tie bound, bit 2 an N_pairs
draw inside the floor bound, bit 4 the N_pairs record.

This module holds no step of the method: it sorts and compares records.
"""
from __future__ import annotations

import numpy as np

TIE, FLOOR, NPAIRS = 1, 2, 4


def canonical(log: np.ndarray) -> np.ndarray:
    """Records sorted by (c0, cell, outcome, slot)."""
    log = np.asarray(log, dtype=np.int32).reshape(-1, 8)
    order = np.lexsort((log[:, 3], log[:, 2], log[:, 1], log[:, 0]))
    return log[order]


def _groups(log: np.ndarray) -> dict:
    out = {}
    if len(log) == 0:
        return out
    keys = log[:, :3]
    cut = np.flatnonzero((np.diff(keys, axis=0) != 0).any(axis=1)) + 1
    for part in np.split(log, cut):
        out[tuple(int(k) for k in part[0, :3])] = part
    return out


def compare_flagged(gpu: np.ndarray, orc: np.ndarray) -> tuple[set, int]:
    """Compare the precision form's full pair list with the oracle's.

    Per (c0, cell, outcome): the N_pairs draws must agree unless the GPU
    flagged its draw (FLOOR); every common slot has the same (p, q), since
    the index draws are integer operations on the same Philox words; the
    accept decisions agree up to the first decision the GPU flagged (TIE),
    after which the velocities of that outcome may differ. Returns the set
    of (c0, cell) holding a flagged decision and the number of flags."""
    gg, go = _groups(canonical(gpu)), _groups(canonical(orc))
    assert set(gg) == set(go), "the (call, cell, outcome) groups differ"
    flagged, nflags = set(), 0
    for key, a in gg.items():
        b = go[key]
        assert a[0, 3] == -1 and b[0, 3] == -1 and a[0, 7] & NPAIRS, key
        na, nb = int(a[0, 6]), int(b[0, 6])
        ca, cb = a[1:], b[1:]
        assert np.array_equal(ca[:, 3], np.arange(na)) and np.array_equal(cb[:, 3], np.arange(nb)), key
        first = None  # first slot at which the GPU's decisions may differ
        if a[0, 7] & FLOOR:
            first = -1
            nflags += 1
        else:
            assert na == nb, (key, na, nb)
        ties = np.flatnonzero(ca[:, 7] & TIE)
        nflags += len(ties)
        if len(ties) and first is None:
            first = int(ca[ties[0], 3])
        m = min(na, nb)
        assert np.array_equal(ca[:m, 4:6], cb[:m, 4:6]), key
        upto = m if first is None else max(0, min(m, first))
        assert np.array_equal(ca[:upto, 6], cb[:upto, 6]), key
        if first is not None:
            flagged.add(key[:2])
    return flagged, nflags


def flagged_cells(gpu: np.ndarray, c0: int) -> set:
    """Cells of call c0 holding a flagged decision in a (flagged-only or
    full) decision log."""
    log = np.asarray(gpu).reshape(-1, 8)
    sel = (log[:, 0] == c0) & ((log[:, 7] & (TIE | FLOOR)) != 0)
    return set(int(c) for c in log[sel, 1])


def step_tracking_flags(g, o, nsteps: int) -> np.ndarray:
    """Advance the library context g (precision form, decision log on in
    flagged mode) and the oracle o one step at a time and return the mask
    of particles a flagged FP32 decision can have reached.

    A particle is reached when, at either collision call of a step, it sits
    (on either side) in a cell that held a flagged decision, or in a cell
    with a particle reached earlier, or when its cell differs between the
    two sides (an FP32 position on the other side of a cell face). Call A
    of step n uses the cells before the drift, call B those after it."""
    reached = np.zeros(g.np, bool)
    step0 = int(g.stats()["step"])
    cg, co = g.get_sort()[0], o.sort()[0]
    for k in range(nsteps):
        g.step(1)
        o.step(1)
        log = g.decision_log()
        cg1, co1 = g.get_sort()[0], o.sort()[0]
        for phase, (a, b) in enumerate(((cg, co), (cg1, co1))):
            reached |= a != b
            hit = flagged_cells(log, 2 * (step0 + k) + phase)
            hit |= set(int(c) for c in a[reached]) | set(int(c) for c in b[reached])
            if hit:
                cells = np.fromiter(hit, dtype=np.int64)
                reached |= np.isin(a, cells) | np.isin(b, cells)
        cg, co = cg1, co1
    return reached
