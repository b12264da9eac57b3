"""Pins of the oracle's displacement step (System.rebucket): SDs regrouped by a new cell index
with the cells' slot ranges fixed.  Checked against properties the definition implies, not by
restating it: conservation, each SD in the cell its index names, old order kept within a cell,
the identity displacement, a round trip, and the capacity rule."""
import numpy as np
import pytest

import oracle
from paper_2101_06318_b300 import inputs


def _system(seed, n_cell=12, spare=3):
    rng = np.random.default_rng(seed)
    counts = rng.integers(0, 9, n_cell)
    width = counts + spare                                  # spare slots: capacity to move into
    n = int(width.sum())
    cs = np.concatenate([[0], np.cumsum(width)]).astype(np.uint32)
    xi = np.zeros(n, np.uint64)
    for c in range(n_cell):
        xi[cs[c]:cs[c] + counts[c]] = rng.integers(1, 10 ** 6, counts[c])
    attr = np.vstack([rng.uniform(1e-15, 1e-12, n), rng.random(n)])
    attr[:, xi == 0] = 0.0
    return oracle.System(xi, attr, cs, 1.0), rng


def _records(s):
    live = np.flatnonzero(s.xi)
    return sorted(zip(s.xi[live].tolist(), s.attr[0, live].tolist(), s.attr[1, live].tolist()))


def test_rebucket_conserves_and_places_every_sd():
    for seed in range(20):
        s, rng = _system(seed)
        before = _records(s)
        live = np.flatnonzero(s.xi)
        tag = {i: (int(s.xi[i]), float(s.attr[1, i])) for i in live}     # identities (xi, attr 1)
        cid = np.full(len(s.xi), -1)
        cid[live] = rng.integers(0, s.n_cell, len(live))
        ok = s.rebucket(cid)
        if not ok:
            continue
        assert _records(s) == before                          # the same SDs, nothing else
        for c in range(s.n_cell):
            lo, hi = int(s.cell_start[c]), int(s.cell_start[c + 1])
            x = s.xi[lo:hi]
            k = int(np.count_nonzero(x))
            assert np.all(x[:k] != 0) and np.all(x[k:] == 0)   # live SDs first
            # every SD here was sent here, and in its old slot order
            olds = [next(i for i in live if tag[i] == (int(x[j]), float(s.attr[1, lo + j]))) for j in range(k)]
            assert all(cid[i] == c for i in olds)
            assert olds == sorted(olds)


def test_rebucket_identity_and_round_trip():
    s, rng = _system(3, spare=10)
    x0, a0 = s.xi.copy(), s.attr.copy()
    cell_of = np.repeat(np.arange(s.n_cell), np.diff(s.cell_start.astype(np.int64)))
    assert s.rebucket(cell_of)                               # nobody moves: nothing changes
    assert np.array_equal(s.xi, x0) and np.array_equal(s.attr, a0)
    # move everything of cell 2 to cell 5, then back: the original layout returns
    live2 = [i for i in np.flatnonzero(s.xi) if cell_of[i] == 2]
    if live2 and np.count_nonzero(s.xi[s.cell_start[5]:s.cell_start[6]]) + len(live2) <= \
            s.cell_start[6] - s.cell_start[5]:
        cid = cell_of.copy()
        cid[live2] = 5
        assert s.rebucket(cid)
        cell_now = np.repeat(np.arange(s.n_cell), np.diff(s.cell_start.astype(np.int64)))
        back = cell_now.copy()
        moved = [i for i in np.flatnonzero(s.xi) if cell_now[i] == 5 and s.attr[1, i] in a0[1, live2]]
        back[moved] = 2
        assert s.rebucket(back)
        assert np.array_equal(s.xi, x0) and np.array_equal(s.attr, a0)


def test_rebucket_capacity_and_range_leave_state_unchanged():
    s, _ = _system(5, spare=0)
    x0 = s.xi.copy()
    live = np.flatnonzero(s.xi)
    cid = np.zeros(len(s.xi), np.int64)                      # all into cell 0: over its width
    if len(live) > s.cell_start[1] - s.cell_start[0]:
        assert not s.rebucket(cid)
        assert np.array_equal(s.xi, x0)
    bad = np.full(len(s.xi), s.n_cell)
    assert not s.rebucket(bad) or len(live) == 0
    assert np.array_equal(s.xi, x0)
