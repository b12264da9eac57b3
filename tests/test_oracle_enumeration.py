"""Exhaustive pins of the oracle's whole step on cells of 4 to 8 SDs.

For a cell of n SDs one step (Sec. 2.2, Steps 1-3) draws a uniformly random
order of the cell's list (Step 1: a random permutation), pairs positions
(2m, 2m+1), and for each pair draws gamma = floor(p) + 1 with probability
p - floor(p), else floor(p) (Step 3, gamma = ceil(p - phi) with phi ~ U[0,1)),
capped at floor(xi_j / xi_k) (eq. (gamma2)), then updates the pair by
eqs. (coal_attr_0)/(coal).  The exact distribution of the state after one
step is therefore a finite sum: all n! orders (each 1/n!) times all
2^floor(n/2) gamma outcomes (weights frac(p) and 1 - frac(p)).  It is built
here from those definitions -- the update written out from the equations in
Python, independently of the oracle's C -- and the oracle's step, run on many
independent copies of the cell at once (one cell index each, so each draws its
own random numbers), must produce outcomes inside that support with the
exact frequencies (chi-square).  Cells below 257 SDs are shuffled by sorting
random keys under both shuffle contracts, so both are run.

The designs include ties (the first SD of the pair is j), case 2 (xi_j =
gamma~ xi_k), caps that bind (floor(p) >= floor(xi_j/xi_k)), and a removal
(xi_k = 1 in case 2: the SD leaves the list and the cell is compacted stably).
"""
import itertools
import math
from collections import defaultdict

import numpy as np
import pytest
from scipy import stats

import oracle

B = 1500.0           # Golovin constant [1/s]
DT = 1.0

# xi, volumes and the largest p (which sets dV) per design
DESIGNS = {
    4: ([9, 2, 4, 4], [2.0e-15, 3.0e-14, 8.0e-15, 1.1e-13], 1.6),
    5: ([1, 1, 3, 2, 9], [4.0e-14, 2.0e-15, 9.0e-14, 5.0e-15, 1.5e-15], 2.6),
    6: ([12, 4, 4, 3, 7, 2], [3.0e-15, 1.2e-13, 5.0e-14, 2.0e-15, 8.0e-14, 6.0e-15], 2.6),
    7: ([8, 2, 5, 5, 3, 11, 4], [9.0e-14, 2.5e-15, 4.0e-14, 6.5e-15, 1.0e-13, 1.5e-15, 3.5e-14], 2.6),
    8: ([12, 4, 4, 3, 7, 2, 9, 6], [3.0e-15, 1.2e-13, 5.0e-14, 2.0e-15, 8.0e-14, 6.0e-15, 1.6e-15, 4.4e-14], 2.6),
}
CELLS = {4: 60000, 5: 100000, 6: 150000, 7: 250000, 8: 400000}


def _scale(n):
    # ratio of all pairs to candidate pairs, eq. (p): ((n^2 - n) / 2) / floor(n / 2)
    return float(n * (n - 1) // 2) / float(n // 2)


def _p(xi, v, a, c, n, dv):
    # eq. (p): a(v_a, v_c) * max(xi) * scale * dt / dV, in the oracle's documented order
    K = B * (v[a] + v[c])
    return ((K * float(max(xi[a], xi[c]))) * _scale(n)) * (DT / dv)


def _update(xi, v, first, second, gamma):
    """eqs. (coal_attr_0)/(coal): j is the SD of larger multiplicity (the first on a tie)."""
    j, k = (first, second) if xi[first] >= xi[second] else (second, first)
    g = min(gamma, xi[j] // xi[k])
    if g == 0:
        return
    if xi[j] - g * xi[k] > 0:                     # case 1
        xi[j] -= g * xi[k]
        v[k] = float(g) * v[j] + v[k]
    else:                                         # case 2
        half = xi[k] // 2
        xi[j], xi[k] = half, xi[k] - half
        v[j] = float(g) * v[j] + v[k]
        v[k] = v[j]


def _compact(xi, v):
    live = [i for i in range(len(xi)) if xi[i] != 0]
    n_dead = len(xi) - len(live)
    return tuple([xi[i] for i in live] + [0] * n_dead), tuple([v[i] for i in live] + [0.0] * n_dead)


def exact_distribution(xi0, v0, dv):
    n = len(xi0)
    oriented = defaultdict(int)
    for perm in itertools.permutations(range(n)):
        oriented[frozenset((perm[2 * m], perm[2 * m + 1]) for m in range(n // 2))] += 1
    total = math.factorial(n)
    dist = defaultdict(float)
    for pairs, cnt in oriented.items():
        pairs = sorted(pairs)
        opts = []
        for a, c in pairs:
            p = _p(xi0, v0, a, c, n, dv)
            fl = math.floor(p)
            f = p - fl
            opts.append([(fl, 1.0 - f), (fl + 1, f)])
        for choice in itertools.product(*opts):
            w = cnt / total
            xi, v = list(xi0), list(v0)
            for (a, c), (g, pw) in zip(pairs, choice):
                w *= pw
                _update(xi, v, a, c, g)
            if w > 0:
                dist[_compact(xi, v)] += w
    return dist


def _dv_for(xi, v, n, pmax):
    worst = max(B * (v[a] + v[c]) * max(xi[a], xi[c]) * _scale(n) * DT for a in range(n) for c in range(n) if a != c)
    return worst / pmax


@pytest.mark.parametrize("shuffle", ["prp", "sort"])
@pytest.mark.parametrize("n", sorted(DESIGNS))
def test_one_step_distribution_matches_enumeration(n, shuffle):
    xi0, v0, pmax = DESIGNS[n]
    dv = _dv_for(xi0, v0, n, pmax)
    ps = [_p(xi0, v0, a, c, n, dv) for a in range(n) for c in range(n) if a != c]
    # the design exercises fractional gammas below and above 1
    assert max(ps) > 1.5 and min(ps) < 0.5
    # the p the oracle computes is the one written above
    for a, c in [(0, 1), (n - 1, 0), (1, 2)]:
        assert oracle.pair_prob(oracle.kernel(0, v0[a], v0[c], B), xi0[a], xi0[c], oracle.pair_scale(n), DT, dv) \
            == _p(xi0, v0, a, c, n, dv)
    exact = exact_distribution(xi0, v0, dv)
    assert abs(sum(exact.values()) - 1.0) < 1e-12
    n_cells = CELLS[n]
    cs = np.arange(n_cells + 1, dtype=np.uint32) * n
    sysm = oracle.System(np.tile(np.array(xi0, np.uint64), n_cells), np.tile(np.array(v0), n_cells)[None, :], cs,
                         dv, 0, B, shuffle)
    sysm.step(DT, 2024 + n, 3)
    X = sysm.xi.reshape(n_cells, n)
    V = sysm.v.reshape(n_cells, n)
    observed = defaultdict(int)
    for row_x, row_v in zip(map(tuple, X.tolist()), map(tuple, V.tolist())):
        observed[(row_x, row_v)] += 1
    outside = [k for k in observed if k not in exact]
    assert not outside, f"{len(outside)} outcomes outside the exact support, e.g. {outside[0]}"
    keys = sorted(exact, key=lambda k: -exact[k])
    big = [k for k in keys if exact[k] * n_cells >= 5.0]
    f_exp = [exact[k] * n_cells for k in big]
    f_obs = [observed.get(k, 0) for k in big]
    rest_exp = n_cells - sum(f_exp)
    if rest_exp > 1e-9:
        f_exp.append(rest_exp)
        f_obs.append(n_cells - sum(f_obs))
    assert len(big) >= 8
    chi2, pval = stats.chisquare(f_obs, f_exp)
    assert pval > 1e-4, (n, shuffle, chi2, pval, len(big))


def test_enumeration_detects_a_biased_pairing():
    """Power of the test above: a step that paired the list in slot order (no shuffle), run on
    the same number of cells, would give a chi-square far beyond any plausible value -- here
    computed from its expected counts against the exact distribution."""
    n = 8
    xi0, v0, pmax = DESIGNS[n]
    dv = _dv_for(xi0, v0, n, pmax)
    exact = exact_distribution(xi0, v0, dv)
    fixed = defaultdict(float)               # outcomes of the fixed pairing (0,1), (2,3), ...
    pairs = [(2 * m, 2 * m + 1) for m in range(n // 2)]
    opts = []
    for a, c in pairs:
        p = _p(xi0, v0, a, c, n, dv)
        fl = math.floor(p)
        opts.append([(fl, 1.0 - (p - fl)), (fl + 1, p - fl)])
    for choice in itertools.product(*opts):
        xi, v = list(xi0), list(v0)
        w = 1.0
        for (a, c), (g, pw) in zip(pairs, choice):
            w *= pw
            _update(xi, v, a, c, g)
        if w > 0:
            fixed[_compact(xi, v)] += w
    n_cells = CELLS[n]
    big = [k for k in exact if exact[k] * n_cells >= 5.0]
    f_exp = np.array([exact[k] * n_cells for k in big])
    f_biased = np.array([fixed.get(k, 0.0) * n_cells for k in big])
    chi2 = float(np.sum((f_biased - f_exp) ** 2 / f_exp))
    assert stats.chi2.sf(chi2, len(big) - 1) < 1e-100


def test_compaction_keeps_slot_order():
    """Step 0 (removal of xi = 0 SDs) keeps the survivors of each cell in slot order and clears
    the freed slots: dead slots scattered through three cells, a marker attribute per slot."""
    rng = np.random.default_rng(3)
    counts = [7, 12, 5]
    n = sum(counts)
    xi = rng.integers(1, 100, n).astype(np.uint64)
    xi[[1, 2, 6, 8, 13, 14, 15, 20]] = 0
    marker = np.arange(n, dtype=np.float64) + 1.0
    attr = np.vstack([rng.random(n) * 1e-12, marker])
    cs = np.r_[0, np.cumsum(counts)].astype(np.uint32)
    s = oracle.System(xi, attr, cs, 1.0, 0, B)
    for c in range(3):
        lo, hi = int(cs[c]), int(cs[c + 1])
        live = [i for i in range(lo, hi) if xi[i] != 0]
        k = len(live)
        assert list(s.attr[1, lo:lo + k]) == [marker[i] for i in live]       # order kept
        assert list(s.xi[lo:lo + k]) == [xi[i] for i in live]
        assert not s.xi[lo + k:hi].any() and not s.attr[:, lo + k:hi].any()   # freed slots cleared


def test_step_with_removals_leaves_live_prefixes():
    """After a step that removes SDs (pairs of multiplicity 1 in case 2) every cell's live SDs
    are a prefix of its slots and the total number of droplets fell by the coalescences."""
    rng = np.random.default_rng(8)
    counts = [40, 300, 9]
    n = sum(counts)
    xi = rng.integers(1, 3, n).astype(np.uint64)
    v = rng.random(n) * 1e-13 + 1e-14
    cs = np.r_[0, np.cumsum(counts)].astype(np.uint32)
    s = oracle.System(xi, v, cs, 1e-10, 0, B, "prp")
    tot0 = int(s.xi.sum())
    st = s.step(DT, 5, 0)
    assert st["n_removed"] > 10
    for c in range(3):
        w = s.xi[cs[c]:cs[c + 1]]
        nz = np.flatnonzero(w)
        assert len(nz) == 0 or nz[-1] == len(nz) - 1
    assert int(s.xi.sum()) < tot0
