"""Statistical and exhaustive pins of the oracle's whole step.

* Pairing is a uniform random set of floor(n/2) non-overlapping pairs
  (Sec. 2.2 Step 1): chi-square over all pairings for n = 4 and n = 5.
* Expected number of real-droplet coalescences per step equals
  sum_{i<j} a(v_i, v_j) xi_i xi_j dt / dV when every p < 1 -- the identity the
  up-scaling of eq. (p) is built to satisfy (Sec. 2.2 Step 2).
* Exact outcome distribution of a 3-SD cell (one candidate pair, any p) by
  enumeration: pair chosen uniformly, gamma = floor(p) + 1 with probability
  frac(p) (Step 3).
* Golovin closed forms (Sec. 4): I1e against scipy.special.ive and the
  analytic pdf's normalisation and mass (the SDM's number and spectrum against
  them, one ensemble per shuffle contract, are in test_oracle_prp_pins.py).
"""
import math
from collections import Counter

import numpy as np
import pytest
from scipy import special, stats

import oracle
from paper_2101_06318_b300 import inputs


SHUFFLES = ["sort", "prp"]


def _one_cell(xi, v, dv, kernel_id=0, b=1500.0, shuffle="prp"):
    n = len(xi)
    return oracle.System(np.array(xi, np.uint64), np.array(v, np.float64), [0, n], dv, kernel_id, b, shuffle)


def _pairing_after_one_step(n, seed, step, shuffle):
    # equal xi = 2: every selected pair collides (p huge) with gamma~ = 1 and case 2,
    # so both partners end with v_i + v_partner; unpaired SDs are unchanged.
    v = np.array([(i + 1) * 1e-12 for i in range(n)])
    s = _one_cell([2] * n, v, dv=1e-30, shuffle=shuffle)
    s.step(1.0, seed, step)
    pairs = set()
    for i in range(n):
        if s.xi[i] == 2:
            continue
        partner = int(round((s.v[i] - v[i]) / 1e-12)) - 1
        pairs.add(tuple(sorted((i, partner))))
    return tuple(sorted(pairs))


@pytest.mark.parametrize("shuffle", SHUFFLES)
@pytest.mark.parametrize("n,n_pairings", [(4, 3), (5, 15), (6, 15)])   # small cells: both shuffles sort
def test_pairing_is_uniform(n, n_pairings, shuffle):
    trials = 300 * n_pairings
    cnt = Counter(_pairing_after_one_step(n, 1234, s, shuffle) for s in range(trials))
    assert len(cnt) == n_pairings
    for pairing in cnt:
        flat = [i for p in pairing for i in p]
        assert len(flat) == len(set(flat)) == 2 * (n // 2)
    chi2, pval = stats.chisquare(list(cnt.values()))
    assert pval > 1e-4, (chi2, pval, cnt)


@pytest.mark.parametrize("shuffle", SHUFFLES)
def test_expected_coalescences_match_all_pairs_sum(shuffle):
    rng = np.random.default_rng(11)
    n = 6
    xi = rng.integers(1000, 10 ** 6, n).astype(np.uint64)
    v = np.exp(rng.uniform(np.log(1e-15), np.log(1e-13), n))
    b, dt = 1500.0, 1.0
    # choose dV so that the largest p is 0.5 (no cap binds: gamma <= 1 <= cap)
    S = n - 1
    pmax = max(b * (v[i] + v[j]) * max(xi[i], xi[j]) * S * dt for i in range(n) for j in range(i + 1, n))
    dv = pmax / 0.5
    want = sum(b * (v[i] + v[j]) * float(xi[i]) * float(xi[j]) * dt / dv
               for i in range(n) for j in range(i + 1, n))
    base = _one_cell(xi, v, dv, 0, b, shuffle)
    tot0 = int(base.xi.sum())
    trials = 40000
    d = np.empty(trials)
    for s in range(trials):
        sys_ = base.copy()
        sys_.step(dt, 77, s)
        d[s] = tot0 - int(sys_.xi.sum())
    mean, sem = d.mean(), d.std(ddof=1) / math.sqrt(trials)
    assert abs(mean - want) < 5 * sem, (mean, want, sem)


@pytest.mark.parametrize("shuffle", SHUFFLES)
def test_three_sd_cell_exact_distribution(shuffle):
    xi = [9, 4, 6]
    v = [3e-14, 5e-14, 1e-14]
    b, dt, dv = 1500.0, 1.0, 1.3e-9
    n = 3
    scale = oracle.pair_scale(n)
    assert scale == 3.0
    # exact distribution of the final (xi, v) over pairings x gamma outcomes
    exact = Counter()
    ps = []
    for a, c in [(0, 1), (0, 2), (1, 2)]:
        K = oracle.kernel(0, v[a], v[c], b)
        p = oracle.pair_prob(K, xi[a], xi[c], scale, dt, dv)
        ps.append(p)
        fl = math.floor(p)
        for extra, w in [(0, 1.0 - (p - fl)), (1, p - fl)]:
            # realise gamma = fl + extra with a phi on the right side of frac(p)
            phi = 0.999999 if extra == 0 else 0.0
            x = np.array(xi, np.uint64)
            at = np.array([v], np.float64)
            oracle.update_pair(x, at, a, c, p, phi)
            exact[(tuple(int(t) for t in x), tuple(at[0]))] += w / 3.0
    assert 0.1 < min(p - math.floor(p) for p in ps) and max(ps) > 1.0   # non-trivial case
    trials = 30000
    mc = Counter()
    for s in range(trials):
        sys_ = _one_cell(xi, v, dv, 0, b, shuffle)
        sys_.step(dt, 99, s)
        mc[(tuple(int(t) for t in sys_.xi), tuple(sys_.v))] += 1
    assert set(mc) <= set(exact)
    keys = sorted(exact)
    f_obs = np.array([mc.get(k, 0) for k in keys], float)
    f_exp = np.array([exact[k] * trials for k in keys])
    chi2, pval = stats.chisquare(f_obs, f_exp)
    assert pval > 1e-4, (chi2, pval)


# --------------------------------------------------------------------------
# Golovin analytic solution
# --------------------------------------------------------------------------

def test_i1e_against_scipy():
    xs = np.concatenate([np.exp(np.linspace(np.log(1e-8), np.log(1e8), 4000)), [29.9, 30.0, 30.1]])
    for x in xs:
        ref = special.ive(1, x)
        assert abs(oracle.i1e(x) - ref) <= 2e-14 * abs(ref), x


def test_golovin_pdf_initial_condition_and_moments():
    vbar, n0, b = inputs.GOLOVIN_VBAR, inputs.GOLOVIN_N0, inputs.GOLOVIN_B
    for v in [1e-15, 1e-13, 1e-12]:
        assert oracle.golovin_phi(v, 0.0, vbar, n0, b) == pytest.approx(math.exp(-v / vbar) / vbar, rel=1e-15)
    # integral of phi is 1 - tau (number), integral of v phi is vbar (mass conserved)
    v = np.exp(np.linspace(np.log(1e-20), np.log(1e-5), 40000))
    for t in [10.0, 1200.0, 3600.0]:
        tau = 1 - math.exp(-n0 * b * vbar * t)
        f = np.array([oracle.golovin_phi(x, t, vbar, n0, b) for x in v])
        num = np.trapezoid(f * v, np.log(v))
        mass = np.trapezoid(f * v * v, np.log(v))
        assert num == pytest.approx(1 - tau, rel=2e-3)
        assert mass == pytest.approx(vbar, rel=2e-3)


# --------------------------------------------------------------------------
# the keyed bijection of the PRP shuffle
# --------------------------------------------------------------------------

def test_prp_is_a_bijection():
    rng = np.random.default_rng(4)
    for n in list(range(2, 70)) + [127, 128, 129, 1000, 4097]:
        K = oracle.prp_keys(int(rng.integers(0, 2 ** 63)), int(rng.integers(0, 1000)), int(rng.integers(0, 1000)))
        img = [oracle.prp(q, n, K) for q in range(n)]
        assert sorted(img) == list(range(n)), n
    # a large n, sampled: distinct and inside [0, n)
    n = (1 << 20) + 12345
    K = oracle.prp_keys(42, 0, 7)
    qs = rng.choice(n, 20000, replace=False)
    img = [oracle.prp(int(q), n, K) for q in qs]
    assert len(set(img)) == len(img) and max(img) < n


@pytest.mark.parametrize("n", [257, 300, 1024, 4097])
def test_prp_pairs_look_like_a_uniform_random_matching(n):
    """For a uniform random matching of n items the distance |i - j| of a pair follows
    P(d) = 2 (n - d) / (n (n - 1)) and the partner of a fixed item is uniform over the
    others; chi-square on integer-aligned bins of both."""
    steps = max(200, 400000 // n)
    dist = np.zeros(n, np.int64)
    partner_of_0 = []
    for step in range(steps):
        K = oracle.prp_keys(7, 3, step)
        img = [oracle.prp(q, n, K) for q in range(n)]
        for m in range(n // 2):
            dist[abs(img[2 * m] - img[2 * m + 1])] += 1
        pos0 = img.index(0)
        if pos0 ^ 1 < n:
            partner_of_0.append(img[pos0 ^ 1])
    d = np.arange(1, n)
    pd = 2.0 * (n - d) / (n * (n - 1))
    cut = np.r_[0, np.unique(np.searchsorted(np.cumsum(pd), np.linspace(0, 1, 31)[1:-1]))]
    obs = np.add.reduceat(dist[1:], cut)
    exp = np.add.reduceat(pd, cut)
    exp = exp * obs.sum() / exp.sum()
    assert stats.chisquare(obs, exp).pvalue > 1e-4
    p0 = np.bincount(np.array(partner_of_0) * 16 // n, minlength=16)
    assert stats.chisquare(p0).pvalue > 1e-4
