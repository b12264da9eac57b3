"""Pins of the oracle's electric-field kernel (project definition).

Sec. 4 names a parametric kernel for electric-field effects on the collision
probability (Berry's case) without giving it.  The project defines it as the
gravitational kernel with the collision efficiency raised toward one by a field
parameter eps in [0, 1]: E_eps = E + eps (1 - E).  What fixes it:

* eps = 0 is the gravitational kernel itself (bit for bit);
* eps = 1 is the geometric sweep-out kernel pi (r1 + r2)^2 |vt1 - vt2| (every
  geometric encounter coalesces), to rounding;
* at the table's nodes E_eps is the node value raised by eps (1 - value);
* E_eps lies in [eps, 1] and grows with eps; the kernel is symmetric and zero
  for equal volumes;
* through a whole step, the expected number of coalescences equals
  sum_{i<j} a_eps(v_i, v_j) xi_i xi_j dt / dV (eq. (p)), so the step uses
  the field parameter it is given.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2101_06318_b300 import inputs

R_NODES = [10e-6, 20e-6, 30e-6, 40e-6, 50e-6, 60e-6, 80e-6, 100e-6, 150e-6, 200e-6, 300e-6, 1000e-6]


def _pairs(n, seed):
    rng = np.random.default_rng(seed)
    r1 = np.exp(rng.uniform(np.log(1e-6), np.log(2e-3), n))
    r2 = np.exp(rng.uniform(np.log(1e-6), np.log(2e-3), n))
    return 4 / 3 * np.pi * r1 ** 3, 4 / 3 * np.pi * r2 ** 3


def test_zero_field_is_the_gravitational_kernel():
    v1, v2 = _pairs(3000, 1)
    for a, b in zip(v1, v2):
        assert oracle.kernel(2, a, b, efield=0.0) == oracle.kernel(1, a, b)


def test_full_field_is_the_geometric_sweep_out_kernel():
    v1, v2 = _pairs(3000, 2)
    for a, b in zip(v1, v2):
        r1, r2 = oracle.radius(a), oracle.radius(b)
        sweep = math.pi * (r1 + r2) ** 2 * abs(oracle.terminal_velocity(r1) - oracle.terminal_velocity(r2))
        assert oracle.kernel(2, a, b, efield=1.0) == pytest.approx(sweep, rel=4e-16 * 8, abs=0.0)


def test_node_values_raised_by_the_field():
    for i, R in enumerate(R_NODES):
        for j in range(11):
            q = j / 10.0
            E = oracle.efficiency(R, q)
            for eps in (0.0, 0.25, 0.5, 1.0):
                want = E + eps * (1.0 - E)
                got = oracle.efficiency_field(R, q, eps)
                assert got == pytest.approx(want, rel=0, abs=2.3e-16), (R, q, eps)
    # one node by hand: R = 50 um, q = 0.5 holds 0.600, so eps = 0.5 gives 0.8
    assert oracle.efficiency_field(50e-6, 0.5, 0.5) == pytest.approx(0.8, abs=2.3e-16)


def test_bounds_monotonicity_symmetry_diagonal():
    v1, v2 = _pairs(1500, 3)
    rng = np.random.default_rng(4)
    for a, b in zip(v1, v2):
        ks = [oracle.kernel(2, a, b, efield=e) for e in (0.0, 0.1, 0.5, 0.9, 1.0)]
        assert all(x <= y for x, y in zip(ks, ks[1:]))
        assert oracle.kernel(2, a, b, efield=0.3) == oracle.kernel(2, b, a, efield=0.3)
        assert oracle.kernel(2, a, a, efield=0.7) == 0.0
        R, q = rng.uniform(5e-6, 2e-3), rng.uniform(0.0, 1.0)
        eps = rng.uniform(0.0, 1.0)
        E = oracle.efficiency_field(R, q, eps)
        assert eps - 1e-15 <= E <= 1.0 + 2.3e-16


@pytest.mark.parametrize("eps", [0.3, 1.0])
def test_expected_coalescences_with_the_field(eps):
    n, n_cells = 300, 4000
    rng = np.random.default_rng(11)
    v = np.sort(inputs.lognormal_volumes(rng, n, 15e-6, 1.6))
    xi = rng.integers(1000, 10 ** 6, n).astype(np.uint64)
    xf = xi.astype(np.float64)
    K = np.array([[oracle.kernel(2, v[i], v[j], efield=eps) if i < j else 0.0 for j in range(n)] for i in range(n)])
    S = oracle.pair_scale(n)
    dv = float(np.max(K * np.maximum.outer(xf, xf))) * S / 0.5
    want = float(np.sum(K * np.outer(xf, xf))) / dv
    K0 = np.array([[oracle.kernel(1, v[i], v[j]) if i < j else 0.0 for j in range(n)] for i in range(n)])
    want0 = float(np.sum(K0 * np.outer(xf, xf))) / dv       # what a step ignoring the field would expect
    cs = np.arange(n_cells + 1, dtype=np.uint32) * n
    s = oracle.System(np.tile(xi, n_cells), np.tile(v, n_cells)[None, :], cs, dv, 2, 1500.0, "prp", efield=eps)
    s.step(1.0, 5, 0)
    d = np.tile(xf, n_cells).reshape(n_cells, n).sum(1) - s.xi.reshape(n_cells, n).astype(np.float64).sum(1)
    mean, sem = d.mean(), d.std(ddof=1) / math.sqrt(n_cells)
    assert abs(mean - want) < 4.5 * sem, (mean, want, sem)
    assert abs(want - want0) > 20 * sem
