"""Pins of the CPU oracle against things other than itself.

* Philox4x32-10 against torch's independent header implementation
  (at::philox_engine), compiled and run here.
* Single-pair updates against the paper's worked example (Sec. 2.2) and cases
  worked by hand from eqs. (gamma2), (coal_attr_0), (coal).
* gamma = ceil(p - phi) against exact rational arithmetic (reading of Step 3).
* The pair-count ratio of eq. (p) against its closed form.
* Cube root, terminal velocity, efficiency table against libm, hand values and
  continuity / node properties.
"""
import json
import math
import os
import subprocess
from fractions import Fraction

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
TORCH_INC = None


def _torch_include():
    import torch
    return os.path.join(os.path.dirname(torch.__file__), "include")


@pytest.fixture(scope="module")
def torch_philox(tmp_path_factory):
    """Compile a tiny program around torch's at::philox_engine (known-answer source)."""
    d = tmp_path_factory.mktemp("kat")
    src = d / "kat.cpp"
    src.write_text(
        "#include <ATen/core/PhiloxRNGEngine.h>\n#include <cstdio>\n#include <cstdlib>\n"
        "int main(int argc, char** argv) {\n"
        "  for (int a = 1; a + 2 < argc; a += 3) {\n"
        "    at::philox_engine e(strtoull(argv[a],0,0), strtoull(argv[a+1],0,0), strtoull(argv[a+2],0,0));\n"
        "    for (int i = 0; i < 4; ++i) printf(\"%u \", e());\n    printf(\"\\n\");\n  }\n}\n")
    exe = d / "kat"
    subprocess.check_call(["g++", "-std=c++17", "-O1", "-I", _torch_include(), "-o", str(exe), str(src)])

    def run(cases):
        args = []
        for seed, sub, off in cases:
            args += [str(seed), str(sub), str(off)]
        out = subprocess.check_output([str(exe), *args]).decode().strip().splitlines()
        return [list(map(int, line.split())) for line in out]
    return run


def test_philox_matches_torch_engine(torch_philox):
    # torch's engine: key = (seed lo, seed hi), counter = (offset lo, offset hi, subseq lo, subseq hi)
    rng = np.random.default_rng(1)
    cases = [(0, 0, 0), (42, 7, 123), (2 ** 64 - 1, 2 ** 64 - 1, 2 ** 64 - 1)]
    for _ in range(40):
        cases.append(tuple(int(x) for x in rng.integers(0, 2 ** 63, 3, dtype=np.int64)))
    ref = torch_philox(cases)
    for (seed, sub, off), want in zip(cases, ref):
        ctr = [off & 0xffffffff, off >> 32, sub & 0xffffffff, sub >> 32]
        key = [seed & 0xffffffff, seed >> 32]
        got = oracle.philox(ctr, key)
        assert list(map(int, got)) == want, (seed, sub, off)


def test_rng_contract_words(torch_philox):
    """Shuffle keys and phi are the documented words of the documented counters."""
    seed, cell, step = (7 << 32) | 11, 5, 9
    for l in range(12):
        off = (l >> 2) | (cell << 32)      # c0 = l >> 2, c1 = cell
        sub = step | (0 << 32)             # c2 = step, c3 = purpose 0
        want = torch_philox([(seed, sub, off)])[0][l & 3]
        assert oracle.shuffle_key(seed, cell, step, l) == want
    for m in range(6):
        off = (m >> 1) | (cell << 32)
        sub = step | (1 << 32)             # purpose 1
        x = torch_philox([(seed, sub, off)])[0]
        w = 2 * (m & 1)
        u53 = ((x[w] << 32) | x[w + 1]) >> 11
        assert oracle.phi_u53(seed, cell, step, m) == u53
        assert oracle.phi(seed, cell, step, m) == u53 / 2.0 ** 53


def _load(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def _apply(first, second, p, phi):
    xi = np.array([first[0], second[0]], np.uint64)
    attr = np.array([[first[1], second[1]]], np.float64)
    g = oracle.update_pair(xi, attr, 0, 1, p, phi)
    return g, [int(xi[0]), float(attr[0, 0])], [int(xi[1]), float(attr[0, 1])]


def test_paper_worked_example():
    ex = _load("paper_worked_example.json")
    # gamma = 5 realised as p in [4,5) with phi below the fractional part
    g = oracle.gamma_tilde(4.5, 0.25, ex["xi_j"], ex["xi_k"])
    assert g == ex["gamma_tilde"]
    g, a, b = _apply([ex["xi_j"], ex["A_j"]], [ex["xi_k"], ex["A_k"]], 4.5, 0.25)
    assert g == ex["gamma_tilde"]
    assert a == [ex["xi_j_after"], ex["A_j_after"]]
    assert b == [ex["xi_k_after"], ex["A_k_after"]]


@pytest.mark.parametrize("case", _load("pair_cases.json")["cases"], ids=lambda c: c["name"])
def test_pair_cases(case):
    g, a, b = _apply(case["first"], case["second"], case["p"], case["phi"])
    assert g == case["gamma_tilde"]
    assert a == case["first_after"]
    assert b == case["second_after"]


def test_gamma_floor_form_equals_ceil_p_minus_phi_exactly():
    """gamma = ceil(p - phi) in exact arithmetic equals floor(p) + [phi < frac(p)]."""
    rng = np.random.default_rng(3)
    ps = list(rng.random(300) * 10.0) + list(rng.random(100) * 1e-3) + [0.0, 1.0, 2.5, 3.0, 1e-300]
    for p in ps:
        for phi in list(rng.random(5)) + [0.0, p - math.floor(p)]:
            if not (0.0 <= phi < 1.0):
                continue
            want = math.ceil(Fraction(p) - Fraction(phi))   # exact rational
            cap = 10 ** 6
            assert oracle.gamma_tilde(p, phi, cap, 1) == min(max(want, 0), cap)


def test_gamma_cap_branch():
    # the cap is floor(xi_j/xi_k) in exact integer arithmetic, also beyond 2^53 / 3
    xi_j, xi_k = 2 ** 52 + 3, 3
    assert oracle.gamma_tilde(1e300, 0.5, xi_j, xi_k) == xi_j // xi_k
    assert oracle.gamma_tilde(float("inf"), 0.5, 100, 7) == 14


def test_pair_scale_closed_form():
    """eq. (p): ((n^2 - n)/2) / floor(n/2) is n - 1 for even n and n for odd n."""
    for n in list(range(2, 200)) + [2 ** 20, 2 ** 20 + 1, 123457, 2 ** 31 - 1]:
        want = n - 1 if n % 2 == 0 else n
        assert oracle.pair_scale(n) == float(want)


def test_golovin_kernel_value():
    assert oracle.kernel(0, 1e-12, 3e-12, 1500.0) == 1500.0 * (1e-12 + 3e-12)


def test_cbrt_against_libm_and_exact_cubes():
    rng = np.random.default_rng(5)
    xs = np.exp(rng.uniform(np.log(1e-30), np.log(1e-3), 20000))
    worst = 0
    for x in xs:
        got = oracle.cbrt(float(x))
        ref = np.cbrt(x)
        ulp = np.spacing(ref)
        worst = max(worst, abs(got - ref) / ulp)
    assert worst <= 1.0, worst
    for k in [1, 2, 3, 5, 10, 100, 12345]:
        assert oracle.cbrt(float(k) ** 3) == float(k)
    assert oracle.cbrt(0.125) == 0.5 and oracle.cbrt(2.0 ** -60) == 2.0 ** -20


def test_radius_of_sphere():
    for r in [1e-8, 1e-6, 15e-6, 1e-3]:
        v = 4.0 / 3.0 * math.pi * r ** 3
        assert abs(oracle.radius(v) - r) <= 4e-16 * r


def test_terminal_velocity_regimes_and_continuity():
    k1, k2, k3 = 1.19e8, 8.0e3, 201.0
    # the written-out regime borders are the rounded quotients they stand for
    import ctypes
    assert oracle.terminal_velocity(k2 / k1) == k2 * (k2 / k1)          # linear law from r12 on
    t = k3 / k2
    assert oracle.terminal_velocity(t * t) == k3 * math.sqrt(t * t)     # square-root law from r23 on
    below = np.nextafter(k2 / k1, 0)
    assert oracle.terminal_velocity(below) == (k1 * below) * below
    # hand values, one per regime
    assert oracle.terminal_velocity(10e-6) == pytest.approx(k1 * 1e-10, rel=1e-15)      # 1.19e-2 m/s
    assert oracle.terminal_velocity(200e-6) == pytest.approx(k2 * 2e-4, rel=1e-15)      # 1.6 m/s
    assert oracle.terminal_velocity(2e-3) == pytest.approx(k3 * math.sqrt(2e-3), rel=1e-15)
    # continuity at the regime borders and monotonicity
    r12, r23 = k2 / k1, (k3 / k2) ** 2
    for rb in (r12, r23):
        lo = oracle.terminal_velocity(rb * (1 - 1e-12))
        hi = oracle.terminal_velocity(rb * (1 + 1e-12))
        assert abs(hi - lo) <= 1e-10 * hi
    rs = np.exp(np.linspace(np.log(1e-8), np.log(5e-3), 2000))
    vts = [oracle.terminal_velocity(r) for r in rs]
    assert all(b >= a for a, b in zip(vts, vts[1:]))


EFF_R = [10e-6, 20e-6, 30e-6, 40e-6, 50e-6, 60e-6, 80e-6, 100e-6, 150e-6, 200e-6, 300e-6, 1000e-6]


def test_efficiency_table_properties():
    # node values reproduce the defining smooth form to the table's 3 decimals
    for R in EFF_R:
        for j in range(11):
            q = j / 10
            e = oracle.efficiency(R, q)
            smooth = R * R / (R * R + (25e-6) ** 2) * (1 - (1 - q) ** 2)
            assert abs(e - smooth) <= 5e-4 + 1e-12, (R, q)
            assert 0.0 <= e <= 1.0
    # bilinear: midpoint between nodes is the mean of the four corners
    e00 = oracle.efficiency(EFF_R[3], 0.3)
    e01 = oracle.efficiency(EFF_R[3], 0.4)
    e10 = oracle.efficiency(EFF_R[4], 0.3)
    e11 = oracle.efficiency(EFF_R[4], 0.4)
    mid = oracle.efficiency(0.5 * (EFF_R[3] + EFF_R[4]), 0.35)
    assert mid == pytest.approx(0.25 * (e00 + e01 + e10 + e11), abs=1e-12)
    # clamping outside the radius nodes
    assert oracle.efficiency(1e-7, 0.5) == oracle.efficiency(EFF_R[0], 0.5)
    assert oracle.efficiency(5e-3, 0.5) == oracle.efficiency(EFF_R[-1], 0.5)


def test_gravitational_kernel_symmetry_and_zero_on_diagonal():
    rng = np.random.default_rng(9)
    for _ in range(500):
        v1, v2 = np.exp(rng.uniform(np.log(1e-22), np.log(1e-8), 2))
        a = oracle.kernel(1, v1, v2)
        b = oracle.kernel(1, v2, v1)
        assert a == b and a >= 0.0
        assert oracle.kernel(1, v1, v1) == 0.0
    # closed form at a chosen pair: r1 = 10 um, r2 = 100 um
    r1, r2 = 10e-6, 100e-6
    v1, v2 = 4 / 3 * math.pi * r1 ** 3, 4 / 3 * math.pi * r2 ** 3
    vt1, vt2 = 1.19e8 * r1 * r1, 8.0e3 * r2
    E = 0.179  # table node R = 100 um, q = 0.1
    want = math.pi * (r1 + r2) ** 2 * abs(vt2 - vt1) * E
    assert oracle.kernel(1, v1, v2) == pytest.approx(want, rel=1e-12)


def test_spectrum_is_the_exactly_summed_definition():
    """Sec. 4 mass spectrum: per bin rho * sum(xi v) / (V dln r), the sum taken exactly over the
    bin's terms (each xi v rounded once) and rounded once -- checked against exact rational
    arithmetic (fractions.Fraction, whose float() rounds correctly), on terms of very different
    magnitudes, with volumes on bin edges (an edge belongs to the bin above it), dead slots and a
    cell range."""
    from fractions import Fraction
    rng = np.random.default_rng(7)
    r_edges = np.exp(np.linspace(np.log(1e-6), np.log(5e-3), 41))
    ve = ((oracle.FOUR_PI_OVER_THREE * r_edges) * r_edges) * r_edges
    counts = [300, 0, 500, 200]
    n = sum(counts)
    v = np.exp(rng.uniform(np.log(ve[0] * 0.5), np.log(ve[-1] * 1.5), n))
    v[:40] = ve[rng.integers(0, len(ve), 40)]                      # exactly on edges
    xi = np.floor(np.exp(rng.uniform(0, np.log(2.0 ** 52), n))).astype(np.uint64) + 1
    xi[rng.random(n) < 0.1] = 0
    cs = np.r_[0, np.cumsum(counts)].astype(np.uint32)
    dv = np.array([1.5e3, 2.0e3, 0.7e3, 1.1e3])
    s = oracle.System(xi, v, cs, dv)
    for lo, hi in ((0, 4), (2, 3)):
        got = s.spectrum(r_edges, cell_lo=lo, cell_hi=hi)
        a, b = int(s.cell_start[lo]), int(s.cell_start[hi])
        V = 0.0
        for c in range(lo, hi):
            V += float(dv[c])
        exact = [Fraction(0)] * (len(r_edges) - 1)
        for i in range(a, b):
            x, vi = int(s.xi[i]), float(s.v[i])
            if x == 0 or not (ve[0] <= vi < ve[-1]):
                continue
            k = max(j for j in range(len(ve) - 1) if ve[j] <= vi)
            exact[k] += Fraction(float(x) * vi)                        # the term, rounded once
        for k in range(len(exact)):
            dlnr = math.log(r_edges[k + 1]) - math.log(r_edges[k])
            assert got[k] == 1000.0 * float(exact[k]) / (V * dlnr), k
