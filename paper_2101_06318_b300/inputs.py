"""Seeded synthetic initial states for the SDM coalescence workloads.

This module only draws initial super-droplet populations (multiplicities xi,
volumes v, cell layout, per-cell dV and kernel choice).  It holds none of the
method's arithmetic and imports neither the CUDA binding nor the oracle, so
both sides (and the benchmark) can start from the same arrays.

Workloads (sizes as given by the workload definitions; ``scale`` shrinks them
for tests):

* ``golovin_box``   -- Sec. 4 of the paper: one cell, V = 1e6 m^3,
  N0 = 2^23 m^-3, exponential volume pdf with mean vbar = 4/3 pi (30.531 um)^3,
  equal multiplicities, each SD one quantile of the distribution between the
  0.001 % and 99.999 % points (quantile points at the bin centres), Golovin
  kernel b = 1500 1/s, dt = 1 s.  Default n_sd = 2^13.
* ``gravitational_box`` -- one cell, n_sd = 2^20, radii lognormal (median
  15 um, sigma_g = 1.4), n0 = 1e8 m^-3, dV = 1e6 m^3, gravitational kernel.
* ``grid_bimodal``  -- 256 x 256 cells of dV = 1e3 m^3, SDs per cell
  Poisson(128), each SD from mode A (0.05 um, sigma_g 1.5) or B (10 um,
  sigma_g 1.3) with probability 1/2, n0 = 1e8 m^-3, gravitational kernel.
* ``ensemble``      -- 1024 independent boxes (one cell each) with
  n_sd = floor(2^(10 + 6u)), u ~ U[0,1); even members Golovin (as
  golovin_box), odd members gravitational (as gravitational_box).
* ``grid_lognormal`` -- 256 x 256 cells of dV = 1e3 m^3, Poisson(256) SDs per
  cell, lognormal 15 um / 1.4, n0 = 1e8 m^-3.
"""
from __future__ import annotations

import math

import numpy as np

GOLOVIN = 0
GRAVITATIONAL = 1

FOUR_PI_OVER_THREE = 4.0 * math.pi / 3.0
GOLOVIN_VBAR = FOUR_PI_OVER_THREE * (30.531e-6) ** 3
GOLOVIN_N0 = 2.0 ** 23
GOLOVIN_DV = 1.0e6
GOLOVIN_B = 1500.0


def _state(xi, v, counts, dv, kernel_id, name, dt=1.0, golovin_b=GOLOVIN_B, **meta):
    counts = np.asarray(counts, np.int64)
    cell_start = np.zeros(len(counts) + 1, np.uint32)
    cell_start[1:] = np.cumsum(counts)
    return {
        "name": name,
        "xi": np.ascontiguousarray(xi, np.uint64),
        "v": np.ascontiguousarray(v, np.float64),
        "cell_start": cell_start,
        "dv": np.ascontiguousarray(np.broadcast_to(np.asarray(dv, np.float64), (len(counts),))),
        "kernel_id": np.ascontiguousarray(np.broadcast_to(np.asarray(kernel_id, np.uint8), (len(counts),))),
        "dt": float(dt),
        "golovin_b": float(golovin_b),
        "meta": meta,
    }


def golovin_volumes(n_sd, vbar=GOLOVIN_VBAR):
    """Quantile points of the exponential pdf between 1e-5 and 1 - 1e-5."""
    i = np.arange(n_sd, dtype=np.float64)
    q = 1e-5 + (i + 0.5) * (1.0 - 2e-5) / n_sd
    return -vbar * np.log1p(-q)


def golovin_box(n_sd=2 ** 13, dv=GOLOVIN_DV, n0=GOLOVIN_N0):
    xi_val = n0 * dv / n_sd
    xi = np.full(n_sd, int(round(xi_val)), np.uint64)
    v = golovin_volumes(n_sd)
    return _state(xi, v, [n_sd], dv, GOLOVIN, "golovin_box", n0=n0, vbar=GOLOVIN_VBAR, n_sd=n_sd)


def lognormal_volumes(rng, n, r_median, sigma_g):
    z = rng.standard_normal(n)
    r = r_median * np.power(sigma_g, z)
    return FOUR_PI_OVER_THREE * r ** 3


def gravitational_box(n_sd=2 ** 20, seed=42, n0=1.0e8, dv=1.0e6):
    rng = np.random.default_rng(seed)
    v = lognormal_volumes(rng, n_sd, 15e-6, 1.4)
    xi = np.full(n_sd, max(1, int(round(n0 * dv / n_sd))), np.uint64)
    return _state(xi, v, [n_sd], dv, GRAVITATIONAL, "gravitational_box", n0=n0, n_sd=n_sd, seed=seed)


def grid_bimodal(nx=256, ny=256, mean_per_cell=128, seed=42, n0=1.0e8, dv=1.0e3):
    rng = np.random.default_rng(seed)
    n_cell = nx * ny
    counts = rng.poisson(mean_per_cell, n_cell).astype(np.int64)
    n = int(counts.sum())
    mode_b = rng.random(n) < 0.5
    z = rng.standard_normal(n)
    r = np.where(mode_b, 10e-6 * np.power(1.3, z), 0.05e-6 * np.power(1.5, z))
    v = FOUR_PI_OVER_THREE * r ** 3
    per_cell_xi = np.maximum(1, np.rint(n0 * dv / np.maximum(counts, 1))).astype(np.uint64)
    xi = np.repeat(per_cell_xi, counts)
    return _state(xi, v, counts, dv, GRAVITATIONAL, "grid_bimodal", n0=n0, nx=nx, ny=ny,
                  mean_per_cell=mean_per_cell, seed=seed)


def ensemble(n_members=1024, log2_lo=10, log2_hi=16, seed=42):
    rng = np.random.default_rng(seed)
    u = rng.random(n_members)
    counts = np.floor(np.power(2.0, log2_lo + (log2_hi - log2_lo) * u)).astype(np.int64)
    xis, vs, dvs, kids = [], [], [], []
    for m, n in enumerate(counts):
        if m % 2 == 0:
            xis.append(np.full(n, int(round(GOLOVIN_N0 * GOLOVIN_DV / n)), np.uint64))
            vs.append(golovin_volumes(int(n)))
            dvs.append(GOLOVIN_DV)
            kids.append(GOLOVIN)
        else:
            xis.append(np.full(n, max(1, int(round(1.0e8 * 1.0e6 / n))), np.uint64))
            vs.append(lognormal_volumes(rng, int(n), 15e-6, 1.4))
            dvs.append(1.0e6)
            kids.append(GRAVITATIONAL)
    return _state(np.concatenate(xis), np.concatenate(vs), counts, np.array(dvs), np.array(kids, np.uint8),
                  "ensemble", n_members=n_members, seed=seed)


def grid_lognormal(nx=256, ny=256, mean_per_cell=256, seed=42, n0=1.0e8, dv=1.0e3):
    rng = np.random.default_rng(seed)
    n_cell = nx * ny
    counts = rng.poisson(mean_per_cell, n_cell).astype(np.int64)
    n = int(counts.sum())
    v = lognormal_volumes(rng, n, 15e-6, 1.4)
    per_cell_xi = np.maximum(1, np.rint(n0 * dv / np.maximum(counts, 1))).astype(np.uint64)
    xi = np.repeat(per_cell_xi, counts)
    return _state(xi, v, counts, dv, GRAVITATIONAL, "grid_lognormal", n0=n0, nx=nx, ny=ny,
                  mean_per_cell=mean_per_cell, seed=seed)


def random_cells(n_cell, mean_per_cell, seed, kernel_mix=True, dead_fraction=0.0, xi_max=10 ** 9,
                 dv=1.0e3, min_per_cell=0):
    """Small irregular multi-cell states for parity tests: Poisson cell sizes
    (with a minimum), log-uniform xi in [1, xi_max], lognormal volumes, a mix
    of kernels, and optionally some dead (xi = 0) slots."""
    rng = np.random.default_rng(seed)
    counts = np.maximum(rng.poisson(mean_per_cell, n_cell), min_per_cell).astype(np.int64)
    n = int(counts.sum())
    xi = np.floor(np.exp(rng.random(n) * math.log(xi_max))).astype(np.uint64)
    xi = np.maximum(xi, 1).astype(np.uint64)
    if dead_fraction > 0:
        xi[rng.random(n) < dead_fraction] = 0
    v = lognormal_volumes(rng, n, 12e-6, 2.0)
    if kernel_mix:
        kid = (rng.random(n_cell) < 0.5).astype(np.uint8)
    else:
        kid = np.zeros(n_cell, np.uint8)
    return _state(xi, v, counts, dv, kid, "random_cells", seed=seed)


def removal_box(n_sd, seed, xi_max=3, p_median=0.5, kernel_id=GOLOVIN, golovin_b=GOLOVIN_B):
    """One cell of small multiplicities (uniform in 1..xi_max) and lognormal
    volumes (median radius 15 um, sigma_g 1.4), its volume dV chosen so that
    the median pair's scaled probability is about p_median: coalescences of
    two SDs of multiplicity 1 remove an SD, so removals happen every step."""
    rng = np.random.default_rng(seed)
    xi = rng.integers(1, xi_max + 1, n_sd).astype(np.uint64)
    v = lognormal_volumes(rng, n_sd, 15e-6, 1.4)
    v_med = FOUR_PI_OVER_THREE * (15e-6) ** 3
    if kernel_id == GOLOVIN:
        k_med = golovin_b * 2.0 * v_med
    else:  # a gravitational pair of median radius and a 1.4x larger partner, roughly 1e-12 m^3/s
        k_med = 1.0e-12
    dv = k_med * xi_max * max(n_sd - 1, 1) / p_median
    return _state(xi, v, [n_sd], dv, kernel_id, "removal_box", golovin_b=golovin_b, seed=seed, n_sd=n_sd)


def concat_states(states, name="concat"):
    """One multi-cell state holding the cells of several states in order."""
    xi = np.concatenate([t["xi"] for t in states])
    v = np.concatenate([t["v"] for t in states])
    counts = np.concatenate([np.diff(t["cell_start"].astype(np.int64)) for t in states])
    dv = np.concatenate([t["dv"] for t in states])
    kid = np.concatenate([t["kernel_id"] for t in states])
    b = {t["golovin_b"] for t in states}
    assert len(b) == 1, "one Golovin constant per state"
    return _state(xi, v, counts, dv, kid, name, dt=states[0]["dt"], golovin_b=b.pop())


WORKLOADS = {
    "golovin_box": golovin_box,
    "gravitational_box": gravitational_box,
    "grid_bimodal": grid_bimodal,
    "ensemble": ensemble,
    "grid_lognormal": grid_lognormal,
}
