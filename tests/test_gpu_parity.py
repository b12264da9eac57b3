"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

FP64 mode must reproduce the oracle bit for bit: multiplicities exactly and
volumes exactly (both sides evaluate the same IEEE operations in the same
order; the CUDA side only settles most decisions from an FP32 bound first).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2101_06318_b300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2101_06318_b300 import sdm  # noqa: E402


SHUFFLES = ["prp", "sort"]


def _oracle_system(s, attr=None, shuffle="prp", efield=0.0):
    a = s["v"][None, :] if attr is None else attr
    return oracle.System(s["xi"], a, s["cell_start"], s["dv"], s["kernel_id"], s["golovin_b"], shuffle, efield)


def _gpu_state(s, attr=None, schedule=None):
    n = len(s["xi"])
    a = s["v"][None, :] if attr is None else attr
    st = sdm.State(max(n, 1), len(s["dv"]), a.shape[0])
    if schedule:
        st.set_schedule(**schedule)
    st.init(s["xi"], a, s["dv"], s["kernel_id"], cell_start=s["cell_start"])
    return st


def _run_both(s, n_steps, seed=42, step0=0, attr=None, schedule=None, precision="fp64", shuffle="prp"):
    o = _oracle_system(s, attr, shuffle)
    ost = o.run(s["dt"], seed, step0, n_steps)
    g = _gpu_state(s, attr, schedule)
    gst = g.step(s["dt"], seed, step0, n_steps, precision=precision, golovin_b=s["golovin_b"], stats=True,
                 shuffle=shuffle)
    g.sync()
    xi, at, cs = g.get_state()
    # invariants the steps keep: live prefixes, and the volume keys the large-cell step gathers
    # (written by every collision and compaction under either contract)
    assert g.check() == (0, 0)
    g.close()
    return o, ost, xi, at, gst


def _assert_bitexact(o, xi, at):
    assert np.array_equal(o.xi, xi), f"xi differs at {np.flatnonzero(o.xi != xi)[:10]}"
    assert np.array_equal(o.attr.view(np.uint64), at.view(np.uint64)), \
        f"attr differs at {np.argwhere(o.attr != at)[:10]}"


@pytest.mark.parametrize("shuffle", SHUFFLES)
def test_golovin_box_bitexact_large_cell_path(shuffle):
    s = inputs.golovin_box()                   # one cell of 2^13 SDs -> large-cell path
    o, ost, xi, at, gst = _run_both(s, 300, shuffle=shuffle)
    _assert_bitexact(o, xi, at)
    for k in ("n_pairs", "n_collisions", "n_removed", "sum_gamma"):
        assert ost[k] == gst[k], k
    assert gst["n_collisions"] > 1000


@pytest.mark.parametrize("shuffle", SHUFFLES)
def test_golovin_box_bitexact_tile_path(shuffle):
    s = inputs.golovin_box(n_sd=4096)          # the whole cell handled in shared memory
    o, ost, xi, at, gst = _run_both(s, 300, schedule=dict(tile_slots=4096, tile_threads=512), shuffle=shuffle)
    _assert_bitexact(o, xi, at)
    assert ost["n_collisions"] == gst["n_collisions"]


@pytest.mark.parametrize("shuffle", SHUFFLES)
@pytest.mark.parametrize("seed", [1, 2, 3])
def test_random_cells_bitexact(seed, shuffle):
    # irregular cells (Poisson sizes incl. empty and 1-SD cells), dead slots, both kernels,
    # log-uniform xi so that case 2 and removals (and so compaction) occur
    s = inputs.random_cells(n_cell=700, mean_per_cell=23, seed=seed, dead_fraction=0.05, xi_max=50, dv=1e-12)
    o, ost, xi, at, gst = _run_both(s, 25, seed=seed, shuffle=shuffle)
    _assert_bitexact(o, xi, at)
    assert ost == {k: gst[k] for k in ost}
    assert gst["n_removed"] > 0 and gst["n_collisions"] > 100


@pytest.mark.parametrize("shuffle", SHUFFLES)
def test_cell_sizes_at_the_kernel_borders_bitexact(shuffle):
    """Cells on both sides of each border between code paths: 256 / 257 live SDs (sorted list or
    bijection), 512 / 513 slots (one warp per cell or a tile), 1024 / 1025 slots (tile or large
    cell), with dead slots so that the live count sits below the width, and small multiplicities
    so that removals (and compaction) happen in every kind of cell."""
    rng = np.random.default_rng(21)
    counts = np.array([2, 3, 255, 256, 257, 258, 300, 511, 512, 513, 600, 1023, 1024, 1025, 1100])
    n = int(counts.sum())
    xi = rng.integers(1, 6, n).astype(np.uint64)
    xi[rng.random(n) < 0.04] = 0                       # dead slots: live counts below the widths
    v = inputs.lognormal_volumes(rng, n, 15e-6, 1.8)
    kid = (np.arange(len(counts)) % 2).astype(np.uint8)
    s = inputs._state(xi, v, counts, 3e-14, kid, "borders")
    o, ost, xi_g, at, gst = _run_both(s, 30, seed=5, schedule=dict(tile_slots=1024), shuffle=shuffle)
    _assert_bitexact(o, xi_g, at)
    assert ost == {k: gst[k] for k in ost}
    assert gst["n_removed"] > 50


@pytest.mark.parametrize("shuffle", SHUFFLES)
def test_big_cells_many_buckets_bitexact(shuffle):
    rng = np.random.default_rng(5)
    parts = []
    for n in (1025, 3000, 4096, 9001, 20000, 2, 1, 0, 777):
        parts.append(n)
    counts = np.array(parts)
    n = int(counts.sum())
    xi = np.maximum(1, np.floor(np.exp(rng.random(n) * math.log(10 ** 6)))).astype(np.uint64)
    v = inputs.lognormal_volumes(rng, n, 20e-6, 2.0)
    s = inputs._state(xi, v, counts, 10.0, (np.arange(len(counts)) % 2).astype(np.uint8), "big_mix")
    o, ost, xi_g, at, gst = _run_both(s, 12, schedule=dict(tile_slots=1024, bucket_target=256), shuffle=shuffle)
    _assert_bitexact(o, xi_g, at)
    assert gst["n_collisions"] > 0


@pytest.mark.parametrize("shuffle", SHUFFLES)
def test_large_cells_with_removals_bitexact(shuffle):
    # small multiplicities and tiny dV: removals every step inside large cells, so the
    # end-of-step compaction of large cells runs, down to fewer than 257 live SDs
    rng = np.random.default_rng(8)
    counts = np.array([3000, 1500, 700])
    n = int(counts.sum())
    xi = rng.integers(1, 4, n).astype(np.uint64)
    v = inputs.lognormal_volumes(rng, n, 20e-6, 2.0)
    s = inputs._state(xi, v, counts, 1e-14, [0, 1, 0], "removals")
    o, ost, xi_g, at, gst = _run_both(s, 40, schedule=dict(tile_slots=512), shuffle=shuffle)
    _assert_bitexact(o, xi_g, at)
    assert gst["n_removed"] > 500
    live = [int(np.count_nonzero(xi_g[a:b])) for a, b in zip(s["cell_start"][:-1], s["cell_start"][1:])]
    assert min(live) < 257


@pytest.mark.parametrize("shuffle", SHUFFLES)
def test_small_cells_with_removals_and_reads_bitexact(shuffle):
    """Cells of one warp (2 to 512 SDs) that lose SDs every step (compacted stably right after the
    step's queued pairs).  Several steps in one call, then single steps with a different read after
    each (state, totals, Step 0 alone, spectrum), then steps again: the state equals the oracle's
    after every leg and the invariants hold."""
    rng = np.random.default_rng(31)
    counts = rng.integers(2, 513, 500)
    n = int(counts.sum())
    xi = rng.integers(1, 4, n).astype(np.uint64)
    v = inputs.lognormal_volumes(rng, n, 20e-6, 2.0)
    s = inputs._state(xi, v, counts, 1e-14, (np.arange(len(counts)) % 2).astype(np.uint8), "small_removals")
    o = _oracle_system(s, None, shuffle)
    g = _gpu_state(s, None, dict(tile_slots=512))
    removed = 0
    step = 0

    def both(k):
        nonlocal step, removed
        o.run(s["dt"], 9, step, k)
        st = g.step(s["dt"], 9, step, k, golovin_b=s["golovin_b"], stats=True, shuffle=shuffle)
        removed += st["n_removed"]
        step += k

    both(6)
    xi_g, at_g, _ = g.get_state()
    _assert_bitexact(o, xi_g, at_g)
    r_edges = np.exp(np.linspace(np.log(1e-6), np.log(5e-3), 41))
    for read in ("state", "totals", "remove_zero", "spectrum"):
        both(1)
        if read == "state":
            xi_g, at_g, _ = g.get_state()
            _assert_bitexact(o, xi_g, at_g)
        elif read == "totals":
            assert g.totals()[2] == int(np.count_nonzero(o.xi))
        elif read == "remove_zero":
            assert g.remove_zero() == int(np.count_nonzero(o.xi))
        else:
            assert np.array_equal(g.spectrum(r_edges), o.spectrum(r_edges))
    both(5)
    xi_g, at_g, _ = g.get_state()
    _assert_bitexact(o, xi_g, at_g)
    assert g.check() == (0, 0)
    g.close()
    assert removed > 2000


def test_removals_across_contracts_and_state_reads_bitexact():
    """Large cells that lose SDs in a PRP step are compacted at the next step's start, or before a
    state read or a SORT step: PRP steps, a totals() read, SORT steps, PRP steps again -- the
    state equals the oracle's after each leg and the invariants hold."""
    rng = np.random.default_rng(18)
    counts = np.array([2600, 1900, 900])
    n = int(counts.sum())
    xi = rng.integers(1, 4, n).astype(np.uint64)
    v = inputs.lognormal_volumes(rng, n, 20e-6, 2.0)
    s = inputs._state(xi, v, counts, 1e-14, [0, 1, 1], "removals_mixed")
    o = _oracle_system(s, None, "prp")
    g = _gpu_state(s, None, dict(tile_slots=512))
    removed = 0
    step = 0
    for shuffle, k in (("prp", 15), ("sort", 6), ("prp", 12)):
        o.shuffle = shuffle
        o.run(s["dt"], 7, step, k)
        st = g.step(s["dt"], 7, step, k, golovin_b=s["golovin_b"], stats=True, shuffle=shuffle)
        removed += st["n_removed"]
        step += k
        n_tot, _, live = g.totals()                      # a state read between the legs
        assert live == int(np.count_nonzero(o.xi))
        xi_g, at_g, _ = g.get_state()
        _assert_bitexact(o, xi_g, at_g)
        assert g.check() == (0, 0)
    assert removed > 300
    g.close()


@pytest.mark.parametrize("shuffle", SHUFFLES)
def test_multiple_attributes_bitexact(shuffle):
    s = inputs.random_cells(n_cell=200, mean_per_cell=30, seed=9, xi_max=1000, dv=1e-11)
    n = len(s["xi"])
    rng = np.random.default_rng(1)
    attr = np.vstack([s["v"], rng.random(n), rng.random(n) * 1e-20]).astype(np.float64)
    o, ost, xi, at, gst = _run_both(s, 10, attr=attr, shuffle=shuffle)
    _assert_bitexact(o, xi, at)


@pytest.mark.parametrize("shuffle", SHUFFLES)
def test_schedule_invariance(shuffle):
    s = inputs.random_cells(n_cell=400, mean_per_cell=60, seed=4, xi_max=10 ** 4, dv=1e-2)
    big = inputs.golovin_box(n_sd=5000)
    # append one larger cell so both paths run in the same step
    xi = np.concatenate([s["xi"], big["xi"]])
    v = np.concatenate([s["v"], big["v"]])
    counts = np.concatenate([np.diff(s["cell_start"].astype(np.int64)), [5000]])
    mix = inputs._state(xi, v, counts, np.concatenate([s["dv"], [1e6]]),
                        np.concatenate([s["kernel_id"], [0]]), "mix")
    ref = None
    for sched in (dict(tile_slots=256, tile_threads=64), dict(tile_slots=1024, tile_threads=256),
                  dict(tile_slots=4096, tile_threads=512, persistent=2), dict(tile_slots=4096, bucket_target=256),
                  dict(tile_slots=512, bucket_target=2048, persistent=1)):
        g = _gpu_state(mix, schedule=sched)
        g.step(1.0, 7, 0, 8, shuffle=shuffle)
        g.sync()
        got = g.get_state()
        g.close()
        if ref is None:
            ref = got
            o = _oracle_system(mix, shuffle=shuffle)
            o.run(1.0, 7, 0, 8)
            _assert_bitexact(o, got[0], got[1])
        else:
            assert np.array_equal(ref[0], got[0]) and np.array_equal(ref[1], got[1]), sched


@pytest.mark.parametrize("shuffle", SHUFFLES)
def test_gravitational_box_full_size_bitexact(shuffle):
    """The benchmarked workload (2^20 SDs in one cell) at full size, a few steps."""
    s = inputs.gravitational_box()
    o, ost, xi, at, gst = _run_both(s, 3, seed=42, shuffle=shuffle)
    _assert_bitexact(o, xi, at)
    assert ost["n_collisions"] == gst["n_collisions"] > 1000
    # most decisions are settled from the FP32 bound
    assert gst["n_fp64"] < 1e-3 * gst["n_pairs"]


@pytest.mark.parametrize("shuffle", SHUFFLES)
def test_grid_lognormal_full_size_bitexact(shuffle):
    """The default benchmark workload at full size (256 x 256 cells, 1.68e7 SDs) in the launch
    configuration bench.py times (the default schedule): two steps against the oracle's, every
    multiplicity and volume."""
    s = inputs.grid_lognormal()
    o, ost, xi, at, gst = _run_both(s, 2, seed=42, shuffle=shuffle)
    _assert_bitexact(o, xi, at)
    assert ost["n_collisions"] == gst["n_collisions"] > 50000


def test_grid_lognormal_full_size_fp32_mode():
    """FP32 mode on the default workload at full size: two steps against the FP64 oracle's; the
    SDs whose outcome differs stay within the mode's stated bound (2e-5 per SD and step), mass is
    conserved to 1e-12."""
    s = inputs.grid_lognormal()
    o, ost, xi, at, gst = _run_both(s, 2, seed=42, precision="fp32")
    differing = int(np.count_nonzero((xi != o.xi) | (at[0] != o.attr[0])))
    print(f"\nFP32 mode, full grid, 2 steps: {differing} of {len(xi)} SDs differ from the FP64 oracle")
    assert differing <= 2e-5 * 2 * len(xi)
    m_o = float(np.sum(o.xi.astype(np.float64) * o.attr[0]))
    m_g = float(np.sum(xi.astype(np.float64) * at[0]))
    assert m_g == pytest.approx(m_o, rel=1e-12)


def test_ensemble_full_size_bitexact():
    """The batched ensemble at full size (1024 boxes, 1.59e7 SDs, Golovin and gravitational
    kernels mixed) in one step, as the bench launches it."""
    s = inputs.ensemble()
    o, ost, xi, at, gst = _run_both(s, 1, seed=42)
    _assert_bitexact(o, xi, at)
    assert ost["n_collisions"] == gst["n_collisions"] > 0


def test_ensemble_graph_replay_full_size_bitexact():
    """The ensemble at full size as its benchmark line runs it: steps captured into a CUDA graph
    with the device step counter and replayed (one step outside the capture, two captured and
    replayed twice), against five oracle steps."""
    s = inputs.ensemble()
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        g = _gpu_state(s)
        d_step = torch.zeros(1, dtype=torch.int32, device="cuda")
        g.step(s["dt"], 42, 0, 1, golovin_b=s["golovin_b"], d_step=d_step)
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=stream):
            g.step(s["dt"], 42, 0, 2, golovin_b=s["golovin_b"], d_step=d_step)
        torch.cuda.synchronize()
        graph.replay()
        graph.replay()
        torch.cuda.synchronize()
        assert int(d_step.item()) == 5
        xi, at, _ = g.get_state()
        g.close()
    o = _oracle_system(s)
    ost = o.run(s["dt"], 42, 0, 5)
    _assert_bitexact(o, xi, at)
    assert ost["n_collisions"] > 0


def test_sort_contract_many_bucket_rounds_bitexact():
    """2^20 SDs in 8192 buckets of 128: the finishing pass takes several buckets per warp (its
    three-CTAs-per-SM form); the queues of surviving pairs carry over from bucket to bucket."""
    s = inputs.gravitational_box()
    o, ost, xi, at, gst = _run_both(s, 2, seed=11, shuffle="sort",
                                    schedule=dict(tile_slots=1024, bucket_target=128))
    _assert_bitexact(o, xi, at)
    assert ost["n_collisions"] == gst["n_collisions"] > 500


def test_sort_contract_sparse_buckets_bitexact():
    """A large cell of multiplicities 1 (every coalescence removes an SD) that loses about a third
    of its SDs every step, until its 1024 buckets hold a record or less on average: many buckets
    are empty, so a bucket's last position often pairs with the first of a bucket several further
    on, and the scatter's chunks past the live count hold no records."""
    s = inputs.removal_box(1 << 16, seed=3, xi_max=1, p_median=0.5)
    o, ost, xi, at, gst = _run_both(s, 16, shuffle="sort", schedule=dict(tile_slots=1024, bucket_target=64))
    _assert_bitexact(o, xi, at)
    assert 50 < int(np.count_nonzero(xi)) < 300


@pytest.mark.parametrize("target", [512, 1024])
def test_sort_contract_wide_buckets_bitexact(target):
    """2^16 SDs in buckets of 512 or 1024 on average: a bucket's sub-bucket counters number 512,
    1024 or 2048 (each form of the warp's 16-bit scan), and the bins past the first 256 of a
    sorted bucket are gathered one by one."""
    s = inputs.removal_box(1 << 16, seed=8, xi_max=3, p_median=0.3)
    o, ost, xi, at, gst = _run_both(s, 6, seed=5, shuffle="sort", schedule=dict(tile_slots=1024, bucket_target=target))
    _assert_bitexact(o, xi, at)
    for k in ("n_pairs", "n_collisions", "n_removed"):
        assert ost[k] == gst[k], k
    assert gst["n_collisions"] > 1000 and gst["n_removed"] > 0


@pytest.mark.parametrize("shuffle", SHUFFLES)
def test_grid_bimodal_sample_bitexact(shuffle):
    s = inputs.grid_bimodal(nx=32, ny=32)      # the 2D-grid workload on a 32 x 32 patch
    o, ost, xi, at, gst = _run_both(s, 10, shuffle=shuffle)
    _assert_bitexact(o, xi, at)


@pytest.mark.parametrize("shuffle", SHUFFLES)
def test_ensemble_sample_bitexact(shuffle):
    s = inputs.ensemble(n_members=24)
    o, ost, xi, at, gst = _run_both(s, 4, shuffle=shuffle)
    _assert_bitexact(o, xi, at)


def test_many_large_cells_with_small_cells_bitexact():
    """70 boxes of 1100 .. 3000 SDs of multiplicity 1 or 2 next to 300 small cells, all losing SDs
    every step: the PRP step of a layout with this many large cells queues their surviving pairs
    with the small cells' pairs (one pair kernel, one compaction for both), and boxes that fall
    below 257 live SDs have all their pairs queued."""
    rng = np.random.default_rng(17)
    boxes = [inputs.removal_box(int(n), seed=100 + i, xi_max=2, p_median=0.25)
             for i, n in enumerate(rng.integers(1100, 3000, 70))]
    small = inputs.random_cells(n_cell=300, mean_per_cell=40, seed=4, dead_fraction=0.05, xi_max=3, dv=1e-12)
    s = inputs.concat_states(boxes + [small])
    o, ost, xi, at, gst = _run_both(s, 15, seed=9)
    _assert_bitexact(o, xi, at)
    for k in ("n_pairs", "n_collisions", "n_removed", "sum_gamma"):
        assert ost[k] == gst[k], k
    live = [int(np.count_nonzero(xi[a:b])) for a, b in zip(s["cell_start"][:70], s["cell_start"][1:71])]
    assert gst["n_removed"] > 10000 and min(live) < 257


def test_many_large_cells_alternating_contracts_bitexact():
    """70 large cells (the PRP step's queue form) losing SDs every step, stepped under the PRP and
    SORT contracts in turn: neither contract's step leaves a cell uncompacted for the other."""
    rng = np.random.default_rng(23)
    boxes = [inputs.removal_box(int(n), seed=200 + i, xi_max=2, p_median=0.25)
             for i, n in enumerate(rng.integers(1100, 3000, 70))]
    s = inputs.concat_states(boxes)
    o = _oracle_system(s)
    g = _gpu_state(s)
    removed = 0
    for k, shuffle in enumerate(["prp", "prp", "sort", "prp", "sort", "sort", "prp", "prp"]):
        o.shuffle = shuffle
        o.run(s["dt"], 13, k, 1)
        st = g.step(s["dt"], 13, k, 1, golovin_b=s["golovin_b"], stats=True, shuffle=shuffle)
        removed += st["n_removed"]
    g.sync()
    xi, at, _ = g.get_state()
    assert g.check() == (0, 0)
    g.close()
    _assert_bitexact(o, xi, at)
    assert removed > 10000


def test_many_large_cells_bitexact():
    """80 boxes of 2^10 .. 2^13 SDs, each a large cell: the PRP step runs in its finer CTAs
    (64 threads) when a layout holds this many large cells."""
    s = inputs.ensemble(n_members=80, log2_lo=10, log2_hi=13, seed=5)
    o, ost, xi, at, gst = _run_both(s, 6, seed=3)
    _assert_bitexact(o, xi, at)
    assert ost["n_collisions"] == gst["n_collisions"]


@pytest.mark.parametrize("shuffle", SHUFFLES)
def test_electric_field_kernel_bitexact(shuffle):
    """The electric-field kernel (project definition: the gravitational kernel with efficiency
    E + eps (1 - E)) on every path: cells of one warp, tiles, large cells; two field parameters
    in turn; against the oracle with the same parameter."""
    rng = np.random.default_rng(17)
    counts = np.r_[rng.poisson(120, 300), rng.poisson(380, 100), [700, 900], [5000, 20000]]
    n = int(counts.sum())
    xi = np.floor(np.exp(rng.random(n) * np.log(1e6))).astype(np.uint64) + 1
    v = inputs.lognormal_volumes(rng, n, 14e-6, 1.8)
    s = inputs._state(xi, v, counts, 1e-3, 2, "electric_cells")
    for eps, step0 in ((0.35, 0), (1.0, 6)):
        o = _oracle_system(s, shuffle=shuffle, efield=eps)
        ost = o.run(s["dt"], 9, step0, 6)
        g = _gpu_state(s)
        gst = g.step(s["dt"], 9, step0, 6, stats=True, shuffle=shuffle, efield=eps)
        xg, ag, _ = g.get_state()
        assert g.check() == (0, 0)
        g.close()
        _assert_bitexact(o, xg, ag)
        assert gst["n_collisions"] == ost["n_collisions"] > 1000


@pytest.mark.parametrize("layout", ["few", "many"])
def test_prp_steps_with_removals_every_step(layout):
    """Large cells that lose SDs in every step, under the PRP contract: each launch compacts the
    cells the previous launch flagged (Step 0) behind its grid barrier.  Thirty one-step calls,
    then thirty steps in one call; the device error word is read after each call (a barrier
    that gave up would show as SDM_ETIMEOUT) and the state matches the oracle bit for bit."""
    if layout == "few":       # four large cells (CTAs of 128 threads) and one small cell
        parts = [inputs.removal_box(n, seed=n, p_median=0.2) for n in (300, 2000, 5000, 70000)]
    else:                     # 70 large cells (CTAs of 64 threads)
        parts = [inputs.removal_box(1100 + 29 * k, seed=k, p_median=0.2) for k in range(70)]
    s = inputs.concat_states(parts)
    o = _oracle_system(s)
    g = _gpu_state(s, schedule=dict(tile_slots=256))
    for step in range(30):
        g.step(s["dt"], 42, step, 1, golovin_b=s["golovin_b"])
        g.sync()                                   # raises on a device error
    g.step(s["dt"], 42, 30, 30, golovin_b=s["golovin_b"])
    g.sync()
    ost = o.run(s["dt"], 42, 0, 60)
    xi, at, _ = g.get_state()
    assert g.check() == (0, 0)
    g.close()
    _assert_bitexact(o, xi, at)
    assert ost["n_removed"] > len(s["xi"]) // 4


def test_edge_cases():
    # n_sd = 2 (one pair), 3 (odd), all-dead cell, huge p (caps bind), xi near 2^53
    xi = np.array([5, 5, 7, 1, 9, 0, 0, (1 << 53) - 1, 3], np.uint64)
    v = np.array([1e-12, 2e-12, 3e-12, 4e-12, 5e-12, 6e-12, 7e-12, 8e-12, 9e-12])
    counts = [2, 3, 2, 2]
    s = inputs._state(xi, v, counts, [1e-20, 1.0, 1.0, 1e-20], [0, 1, 0, 0], "edge")
    o, ost, xi_g, at, gst = _run_both(s, 5)
    _assert_bitexact(o, xi_g, at)
    # empty state
    e = inputs._state(np.zeros(0, np.uint64), np.zeros(0), [0], 1.0, 0, "empty")
    g = _gpu_state(e)
    g.step(1.0, 1, 0, 3)
    g.sync()
    assert g.totals() == (0, 0.0, 0)


def test_fp32_bound_holds_and_fp64_matches_oracle():
    rng = np.random.default_rng(2)
    n = 200000
    r1 = np.exp(rng.uniform(np.log(0.02e-6), np.log(2e-3), n))
    r2 = np.where(rng.random(n) < 0.2, r1 * (1 + rng.normal(0, 1e-6, n)),
                  np.exp(rng.uniform(np.log(0.02e-6), np.log(2e-3), n)))
    # radii near regime joins and table nodes
    joins = np.array([8e3 / 1.19e8, (201 / 8e3) ** 2, 10e-6, 20e-6, 40e-6, 100e-6, 300e-6, 1000e-6])
    r1[:8000] = np.repeat(joins, 1000) * (1 + rng.normal(0, 1e-7, 8000))
    v1 = 4 / 3 * np.pi * r1 ** 3
    v2 = 4 / 3 * np.pi * r2 ** 3
    xi1 = rng.integers(1, 10 ** 9, n).astype(np.uint64)
    xi2 = rng.integers(1, 10 ** 9, n).astype(np.uint64)
    g = sdm.State(16, 1)
    dev = lambda a: torch.from_numpy(a.view(np.int64) if a.dtype == np.uint64 else a).cuda()
    worst = 0.0
    for kid, ncell, dv, eps in ((1, 1 << 20, 1e6, 0.0), (0, 8192, 1e6, 0.0), (1, 127, 1e3, 0.0),
                                (2, 1 << 20, 1e6, 0.4), (2, 300, 1e3, 1.0), (2, 999, 1e3, 0.0)):
        p64, p32, e32 = g.eval_pairs(kid, dev(v1), dev(v2), dev(xi1), dev(xi2), ncell, dv, efield=eps)
        p64, p32, e32 = p64.cpu().numpy(), p32.cpu().numpy().astype(np.float64), e32.cpu().numpy().astype(np.float64)
        # FP64 value equals the oracle's bit for bit (sampled)
        for i in rng.choice(n, 2000, replace=False):
            K = oracle.kernel(kid, v1[i], v2[i], 1500.0, eps)
            po = oracle.pair_prob(K, xi1[i], xi2[i], oracle.pair_scale(ncell), 1.0, dv)
            assert p64[i] == po, (kid, i)
        ratio = np.abs(p64 - p32) / e32
        worst = max(worst, float(ratio.max()))
        assert np.all(np.abs(p64 - p32) <= e32), (kid, ratio.max())
    # the bound is not vacuous either: its width is used, but never exceeded
    assert 0.01 < worst <= 1.0, worst
    # the second filter (gravitational kernel): its FP64 value from refined FP32 seeds stays within
    # its bound of the exact sequence's value, also at regime joins, table nodes and near-equal radii
    worst_lite = 0.0
    for ncell, dv in ((1 << 20, 1e6), (127, 1e3)):
        p64, _, _, pl, el = g.eval_pairs(1, dev(v1), dev(v2), dev(xi1), dev(xi2), ncell, dv, lite=True)
        p64, pl, el = p64.cpu().numpy(), pl.cpu().numpy(), el.cpu().numpy()
        ok = el >= 0
        assert ok.mean() > 0.99
        assert np.all(np.abs(p64[ok] - pl[ok]) <= el[ok])
        worst_lite = max(worst_lite, float((np.abs(p64[ok] - pl[ok]) / el[ok]).max()))
    assert worst_lite < 0.01, worst_lite


def test_early_exit_bound_holds():
    """The early exit's bound of p (table of the two volumes' bins) is above the FP64 value and the
    FP32 value of every pair: wide random pairs, near-equal pairs, volumes on and just below the
    bins' edges, radii at the fall-speed regime joins and at efficiency table nodes, radius ratios
    at the table's ratio nodes."""
    rng = np.random.default_rng(12)
    n = 300000
    r1 = np.exp(rng.uniform(np.log(0.01e-6), np.log(3e-3), n))
    r2 = np.exp(rng.uniform(np.log(0.01e-6), np.log(3e-3), n))
    near = rng.random(n) < 0.2
    r2[near] = r1[near] * (1 + rng.normal(0, 1e-3, near.sum()))
    joins = np.array([8e3 / 1.19e8, (201 / 8e3) ** 2, 10e-6, 20e-6, 30e-6, 60e-6, 100e-6, 150e-6, 300e-6, 1e-3])
    r1[:10000] = np.repeat(joins, 1000) * (1 + rng.normal(0, 1e-7, 10000))
    # radius ratios at and next to the efficiency table's q nodes (the bound's efficiency factor is
    # the interpolant's largest value over the bins' rectangle of radius and ratio)
    qn = np.repeat(np.arange(1, 10) / 10.0, 1000) * (1 + rng.normal(0, 1e-4, 9000))
    r2[50000:59000] = r1[50000:59000] * qn
    v1 = 4 / 3 * np.pi * r1 ** 3
    v2 = 4 / 3 * np.pi * r2 ** 3
    # volumes on a bin edge 2^e (1 + m/4) and one ulp below it
    e = rng.integers(-75, -10, 20000)
    m = rng.integers(0, 4, 20000)
    edge = np.ldexp(1.0 + m / 4.0, e)
    v1[10000:30000] = np.where(rng.random(20000) < 0.5, edge, np.nextafter(edge, 0.0))
    v2[30000:50000] = np.where(rng.random(20000) < 0.5, edge, np.nextafter(edge, 0.0))
    xi1 = rng.integers(1, 10 ** 9, n).astype(np.uint64)
    xi2 = rng.integers(1, 10 ** 9, n).astype(np.uint64)
    g = sdm.State(16, 1)
    dev = lambda a: torch.from_numpy(a.view(np.int64) if a.dtype == np.uint64 else a).cuda()
    for kid, ncell, dv, eps in ((1, 1 << 20, 1e6, 0.0), (0, 8192, 1e6, 0.0), (1, 300, 1e3, 0.0),
                                (2, 1 << 20, 1e6, 0.5), (2, 300, 1e3, 1.0)):
        p64, p32, _, pup = g.eval_pairs(kid, dev(v1), dev(v2), dev(xi1), dev(xi2), ncell, dv, bound=True,
                                        efield=eps)
        p64, p32, pup = p64.cpu().numpy(), p32.cpu().numpy().astype(np.float64), pup.cpu().numpy().astype(np.float64)
        assert np.all(pup >= p64), (kid, np.flatnonzero(pup < p64)[:5])
        assert np.all(pup >= p32), (kid, np.flatnonzero(pup < p32)[:5])
        # not vacuous: within a small factor of p (the multiplicity's power of two alone gives up to 2)
        # for pairs of volumes within a few bins of each other; very unequal or nearly equal radii
        # (fall speeds far apart or nearly the same) leave more room, but there p is small anyway
        q = np.minimum(v1, v2) / np.maximum(v1, v2)
        sel = (p64 > 0) & (q > 0.03) & (q < 0.7) if kid else p64 > 0
        ratio = np.median(pup[sel] / p64[sel])
        print("kernel", kid, "cell", ncell, "median bound / p", ratio)
        # the electric-field kernel's rows bound its efficiency by 1 (E_eps >= eps >= 0.5 here)
        assert ratio < (4.0 if kid < 2 else 8.0), (kid, ratio)


def _spectrum_l1(a, b):
    return float(np.abs(a - b).sum() / max(b.sum(), 1e-300))


@pytest.mark.parametrize("workload", ["box", "cells"])
def test_fp32_mode_against_the_fp64_oracle(workload):
    """FP32 mode (eq. (p) and the decision in FP32, volumes FP64, multiplicities exact) against the
    FP64 oracle, per result:
    * decisions: from the same state (the oracle's, uploaded before each step), one FP32 step and
      one oracle step; SDs whose outcome differs, over all SDs of candidate pairs;
    * after a run of steps from the same start: the number of multiplicities that differ (one
      differing decision changes the trajectory from there on), the mass spectrum's relative L1
      distance and the droplet number's relative difference at t_end; mass conserved to 1e-12."""
    if workload == "box":
        s = inputs.gravitational_box(n_sd=1 << 16)
        n_steps, n_dec = 200, 20
    else:
        s = inputs.random_cells(n_cell=400, mean_per_cell=150, seed=9, xi_max=10 ** 6, dv=1e3)
        n_steps, n_dec = 60, 20
    # decisions from the same state
    o = _oracle_system(s)
    g = _gpu_state(s)
    differing = pairs = 0
    for k in range(n_dec):
        x0, a0 = o.xi.copy(), o.attr.copy()
        st = o.step(s["dt"], 42, k)
        g.set_state(x0, a0)
        g.step(s["dt"], 42, k, 1, precision="fp32", golovin_b=s["golovin_b"])
        xg, ag, _ = g.get_state()
        differing += int(np.count_nonzero((xg != o.xi) | (ag[0] != o.attr[0])))
        pairs += st["n_pairs"]
    g.close()
    frac_sd = differing / (2.0 * pairs)
    # a run of steps from the same start
    o = _oracle_system(s)
    o.run(s["dt"], 42, 0, n_steps)
    g = _gpu_state(s)
    g.step(s["dt"], 42, 0, n_steps, precision="fp32", golovin_b=s["golovin_b"])
    xg, ag, _ = g.get_state()
    n_xi_diff = int(np.count_nonzero(xg != o.xi))
    r_edges = np.exp(np.linspace(np.log(1e-6), np.log(5e-3), 101))
    l1 = _spectrum_l1(g.spectrum(r_edges), o.spectrum(r_edges))
    nt_o, _, m_o = o.totals()                       # oracle: (sum xi, live SDs, mass)
    nt_g, m_g, _ = g.totals()                       # library: (sum xi, mass, live SDs)
    g.close()
    print(f"\nFP32 vs FP64 oracle ({workload}): differing SD outcomes per step {frac_sd:.2e} "
          f"({differing} of {2 * pairs}); after {n_steps} steps: {n_xi_diff} of {len(xg)} multiplicities differ, "
          f"spectrum L1 {l1:.2e}, droplet number {(nt_g - nt_o) / nt_o:+.2e}")
    assert m_g == pytest.approx(m_o, rel=1e-12)
    # the bounds stated for the FP32 mode
    assert frac_sd <= 2e-5
    assert l1 <= 2e-2
    assert abs(nt_g - nt_o) / nt_o <= 1e-3


def test_spectrum_and_totals_match_oracle():
    s = inputs.golovin_box()
    o = _oracle_system(s)
    o.run(1.0, 42, 0, 500)
    g = _gpu_state(s)
    g.step(1.0, 42, 0, 500)
    r_edges = np.exp(np.linspace(np.log(1e-6), np.log(5e-3), 101))
    so = o.spectrum(r_edges)
    sg = g.spectrum(r_edges)
    # both sides sum each bin exactly and round once: equal, and the same on every call
    assert np.array_equal(sg, so)
    assert np.array_equal(g.spectrum(r_edges), sg)
    nt, nl, mo = o.totals()
    gn, gm, gl = g.totals()
    assert gn == nt and gl == nl
    assert gm == pytest.approx(mo, rel=1e-12)
    # multi-cell spectrum of a single cell and of all
    s2 = inputs.random_cells(n_cell=50, mean_per_cell=100, seed=3)
    o2, g2 = _oracle_system(s2), _gpu_state(s2)
    assert np.array_equal(g2.spectrum(r_edges, cell=7), o2.spectrum(r_edges, cell_lo=7, cell_hi=8))
    assert np.array_equal(g2.spectrum(r_edges), o2.spectrum(r_edges))
    # a large state whose terms span many binades (multiplicities 1 .. 2^52), volumes on the edges
    rng = np.random.default_rng(3)
    s3 = inputs.random_cells(n_cell=64, mean_per_cell=4000, seed=5, xi_max=2 ** 52)
    ve = ((oracle.FOUR_PI_OVER_THREE * r_edges) * r_edges) * r_edges
    s3["v"][:500] = ve[rng.integers(0, len(ve), 500)]
    o3, g3 = _oracle_system(s3), _gpu_state(s3)
    assert np.array_equal(g3.spectrum(r_edges), o3.spectrum(r_edges))
    g2.close()
    g3.close()


def test_mass_conservation_and_remove_zero():
    s = inputs.random_cells(n_cell=300, mean_per_cell=40, seed=8, xi_max=20, dv=1e-12)
    g = _gpu_state(s)
    n0, m0, l0 = g.totals()
    st = g.step(1.0, 3, 0, 30, stats=True)
    n1, m1, l1 = g.totals()
    assert m1 == pytest.approx(m0, rel=1e-12)
    assert n0 - n1 >= st["sum_gamma"] > 0
    assert l1 == l0 - st["n_removed"] == g.remove_zero() == g.remove_zero()


def test_checkpoint_resume_bitexact():
    s = inputs.random_cells(n_cell=100, mean_per_cell=50, seed=6, xi_max=1000, dv=1e-3)
    a = _gpu_state(s)
    a.step(1.0, 11, 0, 10)
    xa, aa, _ = a.get_state()
    b = _gpu_state(s)
    b.step(1.0, 11, 0, 5)
    xb, ab, _ = b.get_state()
    c = _gpu_state(s)
    c.set_state(xb, ab)
    c.step(1.0, 11, 5, 5)
    c.sync()
    xc, ac, _ = c.get_state()
    assert np.array_equal(xa, xc) and np.array_equal(aa, ac)


def test_cuda_graph_replay_with_device_step_counter():
    s = inputs.random_cells(n_cell=300, mean_per_cell=40, seed=12, xi_max=10 ** 5, dv=1e-3)
    big = inputs.golovin_box(n_sd=3000)
    xi = np.concatenate([s["xi"], big["xi"]])
    v = np.concatenate([s["v"], big["v"]])
    counts = np.concatenate([np.diff(s["cell_start"].astype(np.int64)), [3000]])
    mix = inputs._state(xi, v, counts, np.concatenate([s["dv"], [1e6]]), np.concatenate([s["kernel_id"], [0]]),
                        "mix")
    ref = _gpu_state(mix)
    ref.step(1.0, 5, 0, 12)
    xr, ar, _ = ref.get_state()
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        g = _gpu_state(mix)
        d_step = torch.zeros(1, dtype=torch.int32, device="cuda")
        g.step(1.0, 5, 0, 1, d_step=d_step)          # warm-up outside capture: steps 0
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=stream):
            g.step(1.0, 5, 0, 4, d_step=d_step)       # captured: 4 steps
        torch.cuda.synchronize()
        # the capture itself did not run; 11 more steps = replay 4 + 4 then 3 host steps
        graph.replay()
        graph.replay()
        torch.cuda.synchronize()
        assert int(d_step.item()) == 9
        g.step(1.0, 5, 9, 3)
        g.sync()
        xg, ag, _ = g.get_state()
    assert np.array_equal(xr, xg) and np.array_equal(ar, ag)
    o = _oracle_system(mix)                         # and both equal the oracle's twelve steps
    o.run(1.0, 5, 0, 12)
    _assert_bitexact(o, xg, ag)


def test_graph_replayed_prp_steps_then_sort_step_bitexact():
    """PRP steps replayed from a CUDA graph can leave large cells flagged for Step 0 where the
    host does not see it; a SORT step after them (with a state read between capture and replay)
    still compacts those cells first."""
    rng = np.random.default_rng(21)
    counts = np.array([2600, 1900, 900])
    n = int(counts.sum())
    xi = rng.integers(1, 4, n).astype(np.uint64)
    v = inputs.lognormal_volumes(rng, n, 20e-6, 2.0)
    s = inputs._state(xi, v, counts, 1e-14, [0, 1, 1], "removals_graph")
    o = _oracle_system(s, None, "prp")
    o.run(s["dt"], 7, 0, 4)
    o.shuffle = "sort"
    o.run(s["dt"], 7, 4, 2)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        g = _gpu_state(s, None, dict(tile_slots=512))
        d_step = torch.zeros(1, dtype=torch.int32, device="cuda")
        g.step(s["dt"], 7, 0, 1, golovin_b=s["golovin_b"], d_step=d_step)      # step 0
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=stream):
            g.step(s["dt"], 7, 0, 3, golovin_b=s["golovin_b"], d_step=d_step)  # steps 1..3, not run here
        torch.cuda.synchronize()
        g.get_state()                                    # a state read between capture and replay
        graph.replay()
        torch.cuda.synchronize()
        assert int(d_step.item()) == 4
        g.step(s["dt"], 7, 4, 2, golovin_b=s["golovin_b"], shuffle="sort")
        g.sync()
        xg, ag, _ = g.get_state()
        assert g.check() == (0, 0)
    _assert_bitexact(o, xg, ag)
    assert int(np.count_nonzero(xg)) < n - 100          # SDs were removed along the way


def test_invalid_inputs_raise():
    s = inputs.random_cells(n_cell=4, mean_per_cell=5, seed=1, min_per_cell=1)
    n = len(s["xi"])
    bad = dict(s)
    bad["v"] = s["v"].copy()
    bad["v"][0] = -1.0
    with pytest.raises(sdm.SDMError) as e:
        _gpu_state(bad)
    assert e.value.code == 1
    bad = dict(s)
    bad["xi"] = s["xi"].copy()
    bad["xi"][0] = 1 << 53
    with pytest.raises(sdm.SDMError) as e:
        _gpu_state(bad)
    assert e.value.code == 4
    st = sdm.State(n - 1, 4)
    with pytest.raises(sdm.SDMError) as e:
        st.init(s["xi"], s["v"][None], s["dv"], s["kernel_id"], cell_start=s["cell_start"])
    assert e.value.code == 3
    g = _gpu_state(s)
    with pytest.raises(sdm.SDMError):
        g.step(dt=-1.0)
    # invalid data streamed in later is reported at the next sync
    xi = s["xi"].copy()
    xi[1] = 1 << 60
    g.set_state(xi, s["v"][None].copy())
    with pytest.raises(sdm.SDMError) as e:
        g.sync()
    assert e.value.code == 4
    g.sync()   # the error word was cleared
    # a live SD behind a removed slot of the same cell breaks the layout rule of set_state
    cs = s["cell_start"]
    c = int(np.flatnonzero(np.diff(cs.astype(np.int64)) >= 2)[0])
    xg = s["xi"].copy()
    xg[cs[c]] = 0
    g.set_state(xg, s["v"][None].copy())
    with pytest.raises(sdm.SDMError) as e:
        g.sync()
    assert e.value.code == 1


def test_device_pointer_init_and_workspace():
    s = inputs.random_cells(n_cell=64, mean_per_cell=30, seed=2)
    n = len(s["xi"])
    ws_bytes = sdm.lib().sdm_workspace_bytes(n, 64, 1)
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device="cuda")
    g = sdm.State(n, 64, 1, workspace=ws)
    g.init(torch.from_numpy(s["xi"].view(np.int64).copy()).cuda(), torch.from_numpy(s["v"][None].copy()).cuda(),
           torch.from_numpy(s["dv"].copy()).cuda(), torch.from_numpy(s["kernel_id"].copy()).cuda(),
           cell_start=torch.from_numpy(s["cell_start"].view(np.int32).copy()).cuda())
    g.step(1.0, 1, 0, 5)
    o = _oracle_system(s)
    o.run(1.0, 1, 0, 5)
    xi_d = torch.empty(n, dtype=torch.int64, device="cuda")
    at_d = torch.empty((1, n), dtype=torch.float64, device="cuda")
    g.get_state(xi_d, at_d)
    torch.cuda.synchronize()
    _assert_bitexact(o, xi_d.cpu().numpy().view(np.uint64), at_d.cpu().numpy())
    small = torch.empty(1024, dtype=torch.uint8, device="cuda")
    with pytest.raises(sdm.SDMError) as e:
        sdm.State(n, 64, 1, workspace=small)
    assert e.value.code == 2


def test_set_schedule_keeps_the_fields_not_given():
    """The binding's set_schedule changes only the fields it is given (the library's defaults:
    1024-slot tiles of 256 threads, 256-SD buckets, no persistent grid)."""
    s = inputs.gravitational_box(n_sd=1 << 12)
    g = _gpu_state(s)
    before = g.schedule
    assert before == {"tile_slots": 1024, "tile_threads": 256, "bucket_target": 256, "persistent": 0}
    g.set_schedule(tile_slots=2048)
    after = g.schedule
    g.close()
    assert after == dict(before, tile_slots=2048)


def test_autotune_keeps_results():
    s = inputs.random_cells(n_cell=500, mean_per_cell=100, seed=3, xi_max=10 ** 4, dv=1e-2)
    a = _gpu_state(s)
    best = a.autotune(n_steps=2)
    assert best["tile_slots"] in (512, 1024, 2048, 4096)
    a.step(1.0, 2, 0, 6)
    xa, aa, _ = a.get_state()
    o = _oracle_system(s)
    o.run(1.0, 2, 0, 6)
    _assert_bitexact(o, xa, aa)


def _displacement_state(seed, n_cell, mean, spare, big=()):
    """Cells with spare slots (capacity to receive SDs), a few large ones, small multiplicities."""
    rng = np.random.default_rng(seed)
    counts = rng.poisson(mean, n_cell)
    for k, nbig in big:
        counts[k] = nbig
    width = counts + spare
    n = int(width.sum())
    cs = np.concatenate([[0], np.cumsum(width)]).astype(np.uint32)
    xi = np.zeros(n, np.uint64)
    for c in range(n_cell):
        xi[cs[c]:cs[c] + counts[c]] = rng.integers(1, 50, counts[c])
    v = inputs.lognormal_volumes(rng, n, 15e-6, 1.8)
    kid = (np.arange(n_cell) % 2).astype(np.uint8)
    return inputs._state(xi, v, width, 1e-13, kid, "displacement"), rng


def test_rebucket_then_steps_bitexact():
    """Displacement between steps (SDs moved to neighbouring or random cells, into the cells' spare
    slots), then steps: the state equals the oracle's after each displacement and each leg of
    steps, for small cells, tiles and large cells alike."""
    s, rng = _displacement_state(31, 300, 60, 40, big=((7, 3000), (150, 1800), (299, 700)))
    o = _oracle_system(s, None, "prp")
    g = _gpu_state(s, None, dict(tile_slots=1024))
    cs = s["cell_start"].astype(np.int64)
    cell_of = np.repeat(np.arange(len(cs) - 1), np.diff(cs))
    step = 0
    for rnd in range(4):
        xi_g, at_g, _ = g.get_state()
        _assert_bitexact(o, xi_g, at_g)
        live = np.flatnonzero(o.xi)
        cid = cell_of.copy()
        move = rng.random(len(live)) < 0.25
        dst = cell_of[live] + rng.integers(-2, 3, len(live))
        far = rng.random(len(live)) < 0.02
        dst = np.where(far, rng.integers(0, len(cs) - 1, len(live)), dst)
        cid[live[move]] = np.clip(dst[move], 0, len(cs) - 2)
        # keep the capacities: drop moves into cells that would overflow (in slot order)
        counts = np.bincount(cid[live], minlength=len(cs) - 1)
        over = counts > np.diff(cs)
        if over.any():
            back = np.isin(cid[live], np.flatnonzero(over))
            cid[live[back]] = cell_of[live[back]]
        assert o.rebucket(cid)
        g.rebucket(cid.astype(np.uint32))
        xi_g, at_g, _ = g.get_state()
        _assert_bitexact(o, xi_g, at_g)
        assert g.check() == (0, 0)
        o.run(s["dt"], 11, step, 6)
        g.step(s["dt"], 11, step, 6, golovin_b=s["golovin_b"])
        step += 6
    xi_g, at_g, _ = g.get_state()
    _assert_bitexact(o, xi_g, at_g)
    g.close()


def test_rebucket_rejects_overflow_and_bad_indices():
    s, rng = _displacement_state(32, 40, 20, 2)
    g = _gpu_state(s)
    x0, a0, _ = g.get_state()
    n = len(s["xi"])
    with pytest.raises(sdm.SDMError):
        g.rebucket(np.zeros(n, np.uint32))                  # everything into cell 0: over its width
    with pytest.raises(sdm.SDMError):
        g.rebucket(np.full(n, 40, np.uint32))               # no cell 40
    x1, a1, _ = g.get_state()
    assert np.array_equal(x0, x1) and np.array_equal(a0.view(np.uint64), a1.view(np.uint64))
    g.close()
