"""Failure detection without faulting the GPU.

* A bounded device wait that runs out: the library's grid barrier (the wait a
  PRP step's blocks take before their Step 0 compaction) is met by a
  cooperative grid whose last block never arrives (a flag nothing sets); the
  waiting blocks give up after the spin limit, record SDM_ETIMEOUT and return.
  sdm_sync reports it once, the context and the state stay usable, and the
  next steps (with removals, so the real barrier runs) match the oracle.
* A SORT-contract bucket that overflows (its capacity lowered for the test):
  the step reports SDM_ECAPACITY and leaves the cell unchanged; with the
  capacity restored the same step matches the oracle.
* The finishing warps' bulk copies announcing more bytes than they deliver
  (a phase nothing completes): every bounded wait runs out, the step reports
  SDM_ETIMEOUT and queues no pair of the cell, so the state is unchanged; with
  the switch off the same step matches the oracle.
"""
import time

import numpy as np
import pytest

import oracle
from paper_2101_06318_b300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2101_06318_b300 import sdm  # noqa: E402

SDM_ECAPACITY, SDM_ETIMEOUT = 3, 6


def _state(s, schedule=None):
    st = sdm.State(len(s["xi"]), len(s["dv"]), 1)
    if schedule:
        st.set_schedule(**schedule)
    st.init(s["xi"], s["v"][None, :], s["dv"], s["kernel_id"], cell_start=s["cell_start"])
    return st


def _oracle(s, shuffle="prp"):
    return oracle.System(s["xi"], s["v"][None, :], s["cell_start"], s["dv"], s["kernel_id"], s["golovin_b"], shuffle)


def test_bounded_wait_runs_out_and_the_state_stays_usable():
    s = inputs.concat_states([inputs.removal_box(n, seed=n, p_median=0.2) for n in (3000, 9000)])
    g = _state(s, dict(tile_slots=1024))
    t0 = time.perf_counter()
    g.debug_wait_timeout(2000, withhold=True)
    with pytest.raises(sdm.SDMError) as e:
        g.sync()
    assert e.value.code == SDM_ETIMEOUT
    assert time.perf_counter() - t0 < 5.0           # ~2000 polls of >= 100 ns, then the kernel returned
    g.sync()                                        # reported once, then cleared
    g.debug_wait_timeout(2000, withhold=False)      # everybody arrives: no error
    g.sync()
    # the real barrier of the PRP step (cells lose SDs every step) still works, bit-exact
    g.step(s["dt"], 42, 0, 12, golovin_b=s["golovin_b"])
    g.sync()
    o = _oracle(s)
    ost = o.run(s["dt"], 42, 0, 12)
    xi, at, _ = g.get_state()
    g.close()
    assert ost["n_removed"] > 100
    assert np.array_equal(o.xi, xi) and np.array_equal(o.attr.view(np.uint64), at.view(np.uint64))


def test_sort_bucket_overflow_reports_capacity_and_leaves_the_cell_unchanged():
    s = inputs.gravitational_box(n_sd=1 << 16)
    g = _state(s)
    sched = g.schedule
    assert sched["bucket_target"] >= 128
    g.debug_bucket_capacity(32)                     # far below the mean bucket count
    g.step(s["dt"], 42, 0, 1, golovin_b=s["golovin_b"], shuffle="sort")
    with pytest.raises(sdm.SDMError) as e:
        g.sync()
    assert e.value.code == SDM_ECAPACITY
    xi, at, _ = g.get_state()
    assert np.array_equal(xi, s["xi"]) and np.array_equal(at[0], s["v"])
    with pytest.raises(sdm.SDMError):
        g.debug_bucket_capacity(1 << 20)            # above the layout's capacity: refused
    g.set_schedule(**sched)                         # a new layout: the computed capacity again
    g.step(s["dt"], 42, 0, 1, golovin_b=s["golovin_b"], shuffle="sort")
    g.sync()
    xi, at, _ = g.get_state()
    g.close()
    o = _oracle(s, "sort")
    st = o.run(s["dt"], 42, 0, 1)
    assert st["n_collisions"] > 0
    assert np.array_equal(o.xi, xi) and np.array_equal(o.attr.view(np.uint64), at.view(np.uint64))


def test_staged_copy_wait_runs_out_and_the_state_stays_usable():
    s = inputs.gravitational_box(n_sd=1 << 16)
    g = _state(s)
    with pytest.raises(sdm.SDMError):
        g.debug_stage_shortfall(8192, 20)           # more than 4096 extra bytes: refused
    with pytest.raises(sdm.SDMError):
        g.debug_stage_shortfall(16, 5)              # a wait below 2^10 cycles: refused
    g.debug_stage_shortfall(16, 20)                 # waits of 2^20 cycles (~0.5 ms)
    t0 = time.perf_counter()
    g.step(s["dt"], 42, 0, 1, golovin_b=s["golovin_b"], shuffle="sort")
    with pytest.raises(sdm.SDMError) as e:
        g.sync()
    assert e.value.code == SDM_ETIMEOUT
    assert time.perf_counter() - t0 < 5.0
    g.sync()                                        # reported once, then cleared
    xi, at, _ = g.get_state()
    assert np.array_equal(xi, s["xi"]) and np.array_equal(at[0], s["v"])
    g.debug_stage_shortfall(0, 0)
    g.step(s["dt"], 42, 0, 2, golovin_b=s["golovin_b"], shuffle="sort")
    g.sync()
    xi, at, _ = g.get_state()
    g.close()
    o = _oracle(s, "sort")
    st = o.run(s["dt"], 42, 0, 2)
    assert st["n_collisions"] > 0
    assert np.array_equal(o.xi, xi) and np.array_equal(o.attr.view(np.uint64), at.view(np.uint64))
