"""The allocation-free single-box step (sdm_coalescence_step_noalloc).

Callers that cannot allocate device memory (processes whose device memory
belongs to another pool with a hard cap, loops that must avoid the device-wide
synchronisation of cudaMalloc/cudaFree) use this entry point; its scratch lives
in a fixed array inside the library.  Here it is called through the C ABI on
device arrays and must give exactly what the allocating path (sdm_alloc +
sdm_coalescence_step on a one-cell state) gives, and exactly what the CPU
oracle gives, for two calls in a row -- the second call reuses the scratch
array left by the first.  Boxes on both sides of the PRP contract's sort
threshold (256/257 SDs) and boxes that lose SDs every step are included.
"""
import ctypes as C

import numpy as np
import pytest

import oracle
from paper_2101_06318_b300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2101_06318_b300 import sdm  # noqa: E402


def _box(n, kind, seed):
    if kind == "golovin":
        return inputs.golovin_box(n_sd=n)
    if kind == "removal":
        return inputs.removal_box(n, seed, p_median=0.2)
    return inputs.gravitational_box(n_sd=n, seed=seed, dv=1e6)


def _device_arrays(s, stride):
    n = len(s["xi"])
    xi_d = torch.from_numpy(s["xi"].view(np.int64).copy()).cuda()
    at_d = torch.zeros((1, stride), dtype=torch.float64, device="cuda")
    at_d[0, :n] = torch.from_numpy(s["v"]).cuda()
    return xi_d, at_d


def _noalloc_step(L, s, xi_d, at_d, stride, step, precision, shuffle):
    n = len(s["xi"])
    p = sdm.StepParams(s["dt"], s["golovin_b"], 42, step, sdm.PREC[precision], sdm.SHUFFLE[shuffle], 0, None)
    stream = torch.cuda.current_stream().cuda_stream
    return L.sdm_coalescence_step_noalloc(C.c_void_p(xi_d.data_ptr()), C.c_void_p(at_d.data_ptr()), 1, stride, n,
                                          float(s["dv"][0]), int(s["kernel_id"][0]), C.byref(p), C.c_void_p(stream))


CASES = [(200000, "grav", "fp64", "prp"), (200000, "grav", "fp64", "sort"), (5000, "golovin", "fp64", "prp"),
         (3, "golovin", "fp64", "sort"), (70000, "grav", "fp32", "prp"),
         (3, "removal", "fp64", "prp"), (256, "removal", "fp64", "prp"), (257, "removal", "fp64", "prp"),
         (1024, "removal", "fp64", "prp"), (5000, "removal", "fp64", "prp"), (5000, "removal", "fp64", "sort"),
         (257, "grav", "fp64", "prp"), (1024, "golovin", "fp64", "prp")]


@pytest.mark.parametrize("n,kind,precision,shuffle", CASES)
def test_noalloc_matches_allocating_path_and_oracle_two_calls(n, kind, precision, shuffle):
    L = sdm.lib()
    s = _box(n, kind, seed=n)
    ref = sdm.from_inputs(s)                    # allocating path: a one-cell state
    o = oracle.System(s["xi"], s["v"][None, :], s["cell_start"], s["dv"], s["kernel_id"], s["golovin_b"], shuffle)
    stride = n + 7                              # the caller's row stride, wider than n on purpose
    xi_d, at_d = _device_arrays(s, stride)
    for step in (0, 1):
        ref.step(s["dt"], 42, step, 1, precision=precision, golovin_b=s["golovin_b"], shuffle=shuffle)
        rc = _noalloc_step(L, s, xi_d, at_d, stride, step, precision, shuffle)
        assert rc == 0, sdm.STATUS.get(rc, rc)
        ref.sync()
        xr, ar, _ = ref.get_state()
        xg = xi_d.cpu().numpy().view(np.uint64)
        ag = at_d[0, :n].cpu().numpy()
        assert np.array_equal(xr, xg), f"step {step}: xi differs from the allocating path"
        assert np.array_equal(ar[0].view(np.uint64), ag.view(np.uint64)), f"step {step}: volumes differ"
        if precision == "fp64":                 # the FP64 mode is bit-exact against the oracle
            o.run(s["dt"], 42, step, 1)
            assert np.array_equal(o.xi, xg), f"step {step}: xi differs from the oracle"
            assert np.array_equal(o.attr[0].view(np.uint64), ag.view(np.uint64)), \
                f"step {step}: volumes differ from the oracle"
    ref.close()


@pytest.mark.parametrize("n,shuffle", [(5000, "prp"), (70000, "prp"), (70000, "sort")])
def test_noalloc_many_steps_with_removals(n, shuffle):
    """Forty calls on a box that loses SDs in every step (its live count falls
    through the 257-SD threshold): every call returns SDM_OK and the result
    matches the oracle bit for bit."""
    L = sdm.lib()
    s = _box(n, "removal", seed=7)
    o = oracle.System(s["xi"], s["v"][None, :], s["cell_start"], s["dv"], s["kernel_id"], s["golovin_b"], shuffle)
    xi_d, at_d = _device_arrays(s, n)
    for step in range(40):
        rc = _noalloc_step(L, s, xi_d, at_d, n, step, "fp64", shuffle)
        assert rc == 0, f"step {step}: {sdm.STATUS.get(rc, rc)}"
    ost = o.run(s["dt"], 42, 0, 40)
    assert ost["n_removed"] > n // 4
    assert np.array_equal(o.xi, xi_d.cpu().numpy().view(np.uint64))
    assert np.array_equal(o.attr[0].view(np.uint64), at_d[0].cpu().numpy().view(np.uint64))


def test_noalloc_rejects_oversized_box():
    L = sdm.lib()
    n = (1 << 18) + 1
    xi_d = torch.ones(n, dtype=torch.int64, device="cuda")
    at_d = torch.full((1, n), 1e-15, dtype=torch.float64, device="cuda")
    p = sdm.StepParams(1.0, 1500.0, 1, 0, 0, 0, 0, None)
    rc = L.sdm_coalescence_step_noalloc(C.c_void_p(xi_d.data_ptr()), C.c_void_p(at_d.data_ptr()), 1, n, n, 1.0, 0,
                                        C.byref(p), C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 3   # SDM_ECAPACITY
    assert torch.all(xi_d == 1)
