"""The allocation-free single-box step (sdm_coalescence_step_noalloc).

Callers that cannot allocate device memory (code running where the CUDA
allocator may not be called, processes whose memory belongs to another pool,
loops that must avoid cudaMalloc's synchronisation) use this entry point; its
scratch lives in a fixed array inside the library.  Here it is called through
the C ABI on device arrays and must give exactly what the allocating path
(sdm_alloc + sdm_coalescence_step on a one-cell state) gives, for two calls in
a row -- the second call reuses the scratch array left by the first.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2101_06318_b300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2101_06318_b300 import sdm  # noqa: E402


def _box(n, kernel, seed):
    if kernel == sdm.KERNEL_GOLOVIN:
        return inputs.golovin_box(n_sd=n)
    return inputs.gravitational_box(n_sd=n, seed=seed, dv=1e6)


@pytest.mark.parametrize("n,kernel,precision,shuffle", [(200000, 1, "fp64", "prp"), (200000, 1, "fp64", "sort"),
                                                        (5000, 0, "fp64", "prp"), (3, 0, "fp64", "sort"),
                                                        (70000, 1, "fp32", "prp")])
def test_noalloc_matches_allocating_path_two_calls(n, kernel, precision, shuffle):
    L = sdm.lib()
    s = _box(n, kernel, seed=n)
    dv = float(s["dv"][0])
    # allocating path: a one-cell state
    ref = sdm.from_inputs(s)
    # allocation-free path: the caller owns xi and the attributes (row stride > n on purpose)
    stride = n + 7
    xi_d = torch.from_numpy(s["xi"].view(np.int64).copy()).cuda()
    at_d = torch.zeros((1, stride), dtype=torch.float64, device="cuda")
    at_d[0, :n] = torch.from_numpy(s["v"]).cuda()
    stream = torch.cuda.current_stream().cuda_stream
    for step in (0, 1):
        ref.step(s["dt"], 42, step, 1, precision=precision, golovin_b=s["golovin_b"], shuffle=shuffle)
        p = sdm.StepParams(s["dt"], s["golovin_b"], 42, step, sdm.PREC[precision], sdm.SHUFFLE[shuffle], 0, None)
        rc = L.sdm_coalescence_step_noalloc(C.c_void_p(xi_d.data_ptr()), C.c_void_p(at_d.data_ptr()), 1, stride, n,
                                            dv, kernel, C.byref(p), C.c_void_p(stream))
        assert rc == 0, sdm.STATUS.get(rc, rc)
        ref.sync()
        xr, ar, _ = ref.get_state()
        xg = xi_d.cpu().numpy().view(np.uint64)
        ag = at_d[0, :n].cpu().numpy()
        assert np.array_equal(xr, xg), f"step {step}: xi differs"
        assert np.array_equal(ar[0].view(np.uint64), ag.view(np.uint64)), f"step {step}: volumes differ"
    ref.close()


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
