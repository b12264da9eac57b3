"""Python binding of libsdm (the C ABI of include/sdm.h): argument marshalling only.

Every step of the coalescence path runs in the library's CUDA kernels; this
module converts numpy arrays (host memory) and torch CUDA tensors (device
memory) to pointers, passes the current torch stream, and turns status codes
into exceptions.  There is no CPU fallback: if the library cannot be built or
loaded, or no GPU is present, the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os
import threading
from dataclasses import dataclass

import numpy as np

from . import build as _build

_lock = threading.Lock()
_lib = None

PREC = {"fp64": 0, "fp32": 1, "surrogate": 2}
KERNEL_GOLOVIN = 0
KERNEL_GRAVITATIONAL = 1
KERNEL_ELECTRIC = 2

STATUS = {0: "SDM_OK", 1: "SDM_EINVAL", 2: "SDM_ENOMEM", 3: "SDM_ECAPACITY", 4: "SDM_ERANGE",
          5: "SDM_ECUDA", 6: "SDM_ETIMEOUT", 7: "SDM_ENOTSUP"}

# every entry point declared in include/sdm.h
EXPORTS = ["sdm_version", "sdm_status_str", "sdm_workspace_bytes", "sdm_alloc", "sdm_init_state",
           "sdm_init_state_segmented", "sdm_set_state", "sdm_get_state", "sdm_coalescence_step",
           "sdm_remove_zero", "sdm_spectrum", "sdm_totals", "sdm_check_state", "sdm_rebucket",
           "sdm_get_schedule", "sdm_set_schedule",
           "sdm_autotune", "sdm_sync", "sdm_free", "sdm_eval_pairs", "sdm_set_profiling", "sdm_get_profile",
           "sdm_launches_per_step", "sdm_coalescence_step_noalloc", "sdm_surrogate_create", "sdm_surrogate_free",
           "sdm_surrogate_train", "sdm_surrogate_build_mask", "sdm_surrogate_params_io", "sdm_surrogate_info",
           "sdm_surrogate_loss_grad", "sdm_surrogate_eval", "sdm_attach_surrogate", "sdm_debug_wait_timeout",
           "sdm_debug_bucket_capacity", "sdm_debug_stage_shortfall"]


class SurrogateParams(C.Structure):
    _fields_ = [("n_train", C.c_uint64), ("seed", C.c_uint64), ("r_min", C.c_double), ("r_max", C.c_double)]


class SDMError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__(f"{where}: {STATUS.get(code, code)}")


SHUFFLE = {"prp": 0, "sort": 1}


class StepParams(C.Structure):
    _fields_ = [("dt", C.c_double), ("golovin_b", C.c_double), ("seed", C.c_uint64), ("step", C.c_uint32),
                ("precision", C.c_uint32), ("shuffle", C.c_uint32), ("reserved", C.c_uint32),
                ("d_step", C.c_void_p), ("efield", C.c_double)]


class StepStats(C.Structure):
    _fields_ = [("n_pairs", C.c_uint64), ("n_collisions", C.c_uint64), ("n_removed", C.c_uint64),
                ("sum_gamma", C.c_uint64), ("n_fp64", C.c_uint64)]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


class Schedule(C.Structure):
    _fields_ = [("tile_slots", C.c_uint32), ("tile_threads", C.c_uint32), ("bucket_target", C.c_uint32),
                ("persistent", C.c_uint32)]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


def lib(build_if_needed: bool = True):
    """Load libsdm.so (building it in-tree first when it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if build_if_needed and _build.stale():
            _build.build()
        if not os.path.exists(_build.LIB):
            raise OSError(f"libsdm.so not built: {_build.LIB}")
        L = C.CDLL(_build.LIB)
        vp, u32, u64, f64, i32, sz = C.c_void_p, C.c_uint32, C.c_uint64, C.c_double, C.c_int, C.c_size_t
        L.sdm_version.restype = C.c_char_p
        L.sdm_status_str.argtypes = [i32]
        L.sdm_status_str.restype = C.c_char_p
        L.sdm_workspace_bytes.argtypes = [u64, u32, u32]
        L.sdm_workspace_bytes.restype = sz
        L.sdm_alloc.argtypes = [C.POINTER(vp), u64, u32, u32, vp, vp, sz]
        L.sdm_init_state.argtypes = [vp, vp, vp, vp, u64, vp, vp, i32]
        L.sdm_init_state_segmented.argtypes = [vp, vp, vp, vp, u64, vp, vp, i32]
        L.sdm_set_state.argtypes = [vp, vp, vp, i32]
        L.sdm_get_state.argtypes = [vp, vp, vp, vp, vp, i32]
        L.sdm_coalescence_step.argtypes = [vp, C.POINTER(StepParams), u32, C.POINTER(StepStats)]
        L.sdm_remove_zero.argtypes = [vp, vp]
        L.sdm_spectrum.argtypes = [vp, vp, u32, u32, vp, i32]
        L.sdm_totals.argtypes = [vp, vp, vp, vp]
        L.sdm_check_state.argtypes = [vp, vp, vp]
        L.sdm_rebucket.argtypes = [vp, vp, i32]
        L.sdm_get_schedule.argtypes = [vp, C.POINTER(Schedule)]
        L.sdm_set_schedule.argtypes = [vp, C.POINTER(Schedule)]
        L.sdm_autotune.argtypes = [vp, C.POINTER(StepParams), u32, C.POINTER(Schedule)]
        L.sdm_sync.argtypes = [vp]
        L.sdm_free.argtypes = [vp]
        L.sdm_free.restype = None
        L.sdm_eval_pairs.argtypes = [vp, u32, vp, vp, vp, vp, u64, u32, f64, f64, f64, f64, vp, vp, vp, vp, vp, vp]
        L.sdm_set_profiling.argtypes = [vp, i32]
        L.sdm_get_profile.argtypes = [vp, vp, vp]
        L.sdm_launches_per_step.argtypes = [vp, u32, vp]
        L.sdm_coalescence_step_noalloc.argtypes = [vp, vp, u32, u64, u32, f64, u32, C.POINTER(StepParams), vp]
        L.sdm_surrogate_create.argtypes = [C.POINTER(vp), C.POINTER(SurrogateParams), vp]
        L.sdm_surrogate_free.argtypes = [vp]
        L.sdm_surrogate_free.restype = None
        L.sdm_surrogate_train.argtypes = [vp, u32, u32, C.c_float, vp]
        L.sdm_surrogate_build_mask.argtypes = [vp, C.c_float, vp, vp]
        L.sdm_surrogate_params_io.argtypes = [vp, vp, i32]
        L.sdm_surrogate_info.argtypes = [vp, vp]
        L.sdm_surrogate_loss_grad.argtypes = [vp, vp, vp, u64, vp, vp]
        L.sdm_surrogate_eval.argtypes = [vp, vp, vp, u64, vp]
        L.sdm_attach_surrogate.argtypes = [vp, vp]
        L.sdm_debug_wait_timeout.argtypes = [vp, u32, i32]
        L.sdm_debug_bucket_capacity.argtypes = [vp, u32]
        L.sdm_debug_stage_shortfall.argtypes = [vp, u32, u32]
        for name in EXPORTS:
            if name not in ("sdm_version", "sdm_status_str", "sdm_workspace_bytes", "sdm_free", "sdm_surrogate_free"):
                getattr(L, name).restype = i32
        _lib = L
        return L


def _check(rc, where):
    if rc != 0:
        raise SDMError(rc, where)


def _torch():
    import torch
    return torch


def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _ptr(x, dtype):
    """(pointer, on_device, keepalive) of a numpy array or torch tensor."""
    if x is None:
        return None, 0, None
    if _is_torch(x):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return C.c_void_p(x.data_ptr()), int(x.is_cuda), x
    a = np.ascontiguousarray(x, dtype=dtype)
    return C.c_void_p(a.ctypes.data), 0, a


def current_stream():
    torch = _torch()
    if not torch.cuda.is_available():
        raise RuntimeError("libsdm needs a CUDA device")
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


class State:
    """One SDM system on the current CUDA device (sdm_state)."""

    def __init__(self, n_slots_cap, n_cell, n_attr=1, stream=None, workspace=None):
        self._L = lib()
        self._h = C.c_void_p()
        self.n_cell = int(n_cell)
        self.n_attr = int(n_attr)
        self.cap = int(n_slots_cap)
        self._ws = workspace
        stream = current_stream() if stream is None else C.c_void_p(stream)
        wsp, wsb = (None, 0)
        if workspace is not None:
            wsp, wsb = C.c_void_p(workspace.data_ptr()), workspace.numel() * workspace.element_size()
        _check(self._L.sdm_alloc(C.byref(self._h), self.cap, self.n_cell, self.n_attr, stream, wsp, wsb),
               "sdm_alloc")
        self.n_sd = 0

    # -- lifetime ------------------------------------------------------------
    def close(self):
        if self._h:
            self._L.sdm_free(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- state -----------------------------------------------------------------
    def init(self, xi, attr, dv, kernel_id=None, cell_id=None, cell_start=None):
        """Load an initial population; give either cell_id (any order) or cell_start (grouped)."""
        n = int(xi.shape[0])
        px, dx, kx = _ptr(xi, np.uint64)
        pa, da, ka = _ptr(attr, np.float64)
        pd, dd, kd = _ptr(dv, np.float64)
        pk, dk, kk = _ptr(kernel_id, np.uint8)
        on_dev = dx
        if len({d for d in (dx, da, dd, dk if kernel_id is not None else dx)}) != 1:
            raise ValueError("all arrays must live on the same side (host or device)")
        if cell_start is not None:
            pc, dc, kc = _ptr(cell_start, np.uint32)
            rc = self._L.sdm_init_state_segmented(self._h, px, pa, pc, n, pd, pk, on_dev)
        else:
            pc, dc, kc = _ptr(cell_id, np.uint32)
            rc = self._L.sdm_init_state(self._h, px, pa, pc, n, pd, pk, on_dev)
        _check(rc, "sdm_init_state")
        self.n_sd = n

    def set_state(self, xi, attr):
        px, dx, kx = _ptr(xi, np.uint64)
        pa, da, ka = _ptr(attr, np.float64)
        _check(self._L.sdm_set_state(self._h, px, pa, dx), "sdm_set_state")
        return kx, ka

    def get_state(self, xi=None, attr=None):
        """Copy out (xi, attr, cell_start).  Fills the given numpy arrays / CUDA tensors, or returns new numpy."""
        n = self.n_sd
        if xi is None and attr is None:
            xi = np.empty(n, np.uint64)
            attr = np.empty((self.n_attr, n), np.float64)
        cs = np.empty(self.n_cell + 1, np.uint32)
        px, dx, _ = _ptr(xi, np.uint64)
        pa, da, _ = _ptr(attr, np.float64)
        _check(self._L.sdm_get_state(self._h, px, pa, None, None, dx), "sdm_get_state")
        _check(self._L.sdm_get_state(self._h, None, None, C.c_void_p(cs.ctypes.data), None, 0), "sdm_get_state")
        return xi, attr, cs

    # -- the step ----------------------------------------------------------------
    def step(self, dt=1.0, seed=42, step=0, n_steps=1, precision="fp64", golovin_b=1500.0, d_step=None,
             stats=False, shuffle="prp", efield=0.0):
        p = StepParams(float(dt), float(golovin_b), int(seed), int(step), PREC[precision], SHUFFLE[shuffle], 0,
                       None if d_step is None else d_step.data_ptr(), float(efield))
        st = StepStats()
        _check(self._L.sdm_coalescence_step(self._h, C.byref(p), int(n_steps), C.byref(st) if stats else None),
               "sdm_coalescence_step")
        return st.as_dict() if stats else None

    def remove_zero(self):
        n = C.c_uint64()
        _check(self._L.sdm_remove_zero(self._h, C.byref(n)), "sdm_remove_zero")
        return int(n.value)

    def spectrum(self, r_edges, cell=None):
        r = np.ascontiguousarray(r_edges, np.float64)
        out = np.zeros(len(r) - 1, np.float64)
        _check(self._L.sdm_spectrum(self._h, C.c_void_p(r.ctypes.data), len(r) - 1,
                                    0xFFFFFFFF if cell is None else int(cell), C.c_void_p(out.ctypes.data), 0),
               "sdm_spectrum")
        return out

    def totals(self):
        n, m, live = C.c_uint64(), C.c_double(), C.c_uint64()
        _check(self._L.sdm_totals(self._h, C.byref(n), C.byref(m), C.byref(live)), "sdm_totals")
        return int(n.value), float(m.value), int(live.value)

    def rebucket(self, cell_id):
        """Move every live SD to the cell cell_id[slot] names (numpy uint32 on the host or a CUDA
        int32/uint32 tensor); within a cell SDs keep their old slot order."""
        if hasattr(cell_id, "data_ptr"):
            _check(self._L.sdm_rebucket(self._h, C.c_void_p(cell_id.data_ptr()), 1), "sdm_rebucket")
        else:
            c = np.ascontiguousarray(cell_id, np.uint32)
            _check(self._L.sdm_rebucket(self._h, c.ctypes.data_as(C.c_void_p), 0), "sdm_rebucket")

    def check(self):
        """Counts of slots breaking the state's invariants: (live-prefix rule, stale volume keys)."""
        bl, bk = C.c_uint64(), C.c_uint64()
        _check(self._L.sdm_check_state(self._h, C.byref(bl), C.byref(bk)), "sdm_check_state")
        return int(bl.value), int(bk.value)

    def attach_surrogate(self, surrogate):
        """Use a trained Surrogate for precision="surrogate" steps (None detaches); the State keeps a
        reference so the surrogate outlives its use."""
        self._surrogate = surrogate
        _check(self._L.sdm_attach_surrogate(self._h, surrogate._h if surrogate is not None else None),
               "sdm_attach_surrogate")

    def sync(self):
        _check(self._L.sdm_sync(self._h), "sdm_sync")

    # -- failure-path self-tests -------------------------------------------------
    def debug_wait_timeout(self, spin_limit, withhold=True):
        _check(self._L.sdm_debug_wait_timeout(self._h, int(spin_limit), int(bool(withhold))),
               "sdm_debug_wait_timeout")

    def debug_bucket_capacity(self, cap):
        _check(self._L.sdm_debug_bucket_capacity(self._h, int(cap)), "sdm_debug_bucket_capacity")

    def debug_stage_shortfall(self, extra_bytes, wait_log2=0):
        _check(self._L.sdm_debug_stage_shortfall(self._h, int(extra_bytes), int(wait_log2)),
               "sdm_debug_stage_shortfall")

    # -- schedule ------------------------------------------------------------------
    @property
    def schedule(self):
        s = Schedule()
        _check(self._L.sdm_get_schedule(self._h, C.byref(s)), "sdm_get_schedule")
        return s.as_dict()

    def set_schedule(self, tile_slots=None, tile_threads=None, bucket_target=None, persistent=None):
        """Set the launch schedule; a field left as None keeps its current value."""
        cur = self.schedule
        s = Schedule(cur["tile_slots"] if tile_slots is None else tile_slots,
                     cur["tile_threads"] if tile_threads is None else tile_threads,
                     cur["bucket_target"] if bucket_target is None else bucket_target,
                     cur["persistent"] if persistent is None else persistent)
        _check(self._L.sdm_set_schedule(self._h, C.byref(s)), "sdm_set_schedule")

    def autotune(self, dt=1.0, seed=42, step=0, n_steps=3, precision="fp64", golovin_b=1500.0, shuffle="prp"):
        p = StepParams(float(dt), float(golovin_b), int(seed), int(step), PREC[precision], SHUFFLE[shuffle], 0, None)
        s = Schedule()
        _check(self._L.sdm_autotune(self._h, C.byref(p), int(n_steps), C.byref(s)), "sdm_autotune")
        return s.as_dict()

    # -- profiling ----------------------------------------------------------------
    KERNEL_KINDS = ("small_cell_kernels", "big_scatter_kernel", "big_finish_kernel", "big_prp_kernel")

    def set_profiling(self, on=True):
        _check(self._L.sdm_set_profiling(self._h, int(bool(on))), "sdm_set_profiling")

    def profile(self):
        """{kernel name: (launches, total ms)} since profiling was enabled."""
        n = (C.c_uint32 * 4)()
        ms = (C.c_double * 4)()
        _check(self._L.sdm_get_profile(self._h, n, ms), "sdm_get_profile")
        return {k: (int(n[i]), float(ms[i])) for i, k in enumerate(self.KERNEL_KINDS)}

    def launches_per_step(self, shuffle="prp"):
        n = C.c_uint32()
        _check(self._L.sdm_launches_per_step(self._h, SHUFFLE[shuffle], C.byref(n)), "sdm_launches_per_step")
        return int(n.value)

    # -- Step 2 alone (testing) ---------------------------------------------------
    def eval_pairs(self, kernel_id, v1, v2, xi1, xi2, n_cell_sd, dv, dt=1.0, golovin_b=1500.0, lite=False,
                   bound=False, efield=0.0):
        """All arguments are CUDA tensors; returns (p64, p32, err32) CUDA tensors, with lite=True
        also the second filter's (plite, errlite), with bound=True also the early exit's bound."""
        torch = _torch()
        n = v1.numel()
        p64 = torch.empty(n, dtype=torch.float64, device=v1.device)
        p32 = torch.empty(n, dtype=torch.float32, device=v1.device)
        e32 = torch.empty(n, dtype=torch.float32, device=v1.device)
        pl = torch.empty(n, dtype=torch.float64, device=v1.device) if lite else None
        el = torch.empty(n, dtype=torch.float64, device=v1.device) if lite else None
        pu = torch.empty(n, dtype=torch.float32, device=v1.device) if bound else None
        _check(self._L.sdm_eval_pairs(self._h, int(kernel_id), C.c_void_p(v1.data_ptr()), C.c_void_p(v2.data_ptr()),
                                      C.c_void_p(xi1.data_ptr()), C.c_void_p(xi2.data_ptr()), n, int(n_cell_sd),
                                      float(dv), float(dt), float(golovin_b), float(efield),
                                      C.c_void_p(p64.data_ptr()),
                                      C.c_void_p(p32.data_ptr()), C.c_void_p(e32.data_ptr()),
                                      C.c_void_p(pl.data_ptr() if lite else None),
                                      C.c_void_p(el.data_ptr() if lite else None),
                                      C.c_void_p(pu.data_ptr() if bound else None)), "sdm_eval_pairs")
        out = (p64, p32, e32) + ((pl, el) if lite else ()) + ((pu,) if bound else ())
        return out


class Surrogate:
    """Learned stand-in for the gravitational kernel (sdm_surrogate_*): create, train on the
    GPU, build the fallback mask, attach to a State for precision="surrogate"."""

    N_PARAM = 8577

    def __init__(self, n_train=10_000_000, seed=7, r_min=1e-6, r_max=3e-3, stream=None):
        self._L = lib()
        torch = _torch()
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        p = SurrogateParams(int(n_train), int(seed), float(r_min), float(r_max))
        h = C.c_void_p()
        _check(self._L.sdm_surrogate_create(C.byref(h), C.byref(p), C.c_void_p(self.stream.cuda_stream)),
               "sdm_surrogate_create")
        self._h = h

    def train(self, steps, batch=8192, lr=2e-3):
        loss = np.zeros(steps, np.float32)
        _check(self._L.sdm_surrogate_train(self._h, int(steps), int(batch), float(lr),
                                           loss.ctypes.data_as(C.c_void_p)), "sdm_surrogate_train")
        return loss

    def build_mask(self, tol=0.01):
        frac = C.c_double()
        err = np.zeros(256 * 256, np.float32)
        _check(self._L.sdm_surrogate_build_mask(self._h, float(tol), C.byref(frac), err.ctypes.data_as(C.c_void_p)),
               "sdm_surrogate_build_mask")
        return float(frac.value), err.reshape(256, 256)

    def params(self):
        w = np.zeros(self.N_PARAM, np.float32)
        _check(self._L.sdm_surrogate_params_io(self._h, w.ctypes.data_as(C.c_void_p), 0), "sdm_surrogate_params_io")
        return w

    def set_params(self, w):
        w = np.ascontiguousarray(w, np.float32)
        _check(self._L.sdm_surrogate_params_io(self._h, w.ctypes.data_as(C.c_void_p), 1), "sdm_surrogate_params_io")

    def info(self):
        out = np.zeros(6, np.float64)
        _check(self._L.sdm_surrogate_info(self._h, out.ctypes.data_as(C.c_void_p)), "sdm_surrogate_info")
        return dict(zip(["c0", "c1", "mu", "sigma", "k_floor", "r_ratio"], out.tolist()))

    def loss_grad(self, x, t):
        """x: CUDA float32 [n, 2], t: CUDA float32 [n] -> (loss, grad numpy [8577])."""
        loss = C.c_float()
        grad = np.zeros(self.N_PARAM, np.float32)
        _check(self._L.sdm_surrogate_loss_grad(self._h, C.c_void_p(x.data_ptr()), C.c_void_p(t.data_ptr()), x.shape[0],
                                               C.byref(loss), grad.ctypes.data_as(C.c_void_p)),
               "sdm_surrogate_loss_grad")
        return float(loss.value), grad

    def eval(self, R, r):
        """R, r: CUDA float64 radii -> CUDA float32 K^ (-1 where the plain kernel is used)."""
        torch = _torch()
        K = torch.empty(R.numel(), dtype=torch.float32, device=R.device)
        _check(self._L.sdm_surrogate_eval(self._h, C.c_void_p(R.data_ptr()), C.c_void_p(r.data_ptr()), R.numel(),
                                          C.c_void_p(K.data_ptr())), "sdm_surrogate_eval")
        return K

    def close(self):
        if getattr(self, "_h", None):
            self._L.sdm_surrogate_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def from_inputs(s, n_attr=1, extra_attrs=None, stream=None, device_arrays=False):
    """Create and initialise a State from an inputs.* workload dict."""
    n = len(s["xi"])
    st = State(max(n, 1), len(s["dv"]), n_attr, stream=stream)
    attr = s["v"][None, :] if extra_attrs is None else np.vstack([s["v"][None, :], extra_attrs])
    if device_arrays:
        torch = _torch()
        st.init(torch.from_numpy(s["xi"].view(np.int64)).cuda(), torch.from_numpy(np.ascontiguousarray(attr)).cuda(),
                torch.from_numpy(s["dv"]).cuda(), torch.from_numpy(s["kernel_id"]).cuda(),
                cell_start=torch.from_numpy(s["cell_start"].view(np.int32)).cuda())
    else:
        st.init(s["xi"], attr, s["dv"], s["kernel_id"], cell_start=s["cell_start"])
    return st
