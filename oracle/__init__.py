"""CPU oracle of the SDM coalescence step (Bartman & Arabas, arXiv:2101.06318).

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package; the product (the CUDA
library and its binding) never does.  It shares no code with the CUDA path.

The arithmetic lives in ``sdm_oracle.c`` (plain C99, FP64, FMA contraction
off); this module compiles it on first use with gcc and exposes it through
ctypes with numpy arrays.  Which passage of the paper each function follows is
stated in the C file's header.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sdm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libsdm_oracle.so")
_CFLAGS = ["-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC"]
_lock = threading.Lock()
_lib = None

KERNEL_GOLOVIN = 0
KERNEL_GRAVITATIONAL = 1
KERNEL_ELECTRIC = 2
SHUFFLE = {"sort": 0, "prp": 1}


def build(force: bool = False) -> str:
    """Compile the oracle shared library (idempotent)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", *_CFLAGS, "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class Stats(C.Structure):
    _fields_ = [("n_pairs", C.c_uint64), ("n_collisions", C.c_uint64),
                ("n_removed", C.c_uint64), ("sum_gamma", C.c_uint64)]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


def _p(t):
    return C.POINTER(t)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            u32, u64, f64, i32 = C.c_uint32, C.c_uint64, C.c_double, C.c_int
            L.sdmo_philox4x32_10.argtypes = [_p(u32), _p(u32), _p(u32)]
            L.sdmo_shuffle_key.argtypes = [u64, u32, u32, u32]
            L.sdmo_shuffle_key.restype = u32
            L.sdmo_phi_u53.argtypes = [u64, u32, u32, u32]
            L.sdmo_phi_u53.restype = u64
            L.sdmo_phi.argtypes = [u64, u32, u32, u32]
            L.sdmo_phi.restype = f64
            L.sdmo_kernel_golovin.argtypes = [f64, f64, f64]
            L.sdmo_kernel_golovin.restype = f64
            L.sdmo_cbrt.argtypes = [f64]
            L.sdmo_cbrt.restype = f64
            L.sdmo_radius.argtypes = [f64]
            L.sdmo_radius.restype = f64
            L.sdmo_terminal_velocity.argtypes = [f64]
            L.sdmo_terminal_velocity.restype = f64
            L.sdmo_efficiency.argtypes = [f64, f64]
            L.sdmo_efficiency.restype = f64
            L.sdmo_kernel_gravitational.argtypes = [f64, f64]
            L.sdmo_kernel_gravitational.restype = f64
            L.sdmo_kernel.argtypes = [i32, f64, f64, f64, f64]
            L.sdmo_kernel.restype = f64
            L.sdmo_kernel_electric.argtypes = [f64, f64, f64]
            L.sdmo_kernel_electric.restype = f64
            L.sdmo_efficiency_field.argtypes = [f64, f64, f64]
            L.sdmo_efficiency_field.restype = f64
            L.sdmo_pair_scale.argtypes = [u64]
            L.sdmo_pair_scale.restype = f64
            L.sdmo_pair_prob.argtypes = [f64, u64, u64, f64, f64, f64]
            L.sdmo_pair_prob.restype = f64
            L.sdmo_gamma_tilde.argtypes = [f64, f64, u64, u64]
            L.sdmo_gamma_tilde.restype = u64
            L.sdmo_update_pair.argtypes = [_p(u64), _p(f64), u32, u64, u64, u64, f64, f64]
            L.sdmo_update_pair.restype = u64
            step_args = [u64, u32, _p(u32), _p(u64), _p(f64), u32, _p(f64), _p(C.c_uint8),
                         f64, f64, f64, u64, u32]
            L.sdmo_step.argtypes = step_args + [i32, _p(Stats)]
            L.sdmo_step.restype = i32
            L.sdmo_run.argtypes = step_args + [u32, i32, _p(Stats)]
            L.sdmo_run.restype = i32
            L.sdmo_compact.argtypes = [u64, u32, _p(u32), _p(u64), _p(f64), u32]
            L.sdmo_prp_keys.argtypes = [u64, u32, u32, _p(u32)]
            L.sdmo_prp.argtypes = [u32, u32, _p(u32)]
            L.sdmo_prp.restype = u32
            L.sdmo_prp_perm.argtypes = [u32, _p(u32), _p(u32)]
            L.sdmo_totals.argtypes = [u64, _p(u64), _p(f64), _p(u64), _p(u64), _p(f64)]
            L.sdmo_i1e.argtypes = [f64]
            L.sdmo_i1e.restype = f64
            L.sdmo_golovin_phi.argtypes = [f64, f64, f64, f64, f64]
            L.sdmo_golovin_phi.restype = f64
            _lib = L
    return _lib


def _ptr(a, t):
    return a.ctypes.data_as(C.POINTER(t))


# ----------------------------------------------------------------------------
# thin numpy-facing wrappers
# ----------------------------------------------------------------------------

def philox(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    o = np.zeros(4, np.uint32)
    lib().sdmo_philox4x32_10(_ptr(c, C.c_uint32), _ptr(k, C.c_uint32), _ptr(o, C.c_uint32))
    return o


def shuffle_key(seed, cell, step, l):
    return int(lib().sdmo_shuffle_key(seed, cell, step, l))


def phi_u53(seed, cell, step, m):
    return int(lib().sdmo_phi_u53(seed, cell, step, m))


def phi(seed, cell, step, m):
    return float(lib().sdmo_phi(seed, cell, step, m))


def kernel(kid, v1, v2, golovin_b=1500.0, efield=0.0):
    return float(lib().sdmo_kernel(int(kid), float(v1), float(v2), float(golovin_b), float(efield)))


def efficiency_field(R, q, eps):
    return float(lib().sdmo_efficiency_field(float(R), float(q), float(eps)))


def cbrt(x):
    return float(lib().sdmo_cbrt(float(x)))


def radius(v):
    return float(lib().sdmo_radius(float(v)))


def terminal_velocity(r):
    return float(lib().sdmo_terminal_velocity(float(r)))


def efficiency(R, q):
    return float(lib().sdmo_efficiency(float(R), float(q)))


def pair_scale(n):
    return float(lib().sdmo_pair_scale(int(n)))


def pair_prob(K, xi_a, xi_b, scale, dt, dv):
    return float(lib().sdmo_pair_prob(float(K), int(xi_a), int(xi_b), float(scale), float(dt), float(dv)))


def gamma_tilde(p, phi_, xi_j, xi_k):
    return int(lib().sdmo_gamma_tilde(float(p), float(phi_), int(xi_j), int(xi_k)))


def update_pair(xi, attr, first, second, p, phi_):
    """In-place single-pair update on numpy arrays; attr is [n_attr, n]."""
    assert xi.dtype == np.uint64 and attr.dtype == np.float64 and attr.flags.c_contiguous
    return int(lib().sdmo_update_pair(_ptr(xi, C.c_uint64), _ptr(attr, C.c_double), attr.shape[0],
                                      attr.shape[1], first, second, float(p), float(phi_)))


PRP_MIN_N = 257          # smaller cells are shuffled by sorting keys
FOUR_PI_OVER_THREE = 4.18879020478639053


def prp_keys(seed, cell, step):
    K = np.zeros(8, np.uint32)
    lib().sdmo_prp_keys(int(seed), int(cell), int(step), _ptr(K, C.c_uint32))
    return K


def prp(q, n, K):
    K = np.ascontiguousarray(K, np.uint32)
    return int(lib().sdmo_prp(int(q), int(n), _ptr(K, C.c_uint32)))


def prp_perm(n, K):
    """The PRP shuffle's whole permutation of [0, n): out[q] = prp(q, n, K)."""
    K = np.ascontiguousarray(K, np.uint32)
    out = np.empty(int(n), np.uint32)
    lib().sdmo_prp_perm(int(n), _ptr(K, C.c_uint32), _ptr(out, C.c_uint32))
    return out


def i1e(x):
    return float(lib().sdmo_i1e(float(x)))


def golovin_phi(v, t, vbar, n0, b):
    return float(lib().sdmo_golovin_phi(float(v), float(t), float(vbar), float(n0), float(b)))


class System:
    """A slot-model SDM system held in numpy arrays, stepped by the oracle.

    The storage is kept compacted (each cell's live SDs first, in order), as
    after every step; ``shuffle`` selects the Step 1 contract ("sort" or "prp").
    """

    def __init__(self, xi, attr, cell_start, dv, kernel_id=None, golovin_b=1500.0, shuffle="prp", efield=0.0):
        self.xi = np.ascontiguousarray(xi, dtype=np.uint64).copy()
        attr = np.asarray(attr, dtype=np.float64)
        if attr.ndim == 1:
            attr = attr[None, :]
        self.attr = np.ascontiguousarray(attr).copy()
        self.cell_start = np.ascontiguousarray(cell_start, dtype=np.uint32).copy()
        self.n_cell = len(self.cell_start) - 1
        self.dv = np.ascontiguousarray(np.broadcast_to(np.asarray(dv, np.float64), (self.n_cell,))).copy()
        if kernel_id is None:
            kernel_id = np.zeros(self.n_cell, np.uint8)
        self.kernel_id = np.ascontiguousarray(
            np.broadcast_to(np.asarray(kernel_id, np.uint8), (self.n_cell,))).copy()
        self.golovin_b = float(golovin_b)
        self.efield = float(efield)           # field parameter of the electric-field kernel
        self.shuffle = shuffle
        assert self.attr.shape[1] == self.xi.shape[0]
        lib().sdmo_compact(self.xi.shape[0], self.n_cell, _ptr(self.cell_start, C.c_uint32),
                           _ptr(self.xi, C.c_uint64), _ptr(self.attr, C.c_double), self.attr.shape[0])

    @property
    def v(self):
        return self.attr[0]

    def _args(self):
        return (self.xi.shape[0], self.n_cell, _ptr(self.cell_start, C.c_uint32),
                _ptr(self.xi, C.c_uint64), _ptr(self.attr, C.c_double), self.attr.shape[0],
                _ptr(self.dv, C.c_double), _ptr(self.kernel_id, C.c_uint8), self.golovin_b, self.efield)

    def step(self, dt, seed, step):
        st = Stats()
        rc = lib().sdmo_step(*self._args(), float(dt), int(seed), int(step), SHUFFLE[self.shuffle], C.byref(st))
        if rc:
            raise RuntimeError(f"sdmo_step failed: {rc}")
        return st.as_dict()

    def run(self, dt, seed, step0, n_steps):
        st = Stats()
        rc = lib().sdmo_run(*self._args(), float(dt), int(seed), int(step0), int(n_steps), SHUFFLE[self.shuffle],
                            C.byref(st))
        if rc:
            raise RuntimeError(f"sdmo_run failed: {rc}")
        return st.as_dict()

    def totals(self):
        nt, nl, m = C.c_uint64(), C.c_uint64(), C.c_double()
        lib().sdmo_totals(self.xi.shape[0], _ptr(self.xi, C.c_uint64), _ptr(self.attr, C.c_double),
                          C.byref(nt), C.byref(nl), C.byref(m))
        return int(nt.value), int(nl.value), float(m.value)

    def spectrum(self, r_edges, rho=1000.0, cell_lo=0, cell_hi=None):
        """Mass spectrum dm/dln r (Sec. 4) of the cells [cell_lo, cell_hi): bin b holds the live SDs
        with ve[b] <= v < ve[b+1], ve = (4 pi/3) r^3 (evaluated as ((4 pi/3) r) r) r);
        out[b] = rho S_b / (V (ln r[b+1] - ln r[b])) with S_b the sum of the bin's terms xi v (each
        product rounded once) taken exactly and rounded once (math.fsum), V the cells' dV summed in
        cell order."""
        r = np.ascontiguousarray(r_edges, np.float64)
        nb = len(r) - 1
        ve = ((FOUR_PI_OVER_THREE * r) * r) * r
        cell_hi = self.n_cell if cell_hi is None else cell_hi
        s0, s1 = int(self.cell_start[cell_lo]), int(self.cell_start[cell_hi])
        xi = self.xi[s0:s1]
        v = self.attr[0, s0:s1]
        sel = (xi != 0) & (ve[0] <= v) & (v < ve[nb])
        t = xi[sel].astype(np.float64) * v[sel]
        b = np.searchsorted(ve, v[sel], side="right") - 1          # ve[b] <= v < ve[b + 1]
        order = np.argsort(b, kind="stable")
        bounds = np.searchsorted(b[order], np.arange(nb + 1))
        V = 0.0
        for c in range(cell_lo, cell_hi):
            V = V + float(self.dv[c])
        out = np.zeros(nb, np.float64)
        for k in range(nb):
            msum = math.fsum(t[order[bounds[k]:bounds[k + 1]]].tolist())
            dlnr = math.log(float(r[k + 1])) - math.log(float(r[k]))
            out[k] = rho * msum / (V * dlnr)
        return out

    def rebucket(self, cell_id):
        """Displacement between steps: every live SD moves to the cell ``cell_id[slot]`` names.

        The paper keeps a cell index per SD and regroups the SDs by it (its cell_start array,
        Sec. 3); the slot model here keeps each cell's slot range fixed, so a cell's width is its
        capacity.  Within a cell the SDs keep their old slot order (a stable sort by the new cell
        index, numpy's stable argsort being the sort), the live ones first.  Returns False, with
        the state unchanged, when an index is out of range or a cell receives more SDs than its
        width; True otherwise.
        """
        cell_id = np.asarray(cell_id, np.int64)
        live = np.flatnonzero(self.xi)
        newc = cell_id[live]
        if len(newc) and (newc.min() < 0 or newc.max() >= self.n_cell):
            return False
        counts = np.bincount(newc, minlength=self.n_cell)
        width = np.diff(self.cell_start.astype(np.int64))
        if np.any(counts > width):
            return False
        order = np.argsort(newc, kind="stable")
        src = live[order]
        cells = newc[order]
        first = np.concatenate([[0], np.cumsum(counts)[:-1]])      # position of each cell's first SD
        dest = self.cell_start[cells].astype(np.int64) + (np.arange(len(order)) - first[cells])
        xi = np.zeros_like(self.xi)
        attr = np.zeros_like(self.attr)
        xi[dest] = self.xi[src]
        attr[:, dest] = self.attr[:, src]
        self.xi, self.attr = xi, attr
        return True

    def copy(self):
        return System(self.xi, self.attr, self.cell_start, self.dv, self.kernel_id, self.golovin_b, self.shuffle,
                      self.efield)
