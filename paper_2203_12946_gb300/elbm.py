"""Thin ctypes binding of the C ABI in ``include/elbm.h`` (argument marshalling only).

Every entry point of the library is exposed under its C name with the same
arguments; pointers may be given as integers, numpy arrays (host memory) or
torch tensors (``data_ptr()``, device memory).  Every step of the method runs in
the CUDA kernels of ``libelbm.so``; if the library cannot be loaded these
functions raise, they never fall back to another implementation.

``Simulation`` is a convenience wrapper that lets PyTorch own the device
buffers and supplies torch's current CUDA stream.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

ELBM_OK = 0
ELBM_ERR_ARG = -1
ELBM_ERR_UNSUPPORTED = -2
ELBM_ERR_CUDA = -3
ELBM_ERR_NONPHYSICAL = -4
ELBM_ERR_TIMEOUT = -5

ELBM_D2Q9 = 9
ELBM_D3Q27 = 27
ELBM_BC_PERIODIC = 0
ELBM_STORE_F64, ELBM_STORE_F32, ELBM_STORE_F16DEV, ELBM_STORE_BF16DEV, ELBM_STORE_F32DEV = 0, 1, 2, 3, 4
ELBM_ALPHA_HIGHER, ELBM_ALPHA_LOWER, ELBM_ALPHA_LBGK, ELBM_ALPHA_ITERATE1 = 0, 1, 2, 3
ELBM_B_DERIVED, ELBM_B_PRINTED = 0, 1
ELBM_MEM_DEVICE, ELBM_MEM_HOST = 0, 1
ELBM_KERNEL_AUTO, ELBM_KERNEL_DIRECT, ELBM_KERNEL_ROWS = 0, 1, 2
ELBM_BATCH_GRAPH, ELBM_BATCH_LAUNCHES, ELBM_BATCH_PER_DOMAIN, ELBM_BATCH_PERSISTENT, ELBM_BATCH_AUTO = 0, 1, 2, 3, 4
ELBM_BRANCH_CUTOFF, ELBM_BRANCH_SOLVED, ELBM_BRANCH_CLAMPED = 0, 1, 2
ELBM_HIST_BINS = 256
ELBM_NOALLOC_SCRATCH_BYTES = 4096

STORAGE_NAMES = {"f64": ELBM_STORE_F64, "f32": ELBM_STORE_F32, "f16dev": ELBM_STORE_F16DEV,
                 "bf16dev": ELBM_STORE_BF16DEV, "f32dev": ELBM_STORE_F32DEV}
STORAGE_BYTES = {ELBM_STORE_F64: 8, ELBM_STORE_F32: 4, ELBM_STORE_F16DEV: 2, ELBM_STORE_BF16DEV: 2,
                 ELBM_STORE_F32DEV: 4}
# numpy type of one stored element (bfloat16 as its raw 16 bits)
STORAGE_NUMPY = {ELBM_STORE_F64: np.float64, ELBM_STORE_F32: np.float32, ELBM_STORE_F16DEV: np.float16,
                 ELBM_STORE_BF16DEV: np.uint16, ELBM_STORE_F32DEV: np.float32}


def dev_unit(D: int, rho0: float = 1.0) -> float:
    """R of the deviation storages (include/elbm.h): 6^-D rho0 rounded to FP32; population i
    is stored as f_i - k_i R with w_i = k_i 6^-D."""
    return float(np.float32((1.0 / 36.0 if D == 2 else 1.0 / 216.0) * rho0))

EXPORTED = ["elbm_default_opts", "elbm_population_bytes", "elbm_create", "elbm_destroy",
            "elbm_last_error", "elbm_bind_buffers", "elbm_set_stream", "elbm_init_equilibrium",
            "elbm_step", "elbm_moments", "elbm_alpha_field", "elbm_diagnostics",
            "elbm_get_populations", "elbm_set_populations", "elbm_step_count", "elbm_synchronize",
            "elbm_diagnostics_noalloc",
            "elbm_batch_create", "elbm_batch_destroy", "elbm_batch_last_error", "elbm_batch_info",
            "elbm_batch_init_equilibrium", "elbm_batch_step", "elbm_batch_tune", "elbm_batch_moments",
            "elbm_batch_diagnostics", "elbm_batch_get_populations", "elbm_batch_set_populations",
            "elbm_batch_synchronize", "elbm_adjoint_step", "elbm_kinetic_energy", "elbm_equilibrium_vjp",
            "elbm_subgrid_viscosity", "elbm_adjoint_step_force", "elbm_set_force", "elbm_step_diag",
            "elbm_batch_check_wait_timeout", "elbm_batch_tune_persistent"]


class elbm_opts(ctypes.Structure):
    _fields_ = [("storage", ctypes.c_int), ("alpha_mode", ctypes.c_int), ("cutoff", ctypes.c_int),
                ("b_variant", ctypes.c_int), ("device", ctypes.c_int), ("rho0", ctypes.c_double),
                ("stream", ctypes.c_void_p), ("kernel", ctypes.c_int)]


class elbm_diag(ctypes.Structure):
    _fields_ = [("mass", ctypes.c_double), ("momentum", ctypes.c_double * 3), ("H", ctypes.c_double),
                ("dH_max", ctypes.c_double), ("alpha_min", ctypes.c_double),
                ("alpha_max", ctypes.c_double), ("alpha_mean", ctypes.c_double),
                ("n_nodes", ctypes.c_int64), ("n_cutoff", ctypes.c_int64),
                ("n_solved", ctypes.c_int64), ("n_clamped", ctypes.c_int64),
                ("n_nonpositive", ctypes.c_int64), ("n_dH_positive", ctypes.c_int64),
                ("n_xmax_band", ctypes.c_int64 * 4)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["momentum"] = list(self.momentum)
        d["n_xmax_band"] = list(self.n_xmax_band)
        return d


class ElbmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"elbm error {code}: {msg}")
        self.code = code


_lib = None
_lock = threading.Lock()


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libelbm.so (building it first if it is missing and nvcc exists)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(_build.LIB):
            if not build_if_missing:
                raise ImportError(f"libelbm.so not built at {_build.LIB}")
            _build.build()
        lib = ctypes.CDLL(_build.LIB)
        P = ctypes.c_void_p
        i64 = ctypes.c_int64
        sig = {
            "elbm_default_opts": (None, [ctypes.POINTER(elbm_opts)]),
            "elbm_population_bytes": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(i64), ctypes.c_int,
                                                     ctypes.POINTER(ctypes.c_size_t)]),
            "elbm_create": (ctypes.c_int, [ctypes.POINTER(P), ctypes.c_int, ctypes.POINTER(i64),
                                           ctypes.c_double, ctypes.c_int, ctypes.POINTER(elbm_opts)]),
            "elbm_destroy": (None, [P]),
            "elbm_last_error": (ctypes.c_char_p, [P]),
            "elbm_bind_buffers": (ctypes.c_int, [P, P, P, ctypes.c_size_t]),
            "elbm_set_stream": (ctypes.c_int, [P, P]),
            "elbm_init_equilibrium": (ctypes.c_int, [P, P, P, ctypes.c_int]),
            "elbm_step": (ctypes.c_int, [P, i64]),
            "elbm_moments": (ctypes.c_int, [P, P, P, ctypes.c_int]),
            "elbm_alpha_field": (ctypes.c_int, [P, P, P, ctypes.c_int]),
            "elbm_diagnostics": (ctypes.c_int, [P, ctypes.POINTER(elbm_diag), P]),
            "elbm_get_populations": (ctypes.c_int, [P, P, ctypes.c_int]),
            "elbm_set_populations": (ctypes.c_int, [P, P, ctypes.c_int]),
            "elbm_step_count": (ctypes.c_int, [P, ctypes.POINTER(i64)]),
            "elbm_synchronize": (ctypes.c_int, [P]),
            "elbm_diagnostics_noalloc": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(i64), ctypes.c_double,
                                                        ctypes.POINTER(elbm_opts), P,
                                                        ctypes.POINTER(elbm_diag), P]),
            "elbm_batch_create": (ctypes.c_int, [ctypes.POINTER(P), ctypes.c_int, ctypes.c_int,
                                                 ctypes.POINTER(i64), ctypes.POINTER(ctypes.c_double),
                                                 ctypes.POINTER(elbm_opts)]),
            "elbm_batch_destroy": (None, [P]),
            "elbm_batch_last_error": (ctypes.c_char_p, [P]),
            "elbm_batch_info": (ctypes.c_int, [P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(i64),
                                               ctypes.POINTER(ctypes.c_int)]),
            "elbm_batch_init_equilibrium": (ctypes.c_int, [P, ctypes.c_int, P, P, ctypes.c_int]),
            "elbm_batch_step": (ctypes.c_int, [P, i64, ctypes.c_int]),
            "elbm_batch_tune": (ctypes.c_int, [P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]),
            "elbm_batch_moments": (ctypes.c_int, [P, ctypes.c_int, P, P, ctypes.c_int]),
            "elbm_batch_diagnostics": (ctypes.c_int, [P, ctypes.c_int, ctypes.POINTER(elbm_diag), P]),
            "elbm_batch_get_populations": (ctypes.c_int, [P, ctypes.c_int, P, ctypes.c_int]),
            "elbm_batch_set_populations": (ctypes.c_int, [P, ctypes.c_int, P, ctypes.c_int]),
            "elbm_batch_synchronize": (ctypes.c_int, [P]),
            "elbm_batch_check_wait_timeout": (ctypes.c_int, [P]),
            "elbm_batch_tune_persistent": (ctypes.c_int, [P, ctypes.POINTER(ctypes.c_int),
                                                          ctypes.POINTER(ctypes.c_double)]),
            "elbm_adjoint_step": (ctypes.c_int, [P, P, P, P]),
            "elbm_kinetic_energy": (ctypes.c_int, [P, P, ctypes.POINTER(ctypes.c_double), P]),
            "elbm_equilibrium_vjp": (ctypes.c_int, [P, P, P, P, P, P]),
            "elbm_subgrid_viscosity": (ctypes.c_int, [P, P, ctypes.c_int]),
            "elbm_adjoint_step_force": (ctypes.c_int, [P, P, P, P, P]),
            "elbm_set_force": (ctypes.c_int, [P, P]),
            "elbm_step_diag": (ctypes.c_int, [P, ctypes.c_int64, P, P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _ptr(x):
    """Address of a numpy array, torch tensor, ctypes object or integer (None -> NULL)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    return ctypes.addressof(x)


def _check(h, code, what):
    if code != ELBM_OK:
        msg = load().elbm_last_error(h)
        raise ElbmError(code, f"{what}: {msg.decode() if msg else ''}")
    return code


def _dims(dims):
    d = (list(dims) + [1, 1])[:3]
    return (ctypes.c_int64 * 3)(*[int(v) for v in d])


# ----------------------------------------------------------------------------
# C entry points (same names and argument order as include/elbm.h; these raise
# ElbmError instead of returning a non-zero status)
# ----------------------------------------------------------------------------

def elbm_default_opts() -> elbm_opts:
    o = elbm_opts()
    load().elbm_default_opts(ctypes.byref(o))
    return o


def elbm_population_bytes(lattice, dims, storage) -> int:
    out = ctypes.c_size_t(0)
    _check(None, load().elbm_population_bytes(int(lattice), _dims(dims), int(storage), ctypes.byref(out)),
           "elbm_population_bytes")
    return int(out.value)


def elbm_create(lattice, dims, beta, bc=ELBM_BC_PERIODIC, opts: elbm_opts | None = None) -> int:
    h = ctypes.c_void_p(None)
    _check(None, load().elbm_create(ctypes.byref(h), int(lattice), _dims(dims), float(beta), int(bc),
                                    None if opts is None else ctypes.byref(opts)), "elbm_create")
    return h.value


def elbm_destroy(h) -> None:
    load().elbm_destroy(h)


def elbm_last_error(h=None) -> str:
    m = load().elbm_last_error(h)
    return m.decode() if m else ""


def elbm_bind_buffers(h, pop_a, pop_b, nbytes) -> None:
    _check(h, load().elbm_bind_buffers(h, _ptr(pop_a), _ptr(pop_b), int(nbytes)), "elbm_bind_buffers")


def elbm_set_stream(h, stream) -> None:
    _check(h, load().elbm_set_stream(h, stream), "elbm_set_stream")


def elbm_init_equilibrium(h, rho, u, where=ELBM_MEM_DEVICE) -> None:
    _check(h, load().elbm_init_equilibrium(h, _ptr(rho), _ptr(u), int(where)), "elbm_init_equilibrium")


def elbm_step(h, n=1) -> None:
    _check(h, load().elbm_step(h, int(n)), "elbm_step")


def elbm_moments(h, rho_out, u_out, where=ELBM_MEM_DEVICE) -> None:
    _check(h, load().elbm_moments(h, _ptr(rho_out), _ptr(u_out), int(where)), "elbm_moments")


def elbm_alpha_field(h, alpha_out, flags_out=None, where=ELBM_MEM_DEVICE) -> None:
    _check(h, load().elbm_alpha_field(h, _ptr(alpha_out), _ptr(flags_out), int(where)), "elbm_alpha_field")


def elbm_diagnostics(h, alpha_hist: np.ndarray | None = None, allow_nonphysical: bool = False) -> dict:
    d = elbm_diag()
    code = load().elbm_diagnostics(h, ctypes.byref(d), _ptr(alpha_hist))
    if not (allow_nonphysical and code == ELBM_ERR_NONPHYSICAL):
        _check(h, code, "elbm_diagnostics")
    out = d.as_dict()
    out["status"] = code
    return out


def elbm_step_diag(h, n: int, alpha_hist: np.ndarray | None = None, allow_nonphysical: bool = False) -> dict:
    """n steps, the first taking the diagnostics of the state before them."""
    d = elbm_diag()
    code = load().elbm_step_diag(h, int(n), ctypes.byref(d), _ptr(alpha_hist))
    if not (allow_nonphysical and code == ELBM_ERR_NONPHYSICAL):
        _check(h, code, "elbm_step_diag")
    out = d.as_dict()
    out["status"] = code
    return out


def elbm_diagnostics_noalloc(lattice, dims, beta, populations, opts: elbm_opts | None = None,
                             alpha_hist: np.ndarray | None = None, allow_nonphysical: bool = False) -> dict:
    """Diagnostics of a caller-owned device population buffer without any device
    allocation (see include/elbm.h); the first call on a device must precede any
    stream capture, and overlapping calls must be serialised by the caller."""
    d = elbm_diag()
    if opts is None:
        opts = elbm_default_opts()
    code = load().elbm_diagnostics_noalloc(int(lattice), _dims(dims), float(beta), ctypes.byref(opts),
                                           _ptr(populations), ctypes.byref(d), _ptr(alpha_hist))
    if not (allow_nonphysical and code == ELBM_ERR_NONPHYSICAL):
        _check(None, code, "elbm_diagnostics_noalloc")
    out = d.as_dict()
    out["status"] = code
    return out


def elbm_subgrid_viscosity(h, nut_out, where=ELBM_MEM_DEVICE) -> None:
    _check(h, load().elbm_subgrid_viscosity(h, _ptr(nut_out), int(where)), "elbm_subgrid_viscosity")


def elbm_adjoint_step_force(h, f_t, g_next, g_t, dforce) -> None:
    _check(h, load().elbm_adjoint_step_force(h, _ptr(f_t), _ptr(g_next), _ptr(g_t), _ptr(dforce)),
           "elbm_adjoint_step_force")


def elbm_set_force(h, force) -> None:
    arr = None if force is None else np.ascontiguousarray(force, dtype=np.float64)
    _check(h, load().elbm_set_force(h, None if arr is None else arr.ctypes.data), "elbm_set_force")


def elbm_adjoint_step(h, f_t, g_next, g_t) -> None:
    _check(h, load().elbm_adjoint_step(h, _ptr(f_t), _ptr(g_next), _ptr(g_t)), "elbm_adjoint_step")


def elbm_kinetic_energy(h, f=None, grad=None) -> float:
    L = ctypes.c_double(0.0)
    _check(h, load().elbm_kinetic_energy(h, _ptr(f), ctypes.byref(L), _ptr(grad)), "elbm_kinetic_energy")
    return float(L.value)


def elbm_equilibrium_vjp(h, rho, u, g, drho=None, du=None) -> None:
    _check(h, load().elbm_equilibrium_vjp(h, _ptr(rho), _ptr(u), _ptr(g), _ptr(drho), _ptr(du)),
           "elbm_equilibrium_vjp")


def elbm_get_populations(h, dst, where=ELBM_MEM_DEVICE) -> None:
    _check(h, load().elbm_get_populations(h, _ptr(dst), int(where)), "elbm_get_populations")


def elbm_set_populations(h, src, where=ELBM_MEM_DEVICE) -> None:
    _check(h, load().elbm_set_populations(h, _ptr(src), int(where)), "elbm_set_populations")


def elbm_step_count(h) -> int:
    s = ctypes.c_int64(0)
    _check(h, load().elbm_step_count(h, ctypes.byref(s)), "elbm_step_count")
    return int(s.value)


def elbm_synchronize(h) -> None:
    _check(h, load().elbm_synchronize(h), "elbm_synchronize")


# ----------------------------------------------------------------------------
# Convenience wrapper: torch owns the device buffers and the stream.
# ----------------------------------------------------------------------------

class Simulation:
    """One periodic lattice on one GPU.

    Parameters mirror ``elbm_create``; ``storage`` is one of "f64", "f32",
    "f16dev", "bf16dev".  Population buffers are torch tensors (uint8 bytes,
    256-byte aligned by the caching allocator) bound with ``elbm_bind_buffers``.
    """

    def __init__(self, lattice, dims, beta, storage="f32", alpha_mode=ELBM_ALPHA_HIGHER,
                 cutoff=True, b_variant=ELBM_B_DERIVED, device=0, rho0=1.0, stream=None,
                 kernel=ELBM_KERNEL_AUTO):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("Simulation needs a CUDA device")
        self.torch = torch
        self.lattice = int(lattice)
        self.D = 2 if self.lattice == ELBM_D2Q9 else 3
        self.Q = self.lattice
        d = (list(dims) + [1, 1])[:3]
        self.dims = tuple(int(v) for v in d)
        self.N = self.dims[0] * self.dims[1] * self.dims[2]
        self.storage = STORAGE_NAMES[storage] if isinstance(storage, str) else int(storage)
        self.device = torch.device("cuda", device)
        o = elbm_default_opts()
        o.storage = self.storage
        o.alpha_mode = int(alpha_mode)
        o.cutoff = int(bool(cutoff))
        o.b_variant = int(b_variant)
        o.device = int(device)
        o.rho0 = float(rho0)
        o.kernel = int(kernel)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        o.stream = self.stream.cuda_stream
        self.h = elbm_create(self.lattice, self.dims, beta, ELBM_BC_PERIODIC, o)
        self.pop_bytes = elbm_population_bytes(self.lattice, self.dims, self.storage)
        self.buffers = [torch.empty(self.pop_bytes, dtype=torch.uint8, device=self.device) for _ in range(2)]
        elbm_bind_buffers(self.h, self.buffers[0], self.buffers[1], self.pop_bytes)

    def close(self):
        if getattr(self, "h", None):
            elbm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- state ---------------------------------------------------------------
    def init_equilibrium(self, rho, u):
        """rho: (N,) or None; u: (D, N).  numpy arrays go through host memory."""
        torch = self.torch
        if isinstance(u, np.ndarray):
            u = np.ascontiguousarray(u, dtype=np.float64)
            rho = None if rho is None else np.ascontiguousarray(rho, dtype=np.float64)
            elbm_init_equilibrium(self.h, rho, u, ELBM_MEM_HOST)
        else:
            u = u.to(self.device, torch.float64).contiguous()
            rho = None if rho is None else rho.to(self.device, torch.float64).contiguous()
            elbm_init_equilibrium(self.h, rho, u, ELBM_MEM_DEVICE)

    def step(self, n=1):
        elbm_step(self.h, n)

    def moments(self):
        torch = self.torch
        rho = torch.empty(self.N, dtype=torch.float64, device=self.device)
        u = torch.empty((self.D, self.N), dtype=torch.float64, device=self.device)
        elbm_moments(self.h, rho, u, ELBM_MEM_DEVICE)
        return rho, u

    def alpha_field(self):
        torch = self.torch
        a = torch.empty(self.N, dtype=torch.float64, device=self.device)
        fl = torch.empty(self.N, dtype=torch.uint8, device=self.device)
        elbm_alpha_field(self.h, a, fl, ELBM_MEM_DEVICE)
        return a, fl

    def subgrid_viscosity(self):
        nut = self.torch.empty(self.N, dtype=self.torch.float64, device=self.device)
        elbm_subgrid_viscosity(self.h, nut, ELBM_MEM_DEVICE)
        return nut

    def step_diag(self, n, with_hist=False, allow_nonphysical=False):
        """n steps; returns the diagnostics of the state before them (one fused pass)."""
        hist = np.zeros(ELBM_HIST_BINS + 2, dtype=np.int64) if with_hist else None
        d = elbm_step_diag(self.h, n, hist, allow_nonphysical)
        if with_hist:
            d["alpha_hist"] = hist
        return d

    def diagnostics(self, with_hist=False, allow_nonphysical=False):
        hist = np.zeros(ELBM_HIST_BINS + 2, dtype=np.int64) if with_hist else None
        d = elbm_diagnostics(self.h, hist, allow_nonphysical)
        if with_hist:
            d["alpha_hist"] = hist
        return d

    def get_populations(self):
        """Host copy of the stored populations as numpy, shape (Q, N), storage dtype
        (bf16 is returned as raw uint16; deviation storages hold f_i - k_i R)."""
        dt = STORAGE_NUMPY[self.storage]
        out = np.empty((self.Q, self.N), dtype=dt)
        elbm_get_populations(self.h, out, ELBM_MEM_HOST)
        return out

    def set_populations(self, f):
        dt = STORAGE_NUMPY[self.storage]
        f = np.ascontiguousarray(f, dtype=dt).reshape(self.Q, self.N)
        elbm_set_populations(self.h, f, ELBM_MEM_HOST)

    def synchronize(self):
        elbm_synchronize(self.h)

    @property
    def steps(self):
        return elbm_step_count(self.h)

    # -- device copies of the state and reverse-mode helpers ----------------
    @property
    def grad_dtype(self):
        return self.torch.float64 if self.storage == ELBM_STORE_F64 else self.torch.float32

    def state_copy(self):
        """Device copy of the current populations (raw storage bytes)."""
        buf = self.torch.empty(self.pop_bytes, dtype=self.torch.uint8, device=self.device)
        elbm_get_populations(self.h, buf, ELBM_MEM_DEVICE)
        return buf

    def restore(self, buf):
        elbm_set_populations(self.h, buf, ELBM_MEM_DEVICE)

    def set_force(self, force=None):
        """Uniform body force (D values, or None for none); see elbm_set_force."""
        elbm_set_force(self.h, None if force is None else np.asarray(force, dtype=np.float64).ravel()[:self.D])

    def adjoint_step(self, f_t, g_next, dforce=None):
        """One reverse step; with ``dforce`` (a float64 device tensor of D values) also
        accumulates the derivative with respect to the body force into it."""
        g_t = self.torch.empty_like(g_next)
        if dforce is None:
            elbm_adjoint_step(self.h, f_t, g_next, g_t)
        else:
            elbm_adjoint_step_force(self.h, f_t, g_next, g_t, dforce)
        return g_t

    def kinetic_energy(self, f=None, with_grad=False):
        grad = (self.torch.empty((self.Q, self.N), dtype=self.grad_dtype, device=self.device)
                if with_grad else None)
        L = elbm_kinetic_energy(self.h, f, grad)
        return (L, grad) if with_grad else L

    def equilibrium_vjp(self, rho, u, g):
        drho = self.torch.empty(self.N, dtype=self.torch.float64, device=self.device)
        du = self.torch.empty((self.D, self.N), dtype=self.torch.float64, device=self.device)
        elbm_equilibrium_vjp(self.h, rho, u, g, drho, du)
        return drho, du


# ----------------------------------------------------------------------------
# Batched ensembles (same names as include/elbm.h)
# ----------------------------------------------------------------------------

def _bcheck(b, code, what):
    if code != ELBM_OK:
        msg = load().elbm_batch_last_error(b)
        raise ElbmError(code, f"{what}: {msg.decode() if msg else ''}")


def elbm_batch_create(lattice, dims_list, betas, opts: elbm_opts | None = None) -> int:
    nd = len(dims_list)
    flat = []
    for d in dims_list:
        flat += [int(v) for v in (list(d) + [1, 1])[:3]]
    b = ctypes.c_void_p(None)
    _bcheck(None, load().elbm_batch_create(ctypes.byref(b), int(lattice), nd, (ctypes.c_int64 * (3 * nd))(*flat),
                                           (ctypes.c_double * nd)(*[float(x) for x in betas]),
                                           None if opts is None else ctypes.byref(opts)), "elbm_batch_create")
    return b.value


def elbm_batch_destroy(b) -> None:
    load().elbm_batch_destroy(b)


def elbm_batch_last_error(b=None) -> str:
    m = load().elbm_batch_last_error(b)
    return m.decode() if m else ""


def elbm_batch_info(b):
    nd, nodes, bx = ctypes.c_int(0), ctypes.c_int64(0), ctypes.c_int(0)
    _bcheck(b, load().elbm_batch_info(b, ctypes.byref(nd), ctypes.byref(nodes), ctypes.byref(bx)),
            "elbm_batch_info")
    return nd.value, nodes.value, bx.value


def elbm_batch_init_equilibrium(b, domain, rho, u, where=ELBM_MEM_HOST) -> None:
    _bcheck(b, load().elbm_batch_init_equilibrium(b, int(domain), _ptr(rho), _ptr(u), int(where)),
            "elbm_batch_init_equilibrium")


def elbm_batch_step(b, n=1, mode=ELBM_BATCH_AUTO) -> None:
    _bcheck(b, load().elbm_batch_step(b, int(n), int(mode)), "elbm_batch_step")


def elbm_batch_tune(b):
    chosen = ctypes.c_int(0)
    ms = (ctypes.c_double * 3)()
    _bcheck(b, load().elbm_batch_tune(b, ctypes.byref(chosen), ms), "elbm_batch_tune")
    return chosen.value, list(ms)


def elbm_batch_tune_persistent(b):
    mode = ctypes.c_int(0)
    ms = (ctypes.c_double * 3)()
    _bcheck(b, load().elbm_batch_tune_persistent(b, ctypes.byref(mode), ms), "elbm_batch_tune_persistent")
    return mode.value, list(ms)


def elbm_batch_moments(b, domain, rho_out, u_out, where=ELBM_MEM_HOST) -> None:
    _bcheck(b, load().elbm_batch_moments(b, int(domain), _ptr(rho_out), _ptr(u_out), int(where)),
            "elbm_batch_moments")


def elbm_batch_diagnostics(b, domain, alpha_hist=None) -> dict:
    d = elbm_diag()
    _bcheck(b, load().elbm_batch_diagnostics(b, int(domain), ctypes.byref(d), _ptr(alpha_hist)),
            "elbm_batch_diagnostics")
    return d.as_dict()


def elbm_batch_get_populations(b, domain, dst, where=ELBM_MEM_HOST) -> None:
    _bcheck(b, load().elbm_batch_get_populations(b, int(domain), _ptr(dst), int(where)),
            "elbm_batch_get_populations")


def elbm_batch_set_populations(b, domain, src, where=ELBM_MEM_HOST) -> None:
    _bcheck(b, load().elbm_batch_set_populations(b, int(domain), _ptr(src), int(where)),
            "elbm_batch_set_populations")


def elbm_batch_synchronize(b) -> None:
    _bcheck(b, load().elbm_batch_synchronize(b), "elbm_batch_synchronize")


def elbm_batch_check_wait_timeout(b) -> None:
    _bcheck(b, load().elbm_batch_check_wait_timeout(b), "elbm_batch_check_wait_timeout")


class Ensemble:
    """Independent periodic domains advanced together (see the batched-ensemble
    section of include/elbm.h)."""

    _DT = STORAGE_NUMPY

    def __init__(self, lattice, dims_list, betas, storage="f32", alpha_mode=ELBM_ALPHA_HIGHER, cutoff=True,
                 b_variant=ELBM_B_DERIVED, device=0, rho0=1.0, stream=None):
        self.lattice = int(lattice)
        self.D = 2 if self.lattice == ELBM_D2Q9 else 3
        self.Q = self.lattice
        self.dims = [tuple(int(v) for v in (list(d) + [1, 1])[:3]) for d in dims_list]
        self.storage = STORAGE_NAMES[storage] if isinstance(storage, str) else int(storage)
        o = elbm_default_opts()
        o.storage = self.storage
        o.alpha_mode = int(alpha_mode)
        o.cutoff = int(bool(cutoff))
        o.b_variant = int(b_variant)
        o.device = int(device)
        o.rho0 = float(rho0)
        o.stream = None if stream is None else int(stream)
        self.b = elbm_batch_create(self.lattice, self.dims, betas, o)

    def close(self):
        if getattr(self, "b", None):
            elbm_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def nodes(self, d):
        nx, ny, nz = self.dims[d]
        return nx * ny * nz

    def init_equilibrium(self, d, rho, u):
        u = np.ascontiguousarray(u, dtype=np.float64)
        rho = None if rho is None else np.ascontiguousarray(rho, dtype=np.float64)
        elbm_batch_init_equilibrium(self.b, d, rho, u, ELBM_MEM_HOST)

    def step(self, n=1, mode=ELBM_BATCH_AUTO):
        """n steps of every domain; AUTO issues the form tune_persistent() found faster
        (the graph of batched launches until it has run)."""
        elbm_batch_step(self.b, n, mode)

    def tune(self):
        return elbm_batch_tune(self.b)

    def tune_persistent(self):
        """(mode ELBM_BATCH_AUTO will issue, ms per step of the persistent mode per width)."""
        return elbm_batch_tune_persistent(self.b)

    def moments(self, d):
        N = self.nodes(d)
        rho = np.empty(N)
        u = np.empty((self.D, N))
        elbm_batch_moments(self.b, d, rho, u, ELBM_MEM_HOST)
        return rho, u

    def diagnostics(self, d):
        return elbm_batch_diagnostics(self.b, d)

    def get_populations(self, d):
        out = np.empty((self.Q, self.nodes(d)), dtype=self._DT[self.storage])
        elbm_batch_get_populations(self.b, d, out, ELBM_MEM_HOST)
        return out

    def set_populations(self, d, f):
        f = np.ascontiguousarray(f, dtype=self._DT[self.storage]).reshape(self.Q, self.nodes(d))
        elbm_batch_set_populations(self.b, d, f, ELBM_MEM_HOST)

    def synchronize(self):
        elbm_batch_synchronize(self.b)
