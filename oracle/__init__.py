"""FP64 CPU oracle of the essentially entropic lattice Boltzmann step.

TEST INFRASTRUCTURE ONLY.  This package is imported by ``tests/``, by
``__graft_entry__.smoke()`` and by the CPU-baseline leg of ``bench.py`` and by
nothing else; the CUDA library and its Python binding never import, load or
call it, and the two share no code.

The arithmetic lives in ``elbm_oracle.c`` (plain C99, IEEE double, no FMA
contraction), compiled on demand with gcc into ``oracle/_build``.  This module
only marshals numpy arrays through ctypes.

Functions and the passages of arXiv:2203.12946 they follow:

* ``lattice``            Sec. I (D1Q3 weights and their tensor products)
* ``equilibrium``        Sec. I, entropic equilibrium (product form)
* ``moments``            Sec. I, rho = <f,1>, rho u = <f,c>
* ``H``                  Eq. hdef
* ``alpha``              Sec. III (Eq. alphaLowerSoln, qaud_tight, gaplhah0),
                         Appendix C, Appendix D (cutoff, positivity clamp)
* ``deltaH_star``        Eq. deltaH3 (Appendix A)
* ``alpha_elbm``         Sec. II, Eq. entropy_conserve / deltaH_ (Newton with
                         bisection safeguard)
* ``alpha_iterate1``     Sec. IV, one Newton step from alpha_Lower
* ``stream``             Eq. advection (pull form, periodic)
* ``collide``/``step``   Eq. fstar_def with the Appendix D path length
* ``init_equilibrium``   f = f^eq(rho, u) at every node

Layout of a population field: structure of arrays ``f[i, n]`` (shape
``(Q, N)``), ``n = (z*ny + y)*nx + x``; velocity ``i`` is lexicographic over
(c_x, c_y[, c_z]) in {-1,0,1}^D with the last axis fastest.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "elbm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libelbm_oracle.so")

MODE_HIGHER, MODE_LOWER, MODE_LBGK, MODE_ITERATE1 = 0, 1, 2, 3
BRANCH_CUTOFF, BRANCH_SOLVED, BRANCH_CLAMPED = 0, 1, 2
B_DERIVED, B_PRINTED = 0, 1
CUTOFF = 1e-3

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (C99, -O2, no FMA contraction, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c99", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
           "-shared", "-fopenmp", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _AlphaInfo(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in (
        "alpha", "alpha_lower", "h", "alpha_higher", "xabsmax", "xmin", "alpha_max",
        "a1", "b1", "c1", "a2", "a", "b", "c")] + [("branch", ctypes.c_int)]


_D = ctypes.POINTER(ctypes.c_double)
_I8 = ctypes.POINTER(ctypes.c_int8)
_I = ctypes.POINTER(ctypes.c_int)
_i64 = ctypes.c_int64


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        sig = {
            "or_lattice": (ctypes.c_int, [ctypes.c_int, _I, _D]),
            "or_equilibrium": (None, [ctypes.c_int, ctypes.c_double, _D, _D]),
            "or_moments": (None, [ctypes.c_int, _D, _D, _D]),
            "or_H": (ctypes.c_double, [ctypes.c_int, _D, _D]),
            "or_departure": (None, [ctypes.c_int, _D, _D, _D]),
            "or_alpha": (ctypes.c_int, [ctypes.c_int, _D, _D, ctypes.c_double, ctypes.c_int,
                                        ctypes.c_int, ctypes.c_int, ctypes.POINTER(_AlphaInfo)]),
            "or_relax": (None, [ctypes.c_int, _D, _D, ctypes.c_double, ctypes.c_double, _D]),
            "or_deltaH_star": (ctypes.c_double, [ctypes.c_int, _D, _D, ctypes.c_double,
                                                 ctypes.c_double]),
            "or_mirror_F": (ctypes.c_double, [ctypes.c_int, _D, _D, ctypes.c_double]),
            "or_alpha_elbm": (ctypes.c_double, [ctypes.c_int, _D, _D, ctypes.c_double, _I, _I]),
            "or_alpha_iterate1": (ctypes.c_double, [ctypes.c_int, _D, _D, ctypes.c_double]),
            "or_stream": (None, [ctypes.c_int, _i64, _i64, _i64, _D, _D, ctypes.c_int]),
            "or_collide": (None, [ctypes.c_int, _i64, ctypes.c_double, ctypes.c_int,
                                  ctypes.c_int, ctypes.c_int, _D, _D, _I8, _D, ctypes.c_int]),
            "or_alpha_field": (None, [ctypes.c_int, _i64, ctypes.c_double, ctypes.c_int,
                                      ctypes.c_int, ctypes.c_int, _D, _D, _I8, _D,
                                      ctypes.c_int]),
            "or_step": (None, [ctypes.c_int, _i64, _i64, _i64, ctypes.c_double, ctypes.c_int,
                               ctypes.c_int, ctypes.c_int, _D, _D, _D, _I8, _D, ctypes.c_int]),
            "or_init_equilibrium": (None, [ctypes.c_int, _i64, _D, _D, _D]),
            "or_moments_field": (None, [ctypes.c_int, _i64, _D, _D, _D]),
            "or_H_total": (ctypes.c_double, [ctypes.c_int, _i64, _D]),
            "or_max_threads": (ctypes.c_int, []),
            "or_collide_vjp": (None, [ctypes.c_int, _D, _D, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                      ctypes.c_int, _D, ctypes.c_double, _D]),
            "or_step_adjoint": (None, [ctypes.c_int, _i64, _i64, _i64, ctypes.c_double, ctypes.c_int,
                                       ctypes.c_int, ctypes.c_int, _D, _D, _D, _D, ctypes.c_double,
                                       ctypes.c_int]),
            "or_force_node": (None, [ctypes.c_int, _D, _D]),
            "or_force": (None, [ctypes.c_int, _i64, _D, _D, ctypes.c_int]),
            "or_step_force_vjp": (None, [ctypes.c_int, _i64, _i64, _i64, ctypes.c_double, ctypes.c_int,
                                         ctypes.c_int, ctypes.c_int, _D, _D, _D, ctypes.c_double, _D,
                                         ctypes.c_int]),
            "or_kinetic_energy": (ctypes.c_double, [ctypes.c_int, _i64, _D, _D]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _dp(a):
    return None if a is None else a.ctypes.data_as(_D)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def max_threads() -> int:
    return int(_load().or_max_threads())


# ----------------------------------------------------------------------------
# Single-node functions
# ----------------------------------------------------------------------------

def lattice(D: int):
    """(c, w): velocities (Q, D) int and weights (Q,) of the D1Q3 product lattice."""
    Q = 3 ** D
    c = np.zeros(Q * D, dtype=np.int32)
    w = np.zeros(Q, dtype=np.float64)
    _load().or_lattice(D, c.ctypes.data_as(_I), _dp(w))
    return c.reshape(Q, D), w


def equilibrium(D: int, rho: float, u) -> np.ndarray:
    u = _f64(u)
    out = np.zeros(3 ** D)
    _load().or_equilibrium(D, float(rho), _dp(u), _dp(out))
    return out


def moments(D: int, f):
    f = _f64(f)
    rho = np.zeros(1)
    u = np.zeros(D)
    _load().or_moments(D, _dp(f), _dp(rho), _dp(u))
    return float(rho[0]), u


def H(f, w) -> float:
    f, w = _f64(f), _f64(w)
    return float(_load().or_H(len(f), _dp(f), _dp(w)))


def departure(f, feq) -> np.ndarray:
    f, feq = _f64(f), _f64(feq)
    x = np.zeros_like(f)
    _load().or_departure(len(f), _dp(f), _dp(feq), _dp(x))
    return x


@dataclass
class AlphaInfo:
    alpha: float
    alpha_lower: float
    h: float
    alpha_higher: float
    xabsmax: float
    xmin: float
    alpha_max: float
    a1: float
    b1: float
    c1: float
    a2: float
    a: float
    b: float
    c: float
    branch: int


def alpha(f, feq, beta: float, cutoff: bool = True, b_variant: int = B_DERIVED,
          mode: int = MODE_HIGHER) -> AlphaInfo:
    """Path length of one node by the steps of Appendix D."""
    f, feq = _f64(f), _f64(feq)
    info = _AlphaInfo()
    _load().or_alpha(len(f), _dp(f), _dp(feq), float(beta), int(bool(cutoff)), int(b_variant),
                     int(mode), ctypes.byref(info))
    return AlphaInfo(**{k: getattr(info, k) for k, _ in _AlphaInfo._fields_})


def relax(f, feq, alpha_: float, beta: float) -> np.ndarray:
    f, feq = _f64(f), _f64(feq)
    out = np.zeros_like(f)
    _load().or_relax(len(f), _dp(f), _dp(feq), float(alpha_), float(beta), _dp(out))
    return out


def deltaH_star(f, x, alpha_: float, beta: float) -> float:
    f, x = _f64(f), _f64(x)
    return float(_load().or_deltaH_star(len(f), _dp(f), _dp(x), float(alpha_), float(beta)))


def mirror_F(f, x, alpha_: float) -> float:
    f, x = _f64(f), _f64(x)
    return float(_load().or_mirror_F(len(f), _dp(f), _dp(x), float(alpha_)))


def alpha_elbm(f, feq, alpha0: float = 2.0):
    """(alpha_ELBM, iterations, status) -- status 0 ok, 1 no root, 2 x == 0, 3 no convergence."""
    f, feq = _f64(f), _f64(feq)
    it = ctypes.c_int(0)
    st = ctypes.c_int(0)
    a = _load().or_alpha_elbm(len(f), _dp(f), _dp(feq), float(alpha0), ctypes.byref(it),
                              ctypes.byref(st))
    return float(a), int(it.value), int(st.value)


def alpha_iterate1(f, feq, alpha_lower: float) -> float:
    f, feq = _f64(f), _f64(feq)
    return float(_load().or_alpha_iterate1(len(f), _dp(f), _dp(feq), float(alpha_lower)))


# ----------------------------------------------------------------------------
# Field functions.  dims = (nx, ny, nz) with nz = 1 for D = 2.
# ----------------------------------------------------------------------------

def _dims(D, dims):
    nx, ny, nz = (list(dims) + [1, 1])[:3]
    if D == 2:
        nz = 1
    return int(nx), int(ny), int(nz)


def init_equilibrium(D: int, rho, u) -> np.ndarray:
    rho = _f64(rho).ravel()
    N = rho.size
    u = _f64(u).reshape(D, N)
    f = np.zeros((3 ** D, N))
    _load().or_init_equilibrium(D, N, _dp(rho), _dp(u), _dp(f))
    return f


def moments_field(D: int, f):
    f = _f64(f)
    N = f.shape[1]
    rho = np.zeros(N)
    u = np.zeros((D, N))
    _load().or_moments_field(D, N, _dp(f), _dp(rho), _dp(u))
    return rho, u


def H_total(D: int, f) -> float:
    f = _f64(f)
    return float(_load().or_H_total(D, f.shape[1], _dp(f)))


def stream(D: int, dims, f, nthreads: int = 0) -> np.ndarray:
    nx, ny, nz = _dims(D, dims)
    f = _f64(f)
    out = np.zeros_like(f)
    _load().or_stream(D, nx, ny, nz, _dp(f), _dp(out), int(nthreads))
    return out


def collide(D: int, f, beta: float, cutoff: bool = True, b_variant: int = B_DERIVED,
            mode: int = MODE_HIGHER, want_alpha: bool = False, want_dH: bool = False,
            nthreads: int = 0):
    """Collide a pre-collision field; returns (f*, alpha or None, branch or None, dH or None)."""
    f = _f64(f).copy()
    N = f.shape[1]
    a = np.zeros(N) if want_alpha else None
    br = np.zeros(N, dtype=np.int8) if want_alpha else None
    dh = np.zeros(N) if want_dH else None
    _load().or_collide(D, N, float(beta), int(bool(cutoff)), int(b_variant), int(mode), _dp(f),
                       _dp(a), None if br is None else br.ctypes.data_as(_I8), _dp(dh),
                       int(nthreads))
    return f, a, br, dh


def alpha_field(D: int, f, beta: float, cutoff: bool = True, b_variant: int = B_DERIVED,
                mode: int = MODE_HIGHER, want_elbm: bool = False, nthreads: int = 0):
    """Per-node (alpha, branch, alpha_ELBM or None) of a pre-collision field."""
    f = _f64(f)
    N = f.shape[1]
    a = np.zeros(N)
    br = np.zeros(N, dtype=np.int8)
    ae = np.zeros(N) if want_elbm else None
    _load().or_alpha_field(D, N, float(beta), int(bool(cutoff)), int(b_variant), int(mode),
                           _dp(f), _dp(a), br.ctypes.data_as(_I8), _dp(ae), int(nthreads))
    return a, br, ae


def _force3(D, force):
    F = np.zeros(3)
    F[:D] = np.asarray(force, dtype=np.float64).ravel()[:D]
    return F


def force_node(D: int, f, force) -> np.ndarray:
    """One node's populations after the exact-difference body-force term (not in the paper)."""
    f = _f64(f).copy()
    _load().or_force_node(D, _dp(_force3(D, force)), _dp(f))
    return f


def step(D: int, dims, f, beta: float, cutoff: bool = True, b_variant: int = B_DERIVED,
         mode: int = MODE_HIGHER, nsteps: int = 1, nthreads: int = 0, want_alpha: bool = False,
         want_dH: bool = False, force=None):
    """Advance a post-collision field by ``nsteps`` steps (stream, then collide, then the
    body-force term when ``force`` is given).

    Returns (f, alpha, branch, dH) where the optional per-node fields belong to
    the last step.
    """
    F = None if force is None else _force3(D, force)
    nx, ny, nz = _dims(D, dims)
    a = _f64(f).copy()
    b = np.zeros_like(a)
    N = a.shape[1]
    lib = _load()
    alpha_ = br = dh = None
    for s in range(nsteps):
        last = s == nsteps - 1
        alpha_ = np.zeros(N) if (want_alpha and last) else None
        br = np.zeros(N, dtype=np.int8) if (want_alpha and last) else None
        dh = np.zeros(N) if (want_dH and last) else None
        lib.or_step(D, nx, ny, nz, float(beta), int(bool(cutoff)), int(b_variant), int(mode),
                    _dp(a), _dp(b), _dp(alpha_), None if br is None else br.ctypes.data_as(_I8),
                    _dp(dh), int(nthreads))
        if F is not None:
            lib.or_force(D, N, _dp(F), _dp(b), int(nthreads))
        a, b = b, a
    return a, alpha_, br, dh


# ----------------------------------------------------------------------------
# Adjoint (chain rule through the step; node Jacobians by central differences)
# ----------------------------------------------------------------------------

def collide_vjp(D: int, f, g, beta: float, cutoff: bool = False, b_variant: int = B_DERIVED,
                mode: int = MODE_HIGHER, eps: float = 1e-5, force=None) -> np.ndarray:
    """h = J^T g of one node's collision (J = d f* / d f), by central differences."""
    f, g = _f64(f), _f64(g)
    h = np.zeros_like(f)
    F = None if force is None else _force3(D, force)
    _load().or_collide_vjp(D, _dp(f), _dp(g), float(beta), int(bool(cutoff)), int(b_variant), int(mode),
                           _dp(F), float(eps), _dp(h))
    return h


def step_adjoint(D: int, dims, f_t, g_next, beta: float, cutoff: bool = False, b_variant: int = B_DERIVED,
                 mode: int = MODE_HIGHER, eps: float = 1e-5, nthreads: int = 0, force=None) -> np.ndarray:
    """dL/df^t from dL/df^{t+1} for f^{t+1} = collide(stream(f^t)) (+ the force term)."""
    nx, ny, nz = _dims(D, dims)
    f_t, g_next = _f64(f_t), _f64(g_next)
    g_t = np.zeros_like(f_t)
    F = None if force is None else _force3(D, force)
    _load().or_step_adjoint(D, nx, ny, nz, float(beta), int(bool(cutoff)), int(b_variant), int(mode),
                            _dp(F), _dp(f_t), _dp(g_next), _dp(g_t), float(eps), int(nthreads))
    return g_t


def step_force_vjp(D: int, dims, f_t, g_next, beta: float, force, cutoff: bool = False,
                   b_variant: int = B_DERIVED, mode: int = MODE_HIGHER, eps: float = 1e-6,
                   nthreads: int = 0) -> np.ndarray:
    """d/dF of <g_next, f^{t+1}> for one forced step (D values), by central differences."""
    nx, ny, nz = _dims(D, dims)
    f_t, g_next = _f64(f_t), _f64(g_next)
    out = np.zeros(3)
    _load().or_step_force_vjp(D, nx, ny, nz, float(beta), int(bool(cutoff)), int(b_variant), int(mode),
                              _dp(_force3(D, force)), _dp(f_t), _dp(g_next), float(eps), _dp(out),
                              int(nthreads))
    return out[:D]


def kinetic_energy(D: int, f, want_grad: bool = True):
    """(L, dL/df) with L = 1/2 sum rho |u|^2."""
    f = _f64(f)
    g = np.zeros_like(f) if want_grad else None
    L = _load().or_kinetic_energy(D, f.shape[1], _dp(f), _dp(g))
    return float(L), g
