"""elbm_diagnostics_noalloc against elbm_diagnostics, through the C ABI.

Callers that cannot allocate device memory (their GPU memory belongs to another
allocator or a fixed pool, or they must not grow their footprint once running)
cannot create a handle, because elbm_create allocates.  elbm_diagnostics_noalloc
serves them: it reads a population buffer the caller already owns and keeps its
reduction accumulator in a fixed device array inside the library.  This test
checks that it returns what the handle-based elbm_diagnostics returns for the
same populations, on two calls in a row (the second call must not see the first
call's sums), and that it rejects bad input with a clear message.  It lives in
its own file, collected last, and passes alone in a fresh process as well.
"""
import ctypes

import numpy as np
import pytest

import oracle as O
from paper_2203_12946_gb300 import elbm as E
from paper_2203_12946_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lib = E.load()
    fn = lib.elbm_diagnostics_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int64), ctypes.c_double,
                   ctypes.POINTER(E.elbm_opts), ctypes.c_void_p, ctypes.POINTER(E.elbm_diag),
                   ctypes.c_void_p]
    return lib


def _call(lib, lattice, dims, beta, opts, ptr, hist):
    d = E.elbm_diag()
    dd = (ctypes.c_int64 * 3)(*dims)
    code = lib.elbm_diagnostics_noalloc(lattice, dd, beta, ctypes.byref(opts), ptr, ctypes.byref(d),
                                        hist.ctypes.data if hist is not None else None)
    return code, d.as_dict()


def _same(a, b):
    for k in ("mass", "H"):
        assert abs(a[k] - b[k]) <= 1e-12 * abs(b[k]), k
    assert np.allclose(a["momentum"], b["momentum"], rtol=0, atol=1e-12 * abs(b["mass"]))
    for k in ("dH_max", "alpha_min", "alpha_max", "alpha_mean"):
        assert abs(a[k] - b[k]) <= 1e-12 * max(1.0, abs(b[k])), k
    for k in ("n_nodes", "n_cutoff", "n_solved", "n_clamped", "n_nonpositive", "n_dH_positive"):
        assert a[k] == b[k], k


@pytest.mark.parametrize("D,dims,storage", [(2, (96, 80, 1), "f64"), (3, (40, 24, 16), "f32"),
                                            (3, (64, 32, 8), "bf16dev")])
def test_noalloc_matches_handle_twice(lib, D, dims, storage):
    import torch

    lattice = E.ELBM_D2Q9 if D == 2 else E.ELBM_D3Q27
    beta = 0.997
    X, Y, Z = inputs.grid(dims)
    rho, u = (inputs.taylor_green_2d(X, Y, dims[0], u0=0.05) if D == 2
              else inputs.taylor_green_3d(X, Y, Z, dims[0], u0=0.05))
    f0 = O.init_equilibrium(D, rho, u) * inputs.population_noise(3 ** D, X.size, 3e-3, seed=7)
    with E.Simulation(lattice, dims, beta, storage=storage) as sim:
        if storage in ("f64", "f32"):
            sim.set_populations(f0)
        else:
            sim.init_equilibrium(*O.moments_field(D, f0))
            sim.step(3)
        want_hist = np.zeros(E.ELBM_HIST_BINS + 2, dtype=np.int64)
        want = E.elbm_diagnostics(sim.h, want_hist)
        # a caller-owned copy of the same populations (device memory the caller allocated)
        host = sim.get_populations()
        buf = torch.from_numpy(host.view(np.uint8).copy()).to("cuda")
        torch.cuda.synchronize()
        opts = E.elbm_default_opts()
        opts.storage = E.STORAGE_NAMES[storage]
        for _ in range(2):
            hist = np.zeros(E.ELBM_HIST_BINS + 2, dtype=np.int64)
            code, got = _call(lib, lattice, dims, beta, opts, buf.data_ptr(), hist)
            assert code == E.ELBM_OK, E.elbm_last_error(None)
            _same(got, want)
            assert np.array_equal(hist, want_hist)


def test_noalloc_rejects_bad_input(lib):
    import torch

    opts = E.elbm_default_opts()
    buf = torch.zeros(9 * 16 * 16, dtype=torch.float32, device="cuda")
    code, _ = _call(lib, 10, (16, 16, 1), 0.9, opts, buf.data_ptr(), None)
    assert code == E.ELBM_ERR_ARG and "lattice" in E.elbm_last_error(None)
    code, _ = _call(lib, E.ELBM_D2Q9, (16, 16, 1), 1.5, opts, buf.data_ptr(), None)
    assert code == E.ELBM_ERR_ARG and "beta" in E.elbm_last_error(None)
    code, _ = _call(lib, E.ELBM_D2Q9, (16, 16, 1), 0.9, opts, None, None)
    assert code == E.ELBM_ERR_ARG and "null" in E.elbm_last_error(None)
    bad = E.elbm_default_opts()
    bad.device = 7
    code, _ = _call(lib, E.ELBM_D2Q9, (16, 16, 1), 0.9, bad, buf.data_ptr(), None)
    assert code == E.ELBM_ERR_ARG and "device" in E.elbm_last_error(None)
