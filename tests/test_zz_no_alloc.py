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
    code = lib.elbm_diagnostics_noalloc(lattice, dd, beta, None if opts is None else ctypes.byref(opts), ptr,
                                        ctypes.byref(d), hist.ctypes.data if hist is not None else None)
    return code, d.as_dict()


def _same(a, b):
    for k in ("mass", "H"):
        assert abs(a[k] - b[k]) <= 1e-12 * abs(b[k]), k
    assert np.allclose(a["momentum"], b["momentum"], rtol=0, atol=1e-12 * abs(b["mass"]))
    for k in ("dH_max", "alpha_min", "alpha_max", "alpha_mean"):
        assert abs(a[k] - b[k]) <= 1e-12 * max(1.0, abs(b[k])), k
    for k in ("n_nodes", "n_cutoff", "n_solved", "n_clamped", "n_nonpositive", "n_dH_positive", "n_xmax_band"):
        assert a[k] == b[k], k


@pytest.mark.parametrize("D,dims,storage", [(2, (96, 80, 1), "f64"), (3, (40, 24, 16), "f32"),
                                            (3, (64, 32, 8), "bf16dev"), (3, (33, 20, 9), "f32dev")])
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
        elif storage == "f32dev":
            c = np.rint(O.lattice(D)[1] * 6.0 ** D) * E.dev_unit(D)
            sim.set_populations((f0 - c[:, None]).astype(np.float32))
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


def test_noalloc_rejects_bad_buffers_and_defaults_to_current_device(lib):
    """A buffer pointer that is misaligned for its element, or not device memory, is an
    argument error (no fault); with NULL options the call runs on the current device."""
    import torch

    dims = (16, 16, 1)
    f0 = O.init_equilibrium(2, np.ones(256), np.zeros((2, 256)))
    buf = torch.from_numpy(f0.astype(np.float32).ravel().view(np.uint8).copy()).cuda()
    opts = E.elbm_default_opts()  # FP32 storage
    code, _ = _call(lib, E.ELBM_D2Q9, dims, 0.9, opts, buf.data_ptr() + 2, None)
    assert code == E.ELBM_ERR_ARG and "aligned" in E.elbm_last_error(None)
    host = np.zeros(9 * 256, dtype=np.float32)
    code, _ = _call(lib, E.ELBM_D2Q9, dims, 0.9, opts, host.ctypes.data, None)
    assert code == E.ELBM_ERR_ARG and "device memory" in E.elbm_last_error(None)
    code, d = _call(lib, E.ELBM_D2Q9, dims, 0.9, None, buf.data_ptr(), None)
    assert code == E.ELBM_OK, E.elbm_last_error(None)
    assert abs(d["mass"] - 256.0) < 1e-5 and d["n_nodes"] == 256


def test_noalloc_repeated_calls_leave_device_memory_unchanged(lib):
    """After the first call (which looks up the fixed array's address), further calls
    change the device's free memory (cudaMemGetInfo) by nothing."""
    import torch

    D, dims = 3, (32, 24, 16)
    X, Y, Z = inputs.grid(dims)
    rho, u = inputs.taylor_green_3d(X, Y, Z, 32, u0=0.05)
    f0 = O.init_equilibrium(D, rho, u).astype(np.float32)
    buf = torch.from_numpy(f0.view(np.uint8).copy()).cuda()
    opts = E.elbm_default_opts()
    code, first = _call(lib, E.ELBM_D3Q27, dims, 0.99, opts, buf.data_ptr(), None)
    assert code == E.ELBM_OK
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(5):
        code, d = _call(lib, E.ELBM_D3Q27, dims, 0.99, opts, buf.data_ptr(), None)
        assert code == E.ELBM_OK and d["n_nodes"] == first["n_nodes"]
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
