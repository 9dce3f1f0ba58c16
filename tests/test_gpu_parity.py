"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle.

Both sides receive the same seeded inputs from ``paper_2203_12946_gb300.inputs``;
the oracle builds its own populations, and where the GPU starts from populations
they are the oracle's (or the oracle's rounded to the GPU's storage type), never
the reverse.  Tolerances:

* FP64 path: 1e-12 relative per population (the rounding-order difference of two
  IEEE double evaluations of the same formulas is ~1e-15 per step);
* FP32 path: x = f^eq/f - 1 carries ~3e-7 absolute error from the FP32
  equilibrium, so f* = f (1 + alpha beta x) moves by <= 2 * 3e-7 relative per step;
  we allow 2e-6 per step on f and 1e-5 relative on u (the stated FP32 target);
* branch decisions (cutoff, clamp) are integers decided by floating point: each
  side decides in its own precision, so a node may take the other branch only
  when its |x|max lies within the decision precision of the 1e-3 threshold
  (1e-12 for FP64, 1e-6 for FP32); such nodes are excluded from the value check
  of that step and counted.
"""
import numpy as np
import pytest

import oracle as O
from paper_2203_12946_gb300 import elbm as E
from paper_2203_12946_gb300 import inputs

pytestmark = pytest.mark.gpu

LAT = {2: E.ELBM_D2Q9, 3: E.ELBM_D3Q27}
MODES = {"higher": (E.ELBM_ALPHA_HIGHER, O.MODE_HIGHER), "lower": (E.ELBM_ALPHA_LOWER, O.MODE_LOWER),
         "lbgk": (E.ELBM_ALPHA_LBGK, O.MODE_LBGK), "iterate1": (E.ELBM_ALPHA_ITERATE1, O.MODE_ITERATE1)}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    E.load()


def noisy_state(D, dims, eps, seed=3, u0=0.05, kind="tgv"):
    """Oracle-made populations: equilibrium of a Taylor-Green field times 1 + eps U(-1,1)."""
    X, Y, Z = inputs.grid(dims)
    L = dims[0]
    if D == 2:
        rho, u = inputs.taylor_green_2d(X, Y, L, u0=u0)
    else:
        rho, u = inputs.taylor_green_3d(X, Y, Z, L, u0=u0)
    f = O.init_equilibrium(D, rho, u)
    return f * inputs.population_noise(3 ** D, X.size, eps, seed=seed)


def dev_ref(D):
    """Reference c_i = k_i R of the deviation storages (rho0 = 1): w_i = k_i 6^-D, R = 6^-D
    rounded to FP32 (include/elbm.h)."""
    _, w = O.lattice(D)
    return np.rint(w * 6.0 ** D) * E.dev_unit(D)


def stored(D, f, storage):
    """(values to hand to set_populations, the FP64 populations they represent exactly)
    for an oracle field f and an FP32 storage."""
    if storage == "f32dev":
        c = dev_ref(D)[:, None]
        s = (f - c).astype(np.float32)
        return s, c + s.astype(np.float64)
    s = f.astype(np.float32)
    return s, s.astype(np.float64)


def populations(D, raw, storage):
    """FP64 populations of a stored field (get_populations output)."""
    if storage == "f32dev":
        return dev_ref(D)[:, None] + raw.astype(np.float64)
    return raw.astype(np.float64)


def gpu_run(D, dims, beta, f0, nsteps, storage="f64", **kw):
    with E.Simulation(LAT[D], dims, beta, storage=storage, **kw) as sim:
        sim.set_populations(f0)
        sim.step(nsteps)
        f = populations(D, sim.get_populations(), storage)
        sim.synchronize()  # also reports an expired device-side wait
    return f


def xabsmax_of(D, f):
    """|x|max per node of a pre-collision field (oracle)."""
    out = np.empty(f.shape[1])
    for n in range(f.shape[1]):
        r, u = O.moments(D, f[:, n])
        out[n] = O.alpha(f[:, n], O.equilibrium(D, r, u), 0.5).xabsmax
    return out


def check_branches(D, f_pre, br_gpu, br_ora, band):
    """Nodes whose branch differs must sit within `band` of the cutoff; returns the mask of
    agreeing nodes."""
    diff = np.nonzero(br_gpu != br_ora)[0]
    if diff.size:
        xm = xabsmax_of(D, f_pre[:, diff])
        assert np.all(np.abs(xm - O.CUTOFF) <= band), (diff[:10], xm[:10])
    agree = np.ones(br_gpu.size, dtype=bool)
    agree[diff] = False
    return agree


# ---------------------------------------------------------------------------
# FP64: one step and several steps, every mode, both b readings, ragged sizes
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("D,dims", [(2, (300, 37, 1)), (3, (37, 19, 11))])
@pytest.mark.parametrize("mode", ["higher", "lower", "lbgk", "iterate1"])
@pytest.mark.parametrize("cutoff", [True, False])
def test_fp64_single_step_every_node(D, dims, mode, cutoff):
    beta = 0.995
    f0 = noisy_state(D, dims, 4e-3)
    gm, om = MODES[mode]
    f_gpu = gpu_run(D, dims, beta, f0, 1, "f64", alpha_mode=gm, cutoff=cutoff)
    f_ora, a_ora, br_ora, _ = O.step(D, dims, f0, beta, cutoff=cutoff, mode=om, want_alpha=True)
    # branch decisions through the alpha field of the same pre-collision state
    with E.Simulation(LAT[D], dims, beta, storage="f64", alpha_mode=gm, cutoff=cutoff) as sim:
        sim.set_populations(f0)
        a_gpu, fl = sim.alpha_field()
        a_gpu, fl = a_gpu.cpu().numpy(), fl.cpu().numpy()
    agree = check_branches(D, O.stream(D, dims, f0), fl, br_ora, 1e-12)
    assert np.max(np.abs(a_gpu[agree] - a_ora[agree])) < 1e-12
    rel = np.abs(f_gpu - f_ora) / np.abs(f_ora)
    assert np.max(rel[:, agree]) < 1e-12
    if mode != "lbgk" and not cutoff:
        assert np.all(fl != E.ELBM_BRANCH_CUTOFF)  # every node on the closed form
    if mode == "lbgk":
        assert np.all(fl == E.ELBM_BRANCH_CUTOFF) and np.all(a_gpu == 2.0)


@pytest.mark.parametrize("b_variant", [E.ELBM_B_DERIVED, E.ELBM_B_PRINTED])
def test_fp64_b_variants(b_variant):
    D, dims, beta = 3, (21, 17, 9), 0.9
    f0 = noisy_state(D, dims, 2e-2, seed=5)
    f_gpu = gpu_run(D, dims, beta, f0, 2, "f64", cutoff=False, b_variant=b_variant)
    f_ora, *_ = O.step(D, dims, f0, beta, cutoff=False, b_variant=b_variant, nsteps=2)
    assert np.max(np.abs(f_gpu - f_ora) / f_ora) < 1e-12


@pytest.mark.parametrize("D,dims,nsteps", [(2, (96, 53, 1), 25), (3, (23, 18, 13), 8)])
def test_fp64_multistep(D, dims, nsteps):
    beta = 0.999
    f0 = noisy_state(D, dims, 1e-2, seed=9)
    f_gpu = gpu_run(D, dims, beta, f0, nsteps, "f64", cutoff=False)
    f_ora, *_ = O.step(D, dims, f0, beta, cutoff=False, nsteps=nsteps)
    assert np.max(np.abs(f_gpu - f_ora) / f_ora) < 1e-12


def test_config1_taylor_green_64_fp64_1000_steps():
    """D2Q9 64^2 Taylor-Green, u0 = 0.01, beta = 0.9, 1000 steps, FP64: u within 1e-12
    relative of the oracle with every node on the closed-form path (cutoff off), and with
    the paper's cutoff on (both sides decide in FP64)."""
    L, beta = 64, 0.9
    dims = (L, L, 1)
    X, Y, _ = inputs.grid(dims)
    rho, u = inputs.taylor_green_2d(X, Y, L, u0=0.01)
    for cutoff in (False, True):
        with E.Simulation(E.ELBM_D2Q9, dims, beta, storage="f64", cutoff=cutoff) as sim:
            sim.init_equilibrium(rho, u)
            f_init = sim.get_populations()
            sim.step(1000)
            r_g, u_g = [t.cpu().numpy() for t in sim.moments()]
        f_o0 = O.init_equilibrium(2, rho, u)
        assert np.max(np.abs(f_init - f_o0) / f_o0) < 1e-15
        f_o, *_ = O.step(2, dims, f_o0, beta, cutoff=cutoff, nsteps=1000)
        r_o, u_o = O.moments_field(2, f_o)
        assert np.linalg.norm(u_g - u_o) / np.linalg.norm(u_o) < 1e-12
        assert np.max(np.abs(r_g - r_o)) < 1e-12


def test_config1_alpha_field_fp64():
    """The 64^2 Taylor-Green configuration (u0 = 0.01, beta = 0.9, cutoff off), every 100
    steps up to 1000: the GPU's FP64 path length of the next collision (elbm_alpha_field) on
    the oracle's state equals the oracle's alpha_H to 1e-12, and on the GPU's own state
    (which differs from the oracle's by rounding order) to 1e-11."""
    L, beta = 64, 0.9
    dims = (L, L, 1)
    X, Y, _ = inputs.grid(dims)
    rho, u = inputs.taylor_green_2d(X, Y, L, u0=0.01)
    f_o = O.init_equilibrium(2, rho, u)
    with E.Simulation(E.ELBM_D2Q9, dims, beta, storage="f64", cutoff=False) as run, \
            E.Simulation(E.ELBM_D2Q9, dims, beta, storage="f64", cutoff=False) as probe:
        run.set_populations(f_o)
        for t in range(100, 1001, 100):
            f_o, *_ = O.step(2, dims, f_o, beta, cutoff=False, nsteps=100)
            run.step(100)
            a_o, br_o, _ = O.alpha_field(2, O.stream(2, dims, f_o), beta, cutoff=False)
            probe.set_populations(f_o)
            a_p, fl_p = [x.cpu().numpy() for x in probe.alpha_field()]
            a_r, _ = [x.cpu().numpy() for x in run.alpha_field()]
            assert np.array_equal(fl_p, br_o)
            assert np.max(np.abs(a_p - a_o)) < 1e-12, t
            assert np.max(np.abs(a_r - a_o)) < 1e-11, t


# ---------------------------------------------------------------------------
# FP32
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("D,dims", [(2, (300, 37, 1)), (3, (37, 19, 11))])
@pytest.mark.parametrize("cutoff", [True, False])
@pytest.mark.parametrize("storage", ["f32", "f32dev"])
def test_fp32_single_step(D, dims, cutoff, storage):
    beta = 0.999
    f0, f_in = stored(D, noisy_state(D, dims, 4e-3), storage)
    f_gpu = gpu_run(D, dims, beta, f0, 1, storage, cutoff=cutoff)
    f_ora, a_ora, br_ora, _ = O.step(D, dims, f_in, beta, cutoff=cutoff, want_alpha=True)
    with E.Simulation(LAT[D], dims, beta, storage=storage, cutoff=cutoff) as sim:
        sim.set_populations(f0)
        a_gpu, fl = [t.cpu().numpy() for t in sim.alpha_field()]
    agree = check_branches(D, O.stream(D, dims, f_in), fl, br_ora, 1e-6)
    assert np.max(np.abs(a_gpu[agree] - a_ora[agree])) < 2e-5
    rel = np.abs(f_gpu - f_ora) / f_ora
    assert np.max(rel[:, agree]) < 2e-6


@pytest.mark.parametrize("D,dims", [(2, (211, 53, 1)), (3, (31, 17, 13))])
@pytest.mark.parametrize("storage", ["f32", "f32dev"])
def test_fp32_series_and_exact_paths(D, dims, storage):
    """Noise levels whose |x|max straddles 0.04, where the FP32 collision switches between
    power-series and per-population forms of its coefficients: both agree with the oracle
    at FP32 precision, and nodes on either side are present."""
    beta = 0.995
    f0, f_in = stored(D, noisy_state(D, dims, 0.032 if D == 2 else 0.024, seed=43), storage)
    f_gpu = gpu_run(D, dims, beta, f0, 1, storage, cutoff=True)
    f_pre = O.stream(D, dims, f_in)
    f_ora, a_ora, br_ora, _ = O.step(D, dims, f_in, beta, cutoff=True, want_alpha=True)
    xm = xabsmax_of(D, f_pre)
    assert np.sum(xm < 0.038) > 50 and np.sum(xm > 0.042) > 50
    with E.Simulation(LAT[D], dims, beta, storage=storage, cutoff=True) as sim:
        sim.set_populations(f0)
        a_gpu, fl = [t.cpu().numpy() for t in sim.alpha_field()]
    agree = check_branches(D, f_pre, fl, br_ora, 1e-6)
    assert np.max(np.abs(a_gpu[agree] - a_ora[agree])) < 2e-5
    rel = np.abs(f_gpu - f_ora) / f_ora
    assert np.max(rel[:, agree]) < 2e-6


@pytest.mark.parametrize("storage", ["f32", "f32dev"])
@pytest.mark.parametrize("mode,b_variant", [("higher", E.ELBM_B_DERIVED), ("higher", E.ELBM_B_PRINTED),
                                            ("lower", E.ELBM_B_DERIVED), ("lbgk", E.ELBM_B_DERIVED)])
def test_fp32_d2q9_two_node_collision_mixed_branches(storage, mode, b_variant):
    """D2Q9 FP32 steps collide two nodes per thread (x and x + 32), one in each lane of the
    paired FP32 instructions.  The noise amplitude rises geometrically along x, from 1e-5
    to 0.9, so the two nodes of a thread often take different branches (cutoff, solved,
    clamped) and different coefficient forms; every mode and both readings of b against
    the oracle, on a ragged width (a thread's second node past the end of its row is not
    stored)."""
    D, dims, beta = 2, (203, 41, 1), 0.99
    X, Y, _ = inputs.grid(dims)
    rho, u = inputs.taylor_green_2d(X, Y, dims[0], u0=0.05)
    amp = 10.0 ** np.interp(X, [0, dims[0] - 1], [-5.0, np.log10(0.9)])
    f = O.init_equilibrium(D, rho, u) * inputs.population_noise(9, X.size, amp, seed=61)
    f0, f_in = stored(D, f, storage)
    gm, om = MODES[mode]
    f_gpu = gpu_run(D, dims, beta, f0, 1, storage, alpha_mode=gm, b_variant=b_variant, cutoff=True)
    f_ora, a_ora, br_ora, _ = O.step(D, dims, f_in, beta, cutoff=True, mode=om, b_variant=b_variant,
                                     want_alpha=True)
    if mode != "lbgk":
        for b, least in ((O.BRANCH_CUTOFF, 500), (O.BRANCH_SOLVED, 5000), (O.BRANCH_CLAMPED, 10)):
            assert np.sum(br_ora == b) > least, b
    with E.Simulation(LAT[D], dims, beta, storage=storage, alpha_mode=gm, b_variant=b_variant,
                      cutoff=True) as sim:
        sim.set_populations(f0)
        _, fl = [t.cpu().numpy() for t in sim.alpha_field()]
    f_pre = O.stream(D, dims, f_in)
    agree = check_branches(D, f_pre, fl, br_ora, 1e-6)
    # far from equilibrium f* = f + alpha beta (f^eq - f) cancels (to 1e-2 of f and below
    # at the highest amplitudes), so the error is measured against the size of its terms
    feq = O.init_equilibrium(D, *O.moments_field(D, f_pre))
    scale = f_pre + 2.5 * np.abs(feq - f_pre)
    err = np.abs(f_gpu - f_ora) / scale
    assert np.max(err[:, agree]) < 2e-6


@pytest.mark.parametrize("storage", ["f32", "f32dev"])
def test_load_policy_after_diagnostics_changes_no_result(storage):
    """The D3Q27 step switches to evict-first population loads once the last diagnostics
    saw most nodes on the longer coefficient forms; the arithmetic is the same, so the
    populations after the steps are identical with and without that switch."""
    D, dims, beta = 3, (40, 12, 9), 0.99
    f0, _ = stored(D, noisy_state(D, dims, 3e-2, seed=71), storage)
    outs = []
    for diag_first in (False, True):
        with E.Simulation(E.ELBM_D3Q27, dims, beta, storage=storage) as sim:
            sim.set_populations(f0)
            if diag_first:
                d = sim.diagnostics()
                assert d["n_xmax_band"][2] + d["n_xmax_band"][3] > d["n_nodes"] // 2
            sim.step(3)
            outs.append(sim.get_populations())
    assert np.array_equal(outs[0], outs[1])


@pytest.mark.parametrize("D,dims", [(2, (131, 29, 1)), (3, (21, 13, 9))])
@pytest.mark.parametrize("storage", ["f32", "f32dev"])
def test_fp32_iterate1_mode(D, dims, storage):
    """alpha_Iterate1 (Sec. IV) in FP32 against the oracle, including nodes far enough
    from equilibrium that the Newton step is undefined and alpha_Lower is kept."""
    beta = 0.99
    f0, f_in = stored(D, noisy_state(D, dims, 0.5, seed=8), storage)
    gm, om = MODES["iterate1"]
    f_gpu = gpu_run(D, dims, beta, f0, 1, storage, alpha_mode=gm, cutoff=True)
    f_ora, a_ora, br_ora, _ = O.step(D, dims, f_in, beta, cutoff=True, mode=om, want_alpha=True)
    with E.Simulation(LAT[D], dims, beta, storage=storage, alpha_mode=gm, cutoff=True) as sim:
        sim.set_populations(f0)
        a_gpu, fl = [t.cpu().numpy() for t in sim.alpha_field()]
    agree = check_branches(D, O.stream(D, dims, f_in), fl, br_ora, 1e-6)
    assert np.sum(br_ora == O.BRANCH_CLAMPED) > 0 and np.sum(br_ora == O.BRANCH_SOLVED) > 0
    err = np.abs(a_gpu - a_ora) / a_ora
    assert np.quantile(err[agree], 0.999) < 1e-4 and np.max(err[agree]) < 1e-2
    rel = np.abs(f_gpu - f_ora) / f_ora
    assert np.quantile(rel[:, agree], 0.999) < 1e-4


@pytest.mark.parametrize("D,dims", [(2, (77, 41, 1)), (3, (19, 17, 10))])
@pytest.mark.parametrize("storage,tol", [("f64", 1e-13), ("f32", 1e-5)])
def test_subgrid_viscosity(D, dims, storage, tol):
    """nu_T = theta (2 - alpha) / (2 alpha beta), theta = 1/3 (Sec. VI, Eq. nuT), from the
    oracle's path length of the same state; zero exactly on cutoff nodes."""
    beta = 0.998
    f0 = noisy_state(D, dims, 0.6e-3, seed=17, u0=0.002)  # |x|max straddles the 1e-3 cutoff
    if storage == "f32":
        f0 = f0.astype(np.float32)
    f_pre = O.stream(D, dims, f0.astype(np.float64))
    with E.Simulation(LAT[D], dims, beta, storage=storage, cutoff=True) as sim:
        sim.set_populations(f0)
        nut = sim.subgrid_viscosity().cpu().numpy()
        _, fl = [t.cpu().numpy() for t in sim.alpha_field()]
    a_ora, br_ora, _ = O.alpha_field(D, f_pre, beta, cutoff=True)
    agree = check_branches(D, f_pre, fl, br_ora, 1e-12 if storage == "f64" else 1e-6)
    want = (1.0 / 3.0) * (2.0 - a_ora) / (2.0 * a_ora * beta)
    assert np.max(np.abs(nut - want)[agree]) < tol
    assert np.all(nut[fl == E.ELBM_BRANCH_CUTOFF] == 0.0)
    assert np.any(fl == E.ELBM_BRANCH_CUTOFF) and np.any(fl == E.ELBM_BRANCH_SOLVED)


@pytest.mark.parametrize("D,L,nsteps", [(2, 96, 40), (3, 32, 20)])
@pytest.mark.parametrize("storage", ["f32", "f32dev"])
def test_fp32_taylor_green_velocity(D, L, nsteps, storage):
    """Taylor-Green vortex (u0 = 0.05, beta = 0.999) from the equilibrium, FP32 storage and
    arithmetic: u within 1e-5 relative (L2) of the FP64 oracle started from the same
    FP32-rounded populations, with the closed-form alpha active on most nodes."""
    beta = 0.999
    dims = (L, L, 1) if D == 2 else (L, L, L)
    X, Y, Z = inputs.grid(dims)
    rho, u = (inputs.taylor_green_2d(X, Y, L, u0=0.05) if D == 2
              else inputs.taylor_green_3d(X, Y, Z, L, u0=0.05))
    with E.Simulation(LAT[D], dims, beta, storage=storage) as sim:
        sim.init_equilibrium(rho, u)
        f_init = populations(D, sim.get_populations(), storage)
        sim.step(nsteps)
        r_g, u_g = [t.cpu().numpy() for t in sim.moments()]
        d = sim.diagnostics()
    _, f_o0 = stored(D, O.init_equilibrium(D, rho, u), storage)
    assert np.array_equal(f_init, f_o0)
    f_o, *_ = O.step(D, dims, f_o0, beta, nsteps=nsteps)
    r_o, u_o = O.moments_field(D, f_o)
    assert np.linalg.norm(u_g - u_o) / np.linalg.norm(u_o) < 1e-5
    assert np.max(np.abs(r_g - r_o)) < 1e-5
    assert d["n_solved"] > 0.5 * X.size


@pytest.mark.parametrize("D,dims,nsteps", [(2, (128, 77, 1), 20), (3, (29, 23, 17), 10)])
@pytest.mark.parametrize("storage", ["f32", "f32dev"])
def test_fp32_noisy_multistep(D, dims, nsteps, storage):
    """Strongly non-equilibrium start (0.3% noise on every population): u within 1e-5
    relative (L2) of the FP64 oracle started from the same stored state, with the cutoff on
    and off."""
    beta = 0.999
    f0, f_in = stored(D, noisy_state(D, dims, 3e-3, seed=13), storage)
    for cutoff in (False, True):
        with E.Simulation(LAT[D], dims, beta, storage=storage, cutoff=cutoff) as sim:
            sim.set_populations(f0)
            sim.step(nsteps)
            r_g, u_g = [t.cpu().numpy() for t in sim.moments()]
            f_g = populations(D, sim.get_populations(), storage)
        f_o, *_ = O.step(D, dims, f_in, beta, cutoff=cutoff, nsteps=nsteps)
        r_o, u_o = O.moments_field(D, f_o)
        assert np.linalg.norm(u_g - u_o) / np.linalg.norm(u_o) < 1e-5
        assert np.max(np.abs(r_g - r_o)) < 1e-5
        assert np.max(np.abs(f_g - f_o) / f_o) < nsteps * 2e-6


def test_fp32dev_taylor_green_1000_steps():
    """D3Q27 Taylor-Green vortex (u0 = 0.05, beta = 0.999, the benchmark flow's parameters)
    on 64^3 for 1000 steps from the equilibrium in FP32 deviation storage: u within 1e-5
    relative (L2) of the FP64 oracle started from the same stored state.  At this length
    the FP32 storage of f_i rounds at the scale of w_i every step and drifts past 1e-5;
    storing d_i = f_i - c_i and colliding on it rounds at the scale of d_i instead."""
    L, beta, nsteps = 64, 0.999, 1000
    dims = (L, L, L)
    X, Y, Z = inputs.grid(dims)
    rho, u = inputs.taylor_green_3d(X, Y, Z, L, u0=0.05)
    with E.Simulation(E.ELBM_D3Q27, dims, beta, storage="f32dev") as sim:
        sim.init_equilibrium(rho, u)
        f_init = populations(3, sim.get_populations(), "f32dev")
        sim.step(nsteps)
        _, u_g = [t.cpu().numpy() for t in sim.moments()]
        d = sim.diagnostics()
    f_o, *_ = O.step(3, dims, f_init, beta, nsteps=nsteps)
    _, u_o = O.moments_field(3, f_o)
    assert np.linalg.norm(u_g - u_o) / np.linalg.norm(u_o) < 1e-5
    assert d["n_solved"] > 0.5 * X.size and d["n_nonpositive"] == 0


def test_fp32_full_size_sampled_nodes():
    """D3Q27 256^3 Taylor-Green (u0 = 0.05, beta = 0.999) in the benchmark's launch
    configuration.  After k = 8 steps, sampled nodes against the oracle, which recomputes
    each from a (2k+3)^3 box of its own initial state (a node after k steps depends only on
    its (2k+1)^3 neighbourhood, so the box's wrap-around never reaches it).  Then 300
    steps in all: conservation, H non-increasing, positivity and the alpha range over the
    whole field (the closed-form branch takes over as the non-equilibrium part grows)."""
    L, beta, k = 256, 0.999, 8
    dims = (L, L, L)
    X, Y, Z = inputs.grid(dims)
    rho, u = inputs.taylor_green_3d(X, Y, Z, L, u0=0.05)
    with E.Simulation(E.ELBM_D3Q27, dims, beta, storage="f32") as sim:
        sim.init_equilibrium(rho, u)
        del X, Y, Z, rho, u
        d0 = sim.diagnostics()
        sim.step(k)
        f_gpu = sim.get_populations()
        dk = sim.diagnostics()
        sim.step(300 - k)
        d1 = sim.diagnostics(with_hist=True)
    rng = np.random.default_rng(17)
    samples = rng.integers(0, L, size=(60, 3))
    samples[:8] = [[0, 0, 0], [L - 1, L - 1, L - 1], [0, L - 1, 5], [L - 1, 0, 200],
                   [128, 0, L - 1], [1, 2, 3], [255, 128, 0], [64, 64, 64]]
    B = 2 * k + 3
    off = np.arange(B) - B // 2
    bz, by, bx = np.meshgrid(off, off, off, indexing="ij")
    centre = (B // 2 * B + B // 2) * B + B // 2
    worst = 0.0
    for (sx, sy, sz) in samples:
        gx, gy, gz = (sx + bx.ravel()) % L, (sy + by.ravel()) % L, (sz + bz.ravel()) % L
        r, uu = inputs.taylor_green_3d(gx, gy, gz, L, u0=0.05)
        fb = O.init_equilibrium(3, r, uu).astype(np.float32).astype(np.float64)
        fb, *_ = O.step(3, (B, B, B), fb, beta, nsteps=k)
        n = (sz * L + sy) * L + sx
        worst = max(worst, np.max(np.abs(f_gpu[:, n].astype(np.float64) - fb[:, centre]) / fb[:, centre]))
    assert worst < k * 2e-6
    # FP32 storage rounds every population every step; the domain sums may drift by a
    # rounding bias of at most ~1e-8 relative per step
    for d, steps in ((dk, k), (d1, 300)):
        assert abs(d["mass"] - d0["mass"]) < 1e-8 * steps * d0["mass"]
        assert np.max(np.abs(np.array(d["momentum"]) - np.array(d0["momentum"]))) < 1e-8 * steps * d0["mass"]
        assert d["n_nonpositive"] == 0
        # with the paper's cutoff, alpha = 2 need not satisfy the H theorem on
        # near-equilibrium nodes (the guarantee is for alpha_H): violations only there
        assert d["n_dH_positive"] <= d["n_cutoff"]
    assert dk["H"] <= d0["H"] and d1["H"] <= dk["H"]
    assert d1["alpha_hist"].sum() == L ** 3
    assert d1["n_solved"] > L ** 3 // 2 and 1.9 < d1["alpha_min"] <= d1["alpha_max"] < 2.1


# ---------------------------------------------------------------------------
# deviation storage (FP16 / BF16 of f - w rho0, FP32 arithmetic)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("storage,mant_bits", [("f16dev", 10), ("bf16dev", 7)])
def test_deviation_storage_single_step(storage, mant_bits):
    D, dims, beta = 3, (31, 17, 9), 0.999
    c, w = O.lattice(D)
    f0 = noisy_state(D, dims, 3e-3, seed=21)
    dev = f0 - w[:, None]
    with E.Simulation(LAT[D], dims, beta, storage=storage) as sim:
        # the stored deviation, rounded to nearest by numpy
        if storage == "f16dev":
            q = dev.astype(np.float16)
            deq = q.astype(np.float64) + w[:, None]
            sim.set_populations(q)
        else:
            b = dev.astype(np.float32).view(np.uint32)
            b = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16).astype(np.uint16)  # RNE to bf16
            deq = (b.astype(np.uint32) << 16).view(np.float32).astype(np.float64) + w[:, None]
            sim.set_populations(b)
        sim.step(1)
        raw = sim.get_populations()
    if storage == "f16dev":
        got = raw.astype(np.float64) + w[:, None]
    else:
        got = (raw.astype(np.uint32) << 16).view(np.float32).astype(np.float64) + w[:, None]
    want, *_ = O.step(D, dims, deq, beta, nsteps=1)
    err = np.abs(got - want)
    bound = 2.0 ** -(mant_bits + 1) * np.abs(want - w[:, None]) * 1.01 + 4e-6 * want + 1e-7
    assert np.all(err <= bound)


# ---------------------------------------------------------------------------
# companions: init, moments, alpha field, diagnostics, edge cases
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("storage", ["f64", "f32", "f32dev"])
def test_init_and_moments(storage):
    D, dims = 3, (19, 13, 7)
    rng = np.random.default_rng(23)
    N = int(np.prod(dims))
    rho = 1 + 0.05 * (2 * rng.random(N) - 1)
    u = 0.1 * rng.standard_normal((3, N))
    with E.Simulation(E.ELBM_D3Q27, dims, 0.9, storage=storage) as sim:
        sim.init_equilibrium(rho, u)
        f = populations(3, sim.get_populations(), storage)
        r_g, u_g = [t.cpu().numpy() for t in sim.moments()]
    f_o = O.init_equilibrium(3, rho, u)
    if storage == "f32dev":
        # f^eq - c_i rounded once to FP32: half an ulp of the deviation
        c = dev_ref(3)[:, None]
        assert np.all(np.abs(f - f_o) <= 2.0 ** -24 * np.abs(f_o - c) + 1e-15)
    else:
        tol = 1e-15 if storage == "f64" else 6e-8
        assert np.max(np.abs(f - f_o) / f_o) < tol
    if storage == "f32":
        # rounded once from a ~44-bit value: the FP32 rounding of the oracle's f^eq, but
        # where f^eq lies within ~2^-43 of a rounding midpoint (none expected here)
        assert np.mean(f == f_o.astype(np.float32).astype(np.float64)) > 0.9999
    r_o, u_o = O.moments_field(3, f)
    assert np.max(np.abs(r_g - r_o)) < 1e-14 and np.max(np.abs(u_g - u_o)) < 1e-14


@pytest.mark.parametrize("storage", ["f32", "f32dev", "f16dev"])
def test_moments_are_exact_sums_of_the_stored_values(storage):
    """elbm_moments sums the stored FP32 values exactly and rounds once to FP64: rho and
    the momentum equal math.fsum of the populations (the correctly rounded exact sums), u
    their quotient to two FP64 ulp, on populations spread over 2^-28 .. 1 and of both signs;
    a node holding a non-finite value gives non-finite moments."""
    import math

    D, dims = 3, (16, 5, 3)
    N = int(np.prod(dims))
    rng = np.random.default_rng(29)
    mag = 2.0 ** rng.uniform(-28, 0, size=(27, N))
    raw = (mag * np.where(rng.random((27, N)) < 0.2, -1.0, 1.0)).astype(np.float32)
    if storage == "f16dev":
        raw = (raw * 1e-2).astype(np.float16)
    raw[:, 5] = 0.0
    with E.Simulation(E.ELBM_D3Q27, dims, 0.9, storage=storage) as sim:
        sim.set_populations(raw)
        f = populations(3, sim.get_populations(), storage) if storage != "f16dev" else (
            dev_ref(3)[:, None] + sim.get_populations().astype(np.float64))
        r_g, u_g = [t.cpu().numpy() for t in sim.moments()]
        bad = raw.copy()
        bad[4, 7] = np.inf
        sim.set_populations(bad)
        r_b, u_b = [t.cpu().numpy() for t in sim.moments()]
    c, _ = O.lattice(3)
    for n in range(N):
        col = [float(v) for v in f[:, n]]
        rho = math.fsum(col)
        assert r_g[n] == rho, n
        if rho == 0.0:  # the all-zero node (FP32 storage): u = 0/0
            continue
        for a in range(3):
            j = math.fsum(c[i, a] * col[i] for i in range(27))
            assert abs(u_g[a, n] - j / rho) <= 2 * np.spacing(abs(j / rho)) + 1e-300, (n, a)
    assert not np.isfinite(r_b[7]) or not np.all(np.isfinite(u_b[:, 7]))
    assert np.all(np.isfinite(r_b[np.arange(N) != 7]))


def test_diagnostics_against_oracle():
    D, dims, beta = 2, (160, 90, 1), 0.995
    f0 = noisy_state(D, dims, 5e-3, seed=29)
    with E.Simulation(E.ELBM_D2Q9, dims, beta, storage="f64", cutoff=False) as sim:
        sim.set_populations(f0)
        d = sim.diagnostics(with_hist=True)
    c, w = O.lattice(D)
    fs = O.stream(D, dims, f0)
    _, a, br, _ = O.collide(D, fs, beta, cutoff=False, want_alpha=True)
    _, _, _, dH = O.collide(D, fs, beta, cutoff=False, want_dH=True)
    assert abs(d["mass"] - f0.sum()) < 1e-12 * f0.sum()
    assert np.allclose(d["momentum"][:2], (c.T @ f0).sum(axis=1), rtol=0, atol=1e-11)
    assert abs(d["H"] - O.H_total(D, f0)) < 1e-12 * abs(d["H"])
    assert d["n_solved"] == np.sum(br == O.BRANCH_SOLVED)
    assert d["n_clamped"] == np.sum(br == O.BRANCH_CLAMPED)
    assert abs(d["alpha_min"] - a.min()) < 1e-12 and abs(d["alpha_max"] - a.max()) < 1e-12
    assert abs(d["alpha_mean"] - a.mean()) < 1e-12
    assert abs(d["dH_max"] - dH.max()) < 1e-14 and d["dH_max"] <= 0
    assert d["n_dH_positive"] == 0 and d["n_nonpositive"] == 0
    hist = d["alpha_hist"]
    assert hist.sum() == a.size
    edges = np.linspace(1.9, 2.1, E.ELBM_HIST_BINS + 1)
    inner = np.histogram(a[(a >= 1.9) & (a < 2.1)], bins=edges)[0]
    # bin edges are decided in two different floating-point formulas: allow a few moves
    assert np.sum(np.abs(hist[1:-1] - inner)) <= 4


@pytest.mark.parametrize("D,dims,storage,kernel,force", [
    (2, (77, 41, 1), "f32", E.ELBM_KERNEL_DIRECT, False),
    (3, (23, 19, 11), "f32", E.ELBM_KERNEL_DIRECT, False),
    (3, (23, 19, 11), "f32dev", E.ELBM_KERNEL_DIRECT, False),
    (3, (23, 19, 11), "f64", E.ELBM_KERNEL_DIRECT, False),
    (2, (64, 40, 1), "f32", E.ELBM_KERNEL_ROWS, False),   # diagnostics pass, then the step
    (2, (61, 33, 1), "f32", E.ELBM_KERNEL_DIRECT, True),  # body force: diagnostics pass first
])
def test_step_diag_equals_diagnostics_then_steps(D, dims, storage, kernel, force):
    """elbm_step_diag(n) reports what elbm_diagnostics reports before elbm_step(n), and
    leaves the same state; called twice in a row."""
    beta = 0.993
    f0 = noisy_state(D, dims, 4e-3, seed=47)
    if storage != "f64":
        f0 = stored(D, f0, storage)[0]
    F = np.array([1e-4, -2e-4, 5e-5])[:D] if force else None
    with E.Simulation(LAT[D], dims, beta, storage=storage, kernel=kernel) as a, \
            E.Simulation(LAT[D], dims, beta, storage=storage, kernel=kernel) as b:
        for sim in (a, b):
            sim.set_populations(f0)
            sim.set_force(F)
        for n in (3, 1):
            want = a.diagnostics(with_hist=True)
            a.step(n)
            got = b.step_diag(n, with_hist=True)
            fa = populations(D, a.get_populations(), storage)
            fb = populations(D, b.get_populations(), storage)
            assert np.max(np.abs(fa - fb) / np.abs(fa)) < (1e-14 if storage == "f64" else 1e-6)
            for k in ("n_nodes", "n_cutoff", "n_solved", "n_clamped", "n_nonpositive", "n_dH_positive"):
                assert got[k] == want[k], k
            assert np.array_equal(got["alpha_hist"], want["alpha_hist"])
            rel = 1e-12 if storage == "f64" else 1e-6
            assert abs(got["mass"] - want["mass"]) <= rel * want["mass"]
            assert abs(got["H"] - want["H"]) <= rel * abs(want["H"])
            assert np.allclose(got["momentum"], want["momentum"], rtol=0, atol=rel * want["mass"])
            for k in ("alpha_min", "alpha_max", "alpha_mean", "dH_max"):
                assert abs(got[k] - want[k]) <= rel * 2.0 + 1e-15, k
            assert a.steps == b.steps


def test_nonphysical_state_is_reported():
    D, dims = 2, (16, 8, 1)
    f0 = noisy_state(D, dims, 1e-3)
    f0[4, 37] = -1e-3
    with E.Simulation(E.ELBM_D2Q9, dims, 0.9, storage="f64") as sim:
        sim.set_populations(f0)
        with pytest.raises(E.ElbmError) as ei:
            sim.diagnostics()
        assert ei.value.code == E.ELBM_ERR_NONPHYSICAL
        d = sim.diagnostics(allow_nonphysical=True)
        assert d["n_nonpositive"] >= 1


def test_clamp_branch_matches_oracle():
    """Far from equilibrium (noise 0.9 on every population) the positivity clamp acts on
    many nodes; GPU and oracle agree on which and on the clamped alpha (FP64)."""
    D, dims, beta = 2, (64, 48, 1), 0.99
    f0 = noisy_state(D, dims, 0.9, seed=31)
    f_gpu = gpu_run(D, dims, beta, f0, 1, "f64")
    f_ora, a_ora, br_ora, _ = O.step(D, dims, f0, beta, want_alpha=True)
    with E.Simulation(E.ELBM_D2Q9, dims, beta, storage="f64") as sim:
        sim.set_populations(f0)
        a_gpu, fl = [t.cpu().numpy() for t in sim.alpha_field()]
    assert np.sum(br_ora == O.BRANCH_CLAMPED) > 20
    assert np.array_equal(fl, br_ora)
    assert np.max(np.abs(a_gpu - a_ora)) < 1e-12
    assert np.max(np.abs(f_gpu - f_ora) / f_ora) < 1e-11
    assert np.all(f_gpu > 0)


@pytest.mark.parametrize("D,dims", [(2, (1, 1, 1)), (2, (1, 7, 1)), (2, (5, 1, 1)),
                                    (3, (1, 1, 1)), (3, (1, 4, 3)), (3, (2, 2, 2))])
def test_degenerate_domains(D, dims):
    """Periodic wrap onto itself (a side of 1 or 2 nodes)."""
    f0 = noisy_state(D, dims, 1e-2, seed=37)
    f_gpu = gpu_run(D, dims, 0.97, f0, 3, "f64", cutoff=False)
    f_ora, *_ = O.step(D, dims, f0, 0.97, cutoff=False, nsteps=3)
    assert np.max(np.abs(f_gpu - f_ora) / f_ora) < 1e-12


@pytest.mark.parametrize("D,dims,storage", [(2, (3, 70001, 1), "f32"), (2, (2, 66000, 1), "f64"),
                                            (3, (2, 2, 65537), "f32"), (3, (2, 65537, 2), "f32dev")])
def test_one_dimensional_launch(D, dims, storage):
    """ny or nz above the grid limit of a 3D launch: the kernel runs on a 1D grid with
    64-bit node indices; same results as the oracle."""
    beta = 0.99
    f0 = noisy_state(D, dims, 3e-3, seed=41)
    f_in = f0
    if storage != "f64":
        f0, f_in = stored(D, f0, storage)
    f_gpu = gpu_run(D, dims, beta, f0, 2, storage, cutoff=False)
    f_ora, *_ = O.step(D, dims, f_in, beta, cutoff=False, nsteps=2)
    tol = 1e-12 if storage == "f64" else 4e-6
    assert np.max(np.abs(f_gpu - f_ora) / f_ora) < tol


def test_zero_steps_and_uniform_fixed_point():
    D, dims = 3, (9, 8, 7)
    N = int(np.prod(dims))
    u = np.repeat(np.array([[0.03], [-0.02], [0.01]]), N, axis=1)
    with E.Simulation(E.ELBM_D3Q27, dims, 0.95, storage="f64") as sim:
        sim.init_equilibrium(np.full(N, 1.2), u)
        f0 = sim.get_populations()
        sim.step(0)
        assert sim.steps == 0 and np.array_equal(sim.get_populations(), f0)
        sim.step(5)
        f5 = sim.get_populations()
        a, fl = [t.cpu().numpy() for t in sim.alpha_field()]
    # re-deriving f^eq from the moments of f^eq reproduces it to a few ulp per step
    assert np.max(np.abs(f5 - f0) / f0) < 1e-14
    assert np.all(a == 2.0) and np.all(fl == E.ELBM_BRANCH_CUTOFF)


@pytest.mark.parametrize("beta", [0.02, 0.5, 0.99999])
def test_beta_extremes(beta):
    D, dims = 2, (40, 30, 1)
    f0 = noisy_state(D, dims, 1e-2, seed=41)
    f_gpu = gpu_run(D, dims, beta, f0, 2, "f64", cutoff=False)
    f_ora, *_ = O.step(D, dims, f0, beta, cutoff=False, nsteps=2)
    assert np.max(np.abs(f_gpu - f_ora) / f_ora) < 1e-12


def test_host_buffers_end_to_end():
    """The C-ABI host-memory forms (init from host arrays, moments into host arrays)."""
    D, dims, beta = 2, (48, 40, 1), 0.99
    X, Y, _ = inputs.grid(dims)
    rho, u = inputs.shear_layer_2d(X, Y, 48)
    h = E.elbm_create(E.ELBM_D2Q9, dims, beta, opts=_opts(E.ELBM_STORE_F64))
    try:
        E.elbm_init_equilibrium(h, np.ascontiguousarray(rho), np.ascontiguousarray(u), E.ELBM_MEM_HOST)
        E.elbm_step(h, 4)
        r = np.empty(X.size)
        uu = np.empty((2, X.size))
        E.elbm_moments(h, r, uu, E.ELBM_MEM_HOST)
        assert E.elbm_step_count(h) == 4
    finally:
        E.elbm_destroy(h)
    f_o, *_ = O.step(2, dims, O.init_equilibrium(2, rho, u), beta, nsteps=4)
    r_o, u_o = O.moments_field(2, f_o)
    assert np.max(np.abs(uu - u_o)) < 1e-12 and np.max(np.abs(r - r_o)) < 1e-12


def _opts(storage):
    o = E.elbm_default_opts()
    o.storage = storage
    return o


# ---------------------------------------------------------------------------
# the two step kernels (DIRECT: L1 gathers; ROWS: bulk-async row staging)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("D,dims,storage", [
    (3, (32, 20, 12), "f32"), (3, (256, 6, 5), "f32"), (3, (512, 3, 2), "f32"), (3, (100, 7, 9), "f32"),
    (2, (1024, 24, 1), "f32"), (2, (300, 37, 1), "f32"), (2, (8, 3, 1), "f32"),
    (2, (64, 64, 1), "f16dev"), (3, (64, 16, 8), "bf16dev"), (3, (48, 5, 7), "f16dev"),
])
def test_rows_kernel_matches_direct(D, dims, storage):
    """Both kernels run the same per-node arithmetic on the same inputs; the compiler may
    contract multiply-adds differently in the two, so they agree to FP32 rounding (a few
    ulp per step), and after quantisation to the same 16-bit value or its neighbour."""
    f0 = noisy_state(D, dims, 5e-3, seed=43)
    c, w = O.lattice(D)
    outs = []
    for kern in (E.ELBM_KERNEL_DIRECT, E.ELBM_KERNEL_ROWS):
        with E.Simulation(LAT[D], dims, 0.999, storage=storage, kernel=kern) as sim:
            if storage == "f32":
                sim.set_populations(f0.astype(np.float32))
            else:
                rho, u = O.moments_field(D, f0)
                sim.init_equilibrium(rho, u)
            sim.step(6)
            outs.append(sim.get_populations())
            sim.synchronize()
    a, b = outs
    if storage == "f32":
        assert np.max(np.abs(a.astype(np.float64) - b) / np.abs(b)) < 6 * 1e-6
    elif storage == "f16dev":
        da, db = a.astype(np.float64), b.astype(np.float64)
        assert np.max(np.abs(da - db)) <= 4 * 2.0 ** -11 * np.max(np.abs(db)) + 1e-6
    else:
        fa = (a.astype(np.uint32) << 16).view(np.float32).astype(np.float64)
        fb = (b.astype(np.uint32) << 16).view(np.float32).astype(np.float64)
        assert np.max(np.abs(fa - fb)) <= 4 * 2.0 ** -8 * np.max(np.abs(fb)) + 1e-6


@pytest.mark.parametrize("D,dims,storage", [(2, (37, 8, 1), "f32"), (3, (30, 4, 4), "f32"),
                                            (2, (64, 8, 1), "f64"), (3, (1028, 2, 2), "f32")])
def test_rows_kernel_rejected_where_it_does_not_apply(D, dims, storage):
    with pytest.raises(E.ElbmError) as ei:
        E.Simulation(LAT[D], dims, 0.9, storage=storage, kernel=E.ELBM_KERNEL_ROWS)
    assert ei.value.code == E.ELBM_ERR_UNSUPPORTED


def test_error_paths_of_the_force_and_fused_diagnostics_calls():
    """Invalid arguments come back as status codes with a message, and leave the handle usable."""
    import torch

    D, dims = 2, (64, 16, 1)
    f0 = noisy_state(D, dims, 1e-3, seed=53)
    with E.Simulation(E.ELBM_D2Q9, dims, 0.95, storage="f32", kernel=E.ELBM_KERNEL_ROWS) as sim:
        sim.set_populations(f0.astype(np.float32))
        with pytest.raises(E.ElbmError) as ei:
            sim.set_force([1e-4, 0.0])  # the body force runs on the DIRECT kernel only
        assert ei.value.code == E.ELBM_ERR_UNSUPPORTED
        sim.set_force(None)  # no force: accepted
        sim.step(1)
    with E.Simulation(E.ELBM_D2Q9, dims, 0.95, storage="f32") as sim:
        sim.set_populations(f0.astype(np.float32))
        with pytest.raises(E.ElbmError) as ei:
            sim.set_force([np.nan, 0.0])
        assert ei.value.code == E.ELBM_ERR_ARG
        with pytest.raises(E.ElbmError) as ei:
            sim.step_diag(0)
        assert ei.value.code == E.ELBM_ERR_ARG
        g = torch.zeros((9, sim.N), dtype=torch.float32, device="cuda")
        with pytest.raises(E.ElbmError) as ei:
            E.elbm_adjoint_step_force(sim.h, sim.state_copy(), g, torch.empty_like(g), None)
        assert ei.value.code == E.ELBM_ERR_ARG
        with pytest.raises(E.ElbmError) as ei:
            E.elbm_adjoint_step_force(sim.h, sim.state_copy(), g, g,
                                      torch.zeros(2, dtype=torch.float64, device="cuda"))
        assert ei.value.code == E.ELBM_ERR_ARG  # g_t aliases g_next
        d = sim.step_diag(2)  # the handle still works
        assert d["n_nodes"] == sim.N and sim.steps == 2


@pytest.mark.parametrize("D,dims", [(3, (32, 20, 12)), (3, (256, 6, 5)), (2, (1024, 24, 1)), (2, (300, 37, 1))])
@pytest.mark.parametrize("storage", ["f32", "f32dev"])
def test_rows_kernel_against_oracle(D, dims, storage):
    """The ROWS kernel (rows staged in shared memory by bulk asynchronous copies) against the
    FP64 oracle directly: one step on every node with the closed form everywhere (cutoff
    off), within the FP32 per-step bound of the DIRECT kernel; then 12 steps with the
    cutoff on, u within 1e-5 relative (L2)."""
    beta = 0.999
    f0, f_in = stored(D, noisy_state(D, dims, 4e-3, seed=61), storage)
    f1 = gpu_run(D, dims, beta, f0, 1, storage, cutoff=False, kernel=E.ELBM_KERNEL_ROWS)
    f_o1, *_ = O.step(D, dims, f_in, beta, cutoff=False, nsteps=1)
    assert np.max(np.abs(f1 - f_o1) / f_o1) < 2e-6
    with E.Simulation(LAT[D], dims, beta, storage=storage, cutoff=True, kernel=E.ELBM_KERNEL_ROWS) as sim:
        sim.set_populations(f0)
        sim.step(12)
        _, u_g = [t.cpu().numpy() for t in sim.moments()]
        sim.synchronize()
    f_o, *_ = O.step(D, dims, f_in, beta, cutoff=True, nsteps=12)
    _, u_o = O.moments_field(D, f_o)
    assert np.linalg.norm(u_g - u_o) / np.linalg.norm(u_o) < 1e-5
