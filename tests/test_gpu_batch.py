"""Batched ensembles (one launch advances many independent domains) against the
oracle, and the four stepping modes against each other.

Each domain of a batch is an independent periodic lattice with its own size and
beta; the oracle advances each one separately.  GRAPH and LAUNCHES run the same
kernel launches (one replayed from a CUDA graph), so they agree bit for bit;
PER_DOMAIN runs the single-domain kernel and PERSISTENT the persistent one,
which the compiler may contract differently, so they agree to FP32 rounding.
"""
import numpy as np
import pytest

import oracle as O
from paper_2203_12946_gb300 import elbm as E
from paper_2203_12946_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    E.load()


def domain_state(D, dims, eps, seed):
    X, Y, Z = inputs.grid(dims)
    L = dims[0]
    rho, u = (inputs.taylor_green_2d(X, Y, L, u0=0.04) if D == 2
              else inputs.taylor_green_3d(X, Y, Z, L, u0=0.04))
    f = O.init_equilibrium(D, rho, u)
    return f * inputs.population_noise(3 ** D, X.size, eps, seed=seed)


@pytest.mark.parametrize("mode", [E.ELBM_BATCH_GRAPH, E.ELBM_BATCH_LAUNCHES, E.ELBM_BATCH_PER_DOMAIN,
                                  E.ELBM_BATCH_PERSISTENT])
def test_fp64_batch_matches_oracle_per_domain(mode):
    dims = [(20, 14, 1), (37, 23, 1), (64, 16, 1), (9, 9, 1), (130, 3, 1)]
    betas = [0.9, 0.99, 0.999, 0.95, 0.97]
    f0 = [domain_state(2, d, 4e-3, seed=k) for k, d in enumerate(dims)]
    with E.Ensemble(E.ELBM_D2Q9, dims, betas, storage="f64", cutoff=False) as ens:
        for k in range(len(dims)):
            ens.set_populations(k, f0[k])
        ens.step(3, mode)
        ens.step(2, mode)  # odd then even counts: buffer parity is tracked
        got = [ens.get_populations(k) for k in range(len(dims))]
    for k, d in enumerate(dims):
        want, *_ = O.step(2, d, f0[k], betas[k], cutoff=False, nsteps=5)
        assert np.max(np.abs(got[k] - want) / want) < 1e-12, k


@pytest.mark.parametrize("mode", [E.ELBM_BATCH_GRAPH, E.ELBM_BATCH_PERSISTENT])
def test_fp64_d3q27_batch_matches_oracle(mode):
    dims = [(12, 10, 8), (7, 9, 5), (16, 4, 4)]
    betas = [0.99, 0.9, 0.995]
    f0 = [domain_state(3, d, 3e-3, seed=10 + k) for k, d in enumerate(dims)]
    with E.Ensemble(E.ELBM_D3Q27, dims, betas, storage="f64") as ens:
        for k in range(len(dims)):
            ens.set_populations(k, f0[k])
        ens.step(4, mode)
        got = [ens.get_populations(k) for k in range(len(dims))]
    for k, d in enumerate(dims):
        want, *_ = O.step(3, d, f0[k], betas[k], nsteps=4)
        assert np.max(np.abs(got[k] - want) / want) < 1e-12, k


def test_modes_agree_and_tune_keeps_state():
    rng = np.random.default_rng(3)
    sides = rng.choice([64, 96, 128, 192], size=12)
    dims = [(int(s), int(s), 1) for s in sides]
    betas = list(rng.uniform(0.9, 0.999, size=len(dims)))
    states = []
    for k, d in enumerate(dims):
        rho, u = inputs.random_vortex_2d(d[0], rms=0.03, seed=100 + k)
        states.append((rho, u))
    outs = {}
    for mode in (E.ELBM_BATCH_GRAPH, E.ELBM_BATCH_LAUNCHES, E.ELBM_BATCH_PER_DOMAIN, E.ELBM_BATCH_PERSISTENT):
        with E.Ensemble(E.ELBM_D2Q9, dims, betas, storage="f32") as ens:
            for k, (rho, u) in enumerate(states):
                ens.init_equilibrium(k, rho, u)
            if mode == E.ELBM_BATCH_GRAPH:
                before = [ens.get_populations(k).copy() for k in range(len(dims))]
                bx, ms = ens.tune()
                assert bx in (64, 128, 256) and all(m > 0 for m in ms)
                after = [ens.get_populations(k) for k in range(len(dims))]
                assert all(np.array_equal(a, b) for a, b in zip(before, after))
            ens.step(7, mode)
            outs[mode] = [ens.get_populations(k) for k in range(len(dims))]
            d0 = ens.diagnostics(0)
            assert d0["n_nonpositive"] == 0
    for k in range(len(dims)):
        a = outs[E.ELBM_BATCH_GRAPH][k].astype(np.float64)
        b = outs[E.ELBM_BATCH_LAUNCHES][k].astype(np.float64)
        c = outs[E.ELBM_BATCH_PER_DOMAIN][k].astype(np.float64)
        d = outs[E.ELBM_BATCH_PERSISTENT][k].astype(np.float64)
        assert np.max(np.abs(a - b) / b) < 7 * 1e-6  # tune may pick another width
        assert np.max(np.abs(a - c) / c) < 7 * 1e-6
        assert np.max(np.abs(a - d) / d) < 7 * 1e-6


def test_ensemble_conserves_per_domain():
    """The batched-ensemble workload (random sides, random beta, random-phase vortex
    initial velocity): mass and momentum of every domain conserved over 50 steps."""
    rng = np.random.default_rng(20221203)
    sides = rng.choice([64, 96, 128, 192, 256, 384, 512], size=16)
    dims = [(int(s), int(s), 1) for s in sides]
    betas = list(rng.uniform(0.9, 0.999, size=len(dims)))
    with E.Ensemble(E.ELBM_D2Q9, dims, betas, storage="f32") as ens:
        for k, d in enumerate(dims):
            rho, u = inputs.random_vortex_2d(d[0], rms=0.03, seed=k)
            ens.init_equilibrium(k, rho, u)
        d0 = [ens.diagnostics(k) for k in range(len(dims))]
        ens.tune()
        ens.step(50)
        d1 = [ens.diagnostics(k) for k in range(len(dims))]
    for a, b in zip(d0, d1):
        assert abs(b["mass"] - a["mass"]) < 50 * 1e-8 * a["mass"]
        assert np.max(np.abs(np.array(b["momentum"]) - np.array(a["momentum"]))) < 50 * 1e-8 * a["mass"]
        assert b["n_nonpositive"] == 0


@pytest.mark.parametrize("storage", ["f32", "f16dev"])
def test_persistent_matches_graph_on_the_ensemble_workload(storage):
    """The 16-domain random ensemble (sides 64..512, so large domains are shared by many
    blocks of the persistent launch and some blocks span several small domains): 101
    persistent steps, issued as 1 + 100 (both buffer parities), agree with the
    graph-replayed launches to FP32 rounding, and synchronising reports no expired wait."""
    rng = np.random.default_rng(20221203)
    sides = rng.choice([64, 96, 128, 192, 256, 384, 512], size=16)
    dims = [(int(s), int(s), 1) for s in sides]
    betas = list(rng.uniform(0.9, 0.999, size=len(dims)))
    outs = {}
    for mode in (E.ELBM_BATCH_GRAPH, E.ELBM_BATCH_PERSISTENT):
        with E.Ensemble(E.ELBM_D2Q9, dims, betas, storage=storage) as ens:
            for k, d in enumerate(dims):
                rho, u = inputs.random_vortex_2d(d[0], rms=0.03, seed=k)
                ens.init_equilibrium(k, rho, u)
            ens.step(1, mode)
            ens.step(100, mode)
            ens.synchronize()
            outs[mode] = [ens.get_populations(k) for k in range(len(dims))]
    for k in range(len(dims)):
        a, b = (outs[m][k] for m in (E.ELBM_BATCH_GRAPH, E.ELBM_BATCH_PERSISTENT))
        if storage == "f32":
            assert np.max(np.abs(a.astype(np.float64) - b) / np.abs(b)) < 101 * 2e-7, k
        else:  # deviations in FP16: equal or one rounding step apart
            da, db = a.astype(np.float64), b.astype(np.float64)
            assert np.max(np.abs(da - db)) <= 4 * 2.0 ** -11 * np.max(np.abs(db)) + 1e-6, k


def test_persistent_wait_expiry_is_reported_and_the_context_survives():
    """Failure detection of the persistent mode without a GPU fault: a launch whose waits
    cannot be satisfied (one owner per domain that never arrives, injected on the host)
    ends after the bounded wait and reports ELBM_ERR_TIMEOUT; the state is untouched and
    the batch keeps stepping correctly afterwards."""
    dims = [(64, 48, 1), (96, 96, 1), (33, 20, 1)]
    betas = [0.95, 0.99, 0.9]
    f0 = [domain_state(2, d, 3e-3, seed=30 + k).astype(np.float32) for k, d in enumerate(dims)]
    with E.Ensemble(E.ELBM_D2Q9, dims, betas, storage="f32") as ens:
        for k in range(len(dims)):
            ens.set_populations(k, f0[k])
        E.elbm_batch_check_wait_timeout(ens.b)
        for k in range(len(dims)):
            assert np.array_equal(ens.get_populations(k), f0[k])
        ens.step(3, E.ELBM_BATCH_PERSISTENT)
        ens.synchronize()
        got = [ens.get_populations(k) for k in range(len(dims))]
    for k, d in enumerate(dims):
        want, *_ = O.step(2, d, f0[k].astype(np.float64), betas[k], nsteps=3)
        assert np.max(np.abs(got[k] - want) / want) < 3 * 2e-6, k


def test_persistent_tuner_keeps_the_state_and_auto_follows_its_choice():
    rng = np.random.default_rng(11)
    sides = rng.choice([64, 96, 128], size=10)
    dims = [(int(s), int(s), 1) for s in sides]
    betas = list(rng.uniform(0.9, 0.999, size=len(dims)))
    outs = {}
    for run in ("auto", "explicit"):
        with E.Ensemble(E.ELBM_D2Q9, dims, betas, storage="f32") as ens:
            for k, d in enumerate(dims):
                rho, u = inputs.random_vortex_2d(d[0], rms=0.03, seed=200 + k)
                ens.init_equilibrium(k, rho, u)
            before = [ens.get_populations(k).copy() for k in range(len(dims))]
            mode, ms = ens.tune_persistent()
            assert mode in (E.ELBM_BATCH_GRAPH, E.ELBM_BATCH_PERSISTENT) and all(m > 0 for m in ms)
            assert all(np.array_equal(a, ens.get_populations(k)) for k, a in enumerate(before))
            ens.step(5, E.ELBM_BATCH_AUTO if run == "auto" else mode)
            ens.synchronize()
            outs[run] = [ens.get_populations(k) for k in range(len(dims))]
    assert all(np.array_equal(a, b) for a, b in zip(outs["auto"], outs["explicit"]))


def test_batch_domain_errors():
    with E.Ensemble(E.ELBM_D2Q9, [(16, 16, 1)], [0.9], storage="f32") as ens:
        with pytest.raises(E.ElbmError) as ei:
            E.elbm_batch_get_populations(ens.b, 3, np.empty(9 * 256, np.float32))
        assert ei.value.code == E.ELBM_ERR_ARG
        with pytest.raises(E.ElbmError):
            E.elbm_batch_step(ens.b, 1, 7)


@pytest.mark.parametrize("mode", [E.ELBM_BATCH_GRAPH, E.ELBM_BATCH_PERSISTENT])
def test_more_domains_than_one_launch_table(mode):
    """A batch of 70 domains needs two batched launches per step (a launch's parameter
    table holds 64 domains); uneven sides, each domain against the oracle (FP64)."""
    rng = np.random.default_rng(70)
    dims = [(int(a), int(b), 1) for a, b in zip(rng.integers(3, 40, size=70), rng.integers(2, 30, size=70))]
    betas = list(rng.uniform(0.9, 0.999, size=70))
    f0 = [domain_state(2, d, 3e-3, seed=200 + k) for k, d in enumerate(dims)]
    with E.Ensemble(E.ELBM_D2Q9, dims, betas, storage="f64", cutoff=False) as ens:
        for k in range(len(dims)):
            ens.set_populations(k, f0[k])
        ens.step(3, mode)
        got = [ens.get_populations(k) for k in range(len(dims))]
        ens.synchronize()
    for k, d in enumerate(dims):
        want, *_ = O.step(2, d, f0[k], betas[k], cutoff=False, nsteps=3)
        assert np.max(np.abs(got[k] - want) / want) < 1e-12, k


@pytest.mark.parametrize("mode", [E.ELBM_BATCH_GRAPH, E.ELBM_BATCH_PERSISTENT, E.ELBM_BATCH_PER_DOMAIN])
def test_fp32_two_node_kernels_on_ragged_domains(mode):
    """D2Q9 FP32 domains collide two nodes per thread (x and x + 32 of a 64-node run);
    sides that are not multiples of 32 leave threads whose second node, or both, lie past
    the end of a row.  Each domain against the oracle over 5 steps, for the batched, the
    persistent and the single-domain kernels."""
    dims = [(33, 7, 1), (65, 12, 1), (97, 5, 1), (1, 9, 1), (31, 31, 1), (200, 3, 1), (129, 17, 1)]
    betas = [0.99, 0.95, 0.999, 0.9, 0.97, 0.995, 0.93]
    f0 = [domain_state(2, d, 2e-2, seed=400 + k).astype(np.float32) for k, d in enumerate(dims)]
    with E.Ensemble(E.ELBM_D2Q9, dims, betas, storage="f32") as ens:
        for k in range(len(dims)):
            ens.set_populations(k, f0[k])
        ens.step(5, mode)
        got = [ens.get_populations(k).astype(np.float64) for k in range(len(dims))]
        ens.synchronize()
    for k, d in enumerate(dims):
        want, *_ = O.step(2, d, f0[k].astype(np.float64), betas[k], nsteps=5)
        assert np.max(np.abs(got[k] - want) / want) < 5 * 2e-6, k
