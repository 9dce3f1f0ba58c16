"""The hand-written adjoint kernels against the oracle's adjoint and against finite
differences of the forward step.

* one backward step (elbm_adjoint_step) against the oracle's reverse step, whose node
  Jacobian-transpose products come from central differences of its own collision:
  FP64 to the differences' accuracy (~1e-8), FP32 to 6e-7 (twice the largest relative
  error measured on these states, 2.8e-7, which is the FP32 rounding of the VJP: the
  FP64 path on the same FP32-rounded inputs agrees with the oracle to 4e-9);
* whole rollouts: <dL/du0, v> from the autograd wrapper (with sqrt(T) checkpointing)
  against central differences of L along v computed with the FP64 forward, and the
  checkpointed gradient against the unsegmented one;
* the kinetic-energy gradient and the equilibrium VJP against the oracle.
The cutoff is off throughout (the shortcut alpha = 2 is a branch; gradients are taken
on the smooth closed-form path).
"""
import numpy as np
import pytest

import oracle as O
from paper_2203_12946_gb300 import elbm as E
from paper_2203_12946_gb300 import inputs

pytestmark = pytest.mark.gpu
LAT = {2: E.ELBM_D2Q9, 3: E.ELBM_D3Q27}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    E.load()


def noisy(D, dims, eps, seed):
    X, Y, Z = inputs.grid(dims)
    L = dims[0]
    rho, u = (inputs.taylor_green_2d(X, Y, L, u0=0.05) if D == 2
              else inputs.taylor_green_3d(X, Y, Z, L, u0=0.05))
    return O.init_equilibrium(D, rho, u) * inputs.population_noise(3 ** D, X.size, eps, seed=seed)


@pytest.mark.parametrize("D,dims", [(2, (23, 17, 1)), (3, (9, 7, 6))])
@pytest.mark.parametrize("mode", [E.ELBM_ALPHA_HIGHER, E.ELBM_ALPHA_LOWER, E.ELBM_ALPHA_LBGK])
@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_adjoint_step_matches_oracle(D, dims, mode, storage):
    import torch

    om = {E.ELBM_ALPHA_HIGHER: O.MODE_HIGHER, E.ELBM_ALPHA_LOWER: O.MODE_LOWER, E.ELBM_ALPHA_LBGK: O.MODE_LBGK}[mode]
    beta = 0.99
    f = noisy(D, dims, 5e-3, seed=11)
    if storage == "f32":
        f = f.astype(np.float32).astype(np.float64)
    rng = np.random.default_rng(5)
    g = rng.standard_normal(f.shape)
    want = O.step_adjoint(D, dims, f, g, beta, cutoff=False, mode=om)
    with E.Simulation(LAT[D], dims, beta, storage=storage, cutoff=False, alpha_mode=mode) as sim:
        sim.set_populations(f)
        ft = sim.state_copy()
        gt = torch.from_numpy(g.astype(np.float64 if storage == "f64" else np.float32)).cuda()
        got = sim.adjoint_step(ft, gt).double().cpu().numpy()
    err = np.linalg.norm(got - want) / np.linalg.norm(want)
    assert err < (1e-7 if storage == "f64" else 6e-7), err


def test_adjoint_through_clamp_matches_oracle():
    """Far from equilibrium many nodes are clamped (alpha from alpha_max)."""
    import torch

    D, dims, beta = 2, (24, 18, 1), 0.99
    f = noisy(D, dims, 0.9, seed=31)
    _, _, br, _ = O.step(D, dims, f, beta, cutoff=False, want_alpha=True)
    assert np.sum(br == O.BRANCH_CLAMPED) > 10
    g = np.random.default_rng(6).standard_normal(f.shape)
    want = O.step_adjoint(D, dims, f, g, beta, cutoff=False)
    with E.Simulation(E.ELBM_D2Q9, dims, beta, storage="f64", cutoff=False) as sim:
        sim.set_populations(f)
        got = sim.adjoint_step(sim.state_copy(), torch.from_numpy(g).cuda()).cpu().numpy()
    assert np.linalg.norm(got - want) / np.linalg.norm(want) < 1e-6


def test_kinetic_energy_and_equilibrium_vjp():
    import torch

    D, dims = 2, (20, 12, 1)
    rng = np.random.default_rng(9)
    N = 240
    rho = 1 + 0.02 * rng.random(N)
    u = 0.05 * rng.standard_normal((2, N))
    f = O.init_equilibrium(D, rho, u)
    L_o, g_o = O.kinetic_energy(D, f)
    with E.Simulation(E.ELBM_D2Q9, dims, 0.9, storage="f64") as sim:
        sim.set_populations(f)
        L, g = sim.kinetic_energy(with_grad=True)
        assert abs(L - L_o) < 1e-14 * L_o
        assert np.max(np.abs(g.cpu().numpy() - g_o)) < 1e-15
        gf = torch.from_numpy(rng.standard_normal(f.shape)).cuda()
        dr, du = sim.equilibrium_vjp(torch.from_numpy(rho).cuda(), torch.from_numpy(u).cuda(), gf)
        dr, du = dr.cpu().numpy(), du.cpu().numpy()
    # against central differences of the oracle's equilibrium
    gh = gf.cpu().numpy()
    h = 1e-6
    for n in (0, 7, 100):
        for a in range(2):
            up, um = u.copy(), u.copy()
            up[a, n] += h
            um[a, n] -= h
            fp = O.equilibrium(2, rho[n], up[:, n])
            fm = O.equilibrium(2, rho[n], um[:, n])
            assert abs(gh[:, n] @ (fp - fm) / (2 * h) - du[a, n]) < 1e-8
        fp = O.equilibrium(2, rho[n] + h, u[:, n])
        fm = O.equilibrium(2, rho[n] - h, u[:, n])
        assert abs(gh[:, n] @ (fp - fm) / (2 * h) - dr[n]) < 1e-8


def _rollout_fd(D, dims, rho0, u0, v, beta, nsteps, h):
    """Central difference of L(u0) along v with the FP64 GPU forward."""
    Ls = []
    for sgn in (1, -1):
        with E.Simulation(LAT[D], dims, beta, storage="f64", cutoff=False) as sim:
            sim.init_equilibrium(rho0, u0 + sgn * h * v)
            sim.step(nsteps)
            Ls.append(sim.kinetic_energy())
    return (Ls[0] - Ls[1]) / (2 * h)


@pytest.mark.parametrize("storage,tol", [("f64", 1e-6), ("f32", 1e-4)])
def test_rollout_gradient_against_finite_differences(storage, tol):
    import torch

    from paper_2203_12946_gb300.adjoint import kinetic_energy_rollout

    D, L, beta, T = 2, 32, 0.95, 40
    dims = (L, L, 1)
    rho0, u0 = inputs.random_vortex_2d(L, rms=0.02, seed=3)
    rng = np.random.default_rng(12)
    with E.Simulation(E.ELBM_D2Q9, dims, beta, storage=storage, cutoff=False) as sim:
        ut = torch.from_numpy(u0).cuda().requires_grad_(True)
        loss = kinetic_energy_rollout(ut, sim, T, rho0=torch.from_numpy(rho0).cuda())
        loss.backward()
        grad = ut.grad.cpu().numpy()
        # the same gradient without segmenting (one checkpoint)
        ut2 = torch.from_numpy(u0).cuda().requires_grad_(True)
        kinetic_energy_rollout(ut2, sim, T, rho0=torch.from_numpy(rho0).cuda(), every=T).backward()
        assert np.max(np.abs(ut2.grad.cpu().numpy() - grad)) <= 1e-12 * np.max(np.abs(grad))
    for k in range(3):
        v = rng.standard_normal(u0.shape) * 0.01
        fd = _rollout_fd(D, dims, rho0, u0, v, beta, T, 1e-4)
        ad = float(np.sum(grad * v))
        assert abs(ad - fd) <= tol * abs(fd), (ad, fd)


def test_rollout_gradient_against_oracle_adjoint():
    """FP64: the GPU gradient dL/df^0 equals the oracle's reverse sweep (oracle forward
    states, oracle reverse steps) on a small D3Q27 box."""
    import torch

    D, dims, beta, T = 3, (6, 5, 4), 0.97, 6
    f0 = noisy(D, dims, 4e-3, seed=21)
    states = [f0]
    for _ in range(T):
        nxt, *_ = O.step(D, dims, states[-1], beta, cutoff=False)
        states.append(nxt)
    _, g = O.kinetic_energy(D, states[-1])
    for t in range(T - 1, -1, -1):
        g = O.step_adjoint(D, dims, states[t], g, beta, cutoff=False)
    with E.Simulation(E.ELBM_D3Q27, dims, beta, storage="f64", cutoff=False) as sim:
        sim.set_populations(f0)
        st = [sim.state_copy()]
        for _ in range(T):
            sim.step(1)
            st.append(sim.state_copy())
        _, gg = sim.kinetic_energy(with_grad=True)
        for t in range(T - 1, -1, -1):
            gg = sim.adjoint_step(st[t], gg)
        got = gg.cpu().numpy()
    assert np.linalg.norm(got - g) / np.linalg.norm(g) < 1e-7


# ---------------------------------------------------------------------------
# Uniform body force (exact-difference term after the collision; not in the paper)
# ---------------------------------------------------------------------------

FORCE = {2: np.array([2e-4, -1e-4]), 3: np.array([2e-4, -1e-4, 3e-4])}


@pytest.mark.parametrize("D,dims", [(2, (29, 17, 1)), (3, (11, 9, 7))])
@pytest.mark.parametrize("storage,tol", [("f64", 1e-12), ("f32", 4e-6)])
def test_forced_step_matches_oracle(D, dims, storage, tol):
    beta = 0.99
    f0 = noisy(D, dims, 3e-3, seed=61)
    if storage == "f32":
        f0 = f0.astype(np.float32).astype(np.float64)
    want, *_ = O.step(D, dims, f0, beta, cutoff=False, nsteps=3, force=FORCE[D])
    with E.Simulation(LAT[D], dims, beta, storage=storage, cutoff=False) as sim:
        sim.set_populations(f0)
        sim.set_force(FORCE[D])
        sim.step(3)
        got = sim.get_populations().astype(np.float64)
    assert np.max(np.abs(got - want) / want) < tol


@pytest.mark.parametrize("storage,tol", [("f64", 1e-13), ("f32", 2e-7)])
def test_uniform_flow_accelerates_on_gpu(storage, tol):
    """u(t) = u0 + t F / rho for a uniform equilibrium under the force (exact in the method)."""
    D, dims = 3, (8, 6, 5)
    N = int(np.prod(dims))
    u0 = np.array([0.01, -0.02, 0.015])
    with E.Simulation(E.ELBM_D3Q27, dims, 0.95, storage=storage) as sim:
        sim.init_equilibrium(np.full(N, 1.02), np.repeat(u0[:, None], N, axis=1))
        sim.set_force(FORCE[3])
        sim.step(40)
        r, u = [t.cpu().numpy() for t in sim.moments()]
    assert np.max(np.abs(u - (u0 + 40 * FORCE[3] / 1.02)[:, None])) < tol
    assert np.max(np.abs(r - 1.02)) < tol


@pytest.mark.parametrize("D,dims", [(2, (13, 11, 1)), (3, (6, 5, 4))])
def test_forced_adjoint_step_matches_oracle(D, dims):
    import torch

    beta = 0.99
    f = noisy(D, dims, 5e-3, seed=67)
    g = np.random.default_rng(68).standard_normal(f.shape)
    want = O.step_adjoint(D, dims, f, g, beta, cutoff=False, force=FORCE[D])
    want_F = O.step_force_vjp(D, dims, f, g, beta, FORCE[D])
    with E.Simulation(LAT[D], dims, beta, storage="f64", cutoff=False) as sim:
        sim.set_populations(f)
        sim.set_force(FORCE[D])
        dF = torch.zeros(D, dtype=torch.float64, device="cuda")
        got = sim.adjoint_step(sim.state_copy(), torch.from_numpy(g).cuda(), dforce=dF).cpu().numpy()
        dF = dF.cpu().numpy()
    assert np.linalg.norm(got - want) / np.linalg.norm(want) < 1e-7
    assert np.max(np.abs(dF - want_F)) < 1e-6 * np.max(np.abs(want_F))


@pytest.mark.parametrize("storage,tol,mean", [("f64", 1e-6, 0.0), ("f32", 1e-4, 0.01)])
def test_rollout_force_gradient_against_finite_differences(storage, tol, mean):
    """dL/dF from the checkpointed reverse sweep against central differences of the FP64
    forward in each component of F, at F = 0 and at a nonzero F.  For a zero-mean vortex
    dL/dF is close to the time-integrated total momentum, a sum over nodes that cancels to
    ~1e-5 of its terms, below what FP32 node sums resolve; the FP32 case adds a mean flow."""
    import torch

    from paper_2203_12946_gb300.adjoint import kinetic_energy_rollout

    L, beta, T = 32, 0.95, 40
    dims = (L, L, 1)
    rho0, u0 = inputs.random_vortex_2d(L, rms=0.02, seed=5)
    u0 = u0 + np.array([mean, -0.5 * mean])[:, None]
    for F in (np.zeros(2), np.array([1e-4, -2e-4])):
        with E.Simulation(E.ELBM_D2Q9, dims, beta, storage=storage, cutoff=False) as sim:
            ut = torch.from_numpy(u0).cuda().requires_grad_(True)
            Ft = torch.from_numpy(F.copy()).requires_grad_(True)
            kinetic_energy_rollout(ut, sim, T, rho0=torch.from_numpy(rho0).cuda(), force=Ft).backward()
            dF = Ft.grad.numpy()
        for a in range(2):
            # L is far from linear in F (its curvature ~ N T^2), so the central differences
            # are Richardson-extrapolated from steps h and h/2 (error O(h^4)).
            fds = []
            for h in (2e-6, 1e-6):
                Ls = []
                for sgn in (1, -1):
                    Fp = F.copy()
                    Fp[a] += sgn * h
                    with E.Simulation(E.ELBM_D2Q9, dims, beta, storage="f64", cutoff=False) as sim:
                        sim.init_equilibrium(rho0, u0)
                        sim.set_force(Fp)
                        sim.step(T)
                        Ls.append(sim.kinetic_energy())
                fds.append((Ls[0] - Ls[1]) / (2 * h))
            fd = (4 * fds[1] - fds[0]) / 3
            assert abs(dF[a] - fd) <= tol * abs(fd), (a, dF[a], fd, fds)


def test_config5_rollout_gradient_at_full_size():
    """The adjoint configuration at its own size: D2Q9 256^2 periodic, beta = 0.9, 2000 steps
    in FP32 with sqrt(T) checkpoints and recompute, u0 from the random-phase vortex field
    (rms 0.02), L = kinetic energy of the final state.  <dL/du0, v> along 4 seeded
    directions agrees with central differences (h = 1e-4) of the FP64 forward to 1e-4."""
    import torch

    from paper_2203_12946_gb300.adjoint import kinetic_energy_rollout

    L, beta, T = 256, 0.9, 2000
    dims = (L, L, 1)
    rho0, u0 = inputs.random_vortex_2d(L, rms=0.02, seed=inputs.DEFAULT_SEED)
    with E.Simulation(E.ELBM_D2Q9, dims, beta, storage="f32", cutoff=False) as sim:
        ut = torch.from_numpy(u0).cuda().requires_grad_(True)
        kinetic_energy_rollout(ut, sim, T, rho0=torch.from_numpy(rho0).cuda()).backward()
        grad = ut.grad.cpu().numpy()
    rng = np.random.default_rng(inputs.DEFAULT_SEED)
    for _ in range(4):
        v = rng.standard_normal(u0.shape) * 0.01
        fd = _rollout_fd(2, dims, rho0, u0, v, beta, T, 1e-4)
        ad = float(np.sum(grad * v))
        assert abs(ad - fd) <= 1e-4 * abs(fd), (ad, fd)
