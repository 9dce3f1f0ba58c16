"""Pins of the oracle's adjoint (the checker of the hand-written backward kernel).

The oracle takes each node's Jacobian-transpose product by central differences of its
own collision and sends it back along the inverse of pull streaming.  Pinned here by
facts that do not depend on how it is computed: the collision conserves mass and
momentum, so the all-ones vector and each velocity component c_a are left eigenvectors
of its Jacobian with eigenvalue 1 (J^T 1 = 1, J^T c_a = c_a); the transpose identity
<g, J v> = <J^T g, v> against an independent directional difference, for one node and
for a whole periodic step (which pins the push direction of the streaming adjoint); and
the kinetic-energy gradient against finite differences.
"""
import numpy as np
import pytest

import oracle as O


def state(rng, D, eps):
    u = rng.uniform(-0.08, 0.08, D)
    f = O.equilibrium(D, 1.0, u) * (1 + eps * (2 * rng.random(3 ** D) - 1))
    return f


@pytest.mark.parametrize("D", [2, 3])
@pytest.mark.parametrize("mode", [O.MODE_HIGHER, O.MODE_LOWER, O.MODE_LBGK])
def test_collision_adjoint_conserved_directions(D, mode):
    rng = np.random.default_rng(7 + D + 3 * mode)
    c, _ = O.lattice(D)
    for _ in range(20):
        f = state(rng, D, 10 ** rng.uniform(-2.5, -1.2))
        one = O.collide_vjp(D, f, np.ones(3 ** D), 0.97, mode=mode)
        assert np.max(np.abs(one - 1.0)) < 1e-7  # central differences, eps = 1e-5
        for a in range(D):
            ca = c[:, a].astype(float)
            assert np.max(np.abs(O.collide_vjp(D, f, ca, 0.97, mode=mode) - ca)) < 1e-7


def _collide(D, f, beta, mode):
    rho, u = O.moments(D, f)
    feq = O.equilibrium(D, rho, u)
    a = O.alpha(f, feq, beta, cutoff=False, mode=mode).alpha
    return O.relax(f, feq, a, beta)


@pytest.mark.parametrize("D", [2, 3])
def test_collision_adjoint_transpose_identity(D):
    rng = np.random.default_rng(17 + D)
    for _ in range(20):
        f = state(rng, D, 10 ** rng.uniform(-2.5, -1.2))
        g = rng.standard_normal(3 ** D)
        v = rng.standard_normal(3 ** D) * f
        h = 1e-6
        Jv = (_collide(D, f + h * v, 0.99, O.MODE_HIGHER) - _collide(D, f - h * v, 0.99, O.MODE_HIGHER)) / (2 * h)
        lhs = g @ Jv
        rhs = O.collide_vjp(D, f, g, 0.99) @ v
        assert abs(lhs - rhs) <= 1e-7 * (abs(lhs) + np.linalg.norm(g) * np.linalg.norm(v) * 1e-3)


@pytest.mark.parametrize("D,dims", [(2, (9, 7, 1)), (3, (5, 4, 3))])
def test_step_adjoint_transpose_identity(D, dims):
    rng = np.random.default_rng(29 + D)
    N = int(np.prod(dims))
    u = 0.05 * rng.standard_normal((D, N))
    f = O.init_equilibrium(D, 1 + 0.01 * rng.random(N), u) * (1 + 3e-3 * (2 * rng.random((3 ** D, N)) - 1))
    g = rng.standard_normal(f.shape)
    v = rng.standard_normal(f.shape) * f
    h = 1e-6
    fp, *_ = O.step(D, dims, f + h * v, 0.995, cutoff=False)
    fm, *_ = O.step(D, dims, f - h * v, 0.995, cutoff=False)
    lhs = np.sum(g * (fp - fm)) / (2 * h)
    rhs = np.sum(O.step_adjoint(D, dims, f, g, 0.995) * v)
    assert abs(lhs - rhs) <= 1e-7 * np.linalg.norm(g) * np.linalg.norm(v)


def test_kinetic_energy_of_uniform_flows():
    """L = 1/2 sum_n rho_n |u_n|^2 (the rollout loss): N nodes of the equilibrium at rho, u
    give N rho |u|^2 / 2; the loss is blind to a rest state's density."""
    for D in (2, 3):
        u = np.array([0.03, -0.02, 0.01])[:D]
        N = 12
        f = O.init_equilibrium(D, np.full(N, 1.2), np.repeat(u[:, None], N, axis=1))
        L, _ = O.kinetic_energy(D, f, want_grad=False)
        assert abs(L - N * 0.5 * 1.2 * float(u @ u)) < 1e-15 * N
        L0, _ = O.kinetic_energy(D, O.init_equilibrium(D, np.full(N, 1.7), np.zeros((D, N))), want_grad=False)
        assert abs(L0) < 1e-30


def test_kinetic_energy_gradient():
    rng = np.random.default_rng(41)
    D, N = 2, 30
    f = O.init_equilibrium(D, 1 + 0.02 * rng.random(N), 0.05 * rng.standard_normal((D, N)))
    L, g = O.kinetic_energy(D, f)
    v = rng.standard_normal(f.shape) * f
    h = 1e-6
    Lp, _ = O.kinetic_energy(D, f + h * v, want_grad=False)
    Lm, _ = O.kinetic_energy(D, f - h * v, want_grad=False)
    assert abs((Lp - Lm) / (2 * h) - np.sum(g * v)) < 1e-8 * np.linalg.norm(g) * np.linalg.norm(v)


# ---------------------------------------------------------------------------
# Body force (exact-difference term after the collision; not in the paper)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("D", [2, 3])
def test_force_term_moments(D):
    """The term f^eq(rho, u + F/rho) - f^eq(rho, u) leaves the mass and adds exactly F to the
    momentum (both equilibria carry their moments exactly); F = 0 changes nothing."""
    rng = np.random.default_rng(31 + D)
    c, _ = O.lattice(D)
    for _ in range(30):
        f = state(rng, D, 10 ** rng.uniform(-3, -1))
        F = rng.uniform(-1e-3, 1e-3, D)
        g = O.force_node(D, f, F)
        r0, u0 = O.moments(D, f)
        r1, u1 = O.moments(D, g)
        assert abs(r1 - r0) < 1e-15
        assert np.max(np.abs(r1 * u1 - (r0 * u0 + F))) < 1e-15
        assert np.array_equal(O.force_node(D, f, np.zeros(D)), f)


@pytest.mark.parametrize("D,dims", [(2, (6, 5, 1)), (3, (4, 3, 3))])
def test_uniform_flow_accelerates_linearly(D, dims):
    """A uniform equilibrium stays an equilibrium under the forced step (x = 0, so alpha = 2
    relaxes nothing), and u grows by F/rho per step: u(t) = u0 + t F / rho."""
    N = int(np.prod(dims))
    rho = np.full(N, 1.02)
    u0 = np.array([0.01, -0.02, 0.015])[:D]
    F = np.array([2e-4, 1e-4, -3e-4])[:D]
    f = O.init_equilibrium(D, rho, np.repeat(u0[:, None], N, axis=1))
    for t in (1, 7, 25):
        ft, *_ = O.step(D, dims, f, 0.95, nsteps=t, force=F)
        r, u = O.moments_field(D, ft)
        assert np.max(np.abs(r - 1.02)) < 1e-13
        assert np.max(np.abs(u - (u0 + t * F / 1.02)[:, None])) < 1e-13


@pytest.mark.parametrize("D,dims", [(2, (7, 6, 1)), (3, (4, 4, 3))])
def test_forced_step_adjoint_transpose_identity(D, dims):
    """<g, d step / d f . v> against an independent directional difference of the forced
    step, and d<g, step>/dF against differences in F."""
    rng = np.random.default_rng(53 + D)
    N = int(np.prod(dims))
    f = np.stack([state(rng, D, 0.02) for _ in range(N)], axis=1)
    F = rng.uniform(-5e-4, 5e-4, D)
    g = rng.standard_normal(f.shape)
    v = rng.standard_normal(f.shape) * f
    h = 1e-6
    fp, *_ = O.step(D, dims, f + h * v, 0.97, cutoff=False, force=F)
    fm, *_ = O.step(D, dims, f - h * v, 0.97, cutoff=False, force=F)
    lhs = np.sum(g * (fp - fm)) / (2 * h)
    rhs = np.sum(O.step_adjoint(D, dims, f, g, 0.97, force=F) * v)
    assert abs(lhs - rhs) <= 1e-6 * abs(lhs)
    dF = O.step_force_vjp(D, dims, f, g, 0.97, F)
    for a in range(D):
        e = np.zeros(D)
        e[a] = 1e-5
        sp, *_ = O.step(D, dims, f, 0.97, cutoff=False, force=F + e)
        sm, *_ = O.step(D, dims, f, 0.97, cutoff=False, force=F - e)
        assert abs(np.sum(g * (sp - sm)) / 2e-5 - dF[a]) <= 1e-6 * np.abs(dF).max()
