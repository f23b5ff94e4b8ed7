"""Pins of the oracle's reverse mode (CPU).  The paper has no adjoint; what fixes it is the
mathematics of the forward operators, each pinned elsewhere:

* the streaming adjoint is the transpose of the streaming: <S x, y> = <x, S^T y> for any
  x, y (exact up to round-off; multi-cell departures, one-cell meshes, synthetic velocities);
* the collision conserves rho, rho u and rho E for every input, so its Jacobian maps the
  moment covectors to themselves: J^T c_M = c_M, and they carry no mu_inf sensitivity;
* at the rest equilibrium (rho = 1, u = 0, T = 1) the BGK Jacobian is the linearised
  operator (1 - omega) I + omega (dE/dM)(dM/dh), whose equilibrium derivatives at rest
  come from the second-order Hermite term alone (App. A: a^(2) = rho (u u + (T - 1) delta))
  and which the test writes out in closed form;
* <lam, J v> from a directional difference of the forward collision equals <J^T lam, v>
  (catches a transposed Jacobian), and likewise for mu_inf;
* the kinetic-energy seed and the initialisation transpose match directional differences
  of the pinned diagnostics and equilibrium initialisation;
* a three-step chain of oracle adjoints reproduces central differences of the oracle's
  forward run, for an initial-velocity perturbation and for mu_inf.
"""
import numpy as np
import pytest

import oracle as O
from paper_2012_05537_gb300 import inputs as I

GAMMA = 1.4
CV = 1.0 / (GAMMA - 1.0)
GFAC = 2.0 * CV - 3.0


def grid(cells, p, dt=0.05, mu=2e-3):
    return O.Grid(cells=tuple(cells), p=p, dt=dt, mu_inf=mu, gamma=GAMMA)


def noneq(g, seed, amp=0.02):
    rho, u, T = I.smooth_fields(g.N[::-1], seed)
    pop = O.init_fields(g, rho, u, T)
    return pop * (1.0 + amp * I.noise(pop.shape, seed + 1))


def rel(a, b):
    return abs(a - b) / max(abs(a), abs(b), 1e-300)


@pytest.mark.parametrize("cells,p,dt", [((2, 3, 2), 2, 0.05), ((1, 2, 1), 3, 0.4), ((3, 1, 2), 4, 0.9),
                                        ((2, 2, 2), 3, 1.7)])
def test_stream_adjoint_is_the_transpose(cells, p, dt):
    g = grid(cells, p, dt=dt)
    rng = np.random.default_rng(3)
    x = rng.standard_normal((2, 45) + g.N[::-1])
    y = rng.standard_normal(x.shape)
    lhs = float(np.sum(O.stream(g, x) * y))
    rhs = float(np.sum(x * O.stream_adjoint(g, y)))
    assert rel(lhs, rhs) < 1e-12


def test_stream_adjoint_with_synthetic_velocities_is_a_back_translation():
    # a velocity that moves exactly two nodes (one cell at p = 2) per step: S is a cyclic
    # shift, S^T the inverse shift
    g = grid((3, 2, 2), 2, dt=1.0)
    N = g.N
    hx = 2 * np.pi / N[0]
    xi = np.array([[hx * 2, 0.0, 0.0]])
    rng = np.random.default_rng(4)
    y = rng.standard_normal((1, 1) + N[::-1])
    back = O.stream_adjoint(g, y, xi=xi)
    assert np.allclose(back, np.roll(y, -2, axis=-1), atol=1e-13)  # S = roll(+2), S^T = roll(-2)


def moment_covectors(xi):
    """c_M for M = rho, j_x, j_y, j_z, E2 as [5][2][45] (f entries, g entries)."""
    x2 = np.sum(xi * xi, axis=1)
    c = np.zeros((5, 2, 45))
    c[0, 0] = 1.0
    for a in range(3):
        c[1 + a, 0] = xi[:, a]
    c[4, 0] = x2
    c[4, 1] = 1.0
    return c


def test_collide_vjp_maps_moment_covectors_to_themselves():
    g = grid((1, 1, 1), 2)
    h = noneq(g, 21, amp=0.05)
    xi, _ = O.velset()
    for cm in moment_covectors(xi):
        lam = np.broadcast_to(cm.reshape(2, 45, 1, 1, 1), h.shape).copy()
        out, dmu = O.collide_vjp(g, h, lam)
        assert np.max(np.abs(out - lam)) < 1e-8 * np.max(np.abs(lam))
        assert abs(dmu) < 1e-8 * h.shape[-1] ** 3 * np.max(np.abs(lam))


def test_collide_vjp_at_rest_is_the_linearised_bgk_operator():
    g = grid((1, 1, 1), 2, dt=0.05, mu=2e-3)
    xi, w = O.velset()
    one = np.ones(g.N[::-1])
    h = O.init_fields(g, one, np.zeros((3,) + g.N[::-1]), one)
    rng = np.random.default_rng(5)
    lam = rng.standard_normal(h.shape)
    out, dmu = O.collide_vjp(g, h, lam)
    tau = g.mu_inf * O.sutherland(1.0) / g.dt + 0.5
    om = 1.0 / tau
    x2 = np.sum(xi * xi, axis=1)
    lf = lam[0].reshape(45, -1)
    lg = lam[1].reshape(45, -1)
    # (dE/dq)^T lam with q = (rho, u, T) at rest: dE_f/drho = w, dE_f/du = w xi,
    # dE_f/dT = w (|xi|^2 - 3)/2; E_g = (2C_v - D) T E_f
    a_rho = np.einsum("i,in->n", w, lf + GFAC * lg)
    a_u = np.einsum("i,ia,in->an", w, xi, lf + GFAC * lg)
    a_T = np.einsum("i,in->n", w * (x2 - 3) / 2, lf) + np.einsum("i,in->n", GFAC * w * (1 + (x2 - 3) / 2), lg)
    # (dq/dM)^T: rho = M_rho, u = j/rho, T = (E2/rho - |u|^2)/(2 C_v)  at rho = 1, u = 0, T = 1
    v_rho = a_rho - a_T
    v_j = a_u
    v_E = a_T / (2 * CV)
    back_f = v_rho[None, :] + np.einsum("ia,an->in", xi, v_j) + x2[:, None] * v_E[None, :]
    back_g = np.broadcast_to(v_E[None, :], lg.shape)
    want = np.stack([(1 - om) * lf + om * back_f, (1 - om) * lg + om * back_g]).reshape(lam.shape)
    assert np.max(np.abs(out - want)) < 1e-8 * np.max(np.abs(want))
    assert abs(dmu) < 1e-8 * np.abs(lam).sum()


def directional(fun, x, v, eps):
    d1 = (fun(x + eps * v) - fun(x - eps * v)) / (2 * eps)
    d2 = (fun(x + 0.5 * eps * v) - fun(x - 0.5 * eps * v)) / eps
    return (4 * d2 - d1) / 3


def test_collide_vjp_is_the_transpose_of_the_forward_derivative():
    g = grid((2, 1, 1), 2, dt=0.08, mu=3e-3)
    h = noneq(g, 31, amp=0.05)
    rng = np.random.default_rng(6)
    lam = rng.standard_normal(h.shape)
    v = rng.standard_normal(h.shape) * np.abs(h)
    out, dmu = O.collide_vjp(g, h, lam)
    jv = directional(lambda x: O.collide(g, x), h, v, 1e-3)
    assert rel(float(np.sum(lam * jv)), float(np.sum(out * v))) < 1e-8

    def with_mu(mu):
        gm = grid((2, 1, 1), 2, dt=0.08, mu=float(mu))
        return O.collide(gm, h)
    dmu_fd = float(np.sum(lam * directional(with_mu, g.mu_inf, 1.0, 1e-3 * g.mu_inf)))
    assert rel(dmu, dmu_fd) < 1e-7


def test_ek_grad_is_the_derivative_of_the_diagnostic():
    g = grid((2, 1, 2), 3)
    pop = noneq(g, 41)
    U0 = 0.59
    lam = O.ek_grad(g, pop, 1.0, U0)
    assert np.all(lam[1] == 0.0)
    rng = np.random.default_rng(7)
    v = rng.standard_normal(pop.shape) * np.abs(pop)
    fd = directional(lambda x: O.diag(g, x, 1.0, 1600.0, U0)[0], pop, v, 1e-3)
    assert rel(float(np.sum(lam * v)), float(fd)) < 1e-8


@pytest.mark.parametrize("k", [0, 1, 2])
def test_diag_grad_is_the_derivative_of_each_diagnostic(k):
    """d(E_k, eps_s, eps_c)/dpop of the oracle against directional differences of its own
    diagnostics (Sec. III.C definitions) along a random direction, on a mesh of several
    cells per direction (cells share face nodes, so the scatter over neighbouring cells is
    exercised) with a non-equilibrium state."""
    g = grid((3, 2, 2), 3)
    pop = noneq(g, 43)
    U0, Re = 0.59, 1600.0
    wts = [0.0, 0.0, 0.0]
    wts[k] = 1.0
    lam = O.diag_grad(g, pop, 1.0, Re, U0, wts)
    rng = np.random.default_rng(17 + k)
    v = rng.standard_normal(pop.shape) * np.abs(pop)
    fd = directional(lambda x: O.diag(g, x, 1.0, Re, U0)[k], pop, v, 1e-3)
    assert rel(float(np.sum(lam * v)), float(fd)) < 1e-7
    if k == 0:  # the E_k part equals the dedicated E_k gradient
        assert np.allclose(lam, O.ek_grad(g, pop, 1.0, U0), rtol=1e-13, atol=1e-18)
    else:  # the dissipation depends on g only through T
        assert np.any(lam[1] != 0.0)


def test_diag_grad_is_linear_in_the_weights():
    g = grid((2, 2, 1), 2)
    pop = noneq(g, 44)
    parts = [O.diag_grad(g, pop, 1.0, 400.0, 0.7, w) for w in ((1, 0, 0), (0, 1, 0), (0, 0, 1))]
    mix = O.diag_grad(g, pop, 1.0, 400.0, 0.7, (0.5, -2.0, 3.0))
    assert np.allclose(mix, 0.5 * parts[0] - 2.0 * parts[1] + 3.0 * parts[2], rtol=1e-12, atol=1e-15)


def test_init_fields_vjp_is_the_transpose_of_the_initialisation():
    g = grid((2, 1, 1), 3)
    rho, u, T = I.smooth_fields(g.N[::-1], 51)
    rng = np.random.default_rng(8)
    lam = rng.standard_normal((2, 45) + g.N[::-1])
    gr, gu, gT = O.init_fields_vjp(g, rho, u, T, lam)
    vr, vu, vT = (rng.standard_normal(a.shape) for a in (rho, u, T))

    def obj(t):
        return float(np.sum(lam * O.init_fields(g, rho + t * vr, u + t * vu, T + t * vT)))
    fd = directional(obj, 0.0, 1.0, 1e-3)
    got = float(np.sum(gr * vr) + np.sum(gu * vu) + np.sum(gT * vT))
    assert rel(got, fd) < 1e-8


def test_adjoint_chain_reproduces_finite_differences_of_the_forward_run():
    """Three steps of the oracle from equilibrium fields; E_k of the final state.  Reverse
    mode: seed, then (stream transpose . collision VJP) per step, then the initialisation
    transpose.  Checked against central differences of the forward oracle."""
    g = grid((2, 1, 1), 2, dt=0.1, mu=4e-3)
    U0, steps = 0.5, 3
    rho, u, T = I.smooth_fields(g.N[::-1], 61)
    rng = np.random.default_rng(9)
    du = 1e-3 * U0 * rng.standard_normal(u.shape)

    def run(uu, gg):
        s = [O.init_fields(gg, rho, uu, T)]
        for _ in range(steps):
            s.append(O.step(gg, s[-1], 1))
        return s

    states = run(u, g)
    lam = O.ek_grad(g, states[-1], 1.0, U0)
    dmu = 0.0
    for k in range(steps, 0, -1):
        lam, d = O.step_adjoint(g, states[k - 1], lam)
        dmu += d
    _, gu, _ = O.init_fields_vjp(g, rho, u, T, lam)
    grad_eps = float(np.sum(gu * du))

    def ek(eps=0.0, mu=g.mu_inf):
        gg = grid((2, 1, 1), 2, dt=0.1, mu=mu)
        return O.diag(gg, run(u + eps * du, gg)[-1], 1.0, 1600.0, U0)[0]
    fd_eps = directional(lambda e: ek(eps=e), 0.0, 1.0, 1.0)
    fd_mu = directional(lambda m: ek(mu=m), g.mu_inf, 1.0, 1e-2 * g.mu_inf)
    assert rel(grad_eps, fd_eps) < 1e-6
    assert rel(dmu, fd_mu) < 1e-6


def test_adjoint_chain_of_the_dissipation_reproduces_finite_differences():
    """The same chain seeded with the dissipation eps_s + eps_c of the final state."""
    g = grid((2, 2, 1), 2, dt=0.1, mu=4e-3)
    U0, Re, steps = 0.5, 1600.0, 3
    rho, u, T = I.smooth_fields(g.N[::-1], 62)
    rng = np.random.default_rng(10)
    du = 1e-3 * U0 * rng.standard_normal(u.shape)

    def run(uu, gg):
        s = [O.init_fields(gg, rho, uu, T)]
        for _ in range(steps):
            s.append(O.step(gg, s[-1], 1))
        return s

    states = run(u, g)
    lam = O.diag_grad(g, states[-1], 1.0, Re, U0, (0.0, 1.0, 1.0))
    dmu = 0.0
    for k in range(steps, 0, -1):
        lam, d = O.step_adjoint(g, states[k - 1], lam)
        dmu += d
    _, gu, _ = O.init_fields_vjp(g, rho, u, T, lam)
    grad_eps = float(np.sum(gu * du))

    def eps(e=0.0, mu=g.mu_inf):
        gg = grid((2, 2, 1), 2, dt=0.1, mu=mu)
        d = O.diag(gg, run(u + e * du, gg)[-1], 1.0, Re, U0)
        return d[1] + d[2]
    fd_eps = directional(lambda e: eps(e=e), 0.0, 1.0, 1.0)
    fd_mu = directional(lambda m: eps(mu=m), g.mu_inf, 1.0, 1e-2 * g.mu_inf)
    assert rel(grad_eps, fd_eps) < 1e-6
    assert rel(dmu, fd_mu) < 1e-6
