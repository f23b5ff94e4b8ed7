"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these tests compares the oracle with itself: each expected value is a closed
form (Gaussian moments, Hermite orthogonality, polynomial exactness, translation,
Chapman-Enskog decay rates, the Taylor-Green integrals) or a constant printed in the
paper (tests/golden/paper_constants.txt).
"""
import itertools
import math
import os

import numpy as np
import pytest

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_constants.txt")


def golden():
    out = {}
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        name, val = line.split()[:2]
        out[name] = float(val)
    return out


def gauss_moment(e):
    """E[x^a y^b z^c] for the unit-variance 3D Gaussian: product of (k-1)!! for even k."""
    if any(k % 2 for k in e):
        return 0.0
    return float(np.prod([math.prod(range(k - 1, 0, -2)) if k > 0 else 1 for k in e]))


# ---------------------------------------------------------------- P1 quadrature
def test_p1_velset_degree_nine_exact_and_not_ten():
    """Sec. II.B: the 45-point set must integrate the Gaussian weight to degree nine."""
    xi, w = O.velset()
    g = golden()
    assert len(w) == int(g["velocity_count"])
    assert np.all(w > 0)
    assert abs(w.sum() - 1.0) < 1e-15
    assert len({tuple(np.round(x, 12)) for x in xi}) == 45
    worst = 0.0
    for deg in range(int(g["cubature_degree"]) + 1):
        for e in itertools.product(range(deg + 1), repeat=3):
            if sum(e) != deg:
                continue
            val = np.sum(w * np.prod(xi ** np.array(e), axis=1))
            worst = max(worst, abs(val - gauss_moment(e)) / max(1.0, gauss_moment(e)))
    assert worst < 1e-13
    deg10 = max(abs(np.sum(w * np.prod(xi ** np.array(e), axis=1)) - gauss_moment(e))
                for e in itertools.product(range(11), repeat=3) if sum(e) == 10)
    assert deg10 > 1.0
    assert abs(np.max(np.linalg.norm(xi, axis=1)) - math.sqrt(15.0)) < 1e-14


def test_p1_velset_shells_and_symmetry():
    """Fig. 2: shells at radii 0, sqrt(3), 3, sqrt(15); the set is closed under xi -> -xi."""
    xi, w = O.velset()
    r = np.linalg.norm(xi, axis=1)
    assert np.allclose(sorted(set(np.round(r, 12))), [0.0, math.sqrt(3), 3.0, math.sqrt(15)])
    for x in xi:
        assert np.min(np.linalg.norm(xi + x, axis=1)) < 1e-14


# ---------------------------------------------------------------- P2 equilibrium moments
def _sym_du(u):
    d = np.eye(3)
    return (np.einsum("ab,c->abc", d, u) + np.einsum("ac,b->abc", d, u)
            + np.einsum("bc,a->abc", d, u))


def _gauss4(u, T):
    """Fourth raw moment of a Maxwellian with mean u and temperature T (closed form)."""
    d = np.eye(3)
    uu = np.einsum("a,b->ab", u, u)
    s6 = sum(np.einsum(spec, d, uu) for spec in
             ["ab,cd->abcd", "ac,bd->abcd", "ad,bc->abcd", "bc,ad->abcd", "bd,ac->abcd",
              "cd,ab->abcd"])
    s3 = (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
          + np.einsum("ad,bc->abcd", d, d))
    return np.einsum("a,b,c,d->abcd", u, u, u, u) + T * s6 + T * T * s3


@pytest.mark.parametrize("seed", range(6))
def test_p2_equilibrium_moments_are_maxwellian(seed):
    """App. A: the fourth-order equilibrium carries the Maxwellian moments up to order 4
    (the quadrature is exact to degree 9 >= 4 + 4)."""
    rng = np.random.default_rng(seed)
    xi, w = O.velset()
    rho = rng.uniform(0.3, 3.0)
    u = rng.uniform(-1.5, 1.5, 3)
    T = rng.uniform(0.5, 2.0)
    f = O.feq(rho, u, T)
    tol = 1e-13 * max(1.0, np.abs(f).sum())
    assert abs(f.sum() - rho) < tol
    assert np.allclose(np.einsum("i,ia->a", f, xi), rho * u, atol=tol, rtol=0)
    M2 = np.einsum("i,ia,ib->ab", f, xi, xi)
    assert np.allclose(M2, rho * (np.outer(u, u) + T * np.eye(3)), atol=tol * 10, rtol=0)
    M3 = np.einsum("i,ia,ib,ic->abc", f, xi, xi, xi)
    assert np.allclose(M3, rho * (np.einsum("a,b,c->abc", u, u, u) + T * _sym_du(u)),
                       atol=tol * 50, rtol=0)
    M4 = np.einsum("i,ia,ib,ic,id->abcd", f, xi, xi, xi, xi)
    assert np.allclose(M4, rho * _gauss4(u, T), atol=tol * 200, rtol=0)


def gauss_product_set(n: int = 5):
    """The Gauss-product alternative of Sec. II.B: the tensor product of the n-point
    Gauss-Hermite rule for the unit-variance Gaussian (nodes and weights from numpy's
    probabilists' Hermite routine), n^3 velocities; n = 5 is the 125-point set."""
    x, wx = np.polynomial.hermite_e.hermegauss(n)
    wx = wx / wx.sum()
    xi = np.array(list(itertools.product(x, x, x)))
    w = np.array([a * b * c for a, b, c in itertools.product(wx, wx, wx)])
    return xi, w


def test_d3q125_gauss_product_set_is_degree_nine_per_direction():
    """Sec. II.B: the 125-point product rule integrates every monomial whose exponents are
    each at most nine, and fails on x^10 (a textbook rule, independent of the 45-point set)."""
    xi, w = gauss_product_set()
    assert len(w) == 125 and np.all(w > 0) and abs(w.sum() - 1.0) < 1e-15
    worst = 0.0
    for e in itertools.product(range(10), repeat=3):
        terms = w * np.prod(xi ** np.array(e), axis=1)
        worst = max(worst, abs(terms.sum() - gauss_moment(e)) / np.abs(terms).sum())
    assert worst < 1e-13
    assert abs(np.sum(w * xi[:, 0] ** 10) - gauss_moment((10, 0, 0))) > 1.0


@pytest.mark.parametrize("seed", range(4))
def test_d3q45_and_d3q125_give_the_same_equilibrium_moments(seed):
    """Any set exact to degree nine yields the same moments of the fourth-order equilibrium
    up to order five (a quartic times a monomial of degree five stays within degree nine),
    so the 45-point set and the 125-point product set, built independently, must agree on
    all of them, including the fifth-order moments that no closed form above checks."""
    rng = np.random.default_rng(100 + seed)
    rho = rng.uniform(0.3, 3.0)
    u = rng.uniform(-1.5, 1.5, 3)
    T = rng.uniform(0.5, 2.0)
    xi45, _ = O.velset()
    xi125, w125 = gauss_product_set()
    f45 = O.feq(rho, u, T)
    f125 = O.feq(rho, u, T, xi125, w125)
    assert not np.allclose(np.sort(f45)[:5], np.sort(f125)[:5])  # different sets, same moments
    worst = 0.0
    for deg in range(6):
        for e in itertools.product(range(deg + 1), repeat=3):
            if sum(e) != deg:
                continue
            m45 = np.sum(f45 * np.prod(xi45 ** np.array(e), axis=1))
            m125 = np.sum(f125 * np.prod(xi125 ** np.array(e), axis=1))
            scale = np.sum(np.abs(f125) * np.prod(np.abs(xi125) ** np.array(e), axis=1))
            worst = max(worst, abs(m45 - m125) / scale)
    assert worst < 1e-13


def test_p2_energy_moment_of_both_populations():
    """Eq. (moments) with g^eq = (2C_v - D) T f^eq: sum(f|xi|^2 + g) = rho|u|^2 + 2 C_v rho T."""
    xi, w = O.velset()
    g = O.Grid(cells=(1, 1, 1), p=2, dt=0.1, mu_inf=0.01)
    rng = np.random.default_rng(7)
    shp = g.N[::-1]
    rho = rng.uniform(0.5, 2.0, shp)
    u = rng.uniform(-1, 1, (3,) + shp)
    T = rng.uniform(0.6, 1.8, shp)
    pop = O.init_fields(g, rho, u, T)
    r2, u2, T2 = O.moments(g, pop)
    assert np.allclose(r2, rho, rtol=1e-13, atol=0)
    assert np.allclose(u2, u, rtol=0, atol=1e-13)
    assert np.allclose(T2, T, rtol=1e-13, atol=0)
    Cv = 1 / (1.4 - 1)
    e2 = (np.einsum("iz...,i->z...", pop[0], (xi ** 2).sum(1)) + pop[1].sum(0))
    assert np.allclose(e2, rho * (u ** 2).sum(0) + 2 * Cv * rho * T, rtol=1e-13, atol=0)


def test_p2_hermite_orthogonality_through_equilibrium():
    """App. B tensors are orthogonal under the weights: the Hermite coefficients of f^eq
    recovered by sum_i f_i H^(n)(xi_i) equal the App. A moments a^(n)."""
    xi, w = O.velset()
    rho, u, T = 1.3, np.array([0.4, -0.7, 0.2]), 1.4
    f = O.feq(rho, u, T)
    d = np.eye(3)
    H2 = np.einsum("ia,ib->iab", xi, xi) - d[None]
    a2 = np.einsum("i,iab->ab", f, H2)
    assert np.allclose(a2, rho * (np.outer(u, u) + (T - 1) * d), atol=1e-13)
    H3 = (np.einsum("ia,ib,ic->iabc", xi, xi, xi)
          - (np.einsum("ia,bc->iabc", xi, d) + np.einsum("ib,ac->iabc", xi, d)
             + np.einsum("ic,ab->iabc", xi, d)))
    a3 = np.einsum("i,iabc->abc", f, H3)
    assert np.allclose(a3, rho * (np.einsum("a,b,c->abc", u, u, u) + (T - 1) * _sym_du(u)),
                       atol=1e-13)


# ---------------------------------------------------------------- P3 Fig. 12
def test_p3_fig12_density_stays_one_while_populations_go_negative():
    """Sec. IV.B / Fig. 12: at rho = theta = 1 the 45 equilibria sweep Ma_x in [0, 4];
    their sum stays exactly 1 while individual values turn negative at high Mach."""
    xi, w = O.velset()
    vals = []
    for ma in np.linspace(0.0, 4.0, 41):
        f = O.feq(1.0, [ma, 0.0, 0.0], 1.0)
        assert abs(f.sum() - 1.0) < 1e-12
        vals.append(f)
    vals = np.array(vals)
    assert np.allclose(vals[0], w, rtol=0, atol=1e-16)
    assert np.all(vals[:5] > -1e-15)           # low Mach: all positive
    assert vals[-1].min() < -0.1               # Ma_x = 4: clearly negative members
    assert np.max(np.abs(vals[-1])) > 10 * np.max(np.abs(vals[20]))  # diverging growth


# ---------------------------------------------------------------- P4 collision
def _noneq_state(g, seed, amp=0.05):
    rng = np.random.default_rng(seed)
    shp = g.N[::-1]
    rho = rng.uniform(0.7, 1.4, shp)
    u = rng.uniform(-0.6, 0.6, (3,) + shp)
    T = rng.uniform(0.7, 1.4, shp)
    pop = O.init_fields(g, rho, u, T)
    return pop * (1.0 + amp * rng.standard_normal(pop.shape))


def _conserved(pop, xi):
    rho = pop[0].sum(0)
    mom = np.einsum("i...,ia->a...", pop[0], xi)
    en = np.einsum("i...,i->...", pop[0], (xi ** 2).sum(1)) + pop[1].sum(0)
    return rho, mom, en


@pytest.mark.parametrize("pr", [False, True])
def test_p4_collision_conserves_mass_momentum_energy(pr):
    """App. C: sum f^(0){1, xi} and sum(f|xi|^2 + g) are collision invariants; the
    Prandtl term of App. D adds no mass, momentum or energy."""
    xi, _ = O.velset()
    g = O.Grid(cells=(2, 1, 1), p=3, dt=0.05, mu_inf=0.02, pr_correction=pr)
    pop = _noneq_state(g, 3)
    post = O.collide(g, pop)
    for a, b in zip(_conserved(pop, xi), _conserved(post, xi)):
        assert np.allclose(a, b, rtol=1e-13, atol=1e-13)
    assert np.max(np.abs(post - pop)) > 1e-3  # it did relax something


@pytest.mark.parametrize("pr", [False, True])
def test_p4_equilibrium_is_a_fixed_point(pr):
    g = O.Grid(cells=(1, 1, 1), p=2, dt=0.05, mu_inf=0.02, pr_correction=pr)
    pop = _noneq_state(g, 5, amp=0.0)
    assert np.allclose(O.collide(g, pop), pop, rtol=1e-13, atol=1e-15)


def _tau(g, rho, T):
    return g.mu_inf * O.sutherland(T) / (rho * T * g.dt) + 0.5


def test_p4_stress_relaxes_with_tau_and_heat_flux_with_tau_pr():
    """Eq. (LBM): the non-equilibrium second moment is scaled by (1 - 1/tau); App. D:
    the centred third moment Qbar is scaled by (1 - 1/tau_Pr), tau_Pr = (tau-1/2)/Pr + 1/2."""
    xi, _ = O.velset()
    g = O.Grid(cells=(1, 1, 1), p=2, dt=0.05, mu_inf=0.03, pr_correction=True, Pr=0.7)
    pop = _noneq_state(g, 11, amp=0.08)
    post = O.collide(g, pop)
    for n in range(g.nodes):
        f = pop[0].reshape(45, -1)[:, n]
        fp = post[0].reshape(45, -1)[:, n]
        gs = pop[1].reshape(45, -1)[:, n].sum()
        rho = f.sum()
        u = f @ xi / rho
        e2 = f @ (xi ** 2).sum(1) + gs
        T = (e2 - rho * u @ u) / (2 * 2.5 * rho)
        tau = _tau(g, rho, T)
        tau_pr = (tau - 0.5) / g.Pr + 0.5
        Pi_eq = rho * (np.outer(u, u) + T * np.eye(3))
        Pi, Pi_p = [np.einsum("i,ia,ib->ab", h, xi, xi) for h in (f, fp)]
        assert np.allclose(Pi_p - Pi_eq, (1 - 1 / tau) * (Pi - Pi_eq), atol=1e-12)
        c = xi - u
        Qb, Qb_p = [np.einsum("i,ia,ib,ic->abc", h, c, c, c) for h in (f, fp)]
        assert np.allclose(Qb_p, (1 - 1 / tau_pr) * Qb, atol=1e-12)


# ---------------------------------------------------------------- P5 Horner vs tensor
def _horner_feq(rho, u, T, xi, w):
    """Equilibrium written as a quartic in s = xi.u per velocity shell (derived
    independently by contracting App. A with App. B in closed form)."""
    th = T - 1.0
    u2 = u @ u
    x2 = (xi ** 2).sum(1)
    s = xi @ u
    c0 = 1 + 0.5 * (-u2 + th * (x2 - 3)) + u2 * u2 / 8 + th * u2 * (5 - x2) / 4 \
        + th * th * (x2 * x2 - 10 * x2 + 15) / 8
    c1 = 1 + 0.5 * (-u2 + th * (x2 - 5))
    c2 = 0.5 - u2 / 4 + th * (x2 - 7) / 4
    return w * rho * (c0 + s * (c1 + s * (c2 + s * (1 / 6 + s / 24))))


@pytest.mark.parametrize("seed", range(4))
def test_p5_tensor_contraction_equals_closed_form_quartic(seed):
    rng = np.random.default_rng(100 + seed)
    xi, w = O.velset()
    rho, u, T = rng.uniform(0.5, 2), rng.uniform(-2, 2, 3), rng.uniform(0.5, 2)
    a = O.feq(rho, u, T)
    b = _horner_feq(rho, u, T, xi, w)
    assert np.max(np.abs(a - b)) <= 1e-14 * np.max(np.abs(a)) * 10


# ---------------------------------------------------------------- P6 interpolation
@pytest.mark.parametrize("p", [2, 3, 4])
def test_p6_lagrange_basis_properties(p):
    """Eq. (interpolation) on GLC points: Kronecker at nodes, partition of unity,
    exactness for degree <= p, inexact at degree p+1."""
    r = O.glc(p)
    assert np.allclose(r, -np.cos(np.pi * np.arange(p + 1) / p), atol=1e-15)
    for a in range(p + 1):
        assert np.allclose(O.lagrange(p, r[a]), np.eye(p + 1)[a], atol=1e-14)
    rng = np.random.default_rng(p)
    for x in rng.uniform(-1, 1, 7):
        ell = O.lagrange(p, x)
        assert abs(ell.sum() - 1) < 1e-14
        for k in range(p + 1):
            assert abs(ell @ r ** k - x ** k) < 1e-13
        assert abs(ell @ r ** (p + 1) - x ** (p + 1)) > 1e-6
        d = O.lagrange_deriv(p, x)
        for k in range(1, p + 1):
            assert abs(d @ r ** k - k * x ** (k - 1)) < 1e-12


def test_p6_quadrature_weights_are_clenshaw_curtis():
    """Textbook Clenshaw-Curtis weights on Chebyshev-Lobatto points."""
    assert np.allclose(O.quad_weights(2), [1 / 3, 4 / 3, 1 / 3], atol=1e-14)
    assert np.allclose(O.quad_weights(4), [1 / 15, 8 / 15, 12 / 15, 8 / 15, 1 / 15], atol=1e-14)
    assert np.allclose(O.quad_weights(3), [1 / 9, 8 / 9, 8 / 9, 1 / 9], atol=1e-14)


@pytest.mark.parametrize("p,shift", [(2, (1, 0, 0)), (3, (-2, 1, 3)), (4, (0, -1, 2))])
def test_p6_whole_cell_shift_is_pure_translation(p, shift):
    """A departure point that is a whole number of cells away lands on a support point,
    so streaming is an exact periodic translation (also for multi-cell departures,
    cf. Fig. 4)."""
    g = O.Grid(cells=(4, 3, 5), p=p, dt=0.25)
    h = [2 * np.pi / c for c in g.cells]
    xi = np.array([[shift[d] * h[d] / g.dt for d in range(3)]])
    rng = np.random.default_rng(1)
    src = rng.standard_normal((1, 1) + g.N[::-1])
    out = O.stream(g, src, xi)
    ref = np.roll(src, shift=(shift[2] * p, shift[1] * p, shift[0] * p), axis=(2, 3, 4))
    assert np.allclose(out, ref, atol=1e-13, rtol=0)


@pytest.mark.parametrize("p", [2, 3])
def test_p6_polynomials_of_degree_p_are_streamed_exactly(p):
    """Inside the departure cell, tensor Lagrange interpolation is exact for polynomials
    of degree <= p in each coordinate (checked where the departure cell does not wrap)."""
    g = O.Grid(cells=(5, 4, 4), p=p, dt=0.1)
    X = [O.node_coords(g, d) for d in range(3)]
    z, y, x = np.meshgrid(X[2], X[1], X[0], indexing="ij")
    rng = np.random.default_rng(p)
    cx, cy, cz = rng.standard_normal((3, p + 1))
    poly = lambda c, t: sum(c[k] * t ** k for k in range(p + 1))
    field = poly(cx, x) * poly(cy, y) * poly(cz, z)
    vel = np.array([[1.3, -0.7, 0.45]])
    out = O.stream(g, field[None, None], vel)[0, 0]
    dx, dy, dz = g.dt * vel[0]
    exact = poly(cx, x - dx) * poly(cy, y - dy) * poly(cz, z - dz)
    # the right-face node of the last cell is node 0 (x = 0), where the global polynomial
    # is not periodic; keep departures whose cell is not the last one in any direction
    L = 2 * np.pi
    h = [L / c for c in g.cells]
    ok = ((x - dx >= 0) & (x - dx < L - h[0]) & (y - dy >= 0) & (y - dy < L - h[1])
          & (z - dz >= 0) & (z - dz < L - h[2]))
    assert ok.sum() > 0.2 * ok.size
    scale = np.max(np.abs(field))
    assert np.max(np.abs(out - exact)[ok]) < 1e-11 * scale


# ---------------------------------------------------------------- P7 advection order
@pytest.mark.parametrize("p", [2, 3])
def test_p7_smooth_advection_converges_at_order_p_plus_1(p):
    """Pure streaming (collision off) of a smooth periodic field: the error of the
    semi-Lagrangian step decreases like h^(p+1) at fixed dt."""
    vel = np.array([[0.731, -0.412, 0.297]])
    errs = []
    for nc in (8, 16):
        g = O.Grid(cells=(nc, nc, nc), p=p, dt=0.3, collide=False)
        X = [O.node_coords(g, d) for d in range(3)]
        z, y, x = np.meshgrid(X[2], X[1], X[0], indexing="ij")
        fn = lambda x, y, z: np.sin(x + 0.3) * np.cos(2 * y) * np.sin(z - 0.2)
        f = fn(x, y, z)[None, None]
        nsteps = 4
        for _ in range(nsteps):
            f = O.stream(g, f, vel)
        t = nsteps * g.dt
        exact = fn(x - t * vel[0, 0], y - t * vel[0, 1], z - t * vel[0, 2])
        errs.append(np.max(np.abs(f[0, 0] - exact)))
    order = math.log2(errs[0] / errs[1])
    assert order > p + 0.5, (errs, order)


# ---------------------------------------------------------------- P8 shear wave
def _wave_run(kind, pr, n0=40, n1=80):
    """Low-Mach wave (k = 1) on an (8,1,1)-cell mesh.  The amplitude is projected on
    sin(x) after n0 start-up steps and again n1 steps later; returns (rate, expected).
    The entropy mode is measured through the linearised entropy s' = C_v T' - rho',
    which acoustic waves (isentropic to leading order) do not carry."""
    p, nc = 4, 8
    nu = 0.05
    dt = 0.05
    Pr = 0.7
    Cv, D = 2.5, 3
    g = O.Grid(cells=(nc, 1, 1), p=p, dt=dt, mu_inf=nu / O.sutherland(1.0), Pr=Pr,
               pr_correction=pr)
    x = O.node_coords(g, 0)
    shp = g.N[::-1]
    X = np.broadcast_to(x, shp)
    eps = 1e-3
    rho = np.ones(shp)
    u = np.zeros((3,) + shp)
    T = np.ones(shp)
    if kind == "shear":
        u[1] = eps * np.sin(X)
    else:  # entropy mode: uniform pressure, temperature perturbation
        T = 1.0 + eps * np.sin(X)
        rho = 1.0 / T
    pop = O.step(g, O.init_fields(g, rho, u, T), n0)
    amp = []
    for s in range(2):
        r, uu, TT = O.moments(g, pop)
        field = uu[1] if kind == "shear" else Cv * (TT - 1.0) - (r - 1.0)
        amp.append(2 * np.mean(field * np.sin(X)))
        if s == 0:
            pop = O.step(g, pop, n1)
    rate = -math.log(amp[1] / amp[0]) / (n1 * dt)
    if kind == "shear":
        expect = nu  # k = 1: decay nu k^2 with nu = mu/rho
    else:
        Cp = Cv + 1
        fac = ((D / 2 + 1) / Pr + Cv - D / 2) if pr else Cp
        expect = nu * fac / Cp
    return rate, expect


def test_p8_shear_wave_decays_at_viscous_rate():
    """App. C: mu = (tau - 1/2) dt P, so a shear wave decays as exp(-nu k^2 t)."""
    rate, expect = _wave_run("shear", False)
    assert abs(rate / expect - 1) < 0.005, (rate, expect)


@pytest.mark.parametrize("pr", [False, True])
def test_p8_entropy_mode_decays_at_thermal_rate(pr):
    """App. C gives lambda = tau P C_p (Pr = 1).  With the App. D term on f and
    g* = (2C_v - D) T f* (which has no first moment) only f's heat flux relaxes at
    tau_Pr, so the thermal diffusivity is nu ((D/2+1)/Pr + C_v - D/2) / C_p; at Pr = 0.7
    this is 0.914 nu/Pr, i.e. an effective Prandtl number of 0.766."""
    rate, expect = _wave_run("entropy", pr)
    assert abs(rate / expect - 1) < 0.015, (rate, expect)
    if pr:
        assert abs(rate / (0.05 / 0.7) - 1) > 0.05  # distinguishable from nu/Pr


# ---------------------------------------------------------------- P9 Taylor-Green
def test_p9_tgv_initial_integrals():
    """Sec. III.C initial condition: E_k(0) = 1/8 (the density correction integrates to
    zero), <|curl u|^2> = 3/4 U0^2, div u = 0.  The discrete values converge to these."""
    g0 = golden()
    errs = []
    for nc in (4, 8):
        Ma, gam, Re = 0.5, 1.4, 1600.0
        U0 = Ma * math.sqrt(gam)
        g = O.Grid(cells=(nc, nc, nc), p=4, dt=0.1, mu_inf=U0 / Re)
        rho, u, T = O.tgv_fields(g, U0)
        pop = O.init_fields(g, rho, u, T)
        ek, es, ec = O.diag(g, pop, 1.0, Re, U0)
        mu1 = g0["sutherland_a"] / (1 + g0["sutherland_b"])
        errs.append((abs(ek - 0.125), abs(es - 0.75 * mu1 / Re), abs(ec)))
    assert errs[1][0] < 1e-6 and errs[1][1] < 1e-3 * 0.75 / 1600 and errs[1][2] < 1e-9
    assert errs[1][1] < errs[0][1]


def _spectral_grad(f, L=2 * np.pi):
    """Exact derivatives of a periodic trigonometric polynomial sampled on a uniform grid
    (numpy FFT), axis order (z, y, x); returns [d/dx, d/dy, d/dz]."""
    out = []
    for ax in (2, 1, 0):
        n = f.shape[ax]
        k = np.fft.fftfreq(n, d=L / n) * 2 * np.pi
        shp = [1, 1, 1]
        shp[ax] = n
        out.append(np.real(np.fft.ifft(1j * k.reshape(shp) * np.fft.fft(f, axis=ax), axis=ax)))
    return out


@pytest.mark.parametrize("Ma", [0.5, 1.25])
def test_p9_tgv_density_is_the_incompressible_pressure(Ma):
    """Sec. III.C initial condition (its density expression is garbled in the paper): at
    uniform T0 the density perturbation must carry the pressure of the incompressible
    Taylor-Green flow, p' = rho' T0 (P = rho T), which the incompressible equations fix by
    the pressure Poisson relation  lap p' = -rho0 d_i u_j d_j u_i  (plus a zero mean).
    A p = 1 mesh puts the oracle's nodes on a uniform grid, where spectral derivatives of
    these band-limited fields are exact; a wrong amplitude (C/8), a missing "+2" or a
    sign error in the density breaks the relation at O(1)."""
    gam, T0, rho0 = 1.4, 1.0, 1.0
    U0 = Ma * math.sqrt(gam * T0)
    g = O.Grid(cells=(16, 16, 16), p=1, dt=0.1)
    x = O.node_coords(g, 0)
    assert np.allclose(np.diff(x), 2 * np.pi / 16, rtol=0, atol=1e-14)  # uniform nodes
    rho, u, T = O.tgv_fields(g, U0, rho0=rho0, T0=T0)
    assert np.all(T == T0)
    pp = (rho - rho0) * T0
    lap = sum(_spectral_grad(gd)[d] for d, gd in enumerate(_spectral_grad(pp)))
    du = [_spectral_grad(u[c]) for c in range(3)]  # du[j][i] = d u_j / d x_i
    rhs = -rho0 * sum(du[j][i] * du[i][j] for i in range(3) for j in range(3))
    scale = np.max(np.abs(rhs))
    assert scale > 0.1 * U0 * U0
    assert np.max(np.abs(lap - rhs)) <= 1e-12 * scale
    assert abs(pp.mean()) <= 1e-14
    # and the incompressible velocity field is divergence free
    assert np.max(np.abs(du[0][0] + du[1][1] + du[2][2])) <= 1e-12 * U0


def test_sutherland_constants_match_paper():
    g = golden()
    for T in (0.5, 1.0, 1.7):
        assert O.sutherland(T) == pytest.approx(g["sutherland_a"] * T ** 1.5
                                                / (T + g["sutherland_b"]), rel=1e-15)


def test_sampled_tgv_step_matches_full_step():
    """The on-demand (sampled) Taylor-Green step used for full-size checks agrees with the
    full-grid step on a small mesh (same departure search and collision)."""
    Ma, gam, Re = 0.5, 1.4, 1600.0
    U0 = Ma * math.sqrt(gam)
    g = O.Grid(cells=(3, 2, 4), p=3, dt=0.2, mu_inf=U0 / Re, pr_correction=True)
    rho, u, T = O.tgv_fields(g, U0)
    full = O.step(g, O.init_fields(g, rho, u, T), 1).reshape(90, -1)
    nodes = np.array([0, 5, 77, g.nodes - 1, 123])
    samp = O.tgv_step_sample(g, nodes, U0)
    assert np.allclose(samp, full[:, nodes].T, rtol=1e-13, atol=1e-15)
