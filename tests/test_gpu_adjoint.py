"""Reverse mode on the GPU against the oracle's reverse mode and against finite differences.

Tolerances:
  * streaming and its transpose, E_k seed: FP64 kernels vs the oracle's literal sums, 1e-12
    relative (different summation order only); FP32 storage 2e-6 (FP32 rounding of a few
    terms of size <= max|x|);
  * adjoint step and initialisation transpose: the oracle builds its Jacobians by
    Richardson-extrapolated central differences, good to about 1e-10 relative; asserted at
    1e-8 of the largest entry (FP64), 2e-4 (FP32 arithmetic through 90 moment-chain terms);
  * gradients through the checkpointed autograd functions on the 16^3-cell, p = 3
    Taylor-Green run (200 steps, checkpoints every 20): FP64 against central differences of
    the FP64 forward run <= 1e-4 relative, FP32 against FP64 at the stated bound.
"""
import numpy as np
import pytest

import oracle as O
from paper_2012_05537_gb300 import build as B
from paper_2012_05537_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.build()
    from paper_2012_05537_gb300 import sllbm
    sllbm.load()
    return sllbm


def make(S, cells, p, storage, courant=2.0, Ma=0.5, Re=1600.0):
    return S.Sim(S.Config(cells=tuple(cells), p=p, Ma=Ma, Re=Re, courant=courant, storage=storage))


def grid_of(sim):
    c = sim.cfg
    return O.Grid(cells=tuple(c.cells), p=c.p, dt=sim.dt, mu_inf=float(sim.info.mu_inf), gamma=c.gamma, Pr=c.Pr)


def to_dev(sim, a):
    """Oracle order [2][45][z][y][x] -> a state-ordered device tensor [45][z][y][x][2]."""
    return torch.as_tensor(np.ascontiguousarray(np.moveaxis(a, 0, -1)), device="cuda").to(sim.pop_dtype)


def to_orc(t):
    return np.moveaxis(t.double().cpu().numpy(), -1, 0)


def noneq(g, seed, amp=0.02):
    rho, u, T = I.smooth_fields(g.N[::-1], seed)
    pop = O.init_fields(g, rho, u, T)
    return pop * (1.0 + amp * I.noise(pop.shape, seed + 1))


def rel_max(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


TOL_EXACT = {"f64": 1e-12, "f32": 2e-6}
TOL_FD = {"f64": 1e-8, "f32": 2e-4}


@pytest.mark.parametrize("storage", ["f64", "f32"])
@pytest.mark.parametrize("cells,p,courant", [((2, 3, 2), 2, 2.0), ((3, 2, 2), 3, 4.0), ((1, 2, 3), 4, 6.0)])
def test_stream_and_its_transpose_match_oracle(S, storage, cells, p, courant):
    sim = make(S, cells, p, storage, courant=courant)
    g = grid_of(sim)
    rng = np.random.default_rng(1)
    x = rng.standard_normal((2, 45) + g.N[::-1])
    out = sim.state_like()
    S.sllbm_stream_apply(sim.ctx, to_dev(sim, x).data_ptr(), out.data_ptr(), False)
    sim.sync()
    assert rel_max(to_orc(out), O.stream(g, x)) < TOL_EXACT[storage]
    S.sllbm_stream_apply(sim.ctx, to_dev(sim, x).data_ptr(), out.data_ptr(), True)
    sim.sync()
    assert rel_max(to_orc(out), O.stream_adjoint(g, x)) < TOL_EXACT[storage]


@pytest.mark.parametrize("storage", ["f64", "f32"])
@pytest.mark.parametrize("cells,p,courant", [((2, 1, 2), 2, 2.0), ((2, 2, 1), 3, 3.0), ((1, 1, 2), 4, 5.0)])
def test_adjoint_step_matches_oracle(S, storage, cells, p, courant):
    sim = make(S, cells, p, storage, courant=courant)
    g = grid_of(sim)
    state = noneq(g, 13)
    rng = np.random.default_rng(2)
    lam = rng.standard_normal(state.shape)
    st, ln = to_dev(sim, state), to_dev(sim, lam)
    g_state = to_orc(st)  # the state as stored (FP32 storage rounds it)
    out = torch.empty_like(ln)
    dmu = torch.zeros(1, dtype=torch.float64, device="cuda")
    S.sllbm_adjoint_step(sim.ctx, st.data_ptr(), ln.data_ptr(), out.data_ptr(), dmu.data_ptr())
    sim.sync()
    want, dmu_want = O.step_adjoint(g, g_state, to_orc(ln))
    assert rel_max(to_orc(out), want) < TOL_FD[storage]
    assert abs(float(dmu) - dmu_want) <= TOL_FD[storage] * 10 * abs(dmu_want)


@pytest.mark.parametrize("cells,p,courant", [((2, 1, 2), 2, 2.0), ((2, 2, 1), 3, 3.0)])
def test_adjoint_step_fp32_state_fp64_adjoint_matches_oracle(S, cells, p, courant):
    """FP32 states, FP64 adjoint populations: the streamed state is computed in FP32 (relative
    error ~1e-7 of the populations), the rest in FP64, so the result sits within 1e-6 of the
    oracle's adjoint at the same (rounded) state."""
    sim = make(S, cells, p, "f32", courant=courant)
    sim.set_adjoint_type("f64")
    g = grid_of(sim)
    st = to_dev(sim, noneq(g, 23))
    rng = np.random.default_rng(6)
    lam = torch.as_tensor(np.ascontiguousarray(np.moveaxis(rng.standard_normal((2, 45) + g.N[::-1]), 0, -1)),
                          device="cuda")
    out = torch.empty_like(lam)
    dmu = torch.zeros(1, dtype=torch.float64, device="cuda")
    S.sllbm_adjoint_step(sim.ctx, st.data_ptr(), lam.data_ptr(), out.data_ptr(), dmu.data_ptr())
    sim.sync()
    want, dmu_want = O.step_adjoint(g, to_orc(st), to_orc(lam))
    assert rel_max(to_orc(out), want) < 1e-6
    assert abs(float(dmu) - dmu_want) <= 1e-5 * abs(dmu_want)


@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_ek_seed_matches_oracle(S, storage):
    sim = make(S, (2, 3, 1), 3, storage)
    g = grid_of(sim)
    st = to_dev(sim, noneq(g, 17))
    lam = sim.state_like()
    S.sllbm_ek_adjoint(sim.ctx, st.data_ptr(), lam.data_ptr())
    sim.sync()
    want = O.ek_grad(g, to_orc(st), sim.cfg.rho0, float(sim.info.U0))
    assert rel_max(to_orc(lam), want) < TOL_EXACT[storage]


@pytest.mark.parametrize("storage", ["f64", "f32"])
@pytest.mark.parametrize("cells,p,wts", [((3, 2, 1), 3, (1.0, 0.0, 0.0)), ((3, 2, 1), 3, (0.0, 1.0, 1.0)),
                                         ((2, 1, 3), 2, (0.3, -2.0, 5.0)), ((2, 2, 2), 4, (0.0, 1.0, 0.0))])
def test_diag_seed_matches_oracle(S, storage, cells, p, wts):
    """sllbm_diag_adjoint (gather form, FP64 arithmetic) against the oracle's derivative of
    the diagnostics (scatter form) at the same state: meshes with one-cell directions (a
    face node held twice by the same cell) and several cells (face nodes held by two)."""
    sim = make(S, cells, p, storage)
    g = grid_of(sim)
    st = to_dev(sim, noneq(g, 29))
    lam = sim.state_like()
    S.sllbm_diag_adjoint(sim.ctx, st.data_ptr(), lam.data_ptr(), *wts)
    sim.sync()
    want = O.diag_grad(g, to_orc(st), sim.cfg.rho0, sim.cfg.Re, float(sim.info.U0), wts)
    assert rel_max(to_orc(lam), want) < TOL_EXACT[storage]


@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_init_fields_adjoint_matches_oracle(S, storage):
    sim = make(S, (2, 1, 2), 4, storage)
    g = grid_of(sim)
    rho, u, T = I.smooth_fields(g.N[::-1], 19)
    rng = np.random.default_rng(3)
    lam = to_dev(sim, rng.standard_normal((2, 45) + g.N[::-1]))
    dev = [torch.as_tensor(np.ascontiguousarray(x), device="cuda") for x in (rho, u, T)]
    out = [torch.empty_like(x) for x in dev]
    S.sllbm_init_fields_adjoint(sim.ctx, *(x.data_ptr() for x in dev), lam.data_ptr(),
                                *(x.data_ptr() for x in out))
    sim.sync()
    want = O.init_fields_vjp(g, rho, u, T, to_orc(lam))
    for got, ref in zip(out, want):
        assert rel_max(got.cpu().numpy(), ref) < 1e-8


def test_reverse_mode_refuses_what_it_does_not_cover(S):
    for kw in ({"storage": "f16dev"}, {"storage": "f32", "pr_correction": True}):
        sim = S.Sim(S.Config(cells=(2, 2, 2), p=2, **kw))
        buf = torch.zeros(int(sim.info.pop_bytes), dtype=torch.uint8, device="cuda")
        dmu = torch.zeros(1, dtype=torch.float64, device="cuda")
        out = torch.zeros_like(buf)
        rc = S.load().sllbm_adjoint_step(sim.ctx, buf.data_ptr(), buf.data_ptr(), out.data_ptr(), dmu.data_ptr())
        assert rc == S.EINVAL


# Relative difference of the FP32 gradients from the FP64 gradients on the 200-step run.
# Measured on GB300: dEk/deps 3.6e-4, dEk/dmu_inf 7.0e-6 (FP64 vs central differences:
# 3.6e-8 and 1.2e-11).  dEk/deps is the projection of the gradient field on a white-noise
# perturbation, about 1/sqrt(3 N_nodes) = 1/576 of |grad| |du| for the smooth gradient, while
# the FP32 rounding of the forward states is itself white and is not suppressed by that
# projection.  Asserted with a factor ~3 margin.
STATED_F32 = {"dEk_deps": 1e-3, "dEk_dmu_inf": 3e-5}
# FP32 forward with FP64 adjoint populations against central differences of the FP64
# forward run.  Measured: dEk/deps 3.5e-4, the same as with FP32 adjoint populations: the
# difference comes from the FP32 forward trajectory (its rounding perturbs the state with
# spatially white noise, which the projection on the white-noise perturbation does not
# suppress), not from the precision of the adjoint.
STATED_F32_ADJ64 = {"dEk_deps": 1e-3, "dEk_dmu_inf": 3e-5}


# FP32 run with compensated moment sums (sllbm_set_compensated) against the FP64 adjoint,
# relative.  Dissipation: the 1e-4 target of finite-difference agreement (measured on GB300:
# d eps/d e 3.6e-7, d eps/d mu_inf 2.0e-5; with plain sums 6.6e-5 and 2.0e-5).  Kinetic
# energy: measured d Ek/d e 1.7e-4 (plain sums 3.6e-4), d Ek/d mu_inf 6.7e-6, asserted at
# about three times that: the projection on the white-noise perturbation keeps the FP32
# rounding of the forward states (see test_gradients_on_the_taylor_green_run).
STATED_F32_COMP = {"deps_deps": 1e-4, "deps_dmu_inf": 1e-4, "dEk_deps": 5e-4, "dEk_dmu_inf": 3e-5}


def test_dissipation_gradients_on_the_taylor_green_run(S):
    """d eps / d e and d eps / d mu_inf (eps = eps_s + eps_c after the 200 steps of the
    reverse-mode workload) by the adjoint chain, against central differences of the FP64
    forward run (<= 1e-4) and, for the FP32 run with compensated moment sums, against the
    FP64 adjoint (the stated bounds above)."""
    from paper_2012_05537_gb300 import adjoint as A

    w = I.WORKLOADS["tgv_16c_p3_adj"]
    every = 20
    cfg = {st: S.Config(cells=w.cells, p=w.p, Ma=w.Ma, Re=w.Re, courant=w.courant, storage=st)
           for st in ("f64", "f32")}
    rho, u, T = A.tgv_fields(cfg["f64"], device="cuda")
    U0 = float(make(S, (1, 1, 1), 2, "f64", Ma=w.Ma).info.U0)
    du = torch.as_tensor(1e-3 * U0 * I.noise(tuple(u.shape), 0), device="cuda")
    res = {}
    for st in ("f64", "f32"):
        sim = S.Sim(cfg[st])
        if st == "f32":
            S.sllbm_set_compensated(sim.ctx, True)
        res[st] = A.diagnostic_gradients(sim, rho, u, T, du, w.steps, every)
        sim.close()
    sim = S.Sim(cfg["f64"])
    mu0 = float(sim.info.mu_inf)

    def eps(e=0.0, mu=mu0):
        sim.set_mu_inf(mu)
        sim.init_fields(rho, u + e * du, T)
        assert sim.step(w.steps) == 0
        d = sim.diag()
        return d[1] + d[2]

    def directional(fun, x, h):
        d1 = (fun(x + h) - fun(x - h)) / (2 * h)
        d2 = (fun(x + h / 2) - fun(x - h / 2)) / h
        return (4 * d2 - d1) / 3

    fd_e = directional(lambda e: eps(e=e), 0.0, 1.0)
    fd_mu = directional(lambda m: eps(mu=m), mu0, 1e-2 * mu0)
    g64, g32 = res["f64"], res["f32"]
    print("FP64 dissipation gradients", g64, "FD", fd_e, fd_mu)
    assert abs(g64["deps_deps"] - fd_e) <= 1e-4 * abs(fd_e)
    assert abs(g64["deps_dmu_inf"] - fd_mu) <= 1e-4 * abs(fd_mu)
    assert abs(g64["eps"] - eps()) <= 1e-12 * abs(g64["eps"])
    for k, bound in STATED_F32_COMP.items():
        r = abs(g32[k] - g64[k]) / abs(g64[k])
        print("FP32 vs FP64", k, r)
        assert r <= bound


def test_gradients_on_the_taylor_green_run(S):
    from paper_2012_05537_gb300 import adjoint as A

    w = I.WORKLOADS["tgv_16c_p3_adj"]
    every = 20
    res = {}
    cfg = {}
    for st in ("f64", "f32"):
        cfg[st] = S.Config(cells=w.cells, p=w.p, Ma=w.Ma, Re=w.Re, courant=w.courant, storage=st)
    rho, u, T = A.tgv_fields(cfg["f64"], device="cuda")
    U0 = float(make(S, (1, 1, 1), 2, "f64", Ma=w.Ma).info.U0)
    du = torch.as_tensor(1e-3 * U0 * I.noise(tuple(u.shape), 0), device="cuda")
    for st in ("f64", "f32"):
        sim = S.Sim(cfg[st])
        res[st] = A.kinetic_energy_gradients(sim, rho, u, T, du, w.steps, every)
        sim.close()
    sim = S.Sim(cfg["f32"])
    res["f32_adj64"] = A.kinetic_energy_gradients(sim, rho, u, T, du, w.steps, every, adjoint="f64")
    sim.close()

    sim = S.Sim(cfg["f64"])
    mu0 = float(sim.info.mu_inf)

    def ek(eps=0.0, mu=mu0):
        sim.set_mu_inf(mu)
        sim.init_fields(rho, u + eps * du, T)
        assert sim.step(w.steps) == 0
        return sim.diag()[0]

    def directional(fun, x, h):
        d1 = (fun(x + h) - fun(x - h)) / (2 * h)
        d2 = (fun(x + h / 2) - fun(x - h / 2)) / h
        return (4 * d2 - d1) / 3

    fd_eps = directional(lambda e: ek(eps=e), 0.0, 1.0)
    fd_mu = directional(lambda m: ek(mu=m), mu0, 1e-2 * mu0)
    g64, g32 = res["f64"], res["f32"]
    print("FP64 adjoint", g64, "FD", fd_eps, fd_mu)
    print("FP32 adjoint", g32)
    assert abs(g64["dEk_deps"] - fd_eps) <= 1e-4 * abs(fd_eps)
    assert abs(g64["dEk_dmu_inf"] - fd_mu) <= 1e-4 * abs(fd_mu)
    for k, bound in STATED_F32.items():
        r = abs(g32[k] - g64[k]) / abs(g64[k])
        print("FP32 vs FP64", k, r)
        assert r <= bound
    # FP32 forward, FP64 adjoint populations: against the finite differences of the FP64 run
    gm = res["f32_adj64"]
    errs = {k: abs(gm[k] - fd) / abs(fd) for k, fd in (("dEk_deps", fd_eps), ("dEk_dmu_inf", fd_mu))}
    print("FP32 forward + FP64 adjoint vs FD", errs)
    for k, r in errs.items():
        assert r <= STATED_F32_ADJ64[k]
