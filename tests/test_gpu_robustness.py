"""High-Mach, low-Reynolds Taylor-Green runs (Sec. III.C, the Re = 100 case): the paper reports
stable runs at Ma 2.5 and Ma 3.0 with time steps 0.015 and 0.03.  Reading of those time
steps: t* = t U0 / L units (the unit of the other Taylor-Green figures).

* Ma 2.5, Re = 100, C = 1 (numerator of the density perturbation), dt* = 0.015, 64^3 nodes:
  the run to t* = 4 stays finite with monotonically decaying kinetic energy, FP32 and FP64
  curves agreeing to 1e-5 (measured on GB300: E_k/E_k0 = 0.4696 at t* = 4, largest step-to-
  step change -1.3e-4).
* Ma 3.0: one step from the Taylor-Green state agrees with the oracle to FP64 round-off (the
  quartic equilibrium's terms reach s^4/24 ~ 1.5e3 here and cancel to O(1)).  The run itself
  does not stay finite on the meshes tried (64^3 to 192^3 nodes, dt* = 0.03 and the same dt in
  lattice units); that gap to the paper is recorded in the design notes, not asserted here.
"""
import math

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


def tgv_sim(S, Ma, dt_star, cells, p, storage):
    U0 = Ma * math.sqrt(1.4)
    return S.Sim(S.Config(cells=(cells,) * 3, p=p, Ma=Ma, Re=100.0, courant=None, dt=dt_star / U0, tgv_C=1.0,
                          storage=storage)).init_tgv()


def test_re100_ma25_run_is_stable_and_decays(S):
    curves = {}
    for st in ("f64", "f32"):
        sim = tgv_sim(S, 2.5, 0.015, 16, 4, st)
        ek = [sim.diag()[0]]
        for _ in range(27):  # t* = 4.05
            assert sim.step(10) == 0
            ek.append(sim.diag()[0])
        rho, _, T = sim.moments()
        assert float(T.min()) > 0.5 and float(rho.min()) > 0.2
        curves[st] = np.array(ek)
        sim.close()
    e = curves["f64"]
    assert np.all(np.isfinite(e))
    assert np.all(np.diff(e) < 0.0)
    assert 0.45 < e[-1] / e[0] < 0.49
    assert np.max(np.abs(curves["f32"] - e)) <= 1e-5 * e[0]


@pytest.mark.parametrize("Ma", [2.5, 3.0])
def test_high_mach_first_step_matches_oracle(S, Ma):
    sim = tgv_sim(S, Ma, 0.03, 6, 4, "f64")
    assert sim.step(1) == 0
    c = sim.cfg
    g = O.Grid(cells=tuple(c.cells), p=c.p, dt=sim.dt, mu_inf=float(sim.info.mu_inf), gamma=c.gamma, Pr=c.Pr)
    nodes = I.sample_nodes(sim.nodes, 64, seed=4)
    ref = O.tgv_step_sample(g, nodes, float(sim.info.U0), C=1.0)
    raw = sim.raw_state().reshape(45, -1, 2)[:, torch.as_tensor(nodes, device="cuda"), :]
    got = raw.permute(1, 2, 0).reshape(len(nodes), 90).double().cpu().numpy()
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.abs(ref).max()
