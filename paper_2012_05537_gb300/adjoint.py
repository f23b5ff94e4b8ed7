"""Reverse mode of the SLLBM step behind ``torch.autograd`` (the paper has no adjoint).

Three autograd functions; the forward and backward arithmetic of each runs in the
library's kernels (PyTorch only holds the tensors and chains the calls):

* :class:`InitFields` -- FP64 fields (rho, u, T) -> equilibrium state
  (``sllbm_init_fields``; backward ``sllbm_init_fields_adjoint``);
* :class:`Steps` -- (state, mu_inf) -> state after n steps (``sllbm_step``).  The forward
  keeps a checkpoint every k steps; the backward recomputes each segment from its
  checkpoint (k states held at a time) and applies ``sllbm_adjoint_step`` step by step in
  reverse, accumulating the mu_inf sensitivity on the device;
* :class:`KineticEnergy` -- state -> E_k of Sec. III.C (``sllbm_diag``; backward
  ``sllbm_ek_adjoint``);
* :class:`Diagnostics` -- state -> (E_k, eps_s, eps_c) of Sec. III.C (``sllbm_diag``;
  backward ``sllbm_diag_adjoint`` with the incoming gradient as the weights).

mu_inf sets the relaxation time through tau = mu_inf (mu/mu_inf)(T)/(rho T dt) + 1/2; the
sensitivity to the reference relaxation time tau_ref = mu_inf (mu/mu_inf)(T0)/(rho0 T0 dt)
+ 1/2 follows by the chain rule (:func:`dtau_ref_dmu`).
"""
from __future__ import annotations

import math

import torch

from . import sllbm as S


def _sutherland(T: float) -> float:
    return 1.4042 * T * math.sqrt(T) / (T + 0.40417)


def dtau_ref_dmu(sim: S.Sim) -> float:
    """d tau_ref / d mu_inf at the reference state (rho0, T0) of the context."""
    c = sim.cfg
    return _sutherland(c.T0) / (c.rho0 * c.T0 * sim.dt)


class InitFields(torch.autograd.Function):
    @staticmethod
    def forward(ctx, rho, u, T, sim):
        f = [x.detach().to(device=sim.device, dtype=torch.float64).contiguous() for x in (rho, u, T)]
        S.sllbm_init_fields(sim.ctx, f[0].data_ptr(), f[1].data_ptr(), f[2].data_ptr(), True)
        out = sim.state_like()
        out.copy_(sim.raw_state())
        ctx.sim = sim
        ctx.save_for_backward(*f)
        return out

    @staticmethod
    def backward(ctx, lam):
        sim = ctx.sim
        rho, u, T = ctx.saved_tensors
        lam = lam.detach().to(sim.adjoint_dtype).contiguous()
        need = ctx.needs_input_grad
        g = [torch.empty_like(x) if need[k] else None for k, x in enumerate((rho, u, T))]
        S.sllbm_init_fields_adjoint(sim.ctx, rho.data_ptr(), u.data_ptr(), T.data_ptr(), lam.data_ptr(),
                                    *(x.data_ptr() if x is not None else 0 for x in g))
        return g[0], g[1], g[2], None


class Steps(torch.autograd.Function):
    @staticmethod
    def forward(ctx, state, mu_inf, sim, n: int, every: int):
        if n < 0 or every < 1:
            raise ValueError("n >= 0 and every >= 1 are required")
        mu = float(mu_inf)
        sim.set_mu_inf(mu)
        st = state.detach().to(sim.pop_dtype).contiguous()
        sim.load_state(st)
        checkpoints = [st.clone()]
        for k in range(1, n + 1):
            rc = sim.step(1)
            if rc != S.OK:
                raise S.SllbmError(rc, "sllbm_step")
            if k % every == 0 and k < n:
                checkpoints.append(sim.raw_state().clone())
        out = sim.raw_state().clone()
        ctx.sim, ctx.n, ctx.every, ctx.mu = sim, n, every, mu
        ctx.checkpoints = checkpoints
        ctx.mu_meta = (mu_inf.shape, mu_inf.device) if torch.is_tensor(mu_inf) else None
        return out

    @staticmethod
    def backward(ctx, lam):
        sim, n, every = ctx.sim, ctx.n, ctx.every
        sim.set_mu_inf(ctx.mu)
        lam = lam.detach().to(sim.adjoint_dtype).contiguous().clone()
        spare = torch.empty_like(lam)
        dmu = torch.zeros(1, dtype=torch.float64, device=sim.device)
        for seg in range(len(ctx.checkpoints) - 1, -1, -1):
            start = seg * every
            end = min(start + every, n)
            states = [ctx.checkpoints[seg]]
            sim.load_state(states[0])
            for _ in range(start + 1, end):
                rc = sim.step(1)
                if rc != S.OK:
                    raise S.SllbmError(rc, "sllbm_step")
                states.append(sim.raw_state().clone())
            # states[k] is the state from which step start+k+1 was taken
            for k in range(end - start - 1, -1, -1):
                S.sllbm_adjoint_step(sim.ctx, states[k].data_ptr(), lam.data_ptr(), spare.data_ptr(),
                                     dmu.data_ptr())
                lam, spare = spare, lam
        gmu = None
        if ctx.mu_meta is not None:
            shape, dev = ctx.mu_meta
            gmu = dmu.reshape(shape).to(dev)
        return lam, gmu, None, None, None


class KineticEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, state, sim):
        st = state.detach().to(sim.pop_dtype).contiguous()
        sim.load_state(st)
        ek = S.sllbm_diag(sim.ctx)[0]
        ctx.sim = sim
        ctx.save_for_backward(st)
        return torch.tensor(ek, dtype=torch.float64, device=sim.device)

    @staticmethod
    def backward(ctx, g):
        sim = ctx.sim
        (st,) = ctx.saved_tensors
        lam = torch.empty(st.shape, dtype=sim.adjoint_dtype, device=st.device)
        S.sllbm_ek_adjoint(sim.ctx, st.data_ptr(), lam.data_ptr())
        return lam * g.to(lam.dtype), None


class Diagnostics(torch.autograd.Function):
    @staticmethod
    def forward(ctx, state, sim):
        st = state.detach().to(sim.pop_dtype).contiguous()
        sim.load_state(st)
        d = S.sllbm_diag(sim.ctx)
        ctx.sim = sim
        ctx.save_for_backward(st)
        return torch.tensor(d, dtype=torch.float64, device=sim.device)

    @staticmethod
    def backward(ctx, g):
        sim = ctx.sim
        (st,) = ctx.saved_tensors
        w = [float(x) for x in g.detach().to("cpu", torch.float64)]
        lam = torch.empty(st.shape, dtype=sim.adjoint_dtype, device=st.device)
        S.sllbm_diag_adjoint(sim.ctx, st.data_ptr(), lam.data_ptr(), w[0], w[1], w[2])
        return lam, None


def tgv_fields(cfg: S.Config, device=None):
    """Taylor-Green initial fields (rho, u[3], T) at the nodes, FP64 on the device: the
    moments of the equilibrium state sllbm_init_tgv builds in an FP64 context."""
    c = S.Config(**{**cfg.__dict__, "storage": "f64"})
    sim = S.Sim(c, device=device)
    sim.init_tgv()
    out = sim.moments()
    sim.close()
    return out


def kinetic_energy_gradients(sim: S.Sim, rho, u, T, du, steps: int, every: int, adjoint: str | None = None):
    """E_k after `steps` steps from the equilibrium of (rho, u + eps du, T) at eps = 0, and
    its gradients with respect to eps and mu_inf (returned as a dict, FP64 scalars).
    adjoint="f64" keeps the adjoint populations of an FP32 run in FP64."""
    if adjoint is not None:
        sim.set_adjoint_type(adjoint)
    eps = torch.zeros((), dtype=torch.float64, device=sim.device, requires_grad=True)
    mu = torch.tensor(float(sim.info.mu_inf), dtype=torch.float64, device=sim.device, requires_grad=True)
    state0 = InitFields.apply(rho, u + eps * du, T, sim)
    stateN = Steps.apply(state0, mu, sim, steps, every)
    ek = KineticEnergy.apply(stateN, sim)
    ek.backward()
    dmu = float(mu.grad)
    return {"Ek": float(ek.detach()), "dEk_deps": float(eps.grad), "dEk_dmu_inf": dmu,
            "dEk_dtau_ref": dmu / dtau_ref_dmu(sim)}


def diagnostic_gradients(sim: S.Sim, rho, u, T, du, steps: int, every: int, adjoint: str | None = None):
    """E_k and the dissipation eps = eps_s + eps_c after `steps` steps from the equilibrium of
    (rho, u + e du, T) at e = 0, with the gradient of each with respect to e and mu_inf: one
    forward run, one reverse sweep per quantity (FP64 scalars in a dict)."""
    if adjoint is not None:
        sim.set_adjoint_type(adjoint)
    e = torch.zeros((), dtype=torch.float64, device=sim.device, requires_grad=True)
    mu = torch.tensor(float(sim.info.mu_inf), dtype=torch.float64, device=sim.device, requires_grad=True)
    state0 = InitFields.apply(rho, u + e * du, T, sim)
    stateN = Steps.apply(state0, mu, sim, steps, every)
    d = Diagnostics.apply(stateN, sim)
    out = {}
    for name, wts in (("Ek", (1.0, 0.0, 0.0)), ("eps", (0.0, 1.0, 1.0))):
        J = d @ torch.tensor(wts, dtype=torch.float64, device=sim.device)
        ge, gm = torch.autograd.grad(J, (e, mu), retain_graph=True)
        out[name] = float(J.detach())
        out[f"d{name}_deps"] = float(ge)
        out[f"d{name}_dmu_inf"] = float(gm)
    return out
