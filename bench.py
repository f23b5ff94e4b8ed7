"""Throughput benchmark of the fused SLLBM step (node-updates/s) on synthetic
Taylor-Green input.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl mine|reference]
                  [--workload tgv_32c_p4] [--storage f32|f64|f16dev|bf16dev]
                  [--mixed-steps 400]

One "step" is one SLLBM time step over the whole mesh: one launch of the fused kernel
(streaming of all 90 populations, moments, equilibrium, collision).  The default
workload is the 32^3-cell, p = 4 (128^3 nodes) Taylor-Green vortex at Ma 0.5, Re 1600,
Courant number 4, FP32 storage.  Each population buffer (755 MB) is larger than the
129 MB L2, so no L2 flush is needed between steps.  With N > 1 (torchrun) every rank
runs an independent replica (the path is not sharded across GPUs: replicas only).

Beside the headline line's FP64 variant, the "mixed" block runs the 64^3-cell, p = 3
(192^3 nodes) Taylor-Green vortex at Ma 1.25, Courant number 1 from the same initial state
in FP64, FP32 and the 16-bit deviation storages for a bounded number of steps and states
each one's throughput, HBM fraction and relative L2 error against the FP64 GPU run (rho, u,
T at the end; kinetic-energy and dissipation curves).

The "batched" block runs 64 seeded Taylor-Green instances of uneven size, order and
parameters one by one and as one CUDA graph per two steps (autotuned kernels), and states
the aggregate node-updates/s of each.  The "adjoint" block times the reverse mode on the 48^3-node Taylor-Green run and states
its gradients' errors against central differences of the FP64 forward run.

The line's "alu_peaks" are measured at the start by the library's FMA microbenchmark
(sllbm_fma_peak: FP32, packed FP32x2, FP64); the FP64 variant and the mixed block quote
their arithmetic against them ("roofline_alu"; for 16-bit storage the bound is the larger of
the HBM time of the algorithmic bytes and the FP32 time of the algorithmic flops).  The
mixed block also runs FP32 arithmetic with compensated moment sums ("*_comp"), and the
"compensated" variant times the headline workload with them.  The "pr" variant times the
headline workload with the Prandtl term of App. D on.  The "long_run"
block runs the throughput mesh for 2000 steps in FP32 and FP64 (Prandtl term on, the
paper's Taylor-Green setting) and compares their E_k(t) and eps(t) curves with each other
and with the oracle's 16^3-cell run at the same time step (tests/golden).

--impl reference times the FP64 CPU oracle (tests-only code) on the host cores on a
bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import dataclasses
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2012_05537_gb300 import inputs as I  # noqa: E402

METRIC = "node-updates/s (×45 pops) vs HBM roofline; mixed vs FP64 at stated error"
UNIT = "node-updates/s"
FALLBACK_HBM_GBS = 6800.0


def algorithmic_flops_per_node(p: int) -> float:
    """Floating-point operations of one node-update (an FMA counts 2): separable streaming of
    90 values, 3 passes of p+1 weights each; moments (45 x 6); the quartic equilibrium by
    Horner per velocity (45 x 9); the BGK update of 90 values (2 each)."""
    fma = 90 * 3 * (p + 1) + 45 * 6 + 45 * 9 + 90 * 2
    return 2.0 * fma


def alu_peaks(S):
    """FMA rates of this GPU in TFLOP/s from the library's microbenchmark (FP32, packed
    FP32x2, FP64), each timed over one launch of a few tens of milliseconds."""
    out = {}
    for name, kind, iters in (("fp32", 0, 32768), ("fp32x2", 1, 16384), ("fp64", 2, 512)):
        f, t = S.sllbm_fma_peak(kind, iters)
        out[name + "_tflops"] = f / 1e12
        out[name + "_ms"] = t * 1e3
    out["how"] = ("sllbm_fma_peak: independent dependent FMA chains on every SM, one timed launch "
                  "after a warm-up launch (CUDA events)")
    return out


def min_roofline(bytes_per_node, flops_per_node, nodes, kernel_ms, hbm_gbs, alu_tflops):
    """Roofline of a step bound by HBM and by the ALU together: the bound is the larger of
    the HBM time of the algorithmic bytes and the ALU time of the algorithmic flops."""
    t_hbm = bytes_per_node * nodes / (hbm_gbs * 1e9)
    t_alu = flops_per_node * nodes / (alu_tflops * 1e12)
    t = kernel_ms / 1e3
    return {"bound": "hbm" if t_hbm >= t_alu else "alu", "frac": max(t_hbm, t_alu) / t,
            "hbm_frac": t_hbm / t, "alu_frac": t_alu / t, "hbm_peak_gbs": hbm_gbs,
            "alu_peak_tflops": alu_tflops, "algorithmic_flops_per_node": flops_per_node,
            "algorithmic_bytes_per_node": bytes_per_node}


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["mine", "reference"], default="mine")
    ap.add_argument("--workload", default="tgv_32c_p4", choices=sorted(I.WORKLOADS))
    ap.add_argument("--storage", choices=["f32", "f64", "f16dev", "bf16dev"], default=None)
    ap.add_argument("--e2e-steps", type=int, default=40)
    ap.add_argument("--kernel", type=int, choices=[0, 1, 2], default=0,
                    help="step kernel of the headline run: 0 automatic, 1 generic, 2 TMA-fed")
    ap.add_argument("--pr", action="store_true",
                    help="headline run with the quasi-equilibrium Prandtl term (App. D) on")
    ap.add_argument("--compensated", action="store_true",
                    help="headline run with compensated moment sums (sllbm_set_compensated)")
    ap.add_argument("--periodic-z", choices=["ghost", "wrap"], default="ghost",
                    help="z boundary of the headline mesh: ghost planes (the mesh as one periodic z-slab, "
                         "refreshed in place before each step) or source boxes wrapping around")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--mixed-steps", type=int, default=400,
                    help="steps of the Ma 1.25 mixed-precision comparison (0: skip)")
    ap.add_argument("--mixed-every", type=int, default=20)
    ap.add_argument("--batch-steps", type=int, default=500,
                    help="steps of the 64-instance batched comparison (0: skip)")
    ap.add_argument("--long-steps", type=int, default=2000,
                    help="steps of the FP32 vs FP64 long run of the throughput mesh (0: skip)")
    ap.add_argument("--long-every", type=int, default=50)
    ap.add_argument("--no-adjoint", action="store_true",
                    help="skip the reverse-mode block (gradients on the 48^3-node run)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


KERNEL_SOURCES = {
    # the TMA-fed kernel and what it is built from
    "tma": ("step_tma.cuh", "step_tma.cu", "collide.cuh", "compsum.cuh", "packed.cuh", "sllbm_internal.h", "tables.h"),
    # the generic tile kernel and its instances
    "generic": ("step_kernel.cuh", "collide.cuh", "compsum.cuh", "packed.cuh", "storage.cuh", "sllbm_internal.h", "tables.h", "step_f32.cu",
                "step_f32_tiles.cu", "step_f64.cu", "step_f16.cu"),
}


def kernel_source_hash(kind: str = "tma") -> str:
    csrc = os.path.join(ROOT, "paper_2012_05537_gb300", "csrc")
    h = hashlib.sha256()
    for name in KERNEL_SOURCES[kind]:
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profiled_traffic(workload: str, storage: str, kind: str = "tma", suffix: str = ""):
    """DRAM bytes per launch recorded from an ncu capture of the current kernel source,
    or None if no summary matches the current source hash of that kernel."""
    path = os.path.join(ROOT, "profiles", f"step_{storage}_{workload}{suffix}.md")
    if not os.path.exists(path):
        return None
    text = open(path).read()
    m_hash = re.search(r"kernel_source_hash:\s*([0-9a-f]+)", text)
    m_bytes = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", text)
    if not m_hash or not m_bytes or m_hash.group(1) != kernel_source_hash(kind):
        return None
    return float(m_bytes.group(1))


class ClockSampler:
    """nvidia-smi clock/throttle samples every 200 ms while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        self.path = None
        self.gpu = gpu_index

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None

        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows),
                "power_w_max": max((num(r[3]) or 0.0) for r in rows)}


def oracle_sample_rate(w: I.Workload, min_seconds: float = 8.0):
    """Oracle node-updates/s on a periodic sub-box of the workload: same cell size h, p,
    dt, Ma, Re; 6 x 6 x 6 cells; Taylor-Green initial fields at those coordinates."""
    import numpy as np

    import oracle as O
    h = 2 * math.pi / w.cells[0]
    sub = (6, 6, 6)
    g = O.Grid(cells=sub, p=w.p, dt=w.dt(), mu_inf=w.mu_inf, gamma=w.gamma, Pr=w.Pr,
               pr_correction=w.pr_correction, L=tuple(c * h for c in sub))
    pop = O.init_fields(g, *O.tgv_fields(g, w.U0))
    steps, t0 = 0, time.perf_counter()
    while True:
        pop = O.step(g, pop, 1)
        steps += 1
        el = time.perf_counter() - t0
        if el >= min_seconds:
            break
    assert np.isfinite(pop).all()
    return g.nodes * steps / el, O.num_threads(), (
        f"{steps} oracle step(s) on a periodic 6^3-cell sub-box ({g.nodes} nodes) of {w.name} "
        f"(same h, p={w.p}, dt, Ma, Re); FP64; {el:.1f} s")


def run_reference(args, rank, world):
    """Reference arm: the FP64 CPU oracle, rank 0 only."""
    if rank != 0:
        return
    import numpy as np

    import oracle as O
    w = I.WORKLOADS[args.workload]
    h = 2 * math.pi / w.cells[0]
    sub = (3, 3, 2)  # bounded sample per step so that K steps stay within minutes
    g = O.Grid(cells=sub, p=w.p, dt=w.dt(), mu_inf=w.mu_inf, gamma=w.gamma, Pr=w.Pr,
               pr_correction=w.pr_correction, L=tuple(c * h for c in sub))
    pop = O.init_fields(g, *O.tgv_fields(g, w.U0))
    pop = O.step(g, pop, max(0, args.warmup))
    t0 = time.perf_counter()
    pop = O.step(g, pop, args.steps)
    el = time.perf_counter() - t0
    assert np.isfinite(pop).all()
    value = g.nodes * args.steps / el
    sample = (f"each step: one oracle step on a periodic 3x3x2-cell sub-box ({g.nodes} nodes) of "
              f"{w.name} (same h, p, dt, Ma, Re); FP64 CPU")
    cores = O.num_threads()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * el / max(1, args.steps), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "note": w.note},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def replica_throughput(total_ms: float, nodes: int, steps: int, dist=None, device="cpu"):
    """Whole-job throughput of N independent replicas: every rank's nodes over the slowest
    rank's time (max over ranks).  Returns (max_ms, node-updates/s)."""
    import torch

    world = 1
    if dist is not None:
        world = dist.get_world_size()
        t = torch.tensor([total_ms], device=device, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    return total_ms, nodes * steps * world / (total_ms / 1e3)


def time_steps(sim, torch, steps, per_launch=True):
    """Times `steps` single-step launches on the context's stream with CUDA events."""
    stream = sim.stream
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)] if per_launch else []
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    start.record(stream)
    for k in range(steps):
        if per_launch:
            ev[k][0].record(stream)
        rc = sim.step(1)
        if rc != 0:
            raise RuntimeError(f"sllbm_step returned {rc}")
        if per_launch:
            ev[k][1].record(stream)
    end.record(stream)
    torch.cuda.synchronize()
    total_ms = start.elapsed_time(end)
    kern = [a.elapsed_time(b) for a, b in ev] if per_launch else []
    return total_ms, kern


ELEM_BYTES = {"f64": 8, "f32": 4, "f16dev": 2, "bf16dev": 2}


def rel_l2(a, b):
    import numpy as np

    den = float(np.linalg.norm(b))
    return float(np.linalg.norm(a - b)) / den if den > 0 else float(np.linalg.norm(a - b))


def mixed_precision_block(S, torch, device, steps, every, hbm, alu):
    """FP64, FP32 and 16-bit deviation storage on the Ma 1.25 Taylor-Green workload, all from
    the same initial state, for `steps` steps, on the periodic mesh with ghost planes along z
    (one slab spanning the mesh, the headline's mode: the same states bit for bit as the
    ordinary periodic context, and no source box wraps around along z; the automatic kernel
    choice is the TMA-fed kernel there for FP32 and the 16-bit storages).  Per storage: median
    kernel time, node-updates/s, fraction of the HBM peak at its algorithmic bytes, and the
    relative L2 error against the FP64 GPU run of rho, u, T after the last step and of the
    E_k(t) and dissipation eps_s(t) + eps_c(t) curves sampled every `every` steps.  The
    FP32-arithmetic storages run a second time with compensated moment sums
    ("<storage>_comp", the same automatic kernel choice).  "periodic_wrap_timing" times the ordinary periodic
    context (boxes wrapping around along z) with the automatic choice (the generic kernel for
    16-bit storage at p = 3) and with the TMA-fed kernel forced."""
    import numpy as np

    w = I.WORKLOADS["tgv_64c_p3_ma125"]
    every = max(1, min(every, steps))
    chunks = steps // every
    out = {"workload": w.name, "note": w.note, "steps": chunks * every,
           "configured_steps": w.steps, "curve_every": every, "reference": "f64 (GPU)",
           "z_boundary": "ghost planes (one slab over the whole mesh)"}
    ref = None
    flops = algorithmic_flops_per_node(w.p)
    nodes = w.nodes
    for name in ("f64", "f32", "f16dev", "bf16dev", "f32_comp", "f16dev_comp", "bf16dev_comp"):
        st = name.split("_")[0]
        sim = S.Sim(S.Config(cells=w.cells, p=w.p, Ma=w.Ma, Re=w.Re, Pr=w.Pr, gamma=w.gamma,
                             courant=w.courant, pr_correction=w.pr_correction, storage=st,
                             slab=(0, w.cells[2])), device=device)
        if name.endswith("_comp"):
            S.sllbm_set_compensated(sim.ctx, True)
        sim.init_tgv()
        curve = [sim.diag()]
        kern = []
        for _ in range(chunks):
            _, k = time_steps(sim, torch, every)
            kern.extend(k)
            curve.append(sim.diag())
        # the interior planes (the ghost planes below and above hold copies)
        g = S.sllbm_slab_info(sim.ctx)[0]
        z = slice(g * w.p, (g + w.cells[2]) * w.p)
        rho, u, T = sim.moments()
        rho, u, T = rho[z].cpu().numpy(), u[:, z].cpu().numpy(), T[z].cpu().numpy()
        curve = np.array(curve)
        ek, eps = curve[:, 0], curve[:, 1] + curve[:, 2]
        kms = statistics.median(kern)
        bpn = 2 * 45 * 2 * ELEM_BYTES[st]
        rec = {"kernel_ms": kms, "value": nodes / (kms / 1e3), "unit": UNIT,
               "hbm_frac": bpn * nodes / (kms / 1e3) / 1e9 / hbm,
               "algorithmic_bytes_per_node": bpn, "step_kernel": int(S.sllbm_get_info(sim.ctx).step_kernel),
               "compensated_moments": name.endswith("_comp"),
               "roofline_alu": min_roofline(bpn, flops, nodes, kms, hbm,
                                            alu["fp64_tflops"] if st == "f64" else alu["fp32_tflops"]),
               "finite": bool(np.isfinite(T).all() and np.isfinite(rho).all())}
        if ref is None:
            ref = (rho, u, T, ek, eps, kms)
            rec["Ek_end"], rec["eps_end"] = float(ek[-1]), float(eps[-1])
        else:
            rec["rel_l2"] = {"rho": rel_l2(rho, ref[0]), "u": rel_l2(u, ref[1]),
                             "T": rel_l2(T, ref[2]), "Ek_curve": rel_l2(ek, ref[3]),
                             "eps_curve": rel_l2(eps, ref[4])}
            rec["speedup_vs_f64"] = ref[5] / kms
        out[name] = rec
        sim.close()
    # the ordinary periodic context, timing only
    wrap = {}
    for name in ("f32", "f16dev", "bf16dev", "f16dev_tma", "bf16dev_tma"):
        st = name.split("_")[0]
        sim = S.Sim(S.Config(cells=w.cells, p=w.p, Ma=w.Ma, Re=w.Re, Pr=w.Pr, gamma=w.gamma,
                             courant=w.courant, pr_correction=w.pr_correction, storage=st,
                             kernel=2 if name.endswith("_tma") else 0, nonfinite_check=True), device=device)
        sim.init_tgv()
        time_steps(sim, torch, 3, per_launch=False)
        _, kern = time_steps(sim, torch, every)
        kms = statistics.median(kern)
        bpn = 2 * 45 * 2 * ELEM_BYTES[st]
        wrap[name] = {"kernel_ms": kms, "value": nodes / (kms / 1e3), "unit": UNIT,
                      "hbm_frac": bpn * nodes / (kms / 1e3) / 1e9 / hbm, "step_kernel": int(sim.info.step_kernel),
                      "steps_timed": every, "status": int(sim.status())}
        sim.close()
    out["periodic_wrap_timing"] = wrap
    return out


def adjoint_block(S, torch, device, hbm, every=20, timed=20):
    """Reverse mode on the 16^3-cell, p = 3 Taylor-Green run (200 steps, checkpoints every
    20): gradients of the final E_k and of the final dissipation eps = eps_s + eps_c with
    respect to a seeded initial-velocity perturbation (amplitude 1e-3 U0) and mu_inf, in FP64,
    FP32 and FP32 with compensated moment sums ("f32_comp"), checked against central
    differences of the FP64 forward run; and the device time of one backward step
    (sllbm_adjoint_step)."""
    from paper_2012_05537_gb300 import adjoint as A

    w = I.WORKLOADS["tgv_16c_p3_adj"]
    cfgs = {st: S.Config(cells=w.cells, p=w.p, Ma=w.Ma, Re=w.Re, courant=w.courant, storage=st.split("_")[0])
            for st in ("f64", "f32", "f32_comp")}
    rho, u, T = A.tgv_fields(cfgs["f64"], device=device)
    out = {"workload": w.name, "note": w.note, "steps": w.steps, "checkpoint_every": every}
    grads = {}
    for st, cfg in cfgs.items():
        sim = S.Sim(cfg, device=device)
        if st == "f32_comp":
            S.sllbm_set_compensated(sim.ctx, True)
        U0 = float(sim.info.U0)
        du = torch.as_tensor(1e-3 * U0 * I.noise(tuple(u.shape), 0), device=device)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        grads[st] = A.diagnostic_gradients(sim, rho, u, T, du, w.steps, every)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        # device time of the backward step alone
        state = sim.raw_state().clone()
        lam = torch.empty_like(state)
        S.sllbm_ek_adjoint(sim.ctx, state.data_ptr(), lam.data_ptr())
        spare = torch.empty_like(lam)
        dmu = torch.zeros(1, dtype=torch.float64, device=device)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        S.sllbm_adjoint_step(sim.ctx, state.data_ptr(), lam.data_ptr(), spare.data_ptr(), dmu.data_ptr())
        torch.cuda.synchronize()
        ev[0].record(sim.stream)
        for _ in range(timed):
            S.sllbm_adjoint_step(sim.ctx, state.data_ptr(), lam.data_ptr(), spare.data_ptr(), dmu.data_ptr())
        ev[1].record(sim.stream)
        torch.cuda.synchronize()
        ms = ev[0].elapsed_time(ev[1]) / timed
        _, fwd = time_steps(sim, torch, timed)
        bpn = 3 * 90 * ELEM_BYTES[st.split("_")[0]]  # read state and lambda, write lambda
        out[st] = {"gradients": grads[st], "wall_s_forward_and_backward": wall,
                   "adjoint_step_ms": ms, "forward_step_ms": statistics.median(fwd),
                   "adjoint_node_updates_per_s": sim.nodes / (ms / 1e3),
                   "adjoint_hbm_frac_of_min_bytes": bpn * sim.nodes / (ms / 1e3) / 1e9 / hbm,
                   "adjoint_min_bytes_per_node": bpn}
        sim.close()
    sim = S.Sim(cfgs["f64"], device=device)
    mu0 = float(sim.info.mu_inf)
    du = torch.as_tensor(1e-3 * float(sim.info.U0) * I.noise(tuple(u.shape), 0), device=device)

    def diag(e=0.0, mu=mu0):
        sim.set_mu_inf(mu)
        sim.init_fields(rho, u + e * du, T)
        sim.step(w.steps)
        d = sim.diag()
        return d[0], d[1] + d[2]

    def central(fun, x, h):
        d1 = [(a - b) / (2 * h) for a, b in zip(fun(x + h), fun(x - h))]
        d2 = [(a - b) / h for a, b in zip(fun(x + h / 2), fun(x - h / 2))]
        return [(4 * b - a) / 3 for a, b in zip(d1, d2)]

    de = central(lambda e: diag(e=e), 0.0, 1.0)
    dm = central(lambda m: diag(mu=m), mu0, 1e-2 * mu0)
    fd = {"dEk_deps": de[0], "dEk_dmu_inf": dm[0], "deps_deps": de[1], "deps_dmu_inf": dm[1]}
    sim.close()
    out["finite_differences_f64"] = fd
    for st in cfgs:
        out[st]["rel_err_vs_fd"] = {k: abs(grads[st][k] - v) / abs(v) for k, v in fd.items()}
        if st != "f64":
            out[st]["rel_err_vs_f64"] = {k: abs(grads[st][k] - grads["f64"][k]) / abs(grads["f64"][k])
                                         for k in fd}
    out["target_rel_err"] = 1e-4
    return out


def golden_curves(name):
    """(steps, E_k, eps) rows of a stored oracle curve file under tests/golden (as text), or
    None if it is absent."""
    import numpy as np

    path = os.path.join(ROOT, "tests", "golden", f"{name}_curves.txt")
    if not os.path.exists(path):
        return None
    rows = np.array([[float(x) for x in line.split()] for line in open(path)
                     if line.strip() and not line.startswith("#")])
    return rows[:, 0].astype(int), rows[:, 1], rows[:, 2] + rows[:, 3]


def long_run_block(S, torch, device, steps, every):
    """The throughput mesh (128^3 nodes, Courant 4) with the Prandtl term on, in FP32 and FP64
    for `steps` steps from the Taylor-Green state: kinetic energy E_k(t) and dissipation
    eps(t) = eps_s + eps_c every `every` steps, the relative L2 of the FP32 curves against the
    FP64 ones, and of both against the FP64 oracle's run of the same flow on 16^3 cells
    (64^3 nodes) at the same time step (tests/golden/tgv_16c_p4_c2_curves.txt; a comparison
    across resolutions, at the steps the file holds)."""
    import numpy as np

    w = I.WORKLOADS["tgv_32c_p4"]
    gold = golden_curves("tgv_16c_p4_c2")
    out = {"workload": w.name, "steps": steps, "every": every, "pr_correction": True,
           "oracle_curves": "tgv_16c_p4_c2 (16^3 cells, p = 4, same dt, Prandtl term on)"}
    curves = {}
    for st in ("f64", "f32"):
        sim = S.Sim(S.Config(cells=w.cells, p=w.p, Ma=w.Ma, Re=w.Re, Pr=w.Pr, gamma=w.gamma,
                             courant=w.courant, pr_correction=True, storage=st), device=device)
        sim.init_tgv()
        rows = [[0] + list(sim.diag())]
        kern = []
        for k in range(every, steps + 1, every):
            _, kk = time_steps(sim, torch, every, per_launch=(k == every))
            kern.extend(kk)
            rows.append([k] + list(sim.diag()))
        rows = np.array(rows)
        curves[st] = (rows[:, 0].astype(int), rows[:, 1], rows[:, 2] + rows[:, 3])
        out[st] = {"kernel_ms": statistics.median(kern), "step_kernel": int(S.sllbm_get_info(sim.ctx).step_kernel),
                   "Ek_end": float(rows[-1, 1]), "eps_end": float(rows[-1, 2] + rows[-1, 3]),
                   "finite": bool(np.isfinite(rows).all()),
                   "eps_peak_step": int(rows[np.argmax(rows[:, 2] + rows[:, 3]), 0])}
        sim.close()
    out["f32_vs_f64_rel_l2"] = {"Ek_curve": rel_l2(curves["f32"][1], curves["f64"][1]),
                                "eps_curve": rel_l2(curves["f32"][2], curves["f64"][2])}
    if gold is not None:
        ks, ek_o, eps_o = gold
        for st in ("f64", "f32"):
            idx = {int(k): n for n, k in enumerate(curves[st][0])}
            sel = [n for n, k in enumerate(ks) if int(k) in idx]
            if not sel:
                continue
            at = [idx[int(ks[n])] for n in sel]
            out[st]["vs_oracle_16c"] = {"steps_compared": int(ks[sel[-1]]),
                                        "Ek_curve_rel_l2": rel_l2(curves[st][1][at], ek_o[sel]),
                                        "eps_curve_rel_l2": rel_l2(curves[st][2][at], eps_o[sel])}
    return out


def decomposed_block(S, torch, device, w, parts=2, steps=50, kernel=1):
    """The workload's mesh as `parts` z-slabs on this one GPU, advanced with one halo
    exchange per step (device copies between the slab contexts), against the undivided mesh
    on the same kernel (generic or TMA-fed): step times with the exchange before the step and overlapped
    with it (a second stream), the exchange alone, the halo bytes moved per step, and whether
    the slabs end bit for bit equal to the whole mesh."""
    import dataclasses

    from paper_2012_05537_gb300 import decomp as D

    cfg = S.Config(cells=w.cells, p=w.p, Ma=w.Ma, Re=w.Re, Pr=w.Pr, gamma=w.gamma, courant=w.courant,
                   storage="f32", kernel=kernel)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    whole = S.Sim(cfg, device=device)
    whole.init_tgv()
    whole.step(3)
    torch.cuda.synchronize()
    ev[0].record(whole.stream)
    whole.step(steps)
    ev[1].record(whole.stream)
    torch.cuda.synchronize()
    whole_ms = ev[0].elapsed_time(ev[1]) / steps
    whole.step(3 + steps)  # the slabs' overlapped run below adds as many steps
    ref = whole.populations()
    whole.close()
    steppers = []
    for r in range(parts):
        sim = S.Sim(dataclasses.replace(cfg, slab=D.slab_bounds(w.cells[2], parts, r)), device=device)
        sim.init_tgv()
        steppers.append(D.SlabStepper(sim))
    D.step_local(steppers, 3)
    torch.cuda.synchronize()
    ev[0].record(steppers[0].sim.stream)
    D.step_local(steppers, steps)
    ev[1].record(steppers[0].sim.stream)
    torch.cuda.synchronize()
    slab_ms = ev[0].elapsed_time(ev[1]) / steps
    ev[0].record(steppers[0].sim.stream)
    for _ in range(steps):
        D.exchange_local(steppers)
    ev[1].record(steppers[0].sim.stream)
    torch.cuda.synchronize()
    exch_ms = ev[0].elapsed_time(ev[1]) / steps
    # the exchange on a second stream, overlapped with the tiles that read no ghost cell
    comm = D.step_local_overlapped(steppers, 3)
    torch.cuda.synchronize()
    ev[0].record(steppers[0].sim.stream)
    D.step_local_overlapped(steppers, steps, comm)
    ev[1].record(steppers[0].sim.stream)
    torch.cuda.synchronize()
    overlap_ms = ev[0].elapsed_time(ev[1]) / steps
    # (the exchange-only loop leaves the state unchanged: the whole mesh and the slabs both
    # ran 2 (3 + steps) steps)
    g, p = steppers[0].ghost, w.p
    inner = [st.sim.populations()[:, :, g * p:(g + st.sim.cfg.slab[1]) * p] for st in steppers]
    equal = bool(torch.equal(torch.cat(inner, dim=2), ref))
    # pack + unpack of both sides; beside it what whole ghost widths for every velocity moved
    halo = sum(2 * (st.sizes["send_low"] + st.sizes["send_high"]) for st in steppers)
    plane = 2 * 45 * ELEM_BYTES["f32"] * w.N[0] * w.N[1] // 45
    halo_full = sum(4 * 45 * g_ * p_ * plane for g_, p_ in [(st.ghost, w.p) for st in steppers])
    for st in steppers:
        st.sim.close()
    nodes = w.nodes
    return {"workload": w.name, "kernel": "TMA-fed" if kernel == 2 else "generic", "parts": parts,
            "ghost_cells": g, "steps": steps,
            "whole_mesh_ms_per_step": whole_ms, "slabs_ms_per_step": slab_ms,
            "slabs_overlapped_ms_per_step": overlap_ms,
            "exchange_ms_per_step": exch_ms, "halo_copy_bytes_per_step": halo,
            "halo_copy_bytes_per_step_whole_ghost_width": halo_full,
            "slabs_value": nodes / (slab_ms / 1e3), "whole_value": nodes / (whole_ms / 1e3),
            "bit_equal_to_whole_mesh": equal,
            "note": "one GPU: the slab contexts exchange by device copies; across GPUs the same "
                    "halos move through torch.distributed point-to-point"}


def batch_block(S, torch, device, count, steps, streams=16, seed=0):
    """`count` Taylor-Green instances of uneven size, order and parameters (seeded mix:
    cells 8^3..24^3, p in {2,3,4}, Ma 0.3..1.25, Re 400..1600, Courant 1..8), FP32, `steps`
    steps each: aggregate node-updates/s run one by one (default kernels, then autotuned
    kernels) against one graph launch per two steps of all instances."""
    from paper_2012_05537_gb300 import batch as BT

    insts = I.batch_instances(count, seed)
    sims = BT.make_instances(insts, device=device)
    nodes = sum(s.nodes for s in sims)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]

    def one_by_one():
        torch.cuda.synchronize()
        ms = 0.0
        for s in sims:
            ev[0].record(s.stream)
            s.step(steps)
            ev[1].record(s.stream)
            torch.cuda.synchronize()
            ms += ev[0].elapsed_time(ev[1])
        return ms

    for s in sims:
        s.step(2)  # warm-up: tables, descriptors, function attributes
    default_ms = one_by_one()
    variants = [s.autotune(3)[0] for s in sims]
    tuned_ms = one_by_one()
    bt = BT.Batch(sims, streams=streams)
    bt.step(2)
    torch.cuda.synchronize()
    ev[0].record(bt.stream)
    bt.step(steps if steps % 2 == 0 else steps + 1)
    ev[1].record(bt.stream)
    torch.cuda.synchronize()
    batch_ms = ev[0].elapsed_time(ev[1])
    bsteps = steps if steps % 2 == 0 else steps + 1
    bt.close()
    # one persistent launch per order and step, tile shape per order autotuned
    pt = BT.Batch(sims, autotune_steps=4, persistent=True)
    shapes = pt.shapes()
    pt.step(2)
    torch.cuda.synchronize()
    ev[0].record(pt.stream)
    pt.step(bsteps)
    ev[1].record(pt.stream)
    torch.cuda.synchronize()
    pers_ms = ev[0].elapsed_time(ev[1])
    pt.close()
    finite = 0
    for s in sims:
        _, _, T = s.moments()
        finite += bool(torch.isfinite(T).all().item())
    for s in sims:
        s.close()
    return {"instances": count, "seed": seed, "steps": steps, "nodes_per_step": nodes,
            "streams": streams, "configured_steps": 500,
            "one_by_one_default": {"ms": default_ms, "value": nodes * steps / (default_ms / 1e3)},
            "one_by_one_autotuned": {"ms": tuned_ms, "value": nodes * steps / (tuned_ms / 1e3)},
            "batched_graph": {"ms": batch_ms, "value": nodes * bsteps / (batch_ms / 1e3)},
            "persistent_graph": {"ms": pers_ms, "value": nodes * bsteps / (pers_ms / 1e3),
                                 "tile_shape_per_order": {str(k): v for k, v in shapes.items()}},
            "speedup_vs_one_by_one_default": (nodes * bsteps / batch_ms) / (nodes * steps / default_ms),
            "persistent_speedup_vs_one_by_one_default": (nodes * bsteps / pers_ms) / (nodes * steps / default_ms),
            "variants_chosen": {str(v): variants.count(v) for v in sorted(set(variants))},
            "instances_finite_at_end": finite, "unit": UNIT}


def run_mine(args, rank, world, local):
    import torch

    from paper_2012_05537_gb300 import build as B
    from paper_2012_05537_gb300 import sllbm as S

    if not torch.cuda.is_available():
        raise RuntimeError("bench.py needs a CUDA device")
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0:
        B.build()
    if dist is not None:
        dist.barrier()
    S.load()
    alu = alu_peaks(S)
    w = I.WORKLOADS[args.workload]
    storage = args.storage or w.storage
    # The periodic mesh with ghost planes along z: one slab spanning all z-cells, whose steps
    # refresh its ghost planes in place (sllbm_halo_periodic, one small launch) so that no
    # source box wraps around along z; bit for bit the same states as the ordinary periodic
    # context (tests/test_gpu_decomp.py), which "--periodic-z wrap" times instead.
    ghost = args.periodic_z == "ghost"
    cfg = S.Config(cells=w.cells, p=w.p, Ma=w.Ma, Re=w.Re, Pr=w.Pr, gamma=w.gamma,
                   courant=w.courant, pr_correction=w.pr_correction or args.pr, storage=storage,
                   slab=(0, w.cells[2]) if ghost else None, kernel=args.kernel)
    sim = S.Sim(cfg, device=f"cuda:{local}")
    if args.compensated:
        sim.set_compensated(True)
    sim.init_tgv()
    for _ in range(max(3, args.warmup)):
        sim.step(1)
    torch.cuda.synchronize()

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = sim.launches()
    total_ms, kern = time_steps(sim, torch, args.steps)
    launches = sim.launches() - launches0
    torch.cuda.synchronize()
    nodes = w.nodes  # the mesh's nodes (a slab's buffers also hold its ghost planes)
    total_ms, value = replica_throughput(total_ms, nodes, args.steps, dist, device=f"cuda:{local}")
    if dist is not None:
        dist.barrier()
    clk = clocks.stop()
    clk["covers"] = "the headline's timed region (nvidia-smi every 200 ms, from 0.3 s before it)"
    _, _, T = sim.moments()
    finite = bool(torch.isfinite(T).all().item())

    elem = ELEM_BYTES[storage]
    bytes_per_node = 2 * 45 * 2 * elem  # read + write of f and g
    kern_avg_ms = statistics.mean(kern)
    hbm, peak_src = measured_peaks()
    achieved = bytes_per_node * nodes / (kern_avg_ms / 1e3) / 1e9
    traffic = profiled_traffic(w.name, storage, "tma" if sim.info.step_kernel == 2 else "generic",
                               ("_ghostz" if ghost else "") + ("_pr" if args.pr else "") +
                               ("_kc" if args.compensated else ""))

    # end to end through the C ABI with host buffers: every step copies a state from pinned
    # host memory to the device, advances it one step and copies the result back.  Headline:
    # a stream of independent states through sllbm_run_host_many (the copies of neighbouring
    # states overlap, in both directions); beside it the same one state at a time
    # (sllbm_run_host, copy in, step, copy out, synchronise).
    # The states here are those of the ordinary periodic context (the call a user makes with
    # host buffers): a slab's state would also carry its ghost planes across the host link.
    e2e = None
    if args.e2e_steps > 0:
        sime = S.Sim(dataclasses.replace(cfg, slab=None), device=f"cuda:{local}") if ghost else sim
        if args.compensated and sime is not sim:
            sime.set_compensated(True)
        if ghost:
            sime.init_tgv()
        nb = int(sime.info.pop_bytes)
        host_in = torch.empty(nb, dtype=torch.uint8).pin_memory()
        host_outs = [torch.empty(nb, dtype=torch.uint8).pin_memory() for _ in range(3)]
        host_in.copy_(sime.raw_state().view(torch.uint8).reshape(-1).cpu())
        sime.run_host(host_in, host_outs[0], 1)
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            sime.run_host(host_in, host_outs[0], 1)
        el_seq = time.perf_counter() - t0
        ins = [host_in] * args.e2e_steps
        outs = [host_outs[k % 3] for k in range(args.e2e_steps)]
        sime.run_host_many(ins[:3], outs[:3], 1)
        t0 = time.perf_counter()
        sime.run_host_many(ins, outs, 1)
        el = time.perf_counter() - t0
        e2e = {"value": nodes * args.e2e_steps * world / el, "unit": UNIT,
               "h2d_bytes_per_step": nb, "d2h_bytes_per_step": nb,
               "steps": args.e2e_steps, "step_kernel": int(sime.info.step_kernel),
               "mode": "independent states streamed through sllbm_run_host_many (copies overlapped), "
                       "ordinary periodic context",
               "sequential": {"value": nodes * args.e2e_steps * world / el_seq, "unit": UNIT,
                              "mode": "one state at a time through sllbm_run_host"}}
        if sime is not sim:
            sime.close()

    variants = {}
    if not args.no_variants and rank == 0 and ghost:
        # the same workload on the ordinary periodic context (source boxes wrap around along z)
        simw = S.Sim(dataclasses.replace(cfg, slab=None), device=f"cuda:{local}")
        simw.init_tgv()
        simw.step(3)
        nw = 50
        tw, kw = time_steps(simw, torch, nw)
        variants["periodic_wrap"] = {"value": nodes * nw / (tw / 1e3), "ms_per_step": tw / nw,
                                     "kernel_ms": statistics.mean(kw), "step_kernel": int(simw.info.step_kernel),
                                     "hbm_frac": bytes_per_node * nodes / (statistics.mean(kw) / 1e3) / 1e9 / hbm,
                                     "steps": nw}
        simw.close()
    if not args.no_variants and rank == 0 and storage != "f64" and not args.pr and not args.compensated:
        # the same workload with compensated moment sums (the same context kind and kernel choice)
        simc = S.Sim(cfg, device=f"cuda:{local}")
        S.sllbm_set_compensated(simc.ctx, True)
        simc.init_tgv()
        simc.step(3)
        nc = 50
        tc, kc = time_steps(simc, torch, nc)
        kc_ms = statistics.mean(kc)
        variants["compensated"] = {"value": nodes * nc / (tc / 1e3), "ms_per_step": tc / nc, "kernel_ms": kc_ms,
                                   "step_kernel": int(S.sllbm_get_info(simc.ctx).step_kernel),
                                   "kernel_time_vs_plain": kc_ms / kern_avg_ms,
                                   "hbm_frac": bytes_per_node * nodes / (kc_ms / 1e3) / 1e9 / hbm, "steps": nc}
        simc.close()
    if not args.no_variants and rank == 0 and storage == "f32":
        # FP64 storage/arithmetic on the same workload (FP64-ALU bound on this part)
        sim64 = S.Sim(S.Config(cells=w.cells, p=w.p, Ma=w.Ma, Re=w.Re, Pr=w.Pr, gamma=w.gamma,
                               courant=w.courant, pr_correction=w.pr_correction, storage="f64"),
                      device=f"cuda:{local}")
        sim64.init_tgv()
        sim64.step(3)
        n64 = 20
        t64, k64 = time_steps(sim64, torch, n64)
        k64_ms = statistics.mean(k64)
        flops = algorithmic_flops_per_node(w.p)
        variants["f64"] = {"value": nodes * n64 / (t64 / 1e3), "ms_per_step": t64 / n64,
                           "kernel_ms": k64_ms,
                           "hbm_gbs_equiv": 2 * 45 * 2 * 8 * nodes / (k64_ms / 1e3) / 1e9,
                           "roofline": {"bound": "alu", "achieved": flops * nodes / (k64_ms / 1e3) / 1e12,
                                        "peak": alu["fp64_tflops"], "unit": "TFLOP/s",
                                        "frac": flops * nodes / (k64_ms / 1e3) / 1e12 / alu["fp64_tflops"],
                                        "peak_source": "measured (sllbm_fma_peak, FP64 FMA)",
                                        "algorithmic_flops_per_node": flops},
                           "steps": n64}
        sim64.close()
        # the paper's Taylor-Green setting: the Prandtl term of App. D on
        simpr = S.Sim(S.Config(cells=w.cells, p=w.p, Ma=w.Ma, Re=w.Re, Pr=w.Pr, gamma=w.gamma,
                               courant=w.courant, pr_correction=True, storage=storage),
                      device=f"cuda:{local}")
        simpr.init_tgv()
        simpr.step(3)
        npr = 50
        tpr, kpr = time_steps(simpr, torch, npr)
        kpr_ms = statistics.mean(kpr)
        variants["pr"] = {"pr_correction": True, "Pr": w.Pr, "value": nodes * npr / (tpr / 1e3),
                          "ms_per_step": tpr / npr, "kernel_ms": kpr_ms,
                          "step_kernel": int(simpr.info.step_kernel),
                          "hbm_frac": bytes_per_node * nodes / (kpr_ms / 1e3) / 1e9 / hbm, "steps": npr}
        simpr.close()
        # the same on the TMA-fed kernel (as fast as the generic one with ghost planes, slower
        # with boxes wrapping along z: the automatic choice keeps the term on the generic kernel)
        for gname, gslab in (("ghost", (0, w.cells[2])), ("wrap", None)):
            simt = S.Sim(S.Config(cells=w.cells, p=w.p, Ma=w.Ma, Re=w.Re, Pr=w.Pr, gamma=w.gamma,
                                  courant=w.courant, pr_correction=True, storage=storage, kernel=2,
                                  slab=gslab), device=f"cuda:{local}")
            simt.init_tgv()
            simt.step(3)
            _, kt = time_steps(simt, torch, npr)
            variants["pr"][f"tma_kernel_ms_{gname}"] = statistics.mean(kt)
            simt.close()
    if not args.no_variants and rank == 0 and args.batch_steps > 0:
        variants["batched"] = batch_block(S, torch, f"cuda:{local}", 64, args.batch_steps)
    if not args.no_variants and rank == 0 and not args.no_adjoint:
        variants["adjoint"] = adjoint_block(S, torch, f"cuda:{local}", hbm)
    if not args.no_variants and rank == 0 and storage == "f32":
        variants["decomposed"] = {"generic": decomposed_block(S, torch, f"cuda:{local}", w, kernel=1),
                                  "tma": decomposed_block(S, torch, f"cuda:{local}", w, kernel=2)}
    if not args.no_variants and rank == 0 and args.mixed_steps > 0:
        variants["mixed"] = mixed_precision_block(S, torch, f"cuda:{local}", args.mixed_steps,
                                                  args.mixed_every, hbm, alu)
    if not args.no_variants and rank == 0 and args.long_steps > 0:
        variants["long_run"] = long_run_block(S, torch, f"cuda:{local}", args.long_steps, args.long_every)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, cores, sample = oracle_sample_rate(w)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": storage, "data": "synthetic",
            "config": {"workload": w.name, "cells": list(w.cells), "p": w.p,
                       "nodes": nodes, "Ma": w.Ma, "Re": w.Re, "courant": w.courant,
                       "pr_correction": bool(w.pr_correction or args.pr),
                       "compensated_moments": bool(args.compensated),
                       "dt": sim.dt, "storage": storage,
                       "z_boundary": ("ghost planes: the mesh as one periodic z-slab (sllbm_create_slab over "
                                      "all cells), refreshed in place before each step by sllbm_halo_periodic "
                                      "inside sllbm_step" if ghost else "source boxes wrap around (periodic images)"),
                       "l2": f"inputs larger than L2 ({sim.info.pop_bytes / 1e6:.0f} MB per buffer)",
                       "parallelism": f"replicas x{world}",
                       "population_updates_per_s": value * 45},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                         "frac": achieved / hbm, "traffic": traffic,
                         "peak_source": peak_src, "kernel_ms": kern_avg_ms,
                         "algorithmic_bytes_per_node": bytes_per_node},
            "roofline_alu": min_roofline(bytes_per_node, algorithmic_flops_per_node(w.p), nodes, kern_avg_ms, hbm,
                                         alu["fp64_tflops"] if storage == "f64" else alu["fp32_tflops"]),
            "alu_peaks": alu,
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clk,
            "finite": finite,
        }
        if variants:
            line["variants"] = variants
        print(json.dumps(line), flush=True)
    sim.close()
    if dist is not None:
        dist.destroy_process_group()


def main():
    args = parse_args()
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    run_mine(args, rank, world, local)


if __name__ == "__main__":
    main()
