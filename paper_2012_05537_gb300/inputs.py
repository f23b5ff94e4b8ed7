"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle runs.

Holds workload definitions (mesh, order, flow parameters) and seeded random-number
helpers only; none of the method's arithmetic (no equilibrium, no streaming, no
moments) lives here, so that the CUDA path and the oracle stay independent.

The workloads stand in for the paper's compressible Taylor-Green vortex runs
(Sec. III.C): periodic [0, 2 pi]^3, constant-temperature initial condition, Re = 1600,
Pr = 0.7, gamma = 1.4, time step given as a Courant number C = dt max|xi| / (L/N).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class Workload:
    name: str
    cells: tuple
    p: int
    Ma: float
    Re: float
    courant: float
    steps: int
    storage: str
    Pr: float = 0.7
    gamma: float = 1.4
    pr_correction: bool = False
    note: str = ""

    @property
    def N(self):
        return tuple(c * self.p for c in self.cells)

    @property
    def nodes(self) -> int:
        n = self.N
        return n[0] * n[1] * n[2]

    @property
    def U0(self) -> float:
        return self.Ma * math.sqrt(self.gamma)

    @property
    def mu_inf(self) -> float:
        return self.U0 / self.Re

    def dt(self, max_xi: float = math.sqrt(15.0)) -> float:
        return self.courant * (2 * math.pi / max(self.N)) / max_xi


WORKLOADS = {
    # small case the oracle finishes in seconds
    "tgv_8c_p3": Workload("tgv_8c_p3", (8, 8, 8), 3, 0.5, 1600.0, 2.0, 50, "f64",
                          note="8^3 cells, p=3 (24^3 nodes), Ma 0.5, C=2, 50 steps"),
    # the throughput workload (about 94 M f-populations)
    "tgv_32c_p4": Workload("tgv_32c_p4", (32, 32, 32), 4, 0.5, 1600.0, 4.0, 2000, "f32",
                           note="32^3 cells, p=4 (128^3 nodes), Ma 0.5, C=4"),
    # profiling size: same resolution per cell as tgv_32c_p4, buffers (318 MB) > L2
    "tgv_24c_p4": Workload("tgv_24c_p4", (24, 24, 24), 4, 0.5, 1600.0, 4.0, 2000, "f32",
                           note="24^3 cells, p=4 (96^3 nodes), Ma 0.5, C=4"),
    # oracle-size companion of the throughput workload (curves)
    "tgv_16c_p4": Workload("tgv_16c_p4", (16, 16, 16), 4, 0.5, 1600.0, 4.0, 2000, "f64",
                           note="16^3 cells, p=4 (64^3 nodes)"),
    # oracle-size companion of the throughput workload's long run: the same time step as
    # tgv_32c_p4 (Courant 4 on 128^3 nodes is Courant 2 on 64^3), 2000 steps (t* = 60), with the
    # Prandtl term the paper's Taylor-Green runs use (Pr 0.7, App. D)
    "tgv_16c_p4_c2": Workload("tgv_16c_p4_c2", (16, 16, 16), 4, 0.5, 1600.0, 2.0, 2000, "f64",
                              pr_correction=True,
                              note="16^3 cells, p=4 (64^3 nodes), Ma 0.5, C=2, Pr term on, 2000 steps"),
    # shocklet case at higher Mach (mixed-precision comparison).  BGK at Ma 1.25 is not stable
    # at Courant 2 and above on this mesh (tau - 1/2 < 0.03 once shocklets form); Courant 1
    # matches the time step the paper uses for this Mach number (dt* = 0.009 at 256^3 points).
    "tgv_64c_p3_ma125": Workload("tgv_64c_p3_ma125", (64, 64, 64), 3, 1.25, 1600.0, 1.0, 5000,
                                 "f32", note="64^3 cells, p=3 (192^3 nodes), Ma 1.25, C=1"),
    # reverse-mode workload: gradients of the final kinetic energy through 200 steps
    "tgv_16c_p3_adj": Workload("tgv_16c_p3_adj", (16, 16, 16), 3, 0.5, 1600.0, 2.0, 200, "f32",
                               note="16^3 cells, p=3 (48^3 nodes), Ma 0.5, C=2, 200 steps"),
    # profiling size of the Ma 1.25 workload's kernel (same cells, order and parameters;
    # 318 MB per FP32 buffer, larger than L2)
    "tgv_32c_p3_ma125": Workload("tgv_32c_p3_ma125", (32, 32, 32), 3, 1.25, 1600.0, 1.0, 200, "f32",
                                 note="32^3 cells, p=3 (96^3 nodes), Ma 1.25, C=1"),
    # large mesh: byte offsets of a buffer beyond 32 bits (FP32 20 GB, FP64 41 GB per buffer)
    "tgv_96c_p4": Workload("tgv_96c_p4", (96, 96, 96), 4, 0.5, 1600.0, 4.0, 1, "f32",
                           note="96^3 cells, p=4 (384^3 nodes), Ma 0.5, C=4 (first step)"),
    # the same mesh at Courant 8 (departures 2.7 cells away): first-step parity only
    "tgv_64c_p3_ma125_c8": Workload("tgv_64c_p3_ma125_c8", (64, 64, 64), 3, 1.25, 1600.0, 8.0, 1,
                                    "f32", note="64^3 cells, p=3, Ma 1.25, C=8 (one step)"),
}


def rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(seed)


def random_fields(shape, seed: int, rho=(0.7, 1.4), u_amp=0.6, T=(0.7, 1.4)):
    """Independent uniform random rho, u (3 components), T at every node (FP64)."""
    g = rng(seed)
    r = g.uniform(rho[0], rho[1], shape)
    u = g.uniform(-u_amp, u_amp, (3,) + tuple(shape))
    t = g.uniform(T[0], T[1], shape)
    return r, u, t


def smooth_fields(shape, seed: int, modes: int = 3, rho_amp=0.1, u_amp=0.4, T_amp=0.1):
    """Smooth periodic random fields on [0, 2 pi)^3 sampled at the given node
    coordinates' index grid (uniform spacing), from a few random Fourier modes."""
    g = rng(seed)
    nz, ny, nx = shape
    z, y, x = np.meshgrid(*(np.arange(n) * 2 * np.pi / n for n in (nz, ny, nx)), indexing="ij")

    def one(amp):
        out = np.zeros(shape)
        for _ in range(modes):
            k = g.integers(-2, 3, 3)
            ph = g.uniform(0, 2 * np.pi)
            out += g.uniform(-amp, amp) * np.cos(k[0] * x + k[1] * y + k[2] * z + ph)
        return out

    r = 1.0 + one(rho_amp)
    u = np.stack([one(u_amp) for _ in range(3)])
    t = 1.0 + one(T_amp)
    return r, u, t


def noise(shape, seed: int) -> np.ndarray:
    """Standard normal array used to push populations away from equilibrium."""
    return rng(seed).standard_normal(shape)


def sample_nodes(nodes: int, count: int, seed: int) -> np.ndarray:
    """Sorted distinct node indices, always including the first and the last node."""
    g = rng(seed)
    pick = g.choice(nodes, size=min(count, nodes), replace=False)
    pick = np.unique(np.concatenate([pick, [0, nodes - 1]]))
    return pick.astype(np.int64)


@dataclass(frozen=True)
class Instance:
    """One member of a batch of independent Taylor-Green runs (cube of cells)."""
    cells: tuple
    p: int
    Ma: float
    Re: float
    courant: float

    @property
    def nodes(self) -> int:
        return (self.cells[0] * self.p) * (self.cells[1] * self.p) * (self.cells[2] * self.p)


def batch_instances(count: int = 64, seed: int = 0):
    """Seeded mix of Taylor-Green instances of uneven size, order and parameters: cells per
    direction uniform in 8..24 (cubes), p in {2, 3, 4}, Ma uniform in [0.3, 1.25], Re uniform
    in [400, 1600], Courant number uniform in [1, 8]."""
    g = rng(seed)
    out = []
    for _ in range(count):
        n = int(g.integers(8, 25))
        p = int(g.choice([2, 3, 4]))
        out.append(Instance(cells=(n, n, n), p=p, Ma=float(g.uniform(0.3, 1.25)),
                            Re=float(g.uniform(400.0, 1600.0)), courant=float(g.uniform(1.0, 8.0))))
    return out
