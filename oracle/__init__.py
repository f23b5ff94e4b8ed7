"""FP64 CPU oracle of the SLLBM time step (arXiv:2012.05537) -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference legs of
``bench.py`` may import this package.  The CUDA library never imports it and shares
no code with it.  The arithmetic lives in ``sllbm_oracle.c`` (plain C, OpenMP over
nodes); this module only compiles that file with gcc and marshals numpy arrays.

Each wrapper cites the passage of the paper its C function follows:

* :func:`velset` -- Sec. II.B / Fig. 2, degree-9 cubature with 45 abscissae;
* :func:`glc`, :func:`lagrange`, :func:`lagrange_deriv`, :func:`quad_weights` --
  the Gauss-Lobatto-Chebyshev support points and Lagrange basis of Eq. (interpolation);
* :func:`feq` -- Eq. (discreteEquilibrium) with App. A moments and App. B Hermite tensors;
* :func:`stream` -- the semi-Lagrangian streaming step of Sec. II.A;
* :func:`collide` -- Eq. (LBM) collision with the App. D Prandtl correction;
* :func:`step` -- stream then collide, the stored state being post-collision;
* :func:`moments` -- Eq. (moments);
* :func:`tgv_fields` -- Sec. III.C Taylor-Green initial fields;
* :func:`diag` -- the E_k, eps_s, eps_c definitions of Sec. III.C;
* :func:`stream_adjoint`, :func:`collide_vjp`, :func:`step_adjoint`, :func:`ek_grad`,
  :func:`diag_grad`, :func:`init_fields_vjp` -- reverse mode of the above (no counterpart
  in the paper):
  the literal transpose of the streaming, and finite-difference (Richardson-extrapolated)
  Jacobians of the collision and the equilibrium initialisation.

Parity unpinned: agreement of the 45-point set with the paper's own (unprinted) table.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sllbm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

Q = 45


def build(force: bool = False) -> str:
    """Compile ``sllbm_oracle.c`` into ``oracle/_build/liboracle.so`` with gcc."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=gnu11", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
           _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            lib.orc_velset.argtypes = [dp, dp]
            lib.orc_velset.restype = ctypes.c_int
            lib.orc_glc.argtypes = [ctypes.c_int, dp]
            lib.orc_lagrange.argtypes = [ctypes.c_int, ctypes.c_double, dp]
            lib.orc_lagrange_deriv.argtypes = [ctypes.c_int, ctypes.c_double, dp]
            lib.orc_quad_weights.argtypes = [ctypes.c_int, dp]
            lib.orc_sutherland.argtypes = [ctypes.c_double]
            lib.orc_sutherland.restype = ctypes.c_double
            lib.orc_feq.argtypes = [dp, dp, ctypes.c_int, ctypes.c_double, dp, ctypes.c_double, dp]
            cfgp = ctypes.POINTER(_Cfg)
            lib.orc_stream.argtypes = [cfgp, ctypes.c_int, ctypes.c_int, dp, dp, dp]
            lib.orc_collide.argtypes = [cfgp, dp]
            lib.orc_step.argtypes = [cfgp, dp, dp, ctypes.c_int]
            lib.orc_moments.argtypes = [cfgp, dp, dp, dp, dp]
            lib.orc_init_fields.argtypes = [cfgp, dp, dp, dp, dp]
            lib.orc_tgv_fields.argtypes = [cfgp, ctypes.c_double, ctypes.c_double,
                                           ctypes.c_double, ctypes.c_double, dp, dp, dp]
            lib.orc_node_coords.argtypes = [cfgp, ctypes.c_int, dp]
            lib.orc_diag.argtypes = [cfgp, dp, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_double, dp]
            lib.orc_tgv_step_sample.argtypes = [cfgp, ctypes.c_double, ctypes.c_double,
                                                ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                                ctypes.POINTER(ctypes.c_long), dp]
            lib.orc_num_threads.restype = ctypes.c_int
            lib.orc_stream_adjoint.argtypes = [cfgp, ctypes.c_int, ctypes.c_int, dp, dp, dp]
            lib.orc_collide_vjp.argtypes = [cfgp, dp, dp, dp, dp]
            lib.orc_ek_grad.argtypes = [cfgp, dp, ctypes.c_double, ctypes.c_double, dp]
            lib.orc_diag_grad.argtypes = [cfgp, dp] + [ctypes.c_double] * 6 + [dp]
            lib.orc_init_fields_vjp.argtypes = [cfgp, dp, dp, dp, dp, dp, dp, dp]
            _lib = lib
    return _lib


class _Cfg(ctypes.Structure):
    _fields_ = [("cells", ctypes.c_int * 3), ("p", ctypes.c_int), ("L", ctypes.c_double * 3),
                ("dt", ctypes.c_double), ("mu_inf", ctypes.c_double),
                ("gamma", ctypes.c_double), ("Pr", ctypes.c_double),
                ("pr_correction", ctypes.c_int), ("collide", ctypes.c_int)]


@dataclass
class Grid:
    """Periodic uniform hexahedral mesh of order-p cells plus the collision constants."""
    cells: tuple
    p: int
    dt: float
    mu_inf: float = 0.0
    gamma: float = 1.4
    Pr: float = 0.7
    pr_correction: bool = False
    collide: bool = True
    L: tuple = (2 * np.pi, 2 * np.pi, 2 * np.pi)

    @property
    def N(self):
        return tuple(c * self.p for c in self.cells)

    @property
    def nodes(self) -> int:
        n = self.N
        return n[0] * n[1] * n[2]

    def _c(self) -> _Cfg:
        c = _Cfg()
        for d in range(3):
            c.cells[d] = int(self.cells[d])
            c.L[d] = float(self.L[d])
        c.p = int(self.p)
        c.dt = float(self.dt)
        c.mu_inf = float(self.mu_inf)
        c.gamma = float(self.gamma)
        c.Pr = float(self.Pr)
        c.pr_correction = int(bool(self.pr_correction))
        c.collide = int(bool(self.collide))
        return c


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def num_threads() -> int:
    return int(_load().orc_num_threads())


def velset():
    """(xi[45,3], w[45]) of the degree-9, 45-abscissa cubature (Sec. II.B)."""
    xi = np.zeros((Q, 3))
    w = np.zeros(Q)
    n = _load().orc_velset(_ptr(xi), _ptr(w))
    assert n == Q
    return xi, w


def glc(p: int) -> np.ndarray:
    r = np.zeros(p + 1)
    _load().orc_glc(p, _ptr(r))
    return r


def lagrange(p: int, r: float) -> np.ndarray:
    ell = np.zeros(p + 1)
    _load().orc_lagrange(p, float(r), _ptr(ell))
    return ell


def lagrange_deriv(p: int, r: float) -> np.ndarray:
    d = np.zeros(p + 1)
    _load().orc_lagrange_deriv(p, float(r), _ptr(d))
    return d


def quad_weights(p: int) -> np.ndarray:
    W = np.zeros(p + 1)
    _load().orc_quad_weights(p, _ptr(W))
    return W


def sutherland(T: float) -> float:
    return float(_load().orc_sutherland(float(T)))


def feq(rho: float, u, T: float, xi=None, w=None) -> np.ndarray:
    """f_i^eq by full tensor contraction (Eq. discreteEquilibrium, App. A, App. B)."""
    if xi is None:
        xi, w = velset()
    xi = np.ascontiguousarray(xi, dtype=np.float64)
    w = np.ascontiguousarray(w, dtype=np.float64)
    u = np.ascontiguousarray(u, dtype=np.float64)
    out = np.zeros(len(w))
    _load().orc_feq(_ptr(xi), _ptr(w), len(w), float(rho), _ptr(u), float(T), _ptr(out))
    return out


def node_coords(g: Grid, d: int) -> np.ndarray:
    x = np.zeros(g.N[d])
    c = g._c()
    _load().orc_node_coords(ctypes.byref(c), d, _ptr(x))
    return x


def stream(g: Grid, src: np.ndarray, xi=None) -> np.ndarray:
    """Semi-Lagrangian pull streaming of every population in ``src`` (shape [nh, nvel, Nz, Ny, Nx])."""
    if xi is None:
        xi, _ = velset()
    xi = np.ascontiguousarray(xi, dtype=np.float64)
    src = np.ascontiguousarray(src, dtype=np.float64)
    nh, nvel = src.shape[0], src.shape[1]
    assert nvel == len(xi)
    dst = np.empty_like(src)
    c = g._c()
    _load().orc_stream(ctypes.byref(c), nh, nvel, _ptr(xi), _ptr(src), _ptr(dst))
    return dst


def collide(g: Grid, pop: np.ndarray) -> np.ndarray:
    out = np.ascontiguousarray(pop, dtype=np.float64).copy()
    c = g._c()
    _load().orc_collide(ctypes.byref(c), _ptr(out))
    return out


def step(g: Grid, pop: np.ndarray, nsteps: int = 1) -> np.ndarray:
    """``nsteps`` SLLBM steps (stream, then collide) of a post-collision state [2,45,Nz,Ny,Nx]."""
    a = np.ascontiguousarray(pop, dtype=np.float64).copy()
    b = np.empty_like(a)
    c = g._c()
    _load().orc_step(ctypes.byref(c), _ptr(a), _ptr(b), int(nsteps))
    return a


def moments(g: Grid, pop: np.ndarray):
    """(rho[Nz,Ny,Nx], u[3,Nz,Ny,Nx], T[Nz,Ny,Nx]) by Eq. (moments)."""
    pop = np.ascontiguousarray(pop, dtype=np.float64)
    shp = g.N[::-1]
    rho = np.zeros(shp)
    u = np.zeros((3,) + shp)
    T = np.zeros(shp)
    c = g._c()
    _load().orc_moments(ctypes.byref(c), _ptr(pop), _ptr(rho), _ptr(u), _ptr(T))
    return rho, u, T


def init_fields(g: Grid, rho, u, T) -> np.ndarray:
    """Equilibrium populations f = f^eq, g = (2C_v - D) T f^eq from given fields."""
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    u = np.ascontiguousarray(u, dtype=np.float64)
    T = np.ascontiguousarray(T, dtype=np.float64)
    pop = np.zeros((2, Q) + g.N[::-1])
    c = g._c()
    _load().orc_init_fields(ctypes.byref(c), _ptr(rho), _ptr(u), _ptr(T), _ptr(pop))
    return pop


def tgv_fields(g: Grid, U0: float, rho0: float = 1.0, T0: float = 1.0, C: float | None = None,
               gamma: float | None = None):
    """Sec. III.C Taylor-Green initial fields; C defaults to gamma*Ma^2 = U0^2/T0."""
    if C is None:
        C = U0 * U0 / T0
    shp = g.N[::-1]
    rho = np.zeros(shp)
    u = np.zeros((3,) + shp)
    T = np.zeros(shp)
    c = g._c()
    _load().orc_tgv_fields(ctypes.byref(c), float(U0), float(rho0), float(T0), float(C),
                           _ptr(rho), _ptr(u), _ptr(T))
    return rho, u, T


def tgv_step_sample(g: Grid, nodes, U0: float, rho0: float = 1.0, T0: float = 1.0,
                    C: float | None = None) -> np.ndarray:
    """One step from the Taylor-Green equilibrium state at the listed node indices only;
    returns [len(nodes), 90] (f then g)."""
    if C is None:
        C = U0 * U0 / T0
    nodes = np.ascontiguousarray(nodes, dtype=np.int64)
    out = np.zeros((len(nodes), 2 * Q))
    c = g._c()
    _load().orc_tgv_step_sample(ctypes.byref(c), float(U0), float(rho0), float(T0), float(C),
                                len(nodes), nodes.ctypes.data_as(ctypes.POINTER(ctypes.c_long)),
                                _ptr(out))
    return out


def diag(g: Grid, pop: np.ndarray, rho_ref: float, Re: float, U0: float) -> np.ndarray:
    """[E_k, eps_s, eps_c] of Sec. III.C, volume-averaged and scaled by U0."""
    pop = np.ascontiguousarray(pop, dtype=np.float64)
    out = np.zeros(3)
    c = g._c()
    _load().orc_diag(ctypes.byref(c), _ptr(pop), float(rho_ref), float(Re), float(U0), _ptr(out))
    return out


# ---- reverse mode --------------------------------------------------------------------------
def stream_adjoint(g: Grid, lam: np.ndarray, xi=None) -> np.ndarray:
    """S^T lam for the pull streaming S of :func:`stream` (same layout): the literal scatter."""
    if xi is None:
        xi, _ = velset()
    xi = np.ascontiguousarray(xi, dtype=np.float64)
    lam = np.ascontiguousarray(lam, dtype=np.float64)
    nh, nvel = lam.shape[0], lam.shape[1]
    assert nvel == len(xi)
    out = np.empty_like(lam)
    c = g._c()
    _load().orc_stream_adjoint(ctypes.byref(c), nh, nvel, _ptr(xi), _ptr(lam), _ptr(out))
    return out


def collide_vjp(g: Grid, h: np.ndarray, lam: np.ndarray):
    """(J^T lam, lam . d collide/d mu_inf) of the collision at the streamed state h [2,45,...]."""
    h = np.ascontiguousarray(h, dtype=np.float64)
    lam = np.ascontiguousarray(lam, dtype=np.float64)
    out = np.empty_like(h)
    dmu = np.zeros(1)
    c = g._c()
    _load().orc_collide_vjp(ctypes.byref(c), _ptr(h), _ptr(lam), _ptr(out), _ptr(dmu))
    return out, float(dmu[0])


def step_adjoint(g: Grid, state_prev: np.ndarray, lam_next: np.ndarray):
    """Adjoint of one :func:`step` taken from state_prev: (lam_prev, d/d mu_inf term)."""
    h = stream(g, state_prev)
    mu_h, dmu = collide_vjp(g, h, lam_next)
    return stream_adjoint(g, mu_h), dmu


def ek_grad(g: Grid, pop: np.ndarray, rho_ref: float, U0: float) -> np.ndarray:
    """d E_k / d pop (E_k as in :func:`diag`), [2,45,Nz,Ny,Nx]; the g half is zero."""
    pop = np.ascontiguousarray(pop, dtype=np.float64)
    lam = np.empty_like(pop)
    c = g._c()
    _load().orc_ek_grad(ctypes.byref(c), _ptr(pop), float(rho_ref), float(U0), _ptr(lam))
    return lam


def diag_grad(g: Grid, pop: np.ndarray, rho_ref: float, Re: float, U0: float,
              weights=(0.0, 1.0, 1.0)) -> np.ndarray:
    """d (wk E_k + ws eps_s + wc eps_c) / d pop for the diagnostics of :func:`diag` (Sec.
    III.C), weights = (wk, ws, wc); [2,45,Nz,Ny,Nx]."""
    pop = np.ascontiguousarray(pop, dtype=np.float64)
    lam = np.empty_like(pop)
    c = g._c()
    wk, ws, wc = (float(x) for x in weights)
    _load().orc_diag_grad(ctypes.byref(c), _ptr(pop), float(rho_ref), float(Re), float(U0), wk, ws, wc,
                          _ptr(lam))
    return lam


def init_fields_vjp(g: Grid, rho, u, T, lam):
    """Gradients of sum(lam * init_fields(rho, u, T)) with respect to rho, u, T."""
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    u = np.ascontiguousarray(u, dtype=np.float64)
    T = np.ascontiguousarray(T, dtype=np.float64)
    lam = np.ascontiguousarray(lam, dtype=np.float64)
    gr, gu, gT = np.empty_like(rho), np.empty_like(u), np.empty_like(T)
    c = g._c()
    _load().orc_init_fields_vjp(ctypes.byref(c), _ptr(rho), _ptr(u), _ptr(T), _ptr(lam),
                                _ptr(gr), _ptr(gu), _ptr(gT))
    return gr, gu, gT
