"""Python binding of libsllbm.so (include/sllbm.h) -- argument marshalling only.

Every function named ``sllbm_*`` here calls the C entry point of the same name; all
arithmetic of the step runs in the library's CUDA kernels.  PyTorch provides device
memory (population buffers are ``torch.uint8`` tensors handed to ``sllbm_set_buffers``)
and the CUDA stream.  There is no CPU fallback: if the library is missing, loading
raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

OK, EINVAL, ENOMEM, ECUDA, ENONFINITE, ETIMEOUT, ENOTREADY, EABORTED, EIO = 0, -1, -2, -3, -4, -5, -6, -7, -8
F64, F32, F16DEV, BF16DEV = 0, 1, 2, 3
STORAGE = {"f64": F64, "f32": F32, "f16dev": F16DEV, "bf16dev": BF16DEV}
Q = 45

_lib = None


class SllbmError(RuntimeError):
    def __init__(self, code: int, where: str, cuda_err: int = 0):
        self.code = code
        msg = f"{where}: {strerror(code)} ({code})"
        if cuda_err:
            msg += f", cudaError {cuda_err}"
        super().__init__(msg)


class Mesh(ctypes.Structure):
    _fields_ = [("cells", ctypes.c_int * 3), ("L", ctypes.c_double * 3)]


class Params(ctypes.Structure):
    _fields_ = [("Ma", ctypes.c_double), ("Re", ctypes.c_double), ("Pr", ctypes.c_double),
                ("gamma", ctypes.c_double), ("T0", ctypes.c_double), ("rho0", ctypes.c_double),
                ("dt_or_courant", ctypes.c_double), ("dt_is_courant", ctypes.c_int),
                ("pr_correction", ctypes.c_int), ("storage", ctypes.c_int),
                ("nonfinite_check", ctypes.c_int), ("tgv_C", ctypes.c_double),
                ("mu_inf_override", ctypes.c_double), ("collide", ctypes.c_int),
                ("kernel", ctypes.c_int)]


class Checkpoint(ctypes.Structure):
    _fields_ = [("storage", ctypes.c_int), ("p", ctypes.c_int), ("velset", ctypes.c_int),
                ("cells", ctypes.c_int * 3), ("pr_correction", ctypes.c_int),
                ("L", ctypes.c_double * 3), ("dt", ctypes.c_double), ("mu_inf", ctypes.c_double),
                ("rho0", ctypes.c_double), ("T0", ctypes.c_double), ("steps", ctypes.c_int64),
                ("payload_bytes", ctypes.c_uint64)]


class Info(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int * 3), ("p", ctypes.c_int), ("nodes", ctypes.c_int64),
                ("Q", ctypes.c_int), ("dt", ctypes.c_double), ("U0", ctypes.c_double),
                ("mu_inf", ctypes.c_double), ("max_xi", ctypes.c_double),
                ("pop_bytes", ctypes.c_size_t), ("storage", ctypes.c_int),
                ("max_cell_shift", ctypes.c_int), ("step_kernel", ctypes.c_int),
                ("step_variant", ctypes.c_int)]


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Loads libsllbm.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError(f"libsllbm.so not built ({path}); run paper_2012_05537_gb300.build.build()")
        _build.build()
    lib = ctypes.CDLL(path)
    vp, dp = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)
    sig = {
        "sllbm_default_params": (None, [ctypes.POINTER(Params)]),
        "sllbm_create": (ctypes.c_int, [ctypes.POINTER(Mesh), ctypes.c_int, ctypes.c_int,
                                        ctypes.POINTER(Params), vp, ctypes.POINTER(vp)]),
        "sllbm_create_slab": (ctypes.c_int, [ctypes.POINTER(Mesh), ctypes.c_int, ctypes.c_int,
                                             ctypes.POINTER(Params), ctypes.c_int, ctypes.c_int, vp,
                                             ctypes.POINTER(vp)]),
        "sllbm_slab_info": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_size_t)]),
        "sllbm_slab_halo_bytes": (ctypes.c_int, [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_size_t)]),
        "sllbm_halo_pack": (ctypes.c_int, [vp, ctypes.c_int, vp, vp]),
        "sllbm_halo_unpack": (ctypes.c_int, [vp, ctypes.c_int, vp, vp]),
        "sllbm_halo_periodic": (ctypes.c_int, [vp, vp]),
        "sllbm_step_begin": (ctypes.c_int, [vp]),
        "sllbm_step_end": (ctypes.c_int, [vp]),
        "sllbm_destroy": (None, [vp]),
        "sllbm_get_info": (ctypes.c_int, [vp, ctypes.POINTER(Info)]),
        "sllbm_velset_table": (ctypes.c_int, [vp, dp, dp]),
        "sllbm_set_buffers": (ctypes.c_int, [vp, vp, vp, ctypes.c_size_t]),
        "sllbm_current_buffer": (vp, [vp]),
        "sllbm_init_tgv": (ctypes.c_int, [vp]),
        "sllbm_init_fields": (ctypes.c_int, [vp, vp, vp, vp, ctypes.c_int]),
        "sllbm_set_populations": (ctypes.c_int, [vp, vp, ctypes.c_int]),
        "sllbm_get_populations": (ctypes.c_int, [vp, vp, ctypes.c_int]),
        "sllbm_step": (ctypes.c_int, [vp, ctypes.c_int]),
        "sllbm_moments": (ctypes.c_int, [vp, vp, vp, vp, ctypes.c_int]),
        "sllbm_diag": (ctypes.c_int, [vp, dp, dp, dp]),
        "sllbm_diag_noalloc": (ctypes.c_int, [vp, dp, dp, dp]),
        "sllbm_run_host": (ctypes.c_int, [vp, vp, vp, ctypes.c_int]),
        "sllbm_run_host_many": (ctypes.c_int, [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.c_int,
                                               ctypes.c_int]),
        "sllbm_sync": (ctypes.c_int, [vp]),
        "sllbm_status": (ctypes.c_int, [vp]),
        "sllbm_last_cuda_error": (ctypes.c_int, [vp]),
        "sllbm_launch_count": (ctypes.c_int64, [vp]),
        "sllbm_strerror": (ctypes.c_char_p, [ctypes.c_int]),
        "sllbm_velset_d3q45": (ctypes.c_int, [dp, dp]),
        "sllbm_stream_table": (ctypes.c_int, [ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                              ctypes.c_int, ctypes.POINTER(ctypes.c_int), dp]),
        "sllbm_set_step_variant": (ctypes.c_int, [vp, ctypes.c_int]),
        "sllbm_autotune": (ctypes.c_int, [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int), dp]),
        "sllbm_batch_plan": (ctypes.c_int, [dp, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
        "sllbm_batch_create": (ctypes.c_int, [ctypes.POINTER(vp), ctypes.c_int, ctypes.c_int, vp,
                                              ctypes.POINTER(vp)]),
        "sllbm_batch_step": (ctypes.c_int, [vp, ctypes.c_int]),
        "sllbm_batch_create_persistent": (ctypes.c_int, [ctypes.POINTER(vp), ctypes.c_int, vp, ctypes.c_int,
                                                         ctypes.POINTER(vp)]),
        "sllbm_batch_shapes": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                              ctypes.POINTER(ctypes.c_int)]),
        "sllbm_batch_destroy": (None, [vp]),
        "sllbm_load_state": (ctypes.c_int, [vp, vp]),
        "sllbm_set_mu_inf": (ctypes.c_int, [vp, ctypes.c_double]),
        "sllbm_stream_apply": (ctypes.c_int, [vp, vp, vp, ctypes.c_int]),
        "sllbm_set_adjoint_type": (ctypes.c_int, [vp, ctypes.c_int]),
        "sllbm_adjoint_step": (ctypes.c_int, [vp, vp, vp, vp, vp]),
        "sllbm_ek_adjoint": (ctypes.c_int, [vp, vp, vp]),
        "sllbm_diag_adjoint": (ctypes.c_int, [vp, vp, vp, ctypes.c_double, ctypes.c_double, ctypes.c_double]),
        "sllbm_init_fields_adjoint": (ctypes.c_int, [vp, vp, vp, vp, vp, vp, vp, vp]),
        "sllbm_set_wait_limit": (ctypes.c_int, [vp, ctypes.c_double]),
        "sllbm_request_abort": (ctypes.c_int, [vp, ctypes.c_int]),
        "sllbm_debug_fail_allocs": (ctypes.c_int, [ctypes.c_int]),
        "sllbm_step_count": (ctypes.c_int64, [vp]),
        "sllbm_set_compensated": (ctypes.c_int, [vp, ctypes.c_int]),
        "sllbm_save": (ctypes.c_int, [vp, ctypes.c_char_p]),
        "sllbm_load": (ctypes.c_int, [vp, ctypes.c_char_p]),
        "sllbm_checkpoint_info": (ctypes.c_int, [ctypes.c_char_p, ctypes.POINTER(Checkpoint)]),
        "sllbm_fma_peak": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, vp, dp, dp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def strerror(code: int) -> str:
    try:
        return load().sllbm_strerror(int(code)).decode()
    except Exception:  # library not loadable: still give a message
        return f"error {code}"


def _check(rc: int, where: str, ctx=None):
    if rc != OK:
        err = load().sllbm_last_cuda_error(ctx) if ctx else 0
        raise SllbmError(rc, where, err)


# ---- thin wrappers with the C names --------------------------------------------------
def sllbm_default_params() -> Params:
    p = Params()
    load().sllbm_default_params(ctypes.byref(p))
    return p


def sllbm_create(mesh: Mesh, p: int, params: Params, stream: int = 0, velset: int = 0):
    ctx = ctypes.c_void_p()
    rc = load().sllbm_create(ctypes.byref(mesh), int(p), int(velset), ctypes.byref(params),
                             ctypes.c_void_p(stream), ctypes.byref(ctx))
    _check(rc, "sllbm_create")
    return ctx


def sllbm_create_slab(mesh: Mesh, p: int, params: Params, z_begin: int, z_cells: int, stream: int = 0,
                      velset: int = 0):
    ctx = ctypes.c_void_p()
    rc = load().sllbm_create_slab(ctypes.byref(mesh), int(p), int(velset), ctypes.byref(params), int(z_begin),
                                  int(z_cells), ctypes.c_void_p(stream), ctypes.byref(ctx))
    _check(rc, "sllbm_create_slab")
    return ctx


def sllbm_slab_info(ctx):
    """(ghost cells per side, bytes of one side's halo buffer)."""
    g, b = ctypes.c_int(), ctypes.c_size_t()
    _check(load().sllbm_slab_info(ctx, ctypes.byref(g), ctypes.byref(b)), "sllbm_slab_info", ctx)
    return int(g.value), int(b.value)


def sllbm_slab_halo_bytes(ctx, side: int) -> int:
    """Bytes sllbm_halo_pack(side) writes (the neighbour's sllbm_halo_unpack(1 - side) reads)."""
    b = ctypes.c_size_t()
    _check(load().sllbm_slab_halo_bytes(ctx, int(side), ctypes.byref(b)), "sllbm_slab_halo_bytes", ctx)
    return int(b.value)


def sllbm_halo_pack(ctx, side: int, halo_ptr: int, stream: int = 0) -> None:
    _check(load().sllbm_halo_pack(ctx, int(side), ctypes.c_void_p(halo_ptr), ctypes.c_void_p(stream)),
           "sllbm_halo_pack", ctx)


def sllbm_halo_unpack(ctx, side: int, halo_ptr: int, stream: int = 0) -> None:
    _check(load().sllbm_halo_unpack(ctx, int(side), ctypes.c_void_p(halo_ptr), ctypes.c_void_p(stream)),
           "sllbm_halo_unpack", ctx)


def sllbm_halo_periodic(ctx, stream: int = 0) -> None:
    _check(load().sllbm_halo_periodic(ctx, ctypes.c_void_p(stream)), "sllbm_halo_periodic", ctx)


def sllbm_step_begin(ctx) -> None:
    _check(load().sllbm_step_begin(ctx), "sllbm_step_begin", ctx)


def sllbm_step_end(ctx) -> None:
    _check(load().sllbm_step_end(ctx), "sllbm_step_end", ctx)


def sllbm_destroy(ctx) -> None:
    load().sllbm_destroy(ctx)


def sllbm_get_info(ctx) -> Info:
    info = Info()
    _check(load().sllbm_get_info(ctx, ctypes.byref(info)), "sllbm_get_info", ctx)
    return info


def sllbm_velset_table(ctx):
    xi = np.zeros((Q, 3))
    w = np.zeros(Q)
    dp = ctypes.POINTER(ctypes.c_double)
    _check(load().sllbm_velset_table(ctx, xi.ctypes.data_as(dp), w.ctypes.data_as(dp)),
           "sllbm_velset_table", ctx)
    return xi, w


def sllbm_set_buffers(ctx, ptr_a: int, ptr_b: int, nbytes: int) -> None:
    _check(load().sllbm_set_buffers(ctx, ctypes.c_void_p(ptr_a), ctypes.c_void_p(ptr_b),
                                    ctypes.c_size_t(nbytes)), "sllbm_set_buffers", ctx)


def sllbm_current_buffer(ctx) -> int:
    return load().sllbm_current_buffer(ctx) or 0


def sllbm_init_tgv(ctx) -> None:
    _check(load().sllbm_init_tgv(ctx), "sllbm_init_tgv", ctx)


def sllbm_init_fields(ctx, rho_ptr: int, u_ptr: int, T_ptr: int, on_device: bool) -> None:
    _check(load().sllbm_init_fields(ctx, ctypes.c_void_p(rho_ptr), ctypes.c_void_p(u_ptr),
                                    ctypes.c_void_p(T_ptr), int(on_device)), "sllbm_init_fields", ctx)


def sllbm_set_populations(ctx, ptr: int, on_device: bool) -> None:
    _check(load().sllbm_set_populations(ctx, ctypes.c_void_p(ptr), int(on_device)),
           "sllbm_set_populations", ctx)


def sllbm_get_populations(ctx, ptr: int, on_device: bool) -> None:
    _check(load().sllbm_get_populations(ctx, ctypes.c_void_p(ptr), int(on_device)),
           "sllbm_get_populations", ctx)


def sllbm_step(ctx, n: int) -> int:
    rc = load().sllbm_step(ctx, int(n))
    if rc not in (OK, ENONFINITE):
        _check(rc, "sllbm_step", ctx)
    return rc


def sllbm_moments(ctx, rho_ptr: int, u_ptr: int, T_ptr: int, on_device: bool) -> None:
    _check(load().sllbm_moments(ctx, ctypes.c_void_p(rho_ptr), ctypes.c_void_p(u_ptr),
                                ctypes.c_void_p(T_ptr), int(on_device)), "sllbm_moments", ctx)


def sllbm_diag(ctx):
    a, b, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(load().sllbm_diag(ctx, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)),
           "sllbm_diag", ctx)
    return a.value, b.value, c.value


def sllbm_diag_noalloc(ctx):
    """sllbm_diag without device allocation (static library scratch, <= 65536 cells)."""
    a, b, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(load().sllbm_diag_noalloc(ctx, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)),
           "sllbm_diag_noalloc", ctx)
    return a.value, b.value, c.value


def sllbm_run_host(ctx, in_ptr: int, out_ptr: int, n: int) -> None:
    _check(load().sllbm_run_host(ctx, ctypes.c_void_p(in_ptr), ctypes.c_void_p(out_ptr), int(n)),
           "sllbm_run_host", ctx)


def sllbm_run_host_many(ctx, in_ptrs, out_ptrs, n: int) -> None:
    assert len(in_ptrs) == len(out_ptrs)
    ins = (ctypes.c_void_p * len(in_ptrs))(*in_ptrs)
    outs = (ctypes.c_void_p * len(out_ptrs))(*out_ptrs)
    _check(load().sllbm_run_host_many(ctx, ins, outs, len(in_ptrs), int(n)), "sllbm_run_host_many", ctx)


def sllbm_status(ctx) -> int:
    rc = load().sllbm_status(ctx)
    if rc not in (OK, ETIMEOUT, EABORTED):
        _check(rc, "sllbm_status", ctx)
    return rc


def sllbm_set_wait_limit(ctx, seconds: float) -> None:
    _check(load().sllbm_set_wait_limit(ctx, float(seconds)), "sllbm_set_wait_limit", ctx)


def sllbm_request_abort(ctx, on: bool) -> None:
    _check(load().sllbm_request_abort(ctx, int(bool(on))), "sllbm_request_abort", ctx)


def sllbm_debug_fail_allocs(after: int) -> None:
    _check(load().sllbm_debug_fail_allocs(int(after)), "sllbm_debug_fail_allocs")


def sllbm_set_compensated(ctx, on: bool) -> None:
    _check(load().sllbm_set_compensated(ctx, int(bool(on))), "sllbm_set_compensated", ctx)


def sllbm_step_count(ctx) -> int:
    return int(load().sllbm_step_count(ctx))


def sllbm_save(ctx, path: str) -> None:
    _check(load().sllbm_save(ctx, os.fsencode(path)), "sllbm_save", ctx)


def sllbm_load(ctx, path: str) -> None:
    _check(load().sllbm_load(ctx, os.fsencode(path)), "sllbm_load", ctx)


def sllbm_checkpoint_info(path: str) -> Checkpoint:
    c = Checkpoint()
    _check(load().sllbm_checkpoint_info(os.fsencode(path), ctypes.byref(c)), "sllbm_checkpoint_info")
    return c


def sllbm_fma_peak(kind: int, iters: int = 4096, stream: int = 0):
    """(flop/s, seconds) of the FMA microbenchmark: kind 0 FP32, 1 packed FP32x2, 2 FP64."""
    f, t = ctypes.c_double(), ctypes.c_double()
    _check(load().sllbm_fma_peak(int(kind), int(iters), ctypes.c_void_p(stream), ctypes.byref(f),
                                 ctypes.byref(t)), "sllbm_fma_peak")
    return float(f.value), float(t.value)


def sllbm_sync(ctx) -> None:
    _check(load().sllbm_sync(ctx), "sllbm_sync", ctx)


def sllbm_velset_d3q45():
    xi = np.zeros((Q, 3))
    w = np.zeros(Q)
    dp = ctypes.POINTER(ctypes.c_double)
    _check(load().sllbm_velset_d3q45(xi.ctypes.data_as(dp), w.ctypes.data_as(dp)), "sllbm_velset_d3q45")
    return xi, w


def sllbm_stream_table(p: int, h: float, dt: float, direction: int):
    shift = np.zeros((Q, p), dtype=np.int32)
    weights = np.zeros((Q, p, p + 1))
    _check(load().sllbm_stream_table(int(p), float(h), float(dt), int(direction),
                                     shift.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                     weights.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
           "sllbm_stream_table")
    return shift, weights


def sllbm_launch_count(ctx) -> int:
    return int(load().sllbm_launch_count(ctx))


def sllbm_set_step_variant(ctx, variant: int) -> None:
    _check(load().sllbm_set_step_variant(ctx, int(variant)), "sllbm_set_step_variant", ctx)


def sllbm_autotune(ctx, steps: int):
    """(chosen variant, ms per step)."""
    v, ms = ctypes.c_int(), ctypes.c_double()
    _check(load().sllbm_autotune(ctx, int(steps), ctypes.byref(v), ctypes.byref(ms)), "sllbm_autotune", ctx)
    return v.value, ms.value


def sllbm_batch_plan(cost, streams: int) -> np.ndarray:
    cost = np.ascontiguousarray(cost, dtype=np.float64)
    assign = np.zeros(len(cost), dtype=np.int32)
    _check(load().sllbm_batch_plan(cost.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), len(cost),
                                   int(streams), assign.ctypes.data_as(ctypes.POINTER(ctypes.c_int))),
           "sllbm_batch_plan")
    return assign


def sllbm_batch_create(ctxs, streams: int, stream: int):
    arr = (ctypes.c_void_p * len(ctxs))(*[c.value if isinstance(c, ctypes.c_void_p) else c for c in ctxs])
    b = ctypes.c_void_p()
    _check(load().sllbm_batch_create(arr, len(ctxs), int(streams), ctypes.c_void_p(stream), ctypes.byref(b)),
           "sllbm_batch_create")
    return b


def sllbm_batch_create_persistent(ctxs, stream: int, tune_steps: int = 0):
    arr = (ctypes.c_void_p * len(ctxs))(*[c.value if isinstance(c, ctypes.c_void_p) else c for c in ctxs])
    b = ctypes.c_void_p()
    _check(load().sllbm_batch_create_persistent(arr, len(ctxs), ctypes.c_void_p(stream), int(tune_steps),
                                                ctypes.byref(b)), "sllbm_batch_create_persistent")
    return b


def sllbm_batch_shapes(b):
    """Tile shape per order (p = 2, 3, 4) of a persistent batch; -1 where the order is absent."""
    v = [ctypes.c_int() for _ in range(3)]
    _check(load().sllbm_batch_shapes(b, *(ctypes.byref(x) for x in v)), "sllbm_batch_shapes")
    return {2: v[0].value, 3: v[1].value, 4: v[2].value}


def sllbm_batch_step(b, nsteps: int) -> None:
    _check(load().sllbm_batch_step(b, int(nsteps)), "sllbm_batch_step")


def sllbm_batch_destroy(b) -> None:
    load().sllbm_batch_destroy(b)


def sllbm_load_state(ctx, state_ptr: int) -> None:
    _check(load().sllbm_load_state(ctx, ctypes.c_void_p(state_ptr)), "sllbm_load_state", ctx)


def sllbm_set_mu_inf(ctx, mu_inf: float) -> None:
    _check(load().sllbm_set_mu_inf(ctx, float(mu_inf)), "sllbm_set_mu_inf", ctx)


def sllbm_set_adjoint_type(ctx, storage: int) -> None:
    _check(load().sllbm_set_adjoint_type(ctx, int(storage)), "sllbm_set_adjoint_type", ctx)


def sllbm_stream_apply(ctx, src_ptr: int, dst_ptr: int, transpose: bool) -> None:
    _check(load().sllbm_stream_apply(ctx, ctypes.c_void_p(src_ptr), ctypes.c_void_p(dst_ptr),
                                     int(bool(transpose))), "sllbm_stream_apply", ctx)


def sllbm_adjoint_step(ctx, state_prev_ptr: int, lam_next_ptr: int, lam_prev_ptr: int,
                       dmu_ptr: int) -> None:
    _check(load().sllbm_adjoint_step(ctx, ctypes.c_void_p(state_prev_ptr), ctypes.c_void_p(lam_next_ptr),
                                     ctypes.c_void_p(lam_prev_ptr), ctypes.c_void_p(dmu_ptr)),
           "sllbm_adjoint_step", ctx)


def sllbm_ek_adjoint(ctx, state_ptr: int, lam_ptr: int) -> None:
    _check(load().sllbm_ek_adjoint(ctx, ctypes.c_void_p(state_ptr), ctypes.c_void_p(lam_ptr)),
           "sllbm_ek_adjoint", ctx)


def sllbm_diag_adjoint(ctx, state_ptr: int, lam_ptr: int, wk: float, ws: float, wc: float) -> None:
    _check(load().sllbm_diag_adjoint(ctx, ctypes.c_void_p(state_ptr), ctypes.c_void_p(lam_ptr), float(wk),
                                     float(ws), float(wc)), "sllbm_diag_adjoint", ctx)


def sllbm_init_fields_adjoint(ctx, rho_ptr: int, u_ptr: int, T_ptr: int, lam_ptr: int,
                              grad_rho_ptr: int, grad_u_ptr: int, grad_T_ptr: int) -> None:
    vp = ctypes.c_void_p
    _check(load().sllbm_init_fields_adjoint(ctx, vp(rho_ptr), vp(u_ptr), vp(T_ptr), vp(lam_ptr),
                                            vp(grad_rho_ptr or None), vp(grad_u_ptr or None),
                                            vp(grad_T_ptr or None)), "sllbm_init_fields_adjoint", ctx)


# ---- convenience object ------------------------------------------------------------------
@dataclass
class Config:
    cells: tuple = (8, 8, 8)
    p: int = 3
    Ma: float = 0.5
    Re: float = 1600.0
    Pr: float = 0.7
    gamma: float = 1.4
    T0: float = 1.0
    rho0: float = 1.0
    courant: float | None = 2.0
    dt: float | None = None
    pr_correction: bool = False
    storage: str = "f32"
    nonfinite_check: bool = False
    tgv_C: float = -1.0
    mu_inf: float | None = None
    collide: bool = True
    kernel: int = 0  # 0 automatic, 1 generic tile kernel, 2 TMA-fed persistent kernel
    slab: tuple | None = None  # (z_begin, z_cells): this part of a mesh decomposed along z
    L: tuple = (2 * np.pi, 2 * np.pi, 2 * np.pi)


class Sim:
    """One SLLBM context with torch-owned ping-pong population buffers."""

    def __init__(self, cfg: Config, device=None, stream=None):
        import torch
        self.cfg = cfg
        self.torch = torch
        self.device = torch.device(device if device is not None else "cuda")
        if self.device.type != "cuda":
            raise RuntimeError("the SLLBM library runs on CUDA devices only")
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        mesh = Mesh()
        for d in range(3):
            mesh.cells[d] = int(cfg.cells[d])
            mesh.L[d] = float(cfg.L[d])
        prm = sllbm_default_params()
        prm.Ma, prm.Re, prm.Pr, prm.gamma = cfg.Ma, cfg.Re, cfg.Pr, cfg.gamma
        prm.T0, prm.rho0 = cfg.T0, cfg.rho0
        if cfg.dt is not None:
            prm.dt_or_courant, prm.dt_is_courant = float(cfg.dt), 0
        else:
            prm.dt_or_courant, prm.dt_is_courant = float(cfg.courant), 1
        prm.pr_correction = int(bool(cfg.pr_correction))
        prm.storage = STORAGE[cfg.storage]
        prm.nonfinite_check = int(bool(cfg.nonfinite_check))
        prm.tgv_C = float(cfg.tgv_C)
        prm.mu_inf_override = float(cfg.mu_inf) if cfg.mu_inf else 0.0
        prm.collide = int(bool(cfg.collide))
        prm.kernel = int(cfg.kernel)
        with torch.cuda.device(self.device):
            if cfg.slab is None:
                self.ctx = sllbm_create(mesh, cfg.p, prm, self.stream.cuda_stream)
            else:
                self.ctx = sllbm_create_slab(mesh, cfg.p, prm, int(cfg.slab[0]), int(cfg.slab[1]),
                                             self.stream.cuda_stream)
        self.info = sllbm_get_info(self.ctx)
        nb = int(self.info.pop_bytes)
        self.buffers = [torch.empty(nb, dtype=torch.uint8, device=self.device) for _ in range(2)]
        sllbm_set_buffers(self.ctx, self.buffers[0].data_ptr(), self.buffers[1].data_ptr(), nb)

    # geometry
    @property
    def N(self):
        return tuple(self.info.N)

    @property
    def nodes(self) -> int:
        return int(self.info.nodes)

    @property
    def dt(self) -> float:
        return float(self.info.dt)

    @property
    def pop_dtype(self):
        t = self.torch
        return {F64: t.float64, F32: t.float32, F16DEV: t.float16, BF16DEV: t.bfloat16}[self.info.storage]

    def velset(self):
        return sllbm_velset_table(self.ctx)

    def init_tgv(self):
        sllbm_init_tgv(self.ctx)
        return self

    def init_fields(self, rho, u, T):
        t = self.torch
        rho = t.as_tensor(rho, dtype=t.float64, device=self.device).contiguous()
        u = t.as_tensor(u, dtype=t.float64, device=self.device).contiguous()
        T = t.as_tensor(T, dtype=t.float64, device=self.device).contiguous()
        sllbm_init_fields(self.ctx, rho.data_ptr(), u.data_ptr(), T.data_ptr(), True)
        return self

    def set_populations(self, pop):
        t = self.torch
        pop = t.as_tensor(pop, dtype=t.float64, device=self.device).contiguous()
        assert pop.numel() == 2 * Q * self.nodes
        sllbm_set_populations(self.ctx, pop.data_ptr(), True)
        self.sync()
        return self

    def populations(self):
        """Current state as a float64 tensor [2, 45, Nz, Ny, Nx] on the device."""
        t = self.torch
        out = t.empty((2, Q) + self.N[::-1], dtype=t.float64, device=self.device)
        sllbm_get_populations(self.ctx, out.data_ptr(), True)
        self.sync()
        return out

    def raw_state(self):
        """Current state buffer viewed in the storage dtype and storage order,
        [45, Nz, Ny, Nx, 2] with the last index 0 for f and 1 for g (no copy)."""
        cur = sllbm_current_buffer(self.ctx)
        idx = 0 if cur == self.buffers[0].data_ptr() else 1
        return self.buffers[idx].view(self.pop_dtype).view((Q,) + self.N[::-1] + (2,))

    def step(self, n: int = 1) -> int:
        return sllbm_step(self.ctx, n)

    def state_like(self):
        """An uninitialised tensor shaped and typed like a state buffer [45, Nz, Ny, Nx, 2]."""
        return self.torch.empty((Q,) + self.N[::-1] + (2,), dtype=self.pop_dtype, device=self.device)

    def set_adjoint_type(self, storage: str) -> None:
        """Type of the adjoint populations of reverse-mode calls: "f64" keeps them in FP64
        next to FP32 forward states; the storage type is the default."""
        sllbm_set_adjoint_type(self.ctx, STORAGE[storage])
        self._adj_f64 = storage == "f64"

    @property
    def adjoint_dtype(self):
        return self.torch.float64 if getattr(self, "_adj_f64", False) else self.pop_dtype

    def set_variant(self, variant: int) -> None:
        """Step kernel: 0 TMA-fed, 1 generic default tile, 2 and 3 generic alternative tiles."""
        sllbm_set_step_variant(self.ctx, variant)
        self.info = sllbm_get_info(self.ctx)

    def set_compensated(self, on: bool = True) -> None:
        """Compensated moment sums for the following steps (the kernel choice is made again)."""
        sllbm_set_compensated(self.ctx, on)
        self.info = sllbm_get_info(self.ctx)

    def autotune(self, steps: int = 5):
        """Times every variant that can run this context from the current state, keeps the
        fastest (the state is restored); returns (variant, ms per step)."""
        out = sllbm_autotune(self.ctx, steps)
        self.info = sllbm_get_info(self.ctx)
        return out

    def load_state(self, state) -> None:
        assert state.is_contiguous() and state.dtype == self.pop_dtype
        assert state.numel() * state.element_size() == int(self.info.pop_bytes)
        sllbm_load_state(self.ctx, state.data_ptr())

    def set_mu_inf(self, mu_inf: float) -> None:
        sllbm_set_mu_inf(self.ctx, mu_inf)
        self.info = sllbm_get_info(self.ctx)

    def moments(self):
        t = self.torch
        shp = self.N[::-1]
        rho = t.empty(shp, dtype=t.float64, device=self.device)
        u = t.empty((3,) + shp, dtype=t.float64, device=self.device)
        T = t.empty(shp, dtype=t.float64, device=self.device)
        sllbm_moments(self.ctx, rho.data_ptr(), u.data_ptr(), T.data_ptr(), True)
        self.sync()
        return rho, u, T

    def diag(self):
        return sllbm_diag(self.ctx)

    def run_host(self, host_in, host_out, n: int):
        sllbm_run_host(self.ctx, host_in.data_ptr(), host_out.data_ptr(), n)

    def run_host_many(self, host_ins, host_outs, n: int):
        """Pipelined end-to-end runs of independent states (pinned host tensors)."""
        sllbm_run_host_many(self.ctx, [t.data_ptr() for t in host_ins], [t.data_ptr() for t in host_outs], n)

    def sync(self):
        sllbm_sync(self.ctx)

    def status(self) -> int:
        return sllbm_status(self.ctx)

    def launches(self) -> int:
        return sllbm_launch_count(self.ctx)

    def close(self):
        if getattr(self, "ctx", None):
            sllbm_sync(self.ctx)
            sllbm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
