"""Run control on the GPU, without faulting or hanging it: a bounded device-side wait that
runs out (a wait limit of zero) and a host abort request both make the TMA-fed persistent
kernel leave early and report through sllbm_status, after which the same context steps
correctly again; injected allocation failures come back as SLLBM_ENOMEM; checkpoints
restore a run bit for bit; the FMA microbenchmark gives plausible rates."""
import numpy as np
import pytest

import oracle as O
from paper_2012_05537_gb300 import build as B

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


# the TMA-fed instances the run-control tests cover: FP32 at p = 4 (without and with the
# Prandtl term, whose epilogue has more barriers), FP16 deviations at p = 3 (a 16-bit box is
# released right after its z pass), BF16 deviations at p = 4
# (storage, p, cells); the suffix "pr" adds the Prandtl term, "kc" compensated moment sums
# (their instances hold a smaller box ring)
TMA_RUN_CASES = [("f32", 4, (16, 8, 8)), ("f32pr", 4, (8, 8, 4)), ("f16dev", 3, (8, 6, 4)), ("bf16dev", 4, (8, 4, 4)),
                 ("f32kc", 4, (8, 8, 4)), ("f16devkc", 3, (8, 6, 4))]


def tma_sim(S, cells=(16, 8, 8), storage="f32", p=4):
    pr, kc = storage.endswith("pr"), storage.endswith("kc")
    storage = storage[:-2] if (pr or kc) else storage
    sim = S.Sim(S.Config(cells=cells, p=p, courant=3.0, storage=storage, kernel=2, pr_correction=pr))
    if kc:
        S.sllbm_set_compensated(sim.ctx, True)
    assert S.sllbm_get_info(sim.ctx).step_kernel == 2
    return sim


def check_against_oracle(S, sim, steps=2, tol=1e-5):
    """FP32: the oracle's run from the FP32-rounded Taylor-Green state.  16-bit deviations: one
    step from the decoded state, in deviation space within the output rounding (2^-11 or 2^-8
    of |d|) plus 1e-5 max|d| for the FP32 arithmetic."""
    sim.init_tgv()
    g = O.Grid(cells=tuple(sim.cfg.cells), p=sim.cfg.p, dt=sim.dt, mu_inf=float(sim.info.mu_inf),
               pr_correction=bool(sim.cfg.pr_correction))
    if sim.cfg.storage == "f32":
        assert sim.step(steps) == 0
        assert S.sllbm_status(sim.ctx) == S.OK
        got = sim.populations().cpu().numpy()
        pop = O.init_fields(g, *O.tgv_fields(g, sim.info.U0)).astype(np.float32).astype(np.float64)
        ref = O.step(g, pop, steps)
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= tol
        return
    start = sim.populations().cpu().numpy()
    assert sim.step(1) == 0
    assert S.sllbm_status(sim.ctx) == S.OK
    ref = O.step(g, start, 1)
    _, w = O.velset()
    c = sim.cfg
    dref = np.array([c.rho0, (2.0 / (c.gamma - 1.0) - 3.0) * c.T0 * c.rho0]).reshape(2, 1, 1, 1, 1)
    dev = lambda pop: pop / np.asarray(w).reshape(1, -1, 1, 1, 1) - dref  # noqa: E731
    d_ref, d_got = dev(ref), dev(sim.populations().cpu().numpy())
    rb = 2.0 ** -11 if c.storage == "f16dev" else 2.0 ** -8
    assert np.all(np.abs(d_got - d_ref) <= rb * np.abs(d_ref) + 1e-5 * np.abs(d_ref).max())


@pytest.mark.parametrize("storage,p,cells", TMA_RUN_CASES)
def test_wait_limit_runs_out_then_context_steps_cleanly(S, storage, p, cells):
    sim = tma_sim(S, cells, storage, p)
    sim.init_tgv()
    S.sllbm_set_wait_limit(sim.ctx, 0.0)  # every wait that is not satisfied at once gives up
    assert sim.step(3) == 0  # (the launches are asynchronous; the status tells)
    assert S.sllbm_status(sim.ctx) == S.ETIMEOUT
    assert S.sllbm_status(sim.ctx) == S.OK  # reported once, then cleared
    torch.cuda.synchronize()  # the CUDA context is intact
    S.sllbm_set_wait_limit(sim.ctx, 2.0)
    check_against_oracle(S, sim)
    sim.close()


@pytest.mark.parametrize("storage,p,cells", TMA_RUN_CASES)
def test_abort_request_stops_the_persistent_kernel(S, storage, p, cells):
    sim = tma_sim(S, cells, storage, p)
    sim.init_tgv()
    S.sllbm_request_abort(sim.ctx, True)
    assert sim.step(2) == 0
    assert S.sllbm_status(sim.ctx) == S.EABORTED
    S.sllbm_request_abort(sim.ctx, False)
    torch.cuda.synchronize()
    check_against_oracle(S, sim)
    sim.close()


def test_injected_allocation_failures(S):
    mesh = S.Mesh()
    for d in range(3):
        mesh.cells[d], mesh.L[d] = 3, 2 * np.pi
    prm = S.sllbm_default_params()
    prm.dt_or_courant, prm.dt_is_courant = 2.0, 1
    stream = torch.cuda.current_stream().cuda_stream
    for after in (0, 1, 3):  # node coordinates (three arrays), then the flag words
        S.sllbm_debug_fail_allocs(after)
        with pytest.raises(S.SllbmError) as e:
            S.sllbm_create(mesh, 3, prm, stream)
        assert e.value.code == S.ENOMEM
    ctx = S.sllbm_create(mesh, 3, prm, stream)  # the hook disarmed itself
    S.sllbm_debug_fail_allocs(0)  # the state buffers the context allocates itself
    assert S.load().sllbm_init_tgv(ctx) == S.ENOMEM
    S.sllbm_init_tgv(ctx)
    assert S.sllbm_step(ctx, 1) == S.OK
    S.sllbm_sync(ctx)
    S.sllbm_destroy(ctx)


@pytest.mark.parametrize("storage,p,kernel", [("f32", 4, 2), ("f64", 3, 1), ("f16dev", 3, 1)])
def test_checkpoint_restores_the_run_bit_for_bit(S, tmp_path, storage, p, kernel):
    cells = (8, 4, 4) if p == 4 else (3, 4, 2)
    cfg = S.Config(cells=cells, p=p, courant=2.0, storage=storage, kernel=kernel)
    a = S.Sim(cfg)
    a.init_tgv()
    a.step(3)
    path = str(tmp_path / "state.ckpt")
    S.sllbm_save(a.ctx, path)
    info = S.sllbm_checkpoint_info(path)
    assert info.steps == 3 and S.sllbm_step_count(a.ctx) == 3 and info.payload_bytes == a.info.pop_bytes
    a.step(4)
    want = a.raw_state().clone()
    b = S.Sim(cfg)
    S.sllbm_load(b.ctx, path)
    assert S.sllbm_step_count(b.ctx) == 3
    b.step(4)
    assert S.sllbm_step_count(b.ctx) == 7
    assert torch.equal(b.raw_state(), want)
    # a context of another order refuses the file; so does a truncated file
    c = S.Sim(S.Config(cells=cells, p=2, courant=2.0, storage=storage))
    with pytest.raises(S.SllbmError) as e:
        S.sllbm_load(c.ctx, path)
    assert e.value.code == S.EINVAL
    raw = open(path, "rb").read()
    open(path, "wb").write(raw[:-100])
    with pytest.raises(S.SllbmError) as e:
        S.sllbm_load(b.ctx, path)
    assert e.value.code == S.EINVAL
    for s in (a, b, c):
        s.close()


def test_fma_peak_rates_are_plausible(S):
    f32, _ = S.sllbm_fma_peak(0, 2048)
    f32x2, _ = S.sllbm_fma_peak(1, 2048)
    f64, _ = S.sllbm_fma_peak(2, 256)
    print(f"FMA peaks: FP32 {f32 / 1e12:.1f}, FP32x2 {f32x2 / 1e12:.1f}, FP64 {f64 / 1e12:.2f} TFLOP/s")
    assert 10e12 < f32 < 200e12
    assert 0.5 * f32 < f32x2 < 4 * f32
    assert 0.05e12 < f64 < f32
