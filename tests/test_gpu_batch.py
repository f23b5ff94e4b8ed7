"""Kernel variants, autotuner and the graph-captured batched launch.

* every tile-shape variant of the generic FP32 kernel against the oracle (one step, the FP32
  tolerance of the other step tests: relative L2 <= 1e-6, elements <= 2e-6 of the scale);
* the autotuner leaves the state as it found it and picks a variant that can run;
* a batch of instances of uneven size and order advanced through the graph equals, bit for
  bit, each instance advanced on its own with the same kernel (same launches, same inputs).
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


def grid_of(sim):
    c = sim.cfg
    return O.Grid(cells=tuple(c.cells), p=c.p, dt=sim.dt, mu_inf=float(sim.info.mu_inf), gamma=c.gamma, Pr=c.Pr)


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("variant", [2, 3])
@pytest.mark.parametrize("cells,p", [((3, 5, 2), 2), ((3, 2, 3), 3), ((3, 1, 2), 4)])
def test_tile_variants_match_oracle(S, variant, cells, p):
    sim = S.Sim(S.Config(cells=cells, p=p, courant=3.0, storage="f32"))
    sim.set_variant(variant)
    assert sim.info.step_variant == variant
    g = grid_of(sim)
    rho, u, T = I.smooth_fields(g.N[::-1], 7)
    pop = O.init_fields(g, rho, u, T) * (1.0 + 0.02 * I.noise((2, 45) + g.N[::-1], 8))
    pop = pop.astype(np.float32).astype(np.float64)
    sim.set_populations(pop)
    assert sim.step(1) == 0
    ref = O.step(g, pop, 1)
    got = sim.populations().cpu().numpy()
    assert rel_l2(got, ref) <= 1e-6
    assert np.max(np.abs(got - ref)) <= 2e-6 * np.abs(ref).max()


def test_variants_refused_where_they_cannot_run(S):
    odd = S.Sim(S.Config(cells=(3, 3, 3), p=4, storage="f32"))
    with pytest.raises(S.SllbmError):
        odd.set_variant(0)  # TMA kernel needs whole tiles
    f64 = S.Sim(S.Config(cells=(2, 2, 2), p=2, storage="f64"))
    with pytest.raises(S.SllbmError):
        f64.set_variant(2)
    with pytest.raises(S.SllbmError):
        f64.set_variant(7)


def test_autotune_restores_the_state(S):
    sim = S.Sim(S.Config(cells=(8, 8, 4), p=4, courant=4.0, storage="f32")).init_tgv()
    assert sim.step(3) == 0
    before = sim.raw_state().clone()
    cur = S.sllbm_current_buffer(sim.ctx)
    v, ms = sim.autotune(3)
    assert v in (0, 1, 2, 3) and ms > 0 and sim.info.step_variant == v
    assert S.sllbm_current_buffer(sim.ctx) == cur
    assert torch.equal(sim.raw_state(), before)


def test_batch_equals_instances_stepped_alone(S):
    insts = I.batch_instances(12, 5)
    insts = [I.Instance(cells=(min(i.cells[0], 12),) * 3, p=i.p, Ma=min(i.Ma, 0.9), Re=i.Re,
                        courant=min(i.courant, 4.0)) for i in insts]
    from paper_2012_05537_gb300 import batch as BT
    sims = BT.make_instances(insts)
    alone = BT.make_instances(insts)
    for k, (a, b) in enumerate(zip(sims, alone)):
        v = k % 4
        try:
            a.set_variant(v)
        except S.SllbmError:
            a.set_variant(1)
        b.set_variant(a.info.step_variant)
    bt = BT.Batch(sims, streams=4)
    bt.step(4)
    for b in alone:
        assert b.step(4) == 0
    torch.cuda.synchronize()
    for a, b in zip(sims, alone):
        assert torch.equal(a.raw_state(), b.raw_state())
    with pytest.raises(S.SllbmError):
        bt.step(3)  # odd step counts would flip the ping-pong parity baked into the graph
    assert sims[0].step(1) == 0
    with pytest.raises(S.SllbmError):
        bt.step(2)  # an instance moved on its own by an odd number of steps
    assert sims[0].step(1) == 0
    bt.step(2)
    torch.cuda.synchronize()
    bt.close()


def test_batch_refuses_the_legacy_stream_and_duplicates(S):
    sim = S.Sim(S.Config(cells=(2, 2, 2), p=2, storage="f32")).init_tgv()
    with pytest.raises(S.SllbmError):
        S.sllbm_batch_create([sim.ctx], 1, 0)
    st = torch.cuda.Stream()
    with pytest.raises(S.SllbmError):
        S.sllbm_batch_create([sim.ctx, sim.ctx], 1, st.cuda_stream)


@pytest.mark.parametrize("tune", [0, 2])
def test_persistent_batch_equals_instances_stepped_alone(S, tune):
    """One persistent launch per order over all instances' tiles.  With the default tile
    shapes, bit for bit the generic kernel's result for every instance (same values, same
    weights, same order).  A tuned smaller tile collides each node on two lanes (even and odd
    velocities summed separately, then added), so there the results agree to FP32 round-off
    (the one-step tolerance of the FP32 parity tests, 2e-6 of the population scale)."""
    insts = I.batch_instances(10, 6)
    insts = [I.Instance(cells=(min(i.cells[0], 11),) * 3, p=i.p, Ma=min(i.Ma, 0.9), Re=i.Re,
                        courant=min(i.courant, 4.0)) for i in insts]
    from paper_2012_05537_gb300 import batch as BT
    sims = BT.make_instances(insts)
    alone = BT.make_instances(insts)
    for b in alone:
        b.set_variant(1)
    bt = BT.Batch(sims, autotune_steps=tune, persistent=True)
    shapes = bt.shapes()
    assert all(shapes[p] in ((0, 1, 2) if p in {i.p for i in insts} else (-1,)) for p in (2, 3, 4))
    bt.step(4)
    for b in alone:
        assert b.step(4) == 0
    torch.cuda.synchronize()
    for a, b in zip(sims, alone):
        if tune == 0:
            assert torch.equal(a.raw_state(), b.raw_state())
        else:
            x, y = a.raw_state().double(), b.raw_state().double()
            assert float((x - y).abs().max()) <= 2e-6 * 4 * float(y.abs().max())
    bt.close()


def test_persistent_batch_refuses_other_storage(S):
    sim = S.Sim(S.Config(cells=(2, 2, 2), p=2, storage="f64")).init_tgv()
    st = torch.cuda.Stream()
    with pytest.raises(S.SllbmError):
        S.sllbm_batch_create_persistent([sim.ctx], st.cuda_stream, 0)
