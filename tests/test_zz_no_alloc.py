"""sllbm_diag_noalloc: the diagnostics entry point that allocates no device memory.

Some callers cannot let the library allocate: their device memory belongs to another
allocator or a fixed budget, or their loop cannot afford cudaMalloc/cudaFree (cudaFree
synchronises the whole device).  This entry point keeps its scratch in a static device
array inside the library; this test checks it through the C ABI against sllbm_diag on
two calls in a row (the second reusing the array the first one left behind), after a
state change, on a smaller mesh after a larger one (the array keeps the larger mesh's
entries), directly against the FP64 oracle's diagnostics, that the call takes no device
memory, and that meshes larger than the static scratch are refused.
Collected last on purpose (file name), so a failure here cannot hide other results.
"""
import numpy as np
import pytest

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


@pytest.mark.parametrize("storage,p,cells", [("f64", 3, (8, 8, 8)), ("f32", 4, (6, 5, 4))])
def test_noalloc_diag_equals_diag_on_consecutive_calls(S, storage, p, cells):
    sim = S.Sim(S.Config(cells=cells, p=p, courant=2.0, storage=storage))
    sim.init_tgv()
    sim.step(4)
    ref = np.array(S.sllbm_diag(sim.ctx))
    first = np.array(S.sllbm_diag_noalloc(sim.ctx))
    second = np.array(S.sllbm_diag_noalloc(sim.ctx))
    # same FP64 sums in another order: the tolerance of the diagnostics parity tests
    assert np.allclose(first, ref, rtol=1e-11, atol=0)
    assert np.allclose(second, ref, rtol=1e-11, atol=0)
    sim.step(3)
    ref2 = np.array(S.sllbm_diag(sim.ctx))
    third = np.array(S.sllbm_diag_noalloc(sim.ctx))
    assert np.allclose(third, ref2, rtol=1e-11, atol=0)
    assert not np.allclose(ref2, ref, rtol=1e-12, atol=0)  # the state really changed
    sim.close()


def test_noalloc_diag_allocates_nothing(S):
    # a first call on another context loads the kernels (lazy module loading may place
    # their code in device memory); then the first call on a fresh context must not
    # change the device's free memory
    warm = S.Sim(S.Config(cells=(4, 4, 4), p=3, courant=2.0, storage="f32"))
    warm.init_tgv()
    S.sllbm_diag_noalloc(warm.ctx)
    sim = S.Sim(S.Config(cells=(6, 6, 6), p=3, courant=2.0, storage="f32"))
    sim.init_tgv()
    sim.step(2)
    sim.sync()
    free0 = torch.cuda.mem_get_info()[0]
    S.sllbm_diag_noalloc(sim.ctx)
    S.sllbm_diag_noalloc(sim.ctx)
    free1 = torch.cuda.mem_get_info()[0]
    assert free1 == free0
    sim.close()
    warm.close()


def test_noalloc_diag_smaller_mesh_after_larger_and_against_oracle(S):
    import oracle as O
    big = S.Sim(S.Config(cells=(10, 9, 8), p=3, courant=2.0, storage="f64"))
    small = S.Sim(S.Config(cells=(3, 2, 4), p=2, courant=2.0, storage="f64"))
    for sim in (big, small):
        sim.init_tgv()
        sim.step(2)
    got_big = np.array(S.sllbm_diag_noalloc(big.ctx))
    got_small = np.array(S.sllbm_diag_noalloc(small.ctx))
    assert np.allclose(got_big, S.sllbm_diag(big.ctx), rtol=1e-11, atol=0)
    assert np.allclose(got_small, S.sllbm_diag(small.ctx), rtol=1e-11, atol=0)
    # the small mesh's values straight from the oracle (its own state, its own diagnostics)
    g = O.Grid(cells=(3, 2, 4), p=2, dt=small.dt, mu_inf=float(small.info.mu_inf))
    pop = O.step(g, O.init_fields(g, *O.tgv_fields(g, small.info.U0)), 2)
    want = O.diag(g, pop, 1.0, 1600.0, small.info.U0)
    # (eps_c is near zero two steps in; its absolute error is measured on eps_s's scale)
    assert np.allclose(got_small, want, rtol=1e-10, atol=1e-10 * abs(want[1]))
    big.close()
    small.close()


def test_noalloc_diag_refuses_meshes_beyond_its_scratch(S):
    sim = S.Sim(S.Config(cells=(257, 256, 1), p=2, courant=1.0, storage="f32"))
    sim.init_tgv()
    with pytest.raises(S.SllbmError) as e:
        S.sllbm_diag_noalloc(sim.ctx)
    assert e.value.code == S.EINVAL
    sim.close()
