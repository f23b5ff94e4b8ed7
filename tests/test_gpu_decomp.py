"""z-decomposition on one GPU: slab contexts that exchange halos before every step
(sllbm_halo_pack / sllbm_halo_unpack, several slabs of one process) must reproduce the
undivided periodic mesh bit for bit: the same source values reach every node, with the same
weights, in the same order.  Also the calls that refuse slab contexts."""
import ctypes
import dataclasses

import numpy as np
import pytest

from paper_2012_05537_gb300 import decomp as D
from paper_2012_05537_gb300 import sllbm as S

pytestmark = pytest.mark.gpu


def _full(cfg, n, kernel=1, compensated=False):
    sim = S.Sim(dataclasses.replace(cfg, kernel=kernel), device="cuda:0")
    if compensated:
        S.sllbm_set_compensated(sim.ctx, True)
    assert sim.info.step_kernel == kernel
    sim.init_tgv()
    init = sim.populations().cpu().numpy()
    assert sim.step(n) == 0
    out = sim.populations().cpu().numpy()
    sim.close()
    return init, out


def _slabs(cfg, parts, n, overlapped=False, kernel=1, compensated=False):
    steppers = []
    for r in range(parts):
        sim = S.Sim(dataclasses.replace(cfg, slab=D.slab_bounds(cfg.cells[2], parts, r), kernel=kernel),
                    device="cuda:0")
        if compensated:
            S.sllbm_set_compensated(sim.ctx, True)
        sim.init_tgv()
        assert sim.info.step_kernel == kernel
        steppers.append(D.SlabStepper(sim))

    def interiors():
        parts_ = []
        for st in steppers:
            g, zc, p = st.ghost, st.sim.cfg.slab[1], cfg.p
            parts_.append(st.sim.populations().cpu().numpy()[:, :, g * p:(g + zc) * p])
        return np.concatenate(parts_, axis=2)

    init = interiors()
    if overlapped:
        D.step_local_overlapped(steppers, n)
    else:
        D.step_local(steppers, n)
    out = interiors()
    ghost = steppers[0].ghost
    for st in steppers:
        st.sim.close()
    return init, out, ghost


@pytest.mark.parametrize("storage", ["f64", "f32"])
@pytest.mark.parametrize("p", [2, 3, 4])
@pytest.mark.parametrize("parts", [1, 2, 3])
def test_slabs_reproduce_the_whole_mesh_bit_for_bit(storage, p, parts):
    cfg = S.Config(cells=(4, 3, 9), p=p, courant=2.0, storage=storage)
    init_full, full = _full(cfg, 4)
    init_slab, slab, ghost = _slabs(cfg, parts, 4)
    assert ghost == 2
    assert np.array_equal(init_slab, init_full)
    assert np.all(np.isfinite(full))
    assert np.array_equal(slab, full)


@pytest.mark.parametrize("storage", ["f64", "f32"])
@pytest.mark.parametrize("p", [3, 4])
@pytest.mark.parametrize("parts", [1, 2, 3])
def test_overlapped_exchange_reproduces_the_whole_mesh(storage, p, parts):
    # the exchange on a second stream while the tiles that read no ghost cell run
    cfg = S.Config(cells=(4, 3, 12), p=p, courant=2.0, storage=storage)
    _, full = _full(cfg, 4)
    _, slab, _ = _slabs(cfg, parts, 4, overlapped=True)
    assert np.array_equal(slab, full)


@pytest.mark.parametrize("p,parts,storage", [(4, 1, "f32"), (4, 2, "f32"), (4, 3, "f32"), (2, 1, "f32"),
                                             (2, 2, "f32"), (3, 1, "f32"), (3, 2, "f32"), (3, 2, "f16dev"),
                                             (2, 2, "f16dev"), (4, 3, "bf16dev")])
@pytest.mark.parametrize("overlapped", [False, True])
def test_tma_fed_slabs_reproduce_the_whole_mesh(p, parts, storage, overlapped):
    # the TMA-fed kernel on slabs (tiles over the interior cells, source boxes reaching into
    # the ghost planes) against the same kernel on the undivided mesh (whose boxes that wrap
    # around along z arrive as zero-filled periodic images, summed exactly)
    cfg = S.Config(cells=(4, 4, 8), p=p, courant=2.0, storage=storage)
    _, full = _full(cfg, 4, kernel=2)
    _, slab, _ = _slabs(cfg, parts, 4, overlapped=overlapped, kernel=2)
    assert np.all(np.isfinite(full))
    assert np.array_equal(slab, full)


@pytest.mark.parametrize("p,parts,storage,overlapped", [(4, 2, "f32", False), (3, 2, "f32", False),
                                                        (2, 2, "f32", True), (3, 2, "f16dev", False),
                                                        (2, 2, "f16dev", False), (4, 3, "bf16dev", True)])
def test_tma_fed_slabs_with_compensated_sums_reproduce_the_whole_mesh(p, parts, storage, overlapped):
    # compensated moment sums (sllbm_set_compensated) run in the epilogue, after the
    # streaming: slabs stay bit-equal to the undivided mesh, the TMA-fed kernel on both
    cfg = S.Config(cells=(4, 4, 8), p=p, courant=2.0, storage=storage)
    _, full = _full(cfg, 4, kernel=2, compensated=True)
    _, plain = _full(cfg, 4, kernel=2)
    _, slab, _ = _slabs(cfg, parts, 4, overlapped=overlapped, kernel=2, compensated=True)
    assert np.all(np.isfinite(full))
    assert np.array_equal(slab, full)
    if storage == "f32":
        assert not np.array_equal(full, plain)  # (the compensated instance did run)


@pytest.mark.parametrize("kernel,p,storage", [(1, 3, "f64"), (1, 4, "f32"), (2, 4, "f32"), (2, 2, "f32"),
                                              (2, 3, "f16dev"), (2, 4, "bf16dev"), (2, 3, "f32")])
def test_periodic_halo_refresh_of_a_whole_mesh_slab(kernel, p, storage):
    # one slab spanning the mesh, its ghost planes refreshed in place before every step (by
    # sllbm_step itself: sllbm_halo_periodic), against the ordinary periodic context on the
    # same kernel
    cfg = S.Config(cells=(4, 4, 8), p=p, courant=2.0, storage=storage)
    _, full = _full(cfg, 4, kernel=kernel)
    sim = S.Sim(dataclasses.replace(cfg, slab=(0, 8), kernel=kernel), device="cuda:0")
    assert sim.info.step_kernel == kernel
    sim.init_tgv()
    g = S.sllbm_slab_info(sim.ctx)[0]
    for k in range(4):
        if k % 2:
            S.sllbm_halo_periodic(sim.ctx)  # explicit refreshes on top of the step's own are harmless
        assert sim.step(1) == 0
    got = sim.populations().cpu().numpy()[:, :, g * p:(g + 8) * p]
    assert np.array_equal(got, full)
    half = S.Sim(dataclasses.replace(cfg, slab=(0, 4)), device="cuda:0")  # not the whole mesh
    with pytest.raises(S.SllbmError):
        S.sllbm_halo_periodic(half.ctx)
    sim.close()
    half.close()


@pytest.mark.parametrize("kernel,p,storage", [(1, 3, "f64"), (2, 4, "f32"), (2, 3, "f16dev")])
def test_diagnostics_of_a_whole_mesh_slab(kernel, p, storage):
    # E_k, eps_s, eps_c of a slab spanning the whole mesh (its interior, the support points
    # wrapping around within it) equal those of the ordinary periodic context bit for bit: the
    # states are the same and the cells are visited in the same order
    cfg = S.Config(cells=(4, 6, 8), p=p, courant=2.0, storage=storage, kernel=kernel)
    a = S.Sim(cfg, device="cuda:0")
    b = S.Sim(dataclasses.replace(cfg, slab=(0, 8)), device="cuda:0")
    for sim in (a, b):
        sim.init_tgv()
        assert sim.step(3) == 0
    da, db = a.diag(), b.diag()
    assert all(np.isfinite(da)) and tuple(da) == tuple(db)
    assert np.allclose(S.sllbm_diag_noalloc(b.ctx), db, rtol=1e-13, atol=0)  # (another summation order)
    a.close()
    b.close()


def test_overlapped_exchange_on_slabs_without_interior_tiles():
    # two-cell slabs with two ghost cells: every tile reads a ghost cell (all in the second launch)
    cfg = S.Config(cells=(3, 3, 6), p=3, courant=2.0, storage="f64")
    _, full = _full(cfg, 3)
    _, slab, ghost = _slabs(cfg, 3, 3, overlapped=True)
    assert ghost == 2
    assert np.array_equal(slab, full)


def test_wider_halo_at_a_larger_courant_number():
    # departures up to two cells: three ghost cells per side, slabs of three cells
    cfg = S.Config(cells=(3, 3, 9), p=2, courant=4.0, storage="f64")
    _, full = _full(cfg, 3)
    _, slab, ghost = _slabs(cfg, 3, 3)
    assert ghost == 3
    assert np.array_equal(slab, full)


def test_slab_refusals():
    base = S.Config(cells=(4, 4, 8), p=4, courant=2.0, storage="f32")
    with pytest.raises(S.SllbmError):  # thinner than its ghost width
        S.Sim(dataclasses.replace(base, slab=(0, 1)), device="cuda:0")
    with pytest.raises(S.SllbmError):  # outside the mesh
        S.Sim(dataclasses.replace(base, slab=(8, 2)), device="cuda:0")
    with pytest.raises(S.SllbmError):  # the TMA-fed kernel cannot tile 3 x 4 x 4 cells at p = 4
        S.Sim(dataclasses.replace(base, cells=(3, 4, 8), slab=(0, 4), kernel=2), device="cuda:0")
    sim = S.Sim(dataclasses.replace(base, slab=(0, 4)), device="cuda:0")
    sim.init_tgv()
    lib = S.load()
    d = [ctypes.c_double() for _ in range(3)]
    assert lib.sllbm_diag(sim.ctx, *[ctypes.byref(x) for x in d]) == S.EINVAL
    assert lib.sllbm_set_step_variant(sim.ctx, 0) == S.OK  # the TMA-fed kernel tiles this slab
    st = D.SlabStepper(sim)
    assert lib.sllbm_halo_pack(sim.ctx, 2, ctypes.c_void_p(st.bufs["send_low"].data_ptr()), None) == S.EINVAL
    assert lib.sllbm_halo_unpack(sim.ctx, 0, None, None) == S.EINVAL
    state = sim.raw_state().clone()
    out = sim.state_like()
    dmu = sim.torch.zeros(1, dtype=sim.torch.float64, device=sim.device)
    assert lib.sllbm_adjoint_step(sim.ctx, ctypes.c_void_p(state.data_ptr()), ctypes.c_void_p(state.data_ptr()),
                                  ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(dmu.data_ptr())) == S.EINVAL
    sim.close()
    whole = S.Sim(base, device="cuda:0")
    with pytest.raises(S.SllbmError):  # not a slab
        S.sllbm_slab_info(whole.ctx)
    assert lib.sllbm_step_begin(whole.ctx) == S.EINVAL
    assert lib.sllbm_step_end(whole.ctx) == S.EINVAL
    whole.close()
