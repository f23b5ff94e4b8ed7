"""Host logic of the z-decomposition on CPU: the slab split, and the ring halo exchange over
torch.distributed point-to-point with gloo ranks (world sizes 1, 2 and 3).  A slab's halo
cells must receive exactly the neighbouring slabs' boundary cells of the periodic mesh."""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_2012_05537_gb300 import decomp as D  # noqa: E402

# mesh cells along z, halo cells below and above a slab (unequal, as when each velocity's
# halo holds only the planes its departure points reach), values per cell
Z, GLOW, GHIGH, K = 10, 2, 1, 3


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _cells(first: int, count: int) -> torch.Tensor:
    """K values per cell, labelled by the cell's index on the periodic mesh."""
    idx = [(first + c) % Z for c in range(count)]
    return torch.tensor([[100.0 * i + k for k in range(K)] for i in idx], dtype=torch.float64).flatten()


def _exchange_on_rank(rank: int, world: int):
    z0, zc = D.slab_bounds(Z, world, rank)
    # down: the lowest cells, which the slab below keeps as its halo above (GHIGH cells);
    # up: the highest cells, the halo below of the slab above (GLOW cells)
    send_low, send_high = _cells(z0, GHIGH), _cells(z0 + zc - GLOW, GLOW)
    recv_low, recv_high = torch.full_like(send_high, -1.0), torch.full_like(send_low, -1.0)
    D.exchange(send_low, send_high, recv_low, recv_high, rank, world)
    return (recv_low.numpy(), recv_high.numpy(), _cells(z0 - GLOW, GLOW).numpy(),
            _cells(z0 + zc, GHIGH).numpy())


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        out[rank] = _exchange_on_rank(rank, world)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_slab_bounds_cover_the_mesh_once_with_even_sizes():
    for z in (3, 7, 10, 64):
        for parts in range(1, min(z, 6) + 1):
            spans = [D.slab_bounds(z, parts, r) for r in range(parts)]
            covered = [c for b, n in spans for c in range(b, b + n)]
            assert covered == list(range(z))
            sizes = [n for _, n in spans]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        D.slab_bounds(3, 4, 0)
    with pytest.raises(ValueError):
        D.slab_bounds(8, 2, 2)


def test_neighbours_form_a_periodic_ring():
    assert D.neighbours(0, 3) == (2, 1)
    assert D.neighbours(2, 3) == (1, 0)
    assert D.neighbours(0, 1) == (0, 0)


def test_single_slab_is_its_own_neighbour():
    got_low, got_high, want_low, want_high = _exchange_on_rank(0, 1)
    assert np.array_equal(got_low, want_low) and np.array_equal(got_high, want_high)


@pytest.mark.parametrize("world", [2, 3])
def test_ring_exchange_fills_halos_with_the_neighbours_cells(world):
    mp_ctx = mp.get_context("spawn")
    out = mp_ctx.Manager().dict()
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, start_method="spawn", join=True)
    for r in range(world):
        got_low, got_high, want_low, want_high = out[r]
        assert np.array_equal(got_low, want_low), f"rank {r}: halo below"
        assert np.array_equal(got_high, want_high), f"rank {r}: halo above"
