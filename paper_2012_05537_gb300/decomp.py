"""Domain decomposition of one periodic mesh along z.

Each part is a slab context (``sllbm_create_slab``): its interior z-cells plus ``ghost``
cells of halo below and above.  The pull streaming of Sec. II.A reads, for a node, the
support points of the cell its departure point falls in, at most ``max_cell_shift`` cells
away, so one halo exchange with the two neighbouring slabs before every step makes the
slabs advance exactly as the whole mesh does.  The exchange is the only data movement
between parts; the collision is node-local.

Parts are ranks of a ``torch.distributed`` group (one GPU each; NCCL point-to-point on GPU
buffers) or, on one device, several slab contexts of one process (``exchange_local``).
"""
from __future__ import annotations


def slab_bounds(z_cells: int, parts: int, part: int) -> tuple[int, int]:
    """(z_begin, z_cells) of part ``part`` of ``parts``: consecutive slabs whose sizes differ
    by at most one cell."""
    if parts < 1 or not 0 <= part < parts or z_cells < parts:
        raise ValueError(f"cannot split {z_cells} cells into {parts} slabs (part {part})")
    base, extra = divmod(z_cells, parts)
    begin = part * base + min(part, extra)
    return begin, base + (1 if part < extra else 0)


def neighbours(rank: int, world: int) -> tuple[int, int]:
    """(rank below, rank above) on the periodic ring of slabs."""
    return (rank - 1) % world, (rank + 1) % world


def exchange(send_low, send_high, recv_low, recv_high, rank: int, world: int, group=None) -> None:
    """One halo exchange on the ring of slabs: ``send_low`` (the slab's lowest interior cells)
    goes to the rank below, whose halo above it becomes; ``send_high`` goes to the rank
    above; ``recv_low`` / ``recv_high`` receive the halos below / above.  With one rank the
    slab is its own neighbour on both sides.  With two ranks both messages of a rank go to
    the same peer; the receives are posted so that they match the sends in order (the
    peer's lowest cells lie above this slab, its highest below)."""
    if world == 1:
        recv_low.copy_(send_high)
        recv_high.copy_(send_low)
        return
    import torch.distributed as dist
    below, above = neighbours(rank, world)
    ops = [dist.P2POp(dist.isend, send_low, below, group),
           dist.P2POp(dist.isend, send_high, above, group),
           dist.P2POp(dist.irecv, recv_high, above, group),
           dist.P2POp(dist.irecv, recv_low, below, group)]
    for req in dist.batch_isend_irecv(ops):
        req.wait()


class SlabStepper:
    """Advances one slab ``Sim`` (created with ``Config(slab=...)``), exchanging its halos
    with the neighbouring ranks before every step."""

    def __init__(self, sim, rank: int = 0, world: int = 1, group=None):
        from . import sllbm as S
        self.sim, self.rank, self.world, self.group = sim, rank, world, group
        self.ghost, self.halo_bytes = S.sllbm_slab_info(sim.ctx)
        # what goes down (the neighbour's ghost planes above) and what goes up differ in
        # size: each velocity's halo holds only the planes its source boxes reach
        down, up = S.sllbm_slab_halo_bytes(sim.ctx, 0), S.sllbm_slab_halo_bytes(sim.ctx, 1)
        self.sizes = {"send_low": down, "recv_high": down, "send_high": up, "recv_low": up}
        torch = sim.torch
        self.bufs = {k: torch.empty(max(n, 1), dtype=torch.uint8, device=sim.device)[:n]
                     for k, n in self.sizes.items()}

    def pack(self, stream=None) -> None:
        from . import sllbm as S
        st = 0 if stream is None else stream.cuda_stream
        S.sllbm_halo_pack(self.sim.ctx, 0, self.bufs["send_low"].data_ptr(), st)
        S.sllbm_halo_pack(self.sim.ctx, 1, self.bufs["send_high"].data_ptr(), st)

    def unpack(self, stream=None) -> None:
        from . import sllbm as S
        st = 0 if stream is None else stream.cuda_stream
        S.sllbm_halo_unpack(self.sim.ctx, 0, self.bufs["recv_low"].data_ptr(), st)
        S.sllbm_halo_unpack(self.sim.ctx, 1, self.bufs["recv_high"].data_ptr(), st)

    def exchange(self) -> None:
        torch = self.sim.torch
        if self.world == 1:
            # the slab is the whole mesh along z: every step refreshes its ghost planes in
            # place (sllbm_halo_periodic inside sllbm_step), nothing to exchange
            return
        self.pack()
        # the collectives run after the packs (enqueued on the slab's stream) and before the
        # unpacks
        cur = torch.cuda.current_stream(self.sim.device)
        cur.wait_stream(self.sim.stream)
        b = self.bufs
        exchange(b["send_low"], b["send_high"], b["recv_low"], b["recv_high"], self.rank, self.world,
                 self.group)
        self.sim.stream.wait_stream(cur)
        self.unpack()

    def step(self, n: int = 1) -> None:
        for _ in range(n):
            self.exchange()
            rc = self.sim.step(1)
            if rc != 0:
                raise RuntimeError(f"sllbm_step returned {rc}")

    def step_overlapped(self, n: int = 1) -> None:
        """n steps with the halo exchange on a second stream, overlapped with the tiles that
        read no ghost cell (sllbm_step_begin); the tiles next to the ghost cells run once the
        halos are in (sllbm_step_end).  Same result as step(), bit for bit."""
        from . import sllbm as S
        torch = self.sim.torch
        if not hasattr(self, "comm"):
            self.comm = torch.cuda.Stream(device=self.sim.device)
        b = self.bufs
        for _ in range(n):
            self.comm.wait_stream(self.sim.stream)  # the current state is complete
            S.sllbm_step_begin(self.sim.ctx)
            self.pack(self.comm)
            with torch.cuda.stream(self.comm):
                exchange(b["send_low"], b["send_high"], b["recv_low"], b["recv_high"], self.rank, self.world,
                         self.group)
            self.unpack(self.comm)
            self.sim.stream.wait_stream(self.comm)
            S.sllbm_step_end(self.sim.ctx)


def exchange_local(steppers) -> None:
    """The halo exchange of several slabs held by one process (a ring in z order), by device
    copies on each slab's stream: every slab packs, then unpacks its neighbours' packed
    buffers directly."""
    from . import sllbm as S
    n = len(steppers)
    for st in steppers:
        st.pack()
    for k, st in enumerate(steppers):
        below, above = steppers[(k - 1) % n], steppers[(k + 1) % n]
        st.sim.stream.wait_stream(below.sim.stream)
        st.sim.stream.wait_stream(above.sim.stream)
        S.sllbm_halo_unpack(st.sim.ctx, 0, below.bufs["send_high"].data_ptr())
        S.sllbm_halo_unpack(st.sim.ctx, 1, above.bufs["send_low"].data_ptr())
    # a slab's next pack overwrites send buffers its neighbours copied from above
    for k, st in enumerate(steppers):
        st.sim.stream.wait_stream(steppers[(k - 1) % n].sim.stream)
        st.sim.stream.wait_stream(steppers[(k + 1) % n].sim.stream)


def step_local(steppers, n: int = 1) -> None:
    """Advances several slabs of one process by n steps (exchange, then one step each)."""
    for _ in range(n):
        exchange_local(steppers)
        for st in steppers:
            rc = st.sim.step(1)
            if rc != 0:
                raise RuntimeError(f"sllbm_step returned {rc}")


def step_local_overlapped(steppers, n: int = 1, comm=None):
    """As step_local, with the exchange on one extra stream `comm` overlapped with every
    slab's interior tiles (sllbm_step_begin / sllbm_step_end).  Returns the stream used."""
    from . import sllbm as S
    torch = steppers[0].sim.torch
    if comm is None:
        comm = torch.cuda.Stream(device=steppers[0].sim.device)
    k = len(steppers)
    for _ in range(n):
        for st in steppers:
            comm.wait_stream(st.sim.stream)  # every current state is complete
        for st in steppers:
            S.sllbm_step_begin(st.sim.ctx)
        for st in steppers:
            st.pack(comm)
        for j, st in enumerate(steppers):
            below, above = steppers[(j - 1) % k], steppers[(j + 1) % k]
            S.sllbm_halo_unpack(st.sim.ctx, 0, below.bufs["send_high"].data_ptr(), comm.cuda_stream)
            S.sllbm_halo_unpack(st.sim.ctx, 1, above.bufs["send_low"].data_ptr(), comm.cuda_stream)
        for st in steppers:
            st.sim.stream.wait_stream(comm)
            S.sllbm_step_end(st.sim.ctx)
    return comm
