"""Many independent SLLBM instances advanced together, as one CUDA graph per two steps of all
instances: either each instance's own step kernel on worker streams (``sllbm_batch_create``,
kernels chosen per instance by ``sllbm_autotune``), or one persistent launch per polynomial
order over a work list of (instance, tile) items (``sllbm_batch_create_persistent``, tile
shape per order chosen by its autotuner).  Argument marshalling only."""
from __future__ import annotations

import torch

from . import sllbm as S


class Batch:
    def __init__(self, sims, streams: int = 16, autotune_steps: int = 0, stream=None, persistent: bool = False):
        self.sims = list(sims)
        dev = self.sims[0].device
        self.stream = stream if stream is not None else torch.cuda.Stream(device=dev)
        self.tuned = []
        self.persistent = persistent
        if autotune_steps > 0 and not persistent:
            for s in self.sims:
                self.tuned.append(s.autotune(autotune_steps))
        torch.cuda.synchronize(dev)
        with torch.cuda.device(dev):
            if persistent:
                self.handle = S.sllbm_batch_create_persistent([s.ctx for s in self.sims], self.stream.cuda_stream,
                                                              autotune_steps)
            else:
                self.handle = S.sllbm_batch_create([s.ctx for s in self.sims], streams, self.stream.cuda_stream)

    def shapes(self):
        """Tile shape per order of a persistent batch."""
        return S.sllbm_batch_shapes(self.handle)

    def step(self, nsteps: int) -> None:
        """Advances every instance by nsteps (even) steps; asynchronous."""
        S.sllbm_batch_step(self.handle, nsteps)

    @property
    def nodes(self) -> int:
        return sum(s.nodes for s in self.sims)

    def close(self) -> None:
        if getattr(self, "handle", None):
            S.sllbm_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def make_instances(instances, storage: str = "f32", device=None):
    """A Sim per inputs.Instance, initialised with its Taylor-Green state."""
    sims = []
    for inst in instances:
        cfg = S.Config(cells=inst.cells, p=inst.p, Ma=inst.Ma, Re=inst.Re, courant=inst.courant, storage=storage)
        sims.append(S.Sim(cfg, device=device).init_tgv())
    return sims
