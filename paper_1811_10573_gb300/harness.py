"""Process-group plumbing for the benchmark: rank discovery, barriers and the
max-over-ranks reduction of timings.  The decomposition itself never
communicates (one independent problem per GPU); only timings cross ranks.
"""
from __future__ import annotations

import os
from dataclasses import dataclass


@dataclass
class Dist:
    rank: int = 0
    world: int = 1
    local_rank: int = 0
    active: bool = False

    def barrier(self):
        if self.active:
            import torch.distributed as dist
            dist.barrier()

    def max(self, value: float) -> float:
        """Maximum of a float over ranks (identity on one process)."""
        if not self.active:
            return float(value)
        import torch
        import torch.distributed as dist
        dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
        t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    def gather(self, value: float) -> list:
        if not self.active:
            return [float(value)]
        import torch
        import torch.distributed as dist
        dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
        t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
        out = [torch.zeros_like(t) for _ in range(self.world)]
        dist.all_gather(out, t)
        return [float(x.item()) for x in out]

    def close(self):
        if self.active:
            import torch.distributed as dist
            dist.destroy_process_group()
            self.active = False


def init(backend: str | None = None) -> Dist:
    """Join the process group when launched by torchrun (WORLD_SIZE > 1)."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if world <= 1:
        return Dist()
    import torch
    import torch.distributed as dist
    rank = int(os.environ["RANK"])
    local = int(os.environ.get("LOCAL_RANK", rank))
    if backend is None:
        backend = "nccl" if torch.cuda.is_available() else "gloo"
    if backend == "nccl":
        torch.cuda.set_device(local)
    os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
    dist.init_process_group(backend=backend, rank=rank, world_size=world)
    return Dist(rank=rank, world=world, local_rank=local, active=True)
