"""Host logic for several GPUs: one process per GPU, work split by independent units.

The propagation, PSF and render of distinct (request, wavelength) slices are independent
(Sec. 3.1 evaluates every wavelength with its own transfer function), so ranks split the
slices and exchange nothing; the benchmark runs one replica of its step per rank.  The
objective of Eq. 4 sums over wavelengths, so its gradient is the sum of per-wavelength
gradients: a wavelength-split gradient ends with one all-reduce (sum) of dL/dh and of the
loss.  Timings are reduced with the maximum over ranks.

Every collective goes through torch.distributed (NCCL between GPUs, gloo on the host), on
tensors of the backend's device.
"""
from __future__ import annotations


def shard(n: int, rank: int, world: int) -> range:
    """Contiguous, balanced block of range(n) owned by `rank` (the first n mod world ranks
    take one extra item); empty when n < world for the surplus ranks."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"rank {rank} outside world of size {world}")
    q, r = divmod(n, world)
    lo = rank * q + min(rank, r)
    return range(lo, lo + q + (1 if rank < r else 0))


def _device():
    import torch
    import torch.distributed as dist

    return torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else torch.device("cpu")


def max_over_ranks(x: float) -> float:
    """Maximum of a per-rank scalar (a multi-GPU step ends when its slowest rank ends); identity
    without a process group."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=_device())
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def grad_split_wavelengths(lambdas, grad_fn, shape):
    """dL/dh and loss of Eq. 4 with the wavelengths split over the ranks.

    grad_fn(sub_lambdas) -> (grad tensor of `shape`, loss scalar tensor) computes this rank's
    share (the GPU path passes a closure over api.grad); a rank with no wavelengths
    contributes zeros.  Returns the all-reduced (grad, loss) on every rank."""
    import torch
    import torch.distributed as dist

    world = dist.get_world_size() if dist.is_available() and dist.is_initialized() else 1
    rank = dist.get_rank() if world > 1 else 0
    mine = shard(len(lambdas), rank, world)
    dev = _device() if world > 1 else None
    if len(mine):
        g, loss = grad_fn([lambdas[j] for j in mine])
        g = g.to(torch.float64)
        loss = torch.as_tensor(loss, dtype=torch.float64).reshape(1)
    else:
        g = torch.zeros(shape, dtype=torch.float64)
        loss = torch.zeros(1, dtype=torch.float64)
    if world > 1:
        g, loss = g.to(dev), loss.to(dev)
        dist.all_reduce(g, op=dist.ReduceOp.SUM)
        dist.all_reduce(loss, op=dist.ReduceOp.SUM)
    return g, loss
