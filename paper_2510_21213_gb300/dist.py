"""Bookkeeping of runs on several GPUs of one node (one process per GPU).

The pair solves of different systems are independent, so ranks never exchange
data: each rank builds its own systems (seeds offset by rank) and the only
collectives are a barrier around a timed region and the maximum over ranks of
its duration. Throughput is the work of all ranks over that maximum (weak
scaling: the work per rank does not depend on the number of ranks).

One system can also be sharded: the pair solves of one exchange build are
independent too, so each rank solves a contiguous share of the sources and
one all-reduce of the partial K (N^2 doubles) and E_H finishes the build.

torch.distributed is plumbing here; any backend works (nccl on GPUs, gloo in
the CPU tests).
"""

from __future__ import annotations

import os

SEED_STRIDE = 1000


def env():
    """(world_size, rank, local_rank) from the torchrun environment (1, 0, 0 without it)."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def init(backend="nccl"):
    """Joins the process group when launched with more than one rank; returns (ws, rank, local)."""
    ws, rank, local = env()
    if ws > 1:
        import torch.distributed as dist

        if not dist.is_initialized():
            dist.init_process_group(backend)
    return ws, rank, local


def finish():
    import torch.distributed as dist

    if dist.is_available() and dist.is_initialized():
        dist.destroy_process_group()


def rank_seed(base, rank):
    """Seed of a rank's system: distinct per rank, the same on every run."""
    return base + SEED_STRIDE * rank


def rank_seeds(base, count, rank):
    """Seeds of a rank's `count` systems (weak scaling: count per rank)."""
    return [rank_seed(base, rank) + k for k in range(count)]


def barrier(sync_cuda=True):
    import torch

    if torch.distributed.is_available() and torch.distributed.is_initialized():
        torch.distributed.barrier()
    if sync_cuda and torch.cuda.is_available():
        torch.cuda.synchronize()


def max_over_ranks(seconds, device="cpu"):
    """The largest of the ranks' values (every rank gets it)."""
    import torch

    if not (torch.distributed.is_available() and torch.distributed.is_initialized()):
        return float(seconds)
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(units_per_rank, steps, max_seconds, world_size):
    """Whole-job throughput: units of all ranks over the slowest rank's time."""
    if max_seconds <= 0:
        raise ValueError("non-positive time")
    return world_size * units_per_rank * steps / max_seconds


# ---------------------------------------------------------------------------
# one system sharded over ranks: each rank solves a contiguous range of the
# sources (0 = Hartree density, then the pairs) and returns its part of K; one
# all-reduce (sum) of the N x N partial K and of E_H gives the whole build
# ---------------------------------------------------------------------------
def shard_range(n_items, world_size, rank):
    """[begin, end) of rank's share of n_items: contiguous, sizes differ by at
    most one (the sources of one system cost about the same)."""
    if world_size < 1 or not 0 <= rank < world_size:
        raise ValueError("bad rank")
    base, extra = divmod(int(n_items), int(world_size))
    begin = rank * base + min(rank, extra)
    return begin, begin + base + (1 if rank < extra else 0)


def allreduce_sum(values, device="cpu"):
    """Element-wise sum over ranks of a float64 array (every rank gets it)."""
    import numpy as np
    import torch

    arr = np.asarray(values, dtype=np.float64)
    if not (torch.distributed.is_available() and torch.distributed.is_initialized()):
        return arr.copy()
    t = torch.tensor(arr, dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.SUM)
    return t.cpu().numpy()


def sharded_exchange(partial, n_orbitals, world_size, rank, device="cpu"):
    """Whole-system K, E_H and E_X = -1/2 tr K from this rank's share.
    partial(begin, end) -> (K_partial [N, N], E_H or 0) computes the share
    (the library's dg_exchange_build_range, or any stand-in with its contract)."""
    import numpy as np

    total = n_orbitals * (n_orbitals + 1) // 2 + 1
    begin, end = shard_range(total, world_size, rank)
    K_part, eh = partial(begin, end)
    red = allreduce_sum(np.concatenate([np.asarray(K_part, dtype=np.float64).reshape(-1), [eh]]), device)
    K = red[:-1].reshape(n_orbitals, n_orbitals)
    return K, float(red[-1]), -0.5 * float(np.trace(K))
