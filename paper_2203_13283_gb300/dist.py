"""Host-side logic of multi-GPU runs (one process per GPU).

The solve of one batch of right-hand sides has no exchange step: every
plane-wave column is an independent solve against the same factors (Eq. 9),
so ranks either hold replicas of the whole setup and solve their own batch
(weak scaling, what the benchmark reports), or split one batch of columns
between them.  Neither needs a collective on the data path; the only
communication is the reduction of timings at the end of a measurement.

The shape gradient shards the same way: its parameters are independent
(each needs only the shared forward and adjoint currents), so each rank
takes a contiguous range of them and the pieces are gathered once at the end.
"""

import os


def world():
    """(rank, world size, local rank) from the launcher's environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def shard_columns(B, rank, world_size):
    """Contiguous share [c0, c1) of B right-hand-side columns for one rank;
    shares differ in size by at most one and cover 0..B-1 exactly once."""
    if world_size < 1 or not 0 <= rank < world_size or B < 0:
        raise ValueError("bad shard request")
    q, r = divmod(B, world_size)
    c0 = rank * q + min(rank, r)
    return c0, c0 + q + (1 if rank < r else 0)


def max_over_ranks(values, device=None):
    """Element-wise maximum of a list of floats over all ranks (the slowest
    rank sets the time of a step); identity on a single process."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return list(values)
    t = torch.tensor(list(values), dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def job_throughput(units_per_rank, world_size, seconds_max):
    """Whole-job rate: units processed by all ranks over the slowest rank's time."""
    return units_per_rank * world_size / seconds_max


def gather_shards(local, n, device=None):
    """The length-n vector whose contiguous shares (as shard_columns assigns
    them) are held by the ranks: every rank passes its own share and gets the
    whole vector.  Identity on a single process."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return list(local)
    w, r = dist.get_world_size(), dist.get_rank()
    c0, c1 = shard_columns(n, r, w)
    if len(local) != c1 - c0:
        raise ValueError("local share has the wrong length")
    width = -(-n // w) if n else 0
    t = torch.zeros(max(width, 1), dtype=torch.float64, device=device)
    if c1 > c0:
        t[:c1 - c0] = torch.as_tensor(list(local), dtype=torch.float64, device=device)
    parts = [torch.zeros_like(t) for _ in range(w)]
    dist.all_gather(parts, t)
    out = []
    for q in range(w):
        a, b = shard_columns(n, q, w)
        out.extend(parts[q][:b - a].tolist())
    return out


def sharded_shape_gradient(solver, angles, phi_obs, M, delta=1e-6, device=None, **kw):
    """(J, grad) of Solver.shape_gradient with the 2M parameters split over
    the ranks of the default process group: each rank evaluates its range on
    its own GPU and the ranges are gathered (one all-gather of 2M numbers)."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        r, w = dist.get_rank(), dist.get_world_size()
    else:
        r, w = 0, 1
    i0, i1 = shard_columns(2 * int(M), r, w)
    J, g = solver.shape_gradient(angles, phi_obs, M, delta=delta, params=(i0, i1), **kw)
    return J, gather_shards(g, 2 * int(M), device=device)
