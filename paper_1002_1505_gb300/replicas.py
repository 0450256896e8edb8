"""Several GPUs as independent replicas (host logic, any torch.distributed backend).

The systems A P = E_inc of different orientations and polarizations are
independent: they share only the Green tensor, which each GPU builds for
itself.  So N GPUs run N replicas with no exchange on the data path -- the
way DDSCAT farms orientations over MPI ranks (guide, sections "MPI: Message
Passing Interface" and "Code Execution Under MPI") -- and
the only communication is the reduction of scalars at the end:

    shard(n, rank, world)                  a rank's contiguous, balanced share of n orientations
    orientation_average_sharded(q, w, ...) the guide's weighted orientation average
                                           (section "Orientational Averaging") from every rank's share
    reduce_max_sum(t, u)                   slowest rank's time and all ranks' work (benchmark line)

Reductions run on CPU tensors under gloo and on the current CUDA device under
NCCL; with no initialised process group they return the local values.
"""
from __future__ import annotations

from typing import Optional, Sequence, Tuple

import numpy as np


def shard(n: int, rank: int, world: int) -> Tuple[int, int]:
    """[start, stop) of rank's share of n items: contiguous, sizes differ by at most one."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    if n < 0:
        raise ValueError("n must be >= 0")
    base, extra = divmod(n, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def _dist():
    try:
        import torch.distributed as dist
    except ImportError:  # pragma: no cover - torch is always present here
        return None
    return dist if dist.is_available() and dist.is_initialized() else None


def _all_reduce(values: np.ndarray, op: str, group=None) -> np.ndarray:
    dist = _dist()
    if dist is None:
        return values
    import torch
    dev = torch.device("cpu")
    if dist.get_backend(group) == "nccl":
        dev = torch.device("cuda", torch.cuda.current_device())
    t = torch.as_tensor(np.ascontiguousarray(values, dtype=np.float64), device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM, group=group)
    return t.cpu().numpy()


def orientation_average_sharded(q_local, w_local: Sequence[float], iorth: int = 2, group=None) -> np.ndarray:
    """Weighted orientation average of per-RHS results over all ranks.

    q_local: this rank's results [n_local * iorth, ...] (RHS order: orientation-major, then
    polarization, as the library solves them); w_local: the guide's weights of this rank's
    orientations (all ranks' weights sum to one).  Returns [iorth, ...], identical on every rank:
    sum over all orientations o of w_o q[o, l].
    """
    q = np.asarray(q_local, dtype=np.float64)
    w = np.asarray(w_local, dtype=np.float64)
    q = q.reshape((len(w), iorth) + q.shape[1:])
    if len(w):
        from . import dda  # the weighted sum is the library's dda_orientation_average
        part = dda.dda_orientation_average(q, w, iorth)
    else:
        part = np.zeros((iorth,) + q.shape[2:])
    return _all_reduce(part, "sum", group).reshape(part.shape)


def reduce_max_sum(time_ms: float, units: float, group=None) -> Tuple[float, float]:
    """(maximum of time_ms, sum of units) over the ranks."""
    t = _all_reduce(np.array([time_ms]), "max", group)
    u = _all_reduce(np.array([units]), "sum", group)
    return float(t[0]), float(u[0])


def local_orientations(orientations: Sequence, weights: Optional[Sequence[float]], rank: int, world: int):
    """This rank's orientations (and their weights, if given) under `shard`."""
    a, b = shard(len(orientations), rank, world)
    return list(orientations[a:b]), (None if weights is None else list(weights[a:b]))
