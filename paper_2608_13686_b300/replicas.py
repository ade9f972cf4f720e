"""Several GPUs as independent replicas (one process per GPU).

The method's trajectories are independent, so N GPUs run N ensembles with no
exchange during propagation: each rank samples its own trajectories with its
own Philox key.  Two host-side steps span the ranks:
  * the job's time is the slowest rank's (max over ranks), and
  * when one estimate over all ranks is wanted, the rank dipoles, each
    normalised 1/N_r over its own N_r trajectories, combine into the estimate
    of the union ensemble, v = sum_r N_r v_r / sum_r N_r: one all-reduce of
    Nt doubles.
These run over any torch.distributed backend (NCCL on GPUs, gloo on CPU).
"""
from __future__ import annotations

import numpy as np


def rank_seed(seed: int, rank: int) -> int:
    """Philox key of a rank: distinct for every rank of one job."""
    return int(seed) + 1000 * int(rank)


def max_over_ranks(x: float) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64)
    if dist.get_backend() == "nccl":
        t = t.cuda()
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def combine_dipoles(vz, n_traj: int):
    """Union-ensemble dipole from every rank's (vz, n_traj); every rank gets it."""
    import torch
    import torch.distributed as dist
    vz = np.asarray(vz, dtype=np.float64)
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return vz.copy()
    buf = torch.from_numpy(np.concatenate([vz * float(n_traj), [float(n_traj)]]))
    if dist.get_backend() == "nccl":
        buf = buf.cuda()
    dist.all_reduce(buf, op=dist.ReduceOp.SUM)
    out = buf.cpu().numpy()
    return out[:-1] / out[-1]
