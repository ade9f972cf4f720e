"""The N > 1 host path on CPU: two gloo ranks, each with its own Philox key,
combine their dipoles into the dipole of the union ensemble (computed here
by the oracle on both ranks' trajectories at once), and agree on the
slowest rank's time."""
import os
import socket

import numpy as np
import torch.multiprocessing as mp

import oracle as O
from paper_2608_13686_b300 import replicas
from paper_2608_13686_b300 import workloads as W

T, P, AL = W.TARGETS["H2"], W.PULSE_800, W.fixed(20.0)
NS = (48, 29)          # trajectories per rank
SEED = 7


def _port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    soa, _, _ = O.sample(T, P, AL, seed=replicas.rank_seed(SEED, rank), n=NS[rank])
    vz, _, _ = O.propagate(T, P, soa, W.GAMMA, cutoff=W.CUTOFF, stab_cutoff=W.STAB_CUTOFF,
                           n_threads=1)
    comb = replicas.combine_dipoles(vz, NS[rank])
    slowest = replicas.max_over_ranks(10.0 + rank)
    q.put((rank, comb, slowest, soa[0].copy()))
    dist.destroy_process_group()


def test_two_gloo_ranks_combine_to_the_union_ensemble():
    O.build()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = {}
    for _ in procs:
        r, comb, slowest, births = q.get(timeout=300)
        res[r] = (comb, slowest, births)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # union ensemble on the oracle, normalised by all trajectories
    s0, _, _ = O.sample(T, P, AL, seed=replicas.rank_seed(SEED, 0), n=NS[0])
    s1, _, _ = O.sample(T, P, AL, seed=replicas.rank_seed(SEED, 1), n=NS[1])
    both = np.concatenate([s0, s1], axis=1)
    vz, _, _ = O.propagate(T, P, both, W.GAMMA, cutoff=W.CUTOFF, stab_cutoff=W.STAB_CUTOFF)
    for r in (0, 1):
        comb, slowest, _ = res[r]
        assert np.max(np.abs(comb - vz)) <= 1e-12 * np.max(np.abs(vz))
        assert slowest == 11.0
    # the ranks drew different trajectories
    assert not np.array_equal(res[0][2][:NS[1]], res[1][2])
