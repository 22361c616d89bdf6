"""The multi-rank path on CPU (gloo, world size 2): each rank draws its own
batch of the same family, the job time is the max over ranks and the job
rate counts every rank's units (weak scaling, no data-path collective)."""
import os
import socket

import numpy as np
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist

    from paper_2604_06575_b300 import dist as pdist
    from paper_2604_06575_b300 import workloads
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, lr = pdist.rank_info()
    polys, Xs = workloads.batched_uneven(seed_off=pdist.workload_seed_offset(r), n_polys=3, t_hi=200, p_hi=300)
    npts = sum(X.shape[0] for X in Xs)
    my_ms = 10.0 * (r + 1)  # a slower second rank
    pdist.barrier()
    mx = pdist.max_over_ranks(my_ms)
    q.put((r, w, npts, float(Xs[0][0, 0]), mx, pdist.job_rate(npts, w, 2, mx)))
    dist.destroy_process_group()


def test_two_ranks_weak_scaling():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, w0, n0, x0, m0, j0), (r1, w1, n1, x1, m1, j1) = res
    assert (r0, r1, w0, w1) == (0, 1, 2, 2)
    assert x0 != x1                      # different batches per rank
    assert m0 == m1 == 20.0              # the slowest rank sets the job time
    assert np.isclose(j0, n0 * 2 * 2 / 20e-3)
