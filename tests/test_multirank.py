"""The multi-rank path of bench.py on CPU (gloo, world size 2): each rank marches a
disjoint, contiguous share of the plane waves that together cover them all, and the
reported time is the largest of the ranks' times (the same helpers the GPU run uses,
with the CPU device)."""
import os
import socket

import numpy as np
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, ws, port, n_waves, out):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    import bench

    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        share = bench.wave_share(n_waves, ws, rank)
        t = bench.reduce_max(1.0 + 0.5 * rank, ws, device="cpu")
        bench.barrier(ws)
        out.put((rank, share.tolist(), t))
    finally:
        dist.destroy_process_group()


def test_two_ranks_share_waves_and_report_the_slowest():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, 16, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    shares = [r[1] for r in res]
    assert shares[0] + shares[1] == list(range(16)) and len(shares[0]) == len(shares[1]) == 8
    assert all(r[2] == 1.5 for r in res)
    # an uneven split stays contiguous, disjoint and covering
    import bench

    assert [bench.wave_share(5, 2, r).tolist() for r in range(2)] == [[0, 1, 2], [3, 4]]
    assert np.concatenate([bench.wave_share(7, 3, r) for r in range(3)]).tolist() == list(range(7))
