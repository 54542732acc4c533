"""Multi-process host logic of bench.py on CPU ranks (gloo, world size 2): each rank runs its
own replica channel (seed + rank) through the CPU oracle, and the job time is the maximum
over ranks. No GPU is used."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out_dir):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import numpy as np
    import bench
    from oracle import oracle as O
    from paper_1512_08042_gb300 import workloads as W

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    cfg = bench.replica_config(W.config(ncx=8, ncy=4, ppc=12, lb_ratio=2, seed=40), rank)
    nodes, cells = W.coupling_sites(cfg, strip_cells=2)
    o = O.Oracle(cfg)
    for _ in range(2):
        o.dsmc_step(1)
        o.map_dsmc_to_lbm(nodes)
        o.lbm_step(1)
        o.map_lbm_to_dsmc(cells)
    checksum = float(np.sum(o.particles()["vx"].astype(np.float64)))
    fake_ms = 10.0 + 5.0 * rank
    job_ms = bench.max_over_ranks(dist, fake_ms, "cpu")
    dist.barrier()
    with open(os.path.join(out_dir, "rank%d.txt" % rank), "w") as fh:
        fh.write("%r %r %d\n" % (checksum, job_ms, cfg["seed"]))
    dist.destroy_process_group()


def test_replicas_on_two_gloo_ranks(tmp_path):
    port = _free_port()
    mp.spawn(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    res = []
    for r in range(2):
        chk, job_ms, seed = open(tmp_path / ("rank%d.txt" % r)).read().split()
        res.append((float(chk), float(job_ms), int(seed)))
    # every rank sees the slowest rank's time
    assert res[0][1] == res[1][1] == 15.0
    # independent replicas: different keys, different particles
    assert res[0][2] != res[1][2]
    assert res[0][0] != res[1][0]
