"""Multi-process host logic of bench.py on CPU ranks (gloo, world size 2): each rank runs its
own replica channel (seed + rank) through the CPU oracle, and the job time is the maximum
over ranks. No GPU is used."""
import os
import socket

import numpy as np
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


# ---------------------------------------------------------------------------------------
# The streamwise slab decomposition on CPU ranks: two oracle ranks, each the slab of half the
# channel's rows, exchange the particles that leave their slab and the LB rows next to their
# boundaries over gloo; their hybrid steps equal the single-rank oracle's bit for bit.

SLAB_CFG = dict(ncx=10, ncy=16, ppc=20, lb_ratio=2, real_bytes=4, seed=44, kn=0.08, ma=0.3)
SLAB_BOUNDS = [0, 8, 16]
SLAB_STEPS = 4


def slab_lists(scfg, cfg, d, nodes, cells):
    """The slab's own node and cell indices of the channel's coupling lists."""
    ncx, ncy, r = cfg["ncx"], cfg["ncy"], cfg["lb_ratio"]
    nly, y0, yh = scfg["ncy"], scfg["y0"], d["yh"]
    nx, ny_s = ncx * r, d["ny"]
    y, x = nodes // nx, nodes % nx
    keep = (y >= y0 * r) & (y < (y0 + nly) * r)
    ln = ((y - y0 * r + yh) * nx + x)[keep]
    cy, cx = cells // ncx, cells % ncx
    keepc = (cy >= y0) & (cy < y0 + nly)
    lc = ((cy - y0) * ncx + cx)[keepc]
    return ln.astype(np.int32), lc.astype(np.int32)


def _sendrecv(rank, world, send_to, send_arr, recv_from, tag):
    """Point-to-point exchange of one float64 array of any length (its length first)."""
    out = torch.from_numpy(np.ascontiguousarray(send_arr, np.float64))
    n_out = torch.tensor([out.numel()], dtype=torch.int64)
    n_in = torch.zeros(1, dtype=torch.int64)

    def send():
        dist.send(n_out, send_to, tag=tag)
        if out.numel():
            dist.send(out, send_to, tag=tag + 1)

    def recv():
        dist.recv(n_in, recv_from, tag=tag)
        buf = torch.zeros(int(n_in.item()), dtype=torch.float64)
        if buf.numel():
            dist.recv(buf, recv_from, tag=tag + 1)
        return buf.numpy()

    if rank % 2 == 0:
        send()
        got = recv()
    else:
        got = recv()
        send()
    return got


def _slab_rank_main(rank, world, port, out_dir):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    from oracle import oracle as O
    from paper_1512_08042_gb300 import workloads as W

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    cfg = W.config(**SLAB_CFG)
    y0, y1 = SLAB_BOUNDS[rank], SLAB_BOUNDS[rank + 1]
    scfg = dict(cfg, ncy=y1 - y0, ncy_global=cfg["ncy"], y0=y0)
    o = O.Oracle(scfg)
    d = O.derive(scfg)
    nodes, cells = W.coupling_sites(cfg)  # the 4-row strip straddles the cut at row 8
    ln, lc = slab_lists(scfg, cfg, d, nodes, cells)
    below, above = (rank - 1) % world, (rank + 1) % world
    yh, ny = d["yh"], d["ny"]
    for step in range(SLAB_STEPS):
        out = o.dsmc_move_out()
        pack = lambda rec, key: np.concatenate([rec, key[:, None].astype(np.float64)], 1).reshape(-1)
        g0 = _sendrecv(rank, world, above, pack(*out[1]), below, 10)  # into the slab above
        g1 = _sendrecv(rank, world, below, pack(*out[0]), above, 20)  # into the slab below
        unpack = lambda a: (a.reshape(-1, 9)[:, :8].copy(), a.reshape(-1, 9)[:, 8].astype(np.uint32))
        o.dsmc_accept(unpack(g0), unpack(g1))
        o.dsmc_phase(1)
        o.dsmc_phase(2)
        if len(ln):
            o.map_dsmc_to_lbm(ln)
        # ghost rows: the yh rows above the lower boundary go to the slab below's top ghost
        # rows, the yh rows below the upper boundary to the slab above's bottom ghost rows
        f = o.f().astype(np.float64)
        top = f[:, ny - 2 * yh:ny - yh].reshape(-1)
        bot = f[:, yh:2 * yh].reshape(-1)
        gb = _sendrecv(rank, world, above, top, below, 30)  # the slab below's top rows
        ga = _sendrecv(rank, world, below, bot, above, 40)  # the slab above's bottom rows
        f[:, 0:yh] = gb.reshape(f.shape[0], yh, -1)
        f[:, ny - yh:ny] = ga.reshape(f.shape[0], yh, -1)
        o.set_f(f.astype(np.float32))
        o.lbm_step(1)
        if len(lc):
            o.map_lbm_to_dsmc(lc)
    p = o.particles()
    np.savez(os.path.join(out_dir, "slab%d.npz" % rank), cs=o.get(O.A_CELL_START),
             crmax=o.get(O.A_CRMAX), rem=o.get(O.A_REM), nbar=o.get(O.A_NBAR_SUM), acc=o.acc(),
             f=o.f()[:, yh:ny - yh], counters=np.array([o.counters()[k] for k in O.COUNTER_NAMES]),
             scalars=np.array([o.scalars()[k] for k in ("step", "nsamples", "status")]), **p)
    dist.barrier()
    dist.destroy_process_group()


def test_slab_oracle_ranks_equal_the_single_rank_oracle(tmp_path):
    import numpy as np
    from oracle import oracle as O
    from paper_1512_08042_gb300 import workloads as W

    port = _free_port()
    mp.spawn(_slab_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    cfg = W.config(**SLAB_CFG)
    o = O.Oracle(cfg)
    nodes, cells = W.coupling_sites(cfg)
    for _ in range(SLAB_STEPS):
        o.dsmc_step(1)
        o.map_dsmc_to_lbm(nodes)
        o.lbm_step(1)
        o.map_lbm_to_dsmc(cells)
    ncx, r = cfg["ncx"], cfg["lb_ratio"]
    wcs = o.get(O.A_CELL_START).astype(np.int64)
    wp = o.particles()
    counters = 0
    for rank in range(2):
        s = np.load(tmp_path / ("slab%d.npz" % rank))
        y0, y1 = SLAB_BOUNDS[rank], SLAB_BOUNDS[rank + 1]
        c0, c1 = y0 * ncx, y1 * ncx
        assert np.array_equal(np.diff(s["cs"].astype(np.int64)), np.diff(wcs)[c0:c1])
        for k in ("x", "y", "vx", "vy", "vz"):
            assert np.array_equal(s[k], wp[k][wcs[c0]:wcs[c1]]), k
        assert np.array_equal(s["crmax"], o.get(O.A_CRMAX)[c0:c1])
        assert np.array_equal(s["rem"], o.get(O.A_REM)[c0:c1])
        assert np.array_equal(s["nbar"], o.get(O.A_NBAR_SUM)[c0:c1])
        assert np.array_equal(s["acc"], o.acc()[c0:c1])
        assert np.array_equal(s["f"], o.f()[:, y0 * r:y1 * r])
        counters = counters + s["counters"]
        sc = o.scalars()
        assert list(s["scalars"][:2]) == [sc["step"], sc["nsamples"]]
    want = np.array([o.counters()[k] for k in O.COUNTER_NAMES])
    assert np.array_equal(counters, want)
    assert want[O.COUNTER_NAMES.index("created")] > 0 and want[O.COUNTER_NAMES.index("collisions")] > 0


# ---------------------------------------------------------------------------------------
# The pairing of the slab exchange between ranks (binding.exchange_dist, which bench.py's
# multi-GPU path uses): with stand-in buffers on CPU ranks over gloo, every rank's receive
# buffers hold exactly its neighbours' send buffers (from below: the lower rank's "towards
# higher rows" buffer; from above: the higher rank's "towards lower rows" one), in a ring of
# two and of three ranks, for the particle buffers and the packed LB rows alike.

class _StandInSlab:
    def __init__(self, rank, nbytes):
        g = torch.Generator().manual_seed(100 + rank)
        self.buf = {("send", d): torch.randint(0, 255, (nbytes,), dtype=torch.uint8, generator=g)
                    for d in (0, 1)}
        self.buf.update({("recv", d): torch.zeros(nbytes, dtype=torch.uint8) for d in (0, 1)})

    def xfer(self, which, d):
        return self.buf[(which, d)]


def _exchange_rank_main(rank, world, port, out_dir):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    from paper_1512_08042_gb300 import binding as B

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    h = _StandInSlab(rank, 1000 + rank * 0)
    B.exchange_dist(h, dist, rank, world)
    halo = [torch.full((37,), float(10 * rank + k)) for k in range(2)] + [torch.zeros(37), torch.zeros(37)]
    B.exchange_dist(h, dist, rank, world, halo)
    torch.save({"send0": h.xfer("send", 0), "send1": h.xfer("send", 1), "recv0": h.xfer("recv", 0),
                "recv1": h.xfer("recv", 1), "halo": halo}, os.path.join(out_dir, "x%d.pt" % rank))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_slab_exchange_pairs_neighbours(tmp_path, world):
    port = _free_port()
    mp.spawn(_exchange_rank_main, args=(world, port, str(tmp_path)), nprocs=world, join=True)
    got = [torch.load(tmp_path / ("x%d.pt" % r)) for r in range(world)]
    for r in range(world):
        below, above = (r - 1) % world, (r + 1) % world
        assert torch.equal(got[r]["recv0"], got[below]["send1"])
        assert torch.equal(got[r]["recv1"], got[above]["send0"])
        # packed LB rows: side 0 holds the slab below's side-1 pack, side 1 the slab above's
        assert torch.equal(got[r]["halo"][2], got[below]["halo"][1])
        assert torch.equal(got[r]["halo"][3], got[above]["halo"][0])


def _ensemble_rank_main(rank, world, port, out_dir):
    # a multi-GPU ensemble's host logic on CPU ranks: every rank runs the same channels with
    # its own seeds (the oracle stands in for the batch) and the ranks sum the replicas' moment
    # sums with one all-reduce
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import numpy as np
    from oracle import oracle as O
    from paper_1512_08042_gb300 import workloads as W

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    cfgs = [dict(c, ncx=min(c["ncx"], 40), ppc=min(c["ppc"], 30)) for c in W.ensemble_configs(3, rank=rank)]
    geom = torch.tensor([[c["ncx"], c["ppc"], c["kn"]] for c in cfgs], dtype=torch.float64)
    seeds = torch.tensor([c["seed"] for c in cfgs], dtype=torch.int64)
    geoms = [torch.zeros_like(geom) for _ in range(world)]
    seedl = [torch.zeros_like(seeds) for _ in range(world)]
    dist.all_gather(geoms, geom)
    dist.all_gather(seedl, seeds)
    accs = []
    for c in cfgs:
        o = O.Oracle(c)
        nodes, cells = W.coupling_sites(c)
        for _ in range(3):
            o.dsmc_step(1)
            o.map_dsmc_to_lbm(nodes)
            o.lbm_step(1)
            o.map_lbm_to_dsmc(cells)
        accs.append(o.get(O.A_ACC).astype(np.float64).reshape(-1))
    flat = torch.from_numpy(np.concatenate(accs))
    mine = flat.clone()
    dist.all_reduce(flat)
    np.save(os.path.join(out_dir, "ens%d_mine.npy" % rank), mine.numpy())
    np.save(os.path.join(out_dir, "ens%d_sum.npy" % rank), flat.numpy())
    same_geom = all(torch.equal(g, geoms[0]) for g in geoms)
    distinct = len(set(int(s) for sl in seedl for s in sl)) == world * len(cfgs)
    with open(os.path.join(out_dir, "ens%d.txt" % rank), "w") as fh:
        fh.write("%d %d\n" % (int(same_geom), int(distinct)))
    dist.destroy_process_group()


def test_ensemble_ranks_share_channels_and_sum_their_moment_sums(tmp_path):
    port = _free_port()
    mp.spawn(_ensemble_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    for r in range(2):
        same_geom, distinct = open(tmp_path / ("ens%d.txt" % r)).read().split()
        assert same_geom == "1" and distinct == "1"
    m0, m1 = np.load(tmp_path / "ens0_mine.npy"), np.load(tmp_path / "ens1_mine.npy")
    assert not np.array_equal(m0, m1)  # different seeds, different samples
    for r in range(2):
        assert np.array_equal(np.load(tmp_path / ("ens%d_sum.npy" % r)), m0 + m1)
