"""The batched ensemble against independent contexts: a replica advanced in a batch must give
bit for bit what the same channel gives when advanced alone (same kernels, same draws)."""
import numpy as np
import pytest

from conftest import LB_TOL_FP32, LB_TOL_FP64, lb_err

torch = pytest.importorskip("torch")

from paper_1512_08042_gb300 import binding as B
from paper_1512_08042_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _cfgs():
    return [W.config(ncx=40, ncy=1, ppc=30, kn=0.05, seed=21),
            W.config(ncx=96, ncy=1, ppc=77, kn=0.3, seed=22),
            W.config(ncx=13, ncy=8, ppc=23, kn=0.1, lb_ratio=2, capacity_factor=1.5, seed=23),
            W.config(ncx=33, ncy=1, ppc=55, kn=0.012, seed=24)]


def _sites(cfgs):
    nodes, cells = zip(*[W.coupling_sites(c) for c in cfgs])
    return list(nodes), list(cells)


def _assert_same(h, g):
    h.sync()
    g.sync()
    assert h.current() == g.current()
    for k, v in h.particles().items():
        assert torch.equal(v, g.particles()[k]), k
    for name in ("cell_start", "crmax", "rem", "nbar_sum", "acc", "f"):
        assert torch.equal(getattr(h, name)(), getattr(g, name)()), name
    assert torch.equal(h.ctrl()[:4], g.ctrl()[:4])
    assert h.counters() == g.counters()


@pytest.mark.parametrize("use_graph,collide", [(False, 256), (True, 256), (True, 128)])
def test_batch_replicas_equal_single_contexts(use_graph, collide):
    # (collide: the batch's collide in blocks of 32 or 16 cells; the single contexts keep theirs)
    cfgs = _cfgs()
    nodes, cells = _sites(cfgs)
    b = B.Batch(cfgs)
    b.set_block("collide", collide)
    assert b.blocks()["collide"] == collide
    singles = [B.Hybrid(c) for c in cfgs]
    b.hybrid_step(nodes, cells, nsteps=4, use_graph=use_graph)
    for h, n, c in zip(singles, nodes, cells):
        h.hybrid_step(torch.from_numpy(n).cuda(), torch.from_numpy(c).cuda(), nsteps=4, use_graph=True)
    b.sync()
    for g, h in zip(b.replicas, singles):
        _assert_same(h, g)
    assert all(g.sync_status()[1] == 0 for g in b.replicas)
    b.close()


def test_batch_tuner_picks_valid_shapes_and_keeps_results():
    cfgs = _cfgs()[:3]
    nodes, cells = _sites(cfgs)
    b = B.Batch(cfgs)
    mb, lb = b.tune(nodes, cells)
    assert mb in (64, 128, 256) and lb in (32, 64, 128)
    shapes = b.blocks()
    assert shapes["move"] == mb and shapes["lbm"] == lb and shapes["dsmc2lb"] in (64, 128, 256)
    assert shapes["collide"] in (256, 128) and shapes["lb2dsmc"] == 256
    with pytest.raises(B.HybError):
        b.set_block("lb2dsmc", 128)  # one shape, fixed by the kernel's design
    with pytest.raises(B.HybError):
        b.set_block("collide", 64)
    b.hybrid_step(nodes, cells, nsteps=2)
    steps = 77 + 2  # 7 steps per shape tried: 3 move, 2 collide, 3 LB, 3 DSMC2LB
    for g, cfg, n, c in zip(b.replicas, cfgs, nodes, cells):
        h = B.Hybrid(cfg)
        h.hybrid_step(torch.from_numpy(n).cuda(), torch.from_numpy(c).cuda(), nsteps=steps, use_graph=True)
        _assert_same(h, g)
    b.close()


def test_batch_refuses_a_replica_out_of_lockstep():
    cfgs = _cfgs()[:2]
    nodes, cells = _sites(cfgs)
    b = B.Batch(cfgs)
    b.hybrid_step(nodes, cells, nsteps=1)
    b.replicas[1].dsmc_step(1)
    with pytest.raises(B.HybError) as ei:
        b.hybrid_step(nodes, cells, nsteps=1)
    assert ei.value.status == B.HYB_ESTATE
    b.close()


def test_full_ensemble_of_64_channels_matches_the_oracle_per_replica():
    # the 64-channel ensemble (heights 32-256 cells, 20-100 per cell, Kn 0.01-0.5, FP32) in
    # one batch: without coupling every replica's DSMC state equals its own oracle bit for
    # bit and its populations match to 1e-5 of w_a rho; with the coupling strip every replica equals
    # the same channel advanced alone
    from oracle import oracle as O
    cfgs = W.ensemble_configs(64)
    empty = [np.zeros(0, np.int32)] * len(cfgs)
    b = B.Batch(cfgs)
    steps = 2
    b.hybrid_step(empty, empty, nsteps=steps)
    b.sync()
    for g, cfg in zip(b.replicas, cfgs):
        o = O.Oracle(cfg)
        for _ in range(steps):
            o.dsmc_step(1)
            o.lbm_step(1)
        assert np.array_equal(g.cell_start().cpu().numpy().astype(np.uint32), o.get(O.A_CELL_START))
        gp, op = g.particles(), o.particles()
        for k in ("x", "y", "vx", "vy", "vz"):
            a, want = gp[k].cpu().numpy(), op[k]
            assert (a == want).mean() >= 0.9999 and np.allclose(a, want, rtol=1e-5, atol=1e-5), k
        assert np.array_equal(g.crmax().cpu().numpy(), o.get(O.A_CRMAX))
        assert np.array_equal(g.rem().cpu().numpy(), o.get(O.A_REM))
        e, w, r = O.lattice(39)
        err = lb_err(g.f().cpu().numpy(), o.f(), w)
        assert err < LB_TOL_FP32, err
    b.close()
    nodes, cells = _sites(cfgs)
    b = B.Batch(cfgs)
    b.hybrid_step(nodes, cells, nsteps=3)
    for k in (0, 17, 63):
        h = B.Hybrid(cfgs[k])
        h.hybrid_step(torch.from_numpy(nodes[k]).cuda(), torch.from_numpy(cells[k]).cuda(),
                      nsteps=3, use_graph=True)
        _assert_same(h, b.replicas[k])
    b.close()
