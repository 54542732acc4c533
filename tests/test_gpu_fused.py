"""The fused multi-step DSMC pass (the collide of step s and the move of step s + 1 in one
pass over the particles, and LB2DSMC moving the particles it creates on at once) gives the
same results as the same steps taken one at a time, bit for bit, and as the oracle; in 2D
and 3D, FP32 and FP64, with walls, body force, coupling and the capacity fallback of
LB2DSMC. The contexts here are small, so the fused pass is forced (HYB_FUSE_ALWAYS); the
automatic choice takes it only where its grid fills the GPU."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1512_08042_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # collected on CPU-only machines, never run there
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1512_08042_gb300 import binding as B  # noqa: E402
from paper_1512_08042_gb300 import build as BUILD  # noqa: E402

BUILD.build()


def fused(cfg):
    h = B.Hybrid(cfg)
    h.set_fuse("always")
    return h


def cfg_small(**kw):
    base = dict(ncx=13, ncy=7, ppc=23, real_bytes=4, seed=11, kn=0.1, ma=0.3, capacity_factor=1.5)
    base.update(kw)
    return W.config(**base)


def assert_same_state(a, b, counters=True):
    a.sync()
    b.sync()
    assert a.current() == b.current()
    assert a.n_tot() == b.n_tot()
    pa, pb = a.particles(), b.particles()
    for k in pa:
        assert torch.equal(pa[k], pb[k]), k
    for name in ("cell_start", "crmax", "rem", "nbar_sum", "acc", "f"):
        assert torch.equal(getattr(a, name)(), getattr(b, name)()), name
    assert torch.equal(a.ctrl()[:4], b.ctrl()[:4])
    if counters:
        assert a.counters() == b.counters()
    # between calls the other half holds no particles
    assert int(a.counts(a.current()[0] ^ 1).sum()) == 0
    assert int(b.counts(b.current()[0] ^ 1).sum()) == 0


@pytest.mark.parametrize("real_bytes,ncz,steps", [(4, 0, 5), (8, 0, 3), (4, 3, 4)])
def test_fused_dsmc_steps_equal_single_steps_and_the_oracle(real_bytes, ncz, steps):
    cfg = cfg_small(real_bytes=real_bytes, ncz=ncz)
    a, b = fused(cfg), B.Hybrid(cfg)
    a.dsmc_step(steps)  # fused: move, steps - 1 fused passes, collide
    for _ in range(steps):
        b.dsmc_step(1)
    assert_same_state(a, b)
    o = O.Oracle(cfg)
    o.dsmc_step(steps)
    assert a.n_tot() == o.scalars()["ntot"]
    assert np.array_equal(a.cell_start().cpu().numpy().astype(np.uint32), o.get(O.A_CELL_START))
    hc, oc = a.counters(), o.counters()
    for k in ("candidates", "collisions", "wall_hits"):
        assert hc[k] == oc[k], k
    pa, op = a.particles(), o.particles()
    for k in op:
        g = pa[k].cpu().numpy()
        if real_bytes == 4:
            assert (g == op[k]).mean() >= 0.9999, k
            assert np.allclose(g, op[k], rtol=1e-5, atol=1e-5), k
        else:
            assert np.allclose(g, op[k], rtol=1e-12, atol=1e-12), k


@pytest.mark.parametrize("real_bytes,ncz,graph", [(4, 0, True), (4, 0, False), (8, 0, True),
                                                  (4, 2, True)])
def test_fused_hybrid_steps_equal_single_steps(real_bytes, ncz, graph):
    cfg = cfg_small(real_bytes=real_bytes, ncz=ncz, lb_ratio=2, ncy=10)
    nodes, cells = W.coupling_sites(cfg, strip_cells=2)
    dn, dc = torch.from_numpy(nodes).cuda(), torch.from_numpy(cells).cuda()
    a, b = fused(cfg), B.Hybrid(cfg)
    for _ in range(2):  # the second call replays the graph captured by the first
        a.hybrid_step(dn, dc, nsteps=4, use_graph=graph)
        for _ in range(4):
            b.hybrid_step(dn, dc, nsteps=1, use_graph=True)
        assert_same_state(a, b)
    c = a.counters()
    assert c["created"] > 0 and c["deleted"] > 0 and c["collisions"] > 0
    assert a.sync_status()[0] == B.HYB_OK
    # an odd step count flips the parities: two graph slots
    a.hybrid_step(dn, dc, nsteps=3, use_graph=graph)
    a.hybrid_step(dn, dc, nsteps=3, use_graph=graph)
    for _ in range(6):
        b.hybrid_step(dn, dc, nsteps=1, use_graph=False)
    assert_same_state(a, b)


def test_fused_hybrid_keeps_cells_whose_new_count_exceeds_the_bin():
    # LB2DSMC only (no DSMC2LB), populations at density 4 everywhere: every coupling cell's new
    # count (about 40) exceeds its bin of 32 slots, so each keeps (and the fused run moves on)
    # its own particles and the capacity status is raised, as in the steps taken one at a time
    cfg = cfg_small(ppc=10, capacity_factor=3.0, lb_ratio=1, ncy=8)
    _, cells = W.coupling_sites(cfg, strip_cells=2)
    dc = torch.from_numpy(cells).cuda()
    e, w, r = O.lattice(39)
    a, b = fused(cfg), B.Hybrid(cfg)
    f = torch.from_numpy((w[:, None] * 4.0 * np.ones((1, a.d["nnodes"]))).astype(np.float32))
    for h in (a, b):
        h.f().copy_(f.view(h.f().shape))
    torch.cuda.synchronize()
    a.hybrid_step(None, dc, nsteps=3, use_graph=False)
    for _ in range(3):
        b.hybrid_step(None, dc, nsteps=1, use_graph=False)
    assert_same_state(a, b)
    for h in (a, b):
        rc, bits = h.sync_status()
        assert rc == B.HYB_ECAPACITY and bits & B.ST_CAPACITY
    assert a.counters()["created"] == 0 and a.n_tot() == cfg["ppc"] * a.L.ncells


def test_fused_hybrid_at_the_819k_particle_channel_equals_single_steps():
    cfg = W.WORKLOADS["poiseuille_64x256_ppc50_fp32"]
    nodes, cells = W.coupling_sites(cfg)
    dn, dc = torch.from_numpy(nodes).cuda(), torch.from_numpy(cells).cuda()
    a, b = fused(cfg), B.Hybrid(cfg)
    a.hybrid_step(dn, dc, nsteps=3, use_graph=True)
    for _ in range(3):
        b.hybrid_step(dn, dc, nsteps=1, use_graph=True)
    assert_same_state(a, b)


def test_fuse_modes_give_the_same_results_and_auto_skips_a_grid_below_the_gpu():
    # HYB_FUSE_AUTO fuses only where the fused grid fills the GPU; a 13 x 10-cell channel (5
    # blocks of 32 cells) takes a move and a collide per step. Every mode gives the same state.
    cfg = cfg_small(lb_ratio=2, ncy=10)
    nodes, cells = W.coupling_sites(cfg, strip_cells=2)
    dn, dc = torch.from_numpy(nodes).cuda(), torch.from_numpy(cells).cuda()
    hs = {}
    for mode in ("auto", "always", "never"):
        h = B.Hybrid(cfg)
        h.set_fuse(mode)
        h.profile("fused")
        h.profile_harvest()
        h.hybrid_step(dn, dc, nsteps=4, use_graph=False)
        h.profile_harvest()
        ms, n = h.profile_read()
        h.profile(-1)
        assert (n > 0) == (mode == "always"), (mode, n)
        h.dsmc_step(3)
        hs[mode] = h
    assert_same_state(hs["always"], hs["never"])
    assert_same_state(hs["auto"], hs["never"])
    with pytest.raises(B.HybError):
        B._check(B.lib().hyb_set_fuse(hs["auto"].ctx, 3))


@pytest.mark.parametrize("real_bytes,ncz", [(4, 0), (8, 0), (4, 2)])
def test_collide_block_shapes_give_the_same_results(real_bytes, ncz):
    # 16-cell blocks (4 warps) and 32-cell blocks (8 warps), fused and plain passes, with
    # coupling: the per-cell work is the same, only its grouping into blocks differs
    cfg = cfg_small(ncx=24, ncy=20, real_bytes=real_bytes, ncz=ncz, lb_ratio=2)
    nodes, cells = W.coupling_sites(cfg, strip_cells=2)
    dn, dc = torch.from_numpy(nodes).cuda(), torch.from_numpy(cells).cuda()
    a, b = fused(cfg), fused(cfg)
    a.set_collide_block(8)
    b.set_collide_block(4)
    assert (a.collide_block(), b.collide_block()) == (8, 4)
    for h in (a, b):
        h.hybrid_step(dn, dc, nsteps=3, use_graph=True)
        h.dsmc_step(2)
        h.hybrid_step(dn, dc, nsteps=1, use_graph=False)
    assert_same_state(a, b)
    with pytest.raises(B.HybError):
        a.set_collide_block(2)


def test_collide_tuner_keeps_results():
    cfg = cfg_small(ncx=24, ncy=20, lb_ratio=2)
    nodes, cells = W.coupling_sites(cfg, strip_cells=2)
    dn, dc = torch.from_numpy(nodes).cuda(), torch.from_numpy(cells).cuda()
    a, b = B.Hybrid(cfg), B.Hybrid(cfg)
    w, fuse = a.tune_collide(dn, dc)
    assert w in (4, 8) and a.collide_block() == w and fuse in ("always", "never")
    a.hybrid_step(dn, dc, nsteps=2, use_graph=True)
    b.hybrid_step(dn, dc, nsteps=192 + 2, use_graph=True)  # the tuner's 192 steps, then 2
    assert_same_state(a, b)


@pytest.mark.parametrize("real_bytes,warps", [(4, 8), (4, 4), (8, 8)])
def test_far_displaced_particles_are_ordered_as_the_oracle_orders_them(real_bytes, warps):
    # a streamwise drift of about 1.2 cells per step: many particles land two or more cells
    # from their old cell (order keys with bit 31), more than the per-cell list of 8 holds in
    # most cells, so the collide ranks them by counting over the records; the fused pass and
    # the plain collide must order them as the oracle does (bit-exact counts, pairs, particles)
    cfg = cfg_small(ncx=12, ncy=10, ppc=40, real_bytes=real_bytes, kn=0.05, ma=0.0, capacity_factor=2.5)
    a = fused(cfg)
    a.set_collide_block(warps)
    p = {k: v.cpu().numpy() for k, v in a.particles().items()}
    cs = a.cell_start().cpu().numpy()
    drift = 1.2 / a.d["dt"]
    vy = p["vy"] + drift
    a.load_particles(p["x"], p["y"], p["vx"], vy, p["vz"], cs)
    o = O.Oracle(cfg)
    o.set_particles(p["x"], p["y"], p["vx"], vy.astype(p["vy"].dtype), p["vz"], cs.astype(np.uint32))
    steps = 3
    a.dsmc_step(steps)
    o.dsmc_step(steps)
    hc, oc = a.counters(), o.counters()
    for k in ("candidates", "collisions", "wall_hits"):
        assert hc[k] == oc[k], k
    assert np.array_equal(a.cell_start().cpu().numpy().astype(np.uint32), o.get(O.A_CELL_START))
    pa, op = a.particles(), o.particles()
    for k in op:
        g = pa[k].cpu().numpy()
        if real_bytes == 4:
            assert (g == op[k]).mean() >= 0.9999, k
        else:
            assert np.allclose(g, op[k], rtol=1e-12, atol=1e-12), k
