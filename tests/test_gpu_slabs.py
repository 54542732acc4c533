"""The streamwise slab decomposition of the channel (the multi-GPU path), as logical slabs on
one GPU: every slab holds a range of the channel's rows, particles that leave a slab are
exchanged through its send and receive buffers, and the LB ghost rows are filled with the
neighbours' outgoing populations before every LB step. Hybrid steps of the slabs must give
the whole channel's results bit for bit: particles, per-cell collision state, moment sums,
populations, counters. The random streams are keyed by the channel's cell ids and the
order keys by the channel's cells (displacements in channel coordinates), which makes this
exact."""
import numpy as np
import pytest

from paper_1512_08042_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # collected on CPU-only machines, never run there
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1512_08042_gb300 import binding as B  # noqa: E402
from paper_1512_08042_gb300 import build as BUILD  # noqa: E402

BUILD.build()


def whole_cells(slab, cfg):
    """The whole channel's cell index of each of the slab's cells, in the slab's order."""
    ncx, ncy = cfg["ncx"], cfg["ncy"]
    nly, y0 = slab.cfg["ncy"], slab.cfg["y0"]
    nz = max(cfg.get("ncz", 0), 1)
    c = np.arange(ncx * nly * nz)
    iz, r = c // (ncx * nly), c % (ncx * nly)
    return (iz * ncy + y0 + r // ncx) * ncx + r % ncx


def local_lists(slab, cfg, nodes, cells):
    """The slab's own node and cell indices of the whole channel's coupling lists."""
    ncx, ncy, r = cfg["ncx"], cfg["ncy"], cfg["lb_ratio"]
    nly, y0, yh = slab.cfg["ncy"], slab.cfg["y0"], int(slab.d["yh"])
    nx, ny_w, ny_s = ncx * r, ncy * r, int(slab.d["ny"])
    z, rem = nodes // (nx * ny_w), nodes % (nx * ny_w)
    y, x = rem // nx, rem % nx
    keep = (y >= y0 * r) & (y < (y0 + nly) * r)
    ln = ((z * ny_s + (y - y0 * r + yh)) * nx + x)[keep]
    cz, crem = cells // (ncx * ncy), cells % (ncx * ncy)
    cy, cx = crem // ncx, crem % ncx
    keepc = (cy >= y0) & (cy < y0 + nly)
    lc = ((cz * nly + (cy - y0)) * ncx + cx)[keepc]
    return (torch.from_numpy(ln.astype(np.int32)).cuda(), torch.from_numpy(lc.astype(np.int32)).cuda())


def assert_slabs_equal_whole(grp, whole, cfg):
    grp.sync()
    whole.sync()
    wa = whole.particle_arrays()
    wcnt = whole.counts()
    r = cfg["lb_ratio"]
    nz_cells = max(cfg.get("ncz", 0), 1)
    tot = {}
    for s in grp.slabs:
        wc = torch.from_numpy(whole_cells(s, cfg)).cuda()
        assert torch.equal(s.counts(), wcnt[wc])
        sa = s.particle_arrays()
        mask = torch.arange(s.L.bin, device="cuda")[None, :] < s.counts()[:, None]
        for k in sa:
            assert torch.equal(sa[k][mask], wa[k][wc][mask]), k
        for name in ("crmax", "rem", "nbar_sum"):
            assert torch.equal(getattr(s, name)(), getattr(whole, name)()[wc]), name
        assert torch.equal(s.acc(), whole.acc()[wc])
        # populations of the slab's own rows (per z layer)
        y0, nly = s.cfg["y0"], s.cfg["ncy"]
        fs = s.f_rows()
        fw = whole.f()
        if s.three_d():
            assert torch.equal(fs, fw[:, :, y0 * r:(y0 + nly) * r, :])
        else:
            assert torch.equal(fs, fw[:, y0 * r:(y0 + nly) * r, :])
        assert torch.equal(s.ctrl()[2:4], whole.ctrl()[2:4])
        for k, v in s.counters().items():
            tot[k] = tot.get(k, 0) + v
        assert s.sync_status()[0] == B.HYB_OK
    assert tot == whole.counters()
    assert nz_cells >= 1


@pytest.mark.parametrize("real_bytes,ncz,cuts,knprof", [
    (4, 0, [8], False),        # two slabs of 8 rows
    (8, 0, [5, 11], False),    # three uneven slabs: distinct neighbours on both sides
    (4, 3, [7], False),        # 3D
    (4, 0, [6], True),         # Kn along the channel
])
def test_slabs_equal_the_whole_channel(real_bytes, ncz, cuts, knprof):
    extra = dict(kn_profile=1, kn=0.02, kn_end=0.3) if knprof else {}
    cfg = W.config(ncx=12, ncy=16, ppc=30, lb_ratio=2, real_bytes=real_bytes, ncz=ncz, ma=0.3,
                   seed=31, **extra)
    # the coupling strip of 4 rows in the middle straddles the cut at row 8
    nodes, cells = W.coupling_sites(cfg)
    whole = B.Hybrid(cfg)
    grp = B.SlabGroup(cfg, cuts)
    lists = [local_lists(s, cfg, nodes, cells) for s in grp.slabs]
    dn, dc = torch.from_numpy(nodes).cuda(), torch.from_numpy(cells).cuda()
    for _ in range(6):
        whole.hybrid_step(dn, dc, nsteps=1, use_graph=False)
        grp.hybrid_step([l[0] for l in lists], [l[1] for l in lists])
    assert_slabs_equal_whole(grp, whole, cfg)
    c = whole.counters()
    assert c["collisions"] > 0 and c["created"] > 0 and c["wall_hits"] > 0


def test_slab_exchange_moves_particles_across_the_periodic_end():
    # fast streamwise flow: many particles cross both slab boundaries every step, including
    # the channel's periodic end (the top slab's particles re-enter the bottom slab)
    cfg = W.config(ncx=8, ncy=8, ppc=40, lb_ratio=1, ma=0.0, seed=5)
    whole = B.Hybrid(cfg)
    grp = B.SlabGroup(cfg, [4])
    for h in [whole] + grp.slabs:
        p = {k: v.cpu().numpy() for k, v in h.particles().items()}
        p["vy"] = p["vy"] + 2.0  # a drift of about one cell per step
        h.load_particles(p["x"], p["y"], p["vx"], p["vy"], p["vz"], h.cell_start().cpu().numpy())
    for _ in range(5):
        whole.dsmc_step(1)
        grp.dsmc_step()
    assert_slabs_equal_whole(grp, whole, cfg)


def test_slab_calls_out_of_order_are_refused():
    cfg = W.config(ncx=8, ncy=8, ppc=10, seed=5)
    grp = B.SlabGroup(cfg, [4])
    s = grp.slabs[0]
    with pytest.raises(B.HybError):
        s.dsmc_step(1)  # a slab steps with the split calls
    with pytest.raises(B.HybError):
        s.dsmc_collide()  # no move yet
    s.dsmc_move()
    with pytest.raises(B.HybError):
        s.dsmc_move()  # the previous move has no collide yet
    grp.exchange_particles()
    s.dsmc_merge()
    s.dsmc_collide()
    whole = B.Hybrid(cfg)
    with pytest.raises(B.HybError):
        whole.halo_size()  # no ghost rows
