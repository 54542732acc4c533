"""Parity of the full 3D path (ncz >= 2: particle z positions periodic over ncz cells, a
lattice of ncz * lb_ratio layers periodic in z, wall densities per streamwise row (y, z),
mappings over the r^3 nodes of a cell) with the CPU oracle, through the C ABI. The paper's
DSMC and LBM solvers are 3D with periodic y and z (Sec. 3.1); the slab (ncz < 2) is one cell
and one LB layer thick. Same tolerances as the slab tests: integers bit-exact, float state
within 1e-5 (FP32) or 1e-12 (FP64)."""
import numpy as np
import pytest

from conftest import LB_TOL_FP32, LB_TOL_FP64, lb_err

from oracle import oracle as O
from paper_1512_08042_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # collected on CPU-only machines, never run there
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1512_08042_gb300 import binding as B  # noqa: E402
from paper_1512_08042_gb300 import build as BUILD  # noqa: E402

BUILD.build()

RTOL = 1e-5
KEYS = ("x", "y", "z", "vx", "vy", "vz")


def cfg3(**kw):
    # 13 x 7 x 3 cells (a ragged last block of 32 cells), 23 per cell
    base = dict(ncx=13, ncy=7, ncz=3, ppc=23, real_bytes=4, seed=17, kn=0.1, capacity_factor=1.5)
    base.update(kw)
    return W.config(**base)


def gpu_particles(h):
    h.sync()
    return {k: v.cpu().numpy() for k, v in h.particles().items()}


def assert_particles_match(gp, op, real_bytes, exact_frac=0.9999):
    assert set(gp) == set(KEYS) and set(op) == set(KEYS)
    for k in KEYS:
        a, b = gp[k], op[k]
        assert a.shape == b.shape, k
        if real_bytes == 4:
            assert ((a == b).mean() if a.size else 1.0) >= exact_frac, k
            assert np.allclose(a, b, rtol=RTOL, atol=RTOL), (k, np.abs(a - b).max())
        else:
            assert np.allclose(a, b, rtol=1e-12, atol=1e-12), (k, np.abs(a - b).max())


def compare_dsmc(h, o, real_bytes):
    assert h.n_tot() == o.scalars()["ntot"]
    assert np.array_equal(h.cell_start().cpu().numpy().astype(np.uint32), o.get(O.A_CELL_START))
    assert_particles_match(gpu_particles(h), o.particles(), real_bytes)
    hc, oc = h.counters(), o.counters()
    for k in ("candidates", "collisions", "wall_hits", "created", "deleted"):
        assert hc[k] == oc[k], (k, hc[k], oc[k])
    assert np.array_equal(h.nbar_sum().cpu().numpy().view(np.uint32), o.get(O.A_NBAR_SUM))
    ga, oa = h.acc().cpu().numpy(), o.acc()
    scale = np.abs(oa).max(axis=0, keepdims=True) + 1e-30
    assert np.all(np.abs(ga - oa) <= 1e-5 * scale), np.abs((ga - oa) / scale).max()
    ctrl = h.ctrl().cpu().numpy()
    s = o.scalars()
    assert ctrl[B.CTRL_STEP] == s["step"] and ctrl[B.CTRL_STATUS] == s["status"]


def cell_of(p, ncx, ncy):
    return ((np.floor(p["z"]).astype(np.int64) * ncy + np.floor(p["y"]).astype(np.int64)) * ncx
            + np.floor(p["x"]).astype(np.int64))


@pytest.mark.parametrize("real_bytes", [4, 8])
def test_init_3d_matches_oracle(real_bytes):
    cfg = cfg3(real_bytes=real_bytes)
    h, o = B.Hybrid(cfg), O.Oracle(cfg)
    assert h.d["ncells"] == 13 * 7 * 3 and h.n_tot() == o.scalars()["ntot"]
    gp, op = gpu_particles(h), o.particles()
    for k in ("x", "y", "z"):
        assert np.array_equal(gp[k], op[k]), k
    assert_particles_match(gp, op, real_bytes)
    # every particle sits in the cell whose bin holds it
    cs = h.cell_start().cpu().numpy()
    own = np.repeat(np.arange(h.d["ncells"]), np.diff(cs))
    assert np.array_equal(cell_of(gp, 13, 7), own)
    f = h.f().cpu().numpy()
    assert f.shape == (39, h.d["nz"], h.d["ny"], h.d["nx"])
    assert np.array_equal(f, o.f())


@pytest.mark.parametrize("real_bytes,steps", [(4, 1), (4, 4), (8, 3)])
def test_dsmc_3d_steps_match_oracle(real_bytes, steps):
    cfg = cfg3(real_bytes=real_bytes, ma=0.3)
    h, o = B.Hybrid(cfg), O.Oracle(cfg)
    for _ in range(steps):
        h.dsmc_step(1)
        o.dsmc_step(1)
    compare_dsmc(h, o, real_bytes)
    gp = gpu_particles(h)
    assert gp["z"].min() >= 0 and gp["z"].max() < 3


def test_dsmc_3d_crowded_cells_take_every_sort_tier():
    # 8 ppc on average with cells of 60, 100 and 200 particles: the register, warp and rank
    # sort tiers of the collision kernel on the same 3D state
    cfg = cfg3(ppc=8, capacity_factor=30.0, ma=0.2)
    h, o = B.Hybrid(cfg), O.Oracle(cfg)
    rng = np.random.default_rng(5)
    nc = h.d["ncells"]
    counts = rng.integers(0, 16, nc)
    counts[[4, 50, 200]] = [60, 100, 200]
    cs = np.zeros(nc + 1, np.int64)
    cs[1:] = np.cumsum(counts)
    cell = np.repeat(np.arange(nc), counts)
    ix, iy, iz = cell % 13, (cell // 13) % 7, cell // 91
    n = cs[-1]
    f32 = np.float32
    # positions below the cell's upper face after rounding to float
    x = np.minimum(ix + rng.random(n), ix + 0.999).astype(f32)
    y = np.minimum(iy + rng.random(n), iy + 0.999).astype(f32)
    z = np.minimum(iz + rng.random(n), iz + 0.999).astype(f32)
    v = rng.normal(size=(3, n)).astype(f32)
    cs = cs.astype(np.uint32)
    h.load_particles(x, y, v[0], v[1], v[2], cs, z=z)
    o.set_particles(x, y, v[0], v[1], v[2], cs, z=z)
    for _ in range(2):
        h.dsmc_step(1)
        o.dsmc_step(1)
    compare_dsmc(h, o, 4)


@pytest.mark.parametrize("lattice,real_bytes,bgk", [(39, 4, 0), (39, 8, 0), (19, 4, 0), (19, 8, 1)])
def test_lbm_3d_steps_match_oracle(lattice, real_bytes, bgk):
    cfg = cfg3(lattice=lattice, real_bytes=real_bytes, lb_ratio=2, ncz=2, ma=0.5, kn=0.3,
               lb_collision=bgk)
    h, o = B.Hybrid(cfg), O.Oracle(cfg)
    e, w, r = O.lattice(lattice)
    f0 = W.gen_populations(w, h.d["nnodes"], seed=23)
    f0 = f0.astype(np.float32 if real_bytes == 4 else np.float64)
    h.f().copy_(torch.from_numpy(f0.reshape(h.f().shape)))
    torch.cuda.synchronize()
    o.set_f(f0)
    tol = LB_TOL_FP32 if real_bytes == 4 else LB_TOL_FP64
    for step in range(3):
        h.lbm_step(1)
        o.lbm_step(1)
        h.sync()
        gf, of = h.f().cpu().numpy(), o.f()
        assert gf.shape == of.shape == (lattice, 4, h.d["ny"], h.d["nx"])
        err = lb_err(gf, of, w)
        assert err < tol, (step, err)
    assert abs(h.f().double().sum().item() / f0.astype(np.float64).sum() - 1) < 1e-6


def test_lbm_3d_with_kn_profile_matches_oracle():
    cfg = cfg3(lb_ratio=2, ncz=2, kn=0.02, kn_profile=1, kn_end=0.4, ma=0.5)
    h, o = B.Hybrid(cfg), O.Oracle(cfg)
    e, w, r = O.lattice(39)
    f0 = W.gen_populations(w, h.d["nnodes"], seed=24).astype(np.float32)
    h.f().copy_(torch.from_numpy(f0.reshape(h.f().shape)))
    torch.cuda.synchronize()
    o.set_f(f0)
    for _ in range(2):
        h.lbm_step(1)
        o.lbm_step(1)
    h.sync()
    gf, of = h.f().cpu().numpy(), o.f()
    err = lb_err(gf, of, w)
    assert err < LB_TOL_FP32, err


@pytest.mark.parametrize("lattice,lb_ratio", [(39, 2), (19, 1)])
def test_dsmc2lb_3d_matches_oracle(lattice, lb_ratio):
    cfg = cfg3(lattice=lattice, lb_ratio=lb_ratio)
    h, o = B.Hybrid(cfg), O.Oracle(cfg)
    src = O.Oracle(cfg3(lattice=lattice, lb_ratio=lb_ratio, ma=0.4))
    src.dsmc_step(5)
    acc, S = src.acc().copy(), src.scalars()["nsamples"]
    h.acc().copy_(torch.from_numpy(acc))
    h.set_counters(nsamples=S)
    o.set(O.A_ACC, acc.reshape(-1))
    o.set_scalars(o.scalars()["step"], S)
    nx, ny, nn = h.d["nx"], h.d["ny"], h.d["nnodes"]
    # nodes in the first, a middle and the last layer, at both walls
    nodes = np.array([0, nx - 1, nx * ny + 5, nx * ny * (h.d["nz"] // 2) + 3 * nx + 7,
                      nn - 1, nn - nx], np.int32)
    h.map_dsmc_to_lbm(torch.from_numpy(nodes).cuda())
    o.map_dsmc_to_lbm(nodes)
    h.sync()
    q = h.d["q"]
    gf = h.f().cpu().numpy().reshape(q, -1)[:, nodes].astype(np.float64)
    of = o.f().reshape(q, -1)[:, nodes].astype(np.float64)
    e, w, r = O.lattice(lattice)
    tol = 2e-6 * (np.abs(of) + w[:, None])
    assert np.all(np.abs(gf - of) <= tol), np.abs((gf - of) / (np.abs(of) + w[:, None])).max()
    assert h.sync_status()[1] == 0


@pytest.mark.parametrize("real_bytes,lb_ratio", [(4, 2), (8, 1)])
def test_lb2dsmc_3d_matches_oracle(real_bytes, lb_ratio):
    cfg = cfg3(real_bytes=real_bytes, lb_ratio=lb_ratio)
    h, o = B.Hybrid(cfg), O.Oracle(cfg)
    h.dsmc_step(1)
    o.dsmc_step(1)
    e, w, r = O.lattice(39)
    f0 = W.gen_populations(w, h.d["nnodes"], seed=8, eps=0.08, rho_eps=0.2)
    f0 = f0.astype(np.float32 if real_bytes == 4 else np.float64)
    h.f().copy_(torch.from_numpy(f0.reshape(h.f().shape)))
    torch.cuda.synchronize()
    o.set_f(f0)
    cells = np.array([0, 12, 91 + 40, 2 * 91 + 90, 2 * 91 + 5, 272], np.int32)
    h.map_lbm_to_dsmc(torch.from_numpy(cells).cuda())
    o.map_lbm_to_dsmc(cells)
    assert h.n_tot() == o.scalars()["ntot"]
    gp = gpu_particles(h)
    assert_particles_match(gp, o.particles(), real_bytes)
    hc, oc = h.counters(), o.counters()
    for k in ("created", "deleted", "l2d_attempts", "envelope"):
        assert hc[k] == oc[k], (k, hc[k], oc[k])
    cs = h.cell_start().cpu().numpy()
    own = np.repeat(np.arange(h.d["ncells"]), np.diff(cs))
    assert np.array_equal(cell_of(gp, 13, 7), own)
    h.dsmc_step(1)
    o.dsmc_step(1)
    compare_dsmc(h, o, real_bytes)


def test_hybrid_3d_fp64_graph_matches_oracle():
    cfg = cfg3(ncx=16, ncy=4, ncz=2, ppc=40, real_bytes=8, lb_ratio=2, seed=3)
    nodes, cells = W.coupling_sites(cfg)
    h, o = B.Hybrid(cfg), O.Oracle(cfg)
    dn, dc = torch.from_numpy(nodes).cuda(), torch.from_numpy(cells).cuda()
    for _ in range(4):
        h.hybrid_step(dn, dc, nsteps=1, use_graph=True)
        o.dsmc_step(1)
        o.map_dsmc_to_lbm(nodes)
        o.lbm_step(1)
        o.map_lbm_to_dsmc(cells)
    compare_dsmc(h, o, 8)
    h.sync()
    assert np.allclose(h.f().cpu().numpy(), o.f(), rtol=1e-11, atol=1e-14)


@pytest.mark.parametrize("lattice", [39, 19])
def test_lbm_step_nodes_3d_matches_oracle(lattice):
    # the differentiated LBM's forward in 3D: per-node g and tau
    cfg = cfg3(ncx=6, ncy=3, ncz=2, lb_ratio=1, lattice=lattice, real_bytes=8, ma=0.5, kn=0.3)
    h, o = B.Hybrid(cfg), O.Oracle(cfg)
    d = h.d
    e, w, r = O.lattice(lattice)
    rng = np.random.default_rng(3)
    f0 = W.gen_populations(w, d["nnodes"], seed=13)
    g = d["g_step"] * (1 + 0.3 * rng.standard_normal(d["nnodes"]))
    tau = d["tau"] * (1 + 0.1 * rng.standard_normal(d["nnodes"]))
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    a_, b_ = dev(f0.reshape(h.f().shape)), torch.empty(h.f().shape, dtype=torch.float64, device="cuda")
    o.set_f(f0)
    o.set_node_params(g, tau)
    for _ in range(2):
        h.lbm_step_nodes(a_, b_, dev(g), dev(tau))
        a_, b_ = b_, a_
    o.lbm_step(2)
    h.sync()
    err = np.abs(a_.cpu().numpy() - o.f()) / (np.abs(o.f()) + 1e-3 * w[:, None, None, None])
    assert err.max() < 1e-12


@pytest.mark.parametrize("lattice", [39, 19])
def test_adjoint_gradient_3d_matches_oracle_central_differences(lattice):
    # the adjoint in 3D (pull transposed over z too, wall sums per (y, z) row) against the
    # oracle's central differences of the FP64 forward, over every node's g and tau
    cfg = cfg3(ncx=6, ncy=3, ncz=2, lb_ratio=1, lattice=lattice, real_bytes=8, ma=0.5, kn=0.3)
    h = B.Hybrid(cfg)
    d = h.d
    assert d["nz"] == 2 and d["nnodes"] == 36
    e, w, r = O.lattice(lattice)
    rng = np.random.default_rng(4)
    f0 = W.gen_populations(w, d["nnodes"], seed=14)
    g = d["g_step"] * (1 + 0.3 * rng.standard_normal(d["nnodes"]))
    tau = d["tau"] * (1 + 0.1 * rng.standard_normal(d["nnodes"]))
    nodes = np.array([1, 8, 13, 20, 27, 34], np.int32)  # both layers, near both walls
    o = O.Oracle(cfg)
    o.set_f(f0)
    o.set_node_params(g, tau)
    o.lbm_step(3)
    targets = np.stack([o.grad_node(n) for n in nodes]) + 0.02 * rng.standard_normal((len(nodes), 20))
    T = 3
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    g_t, tau_t = dev(g).requires_grad_(True), dev(tau).requires_grad_(True)
    f_t = dev(f0.reshape(h.f().shape)).requires_grad_(True)
    loss = B.interface_loss(h, g_t, tau_t, f_t, dev(nodes), dev(targets), T, ckpt_every=2)
    loss.backward()
    want_loss = O.interface_loss_after(cfg, f0, g, tau, nodes, targets, T)
    assert float(loss.detach()) == pytest.approx(want_loss, rel=1e-10)
    want_g, want_t = O.interface_loss_fd_gradient(cfg, f0, g, tau, nodes, targets, T)
    for got, want in ((g_t.grad.cpu().numpy(), want_g), (tau_t.grad.cpu().numpy(), want_t)):
        scale = np.abs(want).max()
        assert scale > 0
        assert np.abs(got - want).max() < 1e-6 * scale, np.abs(got - want).max() / scale
    # populations: a directional derivative of the FP64 forward
    v = rng.standard_normal(f0.shape)
    eps = 1e-6
    lp = O.interface_loss_after(cfg, f0 + eps * v, g, tau, nodes, targets, T)
    lm = O.interface_loss_after(cfg, f0 - eps * v, g, tau, nodes, targets, T)
    got = float((f_t.grad.cpu().numpy().reshape(f0.shape) * v).sum())
    assert got == pytest.approx((lp - lm) / (2 * eps), rel=1e-6)
