"""Parity of the CUDA library with the CPU oracle, through the C ABI, on the same seeded
inputs. Integers (cell keys via cell_start, collision/candidate counts, particle counts) are
compared bit for bit; floating-point state within the tolerances stated per test."""
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

# Float tolerance for state computed in float on both sides (the FP32 path), and the share
# of values allowed to differ in the last bit through double transcendentals rounded to float.
RTOL = 1e-5


def cfg_small(**kw):
    base = dict(ncx=13, ncy=7, ppc=23, real_bytes=4, seed=11, kn=0.1, capacity_factor=1.5)
    base.update(kw)
    return W.config(**base)


def gpu_particles(h):
    h.sync()
    p = h.particles()
    return {k: v.cpu().numpy() for k, v in p.items()}


def assert_particles_match(gp, op, real_bytes, exact_frac=0.9999):
    for k in ("x", "y", "vx", "vy", "vz"):
        a, b = gp[k], op[k]
        assert a.shape == b.shape, k
        eq = (a == b).mean() if a.size else 1.0
        if real_bytes == 4:
            assert eq >= exact_frac, (k, eq)
            assert np.allclose(a, b, rtol=RTOL, atol=RTOL), (k, np.abs(a - b).max())
        else:
            assert np.allclose(a, b, rtol=1e-12, atol=1e-12), (k, np.abs(a - b).max())


def test_philox_matches_oracle_word_for_word():
    rng = np.random.default_rng(0)
    ctr = rng.integers(0, 2 ** 32, size=(100_000, 4), dtype=np.uint64).astype(np.uint32)
    ctr[:3] = [[0, 0, 0, 0], [0xFFFFFFFF] * 4, [0x243f6a88, 0x85a308d3, 0x13198a2e, 0x03707344]]
    seed = 0xDEADBEEF12345678
    want = O.philox(ctr, seed)
    c = torch.from_numpy(ctr.view(np.int32)).cuda()
    out = torch.empty_like(c)
    B.debug_philox(c, seed, out)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy().view(np.uint32), want)


@pytest.mark.parametrize("real_bytes", [4, 8])
def test_init_matches_oracle(real_bytes):
    cfg = cfg_small(real_bytes=real_bytes)
    h = B.Hybrid(cfg)
    o = O.Oracle(cfg)
    assert h.n_tot() == o.scalars()["ntot"]
    gp, op = gpu_particles(h), o.particles()
    assert np.array_equal(gp["x"], op["x"]) and np.array_equal(gp["y"], op["y"])
    assert_particles_match(gp, op, real_bytes)
    assert np.array_equal(h.cell_start().cpu().numpy().astype(np.uint32), o.get(O.A_CELL_START))
    f = h.f().cpu().numpy()
    assert np.array_equal(f, o.f())


def _compare_dsmc(h, o, real_bytes, acc_rtol=1e-5, acc_scale=None):
    """acc_scale: per cell and moment, the sum over the steps of the cell's sums of |term|
    (moment_abs_sums), the scale of each FP64 sum's rounding; else the column's largest sum."""
    assert h.n_tot() == o.scalars()["ntot"]
    assert np.array_equal(h.cell_start().cpu().numpy().astype(np.uint32), o.get(O.A_CELL_START))
    assert_particles_match(gpu_particles(h), o.particles(), real_bytes)
    hc, oc = h.counters(), o.counters()
    for k in ("candidates", "collisions", "wall_hits", "created", "deleted"):
        assert hc[k] == oc[k], (k, hc[k], oc[k])
    if real_bytes == 4:
        assert np.array_equal(h.crmax().cpu().numpy(), o.get(O.A_CRMAX))
        assert np.array_equal(h.rem().cpu().numpy(), o.get(O.A_REM))
    else:
        # double state draws its normals with the platform's double log/sin/cos, which may
        # differ in the last bit between the GPU and the host
        assert np.allclose(h.crmax().cpu().numpy(), o.get(O.A_CRMAX), rtol=1e-12, atol=0)
        assert np.allclose(h.rem().cpu().numpy(), o.get(O.A_REM), rtol=0, atol=1e-9)
    assert np.array_equal(h.nbar_sum().cpu().numpy().view(np.uint32), o.get(O.A_NBAR_SUM))
    ga = h.acc().cpu().numpy()
    oa = o.acc()
    scale = acc_scale if acc_scale is not None else np.abs(oa).max(axis=0, keepdims=True) + 1e-30
    assert np.all(np.abs(ga - oa) <= acc_rtol * scale), np.abs((ga - oa) / (scale + 1e-300)).max()
    ctrl = h.ctrl().cpu().numpy()
    s = o.scalars()
    assert ctrl[B.CTRL_STEP] == s["step"] and ctrl[B.CTRL_NSAMPLES] == s["nsamples"]
    assert ctrl[B.CTRL_STATUS] == s["status"]


@pytest.mark.parametrize("real_bytes,steps", [(4, 1), (4, 4), (8, 3)])
def test_dsmc_steps_match_oracle(real_bytes, steps):
    # the moment sums per element, each to 1e-5 of its own scale (the sum of |term| of the
    # samples it holds)
    cfg = cfg_small(real_bytes=real_bytes, ma=0.3)
    h = B.Hybrid(cfg)
    o = O.Oracle(cfg)
    scale = 0.0
    for _ in range(steps):
        h.dsmc_step(1)
        o.dsmc_step(1)
        scale = scale + moment_abs_sums(o.particles(), o.get(O.A_CELL_START))
    _compare_dsmc(h, o, real_bytes, acc_scale=scale)


def test_dsmc_first_step_full_size_64x256_ppc50():
    # the 819,200-particle channel at its benchmark launch configuration
    cfg = W.WORKLOADS["poiseuille_64x256_ppc50_fp32"]
    h = B.Hybrid(cfg)
    o = O.Oracle(cfg)
    h.dsmc_step(1)
    o.dsmc_step(1)
    _compare_dsmc(h, o, 4, acc_scale=moment_abs_sums(o.particles(), o.get(O.A_CELL_START)))


def test_dsmc_synthetic_state_empty_and_crowded_cells():
    # Poisson cell counts with empty cells and one crowded cell (the largest in-register sort)
    cfg = cfg_small(ncx=9, ncy=5, ppc=20, capacity_factor=12.8, seed=3)
    st = W.gen_particles(9, 5, 20, seed=5, empty_fraction=0.2)
    counts = np.diff(st["cell_start"].astype(np.int64))
    extra = W.gen_particles(1, 1, 170, seed=6)  # crowd cell 17
    c = 17
    ix, iy = c % 9, c // 9
    lo, hi = st["cell_start"][c], st["cell_start"][c + 1]
    ins = {k: np.concatenate([st[k][:hi], (extra[k] + (ix if k == "x" else iy if k == "y" else 0))
                              , st[k][hi:]]) for k in ("x", "y", "vx", "vy", "vz")}
    counts[c] += extra["x"].size
    cs = np.zeros(46, np.uint32)
    cs[1:] = np.cumsum(counts)
    assert 128 < counts[c] <= 256 and (counts == 0).sum() > 3
    args = [ins[k].astype(np.float32) for k in ("x", "y", "vx", "vy", "vz")]
    h = B.Hybrid(cfg)
    o = O.Oracle(cfg)
    h.load_particles(*args, cs)
    o.set_particles(*args, cs)
    for _ in range(2):
        h.dsmc_step(1)
        o.dsmc_step(1)
    _compare_dsmc(h, o, 4)


@pytest.mark.parametrize("lattice,real_bytes", [(39, 4), (39, 8), (19, 4)])
def test_lbm_steps_match_oracle(lattice, real_bytes):
    cfg = cfg_small(lattice=lattice, real_bytes=real_bytes, lb_ratio=2, ma=0.5, kn=0.3)
    h = B.Hybrid(cfg)
    o = O.Oracle(cfg)
    e, w, r = O.lattice(lattice)
    f0 = W.gen_populations(w, h.d["nnodes"], seed=21).astype(np.float32 if real_bytes == 4 else np.float64)
    h.f().copy_(torch.from_numpy(f0.reshape(h.f().shape)))
    torch.cuda.synchronize()
    o.set_f(f0)
    for step in range(3):
        h.lbm_step(1)
        o.lbm_step(1)
        h.sync()
        gf, of = h.f().cpu().numpy(), o.f()
        tol = LB_TOL_FP32 if real_bytes == 4 else LB_TOL_FP64
        err = lb_err(gf, of, w)
        assert err < tol, (step, err)
    # mass is conserved
    assert abs(h.f().double().sum().item() / f0.astype(np.float64).sum() - 1) < 1e-6


def _set_acc(h, o, acc, S):
    h.acc().copy_(torch.from_numpy(acc))
    h.set_counters(nsamples=S)
    o.set(O.A_ACC, acc.reshape(-1))
    o.set_scalars(o.scalars()["step"], S)


@pytest.mark.parametrize("lattice,lb_ratio", [(39, 2), (19, 1), (39, 1)])
def test_dsmc2lb_matches_oracle(lattice, lb_ratio):
    cfg = cfg_small(lattice=lattice, lb_ratio=lb_ratio)
    h = B.Hybrid(cfg)
    o = O.Oracle(cfg)
    # cumulative sums from a few real DSMC steps of the oracle
    src = O.Oracle(cfg_small(lattice=lattice, lb_ratio=lb_ratio, ma=0.4))
    src.dsmc_step(5)
    _set_acc(h, o, src.acc().copy(), src.scalars()["nsamples"])
    nx = h.d["nx"]
    nodes = np.array([0, 1, nx - 1, nx + 5, h.d["nnodes"] - 1, 3 * nx + 7], np.int32)
    h.map_dsmc_to_lbm(torch.from_numpy(nodes).cuda())
    o.map_dsmc_to_lbm(nodes)
    h.sync()
    gf = h.f().cpu().numpy().reshape(h.d["q"], -1)[:, nodes].astype(np.float64)
    of = o.f().reshape(h.d["q"], -1)[:, nodes].astype(np.float64)
    e, w, r = O.lattice(lattice)
    # FP64 coefficients, Hermite series evaluated in the state precision
    tol = (2e-6 if cfg["real_bytes"] == 4 else 1e-13) * (np.abs(of) + w[:, None])
    assert np.all(np.abs(gf - of) <= tol), np.abs((gf - of) / (np.abs(of) + w[:, None])).max()
    assert h.sync_status()[1] == 0


@pytest.mark.parametrize("lattice,real_bytes,lb_ratio", [(39, 4, 2), (39, 8, 1), (19, 4, 1)])
def test_lb2dsmc_matches_oracle(lattice, real_bytes, lb_ratio):
    cfg = cfg_small(lattice=lattice, real_bytes=real_bytes, lb_ratio=lb_ratio)
    h = B.Hybrid(cfg)
    o = O.Oracle(cfg)
    h.dsmc_step(1)
    o.dsmc_step(1)
    # non-equilibrium populations: DSMC2LB projections of sampled moments, perturbed
    e, w, r = O.lattice(lattice)
    f0 = W.gen_populations(w, h.d["nnodes"], seed=8, eps=0.08, rho_eps=0.2)
    f0 = f0.astype(np.float32 if real_bytes == 4 else np.float64)
    h.f().copy_(torch.from_numpy(f0.reshape(h.f().shape)))
    torch.cuda.synchronize()
    o.set_f(f0)
    cells = np.array([0, 5, 12, 13, 40, 90], np.int32)
    n0 = h.n_tot()
    h.map_lbm_to_dsmc(torch.from_numpy(cells).cuda())
    o.map_lbm_to_dsmc(cells)
    assert h.n_tot() == o.scalars()["ntot"]
    assert_particles_match(gpu_particles(h), o.particles(), real_bytes)
    hc, oc = h.counters(), o.counters()
    for k in ("created", "deleted", "l2d_attempts", "envelope"):
        assert hc[k] == oc[k], (k, hc[k], oc[k])
    # the next step compacts the deleted particles away identically
    h.dsmc_step(1)
    o.dsmc_step(1)
    _compare_dsmc(h, o, real_bytes)


def test_lb2dsmc_skips_invalid_cells_like_oracle():
    cfg = cfg_small(lb_ratio=2)
    h = B.Hybrid(cfg)
    o = O.Oracle(cfg)
    h.dsmc_step(1)
    o.dsmc_step(1)
    e, w, r = O.lattice(39)
    f0 = W.gen_populations(w, h.d["nnodes"], seed=9, eps=0.05).astype(np.float32)
    h.f().copy_(torch.from_numpy(f0.reshape(h.f().shape)))
    torch.cuda.synchronize()
    o.set_f(f0)
    cells = np.array([3, -1, 17, 10 ** 6, 30], np.int32)
    h.map_lbm_to_dsmc(torch.from_numpy(cells).cuda())
    o.map_lbm_to_dsmc(cells)
    rc, bits = h.sync_status()
    assert rc == B.HYB_EINVAL and bits & B.ST_BAD_INPUT
    assert o.scalars()["status"] & B.ST_BAD_INPUT
    assert h.n_tot() == o.scalars()["ntot"]
    assert_particles_match(gpu_particles(h), o.particles(), 4)


def test_hybrid_steps_fp64_match_oracle():
    # the 64-cell channel of the paper's mapping tests, FP64, two coupling nodes/cells
    cfg = W.WORKLOADS["poiseuille_64x1_ppc100_fp64"]
    nodes, cells = W.coupling_sites(cfg)
    h = B.Hybrid(cfg)
    o = O.Oracle(cfg)
    dn, dc = torch.from_numpy(nodes).cuda(), torch.from_numpy(cells).cuda()
    for _ in range(4):
        h.hybrid_step(dn, dc, nsteps=1, use_graph=False)
        o.dsmc_step(1)
        o.map_dsmc_to_lbm(nodes)
        o.lbm_step(1)
        o.map_lbm_to_dsmc(cells)
    _compare_dsmc(h, o, 8)
    h.sync()
    assert np.allclose(h.f().cpu().numpy(), o.f(), rtol=1e-11, atol=1e-14)


def test_graph_replay_equals_direct_launches():
    cfg = cfg_small(lb_ratio=2, ncy=8)
    nodes, cells = W.coupling_sites(cfg, strip_cells=2)
    dn, dc = torch.from_numpy(nodes).cuda(), torch.from_numpy(cells).cuda()
    a = B.Hybrid(cfg)
    b = B.Hybrid(cfg)
    a.hybrid_step(dn, dc, nsteps=5, use_graph=False)
    for _ in range(5):
        b.hybrid_step(dn, dc, nsteps=1, use_graph=True)
    a.sync()
    b.sync()
    assert a.current() == b.current()
    # the state is identical; scratch (perm, arrival) holds atomic-order-dependent values
    assert a.n_tot() == b.n_tot()
    for k in ("x", "y", "vx", "vy", "vz"):
        assert torch.equal(a.particles()[k], b.particles()[k]), k
    for name in ("cell_start", "crmax", "rem", "nbar_sum", "acc", "f"):
        assert torch.equal(getattr(a, name)(), getattr(b, name)()), name
    assert torch.equal(a.ctrl()[:4], b.ctrl()[:4])
    assert a.counters() == b.counters()


def test_sample_moments_copy_and_reset():
    cfg = cfg_small()
    h = B.Hybrid(cfg)
    h.dsmc_step(3)
    out = torch.zeros(h.L.ncells, 20, dtype=torch.float64, device="cuda")
    h.sample_moments(out, reset=True)
    h.sync()
    assert out[:, 0].sum().item() == 3 * h.n_tot()
    assert h.acc().abs().sum().item() == 0
    assert int(h.ctrl()[B.CTRL_NSAMPLES].item()) == 0


def test_status_on_capacity_overflow_and_bad_index():
    cfg = cfg_small(capacity_factor=1.0)
    h = B.Hybrid(cfg)
    h.dsmc_step(1)
    e, w, r = O.lattice(39)
    f = torch.from_numpy((w[:, None] * 3.0 * np.ones((1, h.d["nnodes"]))).astype(np.float32))
    h.f().copy_(f.view(h.f().shape))
    torch.cuda.synchronize()
    before = h.n_tot()
    h.map_lbm_to_dsmc(torch.tensor([4, 5], dtype=torch.int32, device="cuda"))
    rc, bits = h.sync_status()
    assert rc == B.HYB_ECAPACITY and bits & B.ST_CAPACITY
    assert h.n_tot() == before  # nothing appended, nothing deleted
    h2 = B.Hybrid(cfg_small())
    h2.dsmc_step(1)
    h2.map_dsmc_to_lbm(torch.tensor([10 ** 6], dtype=torch.int32, device="cuda"))
    rc, bits = h2.sync_status()
    assert rc == B.HYB_EINVAL and bits & B.ST_BAD_INPUT


# ---------------------------------------------------------------------------------------
# The proof-of-concept hybrid of Sec. 4: unregularised BGK, equilibrium DSMC2LB

@pytest.mark.parametrize("lattice,real_bytes", [(19, 4), (19, 8), (39, 8)])
def test_lbm_bgk_steps_match_oracle(lattice, real_bytes):
    cfg = cfg_small(lattice=lattice, real_bytes=real_bytes, lb_ratio=2, ma=0.5, kn=0.3,
                    lb_collision=1)
    h = B.Hybrid(cfg)
    o = O.Oracle(cfg)
    e, w, r = O.lattice(lattice)
    f0 = W.gen_populations(w, h.d["nnodes"], seed=23).astype(np.float32 if real_bytes == 4 else np.float64)
    h.f().copy_(torch.from_numpy(f0.reshape(h.f().shape)))
    torch.cuda.synchronize()
    o.set_f(f0)
    for step in range(3):
        h.lbm_step(1)
        o.lbm_step(1)
        h.sync()
        gf, of = h.f().cpu().numpy(), o.f()
        err = lb_err(gf, of, w)
        assert err < (LB_TOL_FP32 if real_bytes == 4 else LB_TOL_FP64), (step, err)
    # differs from the regularised step (the ghost modes of the perturbed state survive)
    cfg_r = dict(cfg, lb_collision=0)
    o2 = O.Oracle(cfg_r)
    o2.set_f(f0)
    o2.lbm_step(3)
    assert np.abs(o2.f() - o.f()).max() > 1e-6


@pytest.mark.parametrize("lattice", [19, 39])
def test_dsmc2lb_equilibrium_mode_matches_oracle(lattice):
    cfg = cfg_small(lattice=lattice, lb_ratio=1, real_bytes=8, d2l_mode=1)
    h = B.Hybrid(cfg)
    o = O.Oracle(cfg)
    rng = np.random.default_rng(31)
    n = h.d["ncells"]
    S = 9
    acc = np.zeros((n, 20))
    for c in range(n):
        v = rng.standard_normal((cfg["ppc"] * S, 3)) * (1 + 0.2 * rng.random(3)) + 0.1 * rng.standard_normal(3)
        m = [np.ones(len(v))] + [v[:, i] for i in range(3)]
        m += [v[:, i] * v[:, j] for i in range(3) for j in range(i, 3)]
        m += [v[:, i] * v[:, j] * v[:, k] for i in range(3) for j in range(i, 3) for k in range(j, 3)]
        acc[c] = [x.sum() for x in m]
    _set_acc(h, o, acc, S)
    nodes = np.arange(0, h.d["nnodes"], 3, dtype=np.int32)
    h.map_dsmc_to_lbm(torch.from_numpy(nodes).cuda())
    o.map_dsmc_to_lbm(nodes)
    h.sync()
    assert np.allclose(h.f().cpu().numpy(), o.f(), rtol=1e-12, atol=1e-15)


def test_proof_of_concept_hybrid_steps_match_oracle():
    # Sec. 4 at a reduced size: D3Q19 without regularisation, equilibrium DSMC2LB on the
    # buffer row at y = L0/2, no LB2DSMC; FP64, four hybrid steps
    cfg = W.config(ncx=12, ncy=8, ppc=30, lattice=19, lb_ratio=1, kn=0.05, ma=0.1, real_bytes=8,
                   lb_collision=1, d2l_mode=1, coupling="buffer_row", seed=4)
    nodes, cells = W.coupling_sites(cfg)
    assert len(cells) == 0 and len(nodes) == cfg["ncx"]
    h = B.Hybrid(cfg)
    o = O.Oracle(cfg)
    dn, dc = torch.from_numpy(nodes).cuda(), torch.from_numpy(cells).cuda()
    for _ in range(4):
        h.hybrid_step(dn, dc, nsteps=1, use_graph=False)
        o.dsmc_step(1)
        o.map_dsmc_to_lbm(nodes)
        o.lbm_step(1)
    _compare_dsmc(h, o, 8)
    h.sync()
    assert np.allclose(h.f().cpu().numpy(), o.f(), rtol=1e-11, atol=1e-14)


# ---------------------------------------------------------------------------------------
# Kn varying along the channel

@pytest.mark.parametrize("real_bytes,steps", [(4, 3), (8, 2)])
def test_dsmc_steps_with_kn_profile_match_oracle(real_bytes, steps):
    cfg = cfg_small(real_bytes=real_bytes, ncy=12, kn=0.03, kn_profile=1, kn_end=0.6)
    h = B.Hybrid(cfg)
    o = O.Oracle(cfg)
    for _ in range(steps):
        h.dsmc_step(1)
        o.dsmc_step(1)
    _compare_dsmc(h, o, real_bytes)
    c = h.counters()
    oc = o.counters()
    assert c["candidates"] == oc["candidates"] and c["collisions"] == oc["collisions"]


@pytest.mark.parametrize("lattice,real_bytes", [(39, 4), (39, 8)])
def test_lbm_steps_with_kn_profile_match_oracle(lattice, real_bytes):
    cfg = cfg_small(lattice=lattice, real_bytes=real_bytes, lb_ratio=2, ncy=8, ma=0.5, kn=0.05,
                    kn_profile=1, kn_end=0.5)
    h = B.Hybrid(cfg)
    o = O.Oracle(cfg)
    e, w, r = O.lattice(lattice)
    f0 = W.gen_populations(w, h.d["nnodes"], seed=29).astype(np.float32 if real_bytes == 4 else np.float64)
    h.f().copy_(torch.from_numpy(f0.reshape(h.f().shape)))
    torch.cuda.synchronize()
    o.set_f(f0)
    for step in range(3):
        h.lbm_step(1)
        o.lbm_step(1)
        h.sync()
        err = lb_err(h.f().cpu().numpy(), o.f(), w)
        assert err < (LB_TOL_FP32 if real_bytes == 4 else LB_TOL_FP64), (step, err)


def test_hybrid_steps_with_kn_profile_fp64_match_oracle():
    cfg = cfg_small(real_bytes=8, lb_ratio=2, ncy=8, kn=0.05, kn_profile=1, kn_end=0.5)
    nodes, cells = W.coupling_sites(cfg, strip_cells=2)
    h = B.Hybrid(cfg)
    o = O.Oracle(cfg)
    dn, dc = torch.from_numpy(nodes).cuda(), torch.from_numpy(cells).cuda()
    for _ in range(3):
        h.hybrid_step(dn, dc, nsteps=1, use_graph=True)
        o.dsmc_step(1)
        o.map_dsmc_to_lbm(nodes)
        o.lbm_step(1)
        o.map_lbm_to_dsmc(cells)
    _compare_dsmc(h, o, 8)
    h.sync()
    assert np.allclose(h.f().cpu().numpy(), o.f(), rtol=1e-11, atol=1e-14)


@pytest.mark.parametrize("pinned", [True, False])
def test_host_buffer_steps_equal_device_list_steps(pinned):
    # hyb_hybrid_step_host: host lists in, the listed cells' moment sums and the status out;
    # the state equals that of the same steps with device lists, and the returned sums are
    # the arena's rows of the listed cells (zeros for an index out of range)
    cfg = cfg_small(lb_ratio=2, ma=0.3)
    nodes, cells = W.coupling_sites(cfg, strip_cells=2)
    cells_h = np.concatenate([cells, [10 ** 6]]).astype(np.int32)  # one index out of range
    a, b = B.Hybrid(cfg), B.Hybrid(cfg)
    dn, dc = torch.from_numpy(nodes).cuda(), torch.from_numpy(cells_h).cuda()
    mk = (lambda x: torch.from_numpy(x).pin_memory()) if pinned else torch.from_numpy
    hn, hc = mk(nodes), mk(cells_h)
    outs = [mk(np.zeros((len(cells_h), 20))), mk(np.zeros((len(cells_h), 20)))]
    st = [mk(np.zeros(1, np.int32)), mk(np.zeros(1, np.int32))]
    for k in range(5):
        a.hybrid_step(dn, dc, nsteps=1, use_graph=True)
        b.hybrid_step_host(hn, hc, outs[k % 2], st[k % 2])
        if k > 0:
            b.host_wait(1)
    b.host_wait(0)
    a.sync()
    last = outs[4 % 2].numpy()
    acc = b.acc().cpu().numpy()
    assert np.array_equal(last[:-1], acc[cells]) and np.all(last[-1] == 0)
    assert np.array_equal(a.acc().cpu().numpy(), acc)
    for k in ("x", "y", "vx", "vy", "vz"):
        assert np.array_equal(gpu_particles(a)[k], gpu_particles(b)[k]), k
    assert np.array_equal(a.f().cpu().numpy(), b.f().cpu().numpy())
    bits = b.ctrl().cpu().numpy()[B.CTRL_STATUS]
    assert int(st[0].numpy()[0]) == int(st[1].numpy()[0]) == bits
    assert bits & B.ST_BAD_INPUT  # the out-of-range cell was flagged by LB2DSMC
    with pytest.raises(ValueError):
        b.hybrid_step_host(hn, hc, outs[0][:1], st[0])  # result buffer too small
    with pytest.raises(B.HybError):
        b.host_wait(4)


@pytest.mark.parametrize("fuse,pinned", [("always", True), ("never", True), ("always", False)])
def test_multi_step_host_calls_equal_one_step_host_calls(fuse, pinned):
    # hyb_hybrid_steps_host: several steps per call, each copying its lists in and its sums and
    # status out, the DSMC passes fused across the call's steps (or not): every step's returned
    # sums and the final state equal those of one-step host calls. With page-locked buffers
    # the call is a graph, captured at the first two calls and replayed at the third (the same
    # buffers and state halves as the first); pageable buffers take direct launches.
    cfg = cfg_small(lb_ratio=2, ma=0.3)
    nodes, cells = W.coupling_sites(cfg, strip_cells=2)
    a, b = B.Hybrid(cfg), B.Hybrid(cfg)
    b.set_fuse(fuse)
    mk = (lambda x: x.pin_memory()) if pinned else (lambda x: x)
    hn, hc = mk(torch.from_numpy(nodes)), mk(torch.from_numpy(cells))
    n = 9
    one = np.zeros((n, len(cells), 20))
    for k in range(n):
        out = torch.zeros(1, len(cells), 20, dtype=torch.float64).pin_memory()
        st = torch.zeros(1, dtype=torch.int32).pin_memory()
        a.hybrid_step_host(hn, hc, out, st)
        a.host_wait(0)
        one[k] = out.numpy()[0]
    many = [mk(torch.zeros(3, len(cells), 20, dtype=torch.float64)) for _ in range(2)]
    sts = [mk(torch.zeros(3, dtype=torch.int32)) for _ in range(2)]
    got, got_st = [], []
    for call in range(3):
        b.hybrid_step_host(hn, hc, many[call % 2], sts[call % 2], nsteps=3)
        b.host_wait(0)
        got.append(many[call % 2].numpy().copy())
        got_st.append(sts[call % 2].numpy().copy())
    assert np.array_equal(np.concatenate(got), one)
    assert np.all(np.concatenate(got_st) == 0)
    for k in ("x", "y", "vx", "vy", "vz"):
        assert np.array_equal(gpu_particles(a)[k], gpu_particles(b)[k]), k
    assert np.array_equal(a.f().cpu().numpy(), b.f().cpu().numpy())
    assert a.counters() == b.counters()


def test_host_step_graphs_follow_the_fuse_mode_and_3d():
    # a captured host call is replayed only while the step it captured still applies: after
    # hyb_set_fuse changes the pass structure the call is captured again, and the results stay
    # those of one-step host calls; the same on a 3D channel (ncz >= 2)
    for cfg in (cfg_small(lb_ratio=2, ma=0.3), cfg_small(ncz=3, lb_ratio=2, ma=0.3, kn=0.3)):
        nodes, cells = W.coupling_sites(cfg, strip_cells=2)
        a, b = B.Hybrid(cfg), B.Hybrid(cfg)
        hn, hc = torch.from_numpy(nodes).pin_memory(), torch.from_numpy(cells).pin_memory()
        n = 8
        one = np.zeros((n, len(cells), 20))
        out = torch.zeros(1, len(cells), 20, dtype=torch.float64).pin_memory()
        st = torch.zeros(1, dtype=torch.int32).pin_memory()
        for k in range(n):
            a.hybrid_step_host(hn, hc, out, st)
            a.host_wait(0)
            one[k] = out.numpy()[0]
        many = torch.zeros(2, len(cells), 20, dtype=torch.float64).pin_memory()
        sts = torch.zeros(2, dtype=torch.int32).pin_memory()
        got = []
        for call, mode in enumerate(("always", "always", "never", "always")):
            b.set_fuse(mode)
            b.hybrid_step_host(hn, hc, many, sts, nsteps=2)
            b.host_wait(0)
            got.append(many.numpy().copy())
            assert np.all(sts.numpy() == 0)
        assert np.array_equal(np.concatenate(got), one)
        for k in ("x", "y", "vx", "vy", "vz"):
            assert np.array_equal(gpu_particles(a)[k], gpu_particles(b)[k]), k
        assert np.array_equal(a.f().cpu().numpy(), b.f().cpu().numpy())


@pytest.mark.parametrize("pinned", [True, False])
def test_host_steps_with_empty_lists(pinned):
    # host-buffer steps with no coupling nodes or cells: only the status words come back, and
    # the state equals that of uncoupled device steps
    cfg = cfg_small(lb_ratio=2, ma=0.3)
    a, b = B.Hybrid(cfg), B.Hybrid(cfg)
    mk = (lambda x: x.pin_memory()) if pinned else (lambda x: x)
    none = mk(torch.zeros(0, dtype=torch.int32))
    acc = mk(torch.zeros(0, dtype=torch.float64))
    st = mk(torch.full((2,), -1, dtype=torch.int32))
    e = torch.zeros(0, dtype=torch.int32, device="cuda")
    a.hybrid_step(e, e, nsteps=3, use_graph=False)
    b.hybrid_step_host(none, none, acc, st[:1])
    b.hybrid_step_host(none, none, acc, st, nsteps=2)
    b.host_wait(0)
    a.sync()
    assert np.all(st.numpy() == 0)
    for k in ("x", "y", "vx", "vy", "vz"):
        assert np.array_equal(gpu_particles(a)[k], gpu_particles(b)[k]), k
    assert np.array_equal(a.f().cpu().numpy(), b.f().cpu().numpy())


# ---------------------------------------------------------------------------------------
# The benchmarked FP32 coupled step, from the GPU's own state, sub-step by sub-step

def load_oracle_from_gpu(o, h):
    """The oracle takes the GPU's whole state: particles in cell order, the per-cell NTC
    state, the cumulative sums, the populations and the step and sample counts."""
    h.sync()
    p = gpu_particles(h)
    cs = h.cell_start().cpu().numpy().astype(np.uint32)
    o.set_particles(p["x"], p["y"], p["vx"], p["vy"], p["vz"], cs, z=p.get("z"))
    o.set(O.A_CRMAX, h.crmax().cpu().numpy())
    o.set(O.A_REM, h.rem().cpu().numpy())
    o.set(O.A_NBAR_SUM, h.nbar_sum().cpu().numpy().view(np.uint32))
    o.set(O.A_ACC, h.acc().cpu().numpy().reshape(-1))
    o.set_f(h.f().cpu().numpy())
    ctrl = h.ctrl().cpu().numpy()
    o.set_scalars(int(ctrl[B.CTRL_STEP]), int(ctrl[B.CTRL_NSAMPLES]))


def moment_abs_sums(p, cs):
    """Per cell and moment, the sum over the cell's particles of the absolute value of the
    moment's term (1, |v_i|, |v_i v_j|, |v_i v_j v_k|): the scale of the rounding error of a
    sum of those terms."""
    v = np.stack([p["vx"], p["vy"], p["vz"]], 1).astype(np.float64)
    ncell = len(cs) - 1
    cell = np.repeat(np.arange(ncell), np.diff(cs.astype(np.int64)))
    terms = [np.ones(len(v))] + [np.abs(v[:, i]) for i in range(3)]
    terms += [np.abs(v[:, i] * v[:, j]) for i in range(3) for j in range(i, 3)]
    terms += [np.abs(v[:, i] * v[:, j] * v[:, k]) for i in range(3) for j in range(i, 3)
              for k in range(j, 3)]
    return np.stack([np.bincount(cell, weights=t, minlength=ncell) for t in terms], 1)


def test_coupled_fp32_step_of_the_819k_channel_matches_the_oracle_sub_step_by_sub_step():
    # The benchmarked FP32 coupled hybrid step (the 64 x 256-cell channel, 819,200 particles,
    # 8-node strip): from a coupled state reached by the fused run, the oracle takes the GPU's
    # state before each sub-step (DSMC step, DSMC2LB, LB step, LB2DSMC) and both take it.
    # Integers exact (counts, candidates, collisions, created and deleted particles); particle
    # state bit for bit (floats within 1e-5); the step's FP32 moment partials within 1e-5 of
    # each sum's scale, per element; populations within 1e-5 of w_a rho.
    cfg = W.WORKLOADS["poiseuille_64x256_ppc50_fp32"]
    nodes, cells = W.coupling_sites(cfg)
    dn, dc = torch.from_numpy(nodes).cuda(), torch.from_numpy(cells).cuda()
    h = B.Hybrid(cfg)
    h.hybrid_step(dn, dc, nsteps=3, use_graph=True)
    o = O.Oracle(cfg)
    e, w, r = O.lattice(39)
    # DSMC step
    load_oracle_from_gpu(o, h)
    g0, o0, a0 = h.counters(), o.counters(), h.acc().cpu().numpy().copy()
    h.dsmc_step(1)
    o.dsmc_step(1)
    assert np.array_equal(h.cell_start().cpu().numpy().astype(np.uint32), o.get(O.A_CELL_START))
    assert_particles_match(gpu_particles(h), o.particles(), 4)
    g1, o1 = h.counters(), o.counters()
    for k in ("candidates", "collisions", "wall_hits"):
        assert g1[k] - g0[k] == o1[k] - o0[k], k
    assert np.array_equal(h.crmax().cpu().numpy(), o.get(O.A_CRMAX))
    assert np.array_equal(h.rem().cpu().numpy(), o.get(O.A_REM))
    scale = moment_abs_sums(o.particles(), o.get(O.A_CELL_START))
    inc_g, inc_o = h.acc().cpu().numpy() - a0, o.acc() - a0
    assert np.all(np.abs(inc_g - inc_o) <= 1e-5 * scale + 1e-300), np.abs(inc_g - inc_o).max()
    # DSMC2LB from the same sums
    load_oracle_from_gpu(o, h)
    h.map_dsmc_to_lbm(dn)
    o.map_dsmc_to_lbm(nodes)
    h.sync()
    gf = h.f().cpu().numpy().reshape(39, -1)[:, nodes].astype(np.float64)
    of = o.f().reshape(39, -1)[:, nodes].astype(np.float64)
    assert np.all(np.abs(gf - of) <= 2e-6 * (np.abs(of) + w[:, None]))
    # LB step from the same populations
    load_oracle_from_gpu(o, h)
    h.lbm_step(1)
    o.lbm_step(1)
    h.sync()
    gf, of = h.f().cpu().numpy().astype(np.float64), o.f().astype(np.float64)
    rho = of.sum(0)
    assert (np.abs(gf - of) / (w[:, None, None] * rho)).max() < 1e-5
    # LB2DSMC from the same populations
    load_oracle_from_gpu(o, h)
    g0, o0 = h.counters(), o.counters()
    h.map_lbm_to_dsmc(dc)
    o.map_lbm_to_dsmc(cells)
    assert h.n_tot() == o.scalars()["ntot"]
    assert np.array_equal(h.cell_start().cpu().numpy().astype(np.uint32), o.get(O.A_CELL_START))
    gp, op = gpu_particles(h), o.particles()
    for k in op:
        assert np.array_equal(gp[k], op[k]), k
    g1, o1 = h.counters(), o.counters()
    for k in ("created", "deleted", "l2d_attempts", "envelope"):
        assert g1[k] - g0[k] == o1[k] - o0[k], k
    assert g1["created"] > g0["created"]
    assert h.sync_status()[0] == B.HYB_OK


def _grad_populations():
    """Populations at one node of a Grad distribution with a sizable stress and heat flux:
    DSMC2LB (oracle) of cumulative sums with rho 1.05, u (0.04, 0.08, -0.02), <vv> and <vvv>
    of a non-equilibrium gas."""
    import itertools
    rho, u = 1.05, np.array([0.04, 0.08, -0.02])
    I = np.eye(3)
    P = I + np.outer(u, u) + np.array([[0.12, 0.05, 0.0], [0.05, -0.08, 0.03], [0.0, 0.03, -0.04]])
    Q = (np.einsum("i,jk->ijk", u, I) + np.einsum("j,ik->ijk", u, I) + np.einsum("k,ij->ijk", u, I))
    for perm in set(itertools.permutations((0, 1, 1))):
        Q[perm] += 0.06
    for perm in set(itertools.permutations((0, 0, 0))):
        Q[perm] += 0.05
    S, ppc = 1, 100
    NS = rho * ppc * S
    m = np.zeros(20)
    m[0], m[1:4] = NS, NS * u
    o = 4
    for a in range(3):
        for b in range(a, 3):
            m[o] = NS * P[a, b]
            o += 1
    for a in range(3):
        for b in range(a, 3):
            for c in range(b, 3):
                m[o] = NS * Q[a, b, c]
                o += 1
    return O.dsmc2lb_node(39, m, S, ppc)


def test_lb2dsmc_on_2048_cells_matches_the_oracle_and_the_grad_law():
    # 2048 coupling cells (a strip 4 cells wide across a 512-cell channel, as on the large
    # channel) exceed the mapping's grid of 8 blocks per SM, so every block takes several
    # cells. From the same Grad populations in every strip node: new particles bit for bit
    # as the oracle; the FP64 Grad records equal the oracle's FP64 coefficients to 1e-13; and
    # the regenerated gas has E[c c] = I + a2 and E[c c c] = a3 (Table 1) within 5 sigma of
    # the about 100,000 particles' sample.
    cfg = W.config(ncx=512, ncy=16, ppc=50, lb_ratio=2, kn=0.05, seed=23)
    nodes, cells = W.coupling_sites(cfg)
    assert len(cells) == 2048
    h = B.Hybrid(cfg)
    o = O.Oracle(cfg)
    fnode = _grad_populations()
    f = h.f().cpu().numpy().astype(np.float64).reshape(39, -1)
    f[:, nodes] = fnode[:, None]
    f32 = f.astype(np.float32).reshape(h.f().shape)
    h.f().copy_(torch.from_numpy(f32))
    torch.cuda.synchronize()
    o.set_f(f32)
    dc = torch.from_numpy(cells).cuda()
    h.map_lbm_to_dsmc(dc)
    o.map_lbm_to_dsmc(cells)
    assert h.n_tot() == o.scalars()["ntot"]
    gp, op = gpu_particles(h), o.particles()
    for k in op:
        assert np.array_equal(gp[k], op[k]), k
    hc, oc = h.counters(), o.counters()
    for k in ("created", "deleted", "l2d_attempts", "envelope"):
        assert hc[k] == oc[k], k
    rho_g, nnew_g, v_g = h.grad_records(len(cells))
    g = O.grad_coeffs_packed(39, f32.reshape(39, -1)[:, nodes[0]].astype(np.float64), 8)
    want = np.concatenate([g["a2"], g["a3"], g["u"], [g["C"]]])
    assert np.abs(v_g.numpy() - want[None, :]).max() < 1e-13
    assert np.abs(rho_g.numpy() / g["rho"] - 1).max() < 1e-14
    # the regenerated velocities follow the Grad distribution of those coefficients
    cs = h.cell_start().cpu().numpy().astype(np.int64)
    sel = np.concatenate([np.arange(cs[c], cs[c + 1]) for c in cells])
    v = np.stack([gp["vx"][sel], gp["vy"][sel], gp["vz"][sel]], 1).astype(np.float64)
    c = v - g["u"]
    n = len(c)
    assert n > 90_000
    se = 1 / np.sqrt(n)
    pairs = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]
    for k, (i, j) in enumerate(pairs):
        m2 = (c[:, i] * c[:, j]).mean()
        assert abs(m2 - ((1.0 if i == j else 0.0) + g["a2"][k])) < 5 * np.sqrt(3) * se, (i, j)
    triples = [(0, 0, 0), (0, 0, 1), (0, 0, 2), (0, 1, 1), (0, 1, 2), (0, 2, 2), (1, 1, 1),
               (1, 1, 2), (1, 2, 2), (2, 2, 2)]
    for k, (i, j, l) in enumerate(triples):
        m3 = (c[:, i] * c[:, j] * c[:, l]).mean()
        assert abs(m3 - g["a3"][k]) < 5 * np.sqrt(15) * se, (i, j, l)
