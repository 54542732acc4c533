"""The differentiated LBM through the C ABI: the LB step with per-node force increment and
relaxation time against the oracle, the coupling-interface loss against the oracle, and the
adjoint gradient (checkpointed recomputation) against the oracle's central differences and
against directional differences of the GPU forward."""
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


def cfg_lb(**kw):
    base = dict(ncx=6, ncy=4, ppc=10, lb_ratio=2, real_bytes=8, seed=3, kn=0.3, ma=0.5)
    base.update(kw)
    return W.config(**base)


def setup(cfg, seed=1, spread_g=0.3, spread_tau=0.1):
    """A context, seeded populations and per-node parameters around the scalars."""
    h = B.Hybrid(cfg)
    d = h.d
    n = d["nnodes"]
    e, w, r = O.lattice(cfg.get("lattice", 39))
    rng = np.random.default_rng(seed)
    f0 = W.gen_populations(w, n, seed=seed + 100)
    g = d["g_step"] * (1 + spread_g * rng.standard_normal(n))
    tau = d["tau"] * (1 + spread_tau * rng.standard_normal(n))
    real = np.float32 if cfg["real_bytes"] == 4 else np.float64
    f0, g, tau = f0.astype(real), g.astype(real), tau.astype(real)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return h, dev(f0.reshape(h.d["q"], h.d["ny"], h.d["nx"])), dev(g), dev(tau), f0, g, tau


def oracle_after(cfg, f0, g, tau, nsteps):
    o = O.Oracle(cfg)
    o.set_f(f0.astype(np.float32 if cfg["real_bytes"] == 4 else np.float64))
    o.set_node_params(g.astype(np.float64), tau.astype(np.float64))
    o.lbm_step(nsteps)
    return o


def gpu_after(h, f, g, tau, nsteps):
    a, b = f.clone(), torch.empty_like(f)
    for _ in range(nsteps):
        h.lbm_step_nodes(a, b, g, tau)
        a, b = b, a
    h.sync()
    return a


@pytest.mark.parametrize("lattice,real_bytes", [(39, 8), (39, 4), (19, 4)])
def test_lbm_step_nodes_matches_oracle(lattice, real_bytes):
    cfg = cfg_lb(lattice=lattice, real_bytes=real_bytes)
    h, f, g, tau, f0, gn, tn = setup(cfg)
    e, w, r = O.lattice(lattice)
    o = O.Oracle(cfg)
    o.set_f(f0)
    o.set_node_params(gn.astype(np.float64), tn.astype(np.float64))
    a, b = f.clone(), torch.empty_like(f)
    for step in range(3):
        h.lbm_step_nodes(a, b, g, tau)
        a, b = b, a
        o.lbm_step(1)
        h.sync()
        err = lb_err(a.cpu().numpy(), o.f(), w)
        assert err < (LB_TOL_FP32 if real_bytes == 4 else LB_TOL_FP64), (step, err)
    # the context's own populations were not touched
    assert torch.equal(h.f(), torch.from_numpy(np.tile(w[:, None], (1, h.d["nnodes"])).astype(
        f0.dtype).reshape(h.f().shape)).cuda())


@pytest.mark.parametrize("real_bytes", [8, 4])
def test_interface_loss_matches_oracle(real_bytes):
    cfg = cfg_lb(real_bytes=real_bytes)
    h, f, g, tau, f0, gn, tn = setup(cfg, seed=2)
    nodes_np = np.array([5, 17, 30, 30, 77], np.int32)  # a repeated node counts twice
    o = oracle_after(cfg, f0, gn, tn, 2)
    rng = np.random.default_rng(3)
    targets_np = np.stack([o.grad_node(k) for k in nodes_np]) + 0.02 * rng.standard_normal((5, 20))
    want = o.interface_loss(nodes_np, targets_np)
    fT = gpu_after(h, f, g, tau, 2)
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    lam = torch.zeros_like(fT)
    h.lbm_interface_loss(fT, torch.from_numpy(nodes_np).cuda(), torch.from_numpy(
        targets_np.astype(fT.cpu().numpy().dtype)).cuda(), loss, lam)
    h.sync()
    assert loss.item() == pytest.approx(want, rel=1e-10 if real_bytes == 8 else 2e-4)
    # lam is non-zero only at the listed nodes
    nz = (lam.reshape(lam.shape[0], -1) != 0).any(0).nonzero().flatten().cpu().numpy()
    assert set(nz) <= set(nodes_np.tolist())


def gpu_gradient(cfg, h, f, g, tau, nodes, targets, nsteps, ckpt):
    g = g.clone().requires_grad_(True)
    tau = tau.clone().requires_grad_(True)
    f0 = f.clone().requires_grad_(True)
    L = B.interface_loss(h, g, tau, f0, nodes, targets, nsteps, ckpt)
    L.backward()
    torch.cuda.synchronize()
    return L.item(), g.grad.cpu().numpy(), tau.grad.cpu().numpy(), f0.grad


@pytest.mark.parametrize("lattice,real_bytes,tol", [(39, 8, 1e-6), (19, 8, 1e-6), (39, 4, 2e-3)])
def test_adjoint_gradient_matches_oracle_central_differences(lattice, real_bytes, tol):
    cfg = cfg_lb(lattice=lattice, real_bytes=real_bytes)
    h, f, g, tau, f0, gn, tn = setup(cfg, seed=4)
    T, K = 5, 2  # three checkpoint segments
    nodes_np = np.array([2 * h.d["nx"] + 1, 5 * h.d["nx"] + 6, 6 * h.d["nx"] + 11], np.int32)
    o = oracle_after(cfg, f0, gn, tn, T)
    rng = np.random.default_rng(5)
    targets_np = np.stack([o.grad_node(k) for k in nodes_np]) + 0.02 * rng.standard_normal((3, 20))
    loss, dg, dt, _ = gpu_gradient(cfg, h, f, g, tau, torch.from_numpy(nodes_np).cuda(),
                                   torch.from_numpy(targets_np.astype(f0.dtype)).cuda(), T, K)
    cfg64 = dict(cfg, real_bytes=8)
    want_g, want_t = O.interface_loss_fd_gradient(cfg64, f0.astype(np.float64), gn, tn, nodes_np,
                                                  targets_np, T)
    assert loss == pytest.approx(O.interface_loss_after(cfg64, f0.astype(np.float64), gn, tn,
                                                        nodes_np, targets_np, T),
                                 rel=1e-10 if real_bytes == 8 else 1e-3)
    for got, want in ((dg, want_g), (dt, want_t)):
        scale = np.abs(want).max()
        assert scale > 0
        assert np.abs(got - want).max() < tol * scale, np.abs(got - want).max() / scale


def test_adjoint_gradient_is_exactly_zero_outside_the_light_cone():
    cfg = cfg_lb(ncx=6, ncy=10)  # 12 x 20 nodes
    h, f, g, tau, f0, gn, tn = setup(cfg, seed=6)
    nx = h.d["nx"]
    node = 10 * nx + 3
    T = 2
    o = oracle_after(cfg, f0, gn, tn, T)
    targets = o.grad_node(node)[None, :] + 0.01
    _, dg, dt, _ = gpu_gradient(cfg, h, f, g, tau, torch.tensor([node], dtype=torch.int32,
                                device="cuda"), torch.from_numpy(targets).cuda(), T, 1)
    rows = np.arange(h.d["nnodes"]) // nx
    far = np.minimum(np.abs(rows - 10), h.d["ny"] - np.abs(rows - 10)) > 3 * T
    assert np.all(dg[far] == 0) and np.all(dt[far] == 0)
    assert dg[node] != 0 and dt[node] != 0


def test_adjoint_populations_gradient_matches_directional_differences():
    # dL/df0 is the adjoint carried back through every step (streaming transposes and wall
    # densities included); its projection on a random direction must match the central
    # difference of the GPU forward in FP64.
    cfg = cfg_lb()
    h, f, g, tau, f0, gn, tn = setup(cfg, seed=7)
    T = 4
    nodes = torch.tensor([1, h.d["nx"] * 3 + 11, h.d["nx"] * 5 + 4], dtype=torch.int32, device="cuda")
    o = oracle_after(cfg, f0, gn, tn, T)
    targets = torch.from_numpy(np.stack([o.grad_node(int(k)) for k in nodes.cpu()]) + 0.03).cuda()
    _, _, _, gf = gpu_gradient(cfg, h, f, g, tau, nodes, targets, T, 3)
    # a seeded direction, and a step that keeps the difference of the two losses (about 0.05
    # each) well above their FP64 rounding: at eps = 1e-5 (a relative perturbation of 1e-7)
    # that rounding alone was about 1e-7 of the difference and the whole check sat at 1e-6;
    # the truncation error of the central difference is O(eps^2)
    gen = torch.Generator(device="cuda").manual_seed(11)
    v = torch.randn(f.shape, generator=gen, device="cuda", dtype=f.dtype) * 1e-2 * f
    eps = 1e-3

    def loss_at(ff):
        fT = gpu_after(h, ff, g, tau, T)
        L = torch.zeros(1, dtype=torch.float64, device="cuda")
        h.lbm_interface_loss(fT, nodes, targets, L, torch.zeros_like(fT))
        h.sync()
        return L.item()

    fd = (loss_at(f + eps * v) - loss_at(f - eps * v)) / (2 * eps)
    assert (gf * v).sum().item() == pytest.approx(fd, rel=1e-6)


def test_adjoint_at_the_differentiated_lbm_size_256x128_2000_steps():
    # The differentiated configuration: 256 x 128 lattice, 2000 steps, checkpoints every 100,
    # FP32. Checked by properties that hold at any size: a finite gradient, zero outside the
    # rows the loss can reach (none here: 2000 steps cover the channel), and agreement of the
    # FP32 directional derivative in g with central differences of an FP64 run.
    cfg = W.config(ncx=128, ncy=64, ppc=10, lb_ratio=2, real_bytes=4, seed=9, kn=0.1, ma=0.1)
    h, f, g, tau, f0, gn, tn = setup(cfg, seed=9, spread_g=0.1, spread_tau=0.02)
    assert (h.d["nx"], h.d["ny"]) == (256, 128)
    nx = h.d["nx"]
    nodes_np = np.array([y * nx + x for y in range(0, 128, 16) for x in (8, 9, 10, 11)], np.int32)
    nodes = torch.from_numpy(nodes_np).cuda()
    rng = np.random.default_rng(10)
    targets_np = np.zeros((len(nodes_np), 20))
    targets_np[:, 0] = 1.0
    targets_np[:, 2] = 0.05 + 0.01 * rng.standard_normal(len(nodes_np))
    targets = torch.from_numpy(targets_np.astype(np.float32)).cuda()
    loss, dg, dt, _ = gpu_gradient(cfg, h, f, g, tau, nodes, targets, 2000, 100)
    assert np.isfinite(loss) and np.all(np.isfinite(dg)) and np.all(np.isfinite(dt))
    # FP64 directional check along a random perturbation of g
    cfg64 = dict(cfg, real_bytes=8)
    h64 = B.Hybrid(cfg64)
    f64, g64, t64 = (torch.from_numpy(a.astype(np.float64)).cuda() for a in (f0, gn, tn))
    f64 = f64.reshape(h64.d["q"], h64.d["ny"], h64.d["nx"])
    _, dg64, _, _ = gpu_gradient(cfg64, h64, f64, g64, t64, nodes, targets.double(), 2000, 100)
    dirv = torch.from_numpy(rng.standard_normal(h.d["nnodes"])).cuda() * float(np.abs(gn).mean()) * 1e-3

    def loss64(gg):
        fT = gpu_after(h64, f64, gg, t64, 2000)
        L = torch.zeros(1, dtype=torch.float64, device="cuda")
        h64.lbm_interface_loss(fT, nodes, targets.double(), L, torch.zeros_like(fT))
        h64.sync()
        return L.item()

    fd = (loss64(g64 + dirv) - loss64(g64 - dirv)) / 2.0
    got64 = float((torch.from_numpy(dg64).cuda() * dirv).sum())
    got32 = float((torch.from_numpy(dg).cuda().double() * dirv).sum())
    assert got64 == pytest.approx(fd, rel=1e-5)
    assert got32 == pytest.approx(fd, rel=2e-2)


# ---------------------------------------------------------------------------------------
# The differentiated coupling: DSMC2LB of the cumulative sums, LB steps, interface loss

def coupled_inputs(cfg, seed=4):
    """Sums from a few oracle DSMC steps of the same channel, the mapped nodes (the cells of
    column ix = 1, every row), and loss nodes two columns further on."""
    src = O.Oracle(dict(cfg, ma=0.4))
    src.dsmc_step(5)
    acc, S = src.acc().copy(), src.scalars()["nsamples"]
    nx, ny = cfg["ncx"] * cfg["lb_ratio"], cfg["ncy"] * cfg["lb_ratio"]
    d2l = np.array([y * nx + x for y in range(ny) for x in (2, 3)], np.int32)
    nodes = np.array([y * nx + x for y in range(ny) for x in (5, 6)], np.int32)
    rng = np.random.default_rng(seed)
    targets = np.zeros((len(nodes), 20))
    targets[:, 0] = 1.0
    targets[:, 2] = 0.05
    targets[:, 4:] = 0.01 * rng.standard_normal((len(nodes), 16))
    return acc, S, d2l, nodes, targets


@pytest.mark.parametrize("lattice", [39, 19])
def test_coupled_gradient_matches_oracle_central_differences(lattice):
    cfg = cfg_lb(lattice=lattice, real_bytes=8)
    h, f, g, tau, f0, gn, tn = setup(cfg, seed=2)
    acc, S, d2l, nodes, targets = coupled_inputs(cfg)
    T = 3
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    acc_t = dev(acc).requires_grad_(True)
    f_t = f.clone().requires_grad_(True)
    g_t = g.clone().requires_grad_(True)
    loss = B.coupled_interface_loss(h, acc_t, S, dev(d2l), g_t, tau, f_t, dev(nodes),
                                    dev(targets), T, ckpt_every=2)
    loss.backward()
    want_loss = O.coupled_loss_after(cfg, acc, S, d2l, f0, gn, tn, nodes, targets, T)
    assert float(loss.detach()) == pytest.approx(want_loss, rel=1e-10)
    grad = acc_t.grad.cpu().numpy()
    # sums of the mapped cells (column ix = 1) and of an unmapped cell (ix = 4)
    ks = [0, 1, 2, 3, 4, 5, 7, 9, 10, 13, 14, 16, 19]
    entries = [(iy * 6 + 1, k) for iy in (0, 2, 3) for k in ks] + [(2 * 6 + 4, 0), (2 * 6 + 4, 4)]
    want = O.coupled_loss_fd_gradient(cfg, acc, S, d2l, f0, gn, tn, nodes, targets, T, entries)
    got = np.array([grad[c, k] for c, k in entries])
    scale = np.abs(want).max()
    assert scale > 0
    assert np.abs(got - want).max() < 1e-6 * scale, np.abs(got - want).max() / scale
    assert np.all(grad[[iy * 6 + ix for iy in range(4) for ix in (0, 2, 3, 4, 5)]] == 0)
    if lattice == 19:  # the second-order mapping has no third-order coefficients
        assert np.all(grad[:, 10:] == 0)
    # the mapped nodes' populations were overwritten: no gradient reaches them
    gf = f_t.grad.cpu().numpy().reshape(h.d["q"], -1)
    assert np.all(gf[:, d2l] == 0) and np.abs(gf).max() > 0
    assert np.abs(g_t.grad.cpu().numpy()).max() > 0


def test_coupled_gradient_fp32_close_to_fp64():
    grads = []
    for rb in (8, 4):
        cfg = cfg_lb(real_bytes=rb)
        h, f, g, tau, f0, gn, tn = setup(cfg, seed=5)
        acc, S, d2l, nodes, targets = coupled_inputs(cfg)
        real = torch.float32 if rb == 4 else torch.float64
        acc_t = torch.from_numpy(acc).cuda().requires_grad_(True)
        loss = B.coupled_interface_loss(h, acc_t, S, torch.from_numpy(d2l).cuda(), g, tau, f,
                                        torch.from_numpy(nodes).cuda(),
                                        torch.from_numpy(targets).to(real).cuda(), 4, 2)
        loss.backward()
        grads.append(acc_t.grad.cpu().numpy())
    scale = np.abs(grads[0]).max()
    assert scale > 0 and np.abs(grads[1] - grads[0]).max() < 2e-3 * scale


def test_dsmc2lb_adjoint_rejects_the_equilibrium_mapping():
    cfg = cfg_lb(d2l_mode=1)
    h = B.Hybrid(cfg)
    lam = torch.zeros_like(h.f())
    grad = torch.zeros(int(h.L.ncells), 20, dtype=torch.float64, device="cuda")
    with pytest.raises(B.HybError) as ei:
        h.map_dsmc_to_lbm_adjoint(torch.tensor([0, 1], dtype=torch.int32, device="cuda"), lam, grad)
    assert ei.value.status == B.HYB_EINVAL


@pytest.mark.parametrize("real_bytes", [8, 4])
def test_one_call_forward_and_adjoint_segment_equal_the_step_calls(real_bytes):
    # lbm_steps_nodes (7 steps, a checkpoint every 3) and lbm_adjoint_segment (4 and 1 steps)
    # compute what the same lbm_step_nodes and lbm_adjoint_step calls compute: the forward bit
    # for bit; the adjoint up to the order of the wall rows' atomic sums (the populations
    # leaving through a wall take their row's sum, added by several nodes in any order)
    cfg = cfg_lb(real_bytes=real_bytes)
    h, f, g, tau, *_ = setup(cfg, seed=8)
    T, K = 7, 3
    a, b = f.clone(), torch.empty_like(f)
    ck = torch.empty((2,) + tuple(f.shape), dtype=f.dtype, device=f.device)
    fT = h.lbm_steps_nodes(a, b, g, tau, T, K, ck)
    ref, states = f.clone(), [f.clone()]
    for _ in range(T):
        nxt = torch.empty_like(ref)
        h.lbm_step_nodes(ref, nxt, g, tau)
        ref = nxt
        states.append(ref)
    h.sync()
    assert torch.equal(fT, ref)
    assert torch.equal(ck[0], states[3]) and torch.equal(ck[1], states[6])
    rng = np.random.default_rng(5)
    lam_T = torch.from_numpy(rng.standard_normal(tuple(f.shape)).astype(
        np.float32 if real_bytes == 4 else np.float64)).cuda()
    wall = torch.zeros(h.wall_scratch_size(), dtype=f.dtype, device=f.device)
    for n in (4, 1):
        gg1, gt1 = torch.zeros_like(g), torch.zeros_like(tau)
        la, lb = lam_T.clone(), torch.empty_like(lam_T)
        scratch = torch.empty((3,) + tuple(f.shape), dtype=f.dtype, device=f.device)
        out = h.lbm_adjoint_segment(states[2], scratch if n > 1 else None, n, la, lb, g, tau, gg1, gt1,
                                    wall)
        gg2, gt2 = torch.zeros_like(g), torch.zeros_like(tau)
        nxt, cur = lam_T.clone(), torch.empty_like(lam_T)
        for t in reversed(range(2, 2 + n)):
            h.lbm_adjoint_step(states[t], nxt, cur, g, tau, gg2, gt2, wall)
            nxt, cur = cur, nxt
        h.sync()
        tol = 1e-12 if real_bytes == 8 else 1e-5
        for u, v in ((out, nxt), (gg1, gg2), (gt1, gt2)):
            assert float((u - v).abs().max()) <= tol * float(v.abs().max()), n
        assert torch.count_nonzero(wall) == 0


def test_gradient_of_zero_steps_is_the_loss_adjoint_at_f0():
    # T = 0: the loss is taken at f0 itself, so dL/dg = dL/dtau = 0 and dL/df0 is the loss's own
    # adjoint (lbm_interface_loss)
    cfg = cfg_lb()
    h, f, g, tau, *_ = setup(cfg, seed=9)
    nodes = torch.tensor([h.d["nx"] + 2, 3 * h.d["nx"] + 5], dtype=torch.int32, device="cuda")
    targets = torch.full((2, 20), 0.01, dtype=f.dtype, device="cuda")
    loss, dg, dt, df = gpu_gradient(cfg, h, f, g, tau, nodes, targets, 0, 4)
    want_loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    lam = torch.zeros_like(f)
    h.lbm_interface_loss(f, nodes, targets, want_loss, lam)
    h.sync()
    assert loss == want_loss.item()
    assert np.all(dg == 0) and np.all(dt == 0)
    assert torch.equal(df, lam)
