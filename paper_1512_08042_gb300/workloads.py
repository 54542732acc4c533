"""Synthetic workloads and seeded input generators.

The paper measures force-driven plane Poiseuille channels of an Argon-like hard-sphere gas
(Sec. 3.1: T = 273 K, m = 6.63e-26 kg, Ma = 0.1 on the centreline velocity; 100 particles
per cell initially) and publishes no dataset, so every input here is synthetic: a parameter
set plus a seed. This module holds no arithmetic of the method; it only builds parameter
dictionaries, coupling index lists and seeded random arrays that the CUDA library and the
CPU oracle both take as inputs.
"""
import numpy as np

ARGON = dict(T_K=273.0, mass_kg=6.63e-26)

_BASE = dict(lb_ratio=1, lattice=39, real_bytes=4, sample_every=1, kn=0.1, ma=0.1,
             crmax_init=6.0, capacity_factor=2.5, **ARGON)


def config(**kw):
    cfg = dict(_BASE)
    cfg.update(kw)
    return cfg


# Named workloads. Across-channel cells (walls) = ncx, streamwise periodic cells = ncy.
WORKLOADS = {
    # Plain hybrid, 64 cells across x 1 periodic cell, 100 particles/cell, Kn 0.1, FP64,
    # 64-node D3Q39 lattice, mapping at 2 coupling nodes (i = 1 and i = H - 2).
    "poiseuille_64x1_ppc100_fp64": config(ncx=64, ncy=1, ppc=100, real_bytes=8, kn=0.1, seed=1),
    # 2D channel: 64 x 256 DSMC cells, 50 particles/cell (819,200), Kn 0.05, FP32 state,
    # 128 x 512 D3Q39 lattice (two LB nodes per cell per axis), 8-node coupling strip.
    "poiseuille_64x256_ppc50_fp32": config(ncx=64, ncy=256, ppc=50, lb_ratio=2, kn=0.05, seed=2),
    # Mid-size channel for profiling many-wave behaviour on a small device footprint:
    # 128 x 1024 DSMC cells, 50 particles/cell (6,553,600), 256 x 2048 D3Q39 lattice.
    "poiseuille_128x1024_ppc50_fp32": config(ncx=128, ncy=1024, ppc=50, lb_ratio=2, kn=0.05,
                                              seed=7),
    # Large channel: 512 x 4096 DSMC cells, 50 particles/cell (104,857,600), FP32 state,
    # 1024 x 8192 D3Q39 lattice.
    "poiseuille_512x4096_ppc50_fp32": config(ncx=512, ncy=4096, ppc=50, lb_ratio=2, kn=0.05,
                                              seed=5),
    # The large channel with Kn varying along it, log-linear from 0.005 (y = 0) to 0.5
    # (y = L/2) and back: per-cell NTC factors and per-node relaxation times.
    "poiseuille_512x4096_ppc50_knvar_fp32": config(ncx=512, ncy=4096, ppc=50, lb_ratio=2,
                                                    kn=0.005, kn_profile=1, kn_end=0.5, seed=6),
    # Full 3D channel: 64 x 256 x 8 DSMC cells (periodic y and z, Sec. 3.1), 50 per cell
    # (6,553,600), FP32 state, 128 x 512 x 16 D3Q39 lattice, the 4-cell coupling strip in
    # every layer.
    "poiseuille3d_64x256x8_ppc50_fp32": config(ncx=64, ncy=256, ncz=8, ppc=50, lb_ratio=2,
                                                kn=0.05, seed=8),
    # The proof-of-concept hybrid of Sec. 4: plane Poiseuille at Kn 0.05 and Ma 0.1, D3Q19
    # without regularisation, DSMC2LB to the local equilibrium of rho and u (Eq. feq_dsmc)
    # on a buffer layer one cell long at y = L0/2 across the whole height, DSMC solved on its
    # own (no LB2DSMC). The channel sizes are not printed: 64 x 64 cells, 50 per cell, FP64.
    "poc_hybrid_64x64_d3q19_fp64": config(ncx=64, ncy=64, ppc=50, lattice=19, lb_ratio=1,
                                           kn=0.05, ma=0.1, real_bytes=8, lb_collision=1,
                                           d2l_mode=1, coupling="buffer_row", seed=4),
}


# The differentiated LBM: a 256 x 128 D3Q39 lattice (128 x 64 DSMC cells at two LB nodes per
# cell per axis), FP32, differentiated through 2000 steps with checkpoints every 100.
DIFF_LBM = config(ncx=128, ncy=64, ppc=10, lb_ratio=2, kn=0.1, ma=0.1, seed=9)
DIFF_LBM_STEPS, DIFF_LBM_CKPT = 2000, 100


def diff_lbm_inputs(cfg, weights, seed=9, spread_g=0.1, spread_tau=0.02):
    """Seeded populations around rest, per-node force increments and relaxation times around
    the channel's scalars, coupling nodes on an 8-node-wide strip (x = 8..15, every y) and
    targets (rho 1, u_y 0.05, other coefficients 0) for the differentiated LBM."""
    nx, ny = cfg["ncx"] * cfg["lb_ratio"], cfg["ncy"] * cfg["lb_ratio"]
    n = nx * ny
    rng = np.random.default_rng(seed)
    f0 = gen_populations(weights, n, seed=seed + 100)
    g = rng.standard_normal(n)
    tau = rng.standard_normal(n)
    nodes = np.array([y * nx + x for y in range(ny) for x in range(8, 16)], np.int32)
    targets = np.zeros((len(nodes), 20))
    targets[:, 0] = 1.0
    targets[:, 2] = 0.05
    return f0, spread_g * g, spread_tau * tau, nodes, targets


def grad_targets_from_sums(acc, nsamples, ppc, cells):
    """Interface-loss targets sampled from a DSMC gas: for each listed cell, the 20 Grad
    coefficients of its particles from the cumulative sums acc[cell] = (N, S v, S vv, S vvv)
    over `nsamples` samples: rho = N / (S ppc), the mean velocity u, the comoving second
    moments minus the identity (xx xy xz yy yz zz) and the comoving third moments (xxx xxy xxz
    xyy xyz xzz yyy yyz yzz zzz), in thermal units like the populations' coefficients."""
    a = np.asarray(acc, np.float64)[np.asarray(cells)]
    n = a[:, 0]
    u = a[:, 1:4] / n[:, None]
    m2 = a[:, 4:10] / n[:, None]
    m3 = a[:, 10:20] / n[:, None]
    pairs = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]
    triples = [(0, 0, 0), (0, 0, 1), (0, 0, 2), (0, 1, 1), (0, 1, 2), (0, 2, 2), (1, 1, 1),
               (1, 1, 2), (1, 2, 2), (2, 2, 2)]
    p2 = {ij: k for k, ij in enumerate(pairs)}
    raw2 = lambda i, j: m2[:, p2[(min(i, j), max(i, j))]]
    out = np.zeros((len(a), 20))
    out[:, 0] = n / (nsamples * ppc)
    out[:, 1:4] = u
    for k, (i, j) in enumerate(pairs):
        out[:, 4 + k] = raw2(i, j) - u[:, i] * u[:, j] - (1.0 if i == j else 0.0)
    for k, (i, j, l) in enumerate(triples):
        out[:, 10 + k] = (m3[:, k] - u[:, i] * raw2(j, l) - u[:, j] * raw2(i, l) - u[:, l] * raw2(i, j)
                          + 2.0 * u[:, i] * u[:, j] * u[:, l])
    return out


def ensemble_configs(n=64, seed=1000, rank=0):
    """The batched ensemble: n independent channels of the 64 x 1 geometry (walls across,
    one periodic cell), H uniform in 32..256 cells, 20..100 particles per cell, Kn
    log-uniform in [0.01, 0.5], one LB node per cell, FP32 state, seeds seed + k. Rank r of a
    multi-GPU ensemble runs the same n channels with the Philox seeds seed + k + r * 2^20, so
    that channel k of every rank is one more sample of the same flow."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        out.append(config(ncx=int(rng.integers(32, 257)), ncy=1, ppc=int(rng.integers(20, 101)),
                          kn=float(np.exp(rng.uniform(np.log(0.01), np.log(0.5)))), lb_ratio=1,
                          seed=seed + k + (rank << 20)))
    return out


def coupling_sites(cfg, strip_cells=None):
    """Coupling nodes and cells.

    With ncy == 1 (the channel of Sec. 3.2/3.3) the sites are the first fluid node/cell next
    to each wall (i = 1 and i = H - 2). Otherwise a strip `strip_cells` DSMC cells wide
    (default 4, i.e. 8 LB nodes at two nodes per cell) across the whole channel height, in
    the middle of the streamwise period, as the one-cell buffer layer of Sec. 4 widened.
    Returns (nodes, cells) as int32 arrays; node = y * nx + x, cell = iy * ncx + ix. In 3D
    (ncz >= 2) the same sites in every layer: node (z ny + y) nx + x, cell (iz ncy + iy) ncx + ix.
    """
    nodes, cells = _coupling_sites_2d(cfg, strip_cells)
    ncz = cfg.get("ncz", 0)
    if ncz >= 2:
        r = cfg["lb_ratio"]
        nn2, nc2 = cfg["ncx"] * cfg["ncy"] * r * r, cfg["ncx"] * cfg["ncy"]
        nodes = (np.arange(ncz * r, dtype=np.int64)[:, None] * nn2 + nodes[None, :]).reshape(-1)
        cells = (np.arange(ncz, dtype=np.int64)[:, None] * nc2 + cells[None, :]).reshape(-1)
    return nodes.astype(np.int32), cells.astype(np.int32)


def _coupling_sites_2d(cfg, strip_cells):
    ncx, ncy, r = cfg["ncx"], cfg["ncy"], cfg["lb_ratio"]
    nx = ncx * r
    if cfg.get("coupling") == "buffer_row":
        # the buffer layer of Sec. 4: the LB nodes of the cell row at y = L0/2, DSMC2LB only
        y0 = (ncy // 2) * r
        nodes = np.array([y * nx + x for y in range(y0, y0 + r) for x in range(nx)], np.int32)
        return nodes, np.zeros(0, np.int32)
    if ncy == 1:
        cells = np.array([1, ncx - 2], np.int32)
        nodes = []
        for c in cells:
            for dy in range(r):
                for dx in range(r):
                    nodes.append(dy * nx + c * r + dx)
        return np.array(nodes, np.int32), cells
    w = strip_cells if strip_cells is not None else 4
    y0 = ncy // 2 - w // 2
    cells = np.array([iy * ncx + ix for iy in range(y0, y0 + w) for ix in range(ncx)], np.int32)
    nodes = np.array([y * nx + x for y in range(y0 * r, (y0 + w) * r) for x in range(nx)],
                     np.int32)
    return nodes, cells


def gen_populations(weights, nnodes, seed, eps=0.05, rho_eps=0.02):
    """Populations f[a, node] = w_a * rho_node * (1 + eps * U(-1, 1)), rho_node = 1 + rho_eps * U(-1,1)."""
    rng = np.random.default_rng(seed)
    w = np.asarray(weights, np.float64)[:, None]
    rho = 1.0 + rho_eps * rng.uniform(-1, 1, size=(1, nnodes))
    return w * rho * (1.0 + eps * rng.uniform(-1, 1, size=(len(weights), nnodes)))


def gen_particles(ncx, ncy, mean_ppc, seed, empty_fraction=0.0, vel_scale=1.0, drift=(0, 0, 0)):
    """A cell-ordered particle set: per-cell counts ~ Poisson(mean_ppc) (a fraction of cells
    forced empty), positions uniform inside their cell, Gaussian velocities.

    Returns dict of float64 arrays x, y, vx, vy, vz and uint32 cell_start (ncells + 1).
    """
    rng = np.random.default_rng(seed)
    ncells = ncx * ncy
    counts = rng.poisson(mean_ppc, size=ncells)
    if empty_fraction > 0:
        counts[rng.random(ncells) < empty_fraction] = 0
    cell = np.repeat(np.arange(ncells), counts)
    n = cell.size
    ix, iy = cell % ncx, cell // ncx
    out = {
        "x": ix + rng.random(n),
        "y": iy + rng.random(n),
        "vx": drift[0] + vel_scale * rng.standard_normal(n),
        "vy": drift[1] + vel_scale * rng.standard_normal(n),
        "vz": drift[2] + vel_scale * rng.standard_normal(n),
    }
    # keep positions strictly inside their cell after any rounding to float
    out["x"] = np.minimum(out["x"], ix + 0.999)
    out["y"] = np.minimum(out["y"], iy + 0.999)
    cs = np.zeros(ncells + 1, np.uint32)
    cs[1:] = np.cumsum(counts)
    out["cell_start"] = cs
    return out


def slab_config(cfg, rank, world):
    """Rank r of the streamwise decomposition of a channel world times as long as cfg's: the
    rows [r ncy, (r + 1) ncy) of a channel of world * ncy rows (each rank keeps cfg's rows:
    the work per GPU is fixed as ranks are added)."""
    out = dict(cfg)
    out["ncy_global"] = int(world) * int(cfg["ncy"])
    out["y0"] = int(rank) * int(cfg["ncy"])
    return out


def slab_sites(whole_cfg, slab_cfg, yh, nodes, cells):
    """The slab's own node and cell indices of the whole channel's coupling lists (node
    (z ny + y) nx + x and cell (iz ncy + iy) ncx + ix of the whole channel; the slab's lattice
    has yh ghost rows below its rows)."""
    ncx, ncy, r = whole_cfg["ncx"], whole_cfg["ncy"], whole_cfg["lb_ratio"]
    nly, y0 = slab_cfg["ncy"], slab_cfg["y0"]
    nx, ny_w, ny_s = ncx * r, ncy * r, nly * r + 2 * yh
    nodes = np.asarray(nodes, np.int64)
    cells = np.asarray(cells, np.int64)
    z, rem = nodes // (nx * ny_w), nodes % (nx * ny_w)
    y, x = rem // nx, rem % nx
    keep = (y >= y0 * r) & (y < (y0 + nly) * r)
    ln = ((z * ny_s + (y - y0 * r + yh)) * nx + x)[keep]
    cz, crem = cells // (ncx * ncy), cells % (ncx * ncy)
    cy, cx = crem // ncx, crem % ncx
    keepc = (cy >= y0) & (cy < y0 + nly)
    lc = ((cz * nly + (cy - y0)) * ncx + cx)[keepc]
    return ln.astype(np.int32), lc.astype(np.int32)
