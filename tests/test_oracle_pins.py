"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: published known-answer
vectors, closed forms, exact quadrature identities, conservation laws, textbook special cases
and statistical laws with confidence intervals. No GPU is used.
"""
import itertools
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_1512_08042_gb300 import workloads as W
from conftest import read_golden_numbers


def small_cfg(**kw):
    base = dict(ncx=16, ncy=4, ppc=40, real_bytes=8, seed=7, kn=0.1)
    base.update(kw)
    return W.config(**base)


# ---------------------------------------------------------------------------------------
# Philox4x32-10 (Salmon et al., SC'11)

def test_philox_known_answers(golden_dir):
    rows = []
    with open(os.path.join(golden_dir, "philox4x32_10_kat.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                rows.append([int(t, 16) for t in line.split()])
    assert len(rows) == 3
    for r in rows:
        ctr, key, want = r[0:4], r[4:6], r[6:10]
        got = O.philox(ctr, key[0] | (key[1] << 32))[0]
        assert [int(v) for v in got] == want


def test_philox_uniformity_chi2():
    n = 1 << 18
    ctr = np.zeros((n // 4, 4), np.uint32)
    ctr[:, 0] = np.arange(n // 4)
    words = O.philox(ctr, 12345).reshape(-1)
    u = (words >> 8).astype(np.float64) * 2.0 ** -24
    hist, _ = np.histogram(u, bins=64, range=(0, 1))
    e = n / 64
    chi2 = ((hist - e) ** 2 / e).sum()
    # 63 dof: mean 63, sd 11.2; 99.99% upper tail ~ 110
    assert chi2 < 110


# ---------------------------------------------------------------------------------------
# Gauss-Hermite lattices (Sec. 1, Sec. 3.1: D3Q39 has sixth-order isotropy; the quadrature
# must be exact to degree >= 2N, Sec. 2.1)

def gaussian_moment(alpha):
    m = 1.0
    for a in alpha:
        if a % 2:
            return 0.0
        m *= math.prod(range(a - 1, 0, -2)) if a > 0 else 1.0
    return m


def quadrature_max_exact_degree(q):
    e, w, r = O.lattice(q)
    xi = e * r
    deg = 0
    for n in range(0, 10):
        ok = True
        for alpha in itertools.product(range(n + 1), repeat=3):
            if sum(alpha) != n:
                continue
            val = (w * np.prod(xi ** np.array(alpha), axis=1)).sum()
            if abs(val - gaussian_moment(alpha)) > 1e-12 * max(1.0, gaussian_moment(alpha)):
                ok = False
                break
        if not ok:
            return deg
        deg = n
    return deg


def test_d3q39_quadrature_degree_7():
    e, w, r = O.lattice(39)
    assert len(w) == 39 and abs(w.sum() - 1) < 1e-15
    assert abs(r - math.sqrt(1.5)) < 1e-15
    assert len({tuple(v) for v in e}) == 39
    assert quadrature_max_exact_degree(39) == 7


def test_d3q19_quadrature_degree_5():
    e, w, r = O.lattice(19)
    assert len(w) == 19 and abs(w.sum() - 1) < 1e-15
    assert quadrature_max_exact_degree(19) == 5


# ---------------------------------------------------------------------------------------
# Derived constants: Eq. tau, Eq. MFP, Appendix A, Table 3

def test_tau_relation_eq_tau(golden_dir):
    g = read_golden_numbers(os.path.join(golden_dir, "paper_numbers.txt"))
    for q, key in ((39, "c_over_cs_d3q39"), (19, "c_over_cs_d3q19")):
        for kn, H in ((0.1, 64), (0.05, 32), (0.25, 20)):
            d = O.derive(W.config(ncx=H, ncy=1, ppc=10, lattice=q, kn=kn, seed=1))
            assert d["r_lat"] == pytest.approx(g[key], rel=1e-15)
            assert d["tau"] == pytest.approx(math.sqrt(math.pi / 8) * g[key] * kn * H + 0.5,
                                             rel=1e-14)
    d = O.derive(W.WORKLOADS["poiseuille_64x1_ppc100_fp64"])
    assert d["tau"] == pytest.approx(5.412, abs=1e-3)
    d = O.derive(W.WORKLOADS["poiseuille_64x256_ppc50_fp32"])
    assert d["tau"] == pytest.approx(5.412, abs=1e-3)


def test_thermal_speed_matches_table3(golden_dir):
    g = read_golden_numbers(os.path.join(golden_dir, "paper_numbers.txt"))
    cfg = W.config(ncx=16, ncy=1, ppc=10, seed=1, T_K=g["gas_temperature_K"],
                   mass_kg=g["gas_mass_kg"])
    c_th = O.derive(cfg)["c_th_ms"]
    # Table 3's standard deviations of v_y agree with sqrt(kT/m) to 0.5%, not sqrt(2kT/m).
    for k in ("table3_sigma_vy_dsmc_kn015", "table3_sigma_vy_lb2dsmc_kn015",
              "table3_sigma_vy_dsmc_kn025", "table3_sigma_vy_lb2dsmc_kn025"):
        assert abs(g[k] / c_th - 1) < 0.005
        assert abs(g[k] / (math.sqrt(2) * c_th) - 1) > 0.25


def test_force_from_no_slip_parabola():
    # u_max = g H^2 / (8 nu) with u_max = Ma c_s (Sec. 3.1), in lattice units, times r.
    cfg = W.config(ncx=20, ncy=1, ppc=10, seed=1, kn=0.07, ma=0.1, lb_ratio=2)
    d = O.derive(cfg)
    nu = (d["tau"] - 0.5) / 1.5
    g_lat = 8 * nu * 0.1 * math.sqrt(2 / 3) / (40.0 ** 2)
    assert d["g_step"] == pytest.approx(g_lat * math.sqrt(1.5), rel=1e-13)
    assert d["dt"] == pytest.approx(math.sqrt(2 / 3) / 2, rel=1e-15)
    assert d["lam"] == pytest.approx(0.07 * 20, rel=1e-15)


# ---------------------------------------------------------------------------------------
# DSMC: initialisation, NTC collisions, walls, sort

def test_init_maxwellian_and_uniform_positions():
    cfg = small_cfg(ncx=32, ncy=8, ppc=200, capacity_factor=1.25)
    o = O.Oracle(cfg)
    p = o.particles()
    n = p["x"].size
    assert n == 32 * 8 * 200
    v = np.stack([p["vx"], p["vy"], p["vz"]])
    se = 1 / math.sqrt(n)
    assert np.all(np.abs(v.mean(1)) < 5 * se)
    assert np.all(np.abs(v.var(1) - 1) < 5 * math.sqrt(2) * se)
    # fourth moment of a unit Gaussian is 3
    assert np.all(np.abs((v ** 4).mean(1) - 3) < 5 * math.sqrt(96) * se)
    cs = o.get(O.A_CELL_START)
    cell = np.repeat(np.arange(32 * 8), np.diff(cs))
    assert np.all(np.floor(p["x"]) == cell % 32)
    assert np.all(np.floor(p["y"]) == cell // 32)
    frac = p["x"] - np.floor(p["x"])
    hist, _ = np.histogram(frac, bins=16, range=(0, 1))
    assert ((hist - n / 16) ** 2 / (n / 16)).sum() < 45  # 15 dof


def test_ntc_candidate_count_eq_collisionnumber():
    cfg = small_cfg(ma=0.0)
    o = O.Oracle(cfg)
    d = o.d
    o.dsmc_phase(0)
    N = np.diff(o.get(O.A_CELL_START)).astype(np.float64)
    before = o.counters()["candidates"]
    o.dsmc_phase(1)
    got = o.counters()["candidates"] - before
    # first step: N-bar = N, (sigma c_r)_max at its initial value, no remainder
    ncand = 0.5 * N * N * cfg["crmax_init"] * d["coll_dt"]
    want = int(np.floor(ncand[N >= 2]).sum())
    assert got == want


def _cell_sums(o):
    p = o.particles()
    cs = o.get(O.A_CELL_START)
    cell = np.repeat(np.arange(len(cs) - 1), np.diff(cs))
    v = np.stack([p["vx"], p["vy"], p["vz"]], 1)
    mom = np.zeros((len(cs) - 1, 3))
    en = np.zeros(len(cs) - 1)
    np.add.at(mom, cell, v)
    np.add.at(en, cell, (v ** 2).sum(1))
    return mom, en


def test_collisions_conserve_momentum_and_energy_per_cell():
    o = O.Oracle(small_cfg(ppc=60))
    o.dsmc_phase(0)
    m0, e0 = _cell_sums(o)
    c0 = o.counters()["collisions"]
    o.dsmc_phase(1)
    assert o.counters()["collisions"] - c0 > 50
    m1, e1 = _cell_sums(o)
    assert np.abs(m1 - m0).max() < 1e-12
    assert np.abs(e1 - e0).max() < 1e-11
    # and the velocities did change
    p = o.particles()
    assert not np.allclose(e0, 0)


def test_hard_sphere_collision_rate_equals_mean_speed_over_mfp():
    # Equilibrium box: collisions per step = 1/2 N_tot (<c>/lambda) dt with <c> = sqrt(8/pi)
    # (Eq. MFP: lambda = <c>/nu for hard spheres).
    cfg = small_cfg(ncx=24, ncy=8, ppc=50, ma=0.0, kn=0.08, crmax_init=5.0)
    o = O.Oracle(cfg)
    d = o.d
    o.dsmc_step(20)  # let (sigma c_r)_max settle
    c0 = o.counters()["collisions"]
    steps = 200
    o.dsmc_step(steps)
    got = (o.counters()["collisions"] - c0) / steps
    ntot = 24 * 8 * 50
    want = 0.5 * ntot * math.sqrt(8 / math.pi) / d["lam"] * d["dt"]
    # counts per step are ~Poisson with mean `want`; 200 steps, allow 4 sigma + 1% bias
    assert abs(got - want) < 4 * math.sqrt(want / steps) + 0.01 * want


def test_wall_flux_and_equilibrium_is_kept():
    cfg = small_cfg(ncx=20, ncy=6, ppc=80, ma=0.0, kn=0.2)
    o = O.Oracle(cfg)
    d = o.d
    steps = 100
    o.dsmc_step(steps)
    hits = o.counters()["wall_hits"] / steps
    # one-sided Maxwellian flux n <c>/4 through each wall of area ncy (cell units)
    want = 2 * 80 * math.sqrt(8 / math.pi) / 4 * 6 * d["dt"]
    assert abs(hits / want - 1) < 0.05
    p = o.particles()
    v = np.stack([p["vx"], p["vy"], p["vz"]])
    n = v.shape[1]
    assert np.all(np.abs(v.var(1) - 1) < 0.05)
    assert np.all(np.abs(v.mean(1)) < 5 / math.sqrt(n) * 3)
    assert o.scalars()["ntot"] == 20 * 6 * 80


@pytest.mark.parametrize("real_bytes", [4, 8])
def test_body_force_kick_then_drift_on_a_collisionless_wall_free_step(real_bytes):
    # Force-driven Poiseuille flow (Sec. 3.1): each step first adds the body force's velocity
    # increment g to v_y, then moves the particle with the kicked velocity. A collisionless,
    # wall-free step must therefore give exactly v_y' = v_y + g and y' = y + (v_y + g) dt,
    # x' = x + v_x dt, in the state precision. Collisionless: at Kn = 50 the NTC count of
    # Eq. collisionnumber stays below one candidate per cell; wall-free: |v_x| dt keeps x
    # inside the channel. A kick after the drift, a kick scaled by dt, a missing or a doubled
    # kick each fail this.
    cfg = W.config(ncx=16, ncy=6, ppc=1, real_bytes=real_bytes, seed=9, kn=50.0, ma=0.3,
                   lb_ratio=2, capacity_factor=32.0)
    o = O.Oracle(cfg)
    d = o.d
    dt_ = np.float32 if real_bytes == 4 else np.float64
    g, dt = dt_(d["g_step"]), dt_(d["dt"])
    assert 0.1 < g < 2.0  # a kick of the order of the thermal speed: the test resolves it
    rng = np.random.default_rng(17)
    n = 96
    x = rng.uniform(3.0, 13.0, n).astype(dt_)
    y = rng.uniform(1.5, 3.5, n).astype(dt_)
    vx = rng.uniform(-2.0, 2.0, n).astype(dt_)
    vy = rng.uniform(-1.5, 1.5, n).astype(dt_)
    vz = (np.arange(n) * 0.01 + 0.5).astype(dt_)  # distinct: identifies each particle
    cs = np.full(16 * 6 + 1, n, np.uint32)
    cs[0] = 0  # all listed under cell 0; the step sorts them into their cells
    o.set_particles(x, y, vx, vy, vz, cs)
    o.dsmc_step(1)
    assert o.counters()["candidates"] == 0 and o.counters()["wall_hits"] == 0
    p = o.particles()
    k = np.argsort(p["vz"])
    vy1 = (vy + g).astype(dt_)
    assert np.array_equal(p["vy"][k], vy1)
    assert np.array_equal(p["y"][k], (y + vy1 * dt).astype(dt_))
    assert np.array_equal(p["x"][k], (x + vx * dt).astype(dt_))
    assert np.array_equal(p["vx"][k], vx) and np.array_equal(p["vz"][k], vz)


def test_dsmc_poiseuille_bulk_curvature_follows_chapman_enskog_viscosity():
    # Force-driven plane Poiseuille flow (Sec. 3.1) of the DSMC gas at small Kn: in steady
    # state the momentum balance in the bulk, away from the Knudsen layers, is
    # nu u'' = -g / dt (acceleration g / dt per unit time), with nu the kinematic viscosity of
    # hard spheres from Chapman-Enskog, mu = 1.016 (5/16) sqrt(pi m k T) / (pi d^2), i.e.
    # nu = 1.016 (5/16) sqrt(2 pi) lambda c_th for the mean free path lambda of Eq. MFP. The
    # profile's fitted curvature over the central columns is compared with -g / (2 nu dt)
    # within a batch-means confidence interval; the NTC scheme's cell-size bias at
    # cell = lambda / 2 (about 3%, Alexander, Garcia and Alder 1998) is allowed for.
    # The run starts from the expected profile (a parabola plus an estimated slip) so that no
    # start-up transient has to decay.
    H, NY, PPC, KN, MA = 32, 16, 50, 0.0625, 0.2
    cfg = W.config(ncx=H, ncy=NY, ppc=PPC, real_bytes=8, seed=12, kn=KN, ma=MA, lb_ratio=2)
    o = O.Oracle(cfg)
    d = o.d
    lam = KN * H
    nu = 1.016 * 5 / 16 * math.sqrt(2 * math.pi) * lam
    gacc = d["g_step"] / d["dt"]
    c2_want = -gacc / (2 * nu)
    p = o.particles()
    slip = 1.1 * lam * gacc * H / (2 * nu)
    vy = p["vy"] - c2_want * p["x"] * (H - p["x"]) + slip
    o.set_particles(p["x"], p["y"], p["vx"], vy, p["vz"], o.get(O.A_CELL_START))
    o.dsmc_step(300)
    xc = np.arange(H) + 0.5
    sel = (xc > 2 * lam + 1) & (xc < H - 2 * lam - 1)
    a0 = o.acc().copy()
    c2 = []
    for _ in range(8):
        o.dsmc_step(500)
        a1 = o.acc().copy()
        da = (a1 - a0).reshape(NY, H, 20)
        a0 = a1
        u = da[:, :, 2].sum(0) / da[:, :, 0].sum(0)
        c2.append(np.polyfit(xc[sel] - H / 2, u[sel], 2)[0])
    c2 = np.array(c2)
    rel = c2.mean() / c2_want - 1
    se = c2.std(ddof=1) / math.sqrt(len(c2)) / abs(c2_want)
    assert se < 0.08, se
    assert abs(rel) < 4 * se + 0.04, (rel, se)


@pytest.mark.parametrize("ncy,ncz", [(5, 0), (2, 0), (4, 3), (3, 2)])
def test_order_in_a_cell_by_neighbour_offset_then_rank_far_ones_after(ncy, ncz):
    # One collisionless, force-free step of particles displaced by up to two cells along every
    # axis. The order of every cell's particles afterwards is recomputed here from its
    # definition: particles displaced by at most one cell along every axis (streamwise and
    # spanwise periodic, +1 taken where +1 and -1 are the same cell) first, by the offset
    # o = [9 (dz + 1) +] 3 (dy + 1) + dx + 1, then by their rank in their old cell; the others
    # after them, by old cell, then rank. Channels of two rows or layers cover the +1 = -1 case.
    ncx = 8
    cfg = small_cfg(ncx=ncx, ncy=ncy, ncz=ncz, ppc=6, kn=1e6, ma=0.0, capacity_factor=10.0)
    o = O.Oracle(cfg)
    d = o.d
    dt = d["dt"]
    td = ncz >= 2
    nz = ncz if td else 1
    rng = np.random.default_rng(11)
    ncell = ncx * ncy * nz
    per = rng.integers(2, 9, ncell)
    cell = np.repeat(np.arange(ncell), per)  # grouped by old cell: rank = index in the group
    n = len(cell)
    ix, iy, iz = cell % ncx, (cell // ncx) % ncy, cell // (ncx * ncy)
    ix = np.clip(ix, 2, 5)  # keep away from the walls: |vx dt| < 2 hits none
    cell = (iz * ncy + iy) * ncx + ix
    order = np.argsort(cell, kind="stable")
    cell = cell[order]
    ix, iy, iz = ix[order], iy[order], iz[order]
    x = ix + rng.uniform(0.05, 0.95, n)
    y = iy + rng.uniform(0.05, 0.95, n)
    z = iz + rng.uniform(0.05, 0.95, n) if td else np.zeros(n)
    vx = rng.uniform(-1.9, 1.9, n) / dt
    vy = rng.uniform(-2.4, 2.4, n) / dt
    vz = (rng.uniform(-2.4, 2.4, n) / dt) if td else rng.normal(0.0, 1.0, n)
    counts = np.bincount(cell, minlength=ncell)
    cs = np.zeros(ncell + 1, np.uint32)
    cs[1:] = np.cumsum(counts)
    rank = np.arange(n) - cs[cell]
    o.set_particles(x, y, vx, vy, vz, cs, z=z if td else None)
    o.dsmc_step(1)
    assert o.counters()["collisions"] == 0 and o.counters()["wall_hits"] == 0

    def wrap(v, period):
        v = v - period * np.floor(v / period)
        return np.where(v >= period, v - period, v)

    nxp = np.floor(x + vx * dt).astype(int)
    nyp = np.floor(wrap(y + vy * dt, ncy)).astype(int)
    nzp = np.floor(wrap(z + vz * dt, nz)).astype(int) if td else np.zeros(n, int)
    new = (nzp * ncy + nyp) * ncx + nxp

    def disp(dlt, period):  # -1, 0, 1, or None (farther)
        e = dlt % period
        if e == 0:
            return 0
        if e == 1:
            return 1
        if e == period - 1:
            return -1
        return None

    keys = []
    nfar = 0
    for i in range(n):
        dx = int(nxp[i] - ix[i])
        dy = disp(int(nyp[i] - iy[i]), ncy)
        dz = disp(int(nzp[i] - iz[i]), nz) if td else 0
        if abs(dx) <= 1 and dy is not None and dz is not None:
            off = (9 * (dz + 1) if td else 0) + 3 * (dy + 1) + dx + 1
            keys.append((int(new[i]), 0, off, int(rank[i])))
        else:
            nfar += 1
            keys.append((int(new[i]), 1, int(cell[i]), int(rank[i])))
    assert nfar >= 5 and n - nfar >= 20  # both kinds occur
    want = sorted(range(n), key=lambda i: keys[i])
    p = o.particles()
    assert np.array_equal(p["vx"], vx[want]) and np.array_equal(p["vy"], vy[want])
    assert np.array_equal(np.diff(o.get(O.A_CELL_START)), np.bincount(new, minlength=ncell))


def test_sort_is_stable_by_cell_brute_force():
    # zero velocities and no force: a step is sort + sampling only
    cfg = small_cfg(ncx=7, ncy=3, ppc=5, ma=0.0, real_bytes=4, capacity_factor=12.0)
    o = O.Oracle(cfg)
    rng = np.random.default_rng(3)
    n = 60
    x = rng.uniform(0, 7, n).astype(np.float32)
    y = rng.uniform(0, 3, n).astype(np.float32)
    z = np.zeros(n, np.float32)
    cs = np.full(22, n, np.uint32)
    cs[0] = 0  # all 60 listed under cell 0 before the step; the step sorts them
    o.set_particles(x, y, z, z, z, cs)
    o.dsmc_step(1)
    key = (np.floor(y).astype(int) * 7 + np.floor(x).astype(int))
    order = sorted(range(n), key=lambda i: key[i])  # Python's sort is stable
    p = o.particles()
    assert np.array_equal(p["x"], x[order]) and np.array_equal(p["y"], y[order])
    cs = o.get(O.A_CELL_START)
    assert np.array_equal(np.diff(cs), np.bincount(key, minlength=21))


def test_sampling_sums_match_direct_moments():
    o = O.Oracle(small_cfg(ncx=8, ncy=2, ppc=30))
    o.dsmc_step(1)
    acc = o.acc()
    p = o.particles()
    cs = o.get(O.A_CELL_START)
    c = 5
    sl = slice(cs[c], cs[c + 1])
    v = np.stack([p["vx"][sl], p["vy"][sl], p["vz"][sl]], 1)
    assert acc[c, 0] == v.shape[0]
    assert np.allclose(acc[c, 1:4], v.sum(0), rtol=1e-13, atol=1e-13)
    assert acc[c, 4 + 1] == pytest.approx((v[:, 0] * v[:, 1]).sum(), rel=1e-12)  # xy
    assert acc[c, 10 + 4] == pytest.approx((v[:, 0] * v[:, 1] * v[:, 2]).sum(), rel=1e-12)  # xyz
    assert acc[c, 19] == pytest.approx((v[:, 2] ** 3).sum(), rel=1e-12)  # zzz


def test_cell_velocity_scatter_matches_sigma_u():
    # Sec. 5: sigma_u = sqrt(kT / (m <N>)) / sqrt(S) for S independent samples; samples
    # every 50 steps are independent (corr(u_x, u_y) = -0.008).
    cfg = small_cfg(ncx=16, ncy=4, ppc=40, ma=0.0, kn=0.1, sample_every=50)
    o = O.Oracle(cfg)
    o.dsmc_step(50 * 30)
    acc = o.acc()
    S = o.scalars()["nsamples"]
    assert S == 30
    u = acc[:, 2] / acc[:, 0]
    sigma_u = 1 / math.sqrt(40 * S)
    ratio = u.std() / sigma_u
    # 64 cells: the sample sd of a Gaussian has relative sd ~ 1/sqrt(2*63) = 0.09
    assert 0.7 < ratio < 1.3


# ---------------------------------------------------------------------------------------
# LBM: conservation, force moments, Poiseuille

def _lb_moments(q, f):
    e, w, r = O.lattice(q)
    xi = e * r
    rho = f.sum()
    j = (f[:, None] * xi).sum(0)
    Pi = np.einsum("a,ai,aj->ij", f, xi, xi)
    Q = np.einsum("a,ai,aj,ak->ijk", f, xi, xi, xi)
    return rho, j, Pi, Q, xi, w


@pytest.mark.parametrize("q", [39, 19])
def test_lbm_collision_moments(q):
    # Mass kept; momentum gains rho g per step; second moment relaxes as BGK with the Guo
    # force term: Pi' = Pi_eq + (1 - 1/tau)(Pi - Pi_eq) + (1 - 1/2tau) rho (g u + u g).
    cfg = W.config(ncx=16, ncy=1, ppc=10, lattice=q, real_bytes=8, kn=0.2, ma=0.3, seed=1)
    d = O.derive(cfg)
    e, w, r = O.lattice(q)
    rng = np.random.default_rng(1)
    fs = w * (1 + 0.1 * rng.uniform(-1, 1, q))
    out = O.lbm_collide(cfg, fs)
    rho, j, Pi, Q, xi, _ = _lb_moments(q, fs)
    rho2, j2, Pi2, Q2, _, _ = _lb_moments(q, out)
    g = np.array([0, d["g_step"], 0])
    tau = d["tau"]
    assert rho2 == pytest.approx(rho, rel=1e-14)
    assert np.allclose(j2 - j, rho * g, atol=1e-14)
    u = (j + 0.5 * rho * g) / rho
    Pieq = rho * (np.outer(u, u) + np.eye(3))
    want = Pieq + (1 - 1 / tau) * (Pi - Pieq) + (1 - 0.5 / tau) * rho * (
        np.outer(g, u) + np.outer(u, g))
    assert np.allclose(Pi2, want, atol=1e-13)
    if q == 39:
        # third Hermite coefficient: rho uuu + (1 - 1/tau) a3neq + (1 - 1/2tau) rho sym(g u u)
        def h3(F):
            I = np.eye(3)
            m3 = np.einsum("a,ai,aj,ak->ijk", F, xi, xi, xi)
            m1 = (F[:, None] * xi).sum(0)
            return (m3 - np.einsum("i,jk->ijk", m1, I) - np.einsum("j,ik->ijk", m1, I)
                    - np.einsum("k,ij->ijk", m1, I))
        uuu = np.einsum("i,j,k->ijk", u, u, u)
        a3neq = h3(fs) - rho * uuu
        gsym = (np.einsum("i,j,k->ijk", g, u, u) + np.einsum("i,j,k->ijk", u, g, u)
                + np.einsum("i,j,k->ijk", u, u, g))
        want3 = rho * uuu + (1 - 1 / tau) * a3neq + (1 - 0.5 / tau) * rho * gsym
        assert np.allclose(h3(out), want3, atol=1e-13)


def test_lbm_mass_conserved_with_walls_and_force():
    cfg = W.config(ncx=12, ncy=5, ppc=10, lb_ratio=2, real_bytes=8, kn=0.1, ma=0.1, seed=1)
    o = O.Oracle(cfg)
    e, w, r = O.lattice(39)
    f0 = W.gen_populations(w, o.d["nnodes"], seed=4)
    o.set_f(f0)
    m0 = f0.sum()
    o.lbm_step(50)
    assert o.f().sum() == pytest.approx(m0, rel=1e-13)


@pytest.mark.parametrize("q,H,steps,skip,tol", [(19, 16, 6000, 0, 1e-4), (39, 32, 10000, 8, 2e-3)])
def test_lbm_poiseuille_small_kn(q, H, steps, skip, tol):
    # Steady plane Poiseuille: u'' = -g / nu with nu = (tau - 1/2) c_s^2 away from the
    # walls' kinetic layer (the Navier-Stokes limit the paper's LB recovers at small Kn).
    cfg = W.config(ncx=H, ncy=1, ppc=10, lattice=q, real_bytes=8, kn=0.01, ma=0.1, seed=1)
    o = O.Oracle(cfg)
    d = o.d
    o.lbm_step(steps)
    f = o.f()[:, 0, :]
    e, w, r = O.lattice(q)
    rho = f.sum(0)
    u = ((f * (e[:, 1, None] * r)).sum(0) + 0.5 * rho * d["g_step"]) / rho
    nu = (d["tau"] - 0.5) * d["cs_lat"] ** 2
    curv = (u[2:] - 2 * u[1:-1] + u[:-2]) / (-d["g_step"] / nu)
    inner = curv[skip:len(curv) - skip] if skip else curv
    assert np.all(np.abs(inner - 1) < tol)
    assert np.allclose(rho, 1.0, atol=1e-3)
    # the profile is symmetric and peaks mid-channel
    assert np.allclose(u, u[::-1], rtol=1e-9, atol=1e-12)
    assert np.argmax(u) in (H // 2 - 1, H // 2)


# ---------------------------------------------------------------------------------------
# DSMC2LB (Sec. 2.1)

def _sums_from_coeffs(rho, u, P, Q, S, ppc):
    """Cumulative sums of a cell whose per-particle raw moments are u, P (<v v>), Q (<v v v>)."""
    NS = rho * ppc * S
    m = np.zeros(20)
    m[0] = NS
    m[1:4] = NS * u
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
    return m


def _herm_coeffs_of_f(q, f):
    e, w, r = O.lattice(q)
    xi = e * r
    I = np.eye(3)
    a0 = f.sum()
    a1 = (f[:, None] * xi).sum(0)
    a2 = np.einsum("a,ai,aj->ij", f, xi, xi) - a0 * I
    m3 = np.einsum("a,ai,aj,ak->ijk", f, xi, xi, xi)
    a3 = m3 - np.einsum("i,jk->ijk", a1, I) - np.einsum("j,ik->ijk", a1, I) - np.einsum(
        "k,ij->ijk", a1, I)
    return a0, a1, a2, a3


def test_dsmc2lb_round_trip_recovers_moments():
    rng = np.random.default_rng(11)
    rho, u = 1.07, np.array([0.03, 0.11, -0.02])
    A = rng.normal(0, 0.05, (3, 3))
    P = np.eye(3) + np.outer(u, u) + (A + A.T) / 2
    B = rng.normal(0, 0.05, (3, 3, 3))
    Qs = sum(np.transpose(B, p) for p in itertools.permutations(range(3))) / 6
    Q = Qs + np.einsum("i,jk->ijk", u, P) * 0  # arbitrary symmetric third moment
    S, ppc = 37, 50
    f = O.dsmc2lb_node(39, _sums_from_coeffs(rho, u, P, Q, S, ppc), S, ppc)
    a0, a1, a2, a3 = _herm_coeffs_of_f(39, f)
    I = np.eye(3)
    assert a0 == pytest.approx(rho, rel=1e-13)
    assert np.allclose(a1, rho * u, atol=1e-13)
    assert np.allclose(a2, rho * (P - I), atol=1e-13)
    want3 = rho * (Q - np.einsum("i,jk->ijk", u, I) - np.einsum("j,ik->ijk", u, I)
                   - np.einsum("k,ij->ijk", u, I))
    assert np.allclose(a3, want3, atol=1e-13)


def test_dsmc2lb_of_a_maxwellian_is_the_third_order_equilibrium():
    rho, u = 0.93, np.array([-0.04, 0.12, 0.05])
    I = np.eye(3)
    P = I + np.outer(u, u)
    Q = (np.einsum("i,j,k->ijk", u, u, u) + np.einsum("i,jk->ijk", u, I)
         + np.einsum("j,ik->ijk", u, I) + np.einsum("k,ij->ijk", u, I))
    f = O.dsmc2lb_node(39, _sums_from_coeffs(rho, u, P, Q, 10, 100), 10, 100)
    e, w, r = O.lattice(39)
    xu = (e * r) @ u
    u2 = u @ u
    feq = w * rho * (1 + xu + 0.5 * (xu ** 2 - u2) + xu * (xu ** 2 - 3 * u2) / 6)
    assert np.allclose(f, feq, rtol=1e-13, atol=1e-16)


def test_dsmc2lb_d3q19_reduces_to_eq_feq_dsmc():
    # Sec. 4, Eq. feq_dsmc, written in lattice units with c_s^2 = 1/3.
    rho, uH = 1.02, np.array([0.01, 0.09, -0.03])
    I = np.eye(3)
    P = I + np.outer(uH, uH)
    Q = np.zeros((3, 3, 3))
    f = O.dsmc2lb_node(19, _sums_from_coeffs(rho, uH, P, Q, 5, 20), 5, 20)
    e, w, r = O.lattice(19)
    u_lat = uH / r
    cs2 = 1.0 / 3.0
    eu = e @ u_lat
    feq = w * rho * (1 + eu / cs2 + eu ** 2 / (2 * cs2 ** 2) - (u_lat @ u_lat) / (2 * cs2))
    assert np.allclose(f, feq, rtol=1e-13, atol=1e-16)


# ---------------------------------------------------------------------------------------
# LB2DSMC (Sec. 2.2, Table 1)

def _eq_populations(q, rho, u):
    e, w, r = O.lattice(q)
    xu = (e * r) @ u
    u2 = u @ u
    return w * rho * (1 + xu + 0.5 * (xu ** 2 - u2) + xu * (xu ** 2 - 3 * u2) / 6)


def test_lb2dsmc_at_equilibrium_is_textbook_box_muller():
    u = np.array([0.02, 0.08, -0.01])
    f = _eq_populations(39, 1.0, u)
    g = O.grad_coeffs(39, f)
    assert g["M"] < 1e-14 and g["C"] == pytest.approx(1.0, abs=1e-12)
    assert np.allclose(g["u"], u, atol=1e-15)
    n = 2000
    v, info = O.grad_sample(39, f, seed=99, cell=3, t=17, n=n)
    assert info["cap"] == 0 and info["attempts"] == n  # every first trial accepted
    # textbook Box-Muller on the same Philox words (counter: cell, step, tag 6 << 24 | k, 0)
    k = np.arange(n, dtype=np.uint32)
    ctr = np.stack([np.full(n, 3, np.uint32), np.full(n, 17, np.uint32),
                    (np.uint32(6) << np.uint32(24)) | k, np.zeros(n, np.uint32)], 1)
    r = O.philox(ctr, 99).astype(np.float64)
    uo = (r + 0.5) * 2.0 ** -32
    rad1 = np.sqrt(-2 * np.log(uo[:, 0]))
    rad2 = np.sqrt(-2 * np.log(uo[:, 2]))
    xi = np.stack([rad1 * np.cos(2 * np.pi * uo[:, 1]), rad1 * np.sin(2 * np.pi * uo[:, 1]),
                   rad2 * np.cos(2 * np.pi * uo[:, 3])], 1)
    assert np.allclose(v - u, xi, atol=1e-12)


def test_lb2dsmc_sampled_moments_match_grad_coefficients():
    # Non-equilibrium populations from a DSMC2LB projection with stress and heat flux
    rho, u = 1.0, np.array([0.0, 0.1, 0.0])
    I = np.eye(3)
    P = I + np.outer(u, u) + np.array([[0.06, -0.04, 0], [-0.04, -0.03, 0], [0, 0, -0.03]])
    Q = (np.einsum("i,j,k->ijk", u, u, u) + np.einsum("i,jk->ijk", u, I)
         + np.einsum("j,ik->ijk", u, I) + np.einsum("k,ij->ijk", u, I))
    Q = Q.copy()
    for perm in set(itertools.permutations((0, 1, 1))):
        Q[perm] += 0.05
    for perm in set(itertools.permutations((0, 0, 0))):
        Q[perm] += 0.04
    f = O.dsmc2lb_node(39, _sums_from_coeffs(rho, u, P, Q, 1, 100), 1, 100)
    g = O.grad_coeffs(39, f)
    assert 0.03 < g["M"] < 0.1
    n = 2_000_000
    v, info = O.grad_sample(39, f, seed=5, cell=1, t=0, n=n)
    assert info["cap"] == 0
    c = v - g["u"]
    se = 1 / math.sqrt(n)
    m2 = np.einsum("ni,nj->ij", c, c) / n
    # E[c c] = delta + a2; the sd of a product of unit Gaussians is <= sqrt(3)
    assert np.all(np.abs(m2 - (I + g["a2"])) < 5 * math.sqrt(3) * se)
    m3 = np.einsum("ni,nj,nk->ijk", c, c, c) / n
    assert np.all(np.abs(m3 - g["a3"]) < 5 * math.sqrt(15) * se)
    assert np.all(np.abs(c.mean(0)) < 5 * se)
    # acceptance efficiency is 1/C (Table 1 comments), up to the envelope violations
    eff = n / info["attempts"]
    assert abs(eff * g["C"] - 1) < 0.01
    assert info["envelope"] < 1e-3 * info["attempts"]


@pytest.mark.parametrize("q", [39, 19])
def test_lb2dsmc_coefficients_fp64_and_their_rounding_to_the_state(q):
    # Table 1 step 1 is solved in FP64: at a third-order equilibrium with velocity u the
    # comoving coefficients are u and zero to FP64 round-off (closed form), and the values the
    # float sampler takes are exactly the FP64 ones rounded to float.
    u = np.array([0.05, -0.1, 0.02])
    f_eq = _eq_populations(q, 1.1, u)
    g = O.grad_coeffs_packed(q, f_eq, 8)
    assert g["rho"] == pytest.approx(1.1, rel=1e-14)
    assert np.allclose(g["u"], u, rtol=0, atol=1e-15)
    if q == 39:  # D3Q39 integrates the third-order equilibrium exactly
        assert g["M"] < 1e-14
    e, w, r = O.lattice(q)
    f = W.gen_populations(w, 1, seed=11, eps=0.1, rho_eps=0.1)[:, 0]
    gd = O.grad_coeffs_packed(q, f, 8)
    gf = O.grad_coeffs_packed(q, f, 4)
    full = O.grad_coeffs(q, f)
    assert gd["C"] == full["C"] and np.array_equal(gd["u"], full["u"])
    assert gd["M"] > 1e-3
    for k in ("u", "a2", "a3"):
        assert np.array_equal(gf[k], gd[k].astype(np.float32).astype(np.float64)), k
    assert gf["C"] == float(np.float32(gd["C"])) and gf["rho"] == gd["rho"]


def test_lb2dsmc_particle_count_conserves_mass():
    cfg = small_cfg(ncx=10, ncy=3, ppc=40, real_bytes=8)
    o = O.Oracle(cfg)
    e, w, r = O.lattice(39)
    rho_cells = {4: 1.1737, 15: 0.6021, 22: 1.0}
    f = o.f().copy()
    for c, rho in rho_cells.items():
        ix, iy = c % 10, c // 10
        f[:, iy, ix] = w * rho
    o.set_f(f)
    n0 = o.scalars()["ntot"]
    cells = np.array(sorted(rho_cells), np.int32)
    o.map_lbm_to_dsmc(cells)
    s = o.scalars()
    created = o.counters()["created"]
    assert s["ntot"] == n0 - 3 * 40 + created
    assert o.counters()["deleted"] == 3 * 40
    cs = o.get(O.A_CELL_START)
    counts = np.diff(cs.astype(np.int64))
    p = o.particles()
    for c, rho in rho_cells.items():
        # E[N] = rho ppc: floor(rho ppc + U) is one of the two neighbouring integers
        assert math.floor(rho * 40) <= counts[c] <= math.floor(rho * 40) + 1
        sl = slice(cs[c], cs[c + 1])
        assert np.all(np.floor(p["y"][sl]) * 10 + np.floor(p["x"][sl]) == c)
    assert created == sum(counts[c] for c in rho_cells)
    untouched = [c for c in range(30) if c not in rho_cells]
    assert np.all(counts[untouched] == 40)
    o.dsmc_step(1)
    assert o.scalars()["ntot"] == n0 - 3 * 40 + created


def test_lb2dsmc_sigma_matches_table3_in_si_units(golden_dir):
    g = read_golden_numbers(os.path.join(golden_dir, "paper_numbers.txt"))
    c_th = O.derive(small_cfg())["c_th_ms"]
    u = np.array([0.0, 10.5 / c_th, 0.0])
    f = _eq_populations(39, 1.0, u)
    v, info = O.grad_sample(39, f, seed=3, cell=0, t=0, n=200_000)
    sigma = v[:, 1].std() * c_th
    # Table 3: sigma_vy of LB2DSMC particles 239.3 m/s (Kn 0.15), within sampling error
    assert abs(sigma / g["table3_sigma_vy_lb2dsmc_kn015"] - 1) < 0.01
    assert abs(v[:, 1].mean() * c_th - 10.5) < 5 * 240 / math.sqrt(200_000)


# ---------------------------------------------------------------------------------------
# Float series used by the float state path (ln by the atanh series, sin/cos of 2 pi u by
# quadrant reduction and Taylor series): error bounds against numpy's double functions.

def test_float_ln_series_error_bound():
    x = np.concatenate([np.arange(1, 1 << 16, dtype=np.float64) * 2.0 ** -24,
                        np.linspace(2.0 ** -8, 1.0, 200_001), np.linspace(1.0, 4.0, 50_001)])
    x = x.astype(np.float32)
    ln, _, _ = O.float_funcs(x)
    want = np.log(x.astype(np.float64))
    err = np.abs(ln.astype(np.float64) - want)
    assert np.all(err <= 2.5e-7 * np.abs(want) + 1.2e-7), err.max()


def test_float_sincos_series_error_bound():
    u = (np.arange(0, 1 << 24, 37, dtype=np.float64) * 2.0 ** -24).astype(np.float32)
    _, s, c = O.float_funcs(u)
    th = 2 * np.pi * u.astype(np.float64)
    assert np.abs(s - np.sin(th)).max() < 2.5e-7
    assert np.abs(c - np.cos(th)).max() < 2.5e-7
    # exact at the quadrant points
    _, s4, c4 = O.float_funcs(np.array([0, 0.25, 0.5, 0.75], np.float32))
    assert np.array_equal(s4, [0, 1, 0, -1]) and np.array_equal(c4, [1, 0, -1, 0])


@pytest.mark.parametrize("real_bytes", [4, 8])
def test_gaussian_pairs_are_unit_normal(real_bytes):
    n = 400_000
    ctr = np.zeros((n // 4, 4), np.uint32)
    ctr[:, 0] = np.arange(n // 4)
    words = O.philox(ctr, 77).reshape(-1)
    z = O.gauss_pairs(words, real_bytes).reshape(-1)
    se = 1 / math.sqrt(z.size)
    assert abs(z.mean()) < 5 * se
    assert abs(z.var() - 1) < 5 * math.sqrt(2) * se
    assert abs((z ** 4).mean() - 3) < 5 * math.sqrt(96) * se
    # Kolmogorov-Smirnov distance to the normal CDF
    from math import erf
    zs = np.sort(z)
    cdf = 0.5 * (1 + np.vectorize(erf)(zs / math.sqrt(2)))
    ks = np.max(np.abs(cdf - np.arange(1, zs.size + 1) / zs.size))
    assert ks < 1.63 / math.sqrt(zs.size)  # 99% critical value


def test_float_state_init_is_maxwellian():
    cfg = small_cfg(ncx=32, ncy=8, ppc=200, real_bytes=4, capacity_factor=1.25)
    o = O.Oracle(cfg)
    p = o.particles()
    v = np.stack([p["vx"], p["vy"], p["vz"]]).astype(np.float64)
    se = 1 / math.sqrt(v.shape[1])
    assert np.all(np.abs(v.mean(1)) < 5 * se)
    assert np.all(np.abs(v.var(1) - 1) < 5 * math.sqrt(2) * se)


@pytest.mark.parametrize("real_bytes,tol", [(8, 1e-13), (4, 2e-6)])
def test_grad_G_packed_form_equals_full_tensor_sum(real_bytes, tol):
    # the acceptance function G of Eq. distr_outeq in its fixed packed grouping (state
    # precision) against the full-tensor Hermite sum in double
    rho, u = 1.0, np.array([0.02, 0.1, -0.03])
    I = np.eye(3)
    P = I + np.outer(u, u) + np.array([[0.05, -0.03, 0.01], [-0.03, -0.02, 0.02], [0.01, 0.02, -0.03]])
    Q = (np.einsum("i,j,k->ijk", u, u, u) + np.einsum("i,jk->ijk", u, I)
         + np.einsum("j,ik->ijk", u, I) + np.einsum("k,ij->ijk", u, I))
    for perm in set(itertools.permutations((0, 1, 2))):
        Q[perm] += 0.03
    f = O.dsmc2lb_node(39, _sums_from_coeffs(rho, u, P, Q, 1, 100), 1, 100)
    xi = np.random.default_rng(2).standard_normal((5000, 3)).astype(np.float32).astype(np.float64)
    gp, gf = O.grad_G(39, f, xi, real_bytes)
    assert np.all(np.abs(gp - gf) <= tol * (1 + np.abs(gf)))


# ---------------------------------------------------------------------------------------
# Differentiated LBM: per-node parameters, the coupling-interface loss, and the oracle's
# reference gradient (central differences of the FP64 forward)

def _lbm_cfg(**kw):
    base = dict(ncx=6, ncy=4, ppc=10, lb_ratio=2, real_bytes=8, seed=3, kn=0.3, ma=0.5)
    base.update(kw)
    return W.config(**base)


def _perturbed_f(cfg, seed):
    e, w, r = O.lattice(cfg.get("lattice", 39))
    return W.gen_populations(w, O.derive(cfg)["nnodes"], seed=seed)


def test_node_params_equal_to_the_scalars_give_the_plain_step():
    cfg = _lbm_cfg()
    f0 = _perturbed_f(cfg, 5)
    a, b = O.Oracle(cfg), O.Oracle(cfg)
    a.set_f(f0)
    b.set_f(f0)
    n = a.d["nnodes"]
    b.set_node_params(np.full(n, a.d["g_step"]), np.full(n, a.d["tau"]))
    a.lbm_step(3)
    b.lbm_step(3)
    assert np.array_equal(a.f(), b.f())


def test_interface_coefficients_of_dsmc2lb_populations_are_the_central_moments():
    # DSMC2LB builds populations whose raw moments up to order 3 are those of the particle
    # sample (quadrature exact to degree 7), so the Grad coefficients of the loss must be the
    # sample's central moments: rho, u, <cc> - I, <ccc>.
    rng = np.random.default_rng(4)
    rho, u = 0.97, np.array([0.05, -0.08, 0.02])
    A = rng.normal(0, 0.05, (3, 3))
    P = np.eye(3) + np.outer(u, u) + (A + A.T) / 2
    B = rng.normal(0, 0.05, (3, 3, 3))
    Q = sum(np.transpose(B, p) for p in itertools.permutations(range(3))) / 6
    S, ppc = 19, 40
    f = O.dsmc2lb_node(39, _sums_from_coeffs(rho, u, P, Q, S, ppc), S, ppc)
    cfg = _lbm_cfg()
    o = O.Oracle(cfg)
    e, w, r = O.lattice(39)
    full = np.tile(w[:, None], (1, o.d["nnodes"]))
    full[:, 7] = f
    o.set_f(full)
    m = o.grad_node(7)
    C2 = P - np.outer(u, u) - np.eye(3)
    C3 = (Q - np.einsum("i,jk->ijk", u, P) - np.einsum("j,ik->ijk", u, P)
          - np.einsum("k,ij->ijk", u, P) + 2 * np.einsum("i,j,k->ijk", u, u, u))
    p2 = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]
    p3 = [(0, 0, 0), (0, 0, 1), (0, 0, 2), (0, 1, 1), (0, 1, 2), (0, 2, 2), (1, 1, 1),
          (1, 1, 2), (1, 2, 2), (2, 2, 2)]
    assert m[0] == pytest.approx(rho, rel=1e-13)
    assert np.allclose(m[1:4], u, atol=1e-13)
    assert np.allclose(m[4:10], [C2[i, j] for i, j in p2], atol=1e-12)
    assert np.allclose(m[10:20], [C3[i, j, k] for i, j, k in p3], atol=1e-12)
    # at the lattice equilibrium at rest every coefficient but rho vanishes
    o.set_f(np.tile(w[:, None], (1, o.d["nnodes"])))
    m0 = o.grad_node(3)
    assert m0[0] == pytest.approx(1.0, rel=1e-14)
    assert np.abs(m0[1:]).max() < 1e-14


def test_interface_loss_gradient_vanishes_outside_the_light_cone():
    # f_T at a node depends on the parameters within MAXV (= 3) rows per step, walls included
    # (a wall density sums rows y -+ 3), so after T steps rows farther than 3 T are exactly
    # outside: the central differences there are exactly zero.
    cfg = _lbm_cfg(ncx=6, ncy=10)  # 12 x 20 nodes
    d = O.derive(cfg)
    nx, ny, n = d["nx"], d["ny"], d["nnodes"]
    rng = np.random.default_rng(9)
    g = d["g_step"] * (1 + 0.3 * rng.standard_normal(n))
    tau = d["tau"] * (1 + 0.1 * rng.standard_normal(n))
    f0 = _perturbed_f(cfg, 6)
    node = 10 * nx + 3
    o = O.Oracle(cfg)
    o.set_f(f0)
    o.set_node_params(g, tau)
    o.lbm_step(2)
    targets = o.grad_node(node) + 0.01 * rng.standard_normal(20)
    far = [y * nx + x for y in (0, 1, 2, 3, 17, 18, 19) for x in (0, 3, 11)]
    near = [node, node + 1, 9 * nx + 3, 10 * nx + 0]
    dg, dt = O.interface_loss_fd_gradient(cfg, f0, g, tau, [node], targets, 2, which=far + near)
    assert np.all(dg[:len(far)] == 0.0) and np.all(dt[:len(far)] == 0.0)
    assert np.all(np.abs(dg[len(far):]) > 0) and np.abs(dt[len(far)]) > 0


def test_interface_loss_gradient_of_one_step_at_tau_one():
    # At tau = 1 (om = 0, of = 1/2) one step gives j' = j + rho g exactly (the quadrature
    # reproduces the first moment of the series), so u'_y = j_y / rho + g and du'_y/dg = 1.
    # With every target equal to the reached value except u_y (shifted by delta),
    # L = delta^2 and dL/dg at the node is 2 delta.
    cfg = _lbm_cfg()
    d = O.derive(cfg)
    n = d["nnodes"]
    rng = np.random.default_rng(12)
    g = d["g_step"] * (1 + 0.2 * rng.standard_normal(n))
    tau = np.ones(n)
    f0 = _perturbed_f(cfg, 8)
    node = 2 * d["nx"] + 5
    o = O.Oracle(cfg)
    o.set_f(f0)
    o.set_node_params(g, tau)
    o.lbm_step(1)
    targets = o.grad_node(node)
    delta = 0.01
    targets[2] -= delta
    assert O.interface_loss_after(cfg, f0, g, tau, [node], targets, 1) == pytest.approx(
        delta * delta, rel=1e-12)
    dg, dt = O.interface_loss_fd_gradient(cfg, f0, g, tau, [node], targets, 1, which=[node])
    assert dg[0] == pytest.approx(2 * delta, rel=1e-6)


# ---------------------------------------------------------------------------------------
# The proof-of-concept hybrid of Sec. 4: unregularised BGK and the equilibrium DSMC2LB

def _moment_matrix(q):
    """Rows: the 20 moment functions 1, xi, xi xi (6), xi xi xi (10) at the lattice speeds."""
    e, w, r = O.lattice(q)
    xi = e * r
    rows = [np.ones(len(w))] + [xi[:, i] for i in range(3)]
    rows += [xi[:, i] * xi[:, j] for i in range(3) for j in range(i, 3)]
    rows += [xi[:, i] * xi[:, j] * xi[:, k] for i in range(3) for j in range(i, 3)
             for k in range(j, 3)]
    return np.array(rows)


@pytest.mark.parametrize("q", [19, 39])
def test_bgk_relaxes_a_ghost_mode_that_the_regularisation_removes(q):
    # A perturbation with no moment up to order 3 (a "ghost" mode of the lattice): the
    # regularised collision projects it out (f' = f_eq), plain BGK relaxes it by 1 - 1/tau
    # per step (f' = f_eq + (1 - 1/tau) delta). No force, so u is the flow velocity of f.
    e, w, r = O.lattice(q)
    cfg0 = small_cfg(lattice=q, ma=0.0, kn=0.2, lb_ratio=1)
    cfg1 = dict(cfg0, lb_collision=1)
    d = O.derive(cfg0)
    assert d["g_step"] == 0.0
    rho, u = 1.03, np.array([0.04, -0.07, 0.02])
    xu = (e * r) @ u
    u2 = u @ u
    feq = w * rho * (1 + xu + 0.5 * (xu ** 2 - u2)
                     + (xu * (xu ** 2 - 3 * u2) / 6 if q == 39 else 0))
    M = _moment_matrix(q)
    rng = np.random.default_rng(2)
    z = rng.standard_normal(len(w)) * w
    delta = z - np.linalg.pinv(M) @ (M @ z)
    assert np.abs(M @ delta).max() < 1e-14 and np.abs(delta).max() > 1e-4
    fs = feq + 0.05 * delta
    om = 1 - 1 / d["tau"]
    reg = O.lbm_collide(cfg0, fs)
    bgk = O.lbm_collide(cfg1, fs)
    assert np.allclose(reg, feq, rtol=0, atol=1e-15)
    assert np.allclose(bgk, feq + om * 0.05 * delta, rtol=0, atol=1e-15)


def test_bgk_conserves_mass_and_adds_rho_g():
    cfg = small_cfg(lattice=19, lb_ratio=1, lb_collision=1, ma=0.3, kn=0.1)
    d = O.derive(cfg)
    e, w, r = O.lattice(19)
    fs = W.gen_populations(w, 1, seed=3)[:, 0]
    out = O.lbm_collide(cfg, fs)
    xi = e * r
    assert out.sum() == pytest.approx(fs.sum(), rel=1e-14)
    j0, j1 = fs @ xi, out @ xi
    assert np.allclose(j1 - j0, [0, fs.sum() * d["g_step"], 0], atol=1e-15)


def test_equilibrium_dsmc2lb_is_eq_feq_dsmc_for_any_stress():
    # Sec. 4, Eq. feq_dsmc (lattice units, c_s^2 = 1/3): the populations depend on rho and u
    # only, whatever the sample's stress and heat flux; the Grad mapping does not.
    cfg = small_cfg(lattice=19, lb_ratio=1, d2l_mode=1)
    rng = np.random.default_rng(6)
    rho, uH = 0.98, np.array([0.02, 0.11, -0.04])
    A = rng.normal(0, 0.1, (3, 3))
    P = np.eye(3) + np.outer(uH, uH) + (A + A.T) / 2
    B = rng.normal(0, 0.1, (3, 3, 3))
    Q = sum(np.transpose(B, p) for p in itertools.permutations(range(3))) / 6
    S, ppc = 7, cfg["ppc"]
    sums = _sums_from_coeffs(rho, uH, P, Q, S, ppc)
    out = {}
    for mode in (1, 0):
        o = O.Oracle(dict(cfg, d2l_mode=mode))
        acc = o.acc().copy()
        acc[5] = sums
        o.set(O.A_ACC, acc.reshape(-1))
        o.set_scalars(o.scalars()["step"], S)
        o.map_dsmc_to_lbm(np.array([5], np.int32))
        out[mode] = o.f().reshape(19, -1)[:, 5]
    e, w, r = O.lattice(19)
    u_lat = uH / r
    cs2 = 1.0 / 3.0
    eu = e @ u_lat
    feq = w * rho * (1 + eu / cs2 + eu ** 2 / (2 * cs2 ** 2) - (u_lat @ u_lat) / (2 * cs2))
    assert np.allclose(out[1], feq, rtol=1e-13, atol=1e-16)
    assert np.abs(out[0] - feq).max() > 1e-4


# ---------------------------------------------------------------------------------------
# Kn varying along the channel

def test_kn_profile_at_constant_kn_is_the_plain_run():
    cfg = small_cfg(ncx=12, ncy=6, ppc=20, lb_ratio=2, ma=0.3)
    a = O.Oracle(cfg)
    b = O.Oracle(dict(cfg, kn_profile=1, kn_end=cfg["kn"]))
    for o in (a, b):
        o.dsmc_step(3)
        o.lbm_step(3)
    for k in ("x", "y", "vx", "vy", "vz"):
        assert np.array_equal(a.particles()[k], b.particles()[k])
    assert np.array_equal(a.f(), b.f())
    assert a.counters() == b.counters()


def test_kn_profile_collision_rate_follows_the_local_mean_free_path():
    # Equilibrium box with Kn from 0.04 (y = 0) to 0.4 (y = L/2): the collisions per step are
    # the hard-sphere rate 1/2 N <c> dt / lambda(y) summed over the cells, lambda(y) the
    # local mean free path, not the rate of any single Kn.
    cfg = small_cfg(ncx=24, ncy=16, ppc=40, ma=0.0, kn=0.04, kn_profile=1, kn_end=0.4,
                    crmax_init=5.0)
    o = O.Oracle(cfg)
    d = o.d
    o.dsmc_step(20)
    c0 = o.counters()["collisions"]
    steps = 150
    o.dsmc_step(steps)
    got = (o.counters()["collisions"] - c0) / steps
    ys = np.arange(16) + 0.5
    s = 1 - np.abs(2 * ys / 16 - 1)
    kn = 0.04 * (0.4 / 0.04) ** s
    want = sum(0.5 * 24 * 40 * math.sqrt(8 / math.pi) / (k * 24) * d["dt"] for k in kn)
    assert abs(got - want) < 4 * math.sqrt(want / steps) + 0.01 * want
    plain = 0.5 * 24 * 16 * 40 * math.sqrt(8 / math.pi) / d["lam"] * d["dt"]
    assert want < 0.6 * plain  # the profile's rate is far from the rate at kn


# ---------------------------------------------------------------------------------------
# Full 3D (ncz >= 2): periodic z for the particles and the lattice

def test_lbm_3d_with_z_uniform_populations_steps_like_the_slab_in_every_layer():
    # Populations that do not depend on z pull the same values from every layer, and the
    # wall densities of every (y, z) row equal those of the slab row y, so each layer of the
    # 3D step is exactly the quasi-2D step.
    for q in (39, 19):
        cfg2 = small_cfg(ncx=8, ncy=3, lb_ratio=2, lattice=q, ma=0.4, kn=0.15)
        cfg3 = dict(cfg2, ncz=3)
        a, b = O.Oracle(cfg2), O.Oracle(cfg3)
        e, w, r = O.lattice(q)
        f2 = W.gen_populations(w, a.d["nnodes"], seed=3).reshape(q, a.d["ny"], a.d["nx"])
        assert b.d["nz"] == 6
        a.set_f(f2)
        b.set_f(np.repeat(f2[:, None], b.d["nz"], axis=1))
        a.lbm_step(3)
        b.lbm_step(3)
        for z in range(b.d["nz"]):
            assert np.array_equal(b.f()[:, z], a.f()), (q, z)


def test_dsmc_3d_equilibrium_box_collision_rate_and_wall_flux():
    # A 3D box at rest: the hard-sphere collision rate 1/2 N <c> dt / lambda, the one-sided
    # flux n <c> / 4 through each wall of area ncy ncz, z positions inside [0, ncz) and the
    # z velocities of unit variance.
    cfg = small_cfg(ncx=12, ncy=4, ppc=30, ma=0.0, kn=0.1, crmax_init=5.0, ncz=5)
    o = O.Oracle(cfg)
    d = o.d
    assert d["ncells"] == 12 * 4 * 5
    o.dsmc_step(20)
    c0 = o.counters()["collisions"]
    h0 = o.counters()["wall_hits"]
    steps = 120
    o.dsmc_step(steps)
    ntot = 12 * 4 * 5 * 30
    got = (o.counters()["collisions"] - c0) / steps
    want = 0.5 * ntot * math.sqrt(8 / math.pi) / d["lam"] * d["dt"]
    assert abs(got - want) < 4 * math.sqrt(want / steps) + 0.01 * want
    hits = (o.counters()["wall_hits"] - h0) / steps
    want_h = 2 * 30 * math.sqrt(8 / math.pi) / 4 * (4 * 5) * d["dt"]
    assert abs(hits / want_h - 1) < 0.06
    p = o.particles()
    assert p["z"].min() >= 0 and p["z"].max() < 5
    assert abs(p["vz"].var() - 1) < 0.05
    assert o.scalars()["ntot"] == ntot
    # the particles of a cell lie in it
    cs = o.get(O.A_CELL_START)
    for c in (0, 77, 239):
        ix, iy, iz = c % 12, (c // 12) % 4, c // 48
        s = slice(cs[c], cs[c + 1])
        assert np.all(np.floor(p["x"][s]) == ix) and np.all(np.floor(p["y"][s]) == iy)
        assert np.all(np.floor(p["z"][s]) == iz)


def test_lbm_3d_without_force_commutes_with_swapping_y_and_z():
    # y and z are both periodic and the walls are normal to x, so without the body force the
    # lattice step is symmetric under the exchange of y and z (with e_y and e_z exchanged in
    # the velocity set). Populations that vary in x, y and z pin the sign and the layer of
    # the z pull and the per-(y, z) wall rows: stepping the exchanged populations gives the
    # exchanged result.
    for q in (39, 19):
        cfg = small_cfg(ncx=7, ncy=3, ncz=3, lb_ratio=2, lattice=q, ma=0.0, kn=0.2)
        o = O.Oracle(cfg)
        d = o.d
        assert d["g_step"] == 0.0 and d["ny"] == d["nz"] == 6
        e, w, r = O.lattice(q)
        idx = {tuple(v): k for k, v in enumerate(e.tolist())}
        perm = np.array([idx[(v[0], v[2], v[1])] for v in e.tolist()])
        shape = (q, d["nz"], d["ny"], d["nx"])
        fa = W.gen_populations(w, d["nnodes"], seed=19, eps=0.1, rho_eps=0.2).reshape(shape)
        fb = np.empty_like(fa)
        fb[perm] = fa.transpose(0, 2, 1, 3)  # f_b(x, y, z) at e' = f_a(x, z, y) at e
        o.set_f(fa)
        o.lbm_step(2)
        ga = o.f().copy()
        o2 = O.Oracle(cfg)
        o2.set_f(fb)
        o2.lbm_step(2)
        gb = o2.f()
        want = np.empty_like(ga)
        want[perm] = ga.transpose(0, 2, 1, 3)
        assert np.allclose(gb, want, rtol=1e-13, atol=1e-15), (q, np.abs(gb - want).max())
        assert not np.allclose(ga, ga[:, :1])  # the state does vary along z


def test_dsmc_3d_free_flight_moves_z_by_vz_dt_and_wraps():
    # At a huge Kn no pair is selected, and without the body force each particle flies
    # straight: z' = z + vz dt wrapped into [0, ncz), likewise y, x' = x + vx dt (no wall is
    # reached), and the velocities are unchanged. Each particle lands in the bin of the cell
    # holding it.
    cfg = small_cfg(ncx=6, ncy=3, ncz=4, ppc=10, kn=1e6, ma=0.0, capacity_factor=6.0)
    o = O.Oracle(cfg)
    d = o.d
    dt = d["dt"]
    rng = np.random.default_rng(4)
    n = 300
    x = rng.uniform(2.0, 4.0, n)
    y = rng.uniform(0.0, 3.0, n)
    z = rng.uniform(0.0, 4.0, n)
    vx = rng.uniform(-2.0, 2.0, n)  # |vx| dt < 2: no wall
    vy = rng.normal(0.0, 3.0, n)
    vz = rng.normal(0.0, 3.0, n)
    cell = (np.floor(z).astype(int) * 3 + np.floor(y).astype(int)) * 6 + np.floor(x).astype(int)
    order = np.argsort(cell, kind="stable")
    counts = np.bincount(cell, minlength=d["ncells"])
    cs = np.zeros(d["ncells"] + 1, np.uint32)
    cs[1:] = np.cumsum(counts)
    o.set_particles(x[order], y[order], vx[order], vy[order], vz[order], cs, z=z[order])
    o.dsmc_step(1)
    assert o.counters()["collisions"] == 0 and o.counters()["wall_hits"] == 0
    p = o.particles()
    got = np.argsort(p["vx"])
    ref = np.argsort(vx)
    assert np.array_equal(p["vx"][got], vx[ref]) and np.array_equal(p["vz"][got], vz[ref])
    assert np.array_equal(p["vy"][got], vy[ref])
    assert np.allclose(p["x"][got], (x + vx * dt)[ref], rtol=0, atol=1e-12)
    assert np.allclose(p["y"][got], np.mod(y + vy * dt, 3.0)[ref], rtol=0, atol=1e-12)
    assert np.allclose(p["z"][got], np.mod(z + vz * dt, 4.0)[ref], rtol=0, atol=1e-12)
    assert (np.abs(vz * dt) > 1).sum() > 50 and ((z + vz * dt < 0) | (z + vz * dt >= 4)).sum() > 20
    cs1 = o.get(O.A_CELL_START).astype(np.int64)
    own = np.repeat(np.arange(d["ncells"]), np.diff(cs1))
    c1 = (np.floor(p["z"]).astype(int) * 3 + np.floor(p["y"]).astype(int)) * 6 + np.floor(p["x"]).astype(int)
    assert np.array_equal(c1, own)


def test_dsmc2lb_is_linear_in_the_cumulative_sums_for_a_fixed_sample_count():
    # Eq. coefficients with rho = N / (S ppc) and the means M / N: every raw coefficient is
    # a sum over the cell's samples divided by S ppc (the N of rho cancels the N of the
    # means), so the mapped populations are linear in the sums. The adjoint of the mapping
    # is the transpose of this linear map.
    for q in (39, 19):
        cfg = small_cfg(ncx=6, ncy=2, lb_ratio=1, lattice=q)
        src = O.Oracle(dict(cfg, ma=0.4))
        src.dsmc_step(3)
        a = src.acc().copy()
        src.dsmc_step(4)
        b = src.acc().copy() - a
        S = 5
        nodes = np.arange(O.derive(cfg)["nnodes"], dtype=np.int32)

        def mapped(acc):
            o = O.Oracle(cfg)
            o.set(O.A_ACC, acc.reshape(-1))
            o.set_scalars(0, S)
            o.map_dsmc_to_lbm(nodes)
            return o.f().astype(np.float64)

        fa, fb, fab = mapped(a), mapped(b), mapped(0.3 * a + 1.7 * b)
        assert np.allclose(fab, 0.3 * fa + 1.7 * fb, rtol=1e-12, atol=1e-14)
        assert not np.allclose(fa, fb)


def test_kn_profile_rows_and_setters_reproduce_the_built_in_profile():
    # An oracle given the profile's per-cell NTC factors and per-node tau through the setters
    # steps exactly like one that builds the profile itself: this is what lets a window of
    # a large channel take the factors of the channel's own rows.
    cfg = small_cfg(ncx=8, ncy=6, ppc=12, lb_ratio=2, kn=0.01, kn_profile=1, kn_end=0.3,
                    real_bytes=4, ma=0.3)
    d = O.derive(cfg)
    coll, tau = O.kn_profile_rows(cfg, range(0, 6), range(0, d["ny"]))
    assert coll[0] > coll[3] and tau[0] < tau[d["ny"] // 2]  # Kn rises towards y = L/2
    a = O.Oracle(cfg)
    b = O.Oracle(dict(cfg, kn_profile=0))
    b.set_cell_coll(np.repeat(coll, 8))
    b.set_node_params(np.full(d["nnodes"], d["g_step"]), np.repeat(tau, d["nx"]))
    e, w, r = O.lattice(39)
    f0 = W.gen_populations(w, d["nnodes"], seed=5).astype(np.float32)
    for o in (a, b):
        o.set_f(f0)
        o.dsmc_step(3)
        o.lbm_step(2)
    for k in ("x", "y", "vx", "vy", "vz"):
        assert np.array_equal(a.particles()[k], b.particles()[k]), k
    assert a.counters() == b.counters()
    assert np.array_equal(a.f(), b.f())


def test_mappings_3d_reduce_to_the_slab_in_layer_zero():
    # With one LB node per cell and populations uniform in z, the cells and nodes of layer 0
    # keep the slab's ids and Philox keys: LB2DSMC gives the slab's particles exactly (x, y
    # and velocities), with z inside the cell; DSMC2LB of the same sums gives the slab's
    # populations. Cells of other layers draw their own particles, inside their own cells.
    for q in (39, 19):
        cfg2 = small_cfg(ncx=8, ncy=3, ppc=20, lb_ratio=1, lattice=q, real_bytes=8)
        cfg3 = dict(cfg2, ncz=3)
        a, b = O.Oracle(cfg2), O.Oracle(cfg3)
        e, w, r = O.lattice(q)
        f2 = W.gen_populations(w, O.derive(cfg2)["nnodes"], seed=6, eps=0.08, rho_eps=0.2)
        a.set_f(f2)
        b.set_f(np.tile(f2.reshape(q, 1, -1), (1, 3, 1)))
        cells2 = np.array([0, 5, 13, 23], np.int32)
        cells3 = np.concatenate([cells2, cells2 + 24, [47, 71]]).astype(np.int32)
        a.map_lbm_to_dsmc(cells2)
        b.map_lbm_to_dsmc(cells3)
        pa, pb = a.particles(), b.particles()
        csa = a.get(O.A_CELL_START).astype(np.int64)
        csb = b.get(O.A_CELL_START).astype(np.int64)
        for c in cells2:
            sa, sb = slice(csa[c], csa[c + 1]), slice(csb[c], csb[c + 1])
            for k in ("x", "y", "vx", "vy", "vz"):
                assert np.array_equal(pa[k][sa], pb[k][sb]), (q, c, k)
            assert np.all((pb["z"][sb] >= 0) & (pb["z"][sb] < 1))
        for c in cells3[4:]:
            sb = slice(csb[c], csb[c + 1])
            iz, iy, ix = c // 24, (c // 8) % 3, c % 8
            assert np.all(np.floor(pb["z"][sb]) == iz) and np.all(np.floor(pb["y"][sb]) == iy)
            assert np.all(np.floor(pb["x"][sb]) == ix)
        assert not np.array_equal(pb["vx"][csb[24]:csb[25]], pb["vx"][csb[0]:csb[1]])
        # DSMC2LB: layer-0 nodes from the same sums
        # (each layer has its own sums: layer 2 must take its own cells' sums)
        src = O.Oracle(dict(cfg2, ma=0.4))
        src.dsmc_step(4)
        acc0, S = src.acc().copy(), src.scalars()["nsamples"]
        src.dsmc_step(4)
        acc_l2 = src.acc().copy() * 0.5
        acc3 = np.concatenate([acc0, 0.9 * acc0, acc_l2])
        b.set(O.A_ACC, acc3.reshape(-1))
        b.set_scalars(0, S)
        nodes2 = np.arange(24, dtype=np.int32)
        b.map_dsmc_to_lbm(np.concatenate([nodes2, nodes2 + 48]).astype(np.int32))
        fb = b.f().reshape(q, -1)
        for acc, off in ((acc0, 0), (acc_l2, 48)):
            a.set(O.A_ACC, acc.reshape(-1))
            a.set_scalars(0, S)
            a.map_dsmc_to_lbm(nodes2)
            assert np.array_equal(a.f().reshape(q, -1)[:, nodes2], fb[:, nodes2 + off]), (q, off)


def test_interface_loss_3d_with_z_uniform_inputs_is_nz_times_the_slab():
    # populations, force increments and relaxation times that do not depend on z: every
    # layer steps like the slab, so the loss over each layer's copy of the slab's nodes is
    # nz times the slab's loss (the per-node step and the loss in 3D, against the slab)
    cfg2 = small_cfg(ncx=6, ncy=3, lb_ratio=1, ma=0.4, kn=0.2)
    cfg3 = dict(cfg2, ncz=3)
    d2 = O.derive(cfg2)
    e, w, r = O.lattice(39)
    rng = np.random.default_rng(8)
    n2 = d2["nnodes"]
    f2 = W.gen_populations(w, n2, seed=9)
    g2 = d2["g_step"] * (1 + 0.3 * rng.standard_normal(n2))
    t2 = d2["tau"] * (1 + 0.1 * rng.standard_normal(n2))
    nodes2 = np.array([0, 4, 7, 11, 17], np.int32)
    targets2 = 0.05 * rng.standard_normal((len(nodes2), 20))
    targets2[:, 0] += 1.0
    l2 = O.interface_loss_after(cfg2, f2, g2, t2, nodes2, targets2, 3)
    f3 = np.tile(f2.reshape(39, 1, n2), (1, 3, 1))
    nodes3 = np.concatenate([nodes2 + k * n2 for k in range(3)]).astype(np.int32)
    l3 = O.interface_loss_after(cfg3, f3, np.tile(g2, 3), np.tile(t2, 3), nodes3,
                                np.tile(targets2, (3, 1)), 3)
    assert l3 == pytest.approx(3 * l2, rel=1e-13)
    assert l2 > 0
