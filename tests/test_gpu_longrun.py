"""Long runs of the CUDA path against the statistical laws the paper and kinetic theory fix,
within stated confidence intervals: the hard-sphere collision rate of an equilibrium box
(Eq. MFP), the scatter of cell-mean velocities sigma_u (Sec. 5), the bulk curvature of the
DSMC Poiseuille profile against the Chapman-Enskog hard-sphere viscosity at small Kn
(Sec. 3.1), and the steady LB Poiseuille profile (Sec. 3.1, Eq. tau). Each law is written
out here from its definition; the runs are 10^3 to 10^4 steps, cheap on the GPU."""
import math

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


@pytest.mark.parametrize("real_bytes", [4, 8])
def test_equilibrium_box_collision_rate_is_half_n_mean_speed_over_mfp(real_bytes):
    # Hard spheres at rest between walls at the gas temperature: accepted collisions per step
    # = 1/2 N <c>/lambda dt with <c> = sqrt(8/pi) c_th (Eq. MFP: lambda = <c>/nu). Counts per
    # step are about Poisson; 2000 steps of 204,800 particles give a relative sd of 1e-4, and
    # the bound is 5 sd plus 0.3%.
    cfg = W.config(ncx=64, ncy=64, ppc=50, real_bytes=real_bytes, ma=0.0, kn=0.08,
                   crmax_init=5.0, seed=41)
    h = B.Hybrid(cfg)
    d = h.d
    h.dsmc_step(50)  # (sigma c_r)_max settles
    c0 = h.counters()["collisions"]
    steps = 2000
    h.dsmc_step(steps)
    got = (h.counters()["collisions"] - c0) / steps
    ntot = 64 * 64 * 50
    want = 0.5 * ntot * math.sqrt(8 / math.pi) / d["lam"] * d["dt"]
    assert abs(got - want) < 5 * math.sqrt(want / steps) + 0.003 * want, (got, want)
    assert h.n_tot() == ntot and h.sync_status()[0] == B.HYB_OK


def test_cell_mean_velocity_scatter_is_sigma_u():
    # Sec. 5: the cell-mean velocity over S independent samples of <N> particles scatters
    # with sigma_u = sqrt(kT/m) / sqrt(<N> S); samples every 50 steps are independent. 4096
    # cells: the sample sd has a relative sd of about 1/sqrt(2 * 4096) = 1.1%.
    cfg = W.config(ncx=64, ncy=64, ppc=40, ma=0.0, kn=0.1, sample_every=50, seed=43)
    h = B.Hybrid(cfg)
    h.dsmc_step(50 * 40)
    h.sync()
    acc = h.acc().cpu().numpy()
    S = int(h.ctrl().cpu()[B.CTRL_NSAMPLES])
    assert S == 40
    for comp in (1, 2, 3):
        u = acc[:, comp] / acc[:, 0]
        ratio = u.std() / (1 / math.sqrt(40 * S))
        assert 0.94 < ratio < 1.06, (comp, ratio)


def test_dsmc_poiseuille_bulk_curvature_follows_chapman_enskog_viscosity():
    # Force-driven plane Poiseuille flow at Kn = 0.0625 (lambda = 2 cells, H = 32 cells): in
    # steady state the bulk obeys nu u'' = -g / dt with the hard-sphere Chapman-Enskog
    # viscosity nu = 1.016 (5/16) sqrt(2 pi) lambda c_th. The fitted curvature of the mean
    # streamwise velocity over the central columns (2 lambda + 1 from each wall) is compared,
    # by batch means over 8 batches of 2000 steps, within 4 standard errors plus 4% (the NTC
    # cell-size bias at cell = lambda / 2 is about 3%, Alexander, Garcia and Alder 1998).
    H, NY, PPC, KN, MA = 32, 256, 50, 0.0625, 0.2
    cfg = W.config(ncx=H, ncy=NY, ppc=PPC, kn=KN, ma=MA, lb_ratio=2, seed=12)
    h = B.Hybrid(cfg)
    d = h.d
    lam = KN * H
    nu = 1.016 * 5 / 16 * math.sqrt(2 * math.pi) * lam
    gacc = d["g_step"] / d["dt"]
    c2_want = -gacc / (2 * nu)
    # start from the expected profile: a parabola plus an estimated slip
    p = {k: v.cpu().numpy() for k, v in h.particles().items()}
    slip = 1.1 * lam * gacc * H / (2 * nu)
    vy = p["vy"].astype(np.float64) - c2_want * p["x"] * (H - p["x"]) + slip
    h.load_particles(p["x"], p["y"], p["vx"], vy, p["vz"], h.cell_start().cpu().numpy())
    h.dsmc_step(500)
    xc = np.arange(H) + 0.5
    sel = (xc > 2 * lam + 1) & (xc < H - 2 * lam - 1)
    h.sync()
    a0 = h.acc().cpu().numpy().copy()
    c2 = []
    for _ in range(8):
        h.dsmc_step(2000)
        h.sync()
        a1 = h.acc().cpu().numpy().copy()
        da = (a1 - a0).reshape(NY, H, 20)
        a0 = a1
        u = da[:, :, 2].sum(0) / da[:, :, 0].sum(0)
        c2.append(np.polyfit(xc[sel] - H / 2, u[sel], 2)[0])
    c2 = np.array(c2)
    rel = c2.mean() / c2_want - 1
    se = c2.std(ddof=1) / math.sqrt(len(c2)) / abs(c2_want)
    assert se < 0.03, se
    assert abs(rel) < 4 * se + 0.04, (rel, se)


@pytest.mark.parametrize("lattice,real_bytes", [(39, 8), (39, 4), (19, 8)])
def test_lbm_poiseuille_steady_profile_has_curvature_minus_g_over_nu(lattice, real_bytes):
    # The LB channel at small Kn relaxes to the parabola u(x) = g / (2 nu) x (H - x) + slip with
    # nu = (tau - 1/2) c_s^2 in lattice units (Eq. tau, Sec. 3.1): the fitted curvature of u_y
    # over the central nodes is -g / nu. The D3Q39 kinetic walls leave a Knudsen layer of a few
    # nodes, excluded from the fit.
    cfg = W.config(ncx=16, ncy=2, ppc=4, lb_ratio=2, lattice=lattice, real_bytes=real_bytes,
                   kn=0.01, ma=0.1, seed=3)
    h = B.Hybrid(cfg)
    d = h.d
    q, nx = d["q"], d["nx"]
    e, w, r = B.lattice(q)
    e = np.asarray(e, np.float64).reshape(q, 3)
    h.lbm_step(20000)
    h.sync()
    f = h.f().double().cpu().numpy()  # [q, ny, nx]
    rho = f.sum(0)
    jy = np.einsum("a,ayx->yx", e[:, 1] * r, f)
    u = ((jy + 0.5 * rho * d["g_step"]) / rho).mean(0)  # thermal units, per node
    nu = (d["tau"] - 0.5) * d["cs_lat"] ** 2  # lattice units
    x = np.arange(nx) + 0.5
    skip = 8 if q == 39 else 2
    sel = slice(skip, nx - skip)
    c2 = np.polyfit(x[sel], u[sel], 2)[0]
    assert c2 == pytest.approx(-d["g_step"] / (2 * nu), rel=2e-3), (c2, -d["g_step"] / (2 * nu))
    assert np.allclose(u, u[::-1], rtol=1e-5, atol=1e-7)
