"""Parity at the full size of the large channel (512 x 4096 cells, 50 per cell: 104,857,600
particles; 1024 x 8192 D3Q39 nodes), with Kn 0.05 and with Kn 0.005-0.5 along the channel,
in the launch configuration bench.py times.

The oracle cannot step the whole channel in a test's time, so it steps a window: the first
rows of the same channel. Those rows keep the channel's cell ids, order keys and Philox
keys, so their particles are the channel's own from the first draw on. The window is
periodic over its own rows, so only rows within a few cells of its ends see different
neighbours; the rows in between are compared. With the Kn profile the window takes the
channel's per-cell NTC factors and per-node tau of its rows from the oracle (the profile
of the whole channel, evaluated at those rows)."""
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

LARGE = ["poiseuille_512x4096_ppc50_fp32", "poiseuille_512x4096_ppc50_knvar_fp32"]
R = 16              # window rows of DSMC cells
ROWS = range(5, 11)  # compared rows: 5 cells from the window's ends (a particle moves at
                     # most about 2.5 cells per step at these speeds)


def window_oracle(cfg, rows_cells):
    """The oracle of the channel's first `rows_cells` cell rows, with the channel's Kn
    profile at those rows."""
    wcfg = dict(cfg, ncy=rows_cells, kn_profile=0)
    o = O.Oracle(wcfg)
    if cfg.get("kn_profile", 0) == 1:
        d = O.derive(wcfg)
        coll, tau = O.kn_profile_rows(cfg, range(0, rows_cells), range(0, d["ny"]))
        o.set_cell_coll(np.repeat(coll, cfg["ncx"]))
        o.set_node_params(np.full(d["nnodes"], d["g_step"]), np.repeat(tau, d["nx"]))
    return o


@pytest.mark.parametrize("name", LARGE)
def test_large_channel_dsmc_steps_match_an_oracle_window(name):
    cfg = W.WORKLOADS[name]
    ncx = cfg["ncx"]
    h = B.Hybrid(cfg)
    assert h.d["ncells"] * cfg["ppc"] == 104_857_600
    steps = 2
    h.dsmc_step(steps)
    h.sync()
    o = window_oracle(cfg, R)
    o.dsmc_step(steps)
    c0, c1 = ROWS.start * ncx, ROWS.stop * ncx
    # per-cell counts (the sort) and state, bit for bit
    gcount = h.counts().cpu().numpy()[c0:c1]
    ocs = o.get(O.A_CELL_START).astype(np.int64)
    assert np.array_equal(gcount, np.diff(ocs)[c0:c1])
    assert np.array_equal(h.crmax().cpu().numpy()[c0:c1], o.get(O.A_CRMAX)[c0:c1])
    assert np.array_equal(h.rem().cpu().numpy()[c0:c1], o.get(O.A_REM)[c0:c1])
    assert np.array_equal(h.nbar_sum().cpu().numpy().view(np.uint32)[c0:c1],
                          o.get(O.A_NBAR_SUM)[c0:c1])
    ga, oa = h.acc().cpu().numpy()[c0:c1], o.acc()[c0:c1]
    scale = np.abs(oa).max(axis=0, keepdims=True) + 1e-30
    assert np.all(np.abs(ga - oa) <= 1e-5 * scale), np.abs((ga - oa) / scale).max()
    # the particles of those cells, in order
    arr = h.particle_arrays()
    mask = torch.arange(h.d["bin"], device="cuda")[None, :] < h.counts()[c0:c1, None]
    op = o.particles()
    for k in ("x", "y", "vx", "vy", "vz"):
        g = arr[k][c0:c1][mask].cpu().numpy()
        want = op[k][ocs[c0]:ocs[c1]]
        assert g.shape == want.shape, k
        assert (g == want).mean() >= 0.9999, k
        assert np.allclose(g, want, rtol=1e-5, atol=1e-5), (k, np.abs(g - want).max())
    # the window's first row, next to its periodic end, did see other neighbours: the
    # comparison is not vacuous
    assert not np.array_equal(h.counts().cpu().numpy()[:ncx], np.diff(ocs)[:ncx])
    h.close()
    del h, arr, mask
    torch.cuda.empty_cache()


@pytest.mark.parametrize("name", LARGE)
def test_large_channel_lbm_steps_match_an_oracle_window(name):
    cfg = W.WORKLOADS[name]
    h = B.Hybrid(cfg)
    d = h.d
    nx, ny = d["nx"], d["ny"]
    e, w, r = O.lattice(39)
    f0 = W.gen_populations(w, d["nnodes"], seed=31).astype(np.float32)
    h.f().copy_(torch.from_numpy(f0.reshape(h.f().shape)))
    torch.cuda.synchronize()
    steps = 2
    h.lbm_step(steps)
    h.sync()
    rows_nodes = R * cfg["lb_ratio"]
    o = window_oracle(cfg, R)
    o.set_f(np.ascontiguousarray(f0.reshape(39, ny, nx)[:, :rows_nodes]))
    o.lbm_step(steps)
    lo, hi = 3 * steps, rows_nodes - 3 * steps  # the pull reaches 3 rows per step
    gf = h.f()[:, lo:hi].cpu().numpy()
    of = o.f()[:, lo:hi]
    err = lb_err(gf, of, w)
    assert err < LB_TOL_FP32, err
    h.close()
    del h
    torch.cuda.empty_cache()
