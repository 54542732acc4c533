"""Host-side input builders (no GPU): the coupling sites of slab and 3D channels, and the
interface-loss targets sampled from DSMC cumulative sums."""
import numpy as np

from oracle import oracle as O
from paper_1512_08042_gb300 import workloads as W


def test_grad_targets_from_sums_are_the_particles_central_moments():
    # one sample: the sums are those of the cell's particles, so the targets must be rho =
    # N / ppc, the mean velocity, the comoving second moments minus the identity and the
    # comoving third moments of those particles
    cfg = W.config(ncx=8, ncy=2, ppc=100, real_bytes=8, kn=0.1, ma=0.3, seed=3)
    o = O.Oracle(cfg)
    o.dsmc_step(1)
    S = o.scalars()["nsamples"]
    assert S == 1
    cells = np.arange(16)
    t = W.grad_targets_from_sums(o.acc(), S, cfg["ppc"], cells)
    p = o.particles()
    cs = o.get(O.A_CELL_START).astype(np.int64)
    pairs = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]
    triples = [(0, 0, 0), (0, 0, 1), (0, 0, 2), (0, 1, 1), (0, 1, 2), (0, 2, 2), (1, 1, 1),
               (1, 1, 2), (1, 2, 2), (2, 2, 2)]
    for c in cells:
        v = np.stack([p[k][cs[c]:cs[c + 1]] for k in ("vx", "vy", "vz")], 1)
        u = v.mean(0)
        w = v - u
        want = [len(v) / cfg["ppc"], *u]
        want += [(w[:, i] * w[:, j]).mean() - (1.0 if i == j else 0.0) for i, j in pairs]
        want += [(w[:, i] * w[:, j] * w[:, k]).mean() for i, j, k in triples]
        assert np.allclose(t[c], want, rtol=0, atol=1e-13), c


def test_coupling_sites_3d_repeat_the_slab_sites_in_every_layer():
    for r in (1, 2):
        cfg2 = W.config(ncx=16, ncy=8, lb_ratio=r)
        cfg3 = dict(cfg2, ncz=3)
        n2, c2 = W.coupling_sites(cfg2)
        n3, c3 = W.coupling_sites(cfg3)
        nx, ny = 16 * r, 8 * r
        assert len(n3) == 3 * r * len(n2) and len(c3) == 3 * len(c2)
        assert np.array_equal(n3[:len(n2)], n2) and np.array_equal(c3[:len(c2)], c2)
        assert n3.max() < nx * ny * 3 * r and c3.max() < 16 * 8 * 3
        # every mapped node lies in a mapped cell
        z, y, x = n3 // (nx * ny), (n3 // nx) % ny, n3 % nx
        cell = ((z // r) * 8 + y // r) * 16 + x // r
        assert set(cell.tolist()) <= set(c3.tolist())
        assert len(np.unique(n3)) == len(n3)
