"""Host-side checks of the C-ABI library (no GPU): it loads, exports every entry point the
header declares, derives the same constants as the oracle, lays out the arena sanely, uses
the same population order, and rejects invalid parameters without launching anything."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle import oracle as O
from paper_1512_08042_gb300 import binding as B
from paper_1512_08042_gb300 import build as BUILD
from paper_1512_08042_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    BUILD.build()
    return B.lib()


def declared_functions():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*([a-z_][a-z0-9_]*)\s*\(",
                                src, flags=re.M)
    return sorted(set(names))


def test_library_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
    assert set(B.EXPORTS) <= set(names)


@pytest.mark.parametrize("name", sorted(W.WORKLOADS))
def test_derived_constants_equal_oracle(lib, name):
    cfg = W.WORKLOADS[name]
    a = B.derive(cfg)
    b = O.derive(cfg)
    for k in a:
        assert a[k] == b[k], k  # bit-identical: both follow the same written definitions


def test_lattice_order_matches_oracle(lib):
    for q in (39, 19):
        e1, w1, r1 = B.lattice(q)
        e2, w2, r2 = O.lattice(q)
        assert np.array_equal(e1, e2)
        assert np.array_equal(w1, w2)
        assert r1 == r2


def test_layout_is_aligned_and_disjoint(lib):
    cfg = W.WORKLOADS["poiseuille_64x256_ppc50_fp32"]
    L = B.layout(cfg)
    d = B.derive(cfg)
    rb = 4
    assert d["bin"] == 128 and d["capacity"] == 64 * 256 * 128
    regions = []
    for h in range(2):
        regions.append((L.part[h], 8 * rb * d["capacity"]))  # records of 8 Real per particle
        regions.append((L.f[h], d["q"] * d["nnodes"] * rb))
        regions.append((L.count[h], 4 * d["ncells"]))
    for k, sz in (("acc", 160 * d["ncells"]),
                  ("crmax", rb * d["ncells"]), ("rem", rb * d["ncells"]),
                  ("nbar_sum", 4 * d["ncells"]), ("ctrl", 64), ("counters", 128),
                  ("map_scratch", 176 * d["ncells"]), ("coupled", d["ncells"])):
        regions.append((getattr(L, k), sz))
    regions.sort()
    for (o1, s1), (o2, _) in zip(regions, regions[1:]):
        assert o1 % 256 == 0
        assert o1 + s1 <= o2
    assert regions[-1][0] + regions[-1][1] <= L.total_bytes


def test_invalid_parameters_are_rejected(lib):
    good = W.config(ncx=8, ncy=2, ppc=5, seed=1)
    B.derive(good)
    for bad in (dict(ncx=5), dict(lattice=27), dict(real_bytes=2), dict(lb_ratio=3),
                dict(kn=0.0), dict(sample_every=0), dict(capacity_factor=0.5), dict(ppc=0),
                dict(ppc=200), dict(accum_mode=1), dict(accum_mode=2)):
        # accum_mode 1 (Kahan-compensated FP32 sums) is not built: only FP64 sums are
        cfg = dict(good)
        cfg.update(bad)
        with pytest.raises(B.HybError) as ei:
            B.derive(cfg)
        assert ei.value.status == B.HYB_EINVAL
    p = B.make_params(good)
    p.abi_version = 99
    d = B.HybDerived()
    assert lib.hyb_derive(ctypes.byref(p), ctypes.byref(d)) == B.HYB_EINVAL
    # null arguments
    assert lib.dsmc_step(None, 1) == B.HYB_EINVAL
    assert lib.map_lbm_to_dsmc(None, None, 1) == B.HYB_EINVAL
    assert lib.hyb_hybrid_step_host(None, None, 0, None, 0, None, None) == B.HYB_EINVAL
    assert lib.hyb_hybrid_steps_host(None, 2, None, 0, None, 0, None, None) == B.HYB_EINVAL
    assert lib.hyb_host_wait(None, 0) == B.HYB_EINVAL
    assert lib.map_dsmc_to_lbm_adjoint(None, None, 1, None, None) == B.HYB_EINVAL
    assert lib.lbm_adjoint_step(None, None, None, None, None, None, None, None, None) == B.HYB_EINVAL
    assert lib.lbm_steps_nodes(None, None, None, None, None, 4, 2, None) == B.HYB_EINVAL
    assert lib.lbm_adjoint_segment(None, None, None, 2, None, None, None, None, None, None,
                                   None) == B.HYB_EINVAL


def test_batch_layout_places_replicas_and_tables(lib):
    cfgs = [W.config(ncx=40, ncy=1, ppc=30, seed=1), W.config(ncx=13, ncy=8, ppc=23, lb_ratio=2, seed=2)]
    params = (B.HybParams * 2)(*[B.make_params(c) for c in cfgs])
    off = (ctypes.c_uint64 * 4)()
    assert lib.hyb_batch_layout(params, 2, off) == B.HYB_OK
    sizes = [B.layout(c).total_bytes for c in cfgs]
    assert off[0] == 0 and off[1] >= sizes[0] and off[1] % 256 == 0
    assert off[2] >= off[1] + sizes[1] and off[2] % 256 == 0 and off[3] > off[2]
    mixed = [cfgs[0], dict(cfgs[1], real_bytes=8)]
    params = (B.HybParams * 2)(*[B.make_params(c) for c in mixed])
    assert lib.hyb_batch_layout(params, 2, off) == B.HYB_EINVAL
    assert lib.hyb_batch_layout(params, 0, off) == B.HYB_EINVAL


@pytest.mark.parametrize("ncz", [0, 1, 2, 5])
def test_3d_derive_and_layout(lib, ncz):
    # ncz < 2 is the slab; ncz >= 2 adds ncz * lb_ratio LB layers and the z positions
    cfg = W.config(ncx=12, ncy=4, ppc=30, lb_ratio=2, ncz=ncz, real_bytes=8)
    a, b = B.derive(cfg), O.derive(cfg)
    for k in a:
        assert a[k] == b[k], k
    three_d = ncz >= 2
    assert a["ncells"] == 12 * 4 * (ncz if three_d else 1)
    assert a["nz"] == (2 * ncz if three_d else 1)
    assert a["nnodes"] == 24 * 8 * a["nz"]
    L = B.layout(cfg)
    # z lives in the particle records (slot 5) in 3D and the slab alike: the record arrays
    # and populations are disjoint and inside the arena
    regions = sorted([(L.part[h], 8 * 8 * a["capacity"]) for h in range(2)] +
                     [(L.f[h], 8 * a["q"] * a["nnodes"]) for h in range(2)])
    for (o1, s1), (o2, _) in zip(regions, regions[1:]):
        assert o1 % 256 == 0 and o1 + s1 <= o2
    assert regions[-1][0] + regions[-1][1] <= L.total_bytes


def test_3d_restrictions_are_rejected(lib):
    cfg3 = W.config(ncx=8, ncy=2, ppc=5, ncz=2, seed=1)
    B.derive(cfg3)
    with pytest.raises(B.HybError) as ei:
        B.derive(dict(cfg3, ncz=-1))
    assert ei.value.status == B.HYB_EINVAL
    # a batch is for slabs only
    params = (B.HybParams * 2)(*[B.make_params(c) for c in (cfg3, cfg3)])
    off = (ctypes.c_uint64 * 4)()
    assert lib.hyb_batch_layout(params, 2, off) == B.HYB_EINVAL


@pytest.mark.parametrize("ncz", [0, 3])
def test_population_shape_check_uses_the_lattice_shape(lib, ncz):
    # the shape every population argument must have: [q][ny][nx] for the slab and
    # [q][nz][ny][nx] in 3D, formed from the derived constants alone (no device memory)
    cfg = W.config(ncx=8, ncy=3, ppc=5, lb_ratio=2, ncz=ncz, seed=1)
    h = B.Hybrid.__new__(B.Hybrid)
    h.d = B.derive(cfg)
    want = (39, 6, 16) if ncz < 2 else (39, 6, 6, 16)
    assert h._pop_shape() == want
    assert h.wall_scratch_size() == 2 * 6 * (6 if ncz >= 2 else 1) + 1


def test_streamwise_slab_derive_layout_and_limits(lib):
    # a slab of rows [4, 12) of a 20-row channel: the channel's constants, yh ghost rows on
    # each side of its LB rows, two send and two receive buffers of xcap particles each
    cfg = W.config(ncx=10, ncy=8, ppc=20, lb_ratio=2, seed=3, ncy_global=20, y0=4)
    whole = W.config(ncx=10, ncy=20, ppc=20, lb_ratio=2, seed=3)
    a, b, w = B.derive(cfg), O.derive(cfg), B.derive(whole)
    for k in a:
        assert a[k] == b[k], k
    for k in ("tau", "dt", "lam", "coll_dt", "g_step", "bin"):
        assert a[k] == w[k], k
    assert a["yh"] == 3 and a["ny"] == 8 * 2 + 6 and a["xcap"] == 10 * a["bin"]
    L = B.layout(cfg)
    xb = 256 + a["xcap"] * (8 * 4 + 4)
    assert L.xbytes == xb
    regions = sorted([(L.xsend[d], xb) for d in range(2)] + [(L.xrecv[d], xb) for d in range(2)] +
                     [(L.part[h], 32 * a["capacity"]) for h in range(2)] +
                     [(L.f[h], 4 * a["q"] * a["nnodes"]) for h in range(2)])
    for (o1, s1), (o2, _) in zip(regions, regions[1:]):
        assert o1 % 256 == 0 and o1 + s1 <= o2
    assert regions[-1][0] + regions[-1][1] <= L.total_bytes
    d19 = B.derive(dict(cfg, lattice=19))
    assert d19["yh"] == 1 and B.derive(whole)["yh"] == 0 and B.layout(whole).xbytes == 0
    for bad in (dict(y0=13), dict(ncy=3), dict(y0=-1), dict(ncy_global=-2)):
        with pytest.raises(B.HybError):
            B.derive(dict(cfg, **bad))
    with pytest.raises(B.HybError):
        B.derive(dict(whole, y0=2))  # y0 without a channel to cut
    # a batch holds whole channels only
    params = (B.HybParams * 2)(B.make_params(cfg), B.make_params(cfg))
    off = (ctypes.c_uint64 * 4)()
    assert lib.hyb_batch_layout(params, 2, off) == B.HYB_EINVAL
