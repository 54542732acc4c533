"""map_lbm_to_dsmc_noalloc through the C ABI: the entry point for callers that cannot give
the library device memory beyond its state (a host application whose allocator owns the
whole GPU budget, or a loop that may not allocate) must produce exactly what the allocating
map_lbm_to_dsmc produces, call after call, and reject lists longer than its fixed scratch.

Collected last on purpose, so that a run stopping at its first failure has run every other
test before this one."""
import ctypes

import numpy as np
import pytest

from oracle import oracle as O
from paper_1512_08042_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1512_08042_gb300 import binding as B  # noqa: E402
from paper_1512_08042_gb300 import build as BUILD  # noqa: E402

BUILD.build()


def _state(h):
    h.sync()
    out = {k: v.cpu().numpy() for k, v in h.particles().items()}
    out["counts"] = h.counts().cpu().numpy()
    out["counters"] = h.counters()
    out["status"] = h.sync_status()
    return out


def _same(a, b):
    assert np.array_equal(a["counts"], b["counts"])
    for k in ("x", "y", "vx", "vy", "vz"):
        assert np.array_equal(a[k], b[k]), k
    assert a["counters"] == b["counters"]
    assert a["status"] == b["status"] == (B.HYB_OK, 0)


@pytest.mark.parametrize("real_bytes,lb_ratio", [(4, 2), (8, 1)])
def test_noalloc_equals_allocating_entry_point_on_two_calls(real_bytes, lb_ratio):
    cfg = W.config(ncx=13, ncy=7, ppc=23, real_bytes=real_bytes, lb_ratio=lb_ratio, seed=17)
    ref = B.Hybrid(cfg)
    na = B.Hybrid(cfg)
    e, w, r = O.lattice(39)
    f0 = W.gen_populations(w, ref.d["nnodes"], seed=9, eps=0.08, rho_eps=0.2)
    f0 = torch.from_numpy(f0.astype(np.float32 if real_bytes == 4 else np.float64))
    for h in (ref, na):
        h.dsmc_step(1)
        h.sync()
        h.f().copy_(f0.view(h.f().shape))
    torch.cuda.synchronize()
    lists = [np.array([0, 5, 12, 13, 40, 90], np.int32), np.array([3, 4, 88, 7], np.int32)]
    for call, cells in enumerate(lists):
        dc = torch.from_numpy(cells).cuda()
        torch.cuda.synchronize()
        ref.map_lbm_to_dsmc(dc)
        # the new entry point, called directly through the C ABI
        rc = B.lib().map_lbm_to_dsmc_noalloc(na.ctx, ctypes.c_void_p(dc.data_ptr()), dc.numel())
        assert rc == B.HYB_OK
        _same(_state(ref), _state(na))
        assert ref.counters()["created"] > 0
        # the next call regenerates from a moved state
        ref.dsmc_step(1)
        na.dsmc_step(1)
        _same(_state(ref), _state(na))


def test_noalloc_rejects_lists_beyond_its_scratch():
    cfg = W.config(ncx=96, ncy=48, ppc=4, seed=2)
    h = B.Hybrid(cfg)
    n = B.NOALLOC_MAX_CELLS + 1
    cells = torch.arange(n, dtype=torch.int32, device="cuda")
    before = _state(h)
    rc = B.lib().map_lbm_to_dsmc_noalloc(h.ctx, ctypes.c_void_p(cells.data_ptr()), n)
    assert rc == B.HYB_EINVAL
    assert b"HYB_NOALLOC_MAX_CELLS" in B.lib().hyb_last_error(h.ctx)
    after = _state(h)
    assert np.array_equal(before["counts"], after["counts"])


def test_noalloc_3d_and_a_full_scratch_allocate_nothing():
    # a 3D channel (the mappings over the cell's r^3 nodes) and a list of exactly
    # HYB_NOALLOC_MAX_CELLS cells, the largest the fixed scratch holds: results equal the
    # allocating entry point's, and after a warm-up call neither torch's caching allocator
    # nor the device's free memory changes across a call
    cfg = W.config(ncx=64, ncy=32, ncz=2, ppc=6, lb_ratio=2, real_bytes=4, seed=21,
                   capacity_factor=3.0)
    ref = B.Hybrid(cfg)
    na = B.Hybrid(cfg)
    n = B.NOALLOC_MAX_CELLS
    assert ref.L.ncells == n
    e, w, r = O.lattice(39)
    f0 = W.gen_populations(w, ref.d["nnodes"], seed=4, eps=0.05, rho_eps=0.1).astype(np.float32)
    for h in (ref, na):
        h.f().copy_(torch.from_numpy(f0).view(h.f().shape))
    cells = torch.arange(n, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()

    def noalloc():
        return B.lib().map_lbm_to_dsmc_noalloc(na.ctx, ctypes.c_void_p(cells.data_ptr()), n)

    ref.map_lbm_to_dsmc(cells)
    assert noalloc() == B.HYB_OK  # warm-up: the first call looks up the scratch address
    _same(_state(ref), _state(na))
    for h in (ref, na):
        h.dsmc_step(1)
    torch.cuda.synchronize()
    stats0 = torch.cuda.memory_stats()
    free0, _ = torch.cuda.mem_get_info()
    ref.map_lbm_to_dsmc(cells)
    assert noalloc() == B.HYB_OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    stats1 = torch.cuda.memory_stats()
    assert free1 == free0
    for k in ("allocation.all.allocated", "segment.all.allocated", "reserved_bytes.all.current"):
        assert stats1.get(k, 0) == stats0.get(k, 0), k
    _same(_state(ref), _state(na))
    assert ref.counters()["created"] > 0
