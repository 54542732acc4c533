"""Thin ctypes binding of libdsmclbm.so (C ABI in include/dsmclbm.h).

Only argument marshalling lives here: PyTorch allocates the device arena and provides the
stream; every step of the method runs in the library's CUDA kernels. There is no CPU
fallback: if the library is missing or cannot be loaded, `lib()` raises.
"""
import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_build", "libdsmclbm.so")
ABI_VERSION = 12

HYB_OK, HYB_EINVAL, HYB_ENOMEM, HYB_ECUDA, HYB_ECAPACITY, HYB_ETIMEOUT, HYB_ESAMPLING, HYB_ESTATE = range(8)
ST_CAPACITY, ST_BOUNCE_CAP, ST_SCATTER_CAP, ST_SAMPLING_CAP, ST_CELL_OVERFLOW, ST_BAD_INPUT = (
    1, 2, 4, 8, 16, 32)
COUNTER_NAMES = ["wall_hits", "candidates", "collisions", "created", "deleted",
                 "l2d_attempts", "envelope", "bounce_cap"]
KERNELS = {"move": 0, "collide": 1, "lbm": 2, "dsmc2lb": 3, "lb2dsmc": 4, "fused": 5}
CTRL_STATUS, CTRL_NTOT, CTRL_STEP, CTRL_NSAMPLES = 0, 1, 2, 3
NOALLOC_MAX_CELLS = 4096

_u32, _i32, _i64, _u64, _dbl, _vp = (ctypes.c_uint32, ctypes.c_int32, ctypes.c_int64,
                                     ctypes.c_uint64, ctypes.c_double, ctypes.c_void_p)


class HybParams(ctypes.Structure):
    _fields_ = [("abi_version", _u32), ("ncx", _i32), ("ncy", _i32), ("lb_ratio", _i32),
                ("ppc", _i32), ("lattice", _i32), ("real_bytes", _i32), ("sample_every", _i32),
                ("seed", _u64), ("kn", _dbl), ("ma", _dbl), ("crmax_init", _dbl),
                ("capacity_factor", _dbl), ("T_K", _dbl), ("mass_kg", _dbl),
                ("lb_collision", _i32), ("d2l_mode", _i32), ("kn_profile", _i32),
                ("pad0", _i32), ("kn_end", _dbl), ("ncz", _i32), ("accum_mode", _i32),
                ("ncy_global", _i32), ("y0", _i32)]


class HybDerived(ctypes.Structure):
    _fields_ = [("r_lat", _dbl), ("cs_lat", _dbl), ("H_lat", _dbl), ("tau", _dbl), ("dt", _dbl),
                ("lam", _dbl), ("coll_dt", _dbl), ("g_step", _dbl), ("c_th_ms", _dbl),
                ("ncells", _i64), ("nx", _i64), ("ny", _i64), ("nnodes", _i64),
                ("capacity", _i64), ("q", _i32), ("order", _i32), ("bin", _i32), ("pad", _i32),
                ("nz", _i64), ("ncz", _i64), ("yh", _i64), ("xcap", _i64)]


class HybLayout(ctypes.Structure):
    _fields_ = [("total_bytes", _u64), ("capacity", _i64), ("ncells", _i64), ("nnodes", _i64),
                ("q", _i32), ("real_bytes", _i32), ("bin", _i32), ("pad", _i32),
                ("part", _u64 * 2), ("count", _u64 * 2), ("crmax", _u64),
                ("rem", _u64), ("nbar_sum", _u64), ("acc", _u64), ("f", _u64 * 2),
                ("ctrl", _u64), ("counters", _u64), ("map_scratch", _u64), ("coupled", _u64),
                ("coll_cell", _u64), ("tau_node", _u64), ("xsend", _u64 * 2),
                ("xrecv", _u64 * 2), ("xbytes", _u64)]


EXPORTS = ["hyb_derive", "hyb_layout_compute", "hyb_lattice", "hyb_status_string", "dsmc_init",
           "dsmc_step", "dsmc_move", "dsmc_merge", "dsmc_collide", "lbm_halo_size", "lbm_halo_pack",
           "lbm_halo_unpack", "lbm_step", "sample_moments", "map_dsmc_to_lbm", "map_lbm_to_dsmc",
           "map_lbm_to_dsmc_noalloc", "map_dsmc_to_lbm_adjoint", "lbm_step_nodes", "lbm_interface_loss", "lbm_adjoint_step",
           "lbm_steps_nodes", "lbm_adjoint_segment",
           "hyb_hybrid_step", "hyb_hybrid_step_host", "hyb_hybrid_steps_host", "hyb_host_wait", "hyb_batch_layout", "hyb_batch_init", "hyb_batch_replica",
           "hyb_batch_hybrid_step", "hyb_batch_set_blocks", "hyb_batch_set_block", "hyb_batch_get_block",
           "hyb_batch_tune",
           "hyb_batch_last_error", "hyb_batch_destroy", "hyb_current", "hyb_sync_status", "hyb_read_counters",
           "hyb_set_fuse", "hyb_set_collide_block", "hyb_get_collide_block", "hyb_tune_collide",
           "hyb_profile", "hyb_profile_harvest", "hyb_profile_read", "hyb_debug_philox",
           "hyb_last_error", "hyb_destroy"]

_LIB = None


class HybError(RuntimeError):
    def __init__(self, status, msg=""):
        self.status = status
        super().__init__("%s (status %d)%s" % (_status_str(status), status,
                                               (": " + msg) if msg else ""))


def _status_str(s):
    try:
        return lib().hyb_status_string(s).decode()
    except Exception:
        return "status"


def lib():
    """Load libdsmclbm.so; raise if it has not been built."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libdsmclbm.so is not built (%s); run __graft_entry__.build()" % LIB_PATH)
    L = ctypes.CDLL(LIB_PATH)
    P = ctypes.POINTER
    L.hyb_derive.argtypes = [P(HybParams), P(HybDerived)]
    L.hyb_layout_compute.argtypes = [P(HybParams), P(HybLayout)]
    L.hyb_lattice.argtypes = [_i32, _vp, _vp, P(_dbl)]
    L.hyb_status_string.argtypes = [ctypes.c_int]
    L.hyb_status_string.restype = ctypes.c_char_p
    L.dsmc_init.argtypes = [P(HybParams), _vp, _u64, _vp, P(_vp)]
    L.dsmc_step.argtypes = [_vp, _i32]
    L.dsmc_move.argtypes = [_vp]
    L.dsmc_merge.argtypes = [_vp]
    L.dsmc_collide.argtypes = [_vp]
    L.lbm_halo_size.argtypes = [_vp, P(_i64)]
    L.lbm_halo_pack.argtypes = [_vp, _i32, _vp]
    L.lbm_halo_unpack.argtypes = [_vp, _i32, _vp]
    L.lbm_step.argtypes = [_vp, _i32]
    L.sample_moments.argtypes = [_vp, _vp, _i32]
    L.map_dsmc_to_lbm.argtypes = [_vp, _vp, _i32]
    L.map_lbm_to_dsmc.argtypes = [_vp, _vp, _i32]
    L.map_lbm_to_dsmc_noalloc.argtypes = [_vp, _vp, _i32]
    L.map_dsmc_to_lbm_adjoint.argtypes = [_vp, _vp, _i32, _vp, _vp]
    L.lbm_step_nodes.argtypes = [_vp, _vp, _vp, _vp, _vp]
    L.lbm_interface_loss.argtypes = [_vp, _vp, _vp, _i32, _vp, _vp, _vp]
    L.lbm_adjoint_step.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]
    L.lbm_steps_nodes.argtypes = [_vp, _vp, _vp, _vp, _vp, _i32, _i32, _vp]
    L.lbm_adjoint_segment.argtypes = [_vp, _vp, _vp, _i32, _vp, _vp, _vp, _vp, _vp, _vp, _vp]
    L.hyb_hybrid_step.argtypes = [_vp, _vp, _i32, _vp, _i32, _i32, _i32]
    L.hyb_hybrid_step_host.argtypes = [_vp, _vp, _i32, _vp, _i32, _vp, _vp]
    L.hyb_hybrid_steps_host.argtypes = [_vp, _i32, _vp, _i32, _vp, _i32, _vp, _vp]
    L.hyb_host_wait.argtypes = [_vp, _i32]
    L.hyb_batch_layout.argtypes = [_vp, _i32, _vp]
    L.hyb_batch_init.argtypes = [_vp, _i32, _vp, _u64, _vp, P(_vp)]
    L.hyb_batch_replica.argtypes = [_vp, _i32, P(_vp)]
    L.hyb_batch_hybrid_step.argtypes = [_vp, _vp, _vp, _vp, _vp, _i32, _i32]
    L.hyb_batch_set_blocks.argtypes = [_vp, _i32, _i32]
    L.hyb_batch_set_block.argtypes = [_vp, _i32, _i32]
    L.hyb_batch_get_block.argtypes = [_vp, _i32]
    L.hyb_batch_get_block.restype = _i32
    L.hyb_batch_tune.argtypes = [_vp, _vp, _vp, _vp, _vp, P(_i32), P(_i32)]
    L.hyb_batch_last_error.argtypes = [_vp]
    L.hyb_batch_last_error.restype = ctypes.c_char_p
    L.hyb_batch_destroy.argtypes = [_vp]
    L.hyb_current.argtypes = [_vp, P(_i32), P(_i32)]
    L.hyb_set_fuse.argtypes = [_vp, _i32]
    L.hyb_set_collide_block.argtypes = [_vp, _i32]
    L.hyb_get_collide_block.argtypes = [_vp]
    L.hyb_get_collide_block.restype = _i32
    L.hyb_tune_collide.argtypes = [_vp, _vp, _i32, _vp, _i32, P(_i32), P(_i32)]
    L.hyb_sync_status.argtypes = [_vp, P(_u32)]
    L.hyb_read_counters.argtypes = [_vp, _vp]
    L.hyb_profile.argtypes = [_vp, _i32]
    L.hyb_profile_harvest.argtypes = [_vp]
    L.hyb_profile_read.argtypes = [_vp, P(_dbl), P(_i64)]
    L.hyb_debug_philox.argtypes = [_vp, _u64, _vp, _i64, _vp]
    L.hyb_last_error.argtypes = [_vp]
    L.hyb_last_error.restype = ctypes.c_char_p
    L.hyb_destroy.argtypes = [_vp]
    L.hyb_destroy.restype = None
    _LIB = L
    return L


def make_params(cfg):
    p = HybParams()
    p.abi_version = ABI_VERSION
    for name, _ in HybParams._fields_:
        if name != "abi_version" and name in cfg:
            setattr(p, name, cfg[name])
    return p


def _check(rc, ctx=None):
    if rc != HYB_OK:
        msg = lib().hyb_last_error(ctx).decode() if ctx else ""
        raise HybError(rc, msg)


def derive(cfg):
    d = HybDerived()
    _check(lib().hyb_derive(ctypes.byref(make_params(cfg)), ctypes.byref(d)))
    return {n: getattr(d, n) for n, _ in HybDerived._fields_}


def layout(cfg):
    L = HybLayout()
    _check(lib().hyb_layout_compute(ctypes.byref(make_params(cfg)), ctypes.byref(L)))
    return L


def lattice(q):
    e = np.zeros((q, 3), np.int32)
    w = np.zeros(q, np.float64)
    r = ctypes.c_double()
    _check(lib().hyb_lattice(q, e.ctypes.data_as(_vp), w.ctypes.data_as(_vp), ctypes.byref(r)))
    return e, w, r.value


def debug_philox(ctr_dev, seed, out_dev, stream_ptr=0):
    """Philox4x32-10 of device u32 counters [n, 4] into out_dev [n, 4] (torch tensors)."""
    n = ctr_dev.numel() // 4
    _check(lib().hyb_debug_philox(ctr_dev.data_ptr(), seed, out_dev.data_ptr(), n, stream_ptr))


class Hybrid:
    """One channel: DSMC particles, LB populations and the mappings, on one GPU.

    The state lives in a torch uint8 arena on `device`; the library launches on `stream`
    (a dedicated torch.cuda.Stream by default). Methods enqueue work and return; use
    `sync()` (or a synchronising call) before reading views from another stream.
    """

    def __init__(self, cfg, device="cuda:0", stream=None):
        import torch
        self.torch = torch
        self.cfg = dict(cfg)
        self.device = torch.device(device)
        self.params = make_params(cfg)
        self.d = derive(cfg)
        self.L = layout(cfg)
        self.real = torch.float32 if cfg["real_bytes"] == 4 else torch.float64
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.Stream(self.device)
            self.arena = torch.zeros(int(self.L.total_bytes), dtype=torch.uint8, device=self.device)
        torch.cuda.synchronize(self.device)
        ctx = _vp()
        with torch.cuda.device(self.device):
            rc = lib().dsmc_init(ctypes.byref(self.params), self.arena.data_ptr(),
                                 int(self.L.total_bytes), self.stream.cuda_stream, ctypes.byref(ctx))
        _check(rc)
        self.ctx = ctx

    @classmethod
    def _attach(cls, cfg, device, stream, ctx, arena):
        """A view of a context owned elsewhere (a replica of a Batch): no allocation, and
        close() leaves the context to its owner."""
        import torch
        self = cls.__new__(cls)
        self.torch = torch
        self.cfg = dict(cfg)
        self.device = torch.device(device)
        self.params = make_params(cfg)
        self.d = derive(cfg)
        self.L = layout(cfg)
        self.real = torch.float32 if cfg["real_bytes"] == 4 else torch.float64
        self.stream = stream
        self.arena = arena
        self.ctx = ctx
        self._owned = False
        return self

    def close(self):
        if getattr(self, "ctx", None):
            if getattr(self, "_owned", True):
                lib().hyb_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- steps -------------------------------------------------------------------------
    def _inputs(self, *tensors):
        """Order the library's stream after the torch stream that produced `tensors`, and
        keep their memory from being reused before the library's work on them is done."""
        torch = self.torch
        self.stream.wait_stream(torch.cuda.current_stream(self.device))
        for t in tensors:
            if t is not None:
                t.record_stream(self.stream)

    def dsmc_step(self, n=1):
        _check(lib().dsmc_step(self.ctx, n), self.ctx)

    def lbm_step(self, n=1):
        _check(lib().lbm_step(self.ctx, n), self.ctx)

    # -- a streamwise slab (cfg["ncy_global"] > 0): the split DSMC step and the LB ghost rows --
    def dsmc_move(self):
        _check(lib().dsmc_move(self.ctx), self.ctx)

    def dsmc_merge(self):
        _check(lib().dsmc_merge(self.ctx), self.ctx)

    def dsmc_collide(self):
        _check(lib().dsmc_collide(self.ctx), self.ctx)

    def xfer(self, which, d):
        """The exchange buffer `which` ("send" or "recv") of direction d as a uint8 view."""
        off = (self.L.xsend if which == "send" else self.L.xrecv)[d]
        return self.arena[int(off):int(off) + int(self.L.xbytes)]

    def halo_size(self):
        n = ctypes.c_int64()
        _check(lib().lbm_halo_size(self.ctx, ctypes.byref(n)), self.ctx)
        return n.value

    def halo_pack(self, side, buf):
        _check(lib().lbm_halo_pack(self.ctx, int(side), buf.data_ptr()), self.ctx)

    def halo_unpack(self, side, buf):
        self._inputs(buf)
        _check(lib().lbm_halo_unpack(self.ctx, int(side), buf.data_ptr()), self.ctx)

    def f_rows(self, half=None):
        """The populations of the context's own LB rows (a slab's ghost rows left out)."""
        yh = int(self.d["yh"])
        f = self.f(half)
        if yh == 0:
            return f
        return f[..., yh:f.shape[-2] - yh, :]

    def map_dsmc_to_lbm(self, nodes):
        self._inputs(nodes)
        _check(lib().map_dsmc_to_lbm(self.ctx, nodes.data_ptr(), nodes.numel()), self.ctx)

    def map_lbm_to_dsmc(self, cells):
        self._inputs(cells)
        _check(lib().map_lbm_to_dsmc(self.ctx, cells.data_ptr(), cells.numel()), self.ctx)

    def map_lbm_to_dsmc_noalloc(self, cells):
        """map_lbm_to_dsmc with its scratch in the library's fixed device array (for callers
        that cannot give the library device memory beyond the state; at most
        NOALLOC_MAX_CELLS cells per call)."""
        self._inputs(cells)
        _check(lib().map_lbm_to_dsmc_noalloc(self.ctx, cells.data_ptr(), cells.numel()), self.ctx)

    # -- differentiated LBM (per-node g and tau, adjoint, interface loss) ----------------
    def _pop_shape(self):
        # from the derived constants: this check runs on every step call, so it builds no view
        q, ny, nx, nz = (int(self.d[k]) for k in ("q", "ny", "nx", "nz"))
        return (q, nz, ny, nx) if int(self.d["ncz"]) >= 2 else (q, ny, nx)

    def _check_pop(self, *ts):
        for t in ts:
            if tuple(t.shape) != self._pop_shape() or t.dtype != self.real or not t.is_contiguous():
                raise ValueError("populations must be contiguous %s %s" % (self._pop_shape(), self.real))

    def _check_node(self, *ts):
        n = int(self.d["nnodes"])
        for t in ts:
            if t.numel() != n or t.dtype != self.real or not t.is_contiguous():
                raise ValueError("per-node arrays must be contiguous, %d values of %s" % (n, self.real))

    def lbm_step_nodes(self, f_src, f_dst, g, tau):
        """One LB step f_dst = LB(f_src) with per-node force increment g and relaxation time
        tau (the context's own populations are not touched)."""
        self._check_pop(f_src, f_dst)
        self._check_node(g, tau)
        self._inputs(f_src, f_dst, g, tau)
        _check(lib().lbm_step_nodes(self.ctx, f_src.data_ptr(), f_dst.data_ptr(), g.data_ptr(),
                                    tau.data_ptr()), self.ctx)

    def lbm_interface_loss(self, f, nodes, targets, loss, lam):
        """Adds the interface loss of f at `nodes` (int32) against `targets` (n x 20) to
        `loss` (one float64) and dL/df at those nodes to `lam`."""
        self._check_pop(f, lam)
        if targets.dtype != self.real or targets.numel() != 20 * nodes.numel():
            raise ValueError("20 targets per node in the state precision")
        if nodes.dtype != self.torch.int32 or loss.dtype != self.torch.float64:
            raise ValueError("int32 nodes and a float64 loss")
        self._inputs(f, nodes, targets, loss, lam)
        _check(lib().lbm_interface_loss(self.ctx, f.data_ptr(), nodes.data_ptr(), nodes.numel(),
                                        targets.data_ptr(), loss.data_ptr(), lam.data_ptr()),
               self.ctx)

    def wall_scratch_size(self):
        """Values of the adjoint's wall scratch: two sums per streamwise row (y, z), a ticket."""
        return 2 * int(self.d["ny"]) * int(self.d["nz"]) + 1

    def map_dsmc_to_lbm_adjoint(self, nodes, lam, grad_acc):
        """Adds dL/d(acc) to grad_acc (float64 [ncells, 20]) from lam = dL/df after
        map_dsmc_to_lbm at `nodes` (distinct int32), and zeroes lam at those nodes."""
        self._check_pop(lam)
        torch = self.torch
        if nodes.dtype != torch.int32 or grad_acc.dtype != torch.float64 or \
                grad_acc.numel() != 20 * int(self.L.ncells) or not grad_acc.is_contiguous():
            raise ValueError("int32 nodes and a contiguous float64 [ncells, 20] gradient")
        self._inputs(nodes, lam, grad_acc)
        _check(lib().map_dsmc_to_lbm_adjoint(self.ctx, nodes.data_ptr(), nodes.numel(),
                                             lam.data_ptr(), grad_acc.data_ptr()), self.ctx)

    def lbm_adjoint_step(self, f, lam_next, lam, g, tau, grad_g, grad_tau, wall):
        """lam = dL/df_t from f_t and lam_next = dL/df_{t+1}; adds this step's dL/dg and
        dL/dtau to grad_g and grad_tau. wall: 2 ny nz + 1 zeros, left zero."""
        self._check_pop(f, lam_next, lam)
        self._check_node(g, tau, grad_g, grad_tau)
        if wall.numel() != self.wall_scratch_size() or wall.dtype != self.real:
            raise ValueError("wall scratch: 2 ny nz + 1 values in the state precision")
        self._inputs(f, lam_next, lam, g, tau, grad_g, grad_tau, wall)
        _check(lib().lbm_adjoint_step(self.ctx, f.data_ptr(), lam_next.data_ptr(), lam.data_ptr(),
                                      g.data_ptr(), tau.data_ptr(), grad_g.data_ptr(),
                                      grad_tau.data_ptr(), wall.data_ptr()), self.ctx)


    def lbm_steps_nodes(self, f_a, f_b, g, tau, nsteps, ckpt_every=1, ckpt=None):
        """nsteps LB steps alternating between f_a (f_0 on entry) and f_b in one call
        (lbm_steps_nodes); the states f_K, f_2K, ... before the last go to ckpt (a tensor of
        (nsteps - 1) // ckpt_every population arrays, or None when there are none). Returns the
        tensor that holds f_T."""
        self._check_pop(f_a, f_b)
        self._check_node(g, tau)
        nck = (nsteps - 1) // ckpt_every if nsteps > 0 else 0
        if nck > 0 and (ckpt is None or ckpt.dtype != self.real or not ckpt.is_contiguous() or
                        ckpt.numel() < nck * f_a.numel()):
            raise ValueError("ckpt must hold %d contiguous population arrays" % nck)
        self._inputs(f_a, f_b, g, tau, *([ckpt] if ckpt is not None else []))
        _check(lib().lbm_steps_nodes(self.ctx, f_a.data_ptr(), f_b.data_ptr(), g.data_ptr(), tau.data_ptr(),
                                     int(nsteps), int(ckpt_every),
                                     ckpt.data_ptr() if ckpt is not None else None), self.ctx)
        return f_a if nsteps % 2 == 0 else f_b

    def lbm_adjoint_segment(self, state0, states, n, lam_a, lam_b, g, tau, grad_g, grad_tau, wall):
        """The adjoint of n LB steps from state0 in one call (lbm_adjoint_segment): states is
        scratch for n - 1 population arrays (None for n = 1), lam_a holds dL/df at the end of
        the segment on entry. Returns the tensor that holds dL/df at its start."""
        self._check_pop(state0, lam_a, lam_b)
        self._check_node(g, tau, grad_g, grad_tau)
        if n > 1 and (states is None or states.dtype != self.real or not states.is_contiguous() or
                      states.numel() < (n - 1) * state0.numel()):
            raise ValueError("states must hold %d contiguous population arrays" % (n - 1))
        self._inputs(state0, lam_a, lam_b, g, tau, grad_g, grad_tau, wall,
                     *([states] if states is not None else []))
        _check(lib().lbm_adjoint_segment(self.ctx, state0.data_ptr(),
                                         states.data_ptr() if states is not None else None, int(n),
                                         lam_a.data_ptr(), lam_b.data_ptr(), g.data_ptr(), tau.data_ptr(),
                                         grad_g.data_ptr(), grad_tau.data_ptr(), wall.data_ptr()), self.ctx)
        return lam_a if n % 2 == 0 else lam_b
    def hybrid_step(self, nodes=None, cells=None, nsteps=1, use_graph=True, order_inputs=True):
        """`order_inputs=False` skips the stream ordering of `nodes`/`cells` (for callers
        that keep them resident and already ordered, e.g. a timed loop)."""
        if order_inputs:
            self._inputs(nodes, cells)
        np_ = nodes.data_ptr() if nodes is not None else None
        cp_ = cells.data_ptr() if cells is not None else None
        nn = nodes.numel() if nodes is not None else 0
        nc = cells.numel() if cells is not None else 0
        _check(lib().hyb_hybrid_step(self.ctx, np_, nn, cp_, nc, nsteps, 1 if use_graph else 0),
               self.ctx)

    def hybrid_step_host(self, nodes, cells, out_acc, out_status, nsteps=1):
        """Hybrid steps with host lists and host results (hyb_hybrid_step_host for one step,
        hyb_hybrid_steps_host for several, each step copying its lists in and its results out):
        `nodes`, `cells` int32 and `out_acc` float64 [nsteps, len(cells), 20], `out_status`
        int32 [>= nsteps], CPU tensors or arrays (page-locked for asynchronous copies). Returns
        once enqueued; the results are valid after host_wait()."""
        def ptr(a):
            return a.data_ptr() if hasattr(a, "data_ptr") else a.ctypes.data

        def check(a, dtype, n, what):
            if hasattr(a, "data_ptr"):
                ok = (a.device.type == "cpu" and a.is_contiguous() and a.numel() >= n and
                      str(a.dtype) == "torch." + dtype)
            else:
                ok = a.flags["C_CONTIGUOUS"] and a.size >= n and a.dtype == np.dtype(dtype)
            if not ok:
                raise ValueError("%s must be a contiguous host %s buffer of >= %d values" % (what, dtype, n))
        nn, nc = len(nodes), len(cells)
        nsteps = int(nsteps)
        check(nodes, "int32", nn, "nodes")
        check(cells, "int32", nc, "cells")
        check(out_acc, "float64", 20 * nc * nsteps, "out_acc")
        check(out_status, "int32", nsteps, "out_status")
        if nsteps == 1:
            _check(lib().hyb_hybrid_step_host(self.ctx, ptr(nodes) if nn else None, nn,
                                              ptr(cells) if nc else None, nc,
                                              ptr(out_acc) if nc else None, ptr(out_status)), self.ctx)
        else:
            _check(lib().hyb_hybrid_steps_host(self.ctx, nsteps, ptr(nodes) if nn else None, nn,
                                               ptr(cells) if nc else None, nc,
                                               ptr(out_acc) if nc else None, ptr(out_status)), self.ctx)

    def host_wait(self, pending=0):
        """Wait until at most `pending` host steps are in flight (hyb_host_wait)."""
        _check(lib().hyb_host_wait(self.ctx, int(pending)), self.ctx)

    def sample_moments(self, out=None, reset=False):
        self._inputs(out)
        ptr = out.data_ptr() if out is not None else None
        _check(lib().sample_moments(self.ctx, ptr, 1 if reset else 0), self.ctx)

    # -- status ------------------------------------------------------------------------
    def sync(self):
        self.stream.synchronize()

    def sync_status(self):
        bits = _u32()
        rc = lib().hyb_sync_status(self.ctx, ctypes.byref(bits))
        return rc, bits.value

    def counters(self):
        out = np.zeros(16, np.uint64)
        _check(lib().hyb_read_counters(self.ctx, out.ctypes.data_as(_vp)), self.ctx)
        return {n: int(out[i]) for i, n in enumerate(COUNTER_NAMES)}

    def current(self):
        p, f = _i32(), _i32()
        _check(lib().hyb_current(self.ctx, ctypes.byref(p), ctypes.byref(f)))
        return p.value, f.value

    def set_fuse(self, mode):
        """Multi-step calls: "auto" (fuse the DSMC passes when the fused grid fills the GPU),
        "always" or "never"; the results are the same."""
        _check(lib().hyb_set_fuse(self.ctx, {"auto": 0, "always": 1, "never": 2}[mode]))

    def set_collide_block(self, warps):
        """The collide's block shape: 8 warps (32 cells) or 4 (16 cells); the same results."""
        _check(lib().hyb_set_collide_block(self.ctx, int(warps)))

    def collide_block(self):
        return int(lib().hyb_get_collide_block(self.ctx))

    def tune_collide(self, nodes=None, cells=None):
        """Picks the fastest collide block shape and fusion of multi-step calls by timing
        hybrid steps with these coupling lists (device int32 tensors or None); advances the
        context by 192 hybrid steps. Returns (warps, fuse), fuse "always" or "never"."""
        nn = 0 if nodes is None else nodes.numel()
        nc = 0 if cells is None else cells.numel()
        self._inputs(nodes, cells)
        w, f = _i32(), _i32()
        rc = lib().hyb_tune_collide(self.ctx, nodes.data_ptr() if nn else None, nn,
                                    cells.data_ptr() if nc else None, nc, ctypes.byref(w), ctypes.byref(f))
        if rc != HYB_OK:
            raise HybError(rc, lib().hyb_last_error(self.ctx).decode())
        return w.value, {1: "always", 2: "never"}[f.value]

    def profile(self, kernel):
        _check(lib().hyb_profile(self.ctx, KERNELS[kernel] if isinstance(kernel, str) else kernel))

    def profile_harvest(self):
        _check(lib().hyb_profile_harvest(self.ctx), self.ctx)

    def profile_read(self):
        ms, n = _dbl(), _i64()
        _check(lib().hyb_profile_read(self.ctx, ctypes.byref(ms), ctypes.byref(n)))
        return ms.value, n.value

    # -- views into the arena ----------------------------------------------------------
    def _view(self, off, count, dtype):
        torch = self.torch
        esize = torch.empty((), dtype=dtype).element_size()
        return self.arena[int(off):int(off) + int(count) * esize].view(dtype)

    def ctrl(self):
        return self._view(self.L.ctrl, 16, self.torch.int32)

    def n_tot(self):
        self.sync()
        return int(self.counts().sum().item())

    def counts(self, half=None):
        """Particles per cell of the current (or given) half, int64."""
        h = self.current()[0] if half is None else half
        return self._view(self.L.count[h], self.L.ncells, self.torch.int32).long()

    def three_d(self):
        return int(self.d["ncz"]) >= 2

    def _pkeys(self):
        return ("x", "y", "z", "vx", "vy", "vz") if self.three_d() else ("x", "y", "vx", "vy", "vz")

    # slots of a particle record (x, y, vx, vy, vz, z, key bits, unused)
    REC = 8
    SLOT = {"x": 0, "y": 1, "vx": 2, "vy": 3, "vz": 4, "z": 5}

    def particle_arrays(self, half=None):
        """Binned particle arrays [ncells, bin] of the current (or given) half: strided views
        of the particle records; z only in 3D."""
        h = self.current()[0] if half is None else half
        cap, b = self.L.capacity, self.L.bin
        rec = self._view(self.L.part[h], cap * self.REC, self.real).view(cap, self.REC)
        return {k: rec[:, self.SLOT[k]].view(-1, b) for k in self._pkeys()}

    def particles(self):
        """Current particles in cell order (copies, compacted from the bins)."""
        self.sync()
        torch = self.torch
        cnt = self.counts()
        mask = torch.arange(self.L.bin, device=self.device)[None, :] < cnt[:, None]
        return {k: v[mask] for k, v in self.particle_arrays().items()}

    def cell_start(self):
        """First compacted index of each cell (ncells + 1), int32."""
        torch = self.torch
        cs = torch.zeros(self.L.ncells + 1, dtype=torch.int64, device=self.device)
        cs[1:] = torch.cumsum(self.counts(), 0)
        return cs.int()

    def acc(self):
        return self._view(self.L.acc, self.L.ncells * 20, self.torch.float64).view(-1, 20)

    def grad_records(self, n):
        """The Grad records the last map_lbm_to_dsmc wrote for its n listed cells, in list
        order: (rho [n] f64, new counts [n] int64, v [n, 20] f64 = a2 (6), a3 (10), u (3), C),
        the FP64 coefficients of Table 1 step 1 (copies)."""
        torch = self.torch
        self.sync()
        raw = self._view(self.L.map_scratch, n * 176, torch.uint8).view(n, 176).cpu()
        rho = raw[:, 0:8].contiguous().view(torch.float64).view(n)
        nnew = raw[:, 8:12].contiguous().view(torch.int32).view(n).long()
        v = raw[:, 16:176].contiguous().view(torch.float64).view(n, 20)
        return rho, nnew, v

    def crmax(self):
        return self._view(self.L.crmax, self.L.ncells, self.real)

    def rem(self):
        return self._view(self.L.rem, self.L.ncells, self.real)

    def nbar_sum(self):
        return self._view(self.L.nbar_sum, self.L.ncells, self.torch.int32)

    def f(self, half=None):
        """Populations [q, ny, nx] (slab) or [q, nz, ny, nx] (3D) of the current (or given)
        half (a view)."""
        h = self.current()[1] if half is None else half
        q, ny, nx, nz = self.d["q"], self.d["ny"], self.d["nx"], self.d["nz"]
        v = self._view(self.L.f[h], q * nx * ny * nz, self.real)
        return v.view(q, nz, ny, nx) if self.three_d() else v.view(q, ny, nx)

    # -- state transfer (checkpoint / restore, synthetic states) ------------------------
    def load_particles(self, x, y, vx, vy, vz, cell_start, z=None):
        """Write a cell-ordered particle set into the bins of the current half (host arrays);
        z is required in 3D."""
        torch = self.torch
        cs = np.asarray(cell_start, np.int64)
        counts = np.diff(cs)
        if counts.size != self.L.ncells:
            raise ValueError("cell_start must have ncells + 1 entries")
        if counts.max(initial=0) > self.L.bin:
            raise ValueError("a cell holds more particles than its bin (%d)" % self.L.bin)
        cell = np.repeat(np.arange(self.L.ncells), counts)
        slot = torch.as_tensor(cell * self.L.bin + (np.arange(cs[-1]) - cs[cell]),
                               device=self.device)
        arr = self.particle_arrays()
        vals = [("x", x), ("y", y), ("vx", vx), ("vy", vy), ("vz", vz)]
        if self.three_d():
            if z is None:
                raise ValueError("a 3D context needs the z positions")
            vals.append(("z", z))
        for k, v in vals:
            arr[k].view(-1)[slot] = torch.as_tensor(np.asarray(v), dtype=self.real,
                                                    device=self.device)
        h = self.current()[0]
        self._view(self.L.count[h], self.L.ncells, torch.int32).copy_(
            torch.as_tensor(counts.astype(np.int32)))
        self.ctrl()[CTRL_NTOT] = int(cs[-1])
        torch.cuda.synchronize(self.device)

    def set_counters(self, step=None, nsamples=None):
        if step is not None:
            self.ctrl()[CTRL_STEP] = int(step)
        if nsamples is not None:
            self.ctrl()[CTRL_NSAMPLES] = int(nsamples)
        self.torch.cuda.synchronize(self.device)

    def save_state(self):
        """Host copy of the whole arena plus the ping-pong parities (bit-exact resume)."""
        self.sync()
        return {"arena": self.arena.cpu(), "current": self.current(), "cfg": dict(self.cfg)}

    def load_state(self, state):
        if state["cfg"] != self.cfg:
            raise ValueError("state was saved for different parameters")
        if tuple(state["current"]) != self.current():
            raise ValueError("restore into a context with the same ping-pong parity")
        self.sync()
        self.arena.copy_(state["arena"].to(self.device))
        self.torch.cuda.synchronize(self.device)


class Batch:
    """Independent channels (replicas) advanced together: one launch per kernel for all of
    them per hybrid step. `replicas[r]` is a Hybrid view of replica r (state, counters)."""

    def __init__(self, cfgs, device="cuda:0", stream=None):
        import torch
        self.torch = torch
        self.cfgs = [dict(c) for c in cfgs]
        n = len(self.cfgs)
        self.device = torch.device(device)
        params = (HybParams * n)(*[make_params(c) for c in self.cfgs])
        offsets = (ctypes.c_uint64 * (n + 2))()
        _check(lib().hyb_batch_layout(params, n, offsets))
        self.offsets = [int(o) for o in offsets]
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.Stream(self.device)
            self.arena = torch.zeros(self.offsets[n + 1], dtype=torch.uint8, device=self.device)
        torch.cuda.synchronize(self.device)
        b = _vp()
        with torch.cuda.device(self.device):
            rc = lib().hyb_batch_init(params, n, self.arena.data_ptr(), self.offsets[n + 1],
                                      self.stream.cuda_stream, ctypes.byref(b))
        _check(rc)
        self.b = b
        self.replicas = []
        for r in range(n):
            ctx = _vp()
            _check(lib().hyb_batch_replica(self.b, r, ctypes.byref(ctx)))
            size = int(layout(self.cfgs[r]).total_bytes)
            view = self.arena[self.offsets[r]:self.offsets[r] + size]
            self.replicas.append(Hybrid._attach(self.cfgs[r], self.device, self.stream, ctx, view))
        self._lists = None

    def _prepare(self, nodes, cells):
        """Concatenated device lists and host offsets, kept alive while the batch uses them."""
        torch = self.torch
        key = (tuple(id(x) for x in nodes), tuple(id(x) for x in cells))
        if self._lists is not None and self._lists[0] == key:
            return self._lists[1]
        def cat(lists):
            pre = np.zeros(len(lists) + 1, np.int64)
            pre[1:] = np.cumsum([len(x) for x in lists])
            flat = np.concatenate([np.asarray(x, np.int32) for x in lists]) if pre[-1] else np.zeros(1, np.int32)
            dev = torch.from_numpy(flat).to(self.device)
            return dev, pre
        dn, pn = cat(nodes)
        dc, pc = cat(cells)
        self.stream.wait_stream(torch.cuda.current_stream(self.device))
        prepared = (dn, pn, dc, pc)
        self._lists = (key, prepared)
        return prepared

    def moment_sums(self, out=None):
        """The replicas' cumulative FP64 moment sums, one after another in replica order, as one
        flat device tensor (copied into `out` if given): the buffer a multi-GPU ensemble sums
        over its ranks."""
        accs = [r.acc().reshape(-1) for r in self.replicas]
        n = sum(a.numel() for a in accs)
        if out is None:
            out = accs[0].new_empty(n)
        o = 0
        for a in accs:
            out[o:o + a.numel()].copy_(a)
            o += a.numel()
        return out

    def hybrid_step(self, nodes, cells, nsteps=1, use_graph=True):
        """`nodes[r]`, `cells[r]`: replica r's coupling nodes and cells (host int arrays)."""
        dn, pn, dc, pc = self._prepare(nodes, cells)
        rc = lib().hyb_batch_hybrid_step(self.b, dn.data_ptr(), pn.ctypes.data_as(_vp), dc.data_ptr(),
                                         pc.ctypes.data_as(_vp), int(nsteps), 1 if use_graph else 0)
        if rc != HYB_OK:
            raise HybError(rc, lib().hyb_batch_last_error(self.b).decode())

    def set_blocks(self, move_block, lbm_block):
        _check(lib().hyb_batch_set_blocks(self.b, int(move_block), int(lbm_block)))

    def set_block(self, kernel, threads):
        """Block size of one kernel class (a name of KERNELS: move, collide, lbm, dsmc2lb, lb2dsmc)."""
        _check(lib().hyb_batch_set_block(self.b, KERNELS[kernel], int(threads)))

    def blocks(self):
        """The block size of every kernel class of the batch."""
        return {k: int(lib().hyb_batch_get_block(self.b, KERNELS[k]))
                for k in ("move", "collide", "lbm", "dsmc2lb", "lb2dsmc")}

    def tune(self, nodes, cells):
        """Picks the block shapes by timing hybrid steps (advances the batch); returns the move
        and LB sizes (blocks() gives every class)."""
        dn, pn, dc, pc = self._prepare(nodes, cells)
        mb, lb = _i32(), _i32()
        rc = lib().hyb_batch_tune(self.b, dn.data_ptr(), pn.ctypes.data_as(_vp), dc.data_ptr(),
                                  pc.ctypes.data_as(_vp), ctypes.byref(mb), ctypes.byref(lb))
        if rc != HYB_OK:
            raise HybError(rc, lib().hyb_batch_last_error(self.b).decode())
        return mb.value, lb.value

    def sync(self):
        self.stream.synchronize()

    def close(self):
        if getattr(self, "b", None):
            for h in self.replicas:
                h.ctx = None
            lib().hyb_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class SlabGroup:
    """A channel of ncy DSMC rows cut into streamwise slabs (the multi-GPU decomposition), all
    on one device: slab i is a Hybrid of the rows [y0_i, y0_i + rows_i) (periodic channel). A
    step runs every slab's split DSMC step and LB step with the exchanges between them as
    device copies on the slabs' shared stream: the particles that leave a slab (send buffers
    into the neighbours' receive buffers), and before every LB step the outgoing populations
    of the rows next to each boundary (packed by the library into staging, copied, unpacked
    into the neighbours' ghost rows). Across ranks the same buffers go through
    torch.distributed send/recv (see exchange_dist). The results equal the whole channel's."""

    def __init__(self, cfg, cuts, device="cuda:0"):
        import torch
        self.torch = torch
        self.cfg = dict(cfg)
        ncy = cfg["ncy"]
        bounds = [0] + list(cuts) + [ncy]
        self.stream = torch.cuda.Stream(torch.device(device))
        self.slabs = []
        for i in range(len(bounds) - 1):
            c = dict(cfg, ncy=bounds[i + 1] - bounds[i], ncy_global=ncy, y0=bounds[i])
            self.slabs.append(Hybrid(c, device=device, stream=self.stream))
        n = self.slabs[0].halo_size()
        dt = self.slabs[0].real
        self.halo = [[torch.empty(n, dtype=dt, device=device) for _ in range(2)] for _ in self.slabs]

    def close(self):
        for h in self.slabs:
            h.close()

    def _copy(self, dst, src):
        with self.torch.cuda.stream(self.stream):
            dst.copy_(src)

    def exchange_particles(self):
        k = len(self.slabs)
        for i, h in enumerate(self.slabs):
            below, above = self.slabs[(i - 1) % k], self.slabs[(i + 1) % k]
            self._copy(h.xfer("recv", 0), below.xfer("send", 1))
            self._copy(h.xfer("recv", 1), above.xfer("send", 0))

    def exchange_halo(self):
        k = len(self.slabs)
        for i, h in enumerate(self.slabs):
            h.halo_pack(0, self.halo[i][0])
            h.halo_pack(1, self.halo[i][1])
        for i, h in enumerate(self.slabs):
            h.halo_unpack(0, self.halo[(i - 1) % k][1])
            h.halo_unpack(1, self.halo[(i + 1) % k][0])

    def dsmc_step(self):
        for h in self.slabs:
            h.dsmc_move()
        self.exchange_particles()
        for h in self.slabs:
            h.dsmc_merge()
        for h in self.slabs:
            h.dsmc_collide()

    def lbm_step(self):
        self.exchange_halo()
        for h in self.slabs:
            h.lbm_step(1)

    def hybrid_step(self, nodes=None, cells=None):
        """One hybrid step; nodes[i] / cells[i]: slab i's coupling lists (device int32, the
        slab's own node and cell indices, or None)."""
        self.dsmc_step()
        for i, h in enumerate(self.slabs):
            if nodes is not None and nodes[i] is not None and nodes[i].numel():
                h.map_dsmc_to_lbm(nodes[i])
        self.lbm_step()
        for i, h in enumerate(self.slabs):
            if cells is not None and cells[i] is not None and cells[i].numel():
                h.map_lbm_to_dsmc(cells[i])

    def sync(self):
        self.torch.cuda.synchronize()


def exchange_dist(h, dist, rank, world, halo_bufs=None):
    """The exchanges of a slab whose neighbours are other ranks (NCCL or gloo through
    torch.distributed): the send buffers to the ranks below and above into this slab's
    receive buffers, or, with halo_bufs = (packed side 0, packed side 1, received side 0,
    received side 1), the packed populations. Blocking point-to-point pairs, ordered so that
    even ranks send first."""
    below, above = (rank - 1) % world, (rank + 1) % world
    if halo_bufs is None:
        pairs = [(h.xfer("send", 1), above, h.xfer("recv", 0), below),
                 (h.xfer("send", 0), below, h.xfer("recv", 1), above)]
    else:
        p0, p1, r0, r1 = halo_bufs
        pairs = [(p1, above, r0, below), (p0, below, r1, above)]
    for sbuf, sto, rbuf, rfrom in pairs:
        if rank % 2 == 0:
            dist.send(sbuf, sto)
            dist.recv(rbuf, rfrom)
        else:
            dist.recv(rbuf, rfrom)
            dist.send(sbuf, sto)


def interface_loss(h, g, tau, f0, nodes, targets, nsteps, ckpt_every=100):
    """Coupling-interface loss after `nsteps` LB steps from populations f0 with per-node force
    increment g and relaxation time tau (tensors of the context's shape and precision), as a
    differentiable function of g, tau and f0. The backward pass is the library's adjoint
    step, run over the steps in reverse; the states are recomputed segment by segment from
    checkpoints stored every `ckpt_every` steps."""
    return _InterfaceLoss.apply(g, tau, f0, h, nodes, targets, int(nsteps), int(ckpt_every))


def coupled_interface_loss(h, acc, nsamples, d2l_nodes, g, tau, f0, nodes, targets, nsteps,
                           ckpt_every=100):
    """The interface loss of the differentiated coupling: DSMC2LB maps the cumulative sums
    `acc` (float64 [ncells, 20], `nsamples` samples) into the populations f0 at `d2l_nodes`
    (distinct int32), then `nsteps` LB steps run with per-node g and tau, and the loss is
    taken at `nodes` against `targets` (as interface_loss). Differentiable with respect to
    acc, g, tau and f0. The context's own sums, sample count and current populations serve
    as scratch for the mapping."""
    return _CoupledLoss.apply(acc, g, tau, f0, h, int(nsamples), d2l_nodes, nodes, targets,
                              int(nsteps), int(ckpt_every))


def _d2l_into(h, acc, nsamples, d2l_nodes, f0):
    """f0 with DSMC2LB of `acc` written at `d2l_nodes` (a new tensor), through the context."""
    h._inputs(acc, f0)
    with h.torch.cuda.stream(h.stream):
        h.acc().copy_(acc)
        h.f().copy_(f0)
    h.set_counters(nsamples=nsamples)
    h.map_dsmc_to_lbm(d2l_nodes)
    with h.torch.cuda.stream(h.stream):
        return h.f().clone()


def _make_coupled_loss():
    import torch

    class CoupledLoss(torch.autograd.Function):
        @staticmethod
        def forward(ctx, acc, g, tau, f0, h, nsamples, d2l_nodes, nodes, targets, nsteps,
                    ckpt_every):
            g, tau = g.detach().contiguous(), tau.detach().contiguous()
            fm = _d2l_into(h, acc.detach().contiguous(), nsamples, d2l_nodes, f0.detach())
            loss, lam_T, ckpts = _loss_forward(h, g, tau, fm, nodes, targets, nsteps, ckpt_every)
            ctx.h, ctx.nsamples = h, nsamples
            ctx.nsteps, ctx.ckpt_every = nsteps, ckpt_every
            ctx.save_for_backward(g, tau, lam_T, d2l_nodes, *ckpts)
            return loss[0]

        @staticmethod
        def backward(ctx, gout):
            h = ctx.h
            g, tau, lam_T, d2l_nodes, *ckpts = ctx.saved_tensors
            h.stream.wait_stream(torch.cuda.current_stream(g.device))
            grad_g, grad_tau, lam = _loss_adjoint(h, g, tau, lam_T, ckpts, ctx.nsteps,
                                                  ctx.ckpt_every)
            grad_acc = torch.zeros(int(h.L.ncells), 20, dtype=torch.float64, device=g.device)
            h.set_counters(nsamples=ctx.nsamples)
            h.map_dsmc_to_lbm_adjoint(d2l_nodes, lam, grad_acc)  # zeroes lam at d2l_nodes
            with torch.cuda.stream(h.stream):
                s = gout.to(g.dtype)
                out = (grad_acc * gout.to(torch.float64), grad_g * s, grad_tau * s, lam * s)
            torch.cuda.current_stream(g.device).wait_stream(h.stream)
            return out + (None,) * 7

    return CoupledLoss


def _lb_forward(h, g, tau, f0, nsteps, ckpt_every):
    """f_T and the checkpoints f_0, f_K, f_2K, ... (K = ckpt_every), the steps in one library
    call."""
    a = f0.detach().clone()
    b = h.torch.empty_like(a)
    nck = (nsteps - 1) // ckpt_every if nsteps > 0 else 0
    ck = h.torch.empty((max(nck, 1),) + tuple(a.shape), dtype=a.dtype, device=a.device)
    ckpts = [a.clone()]
    fT = h.lbm_steps_nodes(a, b, g, tau, nsteps, ckpt_every, ck if nck else None)
    ckpts += [ck[i] for i in range(nck)]
    return fT, ckpts


def _loss_forward(h, g, tau, f0, nodes, targets, nsteps, ckpt_every):
    """Loss after nsteps LB steps from f0, dL/df_T, and the checkpoints of the states."""
    torch = h.torch
    with torch.cuda.stream(h.stream):
        fT, ckpts = _lb_forward(h, g, tau, f0, nsteps, ckpt_every)
        loss = torch.zeros(1, dtype=torch.float64, device=f0.device)
        lam = torch.zeros_like(fT)
        h.lbm_interface_loss(fT, nodes, targets, loss, lam)
    torch.cuda.current_stream(f0.device).wait_stream(h.stream)
    return loss, lam, ckpts


def _loss_adjoint(h, g, tau, lam_T, ckpts, T, K):
    """The adjoint sweep: (dL/dg, dL/dtau, dL/df_0) from dL/df_T, recomputing the states of
    each checkpoint segment forward and running the adjoint steps over them in reverse."""
    torch = h.torch
    with torch.cuda.stream(h.stream):
        grad_g = torch.zeros_like(g)
        grad_tau = torch.zeros_like(tau)
        wall = torch.zeros(h.wall_scratch_size(), dtype=g.dtype, device=g.device)
        lam_next = lam_T.clone()
        lam = torch.empty_like(lam_next)
        scratch = torch.empty((max(K - 1, 1),) + tuple(lam_next.shape), dtype=lam_next.dtype,
                              device=lam_next.device)
        for s in reversed(range(len(ckpts))):
            t0, t1 = s * K, min(T, (s + 1) * K)
            if t1 <= t0:  # no steps (T = 0)
                continue
            out = h.lbm_adjoint_segment(ckpts[s], scratch if t1 - t0 > 1 else None, t1 - t0, lam_next,
                                        lam, g, tau, grad_g, grad_tau, wall)
            if out is not lam_next:
                lam_next, lam = lam, lam_next
    return grad_g, grad_tau, lam_next


def _make_interface_loss():
    import torch

    class InterfaceLoss(torch.autograd.Function):
        @staticmethod
        def forward(ctx, g, tau, f0, h, nodes, targets, nsteps, ckpt_every):
            g, tau = g.detach().contiguous(), tau.detach().contiguous()
            loss, lam, ckpts = _loss_forward(h, g, tau, f0, nodes, targets, nsteps, ckpt_every)
            ctx.h = h
            ctx.nsteps, ctx.ckpt_every = nsteps, ckpt_every
            ctx.save_for_backward(g, tau, lam, *ckpts)
            return loss[0]

        @staticmethod
        def backward(ctx, gout):
            h = ctx.h
            g, tau, lam_T, *ckpts = ctx.saved_tensors
            h.stream.wait_stream(torch.cuda.current_stream(g.device))
            grad_g, grad_tau, lam = _loss_adjoint(h, g, tau, lam_T, ckpts, ctx.nsteps,
                                                  ctx.ckpt_every)
            with torch.cuda.stream(h.stream):
                s = gout.to(g.dtype)
                gg, gt, gf = grad_g * s, grad_tau * s, lam * s
            torch.cuda.current_stream(g.device).wait_stream(h.stream)
            return gg, gt, gf, None, None, None, None, None

    return InterfaceLoss


class _Lazy:
    def __init__(self, make):
        self._make, self._cls = make, None

    def apply(self, *args):
        if self._cls is None:
            self._cls = self._make()
        return self._cls.apply(*args)


_InterfaceLoss = _Lazy(_make_interface_loss)
_CoupledLoss = _Lazy(_make_coupled_loss)
