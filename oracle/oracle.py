"""ctypes wrapper around the CPU oracle (test infrastructure only).

The oracle is a plain, slow restatement of the DSMC-LBM mapping method (arXiv 1512.08042)
used to check the CUDA library. Only the tests, the smoke check and the CPU-baseline leg of
the benchmark may import this module; the library itself never does.
"""
import ctypes
import os

import numpy as np

from . import build as _build

_LIB = None

A_X, A_Y, A_VX, A_VY, A_VZ, A_CELL_START, A_CRMAX, A_REM, A_NBAR_SUM, A_ACC, A_F, A_Z = range(12)
COUNTER_NAMES = ["wall_hits", "candidates", "collisions", "created", "deleted",
                 "l2d_attempts", "envelope", "bounce_cap"]
ST_CAPACITY, ST_BOUNCE_CAP, ST_SCATTER_CAP, ST_SAMPLING_CAP, ST_CELL_OVERFLOW, ST_BAD_INPUT = (
    1, 2, 4, 8, 16, 32)


class Params(ctypes.Structure):
    _fields_ = [
        ("abi_version", ctypes.c_uint32),
        ("ncx", ctypes.c_int32),
        ("ncy", ctypes.c_int32),
        ("lb_ratio", ctypes.c_int32),
        ("ppc", ctypes.c_int32),
        ("lattice", ctypes.c_int32),
        ("real_bytes", ctypes.c_int32),
        ("sample_every", ctypes.c_int32),
        ("seed", ctypes.c_uint64),
        ("kn", ctypes.c_double),
        ("ma", ctypes.c_double),
        ("crmax_init", ctypes.c_double),
        ("capacity_factor", ctypes.c_double),
        ("T_K", ctypes.c_double),
        ("mass_kg", ctypes.c_double),
        ("lb_collision", ctypes.c_int32),
        ("d2l_mode", ctypes.c_int32),
        ("kn_profile", ctypes.c_int32),
        ("pad0", ctypes.c_int32),
        ("kn_end", ctypes.c_double),
        ("ncz", ctypes.c_int32),
        ("accum_mode", ctypes.c_int32),
        ("ncy_global", ctypes.c_int32),
        ("y0", ctypes.c_int32),
    ]


class Derived(ctypes.Structure):
    _fields_ = [
        ("r_lat", ctypes.c_double),
        ("cs_lat", ctypes.c_double),
        ("H_lat", ctypes.c_double),
        ("tau", ctypes.c_double),
        ("dt", ctypes.c_double),
        ("lam", ctypes.c_double),
        ("coll_dt", ctypes.c_double),
        ("g_step", ctypes.c_double),
        ("c_th_ms", ctypes.c_double),
        ("ncells", ctypes.c_int64),
        ("nx", ctypes.c_int64),
        ("ny", ctypes.c_int64),
        ("nnodes", ctypes.c_int64),
        ("capacity", ctypes.c_int64),
        ("q", ctypes.c_int32),
        ("order", ctypes.c_int32),
        ("bin", ctypes.c_int32),
        ("pad", ctypes.c_int32),
        ("nz", ctypes.c_int64),
        ("ncz", ctypes.c_int64),
        ("yh", ctypes.c_int64),
        ("xcap", ctypes.c_int64),
    ]


def lib():
    global _LIB
    if _LIB is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        vp, i32, i64, u32, u64, dbl = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64,
                                       ctypes.c_uint32, ctypes.c_uint64, ctypes.c_double)
        L.ora_derive.argtypes = [ctypes.POINTER(Params), ctypes.POINTER(Derived)]
        L.ora_philox.argtypes = [vp, u64, vp, i64]
        L.ora_lattice.argtypes = [ctypes.c_int, vp, vp, ctypes.POINTER(dbl)]
        L.ora_create.argtypes = [ctypes.POINTER(Params)]
        L.ora_create.restype = vp
        L.ora_destroy.argtypes = [vp]
        L.ora_dsmc_step.argtypes = [vp, ctypes.c_int]
        L.ora_lbm_step.argtypes = [vp, ctypes.c_int]
        L.ora_dsmc_phase.argtypes = [vp, ctypes.c_int]
        L.ora_map_dsmc_to_lbm.argtypes = [vp, vp, ctypes.c_int]
        L.ora_map_lbm_to_dsmc.argtypes = [vp, vp, ctypes.c_int]
        L.ora_get.argtypes = [vp, ctypes.c_int, vp]
        L.ora_get.restype = i64
        L.ora_set.argtypes = [vp, ctypes.c_int, vp, i64]
        L.ora_scalars.argtypes = [vp, vp]
        L.ora_set_scalars.argtypes = [vp, u64, u64]
        L.ora_counters.argtypes = [vp, vp]
        L.ora_lbm_collide.argtypes = [ctypes.POINTER(Params), vp, vp]
        L.ora_dsmc2lb_node.argtypes = [ctypes.c_int, vp, u64, ctypes.c_int, vp]
        L.ora_grad_coeffs.argtypes = [ctypes.c_int, vp, vp]
        L.ora_dsmc_move.argtypes = [vp]
        L.ora_dsmc_move.restype = None
        L.ora_outbox_size.argtypes = [vp, ctypes.c_int]
        L.ora_outbox_size.restype = i64
        L.ora_outbox_get.argtypes = [vp, ctypes.c_int, vp, vp]
        L.ora_outbox_get.restype = None
        L.ora_dsmc_accept.argtypes = [vp, vp, vp, i64, vp, vp, i64]
        L.ora_dsmc_accept.restype = None
        L.ora_grad_coeffs_packed.argtypes = [ctypes.c_int, vp, ctypes.c_int, vp]
        L.ora_grad_sample.argtypes = [ctypes.c_int, vp, u64, u32, u32, i64, vp, vp]
        L.ora_float_funcs.argtypes = [vp, i64, vp, vp, vp]
        L.ora_grad_G.argtypes = [ctypes.c_int, vp, vp, i64, ctypes.c_int, vp]
        L.ora_gauss_pairs.argtypes = [vp, i64, ctypes.c_int, vp]
        L.ora_lbm_node_params.argtypes = [vp, vp, vp, i64]
        L.ora_dsmc_cell_coll.argtypes = [vp, vp, i64]
        L.ora_kn_profile_rows.argtypes = [ctypes.POINTER(Params), i64, i64, vp, i64, i64, vp]
        L.ora_lbm_grad_node.argtypes = [vp, i64, vp]
        L.ora_lbm_interface_loss.argtypes = [vp, vp, ctypes.c_int, vp]
        L.ora_lbm_interface_loss.restype = ctypes.c_double
        _LIB = L
    return _LIB


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def make_params(cfg):
    p = Params()
    p.abi_version = 1
    for name, _ in Params._fields_:
        if name != "abi_version" and name in cfg:
            setattr(p, name, cfg[name])
    return p


def derive(cfg):
    d = Derived()
    rc = lib().ora_derive(ctypes.byref(make_params(cfg)), ctypes.byref(d))
    if rc != 0:
        raise ValueError("invalid parameters")
    return {name: getattr(d, name) for name, _ in Derived._fields_}


def philox(ctr, seed):
    ctr = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    out = np.empty_like(ctr)
    lib().ora_philox(_ptr(ctr), ctypes.c_uint64(seed), _ptr(out), ctr.shape[0])
    return out


def lattice(q):
    e = np.zeros((q, 3), np.int32)
    w = np.zeros(q, np.float64)
    r = ctypes.c_double()
    if lib().ora_lattice(q, _ptr(e), _ptr(w), ctypes.byref(r)) != 0:
        raise ValueError(q)
    return e, w, r.value


def lbm_collide(cfg, fs):
    fs = np.ascontiguousarray(fs, np.float64)
    out = np.empty_like(fs)
    if lib().ora_lbm_collide(ctypes.byref(make_params(cfg)), _ptr(fs), _ptr(out)) != 0:
        raise ValueError("invalid parameters")
    return out


def dsmc2lb_node(q, m20, S, ppc):
    m = np.ascontiguousarray(m20, np.float64)
    out = np.empty(q, np.float64)
    rc = lib().ora_dsmc2lb_node(q, _ptr(m), S, ppc, _ptr(out))
    if rc != 0:
        raise ValueError(rc)
    return out


def grad_coeffs(q, f):
    f = np.ascontiguousarray(f, np.float64)
    out = np.empty(42, np.float64)
    lib().ora_grad_coeffs(q, _ptr(f), _ptr(out))
    return {"rho": out[0], "u": out[1:4].copy(), "a2": out[4:13].reshape(3, 3).copy(),
            "a3": out[13:40].reshape(3, 3, 3).copy(), "M": out[40], "C": out[41]}


def grad_coeffs_packed(q, f, real_bytes):
    """LB2DSMC coefficients in FP64, packed and rounded to the precision real_bytes (rho and
    M stay FP64), as the sampler takes them."""
    f = np.ascontiguousarray(f, np.float64)
    out = np.empty(22, np.float64)
    if lib().ora_grad_coeffs_packed(q, _ptr(f), real_bytes, _ptr(out)) != 0:
        raise ValueError(q)
    return {"rho": out[0], "u": out[1:4].copy(), "a2": out[4:10].copy(),
            "a3": out[10:20].copy(), "M": out[20], "C": out[21]}


def grad_sample(q, f, seed, cell, t, n):
    f = np.ascontiguousarray(f, np.float64)
    v = np.empty((n, 3), np.float64)
    info = np.zeros(3, np.uint64)
    rc = lib().ora_grad_sample(q, _ptr(f), seed, cell, t, n, _ptr(v), _ptr(info))
    if rc != 0:
        raise ValueError(rc)
    return v, {"attempts": int(info[0]), "envelope": int(info[1]), "cap": int(info[2])}


def grad_G(q, f, xi, real_bytes):
    """G(xi) of the populations f: (packed state-precision form, full-tensor double form)."""
    f = np.ascontiguousarray(f, np.float64)
    xi = np.ascontiguousarray(xi, np.float64).reshape(-1, 3)
    out = np.empty((xi.shape[0], 2), np.float64)
    lib().ora_grad_G(q, _ptr(f), _ptr(xi), xi.shape[0], real_bytes, _ptr(out))
    return out[:, 0], out[:, 1]


def float_funcs(x):
    """ln(x), sin(2 pi x), cos(2 pi x) by the float series of the float state path."""
    x = np.ascontiguousarray(x, np.float32)
    ln, sn, cs = (np.empty_like(x) for _ in range(3))
    lib().ora_float_funcs(_ptr(x), x.size, _ptr(ln), _ptr(sn), _ptr(cs))
    return ln, sn, cs


def gauss_pairs(words, real_bytes):
    w = np.ascontiguousarray(words, np.uint32).reshape(-1, 2)
    out = np.empty((w.shape[0], 2), np.float64)
    lib().ora_gauss_pairs(_ptr(w), w.shape[0], real_bytes, _ptr(out))
    return out


class Oracle:
    """One DSMC + LBM state on the host (float or double, per cfg['real_bytes'])."""

    def __init__(self, cfg):
        self.cfg = dict(cfg)
        self.params = make_params(cfg)
        self.d = derive(cfg)
        self.h = lib().ora_create(ctypes.byref(self.params))
        if not self.h:
            raise ValueError("invalid parameters")
        self.real = np.float32 if cfg["real_bytes"] == 4 else np.float64

    def __del__(self):
        if getattr(self, "h", None):
            lib().ora_destroy(self.h)
            self.h = None

    def dsmc_step(self, n=1):
        lib().ora_dsmc_step(self.h, n)

    # -- a streamwise slab (cfg["ncy_global"] > 0): the split DSMC step -------------------
    def dsmc_move_out(self):
        """Phase 0 without the sort: moves every particle; returns the outboxes towards lower
        (0) and higher (1) rows: (rows of x, y, z, vx, vy, vz, tag >> 32, tag & 0xFFFFFFFF as
        float64, channel cells as uint32)."""
        lib().ora_dsmc_move(self.h)
        out = []
        for d in (0, 1):
            n = lib().ora_outbox_size(self.h, d)
            rec = np.zeros((n, 8), np.float64)
            key = np.zeros(n, np.uint32)
            lib().ora_outbox_get(self.h, d, _ptr(rec), _ptr(key))
            out.append((rec, key))
        return out

    def dsmc_accept(self, in0, in1):
        """The particles received from the slab below (in0) and above (in1), each (rec, key)
        as dsmc_move_out gives them, join; then the sort that ends phase 0."""
        r0, k0 = (np.ascontiguousarray(a) for a in in0)
        r1, k1 = (np.ascontiguousarray(a) for a in in1)
        lib().ora_dsmc_accept(self.h, _ptr(r0), _ptr(k0), len(k0), _ptr(r1), _ptr(k1), len(k1))

    def dsmc_phase(self, phase):
        """0: move + sort, 1: collide, 2: sample + advance the step counter."""
        lib().ora_dsmc_phase(self.h, phase)

    def lbm_step(self, n=1):
        lib().ora_lbm_step(self.h, n)

    def map_dsmc_to_lbm(self, nodes):
        nodes = np.ascontiguousarray(nodes, np.int32)
        lib().ora_map_dsmc_to_lbm(self.h, _ptr(nodes), len(nodes))

    def map_lbm_to_dsmc(self, cells):
        cells = np.ascontiguousarray(cells, np.int32)
        lib().ora_map_lbm_to_dsmc(self.h, _ptr(cells), len(cells))

    _DT = {A_CELL_START: np.uint32, A_NBAR_SUM: np.uint32, A_ACC: np.float64}

    def _dtype(self, which):
        return self._DT.get(which, self.real)

    def get(self, which):
        n = lib().ora_get(self.h, which, None)
        out = np.empty(n, self._dtype(which))
        lib().ora_get(self.h, which, _ptr(out))
        return out

    def set(self, which, arr):
        arr = np.ascontiguousarray(arr, self._dtype(which))
        if lib().ora_set(self.h, which, _ptr(arr), arr.size) != 0:
            raise ValueError("size mismatch for array %d" % which)

    def particles(self):
        keys = [("x", A_X), ("y", A_Y), ("vx", A_VX), ("vy", A_VY), ("vz", A_VZ)]
        if self.d["ncz"] >= 2:
            keys.append(("z", A_Z))
        return {k: self.get(a) for k, a in keys}

    def set_particles(self, x, y, vx, vy, vz, cell_start, z=None):
        for a, v in ((A_X, x), (A_Y, y), (A_VX, vx), (A_VY, vy), (A_VZ, vz)):
            self.set(a, v)
        if z is not None:
            self.set(A_Z, z)
        self.set(A_CELL_START, cell_start)

    def f(self):
        """Populations [q][y][x], or [q][z][y][x] in 3D."""
        if self.d["nz"] > 1:
            return self.get(A_F).reshape(self.d["q"], self.d["nz"], self.d["ny"], self.d["nx"])
        return self.get(A_F).reshape(self.d["q"], self.d["ny"], self.d["nx"])

    def set_f(self, f):
        self.set(A_F, np.asarray(f).reshape(-1))

    def acc(self):
        return self.get(A_ACC).reshape(-1, 20)

    def set_cell_coll(self, coll=None):
        """Per-cell NTC factors (None: the scalar factor)."""
        if coll is None:
            lib().ora_dsmc_cell_coll(self.h, None, 0)
            return
        coll = np.ascontiguousarray(coll, np.float64).reshape(-1)
        if lib().ora_dsmc_cell_coll(self.h, _ptr(coll), coll.size) != 0:
            raise ValueError("one factor per cell")

    def set_node_params(self, g=None, tau=None):
        """Per-node body-force increment g_y and relaxation time tau (None: the scalars)."""
        if g is None:
            lib().ora_lbm_node_params(self.h, None, None, 0)
            return
        g = np.ascontiguousarray(g, np.float64).reshape(-1)
        tau = np.ascontiguousarray(tau, np.float64).reshape(-1)
        if lib().ora_lbm_node_params(self.h, _ptr(g), _ptr(tau), g.size) != 0:
            raise ValueError("one g and one tau per node")

    def grad_node(self, node):
        out = np.empty(20, np.float64)
        lib().ora_lbm_grad_node(self.h, int(node), _ptr(out))
        return out

    def interface_loss(self, nodes, targets):
        nodes = np.ascontiguousarray(nodes, np.int32)
        targets = np.ascontiguousarray(targets, np.float64).reshape(-1)
        return float(lib().ora_lbm_interface_loss(self.h, _ptr(nodes), len(nodes), _ptr(targets)))

    def scalars(self):
        out = np.zeros(4, np.uint64)
        lib().ora_scalars(self.h, _ptr(out))
        return {"step": int(out[0]), "nsamples": int(out[1]), "status": int(out[2]),
                "ntot": int(out[3])}

    def set_scalars(self, step, nsamples):
        lib().ora_set_scalars(self.h, step, nsamples)

    def counters(self):
        out = np.zeros(16, np.uint64)
        lib().ora_counters(self.h, _ptr(out))
        return {n: int(out[i]) for i, n in enumerate(COUNTER_NAMES)}


def kn_profile_rows(cfg, cell_rows, node_rows):
    """The Kn profile of `cfg` at its own rows: NTC factors of the DSMC cell rows `cell_rows`
    and tau of the LB rows `node_rows` (ranges)."""
    coll = np.zeros(len(cell_rows))
    tau = np.zeros(len(node_rows))
    lib().ora_kn_profile_rows(ctypes.byref(make_params(cfg)), cell_rows.start, len(cell_rows),
                              _ptr(coll), node_rows.start, len(node_rows), _ptr(tau))
    return coll, tau


def interface_loss_after(cfg, f0, g, tau, nodes, targets, nsteps):
    """The coupling-interface loss after nsteps LBM steps from f0 with per-node g and tau."""
    o = Oracle(cfg)
    o.set_f(f0)
    o.set_node_params(g, tau)
    o.lbm_step(nsteps)
    return o.interface_loss(nodes, targets)


def coupled_loss_after(cfg, acc, nsamples, d2l_nodes, f0, g, tau, nodes, targets, nsteps):
    """The interface loss after DSMC2LB of the sums `acc` (S = nsamples) into f0 at
    d2l_nodes, then nsteps LBM steps with per-node g and tau."""
    o = Oracle(cfg)
    o.set_f(f0)
    o.set(A_ACC, np.asarray(acc, np.float64).reshape(-1))
    o.set_scalars(0, nsamples)
    o.map_dsmc_to_lbm(np.ascontiguousarray(d2l_nodes, np.int32))
    o.set_node_params(g, tau)
    o.lbm_step(nsteps)
    return o.interface_loss(nodes, targets)


def coupled_loss_fd_gradient(cfg, acc, nsamples, d2l_nodes, f0, g, tau, nodes, targets, nsteps,
                             entries, h=1e-6):
    """Central finite differences of coupled_loss_after with respect to the sums
    acc[cell, k] for each (cell, k) in `entries`: the oracle's reference gradient."""
    acc = np.array(acc, np.float64).reshape(-1, 20)
    out = np.zeros(len(entries))
    for i, (c, k) in enumerate(entries):
        step = h * max(1.0, abs(acc[c, k]))
        save = acc[c, k]
        acc[c, k] = save + step
        lp = coupled_loss_after(cfg, acc, nsamples, d2l_nodes, f0, g, tau, nodes, targets, nsteps)
        acc[c, k] = save - step
        lm = coupled_loss_after(cfg, acc, nsamples, d2l_nodes, f0, g, tau, nodes, targets, nsteps)
        acc[c, k] = save
        out[i] = (lp - lm) / (2.0 * step)
    return out


def interface_loss_fd_gradient(cfg, f0, g, tau, nodes, targets, nsteps, h=1e-6, which=None):
    """Central finite differences of the interface loss with respect to g and tau at the
    nodes `which` (all nodes when None): the oracle's reference gradient."""
    g = np.asarray(g, np.float64).reshape(-1)
    tau = np.asarray(tau, np.float64).reshape(-1)
    idx = np.arange(g.size) if which is None else np.asarray(which)
    o = Oracle(cfg)
    f0 = np.asarray(f0).reshape(-1)

    def loss(gg, tt):
        o.set_f(f0)
        o.set_node_params(gg, tt)
        o.lbm_step(nsteps)
        return o.interface_loss(nodes, targets)

    dg = np.zeros(idx.size)
    dt = np.zeros(idx.size)
    for k, n in enumerate(idx):
        for arr, out, step in ((g, dg, h * max(1e-3, abs(g[n]))), (tau, dt, h * tau[n])):
            save = arr[n]
            arr[n] = save + step
            lp = loss(g, tau)
            arr[n] = save - step
            lm = loss(g, tau)
            arr[n] = save
            out[k] = (lp - lm) / (2.0 * step)
    return dg, dt
