"""Benchmark of the hybrid DSMC-LBM hot path on GB300.

One step = one hybrid step over the whole channel: DSMC step (move, sort, NTC collisions,
sampling), DSMC2LB on the coupling strip, LB stream-collide, LB2DSMC on the coupling strip.
Default workload: the large channel, 512 x 4096 DSMC cells at 50 particles/cell
(104,857,600 particles), Kn varying log-linearly from 0.005 to 0.5 along the channel, FP32
state with FP64 moment sums, 1024 x 8192 D3Q39 lattice with per-node relaxation times,
coupled every step on a 4-cell (8-node) strip. Inputs are synthetic (seeded Maxwellian
start) and larger than the L2 cache (about 23 GB of state); the L2 is also flushed before
every timed step (a 512 MB write), and every step is timed with CUDA events on the library's
stream.

Prints one JSON line. `--impl reference` times the CPU oracle instead (the reference arm:
there is no reference implementation of the paper's method to run, only its restatement),
on windows of the same channel in one process per host core. Under torchrun (N > 1) the
channel is cut into streamwise slabs, one per rank (each rank keeps the single-GPU channel's
rows of a channel N times as long: weak scaling), exchanging the particles that leave a slab
and the LB rows next to its boundaries point to point every step; `--replicas` runs
independent replicas instead.
"""
import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1512_08042_gb300 import workloads as W  # noqa: E402

METRIC = "DSMC particle-updates/s, LBM MLUPS, hybrid steps/s on 1 GB300 at stated tol"
DEFAULT_WORKLOAD = "poiseuille_512x4096_ppc50_knvar_fp32"
WINDOW_ROWS = 16  # DSMC cell rows of the oracle windows (CPU baseline, FP64 error sample)
E2E_CALL = 10  # hybrid steps per host-buffer call of the end-to-end measurement
FLUSH_BYTES = 512 << 20


def launches_in_call(steps, fused, n_nodes, n_cells):
    """The library's kernel launches in one hybrid call of `steps` steps: per step the DSMC
    passes (fused: the collide-and-move pass; else a move and a collide) and the step end, then
    DSMC2LB (with coupling nodes), the LB step and LB2DSMC (with coupling cells); a fused call
    also makes the first move and, with coupling cells, marks and clears them."""
    per_step = (2 if fused else 3) + (n_nodes > 0) + 1 + (n_cells > 0)
    per_call = (1 + 2 * (n_cells > 0 and steps > 1)) if fused else 0
    return steps * per_step + per_call


def kernel_algorithmic_bytes(name, cfg, d, n_particles, n_nodes_map, n_cells_map):
    """Bytes a kernel must move per launch: reads and writes of its inputs and outputs."""
    rb = cfg["real_bytes"]
    ncells = d["ncells"]
    three_d = d["ncz"] >= 2
    pr = 6 if three_d else 5  # Reals per particle: x, y (, z), vx, vy, vz
    if name == "move":
        # pr Real read, pr Real + a u32 key written per particle (into its new cell's bin);
        # per cell: its count read and cleared, the destination counts' atomics
        return n_particles * (2 * pr * rb + 4) + ncells * 12
    if name == "collide":
        # pr Real + key read, pr Real written per particle (in place); per cell: count, crmax,
        # rem, nbar_sum read and written, 20 FP64 sums read and written
        return n_particles * (2 * pr * rb + 4) + ncells * (4 + 2 * rb + 2 * rb + 8 + 320)
    if name == "fused":
        # the collide's reads and per-cell state, then the move's writes: pr Real + key read
        # and written per particle; per cell also the count cleared and the destination atomics
        return n_particles * 2 * (pr * rb + 4) + ncells * (4 + 2 * rb + 2 * rb + 8 + 320 + 8)
    if name == "lbm":
        return d["nnodes"] * 2 * d["q"] * rb
    if name == "dsmc2lb":
        return n_nodes_map * (160 + d["q"] * rb)
    if name == "lb2dsmc":
        # populations of the coupling cells' nodes (r^2, or r^3 in 3D) read; one record and
        # ppc new particles written per coupling cell
        nodes_per_cell = cfg["lb_ratio"] ** (3 if three_d else 2)
        return n_cells_map * (nodes_per_cell * d["q"] * rb + 176 + cfg["ppc"] * pr * rb)
    return 0


def method_bytes(cfg, d):
    """Algorithmic bytes of the method per unit: per DSMC particle-update the particle state
    read and written once (2 x x, y(, z), vx, vy, vz) plus 344 B of per-cell state (20 FP64
    sums read and written, count and offset, (sigma c)max, remainder and N-bar) amortised over
    ppc; per LB node-update the populations read and written once, plus 8 B where tau (and g)
    are per-node fields."""
    rb = cfg["real_bytes"]
    pr = 6 if d["ncz"] >= 2 else 5
    dsmc = 2 * pr * rb + 344.0 / cfg["ppc"]
    lbm = 2 * d["q"] * rb + (8 if cfg.get("kn_profile", 0) == 1 else 0)
    return dsmc, lbm


def sample_clocks(stop, out):
    cmd = ["nvidia-smi", "--query-gpu=clocks.sm,clocks.max.sm,clocks_event_reasons.active,"
           "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
           "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
           "--format=csv,noheader,nounits", "-i", os.environ.get("BENCH_GPU_INDEX", "0")]
    while not stop.is_set():
        try:
            r = subprocess.run(cmd, capture_output=True, text=True, timeout=5)
            if r.returncode == 0 and r.stdout.strip():
                out.append(r.stdout.strip().splitlines()[0])
        except Exception:
            return
        stop.wait(0.2)


def summarize_clocks(lines):
    if not lines:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
    sm, smax, reasons = [], None, set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for ln in lines:
        parts = [p.strip() for p in ln.split(",")]
        try:
            sm.append(float(parts[0]))
            smax = float(parts[1])
        except ValueError:
            continue
        for nm, v in zip(names, parts[3:7]):
            if v.lower() == "active":
                reasons.add(nm)
    sm.sort()
    return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": smax,
            "reasons": sorted(reasons), "samples": len(sm)}


def measured_peak_hbm():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def traffic_record(kernel, workload, units):
    """DRAM bytes per launch of `kernel` from the committed ncu summary (profiles/traffic.json),
    or None if the kernel's source changed since the capture. A capture of a smaller case of
    the same kernel is scaled by the units (particles or nodes) one launch processes: the
    traffic grows in proportion to them (the record states the bytes per unit)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        rec = json.load(open(p))[kernel]
    except Exception:
        return None
    srcs = rec["source"] if isinstance(rec["source"], list) else [rec["source"]]
    sha = hashlib.sha256()
    for f in srcs:  # the kernel's translation unit and the headers it includes, in this order
        sha.update(open(os.path.join(ROOT, "paper_1512_08042_gb300", "csrc", f), "rb").read())
    if sha.hexdigest()[:16] != rec["source_sha"]:
        return None
    if rec.get("workload") == workload:
        return rec["bytes_per_launch"]
    if "bytes_per_unit" in rec:
        return rec["bytes_per_unit"] * units
    return None


def replica_config(cfg, rank):
    """Rank r of a replica ensemble runs the same channel with its own Philox key."""
    out = dict(cfg)
    out["seed"] = int(cfg["seed"]) + int(rank)
    return out


def slab_step(h, dist, rank, world, nodes, cells, halo):
    """One hybrid step of rank `rank`'s streamwise slab: the split DSMC step with the particle
    exchange between neighbouring ranks, DSMC2LB, the exchange of the LB rows next to the
    slab's boundaries, the LB step and LB2DSMC. The exchanges are point-to-point over
    torch.distributed (NCCL between GPUs); the library's stream is synchronised around them."""
    import torch
    from paper_1512_08042_gb300 import binding as B
    h.dsmc_move()
    h.sync()
    B.exchange_dist(h, dist, rank, world)
    torch.cuda.synchronize()
    h.dsmc_merge()
    h.dsmc_collide()
    if nodes.numel():
        h.map_dsmc_to_lbm(nodes)
    h.halo_pack(0, halo[0])
    h.halo_pack(1, halo[1])
    h.sync()
    B.exchange_dist(h, dist, rank, world, halo)
    torch.cuda.synchronize()
    h.halo_unpack(0, halo[2])
    h.halo_unpack(1, halo[3])
    h.lbm_step(1)
    if cells.numel():
        h.map_lbm_to_dsmc(cells)


def run_slab_rank(args, base, rank, world, local_rank, dist):
    """Rank r of the streamwise decomposition (weak scaling: every rank holds base's rows of a
    channel world times as long, with base's coupling strip placed in the middle of the whole
    channel). Returns the rank's line pieces; times are the max over ranks."""
    import torch
    from paper_1512_08042_gb300 import binding as B
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    whole = dict(base, ncy=world * base["ncy"])
    cfg = W.slab_config(base, rank, world)
    h = B.Hybrid(cfg, device=dev)
    d = h.d
    gn, gc = W.coupling_sites(whole)
    ln, lc = W.slab_sites(whole, cfg, d["yh"], gn, gc)
    nodes = torch.from_numpy(ln).to(dev)
    cells = torch.from_numpy(lc).to(dev)
    nh = h.halo_size()
    halo = [torch.empty(nh, dtype=h.real, device=dev) for _ in range(4)]
    for _ in range(args.warmup):
        slab_step(h, dist, rank, world, nodes, cells, halo)
    torch.cuda.synchronize(dev)
    dist.barrier()
    clock_lines, stop = [], threading.Event()
    th = threading.Thread(target=sample_clocks, args=(stop, clock_lines), daemon=True)
    th.start()
    time.sleep(0.3)
    torch.cuda.synchronize(dev)
    dist.barrier()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(h.stream)
    for _ in range(args.steps):
        slab_step(h, dist, rank, world, nodes, cells, halo)
    t1.record(h.stream)
    torch.cuda.synchronize(dev)
    total_ms = max_over_ranks(dist, t0.elapsed_time(t1), dev)
    dist.barrier()
    stop.set()
    th.join(timeout=5)
    # end to end: the same steps with the slab's coupling lists copied in from page-locked
    # host memory and the strip's moment sums read to the host every step
    out = torch.empty((max(1, len(lc)), 20), dtype=torch.float64).pin_memory()
    host_nodes = torch.from_numpy(ln).pin_memory()
    host_cells = torch.from_numpy(lc).pin_memory()
    torch.cuda.synchronize(dev)
    dist.barrier()
    e0 = time.perf_counter()
    e2e_steps = max(5, args.steps // 4)
    for _ in range(e2e_steps):
        with torch.cuda.stream(h.stream):
            nodes.copy_(host_nodes, non_blocking=True)
            cells.copy_(host_cells, non_blocking=True)
        slab_step(h, dist, rank, world, nodes, cells, halo)
        if len(lc):
            with torch.cuda.stream(h.stream):
                out[:len(lc)].copy_(h.acc()[cells.long()])
        torch.cuda.synchronize(dev)
    e2e_s = max_over_ranks(dist, time.perf_counter() - e0, dev)
    rc, bits = h.sync_status()
    n_particles = d["ncells"] * cfg["ppc"]
    value = world * args.steps / (total_ms / 1e3)
    line = {
        "metric": METRIC, "value": value, "unit": "hybrid steps/s (of a rank's slab, times ranks)",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if cfg["real_bytes"] == 4 else "f64", "data": "synthetic",
        "config": {"workload": args.workload, "particles_per_rank": n_particles,
                   "lb_nodes_per_rank": d["nnodes"], "parallelism": "streamwise slabs",
                   "channel_rows": whole["ncy"], "l2": "inputs larger than L2"},
        "dsmc_particle_updates_per_s": value * n_particles,
        "clocks": summarize_clocks(clock_lines),
        # rank 0's launches per step: move, merge, collide, step end, two halo packs, two
        # unpacks, LB step, and DSMC2LB / LB2DSMC where its slab holds coupling sites
        "gpu_launches": args.steps * (9 + int(nodes.numel() > 0) + int(cells.numel() > 0)),
        "status": {"code": rc, "bits": bits},
        "e2e": {"value": world * e2e_steps / e2e_s, "unit": "hybrid steps/s",
                "h2d_bytes_per_step": 4 * (len(ln) + len(lc)), "d2h_bytes_per_step": len(lc) * 160,
                "api": "slab calls with the coupling lists copied in and the strip's moment sums "
                       "read every step"},
    }
    h.close()
    return line


def max_over_ranks(dist, value, device):
    """The largest `value` over all ranks (the job is as slow as its slowest rank)."""
    import torch
    if dist is None:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def window_config(cfg, rows, real_bytes):
    """The channel's first `rows` DSMC cell rows as a periodic channel of their own (the
    oracle window): the same cell ids, Philox keys and derived constants."""
    return dict(cfg, ncy=rows, kn_profile=0, real_bytes=real_bytes)


def window_oracle(cfg, rows, real_bytes):
    """The oracle of the window, with the channel's Kn profile evaluated at its rows."""
    from oracle import oracle as O
    wcfg = window_config(cfg, rows, real_bytes)
    o = O.Oracle(wcfg)
    if cfg.get("kn_profile", 0) == 1:
        d = O.derive(wcfg)
        coll, tau = O.kn_profile_rows(cfg, range(0, rows), range(0, d["ny"]))
        o.set_cell_coll(np.repeat(coll, cfg["ncx"]))
        o.set_node_params(np.full(d["nnodes"], d["g_step"]), np.repeat(tau, d["nx"]))
    return o, wcfg


def oracle_window_worker(job):
    """One host process: hybrid steps (DSMC step, DSMC2LB, LB step, LB2DSMC on the window's own
    strip) of an FP64 oracle window. job = (cfg, rows, nsteps, nwarm, budget_s): nwarm untimed
    steps, then nsteps timed ones, or as many as fit in budget_s if nsteps is 0. Returns
    (steps timed, seconds)."""
    cfg, rows, nsteps, nwarm, budget_s = job
    o, wcfg = window_oracle(cfg, rows, 8)
    nodes, cells = W.coupling_sites(wcfg)

    def one():
        o.dsmc_step(1)
        o.map_dsmc_to_lbm(nodes)
        o.lbm_step(1)
        o.map_lbm_to_dsmc(cells)

    for _ in range(nwarm):
        one()
    done, t0 = 0, time.perf_counter()
    while (nsteps and done < nsteps) or (not nsteps and time.perf_counter() - t0 < budget_s):
        one()
        done += 1
    return done, time.perf_counter() - t0


def run_oracle_windows(cfg, procs, nsteps=0, nwarm=1, budget_s=8.0, rows=WINDOW_ROWS):
    """The FP64 oracle on `procs` windows of the channel at once, one process per window
    (processes started with spawn). Returns the equivalent rate of the whole channel in
    hybrid steps/s (window steps/s summed over the processes, times rows / ncy), the summed
    window steps/s and the steps each process timed."""
    import multiprocessing as mp
    from oracle import build as OB
    OB.build()
    job = (cfg, rows, nsteps, nwarm, budget_s)
    if procs == 1:
        res = [oracle_window_worker(job)]
    else:
        with mp.get_context("spawn").Pool(procs) as pool:
            res = pool.map(oracle_window_worker, [job] * procs)
    win_rate = sum(n / t for n, t in res)
    return win_rate * rows / cfg["ncy"], win_rate, [n for n, _ in res]


def host_cores():
    """Cores of the host: os.cpu_count() and, where lscpu runs, its count."""
    n = os.cpu_count() or 1
    try:
        r = subprocess.run(["lscpu", "-p=CPU"], capture_output=True, text=True, timeout=10)
        cpus = [ln for ln in r.stdout.splitlines() if ln and not ln.startswith("#")]
        if cpus:
            n = min(n, len(cpus)) if n else len(cpus)
    except Exception:
        pass
    return n


def fp64_error_sample(h, cfg, B, cells_np, rows=WINDOW_ROWS):
    """The error of the GPU's results against the FP64 oracle at the benchmarked size.

    (1) LB2DSMC coefficients: the FP64 Grad records the GPU wrote at its last coupling step
    against the oracle's FP64 coefficients of the same populations, for every coupling cell.
    (2) One DSMC step and one LB step from the GPU's own current state: the state of the
    channel's first `rows` cell rows is loaded (in FP64) into an oracle window, both sides
    step, and the interior rows are compared: cells whose count agrees, particles within
    1e-5, the largest velocity error among the rest of the matching particles, the moment
    sums the step added (per particle), and the populations relative to w_a rho."""
    import torch
    from oracle import oracle as O
    d = h.d
    ncx, r, q = cfg["ncx"], cfg["lb_ratio"], d["q"]
    nx = d["nx"]
    e, w, _ = O.lattice(q)
    out = {}
    # (1) LB2DSMC coefficients of the last coupling step
    rho_g, nnew_g, v_g = h.grad_records(len(cells_np))
    y0 = int(cells_np.min()) // ncx
    y1 = int(cells_np.max()) // ncx + 1
    f = h.f()[:, y0 * r:y1 * r].double().cpu().numpy()  # the strip's node rows
    coef_err, rho_err = 0.0, 0.0
    for k, c in enumerate(cells_np):
        ix, iy = c % ncx, c // ncx - y0
        fb = f[:, iy * r:(iy + 1) * r, ix * r:(ix + 1) * r].reshape(q, -1).sum(1) / (r * r)
        g = O.grad_coeffs_packed(q, fb, 8)
        want = np.concatenate([g["a2"], g["a3"], g["u"], [g["C"]]])
        coef_err = max(coef_err, float(np.abs(v_g[k].numpy() - want).max()))
        rho_err = max(rho_err, abs(float(rho_g[k]) / g["rho"] - 1))
    out["lb2dsmc_coefficients"] = {"cells": int(len(cells_np)), "max_abs_err": coef_err,
                                   "rho_max_rel_err": rho_err,
                                   "gpu": "FP64 raw moments and centring identities",
                                   "oracle": "FP64 definition, left-to-right sums"}
    # (2) one step from the GPU's own state
    c1 = rows * ncx
    h.sync()
    cnt = h.counts()[:c1].cpu().numpy()
    arr = h.particle_arrays()
    mask = torch.arange(d["bin"], device=h.device)[None, :] < h.counts()[:c1, None]
    pk = {k: arr[k][:c1][mask].double().cpu().numpy() for k in ("x", "y", "vx", "vy", "vz")}
    cs = np.zeros(c1 + 1, np.int64)
    cs[1:] = np.cumsum(cnt)
    ctrl = h.ctrl().cpu().numpy()
    state = {"crmax": h.crmax()[:c1].double().cpu().numpy(), "rem": h.rem()[:c1].double().cpu().numpy(),
             "nbar": h.nbar_sum()[:c1].cpu().numpy().view(np.uint32).copy(),
             "acc": h.acc()[:c1].cpu().numpy().copy(),
             "f": h.f()[:, :rows * r].double().cpu().numpy().copy()}
    h.dsmc_step(1)
    h.lbm_step(1)
    h.sync()
    o, wcfg = window_oracle(cfg, rows, 8)
    o.set_particles(pk["x"], pk["y"], pk["vx"], pk["vy"], pk["vz"], cs.astype(np.uint32))
    o.set(O.A_CRMAX, state["crmax"])
    o.set(O.A_REM, state["rem"])
    o.set(O.A_NBAR_SUM, state["nbar"])
    o.set(O.A_ACC, state["acc"].reshape(-1))
    o.set_scalars(int(ctrl[B.CTRL_STEP]), int(ctrl[B.CTRL_NSAMPLES]))
    o.set_f(np.ascontiguousarray(state["f"]))
    o.dsmc_step(1)
    o.lbm_step(1)
    lo, hi = 5 * ncx, (rows - 5) * ncx  # rows at least 5 cells from the window's ends
    gcnt = h.counts()[lo:hi].cpu().numpy()
    ocs = o.get(O.A_CELL_START).astype(np.int64)
    ocnt = np.diff(ocs)[lo:hi]
    same = gcnt == ocnt
    arr = h.particle_arrays()
    gmask = torch.arange(d["bin"], device=h.device)[None, :] < h.counts()[lo:hi, None]
    gp = {k: arr[k][lo:hi][gmask].double().cpu().numpy() for k in ("x", "y", "vx", "vy", "vz")}
    op = o.particles()
    gcs = np.zeros(hi - lo + 1, np.int64)
    gcs[1:] = np.cumsum(gcnt)
    within, total, worst = 0, 0, 0.0
    dacc_err = 0.0
    ga_acc = h.acc()[lo:hi].cpu().numpy()
    oa_acc = o.acc()[lo:hi]
    base_acc = state["acc"][lo:hi]
    for j in np.nonzero(same)[0]:
        n = gcnt[j]
        if n == 0:
            continue
        a, b = gcs[j], ocs[lo + j]
        err = np.zeros(n)
        for k in ("x", "y", "vx", "vy", "vz"):
            gv, ov = gp[k][a:a + n], op[k][b:b + n]
            err = np.maximum(err, np.abs(gv - ov) / (1 + np.abs(ov)))
        total += n
        ok = err <= 1e-5
        within += int(ok.sum())
        if ok.all():
            worst = max(worst, float(err.max()))
            inc_g, inc_o = ga_acc[j] - base_acc[j], oa_acc[j] - base_acc[j]
            dacc_err = max(dacc_err, float(np.abs(inc_g - inc_o).max() / n))
    out["dsmc_step"] = {
        "cells": int(hi - lo), "cells_same_count_frac": float(same.mean()),
        "particles_within_1e-5_frac": within / max(1, total),
        "max_rel_err_of_cells_within_1e-5": worst,
        "moment_sums_step_max_err_per_particle": dacc_err,
        "note": "FP32 GPU step against the FP64 oracle from the same (FP32) state"}
    rl, rh = 3, rows * r - 3  # node rows the window's periodic ends do not reach in one step
    gf = h.f()[:, rl:rh].double().cpu().numpy()
    of = o.f()[:, rl:rh]
    rho = of.sum(0)
    out["lbm_step"] = {"node_rows": int(rh - rl),
                       "max_err_over_w_rho": float((np.abs(gf - of) / (w[:, None, None] * rho)).max()),
                       "rho_max_rel_err": float(np.abs(gf.sum(0) / rho - 1).max())}
    return out


def run_ensemble(args):
    """The batched ensemble against plain contexts: n independent channels advanced one hybrid
    step at a time, batched (one launch per kernel for all replicas, tuned block shapes) and
    plain (one context and graph per replica on one stream). Both start from the same states,
    take the same steps and end bit-identical (checked). Under torchrun every rank runs the
    same n channels with its own seeds (weak scaling) and the ranks sum the replicas' moment
    sums every step (one all-reduce: the ensemble average over the GPUs); the plain contexts
    are compared on one GPU only."""
    import torch
    import __graft_entry__ as G
    from paper_1512_08042_gb300 import binding as B

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
        if rank == 0:
            G.build()
        dist.barrier()
        if rank != 0:
            G.build()
    else:
        G.build()
    cfgs = W.ensemble_configs(args.ensemble, rank=rank)
    nodes, cells = zip(*[W.coupling_sites(c) for c in cfgs])
    nodes, cells = list(nodes), list(cells)
    dev = torch.device("cuda", local_rank)
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    tuner = B.Batch(cfgs, device=dev)
    tuner.tune(nodes, cells)
    shapes = tuner.blocks()
    tuner.close()
    batch = B.Batch(cfgs, device=dev)
    for k, v in shapes.items():
        batch.set_block(k, v)
    stream = batch.stream
    plain = [B.Hybrid(c, stream=stream, device=dev) for c in cfgs] if world == 1 else []
    pn = [torch.from_numpy(x).to(dev) for x in nodes]
    pc = [torch.from_numpy(x).to(dev) for x in cells]
    acc_sum = batch.moment_sums() if world > 1 else None

    def step_batch():
        batch.hybrid_step(nodes, cells, nsteps=1, use_graph=True)
        if world > 1:
            with torch.cuda.stream(stream):
                batch.moment_sums(acc_sum)
                dist.all_reduce(acc_sum)

    def step_plain():
        for h, a, b in zip(plain, pn, pc):
            h.hybrid_step(a, b, nsteps=1, use_graph=True, order_inputs=False)

    def timed(step):
        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize(dev)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        for a, b in ev:
            with torch.cuda.stream(stream):
                flush.zero_()
            a.record(stream)
            step()
            b.record(stream)
        torch.cuda.synchronize(dev)
        return sum(a.elapsed_time(b) for a, b in ev) / args.steps

    if dist:
        dist.barrier()
    ms_b = timed(step_batch)
    if dist:
        ms_b = max_over_ranks(dist, ms_b, dev)
        dist.barrier()
        line = {
            "metric": "ensemble hybrid steps/s (every replica of every rank advanced one hybrid step)",
            "value": world * 1e3 / ms_b, "unit": "ensemble steps/s (a rank's ensemble, times ranks)",
            "higher_is_better": True, "ms_per_step": ms_b, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "scaling": "weak", "dtype": "f32", "data": "synthetic",
            "config": {"workload": "ensemble of %d channels per rank (H 32-256 cells, 20-100 ppc, "
                                   "Kn 0.01-0.5), each rank its own seeds" % len(cfgs),
                       "replicas_per_rank": len(cfgs), "block_shapes": shapes,
                       "collective": "all-reduce (sum) of the replicas' FP64 moment sums every step",
                       "l2": "flushed before every timed step (512 MB write)"},
        }
        if rank == 0:
            print(json.dumps(line), flush=True)
        batch.close()
        dist.destroy_process_group()
        return
    ms_p = timed(step_plain)
    identical = True
    for g, h in zip(batch.replicas, plain):
        pg, ph = g.particles(), h.particles()
        identical &= all(torch.equal(pg[k], ph[k]) for k in pg)
        identical &= torch.equal(g.f(), h.f()) and torch.equal(g.acc(), h.acc())
    particles = sum(c["ncx"] * c["ncy"] * c["ppc"] for c in cfgs)
    line = {
        "metric": "ensemble hybrid steps/s (every replica advanced one hybrid step)",
        "value": 1e3 / ms_b, "unit": "ensemble steps/s", "higher_is_better": True,
        "ms_per_step": ms_b, "plain": {"value": 1e3 / ms_p, "ms_per_step": ms_p,
                                       "launches": "%d contexts, one graph each" % len(cfgs)},
        "speedup_vs_plain": ms_p / ms_b, "identical_to_plain": bool(identical),
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": "ensemble of %d channels (H 32-256 cells, 20-100 ppc, Kn 0.01-0.5)"
                               % len(cfgs), "replicas": len(cfgs), "particles": particles,
                   "block_shapes": shapes,
                   "l2": "flushed before every timed step (512 MB write)"},
    }
    print(json.dumps(line), flush=True)
    batch.close()


def run_adjoint(args):
    """The differentiated LBM against the plain forward on the same GPU: one gradient of the
    coupling-interface loss (2000 LB steps with per-node force and relaxation time, forward
    with checkpoints every 100 steps, then recomputation and the adjoint step in reverse)
    against the same 2000 forward steps alone; plus the adjoint kernel's achieved bandwidth
    and the FP32 gradient's error against an FP64 gradient."""
    import torch
    import __graft_entry__ as G
    G.build()
    from paper_1512_08042_gb300 import binding as B

    cfg = dict(W.DIFF_LBM, real_bytes=4)
    T, K = W.DIFF_LBM_STEPS, W.DIFF_LBM_CKPT
    dev = torch.device("cuda", 0)
    h = B.Hybrid(cfg, device=dev)
    d = h.d
    e, w, r = B.lattice(cfg["lattice"])
    f0, sg, st, nodes_np, _ = W.diff_lbm_inputs(cfg, w)
    # targets sampled from the DSMC gas of the same channel: 200 DSMC steps, then the Grad
    # coefficients of the cell holding each coupling node
    h.dsmc_step(200)
    h.sync()
    nsamples = int(h.ctrl().cpu()[B.CTRL_NSAMPLES])
    node_cells = (nodes_np // d["nx"]) // cfg["lb_ratio"] * cfg["ncx"] + (nodes_np % d["nx"]) // cfg["lb_ratio"]
    targets_np = W.grad_targets_from_sums(h.acc().cpu().numpy(), nsamples, cfg["ppc"], node_cells)
    shape = (d["q"], d["ny"], d["nx"])
    mk = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a).astype(dt)).to(dev)
    f = mk(f0, np.float32).reshape(shape)
    g = mk(d["g_step"] * (1 + sg), np.float32)
    tau = mk(d["tau"] * (1 + st), np.float32)
    nodes = mk(nodes_np, np.int32)
    targets = mk(targets_np, np.float32)
    stream = h.stream

    def grad(hh, ff, gg, tt, tg):
        gg = gg.clone().requires_grad_(True)
        tt = tt.clone().requires_grad_(True)
        L = B.interface_loss(hh, gg, tt, ff, nodes, tg, T, K)
        L.backward()
        return L, gg.grad, tt.grad

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize(dev)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize(dev)
        return a.elapsed_time(b) / reps

    def forward_only():
        # the same one-call forward as the gradient's, without its checkpoints
        x, y = f.clone(), torch.empty_like(f)
        h.lbm_steps_nodes(x, y, g, tau, T, T)

    reps = max(1, min(args.steps, 5))
    ms_fwd = timed(forward_only, reps)
    ms_grad = timed(lambda: grad(h, f, g, tau, targets), reps)
    # the adjoint step alone, 200 steps on fixed inputs
    lam_a, lam_b = torch.rand_like(f), torch.empty_like(f)
    gg, gt = torch.zeros_like(g), torch.zeros_like(tau)
    wall = torch.zeros(h.wall_scratch_size(), dtype=torch.float32, device=dev)

    def adj200():
        for _ in range(200):
            h.lbm_adjoint_step(f, lam_a, lam_b, g, tau, gg, gt, wall)

    ms_adj = timed(adj200, 1) / 200
    bytes_adj = d["nnodes"] * (3 * d["q"] * 4 + 4 * 4 + 2 * 4)
    peak, peak_kind = measured_peak_hbm()
    # accuracy of the FP32 gradient against FP64
    cfg64 = dict(cfg, real_bytes=8)
    h64 = B.Hybrid(cfg64, device=dev)
    L32, g32, t32 = grad(h, f, g, tau, targets)
    L64, g64, t64 = grad(h64, f.double(), g.double(), tau.double(), targets.double())
    torch.cuda.synchronize(dev)
    err = lambda a, b: float((a.double() - b).abs().max() / b.abs().max())
    line = {
        "metric": "differentiated LBM: interface-loss gradients/s (2000 LB steps, checkpoints every 100)",
        "value": 1e3 / ms_grad, "unit": "gradients/s", "higher_is_better": True,
        "ms_per_gradient": ms_grad, "forward_only": {"ms": ms_fwd, "lb_steps_per_s": T * 1e3 / ms_fwd,
                                                    "mlups": T * d["nnodes"] / (ms_fwd * 1e3)},
        "gradient_over_forward": ms_grad / ms_fwd,
        "adjoint_step": {"us": ms_adj * 1e3, "achieved_gbs": bytes_adj / (ms_adj * 1e-3) / 1e9,
                         "peak_gbs": peak, "peak_kind": peak_kind,
                         "frac": bytes_adj / (ms_adj * 1e-3) / 1e9 / peak,
                         "bytes_per_node": bytes_adj / d["nnodes"]},
        "fp32_vs_fp64": {"loss_rel": abs(L32.item() - L64.item()) / abs(L64.item()),
                         "grad_g_rel_maxnorm": err(g32, g64), "grad_tau_rel_maxnorm": err(t32, t64)},
        "n_gpus": 1, "steps": reps, "dtype": "f32",
        "data": "synthetic populations; targets sampled from 200 DSMC steps of the same channel",
        "config": {"workload": "differentiated LBM, 256 x 128 D3Q39, %d steps, checkpoints every %d"
                               % (T, K), "coupling_nodes": int(len(nodes_np)),
                   "l2": "inputs not flushed: every gradient sweeps 2000 states"},
    }
    print(json.dumps(line), flush=True)
    h.close()
    h64.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(W.WORKLOADS))
    ap.add_argument("--no-graph", action="store_true")
    ap.add_argument("--collide-block", default="tune", choices=["tune", "4", "8"],
                    help="the collide's block shape in warps (multi-step fusion automatic), or both "
                         "picked by the library's tuner before the warm-up (hyb_tune_collide)")
    ap.add_argument("--profile-kernel", default=None)
    ap.add_argument("--cpu-budget", type=float, default=16.0)
    ap.add_argument("--replicas", action="store_true",
                    help="with several GPUs, independent replicas instead of streamwise slabs")
    ap.add_argument("--no-cpu", action="store_true",
                    help="skip the FP64 oracle error sample and the CPU baseline")
    ap.add_argument("--profile-steps", type=int, default=0,
                    help="run this many hybrid steps with direct launches and exit (for ncu)")
    ap.add_argument("--adjoint", action="store_true",
                    help="time the differentiated LBM (gradient vs forward) on the 256 x 128 lattice")
    ap.add_argument("--ensemble", type=int, default=0,
                    help="time a batched ensemble of this many channels against plain contexts")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.ensemble:
        run_ensemble(args)
        return
    if args.adjoint:
        run_adjoint(args)
        return

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1 and args.impl == "ours" and not args.replicas:
        # several GPUs: the channel in streamwise slabs, one per rank
        import torch
        import torch.distributed as tdist
        import __graft_entry__ as G
        if rank == 0:
            G.build()
        tdist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
        tdist.barrier()
        if rank != 0:
            G.build()
        line = run_slab_rank(args, W.WORKLOADS[args.workload], rank, world, local_rank, tdist)
        if rank == 0:
            print(json.dumps(line), flush=True)
        tdist.destroy_process_group()
        return
    cfg = replica_config(W.WORKLOADS[args.workload], rank)
    nodes_np, cells_np = W.coupling_sites(cfg)

    if args.impl == "reference":
        if rank != 0:
            return
        d = __import__("oracle.oracle", fromlist=["x"]).derive(cfg)
        n = d["ncells"] * cfg["ppc"]
        procs = host_cores()
        # one step = one hybrid step of a window of the channel in every process
        rate, win_rate, done = run_oracle_windows(cfg, procs, nsteps=args.steps,
                                                  nwarm=args.warmup)
        sample = ("%d processes, each an FP64 oracle window of the channel's first %d cell rows "
                  "(%d particles, %d LB node rows, its own 4-row coupling strip); %d timed hybrid "
                  "steps per process after %d warm-up steps; rate scaled to the whole channel by "
                  "rows" % (procs, WINDOW_ROWS, WINDOW_ROWS * cfg["ncx"] * cfg["ppc"],
                            WINDOW_ROWS * cfg["lb_ratio"], done[0], args.warmup))
        line = {
            "impl": "reference", "metric": METRIC, "value": rate, "unit": "hybrid steps/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 / rate, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64",
            "precision": "oracle: FP64 state and arithmetic throughout",
            "data": "synthetic",
            "config": {"workload": args.workload, "particles": n, "lb_nodes": d["nnodes"]},
            "dsmc_particle_updates_per_s": rate * n,
            "cpu_baseline": {"value": rate, "unit": "hybrid steps/s", "cores": procs,
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": rate, "unit": "hybrid steps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0},
        }
        print(json.dumps(line), flush=True)
        return

    import torch
    import __graft_entry__ as G
    G.build() if rank == 0 else None
    dist = None
    if world > 1:
        import torch.distributed as tdist
        dist = tdist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
        dist.barrier()
        if rank != 0:
            G.build()
    from paper_1512_08042_gb300 import binding as B

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    h = B.Hybrid(cfg, device=dev)
    d = h.d
    n_particles = d["ncells"] * cfg["ppc"]
    nodes = torch.from_numpy(nodes_np).to(dev)
    cells = torch.from_numpy(cells_np).to(dev)
    use_graph = not args.no_graph
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = h.stream
    torch.cuda.synchronize(dev)

    def step():
        h.hybrid_step(nodes, cells, nsteps=1, use_graph=use_graph, order_inputs=False)

    def run(n, graph=use_graph):
        # n hybrid steps in one call: the DSMC passes fused across steps
        h.hybrid_step(nodes, cells, nsteps=n, use_graph=graph, order_inputs=False)

    # the collide's block shape (the same results either way): the tuner times both on a
    # second context of this channel from the same initial state (it advances the context it
    # times), outside the timed region
    fuse = "auto"
    if args.collide_block == "tune":
        tuner = B.Hybrid(cfg, device=dev)
        collide_warps, fuse = tuner.tune_collide(nodes, cells)
        tuner.close()
        del tuner
        torch.cuda.empty_cache()
    else:
        collide_warps = int(args.collide_block)
    h.set_collide_block(collide_warps)
    h.set_fuse(fuse)

    if args.profile_steps:
        run(args.profile_steps, graph=False)
        rc, bits = h.sync_status()
        print(json.dumps({"profile_steps": args.profile_steps, "status": rc, "bits": bits}))
        h.close()
        return

    # warm-up (the first fused call of args.steps captures its graph), then every kernel's
    # average time per launch over fused runs of direct launches with CUDA events on the
    # library's stream (kernel timing is taken apart from the timed region)
    for _ in range(args.warmup):
        step()
    run(args.steps)
    h.sync()
    kernel_ms, kernel_launches = {}, {}
    prof_steps = 6
    for name, kid in B.KERNELS.items():
        h.profile(kid)
        h.profile_harvest()
        ms0, n0 = h.profile_read()
        with torch.cuda.stream(stream):
            flush.zero_()
        run(prof_steps, graph=False)
        h.profile_harvest()
        ms1, n1 = h.profile_read()
        if n1 > n0:
            kernel_ms[name] = (ms1 - ms0) / (n1 - n0)
            kernel_launches[name] = (n1 - n0) / prof_steps
    h.profile(-1)
    # the dominant kernel of a step of the timed (fused) run
    # (a channel too small to fill the GPU with the fused pass takes a move and a collide per
    # step: the library's automatic choice)
    kinds = ("fused",) if "fused" in kernel_ms else ("move", "collide")
    per_step = {k: kernel_ms[k] for k in kinds + ("lbm", "dsmc2lb", "lb2dsmc") if k in kernel_ms}
    dominant = args.profile_kernel or max(per_step, key=per_step.get)
    dom_ms = kernel_ms[dominant]

    # single steps (one call per step, L2 flushed before each), for comparison
    single_ms = []
    for _ in range(min(args.steps, 20)):
        with torch.cuda.stream(stream):
            flush.zero_()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        step()
        a1.record(stream)
        single_ms.append((a0, a1))
    torch.cuda.synchronize(dev)
    single_ms = sum(x.elapsed_time(y) for x, y in single_ms) / len(single_ms)

    # timed region: args.steps hybrid steps in one call, inputs larger than L2 (and the L2
    # flushed before the region)
    clock_lines, stop = [], threading.Event()
    th = threading.Thread(target=sample_clocks, args=(stop, clock_lines), daemon=True)
    th.start()
    time.sleep(0.3)
    with torch.cuda.stream(stream):
        flush.zero_()
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    run(args.steps)
    t_end.record(stream)
    torch.cuda.synchronize(dev)
    total_ms = t_start.elapsed_time(t_end)
    if dist:
        total_ms = max_over_ranks(dist, total_ms, dev)
        dist.barrier()
    stop.set()
    th.join(timeout=5)
    rc, bits = h.sync_status()

    # end to end through the C-ABI calls with host buffers: every step copies the coupling
    # lists in from page-locked host memory and the strip's moment sums and the status word
    # out (two of the library's kernels per step, which read and write the host buffers
    # through their device addresses; the call is one CUDA graph). The headline form takes E2E_CALL steps per call (hyb_hybrid_steps_host: the DSMC
    # passes fused across the call's steps as in the device-timed run), pipelined: the host
    # reads call j's results (two result buffers) while call j + 1 runs. One step per call
    # (hyb_hybrid_step_host), pipelined and synchronous, is reported beside it.
    h.profile(-1)
    pin_nodes = torch.from_numpy(nodes_np).pin_memory()
    pin_cells = torch.from_numpy(cells_np).pin_memory()
    e2e_steps = max(20 * E2E_CALL, args.steps)  # at least 20 calls: the pipeline's fill is amortised

    def e2e_run(per_call, pipelined, seen):
        out_acc = [torch.empty(per_call, len(cells_np), 20, dtype=torch.float64).pin_memory() for _ in range(2)]
        out_status = [torch.zeros(per_call, dtype=torch.int32).pin_memory() for _ in range(2)]
        acc_np = [t.numpy() for t in out_acc]
        st_np = [t.numpy() for t in out_status]

        def read(b):
            seen["n"] = float(acc_np[b][-1][:, 0].sum())  # the strip's sampled particle count
            seen["bad"] |= int(np.bitwise_or.reduce(st_np[b]))

        calls = max(1, e2e_steps // per_call)
        h.host_wait(0)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for k in range(calls):
            b = k % 2
            h.hybrid_step_host(pin_nodes, pin_cells, out_acc[b], out_status[b], nsteps=per_call)
            if pipelined:
                if k > 0:
                    h.host_wait(1)
                    read(1 - b)
            else:
                h.host_wait(0)
                read(b)
        if pipelined:
            h.host_wait(0)
            read((calls - 1) % 2)
        return calls * per_call / (time.perf_counter() - t0)

    seen = {"n": 0.0, "bad": 0}
    e2e_run(E2E_CALL, True, seen)  # first use: staging allocation
    e2e_rate = e2e_run(E2E_CALL, True, seen)
    e2e_run(1, True, seen)  # graph capture of the one-step call
    e2e_one_sync = e2e_run(1, False, seen)
    e2e_one = e2e_run(1, True, seen)
    h2d = pin_nodes.numel() * 4 + pin_cells.numel() * 4
    d2h = len(cells_np) * 20 * 8 + 4

    value = world * args.steps / (total_ms / 1e3)
    peak, peak_kind = measured_peak_hbm()
    dsmc_b, lbm_b = method_bytes(cfg, d)
    units = {"move": n_particles * dsmc_b, "collide": n_particles * dsmc_b,
             "fused": n_particles * dsmc_b, "lbm": d["nnodes"] * lbm_b}
    alg_design = kernel_algorithmic_bytes(dominant, cfg, d, n_particles, len(nodes_np), len(cells_np))
    alg = units.get(dominant, alg_design)
    achieved = alg / (dom_ms / 1e3) / 1e9 if dom_ms > 0 else None
    step_bytes = n_particles * dsmc_b + d["nnodes"] * lbm_b
    step_ms = total_ms / args.steps / world
    dsmc_ms = kernel_ms.get("fused", 0.0)
    line = {
        "metric": METRIC, "value": value, "unit": "hybrid steps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if cfg["real_bytes"] == 4 else "f64", "data": "synthetic",
        "config": {"workload": args.workload, "particles": n_particles, "lb_nodes": d["nnodes"],
                   "lattice": "D3Q%d" % d["q"], "coupling_nodes": len(nodes_np),
                   "coupling_cells": len(cells_np), "graph": use_graph,
                   "collide_block_warps": collide_warps, "fuse": fuse,
                   "kn": [cfg["kn"], cfg.get("kn_end", cfg["kn"])] if cfg.get("kn_profile") else cfg["kn"],
                   "l2": "inputs larger than L2, and flushed before every timed step (512 MB write)",
                   "parallelism": "replicas" if world > 1 else "single"},
        "dsmc_particle_updates_per_s": value * n_particles,
        "lbm_mlups": value * d["nnodes"] / 1e6,
        "roofline": {"kernel": dominant, "bound": "hbm", "achieved": achieved, "peak": peak,
                     "peak_kind": peak_kind, "unit": "GB/s",
                     "frac": achieved / peak if achieved else None,
                     "algorithmic_bytes_per_launch": alg,
                     "bytes_basis": "method bytes per unit (%.1f B per particle-update, %d B per "
                                    "node-update) x units per launch" % (dsmc_b, lbm_b)
                                    if dominant in units else "design bytes (no method figure)",
                     "ms_per_launch": dom_ms,
                     "traffic": traffic_record(dominant, args.workload,
                                               n_particles if dominant in ("move", "collide", "fused")
                                               else d["nnodes"]),
                     "design_bytes_per_launch": alg_design,
                     "design_frac": (alg_design / (dom_ms / 1e3) / 1e9 / peak) if dom_ms > 0 else None},
        "roofline_step": {"bytes_per_step": step_bytes, "achieved": step_bytes / (step_ms / 1e3) / 1e9,
                          "peak": peak, "unit": "GB/s",
                          "frac": step_bytes / (step_ms / 1e3) / 1e9 / peak,
                          "steps_per_s_at_peak": peak * 1e9 / step_bytes,
                          "dsmc_frac": (n_particles * dsmc_b) / (dsmc_ms / 1e3) / 1e9 / peak
                          if dsmc_ms > 0 else None,
                          "lbm_frac": (d["nnodes"] * lbm_b) / (kernel_ms["lbm"] / 1e3) / 1e9 / peak
                          if kernel_ms.get("lbm") else None,
                          "note": "per-kernel times are CUDA-event brackets taken apart from the "
                                  "timed steps (upper bounds: they break the overlap of "
                                  "programmatic dependent launch)"},
        "kernel_ms": kernel_ms,
        "kernel_launches_per_step": kernel_launches,
        "single_step": {"ms_per_step": single_ms, "value": world * 1e3 / single_ms,
                        "note": "one call per hybrid step (move and collide as two passes), "
                                "L2 flushed before each"},
        "clocks": summarize_clocks(clock_lines),
        "gpu_launches": launches_in_call(args.steps, "fused" in kernel_ms, len(nodes_np), len(cells_np)),
        "status": {"code": rc, "bits": bits},
        "e2e": {"value": world * e2e_rate, "unit": "hybrid steps/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "api": "hyb_hybrid_steps_host, %d steps per call (every step: host lists in, "
                       "strip moments and status out)" % E2E_CALL,
                "mode": "pipelined: the host reads a call's results while the next call runs",
                "transfers": "page-locked host buffers read and written by two library kernels per "
                             "step through their device addresses; each call one CUDA graph",
                "gpu_launches_per_call": launches_in_call(E2E_CALL, "fused" in kernel_ms, len(nodes_np),
                                                          len(cells_np)) + 2 * E2E_CALL,
                "one_step_per_call": {"api": "hyb_hybrid_step_host", "value": world * e2e_one,
                                      "synchronous_value": world * e2e_one_sync},
                "status_bits_seen": seen["bad"]},
    }
    if rank == 0 and world == 1 and not args.no_cpu:
        # the FP64 oracle: its error against the GPU at this size, then its speed on windows
        # of the channel, single-threaded and in one process per host core
        line["error_vs_fp64_oracle"] = fp64_error_sample(h, cfg, B, cells_np)
        rate1, win1, done1 = run_oracle_windows(cfg, 1, budget_s=args.cpu_budget / 2)
        procs = host_cores()
        rate_n, win_n, done_n = run_oracle_windows(cfg, procs, budget_s=args.cpu_budget / 2)
        line["cpu_baseline"] = {
            "value": rate_n, "unit": "hybrid steps/s", "cores": procs, "kind": "oracle",
            "sample": "FP64 oracle windows of the channel's first %d cell rows (%d particles, "
                      "its own 4-row coupling strip), one process per core, %d hybrid steps each "
                      "in %.0f s; rate scaled to the whole channel by rows"
                      % (WINDOW_ROWS, WINDOW_ROWS * cfg["ncx"] * cfg["ppc"], min(done_n),
                         args.cpu_budget / 2),
            "single_thread": {"value": rate1, "cores": 1,
                              "particle_updates_per_s": win1 * WINDOW_ROWS * cfg["ncx"] * cfg["ppc"]},
            "particle_updates_per_s": win_n * WINDOW_ROWS * cfg["ncx"] * cfg["ppc"]}
    if rank == 0:
        print(json.dumps(line), flush=True)
    h.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
