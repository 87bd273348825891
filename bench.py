#!/usr/bin/env python
"""Benchmark of the batched block solves of the 4D domain decomposition.

Workload (one step): x = D_{Omega0^a}^{-1} b for every framed block Omega0^a
of a 32^4 lattice (256 blocks of 9^4 sites: 7^4 cores and a one-site frame)
and 12 Gaussian right-hand sides per block (3072 systems, 20.15 M site-rhs),
kappa = 0.135, links exp(i 0.5 H) with seed 2, every system solved to
|b - D x| <= 1e-10 |b| with the FP32 inner BiCGstab and FP64 defect
correction of libdd4d.  Inputs are resident on the GPU when the timed region
starts and are larger than L2.  The line also reports the plain FP64 solve
of the same batch, the stencil's roofline, the multi-boson action rate on the
8^4 lattice, an end-to-end number through the C ABI with host buffers, and
the FP64 CPU oracle on a bounded sample (the reference arm).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun each rank solves its own batch (weak scaling, no collective on
the data path); rank 0 prints the JSON line.
"""

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

LATTICE = (32, 32, 32, 32)
KAPPA, EPS, SEED = 0.135, 0.5, 2
CORE, FRAME, NRHS = 7, 1, 12
TOL = 1e-10
CSW = 1.0            # clover coefficient of the clover side figure
WORKLOAD = ("32^4 Wilson-Dirac (kappa 0.135, links exp(i 0.5 H), seed 2): 256 framed blocks "
            "Omega0^a of 9^4 sites (7^4 cores, frame 1) x 12 Gaussian rhs = 3072 block "
            "systems solved to 1e-10")
METRIC = "block-solve sites/s to 1e-10"
UNIT = "site-rhs/s"


def cores_uniform(L, core, frame):
    out = []
    for mu in range(4):
        period = core + frame
        out.append([(i * period, i * period + core - 1) for i in range(L[mu] // period)])
    return out


def site_rhs():
    nb = 1
    for mu in range(4):
        nb *= LATTICE[mu] // (CORE + FRAME)
    return nb * (CORE + 2 * FRAME) ** 4 * NRHS


# ---------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile(mode="w+", suffix=".csv", delete=False)
            cmd = ["nvidia-smi", "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                   "-lms", "200"]
            if self.gpu_id is not None:
                cmd += ["-i", str(self.gpu_id)]
            self.proc = subprocess.Popen(cmd, stdout=self.file, stderr=subprocess.DEVNULL)
        except (OSError, ValueError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.file.flush()
        rows = []
        with open(self.file.name) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 7:
                    rows.append(parts)
        os.unlink(self.file.name)
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[3 + k] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


def gpu_smi_id(torch, dev):
    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        vis = os.environ.get("CUDA_VISIBLE_DEVICES")
        return vis.split(",")[dev] if vis else dev


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def traffic_record():
    """ncu DRAM bytes per launch of the FP32 hop kernel (profiles/), or None."""
    path = os.path.join(ROOT, "profiles", "hop_lb_f32_traffic.json")
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return None


# ---------------------------------------------------------------------------
# The FP64 CPU oracle on a bounded sample of the workload, on every host core:
# one worker process per core, each with its own framed block (links copied
# from the workload's lattice into a box with one spare layer, so the
# restricted operator D_Omega is the same matrix), its own 2 Gaussian rhs, the
# matrix assembled before the timed region, the oracle's BiCGstab to 1e-13
# inside it.  All workers start the timed region together (a barrier); the wall
# time is from the first start to the last finish.  The systems are all alike,
# so the full batch of 3072 systems takes (3072 / sample systems) times as long.
SAMPLE_RHS = 2


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _sample_blocks(n):
    """n framed blocks whose boxes do not cross the lattice boundary."""
    per = LATTICE[0] // (CORE + FRAME)
    out = []
    for k in range(per ** 4):
        idx = [(k // per ** (3 - m)) % per for m in range(4)]
        if min(idx) >= 1:
            out.append(idx)
        if len(out) == n:
            break
    return out


def _block_box(U, idx):
    """Links of a framed block's box (9^4 sites) in a 10^4 array with an identity spare layer."""
    side = CORE + 2 * FRAME
    org = [(CORE + FRAME) * i - FRAME for i in idx]
    box = np.zeros((side + 1,) * 4 + (4, 3, 3), dtype=np.complex128)
    box[...] = np.eye(3)
    sl = tuple(slice(o, o + side) for o in org)
    box[:side, :side, :side, :side] = U[sl]
    return box


def _oracle_worker(box, k, barrier, q):
    from oracle.dd import DomainSolver
    from paper_2211_06902_gb300 import synth
    side = CORE + 2 * FRAME
    mask = np.zeros(box.shape[:4], dtype=bool)
    mask[:side, :side, :side, :side] = True
    sol = DomainSolver(box, KAPPA, mask)                      # assembly: outside the timed region
    n = len(sol.sites)
    b = synth.complex_gaussian(SEED, synth.TAG_RHS + k, (SAMPLE_RHS, 12 * n))
    barrier.wait()
    t0 = time.monotonic()
    for r in range(SAMPLE_RHS):
        sol.solve_vec(b[r])
    q.put((t0, time.monotonic(), SAMPLE_RHS * n))


def oracle_parallel(U, runs):
    """Wall times of ``runs`` parallel runs of the sample, site-rhs per run, workers."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    nw = host_cores()
    boxes = [_block_box(U, idx) for idx in _sample_blocks(nw)]
    nw = len(boxes)
    walls, units = [], 0
    # one thread per worker: the spawned interpreters read these when they import numpy
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in saved:
        os.environ[k] = "1"
    try:
        walls, units = _parallel_runs(ctx, boxes, runs)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    return walls, units, nw


def _parallel_runs(ctx, boxes, runs):
    nw = len(boxes)
    walls, units = [], 0
    for _ in range(runs):
        barrier = ctx.Barrier(nw)
        q = ctx.Queue()
        procs = [ctx.Process(target=_oracle_worker, args=(boxes[k], k, barrier, q)) for k in range(nw)]
        for pr in procs:
            pr.start()
        res = [q.get() for _ in range(nw)]
        for pr in procs:
            pr.join()
        walls.append(max(r[1] for r in res) - min(r[0] for r in res))
        units = sum(r[2] for r in res)
    return walls, units


def cpu_sample_text(nw, wall, runs):
    full = site_rhs() // ((CORE + 2 * FRAME) ** 4)          # systems in the full batch
    return ("%d framed 9^4 blocks x %d rhs (%d of the %d systems), one worker process per "
            "host core; oracle BiCGstab to 1e-13 on the assembled sparse D_Omega, assembly "
            "outside the timed region; median wall %.2f s over %d runs; the full batch "
            "extrapolates linearly to %.0f s" % (nw, SAMPLE_RHS, nw * SAMPLE_RHS, full, wall, runs,
                                                   wall * full / (nw * SAMPLE_RHS)))


def cpu_baseline_entry(U):
    walls, units, nw = oracle_parallel(U, 3)
    wall = statistics.median(walls)
    return {"value": units / wall, "unit": UNIT, "cores": nw, "kind": "oracle",
            "sample": cpu_sample_text(nw, wall, len(walls))}


# ---------------------------------------------------------------------------
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from paper_2211_06902_gb300 import synth
    U = synth.gauge_field(LATTICE, EPS, SEED)
    if args.warmup:
        oracle_parallel(U, args.warmup)
    walls, units, nw = oracle_parallel(U, args.steps)
    t = sum(walls) / len(walls)
    value = units / t
    sample = cpu_sample_text(nw, statistics.median(walls), len(walls))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": "per step: " + sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": nw, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2211_06902_gb300 import dd4d, ranks, synth

    world, rank, local = ranks.rank_info()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    torch.cuda.init()
    dev = torch.device("cuda", local)

    def barrier():
        ranks.barrier(world)
        torch.cuda.synchronize()

    if not os.path.exists(dd4d.LIB_PATH):
        from paper_2211_06902_gb300 import build
        build.build()

    U = synth.gauge_field(LATTICE, EPS, SEED)
    ctx = dd4d.Context(LATTICE, KAPPA)
    ctx.gauge_upload(U)
    info = ctx.set_geometry(cores_uniform(LATTICE, CORE, FRAME))
    ids = list(range(info["nblocks"]))
    n_om = info["max_omega"]
    b_h = synth.complex_gaussian(ranks.batch_seed(SEED, rank), synth.TAG_RHS, (len(ids), NRHS, n_om, 12))
    b = torch.from_numpy(b_h.view(np.float64)).to(dev)
    x = torch.zeros_like(b)
    units = site_rhs()
    assert units == len(ids) * NRHS * n_om
    mixed = dd4d.params(TOL, inner_prec="f32", inner_tol=args.inner_tol, check_every=8,
                        autotune=True)
    plain = dd4d.params(TOL, inner_prec="f64", check_every=8)

    def step(prm):
        st = ctx.solve_blocks("omega", ids, NRHS, b, x, prm)
        if st["status"] != 0 or st["max_relres"] > TOL:
            raise RuntimeError("solve missed tolerance: %s" % st)
        return st

    for _ in range(args.warmup):
        step(mixed)
    stream = torch.cuda.current_stream()
    sampler = ClockSampler(gpu_smi_id(torch, local))
    barrier()
    sampler.start()
    time.sleep(0.3)
    ctx.timing_enable(True)
    ctx.timing_get(0)
    ctx.timing_get(1)
    launches0 = dd4d.launch_count()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    stats = None
    for _ in range(args.steps):
        stats = step(mixed)
    e1.record(stream)
    barrier()
    ms = e0.elapsed_time(e1) / args.steps
    launches = dd4d.launch_count() - launches0
    hop32_ms, hop32_n, hop32_bytes = ctx.timing_get(1)
    hop64_ms, hop64_n, hop64_bytes = ctx.timing_get(0)
    ctx.timing_enable(False)
    clocks = sampler.stop()
    ms = ranks.max_over_ranks(ms, world, dev)
    value = ranks.aggregate_rate(units, world, ms * 1e-3)

    # plain FP64 form of the same batch (the reference form of the ratio)
    step(plain)
    p0 = torch.cuda.Event(enable_timing=True)
    p1 = torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    pst = step(plain)
    p1.record(stream)
    torch.cuda.synchronize()
    plain_ms = p0.elapsed_time(p1)

    # the same mixed solve with each inner solve as one graph launch (device-side loop)
    loop_prm = dd4d.params(TOL, inner_prec="f32", inner_tol=args.inner_tol, autotune=True, graph_loop=True)
    step(loop_prm)
    l0 = torch.cuda.Event(enable_timing=True)
    l1 = torch.cuda.Event(enable_timing=True)
    la = dd4d.launch_count()
    l0.record(stream)
    lst = step(loop_prm)
    l1.record(stream)
    torch.cuda.synchronize()
    device_loop = {"ms_per_step": l0.elapsed_time(l1), "max_iters": lst["max_iters"],
                   "max_relres": lst["max_relres"], "kernel_launches_per_step": dd4d.launch_count() - la,
                   "host_polls_per_inner_solve": 0}
    # the whole solve (outer cycles included) as one graph launch
    solve_prm = dd4d.params(TOL, inner_prec="f32", inner_tol=args.inner_tol, autotune=True, graph_solve=True)
    step(solve_prm)
    la = dd4d.launch_count()
    l0.record(stream)
    gst = step(solve_prm)
    l1.record(stream)
    torch.cuda.synchronize()
    whole_graph = {"ms_per_step": l0.elapsed_time(l1), "value": world * units / (l0.elapsed_time(l1) * 1e-3),
                   "max_iters": gst["max_iters"], "outer_cycles": gst["outer_cycles"],
                   "max_relres": gst["max_relres"], "kernel_launches_per_step": dd4d.launch_count() - la,
                   "graph_launches_per_step": 1, "host_polls_per_step": 0}

    # BF16-storage inner solve of the same batch (FP32 arithmetic, double-float residuals)
    bf16 = None
    if rank == 0:
        bprm = dd4d.params(TOL, inner_prec="bf16", inner_tol=1e-3, check_every=8, autotune=True)
        try:
            step(bprm)
            q0 = torch.cuda.Event(enable_timing=True)
            q1 = torch.cuda.Event(enable_timing=True)
            q0.record(stream)
            qst = step(bprm)
            q1.record(stream)
            torch.cuda.synchronize()
            bms = q0.elapsed_time(q1)
            bf16 = {"value": units / (bms * 1e-3), "ms_per_step": bms, "inner_tol": 1e-3,
                    "max_iters": qst["max_iters"], "outer_cycles": qst["outer_cycles"],
                    "max_relres": qst["max_relres"], "hop_variant": dd4d.hop_variant_name("bf16", qst["hop_variant"])}
        except (dd4d.DDError, RuntimeError) as err:
            bf16 = {"unavailable": str(err)[:200]}

    learned = None
    if rank == 0 and not args.no_learned:
        learned = learned_ab(dd4d, synth, torch, ctx, ids, b, x, units, ms)
        learned["max_iters_without"] = stats["max_iters"]
        # the learned mixed-precision forms against the plain FP64 GPU form of the same batch
        learned["speedup_vs_plain_f64"] = {
            "bicgstab_net_guess": plain_ms / learned["ms_per_step_with_net"],
            "fgmres10_net_preconditioned": plain_ms / learned["fgmres10_net_preconditioned"]["ms_per_step"]}

    # end to end through the C ABI with pinned host buffers: the solve of each
    # pipelined chunk as one graph launch (no host poll between the chunks)
    e2e_prm = dd4d.params(TOL, inner_prec="f32", inner_tol=args.inner_tol, check_every=8, autotune=True,
                          graph_solve=True)
    bh = torch.from_numpy(b_h.view(np.float64)).pin_memory()
    xh = torch.empty_like(bh).pin_memory()
    for _ in range(2):
        ctx.solve_blocks("omega", ids, NRHS, bh, xh, e2e_prm)
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        st = ctx.solve_blocks("omega", ids, NRHS, bh, xh, e2e_prm)
        if st["status"] != 0 or st["max_relres"] > TOL:
            raise RuntimeError("e2e solve failed: %s" % st)
    barrier()
    e2e_s = (time.perf_counter() - t0) / args.steps
    e2e = {"value": world * units / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": int(bh.numel() * 8), "d2h_bytes_per_step": int(xh.numel() * 8),
           "form": "dd_solve_blocks on page-locked host b and x, pipelined chunks, each chunk's mixed "
                   "solve one graph launch (DD_SOLVE_GRAPH_SOLVE)", "ms_per_step": e2e_s * 1e3}
    del bh, xh

    # multi-boson action on the 8^4 lattice (16 blocks of 5^4, N = 4, 2 fields)
    action = uneven = heatbath = reweight = config5 = None
    if rank == 0:
        action = action_rate(dd4d, synth, torch)
        heatbath = heatbath_rate(dd4d, synth, torch)
        reweight = reweight_rate(dd4d, synth, torch)
        if not args.no_uneven:
            uneven = uneven_action_rate(dd4d, synth, torch)
    stencil = None
    if rank == 0 and not args.no_stencil:
        stencil = stencil_rates(dd4d, synth, torch, ctx, ids, b, n_om)
    force = None
    if rank == 0:
        try:
            force = force_rate(dd4d, torch, ctx, info, mixed)
        except (dd4d.DDError, RuntimeError) as err:          # e.g. device memory
            force = {"unavailable": str(err)[:200]}
    md = None
    if rank == 0:
        try:
            md = md_rate(dd4d, torch, ctx, info, mixed, U)
        except (dd4d.DDError, RuntimeError) as err:
            ctx.gauge_upload(U)
            md = {"unavailable": str(err)[:200]}
    # the same batch with the clover term (left-preconditioned by A^{-1}): the
    # mixed form (FP32 inner with the FP32 A^{-1} epilogue, double-float
    # residual with the double-float one) and the plain FP64 form
    clover = None
    if rank == 0:
        try:
            t0 = time.perf_counter()
            ctx.set_clover(CSW)
            build_s = time.perf_counter() - t0

            def clover_time(prm):
                step(prm)
                c0 = torch.cuda.Event(enable_timing=True)
                c1 = torch.cuda.Event(enable_timing=True)
                c0.record(stream)
                cst = step(prm)
                c1.record(stream)
                torch.cuda.synchronize()
                return c0.elapsed_time(c1), cst
            c_A = ctx.clover_cond()
            mms, mst = clover_time(mixed)
            cms, cst = clover_time(plain)
            ctx.set_clover(0.0)
            clover = {"metric": "block-solve sites/s to 1e-10 with the clover term", "value": units / (mms * 1e-3),
                      "unit": UNIT, "ms_per_step": mms, "c_sw": CSW, "max_iters": mst["max_iters"],
                      "outer_cycles": mst["outer_cycles"], "max_relres": mst["max_relres"],
                      "plain_f64": {"value": units / (cms * 1e-3), "ms_per_step": cms,
                                    "max_iters": cst["max_iters"], "max_relres": cst["max_relres"]},
                      "mixed_speedup_vs_plain_f64": cms / mms,
                      "cond_bound_c_A": c_A,
                      "tol_preconditioned": TOL / c_A,
                      "mixed_ms_without_clover": ms,
                      "table_build_s": build_s,
                      "workload": "the bench batch (256 framed blocks of 9^4 x 12 rhs, 32^4) with "
                                  "A(x) = 1 + i kappa c_sw sum sigma F; FP32 inner + double-float "
                                  "correction, A^{-1} in every hop"}
        except (dd4d.DDError, RuntimeError) as err:
            ctx.set_clover(0.0)
            clover = {"unavailable": str(err)[:200]}

    peak, peak_kind = measured_peaks()
    achieved = hop32_bytes / (hop32_ms * 1e-3) / 1e9 if hop32_ms > 0 else None
    # stored ncu traffic counts only for the launch variant they were taken on
    tr = traffic_record()
    hv = stats["hop_variant"]
    if tr and tr.get("variant_name") != dd4d.hop_variant_name("f32", hv):
        tr = None
    alg_per_launch = hop32_bytes / hop32_n if hop32_n else None
    # ncu DRAM bytes of fully active launches, scaled to the timed region's
    # average launch by its algorithmic bytes (systems that converged skip)
    traffic = tr["dram_over_algorithmic"] * alg_per_launch if (tr and alg_per_launch) else None
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak if achieved else None,
                "traffic": traffic,
                "traffic_dram_over_algorithmic": tr["dram_over_algorithmic"] if tr else None,
                "kernel": "FP32 even-odd hop inside the inner BiCGstab, autotuned variant %d: %s"
                          % (hv, dd4d.hop_variant_name("f32", hv)),
                "peak_kind": peak_kind, "launches": hop32_n,
                "avg_launch_ms": hop32_ms / hop32_n if hop32_n else None,
                "algorithmic_bytes_per_launch": alg_per_launch}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+df64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "lattice": list(LATTICE), "blocks": len(ids),
                   "omega_sites": n_om, "rhs_per_block": NRHS, "systems": len(ids) * NRHS,
                   "site_rhs_per_step": units, "inner": "f32",
                   "residual": "double-float (f32 pairs)", "inner_tol": args.inner_tol,
                   "tol": TOL, "l2": "inputs larger than L2 (3.9 GB rhs, ~15 GB working set)"},
        "roofline": roofline,
        "clocks": clocks,
        "e2e": e2e,
        "gpu_launches": launches,
        "solver": {"max_relres": stats["max_relres"], "max_iters": stats["max_iters"],
                   "outer_cycles": stats["outer_cycles"], "hop_variant": stats["hop_variant"]},
        "bf16_inner": bf16,
        "device_loop_graph": device_loop,
        "whole_solve_graph": whole_graph,
        "plain_f64": {"value": world * units / (plain_ms * 1e-3), "ms_per_step": plain_ms,
                      "max_iters": pst["max_iters"], "speedup_of_mixed": plain_ms / ms,
                      "residual_hop_ms_in_mixed_step": hop64_ms / args.steps},
        "action": action,
        "action_uneven": uneven,
        "action_48x4": config5,
        "heatbath": heatbath,
        "reweight": reweight,
        "force": force,
        "clover": clover,
        "md": md,
        "learned_guess": learned,
        "stencil": stencil,
    }
    ctx.close()
    # the config-3 action with its blocks split over every rank (all ranks take part)
    sharded = None
    if not args.no_uneven:
        torch.cuda.empty_cache()
        try:
            sharded = sharded_action_rate(dd4d, synth, torch, world, rank, local)
        except (dd4d.DDError, RuntimeError) as err:
            sharded = {"unavailable": str(err)[:200]}
        line["action_uneven_sharded"] = sharded
    # the 48^4 action holds ~100 GB of batched work vectors: measured after the
    # bench context has released its memory
    if rank == 0 and not args.no_config5:
        del b, x
        torch.cuda.empty_cache()
        try:
            config5 = config5_action_rate(dd4d, synth, torch)
        except (dd4d.DDError, RuntimeError) as err:          # e.g. device memory
            config5 = {"unavailable": str(err)[:200]}
        line["action_48x4"] = config5
    if rank == 0:
        line["cpu_baseline"] = cpu_baseline_entry(U) if world == 1 else None
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


def learned_ab(dd4d, synth, torch, ctx, ids, b, x, units, ms_plain_guess):
    """Trains the parallel-transport network on three other 16^4 lattices
    (eps 0.4, 0.5, 0.6; 16 framed blocks x 4 rhs each; targets from the FP64
    solver) and times the bench batch (held-out lattice) with the network as
    initial guess, against the same solve without it."""
    net = dd4d.Net(ctx, synth.net_init_weights(11))
    train = []
    for k, eps in enumerate((0.4, 0.5, 0.6)):
        L = (16, 16, 16, 16)
        c = dd4d.Context(L, KAPPA)
        c.gauge_upload(synth.gauge_field(L, eps, 100 + k))
        info = c.set_geometry(cores_uniform(L, CORE, FRAME))
        bt = synth.complex_gaussian(100 + k, synth.TAG_RHS, (info["nblocks"], 4, info["max_omega"], 12))
        st = net.train(list(range(info["nblocks"])), 4,
                       torch.from_numpy(bt.view(np.float64)).cuda(), steps=80, lr=3e-3, ctx=c)
        train.append({"eps": eps, "loss_first": st["loss_first"], "loss_last": st["loss_last"],
                      "seconds": st["seconds"], "pairs": st["pairs"]})
        c.close()
    net.attach(ctx)

    def timed(prm):
        ctx.solve_blocks("omega", ids, NRHS, b, x, prm)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        st = ctx.solve_blocks("omega", ids, NRHS, b, x, prm)
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), st
    ms, st = timed(dd4d.params(TOL, inner_prec="f32", inner_tol=3e-6, net_guess=True, autotune=True))
    # FGMRES(10) inner solves, without and with the network as right preconditioner
    fg0_ms, fg0 = timed(dd4d.params(TOL, inner_prec="f32", inner_tol=3e-6, autotune=True, fgmres=True, restart=10))
    fg1_ms, fg1 = timed(dd4d.params(TOL, inner_prec="f32", inner_tol=3e-6, autotune=True, fgmres=True, restart=10,
                                    net_precond=True))
    # one application of the network to the whole batch (tensor cores), and on the CUDA cores
    y = torch.empty_like(b)
    app = {}
    for tcm in (True, False):
        net.tensor_cores(tcm)
        net.apply(ids, NRHS, b, y)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        net.apply(ids, NRHS, b, y)
        e1.record()
        torch.cuda.synchronize()
        app["tensor_cores" if tcm else "fp32_cuda_cores"] = e0.elapsed_time(e1)
    net.tensor_cores(True)
    del y
    net.detach(ctx)
    net.close()
    return {"workload": "network trained on 3 x 16^4 lattices (eps 0.4/0.5/0.6, 64 pairs each), "
                        "4 layers 4-16-16-16-4, BF16 weights, applied on the held-out bench lattice (seed 2)",
            "training": train, "ms_per_step_with_net": ms, "ms_per_step_without": ms_plain_guess,
            "value_with_net": units / (ms * 1e-3), "max_iters_with_net": st["max_iters"],
            "max_relres_with_net": st["max_relres"], "status": st["status"],
            "fgmres10_plain": {"ms_per_step": fg0_ms, "max_iters": fg0["max_iters"],
                               "max_relres": fg0["max_relres"], "status": fg0["status"]},
            "fgmres10_net_preconditioned": {"ms_per_step": fg1_ms, "max_iters": fg1["max_iters"],
                                            "max_relres": fg1["max_relres"], "status": fg1["status"]},
            "net_application_ms": app}


def stencil_rates(dd4d, synth, torch, ctx, ids, b12, n_om):
    """D_X on the config-2 framed blocks (dd_apply_D_block) per storage precision
    and rhs count: the best launch form's algorithmic bandwidth (bytes of the
    formula in the library's accounting / event-timed hop launches) and its
    fraction of the measured HBM peak."""
    peak, _ = measured_peaks()
    out = {"workload": "32^4, 256 framed blocks of 9^4, even-odd hop launches of D_X (2 per apply)"}
    b1 = torch.from_numpy(synth.complex_gaussian(4, synth.TAG_RHS, (len(ids), 1, n_om, 12))
                          .view(np.float64).copy()).to(b12.device)
    for prec, which in (("f64", 0), ("f32", 1), ("bf16", 2)):
        for nrhs, inp in ((1, b1), (12, b12)):
            o = torch.empty_like(inp)
            best = None
            for v in range(dd4d.lib().dd_hop_variants(dd4d.PREC[prec])):
                ctx.set_hop_variant(prec, v)
                ctx.apply_D_block("omega", ids, nrhs, inp, o, prec)
                torch.cuda.synchronize()
                ctx.timing_enable(True)
                ctx.timing_get(which)
                for _ in range(3):
                    ctx.apply_D_block("omega", ids, nrhs, inp, o, prec)
                ms, n, by = ctx.timing_get(which)
                ctx.timing_enable(False)
                gbs = by / (ms * 1e-3) / 1e9
                if best is None or gbs > best[0]:
                    best = (gbs, ms / n, v)
            ctx.set_hop_variant(prec, -1)
            del o
            entry = {"GB_s": best[0], "frac_of_hbm": best[0] / peak if peak else None,
                     "ms_per_launch": best[1], "variant": dd4d.hop_variant_name(prec, best[2])}
            if prec == "f64":
                # the FP64 form is bound by the FP64 pipes: 1320 flops per output (site, rhs)
                # for the hop and 48 for the self term, against the measured FP64 FMA rate
                units = len(ids) * n_om * nrhs / 2.0
                tf = units * 1368.0 / (best[1] * 1e-3) / 1e12
                fma = dd4d.fp64_fma_rate()
                entry.update({"fp64_tflops": tf, "fp64_fma_peak_tflops": fma, "frac_of_fp64_fma": tf / fma,
                              "bound": "alu (FP64)"})
            out["%s_%drhs" % (prec, nrhs)] = entry
    return out


def action_rate(dd4d, synth, torch, evals=5):
    """Multi-boson action on the 8^4 lattice (16 blocks of 5^4, N = 4)."""
    L = (8, 8, 8, 8)
    U = synth.gauge_field(L, 0.3, 1)
    c = dd4d.Context(L, 0.13)
    c.gauge_upload(U)
    c.set_geometry(cores_uniform(L, 3, 1))
    dpi = c.geom_sites(dd4d.SET_DPI)
    u = dd4d.roots(4, 0.5)
    chi = synth.complex_gaussian(1, synth.TAG_CHI, (2, len(dpi), 12))
    d = torch.from_numpy(chi.view(np.float64)).cuda()
    prm = dd4d.params(TOL, inner_prec="f64", graph=True, autotune=True)
    for _ in range(2):
        c.multiboson_action(u, d, prm)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(evals):
        S, Sb, Sr, st = c.multiboson_action(u, d, prm)
    dt = (time.perf_counter() - t0) / evals
    stats = c.last_solve_stats()
    c.close()
    return {"metric": "action evals/s", "value": 1.0 / dt, "unit": "evals/s",
            "workload": "8^4, kappa 0.13, eps 0.3, 16 blocks of 5^4 + frame in one batch, "
                        "N = 4 (2 fields), FP64 solves to 1e-10, CUDA graphs, autotuned",
            "S": S, "max_relres": stats["max_relres"]}


def heatbath_rate(dd4d, synth, torch, reps=3):
    """Multi-boson fields by heat-bath on the 8^4 lattice: chi_k = W_{u_k}^{-1} eta_k for
    the N/2 = 4 fields of N = 8 (c = 0.5), checked by S_MB(chi) = sum |eta|^2."""
    L = (8, 8, 8, 8)
    c = dd4d.Context(L, 0.13)
    c.gauge_random(0.3, 1)
    c.set_geometry(cores_uniform(L, 3, 1))
    dpi = c.geom_sites(dd4d.SET_DPI)
    u = dd4d.roots(8, 0.5)
    eta = synth.complex_gaussian(1, synth.TAG_CHI, (len(u), len(dpi), 12))
    de = torch.from_numpy(eta.view(np.float64)).cuda()
    dx = torch.zeros_like(de)
    prm = dd4d.params(1e-11, inner_prec="f64", graph=True, autotune=True)
    c.multiboson_heatbath(u, de, dx, tol=1e-10, prm=prm)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(reps):
        st = c.multiboson_heatbath(u, de, dx, tol=1e-10, prm=prm)
    dt = (time.perf_counter() - t0) / reps
    S = c.multiboson_action(u, dx, prm)[0]
    ref = float(np.vdot(eta, eta).real)
    c.close()
    return {"metric": "heat-bath field sets/s", "value": 1.0 / dt, "unit": "sets/s",
            "workload": "8^4, kappa 0.13, eps 0.3 (links drawn on the device), 16 blocks of 5^4 + frame, "
                        "N = 8 (4 fields), BiCGstab on dPi to 1e-10 over apply_w with FP64 solves to 1e-11",
            "iterations": st["iterations"], "matvecs": st["matvecs"], "max_relres": st["max_relres"],
            "action_identity_relerr": abs(S - ref) / ref}


def reweight_rate(dd4d, synth, torch, n_src=16, N=12, cpar=0.5, reps=2):
    """Stochastic samples of the reweighting factor W_N = det{1 - R_{N+1}(W_1)} (Eq. rw)
    on the 8^4 lattice: s = |eta|^2 - |M eta|^2 for 16 complex Gaussian sources, each
    R_{N+1}(W_1) eta built from N + 1 = 13 apply_w batches; mean(exp(s)) estimates |W_N|^-2."""
    L = (8, 8, 8, 8)
    c = dd4d.Context(L, 0.13)
    c.gauge_random(0.3, 1)
    c.set_geometry(cores_uniform(L, 3, 1))
    dpi = c.geom_sites(dd4d.SET_DPI)
    eta = synth.complex_gaussian(2, synth.TAG_CHI, (n_src, len(dpi), 12))
    de = torch.from_numpy(eta.view(np.float64)).cuda()
    prm = dd4d.params(1e-11, inner_prec="f64", graph=True, autotune=True)
    c.reweight_samples(N, cpar, de, None, prm)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(reps):
        smp, st = c.reweight_samples(N, cpar, de, None, prm)
    dt = (time.perf_counter() - t0) / reps
    c.close()
    ex = np.exp(smp)
    mean, err = float(ex.mean()), float(ex.std(ddof=1) / np.sqrt(n_src))
    return {"metric": "reweighting samples/s", "value": n_src / dt, "unit": "samples/s",
            "workload": "8^4, kappa 0.13, eps 0.3 (links drawn on the device), 16 blocks of 5^4 + frame, "
                        "N = 12, c = 0.5, 16 sources, 13 apply_w batches with FP64 solves to 1e-11",
            "status": st, "mean_exp_s": mean, "stderr": err,
            "ln_abs_W_N": -0.5 * float(np.log(mean))}


def force_rate(dd4d, torch, ctx, info, prm, n_f=12, reps=2):
    """Force of the multi-boson action on the active links of the 32^4 lattice (256
    blocks, cores 7^4): 12 fields (N = 24, c = 0.5), two batched block solves of
    3072 systems each (mixed precision to 1e-10) and one FP64 thread per link."""
    n_dpi = info["n_dpi"]
    L = LATTICE
    gen = torch.Generator(device="cuda")
    gen.manual_seed(11)
    chi = torch.randn((n_f, n_dpi, 24), generator=gen, device="cuda", dtype=torch.float64) * (0.5 ** 0.5)
    F = torch.zeros(tuple(L) + (4, 8), dtype=torch.float64, device="cuda")
    u = dd4d.roots(2 * n_f, 0.5)
    ctx.mb_force(u, chi, F=F, prm=prm)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(reps):
        _, st = ctx.mb_force(u, chi, F=F, prm=prm)
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / reps
    # the force kernel alone (CUDA events on its stream), one more call
    ctx.timing_get(3)
    ctx.timing_enable(True)
    ctx.mb_force(u, chi, F=F, prm=prm)
    ctx.timing_enable(False)
    kms, kn, kflops = ctx.timing_get(3)
    for w in range(3):
        ctx.timing_get(w)
    links = int((F != 0).any(dim=-1).sum().item())
    fmax = float(F.abs().max().item())
    # the other block-local term: noise estimate of d ln|det D_Omega| / d eps, 4 noise
    # vectors per block (one batched solve of 1024 systems and the same link kernel)
    n_noise = 4
    eta = torch.randn((info["nblocks"], n_noise, info["max_omega"], 24), generator=gen, device="cuda",
                      dtype=torch.float64) * (0.5 ** 0.5)
    ctx.logdet_force(n_noise, eta, G=F, prm=prm)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    _, gst = ctx.logdet_force(n_noise, eta, G=F, prm=prm)
    torch.cuda.synchronize()
    ld_s = time.perf_counter() - t1
    del chi, F, eta
    fp64 = dd4d.fp64_fma_rate()
    kg = kflops / max(kn, 1) / (kms / max(kn, 1) * 1e-3) / 1e9 if kms > 0 else None
    return {"metric": "force evaluations/s", "value": 1.0 / dt, "unit": "evals/s",
            "logdet_force": {"seconds_per_eval": ld_s, "noise_per_block": n_noise, "status": gst},
            "force_kernel_roofline": {"bound": "alu", "achieved": kg, "unit": "GFLOP/s FP64",
                                      "peak": fp64 * 1e3, "peak_kind": "measured FP64 FMA rate (dd_fp64_fma_rate)",
                                      "frac": kg / (fp64 * 1e3) if kg and fp64 > 0 else None},
            "workload": "32^4 bench lattice, 256 blocks (cores 7^4, frame 1), 12 fields (N = 24, c = 0.5), "
                        "two batched block solves of 3072 systems (FP32 inner + double-float correction "
                        "to 1e-10), FP64 force kernel",
            "seconds_per_eval": dt, "active_links": links, "links_per_s": links / dt,
            "force_kernel_ms": kms / max(kn, 1),
            "force_kernel_fp64_gflops": kg,
            "max_abs_force": fmax, "status": st}


def md_rate(dd4d, torch, ctx, info, prm, U, n_f=12, tau=0.1, nsteps=2):
    """One block-local molecular-dynamics trajectory of the active links of the 32^4
    lattice (256 blocks): 12 multi-boson fields and one pseudofermion per block,
    leapfrog with nsteps steps (nsteps + 1 force evaluations: the multi-boson force
    and the pseudofermion force, four batched block solves), mixed-precision solves
    to 1e-10.  The context's links are restored afterwards."""
    gen = torch.Generator(device="cuda")
    gen.manual_seed(13)
    chi = torch.randn((n_f, info["n_dpi"], 24), generator=gen, device="cuda", dtype=torch.float64) * (0.5 ** 0.5)
    eta = torch.randn((info["nblocks"], 1, info["max_omega"], 24), generator=gen, device="cuda",
                      dtype=torch.float64) * (0.5 ** 0.5)
    phi = torch.zeros_like(eta)
    ctx.pf_heatbath(eta, phi)
    P = torch.randn(tuple(LATTICE) + (4, 8), generator=gen, device="cuda", dtype=torch.float64)
    u = dd4d.roots(2 * n_f, 0.5)
    st = ctx.md_trajectory(u, chi, phi, P, tau, nsteps, prm)
    ctx.gauge_upload(U)
    del chi, eta, phi, P
    return {"metric": "MD trajectories/s", "value": 1.0 / st["seconds"], "unit": "trajectories/s",
            "seconds_per_trajectory": st["seconds"], "force_evals": st["force_evals"],
            "seconds_per_force_eval": st["seconds"] / st["force_evals"], "tau": tau, "steps": nsteps,
            "dH": st["H1"] - st["H0"], "H0": st["H0"], "status": st["status"],
            "workload": "32^4 bench lattice, 256 blocks (cores 7^4, frame 1): active links of every block, "
                        "12 multi-boson fields (N = 24, c = 0.5) + one pseudofermion per block, leapfrog, "
                        "FP32 inner + double-float correction to 1e-10"}


def config5_action_rate(dd4d, synth, torch, group=8):
    """Multi-boson action on 48^4 (1296 framed blocks of 9^4, N = 48: 24 fields), FP32
    inner solves with double-float defect correction to 1e-10.  The 24 fields go
    through the action in groups (S is a sum over fields), which keeps the block
    and frame solves of one group within one GPU's memory."""
    L = (48, 48, 48, 48)
    c = dd4d.Context(L, 0.1365)
    c.gauge_random(0.6, 5)
    info = c.set_geometry(cores_uniform(L, 7, 1))
    n_dpi = info["n_dpi"]
    u = dd4d.roots(48, 0.5)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(5)
    prm = dd4d.params(TOL, inner_prec="f32", inner_tol=3e-6, autotune=True)
    groups = [u[k:k + group] for k in range(0, len(u), group)]
    chis = [torch.randn((len(g), n_dpi, 24), generator=gen, device="cuda", dtype=torch.float64) * (0.5 ** 0.5)
            for g in groups]
    c.multiboson_action(groups[0], chis[0], prm)        # autotune the batch shape
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    S, relres = 0.0, 0.0
    for g, ch in zip(groups, chis):
        S += c.multiboson_action(g, ch, prm)[0]
        relres = max(relres, c.last_solve_stats()["max_relres"])
    dt = time.perf_counter() - t0
    site_rhs = len(u) * (info["nblocks"] * info["max_omega"] + info["n_lambda1"])
    # the first group of fields in three forms: FP32 inner (as above), plain FP64
    # inner solves (the reference form) and BF16-storage inner solves; each one's
    # time and the relative difference of its S^r and S^a to the FP64 form's
    forms = {}
    for name, fprm in (("f32_inner", prm),
                       ("plain_f64", dd4d.params(TOL, inner_prec="f64")),
                       ("bf16_inner", dd4d.params(TOL, inner_prec="bf16", inner_tol=1e-3, autotune=True))):
        c.multiboson_action(groups[0], chis[0], fprm)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        Sg, Sb, Sr, _ = c.multiboson_action(groups[0], chis[0], fprm)
        forms[name] = {"seconds": time.perf_counter() - t1, "S": Sg, "S_r": Sr, "S_blocks": np.asarray(Sb),
                       "max_relres": c.last_solve_stats()["max_relres"]}
    ref = forms["plain_f64"]
    out_forms = {}
    for name, f in forms.items():
        out_forms[name] = {"seconds_first_group": f["seconds"], "max_relres": f["max_relres"],
                           "rel_diff_S_vs_f64": abs(f["S"] - ref["S"]) / ref["S"],
                           "rel_diff_S_r_vs_f64": abs(f["S_r"] - ref["S_r"]) / ref["S_r"],
                           "max_rel_diff_S_block_vs_f64": float(np.max(np.abs(f["S_blocks"] - ref["S_blocks"])
                                                                       / ref["S_blocks"]))}
    c.close()
    return {"metric": "action evals/s", "value": 1.0 / dt, "unit": "evals/s",
            "workload": "48^4, kappa 0.1365, eps 0.6 (links drawn on the device, seed 5), 1296 framed blocks "
                        "of 9^4 + frame Lambda1, N = 48 (24 fields, c = 0.5, Gaussian chi on dPi from a seeded "
                        "device generator), FP32 inner + double-float defect correction to 1e-10, fields in "
                        "groups of %d" % group,
            "seconds_per_eval": dt, "block_and_frame_site_rhs_per_eval": site_rhs,
            "site_rhs_per_s": site_rhs / dt, "S": S, "max_relres": relres,
            "first_group_forms": out_forms,
            "mixed_speedup_vs_plain_f64": forms["plain_f64"]["seconds"] / forms["f32_inner"]["seconds"]}


def uneven_action_rate(dd4d, synth, torch, evals=2):
    """Multi-boson action on 64x32^3 with uneven blocks (cores 6 and 8 mixed,
    frame 1: 512 framed blocks of 8^4..10^4 sites in 16 shapes) plus the frame
    Lambda1, 12 fields (N = 24), FP32 inner solves + FP64 defect correction,
    every block and the frame in one batch, CUDA graphs, autotuned launches."""
    L = (64, 32, 32, 32)

    def cores(n, sizes):
        out, x = [], 0
        for k in range(n):
            c = sizes[k % 2]
            out.append((x, x + c - 1))
            x += c + 1
        return out
    cl = [cores(8, (6, 8))] + [cores(4, (6, 8))] * 3
    t0 = time.perf_counter()
    U = synth.gauge_field(L, 0.6, 3)
    c = dd4d.Context(L, 0.136)
    c.gauge_upload(U)
    info = c.set_geometry(cl)
    dpi = c.geom_sites(dd4d.SET_DPI)
    n_f = 12
    u = dd4d.roots(2 * n_f, 0.5)
    chi = synth.complex_gaussian(3, synth.TAG_CHI, (n_f, len(dpi), 12))
    d = torch.from_numpy(chi.view(np.float64)).cuda()
    setup = time.perf_counter() - t0
    prm = dd4d.params(TOL, inner_prec="f32", graph=True, autotune=True)
    c.multiboson_action(u, d, prm)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(evals):
        S, Sb, Sr, st = c.multiboson_action(u, d, prm)
    dt = (time.perf_counter() - t0) / evals
    stats = c.last_solve_stats()
    sizes = sorted({len(c.geom_sites(dd4d.SET_OMEGA, b)) for b in range(0, info["nblocks"], 7)})
    # the error of the mixed form against the plain FP64 form of the same action
    # (the FP64 form is the one the oracle pins, on smaller uneven lattices)
    t1 = time.perf_counter()
    S64, Sb64, Sr64, _ = c.multiboson_action(u, d, dd4d.params(TOL, inner_prec="f64"))
    f64_s = time.perf_counter() - t1
    c.close()
    err = {"rel_diff_S_vs_f64": abs(S - S64) / abs(S64), "rel_diff_S_r_vs_f64": abs(Sr - Sr64) / abs(Sr64),
           "max_rel_diff_S_block_vs_f64": max(abs(a - b) / abs(b) for a, b in zip(Sb, Sb64)),
           "plain_f64_seconds_per_eval": f64_s, "mixed_speedup_vs_plain_f64": f64_s / dt}
    return {"metric": "action evals/s", "value": 1.0 / dt, "unit": "evals/s", "error_vs_f64": err,
            "workload": "64x32^3, kappa 0.136, eps 0.6, seed 3: 512 uneven framed blocks "
                        "(cores 6/8 per direction, frame 1) + frame Lambda1 (%d sites), "
                        "12 fields (N = 24, c = 0.5), FP32 inner + FP64 defect correction "
                        "to 1e-10, one batch, CUDA graphs, autotuned" % info["n_lambda1"],
            "omega_sizes_seen": sizes, "n_dpi": info["n_dpi"], "S": S,
            "max_relres": stats["max_relres"], "max_iters": stats["max_iters"],
            "setup_s": setup, "s_per_eval": dt}


def sharded_action_rate(dd4d, synth, torch, world, rank, local, evals=2):
    """The config-3 multi-boson action (64x32^3, 512 uneven framed blocks + frame,
    12 fields) with the blocks split over the ranks (partition.py): each rank solves
    its blocks' frame pieces and framed blocks, rank 0 also the frame; two sums
    across the ranks per evaluation (NCCL under torchrun).  Strong scaling: the
    same lattice at every rank count; the slowest rank sets the time."""
    from paper_2211_06902_gb300 import partition, ranks
    L = (64, 32, 32, 32)

    def cores(n, sizes):
        out, x = [], 0
        for k in range(n):
            c = sizes[k % 2]
            out.append((x, x + c - 1))
            x += c + 1
        return out
    cl = [cores(8, (6, 8))] + [cores(4, (6, 8))] * 3
    c = dd4d.Context(L, 0.136)
    c.gauge_random(0.6, 3)
    info = c.set_geometry(cl)
    nb = info["nblocks"]
    dev = torch.device("cuda", local)
    dpi = c.geom_sites(dd4d.SET_DPI)
    n_f = 12
    u = torch.from_numpy(np.asarray(dd4d.roots(2 * n_f, 0.5))).to(dev)
    chi = torch.from_numpy(synth.complex_gaussian(3, synth.TAG_CHI, (n_f, len(dpi), 12))).to(dev)
    ops = partition.LibraryOps(c, dd4d.params(TOL, inner_prec="f32", graph=True, autotune=True))
    bod = partition.block_of_dpi(c, nb, device=dev)
    comm = partition.Comm(world)
    S, Sa, Sr = partition.multiboson_action(ops, comm, rank, world, u, chi, bod)
    ranks.barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(evals):
        S, Sa, Sr = partition.multiboson_action(ops, comm, rank, world, u, chi, bod)
    torch.cuda.synchronize()
    dt = ranks.max_over_ranks((time.perf_counter() - t0) / evals, world, dev)
    c.close()
    return {"metric": "action evals/s, blocks sharded over the ranks", "value": 1.0 / dt,
            "unit": "evals/s", "ranks": world, "scaling": "strong", "S": S, "S_r": Sr,
            "blocks_per_rank": [len(partition.owned_blocks(nb, r, world)) for r in range(world)],
            "workload": "64x32^3, kappa 0.136, eps 0.6 (links drawn on the device), 512 uneven framed "
                        "blocks + frame Lambda1, 12 fields (N = 24, c = 0.5), FP32 inner + FP64 defect "
                        "correction to 1e-10; frame-piece and block solves split by block index, the "
                        "frame solved on rank 0; sums across ranks per evaluation: Q chi on dPi1 and the "
                        "per-block parts of S"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--inner-tol", type=float, default=3e-6)
    ap.add_argument("--no-uneven", action="store_true",
                    help="omit the 64x32^3 uneven-block action measurement")
    ap.add_argument("--no-learned", action="store_true",
                    help="omit the learned-initial-guess A/B measurement")
    ap.add_argument("--no-config5", action="store_true",
                    help="omit the 48^4, 24-field action measurement")
    ap.add_argument("--no-stencil", action="store_true",
                    help="omit the per-precision stencil bandwidth measurement")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
