"""Benchmark of the Monte Carlo NEGF walk path on GB300.

One step = one pass of the whole hot path over the benchmark workload: transition tables for
every (wire, energy) task (lead self-energies, RGF sweeps, block columns -> Step 6' weights,
alias tables), the walks (walkers_per_task per task, start lead L) with their tally, and the
current with its standard error.  Workload (default): 2D wire W = 10 x L = 50, t = 1, onsite
U[-1, 1], eta = 0.05, 64 midpoint energies on [-3.5, 3.5], 1e6 walkers per energy, FP32 tables,
FP64 tally/current; inputs resident on the device.

  python bench.py [--gpus N --steps K --warmup W] [--impl gb300|reference] [--workload NAME]

Prints one JSON line on rank 0.  --impl reference times the CPU FP64 oracle (test
infrastructure) on a bounded sample of the same workload.
"""
import argparse
import json
import os
import subprocess
import sys
import time

for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")      # the CPU baseline is the oracle as it stands: 1 thread

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1805_10164_gb300 import dist as ndist, inputs  # noqa: E402

METRIC = "walker steps/s and s per lead current at 1% std error on 1 GB300; frac of roofline"
UNIT = "walker steps/s"
L2_BYTES = 129 * 1024 * 1024


def workload(name, energies=0):
    if name == "wire_10x50":
        wl = inputs.wire_10x50()
    elif name == "chain_l20":
        wl = inputs.chain_l20()
    elif name == "wire_16x100":
        wl = inputs.wire_16x100(precision="fp32")
    elif name == "wire_32x100":
        wl = inputs.wire_32x100()
    elif name == "wire_64x100":
        wl = inputs.wire_64x100()
    elif name == "wire_64x1000":
        wl = inputs.wire_64x1000()
    elif name == "batched_uneven":
        wl = inputs.batched_uneven()
    else:
        raise SystemExit(f"unknown workload {name}")
    if energies:
        # an evenly spread subset of each wire's energy grid (same weights)
        for w in wl.wires:
            idx = np.unique(np.linspace(0, len(w.energy) - 1, energies).round().astype(int))
            w.energy, w.energy_weight = w.energy[idx], w.energy_weight[idx]
        wl.name += f"_sub{energies}E"
    return wl


def tensor_peak(kind):
    """Dense tensor peak for TF32 from the measured BF16 burst peak and the nominal ratio
    (1.1 / 2.25 PFLOP/s)."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            bf16 = float(json.load(f)["bf16_tflops"])
        return bf16 * 1.1 / 2.25, "measured BF16 burst x nominal TF32/BF16 ratio (1.1/2.25)"
    except Exception:
        return 1900.0 * 1.1 / 2.25, "fallback BF16 1.9 PFLOP/s x nominal TF32/BF16 ratio"


# DRAM traffic per launch (dram__bytes_read.sum + dram__bytes_write.sum, one ncu capture of a
# timed launch, see profiles/) keyed by kernel, workload and a hash of the kernel's sources: a
# kernel changed since its counters were taken reports null.
MEASURED_TRAFFIC = {
    ("walk_kernel", "wire_W10_L50_eta0.05_64E", "6f10e941e2fe02bd"): 133336576,
}
TRAFFIC_SOURCES = {"walk_kernel": ["k_walk.cu", "philox.cuh"]}


def measured_traffic(kernel, workload):
    import hashlib
    files = TRAFFIC_SOURCES.get(kernel)
    if not files:
        return None
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_1805_10164_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return MEASURED_TRAFFIC.get((kernel, workload, h.hexdigest()[:16]))


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampler running during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.proc = None
        self.index = index
        self.t0 = time.perf_counter()
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def elapsed(self):
        return time.perf_counter() - self.t0

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)),
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(n_gpus):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if os.environ.get("NEGF_BENCH_GLOO") is None else "gloo")
    return rank, world, local


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ------------------------------------------------------------------ algorithmic bytes per kernel

def two_level(W, L, precision):
    """Layout the library picks by default (NEGF_LAYOUT_AUTO)."""
    return (precision == "split_tf32" and W == 64) or W * L > 2048


def level2_words(W):
    """u32 words of one level-2 inverse-CDF block (NEGF_LEVEL2_WORDS)."""
    return 8 if W <= 8 else 8 + 8 * ((W + 7) // 8)


def algorithmic_bytes(kernel, wl, precision, counts):
    """Bytes a kernel must move per launch by its definition (tables in, tables out)."""
    tasks = [(w.W, w.L) for w in wl.wires for _ in w.energy]
    rows = [W * L + 2 * W for W, L in tasks]
    one = [(r, W * L + 2) for r, (W, L) in zip(rows, tasks) if not two_level(W, L, precision)]
    two = [(r, W, L) for r, (W, L) in zip(rows, tasks) if two_level(W, L, precision)]
    wsz = 8 if precision == "fp64" else 4
    if kernel == "walk_kernel":
        walkers = int(counts[:, 0].sum())
        steps = int(counts[:, 4].sum())
        absorbed = int(counts[:, 1].sum() + counts[:, 2].sum())
        # one 8-byte entry per draw; two-level tables: a level-1 entry per transition and, per
        # transition that stays in the wire, the level-2 guide and one octet (32 B each; the
        # octet alone for W <= 8)
        if two and not one:
            Ws = {W for _, W, _ in two}
            if len(Ws) != 1:
                return None
            l2 = 32 if min(Ws) <= 8 else 64
            return 8 * (walkers + steps) + l2 * (steps - absorbed)
        if two:
            return None
        return 8 * (steps + walkers)
    if kernel == "alias_kernel":           # one-level rows, or the level-1 rows
        return sum(r * K for r, K in one) * (wsz + 8) + sum(r * (L + 2) for r, W, L in two) * (wsz + 8)
    if kernel == "two_level_kernel":       # read the weights, write level-2 blocks and level-1 weights
        return sum(r * (W * L) * wsz + r * L * (4 * level2_words(W) + wsz) for r, W, L in two)
    if kernel in ("diag_chain_kernels", "chain_cta_kernel", "chain_tc_kernel"):
        return sum(r * K for r, K in one) * wsz + sum(r * (W * L + 2) for r, W, L in two) * wsz
    return None


# ------------------------------------------------------------------ GPU arm

def run_gpu(args):
    import torch
    from paper_1805_10164_gb300 import build, negf

    rank, world, local = dist_setup(args.gpus)
    torch.cuda.set_device(local)
    build.build()
    wl = workload(args.workload, args.energies)
    prec = args.precision or wl.precision
    N = args.walkers or wl.walkers_per_task
    dev_wires = [inputs.Wire(W=w.W, L=w.L, t=w.t, onsite=torch.from_numpy(w.onsite).cuda(),
                             eta=torch.from_numpy(w.eta).cuda(),
                             energy=torch.from_numpy(w.energy).cuda(),
                             energy_weight=torch.from_numpy(w.energy_weight).cuda())
                 for w in wl.wires]
    stream = torch.cuda.current_stream()
    ctx = negf.negf_create(local, stream)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
    n_tasks = sum(len(w.energy) for w in wl.wires)
    plan = None
    plan_prec = prec
    tuning = None
    if args.mode == "graph":
        # the whole step captured once (device-resident inputs re-read by every launch);
        # launch shapes picked by the library's autotuner on this workload
        plan = negf.negf_plan_create(ctx, dev_wires, 0, N, wl.mu_p, wl.mu_q, wl.kT,
                                     precision=prec, memspace="device", max_steps=args.max_steps,
                                     tasks_per_wave=args.plan_tasks_per_wave, autotune=True)
        tuning = negf.negf_plan_get_tuning(plan)

    def one_step(step_idx, wires, memspace, prec=prec, end_event=None):
        """One step; `end_event` (if given) is recorded on the stream once the step's device work
        is enqueued, before the host reads the results (the host path is timed by e2e)."""
        wid0 = ndist.weak_walker_offset(rank, step_idx, N)
        if plan is not None and memspace == "device" and prec == plan_prec:
            negf.negf_plan_launch(ctx, plan, args.seed, wid0)
            if end_event is not None:
                end_event.record(stream)
            r = negf.negf_plan_result(ctx, plan)
            return r, r["counts"]
        if args.mode in ("pipeline", "graph"):
            # build wave w+1 while wave w walks; tables are freed wave by wave
            tables, tally = negf.negf_run(ctx, wires, 0, args.seed, N, precision=prec,
                                          memspace=memspace, walker_id_offset=wid0,
                                          max_steps=args.max_steps,
                                          # graph mode's host-buffer leg: waves only as
                                          # the memory budget requires
                                          tasks_per_wave=(args.tasks_per_wave
                                                          if args.mode == "pipeline" else 1 << 30),
                                          walk_blocks_per_sm=args.walk_blocks_per_sm)
        else:
            tables = negf.negf_build_tables(ctx, wires, precision=prec, memspace=memspace)
            tally = negf.negf_walk(ctx, tables, 0, args.seed, N, walker_id_offset=wid0,
                                   max_steps=args.max_steps)
        res = negf.negf_current(ctx, tables, tally, wl.mu_p, wl.mu_q, wl.kT)
        if end_event is not None:
            end_event.record(stream)
        counts = negf.negf_tally_counts(ctx, tally, n_tasks)
        negf.negf_tally_free(tally)
        negf.negf_tables_free(tables)
        return res, counts

    for i in range(args.warmup):
        one_step(10_000 + i, dev_wires, "device")
    torch.cuda.synchronize()
    # ---- timed region (device-resident inputs)
    barrier(world)
    torch.cuda.synchronize()
    clocks = Clocks(local) if rank == 0 else None
    negf.negf_profile_enable(ctx, True)
    total_ms, tot_steps, tot_walkers = 0.0, 0, 0
    last = None
    for i in range(args.steps):
        flush.fill_(float(i))                      # evict the previous step's tables from L2
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        res, counts = one_step(i, dev_wires, "device", end_event=e1)
        e1.synchronize()
        total_ms += e0.elapsed_time(e1)
        tot_steps += int(counts[:, 4].sum())
        tot_walkers += int(counts[:, 0].sum())
        last = (res, counts)
    torch.cuda.synchronize()
    prof = negf.negf_profile_read(ctx)
    negf.negf_profile_enable(ctx, False)
    if clocks is not None:
        # nvidia-smi samples every 200 ms: when the timed steps were shorter than a second,
        # keep running the same step (untimed) so that the clock record holds a few samples
        t_soak = time.perf_counter()
        i = 0
        while clocks.elapsed() < 1.2 and time.perf_counter() - t_soak < 5.0:
            flush.fill_(float(i))
            one_step(30_000 + i, dev_wires, "device")
            torch.cuda.synchronize()
            i += 1
    clk = clocks.stop() if clocks else None
    if clk is not None:
        clk["window"] = "timed steps, then repeats of the same step until 1.2 s had passed"
    barrier(world)
    t_max = max_over_ranks(total_ms, world)
    all_steps = sum_over_ranks(float(tot_steps), world)
    # ---- end-to-end through the public API with host buffers (copies inside the region)
    e2e_ms, e2e_steps = 0.0, 0
    h2d = sum(w.onsite.nbytes + w.eta.nbytes + w.energy.nbytes + w.energy_weight.nbytes
              for w in wl.wires)
    d2h = 8 * (2 * len(wl.wires) + 2 * n_tasks + 1) + 4 + 8 * n_tasks * negf.TALLY_FIELDS
    # graph mode: the step's inputs come from pinned host buffers into the device arrays the
    # captured plan reads, then the plan runs and its results are read back (the serving path);
    # the other modes pass the host arrays to the library, which copies them itself
    pinned = None
    if plan is not None:
        pinned = [[torch.from_numpy(a).pin_memory() for a in (w.onsite, w.eta, w.energy,
                                                                w.energy_weight)]
                  for w in wl.wires]
    for i in range(max(1, min(args.steps, 3))):
        flush.fill_(float(i))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        if pinned is not None:
            for dw, hp in zip(dev_wires, pinned):
                for dst, src in zip((dw.onsite, dw.eta, dw.energy, dw.energy_weight), hp):
                    dst.copy_(src, non_blocking=True)
            _, counts = one_step(20_000 + i, dev_wires, "device")
        else:
            _, counts = one_step(20_000 + i, wl.wires, "host")
        torch.cuda.synchronize()
        e2e_ms += 1e3 * (time.perf_counter() - t0)
        e2e_steps += int(counts[:, 4].sum())
    e2e_ms = max_over_ranks(e2e_ms, world)
    e2e_steps = sum_over_ranks(float(e2e_steps), world)
    # ceiling for the walk's 8-byte alias-entry gathers (measured, this GPU, this run)
    per_task_bytes = 8 * max((w.W * w.L + 2 * w.W) * (w.W * w.L + 2) for w in wl.wires)
    probe_tab = min(2 * per_task_bytes, 16 << 30)
    probe_gps = negf.negf_probe_gather(ctx, probe_tab, ilp=8, chain=64)
    probe_gps1 = negf.negf_probe_gather(ctx, probe_tab, ilp=1, chain=64)
    probe_gbs = 8 * probe_gps / 1e9
    probe_src = (f"measured: negf_probe_gather, random 8-byte gathers over {probe_tab >> 20} MiB "
                 f"(two tasks' alias tables, at most 16 GiB), 8 independent chains per thread "
                 f"({probe_gps:.3g}/s; 1 chain: {probe_gps1:.3g}/s)")
    # seconds per current at 1 % SE with FP64 tables (the plain FP64 form), for comparison
    fp64_cmp = None
    if args.compare_fp64 and prec != "fp64":
        fp64_cmp = time_precision("fp64", one_step, dev_wires, negf, ctx, stream, flush, args)
    if plan is not None:
        negf.negf_plan_destroy(plan)
    negf.negf_destroy(ctx)
    if rank != 0:
        return
    res, counts = last
    ms_per_step = t_max / args.steps
    value = all_steps / (t_max / 1e3)
    # roofline of the dominant kernel
    dom = max(prof.items(), key=lambda kv: kv[1][1])
    kname, (klaunch, kms) = dom
    peak, src = peaks()
    abytes = algorithmic_bytes(kname, wl, prec, counts)
    roof = roof_hbm = None
    if abytes is not None and klaunch > 0:
        launches_per_step = klaunch / args.steps
        per_launch_bytes = abytes / max(1, launches_per_step)
        per_launch_s = kms / 1e3 / klaunch
        ach = per_launch_bytes / per_launch_s / 1e9
        roof_hbm = {"kernel": kname, "bound": "hbm", "achieved": round(ach, 1), "peak": peak,
                    "unit": "GB/s", "frac": round(ach / peak, 4), "peak_source": src + " HBM copy",
                    "traffic": None, "algorithmic_bytes_per_launch": int(per_launch_bytes),
                    "avg_launch_ms": round(kms / klaunch, 5)}
        roof_hbm["traffic"] = measured_traffic(kname, wl.name)
        roof = dict(roof_hbm)
        if kname == "walk_kernel" and probe_gbs and (probe_tab < 2 * per_task_bytes):
            # the probe could not cover two tasks' tables: HBM-resident gathers, keep the HBM
            # copy peak
            pass
        elif kname == "walk_kernel" and probe_gbs:
            # the alias tables of the tasks in flight sit in L2: the ceiling is the measured
            # random 8-byte gather rate over a table of that size
            roof.update(bound="l2", peak=round(probe_gbs, 1), frac=round(ach / probe_gbs, 4),
                        peak_source=probe_src)
    if kname == "chain_tc_kernel" and klaunch > 0:
        # tensor-core roofline: TF32 operations of the 3xTF32 products (3 GEMMs of 128 x 128 x
        # 128 real per CTA step, a pair of block columns advanced by one slice)
        steps_ct = 0
        for w in wl.wires:
            if w.W == 64:
                steps_ct += len(w.energy) * ((w.L + 2) * (w.L - 1) + 1) // 2
        flops = 3 * 2 * 128 ** 3 * steps_ct / max(1, klaunch / args.steps / 2)
        tflops = flops / (kms / 1e3 / (klaunch / 2)) / 1e12
        tf32_peak = tensor_peak("tf32")
        roof = {"kernel": kname, "bound": "tensor", "achieved": round(tflops, 1),
                "peak": round(tf32_peak[0], 1), "unit": "TFLOP/s",
                "frac": round(tflops / tf32_peak[0], 4), "peak_source": tf32_peak[1],
                "traffic": None, "algorithmic_flops_per_launch": int(flops),
                "avg_launch_ms": round(kms / klaunch * 2, 5)}
    # seconds per current at 1 % relative standard error: fixed table cost + walks scaled by
    # the binomial variance (N_needed = N (rel_se / 0.01)^2)
    walk_ms = prof.get("walk_kernel", (0, 0.0))[1] / args.steps
    rel = float(res["se"][0] / abs(res["I"][0])) if res["I"][0] != 0 else float("nan")
    s_per_current = ((ms_per_step - walk_ms) + walk_ms * (rel / 0.01) ** 2) / 1e3
    launches = int(sum(v[0] for v in prof.values()))
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp64": "f64 tables, u32 walks, f64 tally",
                  "fp32": "f32 tables, u32 walks, f64 tally",
                  "split_tf32": "tf32x3 block products (f32 accumulate), f32 tables, u32 walks, "
                                "f64 tally"}[prec],
        "data": "synthetic (seeded square-lattice wire standing in for the paper's CdTe nanowires)",
        "config": {"workload": wl.name, "wires": len(wl.wires), "tasks": n_tasks,
                   "walkers_per_task": N, "precision": prec, "start_lead": "L",
                   "mu_p": wl.mu_p, "mu_q": wl.mu_q, "kT": wl.kT,
                   "l2": "flushed between timed steps (258 MiB write, outside the timed events)",
                   "mode": args.mode,
                   "tasks_per_wave": (args.plan_tasks_per_wave if args.mode == "graph"
                                      else args.tasks_per_wave),
                   "launch_shapes": tuning,
                   "parallelism": f"tasks replicated per rank, walker ids disjoint ({world} GPU)"},
        "walker_steps_per_step": all_steps / args.steps / world,
        "walkers_per_step": tot_walkers / args.steps,
        "current": float(res["I"][0]), "current_rel_se": rel,
        "s_per_current_1pct": s_per_current,
        "kernel_ms_per_step": {k: round(v[1] / args.steps, 4) for k, v in prof.items()},
        "roofline": roof,
        "roofline_hbm": roof_hbm,
        "e2e": {"value": e2e_steps / (e2e_ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h),
                "path": ("pinned host inputs copied into the plan's device inputs, captured plan "
                         "launched, results read back (wall clock)" if plan is not None else
                         "host arrays passed to the library, results read back (wall clock)")},
        "gpu_launches": launches,
        "clocks": clk,
    }
    if fp64_cmp is not None:
        fp64_cmp["s_per_current_1pct_" + prec] = s_per_current
        fp64_cmp["speedup_" + prec + "_over_fp64"] = fp64_cmp["s_per_current_1pct"] / s_per_current
        out["fp64_tables"] = fp64_cmp
    if world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(wl, args, budget_s=args.cpu_budget)
    print(json.dumps(out), flush=True)


def time_precision(prec, one_step, dev_wires, negf, ctx, stream, flush, args, steps=3):
    """ms per step, walk ms and s per current at 1 % SE of the same workload with tables of
    precision ``prec`` (device-resident inputs, L2 flushed between steps)."""
    import torch
    for i in range(2):
        one_step(40_000 + i, dev_wires, "device", prec)
    torch.cuda.synchronize()
    negf.negf_profile_enable(ctx, True)
    tot = 0.0
    res = None
    for i in range(steps):
        flush.fill_(float(i))
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        res, _ = one_step(41_000 + i, dev_wires, "device", prec, end_event=e1)
        e1.synchronize()
        tot += e0.elapsed_time(e1)
    prof = negf.negf_profile_read(ctx)
    negf.negf_profile_enable(ctx, False)
    ms = tot / steps
    walk_ms = prof.get("walk_kernel", (0, 0.0))[1] / steps
    rel = float(res["se"][0] / abs(res["I"][0])) if res["I"][0] != 0 else float("nan")
    return {"precision": prec, "ms_per_step": ms, "walk_ms": walk_ms, "current": float(res["I"][0]),
            "current_rel_se": rel,
            "s_per_current_1pct": ((ms - walk_ms) + walk_ms * (rel / 0.01) ** 2) / 1e3,
            "kernel_ms_per_step": {k: round(v[1] / steps, 4) for k, v in prof.items()}}


# ------------------------------------------------------------------ gradient (forward + backward)


def run_gradient(args):
    """One step = the differentiable current of the workload's first wire through the public
    torch API (autograd.NegfCurrent: tables keeping G, walks with score tallies, current) and
    its backward (negf_current_backward: the gradient w.r.t. every onsite energy and every
    dephasing rate).  The API is synchronous (the current and the gradient come back to the
    host), so the timed region is wall time on the device between the step's first launch and
    the gradient's arrival."""
    import torch
    from paper_1805_10164_gb300 import autograd, build, negf

    rank, world, local = dist_setup(args.gpus)
    torch.cuda.set_device(local)
    build.build()
    name = args.workload if args.workload != "wire_10x50" else "wire_16x100"
    wl = workload(name, args.energies)
    prec = args.precision or wl.precision
    w = wl.wires[0]
    N = args.walkers or wl.walkers_per_task
    stream = torch.cuda.current_stream()
    ctx = negf.negf_create(local, stream)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
    onsite_h = torch.from_numpy(w.onsite).pin_memory()
    eta_h = torch.from_numpy(w.eta).pin_memory()

    def spec_for(i):
        return autograd.CurrentSpec(W=w.W, L=w.L, t=w.t, energy=w.energy,
                                    energy_weight=w.energy_weight, mu_p=wl.mu_p, mu_q=wl.mu_q,
                                    kT=wl.kT, start_lead=0, walkers_per_task=N, seed=args.seed,
                                    walker_id_offset=ndist.weak_walker_offset(rank, i, N),
                                    max_steps=args.max_steps, precision=prec)

    def one_step(i, onsite, eta):
        onsite = onsite.detach().requires_grad_(True)
        eta = eta.detach().requires_grad_(True)
        I, se = autograd.NegfCurrent.apply(onsite, eta, ctx, spec_for(i))
        I.backward()
        return float(I), float(se), onsite.grad, eta.grad

    on_d = onsite_h.cuda()
    eta_d = eta_h.cuda()
    for i in range(args.warmup):
        one_step(10_000 + i, on_d, eta_d)
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    clocks = Clocks(local) if rank == 0 else None
    negf.negf_profile_enable(ctx, True)
    total_ms, res = 0.0, None
    for i in range(args.steps):
        flush.fill_(float(i))
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        res = one_step(i, on_d, eta_d)
        e1.record(stream)
        e1.synchronize()
        total_ms += e0.elapsed_time(e1)
    prof = negf.negf_profile_read(ctx)
    negf.negf_profile_enable(ctx, False)
    if clocks is not None:
        t_soak = time.perf_counter()
        i = 0
        while clocks.elapsed() < 1.2 and time.perf_counter() - t_soak < 10.0:
            flush.fill_(float(i))
            one_step(30_000 + i, on_d, eta_d)
            torch.cuda.synchronize()
            i += 1
    clk = clocks.stop() if clocks else None
    if clk is not None:
        clk["window"] = "timed steps, then repeats of the same step until 1.2 s had passed"
    # walker steps of one step: the same walks (same seed and walker ids) without score
    # tallies, outside the timed region
    dev = inputs.Wire(W=w.W, L=w.L, t=w.t, onsite=on_d, eta=eta_d,
                      energy=torch.from_numpy(w.energy).cuda(),
                      energy_weight=torch.from_numpy(w.energy_weight).cuda())
    tab = negf.negf_build_tables(ctx, [dev], precision=prec, memspace="device")
    steps_per_step = 0.0
    for i in range(args.steps):
        tl = negf.negf_walk(ctx, tab, 0, args.seed, N,
                            walker_id_offset=ndist.weak_walker_offset(rank, i, N),
                            max_steps=args.max_steps)
        steps_per_step += float(negf.negf_tally_counts(ctx, tl, len(w.energy))[:, 4].sum())
        negf.negf_tally_free(tl)
    negf.negf_tables_free(tab)
    steps_per_step /= args.steps
    barrier(world)
    t_max = max_over_ranks(total_ms, world)
    # end to end: onsite and eta from pinned host memory, the gradient back to the host
    e2e_ms = 0.0
    n_e2e = max(1, min(args.steps, 3))
    for i in range(n_e2e):
        flush.fill_(float(i))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, _, gV, gE = one_step(20_000 + i, onsite_h.cuda(non_blocking=True),
                                eta_h.cuda(non_blocking=True))
        gV.cpu()
        gE.cpu()
        torch.cuda.synchronize()
        e2e_ms += (time.perf_counter() - t0) * 1e3
    negf.negf_destroy(ctx)
    if rank != 0:
        return
    I, se, gV, gE = res
    n_par = 2 * w.W * w.L
    out = {
        "metric": METRIC, "value": steps_per_step * world / (t_max / args.steps / 1e3),
        "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None,
        "dtype": {"fp64": "f64 tables and adjoint, u32 walks, f64 tally",
                  "fp32": "f32 tables and adjoint, u32 walks, f64 tally"}.get(prec, prec),
        "data": "synthetic (seeded square-lattice wire standing in for the paper's CdTe nanowires)",
        "config": {"workload": wl.name + "_gradient", "walkers_per_task": N,
                   "tasks": len(w.energy), "precision": prec,
                   "parameters": n_par,
                   "step": "forward (tables keeping G, walks with score tallies, current) + "
                           "backward (gradient w.r.t. every onsite energy and dephasing rate) "
                           "through autograd.NegfCurrent",
                   "l2": "flushed between timed steps (258 MiB write, outside the timed events)",
                   "mode": "gradient"},
        "walker_steps_per_step": steps_per_step,
        "gradient": {"ms_per_gradient": t_max / args.steps, "parameters": n_par, "I": I,
                     "se": se, "dI_donsite_norm": float(gV.norm()),
                     "dI_deta_norm": float(gE.norm())},
        "kernel_ms_per_step": {k: round(v[1] / args.steps, 4) for k, v in prof.items()},
        "e2e": {"value": steps_per_step / (e2e_ms / n_e2e / 1e3), "unit": UNIT,
                "h2d_bytes_per_step": int(2 * w.onsite.nbytes),
                "d2h_bytes_per_step": int(2 * w.onsite.nbytes + 16)},
        "gpu_launches": int(sum(v[0] for v in prof.values())),
        "clocks": clk,
    }
    print(json.dumps(out), flush=True)


# ------------------------------------------------------------------ thermal-window sampler

THERMAL_GRID = 17          # grid energies spanning mu +- 8 kT


def thermal_wire(wl):
    """The workload's first wire on a grid of THERMAL_GRID energies spanning mu +- 8 kT around
    mu = 0 (the linear-response reading: E_F = 0) at the workload's kT."""
    w = wl.wires[0]
    grid = np.linspace(-8.0 * wl.kT, 8.0 * wl.kT, THERMAL_GRID)
    return inputs.Wire(W=w.W, L=w.L, t=w.t, onsite=w.onsite, eta=w.eta, energy=grid,
                       energy_weight=np.ones_like(grid)), 0.0, wl.kT


def run_thermal(args):
    """One step = tables on the grid + the thermal-window walks of the linear conductance
    (negf_walk_thermal) + their tally; walkers per step = the workload's walkers per task times
    its number of energies."""
    import torch
    from paper_1805_10164_gb300 import build, negf
    from oracle import alias, pipeline, thermal

    rank, world, local = dist_setup(args.gpus)
    torch.cuda.set_device(local)
    build.build()
    wl = workload(args.workload, args.energies)
    prec = args.precision or wl.precision
    w, mu, kT = thermal_wire(wl)
    N = (args.walkers or wl.walkers_per_task) * len(wl.wires[0].energy)
    dev = inputs.Wire(W=w.W, L=w.L, t=w.t, onsite=torch.from_numpy(w.onsite).cuda(),
                      eta=torch.from_numpy(w.eta).cuda(), energy=torch.from_numpy(w.energy).cuda(),
                      energy_weight=torch.from_numpy(w.energy_weight).cuda())
    stream = torch.cuda.current_stream()
    ctx = negf.negf_create(local, stream)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")

    def one_step(i, wire, memspace):
        wid0 = ndist.weak_walker_offset(rank, i, N)
        t = negf.negf_build_tables(ctx, [wire], precision=prec, memspace=memspace)
        try:
            return negf.negf_walk_thermal(ctx, t, 0, 0, args.seed, N, mu, kT,
                                          walker_id_offset=wid0, max_steps=args.max_steps)
        finally:
            negf.negf_tables_free(t)

    for i in range(args.warmup):
        one_step(10_000 + i, dev, "device")
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    clocks = Clocks(local) if rank == 0 else None
    negf.negf_profile_enable(ctx, True)
    total_ms, tot_steps, res = 0.0, 0.0, None
    for i in range(args.steps):
        flush.fill_(float(i))
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        res = one_step(i, dev, "device")
        e1.record(stream)
        e1.synchronize()
        total_ms += e0.elapsed_time(e1)
        tot_steps += res["mean_steps"] * res["walkers"]
    prof = negf.negf_profile_read(ctx)
    negf.negf_profile_enable(ctx, False)
    if clocks is not None:
        t_soak = time.perf_counter()
        i = 0
        while clocks.elapsed() < 1.2 and time.perf_counter() - t_soak < 5.0:
            flush.fill_(float(i))
            one_step(30_000 + i, dev, "device")
            torch.cuda.synchronize()
            i += 1
    clk = clocks.stop() if clocks else None
    if clk is not None:
        clk["window"] = "timed steps, then repeats of the same step until 1.2 s had passed"
    barrier(world)
    t_max = max_over_ranks(total_ms, world)
    all_steps = sum_over_ranks(tot_steps, world)
    # end to end with host buffers (inputs copied in, results copied out, inside the region)
    e2e_ms, e2e_steps = 0.0, 0.0
    for i in range(max(1, min(args.steps, 3))):
        flush.fill_(float(i))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = one_step(20_000 + i, w, "host")
        torch.cuda.synchronize()
        e2e_ms += (time.perf_counter() - t0) * 1e3
        e2e_steps += r["mean_steps"] * r["walkers"]
    h2d = w.onsite.nbytes + w.eta.nbytes + w.energy.nbytes + w.energy_weight.nbytes
    # roofline: one 8-byte alias entry per draw (injection + transitions); the grid's tables
    # sit in L2, so the ceiling is the measured random-gather rate over their size
    tab_bytes = THERMAL_GRID * (w.W * w.L + 2 * w.W) * (w.W * w.L + 2) * 8
    probe_tab = min(tab_bytes, 16 << 30)
    gps = negf.negf_probe_gather(ctx, probe_tab, ilp=8, chain=64)
    negf.negf_destroy(ctx)
    if rank != 0:
        return
    kname = "thermal_walk_kernel"
    klaunch, kms = prof.get(kname, (0, 0.0))
    walkers = res["walkers"]
    per_launch_bytes = 8.0 * (res["mean_steps"] * walkers + walkers)
    ach = per_launch_bytes / (kms / 1e3 / max(klaunch, 1)) / 1e9 if klaunch else 0.0
    peak = 8 * gps / 1e9
    out = {
        "metric": METRIC, "value": all_steps / (t_max / 1e3), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp64": "f64 tables, u32 walks, integer tally",
                  "fp32": "f32 tables, u32 walks, integer tally"}.get(prec, prec),
        "data": "synthetic (seeded square-lattice wire standing in for the paper's CdTe nanowires)",
        "config": {"workload": f"thermal_{wl.name.split('_64E')[0]}_{THERMAL_GRID}E_kT{kT}",
                   "sampler": "energies from Th = -df/dE on the grid span, chain interpolated "
                              "between grid energies",
                   "grid": [float(w.energy[0]), float(w.energy[-1]), THERMAL_GRID], "mu": mu,
                   "kT": kT, "walkers_per_step": walkers, "precision": prec,
                   "l2": "flushed between timed steps (258 MiB write, outside the timed events)",
                   "mode": "thermal"},
        "conductance": {"G": res["G"], "se": res["se"], "window": res["window"],
                        "unit": "e^2/h"},
        "kernel_ms_per_step": {k: round(v[1] / args.steps, 4) for k, v in prof.items()},
        "roofline": {"kernel": kname, "bound": "l2", "achieved": round(ach, 1),
                     "peak": round(peak, 1), "unit": "GB/s",
                     "frac": round(ach / peak, 4) if peak else None, "traffic": None,
                     "peak_source": f"measured: negf_probe_gather over {probe_tab >> 20} MiB "
                                    f"(the grid's alias tables), 8 chains per thread",
                     "algorithmic_bytes_per_launch": int(per_launch_bytes),
                     "avg_launch_ms": round(kms / max(klaunch, 1), 5)},
        "e2e": {"value": e2e_steps / (e2e_ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": 8 * 10},
        "gpu_launches": int(sum(v[0] for v in prof.values())),
        "clocks": clk,
    }
    if world == 1 and not args.no_cpu_baseline:
        # the oracle's tables and replay walker on the same grid, a bounded sample of walkers
        t0 = time.perf_counter()
        tabs = [pipeline.task_reference(w.onsite, w.eta, w.t, E, with_alias=False,
                                        with_direct=False)["tab"] for E in w.energy]
        ent = [alias.build_tables(tb["w"]) for tb in tabs]
        ment = [np.stack([alias.build_tables(tb["mode_w"][p][None, :])[0] for p in (0, 1)])
                for tb in tabs]
        c = [tb["c"] for tb in tabs]
        n_w, steps = 0, 0
        while time.perf_counter() - t0 < min(args.cpu_budget, 20.0) or n_w == 0:
            lead, st, _, _ = thermal.walk(ent, ment, c, tabs[0]["n"], w.W, 0, 0, args.seed,
                                          np.arange(n_w, n_w + 2000, dtype=np.uint64), w.energy,
                                          mu, kT, 1 << 20)
            n_w += 2000
            steps += int(st.sum())
        dt = time.perf_counter() - t0
        out["cpu_baseline"] = {"value": steps / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
                               "sample": f"{THERMAL_GRID} grid tables + {n_w} walkers "
                                         f"({dt:.1f} s, numpy/LAPACK single thread)"}
    print(json.dumps(out), flush=True)


# ------------------------------------------------------------------ CPU oracle (baseline)

def cpu_sample(wl, n_energy, walkers, seed, t_budget=None):
    """Oracle on a sample of the workload: tables for n_energy energies spread over the grid
    and `walkers` walks each.  Returns (walker steps, seconds, sample description)."""
    from oracle import pipeline, walker
    w = wl.wires[0]
    idx = np.linspace(0, len(w.energy) - 1, n_energy).round().astype(int)
    steps = 0
    t0 = time.perf_counter()
    for k in idx:
        ref = pipeline.task_reference(w.onsite, w.eta, w.t, w.energy[k], w.lead_model,
                                      w.gamma_lead, with_direct=False)
        lead, st = walker.walk(ref["entries"], ref["mode_entries"], ref["n"], w.W, ref["c_open"],
                               int(k), 0, seed, np.arange(walkers, dtype=np.uint64), 1 << 20)
        steps += int(st.sum())
    dt = time.perf_counter() - t0
    return steps, dt, f"{n_energy} of {len(w.energy)} energies x {walkers} walkers"


def cpu_baseline(wl, args, budget_s=20.0):
    walkers = wl.walkers_per_task
    steps, dt, desc = cpu_sample(wl, min(16, len(wl.wires[0].energy)), walkers, args.seed)
    return {"value": steps / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": desc + f" ({dt:.1f} s, numpy/LAPACK single thread)"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    wl = workload(args.workload, args.energies)
    walkers = wl.walkers_per_task
    for i in range(args.warmup):
        cpu_sample(wl, 1, 1000, args.seed + i)
    tot_steps, tot_s = 0, 0.0
    desc = ""
    for i in range(args.steps):
        st, dt, desc = cpu_sample(wl, min(2, len(wl.wires[0].energy)), walkers,
                                  args.seed + 100 + i)
        tot_steps += st
        tot_s += dt
    value = tot_steps / tot_s
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1e3 * tot_s / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "impl": "reference",
           "config": {"workload": wl.name, "walkers_per_task": wl.walkers_per_task,
                      "sampled": desc},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                            "sample": desc + " per step"},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="wire_10x50")
    ap.add_argument("--precision", default=None)
    ap.add_argument("--walkers", type=int, default=None)
    ap.add_argument("--seed", type=int, default=20240607)
    ap.add_argument("--max-steps", type=int, default=1 << 20)
    ap.add_argument("--cpu-budget", type=float, default=20.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--mode", default="graph",
                    choices=["graph", "pipeline", "separate", "thermal", "gradient"])
    ap.add_argument("--tasks-per-wave", type=int, default=8)
    ap.add_argument("--walk-blocks-per-sm", type=int, default=4)
    ap.add_argument("--no-compare-fp64", dest="compare_fp64", action="store_false")
    ap.add_argument("--plan-tasks-per-wave", type=int, default=0,
                    help="graph mode: tasks per wave (0: all tasks in one wave, or 1024 for "
                         "the batched workload, whose 8192 tasks' tables need 548 GB)")
    ap.add_argument("--energies", type=int, default=0,
                    help="use an evenly spread subset of this many grid energies")
    args = ap.parse_args()
    if args.workload == "batched_uneven" and args.plan_tasks_per_wave == 0:
        args.plan_tasks_per_wave = 1024
    if args.impl == "reference":
        run_reference(args)
    elif args.mode == "thermal":
        run_thermal(args)
    elif args.mode == "gradient":
        run_gradient(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
