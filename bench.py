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


# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum, one ncu capture, see profiles/)
# per step of the named workload, keyed by kernel, workload and a hash of the kernel's sources:
# a kernel changed since its counters were taken reports null.  The headline's chain figure
# (which writes the level-2 blocks itself) is scaled from a capture of the W = 64 x L = 100
# wire (8 tasks) by the units processed (the blocks written and the g blocks read both grow as
# n^2 per task): x 100 per task, x 256 / 8 tasks.
MEASURED_TRAFFIC = {
    ("walk_kernel", "wire_W10_L50_eta0.05_64E", "83e0ebef3d6f1969"): 133926400,
    ("chain_cta_kernel", "wire_W64_L1000_eta0.005_256E", "a3bffe9ce92a6da4"): 5145210496000,
}
TRAFFIC_SOURCES = {"walk_kernel": ["k_walk.cu", "philox.cuh"],
                   "chain_cta_kernel": ["k_chain_cta.cu", "level2.cuh"]}


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

DEFAULT_WORKLOAD = "wire_64x1000"
SUB_RECORDS = ("wire_10x50", "batched_uneven")
FP64_ENERGIES = 2          # the FP64 comparison runs on this many energies of the first wire


def fp32_peak():
    """FP32 fused-multiply-add peak of the GPU from its unit counts and clock: 152 SMs x 128
    FP32 lanes x 2 flop per clock at the maximum SM clock (MEASURED_PEAKS.json sm_max_mhz,
    else the nominal 2070 MHz)."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            mhz = float(json.load(f)["sm_max_mhz"])
        src = "152 SMs x 128 FP32 lanes x 2 flop x measured max SM clock"
    except Exception:
        mhz, src = 2070.0, "152 SMs x 128 FP32 lanes x 2 flop x nominal 2070 MHz"
    return 152 * 128 * 2 * mhz * 1e6 / 1e12, f"{src} ({mhz:.0f} MHz)"


CKPT_STRIDE = 10          # the gradient's RGF blocks kept every this many slices


def adjoint_flops(w):
    """Flops of the block-column adjoint's block products for one task of wire w: per column
    m, the chain of G[:, m] (L - 1 products), the elimination and back substitution (2 L - 1),
    the lead-column products of the two boundary slices (2), and for the start lead's column
    also G Phi and the injection seeds' products (2 L); 8 W^3 flops per W x W complex
    product."""
    W, L = w.W, w.L
    prods = L * (3 * L - 2 + 2) + 2 * L
    return 8.0 * W ** 3 * prods


def cta_chain_flops(wl, precision):
    """FP32 flops of the CTA-wide block-column products per step: 8 W^3 per block-column step
    (one W x W complex block times a W x W block); W = 64 runs towards slice 0 only
    (G = G^T) plus the lead-L injection column: L(L-1)/2 + 2(L-1) steps per task; 16 < W <= 32
    runs both directions: (L + 2)(L - 1) steps."""
    if precision != "fp32":
        return 0
    total = 0
    for w in wl.wires:
        W, L = w.W, w.L
        if W == 64:
            st = L * (L - 1) // 2 + 2 * (L - 1)
        elif 16 < W <= 32:
            st = (L + 2) * (L - 1)
        else:
            continue
        total += len(w.energy) * 8 * W ** 3 * st
    return total


def tc_chain_flops(wl):
    """TF32 operations of the split-TF32 tensor-core chain per step (3 GEMMs of 128 x 128 x
    128 real per CTA step, a pair of block columns advanced by one slice)."""
    steps_ct = 0
    for w in wl.wires:
        if w.W == 64:
            steps_ct += len(w.energy) * ((w.L + 2) * (w.L - 1) + 1) // 2
    return 3 * 2 * 128 ** 3 * steps_ct


def rooflines(prof, wl, prec, counts, steps, probe_gbs=None, probe_src=None):
    """Roofline entry per kernel group of the step: achieved = algorithmic bytes (or flops) per
    step / the group's device time per step (prof: totals over ``steps`` steps; counts: the
    tallies of one step)."""
    hbm, hsrc = peaks()
    out = {}
    for kname, (launches, ms) in prof.items():
        if launches == 0 or ms <= 0:
            continue
        sec = ms / 1e3 / steps
        ent = None
        if kname == "chain_cta_kernel" and cta_chain_flops(wl, prec):
            fl = cta_chain_flops(wl, prec)
            pk, src = fp32_peak()
            ach = fl / sec / 1e12
            ent = {"bound": "alu", "achieved": round(ach, 2), "peak": round(pk, 2),
                   "unit": "TFLOP/s", "frac": round(ach / pk, 4), "peak_source": src,
                   "algorithmic_flops_per_step": int(fl)}
        elif kname == "chain_tc_kernel":
            fl = tc_chain_flops(wl)
            pk, src = tensor_peak("tf32")
            ach = fl / sec / 1e12
            ent = {"bound": "tensor", "achieved": round(ach, 1), "peak": round(pk, 1),
                   "unit": "TFLOP/s", "frac": round(ach / pk, 4), "peak_source": src,
                   "algorithmic_flops_per_step": int(fl)}
        elif kname in ("walk_kernel", "alias_kernel", "two_level_kernel"):
            b = algorithmic_bytes(kname, wl, prec, counts)
            if b is not None:
                ach = b / sec / 1e9
                ent = {"bound": "hbm", "achieved": round(ach, 1), "peak": hbm, "unit": "GB/s",
                       "frac": round(ach / hbm, 4), "peak_source": hsrc + " HBM copy",
                       "algorithmic_bytes_per_step": int(b)}
                if kname == "walk_kernel" and probe_gbs:
                    ent.update(bound="l2", peak=round(probe_gbs, 1),
                               frac=round(ach / probe_gbs, 4), peak_source=probe_src)
        if ent is not None:
            # traffic: the measured DRAM bytes per step over the launches of a step (the
            # average launch, as achieved is the average launch's rate)
            tps = measured_traffic(kname, wl.name)
            lps = launches / steps
            ent.update(kernel=kname, launches_per_step=lps, ms_per_step=round(ms / steps, 4),
                       traffic=int(tps / lps) if tps is not None else None,
                       traffic_per_step=tps)
            out[kname] = ent
    return out


def local_workload(wl, rank, world):
    """The energies of every wire that this rank owns (task partition, no data exchange)."""
    if world == 1:
        return wl
    import copy
    sub = copy.deepcopy(wl)
    for w in sub.wires:
        idx = ndist.task_partition(len(w.energy), rank, world)
        w.energy, w.energy_weight = w.energy[idx], w.energy_weight[idx]
    return sub


class Runner:
    """One workload through the library on this rank: a captured plan over device-resident
    inputs (the timed step), and negf_run over host arrays (the end-to-end path)."""

    def __init__(self, negf, ctx, stream, wl, prec, N, args, seed, tasks_per_wave=0):
        import torch
        self.negf, self.ctx, self.stream, self.wl, self.prec, self.N = negf, ctx, stream, wl, prec, N
        self.args, self.seed = args, seed
        self.dev = [inputs.Wire(W=w.W, L=w.L, t=w.t, onsite=torch.from_numpy(w.onsite).cuda(),
                                eta=torch.from_numpy(w.eta).cuda(),
                                energy=torch.from_numpy(w.energy).cuda(),
                                energy_weight=torch.from_numpy(w.energy_weight).cuda())
                    for w in wl.wires]
        self.n_tasks = sum(len(w.energy) for w in wl.wires)
        self.plan = negf.negf_plan_create(ctx, self.dev, 0, N, wl.mu_p, wl.mu_q, wl.kT,
                                          precision=prec, memspace="device",
                                          max_steps=args.max_steps,
                                          tasks_per_wave=tasks_per_wave, autotune=True)
        self.tuning = negf.negf_plan_get_tuning(self.plan)

    def step(self, wid0, end_event=None):
        self.negf.negf_plan_launch(self.ctx, self.plan, self.seed, wid0)
        if end_event is not None:
            end_event.record(self.stream)
        r = self.negf.negf_plan_result(self.ctx, self.plan)
        return r, r["counts"]

    def host_step(self, wid0):
        """End to end through the public API with host buffers: the library copies the inputs,
        builds, walks, and the current, SE and tallies come back to host memory."""
        negf = self.negf
        tables, tally = negf.negf_run(self.ctx, self.wl.wires, 0, self.seed, self.N,
                                      precision=self.prec, memspace="host",
                                      walker_id_offset=wid0, max_steps=self.args.max_steps)
        res = negf.negf_current(self.ctx, tables, tally, self.wl.mu_p, self.wl.mu_q, self.wl.kT)
        counts = negf.negf_tally_counts(self.ctx, tally, self.n_tasks)
        negf.negf_tally_free(tally)
        negf.negf_tables_free(tables)
        return res, counts

    def close(self):
        self.negf.negf_plan_destroy(self.plan)


def timed(runner, negf, ctx, stream, flush, steps, warmup, rank, world, step0=0, clocks=None):
    """W untimed steps, then K steps bracketed by a barrier and synchronize, each timed with
    CUDA events on the launching stream (L2 flushed between steps, outside the events)."""
    import torch
    N = runner.N
    for i in range(warmup):
        runner.step(ndist.weak_walker_offset(rank, 10_000 + step0 + i, N))
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    clk = Clocks(torch.cuda.current_device()) if (clocks and rank == 0) else None
    negf.negf_profile_enable(ctx, True)
    total_ms, tot_steps, tot_walkers, last = 0.0, 0, 0, None
    for i in range(steps):
        flush.fill_(float(i))
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        res, counts = runner.step(ndist.weak_walker_offset(rank, step0 + i, N), end_event=e1)
        e1.synchronize()
        total_ms += e0.elapsed_time(e1)
        tot_steps += int(counts[:, 4].sum())
        tot_walkers += int(counts[:, 0].sum())
        last = (res, counts)
    torch.cuda.synchronize()
    prof = negf.negf_profile_read(ctx)
    negf.negf_profile_enable(ctx, False)
    if clk is not None:
        # nvidia-smi samples every 200 ms: keep running the same step (untimed) until the clock
        # record holds a few samples
        t_soak = time.perf_counter()
        i = 0
        while clk.elapsed() < 1.2 and time.perf_counter() - t_soak < 5.0:
            flush.fill_(float(i))
            runner.step(ndist.weak_walker_offset(rank, 30_000 + step0 + i, N))
            torch.cuda.synchronize()
            i += 1
    clk_out = clk.stop() if clk else None
    if clk_out is not None:
        clk_out["window"] = "timed steps, then repeats of the same step until 1.2 s had passed"
    barrier(world)
    t_max = max_over_ranks(total_ms, world)
    all_steps = sum_over_ranks(float(tot_steps), world)
    return dict(t_max=t_max, all_steps=all_steps, tot_walkers=tot_walkers, prof=prof,
                last=last, clocks=clk_out)


def s_per_current(ms_per_step, walk_ms, rel):
    """Seconds per current at 1 % relative SE: the step's fixed table cost plus its walks scaled
    by the binomial variance (N_needed = N (rel / 0.01)^2)."""
    return ((ms_per_step - walk_ms) + walk_ms * (rel / 0.01) ** 2) / 1e3


def fp64_comparison(negf, ctx, stream, flush, wl, args):
    """Seconds per current at 1 % SE with FP64 tables (the plain FP64 form) and with the
    workload's tables, on the same labelled energy subset of the first wire (the FP64 chains of
    wide slices take seconds per energy, so the comparison is bounded)."""
    import copy
    import torch
    sub = copy.deepcopy(wl)
    sub.wires = sub.wires[:1]
    w = sub.wires[0]
    idx = np.unique(np.linspace(0, len(w.energy) - 1, FP64_ENERGIES).round().astype(int))
    w.energy, w.energy_weight = w.energy[idx], w.energy_weight[idx]
    out = {"energies": [int(i) for i in idx], "wire": f"W={w.W} L={w.L}"}
    dev = [inputs.Wire(W=w.W, L=w.L, t=w.t, onsite=torch.from_numpy(w.onsite).cuda(),
                       eta=torch.from_numpy(w.eta).cuda(), energy=torch.from_numpy(w.energy).cuda(),
                       energy_weight=torch.from_numpy(w.energy_weight).cuda())]
    N = args.walkers or sub.walkers_per_task
    for prec in (args.precision or wl.precision, "fp64"):
        def one(i, e1=None):
            t = negf.negf_build_tables(ctx, dev, precision=prec, memspace="device")
            tl = negf.negf_walk(ctx, t, 0, args.seed, N, walker_id_offset=i * N,
                                max_steps=args.max_steps)
            r = negf.negf_current(ctx, t, tl, sub.mu_p, sub.mu_q, sub.kT)
            if e1 is not None:
                e1.record(stream)
            negf.negf_tally_free(tl)
            negf.negf_tables_free(t)
            return r
        one(0)
        torch.cuda.synchronize()
        negf.negf_profile_enable(ctx, True)
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = one(1, e1)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        prof = negf.negf_profile_read(ctx)
        negf.negf_profile_enable(ctx, False)
        walk_ms = prof.get("walk_kernel", (0, 0.0))[1]
        rel = float(r["se"][0] / abs(r["I"][0])) if r["I"][0] != 0 else float("nan")
        out[prec] = {"ms_per_step": ms, "walk_ms": walk_ms, "current": float(r["I"][0]),
                     "current_rel_se": rel, "s_per_current_1pct": s_per_current(ms, walk_ms, rel),
                     "kernel_ms_per_step": {k: round(v[1], 4) for k, v in prof.items()}}
    p32 = args.precision or wl.precision
    out["speedup_" + p32 + "_over_fp64"] = (out["fp64"]["s_per_current_1pct"]
                                            / out[p32]["s_per_current_1pct"])
    return out


def sub_record(negf, ctx, stream, flush, name, args, rank, world):
    """One more workload measured the same way (graph mode, device-resident inputs)."""
    wl = workload(name)
    prec = wl.precision
    N = wl.walkers_per_task
    steps = min(args.steps, 20) if name == "wire_10x50" else min(args.steps, 3)
    r = Runner(negf, ctx, stream, wl, prec, N, args, args.seed,
               tasks_per_wave=1024 if name == "batched_uneven" else 0)
    try:
        t = timed(r, negf, ctx, stream, flush, steps, 3, rank, world, step0=50_000)
    finally:
        r.close()
    res, counts = t["last"]
    probe_gbs = probe_src = None
    if name == "wire_10x50":
        per_task = 8 * max((w.W * w.L + 2 * w.W) * (w.W * w.L + 2) for w in wl.wires)
        probe_tab = min(2 * per_task, 16 << 30)
        probe_gbs = 8 * negf.negf_probe_gather(ctx, probe_tab, ilp=8, chain=64) / 1e9
        probe_src = (f"measured: negf_probe_gather, random 8-byte gathers over {probe_tab >> 20}"
                     f" MiB (two tasks' alias tables), 8 independent chains per thread")
    roofs = rooflines(t["prof"], wl, prec, counts, steps, probe_gbs, probe_src)
    ms = t["t_max"] / steps
    dom = max(t["prof"].items(), key=lambda kv: kv[1][1])[0]
    walk_ms = t["prof"].get("walk_kernel", (0, 0.0))[1] / steps
    rel = float(res["se"][0] / abs(res["I"][0])) if res["I"][0] != 0 else float("nan")
    return {"workload": wl.name, "value": t["all_steps"] / (t["t_max"] / 1e3), "unit": UNIT,
            "steps": steps, "warmup": 3, "ms_per_step": ms, "precision": prec,
            "walkers_per_task": N, "tasks": r.n_tasks, "launch_shapes": r.tuning,
            "s_per_current_1pct": s_per_current(ms, walk_ms, rel),
            "kernel_ms_per_step": {k: round(v[1] / steps, 4) for k, v in t["prof"].items()},
            "roofline": roofs.get(dom), "roofline_kernels": roofs}


def run_gpu(args):
    import torch
    from paper_1805_10164_gb300 import build, negf

    rank, world, local = dist_setup(args.gpus)
    torch.cuda.set_device(local)
    build.build()
    wl_all = workload(args.workload or DEFAULT_WORKLOAD, args.energies)
    prec = args.precision or wl_all.precision
    wl = local_workload(wl_all, rank, world)
    N = args.walkers or wl.walkers_per_task
    seed = args.seed + rank          # ranks own different tasks: independent Philox keys
    stream = torch.cuda.current_stream()
    ctx = negf.negf_create(local, stream)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
    runner = Runner(negf, ctx, stream, wl, prec, N, args, seed,
                    tasks_per_wave=args.plan_tasks_per_wave)
    t = timed(runner, negf, ctx, stream, flush, args.steps, args.warmup, rank, world,
              clocks=True)
    res, counts = t["last"]
    # the one exchange step: the wires' partial currents and SE^2 add over ranks
    I_all, se_all = ndist.reduce_current(res["I"], res["se"])
    # end to end through the public API with host buffers (copies inside the region)
    e2e_ms, e2e_steps = 0.0, 0
    n_e2e = max(1, min(args.steps, 2))
    for i in range(n_e2e):
        flush.fill_(float(i))
        torch.cuda.synchronize()
        barrier(world)
        t0 = time.perf_counter()
        _, c2 = runner.host_step(ndist.weak_walker_offset(rank, 20_000 + i, N))
        torch.cuda.synchronize()
        e2e_ms += 1e3 * (time.perf_counter() - t0)
        e2e_steps += int(c2[:, 4].sum())
    e2e_ms = max_over_ranks(e2e_ms, world)
    e2e_steps = sum_over_ranks(float(e2e_steps), world)
    h2d = sum(w.onsite.nbytes + w.eta.nbytes + w.energy.nbytes + w.energy_weight.nbytes
              for w in wl.wires)
    d2h = 8 * (2 * len(wl.wires) + 2 * runner.n_tasks) + 8 * runner.n_tasks * negf.TALLY_FIELDS
    tuning = runner.tuning
    runner.close()
    extra = {}
    if world == 1 and args.compare_fp64 and prec != "fp64":
        extra["fp64_tables"] = fp64_comparison(negf, ctx, stream, flush, wl, args)
    if world == 1 and args.sub_records:
        extra["sub_records"] = {name: sub_record(negf, ctx, stream, flush, name, args, rank, world)
                                for name in SUB_RECORDS if name != (args.workload or DEFAULT_WORKLOAD)}
    negf.negf_destroy(ctx)
    if rank != 0:
        return
    ms_per_step = t["t_max"] / args.steps
    prof = t["prof"]
    roofs = rooflines(prof, wl, prec, counts, args.steps)
    dom = max(prof.items(), key=lambda kv: kv[1][1])[0]
    walk_ms = prof.get("walk_kernel", (0, 0.0))[1] / args.steps
    rel = float(se_all[0] / abs(I_all[0])) if I_all[0] != 0 else float("nan")
    out = {
        "metric": METRIC, "value": t["all_steps"] / (t["t_max"] / 1e3), "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
        "higher_is_better": True, "scaling": "strong" if world > 1 else "weak",
        "vs_baseline": None,
        "dtype": {"fp64": "f64 tables, u32 walks, f64 tally",
                  "fp32": "f32 tables, u32 walks, f64 tally",
                  "split_tf32": "tf32x3 block products (f32 accumulate), f32 tables, u32 walks, "
                                "f64 tally"}[prec],
        "data": "synthetic (seeded square-lattice wire standing in for the paper's CdTe nanowires)",
        "config": {"workload": wl_all.name, "wires": len(wl_all.wires),
                   "tasks": sum(len(w.energy) for w in wl_all.wires),
                   "walkers_per_task": N, "precision": prec, "start_lead": "L",
                   "mu_p": wl.mu_p, "mu_q": wl.mu_q, "kT": wl.kT,
                   "l2": "inputs larger than L2 (tables of one task: tens of GB) and L2 flushed "
                         "between timed steps (258 MiB write, outside the timed events)",
                   "mode": "graph", "launch_shapes": tuning,
                   "parallelism": (f"task partition: each of {world} ranks builds and walks its "
                                   f"own energies; one all-reduce of the partial current"
                                   if world > 1 else "1 GPU, all tasks")},
        "walker_steps_per_step": t["all_steps"] / args.steps,
        "walkers_per_step": t["tot_walkers"] / args.steps * world,
        "current": float(I_all[0]), "current_rel_se": rel,
        "s_per_current_1pct": s_per_current(ms_per_step, walk_ms, rel),
        "kernel_ms_per_step": {k: round(v[1] / args.steps, 4) for k, v in prof.items()},
        "roofline": roofs.get(dom),
        "roofline_kernels": roofs,
        "e2e": {"value": e2e_steps / (e2e_ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h),
                "path": "negf_run over host arrays (the library copies the inputs, builds, "
                        "walks) + negf_current and the tallies read back, wall clock"},
        "gpu_launches": int(sum(v[0] for v in prof.values())),
        "clocks": t["clocks"],
    }
    out.update(extra)
    if world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(wl_all, args)
    print(json.dumps(out), flush=True)

# ------------------------------------------------------------------ gradient (forward + backward)


def run_gradient(args):
    """One step = the differentiable current of the workload's first wire through the public
    torch API (autograd.NegfCurrent: tables keeping their weights, walks with score tallies,
    current) and its backward (negf_current_backward_rgf: the block-column adjoint with the
    RGF blocks checkpointed every CKPT_STRIDE slices; the gradient w.r.t. every onsite energy
    and every dephasing rate).  The API is synchronous (the current and the gradient come back to the
    host), so the timed region is wall time on the device between the step's first launch and
    the gradient's arrival."""
    import torch
    from paper_1805_10164_gb300 import autograd, build, negf

    rank, world, local = dist_setup(args.gpus)
    torch.cuda.set_device(local)
    build.build()
    name = args.workload or "wire_16x100"
    wl = workload(name, args.energies)
    prec = args.precision or wl.precision
    w = wl.wires[0]
    N = args.walkers or wl.walkers_per_task
    stream = torch.cuda.current_stream()
    ctx = negf.negf_create(local, stream)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
    onsite_h = torch.from_numpy(w.onsite).pin_memory()
    eta_h = torch.from_numpy(w.eta).pin_memory()

    def spec_for(i, adjoint="rgf"):
        return autograd.CurrentSpec(W=w.W, L=w.L, t=w.t, energy=w.energy,
                                    energy_weight=w.energy_weight, mu_p=wl.mu_p, mu_q=wl.mu_q,
                                    kT=wl.kT, start_lead=0, walkers_per_task=N, seed=args.seed,
                                    walker_id_offset=ndist.weak_walker_offset(rank, i, N),
                                    max_steps=args.max_steps, precision=prec, adjoint=adjoint,
                                    ckpt_stride=CKPT_STRIDE)

    def one_step(i, onsite, eta, adjoint="rgf"):
        onsite = onsite.detach().requires_grad_(True)
        eta = eta.detach().requires_grad_(True)
        I, se = autograd.NegfCurrent.apply(onsite, eta, ctx, spec_for(i, adjoint))
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
    # context: the same step with the dense adjoint (n x n G kept per task), one-level wires only
    dense_ms = None
    if w.W * w.L <= 6400:
        for i in range(2):
            flush.fill_(float(i))
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            one_step(40_000 + i, on_d, eta_d, adjoint="dense")
            e1.record(stream)
            e1.synchronize()
            dense_ms = e0.elapsed_time(e1)
    negf.negf_destroy(ctx)
    if rank != 0:
        return
    I, se, gV, gE = res
    n_par = 2 * w.W * w.L
    kname = "adjoint_column_kernel"
    klaunch, kms = prof.get(kname, (0, 0.0))
    fl = adjoint_flops(w) * len(w.energy)
    per_launch = fl * args.steps / max(klaunch, 1)
    ach = per_launch / (kms / 1e3 / max(klaunch, 1)) / 1e12 if klaunch else 0.0
    if prec == "fp32":
        peak, psrc = fp32_peak()
    else:
        peak, psrc = 1.25, "nominal FP64 rate of the part (no measured FP64 peak)"
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
                   "step": "forward (tables keeping their weights, walks with score tallies, "
                           "current) + backward (block-column adjoint: gradient w.r.t. every "
                           "onsite energy and dephasing rate) through autograd.NegfCurrent",
                   "adjoint": "block-column RGF adjoint, no dense G",
                   "ckpt_stride": CKPT_STRIDE,
                   "l2": "flushed between timed steps (258 MiB write, outside the timed events)",
                   "mode": "gradient"},
        "walker_steps_per_step": steps_per_step,
        "gradient": {"ms_per_gradient": t_max / args.steps, "parameters": n_par, "I": I,
                     "se": se, "dI_donsite_norm": float(gV.norm()),
                     "dI_deta_norm": float(gE.norm()),
                     "dense_adjoint_ms_per_step": dense_ms},
        "roofline": {"kernel": kname, "bound": "alu", "achieved": round(ach, 3),
                     "peak": peak, "unit": "TFLOP/s", "frac": round(ach / peak, 4),
                     "traffic": None, "peak_source": psrc,
                     "algorithmic_flops_per_launch": per_launch,
                     "avg_launch_ms": round(kms / max(klaunch, 1), 4)},
        "kernel_ms_per_step": {k: round(v[1] / args.steps, 4) for k, v in prof.items()},
        "e2e": {"value": steps_per_step / (e2e_ms / n_e2e / 1e3), "unit": UNIT,
                "h2d_bytes_per_step": int(2 * w.onsite.nbytes),
                "d2h_bytes_per_step": int(2 * w.onsite.nbytes + 16)},
        "gpu_launches": int(sum(v[0] for v in prof.values())),
        "clocks": clk,
    }
    print(json.dumps(out), flush=True)


# ------------------------------------------------------------------ thermal-window sampler

THERMAL_INIT = 9           # evenly spaced energies the adaptive grid starts from (mu +- 8 kT)
THERMAL_TOL = 0.05         # split an interval whose ends' probabilities differ by more than 5 %
THERMAL_MAX = 257          # at most this many grid energies
PLAIN_ENERGIES = 256       # the plain sampler's drawn energies (tables built at each)
PLAIN_WALKERS = 1 << 16    # walkers per drawn energy


def on_grid(w, grid):
    grid = np.asarray(grid, dtype=np.float64)
    return inputs.Wire(W=w.W, L=w.L, t=w.t, onsite=w.onsite, eta=w.eta, energy=grid,
                       energy_weight=np.ones_like(grid))


def plain_thermal(ctx, negf, w, mu, kT, prec, seed):
    """The plain sampler the interpolation replaces: PLAIN_ENERGIES energies drawn from Th on
    mu +- 8 kT (inverse CDF of seeded uniforms), tables built at every drawn energy, walks there,
    G = window x the mean transmission.  Returns (G, se, seconds) with the build, the walks and
    the tally read inside the wall-clock region."""
    F = lambda E: 1.0 / (1.0 + np.exp(-(E - mu) / kT))            # noqa: E731
    F0, F1 = F(mu - 8 * kT), F(mu + 8 * kT)
    u = np.sort(np.random.default_rng(seed).random(PLAIN_ENERGIES))
    Fd = F0 + u * (F1 - F0)
    wd = on_grid(w, mu + kT * np.log(Fd / (1.0 - Fd)))
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    tables, tally = negf.negf_run(ctx, [wd], 0, seed, PLAIN_WALKERS, precision=prec)
    cur = negf.negf_current(ctx, tables, tally, mu + 1.0, mu - 1.0, kT)
    dt = time.perf_counter() - t0
    negf.negf_tally_free(tally)
    negf.negf_tables_free(tables)
    T = cur["T"]
    return (F1 - F0) * T.mean(), (F1 - F0) * T.std(ddof=1) / np.sqrt(T.size), dt


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
    wl = workload(args.workload or "wire_10x50", args.energies)
    prec = args.precision or wl.precision
    mu, kT = 0.0, wl.kT                  # the linear-response reading: E_F = 0
    stream = torch.cuda.current_stream()
    ctx = negf.negf_create(local, stream)
    # the interpolating sampler's grid (adaptive rule), once, outside the timed steps
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    grid = negf.negf_thermal_grid(ctx, wl.wires[0], mu - 8 * kT, mu + 8 * kT, THERMAL_INIT,
                                  THERMAL_TOL, THERMAL_MAX, precision=prec)
    grid_s = time.perf_counter() - t0
    w = on_grid(wl.wires[0], grid)
    N = (args.walkers or wl.walkers_per_task) * len(wl.wires[0].energy)
    dev = inputs.Wire(W=w.W, L=w.L, t=w.t, onsite=torch.from_numpy(w.onsite).cuda(),
                      eta=torch.from_numpy(w.eta).cuda(), energy=torch.from_numpy(w.energy).cuda(),
                      energy_weight=torch.from_numpy(w.energy_weight).cuda())
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
    # seconds per conductance at 1 % SE: interpolating (grid once + tables on it + walks scaled
    # to the walkers 1 % needs) against plain (tables at every drawn energy, scaled to the
    # energies 1 % needs); both wall clock through the public calls
    wall = []
    for i in range(2):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        tb = negf.negf_build_tables(ctx, [dev], precision=prec, memspace="device")
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        r = negf.negf_walk_thermal(ctx, tb, 0, 0, args.seed + 7, N, mu, kT,
                                   walker_id_offset=(40_000 + i) * N, max_steps=args.max_steps)
        t2 = time.perf_counter()
        negf.negf_tables_free(tb)
        wall.append((t1 - t0, t2 - t1, r))
    tab_s, walk_s, ri = wall[-1]
    Gp, sep, plain_s = plain_thermal(ctx, negf, wl.wires[0], mu, kT, prec, args.seed)
    # s(eps) to a relative SE eps: interpolating = fixed (grid + tables) + walk_s (se/G)^2 /
    # eps^2; plain = plain_s (se/G)^2 / eps^2 (its energies scale with 1 / eps^2)
    fixed_i = grid_s + tab_s
    coef_i = walk_s * (ri["se"] / ri["G"]) ** 2 if ri["G"] > 0 else float("inf")
    coef_p = plain_s * (sep / Gp) ** 2 if Gp > 0 else float("inf")
    s_i = lambda eps: fixed_i + coef_i / eps ** 2                  # noqa: E731
    s_p = lambda eps: coef_p / eps ** 2                            # noqa: E731
    comparison = {
        "target": "seconds to G at relative standard error eps, wall clock through the public "
                  "calls, scaled from the measured runs (walkers or drawn energies ~ 1 / eps^2)",
        "interpolating": {
            "grid_points": int(grid.size), "rule": f"split where the distance > {THERMAL_TOL}",
            "grid_s": round(grid_s, 4), "tables_s": round(tab_s, 4),
            "walkers": int(N), "walk_s": round(walk_s, 4), "G": ri["G"], "se": ri["se"],
            "s_per_G_1pct": round(s_i(1e-2), 5), "s_per_G_0.1pct": round(s_i(1e-3), 5)},
        "plain": {
            "energies": PLAIN_ENERGIES, "walkers_per_energy": PLAIN_WALKERS,
            "s": round(plain_s, 4), "G": Gp, "se": sep,
            "s_per_G_1pct": round(s_p(1e-2), 5), "s_per_G_0.1pct": round(s_p(1e-3), 5)},
        "z_interp_vs_plain": (ri["G"] - Gp) / np.hypot(ri["se"], sep),
        "speedup_1pct": round(s_p(1e-2) / s_i(1e-2), 3),
        "speedup_0.1pct": round(s_p(1e-3) / s_i(1e-3), 3),
        # below this relative SE the interpolating sampler is the faster one
        "crossover_eps": (float(np.sqrt((coef_p - coef_i) / fixed_i))
                          if coef_p > coef_i else None),
    }
    # roofline: one 8-byte alias entry per draw (injection + transitions); the grid's tables
    # sit in L2, so the ceiling is the measured random-gather rate over their size
    tab_bytes = grid.size * (w.W * w.L + 2 * w.W) * (w.W * w.L + 2) * 8
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
        "config": {"workload": f"thermal_{wl.name.split('_64E')[0]}_adaptive_kT{kT}",
                   "sampler": "energies from Th = -df/dE on the grid span, chain interpolated "
                              "between grid energies",
                   "grid": [float(w.energy[0]), float(w.energy[-1]), int(grid.size)], "mu": mu,
                   "kT": kT, "walkers_per_step": walkers, "precision": prec,
                   "l2": "flushed between timed steps (258 MiB write, outside the timed events)",
                   "mode": "thermal"},
        "conductance": {"G": res["G"], "se": res["se"], "window": res["window"],
                        "unit": "e^2/h"},
        "comparison": comparison,
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
        while time.perf_counter() - t0 < 20.0 or n_w == 0:
            lead, st, _, _ = thermal.walk(ent, ment, c, tabs[0]["n"], w.W, 0, 0, args.seed,
                                          np.arange(n_w, n_w + 2000, dtype=np.uint64), w.energy,
                                          mu, kT, 1 << 20)
            n_w += 2000
            steps += int(st.sum())
        dt = time.perf_counter() - t0
        out["cpu_baseline"] = {"value": steps / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
                               "sample": f"{grid.size} grid tables + {n_w} walkers "
                                         f"({dt:.1f} s, numpy/LAPACK single thread)"}
    print(json.dumps(out), flush=True)


INELASTIC_SIGMA = 0.1      # width of the Step 7' energy redistribution (about one grid spacing)


def run_inelastic(args):
    """One step = the tables of every grid energy + the Step 7' energy rows + walks whose energy
    changes at every probe visited (negf_walk_inelastic) + the tally read; walker steps/s as the
    headline metric, with the elastic walk of the same tables (sigma = 0) beside it."""
    import torch
    from paper_1805_10164_gb300 import build, negf

    rank, world, local = dist_setup(args.gpus)
    torch.cuda.set_device(local)
    build.build()
    wl = workload(args.workload or "wire_10x50", args.energies)
    prec = args.precision or wl.precision
    w = wl.wires[0]
    nE = len(w.energy)
    N = args.walkers or wl.walkers_per_task
    stream = torch.cuda.current_stream()
    ctx = negf.negf_create(local, stream)
    dev = inputs.Wire(W=w.W, L=w.L, t=w.t, onsite=torch.from_numpy(w.onsite).cuda(),
                      eta=torch.from_numpy(w.eta).cuda(), energy=torch.from_numpy(w.energy).cuda(),
                      energy_weight=torch.from_numpy(w.energy_weight).cuda())
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")

    def one_step(i, wire, memspace, sigma=INELASTIC_SIGMA):
        wid0 = ndist.weak_walker_offset(rank, i, N)
        t = negf.negf_build_tables(ctx, [wire], precision=prec, memspace=memspace)
        try:
            tl = negf.negf_walk_inelastic(ctx, t, 0, args.seed, N, sigma, walker_id_offset=wid0,
                                          max_steps=args.max_steps)
            try:
                cnt = negf.negf_tally_counts(ctx, tl, nE)
                res = negf.negf_current(ctx, t, tl, wl.mu_p, wl.mu_q, wl.kT)
            finally:
                negf.negf_tally_free(tl)
        finally:
            negf.negf_tables_free(t)
        return cnt, res

    for i in range(args.warmup):
        one_step(10_000 + i, dev, "device")
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    clocks = Clocks(local) if rank == 0 else None
    negf.negf_profile_enable(ctx, True)
    total_ms, tot_steps, cnt, res = 0.0, 0.0, None, None
    for i in range(args.steps):
        flush.fill_(float(i))
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        cnt, res = one_step(i, dev, "device")
        e1.record(stream)
        e1.synchronize()
        total_ms += e0.elapsed_time(e1)
        tot_steps += float(cnt[:, 4].sum())
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
    # end to end with host buffers (inputs copied in, the tally and current copied out)
    e2e_ms, e2e_steps = 0.0, 0.0
    for i in range(max(1, min(args.steps, 3))):
        flush.fill_(float(i))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        c2, _ = one_step(20_000 + i, w, "host")
        torch.cuda.synchronize()
        e2e_ms += (time.perf_counter() - t0) * 1e3
        e2e_steps += float(c2[:, 4].sum())
    h2d = w.onsite.nbytes + w.eta.nbytes + w.energy.nbytes + w.energy_weight.nbytes
    cnt0, res0 = one_step(50_000, dev, "device", sigma=0.0)      # the elastic law, same kernel
    # roofline: 8 B per Step 6' entry drawn (injection + transitions) + 8 B per Step 7' entry
    # (every transition to a site); the tables and energy rows of the wire sit mostly in L2, so
    # the ceiling is the measured random-gather rate over their size
    n, K = w.W * w.L, w.W * w.L + 2
    tab_bytes = nE * (n + 2 * w.W) * K * 8 + n * nE * nE * 8
    probe_tab = min(tab_bytes, 16 << 30)
    gps = negf.negf_probe_gather(ctx, probe_tab, ilp=8, chain=64)
    negf.negf_destroy(ctx)
    if rank != 0:
        return
    kname = "inelastic_walk_kernel"
    klaunch, kms = prof.get(kname, (0, 0.0))
    walkers = float(cnt[:, 0].sum())
    absorbed = float(cnt[:, 1].sum() + cnt[:, 2].sum())
    trans = float(cnt[:, 4].sum())
    per_launch = 8.0 * (walkers + trans + (trans - absorbed)) * args.steps / max(klaunch, 1)
    ach = per_launch / (kms / 1e3 / max(klaunch, 1)) / 1e9 if klaunch else 0.0
    peak = 8 * gps / 1e9
    out = {
        "metric": METRIC, "value": all_steps / (t_max / 1e3), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp64": "f64 tables, u32 walks, integer tally",
                  "fp32": "f32 tables, u32 walks, integer tally"}.get(prec, prec),
        "data": "synthetic (seeded square-lattice wire standing in for the paper's CdTe nanowires)",
        "config": {"workload": f"inelastic_{wl.name}_sigma{INELASTIC_SIGMA}",
                   "model": "Buttiker probes with Step 7' energy redistribution: Gaussian kernel "
                            "of width sigma on the energy grid, scaled so that gamma = eta",
                   "walkers_per_task": N, "tasks": nE, "precision": prec,
                   "l2": "flushed between timed steps (258 MiB write, outside the timed events)",
                   "mode": "inelastic"},
        "transmission": {"T_inelastic": [float(x) for x in res["T"]],
                         "T_elastic": [float(x) for x in res0["T"]],
                         "mean_steps_inelastic": trans / max(walkers, 1.0),
                         "mean_steps_elastic": float(cnt0[:, 4].sum()) / max(float(cnt0[:, 0].sum()), 1.0)},
        "kernel_ms_per_step": {k: round(v[1] / args.steps, 4) for k, v in prof.items()},
        "roofline": {"kernel": kname, "bound": "l2", "achieved": round(ach, 1),
                     "peak": round(peak, 1), "unit": "GB/s",
                     "frac": round(ach / peak, 4) if peak else None, "traffic": None,
                     "peak_source": f"measured: negf_probe_gather over {probe_tab >> 20} MiB "
                                    f"(the tables and energy rows), 8 chains per thread",
                     "algorithmic_bytes_per_launch": int(per_launch),
                     "avg_launch_ms": round(kms / max(klaunch, 1), 5)},
        "e2e": {"value": e2e_steps / (e2e_ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(8 * nE * (negf.TALLY_FIELDS + 2) + 16)},
        "gpu_launches": int(sum(v[0] for v in prof.values())),
        "clocks": clk,
    }
    print(json.dumps(out), flush=True)


# ------------------------------------------------------------------ CPU oracle (baseline)

CPU_SLICES = 32            # the oracle's sample: the first slices of the workload's first wire
CPU_WALKERS = 1_000_000    # walkers per sampled energy


def _oracle_energy(job):
    """The oracle (test infrastructure) on one energy of the sample: dense G, Step 6' weights,
    tables (two-level for wide slices, as the library lays them out), walks.  Returns
    (walker steps, seconds)."""
    import numpy as _np
    from oracle import alias, markov, walker, wire
    onsite, eta, t_hop, E, task, seed, walkers = job
    L, W = onsite.shape
    t0 = time.perf_counter()
    g = wire.green_retarded(E, onsite, eta, t_hop)
    phi, _, gam = wire.lead_modes(E, W, t_hop)
    tab = markov.transition_weights(g, (phi, gam))
    ment = _np.stack([alias.vose(tab["mode_w"][p]) for p in range(2)])
    wids = _np.arange(walkers, dtype=_np.uint64)
    if W * L > 2048 or W == 64:
        l1, l2 = alias.build_two_level(tab["w"], L, W)
        _, st = walker.walk_two_level(l1, l2, ment, W * L, L, W, tab["c"] > 0, task, 0, seed,
                                      wids, 1 << 20)
    else:
        ent = alias.build_tables(tab["w"])
        _, st = walker.walk(ent, ment, W * L, W, tab["c"] > 0, task, 0, seed, wids, 1 << 20)
    return int(st.astype(_np.uint64).sum()), time.perf_counter() - t0


def cpu_sample(wl, cores, seed):
    """The oracle on ``cores`` energies of the workload's first wire, truncated to its first
    CPU_SLICES slices, one energy per process (spawned, one thread each).  Returns (walker
    steps, wall seconds, description)."""
    import multiprocessing as mp
    w = wl.wires[0]
    Ls = min(w.L, CPU_SLICES)
    idx = np.unique(np.linspace(0, len(w.energy) - 1, cores).round().astype(int))
    jobs = [(w.onsite[:Ls], w.eta[:Ls], w.t, float(w.energy[k]), int(k), seed,
             CPU_WALKERS) for k in idx]
    t0 = time.perf_counter()
    with mp.get_context("spawn").Pool(len(jobs)) as pool:
        res = pool.map(_oracle_energy, jobs)
    dt = time.perf_counter() - t0
    steps = sum(r[0] for r in res)
    desc = (f"oracle on W={w.W} x L={Ls} (the first {Ls} of {w.L} slices), {len(jobs)} of "
            f"{len(w.energy)} energies x {CPU_WALKERS} walkers, one energy per process "
            f"(numpy/LAPACK, one thread each), tables included")
    return steps, dt, desc, len(jobs)


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def cpu_baseline(wl, args):
    steps, dt, desc, used = cpu_sample(wl, host_cores(), args.seed)
    return {"value": steps / dt, "unit": UNIT, "cores": used, "kind": "oracle",
            "sample": desc + f" ({dt:.1f} s)"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    wl = workload(args.workload or DEFAULT_WORKLOAD, args.energies)
    cores = host_cores()
    for i in range(args.warmup):
        cpu_sample(wl, min(cores, 2), args.seed + i)
    tot_steps, tot_s, desc, used = 0, 0.0, "", 0
    for i in range(args.steps):
        st, dt, desc, used = cpu_sample(wl, cores, args.seed + 100 + i)
        tot_steps += st
        tot_s += dt
    value = tot_steps / tot_s
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1e3 * tot_s / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "impl": "reference",
           "config": {"workload": wl.name, "walkers_per_task": CPU_WALKERS, "sampled": desc},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": used, "kind": "oracle",
                            "sample": desc + " per step"},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default=None,
                    help=f"default {DEFAULT_WORKLOAD} (wire_10x50 for --mode thermal, "
                         f"wire_16x100 for --mode gradient)")
    ap.add_argument("--precision", default=None)
    ap.add_argument("--walkers", type=int, default=None)
    ap.add_argument("--seed", type=int, default=20240607)
    ap.add_argument("--max-steps", type=int, default=1 << 20)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-sub-records", dest="sub_records", action="store_false")
    ap.add_argument("--mode", default="graph", choices=["graph", "thermal", "gradient", "inelastic"])
    ap.add_argument("--no-compare-fp64", dest="compare_fp64", action="store_false")
    ap.add_argument("--plan-tasks-per-wave", type=int, default=0,
                    help="tasks per wave of the captured plan (0: as the memory budget allows; "
                         "1024 for the batched workload)")
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
    elif args.mode == "inelastic":
        run_inelastic(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
