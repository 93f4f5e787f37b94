"""Benchmark of the signature-kernel PDE solve on GB300.

One step = one pass of the whole hot path over one batch: the Gram matrix of
256 x 256 pairs of 128-point, 8-channel time-augmented random walks at dyadic
order 2 (xi ~ N(0, 1/(L d))), FP32 recurrence: increments, coarse-cell
coefficients, the anti-diagonal sweep of 508 x 508 refined cells per pair,
and the corner values, all inside one kernel launch.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line (rank 0).  `value` is refined grid cells per second over
the whole job (inputs resident in HBM, L2 flushed between timed steps);
`e2e` is the same metric through the public API with the inputs copied from
pinned host memory and the Gram read back every step.  `--impl reference`
times the FP64 CPU oracle on this host's cores on a bounded sample of the
same workload.
"""
from __future__ import annotations

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

METRIC = "PDE grid cells/s and kernel pairs/s at stated rel err vs FP64 oracle; % FP32 FMA peak"
WORKLOAD = "gram 256x256, L=M=128, d=8 time-augmented random walks, dyadic order 2, fp32 recurrence"
BX = BY = 256
L = M = 128
D = 8
LAM = 2
NI = (L - 1) << LAM
NJ = (M - 1) << LAM
CELLS_PER_PAIR = NI * NJ
COARSE_PER_PAIR = (L - 1) * (M - 1)
FLOP_PER_CELL = 3           # add, multiply, add of the printed scheme (h precomputed per coarse cell)
L2_FLUSH_BYTES = 256 << 20  # > 129 MB of L2


def peaks():
    p = {}
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            p = json.load(f)
    return p


def fp32_peak_tflops(sms: int):
    """FP32 FMA peak: SMs x 128 lanes x 2 flop x max SM clock."""
    p = peaks()
    mhz = float(p.get("sm_max_mhz", 2070.0))
    return sms * 128 * 2 * mhz * 1e6 / 1e12, mhz, ("measured" if "sm_max_mhz" in p else "fallback")


def profile_traffic():
    """DRAM bytes per launch of the chained kernel from the committed ncu
    summary, when that summary was taken on the current kernel source."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "chain_f32_gram256.md")
    src = os.path.join(ROOT, "paper_2006_14794_gb300", "csrc", "fwd_chain.cu")
    if not (os.path.exists(path) and os.path.exists(src)):
        return None, None
    fields = {}
    for line in open(path):
        if ":" in line and not line.startswith("|"):
            k, _, v = line.partition(":")
            fields[k.strip()] = v.strip()
    sha = hashlib.sha256(open(src, "rb").read()).hexdigest()
    if fields.get("source_sha256") != sha:
        return None, None
    try:
        return int(fields["traffic_bytes_per_launch"]), "profiles/chain_f32_gram256.md"
    except (KeyError, ValueError):
        return None, None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        # the raw samples: SIGK_CLOCKS_DIR if set, else the temporary directory
        out_dir = os.environ.get("SIGK_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(out_dir, "sigk_clocks_rank%d.csv" % gpu_index)

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.fh,
                stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [s.strip() for s in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


def make_inputs(rank: int):
    from paper_2006_14794_gb300 import inputs
    w = inputs.gram_256(seed=inputs.SEEDS[2] + 1000 * rank)
    X32, X64 = inputs.f32(w["X"])
    Y32, Y64 = inputs.f32(w["Y"])
    return X32, Y32, X64, Y64


def oracle_sample_rate(X64, Y64, budget_s: float):
    """Oracle cells/s on this host's cores: whole rows of the Gram, until the
    time budget is spent (at least one row)."""
    import oracle
    t0 = time.perf_counter()
    rows = 0
    while True:
        oracle.gram(X64[rows:rows + 1], Y64, LAM)
        rows += 1
        if time.perf_counter() - t0 >= budget_s or rows == BX:
            break
    dt = time.perf_counter() - t0
    pairs = rows * BY
    return pairs * CELLS_PER_PAIR / dt, pairs, dt, oracle.num_threads()


def max_over_ranks(value: float, device=None) -> float:
    """The slowest rank's time: every rank passes its own, every rank gets the max
    (no-op without an initialised process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    _, _, X64, Y64 = make_inputs(0)
    vals = []
    budget = float(os.environ.get("SIGK_REF_STEP_SECONDS", "8"))
    for _ in range(args.warmup):
        oracle_sample_rate(X64, Y64, 0.5)
    samples = []
    for _ in range(args.steps):
        rate, pairs, dt, cores = oracle_sample_rate(X64, Y64, budget)
        vals.append(rate)
        samples.append(pairs)
    value = statistics.median(vals)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "cells/s",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * BX * BY * CELLS_PER_PAIR / value,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "l2": "n/a (host)"},
        "pairs_per_s": value / CELLS_PER_PAIR,
        "cpu_baseline": {"value": value, "unit": "cells/s", "cores": cores, "kind": "oracle",
                         "sample": "%d of 65536 pairs (whole Gram rows) per step, ~%gs each" % (
                             min(samples), budget)},
        "e2e": {"value": value, "unit": "cells/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_gpu(args):
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if ws > 1 else 0)
    torch.cuda.set_device(dev)
    from paper_2006_14794_gb300 import sigk
    sigk.lib()
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count

    X32, Y32, X64, Y64 = make_inputs(rank)
    Xd = torch.from_numpy(X32).to(dev)
    Yd = torch.from_numpy(Y32).to(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize(dev)

    # ---- warm-up (also the parity sample)
    out = None
    for _ in range(max(args.warmup, 3)):
        out = sigk.gram(Xd, Yd, LAM)
    torch.cuda.synchronize(dev)

    # ---- timed region: inputs resident, L2 flushed before each step
    st = torch.cuda.current_stream(dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    clocks = ClockSampler(local if ws > 1 else 0)
    clocks.start()
    time.sleep(0.3)
    barrier()
    t_wall0 = time.perf_counter()
    for i in range(args.steps):
        flush.fill_(float(i))
        ev[i][0].record(st)
        out = sigk.gram(Xd, Yd, LAM)
        ev[i][1].record(st)
    barrier()
    t_wall = time.perf_counter() - t_wall0
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    ms = max_over_ranks(sum(step_ms) / len(step_ms), dev)
    cells_step = BX * BY * CELLS_PER_PAIR
    value = ws * cells_step / (ms * 1e-3)

    # ---- end to end through the public API, host buffers (pinned)
    Xh = torch.from_numpy(X32).pin_memory()
    Yh = torch.from_numpy(Y32).pin_memory()
    Oh = torch.empty(BX, BY, dtype=torch.float32).pin_memory()
    e2e_steps = max(1, args.steps)
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for i in range(e2e_steps):
        xd = Xh.to(dev, non_blocking=True)
        yd = Yh.to(dev, non_blocking=True)
        o = sigk.gram(xd, yd, LAM)
        Oh.copy_(o, non_blocking=True)
    e1.record(st)
    barrier()
    e2e_ms = max_over_ranks(e0.elapsed_time(e1) / e2e_steps, dev)
    e2e_value = ws * cells_step / (e2e_ms * 1e-3)

    # ---- parity of the timed output with the oracle on sampled entries
    line = None
    if rank == 0:
        import oracle
        got = out.cpu().numpy()
        rng = np.random.default_rng(11)
        idx = rng.integers(0, BX, size=(48, 2))
        ref = np.array([oracle.sigkernel(X64[i], Y64[j], LAM) for i, j in idx])
        g = got[idx[:, 0], idx[:, 1]]
        rel = float(np.max(np.abs(g - ref) / np.maximum(np.abs(ref), 1e-3)))

        peak_tf, mhz, peak_src = fp32_peak_tflops(sms)
        traffic, traffic_src = profile_traffic()
        flop = BX * BY * (CELLS_PER_PAIR * FLOP_PER_CELL + COARSE_PER_PAIR * 2 * D)
        achieved_tf = flop / (ms * 1e-3) / 1e12

        # plain FP64 per-pair GPU sweep on the same workload (comparison baseline)
        f64 = None
        if not args.skip_fp64:
            Xd64 = torch.from_numpy(X64).to(dev)
            Yd64 = torch.from_numpy(Y64).to(dev)
            sigk.gram(Xd64[:8], Yd64[:8], LAM)
            torch.cuda.synchronize(dev)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(st)
            o64 = sigk.gram(Xd64, Yd64, LAM)
            b.record(st)
            torch.cuda.synchronize(dev)
            ms64 = a.elapsed_time(b)
            rel64 = float(np.max(np.abs(o64.cpu().numpy()[idx[:, 0], idx[:, 1]] - ref) /
                                 np.maximum(np.abs(ref), 1e-3)))
            f64 = {"value": cells_step / (ms64 * 1e-3), "unit": "cells/s", "ms_per_step": ms64,
                   "rel_err_vs_oracle": rel64, "kernel": "plain per-pair anti-diagonal FP64"}

        cpu = None
        if not args.skip_cpu:
            rate, pairs, dt, cores = oracle_sample_rate(X64, Y64, args.cpu_seconds)
            cpu = {"value": rate, "unit": "cells/s", "cores": cores, "kind": "oracle",
                   "sample": "%d of 65536 pairs (whole Gram rows), %.1f s" % (pairs, dt)}

        line = {
            "metric": METRIC, "value": value, "unit": "cells/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "pairs_per_step": BX * BY,
                       "cells_per_pair": CELLS_PER_PAIR, "l2": "flushed (256 MB write) before each step",
                       "parallelism": "dp%d (independent Gram per GPU)" % ws},
            "pairs_per_s": value / CELLS_PER_PAIR,
            "rel_err_vs_oracle": rel,
            "fp32_fma_peak_frac": achieved_tf / peak_tf,
            "roofline": {"bound": "alu", "achieved": achieved_tf, "peak": peak_tf,
                         "unit": "TFLOP/s", "frac": achieved_tf / peak_tf, "traffic": traffic,
                         "traffic_source": traffic_src,
                         "peak_source": "%s SMs x 128 FP32 lanes x 2 flop x %.0f MHz (%s max SM clock)" % (
                             sms, mhz, peak_src),
                         "work": "3 flop per refined cell + 2d flop per coarse cell"},
            "clocks": clk,
            "e2e": {"value": e2e_value, "unit": "cells/s",
                    "h2d_bytes_per_step": int(X32.nbytes + Y32.nbytes),
                    "d2h_bytes_per_step": int(BX * BY * 4), "ms_per_step": e2e_ms},
            "gpu_launches": args.steps,
            "wall_s_timed_region": t_wall,
            "fp64_plain_gpu": f64,
            "cpu_baseline": cpu,
        }
        if ws == 1 and not args.skip_workloads:
            # the other configurations, measured in the same run (one GPU)
            del flush
            torch.cuda.empty_cache()
            line["workloads"] = run_workloads(args)
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()
    return 0


# ---- the other workloads ----------------------------------------------------
#
# Each is a parity case of the test suite at full size, measured the same way
# as the headline: W >= 3 untimed calls, then >= 5 timed calls bracketed by
# CUDA events on the launching stream with a 256 MB L2 flush before each, the
# result checked against the oracle on sampled outputs, and the oracle timed
# on this host's cores on a bounded sample of the same workload.  The default
# run reports all of them under the headline line's "workloads" key;
# `--workload NAME` prints one of them as a line of its own (with e2e).

# Dense FP64 of the GB300, nominal (MEASURED_PEAKS.json has no FP64 figure).
FP64_PEAK_NOMINAL_TF = 1.25


def _pick(rng_seed, n, k, must=()):
    rng = np.random.default_rng(rng_seed)
    idx = list(must) + [int(v) for v in rng.choice(n, size=min(k, n), replace=False)]
    return sorted(set(idx))


def _timed_oracle(fn):
    t0 = time.perf_counter()
    r = fn()
    return r, time.perf_counter() - t0


def _workload(name, batch=0, cache=None):
    """The workload `name` as a dict:
    desc, dtype ("f32" | "f64"), step() (one timed call; returns what parity
    reads), cells and pairs per step, flop per step (the algorithmic work),
    kernels (the launches of one step, dominant first), oracle_rate(budget)
    -> (cells/s, sample, threads), parity(out) -> (rel err, sample),
    host_step(*host) with host buffers and its h2d / d2h bytes.
    batch > 0 keeps the first `batch` pairs / paths (a small case for
    profilers); cache: dict shared between workloads (oracle results)."""
    import torch
    from paper_2006_14794_gb300 import inputs, sigk, tune
    import oracle
    cache = {} if cache is None else cache

    if name in ("gram_small_f64", "gram_small_f32"):
        # config 1: Gram 8 x 8, L=32, d=3 (time + 2 walks), dyadic order 1,
        # plus the 8 straight-line pairs of the closed-form check
        w = inputs.gram_small()
        lam = w["dyadic_order"]
        f64 = name.endswith("f64")
        tdt = torch.float64 if f64 else torch.float32
        X32, X64 = inputs.f32(w["X"])
        Y32, Y64 = inputs.f32(w["Y"])
        lx32, lx64 = inputs.f32(w["lines_x"])
        ly32, ly64 = inputs.f32(w["lines_y"])
        src = (X64, Y64, lx64, ly64) if f64 else (X32, Y32, lx32, ly32)
        Xd, Yd, LXd, LYd = [torch.as_tensor(a, dtype=tdt).cuda() for a in src]
        n = (32 - 1) << lam
        cells = (64 + 8) * n * n
        coarse = (64 + 8) * 31 * 31

        def step():
            return sigk.gram(Xd, Yd, lam), sigk.pairs(LXd, LYd, lam)

        def refs():
            if "gram_small" not in cache:
                cache["gram_small"] = _timed_oracle(
                    lambda: (oracle.gram(X64, Y64, lam), oracle.pairs(lx64, ly64, lam)))
            return cache["gram_small"]

        def oracle_rate(budget):
            _, dt = refs()
            return cells / dt, "the whole step (64 Gram entries + 8 straight-line pairs)", oracle.num_threads()

        def parity(out):
            (K, Ln), _ = refs()
            g = np.concatenate([out[0].double().cpu().numpy().ravel(), out[1].double().cpu().numpy()])
            r = np.concatenate([K.ravel(), Ln])
            return float(np.max(np.abs(g - r) / np.maximum(np.abs(r), 1e-3))), "all 72 outputs"

        host = tuple(torch.as_tensor(a, dtype=tdt).pin_memory() for a in src) + (
            torch.empty(8, 8, dtype=tdt).pin_memory(), torch.empty(8, dtype=tdt).pin_memory())

        def host_step(hx, hy, hlx, hly, hk, hl):
            k = sigk.gram(hx.cuda(non_blocking=True), hy.cuda(non_blocking=True), lam)
            l = sigk.pairs(hlx.cuda(non_blocking=True), hly.cuda(non_blocking=True), lam)
            hk.copy_(k, non_blocking=True)
            hl.copy_(l, non_blocking=True)
        es = 8 if f64 else 4
        return dict(
            desc="Gram 8x8, L=M=32, d=3 (time + 2 walks), dyadic order 1, plus 8 straight-line pairs, %s"
                 % ("fp64 (plain per-pair sweep, the printed scheme)" if f64 else "fp32 (chained register sweep)"),
            dtype="f64" if f64 else "f32", step=step, cells=cells, pairs=72,
            flop=3 * cells + 2 * 3 * coarse,
            kernels="plain_kernel<double>" if f64 else "chain_f32_kernel",
            oracle_rate=oracle_rate, parity=parity, host_step=host_step, host=host,
            h2d=sum(a.nbytes for a in src), d2h=72 * es)

    if name == "uneven4096":
        # config 3: 4096 pairs, L, M ~ U{16..512}, d=16 walks, dyadic order 1
        # (batch > 0: the first `batch` pairs, 4096 for all, on the warp-stack
        # schedule, untuned: a case for profilers without the tuner's runs)
        w = inputs.uneven_pairs()
        lam = w["dyadic_order"]
        np_all = 4096
        tuned = batch <= 0
        if 0 < batch < 4096:
            np_all = batch
            w = dict(w, Xp=w["Xp"][:w["x_off"][batch]], Yp=w["Yp"][:w["y_off"][batch]],
                     x_off=w["x_off"][:batch + 1], y_off=w["y_off"][:batch + 1])
        X32, X64 = inputs.f32(w["Xp"])
        Y32, Y64 = inputs.f32(w["Yp"])
        xo, yo = w["x_off"], w["y_off"]
        lx, ly = xo[1:] - xo[:-1], yo[1:] - yo[:-1]
        cells = int(np.sum(((lx - 1) << lam) * ((ly - 1) << lam)))
        coarse = int(np.sum((lx - 1) * (ly - 1)))
        Xd, Yd = torch.from_numpy(X32).cuda(), torch.from_numpy(Y32).cuda()
        xod, yod = torch.as_tensor(xo).cuda(), torch.as_tensor(yo).cuda()
        # the schedule chosen by timing the candidates on these inputs (before
        # the timed region), then the whole call captured as one CUDA graph
        if tuned:
            sched, _ = tune.tune("pairs_varlen", Xd, xod, Yd, yod, lam, 512, store=False)
        else:
            sched = sigk.Schedule(sigk.REC_CHAIN)
        g = sigk.graphed(sigk.pairs_varlen, Xd, xod, Yd, yod, lam, max_len=512, schedule=sched)

        def step():
            return g.replay()

        def host_step(hx, hy, hxo, hyo, ho):
            o = g(hx, hxo, hy, hyo)
            ho.copy_(o, non_blocking=True)

        def oracle_rate(budget):
            t0 = time.perf_counter(); done = 0; cc = 0
            while time.perf_counter() - t0 < budget and done < np_all:
                b = np.arange(done, min(done + 64, np_all))
                sub_x = np.concatenate([X64[xo[i]:xo[i + 1]] for i in b])
                sub_y = np.concatenate([Y64[yo[i]:yo[i + 1]] for i in b])
                sxo = np.concatenate([[0], np.cumsum(lx[b])]); syo = np.concatenate([[0], np.cumsum(ly[b])])
                oracle.pairs_varlen(sub_x, sxo, sub_y, syo, lam)
                cc += int(np.sum(((lx[b] - 1) << lam) * ((ly[b] - 1) << lam))); done = b[-1] + 1
            return cc / (time.perf_counter() - t0), "pairs 0..%d of %d" % (done - 1, np_all), oracle.num_threads()

        def parity(out):
            o = out.cpu().numpy()
            cl = (lx - 1) * (ly - 1)
            idx = _pick(8, np_all, 60, must=(0, np_all - 1, int(np.argmax(cl)), int(np.argmin(cl))))
            ref = np.array([oracle.sigkernel(X64[xo[b]:xo[b + 1]], Y64[yo[b]:yo[b + 1]], lam) for b in idx])
            return float(np.max(np.abs(o[idx] - ref) / np.maximum(np.abs(ref), 1e-3))), \
                "%d pairs (60 random, the first, the last, the most and the fewest cells)" % len(idx)
        host = (torch.from_numpy(X32).pin_memory(), torch.from_numpy(Y32).pin_memory(),
                torch.as_tensor(xo).pin_memory(), torch.as_tensor(yo).pin_memory(),
                torch.empty(np_all).pin_memory())
        return dict(
            desc="%d pairs, L,M ~ U{16..512}, d=16 walks, dyadic order 1, fp32; %s schedule "
                 "rec=%d rows_per_lane=%d coef_path=%d orient=%d, one CUDA graph per call"
                 % (np_all, "tuned" if tuned else "warp-stack", sched.rec, sched.rows_per_lane,
                    sched.coef_path, sched.orient),
            dtype="f32", step=step, cells=cells, pairs=np_all, flop=3 * cells + 2 * 16 * coarse,
            kernels=_uneven_kernels(sched), oracle_rate=oracle_rate, parity=parity,
            host_step=host_step, host=host, h2d=X32.nbytes + Y32.nbytes + xo.nbytes + yo.nbytes,
            d2h=np_all * 4)

    if name.startswith("long64") and not name.endswith("_grad"):
        # config 5: 64 pairs, L=M=4096, d=64 (time + 63 walks), dyadic order 0 / 1
        lam = int(name[len("long64_l")])
        f64 = name.endswith("_f64")
        w = inputs.long_pairs()
        nb = batch if 0 < batch < 64 else 64
        X32, X64 = inputs.f32(w["X"][:nb])
        Y32, Y64 = inputs.f32(w["Y"][:nb])
        n = (4095 << lam)
        cells = nb * n * n
        tdt = torch.float64 if f64 else torch.float32
        Xd = torch.as_tensor(X64 if f64 else X32, dtype=tdt).cuda()
        Yd = torch.as_tensor(Y64 if f64 else Y32, dtype=tdt).cuda()
        # FP64 takes the strip path (the recurrence precision form); FP32 the
        # library's default (strip path, tensor-core coefficients)
        rec = sigk.REC_CHAIN if f64 else sigk.REC_AUTO

        def step():
            return sigk.pairs(Xd, Yd, lam, rec=rec)

        def host_step(hx, hy, ho):
            o = sigk.pairs(hx.cuda(non_blocking=True), hy.cuda(non_blocking=True), lam, rec=rec)
            ho.copy_(o, non_blocking=True)

        # the oracle on 8 of the pairs (spread over the batch), timed, and
        # their values as the parity reference; the rate extrapolates to 64
        sample = sorted(set(int(v) for v in np.linspace(0, nb - 1, min(8, nb)).round()))

        def refs():
            key = ("long64", lam, nb)
            if key not in cache:
                cache[key] = _timed_oracle(lambda: oracle.pairs(X64[sample], Y64[sample], lam))
            return cache[key]

        def oracle_rate(budget):
            _, dt = refs()
            return len(sample) * n * n / dt, "%d of %d pairs (indices %s), one OpenMP thread per pair; " \
                "the rate extrapolates to the whole batch" % (len(sample), nb, sample), \
                min(len(sample), oracle.num_threads())

        def parity(out):
            ref, _ = refs()
            o = out.double().cpu().numpy()[sample]
            return float(np.max(np.abs(o - ref) / np.maximum(np.abs(ref), 1e-3))), \
                "%d pairs %s" % (len(sample), sample)
        host = (torch.as_tensor(X64 if f64 else X32, dtype=tdt).pin_memory(),
                torch.as_tensor(Y64 if f64 else Y32, dtype=tdt).pin_memory(),
                torch.empty(nb, dtype=tdt).pin_memory())
        es = 8 if f64 else 4
        kern = ("coef_kernel<double> (FMA contraction) + strip_kernel<double, 8, lambda> (256-row strips)"
                if f64 else "coef_tc5_kernel (split-TF32 tcgen05 contraction) + strip_kernel<float> "
                            "(%d-row strips)" % (256 if lam == 0 else 512))
        return dict(
            desc="%d pairs, L=M=4096, d=64 time-augmented walks, dyadic order %d, %s"
                 % (nb, lam, "fp64 recurrence and contraction (strip path)" if f64 else "fp32 recurrence, "
                    "split-TF32 increment Gram"),
            dtype="f64" if f64 else "f32", step=step, cells=cells, pairs=nb,
            flop=3 * cells + 2 * 64 * nb * 4095 * 4095, kernels=kern, oracle_rate=oracle_rate,
            parity=parity, host_step=host_step, host=host, h2d=2 * nb * 4096 * 64 * es, d2h=nb * es)

    if name == "long64_l1_grad":
        # config 5's backward: the gradient of sum_b g_b k(X_b, Y_b) for the
        # 64 long pairs at dyadic order 1 (strip path: the forward with
        # checkpoints, the adjoint undoing it in place, the chain rule)
        lam = 1
        w = inputs.long_pairs()
        nb = batch if 0 < batch < 64 else 64
        X32, X64 = inputs.f32(w["X"][:nb])
        Y32, Y64 = inputs.f32(w["Y"][:nb])
        n = 4095 << lam
        cells = nb * n * n
        coarse = nb * 4095 * 4095
        Xd, Yd = torch.from_numpy(X32).cuda(), torch.from_numpy(Y32).cuda()
        gv = np.random.default_rng(55).normal(size=nb)
        gd = torch.as_tensor(gv, dtype=torch.float32).cuda()

        def step():
            return sigk.pairs_backward(gd, Xd, Yd, lam)

        sample = [0, nb - 1] if nb > 1 else [0]

        def refs():
            key = ("long64_grad", nb)
            if key not in cache:
                cache[key] = _timed_oracle(lambda: oracle.pairs_grad(X64[sample], Y64[sample], lam, gv[sample]))
            return cache[key]

        def oracle_rate(budget):
            _, dt = refs()
            return len(sample) * n * n / dt, "values and gradients of pairs %s; forward cells of those pairs " \
                "per second" % sample, min(len(sample), oracle.num_threads())

        def parity(out):
            (rX, rY), _ = refs()
            dX, dY = out
            e = 0.0
            for got, ref in ((dX.double().cpu().numpy()[sample], rX), (dY.double().cpu().numpy()[sample], rY)):
                e = max(e, float(np.max(np.abs(got - ref)) / np.max(np.abs(ref))))
            return e, "dX, dY of pairs %s (max |g - g_ref| / max |g_ref|)" % sample

        host = (torch.from_numpy(X32).pin_memory(), torch.from_numpy(Y32).pin_memory(),
                torch.empty(X32.shape).pin_memory())

        def host_step(hx, hy, hg):
            dX, _ = sigk.pairs_backward(gd, hx.cuda(non_blocking=True), hy.cuda(non_blocking=True), lam)
            hg.copy_(dX, non_blocking=True)
        # flop: the coefficients (2d a coarse cell), the forward sweep (3 a
        # refined cell), the adjoint (7: two multiply-adds, an add, the dk/dc
        # multiply-add) and the undone forward step (3), the chain rule
        # (2 x 2d a coarse cell)
        return dict(
            desc="gradient of sum_b g_b k(X_b, Y_b), %d pairs, L=M=4096, d=64 time-augmented walks, dyadic "
                 "order 1, fp32 (strip adjoint with checkpoints every 64 steps)" % nb,
            dtype="f32", step=step, cells=cells, pairs=nb, flop=2 * 64 * coarse + 13 * cells + 4 * 64 * coarse,
            kernels="strip_adj_kernel + strip_kernel (checkpointing forward) + coef_tc5_kernel + grad_chain_kernel",
            oracle_rate=oracle_rate, parity=parity, host_step=host_step, host=host,
            h2d=X32.nbytes + Y32.nbytes, d2h=X32.nbytes)

    if name in ("mmd128", "mmd128_rbf"):
        # config 4: MMD^2 between 128 and 128 paths, L=256, d=32, dyadic order 1;
        # one step = the loss and dL/dX.  mmd128_rbf: the same with the RBF
        # lift (sigma = 1) of Sec. 2.2
        rbf_sigma = 1.0 if name == "mmd128_rbf" else None
        var = sigk.Variant(static_kernel="rbf", sigma=rbf_sigma) if rbf_sigma else None
        okw = dict(static_kernel="rbf", sigma=rbf_sigma) if rbf_sigma else {}
        w = inputs.mmd_batches()
        lam = w["dyadic_order"]
        nb = batch if 1 < batch < 128 else 128
        X32, X64 = inputs.f32(w["X"][:nb])
        Y32, Y64 = inputs.f32(w["Y"][:nb])
        Yd = torch.from_numpy(Y32).cuda()
        Xd = torch.from_numpy(X32).cuda()
        nc, nn = 510 * 510, 255 * 255
        # the pairs the U-statistic uses: i < j of Kxx and Kyy, all of Kxy
        u_pairs = nb * (nb - 1) + nb * nb
        cells = u_pairs * nc
        # algorithmic flop of the step as it runs: Kxx and Kyy are symmetric
        # Grams (pairs i <= j, n(n+1)/2 of them), Kxy is full.  Coefficients
        # (2d per coarse cell) and forward sweeps (3 per refined cell) of all
        # three; adjoint sweeps of Kxx and Kxy, the Grams with X in them (7 per
        # refined cell: two multiply-adds, an add and the dk/dc multiply-add);
        # chain-rule contractions into dX, 2 (255 nb)^2 d each: one for Kxy,
        # and for Kxx the row-role and column-role contractions over i <= j,
        # together one full contraction
        sym = nb * (nb + 1) // 2
        fwd_pairs = 2 * sym + nb * nb
        adj_pairs = sym + nb * nb
        nch = 32
        flop = (fwd_pairs * nn * 2 * nch + fwd_pairs * nc * 3 + adj_pairs * nc * 7
                + 2 * 2 * (255 * nb) ** 2 * nch)
        if rbf_sigma:
            # the lift: 9d flop per coarse cell for its coefficient (exponentials
            # not counted); its chain rule: squared distances (3d per point pair)
            # and the contractions over points
            flop = (fwd_pairs * nn * 9 * nch + fwd_pairs * nc * 3 + adj_pairs * nc * 7
                    + adj_pairs * 256 * 256 * 3 * nch + 2 * 2 * (256 * nb) ** 2 * nch)

        def step():
            X = Xd.clone().requires_grad_(True)
            v = sigk.mmd2_loss(X, Yd, lam, variant=var)
            v.backward()
            return X.grad

        def host_step(hx, hy, hg):
            X = hx.cuda(non_blocking=True).requires_grad_(True)
            v = sigk.mmd2_loss(X, hy.cuda(non_blocking=True), lam, variant=var)
            v.backward()
            hg.copy_(X.grad, non_blocking=True)

        rows = [0, min(77, nb - 1)]

        def refs():
            key = (name, nb)
            if key not in cache:
                m = n = nb

                def run():
                    gxx = np.full((1, m), 1.0 / (m * (m - 1)))
                    gxy = np.full((1, n), -2.0 / (m * n))
                    out = []
                    for i in rows:
                        gi = gxx.copy()
                        gi[0, i] = 0.0
                        a, _ = oracle.gram_grad(X64[i:i + 1], X64, lam, gi, want_dy=False, **okw)
                        b, _ = oracle.gram_grad(X64[i:i + 1], Y64, lam, gxy, want_dy=False, **okw)
                        out.append(2.0 * a[0] + b[0])
                    return out
                cache[key] = _timed_oracle(run)
            return cache[key]

        def oracle_rate(budget):
            _, dt = refs()
            pairs_done = len(rows) * 2 * nb
            return pairs_done * nc / dt, "values and gradients of the %d pairs of rows %s of Kxx and Kxy " \
                "(dL/dX_i for those rows); forward cells of those pairs per second" % (pairs_done, rows), \
                oracle.num_threads()

        def parity(out):
            want, _ = refs()
            g = out.double().cpu().numpy()
            err = max(float(np.max(np.abs(g[i] - wv)) / np.max(np.abs(wv))) for i, wv in zip(rows, want))
            return err, "dL/dX rows %s (max |g - g_ref| / max |g_ref| per row)" % rows
        host = (torch.from_numpy(X32).pin_memory(), torch.from_numpy(Y32).pin_memory(),
                torch.empty(X32.shape).pin_memory())
        return dict(
            desc="MMD^2 %d vs %d, L=256, d=32 walks + drift, dyadic order 1, %sloss + dL/dX, fp32 "
                 "(cells: the forward cells of the U-statistic's %d distinct pairs)"
                 % (nb, nb, "RBF lift (sigma 1), " if rbf_sigma else "", u_pairs),
            dtype="f32", step=step, cells=cells, pairs=u_pairs, flop=flop,
            kernels=("rbf_coef_kernel + chain_band_kernel + chain_band_adj_kernel + rbf_wt_kernel + "
                     "dense_gemm_kernel (band form; fused value-and-gradient calls for Kxx and Kxy)" if rbf_sigma else
                     "chain_band_adj_kernel + band_gemm_kernel + band_coef_kernel + chain_band_kernel "
                     "(band form; fused value-and-gradient calls for Kxx and Kxy)"),
            oracle_rate=oracle_rate, parity=parity, host_step=host_step, host=host,
            h2d=X32.nbytes + Y32.nbytes, d2h=X32.nbytes)

    if name in ("gram256_implicit", "gram256_rbf"):
        # the benchmark Gram with the implicit scheme (Sec. 3.1 remark) or the
        # RBF static-kernel lift (Sec. 2.2, sigma = 1)
        w = inputs.gram_256()
        lam = w["dyadic_order"]
        nb = batch if 0 < batch < 256 else 256
        X32, X64 = inputs.f32(w["X"][:nb])
        Y32, Y64 = inputs.f32(w["Y"][:nb])
        nbx, nby, L, d = X32.shape[0], Y32.shape[0], X32.shape[1], X32.shape[2]
        if name == "gram256_implicit":
            v = sigk.Variant(scheme="implicit")
            okw = dict(scheme="implicit")
            cflop = 2 * d + 2          # <dx, dy>, then c / (1 - c/2)
            what = "implicit scheme"
            kern = "chain_f32_kernel (implicit instance)"
        else:
            v = sigk.Variant(static_kernel="rbf", sigma=1.0)
            okw = dict(static_kernel="rbf", sigma=1.0)
            cflop = 9 * d              # |u|^2, <u,dx>, <u,dy>, <dx,dy> and u = x_p - y_q per channel
            what = "RBF lift (sigma = 1), explicit scheme"
            kern = "rbf_coef_kernel + chain_band_kernel"
        n = (L - 1) << lam
        cells = nbx * nby * n * n
        coarse = nbx * nby * (L - 1) * (L - 1)
        Xd, Yd = torch.from_numpy(X32).cuda(), torch.from_numpy(Y32).cuda()

        def step():
            return sigk.gram(Xd, Yd, lam, variant=v)

        def host_step(hx, hy, ho):
            o = sigk.gram(hx.cuda(non_blocking=True), hy.cuda(non_blocking=True), lam, variant=v)
            ho.copy_(o, non_blocking=True)

        def oracle_rate(budget):
            t0 = time.perf_counter(); rows = 0
            while time.perf_counter() - t0 < budget and rows < nbx:
                oracle.gram(X64[rows:rows + 1], Y64, lam, **okw)
                rows += 1
            return rows * nby * n * n / (time.perf_counter() - t0), "%d Gram rows of %d" % (rows, nbx), \
                oracle.num_threads()

        def parity(out):
            rng = np.random.default_rng(7)
            idx = rng.choice(nbx * nby, 16, replace=False)
            o = out.cpu().numpy()
            errs = []
            for t in idx:
                i, j = divmod(int(t), nby)
                ref = oracle.sigkernel(X64[i], Y64[j], lam, **okw)
                errs.append(abs(o[i, j] - ref) / max(abs(ref), 1e-3))
            return float(max(errs)), "16 sampled entries"
        host = (torch.from_numpy(X32).pin_memory(), torch.from_numpy(Y32).pin_memory(),
                torch.empty(nbx, nby).pin_memory())
        return dict(
            desc="gram %dx%d, L=M=128, d=8 time-augmented random walks, dyadic order 2, fp32, %s"
                 % (nbx, nby, what),
            dtype="f32", step=step, cells=cells, pairs=nbx * nby, flop=3 * cells + cflop * coarse,
            kernels=kern, oracle_rate=oracle_rate, parity=parity, host_step=host_step, host=host,
            h2d=X32.nbytes + Y32.nbytes, d2h=nbx * nby * 4)

    if name == "surface256":
        # the solution surface on the sample grid for the benchmark's 65536
        # pairs (X_i, Y_j) of the 256 x 256 Gram, as a batch of pairs
        w = inputs.gram_256()
        lam = w["dyadic_order"]
        nb = batch if 0 < batch < 256 else 256
        X32, X64 = inputs.f32(w["X"][:nb])
        Y32, Y64 = inputs.f32(w["Y"][:nb])
        L, d = X32.shape[1], X32.shape[2]
        B = nb * nb
        Xd = torch.from_numpy(X32).cuda().repeat_interleave(nb, 0).contiguous()
        Yd = torch.from_numpy(Y32).cuda().repeat(nb, 1, 1).contiguous()
        n = (L - 1) << lam
        cells = B * n * n
        coarse = B * (L - 1) * (L - 1)

        def step():
            return sigk.pairs_surface(Xd, Yd, lam)[1]

        hx, hy = Xd.cpu().pin_memory(), Yd.cpu().pin_memory()
        hs = torch.empty(B, L, L).pin_memory()

        def host_step(hx, hy, hs):
            _, sf = sigk.pairs_surface(hx.cuda(non_blocking=True), hy.cuda(non_blocking=True), lam)
            hs.copy_(sf, non_blocking=True)

        def oracle_rate(budget):
            t0 = time.perf_counter(); done = 0
            while time.perf_counter() - t0 < budget and done < nb:
                oracle.pairs_surface(np.repeat(X64[done:done + 1], nb, 0), Y64, lam)
                done += 1
            return done * nb * n * n / (time.perf_counter() - t0), "%d x %d pairs" % (done, nb), \
                oracle.num_threads()

        def parity(out):
            rng = np.random.default_rng(8)
            s = out.cpu().numpy()
            errs = []
            for t in rng.choice(B, 6, replace=False):
                i, j = divmod(int(t), nb)
                ref = oracle.surface(X64[i], Y64[j], lam)
                errs.append(float(np.max(np.abs(s[t] - ref) / np.maximum(np.abs(ref), 1e-3))))
            return max(errs), "6 sampled pairs, every node"
        return dict(
            desc="%d pairs (X_i, Y_j) of the 256x256 Gram inputs, L=M=128, d=8, dyadic order 2, fp32: "
                 "the solution surface on the sample grid (%d x %d nodes per pair, %.2f GB written)"
                 % (B, L, L, B * L * L * 4 / 1e9),
            dtype="f32", step=step, cells=cells, pairs=B, flop=3 * cells + 2 * d * coarse,
            kernels="chain_f32_kernel (surface instance, inline coefficients) + band_gbar_kernel (surface unpack)",
            oracle_rate=oracle_rate, parity=parity, host_step=host_step, host=(hx, hy, hs),
            h2d=hx.numel() * 4 + hy.numel() * 4, d2h=B * L * L * 4)

    if name == "support_fbm30":
        # the support-reduction example of Sec. 5.3: 30 fBM paths (Hurst
        # exponents from {0.2, 0.5, 0.8}), their signature-kernel Gram, then
        # proximal gradient descent on the weights; one step = the Gram + 2000
        # iterations
        X, H = inputs.fbm_paths()
        X[:, :, 1] *= 0.5 / np.abs(X[:, :, 1]).max()
        X32, X64 = inputs.f32(X)
        lam_d, iters, pen = 3, 2000, 0.5
        n, L = X32.shape[0], X32.shape[1]
        Xd = torch.from_numpy(X32).cuda()
        K0 = sigk.gram(Xd, Xd, lam_d)
        gamma = float(0.5 / np.abs(np.linalg.eigvalsh(K0.double().cpu().numpy())).max())
        a = torch.full((n,), 1.0 / n, device="cuda")
        b0 = torch.zeros(n, device="cuda")
        cells = n * n * ((L - 1) << lam_d) ** 2

        def step():
            K = sigk.gram(Xd, Xd, lam_d)
            return sigk.support_reduction(K, a, b0, gamma, pen, iters)[0]

        def host_step(hx, hb):
            xd = hx.cuda(non_blocking=True)
            K = sigk.gram(xd, xd, lam_d)
            hb.copy_(sigk.support_reduction(K, a, b0, gamma, pen, iters)[0], non_blocking=True)

        def oracle_rate(budget):
            t0 = time.perf_counter()
            K = oracle.gram(X64, X64, lam_d)
            oracle.support_reduction(K, np.full(n, 1.0 / n), np.zeros(n), gamma, pen, iters)
            return cells / (time.perf_counter() - t0), "the whole step (Gram + %d iterations)" % iters, \
                oracle.num_threads()

        def parity(out):
            K = oracle.gram(X64, X64, lam_d)
            rb, _ = oracle.support_reduction(K, np.full(n, 1.0 / n), np.zeros(n), gamma, pen, iters)
            o = out.double().cpu().numpy()
            return float(np.max(np.abs(o - rb)) / np.max(np.abs(rb))), "beta after %d iterations" % iters
        return dict(
            desc="support reduction (Sec. 5.3): 30 fBM paths, L=%d, d=2, Gram at dyadic order %d, then %d "
                 "proximal gradient steps (lam = %g), fp32" % (L, lam_d, iters, pen),
            dtype="f32", step=step, cells=cells, pairs=n * n, flop=3 * cells,
            kernels="chain_f32_kernel + support_kernel", oracle_rate=oracle_rate, parity=parity,
            host_step=host_step, host=(torch.from_numpy(X32).pin_memory(), torch.empty(n).pin_memory()),
            h2d=X32.nbytes, d2h=n * 4)
    raise SystemExit("unknown workload " + name)


def _uneven_kernels(sched):
    from paper_2006_14794_gb300 import sigk
    if sched.rec == sigk.REC_CHAIN:
        return ("vstack_kernel (one launch per stack height; coefficients formed in the sweep) + "
                "vs_inc_kernel (increments) + vs_pairs_kernel + vs_plan_kernel (device planning)")
    if sched.rec == sigk.REC_BAND:
        return ("vband_sweep_kernel (one launch per band class) + vb_coef_kernel (FMA contraction into "
                "the band) + vb_pairs_kernel + vb_plan_kernel (device planning)")
    return ("plan_kernel + inc_kernel + coef_kernel (FMA contraction) + strip_kernel<float> "
            "(strip path, %s-row strips)" % (32 * sched.rows_per_lane if sched.rows_per_lane else "default"))


def _peak(dtype, sms):
    if dtype == "f64":
        return FP64_PEAK_NOMINAL_TF, "nominal dense FP64 of the GB300 (no measured FP64 figure)"
    tf, mhz, src = fp32_peak_tflops(sms)
    return tf, "%d SMs x 128 FP32 lanes x 2 flop x %.0f MHz (%s max SM clock)" % (sms, mhz, src)


def measure_workload(name, args, cache=None, with_e2e=False, with_clocks=True):
    """Times one workload as described above; returns its result dict."""
    import torch
    wl = _workload(name, args.batch, cache)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    for _ in range(max(args.warmup, 3)):
        wl["step"]()
    torch.cuda.synchronize()
    steps = max(args.wl_steps, 5)
    st = torch.cuda.current_stream()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    clocks = ClockSampler(0) if with_clocks else None
    if clocks:
        clocks.start()
        time.sleep(0.3)
    out = None
    for i in range(steps):
        flush.fill_(float(i))
        ev[i][0].record(st)
        out = wl["step"]()
        ev[i][1].record(st)
    torch.cuda.synchronize()
    clk = clocks.stop() if clocks else None
    ms = sum(a.elapsed_time(b) for a, b in ev) / steps
    rel, rel_sample = wl["parity"](out)
    props = torch.cuda.get_device_properties(0)
    peak_tf, peak_src = _peak(wl["dtype"], props.multi_processor_count)
    ach = wl["flop"] / (ms * 1e-3) / 1e12
    if args.skip_cpu:
        cpu = {"value": None, "unit": "cells/s", "cores": 0, "kind": "oracle", "sample": "skipped (--skip-cpu)"}
    else:
        rate, sample, cores = wl["oracle_rate"](args.wl_cpu_seconds)
        cpu = {"value": rate, "unit": "cells/s", "cores": cores, "kind": "oracle", "sample": sample}
    res = {
        "config": wl["desc"], "dtype": wl["dtype"], "steps": steps, "ms_per_step": ms,
        "cells_per_s": wl["cells"] / (ms * 1e-3), "pairs_per_s": wl["pairs"] / (ms * 1e-3),
        "cells_per_step": wl["cells"], "pairs_per_step": wl["pairs"],
        "rel_err_vs_oracle": {"max": rel, "sample": rel_sample},
        "roofline": {"bound": "alu", "work_flop_per_step": wl["flop"], "achieved": ach, "peak": peak_tf,
                     "unit": "TFLOP/s", "frac": ach / peak_tf, "peak_source": peak_src,
                     "kernels": wl["kernels"],
                     "note": "whole call (all of its kernels) over CUDA events"},
        "clocks": clk, "cpu_baseline": cpu,
    }
    if with_e2e:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(steps):
            wl["host_step"](*wl["host"])
        e1.record(st)
        torch.cuda.synchronize()
        e2e_ms = e0.elapsed_time(e1) / steps
        res["e2e"] = {"value": wl["cells"] / (e2e_ms * 1e-3), "unit": "cells/s",
                      "h2d_bytes_per_step": int(wl["h2d"]), "d2h_bytes_per_step": int(wl["d2h"]),
                      "ms_per_step": e2e_ms}
    del flush
    torch.cuda.empty_cache()
    return res


# the configurations of the workload statement besides the headline Gram
# (configs 1, 3, 4, 5; config 5 in FP32 and FP64 at both dyadic orders, and
# its backward at dyadic order 1)
DEFAULT_WORKLOADS = ["gram_small_f64", "gram_small_f32", "uneven4096", "mmd128", "mmd128_rbf", "long64_l0",
                     "long64_l1", "long64_l0_f64", "long64_l1_f64", "long64_l1_grad"]


def run_workloads(args):
    cache = {}
    res = {}
    for name in DEFAULT_WORKLOADS:
        try:
            res[name] = measure_workload(name, args, cache)
        except Exception as e:   # one broken workload must not hide the others
            res[name] = {"error": "%s: %s" % (type(e).__name__, e)}
    return res


def run_extra(args):
    import torch
    torch.cuda.set_device(0)
    from paper_2006_14794_gb300 import sigk
    sigk.lib()
    r = measure_workload(args.workload, args, with_e2e=True)
    import oracle  # noqa: F401
    line = {
        "metric": METRIC, "value": r["cells_per_s"], "unit": "cells/s", "n_gpus": 1,
        "steps": r["steps"], "warmup": args.warmup, "ms_per_step": r["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": r["dtype"],
        "data": "synthetic",
        "config": {"workload": r["config"], "l2": "flushed (256 MB write) before each step"},
        "pairs_per_s": r["pairs_per_s"],
        "roofline": r["roofline"], "clocks": r["clocks"], "e2e": r["e2e"],
        "cpu_baseline": r["cpu_baseline"], "rel_err_vs_oracle": r["rel_err_vs_oracle"],
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--skip-fp64", action="store_true")
    ap.add_argument("--skip-workloads", action="store_true",
                    help="the headline line only (no 'workloads' key)")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--wl-steps", type=int, default=5, help="timed steps per workload (>= 5)")
    ap.add_argument("--wl-cpu-seconds", type=float, default=3.0,
                    help="oracle time budget per workload where the sample is time-bounded")
    ap.add_argument("--batch", type=int, default=0,
                    help="uneven4096 / long64 / mmd128 / gram256_*: only the first BATCH pairs / paths per batch "
                         "(profiling)")
    ap.add_argument("--workload", default="gram256",
                    choices=["gram256"] + DEFAULT_WORKLOADS + ["gram256_implicit", "gram256_rbf",
                                                               "surface256", "support_fbm30"])
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.workload != "gram256":
        return run_extra(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
