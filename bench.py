#!/usr/bin/env python
"""Benchmark of the tensor-train contraction library on GB300.

Workload (one "step"): the order-10 TT pair with mode sizes 16 and internal
ranks 64 in float32 (seeded Gaussian cores, sigma = 1/sqrt(I R)); one full
contraction <X, Y> and one partial contraction over modes 1-6 (chain layout).
Metric: contractions per second (2 per step), with GFLOP/s and the roofline
fraction of the dominant kernel (the environment sweep).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun every rank runs its own replica of the pair (the path has no
exchange step: replicas only); rank 0 prints one JSON line.  The reference arm
times the float64 CPU oracle on the host cores.
"""
from __future__ import annotations

import os

os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
os.environ.setdefault("OMP_NUM_THREADS", "1")

import argparse  # noqa: E402
import json  # noqa: E402
import math  # noqa: E402
import statistics  # noqa: E402
import subprocess  # noqa: E402
import tempfile  # noqa: E402
import sys  # noqa: E402
import time  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_2109_00626_gb300 import inputs as G  # noqa: E402
from paper_2109_00626_gb300 import workload as W  # noqa: E402

# DRAM bytes read + written by one launch of sweep_two_sided_kernel<float,64> on
# this workload (ncu dram__bytes_read.sum + dram__bytes_write.sum, cold L2; the
# capture is in profiles/launches_order10_r64_step.md).  Reset to None whenever
# that kernel or the sweep body changes.
TWO_SIDED_TRAFFIC = 4299776

METRIC = "TT contractions/s (order-10, I=16, R=64, fp32: full + partial over modes 1-6)"
UNIT = "contractions/s"
MASK = [1] * 6 + [0] * 4
WORKLOAD = "order-10 TT pair, modes 16, internal ranks 64, float32; full contraction + partial contraction over modes 1-6 (chain layout)"


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def fp32_simt_peak_tflops():
    """152 SMs x 128 FP32 lanes x 2 flop (FMA) x 2.07 GHz maximum SM clock."""
    sm_mhz = _peaks().get("sm_max_mhz", 2070.0)
    return 152 * 128 * 2 * sm_mhz * 1e6 / 1e12


def measure_peaks():
    """Reference peaks beside the measured HBM copy and bf16 GEMM: cuBLAS SGEMM with TF32 off
    (the float32 FMA pipe) and DGEMM, square n x n, timed with CUDA events
    after warm-up; one JSON line.  Context for the float32 roofline, whose
    denominator stays the derived FMA peak."""
    import torch

    dev = torch.device("cuda", 0)
    torch.backends.cuda.matmul.allow_tf32 = False
    out = {"derived_fp32_fma_tflops": fp32_simt_peak_tflops()}
    for name, dt, n, reps in (("sgemm", torch.float32, 8192, 20), ("dgemm", torch.float64, 4096, 5)):
        a = torch.randn(n, n, dtype=dt, device=dev)
        b = torch.randn(n, n, dtype=dt, device=dev)
        c = torch.empty(n, n, dtype=dt, device=dev)
        for _ in range(3):
            torch.mm(a, b, out=c)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        sampler = ClockSampler(0)
        sampler.start()
        e0.record()
        for _ in range(reps):
            torch.mm(a, b, out=c)
        e1.record()
        torch.cuda.synchronize(dev)
        clocks = sampler.stop()
        ms = e0.elapsed_time(e1) / reps
        out[name + "_tflops"] = 2.0 * n**3 / (ms / 1e3) / 1e12
        out[name + "_n"] = n
        out[name + "_clocks"] = clocks
    print(json.dumps(out))
    return 0


def work_per_step():
    modes = [16] * 10
    r = G.tt_ranks(10, 64)
    f_full = W.full_flops(modes, r, r)
    f_part = W.partial_chain_flops(modes, r, r, MASK)
    b_full = W.full_bytes(modes, r, r, 4)
    b_part = W.partial_chain_bytes(modes, r, r, MASK, 4)
    return f_full, f_part, b_full, b_part


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms."""

    Q = (
        "index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
        "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
        "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap"
    )

    def __init__(self, gpu_index=0):
        self.proc = None
        self.lines = []
        self.gpu = gpu_index

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE,
                stderr=subprocess.DEVNULL,
                text=True,
            )
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out = ""
        rows = []
        for ln in out.strip().splitlines():
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append(
                    {
                        "sm": float(parts[1]),
                        "max": float(parts[2]),
                        "hw": parts[5],
                        "hwt": parts[6],
                        "swt": parts[7],
                        "pcap": parts[8],
                    }
                )
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        reasons = set()
        for r in rows:
            if r["hw"] == "Active":
                reasons.add("hw_slowdown")
            if r["hwt"] == "Active":
                reasons.add("hw_thermal_slowdown")
            if r["swt"] == "Active":
                reasons.add("sw_thermal_slowdown")
            if r["pcap"] == "Active":
                reasons.add("sw_power_cap")
        return {
            "sm_mhz": statistics.median(r["sm"] for r in rows),
            "sm_max_mhz": max(r["max"] for r in rows),
            "reasons": sorted(reasons),
            "samples": len(rows),
        }


def _oracle_pair_seconds(p):
    """Worker of the batched CPU baseline: host time of the float64 oracle on
    pair p of the uneven batch (its cores drawn on the host from the pair's
    seed; drawing is not timed)."""
    import oracle as O

    spec, x, y = G.batch_pair(p, 0, np.float64)
    t0 = time.perf_counter()
    if spec["kind"] == "full":
        O.contract_full(x, y)
    else:
        O.partial_chain(x, y, spec["mask"])
    return time.perf_counter() - t0


def cpu_baseline_batched(stride=2, n_pairs=4096):
    """The float64 oracle over every `stride`-th pair of the 4096-pair batch,
    the pairs spread over every host core by a process pool (spawned: the
    calling process already holds a CUDA context).  The rate for the whole
    batch is the sample's wall time scaled by the batch's flops over the
    sample's (the flop model of the benchmark)."""
    import multiprocessing as mp

    specs = G.batch4096_spec(n_pairs, 0)

    def flops_of(sp):
        if sp["kind"] == "full":
            return W.full_flops(sp["modes"], sp["ranks_x"], sp["ranks_y"])
        return W.partial_chain_flops(sp["modes"], sp["ranks_x"], sp["ranks_y"], sp["mask"])

    sample = list(range(0, n_pairs, stride))
    f_all = sum(flops_of(sp) for sp in specs)
    f_sample = sum(flops_of(specs[p]) for p in sample)
    cores = os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        pool.map(_oracle_pair_seconds, sample[: 2 * cores])  # workers started and warm
        t0 = time.perf_counter()
        per_pair = pool.map(_oracle_pair_seconds, sample, chunksize=1)
        wall = time.perf_counter() - t0
    batch_s = wall * f_all / f_sample
    return {
        "value": n_pairs / batch_s,
        "unit": "contractions/s",
        "cores": cores,
        "kind": "oracle",
        "sample": f"every {stride}th pair ({len(sample)} of {n_pairs}, {f_sample / f_all:.1%} of the batch's flops) in {wall:.1f} s wall on {cores} host processes (one thread each); {sum(per_pair):.1f} s of oracle time; rate scaled to the whole batch by flops",
    }


def cpu_baseline(seconds=10.0):
    """The float64 oracle, as it stands, on the same pair (one host thread)."""
    import oracle as O

    x, y = G.order10_r64(0, np.float64)
    t0 = time.perf_counter()
    n = 0
    while True:
        O.contract_full(x, y)
        O.partial_chain(x, y, MASK)
        n += 1
        if time.perf_counter() - t0 >= seconds:
            break
    dt = time.perf_counter() - t0
    return {
        "value": 2 * n / dt,
        "unit": UNIT,
        "cores": 1,
        "kind": "oracle",
        "sample": f"{n} steps (full + partial over modes 1-6 of the same order-10 pair) in {dt:.1f} s, numpy float64, OPENBLAS_NUM_THREADS=1",
    }


def accuracy(x32, y32, z_gpu, zc_gpu):
    """Part of the CPU-baseline leg: errors of the headline step's GPU results
    against the float64 oracle on the same float32 cores.  Full contraction:
    eps = |z - z*| / (||X|| ||Y||) (norms from the oracle's <X,X>, <Y,Y>), the
    plain relative error and kappa = ||X|| ||Y|| / |z*|.  Partial contraction:
    the joined core C's largest error relative to its largest entry, and
    whether the copied cores are bit-exact."""
    import oracle as O

    x = [np.asarray(c, dtype=np.float64) for c in x32]
    y = [np.asarray(c, dtype=np.float64) for c in y32]
    z_star = O.contract_full(x, y)
    nrm = math.sqrt(O.contract_full(x, x) * O.contract_full(y, y))
    want, _ = O.partial_chain(x, y, MASK)
    _, s = O.end_block(MASK)
    c_at = len(x) - s - 1  # position of the joined core C in the chain (leading block)
    got = [np.asarray(g, dtype=np.float64).reshape(w.shape) for g, w in zip(zc_gpu, want)]
    c_err = float(np.abs(got[c_at] - want[c_at]).max() / np.abs(want[c_at]).max())
    copies_exact = all(np.array_equal(g, w) for p, (g, w) in enumerate(zip(got, want)) if p != c_at)

    def fin(v):
        return float(v) if math.isfinite(v) else None

    return {
        "reference": "float64 oracle on the same float32 cores",
        "full_eps": fin(abs(z_gpu - z_star) / nrm),
        "full_rel": fin(abs(z_gpu - z_star) / abs(z_star)),
        "kappa": fin(nrm / abs(z_star)),
        "partial_c_rel": fin(c_err),
        "partial_copies_exact": bool(copies_exact),
        "bound_eps": 1e-5,
    }


def tc_accuracy(results):
    """Part of the CPU-baseline leg: each tensor-core form's z (mantissa,
    exponent) against the float64 oracle on the order-16 rank-256 pair, as
    eps = |z - z*| / (||X|| ||Y||) on the float32 cores (end to end) and, for
    the bfloat16 form, on the bfloat16-rounded cores it reads (arithmetic
    error); with kappa and the bound the tests hold each form to (the
    rounding-error model's 8 sigma plus twice its coherent bias, relative to
    |z*| of the cores the form reads)."""
    import oracle as O
    import torch
    from oracle import error_model as M

    x, y = G.order16_r256(0)
    x64 = [c.astype(np.float64) for c in x]
    y64 = [c.astype(np.float64) for c in y]
    z32 = O.contract_full(x64, y64)
    nrm = math.sqrt(O.contract_full(x64, x64) * O.contract_full(y64, y64))

    def fin(v):
        return float(v) if math.isfinite(v) else None

    out = {}
    for prec, (m, e) in results.items():
        z = math.ldexp(m, e)
        rep = {
            "reference": "float64 oracle",
            "eps_vs_fp32_cores": fin(abs(z - z32) / nrm),
            "rel_vs_fp32_cores": fin(abs(z - z32) / abs(z32)),
            "kappa": fin(nrm / abs(z32)),
        }
        if prec == "native":
            xb = [torch.from_numpy(c).bfloat16().double().numpy() for c in x]
            yb = [torch.from_numpy(c).bfloat16().double().numpy() for c in y]
            z16 = O.contract_full(xb, yb)
            rep["eps_vs_bf16_cores"] = fin(abs(z - z16) / nrm)
            rep["rel_vs_bf16_cores"] = fin(abs(z - z16) / abs(z16))
            rep["bound_rel"] = fin(M.tc_bound(xb, yb, "bf16", z16) / abs(z16))
        else:
            rep["bound_rel"] = fin(M.tc_bound(x64, y64, "bf16x3", z32) / abs(z32))
        out[prec] = rep
    return out


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def step_config(world):
    """The `config` of both arms' JSON lines (same keys and values)."""
    return {
        "workload": WORKLOAD,
        "seed": 0,
        "l2": "flushed between timed steps (256 MiB write)",
        "parallelism": "replicas" if world > 1 else "none",
    }


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import oracle as O

    x, y = G.order10_r64(0, np.float64)
    for _ in range(args.warmup):
        O.contract_full(x, y)
        O.partial_chain(x, y, MASK)
    # the host caches are flushed between timed steps too (a 256 MiB write),
    # outside the timed region
    flush = np.empty(256 << 20, dtype=np.uint8)
    dt = 0.0
    for _ in range(args.steps):
        flush.fill(1)
        t0 = time.perf_counter()
        O.contract_full(x, y)
        O.partial_chain(x, y, MASK)
        dt += time.perf_counter() - t0
    val = 2 * args.steps / dt
    line = {
        "impl": "reference",
        "metric": METRIC,
        "value": val,
        "unit": UNIT,
        "n_gpus": args.gpus,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": step_config(world),
        "cpu_baseline": {
            "value": val,
            "unit": UNIT,
            "cores": 1,
            "kind": "oracle",
            "sample": f"{args.steps} steps of the full workload, numpy float64 oracle, one host thread on rank 0 (host caches flushed between steps)",
        },
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def arena(shapes, dtype, device, pin=False):
    """One buffer holding tensors of the given shapes back to back, each view
    starting on a 16-byte boundary; returns (buffer, views)."""
    import torch

    esize = torch.tensor([], dtype=dtype).element_size()
    align = max(1, 16 // esize)
    offs, n = [], 0
    for sh in shapes:
        offs.append(n)
        n += (int(np.prod(sh)) + align - 1) // align * align
    buf = torch.zeros(max(n, 1), dtype=dtype, device=device)
    if pin:
        buf = buf.pin_memory()
    views = [buf[o : o + int(np.prod(sh))].view(*sh) for o, sh in zip(offs, shapes)]
    return buf, views


def run_ours(args):
    import torch

    import paper_2109_00626_gb300 as T

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)

    x, y = G.order10_r64(0, np.float32)
    # every input core in one device arena (and a pinned host mirror), every
    # output core of the partial contraction in another: the end-to-end step
    # moves its inputs with one host-to-device copy and its results with two
    # device-to-host copies
    din, xyd = arena([c.shape for c in x + y], torch.float32, dev)
    hin, xyh = arena([c.shape for c in x + y], torch.float32, "cpu", pin=True)
    for d, h, c in zip(xyd, xyh, x + y):
        h.copy_(torch.from_numpy(c))
        d.copy_(h)
    xd, yd = xyd[: len(x)], xyd[len(x) :]
    zm, zr, _ = T.partial_shape(T.Desc(xd), T.Desc(yd), MASK)
    zshapes = [(zr[t], zm[t], zr[t + 1]) for t in range(len(zm))]
    dz, zd = arena(zshapes, torch.float32, dev)
    full = T.FullContraction(xd, yd)
    part = T.PartialContraction(xd, yd, MASK, out=zd)
    stream = torch.cuda.current_stream(dev)
    side = torch.cuda.Stream(dev)  # the full and the partial contraction are independent: run them side by side
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def step(evs=None, fc=full, pc=part):
        fork = torch.cuda.Event()
        fork.record(stream)
        side.wait_event(fork)
        if evs is not None:
            evs[0].record(side)
        fc(side)
        if evs is not None:
            evs[1].record(side)
        pc(stream)
        join = torch.cuda.Event()
        join.record(side)
        stream.wait_event(join)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)

    K = args.steps
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(K)]
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    l0 = T.launch_count()
    for k in range(K):
        flush.fill_(float(k))  # L2 flush between timed steps (256 MiB write, untimed)
        ev[k][0].record(stream)
        step(ev[k][2:4])
        ev[k][1].record(stream)
    torch.cuda.synchronize(dev)
    launches = T.launch_count() - l0
    if world > 1:
        torch.distributed.barrier()
    clocks = sampler.stop()
    t_step = [ev[k][0].elapsed_time(ev[k][1]) for k in range(K)]
    t_full = [ev[k][2].elapsed_time(ev[k][3]) for k in range(K)]
    tot_ms = sum(t_step)
    if world > 1:
        t = torch.tensor([tot_ms], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        tot_ms = float(t.item())
    ms = tot_ms / K
    value = 2 * K * world / (tot_ms / 1e3)

    f_full, f_part, b_full, b_part = work_per_step()
    full_ms = statistics.mean(t_full)
    achieved = f_full / (full_ms / 1e3) / 1e12
    peak = fp32_simt_peak_tflops()

    # end to end through the C ABI with host buffers, every step: H2D of every
    # core (one copy of the input arena), both contractions, D2H of z and of
    # the partial result's cores (one copy of the output arena).  Two sets of
    # arenas alternate, so step k+1's upload and step k-1's download run on
    # copy streams while step k computes.
    hz = [arena(zshapes, torch.float32, "cpu", pin=True)[0] for _ in range(2)]
    outh = [torch.empty(1, dtype=torch.float64).pin_memory() for _ in range(2)]
    din2, xyd2 = arena([c.shape for c in x + y], torch.float32, dev)
    din2.copy_(din)
    dz2, zd2 = arena(zshapes, torch.float32, dev)
    full2 = T.FullContraction(xyd2[: len(x)], xyd2[len(x) :])
    part2 = T.PartialContraction(xyd2[: len(x)], xyd2[len(x) :], MASK, out=zd2)
    sets = [(din, dz, full, part), (din2, dz2, full2, part2)]
    h2d = hin.numel() * 4
    d2h = 8 + hz[0].numel() * 4
    cin, cout = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    ev_in = [torch.cuda.Event() for _ in range(2)]
    ev_done = [torch.cuda.Event() for _ in range(2)]
    ev_out = [torch.cuda.Event() for _ in range(2)]
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    K2 = max(2, K // 2)
    torch.cuda.synchronize(dev)
    e0.record(cin)
    for k in range(K2):
        j = k & 1
        d_in, d_z, fc, pc = sets[j]
        cin.wait_event(ev_done[j])  # step k-2 has finished reading this input arena
        with torch.cuda.stream(cin):
            d_in.copy_(hin, non_blocking=True)
        ev_in[j].record(cin)
        stream.wait_event(ev_in[j])
        stream.wait_event(ev_out[j])  # step k-2's results have left this output arena
        step(fc=fc, pc=pc)
        ev_done[j].record(stream)
        cout.wait_event(ev_done[j])
        with torch.cuda.stream(cout):
            outh[j].copy_(fc.out, non_blocking=True)
            hz[j].copy_(d_z, non_blocking=True)
        ev_out[j].record(cout)
    e1.record(cout)
    torch.cuda.synchronize(dev)
    e2e_ms = e0.elapsed_time(e1) / K2
    # the same, one step at a time on one stream (no overlap of copies and work)
    torch.cuda.synchronize(dev)
    e0.record(stream)
    for _ in range(K2):
        din.copy_(hin, non_blocking=True)
        step()
        outh[0].copy_(full.out, non_blocking=True)
        hz[0].copy_(dz, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    serial_ms = e0.elapsed_time(e1) / K2

    status = int(full.status.item()) | int(part.status.item()) | int(full2.status.item()) | int(part2.status.item())
    forms = {}
    if not args.no_forms:
        runners = {
            "tf32x3": lambda: bench_step_prec(T, dev, args, "tf32x3"),
            "tf32": lambda: bench_step_prec(T, dev, args, "tf32"),
            "batched": lambda: bench_batched(T, dev, args),
            "bf16": lambda: bench_bf16(T, dev, args, "native"),
            "bf16x3": lambda: bench_bf16(T, dev, args, "bf16x3"),
            "backward": lambda: bench_backward(T, dev, args),
            "merged": lambda: bench_merged(T, dev, args),
            "dense_ttcp": lambda: bench_dense_ttcp(T, dev, args),
            "factored": lambda: bench_factored(T, dev, args),
            "random_sets": lambda: bench_random_sets(T, dev, args),
            "round": lambda: bench_round(T, dev, args),
        }
        wanted = list(runners) if args.forms == "all" else [f for f in args.forms.split(",") if f]
        for name in wanted:
            forms[name] = runners[name]()

    if rank == 0:
        line = {
            "metric": METRIC,
            "value": value,
            "unit": UNIT,
            "n_gpus": world,
            "steps": K,
            "warmup": args.warmup,
            "ms_per_step": ms,
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "f32",
            "data": "synthetic",
            "config": step_config(world),
            "gflops": (f_full + f_part) / (ms / 1e3) / 1e9,
            "roofline": {
                "kernel": "sweep_two_sided_kernel<float,64> (full contraction, two clusters from both ends)",
                "bound": "alu",
                "achieved": achieved,
                "peak": peak,
                "unit": "TFLOP/s",
                "frac": achieved / peak,
                "traffic": TWO_SIDED_TRAFFIC,
                "note": "fp32 FMA peak = 152 SMs x 128 lanes x 2 x 2.07 GHz (derived); single latency-bound contraction; traffic = ncu dram bytes read+write of one launch of this kernel (cold L2) against %d bytes of cores, null while the kernel has changed since the last capture" % (b_full,),
            },
            "e2e": {
                "value": 2 / (e2e_ms / 1e3) * world,
                "unit": UNIT,
                "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h,
                "serial_value": 2 / (serial_ms / 1e3) * world,
                "note": "every step uploads all cores (one pinned-arena copy) and downloads z and the partial "
                "result (one arena copy); two buffer sets alternate so copies of neighbouring steps overlap "
                "the contractions on copy streams; serial_value: the same steps one at a time on one stream",
            },
            "gpu_launches": launches,
            "clocks": clocks,
            "device_status": status,
            "forms": forms,
        }
        if not args.no_cpu_baseline and world == 1:
            line["cpu_baseline"] = cpu_baseline(args.cpu_seconds)
            try:
                line["accuracy"] = accuracy(x, y, float(full.out.item()), [c.detach().cpu().numpy() for c in part.z])
            except Exception as e:  # a report, never a reason to lose the measurement line
                line["accuracy"] = {"error": repr(e)[:200]}
            if _TC_RESULTS:
                try:
                    for prec, rep in tc_accuracy(_TC_RESULTS).items():
                        forms["bf16" if prec == "native" else prec]["accuracy"] = rep
                except Exception as e:
                    forms["bf16"]["accuracy"] = {"error": repr(e)[:200]}
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def tf32_peak_tflops():
    """Dense tf32 tensor peak: the measured bf16 burst peak times the nominal
    tf32 / bf16 ratio of the part (1.1 / 2.25 PFLOP/s dense)."""
    return _bf16_peak()[0] * 1.1 / 2.25


def tf32_issued_flops(x, y, mask=None):
    """Tensor-core flops the tf32x3 sweep issues for a full contraction (mask
    None: every mode but the last) or a chain partial one (the contracted
    modes and the boundary core): per slice, GEMM 1 and GEMM 2 of 128 x 64 x
    (8 ceil(K / 8)) in two passes."""
    n = len(x)
    if mask is None:
        modes = list(range(n - 1))
        extra = []
    else:
        side, s = W.end_block(mask)
        modes = list(range(s)) if side == "lead" else list(range(n - s, n))
        extra = [s if side == "lead" else n - s - 1]
    tot = 0
    for k in modes:
        i_dim = x[k].shape[1]
        k1 = -(-y[k].shape[0] // 8)
        k2 = -(-x[k].shape[0] // 8)
        tot += i_dim * 2 * 2 * 128 * 64 * 8 * (k1 + k2)
    for k in extra:
        tot += x[k].shape[1] * 2 * 2 * 128 * 64 * 8 * -(-x[k].shape[0] // 8)
    return tot


def bench_step_prec(T, dev, args, prec):
    """The headline step (full and partial contraction of the order-10 pair,
    side by side on two streams, L2 flushed between steps) with the products
    of `prec` on the tensor cores; CUDA events on the launching streams; the
    full contraction's launch timed alone for its roofline; accuracy against
    the float64 oracle on the same float32 cores."""
    import torch

    import oracle as O

    x, y = G.order10_r64(0, np.float32)
    xd = [torch.from_numpy(c).to(dev) for c in x]
    yd = [torch.from_numpy(c).to(dev) for c in y]
    full = T.FullContraction(xd, yd, prec=prec)
    part = T.PartialContraction(xd, yd, MASK, prec=prec)
    stream = torch.cuda.current_stream(dev)
    side = torch.cuda.Stream(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def step(evs=None):
        fork = torch.cuda.Event()
        fork.record(stream)
        side.wait_event(fork)
        if evs is not None:
            evs[0].record(side)
        full(side)
        if evs is not None:
            evs[1].record(side)
        part(stream)
        join = torch.cuda.Event()
        join.record(side)
        stream.wait_event(join)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize(dev)
    K = args.steps
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(K)]
    for k in range(K):
        flush.fill_(float(k))
        ev[k][0].record(stream)
        step(ev[k][2:4])
        ev[k][1].record(stream)
    torch.cuda.synchronize(dev)
    ms = statistics.mean(ev[k][0].elapsed_time(ev[k][1]) for k in range(K))
    full_ms = statistics.mean(ev[k][2].elapsed_time(ev[k][3]) for k in range(K))
    f_full, f_part, _, _ = work_per_step()
    issued = tf32_issued_flops(x, y)
    peak = tf32_peak_tflops()
    out = {
        "workload": WORKLOAD + "; products on the tensor cores (" + prec + ")",
        "value": 2 / (ms / 1e3),
        "unit": UNIT,
        "ms_per_step": ms,
        "ms_full": full_ms,
        "gflops": (f_full + f_part) / (ms / 1e3) / 1e9,
        "roofline": {
            "kernel": "tf_two_sided_kernel<%s> (full contraction, two clusters from both ends)"
                      % ("true" if prec == "tf32x3" else "false"),
            "bound": "tensor",
            "achieved": issued / (full_ms / 1e3) / 1e12,
            "peak": peak,
            "unit": "TFLOP/s",
            "frac": issued / (full_ms / 1e3) / 1e12 / peak,
            "note": "tensor flops issued (128 x 64 tiles, hi and lo stacked, two passes) per launch over its CUDA-event "
                    "time; peak = measured bf16 burst x 1.1 / 2.25 (nominal dense tf32 / bf16); latency-bound single "
                    "contraction",
        },
        "device_status": int(full.status.item()) | int(part.status.item()),
        "l2": "flushed between timed steps (256 MiB write)",
    }
    if not args.no_cpu_baseline:
        try:
            x64 = [c.astype(np.float64) for c in x]
            y64 = [c.astype(np.float64) for c in y]
            z = float(full.out.item())
            zs = O.contract_full(x64, y64)
            nrm = math.sqrt(O.contract_full(x64, x64) * O.contract_full(y64, y64))
            zc, _ = O.partial_chain(x64, y64, MASK)
            got = [c.detach().cpu().double().numpy() for c in part.z]
            c_rel = max(float(np.abs(g - w).max() / np.abs(w).max()) for g, w in zip(got, zc))
            out["accuracy"] = {
                "reference": "float64 oracle on the same float32 cores",
                "full_eps": abs(z - zs) / nrm,
                "full_rel": abs(z - zs) / abs(zs),
                "kappa": nrm / abs(zs),
                "partial_core_rel": c_rel,
                "bound_eps": 1e-5,
            }
        except Exception as e:  # a report, never a reason to lose the measurement line
            out["accuracy"] = {"error": repr(e)[:200]}
        if "order10_step" not in _ORACLE_TIMES:
            def oracle_step():
                O.contract_full(x, y)
                O.partial_chain(x, y, MASK)

            t = _oracle_once(oracle_step, "contractions/s", "one step (full + partial over modes 1-6), numpy float64")
            t["value"] *= 2  # two contractions a step, as the form's value counts them
            _ORACLE_TIMES["order10_step"] = t
        out["cpu_baseline"] = _ORACLE_TIMES["order10_step"]
    return out


def bench_batched(T, dev, args):
    """4096 uneven pairs in one graph-captured persistent launch (inputs 15 GB,
    larger than L2: no flush needed)."""
    import torch

    from paper_2109_00626_gb300 import shard as S

    rank, world, _ = dist_env()
    t0 = time.perf_counter()
    specs_all = G.batch4096_spec(4096, 0)
    flops = 0
    nbytes = 0
    costs = []
    for sp in specs_all:
        m, rx, ry = sp["modes"], sp["ranks_x"], sp["ranks_y"]
        if sp["kind"] == "full":
            f = W.full_flops(m, rx, ry)
            nbytes += W.full_bytes(m, rx, ry, 4)
        else:
            f = W.partial_chain_flops(m, rx, ry, sp["mask"])
            nbytes += W.partial_chain_bytes(m, rx, ry, sp["mask"], 4)
        flops += f
        costs.append(f)
    # N > 1: every rank contracts its own LPT shard of the pairs (no exchange)
    subset = S.lpt_shards(costs, world)[rank] if world > 1 else None
    specs, pairs = G.batch4096_device(4096, 0, dev, subset=subset)
    stream = torch.cuda.current_stream(dev)
    K = max(3, args.steps // 20)

    def time_graph(bat):
        g = bat.graph()
        for _ in range(max(3, args.warmup // 4)):
            g.replay()
        torch.cuda.synchronize(dev)
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)
        for a, b in evs:
            a.record(stream)
            g.replay()
            b.record(stream)
        torch.cuda.synchronize(dev)
        t_ms = statistics.mean(a.elapsed_time(b) for a, b in evs)
        if world > 1:
            t = torch.tensor([t_ms], device=dev)
            torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
            t_ms = float(t.item())
        del g
        return t_ms

    # untuned (the default tile configuration for every pair), then the
    # autotuner's cache (built here, before timing) and the tuned plan
    saved = os.environ.pop("TTC_AUTOTUNE_CACHE", None)
    bat0 = T.BatchedContraction(pairs)
    ms_untuned = time_graph(bat0)
    del bat0
    t_tune = time.perf_counter()
    cache = os.path.join(tempfile.gettempdir(), f"ttc_autotune_f32_rank{rank}.txt")
    T.autotune("f32", cache)
    tune_s = time.perf_counter() - t_tune
    os.environ["TTC_AUTOTUNE_CACHE"] = cache
    bat = T.BatchedContraction(pairs)
    setup_s = time.perf_counter() - t0
    ms = time_graph(bat)
    if saved is not None:
        os.environ["TTC_AUTOTUNE_CACHE"] = saved
    else:
        os.environ.pop("TTC_AUTOTUNE_CACHE", None)
    achieved = flops / (ms / 1e3) / 1e12
    peak = fp32_simt_peak_tflops()
    hbm = _peaks().get("hbm_gbs", 6683.2)
    out = {
        "workload": "4096 TT pairs, order U{4..12}, modes U{2..32}, ranks U{4..128}, float32; even pairs full, odd pairs partial over an end block of floor(N/2) modes; one CUDA-graph replay of one persistent launch",
        "sharding": "pairs dealt to ranks longest-first by predicted flops; whole-job time = slowest rank" if world > 1 else "single GPU",
        "pairs_this_rank": len(specs),
        "value": 4096 / (ms / 1e3),
        "unit": "contractions/s",
        "ms_per_launch": ms,
        "launches": K,
        "gflops": flops / (ms / 1e3) / 1e9,
        "alg_flops": flops,
        "alg_bytes": nbytes,
        "roofline": {
            "kernel": "batched_kernel<float>",
            "bound": "alu",
            "achieved": achieved,
            "peak": peak,
            "unit": "TFLOP/s",
            "frac": achieved / peak,
            "hbm_gbs": nbytes / (ms / 1e3) / 1e9,
            "hbm_frac": nbytes / (ms / 1e3) / 1e9 / hbm,
        },
        "tiles": {str(int(t)): int(c) for t, c in zip(*np.unique(bat.tiles(), return_counts=True))},
        "tiles_note": "tile configuration = panel-budget level + 3 x replica-cap index (caps none, 1, 2, 4); "
                      "chosen per (rank, mode size) bucket by the autotuner, run before timing",
        "value_untuned": 4096 / (ms_untuned / 1e3),
        "ms_per_launch_untuned": ms_untuned,
        "autotune_s": tune_s,
        "setup_s": setup_s,
        "device_status": int(bat.status.item()),
        "gpu_launches_per_replay": 1,
    }
    del bat, pairs
    torch.cuda.empty_cache()
    if world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline_batched()
    return out


def _bf16_peak():
    pk = _peaks()
    return pk.get("bf16_tflops", 1933.5), pk.get("bf16_tflops_sustained", 1747.6)


def merged_masks(draws=8, order=6, size=3):
    """Seeded random contracted sets S, |S| = size of order modes."""
    out = []
    for d in range(draws):
        mask = [0] * order
        for k in np.random.default_rng([2109, d]).choice(order, size, replace=False):
            mask[int(k)] = 1
        out.append(mask)
    return out


def merged_bytes(x, y, zs, ebytes):
    """Cores read once plus the merged output cores written once."""
    return ebytes * (sum(c.size for c in x) + sum(c.size for c in y) + sum(int(np.prod(s)) for s in zs))


def bench_merged(T, dev, args):
    """Partial contraction over a random set of three of six modes, merged
    (TT-matrix) layout: modes 8, ranks 16, float32; eight seeded draws of S,
    timed in turn with an L2 flush before each contraction."""
    import torch

    x, y = G.pair(13, [8] * 6, G.tt_ranks(6, 16), G.tt_ranks(6, 16), np.float32)
    xd = [torch.from_numpy(c).to(dev) for c in x]
    yd = [torch.from_numpy(c).to(dev) for c in y]
    masks = merged_masks()
    ops = [T.PartialContraction(xd, yd, m, layout="merged") for m in masks]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    for _ in range(3):
        for op in ops:
            op(stream)
    torch.cuda.synchronize(dev)
    R = max(3, args.steps // 40)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(R * len(ops))]
    for r in range(R):
        for k, op in enumerate(ops):
            flush.fill_(float(r))  # L2 flush between timed contractions (untimed)
            a, b = ev[r * len(ops) + k]
            a.record(stream)
            op(stream)
            b.record(stream)
    torch.cuda.synchronize(dev)
    per = [statistics.mean(ev[r * len(ops) + k][0].elapsed_time(ev[r * len(ops) + k][1]) for r in range(R))
           for k in range(len(ops))]
    ms = statistics.mean(per)
    nbytes = statistics.mean(merged_bytes(x, y, [tuple(c.shape) for c in op.z], 4) for op in ops)
    hbm = _peaks().get("hbm_gbs", 6683.2)
    status = 0
    for op in ops:
        status |= int(op.status.item())
    extra = {}
    if not args.no_cpu_baseline:
        import oracle as O

        extra["cpu_baseline"] = _oracle_once(lambda: O.partial_merged(x, y, masks[0]), "contractions/s",
                                             "one contraction over the first set, numpy float64 merged cores")
    return {
        **extra,
        "workload": "order-6 TT pair, modes 8, ranks 16, float32; partial contraction over a random S, |S| = 3, "
                    "merged layout; eight seeded draws of S timed in turn",
        "sets": ["".join(str(v) for v in m) for m in masks],
        "value": 1.0 / (ms / 1e3),
        "unit": "contractions/s",
        "ms_per_contraction": ms,
        "ms_per_set": per,
        "alg_bytes": nbytes,
        "roofline": {
            "kernel": "whole contraction (zrows_kernel writes the merged cores)",
            "bound": "hbm",
            "achieved": nbytes / (ms / 1e3) / 1e9,
            "peak": hbm,
            "unit": "GB/s",
            "frac": nbytes / (ms / 1e3) / 1e9 / hbm,
            "note": "bytes = cores read once + merged cores written once, mean over the draws; "
                    "peak = measured HBM copy bandwidth",
        },
        "device_status": status,
        "l2": "flushed before each contraction",
    }


FACTORED_MASK = [1, 0, 0, 1, 1, 1, 0, 0]


def _oracle_once(fn, unit, sample):
    """The float64 oracle timed beside a GPU form: one call of fn on one host
    thread (OPENBLAS_NUM_THREADS=1), as a rate in the form's unit."""
    t0 = time.perf_counter()
    fn()
    dt = time.perf_counter() - t0
    return {"value": 1.0 / dt, "unit": unit, "cores": 1, "kind": "oracle", "sample": sample, "seconds": dt}


def bench_factored(T, dev, args):
    """General-S partial contraction at rank 64 in factored form: order 8,
    modes 16, ranks 64, float32, S = {0, 3, 4, 5} (the left environment of mode
    0 and the 4096 x 4096 transfer matrix of the interior run 3-5; the merged
    layout's cores would hold 4096 x 16 x 16 x 4096 entries).  CUDA events on
    the launching stream, L2 flushed before each call."""
    import torch

    x, y = G.pair(3, [16] * 8, G.tt_ranks(8, 64), G.tt_ranks(8, 64), np.float32)
    xd = [torch.from_numpy(c).to(dev) for c in x]
    yd = [torch.from_numpy(c).to(dev) for c in y]
    op = T.FactoredContraction(xd, yd, FACTORED_MASK)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    for _ in range(2):
        op(stream)
    torch.cuda.synchronize(dev)
    ts = []
    for r in range(5):
        flush.fill_(float(r))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        op(stream)
        b.record(stream)
        torch.cuda.synchronize(dev)
        ts.append(a.elapsed_time(b))
    ms = statistics.median(ts)
    rx = [c.shape[0] for c in x] + [1]
    ry = [c.shape[0] for c in y] + [1]
    flops = W.factored_flops([16] * 8, rx, ry, FACTORED_MASK)
    peak = fp32_simt_peak_tflops()
    out_bytes = sum(r[0].numel() * 4 + r[1].numel() * 8 for r in op.runs() if r is not None)
    extra = {}
    if not args.no_cpu_baseline:
        import oracle as O

        extra["cpu_baseline"] = _oracle_once(lambda: O.partial_factored(x, y, FACTORED_MASK), "contractions/s",
                                             "one contraction, numpy float64 transfer matrices (4096 x 4096)")
    return {
        **extra,
        "workload": "order-8 TT pair, modes 16, ranks 64, float32; partial contraction over S = {0, 3, 4, 5} "
                    "in factored form (left environment + 4096 x 4096 transfer matrix)",
        "value": 1.0 / (ms / 1e3),
        "unit": "contractions/s",
        "ms_per_contraction": ms,
        "alg_flops": flops,
        "out_bytes": out_bytes,
        "roofline": {
            "kernel": "transfer_kernel<float> (the interior run's rows)",
            "bound": "alu",
            "achieved": flops / (ms / 1e3) / 1e12,
            "peak": peak,
            "unit": "TFLOP/s",
            "frac": flops / (ms / 1e3) / 1e12 / peak,
            "note": "flops = 4096 basis sweeps of the run (the first mode from a unit environment) + the left "
                    "environment; fp32 FMA peak derived",
        },
        "device_status": int(op.status.item()),
        "l2": "flushed before each call",
    }


RS_STREAMS = 16  # streams the random-set batch's independent calls are dealt over


def bench_random_sets(T, dev, args, n_pairs=512):
    """The batch's secondary run over truly random contracted sets: 512 pairs
    of order U{4..12}, modes U{2..32}, ranks U{4..16}, float32, S = a random
    set of floor(N/2) modes at any positions, factored output (the merged
    layout's Kronecker factors; the merged cores themselves would reach
    256 x 32 x 32 x 256 entries).  One contraction call per pair (each call
    its own few launches, none using more than one cluster), dealt round-robin
    over RS_STREAMS streams forked from and joined back into the timing
    stream between two CUDA events, so independent pairs share the GPU; also
    the same calls captured once in a CUDA graph and replayed; beside it the
    float64 oracle on a sample of pairs on one host thread."""
    import time as _time

    import torch

    import oracle as O

    pairs = [G.random_sets_pair(p) for p in range(n_pairs)]
    ops = []
    for mask, x, y in pairs:
        xd = [torch.from_numpy(c).to(dev) for c in x]
        yd = [torch.from_numpy(c).to(dev) for c in y]
        ops.append(T.FactoredContraction(xd, yd, mask))
    stream = torch.cuda.current_stream(dev)
    lanes = [torch.cuda.Stream(dev) for _ in range(RS_STREAMS)]

    def run_all(base):
        for ln in lanes:
            ln.wait_stream(base)
        for q, op in enumerate(ops):
            op(lanes[q % RS_STREAMS])
        for ln in lanes:
            base.wait_stream(ln)

    run_all(stream)  # first calls (and per-stream library handles) outside the timing
    torch.cuda.synchronize(dev)
    ts = []
    for r in range(3):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        run_all(stream)
        b.record(stream)
        torch.cuda.synchronize(dev)
        ts.append(a.elapsed_time(b))
    ms = statistics.median(ts)
    # the same 512 calls captured once in a CUDA graph and replayed: the
    # device time of the batch without the host's per-call launch overhead
    graph_ms = None
    try:
        side = torch.cuda.Stream(dev)
        side.wait_stream(stream)
        run_all(side)
        stream.wait_stream(side)
        torch.cuda.synchronize(dev)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=side):
            run_all(side)
        g.replay()
        torch.cuda.synchronize(dev)
        gts = []
        for r in range(3):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            g.replay()
            b.record(stream)
            torch.cuda.synchronize(dev)
            gts.append(a.elapsed_time(b))
        graph_ms = statistics.median(gts)
        del g
    except RuntimeError as e:  # a call the capture refuses: report the eager number alone
        graph_ms = None
        print(f"random_sets: graph capture failed: {e}", file=sys.stderr)
    flops = sum(W.factored_flops([c.shape[1] for c in x_], [c.shape[0] for c in x_] + [1],
                                 [c.shape[0] for c in y_] + [1], m) for m, x_, y_ in pairs)
    status = 0
    for op in ops:
        status |= int(op.status.item())
    out = {
        "workload": "512 TT pairs, order U{4..12}, modes U{2..32}, ranks U{4..16}, float32; partial contraction "
                    "over a random set of floor(N/2) modes (any positions), factored output; one call per pair, "
                    f"dealt round-robin over {RS_STREAMS} streams",
        "value": n_pairs / (ms / 1e3),
        "unit": "contractions/s",
        "ms_per_batch": ms,
        "ms_per_batch_graph": graph_ms,
        "value_graph": n_pairs / (graph_ms / 1e3) if graph_ms else None,
        "alg_flops": flops,
        "gflops": flops / (ms / 1e3) / 1e9,
        "device_status": status,
    }
    if not args.no_cpu_baseline:
        t0 = _time.perf_counter()
        k = 0
        while k < n_pairs and _time.perf_counter() - t0 < 5.0:
            m, x_, y_ = pairs[k]
            O.partial_factored(x_, y_, m)
            k += 1
        dt = _time.perf_counter() - t0
        out["cpu_baseline"] = {"value": k / dt, "unit": "contractions/s", "cores": 1, "kind": "oracle",
                               "sample": f"the first {k} pairs, numpy float64 transfer matrices, one thread"}
    return out


def bench_round(T, dev, args):
    """TT rounding of a merged-layout result: order-5 operands, modes 8, ranks
    8, float32, S = {1, 3}: merged cores of ranks up to 64 and modes 8 x 8,
    rounded at eps 1e-4 (tt_round on the GPU, CUDA events around the call
    and the read of the new ranks); the error of the rounded result against
    Eq. 8 on the dense operands and the float64 oracle's rounding timed
    beside it."""
    import time as _time

    import torch

    import oracle as O

    x, y = G.pair(6, [8] * 5, G.tt_ranks(5, 8), G.tt_ranks(5, 8), np.float32)
    mask = [0, 1, 0, 1, 0]
    xd = [torch.from_numpy(c).to(dev) for c in x]
    yd = [torch.from_numpy(c).to(dev) for c in y]
    op = T.PartialContraction(xd, yd, mask, layout="merged")
    op()
    torch.cuda.synchronize(dev)
    eps = 1e-4
    stream = torch.cuda.current_stream(dev)
    for _ in range(2):
        out = T.round_merged(op.z, eps)
    torch.cuda.synchronize(dev)
    ts = []
    for _ in range(5):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        out = T.round_merged(op.z, eps)
        b.record(stream)
        torch.cuda.synchronize(dev)
        ts.append(a.elapsed_time(b))
    ms = statistics.median(ts)
    got = O.merged_to_dense([c.cpu().numpy().astype(np.float64).reshape(c.shape[0], 8, 8, c.shape[2]) for c in out],
                            op.perm)
    want = O.tcp(O.tt_to_dense([c.astype(np.float64) for c in x]), O.tt_to_dense([c.astype(np.float64) for c in y]),
                 [1, 3])
    res = {
        "workload": "merged result of an order-5 pair (modes 8, ranks 8, float32, S = {1, 3}): cores of ranks "
                    "up to 64 and modes 8 x 8, TT-rounded at eps 1e-4",
        "ms": ms,
        "value": 1.0 / (ms / 1e3),
        "unit": "roundings/s",
        "ranks_in": [int(c.shape[0]) for c in op.z] + [1],
        "ranks_out": [int(c.shape[0]) for c in out] + [1],
        "err_rel_frobenius": float(np.linalg.norm(got - want) / np.linalg.norm(want)),
        "roofline": {"bound": "latency", "note": "one cluster launch runs both sweeps of per-core Jacobi SVDs "
                                                "(dependent rounds; unfoldings too large for one CTA spread over "
                                                "16 CTAs, two cluster barriers per round)"},
    }
    if not args.no_cpu_baseline:
        flat = [c.cpu().numpy().astype(np.float64) for c in op.z]
        t0 = _time.perf_counter()
        O.tt_round(flat, eps)
        res["cpu_baseline"] = {"value": 1.0 / (_time.perf_counter() - t0), "unit": "roundings/s", "cores": 1,
                               "kind": "oracle", "sample": "one rounding, numpy float64 (QR and SVD), one thread"}
    return res


EXAMPLE2_Y = [(20, 20, 20), (20, 20, 20, 5), (20, 20, 20, 5, 4)]


def bench_dense_ttcp(T, dev, args):
    """Dense-input contraction (Alg. 2 on dense operands): Example 2's
    X x_1^1 Y with X in R^{20x20x20} and Y of 20^3, 20^3 x 5 and
    20^3 x 5 x 4, Gaussian, float32, eps = 1e-6 (full ranks): both TT-SVDs
    and the contraction of the leading pair, timed end to end with CUDA
    events (the call reads the chosen ranks back to size the contraction);
    beside it the float64 oracle (its TT decomposition of both operands and
    the chain contraction) on one host thread, and the accuracy of the GPU
    result against Eq. 8 on the dense tensors."""
    import time as _time

    import torch

    import oracle as O

    rng = np.random.default_rng(2109)
    xh = rng.standard_normal((20, 20, 20)).astype(np.float32)
    stream = torch.cuda.current_stream(dev)
    out = {"workload": "Example 2 shapes: X 20^3 x_1^1 Y (Y = 20^3, 20^3x5, 20^3x5x4), Gaussian, float32, "
                       "eps 1e-6; TT-SVD of both operands on the GPU, then the leading-pair chain contraction",
           "cases": []}
    status = 0
    for ys in EXAMPLE2_Y:
        yh = rng.standard_normal(ys).astype(np.float32)
        x = torch.from_numpy(xh).to(dev)
        y = torch.from_numpy(yh).to(dev)
        for _ in range(2):
            z, perm = T.contract_dense_pairs(x, y, [(0, 0)], 1e-6)
        torch.cuda.synchronize(dev)
        R = 5
        ts = []
        for _ in range(R):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            z, perm = T.contract_dense_pairs(x, y, [(0, 0)], 1e-6)
            b.record(stream)
            torch.cuda.synchronize(dev)
            ts.append(a.elapsed_time(b))
        ms = statistics.median(ts)
        got = O.chain_to_dense([c.detach().cpu().numpy().astype(np.float64) for c in z], perm)
        want = O.tcp_pairs(xh.astype(np.float64), yh.astype(np.float64), [(0, 0)])
        rel = float(np.linalg.norm(got - want) / (np.linalg.norm(xh) * np.linalg.norm(yh)))
        case = {"y_shape": list(ys), "ms": ms, "value": 1.0 / (ms / 1e3), "unit": "dense contractions/s",
                "ranks_z": [int(c.shape[0]) for c in z] + [1], "err_rel_frobenius": rel}
        if not args.no_cpu_baseline:
            t0 = _time.perf_counter()
            xc = O.tt_svd(xh.astype(np.float64), 1e-6)
            yc = O.tt_svd(yh.astype(np.float64), 1e-6)
            O.partial_chain_pairs(xc, yc, [(0, 0)])
            dt = _time.perf_counter() - t0
            case["cpu_baseline"] = {"value": 1.0 / dt, "unit": "dense contractions/s", "cores": 1, "kind": "oracle",
                                    "sample": "one call: numpy float64 TT decomposition of both operands and the "
                                              "chain contraction"}
        out["cases"].append(case)
    out["value"] = statistics.mean(c["value"] for c in out["cases"])
    out["unit"] = "dense contractions/s (mean over the three shapes)"
    out["roofline"] = {"bound": "latency", "note": "one cluster launch runs each decomposition, X's and Y's "
                                                   "concurrently on two streams (dependent Jacobi rounds); "
                                                   "a few MB of data, no roofline fraction is meaningful"}
    out["device_status"] = status
    return out


_TC_RESULTS = {}  # precision form -> (mantissa, exponent) of its last z, for the accuracy report
_ORACLE_TIMES = {}  # workload -> the oracle's timing, shared by the forms that run it


def bench_bf16(T, dev, args, prec):
    """Order 16, modes 32, ranks 256, log-normal core scales; full contraction
    on the tensor cores: bfloat16 cores with float32 sums ("native"), or the
    split-bfloat16 x3 products on the float32 cores ("bf16x3")."""
    import torch

    x, y = G.order16_r256(0)
    if prec == "native":
        xd = [torch.from_numpy(c).to(dev).bfloat16() for c in x]
        yd = [torch.from_numpy(c).to(dev).bfloat16() for c in y]
        ebytes = 2
    else:
        xd = [torch.from_numpy(c).to(dev) for c in x]
        yd = [torch.from_numpy(c).to(dev) for c in y]
        ebytes = 4
    op = T.FullContraction(xd, yd, prec=prec, split=True)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    for _ in range(max(3, args.warmup // 4)):
        op()
    torch.cuda.synchronize(dev)
    K = max(5, args.steps // 10)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    for a, b in evs:
        flush.fill_(1.0)
        a.record(stream)
        op()
        b.record(stream)
    torch.cuda.synchronize(dev)
    ms = statistics.mean(a.elapsed_time(b) for a, b in evs)
    _TC_RESULTS[prec] = (float(op.out.item()), int(op.log2.item()))
    modes, r = [32] * 16, G.tt_ranks(16, 256)
    flops = W.full_flops(modes, r, r)
    nprod = 3 if prec == "bf16x3" else 1
    burst, sustained = _bf16_peak()
    achieved = flops * nprod / (ms / 1e3) / 1e12
    del op, xd, yd, flush
    torch.cuda.empty_cache()
    extra = {}
    if not args.no_cpu_baseline:
        import oracle as O

        if "order16" not in _ORACLE_TIMES:
            _ORACLE_TIMES["order16"] = _oracle_once(lambda: O.contract_full(x, y), "contractions/s",
                                                    "one contraction of the float32 cores, numpy float64 sweep")
        extra["cpu_baseline"] = _ORACLE_TIMES["order16"]
    return {
        **extra,
        "workload": "order-16 TT pair, modes 32, ranks 256, log-normal core scales (sigma 1); full contraction on tcgen05 tensor cores" + (", bf16 cores, fp32 sums, fp64 final sum" if prec == "native" else ", fp32 cores split into hi+lo bf16, 3 products per step"),
        "value": 1.0 / (ms / 1e3),
        "unit": "contractions/s",
        "ms_per_contraction": ms,
        "gflops": flops / (ms / 1e3) / 1e9,
        "alg_flops": flops,
        "alg_bytes": W.full_bytes(modes, r, r, ebytes),
        "roofline": {
            "kernel": "tc_mode_kernel<%s>" % ("true" if prec == "bf16x3" else "false"),
            "bound": "tensor",
            "achieved": achieved,
            "peak": burst,
            "unit": "TFLOP/s",
            "frac": achieved / burst,
            "note": "tensor products counted (x3 for the split variant); peak = measured bf16 burst",
        },
        "l2": "flushed before each contraction",
    }


def bench_backward(T, dev, args):
    """Gradients of loss = sum(Z), Z = partial contraction over modes 1-8 of the
    order-12, mode 16, rank 64 float32 pair, with respect to all 24 cores."""
    import torch

    x, y = G.order12_r64(0)
    xd = [torch.from_numpy(c).to(dev).requires_grad_(True) for c in x]
    yd = [torch.from_numpy(c).to(dev).requires_grad_(True) for c in y]
    mask = [1] * 8 + [0] * 4
    stream = torch.cuda.current_stream(dev)

    def step():
        for c in xd + yd:
            c.grad = None
        zc = T.tt_partial(xd, yd, mask)
        loss = T.tt_sum(zc)
        loss.backward()

    for _ in range(max(3, args.warmup // 4)):
        step()
    torch.cuda.synchronize(dev)
    K = max(5, args.steps // 10)
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(K):
        step()
    b.record(stream)
    torch.cuda.synchronize(dev)
    ms = a.elapsed_time(b) / K
    # the same step captured once in a CUDA graph and replayed (how a training
    # loop would run it: no Python between the kernels)
    side = torch.cuda.Stream(dev)
    side.wait_stream(stream)
    with torch.cuda.stream(side):
        for _ in range(3):
            step()
    stream.wait_stream(side)
    for c in xd + yd:
        c.grad = None
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        zc = T.tt_partial(xd, yd, mask)
        loss = T.tt_sum(zc)
        loss.backward()
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize(dev)
    a.record(stream)
    for _ in range(K):
        g.replay()
    b.record(stream)
    torch.cuda.synchronize(dev)
    graph_ms = a.elapsed_time(b) / K
    del g
    extra = {}
    if not args.no_cpu_baseline:
        import oracle as O

        def oracle_step():
            zo, _ = O.partial_chain(x, y, mask)
            ones = [np.ones((1, c.shape[1], 1)) for c in zo]
            O.contract_full(zo, ones)
            dz, _ = O.grad_full(zo, ones)
            O.grad_partial_chain(x, y, mask, dz)

        extra["cpu_baseline"] = _oracle_once(oracle_step, "gradient evaluations/s",
                                             "one step (partial contraction, its sum, the gradients of every "
                                             "core), numpy float64")
    modes, r = [16] * 12, G.tt_ranks(12, 64)
    fwd = W.partial_chain_flops(modes, r, r, mask)
    # adjoint: five products per contracted mode (U, dGx, W, dGy, next F), counted without recompute
    bwd = sum(5 * W.mode_flops(r[k], r[k + 1], r[k], r[k + 1], modes[k]) // 2 for k in range(8))
    return {
        "workload": "order-12 TT pair, modes 16, ranks 64, float32; loss = sum of the partial contraction over modes 1-8; gradients of all 24 cores through torch.autograd (TTPartial, TTFull)",
        "value": 1.0 / (graph_ms / 1e3),
        "unit": "gradient evaluations/s",
        "ms_per_step": graph_ms,
        "ms_per_step_graph": graph_ms,
        "ms_per_step_eager": ms,
        "value_eager": 1.0 / (ms / 1e3),
        "gflops": (fwd + bwd) / (graph_ms / 1e3) / 1e9,
        "alg_flops": fwd + bwd,
        "roofline": {
            "kernel": "whole gradient step (sweep_cluster_kernel: the forward partial and the right-environment "
                      "sweep; adjoint_grads_kernel; the rank-1 chains of the sum)",
            "bound": "alu",
            "achieved": (fwd + bwd) / (graph_ms / 1e3) / 1e12,
            "peak": fp32_simt_peak_tflops(),
            "unit": "TFLOP/s",
            "frac": (fwd + bwd) / (graph_ms / 1e3) / 1e12 / fp32_simt_peak_tflops(),
            "note": "latency-bound single instance (environment sweeps on clusters of 16 SMs); forward + adjoint "
            "products (five per contracted mode); timed as a CUDA-graph replay of the whole step "
            "(value_eager / ms_per_step_eager: the same step launched from Python through torch.autograd)",
        },
        **extra,
    }


def run_profile_case(case):
    """Small cases for ncu captures (a few GB at most on the device)."""
    import torch

    import paper_2109_00626_gb300 as T

    dev = torch.device("cuda", 0)
    if case in ("tc_native", "tc_x3"):
        x, y = G.order16_r256(0)
        conv = (lambda c: torch.from_numpy(c).to(dev).bfloat16()) if case == "tc_native" else (lambda c: torch.from_numpy(c).to(dev))
        op = T.FullContraction([conv(c) for c in x], [conv(c) for c in y],
                               prec="native" if case == "tc_native" else "bf16x3", split=True)
        for _ in range(2):
            op()
        status = op.status
    elif case == "backward":
        x, y = G.order12_r64(0)
        xd = [torch.from_numpy(c).to(dev).requires_grad_(True) for c in x]
        yd = [torch.from_numpy(c).to(dev).requires_grad_(True) for c in y]
        mask = [1] * 8 + [0] * 4
        for _ in range(2):
            for c in xd + yd:
                c.grad = None
            loss = T.tt_sum(T.tt_partial(xd, yd, mask))
            loss.backward()
        torch.cuda.synchronize(dev)
        status = torch.tensor([0 if math.isfinite(float(loss.detach())) else 1])
    elif case == "merged":
        x, y = G.pair(13, [8] * 6, G.tt_ranks(6, 16), G.tt_ranks(6, 16), np.float32)
        xd, yd = [torch.from_numpy(c).to(dev) for c in x], [torch.from_numpy(c).to(dev) for c in y]
        status = torch.zeros(1, dtype=torch.int32, device=dev)
        for m in merged_masks():
            op = T.PartialContraction(xd, yd, m, layout="merged")
            op()
            status |= op.status
    elif case == "order10_tf32x3":
        x, y = G.order10_r64(0, np.float32)
        xd, yd = [torch.from_numpy(c).to(dev) for c in x], [torch.from_numpy(c).to(dev) for c in y]
        full = T.FullContraction(xd, yd, prec="tf32x3")
        part = T.PartialContraction(xd, yd, MASK, prec="tf32x3")
        for _ in range(2):
            full()
            part()
        status = full.status | part.status
    elif case == "dense_ttcp":
        rng = np.random.default_rng(2109)
        x = torch.from_numpy(rng.standard_normal((20, 20, 20)).astype(np.float32)).to(dev)
        y = torch.from_numpy(rng.standard_normal((20, 20, 20, 5, 4)).astype(np.float32)).to(dev)
        for _ in range(2):
            T.contract_dense_pairs(x, y, [(0, 0)], 1e-6)
        status = torch.zeros(1, dtype=torch.int32)
    elif case == "factored":
        x, y = G.pair(3, [16] * 8, G.tt_ranks(8, 64), G.tt_ranks(8, 64), np.float32)
        op = T.FactoredContraction([torch.from_numpy(c).to(dev) for c in x], [torch.from_numpy(c).to(dev) for c in y],
                                   FACTORED_MASK)
        for _ in range(2):
            op()
        status = op.status
    elif case == "round":
        x, y = G.pair(6, [8] * 5, G.tt_ranks(5, 8), G.tt_ranks(5, 8), np.float32)
        op = T.PartialContraction([torch.from_numpy(c).to(dev) for c in x], [torch.from_numpy(c).to(dev) for c in y],
                                  [0, 1, 0, 1, 0], layout="merged")
        op()
        for _ in range(2):
            T.round_merged(op.z, 1e-4)
        status = op.status
    elif case == "batched512":
        _, pairs = G.batch4096_device(512, 0, dev)
        op = T.BatchedContraction(pairs)
        for _ in range(2):
            op()
        status = op.status
    else:
        x, y = G.order10_r64(0, np.float32)
        op = T.FullContraction([torch.from_numpy(c).to(dev) for c in x], [torch.from_numpy(c).to(dev) for c in y])
        for _ in range(2):
            op()
        status = op.status
    torch.cuda.synchronize(dev)
    print(json.dumps({"profile_case": case, "device_status": int(status.item())}))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true")
    ap.add_argument("--forms", default="all", help="comma-separated subset of the secondary forms to run (default all)")
    ap.add_argument("--profile-case", choices=["tc_native", "tc_x3", "batched512", "order10", "order10_tf32x3", "backward",
                                               "merged", "dense_ttcp", "factored", "round"],
                    default=None,
                    help="run a small case twice for an ncu capture and exit (no JSON line)")
    ap.add_argument("--measure-peaks", action="store_true",
                    help="time cuBLAS SGEMM (TF32 off) and DGEMM as reference peaks and exit")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.profile_case:
        return run_profile_case(args.profile_case)
    if args.measure_peaks:
        return measure_peaks()
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
