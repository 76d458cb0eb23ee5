#!/usr/bin/env python3
"""Decoded Mbit/s of the GB300 layered BP syndrome decoder (arXiv 2004.09084).

Workload (default): the rate-0.1 QC-MET-LDPC stand-in code with Z = 12500
(n = 10^6), 128 codewords per GPU of random bits with syndromes s = Hx, BIAWGN
channel LLRs at SNR 0.161, 100 layered iterations, no early termination.  A
step is one full decode of the 128 codewords (one kernel launch).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank decodes its own 128 codewords (frames are
independent: weak scaling, no collective on the data path); the step time is
the maximum over ranks.  ``--impl reference`` times the FP64 CPU oracle on the
host cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
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

import synth  # noqa: E402

METRIC = "decoded Mbit/s (128x1e6-bit codewords, fixed iters) and FER vs plain FP32 BP"
RATE = "0.1"
Z = 12500
K_FRAMES = 128
ITERS = 100
SNR = 0.161
BYTES_PER_EDGE = {"fp32": 16, "fp16": 12, "bf16": 12}   # per edge, frame and iteration
# ncu DRAM counts of the dominant kernel, one per decode kernel
PROFILES = {
    "group": os.path.join(ROOT, "profiles", "decode_group_kernel_rate0.1_Z12500_K128_T100.txt"),
    "frame": os.path.join(ROOT, "profiles", "decode_kernel_rate0.1_Z12500_K128_T100.txt"),
}
KERNEL_SOURCES = {
    "group": ("decode_group.cu", "check_rule.cuh", "qcmet_internal.h"),
    "frame": ("decode.cu", "check_rule.cuh", "qcmet_internal.h"),
}


def workload_name(msg: str) -> str:
    return (f"rate-{RATE} QC-MET-LDPC [[A,0],[B,I70]] 72x80, Z={Z} (n=1e6), {K_FRAMES} codewords/GPU, "
            f"SNR {SNR}, {ITERS} layered iterations, {msg.upper()} messages, no early termination")


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def kernel_hash(kernel: str = "group") -> str:
    """sha256 (first 16 hex digits) of a kernel's sources with // comments and
    blank lines removed, so that a comment edit keeps a profile valid."""
    h = hashlib.sha256()
    for name in KERNEL_SOURCES[kernel]:
        with open(os.path.join(ROOT, "paper_2004_09084_gb300", "csrc", name)) as f:
            for line in f:
                code = line.split("//", 1)[0].rstrip()
                if code:
                    h.update(code.encode() + b"\n")
    return h.hexdigest()[:16]


def profiled_traffic(kernel: str = "group"):
    """DRAM bytes per launch from the committed ncu summary, if it still matches the kernel."""
    path = PROFILES[kernel]
    if not os.path.exists(path):
        return None
    vals = {}
    with open(path) as f:
        for line in f:
            if ":" in line and not line.startswith("#"):
                k, v = line.split(":", 1)
                vals[k.strip()] = v.strip()
    if vals.get("kernel_source_sha256_16") != kernel_hash(kernel):
        return None
    try:
        return float(vals["dram_bytes_per_launch_full"])
    except (KeyError, ValueError):
        return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (FileNotFoundError, OSError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None or not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx.append(float(parts[2]))
                except ValueError:
                    continue
                for name, val in zip(names, parts[5:9]):
                    if val.lower().startswith("active"):
                        reasons.add(name)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU oracle timing (the reference arm and the cpu_baseline)

def oracle_sample(code, cores: int, iters: int = 20):
    """Time the FP64 oracle on `cores` frames x `iters` iterations; returns (Mbit/s, seconds, desc)."""
    import oracle
    fr = synth.make_frames(code, cores, SNR, first=10_000)
    oracle.build()
    t0 = time.perf_counter()
    oracle.decode(code.base, code.shifts, code.Z, fr.llr, fr.syn, iters, nthreads=cores)
    dt = time.perf_counter() - t0
    edge_updates = cores * iters * code.edges
    rate = edge_updates / dt                                    # edge updates per second
    mbit = code.n * rate / (code.edges * ITERS) / 1e6           # Mbit/s at 100 iterations
    desc = (f"{cores} frames x {iters} iterations of the Z={code.Z} code ({edge_updates:.3g} edge "
            f"updates, {dt:.1f} s wall on {cores} threads), scaled linearly to {ITERS} iterations")
    return mbit, dt, desc


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    code = synth.make_code(RATE, Z)
    cores = os.cpu_count() or 1
    oracle_sample(code, 1, 1)   # untimed warm-up (build, page-in)
    vals = []
    desc = ""
    for _ in range(max(args.steps, 1)):
        v, dt, desc = oracle_sample(code, cores)
        vals.append(v)
    value = statistics.median(vals)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "Mbit/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": K_FRAMES * code.n / (value * 1e6) * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": workload_name("fp64 (oracle)"),
                                        "parallelism": "host threads, one frame per thread"},
        "cpu_baseline": {"value": value, "unit": "Mbit/s", "cores": cores, "kind": "oracle",
                         "sample": desc},
        "e2e": {"value": value, "unit": "Mbit/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------

def frame_offset(rank: int, frames_per_rank: int) -> int:
    """First frame index of a rank: ranks decode disjoint frame sets (weak scaling)."""
    return rank * frames_per_rank


def max_over_ranks(value: float, device=None) -> float:
    """Step time of the whole job: the slowest rank's (identity without a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_mbit_per_s(world: int, frames_per_rank: int, n: int, seconds: float) -> float:
    """Whole-job decoded Mbit/s: all ranks' bits over the slowest rank's time."""
    return world * frames_per_rank * n / seconds / 1e6


def progress(msg: str):
    print(f"[bench {time.strftime('%H:%M:%S')}] {msg}", file=sys.stderr, flush=True)


def run_ours(args):
    import torch
    import torch.distributed as dist

    import paper_2004_09084_gb300 as q

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local if world > 1 else torch.cuda.current_device())
    torch.cuda.set_device(dev)

    code = synth.make_code(RATE, Z)
    qc = q.Code(code.base, code.shifts, code.Z)
    fr = synth.make_frames(code, K_FRAMES, SNR, first=frame_offset(rank, K_FRAMES))
    n = code.n
    llr = torch.from_numpy(fr.llr).to(dev)
    syn = torch.from_numpy(fr.syn).to(dev)
    hard = torch.empty((K_FRAMES, n), dtype=torch.uint8, device=dev)
    post = torch.empty((K_FRAMES, n), dtype=torch.float32, device=dev)
    ok = torch.empty((K_FRAMES,), dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        q.decode(qc, llr, syn, ITERS, hard=hard, llr_post=post, ok=ok, msg=args.msg,
                 stream=stream, l2_persist=args.l2_persist == "on", kernel=args.kernel,
                 cluster=args.cluster)

    progress("inputs resident; warm-up")
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    progress("timed region")

    def barrier():
        if world > 1:
            dist.barrier()

    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    with ClockSampler(dev.index if dev.index is not None else 0) as clk:
        barrier()
        torch.cuda.synchronize(dev)
        start.record(stream)
        for _ in range(args.steps):
            step()
        end.record(stream)
        torch.cuda.synchronize(dev)
        barrier()
    ms = max_over_ranks(start.elapsed_time(end) / args.steps, dev)
    clocks = clk.summary()
    progress(f"timed region done: {ms:.2f} ms/step; end-to-end leg")

    # decode quality of the last step (outside the timed region)
    h_cpu = hard.cpu().numpy()
    ok_cpu = ok.cpu().numpy()
    fer = float(np.mean(np.any(h_cpu != fr.x, axis=1)))
    ok_rate = float(np.mean(ok_cpu))

    # end to end through the host-buffer entry point, pinned memory
    pin_llr = torch.from_numpy(fr.llr).pin_memory()
    pin_syn = torch.from_numpy(fr.syn).pin_memory()
    pin_hard = torch.empty((K_FRAMES, n), dtype=torch.uint8).pin_memory()
    pin_post = torch.empty((K_FRAMES, n), dtype=torch.float32).pin_memory()
    pin_ok = torch.empty((K_FRAMES,), dtype=torch.uint8).pin_memory()
    # all three outputs of the call cross back: hard decisions, posteriors, ok flags
    host_out = (pin_hard.numpy(), pin_post.numpy(), pin_ok.numpy())
    q.decode_host(qc, pin_llr.numpy(), pin_syn.numpy(), ITERS, msg=args.msg,
                  stream=stream, out=host_out, l2_persist=args.l2_persist == "on",
                  kernel=args.kernel, cluster=args.cluster)
    # each call timed on its own (the call is synchronous); the median is the
    # figure, every call's time is reported beside it
    e2e_steps = 5
    barrier()
    e2e_each = []
    for _ in range(e2e_steps):
        t0 = time.perf_counter()
        q.decode_host(qc, pin_llr.numpy(), pin_syn.numpy(), ITERS, msg=args.msg,
                      stream=stream, out=host_out, l2_persist=args.l2_persist == "on",
                      kernel=args.kernel, cluster=args.cluster)
        e2e_each.append(time.perf_counter() - t0)
    e2e_s = max_over_ranks(statistics.median(e2e_each), dev)
    h2d = pin_llr.numel() * pin_llr.element_size() + pin_syn.numel() * pin_syn.element_size()
    d2h = sum(t.numel() * t.element_size() for t in (pin_hard, pin_post, pin_ok))

    # the committed ncu figure is for this workload with FP32 messages; the
    # library takes the grouped kernel for it unless --kernel frame
    kern = "frame" if args.kernel == "frame" else "group"
    traffic = profiled_traffic(kern) if args.msg == "fp32" else None
    bits = world * K_FRAMES * n
    value = job_mbit_per_s(world, K_FRAMES, n, ms * 1e-3)
    peak, peak_kind = peaks()
    algo_bytes = BYTES_PER_EDGE[args.msg] * code.edges * K_FRAMES * ITERS
    achieved = algo_bytes / (ms * 1e-3) / 1e9
    info = qc.info()
    # bytes the stateful part must move: messages and posteriors of the core
    # columns, channel LLRs of the degree-1 columns (read once per iteration)
    mbytes = 4 if args.msg == "fp32" else 2
    core_edges = info["msg_slots"] * Z
    deg1_edges = code.edges - core_edges
    state_bytes = (core_edges * (8 + 2 * mbytes) + deg1_edges * 4) * K_FRAMES * ITERS

    progress("end-to-end leg done")
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cores = os.cpu_count() or 1
        v, dt, desc = oracle_sample(code, cores)
        cpu = {"value": v, "unit": "Mbit/s", "cores": cores, "kind": "oracle", "sample": desc}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "Mbit/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if args.msg == "fp32" else f"f32 ({args.msg} messages)",
            "data": "synthetic",
            "config": {"workload": workload_name(args.msg), "K": K_FRAMES, "Z": Z, "n": n,
                       "iterations": ITERS, "snr": SNR, "msg": args.msg,
                       "l2_persist": args.l2_persist, "kernel": args.kernel,
                       "cluster": args.cluster,
                       "parallelism": f"dp{world} (frames sharded, no collective)",
                       "l2": "inputs larger than L2 (message state "
                             f"{K_FRAMES * info['msg_slots'] * Z * mbytes / 1e9:.2f} GB per GPU)"},
            "fer": fer, "ok_rate": ok_rate,
            "e2e": {"value": job_mbit_per_s(world, K_FRAMES, n, e2e_s), "unit": "Mbit/s",
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "outputs": "hard, llr_post, ok", "steps": e2e_steps, "statistic": "median",
                    "ms_each": [round(t * 1e3, 2) for t in e2e_each]},
            "gpu_launches": args.steps,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "traffic_frac": (traffic / (ms * 1e-3) / 1e9 / peak) if traffic else None,
                         "peak_source": f"{peak_kind} hbm_gbs",
                         "model": f"{BYTES_PER_EDGE[args.msg]} B per edge per frame per iteration",
                         "stateful_bytes_frac": state_bytes / (ms * 1e-3) / 1e9 / peak,
                         "kernel": "decode_group_kernel" if kern == "group" else "decode_kernel",
                         "note": "the model counts every core-posterior access as DRAM traffic; "
                                 "the L2 serves most of them, so frac can exceed 1. traffic: "
                                 "ncu-counted DRAM bytes per launch (1-pass capture, caches "
                                 "not flushed); traffic_frac: those bytes over the timed "
                                 "duration"},
            "clocks": clocks,
        }
        if cpu:
            line["cpu_baseline"] = cpu
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def run_profile(args):
    """Plain decode launches of a chosen size (no timing report); used under ncu."""
    import torch

    import paper_2004_09084_gb300 as q
    code = synth.make_code(RATE, Z)
    qc = q.Code(code.base, code.shifts, code.Z)
    fr = synth.make_frames(code, args.frames, SNR)
    dev = torch.device("cuda", 0)
    llr = torch.from_numpy(fr.llr).to(dev)
    syn = torch.from_numpy(fr.syn).to(dev)
    progress("profile case: inputs resident")
    for k in range(args.launches):
        hard, post, ok = q.decode(qc, llr, syn, args.iters, msg=args.msg,
                                  l2_persist=args.l2_persist == "on", kernel=args.kernel,
                                  cluster=args.cluster)
        torch.cuda.synchronize(dev)
        progress(f"profile case: launch {k} done")
    print(json.dumps({"profile_case": {"frames": args.frames, "iters": args.iters,
                                       "launches": args.launches, "msg": args.msg,
                                       "l2_persist": args.l2_persist,
                                       "ok_rate": float(ok.float().mean().item())}}))
    return 0


def run_report(args):
    """Secondary measurements printed as one JSON line per case (not the bench line)."""
    import torch

    import paper_2004_09084_gb300 as q
    dev = torch.device("cuda", 0)
    # the decodes use the persisting L2 window as the bench line does (--l2-persist)
    l2p = args.l2_persist == "on"

    def timed(fn, reps=3):
        fn()
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            out = fn()
        e1.record()
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) / reps, out

    if args.report == "early-stop":
        # Discussion, Table tabearly: fixed iterations against early termination
        code = synth.make_code(RATE, Z)
        qc = q.Code(code.base, code.shifts, code.Z)
        T = args.iters if args.iters != ITERS else 50
        for snr in (0.161, 0.2, 0.22, 0.25):
            fr = synth.make_frames(code, K_FRAMES, snr, first=50_000)
            llr = torch.from_numpy(fr.llr).to(dev)
            syn = torch.from_numpy(fr.syn).to(dev)
            ms_fix, (h, _, ok) = timed(lambda: q.decode(qc, llr, syn, T, l2_persist=l2p))
            fer_fix = float(np.mean(np.any(h.cpu().numpy() != fr.x, axis=1)))
            for every in (1, 5):
                ms_et, (h2, _, ok2, it) = timed(
                    lambda: q.decode_early_stop(qc, llr, syn, T, every, l2_persist=l2p))
                it = it.cpu().numpy()
                print(json.dumps({
                    "report": "early-stop", "snr": snr, "max_iterations": T, "check_every": every,
                    "fixed": {"ms": ms_fix, "mbit_s": K_FRAMES * code.n / ms_fix / 1e3, "fer": fer_fix},
                    "early": {"ms": ms_et, "mbit_s": K_FRAMES * code.n / ms_et / 1e3,
                              "fer": float(np.mean(np.any(h2.cpu().numpy() != fr.x, axis=1))),
                              "avg_iterations": float(it.mean()), "max_iterations_used": int(it.max())},
                }), flush=True)
        return 0

    if args.report == "precision":
        # 16-bit message storage: rates 0.1 / 0.05 / 0.02 at their SNRs, against the FP64 oracle
        import oracle
        # each rate at its configured SNR (where the stand-in codes do not
        # decode: FER 1) and at SNRs on their waterfall, where FER lies between
        # about 0.05 and 0.6 and the formats can differ
        plan = [("0.1", 100, [0.161, 0.20, 0.21]), ("0.05", 75, [0.076, 0.104, 0.106]),
                ("0.02", 100, [0.029, 0.08, 0.085, 0.09])]
        for rate, T, snrs in plan:
          code = synth.make_code(rate, Z)
          qc = q.Code(code.base, code.shifts, code.Z)
          for snr in snrs:
            fr = synth.make_frames(code, K_FRAMES, snr, first=60_000)
            llr = torch.from_numpy(fr.llr).to(dev)
            syn = torch.from_numpy(fr.syn).to(dev)
            _, rp, _ = oracle.decode(code.base, code.shifts, code.Z, fr.llr[:1], fr.syn[:1], 5)
            rp16 = {m: oracle.decode(code.base, code.shifts, code.Z, fr.llr[:1], fr.syn[:1], 5,
                                     msg_fmt=f)[1] for m, f in (("fp16", oracle.MSG_FP16),
                                                                ("bf16", oracle.MSG_BF16))}
            for msg in ("fp32", "fp16", "bf16"):
                ms, (h, _, ok) = timed(lambda: q.decode(qc, llr, syn, T, msg=msg, l2_persist=l2p))
                hn = h.cpu().numpy()
                _, p5, _ = q.decode(qc, llr[:1], syn[:1], 5, msg=msg)
                p5 = p5.cpu().numpy().astype(np.float64)[0]
                err = np.abs(p5 - rp[0]) / np.maximum(np.abs(rp[0]), 1.0)
                line = {
                    "report": "precision", "rate": rate, "snr": snr, "iterations": T, "msg": msg,
                    "edges": code.edges, "ms": ms, "mbit_s": K_FRAMES * code.n / ms / 1e3,
                    "fer": float(np.mean(np.any(hn != fr.x, axis=1))), "ber": float(np.mean(hn != fr.x)),
                    "ok_rate": float(ok.float().mean().item()),
                    "llr_err_vs_fp64_T5": {"max": float(err.max()), "p999": float(np.quantile(err, 0.999)),
                                           "hard_agree": float(np.mean((p5 < 0) == (rp[0] < 0)))},
                }
                if msg != "fp32":
                    # against the oracle that rounds its stored messages the same way
                    e16 = np.abs(p5 - rp16[msg][0]) / np.maximum(np.abs(rp16[msg][0]), 1.0)
                    line["llr_err_vs_fp64_rounded_T5"] = {"max": float(e16.max()),
                                                          "p999": float(np.quantile(e16, 0.999))}
                print(json.dumps(line), flush=True)
        return 0
    if args.report == "learned":
        # learned offset/scaled min-sum: train on decoder-generated frames over an
        # SNR range, then compare with plain min-sum and tanh-rule BP on held-out
        # frames.  Two training ranges: the configured one (0.15-0.17, where BP
        # itself does not converge on this stand-in code) and one where BP does
        # (0.20-0.22).
        from paper_2004_09084_gb300 import learned
        code = synth.make_code(RATE, Z)
        qc = q.Code(code.base, code.shifts, code.Z)
        T = 30
        frames, batch = args.train_frames, args.train_batch
        plain_s, plain_o = learned.init_weights(qc, T, device=dev)
        for lo, hi in ((0.15, 0.17), (0.20, 0.22)):
            gen = torch.Generator(device=dev)
            gen.manual_seed(2004)
            ws, wo = learned.init_weights(qc, T, scale=args.init_scale, device=dev)
            ws.requires_grad_()
            wo.requires_grad_()
            opt = torch.optim.Adam([ws, wo], lr=0.01)
            t0 = time.perf_counter()
            losses = []
            for step in range(max(1, frames // batch)):
                llr, syn, x = learned.make_batch(qc, batch, lo, hi, gen)
                opt.zero_grad()
                loss = learned.minsum_loss(ws, wo, qc, llr, syn, x).mean()
                loss.backward()
                opt.step()
                with torch.no_grad():
                    ws.clamp_(0.0, 2.0)
                    wo.clamp_(0.0, 5.0)
                losses.append(float(loss.item()))
            torch.cuda.synchronize(dev)
            train_s = time.perf_counter() - t0
            print(json.dumps({"report": "learned-training", "frames": frames, "batch": batch,
                              "iterations": T, "snr_range": [lo, hi], "init_scale": args.init_scale,
                              "seconds": train_s, "loss_first": losses[0],
                              "loss_last10": float(np.mean(losses[-10:]))}), flush=True)
            for snr in (0.161, 0.2, 0.22, 0.25):
                gen.manual_seed(777)
                llr, syn, x = learned.make_batch(qc, K_FRAMES, snr, snr, gen)
                res = {}
                # no L2 window here: qcmet_minsum_decode takes no options, so BP runs
                # the same way for a like-for-like time
                for name, fn in (("bp", lambda: q.decode(qc, llr, syn, T)),
                                 ("minsum", lambda: learned.decode(qc, llr, syn, plain_s, plain_o)),
                                 ("learned", lambda: learned.decode(qc, llr, syn, ws, wo))):
                    ms, (h, _, ok) = timed(fn)
                    res[name] = {"ms": ms, "mbit_s": K_FRAMES * code.n / ms / 1e3,
                                 "fer": float((h != x).any(dim=1).float().mean().item()),
                                 "ber": float((h != x).float().mean().item()),
                                 "ok_rate": float(ok.float().mean().item())}
                print(json.dumps({"report": "learned", "trained_on": [lo, hi], "snr": snr,
                                  "iterations": T, **res}), flush=True)
            if args.save_weights:
                # flat FP32 file + JSON header (learned.save_weights)
                learned.save_weights(f"{args.save_weights}_{lo}_{hi}.f32", ws, wo, code.base,
                                     code.shifts, code.Z,
                                     info={"snr_range": [lo, hi], "frames": frames,
                                           "batch": batch, "init_scale": args.init_scale})
        return 0
    if args.report == "batch":
        # mixed batch: 192 codewords across rates 0.1/0.05/0.02 and lengths
        # 1e5 / 5e5 / 1e6 (Z = 1250 / 6250 / 12500) in one graph-captured launch
        plan = [(Zl, Kl) for Zl, Kl in ((1250, 22), (6250, 21), (12500, 21))]
        frames, bits, groups = [], 0, []
        for rate in ("0.1", "0.05", "0.02"):
            for j, (Zl, Kl) in enumerate(plan):
                code = synth.make_code(rate, Zl)
                qc = q.Code(code.base, code.shifts, code.Z)
                fr = synth.make_frames(code, Kl, synth.RATE_SNR[rate], first=70_000 + 100 * j)
                llr = torch.from_numpy(fr.llr).to(dev)
                syn = torch.from_numpy(fr.syn).to(dev)
                groups.append((qc, llr, syn))
                for k in range(Kl):   # one allocation per frame keeps every row 16-byte aligned
                    frames.append((qc, llr[k].clone(), syn[k].clone()))
                bits += Kl * code.n
        T = ITERS
        for msg in ("fp16", "fp32"):
            t0 = time.perf_counter()
            b = q.Batch(frames, T, msg=msg, autotune=True)
            create_s = time.perf_counter() - t0
            ms, _ = timed(lambda: b.run())
            # the same frames as one launch per (rate, length) group
            ms_sep, _ = timed(lambda: [q.decode(qc, llr, syn, T, msg=msg, l2_persist=l2p)
                                       for qc, llr, syn in groups])
            print(json.dumps({"report": "batch", "frames": len(frames), "bits": bits, "msg": msg,
                              "iterations": T, "ms": ms, "mbit_s": bits / ms / 1e3,
                              "separate_launches_ms": ms_sep,
                              "separate_launches_mbit_s": bits / ms_sep / 1e3,
                              "create_s": create_s, "config": b.config()}), flush=True)
            b.close()
        return 0
    raise SystemExit(f"unknown report {args.report}")


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawTextHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--msg", choices=["fp32", "fp16", "bf16"], default="fp32")
    ap.add_argument("--l2-persist", choices=["on", "off"], default="on",
                    help="persisting L2 window over the core posteriors")
    ap.add_argument("--kernel", choices=["auto", "frame", "group"], default="auto",
                    help="decode kernel (QCMET_KERNEL_*)")
    ap.add_argument("--cluster", type=int, default=0,
                    help="grouped kernel: cluster size (0 = chosen by the library)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile", action="store_true",
                    help="only run --launches decodes of --frames x --iters (for ncu captures)")
    ap.add_argument("--frames", type=int, default=K_FRAMES)
    ap.add_argument("--iters", type=int, default=ITERS)
    ap.add_argument("--launches", type=int, default=2)
    ap.add_argument("--train-frames", type=int, default=10_000,
                    help="--report learned: training frames (decoder-generated)")
    ap.add_argument("--save-weights", default="",
                    help="--report learned: write the weights to <prefix>_<lo>_<hi>.f32 (+ .json)")
    ap.add_argument("--init-scale", type=float, default=0.25,
                    help="--report learned: initial min-sum scale (offsets start at 0)")
    ap.add_argument("--train-batch", type=int, default=128,
                    help="--report learned: frames per training step (one CTA per frame)")
    ap.add_argument("--report", choices=["early-stop", "precision", "learned", "batch"],
                    help="print secondary measurements instead of the bench line")
    args = ap.parse_args()
    if args.report:
        return run_report(args)
    if args.profile:
        return run_profile(args)
    if args.warmup < 3 and args.impl == "ours":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
