"""Throughput benchmark of GF(q) belief-propagation decoding on GB300.

One step decodes one batch of the GF(16) regular (3,6) rate-1/2 N=1000
workload over BI-AWGN (Eb/N0 1.0 / 1.5 / 2.0 dB round-robin over frames,
4096 frames, max 200 iterations, early stop) under both schedules of the
paper, PUS then SUS, with inputs resident in HBM.  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank decodes its own 4096 frames (weak
scaling, no data-path collective); the slowest rank's time is reported.
"""
from __future__ import annotations

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

METRIC = "decoded frames/s and symbol-iter/s, SUS vs PUS, at matched BER; p50/p99 latency; % HBM roofline"
WORKLOAD = "gf16_n1000_awgn"
# Algorithmic bytes per symbol-iteration (FP32 messages, d_v = 3): PUS reads and
# writes every edge message twice per iteration plus the prior (52 q bytes); SUS
# reads and writes the single stored slab once per sweep plus the prior (28 q).
ALG_BYTES_PER_SYMITER = {"pus": 52, "sus": 28}
# FP32 FMAs per symbol-iteration of the probability-domain check node (the
# route whose every entry keeps relative precision; d_v = 3, d_c = 6, M/N =
# 1/2), convolutions of q^2 FMAs: PUS runs 3 (d_c - 2) = 12 per check, M/N
# checks per symbol: 6 q^2.  SUS with running partials: d_c - 2 suffixes per
# check at the sweep start plus, at each of the d_c - 2 inner positions, one
# for r and one for the prefix: also 3 (d_c - 2) per check, 6 q^2.  SUS
# folding per visit: d_c - 2 for each of a column's 3 checks, 12 q^2.
ALG_FMA_PER_SYMITER_Q2 = {"pus": 6, "sus": 6, "sus_fold": 12}
# FP32 FMA rate: 152 SMs x 4 schedulers x 32 lanes, one FMA (2 flop) per lane
# per clock, at the sampled SM clock (2070 MHz maximum).
FP32_LANES = 152 * 4 * 32
# The kernel of each schedule on the benchmark path (layout AUTO at 4096
# frames): PUS frame-resident (a frame's messages in one CTA's shared memory),
# SUS by levels folding each check's messages per visit (with 27 frames per
# SM; up to 4 frames per SM AUTO takes the frame-resident SUS kernel).
BENCH_KERNEL = {"pus": "k_pus_res<16,256,6,4>", "sus": "k_sus_level<16,8,64,false>"}
RESIDENT_SUS_FRAMES_PER_SM = 4


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--frames", type=int, default=4096)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--schedules", default="pus,sus", help="comma list (profiling cases)")
    ap.add_argument("--max-iter", type=int, default=0, help="override the workload's max_iter (profiling cases)")
    ap.add_argument("--method", default="auto", choices=["auto", "direct", "transform"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--sus-width", type=int, default=0, help="SUS lane teams per frame (0 = automatic)")
    ap.add_argument("--layout", default="auto", choices=["auto", "lanes", "thread", "resident", "l2resident"])
    ap.add_argument("--partials", default="auto", choices=["auto", "fold", "running", "running_global"],
                    help="SUS level kernel: check messages folded per visit or carried as running partials")
    ap.add_argument("--workload", default="batch", choices=["batch", "mixed", "serve", "wht", "markov", "paper", "fig1"],
                    help="batch: the GF(16) N=1000 benchmark (default); mixed: frames of 12 (q, N) classes in one "
                         "persistent launch; serve: Poisson arrivals to the continuous-batching server")
    ap.add_argument("--duration", type=float, default=6.0, help="serve: seconds per offered load")
    ap.add_argument("--noise-scale", type=float, default=1.0, help="paper: multiplier of Table 1's noise levels")
    ap.add_argument("--wht-q", type=int, default=0, help="wht: one field size only (profiling cases)")
    ap.add_argument("--wht-mb", type=int, default=2048, help="wht: MiB of input vectors per field size")
    return ap.parse_args()


def shard_first_frame(rank: int, frames_per_rank: int) -> int:
    """Weak scaling: rank r decodes frames r*F .. r*F + F - 1 of the workload."""
    return rank * frames_per_rank


def max_over_ranks(x: float, world: int, device) -> float:
    """The slowest rank's value (an all-reduce MAX; the only collective, outside
    the timed region)."""
    if world == 1:
        return float(x)
    import torch
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_frames_per_s(frames_per_rank_step: int, world: int, ms_per_step: float) -> float:
    """Whole-job throughput: every rank's frames over the slowest rank's time."""
    return frames_per_rank_step * world / (ms_per_step / 1e3)


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def measured_peaks():
    """The measured HBM copy bandwidth and bf16 GEMM rates, or None."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    return json.load(open(path)) if os.path.exists(path) else None


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self._t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self._t:
            self._t.join(timeout=2)
        return summarise_clocks(self.lines)


def summarise_clocks(lines):
    """Median SM clock, the largest maximum clock and the throttle reasons seen
    active, from ClockSampler.FIELDS lines (csv, no header, no units)."""
    sm, mx, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for ln in lines:
        parts = [p.strip() for p in ln.split(",")]
        if len(parts) < 9:
            continue
        try:
            sm.append(float(parts[1]))
            mx.append(float(parts[2]))
        except ValueError:
            continue
        for n, v in zip(names, parts[5:9]):
            if v.lower() == "active":
                reasons.add(n)
    return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
            "reasons": sorted(reasons), "samples": len(sm)}


def source_hash() -> str:
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_cs_0605069_gb300", "csrc")
    for f in sorted(os.listdir(d)):
        if f.endswith((".cu", ".cuh")):
            h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()[:16]


def code_tokens(text: str) -> str:
    """C/C++/CUDA source without comments and with whitespace runs collapsed:
    what the compiler sees, so that an edit of comments alone keeps it."""
    out, i, n = [], 0, len(text)
    while i < n:
        c = text[i]
        if text.startswith("//", i):
            j = text.find("\n", i)
            i = n if j < 0 else j
        elif text.startswith("/*", i):
            j = text.find("*/", i + 2)
            i = n if j < 0 else j + 2
            out.append(" ")
        elif c in "\"'":
            j = i + 1
            while j < n and text[j] != c:
                j += 2 if text[j] == "\\" else 1
            out.append(text[i:j + 1])
            i = j + 1
        else:
            out.append(c)
            i += 1
    return " ".join("".join(out).split())


def files_hash(files) -> str:
    """Hash of the code (comments and layout aside) of the given source files."""
    h = hashlib.sha256()
    for f in files:
        h.update(code_tokens(open(os.path.join(ROOT, f), encoding="utf-8").read()).encode())
        h.update(b"\0")
    return h.hexdigest()[:16]


def profiled_traffic(kernel: str, symiters: float):
    """DRAM bytes of the kernel for this launch, scaled from the committed ncu
    summary when it was taken on the kernel's current source files; else None."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        t = json.load(open(path))
        ent = t.get(kernel)
        if not ent or ent.get("source_hash") != files_hash(ent["files"]):
            return None
    except (OSError, ValueError, KeyError):
        return None
    return ent["dram_bytes_per_symiter"] * symiters


def error_rates(x_hat, x, q: int, levels=(1.0, 1.5, 2.0)):
    """Frame, symbol and bit error rates of the decided words against the sent
    codewords, per noise level (frame f is at level f mod len(levels)) and
    over the batch."""
    p = q.bit_length() - 1
    x_hat = np.asarray(x_hat, np.int64)
    x = np.asarray(x, np.int64)
    sym = x_hat != x
    bits = np.zeros(x.shape, np.int64)
    d = x_hat ^ x
    for k in range(p):
        bits += (d >> k) & 1

    def rates(sel):
        if not sel.any():
            return None
        return {"fer": float(sym[sel].any(1).mean()), "ser": float(sym[sel].mean()),
                "ber": float(bits[sel].sum() / (sel.sum() * x.shape[1] * p)), "frames": int(sel.sum())}

    idx = np.arange(x.shape[0])
    out = {str(db): rates(idx % len(levels) == k) for k, db in enumerate(levels)}
    out["all"] = rates(idx >= 0)
    return out


def cpu_baseline(batch, frames: int, max_iter: int):
    """The FP64 oracle on the host cores, on the first `frames` frames."""
    from oracle import oracle as O
    threads = os.cpu_count() or 1
    t0 = time.perf_counter()
    it = 0
    for s in ("pus", "sus"):
        r = O.decode(batch.code, batch.obs[:frames], "awgn", batch.param[:frames], s, max_iter=max_iter,
                     threads=threads)
        it += int(r["iters"].sum())
    dt = time.perf_counter() - t0
    return {"value": 2 * frames / dt, "unit": "frames/s", "cores": threads, "kind": "oracle",
            "sample": f"first {frames} frames of the batch, PUS and SUS, {dt:.1f} s",
            "sym_iter_per_s": it * batch.code.N / dt}


def run_reference(args, rank, world):
    """--impl reference: the FP64 oracle as it stands, timed on the host cores."""
    if rank != 0:
        return
    from paper_cs_0605069_gb300 import workload as W
    frames = 24
    b = W.make_batch(WORKLOAD, frames=frames)
    from oracle import oracle as O
    threads = os.cpu_count() or 1
    times, its = [], []
    for k in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        it = 0
        for s in ("pus", "sus"):
            r = O.decode(b.code, b.obs, "awgn", b.param, s, max_iter=b.max_iter, threads=threads)
            it += int(r["iters"].sum())
        if k >= args.warmup:
            times.append(time.perf_counter() - t0)
            its.append(it)
    dt = float(np.mean(times))
    val = 2 * frames / dt
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "frames/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{WORKLOAD} sample of {frames} frames per step (first frames of the batch)",
                       "q": 16, "N": 1000, "code": "regular (3,6) rate 1/2", "channel": "BI-AWGN 1.0/1.5/2.0 dB",
                       "max_iter": b.max_iter, "schedules": ["pus", "sus"]},
            "cpu_baseline": {"value": val, "unit": "frames/s", "cores": threads, "kind": "oracle",
                             "sample": f"{frames} frames x 2 schedules per step"},
            "e2e": {"value": val, "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "sym_iter_per_s": float(np.mean(its)) * b.code.N / dt}
    print(json.dumps(line), flush=True)


def sus_folds(args, frames: int, sms: int = 152) -> bool:
    """Whether SUS runs the level kernel that folds each check's messages per
    visit (AUTO above RESIDENT_SUS_FRAMES_PER_SM frames per SM, or asked for)."""
    if args.partials == "fold":
        return True
    if args.layout in ("resident", "l2resident") or args.partials != "auto":
        return False
    return args.layout != "auto" or frames > RESIDENT_SUS_FRAMES_PER_SM * sms


def launches_per_decode(schedule: str, args, frames: int) -> int:
    """Kernels one gfbp_decode of the benchmark launches: the channel
    likelihoods and the schedule's kernel, plus the message initialisation
    for SUS unless a frame-resident kernel (which initialises on chip) runs."""
    if schedule == "pus":
        return 2
    resident = (args.layout in ("resident", "l2resident") or
                (args.layout == "auto" and args.partials == "auto" and not sus_folds(args, frames)))
    return 2 if resident else 3


def main():
    args = parse()
    rank, world, local = dist_info()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.workload == "mixed":
        from bench_modes import run_mixed
        run_mixed(args)
        return
    if args.workload == "serve":
        from bench_modes import run_serve
        run_serve(args)
        return
    if args.workload == "wht":
        from bench_modes import run_wht
        run_wht(args)
        return
    if args.workload == "markov":
        from bench_modes import run_markov
        run_markov(args)
        return
    if args.workload == "paper":
        from bench_modes import run_paper
        run_paper(args)
        return
    if args.workload == "fig1":
        from bench_modes import run_fig1
        run_fig1(args)
        return
    import torch
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_cs_0605069_gb300 import gfbp, workload as W

    F = args.frames
    b = W.make_batch(WORKLOAD, frames=F, first_frame=shard_first_frame(rank, F))
    code = gfbp.Code.from_coo(b.code)
    N, q = b.code.N, b.code.q
    dev = torch.device("cuda", local)
    obs = torch.from_numpy(b.obs).to(dev)
    sig = torch.from_numpy(b.param.astype(np.float32)).to(dev)
    scheds = tuple(args.schedules.split(","))
    max_iter = args.max_iter or b.max_iter
    ws = {s: torch.empty(gfbp.workspace_size(code, F, s), dtype=torch.uint8, device=dev) for s in scheds}
    outs = {s: dict(x_hat=torch.empty((F, N), dtype=torch.uint8, device=dev),
                    iters=torch.empty(F, dtype=torch.int32, device=dev),
                    converged=torch.empty(F, dtype=torch.uint8, device=dev)) for s in scheds}
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > 129 MB L2
    stream = torch.cuda.current_stream()

    def step(record=None):
        for s in scheds:
            ev = record[s] if record else None
            gfbp.decode(code, obs, "awgn", 0.0, schedule=s, max_iter=max_iter, frame_param=sig,
                        workspace=ws[s], out=outs[s], kernel_events=ev, check_method=args.method,
                        sus_width=args.sus_width, layout=args.layout, partials=args.partials)

    for _ in range(args.warmup):
        flush.fill_(1.0)
        step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = ClockSampler(local)
    clk.start()
    step_ms, kern_ms = [], {s: [] for s in scheds}
    iters = {s: [] for s in scheds}
    for _ in range(args.steps):
        flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        kev = {s: (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for s in scheds}
        e0.record(stream)
        step(kev)
        e1.record(stream)
        torch.cuda.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        for s in scheds:
            kern_ms[s].append(kev[s][0].elapsed_time(kev[s][1]))
            iters[s].append(outs[s]["iters"].cpu().numpy().copy())
    torch.cuda.synchronize()
    clocks = clk.stop()
    total_ms = max_over_ranks(float(np.sum(step_ms)), world, dev)
    if world > 1:
        torch.distributed.barrier()
    ms_per_step = total_ms / args.steps
    frames_per_step = len(scheds) * F * world
    value = job_frames_per_s(len(scheds) * F, world, ms_per_step)

    # end to end through the public API: pinned host obs in, results out, every step
    e2e = None
    if not args.no_e2e:
        host_obs = torch.from_numpy(b.obs).pin_memory()
        host_sig = torch.from_numpy(b.param.astype(np.float32)).pin_memory()
        host_out = {s: {k: torch.empty(v.shape, dtype=v.dtype).pin_memory() for k, v in outs[s].items()} for s in scheds}
        obs_d = torch.empty_like(obs)
        sig_d = torch.empty_like(sig)
        h2d = host_obs.numel() * 4 + host_sig.numel() * 4
        d2h = sum(v.numel() * v.element_size() for s in scheds for v in outs[s].values())

        def e2e_step():
            obs_d.copy_(host_obs, non_blocking=True)
            sig_d.copy_(host_sig, non_blocking=True)
            for s in scheds:
                gfbp.decode(code, obs_d, "awgn", 0.0, schedule=s, max_iter=max_iter, frame_param=sig_d,
                            workspace=ws[s], out=outs[s], check_method=args.method, sus_width=args.sus_width,
                            layout=args.layout, partials=args.partials)
                for k in outs[s]:
                    host_out[s][k].copy_(outs[s][k], non_blocking=True)

        e2e_step()
        torch.cuda.synchronize()
        e_ms = []
        for _ in range(args.steps):
            flush.fill_(1.0)
            a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            e2e_step()
            z.record(stream)
            torch.cuda.synchronize()
            e_ms.append(a.elapsed_time(z))
        em = max_over_ranks(float(np.mean(e_ms)), world, dev)
        e2e = {"value": job_frames_per_s(len(scheds) * F, world, em), "unit": "frames/s", "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h)}

    per = {}
    for s in scheds:
        it = np.stack(iters[s])
        symit = float(it.sum()) * N / args.steps
        kms = float(np.mean(kern_ms[s]))
        conv = outs[s]["converged"].cpu().numpy().astype(bool)
        last = it[-1]
        per[s] = {"kernel_ms": kms, "frames_per_s": F / (kms / 1e3), "sym_iter_per_s": symit / (kms / 1e3),
                  "mean_iters": float(it.mean()),
                  "mean_iters_converged": float(last[conv].mean()) if conv.any() else None,
                  "iters_by_ebn0_db": {str(db): float(it[:, k::3].mean()) for k, db in enumerate((1.0, 1.5, 2.0))},
                  "converged": float(conv.mean()),
                  "errors_by_ebn0_db": error_rates(outs[s]["x_hat"].cpu().numpy(), b.x, q)}
    # roofline of the dominant kernel: the FP32 FMA pipe (the probability-domain
    # check node's q^2 convolutions) and the HBM model of the paper's passes;
    # "bound" is the nearer of the two ceilings
    dom = max(scheds, key=lambda s: per[s]["kernel_ms"])
    peaks = measured_peaks()
    hbm_peak = peaks["hbm_gbs"] if peaks else 6800.0
    symit_launch = float(np.stack(iters[dom]).sum()) * N / args.steps
    secs = per[dom]["kernel_ms"] / 1e3
    hbm_gbs = ALG_BYTES_PER_SYMITER[dom] * q * symit_launch / secs / 1e9
    sm_mhz = (clocks or {}).get("sm_mhz") or 2070.0
    alu_peak = FP32_LANES * 2 * sm_mhz * 1e6 / 1e12
    fma_key = "sus_fold" if dom == "sus" and sus_folds(args, F) else dom
    alu_tf = 2 * ALG_FMA_PER_SYMITER_Q2[fma_key] * q * q * symit_launch / secs / 1e12
    kernel = (BENCH_KERNEL[dom] if args.layout == "auto" and args.method == "auto" and args.partials == "auto"
              and not (dom == "sus" and not sus_folds(args, F)) else None)
    traffic = profiled_traffic(kernel, symit_launch) if kernel else None
    hbm = {"achieved": hbm_gbs, "peak": hbm_peak, "unit": "GB/s", "frac": hbm_gbs / hbm_peak,
           "peak_source": "measured" if peaks else "fallback",
           "algorithmic_bytes_per_symiter": ALG_BYTES_PER_SYMITER[dom] * q}
    alu = {"achieved": alu_tf, "peak": alu_peak, "unit": "TFLOP/s", "frac": alu_tf / alu_peak,
           "peak_source": f"derived: {FP32_LANES} FP32 lanes x 2 flop x {sm_mhz:.0f} MHz (sampled SM clock)",
           "algorithmic_flops_per_symiter": 2 * ALG_FMA_PER_SYMITER_Q2[fma_key] * q * q}
    # headline: the HBM roofline of the method's algorithmic bytes per
    # symbol-iteration; the FP32 FMA figure of the same launch beside it
    roof = {"bound": "hbm", **hbm, "traffic": traffic, "kernel": kernel or f"{dom} ({args.layout}/{args.method})",
            "alu_model": alu}
    gpu_launches = args.steps * sum(launches_per_decode(s, args, F) for s in scheds)

    line = {"metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "q": q, "N": N, "M": b.code.M, "code": "regular (3,6) rate 1/2",
                       "channel": "BI-AWGN, Eb/N0 1.0/1.5/2.0 dB round-robin", "frames_per_gpu": F,
                       "max_iter": max_iter, "schedules": list(scheds), "check_method": args.method,
                       "layout": args.layout, "sus_width": args.sus_width, "sus_partials": args.partials,
                       "l2": "flushed between steps (256 MB write)",
                       "parallelism": f"frames sharded over {world} GPU(s), no collective"},
            "sym_iter_per_s": sum(per[s]["sym_iter_per_s"] for s in scheds) / len(scheds),
            **{s: per[s] for s in scheds},
            "sus_pus_iteration_ratio": (per["sus"]["mean_iters"] / per["pus"]["mean_iters"]
                                        if len(scheds) == 2 else None),
            "latency_ms": {f"batch_{s}": per[s]["kernel_ms"] for s in scheds},
            "roofline": roof, "clocks": clocks, "gpu_launches": gpu_launches, "e2e": e2e}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(b, 96, max_iter)
    if rank == 0:
        print(json.dumps(line), flush=True)
    code.close()
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
