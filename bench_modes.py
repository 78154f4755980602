"""Measurements of the batched and served forms and of the transform kernels
(python bench.py --workload mixed | serve | wht); one JSON line each.  Inputs are synthetic: noisy all-zero
codewords over symmetric channels (a linear code's BP trajectory does not
depend on the codeword), regular (3,6) codes from the seeded generator."""
from __future__ import annotations

import json
import os
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))


def _clock_sampler():
    from bench import ClockSampler
    import torch
    return ClockSampler(torch.cuda.current_device())


def run_mixed(args):
    """12 classes (q in {4,16,64,256} x N in {256,1000,4000}), frames
    round-robin over the classes, BI-AWGN 1.5 dB, SUS, max 200 iterations:
    one persistent launch captured in a CUDA graph (kernel variants from the
    autotuner) against one gfbp_decode launch per class, and the same graph
    with the q >= 64 classes on the tensor-core transforms (FP16 hi/lo split,
    FP32 accumulation) instead of the FP32 CUDA-core transforms."""
    import torch
    from paper_cs_0605069_gb300 import gfbp, workload as W
    total = args.frames if args.frames != 4096 else 8192
    qs, Ns = (4, 16, 64, 256), (256, 1000, 4000)
    classes = [(q, N) for q in qs for N in Ns]
    per = total // len(classes)
    sig = W.ebn0_to_sigma(1.5)
    max_iter = args.max_iter or 200
    items, codes, hcodes = [], [], []
    for k, (q, N) in enumerate(classes):
        code = W.regular_code(q, N, cfg=f"mixed{q}_{N}", encodable=False)
        rng = W.rng_for(f"mixed{q}_{N}", "noise", 0)
        obs = torch.from_numpy(W.biawgn(rng, np.zeros((per, N), np.int64), code.p, sig)).cuda()
        cd = gfbp.Code.from_coo(code)
        hcodes.append(code)
        codes.append(cd)
        items.append(dict(code=cd, obs=obs, channel="awgn", param=sig))
    tuned = {}
    for it in items:
        n = min(64, int(it["obs"].shape[0]))
        tuned[f"q{it['code'].q}_N{it['code'].N}"] = gfbp.autotune(it["code"], it["obs"][:n], "awgn", sig,
                                                                 schedule="sus", max_iter=10)
    b = gfbp.Batch(items, schedule="sus", max_iter=max_iter)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        b.run(stream=s)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        b.run(stream=torch.cuda.current_stream())
    for _ in range(args.warmup):
        g.replay()
    torch.cuda.synchronize()
    clk = _clock_sampler()
    clk.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for a, z in ev:
        a.record()
        g.replay()
        z.record()
    torch.cuda.synchronize()
    clocks = clk.stop()
    ms = float(np.mean([a.elapsed_time(z) for a, z in ev]))
    symit = sum(int(o["iters"].sum().item()) * it["code"].N for o, it in zip(b.outputs, items))
    # plain: one gfbp_decode launch per class, back to back
    torch.cuda.synchronize()
    a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for it in items:
        gfbp.decode(it["code"], it["obs"], "awgn", sig, schedule="sus", max_iter=max_iter)
    z.record()
    torch.cuda.synchronize()
    plain_ms = a.elapsed_time(z)
    frames = per * len(classes)

    # the q >= 64 classes on the tensor-core route (variant numbers of gfbp_autotune)
    tensor_variant = {64: 21, 128: 22, 256: 23}
    bt = gfbp.Batch(items, schedule="sus", max_iter=max_iter)
    bt.set_variants([tensor_variant.get(it["code"].q, v) for it, v in zip(items, b.variants())])
    with torch.cuda.stream(s):
        bt.run(stream=s)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    gt = torch.cuda.CUDAGraph()
    with torch.cuda.graph(gt):
        bt.run(stream=torch.cuda.current_stream())
    for _ in range(args.warmup):
        gt.replay()
    evt = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for a, z in evt:
        a.record()
        gt.replay()
        z.record()
    torch.cuda.synchronize()
    ms_t = float(np.mean([a.elapsed_time(z) for a, z in evt]))
    agree = {}
    for (q, N), o, ot in zip(classes, b.outputs, bt.outputs):
        if q in tensor_variant:
            same = (o["x_hat"] == ot["x_hat"]).all(1) & (o["iters"] == ot["iters"])
            agree[f"q{q}_N{N}"] = {"same_decisions_and_iters": float(same.float().mean().item()),
                                   "converged_fp32": float(o["converged"].float().mean().item()),
                                   "converged_tensor": float(ot["converged"].float().mean().item())}
    tensor = {"ms_per_step": ms_t, "value": frames / (ms_t / 1e3), "variants": dict(zip([f"q{q}_N{N}" for q, N in classes],
                                                                                    bt.variants())),
              "vs_fp32_transforms": agree,
              "posterior_accuracy": "both routes within 1e-4 posterior max-abs of the FP64 oracle per iteration "
                                    "(tests/test_gpu_parity.py lock-step)"}
    line = {"metric": "decoded frames/s, mixed (q, N) batch in one persistent graph-captured launch", "workload": "mixed",
            "value": frames / (ms / 1e3), "unit": "frames/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "dtype": "f32",
            "data": "synthetic (noisy all-zero codewords)",
            "config": {"classes": [f"q{q}_N{N}" for q, N in classes], "frames": frames, "schedule": "sus",
                       "channel": "BI-AWGN Eb/N0 1.5 dB", "max_iter": max_iter, "graph": True},
            "sym_iter_per_s": symit / (ms / 1e3), "variants": dict(zip([f"q{q}_N{N}" for q, N in classes],
                                                                       b.variants())),
            "autotuned": tuned, "plain_per_class_ms": plain_ms, "tensor_core_transforms": tensor,
            "mean_iters": {f"q{q}_N{N}": float(o["iters"].float().mean().item())
                           for (q, N), o in zip(classes, b.outputs)},
            "clocks": clocks}
    print(json.dumps(line), flush=True)


def run_serve(args):
    """Poisson arrivals of single-frame requests: q in {2,16,256}, N uniform in
    {128, 256, ..., 8192} (a pool of 8 lengths per field), channel uniform in
    {BSC 0.05, BEC 0.35, BI-AWGN 1.5 dB}, i.i.d. or Markov (self-transition
    0.8) prior with probability 1/2, SUS, max 200 iterations, 40 GB pool;
    offered load swept as fractions of the measured saturation throughput."""
    import torch
    from paper_cs_0605069_gb300 import gfbp, workload as W
    rng = np.random.default_rng(0)
    Ns = (128, 256, 512, 1024, 2048, 4096, 6144, 8192)
    pool = {}
    for q in (2, 16, 256):
        for N in Ns:
            pool[(q, N)] = (gfbp.Code.from_coo(W.regular_code(q, N, cfg=f"serve{q}_{N}", encodable=False)), q, N)
    chans = (("bsc", 0.05), ("bec", 0.35), ("awgn", W.ebn0_to_sigma(1.5)))

    def make_req():
        q = int(rng.choice((2, 16, 256)))
        N = int(rng.choice(Ns))
        ch, prm = chans[int(rng.integers(3))]
        cd = pool[(q, N)][0]
        p = q.bit_length() - 1
        x = np.zeros((1, N), np.int64)
        if ch == "bsc":
            obs = W.bsc(rng, x, p, prm)
        elif ch == "bec":
            obs = W.bec(rng, x, p, prm)
        else:
            obs = W.biawgn(rng, x, p, prm)
        markov = rng.random() < 0.5
        T = W.self_transition_chain(q, 0.8) if markov else None
        return dict(code=cd, obs=obs, channel=ch, param=prm, T=T, K=N // 2 if markov else 0, N=N)

    budget = 40 << 30
    srv = gfbp.Server(budget, round_iters=4)
    # saturation: a burst of requests, completed frames per second
    burst = [make_req() for _ in range(400)]
    t0 = time.perf_counter()
    ids = [srv.submit(r["code"], r["obs"], r["channel"], r["param"], T=r["T"], K=r["K"], schedule="sus",
                      max_iter=200) for r in burst]
    for i in ids:
        srv.wait(i, timeout_s=600)
    sat = len(burst) / (time.perf_counter() - t0)
    sweep = []
    clk = _clock_sampler()
    clk.start()
    for frac in (0.1, 0.3, 0.5, 0.8, 1.0, 1.2):
        lam = frac * sat
        reqs, lat = [], []
        t_end = time.perf_counter() + args.duration
        submitted = []
        t_next = time.perf_counter()
        while time.perf_counter() < t_end:
            t_next += rng.exponential(1.0 / lam)
            while time.perf_counter() < t_next:
                time.sleep(min(0.0005, max(0.0, t_next - time.perf_counter())))
            r = make_req()
            submitted.append((srv.submit(r["code"], r["obs"], r["channel"], r["param"], T=r["T"], K=r["K"],
                                         schedule="sus", max_iter=200), r["N"]))
        t_sub = time.perf_counter()
        for i, _N in submitted:
            lat.append(srv.wait(i, timeout_s=600)["latency_us"] / 1e3)
        elapsed = time.perf_counter() - (t_end - args.duration)
        sweep.append({"offered_frac": frac, "offered_per_s": lam, "requests": len(submitted),
                      "frames_per_s": len(submitted) / elapsed, "p50_ms": float(np.percentile(lat, 50)),
                      "p99_ms": float(np.percentile(lat, 99)),
                      "symbols_per_s": sum(N for _, N in submitted) / elapsed})
    clocks = clk.stop()
    st = srv.stats()
    srv.close()
    line = {"metric": "served frames/s and p50/p99 latency vs offered load", "workload": "serve",
            "value": max(x["frames_per_s"] for x in sweep), "unit": "frames/s", "n_gpus": 1,
            "higher_is_better": True, "dtype": "f32", "data": "synthetic (noisy all-zero codewords)",
            "config": {"q": [2, 16, 256], "N": list(Ns), "channels": ["bsc 0.05", "bec 0.35", "awgn 1.5 dB"],
                       "prior": "iid or markov(0.8), p=1/2", "schedule": "sus", "max_iter": 200,
                       "budget_bytes": budget, "round_iters": 4, "duration_s": args.duration},
            "saturation_frames_per_s": sat, "sweep": sweep, "server": st, "clocks": clocks}
    print(json.dumps(line), flush=True)


def run_wht(args):
    """gfbp_wht on 2 GB of q-vectors per q in {64, 128, 256}: FP32 butterflies
    on the CUDA cores against the FP16 hi/lo contraction on the tensor cores
    (bytes moved: the vectors read once and written once; tensor flops: 2 q^2
    per vector per FP16 part)."""
    import torch
    from bench import ClockSampler, measured_peaks
    from paper_cs_0605069_gb300 import gfbp
    torch.cuda.set_device(0)
    peaks = measured_peaks()
    res = {}
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    for q in (64, 128, 256):
        n = (2 << 30) // (4 * q)
        g = torch.Generator(device="cuda").manual_seed(q)
        x = torch.rand((n, q), device="cuda", generator=g)
        x /= x.sum(1, keepdim=True)
        y = torch.empty_like(x)
        row = {}
        for m in ("simt", "tensor"):
            for _ in range(max(args.warmup, 3)):
                gfbp.wht(x, m, out=y)
            ts = []
            for _ in range(args.steps):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record()
                gfbp.wht(x, m, out=y)
                b.record()
                torch.cuda.synchronize()
                ts.append(a.elapsed_time(b))
            ms = float(np.median(ts))
            gbs = 2 * x.numel() * 4 / (ms / 1e3) / 1e9
            row[m] = {"ms": ms, "vectors_per_s": n / (ms / 1e3), "GB_s": gbs,
                      "frac_hbm": gbs / peaks["hbm_gbs"] if peaks else None}
            if m == "tensor":
                tf = 2 * 2 * n * q * q / (ms / 1e3) / 1e12
                row[m]["tensor_TFLOP_s"] = tf
        ys = gfbp.wht(x[:4096], "simt")
        yt = gfbp.wht(x[:4096], "tensor")
        row["max_abs_diff_tensor_vs_simt"] = float((ys - yt).abs().max().item())
        res[f"q{q}"] = row
        del x, y
    cl = clocks.stop()
    line = {"metric": "Walsh-Hadamard transforms/s, FP32 CUDA-core butterflies vs FP16 hi/lo tensor cores",
            "workload": "wht", "unit": "vectors/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "value": res["q256"]["tensor"]["vectors_per_s"], "higher_is_better": True, "dtype": "f32 (tensor: f16x2 in, f32 acc)",
            "data": "synthetic probability vectors, 2 GB per q (above L2)", "config": {"bytes_per_q": 2 << 30},
            "per_q": res, "clocks": cl}
    print(json.dumps(line))
