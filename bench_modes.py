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
    # plain: one gfbp_decode launch per class, back to back (each also timed alone)
    torch.cuda.synchronize()
    a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    cls_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in items]
    a.record()
    for it, (c0, c1) in zip(items, cls_ev):
        c0.record()
        gfbp.decode(it["code"], it["obs"], "awgn", sig, schedule="sus", max_iter=max_iter)
        c1.record()
    z.record()
    torch.cuda.synchronize()
    plain_ms = a.elapsed_time(z)
    plain_class_ms = {f"q{q}_N{N}": c0.elapsed_time(c1) for (q, N), (c0, c1) in zip(classes, cls_ev)}
    frames = per * len(classes)

    def graph_arm(variant_of_q):
        """The batch with the q >= 64 classes pinned to other variants: mean
        ms per graph replay and the batch (for its outputs and variants)."""
        bx = gfbp.Batch(items, schedule="sus", max_iter=max_iter)
        bx.set_variants([variant_of_q.get(it["code"].q, v) for it, v in zip(items, b.variants())])
        with torch.cuda.stream(s):
            bx.run(stream=s)
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        gx = torch.cuda.CUDAGraph()
        with torch.cuda.graph(gx):
            bx.run(stream=torch.cuda.current_stream())
        for _ in range(args.warmup):
            gx.replay()
        evx = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        for a0, z0 in evx:
            a0.record()
            gx.replay()
            z0.record()
        torch.cuda.synchronize()
        return float(np.mean([a0.elapsed_time(z0) for a0, z0 in evx])), bx

    # the q >= 64 classes on the tensor-core transforms, and on the FP32
    # transform route (the same accuracy class: both are transforms, ~1e-4),
    # variant numbers of gfbp_autotune
    tensor_variant = {64: 21, 128: 22, 256: 23}
    ms_t, bt = graph_arm(tensor_variant)
    ms_f, bf = graph_arm({64: 16, 128: 17, 256: 18})
    agree = {}
    for (q, N), o, ot in zip(classes, bf.outputs, bt.outputs):
        if q in tensor_variant:
            same = (o["x_hat"] == ot["x_hat"]).all(1) & (o["iters"] == ot["iters"])
            agree[f"q{q}_N{N}"] = {"same_decisions_and_iters": float(same.float().mean().item()),
                                   "converged_fp32": float(o["converged"].float().mean().item()),
                                   "converged_tensor": float(ot["converged"].float().mean().item())}
    tensor = {"ms_per_step": ms_t, "value": frames / (ms_t / 1e3), "variants": dict(zip([f"q{q}_N{N}" for q, N in classes],
                                                                                    bt.variants())),
              "fp32_transforms_ms_per_step": ms_f,
              "vs_fp32_transforms": agree,
              "posterior_accuracy": "both transform routes within 1e-4 posterior max-abs of the FP64 oracle per "
                                    "iteration (tests/test_gpu_parity.py lock-step)"}
    line = {"metric": "decoded frames/s, mixed (q, N) batch in one persistent graph-captured launch", "workload": "mixed",
            "value": frames / (ms / 1e3), "unit": "frames/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "dtype": "f32",
            "data": "synthetic (noisy all-zero codewords)",
            "config": {"classes": [f"q{q}_N{N}" for q, N in classes], "frames": frames, "schedule": "sus",
                       "channel": "BI-AWGN Eb/N0 1.5 dB", "max_iter": max_iter, "graph": True},
            "sym_iter_per_s": symit / (ms / 1e3), "variants": dict(zip([f"q{q}_N{N}" for q, N in classes],
                                                                       b.variants())),
            "autotuned": tuned, "plain_per_class_ms": plain_ms, "plain_class_ms": plain_class_ms,
            "tensor_core_transforms": tensor,
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


def run_markov(args):
    """The Markov-source configuration: GF(8), regular (3,6), N = 2000, a
    stationary chain with self-transition 0.8, BSC 0.08 / 0.10 (round-robin
    over frames) and BEC 0.40, 2048 frames each, PUS and SUS, max 200
    iterations, the dynamical block priors (Eqs. 6-7) on; the same frames
    decoded with the i.i.d. prior give the gain of the source model.  Each
    decode is timed alone (CUDA events around the schedule kernel, L2 flushed
    before it); symbol-iterations/s and the HBM model (PUS 52q, SUS 28q bytes
    per symbol-iteration; the block priors add 2q per source symbol and
    iteration, not counted) as in the main benchmark."""
    import torch
    from bench import ALG_BYTES_PER_SYMITER, measured_peaks
    from paper_cs_0605069_gb300 import gfbp, workload as W
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    peaks = measured_peaks()
    hbm_peak = peaks["hbm_gbs"] if peaks else 6800.0
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    clocks = _clock_sampler()
    clocks.start()
    res = {}
    F = args.frames if args.frames != 4096 else 2048
    for name in ("gf8_n2000_markov_bsc", "gf8_n2000_markov_bec"):
        b = W.make_batch(name, frames=F)
        code = gfbp.Code.from_coo(b.code)
        N, q = b.code.N, b.code.q
        obs = torch.from_numpy(b.obs).to(dev)
        fp = torch.from_numpy(b.param.astype(np.float32)).to(dev)
        levels = sorted(set(float(v) for v in b.param))
        row = {}
        for prior in ("markov", "iid"):
            pk = dict(T=b.T, K=b.K) if prior == "markov" else {}
            for sched in ("pus", "sus"):
                ws = torch.empty(gfbp.workspace_size(code, F, sched, pk.get("T"), pk.get("K", 0)), dtype=torch.uint8,
                                 device=dev)
                out = dict(x_hat=torch.empty((F, N), dtype=torch.uint8, device=dev),
                           iters=torch.empty(F, dtype=torch.int32, device=dev),
                           converged=torch.empty(F, dtype=torch.uint8, device=dev))

                def run(ev=None):
                    gfbp.decode(code, obs, b.channel, 0.0, schedule=sched, max_iter=b.max_iter, frame_param=fp,
                                workspace=ws, out=out, kernel_events=ev, **pk)

                for _ in range(max(args.warmup, 3)):
                    flush.fill_(1.0)
                    run()
                ms = []
                for _ in range(args.steps):
                    flush.fill_(1.0)
                    ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                    run(ev)
                    torch.cuda.synchronize()
                    ms.append(ev[0].elapsed_time(ev[1]))
                kms = float(np.mean(ms))
                it = out["iters"].cpu().numpy()
                conv = out["converged"].cpu().numpy().astype(bool)
                xh = out["x_hat"].cpu().numpy()
                symit = float(it.sum()) * N
                gbs = ALG_BYTES_PER_SYMITER[sched] * q * symit / (kms / 1e3) / 1e9
                by = {}
                for lv in levels:
                    sel = b.param.astype(np.float64) == lv
                    by[str(lv)] = {"ser": float((xh[sel] != b.x[sel]).mean()),
                                   "fer": float((xh[sel] != b.x[sel]).any(1).mean()),
                                   "converged": float(conv[sel].mean()), "mean_iters": float(it[sel].mean())}
                row[f"{sched}_{prior}"] = {"kernel_ms": kms, "frames_per_s": F / (kms / 1e3),
                                           "sym_iter_per_s": symit / (kms / 1e3), "mean_iters": float(it.mean()),
                                           "converged": float(conv.mean()), "hbm_model_GB_s": gbs,
                                           "hbm_model_frac": gbs / hbm_peak, "by_param": by}
        for sched in ("pus", "sus"):
            m, i = row[f"{sched}_markov"], row[f"{sched}_iid"]
            row[f"{sched}_gain"] = {"iters_iid_over_markov": i["mean_iters"] / m["mean_iters"],
                                    "converged_markov_minus_iid": m["converged"] - i["converged"]}
        row["sus_pus_iteration_ratio"] = row["sus_markov"]["mean_iters"] / row["pus_markov"]["mean_iters"]
        res[name] = row
    cl = clocks.stop()
    total_frames = 2 * 2 * F   # both channels, both schedules, Markov prior
    total_ms = sum(res[n][f"{s}_markov"]["kernel_ms"] for n in res for s in ("pus", "sus"))
    line = {"metric": "decoded frames/s, Markov source with dynamical block priors, SUS and PUS", "workload": "markov",
            "unit": "frames/s", "n_gpus": 1, "steps": args.steps, "warmup": max(args.warmup, 3),
            "value": total_frames / (total_ms / 1e3), "higher_is_better": True, "dtype": "f32",
            "data": "synthetic (seeded Markov sources, systematic encoding)",
            "config": {"q": 8, "N": 2000, "code": "regular (3,6) rate 1/2", "frames": F, "max_iter": 200,
                       "source": "stationary chain, self-transition 0.8", "l2": "flushed before every decode"},
            "per_workload": res, "clocks": cl}
    print(json.dumps(line))


def run_wht(args):
    """gfbp_wht on 2 GB of q-vectors per q in {16, ..., 256}: FP32 butterflies
    on the CUDA cores against the tensor-core form (each 16-entry chunk
    contracted with H_16 in FP16 hi/lo parts, the chunk index transformed by
    FP32 butterflies).  Bytes moved: the vectors read once and written once;
    tensor flops: 2 q 16 per vector per FP16 part."""
    import torch
    from bench import ClockSampler, measured_peaks
    from paper_cs_0605069_gb300 import gfbp
    torch.cuda.set_device(0)
    peaks = measured_peaks()
    res = {}
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    for q in ((args.wht_q,) if args.wht_q else (16, 32, 64, 128, 256)):
        n = (args.wht_mb << 20) // (4 * q)
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
                tf = 2 * 2 * n * q * 16 / (ms / 1e3) / 1e12
                row[m]["tensor_TFLOP_s"] = tf
        ys = gfbp.wht(x[:4096], "simt")
        yt = gfbp.wht(x[:4096], "tensor")
        row["max_abs_diff_tensor_vs_simt"] = float((ys - yt).abs().max().item())
        res[f"q{q}"] = row
        del x, y
    cl = clocks.stop()
    line = {"metric": "Walsh-Hadamard transforms/s, FP32 CUDA-core butterflies vs FP16 hi/lo tensor cores",
            "workload": "wht", "unit": "vectors/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "value": res[max(res, key=lambda k: int(k[1:]))]["tensor"]["vectors_per_s"], "higher_is_better": True,
            "dtype": "f32 (tensor: f16x2 in, f32 acc)",
            "data": f"synthetic probability vectors, {args.wht_mb} MiB per q", "config": {"bytes_per_q": args.wht_mb << 20},
            "per_q": res, "clocks": cl}
    print(json.dumps(line))


# Table 1 of the paper (context: its Kanter-Saad code is not given): mean
# SUS and PUS iterations, their ratio, mean and deviation of per-frame ratios,
# BER x 1e-6 (SUS, PUS); None where the table prints "<1".
TABLE1 = {
    ("bsc", 2): (0.155, 25.06, 50.73, 0.494, 0.541, 0.080, 5.28, 5.50),
    ("bsc", 4): (0.227, 28.22, 55.66, 0.507, 0.513, 0.055, 1.54, 1.53),
    ("bsc", 8): (0.230, 25.57, 50.04, 0.511, 0.518, 0.073, 1.74, 1.74),
    ("bec", 2): (0.58, 17.60, 35.07, 0.502, 0.503, 0.051, None, None),
    ("bec", 4): (0.78, 22.98, 44.54, 0.516, 0.527, 0.070, 1.9, 2.0),
    ("bec", 8): (0.76, 20.02, 40.70, 0.492, 0.498, 0.063, None, None),
    ("awgn", 2): (0.98, 20.77, 42.64, 0.487, 0.497, 0.026, None, None),
    ("awgn", 4): (1.64, 19.27, 37.28, 0.517, 0.534, 0.087, 6.2, 6.0),
    ("awgn", 8): (1.66, 16.55, 32.14, 0.515, 0.511, 0.058, 2.6, 2.5),
}


def run_paper(args):
    """The shape of Table 1: rate 1/3, N = 10000/log2 q symbols, GF(2) with an
    i.i.d. source, GF(4) with the 4S Markov chain, GF(8) with the 2S bit chain
    taken 3 bits per symbol, BSC / BEC / BI-AWGN; PUS and SUS decode the same
    frames.  The paper's Kanter-Saad code is replaced by a regular (4,6) code
    (rate 1/3), whose BP threshold lies well below the KS code's: per setting
    the noise is Table 1's scaled by the largest of 1.0, 0.9, ..., 0.3 at
    which at least 90% of 256 trial frames converge under PUS (or by
    --noise-scale when given).  With the i.i.d. source the frames are random
    words x decoded in the syndrome form H x = z (Eq. 2; over GF(2) a (4,6) H
    of even column weight is never of full rank, so it has no systematic
    encoder, and an all-zero word would let ties pass as correct); with a
    Markov source the source symbols are encoded systematically.  BER counts
    all code bits (i.i.d.) or the source bits (Markov)."""
    import torch
    from paper_cs_0605069_gb300 import gfbp, workload as W
    torch.cuda.set_device(0)
    F = args.frames if args.frames != 4096 else 6000
    max_iter = args.max_iter or 500
    sizes = {2: 9999, 4: 5001, 8: 3333}
    chains = {2: None, 4: W.MARKOV_4S, 8: W.bit_chain_symbols(W.MARKOV_2S, 3)}

    def frames(code, ch, q, T, noise, n, seed):
        p = q.bit_length() - 1
        rng = W.rng_for(f"paper_{ch}_q{q}", "frames", seed)
        if T is None:
            x = rng.integers(0, q, size=(n, code.N)).astype(np.int64)
            src, K, syn = x, code.N, code.syndrome(x).astype(np.uint8)
        else:
            K = code.K
            src = W.markov_source(rng.random((n, K)), T / T.sum(1, keepdims=True))
            x, syn = W.encode(code, src), None
        if ch == "bsc":
            obs = W.bsc(rng, x, p, noise)
        elif ch == "bec":
            obs = W.bec(rng, x, p, noise)
        else:
            obs = W.biawgn(rng, x, p, noise)
        return obs, x, src, K, syn

    def decode(cd, code, ch, noise, T, obs, syn, sched):
        kw = dict(T=T, K=code.K) if T is not None else {}
        synd = torch.from_numpy(syn).cuda() if syn is not None else None
        return gfbp.decode(cd, torch.from_numpy(obs).cuda(), ch, noise, schedule=sched, max_iter=max_iter,
                           syndrome=synd, **kw)

    rows = []
    for (ch, q), tab in TABLE1.items():
        p = q.bit_length() - 1
        N = sizes[q]
        T = chains[q]
        code = W.regular_code(q, N, dv=4, dc=6, cfg=f"paper_rate13_q{q}", encodable=T is not None)
        cd = gfbp.Code.from_coo(code)
        scale = args.noise_scale if args.noise_scale != 1.0 else None
        trials = []
        if scale is None:
            for s in (1.0, 0.9, 0.8, 0.7, 0.6, 0.5, 0.4, 0.3):
                obs, x, src, K, syn = frames(code, ch, q, T, tab[0] * s, 256, 1)
                out = decode(cd, code, ch, tab[0] * s, T, obs, syn, "pus")
                conv = float(out["converged"].float().mean().item())
                trials.append({"scale": s, "converged_pus": conv})
                if conv >= 0.9:
                    scale = s
                    break
            scale = scale or 0.3
        noise = tab[0] * scale
        obs, x, src, K, syn = frames(code, ch, q, T, noise, F, 0)
        res = {}
        for sched in ("pus", "sus"):
            decode(cd, code, ch, noise, T, obs[:64], None if syn is None else syn[:64], sched)   # warm-up
            a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            out = decode(cd, code, ch, noise, T, obs, syn, sched)
            z.record()
            torch.cuda.synchronize()
            ms = a.elapsed_time(z)
            xh = out["x_hat"].cpu().numpy().astype(np.int64)
            it = out["iters"].cpu().numpy().astype(np.float64)
            sb = ((xh[:, :K] ^ src[:, :K])[..., None] >> np.arange(p)) & 1
            res[sched] = {"iters": it, "conv": out["converged"].cpu().numpy().astype(bool),
                          "ber": float(sb.mean()), "fer": float((xh != x).any(1).mean()), "ms": ms}
        ts, tp = res["sus"]["iters"], res["pus"]["iters"]
        ratio = ts / tp
        rows.append({
            "channel": ch, "q": q, "N": N, "source": "iid" if T is None else ("4S" if q == 4 else "2S bits"),
            "noise": noise, "noise_scale": scale, "scale_trials": trials, "frames": F,
            "t_sus": float(ts.mean()), "t_pus": float(tp.mean()), "ratio_of_means": float(ts.mean() / tp.mean()),
            "mean_of_ratios": float(ratio.mean()), "stdev_ratio": float(ratio.std()),
            "ber_sus": res["sus"]["ber"], "ber_pus": res["pus"]["ber"],
            "fer_sus": res["sus"]["fer"], "fer_pus": res["pus"]["fer"],
            "converged_sus": float(res["sus"]["conv"].mean()), "converged_pus": float(res["pus"]["conv"].mean()),
            "frames_per_s": {s: F / (res[s]["ms"] / 1e3) for s in ("pus", "sus")},
            "table1": {"noise": tab[0], "t_sus": tab[1], "t_pus": tab[2], "ratio_of_means": tab[3],
                       "mean_of_ratios": tab[4], "stdev_ratio": tab[5], "ber_e6": [tab[6], tab[7]]},
        })
        print(json.dumps({k: (round(v, 4) if isinstance(v, float) else v) for k, v in rows[-1].items()
                          if k not in ("frames_per_s", "table1", "scale_trials")}), flush=True)
    line = {"metric": "SUS/PUS mean iterations beside Table 1 (regular (4,6) rate-1/3 stand-in code)",
            "workload": "paper", "unit": "ratio", "value": float(np.mean([r["ratio_of_means"] for r in rows])),
            "higher_is_better": False, "n_gpus": 1, "config": {"frames": F, "max_iter": max_iter},
            "rows": rows}
    print(json.dumps(line), flush=True)


def fig1_trajectory(P0, P, iters):
    """P[f][t], t = 0..max_iter, for the Fig. 1 statistic: P0 [F] the fraction
    of symbols the channel alone decides correctly, P [F][max_iter] the
    fraction after each iteration; after a frame stops (iters [F]) its last
    iteration's value holds."""
    P = np.asarray(P, np.float64)
    F, T = P.shape
    it = np.asarray(iters, np.int64)
    last = P[np.arange(F), np.maximum(it - 1, 0)]
    P = np.where(np.arange(T)[None, :] < it[:, None], P, last[:, None])
    return np.concatenate([np.asarray(P0, np.float64)[:, None], P], 1)


def fig1_gains(Pall, iters, bins):
    """Sum and count of the gains dP = P_t - P_{t-1} over the iterations each
    frame ran, binned by the level P_{t-1} they start from (bins: edges)."""
    dP = np.diff(Pall, axis=1)
    Pprev = Pall[:, :-1]
    live = np.arange(dP.shape[1])[None, :] < np.asarray(iters)[:, None]
    nb = len(bins) - 1
    b = np.clip(np.digitize(Pprev, bins) - 1, 0, nb - 1)
    sums, cnts = np.zeros(nb), np.zeros(nb)
    np.add.at(sums, b[live], dP[live])
    np.add.at(cnts, b[live], 1)
    return sums, cnts


def run_fig1(args):
    """The statistic of Fig. 1: P = fraction of correctly decided symbols after
    an iteration, dP = its gain in that iteration; the mean gain of PUS over
    the mean gain of SUS at equal P (20 bins).  GF(8), N = 3333 symbols (9999
    bits), rate 1/3 (regular (4,6) stand-in for the KS code), the 2S bit chain
    as source (3 bits per symbol), block priors on, BSC at Table 1's f = 0.23
    scaled by --noise-scale (default 0.6, where the stand-in code decodes:
    see --workload paper).  Both schedules decode the same frames."""
    import torch
    from paper_cs_0605069_gb300 import gfbp, workload as W
    torch.cuda.set_device(0)
    F = args.frames if args.frames != 4096 else 2000
    max_iter = args.max_iter or 200
    scale = args.noise_scale if args.noise_scale != 1.0 else 0.6
    f = 0.23 * scale
    q, N, p = 8, 3333, 3
    T = W.bit_chain_symbols(W.MARKOV_2S, 3)
    code = W.regular_code(q, N, dv=4, dc=6, cfg="paper_rate13_q8")
    cd = gfbp.Code.from_coo(code)
    bins = np.linspace(0.0, 1.0, 21)
    sums = {s: np.zeros(20) for s in ("pus", "sus")}
    cnts = {s: np.zeros(20) for s in ("pus", "sus")}
    iters = {s: [] for s in ("pus", "sus")}
    chunk = 500
    for c0 in range(0, F, chunk):
        n = min(chunk, F - c0)
        rng = W.rng_for("fig1_gf8", "frames", c0)
        src = W.markov_source(rng.random((n, code.K)), T / T.sum(1, keepdims=True))
        x = W.encode(code, src)
        obs = torch.from_numpy(W.bsc(rng, x, p, f)).cuda()
        xd = torch.from_numpy(x.astype(np.uint8)).cuda()
        for sched in ("pus", "sus"):
            out = gfbp.decode(cd, obs, "bsc", f, schedule=sched, max_iter=max_iter, T=T, K=code.K, trace=True)
            tr = out["trace"]                                           # [n][max_iter][N], 255 after the stop
            it = out["iters"].long()
            iters[sched].append(it.cpu().numpy())
            P = (tr == xd[:, None, :]).float().mean(2).cpu().numpy()    # [n][max_iter]
            # P before the first iteration: the channel's own decisions
            x0 = (np.asarray(obs.cpu().numpy() > 0.5, np.int64) * (1 << np.arange(p))).sum(2)
            P0 = (x0 == x).mean(1)
            sm, cn = fig1_gains(fig1_trajectory(P0, P, it.cpu().numpy()), it.cpu().numpy(), bins)
            sums[sched] += sm
            cnts[sched] += cn
    rows = []
    for k in range(20):
        if cnts["pus"][k] > 0 and cnts["sus"][k] > 0:
            mp, ms = sums["pus"][k] / cnts["pus"][k], sums["sus"][k] / cnts["sus"][k]
            rows.append({"P": float((bins[k] + bins[k + 1]) / 2), "dP_pus": float(mp), "dP_sus": float(ms),
                         "ratio_pus_over_sus": float(mp / ms) if ms != 0 else None,
                         "iters_in_bin": [int(cnts["pus"][k]), int(cnts["sus"][k])]})
    ratios = [r["ratio_pus_over_sus"] for r in rows if r["ratio_pus_over_sus"] is not None]
    line = {"metric": "mean dP(PUS) / mean dP(SUS) at equal P (Fig. 1 statistic)", "workload": "fig1",
            "unit": "ratio", "value": float(np.median(ratios)) if ratios else None, "n_gpus": 1,
            "config": {"q": q, "N": N, "rate": "1/3 (regular (4,6))", "source": "2S bits, 3 per symbol",
                       "channel": f"BSC f={f:.4f} (Table 1 f=0.23 x {scale})", "frames": F, "max_iter": max_iter},
            "mean_iters": {s: float(np.concatenate(iters[s]).mean()) for s in iters}, "bins": rows}
    print(json.dumps(line), flush=True)
