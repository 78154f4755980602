"""Helpers shared by the GPU parity tests: run the CUDA library through its
Python binding and compare with the oracle."""
import numpy as np

# Tolerances: lock-step posteriors and messages, FP32 device vs FP64 oracle
# from the same state (max-abs per iteration); a hard decision whose oracle
# top-two posterior gap is at most TIE_GAP may differ (tie).
LOCKSTEP_ATOL = 1e-5
TIE_GAP = 1e-3


def to_dev(a, dtype=None):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def gpu_decode(code_dev, obs, channel, param, schedule, max_iter, T=None, K=0, src_pos=None, punct=None,
               syndrome=None, trace=False, post=False, no_early_stop=False, check_method="auto", sus_width=0,
               layout="auto", partials="auto", gauss_seidel=False):
    import torch
    from paper_cs_0605069_gb300 import gfbp
    fp = np.asarray(param, np.float32)
    frame_param = to_dev(np.broadcast_to(fp, (obs.shape[0],)).copy()) if fp.ndim else None
    out = gfbp.decode(code_dev, to_dev(obs, torch.float32), channel=channel, param=float(fp) if fp.ndim == 0 else 0.0,
                      schedule=schedule, max_iter=max_iter, T=T, K=K, src_pos=src_pos, frame_param=frame_param,
                      punct=None if punct is None else to_dev(punct),
                      syndrome=None if syndrome is None else to_dev(syndrome), post=post, trace=trace,
                      no_early_stop=no_early_stop, check_method=check_method, sus_width=sus_width,
                      layout=layout, partials=partials, gauss_seidel=gauss_seidel)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


# Relative perturbation of the channel parameter used to find each frame's
# conditioning horizon (BP past the code's threshold iterates chaotically, and
# FP32 and FP64 trajectories of such frames separate whatever the FP32
# arithmetic): the per-iteration deviation the FP32 path is held to in
# lock-step (LOCKSTEP_ATOL), so that the probes perturb at least as much as
# the device path may.  Measured on GF(4), N = 96, BSC 0.05, 1000 frames: an
# FP32 decoder left a chaotic frame's FP64 trajectory 3 iterations before
# probes at 1e-6 (and FP64 runs storing every message rounded to FP32) did;
# at 1e-5 the horizon frames are 17 of the 1000, all of them non-converging,
# against 14 at 1e-6.  The transform route, whose per-iteration deviation
# reaches 1e-4, is measured against a horizon at that scale
# (HORIZON_REL_TRANSFORM).
HORIZON_REL = LOCKSTEP_ATOL
HORIZON_REL_TRANSFORM = 1e-4


def oracle_horizon(oracle, code, obs, kind, param, schedule, max_iter, gap_thr=TIE_GAP, rel=None, draws=3, **kw):
    """Per frame, the first iteration at which the oracle's own hard decisions
    change (on a symbol with top-two gap > gap_thr) when the channel parameter
    is perturbed by a relative +rel or -rel (default HORIZON_REL), or under
    the oracle's conditioning probes (every message stored rounded to FP32,
    alone and with the likelihoods moved by one float ulp in `draws` seeded
    patterns): the earliest of them; max_iter + 1 when they never do.  Beyond
    it the frame's trajectory is not determined to FP32 precision (BP past the
    code's threshold iterates chaotically), so no FP32 result can follow it."""
    rel = HORIZON_REL if rel is None else rel
    a = oracle.decode(code, obs, kind, param, schedule, max_iter=max_iter, trace=True, early_stop=False, **kw)
    F = a["trace_x"].shape[0]
    hz = np.full(F, max_iter + 1, np.int64)
    probes = [(1.0, 0), (-1.0, 0)] + [(0.0, k) for k in range(1, draws + 2)]
    for sgn, r32 in probes:
        prm = np.asarray(param, np.float64) * (1.0 + sgn * rel)
        ob = np.asarray(obs, np.float32) * np.float32(1.0 + sgn * rel) if kind == "loglik" else obs
        b = oracle.decode(code, ob, kind, prm, schedule, max_iter=max_iter, trace=True, early_stop=False,
                          round32=r32, **kw)
        bad = (a["trace_x"] != b["trace_x"]) & (a["trace_gap"] > gap_thr)
        for f in range(F):
            t = np.nonzero(bad[f].any(1))[0]
            if t.size:
                hz[f] = min(hz[f], int(t[0]) + 1)
    return hz


def classify_frames(gpu, ora, gap_thr=TIE_GAP, horizon=None):
    """Per frame: 'match' (identical decisions, count and flag), 'tie' (every
    per-iteration hard-decision disagreement up to the earlier stop sits on a
    symbol whose oracle top-two gap <= gap_thr), 'horizon' (the frame runs past
    its conditioning horizon and the decisions agree, ties aside, before it)
    or 'fail'."""
    F = len(ora["iters"])
    kinds = []
    for f in range(F):
        same = (gpu["iters"][f] == ora["iters"][f] and gpu["converged"][f] == ora["conv"][f]
                and (gpu["x_hat"][f] == ora["xhat"][f]).all())
        tmax = int(min(gpu["iters"][f], ora["iters"][f]))
        hz = int(horizon[f]) if horizon is not None else 10 ** 9
        tcmp = min(tmax, hz - 1)
        tg = gpu["trace"][f, :tcmp]
        to = ora["trace_x"][f, :tcmp]
        gap = ora["trace_gap"][f, :tcmp]
        dis = tg != to
        clean = (not dis.any()) or (gap[dis] <= gap_thr).all()
        if same and not dis.any():
            kinds.append("match")
        elif clean and tmax < hz and dis.any():
            kinds.append("tie")
        elif clean and max(gpu["iters"][f], ora["iters"][f]) >= hz:
            kinds.append("horizon")
        else:
            kinds.append("fail")
    return np.array(kinds)


def classify_final(gpu, ora, gap_thr=TIE_GAP, horizon=None):
    """The parity classes of classify_frames for outputs without a per-iteration
    trace (batches, served requests): 'match' (identical decisions, count and
    flag), 'tie' (identical count and flag, every differing decision on a
    symbol whose oracle top-two gap after the last iteration is <= gap_thr),
    'horizon' (the frame runs past its conditioning horizon) or 'fail'.  ora
    must hold the oracle's trace (trace=True)."""
    F = len(ora["iters"])
    kinds = []
    for f in range(F):
        same = (gpu["iters"][f] == ora["iters"][f] and gpu["converged"][f] == ora["conv"][f])
        dis = gpu["x_hat"][f] != ora["xhat"][f]
        if same and not dis.any():
            kinds.append("match")
            continue
        t = int(ora["iters"][f]) - 1
        gap = ora["trace_gap"][f, t]
        hz = int(horizon[f]) if horizon is not None else 10 ** 9
        if same and (gap[dis] <= gap_thr).all():
            kinds.append("tie")
        elif max(int(gpu["iters"][f]), int(ora["iters"][f])) >= hz:
            kinds.append("horizon")
        else:
            kinds.append("fail")
    return np.array(kinds)


def fail_report(gpu, ora, hz, frames):
    """Where each failing frame first left the oracle's decisions on a firm symbol."""
    out = []
    for f in frames:
        t = int(min(gpu["iters"][f], ora["iters"][f]))
        dis = gpu["trace"][f, :t] != ora["trace_x"][f, :t]
        firm = dis & (ora["trace_gap"][f, :t] > TIE_GAP)
        it = np.nonzero(firm.any(1))[0]
        first = int(it[0]) + 1 if it.size else None
        out.append(f"frame {f}: iters gpu {gpu['iters'][f]} oracle {ora['iters'][f]}, horizon {hz[f]}, "
                   f"first firm disagreement at iteration {first}")
    return "; ".join(out)


class Batchlike:
    """The fields of a workload batch that the free-running parity check reads,
    for inputs built in a test (i.i.d. source)."""

    def __init__(self, code, obs, param, max_iter):
        self.code, self.obs, self.param, self.max_iter = code, obs, param, max_iter
        self.T, self.K = None, 0
