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
               syndrome=None, trace=False, post=False, no_early_stop=False):
    import torch
    from paper_cs_0605069_gb300 import gfbp
    fp = np.asarray(param, np.float32)
    frame_param = to_dev(np.broadcast_to(fp, (obs.shape[0],)).copy()) if fp.ndim else None
    out = gfbp.decode(code_dev, to_dev(obs, torch.float32), channel=channel, param=float(fp) if fp.ndim == 0 else 0.0,
                      schedule=schedule, max_iter=max_iter, T=T, K=K, src_pos=src_pos, frame_param=frame_param,
                      punct=None if punct is None else to_dev(punct),
                      syndrome=None if syndrome is None else to_dev(syndrome), post=post, trace=trace,
                      no_early_stop=no_early_stop)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


def classify_frames(gpu, ora, gap_thr=TIE_GAP):
    """Per frame: 'match' (identical decisions, count and flag), 'tie' (every
    per-iteration hard-decision disagreement up to the earlier stop sits on a
    symbol whose oracle top-two gap <= gap_thr) or 'fail'."""
    F = len(ora["iters"])
    kinds = []
    for f in range(F):
        same = (gpu["iters"][f] == ora["iters"][f] and gpu["converged"][f] == ora["conv"][f]
                and (gpu["x_hat"][f] == ora["xhat"][f]).all())
        tmax = int(min(gpu["iters"][f], ora["iters"][f]))
        tg = gpu["trace"][f, :tmax]
        to = ora["trace_x"][f, :tmax]
        gap = ora["trace_gap"][f, :tmax]
        dis = tg != to
        if not dis.any() and same:
            kinds.append("match")
        elif dis.any() and (gap[dis] <= gap_thr).all():
            kinds.append("tie")
        elif not dis.any():
            # identical decisions up to the earlier stop but different stops
            kinds.append("fail")
        else:
            kinds.append("fail")
    return np.array(kinds)
