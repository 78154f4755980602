"""The parity bookkeeping itself, on the CPU: the oracle standing in for the
GPU must classify every frame as a match, whether a batch is compared whole
or on sampled frames (the full-size GPU test samples frames of one batch)."""
import numpy as np
import pytest


def _as_gpu(out):
    return {"x_hat": out["xhat"], "iters": out["iters"], "converged": out["conv"], "trace": out["trace_x"]}


@pytest.mark.parametrize("schedule", ["pus", "sus"])
def test_oracle_against_itself_matches_whole_and_sampled(oracle, schedule):
    from paper_cs_0605069_gb300 import workload as W
    from tests.parity_util import classify_frames, oracle_horizon
    from tests.test_gpu_parity import sampled_parity
    b = W.make_batch("gf4_n96_bsc005", frames=30)
    whole = oracle.decode(b.code, b.obs, b.channel, b.param, schedule, max_iter=b.max_iter, trace=True)
    hz = oracle_horizon(oracle, b.code, b.obs, b.channel, b.param, schedule, b.max_iter)
    kinds = classify_frames(_as_gpu(whole), whole, horizon=hz)
    assert (kinds == "match").all()
    sample = [0, 5, 17, 29]
    kinds = sampled_parity(oracle, b, b.channel, schedule, _as_gpu(whole), sample)
    assert list(kinds) == ["match"] * len(sample)
    # a planted mistake on one sampled frame (its decisions flipped from the
    # first iteration on) is caught
    bad = {k: np.array(v, copy=True) for k, v in _as_gpu(whole).items()}
    bad["trace"][17, :, :5] ^= 1
    bad["x_hat"][17, :5] ^= 1
    kinds = sampled_parity(oracle, b, b.channel, schedule, bad, sample)
    assert list(kinds) == ["match", "match", "fail", "match"]
