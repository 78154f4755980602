"""The MN form of Sec. 2 (Eqs. 1-2) end to end on the GPU against the FP64
oracle: H = [A | B], the source columns punctured and under the Markov block
prior, the noise columns under the noise prior, decoded from the syndrome
z = B r (z != 0), lock-step and free-running."""
import numpy as np
import pytest

from tests.parity_util import LOCKSTEP_ATOL, classify_frames, gpu_decode, oracle_horizon, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_cs_0605069_gb300 import gfbp
    gfbp.lib()
    return torch


def _batch(q, M=150, frames=48, f=0.01):
    """A source that stays with probability 0.95 and noise bits flipped with
    probability 0.01: nearly every frame decodes (the horizon class is for
    frames that do not; at stay 0.8, f = 0.06 the code is past its threshold
    and nearly none decode)."""
    from paper_cs_0605069_gb300 import workload as W
    return W.mn_batch(q, M, frames, f, stay=0.95, cfg=f"mn_test_{q}")


def test_mn_syndromes_are_those_of_the_received_word():
    from paper_cs_0605069_gb300 import workload as W
    b = _batch(4)
    w = np.concatenate([b.s, b.n], axis=1)
    np.testing.assert_array_equal(b.code.syndrome(w), b.z)   # H [s; n] = z (Eq. 2)
    assert (b.z != 0).any() and b.punct[:b.K].all() and not b.punct[b.K:].any()


@pytest.mark.parametrize("q", [4, 8, 16])
@pytest.mark.parametrize("schedule", ["pus", "sus"])
def test_mn_lockstep(torch_cuda, oracle, q, schedule):
    import torch
    from paper_cs_0605069_gb300 import gfbp
    b = _batch(q, frames=6, f=0.02)
    cd = gfbp.Code.from_coo(b.code)
    F = b.obs.shape[0]
    msg = oracle.initial_messages(b.code, b.obs, "bsc", b.f, T=b.T, K=b.K, punct=b.punct)
    _, pi = oracle.markov(b.T, np.full((1, q), 1.0 / q))
    prior = np.broadcast_to(pi, (F, b.K, q)).copy()
    fp = to_dev(np.full(F, b.f, np.float32))
    for it in range(6):
        ref = oracle.step(b.code, b.obs, "bsc", b.f, msg, schedule, T=b.T, K=b.K, prior=prior, punct=b.punct,
                          syn=b.z)
        m = to_dev(msg.astype(np.float32))
        out = gfbp.step(cd, to_dev(b.obs, torch.float32), m, channel="bsc", schedule=schedule, T=b.T, K=b.K,
                        prior_in=to_dev(prior.astype(np.float32)), frame_param=fp, punct=to_dev(b.punct),
                        syndrome=to_dev(b.z))
        torch.cuda.synchronize()
        assert np.abs(out["post"].cpu().numpy() - ref["post"]).max() <= LOCKSTEP_ATOL, it
        assert np.abs(out["msg"].cpu().numpy() - ref["msg"]).max() <= LOCKSTEP_ATOL, it
        assert np.abs(out["prior_out"].cpu().numpy() - ref["prior_out"]).max() <= LOCKSTEP_ATOL, it
        msg, prior = ref["msg"], ref["prior_out"]


@pytest.mark.parametrize("q", [4, 8])
@pytest.mark.parametrize("schedule", ["pus", "sus"])
def test_mn_free_running(torch_cuda, oracle, q, schedule):
    from paper_cs_0605069_gb300 import gfbp
    b = _batch(q)
    cd = gfbp.Code.from_coo(b.code)
    kw = dict(T=b.T, K=b.K, punct=b.punct, syn=b.z)
    ora = oracle.decode(b.code, b.obs, "bsc", b.f, schedule, max_iter=b.max_iter, trace=True, **kw)
    hz = oracle_horizon(oracle, b.code, b.obs, "bsc", b.f, schedule, b.max_iter, **kw)
    gpu = gpu_decode(cd, b.obs, "bsc", b.f, schedule, b.max_iter, T=b.T, K=b.K, punct=b.punct, syndrome=b.z,
                     trace=True)
    kinds = classify_frames(gpu, ora, horizon=hz)
    n = {k: int((kinds == k).sum()) for k in ("match", "tie", "horizon", "fail")}
    print(f"MN form GF({q}) {schedule}: {n}")
    assert n["fail"] == 0 and n["horizon"] <= 0.05 * len(kinds) + 1
    # converged frames recover the source word and the noise (a converged word
    # satisfies H w = z; at this noise level it is the sent one)
    ok = gpu["converged"].astype(bool)
    assert ok.mean() > 0.5
    right = (gpu["x_hat"][ok, :b.K] == b.s[ok]).all(1) & (gpu["x_hat"][ok, b.K:] == b.n[ok]).all(1)
    assert right.mean() >= 0.95
