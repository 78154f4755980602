"""The Gauss-Seidel block prior inside SUS (a variant the paper leaves open:
each source symbol's prior re-estimated by Eq. 6 as the sweep reaches it)
against the FP64 oracle's same mode: free-running decisions, counts and flags
on Markov sources over BSC and BEC, and exact posteriors on source columns
that meet no check."""
import numpy as np
import pytest

from tests.parity_util import TIE_GAP, classify_frames, gpu_decode, oracle_horizon

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_cs_0605069_gb300 import gfbp
    gfbp.lib()
    return torch


@pytest.mark.parametrize("name,N,frames", [("gf8_n2000_markov_bsc", 400, 24), ("gf8_n2000_markov_bec", 400, 24)])
def test_gauss_seidel_free_running_against_the_oracle(torch_cuda, oracle, name, N, frames):
    from paper_cs_0605069_gb300 import gfbp, workload as W
    b = W.make_batch(name, frames=frames, N=N)
    cd = gfbp.Code.from_coo(b.code)
    kw = dict(T=b.T, K=b.K, gauss_seidel=True)
    ora = oracle.decode(b.code, b.obs, b.channel, b.param, "sus", max_iter=60, trace=True, **kw)
    hz = oracle_horizon(oracle, b.code, b.obs, b.channel, b.param, "sus", 60, **kw)
    gpu = gpu_decode(cd, b.obs, b.channel, b.param, "sus", 60, trace=True, **kw)
    kinds = classify_frames(gpu, ora, horizon=hz)
    n = {k: int((kinds == k).sum()) for k in ("match", "tie", "horizon", "fail")}
    print(f"{name} Gauss-Seidel prior: {n}")
    assert n["fail"] == 0
    assert n["horizon"] <= 0.05 * len(kinds) + 1
    # and it is a different decoder from the Jacobi reading
    jac = gpu_decode(cd, b.obs, b.channel, b.param, "sus", 60, **{k: v for k, v in kw.items() if k != "gauss_seidel"})
    assert (jac["iters"] != gpu["iters"]).any() or (jac["x_hat"] != gpu["x_hat"]).any()


def test_gauss_seidel_posteriors_on_free_source_columns(torch_cuda, oracle):
    """Source columns that meet no check: the posteriors follow the prior's
    Gauss-Seidel trajectory; device within 1e-5 of the oracle after each of
    three sweeps."""
    from paper_cs_0605069_gb300 import gfbp, workload as W
    q, K = 8, 9
    H = np.zeros((2, K + 3), np.int64)
    H[0, K:K + 2] = 1
    H[1, K + 1:K + 3] = [3, 5]
    code = W.code_from_dense(H, q)
    rng = np.random.default_rng(9)
    T = rng.random((q, q)) + 0.05
    T /= T.sum(1, keepdims=True)
    src_pos = np.array([3, 0, 7, 1, 8, 2, 6, 4, 5], np.int32)
    obs = rng.integers(0, 2, size=(4, K + 3, 3)).astype(np.float32)
    obs[:, K:] = 0.0
    cd = gfbp.Code.from_coo(code)
    for t_max in (1, 2, 3):
        ora = oracle.decode(code, obs, "bsc", 0.2, "sus", max_iter=t_max, T=T, K=K, src_pos=src_pos,
                            early_stop=False, post=True, gauss_seidel=True)
        gpu = gpu_decode(cd, obs, "bsc", 0.2, "sus", t_max, T=T, K=K, src_pos=src_pos, post=True,
                         no_early_stop=True, gauss_seidel=True)
        assert np.abs(gpu["post"] - ora["post"]).max() <= 1e-5, t_max


def test_gauss_seidel_refused_where_it_does_not_apply(torch_cuda):
    import torch
    from paper_cs_0605069_gb300 import gfbp, workload as W
    b = W.make_batch("gf8_n2000_markov_bsc", frames=2, N=200)
    cd = gfbp.Code.from_coo(b.code)
    obs = torch.from_numpy(b.obs).cuda()
    with pytest.raises(gfbp.GfbpError):
        gfbp.decode(cd, obs, "bsc", 0.08, schedule="pus", T=b.T, K=b.K, gauss_seidel=True)
