"""gfbp_decode_noalloc: decoding for callers that cannot allocate device
memory on their decode path (its scratch is a static device array inside the
library).  Two calls in a row, through the C ABI, must give what gfbp_decode
gives on the same inputs: identical decisions, counts and flags, posteriors
within the lock-step tolerance.  The second call runs on the scratch the first
one left behind, with a different batch and schedule."""
import numpy as np
import pytest

from tests.parity_util import LOCKSTEP_ATOL

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_cs_0605069_gb300 import gfbp, workload as W
    return torch, gfbp, W


def _check_same(torch, a, b):
    torch.cuda.synchronize()
    for k in ("x_hat", "iters", "converged"):
        assert torch.equal(a[k], b[k]), k
    err = (a["post"] - b["post"]).abs().max().item()
    assert err <= LOCKSTEP_ATOL, err


def test_noalloc_matches_decode_on_two_calls(env):
    torch, gfbp, W = env
    cases = [("gf4_n96_bsc005", 200, "pus", 60), ("gf16_n1000_awgn", 24, "sus", 200)]
    for name, frames, sched, max_iter in cases:
        b = W.make_batch(name, frames=frames, first_frame=7)
        code = gfbp.Code.from_coo(b.code)
        obs = torch.from_numpy(b.obs).cuda()
        fp = torch.from_numpy(b.param.astype(np.float32)).cuda()
        ref = gfbp.decode(code, obs, b.channel, 0.0, schedule=sched, max_iter=max_iter, frame_param=fp, post=True)
        got = gfbp.decode_noalloc(code, obs, b.channel, 0.0, schedule=sched, max_iter=max_iter, frame_param=fp,
                                  post=True)
        _check_same(torch, ref, got)
        code.close()


def test_noalloc_rejects_batches_beyond_the_static_scratch(env):
    torch, gfbp, W = env
    b = W.make_batch("gf16_n1000_awgn", frames=1)
    code = gfbp.Code.from_coo(b.code)
    big = torch.zeros((4096, b.code.N, 4), dtype=torch.float32, device="cuda")
    with pytest.raises(gfbp.GfbpError) as e:
        gfbp.decode_noalloc(code, big, "awgn", 0.8)
    assert e.value.status == gfbp.GFBP_EINVAL and "static" in str(e.value)
    code.close()


def test_noalloc_refuses_partials_that_allocate(env):
    torch, gfbp, W = env
    b = W.make_batch("gf16_n1000_awgn", frames=2)
    code = gfbp.Code.from_coo(b.code)
    obs = torch.from_numpy(b.obs).cuda()
    with pytest.raises(gfbp.GfbpError) as e:
        gfbp.decode_noalloc(code, obs, "awgn", 0.8, schedule="sus", partials="running_global")
    assert e.value.status == gfbp.GFBP_EINVAL
    code.close()
