"""Device-side anomaly status words.

* zero_sums: per frame, the normalisations of r (Eq. 3), q (Eq. 4) and Q
  (Eq. 5) whose sum vanished and that fell back to the uniform vector,
  against the FP64 oracle's count on inputs whose evidence contradicts
  itself.  On the BEC every message is uniform over a coset of a subgroup of
  GF(q)'s additive group (its entries are 0 or one power of two), so FP32 and
  FP64 compute the same numbers on either check-node route and the counts,
  decisions and iteration counts must be equal, not merely close.
* Bounded device waits: each wait the kernels use is run on a condition that
  never comes true (gfbp_wait_selftest); it must give up within its bound,
  report a timeout status, and leave the context usable.
"""
import time

import numpy as np
import pytest

from tests.parity_util import to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_cs_0605069_gb300 import gfbp
    gfbp.lib()
    return torch


def _contradicting(q, F=16, N=96, eps=0.25):
    """Codewords through a BEC (bits erased with probability eps), decoded
    against a syndrome that three checks of every other frame contradict."""
    from paper_cs_0605069_gb300 import workload as W
    code = W.regular_code(q, N, cfg=f"zero_sums_q{q}")
    rng = np.random.default_rng(100 + q)
    s = rng.integers(0, q, size=(F, code.K))
    x = W.encode(code, s)
    obs = W.bec(rng, x, W.log2q(q), eps)
    z = code.syndrome(x).astype(np.uint8)
    for f in range(0, F, 2):
        rows = rng.choice(code.M, 3, replace=False)
        z[f, rows] ^= rng.integers(1, q, size=3).astype(np.uint8)
    return code, obs, z


# (schedule, layout, partials, q): each schedule kernel family at least once —
# frame-resident (AUTO at 16 frames, q <= 16), thread-per-check / per-pair
# level kernels, running partials in shared memory, lane teams, and for
# q = 64 / 128 the lane-group kernels on the probability and transform routes.
CASES = [
    ("pus", "auto", "auto", 4), ("pus", "thread", "auto", 4), ("pus", "lanes", "auto", 4),
    ("sus", "auto", "auto", 4), ("sus", "thread", "fold", 4), ("sus", "thread", "running", 4),
    ("sus", "lanes", "auto", 4), ("pus", "auto", "auto", 16), ("sus", "auto", "auto", 16),
    ("sus", "thread", "fold", 16), ("pus", "auto", "auto", 64), ("sus", "auto", "auto", 64),
    ("pus", "auto", "auto", 128), ("sus", "auto", "auto", 128),
]


@pytest.mark.parametrize("schedule,layout,partials,q", CASES)
def test_zero_sum_counts_match_the_oracle(torch_cuda, oracle, schedule, layout, partials, q):
    from paper_cs_0605069_gb300 import gfbp
    code, obs, z = _contradicting(q)
    ora = oracle.decode(code, obs, "bec", 0.25, schedule, max_iter=20, syn=z)
    assert (ora["zero_sums"][1::2] == 0).all() and (ora["zero_sums"][0::2] > 0).all()
    out = gfbp.decode(gfbp.Code.from_coo(code), to_dev(obs), "bec", 0.25, schedule=schedule, max_iter=20,
                      syndrome=to_dev(z), layout=layout, partials=partials, zero_sums=True)
    np.testing.assert_array_equal(out["zero_sums"].cpu().numpy(), ora["zero_sums"])
    np.testing.assert_array_equal(out["iters"].cpu().numpy(), ora["iters"])
    np.testing.assert_array_equal(out["x_hat"].cpu().numpy(), ora["xhat"])


def test_zero_sums_are_zero_on_ordinary_frames(torch_cuda):
    """The benchmark-shaped decode (BI-AWGN, consistent syndromes) reports no
    fallback on any frame, and asking for the count changes no result."""
    import torch
    from paper_cs_0605069_gb300 import gfbp, workload as W
    b = W.make_batch("gf16_n1000_awgn", frames=64)
    cd = gfbp.Code.from_coo(b.code)
    fp = to_dev(b.param.astype(np.float32))
    for s in ("pus", "sus"):
        a = gfbp.decode(cd, to_dev(b.obs), "awgn", 0.0, schedule=s, max_iter=50, frame_param=fp, zero_sums=True)
        c = gfbp.decode(cd, to_dev(b.obs), "awgn", 0.0, schedule=s, max_iter=50, frame_param=fp)
        torch.cuda.synchronize()
        assert int(a["zero_sums"].sum()) == 0
        for k in ("x_hat", "iters", "converged"):
            assert torch.equal(a[k], c[k]), k


@pytest.mark.parametrize("which", ["mbarrier", "watermark"])
def test_bounded_waits_run_out_and_report(torch_cuda, which):
    """A wait on a condition that never comes true gives up (GFBP_ETIMEOUT,
    not completed) within a few seconds, and a decode afterwards on the same
    context gives the same results as before it."""
    import torch
    from paper_cs_0605069_gb300 import gfbp, workload as W
    b = W.make_batch("gf4_n96_bsc005", frames=32)
    cd = gfbp.Code.from_coo(b.code)
    before = gfbp.decode(cd, to_dev(b.obs), "bsc", 0.05, schedule="sus", max_iter=30)
    torch.cuda.synchronize()
    t0 = time.time()
    rc, done = gfbp.wait_selftest(which)
    dt = time.time() - t0
    print(f"{which} wait ran out after {dt:.3f} s")
    assert rc == gfbp.GFBP_ETIMEOUT and done == 0
    assert "ran out" in gfbp.last_error()
    assert dt < 30
    after = gfbp.decode(cd, to_dev(b.obs), "bsc", 0.05, schedule="sus", max_iter=30)
    torch.cuda.synchronize()
    for k in ("x_hat", "iters", "converged"):
        assert torch.equal(before[k], after[k]), k
