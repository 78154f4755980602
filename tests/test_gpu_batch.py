"""Batched decoding (one persistent launch over frames of several codes with
uneven q and N) against the FP64 oracle item by item and against gfbp_decode
of each code alone in the same kernel routine, CUDA-graph replay of a batch
run, and the autotuner.

Batch items run the level kernels that fold a check's messages per visit
(q <= 16) or the lane-group level kernels (q >= 32), and the lane-group PUS
routine; gfbp_decode's AUTO takes the frame-resident kernels for q <= 16,
whose SUS arithmetic (running partial convolutions) rounds differently, so
the bit-for-bit comparisons decode alone with partials FOLD."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_cs_0605069_gb300 import gfbp, workload as W
    return torch, gfbp, W


def _mixed_items(torch, gfbp, W, frames=24, keep_host=False):
    """Codes with q in {2, 4, 16, 64, 256} and uneven N, BI-AWGN at 1.5 dB,
    noisy all-zero or random codewords (the channel is symmetric)."""
    items, refs = [], []
    specs = [(4, 96, True), (16, 200, True), (64, 96, False), (256, 48, False), (2, 120, True)]
    for k, (q, N, enc) in enumerate(specs):
        code = W.regular_code(q, N, cfg=f"batch{q}_{N}", encodable=enc)
        rng = np.random.default_rng(k)
        x = W.encode(code, rng.integers(0, q, size=(frames, code.K))) if enc else np.zeros((frames, N), np.int64)
        sig = W.ebn0_to_sigma(1.5)
        obs = torch.from_numpy(W.biawgn(rng, x, code.p, sig)).cuda()
        cd = gfbp.Code.from_coo(code)
        items.append(dict(code=cd, obs=obs, channel="awgn", param=sig))
        if keep_host:
            items[-1]["host"] = (code, obs.cpu().numpy())
    return items


def _alone_kw(q, schedule):
    return dict(partials="fold") if schedule == "sus" and q <= 16 else {}


@pytest.mark.parametrize("schedule", ["pus", "sus"])
def test_batch_equals_each_code_alone(env, schedule):
    torch, gfbp, W = env
    items = _mixed_items(torch, gfbp, W)
    b = gfbp.Batch(items, schedule=schedule, max_iter=40)
    outs = b.run()
    torch.cuda.synchronize()
    for it, o in zip(items, outs):
        ref = gfbp.decode(it["code"], it["obs"], "awgn", it["param"], schedule=schedule, max_iter=40,
                          **_alone_kw(it["code"].q, schedule))
        torch.cuda.synchronize()
        for k in ("x_hat", "iters", "converged"):
            assert torch.equal(ref[k], o[k]), (it["code"].q, k)
    b.close()


@pytest.mark.parametrize("schedule", ["pus", "sus"])
def test_batch_items_against_the_oracle(env, oracle, schedule):
    """Every frame of every item of a mixed batch (q in {2, 4, 16, 64, 256})
    against the FP64 oracle's decode of that item (Sec. 2): identical
    decisions, counts and flags except tie and horizon frames."""
    from tests.parity_util import classify_final, oracle_horizon
    torch, gfbp, W = env
    items = _mixed_items(torch, gfbp, W, frames=24, keep_host=True)
    b = gfbp.Batch(items, schedule=schedule, max_iter=40)
    outs = b.run()
    torch.cuda.synchronize()
    for it, o in zip(items, outs):
        code, obs = it["host"]
        ora = oracle.decode(code, obs, "awgn", it["param"], schedule, max_iter=40, trace=True)
        hz = oracle_horizon(oracle, code, obs, "awgn", it["param"], schedule, 40)
        g = {k: v.cpu().numpy() for k, v in o.items()}
        kinds = classify_final(g, ora, horizon=hz)
        n = {k: int((kinds == k).sum()) for k in ("match", "tie", "horizon", "fail")}
        print(f"batch {schedule} q={code.q} N={code.N}: {n}")
        assert n["fail"] == 0, (code.q, np.nonzero(kinds == "fail")[0])
        assert n["horizon"] <= 0.05 * len(kinds) + 1
    b.close()


def test_batch_run_replays_in_a_cuda_graph(env):
    torch, gfbp, W = env
    items = _mixed_items(torch, gfbp, W, frames=16)
    b = gfbp.Batch(items, schedule="sus", max_iter=30)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        b.run(stream=s)           # warm up outside capture
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    first = [{k: v.clone() for k, v in o.items()} for o in b.outputs]
    for o in b.outputs:
        for v in o.values():
            v.zero_()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        b.run(stream=torch.cuda.current_stream())
    for rep in range(2):
        for o in b.outputs:
            for v in o.values():
                v.zero_()
        g.replay()
        torch.cuda.synchronize()
        for a, o in zip(first, b.outputs):
            for k in a:
                assert torch.equal(a[k], o[k]), k
    b.close()


def test_autotune_picks_a_valid_variant_and_batches_use_it(env):
    torch, gfbp, W = env
    b0 = W.make_batch("gf16_n1000_awgn", frames=64)
    code = gfbp.Code.from_coo(b0.code)
    obs = torch.from_numpy(b0.obs).cuda()
    fp = torch.from_numpy(b0.param.astype(np.float32)).cuda()
    v = gfbp.autotune(code, obs, "awgn", 0.0, schedule="sus", max_iter=10, frame_param=fp)
    assert v in (14, 2, 6)                  # levels, team or group: the probability route for q = 16
    b = gfbp.Batch([dict(code=code, obs=obs, channel="awgn", frame_param=fp)], schedule="sus", max_iter=30)
    assert b.variants() == [v]
    outs = b.run()
    ref = gfbp.decode(code, obs, "awgn", 0.0, schedule="sus", max_iter=30, frame_param=fp)
    torch.cuda.synchronize()
    assert torch.equal(ref["converged"], outs[0]["converged"])
    same = (ref["x_hat"] == outs[0]["x_hat"]).all(1) & (ref["iters"] == outs[0]["iters"])
    assert same.float().mean().item() > 0.95   # the team and group routes round differently
    b.close()


def test_batch_rejects_bad_items(env):
    torch, gfbp, W = env
    code = W.code_from_dense(np.array([[1, 1, 1, 1, 1, 1, 1, 1]]), 4)
    cd = gfbp.Code.from_coo(code)
    with pytest.raises(gfbp.GfbpError) as e:
        gfbp.Batch([dict(code=cd, obs=torch.zeros((2, 8, 2), device="cuda"), channel="bsc", param=0.1)])
    assert e.value.status == gfbp.GFBP_EUNSUPPORTED


# variant numbers of gfbp_autotune
TEAM = {4: 0, 8: 1, 16: 2}
GROUP_D = {2: 3, 4: 4, 8: 5, 16: 6}
GROUP_T = {32: 7, 64: 8, 128: 9, 256: 10}
LEVEL_T = {32: 15, 64: 16, 128: 17, 256: 18}
# AUTO's route: the probability route up to q = 64, the transform route above
LEVEL = {2: 11, 4: 12, 8: 13, 16: 14, 32: 24, 64: 25, 128: 17, 256: 18}


def test_batch_default_variants_are_level_schedules(env):
    torch, gfbp, W = env
    items = _mixed_items(torch, gfbp, W, frames=4)
    b = gfbp.Batch(items, schedule="sus", max_iter=5)
    assert b.variants() == [LEVEL[it["code"].q] for it in items]
    b.close()


def test_batch_with_both_kernel_families_equals_each_code_alone(env):
    """Items pinned to warp-per-frame variants (team q=4, group transform
    q=64) beside items on the level schedules (q=16, q=256, q=2): the two
    persistent kernels of one run split the frame table between them, and
    every item still equals gfbp_decode of its code alone in the same kernel
    (the team item against the lane layout)."""
    torch, gfbp, W = env
    items = _mixed_items(torch, gfbp, W)
    qs = [it["code"].q for it in items]
    pin = {4: TEAM[4], 16: LEVEL[16], 64: GROUP_T[64], 256: LEVEL[256], 2: LEVEL[2]}
    b = gfbp.Batch(items, schedule="sus", max_iter=40)
    b.set_variants([pin[q] for q in qs])
    assert b.variants() == [pin[q] for q in qs]
    outs = b.run()
    torch.cuda.synchronize()
    for it, o in zip(items, outs):
        q = it["code"].q
        kw = dict(layout="lanes") if q == 4 else _alone_kw(q, "sus")
        if q == 64:
            kw = dict(layout="lanes", check_method="transform")   # the group kernel, transform route
        ref = gfbp.decode(it["code"], it["obs"], "awgn", it["param"], schedule="sus", max_iter=40, **kw)
        torch.cuda.synchronize()
        for k in ("x_hat", "iters", "converged"):
            assert torch.equal(ref[k], o[k]), (it["code"].q, k)
    with pytest.raises(gfbp.GfbpError):
        b.set_variants([TEAM[16] for _ in qs])   # a q=16 variant for every item
    b.close()


def test_batch_tensor_route_variants_equal_decode(env):
    """Items pinned to the tensor-core route (variants 21, 23) decode as
    gfbp_decode with check_method TENSOR does, bit for bit; the other items keep
    the FP32 routes in the same run."""
    torch, gfbp, W = env
    items = _mixed_items(torch, gfbp, W, frames=12)
    qs = [it["code"].q for it in items]
    b = gfbp.Batch(items, schedule="sus", max_iter=30)
    b.set_variants([{64: 21, 256: 23}.get(q, LEVEL[q]) for q in qs])
    outs = b.run()
    torch.cuda.synchronize()
    for it, o in zip(items, outs):
        q = it["code"].q
        kw = dict(check_method="tensor") if q in (64, 256) else _alone_kw(q, "sus")
        ref = gfbp.decode(it["code"], it["obs"], "awgn", it["param"], schedule="sus", max_iter=30, **kw)
        torch.cuda.synchronize()
        for k in ("x_hat", "iters", "converged"):
            assert torch.equal(ref[k], o[k]), (q, k)
    b.close()
