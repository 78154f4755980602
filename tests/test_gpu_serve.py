"""Serving (continuous batching): every request decodes to exactly what it
decodes to alone, whatever else is resident when it arrives; admission by
footprint, bounded waits and draining."""
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


def _requests(W, n=18, seed=0):
    """Mixed requests: q in {2, 4, 16, 64, 256}, uneven N, BSC / BEC /
    BI-AWGN, i.i.d. or Markov prior, SUS or PUS."""
    rng = np.random.default_rng(seed)
    codes = {}
    reqs = []
    for k in range(n):
        q = [2, 4, 16, 64, 256][k % 5]
        N = [48, 96, 144][(k // 5) % 3]
        if (q, N) not in codes:
            codes[(q, N)] = W.regular_code(q, N, cfg=f"serve{q}_{N}", encodable=q <= 16)
        code = codes[(q, N)]
        F = 1 + k % 3
        ch = ["bsc", "bec", "awgn"][k % 3]
        markov = (k % 4 == 1) and code.enc is not None
        T = W.self_transition_chain(q, 0.8) if markov else None
        if code.enc is not None:
            src = W.markov_source(rng.random((F, code.K)), T) if markov else rng.integers(0, q, size=(F, code.K))
            x = W.encode(code, src)
        else:
            x = np.zeros((F, N), np.int64)
        p = code.p
        if ch == "bsc":
            obs, param = W.bsc(rng, x, p, 0.05), 0.05
        elif ch == "bec":
            obs, param = W.bec(rng, x, p, 0.3), 0.3
        else:
            param = W.ebn0_to_sigma(2.0)
            obs = W.biawgn(rng, x, p, param)
        reqs.append(dict(code=code, obs=obs, channel=ch, param=param, T=T, K=code.K if markov else 0,
                         schedule="sus" if k % 2 == 0 else "pus", max_iter=[20, 40][k % 2]))
    return reqs


def _alone(torch, gfbp, dev_codes, r):
    cd = dev_codes[id(r["code"])]
    # served requests run the batch kernels: for SUS with q <= 16 the level
    # kernel folding a check's messages per visit (decode alone with FOLD)
    kw = dict(partials="fold") if r["schedule"] == "sus" and r["code"].q <= 16 else {}
    out = gfbp.decode(cd, torch.from_numpy(r["obs"]).cuda(), r["channel"], r["param"], schedule=r["schedule"],
                      max_iter=r["max_iter"], T=r["T"], K=r["K"], **kw)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


def test_each_request_decodes_as_alone_while_others_run(env):
    torch, gfbp, W = env
    reqs = _requests(W)
    dev_codes = {}
    for r in reqs:
        if id(r["code"]) not in dev_codes:
            dev_codes[id(r["code"])] = gfbp.Code.from_coo(r["code"])
    srv = gfbp.Server(1 << 30, round_iters=4)
    ids = []
    for r in reqs[:9]:
        ids.append(srv.submit(dev_codes[id(r["code"])], r["obs"], r["channel"], r["param"], T=r["T"], K=r["K"],
                              schedule=r["schedule"], max_iter=r["max_iter"]))
    first = srv.wait(ids[0])
    for r in reqs[9:]:                        # these arrive while the first ones are resident
        ids.append(srv.submit(dev_codes[id(r["code"])], r["obs"], r["channel"], r["param"], T=r["T"], K=r["K"],
                              schedule=r["schedule"], max_iter=r["max_iter"]))
    results = [first] + [srv.wait(i) for i in ids[1:]]
    st = srv.stats()
    srv.close()
    assert st["completed"] == len(reqs) and st["peak_resident"] >= 2
    for r, res in zip(reqs, results):
        ref = _alone(torch, gfbp, dev_codes, r)
        for k in ("x_hat", "iters", "converged"):
            np.testing.assert_array_equal(res[k], ref[k], err_msg=f"q={r['code'].q} {r['schedule']} {k}")
        assert res["latency_us"] > 0 and res["rounds"] >= 1


def test_heavy_and_light_lanes_decode_as_alone(env):
    """Requests whose iteration costs eight GF(16), N = 1000 frame-iterations
    or more (here GF(256), N = 384 and GF(64), N = 1000) run in their own lane
    of rounds, beside the light ones: every result is still what the request
    decodes to alone, for requests in both lanes arriving while others run."""
    torch, gfbp, W = env
    rng = np.random.default_rng(11)
    heavy = [W.regular_code(256, 384, cfg="serve_heavy_256", encodable=False),
             W.regular_code(64, 1000, cfg="serve_heavy_64", encodable=False)]
    light = [W.regular_code(4, 96, cfg="serve_light_4", encodable=False),
             W.regular_code(16, 96, cfg="serve_light_16", encodable=False)]
    reqs = []
    for k in range(12):
        code = heavy[(k // 3) % 2] if k % 3 == 0 else light[k % 2]
        F = 1 + k % 2
        x = np.zeros((F, code.N), np.int64)
        sig = W.ebn0_to_sigma(2.0)
        reqs.append(dict(code=code, obs=W.biawgn(rng, x, code.p, sig), channel="awgn", param=sig, T=None, K=0,
                         schedule="sus" if k % 2 == 0 else "pus", max_iter=[30, 60][k % 2]))
    dev_codes = {}
    for r in reqs:
        if id(r["code"]) not in dev_codes:
            dev_codes[id(r["code"])] = gfbp.Code.from_coo(r["code"])
    srv = gfbp.Server(1 << 30, round_iters=4)
    ids = [srv.submit(dev_codes[id(r["code"])], r["obs"], r["channel"], r["param"], schedule=r["schedule"],
                      max_iter=r["max_iter"]) for r in reqs[:6]]
    first = srv.wait(ids[1])                  # a light request, while the heavy ones run
    ids += [srv.submit(dev_codes[id(r["code"])], r["obs"], r["channel"], r["param"], schedule=r["schedule"],
                       max_iter=r["max_iter"]) for r in reqs[6:]]
    results = {i: srv.wait(i) for i in ids if i != ids[1]}
    results[ids[1]] = first
    st = srv.stats()
    srv.close()
    assert st["completed"] == len(reqs)
    for r, i in zip(reqs, ids):
        ref = _alone(torch, gfbp, dev_codes, r)
        for k in ("x_hat", "iters", "converged"):
            np.testing.assert_array_equal(results[i][k], ref[k], err_msg=f"q={r['code'].q} N={r['code'].N} "
                                                                          f"{r['schedule']} {k}")


def test_served_requests_against_the_oracle(env, oracle):
    """Each served request (mixed q, channels, priors, schedules, admitted while
    others are resident) against the FP64 oracle's decode of it (Sec. 2):
    identical decisions, counts and flags except tie and horizon frames."""
    from tests.parity_util import classify_final, oracle_horizon
    torch, gfbp, W = env
    reqs = _requests(W, n=20, seed=5)
    dev_codes = {}
    for r in reqs:
        if id(r["code"]) not in dev_codes:
            dev_codes[id(r["code"])] = gfbp.Code.from_coo(r["code"])
    srv = gfbp.Server(1 << 30, round_iters=3)
    ids = [srv.submit(dev_codes[id(r["code"])], r["obs"], r["channel"], r["param"], T=r["T"], K=r["K"],
                      schedule=r["schedule"], max_iter=r["max_iter"]) for r in reqs]
    results = [srv.wait(i) for i in ids]
    srv.close()
    total = {"match": 0, "tie": 0, "horizon": 0, "fail": 0}
    for r, res in zip(reqs, results):
        kw = dict(T=r["T"], K=r["K"]) if r["T"] is not None else {}
        ora = oracle.decode(r["code"], r["obs"], r["channel"], r["param"], r["schedule"], max_iter=r["max_iter"],
                            trace=True, **kw)
        hz = oracle_horizon(oracle, r["code"], r["obs"], r["channel"], r["param"], r["schedule"], r["max_iter"],
                            **kw)
        kinds = classify_final(res, ora, horizon=hz)
        for k in total:
            total[k] += int((kinds == k).sum())
        assert not (kinds == "fail").any(), (r["code"].q, r["schedule"], r["channel"], kinds)
    print(f"served requests against the oracle: {total}")
    assert total["horizon"] <= 0.05 * sum(total.values()) + 1


def test_admission_budget_timeouts_and_drain(env):
    torch, gfbp, W = env
    code = W.regular_code(16, 96, cfg="serve-budget")
    cd = gfbp.Code.from_coo(code)
    rng = np.random.default_rng(1)
    obs = W.biawgn(rng, np.zeros((4, 96), np.int64), 4, W.ebn0_to_sigma(1.0))
    srv = gfbp.Server(1 << 20, round_iters=1)          # 1 MiB: room for a few frames only
    with pytest.raises(gfbp.GfbpError) as e:
        srv.submit(cd, np.zeros((64, 96, 4), np.float32), "awgn", 0.8)
    assert e.value.status == gfbp.GFBP_EINVAL and "budget" in str(e.value)
    ids = [srv.submit(cd, obs, "awgn", W.ebn0_to_sigma(1.0), max_iter=200) for _ in range(6)]
    with pytest.raises(gfbp.GfbpError) as e:
        srv.wait(ids[-1], timeout_s=0.0)
    assert e.value.status == gfbp.GFBP_ETIMEOUT
    srv.drain()
    with pytest.raises(gfbp.GfbpError) as e:
        srv.submit(cd, obs, "awgn", 0.8)
    assert e.value.status == gfbp.GFBP_EBUSY
    outs = [srv.wait(i, timeout_s=5.0) for i in ids]
    assert all(o["iters"].max() <= 200 for o in outs)
    st = srv.stats()
    assert st["peak_bytes"] <= (1 << 20) and st["completed"] == 6
    srv.close()
