"""GPU parity: the CUDA library (through its C ABI) against the FP64 oracle on
the same seeded inputs.

Lock-step: from the oracle's message state at iteration t, one device
iteration must give the oracle's Q (Eq. 5), q (Eq. 4) and block priors
(Eqs. 6-7) within LOCKSTEP_ATOL = 1e-5 max-abs on the default path (AUTO:
the probability-domain check node for every q).  The transform check node is
an explicit, non-default route: it keeps an absolute error of ~1e-7 of each
message's largest entry, which conflicts between checks and channel can
amplify and SUS compounds over a sweep; its tests hold it to the accuracy the
header states for it (TRANSFORM_ATOL).  Free-running: decided symbols,
iteration counts and converged flags identical on every frame except tie
frames (every disagreement on a symbol with oracle top-two gap <= TIE_GAP) and
frames that run past their conditioning horizon at FP32 rounding scale (see
parity_util.oracle_horizon); both kinds are counted and reported.
"""
import numpy as np
import pytest

from tests.parity_util import LOCKSTEP_ATOL, TIE_GAP, classify_frames, fail_report, gpu_decode, oracle_horizon, to_dev

# The transform route's stated accuracy (not the default path's bar).
TRANSFORM_ATOL = {"pus": 1e-4, "sus": 1e-3}


def _atol(method, schedule):
    return LOCKSTEP_ATOL if method == "direct" else TRANSFORM_ATOL[schedule]

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_cs_0605069_gb300 import gfbp
    gfbp.lib()
    return torch


def _workload(name, frames, N=None):
    from paper_cs_0605069_gb300 import workload as W
    return W.make_batch(name, frames=frames, N=N)


def _lockstep(torch_cuda, oracle, code, obs, kind, param, schedule, iters, T=None, K=0, atol=LOCKSTEP_ATOL,
              method="auto", layout="auto", syn=None):
    import torch
    from paper_cs_0605069_gb300 import gfbp
    cd = gfbp.Code.from_coo(code)
    F = obs.shape[0]
    msg = oracle.initial_messages(code, obs, kind, param, T=T, K=K)
    prior = None
    if T is not None:
        _, pi = oracle.markov(T, np.full((1, code.q), 1.0 / code.q))
        prior = np.broadcast_to(pi, (F, K, code.q)).copy()
    fp = to_dev(np.broadcast_to(np.asarray(param, np.float32), (F,)).copy())
    worst = 0.0
    for t in range(iters):
        ref = oracle.step(code, obs, kind, param, msg, schedule, T=T, K=K, prior=prior, syn=syn)
        m = to_dev(msg.astype(np.float32))
        out = gfbp.step(cd, to_dev(obs, torch.float32), m, channel=kind, schedule=schedule, T=T, K=K,
                        prior_in=None if prior is None else to_dev(prior.astype(np.float32)), frame_param=fp,
                        check_method=method, layout=layout, syndrome=None if syn is None else to_dev(syn))
        torch.cuda.synchronize()
        post = out["post"].cpu().numpy()
        dpost = np.abs(post - ref["post"]).max()
        dmsg = np.abs(out["msg"].cpu().numpy() - ref["msg"]).max()
        worst = max(worst, dpost, dmsg)
        assert dpost <= atol, f"iteration {t + 1}: Q max-abs {dpost}"
        assert dmsg <= atol, f"iteration {t + 1}: q max-abs {dmsg}"
        # hard decisions agree wherever the oracle's decision is not a near tie
        srt = np.sort(ref["post"], axis=2)
        gap = srt[..., -1] - srt[..., -2]
        xh = out["x_hat"].cpu().numpy()
        firm = gap > TIE_GAP
        assert (xh[firm] == ref["xhat"][firm]).all()
        if T is not None:
            dP = np.abs(out["prior_out"].cpu().numpy() - ref["prior_out"]).max()
            assert dP <= atol, f"iteration {t + 1}: block prior max-abs {dP}"
            prior = ref["prior_out"]
        msg = ref["msg"]
    return worst


METHODS = ["direct", "transform"]


@pytest.mark.parametrize("method", METHODS)
@pytest.mark.parametrize("schedule", ["pus", "sus"])
def test_lockstep_gf4_n96_bsc(torch_cuda, oracle, schedule, method):
    b = _workload("gf4_n96_bsc005", 64)
    _lockstep(torch_cuda, oracle, b.code, b.obs, "bsc", b.param, schedule, iters=10, method=method,
              atol=_atol(method, schedule))


@pytest.mark.parametrize("method", METHODS)
@pytest.mark.parametrize("schedule", ["pus", "sus"])
def test_lockstep_gf16_n1000_awgn(torch_cuda, oracle, schedule, method):
    b = _workload("gf16_n1000_awgn", 12)
    _lockstep(torch_cuda, oracle, b.code, b.obs, "awgn", b.param, schedule, iters=8, method=method,
              atol=_atol(method, schedule))


@pytest.mark.parametrize("schedule", ["pus", "sus"])
def test_lockstep_benchmark_kernels_many_frames(torch_cuda, oracle, schedule):
    """The benchmark's own kernels (AUTO at GF(16), N = 1000: the frame-resident
    kernels, whatever the frame count) with more frames than SMs, so CTAs decode
    several frames in turn: 10 iterations within 1e-5 of the oracle."""
    b = _workload("gf16_n1000_awgn", 320)
    worst = _lockstep(torch_cuda, oracle, b.code, b.obs, "awgn", b.param, schedule, iters=10)
    print(f"{schedule}: worst lock-step deviation over 320 frames x 10 iterations {worst:.2e}")


@pytest.mark.parametrize("method", METHODS)
@pytest.mark.parametrize("schedule", ["pus", "sus"])
def test_lockstep_gf8_markov(torch_cuda, oracle, schedule, method):
    b = _workload("gf8_n2000_markov_bsc", 6, N=400)
    _lockstep(torch_cuda, oracle, b.code, b.obs, "bsc", b.param, schedule, iters=6, T=b.T, K=b.K, method=method,
              atol=_atol(method, schedule))


def _free_running(oracle, b, kind, schedule, method="auto", max_horizon_frac=0.05):
    from tests.parity_util import HORIZON_REL, HORIZON_REL_TRANSFORM
    from paper_cs_0605069_gb300 import gfbp
    cd = gfbp.Code.from_coo(b.code)
    T = b.T
    K = b.K
    ora = oracle.decode(b.code, b.obs, kind, b.param, schedule, max_iter=b.max_iter, T=T, K=K, trace=True)
    rel = HORIZON_REL_TRANSFORM if method == "transform" else HORIZON_REL
    hz = oracle_horizon(oracle, b.code, b.obs, kind, b.param, schedule, b.max_iter, T=T, K=K, rel=rel)
    gpu = gpu_decode(cd, b.obs, kind, b.param, schedule, b.max_iter, T=T, K=K, trace=True, check_method=method)
    kinds = classify_frames(gpu, ora, horizon=hz)
    n = {k: int((kinds == k).sum()) for k in ("match", "tie", "horizon", "fail")}
    print(f"{schedule}/{method}: frames {len(kinds)} {n}")
    assert n["fail"] == 0, fail_report(gpu, ora, hz, np.nonzero(kinds == "fail")[0][:5])
    assert n["horizon"] <= max_horizon_frac * len(kinds) + 1
    return kinds


@pytest.mark.parametrize("schedule", ["pus", "sus"])
def test_free_running_gf4_n96_bsc_1000_frames(torch_cuda, oracle, schedule):
    _free_running(oracle, _workload("gf4_n96_bsc005", 1000), "bsc", schedule)


@pytest.mark.parametrize("method", METHODS)
@pytest.mark.parametrize("schedule", ["pus", "sus"])
def test_free_running_gf16_n1000_awgn(torch_cuda, oracle, schedule, method):
    _free_running(oracle, _workload("gf16_n1000_awgn", 96), "awgn", schedule, method=method)


@pytest.mark.parametrize("schedule", ["pus", "sus"])
def test_free_running_gf8_markov_bsc(torch_cuda, oracle, schedule):
    _free_running(oracle, _workload("gf8_n2000_markov_bsc", 24), "bsc", schedule)


@pytest.mark.parametrize("schedule", ["pus", "sus"])
def test_free_running_gf8_markov_bec(torch_cuda, oracle, schedule):
    _free_running(oracle, _workload("gf8_n2000_markov_bec", 24), "bec", schedule)


def sampled_parity(oracle, b, kind, schedule, gpu, frames):
    """The parity criterion on chosen frames of a batch the GPU decoded whole:
    the oracle decodes those frames alone (frames are independent).  gpu:
    outputs of the whole batch (x_hat, iters, converged, trace)."""
    from tests.parity_util import Batchlike
    idx = np.asarray(frames)
    sub = Batchlike(b.code, b.obs[idx], np.asarray(b.param)[idx], b.max_iter)
    ora = oracle.decode(sub.code, sub.obs, kind, sub.param, schedule, max_iter=sub.max_iter, trace=True)
    hz = oracle_horizon(oracle, sub.code, sub.obs, kind, sub.param, schedule, sub.max_iter)
    g = {k: np.asarray(gpu[k])[idx] for k in ("x_hat", "iters", "converged", "trace")}
    return classify_frames(g, ora, horizon=hz)


# The benchmark's launch: 4096 frames of GF(16), N = 1000 at 1.0/1.5/2.0 dB
# (frame f at the (f mod 3)-th level), max 200 iterations, AUTO kernels.  The
# oracle decodes 132 frames spread over the batch, 44 at each noise level, one
# by one: no frame may fail; ties and horizon frames are counted, the latter
# capped as in the free-running tests.
_BASES = np.linspace(0, 4093, 44).astype(int) // 3 * 3
BENCH_SAMPLE = sorted(int(b) + r for b in _BASES for r in range(3))


def test_benchmark_sample_spans_the_batch_and_noise_levels():
    f = np.asarray(BENCH_SAMPLE)
    assert len(f) == 132 and f.min() == 0 and f.max() >= 4090
    assert all(int((f % 3 == r).sum()) == 44 for r in range(3))


@pytest.mark.parametrize("schedule", ["pus", "sus"])
def test_benchmark_configuration_sampled_frames(torch_cuda, oracle, schedule):
    b = _workload("gf16_n1000_awgn", 4096)
    from paper_cs_0605069_gb300 import gfbp
    cd = gfbp.Code.from_coo(b.code)
    gpu = gpu_decode(cd, b.obs, "awgn", b.param, schedule, b.max_iter, trace=True)
    kinds = sampled_parity(oracle, b, "awgn", schedule, gpu, BENCH_SAMPLE)
    n = {k: int((kinds == k).sum()) for k in ("match", "tie", "horizon", "fail")}
    print(f"{schedule} benchmark configuration, {len(BENCH_SAMPLE)} sampled frames: {n}")
    assert n["fail"] == 0, np.asarray(BENCH_SAMPLE)[kinds == "fail"]
    assert n["horizon"] <= 0.05 * len(BENCH_SAMPLE) + 1


# ---------------------------------------------------------------- edge cases
def _tiny_codes():
    from tests.test_oracle_decoder import chain_code, random_tree_code
    rng = np.random.default_rng(11)
    yield "tree-q8", random_tree_code(rng, 6, 8)
    yield "tree-q2", random_tree_code(rng, 11, 2)
    yield "chain-q4", chain_code(7, 4, rng)


@pytest.mark.parametrize("schedule", ["pus", "sus"])
def test_tree_codes_exact_marginals_on_gpu(torch_cuda, oracle, schedule):
    """Cycle-free graphs: the device reaches the exact marginals (enumeration)
    and the oracle's posteriors, with a non-zero syndrome."""
    from paper_cs_0605069_gb300 import gfbp
    from tests.test_oracle_decoder import exact_marginals
    for name, code in _tiny_codes():
        rng = np.random.default_rng(len(name))
        ll = rng.normal(0, 1.5, size=(3, code.N, code.q)).astype(np.float32)
        z = rng.integers(0, code.q, size=(3, code.M)).astype(np.uint8)
        it = code.N + code.M + 2
        ora = oracle.decode(code, ll, "loglik", 0.0, schedule, max_iter=it, syn=z, early_stop=False, post=True)
        gpu = gpu_decode(gfbp.Code.from_coo(code), ll, "loglik", 0.0, schedule, it, syndrome=z, post=True,
                         no_early_stop=True)
        for f in range(3):
            L = oracle.channel(code.q, "loglik", 0.0, ll[f])
            want = exact_marginals(code, L, z[f])
            np.testing.assert_allclose(gpu["post"][f], want, atol=2e-6)
            np.testing.assert_allclose(gpu["post"][f], ora["post"][f], atol=2e-6)


@pytest.mark.parametrize("q", [2, 32, 64, 128, 256])
@pytest.mark.parametrize("schedule", ["pus", "sus"])
def test_other_field_sizes(torch_cuda, oracle, q, schedule):
    """Every field size the library instantiates, on a small regular code
    over the BI-AWGN channel: lock-step Q and q from the oracle's state."""
    from paper_cs_0605069_gb300 import workload as W
    code = W.regular_code(q, 48, cfg=f"fields{q}")
    rng = np.random.default_rng(q)
    x = W.encode(code, rng.integers(0, q, size=(4, code.K)))
    obs = W.biawgn(rng, x, code.p, 0.8)
    _lockstep(torch_cuda, oracle, code, obs, "awgn", 0.8, schedule, iters=3)


@pytest.mark.parametrize("q", [32, 64, 128, 256])
@pytest.mark.parametrize("schedule", ["pus", "sus"])
def test_lockstep_large_fields_probability_route(torch_cuda, oracle, q, schedule):
    """The probability route for q >= 32 (shared-memory XOR-convolutions by
    lane groups; AUTO's route up to q = 64, an explicit choice above) on
    N = 400 symbols near the code's threshold, 8 iterations, every posterior
    and message within 1e-5 of the oracle."""
    from paper_cs_0605069_gb300 import workload as W
    code = W.regular_code(q, 400, cfg=f"bigfield{q}", encodable=False)
    rng = np.random.default_rng(q + 1)
    F = 3
    x = rng.integers(0, q, size=(F, code.N))
    z = code.syndrome(x)
    sig = W.ebn0_to_sigma(1.5)
    obs = W.biawgn(rng, x, code.p, sig)
    _lockstep(torch_cuda, oracle, code, obs, "awgn", sig, schedule, iters=8, syn=z.astype(np.uint8),
              method="auto" if q <= 64 else "direct")


@pytest.mark.parametrize("q", [128, 256])
@pytest.mark.parametrize("schedule", ["pus", "sus"])
def test_lockstep_large_fields_transform_route(torch_cuda, oracle, q, schedule):
    """AUTO's route for q = 128, 256 (the transform route): held to the
    accuracy stated for it, its largest deviation printed."""
    from paper_cs_0605069_gb300 import workload as W
    code = W.regular_code(q, 400, cfg=f"bigfield{q}", encodable=False)
    rng = np.random.default_rng(q + 1)
    x = rng.integers(0, q, size=(3, code.N))
    z = code.syndrome(x)
    sig = W.ebn0_to_sigma(1.5)
    obs = W.biawgn(rng, x, code.p, sig)
    worst = _lockstep(torch_cuda, oracle, code, obs, "awgn", sig, schedule, iters=8, syn=z.astype(np.uint8),
                      atol=TRANSFORM_ATOL[schedule])
    print(f"GF({q}) {schedule} transform route: worst lock-step deviation {worst:.2e}")


@pytest.mark.parametrize("schedule", ["pus", "sus"])
def test_irregular_code_generic_kernel(torch_cuda, oracle, schedule):
    """Row degrees up to 16 and column degrees up to 8 use the generic kernel."""
    rng = np.random.default_rng(3)
    q, M, N = 8, 30, 40
    H = np.zeros((M, N), np.int64)
    for j in range(N):
        dv = int(rng.integers(1, 8))
        for i in rng.choice(np.arange(1, M), size=dv, replace=False):
            H[i, j] = rng.integers(1, q)
    H[0, :16] = rng.integers(1, q, size=16)
    from paper_cs_0605069_gb300 import workload as W
    code = W.code_from_dense(H, q)
    assert max(np.bincount(code.rows)) <= 16 and max(np.bincount(code.cols)) <= 8
    obs = rng.integers(0, 2, size=(5, N, 3)).astype(np.float32)
    _lockstep(torch_cuda, oracle, code, obs, "bsc", 0.07, schedule, iters=4)


@pytest.mark.parametrize("schedule", ["pus", "sus"])
def test_punctured_symbols_and_syndrome_form(torch_cuda, oracle, schedule):
    """MN-style input (Eq. 2): punctured symbols and a non-zero syndrome."""
    from paper_cs_0605069_gb300 import gfbp
    b = _workload("gf4_n96_bsc005", 40)
    code = b.code
    rng = np.random.default_rng(9)
    v = rng.integers(0, code.q, size=(40, code.N))
    z = code.syndrome(v).astype(np.uint8)
    punct = np.zeros(code.N, np.uint8)
    punct[:10] = 1
    obs = (b.obs.astype(np.int64) ^ rng.integers(0, 2, size=b.obs.shape)).astype(np.float32)
    ora = oracle.decode(code, obs, "bsc", 0.05, schedule, max_iter=40, punct=punct, syn=z, trace=True)
    gpu = gpu_decode(gfbp.Code.from_coo(code), obs, "bsc", 0.05, schedule, 40, punct=punct, syndrome=z, trace=True)
    kinds = classify_frames(gpu, ora)
    assert (kinds != "fail").all()


def test_empty_batch_and_errors(torch_cuda):
    import torch
    from paper_cs_0605069_gb300 import gfbp, workload as W
    b = W.make_batch("gf4_n96_bsc005", frames=1)
    cd = gfbp.Code.from_coo(b.code)
    out = gfbp.decode(cd, torch.empty((0, b.code.N, 2), device="cuda"), "bsc", 0.05)
    assert out["x_hat"].shape == (0, b.code.N)
    with pytest.raises(gfbp.GfbpError) as e:
        gfbp.decode(cd, to_dev(b.obs), "bsc", 1.5)
    assert e.value.status == gfbp.GFBP_EINVAL and "flip rate" in str(e.value)
    with pytest.raises(gfbp.GfbpError):
        gfbp.decode(cd, to_dev(b.obs), "bsc", 0.05, max_iter=0)
    with pytest.raises(gfbp.GfbpError):
        gfbp.decode(cd, to_dev(b.obs), "bsc", 0.05, T=np.eye(4), K=0)


@pytest.mark.parametrize("schedule,partials,frames", [("pus", "auto", 300), ("sus", "fold", 300),
                                                      ("sus", "running", 120)])
def test_single_frame_and_large_batch_agree(torch_cuda, schedule, partials, frames):
    """A frame decodes to the same bits alone and inside a batch run by the
    same kernel (frames are independent; the persistent kernels take them in
    any order).  SUS with AUTO partials picks its kernel by the frame count,
    so each SUS kernel is pinned here."""
    from paper_cs_0605069_gb300 import gfbp
    b = _workload("gf16_n1000_awgn", frames)
    cd = gfbp.Code.from_coo(b.code)
    full = gpu_decode(cd, b.obs, "awgn", b.param, schedule, 50, post=True, partials=partials)
    for f in (0, 1, frames // 2 + 7, frames - 1):
        one = gpu_decode(cd, b.obs[f:f + 1], "awgn", b.param[f:f + 1], schedule, 50, post=True,
                         partials=partials)
        assert one["iters"][0] == full["iters"][f]
        np.testing.assert_array_equal(one["x_hat"][0], full["x_hat"][f])
        np.testing.assert_array_equal(one["post"][0], full["post"][f])


# The TENSOR check method (SUS, q >= 16): transforms on the tensor cores with an
# FP16 hi/lo split and FP32 accumulation; the stated bound is 1e-4 posterior
# max-abs per iteration against the FP64 oracle.
TENSOR_ATOL = 1e-4


@pytest.mark.parametrize("q,N,db", [(64, 128, 2.0), (256, 48, 2.5), (16, 240, 1.5)])
def test_lockstep_tensor_route(torch_cuda, oracle, q, N, db):
    from paper_cs_0605069_gb300 import workload as W
    code = W.regular_code(q, N, cfg=f"tensor_route_{q}", encodable=False)
    rng = np.random.default_rng(q + 7)
    F = 8
    x = rng.integers(0, q, size=(F, code.N))
    sig = W.ebn0_to_sigma(db)
    obs = W.biawgn(rng, x, code.p, sig)
    worst = _lockstep(torch_cuda, oracle, code, obs, "awgn", np.full(F, sig), "sus", iters=6,
                      method="tensor", atol=TENSOR_ATOL)
    print(f"GF({q}) tensor route lock-step worst {worst:.2e}")


def test_lockstep_tensor_route_markov(torch_cuda, oracle):
    from paper_cs_0605069_gb300 import workload as W
    b = W.make_batch("gf8_n2000_markov_bsc", frames=4, N=300)
    # GF(8) is below the tensor route's q >= 16: the route is refused there
    from paper_cs_0605069_gb300 import gfbp
    import torch
    cd = gfbp.Code.from_coo(b.code)
    with pytest.raises(gfbp.GfbpError):
        gfbp.decode(cd, to_dev(b.obs, torch.float32), "bsc", 0.08, schedule="sus", check_method="tensor")
    with pytest.raises(gfbp.GfbpError):
        code64 = W.regular_code(64, 64, cfg="tensor_pus", encodable=False)
        c64 = gfbp.Code.from_coo(code64)
        obs = torch.zeros((2, 64, 6), device="cuda")
        gfbp.decode(c64, obs, "awgn", 0.8, schedule="pus", check_method="tensor")


def test_free_running_tensor_route_gf64(torch_cuda, oracle):
    from paper_cs_0605069_gb300 import workload as W
    from tests.parity_util import Batchlike
    code = W.regular_code(64, 256, cfg="tensor_free_64", encodable=False)
    rng = np.random.default_rng(64)
    F = 48
    x = np.zeros((F, code.N), np.int64)
    sig = np.array([W.ebn0_to_sigma(db) for db in (1.5, 2.0, 2.5)])[np.arange(F) % 3]
    obs = W.biawgn(rng, x, code.p, sig)
    _free_running(oracle, Batchlike(code, obs, sig, 40), "awgn", "sus", method="tensor")


def _code_with_empty_columns(q, seed):
    """A 6 x 12 H over GF(q) whose columns 5 and 11 meet no check (a symbol the
    code leaves free: its posterior is its channel likelihood alone)."""
    from paper_cs_0605069_gb300 import workload as W
    rng = np.random.default_rng(seed)
    H = np.zeros((6, 12), np.int64)
    for j in range(12):
        if j in (5, 11):
            continue
        # column degrees 1 to 3 and row degrees at most 8 keep the code within
        # the single-team SUS kernel, the lane layout's route for q <= 16
        rows = rng.choice(6, size=1 + j % 3, replace=False)
        H[rows, j] = rng.integers(1, q, size=rows.size)
    for i in range(6):
        while np.count_nonzero(H[i]) < 2:
            j = rng.choice([c for c in range(12) if c not in (5, 11) and H[i, c] == 0])
            H[i, j] = rng.integers(1, q)
    return W.code_from_dense(H, q), rng


@pytest.mark.parametrize("q,method,layout", [
    (4, "direct", "thread"), (4, "direct", "lanes"), (16, "direct", "thread"),
    (32, "transform", "thread"), (32, "transform", "lanes"), (16, "tensor", "auto"), (64, "tensor", "auto"),
])
@pytest.mark.parametrize("schedule", ["sus", "pus"])
def test_lockstep_columns_without_checks(torch_cuda, oracle, q, method, layout, schedule):
    if method == "tensor" and schedule == "pus":
        pytest.skip("the tensor check method is a SUS route")
    from paper_cs_0605069_gb300 import workload as W
    code, rng = _code_with_empty_columns(q, q)
    F = 5
    obs = W.bsc(rng, np.zeros((F, code.N), np.int64), code.p, 0.1)
    atol = TENSOR_ATOL if method == "tensor" else _atol(method, schedule)
    _lockstep(torch_cuda, oracle, code, obs, "bsc", np.full(F, 0.1), schedule, iters=4, method=method,
              atol=atol, layout=layout)


@pytest.mark.parametrize("q,method", [(4, "direct"), (32, "transform"), (16, "tensor")])
def test_free_running_columns_without_checks(torch_cuda, oracle, q, method):
    """Decoding to the end: the free columns' decisions are their channel
    argmax, and the level kernels agree with the lane kernels bit for bit."""
    from paper_cs_0605069_gb300 import gfbp, workload as W
    from tests.parity_util import gpu_decode
    code, rng = _code_with_empty_columns(q, 100 + q)
    F = 12
    obs = W.bsc(rng, np.zeros((F, code.N), np.int64), code.p, 0.15)
    cd = gfbp.Code.from_coo(code)
    outs = {}
    for lay in (("auto",) if method == "tensor" else ("lanes", "thread", "auto")):
        outs[lay] = gpu_decode(cd, obs, "bsc", 0.15, "sus", 20, post=True, trace=True, check_method=method,
                               layout=lay, partials="fold" if lay == "thread" else "auto")
    if method != "tensor":
        a, b = outs["lanes"], outs["thread"]
        for k in a:
            x, y = np.asarray(a[k]), np.asarray(b[k])
            if x.dtype == np.float32:
                x, y = x.view(np.uint32), y.view(np.uint32)
            assert np.array_equal(x, y), f"{k} differs between the lane and level kernels"
    # BSC likelihood of each symbol value from the received bits, normalised
    a = np.arange(q)
    bits = (a[:, None] >> np.arange(code.p)[None, :]) & 1            # [q, p]
    for j in (5, 11):
        rx = obs[:, j, :].astype(np.int64)                            # [F, p]
        flips = (bits[None, :, :] != rx[:, None, :]).sum(axis=2)      # [F, q]
        lik = 0.15 ** flips * 0.85 ** (code.p - flips)
        lik /= lik.sum(axis=1, keepdims=True)
        for out in outs.values():
            np.testing.assert_allclose(out["post"][:, j], lik, atol=1e-6)
            np.testing.assert_array_equal(out["x_hat"][:, j], (rx << np.arange(code.p)).sum(axis=1))
