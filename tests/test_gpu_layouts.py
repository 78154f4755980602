"""Kernels that hold or order the work differently must give the same bits.

SUS: the multi-team kernel starts a column once the last earlier column sharing
a check with it has finished; the level kernel (thread layout, check messages
folded afresh at every visit) updates the columns level by level (one level's
columns share no check).  Both give every column the operands of the strictly
sequential order with the single-team kernel's arithmetic.  PUS: the thread layout (a check or a column per thread,
vectors in registers) runs the lane-group kernel's arithmetic in the same
order.  So x_hat, iters, converged, posteriors, traces and lock-step messages
must match the lane kernels bit for bit."""
import numpy as np
import pytest

from tests.parity_util import gpu_decode, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_cs_0605069_gb300 import gfbp
    gfbp.lib()
    return torch


def _same(a, b, what):
    for k in a:
        x, y = np.asarray(a[k]), np.asarray(b[k])
        if x.dtype == np.float32:
            x, y = x.view(np.uint32), y.view(np.uint32)
        assert np.array_equal(x, y), f"{what}: {k} differs"


def _widths(cd, obs, kind, param, max_iter, widths=(2, 4, 8), levels=True, **kw):
    ref = gpu_decode(cd, obs, kind, param, "sus", max_iter, post=True, trace=True, layout="lanes", sus_width=1,
                     **kw)
    runs = [(f"width {w}", dict(layout="lanes", sus_width=w)) for w in widths]
    if levels:
        runs.append(("levels", dict(layout="thread", partials="fold")))
    for what, v in runs:
        out = gpu_decode(cd, obs, kind, param, "sus", max_iter, post=True, trace=True, **v, **kw)
        _same(ref, out, what)
    return ref


@pytest.mark.parametrize("name,N,frames,max_iter", [
    ("gf4_n96_bsc005", None, 64, 60),
    ("gf16_n1000_awgn", 400, 36, 60),
    ("gf8_n2000_markov_bsc", 300, 18, 40),
    ("gf8_n2000_markov_bec", 300, 18, 40),
])
def test_wave_equals_single_team(torch_cuda, name, N, frames, max_iter):
    from paper_cs_0605069_gb300 import gfbp, workload as W
    b = W.make_batch(name, frames=frames, N=N)
    cd = gfbp.Code.from_coo(b.code)
    ref = _widths(cd, b.obs, b.channel, b.param, max_iter, T=b.T, K=b.K)
    assert ref["iters"].min() >= 1


def test_wave_row_degree_8_with_syndrome(torch_cuda):
    from paper_cs_0605069_gb300 import gfbp, workload as W
    code = W.regular_code(16, 240, dv=4, dc=8, cfg="wave_dc8", encodable=False)
    rng = np.random.default_rng(7)
    F = 20
    x = rng.integers(0, 16, size=(F, code.N))
    z = code.syndrome(x).astype(np.uint8)   # H x = z holds for the sent word
    sig = W.ebn0_to_sigma(2.5, rate=0.5)
    obs = W.biawgn(rng, x, code.p, sig)
    cd = gfbp.Code.from_coo(code)
    ref = _widths(cd, obs, "awgn", sig, 50, syndrome=z)
    assert ref["converged"].sum() > F // 2


def test_wave_more_frames_than_resident_ctas(torch_cuda):
    """Every CTA takes several frames in turn."""
    from paper_cs_0605069_gb300 import gfbp, workload as W
    b = W.make_batch("gf4_n96_bsc005", frames=3000)
    cd = gfbp.Code.from_coo(b.code)
    _widths(cd, b.obs, b.channel, b.param, 30, widths=(2, 8))


def test_wave_code_shorter_than_team_count(torch_cuda):
    """N = 5 columns, 8 teams: teams without columns must not block."""
    from paper_cs_0605069_gb300 import gfbp, workload as W
    H = np.array([[1, 2, 0, 3, 1],
                  [0, 1, 1, 0, 2],
                  [3, 0, 2, 1, 0]])
    code = W.code_from_dense(H, 4)
    rng = np.random.default_rng(3)
    obs = W.bsc(rng, np.zeros((6, 5), np.int64), code.p, 0.1)
    cd = gfbp.Code.from_coo(code)
    _widths(cd, obs, "bsc", 0.1, 20, no_early_stop=True)


def test_wave_lockstep_step_equals_single_team(torch_cuda, oracle):
    import torch
    from paper_cs_0605069_gb300 import gfbp, workload as W
    b = W.make_batch("gf8_n2000_markov_bsc", frames=8, N=300)
    cd = gfbp.Code.from_coo(b.code)
    F = b.obs.shape[0]
    msg0 = oracle.initial_messages(b.code, b.obs, b.channel, b.param, T=b.T, K=b.K)
    _, pi = oracle.markov(b.T, np.full((1, b.code.q), 1.0 / b.code.q))
    prior = to_dev(np.broadcast_to(pi, (F, b.K, b.code.q)).astype(np.float32).copy())
    fp = to_dev(np.asarray(b.param, np.float32))
    outs = {}
    for name, v in (("one team", dict(layout="lanes", sus_width=1)), ("width 4", dict(layout="lanes",
                    sus_width=4)), ("levels", dict(layout="thread", partials="fold"))):
        m = to_dev(msg0.astype(np.float32))
        o = gfbp.step(cd, to_dev(b.obs, torch.float32), m, channel=b.channel, schedule="sus", T=b.T, K=b.K,
                      prior_in=prior, frame_param=fp, **v)
        torch.cuda.synchronize()
        outs[name] = {k: x.cpu().numpy() for k, x in o.items() if x is not None}
    _same(outs["one team"], outs["width 4"], "step width 4")
    _same(outs["one team"], outs["levels"], "step levels")


@pytest.mark.parametrize("name,N,frames,max_iter", [
    ("gf4_n96_bsc005", None, 64, 60),
    ("gf16_n1000_awgn", 400, 36, 60),
    ("gf8_n2000_markov_bsc", 300, 18, 40),
    ("gf8_n2000_markov_bec", 300, 18, 40),
])
def test_pus_thread_layout_equals_lanes(torch_cuda, name, N, frames, max_iter):
    from paper_cs_0605069_gb300 import gfbp, workload as W
    b = W.make_batch(name, frames=frames, N=N)
    cd = gfbp.Code.from_coo(b.code)
    kw = dict(T=b.T, K=b.K, post=True, trace=True)
    ref = gpu_decode(cd, b.obs, b.channel, b.param, "pus", max_iter, layout="lanes", **kw)
    out = gpu_decode(cd, b.obs, b.channel, b.param, "pus", max_iter, layout="thread", **kw)
    _same(ref, out, "pus thread layout")


def test_pus_thread_layout_irregular_and_syndrome(torch_cuda):
    """Row degree 12, column degree 6 (the lane kernel's large-degree variant)
    and a nonzero syndrome."""
    from paper_cs_0605069_gb300 import gfbp, workload as W
    code = W.regular_code(8, 120, dv=6, dc=12, cfg="levels_dv6", encodable=False)
    rng = np.random.default_rng(5)
    F = 12
    x = rng.integers(0, 8, size=(F, code.N))
    z = code.syndrome(x).astype(np.uint8)
    obs = W.bsc(rng, x, code.p, 0.04)
    cd = gfbp.Code.from_coo(code)
    for sched in ("pus", "sus"):
        ref = gpu_decode(cd, obs, "bsc", 0.04, sched, 30, syndrome=z, post=True, trace=True, layout="lanes")
        out = gpu_decode(cd, obs, "bsc", 0.04, sched, 30, syndrome=z, post=True, trace=True, layout="thread")
        if sched == "pus":
            _same(ref, out, "pus thread layout")
        else:
            # column degree 6 is beyond the SUS team kernels: the lane layout
            # ran the generic group kernel, whose sums run in another order
            assert np.mean(ref["x_hat"] == out["x_hat"]) > 0.99


def test_pus_lockstep_thread_equals_lanes(torch_cuda, oracle):
    import torch
    from paper_cs_0605069_gb300 import gfbp, workload as W
    b = W.make_batch("gf8_n2000_markov_bsc", frames=8, N=300)
    cd = gfbp.Code.from_coo(b.code)
    F = b.obs.shape[0]
    msg0 = oracle.initial_messages(b.code, b.obs, b.channel, b.param, T=b.T, K=b.K)
    _, pi = oracle.markov(b.T, np.full((1, b.code.q), 1.0 / b.code.q))
    prior = to_dev(np.broadcast_to(pi, (F, b.K, b.code.q)).astype(np.float32).copy())
    fp = to_dev(np.asarray(b.param, np.float32))
    outs = {}
    for lay in ("lanes", "thread"):
        m = to_dev(msg0.astype(np.float32))
        o = gfbp.step(cd, to_dev(b.obs, torch.float32), m, channel=b.channel, schedule="pus", T=b.T, K=b.K,
                      prior_in=prior, frame_param=fp, layout=lay)
        torch.cuda.synchronize()
        outs[lay] = {k: x.cpu().numpy() for k, x in o.items() if x is not None}
    _same(outs["lanes"], outs["thread"], "pus step thread layout")


def test_levels_column_degree_above_team_limit(torch_cuda, oracle):
    """Column degree 6 (beyond the team kernels): the level kernel against the
    oracle in lock-step (one SUS iteration from the same messages)."""
    import torch
    from paper_cs_0605069_gb300 import gfbp, workload as W
    from tests.parity_util import LOCKSTEP_ATOL
    code = W.regular_code(8, 120, dv=6, dc=12, cfg="levels_dv6", encodable=False)
    rng = np.random.default_rng(11)
    F = 6
    obs = W.bsc(rng, np.zeros((F, code.N), np.int64), code.p, 0.03)
    cd = gfbp.Code.from_coo(code)
    fp = to_dev(np.full(F, 0.03, np.float32))
    msg = oracle.initial_messages(code, obs, "bsc", 0.03)
    for it in range(3):
        ref = oracle.step(code, obs, "bsc", 0.03, msg, "sus")
        o = gfbp.step(cd, to_dev(obs, torch.float32), to_dev(msg.astype(np.float32)), channel="bsc",
                      schedule="sus", frame_param=fp, layout="thread")
        torch.cuda.synchronize()
        assert np.abs(o["post"].cpu().numpy() - ref["post"]).max() <= LOCKSTEP_ATOL
        assert np.abs(o["msg"].cpu().numpy() - ref["msg"]).max() <= LOCKSTEP_ATOL
        msg = ref["msg"]


def test_wave_width_is_validated(torch_cuda):
    import torch
    from paper_cs_0605069_gb300 import gfbp, workload as W
    b = W.make_batch("gf4_n96_bsc005", frames=2)
    cd = gfbp.Code.from_coo(b.code)
    with pytest.raises(gfbp.GfbpError):
        gfbp.decode(cd, to_dev(b.obs, torch.float32), b.channel, float(b.param[0]), schedule="sus", sus_width=3)
    with pytest.raises(KeyError):
        gfbp.decode(cd, to_dev(b.obs, torch.float32), b.channel, float(b.param[0]), schedule="sus",
                    layout="fastest")


@pytest.mark.parametrize("q,N,db", [(32, 192, 2.0), (64, 128, 2.5), (256, 96, 3.0), (16, 240, 1.5)])
def test_sus_levels_transform_route_equals_lanes(torch_cuda, q, N, db):
    """The level schedule with the transform check node (one lane group per
    (column, check) pair) against the lane kernel walking the columns."""
    from paper_cs_0605069_gb300 import gfbp, workload as W
    code = W.regular_code(q, N, cfg=f"levels_tr_{q}", encodable=False)
    rng = np.random.default_rng(q)
    F = 10
    x = rng.integers(0, q, size=(F, code.N))
    z = code.syndrome(x).astype(np.uint8)
    sig = W.ebn0_to_sigma(db)
    obs = W.biawgn(rng, x, code.p, sig)
    cd = gfbp.Code.from_coo(code)
    kw = dict(syndrome=z, post=True, trace=True, check_method="transform")
    ref = gpu_decode(cd, obs, "awgn", sig, "sus", 25, layout="lanes", **kw)
    out = gpu_decode(cd, obs, "awgn", sig, "sus", 25, layout="thread", **kw)
    _same(ref, out, f"GF({q}) levels, transform route")


def test_sus_levels_transform_route_markov_step(torch_cuda, oracle):
    import torch
    from paper_cs_0605069_gb300 import gfbp, workload as W
    b = W.make_batch("gf8_n2000_markov_bsc", frames=6, N=300)
    cd = gfbp.Code.from_coo(b.code)
    F = b.obs.shape[0]
    msg0 = oracle.initial_messages(b.code, b.obs, b.channel, b.param, T=b.T, K=b.K)
    _, pi = oracle.markov(b.T, np.full((1, b.code.q), 1.0 / b.code.q))
    prior = to_dev(np.broadcast_to(pi, (F, b.K, b.code.q)).astype(np.float32).copy())
    fp = to_dev(np.asarray(b.param, np.float32))
    outs = {}
    for lay in ("lanes", "thread"):
        m = to_dev(msg0.astype(np.float32))
        o = gfbp.step(cd, to_dev(b.obs, torch.float32), m, channel=b.channel, schedule="sus", T=b.T, K=b.K,
                      prior_in=prior, frame_param=fp, layout=lay, check_method="transform")
        torch.cuda.synchronize()
        outs[lay] = {k: x.cpu().numpy() for k, x in o.items() if x is not None}
    _same(outs["lanes"], outs["thread"], "sus step, transform route, levels")
    full = {}
    for lay in ("lanes", "thread"):
        full[lay] = gpu_decode(cd, b.obs, b.channel, b.param, "sus", 30, T=b.T, K=b.K, post=True,
                               check_method="transform", layout=lay)
    _same(full["lanes"], full["thread"], "sus decode, transform route, Markov, levels")


def test_pus_bulk_staged_equals_plain_staging(torch_cuda):
    """Up to 8 frames per SM the PUS kernel fetches each check by bulk copies
    one check ahead; above that it loads them in place.  Both give the same
    bits: a 64-frame decode (bulk) against the same frames inside a 2000-frame
    decode (plain), and the 2000-frame decode against the thread layout."""
    import torch
    from paper_cs_0605069_gb300 import gfbp, workload as W
    b = W.make_batch("gf4_n96_bsc005", frames=2000)
    cd = gfbp.Code.from_coo(b.code)
    big = gpu_decode(cd, b.obs, b.channel, b.param, "pus", 60, post=True, layout="lanes")
    small = gpu_decode(cd, b.obs[:64], b.channel, b.param[:64], "pus", 60, post=True, layout="lanes")
    _same(small, {k: v[:64] for k, v in big.items()}, "bulk vs plain staging")
    thr = gpu_decode(cd, b.obs, b.channel, b.param, "pus", 60, post=True, layout="thread")
    _same(big, thr, "plain staging vs thread layout")


# SUS with running partial convolutions: the kernel holding a frame's partials
# in shared memory against the one holding them in the workspace.
@pytest.mark.parametrize("name,N,frames,max_iter", [
    ("gf4_n96_bsc005", None, 64, 60),
    ("gf16_n1000_awgn", None, 20, 60),
    ("gf8_n2000_markov_bsc", 300, 18, 40),
    ("gf8_n2000_markov_bec", 300, 18, 40),
])
def test_sus_partials_in_shared_memory_equal_global(torch_cuda, name, N, frames, max_iter):
    from paper_cs_0605069_gb300 import gfbp, workload as W
    b = W.make_batch(name, frames=frames, N=N)
    cd = gfbp.Code.from_coo(b.code)
    kw = dict(T=b.T, K=b.K, post=True, trace=True, layout="thread")
    ref = gpu_decode(cd, b.obs, b.channel, b.param, "sus", max_iter, partials="running_global", **kw)
    out = gpu_decode(cd, b.obs, b.channel, b.param, "sus", max_iter, partials="running", **kw)
    _same(ref, out, "running partials, shared vs global memory")
    assert ref["iters"].min() >= 1


@pytest.mark.parametrize("q,dv,dc,N", [(2, 3, 6, 240), (8, 6, 12, 120), (16, 4, 8, 240), (4, 3, 16, 256)])
def test_sus_partials_irregular_degrees_and_syndrome(torch_cuda, q, dv, dc, N):
    from paper_cs_0605069_gb300 import gfbp, workload as W
    code = W.regular_code(q, N, dv=dv, dc=dc, cfg=f"partials_{q}_{dv}_{dc}", encodable=False)
    rng = np.random.default_rng(q * 31 + dc)
    F = 12
    x = rng.integers(0, q, size=(F, code.N))
    z = code.syndrome(x).astype(np.uint8)
    obs = W.bsc(rng, x, code.p, 0.04)
    cd = gfbp.Code.from_coo(code)
    kw = dict(syndrome=z, post=True, trace=True, layout="thread")
    ref = gpu_decode(cd, obs, "bsc", 0.04, "sus", 30, partials="running_global", **kw)
    out = gpu_decode(cd, obs, "bsc", 0.04, "sus", 30, partials="running", **kw)
    _same(ref, out, f"GF({q}) ({dv},{dc}) running partials, shared vs global memory")


def test_sus_partials_lockstep_step_shared_equals_global(torch_cuda, oracle):
    import torch
    from paper_cs_0605069_gb300 import gfbp, workload as W
    b = W.make_batch("gf8_n2000_markov_bsc", frames=8, N=300)
    cd = gfbp.Code.from_coo(b.code)
    F = b.obs.shape[0]
    msg0 = oracle.initial_messages(b.code, b.obs, b.channel, b.param, T=b.T, K=b.K)
    _, pi = oracle.markov(b.T, np.full((1, b.code.q), 1.0 / b.code.q))
    prior = to_dev(np.broadcast_to(pi, (F, b.K, b.code.q)).astype(np.float32).copy())
    fp = to_dev(np.asarray(b.param, np.float32))
    outs = {}
    for part in ("running", "running_global"):
        m = to_dev(msg0.astype(np.float32))
        o = gfbp.step(cd, to_dev(b.obs, torch.float32), m, channel=b.channel, schedule="sus", T=b.T, K=b.K,
                      prior_in=prior, frame_param=fp, layout="thread", partials=part)
        torch.cuda.synchronize()
        outs[part] = {k: x.cpu().numpy() for k, x in o.items() if x is not None}
    _same(outs["running_global"], outs["running"], "sus step, running partials")
