"""The frame-resident kernels (a frame's whole edge slab on chip for its whole
decode: in one CTA's shared memory, or for SUS in an L2-sized set of
workspace slabs) against the global-memory kernels of the same arithmetic,
bit for bit: PUS against the thread layout, SUS against the level kernel with
running partial convolutions in a second global slab.  x_hat, iteration
counts, flags, posteriors, traces and lock-step messages must all agree."""
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


REF = {"pus": dict(layout="thread"), "sus": dict(layout="thread", partials="running_global")}


LAYOUTS = {"pus": ("resident", "auto"), "sus": ("resident", "l2resident", "auto")}


def _both(cd, obs, kind, param, max_iter, auto_sus=True, **kw):
    for sched in ("pus", "sus"):
        ref = gpu_decode(cd, obs, kind, param, sched, max_iter, post=True, trace=True, **REF[sched], **kw)
        for lay in LAYOUTS[sched]:
            if sched == "sus" and lay == "auto" and not auto_sus:
                continue
            out = gpu_decode(cd, obs, kind, param, sched, max_iter, post=True, trace=True, layout=lay, **kw)
            _same(ref, out, f"{sched} {lay}")


@pytest.mark.parametrize("name,N,frames,max_iter", [
    ("gf4_n96_bsc005", None, 64, 60),
    ("gf16_n1000_awgn", None, 24, 60),
    ("gf8_n2000_markov_bsc", 1200, 12, 40),   # (N = 2000 does not fit one CTA for PUS)
    ("gf8_n2000_markov_bec", 500, 18, 40),
])
def test_resident_equals_global(torch_cuda, name, N, frames, max_iter):
    from paper_cs_0605069_gb300 import gfbp, workload as W
    b = W.make_batch(name, frames=frames, N=N)
    cd = gfbp.Code.from_coo(b.code)
    _both(cd, b.obs, b.channel, b.param, max_iter, T=b.T, K=b.K)


def test_resident_many_frames_per_cta(torch_cuda):
    """Far more frames than resident CTAs: every CTA decodes frames in turn in
    the same shared memory (GF(16), N = 1000: one frame per SM).  (SUS AUTO
    takes the folding level kernel at this frame count.)"""
    from paper_cs_0605069_gb300 import gfbp, workload as W
    b = W.make_batch("gf16_n1000_awgn", frames=700)
    cd = gfbp.Code.from_coo(b.code)
    _both(cd, b.obs, b.channel, b.param, 25, auto_sus=False)


@pytest.mark.parametrize("q,dv,dc,N", [(2, 3, 6, 240), (16, 4, 6, 300), (4, 2, 4, 128), (8, 3, 5, 150)])
def test_resident_degrees_and_syndrome(torch_cuda, q, dv, dc, N):
    from paper_cs_0605069_gb300 import gfbp, workload as W
    code = W.regular_code(q, N, dv=dv, dc=dc, cfg=f"resident_{q}_{dv}_{dc}", encodable=False)
    rng = np.random.default_rng(q * 7 + dc)
    F = 16
    x = rng.integers(0, q, size=(F, code.N))
    z = code.syndrome(x).astype(np.uint8)
    obs = W.bsc(rng, x, code.p, 0.04)
    cd = gfbp.Code.from_coo(code)
    _both(cd, obs, "bsc", 0.04, 30, syndrome=z)


def test_resident_small_code_with_free_column_and_degree_one_check(torch_cuda):
    """A column without checks, a check of degree 1 and one of degree 2."""
    from paper_cs_0605069_gb300 import gfbp, workload as W
    H = np.array([[1, 2, 0, 3, 1, 0],
                  [0, 1, 1, 0, 2, 0],
                  [3, 0, 2, 1, 0, 0],
                  [0, 0, 0, 2, 0, 0],
                  [0, 3, 0, 0, 1, 0]])
    code = W.code_from_dense(H, 4)
    rng = np.random.default_rng(4)
    obs = W.bsc(rng, np.zeros((9, 6), np.int64), code.p, 0.1)
    cd = gfbp.Code.from_coo(code)
    _both(cd, obs, "bsc", 0.1, 20, no_early_stop=True)


@pytest.mark.parametrize("sched", ["pus", "sus"])
def test_resident_lockstep_step(torch_cuda, oracle, sched):
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
    runs = [("ref", REF[sched])] + [(lay, dict(layout=lay)) for lay in LAYOUTS[sched]]
    for name, v in runs:
        m = to_dev(msg0.astype(np.float32))
        o = gfbp.step(cd, to_dev(b.obs, torch.float32), m, channel=b.channel, schedule=sched, T=b.T, K=b.K,
                      prior_in=prior, frame_param=fp, **v)
        torch.cuda.synchronize()
        outs[name] = {k: x.cpu().numpy() for k, x in o.items() if x is not None}
    for lay in LAYOUTS[sched]:
        _same(outs["ref"], outs[lay], f"{sched} step {lay}")


def test_resident_refused_where_it_does_not_apply(torch_cuda):
    import torch
    from paper_cs_0605069_gb300 import gfbp, workload as W
    b = W.make_batch("gf4_n96_bsc005", frames=2)
    cd = gfbp.Code.from_coo(b.code)
    obs = to_dev(b.obs, torch.float32)
    with pytest.raises(gfbp.GfbpError):
        gfbp.decode(cd, obs, b.channel, float(b.param[0]), schedule="sus", layout="resident", partials="fold")
    code = W.regular_code(32, 64, cfg="resident_q32", encodable=False)
    cd32 = gfbp.Code.from_coo(code)
    o32 = to_dev(W.bsc(np.random.default_rng(1), np.zeros((2, 64), np.int64), code.p, 0.02), torch.float32)
    with pytest.raises(gfbp.GfbpError):
        gfbp.decode(cd32, o32, "bsc", 0.02, schedule="pus", layout="resident")
