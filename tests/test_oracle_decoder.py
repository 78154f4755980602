"""Pins of the oracle's whole decoder (Sec. 2): exact marginals on cycle-free
graphs, the sequential schedule's in-place order, the BEC peeling decoder,
the syndrome form, the stopping rule and the one-step entry point."""
import itertools
from types import SimpleNamespace

import numpy as np
import pytest

from tests import _gf


def _code(rows, cols, vals, M, N, q):
    order = np.lexsort((cols, rows))
    return SimpleNamespace(q=q, M=M, N=N, rows=np.asarray(rows)[order], cols=np.asarray(cols)[order],
                           vals=np.asarray(vals)[order], poly=0, E=len(rows))


def random_tree_code(rng, N, q, max_deg=4):
    """Random connected cycle-free factor graph with N symbols; columns are
    relabelled at random so that index order does not follow the tree."""
    rows, cols = [], []
    used = [0]
    nxt = 1
    i = 0
    while nxt < N:
        d = int(rng.integers(2, max_deg + 1))
        members = [int(rng.choice(used))] + list(range(nxt, min(N, nxt + d - 1)))
        nxt = min(N, nxt + d - 1)
        for v in members:
            rows.append(i)
            cols.append(v)
        used += members[1:]
        i += 1
    perm = rng.permutation(N)
    cols = [int(perm[c]) for c in cols]
    vals = rng.integers(1, q, size=len(rows))
    return _code(np.array(rows), np.array(cols), vals, i, N, q)


def exact_marginals(code, L, z):
    """Pr(x_j = a | obs, H x = z) by enumerating every word."""
    q, N = code.q, code.N
    words = np.array(list(itertools.product(range(q), repeat=N)))
    ok = np.ones(len(words), bool)
    for i in range(code.M):
        s = np.zeros(len(words), np.int64)
        for r, c, h in zip(code.rows, code.cols, code.vals):
            if r == i:
                s ^= np.array([_gf.mul(int(h), int(x), q.bit_length() - 1) for x in range(q)])[words[:, c]]
        ok &= s == z[i]
    words = words[ok]
    w = np.prod(L[np.arange(N)[None, :], words], axis=1)
    out = np.zeros((N, q))
    for j in range(N):
        np.add.at(out[j], words[:, j], w)
    return out / out.sum(1, keepdims=True)


@pytest.mark.parametrize("q,N", [(2, 11), (4, 7), (8, 5)])
@pytest.mark.parametrize("schedule", ["pus", "sus"])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_tree_codes_reach_exact_marginals(oracle, q, N, schedule, seed):
    rng = np.random.default_rng(100 * seed + q)
    code = random_tree_code(rng, N, q)
    ll = rng.normal(0, 1.5, size=(1, N, q)).astype(np.float32)
    z = rng.integers(0, q, size=code.M) if seed == 2 else np.zeros(code.M, np.int64)
    L = oracle.channel(q, "loglik", 0.0, ll[0])
    want = exact_marginals(code, L, z)
    out = oracle.decode(code, ll, "loglik", 0.0, schedule, max_iter=N + code.M + 2, syn=z[None].astype(np.uint8),
                        early_stop=False, post=True)
    np.testing.assert_allclose(out["post"][0], want, rtol=0, atol=1e-12)


@pytest.mark.parametrize("q,N", [(4, 7), (8, 5)])
@pytest.mark.parametrize("schedule", ["pus", "sus"])
def test_tree_codes_bit_erasures_reach_exact_marginals(oracle, q, N, schedule):
    """BEC with bits erased at random (exact-zero likelihoods for every symbol
    that disagrees with a received bit): on a cycle-free graph BP still
    reaches the exact marginals of the words consistent with the received
    bits and H x = z, z the sent word's syndrome."""
    rng = np.random.default_rng(7 * q + N)
    code = random_tree_code(rng, N, q)
    p = q.bit_length() - 1
    x = rng.integers(0, q, size=N)
    z = np.asarray(_gf.syndrome(code.rows, code.cols, code.vals, code.M, x, q), np.int64)
    bits = ((x[:, None] >> np.arange(p)[None, :]) & 1).astype(np.float32)
    bits[rng.random(bits.shape) < 0.5] = 2.0   # erased
    L = oracle.channel(q, "bec", 0.5, bits)
    assert np.all(L[np.arange(N), x] > 0)       # the sent word stays possible
    want = exact_marginals(code, L, z)
    out = oracle.decode(code, bits[None], "bec", 0.5, schedule, max_iter=N + code.M + 2,
                        syn=z[None].astype(np.uint8), early_stop=False, post=True)
    np.testing.assert_allclose(out["post"][0], want, rtol=0, atol=1e-12)


def chain_code(N, q, rng):
    rows = np.repeat(np.arange(N - 1), 2)
    cols = np.stack([np.arange(N - 1), np.arange(1, N)], 1).ravel()
    return _code(rows, cols, rng.integers(1, q, size=2 * (N - 1)), N - 1, N, q)


@pytest.mark.parametrize("q", [2, 4, 8])
def test_sus_sweep_carries_information_along_column_order(oracle, q):
    """On a chain whose columns are numbered along it, one SUS sweep moves
    information from column 0 to column N-1 (each column uses the messages
    its predecessor updated in the same sweep), so Q_{N-1} is already the
    exact marginal; one PUS iteration only reaches one hop."""
    rng = np.random.default_rng(q)
    N = 6
    code = chain_code(N, q, rng)
    ll = rng.normal(0, 2.0, size=(1, N, q)).astype(np.float32)
    L = oracle.channel(q, "loglik", 0.0, ll[0])
    z = np.zeros(code.M, np.int64)
    want = exact_marginals(code, L, z)
    sus = oracle.decode(code, ll, "loglik", 0.0, "sus", max_iter=1, early_stop=False, post=True)["post"][0]
    pus = oracle.decode(code, ll, "loglik", 0.0, "pus", max_iter=1, early_stop=False, post=True)["post"][0]
    np.testing.assert_allclose(sus[N - 1], want[N - 1], atol=1e-12)
    assert np.abs(pus[N - 1] - want[N - 1]).max() > 1e-4
    assert np.abs(sus[0] - want[0]).max() > 1e-4


def peel(code, x, erased):
    """Classic peeling decoder over GF(q) for whole-symbol erasures."""
    q = code.q
    p = q.bit_length() - 1
    known = ~erased.copy()
    val = np.where(known, x.astype(np.int64), -1)
    inv = {a: next(b for b in range(1, q) if _gf.mul(a, b, p) == 1) for a in range(1, q)}
    checks = {}
    for r, c, h in zip(code.rows, code.cols, code.vals):
        checks.setdefault(int(r), []).append((int(c), int(h)))
    changed = True
    while changed:
        changed = False
        for i, edges in checks.items():
            unk = [(c, h) for c, h in edges if not known[c]]
            if len(unk) == 1:
                c, h = unk[0]
                s = 0
                for c2, h2 in edges:
                    if known[c2]:
                        s ^= _gf.mul(h2, int(val[c2]), p)
                val[c] = _gf.mul(inv[h], s, p)
                known[c] = True
                changed = True
    return known, val


@pytest.mark.parametrize("q", [4, 16])
@pytest.mark.parametrize("eps", [0.3, 0.45])
@pytest.mark.parametrize("schedule", ["pus", "sus"])
def test_bec_symbol_erasures_match_peeling(oracle, q, eps, schedule):
    from paper_cs_0605069_gb300 import workload as W
    code = W.regular_code(q, 96, cfg=f"peel{q}")
    p = code.p
    rng = np.random.default_rng(int(eps * 100) + q)
    F = 12
    x = W.encode(code, rng.integers(0, q, size=(F, code.K)))
    obs = W.to_bits(x, p).astype(np.float32)
    erased = rng.random((F, code.N)) < eps
    obs[erased] = 2.0
    out = oracle.decode(code, obs, "bec", eps, schedule, max_iter=80, early_stop=False, post=True)
    for f in range(F):
        known, val = peel(code, x[f], erased[f])
        det = out["post"][f].max(1) == 1.0
        np.testing.assert_array_equal(det, known)
        np.testing.assert_array_equal(out["xhat"][f][known], x[f][known])


@pytest.mark.parametrize("schedule", ["pus", "sus"])
def test_syndrome_form_is_relabelled_codeword_form(oracle, schedule):
    """Decoding H w = z with w = x + v (symbolwise XOR) and z = H v gives the
    messages of the codeword problem relabelled by a -> a + v_j (Sec. 2, Eq. 2)."""
    from paper_cs_0605069_gb300 import workload as W
    b = W.make_batch("gf4_n96_bsc005", frames=16)
    code = b.code
    rng = np.random.default_rng(5)
    v = rng.integers(0, code.q, size=(16, code.N))
    z = code.syndrome(v).astype(np.uint8)
    obs_w = (b.obs.astype(np.int64) ^ W.to_bits(v, code.p)).astype(np.float32)
    a = oracle.decode(code, b.obs, "bsc", b.param, schedule, max_iter=30, post=True)
    c = oracle.decode(code, obs_w, "bsc", b.param, schedule, max_iter=30, post=True, syn=z)
    np.testing.assert_array_equal(a["iters"], c["iters"])
    np.testing.assert_array_equal(a["conv"], c["conv"])
    for f in range(16):
        idx = np.arange(code.q)[None, :] ^ v[f][:, None]   # Q^w_j(a) = Q^x_j(a + v_j)
        np.testing.assert_allclose(c["post"][f], np.take_along_axis(a["post"][f], idx, 1), atol=1e-12)


@pytest.mark.parametrize("schedule", ["pus", "sus"])
@pytest.mark.parametrize("q", [2, 4])
def test_zero_sums_count_contradicted_posteriors(oracle, schedule, q):
    """One check x_0 + x_1 = z over two symbols observed without erasure as
    (0, 0), with z = 1: in every iteration the check tells each symbol the
    other value (r = delta at 1), each column's only message q_ij is its own
    likelihood (it meets no other check), and each posterior Q_j = p_j r_ij
    vanishes and falls back to uniform: two zero sums per iteration, the
    decisions (0, 0) (lowest symbol of a uniform posterior), never converged."""
    code = _code([0, 0], [0, 1], [1, 1], 1, 2, q)
    obs = np.zeros((1, 2, q.bit_length() - 1), np.float32)   # BEC, every bit seen as 0
    z = np.array([[1]], np.uint8)
    for T in (1, 3, 7):
        a = oracle.decode(code, obs, "bec", 0.0, schedule, max_iter=T, syn=z)
        assert a["zero_sums"][0] == 2 * T and a["iters"][0] == T and a["conv"][0] == 0
        np.testing.assert_array_equal(a["xhat"][0], [0, 0])
    a = oracle.decode(code, obs, "bec", 0.0, schedule, max_iter=5, syn=np.zeros((1, 1), np.uint8))
    assert a["zero_sums"][0] == 0 and a["iters"][0] == 1 and a["conv"][0] == 1


def test_converged_words_satisfy_all_checks(oracle):
    from paper_cs_0605069_gb300 import workload as W
    b = W.make_batch("gf4_n96_bsc005", frames=200)
    for s in ("pus", "sus"):
        out = oracle.decode(b.code, b.obs, "bsc", b.param, s, max_iter=100)
        assert (out["iters"] >= 1).all() and (out["iters"] <= 100).all()
        assert out["conv"].sum() > 150
        for f in np.nonzero(out["conv"])[0][:60]:
            z = _gf.syndrome(b.code.rows, b.code.cols, b.code.vals, b.code.M, out["xhat"][f], b.code.q)
            assert not any(z)
        for f in np.nonzero(out["conv"] == 0)[0]:
            assert out["iters"][f] == 100


def test_generator_codewords_satisfy_oracle_field(oracle):
    """The workload generator's encoder and the oracle's field agree: every
    transmitted word has zero syndrome under the oracle's tables."""
    from paper_cs_0605069_gb300 import workload as W
    for name in ("gf4_n96_bsc005", "gf16_n1000_awgn"):
        b = W.make_batch(name, frames=4)
        mul, _ = oracle.gf_tables(b.code.q)
        for f in range(4):
            z = np.zeros(b.code.M, np.int64)
            np.bitwise_xor.at(z, b.code.rows, mul[b.code.vals, b.x[f][b.code.cols]])
            assert not z.any()


@pytest.mark.parametrize("schedule", ["pus", "sus"])
@pytest.mark.parametrize("markov", [False, True])
def test_step_reproduces_decode(oracle, schedule, markov):
    """Iterating the one-step entry point from q_ij = p_j gives decode's
    trajectory: same hard decisions per iteration and the same stop."""
    from paper_cs_0605069_gb300 import workload as W
    if markov:
        code = W.regular_code(8, 96, cfg="step-markov")
        T = W.self_transition_chain(8, 0.8)
        rng = np.random.default_rng(1)
        x = W.encode(code, W.markov_source(rng.random((6, code.K)), T))
        obs = W.bsc(rng, x, 3, 0.12)
        K, param, kind = code.K, 0.12, "bsc"
    else:
        b = W.make_batch("gf4_n96_bsc005", frames=6)
        code, obs, T, K, param, kind = b.code, b.obs, None, 0, b.param, "bsc"
    ref = oracle.decode(code, obs, kind, param, schedule, max_iter=25, T=T, K=K, trace=True, post=True)
    msg = oracle.initial_messages(code, obs, kind, param, T=T, K=K)
    F = obs.shape[0]
    prior = None
    if markov:
        _, pi = oracle.markov(T, np.full((1, code.q), 1.0 / code.q))
        prior = np.broadcast_to(pi, (F, K, code.q)).copy()
    done = np.zeros(F, bool)
    for t in range(1, 26):
        st = oracle.step(code, obs, kind, param, msg, schedule, T=T, K=K, prior=prior)
        msg = st["msg"]
        for f in range(F):
            if done[f]:
                continue
            np.testing.assert_array_equal(st["xhat"][f], ref["trace_x"][f, t - 1])
            if st["sat"][f]:
                done[f] = True
                assert ref["iters"][f] == t and ref["conv"][f] == 1
                np.testing.assert_allclose(st["post"][f], ref["post"][f], atol=1e-12)
        if markov:
            prior = st["prior_out"]
        if done.all():
            break


def _support_propagation(code, C, z, schedule, iters):
    """BP on the BEC as set propagation: every message is uniform over its
    support, a coset of GF(2)^p.  Check node: the support of x_j given the
    others is h_j^-1 (z XOR the sumset of h_j' supp(q_j')); variable node:
    the intersection of the channel's consistent set with the other checks'
    supports.  Returns the posterior supports after each iteration."""
    q = code.q
    p = q.bit_length() - 1
    M, N = code.M, code.N
    rows, cols, vals = (np.asarray(a) for a in (code.rows, code.cols, code.vals))
    E = len(rows)
    mul = [[_gf.mul(a, b, p) for b in range(q)] for a in range(q)]
    inv = [0] + [next(b for b in range(1, q) if mul[a][b] == 1) for a in range(1, q)]
    edges_of_row = [[e for e in range(E) if rows[e] == i] for i in range(M)]
    edges_of_col = [[e for e in range(E) if cols[e] == j] for j in range(N)]
    Qs = [set(C[cols[e]]) for e in range(E)]     # q_ij <- p_j
    R = [set(range(q)) for _ in range(E)]

    def check(e):
        i = rows[e]
        s = {int(z[i])}
        for e2 in edges_of_row[i]:
            if e2 != e:
                s = {a ^ mul[int(vals[e2])][b] for a in s for b in Qs[e2]}
        return {mul[inv[int(vals[e])]][a] for a in s}

    def var(j):
        for e in edges_of_col[j]:
            s = set(C[j])
            for e2 in edges_of_col[j]:
                if e2 != e:
                    s &= R[e2]
            Qs[e] = s

    def post(j):
        s = set(C[j])
        for e in edges_of_col[j]:
            s &= R[e]
        return s

    out = []
    for _ in range(iters):
        P = [None] * N
        if schedule == "pus":
            R = [check(e) for e in range(E)]
            for j in range(N):
                var(j)
                P[j] = post(j)
        else:
            for j in range(N):
                for e in edges_of_col[j]:
                    R[e] = check(e)
                P[j] = post(j)
                var(j)
        out.append(P)
    return out


# (q, N, erasure rate, seed): cases where decoding progresses over several
# iterations and the two schedules' support trajectories differ
BEC_COSET_CASES = [(4, 48, 0.35, 0), (8, 36, 0.30, 5)]


@pytest.mark.parametrize("q,N,eps,seed", BEC_COSET_CASES)
@pytest.mark.parametrize("schedule", ["pus", "sus"])
def test_bec_bit_erasures_follow_coset_propagation(oracle, q, N, eps, seed, schedule):
    """On a loopy code under random bit erasures every BP posterior is uniform
    over the support that set propagation predicts, iteration by iteration,
    in the schedule's own update order (the two orders' trajectories differ
    here, so the pin tells them apart)."""
    from paper_cs_0605069_gb300 import workload as W
    code = W.regular_code(q, N, cfg=f"bec_cosets_{q}_{N}", encodable=False)
    rng = np.random.default_rng(1000 * seed + q * N)
    p = q.bit_length() - 1
    x = rng.integers(0, q, size=N)
    z = np.asarray(_gf.syndrome(code.rows, code.cols, code.vals, code.M, x, q), np.int64)
    bits = ((x[:, None] >> np.arange(p)[None, :]) & 1).astype(np.float32)
    bits[rng.random(bits.shape) < eps] = 2.0
    C = [{a for a in range(q) if all(bits[j, k] == 2.0 or ((a >> k) & 1) == bits[j, k] for k in range(p))}
         for j in range(N)]
    iters = 6
    want = _support_propagation(code, C, z, schedule, iters)
    other = _support_propagation(code, C, z, "sus" if schedule == "pus" else "pus", iters)
    assert want != other
    msg = oracle.initial_messages(code, bits[None], "bec", eps)
    for t in range(iters):
        r = oracle.step(code, bits[None], "bec", eps, msg, schedule, syn=z[None].astype(np.uint8))
        for j in range(N):
            S = want[t][j]
            assert x[j] in S
            expect = np.array([1.0 / len(S) if a in S else 0.0 for a in range(q)])
            np.testing.assert_allclose(r["post"][0, j], expect, rtol=0, atol=1e-12, err_msg=f"t={t} j={j}")
        msg = r["msg"]
