"""Pins of the oracle's decode loop where it uses the dynamical block priors
(Sec. 2: the priors of the source symbols are re-estimated after every
iteration by Eq. 6 from the pseudo-posteriors of Eq. 5 and used in the next
iteration) and of its hard decision ("clipping", lowest symbol among equal
maxima).

On a code whose source columns meet no check, BP leaves a source symbol's
pseudo-posterior at its prior belief: Q_j = p_j = normalise(L_j P_j) exactly,
with L_j the channel likelihood and P_j its block prior.  The trajectory of
the block priors then follows from Eq. 6 alone, which the test writes out in
numpy with an independently computed stationary distribution.  That fixes:
the initial prior (pi, before the first iteration), the Jacobi timing (P used
in iteration t comes from the Q of iteration t-1), the orientation of the
transition matrix on both sides, the boundaries, the use of the full Q
rather than an extrinsic one, and the mapping of source index to column
through a non-identity src_pos.
"""
import numpy as np
import pytest

from paper_cs_0605069_gb300 import workload as W


def _bsc_likelihood(q, f, bits):
    """Sec. 2 BSC likelihood of every symbol for received bits [p]."""
    p = q.bit_length() - 1
    L = np.ones(q)
    for a in range(q):
        for k in range(p):
            L[a] *= (1 - f) if ((a >> k) & 1) == bits[k] else f
    return L / L.sum()


def _stationary_eig(T):
    """Left eigenvector of T for eigenvalue 1 (numpy eig; the oracle solves a
    linear system instead)."""
    w, v = np.linalg.eig(T.T)
    pi = np.real(v[:, np.argmin(np.abs(w - 1.0))])
    return pi / pi.sum()


def _eq6(T, pi, Qm, Qp):
    """Eq. 6 for one source symbol: P^b ∝ (sum_a Qm^a T_ab)(sum_c T_bc Qp^c),
    with pi_b for the missing left neighbour and 1 for the missing right one."""
    left = pi if Qm is None else Qm @ T
    right = np.ones(len(pi)) if Qp is None else T @ Qp
    P = left * right
    return P / P.sum()


def _free_source_code(q, K):
    """K source columns that meet no check, then two columns joined by one
    check (so the code has a check at all)."""
    H = np.zeros((1, K + 2), np.int64)
    H[0, K] = 1
    H[0, K + 1] = 1
    return W.code_from_dense(H, q)


@pytest.mark.parametrize("q,schedule", [(2, "pus"), (4, "sus"), (8, "pus"), (8, "sus")])
def test_markov_prior_trajectory_on_free_source_symbols(oracle, q, schedule):
    rng = np.random.default_rng(100 + q)
    K = 7
    code = _free_source_code(q, K)
    p = code.p
    f = 0.2
    # an asymmetric chain: a transposed matrix gives other priors
    T = rng.random((q, q)) + 0.05
    T[np.arange(q), (np.arange(q) + 1) % q] += 2.0
    T /= T.sum(1, keepdims=True)
    pi = _stationary_eig(T)
    src_pos = np.array([4, 0, 6, 2, 5, 1, 3], np.int32)   # source order != column order
    F = 3
    obs = rng.integers(0, 2, size=(F, K + 2, p)).astype(np.float32)
    obs[:, K:] = 0.0
    for t_max in range(1, 5):
        out = oracle.decode(code, obs, "bsc", f, schedule, max_iter=t_max, T=T, K=K, src_pos=src_pos,
                            early_stop=False, post=True)
        for fr in range(F):
            L = np.array([_bsc_likelihood(q, f, obs[fr, j].astype(int)) for j in range(K)])
            P = np.tile(pi, (K, 1))   # block priors in use during the first iteration
            for t in range(1, t_max + 1):
                Q = np.zeros((K, q))
                for i in range(K):
                    x = L[src_pos[i]] * P[i]
                    Q[i] = x / x.sum()
                if t < t_max:   # re-estimated after the iteration, for the next one
                    P = np.array([_eq6(T, pi, Q[i - 1] if i > 0 else None, Q[i + 1] if i < K - 1 else None)
                                  for i in range(K)])
            got = out["post"][fr][src_pos]
            np.testing.assert_allclose(got, Q, rtol=0, atol=1e-12,
                                       err_msg=f"t_max={t_max} frame {fr}")


def test_markov_pin_detects_a_prior_updated_one_iteration_early(oracle):
    """The trajectory test above would fail for a decoder that re-estimated
    the priors before the first iteration: the two readings differ."""
    q, K, f = 4, 5, 0.2
    rng = np.random.default_rng(3)
    code = _free_source_code(q, K)
    T = rng.random((q, q)) + 0.1
    T /= T.sum(1, keepdims=True)
    pi = _stationary_eig(T)
    obs = rng.integers(0, 2, size=(1, K + 2, 2)).astype(np.float32)
    obs[:, K:] = 0.0
    out = oracle.decode(code, obs, "bsc", f, "pus", max_iter=1, T=T, K=K, early_stop=False, post=True)
    L = np.array([_bsc_likelihood(q, f, obs[0, j].astype(int)) for j in range(K)])
    Q0 = L * pi / (L * pi).sum(1, keepdims=True)
    early = np.array([_eq6(T, pi, Q0[i - 1] if i > 0 else None, Q0[i + 1] if i < K - 1 else None)
                      for i in range(K)])
    wrong = L * early / (L * early).sum(1, keepdims=True)
    assert np.abs(out["post"][0][:K] - Q0).max() < 1e-12
    assert np.abs(wrong - Q0).max() > 1e-3


@pytest.mark.parametrize("schedule", ["pus", "sus"])
def test_hard_decision_takes_the_lowest_of_equal_maxima(oracle, schedule):
    """Bit erasures on columns that meet no check leave exact ties in Q:
    GF(4) bit 0 erased, bit 1 = 1 -> {2, 3}; GF(8) bits 0 and 2 erased, bit 1 =
    1 -> {2, 3, 6, 7}; every bit erased -> all symbols.  Clipping picks the
    lowest tied symbol."""
    for q, bits, want in [(4, [2, 1], 2), (8, [2, 1, 2], 2), (8, [2, 2, 2], 0), (4, [1, 2], 1)]:
        code = _free_source_code(q, 3)
        p = code.p
        obs = np.zeros((1, 5, p), np.float32)
        obs[0, :3] = np.array(bits, np.float32)
        out = oracle.decode(code, obs, "bec", 0.5, schedule, max_iter=3, post=True)
        Q = out["post"][0]
        assert Q[0].max() == Q[0][want], (q, bits)
        assert (out["xhat"][0, :3] == want).all(), (q, bits, out["xhat"][0])


@pytest.mark.parametrize("q", [2, 4, 8])
def test_gauss_seidel_prior_trajectory_on_free_source_symbols(oracle, q):
    """Markov priors re-estimated inside the SUS sweep: when the sweep reaches
    the column of source symbol i, P_i follows Eq. 6 from its neighbours'
    pseudo-posteriors as they stand (already updated in this sweep when their
    column came earlier, else from the previous sweep, or their initial belief
    L pi before their first visit); on columns that meet no check Q_j =
    normalise(L_j P_j)."""
    rng = np.random.default_rng(200 + q)
    K = 7
    code = _free_source_code(q, K)
    p = code.p
    f = 0.2
    T = rng.random((q, q)) + 0.05
    T[np.arange(q), (np.arange(q) + 1) % q] += 2.0
    T /= T.sum(1, keepdims=True)
    pi = _stationary_eig(T)
    src_pos = np.array([4, 0, 6, 2, 5, 1, 3], np.int32)
    src_index = {int(j): i for i, j in enumerate(src_pos)}
    F = 3
    obs = rng.integers(0, 2, size=(F, K + 2, p)).astype(np.float32)
    obs[:, K:] = 0.0
    for t_max in range(1, 4):
        out = oracle.decode(code, obs, "bsc", f, "sus", max_iter=t_max, T=T, K=K, src_pos=src_pos,
                            early_stop=False, post=True, gauss_seidel=True)
        jac = oracle.decode(code, obs, "bsc", f, "sus", max_iter=t_max, T=T, K=K, src_pos=src_pos,
                            early_stop=False, post=True)
        for fr in range(F):
            L = np.array([_bsc_likelihood(q, f, obs[fr, j].astype(int)) for j in range(K)])
            Qc = L * pi / (L * pi).sum(1, keepdims=True)   # by column, initial beliefs
            for _ in range(t_max):
                for j in range(K):                           # the sweep, in column order
                    i = src_index[j]
                    Qm = Qc[src_pos[i - 1]] if i > 0 else None
                    Qp = Qc[src_pos[i + 1]] if i < K - 1 else None
                    P = _eq6(T, pi, Qm, Qp)
                    x = L[j] * P
                    Qc[j] = x / x.sum()
            np.testing.assert_allclose(out["post"][fr][:K], Qc, rtol=0, atol=1e-12, err_msg=f"t_max={t_max}")
            if t_max == 1:
                # the Jacobi reading uses pi throughout the first iteration
                assert np.abs(jac["post"][fr][:K] - Qc).max() > 1e-6


def test_gauss_seidel_is_refused_for_pus(oracle):
    code = _free_source_code(4, 3)
    obs = np.zeros((1, 5, 2), np.float32)
    T = np.full((4, 4), 0.25)
    with pytest.raises(ValueError):
        oracle.decode(code, obs, "bsc", 0.1, "pus", max_iter=2, T=T, K=3, gauss_seidel=True)
