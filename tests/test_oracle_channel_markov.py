"""Pins of the oracle's channel likelihoods (Sec. 2) and Markov priors (Eqs. 6-7)."""
import os

import numpy as np
import pytest
from scipy.stats import norm

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("q", [2, 4, 8, 16, 256])
@pytest.mark.parametrize("f", [0.01, 0.155, 0.23])
def test_bsc_noise_symbol_formula(oracle, q, f):
    """Sec. 2: Q_j^a = f^L (1-f)^(log2 q - L), L = number of 1 bits of a,
    for a received all-zero symbol; with received bits y, L counts a XOR y."""
    p = q.bit_length() - 1
    L = np.array([bin(a).count("1") for a in range(q)])
    want = f ** L * (1 - f) ** (p - L)
    got = oracle.channel(q, "bsc", f, np.zeros((1, p), np.float32))[0]
    np.testing.assert_allclose(got, want / want.sum(), rtol=1e-13, atol=0)
    y = 5 % q
    bits = np.array([(y >> k) & 1 for k in range(p)], np.float32)
    Ly = np.array([bin(a ^ y).count("1") for a in range(q)])
    want = f ** Ly * (1 - f) ** (p - Ly)
    got = oracle.channel(q, "bsc", f, bits[None])[0]
    np.testing.assert_allclose(got, want / want.sum(), rtol=1e-13, atol=0)


@pytest.mark.parametrize("q", [4, 8, 16])
def test_bec_uniform_over_consistent_symbols(oracle, q):
    p = q.bit_length() - 1
    rng = np.random.default_rng(q)
    for _ in range(20):
        a0 = int(rng.integers(q))
        y = np.array([(a0 >> k) & 1 for k in range(p)], np.float32)
        y[rng.random(p) < 0.5] = 2.0
        got = oracle.channel(q, "bec", 0.5, y[None])[0]
        ok = np.array([all(y[k] == 2 or ((a >> k) & 1) == y[k] for k in range(p)) for a in range(q)])
        np.testing.assert_array_equal(got, ok / ok.sum())


@pytest.mark.parametrize("q", [2, 16, 256])
@pytest.mark.parametrize("sigma", [0.5, 0.84, 1.66])
def test_biawgn_gaussian_product(oracle, q, sigma):
    p = q.bit_length() - 1
    rng = np.random.default_rng(3)
    y = rng.normal(0, 1.5, size=p).astype(np.float32)
    s = np.array([[1.0 - 2.0 * ((a >> k) & 1) for k in range(p)] for a in range(q)])
    want = np.prod(norm.pdf(y.astype(np.float64)[None, :], loc=s, scale=sigma), axis=1)
    got = oracle.channel(q, "awgn", sigma, y[None])[0]
    np.testing.assert_allclose(got, want / want.sum(), rtol=1e-11, atol=1e-300)


def test_punctured_and_loglik(oracle):
    q = 8
    got = oracle.channel(q, "bsc", 0.1, np.ones((2, 3), np.float32), punct=np.array([1, 0], np.uint8))
    np.testing.assert_allclose(got[0], np.full(q, 1.0 / q))
    ll = np.log(np.arange(1, q + 1, dtype=np.float64)).astype(np.float32)
    got = oracle.channel(q, "loglik", 0.0, ll[None])[0]
    want = np.exp(ll.astype(np.float64))
    np.testing.assert_allclose(got, want / want.sum(), rtol=1e-12)


def test_markov_hand_worked_example(oracle):
    rows = np.loadtxt(os.path.join(GOLDEN, "markov_q2_hand.txt"))
    T = np.array([[0.9, 0.1], [0.3, 0.7]])
    Q = np.array([[0.6, 0.4], [0.3, 0.7], [0.2, 0.8]])
    for form in (6, 7):
        P, pi = oracle.markov(T, Q, form=form)
        np.testing.assert_allclose(pi, [0.75, 0.25], atol=1e-15)
        np.testing.assert_allclose(P, rows[:, 1:], atol=1e-14)


@pytest.mark.parametrize("q", [2, 3, 4, 8, 16])
def test_eq6_equals_eq7(oracle, q):
    rng = np.random.default_rng(q)
    T = rng.random((q, q)) + 0.05
    Q = rng.random((7, q))
    Q /= Q.sum(1, keepdims=True)
    P6, _ = oracle.markov(T, Q, form=6)
    P7, _ = oracle.markov(T, Q, form=7)
    np.testing.assert_allclose(P6, P7, rtol=0, atol=1e-15)
    np.testing.assert_allclose(P6.sum(1), 1.0, atol=1e-15)


def _stationary_by_eig(T):
    T = np.asarray(T, float)
    T = T / T.sum(1, keepdims=True)
    w, v = np.linalg.eig(T.T)
    x = np.real(v[:, np.argmin(abs(w - 1))])
    return x / x.sum()


def test_stationary_distributions(oracle):
    from paper_cs_0605069_gb300.workload import MARKOV_2S, MARKOV_4S, self_transition_chain
    one = np.full((1, 2), 0.5)
    _, pi2 = oracle.markov(MARKOV_2S, one)
    np.testing.assert_allclose(pi2, [0.5, 0.5], atol=1e-15)
    _, pi4 = oracle.markov(MARKOV_4S, np.full((1, 4), 0.25))
    np.testing.assert_allclose(pi4, _stationary_by_eig(MARKOV_4S), atol=1e-12)
    np.testing.assert_allclose(pi4, [0.7625, 0.0764, 0.0284, 0.1328], atol=6e-5)
    T = MARKOV_4S / MARKOV_4S.sum(1, keepdims=True)
    np.testing.assert_allclose(pi4 @ T, pi4, atol=1e-15)
    _, pi8 = oracle.markov(self_transition_chain(8, 0.8), np.full((1, 8), 1 / 8))
    np.testing.assert_allclose(pi8, np.full(8, 1 / 8), atol=1e-15)


def test_single_source_position_gets_pi(oracle):
    T = np.array([[0.9, 0.1], [0.3, 0.7]])
    P, _ = oracle.markov(T, np.array([[0.1, 0.9]]))
    np.testing.assert_allclose(P[0], [0.75, 0.25], atol=1e-15)
