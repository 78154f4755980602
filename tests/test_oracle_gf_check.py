"""Pins of the oracle's field arithmetic and horizontal pass (Eq. 3).

The field is pinned to shift-and-add multiplication written in the test and to
the field axioms; Eq. 3 is pinned to its definition (enumeration of every
configuration of the other symbols of a check), to the q = 2 closed form
(product of differences), and to special cases.
"""
import itertools

import numpy as np
import pytest

from tests import _gf


@pytest.mark.parametrize("q", [2, 4, 8, 16, 32, 64, 128, 256])
def test_field_tables_match_shift_and_add(oracle, q):
    mul, inv = oracle.gf_tables(q)
    ref = np.array(_gf.table(q))
    assert (mul == ref).all()
    for a in range(1, q):
        assert mul[a, inv[a]] == 1


@pytest.mark.parametrize("q", [2, 4, 8, 16, 64, 256])
def test_field_axioms_exhaustive(oracle, q):
    mul, inv = oracle.gf_tables(q)
    a = np.arange(q)
    A, B, Cc = np.meshgrid(a, a, a, indexing="ij")
    assert (mul[mul[A, B], Cc] == mul[A, mul[B, Cc]]).all()          # associativity
    assert (mul[A, B ^ Cc] == (mul[A, B] ^ mul[A, Cc])).all()         # distributivity over XOR
    assert (mul == mul.T).all()                                      # commutativity
    assert (mul[1] == a).all() and (mul[0] == 0).all()                # identities
    nz = mul[1:, 1:]
    assert (nz != 0).all()                                           # no zero divisors
    for r in nz:
        assert sorted(r.tolist()) == list(range(1, q))                # rows are permutations


@pytest.mark.parametrize("q", [4, 8, 16, 32, 64, 128, 256])
def test_field_generator_is_primitive(oracle, q):
    mul, _ = oracle.gf_tables(q)
    x, v, order = 2, 2, 1
    while v != 1:
        v = mul[v, x]
        order += 1
    assert order == q - 1


def test_non_primitive_polynomial_rejected(oracle):
    # x^4+x^3+x^2+x+1 is irreducible but x has order 5 in it.
    with pytest.raises(ValueError):
        oracle.gf_tables(16, 0x1F)


def _brute_force_check(q, h, z, qin):
    """Eq. 3 literally: for x_k = a, sum over every configuration of the
    other symbols that satisfies sum_m h_m x_m = z of the product of their q's."""
    p = q.bit_length() - 1
    d = len(h)
    r = np.zeros((d, q))
    for k in range(d):
        others = [m for m in range(d) if m != k]
        for a in range(q):
            tot = 0.0
            for conf in itertools.product(range(q), repeat=len(others)):
                s = _gf.mul(h[k], a, p)
                w = 1.0
                for m, xm in zip(others, conf):
                    s ^= _gf.mul(h[m], xm, p)
                    w *= qin[m][xm]
                if s == z:
                    tot += w
            r[k, a] = tot
        r[k] /= r[k].sum()
    return r


def _random_messages(rng, d, q, kind):
    qin = rng.random((d, q))
    if kind == "zeros":
        qin[rng.random((d, q)) < 0.3] = 0.0
        qin[:, 0] += 0.1
    elif kind == "onehot":
        qin[0] = 0.0
        qin[0, rng.integers(q)] = 1.0
    elif kind == "tiny":
        qin[:, 1:] *= 1e-30
    return qin / qin.sum(1, keepdims=True)


@pytest.mark.parametrize("q,d", [(2, 1), (2, 2), (2, 6), (4, 2), (4, 3), (4, 5), (8, 3), (8, 4)])
@pytest.mark.parametrize("kind", ["random", "zeros", "onehot", "tiny"])
def test_check_matches_configuration_sum(oracle, q, d, kind):
    rng = np.random.default_rng(1000 * q + 10 * d + len(kind))
    for trial in range(3):
        h = rng.integers(1, q, size=d)
        z = int(rng.integers(q))
        qin = _random_messages(rng, d, q, kind)
        ref = _brute_force_check(q, list(h), z, qin)
        got = oracle.check(q, h, z, qin)
        np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12)
        got_wht = oracle.check(q, h, z, qin, use_wht=True)
        np.testing.assert_allclose(got_wht, ref, rtol=0, atol=1e-12)


@pytest.mark.parametrize("d", [2, 3, 6, 10])
@pytest.mark.parametrize("z", [0, 1])
def test_check_binary_closed_form(oracle, d, z):
    """q = 2: r^0 - r^1 = (-1)^z prod_{m != k} (q_m^0 - q_m^1)."""
    rng = np.random.default_rng(d)
    qin = rng.random((d, 2))
    qin /= qin.sum(1, keepdims=True)
    r = oracle.check(2, np.ones(d, int), z, qin)
    diff = qin[:, 0] - qin[:, 1]
    for k in range(d):
        want = (-1) ** z * np.prod(np.delete(diff, k))
        assert abs((r[k, 0] - r[k, 1]) - want) < 1e-14


@pytest.mark.parametrize("q", [4, 16, 256])
def test_degree_one_check_forces_symbol(oracle, q):
    """A check with one symbol forces h x = z, i.e. x = h^-1 z."""
    mul, inv = oracle.gf_tables(q)
    for h in (1, 2, q - 1):
        for z in (0, 1, q - 1):
            r = oracle.check(q, [h], z, np.full((1, q), 1.0 / q))
            want = np.zeros(q)
            want[mul[inv[h], z]] = 1.0
            np.testing.assert_array_equal(r[0], want)


@pytest.mark.parametrize("q", [16, 32, 64, 128, 256])
def test_transform_route_equals_direct_route(oracle, q):
    rng = np.random.default_rng(q)
    d = 6
    h = rng.integers(1, q, size=d)
    qin = rng.random((d, q)) ** 4
    qin /= qin.sum(1, keepdims=True)
    a = oracle.check(q, h, 3, qin)
    b = oracle.check(q, h, 3, qin, use_wht=True)
    np.testing.assert_allclose(a, b, rtol=0, atol=1e-13)


@pytest.mark.parametrize("q", [4, 8, 16])
def test_check_uniform_neighbour_gives_uniform(oracle, q):
    """If any other symbol of the check is uniform, its sum hides the rest."""
    rng = np.random.default_rng(7)
    qin = rng.random((4, q))
    qin /= qin.sum(1, keepdims=True)
    qin[2] = 1.0 / q
    r = oracle.check(q, rng.integers(1, q, size=4), 1, qin)
    for k in (0, 1, 3):
        np.testing.assert_allclose(r[k], np.full(q, 1.0 / q), atol=1e-15)
