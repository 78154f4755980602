"""Seeded synthetic workloads for GF(q) LDPC decoding.

This module only makes inputs: parity-check matrices, source words,
codewords and channel observations.  It holds no step of the decoder
(no likelihoods, no messages, no priors); the CUDA library and the FP64
oracle both take what it produces as plain arrays.

Workload shapes follow the paper's experiments (Sec. 3): LDPC codes over
GF(q=2^p) whose non-zero entries are uniform in {1..q-1} (Sec. 2), i.i.d.
or Markov sources (Sec. 3 and its footnote matrices), binary images of the
symbols sent over a BSC, a BEC or a BI-AWGN channel (Sec. 2, Eq. 1 and the
footnote on other channels).  The paper's Kanter-Saad construction is not
given in the paper, so regular (d_v, d_c) codes built from a random socket
permutation stand in for it.

GF(2^p) arithmetic here is a bitwise carry-less multiply reduced by the
field polynomial; it is used only to encode and to compute syndromes of
generated words.
"""
from __future__ import annotations

import hashlib
from dataclasses import dataclass, field

import numpy as np

# Primitive polynomials (bit k = coefficient of x^k), one per field size.
FIELD_POLY = {1: 0x3, 2: 0x7, 3: 0xB, 4: 0x13, 5: 0x25, 6: 0x43, 7: 0x89, 8: 0x11D}


def log2q(q: int) -> int:
    p = int(q).bit_length() - 1
    if q < 2 or (1 << p) != q or p > 8:
        raise ValueError(f"q must be 2^p with 1 <= p <= 8, got {q}")
    return p


def gf_mul_bitwise(a, b, p: int, poly: int):
    """Carry-less product of a and b reduced modulo poly (numpy arrays or ints)."""
    a = np.asarray(a, dtype=np.int64)
    b = np.asarray(b, dtype=np.int64)
    acc = np.zeros(np.broadcast(a, b).shape, dtype=np.int64)
    aa = np.broadcast_to(a, acc.shape).copy()
    for k in range(p):
        acc ^= np.where((b >> k) & 1, aa, 0)
        aa <<= 1
        aa = np.where(aa & (1 << p), aa ^ poly, aa)
    return acc


def gf_mul_table(q: int, poly: int | None = None) -> np.ndarray:
    p = log2q(q)
    poly = FIELD_POLY[p] if poly is None else poly
    a = np.arange(q)[:, None]
    b = np.arange(q)[None, :]
    return gf_mul_bitwise(a, b, p, poly).astype(np.uint8)


def rng_for(cfg: str, role: str, index: int = 0) -> np.random.Generator:
    """Independent, reproducible stream for (workload, role, index)."""
    h = hashlib.sha256(f"{cfg}|{role}|{index}".encode()).digest()
    words = [int.from_bytes(h[i:i + 4], "little") for i in range(0, 32, 4)]
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence(words)))


@dataclass
class Code:
    """Sparse parity-check matrix H over GF(q) in COO form, sorted by (row, col).

    When `enc` is set the code is systematic: columns 0..K-1 carry the
    information symbols and the last M columns the parity symbols, and
    `enc` is the binary (M*p x K*p) matrix that maps information bits to
    parity bits (bit k of a symbol is (a >> k) & 1).
    """
    q: int
    M: int
    N: int
    rows: np.ndarray
    cols: np.ndarray
    vals: np.ndarray
    poly: int
    K: int = 0
    enc: np.ndarray | None = field(default=None, repr=False)

    @property
    def p(self) -> int:
        return log2q(self.q)

    @property
    def E(self) -> int:
        return int(self.rows.size)

    def dense(self) -> np.ndarray:
        H = np.zeros((self.M, self.N), dtype=np.int64)
        H[self.rows, self.cols] = self.vals
        return H

    def syndrome(self, x: np.ndarray) -> np.ndarray:
        """z = H x over GF(q) for words x of shape [F, N]; returns [F, M]."""
        x = np.atleast_2d(np.asarray(x, dtype=np.int64))
        prod = gf_mul_bitwise(self.vals[None, :], x[:, self.cols], self.p, self.poly)
        z = np.zeros((x.shape[0], self.M), dtype=np.int64)
        for e in range(self.E):  # XOR-accumulate per edge, vectorised over frames
            z[:, self.rows[e]] ^= prod[:, e]
        return z


def _sort_coo(rows, cols, vals):
    order = np.lexsort((cols, rows))
    return rows[order].astype(np.int32), cols[order].astype(np.int32), vals[order].astype(np.int32)


def _count_local_4cycles(c, chk, var):
    """4-cycles through check c: sum over other checks c' of C(|N(c) & N(c')|, 2)."""
    cnt = {}
    for v in chk[c]:
        for c2 in var[v]:
            if c2 != c:
                cnt[c2] = cnt.get(c2, 0) + 1
    return sum(k * (k - 1) // 2 for k in cnt.values()), cnt


def _edges_in_4cycles(chk, var):
    bad = []
    for c in range(len(chk)):
        _, cnt = _count_local_4cycles(c, chk, var)
        shared = {c2 for c2, k in cnt.items() if k >= 2}
        if not shared:
            continue
        for v in chk[c]:
            if any(c2 in shared for c2 in var[v] if c2 != c):
                bad.append((c, v))
    return bad


def regular_graph(N: int, dv: int, dc: int, rng: np.random.Generator, swap_budget_per_edge: int = 100):
    """Random (dv, dc)-regular bipartite graph without multi-edges; 4-cycles
    removed by swaps that strictly lower their count, while the budget lasts."""
    if (N * dv) % dc:
        raise ValueError("N*dv must be divisible by dc")
    M = N * dv // dc
    E = N * dv
    var_sock = np.repeat(np.arange(N), dv)
    for _attempt in range(1000):
        perm = rng.permutation(E)
        vs = var_sock[perm].reshape(M, dc)
        chk = [list(r) for r in vs]
        # repair multi-edges by swapping with random sockets
        ok = True
        for _ in range(100 * E):
            dup = next(((c, k) for c in range(M) for k in range(dc) if chk[c].count(chk[c][k]) > 1), None)
            if dup is None:
                break
            c, k = dup
            c2 = int(rng.integers(M))
            k2 = int(rng.integers(dc))
            v, v2 = chk[c][k], chk[c2][k2]
            if c2 != c and v2 not in chk[c] and v not in chk[c2]:
                chk[c][k], chk[c2][k2] = v2, v
        else:
            ok = False
        if ok:
            break
    else:
        raise RuntimeError("could not build a simple regular graph")
    var = [[] for _ in range(N)]
    for c in range(M):
        for v in chk[c]:
            var[v].append(c)
    budget = swap_budget_per_edge * E
    while budget > 0:
        bad = _edges_in_4cycles(chk, var)
        if not bad:
            break
        improved = False
        for (c1, v1) in bad:
            if budget <= 0:
                break
            budget -= 1
            if v1 not in chk[c1]:
                continue
            c2 = int(rng.integers(M))
            v2 = chk[c2][int(rng.integers(dc))]
            if c2 == c1 or v2 == v1 or v2 in chk[c1] or v1 in chk[c2]:
                continue
            before = _count_local_4cycles(c1, chk, var)[0] + _count_local_4cycles(c2, chk, var)[0]
            _swap(chk, var, c1, v1, c2, v2)
            after = _count_local_4cycles(c1, chk, var)[0] + _count_local_4cycles(c2, chk, var)[0]
            if after < before:
                improved = True
            else:
                _swap(chk, var, c1, v2, c2, v1)
        if not improved and budget <= 0:
            break
    rows = np.array([c for c in range(M) for _ in chk[c]], dtype=np.int64)
    cols = np.array([v for c in range(M) for v in chk[c]], dtype=np.int64)
    return M, rows, cols


def _swap(chk, var, c1, v1, c2, v2):
    """Replace edges (c1,v1),(c2,v2) by (c1,v2),(c2,v1)."""
    chk[c1][chk[c1].index(v1)] = v2
    chk[c2][chk[c2].index(v2)] = v1
    var[v1][var[v1].index(c1)] = c2
    var[v2][var[v2].index(c2)] = c1


def count_4cycles(rows, cols, M, N) -> int:
    chk = [[] for _ in range(M)]
    var = [[] for _ in range(N)]
    for r, c in zip(rows, cols):
        chk[int(r)].append(int(c))
        var[int(c)].append(int(r))
    total = sum(_count_local_4cycles(c, chk, var)[0] for c in range(M))
    return total // 2


def _mul_matrix(h: int, p: int, poly: int) -> np.ndarray:
    """Binary p x p matrix of y = h*x over GF(2^p): column k = bits of h * x^k."""
    Mx = np.zeros((p, p), dtype=np.uint8)
    for k in range(p):
        v = int(gf_mul_bitwise(h, 1 << k, p, poly))
        for b in range(p):
            Mx[b, k] = (v >> b) & 1
    return Mx


def _binary_image(q, M, N, rows, cols, vals, poly) -> np.ndarray:
    p = log2q(q)
    Hb = np.zeros((M * p, N * p), dtype=np.uint8)
    cache = {}
    for r, c, h in zip(rows, cols, vals):
        h = int(h)
        if h not in cache:
            cache[h] = _mul_matrix(h, p, poly)
        Hb[r * p:(r + 1) * p, c * p:(c + 1) * p] = cache[h]
    return Hb


def _rref_gf2(Hb: np.ndarray, col_order: np.ndarray):
    """Reduced row echelon form over GF(2) of a bit matrix, pivots taken in col_order.
    Returns (packed reduced rows, pivot columns per row)."""
    R, C = Hb.shape
    W = np.packbits(Hb, axis=1, bitorder="little").view(np.uint8)
    nbytes = W.shape[1]
    pad = (-nbytes) % 8
    W = np.concatenate([W, np.zeros((R, pad), np.uint8)], axis=1).view(np.uint64).copy()
    piv = []
    r = 0
    for c in col_order:
        if r == R:
            break
        word, bit = divmod(int(c), 64)
        colbits = (W[:, word] >> np.uint64(bit)) & np.uint64(1)
        cand = np.nonzero(colbits[r:])[0]
        if cand.size == 0:
            continue
        pr = r + int(cand[0])
        if pr != r:
            W[[r, pr]] = W[[pr, r]]
        colbits = (W[:, word] >> np.uint64(bit)) & np.uint64(1)
        mask = colbits.astype(bool)
        mask[r] = False
        W[mask] ^= W[r]
        piv.append(int(c))
        r += 1
    return W[:r], piv


def systematic(q, M, N, rows, cols, vals, poly):
    """Relabel columns so that the last M columns of H are invertible and
    return (rows, cols, vals, K, enc) of the relabelled code; None if H is
    rank deficient."""
    p = log2q(q)
    Hb = _binary_image(q, M, N, rows, cols, vals, poly)
    # pivot search from the last symbol column backwards, whole symbols at a time
    order = np.concatenate([np.arange(c * p, (c + 1) * p) for c in range(N - 1, -1, -1)])
    W, piv = _rref_gf2(Hb, order)
    if len(piv) != M * p:
        return None
    piv_sym = sorted({c // p for c in piv})
    if len(piv_sym) != M or any(sum(1 for c in piv if c // p == s) != p for s in piv_sym):
        return None
    info_sym = [s for s in range(N) if s not in set(piv_sym)]
    new_of_old = np.empty(N, dtype=np.int64)
    for i, s in enumerate(info_sym + piv_sym):
        new_of_old[s] = i
    K = N - M
    # unpack reduced rows; pivot bit b is the XOR of the information bits on its row
    Wb = np.unpackbits(W.view(np.uint8), axis=1, bitorder="little")[:, :N * p]
    info_bits = np.concatenate([np.arange(s * p, (s + 1) * p) for s in info_sym])
    enc = np.zeros((M * p, K * p), dtype=np.uint8)
    for row, pb in enumerate(piv):
        sym, bit = divmod(pb, p)
        t = int(new_of_old[sym]) - K
        enc[t * p + bit] = Wb[row, info_bits]
    r2, c2, v2 = _sort_coo(np.asarray(rows), new_of_old[np.asarray(cols)], np.asarray(vals))
    return r2, c2, v2, K, enc


def regular_code(q: int, N: int, dv: int = 3, dc: int = 6, cfg: str = "code", poly: int | None = None,
                 encodable: bool = True, max_tries: int = 50) -> Code:
    """Random regular (dv, dc) LDPC code over GF(q) with N symbols.

    With `encodable` the columns are relabelled into systematic order
    (information symbols first) and a binary encoder is attached; codes
    whose H is rank deficient are redrawn from the next seed.
    """
    p = log2q(q)
    poly = FIELD_POLY[p] if poly is None else poly
    for t in range(max_tries):
        rng = rng_for(cfg, "H", t)
        M, rows, cols = regular_graph(N, dv, dc, rng)
        vals = rng.integers(1, q, size=rows.size)
        rows, cols, vals = _sort_coo(rows, cols, vals)
        if not encodable:
            return Code(q, M, N, rows, cols, vals, poly)
        s = systematic(q, M, N, rows, cols, vals, poly)
        if s is None:
            continue
        r2, c2, v2, K, enc = s
        return Code(q, M, N, r2, c2, v2, poly, K=K, enc=enc)
    raise RuntimeError("no full-rank code found")


def code_from_dense(H: np.ndarray, q: int, poly: int | None = None, encodable: bool = False) -> Code:
    p = log2q(q)
    poly = FIELD_POLY[p] if poly is None else poly
    H = np.asarray(H)
    rows, cols = np.nonzero(H)
    vals = H[rows, cols]
    rows, cols, vals = _sort_coo(rows, cols, vals)
    M, N = H.shape
    if encodable:
        s = systematic(q, M, N, rows, cols, vals, poly)
        if s is None:
            raise ValueError("H is rank deficient")
        r2, c2, v2, K, enc = s
        return Code(q, M, N, r2, c2, v2, poly, K=K, enc=enc)
    return Code(q, M, N, rows, cols, vals, poly)


def to_bits(x: np.ndarray, p: int) -> np.ndarray:
    """[..., n] symbols -> [..., n, p] bits, bit k = (a >> k) & 1."""
    x = np.asarray(x, dtype=np.int64)
    return ((x[..., None] >> np.arange(p)) & 1).astype(np.uint8)


def from_bits(b: np.ndarray) -> np.ndarray:
    p = b.shape[-1]
    return (b.astype(np.int64) << np.arange(p)).sum(-1)


def encode(code: Code, s: np.ndarray) -> np.ndarray:
    """Codewords x = [s; t] with H x = 0 for information words s of shape [F, K]."""
    if code.enc is None:
        raise ValueError("code has no encoder")
    s = np.atleast_2d(np.asarray(s, dtype=np.int64))
    F = s.shape[0]
    sb = to_bits(s, code.p).reshape(F, -1).astype(np.float32)
    tb = (sb @ code.enc.T.astype(np.float32)).astype(np.int64) & 1
    t = from_bits(tb.reshape(F, code.M, code.p))
    return np.concatenate([s, t], axis=1).astype(np.uint8)


def iid_source(rng: np.random.Generator, F: int, K: int, q: int) -> np.ndarray:
    return rng.integers(0, q, size=(F, K)).astype(np.int64)


def stationary(T: np.ndarray) -> np.ndarray:
    T = np.asarray(T, dtype=np.float64)
    T = T / T.sum(1, keepdims=True)
    w, v = np.linalg.eig(T.T)
    k = int(np.argmin(np.abs(w - 1)))
    pi = np.abs(np.real(v[:, k]))
    return pi / pi.sum()


def markov_source(u: np.ndarray, T: np.ndarray, start: np.ndarray | None = None) -> np.ndarray:
    """First-order chain with row-stochastic T[a, b] = Pr(next = b | current = a),
    driven by uniforms u of shape [F, K].  The first symbol is drawn from
    `start` (default: the stationary distribution)."""
    T = np.asarray(T, dtype=np.float64)
    T = T / T.sum(1, keepdims=True)
    q = T.shape[0]
    start = stationary(T) if start is None else np.asarray(start, dtype=np.float64)
    cdf = np.cumsum(T, axis=1)
    cdf[:, -1] = 1.0
    F, K = u.shape
    s = np.empty((F, K), dtype=np.int64)
    s[:, 0] = np.minimum(np.searchsorted(np.cumsum(start), u[:, 0], side="right"), q - 1)
    for i in range(1, K):
        s[:, i] = np.minimum((u[:, i:i + 1] >= cdf[s[:, i - 1]]).sum(1), q - 1)
    return s


def bit_chain_symbols(Tb: np.ndarray, p: int) -> np.ndarray:
    """The first-order chain over p-bit symbols induced by a two-state bit
    chain Tb run through bits 0..p-1 of every symbol in turn: Pr(next = b |
    current = a) = Tb[a_{p-1}, b_0] Tb[b_0, b_1] ... Tb[b_{p-2}, b_{p-1}]."""
    q = 1 << p
    T = np.ones((q, q))
    for a in range(q):
        for b in range(q):
            prev = (a >> (p - 1)) & 1
            for k in range(p):
                bit = (b >> k) & 1
                T[a, b] *= Tb[prev, bit]
                prev = bit
    return T


def self_transition_chain(q: int, stay: float) -> np.ndarray:
    """q-state chain that stays with probability `stay`, else moves uniformly."""
    T = np.full((q, q), (1.0 - stay) / (q - 1))
    np.fill_diagonal(T, stay)
    return T


# Markov matrices printed in the paper's footnote to Sec. 3.
MARKOV_2S = np.array([[0.89, 0.11], [0.11, 0.89]])
MARKOV_4S = np.array([[0.808022, 0.0883281, 0.0130689, 0.0905813],
                      [0.128676, 0.0514706, 0.0772059, 0.742647],
                      [0.755814, 0.108527, 0.0116279, 0.124031],
                      [0.866667, 0.0151111, 0.091556, 0.0266659]])


def bsc(rng, x: np.ndarray, p: int, f: float) -> np.ndarray:
    """Binary images of x with each bit flipped with probability f -> [F, N, p] float32 0/1."""
    b = to_bits(x, p)
    flip = rng.random(b.shape) < f
    return (b ^ flip).astype(np.float32)


def bec(rng, x: np.ndarray, p: int, eps: float) -> np.ndarray:
    """Bits erased with probability eps (marked 2.0)."""
    b = to_bits(x, p).astype(np.float32)
    b[rng.random(b.shape) < eps] = 2.0
    return b


def biawgn(rng, x: np.ndarray, p: int, sigma) -> np.ndarray:
    """BPSK (bit 0 -> +1, bit 1 -> -1) plus white Gaussian noise of std sigma
    (scalar or one value per frame)."""
    b = to_bits(x, p).astype(np.float32)
    sig = np.asarray(sigma, dtype=np.float64).reshape(-1, 1, 1) if np.ndim(sigma) else float(sigma)
    return (1.0 - 2.0 * b + sig * rng.standard_normal(b.shape)).astype(np.float32)


def ebn0_to_sigma(ebn0_db: float, rate: float = 0.5) -> float:
    """sigma of unit-energy BPSK at the given Eb/N0 and code rate."""
    return float(np.sqrt(1.0 / (2.0 * rate * 10.0 ** (ebn0_db / 10.0))))


# ---------------------------------------------------------------------------
# Named workloads: regular (3,6) rate-1/2 codes shaped like the paper's settings.
WORKLOADS = {
    "gf4_n96_bsc005": dict(q=4, N=96, source="iid", channel="bsc", params=[0.05], frames=1000, max_iter=100),
    "gf16_n1000_awgn": dict(q=16, N=1000, source="iid", channel="awgn", params=[1.0, 1.5, 2.0],
                            frames=4096, max_iter=200),
    "gf8_n2000_markov_bsc": dict(q=8, N=2000, source="markov", stay=0.8, channel="bsc", params=[0.08, 0.10],
                                 frames=2048, max_iter=200),
    "gf8_n2000_markov_bec": dict(q=8, N=2000, source="markov", stay=0.8, channel="bec", params=[0.40],
                                 frames=2048, max_iter=200),
}


@dataclass
class Batch:
    code: Code
    x: np.ndarray          # [F, N] transmitted codewords (uint8)
    obs: np.ndarray        # [F, N, p] float32 observations
    channel: str           # "bsc" | "bec" | "awgn"
    param: np.ndarray      # [F] channel parameter per frame (f, eps or sigma)
    T: np.ndarray | None   # Markov transition matrix or None
    K: int                 # number of source positions (0..K-1)
    max_iter: int


def make_batch(name: str, frames: int | None = None, first_frame: int = 0, N: int | None = None) -> Batch:
    """Frames first_frame .. first_frame+frames-1 of a named workload.  Frame f
    uses channel parameter params[f % len(params)]."""
    w = WORKLOADS[name]
    q = w["q"]
    N = w["N"] if N is None else N
    p = log2q(q)
    cfg = f"{name}/N{N}"
    code = regular_code(q, N, cfg=cfg)
    F = w["frames"] if frames is None else frames
    fidx = np.arange(first_frame, first_frame + F)
    params = np.asarray(w["params"], dtype=np.float64)[fidx % len(w["params"])]
    T = None
    src = np.empty((F, code.K), dtype=np.int64)
    if w["source"] == "markov":
        T = self_transition_chain(q, w["stay"])
    if T is not None:
        u = np.stack([rng_for(cfg, "src", int(f)).random(code.K) for f in fidx])
        src[:] = markov_source(u, T)
    else:
        for i, f in enumerate(fidx):
            src[i] = iid_source(rng_for(cfg, "src", int(f)), 1, code.K, q)[0]
    x = encode(code, src)
    obs = np.empty((F, N, p), dtype=np.float32)
    for i, f in enumerate(fidx):
        r = rng_for(cfg, "noise", int(f))
        if w["channel"] == "bsc":
            obs[i] = bsc(r, x[i:i + 1], p, params[i])[0]
        elif w["channel"] == "bec":
            obs[i] = bec(r, x[i:i + 1], p, params[i])[0]
        else:
            sig = ebn0_to_sigma(params[i])
            params[i] = sig
            obs[i] = biawgn(r, x[i:i + 1], p, sig)[0]
    return Batch(code, x, obs, w["channel"], params, T, code.K if T is not None else 0, w["max_iter"])


# ---------------------------------------------------------------------------
# The MN form of Sec. 2 (Eqs. 1-2): H = [A | B] with the source symbols s on
# the first K columns and B (the last M columns) invertible; the sender
# transmits t = B^-1 A s, the channel adds noise n (r = t + n on the bits),
# and the receiver decodes the unknowns w = [s; n] from the syndrome
# z = H [0; r] = B r, with the source columns never observed (punctured) and
# a block prior on them, the noise columns carrying the noise prior.
@dataclass
class MNBatch:
    code: Code
    s: np.ndarray          # [F, K] source words
    n: np.ndarray          # [F, M] noise symbols (r = t XOR n)
    obs: np.ndarray        # [F, N, p] decoder observations: 0 bits on the noise columns
    punct: np.ndarray      # [N] 1 on the source columns
    z: np.ndarray          # [F, M] syndromes B r
    f: float               # BSC flip rate of the noise bits
    T: np.ndarray          # Markov transition matrix of the source
    K: int
    max_iter: int


def mn_batch(q: int, M: int, frames: int, f: float, stay: float = 0.8, dv: int = 3, dc: int = 6,
             cfg: str = "mn", max_iter: int = 100) -> MNBatch:
    """Frames of the MN form over a systematic regular code (N = K + M, source
    first): a stationary Markov source (self-transition `stay`) and a BSC of
    flip rate f on the bits of t."""
    N = M * dc // (dc - dv) if dc != dv else 2 * M
    code = regular_code(q, N, dv=dv, dc=dc, cfg=cfg)
    K, p = code.K, code.p
    T = self_transition_chain(q, stay)
    u = np.stack([rng_for(cfg, "src", i).random(K) for i in range(frames)])
    s = markov_source(u, T)
    x = encode(code, s)
    t = x[:, K:].astype(np.int64)
    nb = np.stack([(rng_for(cfg, "noise", i).random((code.M, p)) < f) for i in range(frames)]).astype(np.int64)
    n = from_bits(nb)
    r = t ^ n
    w = np.concatenate([np.zeros((frames, K), np.int64), r], axis=1)
    z = code.syndrome(w)
    obs = np.zeros((frames, code.N, p), np.float32)   # the noise prior: bits observed as 0 through BSC(f)
    punct = np.zeros(code.N, np.uint8)
    punct[:K] = 1
    return MNBatch(code, s, n, obs, punct, z.astype(np.uint8), f, T, K, max_iter)
