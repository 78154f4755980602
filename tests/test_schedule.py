"""The SUS level schedule that gfbp_code_create builds (host logic, read back
through gfbp_level_schedule with no GPU), checked against its definition:
level(j) = 1 + the highest level of the earlier columns sharing a check with
j (0 if none), so that the columns of one level share no check; pieces of
whole columns of one level with at most 128 (column, slot) pairs; inside a
piece the pairs at an inner position of their check first, then those at
position 0, then the rest, each with its row in the piece's column order."""
import os
import shutil

import numpy as np
import pytest


@pytest.fixture(scope="module")
def G():
    from paper_cs_0605069_gb300 import build, gfbp
    if not os.path.exists(gfbp.LIB_PATH):
        if not (shutil.which("nvcc") or os.path.exists("/usr/local/cuda/bin/nvcc")):
            pytest.skip("libgfbp.so not built and nvcc unavailable")
        build.build()
    gfbp.lib()
    return gfbp


def _adjacency(code):
    cols_of = [[] for _ in range(code.M)]
    rows_of = [[] for _ in range(code.N)]
    for r, c in zip(np.asarray(code.rows), np.asarray(code.cols)):
        cols_of[int(r)].append(int(c))
        rows_of[int(c)].append(int(r))
    return [sorted(x) for x in cols_of], [sorted(x) for x in rows_of]


def _check(code, s):
    cols_of, rows_of = _adjacency(code)
    level = s["level"]
    # the definition, column by column in order
    for j in range(code.N):
        earlier = {c for r in rows_of[j] for c in cols_of[r] if c < j}
        want = 1 + max(level[c] for c in earlier) if earlier else 0
        assert level[j] == want, j
    assert s["n_levels"] == int(level.max()) + 1
    # one level's columns share no check
    for r in range(code.M):
        lv = [level[c] for c in cols_of[r]]
        assert len(set(lv)) == len(lv), r
    # pieces: whole columns of one level, <= 128 pairs, levels in order, and
    # every (column, slot) pair exactly once (a column without checks: slot 0)
    pp = s["piece_ptr"]
    assert pp[0] == 0 and pp[-1] == len(s["pair_col"]) and np.all(np.diff(pp) > 0)
    seen = set()
    last = (-1, -1)   # (level, column) of the previous piece's last column
    for p in range(len(pp) - 1):
        a, b = pp[p], pp[p + 1]
        assert b - a <= 128
        cols = s["pair_col"][a:b]
        slots = s["pair_slot"][a:b]
        rowsi = s["pair_row"][a:b]
        lv = {int(level[c]) for c in cols}
        assert len(lv) == 1, p
        ucols = sorted(set(int(c) for c in cols))
        assert (lv.pop(), ucols[0]) > last
        last = (int(level[ucols[-1]]), ucols[-1])
        # whole columns, with rows in the piece's column order
        base = 0
        expect_row = {}
        for c in ucols:
            n = max(len(rows_of[c]), 1)
            for k in range(n):
                expect_row[(c, k)] = base + k
            base += n
        got = {(int(c), int(k)): int(r) for c, k, r in zip(cols, slots, rowsi)}
        assert got == expect_row, p
        for key in got:
            assert key not in seen
            seen.add(key)
        # work classes in order: inner positions, position 0, the rest
        cls = []
        for c, k in zip(cols, slots):
            c, k = int(c), int(k)
            if not rows_of[c]:
                cls.append(2)
                continue
            r = rows_of[c][k]
            t, dc = cols_of[r].index(c), len(cols_of[r])
            cls.append(0 if 1 <= t <= dc - 2 else (1 if t == 0 and dc >= 2 else 2))
        assert cls == sorted(cls), p
    assert len(seen) == sum(max(len(x), 1) for x in rows_of)


def test_schedule_of_the_benchmark_code(G):
    from paper_cs_0605069_gb300 import workload as W
    b = W.make_batch("gf16_n1000_awgn", frames=1)
    s = G.level_schedule(b.code)
    _check(b.code, s)
    assert 20 <= s["n_levels"] <= 40   # a random (3,6) code with N = 1000


@pytest.mark.parametrize("q,N,dv,dc", [(8, 120, 6, 12), (4, 256, 3, 16), (2, 240, 3, 6), (16, 64, 4, 8)])
def test_schedule_of_regular_codes(G, q, N, dv, dc):
    from paper_cs_0605069_gb300 import workload as W
    code = W.regular_code(q, N, dv=dv, dc=dc, cfg=f"sched_{q}_{dv}_{dc}", encodable=False)
    _check(code, G.level_schedule(code))


def test_schedule_of_irregular_code_with_free_columns_and_degree_one_checks(G):
    from paper_cs_0605069_gb300 import workload as W
    rng = np.random.default_rng(5)
    M, N, q = 40, 90, 4
    H = np.zeros((M, N), np.int64)
    for j in range(N):
        if j % 11 == 5:
            continue   # a column without checks
        d = 1 + int(rng.integers(0, 4))
        H[rng.choice(M, size=d, replace=False), j] = rng.integers(1, q, size=d)
    for i in range(M):
        while np.count_nonzero(H[i]) > 12:
            H[i, rng.choice(np.nonzero(H[i])[0])] = 0
    H[0, :] = 0
    H[0, 7] = 3   # a check of degree 1
    code = W.code_from_dense(H, q)
    s = G.level_schedule(code)
    _check(code, s)
    assert s["level"][5] == 0


def test_schedule_validates_like_code_create(G):
    from types import SimpleNamespace
    bad = SimpleNamespace(q=4, M=1, N=2, rows=[0], cols=[0], vals=[4])
    with pytest.raises(G.GfbpError) as e:
        G.level_schedule(bad)
    assert e.value.status == G.GFBP_EINVAL and "out of range" in str(e.value)
    dup = SimpleNamespace(q=4, M=1, N=2, rows=[0, 0], cols=[1, 1], vals=[1, 2])
    with pytest.raises(G.GfbpError):
        G.level_schedule(dup)


def test_schedule_edge_cases(G):
    from types import SimpleNamespace
    # no checks at all: every column is free, level 0, one pseudo-pair each
    free = SimpleNamespace(q=4, M=0, N=5, rows=[], cols=[], vals=[])
    s = G.level_schedule(free)
    assert list(s["level"]) == [0] * 5 and s["n_levels"] == 1
    assert sorted(zip(s["pair_col"], s["pair_slot"])) == [(j, 0) for j in range(5)]
    _check(free, s)
    # a single column with one check of degree 1
    one = SimpleNamespace(q=2, M=1, N=1, rows=[0], cols=[0], vals=[1])
    s = G.level_schedule(one)
    assert list(s["level"]) == [0] and list(s["piece_ptr"]) == [0, 1]
    _check(one, s)
    # one check over 16 columns: a chain of 16 levels of one column each
    chain = SimpleNamespace(q=4, M=1, N=16, rows=[0] * 16, cols=list(range(16)), vals=[1, 2, 3, 1] * 4)
    s = G.level_schedule(chain)
    assert list(s["level"]) == list(range(16)) and len(s["piece_ptr"]) == 17
    _check(chain, s)
