"""Python access to the FP64 CPU oracle (oracle/gfbp_oracle.c).

TEST INFRASTRUCTURE: the slow, literal reference of the paper's decoder that
the CUDA library is checked against.  Only the tests, the smoke check and the
benchmark's CPU-baseline leg use it; the decoding library never imports it.

Arrays in, arrays out (numpy, float64 for probabilities).  Channel kinds:
"bsc" (param f), "bec" (param eps), "awgn" (param sigma), "loglik".
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gfbp_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None
_lock = threading.Lock()

KIND = {"bsc": 0, "bec": 1, "awgn": 2, "loglik": 3}


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/liboracle.so (gcc, OpenMP, no fast-math)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-shared", "-fPIC",
                               _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = C.CDLL(_LIB_PATH)
            P = C.c_void_p
            i, u, l, d = C.c_int, C.c_uint, C.c_long, C.c_double
            _lib.oracle_decode.argtypes = [i, u, i, i, l, P, P, P, i, i, P, P, P, P, i, i, i, i, i, P, i, P,
                                           P, P, P, P, P, P, P, i, i]
            _lib.oracle_step.argtypes = [i, u, i, i, l, P, P, P, i, i, P, P, P, P, i, i, i, P, i, P,
                                         P, P, P, P, P, P, i]
            _lib.oracle_gf_tables.argtypes = [i, u, P, P]
            _lib.oracle_check.argtypes = [i, u, i, P, i, P, P, i]
            _lib.oracle_channel.argtypes = [i, i, d, i, P, P, P]
            _lib.oracle_markov.argtypes = [i, P, i, P, P, i, P]
            for fn in ("oracle_decode", "oracle_step", "oracle_gf_tables", "oracle_check",
                       "oracle_channel", "oracle_markov"):
                getattr(_lib, fn).restype = C.c_int
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _c(a, dt):
    return None if a is None else np.ascontiguousarray(a, dtype=dt)


def _check(rc, what):
    if rc != 0:
        raise ValueError(f"{what} failed with status {rc}")


def gf_tables(q: int, poly: int = 0):
    mul = np.zeros((q, q), np.int32)
    inv = np.zeros(q, np.int32)
    _check(lib().oracle_gf_tables(q, poly, _p(mul), _p(inv)), "oracle_gf_tables")
    return mul, inv


def check(q: int, h, z: int, qin, use_wht: bool = False, poly: int = 0) -> np.ndarray:
    """Eq. 3 for every edge of one check: qin [d][q] -> r [d][q]."""
    h = _c(h, np.int32)
    qin = _c(qin, np.float64)
    r = np.zeros_like(qin)
    _check(lib().oracle_check(q, poly, int(h.size), _p(h), int(z), _p(qin), _p(r), int(use_wht)), "oracle_check")
    return r


def channel(q: int, kind: str, param: float, obs, punct=None) -> np.ndarray:
    obs = _c(obs, np.float32)
    p = q.bit_length() - 1
    n = obs.size // (q if kind == "loglik" else p)
    L = np.zeros((n, q), np.float64)
    _check(lib().oracle_channel(q, KIND[kind], float(param), n, _p(obs), _p(_c(punct, np.uint8)), _p(L)),
           "oracle_channel")
    return L


def markov(T, Q, form: int = 6):
    """Priors of K ordered source positions from their posteriors Q [K][q];
    returns (P [K][q], pi [q])."""
    T = _c(T, np.float64)
    Q = _c(Q, np.float64)
    K, q = Q.shape
    P = np.zeros_like(Q)
    pi = np.zeros(q, np.float64)
    _check(lib().oracle_markov(q, _p(T), K, _p(Q), _p(P), form, _p(pi)), "oracle_markov")
    return P, pi


def _code_arrays(code):
    rows = _c(code.rows, np.int32)
    cols = _c(code.cols, np.int32)
    vals = _c(code.vals, np.int32)
    return rows, cols, vals


def _params(param, F):
    a = np.asarray(param, dtype=np.float64)
    return np.ascontiguousarray(np.broadcast_to(a, (F,)) if a.ndim == 0 else a.reshape(F))


def decode(code, obs, kind: str, param, schedule: str = "pus", max_iter: int = 100, T=None, K: int = 0,
           src_pos=None, punct=None, syn=None, use_wht: bool | None = None, early_stop: bool = True,
           trace: bool = False, post: bool = False, threads: int = 0, gauss_seidel: bool = False,
           round32: int = 0):
    """Decode F frames.  obs: [F][N][p] (or [F][N][q] for loglik).  With a
    Markov source (T), gauss_seidel re-estimates each block prior as the SUS
    sweep reaches its symbol instead of after every iteration.  round32 is a
    conditioning probe, not the decoder: with round32 != 0 every message is
    stored rounded to the nearest float, as a decoder keeping FP32 messages
    does, and with round32 = k >= 2 the channel likelihoods are also moved by
    one float ulp in a pattern seeded by k."""
    obs = _c(obs, np.float32)
    F = obs.shape[0]
    q, M, N = code.q, code.M, code.N
    rows, cols, vals = _code_arrays(code)
    if use_wht is None:
        use_wht = q >= 64
    xhat = np.zeros((F, N), np.uint8)
    iters = np.zeros(F, np.int32)
    conv = np.zeros(F, np.uint8)
    zs = np.zeros(F, np.int64)
    Q = np.zeros((F, N, q), np.float64) if post else None
    tx = np.zeros((F, max_iter, N), np.uint8) if trace else None
    tg = np.zeros((F, max_iter, N), np.float32) if trace else None
    markov_on = T is not None
    Tc = _c(T, np.float64) if markov_on else None
    sp = _c(src_pos, np.int32) if src_pos is not None else None
    rc = lib().oracle_decode(q, int(getattr(code, "poly", 0) or 0), M, N, rows.size, _p(rows), _p(cols), _p(vals),
                             F, KIND[kind], _p(_params(param, F)), _p(obs), _p(_c(punct, np.uint8)),
                             _p(_c(syn, np.uint8)), 1 if schedule == "sus" else 0, int(use_wht), int(early_stop),
                             int(max_iter), (2 if gauss_seidel else 1) if markov_on else 0, _p(Tc), int(K if markov_on else 0), _p(sp),
                             _p(xhat), _p(iters), _p(conv), _p(Q), _p(tx), _p(tg), _p(zs), int(threads),
                             int(round32))
    _check(rc, "oracle_decode")
    out = dict(xhat=xhat, iters=iters, conv=conv, zero_sums=zs)
    if post:
        out["post"] = Q
    if trace:
        out["trace_x"] = tx
        out["trace_gap"] = tg
    return out


def step(code, obs, kind: str, param, msg, schedule: str = "pus", T=None, K: int = 0, src_pos=None,
         prior=None, punct=None, syn=None, use_wht: bool | None = None, threads: int = 0):
    """One iteration from the q-message state msg [F][E][q] (edges in (row, col)
    order).  Returns dict(msg, post, xhat, sat, prior_out)."""
    obs = _c(obs, np.float32)
    F = obs.shape[0]
    q, M, N = code.q, code.M, code.N
    rows, cols, vals = _code_arrays(code)
    if use_wht is None:
        use_wht = q >= 64
    msg = np.array(msg, dtype=np.float64, order="C", copy=True)
    post = np.zeros((F, N, q), np.float64)
    xhat = np.zeros((F, N), np.uint8)
    sat = np.zeros(F, np.uint8)
    markov_on = T is not None
    prior = _c(prior, np.float64) if markov_on else None
    prior_out = np.zeros((F, K, q), np.float64) if markov_on else None
    sp = _c(src_pos, np.int32) if src_pos is not None else None
    rc = lib().oracle_step(q, int(getattr(code, "poly", 0) or 0), M, N, rows.size, _p(rows), _p(cols), _p(vals),
                           F, KIND[kind], _p(_params(param, F)), _p(obs), _p(_c(punct, np.uint8)),
                           _p(_c(syn, np.uint8)), 1 if schedule == "sus" else 0, int(use_wht), int(markov_on),
                           _p(_c(T, np.float64) if markov_on else None), int(K if markov_on else 0), _p(sp),
                           _p(msg), _p(prior), _p(prior_out), _p(post), _p(xhat), _p(sat), int(threads))
    _check(rc, "oracle_step")
    return dict(msg=msg, post=post, xhat=xhat, sat=sat, prior_out=prior_out)


def initial_messages(code, obs, kind: str, param, T=None, K: int = 0, src_pos=None, punct=None) -> np.ndarray:
    """q_ij <- p_j on every edge (Sec. 2 initialisation), [F][E][q]; with a
    Markov source, p_j includes the stationary prior of source positions."""
    obs = np.asarray(obs, np.float32)
    F = obs.shape[0]
    q, N = code.q, code.N
    out = np.zeros((F, code.E, q), np.float64)
    pi = None
    if T is not None:
        _, pi = markov(T, np.full((1, q), 1.0 / q))
        pos = np.arange(K) if src_pos is None else np.asarray(src_pos)
    for f in range(F):
        prm = float(np.broadcast_to(np.asarray(param, np.float64), (F,))[f]) if np.ndim(param) == 0 else float(np.asarray(param)[f])
        L = channel(q, kind, prm, obs[f], punct)
        if pi is not None:
            L[pos] *= pi[None, :]
            L /= L.sum(1, keepdims=True)
        out[f] = L[np.asarray(code.cols)]
    return out
