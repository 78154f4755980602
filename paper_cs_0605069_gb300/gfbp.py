"""Python binding of the gfbp C ABI (include/gfbp.h).

Argument marshalling only: every step of decoding runs in the CUDA library
libgfbp.so.  PyTorch supplies device memory (CUDA tensors, whose raw
pointers are passed) and the current stream.  If the library is missing the
import of this module's functions fails loudly; there is no CPU path.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgfbp.so")
_lib = None
_lock = threading.Lock()

GFBP_OK, GFBP_EINVAL, GFBP_ENOMEM, GFBP_ECUDA, GFBP_ETIMEOUT, GFBP_EBUSY, GFBP_EUNSUPPORTED = range(7)
CHANNEL = {"bsc": 0, "bec": 1, "awgn": 2, "biawgn": 2, "loglik": 3}
SCHEDULE = {"pus": 0, "sus": 1}
CHECK_METHOD = {"auto": 0, "transform": 1, "direct": 2, "tensor": 3}
LAYOUT = {"auto": 0, "lanes": 1, "thread": 2, "resident": 3, "l2resident": 4}
PARTIALS = {"auto": 0, "fold": 1, "running": 2, "running_global": 3}

# Functions declared in include/gfbp.h (the CPU test checks that every one is exported).
EXPORTS = ("gfbp_last_error", "gfbp_code_create", "gfbp_code_destroy", "gfbp_code_info", "gfbp_level_schedule",
           "gfbp_workspace_size", "gfbp_decode", "gfbp_step", "gfbp_decode_noalloc",
           "gfbp_batch_create", "gfbp_batch_run", "gfbp_batch_variants", "gfbp_batch_set_variants",
           "gfbp_batch_destroy", "gfbp_autotune", "gfbp_wht", "gfbp_wait_selftest",
           "gfbp_server_create", "gfbp_server_submit", "gfbp_server_wait", "gfbp_server_stats",
           "gfbp_server_drain", "gfbp_server_destroy")


class GfbpError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: status {status}: {last_error()}")


class gfbp_channel(C.Structure):
    _fields_ = [("kind", C.c_int32), ("param", C.c_float), ("frame_param", C.c_void_p)]


class gfbp_prior(C.Structure):
    _fields_ = [("kind", C.c_int32), ("T", C.c_void_p), ("K", C.c_int32), ("src_pos", C.c_void_p)]


class gfbp_options(C.Structure):
    _fields_ = [("punct", C.c_void_p), ("syndrome", C.c_void_p), ("post", C.c_void_p),
                ("xhat_trace", C.c_void_p), ("no_early_stop", C.c_int32), ("workspace", C.c_void_p),
                ("workspace_bytes", C.c_size_t), ("kernel_events", C.c_void_p * 2), ("check_method", C.c_int32),
                ("sus_width", C.c_int32), ("layout", C.c_int32), ("sus_partials", C.c_int32),
                ("zero_sums", C.c_void_p)]


def lib() -> C.CDLL:
    """The loaded CUDA library; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: run paper_cs_0605069_gb300/build.py (no CPU fallback)")
            L = C.CDLL(LIB_PATH)
            P, i32, i64, u32 = C.c_void_p, C.c_int32, C.c_int64, C.c_uint32
            L.gfbp_last_error.restype = C.c_char_p
            L.gfbp_last_error.argtypes = []
            L.gfbp_code_create.argtypes = [i32, i32, i32, i64, P, P, P, u32, C.POINTER(C.c_void_p)]
            L.gfbp_level_schedule.argtypes = [i32, i32, i32, i64, P, P, P, P, C.POINTER(i32), P, C.POINTER(i32), P,
                                              P, P, C.POINTER(i32)]
            L.gfbp_code_destroy.argtypes = [P]
            L.gfbp_code_destroy.restype = None
            L.gfbp_code_info.argtypes = [P] + [C.POINTER(i32)] * 3 + [C.POINTER(i64)] + [C.POINTER(i32)] * 2
            L.gfbp_workspace_size.argtypes = [P, i32, i32, C.POINTER(gfbp_prior), i32, C.POINTER(C.c_size_t)]
            L.gfbp_decode.argtypes = [P, i32, P, gfbp_channel, i32, C.POINTER(gfbp_prior), i32, P, P, P,
                                      C.POINTER(gfbp_options), P]
            L.gfbp_step.argtypes = [P, i32, P, gfbp_channel, i32, C.POINTER(gfbp_prior), P, P, P, P, P, P,
                                    C.POINTER(gfbp_options), P]
            L.gfbp_decode_noalloc.argtypes = L.gfbp_decode.argtypes
            L.gfbp_wht.argtypes = [P, P, i64, i32, i32, P]
            L.gfbp_wait_selftest.argtypes = [i32, C.POINTER(i32), P]
            for fn in ("gfbp_code_create", "gfbp_code_info", "gfbp_workspace_size", "gfbp_decode", "gfbp_step",
                       "gfbp_decode_noalloc", "gfbp_wht", "gfbp_wait_selftest"):
                getattr(L, fn).restype = C.c_int
            _lib = L
    return _lib


def last_error() -> str:
    return (lib().gfbp_last_error() or b"").decode()


def _ok(rc: int, where: str):
    if rc != GFBP_OK:
        raise GfbpError(rc, where)


class Code:
    """A parity-check matrix H over GF(q) on the current CUDA device (gfbp_code_create)."""

    def __init__(self, q: int, M: int, N: int, rows, cols, vals, poly: int = 0):
        r = np.ascontiguousarray(rows, dtype=np.int32)
        c = np.ascontiguousarray(cols, dtype=np.int32)
        v = np.ascontiguousarray(vals, dtype=np.int32)
        h = C.c_void_p()
        _ok(lib().gfbp_code_create(int(q), int(M), int(N), int(r.size), r.ctypes.data, c.ctypes.data,
                                   v.ctypes.data, int(poly), C.byref(h)), "gfbp_code_create")
        self.handle = h
        vals_ = [C.c_int32() for _ in range(3)]
        E = C.c_int64()
        dc, dv = C.c_int32(), C.c_int32()
        _ok(lib().gfbp_code_info(h, C.byref(vals_[0]), C.byref(vals_[1]), C.byref(vals_[2]), C.byref(E),
                                 C.byref(dc), C.byref(dv)), "gfbp_code_info")
        self.q, self.M, self.N = (x.value for x in vals_)
        self.E, self.max_row_degree, self.max_col_degree = E.value, dc.value, dv.value

    @classmethod
    def from_coo(cls, code) -> "Code":
        """From any object with q, M, N, rows, cols, vals (and optionally poly)."""
        return cls(code.q, code.M, code.N, code.rows, code.cols, code.vals, getattr(code, "poly", 0) or 0)

    def close(self):
        if getattr(self, "handle", None):
            lib().gfbp_code_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def level_schedule(code) -> dict:
    """gfbp_level_schedule (host only) for an object with q, M, N, rows, cols,
    vals: the SUS level of every column, the pieces (pair offsets) and the
    pairs (column, slot, row index in the piece's column order) in the order
    the level kernel takes them."""
    r = np.ascontiguousarray(code.rows, dtype=np.int32)
    c = np.ascontiguousarray(code.cols, dtype=np.int32)
    v = np.ascontiguousarray(code.vals, dtype=np.int32)
    cap = int(r.size) + int(code.N)
    level = np.empty(int(code.N), np.int32)
    piece_ptr = np.empty(cap + 1, np.int32)
    pair_col, pair_slot, pair_row = (np.empty(cap, np.int32) for _ in range(3))
    nl, npc, npr = C.c_int32(), C.c_int32(), C.c_int32()
    _ok(lib().gfbp_level_schedule(int(code.q), int(code.M), int(code.N), int(r.size), r.ctypes.data, c.ctypes.data,
                                  v.ctypes.data, level.ctypes.data, C.byref(nl), piece_ptr.ctypes.data, C.byref(npc),
                                  pair_col.ctypes.data, pair_slot.ctypes.data, pair_row.ctypes.data, C.byref(npr)),
        "gfbp_level_schedule")
    n = npr.value
    return dict(level=level, n_levels=nl.value, piece_ptr=piece_ptr[:npc.value + 1].copy(),
                pair_col=pair_col[:n].copy(), pair_slot=pair_slot[:n].copy(), pair_row=pair_row[:n].copy())


def _ptr(t) -> int | None:
    return None if t is None else int(t.data_ptr())


def _stream(stream):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


def _prior(T, K, src_pos, gauss_seidel=False):
    if T is None:
        return gfbp_prior(0, None, 0, None), None
    T = np.ascontiguousarray(T, dtype=np.float64)
    sp = None if src_pos is None else np.ascontiguousarray(src_pos, dtype=np.int32)
    pr = gfbp_prior(2 if gauss_seidel else 1, T.ctypes.data, int(K), None if sp is None else sp.ctypes.data)
    return pr, (T, sp)


def workspace_size(code: Code, n_frames: int, schedule: str = "pus", T=None, K: int = 0, src_pos=None,
                   step: bool = False) -> int:
    pr, _keep = _prior(T, K, src_pos)
    n = C.c_size_t()
    _ok(lib().gfbp_workspace_size(code.handle, int(n_frames), SCHEDULE[schedule], C.byref(pr), int(step),
                                  C.byref(n)), "gfbp_workspace_size")
    return n.value


def decode(code: Code, obs, channel: str = "bsc", param: float = 0.0, schedule: str = "pus", max_iter: int = 100,
           T=None, K: int = 0, src_pos=None, frame_param=None, punct=None, syndrome=None, post: bool = False,
           trace: bool = False, no_early_stop: bool = False, workspace=None, out=None, stream=None,
           kernel_events=None, check_method: str = "auto", sus_width: int = 0,
           layout: str = "auto", partials: str = "auto", gauss_seidel: bool = False, zero_sums: bool = False):
    """gfbp_decode on CUDA tensors.  obs: float32 [F][N][p] (or [F][N][q] for
    loglik).  Returns dict of device tensors x_hat [F][N] uint8, iters [F]
    int32, converged [F] uint8 (+ post [F][N][q], trace [F][max_iter][N],
    zero_sums [F] int32: the normalisations that fell back to uniform).
    layout: "auto", "lanes" or "thread" (kernels for q = 4, 8, 16 with the
    direct check node, same results); sus_width: SUS lane teams per frame of
    the "lanes" layout (0 = automatic); partials: "auto", "fold", "running" or
    "running_global" (how the SUS level kernel gathers a check's other
    messages); gauss_seidel: with a Markov source (T), re-estimate each block
    prior as the SUS sweep reaches it (prior kind MARKOV_GS)."""
    import torch
    F = int(obs.shape[0])
    dev = obs.device
    if out is None:
        out = dict(x_hat=torch.empty((F, code.N), dtype=torch.uint8, device=dev),
                   iters=torch.empty(F, dtype=torch.int32, device=dev),
                   converged=torch.empty(F, dtype=torch.uint8, device=dev))
        if post:
            out["post"] = torch.empty((F, code.N, code.q), dtype=torch.float32, device=dev)
        if trace:
            out["trace"] = torch.empty((F, max_iter, code.N), dtype=torch.uint8, device=dev)
        if zero_sums:
            out["zero_sums"] = torch.empty(F, dtype=torch.int32, device=dev)
    pr, _keep = _prior(T, K, src_pos, gauss_seidel)
    if workspace is None:
        nbytes = workspace_size(code, F, schedule, T, K, src_pos)
        workspace = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    opt = gfbp_options(_ptr(punct), _ptr(syndrome), _ptr(out.get("post")), _ptr(out.get("trace")),
                       int(no_early_stop), _ptr(workspace), int(workspace.numel()))
    opt.check_method = CHECK_METHOD[check_method]
    opt.sus_width = int(sus_width)
    opt.layout = LAYOUT[layout]
    opt.sus_partials = PARTIALS[partials]
    opt.zero_sums = _ptr(out.get("zero_sums"))
    if kernel_events is not None:   # (torch.cuda.Event, torch.cuda.Event) timing the schedule kernel alone
        for ev in kernel_events:    # torch creates the CUDA event on its first record
            if not ev.cuda_event:
                ev.record(stream if stream is not None else torch.cuda.current_stream())
        opt.kernel_events[0] = kernel_events[0].cuda_event
        opt.kernel_events[1] = kernel_events[1].cuda_event
    ch = gfbp_channel(CHANNEL[channel], float(param), _ptr(frame_param))
    _ok(lib().gfbp_decode(code.handle, F, _ptr(obs), ch, SCHEDULE[schedule], C.byref(pr), int(max_iter),
                          _ptr(out["x_hat"]), _ptr(out["iters"]), _ptr(out["converged"]), C.byref(opt),
                          _stream(stream)), "gfbp_decode")
    return out


def step(code: Code, obs, msg, channel: str = "bsc", param: float = 0.0, schedule: str = "pus", T=None, K: int = 0,
         src_pos=None, prior_in=None, frame_param=None, punct=None, syndrome=None, stream=None,
         check_method: str = "auto", sus_width: int = 0, layout: str = "auto", partials: str = "auto"):
    """gfbp_step: one iteration from msg (float32 [F][E][q], updated in place).
    Returns dict(msg, post, x_hat, sat, prior_out)."""
    import torch
    F = int(obs.shape[0])
    dev = obs.device
    post = torch.empty((F, code.N, code.q), dtype=torch.float32, device=dev)
    x_hat = torch.empty((F, code.N), dtype=torch.uint8, device=dev)
    sat = torch.empty(F, dtype=torch.uint8, device=dev)
    prior_out = torch.empty((F, K, code.q), dtype=torch.float32, device=dev) if T is not None else None
    pr, _keep = _prior(T, K, src_pos)
    ws = torch.empty(workspace_size(code, F, schedule, T, K, src_pos, step=True), dtype=torch.uint8, device=dev)
    opt = gfbp_options(_ptr(punct), _ptr(syndrome), None, None, 0, _ptr(ws), int(ws.numel()))
    opt.check_method = CHECK_METHOD[check_method]
    opt.sus_width = int(sus_width)
    opt.layout = LAYOUT[layout]
    opt.sus_partials = PARTIALS[partials]
    ch = gfbp_channel(CHANNEL[channel], float(param), _ptr(frame_param))
    _ok(lib().gfbp_step(code.handle, F, _ptr(obs), ch, SCHEDULE[schedule], C.byref(pr), _ptr(msg), _ptr(prior_in),
                        _ptr(prior_out), _ptr(post), _ptr(x_hat), _ptr(sat), C.byref(opt), _stream(stream)),
        "gfbp_step")
    return dict(msg=msg, post=post, x_hat=x_hat, sat=sat, prior_out=prior_out)


WHT_METHOD = {"simt": 0, "tensor": 1}


def wht(x, method: str = "simt", out=None, stream=None):
    """gfbp_wht on a CUDA float32 tensor [n, q] (unnormalised Walsh-Hadamard
    transform of every row); method "simt" (FP32 butterflies) or "tensor"
    (FP16 hi/lo split on the tensor cores, FP32 accumulation)."""
    import torch
    x = x.contiguous()
    n, q = int(x.shape[0]), int(x.shape[1])
    y = torch.empty_like(x) if out is None else out
    _ok(lib().gfbp_wht(_ptr(x), _ptr(y), n, q, WHT_METHOD[method], _stream(stream)), "gfbp_wht")
    return y


WAIT = {"mbarrier": 0, "watermark": 1}


def wait_selftest(which: str, stream=None):
    """gfbp_wait_selftest: run one of the kernels' bounded waits on a
    condition that never comes true.  Returns (status, completed): the
    expected outcome is (GFBP_ETIMEOUT, 0)."""
    done = C.c_int32(-1)
    rc = lib().gfbp_wait_selftest(WAIT[which], C.byref(done), _stream(stream))
    return int(rc), int(done.value)


def decode_noalloc(code: Code, obs, channel: str = "bsc", param: float = 0.0, schedule: str = "pus",
                   max_iter: int = 100, T=None, K: int = 0, src_pos=None, frame_param=None, post: bool = False,
                   check_method: str = "auto", out=None, stream=None, sus_width: int = 0,
                   layout: str = "auto", partials: str = "auto"):
    """gfbp_decode_noalloc on CUDA tensors: like decode(), with the library's
    static device scratch instead of a workspace (no device allocation inside
    the library; the outputs here are caller tensors)."""
    import torch
    F = int(obs.shape[0])
    dev = obs.device
    if out is None:
        out = dict(x_hat=torch.empty((F, code.N), dtype=torch.uint8, device=dev),
                   iters=torch.empty(F, dtype=torch.int32, device=dev),
                   converged=torch.empty(F, dtype=torch.uint8, device=dev))
        if post:
            out["post"] = torch.empty((F, code.N, code.q), dtype=torch.float32, device=dev)
    pr, _keep = _prior(T, K, src_pos)
    opt = gfbp_options(None, None, _ptr(out.get("post")), None, 0, None, 0)
    opt.check_method = CHECK_METHOD[check_method]
    opt.sus_width = int(sus_width)
    opt.layout = LAYOUT[layout]
    opt.sus_partials = PARTIALS[partials]
    ch = gfbp_channel(CHANNEL[channel], float(param), _ptr(frame_param))
    _ok(lib().gfbp_decode_noalloc(code.handle, F, _ptr(obs), ch, SCHEDULE[schedule], C.byref(pr), int(max_iter),
                                  _ptr(out["x_hat"]), _ptr(out["iters"]), _ptr(out["converged"]), C.byref(opt),
                                  _stream(stream)), "gfbp_decode_noalloc")
    return out


class gfbp_batch_item(C.Structure):
    _fields_ = [("code", C.c_void_p), ("n_frames", C.c_int32), ("obs", C.c_void_p), ("channel", gfbp_channel),
                ("prior", C.c_void_p), ("x_hat", C.c_void_p), ("iters", C.c_void_p), ("converged", C.c_void_p)]


def _batch_lib():
    L = lib()
    if not getattr(L, "_batch_typed", False):
        P, i32 = C.c_void_p, C.c_int32
        L.gfbp_batch_create.argtypes = [C.POINTER(gfbp_batch_item), i32, i32, i32, C.POINTER(gfbp_options),
                                        C.POINTER(C.c_void_p)]
        L.gfbp_batch_run.argtypes = [P, P]
        L.gfbp_batch_variants.argtypes = [P, C.POINTER(i32)]
        L.gfbp_batch_set_variants.argtypes = [P, C.POINTER(i32)]
        L.gfbp_batch_destroy.argtypes = [P]
        L.gfbp_batch_destroy.restype = None
        L.gfbp_autotune.argtypes = [P, i32, P, gfbp_channel, i32, C.POINTER(gfbp_prior), i32, P, C.POINTER(i32)]
        for fn in ("gfbp_batch_create", "gfbp_batch_run", "gfbp_batch_variants", "gfbp_batch_set_variants",
                   "gfbp_autotune"):
            getattr(L, fn).restype = C.c_int
        L._batch_typed = True
    return L


class Batch:
    """gfbp_batch: frames of several codes decoded by one persistent launch.
    items: list of dict(code=Code, obs=tensor, channel=str, param=float,
    frame_param=tensor|None, T=None, K=0).  Outputs are allocated here
    (self.outputs[i] = dict(x_hat, iters, converged))."""

    def __init__(self, items, schedule: str = "sus", max_iter: int = 100):
        import torch
        L = _batch_lib()
        self._keep = []
        arr = (gfbp_batch_item * len(items))()
        self.outputs = []
        for i, it in enumerate(items):
            code, obs = it["code"], it["obs"]
            F = int(obs.shape[0])
            o = dict(x_hat=torch.empty((F, code.N), dtype=torch.uint8, device=obs.device),
                     iters=torch.empty(F, dtype=torch.int32, device=obs.device),
                     converged=torch.empty(F, dtype=torch.uint8, device=obs.device))
            self.outputs.append(o)
            pr, keep = _prior(it.get("T"), it.get("K", 0), it.get("src_pos"))
            self._keep += [pr, keep, obs, it.get("frame_param")]
            arr[i] = gfbp_batch_item(code.handle, F, _ptr(obs),
                                     gfbp_channel(CHANNEL[it["channel"]], float(it.get("param", 0.0)),
                                                  _ptr(it.get("frame_param"))),
                                     C.cast(C.pointer(pr), C.c_void_p) if it.get("T") is not None else None,
                                     _ptr(o["x_hat"]), _ptr(o["iters"]), _ptr(o["converged"]))
        h = C.c_void_p()
        _ok(L.gfbp_batch_create(arr, len(items), SCHEDULE[schedule], int(max_iter), None, C.byref(h)),
            "gfbp_batch_create")
        self.handle = h
        self.n = len(items)

    def run(self, stream=None):
        _ok(_batch_lib().gfbp_batch_run(self.handle, _stream(stream)), "gfbp_batch_run")
        return self.outputs

    def variants(self):
        v = (C.c_int32 * self.n)()
        _ok(_batch_lib().gfbp_batch_variants(self.handle, v), "gfbp_batch_variants")
        return list(v)

    def set_variants(self, variants):
        """Pin every item's kernel variant (numbering of gfbp_autotune)."""
        v = (C.c_int32 * self.n)(*[int(x) for x in variants])
        _ok(_batch_lib().gfbp_batch_set_variants(self.handle, v), "gfbp_batch_set_variants")

    def close(self):
        if getattr(self, "handle", None):
            _batch_lib().gfbp_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def autotune(code: Code, obs, channel: str, param: float = 0.0, schedule: str = "sus", max_iter: int = 20,
             frame_param=None, T=None, K: int = 0, stream=None) -> int:
    """gfbp_autotune on a sample batch; returns the chosen kernel variant."""
    pr, _keep = _prior(T, K, None)
    v = C.c_int32()
    _ok(_batch_lib().gfbp_autotune(code.handle, int(obs.shape[0]), _ptr(obs),
                                   gfbp_channel(CHANNEL[channel], float(param), _ptr(frame_param)),
                                   SCHEDULE[schedule], C.byref(pr), int(max_iter), _stream(stream), C.byref(v)),
        "gfbp_autotune")
    return v.value


class gfbp_request(C.Structure):
    _fields_ = [("code", C.c_void_p), ("n_frames", C.c_int32), ("obs", C.c_void_p), ("channel", gfbp_channel),
                ("prior", C.c_void_p), ("schedule", C.c_int32), ("max_iter", C.c_int32), ("x_hat", C.c_void_p),
                ("iters", C.c_void_p), ("converged", C.c_void_p)]


class gfbp_result(C.Structure):
    _fields_ = [("latency_us", C.c_double), ("queue_us", C.c_double), ("rounds", C.c_int32)]


class gfbp_server_stats_t(C.Structure):
    _fields_ = [("queued", C.c_int32), ("resident", C.c_int32), ("peak_resident", C.c_int32),
                ("rounds", C.c_int64), ("completed", C.c_int64), ("bytes_in_use", C.c_size_t),
                ("peak_bytes", C.c_size_t)]


def _server_lib():
    L = lib()
    if not getattr(L, "_server_typed", False):
        P = C.c_void_p
        L.gfbp_server_create.argtypes = [C.c_size_t, C.c_int32, C.POINTER(C.c_void_p)]
        L.gfbp_server_submit.argtypes = [P, C.POINTER(gfbp_request), C.POINTER(C.c_uint64)]
        L.gfbp_server_wait.argtypes = [P, C.c_uint64, C.c_int64, C.POINTER(gfbp_result)]
        L.gfbp_server_stats.argtypes = [P, C.POINTER(gfbp_server_stats_t)]
        L.gfbp_server_drain.argtypes = [P]
        L.gfbp_server_destroy.argtypes = [P]
        L.gfbp_server_destroy.restype = None
        for fn in ("gfbp_server_create", "gfbp_server_submit", "gfbp_server_wait", "gfbp_server_stats",
                   "gfbp_server_drain"):
            getattr(L, fn).restype = C.c_int
        L._server_typed = True
    return L


class Server:
    """gfbp_server: continuous batching of decode requests with host inputs and
    outputs (numpy arrays)."""

    def __init__(self, hbm_budget_bytes: int, round_iters: int = 8):
        h = C.c_void_p()
        _ok(_server_lib().gfbp_server_create(int(hbm_budget_bytes), int(round_iters), C.byref(h)),
            "gfbp_server_create")
        self.handle = h
        self._pending = {}

    def submit(self, code: Code, obs, channel: str = "bsc", param: float = 0.0, frame_param=None, T=None,
               K: int = 0, schedule: str = "sus", max_iter: int = 100) -> int:
        obs = np.ascontiguousarray(obs, dtype=np.float32)
        F = int(obs.shape[0])
        out = dict(x_hat=np.zeros((F, code.N), np.uint8), iters=np.zeros(F, np.int32),
                   converged=np.zeros(F, np.uint8))
        fp = None if frame_param is None else np.ascontiguousarray(frame_param, dtype=np.float32)
        pr, keep = _prior(T, K, None)
        req = gfbp_request(code.handle, F, obs.ctypes.data,
                           gfbp_channel(CHANNEL[channel], float(param), None if fp is None else fp.ctypes.data),
                           C.cast(C.pointer(pr), C.c_void_p) if T is not None else None, SCHEDULE[schedule],
                           int(max_iter), out["x_hat"].ctypes.data, out["iters"].ctypes.data,
                           out["converged"].ctypes.data)
        rid = C.c_uint64()
        _ok(_server_lib().gfbp_server_submit(self.handle, C.byref(req), C.byref(rid)), "gfbp_server_submit")
        self._pending[rid.value] = (out, obs, fp, pr, keep)
        return rid.value

    def wait(self, rid: int, timeout_s: float = 60.0):
        res = gfbp_result()
        _ok(_server_lib().gfbp_server_wait(self.handle, C.c_uint64(rid), int(timeout_s * 1e6), C.byref(res)),
            "gfbp_server_wait")
        out = self._pending.pop(rid)[0]
        out.update(latency_us=res.latency_us, queue_us=res.queue_us, rounds=res.rounds)
        return out

    def stats(self):
        st = gfbp_server_stats_t()
        _ok(_server_lib().gfbp_server_stats(self.handle, C.byref(st)), "gfbp_server_stats")
        return {k: getattr(st, k) for k, _ in gfbp_server_stats_t._fields_}

    def drain(self):
        _ok(_server_lib().gfbp_server_drain(self.handle), "gfbp_server_drain")

    def close(self):
        if getattr(self, "handle", None):
            _server_lib().gfbp_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
