"""Thin ctypes binding of the C ABI in include/sfft.h (argument marshalling only).

Every function keeps the C name and forwards to the CUDA library
``libsfft.so``; nothing here computes any step of the method.  Device buffers
are torch CUDA tensors (or raw integer addresses); streams are torch streams,
raw ``cudaStream_t`` integers, or None for the current torch stream.  A failed
call raises ``SfftError`` carrying the library's status and reason.  If the
library cannot be built or loaded the import of the first call fails loudly:
there is no fallback path.
"""
from __future__ import annotations

import ctypes
import threading

from . import build as _build

_lock = threading.Lock()
_lib = None

_i32 = ctypes.c_int32
_i64 = ctypes.c_int64
_u64 = ctypes.c_uint64
_p = ctypes.c_void_p

SFFT_OK, SFFT_EINVAL, SFFT_ENOMEM, SFFT_ECUDA, SFFT_EBUSY, SFFT_ETIMEDOUT, SFFT_EPENDING, SFFT_ENOTIMPL = range(8)


class sfft_opts(ctypes.Structure):
    _fields_ = [("c", _i32), ("T", _i32), ("precision", _i32), ("method", _i32), ("comb", _i32),
                ("estimator", _i32), ("refine", _i32), ("search_bits", _i32), ("residual", _i32),
                ("mode", _i32)]


class sfft_plan_info(ctypes.Structure):
    _fields_ = [("N", _i64), ("w", _i64), ("K", _i32), ("B", _i32), ("L", _i32), ("c", _i32), ("T", _i32),
                ("nsel", _i32), ("seed", _u64), ("samples_touched", _i64), ("candidate_capacity", _i64),
                ("device_bytes", ctypes.c_size_t), ("method", _i32), ("estimator", _i32), ("refine", _i32)]


class sfft_exec_stats(ctypes.Structure):
    _fields_ = [("candidates", _i64), ("estimated", _i64), ("recorded", _i64), ("fallback", _i32),
                ("theta", ctypes.c_float), ("iterations", _i32), ("residual_energy", ctypes.c_double),
                ("bucket_energy", ctypes.c_double), ("device_error", _i32)]


class sfft_request(ctypes.Structure):
    _fields_ = [("N", _i64), ("w", _i64), ("K", _i32), ("B", _i32), ("L", _i32), ("seed", _u64),
                ("opts", sfft_opts), ("x_dev", _p), ("idx_dev", _p), ("val_dev", _p), ("count_samples", _i32)]


class sfft_result(ctypes.Structure):
    _fields_ = [("k_out", _i32), ("status", _i32), ("samples_touched", _i64), ("latency_ns", _i64)]


_SIGS = {
    "sfft_plan_create": (_i32, [ctypes.POINTER(_p), _i64, _i32, _i32, _i64, _i32, _u64]),
    "sfft_plan_create_ex": (_i32, [ctypes.POINTER(_p), _i64, _i32, _i32, _i64, _i32, _u64,
                                   ctypes.POINTER(sfft_opts)]),
    "sfft_plan_destroy": (None, [_p]),
    "sfft_plan_reseed": (_i32, [_p, _u64, _p]),
    "sfft_plan_get_info": (_i32, [_p, ctypes.POINTER(sfft_plan_info)]),
    "sfft_plan_get_loops": (_i32, [_p, _p, _p, _p]),
    "sfft_loop_params": (_i32, [_i64, _i32, _u64, _p, _p, _p]),
    "sfft_suggest_params": (_i32, [_i64, _i32, ctypes.c_double, _p, _p, _p]),
    "sfft_window_walk": (_i32, [_i64, _i64, _u64, _u64, _i64, _p]),
    "sfft_tuning_load": (_i32, [ctypes.c_char_p]),
    "sfft_tuning_clear": (None, []),
    "sfft_tuning_classes": (_i32, []),
    "sfft_plan_last_stats": (_i32, [_p, ctypes.POINTER(sfft_exec_stats)]),
    "sfft_execute": (_i32, [_p, _p, _p, _p, _p, _p]),
    "sfft_execute_host": (_i32, [_p, _p, _p, _p, _p, _p]),
    "sfft_execute_batch": (_i32, [_p, _p, _p, _p, _p, _i32, _p]),
    "sfft_execute_batch_timed": (_i32, [_p, _p, _p, _p, _p, _i32, _i32, ctypes.POINTER(ctypes.c_float),
                                        ctypes.POINTER(ctypes.c_float), _p]),
    "sfft_execute_batch_host": (_i32, [_p, _p, _p, _p, _p, _i32, _p]),
    "sfft_bucketize": (_i32, [_p, _p, _p, _p]),
    "sfft_select": (_i32, [_p, _p, _p, _p]),
    "sfft_vote": (_i32, [_p, _p, _p, _p, _i64, _p]),
    "sfft_estimate": (_i32, [_p, _p, _p, _i64, _p, _p]),
    "sfft_bucketize_noalloc": (_i32, [_i64, _i32, _i64, _i32, _u64, _p, _p, _p]),
    "sfft_server_create": (_i32, [ctypes.POINTER(_p), ctypes.c_size_t, _i32]),
    "sfft_submit": (_i32, [_p, ctypes.POINTER(sfft_request), ctypes.POINTER(_u64)]),
    "sfft_poll": (_i32, [_p, _u64, ctypes.POINTER(sfft_result)]),
    "sfft_wait": (_i32, [_p, _u64, _i64, ctypes.POINTER(sfft_result)]),
    "sfft_server_set_paused": (_i32, [_p, _i32]),
    "sfft_server_destroy": (None, [_p]),
    "sfft_status_string": (ctypes.c_char_p, [_i32]),
    "sfft_last_error": (ctypes.c_char_p, []),
}

EXPORTED = tuple(_SIGS)


class SfftError(RuntimeError):
    def __init__(self, status: int, reason: str):
        super().__init__(f"{status_string(status)} ({status}): {reason}")
        self.status = status


def lib():
    """Load (building first if needed) the CUDA library; raises if unavailable."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            so = ctypes.CDLL(path)
            for name, (res, args) in _SIGS.items():
                fn = getattr(so, name)
                fn.restype = res
                fn.argtypes = args
            _lib = so
    return _lib


def library_path() -> str:
    return _build.LIB


def status_string(status: int) -> str:
    return lib().sfft_status_string(status).decode()


def _check(status: int):
    if status != SFFT_OK:
        raise SfftError(status, lib().sfft_last_error().decode())
    return status


def _addr(t) -> int | None:
    """Device address of a tensor (must be contiguous) or an integer address."""
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if not t.is_contiguous():
        raise ValueError("buffers must be contiguous")
    return t.data_ptr()


def _stream(stream) -> int | None:
    if stream is None:
        import torch

        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class Plan:
    """Owning handle of an ``sfft_plan*`` (destroyed with the object)."""

    def __init__(self, handle: int):
        self.handle = handle
        self._info = None

    @property
    def info(self) -> sfft_plan_info:
        if self._info is None:
            self._info = sfft_plan_get_info(self)
        return self._info

    def destroy(self):
        if self.handle:
            lib().sfft_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass

    @property
    def _as_parameter_(self):
        return ctypes.c_void_p(self.handle)


def sfft_plan_create(N, K, B, w, L, seed, opts: sfft_opts | None = None) -> Plan:
    h = _p()
    if opts is None:
        _check(lib().sfft_plan_create(ctypes.byref(h), N, K, B, w, L, seed))
    else:
        _check(lib().sfft_plan_create_ex(ctypes.byref(h), N, K, B, w, L, seed, ctypes.byref(opts)))
    return Plan(h.value)


SFFT_METHOD_VOTING = 0
SFFT_METHOD_PHASE = 1
SFFT_METHOD_COMB = 2
SFFT_METHOD_SEARCH = 3
SFFT_ESTIMATOR_MEDIAN = 0
SFFT_ESTIMATOR_MEAN = 1
SFFT_MAX_REFINE = 8
SFFT_GATHER_AUTO = 0
SFFT_GATHER_PERMUTED = 1
SFFT_GATHER_STREAM = 2


def sfft_plan_create_ex(N, K, B, w, L, seed, c=0, T=0, precision=0, method=SFFT_METHOD_VOTING, comb=0,
                        estimator=SFFT_ESTIMATOR_MEDIAN, refine=0, search_bits=0, residual=0,
                        mode=SFFT_GATHER_AUTO) -> Plan:
    return sfft_plan_create(N, K, B, w, L, seed,
                            sfft_opts(c, T, precision, method, comb, estimator, refine, search_bits, residual,
                                      mode))


def sfft_window_walk(N, w, sigma, tau, p0):
    """(first read p >= p0, its tap, k+, alpha, k-, beta) of one loop's window (host only)."""
    out = (ctypes.c_int64 * 6)()
    _check(lib().sfft_window_walk(N, w, sigma, tau, p0, out))
    return tuple(out)


def sfft_plan_destroy(plan: Plan):
    plan.destroy()


def sfft_plan_reseed(plan: Plan, seed: int, stream=None):
    """New loop parameters for `seed`, uploaded on `stream` (scratch and tables kept)."""
    _check(lib().sfft_plan_reseed(plan.handle, seed, _stream(stream)))
    plan._info = None


def sfft_plan_get_info(plan: Plan) -> sfft_plan_info:
    info = sfft_plan_info()
    _check(lib().sfft_plan_get_info(plan.handle, ctypes.byref(info)))
    return info


def sfft_plan_get_loops(plan: Plan):
    L = plan.info.L
    s, t, si = (ctypes.c_uint32 * L)(), (ctypes.c_uint32 * L)(), (ctypes.c_uint32 * L)()
    _check(lib().sfft_plan_get_loops(plan.handle, s, t, si))
    return list(s), list(t), list(si)


def sfft_plan_last_stats(plan: Plan) -> sfft_exec_stats:
    st = sfft_exec_stats()
    _check(lib().sfft_plan_last_stats(plan.handle, ctypes.byref(st)))
    return st


def sfft_loop_params(N, L, seed):
    s, t, si = (ctypes.c_uint32 * L)(), (ctypes.c_uint32 * L)(), (ctypes.c_uint32 * L)()
    _check(lib().sfft_loop_params(N, L, seed, s, t, si))
    return list(s), list(t), list(si)


def sfft_suggest_params(N, K, snr_db=None):
    """(B, w, L) for a signal shape by the library's size-class rule (snr_db None: noiseless)."""
    B, w, L = ctypes.c_int32(), ctypes.c_int64(), ctypes.c_int32()
    snr = float("nan") if snr_db is None else float(snr_db)
    _check(lib().sfft_suggest_params(N, K, snr, ctypes.byref(B), ctypes.byref(w), ctypes.byref(L)))
    return B.value, w.value, L.value


def sfft_tuning_load(path: str):
    """Load the autotuner's JSON cache of per-size-class plan sizes."""
    _check(lib().sfft_tuning_load(str(path).encode()))


def sfft_tuning_clear():
    lib().sfft_tuning_clear()


def sfft_tuning_classes() -> int:
    return int(lib().sfft_tuning_classes())


def sfft_execute(plan: Plan, x, idx, val, k_out, stream=None):
    _check(lib().sfft_execute(plan.handle, _addr(x), _addr(idx), _addr(val), _addr(k_out), _stream(stream)))


def sfft_execute_host(plan: Plan, x_host, idx_host, val_host, k_out_host, stream=None):
    """Host-buffer variant: numpy arrays or pinned CPU tensors (contiguous)."""
    def hp(a):
        if hasattr(a, "ctypes"):
            return a.ctypes.data
        return _addr(a)

    _check(lib().sfft_execute_host(plan.handle, hp(x_host), hp(idx_host), hp(val_host), hp(k_out_host),
                                   _stream(stream)))


def sfft_execute_batch(plans, xs, idxs, vals, k_out, stream=None):
    n = len(plans)
    arr = lambda vals_: (_p * n)(*vals_)  # noqa: E731
    _check(lib().sfft_execute_batch(arr([p.handle for p in plans]), arr([_addr(x) for x in xs]),
                                    arr([_addr(i) for i in idxs]), arr([_addr(v) for v in vals]),
                                    _addr(k_out), n, _stream(stream)))


STAGES = ("gather_fold", "fft_select", "vote_scan", "estimate", "refine", "residual")


def sfft_execute_batch_timed(plans, xs, idxs, vals, k_out, steps, stream=None):
    """Returns (total_ms, {stage: summed ms}) over `steps` back-to-back runs."""
    n = len(plans)
    arr = lambda vals_: (_p * n)(*vals_)  # noqa: E731
    total = ctypes.c_float()
    stages = (ctypes.c_float * len(STAGES))()
    _check(lib().sfft_execute_batch_timed(arr([p.handle for p in plans]), arr([_addr(x) for x in xs]),
                                          arr([_addr(i) for i in idxs]), arr([_addr(v) for v in vals]),
                                          _addr(k_out), n, steps, ctypes.byref(total), stages, _stream(stream)))
    return total.value, dict(zip(STAGES, list(stages)))


def _host_addr(a):
    if hasattr(a, "ctypes"):
        return a.ctypes.data
    return _addr(a)


def sfft_execute_batch_host(plans, xs, idxs, vals, k_out, stream=None):
    """Host-buffer batch: numpy arrays or (pinned) CPU tensors."""
    n = len(plans)
    arr = lambda vals_: (_p * n)(*vals_)  # noqa: E731
    _check(lib().sfft_execute_batch_host(arr([p.handle for p in plans]), arr([_host_addr(x) for x in xs]),
                                         arr([_host_addr(i) for i in idxs]), arr([_host_addr(v) for v in vals]),
                                         _host_addr(k_out), n, _stream(stream)))


def sfft_bucketize(plan: Plan, x, zhat, stream=None):
    _check(lib().sfft_bucketize(plan.handle, _addr(x), _addr(zhat), _stream(stream)))


def sfft_select(plan: Plan, zhat, sel, stream=None):
    _check(lib().sfft_select(plan.handle, _addr(zhat), _addr(sel), _stream(stream)))


def sfft_vote(plan: Plan, sel, cand, n_cand, cap, stream=None):
    _check(lib().sfft_vote(plan.handle, _addr(sel), _addr(cand), _addr(n_cand), cap, _stream(stream)))


def sfft_estimate(plan: Plan, zhat, cand, n_cand, est, stream=None):
    _check(lib().sfft_estimate(plan.handle, _addr(zhat), _addr(cand), n_cand, _addr(est), _stream(stream)))


def sfft_bucketize_noalloc(N, B, w, L, seed, x, zhat, stream=None):
    """Bucket values without allocating (scratch in the library's static
    device memory); see include/sfft.h for the limits and the sharing rule."""
    _check(lib().sfft_bucketize_noalloc(N, B, w, L, seed, _addr(x), _addr(zhat), _stream(stream)))


class Server:
    def __init__(self, handle: int):
        self.handle = handle

    def destroy(self):
        if self.handle:
            lib().sfft_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def sfft_server_create(hbm_budget_bytes: int, max_slots: int) -> Server:
    h = _p()
    _check(lib().sfft_server_create(ctypes.byref(h), hbm_budget_bytes, max_slots))
    return Server(h.value)


def sfft_server_set_paused(srv: Server, paused: bool):
    _check(lib().sfft_server_set_paused(srv.handle, int(bool(paused))))


def sfft_server_destroy(srv: Server):
    srv.destroy()


def sfft_submit(srv: Server, N, K, B, w, L, seed, x, idx, val, c=0, T=0, method=0, comb=0, estimator=0,
                refine=0, search_bits=0, residual=0, count_samples=1, precision=0, mode=0) -> int:
    req = sfft_request(N, w, K, B, L, seed,
                       sfft_opts(c, T, precision, method, comb, estimator, refine, search_bits, residual, mode),
                       _addr(x), _addr(idx), _addr(val), int(count_samples))
    ticket = _u64()
    _check(lib().sfft_submit(srv.handle, ctypes.byref(req), ctypes.byref(ticket)))
    return ticket.value


def sfft_poll(srv: Server, ticket: int):
    """Returns an sfft_result once done, None while pending."""
    res = sfft_result()
    st = lib().sfft_poll(srv.handle, ticket, ctypes.byref(res))
    if st == SFFT_EPENDING:
        return None
    _check(st)
    return res


def sfft_wait(srv: Server, ticket: int, timeout_ms: int = 60000):
    res = sfft_result()
    _check(lib().sfft_wait(srv.handle, ticket, timeout_ms, ctypes.byref(res)))
    return res
