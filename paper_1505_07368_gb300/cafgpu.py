"""Python binding of libcafgpu.so (the C ABI in include/caf_gpu.h).

Argument marshalling only: every step of the actor path -- mailboxes,
scheduling, payloads, replies -- runs in the library's CUDA kernels.  There
is no fallback: if the library cannot be loaded, or no CUDA device is
present, the calls raise.

PyTorch is used by callers for device memory (``tensor.data_ptr()``) and
streams; this module takes plain integers for device addresses.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _build

# ---- constants (caf_gpu.h) ------------------------------------------------
OK, EINVAL, ENOMEM, EAGAIN, ETIMEDOUT, EDEAD, EWAITLIMIT, ESTATE, ECUDA, EBOUNDS = 0, -1, -2, -3, -4, -5, -6, -7, -8, -9
FACTOR_U64, GEMM_BF16, GEMM_SPLIT_BF16X3, RING_TOKEN, SINK, SOURCE, MANDELBROT, FORK = 1, 2, 3, 4, 5, 6, 7, 8
BACKEND_PERSISTENT, BACKEND_PER_MESSAGE_LAUNCH = 0, 1
SCHED_GLOBAL, SCHED_STEAL = 0, 1
REPLY_OK, REPLY_NOFACTOR, REPLY_DEAD, REPLY_REJECTED = 0, 1, 2, 3
MSG_START = 1
ACTOR_MASTER = 1
ACTOR_RECREATE = 2

DMSG_DTYPE = np.dtype([("actor", "<u4"), ("kind", "<u4"), ("sender", "<u4"), ("sender_seq", "<u4"),
                       ("u64", "<u8"), ("tag", "<u8")])
DREPLY_DTYPE = np.dtype([("status", "<i4"), ("done", "<u4"), ("r0", "<u8"), ("r1", "<u8"), ("t_done", "<u8")])
GEMM_DESC_DTYPE = np.dtype([("A", "<u8"), ("B", "<u8"), ("C", "<u8"), ("n", "<u4"), ("pad", "<u4")])
MANDEL_DESC_DTYPE = np.dtype([("out", "<u8"), ("width", "<u4"), ("rows", "<u4"), ("row0", "<u4"),
                              ("max_iter", "<u4"), ("x0", "<f4"), ("y0", "<f4"), ("dx", "<f4"), ("dy", "<f4")])
MANDEL_MAX_PIXELS = 1 << 24
MANDEL_MAX_ITER = 1 << 16
LOG_DTYPE = np.dtype([("actor", "<u4"), ("sender", "<u4"), ("sender_seq", "<u4"), ("kind", "<u4"),
                      ("stamp", "<u8"), ("tag", "<u8"), ("value", "<u8")])


class CafGpuError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(f"{what}: {strerror(code)} ({code})")


class RuntimeCfg(ctypes.Structure):
    _fields_ = [("max_actors", ctypes.c_uint32), ("mailbox_capacity", ctypes.c_uint32),
                ("max_inflight_requests", ctypes.c_uint32), ("ingress_capacity", ctypes.c_uint32),
                ("ctas_per_sm", ctypes.c_uint32), ("max_msgs_per_claim", ctypes.c_uint32),
                ("factor_batch", ctypes.c_uint32), ("factor_warps", ctypes.c_uint32),
                ("max_factor_n", ctypes.c_uint64), ("mem_budget_bytes", ctypes.c_uint64),
                ("wait_limit_ns", ctypes.c_uint64), ("idle_exit_ns", ctypes.c_uint64),
                ("validation_mode", ctypes.c_uint32), ("log_capacity", ctypes.c_uint32),
                ("cuda_stream", ctypes.c_void_p), ("gemm_items_per_round", ctypes.c_uint32),
                ("fork_pool", ctypes.c_uint32), ("scheduler", ctypes.c_uint32), ("factor_split", ctypes.c_uint32),
                ("gemm_tile_n", ctypes.c_uint32)]


class ActorCfg(ctypes.Structure):
    _fields_ = [("mailbox_capacity", ctypes.c_uint32), ("flags", ctypes.c_uint32),
                ("next", ctypes.c_uint64), ("worker", ctypes.c_uint64), ("init_state", ctypes.c_int32),
                ("factor_count", ctypes.c_uint32), ("factor_n", ctypes.c_void_p),
                ("factor_replies", ctypes.c_void_p), ("ring_len", ctypes.c_uint32),
                ("incarnations", ctypes.c_uint32)]


class Msg(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_uint32), ("flags", ctypes.c_uint32), ("sender", ctypes.c_uint32),
                ("n", ctypes.c_uint32), ("u64", ctypes.c_uint64), ("tag", ctypes.c_uint64),
                ("A", ctypes.c_void_p), ("B", ctypes.c_void_p), ("C", ctypes.c_void_p)]


class MandelDesc(ctypes.Structure):
    """caf_gpu_mandel_desc: rows row0 .. row0+rows-1 of an image `width` wide;
    pixel (i, j) is c = (x0 + i dx) + (y0 + j dy) i; out: device uint32 counts."""
    _fields_ = [("out", ctypes.c_void_p), ("width", ctypes.c_uint32), ("rows", ctypes.c_uint32),
                ("row0", ctypes.c_uint32), ("max_iter", ctypes.c_uint32), ("x0", ctypes.c_float),
                ("y0", ctypes.c_float), ("dx", ctypes.c_float), ("dy", ctypes.c_float)]


class Reply(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("kind", ctypes.c_uint32), ("r0", ctypes.c_uint64),
                ("r1", ctypes.c_uint64), ("t_done", ctypes.c_uint64)]


class Stats(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_uint64), ("messages", ctypes.c_uint64),
                ("device_sends", ctypes.c_uint64), ("claims", ctypes.c_uint64),
                ("factor_items", ctypes.c_uint64), ("prime_tests", ctypes.c_uint64),
                ("gemm_tiles", ctypes.c_uint64), ("error_word", ctypes.c_uint32), ("pad", ctypes.c_uint32),
                ("diag0", ctypes.c_uint64), ("diag1", ctypes.c_uint64), ("t_mark", ctypes.c_uint64),
                ("device_spawns", ctypes.c_uint64)]


SERVE_REQ_DTYPE = np.dtype([("actor", "<u8"), ("t_arrival", "<f8"), ("u64", "<u8"), ("n", "<u4"), ("pad", "<u4"),
                            ("A", "<u8"), ("B", "<u8")])
SERVE_RESULT_DTYPE = np.dtype([("status", "<i4"), ("pad", "<u4"), ("r0", "<u8"), ("r1", "<u8"),
                               ("c_offset", "<u8"), ("t_admit", "<f8"), ("t_done", "<f8")])


class ServeCfg(ctypes.Structure):
    _fields_ = [("mem_budget_bytes", ctypes.c_uint64), ("c_arena", ctypes.c_void_p),
                ("c_arena_bytes", ctypes.c_uint64), ("timeout_ns", ctypes.c_uint64)]


class ServeStats(ctypes.Structure):
    _fields_ = [("wall_s", ctypes.c_double), ("peak_inflight_bytes", ctypes.c_uint64),
                ("peak_inflight", ctypes.c_uint32), ("pad", ctypes.c_uint32), ("launches", ctypes.c_uint64)]


# Every symbol include/caf_gpu.h declares (checked by the CPU tests).
EXPORTS = [
    "caf_gpu_runtime_create", "caf_gpu_runtime_destroy", "caf_gpu_spawn", "caf_gpu_send",
    "caf_gpu_request", "caf_gpu_await", "caf_gpu_request_batch", "caf_gpu_await_batch",
    "caf_gpu_request_batch_device", "caf_gpu_sync", "caf_gpu_stream_sync", "caf_gpu_set_backend",
    "caf_gpu_reset_actors", "caf_gpu_actor_state", "caf_gpu_stats_read", "caf_gpu_read_log",
    "caf_gpu_stream", "caf_gpu_mark", "caf_gpu_prime_table", "caf_gpu_debug_wait_expiry", "caf_gpu_clear_error",
    "caf_gpu_measure_mul_rates", "caf_gpu_measure_fp32_rate", "caf_gpu_measure_latency", "caf_gpu_sink_totals",
    "caf_gpu_graph_begin", "caf_gpu_graph_end", "caf_gpu_graph_launch", "caf_gpu_graph_destroy",
    "caf_gpu_serve_run", "caf_gpu_factor_static", "caf_gpu_check_guards", "caf_gpu_debug_inject",
    "caf_gpu_strerror",
]
FACTOR_STATIC_MAX = 4096

_lib = None


def load(build: bool = True):
    """Load libcafgpu.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if build:
        _build.build()
    if not os.path.exists(_build.LIB):
        raise OSError(f"libcafgpu.so not built ({_build.LIB})")
    L = ctypes.CDLL(_build.LIB)
    vp, u32, u64, i32 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int32
    P = ctypes.POINTER
    sig = {
        "caf_gpu_runtime_create": [P(RuntimeCfg), P(vp)],
        "caf_gpu_runtime_destroy": [vp],
        "caf_gpu_spawn": [vp, u32, P(ActorCfg), P(u64)],
        "caf_gpu_send": [vp, u64, P(Msg)],
        "caf_gpu_request": [vp, u64, P(Msg), P(u64)],
        "caf_gpu_await": [vp, u64, u64, P(Reply)],
        "caf_gpu_request_batch": [vp, vp, vp, u32, vp],
        "caf_gpu_await_batch": [vp, vp, u32, u64, vp],
        "caf_gpu_request_batch_device": [vp, vp, u32, vp],
        "caf_gpu_sync": [vp],
        "caf_gpu_stream_sync": [vp],
        "caf_gpu_set_backend": [vp, ctypes.c_int],
        "caf_gpu_reset_actors": [vp],
        "caf_gpu_actor_state": [vp, u64, P(u32), P(i32)],
        "caf_gpu_stats_read": [vp, P(Stats)],
        "caf_gpu_read_log": [vp, vp, u32, P(u32)],
        "caf_gpu_prime_table": [vp, P(vp), P(u32)],
        "caf_gpu_debug_wait_expiry": [vp, u64],
        "caf_gpu_measure_mul_rates": [vp],
        "caf_gpu_measure_fp32_rate": [vp],
        "caf_gpu_measure_latency": [vp],
        "caf_gpu_sink_totals": [vp, u64, P(u64), P(u64)],
        "caf_gpu_clear_error": [vp],
        "caf_gpu_mark": [vp],
        "caf_gpu_factor_static": [vp, u32, vp, vp],
        "caf_gpu_graph_begin": [vp],
        "caf_gpu_graph_end": [vp, P(vp)],
        "caf_gpu_graph_launch": [vp, vp],
        "caf_gpu_graph_destroy": [vp],
        "caf_gpu_serve_run": [vp, vp, u32, P(ServeCfg), vp, P(ServeStats)],
        "caf_gpu_check_guards": [vp, P(u32)],
        "caf_gpu_debug_inject": [vp, u32, u64],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    L.caf_gpu_stream.argtypes = [vp]
    L.caf_gpu_stream.restype = vp
    L.caf_gpu_strerror.argtypes = [ctypes.c_int]
    L.caf_gpu_strerror.restype = ctypes.c_char_p
    _lib = L
    return L


def measure_mul_rates() -> dict:
    """Measured low-multiply, high-multiply and divisibility-test-chain rates (multiplies/s)."""
    out = (ctypes.c_double * 3)()
    _check(load().caf_gpu_measure_mul_rates(out), "caf_gpu_measure_mul_rates")
    return {"mul_lo_per_s": out[0], "mul_hi_per_s": out[1], "test_chain_mul_per_s": out[2]}


def measure_fp32_rate() -> float:
    """Measured float32 multiply + add rate (operations/s, each rounded on its own)."""
    out = ctypes.c_double()
    _check(load().caf_gpu_measure_fp32_rate(ctypes.byref(out)), "caf_gpu_measure_fp32_rate")
    return out.value


def measure_latency() -> dict:
    """Measured latencies (ns): returning L2 atomic, L2 acquire load, store +
    fence.sc, and one-way flag handoff between two SMs."""
    out = (ctypes.c_double * 4)()
    _check(load().caf_gpu_measure_latency(out), "caf_gpu_measure_latency")
    return {"atomic_ns": out[0], "load_acquire_ns": out[1], "store_fence_sc_ns": out[2], "handoff_ns": out[3]}


def factor_static(d_n: int, count: int, d_replies: int, stream: int = 0) -> int:
    """caf_gpu_factor_static: factor `count` numbers at device address `d_n`
    into the caf_gpu_dreply array at `d_replies`, allocating nothing.  Returns
    the status code (0 on success)."""
    return load().caf_gpu_factor_static(d_n, count, d_replies, stream or None)


def strerror(code: int) -> str:
    try:
        return load(build=False).caf_gpu_strerror(code).decode()
    except OSError:
        return f"error {code}"


def _check(code: int, what: str) -> int:
    if code != 0:
        raise CafGpuError(code, what)
    return code


class Runtime:
    """One caf_gpu runtime (actor table, mailboxes, prime table) on the current CUDA device."""

    def __init__(self, **cfg):
        self.L = load()
        c = RuntimeCfg()
        for k, v in cfg.items():
            if not hasattr(c, k):
                raise TypeError(f"unknown runtime cfg field {k}")
            setattr(c, k, v)
        h = ctypes.c_void_p()
        _check(self.L.caf_gpu_runtime_create(ctypes.byref(c), ctypes.byref(h)), "caf_gpu_runtime_create")
        self.h = h
        self._keep = []

    def close(self):
        if self.h:
            rc = self.L.caf_gpu_runtime_destroy(self.h)
            self.h = None
            _check(rc, "caf_gpu_runtime_destroy")

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- actors -------------------------------------------------------------
    def spawn(self, kernel_id: int, mailbox_capacity: int = 0, flags: int = 0, next: int = 0,
              worker: int = 0, init_state: int = 0, factor_n: int = 0, factor_count: int = 0,
              factor_replies: int = 0, ring_len: int = 0, incarnations: int = 0) -> int:
        c = ActorCfg(mailbox_capacity, flags, next, worker, init_state, factor_count, factor_n or None,
                     factor_replies or None, ring_len, incarnations)
        out = ctypes.c_uint64()
        _check(self.L.caf_gpu_spawn(self.h, kernel_id, ctypes.byref(c), ctypes.byref(out)), "caf_gpu_spawn")
        return out.value

    def check_guards(self) -> int:
        """Guard regions after the device arrays whose bytes changed (0: intact)."""
        out = ctypes.c_uint32()
        _check(self.L.caf_gpu_check_guards(self.h, ctypes.byref(out)), "caf_gpu_check_guards")
        return out.value

    def debug_inject(self, what: int, arg: int) -> int:
        """Host-side fault injection for tests (returns the status code)."""
        return self.L.caf_gpu_debug_inject(self.h, what, arg)

    def actor_state(self, actor: int):
        lc = ctypes.c_uint32()
        us = ctypes.c_int32()
        _check(self.L.caf_gpu_actor_state(self.h, actor, ctypes.byref(lc), ctypes.byref(us)), "caf_gpu_actor_state")
        return lc.value, us.value

    def sink_totals(self, actor: int):
        """(messages handled, sum of their values) of a SINK."""
        c = ctypes.c_uint64()
        t = ctypes.c_uint64()
        _check(self.L.caf_gpu_sink_totals(self.h, actor, ctypes.byref(c), ctypes.byref(t)), "caf_gpu_sink_totals")
        return c.value, t.value

    # -- messages -----------------------------------------------------------
    @staticmethod
    def msg(kind: int, u64: int = 0, sender: int = 0, flags: int = 0, tag: int = 0, n: int = 0,
            A: int = 0, B: int = 0, C: int = 0) -> Msg:
        return Msg(kind, flags, sender, n, u64, tag, A or None, B or None, C or None)

    @staticmethod
    def mandel_msg(desc: MandelDesc, sender: int = 0, tag: int = 0) -> Msg:
        """A MANDELBROT message naming `desc` (the runtime copies it at the call)."""
        return Msg(MANDELBROT, 0, sender, 0, ctypes.addressof(desc), tag, None, None, None)

    def send(self, actor: int, m: Msg) -> None:
        _check(self.L.caf_gpu_send(self.h, actor, ctypes.byref(m)), "caf_gpu_send")

    def try_send(self, actor: int, m: Msg) -> int:
        return self.L.caf_gpu_send(self.h, actor, ctypes.byref(m))

    def request(self, actor: int, m: Msg) -> int:
        out = ctypes.c_uint64()
        _check(self.L.caf_gpu_request(self.h, actor, ctypes.byref(m), ctypes.byref(out)), "caf_gpu_request")
        return out.value

    def await_(self, handle: int, timeout_ns: int = 0):
        r = Reply()
        self._diag(self.L.caf_gpu_await(self.h, handle, timeout_ns, ctypes.byref(r)), "caf_gpu_await")
        return r.status, r.r0, r.r1

    def try_await(self, handle: int, timeout_ns: int = 0):
        r = Reply()
        rc = self.L.caf_gpu_await(self.h, handle, timeout_ns, ctypes.byref(r))
        return rc, (r.status, r.r0, r.r1)

    def request_batch(self, actors: np.ndarray, msgs) -> np.ndarray:
        """actors: uint64 array of actor ids; msgs: ctypes array of Msg."""
        actors = np.ascontiguousarray(actors, dtype=np.uint64)
        n = actors.size
        out = np.zeros(n, dtype=np.uint64)
        _check(self.L.caf_gpu_request_batch(self.h, actors.ctypes.data, ctypes.addressof(msgs), n,
                                            out.ctypes.data), "caf_gpu_request_batch")
        return out

    def _diag(self, code: int, what: str):
        if code == EWAITLIMIT:
            s = self.stats()
            what = f"{what} [error_word={s['error_word']:#x} diag=({s['diag0']}, {s['diag1']})]"
        _check(code, what)

    def await_batch(self, handles: np.ndarray, timeout_ns: int = 0):
        handles = np.ascontiguousarray(handles, dtype=np.uint64)
        out = (Reply * handles.size)()
        self._diag(self.L.caf_gpu_await_batch(self.h, handles.ctypes.data, handles.size, timeout_ns,
                                              ctypes.addressof(out)), "caf_gpu_await_batch")
        a = np.frombuffer(out, dtype=np.dtype([("status", "<i4"), ("kind", "<u4"), ("r0", "<u8"), ("r1", "<u8"),
                                               ("t_done", "<u8")]))
        return a.copy()

    def request_batch_device(self, d_msgs: int, count: int, d_replies: int) -> None:
        _check(self.L.caf_gpu_request_batch_device(self.h, d_msgs, count, d_replies),
               "caf_gpu_request_batch_device")

    # -- control --------------------------------------------------------------
    def sync(self):
        self._diag(self.L.caf_gpu_sync(self.h), "caf_gpu_sync")

    def stream_sync(self):
        self._diag(self.L.caf_gpu_stream_sync(self.h), "caf_gpu_stream_sync")

    def set_backend(self, backend: int):
        _check(self.L.caf_gpu_set_backend(self.h, backend), "caf_gpu_set_backend")

    def reset_actors(self):
        _check(self.L.caf_gpu_reset_actors(self.h), "caf_gpu_reset_actors")

    def stats(self) -> dict:
        s = Stats()
        _check(self.L.caf_gpu_stats_read(self.h, ctypes.byref(s)), "caf_gpu_stats_read")
        return {k: getattr(s, k) for k, _ in Stats._fields_ if k != "pad"}

    def read_log(self, cap: int = 1 << 22) -> np.ndarray:
        out = np.zeros(cap, dtype=LOG_DTYPE)
        cnt = ctypes.c_uint32()
        _check(self.L.caf_gpu_read_log(self.h, out.ctypes.data, cap, ctypes.byref(cnt)), "caf_gpu_read_log")
        return out[:cnt.value].copy()

    # -- serving -----------------------------------------------------------------
    def serve_run(self, reqs: np.ndarray, c_arena: int = 0, c_arena_bytes: int = 0, mem_budget_bytes: int = 0,
                  timeout_ns: int = 0):
        """Run the open-loop serving loop over `reqs` (SERVE_REQ_DTYPE, sorted by
        t_arrival).  Returns (results as SERVE_RESULT_DTYPE, stats dict)."""
        reqs = np.ascontiguousarray(reqs, dtype=SERVE_REQ_DTYPE)
        res = np.zeros(reqs.size, dtype=SERVE_RESULT_DTYPE)
        cfg = ServeCfg(mem_budget_bytes, c_arena or None, c_arena_bytes, timeout_ns)
        st = ServeStats()
        self._diag(self.L.caf_gpu_serve_run(self.h, reqs.ctypes.data, reqs.size, ctypes.byref(cfg),
                                            res.ctypes.data, ctypes.byref(st)), "caf_gpu_serve_run")
        return res, {k: getattr(st, k) for k, _ in ServeStats._fields_ if k != "pad"}

    # -- CUDA graphs ----------------------------------------------------------
    def graph_begin(self):
        _check(self.L.caf_gpu_graph_begin(self.h), "caf_gpu_graph_begin")

    def graph_end(self) -> int:
        g = ctypes.c_void_p()
        _check(self.L.caf_gpu_graph_end(self.h, ctypes.byref(g)), "caf_gpu_graph_end")
        return g.value

    def graph_launch(self, g: int):
        _check(self.L.caf_gpu_graph_launch(self.h, g), "caf_gpu_graph_launch")

    def graph_destroy(self, g: int):
        _check(self.L.caf_gpu_graph_destroy(g), "caf_gpu_graph_destroy")

    def mark(self):
        _check(self.L.caf_gpu_mark(self.h), "caf_gpu_mark")

    def stream(self) -> int:
        return self.L.caf_gpu_stream(self.h) or 0

    def prime_table(self):
        p = ctypes.c_void_p()
        n = ctypes.c_uint32()
        _check(self.L.caf_gpu_prime_table(self.h, ctypes.byref(p), ctypes.byref(n)), "caf_gpu_prime_table")
        return p.value or 0, n.value

    def debug_wait_expiry(self, limit_ns: int) -> int:
        return self.L.caf_gpu_debug_wait_expiry(self.h, limit_ns)

    def clear_error(self):
        _check(self.L.caf_gpu_clear_error(self.h), "caf_gpu_clear_error")
