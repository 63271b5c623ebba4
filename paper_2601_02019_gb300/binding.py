"""ctypes binding of include/aerosketch.h (argument marshalling only)."""
from __future__ import annotations

import ctypes as ct
import math
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "libaerosketch.so")

AS_OK, AS_EINVAL, AS_ENOMEM, AS_EDEVICE, AS_ENUMERIC, AS_ETIMEOUT, AS_EBUSY, AS_ENOTSUP = range(8)
AS_PERSISTENT, AS_FIXED_THETA, AS_SLIDING, AS_SITE, AS_COORDINATOR = range(5)
AS_FP32_PLAIN, AS_BF16, AS_BF16X3, AS_BF16X6 = 0, 1, 2, 3
AS_TRACE_DECISIONS = 0x1
AS_PROFILE = 0x2
AS_QUERY_DENSE = 0x4

EXPORTED = ("sketch_create", "sketch_update", "sketch_query", "sketch_query_gram", "sketch_get_buffer", "sketch_get_gram",
            "sketch_merge", "sketch_stats", "sketch_trace", "sketch_profile", "sketch_profile_reset",
            "sketch_profile_select",
            "sketch_destroy", "as_symeig", "as_symeig_noalloc", "as_tc_gemm", "as_status_str", "as_last_error",
            "as_inject_alloc_failure",
            "sketch_set_theta", "sketch_send_snapshots", "as_p5_create", "as_p5_round", "as_p5_query",
            "as_p5_query_gram", "as_p5_stats", "as_p5_site", "as_p5_coordinator", "as_p5_destroy",
            "as_sw_create", "as_sw_update", "as_sw_query", "as_sw_query_gram", "as_sw_stats", "as_sw_level",
            "as_sw_destroy", "sketch_footprint", "sketch_reserve", "sketch_update_many", "sketch_update_grouped",
            "as_server_create",
            "as_server_open", "as_server_submit", "as_server_wait", "as_server_drain", "as_server_session",
            "as_server_close", "as_server_stats", "as_server_reset_stats", "as_server_destroy", "as_wait_selftest")


class AsConfig(ct.Structure):
    _fields_ = [("d", ct.c_int32), ("ell", ct.c_int32), ("eps", ct.c_double), ("mode", ct.c_int32),
                ("prec", ct.c_int32), ("theta", ct.c_double), ("eps_si", ct.c_double), ("k_pi", ct.c_int32),
                ("q_si", ct.c_int32), ("seed", ct.c_uint64), ("stream_id", ct.c_uint64), ("flags", ct.c_uint32),
                ("reserved", ct.c_uint32), ("delta", ct.c_double)]


class AsServerConfig(ct.Structure):
    _fields_ = [("hbm_budget", ct.c_int64), ("workers", ct.c_int32), ("reserved", ct.c_int32)]


class AsServerCounters(ct.Structure):
    _fields_ = [("sessions_open", ct.c_int64), ("sessions_refused", ct.c_int64), ("footprint_bytes", ct.c_int64),
                ("requests_done", ct.c_int64), ("requests_failed", ct.c_int64), ("rows_done", ct.c_int64),
                ("p50_ms", ct.c_double), ("p99_ms", ct.c_double), ("max_ms", ct.c_double), ("mean_ms", ct.c_double),
                ("span_s", ct.c_double)]


class AsStats(ct.Structure):
    _fields_ = [("rows", ct.c_int64), ("ell", ct.c_int32), ("d", ct.c_int32), ("rows_in_buffer", ct.c_int32),
                ("reserved0", ct.c_int32), ("fro2", ct.c_double), ("theta", ct.c_double),
                ("shrinks", ct.c_int64), ("gates", ct.c_int64), ("dumps", ct.c_int64),
                ("snapshot_rank", ct.c_int64), ("si_runs", ct.c_int64), ("device_bytes", ct.c_int64),
                ("device_status", ct.c_int32), ("reserved1", ct.c_int32), ("kernel_launches", ct.c_int64),
                ("snapshots_sent", ct.c_int64), ("snapshots_received", ct.c_int64),
                ("grouped_batches", ct.c_int64)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_ if not f.startswith("reserved")}


class AsP5Counters(ct.Structure):
    _fields_ = [("rounds", ct.c_int64), ("messages", ct.c_int64), ("broadcasts", ct.c_int64),
                ("snapshots_sent", ct.c_int64), ("f_hat", ct.c_double), ("f_site", ct.c_double)]


class AsSwCounters(ct.Structure):
    _fields_ = [("rows", ct.c_int64), ("levels", ct.c_int32), ("last_level", ct.c_int32),
                ("raw_queued", ct.c_int64), ("snapshots_queued", ct.c_int64),
                ("popped_expired", ct.c_int64), ("popped_cap", ct.c_int64)]


class AsEvent(ct.Structure):
    _fields_ = [("i", ct.c_int64), ("sig2_pi", ct.c_double), ("theta", ct.c_double), ("j_stop", ct.c_int32),
                ("xi", ct.c_int32), ("ritz_k", ct.c_double), ("ritz_1", ct.c_double),
                ("amp_choice", ct.c_uint64)]


class AsKernelStat(ct.Structure):
    _fields_ = [("name", ct.c_char * 32), ("launches", ct.c_int64), ("total_ms", ct.c_double),
                ("flops", ct.c_double), ("bytes", ct.c_double), ("issued_flops", ct.c_double)]


class AeroSketchError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        msg = f"{what}: {lib().as_status_str(code).decode()}"
        cuda = lib().as_last_error().decode()
        if cuda and code == AS_EDEVICE:   # name the CUDA call that failed
            msg += f" [{cuda}]"
        super().__init__(msg)


_LIB = None


def load_library(path: str = LIB_PATH) -> ct.CDLL:
    """Load libaerosketch.so and declare every exported signature."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with paper_2601_02019_gb300/build.py")
    L = ct.CDLL(path)
    P, I64, I32 = ct.c_void_p, ct.c_int64, ct.c_int32
    L.sketch_create.argtypes = [ct.POINTER(AsConfig), P, ct.POINTER(P)]
    L.sketch_update.argtypes = [P, P, I64, I64]
    L.sketch_query.argtypes = [P, I64, P, I64, ct.POINTER(I32)]
    L.sketch_query_gram.argtypes = [P, I64, P]
    L.sketch_get_buffer.argtypes = [P, P, ct.POINTER(I32)]
    L.sketch_get_gram.argtypes = [P, P]
    L.sketch_merge.argtypes = [P, P]
    L.sketch_stats.argtypes = [P, ct.POINTER(AsStats)]
    L.sketch_trace.argtypes = [P, ct.POINTER(AsEvent), I64, ct.POINTER(I64)]
    L.sketch_profile.argtypes = [P, ct.POINTER(AsKernelStat), I32, ct.POINTER(I32)]
    L.sketch_profile_reset.argtypes = [P]
    L.sketch_profile_select.argtypes = [P, ct.c_uint32]
    L.sketch_destroy.argtypes = [P]
    L.as_symeig.argtypes = [I32, P, I32, P, P]
    L.as_symeig_noalloc.argtypes = [I32, P, I32, P, P, P]
    L.as_inject_alloc_failure.argtypes = [I32]
    L.as_tc_gemm.argtypes = [I32, I32, I32, P, P, I32, I32, P]
    L.sketch_set_theta.argtypes = [P, ct.c_double]
    L.sketch_send_snapshots.argtypes = [P, P, ct.POINTER(I32)]
    L.as_p5_create.argtypes = [ct.POINTER(AsConfig), I32, P, ct.POINTER(P)]
    L.as_p5_round.argtypes = [P, ct.POINTER(P), ct.POINTER(I64), ct.POINTER(I64)]
    L.as_p5_query.argtypes = [P, P, I64, ct.POINTER(I32)]
    L.as_p5_query_gram.argtypes = [P, P]
    L.as_p5_stats.argtypes = [P, ct.POINTER(AsP5Counters)]
    L.as_p5_site.argtypes = [P, I32, ct.POINTER(P)]
    L.as_p5_coordinator.argtypes = [P, ct.POINTER(P)]
    L.as_p5_destroy.argtypes = [P]
    L.as_sw_create.argtypes = [ct.POINTER(AsConfig), I64, ct.c_double, P, ct.POINTER(P)]
    L.as_sw_update.argtypes = [P, P, I64, I64]
    L.as_sw_query.argtypes = [P, P, I64, ct.POINTER(I32), ct.POINTER(I32)]
    L.as_sw_query_gram.argtypes = [P, P, ct.POINTER(I32)]
    L.as_sw_stats.argtypes = [P, ct.POINTER(AsSwCounters)]
    L.as_sw_level.argtypes = [P, I32, ct.POINTER(P)]
    L.as_sw_destroy.argtypes = [P]
    L.sketch_footprint.argtypes = [ct.POINTER(AsConfig), I64, ct.POINTER(I64)]
    L.sketch_reserve.argtypes = [P, I64]
    L.sketch_update_many.argtypes = [ct.POINTER(P), ct.POINTER(P), ct.POINTER(I64), ct.POINTER(I64), I32]
    L.sketch_update_grouped.argtypes = [ct.POINTER(P), ct.POINTER(P), ct.POINTER(I64), ct.POINTER(I64), I32]
    L.as_server_create.argtypes = [ct.POINTER(AsServerConfig), ct.POINTER(P)]
    L.as_server_open.argtypes = [P, ct.POINTER(AsConfig), ct.c_double, ct.POINTER(I64)]
    L.as_server_submit.argtypes = [P, I64, P, I64, I64, ct.POINTER(I64)]
    L.as_server_wait.argtypes = [P, I64, ct.POINTER(ct.c_double)]
    L.as_server_drain.argtypes = [P]
    L.as_server_session.argtypes = [P, I64, ct.POINTER(P)]
    L.as_server_close.argtypes = [P, I64]
    L.as_server_stats.argtypes = [P, ct.POINTER(AsServerCounters)]
    L.as_server_reset_stats.argtypes = [P]
    L.as_server_destroy.argtypes = [P]
    L.as_wait_selftest.argtypes = [I32, I32, P]
    L.as_status_str.argtypes = [ct.c_int]
    L.as_status_str.restype = ct.c_char_p
    L.as_last_error.argtypes = []
    L.as_last_error.restype = ct.c_char_p
    for name in EXPORTED:
        if name not in ("as_status_str", "as_last_error"):
            getattr(L, name).restype = ct.c_int
    _LIB = L
    return L


def lib() -> ct.CDLL:
    return load_library()


def _check(code: int, what: str) -> None:
    if code != AS_OK:
        raise AeroSketchError(code, what)


def _ptr(x) -> int:
    """Address of a numpy array (host) or a torch tensor (host or device)."""
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return int(x.data_ptr())


class Sketch:
    """One AeroSketch stream on the current CUDA device (the C ABI's as_sketch)."""

    def __init__(self, d: int, ell: int = 0, eps: float = 0.0, *, mode: int = AS_PERSISTENT,
                 prec: int = AS_FP32_PLAIN, theta: float = 0.0, eps_si: float = 0.0, k_pi: int = 0,
                 q_si: int = 0, seed: int = 0, stream_id: int = 0, trace: bool = False, profile: bool = False,
                 delta: float = 0.0, stream=None, dense_query: bool = False):
        L = lib()
        flags = ((AS_TRACE_DECISIONS if trace else 0) | (AS_PROFILE if profile else 0)
                 | (AS_QUERY_DENSE if dense_query else 0))
        cfg = AsConfig(d=d, ell=ell, eps=eps, mode=mode, prec=prec, theta=theta, eps_si=eps_si, k_pi=k_pi,
                       q_si=q_si, seed=seed, stream_id=stream_id, flags=flags, delta=delta)
        h = ct.c_void_p()
        sp = None if stream is None else ct.c_void_p(int(getattr(stream, "cuda_stream", stream)))
        _check(L.sketch_create(ct.byref(cfg), sp, ct.byref(h)), "sketch_create")
        self._h = h
        self.d = d
        self.ell = self.stats()["ell"]

    def close(self) -> None:
        if getattr(self, "_h", None):
            lib().sketch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def reserve(self, snapshot_rank: int) -> None:
        """Allocate the on-demand buffers at their maxima and room for
        `snapshot_rank` more units of snapshot rank (sketch_reserve)."""
        _check(lib().sketch_reserve(self._h, int(snapshot_rank)), "sketch_reserve")

    def update(self, rows, ld: int | None = None) -> None:
        """rows: (n, d) float32 numpy array (host) or torch tensor (host or device)."""
        n = int(rows.shape[0])
        if n == 0:
            _check(lib().sketch_update(self._h, ct.c_void_p(_ptr(rows)), 0, self.d), "sketch_update")
            return
        if ld is None:
            ld = int(rows.strides[0] // 4) if isinstance(rows, np.ndarray) else int(rows.stride(0))
        if isinstance(rows, np.ndarray):
            assert rows.dtype == np.float32 and rows.strides[1] == 4
        _check(lib().sketch_update(self._h, ct.c_void_p(_ptr(rows)), n, ld), "sketch_update")

    def query(self, t: int = -1) -> np.ndarray:
        """Query(t) of Algorithm 8 (t = -1: the current time)."""
        out = np.zeros((self.ell, self.d), dtype=np.float32)
        rows = ct.c_int32()
        _check(lib().sketch_query(self._h, t, ct.c_void_p(out.ctypes.data), self.d, ct.byref(rows)),
               "sketch_query")
        return out[: rows.value]

    def query_gram(self, t: int = -1) -> np.ndarray:
        out = np.zeros((self.d, self.d), dtype=np.float64)
        _check(lib().sketch_query_gram(self._h, t, ct.c_void_p(out.ctypes.data)), "sketch_query_gram")
        return out

    def buffer(self) -> tuple[np.ndarray, int]:
        out = np.zeros((2 * self.ell, self.d), dtype=np.float32)
        r = ct.c_int32()
        _check(lib().sketch_get_buffer(self._h, ct.c_void_p(out.ctypes.data), ct.byref(r)), "sketch_get_buffer")
        return out, r.value

    def gram(self) -> np.ndarray:
        out = np.zeros((2 * self.ell, 2 * self.ell), dtype=np.float64)
        _check(lib().sketch_get_gram(self._h, ct.c_void_p(out.ctypes.data)), "sketch_get_gram")
        return out

    def stats(self) -> dict:
        s = AsStats()
        _check(lib().sketch_stats(self._h, ct.byref(s)), "sketch_stats")
        return s.as_dict()

    def trace(self) -> list[dict]:
        n = ct.c_int64()
        _check(lib().sketch_trace(self._h, None, 0, ct.byref(n)), "sketch_trace")
        arr = (AsEvent * max(1, n.value))()
        _check(lib().sketch_trace(self._h, arr, n.value, ct.byref(n)), "sketch_trace")
        return [{f: getattr(arr[t], f) for f, _ in AsEvent._fields_} for t in range(n.value)]

    def profile(self) -> list[dict]:
        arr = (AsKernelStat * 32)()
        n = ct.c_int32()
        _check(lib().sketch_profile(self._h, arr, 32, ct.byref(n)), "sketch_profile")
        return [{"name": arr[t].name.decode(), "launches": arr[t].launches, "total_ms": arr[t].total_ms,
                 "flops": arr[t].flops, "bytes": arr[t].bytes, "issued_flops": arr[t].issued_flops}
                for t in range(min(n.value, 32))]

    def profile_reset(self) -> None:
        _check(lib().sketch_profile_reset(self._h), "sketch_profile_reset")

    def profile_select(self, names: list[str] | None) -> None:
        """Time only the named kernel classes (None: all of them)."""
        order = [k["name"] for k in self.profile()]
        if names is None:
            mask = 0xFFFFFFFF
        else:
            unknown = [n for n in names if n not in order]
            if unknown:
                raise ValueError(f"unknown kernel classes {unknown}; known: {order}")
            mask = 0
            for n in names:
                mask |= 1 << order.index(n)
        _check(lib().sketch_profile_select(self._h, mask), "sketch_profile_select")

    def merge(self, other: "Sketch") -> None:
        """Absorb other's whole query Gram (decomposability); other is unchanged."""
        _check(lib().sketch_merge(self._h, other._h), "sketch_merge")

    def set_theta(self, theta: float) -> None:
        _check(lib().sketch_set_theta(self._h, float(theta)), "sketch_set_theta")

    def send_snapshots(self, dst: "Sketch") -> int:
        """Move every queued snapshot term into dst's accumulator; returns how many."""
        n = ct.c_int32()
        _check(lib().sketch_send_snapshots(self._h, dst._h, ct.byref(n)), "sketch_send_snapshots")
        return n.value


class _Borrowed(Sketch):
    """A sketch handle owned by someone else (a P5 site or coordinator)."""

    def __init__(self, h, d: int, owner):
        self._h = h
        self.d = d
        self._owner = owner
        self.ell = self.stats()["ell"]

    def close(self) -> None:
        self._h = None


class P5:
    """Algorithm 10: m sites and a coordinator in synchronous rounds (C ABI as_p5)."""

    def __init__(self, d: int, ell: int, m: int, *, eps: float = 0.0, prec: int = AS_FP32_PLAIN,
                 seed: int = 0, stream_id: int = 0, trace: bool = False, stream=None):
        cfg = AsConfig(d=d, ell=ell, eps=eps, mode=AS_SITE, prec=prec, seed=seed, stream_id=stream_id,
                       flags=AS_TRACE_DECISIONS if trace else 0)
        h = ct.c_void_p()
        sp = None if stream is None else ct.c_void_p(int(getattr(stream, "cuda_stream", stream)))
        _check(lib().as_p5_create(ct.byref(cfg), m, sp, ct.byref(h)), "as_p5_create")
        self._h, self.d, self.m = h, d, m

    def close(self) -> None:
        if getattr(self, "_h", None):
            lib().as_p5_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def round(self, blocks) -> None:
        """blocks[j]: site j's rows of this round (numpy FP32 or torch tensors, contiguous)."""
        assert len(blocks) == self.m
        keep = [np.ascontiguousarray(b, dtype=np.float32) if isinstance(b, np.ndarray) else b for b in blocks]
        ptrs = (ct.c_void_p * self.m)(*[_ptr(b) for b in keep])
        ns = (ct.c_int64 * self.m)(*[int(b.shape[0]) for b in keep])
        lds = (ct.c_int64 * self.m)(*[self.d] * self.m)
        _check(lib().as_p5_round(self._h, ptrs, ns, lds), "as_p5_round")

    def query(self) -> np.ndarray:
        out = np.zeros((self.site(0).ell, self.d), dtype=np.float32)
        rows = ct.c_int32()
        _check(lib().as_p5_query(self._h, ct.c_void_p(out.ctypes.data), self.d, ct.byref(rows)), "as_p5_query")
        return out[: rows.value]

    def query_gram(self) -> np.ndarray:
        out = np.zeros((self.d, self.d), dtype=np.float64)
        _check(lib().as_p5_query_gram(self._h, ct.c_void_p(out.ctypes.data)), "as_p5_query_gram")
        return out

    def stats(self) -> dict:
        c = AsP5Counters()
        _check(lib().as_p5_stats(self._h, ct.byref(c)), "as_p5_stats")
        return {f: getattr(c, f) for f, _ in AsP5Counters._fields_}

    def site(self, j: int) -> Sketch:
        h = ct.c_void_p()
        _check(lib().as_p5_site(self._h, j, ct.byref(h)), "as_p5_site")
        return _Borrowed(h, self.d, self)

    def coordinator(self) -> Sketch:
        h = ct.c_void_p()
        _check(lib().as_p5_coordinator(self._h, ct.byref(h)), "as_p5_coordinator")
        return _Borrowed(h, self.d, self)


def symeig(A: np.ndarray, nev: int) -> tuple[np.ndarray, np.ndarray]:
    """The library's FP64 symmetric eigensolver (descending nev pairs)."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    n = A.shape[0]
    lam = np.zeros(nev)
    V = np.zeros((n, nev))
    _check(lib().as_symeig(n, ct.c_void_p(A.ctypes.data), nev, ct.c_void_p(lam.ctypes.data),
                           ct.c_void_p(V.ctypes.data)), "as_symeig")
    return lam, V


def tc_gemm(A: np.ndarray, B: np.ndarray, npass: int = 3, splits: int = 1) -> np.ndarray:
    """A B^T on the tensor cores (tcgen05, BF16 operands, FP32 accumulation)."""
    A = np.ascontiguousarray(A, dtype=np.float32)
    B = np.ascontiguousarray(B, dtype=np.float32)
    out = np.zeros((A.shape[0], B.shape[0]))
    _check(lib().as_tc_gemm(A.shape[0], B.shape[0], A.shape[1], ct.c_void_p(A.ctypes.data), ct.c_void_p(B.ctypes.data),
                            npass, splits, ct.c_void_p(out.ctypes.data)), "as_tc_gemm")
    return out


def replay_from_trace(events: list[dict]) -> dict:
    """Decision record in the oracle's replay format (rows whose gate passed,
    the doubling step and xi of each, and with probability amplification the
    simultaneous iteration kept at each doubling step, keyed ("amp", i, j))."""
    rec = {"fired": {int(e["i"]) for e in events},
           "si": {int(e["i"]): (int(e["j_stop"]), int(e["xi"])) for e in events}}
    for e in events:
        c = int(e.get("amp_choice", 0))
        j = 1
        while c:
            if c & 15:
                rec[("amp", int(e["i"]), j)] = c & 15
            c >>= 4
            j += 1
    return rec


def _row_args(rows) -> tuple[int, int, int]:
    """(pointer, n, ld) of a float32 row block: numpy (host) or torch (host or device)."""
    n = int(rows.shape[0])
    if isinstance(rows, np.ndarray):
        assert rows.dtype == np.float32 and rows.strides[1] == 4
        ld = int(rows.strides[0] // 4) if n > 0 else int(rows.shape[1])
    else:
        ld = int(rows.stride(0))
    return _ptr(rows), n, ld


def footprint(d: int, ell: int = 0, eps: float = 0.0, *, prec: int = AS_FP32_PLAIN, snapshot_rank: int = 0,
              delta: float = 0.0) -> int:
    """Device bytes of a sketch after sketch_reserve(snapshot_rank) (sketch_footprint; host arithmetic)."""
    cfg = AsConfig(d=d, ell=ell, eps=eps, mode=AS_PERSISTENT, prec=prec, delta=delta)
    b = ct.c_int64()
    _check(lib().sketch_footprint(ct.byref(cfg), int(snapshot_rank), ct.byref(b)), "sketch_footprint")
    return b.value


def _many(fn: str, sketches: list, blocks: list) -> None:
    assert len(sketches) == len(blocks)
    k = len(sketches)
    hs = (ct.c_void_p * max(1, k))(*[s._h.value for s in sketches])
    args = [_row_args(b) for b in blocks]
    rp = (ct.c_void_p * max(1, k))(*[a[0] for a in args])
    ns = (ct.c_int64 * max(1, k))(*[a[1] for a in args])
    lds = (ct.c_int64 * max(1, k))(*[a[2] for a in args])
    _check(getattr(lib(), fn)(hs, rp, ns, lds, k), fn)


def update_many(sketches: list, blocks: list) -> None:
    """sketch_update_many: sketch k gets blocks[k]; the sketches progress
    independently on the library's worker threads, each on its own stream."""
    _many("sketch_update_many", sketches, blocks)


def update_grouped(sketches: list, blocks: list) -> None:
    """sketch_update_grouped: the same update, each sketch on its own worker
    thread, with the blocks' batched iterations sharing cooperative launches
    through the launch combiner (bitwise the same results)."""
    _many("sketch_update_grouped", sketches, blocks)


class Server:
    """The serving runtime (C ABI as_server): sessions admitted against an HBM
    budget by their footprint, requests run with continuous batching."""

    def __init__(self, hbm_budget: int = 0, workers: int = 0):
        cfg = AsServerConfig(hbm_budget=int(hbm_budget), workers=int(workers))
        h = ct.c_void_p()
        _check(lib().as_server_create(ct.byref(cfg), ct.byref(h)), "as_server_create")
        self._h = h
        self._keep: dict[int, object] = {}   # rows of pending requests, kept alive until completion
        self._dims: dict[int, int] = {}

    def close(self) -> None:
        if getattr(self, "_h", None):
            lib().as_server_destroy(self._h)
            self._h = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def open(self, d: int, ell: int = 0, eps: float = 0.0, *, mass_ratio: float = 1e6, prec: int = AS_FP32_PLAIN,
             seed: int = 0, stream_id: int = 0, trace: bool = False) -> int:
        """A persistent-mode session; raises AeroSketchError(AS_EBUSY) when the budget refuses it."""
        cfg = AsConfig(d=d, ell=ell, eps=eps, mode=AS_PERSISTENT, prec=prec, seed=seed, stream_id=stream_id,
                       flags=AS_TRACE_DECISIONS if trace else 0)
        sid = ct.c_int64()
        _check(lib().as_server_open(self._h, ct.byref(cfg), float(mass_ratio), ct.byref(sid)), "as_server_open")
        self._dims[sid.value] = d
        return sid.value

    def submit(self, session: int, rows) -> int:
        p, n, ld = _row_args(rows)
        t = ct.c_int64()
        _check(lib().as_server_submit(self._h, int(session), ct.c_void_p(p), n, ld, ct.byref(t)), "as_server_submit")
        self._keep[t.value] = rows
        return t.value

    def wait(self, ticket: int) -> float:
        lat = ct.c_double()
        code = lib().as_server_wait(self._h, int(ticket), ct.byref(lat))
        self._keep.pop(ticket, None)
        _check(code, "as_server_wait")
        return lat.value

    def drain(self) -> None:
        code = lib().as_server_drain(self._h)
        self._keep.clear()
        _check(code, "as_server_drain")

    def sketch(self, session: int) -> "Sketch":
        h = ct.c_void_p()
        _check(lib().as_server_session(self._h, int(session), ct.byref(h)), "as_server_session")
        return _Borrowed(h, self._dims[session], self)

    def close_session(self, session: int) -> None:
        _check(lib().as_server_close(self._h, int(session)), "as_server_close")
        self._dims.pop(session, None)

    def stats(self) -> dict:
        c = AsServerCounters()
        _check(lib().as_server_stats(self._h, ct.byref(c)), "as_server_stats")
        return {f: getattr(c, f) for f, _ in AsServerCounters._fields_}

    def reset_stats(self) -> None:
        _check(lib().as_server_reset_stats(self._h), "as_server_reset_stats")


def default_k_pi(d: int) -> int:
    return int(math.ceil(math.log2(d))) + 1


class SlidingWindow:
    """Algorithm 6: the sketch of the last N rows (C ABI as_sw)."""

    def __init__(self, d: int, ell: int, N: int, R: float, *, eps: float = 0.0, prec: int = AS_FP32_PLAIN,
                 seed: int = 0, stream_id: int = 0, trace: bool = False, stream=None):
        cfg = AsConfig(d=d, ell=ell, eps=eps, mode=AS_FIXED_THETA, prec=prec, seed=seed, stream_id=stream_id,
                       flags=AS_TRACE_DECISIONS if trace else 0)
        h = ct.c_void_p()
        sp = None if stream is None else ct.c_void_p(int(getattr(stream, "cuda_stream", stream)))
        _check(lib().as_sw_create(ct.byref(cfg), int(N), float(R), sp, ct.byref(h)), "as_sw_create")
        self._h, self.d, self.N = h, d, N
        self.ell = self.level(0).ell

    def close(self) -> None:
        if getattr(self, "_h", None):
            lib().as_sw_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def update(self, rows) -> None:
        if isinstance(rows, np.ndarray):
            rows = np.ascontiguousarray(rows, dtype=np.float32)
        _check(lib().as_sw_update(self._h, ct.c_void_p(_ptr(rows)), int(rows.shape[0]), self.d), "as_sw_update")

    def query(self) -> tuple[np.ndarray, int]:
        out = np.zeros((self.ell, self.d), dtype=np.float32)
        rows, lvl = ct.c_int32(), ct.c_int32()
        _check(lib().as_sw_query(self._h, ct.c_void_p(out.ctypes.data), self.d, ct.byref(rows), ct.byref(lvl)),
               "as_sw_query")
        return out[: rows.value], lvl.value

    def query_gram(self) -> tuple[np.ndarray, int]:
        out = np.zeros((self.d, self.d), dtype=np.float64)
        lvl = ct.c_int32()
        _check(lib().as_sw_query_gram(self._h, ct.c_void_p(out.ctypes.data), ct.byref(lvl)), "as_sw_query_gram")
        return out, lvl.value

    def stats(self) -> dict:
        c = AsSwCounters()
        _check(lib().as_sw_stats(self._h, ct.byref(c)), "as_sw_stats")
        return {f: getattr(c, f) for f, _ in AsSwCounters._fields_}

    def level(self, j: int) -> Sketch:
        h = ct.c_void_p()
        _check(lib().as_sw_level(self._h, j, ct.byref(h)), "as_sw_level")
        return _Borrowed(h, self.d, self)
