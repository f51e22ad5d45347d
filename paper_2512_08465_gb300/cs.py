"""Thin Python binding of libcs (argument marshalling only).

Every step of the evaluation runs in the CUDA library; this module converts
arguments (numpy arrays, torch tensors, stream handles) into the plain pointers
and sizes of the C ABI declared in ``include/cs.h``.  Importing it loads
``_lib/libcs.so`` (building it with nvcc if it is missing) and raises if the
library cannot be loaded: there is no CPU fallback.

PyTorch is used only to own device memory and to name CUDA streams.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

_LIB = None

CS_OK, CS_PENDING = 0, 1
CS_E_ARG, CS_E_NOMEM, CS_E_UNKNOWN_ID = -1, -2, -6
ERRORS = {-1: "CS_E_ARG", -2: "CS_E_NOMEM", -3: "CS_E_BASE_INSECURE", -4: "CS_E_TIMEOUT",
          -5: "CS_E_CUDA", -6: "CS_E_UNKNOWN_ID", -7: "CS_E_NUMERIC"}
CLASSES = ("SECURE", "ISLANDED", "OPF_NONCONV", "LIMIT", "SS_UNSTABLE", "SS_POORLY_DAMPED", "EIG_FAIL")
RISK_EQ3, RISK_ORDERED = 0, 1
PREC_FP64, PREC_MIXED = 0, 1

EXPORTS = ("cs_default_options", "cs_create", "cs_destroy", "cs_load_network", "cs_unload_network",
           "cs_base_result", "cs_evaluate_device", "cs_sync", "cs_submit_contingencies", "cs_poll",
           "cs_risk_index", "cs_risk_reduce_device", "cs_enumerate_pairs_device", "cs_last_error",
           "cs_last_launch_count", "cs_set_timing", "cs_kernel_times", "cs_alu_peak", "cs_eigen_reruns",
           "cs_risk_index_static", "cs_network_stats", "cs_serving_stats", "cs_risk_index_batch",
           "cs_evaluate_device_n3", "cs_enumerate_triples_device", "cs_risk_index_pair_freq",
           "cs_symbolic_pattern", "cs_check_network", "cs_tc_gemm_update", "cs_hessenberg_tc")

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int32)


class Options(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int32), ("damping_min", ctypes.c_double), ("opf_tol", ctypes.c_double),
                ("opf_max_it", ctypes.c_int32), ("require_secure_base", ctypes.c_int32),
                ("ctas_per_sm", ctypes.c_int32), ("chunk", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("hbm_budget", ctypes.c_int64), ("serve_slots", ctypes.c_int32), ("batch_cap", ctypes.c_int32),
                ("main_island", ctypes.c_int32), ("autotune", ctypes.c_int32)]


class NetworkDesc(ctypes.Structure):
    _fields_ = [("n_bus", ctypes.c_int32), ("n_branch", ctypes.c_int32), ("n_gen", ctypes.c_int32),
                ("n_levels", ctypes.c_int32), ("ref_bus", ctypes.c_int32),
                ("base_mva", ctypes.c_double), ("f_hz", ctypes.c_double)] + \
               [(k, _dp) for k in ("Vmin", "Vmax", "Gs", "Bs", "Pd", "Qd")] + \
               [("f", _ip), ("t", _ip)] + [(k, _dp) for k in ("r", "x", "b", "rate", "tap")] + \
               [("gbus", _ip)] + [(k, _dp) for k in ("Pmin", "Pmax", "Qmin", "Qmax", "c2", "c1", "c0",
                                                      "H", "D", "xd", "xq", "xdp", "Td0p", "Tq0p", "KA", "TA")] + \
               [("opf_max_it", ctypes.c_int32)]


class Result(ctypes.Structure):
    _fields_ = [("klass", ctypes.c_void_p), ("severe", ctypes.c_void_p), ("n_islands", ctypes.c_void_p),
                ("opf_iters", ctypes.c_void_p), ("cost", ctypes.c_void_p), ("max_re", ctypes.c_void_p),
                ("min_zeta", ctypes.c_void_p), ("Vm", ctypes.c_void_p), ("Va", ctypes.c_void_p),
                ("v_margin", ctypes.c_void_p), ("max_loading", ctypes.c_void_p),
                ("shed_mw", ctypes.c_void_p), ("main_klass", ctypes.c_void_p)]


RESULT_FIELDS = (("klass", np.uint8), ("severe", np.uint8), ("n_islands", np.int16), ("opf_iters", np.int16),
                 ("cost", np.float64), ("max_re", np.float64), ("min_zeta", np.float64))
# optional per-scenario fields, in Result order after Vm / Va; the request path returns them too
EXTRA_FIELDS = (("v_margin", np.float64), ("max_loading", np.float64), ("shed_mw", np.float64),
                ("main_klass", np.uint8))


class CSError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{ERRORS.get(status, status)}: {msg}")
        self.status = status


def _network_desc(net):
    """cs_network_desc of a ``synth.Network``; the arrays it points to are returned
    with it and must stay alive while it is used."""
    arrs = {}

    def d(name, v):
        a = np.ascontiguousarray(v, dtype=np.float64)
        arrs[name] = a
        return a.ctypes.data_as(_dp)

    def i(name, v):
        a = np.ascontiguousarray(v, dtype=np.int32)
        arrs[name] = a
        return a.ctypes.data_as(_ip)

    D = NetworkDesc()
    D.n_bus, D.n_branch, D.n_gen = net.n_bus, net.n_branch, net.n_gen
    D.n_levels, D.ref_bus = len(net.levels), int(net.ref_bus)
    D.base_mva, D.f_hz = float(net.base_mva), float(net.f_hz)
    for k in ("Vmin", "Vmax", "Gs", "Bs"):
        setattr(D, k, d(k, getattr(net, k)))
    D.Pd = d("Pd", np.asarray(net.Pd).reshape(-1))
    D.Qd = d("Qd", np.asarray(net.Qd).reshape(-1))
    D.f = i("f", net.f)
    D.t = i("t", net.t)
    for k in ("r", "x", "b", "rate", "tap"):
        setattr(D, k, d(k, getattr(net, k)))
    D.gbus = i("gbus", net.gbus)
    for k in ("Pmin", "Pmax", "Qmin", "Qmax", "c2", "c1", "c0", "H", "D", "xd", "xq", "xdp", "Td0p",
              "Tq0p", "KA", "TA"):
        setattr(D, k, d(k, getattr(net, k)))
    D.opf_max_it = int(getattr(net, "opf_max_it", 0) or 0)   # optional attribute; 0: the context's cap
    return D, arrs


def check_network(net) -> None:
    """cs_check_network: the descriptor checks of cs_load_network, on the host only.
    Raises CSError (CS_E_ARG) with the library's message for an invalid network."""
    lib = load_library()
    D, arrs = _network_desc(net)
    msg = ctypes.create_string_buffer(256)
    st = lib.cs_check_network(ctypes.byref(D), msg, len(msg))
    if st != 0:
        raise CSError(st, "cs_check_network: " + msg.value.decode())


def lib_path() -> str:
    return _build.LIB


def load_library(build_if_missing: bool = True):
    """Load libcs (compiling it first if needed).  Raises if it cannot be loaded."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = _build.build() if build_if_missing else _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"libcs not found at {path}; run paper_2512_08465_gb300.build.build()")
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    i32, i64, u64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64
    sig = {
        "cs_default_options": (None, [ctypes.POINTER(Options)]),
        "cs_create": (i32, [ctypes.POINTER(Options), ctypes.POINTER(P)]),
        "cs_destroy": (i32, [P]),
        "cs_load_network": (i32, [P, ctypes.POINTER(NetworkDesc), ctypes.POINTER(i32)]),
        "cs_unload_network": (i32, [P, i32]),
        "cs_base_result": (i32, [P, i32, i32, ctypes.POINTER(Result)]),
        "cs_evaluate_device": (i32, [P, i32, i32, P, P, i64, ctypes.POINTER(Result), P]),
        "cs_sync": (i32, [P, P]),
        "cs_submit_contingencies": (i32, [P, i32, i32, P, P, i64, ctypes.POINTER(u64)]),
        "cs_poll": (i32, [P, u64, i32, ctypes.POINTER(Result)]),
        "cs_risk_index": (i32, [P, i32, i32, P, i32, P, ctypes.POINTER(i64)]),
        "cs_risk_index_static": (i32, [P, i32, i32, P, i32, P, ctypes.POINTER(i64)]),
        "cs_network_stats": (i32, [P, i32, P, i32]),
        "cs_symbolic_pattern": (i32, [i32, i32, P, P, i32, P, P, P, i64, P, P]),
        "cs_check_network": (i32, [ctypes.POINTER(NetworkDesc), ctypes.c_char_p, i32]),
        "cs_tc_gemm_update": (i32, [P, i32, i32, i32, i32, P, i64, i64, P, i64, i64, P, i64, i64, ctypes.c_float, P]),
        "cs_hessenberg_tc": (i32, [P, i32, i32, P, i64, P]),
        "cs_serving_stats": (i32, [P, P, i32]),
        "cs_risk_index_batch": (i32, [P, i32, i32, P, i64, i32, P, P]),
        "cs_evaluate_device_n3": (i32, [P, i32, i32, P, P, P, i64, ctypes.POINTER(Result), P]),
        "cs_enumerate_triples_device": (i32, [i32, i64, i64, P, P, P, P]),
        "cs_risk_index_pair_freq": (i32, [P, i32, i32, P, P, i32, P, ctypes.POINTER(i64)]),
        "cs_risk_reduce_device": (i32, [i32, P, P, P, i32, P, P]),
        "cs_enumerate_pairs_device": (i32, [i32, i64, i64, P, P, P]),
        "cs_last_error": (ctypes.c_char_p, [P]),
        "cs_last_launch_count": (i64, [P]),
        "cs_set_timing": (i32, [P, i32]),
        "cs_kernel_times": (i32, [P, P, P]),
        "cs_alu_peak": (i32, [i32, P, P]),
        "cs_eigen_reruns": (i32, [P, ctypes.POINTER(i64)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


def _ptr(x):
    """Data pointer of a torch tensor or numpy array (None -> NULL)."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return ctypes.c_void_p(x.data_ptr())
    return ctypes.c_void_p(x.ctypes.data)


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def default_options(**kw) -> Options:
    """cs_default_options with the given fields overridden; an unknown field name raises."""
    o = Options()
    load_library().cs_default_options(ctypes.byref(o))
    names = {f for f, _ in Options._fields_}
    for k, v in kw.items():
        if k not in names:
            raise TypeError(f"unknown cs_options field {k!r} (known: {', '.join(sorted(names))})")
        setattr(o, k, v)
    return o


class Context:
    """One libcs context on one CUDA device."""

    def __init__(self, **options):
        self.lib = load_library()
        self.opt = default_options(**options)
        h = ctypes.c_void_p()
        st = self.lib.cs_create(ctypes.byref(self.opt), ctypes.byref(h))
        if st != CS_OK:
            raise CSError(st, "cs_create failed (no usable CUDA device?)")
        self.h = h
        self._keep = {}

    def close(self):
        if getattr(self, "h", None):
            self.lib.cs_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st, what):
        if st < 0:
            raise CSError(st, f"{what}: {self.lib.cs_last_error(self.h).decode()}")
        return st

    # -------------------------------------------------------------- networks --
    def load_network(self, net) -> int:
        """Copy a ``synth.Network`` (or any object with the same fields) to the device."""
        D, arrs = _network_desc(net)
        nid = ctypes.c_int32()
        self._check(self.lib.cs_load_network(self.h, ctypes.byref(D), ctypes.byref(nid)), "cs_load_network")
        return nid.value

    def unload_network(self, net_id: int):
        self._check(self.lib.cs_unload_network(self.h, net_id), "cs_unload_network")

    def base_result(self, net_id: int, level: int) -> dict:
        out = {k: np.zeros(1, dt) for k, dt in RESULT_FIELDS}
        R = Result(*[_ptr(out[k]) for k, _ in RESULT_FIELDS], None, None, None, None)
        self._check(self.lib.cs_base_result(self.h, net_id, level, ctypes.byref(R)), "cs_base_result")
        return {k: v[0] for k, v in out.items()}

    # ------------------------------------------------------------ evaluation --
    @staticmethod
    def alloc_results(n: int, device="cuda", n_bus: int = 0, indices: bool = False, main_island: bool = False):
        """Result tensors for n records (torch, on ``device``); Vm/Va if n_bus > 0; the
        non-binary severity indices (v_margin, max_loading) if indices; the main-island
        fields (shed_mw, main_klass) if main_island."""
        import torch
        tmap = {np.uint8: torch.uint8, np.int16: torch.int16, np.float64: torch.float64}
        out = {k: torch.empty(n, dtype=tmap[dt], device=device) for k, dt in RESULT_FIELDS}
        if n_bus:
            out["Vm"] = torch.empty(n * n_bus, dtype=torch.float64, device=device)
            out["Va"] = torch.empty(n * n_bus, dtype=torch.float64, device=device)
        if indices:
            out["v_margin"] = torch.empty(n, dtype=torch.float64, device=device)
            out["max_loading"] = torch.empty(n, dtype=torch.float64, device=device)
        if main_island:
            out["shed_mw"] = torch.empty(n, dtype=torch.float64, device=device)
            out["main_klass"] = torch.empty(n, dtype=torch.uint8, device=device)
        return out

    @staticmethod
    def _result_struct(out):
        return Result(*[_ptr(out[k]) for k, _ in RESULT_FIELDS], _ptr(out.get("Vm")), _ptr(out.get("Va")),
                      _ptr(out.get("v_margin")), _ptr(out.get("max_loading")),
                      _ptr(out.get("shed_mw")), _ptr(out.get("main_klass")))

    def evaluate_device(self, net_id: int, level: int, ei, ej, out: dict, stream=None):
        """Asynchronous evaluation of len(ei) scenarios with device tensors."""
        n = int(ei.numel())
        R = self._result_struct(out)
        st = self.lib.cs_evaluate_device(self.h, net_id, level, _ptr(ei), _ptr(ej), n, ctypes.byref(R),
                                         _stream_handle(stream))
        self._check(st, "cs_evaluate_device")

    def evaluate_device_n3(self, net_id: int, level: int, ei, ej, ek, out: dict, stream=None):
        """N-3 extension: like evaluate_device with a third element per scenario (-1 = none)."""
        n = int(ei.numel())
        R = self._result_struct(out)
        st = self.lib.cs_evaluate_device_n3(self.h, net_id, level, _ptr(ei), _ptr(ej), _ptr(ek), n,
                                            ctypes.byref(R), _stream_handle(stream))
        self._check(st, "cs_evaluate_device_n3")

    def sync(self, stream=None):
        self._check(self.lib.cs_sync(self.h, _stream_handle(stream)), "cs_sync")

    def last_launch_count(self) -> int:
        return int(self.lib.cs_last_launch_count(self.h))

    def eigen_reruns(self) -> int:
        c = ctypes.c_int64()
        self._check(self.lib.cs_eigen_reruns(self.h, ctypes.byref(c)), "cs_eigen_reruns")
        return c.value

    def set_timing(self, enable: bool = True):
        self._check(self.lib.cs_set_timing(self.h, int(enable)), "cs_set_timing")

    def kernel_times(self):
        """(ms per kernel, launches per kernel) for islanding, OPF, small-signal."""
        ms = np.zeros(3)
        cnt = np.zeros(3, np.int64)
        self._check(self.lib.cs_kernel_times(self.h, _ptr(ms), _ptr(cnt)), "cs_kernel_times")
        return dict(zip(("islands", "opf", "dyn"), ms.tolist())), dict(zip(("islands", "opf", "dyn"), cnt.tolist()))

    def submit(self, net_id: int, level: int, ei, ej) -> int:
        """Non-blocking submission with host arrays; returns a request id."""
        ei = np.ascontiguousarray(ei, dtype=np.int32)
        ej = np.ascontiguousarray(ej, dtype=np.int32)
        rid = ctypes.c_uint64()
        st = self.lib.cs_submit_contingencies(self.h, net_id, level, _ptr(ei), _ptr(ej), ei.size,
                                              ctypes.byref(rid))
        self._check(st, "cs_submit_contingencies")
        self._keep[rid.value] = ei.size
        return rid.value

    def poll(self, request_id: int, timeout_us: int = 0, out: dict | None = None):
        """Results of a finished request as numpy arrays (every per-scenario field: the
        seven record fields, the severity indices and the main-island fields), or None
        while pending."""
        n = self._keep.get(request_id, 0)
        if out is None:
            out = {k: np.empty(n, dt) for k, dt in RESULT_FIELDS + EXTRA_FIELDS}
        R = Result(*[_ptr(out[k]) for k, _ in RESULT_FIELDS], None, None,
                   *[_ptr(out.get(k)) for k, _ in EXTRA_FIELDS])
        st = self.lib.cs_poll(self.h, request_id, int(timeout_us), ctypes.byref(R))
        if st == CS_PENDING:
            return None
        self._check(st, "cs_poll")
        self._keep.pop(request_id, None)
        return out

    def evaluate(self, net_id: int, level: int, ei, ej, timeout_us: int = 600_000_000):
        """Blocking convenience: submit host arrays and wait for the results."""
        rid = self.submit(net_id, level, ei, ej)
        out = self.poll(rid, timeout_us)
        if out is None:
            raise CSError(-4, "request did not finish in time")
        return out

    def serving_stats(self) -> dict:
        """Counters of the serving path (cs_serving_stats)."""
        v = np.zeros(9, np.int64)
        self._check(self.lib.cs_serving_stats(self.h, _ptr(v), 9), "cs_serving_stats")
        keys = ("batches", "completed", "merged", "admission_waits", "nomem", "peak_bytes", "bytes_now",
                "queued", "in_flight")
        return dict(zip(keys, (int(x) for x in v)))

    def network_stats(self, net_id: int) -> dict:
        """Sizes of a loaded network and its symbolic analysis (cs_network_stats)."""
        v = np.zeros(12, np.int64)
        self._check(self.lib.cs_network_stats(self.h, net_id, _ptr(v), 12), "cs_network_stats")
        keys = ("n_bus", "n_branch", "n_gen", "l_blocks", "block_updates", "levels", "states_max", "levels_load",
                "opf_ctas_per_sm", "dyn_ctas_per_sm", "autotuned", "opf_max_it")
        return dict(zip(keys, (int(x) for x in v)))

    # ------------------------------------------------------------ Risk Index --
    def risk_index(self, net_id: int, level: int, lam, mode: int = RISK_ORDERED):
        lam = np.ascontiguousarray(lam, dtype=np.float64)
        R = np.empty_like(lam)
        miss = ctypes.c_int64()
        st = self.lib.cs_risk_index(self.h, net_id, level, _ptr(lam), mode, _ptr(R), ctypes.byref(miss))
        self._check(st, "cs_risk_index")
        return R, miss.value

    def risk_index_pair_freq(self, net_id: int, level: int, lam, F, mode: int = RISK_ORDERED):
        """cs_risk_index_pair_freq: Eq. 3 with explicit pair frequencies F (E x E, host)."""
        lam = np.ascontiguousarray(lam, dtype=np.float64)
        F = np.ascontiguousarray(F, dtype=np.float64)
        R = np.empty_like(lam)
        miss = ctypes.c_int64()
        st = self.lib.cs_risk_index_pair_freq(self.h, net_id, level, _ptr(lam), _ptr(F), mode, _ptr(R),
                                              ctypes.byref(miss))
        self._check(st, "cs_risk_index_pair_freq")
        return R, miss.value

    def risk_index_batch(self, net_id: int, level: int, lam, R, mode: int = RISK_ORDERED, stream=None):
        """cs_risk_index_batch: R[s, i] for device rate samples lam[s, i] (float64, sample-major)."""
        st = self.lib.cs_risk_index_batch(self.h, net_id, level, _ptr(lam), lam.shape[0], mode, _ptr(R),
                                          _stream_handle(stream))
        self._check(st, "cs_risk_index_batch")

    def hessenberg_tc(self, A, stream=None):
        """cs_hessenberg_tc: reduce a float32 device tensor of shape (n, n) or (batch, n, n)
        (contiguous) to upper Hessenberg form in place."""
        a3 = A if A.dim() == 3 else A.unsqueeze(0)
        if A.dtype.itemsize != 4 or not a3.is_contiguous() or a3.shape[1] != a3.shape[2]:
            raise ValueError("hessenberg_tc wants contiguous square float32 matrices")
        b, n, _ = a3.shape
        self._check(self.lib.cs_hessenberg_tc(self.h, b, n, _ptr(a3), n * n, _stream_handle(stream)),
                    "cs_hessenberg_tc")

    def risk_index_static(self, net_id: int, level: int, lam, mode: int = RISK_ORDERED):
        """cs_risk_index_static: the same reduction with its device scratch in a
        static array (no device allocation; at most 4096 outage elements)."""
        lam = np.ascontiguousarray(lam, dtype=np.float64)
        R = np.empty_like(lam)
        miss = ctypes.c_int64()
        st = self.lib.cs_risk_index_static(self.h, net_id, level, _ptr(lam), mode, _ptr(R), ctypes.byref(miss))
        self._check(st, "cs_risk_index_static")
        return R, miss.value


def tc_gemm_update(A, B, C, alpha: float = 1.0, ctx=None, stream=None):
    """cs_tc_gemm_update: C[b] += alpha A[b] @ B[b] on the tensor cores (float32 torch
    tensors on the device, 2-D or a batch of 3-D, each matrix row-major contiguous)."""
    lib = load_library()
    a3, b3, c3 = (x if x.dim() == 3 else x.unsqueeze(0) for x in (A, B, C))
    batch, M, K = a3.shape
    N = b3.shape[2]
    for x in (a3, b3, c3):
        if x.dtype.itemsize != 4 or not x.is_contiguous():
            raise ValueError("tc_gemm_update wants contiguous float32 tensors")
    if b3.shape[:2] != (batch, K) or c3.shape != (batch, M, N):
        raise ValueError("shape mismatch")
    st = lib.cs_tc_gemm_update(ctx.h if ctx is not None else None, batch, M, N, K, _ptr(a3), K, M * K, _ptr(b3), N,
                               K * N, _ptr(c3), N, M * N, float(alpha), _stream_handle(stream))
    if st != CS_OK:
        raise CSError(st, "cs_tc_gemm_update")


def risk_reduce_device(n_elem: int, S1, S2, lam, R, mode: int = RISK_ORDERED, stream=None):
    st = load_library().cs_risk_reduce_device(n_elem, _ptr(S1), _ptr(S2), _ptr(lam), mode, _ptr(R),
                                              _stream_handle(stream))
    if st != CS_OK:
        raise CSError(st, "cs_risk_reduce_device")


def alu_peak(device: int = 0):
    """Measured (fp64, fp32) FMA-pipe peaks in TFLOP/s."""
    a, b = ctypes.c_double(), ctypes.c_double()
    st = load_library().cs_alu_peak(device, ctypes.byref(a), ctypes.byref(b))
    if st != CS_OK:
        raise CSError(st, "cs_alu_peak")
    return a.value, b.value


def enumerate_triples_device(n_elem: int, first: int, count: int, ei, ej, ek, stream=None):
    st = load_library().cs_enumerate_triples_device(n_elem, first, count, _ptr(ei), _ptr(ej), _ptr(ek),
                                                    _stream_handle(stream))
    if st != CS_OK:
        raise CSError(st, "cs_enumerate_triples_device")


def enumerate_pairs_device(n_elem: int, first: int, count: int, ei, ej, stream=None):
    st = load_library().cs_enumerate_pairs_device(n_elem, first, count, _ptr(ei), _ptr(ej),
                                                  _stream_handle(stream))
    if st != CS_OK:
        raise CSError(st, "cs_enumerate_pairs_device")


def symbolic_pattern(n_bus: int, f, t, ref_bus: int = -1) -> dict:
    """cs_symbolic_pattern on host arrays (no device): the elimination order
    (perm[new] = old bus), the CSC pattern of L's off-diagonal blocks (col_ptr, row),
    the elimination-tree height of each column (level) and the counts (blocks,
    levels, block updates)."""
    lib = load_library()
    f = np.ascontiguousarray(f, dtype=np.int32)
    t = np.ascontiguousarray(t, dtype=np.int32)
    stats = np.zeros(4, np.int64)
    st = lib.cs_symbolic_pattern(int(n_bus), int(f.size), _ptr(f), _ptr(t), int(ref_bus),
                                 None, None, None, 0, None, _ptr(stats))
    if st != CS_OK:
        raise CSError(st, "cs_symbolic_pattern")
    perm = np.zeros(n_bus, np.int32)
    col_ptr = np.zeros(n_bus + 1, np.int32)
    row = np.zeros(max(1, int(stats[3])), np.int32)
    level = np.zeros(n_bus, np.int32)
    st = lib.cs_symbolic_pattern(int(n_bus), int(f.size), _ptr(f), _ptr(t), int(ref_bus),
                                 _ptr(perm), _ptr(col_ptr), _ptr(row), int(row.size), _ptr(level), _ptr(stats))
    if st != CS_OK:
        raise CSError(st, "cs_symbolic_pattern")
    return dict(perm=perm, col_ptr=col_ptr, row=row[:int(stats[3])], level=level,
                blocks=int(stats[0]), levels=int(stats[1]), updates=int(stats[2]))
