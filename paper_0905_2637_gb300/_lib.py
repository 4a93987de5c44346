"""ctypes binding of ``libpetfmm.so`` (argument marshalling only).

The functions named ``petfmm_*`` mirror the C ABI of ``include/petfmm.h``
one to one; ``Context`` and ``Server`` wrap them for use with torch tensors.
Every step of the evaluation runs in the library's CUDA kernels: there is no
Python or CPU fallback, and a missing library raises ``ImportError``.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# PETFMM_CHECKED=1 loads the bounds-checked build (libpetfmm_checked.so)
LIB_PATH = os.path.join(HERE, "libpetfmm_checked.so" if os.environ.get("PETFMM_CHECKED") == "1"
                        else "libpetfmm.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "petfmm.h")

PETFMM_OK, PETFMM_EINVAL, PETFMM_ENOMEM, PETFMM_EDOMAIN = 0, -1, -2, -3
PETFMM_ECUDA, PETFMM_ETIMEOUT, PETFMM_EBUSY, PETFMM_ENOTREADY = -4, -5, -6, -7
PETFMM_FP64, PETFMM_MIXED = 0, 1
PETFMM_F64, PETFMM_F32 = 0, 1
PETFMM_OPT_TIMING, PETFMM_OPT_SPIN_LIMIT, PETFMM_OPT_P2P_MODE, PETFMM_OPT_POISON = 1, 2, 3, 4
PETFMM_OPT_M2L_TC, PETFMM_OPT_TC_DENSE, PETFMM_OPT_TC_SEG, PETFMM_OPT_NEAR_TOL = 5, 6, 8, 9
PETFMM_OPT_GRAPH, PETFMM_OPT_P2P_PAIRS, PETFMM_OPT_KERNEL, PETFMM_OPT_TC_BLOCKS = 10, 11, 12, 13
PETFMM_OPT_TC_PIPE, PETFMM_OPT_OVERLAP = 14, 15
PETFMM_KERNEL_VORTEX, PETFMM_KERNEL_LAPLACE = 0, 1
PETFMM_NOALLOC_MAX_N = 1048576
STAGES = ("morton", "sort", "gather", "p2m", "m2m", "m2l", "l2l", "worklist", "pairs", "p2p",
          "final")


class Domain(ctypes.Structure):
    _fields_ = [("x0", ctypes.c_double), ("y0", ctypes.c_double), ("width", ctypes.c_double)]


class Instance(ctypes.Structure):
    _fields_ = [("domain", Domain), ("levels", ctypes.c_int), ("order", ctypes.c_int),
                ("sigma", ctypes.c_double), ("n", ctypes.c_int64),
                ("x", ctypes.c_void_p), ("y", ctypes.c_void_p), ("gamma", ctypes.c_void_p),
                ("u", ctypes.c_void_p), ("v", ctypes.c_void_p)]


class Request(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("x", ctypes.c_void_p), ("y", ctypes.c_void_p),
                ("gamma", ctypes.c_void_p), ("levels", ctypes.c_int), ("order", ctypes.c_int),
                ("sigma", ctypes.c_double), ("dt", ctypes.c_double), ("n_steps", ctypes.c_int),
                ("precision", ctypes.c_int)]


class Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("latency_ms", ctypes.c_double),
                ("queue_ms", ctypes.c_double), ("n", ctypes.c_int64),
                ("x", ctypes.POINTER(ctypes.c_double)), ("y", ctypes.POINTER(ctypes.c_double)),
                ("rounds", ctypes.c_int32), ("max_shared", ctypes.c_int32)]


class ServeStats(ctypes.Structure):
    _fields_ = [("rounds", ctypes.c_uint64), ("submitted", ctypes.c_uint64),
                ("admitted", ctypes.c_uint64), ("completed", ctypes.c_uint64),
                ("queued", ctypes.c_int32), ("max_active", ctypes.c_int32),
                ("mean_active", ctypes.c_double), ("busy_ms", ctypes.c_double),
                ("up_ms", ctypes.c_double), ("admit_ms", ctypes.c_double),
                ("launch_ms", ctypes.c_double), ("wait_ms", ctypes.c_double),
                ("post_ms", ctypes.c_double), ("gpu_ms", ctypes.c_double)]


class Stats(ctypes.Structure):
    _fields_ = [("kernel_launches", ctypes.c_uint64), ("evaluations", ctypes.c_uint64),
                ("p2p_pairs", ctypes.c_int64), ("m2l_pairs", ctypes.c_int64),
                ("p2p_items", ctypes.c_int64), ("p2p_load_balance", ctypes.c_float),
                ("p2p_pair_items", ctypes.c_int64), ("p2p_split_entries", ctypes.c_int64),
                ("p2p_sym_pairs", ctypes.c_int64), ("pairs_load_balance", ctypes.c_float),
                ("occupied_leaves", ctypes.c_int64)]


class LevelRule(ctypes.Structure):
    _fields_ = [("order", ctypes.c_int32), ("log2n", ctypes.c_int32), ("levels", ctypes.c_int32),
                ("ms", ctypes.c_float)]


class TuneReport(ctypes.Structure):
    _fields_ = [("tc_blocks", ctypes.c_int), ("tc_dense_pct", ctypes.c_int),
                ("nrules", ctypes.c_int), ("changed", ctypes.c_int),
                ("evaluations", ctypes.c_int), ("ms_model", ctypes.c_float),
                ("ms_tuned", ctypes.c_float)]


class PetfmmError(RuntimeError):
    def __init__(self, code, what=""):
        self.code = code
        super().__init__(f"{what}: {_strerror(code)} ({code})" if what else _strerror(code))


_lock = threading.Lock()
_lib = None


def _strerror(code):
    try:
        return load().petfmm_strerror(code).decode()
    except Exception:  # pragma: no cover - only when the library is absent
        return str(code)


def header_symbols():
    """Names of the functions the public header declares."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(petfmm(?:3d)?_[a-z_0-9]+)\s*\(", text)))


def load():
    """Load the CUDA library (build it first with ``build.build()``)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: run paper_0905_2637_gb300.build.build() "
                              "(needs nvcc); there is no CPU fallback")
        lib = ctypes.CDLL(LIB_PATH)
        P, I, I64, D, SZ = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_size_t
        PP = ctypes.POINTER(ctypes.c_void_p)
        sig = {
            "petfmm_create": (I, [ctypes.POINTER(Domain), I, I, D, I, I, P, PP]),
            "petfmm_evaluate": (I, [P, I64, P, P, P, P, P]),
            "petfmm_evaluate_host": (I, [P, I64, P, P, P, P, P]),
            "petfmm_sync": (I, [P]),
            "petfmm_destroy": (I, [P]),
            "petfmm_evaluate_batch": (I, [P, I, ctypes.POINTER(Instance)]),
            "petfmm_choose_levels": (I, [I64, I, D, ctypes.POINTER(Domain)]),
            "petfmm_serve_create": (I, [SZ, I, I, PP]),
            "petfmm_serve_submit": (I, [P, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_uint64)]),
            "petfmm_serve_poll": (I, [P, ctypes.c_uint64, ctypes.POINTER(Result)]),
            "petfmm_serve_release": (I, [P, ctypes.c_uint64]),
            "petfmm_serve_destroy": (I, [P]),
            "petfmm_serve_estimate_bytes": (SZ, [I64, I, I, I]),
            "petfmm_serve_stats": (I, [P, ctypes.POINTER(ServeStats)]),
            "petfmm_serve_trace": (I, [P, P, P, P, I]),
            "petfmm_debug_tree": (I, [P, P, P, P]),
            "petfmm_debug_expansions": (I, [P, I, I, P]),
            "petfmm_debug_interaction_list": (I, [I, I, I, P]),
            "petfmm_debug_m2l_images": (I, [I, I, I, P, ctypes.c_int64]),
            "petfmm_debug_op_table": (I, [I, I, I, P, ctypes.c_int64]),
            "petfmm_debug_near_fit": (I, [ctypes.c_double, ctypes.c_double, ctypes.c_double, P]),
            "petfmm_debug_plan": (I, [I, I, ctypes.POINTER(Instance), P, I]),
            "petfmm_set_option": (I, [P, I, I64]),
            "petfmm_stage_times": (I, [P, P, I]),
            "petfmm_get_stats": (I, [P, ctypes.POINTER(Stats)]),
            "petfmm_strerror": (ctypes.c_char_p, [I]),
            "petfmm_version": (I, []),
            "petfmm_measure_peaks": (I, [ctypes.POINTER(Peaks)]),
            "petfmm_tree_noalloc": (I, [ctypes.POINTER(Domain), I, I, I64, P, P, P, P, P, P]),
            "petfmm_debug_checks": (I, [P]),
            "petfmm_rule_levels": (I, [ctypes.POINTER(LevelRule), I, I64, I, D,
                                       ctypes.POINTER(Domain)]),
            "petfmm_set_level_rules": (I, [P, ctypes.POINTER(LevelRule), I]),
            "petfmm_tune_batch": (I, [P, I, ctypes.POINTER(Instance), I,
                                      ctypes.POINTER(LevelRule), I, ctypes.POINTER(TuneReport)]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


# --------------------------------------------------------------------------- C-ABI mirror

def _ck(rc, what):
    if rc < 0:
        raise PetfmmError(rc, what)
    return rc


def petfmm_create(domain, levels, order, sigma, precision, dtype, cuda_stream):
    h = ctypes.c_void_p()
    dom = Domain(*map(float, domain))
    _ck(load().petfmm_create(ctypes.byref(dom), int(levels), int(order), float(sigma),
                             int(precision), int(dtype), cuda_stream, ctypes.byref(h)),
        "petfmm_create")
    return h


def petfmm_evaluate(ctx, n, x, y, gamma, u, v):
    return _ck(load().petfmm_evaluate(ctx, int(n), x, y, gamma, u, v), "petfmm_evaluate")


def petfmm_evaluate_host(ctx, n, x, y, gamma, u, v):
    return _ck(load().petfmm_evaluate_host(ctx, int(n), x, y, gamma, u, v), "petfmm_evaluate_host")


def petfmm_sync(ctx):
    return _ck(load().petfmm_sync(ctx), "petfmm_sync")


def petfmm_destroy(ctx):
    return _ck(load().petfmm_destroy(ctx), "petfmm_destroy")


def petfmm_choose_levels(n, order, sigma, domain):
    dom = Domain(*map(float, domain))
    return _ck(load().petfmm_choose_levels(int(n), int(order), float(sigma), ctypes.byref(dom)),
               "petfmm_choose_levels")


def _rules_array(rules):
    arr = (LevelRule * max(1, len(rules)))()
    for i, r in enumerate(rules):
        arr[i] = LevelRule(int(r["order"]), int(r["log2n"]), int(r["levels"]),
                           float(r.get("ms", 0.0)))
    return arr


def petfmm_rule_levels(rules, n, order, sigma, domain):
    """Automatic L of one problem under level rules (list of dicts with order,
    log2n, levels); host only."""
    dom = Domain(*map(float, domain))
    return _ck(load().petfmm_rule_levels(_rules_array(rules), len(rules), int(n), int(order),
                                         float(sigma), ctypes.byref(dom)), "petfmm_rule_levels")


def petfmm_debug_near_fit(sigma, wleaf, tol):
    """The near-field polynomial fit: dict(deg, general, kappa, split_rho2, coef)."""
    out = np.zeros(4 + 15, np.float64)
    _ck(load().petfmm_debug_near_fit(float(sigma), float(wleaf), float(tol), out.ctypes.data),
        "petfmm_debug_near_fit")
    return dict(deg=int(out[0]), general=int(out[1]), kappa=float(out[2]),
                split_rho2=float(out[3]), coef=out[4:].copy())


def petfmm_debug_op_table(order, kernel=0, which=0):
    """FP64 M2M (which 0), L2L (1) or M2L (2) operators as a complex array
    [4 or 40][p][p] (layout in petfmm.h)."""
    n = _ck(load().petfmm_debug_op_table(int(order), int(kernel), int(which), None, 0),
            "petfmm_debug_op_table")
    out = np.zeros(n, np.float64)
    _ck(load().petfmm_debug_op_table(int(order), int(kernel), int(which), out.ctypes.data, n),
        "petfmm_debug_op_table")
    return out.view(np.complex128).reshape(-1, int(order), int(order))


def petfmm_debug_m2l_images(order, kernel=0, blocks=0):
    """The tensor-core M2L operator images (float32 array; layout in petfmm.h)."""
    n = _ck(load().petfmm_debug_m2l_images(int(order), int(kernel), int(blocks), None, 0),
            "petfmm_debug_m2l_images")
    out = np.zeros(n, np.float32)
    _ck(load().petfmm_debug_m2l_images(int(order), int(kernel), int(blocks), out.ctypes.data, n),
        "petfmm_debug_m2l_images")
    return out


def petfmm_debug_interaction_list(level, ix, iy):
    out = np.zeros(2 * 27, np.int32)
    cnt = _ck(load().petfmm_debug_interaction_list(int(level), int(ix), int(iy), out.ctypes.data),
              "petfmm_debug_interaction_list")
    return out[: 2 * cnt].reshape(cnt, 2).copy()


def petfmm_debug_plan(precision, instances):
    """Host-side launch plan: list of (range, inst, level, units, block0)."""
    arr = (Instance * max(1, len(instances)))()
    for i, it in enumerate(instances):
        arr[i] = Instance(Domain(*map(float, it["domain"])), int(it.get("levels", 0)),
                          int(it["order"]), float(it["sigma"]), int(it["n"]), 8, 8, 8, 8, 8)
    n = _ck(load().petfmm_debug_plan(int(precision), len(instances), arr, None, 0), "petfmm_debug_plan")
    out = np.zeros((max(n, 1), 5), np.int64)
    _ck(load().petfmm_debug_plan(int(precision), len(instances), arr, out.ctypes.data, n),
        "petfmm_debug_plan")
    return out[:n]


def petfmm_serve_estimate_bytes(n, levels, order, precision):
    return int(load().petfmm_serve_estimate_bytes(int(n), int(levels), int(order), int(precision)))


def petfmm_strerror(code):
    return load().petfmm_strerror(int(code)).decode()


def petfmm_version():
    return int(load().petfmm_version())


class Peaks(ctypes.Structure):
    _fields_ = [("fp32_ops", ctypes.c_double), ("fp64_ops", ctypes.c_double),
                ("mufu_rcp_ops", ctypes.c_double), ("mufu_ex2_ops", ctypes.c_double),
                ("tf32_flops", ctypes.c_double), ("sms", ctypes.c_int)]


def petfmm_measure_peaks():
    """Measured pipe rates of the current device (petfmm_measure_peaks)."""
    pk = Peaks()
    _ck(load().petfmm_measure_peaks(ctypes.byref(pk)), "petfmm_measure_peaks")
    return {f: getattr(pk, f) for f, _ in Peaks._fields_}


# --------------------------------------------------------------------------- torch wrappers

def _torch():
    import torch
    return torch


def _dev_ptr(t, dtype, n, name):
    torch = _torch()
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype or not t.is_contiguous() or t.numel() != n:
        raise TypeError(f"{name} must be a contiguous {dtype} tensor of {n} elements")
    return t.data_ptr()


class Context:
    """One FMM configuration bound to a CUDA stream (``petfmm_create``)."""

    def __init__(self, domain, levels, order, sigma, precision="mixed", dtype="f32", stream=None,
                 kernel="vortex"):
        torch = _torch()
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required (no CPU fallback)")
        self.precision = {"fp64": PETFMM_FP64, "mixed": PETFMM_MIXED}[precision]
        self.dtype_code = {"f64": PETFMM_F64, "f32": PETFMM_F32}[dtype]
        self.torch_dtype = torch.float32 if dtype == "f32" else torch.float64
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.domain, self.levels, self.order, self.sigma = tuple(domain), levels, order, sigma
        self.handle = petfmm_create(domain, levels, order, sigma, self.precision, self.dtype_code,
                                    ctypes.c_void_p(self.stream.cuda_stream))
        if kernel != "vortex":
            self.set_option(PETFMM_OPT_KERNEL,
                            {"laplace": PETFMM_KERNEL_LAPLACE}[kernel])

    def close(self):
        if self.handle is not None:
            petfmm_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def evaluate(self, x, y, gamma, u=None, v=None):
        """Enqueue one evaluation; returns (u, v).  Call ``sync()`` before use."""
        torch = _torch()
        n = x.numel()
        if u is None:
            u = torch.empty(n, dtype=self.torch_dtype, device=x.device)
        if v is None:
            v = torch.empty(n, dtype=self.torch_dtype, device=x.device)
        ptrs = [_dev_ptr(t, self.torch_dtype, n, nm) for t, nm in
                ((x, "x"), (y, "y"), (gamma, "gamma"), (u, "u"), (v, "v"))]
        petfmm_evaluate(self.handle, n, *ptrs)
        return u, v

    def evaluate_host(self, x, y, gamma):
        """Host arrays in, host arrays out (copies inside the call)."""
        npd = np.float32 if self.dtype_code == PETFMM_F32 else np.float64
        x, y, g = (np.ascontiguousarray(a, dtype=npd) for a in (x, y, gamma))
        u, v = np.empty_like(x), np.empty_like(x)
        petfmm_evaluate_host(self.handle, x.size, x.ctypes.data, y.ctypes.data, g.ctypes.data,
                             u.ctypes.data, v.ctypes.data)
        return u, v

    def evaluate_host_ptrs(self, n, x, y, gamma, u, v):
        return petfmm_evaluate_host(self.handle, n, x, y, gamma, u, v)

    def sync(self):
        return petfmm_sync(self.handle)

    def set_option(self, option, value):
        _ck(load().petfmm_set_option(self.handle, int(option), int(value)), "petfmm_set_option")

    def stage_times(self):
        ms = (ctypes.c_float * len(STAGES))()
        rc = load().petfmm_stage_times(self.handle, ctypes.cast(ms, ctypes.c_void_p), len(STAGES))
        _ck(rc, "petfmm_stage_times")
        return {s: float(ms[i]) for i, s in enumerate(STAGES)}

    def stats(self):
        st = Stats()
        _ck(load().petfmm_get_stats(self.handle, ctypes.byref(st)), "petfmm_get_stats")
        return {f: getattr(st, f) for f, _ in Stats._fields_}

    def debug_tree(self, n):
        keys = np.zeros(n, np.uint32)
        perm = np.zeros(n, np.uint32)
        start = np.zeros((1 << (2 * self.levels)) + 1, np.uint32)
        _ck(load().petfmm_debug_tree(self.handle, keys.ctypes.data, perm.ctypes.data, start.ctypes.data),
            "petfmm_debug_tree")
        return keys, perm, start

    def debug_expansions(self, level, which):
        out = np.zeros((1 << (2 * level)) * self.order * 2, np.float64)
        _ck(load().petfmm_debug_expansions(self.handle, int(level), int(which), out.ctypes.data),
            "petfmm_debug_expansions")
        return out.view(np.complex128).reshape(1 << (2 * level), self.order)

    def _instances(self, instances):
        arr = (Instance * max(1, len(instances)))()
        for i, it in enumerate(instances):
            n = it["x"].numel()
            ptrs = [_dev_ptr(it[k], self.torch_dtype, n, k) for k in ("x", "y", "gamma", "u", "v")]
            arr[i] = Instance(Domain(*map(float, it["domain"])), int(it.get("levels", 0)),
                              int(it["order"]), float(it["sigma"]), n, *ptrs)
        return arr

    def evaluate_batch(self, instances):
        """instances: list of dicts with domain, levels (<= 0: automatic), order,
        sigma, x, y, gamma, u, v (CUDA tensors of the context's dtype)."""
        _ck(load().petfmm_evaluate_batch(self.handle, len(instances), self._instances(instances)),
            "petfmm_evaluate_batch")

    def set_level_rules(self, rules):
        """Install level rules (list of dicts with order, log2n, levels)."""
        _ck(load().petfmm_set_level_rules(self.handle, _rules_array(rules), len(rules)),
            "petfmm_set_level_rules")

    def tune_batch(self, instances, reps=3):
        """Run the autotuner on a batch (petfmm_tune_batch); returns (rules,
        report) as a list of dicts and a dict.  The context keeps the result."""
        cap = 4 * max(1, len(instances))
        out = (LevelRule * cap)()
        rep = TuneReport()
        _ck(load().petfmm_tune_batch(self.handle, len(instances), self._instances(instances),
                                     int(reps), out, cap, ctypes.byref(rep)), "petfmm_tune_batch")
        rules = [dict(order=out[i].order, log2n=out[i].log2n, levels=out[i].levels, ms=out[i].ms)
                 for i in range(rep.nrules)]
        return rules, {f: getattr(rep, f) for f, _ in TuneReport._fields_}


class Server:
    """Request loop with continuous batching (``petfmm_serve_*``)."""

    def __init__(self, hbm_budget_bytes, max_slots=64, max_queue=4096):
        h = ctypes.c_void_p()
        _ck(load().petfmm_serve_create(int(hbm_budget_bytes), int(max_slots), int(max_queue),
                                       ctypes.byref(h)), "petfmm_serve_create")
        self.handle = h

    def submit(self, x, y, gamma, sigma, order, dt, n_steps, levels=0, precision="mixed"):
        x, y, g = (np.ascontiguousarray(a, dtype=np.float64) for a in (x, y, gamma))
        req = Request(x.size, x.ctypes.data, y.ctypes.data, g.ctypes.data, int(levels), int(order),
                      float(sigma), float(dt), int(n_steps),
                      {"fp64": PETFMM_FP64, "mixed": PETFMM_MIXED}[precision])
        t = ctypes.c_uint64()
        _ck(load().petfmm_serve_submit(self.handle, ctypes.byref(req), ctypes.byref(t)),
            "petfmm_serve_submit")
        return int(t.value)

    def poll(self, ticket, positions=True):
        """None while running; else dict(status, latency_ms, queue_ms, rounds,
        max_shared and, with positions, x, y); the result is then released."""
        r = Result()
        rc = load().petfmm_serve_poll(self.handle, ctypes.c_uint64(ticket), ctypes.byref(r))
        if rc == PETFMM_ENOTREADY:
            return None
        _ck(rc, "petfmm_serve_poll")
        out = {"status": r.status, "latency_ms": r.latency_ms, "queue_ms": r.queue_ms,
               "rounds": r.rounds, "max_shared": r.max_shared}
        if positions and r.status == PETFMM_OK and r.n > 0:
            out["x"] = np.ctypeslib.as_array(r.x, shape=(r.n,)).copy()
            out["y"] = np.ctypeslib.as_array(r.y, shape=(r.n,)).copy()
        load().petfmm_serve_release(self.handle, ctypes.c_uint64(ticket))
        return out

    def stats(self):
        st = ServeStats()
        _ck(load().petfmm_serve_stats(self.handle, ctypes.byref(st)), "petfmm_serve_stats")
        return {f: getattr(st, f) for f, _ in ServeStats._fields_}

    def trace(self):
        """Per round: (start ms since creation, queued, resident) arrays."""
        n = _ck(load().petfmm_serve_trace(self.handle, None, None, None, 0), "petfmm_serve_trace")
        t = np.zeros(max(n, 1), np.float64)
        q = np.zeros(max(n, 1), np.int32)
        a = np.zeros(max(n, 1), np.int32)
        n = _ck(load().petfmm_serve_trace(self.handle, t.ctypes.data, q.ctypes.data, a.ctypes.data,
                                          n), "petfmm_serve_trace")
        return t[:n], q[:n], a[:n]

    def close(self):
        if self.handle is not None:
            _ck(load().petfmm_serve_destroy(self.handle), "petfmm_serve_destroy")
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
