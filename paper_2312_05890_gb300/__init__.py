"""Python binding of libslrcount, the GB300 exact #DNN-Verification counter.

The functions below carry the names of the C ABI in ``include/slrcount.h`` and
only marshal arguments (numpy arrays or CUDA tensors in, numbers out); every
step of the computation runs in the library's CUDA kernels.  ``Counter`` wraps
one context for convenience.  There is no CPU fallback: when the shared library
has not been built, or no GPU is present, the calls raise.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libslrcount.so")

SLR_OK = 0
SLR_EINVAL = -1
STATUS = {0: "SLR_OK", -1: "SLR_EINVAL", -2: "SLR_ENOMEM", -3: "SLR_ECUDA", -4: "SLR_ESTATE",
          -5: "SLR_EOVERFLOW", -6: "SLR_ETIMEOUT", -7: "SLR_EUNSUPPORTED"}
SAFE, UNSAFE, UNDECIDED = 0, 1, 2
RELAX_NEURIFY, RELAX_PAPER_LITERAL, RELAX_INTERVAL = 0, 1, 2
PREC_FP32 = 0
PREC_TC_TF32 = 1
SPLIT_WIDEST = 0
SPLIT_GRADIENT = 1
SPLIT_PATH_BITS = 16     # SPLIT_GRADIENT codes: path below, one 4-bit split-set position per level above
MAX_LEVELS = 63

# Names the header declares (checked by the CPU test that loads the library).
EXPORTS = ("slr_create", "slr_destroy", "slr_default_options", "slr_set_options", "slr_load_network",
           "slr_set_activations",
           "slr_set_box", "slr_set_property", "slr_count", "slr_bounds", "slr_leaves", "slr_schedule",
           "slr_split_set", "slr_wait_selfcheck", "slr_count_noalloc", "slr_count_batch", "slr_alpha_width", "slr_margin_backward",
           "slr_optimize_alpha", "slr_count_checkpoint", "slr_count_resume", "slr_measure_fp32_peak",
           "slr_default_approx_options", "slr_count_approx",
           "slr_last_error")


class SlrError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class slr_options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("relax_mode", ctypes.c_int32),
                ("fp64_recheck", ctypes.c_int32), ("record_leaves", ctypes.c_int32),
                ("profile", ctypes.c_int32), ("split_rule", ctypes.c_int32),
                ("frontier_cap", ctypes.c_int64), ("leaf_cap", ctypes.c_int64),
                ("alpha_steps", ctypes.c_int32), ("alpha_lr", ctypes.c_float), ("alpha_cap", ctypes.c_int64),
                ("tile_boxes", ctypes.c_int32), ("tile_threads", ctypes.c_int32),
                ("wide", ctypes.c_int32), ("shard_count", ctypes.c_int32), ("shard_index", ctypes.c_int32),
                ("shard_level", ctypes.c_int32), ("recheck_cluster", ctypes.c_int32),
                ("alpha_margin", ctypes.c_float), ("recheck_pairs", ctypes.c_int32)]


_U64A = ctypes.c_uint64 * (MAX_LEVELS + 1)


class slr_result(ctypes.Structure):
    _fields_ = [("unsafe_lo", ctypes.c_uint64), ("unsafe_hi", ctypes.c_uint64), ("boxes", ctypes.c_uint64),
                ("rechecked", ctypes.c_uint64), ("tie_leaves", ctypes.c_uint64), ("depth", ctypes.c_int32),
                ("levels", ctypes.c_int32), ("level_boxes", _U64A), ("level_safe", _U64A),
                ("level_unsafe", _U64A), ("level_undecided", _U64A), ("device_ms", ctypes.c_double),
                ("kernel_ms", ctypes.c_double * 3), ("launches", ctypes.c_int64),
                ("h2d_bytes", ctypes.c_int64), ("d2h_bytes", ctypes.c_int64),
                ("tile_boxes", ctypes.c_int32), ("tile_threads", ctypes.c_int32),
                ("rechecked_fp32", ctypes.c_uint64), ("alpha_boxes", ctypes.c_uint64),
                ("alpha_decided", ctypes.c_uint64), ("alpha_ms", ctypes.c_double),
                ("gemm_ms", ctypes.c_double), ("gemm_launches", ctypes.c_int64), ("gemm_flop", ctypes.c_double),
                ("completion_ms", ctypes.c_double), ("rechecked_fp64", ctypes.c_uint64)]

    def to_dict(self):
        n = self.depth + 1
        return dict(unsafe_lo=int(self.unsafe_lo), unsafe_hi=int(self.unsafe_hi), boxes=int(self.boxes),
                    rechecked=int(self.rechecked), tie_leaves=int(self.tie_leaves), depth=int(self.depth),
                    levels=int(self.levels), device_ms=float(self.device_ms),
                    kernel_ms=[float(x) for x in self.kernel_ms], launches=int(self.launches),
                    h2d_bytes=int(self.h2d_bytes), d2h_bytes=int(self.d2h_bytes),
                    tile=(int(self.tile_boxes), int(self.tile_threads)),
                    rechecked_fp32=int(self.rechecked_fp32), alpha_boxes=int(self.alpha_boxes),
                    alpha_decided=int(self.alpha_decided), alpha_ms=float(self.alpha_ms),
                    gemm_ms=float(self.gemm_ms), gemm_launches=int(self.gemm_launches),
                    gemm_flop=float(self.gemm_flop), completion_ms=float(self.completion_ms),
                    rechecked_fp64=int(self.rechecked_fp64),
                    level_boxes=list(self.level_boxes[:n]), level_safe=list(self.level_safe[:n]),
                    level_unsafe=list(self.level_unsafe[:n]), level_undecided=list(self.level_undecided[:n]))


APPROX_MAX_TRIALS = 64
_AT = APPROX_MAX_TRIALS


class slr_approx_options(ctypes.Structure):
    _fields_ = [("trials", ctypes.c_int32), ("splits", ctypes.c_int32), ("samples", ctypes.c_int32),
                ("leaf_depth", ctypes.c_int32), ("beta", ctypes.c_double), ("seed", ctypes.c_uint64)]


class slr_approx_result(ctypes.Structure):
    _fields_ = [("vr_lower", ctypes.c_double), ("confidence", ctypes.c_double), ("vr_mean", ctypes.c_double),
                ("trials", ctypes.c_int32), ("splits_done", ctypes.c_int32 * _AT),
                ("leaf_unsafe_lo", ctypes.c_uint64 * _AT), ("leaf_unsafe_hi", ctypes.c_uint64 * _AT),
                ("leaf_volume", ctypes.c_double * _AT), ("estimate", ctypes.c_double * _AT),
                ("estimate_hi", ctypes.c_double * _AT), ("boxes", ctypes.c_uint64),
                ("samples_unsafe", ctypes.c_uint64), ("device_ms", ctypes.c_double)]

    def to_dict(self):
        n = int(self.trials)
        return dict(vr_lower=float(self.vr_lower), confidence=float(self.confidence), vr_mean=float(self.vr_mean),
                    trials=n, splits_done=list(self.splits_done[:n]), leaf_unsafe_lo=list(self.leaf_unsafe_lo[:n]),
                    leaf_unsafe_hi=list(self.leaf_unsafe_hi[:n]), leaf_volume=list(self.leaf_volume[:n]),
                    estimate=list(self.estimate[:n]), estimate_hi=list(self.estimate_hi[:n]),
                    boxes=int(self.boxes), samples_unsafe=int(self.samples_unsafe),
                    device_ms=float(self.device_ms))


class slr_problem(ctypes.Structure):
    _fields_ = [("K", ctypes.c_int32), ("widths", ctypes.c_void_p), ("W", ctypes.c_void_p), ("b", ctypes.c_void_p),
                ("lo", ctypes.c_void_p), ("hi", ctypes.c_void_p), ("n_clauses", ctypes.c_int32),
                ("rows_per_clause", ctypes.c_void_p), ("C", ctypes.c_void_p), ("e", ctypes.c_void_p),
                ("strict", ctypes.c_void_p), ("depth", ctypes.c_int32)]


_lib_handle = None


def load_library(path: str = LIB_PATH):
    """Load the shared library (raises if it has not been built)."""
    global _lib_handle
    if _lib_handle is not None:
        return _lib_handle
    if not os.path.exists(path):
        raise RuntimeError(f"libslrcount.so not built at {path}; run paper_2312_05890_gb300.build.build()")
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    i32, i64 = ctypes.c_int32, ctypes.c_int64
    sig = {
        "slr_create": (ctypes.c_int, [ctypes.POINTER(P), ctypes.c_int, P]),
        "slr_destroy": (ctypes.c_int, [P]),
        "slr_default_options": (None, [ctypes.POINTER(slr_options)]),
        "slr_set_options": (ctypes.c_int, [P, ctypes.POINTER(slr_options)]),
        "slr_load_network": (ctypes.c_int, [P, ctypes.c_int, P, P, P]),
        "slr_set_box": (ctypes.c_int, [P, ctypes.c_int, P, P]),
        "slr_set_activations": (ctypes.c_int, [P, ctypes.c_int, P]),
        "slr_set_property": (ctypes.c_int, [P, ctypes.c_int, P, ctypes.c_int, P, P, P]),
        "slr_count": (ctypes.c_int, [P, ctypes.c_int, ctypes.POINTER(slr_result)]),
        "slr_bounds": (ctypes.c_int, [P, i64, P, P, P, P, P, P, P, ctypes.c_int]),
        "slr_alpha_width": (ctypes.c_int, [P, ctypes.POINTER(i64)]),
        "slr_margin_backward": (ctypes.c_int, [P, i64, P, P, P, P, P, P, P, P, P, P, P, P, ctypes.c_int]),
        "slr_optimize_alpha": (ctypes.c_int, [P, i64, P, P, ctypes.c_int, ctypes.c_float, P, P, P, P,
                                              ctypes.c_int]),
        "slr_leaves": (ctypes.c_int, [P, i64, P, P, P, ctypes.POINTER(i64)]),
        "slr_schedule": (ctypes.c_int, [P, ctypes.c_int, P]),
        "slr_split_set": (ctypes.c_int, [P, P, ctypes.POINTER(i32)]),
        "slr_wait_selfcheck": (ctypes.c_int, [P, ctypes.c_int32]),
        "slr_count_noalloc": (ctypes.c_int, [P, ctypes.c_int, ctypes.POINTER(slr_result)]),
        "slr_count_batch": (ctypes.c_int, [P, ctypes.c_int, ctypes.POINTER(slr_problem), ctypes.POINTER(slr_result)]),
        "slr_count_checkpoint": (ctypes.c_int, [P, ctypes.c_int, ctypes.c_int, P, ctypes.c_size_t,
                                                ctypes.POINTER(ctypes.c_size_t)]),
        "slr_count_resume": (ctypes.c_int, [P, ctypes.c_char_p, ctypes.c_size_t, ctypes.POINTER(slr_result)]),
        "slr_measure_fp32_peak": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                                 ctypes.POINTER(ctypes.c_double)]),
        "slr_default_approx_options": (None, [ctypes.POINTER(slr_approx_options)]),
        "slr_count_approx": (ctypes.c_int, [P, ctypes.POINTER(slr_approx_options), ctypes.POINTER(slr_approx_result),
                                            P, P]),
        "slr_last_error": (ctypes.c_char_p, [P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _ = i32
    _lib_handle = lib
    return lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _check(lib, ctx, rc):
    if rc != SLR_OK:
        raise SlrError(rc, lib.slr_last_error(ctx).decode())


# ---------------------------------------------------------------------------
# functions named as in the C ABI
# ---------------------------------------------------------------------------

def slr_create(device: int = 0, stream: int | None = None):
    lib = load_library()
    ctx = ctypes.c_void_p()
    _check(lib, None, lib.slr_create(ctypes.byref(ctx), device, stream))
    return ctx


def slr_destroy(ctx):
    lib = load_library()
    _check(lib, ctx, lib.slr_destroy(ctx))


def slr_default_options() -> slr_options:
    o = slr_options()
    load_library().slr_default_options(ctypes.byref(o))
    return o


def slr_set_options(ctx, opt: slr_options):
    lib = load_library()
    _check(lib, ctx, lib.slr_set_options(ctx, ctypes.byref(opt)))


def slr_load_network(ctx, W, b):
    lib = load_library()
    Ws = [np.ascontiguousarray(w, dtype=np.float32) for w in W]
    bs = [np.ascontiguousarray(x, dtype=np.float32).reshape(-1) for x in b]
    K = len(Ws)
    widths = np.array([Ws[0].shape[1]] + [w.shape[0] for w in Ws], dtype=np.int32)
    wp = (ctypes.c_void_p * K)(*[w.ctypes.data for w in Ws])
    bp = (ctypes.c_void_p * K)(*[x.ctypes.data for x in bs])
    _check(lib, ctx, lib.slr_load_network(ctx, K, _ptr(widths), wp, bp))


ACTIVATIONS = {"relu": 0, "tanh": 1, "sigmoid": 2}


def slr_set_activations(ctx, act):
    """Activation of each hidden layer ('relu', 'tanh', 'sigmoid' or the SLR_ACT_* numbers)."""
    lib = load_library()
    a = np.ascontiguousarray([ACTIVATIONS.get(x, x) for x in act], dtype=np.int32)
    _check(lib, ctx, lib.slr_set_activations(ctx, int(a.shape[0]), _ptr(a) if a.size else None))


def slr_set_box(ctx, lo, hi):
    lib = load_library()
    lo = np.ascontiguousarray(lo, dtype=np.float32)
    hi = np.ascontiguousarray(hi, dtype=np.float32)
    _check(lib, ctx, lib.slr_set_box(ctx, int(lo.shape[0]), _ptr(lo), _ptr(hi)))


def slr_set_property(ctx, rows_per_clause, C, e, strict):
    lib = load_library()
    rpc = np.ascontiguousarray(rows_per_clause, dtype=np.int32)
    C = np.ascontiguousarray(C, dtype=np.float32)
    e = np.ascontiguousarray(e, dtype=np.float32)
    st = np.ascontiguousarray(strict, dtype=np.uint8)
    _check(lib, ctx, lib.slr_set_property(ctx, int(rpc.shape[0]), _ptr(rpc), int(C.shape[1]), _ptr(C), _ptr(e), _ptr(st)))


def slr_count(ctx, D: int) -> dict:
    lib = load_library()
    res = slr_result()
    rc = lib.slr_count(ctx, int(D), ctypes.byref(res))
    _check(lib, ctx, rc)
    return res.to_dict()


class _Buffers:
    """Inputs and outputs of one call, all on the host (numpy) or all on the device (CUDA tensors)."""

    def __init__(self, like):
        self.device = hasattr(like, "data_ptr")
        self.keep = []

    def inp(self, a, dtype=np.float32):
        if a is None:
            return None
        if self.device:
            import torch
            t = a.detach().to(dtype=torch.float32 if dtype == np.float32 else torch.uint8).contiguous()
            self.keep.append(t)
            return ctypes.c_void_p(t.data_ptr())
        x = np.ascontiguousarray(a, dtype=dtype)
        self.keep.append(x)
        return _ptr(x)

    def out(self, shape, dtype=np.float32, like=None):
        if self.device:
            import torch
            return torch.empty(shape, dtype=torch.float32 if dtype == np.float32 else torch.uint8, device=like.device)
        return np.empty(shape, dtype=dtype)

    @staticmethod
    def ptr(a):
        if a is None:
            return None
        return ctypes.c_void_p(a.data_ptr()) if hasattr(a, "data_ptr") else _ptr(a)


def slr_bounds(ctx, box_lo, box_hi, R: int, want_rows=True, want_cls=True, want_err=False, alpha=None):
    """Bounds of n boxes: (row_lo, row_hi, cls) or, with want_err, (row_lo, row_hi, cls, row_err).

    numpy inputs use host memory; CUDA tensors (with .data_ptr) stay on the device.
    alpha (n x H, optional) gives the lower ReLU slopes.
    """
    lib = load_library()
    io = _Buffers(box_lo)
    n = int(box_lo.shape[0])
    lo, hi, al = io.inp(box_lo), io.inp(box_hi), io.inp(alpha)
    rl = io.out((n, R), like=box_lo) if want_rows else None
    rh = io.out((n, R), like=box_lo) if want_rows else None
    re_ = io.out((n, R), like=box_lo) if want_err else None
    cl = io.out((n,), np.uint8, like=box_lo) if want_cls else None
    q = io.ptr
    _check(lib, ctx, lib.slr_bounds(ctx, n, lo, hi, al, q(rl), q(rh), q(re_), q(cl), 1 if io.device else 0))
    return (rl, rh, cl, re_) if want_err else (rl, rh, cl)


def slr_alpha_width(ctx) -> int:
    lib = load_library()
    h = ctypes.c_int64()
    _check(lib, ctx, lib.slr_alpha_width(ctx, ctypes.byref(h)))
    return int(h.value)


def slr_margin_backward(ctx, box_lo, box_hi, R: int, g_lo, g_hi, alpha=None, widths=None, want_rows=True,
                        want_alpha=True, want_box=True):
    """Gradients of J = sum(g_lo * lo + g_hi * hi) over the float32 SLR row bounds of n boxes.

    Returns a dict with 'row_lo', 'row_hi' (n x R), 'd_alpha' (n x H), 'd_lo', 'd_hi' (n x d) and,
    when `widths` (the network's widths[0..K]) is given, 'd_W' and 'd_b' (lists over layers).
    """
    lib = load_library()
    io = _Buffers(box_lo)
    n, d = int(box_lo.shape[0]), int(box_lo.shape[1])
    H = slr_alpha_width(ctx)
    lo, hi, al = io.inp(box_lo), io.inp(box_hi), io.inp(alpha)
    gl, gh = io.inp(g_lo), io.inp(g_hi)
    out = {}
    out["row_lo"] = io.out((n, R), like=box_lo) if want_rows else None
    out["row_hi"] = io.out((n, R), like=box_lo) if want_rows else None
    out["d_alpha"] = io.out((n, H), like=box_lo) if want_alpha else None
    out["d_lo"] = io.out((n, d), like=box_lo) if want_box else None
    out["d_hi"] = io.out((n, d), like=box_lo) if want_box else None
    wp = bp = None
    if widths is not None:
        K = len(widths) - 1
        out["d_W"] = [io.out((int(widths[k + 1]), int(widths[k])), like=box_lo) for k in range(K)]
        out["d_b"] = [io.out((int(widths[k + 1]),), like=box_lo) for k in range(K)]
        wp = (ctypes.c_void_p * K)(*[io.ptr(x).value for x in out["d_W"]])
        bp = (ctypes.c_void_p * K)(*[io.ptr(x).value for x in out["d_b"]])
    q = io.ptr
    _check(lib, ctx, lib.slr_margin_backward(ctx, n, lo, hi, al, gl, gh, q(out["row_lo"]), q(out["row_hi"]),
                                             q(out["d_alpha"]), q(out["d_lo"]), q(out["d_hi"]),
                                             ctypes.cast(wp, ctypes.c_void_p) if wp is not None else None,
                                             ctypes.cast(bp, ctypes.c_void_p) if bp is not None else None,
                                             1 if io.device else 0))
    return out


def slr_optimize_alpha(ctx, box_lo, box_hi, R: int, steps: int = 20, lr: float = 0.1, want_alpha=True):
    """Projected-Adam steps on the lower slopes: (row_lo, row_hi, cls, alpha) with sound, intersected bounds."""
    lib = load_library()
    io = _Buffers(box_lo)
    n = int(box_lo.shape[0])
    H = slr_alpha_width(ctx)
    lo, hi = io.inp(box_lo), io.inp(box_hi)
    rl = io.out((n, R), like=box_lo)
    rh = io.out((n, R), like=box_lo)
    cl = io.out((n,), np.uint8, like=box_lo)
    al = io.out((n, H), like=box_lo) if want_alpha else None
    q = io.ptr
    _check(lib, ctx, lib.slr_optimize_alpha(ctx, n, lo, hi, int(steps), float(lr), q(al), q(rl), q(rh), q(cl),
                                            1 if io.device else 0))
    return rl, rh, cl, al


def slr_leaves(ctx, cap: int):
    lib = load_library()
    codes = np.empty(cap, dtype=np.uint64)
    depth = np.empty(cap, dtype=np.uint8)
    cls = np.empty(cap, dtype=np.uint8)
    n = ctypes.c_int64()
    _check(lib, ctx, lib.slr_leaves(ctx, cap, _ptr(codes), _ptr(depth), _ptr(cls), ctypes.byref(n)))
    m = min(cap, n.value)
    return codes[:m], depth[:m], cls[:m]


def slr_schedule(ctx, D: int):
    lib = load_library()
    out = np.empty(D, dtype=np.int32)
    _check(lib, ctx, lib.slr_schedule(ctx, D, _ptr(out)))
    return out


def slr_split_set(ctx):
    lib = load_library()
    out = np.empty(16, dtype=np.int32)
    n = ctypes.c_int32()
    _check(lib, ctx, lib.slr_split_set(ctx, _ptr(out), ctypes.byref(n)))
    return out[:n.value].copy()


def slr_wait_selfcheck(ctx, limit: int = 4096):
    """A bounded device wait on a barrier nothing completes; raises SlrError (SLR_ETIMEOUT)."""
    lib = load_library()
    _check(lib, ctx, lib.slr_wait_selfcheck(ctx, int(limit)))


def split_code_dims(code: int, depth: int, split_set):
    """(path, dims) of a SPLIT_GRADIENT code: the halves taken (bit depth-1-j for
    split j) and the input dimension of each split."""
    code = int(code)
    path = code & ((1 << SPLIT_PATH_BITS) - 1)
    dims = [int(split_set[(code >> (SPLIT_PATH_BITS + 4 * j)) & 15]) for j in range(depth)]
    return path, dims


def slr_count_noalloc(ctx, D: int) -> dict:
    """slr_count without any GPU allocation (fixed scratch inside the library; see the header)."""
    lib = load_library()
    res = slr_result()
    _check(lib, ctx, lib.slr_count_noalloc(ctx, int(D), ctypes.byref(res)))
    return res.to_dict()


def slr_count_approx(ctx, d: int, **kw) -> dict:
    """CountingProVe_SLR (see the header): the lower bound of the violation rate with its
    confidence, per-trial splits, leaf counts, volumes and estimates, and each trial's leaf box."""
    lib = load_library()
    o = slr_approx_options()
    lib.slr_default_approx_options(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    res = slr_approx_result()
    n = max(1, int(o.trials))
    llo = np.zeros((n, d), dtype=np.float32)
    lhi = np.zeros((n, d), dtype=np.float32)
    _check(lib, ctx, lib.slr_count_approx(ctx, ctypes.byref(o), ctypes.byref(res), _ptr(llo), _ptr(lhi)))
    out = res.to_dict()
    out["leaf_lo"], out["leaf_hi"] = llo, lhi
    return out


def slr_measure_fp32_peak(device: int = 0, iters: int = 1 << 19) -> dict:
    """FP32 FMA rate of the device in TFLOP/s, measured by the library's FFMA kernel."""
    lib = load_library()
    tf = ctypes.c_double(0.0)
    ms = ctypes.c_double(0.0)
    rc = lib.slr_measure_fp32_peak(int(device), int(iters), ctypes.byref(tf), ctypes.byref(ms))
    if rc != SLR_OK:
        raise SlrError(rc, "slr_measure_fp32_peak failed")
    return {"tflops": tf.value, "ms": ms.value, "iters": int(iters)}


def slr_count_checkpoint(ctx, D: int, t: int, size_hint: int = 1 << 22) -> bytes:
    """Levels 0..t of a count to depth D; returns the state to resume from (see the header)."""
    lib = load_library()
    used = ctypes.c_size_t(0)
    buf = ctypes.create_string_buffer(size_hint)
    rc = lib.slr_count_checkpoint(ctx, int(D), int(t), ctypes.cast(buf, ctypes.c_void_p), size_hint, ctypes.byref(used))
    if rc == SLR_EINVAL and used.value > size_hint:
        buf = ctypes.create_string_buffer(used.value)
        rc = lib.slr_count_checkpoint(ctx, int(D), int(t), ctypes.cast(buf, ctypes.c_void_p), used.value,
                                      ctypes.byref(used))
    _check(lib, ctx, rc)
    return buf.raw[:used.value]


def slr_count_resume(ctx, state: bytes) -> dict:
    """Finish a count from a checkpoint; the result covers the whole count."""
    lib = load_library()
    res = slr_result()
    _check(lib, ctx, lib.slr_count_resume(ctx, bytes(state), len(state), ctypes.byref(res)))
    return res.to_dict()


def slr_count_batch(ctx, problems, depths=None):
    """Count many workloads.Problem-like objects together; returns one result dict per problem."""
    lib = load_library()
    keep = []
    arr = (slr_problem * len(problems))()
    for i, p in enumerate(problems):
        Ws = [np.ascontiguousarray(w, dtype=np.float32) for w in p.net.W]
        bs = [np.ascontiguousarray(x, dtype=np.float32).reshape(-1) for x in p.net.b]
        widths = np.array([Ws[0].shape[1]] + [w.shape[0] for w in Ws], dtype=np.int32)
        wp = (ctypes.c_void_p * len(Ws))(*[w.ctypes.data for w in Ws])
        bp = (ctypes.c_void_p * len(bs))(*[x.ctypes.data for x in bs])
        lo = np.ascontiguousarray(p.lo, dtype=np.float32)
        hi = np.ascontiguousarray(p.hi, dtype=np.float32)
        rpc = np.ascontiguousarray(p.prop.rows_per_clause, dtype=np.int32)
        C = np.ascontiguousarray(p.prop.C, dtype=np.float32)
        e = np.ascontiguousarray(p.prop.e, dtype=np.float32)
        st = np.ascontiguousarray(p.prop.strict, dtype=np.uint8)
        keep += [Ws, bs, widths, wp, bp, lo, hi, rpc, C, e, st]
        D = p.depth if depths is None else depths[i]
        arr[i] = slr_problem(len(Ws), widths.ctypes.data, ctypes.cast(wp, ctypes.c_void_p),
                             ctypes.cast(bp, ctypes.c_void_p), lo.ctypes.data, hi.ctypes.data, int(rpc.shape[0]),
                             rpc.ctypes.data, C.ctypes.data, e.ctypes.data, st.ctypes.data, int(D))
    res = (slr_result * len(problems))()
    _check(lib, ctx, lib.slr_count_batch(ctx, len(problems), arr, res))
    return [r.to_dict() for r in res]


def slr_last_error(ctx) -> str:
    return load_library().slr_last_error(ctx).decode()


# ---------------------------------------------------------------------------
# convenience wrapper
# ---------------------------------------------------------------------------

class Counter:
    """One counting context on one GPU: network, box, property, options."""

    def __init__(self, device: int = 0, stream: int | None = None):
        self.ctx = slr_create(device, stream)
        self.R = None

    def close(self):
        if self.ctx is not None:
            slr_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass

    def load_network(self, W, b):
        slr_load_network(self.ctx, W, b)
        self.widths = [int(np.asarray(W[0]).shape[1])] + [int(np.asarray(w).shape[0]) for w in W]

    def set_box(self, lo, hi):
        slr_set_box(self.ctx, lo, hi)

    def set_property(self, rows_per_clause, C, e, strict):
        slr_set_property(self.ctx, rows_per_clause, C, e, strict)
        self.R = int(np.asarray(e).shape[0])

    def set_problem(self, problem):
        """Load a workloads.Problem (network, box and property)."""
        self.load_network(problem.net.W, problem.net.b)
        act = list(getattr(problem.net, "act", None) or [])
        if act:
            slr_set_activations(self.ctx, act)
        self.set_box(problem.lo, problem.hi)
        p = problem.prop
        self.set_property(p.rows_per_clause, p.C, p.e, p.strict)

    def set_options(self, **kw):
        o = slr_default_options()
        for k, v in kw.items():
            setattr(o, k, v)
        slr_set_options(self.ctx, o)

    def count(self, D: int) -> dict:
        return slr_count(self.ctx, D)

    def count_batch(self, problems, depths=None):
        return slr_count_batch(self.ctx, problems, depths)

    def count_approx(self, **kw) -> dict:
        return slr_count_approx(self.ctx, self.widths[0], **kw)

    def count_noalloc(self, D: int) -> dict:
        return slr_count_noalloc(self.ctx, D)

    def checkpoint(self, D: int, t: int) -> bytes:
        return slr_count_checkpoint(self.ctx, D, t)

    def resume(self, state: bytes) -> dict:
        return slr_count_resume(self.ctx, state)

    def bounds(self, lo, hi, want_rows=True, want_cls=True, want_err=False, alpha=None):
        return slr_bounds(self.ctx, lo, hi, self.R, want_rows, want_cls, want_err, alpha)

    def alpha_width(self) -> int:
        return slr_alpha_width(self.ctx)

    def margin_backward(self, lo, hi, g_lo, g_hi, alpha=None, weights=False, **kw):
        return slr_margin_backward(self.ctx, lo, hi, self.R, g_lo, g_hi, alpha,
                                   self.widths if weights else None, **kw)

    def optimize_alpha(self, lo, hi, steps: int = 20, lr: float = 0.1, want_alpha=True):
        return slr_optimize_alpha(self.ctx, lo, hi, self.R, steps, lr, want_alpha)

    def leaves(self, cap: int = 1 << 22):
        return slr_leaves(self.ctx, cap)

    def schedule(self, D: int):
        return slr_schedule(self.ctx, D)

    def split_set(self):
        return slr_split_set(self.ctx)

    def wait_selfcheck(self, limit: int = 4096):
        return slr_wait_selfcheck(self.ctx, limit)
