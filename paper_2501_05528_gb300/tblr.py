"""Python binding of libtblr.so (include/tblr.h): argument marshalling only.

Every function named ``tblr_*`` here calls the C entry point of the same name;
PyTorch supplies device memory (torch tensors) and the current CUDA stream.
Nothing here computes any step of the method: all of it runs in the CUDA
library, and a missing library or GPU raises instead of falling back.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libtblr.so")

TBLR_OK, TBLR_EINVAL, TBLR_ECUDA, TBLR_EUNSUPPORTED, TBLR_EWORKSPACE, TBLR_ETIMEOUT = 0, -1, -2, -3, -4, -5
KERNELS = {"laplace2d": 1, "laplace3d": 2, "dense": 3}
FP64, MIXED = 0, 1
NEARFIELD_PROBE, NEARFIELD_EXACT = 0, 1
SKETCH_BLACKBOX, SKETCH_TAGGED, SKETCH_SELFADJOINT = 0, 1, 2
Z_PROJECT, Z_MINRATIO = 0, 1


class TblrError(RuntimeError):
    def __init__(self, status, where):
        msg = lib().tblr_last_error().decode(errors="replace")
        super().__init__(f"{where}: status {status}: {msg}")
        self.status = status


class Problem(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int32), ("kernel", ctypes.c_int32), ("n", ctypes.c_int64),
                ("grid", ctypes.c_int32 * 3), ("lo", ctypes.c_double * 3),
                ("hi", ctypes.c_double * 3), ("k", ctypes.c_int32), ("p", ctypes.c_int32),
                ("e", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("nearfield", ctypes.c_int32), ("sketch", ctypes.c_int32),
                ("zrule", ctypes.c_int32)]


class Sizes(ctypes.Structure):
    _fields_ = [("b", ctypes.c_int64), ("ell", ctypes.c_int32), ("r", ctypes.c_int32),
                ("s3", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("sketch_cols", ctypes.c_int64)]


class LayoutStruct(ctypes.Structure):
    _fields_ = [(name, ctypes.c_void_p) for name in
                ("perm", "box_of", "offsets", "nbr", "nnbr", "colour", "pts")]


class Job(ctypes.Structure):
    _fields_ = [("prob", Problem)] + [(n, ctypes.c_void_p) for n in
                                      ("points", "T", "G", "H", "dense")] + [
        ("lay", LayoutStruct), ("nf_off", ctypes.c_void_p), ("m_max_dev", ctypes.c_void_p),
        ("m_max", ctypes.c_int32), ("reserved", ctypes.c_int32), ("nf_total", ctypes.c_int64)] + [
        (n, ctypes.c_void_p) for n in ("yz", "z", "tau", "rho", "u", "v", "ranks", "at", "bnear",
                                       "ws")] + [("ws_bytes", ctypes.c_size_t)]


class Request(ctypes.Structure):
    _fields_ = [("prob", Problem)] + [(n, ctypes.c_void_p) for n in (
        "points_h", "T_h", "G_h", "H_h", "perm_h", "offsets_h", "nbr_h", "ranks_h", "u_h", "v_h",
        "at_h", "bnear_h")] + [("bnear_capacity", ctypes.c_int64)]


class ServerReport(ctypes.Structure):
    _fields_ = [("completed", ctypes.c_uint64), ("failed", ctypes.c_uint64),
                ("pending", ctypes.c_uint64), ("active", ctypes.c_uint64),
                ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double),
                ("throughput", ctypes.c_double), ("mem_in_use", ctypes.c_size_t),
                ("mem_peak", ctypes.c_size_t)]


_VP, _I64, _SZ, _I32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_size_t, ctypes.c_int32
_PP = ctypes.POINTER(Problem)
_PL = ctypes.POINTER(LayoutStruct)
_SIGNATURES = {
    "tblr_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "tblr_last_error": (ctypes.c_char_p, []),
    "tblr_sizes_of": (ctypes.c_int, [_PP, ctypes.POINTER(Sizes)]),
    "tblr_tessellate_workspace": (_SZ, [_PP]),
    "tblr_tessellate": (ctypes.c_int, [_PP, _VP, _PL, _VP, _SZ, _VP]),
    "tblr_tessellate_noalloc": (ctypes.c_int, [_PP, _VP, _PL, _VP]),
    "tblr_nearfield_offsets": (ctypes.c_int, [_PP, _PL, _VP, _VP, _VP]),
    "tblr_test_matrices": (ctypes.c_int, [_PP, _PL, _VP, _VP, _VP, _VP, _VP]),
    "tblr_apply_workspace": (_SZ, [_PP, _I64, ctypes.c_int]),
    "tblr_apply": (ctypes.c_int, [_PP, _PL, _VP, _VP, _I64, _VP, _I64, ctypes.c_int, ctypes.c_int,
                                  _VP, _SZ, _VP]),
    "tblr_sketch_workspace": (_SZ, [_PP]),
    "tblr_sketch": (ctypes.c_int, [_PP, _PL, _VP, _VP, _VP, _VP, _SZ, _VP]),
    "tblr_decode": (ctypes.c_int, [_PP, _PL, _VP, _VP, _VP, _VP, _VP]),
    "tblr_far_indicator": (ctypes.c_int, [_PP, _PL, _VP, _VP]),
    "tblr_tagged_sketch_workspace": (_SZ, [_PP]),
    "tblr_tagged_sketch": (ctypes.c_int, [_PP, _PL, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _SZ, _VP]),
    "tblr_tune_tagged_sketch": (ctypes.c_int, [_PP, _PL, _VP, _VP, _VP, _VP, _VP, _VP, _SZ,
                                               ctypes.POINTER(ctypes.c_int32), _VP]),
    "tblr_tuned_width": (ctypes.c_int, [_PP, ctypes.POINTER(ctypes.c_int32)]),
    "tblr_tune_clear": (None, []),
    "tblr_combine": (ctypes.c_int, [_PP, _PL, _VP, _VP, _VP, _VP, _VP]),
    "tblr_col_workspace": (_SZ, [_PP]),
    "tblr_col": (ctypes.c_int, [_PP, _PL, _VP, _VP, _VP, _VP, _SZ, _VP]),
    "tblr_coupling_workspace": (_SZ, [_PP]),
    "tblr_coupling": (ctypes.c_int, [_PP, _PL, _VP, _VP, _VP, _VP, _I32, _VP, _VP, _SZ, _VP]),
    "tblr_nearfield_workspace": (_SZ, [_PP, _I32]),
    "tblr_nearfield": (ctypes.c_int, [_PP, _PL, _VP, _VP, _VP, _VP, _VP, _VP, _I32, _VP, _VP, _SZ,
                                      _VP]),
    "tblr_compress_workspace": (_SZ, [_PP, _I32]),
    "tblr_compress": (ctypes.c_int, [_PP, _PL, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP,
                                     _VP, _VP, _VP, _I32, _VP, _VP, _SZ, _VP]),
    "tblr_compress_host": (ctypes.c_int, [_PP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP,
                                          _VP, _VP, _VP, _I64, ctypes.POINTER(_I64), _VP]),
    "tblr_release_device_cache": (ctypes.c_int, []),
    "tblr_device_timeouts": (ctypes.c_int, [ctypes.POINTER(ctypes.c_uint)]),
    "tblr_decode_lp_failures": (ctypes.c_int, [ctypes.POINTER(ctypes.c_uint)]),
    "tblr_batch_plan": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(Job), _VP]),
    "tblr_batch_run": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(Job), ctypes.c_int, _VP]),
    "tblr_graph_create": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(Job), ctypes.c_int, _VP,
                                         ctypes.POINTER(_VP)]),
    "tblr_graph_launch": (ctypes.c_int, [_VP, _VP]),
    "tblr_graph_destroy": (None, [_VP]),
    "tblr_server_create": (ctypes.c_int, [ctypes.POINTER(_VP), ctypes.c_int, _SZ, ctypes.c_int]),
    "tblr_server_submit": (ctypes.c_int, [_VP, ctypes.POINTER(Request),
                                          ctypes.POINTER(ctypes.c_uint64)]),
    "tblr_server_wait": (ctypes.c_int, [_VP, ctypes.c_uint64, ctypes.c_int,
                                        ctypes.POINTER(ctypes.c_int),
                                        ctypes.POINTER(ctypes.c_double)]),
    "tblr_server_stats": (ctypes.c_int, [_VP, ctypes.POINTER(ServerReport)]),
    "tblr_server_destroy": (None, [_VP]),
}

_lib = None


def lib():
    """Load libtblr.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -m paper_2501_05528_gb300.build`")
        handle = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGNATURES.items():
            fn = getattr(handle, name)
            fn.restype = res
            fn.argtypes = args
        _lib = handle
    return _lib


def _require_cuda():
    if not torch.cuda.is_available():
        raise RuntimeError("tblr needs a CUDA device; there is no CPU fallback")


def _check(status, where):
    if status != TBLR_OK:
        raise TblrError(status, where)


def _p(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _dev():
    return torch.device("cuda", torch.cuda.current_device())


def make_problem(d, kernel, n, grid, lo, hi, k, p=10, e=3, precision=FP64,
                 nearfield=NEARFIELD_PROBE, sketch=SKETCH_BLACKBOX, selfadjoint=False,
                 zrule=Z_PROJECT) -> Problem:
    g = list(grid) + [1] * (3 - len(grid))
    lo3 = list(lo) + [0.0] * (3 - len(lo))
    hi3 = list(hi) + [1.0] * (3 - len(hi))
    kind = KERNELS[kernel] if isinstance(kernel, str) else int(kernel)
    return Problem(d, kind, n, (ctypes.c_int32 * 3)(*g), (ctypes.c_double * 3)(*lo3),
                   (ctypes.c_double * 3)(*hi3), k, p, e, precision, nearfield,
                   sketch | (SKETCH_SELFADJOINT if selfadjoint else 0), zrule)


def tblr_sizes_of(prob: Problem) -> Sizes:
    out = Sizes()
    _check(lib().tblr_sizes_of(ctypes.byref(prob), ctypes.byref(out)), "tblr_sizes_of")
    return out


class Layout:
    """Device tensors of a tessellation and the C struct pointing at them."""

    def __init__(self, prob: Problem):
        sz = tblr_sizes_of(prob)
        dev = _dev()
        n, b, s3 = prob.n, sz.b, sz.s3
        i32 = dict(dtype=torch.int32, device=dev)
        self.perm = torch.empty(n, **i32)
        self.box_of = torch.empty(n, **i32)
        self.offsets = torch.empty(b + 1, **i32)
        self.nbr = torch.empty(b * s3, **i32)
        self.nnbr = torch.empty(b, **i32)
        self.colour = torch.empty(b, **i32)
        self.pts = torch.empty(prob.d * n, dtype=torch.float64, device=dev)
        self.struct = LayoutStruct(*[t.data_ptr() for t in (
            self.perm, self.box_of, self.offsets, self.nbr, self.nnbr, self.colour, self.pts)])

    @property
    def ref(self):
        return ctypes.byref(self.struct)


def tblr_tessellate(prob: Problem, points: torch.Tensor) -> Layout:
    _require_cuda()
    points = points.contiguous()
    lay = Layout(prob)
    nbytes = lib().tblr_tessellate_workspace(ctypes.byref(prob))
    ws = torch.empty(max(nbytes, 1), dtype=torch.uint8, device=_dev())
    _check(lib().tblr_tessellate(ctypes.byref(prob), _p(points), lay.ref, _p(ws), nbytes, _stream()),
           "tblr_tessellate")
    lay._ws = ws
    return lay


def tblr_tessellate_noalloc(prob: Problem, points: torch.Tensor) -> Layout:
    """Tessellation whose scratch is the library's fixed static device array
    (no allocation inside the call; the caller still owns inputs and outputs)."""
    _require_cuda()
    points = points.contiguous()
    lay = Layout(prob)
    _check(lib().tblr_tessellate_noalloc(ctypes.byref(prob), _p(points), lay.ref, _stream()),
           "tblr_tessellate_noalloc")
    return lay


def tblr_nearfield_offsets(prob: Problem, lay: Layout):
    sz = tblr_sizes_of(prob)
    nf_off = torch.empty(sz.b * sz.s3 + 1, dtype=torch.int64, device=_dev())
    m_max = torch.empty(1, dtype=torch.int32, device=_dev())
    _check(lib().tblr_nearfield_offsets(ctypes.byref(prob), lay.ref, _p(nf_off), _p(m_max),
                                        _stream()), "tblr_nearfield_offsets")
    return nf_off, m_max


def tblr_test_matrices(prob, lay, T, G, H):
    sz = tblr_sizes_of(prob)
    out = torch.empty(sz.sketch_cols * prob.n, dtype=torch.float64, device=_dev())
    _check(lib().tblr_test_matrices(ctypes.byref(prob), lay.ref, _p(T), _p(G), _p(H), _p(out),
                                    _stream()), "tblr_test_matrices")
    return out


def tblr_apply(prob, lay, xt, ncols, adjoint=0, precision=FP64, dense=None):
    """Y = A X (or A^T X); xt is K-major [ncols * n]; returns Y as [n, ncols]."""
    y = torch.empty(prob.n, ncols, dtype=torch.float64, device=_dev())
    nbytes = lib().tblr_apply_workspace(ctypes.byref(prob), ncols, precision)
    ws = torch.empty(max(nbytes, 1), dtype=torch.uint8, device=_dev())
    _check(lib().tblr_apply(ctypes.byref(prob), lay.ref, _p(dense), _p(xt), ncols, _p(y), ncols,
                            adjoint, precision, _p(ws), nbytes, _stream()), "tblr_apply")
    return y


def tblr_sketch(prob, lay, omega_psi, dense=None):
    sz = tblr_sizes_of(prob)
    yz = torch.empty(prob.n, sz.sketch_cols, dtype=torch.float64, device=_dev())
    nbytes = lib().tblr_sketch_workspace(ctypes.byref(prob))
    ws = torch.empty(max(nbytes, 1), dtype=torch.uint8, device=_dev())
    _check(lib().tblr_sketch(ctypes.byref(prob), lay.ref, _p(dense), _p(omega_psi), _p(yz), _p(ws),
                             nbytes, _stream()), "tblr_sketch")
    return yz


def tblr_decode(prob, lay, T):
    sz = tblr_sizes_of(prob)
    dev = _dev()
    z = torch.empty(sz.b, sz.ell, dtype=torch.float64, device=dev)
    tau = torch.empty(sz.b, sz.b, dtype=torch.float64, device=dev)
    rho = torch.empty(sz.b, dtype=torch.float64, device=dev)
    _check(lib().tblr_decode(ctypes.byref(prob), lay.ref, _p(T), _p(z), _p(tau), _p(rho),
                             _stream()), "tblr_decode")
    return z, tau, rho


def tblr_tagged_sketch(prob, lay, tau, G, H, dense=None):
    """S, R from the projected tags (TBLR_SKETCH_TAGGED), without forming Y, Z.  With the
    self-adjoint flag only S is formed and R is returned as S."""
    sz = tblr_sizes_of(prob)
    s = torch.empty(prob.n, sz.r, dtype=torch.float64, device=_dev())
    rr = torch.empty_like(s)
    nbytes = lib().tblr_tagged_sketch_workspace(ctypes.byref(prob))
    ws = torch.empty(max(nbytes, 1), dtype=torch.uint8, device=_dev())
    _check(lib().tblr_tagged_sketch(ctypes.byref(prob), lay.ref, _p(dense), _p(tau), _p(G), _p(H),
                                    _p(s), _p(rr), _p(ws), nbytes, _stream()), "tblr_tagged_sketch")
    return (s, s) if prob.sketch & SKETCH_SELFADJOINT else (s, rr)


def tblr_tune_tagged_sketch(prob, lay, tau, G, H):
    """Time every admissible tile width of the mixed tagged sketch on this problem and record
    the fastest for its class (this process).  Returns (width, S, R) with the chosen width's S, R."""
    sz = tblr_sizes_of(prob)
    s = torch.empty(prob.n, sz.r, dtype=torch.float64, device=_dev())
    rr = torch.empty_like(s)
    nbytes = lib().tblr_tagged_sketch_workspace(ctypes.byref(prob))
    ws = torch.empty(max(nbytes, 1), dtype=torch.uint8, device=_dev())
    w = ctypes.c_int32(0)
    _check(lib().tblr_tune_tagged_sketch(ctypes.byref(prob), lay.ref, _p(tau), _p(G), _p(H), _p(s),
                                         _p(rr), _p(ws), nbytes, ctypes.byref(w), _stream()),
           "tblr_tune_tagged_sketch")
    return w.value, s, (s if prob.sketch & SKETCH_SELFADJOINT else rr)


def tblr_tuned_width(prob) -> int:
    w = ctypes.c_int32(0)
    _check(lib().tblr_tuned_width(ctypes.byref(prob), ctypes.byref(w)), "tblr_tuned_width")
    return w.value


def tblr_tune_clear() -> None:
    lib().tblr_tune_clear()


def tblr_combine(prob, lay, yz, z):
    sz = tblr_sizes_of(prob)
    s = torch.empty(prob.n, sz.r, dtype=torch.float64, device=_dev())
    rr = torch.empty_like(s)
    _check(lib().tblr_combine(ctypes.byref(prob), lay.ref, _p(yz), _p(z), _p(s), _p(rr), _stream()),
           "tblr_combine")
    return s, rr


def tblr_col(prob, lay, s):
    sz = tblr_sizes_of(prob)
    u = torch.empty(prob.n, prob.k, dtype=torch.float64, device=_dev())
    ranks = torch.empty(sz.b, dtype=torch.int32, device=_dev())
    nbytes = lib().tblr_col_workspace(ctypes.byref(prob))
    ws = torch.empty(max(nbytes, 1), dtype=torch.uint8, device=_dev())
    _check(lib().tblr_col(ctypes.byref(prob), lay.ref, _p(s), _p(u), _p(ranks), _p(ws), nbytes,
                          _stream()), "tblr_col")
    return u, ranks


def tblr_coupling(prob, lay, u, v, ranks, m_max: int, dense=None):
    sz = tblr_sizes_of(prob)
    at = torch.empty(sz.b, sz.b, prob.k, prob.k, dtype=torch.float64, device=_dev())
    nbytes = lib().tblr_coupling_workspace(ctypes.byref(prob))
    ws = torch.empty(max(nbytes, 1), dtype=torch.uint8, device=_dev())
    _check(lib().tblr_coupling(ctypes.byref(prob), lay.ref, _p(dense), _p(u), _p(v), _p(ranks),
                               m_max, _p(at), _p(ws), nbytes, _stream()), "tblr_coupling")
    return at


def tblr_nearfield(prob, lay, u, at, v, ranks, nf_off, m_max: int, total: int, dense=None):
    bnear = torch.empty(max(total, 1), dtype=torch.float64, device=_dev())
    nbytes = lib().tblr_nearfield_workspace(ctypes.byref(prob), m_max)
    ws = torch.empty(max(nbytes, 1), dtype=torch.uint8, device=_dev())
    _check(lib().tblr_nearfield(ctypes.byref(prob), lay.ref, _p(dense), _p(u), _p(at), _p(v),
                                _p(ranks), _p(nf_off), m_max, _p(bnear), _p(ws), nbytes, _stream()),
           "tblr_nearfield")
    return bnear


def tblr_far_indicator(prob, lay):
    """Algorithm 3's far-field mask as tags: tau[i, c] = 0 for c in N_i, else 1."""
    sz = tblr_sizes_of(prob)
    tau = torch.empty(sz.b, sz.b, dtype=torch.float64, device=_dev())
    _check(lib().tblr_far_indicator(ctypes.byref(prob), lay.ref, _p(tau), _stream()),
           "tblr_far_indicator")
    return tau


def tblr_decode_lp_failures() -> int:
    """Synchronise the device; return and reset the count of §5.3 programs without an optimum."""
    out = ctypes.c_uint(0)
    _check(lib().tblr_decode_lp_failures(ctypes.byref(out)), "tblr_decode_lp_failures")
    return int(out.value)


def tblr_device_timeouts() -> int:
    """Synchronise the device; return and reset the count of timed-out device waits."""
    out = ctypes.c_uint(0)
    _check(lib().tblr_device_timeouts(ctypes.byref(out)), "tblr_device_timeouts")
    return int(out.value)


class Compressed:
    """Device-resident result of one compression (reconstruct_tag, Table 1)."""

    def __init__(self, **kw):
        self.__dict__.update(kw)


def tblr_compress(prob, lay, T, G, H, dense=None, nf=None, out=None, ws=None):
    """Steps a2..a8 on a tessellated problem.  ``nf`` = (nf_off, m_max_int, total_int);
    ``out``/``ws`` may be a previous result and workspace to reuse."""
    sz = tblr_sizes_of(prob)
    dev = _dev()
    if nf is None:
        nf_off, m_max_t = tblr_nearfield_offsets(prob, lay)
        m_max = int(m_max_t.item())
        total = int(nf_off[-1].item())
    else:
        nf_off, m_max, total = nf
    f64 = dict(dtype=torch.float64, device=dev)
    if out is None:
        out = Compressed(
            yz=torch.empty(prob.n, sz.sketch_cols, **f64), z=torch.empty(sz.b, sz.ell, **f64),
            tau=torch.empty(sz.b, sz.b, **f64), rho=torch.empty(sz.b, **f64),
            u=torch.empty(prob.n, prob.k, **f64), v=torch.empty(prob.n, prob.k, **f64),
            ranks=torch.empty(sz.b, dtype=torch.int32, device=dev),
            at=torch.empty(sz.b, sz.b, prob.k, prob.k, **f64),
            bnear=torch.empty(max(total, 1), **f64))
    out.nf_off, out.m_max, out.total, out.layout = nf_off, m_max, total, lay
    nbytes = lib().tblr_compress_workspace(ctypes.byref(prob), m_max)
    if ws is None or ws.numel() < nbytes:
        ws = torch.empty(max(nbytes, 1), dtype=torch.uint8, device=dev)
    out.ws = ws
    _check(lib().tblr_compress(ctypes.byref(prob), lay.ref, _p(dense), _p(T), _p(G), _p(H),
                               _p(out.yz), _p(out.z), _p(out.tau), _p(out.rho), _p(out.u),
                               _p(out.v), _p(out.ranks), _p(out.at), _p(nf_off), m_max,
                               _p(out.bnear), _p(ws), nbytes, _stream()), "tblr_compress")
    return out


def compress(prob, points, T, G, H, dense=None):
    """Tessellate and compress in one call (device tensors in, device tensors out)."""
    lay = tblr_tessellate(prob, points)
    return tblr_compress(prob, lay, T, G, H, dense=dense)


def tblr_compress_host(prob, points, T, G, H, dense=None, outputs=None, stream=None):
    """End to end from host arrays (numpy or pinned CPU tensors).  Returns a dict of
    host arrays.  ``outputs`` may hold preallocated (pinned) buffers to reuse."""
    sz = tblr_sizes_of(prob)
    n, b, k, s3 = prob.n, sz.b, prob.k, sz.s3

    def host(arr, dtype):
        t = torch.as_tensor(np.ascontiguousarray(arr)) if isinstance(arr, np.ndarray) else arr
        return t.to(dtype).contiguous()

    pts, Th, Gh, Hh = (host(x, torch.float64) for x in (points, T, G, H))
    dn = None if dense is None else host(dense, torch.float64)
    o = outputs
    if o is None:
        o = dict(perm=torch.empty(n, dtype=torch.int32), offsets=torch.empty(b + 1, dtype=torch.int32),
                 nbr=torch.empty(b * s3, dtype=torch.int32), ranks=torch.empty(b, dtype=torch.int32),
                 u=torch.empty(n, k, dtype=torch.float64), v=torch.empty(n, k, dtype=torch.float64),
                 at=torch.empty(b, b, k, k, dtype=torch.float64),
                 bnear=torch.empty(1, dtype=torch.float64))
    need = ctypes.c_int64(0)
    st = ctypes.c_void_p(stream) if stream is not None else _stream()
    args = (ctypes.byref(prob), _p(pts), _p(Th), _p(Gh), _p(Hh), _p(dn), _p(o["perm"]),
            _p(o["offsets"]), _p(o["nbr"]), _p(o["ranks"]), _p(o["u"]), _p(o["v"]), _p(o["at"]))
    status = lib().tblr_compress_host(*args, _p(o["bnear"]), o["bnear"].numel(),
                                      ctypes.byref(need), st)
    if status == TBLR_EWORKSPACE:
        pin = o["u"].is_pinned()
        o["bnear"] = torch.empty(need.value, dtype=torch.float64, pin_memory=pin)
        status = lib().tblr_compress_host(*args, _p(o["bnear"]), o["bnear"].numel(),
                                          ctypes.byref(need), st)
    _check(status, "tblr_compress_host")
    o["bnear_size"] = need.value
    return o


# ------------------------------------------------------------------ batches

class BatchJob:
    """Device buffers of one job of a batch and its C descriptor (tblr_job)."""

    def __init__(self, prob, points, T, G, H):
        self.prob = prob
        self.points, self.T, self.G, self.H = (x.contiguous() for x in (points, T, G, H))
        sz = tblr_sizes_of(prob)
        dev = _dev()
        self.sz = sz
        self.lay = Layout(prob)
        self.nf_off = torch.empty(sz.b * sz.s3 + 1, dtype=torch.int64, device=dev)
        self.m_max_dev = torch.empty(1, dtype=torch.int32, device=dev)
        tws = lib().tblr_tessellate_workspace(ctypes.byref(prob))
        self.ws = torch.empty(max(tws, 1), dtype=torch.uint8, device=dev)
        self.c = Job(prob=prob, points=self.points.data_ptr(), T=self.T.data_ptr(),
                     G=self.G.data_ptr(), H=self.H.data_ptr(), dense=None, lay=self.lay.struct,
                     nf_off=self.nf_off.data_ptr(), m_max_dev=self.m_max_dev.data_ptr(),
                     ws=self.ws.data_ptr(), ws_bytes=self.ws.numel())

    def allocate_outputs(self):
        """After tblr_batch_plan: outputs and the full workspace, sized from the plan."""
        sz, dev, n, k = self.sz, _dev(), self.prob.n, self.prob.k
        f64 = dict(dtype=torch.float64, device=dev)
        tagged = bool(self.prob.sketch & SKETCH_TAGGED)   # Y, Z are never formed
        self.out = Compressed(
            yz=torch.empty(1 if tagged else n * sz.sketch_cols, **f64),
            z=torch.empty(sz.b, sz.ell, **f64),
            tau=torch.empty(sz.b, sz.b, **f64), rho=torch.empty(sz.b, **f64),
            u=torch.empty(n, k, **f64), v=torch.empty(n, k, **f64),
            ranks=torch.empty(sz.b, dtype=torch.int32, device=dev),
            at=torch.empty(sz.b, sz.b, k, k, **f64),
            bnear=torch.empty(max(self.c.nf_total, 1), **f64),
            nf_off=self.nf_off, m_max=self.c.m_max, total=self.c.nf_total, layout=self.lay)
        need = max(lib().tblr_compress_workspace(ctypes.byref(self.prob), self.c.m_max),
                   self.ws.numel())
        self.ws = torch.empty(need, dtype=torch.uint8, device=dev)
        o = self.out
        for name in ("yz", "z", "tau", "rho", "u", "v", "ranks", "at", "bnear"):
            setattr(self.c, name, getattr(o, name).data_ptr())
        self.c.ws = self.ws.data_ptr()
        self.c.ws_bytes = self.ws.numel()


def _job_array(jobs):
    arr = (Job * len(jobs))()
    for i, j in enumerate(jobs):
        arr[i] = j.c
    return arr


def tblr_batch_plan(jobs):
    _require_cuda()
    arr = _job_array(jobs)
    _check(lib().tblr_batch_plan(len(jobs), arr, _stream()), "tblr_batch_plan")
    for i, j in enumerate(jobs):
        j.c.m_max, j.c.nf_total = arr[i].m_max, arr[i].nf_total
        j.allocate_outputs()


def tblr_batch_run(jobs, n_streams=4):
    arr = _job_array(jobs)
    _check(lib().tblr_batch_run(len(jobs), arr, n_streams, _stream()), "tblr_batch_run")


class Graph:
    """A batch captured into one CUDA graph (tblr_graph_create / launch / destroy)."""

    def __init__(self, jobs, n_streams=4):
        self._jobs = jobs
        self.h = ctypes.c_void_p()
        arr = _job_array(jobs)
        _check(lib().tblr_graph_create(len(jobs), arr, n_streams, _stream(), ctypes.byref(self.h)),
               "tblr_graph_create")

    def launch(self):
        _check(lib().tblr_graph_launch(self.h, _stream()), "tblr_graph_launch")

    def __del__(self):
        if getattr(self, "h", None) and self.h.value:
            lib().tblr_graph_destroy(self.h)
            self.h = ctypes.c_void_p()


# ------------------------------------------------------------------ serving

class Server:
    """Continuous-batching server (tblr_server_*).  submit() takes pinned host arrays."""

    def __init__(self, mem_budget_bytes, max_inflight=8, device=None):
        _require_cuda()
        self.h = ctypes.c_void_p()
        dev = torch.cuda.current_device() if device is None else device
        _check(lib().tblr_server_create(ctypes.byref(self.h), dev, int(mem_budget_bytes),
                                        max_inflight), "tblr_server_create")
        self._keep = {}

    def submit(self, prob, points, T, G, H, outputs):
        """points/T/G/H and outputs (dict as from host_outputs) are CPU tensors, pinned."""
        o = outputs
        req = Request(prob=prob, points_h=points.data_ptr(), T_h=T.data_ptr(), G_h=G.data_ptr(),
                      H_h=H.data_ptr(), perm_h=o["perm"].data_ptr(),
                      offsets_h=o["offsets"].data_ptr(), nbr_h=o["nbr"].data_ptr(),
                      ranks_h=o["ranks"].data_ptr(), u_h=o["u"].data_ptr(), v_h=o["v"].data_ptr(),
                      at_h=o["at"].data_ptr(), bnear_h=o["bnear"].data_ptr(),
                      bnear_capacity=o["bnear"].numel())
        ticket = ctypes.c_uint64()
        _check(lib().tblr_server_submit(self.h, ctypes.byref(req), ctypes.byref(ticket)),
               "tblr_server_submit")
        self._keep[ticket.value] = (points, T, G, H, outputs)
        return ticket.value

    def wait(self, ticket, timeout_ms=600000):
        st, lat = ctypes.c_int(), ctypes.c_double()
        _check(lib().tblr_server_wait(self.h, ticket, timeout_ms, ctypes.byref(st),
                                      ctypes.byref(lat)), "tblr_server_wait")
        self._keep.pop(ticket, None)
        return st.value, lat.value

    def stats(self):
        r = ServerReport()
        _check(lib().tblr_server_stats(self.h, ctypes.byref(r)), "tblr_server_stats")
        return {f: getattr(r, f) for f, _ in ServerReport._fields_}

    def close(self):
        if self.h.value:
            lib().tblr_server_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        self.close()


def host_outputs(prob, bnear_capacity, pin=True):
    """Host output buffers for one request (sizes as in tblr_compress_host)."""
    sz = tblr_sizes_of(prob)
    n, b, k = prob.n, sz.b, prob.k

    def e(*shape, dtype):
        t = torch.empty(*shape, dtype=dtype)
        return t.pin_memory() if pin else t
    return dict(perm=e(n, dtype=torch.int32), offsets=e(b + 1, dtype=torch.int32),
                nbr=e(b * sz.s3, dtype=torch.int32), ranks=e(b, dtype=torch.int32),
                u=e(n, k, dtype=torch.float64), v=e(n, k, dtype=torch.float64),
                at=e(b, b, k, k, dtype=torch.float64),
                bnear=e(max(int(bnear_capacity), 1), dtype=torch.float64))
