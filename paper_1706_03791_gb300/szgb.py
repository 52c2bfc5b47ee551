"""Python binding of the C ABI in include/szgb.h (argument marshalling only).

Every step of compression and decompression runs in the CUDA library
``libszgb.so`` built in-tree for sm_103a; this module only passes pointers
and sizes.  PyTorch tensors provide device memory and streams; NumPy arrays
are passed as host buffers.  If the library is missing or cannot be loaded
the import fails: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import json
import os
import time

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libszgb.so")

OK, EINVAL, ENONFINITE, ETRUNC, ECORRUPT, ENOMEM, EBUDGET, ETIMEOUT, ECUDA, EUNSUPPORTED = \
    0, -1, -2, -3, -4, -5, -6, -7, -8, -9
ESCRATCH = -10
ABS, REL, ABS_AND_REL = 0, 1, 2
CHUNK_ROWS = 0xFFFFFFFF  # chunk_points: one Huffman chunk per row


class SzgbError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        super().__init__("%s: %s (%d)" % (what, strerror(code), code))


class Params(C.Structure):
    _fields_ = [("ndim", C.c_int), ("shape", C.c_uint64 * 4), ("mode", C.c_int),
                ("eb_abs", C.c_double), ("eb_rel", C.c_double), ("layers", C.c_int),
                ("m", C.c_int), ("theta", C.c_double), ("variant", C.c_int), ("chunk_points", C.c_uint32)]


class Stats(C.Structure):
    _fields_ = [("n_points", C.c_uint64), ("n_unpred", C.c_uint64), ("stream_bytes", C.c_uint64),
                ("m", C.c_int), ("maxlen", C.c_int), ("nsym", C.c_uint32), ("eb_f", C.c_float),
                ("xmin", C.c_float), ("xmax", C.c_float), ("status", C.c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class Quality(C.Structure):
    _fields_ = [("max_abs_err", C.c_double), ("max_rel_err", C.c_double), ("rmse", C.c_double),
                ("nrmse", C.c_double), ("psnr", C.c_double), ("pearson", C.c_double), ("x_min", C.c_double),
                ("x_max", C.c_double), ("n", C.c_uint64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


OP_COMPRESS, OP_DECOMPRESS = 0, 1


class Request(C.Structure):
    _fields_ = [("op", C.c_int), ("in_", C.c_void_p), ("in_bytes", C.c_size_t), ("params", Params),
                ("out", C.c_void_p), ("out_cap", C.c_size_t)]


_lib = None


def lib():
    """Load libszgb.so (raises if it is not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libszgb.so is not built (run __graft_entry__.build())")
        L = C.CDLL(LIB_PATH)
        vp, sz = C.c_void_p, C.c_size_t
        L.szgb_create.argtypes = [C.POINTER(vp), C.c_int, sz]
        L.szgb_destroy.argtypes = [vp]
        L.szgb_destroy.restype = None
        L.szgb_set_stream.argtypes = [vp, vp]
        L.szgb_compress_bound.argtypes = [C.POINTER(Params)]
        L.szgb_compress_bound.restype = sz
        L.szgb_compress.argtypes = [vp, vp, C.c_int, C.POINTER(Params), vp, sz, C.c_int,
                                    C.POINTER(sz), C.POINTER(Stats)]
        L.szgb_compress_trace.argtypes = [vp, vp, C.POINTER(Params), vp, sz, C.POINTER(sz),
                                          C.POINTER(Stats), vp, vp]
        L.szgb_compress_4d.argtypes = [vp, vp, C.POINTER(C.c_uint64), C.POINTER(Params), vp, sz, C.POINTER(sz),
                                       C.POINTER(Stats), vp, vp]
        L.szgb_decompress.argtypes = [vp, vp, sz, C.c_int, vp, sz, C.c_int]
        L.szgb_stream_info.argtypes = [vp, sz, C.POINTER(Params), C.POINTER(C.c_uint64)]
        L.szgb_set_profiling.argtypes = [vp, C.c_int]
        L.szgb_num_phases.argtypes = []
        L.szgb_phase_name.argtypes = [C.c_int]
        L.szgb_phase_name.restype = C.c_char_p
        L.szgb_phase_times.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(C.c_uint64), C.c_int,
                                       C.c_int]
        L.szgb_decompress_noalloc.argtypes = [vp, sz, vp, sz, vp]
        L.szgb_compress_batch.argtypes = [vp, C.c_int, C.POINTER(vp), C.POINTER(Params), C.POINTER(vp),
                                          C.POINTER(sz), C.POINTER(sz), C.POINTER(Stats)]
        L.szgb_decompress_batch.argtypes = [vp, C.c_int, C.POINTER(vp), C.POINTER(sz), C.POINTER(vp),
                                            C.POINTER(sz), C.POINTER(C.c_int)]
        L.szgb_set_graphs.argtypes = [vp, C.c_int]
        L.szgb_set_wave_ctas.argtypes = [vp, C.c_int]
        L.szgb_debug_set_wait_limit.argtypes = [vp, C.c_uint64]
        L.szgb_debug_skip_item.argtypes = [vp, C.c_int]
        L.szgb_quality_dev.argtypes = [vp, vp, vp, sz, C.POINTER(Quality)]
        L.szgb_suggest_m.argtypes = [C.POINTER(Stats), C.c_double, C.POINTER(C.c_double)]
        L.szgb_hit_count_dev.argtypes = [vp, vp, vp, C.c_int, C.POINTER(C.c_uint64), C.c_int, C.c_double,
                                         C.POINTER(C.c_uint64)]
        L.szgb_autotune.argtypes = [vp, vp, C.POINTER(Params), C.c_int, C.POINTER(C.c_int),
                                    C.POINTER(C.c_int), C.POINTER(C.c_double)]
        L.szgb_autotune_batch.argtypes = [vp, C.c_int, C.POINTER(vp), C.POINTER(Params), C.c_int,
                                          C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_double)]
        L.szgb_tune_save.argtypes = [vp, C.c_char_p]
        L.szgb_tune_load.argtypes = [vp, C.c_char_p]
        L.szgb_server_create.argtypes = [C.POINTER(vp), C.c_int, sz, C.c_int, C.c_int]
        L.szgb_submit.argtypes = [vp, C.POINTER(Request), C.POINTER(C.c_uint64)]
        L.szgb_poll.argtypes = [vp, C.c_uint64, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(sz)]
        L.szgb_wait.argtypes = [vp, C.c_uint64, C.POINTER(C.c_int), C.POINTER(sz)]
        L.szgb_server_stats.argtypes = [vp, C.POINTER(C.c_uint64), C.POINTER(C.c_uint64), C.POINTER(sz)]
        L.szgb_server_destroy.argtypes = [vp]
        L.szgb_server_destroy.restype = None
        L.szgb_strerror.argtypes = [C.c_int]
        L.szgb_strerror.restype = C.c_char_p
        _lib = L
    return _lib


def strerror(code: int) -> str:
    return lib().szgb_strerror(code).decode()


# names of every entry point declared in include/szgb.h
EXPORTS = ["szgb_create", "szgb_destroy", "szgb_set_stream", "szgb_compress_bound", "szgb_compress",
           "szgb_compress_trace", "szgb_decompress", "szgb_stream_info", "szgb_set_profiling",
           "szgb_num_phases", "szgb_phase_name", "szgb_phase_times", "szgb_strerror",
           "szgb_decompress_noalloc", "szgb_compress_batch", "szgb_decompress_batch", "szgb_set_graphs", "szgb_set_wave_ctas",
           "szgb_server_create", "szgb_submit", "szgb_poll", "szgb_wait", "szgb_server_stats",
           "szgb_server_destroy", "szgb_autotune", "szgb_autotune_batch", "szgb_tune_save", "szgb_tune_load",
           "szgb_quality_dev", "szgb_hit_count_dev", "szgb_suggest_m", "szgb_compress_4d",
           "szgb_debug_set_wait_limit", "szgb_debug_skip_item"]


VARIANT_EXACT, VARIANT_LATTICE = 0, 1


def make_params(shape, mode=REL, eb_abs=0.0, eb_rel=1e-4, layers=1, m=0, theta=0.99, variant=0,
                chunk_points=0) -> Params:
    p = Params()
    shape = tuple(int(s) for s in shape)
    p.ndim = len(shape)
    for i in range(4):
        p.shape[i] = shape[i] if i < len(shape) else 0
    p.mode, p.eb_abs, p.eb_rel, p.layers, p.m, p.theta = mode, float(eb_abs), float(eb_rel), \
        int(layers), int(m), float(theta)
    p.variant = int(variant)
    p.chunk_points = int(chunk_points)
    return p


def compress_bound(shape, **kw) -> int:
    p = make_params(shape, **kw)
    return int(lib().szgb_compress_bound(C.byref(p)))


def suggest_m(stats, theta: float = 0.99):
    """Algorithm 1, last step: (suggested m, interval hit rate) from the
    Stats of a compression -- m + 1 (at most 16) when fewer than theta of
    the points fell into one of the 2^m - 1 intervals, else m."""
    r = C.c_double()
    m = lib().szgb_suggest_m(C.byref(stats), float(theta), C.byref(r))
    if m < 0:
        raise SzgbError(m, "szgb_suggest_m")
    return m, r.value


def stream_info(stream) -> dict:
    s = np.ascontiguousarray(np.asarray(stream, dtype=np.uint8))
    p = Params()
    k = C.c_uint64()
    rc = lib().szgb_stream_info(s.ctypes.data, s.size, C.byref(p), C.byref(k))
    if rc:
        raise SzgbError(rc, "szgb_stream_info")
    return {"ndim": p.ndim, "shape": tuple(p.shape[i] for i in range(p.ndim)), "mode": p.mode,
            "eb_abs": p.eb_abs, "eb_rel": p.eb_rel, "layers": p.layers, "m": p.m,
            "theta": p.theta, "chunk_points": p.chunk_points, "n_unpred": k.value}


def _is_torch(a):
    return type(a).__module__.startswith("torch")


def _require_cuda(t, dtype, name, device=None):
    """Raise unless `t` is a contiguous CUDA tensor of `dtype` (on `device`
    when given): the library reads and writes through its raw pointer."""
    if not _is_torch(t) or not getattr(t, "is_cuda", False):
        raise TypeError("%s must be a CUDA tensor" % name)
    if t.dtype != dtype:
        raise TypeError("%s must be %s, not %s" % (name, dtype, t.dtype))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    if device is not None and t.device.index != device:
        raise ValueError("%s is on cuda:%s, the context on cuda:%d" % (name, t.device.index, device))


def _require_host(a, dtype, name):
    """Raise unless `a` is a C-contiguous NumPy array of `dtype`."""
    if not isinstance(a, np.ndarray):
        raise TypeError("%s must be a NumPy array" % name)
    if a.dtype != dtype:
        raise TypeError("%s must be %s, not %s" % (name, np.dtype(dtype), a.dtype))
    if not a.flags.c_contiguous:
        raise ValueError("%s must be C-contiguous" % name)


class Context:
    """A library context (device scratch and a stream) on one CUDA device."""

    def __init__(self, device: int = 0, budget: int = 0):
        self._h = C.c_void_p()
        rc = lib().szgb_create(C.byref(self._h), int(device), int(budget))
        if rc:
            raise SzgbError(rc, "szgb_create")
        self.device = device

    def close(self):
        if self._h:
            lib().szgb_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream_ptr: int | None):
        lib().szgb_set_stream(self._h, C.c_void_p(stream_ptr or 0))

    def set_profiling(self, on: bool):
        lib().szgb_set_profiling(self._h, 1 if on else 0)

    def phase_times(self, reset: bool = False) -> dict:
        L = lib()
        n = L.szgb_num_phases()
        ms = (C.c_double * n)()
        calls = (C.c_uint64 * n)()
        L.szgb_phase_times(self._h, ms, calls, n, 1 if reset else 0)
        return {L.szgb_phase_name(i).decode(): (ms[i], calls[i]) for i in range(n)}

    # -- compression ---------------------------------------------------------
    def compress(self, x, out=None, **kw):
        """Compress `x` (a CUDA float32 tensor, or a NumPy float32 array on the
        host; 1D-4D).
        Returns (stream, stats): with a CUDA input, `stream` is a view of the
        uint8 CUDA tensor `out` (allocated when None); with a NumPy input, a
        NumPy uint8 array."""
        p = make_params(tuple(x.shape), **kw)
        L = lib()
        bound = int(L.szgb_compress_bound(C.byref(p)))
        st = Stats()
        olen = C.c_size_t()
        if _is_torch(x):
            import torch
            _require_cuda(x, torch.float32, "x", self.device)
            if out is None:
                out = torch.empty(bound, dtype=torch.uint8, device=x.device)
            _require_cuda(out, torch.uint8, "out", self.device)
            rc = L.szgb_compress(self._h, C.c_void_p(x.data_ptr()), 1, C.byref(p),
                                 C.c_void_p(out.data_ptr()), out.numel(), 1, C.byref(olen), C.byref(st))
            if rc:
                raise SzgbError(rc, "szgb_compress")
            return out[:olen.value], st
        xa = np.ascontiguousarray(x, dtype=np.float32)
        if out is None:
            out = np.empty(bound, np.uint8)
        _require_host(out, np.uint8, "out")
        rc = L.szgb_compress(self._h, C.c_void_p(xa.ctypes.data), 0, C.byref(p),
                             C.c_void_p(out.ctypes.data), out.size, 0, C.byref(olen), C.byref(st))
        if rc:
            raise SzgbError(rc, "szgb_compress")
        return out[:olen.value], st

    def compress_host_ptr(self, x_ptr: int, shape, out_ptr: int, out_cap: int, **kw):
        """Compress from a host pointer into a host buffer (pinned or pageable)."""
        p = make_params(shape, **kw)
        st = Stats()
        olen = C.c_size_t()
        rc = lib().szgb_compress(self._h, C.c_void_p(x_ptr), 0, C.byref(p), C.c_void_p(out_ptr),
                                 int(out_cap), 0, C.byref(olen), C.byref(st))
        if rc:
            raise SzgbError(rc, "szgb_compress")
        return olen.value, st

    def compress_trace(self, x, **kw):
        """Device-only compression that also returns the recorded (exact
        decompressed) values and the quantization codes, for testing."""
        import torch
        _require_cuda(x, torch.float32, "x", self.device)
        p = make_params(tuple(x.shape), **kw)
        L = lib()
        bound = int(L.szgb_compress_bound(C.byref(p)))
        out = torch.empty(bound, dtype=torch.uint8, device=x.device)
        rec = torch.empty_like(x)
        codes = torch.empty(x.shape, dtype=torch.int16, device=x.device)
        if x.dim() == 4:
            s_, st = self._compress_4d(x, p, out, rec, codes)
            return s_, rec, codes, st
        st = Stats()
        olen = C.c_size_t()
        rc = L.szgb_compress_trace(self._h, C.c_void_p(x.data_ptr()), C.byref(p),
                                   C.c_void_p(out.data_ptr()), out.numel(), C.byref(olen),
                                   C.byref(st), C.c_void_p(rec.data_ptr()),
                                   C.c_void_p(codes.data_ptr()))
        if rc:
            raise SzgbError(rc, "szgb_compress_trace")
        return out[:olen.value], rec, codes, st

    def _compress_4d(self, x, p, out, rec, codes):
        """szgb_compress_4d on the CUDA tensor x (4 dimensions)."""
        shp = (C.c_uint64 * 4)(*[int(a) for a in x.shape])
        st = Stats()
        olen = C.c_size_t()
        rc = lib().szgb_compress_4d(self._h, C.c_void_p(x.data_ptr()), shp, C.byref(p), C.c_void_p(out.data_ptr()),
                                    out.numel(), C.byref(olen), C.byref(st),
                                    C.c_void_p(rec.data_ptr()) if rec is not None else None,
                                    C.c_void_p(codes.data_ptr()) if codes is not None else None)
        if rc:
            raise SzgbError(rc, "szgb_compress_4d")
        return out[:olen.value], st

    # -- decompression -------------------------------------------------------
    def decompress(self, stream, out=None, shape=None):
        """Decompress a stream (uint8 CUDA tensor or NumPy array).  Returns a
        float32 CUDA tensor (CUDA stream input) or NumPy array."""
        L = lib()
        if _is_torch(stream):
            import torch
            _require_cuda(stream, torch.uint8, "stream", self.device)
            if out is None:  # the shape is in the header (one small device-to-host read)
                info = stream_info_header(stream[:128].cpu().numpy())
                out = torch.empty(info["shape"], dtype=torch.float32, device=stream.device)
            _require_cuda(out, torch.float32, "out", self.device)
            rc = L.szgb_decompress(self._h, C.c_void_p(stream.data_ptr()), stream.numel(), 1,
                                   C.c_void_p(out.data_ptr()), out.numel(), 1)
            if rc:
                raise SzgbError(rc, "szgb_decompress")
            return out
        s = np.ascontiguousarray(np.asarray(stream, dtype=np.uint8))
        info = stream_info_header(s[:128])
        if out is None:
            out = np.empty(info["shape"], np.float32)
        _require_host(out, np.float32, "out")
        rc = L.szgb_decompress(self._h, C.c_void_p(s.ctypes.data), s.size, 0,
                               C.c_void_p(out.ctypes.data), out.size, 0)
        if rc:
            raise SzgbError(rc, "szgb_decompress")
        return out

    # -- autotuner -----------------------------------------------------------
    def autotune(self, x, reps: int = 2, **kw) -> dict:
        """Pick the wavefront shape for the shape class of the CUDA tensor `x`."""
        import torch
        _require_cuda(x, torch.float32, "x", self.device)
        p = make_params(tuple(x.shape), **kw)
        W, ch, ms = C.c_int(), C.c_int(), C.c_double()
        rc = lib().szgb_autotune(self._h, C.c_void_p(x.data_ptr()), C.byref(p), int(reps), C.byref(W),
                                 C.byref(ch), C.byref(ms))
        if rc:
            raise SzgbError(rc, "szgb_autotune")
        return {"W": W.value, "chunk": ch.value & 0xFFFFFFFF, "ms": ms.value}

    def autotune_batch(self, xs, params, reps: int = 1) -> dict:
        """Pick one wavefront shape for the batch of CUDA tensors `xs`
        (timed as batched passes) and keep it for every shape class in it."""
        import torch
        n = len(xs)
        if isinstance(params, dict):
            params = [params] * n
        P = (Params * n)()
        for i, (x, kw) in enumerate(zip(xs, params)):
            _require_cuda(x, torch.float32, "xs[%d]" % i, self.device)
            P[i] = make_params(tuple(x.shape), **kw)
        dp = (C.c_void_p * n)(*[x.data_ptr() for x in xs])
        W, ch, ms = C.c_int(), C.c_int(), C.c_double()
        rc = lib().szgb_autotune_batch(self._h, n, dp, P, int(reps), C.byref(W), C.byref(ch), C.byref(ms))
        if rc:
            raise SzgbError(rc, "szgb_autotune_batch")
        return {"W": W.value, "chunk": ch.value & 0xFFFFFFFF, "ms": ms.value}

    def tune_save(self, path: str):
        rc = lib().szgb_tune_save(self._h, path.encode())
        if rc:
            raise SzgbError(rc, "szgb_tune_save")

    def tune_load(self, path: str):
        rc = lib().szgb_tune_load(self._h, path.encode())
        if rc:
            raise SzgbError(rc, "szgb_tune_load")

    # -- batches -------------------------------------------------------------
    def set_graphs(self, on: bool):
        lib().szgb_set_graphs(self._h, 1 if on else 0)

    def set_wave_ctas(self, max_ctas: int):
        """Cap the persistent wavefront launches of this context at max_ctas
        CTAs (0 = one per SM), leaving the other SMs to other streams."""
        rc = lib().szgb_set_wave_ctas(self._h, int(max_ctas))
        if rc:
            raise SzgbError(rc, "szgb_set_wave_ctas")

    def debug_set_wait_limit(self, ns: int):
        """Test hook: limit of the device-side waits of later calls (0 = the
        default, 4 s)."""
        rc = lib().szgb_debug_set_wait_limit(self._h, int(ns))
        if rc:
            raise SzgbError(rc, "szgb_debug_set_wait_limit")

    def debug_skip_item(self, item: int):
        """Test hook: the wavefront work item `item` is never run (-1 = off),
        so the waits of its consumers run out and calls return ETIMEOUT."""
        rc = lib().szgb_debug_skip_item(self._h, int(item))
        if rc:
            raise SzgbError(rc, "szgb_debug_skip_item")

    def quality(self, x, y) -> dict:
        """Reconstruction quality of y against x (CUDA float32 tensors of one
        size): maximum absolute / range-relative error, RMSE, NRMSE, PSNR and
        Pearson's coefficient (Sec. II, Metrics 1-3), computed on the device."""
        import torch
        _require_cuda(x, torch.float32, "x", self.device)
        _require_cuda(y, torch.float32, "y", self.device)
        if x.numel() != y.numel():
            raise ValueError("x and y need the same number of values")
        q = Quality()
        rc = lib().szgb_quality_dev(self._h, C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()), x.numel(),
                                    C.byref(q))
        if rc:
            raise SzgbError(rc, "szgb_quality_dev")
        return q.as_dict()

    def hit_count(self, x, v, layers: int, eb: float) -> int:
        """Points of x whose n-layer prediction from the values v at the
        preceding neighbours lies within eb of x (Sec. III): v = x counts the
        hits behind R_PH^orig, v = the compressor's recorded values (see
        compress_trace) those behind R_PH^decomp.  CUDA float32 tensors of
        one shape, computed on the device."""
        import torch
        _require_cuda(x, torch.float32, "x", self.device)
        _require_cuda(v, torch.float32, "v", self.device)
        if tuple(x.shape) != tuple(v.shape) or not 1 <= x.dim() <= 4:
            raise ValueError("x and v need one 1D..4D shape")
        shp = (C.c_uint64 * max(1, x.dim()))(*[int(a) for a in x.shape])
        n = C.c_uint64()
        rc = lib().szgb_hit_count_dev(self._h, C.c_void_p(x.data_ptr()), C.c_void_p(v.data_ptr()), x.dim(), shp,
                                      int(layers), float(eb), C.byref(n))
        if rc:
            raise SzgbError(rc, "szgb_hit_count_dev")
        return int(n.value)

    def hit_rates(self, x, layers: int, **kw) -> dict:
        """R_PH^orig and R_PH^decomp of the CUDA float32 field x for the
        n-layer predictor under the bound in kw (Sec. III, Table 2): the
        second is taken from this compressor's own recorded values, with the
        effective float32 bound eb_f of the compression."""
        _, rec, _, st = self.compress_trace(x, layers=layers, **kw)
        N = x.numel()
        h_o = self.hit_count(x, x, layers, st.eb_f)
        h_d = self.hit_count(x, rec, layers, st.eb_f)
        return {"n": layers, "N": N, "eb_f": st.eb_f, "m": st.m, "hits_orig": h_o, "hits_decomp": h_d,
                "R_orig": h_o / N, "R_decomp": h_d / N}

    def compress_batch(self, xs, params, outs=None):
        """Compress the CUDA float32 tensors `xs` in one batched call.
        `params` is one dict of make_params keywords for all fields or a list
        of them.  `outs` (optional) are uint8 CUDA tensors to write into.
        Returns (streams, stats): views of the output tensors and a list of
        Stats."""
        import torch
        n = len(xs)
        if isinstance(params, dict):
            params = [params] * n
        P = (Params * n)()
        for i, (x, kw) in enumerate(zip(xs, params)):
            _require_cuda(x, torch.float32, "xs[%d]" % i, self.device)
            P[i] = make_params(tuple(x.shape), **kw)
        L = lib()
        if outs is None:
            outs = [torch.empty(int(L.szgb_compress_bound(C.byref(P[i]))), dtype=torch.uint8, device=xs[i].device)
                    for i in range(n)]
        if len(outs) != n:
            raise ValueError("one output per field")
        for i, o in enumerate(outs):
            _require_cuda(o, torch.uint8, "outs[%d]" % i, self.device)
        dp = (C.c_void_p * n)(*[x.data_ptr() for x in xs])
        op = (C.c_void_p * n)(*[o.data_ptr() for o in outs])
        cap = (C.c_size_t * n)(*[o.numel() for o in outs])
        olen = (C.c_size_t * n)()
        st = (Stats * n)()
        rc = L.szgb_compress_batch(self._h, n, dp, P, op, cap, olen, st)
        if rc:
            raise SzgbError(rc, "szgb_compress_batch")
        return [outs[i][:olen[i]] for i in range(n)], [st[i] for i in range(n)]

    def decompress_batch(self, streams, outs=None):
        """Decompress the uint8 CUDA tensors `streams` in one batched call into
        float32 CUDA tensors (allocated from the headers when `outs` is None)."""
        import torch
        n = len(streams)
        for i, s in enumerate(streams):
            _require_cuda(s, torch.uint8, "streams[%d]" % i, self.device)
        if outs is None:
            outs = []
            for s in streams:
                info = stream_info_header(s[:128].cpu().numpy())
                outs.append(torch.empty(info["shape"], dtype=torch.float32, device=s.device))
        if len(outs) != n:
            raise ValueError("one output per stream")
        for i, o in enumerate(outs):
            _require_cuda(o, torch.float32, "outs[%d]" % i, self.device)
        ip = (C.c_void_p * n)(*[s.data_ptr() for s in streams])
        il = (C.c_size_t * n)(*[s.numel() for s in streams])
        op = (C.c_void_p * n)(*[o.data_ptr() for o in outs])
        oc = (C.c_size_t * n)(*[o.numel() for o in outs])
        rc = lib().szgb_decompress_batch(self._h, n, ip, il, op, oc, None)
        if rc:
            raise SzgbError(rc, "szgb_decompress_batch")
        return outs

    def decompress_ptr(self, in_ptr: int, in_len: int, in_on_device: bool, out_ptr: int,
                       out_elems: int, out_on_device: bool) -> int:
        return lib().szgb_decompress(self._h, C.c_void_p(in_ptr), int(in_len), int(in_on_device),
                                     C.c_void_p(out_ptr), int(out_elems), int(out_on_device))


def stream_info_header(hdr) -> dict:
    """Shape and parameters from the 128-byte header alone (no length check)."""
    import struct
    b = bytes(np.asarray(hdr[:128], dtype=np.uint8))
    ndim = b[8]
    d = struct.unpack_from("<3Q", b, 16)
    if ndim == 4:  # a 4D field keeps its slowest extent at byte 120
        shape = (int(struct.unpack_from("<Q", b, 120)[0]),) + tuple(int(v) for v in d)
    else:
        shape = tuple(int(v) for v in d[3 - ndim:])
    return {"ndim": ndim, "shape": shape, "m": b[10], "layers": b[9]}


def decompress_noalloc(stream, out, cuda_stream: int = 0) -> int:
    """szgb_decompress_noalloc on a uint8 CUDA tensor `stream` into the
    float32 CUDA tensor `out`; returns the C status code.  No memory is
    allocated by the library (the caller provides `out`).  `stream` and `out`
    must be on the same device; the call runs with that device current, and
    `cuda_stream` (a cudaStream_t handle, 0 = the legacy default stream) must
    belong to it."""
    import torch
    _require_cuda(stream, torch.uint8, "stream")
    _require_cuda(out, torch.float32, "out")
    if stream.device != out.device:
        raise ValueError("stream is on %s but out is on %s" % (stream.device, out.device))
    with torch.cuda.device(stream.device):
        return lib().szgb_decompress_noalloc(C.c_void_p(stream.data_ptr()), stream.numel(),
                                             C.c_void_p(out.data_ptr()), out.numel(),
                                             C.c_void_p(cuda_stream or 0))


class Server:
    """The serving loop (szgb_server_*): host buffers in, host buffers out.
    The buffers of a request are kept referenced here until it is done.

    With `log_path`, one JSON line per completed request is appended there:
    ticket, op, shape, input and output bytes, status, latency from submit
    to the completion seen by poll/wait, and for a compressed stream its
    compression factor, bit-rate (Sec. II, Metric 4), m and unpredictable
    count from the stream header."""

    def __init__(self, device: int = 0, budget: int = 100 << 30, workers: int = 2, max_batch: int = 64,
                 log_path: str | None = None):
        self._h = C.c_void_p()
        self._keep = {}
        self._meta = {}
        self._log = None
        rc = lib().szgb_server_create(C.byref(self._h), int(device), int(budget), int(workers), int(max_batch))
        if rc:
            raise SzgbError(rc, "szgb_server_create")
        if log_path:
            self._log = open(log_path, "a")

    def close(self):
        if self._h:
            lib().szgb_server_destroy(self._h)
            self._h = C.c_void_p()
            self._keep.clear()
            self._meta.clear()
        if self._log is not None:
            self._log.close()
            self._log = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _submit(self, req, keep, meta):
        t = C.c_uint64()
        t0 = time.perf_counter()
        rc = lib().szgb_submit(self._h, C.byref(req), C.byref(t))
        if rc:
            raise SzgbError(rc, "szgb_submit")
        self._keep[t.value] = keep
        meta["t0"] = t0
        self._meta[t.value] = meta
        return t.value

    def _finish(self, ticket: int, status: int, out_len: int):
        keep = self._keep.pop(ticket, None)
        meta = self._meta.pop(ticket, None)
        if self._log is None or meta is None:
            return
        rec = {"ticket": ticket, "op": meta["op"], "shape": meta["shape"], "in_bytes": meta["in_bytes"],
               "out_bytes": int(out_len), "status": int(status),
               "latency_s": time.perf_counter() - meta["t0"]}
        if status == OK and meta["op"] == "compress" and out_len >= 128:
            n = int(np.prod(meta["shape"], dtype=np.int64))
            hdr = stream_info_header(keep[1][:128])
            rec.update(compression_factor=meta["in_bytes"] / out_len, bit_rate=8.0 * out_len / n,
                       m=int(hdr["m"]), n_unpred=int(np.frombuffer(bytes(keep[1][80:88]), "<u8")[0]))
        self._log.write(json.dumps(rec) + "\n")
        self._log.flush()

    def submit_compress(self, x: np.ndarray, out: np.ndarray, **kw) -> int:
        """Queue compression of the host float32 array `x` into the host uint8
        array `out`; returns the ticket."""
        _require_host(x, np.float32, "x")
        _require_host(out, np.uint8, "out")
        r = Request()
        r.op = OP_COMPRESS
        r.in_ = x.ctypes.data
        r.in_bytes = x.nbytes
        r.params = make_params(x.shape, **kw)
        r.out = out.ctypes.data
        r.out_cap = out.nbytes
        return self._submit(r, (x, out), {"op": "compress", "shape": list(x.shape), "in_bytes": x.nbytes})

    def submit_decompress(self, stream: np.ndarray, out: np.ndarray) -> int:
        """Queue decompression of the host stream into the host float32 array `out`."""
        _require_host(stream, np.uint8, "stream")
        _require_host(out, np.float32, "out")
        r = Request()
        r.op = OP_DECOMPRESS
        r.in_ = stream.ctypes.data
        r.in_bytes = stream.nbytes
        r.out = out.ctypes.data
        r.out_cap = out.nbytes
        return self._submit(r, (stream, out), {"op": "decompress", "shape": list(out.shape),
                                                "in_bytes": stream.nbytes})

    def poll(self, ticket: int):
        """(done, status, out_len); status and out_len are None until done."""
        d, st, n = C.c_int(), C.c_int(), C.c_size_t()
        rc = lib().szgb_poll(self._h, C.c_uint64(ticket), C.byref(d), C.byref(st), C.byref(n))
        if rc:
            raise SzgbError(rc, "szgb_poll")
        if d.value:
            self._finish(ticket, st.value, n.value)
            return True, st.value, n.value
        return False, None, None

    def wait(self, ticket: int):
        """(status, out_len) once the request is done."""
        st, n = C.c_int(), C.c_size_t()
        rc = lib().szgb_wait(self._h, C.c_uint64(ticket), C.byref(st), C.byref(n))
        if rc:
            raise SzgbError(rc, "szgb_wait")
        self._finish(ticket, st.value, n.value)
        return st.value, n.value

    def stats(self) -> dict:
        b, c_, p = C.c_uint64(), C.c_uint64(), C.c_size_t()
        lib().szgb_server_stats(self._h, C.byref(b), C.byref(c_), C.byref(p))
        return {"batches": b.value, "completed": c_.value, "peak_reserved": p.value}
