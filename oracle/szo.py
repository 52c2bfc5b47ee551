"""ctypes binding of the C oracle (oracle/szo.c).

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the
benchmark's CPU baseline.  ``build()`` compiles ``libszo.so`` next to this
file with ``-O2 -ffp-contract=off`` (no FMA contraction, IEEE float order as
written), which the oracle's bit-exact definition relies on.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = os.path.join(_HERE, "libszo.so")
_SRC = os.path.join(_HERE, "szo.c")
_lib = None

OK, EINVAL, ENONFINITE, ETRUNC, ECORRUPT, ENOMEM = 0, -1, -2, -3, -4, -5
ABS, REL, ABS_AND_REL = 0, 1, 2


def build(force: bool = False) -> str:
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11",
                               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        u64p = C.POINTER(C.c_uint64)
        L.szo_num_terms.argtypes = [C.c_int, C.c_int]
        L.szo_terms.argtypes = [C.c_int, C.c_int, C.c_void_p, C.c_void_p]
        L.szo_terms4.argtypes = [C.c_int, C.c_int, C.c_void_p, C.c_void_p]
        L.szo_predict_field.argtypes = [C.c_void_p, C.c_int, u64p, C.c_int, C.c_void_p]
        L.szo_effective_eb.argtypes = [C.c_int, C.c_double, C.c_double, C.c_float, C.c_float,
                                       C.POINTER(C.c_float)]
        L.szo_effective_eb.restype = C.c_double
        L.szo_quantize.argtypes = [C.c_float, C.c_float, C.c_float, C.c_int, C.POINTER(C.c_float)]
        L.szo_truncate.argtypes = [C.c_float, C.c_float, C.POINTER(C.c_float)]
        L.szo_huffman_lengths.argtypes = [C.c_void_p, C.c_int, C.c_void_p]
        L.szo_canonical_codes.argtypes = [C.c_void_p, C.c_int, C.c_void_p]
        L.szo_choose_m.argtypes = [C.c_void_p, C.c_int, u64p, C.c_int, C.c_float, C.c_double]
        L.szo_stream_bound.argtypes = [C.c_int, u64p]
        L.szo_stream_bound.restype = C.c_size_t
        L.szo_compress.argtypes = [C.c_void_p, C.c_int, u64p, C.c_int, C.c_double, C.c_double,
                                   C.c_int, C.c_int, C.c_double, C.c_int, C.c_void_p, C.c_size_t,
                                   C.POINTER(C.c_size_t), C.c_void_p, C.c_void_p]
        L.szo_compress_chunked.argtypes = [C.c_void_p, C.c_int, u64p, C.c_int, C.c_double, C.c_double,
                                           C.c_int, C.c_int, C.c_double, C.c_int, C.c_uint32, C.c_void_p,
                                           C.c_size_t, C.POINTER(C.c_size_t), C.c_void_p, C.c_void_p]
        L.szo_decompress.argtypes = [C.c_void_p, C.c_size_t, C.c_void_p, C.c_size_t]
        L.szo_lattice_point.argtypes = [C.c_float, C.c_float, C.POINTER(C.c_int)]
        L.szo_lattice_point.restype = C.c_int64
        L.szo_lattice_value.argtypes = [C.c_int64, C.c_float]
        L.szo_lattice_value.restype = C.c_float
        L.szo_choose_m_lattice.argtypes = [C.c_void_p, C.c_int, u64p, C.c_int, C.c_float, C.c_double]
        L.szo_compress_lattice.argtypes = [C.c_void_p, C.c_int, u64p, C.c_int, C.c_double, C.c_double,
                                           C.c_int, C.c_int, C.c_double, C.c_void_p, C.c_size_t,
                                           C.POINTER(C.c_size_t), C.c_void_p, C.c_void_p]
        _lib = L
    return _lib


def _shape(a):
    if not 1 <= a.ndim <= 4:
        raise ValueError("1D..4D fields only")
    return (C.c_uint64 * 4)(*[int(s) for s in a.shape] + [1] * (4 - a.ndim))


def terms(ndim: int, n: int):
    """(k offsets [T, max(3, ndim)], integer coefficients [T]) in summation
    order; offsets have leading zeros for the absent axes."""
    T = lib().szo_num_terms(ndim, n)
    c = np.zeros(T, np.int64)
    if ndim <= 3:
        k = np.zeros((T, 3), np.int32)
        lib().szo_terms(ndim, n, k.ctypes.data, c.ctypes.data)
    else:
        k = np.zeros((T, 4), np.int32)
        lib().szo_terms4(ndim, n, k.ctypes.data, c.ctypes.data)
    return k, c


def predict_field(V: np.ndarray, n: int) -> np.ndarray:
    V = np.ascontiguousarray(V, dtype=np.float32)
    out = np.empty_like(V)
    rc = lib().szo_predict_field(V.ctypes.data, V.ndim, _shape(V), n, out.ctypes.data)
    assert rc == 0
    return out


def effective_eb(mode, eb_abs, eb_rel, xmin, xmax):
    f = C.c_float()
    e = lib().szo_effective_eb(mode, eb_abs, eb_rel, xmin, xmax, C.byref(f))
    return e, f.value


def quantize(x, pred, eb_f, m):
    r = C.c_float()
    code = lib().szo_quantize(x, pred, eb_f, m, C.byref(r))
    return code, r.value


def truncate(x, eb_f):
    r = C.c_float()
    t = lib().szo_truncate(x, eb_f, C.byref(r))
    return t, r.value


def huffman_lengths(freq) -> np.ndarray:
    f = np.ascontiguousarray(freq, dtype=np.uint64)
    ln = np.zeros(f.size, np.uint8)
    rc = lib().szo_huffman_lengths(f.ctypes.data, f.size, ln.ctypes.data)
    assert rc >= 0
    return ln


def canonical_codes(lens) -> np.ndarray:
    ln = np.ascontiguousarray(lens, dtype=np.uint8)
    c = np.zeros(ln.size, np.uint64)
    lib().szo_canonical_codes(ln.ctypes.data, ln.size, c.ctypes.data)
    return c


def choose_m(x, n, eb_f, theta=0.99):
    x = np.ascontiguousarray(x, dtype=np.float32)
    return lib().szo_choose_m(x.ctypes.data, x.ndim, _shape(x), n, eb_f, theta)


def compress(x, mode=REL, eb_abs=0.0, eb_rel=1e-4, n=1, m=0, theta=0.99, order=0,
             want_aux=False, layers=None, chunk_points=0):
    """Returns the stream bytes (and, with want_aux, the recorded values and
    the quantization codes).  `layers` is an alias of n.  `chunk_points`
    cuts every row's Huffman payload into chunks of that many points (a
    power of two >= 32; 0: one chunk per row)."""
    if layers is not None:
        n = layers
    x = np.ascontiguousarray(x, dtype=np.float32)
    L = lib()
    cap = L.szo_stream_bound(x.ndim, _shape(x))
    out = np.zeros(cap, np.uint8)
    olen = C.c_size_t()
    rec = np.empty_like(x) if want_aux else None
    codes = np.empty(x.shape, np.uint16) if want_aux else None
    rc = L.szo_compress_chunked(x.ctypes.data, x.ndim, _shape(x), mode, eb_abs, eb_rel, n, m, theta,
                                order, int(chunk_points), out.ctypes.data, cap, C.byref(olen),
                                rec.ctypes.data if want_aux else None,
                                codes.ctypes.data if want_aux else None)
    if rc != 0:
        raise RuntimeError("szo_compress failed: %d" % rc)
    s = out[:olen.value].copy()
    return (s, rec, codes) if want_aux else s


def lattice_point(x, eb_f):
    """(p, ok): the lattice integer of x and whether its lattice value is
    within the bound (the lattice variant)."""
    ok = C.c_int()
    p = lib().szo_lattice_point(x, eb_f, C.byref(ok))
    return p, bool(ok.value)


def lattice_value(p, eb_f):
    return lib().szo_lattice_value(int(p), eb_f)


def choose_m_lattice(x, n, eb_f, theta=0.99):
    x = np.ascontiguousarray(x, dtype=np.float32)
    return lib().szo_choose_m_lattice(x.ctypes.data, x.ndim, _shape(x), n, eb_f, theta)


def compress_lattice(x, mode=REL, eb_abs=0.0, eb_rel=1e-4, n=1, m=0, theta=0.99, want_aux=False,
                     layers=None):
    """The lattice variant (not the paper's method; labelled separately).
    Returns the stream (and, with want_aux, the reconstructed values and the
    codes)."""
    if layers is not None:
        n = layers
    x = np.ascontiguousarray(x, dtype=np.float32)
    L = lib()
    cap = L.szo_stream_bound(x.ndim, _shape(x)) + 11 * x.size + 64
    out = np.zeros(cap, np.uint8)
    olen = C.c_size_t()
    rec = np.empty_like(x) if want_aux else None
    codes = np.empty(x.shape, np.uint16) if want_aux else None
    rc = L.szo_compress_lattice(x.ctypes.data, x.ndim, _shape(x), mode, eb_abs, eb_rel, n, m, theta,
                                out.ctypes.data, cap, C.byref(olen),
                                rec.ctypes.data if want_aux else None,
                                codes.ctypes.data if want_aux else None)
    if rc != 0:
        raise RuntimeError("szo_compress_lattice failed: %d" % rc)
    s = out[:olen.value].copy()
    return (s, rec, codes) if want_aux else s


def compress_rc(x, **kw):
    try:
        compress(x, **kw)
        return 0
    except RuntimeError as e:
        return int(str(e).split(":")[-1])


def decompress(stream, shape=None):
    s = np.ascontiguousarray(stream, dtype=np.uint8)
    hdr = header(s)
    dims = hdr["dims"]
    N = int(np.prod(dims, dtype=np.uint64))
    out = np.empty(N, np.float32)
    rc = lib().szo_decompress(s.ctypes.data, s.size, out.ctypes.data, N)
    if rc != 0:
        raise RuntimeError("szo_decompress failed: %d" % rc)
    return out.reshape(dims)


def decompress_rc(stream):
    s = np.ascontiguousarray(stream, dtype=np.uint8)
    out = np.empty(max(1, 1 << 20), np.float32)
    try:
        hdr = header(s)
        N = int(np.prod(hdr["dims"], dtype=np.uint64))
        if N > out.size:
            out = np.empty(N, np.float32)
    except Exception:
        pass
    return lib().szo_decompress(s.ctypes.data, s.size, out.ctypes.data, out.size)


def header(s):
    """Parse the fixed 128-byte header (little-endian)."""
    b = bytes(np.asarray(s[:128], dtype=np.uint8))
    import struct
    if len(b) < 128:
        raise ValueError("short stream")
    f = {}
    f["magic"] = b[0:4]
    f["version"], f["header_bytes"] = struct.unpack_from("<HH", b, 4)
    f["ndim"], f["layers"], f["m"], f["mode"], f["maxlen"], f["table_width"] = b[8], b[9], b[10], b[11], b[12], b[13]
    f["shape"] = struct.unpack_from("<3Q", b, 16)
    f["eb_abs"], f["eb_rel"] = struct.unpack_from("<2d", b, 40)
    f["eb_f"], f["xmin"], f["xmax"] = struct.unpack_from("<3f", b, 56)
    f["nsym"], = struct.unpack_from("<I", b, 68)
    f["nchunks"], f["K"], f["payload_bytes"], f["total_bytes"] = struct.unpack_from("<4Q", b, 72)
    f["theta"], = struct.unpack_from("<d", b, 104)
    f["adaptive"] = b[112]
    f["lattice"] = b[113]
    f["chunk_points"], = struct.unpack_from("<I", b, 116)  # 0: one chunk per row
    # all four extents (a 4D field keeps its slowest one at byte 120) and the
    # field's own shape
    d0, = struct.unpack_from("<Q", b, 120)
    f["shape4"] = ((d0 if f["ndim"] == 4 else 1),) + tuple(f["shape"])
    f["dims"] = tuple(int(v) for v in f["shape4"][4 - f["ndim"]:]) if 1 <= f["ndim"] <= 4 else ()
    return f
