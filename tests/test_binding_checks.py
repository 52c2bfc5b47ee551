"""The Python binding rejects buffers the library cannot take (host tensors
where device memory is required, wrong dtypes, strided arrays) before any
pointer reaches the C library.  No GPU needed: the checks run first."""
import numpy as np
import pytest
import torch

from paper_1706_03791_gb300 import build

build.build()
from paper_1706_03791_gb300 import szgb  # noqa: E402


@pytest.fixture()
def ctx():
    c = szgb.Context.__new__(szgb.Context)  # no device context: only the checks run
    c._h = None
    c.device = 0
    return c


def test_device_calls_reject_host_tensors(ctx):
    x = torch.zeros(8, 8)
    with pytest.raises(TypeError):
        ctx.compress(x, eb_rel=1e-3)
    with pytest.raises(TypeError):
        ctx.compress_trace(x, eb_rel=1e-3)
    with pytest.raises(TypeError):
        ctx.decompress(torch.zeros(200, dtype=torch.uint8))
    with pytest.raises(TypeError):
        ctx.quality(x, x)
    with pytest.raises(TypeError):
        ctx.hit_count(x, x, 1, 0.1)
    with pytest.raises(TypeError):
        ctx.compress_batch([x], dict(eb_rel=1e-3))
    with pytest.raises(TypeError):
        ctx.decompress_batch([torch.zeros(200, dtype=torch.uint8)])
    with pytest.raises(TypeError):
        ctx.autotune(x, eb_rel=1e-3)
    with pytest.raises(TypeError):
        szgb.decompress_noalloc(torch.zeros(200, dtype=torch.uint8), x)


def test_4d_params(ctx):
    p = szgb.make_params((2, 3, 4, 5), eb_rel=1e-3)
    assert p.ndim == 4 and tuple(p.shape) == (2, 3, 4, 5)
    with pytest.raises(TypeError):  # a CPU tensor is neither a CUDA tensor nor a NumPy array
        ctx.compress(torch.zeros(2, 3, 4, 5), eb_rel=1e-3)
    # the 4D bound is the bound of the (D P) x M x N view
    assert szgb.compress_bound((2, 3, 4, 5), eb_rel=1e-3) == szgb.compress_bound((6, 4, 5), eb_rel=1e-3) > 0
    # extents: each 1..2^32-1, D x P below 2^32, the lattice variant not in 4D
    assert szgb.compress_bound((2, 0, 4, 5), eb_rel=1e-3) == 0
    assert szgb.compress_bound((1 << 16, 1 << 16, 1, 1), eb_rel=1e-3) == 0


def test_4d_header_shape():
    from oracle import szo
    x = np.random.default_rng(3).normal(size=(2, 3, 4, 5)).astype(np.float32)
    s = szo.compress(x, eb_rel=1e-3, m=8)
    info = szgb.stream_info_header(s[:128])
    assert info["ndim"] == 4 and info["shape"] == x.shape
    # the library's own header parser describes the 4D field as such
    full = szgb.stream_info(s)
    assert full["ndim"] == 4 and full["shape"] == x.shape and full["layers"] == 1 and full["m"] == 8


def test_host_outputs_checked(ctx):
    x = np.zeros((8, 8), np.float32)
    with pytest.raises(TypeError):
        ctx.compress(x, out=np.zeros(4096, np.int8), eb_rel=1e-3)
    with pytest.raises(ValueError):
        ctx.compress(x, out=np.zeros(8192, np.uint8)[::2], eb_rel=1e-3)
    stream = np.zeros(256, np.uint8)
    stream[8] = 2
    stream[16] = 8
    stream[24] = 8
    with pytest.raises(TypeError):
        ctx.decompress(stream, out=np.zeros((8, 8), np.float16))


def test_server_requests_checked():
    srv = szgb.Server.__new__(szgb.Server)
    srv._h = None
    srv._keep = {}
    x = np.zeros((16, 16), np.float32)
    out = np.zeros(4096, np.uint8)
    with pytest.raises(TypeError):
        srv.submit_compress(x.astype(np.float64), out, eb_rel=1e-3)
    with pytest.raises(ValueError):
        srv.submit_compress(x[:, ::2], out, eb_rel=1e-3)
    with pytest.raises(ValueError):
        srv.submit_decompress(out[::2], np.zeros(256, np.float32))
    with pytest.raises(TypeError):
        srv.submit_decompress(out, np.zeros(256, np.float64))
