"""Pins of the oracle's chunked Huffman payload (the chunk size is this
build's choice: the paper codes one stream, Sec. IV-A; rows are cut into
chunks so that they can be coded and decoded in parallel).

The format: every row of N points is cut into chunks of C points (a power of
two >= 32; the last chunk of a row is shorter), chunks follow row by row,
each is its own MSB-first bit string padded to a byte, the chunk table holds
their byte lengths and header byte 116 holds C (0: one chunk per row).

Checked against things the oracle's writer does not compute the same way:
  * a plain Python bit reader decodes every chunk on its own, with the
    canonical code rebuilt from the codebook section, and must give exactly
    the quantization codes of that chunk's points (pins which points a chunk
    holds and that each chunk starts on its own byte);
  * C at least the row length gives the byte-identical whole-row stream;
  * table length, payload size and header fields follow from the definition;
  * the round trip is bit-exact at every chunk size, ragged last chunks
    included, in 1D-4D;
  * sizes that are not a power of two >= 32 are rejected, and so is a stream
    whose chunk field is inconsistent."""
import struct

import numpy as np
import pytest

from synthetic import fields


def _canonical(lens):
    """symbol -> (code, length) from a {symbol: length} map, by the canonical
    rule: symbols in (length, symbol) order take consecutive codes, shifted
    left whenever the length grows."""
    out, code, prev = {}, 0, None
    for s in sorted(lens, key=lambda s: (lens[s], s)):
        L = lens[s]
        code = 0 if prev is None else (code + 1) << (L - prev)
        prev = L
        out[s] = (code, L)
    return out


def _decode_chunk(buf, npts, decode, e_eb):
    """Codes of npts points from one chunk's bytes (MSB first); after a code
    0 skip its 9 + t record bits (t from the stored exponent)."""
    bits = "".join(format(b, "08b") for b in buf)
    pos, codes = 0, []
    for _ in range(npts):
        c = ""
        while c not in decode:
            c += bits[pos]
            pos += 1
            assert len(c) <= 64
        sym = decode[c]
        codes.append(sym)
        if sym == 0:
            ex = int(bits[pos + 1:pos + 9], 2)
            t = 23 if e_eb == 0 else min(23, max(0, max(ex, 1) - e_eb))
            pos += 9 + t
    # only padding after the last point, less than a byte
    assert len(bits) - pos < 8 and set(bits[pos:]) <= {"0"}
    return codes


def _sections(s):
    h = bytes(s[:128])
    nsym, = struct.unpack_from("<I", h, 68)
    nch, = struct.unpack_from("<Q", h, 72)
    tw = h[13]
    cb = 128
    lens = {}
    for e in range(nsym):
        sym, = struct.unpack_from("<H", bytes(s[cb + 3 * e:cb + 3 * e + 2]))
        lens[sym] = int(s[cb + 3 * e + 2])
    tb = cb + ((3 * nsym + 3) & ~3)
    table = [int.from_bytes(bytes(s[tb + tw * i:tb + tw * i + tw]), "little") for i in range(nch)]
    pl = tb + ((tw * nch + 3) & ~3)
    return lens, table, pl


@pytest.mark.parametrize("C", [32, 64, 128])
def test_each_chunk_decodes_to_its_points(szo, C):
    x = fields.grf2d(6, 150, seed=40)  # rows of 150: chunks 150 = 4*32 + 22, 2*64 + 22, 128 + 22
    kw = dict(eb_rel=1e-5, m=0)  # a tight bound: some unpredictable points
    s, rec, codes = szo.compress(x, want_aux=True, chunk_points=C, **kw)
    h = szo.header(s)
    assert h["chunk_points"] == C
    lens, table, pl = _sections(s)
    decode = {format(c, "0%db" % L): sym for sym, (c, L) in _canonical(lens).items()}
    e_eb = (struct.unpack("<I", struct.pack("<f", h["eb_f"]))[0] >> 23) & 0xFF
    nseg = -(-x.shape[1] // C)
    assert len(table) == x.shape[0] * nseg == h["nchunks"]
    assert sum(table) == h["payload_bytes"] and h["total_bytes"] == s.size
    off = pl
    for ch, nb in enumerate(table):
        r, sg = divmod(ch, nseg)
        l0, l1 = sg * C, min(x.shape[1], (sg + 1) * C)
        got = _decode_chunk(s[off:off + nb], l1 - l0, decode, e_eb)
        assert got == codes[r, l0:l1].tolist(), "chunk %d" % ch
        off += nb
    assert off == s.size
    assert (codes == 0).any()


CASES = [
    ("1d", lambda: fields.grf2d(1, 1000, seed=41).reshape(1000), dict(eb_rel=1e-4, m=0)),
    ("2d-n2", lambda: fields.grf2d(23, 211, seed=42), dict(eb_rel=1e-4, n=2, m=0)),
    ("3d", lambda: fields.blobs3d(5, 9, 97, seed=43, nblobs=3), dict(eb_rel=1e-5, m=0)),
    ("4d", lambda: fields.blobs3d(6, 8, 70, seed=44, nblobs=3).reshape(2, 3, 8, 70), dict(eb_rel=1e-4, m=8)),
]


@pytest.mark.parametrize("name,gen,kw", CASES, ids=[c[0] for c in CASES])
def test_round_trip_every_chunk_size(szo, name, gen, kw):
    x = np.ascontiguousarray(gen())
    N = x.shape[-1]
    s0, rec0, codes0 = szo.compress(x, want_aux=True, **kw)
    for C in (32, 64, 128, 256, 512, 1024, 2048):
        s, rec, codes = szo.compress(x, want_aux=True, chunk_points=C, **kw)
        # the chunking changes only the coding of the codes
        assert np.array_equal(rec.view(np.uint32), rec0.view(np.uint32)) and np.array_equal(codes, codes0)
        y = szo.decompress(s)
        assert np.array_equal(y.view(np.uint32), rec0.view(np.uint32)), C
        h = szo.header(s)
        if C >= N:  # one chunk per row: the whole-row stream itself
            assert np.array_equal(s, s0) and h["chunk_points"] == 0
        else:
            assert h["chunk_points"] == C
            assert h["nchunks"] == (x.size // N) * (-(-N // C))
            # a chunk boundary costs at most a table entry and a pad byte
            assert s0.size <= s.size <= s0.size + 5 * h["nchunks"] + 4


def test_invalid_chunk_sizes(szo):
    x = fields.grf2d(8, 100, seed=45)
    for C in (1, 16, 48, 100, 33):
        assert szo.compress_rc(x, eb_rel=1e-3, m=8, chunk_points=C) == szo.EINVAL
    assert szo.compress_rc(x, eb_rel=1e-3, m=8, chunk_points=64) == 0


def test_inconsistent_chunk_field_rejected(szo):
    x = fields.grf2d(8, 100, seed=46)
    s = szo.compress(x, eb_rel=1e-3, m=8, chunk_points=32)
    for v in (48, 16, 128, 0):  # not a power of two, below 32, >= the row, or the table no longer fits
        bad = s.copy()
        bad[116:120] = np.frombuffer(struct.pack("<I", v), np.uint8)
        assert szo.decompress_rc(bad) == szo.ECORRUPT, v
