"""Format variant R4c (LUDA_F_COMPRESS): data blocks stored in the Snappy stream format
when that saves an eighth of their bytes. The oracle's decoder is checked against streams
worked out by hand from the published format and against an independent pure-Python
decoder; its compressor against hand-worked outputs and by round trips through the
independent decoder; the table builder and the compaction by reading their output with
the independent reader."""
import struct

import numpy as np
import pytest

import oracle
import sstpy
from helpers import U64MAX
from paper_2004_03054_b300 import workloads as W

# (stream, decoded bytes), each element worked out from the format description
STREAMS = [
    ("00", b""),                                           # length 0, no elements
    ("05" "10" + b"hello".hex(), b"hello"),                  # literal of 5: tag (5 - 1) << 2
    ("0a" "04" + b"ab".hex() + "1e0200", b"ababababab"),     # 2-byte-offset copy, length 8 at offset 2 (overlap)
    ("09" "10" + b"abcde".hex() + "0105", b"abcdeabcd"),     # 1-byte-offset copy: length 4 + 0, offset 5
    ("06" "08" + b"xyz".hex() + "0b03000000", b"xyzxyz"),    # 4-byte-offset copy: length 1 + 2, offset 3
    ("64" "f063" + bytes(range(100)).hex(), bytes(range(100))),  # literal length 100 in one extra byte (tag 60)
    ("8002" "f4ff00" + bytes(256).hex(), bytes(256)),        # length 256: varint 80 02, tag 61, two bytes 0x00ff
]

BAD = [
    "05" "10" + b"hell".hex(),        # literal runs past the stream
    "04" "04" + b"ab".hex() + "0a00", # copy offset 0
    "04" "04" + b"ab".hex() + "0a03", # 2-byte copy offset 3 beyond the 2 bytes written (kind 2 needs 2 bytes: truncated)
    "06" "04" + b"ab".hex() + "0a0300",  # offset 3 beyond the 2 bytes written
    "03" "04" + b"ab".hex(),          # decoded length 2, header says 3
    "01" "04" + b"ab".hex(),          # decoded length 2, header says 1
    "",                               # no length
]


@pytest.mark.parametrize("stream,want", STREAMS)
def test_decode_hand_worked(stream, want):
    b = bytes.fromhex(stream)
    assert oracle.snappy_uncompress(b) == (0, want)
    assert sstpy.snappy_uncompress(b) == want


@pytest.mark.parametrize("stream", BAD)
def test_decode_rejects(stream):
    b = bytes.fromhex(stream)
    assert oracle.snappy_uncompress(b)[0] == oracle.ERR_CORRUPTION
    with pytest.raises((ValueError, IndexError)):
        sstpy.snappy_uncompress(b)


# Compressor outputs worked out by hand. H(i) = (x * 2654435761 mod 2^32) >> 20 of the
# word at i; the inputs are chosen so that only the intended positions share a hash:
#   "a" * 10: position 1 finds 0; copy of length 9 (the rest of the input), offset 1 ->
#     varint 10, literal "a" (tag 00), kind-1 copy tag 1 | (9 - 4) << 2 = 0x15, offset 01;
#   "ab" * 6: H("abab") = 0x0da != H("baba") = 0x3d1, so position 2 finds 0 with length
#     10 -> literal "ab" (tag 04), kind-1 copy 1 | 6 << 2 = 0x19, offset 02;
#   "abcdefgh" * 4: the eight 4-grams of the first period hash apart (0x630 0x637 0x63d
#     0x643 0x649 0xdcf 0x0fd 0x546); position 8 finds 0 with length 24 > 11 -> literal
#     of 8 (tag 0x1c), kind-2 copy 2 | 23 << 2 = 0x5e, offset 08 00;
#   100 zero bytes: segment [0, 64): literal 00, then position 1 finds 0 and copies to the
#     segment's end (length 63 > 11: kind 2, 2 | 62 << 2 = 0xfa, offset 01 00); segment
#     [64, 100) starts its own parse: position 64 finds 63, copy of length 36 (0x8e 01 00);
#   66 zero bytes: as above, then segment [64, 66) has fewer than 4 bytes: literal 00 00.
@pytest.mark.parametrize("data,stream", [
    (bytes(100), "64" "0000" "fa0100" "8e0100"),
    (bytes(66), "42" "0000" "fa0100" "040000"),
    (b"a" * 10, "0a" "0061" "1501"),
    (b"ab" * 6, "0c" "046162" "1902"),
    (b"abcdefgh" * 4, "20" "1c" + b"abcdefgh".hex() + "5e0800"),
    (b"", "00"),
    (b"abc", "03" "08616263"),
])
def test_compress_hand_worked(data, stream):
    assert oracle.snappy_compress(data).hex() == stream


def _compressible(rng, n, words=None):
    """Bytes with repeats at many distances: a few random words (given, or drawn here) and
    their copies, with short random runs between them."""
    words = words or [rng.bytes(int(rng.integers(1, 24))) for _ in range(12)]
    out = bytearray()
    while len(out) < n:
        out += words[int(rng.integers(0, len(words)))] if rng.random() < 0.8 else rng.bytes(int(rng.integers(1, 9)))
    return bytes(out[:n])


@pytest.mark.parametrize("seed", range(20))
def test_round_trip(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.choice([1, 3, 4, 5, 63, 64, 65, 300, 4096, 70000]))
    for data in (_compressible(rng, n), rng.bytes(n), bytes(n)):
        c = oracle.snappy_compress(data)
        assert sstpy.snappy_uncompress(c) == data
        assert oracle.snappy_uncompress(c) == (0, data)
    # a long run of zeros: one literal byte, then one copy of offset 1 per 64-byte segment
    z = oracle.snappy_compress(bytes(1000))
    assert len(z) < 60 and sstpy.snappy_uncompress(z) == bytes(1000)


def _run(n, vlen, seed, compressible=True):
    rng = np.random.default_rng(seed)
    users = sorted({rng.bytes(16) for _ in range(n)})
    n = len(users)
    words = [rng.bytes(int(rng.integers(4, 24))) for _ in range(16)]   # shared by the run's values
    vals = [(_compressible(rng, vlen, words) if compressible else rng.bytes(vlen)) for _ in range(n)]
    voff = np.zeros(n + 1, np.uint64)
    np.cumsum([len(v) for v in vals], out=voff[1:])
    km = np.frombuffer(b"".join(users), np.uint8).copy()
    return W.Run(km, np.arange(n + 1, dtype=np.uint64) * 16, np.arange(1, n + 1, dtype=np.uint64),
                 np.ones(n, np.uint8), np.frombuffer(b"".join(vals), np.uint8).copy(), voff, 0)


@pytest.mark.parametrize("n,T,vlen,target", [(300, 4096, 200, U64MAX), (400, 1024, 50, 16 << 10),
                                             (100, 1, 300, U64MAX), (120, 16384, 1000, 64 << 10)])
def test_builder(n, T, vlen, target):
    run = _run(n, vlen, seed=T + vlen)
    comp = oracle.build_tables(run, T, 16, 10, target, flags=oracle.F_COMPRESS)
    raw = oracle.build_tables(run, T, 16, 10, target)
    assert comp.status == raw.status == 0
    rc_ = [sstpy.read(t.data) for t in comp.tables]
    rr = [sstpy.read(t.data) for t in raw.tables]
    # the same entries; with one table, cut into the same blocks (the block cut uses the
    # uncompressed sizes; the file cut the stored ones)
    assert [e for r in rc_ for e in r["entries"]] == [e for r in rr for e in r["entries"]]
    if target == U64MAX:
        assert [[b[2] for b in r["blocks"]] for r in rc_] == [[b[2] for b in r["blocks"]] for r in rr]
    assert any(t == 1 for r in rc_ for t in r["types"])
    for t, r in zip(comp.tables, rc_):
        for (off, size, ents), typ in zip(r["blocks"], r["types"]):
            if typ == 1:   # kept compressed only when that saves an eighth
                raw_len = len(sstpy.snappy_uncompress(t.data[off:off + size]))
                assert size < raw_len - raw_len // 8
        ok, rt, _ = oracle.read_table(t.data)
        assert ok == 0 and rt.layout_ok and rt.index_keys_ok


def test_incompressible_blocks_stay_raw():
    run = _run(100, 500, seed=7, compressible=False)
    res = oracle.build_tables(run, 4096, 16, 10, U64MAX, flags=oracle.F_COMPRESS)
    plain = oracle.build_tables(run, 4096, 16, 10, U64MAX)
    assert [t.data for t in res.tables] == [t.data for t in plain.tables]


def _compact(inputs, flags=0, T=4096, target=2 << 20):
    return oracle.compact(inputs, oracle.MAX_SEQ, False, T, 16, 10, target, flags)


def test_compaction_of_compressed_inputs():
    runs = [_run(150, 150, seed=s) for s in (1, 2, 3)]
    for i, r in enumerate(runs):
        r.seqs[:] = r.seqs + np.uint64(1000 * (3 - i))   # newer inputs first
    comp = [oracle.build_tables(r, 2048, 16, 10, U64MAX, flags=oracle.F_COMPRESS).tables[0].data for r in runs]
    raw = [oracle.build_tables(r, 2048, 16, 10, U64MAX).tables[0].data for r in runs]
    assert any(t == 1 for d in comp for t in sstpy.read(d)["types"])
    a, b = _compact(comp), _compact(raw)
    assert a.status == b.status == 0
    assert [t.data for t in a.tables] == [t.data for t in b.tables]
    c = _compact(comp, flags=oracle.F_COMPRESS)
    assert c.status == 0
    assert [e for t in c.tables for e in sstpy.read(t.data)["entries"]] == \
        [e for t in b.tables for e in sstpy.read(t.data)["entries"]]


def _reseal(img: bytearray, off: int, size: int):
    """Recompute a block's masked CRC trailer after an edit."""
    c = sstpy.crc32c(bytes(img[off:off + size + 1]))
    m = ((((c >> 15) | (c << 17)) & 0xFFFFFFFF) + 0xA282EAD8) & 0xFFFFFFFF
    img[off + size + 1:off + size + 5] = struct.pack("<I", m)


def test_malformed_stream_with_valid_checksum():
    run = _run(60, 300, seed=11)
    img = bytearray(oracle.build_tables(run, 4096, 16, 10, U64MAX, flags=oracle.F_COMPRESS).tables[0].data)
    r = sstpy.read(bytes(img))
    b = next(i for i, t in enumerate(r["types"]) if t == 1)
    off, size, _ = r["blocks"][b]
    bad = bytearray(img)
    bad[off] ^= 0x01          # the uncompressed-length varint: decoded length no longer matches
    _reseal(bad, off, size)
    assert _compact([bytes(bad)]).status == oracle.ERR_CORRUPTION
    other = bytearray(img)
    other[off + size] = 2     # an unknown block type, checksum resealed
    _reseal(other, off, size)
    assert _compact([bytes(other)]).status == oracle.ERR_NOT_SUPPORTED
