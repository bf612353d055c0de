"""An independent, pure-Python reader of the table format, for small tables in tests.

It shares nothing with the C oracle or the CUDA path: its own varint decoder, its own
bit-at-a-time CRC-32C (from the reflected polynomial) and its own block walker. Reading
the oracle's output with it (and comparing against the brute-force replay) pins the
oracle's encoder without trusting the oracle's own reader.
"""
from __future__ import annotations

import struct

MAGIC = 0x4C55444153535431
POLY = 0x82F63B78


def crc32c(data: bytes) -> int:
    c = 0xFFFFFFFF
    for b in data:
        c ^= b
        for _ in range(8):
            c = (c >> 1) ^ POLY if c & 1 else c >> 1
    return c ^ 0xFFFFFFFF


def unmask(m: int) -> int:
    r = (m - 0xA282EAD8) & 0xFFFFFFFF
    return ((r >> 17) | (r << 15)) & 0xFFFFFFFF


def varint(buf: bytes, pos: int, limit: int):
    shift = 0
    val = 0
    while True:
        if pos >= limit or shift > 63:
            raise ValueError("bad varint")
        b = buf[pos]
        pos += 1
        val |= (b & 0x7F) << shift
        if not b & 0x80:
            return val, pos
        shift += 7


def block(buf: bytes, off: int, size: int) -> bytes:
    contents = buf[off:off + size]
    typ = buf[off + size]
    (m,) = struct.unpack_from("<I", buf, off + size + 1)
    if crc32c(buf[off:off + size + 1]) != unmask(m):
        raise ValueError("crc")
    if typ != 0:
        raise ValueError("compressed")
    return contents


def entries(contents: bytes):
    """[(key, value, is_restart)] of a block, keys rebuilt from shared prefixes."""
    (nr,) = struct.unpack_from("<I", contents, len(contents) - 4)
    rstart = len(contents) - 4 - 4 * nr
    restarts = set(struct.unpack_from(f"<{nr}I", contents, rstart))
    out = []
    pos = 0
    key = b""
    while pos < rstart:
        is_restart = pos in restarts
        shared, pos = varint(contents, pos, rstart)
        nonshared, pos = varint(contents, pos, rstart)
        vlen, pos = varint(contents, pos, rstart)
        if is_restart and shared:
            raise ValueError("restart with shared bytes")
        key = key[:shared] + contents[pos:pos + nonshared]
        pos += nonshared
        out.append((key, contents[pos:pos + vlen], is_restart))
        pos += vlen
    if pos != rstart:
        raise ValueError("entries overrun")
    return out


def handle(b: bytes, pos=0):
    off, pos = varint(b, pos, len(b))
    size, pos = varint(b, pos, len(b))
    return off, size, pos


def read(buf: bytes):
    """dict(entries=[(internal_key, value)], blocks=[(off, size, [entries])], filter=bytes)."""
    (magic,) = struct.unpack_from("<Q", buf, len(buf) - 8)
    if magic != MAGIC:
        raise ValueError("magic")
    ft = buf[len(buf) - 48:len(buf) - 8]
    moff, msize, p = handle(ft)
    ioff, isize, _ = handle(ft, p)
    index = entries(block(buf, ioff, isize))
    meta = entries(block(buf, moff, msize))
    fh = [v for k, v, _ in meta if k == b"filter.luda.bloom"]
    foff, fsize, _ = handle(fh[0])
    filt = block(buf, foff, fsize)
    blocks = []
    allents = []
    for i, (k, v, _) in enumerate(index):
        off, size, _ = handle(v)
        ents = entries(block(buf, off, size))
        # R9: last key <= index key < the next block's first key (internal key order)
        if len(k) < 8 or _order(ents[-1][0]) > _order(k):
            raise ValueError("index key is below its block's last key")
        if blocks and _order(index[i - 1][0]) >= _order(ents[0][0]):
            raise ValueError("index key is not below the next block's first key")
        blocks.append((off, size, ents))
        allents.extend((e[0], e[1]) for e in ents)
    return dict(entries=allents, blocks=blocks, filter=filt, index_keys=[k for k, _, _ in index],
                handles=dict(filter=(foff, fsize), meta=(moff, msize), index=(ioff, isize)))


def _order(ikey: bytes):
    """Sort key of an internal key: user key ascending, then the trailer descending."""
    (tr,) = struct.unpack("<Q", ikey[-8:])
    return (ikey[:-8], -tr)


def split_internal(ikey: bytes):
    (tr,) = struct.unpack("<Q", ikey[-8:])
    return ikey[:-8], tr >> 8, tr & 0xFF
