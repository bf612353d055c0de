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


def block(buf: bytes, off: int, size: int, data: bool = False) -> bytes:
    """A block's contents after its checksum check; a data block may be stored compressed
    (type 1, R4c)."""
    contents = buf[off:off + size]
    typ = buf[off + size]
    (m,) = struct.unpack_from("<I", buf, off + size + 1)
    if crc32c(buf[off:off + size + 1]) != unmask(m):
        raise ValueError("crc")
    if typ == 1 and data:
        return snappy_uncompress(contents)
    if typ != 0:
        raise ValueError("compressed")
    return contents


def snappy_uncompress(b: bytes) -> bytes:
    """A Snappy-format stream, decoded element by element from the format's published
    description (varint length; literal, 1-, 2- and 4-byte-offset copy elements)."""
    ulen, p = varint(b, 0, len(b))
    out = bytearray()
    while p < len(b):
        tag = b[p]
        p += 1
        kind = tag & 3
        if kind == 0:
            n = tag >> 2
            if n >= 60:
                nb = n - 59
                if p + nb > len(b):
                    raise ValueError("truncated literal length")
                n = int.from_bytes(b[p:p + nb], "little")
                p += nb
            n += 1
            if p + n > len(b):
                raise ValueError("truncated literal")
            out += b[p:p + n]
            p += n
            continue
        if kind == 1:
            if p + 1 > len(b):
                raise ValueError("truncated copy")
            n, off = 4 + ((tag >> 2) & 7), ((tag >> 5) << 8) | b[p]
            p += 1
        else:
            nb = 2 if kind == 2 else 4
            if p + nb > len(b):
                raise ValueError("truncated copy")
            n, off = 1 + (tag >> 2), int.from_bytes(b[p:p + nb], "little")
            p += nb
        if off == 0 or off > len(out):
            raise ValueError("copy offset")
        for _ in range(n):
            out.append(out[-off])
    if len(out) != ulen:
        raise ValueError("length")
    return bytes(out)


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
    fh = [(k, v) for k, v, _ in meta if k in (b"filter.luda.bloom", b"filter.luda.bloom2k")]
    if len(fh) != 1:
        raise ValueError("metaindex must name exactly one filter")
    fname = fh[0][0].decode()
    foff, fsize, _ = handle(fh[0][1])
    filt = block(buf, foff, fsize)
    blocks = []
    types = []
    allents = []
    for i, (k, v, _) in enumerate(index):
        off, size, _ = handle(v)
        ents = entries(block(buf, off, size, data=True))
        types.append(buf[off + size])
        # R9: last key <= index key < the next block's first key (internal key order)
        if len(k) < 8 or _order(ents[-1][0]) > _order(k):
            raise ValueError("index key is below its block's last key")
        if blocks and _order(index[i - 1][0]) >= _order(ents[0][0]):
            raise ValueError("index key is not below the next block's first key")
        blocks.append((off, size, ents))
        allents.extend((e[0], e[1]) for e in ents)
    return dict(entries=allents, blocks=blocks, types=types, filter=filt, filter_name=fname,
                index_keys=[k for k, _, _ in index],
                handles=dict(filter=(foff, fsize), meta=(moff, msize), index=(ioff, isize)))


def _order(ikey: bytes):
    """Sort key of an internal key: user key ascending, then the trailer descending."""
    (tr,) = struct.unpack("<Q", ikey[-8:])
    return (ikey[:-8], -tr)


def split_internal(ikey: bytes):
    (tr,) = struct.unpack("<Q", ikey[-8:])
    return ikey[:-8], tr >> 8, tr & 0xFF


def murmur3_32(data: bytes, seed: int = 0) -> int:
    """MurmurHash3 x86_32, written from its published definition (4-byte little-endian
    blocks mixed with c1 = 0xcc9e2d51, c2 = 0x1b873593, rotations 15 and 13, then the
    tail, the length and the fmix32 finaliser)."""
    M = 0xFFFFFFFF
    h = seed & M
    n = len(data)
    c1, c2 = 0xCC9E2D51, 0x1B873593

    def rotl(x, r):
        return ((x << r) | (x >> (32 - r))) & M

    for i in range(0, n - n % 4, 4):
        k = int.from_bytes(data[i:i + 4], "little")
        k = rotl((k * c1) & M, 15) * c2 & M
        h = (rotl(h ^ k, 13) * 5 + 0xE6546B64) & M
    t = data[n - n % 4:]
    if t:
        k = int.from_bytes(t, "little")
        h ^= rotl((k * c1) & M, 15) * c2 & M
    h ^= n
    h ^= h >> 16
    h = (h * 0x85EBCA6B) & M
    h ^= h >> 13
    h = (h * 0xC2B2AE35) & M
    return h ^ (h >> 16)


def bloom(ukeys, bpk: int) -> bytes:
    """One R10 bloom filter (bitmap || k) over the user keys, bit by bit."""
    bits = max(64, len(ukeys) * bpk)
    nbytes = (bits + 7) // 8
    bits = nbytes * 8
    k = min(30, max(1, bpk * 69 // 100))
    bm = bytearray(nbytes)
    for u in ukeys:
        h = murmur3_32(u)
        d = ((h >> 17) | (h << 15)) & 0xFFFFFFFF
        for _ in range(k):
            b = h % bits
            bm[b >> 3] |= 1 << (b & 7)
            h = (h + d) & 0xFFFFFFFF
    return bytes(bm) + bytes([k])


def filter_array(blocks, data_end: int, bpk: int, base_lg: int = 11) -> bytes:
    """The R10 variant's filter block, from a table's data blocks [(off, size, entries)]
    and the offset where its data blocks end: filter i holds the user keys of the blocks
    with off >> base_lg == i; there are max(data_end >> base_lg, (last off >> base_lg) + 1)
    filters, the ones without keys empty."""
    n = max(data_end >> base_lg, (blocks[-1][0] >> base_lg) + 1) if blocks else 0
    keys = [[] for _ in range(n)]
    for off, _, ents in blocks:
        keys[off >> base_lg].extend(e[0][:-8] for e in ents)
    body, offs = b"", []
    for ks in keys:
        offs.append(len(body))
        if ks:
            body += bloom(ks, bpk)
    return body + b"".join(struct.pack("<I", o) for o in offs) + struct.pack("<I", len(body)) + bytes([base_lg])
