"""CPU oracle for the LUDA compaction job -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import this package. The product path (``paper_2004_03054_b300``) never does.

The arithmetic lives in ``luda_oracle.c`` (plain C, single-threaded); this module only
marshals arguments through ctypes. See that file's header for what is computed and which
part of the paper each step follows (LUDA, §II-A Phases 1-3).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import time
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "luda_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_HDR = os.path.join(os.path.dirname(_HERE), "include", "luda_oracle.h")  # its C ABI (luda_oracle_compact)

OK = 0
ERR_INVALID_ARG = -1
ERR_CORRUPTION = -2
ERR_NOT_SUPPORTED = -3
ERR_OOM = -4
ERR_DUPLICATE_KEY = -7
F_STRICT_DUP = 1
F_SHORT_INDEX = 4  # index keys shortened (format variant of R9)
F_FILTER_ARRAY = 8  # one filter per 2 KiB of data block offsets (format variant of R10)
F_COMPRESS = 16  # data blocks stored Snappy-compressed when that saves an eighth (R4c)
MAX_SEQ = (1 << 56) - 1


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (plain -O2, no vectorisation pragmas)."""
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-Wall", "-shared", "-fPIC", "-I", os.path.dirname(_HDR),
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


class _Table(C.Structure):
    _fields_ = [("data", C.POINTER(C.c_uint8)), ("size", C.c_uint64), ("n_entries", C.c_uint64),
                ("smallest", C.POINTER(C.c_uint8)), ("smallest_len", C.c_uint32),
                ("largest", C.POINTER(C.c_uint8)), ("largest_len", C.c_uint32)]


class _Result(C.Structure):
    _fields_ = [("tables", C.POINTER(_Table)), ("n_tables", C.c_uint32),
                ("n_in_entries", C.c_uint64), ("n_dropped", C.c_uint64)]


class _Read(C.Structure):
    _fields_ = [("keys", C.POINTER(C.c_uint8)), ("koff", C.POINTER(C.c_uint64)),
                ("vals", C.POINTER(C.c_uint8)), ("voff", C.POINTER(C.c_uint64)), ("n", C.c_uint64),
                ("n_blocks", C.c_uint64), ("blk_off", C.POINTER(C.c_uint64)),
                ("blk_size", C.POINTER(C.c_uint64)), ("blk_last", C.POINTER(C.c_uint64)),
                ("index_keys_ok", C.c_uint32), ("index_keys_exact", C.c_uint32), ("layout_ok", C.c_uint32),
                ("filter_off", C.c_uint64), ("filter_size", C.c_uint64), ("filter_array", C.c_uint32)]


_lib = None
_EMPTY = np.zeros(1, np.uint8)  # a valid address for an empty bound key


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        u8p, u64p = C.POINTER(C.c_uint8), C.POINTER(C.c_uint64)
        L.ora_crc32c.restype = C.c_uint32
        L.ora_crc32c.argtypes = [C.c_void_p, C.c_uint64]
        L.ora_crc32c_bitwise.restype = C.c_uint32
        L.ora_crc32c_bitwise.argtypes = [C.c_void_p, C.c_uint64]
        L.ora_mask.restype = C.c_uint32
        L.ora_mask.argtypes = [C.c_uint32]
        L.ora_unmask.restype = C.c_uint32
        L.ora_unmask.argtypes = [C.c_uint32]
        L.ora_murmur3_32.restype = C.c_uint32
        L.ora_murmur3_32.argtypes = [C.c_void_p, C.c_uint64, C.c_uint32]
        L.ora_put_varint.restype = C.c_uint32
        L.ora_put_varint.argtypes = [C.c_void_p, C.c_uint64]
        L.ora_get_varint64.restype = C.c_uint64
        L.ora_get_varint64.argtypes = [C.c_void_p, C.c_uint64, u64p]
        L.ora_encode_block.restype = C.c_int
        L.ora_encode_block.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_uint64,
                                       C.c_uint32, C.c_void_p, C.c_uint64, u64p]
        L.ora_compact.restype = C.c_int
        L.ora_compact.argtypes = [C.c_void_p, C.c_void_p, C.c_uint32, C.c_uint64, C.c_int32, C.c_uint64,
                                  C.c_uint32, C.c_uint32, C.c_uint64, C.c_uint32, C.POINTER(C.POINTER(_Result))]
        L.ora_compact_range.restype = C.c_int
        L.ora_compact_range.argtypes = [C.c_void_p, C.c_void_p, C.c_uint32, C.c_uint64, C.c_int32, C.c_uint64,
                                        C.c_uint32, C.c_uint32, C.c_uint64, C.c_uint32, C.c_void_p, C.c_uint64,
                                        C.c_void_p, C.c_uint64, C.POINTER(C.POINTER(_Result))]
        L.ora_build.restype = C.c_int
        L.ora_build.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                C.c_uint64, C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint64, C.c_uint32,
                                C.POINTER(C.POINTER(_Result))]
        L.ora_free_result.argtypes = [C.POINTER(_Result)]
        L.ora_read_table.restype = C.c_int
        L.ora_read_table.argtypes = [C.c_void_p, C.c_uint64, C.POINTER(C.POINTER(_Read))]
        L.ora_free_read.argtypes = [C.POINTER(_Read)]
        L.ora_bloom_may_contain.restype = C.c_int
        L.ora_bloom_may_contain.argtypes = [C.c_void_p, C.c_uint64, C.c_void_p, C.c_uint64]
        for name in ("ora_snappy_compress", "ora_snappy_uncompress"):
            f = getattr(L, name)
            f.restype = C.c_int
            f.argtypes = [C.c_void_p, C.c_uint64, C.POINTER(C.c_void_p), C.POINTER(C.c_uint64)]
        L.ora_filter_array_may_contain.restype = C.c_int
        L.ora_filter_array_may_contain.argtypes = [C.c_void_p, C.c_uint64, C.c_uint64, C.c_void_p, C.c_uint64]
        L.ora_last_detail.restype = C.c_char_p
        del u8p
        _lib = L
    return _lib


def _ptr(a) -> int:
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    raise TypeError(type(a))


def _u8(b) -> np.ndarray:
    if isinstance(b, np.ndarray):
        return np.ascontiguousarray(b, dtype=np.uint8)
    return np.frombuffer(bytes(b), dtype=np.uint8) if len(b) else np.zeros(1, np.uint8)[:0]


def crc32c(data: bytes) -> int:
    a = _u8(data)
    return lib().ora_crc32c(a.ctypes.data, len(a))


def crc32c_bitwise(data: bytes) -> int:
    a = _u8(data)
    return lib().ora_crc32c_bitwise(a.ctypes.data, len(a))


def mask(c: int) -> int:
    return lib().ora_mask(c)


def unmask(m: int) -> int:
    return lib().ora_unmask(m)


def murmur3_32(data: bytes, seed: int = 0) -> int:
    a = _u8(data)
    return lib().ora_murmur3_32(a.ctypes.data, len(a), seed)


def put_varint(v: int) -> bytes:
    buf = (C.c_uint8 * 10)()
    n = lib().ora_put_varint(buf, v)
    return bytes(buf[:n])


def get_varint64(data: bytes):
    """(value, bytes consumed); consumed == 0 means malformed."""
    a = _u8(data)
    v = C.c_uint64()
    n = lib().ora_get_varint64(a.ctypes.data, len(a), C.byref(v))
    return v.value, int(n)


def _blob(items):
    offs = np.zeros(len(items) + 1, np.uint64)
    if items:
        offs[1:] = np.cumsum([len(x) for x in items], dtype=np.uint64)
    blob = np.frombuffer(b"".join(items), np.uint8) if items else np.zeros(0, np.uint8)
    return np.ascontiguousarray(blob), offs


def encode_block(entries, restart_interval: int) -> bytes:
    """Contents of one block holding raw (key, value) entries (no trailer)."""
    kb, ko = _blob([k for k, _ in entries])
    vb, vo = _blob([v for _, v in entries])
    cap = sum(len(k) + len(v) + 15 for k, v in entries) + 4 * (len(entries) + 1) + 16
    out = np.zeros(cap, np.uint8)
    n = C.c_uint64()
    rc = lib().ora_encode_block(kb.ctypes.data, ko.ctypes.data, vb.ctypes.data, vo.ctypes.data, len(entries),
                                restart_interval, out.ctypes.data, cap, C.byref(n))
    if rc:
        raise ValueError(f"encode_block rc={rc}")
    return out[: n.value].tobytes()


@dataclass
class Table:
    data: bytes
    n_entries: int
    smallest: bytes
    largest: bytes


@dataclass
class Result:
    status: int
    tables: list
    n_in_entries: int = 0
    n_dropped: int = 0
    detail: str = ""


def _take(rc, res_p) -> Result:
    L = lib()
    if rc != OK:
        return Result(rc, [], detail=L.ora_last_detail().decode(errors="replace"))
    r = res_p.contents
    tables = []
    for i in range(r.n_tables):
        t = r.tables[i]
        tables.append(Table(C.string_at(t.data, t.size), int(t.n_entries),
                            C.string_at(t.smallest, t.smallest_len), C.string_at(t.largest, t.largest_len)))
    out = Result(OK, tables, int(r.n_in_entries), int(r.n_dropped))
    L.ora_free_result(res_p)
    return out


def compact(inputs, smallest_snapshot: int = MAX_SEQ, bottommost: bool = False, block_size: int = 4096,
            restart_interval: int = 16, bloom_bits_per_key: int = 10, target_file_size: int = 2 << 20,
            flags: int = 0, timing: dict | None = None, lo: bytes | None = None, hi: bytes | None = None) -> Result:
    """Compact input tables (listed newest first) into new tables. When `timing` is a
    dict, timing["seconds"] receives the wall time of the C call alone. lo / hi restrict
    the compaction to the user keys [lo, hi) (R13; None = unbounded)."""
    arrs = [_u8(x) for x in inputs]
    ptrs = (C.c_void_p * max(1, len(arrs)))(*[a.ctypes.data for a in arrs])
    sizes = (C.c_uint64 * max(1, len(arrs)))(*[len(a) for a in arrs])
    res = C.POINTER(_Result)()
    L = lib()
    t0 = time.perf_counter()
    lo_a = _u8(lo) if lo is not None else None
    hi_a = _u8(hi) if hi is not None else None
    rc = L.ora_compact_range(ptrs, sizes, len(arrs), smallest_snapshot, int(bool(bottommost)), block_size,
                             restart_interval, bloom_bits_per_key, target_file_size, flags,
                             (lo_a.ctypes.data if len(lo_a) else _EMPTY.ctypes.data) if lo_a is not None else None,
                             len(lo_a) if lo_a is not None else 0,
                             (hi_a.ctypes.data if len(hi_a) else _EMPTY.ctypes.data) if hi_a is not None else None,
                             len(hi_a) if hi_a is not None else 0, C.byref(res))
    if timing is not None:
        timing["seconds"] = time.perf_counter() - t0
    return _take(rc, res)


def build_tables(run, block_size: int = 4096, restart_interval: int = 16, bloom_bits_per_key: int = 10,
                 target_file_size: int = (1 << 64) - 1, flags: int = 0) -> Result:
    """Build tables from one sorted run (a ``workloads.Run``): the memtable-flush path."""
    ukeys = np.ascontiguousarray(run.ukeys, np.uint8)
    ukoff = np.ascontiguousarray(run.ukoff, np.uint64)
    seqs = np.ascontiguousarray(run.seqs, np.uint64)
    types = np.ascontiguousarray(run.types, np.uint8)
    vals = np.ascontiguousarray(run.vals, np.uint8)
    voff = np.ascontiguousarray(run.voff, np.uint64)
    res = C.POINTER(_Result)()
    rc = lib().ora_build(ukeys.ctypes.data, ukoff.ctypes.data, seqs.ctypes.data, types.ctypes.data,
                         vals.ctypes.data, voff.ctypes.data, len(seqs), block_size, restart_interval,
                         bloom_bits_per_key, target_file_size, flags, C.byref(res))
    return _take(rc, res)


@dataclass
class ReadTable:
    keys: list          # internal keys
    values: list
    n_blocks: int
    blk_off: list
    blk_size: list
    blk_last: list
    index_keys_ok: bool       # every index key in [its block's last key, the next block's first key)
    index_keys_exact: bool    # every index key equals its block's last key
    layout_ok: bool
    filter: bytes       # filter block contents (bitmap || k, or a filter array)
    filter_array: bool = False  # the metaindex names a filter array


def read_table(data: bytes):
    """(status, ReadTable | None, detail)."""
    a = _u8(data)
    r = C.POINTER(_Read)()
    L = lib()
    rc = L.ora_read_table(a.ctypes.data, len(a), C.byref(r))
    if rc != OK:
        return rc, None, L.ora_last_detail().decode(errors="replace")
    t = r.contents
    n = int(t.n)
    koff = np.ctypeslib.as_array(t.koff, shape=(n + 1,)).copy()
    voff = np.ctypeslib.as_array(t.voff, shape=(n + 1,)).copy()
    kb = C.string_at(t.keys, int(koff[-1])) if koff[-1] else b""
    vb = C.string_at(t.vals, int(voff[-1])) if voff[-1] else b""
    nb = int(t.n_blocks)
    out = ReadTable(
        keys=[kb[koff[i]:koff[i + 1]] for i in range(n)],
        values=[vb[voff[i]:voff[i + 1]] for i in range(n)],
        n_blocks=nb,
        blk_off=[int(t.blk_off[i]) for i in range(nb)],
        blk_size=[int(t.blk_size[i]) for i in range(nb)],
        blk_last=[int(t.blk_last[i]) for i in range(nb)],
        index_keys_ok=bool(t.index_keys_ok), index_keys_exact=bool(t.index_keys_exact), layout_ok=bool(t.layout_ok),
        filter=bytes(a[int(t.filter_off): int(t.filter_off) + int(t.filter_size)]),
        filter_array=bool(t.filter_array),
    )
    L.ora_free_read(r)
    return OK, out, ""


def bloom_may_contain(filter_contents: bytes, ukey: bytes) -> bool:
    f = _u8(filter_contents)
    k = _u8(ukey)
    return bool(lib().ora_bloom_may_contain(f.ctypes.data, len(f), k.ctypes.data, len(k)))


def _codec(name, data: bytes):
    a = _u8(data)
    p = C.c_void_p()
    n = C.c_uint64()
    rc = getattr(lib(), name)(a.ctypes.data, len(a), C.byref(p), C.byref(n))
    if rc != OK:
        return rc, None
    out = C.string_at(p, n.value) if n.value else b""
    C.CDLL(None).free(p)
    return OK, out


def snappy_compress(data: bytes) -> bytes:
    """This format's compressor (R4c): a Snappy-format stream."""
    rc, out = _codec("ora_snappy_compress", data)
    assert rc == OK
    return out


def snappy_uncompress(stream: bytes):
    """(status, bytes | None) of a Snappy-format stream."""
    return _codec("ora_snappy_uncompress", stream)


def filter_array_may_contain(filter_contents: bytes, block_off: int, ukey: bytes) -> bool:
    """Query of a filter array for a key of the data block at table offset block_off."""
    f = _u8(filter_contents)
    k = _u8(ukey)
    return bool(lib().ora_filter_array_may_contain(f.ctypes.data, len(f), block_off, k.ctypes.data, len(k)))


def subcompact(inputs, bounds, smallest_snapshot: int = MAX_SEQ, bottommost: bool = False, block_size: int = 4096,
               restart_interval: int = 16, bloom_bits_per_key: int = 10, target_file_size: int = 2 << 20,
               flags: int = 0) -> Result:
    """R13 subcompactions: the job split at the strictly increasing user keys `bounds` into
    len(bounds) + 1 ranged compactions, whose tables are concatenated in key order (entry
    counts summed; the first failing range's status)."""
    edges = [None] + list(bounds) + [None]
    out = Result(0, [])
    for lo, hi in zip(edges[:-1], edges[1:]):
        r = compact(inputs, smallest_snapshot, bottommost, block_size, restart_interval, bloom_bits_per_key,
                    target_file_size, flags, lo=lo, hi=hi)
        if r.status != 0:
            return r
        out.tables.extend(r.tables)
        out.n_in_entries += r.n_in_entries
        out.n_dropped += r.n_dropped
    return out
