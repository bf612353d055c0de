"""Pins of the oracle's primitives against published values and hand-worked examples."""
import ast
import os

import numpy as np
import pytest

import oracle
import sstpy

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _lines(name, fields=None):
    """Non-comment lines split on whitespace (the first field may hold spaces when
    `fields` is given: the rest are split from the right)."""
    with open(os.path.join(GOLD, name)) as f:
        rows = [ln.rstrip("\n") for ln in f if ln.strip() and not ln.startswith("#")]
    return [r.rsplit(None, fields - 1) if fields else r.split() for r in rows]


def _crc_message(spec):
    kind, arg = spec.split(":", 1)
    if kind == "ascii":
        return arg.encode()
    n = int(arg)
    return {"zeros": bytes(n), "ones": b"\xff" * n, "incr": bytes(range(n)),
            "decr": bytes(range(n - 1, -1, -1))}[kind]


@pytest.mark.parametrize("spec,want", _lines("crc32c_vectors.txt"))
def test_crc32c_published(spec, want):
    msg = _crc_message(spec)
    assert oracle.crc32c(msg) == int(want, 16)
    assert oracle.crc32c_bitwise(msg) == int(want, 16)


def test_crc32c_table_equals_bitwise_random():
    rng = np.random.default_rng(0)
    for n in [0, 1, 2, 3, 4, 5, 7, 8, 31, 64, 100, 1000, 4097]:
        msg = rng.bytes(n)
        assert oracle.crc32c(msg) == oracle.crc32c_bitwise(msg) == sstpy.crc32c(msg)


def test_mask_roundtrip():
    rng = np.random.default_rng(1)
    for c in [0, 1, 0xFFFFFFFF, 0xA282EAD8] + rng.integers(0, 2**32, size=200).tolist():
        m = oracle.mask(int(c))
        assert oracle.unmask(m) == c
        assert m == ((((c >> 15) | (c << 17)) & 0xFFFFFFFF) + 0xA282EAD8) & 0xFFFFFFFF
    assert oracle.mask(0) == 0xA282EAD8


@pytest.mark.parametrize("msg,seed,want", _lines("murmur3_vectors.txt", 3))
def test_murmur3_published(msg, seed, want):
    assert oracle.murmur3_32(ast.literal_eval(msg), int(seed, 16)) == int(want, 16)


@pytest.mark.parametrize("value,enc", _lines("varint_vectors.txt"))
def test_varint_vectors(value, enc):
    assert oracle.put_varint(int(value)).hex() == enc
    v, n = oracle.get_varint64(bytes.fromhex(enc))
    assert (v, n) == (int(value), len(enc) // 2)


def test_varint_malformed():
    assert oracle.get_varint64(b"\x80")[1] == 0                       # truncated
    assert oracle.get_varint64(b"\x80" * 10 + b"\x01")[1] == 0        # 11 bytes
    assert oracle.get_varint64(b"\xff" * 9 + b"\x02")[1] == 0         # > 2^64
    assert oracle.get_varint64(b"\x80\x00") == (0, 2)                  # non-minimal accepted


@pytest.mark.parametrize("R,contents", _lines("block_example.txt"))
def test_block_worked_example(R, contents):
    got = oracle.encode_block([(b"abc", b"1"), (b"abd", b"22"), (b"abe", b"")], int(R))
    assert got.hex() == contents
    ents = sstpy.entries(got)
    assert [(k, v) for k, v, _ in ents] == [(b"abc", b"1"), (b"abd", b"22"), (b"abe", b"")]


def test_block_restart_rule_random():
    """Random blocks decode back with the independent Python walker; entry j is a restart
    iff j % R == 0."""
    rng = np.random.default_rng(2)
    for R in [1, 2, 3, 5, 16]:
        keys = sorted({rng.bytes(int(rng.integers(0, 12))) for _ in range(60)})
        ents = [(k, rng.bytes(int(rng.integers(0, 9)))) for k in keys]
        got = oracle.encode_block(ents, R)
        dec = sstpy.entries(got)
        assert [(k, v) for k, v, _ in dec] == ents
        assert [r for _, _, r in dec] == [j % R == 0 for j in range(len(ents))]
