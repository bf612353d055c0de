"""Shared test helpers: building input tables with the oracle, reading results."""
from __future__ import annotations

import struct

import oracle
import sstpy

U64MAX = (1 << 64) - 1


def oracle_inputs(job):
    """Each run of the job becomes one input table, built by the oracle's builder."""
    out = []
    for r in job.inputs:
        res = oracle.build_tables(r, job.block_size, job.restart_interval, job.bloom_bits_per_key, U64MAX)
        assert res.status == 0, res.detail
        assert len(res.tables) == 1
        out.append(res.tables[0].data)
    return out


def oracle_compact(job, inputs=None, flags=0):
    inputs = oracle_inputs(job) if inputs is None else inputs
    return oracle.compact(inputs, job.smallest_snapshot, job.bottommost, job.block_size, job.restart_interval,
                          job.bloom_bits_per_key, job.target_file_size, flags)


def decoded(tables, reader="oracle"):
    """[(ukey, seq, type, value)] of a list of table images, in file order."""
    out = []
    for t in tables:
        data = t.data if hasattr(t, "data") else t
        if reader == "py":
            ents = sstpy.read(data)["entries"]
        else:
            st, rt, det = oracle.read_table(data)
            assert st == 0, det
            ents = list(zip(rt.keys, rt.values))
        for k, v in ents:
            (tr,) = struct.unpack("<Q", k[-8:])
            out.append((k[:-8], tr >> 8, tr & 0xFF, v))
    return out
