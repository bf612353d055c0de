"""Brute-force map replay of a job's writes: what a compaction must keep.

Every version of every user key goes into a Python dict. Per key, the versions are taken
newest first and LevelDB's compaction rule is applied directly: a version is dropped when
a newer version of the same key is visible at the smallest snapshot, or when it is a
tombstone visible at that snapshot and the job is bottommost (LUDA §II-A, Phase 2: pairs
are merged in key order and deleted or stale ones are removed). The result is the expected entry list in output order.
"""
from __future__ import annotations

from collections import defaultdict

INF = float("inf")


def replay(job):
    versions = defaultdict(list)
    for r in job.inputs:
        for i in range(r.n):
            versions[r.key(i)].append((int(r.seqs[i]), int(r.types[i]), r.value(i)))
    S = job.smallest_snapshot
    out = []
    for k in sorted(versions):
        last = INF
        for seq, typ, val in sorted(versions[k], key=lambda t: (-t[0], -t[1])):
            drop = last <= S or (typ == 0 and seq <= S and job.bottommost)
            last = seq
            if not drop:
                out.append((k, seq, typ, val))
    return out


def newest_only(job):
    """Closed form for S = max: the newest version of each key, minus tombstones when
    bottommost."""
    newest = {}
    for r in job.inputs:
        for i in range(r.n):
            k = r.key(i)
            s = int(r.seqs[i])
            if k not in newest or s > newest[k][0]:
                newest[k] = (s, int(r.types[i]), r.value(i))
    return [(k,) + newest[k] for k in sorted(newest) if not (job.bottommost and newest[k][1] == 0)]
