"""Seeded synthetic compaction jobs shaped like the paper's workloads.

This module only draws data: user keys, sequence numbers, put/delete labels and value
bytes, grouped into runs (one run per input table, user keys unique and in byte order
within a run). It holds none of the compaction's arithmetic: no key encoding, checksum,
hash, varint or table layout. Both the CUDA path's table builder and the oracle's turn a
run into table bytes themselves.

The shapes follow the paper's evaluation (LUDA, §IV-A "Configuration and Methodology":
16 B keys, 128 B-1 KB values, 4 KB data blocks, 10 bits/key bloom filters, update-heavy
YCSB-A traffic with zipfian skew). No dataset or benchmark item is reproduced: every byte
comes from ``numpy.random.Generator(PCG64(seed))``.

Configs (sizes at ``scale=1``):
  1 single plain job: 1 level-1 table + 2 overlapping level-2 tables of ~2 MiB; 16 B keys
    u64_be(x) || u64_be(splitmix64(x)), x uniform in [0, 2^40); 15% of level-1 keys reuse a
    level-2 key; 100 B values; 2% deletions; 4 KiB blocks, 2 MiB files.
  2 LevelDB-default job: 1 level-L table + 10 level-L+1 tables of ~2 MiB; 16 B keys drawn
    zipf(0.99) over a 2^24-key universe; 128 B values; 5% deletions; bottommost.
  3 large job: 4 overlapping 64 MiB L0 tables + 12 disjoint 64 MiB L1 tables (~1 GiB);
    keys of 8-64 B built from a pool of 4096 prefixes of 0-24 B plus random suffixes;
    1 KiB values; 10% overwrites; 3% deletions; 16 KiB blocks, 64 MiB files.
  4 batch of 256 jobs, per-job input lognormal (median 4 MiB, sigma 1.2) clipped to
    [256 KiB, 64 MiB]; 16-32 B keys; 32 B-4 KiB values; 10% overwrites; 3% deletions.
  5 served: a write stream for a simulated LSM tree (``config5_stream``): Poisson
    arrivals, 16 B keys (half uniform, half zipf(0.99) over a 2^24-key universe), 256 B
    values, no deletions, cut into 64 MiB memtables.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

MAX_SEQ = (1 << 56) - 1
PUT, DEL = 1, 0
MiB = 1 << 20


@dataclass
class Run:
    """One input table's entries, user keys strictly increasing (byte order)."""
    ukeys: np.ndarray   # uint8 blob of user keys
    ukoff: np.ndarray   # uint64 [n+1]
    seqs: np.ndarray    # uint64 [n]
    types: np.ndarray   # uint8 [n]: 1 put, 0 delete
    vals: np.ndarray    # uint8 blob of values
    voff: np.ndarray    # uint64 [n+1]
    level: int = 0

    @property
    def n(self) -> int:
        return len(self.seqs)

    def key(self, i: int) -> bytes:
        return self.ukeys[self.ukoff[i]:self.ukoff[i + 1]].tobytes()

    def value(self, i: int) -> bytes:
        return self.vals[self.voff[i]:self.voff[i + 1]].tobytes()

    @property
    def nbytes(self) -> int:
        return int(self.ukoff[-1]) + int(self.voff[-1]) + 8 * self.n


@dataclass
class Job:
    name: str
    seed: int
    inputs: list                     # [Run], newest first
    smallest_snapshot: int = MAX_SEQ
    bottommost: bool = False
    block_size: int = 4096
    restart_interval: int = 16
    bloom_bits_per_key: int = 10
    target_file_size: int = 2 * MiB
    level: int = 1
    meta: dict = field(default_factory=dict)

    def opts(self) -> dict:
        return dict(block_size=self.block_size, restart_interval=self.restart_interval,
                    bloom_bits_per_key=self.bloom_bits_per_key, target_file_size=self.target_file_size)

    @property
    def n_entries(self) -> int:
        return sum(r.n for r in self.inputs)


def _splitmix64(x: np.ndarray) -> np.ndarray:
    """SplitMix64 output function (Steele, Lea, Flood 2014), vectorised, mod 2^64."""
    with np.errstate(over="ignore"):
        z = x.astype(np.uint64) + np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def _fixed_keys(hi: np.ndarray) -> np.ndarray:
    """16-byte keys u64_be(x) || u64_be(splitmix64(x)) as an [n, 16] byte matrix."""
    a = np.empty((len(hi), 2), dtype=">u8")
    a[:, 0] = hi
    a[:, 1] = _splitmix64(hi)
    return a.view(np.uint8).reshape(len(hi), 16)


def _make_run(keymat_or_list, seqs, types, vlens, rng, level) -> Run:
    """Assemble a run from keys already in increasing byte order."""
    n = len(seqs)
    if isinstance(keymat_or_list, np.ndarray):
        km = np.ascontiguousarray(keymat_or_list)
        ukeys = km.reshape(-1)
        ukoff = np.arange(n + 1, dtype=np.uint64) * np.uint64(km.shape[1])
    else:
        lens = np.fromiter((len(k) for k in keymat_or_list), dtype=np.uint64, count=n)
        ukeys = np.frombuffer(b"".join(keymat_or_list), dtype=np.uint8).copy() if n else np.zeros(0, np.uint8)
        ukoff = np.zeros(n + 1, np.uint64)
        np.cumsum(lens, out=ukoff[1:])
    vlens = np.where(np.asarray(types) == DEL, 0, np.asarray(vlens)).astype(np.uint64)
    voff = np.zeros(n + 1, np.uint64)
    np.cumsum(vlens, out=voff[1:])
    total = int(voff[-1])
    vals = np.frombuffer(rng.bytes(total), dtype=np.uint8).copy() if total else np.zeros(0, np.uint8)
    return Run(ukeys, ukoff, np.asarray(seqs, np.uint64), np.asarray(types, np.uint8), vals, voff, level)


def _types(rng, n, p_del):
    return np.where(rng.random(n) < p_del, DEL, PUT).astype(np.uint8)


def _split_even(n, parts):
    b = np.linspace(0, n, parts + 1).round().astype(np.int64)
    return [(int(b[i]), int(b[i + 1])) for i in range(parts)]


# ----------------------------------------------------------------------------------------
def config1(seed: int = 1, scale: float = 1.0) -> Job:
    rng = np.random.default_rng(seed)
    per = max(8, int(round(2 * MiB * scale / 125.5)))
    space = 1 << 40
    xs = np.unique(rng.integers(0, space, size=int(per * 3.3), dtype=np.uint64))
    rng.shuffle(xs)
    lower_x = np.sort(xs[: 2 * per])
    fresh = xs[2 * per: 2 * per + per]
    n_re = int(round(0.15 * per))
    reuse = rng.choice(lower_x, size=n_re, replace=False)
    upper_x = np.sort(np.concatenate([reuse, fresh[: per - n_re]]))
    seq_lower = rng.permutation(np.arange(1, 2 * per + 1, dtype=np.uint64))
    seq_upper = rng.permutation(np.arange(2 * per + 1, 3 * per + 1, dtype=np.uint64))
    inputs = [_make_run(_fixed_keys(upper_x), seq_upper, _types(rng, per, 0.02), np.full(per, 100), rng, 1)]
    for a, b in _split_even(2 * per, 2):
        inputs.append(_make_run(_fixed_keys(lower_x[a:b]), seq_lower[a:b], _types(rng, b - a, 0.02),
                                np.full(b - a, 100), rng, 2))
    return Job("cfg1_single_plain", seed, inputs, MAX_SEQ, False, 4096, 16, 10,
               max(4096, int(2 * MiB * scale)), level=2)


_ZIPF_CDF = {}


def _zipf_cdf(n: int, s: float) -> np.ndarray:
    key = (n, s)
    if key not in _ZIPF_CDF:
        w = np.arange(1, n + 1, dtype=np.float64) ** (-s)
        c = np.cumsum(w)
        _ZIPF_CDF[key] = c / c[-1]
    return _ZIPF_CDF[key]


def _zipf_distinct(rng, count, universe_bits, s, taken=None):
    """`count` distinct universe indices in first-draw order of a zipf(s) stream."""
    n = 1 << universe_bits
    cdf = _zipf_cdf(n, s)
    got = []
    seen = set() if taken is None else set(taken)
    draws = max(64, count * 2)
    while len(got) < count:
        r = np.searchsorted(cdf, rng.random(draws))
        u = (r.astype(np.uint64) * np.uint64(0x9E3779B1)) & np.uint64(n - 1)   # scatter ranks
        for v in u.tolist():
            if v not in seen:
                seen.add(v)
                got.append(v)
                if len(got) == count:
                    break
        draws *= 2
    return np.array(got, dtype=np.uint64)


def config2(seed: int = 2, scale: float = 1.0) -> Job:
    rng = np.random.default_rng(seed)
    per = max(8, int(round(2 * MiB * scale / 150.0)))
    lower_u = np.sort(_zipf_distinct(rng, 10 * per, 24, 0.99))
    upper_u = np.sort(_zipf_distinct(rng, per, 24, 0.99))
    seq_lower = rng.permutation(np.arange(1, 10 * per + 1, dtype=np.uint64))
    seq_upper = rng.permutation(np.arange(10 * per + 1, 11 * per + 1, dtype=np.uint64))
    inputs = [_make_run(_fixed_keys(upper_u), seq_upper, _types(rng, per, 0.05), np.full(per, 128), rng, 1)]
    for a, b in _split_even(10 * per, 10):
        inputs.append(_make_run(_fixed_keys(lower_u[a:b]), seq_lower[a:b], _types(rng, b - a, 0.05),
                                np.full(b - a, 128), rng, 2))
    return Job("cfg2_leveldb_default", seed, inputs, MAX_SEQ, True, 4096, 16, 10,
               max(4096, int(2 * MiB * scale)), level=2)


def _prefix_keys(rng, count, pool, lo, hi, seen):
    """`count` fresh distinct keys: a pool prefix (capped at the key length) + random tail."""
    out = []
    while len(out) < count:
        m = (count - len(out)) + 16
        lens = rng.integers(lo, hi + 1, size=m)
        pidx = rng.integers(0, len(pool), size=m)
        raw = rng.bytes(int(lens.sum()))
        pos = 0
        for L, pi in zip(lens.tolist(), pidx.tolist()):
            p = pool[pi][:L]
            k = p + raw[pos: pos + L - len(p)]
            pos += L
            if k not in seen:
                seen.add(k)
                out.append(k)
                if len(out) == count:
                    break
    return out


def with_compressible_values(job: Job, seed: int = 17, vocab: int = 256, word: int = 8) -> Job:
    """The job with every value rewritten (same lengths) as a stream of `word`-byte words
    drawn uniformly from a vocabulary of `vocab` random words, so that blocks compress
    (format variant R4c): most words recur within a block at distances below 2 KiB. The
    paper's YCSB values are random; this stands in for the text-like values of LevelDB's
    own benchmark, which compress to about half."""
    rng = np.random.default_rng(seed)
    words = np.frombuffer(rng.bytes(vocab * word), np.uint8).reshape(vocab, word)
    for r in job.inputs:
        total = int(r.voff[-1])
        if total:
            idx = rng.integers(0, vocab, size=(total + word - 1) // word)
            r.vals = np.ascontiguousarray(words[idx].reshape(-1)[:total])
    return job


def config3(seed: int = 3, scale: float = 1.0) -> Job:
    rng = np.random.default_rng(seed)
    per = max(8, int(round(64 * MiB * scale / 1076.0)))
    pool = [rng.bytes(int(n)) for n in rng.integers(0, 25, size=4096)]
    seen = set()
    lower = sorted(_prefix_keys(rng, 12 * per, pool, 8, 64, seen))
    seq = 1
    seq_lower = rng.permutation(np.arange(seq, seq + 12 * per, dtype=np.uint64))
    seq += 12 * per
    runs_l1 = []
    for a, b in _split_even(12 * per, 12):
        runs_l1.append(_make_run(lower[a:b], seq_lower[a:b], _types(rng, b - a, 0.03), np.full(b - a, 1024),
                                 rng, 1))
    existing = list(lower)
    runs_l0 = []
    for f in range(4):
        n_ow = int(round(0.10 * per))
        ow_idx = rng.choice(len(existing), size=n_ow, replace=False)
        ow = [existing[i] for i in ow_idx.tolist()]
        fresh = _prefix_keys(rng, per - n_ow, pool, 8, 64, seen)
        keys = sorted(set(ow) | set(fresh))
        existing.extend(fresh)
        s = rng.permutation(np.arange(seq, seq + len(keys), dtype=np.uint64))
        seq += len(keys)
        runs_l0.append(_make_run(keys, s, _types(rng, len(keys), 0.03), np.full(len(keys), 1024), rng, 0))
    inputs = list(reversed(runs_l0)) + runs_l1
    return Job("cfg3_large", seed, inputs, MAX_SEQ, False, 16384, 16, 10,
               max(16384, int(64 * MiB * scale)), level=1)


def config4_job(rng, total_bytes: int, name: str, seed: int) -> Job:
    """One job of the batch: 1 upper table + ceil(rest / 2 MiB) lower tables."""
    avg_entry = 24 + 8 + 3 + 2064
    upper_bytes = min(2 * MiB, total_bytes // 2)
    rest = total_bytes - upper_bytes
    n_lower_files = max(1, -(-rest // (2 * MiB)))
    n_lower = max(n_lower_files * 2, rest // avg_entry)
    n_upper = max(2, upper_bytes // avg_entry)
    seen = set()

    def rnd_keys(count):
        out = []
        while len(out) < count:
            lens = rng.integers(16, 33, size=count - len(out) + 8)
            raw = rng.bytes(int(lens.sum()))
            pos = 0
            for L in lens.tolist():
                k = raw[pos: pos + L]
                pos += L
                if k not in seen:
                    seen.add(k)
                    out.append(k)
                    if len(out) == count:
                        break
        return out

    lower = sorted(rnd_keys(int(n_lower)))
    n_ow = int(round(0.10 * n_upper))
    ow = [lower[i] for i in rng.choice(len(lower), size=min(n_ow, len(lower)), replace=False).tolist()]
    upper = sorted(set(ow) | set(rnd_keys(int(n_upper) - len(ow))))
    seq_lower = rng.permutation(np.arange(1, len(lower) + 1, dtype=np.uint64))
    seq_upper = rng.permutation(np.arange(len(lower) + 1, len(lower) + len(upper) + 1, dtype=np.uint64))
    inputs = [_make_run(upper, seq_upper, _types(rng, len(upper), 0.03),
                        rng.integers(32, 4097, size=len(upper)), rng, 1)]
    for a, b in _split_even(len(lower), int(n_lower_files)):
        inputs.append(_make_run(lower[a:b], seq_lower[a:b], _types(rng, b - a, 0.03),
                                rng.integers(32, 4097, size=b - a), rng, 2))
    return Job(name, seed, inputs, MAX_SEQ, False, 4096, 16, 10, 2 * MiB, level=2)


def config4(seed: int = 4, scale: float = 1.0, n_jobs: int = 256) -> list:
    rng = np.random.default_rng(seed)
    sizes = np.exp(rng.normal(np.log(4 * MiB), 1.2, size=n_jobs))
    sizes = np.clip(sizes, 256 * 1024, 64 * MiB) * scale
    sizes = np.maximum(sizes, 16 * 1024).astype(np.int64)
    return [config4_job(rng, int(s), f"cfg4_job{j}", seed) for j, s in enumerate(sizes.tolist())]


@dataclass
class Memtable:
    """One memtable's worth of writes in arrival order. User key i is
    u64_be(hi[i]) || u64_be(lo[i]); sequence numbers increase with arrival; every write is a
    put of a 256-byte value (the values themselves are drawn by the consumer, e.g. as
    slices of a random pool)."""
    t_full: float        # stream time (s) at which the memtable is full
    hi: np.ndarray       # uint64 [n]
    lo: np.ndarray       # uint64 [n]
    seqs: np.ndarray     # uint64 [n]
    value_len: int = 256

    @property
    def n(self) -> int:
        return len(self.seqs)


def config5_stream(seed: int = 5, n_memtables: int = 24, memtable_bytes: int = 64 * MiB,
                   write_rate: float = 8e6, value_len: int = 256, universe_bits: int = 24, zipf_s: float = 0.99,
                   first_seq: int = 1):
    """Seeded Poisson write stream (rate `write_rate` writes/s) cut into memtables of
    `memtable_bytes` (key + value + 8 bytes of sequence/type per write). Half of the keys
    are uniform 16-byte strings, half are zipf(`zipf_s`) draws over 2^universe_bits keys
    u64_be(splitmix64(r)) || u64_be(r)."""
    rng = np.random.default_rng(seed)
    per = max(1, memtable_bytes // (16 + value_len + 8))
    cdf = _zipf_cdf(1 << universe_bits, zipf_s)
    t, seq = 0.0, first_seq
    for _ in range(n_memtables):
        t += float(rng.gamma(per, 1.0 / write_rate))   # sum of `per` exponential gaps
        hi = rng.integers(0, 1 << 63, size=per, dtype=np.uint64) * np.uint64(2) + \
            rng.integers(0, 2, size=per, dtype=np.uint64)
        lo = rng.integers(0, 1 << 63, size=per, dtype=np.uint64) * np.uint64(2) + \
            rng.integers(0, 2, size=per, dtype=np.uint64)
        z = rng.random(per) < 0.5
        r = np.searchsorted(cdf, rng.random(int(z.sum()))).astype(np.uint64)
        hi[z] = _splitmix64(r)
        lo[z] = r
        seqs = np.arange(seq, seq + per, dtype=np.uint64)
        seq += per
        yield Memtable(t, hi, lo, seqs, value_len)


CONFIGS = {1: config1, 2: config2, 3: config3}


def make(config: int, seed: int | None = None, scale: float = 1.0) -> Job:
    fn = CONFIGS[config]
    return fn(seed if seed is not None else config, scale)


# ----------------------------------------------------------------------------------------
def tiny_job(rng, n_keys: int = 3, max_versions: int = 6, n_inputs: int = 3, key_len=(1, 3),
             val_len=(0, 4), p_del: float = 0.3, snapshot=None, bottommost=None, opts=None) -> Job:
    """A small random job for exhaustive-style tests: a few user keys, each with up to
    `max_versions` versions spread across `n_inputs` inputs (newer inputs hold newer
    versions), arbitrary snapshot and bottommost flag."""
    alphabet = [bytes([c]) for c in b"ab\x00\xff"]
    keys = set()
    while len(keys) < n_keys:
        L = int(rng.integers(key_len[0], key_len[1] + 1))
        keys.add(b"".join(alphabet[int(i)] for i in rng.integers(0, len(alphabet), size=L)))
    keys = sorted(keys)
    versions = []   # (ukey, input)
    for k in keys:
        nv = int(rng.integers(1, max_versions + 1))
        ins = sorted(rng.choice(n_inputs, size=min(nv, n_inputs), replace=False).tolist())
        for i in ins:
            versions.append((k, i))
    # input 0 is newest: assign seqs so that lower input index => higher seq
    n = len(versions)
    seqs = rng.permutation(np.arange(1, n + 1)).tolist()
    by_input = {i: [] for i in range(n_inputs)}
    # give the newest inputs the largest sequence numbers
    order = sorted(range(n), key=lambda j: (versions[j][1], seqs[j]))
    ranked = sorted(seqs, reverse=True)
    for rank, j in enumerate(order):
        k, i = versions[j]
        by_input[i].append((k, ranked[rank]))
    runs = []
    for i in range(n_inputs):
        ents = sorted(by_input[i])
        if not ents:
            continue
        ks = [k for k, _ in ents]
        ss = np.array([s for _, s in ents], np.uint64)
        ts = _types(rng, len(ents), p_del)
        vl = rng.integers(val_len[0], val_len[1] + 1, size=len(ents))
        runs.append(_make_run(ks, ss, ts, vl, rng, 0 if i == 0 else 1))
    max_seq = n
    if snapshot is None:
        snapshot = int(rng.integers(0, max_seq + 2)) if rng.random() < 0.7 else MAX_SEQ
    if bottommost is None:
        bottommost = bool(rng.random() < 0.5)
    o = dict(block_size=int(rng.choice([1, 16, 48, 4096])), restart_interval=int(rng.choice([1, 2, 3, 16])),
             bloom_bits_per_key=int(rng.choice([1, 5, 10])), target_file_size=int(rng.choice([1, 64, 200, 1 << 30])))
    if opts:
        o.update(opts)
    return Job("tiny", 0, runs, snapshot, bottommost, o["block_size"], o["restart_interval"],
               o["bloom_bits_per_key"], o["target_file_size"])
