"""The oracle under AddressSanitizer and UndefinedBehaviorSanitizer (CPU): built from its
source with the sanitizers, it compacts the same jobs (valid and corrupt) to the same bytes
and status as the plain build, with no sanitizer report."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
from helpers import U64MAX, oracle_inputs
from paper_2004_03054_b300 import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def exe(tmp_path_factory):
    if shutil.which("gcc") is None:
        pytest.skip("no gcc")
    path = str(tmp_path_factory.mktemp("asan") / "oracle_asan")
    r = subprocess.run(["gcc", "-std=c11", "-O1", "-g", "-fno-omit-frame-pointer", "-fsanitize=address,undefined",
                        "-I", os.path.join(os.path.dirname(HERE), "include"),
                        "-fno-sanitize-recover=undefined", "-o", path, os.path.join(HERE, "oracle_sanitize_main.c")],
                       capture_output=True, text=True)
    if r.returncode != 0 and "sanitize" in r.stderr:
        pytest.skip("this gcc has no sanitizer runtime: " + r.stderr[-200:])
    assert r.returncode == 0, r.stderr
    return path


def _run(exe, tmp_path, job, inputs, flags=0):
    files = []
    for i, b in enumerate(inputs):
        p = tmp_path / f"in{i}.sst"
        p.write_bytes(b)
        files.append(str(p))
    out = tmp_path / "out.bin"
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=1:abort_on_error=1", UBSAN_OPTIONS="print_stacktrace=1")
    r = subprocess.run([exe, str(out), str(job.smallest_snapshot), str(int(job.bottommost)), str(job.block_size),
                        str(job.restart_interval), str(job.bloom_bits_per_key), str(job.target_file_size), str(flags)]
                       + files, capture_output=True, text=True, env=env, timeout=300)
    assert r.returncode == 0 and "runtime error" not in r.stderr and "ERROR: AddressSanitizer" not in r.stderr, \
        r.stderr[-2000:]
    data = out.read_bytes()
    head, rest = data.split(b"\n", 1)
    rc, n = (int(x) for x in head.split())
    tables = []
    for _ in range(n):
        size_line, rest = rest.split(b"\n", 1)
        size = int(size_line)
        tables.append(rest[:size])
        rest = rest[size:]
    return rc, tables


def _plain(job, inputs, flags=0):
    res = oracle.compact(inputs, job.smallest_snapshot, job.bottommost, job.block_size, job.restart_interval,
                         job.bloom_bits_per_key, job.target_file_size, flags)
    return res.status, [t.data for t in res.tables]


@pytest.mark.parametrize("seed", range(4))
def test_sanitized_oracle_matches_plain_build(exe, tmp_path, seed):
    rng = np.random.default_rng(900 + seed)
    job = W.tiny_job(rng, n_keys=int(rng.integers(20, 300)), max_versions=4, n_inputs=int(rng.integers(1, 5)),
                     key_len=(0, 40), val_len=(0, 600))
    job.block_size, job.target_file_size = 512, 8192
    ins = oracle_inputs(job)
    assert _run(exe, tmp_path, job, ins) == _plain(job, ins)


def test_sanitized_oracle_on_config1_and_corrupt_inputs(exe, tmp_path):
    job = W.config1(seed=7, scale=1 / 64)
    ins = oracle_inputs(job)
    assert _run(exe, tmp_path, job, ins) == _plain(job, ins)
    bad = bytearray(ins[1])
    bad[40] ^= 0x10                          # a data block's bytes: checksum mismatch
    cases = [[ins[0], bytes(bad)] + ins[2:], [ins[0][:-7]] + ins[1:], [b"\x00" * 47] + ins[1:],
             [bytes(np.random.default_rng(1).integers(0, 256, 3000, dtype=np.uint8))] + ins[1:]]
    for c in cases:
        rc, tables = _run(exe, tmp_path, job, c)
        assert (rc, tables) == _plain(job, c) and rc != 0 and not tables


def test_sanitized_oracle_strict_duplicates(exe, tmp_path):
    job = W.config1(seed=8, scale=1 / 128)
    ins = oracle_inputs(job)
    job.target_file_size = U64MAX
    assert _run(exe, tmp_path, job, [ins[0], ins[0]], flags=1) == _plain(job, [ins[0], ins[0]], flags=1)
