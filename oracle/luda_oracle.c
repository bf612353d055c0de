/*
 * luda_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded CPU compactor for the LUDA table format. It exists so
 * that the tests, the smoke check and the benchmark's CPU-baseline leg can check the CUDA
 * path byte for byte. Nothing in the product links, loads or calls it, and it shares no
 * code, header, table or constant generator with the CUDA path.
 *
 * The method (LUDA, arXiv 2004.03054, §II-A "LSM-tree Compaction") is exact: a
 * compaction decodes the input tables (Phase 1, unpack), orders all pairs by key and
 * removes stale and deleted ones (Phase 2, delete and sort), and packs the survivors into
 * new tables with data blocks, checksums, an index and a bloom filter (Phase 3, pack).
 * The paper defers the byte layout to LevelDB; the layout used here is the written
 * LevelDB-style format of this project (varints, prefix-compressed keys with restart
 * points, masked CRC32C trailers, full-key index, per-table bloom filter, no
 * compression). So the oracle is that definition written out, step by step:
 *   1. decode every entry of every input, verifying every checksum and structure rule;
 *   2. sort all entries by the total order (user key asc, trailer desc, input, position);
 *   3. apply the snapshot-aware drop rule in that order;
 *   4. re-encode with the sequential, one-entry-at-a-time table builder loop (flush a
 *      block when its size estimate reaches the block size, finish a file when its
 *      flushed size reaches the target).
 * Format variants, each behind a flag: shortened index keys, ranged compactions, and
 * LevelDB's filter array (one filter per 2 KiB of data block offsets; the paper's
 * prototype is built on LevelDB 1.22, §IV-A, whose tables carry a bloom filter block,
 * §II-A) built by the same loop's block-start steps.
 *
 * Parity pins (tests/test_oracle_*.py): published CRC-32C check values, a bit-at-a-time
 * CRC from the polynomial, MurmurHash3 published values, a hand-worked block example,
 * a brute-force dictionary replay of the generated writes, an independent pure-Python
 * table reader, bloom false-positive rate against its closed form, and structural
 * invariants of every produced table; the filter array against the independent reader's
 * own construction and a hand-worked layout.
 */
#define _POSIX_C_SOURCE 199309L /* clock_gettime */
#include <stdarg.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>

#include "luda_oracle.h"

#define ORA_OK 0
#define ORA_ERR_INVALID_ARG (-1)
#define ORA_ERR_CORRUPTION (-2)
#define ORA_ERR_NOT_SUPPORTED (-3)
#define ORA_ERR_OOM (-4)
#define ORA_ERR_DUPLICATE_KEY (-7)

#define ORA_F_STRICT_DUP 1u
#define ORA_F_SHORT_INDEX 4u /* R9 variant: shortened index keys */
#define ORA_F_FILTER_ARRAY 8u /* R10 variant: one filter per 2 KiB of data block offsets */
#define ORA_F_COMPRESS 16u    /* R4c: data blocks stored Snappy-compressed when that saves 1/8 */

#define ORA_MAGIC 0x4C55444153535431ull
#define ORA_FOOTER 48
#define ORA_TRAILER 5
#define ORA_MAX_SEQ ((1ull << 56) - 1)
static const char ORA_FILTER_NAME[] = "filter.luda.bloom";
static const char ORA_FILTER_ARRAY_NAME[] = "filter.luda.bloom2k";
#define ORA_FILTER_BASE_LG 11u

static char g_detail[512];

static void detail(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_detail, sizeof g_detail, fmt, ap);
  va_end(ap);
}

const char* ora_last_detail(void) { return g_detail; }

/* ------------------------------------------------------------------------------------
 * CRC-32C (Castagnoli), reflected polynomial 0x82F63B78, init and final XOR 0xFFFFFFFF.
 * Every data block carries a checksum over its keys and values (§II-A), computed per
 * block when packing (§III-C, encode kernel) and verified when unpacking.
 * ------------------------------------------------------------------------------------ */
#define ORA_CRC_POLY 0x82F63B78u

/* Bit at a time, straight from the polynomial: shift the register right, XOR the
 * polynomial when the bit shifted out is 1. */
uint32_t ora_crc32c_bitwise(const uint8_t* p, uint64_t n) {
  uint32_t c = 0xFFFFFFFFu;
  for (uint64_t i = 0; i < n; i++) {
    c ^= p[i];
    for (int b = 0; b < 8; b++) c = (c & 1u) ? (c >> 1) ^ ORA_CRC_POLY : (c >> 1);
  }
  return c ^ 0xFFFFFFFFu;
}

/* Byte at a time with a 256-entry table; entry v is the bitwise register update of the
 * single byte v from a zero register. */
static uint32_t g_crc_table[256];
static int g_crc_ready = 0;

static void crc_init(void) {
  if (g_crc_ready) return;
  for (uint32_t v = 0; v < 256; v++) {
    uint32_t c = v;
    for (int b = 0; b < 8; b++) c = (c & 1u) ? (c >> 1) ^ ORA_CRC_POLY : (c >> 1);
    g_crc_table[v] = c;
  }
  g_crc_ready = 1;
}

static uint32_t crc_extend(uint32_t c, const uint8_t* p, uint64_t n) {
  for (uint64_t i = 0; i < n; i++) c = g_crc_table[(c ^ p[i]) & 0xFFu] ^ (c >> 8);
  return c;
}

uint32_t ora_crc32c(const uint8_t* p, uint64_t n) {
  crc_init();
  return crc_extend(0xFFFFFFFFu, p, n) ^ 0xFFFFFFFFu;
}

/* Masked form stored in block trailers: rotate right by 15, add a constant. */
uint32_t ora_mask(uint32_t c) { return ((c >> 15) | (c << 17)) + 0xA282EAD8u; }
uint32_t ora_unmask(uint32_t m) {
  uint32_t r = m - 0xA282EAD8u;
  return (r >> 17) | (r << 15);
}

/* ------------------------------------------------------------------------------------
 * MurmurHash3 x86_32 (A. Appleby, public domain), restated from its published
 * description: 4-byte little-endian blocks mixed with c1/c2 and rotations, a 1-3 byte
 * tail, then the length and the fmix32 finaliser.
 * ------------------------------------------------------------------------------------ */
static uint32_t rotl32(uint32_t x, int r) { return (x << r) | (x >> (32 - r)); }

uint32_t ora_murmur3_32(const uint8_t* p, uint64_t n, uint32_t seed) {
  const uint32_t c1 = 0xcc9e2d51u, c2 = 0x1b873593u;
  uint32_t h = seed;
  uint64_t nblocks = n / 4;
  for (uint64_t i = 0; i < nblocks; i++) {
    uint32_t k = (uint32_t)p[4 * i] | ((uint32_t)p[4 * i + 1] << 8) |
                 ((uint32_t)p[4 * i + 2] << 16) | ((uint32_t)p[4 * i + 3] << 24);
    k *= c1;
    k = rotl32(k, 15);
    k *= c2;
    h ^= k;
    h = rotl32(h, 13);
    h = h * 5u + 0xe6546b64u;
  }
  const uint8_t* tail = p + nblocks * 4;
  uint32_t k = 0;
  switch (n & 3) {
    case 3: k ^= (uint32_t)tail[2] << 16; /* fall through */
    case 2: k ^= (uint32_t)tail[1] << 8;  /* fall through */
    case 1:
      k ^= (uint32_t)tail[0];
      k *= c1;
      k = rotl32(k, 15);
      k *= c2;
      h ^= k;
  }
  h ^= (uint32_t)n;
  h ^= h >> 16;
  h *= 0x85ebca6bu;
  h ^= h >> 13;
  h *= 0xc2b2ae35u;
  h ^= h >> 16;
  return h;
}

/* ------------------------------------------------------------------------------------
 * Growable byte buffer and LEB128 varints.
 * ------------------------------------------------------------------------------------ */
typedef struct {
  uint8_t* p;
  uint64_t n, cap;
} buf_t;

static int buf_reserve(buf_t* b, uint64_t extra) {
  if (b->n + extra <= b->cap) return 0;
  uint64_t cap = b->cap ? b->cap : 256;
  while (cap < b->n + extra) cap *= 2;
  uint8_t* q = (uint8_t*)realloc(b->p, cap);
  if (!q) return -1;
  b->p = q;
  b->cap = cap;
  return 0;
}

static int buf_put(buf_t* b, const void* src, uint64_t n) {
  if (buf_reserve(b, n)) return -1;
  if (n) memcpy(b->p + b->n, src, n);
  b->n += n;
  return 0;
}

static int buf_put_u32(buf_t* b, uint32_t v) {
  uint8_t t[4] = {(uint8_t)v, (uint8_t)(v >> 8), (uint8_t)(v >> 16), (uint8_t)(v >> 24)};
  return buf_put(b, t, 4);
}

static int buf_put_u64(buf_t* b, uint64_t v) {
  uint8_t t[8];
  for (int i = 0; i < 8; i++) t[i] = (uint8_t)(v >> (8 * i));
  return buf_put(b, t, 8);
}

/* Minimal LEB128: 7 bits per byte, low group first, continuation bit 0x80. */
uint32_t ora_put_varint(uint8_t* dst, uint64_t v) {
  uint32_t i = 0;
  while (v >= 0x80) {
    dst[i++] = (uint8_t)(v | 0x80);
    v >>= 7;
  }
  dst[i++] = (uint8_t)v;
  return i;
}

static int buf_put_varint(buf_t* b, uint64_t v) {
  uint8_t t[10];
  return buf_put(b, t, ora_put_varint(t, v));
}

/* Decode a varint of at most max_bytes bytes (5 for 32-bit, 10 for 64-bit) from [p,end).
 * Returns the bytes consumed, or 0 when the run passes `end`, is too long, or the value
 * does not fit in the target width. */
static uint32_t get_varint(const uint8_t* p, const uint8_t* end, int bits, uint64_t* out) {
  int max_bytes = bits == 32 ? 5 : 10;
  uint64_t v = 0;
  for (int i = 0; i < max_bytes; i++) {
    if (p + i >= end) return 0;
    uint64_t b = p[i];
    if (i == 9 && (b & 0x7F) > 1) return 0; /* 64-bit overflow */
    v |= (b & 0x7F) << (7 * i);
    if (!(b & 0x80)) {
      if (bits == 32 && v > 0xFFFFFFFFull) return 0;
      *out = v;
      return (uint32_t)(i + 1);
    }
  }
  return 0;
}

uint64_t ora_get_varint64(const uint8_t* p, uint64_t n, uint64_t* value) {
  return get_varint(p, p + n, 64, value);
}

static uint32_t rd_u32(const uint8_t* p) {
  return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
}

static uint64_t rd_u64(const uint8_t* p) {
  uint64_t v = 0;
  for (int i = 0; i < 8; i++) v |= (uint64_t)p[i] << (8 * i);
  return v;
}

/* ------------------------------------------------------------------------------------
 * Internal keys and their order.
 * ------------------------------------------------------------------------------------ */

/* User keys by memcmp over the common length, a proper prefix first. */
static int cmp_user(const uint8_t* a, uint64_t na, const uint8_t* b, uint64_t nb) {
  uint64_t m = na < nb ? na : nb;
  int c = m ? memcmp(a, b, m) : 0;
  if (c) return c < 0 ? -1 : 1;
  return na < nb ? -1 : (na > nb ? 1 : 0);
}

/* Internal keys: user key ascending, then the trailer (seq << 8 | type) descending. */
static int cmp_internal(const uint8_t* a, uint64_t na, const uint8_t* b, uint64_t nb) {
  int c = cmp_user(a, na - 8, b, nb - 8);
  if (c) return c;
  uint64_t ta = rd_u64(a + na - 8), tb = rd_u64(b + nb - 8);
  return ta > tb ? -1 : (ta < tb ? 1 : 0);
}

/* ------------------------------------------------------------------------------------
 * Block builder (restart interval R) and table builder.
 * Phase 3 "Pack" of §II-A: group pairs into data blocks by the block size, compute
 * the shared key parts and each block's checksum, then the index and bloom filter.
 * ------------------------------------------------------------------------------------ */
typedef struct {
  buf_t buf;
  uint32_t* restarts;
  uint64_t nrest, caprest;
  uint32_t R, counter;
  buf_t last_key;
  uint64_t n;
} bb_t;

static int bb_push_restart(bb_t* bb, uint32_t off) {
  if (bb->nrest == bb->caprest) {
    uint64_t cap = bb->caprest ? bb->caprest * 2 : 16;
    uint32_t* q = (uint32_t*)realloc(bb->restarts, cap * sizeof(uint32_t));
    if (!q) return -1;
    bb->restarts = q;
    bb->caprest = cap;
  }
  bb->restarts[bb->nrest++] = off;
  return 0;
}

static int bb_reset(bb_t* bb) {
  bb->buf.n = 0;
  bb->nrest = 0;
  bb->counter = 0;
  bb->last_key.n = 0;
  bb->n = 0;
  return bb_push_restart(bb, 0);
}

static void bb_free(bb_t* bb) {
  free(bb->buf.p);
  free(bb->restarts);
  free(bb->last_key.p);
  memset(bb, 0, sizeof *bb);
}

/* Append one entry. Entry j of the block is a restart iff j % R == 0; a restart stores
 * shared = 0, every other entry shares its longest common prefix with the previous key. */
static int bb_add(bb_t* bb, const uint8_t* key, uint64_t klen, const uint8_t* val, uint64_t vlen) {
  uint64_t shared = 0;
  if (bb->counter < bb->R) {
    uint64_t m = bb->last_key.n < klen ? bb->last_key.n : klen;
    while (shared < m && bb->last_key.p[shared] == key[shared]) shared++;
  } else {
    if (bb_push_restart(bb, (uint32_t)bb->buf.n)) return -1;
    bb->counter = 0;
  }
  if (buf_put_varint(&bb->buf, shared) || buf_put_varint(&bb->buf, klen - shared) ||
      buf_put_varint(&bb->buf, vlen) || buf_put(&bb->buf, key + shared, klen - shared) ||
      buf_put(&bb->buf, val, vlen))
    return -1;
  bb->last_key.n = 0;
  if (buf_put(&bb->last_key, key, klen)) return -1;
  bb->counter++;
  bb->n++;
  return 0;
}

/* Contents size if the block were finished now: entries, restart array, its count. */
static uint64_t bb_estimate(const bb_t* bb) { return bb->buf.n + bb->nrest * 4 + 4; }

static int bb_finish(bb_t* bb) {
  for (uint64_t i = 0; i < bb->nrest; i++)
    if (buf_put_u32(&bb->buf, bb->restarts[i])) return -1;
  return buf_put_u32(&bb->buf, (uint32_t)bb->nrest);
}

/* Encode a single block of raw (key, value) entries, for the hand-worked example test. */
int ora_encode_block(const uint8_t* keys, const uint64_t* koff, const uint8_t* vals,
                     const uint64_t* voff, uint64_t n, uint32_t R, uint8_t* out, uint64_t cap,
                     uint64_t* out_len) {
  bb_t bb;
  memset(&bb, 0, sizeof bb);
  bb.R = R;
  int rc = ORA_OK;
  if (R == 0 || bb_reset(&bb)) rc = ORA_ERR_INVALID_ARG;
  for (uint64_t i = 0; rc == ORA_OK && i < n; i++)
    if (bb_add(&bb, keys + koff[i], koff[i + 1] - koff[i], vals + voff[i], voff[i + 1] - voff[i]))
      rc = ORA_ERR_OOM;
  if (rc == ORA_OK && bb_finish(&bb)) rc = ORA_ERR_OOM;
  if (rc == ORA_OK) {
    *out_len = bb.buf.n;
    if (bb.buf.n > cap) rc = ORA_ERR_INVALID_ARG;
    else memcpy(out, bb.buf.p, bb.buf.n);
  }
  bb_free(&bb);
  return rc;
}

typedef struct {
  uint8_t* data;
  uint64_t size;
  uint64_t n_entries;
  uint8_t* smallest;
  uint32_t smallest_len;
  uint8_t* largest;
  uint32_t largest_len;
} ora_table;

typedef struct {
  ora_table* tables;
  uint32_t n_tables;
  uint64_t n_in_entries;
  uint64_t n_dropped;
} ora_result;

typedef struct {
  uint64_t T, target;
  uint32_t R, bpk;
  /* the open file */
  int open;
  buf_t file;
  bb_t data, index;
  buf_t fkeys;      /* user keys of the open table, concatenated */
  uint64_t* fkoff;  /* their offsets, n_entries + 1 */
  uint64_t fkcap;
  uint64_t n_entries;
  buf_t smallest, largest;
  /* R9 variant: a flushed block's index entry waits for the next block's first key */
  int short_index, pending;
  buf_t pend_key;
  uint64_t pend_off, pend_size;
  /* R10 variant: the filters generated so far (concatenated), their offsets, and the first
   * entry not yet in a filter */
  int filter_array;
  int compress;     /* R4c */
  buf_t farr;
  uint32_t* foffs;
  uint64_t nfilt, capfilt, fgen;
  /* finished tables */
  ora_table* tables;
  uint32_t n_tables, cap_tables;
} tb_t;

/* Write a block: its stored bytes, then the trailer (type byte, masked CRC32C over the
 * stored bytes and the type). Returns the handle of the block. */
static int write_block_t(buf_t* file, const uint8_t* contents, uint64_t n, uint8_t type, uint64_t* off,
                         uint64_t* size) {
  crc_init();
  *off = file->n;
  *size = n;
  uint32_t c = crc_extend(0xFFFFFFFFu, contents, n);
  c = crc_extend(c, &type, 1) ^ 0xFFFFFFFFu;
  if (buf_put(file, contents, n) || buf_put(file, &type, 1) || buf_put_u32(file, ora_mask(c))) return -1;
  return 0;
}

static int write_block(buf_t* file, const uint8_t* contents, uint64_t n, uint64_t* off, uint64_t* size) {
  return write_block_t(file, contents, n, 0, off, size);
}

/* ------------------------------------------------------------------------------------
 * R4c block compression. The paper leaves Snappy compression to future work (§IV-A);
 * LevelDB, which it builds on, stores a data block compressed (trailer type 1) when
 * that saves at least an eighth of its bytes. The stream is the public Snappy format:
 * varint32 uncompressed length, then elements whose tag's low two bits give the kind:
 *   0 literal: length - 1 in the tag's upper six bits when below 60, else in the next
 *     1..4 bytes (little-endian) for the values 60..63; then the literal bytes;
 *   1 copy: length 4 + bits 2..4, offset = bits 5..7 << 8 | next byte;
 *   2 copy: length 1 + bits 2..7, offset = next 2 bytes (little-endian);
 *   3 copy: length 1 + bits 2..7, offset = next 4 bytes;
 * a copy repeats `length` bytes from `offset` bytes back (1 <= offset <= bytes so far;
 * overlapping copies repeat a pattern).
 * ------------------------------------------------------------------------------------ */
int ora_snappy_uncompress(const uint8_t* in, uint64_t n, uint8_t** out, uint64_t* out_len) {
  *out = NULL;
  *out_len = 0;
  const uint8_t* p = in;
  const uint8_t* end = in + n;
  uint64_t ulen;
  uint32_t a = get_varint(p, end, 32, &ulen);
  if (!a) return ORA_ERR_CORRUPTION;
  p += a;
  uint8_t* o = (uint8_t*)malloc(ulen ? ulen : 1);
  if (!o) return ORA_ERR_OOM;
  uint64_t w = 0;
  while (p < end) {
    const uint8_t tag = *p++;
    const uint32_t kind = tag & 3u;
    uint64_t len, off = 0;
    if (kind == 0) {
      len = tag >> 2;
      if (len >= 60) {
        const uint32_t nb = (uint32_t)len - 59;
        if ((uint64_t)(end - p) < nb) goto bad;
        len = 0;
        for (uint32_t i = 0; i < nb; i++) len |= (uint64_t)p[i] << (8 * i);
        p += nb;
      }
      len += 1;
      if ((uint64_t)(end - p) < len || ulen - w < len) goto bad;
      memcpy(o + w, p, len);
      p += len;
      w += len;
      continue;
    }
    const uint32_t nb = kind == 1 ? 1 : (kind == 2 ? 2 : 4);
    if ((uint64_t)(end - p) < nb) goto bad;
    if (kind == 1) {
      len = 4 + ((tag >> 2) & 7u);
      off = ((uint64_t)(tag >> 5) << 8) | p[0];
    } else {
      len = 1 + (tag >> 2);
      for (uint32_t i = 0; i < nb; i++) off |= (uint64_t)p[i] << (8 * i);
    }
    p += nb;
    if (off == 0 || off > w || ulen - w < len) goto bad;
    for (uint64_t i = 0; i < len; i++, w++) o[w] = o[w - off];
  }
  if (w != ulen) goto bad;
  *out = o;
  *out_len = ulen;
  return ORA_OK;
bad:
  free(o);
  return ORA_ERR_CORRUPTION;
}

/* One literal element of len >= 1 bytes (shortest length form). */
static int sn_literal(buf_t* out, const uint8_t* p, uint64_t len) {
  const uint64_t v = len - 1;
  uint8_t hdr[5];
  uint32_t h = 0;
  if (v < 60) {
    hdr[h++] = (uint8_t)(v << 2);
  } else {
    const uint32_t nb = v < (1u << 8) ? 1 : v < (1u << 16) ? 2 : v < (1u << 24) ? 3 : 4;
    hdr[h++] = (uint8_t)((59 + nb) << 2);
    for (uint32_t i = 0; i < nb; i++) hdr[h++] = (uint8_t)(v >> (8 * i));
  }
  return buf_put(out, hdr, h) || buf_put(out, p, len);
}

static int sn_copy(buf_t* out, uint64_t off, uint64_t len) {
  uint8_t e[3];
  if (len <= 11 && off < 2048) {
    e[0] = (uint8_t)(1u | (uint32_t)(len - 4) << 2 | (uint32_t)(off >> 8) << 5);
    e[1] = (uint8_t)off;
    return buf_put(out, e, 2);
  }
  e[0] = (uint8_t)(2u | (uint32_t)(len - 1) << 2);
  e[1] = (uint8_t)off;
  e[2] = (uint8_t)(off >> 8);
  return buf_put(out, e, 3);
}

/* This format's compressor (the stream format admits many encodings of one block; this
 * one is fixed so that every implementation writes the same bytes). Let H(i) be the
 * 12-bit hash (x * 2654435761 mod 2^32) >> 20 of the little-endian 32-bit word x at
 * position i (defined for i + 4 <= n), and cand(i) the largest j < i with H(j) = H(i),
 * over every position of the block. The block is cut into 64-byte segments [64s, e),
 * e = min(64s + 64, n), each parsed greedily from its start on its own: at position i,
 * if e - i >= 4, cand(i) exists, i - cand(i) < 65536 and the four bytes at cand(i) equal
 * those at i, a copy of offset i - cand(i) and length L = the common length of the two
 * positions' suffixes, at most e - i, is emitted and i moves by L; otherwise byte i joins
 * the pending literal and i moves by one. Pending literal bytes are emitted as one literal
 * element before each copy and at the segment's end. A copy takes the 2-byte form (kind 1)
 * when L <= 11 and the offset is below 2048, else the 3-byte form (kind 2). Segments make
 * the parses independent of each other (a parallel compressor gives each its own thread)
 * and keep every copy within 64 bytes. */
int ora_snappy_compress(const uint8_t* in, uint64_t n, uint8_t** out, uint64_t* out_len) {
  buf_t o = {0};
  int64_t last[4096];
  for (int k = 0; k < 4096; k++) last[k] = -1;
  /* cand of every position, entered in position order */
  int64_t* cand = (int64_t*)malloc((n ? n : 1) * sizeof(int64_t));
  if (!cand) return ORA_ERR_OOM;
  for (uint64_t p = 0; p < n; p++) {
    cand[p] = -1;
    if (p + 4 > n) continue;
    const uint32_t h = (uint32_t)(rd_u32(in + p) * 2654435761u) >> 20;
    cand[p] = last[h];
    last[h] = (int64_t)p;
  }
  int rc = buf_put_varint(&o, n);
  for (uint64_t s0 = 0; rc == 0 && s0 < n; s0 += 64) {
    const uint64_t e = s0 + 64 < n ? s0 + 64 : n;
    uint64_t i = s0, lit = s0;
    while (rc == 0 && i < e) {
      const int64_t j = cand[i];
      if (e - i >= 4 && j >= 0 && i - (uint64_t)j < 65536 && memcmp(in + j, in + i, 4) == 0) {
        uint64_t L = 4;
        while (i + L < e && in[j + L] == in[i + L]) L++;
        rc = (i > lit ? sn_literal(&o, in + lit, i - lit) : 0) || sn_copy(&o, i - (uint64_t)j, L);
        i += L;
        lit = i;
      } else {
        i++;
      }
    }
    if (rc == 0 && e > lit) rc = sn_literal(&o, in + lit, e - lit);
  }
  free(cand);
  if (rc) {
    free(o.p);
    *out = NULL;
    return ORA_ERR_OOM;
  }
  *out = o.p;
  *out_len = o.n;
  return ORA_OK;
}

static int put_handle(buf_t* b, uint64_t off, uint64_t size) {
  return buf_put_varint(b, off) || buf_put_varint(b, size);
}

/* R9 with short index keys. For the last internal key `last` of a block (user key a) and,
 * when another block of the same table follows, that block's first internal key `next`
 * (user key b): let d be the first byte position where a and b differ (next == NULL: the
 * first byte of a that is not 0xFF). If such a position exists, a[d] can be raised by one
 * (below 0xFF; with a next key also still below b[d]) and d + 1 is shorter than a, the
 * index key is a[0..d) || (a[d] + 1) followed by the trailer of the largest sequence
 * number with type 1; otherwise it is `last` itself. Either way last <= key < next in the
 * internal key order. */
static int index_key(const uint8_t* last, uint64_t llen, const uint8_t* next, uint64_t nlen, buf_t* out) {
  const uint64_t ua = llen - 8;
  uint64_t d = 0;
  int shorten = 0;
  if (next) {
    const uint64_t ub = nlen - 8, m = ua < ub ? ua : ub;
    while (d < m && last[d] == next[d]) d++;
    shorten = d < m && last[d] < 0xFF && last[d] + 1 < next[d] && d + 1 < ua;
  } else {
    while (d < ua && last[d] == 0xFF) d++;
    shorten = d < ua && d + 1 < ua;
  }
  out->n = 0;
  if (!shorten) return buf_put(out, last, llen);
  const uint8_t up = (uint8_t)(last[d] + 1);
  return buf_put(out, last, d) || buf_put(out, &up, 1) || buf_put_u64(out, ORA_MAX_SEQ << 8 | 1u);
}

static int tb_add_index(tb_t* tb, const uint8_t* key, uint64_t klen, uint64_t off, uint64_t size) {
  buf_t h = {0};
  int rc = put_handle(&h, off, size) || bb_add(&tb->index, key, klen, h.p, h.n);
  free(h.p);
  return rc;
}

/* The pending index entry, now that the next block's first key (or the end of the table,
 * next == NULL) is known. */
static int tb_resolve_index(tb_t* tb, const uint8_t* next, uint64_t nlen) {
  if (!tb->pending) return 0;
  tb->pending = 0;
  buf_t k = {0};
  int rc = index_key(tb->pend_key.p, tb->pend_key.n, next, nlen, &k) ||
           tb_add_index(tb, k.p, k.n, tb->pend_off, tb->pend_size);
  free(k.p);
  return rc;
}

static int fa_start_block(tb_t* tb, uint64_t off);

static int tb_flush_block(tb_t* tb) {
  uint64_t off, size;
  if (bb_finish(&tb->data)) return -1;
  int stored = 0;
  if (tb->compress) {
    /* R4c: kept compressed when that saves at least an eighth of the raw bytes */
    uint8_t* c;
    uint64_t cn;
    const uint64_t raw = tb->data.buf.n;
    if (ora_snappy_compress(tb->data.buf.p, raw, &c, &cn)) return -1;
    if (cn < raw - raw / 8) {
      stored = 1;
      if (write_block_t(&tb->file, c, cn, 1, &off, &size)) {
        free(c);
        return -1;
      }
    }
    free(c);
  }
  if (!stored && write_block(&tb->file, tb->data.buf.p, tb->data.buf.n, &off, &size)) return -1;
  if (tb->filter_array && fa_start_block(tb, tb->file.n)) return -1;
  if (tb->short_index) {
    tb->pending = 1;
    tb->pend_key.n = 0;
    tb->pend_off = off;
    tb->pend_size = size;
    if (buf_put(&tb->pend_key, tb->data.last_key.p, tb->data.last_key.n)) return -1;
  } else if (tb_add_index(tb, tb->data.last_key.p, tb->data.last_key.n, off, size)) {
    /* Index entry: the block's last internal key, unshortened, and the block's handle. */
    return -1;
  }
  return bb_reset(&tb->data);
}

/* Bloom filter over the user keys of the open table's entries [first, last), appended to
 * out: m = max(64, n*bpk) bits rounded up to whole bytes, k = clamp(bpk*69/100, 1, 30)
 * probes by double hashing h, h+d, h+2d, ... with h = MurmurHash3_x86_32(key, 0) and d = h
 * rotated right by 17; then the byte k. */
static int bloom_append(tb_t* tb, uint64_t first, uint64_t last, buf_t* out) {
  uint64_t n = last - first;
  uint64_t bits = n * tb->bpk;
  if (bits < 64) bits = 64;
  uint64_t bytes = (bits + 7) / 8;
  bits = bytes * 8;
  uint32_t k = tb->bpk * 69 / 100;
  if (k < 1) k = 1;
  if (k > 30) k = 30;
  const uint64_t at = out->n;
  if (buf_reserve(out, bytes + 1)) return -1;
  memset(out->p + at, 0, bytes);
  out->n = at + bytes;
  uint8_t* bm = out->p + at;
  for (uint64_t i = first; i < last; i++) {
    uint32_t h = ora_murmur3_32(tb->fkeys.p + tb->fkoff[i], tb->fkoff[i + 1] - tb->fkoff[i], 0);
    uint32_t d = (h >> 17) | (h << 15);
    for (uint32_t j = 0; j < k; j++) {
      uint64_t b = h % bits;
      bm[b >> 3] |= (uint8_t)(1u << (b & 7));
      h += d;
    }
  }
  uint8_t kb = (uint8_t)k;
  return buf_put(out, &kb, 1);
}

/* R10 filter block: one bloom filter over every entry of the table. */
static int build_filter(tb_t* tb, buf_t* out) {
  out->n = 0;
  return bloom_append(tb, 0, tb->n_entries, out);
}

/* R10 variant, filter array (LevelDB's filter block builder): filter i covers the data
 * blocks whose offset in the table lies in [i * 2 KiB, (i + 1) * 2 KiB). The next filter
 * takes the entries added since the previous one; with none it is empty. */
static int fa_generate(tb_t* tb) {
  if (tb->nfilt == tb->capfilt) {
    uint64_t cap = tb->capfilt ? tb->capfilt * 2 : 64;
    uint32_t* q = (uint32_t*)realloc(tb->foffs, cap * sizeof(uint32_t));
    if (!q) return -1;
    tb->foffs = q;
    tb->capfilt = cap;
  }
  tb->foffs[tb->nfilt++] = (uint32_t)tb->farr.n;
  if (tb->fgen < tb->n_entries && bloom_append(tb, tb->fgen, tb->n_entries, &tb->farr)) return -1;
  tb->fgen = tb->n_entries;
  return 0;
}

/* A data block starts at offset `off` of the table: every filter index below off / 2 KiB
 * is generated (the first of them holds the entries added so far). */
static int fa_start_block(tb_t* tb, uint64_t off) {
  while (tb->nfilt < (off >> ORA_FILTER_BASE_LG))
    if (fa_generate(tb)) return -1;
  return 0;
}

/* Filter array contents: the filters, u32 offset of each, u32 offset of that array, the
 * byte base_lg = 11. The entries of the last block, if no filter holds them yet, get one. */
static int build_filter_array(tb_t* tb, buf_t* out) {
  if (tb->fgen < tb->n_entries && fa_generate(tb)) return -1;
  out->n = 0;
  if (buf_put(out, tb->farr.p, tb->farr.n)) return -1;
  for (uint64_t i = 0; i < tb->nfilt; i++)
    if (buf_put_u32(out, tb->foffs[i])) return -1;
  uint8_t lg = (uint8_t)ORA_FILTER_BASE_LG;
  return buf_put_u32(out, (uint32_t)tb->farr.n) || buf_put(out, &lg, 1);
}

static int tb_finish_file(tb_t* tb) {
  if (tb->data.n > 0 && tb_flush_block(tb)) return -1;
  if (tb_resolve_index(tb, NULL, 0)) return -1;
  uint64_t foff, fsize, moff, msize, ioff, isize;
  buf_t f = {0};
  int rc = (tb->filter_array ? build_filter_array(tb, &f) : build_filter(tb, &f)) ||
           write_block(&tb->file, f.p, f.n, &foff, &fsize);
  free(f.p);
  if (rc) return -1;
  const char* fname = tb->filter_array ? ORA_FILTER_ARRAY_NAME : ORA_FILTER_NAME;
  /* Metaindex: one entry naming the filter block. */
  bb_t meta;
  memset(&meta, 0, sizeof meta);
  meta.R = 1;
  buf_t h = {0};
  rc = bb_reset(&meta) || put_handle(&h, foff, fsize) ||
       bb_add(&meta, (const uint8_t*)fname, strlen(fname), h.p, h.n) ||
       bb_finish(&meta) || write_block(&tb->file, meta.buf.p, meta.buf.n, &moff, &msize);
  free(h.p);
  bb_free(&meta);
  if (rc) return -1;
  if (bb_finish(&tb->index) || write_block(&tb->file, tb->index.buf.p, tb->index.buf.n, &ioff, &isize))
    return -1;
  /* Footer: two handles, zero padding to 40 bytes, the magic. */
  buf_t ft = {0};
  rc = put_handle(&ft, moff, msize) || put_handle(&ft, ioff, isize) || buf_reserve(&ft, 48);
  if (!rc) {
    memset(ft.p + ft.n, 0, 40 - ft.n);
    ft.n = 40;
    rc = buf_put_u64(&ft, ORA_MAGIC) || buf_put(&tb->file, ft.p, ft.n);
  }
  free(ft.p);
  if (rc) return -1;
  /* Emit the table. */
  if (tb->n_tables == tb->cap_tables) {
    uint32_t cap = tb->cap_tables ? tb->cap_tables * 2 : 8;
    ora_table* q = (ora_table*)realloc(tb->tables, cap * sizeof(ora_table));
    if (!q) return -1;
    tb->tables = q;
    tb->cap_tables = cap;
  }
  ora_table* t = &tb->tables[tb->n_tables++];
  memset(t, 0, sizeof *t);
  t->data = tb->file.p;
  t->size = tb->file.n;
  t->n_entries = tb->n_entries;
  t->smallest = tb->smallest.p;
  t->smallest_len = (uint32_t)tb->smallest.n;
  t->largest = tb->largest.p;
  t->largest_len = (uint32_t)tb->largest.n;
  memset(&tb->file, 0, sizeof tb->file);
  memset(&tb->smallest, 0, sizeof tb->smallest);
  memset(&tb->largest, 0, sizeof tb->largest);
  tb->open = 0;
  return 0;
}

/* One builder step, exactly as the sequential loop of a LevelDB-style compaction:
 * add the entry to the open block; if the block's size estimate reached the block size,
 * flush it; if the file's flushed size reached the target, finish the file. */
static int tb_add(tb_t* tb, const uint8_t* key, uint64_t klen, const uint8_t* val, uint64_t vlen) {
  if (!tb->open) {
    tb->open = 1;
    tb->file.n = 0;
    tb->fkeys.n = 0;
    tb->n_entries = 0;
    tb->farr.n = 0;
    tb->nfilt = tb->fgen = 0;
    if (bb_reset(&tb->data) || bb_reset(&tb->index)) return -1;
    if (buf_put(&tb->smallest, key, klen)) return -1;
  }
  if (tb_resolve_index(tb, key, klen)) return -1;
  if (bb_add(&tb->data, key, klen, val, vlen)) return -1;
  if (tb->n_entries + 2 > tb->fkcap) {
    uint64_t cap = tb->fkcap ? tb->fkcap * 2 : 1024;
    uint64_t* q = (uint64_t*)realloc(tb->fkoff, cap * sizeof(uint64_t));
    if (!q) return -1;
    tb->fkoff = q;
    tb->fkcap = cap;
  }
  tb->fkoff[tb->n_entries] = tb->fkeys.n;
  if (buf_put(&tb->fkeys, key, klen - 8)) return -1;
  tb->n_entries++;
  tb->fkoff[tb->n_entries] = tb->fkeys.n;
  tb->largest.n = 0;
  if (buf_put(&tb->largest, key, klen)) return -1;
  if (bb_estimate(&tb->data) >= tb->T && tb_flush_block(tb)) return -1;
  if (tb->file.n >= tb->target && tb_finish_file(tb)) return -1;
  return 0;
}

static void tb_free(tb_t* tb) {
  free(tb->file.p);
  bb_free(&tb->data);
  bb_free(&tb->index);
  free(tb->fkeys.p);
  free(tb->fkoff);
  free(tb->smallest.p);
  free(tb->largest.p);
  free(tb->pend_key.p);
  free(tb->farr.p);
  free(tb->foffs);
}

void ora_free_result(ora_result* r) {
  if (!r) return;
  for (uint32_t i = 0; i < r->n_tables; i++) {
    free(r->tables[i].data);
    free(r->tables[i].smallest);
    free(r->tables[i].largest);
  }
  free(r->tables);
  free(r);
}

static int check_opts(uint64_t T, uint32_t R, uint32_t bpk, uint64_t target) {
  if (T < 1 || R < 1 || R > 65535 || bpk < 1 || bpk > 64 || target < 1) {
    detail("invalid options: block_size=%llu restart_interval=%u bloom_bits_per_key=%u target=%llu",
           (unsigned long long)T, R, bpk, (unsigned long long)target);
    return ORA_ERR_INVALID_ARG;
  }
  return ORA_OK;
}

static void tb_init(tb_t* tb, uint64_t T, uint32_t R, uint32_t bpk, uint64_t target, uint32_t flags) {
  memset(tb, 0, sizeof *tb);
  tb->short_index = (flags & ORA_F_SHORT_INDEX) != 0;
  tb->filter_array = (flags & ORA_F_FILTER_ARRAY) != 0;
  tb->compress = (flags & ORA_F_COMPRESS) != 0;
  tb->T = T;
  tb->R = R;
  tb->bpk = bpk;
  tb->target = target;
  tb->data.R = R;
  tb->index.R = 1;
}

static int tb_take(tb_t* tb, ora_result* res) {
  if (tb->open && tb_finish_file(tb)) return -1;
  res->tables = tb->tables;
  res->n_tables = tb->n_tables;
  tb->tables = NULL;
  tb->n_tables = tb->cap_tables = 0;
  return 0;
}

/* ------------------------------------------------------------------------------------
 * Decoding (Phase 1 "Unpack" of §II-A): verify each block's checksum, then restore
 * the full keys from the shared prefixes.
 * ------------------------------------------------------------------------------------ */
typedef struct {
  uint64_t koff;  /* offset of the full internal key in the key arena */
  uint32_t klen;
  const uint8_t* val;
  uint64_t vlen;
  uint32_t input;
  uint64_t pos;   /* position within its input, in key order */
} ent_t;

typedef struct {
  buf_t keys;
  ent_t* e;
  uint64_t n, cap;
  uint8_t** owned;  /* decompressed blocks the entries' values point into */
  uint64_t n_owned, cap_owned;
} ents_t;

static int ents_own(ents_t* es, uint8_t* p) {
  if (!p) return 0;
  if (es->n_owned == es->cap_owned) {
    uint64_t cap = es->cap_owned ? es->cap_owned * 2 : 64;
    uint8_t** q = (uint8_t**)realloc(es->owned, cap * sizeof(uint8_t*));
    if (!q) {
      free(p);
      return -1;
    }
    es->owned = q;
    es->cap_owned = cap;
  }
  es->owned[es->n_owned++] = p;
  return 0;
}

static void ents_free(ents_t* es) {
  for (uint64_t i = 0; i < es->n_owned; i++) free(es->owned[i]);
  free(es->owned);
  free(es->e);
  free(es->keys.p);
}

static int ents_push(ents_t* es, const uint8_t* key, uint64_t klen, const uint8_t* val, uint64_t vlen,
                     uint32_t input, uint64_t pos) {
  if (es->n == es->cap) {
    uint64_t cap = es->cap ? es->cap * 2 : 1024;
    ent_t* q = (ent_t*)realloc(es->e, cap * sizeof(ent_t));
    if (!q) return -1;
    es->e = q;
    es->cap = cap;
  }
  ent_t* t = &es->e[es->n++];
  t->koff = es->keys.n;
  t->klen = (uint32_t)klen;
  t->val = val;
  t->vlen = vlen;
  t->input = input;
  t->pos = pos;
  return buf_put(&es->keys, key, klen);
}

/* Read the block at handle (off, size) of a file: check bounds, the CRC over the stored
 * bytes and type, then the type byte: 0, or with `type` given also 1 (R4c, compressed),
 * returned there. */
static int read_block_t(const uint8_t* f, uint64_t fsize, uint64_t off, uint64_t size, const char* what,
                        uint32_t input, uint8_t* type) {
  uint64_t limit = fsize - ORA_FOOTER;
  if (off > limit || size > limit - off || ORA_TRAILER > limit - off - size) {
    detail("input %u: %s block handle (%llu,%llu) outside the file", input, what,
           (unsigned long long)off, (unsigned long long)size);
    return ORA_ERR_CORRUPTION;
  }
  crc_init();
  uint32_t want = ora_unmask(rd_u32(f + off + size + 1));
  uint32_t got = crc_extend(0xFFFFFFFFu, f + off, size + 1) ^ 0xFFFFFFFFu;
  if (want != got) {
    detail("input %u: %s block at %llu: checksum mismatch", input, what, (unsigned long long)off);
    return ORA_ERR_CORRUPTION;
  }
  if (f[off + size] != 0 && !(type && f[off + size] == 1)) {
    detail("input %u: %s block at %llu: compression type %u not supported", input, what,
           (unsigned long long)off, f[off + size]);
    return ORA_ERR_NOT_SUPPORTED;
  }
  if (type) *type = f[off + size];
  return ORA_OK;
}

static int read_block(const uint8_t* f, uint64_t fsize, uint64_t off, uint64_t size, const char* what,
                      uint32_t input) {
  return read_block_t(f, fsize, off, size, what, input, NULL);
}

/* A data block's contents: the stored bytes, or for type 1 their decompression (a new
 * buffer in *owned, which the caller frees). */
static int load_data_block(const uint8_t* f, uint64_t fsize, uint64_t off, uint64_t size, uint32_t input,
                           const uint8_t** contents, uint64_t* csize, uint8_t** owned) {
  uint8_t type = 0;
  *owned = NULL;
  int rc = read_block_t(f, fsize, off, size, "data", input, &type);
  if (rc) return rc;
  *contents = f + off;
  *csize = size;
  if (type == 1) {
    rc = ora_snappy_uncompress(f + off, size, owned, csize);
    if (rc == ORA_ERR_CORRUPTION)
      detail("input %u: data block at %llu: malformed compressed stream", input, (unsigned long long)off);
    if (rc) return rc;
    *contents = *owned;
  }
  return ORA_OK;
}

/* Walk a verified block's entries in order, calling `cb` with each full key and value.
 * Enforces the structure rules: at least one restart, offsets strictly increasing from 0,
 * every restart segment starting with shared = 0 and ending exactly at its end. */
typedef int (*entry_cb)(void* ctx, const uint8_t* key, uint64_t klen, const uint8_t* val, uint64_t vlen,
                        int at_restart);

static int walk_block(const uint8_t* b, uint64_t size, buf_t* key, entry_cb cb, void* ctx, const char* what,
                      uint32_t input, uint64_t off) {
  if (size < 4) goto bad;
  uint64_t nr = rd_u32(b + size - 4);
  if (nr < 1 || nr > (size - 4) / 4) goto bad;
  uint64_t rstart = size - 4 - 4 * nr;
  for (uint64_t r = 0; r < nr; r++) {
    uint64_t s = rd_u32(b + rstart + 4 * r);
    uint64_t e = r + 1 < nr ? rd_u32(b + rstart + 4 * (r + 1)) : rstart;
    if ((r == 0 && s != 0) || s >= e || e > rstart) goto bad;
    const uint8_t* p = b + s;
    const uint8_t* end = b + e;
    int first = 1;
    key->n = 0;
    while (p < end) {
      uint64_t shared, nonshared, vlen;
      uint32_t a = get_varint(p, end, 32, &shared);
      if (!a) goto bad;
      p += a;
      a = get_varint(p, end, 32, &nonshared);
      if (!a) goto bad;
      p += a;
      a = get_varint(p, end, 32, &vlen);
      if (!a) goto bad;
      p += a;
      if ((first && shared != 0) || shared > key->n) goto bad;
      if (nonshared > (uint64_t)(end - p) || vlen > (uint64_t)(end - p) - nonshared) goto bad;
      key->n = shared;
      if (buf_put(key, p, nonshared)) return ORA_ERR_OOM;
      p += nonshared;
      int rc = cb(ctx, key->p, key->n, p, vlen, first);
      if (rc) return rc;
      p += vlen;
      first = 0;
    }
  }
  return ORA_OK;
bad:
  detail("input %u: %s block at %llu: malformed contents", input, what, (unsigned long long)off);
  return ORA_ERR_CORRUPTION;
}

typedef struct {
  const uint8_t* f;
  uint64_t fsize;
  uint32_t input;
  uint64_t* off;
  uint64_t* size;
  uint64_t n, cap;
  buf_t keys;       /* index keys, back to back */
  uint64_t* kend;   /* end of index key b in `keys` */
} index_ctx;

static int index_cb(void* vctx, const uint8_t* key, uint64_t klen, const uint8_t* val, uint64_t vlen,
                    int at_restart) {
  index_ctx* c = (index_ctx*)vctx;
  uint64_t off, size;
  uint32_t a, b;
  if (!at_restart) goto bad; /* restart interval 1: every entry starts its own segment */
  a = get_varint(val, val + vlen, 64, &off);
  if (!a) goto bad;
  b = get_varint(val + a, val + vlen, 64, &size);
  if (!b || a + b != vlen) goto bad;
  if (c->n == c->cap) {
    uint64_t cap = c->cap ? c->cap * 2 : 64;
    uint64_t* q1 = (uint64_t*)realloc(c->off, cap * sizeof(uint64_t));
    if (!q1) return ORA_ERR_OOM;
    c->off = q1;
    uint64_t* q2 = (uint64_t*)realloc(c->size, cap * sizeof(uint64_t));
    if (!q2) return ORA_ERR_OOM;
    c->size = q2;
    uint64_t* q3 = (uint64_t*)realloc(c->kend, cap * sizeof(uint64_t));
    if (!q3) return ORA_ERR_OOM;
    c->kend = q3;
    c->cap = cap;
  }
  if (buf_put(&c->keys, key, klen)) return ORA_ERR_OOM;
  c->off[c->n] = off;
  c->size[c->n] = size;
  c->kend[c->n] = c->keys.n;
  c->n++;
  return ORA_OK;
bad:
  detail("input %u: malformed index entry", c->input);
  return ORA_ERR_CORRUPTION;
}

typedef struct {
  ents_t* es;
  uint32_t input;
  uint64_t pos;
} data_ctx;

static int data_cb(void* vctx, const uint8_t* key, uint64_t klen, const uint8_t* val, uint64_t vlen,
                   int at_restart) {
  data_ctx* c = (data_ctx*)vctx;
  (void)at_restart;
  if (klen < 8 || (key[klen - 8] != 0 && key[klen - 8] != 1)) {
    detail("input %u: entry %llu: malformed internal key", c->input, (unsigned long long)c->pos);
    return ORA_ERR_CORRUPTION;
  }
  if (ents_push(c->es, key, klen, val, vlen, c->input, c->pos)) return ORA_ERR_OOM;
  c->pos++;
  return ORA_OK;
}

/* Footer: size >= 48, the magic, two handles inside the file. */
static int read_footer(const uint8_t* f, uint64_t fsize, uint32_t input, uint64_t* moff, uint64_t* msize,
                       uint64_t* ioff, uint64_t* isize) {
  if (fsize < ORA_FOOTER || rd_u64(f + fsize - 8) != ORA_MAGIC) {
    detail("input %u: missing or bad footer", input);
    return ORA_ERR_CORRUPTION;
  }
  const uint8_t* p = f + fsize - ORA_FOOTER;
  const uint8_t* end = p + 40;
  uint32_t a;
  if (!(a = get_varint(p, end, 64, moff))) goto bad;
  p += a;
  if (!(a = get_varint(p, end, 64, msize))) goto bad;
  p += a;
  if (!(a = get_varint(p, end, 64, ioff))) goto bad;
  p += a;
  if (!(a = get_varint(p, end, 64, isize))) goto bad;
  uint64_t limit = fsize - ORA_FOOTER;
  if (*moff > limit || *msize > limit - *moff || ORA_TRAILER > limit - *moff - *msize) goto bad;
  if (*ioff > limit || *isize > limit - *ioff || ORA_TRAILER > limit - *ioff - *isize) goto bad;
  return ORA_OK;
bad:
  detail("input %u: malformed footer handles", input);
  return ORA_ERR_CORRUPTION;
}

/* Decode one input table into `es`, entries in file order; check strict key order. */
/* A user-key range [lo, hi) of a ranged compaction (R13); a NULL bound is unbounded. */
typedef struct {
  const uint8_t* lo;
  uint64_t lo_len;
  const uint8_t* hi;
  uint64_t hi_len;
} range_t;

static int in_range(const range_t* rg, const uint8_t* u, uint64_t n) {
  if (!rg) return 1;
  if (rg->lo && cmp_user(u, n, rg->lo, rg->lo_len) < 0) return 0;
  if (rg->hi && cmp_user(u, n, rg->hi, rg->hi_len) >= 0) return 0;
  return 1;
}

static int decode_input(const uint8_t* f, uint64_t fsize, uint32_t input, ents_t* es, const range_t* rg) {
  uint64_t moff, msize, ioff, isize;
  int rc = read_footer(f, fsize, input, &moff, &msize, &ioff, &isize);
  if (rc) return rc;
  if ((rc = read_block(f, fsize, ioff, isize, "index", input))) return rc;
  index_ctx ic = {f, fsize, input, NULL, NULL, 0, 0, {0}, NULL};
  buf_t key = {0};
  rc = walk_block(f + ioff, isize, &key, index_cb, &ic, "index", input, ioff);
  uint64_t first = es->n;
  data_ctx dc = {es, input, 0};
  int prev_read = 0;
  for (uint64_t b = 0; rc == ORA_OK && b < ic.n; b++) {
    const uint64_t before = es->n;
    /* R13: a ranged compaction reads block b only when it can hold keys of [lo, hi): its
     * index key's user key is not below lo, and the previous block's is below hi */
    if (rg) {
      const uint64_t k0 = b ? ic.kend[b - 1] : 0, kl = ic.kend[b] - k0;
      int rd = 1;
      if (rg->lo && kl >= 8 && cmp_user(ic.keys.p + k0, kl - 8, rg->lo, rg->lo_len) < 0) rd = 0;
      if (rd && b > 0 && rg->hi) {
        const uint64_t p0 = b > 1 ? ic.kend[b - 2] : 0, pl = ic.kend[b - 1] - p0;
        if (pl >= 8 && cmp_user(ic.keys.p + p0, pl - 8, rg->hi, rg->hi_len) >= 0) rd = 0;
      }
      if (!rd) {
        prev_read = 0;
        continue;
      }
    }
    const uint8_t* contents = NULL;
    uint64_t csize = 0;
    uint8_t* owned = NULL;
    rc = load_data_block(f, fsize, ic.off[b], ic.size[b], input, &contents, &csize, &owned);
    if (rc == ORA_OK && ents_own(es, owned)) rc = ORA_ERR_OOM;
    if (rc == ORA_OK) rc = walk_block(contents, csize, &key, data_cb, &dc, "data", input, ic.off[b]);
    /* R9: a data block's index key is at or above its last internal key, and the previous
     * block's index key is below this block's first internal key */
    if (rc == ORA_OK) {
      const uint64_t k0 = b ? ic.kend[b - 1] : 0, kl = ic.kend[b] - k0;
      const ent_t* last = es->n > before ? &es->e[es->n - 1] : NULL;
      if (!last || kl < 8 || cmp_internal(es->keys.p + last->koff, last->klen, ic.keys.p + k0, kl) > 0) {
        detail("input %u: index key of data block %llu is below its last key", input, (unsigned long long)b);
        rc = ORA_ERR_CORRUPTION;
      } else if (b > 0 && prev_read) {
        const uint64_t p0 = b > 1 ? ic.kend[b - 2] : 0, pl = ic.kend[b - 1] - p0;
        const ent_t* first = &es->e[before];
        if (cmp_internal(ic.keys.p + p0, pl, es->keys.p + first->koff, first->klen) >= 0) {
          detail("input %u: index key of data block %llu is not below the next block's first key", input,
                 (unsigned long long)(b - 1));
          rc = ORA_ERR_CORRUPTION;
        }
      }
    }
    prev_read = 1;
  }
  free(ic.off);
  free(ic.size);
  free(ic.kend);
  free(ic.keys.p);
  free(key.p);
  for (uint64_t i = first + 1; rc == ORA_OK && i < es->n; i++) {
    const ent_t* a = &es->e[i - 1];
    const ent_t* b = &es->e[i];
    if (cmp_internal(es->keys.p + a->koff, a->klen, es->keys.p + b->koff, b->klen) >= 0) {
      detail("input %u: entries %llu and %llu out of order", input, (unsigned long long)a->pos,
             (unsigned long long)b->pos);
      rc = ORA_ERR_CORRUPTION;
    }
  }
  return rc;
}

/* ------------------------------------------------------------------------------------
 * Compaction: Phases 1-3 of §II-A, in order.
 * ------------------------------------------------------------------------------------ */
static const uint8_t* g_sort_keys;

/* The total order: internal key order, then input index, then position. */
static int cmp_entry(const void* va, const void* vb) {
  const ent_t* a = (const ent_t*)va;
  const ent_t* b = (const ent_t*)vb;
  int c = cmp_internal(g_sort_keys + a->koff, a->klen, g_sort_keys + b->koff, b->klen);
  if (c) return c;
  if (a->input != b->input) return a->input < b->input ? -1 : 1;
  return a->pos < b->pos ? -1 : (a->pos > b->pos ? 1 : 0);
}

int ora_compact_range(const uint8_t* const* datas, const uint64_t* sizes, uint32_t n_inputs,
                      uint64_t smallest_snapshot, int32_t bottommost, uint64_t block_size, uint32_t restart_interval,
                      uint32_t bloom_bits_per_key, uint64_t target_file_size, uint32_t flags, const uint8_t* lo,
                      uint64_t lo_len, const uint8_t* hi, uint64_t hi_len, ora_result** out) {
  range_t range = {lo, lo_len, hi, hi_len};
  const range_t* rg = (lo || hi) ? &range : NULL;
  g_detail[0] = 0;
  *out = NULL;
  int rc = check_opts(block_size, restart_interval, bloom_bits_per_key, target_file_size);
  if (rc) return rc;
  if (n_inputs > 0 && (!datas || !sizes)) return ORA_ERR_INVALID_ARG;
  ents_t es;
  memset(&es, 0, sizeof es);
  /* Phase 1: unpack every input. */
  for (uint32_t i = 0; rc == ORA_OK && i < n_inputs; i++) rc = decode_input(datas[i], sizes[i], i, &es, rg);
  ora_result* res = (ora_result*)calloc(1, sizeof(ora_result));
  if (!res && rc == ORA_OK) rc = ORA_ERR_OOM;
  /* Phase 2: sort all pairs in the total order, then drop stale versions and, at the
   * bottommost level, tombstones (the snapshot-aware rule of LevelDB compactions). */
  if (rc == ORA_OK && es.n > 1) {
    g_sort_keys = es.keys.p;
    qsort(es.e, es.n, sizeof(ent_t), cmp_entry);
  }
  if (rc == ORA_OK && (flags & ORA_F_STRICT_DUP)) {
    for (uint64_t i = 1; i < es.n; i++) {
      const ent_t* a = &es.e[i - 1];
      const ent_t* b = &es.e[i];
      if (a->klen == b->klen && memcmp(es.keys.p + a->koff, es.keys.p + b->koff, a->klen) == 0) {
        detail("duplicate internal key in inputs %u and %u", a->input, b->input);
        rc = ORA_ERR_DUPLICATE_KEY;
        break;
      }
    }
  }
  tb_t tb;
  tb_init(&tb, block_size, restart_interval, bloom_bits_per_key, target_file_size, flags);
  uint64_t dropped = 0;
  if (rc == ORA_OK) {
    const uint64_t INF = ~0ull;
    uint64_t last_seq = INF;
    for (uint64_t i = 0; rc == ORA_OK && i < es.n; i++) {
      const ent_t* e = &es.e[i];
      const uint8_t* k = es.keys.p + e->koff;
      if (i > 0) {
        const ent_t* p = &es.e[i - 1];
        if (cmp_user(es.keys.p + p->koff, p->klen - 8, k, e->klen - 8) != 0) last_seq = INF;
      }
      uint64_t tr = rd_u64(k + e->klen - 8);
      uint64_t seq = tr >> 8;
      int is_del = (tr & 0xFF) == 0;
      int drop = 0;
      if (!in_range(rg, k, e->klen - 8)) drop = 1; /* R13: only keys of the range are written */
      else if (last_seq != INF && last_seq <= smallest_snapshot) drop = 1;
      else if (is_del && seq <= smallest_snapshot && bottommost) drop = 1;
      last_seq = seq;
      if (drop) {
        dropped++;
        continue;
      }
      /* Phase 3: pack the survivor. */
      if (tb_add(&tb, k, e->klen, e->val, e->vlen)) rc = ORA_ERR_OOM;
    }
    if (rc == ORA_OK && tb_take(&tb, res)) rc = ORA_ERR_OOM;
    if (rc == ORA_OK) {
      res->n_in_entries = es.n;
      res->n_dropped = dropped;
    }
  }
  tb_free(&tb);
  for (uint32_t i = 0; i < tb.n_tables; i++) {
    free(tb.tables[i].data);
    free(tb.tables[i].smallest);
    free(tb.tables[i].largest);
  }
  free(tb.tables);
  ents_free(&es);
  if (rc != ORA_OK) {
    ora_free_result(res);
    return rc;
  }
  *out = res;
  return ORA_OK;
}

int ora_compact(const uint8_t* const* datas, const uint64_t* sizes, uint32_t n_inputs, uint64_t smallest_snapshot,
                int32_t bottommost, uint64_t block_size, uint32_t restart_interval, uint32_t bloom_bits_per_key,
                uint64_t target_file_size, uint32_t flags, ora_result** out) {
  return ora_compact_range(datas, sizes, n_inputs, smallest_snapshot, bottommost, block_size, restart_interval,
                           bloom_bits_per_key, target_file_size, flags, NULL, 0, NULL, 0, out);
}

/* Build tables from entries the caller already sorted (a memtable flush): user keys,
 * sequence numbers and types form the internal keys; the same builder loop as a
 * compaction packs them, cutting files at the target size. Unsorted input, seq >= 2^56 or
 * a type other than 0/1 is an invalid argument. */
int ora_build(const uint8_t* ukeys, const uint64_t* ukoff, const uint64_t* seqs, const uint8_t* types,
              const uint8_t* vals, const uint64_t* voff, uint64_t n, uint64_t block_size, uint32_t restart_interval,
              uint32_t bloom_bits_per_key, uint64_t target_file_size, uint32_t flags, ora_result** out) {
  g_detail[0] = 0;
  *out = NULL;
  int rc = check_opts(block_size, restart_interval, bloom_bits_per_key, target_file_size);
  if (rc) return rc;
  ora_result* res = (ora_result*)calloc(1, sizeof(ora_result));
  if (!res) return ORA_ERR_OOM;
  tb_t tb;
  tb_init(&tb, block_size, restart_interval, bloom_bits_per_key, target_file_size, flags);
  buf_t prev = {0}, cur = {0};
  for (uint64_t i = 0; rc == ORA_OK && i < n; i++) {
    if (seqs[i] > ORA_MAX_SEQ || types[i] > 1) {
      detail("entry %llu: sequence or type out of range", (unsigned long long)i);
      rc = ORA_ERR_INVALID_ARG;
      break;
    }
    cur.n = 0;
    if (buf_put(&cur, ukeys + ukoff[i], ukoff[i + 1] - ukoff[i]) || buf_put_u64(&cur, seqs[i] << 8 | types[i])) {
      rc = ORA_ERR_OOM;
      break;
    }
    if (i > 0 && cmp_internal(prev.p, prev.n, cur.p, cur.n) >= 0) {
      detail("entries %llu and %llu are not in increasing internal key order", (unsigned long long)(i - 1),
             (unsigned long long)i);
      rc = ORA_ERR_INVALID_ARG;
      break;
    }
    if (tb_add(&tb, cur.p, cur.n, vals + voff[i], voff[i + 1] - voff[i])) rc = ORA_ERR_OOM;
    buf_t t = prev;
    prev = cur;
    cur = t;
  }
  if (rc == ORA_OK && tb_take(&tb, res)) rc = ORA_ERR_OOM;
  if (rc == ORA_OK) res->n_in_entries = n;
  tb_free(&tb);
  for (uint32_t i = 0; i < tb.n_tables; i++) {
    free(tb.tables[i].data);
    free(tb.tables[i].smallest);
    free(tb.tables[i].largest);
  }
  free(tb.tables);
  free(prev.p);
  free(cur.p);
  if (rc != ORA_OK) {
    ora_free_result(res);
    return rc;
  }
  *out = res;
  return ORA_OK;
}

/* ------------------------------------------------------------------------------------
 * Table reader for the invariant tests: every block verified, entries returned in order,
 * plus the layout facts the invariants need.
 * ------------------------------------------------------------------------------------ */
typedef struct {
  uint8_t* keys;       /* internal keys, concatenated */
  uint64_t* koff;      /* n + 1 */
  uint8_t* vals;
  uint64_t* voff;      /* n + 1 */
  uint64_t n;
  uint64_t n_blocks;
  uint64_t* blk_off;   /* data block handles */
  uint64_t* blk_size;
  uint64_t* blk_last;  /* entry index of each block's last entry */
  uint32_t index_keys_ok;   /* every index key lies in [its block's last key, the next block's first key) */
  uint32_t index_keys_exact; /* every index key equals its block's last key */
  uint32_t layout_ok;       /* data blocks tile [0, filter) and the blocks follow in order */
  uint64_t filter_off, filter_size;
  uint32_t filter_array;    /* the filter block is a filter array (R10 variant) */
} ora_read;

typedef struct {
  buf_t keys, vals;
  uint64_t *koff, *voff;
  uint64_t n, cap;
} rd_ctx;

static int rd_cb(void* vctx, const uint8_t* key, uint64_t klen, const uint8_t* val, uint64_t vlen, int at_restart) {
  rd_ctx* c = (rd_ctx*)vctx;
  (void)at_restart;
  if (klen < 8 || (key[klen - 8] != 0 && key[klen - 8] != 1)) return ORA_ERR_CORRUPTION;
  if (c->n + 2 > c->cap) {
    uint64_t cap = c->cap ? c->cap * 2 : 1024;
    uint64_t* q1 = (uint64_t*)realloc(c->koff, cap * sizeof(uint64_t));
    if (!q1) return ORA_ERR_OOM;
    c->koff = q1;
    uint64_t* q2 = (uint64_t*)realloc(c->voff, cap * sizeof(uint64_t));
    if (!q2) return ORA_ERR_OOM;
    c->voff = q2;
    c->cap = cap;
  }
  c->koff[c->n] = c->keys.n;
  c->voff[c->n] = c->vals.n;
  if (buf_put(&c->keys, key, klen) || buf_put(&c->vals, val, vlen)) return ORA_ERR_OOM;
  c->n++;
  c->koff[c->n] = c->keys.n;
  c->voff[c->n] = c->vals.n;
  return ORA_OK;
}

typedef struct {
  buf_t name;
  uint64_t off, size;
  int found, array;
} meta_ctx;

static int meta_cb(void* vctx, const uint8_t* key, uint64_t klen, const uint8_t* val, uint64_t vlen, int at_restart) {
  meta_ctx* c = (meta_ctx*)vctx;
  (void)at_restart;
  const int plain = klen == sizeof ORA_FILTER_NAME - 1 && memcmp(key, ORA_FILTER_NAME, klen) == 0;
  const int array = klen == sizeof ORA_FILTER_ARRAY_NAME - 1 && memcmp(key, ORA_FILTER_ARRAY_NAME, klen) == 0;
  if (plain || array) {
    if (c->found) return ORA_ERR_CORRUPTION;
    c->array = array;
    uint32_t a = get_varint(val, val + vlen, 64, &c->off);
    if (!a) return ORA_ERR_CORRUPTION;
    uint32_t b = get_varint(val + a, val + vlen, 64, &c->size);
    if (!b || a + b != vlen) return ORA_ERR_CORRUPTION;
    c->found = 1;
  }
  return ORA_OK;
}

typedef struct {
  index_ctx ic;
  buf_t lastkeys;
  uint64_t* lkoff;
  uint64_t lcap;
} ridx_ctx;

static int ridx_cb(void* vctx, const uint8_t* key, uint64_t klen, const uint8_t* val, uint64_t vlen, int at_restart) {
  ridx_ctx* c = (ridx_ctx*)vctx;
  int rc = index_cb(&c->ic, key, klen, val, vlen, at_restart);
  if (rc) return rc;
  if (c->ic.n + 1 > c->lcap) {
    uint64_t cap = c->lcap ? c->lcap * 2 : 64;
    uint64_t* q = (uint64_t*)realloc(c->lkoff, cap * sizeof(uint64_t));
    if (!q) return ORA_ERR_OOM;
    c->lkoff = q;
    c->lcap = cap;
  }
  c->lkoff[c->ic.n - 1] = c->lastkeys.n;
  c->lkoff[c->ic.n] = c->lastkeys.n + klen;
  return buf_put(&c->lastkeys, key, klen) ? ORA_ERR_OOM : ORA_OK;
}

void ora_free_read(ora_read* r) {
  if (!r) return;
  free(r->keys);
  free(r->koff);
  free(r->vals);
  free(r->voff);
  free(r->blk_off);
  free(r->blk_size);
  free(r->blk_last);
  free(r);
}

int ora_read_table(const uint8_t* f, uint64_t fsize, ora_read** out) {
  g_detail[0] = 0;
  *out = NULL;
  uint64_t moff, msize, ioff, isize;
  int rc = read_footer(f, fsize, 0, &moff, &msize, &ioff, &isize);
  if (rc) return rc;
  if ((rc = read_block(f, fsize, ioff, isize, "index", 0))) return rc;
  if ((rc = read_block(f, fsize, moff, msize, "metaindex", 0))) return rc;
  buf_t key = {0};
  ridx_ctx ri;
  memset(&ri, 0, sizeof ri);
  ri.ic.f = f;
  ri.ic.fsize = fsize;
  rc = walk_block(f + ioff, isize, &key, ridx_cb, &ri, "index", 0, ioff);
  meta_ctx mc;
  memset(&mc, 0, sizeof mc);
  if (rc == ORA_OK) rc = walk_block(f + moff, msize, &key, meta_cb, &mc, "metaindex", 0, moff);
  if (rc == ORA_OK && !mc.found) rc = ORA_ERR_CORRUPTION;
  if (rc == ORA_OK) rc = read_block(f, fsize, mc.off, mc.size, "filter", 0);
  ora_read* r = (ora_read*)calloc(1, sizeof(ora_read));
  rd_ctx dc;
  memset(&dc, 0, sizeof dc);
  uint64_t* blk_last = (uint64_t*)calloc(ri.ic.n + 1, sizeof(uint64_t));
  if (!r || !blk_last) rc = rc ? rc : ORA_ERR_OOM;
  uint32_t keys_ok = 1, keys_exact = 1, layout_ok = 1;
  uint64_t expect = 0;
  for (uint64_t b = 0; rc == ORA_OK && b < ri.ic.n; b++) {
    if (ri.ic.off[b] != expect) layout_ok = 0;
    expect = ri.ic.off[b] + ri.ic.size[b] + ORA_TRAILER;
    const uint8_t* contents = NULL;
    uint64_t csize = 0;
    uint8_t* owned = NULL;
    rc = load_data_block(f, fsize, ri.ic.off[b], ri.ic.size[b], 0, &contents, &csize, &owned);
    if (rc == ORA_OK) rc = walk_block(contents, csize, &key, rd_cb, &dc, "data", 0, ri.ic.off[b]);
    free(owned);
    if (rc == ORA_OK) {
      if (dc.n == 0) {
        rc = ORA_ERR_CORRUPTION;
        break;
      }
      const uint64_t first = b ? blk_last[b - 1] + 1 : 0;
      blk_last[b] = dc.n - 1;
      const uint64_t lk = dc.koff[dc.n] - dc.koff[dc.n - 1], ik = ri.lkoff[b + 1] - ri.lkoff[b];
      const uint8_t* ikey = ri.lastkeys.p + ri.lkoff[b];
      if (lk != ik || memcmp(dc.keys.p + dc.koff[dc.n - 1], ikey, lk) != 0) keys_exact = 0;
      if (ik < 8 || cmp_internal(dc.keys.p + dc.koff[dc.n - 1], lk, ikey, ik) > 0) keys_ok = 0;
      if (b > 0) {
        const uint64_t pk = ri.lkoff[b] - ri.lkoff[b - 1];
        if (pk < 8 || cmp_internal(ri.lastkeys.p + ri.lkoff[b - 1], pk, dc.keys.p + dc.koff[first],
                                   dc.koff[first + 1] - dc.koff[first]) >= 0)
          keys_ok = 0;
      }
    }
  }
  if (rc == ORA_OK) {
    /* data blocks, filter, metaindex, index, footer: back to back */
    if (mc.off != expect) layout_ok = 0;
    if (moff != mc.off + mc.size + ORA_TRAILER) layout_ok = 0;
    if (ioff != moff + msize + ORA_TRAILER) layout_ok = 0;
    if (ioff + isize + ORA_TRAILER + ORA_FOOTER != fsize) layout_ok = 0;
    if (ri.ic.n == 0) layout_ok = 0;
  }
  free(key.p);
  free(ri.lastkeys.p);
  free(ri.lkoff);
  free(ri.ic.keys.p);
  free(ri.ic.kend);
  if (rc != ORA_OK) {
    free(ri.ic.off);
    free(ri.ic.size);
    free(blk_last);
    free(dc.keys.p);
    free(dc.vals.p);
    free(dc.koff);
    free(dc.voff);
    free(r);
    return rc;
  }
  if (dc.n == 0) {
    dc.koff = (uint64_t*)calloc(1, sizeof(uint64_t));
    dc.voff = (uint64_t*)calloc(1, sizeof(uint64_t));
  }
  r->keys = dc.keys.p;
  r->koff = dc.koff;
  r->vals = dc.vals.p;
  r->voff = dc.voff;
  r->n = dc.n;
  r->n_blocks = ri.ic.n;
  r->blk_off = ri.ic.off;
  r->blk_size = ri.ic.size;
  r->blk_last = blk_last;
  r->index_keys_ok = keys_ok;
  r->index_keys_exact = keys_exact;
  r->layout_ok = layout_ok;
  r->filter_off = mc.off;
  r->filter_size = mc.size;
  r->filter_array = (uint32_t)mc.array;
  *out = r;
  return ORA_OK;
}

/* Membership query against a filter array's contents for a key of the data block at
 * offset block_off: the filter of index block_off >> base_lg decides; an empty one holds
 * nothing; a malformed array answers "may contain". */
int ora_bloom_may_contain(const uint8_t* filter, uint64_t len, const uint8_t* ukey, uint64_t ulen);
int ora_filter_array_may_contain(const uint8_t* fa, uint64_t len, uint64_t block_off, const uint8_t* ukey,
                                 uint64_t ulen) {
  if (len < 5) return 1;
  const uint32_t lg = fa[len - 1];
  const uint64_t arr = rd_u32(fa + len - 5);
  if (arr > len - 5 || lg > 63) return 1;
  const uint64_t num = (len - 5 - arr) / 4, i = block_off >> lg;
  if (i >= num) return 1;
  const uint64_t start = rd_u32(fa + arr + 4 * i);
  const uint64_t limit = i + 1 < num ? rd_u32(fa + arr + 4 * (i + 1)) : arr;
  if (start == limit) return 0;
  if (start > limit || limit > arr) return 1;
  return ora_bloom_may_contain(fa + start, limit - start, ukey, ulen);
}

/* Bloom membership query against a filter block's contents (bitmap || k). */
int ora_bloom_may_contain(const uint8_t* filter, uint64_t len, const uint8_t* ukey, uint64_t ulen) {
  if (len < 2) return 1;
  uint64_t bits = (len - 1) * 8;
  uint32_t k = filter[len - 1];
  uint32_t h = ora_murmur3_32(ukey, ulen, 0);
  uint32_t d = (h >> 17) | (h << 15);
  for (uint32_t j = 0; j < k; j++) {
    uint64_t b = h % bits;
    if (!(filter[b >> 3] & (1u << (b & 7)))) return 0;
    h += d;
  }
  return 1;
}

/* ------------------------------------------------------------------------------------
 * luda_compact's C ABI (include/luda_oracle.h): the same arguments, served by
 * ora_compact above. Only marshalling: the flags are checked, the inputs handed over,
 * the result's tables moved into the caller's outputs.
 * ------------------------------------------------------------------------------------ */
int luda_oracle_compact(const luda_oracle_input* inputs, uint32_t n_inputs, int32_t level,
                        uint64_t smallest_snapshot, const luda_oracle_options* opts, luda_oracle_outputs* out) {
  (void)level;
  if (!out) return ORA_ERR_INVALID_ARG;
  memset(out, 0, sizeof *out);
  const uint32_t known = ORA_F_STRICT_DUP | 2u /* trace: nothing to record */ | ORA_F_SHORT_INDEX |
                         ORA_F_FILTER_ARRAY | ORA_F_COMPRESS;
  if (!opts || (n_inputs && !inputs) || (opts->flags & ~known)) {
    out->status = ORA_ERR_INVALID_ARG;
    return ORA_ERR_INVALID_ARG;
  }
  const uint8_t** datas = (const uint8_t**)malloc(sizeof(uint8_t*) * (n_inputs ? n_inputs : 1));
  uint64_t* sizes = (uint64_t*)malloc(sizeof(uint64_t) * (n_inputs ? n_inputs : 1));
  if (!datas || !sizes) {
    free(datas);
    free(sizes);
    out->status = ORA_ERR_OOM;
    return ORA_ERR_OOM;
  }
  int rc = ORA_OK;
  for (uint32_t i = 0; i < n_inputs; i++) {
    datas[i] = inputs[i].data;
    sizes[i] = inputs[i].size;
    if (!datas[i] && sizes[i]) rc = ORA_ERR_INVALID_ARG;
  }
  ora_result* res = NULL;
  struct timespec t0, t1;
  clock_gettime(CLOCK_MONOTONIC, &t0);
  if (rc == ORA_OK)
    rc = ora_compact(datas, sizes, n_inputs, smallest_snapshot, opts->bottommost, opts->block_size,
                     opts->restart_interval, opts->bloom_bits_per_key, opts->target_file_size,
                     opts->flags & ~2u, &res);
  clock_gettime(CLOCK_MONOTONIC, &t1);
  free(datas);
  free(sizes);
  if (rc == ORA_OK) {
    out->tables = (luda_oracle_table*)calloc(res->n_tables ? res->n_tables : 1, sizeof(luda_oracle_table));
    if (!out->tables) {
      ora_free_result(res);
      rc = ORA_ERR_OOM;
    }
  }
  if (rc != ORA_OK) {
    out->status = rc;
    return rc;
  }
  for (uint32_t i = 0; i < res->n_tables; i++) {
    const ora_table* t = &res->tables[i];
    luda_oracle_table* o = &out->tables[i];
    o->data = t->data;
    o->size = t->size;
    o->n_entries = t->n_entries;
    o->smallest = t->smallest;
    o->smallest_len = t->smallest_len;
    o->largest = t->largest;
    o->largest_len = t->largest_len;
  }
  out->n_tables = res->n_tables;
  out->n_in_entries = res->n_in_entries;
  out->n_dropped = res->n_dropped;
  out->ms_device = (double)(t1.tv_sec - t0.tv_sec) * 1e3 + (double)(t1.tv_nsec - t0.tv_nsec) * 1e-6;
  out->_priv = res; /* owns the table bytes and keys */
  return ORA_OK;
}

void luda_oracle_outputs_free(luda_oracle_outputs* out) {
  if (!out) return;
  ora_free_result((ora_result*)out->_priv);
  free(out->tables);
  memset(out, 0, sizeof *out);
}
