// crc_tables.cu -- host-side generation of the CRC-32C lookup tables used on the device.
//
// Everything is derived from the reflected Castagnoli polynomial 0x82F63B78:
//   * slice[0][v]: eight bit-steps of the register holding v (shift right, XOR the
//     polynomial when the bit shifted out is 1); slice[k][v] = slice[0] step applied to
//     slice[k-1][v] (slicing-by-4).
//   * Z1, the 32x32 GF(2) matrix of "feed one zero byte", its powers Z_{16 * 2^j} by
//     repeated squaring and its inverse by Gauss-Jordan elimination; each matrix M is
//     stored as four byte tables tab[b][v] = M(v << 8b).
#include <cstdint>
#include <utility>

#include "crc.cuh"

namespace luda {

namespace {

constexpr uint32_t kPoly = 0x82F63B78u;

struct Mat {
  uint32_t col[32];  // col[i] = image of bit i
};

uint32_t apply(const Mat& m, uint32_t v) {
  uint32_t r = 0;
  for (int i = 0; i < 32; ++i)
    if (v >> i & 1u) r ^= m.col[i];
  return r;
}

Mat mul(const Mat& a, const Mat& b) {  // a after b
  Mat r;
  for (int i = 0; i < 32; ++i) r.col[i] = apply(a, b.col[i]);
  return r;
}

bool invert(const Mat& m, Mat* out) {
  // Solve with rows: row r of m is the set of columns i whose image has bit r.
  uint64_t rows[32];
  for (int r = 0; r < 32; ++r) {
    uint32_t bits = 0;
    for (int i = 0; i < 32; ++i)
      if (m.col[i] >> r & 1u) bits |= 1u << i;
    rows[r] = uint64_t(bits) | (uint64_t(1u << r) << 32);  // [m | I]
  }
  for (int c = 0; c < 32; ++c) {
    int piv = -1;
    for (int r = c; r < 32; ++r)
      if (rows[r] >> c & 1u) {
        piv = r;
        break;
      }
    if (piv < 0) return false;
    std::swap(rows[c], rows[piv]);
    for (int r = 0; r < 32; ++r)
      if (r != c && (rows[r] >> c & 1u)) rows[r] ^= rows[c];
  }
  // rows now [I | m^-1]; row r of the inverse in the high half.
  for (int i = 0; i < 32; ++i) {
    uint32_t col = 0;
    for (int r = 0; r < 32; ++r)
      if (rows[r] >> (32 + i) & 1u) col |= 1u << r;
    out->col[i] = col;
  }
  return true;
}

void to_tables(const Mat& m, uint32_t* tab) {
  for (int b = 0; b < 4; ++b)
    for (uint32_t v = 0; v < 256; ++v) tab[b * 256 + v] = apply(m, v << (8 * b));
}

Mat power(const Mat& m, uint32_t e) {  // m^e by square-and-multiply
  Mat acc;
  for (int i = 0; i < 32; ++i) acc.col[i] = 1u << i;
  Mat base = m;
  for (; e; e >>= 1) {
    if (e & 1u) acc = mul(acc, base);
    base = mul(base, base);
  }
  return acc;
}

}  // namespace

// Fills `slice` (1024 words) and `shift` (kShiftTables * 1024 words).
bool make_crc_tables(uint32_t* slice, uint32_t* shift) {
  for (uint32_t v = 0; v < 256; ++v) {
    uint32_t c = v;
    for (int b = 0; b < 8; ++b) c = (c & 1u) ? (c >> 1) ^ kPoly : (c >> 1);
    slice[v] = c;
  }
  for (int k = 1; k < 4; ++k)
    for (uint32_t v = 0; v < 256; ++v) {
      const uint32_t prev = slice[(k - 1) * 256 + v];
      slice[k * 256 + v] = (prev >> 8) ^ slice[prev & 0xFFu];
    }
  Mat z1;
  for (int i = 0; i < 32; ++i) {
    const uint32_t r = 1u << i;
    z1.col[i] = slice[r & 0xFFu] ^ (r >> 8);
  }
  Mat z = z1;  // Z_16
  for (int s = 0; s < 4; ++s) z = mul(z, z);
  for (int j = 0; j < kShiftPow; ++j) {
    to_tables(z, shift + size_t(j) * 1024);
    z = mul(z, z);
  }
  to_tables(power(z1, 992), shift + size_t(kShift992) * 1024);
  Mat inv;
  if (!invert(z1, &inv)) return false;
  Mat zp = inv;
  for (int p = 1; p <= kShiftInv; ++p) {
    to_tables(zp, shift + size_t(kShiftPow + p - 1) * 1024);
    zp = mul(zp, inv);
  }
  return true;
}

// Fills `out` (kChunkTables * 1024 words) with the matrices Z_L listed at kCZ16 ... kCZ4608.
bool make_chunk_tables(uint32_t* out) {
  uint32_t slice[256];
  for (uint32_t v = 0; v < 256; ++v) {
    uint32_t c = v;
    for (int b = 0; b < 8; ++b) c = (c & 1u) ? (c >> 1) ^ kPoly : (c >> 1);
    slice[v] = c;
  }
  Mat z1;
  for (int i = 0; i < 32; ++i) {
    const uint32_t r = 1u << i;
    z1.col[i] = slice[r & 0xFFu] ^ (r >> 8);
  }
  static const uint32_t kLen[kChunkTables] = {16, 32, 64, 128, 80, kChunk, 2 * kChunk, 4 * kChunk,
                                              8 * kChunk, 16 * kChunk, 32 * kChunk};
  for (int t = 0; t < kChunkTables; ++t) to_tables(power(z1, kLen[t]), out + size_t(t) * 1024);
  return true;
}

}  // namespace luda
