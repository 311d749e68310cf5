// rb_opfile.cu -- operator files: the reduced operators of one n_max set (the output of the
// offline stage, Sec. 3.5-3.6) in a versioned binary file with a checksum, written from host
// arrays and loaded into a context. Host code only.
//
// Layout (little-endian):
//   offset  0  magic "RBOPS\0\0\0" (8 bytes)
//           8  u32 version (1)          12  u32 header bytes (64)
//          16  i32 n_max, m, q_a, q_c, q_f, q_b, dtype_c (7 x 4 bytes)
//          44  u32 flags (bit 0: pressure operators present)
//          48  u64 payload bytes        56  u64 checksum of the payload
//          64  payload: A, C, f, then (with pressure) B, As, Cs, fs, each C-contiguous as
//              rb_operators documents; C and Cs in their storage type (dtype_c).
// Checksum: FNV-1a (64-bit offset basis and prime) over the payload taken as 8-byte
// little-endian words, a last partial word zero-padded.
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "rb_ctx.h"

namespace rb {

constexpr char kOpMagic[8] = {'R', 'B', 'O', 'P', 'S', 0, 0, 0};
constexpr uint32_t kOpVersion = 1, kOpHeader = 64;

struct OpShape {
  int n, m, q_a, q_c, q_f, q_b, dtype_c;
  bool pres;
  size_t csz() const { return dtype_c == RB_F64 ? 8 : (dtype_c == RB_F32 ? 4 : 2); }
  // byte sizes of the arrays in file order
  void sizes(size_t out[7]) const {
    const size_t nn = (size_t)n, mm = (size_t)m;
    out[0] = 8 * (size_t)q_a * nn * nn;
    out[1] = csz() * (size_t)q_c * nn * nn * nn;
    out[2] = 8 * (size_t)q_f * nn;
    out[3] = pres ? 8 * (size_t)q_b * mm * mm : 0;
    out[4] = pres ? 8 * (size_t)q_a * mm * nn : 0;
    out[5] = pres ? csz() * (size_t)q_c * nn * nn * mm : 0;
    out[6] = pres ? 8 * (size_t)q_f * mm : 0;
  }
  size_t payload() const {
    size_t s[7];
    sizes(s);
    size_t t = 0;
    for (size_t v : s) t += v;
    return t;
  }
};

struct Fnv {
  uint64_t h = 0xcbf29ce484222325ull;
  uint8_t tail[8];
  int nt = 0;
  void word(uint64_t w) {
    h ^= w;
    h *= 0x100000001b3ull;
  }
  void add(const void *p, size_t bytes) {
    const uint8_t *b = (const uint8_t *)p;
    while (bytes && nt) {  // complete a pending partial word
      tail[nt++] = *b++;
      --bytes;
      if (nt == 8) {
        uint64_t w;
        memcpy(&w, tail, 8);
        word(w);
        nt = 0;
      }
    }
    for (; bytes >= 8; bytes -= 8, b += 8) {
      uint64_t w;
      memcpy(&w, b, 8);
      word(w);
    }
    while (bytes--) tail[nt++] = *b++;
  }
  uint64_t done() {
    if (nt) {
      memset(tail + nt, 0, 8 - nt);
      uint64_t w;
      memcpy(&w, tail, 8);
      word(w);
      nt = 0;
    }
    return h;
  }
};

static int check_shape(const rb_ctx *ctx, const OpShape &s) {
  if (s.n < 1 || s.n > RB_N_MAX) return set_error(ctx, RB_ERR_ARG, "n_max %d out of range", s.n);
  if (s.q_a < 1 || s.q_c < 1 || s.q_f < 1 || s.q_a > RB_Q_MAX || s.q_c > RB_Q_MAX ||
      s.q_f > RB_Q_MAX || s.q_b < 0 || s.q_b > RB_Q_MAX)
    return set_error(ctx, RB_ERR_ARG, "affine term counts out of range");
  if (s.dtype_c != RB_F64 && s.dtype_c != RB_F32 && s.dtype_c != RB_BF16)
    return set_error(ctx, RB_ERR_ARG, "bad dtype_c");
  if (s.pres && (s.m < 1 || s.m > RB_M_MAX || s.q_b < 1))
    return set_error(ctx, RB_ERR_ARG, "pressure sizes out of range");
  return RB_OK;
}

static void put32(uint8_t *h, int off, uint32_t v) { memcpy(h + off, &v, 4); }
static void put64(uint8_t *h, int off, uint64_t v) { memcpy(h + off, &v, 8); }
static uint32_t get32(const uint8_t *h, int off) {
  uint32_t v;
  memcpy(&v, h + off, 4);
  return v;
}
static uint64_t get64(const uint8_t *h, int off) {
  uint64_t v;
  memcpy(&v, h + off, 8);
  return v;
}

}  // namespace rb

using namespace rb;

extern "C" {

int rb_save_operators(const rb_operators *ops, const char *path) {
  if (!ops || !path) return set_error(nullptr, RB_ERR_ARG, "rb_save_operators: NULL argument");
  OpShape s{ops->n_max, ops->B ? ops->m : 0, ops->q_a, ops->q_c, ops->q_f, ops->B ? ops->q_b : 0,
            ops->dtype_c, ops->B != nullptr};
  int rc = check_shape(nullptr, s);
  if (rc != RB_OK) return rc;
  if (!ops->A || !ops->C || !ops->f || (s.pres && (!ops->As || !ops->Cs || !ops->fs)))
    return set_error(nullptr, RB_ERR_ARG, "rb_save_operators: operator arrays missing");
  const void *arr[7] = {ops->A, ops->C, ops->f, ops->B, ops->As, ops->Cs, ops->fs};
  size_t sz[7];
  s.sizes(sz);
  Fnv f;
  for (int i = 0; i < 7; ++i)
    if (sz[i]) f.add(arr[i], sz[i]);
  uint8_t h[kOpHeader] = {};
  memcpy(h, kOpMagic, 8);
  put32(h, 8, kOpVersion);
  put32(h, 12, kOpHeader);
  const int32_t dims[7] = {s.n, s.m, s.q_a, s.q_c, s.q_f, s.q_b, s.dtype_c};
  for (int i = 0; i < 7; ++i) put32(h, 16 + 4 * i, (uint32_t)dims[i]);
  put32(h, 44, s.pres ? 1u : 0u);
  put64(h, 48, s.payload());
  put64(h, 56, f.done());
  FILE *fp = fopen(path, "wb");
  if (!fp) return set_error(nullptr, RB_ERR_ARG, "rb_save_operators: cannot open %s", path);
  bool ok = fwrite(h, 1, kOpHeader, fp) == kOpHeader;
  for (int i = 0; i < 7 && ok; ++i)
    if (sz[i]) ok = fwrite(arr[i], 1, sz[i], fp) == sz[i];
  ok = (fclose(fp) == 0) && ok;
  if (!ok) return set_error(nullptr, RB_ERR_ARG, "rb_save_operators: write to %s failed", path);
  return RB_OK;
}

int rb_load_operator_file(rb_ctx *ctx, const char *path) {
  if (!ctx) return RB_ERR_ARG;
  if (!path) return set_error(ctx, RB_ERR_ARG, "path is NULL");
  FILE *fp = fopen(path, "rb");
  if (!fp) return set_error(ctx, RB_ERR_ARG, "cannot open %s", path);
  uint8_t h[kOpHeader];
  if (fread(h, 1, kOpHeader, fp) != kOpHeader) {
    fclose(fp);
    return set_error(ctx, RB_ERR_ARG, "%s: shorter than the header", path);
  }
  if (memcmp(h, kOpMagic, 8) != 0 || get32(h, 8) != kOpVersion || get32(h, 12) != kOpHeader) {
    fclose(fp);
    return set_error(ctx, RB_ERR_ARG, "%s: not an operator file of version %u", path, kOpVersion);
  }
  int32_t d[7];
  for (int i = 0; i < 7; ++i) d[i] = (int32_t)get32(h, 16 + 4 * i);
  const uint32_t flags = get32(h, 44);
  OpShape s{d[0], d[1], d[2], d[3], d[4], d[5], d[6], (flags & 1u) != 0};
  int rc = check_shape(ctx, s);
  if (rc != RB_OK) {
    fclose(fp);
    return rc;
  }
  const uint64_t payload = get64(h, 48), sum = get64(h, 56);
  if (payload != s.payload()) {
    fclose(fp);
    return set_error(ctx, RB_ERR_ARG, "%s: payload size does not match the shapes", path);
  }
  std::vector<uint8_t> buf;
  try {
    buf.resize(payload);
  } catch (...) {
    fclose(fp);
    return set_error(ctx, RB_ERR_OOM, "%s: %llu bytes of host memory", path, (unsigned long long)payload);
  }
  const size_t got = fread(buf.data(), 1, payload, fp);
  const bool extra = fgetc(fp) != EOF;
  fclose(fp);
  if (got != payload || extra) return set_error(ctx, RB_ERR_ARG, "%s: file size does not match its header", path);
  Fnv f;
  f.add(buf.data(), payload);
  if (f.done() != sum) return set_error(ctx, RB_ERR_ARG, "%s: checksum mismatch", path);
  size_t sz[7];
  s.sizes(sz);
  const uint8_t *p[7];
  size_t off = 0;
  for (int i = 0; i < 7; ++i) {
    p[i] = sz[i] ? buf.data() + off : nullptr;
    off += sz[i];
  }
  rb_operators ops{};
  ops.n_max = s.n;
  ops.m = s.m;
  ops.q_a = s.q_a;
  ops.q_c = s.q_c;
  ops.q_f = s.q_f;
  ops.q_b = s.q_b;
  ops.dtype_c = s.dtype_c;
  ops.A = (const double *)p[0];
  ops.C = p[1];
  ops.f = (const double *)p[2];
  ops.B = (const double *)p[3];
  ops.As = (const double *)p[4];
  ops.Cs = p[5];
  ops.fs = (const double *)p[6];
  return rb_load_operators(ctx, &ops);
}

}  // extern "C"
