// Checkpoint of a decomposition: the premise of the method is that the
// eigenpairs are computed once and reused for any number of forcings,
// orders and times (Sec. II), so (n, lambda, V) can be written to a file and
// read back, tagged with a hash of the domain they belong to.
//
// File layout (every field little-endian, whatever the host):
//   offset  0  magic "FRACLAPD" (8 bytes)
//           8  u32 version (1)
//          12  i32 dim (2 or 3; 0 = no grid recorded)
//          16  i64 n
//          24  i64 ext[3] (nx, ny, nz)
//          48  f64 h
//          56  u64 mask hash (0 = none)
//          64  u32 reserved (0)
//          68  f64 lambda[n], then f64 V[n*n] column-major, packed (ld = n)
//   end - 8    u64 FNV-1a-64 of every byte before it
// Host buffers only: the caller moves V between device and host.
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <string>
#include <vector>

#include "../../include/fraclap.h"

namespace {

constexpr char kMagic[8] = {'F', 'R', 'A', 'C', 'L', 'A', 'P', 'D'};
constexpr uint32_t kVersion = 1;
constexpr size_t kHeaderBytes = 68;

// FNV-1a, 64-bit (Fowler, Noll, Vo): h = (h xor byte) * 1099511628211,
// starting from 14695981039346656037.
struct Fnv {
  uint64_t h = 14695981039346656037ull;
  void add(const unsigned char* p, size_t len) {
    for (size_t i = 0; i < len; ++i) {
      h ^= p[i];
      h *= 1099511628211ull;
    }
  }
};

void put_u64(unsigned char* p, uint64_t v) {
  for (int i = 0; i < 8; ++i) p[i] = (unsigned char)(v >> (8 * i));
}
uint64_t get_u64(const unsigned char* p) {
  uint64_t v = 0;
  for (int i = 0; i < 8; ++i) v |= (uint64_t)p[i] << (8 * i);
  return v;
}
void put_u32(unsigned char* p, uint32_t v) {
  for (int i = 0; i < 4; ++i) p[i] = (unsigned char)(v >> (8 * i));
}
uint32_t get_u32(const unsigned char* p) {
  uint32_t v = 0;
  for (int i = 0; i < 4; ++i) v |= (uint32_t)p[i] << (8 * i);
  return v;
}
uint64_t bits_of(double x) {
  uint64_t u;
  memcpy(&u, &x, 8);
  return u;
}
double double_of(uint64_t u) {
  double x;
  memcpy(&x, &u, 8);
  return x;
}

// Writes `len` bytes and feeds them to the checksum.
bool put(FILE* f, Fnv* sum, const unsigned char* p, size_t len) {
  sum->add(p, len);
  return fwrite(p, 1, len, f) == len;
}
bool get(FILE* f, Fnv* sum, unsigned char* p, size_t len) {
  if (fread(p, 1, len, f) != len) return false;
  sum->add(p, len);
  return true;
}

}  // namespace

extern "C" uint64_t fraclap_mask_hash(const uint8_t* mask_host, int dim, const int64_t ext[3], double h) {
  if (!mask_host || !ext || (dim != 2 && dim != 3) || ext[0] < 0 || ext[1] < 0 || ext[2] < 0) return 0;
  Fnv s;
  unsigned char b[8];
  put_u32(b, (uint32_t)dim);
  s.add(b, 4);
  for (int d = 0; d < 3; ++d) {
    put_u64(b, (uint64_t)ext[d]);
    s.add(b, 8);
  }
  put_u64(b, bits_of(h));
  s.add(b, 8);
  const int64_t total = ext[0] * ext[1] * (dim == 3 ? ext[2] : 1);
  for (int64_t g = 0; g < total; ++g) {
    const unsigned char v = mask_host[g] ? 1 : 0;
    s.add(&v, 1);
  }
  return s.h ? s.h : 1;  // 0 means "no hash" in the file
}

extern "C" int fraclap_save_decomposition(const char* path, int64_t n, const double* lambda_host,
                                          const double* V_host, int64_t ldv, int dim, const int64_t ext[3],
                                          double h, uint64_t mask_hash) {
  if (!path || n < 0 || (n > 0 && (!lambda_host || !V_host || ldv < n))) return FRACLAP_ERR_INVALID_ARG;
  if (dim != 0 && dim != 2 && dim != 3) return FRACLAP_ERR_INVALID_ARG;
  const std::string tmp = std::string(path) + ".partial";
  FILE* f = fopen(tmp.c_str(), "wb");
  if (!f) return FRACLAP_ERR_IO;
  Fnv sum;
  unsigned char hdr[kHeaderBytes] = {};
  memcpy(hdr, kMagic, 8);
  put_u32(hdr + 8, kVersion);
  put_u32(hdr + 12, (uint32_t)dim);
  put_u64(hdr + 16, (uint64_t)n);
  for (int d = 0; d < 3; ++d) put_u64(hdr + 24 + 8 * d, ext ? (uint64_t)ext[d] : 0);
  put_u64(hdr + 48, bits_of(h));
  put_u64(hdr + 56, mask_hash);
  bool ok = put(f, &sum, hdr, kHeaderBytes);
  std::vector<unsigned char> col((size_t)(n > 0 ? n : 1) * 8);
  for (int64_t i = 0; ok && i < n; ++i) put_u64(&col[8 * i], bits_of(lambda_host[i]));
  if (ok && n > 0) ok = put(f, &sum, col.data(), (size_t)n * 8);
  for (int64_t j = 0; ok && j < n; ++j) {
    const double* v = V_host + j * ldv;
    for (int64_t i = 0; i < n; ++i) put_u64(&col[8 * i], bits_of(v[i]));
    ok = put(f, &sum, col.data(), (size_t)n * 8);
  }
  unsigned char tr[8];
  put_u64(tr, sum.h);
  ok = ok && fwrite(tr, 1, 8, f) == 8;
  ok = (fclose(f) == 0) && ok;
  if (!ok || rename(tmp.c_str(), path) != 0) {
    remove(tmp.c_str());
    return FRACLAP_ERR_IO;
  }
  return 0;
}

extern "C" int fraclap_load_decomposition(const char* path, int64_t* n_out, int* dim_out, int64_t ext_out[3],
                                          double* h_out, uint64_t* mask_hash_out, double* lambda_host,
                                          double* V_host, int64_t ldv, uint64_t expect_mask_hash) {
  if (!path) return FRACLAP_ERR_INVALID_ARG;
  FILE* f = fopen(path, "rb");
  if (!f) return FRACLAP_ERR_IO;
  Fnv sum;
  unsigned char hdr[kHeaderBytes];
  int rc = 0;
  int64_t n = -1;
  uint64_t mh = 0;
  if (!get(f, &sum, hdr, kHeaderBytes) || memcmp(hdr, kMagic, 8) != 0 || get_u32(hdr + 8) != kVersion) {
    rc = FRACLAP_ERR_IO;
  } else {
    n = (int64_t)get_u64(hdr + 16);
    const int dim = (int)get_u32(hdr + 12);
    mh = get_u64(hdr + 56);
    // the file must hold exactly header + lambda + V + checksum
    long long want = -1;
    if (n >= 0 && n <= (int64_t)3037000499ll / 8 && (dim == 0 || dim == 2 || dim == 3))
      want = (long long)kHeaderBytes + 8ll * n + 8ll * n * n + 8ll;
    long long here = ftell(f), size = -1;
    if (here >= 0 && fseek(f, 0, SEEK_END) == 0) size = ftell(f);
    if (want < 0 || size != want || fseek(f, here, SEEK_SET) != 0) {
      rc = FRACLAP_ERR_IO;
    } else {
      if (n_out) *n_out = n;
      if (dim_out) *dim_out = dim;
      for (int d = 0; d < 3; ++d)
        if (ext_out) ext_out[d] = (int64_t)get_u64(hdr + 24 + 8 * d);
      if (h_out) *h_out = double_of(get_u64(hdr + 48));
      if (mask_hash_out) *mask_hash_out = mh;
      if (expect_mask_hash != 0 && mh != expect_mask_hash) rc = FRACLAP_ERR_INVALID_ARG;
    }
  }
  if (rc == 0 && lambda_host) {  // second call: the payload
    if (n > 0 && (!V_host || ldv < n)) {
      rc = FRACLAP_ERR_INVALID_ARG;
    } else {
      std::vector<unsigned char> col((size_t)(n > 0 ? n : 1) * 8);
      bool ok = n == 0 || get(f, &sum, col.data(), (size_t)n * 8);
      for (int64_t i = 0; ok && i < n; ++i) lambda_host[i] = double_of(get_u64(&col[8 * i]));
      for (int64_t j = 0; ok && j < n; ++j) {
        ok = get(f, &sum, col.data(), (size_t)n * 8);
        double* v = V_host + j * ldv;
        for (int64_t i = 0; ok && i < n; ++i) v[i] = double_of(get_u64(&col[8 * i]));
      }
      unsigned char tr[8];
      if (!ok || fread(tr, 1, 8, f) != 8 || get_u64(tr) != sum.h) rc = FRACLAP_ERR_IO;
    }
  }
  fclose(f);
  return rc;
}
