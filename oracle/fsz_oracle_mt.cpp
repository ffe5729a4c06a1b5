// All-core timing driver for the CPU oracle: TEST INFRASTRUCTURE ONLY.
//
// Runs the oracle's own functions on every host core, for the reported CPU baseline: the
// value range over element ranges (combined: min of minima, max of maxima, all finite),
// the tiles' encoding over contiguous tile ranges (fszo_compress_tiles), then a serial
// exclusive scan of the ranges' byte counts to place them; decoding the same way
// (fszo_decompress_tiles over tile ranges after a serial scan of the rate header). The
// oracle itself stays single-threaded; this file adds no arithmetic of the method, only
// the split into ranges, and its streams equal the oracle's byte for byte.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>

#include "fsz_oracle.h"

namespace {

constexpr uint64_t kTile = 256;
constexpr uint64_t kMaxTileBytes = 772;

template <typename F>
void parallel_ranges(uint64_t count, int nthreads, F&& body) {
  const uint64_t parts = std::max<uint64_t>(1, std::min<uint64_t>(uint64_t(nthreads), count));
  std::vector<std::thread> pool;
  for (uint64_t k = 0; k < parts; ++k) {
    const uint64_t a = count * k / parts, b = count * (k + 1) / parts;
    pool.emplace_back([&body, k, a, b] { body(k, a, b); });
  }
  for (auto& t : pool) t.join();
}

}  // namespace

extern "C" {

int fszo_mt_compress(const float* d, uint32_t ndim, const uint64_t* dims, int mode, double eb_req,
                     uint8_t* out, uint64_t out_capacity, uint64_t* out_bytes, int nthreads) {
  if (ndim < 1 || ndim > 3 || dims == nullptr || nthreads < 1) return FSZO_ERR_INVALID_ARG;
  uint64_t n = 1;
  for (uint32_t k = 0; k < ndim; ++k) n *= dims[k];
  // value range
  const uint64_t parts = std::max<uint64_t>(1, std::min<uint64_t>(uint64_t(nthreads), n));
  std::vector<float> lo(parts, 0.0f), hi(parts, 0.0f);
  std::vector<int> fin(parts, 1);
  if (n > 0)
    parallel_ranges(n, nthreads, [&](uint64_t k, uint64_t a, uint64_t b) {
      fszo_stats(d + a, b - a, &lo[k], &hi[k], &fin[k]);
    });
  float vmin = 0.0f, vmax = 0.0f;
  int all_finite = 1;
  for (uint64_t k = 0; k < parts; ++k) all_finite &= fin[k];
  if (all_finite && n > 0) {
    vmin = lo[0];
    vmax = hi[0];
    for (uint64_t k = 1; k < parts; ++k) {
      if (lo[k] < vmin) vmin = lo[k];
      if (hi[k] > vmax) vmax = hi[k];
    }
  }
  fszo_params_t p;
  int st = fszo_params(mode, eb_req, vmin, vmax, all_finite, n, &p);
  if (st != FSZO_OK) return st;
  // tiles over ranges, each into a buffer of its own
  const uint64_t T = (n + kTile - 1) / kTile;
  if (out_capacity < 64 + 8 * T) return FSZO_ERR_CAPACITY;
  const uint64_t tparts = std::max<uint64_t>(1, std::min<uint64_t>(uint64_t(nthreads), T));
  std::vector<std::vector<uint8_t>> data(tparts);
  std::vector<uint64_t> bytes(tparts, 0), t0s(tparts, 0);
  std::vector<int> sts(tparts, FSZO_OK);
  if (T > 0)
    parallel_ranges(T, nthreads, [&](uint64_t k, uint64_t a, uint64_t b) {
      t0s[k] = a;
      data[k].resize((b - a) * kMaxTileBytes);
      sts[k] = fszo_compress_tiles(d, n, p.r, a, b, out + 64 + 8 * a, data[k].data(),
                                   data[k].size(), &bytes[k]);
    });
  for (int s : sts)
    if (s != FSZO_OK) return s;
  // serial exclusive scan of the ranges' byte counts, then the copies
  std::vector<uint64_t> off(tparts + 1, 0);
  for (uint64_t k = 0; k < tparts; ++k) off[k + 1] = off[k] + bytes[k];
  const uint64_t total = 64 + 8 * T + off[tparts];
  if (out_bytes) *out_bytes = total;
  if (total > out_capacity) return FSZO_ERR_CAPACITY;
  fszo_write_preamble(out, ndim, dims, n, mode, eb_req, p.s, 0u, off[tparts]);
  if (T > 0)
    parallel_ranges(tparts, nthreads, [&](uint64_t, uint64_t a, uint64_t b) {
      for (uint64_t k = a; k < b; ++k)
        if (bytes[k]) std::memcpy(out + 64 + 8 * T + off[k], data[k].data(), bytes[k]);
    });
  return FSZO_OK;
}

int fszo_mt_decompress(const uint8_t* in, uint64_t in_bytes, float* out, uint64_t out_capacity_elems,
                       uint64_t* n_out, int nthreads) {
  if (nthreads < 1) return FSZO_ERR_INVALID_ARG;
  uint64_t n, db, dims[3];
  uint32_t nd, word;
  double eb;
  float s;
  int st = fszo_read_preamble_f(in, in_bytes, &n, &nd, dims, &eb, &s, &db, &word);
  if (st != FSZO_OK) return st;
  if (word & 0xFF00u) return FSZO_ERR_INVALID_ARG;  // the default tile configuration only
  if (n > out_capacity_elems) return FSZO_ERR_CAPACITY;
  const uint64_t T = (n + kTile - 1) / kTile;
  // serial scan of the rate header: each range's first data byte
  const uint64_t tparts = std::max<uint64_t>(1, std::min<uint64_t>(uint64_t(nthreads), T));
  std::vector<uint64_t> start(tparts, 0);
  const uint8_t* header = in + 64;
  uint64_t acc = 0, k = 0;
  for (uint64_t t = 0; t < T; ++t) {
    while (k < tparts && T * k / tparts == t) start[k++] = acc;
    const uint8_t* h = header + 8 * t;
    uint64_t bytes = (h[0] & 0x40) ? 4 : 0;
    for (int b = 0; b < 8; ++b) bytes += fszo_block_cost(h[b] & 0x1F);
    acc += bytes;
  }
  if (acc != db) return FSZO_ERR_CORRUPT;
  std::vector<int> sts(tparts, FSZO_OK);
  if (T > 0)
    parallel_ranges(T, nthreads, [&](uint64_t k, uint64_t a, uint64_t b) {
      sts[k] = fszo_decompress_tiles(in, in_bytes, a, b, start[k], out + a * kTile);
    });
  for (int x : sts)
    if (x != FSZO_OK) return x;
  if (n_out) *n_out = n;
  return FSZO_OK;
}

}  // extern "C"
