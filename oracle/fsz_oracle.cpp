// FSZ CPU oracle: TEST INFRASTRUCTURE ONLY (see fsz_oracle.h).
//
// Plain single-threaded C++17. Build with -O2 -ffp-contract=off -fno-fast-math so
// that every float32 multiply and add is one IEEE round-to-nearest operation.
// Each function follows the paper's steps in its order and notation; where the
// paper is silent the reading used is stated next to the code.
#include "fsz_oracle.h"

#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

namespace {

constexpr int kTile = 256;        // Sec. 3.1: a tile is 8 blocks of 32 elements
constexpr int kBlock = 32;
constexpr int kBlocksPerTile = 8;
constexpr uint64_t kPreamble = 64; // the 64-byte preamble is this project's addition
// The margin eps = (3Q + 4) 2^-23 of reading R2 is capped at 2^-4 (first tier); a field
// that needs more takes the second tier, capped at 2^-1. Q bounds |q|.
constexpr uint32_t kQmax1 = 174761;   // largest Q with (3Q + 4) 2^-23 <= 2^-4
constexpr uint32_t kQmax2 = 1398100;  // largest Q with (3Q + 4) 2^-23 <= 2^-1
constexpr uint64_t kMaxElems = uint64_t(1) << 40;

uint64_t tiles_of(uint64_t n) { return (n + kTile - 1) / kTile; }

void put_u16(uint8_t* p, uint16_t v) { p[0] = uint8_t(v); p[1] = uint8_t(v >> 8); }
void put_u32(uint8_t* p, uint32_t v) { for (int i = 0; i < 4; ++i) p[i] = uint8_t(v >> (8 * i)); }
void put_u64(uint8_t* p, uint64_t v) { for (int i = 0; i < 8; ++i) p[i] = uint8_t(v >> (8 * i)); }
uint16_t get_u16(const uint8_t* p) { return uint16_t(p[0] | (p[1] << 8)); }
uint32_t get_u32(const uint8_t* p) {
  uint32_t v = 0;
  for (int i = 3; i >= 0; --i) v = (v << 8) | p[i];
  return v;
}
uint64_t get_u64(const uint8_t* p) {
  uint64_t v = 0;
  for (int i = 7; i >= 0; --i) v = (v << 8) | p[i];
  return v;
}

// A payload word holds one bit per element of a 32-element block: element j at
// bit 31 - j (Sec. 4.3). It is serialised most significant byte first, so byte 0
// carries elements 0..7 with element 0 in its top bit (reading of the uchar4 store).
void put_word_be(std::vector<uint8_t>& out, uint32_t w) {
  out.push_back(uint8_t(w >> 24));
  out.push_back(uint8_t(w >> 16));
  out.push_back(uint8_t(w >> 8));
  out.push_back(uint8_t(w));
}
uint32_t get_word_be(const uint8_t* p) {
  return (uint32_t(p[0]) << 24) | (uint32_t(p[1]) << 16) | (uint32_t(p[2]) << 8) | uint32_t(p[3]);
}

// Two's-complement wrap-around arithmetic (well defined in C++ via uint32).
int32_t wsub(int32_t a, int32_t b) { return int32_t(uint32_t(a) - uint32_t(b)); }
int32_t wadd(int32_t a, int32_t b) { return int32_t(uint32_t(a) + uint32_t(b)); }
uint32_t uabs(int32_t v) { return v < 0 ? uint32_t(0) - uint32_t(v) : uint32_t(v); }

// The tile configuration in bits 8-15 of the preamble's method word (Sec. 6.5): B code 0
// (32) or 1 (64), T code 0 (8), 1 (4) or 2 (16).
bool tile_cfg_from_word(uint32_t word, int* B, int* T) {
  const uint32_t bc = (word >> 8) & 0xF, tc = (word >> 12) & 0xF;
  if (bc > 1 || tc > 2) return false;
  *B = bc == 1 ? 64 : 32;
  *T = tc == 1 ? 4 : tc == 2 ? 16 : 8;
  return true;
}

}  // namespace

extern "C" {

int fszo_stats(const float* d, uint64_t n, float* vmin, float* vmax, int* all_finite) {
  int fin = 1;
  for (uint64_t i = 0; i < n; ++i)
    if (!std::isfinite(d[i])) fin = 0;
  float lo = 0.0f, hi = 0.0f;
  if (fin && n > 0) {
    lo = d[0];
    hi = d[0];
    for (uint64_t i = 1; i < n; ++i) {
      if (d[i] < lo) lo = d[i];
      if (d[i] > hi) hi = d[i];
    }
  }
  *vmin = lo;
  *vmax = hi;
  *all_finite = fin;
  return FSZO_OK;
}

// Reading of Sec. 5.1 and of the error-bound argument of Sec. 4.2.2:
//  * ABS: eb as given. REL: eb = REL x (max - min) in float64; a constant field
//    uses REL x |max|, or REL itself when that is 0 (the paper is silent).
//  * The paper's |d - 2eb q| <= eb holds in exact arithmetic only. In float32 the
//    quantizer and the reconstruction each round, so the half step e is shrunk by
//    a margin eps that covers both roundings for |q| <= Q, with Q bounded from the
//    field's max |d| (A). e is rounded toward zero to float32, s = 2e, r = fl(1/s).
//  * eps = (3Q + 4) 2^-23 is capped at 2^-4, Q = ceil(A / (2 eb (1 - 2^-4))) + 1; a field
//    beyond that cap takes a second tier, Q = ceil(A / (2 eb (1 - 2^-1))) + 1 with eps
//    capped at 2^-1 (a finer step: a field the first tier accepts keeps its stream).
int fszo_params(int mode, double eb_req, float vmin, float vmax, int all_finite, uint64_t n,
                fszo_params_t* p) {
  if (!(eb_req > 0.0) || !std::isfinite(eb_req)) return FSZO_ERR_INVALID_ARG;
  if (mode != FSZO_EB_ABS && mode != FSZO_EB_REL) return FSZO_ERR_INVALID_ARG;
  if (!all_finite) return FSZO_ERR_NONFINITE;
  if (n == 0) { vmin = 0.0f; vmax = 0.0f; }
  double eb = eb_req;
  if (mode == FSZO_EB_REL) {
    double range = double(vmax) - double(vmin);
    if (range > 0.0) {
      eb = eb_req * range;
    } else {
      double mag = std::fabs(double(vmax));
      eb = mag > 0.0 ? eb_req * mag : eb_req;
    }
  }
  if (!(eb > 0.0) || !std::isfinite(eb)) return FSZO_ERR_EB_TOO_SMALL;
  const double two100 = std::ldexp(1.0, 100);
  double eb_eff = eb < two100 ? eb : two100;
  double A = std::fmax(std::fabs(double(vmin)), std::fabs(double(vmax)));
  // First tier: K = A / (2 eb (1 - 2^-4)) bounds A / (2e) whenever eps <= 2^-4.
  double K = A / (2.0 * eb_eff * (1.0 - 0.0625));
  uint32_t Q = 0;
  if (K <= double(kQmax1) && uint32_t(std::ceil(K)) + 1u <= kQmax1) {
    Q = uint32_t(std::ceil(K)) + 1u;
  } else {
    // Second tier, for fields the first refuses: K = A / (2 eb (1 - 2^-1)) bounds A / (2e)
    // whenever eps <= 2^-1 (a step up to half the first tier's).
    K = A / (2.0 * eb_eff * (1.0 - 0.5));
    if (!(K <= double(kQmax2))) return FSZO_ERR_EB_TOO_SMALL;
    Q = uint32_t(std::ceil(K)) + 1u;
    if (Q > kQmax2) return FSZO_ERR_EB_TOO_SMALL;
  }
  double eps = double(3u * Q + 4u) * std::ldexp(1.0, -23);
  double x = eb_eff * (1.0 - eps);
  float e = float(x);
  if (double(e) > x) e = std::nextafter(e, 0.0f);
  if (!(e >= std::ldexp(1.0f, -100))) return FSZO_ERR_EB_TOO_SMALL;
  float s = 2.0f * e;
  float r = 1.0f / s;
  p->eb = eb; p->eb_eff = eb_eff; p->K = K; p->Q = Q; p->e = e; p->s = s; p->r = r;
  return FSZO_OK;
}

// Sec. 4.2.2: q_i = round(d_i / (2 eb)). Here t = fl32(d x r) and the rounding is to
// the nearest integer with ties to even (the default IEEE rounding mode).
int32_t fszo_quantize(float d, float r) {
  float t = d * r;
  return int32_t(std::nearbyint(t));
}

float fszo_dequantize(int32_t q, float s) { return float(q) * s; }

// Sec. 4.2.2, variant 3: mu = round(dbar / (2 eb)), dbar = (1/256) sum_j d_j, the tile's
// floating-point mean. The paper leaves the summation order open; the order fixed
// here is: 32 partial sums P_j over elements 8j..8j+7 added left to right, then
// P_j += P_{j+h} for j < h, h = 16, 8, 4, 2, 1, and S = P_0. dbar = S x 2^-8.
// Padding elements of a partial last tile are zeros and are included.
int32_t fszo_tile_mu(const float d[256], float r) {
  float P[32];
  for (int j = 0; j < 32; ++j) {
    float acc = d[8 * j];
    for (int i = 1; i < 8; ++i) acc = acc + d[8 * j + i];
    P[j] = acc;
  }
  for (int h = 16; h >= 1; h /= 2)
    for (int j = 0; j < h; ++j) P[j] = P[j] + P[j + h];
  float dbar = P[0] * 0.00390625f;
  return fszo_quantize(dbar, r);
}

// Eqs. 1-2 and the variant list of Sec. 4.2.2. qh = q - mu for centred variants.
// The state carries across all 8 block boundaries (Eq. 2); only the tile's first
// element(s) lack predecessors, which are read as zero (reading: zero-initialised
// state, so l1_0 = qh_0, l2_0 = qh_0 and l2_1 = qh_1 - 2 qh_0).
void fszo_tile_residuals(const int32_t q[256], int32_t mu, int variant, int32_t l[256]) {
  fszo_tile_residuals_f(q, mu, variant, 0, l);
}

// The same with features switched off (Sec. 6.4 ablation). Without the cross-block state
// (FSZO_OFF_CROSS) every block restarts from zero predecessors, as its first element(s)
// would at a tile start (Sec. 2, C1: "restart prediction state at every boundary").
void fszo_tile_residuals_f(const int32_t q[256], int32_t mu, int variant, uint32_t off,
                           int32_t l[256]) {
  const bool centred = (variant == FSZO_LZ1C || variant == FSZO_LZ2C);
  const bool second = (variant == FSZO_LZ2 || variant == FSZO_LZ2C);
  int32_t prev1 = 0, prev2 = 0;  // qh_{i-1}, qh_{i-2}
  for (int i = 0; i < kTile; ++i) {
    if ((off & FSZO_OFF_CROSS) && i % kBlock == 0) prev1 = prev2 = 0;
    int32_t qh = centred ? wsub(q[i], mu) : q[i];
    if (!second) {
      l[i] = wsub(qh, prev1);
    } else {
      l[i] = wadd(wsub(qh, wadd(prev1, prev1)), prev2);
    }
    prev2 = prev1;
    prev1 = qh;
  }
}

// Sec. 4.1.2: r_b = ceil(log2(max_j |l_j| + 1)), the bit length of the block maximum.
uint32_t fszo_rate(uint32_t maxabs) {
  uint32_t r = 0;
  while (r < 32 && (uint64_t(1) << r) <= maxabs) ++r;
  return r;
}

// Eq. 3: S_b = 0 for r_b = 0, else a 4-byte sign map plus r_b 4-byte bit-planes.
uint32_t fszo_block_cost(uint32_t rate) { return rate == 0 ? 0u : 4u + 4u * rate; }

void fszo_tile_costs_four_pass(const int32_t q[256], int32_t mu, uint32_t C[4], uint8_t rates[32]) {
  fszo_tile_costs_four_pass_f(q, mu, 0, C, rates);
}

void fszo_tile_costs_four_pass_f(const int32_t q[256], int32_t mu, uint32_t off, uint32_t C[4],
                                 uint8_t rates[32]) {
  int32_t l[kTile];
  for (int v = 0; v < 4; ++v) {
    fszo_tile_residuals_f(q, mu, v, off, l);
    uint32_t cost = (v == FSZO_LZ1C || v == FSZO_LZ2C) ? 4u : 0u;  // the 4-byte mean
    for (int b = 0; b < kBlocksPerTile; ++b) {
      uint32_t m = 0;
      for (int j = 0; j < kBlock; ++j) { uint32_t a = uabs(l[b * kBlock + j]); if (a > m) m = a; }
      uint32_t rb = fszo_rate(m);
      rates[v * 8 + b] = uint8_t(rb);
      cost += fszo_block_cost(rb);
    }
    C[v] = cost;
  }
}

// Sec. 4.2.3: one loop computes the LZ1 and LZ2 residuals with cross-block state and
// the per-block maxima. By Eq. 4, Delta^k (q - mu) = Delta^k q for i >= k, so centring
// changes only the first k residuals of the tile, all inside block 0: the loop also
// keeps block 0's maxima over i >= k, and the centred block-0 rate is that maximum
// joined with the centred boundary residuals, computed after the loop.
void fszo_tile_costs_single_pass(const int32_t q[256], int32_t mu, uint32_t C[4], uint8_t rates[32]) {
  fszo_tile_costs_single_pass_f(q, mu, 0, C, rates);
}

// With features switched off: without the cross-block state the loop restarts at every
// block and only LZ1 and LZ2 are costed (centring needs the carried state: its costs are
// left at UINT32_MAX and its rates at 0).
void fszo_tile_costs_single_pass_f(const int32_t q[256], int32_t mu, uint32_t off, uint32_t C[4],
                                   uint8_t rates[32]) {
  if (off & FSZO_OFF_CROSS) {
    int32_t prev1 = 0, prev2 = 0;
    C[FSZO_LZ1] = C[FSZO_LZ2] = 0;
    C[FSZO_LZ1C] = C[FSZO_LZ2C] = UINT32_MAX;
    for (int b = 0; b < kBlocksPerTile; ++b) {
      uint32_t M1 = 0, M2 = 0;
      prev1 = prev2 = 0;
      for (int j = 0; j < kBlock; ++j) {
        int32_t qi = q[b * kBlock + j];
        uint32_t a1 = uabs(wsub(qi, prev1));
        uint32_t a2 = uabs(wadd(wsub(qi, wadd(prev1, prev1)), prev2));
        if (a1 > M1) M1 = a1;
        if (a2 > M2) M2 = a2;
        prev2 = prev1;
        prev1 = qi;
      }
      uint32_t r1 = fszo_rate(M1), r2 = fszo_rate(M2);
      rates[FSZO_LZ1 * 8 + b] = uint8_t(r1);
      rates[FSZO_LZ2 * 8 + b] = uint8_t(r2);
      rates[FSZO_LZ1C * 8 + b] = rates[FSZO_LZ2C * 8 + b] = 0;
      C[FSZO_LZ1] += fszo_block_cost(r1);
      C[FSZO_LZ2] += fszo_block_cost(r2);
    }
    return;
  }
  uint32_t M1[8] = {0}, M2[8] = {0};
  uint32_t M1_rest0 = 0, M2_rest0 = 0;  // block 0 over i >= 1 (LZ1) and i >= 2 (LZ2)
  int32_t prev1 = 0, prev2 = 0;
  for (int i = 0; i < kTile; ++i) {
    int32_t l1 = wsub(q[i], prev1);
    int32_t l2 = wadd(wsub(q[i], wadd(prev1, prev1)), prev2);
    int b = i / kBlock;
    uint32_t a1 = uabs(l1), a2 = uabs(l2);
    if (a1 > M1[b]) M1[b] = a1;
    if (a2 > M2[b]) M2[b] = a2;
    if (b == 0 && i >= 1 && a1 > M1_rest0) M1_rest0 = a1;
    if (b == 0 && i >= 2 && a2 > M2_rest0) M2_rest0 = a2;
    prev2 = prev1;
    prev1 = q[i];
  }
  // Centred boundary residuals: l1c_0 = q_0 - mu; l2c_0 = q_0 - mu;
  // l2c_1 = (q_1 - mu) - 2 (q_0 - mu) = q_1 - 2 q_0 + mu.
  uint32_t c10 = uabs(wsub(q[0], mu));
  uint32_t c21 = uabs(wadd(wsub(q[1], wadd(q[0], q[0])), mu));
  uint32_t M1c0 = M1_rest0 > c10 ? M1_rest0 : c10;
  uint32_t M2c0 = M2_rest0 > c10 ? M2_rest0 : c10;
  if (c21 > M2c0) M2c0 = c21;

  uint32_t tail1 = 0, tail2 = 0;  // blocks 1..7, shared by centred and plain variants
  for (int b = 0; b < kBlocksPerTile; ++b) {
    uint32_t r1 = fszo_rate(M1[b]), r2 = fszo_rate(M2[b]);
    rates[FSZO_LZ1 * 8 + b] = uint8_t(r1);
    rates[FSZO_LZ2 * 8 + b] = uint8_t(r2);
    rates[FSZO_LZ1C * 8 + b] = uint8_t(r1);
    rates[FSZO_LZ2C * 8 + b] = uint8_t(r2);
    if (b > 0) { tail1 += fszo_block_cost(r1); tail2 += fszo_block_cost(r2); }
  }
  uint32_t r1c0 = fszo_rate(M1c0), r2c0 = fszo_rate(M2c0);
  rates[FSZO_LZ1C * 8 + 0] = uint8_t(r1c0);
  rates[FSZO_LZ2C * 8 + 0] = uint8_t(r2c0);
  C[FSZO_LZ1] = fszo_block_cost(rates[0]) + tail1;
  C[FSZO_LZ2] = fszo_block_cost(rates[8]) + tail2;
  C[FSZO_LZ1C] = 4u + fszo_block_cost(r1c0) + tail1;
  C[FSZO_LZ2C] = 4u + fszo_block_cost(r2c0) + tail2;
}

// Reading: the first strict minimum in the listed order, so ties go to LZ1 over LZ2
// and centring is taken only when strictly cheaper ("enabled only when its 4-byte
// cost for mu is outweighed by the savings", Sec. 4.2.2).
int fszo_select(const uint32_t C[4]) { return fszo_select_f(C, 0); }

// Among the variants whose features are on: LZ2 needs FSZO_OFF_LZ2 clear, the centred
// ones FSZO_OFF_CENTER clear (and LZ2C both).
int fszo_select_f(const uint32_t C[4], uint32_t off) {
  const bool on[4] = {true, !(off & FSZO_OFF_LZ2), !(off & FSZO_OFF_CENTER),
                      !(off & FSZO_OFF_LZ2) && !(off & FSZO_OFF_CENTER)};
  int best = 0;
  for (int v = 1; v < 4; ++v)
    if (on[v] && C[v] < C[best]) best = v;
  return best;
}

int fszo_features_valid(uint32_t off) {
  // bits 8-15 name the tile configuration (fszo_tile_word); the rest are features
  if (((off >> 8) & 0xF) > 1 || ((off >> 12) & 0xF) > 2) return 0;
  off &= ~uint32_t(0xFF00);
  if (off & ~uint32_t(FSZO_OFF_CROSS | FSZO_OFF_CENTER | FSZO_OFF_LZ2)) return 0;
  // centring is defined on the carried state (Eq. 4): off with it
  if ((off & FSZO_OFF_CROSS) && !(off & FSZO_OFF_CENTER)) return 0;
  return 1;
}

uint64_t fszo_compress_bound(uint64_t n) {
  uint64_t T = tiles_of(n);
  return kPreamble + 8 * T + 772 * T;
}

}  // extern "C"

namespace {

// Steps 1-5 of Sec. 3.1 for one tile: quantize, tile mean, four-way costs, select, then the
// 8 rate-header bytes and the tile's data appended to `data`.
void encode_tile(const float dt[256], float r, int force_variant, uint32_t off, uint8_t header[8],
                 std::vector<uint8_t>& data) {
  int32_t q[kTile], l[kTile];
  // Step 1: quantize (Sec. 3.1, Sec. 4.2.2).
  for (int i = 0; i < kTile; ++i) q[i] = fszo_quantize(dt[i], r);
  int32_t mu = fszo_tile_mu(dt, r);
  // Steps 2-3: four-way evaluation and adaptive select.
  uint32_t C[4];
  uint8_t rates[32];
  fszo_tile_costs_single_pass_f(q, mu, off, C, rates);
  const int v = force_variant >= 0 ? force_variant : fszo_select_f(C, off);
  const bool centred = (v == FSZO_LZ1C || v == FSZO_LZ2C);
  const bool second = (v == FSZO_LZ2 || v == FSZO_LZ2C);
  // Rate header (Sec. 3.1 "Compressed format"): block 0 carries bit 7 = LZ order
  // (set for second order), bit 6 = centring, bits 4-0 = rate; blocks 1-7 the rate.
  for (int b = 0; b < kBlocksPerTile; ++b) header[b] = rates[v * 8 + b];
  header[0] = uint8_t(header[0] | (second ? 0x80 : 0) | (centred ? 0x40 : 0));
  // Step 5: encode with the selected variant.
  fszo_tile_residuals_f(q, mu, v, off, l);
  if (centred) {
    // Tile mean: a 4-byte float stored inline, first in the tile's data (reading
    // of "stored inline"); it holds the integer mu exactly.
    float muf = float(mu);
    uint32_t bits;
    std::memcpy(&bits, &muf, 4);
    uint8_t tmp[4];
    put_u32(tmp, bits);
    data.insert(data.end(), tmp, tmp + 4);
  }
  for (int b = 0; b < kBlocksPerTile; ++b) {
    uint32_t rb = rates[v * 8 + b];
    if (rb == 0) continue;  // zero-rate blocks store nothing
    uint32_t sign = 0;
    for (int j = 0; j < kBlock; ++j)
      if (l[b * kBlock + j] < 0) sign |= 1u << (31 - j);
    put_word_be(data, sign);
    for (uint32_t k = 0; k < rb; ++k) {  // bit-plane k, least significant plane first
      uint32_t w = 0;
      for (int j = 0; j < kBlock; ++j)
        if ((uabs(l[b * kBlock + j]) >> k) & 1u) w |= 1u << (31 - j);
      put_word_be(data, w);
    }
  }
}

void load_tile(const float* d, uint64_t n, uint64_t t, float dt[256]) {
  // Zero padding of a partial last tile (reading: the paper is silent).
  for (int i = 0; i < kTile; ++i) {
    uint64_t g = t * kTile + uint64_t(i);
    dt[i] = g < n ? d[g] : 0.0f;
  }
}

}  // namespace

extern "C" {

int fszo_compress_tiles(const float* d, uint64_t n, float r, uint64_t t0, uint64_t t1,
                        uint8_t* header_out, uint8_t* data_out, uint64_t data_cap,
                        uint64_t* data_bytes) {
  return fszo_compress_tiles_f(d, n, r, t0, t1, 0, header_out, data_out, data_cap, data_bytes);
}

int fszo_compress_tiles_f(const float* d, uint64_t n, float r, uint64_t t0, uint64_t t1,
                          uint32_t off, uint8_t* header_out, uint8_t* data_out,
                          uint64_t data_cap, uint64_t* data_bytes) {
  if (t1 < t0 || t1 > tiles_of(n) || !fszo_features_valid(off)) return FSZO_ERR_INVALID_ARG;
  std::vector<uint8_t> data;
  float dt[kTile];
  for (uint64_t t = t0; t < t1; ++t) {
    load_tile(d, n, t, dt);
    encode_tile(dt, r, -1, off, header_out + 8 * (t - t0), data);
  }
  if (data_bytes) *data_bytes = data.size();
  if (data.size() > data_cap) return FSZO_ERR_CAPACITY;
  if (!data.empty()) std::memcpy(data_out, data.data(), data.size());
  return FSZO_OK;
}

// Preamble (this project's addition; little-endian fields): magic, version, ndim, mode, n,
// dims, requested eb, step s, method word (features switched off; 0: the full method),
// data bytes.
void fszo_write_preamble(uint8_t* out, uint32_t ndim, const uint64_t* dims, uint64_t n, int mode,
                         double eb_req, float s, uint32_t method_word, uint64_t data_bytes) {
  std::memset(out, 0, kPreamble);
  out[0] = 'F'; out[1] = 'S'; out[2] = 'Z'; out[3] = '1';
  put_u16(out + 4, 1);
  out[6] = uint8_t(ndim);
  out[7] = uint8_t(mode);
  put_u64(out + 8, n);
  for (uint32_t k = 0; k < 3; ++k) put_u64(out + 16 + 8 * k, k < ndim ? dims[k] : 0);
  uint64_t ebits;
  std::memcpy(&ebits, &eb_req, 8);
  put_u64(out + 40, ebits);
  uint32_t sbits;
  std::memcpy(&sbits, &s, 4);
  put_u32(out + 48, sbits);
  put_u32(out + 52, method_word);
  put_u64(out + 56, data_bytes);
}

int fszo_compress(const float* d, uint32_t ndim, const uint64_t* dims, int mode, double eb_req,
                  uint8_t* out, uint64_t out_capacity, uint64_t* out_bytes, int force_variant) {
  return fszo_compress_f(d, ndim, dims, mode, eb_req, 0, out, out_capacity, out_bytes,
                         force_variant);
}

int fszo_compress_f(const float* d, uint32_t ndim, const uint64_t* dims, int mode, double eb_req,
                    uint32_t off, uint8_t* out, uint64_t out_capacity, uint64_t* out_bytes,
                    int force_variant) {
  if (ndim < 1 || ndim > 3 || dims == nullptr) return FSZO_ERR_INVALID_ARG;
  if (force_variant < -1 || force_variant > 3) return FSZO_ERR_INVALID_ARG;
  if (!fszo_features_valid(off)) return FSZO_ERR_INVALID_ARG;
  if (force_variant >= 0) {  // a forced variant must be one whose features are on
    if ((force_variant == FSZO_LZ2 || force_variant == FSZO_LZ2C) && (off & FSZO_OFF_LZ2))
      return FSZO_ERR_INVALID_ARG;
    if (force_variant >= FSZO_LZ1C && (off & FSZO_OFF_CENTER)) return FSZO_ERR_INVALID_ARG;
  }
  uint64_t n = 1;
  for (uint32_t k = 0; k < ndim; ++k) {
    if (dims[k] != 0 && n > kMaxElems / dims[k]) return FSZO_ERR_INVALID_ARG;
    n *= dims[k];
  }
  if (n > kMaxElems) return FSZO_ERR_INVALID_ARG;
  float vmin, vmax;
  int fin;
  fszo_stats(d, n, &vmin, &vmax, &fin);
  fszo_params_t p;
  int st = fszo_params(mode, eb_req, vmin, vmax, fin, n, &p);
  if (st != FSZO_OK) return st;

  const uint64_t T = tiles_of(n);
  std::vector<uint8_t> header(8 * T);
  std::vector<uint8_t> data;
  data.reserve(size_t(n));
  float dt[kTile];
  for (uint64_t t = 0; t < T; ++t) {
    load_tile(d, n, t, dt);
    encode_tile(dt, p.r, force_variant, off, header.data() + 8 * t, data);
  }
  const uint64_t total = kPreamble + 8 * T + uint64_t(data.size());
  if (out_bytes) *out_bytes = total;
  if (total > out_capacity) return FSZO_ERR_CAPACITY;
  fszo_write_preamble(out, ndim, dims, n, mode, eb_req, p.s, off, uint64_t(data.size()));
  if (T) std::memcpy(out + kPreamble, header.data(), header.size());
  if (!data.empty()) std::memcpy(out + kPreamble + 8 * T, data.data(), data.size());
  return FSZO_OK;
}

int fszo_read_preamble(const uint8_t* in, uint64_t in_bytes, uint64_t* n, uint32_t* ndim,
                       uint64_t dims[3], double* eb_req, float* s, uint64_t* data_bytes) {
  return fszo_read_preamble_f(in, in_bytes, n, ndim, dims, eb_req, s, data_bytes, nullptr);
}

int fszo_read_preamble_f(const uint8_t* in, uint64_t in_bytes, uint64_t* n, uint32_t* ndim,
                         uint64_t dims[3], double* eb_req, float* s, uint64_t* data_bytes,
                         uint32_t* features_off) {
  if (in == nullptr || in_bytes < kPreamble) return FSZO_ERR_CORRUPT;
  if (in[0] != 'F' || in[1] != 'S' || in[2] != 'Z' || in[3] != '1') return FSZO_ERR_CORRUPT;
  if (get_u16(in + 4) != 1) return FSZO_ERR_CORRUPT;
  uint32_t nd = in[6];
  if (nd < 1 || nd > 3 || in[7] > 1) return FSZO_ERR_CORRUPT;
  uint64_t nn = get_u64(in + 8);
  uint64_t prod = 1;
  for (uint32_t k = 0; k < 3; ++k) {
    uint64_t dk = get_u64(in + 16 + 8 * k);
    if (k >= nd) { if (dk != 0) return FSZO_ERR_CORRUPT; continue; }
    if (dk != 0 && prod > kMaxElems / dk) return FSZO_ERR_CORRUPT;
    prod *= dk;
    if (dims) dims[k] = dk;
  }
  if (prod != nn || nn > kMaxElems) return FSZO_ERR_CORRUPT;
  uint64_t ebits = get_u64(in + 40); double eb; std::memcpy(&eb, &ebits, 8);
  uint32_t sbits = get_u32(in + 48); float sv; std::memcpy(&sv, &sbits, 4);
  if (!(eb > 0.0) || !std::isfinite(eb)) return FSZO_ERR_CORRUPT;
  if (!(sv >= std::ldexp(1.0f, -99)) || !std::isfinite(sv)) return FSZO_ERR_CORRUPT;
  const uint32_t off = get_u32(in + 52);
  if (!fszo_features_valid(off)) return FSZO_ERR_CORRUPT;
  uint64_t db = get_u64(in + 56);
  int cfgB = 32, cfgT = 8;
  tile_cfg_from_word(off, &cfgB, &cfgT);
  const uint64_t hdr = uint64_t(cfgT) * ((nn + uint64_t(cfgB * cfgT) - 1) / uint64_t(cfgB * cfgT));
  if (in_bytes - kPreamble < hdr) return FSZO_ERR_CORRUPT;
  if (db > in_bytes - kPreamble - hdr) return FSZO_ERR_CORRUPT;
  if (n) *n = nn;
  if (ndim) *ndim = nd;
  if (eb_req) *eb_req = eb;
  if (s) *s = sv;
  if (data_bytes) *data_bytes = db;
  if (features_off) *features_off = off;
  return FSZO_OK;
}

// ------------------------------------------------------------------ tile configurations
//
// Sec. 6.5 (Table 8) sweeps the block size B (elements per block) and the blocks per tile
// T. A configured tile has B T elements and T header bytes (block 0's byte carries the
// order and centring flags as in the default). For B = 64 a sign map or bit-plane is an
// 8-byte word, element j at bit 63 - j, serialised most significant byte first (the B = 32
// word's rule at twice the width), so S_b = (B / 8)(1 + r_b) bytes for r_b > 0 (Eq. 3).
// The tile mean sums 8-element runs left to right and then pairs them as the default does
// (P_j += P_{j+h}, h = R/2 .. 1 for R runs), times 1/(B T). This path evaluates the four
// variants by their definition (one residual pass per variant) and takes the first strict
// minimum among the enabled ones. With B = 32, T = 8 it reproduces the default stream.

extern "C" uint32_t fszo_tile_word(int B, int T) {
  const uint32_t bcode = B == 64 ? 1u : 0u;
  const uint32_t tcode = T == 4 ? 1u : T == 16 ? 2u : 0u;
  return (bcode << 8) | (tcode << 12);
}

namespace {

uint32_t cfg_block_cost(uint32_t rate, int B) {
  return rate == 0 ? 0u : uint32_t(B / 8) * (1u + rate);
}

// Serialises the low B bits of w most significant first (B / 8 bytes).
void put_bits_be(std::vector<uint8_t>& out, uint64_t w, int B) {
  for (int k = B / 8 - 1; k >= 0; --k) out.push_back(uint8_t(w >> (8 * k)));
}
uint64_t get_bits_be(const uint8_t* p, int B) {
  uint64_t w = 0;
  for (int k = 0; k < B / 8; ++k) w = (w << 8) | p[k];
  return w;
}

int32_t cfg_tile_mu(const std::vector<float>& dt, float r) {
  const int R = int(dt.size()) / 8;
  std::vector<float> P(R);
  for (int j = 0; j < R; ++j) {
    float acc = dt[8 * j];
    for (int i = 1; i < 8; ++i) acc = acc + dt[8 * j + i];
    P[j] = acc;
  }
  for (int h = R / 2; h >= 1; h /= 2)
    for (int j = 0; j < h; ++j) P[j] = P[j] + P[j + h];
  const float dbar = P[0] * (1.0f / float(dt.size()));  // a power of two: exact
  return fszo_quantize(dbar, r);
}

void cfg_residuals(const std::vector<int32_t>& q, int32_t mu, int variant, uint32_t off, int B,
                   std::vector<int32_t>& l) {
  const bool centred = (variant == FSZO_LZ1C || variant == FSZO_LZ2C);
  const bool second = (variant == FSZO_LZ2 || variant == FSZO_LZ2C);
  int32_t prev1 = 0, prev2 = 0;
  l.assign(q.size(), 0);
  for (size_t i = 0; i < q.size(); ++i) {
    if ((off & FSZO_OFF_CROSS) && i % size_t(B) == 0) prev1 = prev2 = 0;
    const int32_t qh = centred ? wsub(q[i], mu) : q[i];
    l[i] = second ? wadd(wsub(qh, wadd(prev1, prev1)), prev2) : wsub(qh, prev1);
    prev2 = prev1;
    prev1 = qh;
  }
}

// One configured tile: header (T bytes) and data appended (steps 1-5 of Sec. 3.1).
void cfg_encode_tile(const std::vector<float>& dt, float r, uint32_t off, int B, int T,
                     uint8_t* header, std::vector<uint8_t>& data) {
  const int tile = B * T;
  std::vector<int32_t> q(tile), l;
  for (int i = 0; i < tile; ++i) q[i] = fszo_quantize(dt[i], r);
  const int32_t mu = cfg_tile_mu(dt, r);
  uint32_t C[4];
  std::vector<uint8_t> rates(4 * size_t(T));
  for (int v = 0; v < 4; ++v) {
    cfg_residuals(q, mu, v, off, B, l);
    uint32_t cost = (v == FSZO_LZ1C || v == FSZO_LZ2C) ? 4u : 0u;
    for (int b = 0; b < T; ++b) {
      uint32_t m = 0;
      for (int j = 0; j < B; ++j) { const uint32_t a = uabs(l[b * B + j]); if (a > m) m = a; }
      rates[size_t(v) * T + b] = uint8_t(fszo_rate(m));
      cost += cfg_block_cost(rates[size_t(v) * T + b], B);
    }
    C[v] = cost;
  }
  const int v = fszo_select_f(C, off);
  const bool centred = (v == FSZO_LZ1C || v == FSZO_LZ2C);
  const bool second = (v == FSZO_LZ2 || v == FSZO_LZ2C);
  for (int b = 0; b < T; ++b) header[b] = rates[size_t(v) * T + b];
  header[0] = uint8_t(header[0] | (second ? 0x80 : 0) | (centred ? 0x40 : 0));
  cfg_residuals(q, mu, v, off, B, l);
  if (centred) {
    const float muf = float(mu);
    uint32_t bits;
    std::memcpy(&bits, &muf, 4);
    uint8_t tmp[4];
    put_u32(tmp, bits);
    data.insert(data.end(), tmp, tmp + 4);
  }
  for (int b = 0; b < T; ++b) {
    const uint32_t rb = rates[size_t(v) * T + b];
    if (rb == 0) continue;
    uint64_t sign = 0;
    for (int j = 0; j < B; ++j)
      if (l[b * B + j] < 0) sign |= uint64_t(1) << (B - 1 - j);
    put_bits_be(data, sign, B);
    for (uint32_t k = 0; k < rb; ++k) {
      uint64_t w = 0;
      for (int j = 0; j < B; ++j)
        if ((uabs(l[b * B + j]) >> k) & 1u) w |= uint64_t(1) << (B - 1 - j);
      put_bits_be(data, w, B);
    }
  }
}

// Decodes a configured stream (preamble already checked) into q.
int cfg_decode_to_q(const uint8_t* in, uint64_t in_bytes, uint64_t n, uint32_t word, uint64_t db,
                    std::vector<int32_t>& qout) {
  int B, T;
  if (!tile_cfg_from_word(word, &B, &T)) return FSZO_ERR_CORRUPT;
  const int tile = B * T;
  const uint64_t NT = (n + uint64_t(tile) - 1) / uint64_t(tile);
  if ((in_bytes - kPreamble) / uint64_t(T) < NT) return FSZO_ERR_CORRUPT;
  const uint8_t* header = in + kPreamble;
  const uint8_t* data = header + uint64_t(T) * NT;
  if (db > in_bytes - kPreamble - uint64_t(T) * NT) return FSZO_ERR_CORRUPT;
  std::vector<uint64_t> offs(NT + 1, 0);
  for (uint64_t t = 0; t < NT; ++t) {
    const uint8_t* h = header + uint64_t(T) * t;
    if (h[0] & 0x20) return FSZO_ERR_CORRUPT;
    if ((h[0] & 0x80) && (word & FSZO_OFF_LZ2)) return FSZO_ERR_CORRUPT;
    if ((h[0] & 0x40) && (word & FSZO_OFF_CENTER)) return FSZO_ERR_CORRUPT;
    uint64_t bytes = (h[0] & 0x40) ? 4 : 0;
    for (int b = 0; b < T; ++b) {
      if (b > 0 && (h[b] & 0xE0)) return FSZO_ERR_CORRUPT;
      bytes += cfg_block_cost(h[b] & 0x1F, B);
    }
    offs[t + 1] = offs[t] + bytes;
  }
  if (offs[NT] != db) return FSZO_ERR_CORRUPT;
  qout.assign(size_t(NT) * size_t(tile), 0);
  std::vector<int32_t> l(tile);
  for (uint64_t t = 0; t < NT; ++t) {
    const uint8_t* h = header + uint64_t(T) * t;
    const bool second = (h[0] & 0x80) != 0, centred = (h[0] & 0x40) != 0;
    const uint8_t* p = data + offs[t];
    int32_t mu = 0;
    if (centred) {
      const uint32_t bits = get_u32(p);
      float muf;
      std::memcpy(&muf, &bits, 4);
      if (!(std::fabs(muf) <= 16777216.0f) || std::nearbyint(muf) != muf) return FSZO_ERR_CORRUPT;
      mu = int32_t(muf);
      p += 4;
    }
    for (int b = 0; b < T; ++b) {
      const uint32_t rb = h[b] & 0x1F;
      for (int j = 0; j < B; ++j) l[b * B + j] = 0;
      if (rb == 0) continue;
      const uint64_t sign = get_bits_be(p, B);
      p += B / 8;
      std::vector<uint32_t> mag(B, 0);
      for (uint32_t k = 0; k < rb; ++k) {
        const uint64_t w = get_bits_be(p, B);
        p += B / 8;
        for (int j = 0; j < B; ++j)
          if ((w >> (B - 1 - j)) & 1u) mag[j] |= 1u << k;
      }
      for (int j = 0; j < B; ++j) {
        const bool neg = (sign >> (B - 1 - j)) & 1u;
        l[b * B + j] = neg ? int32_t(uint32_t(0) - mag[j]) : int32_t(mag[j]);
      }
    }
    int32_t prev1 = 0, prev2 = 0;
    for (int i = 0; i < tile; ++i) {
      if ((word & FSZO_OFF_CROSS) && i % B == 0) prev1 = prev2 = 0;
      const int32_t qh = second ? wsub(wadd(l[i], wadd(prev1, prev1)), prev2) : wadd(l[i], prev1);
      prev2 = prev1;
      prev1 = qh;
      qout[size_t(t) * size_t(tile) + size_t(i)] = wadd(qh, mu);
    }
  }
  return FSZO_OK;
}

}  // namespace

extern "C" {

uint64_t fszo_compress_bound_cfg(uint64_t n, int B, int T) {
  const uint64_t NT = (n + uint64_t(B * T) - 1) / uint64_t(B * T);
  return kPreamble + uint64_t(T) * NT + (uint64_t(T) * uint64_t(B / 8) * 24 + 4) * NT;
}

int fszo_compress_cfg(const float* d, uint32_t ndim, const uint64_t* dims, int mode, double eb_req,
                      uint32_t off, int B, int T, uint8_t* out, uint64_t out_capacity,
                      uint64_t* out_bytes) {
  if ((B != 32 && B != 64) || (T != 4 && T != 8 && T != 16)) return FSZO_ERR_INVALID_ARG;
  if (ndim < 1 || ndim > 3 || dims == nullptr || !fszo_features_valid(off & 7u)) return FSZO_ERR_INVALID_ARG;
  uint64_t n = 1;
  for (uint32_t k = 0; k < ndim; ++k) {
    if (dims[k] != 0 && n > kMaxElems / dims[k]) return FSZO_ERR_INVALID_ARG;
    n *= dims[k];
  }
  float vmin, vmax;
  int fin;
  fszo_stats(d, n, &vmin, &vmax, &fin);
  fszo_params_t p;
  const int st = fszo_params(mode, eb_req, vmin, vmax, fin, n, &p);
  if (st != FSZO_OK) return st;
  const int tile = B * T;
  const uint64_t NT = (n + uint64_t(tile) - 1) / uint64_t(tile);
  std::vector<uint8_t> header(uint64_t(T) * NT), data;
  std::vector<float> dt(tile);
  for (uint64_t t = 0; t < NT; ++t) {
    for (int i = 0; i < tile; ++i) {  // zero padding of a partial last tile
      const uint64_t g = t * uint64_t(tile) + uint64_t(i);
      dt[i] = g < n ? d[g] : 0.0f;
    }
    cfg_encode_tile(dt, p.r, off & 7u, B, T, header.data() + uint64_t(T) * t, data);
  }
  const uint64_t total = kPreamble + header.size() + data.size();
  if (out_bytes) *out_bytes = total;
  if (total > out_capacity) return FSZO_ERR_CAPACITY;
  std::memset(out, 0, kPreamble);
  out[0] = 'F'; out[1] = 'S'; out[2] = 'Z'; out[3] = '1';
  put_u16(out + 4, 1);
  out[6] = uint8_t(ndim);
  out[7] = uint8_t(mode);
  put_u64(out + 8, n);
  for (uint32_t k = 0; k < 3; ++k) put_u64(out + 16 + 8 * k, k < ndim ? dims[k] : 0);
  uint64_t ebits;
  std::memcpy(&ebits, &eb_req, 8);
  put_u64(out + 40, ebits);
  uint32_t sbits;
  std::memcpy(&sbits, &p.s, 4);
  put_u32(out + 48, sbits);
  put_u32(out + 52, (off & 7u) | fszo_tile_word(B, T));
  put_u64(out + 56, uint64_t(data.size()));
  if (!header.empty()) std::memcpy(out + kPreamble, header.data(), header.size());
  if (!data.empty()) std::memcpy(out + kPreamble + header.size(), data.data(), data.size());
  return FSZO_OK;
}

}  // extern "C"

namespace {

// Decompression steps d4-d5 (Sec. 3.1 "Decompression") for one tile: its 8 header bytes h,
// its data p (validated by the caller's scan of the header), writing its 256 integers q.
int decode_tile(const uint8_t* h, const uint8_t* p, uint32_t feat_off, int32_t q[256]) {
  int32_t l[kTile];
  const bool second = (h[0] & 0x80) != 0;
  const bool centred = (h[0] & 0x40) != 0;
  int32_t mu = 0;
  if (centred) {
    uint32_t bits = get_u32(p); float muf; std::memcpy(&muf, &bits, 4);
    // The mean slot must hold an integer of magnitude at most 2^24.
    if (!(std::fabs(muf) <= 16777216.0f) || std::nearbyint(muf) != muf) return FSZO_ERR_CORRUPT;
    mu = int32_t(muf);
    p += 4;
  }
  // d4: decode and bit-unshuffle.
  for (int b = 0; b < kBlocksPerTile; ++b) {
    uint32_t rb = h[b] & 0x1F;
    for (int j = 0; j < kBlock; ++j) l[b * kBlock + j] = 0;
    if (rb == 0) continue;
    uint32_t sign = get_word_be(p); p += 4;
    uint32_t mag[kBlock] = {0};
    for (uint32_t k = 0; k < rb; ++k) {
      uint32_t w = get_word_be(p); p += 4;
      for (int j = 0; j < kBlock; ++j)
        if ((w >> (31 - j)) & 1u) mag[j] |= 1u << k;
    }
    for (int j = 0; j < kBlock; ++j) {
      bool neg = (sign >> (31 - j)) & 1u;
      l[b * kBlock + j] = neg ? int32_t(uint32_t(0) - mag[j]) : int32_t(mag[j]);
    }
  }
  // d5: inverse prediction with the carried state, then + mu.
  int32_t prev1 = 0, prev2 = 0;
  for (int i = 0; i < kTile; ++i) {
    if ((feat_off & FSZO_OFF_CROSS) && i % kBlock == 0) prev1 = prev2 = 0;  // independent blocks
    int32_t qh = second ? wsub(wadd(l[i], wadd(prev1, prev1)), prev2) : wadd(l[i], prev1);
    prev2 = prev1;
    prev1 = qh;
    q[i] = wadd(qh, mu);
  }
  return FSZO_OK;
}

// Decompression steps d1-d5 (Sec. 3.1 "Decompression"), writing the integers q.
int decode_to_q(const uint8_t* in, uint64_t in_bytes, std::vector<int32_t>& qout, uint64_t cap,
                uint64_t* n_out, float* s_out) {
  uint64_t n, db; uint32_t nd; uint64_t dims[3]; double eb; float s; uint32_t feat_off;
  int st = fszo_read_preamble_f(in, in_bytes, &n, &nd, dims, &eb, &s, &db, &feat_off);
  if (st != FSZO_OK) return st;
  if (n > cap) return FSZO_ERR_CAPACITY;
  if (feat_off & 0xFF00u) {  // a configured tile (Sec. 6.5)
    st = cfg_decode_to_q(in, in_bytes, n, feat_off, db, qout);
    if (st != FSZO_OK) return st;
    if (n_out) *n_out = n;
    if (s_out) *s_out = s;
    return FSZO_OK;
  }
  const uint64_t T = tiles_of(n);
  const uint8_t* header = in + kPreamble;
  const uint8_t* data = header + 8 * T;
  // d1-d3: rates and tile metadata, block sizes, and tile offsets by an exclusive scan.
  std::vector<uint64_t> off(T + 1, 0);
  for (uint64_t t = 0; t < T; ++t) {
    const uint8_t* h = header + 8 * t;
    if (h[0] & 0x20) return FSZO_ERR_CORRUPT;  // bit 5 of block 0 is unused
    // a tile may not use a feature the stream has switched off
    if ((h[0] & 0x80) && (feat_off & FSZO_OFF_LZ2)) return FSZO_ERR_CORRUPT;
    if ((h[0] & 0x40) && (feat_off & FSZO_OFF_CENTER)) return FSZO_ERR_CORRUPT;
    uint64_t bytes = (h[0] & 0x40) ? 4 : 0;
    for (int b = 0; b < kBlocksPerTile; ++b) {
      if (b > 0 && (h[b] & 0xE0)) return FSZO_ERR_CORRUPT;  // blocks 1-7 carry only a rate
      bytes += fszo_block_cost(h[b] & 0x1F);
    }
    off[t + 1] = off[t] + bytes;
  }
  if (off[T] != db) return FSZO_ERR_CORRUPT;
  qout.assign(size_t(T * kTile), 0);
  for (uint64_t t = 0; t < T; ++t) {
    st = decode_tile(header + 8 * t, data + off[t], feat_off, qout.data() + t * kTile);
    if (st != FSZO_OK) return st;
  }
  if (n_out) *n_out = n;
  if (s_out) *s_out = s;
  return FSZO_OK;
}

}  // namespace

// PSNR against the original's value range, the usual definition of the error-bounded
// compression literature (the paper plots it, Fig. 8, without printing the formula).
int fszo_quality(const float* d, const float* y, uint64_t n, double eb, uint64_t stream_bytes,
                 fszo_quality_t* q) {
  if (q == nullptr || n == 0 || d == nullptr || y == nullptr) return FSZO_ERR_INVALID_ARG;
  q->n = n;
  q->over_bound = 0;
  q->max_abs_err = 0.0;
  q->sum_sq_err = 0.0;
  q->vmin = double(d[0]);
  q->vmax = double(d[0]);
  for (uint64_t i = 0; i < n; ++i) {
    const double e = double(d[i]) - double(y[i]);
    const double a = std::fabs(e);
    if (a > q->max_abs_err) q->max_abs_err = a;
    if (a > eb) q->over_bound += 1;
    q->sum_sq_err += e * e;
    if (double(d[i]) < q->vmin) q->vmin = double(d[i]);
    if (double(d[i]) > q->vmax) q->vmax = double(d[i]);
  }
  const double range = q->vmax - q->vmin;
  const double mse = q->sum_sq_err / double(n);
  q->psnr_db = mse > 0.0 ? 20.0 * std::log10(range) - 10.0 * std::log10(mse) : INFINITY;
  q->nrmse = range > 0.0 ? std::sqrt(mse) / range : 0.0;
  q->bit_rate = 8.0 * double(stream_bytes) / double(n);
  return FSZO_OK;
}

int fszo_decompress_q(const uint8_t* in, uint64_t in_bytes, int32_t* q_out,
                      uint64_t out_capacity_elems, uint64_t* n_out) {
  std::vector<int32_t> q; uint64_t n = 0; float s;
  int st = decode_to_q(in, in_bytes, q, out_capacity_elems, &n, &s);
  if (st != FSZO_OK) return st;
  for (uint64_t i = 0; i < n; ++i) q_out[i] = q[size_t(i)];
  if (n_out) *n_out = n;
  return FSZO_OK;
}

// Tiles [t0, t1) of a stream of the default tile configuration, the first of them starting
// data_off bytes into the data region (the caller's scan of the header): their elements
// [256 t0, min(n, 256 t1)) dequantized into out (indexed from element 256 t0).
int fszo_decompress_tiles(const uint8_t* in, uint64_t in_bytes, uint64_t t0, uint64_t t1,
                          uint64_t data_off, float* out) {
  uint64_t n, db; uint32_t nd; uint64_t dims[3]; double eb; float s; uint32_t feat_off;
  int st = fszo_read_preamble_f(in, in_bytes, &n, &nd, dims, &eb, &s, &db, &feat_off);
  if (st != FSZO_OK) return st;
  const uint64_t T = tiles_of(n);
  if ((feat_off & 0xFF00u) || t1 < t0 || t1 > T || data_off > db) return FSZO_ERR_INVALID_ARG;
  const uint8_t* header = in + kPreamble;
  const uint8_t* p = header + 8 * T + data_off;
  int32_t q[kTile];
  for (uint64_t t = t0; t < t1; ++t) {
    const uint8_t* h = header + 8 * t;
    st = decode_tile(h, p, feat_off, q);
    if (st != FSZO_OK) return st;
    uint64_t bytes = (h[0] & 0x40) ? 4 : 0;
    for (int b = 0; b < kBlocksPerTile; ++b) bytes += fszo_block_cost(h[b] & 0x1F);
    p += bytes;
    for (int i = 0; i < kTile; ++i) {
      const uint64_t g = t * kTile + uint64_t(i);
      if (g < n) out[g - t0 * kTile] = fszo_dequantize(q[i], s);
    }
  }
  return FSZO_OK;
}

int fszo_decompress(const uint8_t* in, uint64_t in_bytes, float* out, uint64_t out_capacity_elems,
                    uint64_t* n_out) {
  std::vector<int32_t> q; uint64_t n = 0; float s;
  int st = decode_to_q(in, in_bytes, q, out_capacity_elems, &n, &s);
  if (st != FSZO_OK) return st;
  // d5 (dequantize): d' = fl32(float(q) x s); padding elements are dropped.
  for (uint64_t i = 0; i < n; ++i) out[i] = fszo_dequantize(q[size_t(i)], s);
  if (n_out) *n_out = n;
  return FSZO_OK;
}

}  // extern "C"
