// Tile configurations of Sec. 6.5 (Table 8): B elements per block (32 or 64) and T blocks
// per tile (4, 8 or 16). A configured stream has T header bytes per tile (block 0's byte
// carries the order and centring flags) and B-bit sign and plane words (B / 8 bytes,
// element j at bit B - 1 - j, most significant byte first), so S_b = (B / 8)(1 + r_b) for
// r_b > 0. The preamble's method word (byte 52) carries the configuration in bits 8-15.
//
// A generic path for the configuration sweep, in the paper's two-read structure: the
// value-range pass; a cost pass (one warp per tile: the four variants' costs, the
// selection, the rate header, the tile's size); an exclusive scan of the sizes; an
// encoding pass (the tile read again, each 32-element row's bit-planes built by one
// warp bit transpose); the preamble. Element i of a tile sits in register i / 32 of lane
// i % 32, so every load and store of a register is one coalesced 128-byte row. The
// decoder mirrors it (the same transpose, then prefix sums in element order). The
// specialised single-pass kernels cover the default configuration only.
#include <algorithm>

#include "fsz_internal.cuh"

namespace fsz {

namespace {

constexpr int kTiledThreads = 256;  // 8 warps, a tile each at a time
constexpr int kTiledWarps = kTiledThreads / 32;
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4 * kScanThreads;  // tile sizes per CTA in the scan
constexpr uint32_t FULL = 0xffffffffu;

uint32_t tile_word_of(int B, int T) {
  return (B == 64 ? 1u : 0u) << 8 | (T == 4 ? 1u : T == 16 ? 2u : 0u) << 12;
}

__host__ __device__ __forceinline__ bool config_of(uint32_t word, int* B, int* T) {
  const uint32_t bc = (word >> 8) & 0xF, tc = (word >> 12) & 0xF;
  if (bc > 1 || tc > 2 || (word & 0xFFFF00F8u)) return false;
  *B = bc == 1 ? 64 : 32;
  *T = tc == 1 ? 4 : tc == 2 ? 16 : 8;
  return true;
}

// Per-call arrays after the value-range pass's workspace.
struct TiledPtrs {
  uint32_t* sizes;   // tile bytes
  uint64_t* offs;    // exclusive byte offsets inside the tile data
  uint64_t* rec;     // cost pass -> encoding pass: variant | mu << 32
  uint64_t* part;    // scan: CTA sums, then their exclusive prefix; part[nparts] = total
  uint64_t ntiles;
};

struct TiledLayout {
  WsLayout L;
  uint64_t sizes_off, offs_off, rec_off, part_off, bytes, max_tiles;
};

TiledLayout tiled_layout(uint64_t n) {
  TiledLayout t;
  t.L = ws_layout((n + kTile - 1) / kTile, 1);
  t.max_tiles = (n + 127) / 128 + 1;  // the smallest tile has 128 elements
  auto a16 = [](uint64_t x) { return (x + 15) & ~uint64_t(15); };
  t.sizes_off = a16(t.L.bytes);
  t.offs_off = a16(t.sizes_off + 4 * t.max_tiles);
  t.rec_off = a16(t.offs_off + 8 * t.max_tiles);
  t.part_off = a16(t.rec_off + 8 * t.max_tiles);
  t.bytes = t.part_off + 8 * (t.max_tiles / kScanItems + 2);
  return t;
}

TiledPtrs tiled_ptrs(void* ws, const TiledLayout& t, uint64_t ntiles) {
  uint8_t* b = static_cast<uint8_t*>(ws);
  return TiledPtrs{reinterpret_cast<uint32_t*>(b + t.sizes_off), reinterpret_cast<uint64_t*>(b + t.offs_off),
                   reinterpret_cast<uint64_t*>(b + t.rec_off), reinterpret_cast<uint64_t*>(b + t.part_off),
                   ntiles};
}

__device__ __forceinline__ uint32_t quantize_bits(float d, float r) {
  return uint32_t(__float_as_int(__fadd_rn(__fmul_rn(d, r), kMagic)) - kMagicBits);
}

__device__ __forceinline__ uint32_t bswap32(uint32_t w) { return __byte_perm(w, 0, 0x0123); }

// A warp's tile buffer in shared memory holds each 32-element row (one register of the
// warp) in kRowWords words, so element e sits at word e + 4 (e / 32). Row writes stay
// conflict-free, and the 128-bit reads of any 8 consecutive lanes at a stride of 4, 8, 16
// or 32 words (a lane's 8-element run, or its E consecutive elements) fall in 8 distinct
// bank groups.
constexpr int kRowWords = 36;
__device__ __forceinline__ int padded(int e) { return e + 4 * (e >> 5); }

// The predecessor of every element of the tile (element 32 k + L sits in register k of
// lane L): one rotation of each register by a lane, lane 0 taking the previous register's
// rotated value (element 32 k - 1); zero before the tile, and before every block when
// `restart` holds (no cross-block state).
template <int B, int E>
__device__ __forceinline__ void predecessors(const uint32_t (&v)[E], bool restart, int lane,
                                             uint32_t (&p)[E]) {
  uint32_t before = 0;  // at lane 0: the element before register k's first
#pragma unroll
  for (int k = 0; k < E; ++k) {
    const uint32_t rot = __shfl_sync(FULL, v[k], (lane + 31) & 31);
    uint32_t pk = lane == 0 ? before : rot;
    if (restart && ((32 * k + lane) % B) == 0) pk = 0;
    p[k] = pk;
    before = rot;
  }
}

// Residuals of one variant (Eqs. 1-2) for the tile held in qh (q, less mu when centred):
// LZ1 from zero predecessors, LZ2 as the LZ1 residuals' own first differences (so
// l2_0 = qh_0 and l2_1 = qh_1 - 2 qh_0), the state running across the whole tile, or
// restarting at every block without the cross-block state.
template <int B, int E>
__device__ __forceinline__ void tile_residuals(const uint32_t (&qh)[E], bool second, bool indep,
                                               int lane, uint32_t (&l)[E]) {
  uint32_t p[E];
  predecessors<B, E>(qh, indep, lane, p);
#pragma unroll
  for (int k = 0; k < E; ++k) l[k] = qh[k] - p[k];
  if (second) {
    predecessors<B, E>(l, indep, lane, p);
#pragma unroll
    for (int k = 0; k < E; ++k) l[k] -= p[k];
  }
}

// Lane constants of warp_transpose32, one per exchange step (j = 16, 8, 4, 2, 1): the
// lane's own bits (the lower lane of a pair keeps the bits outside the low j of each 2j,
// the upper lane those inside) and the rotation that lines the partner's bits up.
struct Xpose {
  uint32_t keep[5];
  uint32_t amt[5];
};

__device__ __forceinline__ Xpose xpose_consts(int lane) {
  Xpose c;
#pragma unroll
  for (int s = 0; s < 5; ++s) {
    const int j = 16 >> s;
    const uint32_t m = j == 16 ? 0x0000FFFFu : j == 8 ? 0x00FF00FFu : j == 4 ? 0x0F0F0F0Fu
                     : j == 2 ? 0x33333333u : 0x55555555u;
    const bool upper = (lane & j) != 0;
    c.keep[s] = upper ? m : ~m;
    c.amt[s] = upper ? uint32_t(32 - j) : uint32_t(j);
  }
  return c;
}

// 32 x 32 bit transpose across the warp, anti-diagonal form: on return bit c of lane L is
// bit 31 - L of lane 31 - c on entry. Five exchange steps (j = 16 .. 1): lanes L and L ^ j
// trade the j x j bit blocks off the diagonal of their 2j x 2j block, each taking a
// rotated copy of the partner's word and a bit-select. Lane L holds plane 31 - L of the
// 32 elements given one per lane (element e at bit 31 - e), and the converse.
__device__ __forceinline__ uint32_t warp_transpose32(uint32_t v, const Xpose& c) {
#pragma unroll
  for (int s = 0; s < 5; ++s) {
    const int j = 16 >> s;
    const uint32_t x = __shfl_xor_sync(FULL, v, j);
    const uint32_t sh = __funnelshift_r(x, x, j == 16 ? 16u : c.amt[s]);  // rotate right
    v = (v & c.keep[s]) | (sh & ~c.keep[s]);
  }
  return v;
}

// OR of |l| over block b (B / 32 registers), warp-wide: the block's rate (Sec. 4.1.2).
template <int B, int E>
__device__ __forceinline__ uint32_t block_rate(const uint32_t (&l)[E], int b) {
  uint32_t m = uabs32(int32_t(l[b * (B / 32)]));
  if (B == 64) m |= uabs32(int32_t(l[b * (B / 32) + (B == 64 ? 1 : 0)]));
  m = __reduce_or_sync(FULL, m);
  return 32u - uint32_t(__clz(int(m)));
}

__device__ __forceinline__ uint32_t cfg_block_cost(uint32_t rate, int B) {
  return rate == 0 ? 0u : uint32_t(B / 8) * (1u + rate);
}

// The tile's elements (zero past n) and their quantized values.
template <int B, int T, int E>
__device__ __forceinline__ void load_tile(const float* in, uint64_t n, uint64_t t, float r, int lane,
                                          float (&d)[E], uint32_t (&q)[E]) {
#pragma unroll
  for (int k = 0; k < E; ++k) {
    const uint64_t i = t * uint64_t(B * T) + uint64_t(32 * k + lane);
    d[k] = i < n ? in[i] : 0.0f;
    q[k] = quantize_bits(d[k], r);
  }
}

// The tile mean in the fixed order: the 8-element runs P_j (elements 8j..8j+7) added left
// to right, then P_j += P_{j+h} for h = R/2 .. 1 (R runs). The tile goes through the
// warp's shared buffer so that lane j adds run j (and j + 32, ...); the first levels of
// the tree stay inside a lane, the last five are shuffles.
template <int B, int T, int E>
__device__ __forceinline__ uint32_t tile_mu(const float (&d)[E], float r, int lane, float* tile) {
  constexpr int R = B * T / 8;
  constexpr int U = (R + 31) / 32;  // runs per lane: 1, 2 or 4
#pragma unroll
  for (int k = 0; k < E; ++k) tile[kRowWords * k + lane] = d[k];
  __syncwarp();
  float P[U];
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int j = lane + 32 * u;
    float acc = 0.0f;
    if (j < R) {
      const float4 x = *reinterpret_cast<const float4*>(tile + padded(8 * j));
      const float4 y = *reinterpret_cast<const float4*>(tile + padded(8 * j + 4));
      acc = __fadd_rn(x.x, x.y);
      acc = __fadd_rn(acc, x.z);
      acc = __fadd_rn(acc, x.w);
      acc = __fadd_rn(acc, y.x);
      acc = __fadd_rn(acc, y.y);
      acc = __fadd_rn(acc, y.z);
      acc = __fadd_rn(acc, y.w);
    }
    P[u] = acc;
  }
  __syncwarp();  // the buffer is the next tile's
  if constexpr (U == 4) {  // h = 64: runs j += j + 64 and j + 32 += j + 96
    P[0] = __fadd_rn(P[0], P[2]);
    P[1] = __fadd_rn(P[1], P[3]);
  }
  if constexpr (U >= 2) P[0] = __fadd_rn(P[0], P[1]);  // h = 32
#pragma unroll
  for (int h = R >= 32 ? 16 : R / 2; h >= 1; h >>= 1) {
    const float y = __shfl_down_sync(FULL, P[0], h);
    if (lane < h) P[0] = __fadd_rn(P[0], y);
  }
  const uint32_t mu = quantize_bits(__fmul_rn(P[0], 1.0f / float(B * T)), r);
  return __shfl_sync(FULL, mu, 0);
}

template <int B, int T>
__global__ void __launch_bounds__(kTiledThreads) fsz_tiled_cost_kernel(KernelArgs a, TiledPtrs p) {
  constexpr int E = B * T / 32;
  __shared__ __align__(16) float s_tile[kTiledWarps][kRowWords * E];
  __shared__ uint8_t s_rates[kTiledWarps][4][T];
  FieldInfo* fi = a.fields;
  if (fi->status != 0) return;
  const float r = fi->r;
  const uint64_t n = fi->n;
  const uint32_t off = fi->features_off & 7u;
  const bool indep = (off & kOffCross) != 0;
  const bool lz2_on = !(off & kOffLz2), cen_on = !(off & kOffCenter);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint64_t hdr_base = 64;
  // the record's pointers once: the byte stores below may alias anything
  const float* const in = fi->in;
  uint8_t* const out = fi->out;
  for (uint64_t t = uint64_t(blockIdx.x) * kTiledWarps + warp; t < p.ntiles;
       t += uint64_t(gridDim.x) * kTiledWarps) {
    float d[E];
    uint32_t q[E], l[E];
    load_tile<B, T, E>(in, n, t, r, lane, d, q);
    const uint32_t mu = cen_on ? tile_mu<B, T, E>(d, r, lane, s_tile[warp]) : 0u;
    uint32_t C[4] = {0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu};
    if (!indep) {
      // With the state carried across blocks, centring changes the tile's first residual
      // of LZ1 and the first two of LZ2 only (Eq. 4): both variants' residuals once, and
      // block 0's centred rates from the rest of the block and the changed residuals.
      uint32_t p1[E], l2[E];
      predecessors<B, E>(q, false, lane, p1);
#pragma unroll
      for (int k = 0; k < E; ++k) l[k] = q[k] - p1[k];
      predecessors<B, E>(l, false, lane, p1);
#pragma unroll
      for (int k = 0; k < E; ++k) l2[k] = l[k] - p1[k];
      uint32_t c1 = 0, c2 = 0, r10 = 0, r20 = 0;
#pragma unroll
      for (int b = 0; b < T; ++b) {
        const uint32_t ra = block_rate<B, E>(l, b), rb = block_rate<B, E>(l2, b);
        if (lane == 0) {
          s_rates[warp][0][b] = s_rates[warp][2][b] = uint8_t(ra);
          s_rates[warp][1][b] = s_rates[warp][3][b] = uint8_t(rb);
        }
        if (b == 0) {
          r10 = ra;
          r20 = rb;
        }
        c1 += cfg_block_cost(ra, B);
        c2 += cfg_block_cost(rb, B);
      }
      C[0] = c1;
      if (lz2_on) C[1] = c2;
      if (cen_on) {
        uint32_t m1 = lane == 0 ? 0u : uabs32(int32_t(l[0]));
        uint32_t m2 = lane <= 1 ? 0u : uabs32(int32_t(l2[0]));
        if (B == 64) {
          m1 |= uabs32(int32_t(l[B == 64 ? 1 : 0]));
          m2 |= uabs32(int32_t(l2[B == 64 ? 1 : 0]));
        }
        m1 = __reduce_or_sync(FULL, m1);
        m2 = __reduce_or_sync(FULL, m2);
        const uint32_t q0 = __shfl_sync(FULL, q[0], 0);
        const uint32_t l21 = __shfl_sync(FULL, l2[0], 1);
        const uint32_t c0 = uabs32(int32_t(q0 - mu));  // centred l1_0 = l2_0 = q_0 - mu
        const uint32_t r1c = 32u - uint32_t(__clz(int(m1 | c0)));
        const uint32_t r2c = 32u - uint32_t(__clz(int(m2 | c0 | uabs32(int32_t(l21 + mu)))));
        C[2] = 4u + c1 - cfg_block_cost(r10, B) + cfg_block_cost(r1c, B);
        if (lz2_on) C[3] = 4u + c2 - cfg_block_cost(r20, B) + cfg_block_cost(r2c, B);
        if (lane == 0) {
          s_rates[warp][2][0] = uint8_t(r1c);
          s_rates[warp][3][0] = uint8_t(r2c);
        }
      }
    } else {
      // Without it every block restarts, so centring changes every block: each variant's
      // residuals in turn.
      uint32_t qh[E];
#pragma unroll 1
      for (int v = 0; v < 4; ++v) {
        const bool centred = v >= 2, second = (v & 1) != 0;
        if ((second && !lz2_on) || (centred && !cen_on)) continue;
#pragma unroll
        for (int k = 0; k < E; ++k) qh[k] = centred ? q[k] - mu : q[k];
        tile_residuals<B, E>(qh, second, true, lane, l);
        uint32_t cost = centred ? 4u : 0u;
#pragma unroll
        for (int b = 0; b < T; ++b) {
          const uint32_t rate = block_rate<B, E>(l, b);
          if (lane == 0) s_rates[warp][v][b] = uint8_t(rate);
          cost += cfg_block_cost(rate, B);
        }
        C[v] = cost;
      }
    }
    int vs = 0;  // first strict minimum in the listed order (Sec. 4.2.2)
#pragma unroll
    for (int v = 1; v < 4; ++v)
      if (C[v] < C[vs]) vs = v;
    __syncwarp();
    if (lane < T) {
      uint32_t hb = s_rates[warp][vs][lane];
      if (lane == 0) hb |= ((vs & 1) ? 0x80u : 0u) | (vs >= 2 ? 0x40u : 0u);
      out[hdr_base + uint64_t(T) * t + lane] = uint8_t(hb);
    }
    if (lane == 0) {
      p.sizes[t] = C[vs];
      p.rec[t] = uint64_t(vs) | (uint64_t(mu) << 32);
    }
    __syncwarp();
  }
}

// Exclusive scan of the tile sizes: CTA sums, their prefix (one CTA), then each CTA's
// tiles. part[nparts] holds the total.
__device__ __forceinline__ uint64_t block_exclusive_scan(uint64_t v, uint64_t* s_warp, uint64_t* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint64_t inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint64_t y = __shfl_up_sync(FULL, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) s_warp[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    uint64_t w = lane < int(blockDim.x / 32) ? s_warp[lane] : 0;
    uint64_t wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint64_t y = __shfl_up_sync(FULL, wi, o);
      if (lane >= o) wi += y;
    }
    s_warp[lane] = wi - w;
    if (lane == 31) s_warp[32] = wi;
  }
  __syncthreads();
  const uint64_t r = inc - v + s_warp[warp];
  *total = s_warp[32];
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(kScanThreads) fsz_tiled_scan_sums(TiledPtrs p) {
  __shared__ uint64_t s_warp[33];
  uint64_t sum = 0;
  const uint64_t base = uint64_t(blockIdx.x) * kScanItems;
  for (int k = threadIdx.x; k < kScanItems; k += kScanThreads)
    if (base + k < p.ntiles) sum += p.sizes[base + k];
  uint64_t total;
  block_exclusive_scan(sum, s_warp, &total);
  if (threadIdx.x == 0) p.part[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScanThreads) fsz_tiled_scan_parts(TiledPtrs p, uint32_t nparts) {
  __shared__ uint64_t s_warp[33];
  uint64_t carry = 0;
  for (uint32_t base = 0; base < nparts; base += kScanThreads) {
    const uint32_t i = base + threadIdx.x;
    const uint64_t v = i < nparts ? p.part[i] : 0;
    uint64_t total;
    const uint64_t ex = block_exclusive_scan(v, s_warp, &total);
    if (i < nparts) p.part[i] = carry + ex;
    carry += total;
  }
  if (threadIdx.x == 0) p.part[nparts] = carry;
}

__global__ void __launch_bounds__(kScanThreads) fsz_tiled_scan_apply(TiledPtrs p) {
  __shared__ uint64_t s_warp[33];
  const uint64_t base = uint64_t(blockIdx.x) * kScanItems;
  uint64_t carry = p.part[blockIdx.x];
  for (int k0 = 0; k0 < kScanItems; k0 += kScanThreads) {
    const uint64_t i = base + k0 + threadIdx.x;
    const uint64_t v = i < p.ntiles ? p.sizes[i] : 0;
    uint64_t total;
    const uint64_t ex = block_exclusive_scan(v, s_warp, &total);
    if (i < p.ntiles) p.offs[i] = carry + ex;
    carry += total;
  }
}

template <int B, int T>
__global__ void __launch_bounds__(kTiledThreads) fsz_tiled_encode_kernel(KernelArgs a, TiledPtrs p,
                                                                         uint32_t nparts) {
  constexpr int E = B * T / 32;
  FieldInfo* fi = a.fields;
  if (fi->status != 0) return;
  const uint64_t data_bytes = p.part[nparts];
  const uint64_t data_base = 64 + uint64_t(T) * p.ntiles;
  if (data_base + data_bytes > fi->cap) {  // the stream does not fit: nothing is written
    if (blockIdx.x == 0 && threadIdx.x == 0) set_error(a.ctrl, fi, FSZ_ERR_CAPACITY);
    return;
  }
  const float r = fi->r;
  const uint64_t n = fi->n;
  const bool indep = (fi->features_off & kOffCross) != 0;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const Xpose xc = xpose_consts(lane);
  const float* const in = fi->in;
  uint8_t* const out = fi->out;
  for (uint64_t t = uint64_t(blockIdx.x) * kTiledWarps + warp; t < p.ntiles;
       t += uint64_t(gridDim.x) * kTiledWarps) {
    float d[E];
    uint32_t q[E], l[E];
    load_tile<B, T, E>(in, n, t, r, lane, d, q);
    const uint64_t rec = p.rec[t];
    const int vs = int(rec & 3u);
    const uint32_t mu = uint32_t(rec >> 32);
    const bool centred = vs >= 2, second = (vs & 1) != 0;
    if (centred) {
#pragma unroll
      for (int k = 0; k < E; ++k) q[k] -= mu;
    }
    tile_residuals<B, E>(q, second, indep, lane, l);
    uint32_t vv[E];  // sign-magnitude: bit 0 the sign, bit k + 1 magnitude plane k
#pragma unroll
    for (int k = 0; k < E; ++k) vv[k] = (uabs32(int32_t(l[k])) << 1) | (l[k] >> 31);
    uint8_t* dst = out + data_base + p.offs[t];
    const uint8_t* hdr = out + 64 + uint64_t(T) * t;
    uint32_t pos = 0;
    if (centred) {
      if (lane == 0) *reinterpret_cast<float*>(dst) = __int2float_rn(int32_t(mu));
      pos = 4;
    }
#pragma unroll
    for (int b = 0; b < T; ++b) {
      const uint32_t rate = hdr[b] & 0x1Fu;
      if (rate == 0) continue;
      // words 0..rate: word w holds bit w of every element's sign-magnitude value; after
      // the transpose lane L holds word 31 - L (B = 64: both 32-element halves)
      const uint32_t w = 31u - uint32_t(lane);
      const uint32_t hi = warp_transpose32(vv[b * (B / 32)], xc);
      uint32_t lo = 0;
      if (B == 64) lo = warp_transpose32(vv[b * (B / 32) + (B == 64 ? 1 : 0)], xc);
      if (w <= rate) {
        uint32_t* o = reinterpret_cast<uint32_t*>(dst + pos + uint32_t(B / 8) * w);
        o[0] = bswap32(hi);
        if (B == 64) o[1] = bswap32(lo);
      }
      pos += uint32_t(B / 8) * (rate + 1);
    }
    __syncwarp();
  }
}

__global__ void fsz_tiled_preamble_kernel(KernelArgs a, TiledPtrs p, uint32_t nparts, int T) {
  FieldInfo* fi = a.fields;
  if (threadIdx.x != 0 || fi->status != 0) return;
  const uint64_t data_bytes = p.part[nparts];
  const uint64_t total = 64 + uint64_t(T) * p.ntiles + data_bytes;
  if (total > fi->cap) return;
  uint32_t w[16];
  w[0] = 0x315A5346u;  // "FSZ1"
  w[1] = 1u | (fi->ndim << 16) | (fi->mode << 24);
  w[2] = uint32_t(fi->n);
  w[3] = uint32_t(fi->n >> 32);
  for (int k = 0; k < 3; ++k) {
    const uint64_t dk = uint32_t(k) < fi->ndim ? fi->dims[k] : 0;
    w[4 + 2 * k] = uint32_t(dk);
    w[5 + 2 * k] = uint32_t(dk >> 32);
  }
  const uint64_t eb = static_cast<uint64_t>(__double_as_longlong(fi->eb_req));
  w[10] = uint32_t(eb);
  w[11] = uint32_t(eb >> 32);
  w[12] = __float_as_uint(fi->s);
  w[13] = fi->features_off;  // switched-off features and the tile configuration
  w[14] = uint32_t(data_bytes);
  w[15] = uint32_t(data_bytes >> 32);
  uint4* dst = reinterpret_cast<uint4*>(fi->out);
  for (int k = 0; k < 4; ++k) dst[k] = make_uint4(w[4 * k], w[4 * k + 1], w[4 * k + 2], w[4 * k + 3]);
  fi->data_bytes = data_bytes;
  if (fi->out_bytes) *fi->out_bytes = total;
}

// ------------------------------------------------------------------ decompression

// Reads and checks a configured stream's preamble (the rules of plan_dfield plus the
// configuration) into the field record.
__global__ void fsz_tiled_setup_decompress(KernelArgs a, const uint8_t* in, uint64_t in_bytes,
                                           float* out, uint64_t cap_elems, uint64_t max_tiles) {
  if (threadIdx.x != 0) return;
  FieldInfo* fi = a.fields;
  fi->sin = in;
  fi->in_bytes = in_bytes;
  fi->dout = out;
  fi->nchunks = 0;
  uint32_t st = FSZ_OK;
  int B = 32, T = 8;
  if (in_bytes < 64) st = FSZ_ERR_CORRUPT;
  uint32_t w[16] = {0};
  if (st == FSZ_OK) {
    const uint4* pw = reinterpret_cast<const uint4*>(in);
    for (int k = 0; k < 4; ++k) {
      const uint4 v = pw[k];
      w[4 * k] = v.x; w[4 * k + 1] = v.y; w[4 * k + 2] = v.z; w[4 * k + 3] = v.w;
    }
    if (w[0] != 0x315A5346u || (w[1] & 0xFFFFu) != 1u) st = FSZ_ERR_CORRUPT;
  }
  const uint32_t ndim = (w[1] >> 16) & 0xFFu, mode = w[1] >> 24;
  if (st == FSZ_OK && (ndim < 1 || ndim > 3 || mode > 1)) st = FSZ_ERR_CORRUPT;
  const uint64_t n = uint64_t(w[2]) | (uint64_t(w[3]) << 32);
  uint64_t prod = 1;
  for (uint32_t k = 0; st == FSZ_OK && k < 3; ++k) {
    const uint64_t dk = uint64_t(w[4 + 2 * k]) | (uint64_t(w[5 + 2 * k]) << 32);
    if (k >= ndim) {
      if (dk != 0) st = FSZ_ERR_CORRUPT;
      continue;
    }
    if (dk != 0 && prod > kMaxElems / dk) st = FSZ_ERR_CORRUPT;
    prod *= dk;
  }
  if (st == FSZ_OK && (prod != n || n > kMaxElems)) st = FSZ_ERR_CORRUPT;
  const double eb = __longlong_as_double(static_cast<long long>(uint64_t(w[10]) | (uint64_t(w[11]) << 32)));
  const float sv = __uint_as_float(w[12]);
  if (st == FSZ_OK && (!(eb > 0.0) || isinf(eb) || !(sv >= 1.5777218104420236e-30f) || isinf(sv)))
    st = FSZ_ERR_CORRUPT;
  if (st == FSZ_OK && (!config_of(w[13], &B, &T) || !features_valid(w[13] & 7u))) st = FSZ_ERR_CORRUPT;
  const uint64_t db = uint64_t(w[14]) | (uint64_t(w[15]) << 32);
  const uint64_t NT = (n + uint64_t(B * T) - 1) / uint64_t(B * T);
  if (st == FSZ_OK && ((in_bytes - 64) / uint64_t(T) < NT || db > in_bytes - 64 - uint64_t(T) * NT))
    st = FSZ_ERR_CORRUPT;
  if (st == FSZ_OK && n > cap_elems) st = FSZ_ERR_CAPACITY;
  if (st == FSZ_OK && NT > max_tiles) st = FSZ_ERR_WORKSPACE;
  fi->n = st == FSZ_OK ? n : 0;
  fi->T = st == FSZ_OK ? NT : 0;
  fi->s = sv;
  fi->data_bytes = db;
  fi->features_off = w[13];
  if (st != FSZ_OK) set_error(a.ctrl, fi, st);
}

// Tile sizes from the rate headers (any configuration: B and T from the method word);
// zero for the slots past the stream's tiles, which the scan also covers.
__global__ void __launch_bounds__(kTiledThreads) fsz_tiled_sizes_kernel(KernelArgs a, TiledPtrs p) {
  FieldInfo* fi = a.fields;
  const bool ok = fi->status == 0;
  int B = 32, T = 8;
  config_of(fi->features_off, &B, &T);
  const uint32_t foff = fi->features_off & 7u;
  const uint64_t NT = ok ? fi->T : 0;
  for (uint64_t t = uint64_t(blockIdx.x) * kTiledThreads + threadIdx.x; t < p.ntiles;
       t += uint64_t(gridDim.x) * kTiledThreads) {
    if (t >= NT) {
      p.sizes[t] = 0;
      continue;
    }
    const uint8_t* h = fi->sin + 64 + uint64_t(T) * t;
    uint32_t bytes = (h[0] & 0x40u) ? 4u : 0u;
    bool bad = (h[0] & 0x20u) || ((h[0] & 0x80u) && (foff & kOffLz2)) ||
               ((h[0] & 0x40u) && (foff & kOffCenter));
    for (int b = 0; b < T; ++b) {
      if (b > 0 && (h[b] & 0xE0u)) bad = true;
      bytes += cfg_block_cost(h[b] & 0x1Fu, B);
    }
    if (bad) set_error(a.ctrl, fi, FSZ_ERR_CORRUPT);
    p.sizes[t] = bytes;
  }
}

template <int B, int T>
__global__ void __launch_bounds__(kTiledThreads) fsz_tiled_decode_kernel(KernelArgs a, TiledPtrs p,
                                                                         uint32_t nparts) {
  constexpr int E = B * T / 32;
  static_assert(E % 4 == 0, "each lane's run is whole 128-bit words");
  __shared__ __align__(16) uint32_t s_tile[kTiledWarps][E <= 16 ? kRowWords * E : 4];
  FieldInfo* fi = a.fields;
  int cb = 0, ct = 0;
  if (!config_of(fi->features_off, &cb, &ct) || cb != B || ct != T) return;  // another instance's
  if (fi->status != 0) return;
  if (p.part[nparts] != fi->data_bytes) {
    if (blockIdx.x == 0 && threadIdx.x == 0) set_error(a.ctrl, fi, FSZ_ERR_CORRUPT);
    return;
  }
  const float s = fi->s;
  const uint64_t n = fi->n;
  const bool indep = (fi->features_off & kOffCross) != 0;
  const uint64_t NT = fi->T;
  const uint64_t data_base = 64 + uint64_t(T) * NT;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const Xpose xc = xpose_consts(lane);
  const uint8_t* const sin = fi->sin;
  float* const dout = fi->dout;
  for (uint64_t t = uint64_t(blockIdx.x) * kTiledWarps + warp; t < NT;
       t += uint64_t(gridDim.x) * kTiledWarps) {
    const uint8_t* h = sin + 64 + uint64_t(T) * t;
    const uint8_t* src = sin + data_base + p.offs[t];
    const bool second = (h[0] & 0x80u) != 0, centred = (h[0] & 0x40u) != 0;
    uint32_t mu = 0;
    bool good = true;
    uint32_t pos = 0;
    if (centred) {
      const float muf = *reinterpret_cast<const float*>(src);
      const int m = __float2int_rn(muf);
      if (!(fabsf(muf) <= 16777216.0f) || __int2float_rn(m) != muf) good = false;
      mu = uint32_t(m);
      pos = 4;
    }
    uint32_t x[E];
#pragma unroll
    for (int k = 0; k < E; ++k) x[k] = 0;
#pragma unroll
    for (int b = 0; b < T; ++b) {
      const uint32_t rate = h[b] & 0x1Fu;
      if (rate == 0) continue;
      // lane L loads word 31 - L (zero past the block's rate + 1 words); the transpose
      // leaves this lane's element's sign-magnitude value, bit w from word w
      const uint32_t w = 31u - uint32_t(lane);
      uint32_t g0 = 0, g1 = 0;
      if (w <= rate) {
        const uint32_t* wp = reinterpret_cast<const uint32_t*>(src + pos + uint32_t(B / 8) * w);
        g0 = bswap32(wp[0]);
        if (B == 64) g1 = bswap32(wp[B == 64 ? 1 : 0]);
      }
      const uint32_t v0 = warp_transpose32(g0, xc);
      uint32_t v1 = 0;
      if (B == 64) v1 = warp_transpose32(g1, xc);
      const uint32_t m0 = v0 >> 1, m1 = v1 >> 1;
      x[b * (B / 32)] = (v0 & 1u) ? 0u - m0 : m0;
      if (B == 64) x[b * (B / 32) + (B == 64 ? 1 : 0)] = (v1 & 1u) ? 0u - m1 : m1;
      pos += uint32_t(B / 8) * (rate + 1);
    }
    // inverse prediction: inclusive prefix sums in element order (once for LZ1, twice for
    // LZ2), restarting at every block without the cross-block state.
    if constexpr (E <= 16) {
      // Through the warp's buffer each lane takes E consecutive elements: a sum runs along
      // the lane, then one scan of the lanes' totals (over the 32 / T lanes of a block
      // when blocks restart) gives each lane its offset; mu comes in with the last offset.
      uint32_t* const tb = s_tile[warp];
#pragma unroll
      for (int k = 0; k < E; ++k) tb[kRowWords * k + lane] = x[k];
      __syncwarp();
      uint32_t v[E];
#pragma unroll
      for (int u = 0; u < E / 4; ++u) {
        const uint4 w4 = *reinterpret_cast<const uint4*>(tb + padded(E * lane + 4 * u));
        v[4 * u] = w4.x; v[4 * u + 1] = w4.y; v[4 * u + 2] = w4.z; v[4 * u + 3] = w4.w;
      }
      __syncwarp();  // the buffer is the next tile's
      auto prefix = [&](const uint32_t add) {
#pragma unroll
        for (int i = 1; i < E; ++i) v[i] += v[i - 1];
        const uint32_t tot = v[E - 1];
        uint32_t inc = tot;
        if (indep) {
#pragma unroll
          for (int o = 1; o < 32 / T; o <<= 1) inc = scan_step_up<32 / T>(inc, o);
        } else {
#pragma unroll
          for (int o = 1; o < 32; o <<= 1) inc = scan_step_up(inc, o);
        }
        const uint32_t ex = inc - tot + add;
#pragma unroll
        for (int i = 0; i < E; ++i) v[i] += ex;
      };
      if (second) prefix(0u);
      prefix(mu);
      float o[E];
#pragma unroll
      for (int i = 0; i < E; ++i) o[i] = __fmul_rn(__int2float_rn(int32_t(v[i])), s);
      const uint64_t e0 = t * uint64_t(B * T) + uint64_t(E) * uint64_t(lane);
      if (t * uint64_t(B * T) + uint64_t(B * T) <= n) {  // a whole tile: 128-bit stores
#pragma unroll
        for (int u = 0; u < E / 4; ++u)
          reinterpret_cast<float4*>(dout + e0)[u] = make_float4(o[4 * u], o[4 * u + 1], o[4 * u + 2], o[4 * u + 3]);
      } else {
#pragma unroll
        for (int i = 0; i < E; ++i)
          if (e0 + uint64_t(i) < n) dout[e0 + i] = o[i];
      }
    } else {
      // 32 elements per lane would make a 31-step chain per sum: a warp scan per register
      // instead, the running total carried from one register to the next.
#pragma unroll 1
      for (int pass = 0; pass < (second ? 2 : 1); ++pass) {
        uint32_t carry = 0;
#pragma unroll
        for (int k = 0; k < E; ++k) {
          if (indep && ((32 * k) % B) == 0) carry = 0;
          uint32_t inc = x[k];
#pragma unroll
          for (int o = 1; o < 32; o <<= 1) inc = scan_step_up(inc, o);
          x[k] = inc + carry;
          carry = __shfl_sync(FULL, x[k], 31);
        }
      }
#pragma unroll
      for (int k = 0; k < E; ++k) {
        const uint64_t i = t * uint64_t(B * T) + uint64_t(32 * k + lane);
        if (i < n) dout[i] = __fmul_rn(__int2float_rn(int32_t(x[k] + mu)), s);
      }
    }
    if (!__all_sync(FULL, good) && lane == 0) set_error(a.ctrl, fi, FSZ_ERR_CORRUPT);
  }
}

int tiled_grid() {
  static DeviceCfgCache cache;  // per device
  return cache.get([] {
    LaunchCfg c;
    c.grid = [&] {
      int dev = 0, sms = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      return sms * 8;
    }();
    return c;
  }).grid;
}

template <int B, int T>
void launch_tiled_compress(const KernelArgs& a, const TiledPtrs& p, uint32_t nparts, cudaStream_t s) {
  const int g = int(std::min<uint64_t>(uint64_t(tiled_grid()), (p.ntiles + kTiledWarps - 1) / kTiledWarps));
  fsz_tiled_cost_kernel<B, T><<<g, kTiledThreads, 0, s>>>(a, p);
  fsz_tiled_scan_sums<<<nparts, kScanThreads, 0, s>>>(p);
  fsz_tiled_scan_parts<<<1, kScanThreads, 0, s>>>(p, nparts);
  fsz_tiled_scan_apply<<<nparts, kScanThreads, 0, s>>>(p);
  fsz_tiled_encode_kernel<B, T><<<g, kTiledThreads, 0, s>>>(a, p, nparts);
  fsz_tiled_preamble_kernel<<<1, 32, 0, s>>>(a, p, nparts, T);
}

}  // namespace

}  // namespace fsz

using namespace fsz;

extern "C" {

uint64_t fsz_compress_bound_tiled(uint64_t n, uint32_t block, uint32_t tile_blocks) {
  const uint64_t tile = uint64_t(block) * tile_blocks;
  if ((block != 32 && block != 64) || (tile_blocks != 4 && tile_blocks != 8 && tile_blocks != 16))
    return 0;
  const uint64_t NT = (n + tile - 1) / tile;
  return 64 + uint64_t(tile_blocks) * NT + (uint64_t(tile_blocks) * (block / 8) * 24 + 4) * NT;
}

uint64_t fsz_tiled_workspace_bytes(uint64_t n) { return tiled_layout(n).bytes; }

fsz_status fsz_compress_tiled(const float* d_in, fsz_dims dims, fsz_eb_mode mode, double eb,
                              uint32_t block, uint32_t tile_blocks, uint32_t features_off,
                              void* d_out, uint64_t out_capacity, uint64_t* d_out_bytes, void* d_ws,
                              uint64_t ws_bytes, fsz_stream stream) {
  const int B = int(block), T = int(tile_blocks);
  if ((B != 32 && B != 64) || (T != 4 && T != 8 && T != 16)) return FSZ_ERR_INVALID_ARG;
  if (!features_valid(features_off)) return FSZ_ERR_INVALID_ARG;
  uint64_t n = 1;
  if (dims.ndim < 1 || dims.ndim > 3 || dims.reserved != 0) return FSZ_ERR_INVALID_ARG;
  for (uint32_t k = 0; k < dims.ndim; ++k) {
    if (dims.dims[k] != 0 && n > kMaxElems / dims.dims[k]) return FSZ_ERR_INVALID_ARG;
    n *= dims.dims[k];
  }
  if (n == 0) return FSZ_ERR_INVALID_ARG;
  const TiledLayout lay = tiled_layout(n);
  if (d_ws == nullptr || ws_bytes < lay.bytes) return FSZ_ERR_WORKSPACE;
  const uint64_t NT = (n + uint64_t(B * T) - 1) / uint64_t(B * T);
  if (out_capacity < 64 + uint64_t(T) * NT) return FSZ_ERR_CAPACITY;
  // value-range pass and step (the field record gets the method word)
  fsz_status st = fsz_compress_prepare(d_in, dims, mode, eb, d_out, out_capacity, d_out_bytes, d_ws,
                                       lay.L.bytes, stream);
  if (st != FSZ_OK) return st;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  uint8_t* ws = static_cast<uint8_t*>(d_ws);
  KernelArgs a;
  a.ctrl = reinterpret_cast<Ctrl*>(ws);
  a.fields = reinterpret_cast<FieldInfo*>(ws + lay.L.fields_off);
  a.chunk_field = reinterpret_cast<const uint32_t*>(ws + lay.L.map_off);
  a.flags = reinterpret_cast<uint64_t*>(ws + lay.L.flags_off);
  a.skip_chunk = ~uint64_t(0);
  a.timeout_ns = kDefaultTimeoutNs;
  const uint32_t word = features_off | tile_word_of(B, T);
  if (cudaMemcpyAsync(&a.fields->features_off, &word, 4, cudaMemcpyHostToDevice, s) != cudaSuccess)
    return FSZ_ERR_CUDA;
  const TiledPtrs p = tiled_ptrs(d_ws, lay, NT);
  const uint32_t nparts = uint32_t((NT + kScanItems - 1) / kScanItems);
  if (B == 32 && T == 4) launch_tiled_compress<32, 4>(a, p, nparts, s);
  else if (B == 32 && T == 8) launch_tiled_compress<32, 8>(a, p, nparts, s);
  else if (B == 32 && T == 16) launch_tiled_compress<32, 16>(a, p, nparts, s);
  else if (B == 64 && T == 4) launch_tiled_compress<64, 4>(a, p, nparts, s);
  else if (B == 64 && T == 8) launch_tiled_compress<64, 8>(a, p, nparts, s);
  else launch_tiled_compress<64, 16>(a, p, nparts, s);
  return cudaGetLastError() == cudaSuccess ? FSZ_OK : FSZ_ERR_CUDA;
}

fsz_status fsz_decompress_tiled(const void* d_in, uint64_t in_bytes, float* d_out,
                                uint64_t out_capacity_elems, void* d_ws, uint64_t ws_bytes,
                                fsz_stream stream) {
  if (d_in == nullptr || d_out == nullptr || d_ws == nullptr) return FSZ_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(d_in) | reinterpret_cast<uintptr_t>(d_out) |
       reinterpret_cast<uintptr_t>(d_ws)) & 15)
    return FSZ_ERR_ALIGN;
  if (out_capacity_elems > kMaxElems) out_capacity_elems = kMaxElems;
  const TiledLayout lay = tiled_layout(out_capacity_elems);
  if (ws_bytes < lay.bytes) return FSZ_ERR_WORKSPACE;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (cudaMemsetAsync(d_ws, 0, lay.L.bytes, s) != cudaSuccess) return FSZ_ERR_CUDA;
  uint8_t* ws = static_cast<uint8_t*>(d_ws);
  KernelArgs a;
  a.ctrl = reinterpret_cast<Ctrl*>(ws);
  a.fields = reinterpret_cast<FieldInfo*>(ws + lay.L.fields_off);
  a.chunk_field = reinterpret_cast<const uint32_t*>(ws + lay.L.map_off);
  a.flags = reinterpret_cast<uint64_t*>(ws + lay.L.flags_off);
  a.skip_chunk = ~uint64_t(0);
  a.timeout_ns = kDefaultTimeoutNs;
  fsz_tiled_setup_decompress<<<1, 32, 0, s>>>(a, static_cast<const uint8_t*>(d_in), in_bytes, d_out,
                                              out_capacity_elems, lay.max_tiles);
  // the tile count is on the device: the sizes, the scan and the decoders cover the most
  // tiles this output can hold and stop at the stream's own count
  const TiledPtrs p = tiled_ptrs(d_ws, lay, lay.max_tiles);
  const uint32_t nparts = uint32_t((lay.max_tiles + kScanItems - 1) / kScanItems);
  const int g = tiled_grid();
  fsz_tiled_sizes_kernel<<<g, kTiledThreads, 0, s>>>(a, p);
  fsz_tiled_scan_sums<<<nparts, kScanThreads, 0, s>>>(p);
  fsz_tiled_scan_parts<<<1, kScanThreads, 0, s>>>(p, nparts);
  fsz_tiled_scan_apply<<<nparts, kScanThreads, 0, s>>>(p);
  fsz_tiled_decode_kernel<32, 4><<<g, kTiledThreads, 0, s>>>(a, p, nparts);
  fsz_tiled_decode_kernel<32, 8><<<g, kTiledThreads, 0, s>>>(a, p, nparts);
  fsz_tiled_decode_kernel<32, 16><<<g, kTiledThreads, 0, s>>>(a, p, nparts);
  fsz_tiled_decode_kernel<64, 4><<<g, kTiledThreads, 0, s>>>(a, p, nparts);
  fsz_tiled_decode_kernel<64, 8><<<g, kTiledThreads, 0, s>>>(a, p, nparts);
  fsz_tiled_decode_kernel<64, 16><<<g, kTiledThreads, 0, s>>>(a, p, nparts);
  return cudaGetLastError() == cudaSuccess ? FSZ_OK : FSZ_ERR_CUDA;
}

}  // extern "C"
