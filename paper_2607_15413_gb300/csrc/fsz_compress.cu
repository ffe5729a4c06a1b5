// FSZ single-pass compression kernel (Sec. 3.1 steps 1-5, Sec. 4).
//
// Persistent, warp-specialised CTAs (no CTA-wide barrier in the main loop; the roles
// hand work to one another through mbarriers):
//   producer warp  takes a ticket per chunk of kCChunkTiles tiles and stages the chunk
//                  in shared memory, one half of kStageTiles tiles per 1-D TMA bulk copy;
//   compute warps  (8) quantize, predict, evaluate the four variants, select and encode
//                  two tiles at a time (16 elements per lane) from registers into the
//                  warp's own ring buffer in shared memory, and write the tiles' rate
//                  headers (steps 1-3 and 5; each tile is read from HBM once). The last
//                  warp through a chunk scans its tile sizes and publishes the chunk's
//                  aggregate flag;
//   resolver warp  looks back for the chunk's exclusive byte offset (step 4, Sec. 4.4)
//                  and publishes the inclusive prefix;
//   compute warps  copy their tiles of each resolved chunk from the ring to the stream,
//                  whenever one has resolved (between stages and while waiting for input);
//                  they wait for an offset only when their ring is full.
// The ring decouples encoding from the device-wide scan: chunks finish out of ticket order
// across the grid, and a chunk's offset is known only when every earlier chunk has
// published its size, so the encoded bytes wait in shared memory meanwhile (about
// kRingBytes / 250 B tiles per warp at the typical rate, at least one chunk at the worst).
#include "fsz_internal.cuh"

namespace fsz {

namespace {

constexpr int kComputeWarps = 8;
constexpr int kProducerWarp = kComputeWarps;
constexpr int kResolverWarp = kComputeWarps + 1;
constexpr int kThreads = (kComputeWarps + 2) * 32;
constexpr int kStageTiles = 16;                    // tiles per TMA stage (half a chunk)
constexpr int kStageElems = kStageTiles * kTile;
constexpr int kStages = 2;                         // TMA input stages
constexpr int kSets = 8;                           // chunks in flight per CTA
constexpr int kCtasPerSm = 2;                      // 96 registers per thread
constexpr int kRingBytes = 8192;                   // encoded-tile ring per compute warp
constexpr int kLookbackPerLane = 4;                // lookback window: 128 flags
constexpr int kTicketAhead = 2;                    // chunk tickets taken ahead of use
constexpr uint32_t kNone = 0xffffffffu;
static_assert(kCChunkTiles == 2 * kStageTiles, "a chunk is two stages");
static_assert(kCChunkTiles <= 32, "one lane per tile in the chunk scan");
static_assert(kRingBytes >= 3 * 2 * kMaxTileBytes,
              "with only the current chunk's first pair live, a free pair gap exists");
static_assert((kRingBytes & (kRingBytes - 1)) == 0, "ring counters wrap with the ring");
static_assert(kStageTiles == 2 * kComputeWarps, "one pair per warp per stage");
static_assert(kRingBytes <= 65536, "ring offsets are 16-bit");
static_assert(kMaxTileBytes % 4 == 0, "tiles are 32-bit words");

// A chunk's parameters, read once from the field record by the producer and kept in the
// chunk's set until every compute warp has placed the chunk.
constexpr uint32_t kInfoOk = 1u, kInfoLast = 2u, kInfoFirst = 4u, kInfoSkip = 8u;
struct ChunkInfo {
  const float* in;       // the chunk's first element
  uint8_t* out;          // the field's stream
  FieldInfo* fi;
  uint64_t tile0;        // field-local index of the chunk's first tile
  uint64_t data_base;    // 64 + 8T: start of the field's tile data
  uint64_t cap;          // the field's output capacity
  uint64_t chunk_first;  // global index of the field's first chunk
  uint32_t chunk;        // global ticket, or kNone
  uint32_t ntiles;
  uint32_t cnt;          // valid elements in the chunk
  float r;
  uint32_t flags;        // kInfo* bits
  uint32_t off;          // the field's switched-off features (kOff* bits)
};

struct StageInfo {
  uint32_t seq;   // the CTA's chunk sequence number of the staged chunk
  uint32_t half;  // which half of it
};

struct __align__(16) CompressSmem {
  float in[kStages][kStageElems];                 // TMA stages
  uint8_t ring[kComputeWarps][kRingBytes];        // encoded tiles awaiting their offset
  ChunkInfo meta[kSets];
  ChunkInfo pre[kTicketAhead];                    // producer's tickets taken ahead
  uint64_t set_excl[kSets];
  uint32_t toff[kSets][kCChunkTiles];             // tile offsets inside the chunk
  uint32_t ring_mark[kComputeWarps][kSets];       // ring head after the warp's share
  uint32_t set_tot[kSets];
  uint32_t done_cnt[kSets];
  uint32_t tinfo[kSets][kCChunkTiles];            // ring offset << 16 | encoded size
  StageInfo stage[kStages];
  uint64_t full[kStages], empty[kStages], computed[kSets], resolved[kSets], setfree[kSets];
};

// Eq. 3: S_b = 0 for r_b = 0, else 4 + 4 r_b.
__device__ __forceinline__ uint32_t block_cost(int R) { return (uint32_t(R) + (R != 0 ? 1u : 0u)) << 2; }

// v = 2|l| + sign: bit 0 is the sign-map bit, bit k + 1 magnitude bit-plane k (Sec. 4.3).
__device__ __forceinline__ uint32_t sign_mag(int l) { return (uabs32(l) << 1) | (uint32_t(l) >> 31); }

// The sign-magnitude word by multiply-adds: 2|l| + s = l (2 - 4s) + s with s the sign bit.
__device__ __forceinline__ uint32_t sign_mag_fma(int l) {
  const int sg = int(uint32_t(l) >> 31);
  return uint32_t(mad_s32(l, mad_s32(sg, -4, 2), sg));
}

// Loads lane hl = lane & 15's 16 elements (16 hl..16 hl + 15) of its half's tile from
// the stage into registers, in element order.
__device__ __forceinline__ void load_pair(const float* __restrict__ tile, const int lane,
                                          float (&d)[16]) {
  const int hl = lane & 15;
  const float4* t4 = reinterpret_cast<const float4*>(tile) + 4 * hl;
  // Load k of lane hl reads chunk (k + 2 (hl/2 mod 2)) mod 4 of its 64 bytes, so each
  // 128-bit phase of 8 lanes hits every bank group twice rather than two of them four
  // times; one select stage puts the chunks back in order.
  const int rot = (hl >> 1) & 1;
  float4 u[4], q[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) u[k] = t4[(k + 2 * rot) & 3];
#pragma unroll
  for (int c = 0; c < 4; ++c) q[c] = rot ? u[(c + 2) & 3] : u[c];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    d[4 * k] = q[k].x; d[4 * k + 1] = q[k].y; d[4 * k + 2] = q[k].z; d[4 * k + 3] = q[k].w;
  }
}

// Compresses two tiles with one warp: lanes 0-15 take one tile and lanes 16-31 the next
// (half = lane >> 4). Lane hl = lane & 15 holds elements 16 hl..16 hl + 15 of its tile in
// d, so lanes 2g, 2g + 1 of a half own block g (Sec. 3.1: a tile is 8 blocks of 32
// elements). The halves run in lockstep but each takes its own decisions (variant, rates).
// `hdr` is this half's; the first half's bytes go to `slot`, the second half's right after
// them. A half with `live` false computes but stores nothing. Returns this half's byte
// count (uniform within the half). Switched-off features (kOff* bits) arrive as `restart`
// (this lane starts from zero predecessors: the tile's first lane, and without the
// cross-block state every block's first lane) and as penalties pen2, pen3 (2^16 for the
// second-order and the centred variants when off), which raise a switched-off variant's
// cost past any tile's so that it is never selected.
// With kGiven the four tile costs come from `given` (this half's tile, stride gT between
// variants) rather than from the costs computed here: the multipass evaluation's
// encoding pass. They are equal, so the stream is the same.
template <bool kGiven>
__device__ __forceinline__ uint32_t compress_pair(const float (&d)[16],
                                                  uint8_t* __restrict__ slot,
                                                  uint8_t* __restrict__ hdr, const float r,
                                                  const int lane, const bool live,
                                                  const bool restart, const int pen2,
                                                  const int pen3,
                                                  const uint32_t* __restrict__ given,
                                                  const uint64_t gT) {
  constexpr uint32_t FULL = 0xffffffffu;
  const int hl = lane & 15;
  // Step 1, quantize (Sec. 4.2.2): t = fl(d r) then the nearest integer, ties to even.
  // Y holds q + bits(M); differences of Y are differences of q.
  int Y[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) Y[i] = __float_as_int(__fadd_rn(__fmul_rn(d[i], r), kMagic));

  // Tile sum for centring (Sec. 4.2.2, variant 3) in the fixed order: the sums of elements
  // 8j..8j+7 left to right (two per lane: V0 for j even, V1 for j odd), then a butterfly
  // over j by 16, 8, 4, 2 (lanes xor 8, 4, 2, 1 within the half) and finally by 1
  // (V0 + V1). Float addition is commutative, so both partners of a step get equal sums.
  float V0 = d[0], V1 = d[8];
#pragma unroll
  for (int i = 1; i < 8; ++i) {
    V0 = __fadd_rn(V0, d[i]);
    V1 = __fadd_rn(V1, d[8 + i]);
  }
#pragma unroll
  for (int o = 8; o >= 1; o >>= 1) {
    V0 = __fadd_rn(V0, __shfl_xor_sync(FULL, V0, o));
    V1 = __fadd_rn(V1, __shfl_xor_sync(FULL, V1, o));
  }
  const float P = __fadd_rn(V0, V1);
  const int mu =
      __float_as_int(__fadd_rn(__fmul_rn(__fmul_rn(P, 0.00390625f), r), kMagic)) - kMagicBits;

  // LZ1 residuals with the state carried across lane and block boundaries (Eq. 2); the
  // tile's first predecessor is zero. LZ2 as the difference of LZ1 residuals:
  // l2_i = (q_i - q_{i-1}) - (q_{i-1} - q_{i-2}).
  int prevY = __shfl_up_sync(FULL, Y[15], 1, 16);
  if (restart) prevY = kMagicBits;
  int l1[16], l2[16];
  l1[0] = Y[0] - prevY;
#pragma unroll
  for (int i = 1; i < 16; ++i) l1[i] = Y[i] - Y[i - 1];
  int prevL = __shfl_up_sync(FULL, l1[15], 1, 16);
  if (restart) prevL = 0;
  l2[0] = l1[0] - prevL;
#pragma unroll
  for (int i = 1; i < 16; ++i) l2[i] = l1[i] - l1[i - 1];

  // Block maxima as ORs (same bit length); the block's two lanes combine by one shuffle.
  // rest* leave out the tile's first residual(s), the only ones centring changes (Eq. 4).
  uint32_t rest1 = 0, rest2 = 0;
#pragma unroll
  for (int i = 1; i < 16; ++i) rest1 |= uabs32(l1[i]);
#pragma unroll
  for (int i = 2; i < 16; ++i) rest2 |= uabs32(l2[i]);
  const uint32_t o1 = rest1 | uabs32(l1[0]);
  const uint32_t o2 = rest2 | uabs32(l2[0]) | uabs32(l2[1]);
  const uint32_t x1 = __shfl_xor_sync(FULL, o1, 1);
  const uint32_t y1 = __shfl_xor_sync(FULL, o2, 1);
  // Rate r_b = bit length of the block maximum (Sec. 4.1.2).
  const int R1 = 32 - __clz(int(o1 | x1));
  const int R2 = 32 - __clz(int(o2 | y1));

  // Centred block-0 rates (lane hl = 0): l1c_0 = q_0 - mu, l2c_0 = q_0 - mu,
  // l2c_1 = q_1 - 2 q_0 + mu = l2_1 + mu; the rest of block 0 is unchanged (Eq. 4).
  const int q0 = Y[0] - kMagicBits;
  const uint32_t c10 = uabs32(q0 - mu);
  const uint32_t c21 = uabs32(l2[1] + mu);
  const int R1c = 32 - __clz(int(rest1 | x1 | c10));
  const int R2c = 32 - __clz(int(rest2 | y1 | c10 | c21));

  // Block costs S_b (Eq. 3) of LZ1 and LZ2 as 16-bit halves. An inclusive scan over the
  // 8 blocks (lanes 2 apart) gives every block's end offset for both variants; lane 15 of
  // the half holds the tile costs C = sum of S_b. Centring changes block 0 only: its cost
  // deltas and rates come from lane 0; variants 3 and 4 pay 4 bytes for mu (step 2).
  const uint32_t pk = block_cost(R1) | (block_cost(R2) << 16);
  uint32_t pinc = pk;
  pinc = scan_step_up<16>(pinc, 2);
  pinc = scan_step_up<16>(pinc, 4);
  pinc = scan_step_up<16>(pinc, 8);
  const uint32_t ptot = __shfl_sync(FULL, pinc, 15, 16);
  int C1 = int(ptot & 0xffffu), C2 = int(ptot >> 16);
  uint32_t bc = (block_cost(R1c) - block_cost(R1) + 1024u) |
                ((block_cost(R2c) - block_cost(R2) + 1024u) << 11) | (uint32_t(R1c) << 22) |
                (uint32_t(R2c) << 27);
  bc = __shfl_sync(FULL, bc, 0, 16);
  const int dC1 = int(bc & 0x7ffu) - 1024, dC2 = int((bc >> 11) & 0x7ffu) - 1024;
  int C3 = 4 + C1 + dC1 + pen3;
  int C4 = 4 + C2 + dC2 + pen2 + pen3;
  if constexpr (kGiven) {
    C1 = int(given[0]);
    C2 = int(given[gT]);
    C3 = int(given[2 * gT]);
    C4 = int(given[3 * gT]);
  }
  const int R1c0 = int((bc >> 22) & 31u), R2c0 = int(bc >> 27);

  // Step 3: first strict minimum in the order LZ1, LZ2, LZ1c, LZ2c.
  int v = 0, best = C1;
  if (C2 + pen2 < best) { v = 1; best = C2; }
  if (C3 < best) { v = 2; best = C3; }
  if (C4 < best) { v = 3; best = C4; }
  const bool second = (v & 1) != 0, centred = v >= 2;

  const int g = hl >> 1, t2 = hl & 1;
  int Rg = second ? R2 : R1;
  if (g == 0 && centred) Rg = second ? R2c0 : R1c0;
  // Rate header (Sec. 3.1): block 0 carries bit 7 = order 2, bit 6 = centred.
  if (t2 == 0 && live) {
    uint32_t hb = uint32_t(Rg);
    if (g == 0) hb |= (second ? 0x80u : 0u) | (centred ? 0x40u : 0u);
    hdr[g] = uint8_t(hb);
  }

  // Step 5: residuals of the selected variant as sign-magnitude words v = 2|l| + sign,
  // so that bit 0 is the sign map and bit k + 1 is magnitude bit-plane k (Sec. 4.3). The
  // halves may select different variants: select per element rather than branch.
  // The selected residual is l1_i + m l1_{i-1} with m = 0 (LZ1) or -1 (LZ2).
  const int m = second ? -1 : 0;
  uint32_t vv[16];
  vv[0] = sign_mag_fma(mad_s32(prevL, m, l1[0]));
#pragma unroll
  for (int i = 1; i < 16; ++i) vv[i] = sign_mag_fma(mad_s32(l1[i - 1], m, l1[i]));
  const bool fix = centred && hl == 0;
  vv[0] = fix ? sign_mag(q0 - mu) : vv[0];
  vv[1] = (fix && second) ? sign_mag(l2[1] + mu) : vv[1];

  // Byte offset of block g inside the tile's data: the variant's exclusive prefix; when
  // centred, mu's 4 bytes come first and block 0's cost changes by its delta.
  const uint32_t pexc = pinc - pk;
  int off = int(second ? (pexc >> 16) : (pexc & 0xffffu));
  if (centred) off += 4 + (g > 0 ? (second ? dC2 : dC1) : 0);
  const uint32_t size_first = __shfl_sync(FULL, uint32_t(best), 0);
  uint8_t* const my_slot = slot + (lane >= 16 ? size_first : 0u);
  uint8_t* const blk = my_slot + off;
  if (fix && live) *reinterpret_cast<float*>(my_slot) = __int2float_rn(mu);

  const int nwords = live && Rg > 0 ? Rg + 1 : 0;  // block g's words: sign map + Rg planes
  const int Rmax = int(__reduce_max_sync(FULL, live ? uint32_t(Rg) : 0u));
  if (Rmax > 0) {
    const int nch = (Rmax + 8) >> 3;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      if (c < nch) {
        // Byte c of v_7..v_4 into lo, of v_3..v_0 into hi (element order reversed), so the
        // 8x8 transpose leaves plane 8c + b in byte b with element i at bit 7 - i; the
        // same for the lane's elements 8-15.
        const uint32_t sel = uint32_t(c) | (uint32_t(4 + c) << 4);
        uint32_t lo0 = __byte_perm(__byte_perm(vv[7], vv[6], sel), __byte_perm(vv[5], vv[4], sel), 0x5410);
        uint32_t hi0 = __byte_perm(__byte_perm(vv[3], vv[2], sel), __byte_perm(vv[1], vv[0], sel), 0x5410);
        uint32_t lo1 = __byte_perm(__byte_perm(vv[15], vv[14], sel), __byte_perm(vv[13], vv[12], sel), 0x5410);
        uint32_t hi1 = __byte_perm(__byte_perm(vv[11], vv[10], sel), __byte_perm(vv[9], vv[8], sel), 0x5410);
        transpose8x8(lo0, hi0);
        transpose8x8(lo1, hi1);
        // Lane t2 = 0 builds the words of planes 8c..8c+3, lane t2 = 1 those of 8c+4..8c+7;
        // each needs the partner's bytes of those planes.
        const uint32_t r0 = __shfl_xor_sync(FULL, t2 ? lo0 : hi0, 1);
        const uint32_t r1 = __shfl_xor_sync(FULL, t2 ? lo1 : hi1, 1);
        const uint32_t X0 = t2 ? r0 : lo0, X1 = t2 ? r1 : lo1;
        const uint32_t Y0 = t2 ? hi0 : r0, Y1 = t2 ? hi1 : r1;
        // word b = [X0.b, X1.b, Y0.b, Y1.b] in memory order: elements 0-7, 8-15, 16-23,
        // 24-31, each byte with its first element in the top bit (Sec. 4.3)
        const uint32_t u0 = __byte_perm(X0, X1, 0x5140), u1 = __byte_perm(X0, X1, 0x7362);
        const uint32_t u2 = __byte_perm(Y0, Y1, 0x5140), u3 = __byte_perm(Y0, Y1, 0x7362);
        const uint32_t w[4] = {__byte_perm(u0, u2, 0x5410), __byte_perm(u0, u2, 0x7632),
                               __byte_perm(u1, u3, 0x5410), __byte_perm(u1, u3, 0x7632)};
        const int wb = 8 * c + 4 * t2;
#pragma unroll
        for (int b = 0; b < 4; ++b)
          if (wb + b < nwords) reinterpret_cast<uint32_t*>(blk)[wb + b] = w[b];
      }
    }
  }
  return uint32_t(best);
}

// kGiven: the multipass evaluation's encoding pass (selection from a.given_costs).
// kFeat: fields' switched-off features honoured; without it the full method is compiled
// with none of that handling.
template <bool kGiven, bool kFeat>
__global__ void __launch_bounds__(kThreads, kCtasPerSm) fsz_compress_kernel(KernelArgs a) {
  extern __shared__ __align__(128) uint8_t smem_raw[];
  CompressSmem& S = *reinterpret_cast<CompressSmem*>(smem_raw);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint64_t total = a.ctrl->total_chunks;
  // mbarrier waits outlast the longest lookback wait, so a lookback that runs out is
  // reported as such rather than as a stalled pipeline.
  const uint64_t wait_ns = 4 * a.timeout_ns;

  if (tid == 0) {
    for (int k = 0; k < kStages; ++k) {
      mbar_init(&S.full[k], 1);
      mbar_init(&S.empty[k], kComputeWarps);
    }
    for (int k = 0; k < kSets; ++k) {
      mbar_init(&S.computed[k], 1);
      mbar_init(&S.resolved[k], 1);
      mbar_init(&S.setfree[k], kComputeWarps);
      S.done_cnt[k] = 0;
    }
    fence_mbar_init();
  }
  __syncthreads();

  if (warp == kProducerWarp) {
    // ---------------------------------------------------------------- producer
    // Tickets are taken two chunks ahead, so the ticket atomic and the field-record loads
    // overlap the waits; a chunk's record goes to its set once the chunk kSets earlier has
    // been placed by every compute warp, and each half goes out as soon as a stage frees.
    if (lane != 0) return;
    const bool single = a.ctrl->nfields == 1;
    auto fetch = [&](ChunkInfo& ci) {
      const uint32_t c = atomicAdd(&a.ctrl->ticket, 1u);
      ci.chunk = c;
      if (c >= total) return;
      FieldInfo* fi = single ? a.fields : a.fields + a.chunk_field[c];
      const uint64_t first = fi->chunk_first;
      const uint64_t lc = c - first;
      const uint64_t tile0 = lc * kCChunkTiles;
      const uint64_t e0 = tile0 * kTile;
      const uint64_t T = fi->T;
      ci.in = fi->in + e0;
      ci.out = fi->out;
      ci.fi = fi;
      ci.tile0 = tile0;
      ci.data_base = 64 + 8 * T;
      ci.cap = fi->cap;
      ci.chunk_first = first;
      ci.ntiles = uint32_t(min(uint64_t(kCChunkTiles), T - tile0));
      ci.cnt = uint32_t(min(fi->n - e0, uint64_t(kCChunkElems)));
      ci.r = fi->r;
      ci.off = fi->features_off;
      ci.flags = (fi->s > 0.0f ? kInfoOk : 0u) |  // a field without a step has nothing to load
                 (lc + 1 == fi->nchunks ? kInfoLast : 0u) | (lc == 0 ? kInfoFirst : 0u) |
                 (uint64_t(c) == a.skip_chunk ? kInfoSkip : 0u);
    };
    for (int k = 0; k < kTicketAhead; ++k) fetch(S.pre[k]);
    uint32_t u = 0;  // stage uses so far
    auto take_stage = [&](uint32_t seq, uint32_t h) -> int {
      const int s = int(u % kStages);
      if (u >= uint32_t(kStages) && !mbar_wait(&S.empty[s], ((u / kStages) - 1) & 1u, wait_ns)) {
        set_error(a.ctrl, nullptr, FSZ_ERR_TIMEOUT);
        return -1;
      }
      S.stage[s].seq = seq;
      S.stage[s].half = h;
      ++u;
      return s;
    };
    for (uint32_t seq = 0;; ++seq) {
      const int b = int(seq % kSets);
      if (seq >= uint32_t(kSets) && !mbar_wait(&S.setfree[b], ((seq / kSets) - 1) & 1u, wait_ns)) {
        set_error(a.ctrl, nullptr, FSZ_ERR_TIMEOUT);
        return;
      }
      ChunkInfo& q = S.pre[seq % kTicketAhead];
      S.meta[b] = q;
      if (q.chunk >= total) {
        S.meta[b].chunk = kNone;
        const int s = take_stage(seq, 0);
        if (s >= 0) mbar_arrive(&S.full[s]);
        return;
      }
      const uint32_t halves = q.ntiles > uint32_t(kStageTiles) ? 2u : 1u;
      for (uint32_t h = 0; h < halves; ++h) {
        const int s = take_stage(seq, h);
        if (s < 0) return;
        const uint32_t e_h = h * kStageElems;
        const uint32_t valid = min(q.cnt - e_h, uint32_t(kStageElems));
        const uint32_t bulk = (q.flags & kInfoOk) ? ((valid * 4) & ~15u) : 0u;
        fence_proxy_async();
        mbar_arrive_expect_tx(&S.full[s], bulk);
        if (bulk) tma_load_1d(S.in[s], q.in + e_h, bulk, &S.full[s]);
      }
      fetch(q);  // the ticket kTicketAhead chunks ahead
    }
  }

  if (warp == kResolverWarp) {
    // ---------------------------------------------------------------- resolver
    // Step 4 at device level, one chunk after another in this CTA's ticket order, as soon
    // as the chunk's aggregate is out: the compute warps keep encoding meanwhile.
    for (uint32_t seq = 0;; ++seq) {
      const int b = int(seq % kSets);
      if (!mbar_wait(&S.computed[b], (seq / kSets) & 1u, wait_ns)) {
        if (lane == 0) set_error(a.ctrl, nullptr, FSZ_ERR_TIMEOUT);
        return;
      }
      const ChunkInfo& ci = S.meta[b];
      const uint32_t c = ci.chunk;
      if (c == kNone) return;
      const uint32_t flags = ci.flags;
      const uint32_t tot = S.set_tot[b];
      uint64_t excl = 0;
      if (!(flags & kInfoFirst)) {
        bool to = false;
        excl = lookback<kLookbackPerLane>(a.flags, int64_t(c), int64_t(ci.chunk_first),
                                          globaltimer_ns() + a.timeout_ns, &to);
        if (lane == 0) {
          if (to) set_error(a.ctrl, ci.fi, FSZ_ERR_TIMEOUT);
          if (!(flags & kInfoSkip)) st_flag(a.flags + c, kFlagIncl | (excl + tot));
        }
      }
      __syncwarp();
      if (lane == 0) {
        S.set_excl[b] = excl;
        mbar_arrive(&S.resolved[b]);
      }
    }
  }

  // ------------------------------------------------------------------ compute warps
  uint8_t* const ring = S.ring[warp];
  uint32_t head = 0, tail = 0;  // ring byte counters (warp-uniform)
  uint32_t placed = 0;          // this CTA's chunks placed by this warp so far
  uint32_t done = 0;            // ... encoded by this warp so far

  // Copies this warp's tiles of chunk `placed` (resolved) into the stream and frees them.
  auto place = [&]() {
    const int b = int(placed % kSets);
    const ChunkInfo& ci = S.meta[b];
    if ((ci.flags & (kInfoOk | kInfoSkip)) == kInfoOk) {
      const uint64_t excl = S.set_excl[b];
      const uint32_t tot = S.set_tot[b];
      if (ci.data_base + excl + tot > ci.cap) {
        if (lane == 0) set_error(a.ctrl, ci.fi, FSZ_ERR_CAPACITY);
      } else {
        uint8_t* base = ci.out + ci.data_base + excl;
        // the warp's pair of each stage: contiguous in the ring and in the stream
        const int nt = int(ci.ntiles);
        for (int t0 = 2 * warp; t0 < nt; t0 += kStageTiles) {
          const uint32_t ti = S.tinfo[b][t0];
          const uint32_t nw = ((ti & 0xffffu) + (t0 + 1 < nt ? (S.tinfo[b][t0 + 1] & 0xffffu) : 0u)) >> 2;
          const uint32_t* src = reinterpret_cast<const uint32_t*>(ring + (ti >> 16));
          uint32_t* dst = reinterpret_cast<uint32_t*>(base + S.toff[b][t0]);
          for (uint32_t q0 = 0; q0 < nw; q0 += 128) {  // 4 words per lane in flight
            uint32_t v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const uint32_t q = q0 + 32 * u + lane;
              if (q < nw) v[u] = src[q];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const uint32_t q = q0 + 32 * u + lane;
              if (q < nw) dst[q] = v[u];
            }
          }
        }
        if (warp == 0 && lane == 0 && (ci.flags & kInfoLast)) write_preamble(ci.fi, excl + tot);
      }
    }
    tail = S.ring_mark[warp][b];
    ++placed;
    __syncwarp();
    if (lane == 0) mbar_arrive(&S.setfree[b]);
  };
  // Places every chunk that has resolved, without waiting.
  auto place_ready = [&]() {
    while (placed < done && mbar_test(&S.resolved[placed % kSets], (placed / kSets) & 1u)) place();
  };
  // Places the oldest chunk, waiting for its offset.
  auto place_oldest = [&]() -> bool {
    if (!mbar_wait(&S.resolved[placed % kSets], (placed / kSets) & 1u, wait_ns)) return false;
    place();
    return true;
  };

  bool ok_run = true;
  for (uint32_t u = 0;; ++u) {
    const int s = int(u % kStages);
    const uint32_t par = (u / kStages) & 1u;
    // Wait for the stage, placing resolved chunks meanwhile (the producer may be waiting
    // for this warp to free a set). The stage is usually full already: one test, no timer.
    if (!mbar_test(&S.full[s], par)) {
      const uint64_t deadline = globaltimer_ns() + wait_ns;
      bool got = false;
      while (!got) {
        if (placed < done) {
          if (mbar_test(&S.resolved[placed % kSets], (placed / kSets) & 1u)) {
            place();
            continue;
          }
          got = mbar_try_wait_for(&S.full[s], par, 2000u);
        } else {
          got = mbar_try_wait_sleep(&S.full[s], par);
        }
        if (!got && globaltimer_ns() > deadline) break;
      }
      if (!got) {
        if (lane == 0) set_error(a.ctrl, nullptr, FSZ_ERR_TIMEOUT);
        ok_run = false;
        break;
      }
    }
    const uint32_t seq = S.stage[s].seq, h = S.stage[s].half;
    const int b = int(seq % kSets);
    const ChunkInfo& ci = S.meta[b];
    const uint32_t c = ci.chunk;
    const uint32_t flags = ci.flags;
    const int ntiles = int(ci.ntiles);
    const bool end = (c == kNone);
    const bool last_half = end || (h + 1 == (ntiles > kStageTiles ? 2u : 1u));
    bool released = false;
    if (!end && (flags & kInfoOk)) {
      const float r = ci.r;
      const uint32_t e_h = h * kStageElems;
      const uint32_t cnt = min(ci.cnt - e_h, uint32_t(kStageElems));
      const uint32_t bulk_elems = ((cnt * 4) & ~15u) / 4;
      const float* gin = ci.in + e_h;
      uint8_t* hdr_out = ci.out + 64 + 8 * ci.tile0;
      const int t_end = min(ntiles, int(h + 1) * kStageTiles);
      const bool ragged = cnt < uint32_t(kStageElems);
      const int ta = int(h) * kStageTiles + 2 * warp;  // this warp's pair in the stage
      if (ta < t_end) {
        const int half = lane >> 4;
        const bool live = ta + half < t_end;
        const int tl = live ? ta + half : ta;          // a missing second tile repeats the first
        const int ts = tl - int(h) * kStageTiles;
        float* tile = S.in[s] + ts * kTile;
        // ragged end of a field: this lane's 16 elements past the bulk copy by plain loads
        const uint32_t k0 = uint32_t(ts) * kTile + 16u * uint32_t(lane & 15);
        if (ragged && live && k0 + 16 > bulk_elems) {
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            const uint32_t k = k0 + uint32_t(i);
            if (k >= bulk_elems) tile[16 * (lane & 15) + i] = k < cnt ? gin[k] : 0.0f;
          }
        }
        __syncwarp();
        float d[16];
        load_pair(tile, lane, d);
        __syncwarp();
        if (lane == 0) mbar_arrive(&S.empty[s]);  // the pair is in registers
        released = true;
        // room for a worst-case pair, contiguous in the ring
        constexpr uint32_t kPair = 2 * kMaxTileBytes;
        uint32_t pos = head % kRingBytes;
        uint32_t skip = pos + kPair > uint32_t(kRingBytes) ? kRingBytes - pos : 0u;
        while (kRingBytes - (head - tail) < skip + kPair) {
          if (placed == done || !place_oldest()) {  // cannot happen with <= one pair live
            if (lane == 0) set_error(a.ctrl, nullptr, FSZ_ERR_TIMEOUT);
            ok_run = false;
            break;
          }
          pos = head % kRingBytes;
          skip = pos + kPair > uint32_t(kRingBytes) ? kRingBytes - pos : 0u;
        }
        if (!ok_run) break;
        head += skip;
        pos = head % kRingBytes;
        // switched-off features: zero predecessors for every block's first lane without
        // the carried state; cost penalties for switched-off variants
        const uint32_t foff = kFeat ? ci.off : 0u;
        const bool restart = (lane & 15) == 0 || ((foff & kOffCross) && (lane & 1) == 0);
        const int pen2 = (foff & kOffLz2) ? 0x10000 : 0;
        const int pen3 = (foff & kOffCenter) ? 0x10000 : 0;
        const uint32_t nb = compress_pair<kGiven>(d, ring + pos, hdr_out + 8 * tl, r, lane, live,
                                                  restart, pen2, pen3,
                                                  a.given_costs + ci.tile0 + tl, a.given_T);
        const uint32_t na = __shfl_sync(0xffffffffu, nb, 0);
        const uint32_t nbb = __shfl_sync(0xffffffffu, nb, 16);
        const bool second_live = ta + 1 < t_end;
        if (lane == 0) S.tinfo[b][ta] = (pos << 16) | na;
        if (lane == 16 && second_live) S.tinfo[b][ta + 1] = ((pos + na) << 16) | nbb;
        head += na + (second_live ? nbb : 0u);
      }
      if (!ok_run) break;
    }
    __syncwarp();
    if (!end && !released && lane == 0) mbar_arrive(&S.empty[s]);  // done reading the stage
    if (last_half) {
      // This warp is through the chunk: the last warp to get here scans the chunk's tile
      // sizes and publishes its aggregate (step 4, thread and warp levels).
      uint32_t last = 0;
      S.ring_mark[warp][b] = head;  // every lane (the same value): read by every lane
      if (lane == 0) {
        __threadfence_block();
        last = atomicAdd(&S.done_cnt[b], 1u) == uint32_t(kComputeWarps - 1) ? 1u : 0u;
        __threadfence_block();
      }
      last = __shfl_sync(0xffffffffu, last, 0);
      __syncwarp();
      if (last) {
        if (!end) {
          const uint32_t mine = ((flags & kInfoOk) && lane < ntiles) ? (S.tinfo[b][lane] & 0xffffu) : 0u;
          uint32_t inc = mine;
#pragma unroll
          for (int o = 1; o < 32; o <<= 1) {
            const uint32_t x = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += x;
          }
          S.toff[b][lane] = inc - mine;
          const uint32_t tot = __shfl_sync(0xffffffffu, inc, 31);
          if (lane == 0) {
            S.set_tot[b] = tot;
            if (!(flags & kInfoSkip)) st_flag(a.flags + c, ((flags & kInfoFirst) ? kFlagIncl : kFlagAgg) | tot);
          }
        }
        __syncwarp();
        if (lane == 0) {
          S.done_cnt[b] = 0;
          mbar_arrive(&S.computed[b]);
        }
      }
      if (end) break;
      ++done;
    }
    place_ready();
  }
  // Chunks encoded but not yet placed.
  while (ok_run && placed < done) {
    if (!place_oldest()) {
      if (lane == 0) set_error(a.ctrl, nullptr, FSZ_ERR_TIMEOUT);
      break;
    }
  }
}

}  // namespace

LaunchCfg compress_cfg() {
  static LaunchCfg cfg = [] {
    LaunchCfg c;
    c.smem = int(sizeof(CompressSmem));
    cudaFuncSetAttribute(fsz_compress_kernel<false, false>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, c.smem);
    cudaFuncSetAttribute(fsz_compress_kernel<false, true>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, c.smem);
    cudaFuncSetAttribute(fsz_compress_kernel<true, false>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, c.smem);
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fsz_compress_kernel<false, false>, kThreads,
                                                  c.smem);
    c.sms = sms;
    c.per = per > 0 ? per : 1;
    c.grid = sms * c.per;
    return c;
  }();
  return cfg;
}

void launch_compress(const KernelArgs& a, cudaStream_t st, CompressKind kind) {
  const LaunchCfg c = compress_cfg();
  const int g = sched_grid(c, kSchedCompress);
  if (kind == kCompressFeatures)
    fsz_compress_kernel<false, true><<<g, kThreads, c.smem, st>>>(a);
  else if (kind == kCompressGiven)
    fsz_compress_kernel<true, false><<<g, kThreads, c.smem, st>>>(a);
  else
    fsz_compress_kernel<false, false><<<g, kThreads, c.smem, st>>>(a);
}

}  // namespace fsz
