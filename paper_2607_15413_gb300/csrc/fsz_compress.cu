// FSZ single-pass compression kernel (Sec. 3.1 steps 1-5, Sec. 4).
//
// Persistent, warp-specialised CTAs (no CTA-wide barrier in the main loop; the roles
// hand chunks to one another through mbarriers):
//   producer warp  takes chunk tickets and stages each chunk of kChunkTiles tiles in
//                  shared memory with a 1-D TMA bulk copy, kStages chunks ahead;
//   compute warps  (8) quantize, predict, evaluate the four variants, select and encode
//                  one tile at a time from registers into a per-tile slot in shared
//                  memory, and write the tile's rate header (steps 1-3 and 5; the tile is
//                  read from HBM once);
//   scanner warp   scans the chunk's tile sizes, publishes the chunk's aggregate flag,
//                  looks back for the chunk's exclusive byte offset (step 4, Sec. 4.4) and
//                  publishes the inclusive prefix;
//   compute warps  copy each chunk's slots to their place in the stream kDefer chunks
//                  later, by which time the scanner has resolved the chunk's offset.
#include "fsz_internal.cuh"

namespace fsz {

namespace {

constexpr int kComputeWarps = 8;
constexpr int kProducerWarp = kComputeWarps;
constexpr int kScannerWarp = kComputeWarps + 1;
constexpr int kThreads = (kComputeWarps + 2) * 32;
constexpr int kStages = 2;            // TMA input stages
constexpr int kSets = 3;              // slot sets of encoded tiles
constexpr int kDefer = kSets - 1;     // chunk j is copied out while computing chunk j + kDefer
constexpr uint32_t kNone = 0xffffffffu;
constexpr int kSlot = kMaxTileBytes;
static_assert(kChunkTiles <= 32, "one lane per tile in the chunk scan");
static_assert(kSlot % 4 == 0, "slots hold 32-bit words");

// A chunk's parameters, read once from the field record by the producer and handed to the
// other warps through shared memory (keeps dependent global loads off the compute path).
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
  uint32_t bulk_elems;   // elements covered by the TMA copy
  float r;
  uint32_t flags;        // kInfo* bits
};

struct __align__(16) CompressSmem {
  float in[kStages][kChunkElems];            // TMA stages
  uint8_t slot[kSets][kChunkTiles][kSlot];   // encoded tiles awaiting their offset
  uint64_t hdr[kComputeWarps];               // per-warp scratch: one tile's 8 header bytes
  uint32_t tbytes[kSets][kChunkTiles];
  uint32_t toff[kSets][kChunkTiles];
  uint64_t set_excl[kSets];
  uint32_t set_total[kSets];
  ChunkInfo stage_info[kStages];             // producer -> compute warps
  ChunkInfo pre[2];                          // producer's tickets taken ahead
  ChunkInfo set_info[kSets];                 // compute warp 0 -> scanner
  ChunkInfo warp_info[kComputeWarps][kSets]; // each compute warp's own copy, for its copy-out
  uint64_t full[kStages], empty[kStages], computed[kSets], resolved[kSets];
};

// Eq. 3: S_b = 0 for r_b = 0, else 4 + 4 r_b.
__device__ __forceinline__ uint32_t block_cost(int R) { return (uint32_t(R) + (R != 0 ? 1u : 0u)) << 2; }

// v = 2|l| + sign: bit 0 is the sign-map bit, bit k + 1 magnitude bit-plane k (Sec. 4.3).
__device__ __forceinline__ uint32_t sign_mag(int l) { return (uabs32(l) << 1) | (uint32_t(l) >> 31); }

// Compresses the 256-element tile at `tile` (shared memory) with one warp. Lane j owns
// elements 8j..8j+7; the 4 lanes 4g..4g+3 own block g. Writes the tile's 8 rate-header
// bytes to hdr and its encoded bytes to slot; returns the byte count (warp-uniform).
__device__ __forceinline__ uint32_t compress_tile(const float* __restrict__ tile,
                                                  uint8_t* __restrict__ slot,
                                                  uint8_t* __restrict__ hdr, const float r,
                                                  const int lane) {
  constexpr uint32_t FULL = 0xffffffffu;
  const float4 A = reinterpret_cast<const float4*>(tile)[2 * lane];
  const float4 B = reinterpret_cast<const float4*>(tile)[2 * lane + 1];
  const float d[8] = {A.x, A.y, A.z, A.w, B.x, B.y, B.z, B.w};

  // Step 1, quantize (Sec. 4.2.2): t = fl(d r) then the nearest integer, ties to even.
  // Y holds q + bits(M); differences of Y are differences of q.
  int Y[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) Y[i] = __float_as_int(__fadd_rn(__fmul_rn(d[i], r), kMagic));

  // Tile sum for centring (Sec. 4.2.2, variant 3), in the fixed order: the lane's 8
  // elements left to right, then a butterfly over lanes 16, 8, 4, 2, 1.
  float P = d[0];
#pragma unroll
  for (int i = 1; i < 8; ++i) P = __fadd_rn(P, d[i]);
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) P = __fadd_rn(P, __shfl_xor_sync(FULL, P, o));
  const int mu =
      __float_as_int(__fadd_rn(__fmul_rn(__fmul_rn(P, 0.00390625f), r), kMagic)) - kMagicBits;

  // LZ1 residuals with the state carried across lane and block boundaries (Eq. 2); the
  // tile's first predecessor is zero. LZ2 as the difference of LZ1 residuals:
  // l2_i = (q_i - q_{i-1}) - (q_{i-1} - q_{i-2}).
  int prevY = __shfl_up_sync(FULL, Y[7], 1);
  if (lane == 0) prevY = kMagicBits;
  int l1[8], l2[8];
  l1[0] = Y[0] - prevY;
#pragma unroll
  for (int i = 1; i < 8; ++i) l1[i] = Y[i] - Y[i - 1];
  int prevL = __shfl_up_sync(FULL, l1[7], 1);
  if (lane == 0) prevL = 0;
  l2[0] = l1[0] - prevL;
#pragma unroll
  for (int i = 1; i < 8; ++i) l2[i] = l1[i] - l1[i - 1];

  // Block maxima as ORs (same bit length). rest* leave out the tile's first residual(s),
  // the only ones centring changes (Eq. 4); they are used by lane 0 only.
  uint32_t rest1 = 0, rest2 = 0;
#pragma unroll
  for (int i = 1; i < 8; ++i) rest1 |= uabs32(l1[i]);
#pragma unroll
  for (int i = 2; i < 8; ++i) rest2 |= uabs32(l2[i]);
  const uint32_t o1 = rest1 | uabs32(l1[0]);
  const uint32_t o2 = rest2 | uabs32(l2[0]) | uabs32(l2[1]);
  const uint32_t x1 = __shfl_xor_sync(FULL, o1, 1);
  uint32_t b1 = o1 | x1;
  const uint32_t x2 = __shfl_xor_sync(FULL, b1, 2);
  b1 |= x2;
  const uint32_t y1 = __shfl_xor_sync(FULL, o2, 1);
  uint32_t b2 = o2 | y1;
  const uint32_t y2 = __shfl_xor_sync(FULL, b2, 2);
  b2 |= y2;
  // Rate r_b = bit length of the block maximum (Sec. 4.1.2).
  const int R1 = 32 - __clz(int(b1));
  const int R2 = 32 - __clz(int(b2));

  // Centred block-0 rates (lane 0): l1c_0 = q_0 - mu, l2c_0 = q_0 - mu,
  // l2c_1 = q_1 - 2 q_0 + mu = l2_1 + mu; the rest of block 0 is unchanged.
  const int q0 = Y[0] - kMagicBits;
  const uint32_t c10 = uabs32(q0 - mu);
  const uint32_t c21 = uabs32(l2[1] + mu);
  const int R1c = 32 - __clz(int(rest1 | x1 | x2 | c10));
  const int R2c = 32 - __clz(int(rest2 | y1 | y2 | c10 | c21));

  // Tile costs C = sum of S_b (Eq. 3), plus 4 bytes for mu when centred (step 2).
  uint32_t pk = block_cost(R1) | (block_cost(R2) << 16);
  pk += __shfl_xor_sync(FULL, pk, 4);
  pk += __shfl_xor_sync(FULL, pk, 8);
  pk += __shfl_xor_sync(FULL, pk, 16);
  const int C1 = int(pk & 0xffffu), C2 = int(pk >> 16);
  uint32_t bc = (block_cost(R1c) - block_cost(R1) + 1024u) |
                ((block_cost(R2c) - block_cost(R2) + 1024u) << 11) | (uint32_t(R1c) << 22) |
                (uint32_t(R2c) << 27);
  bc = __shfl_sync(FULL, bc, 0);
  const int C3 = 4 + C1 + int(bc & 0x7ffu) - 1024;
  const int C4 = 4 + C2 + int((bc >> 11) & 0x7ffu) - 1024;
  const int R1c0 = int((bc >> 22) & 31u), R2c0 = int(bc >> 27);

  // Step 3, adaptive select: first strict minimum in the order LZ1, LZ2, LZ1c, LZ2c.
  int v = 0, best = C1;
  if (C2 < best) { v = 1; best = C2; }
  if (C3 < best) { v = 2; best = C3; }
  if (C4 < best) { v = 3; best = C4; }
  const bool second = (v & 1) != 0, centred = v >= 2;

  const int g = lane >> 2, t = lane & 3;
  int Rg = second ? R2 : R1;
  if (g == 0 && centred) Rg = second ? R2c0 : R1c0;
  // Rate header (Sec. 3.1): block 0 carries bit 7 = order 2, bit 6 = centred.
  if (t == 0) {
    uint32_t hb = uint32_t(Rg);
    if (g == 0) hb |= (second ? 0x80u : 0u) | (centred ? 0x40u : 0u);
    hdr[g] = uint8_t(hb);
  }

  // Step 5: residuals of the selected variant as sign-magnitude words v = 2|l| + sign,
  // so that bit 0 is the sign map and bit k + 1 is magnitude bit-plane k (Sec. 4.3).
  uint32_t vv[8];
  if (second) {  // the variant is warp-uniform
#pragma unroll
    for (int i = 0; i < 8; ++i) vv[i] = sign_mag(l2[i]);
  } else {
#pragma unroll
    for (int i = 0; i < 8; ++i) vv[i] = sign_mag(l1[i]);
  }
  if (centred && lane == 0) {
    vv[0] = sign_mag(q0 - mu);
    if (second) vv[1] = sign_mag(l2[1] + mu);
  }

  // Byte offset of block g inside the tile's data (after mu when centred).
  const int Sg = int(block_cost(Rg));
  int inc = Sg, tmp;
  tmp = __shfl_up_sync(FULL, inc, 4); if (lane >= 4) inc += tmp;
  tmp = __shfl_up_sync(FULL, inc, 8); if (lane >= 8) inc += tmp;
  tmp = __shfl_up_sync(FULL, inc, 16); if (lane >= 16) inc += tmp;
  uint8_t* blk = slot + (centred ? 4 : 0) + (inc - Sg);
  if (centred && lane == 0) *reinterpret_cast<float*>(slot) = __int2float_rn(mu);

  const int Rmax = int(__reduce_max_sync(FULL, uint32_t(Rg)));
  if (Rmax > 0) {
    const int nch = (Rmax + 8) >> 3;  // 8-plane slices of v covering bits 0..Rmax
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      if (c < nch) {
        // Byte c of v_7..v_4 into lo, of v_3..v_0 into hi (element order reversed), so the
        // 8x8 transpose leaves plane 8c + b in byte b with element i at bit 7 - i.
        const uint32_t sel = uint32_t(c) | (uint32_t(4 + c) << 4);
        uint32_t lo = __byte_perm(__byte_perm(vv[7], vv[6], sel), __byte_perm(vv[5], vv[4], sel), 0x5410);
        uint32_t hi = __byte_perm(__byte_perm(vv[3], vv[2], sel), __byte_perm(vv[1], vv[0], sel), 0x5410);
        transpose8x8(lo, hi);
        // Gather the 4 lanes' bytes of one plane into a 32-element word: lane t then
        // holds words 8c + t and 8c + 4 + t of its block, bytes in memory order.
        lo = transpose4x4_bytes(lo, t);
        hi = transpose4x4_bytes(hi, t);
        const int w0 = 8 * c + t, w1 = w0 + 4;
        if (Rg > 0 && w0 <= Rg) reinterpret_cast<uint32_t*>(blk)[w0] = lo;
        if (Rg > 0 && w1 <= Rg) reinterpret_cast<uint32_t*>(blk)[w1] = hi;
      }
    }
  }
  return uint32_t(best);
}

__global__ void __launch_bounds__(kThreads, 3) fsz_compress_kernel(KernelArgs a) {
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
      mbar_init(&S.computed[k], kComputeWarps);
      mbar_init(&S.resolved[k], 1);
    }
    fence_mbar_init();
  }
  __syncthreads();

  if (warp == kProducerWarp) {
    // ---------------------------------------------------------------- producer
    // Tickets are taken two chunks ahead, so the ticket atomic and the field-record loads
    // overlap the wait for a free stage; a free stage is refilled at once.
    if (lane != 0) return;
    const bool single = a.ctrl->nfields == 1;
    auto fetch = [&](ChunkInfo& ci) {
      const uint32_t c = atomicAdd(&a.ctrl->ticket, 1u);
      ci.chunk = c;
      if (c >= total) return;
      FieldInfo* fi = single ? a.fields : a.fields + a.chunk_field[c];
      const uint64_t first = fi->chunk_first;
      const uint64_t lc = c - first;
      const uint64_t tile0 = lc * kChunkTiles;
      const uint64_t e0 = tile0 * kTile;
      const uint64_t T = fi->T;
      const uint32_t cnt = uint32_t(min(fi->n - e0, uint64_t(kChunkElems)));
      const bool ok = fi->s > 0.0f;  // a field without a step has nothing to load
      ci.in = fi->in + e0;
      ci.out = fi->out;
      ci.fi = fi;
      ci.tile0 = tile0;
      ci.data_base = 64 + 8 * T;
      ci.cap = fi->cap;
      ci.chunk_first = first;
      ci.ntiles = uint32_t(min(uint64_t(kChunkTiles), T - tile0));
      ci.cnt = cnt;
      ci.bulk_elems = ok ? ((cnt * 4) & ~15u) / 4 : 0u;
      ci.r = fi->r;
      ci.flags = (ok ? kInfoOk : 0u) | (lc + 1 == fi->nchunks ? kInfoLast : 0u) |
                 (lc == 0 ? kInfoFirst : 0u) | (uint64_t(c) == a.skip_chunk ? kInfoSkip : 0u);
    };
    fetch(S.pre[0]);
    fetch(S.pre[1]);
    for (uint32_t j = 0;; ++j) {
      const int s = int(j % kStages);
      if (j >= uint32_t(kStages) && !mbar_wait(&S.empty[s], ((j / kStages) - 1) & 1u, wait_ns)) {
        set_error(a.ctrl, nullptr, FSZ_ERR_TIMEOUT);
        return;
      }
      ChunkInfo& q = S.pre[j & 1];
      S.stage_info[s] = q;
      if (q.chunk >= total) {
        S.stage_info[s].chunk = kNone;
        mbar_arrive(&S.full[s]);
        return;
      }
      const uint32_t bulk = q.bulk_elems * 4;
      fence_proxy_async();
      mbar_arrive_expect_tx(&S.full[s], bulk);
      if (bulk) tma_load_1d(S.in[s], q.in, bulk, &S.full[s]);
      fetch(q);  // the ticket two chunks ahead
    }
  }

  if (warp == kScannerWarp) {
    // ---------------------------------------------------------------- scanner
    // Chunk j's aggregate is published as soon as its tiles are encoded; chunk j's
    // lookback waits until chunk j + 1 is encoded, so that the chunks ticketed next to
    // chunk j on other SMs have published theirs by then.
    uint32_t prev_c = kNone, prev_tot = 0, prev_flags = 0;
    uint64_t prev_first = 0;
    FieldInfo* prev_fi = nullptr;
    int prev_b = 0;
    auto resolve = [&](uint32_t c, uint64_t first, uint32_t flags, FieldInfo* fi, uint32_t tot, int b) {
      uint64_t excl = 0;
      if (!(flags & kInfoFirst)) {
        bool to = false;
        excl = lookback(a.flags, int64_t(c), int64_t(first), globaltimer_ns() + a.timeout_ns, &to);
        if (lane == 0) {
          if (to) set_error(a.ctrl, fi, FSZ_ERR_TIMEOUT);
          if (!(flags & kInfoSkip)) st_flag(a.flags + c, kFlagIncl | (excl + tot));
        }
      }
      __syncwarp();
      if (lane == 0) {
        S.set_excl[b] = excl;
        S.set_total[b] = tot;
        mbar_arrive(&S.resolved[b]);
      }
    };
    for (uint32_t j = 0;; ++j) {
      const int b = int(j % kSets);
      if (!mbar_wait(&S.computed[b], (j / kSets) & 1u, wait_ns)) {
        if (lane == 0) set_error(a.ctrl, nullptr, FSZ_ERR_TIMEOUT);
        return;
      }
      const ChunkInfo& ci = S.set_info[b];
      const uint32_t c = ci.chunk;
      if (c == kNone) break;
      const uint32_t flags = ci.flags;
      const int ntiles = int(ci.ntiles);
      // Thread and warp levels of the scan over the chunk's tiles; the chunk's aggregate.
      const uint32_t mine = ((flags & kInfoOk) && lane < ntiles) ? S.tbytes[b][lane] : 0u;
      uint32_t inc = mine;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t x = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += x;
      }
      if (lane < kChunkTiles) S.toff[b][lane] = inc - mine;
      const uint32_t tot = __shfl_sync(0xffffffffu, inc, 31);
      if (lane == 0 && !(flags & kInfoSkip))
        st_flag(a.flags + c, ((flags & kInfoFirst) ? kFlagIncl : kFlagAgg) | tot);
      // Device level for the previous chunk.
      if (prev_c != kNone) resolve(prev_c, prev_first, prev_flags, prev_fi, prev_tot, prev_b);
      prev_c = c;
      prev_first = ci.chunk_first;
      prev_flags = flags;
      prev_fi = ci.fi;
      prev_tot = tot;
      prev_b = b;
    }
    if (prev_c != kNone) resolve(prev_c, prev_first, prev_flags, prev_fi, prev_tot, prev_b);
    return;
  }

  // ------------------------------------------------------------------ compute warps
  // Copies this warp's tiles of chunk k (slot set k % kSets) into the stream.
  auto copy_out = [&](uint32_t k) -> bool {
    const int b = int(k % kSets);
    if (!mbar_wait(&S.resolved[b], (k / kSets) & 1u, wait_ns)) return false;
    const ChunkInfo& ci = S.warp_info[warp][b];
    if ((ci.flags & (kInfoOk | kInfoSkip)) != kInfoOk) return true;
    const uint64_t excl = S.set_excl[b];
    const uint32_t tot = S.set_total[b];
    if (ci.data_base + excl + tot > ci.cap) {
      if (lane == 0) set_error(a.ctrl, ci.fi, FSZ_ERR_CAPACITY);
    } else {
      uint8_t* base = ci.out + ci.data_base + excl;
      for (int tl = warp; tl < int(ci.ntiles); tl += kComputeWarps) {
        const uint32_t nw = S.tbytes[b][tl] >> 2;
        const uint32_t* src = reinterpret_cast<const uint32_t*>(S.slot[b][tl]);
        uint32_t* dst = reinterpret_cast<uint32_t*>(base + S.toff[b][tl]);
        for (uint32_t q = lane; q < nw; q += 32) dst[q] = src[q];
      }
      if (warp == 0 && lane == 0 && (ci.flags & kInfoLast)) write_preamble(ci.fi, excl + tot);
    }
    return true;
  };

  uint32_t j = 0;
  for (;; ++j) {
    const int s = int(j % kStages), b = int(j % kSets);
    if (!mbar_wait(&S.full[s], (j / kStages) & 1u, wait_ns)) {
      if (lane == 0) set_error(a.ctrl, nullptr, FSZ_ERR_TIMEOUT);
      return;
    }
    const ChunkInfo& ci = S.stage_info[s];
    // Keep the chunk's parameters past the stage's reuse: this warp's copy, and warp 0's
    // copy for the scanner (16 lanes copy 4 bytes each).
    static_assert(sizeof(ChunkInfo) % 4 == 0 && sizeof(ChunkInfo) <= 128, "ChunkInfo copy");
    if (lane < int(sizeof(ChunkInfo) / 4)) {
      const uint32_t w = reinterpret_cast<const uint32_t*>(&ci)[lane];
      reinterpret_cast<uint32_t*>(&S.warp_info[warp][b])[lane] = w;
      if (warp == 0) reinterpret_cast<uint32_t*>(&S.set_info[b])[lane] = w;
    }
    if (warp == 0) __threadfence_block();  // all lanes' copies before lane 0's arrival
    const uint32_t c = ci.chunk;
    if (c == kNone) {
      __syncwarp();
      if (lane == 0) mbar_arrive(&S.computed[b]);  // tells the scanner to stop
      break;
    }
    const uint32_t flags = ci.flags;
    if (flags & kInfoOk) {
      const float r = ci.r;
      const int ntiles = int(ci.ntiles);
      const uint32_t cnt = ci.cnt, bulk_elems = ci.bulk_elems;
      const float* gin = ci.in;
      uint64_t* hdr_out = reinterpret_cast<uint64_t*>(ci.out + 64) + ci.tile0;
      for (int tl = warp; tl < ntiles; tl += kComputeWarps) {
        float* tile = S.in[s] + tl * kTile;
        // Ragged end of a field: this lane's elements past the last 16-byte boundary of
        // the bulk copy by plain loads; padding elements are zeros (they quantize to 0).
        const uint32_t k0 = uint32_t(tl) * kTile + 8u * uint32_t(lane);
        if (k0 + 8 > bulk_elems) {
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const uint32_t k = k0 + uint32_t(i);
            if (k >= bulk_elems) tile[8 * lane + i] = k < cnt ? gin[k] : 0.0f;
          }
        }
        const uint32_t nb = compress_tile(tile, S.slot[b][tl],
                                          reinterpret_cast<uint8_t*>(&S.hdr[warp]), r, lane);
        __syncwarp();
        if (lane == 0) {
          S.tbytes[b][tl] = nb;
          hdr_out[tl] = S.hdr[warp];
        }
        __syncwarp();
      }
    }
    __syncwarp();
    if (lane == 0) {
      mbar_arrive(&S.empty[s]);     // done reading the stage
      mbar_arrive(&S.computed[b]);  // tile sizes ready for the scanner
    }
    if (j >= uint32_t(kDefer) && !copy_out(j - kDefer)) {
      if (lane == 0) set_error(a.ctrl, nullptr, FSZ_ERR_TIMEOUT);
      return;
    }
  }
  // Chunks computed but not yet placed.
  for (uint32_t k = j >= uint32_t(kDefer) ? j - kDefer : 0; k < j; ++k) {
    if (!copy_out(k)) {
      if (lane == 0) set_error(a.ctrl, nullptr, FSZ_ERR_TIMEOUT);
      return;
    }
  }
}

}  // namespace

LaunchCfg compress_cfg() {
  static LaunchCfg cfg = [] {
    LaunchCfg c;
    c.smem = int(sizeof(CompressSmem));
    cudaFuncSetAttribute(fsz_compress_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, c.smem);
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fsz_compress_kernel, kThreads, c.smem);
    c.sms = sms;
    c.per = per > 0 ? per : 1;
    c.grid = sms * c.per;
    return c;
  }();
  return cfg;
}

void launch_compress(const KernelArgs& a, cudaStream_t st) {
  const LaunchCfg c = compress_cfg();
  fsz_compress_kernel<<<sched_grid(c, kSchedCompress), kThreads, c.smem, st>>>(a);
}

}  // namespace fsz
