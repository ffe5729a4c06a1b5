// FSZ decompression kernel (Sec. 3.1 "Decompression", steps d1-d5).
//
// Persistent, warp-specialised CTAs; the roles hand chunks to one another through
// mbarriers:
//   header warp   takes a ticket, d1 reads the chunk's rate header, d2 derives the tile
//                 sizes and scans them, publishes the chunk's aggregate flag at once and
//                 leaves the chunk's record (headers, offsets, field parameters) in a ring
//                 of records, running ahead of decoding;
//   loader warp   d3 looks back for the chunk's byte offset (decoupled lookback) as soon
//                 as the record is in, publishes the inclusive prefix, then takes the
//                 chunk's payload bytes (its actual size, not the worst case) from a byte
//                 ring, waiting for the oldest chunks' decoding to release space, and loads
//                 the payload there with a 1-D TMA bulk copy. Compressed chunks being far
//                 below the worst case, several are in flight per CTA;
//   decode warps  (8) each decode a quad of 4 tiles at a time, lane L holding block L & 7
//                 of tile L >> 3 (32 consecutive elements): d4 reads the block's sign map
//                 and planes and undoes the bit shuffle with the register-pair delta swaps
//                 of the compressor, run backwards; d5 inverts the prediction as prefix sums
//                 inside the lane with the carry from the tile's earlier blocks by an 8-lane
//                 scan (once for LZ1, twice for LZ2), adds mu, d' = fl(float(q) s); the
//                 floats go through a per-warp swizzled buffer so that each store of the
//                 warp writes 512 consecutive bytes.
#include "fsz_internal.cuh"

namespace fsz {

namespace {

constexpr int kDecodeWarps = 8;
constexpr int kHeaderWarp = kDecodeWarps;
constexpr int kLoaderWarp = kDecodeWarps + 1;
constexpr int kThreads = (kDecodeWarps + 2) * 32;
#ifndef FSZ_DEC_RING_BYTES
#define FSZ_DEC_RING_BYTES 65536
#endif
constexpr int kMaxRecs = kMaxDecRecords;  // chunk records (fetched .. decoded): up to
constexpr uint32_t kRingBytes = FSZ_DEC_RING_BYTES;  // payload byte ring
constexpr int kQuadTiles = 4;  // tiles per decode warp and iteration
// Ring bytes a chunk can take: its payload (at most kDChunkTiles header-valid tiles) from
// the 16-byte boundary below its start, rounded up to 16 bytes.
constexpr uint32_t kMaxChunkRingBytes = kDChunkTiles * kMaxDecTileBytes + 32;
static_assert(kDChunkTiles <= 32, "one lane per tile in the chunk scan");
static_assert(kRingBytes % 16 == 0 && kRingBytes >= kMaxChunkRingBytes, "the ring holds the largest chunk");

constexpr uint32_t kNoneChunk = 0xffffffffu;
#ifndef FSZ_DEC_LOOKBACK_K
#define FSZ_DEC_LOOKBACK_K 1
#endif
constexpr int kLookbackPerLane = FSZ_DEC_LOOKBACK_K;  // lookback window: 32 K flags
// The schedule's work assignment (kernel arguments): a ticket hands a CTA ticket_chunks
// consecutive chunks (at most kMaxTicketChunks). Their rate headers are read together,
// and a chunk that follows its group's previous chunk in the same field takes its byte
// offset from that chunk (no lookback), so the atomics and the lookbacks per chunk drop by
// that factor. A CTA holds `records` chunks (2 x ticket_chunks .. kMaxRecs) between
// ticket and decode.

// A chunk's header and parameters, from the header warp to the loader and the decode
// warps through shared memory (keeps dependent global loads off the decode path).
struct ChunkRec {
  uint64_t hdr[kDChunkTiles];
  uint64_t boff[kDChunkTiles];  // block word offsets of each tile (block_word_offsets)
  uint32_t toff[kDChunkTiles];
  FieldInfo* fi;
  float* dout;           // the chunk's first output element
  const uint8_t* sin;    // the field's stream
  uint64_t in_bytes;     // its size
  uint64_t data_bytes;   // tile data bytes the preamble declares
  uint64_t data_base;    // 64 + 8T: start of the tile data
  uint64_t excl;         // byte offset of the chunk's payload in the tile data
  uint32_t chunk;        // ticket, or kNoneChunk
  uint32_t lc;           // chunk index inside the field
  uint32_t last;         // the field's last chunk
  uint32_t tot;          // payload bytes of the chunk
  uint32_t bad;          // reserved header bits seen
  uint32_t valid;        // payload loaded and decodable
  uint32_t pay;          // payload start inside the ring
  uint32_t ntiles;
  uint32_t cnt;          // valid elements of the chunk
  uint32_t indep;        // the stream's blocks are independent (no carried state)
  uint32_t chain;        // the previous record holds chunk - 1 of the same field
  float step;
};

struct __align__(16) DecompressSmem {
  uint8_t ring[kRingBytes];
  float out[kDecodeWarps][kQuadTiles * kTile];  // per-warp re-layout of a quad's floats
  ChunkRec rec[kMaxRecs];
  uint32_t ring_end[kMaxRecs];  // loader only: ring position (mod 2^32) after each chunk's bytes
  // fetched: record in (header -> loader); full: payload in (loader -> decode warps);
  // done: chunk decoded, its record and ring bytes free (decode warps -> header, loader)
  uint64_t fetched[kMaxRecs], full[kMaxRecs], done[kMaxRecs];
};
// two CTAs per SM (228 KiB of shared memory, 1 KiB of it reserved per CTA)
static_assert(sizeof(DecompressSmem) <= 113 * 1024, "shared memory of one CTA");

// Bytes of a tile from its 8 header bytes: sum of S_b (Eq. 3) + 4 for a centred tile.
__device__ __forceinline__ uint32_t tile_bytes_from_header(uint64_t h) {
  const uint64_t R = h & 0x1F1F1F1F1F1F1F1FULL;
  const uint64_t W = R + (((R + 0x7F7F7F7F7F7F7F7FULL) & 0x8080808080808080ULL) >> 7);
  const uint32_t lo = uint32_t(W), hi = uint32_t(W >> 32);
  const uint32_t words = ((lo * 0x01010101u) >> 24) + ((hi * 0x01010101u) >> 24);
  return 4u * words + ((h & 0x40u) ? 4u : 0u);
}

// Word offsets of the 8 blocks inside the tile's data (after mu), one per byte: the
// exclusive byte-wise prefix sum of the blocks' word counts (rate + 1, or 0; <= 224).
__device__ __forceinline__ uint64_t block_word_offsets(uint64_t h) {
  const uint64_t R = h & 0x1F1F1F1F1F1F1F1FULL;
  const uint64_t W = R + (((R + 0x7F7F7F7F7F7F7F7FULL) & 0x8080808080808080ULL) >> 7);
  return (W * 0x0101010101010101ULL) << 8;
}

__device__ __forceinline__ bool header_reserved_bits_set(uint64_t h) {
  return (h & 0x20u) || (h & 0xE0E0E0E0E0E0E000ULL);
}

// Byte permute with the generic mode's sign replication (a selector nibble with bit 3 set
// fills the result byte with the top bit of the byte it selects).
__device__ __forceinline__ uint32_t prmt(uint32_t a, uint32_t b, uint32_t sel) {
  uint32_t d;
  asm("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(sel));
  return d;
}
__device__ __forceinline__ uint32_t lds32(uint32_t addr) {
  uint32_t v;
  asm volatile("ld.shared.b32 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
  return v;
}
__device__ __forceinline__ void sts128(uint32_t addr, float4 v) {
  asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "f"(v.x), "f"(v.y),
               "f"(v.z), "f"(v.w)
               : "memory");
}
__device__ __forceinline__ float4 lds128(uint32_t addr) {
  float4 v;
  asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "r"(addr)
               : "memory");
  return v;
}

// Inclusive prefix sum over a tile of x[0..31] in each lane (the lane's block), the 8
// lanes of a tile carrying block to block: the lane's own prefix, then the exclusive scan
// of the blocks' totals over the tile's lanes, plus `add`. Without the carried state
// (indep) each block restarts. Lanes with `apply` false keep x; every lane of the warp
// must call this (the scan's shuffles take the full warp), and the 8 lanes of a tile
// agree on `apply`, so the scan segments of applying tiles see only their own lanes.
template <bool kAny>
__device__ __forceinline__ void tile_prefix(uint32_t (&x)[32], const uint32_t add, const bool indep,
                                            const bool apply) {
  // the lane's prefix as four independent 8-element runs (short dependency chains), the
  // runs' offsets folded into the final additions
  uint32_t o1 = 0, o2 = 0, o3 = 0, tot = 0;
  if (apply) {
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
      for (int i = 1; i < 8; ++i) x[8 * k + i] += x[8 * k + i - 1];
    o1 = x[7];
    o2 = o1 + x[15];
    o3 = o2 + x[23];
    tot = o3 + x[31];
  }
  uint32_t inc = tot;
#pragma unroll
  for (int o = 1; o < 8; o <<= 1) inc = scan_step_up<8>(inc, o);
  uint32_t ex = inc - tot;
  if (kAny && indep) ex = 0;
  ex += add;
  if (apply) {
    const uint32_t e[4] = {ex, ex + o1, ex + o2, ex + o3};
#pragma unroll
    for (int i = 0; i < 32; ++i) x[i] += e[i >> 3];
  }
}

// Decodes one quad (4 tiles) with one warp into o (lane L: block L & 7 of tile L >> 3).
// h, boff: the lane's tile's header and block word offsets; tp: shared-memory address of
// the tile's data; live: the tile exists. Returns false if a tile's mean slot is
// malformed. kAny: the instance that also decodes streams without the cross-block state
// (`indep`: every block restarts from zero predecessors).
template <bool kAny>
__device__ __forceinline__ bool decompress_quad(const uint64_t h, const uint64_t boff,
                                                const uint32_t tp, const bool live, const float s,
                                                const int lane, const bool indep, float (&o)[32]) {
  constexpr uint32_t FULL = 0xffffffffu;
  const int g = lane & 7;
  const bool second = (h & 0x80u) != 0, centred = (h & 0x40u) != 0;
  const int Rg = live ? int((h >> (8 * g)) & 31u) : 0;
  // d2: block offsets by a byte-wise prefix sum (done by the header warp)
  const uint32_t blk = tp + (centred ? 4u : 0u) + 4u * uint32_t((boff >> (8 * g)) & 0xFFu);
  bool good = true;
  int mu = 0;
  if (live && centred) {
    const float muf = __uint_as_float(lds32(tp));
    if (!(fabsf(muf) <= 16777216.0f)) {
      good = false;
    } else {
      mu = __float2int_rn(muf);
      if (__int2float_rn(mu) != muf) good = false;
    }
  }
  // d4: the block's planes (sign map, then the magnitude bits) become the planes of the
  // two's-complement residuals by a bit-sliced negation of the negative elements,
  // x = (m ^ S) + S over all 32 elements at once (S the sign map); the planes above the
  // rate then all equal the result's sign plane. They go back through the plane network,
  // and each element is gathered from its bytes by permutes that replicate the top byte's
  // sign, which sign-extends it.
  const int Rmax = int(__reduce_max_sync(FULL, uint32_t(Rg)));
  const int nch = Rmax > 0 ? (Rmax + 8) >> 3 : 0;
  uint32_t X[4][8];
  {
    const uint32_t S = Rg > 0 ? lds32(blk) : 0u;
    uint32_t carry = S;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      if (c < nch) {
#pragma unroll
        for (int b = 0; b < 8; ++b) {
          const int j = 8 * c + b;  // plane j of x: magnitude plane j is the block's word j + 1
          const uint32_t M = j < Rg ? lds32(blk + 4u * uint32_t(j + 1)) : 0u;
          const uint32_t y = M ^ S;
          X[c][b] = y ^ carry;
          carry &= y;
        }
        swap_planes(X[c]);
      }
    }
  }
  // byte m of X[c][k] is byte c of element 8 m + 7 - k
  uint32_t x[32];
  if (nch == 0) {
#pragma unroll
    for (int i = 0; i < 32; ++i) x[i] = 0u;
  } else if (nch == 1) {
#pragma unroll
    for (int k = 0; k < 8; ++k)
#pragma unroll
      for (int m = 0; m < 4; ++m)
        x[8 * m + 7 - k] = prmt(X[0][k], 0u, m | ((8 | m) << 4) | ((8 | m) << 8) | ((8 | m) << 12));
  } else if (nch == 2) {
#pragma unroll
    for (int k = 0; k < 8; ++k)
#pragma unroll
      for (int m = 0; m < 4; ++m)
        x[8 * m + 7 - k] = prmt(X[0][k], X[1][k], m | ((4 + m) << 4) | ((12 + m) << 8) | ((12 + m) << 12));
  } else if (nch == 3) {
#pragma unroll
    for (int k = 0; k < 8; ++k)
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        const uint32_t t = prmt(X[0][k], X[1][k], m | ((4 + m) << 4));
        x[8 * m + 7 - k] = prmt(t, X[2][k], 0x0010u | ((4 + m) << 8) | ((12 + m) << 12));
      }
  } else {
#pragma unroll
    for (int k = 0; k < 8; ++k)
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        const uint32_t t = prmt(X[0][k], X[1][k], m | ((4 + m) << 4));
        const uint32_t u = prmt(X[2][k], X[3][k], (m << 8) | ((4 + m) << 12));
        x[8 * m + 7 - k] = prmt(t, u, 0x7610u);
      }
  }
  // d5: inverse prediction. With zero predecessors, LZ1's q_i = l_i + q_{i-1} is an
  // inclusive prefix sum over the tile; LZ2's q_i = l_i + 2 q_{i-1} - q_{i-2} is the prefix
  // sum of the prefix sum (the first sum rebuilds the LZ1 residuals); then + mu. The
  // quad's tiles may differ in their predictor: the first sum runs on the whole warp and
  // applies to the LZ2 tiles only.
  if (__any_sync(FULL, second)) tile_prefix<kAny>(x, 0u, indep, second);
  tile_prefix<kAny>(x, uint32_t(mu), indep, true);
#pragma unroll
  for (int i = 0; i < 32; ++i) o[i] = __fmul_rn(__int2float_rn(int(x[i])), s);
  return __all_sync(FULL, good);
}

// kAny: also decodes streams without the cross-block state. kPrezero: the output already
// holds zeros; tiles whose 8 blocks all have rate 0 and no mean (all +0.0) are neither
// decoded nor written (the adaptive pre-zero of Sec. 3.1 for high compression ratios).
template <bool kAny, bool kPrezero>
__global__ void __launch_bounds__(kThreads, 2) fsz_decompress_kernel(KernelArgs a) {
  extern __shared__ __align__(128) uint8_t smem_raw[];
  DecompressSmem& S = *reinterpret_cast<DecompressSmem*>(smem_raw);
  constexpr uint32_t FULL = 0xffffffffu;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint64_t total = a.ctrl->total_chunks;
  const uint64_t wait_ns = 4 * a.timeout_ns;
  const uint32_t group = launch_ticket_chunks(a.ticket_chunks, a.min_tickets, total, gridDim.x);
  const uint32_t recs = a.records;

  if (tid == 0) {
    for (int k = 0; k < kMaxRecs; ++k) {
      mbar_init(&S.fetched[k], 1);
      mbar_init(&S.full[k], 1);
      mbar_init(&S.done[k], kDecodeWarps);
    }
    fence_mbar_init();
  }
  __syncthreads();

  if (warp == kHeaderWarp) {
    // ---------------------------------------------------------------- header warp
    const bool single = a.ctrl->nfields == 1;
    for (uint32_t seq = 0;; seq += group) {
      // the group's records must be free: their previous chunks decoded
      bool ok = true;
      for (uint32_t g = 0; g < group; ++g) {
        const uint32_t sg = seq + g;
        if (ok && sg >= recs) ok = mbar_wait(&S.done[sg % recs], ((sg / recs) - 1) & 1u, wait_ns);
      }
      if (!ok) {
        if (lane == 0) set_error(a.ctrl, nullptr, FSZ_ERR_TIMEOUT);
        return;
      }
      // (tickets only go to running CTAs: a CTA that is not resident yet, e.g. behind
      // another stream's kernel, holds no chunk that the others' lookbacks wait for)
      uint32_t t = 0;
      if (lane == 0) t = atomicAdd(&a.ctrl->ticket, 1u);
      t = __shfl_sync(FULL, t, 0);
      const uint64_t c0 = uint64_t(t) * group;
      // field, position and rate header of each chunk of the group (loads issued together)
      FieldInfo* fis[kMaxTicketChunks];
      uint64_t hbs[kMaxTicketChunks];
#pragma unroll
      for (int g = 0; g < kMaxTicketChunks; ++g) {
        const uint64_t c = c0 + g;
        fis[g] = nullptr;
        hbs[g] = 0;
        if (uint32_t(g) < group && c < total) {
          FieldInfo* fi = single ? a.fields : a.fields + a.chunk_field[c];
          fis[g] = fi;
          const uint64_t tile0 = (c - fi->chunk_first) * kDChunkTiles;
          if (tile0 + lane < fi->T)
            hbs[g] = __ldg(reinterpret_cast<const unsigned long long*>(fi->sin + 64) + tile0 + lane);
        }
      }
      bool end = false;
      uint64_t prev_lc = 0;
#pragma unroll
      for (int g = 0; g < kMaxTicketChunks; ++g) {
        if (uint32_t(g) >= group) break;
        const uint32_t sg = seq + g;
        const int r = int(sg % recs);
        ChunkRec& q = S.rec[r];
        const uint64_t c = c0 + g;
        if (end) continue;
        if (c >= total) {
          if (lane == 0) {
            q.chunk = kNoneChunk;
            mbar_arrive(&S.fetched[r]);
          }
          end = true;
          continue;
        }
        FieldInfo* fi = fis[g];
        const uint64_t hb = hbs[g];
        const uint64_t first = fi->chunk_first;
        const uint64_t lc = c - first;
        const uint64_t T = fi->T;
        const uint64_t tile0 = lc * kDChunkTiles;
        const int ntiles = int(min(uint64_t(kDChunkTiles), T - tile0));
        if (lane < kDChunkTiles) {
          q.hdr[lane] = hb;
          q.boff[lane] = block_word_offsets(hb);
        }
        // a tile may not use a feature the stream has switched off
        const uint32_t foff = fi->features_off;
        const uint64_t forbid = ((foff & kOffLz2) ? 0x80u : 0u) | ((foff & kOffCenter) ? 0x40u : 0u);
        // streams without the cross-block state are decoded by the kAny instance only
        const bool unsupported = !kAny && (foff & kOffCross);
        if (unsupported && lane == 0) set_error(a.ctrl, fi, FSZ_ERR_INVALID_ARG);
        const bool bad_hdr = unsupported ||
            __any_sync(FULL, lane < ntiles && (header_reserved_bits_set(hb) || (hb & forbid)));
        const uint32_t mine = lane < ntiles ? tile_bytes_from_header(hb) : 0u;
        uint32_t inc = mine;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t y = __shfl_up_sync(FULL, inc, o);
          if (lane >= o) inc += y;
        }
        if (lane < kDChunkTiles) q.toff[lane] = inc - mine;
        const uint32_t tot = __shfl_sync(FULL, inc, 31);
        // the chunk follows the group's previous one (unless that one is held back by the
        // test hook, whose successors must meet its missing flag)
        const bool chain = g > 0 && fis[g - 1] == fi && lc == prev_lc + 1 && c - 1 != a.skip_chunk;
        prev_lc = lc;
        if (lane == 0) {
          if (c != a.skip_chunk) st_flag(a.flags + c * kFlagStride, (lc == 0 ? kFlagIncl : kFlagAgg) | tot);
          q.chunk = uint32_t(c);
          q.lc = uint32_t(lc);
          q.last = (lc + 1 == fi->nchunks) ? 1u : 0u;
          q.tot = tot;
          q.bad = bad_hdr ? 1u : 0u;
          q.fi = fi;
          q.sin = fi->sin;
          q.in_bytes = fi->in_bytes;
          q.data_bytes = fi->data_bytes;
          q.data_base = 64 + 8 * T;
          q.dout = fi->dout + tile0 * kTile;
          q.ntiles = uint32_t(ntiles);
          q.cnt = uint32_t(min(fi->n - tile0 * kTile, uint64_t(kDChunkElems)));
          q.step = fi->s;
          q.indep = (foff & kOffCross) ? 1u : 0u;
          q.chain = chain ? 1u : 0u;
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&S.fetched[r]);
      }
      if (end) return;
    }
  }

  if (warp == kLoaderWarp) {
    // ---------------------------------------------------------------- loader warp
    // Ring positions count bytes modulo 2^32: head = where the next payload goes, freed =
    // how far the decoded chunks have released. Chunks take and release space in ticket
    // order, so the bytes in use are head - freed; pos is head's place in the ring.
    uint32_t head = 0, freed = 0, pos = 0;
    uint32_t oldest = 0;  // the oldest chunk whose bytes are not yet known to be released
    uint64_t prev_excl = 0, prev_tot = 0;  // the previous record's chunk: offset and bytes
    for (uint32_t seq = 0;; ++seq) {
      const int r = int(seq % recs);
      if (!mbar_wait(&S.fetched[r], (seq / recs) & 1u, wait_ns)) {
        if (lane == 0) set_error(a.ctrl, nullptr, FSZ_ERR_TIMEOUT);
        return;
      }
      ChunkRec& q = S.rec[r];
      const uint32_t c = q.chunk;
      const bool none = c == kNoneChunk;
      FieldInfo* fi = q.fi;
      const uint32_t tot = q.tot;
      const bool skip = !none && uint64_t(c) == a.skip_chunk;
      uint64_t excl = 0;
      if (!none && q.lc != 0) {
        bool to = false;
        if (q.chain)  // d3 from the group's previous chunk, resolved just before
          excl = prev_excl + prev_tot;
        else
          excl = lookback<kLookbackPerLane>(a.flags, int64_t(c), int64_t(c) - int64_t(q.lc),
                                            globaltimer_ns() + a.timeout_ns, &to);
        if (lane == 0) {
          if (to) set_error(a.ctrl, fi, FSZ_ERR_TIMEOUT);
          if (!skip) st_flag(a.flags + uint64_t(c) * kFlagStride, kFlagIncl | (excl + tot));
        }
      }
      prev_excl = excl;
      prev_tot = tot;
      if (none) {
        if (lane == 0) mbar_arrive(&S.full[r]);
        return;
      }
      bool valid = q.bad == 0 && !skip;
      if (q.data_base + excl + tot > q.in_bytes) valid = false;
      if (q.last && excl + tot != q.data_bytes) valid = false;
      const uint64_t base = reinterpret_cast<uint64_t>(q.sin);
      const uint64_t src = base + q.data_base + excl;
      const uint64_t a0 = src & ~uint64_t(15);
      // Round the copy's end up to 16 bytes while that stays inside the stream buffer;
      // otherwise the last few bytes come by plain loads.
      const uint64_t end_up = (src + tot + 15) & ~uint64_t(15);
      const uint64_t a1 = end_up <= base + q.in_bytes ? end_up : ((src + tot) & ~uint64_t(15));
      const uint32_t bulk = (valid && a1 > a0) ? uint32_t(a1 - a0) : 0u;
      // ring space: the payload from a0, rounded up to 16 bytes, in one piece (a payload
      // that would run past the ring's end starts at the ring's start instead)
      const uint32_t need = valid ? (uint32_t(src - a0) + tot + 15u) & ~15u : 0u;
      uint32_t start = head, phys = pos;
      if (pos + need > kRingBytes) {
        start += kRingBytes - pos;
        phys = 0;
      }
      // Chunks seq - recs and older are decoded: the header warp reused their records.
      while (oldest + recs <= seq) freed = S.ring_end[oldest++ % recs];
      bool space = true;
      while (start + need - freed > kRingBytes) {
        if (oldest == seq) {  // nothing in flight: the skipped end of the ring is free too
          freed = start;
          break;
        }
        // wait for the oldest chunk in flight; its record is not reused before it is done
        if (!mbar_wait(&S.done[oldest % recs], (oldest / recs) & 1u, wait_ns)) {
          space = false;
          break;
        }
        freed = S.ring_end[oldest % recs];
        ++oldest;
      }
      if (!space) {
        if (lane == 0) set_error(a.ctrl, nullptr, FSZ_ERR_TIMEOUT);
        return;
      }
      head = start + need;
      pos = phys + need;
      if (lane == 0) S.ring_end[r] = head;
      if (lane == 0) {
        if (!valid && !skip) set_error(a.ctrl, fi, FSZ_ERR_CORRUPT);
        q.pay = phys + uint32_t(src - a0);
        q.valid = valid ? 1u : 0u;
        if (bulk) {
          fence_proxy_async();
          mbar_expect_tx(&S.full[r], bulk);
          tma_load_1d(S.ring + phys, reinterpret_cast<const void*>(a0), bulk, &S.full[r]);
        }
      }
      if (valid) {
        // Payload bytes past the last 16-byte boundary of the bulk copy: plain loads.
        const uint32_t lo = uint32_t(max(a1, src) - a0), hi = uint32_t(src + tot - a0);
        const uint8_t* gb = reinterpret_cast<const uint8_t*>(a0);
        for (uint32_t k = lo + 4 * uint32_t(lane); k < hi; k += 128)
          *reinterpret_cast<uint32_t*>(S.ring + phys + k) = *reinterpret_cast<const uint32_t*>(gb + k);
      }
      __threadfence_block();  // every lane's tail bytes before lane 0's arrival
      __syncwarp();
      if (lane == 0) mbar_arrive(&S.full[r]);
    }
  }

  // ------------------------------------------------------------------ decode warps
  const uint32_t obuf = smem_u32(S.out[warp]);
  bool good = true;
  for (uint32_t seq = 0;; ++seq) {
    const int r = int(seq % recs);
    if (!mbar_wait(&S.full[r], (seq / recs) & 1u, wait_ns)) {
      if (lane == 0) set_error(a.ctrl, nullptr, FSZ_ERR_TIMEOUT);
      break;
    }
    const ChunkRec& st = S.rec[r];
    const uint32_t c = st.chunk;
    if (c == kNoneChunk) break;
    FieldInfo* fi = st.fi;
    if (st.valid) {
      const float step = st.step;
      const int ntiles = int(st.ntiles);
      const uint32_t cnt = st.cnt;
      float* dout = st.dout;
      const uint32_t pay = smem_u32(S.ring) + st.pay;
      const int nquads = (ntiles + kQuadTiles - 1) / kQuadTiles;
      for (int qd = warp; qd < nquads; qd += kDecodeWarps) {
        const int t = kQuadTiles * qd + (lane >> 3);
        const bool live = t < ntiles;
        const uint64_t h = live ? st.hdr[t] : 0ull;
        // a pre-zeroed output: a tile whose rates are all 0 and that has no mean is +0.0
        // throughout, neither decoded nor written; a quad of such tiles is skipped
        const bool write_tile = live && (!kPrezero || (h & 0x1F1F1F1F1F1F1F5FULL) != 0);
        if (kPrezero && !__any_sync(FULL, write_tile)) continue;
        float o[32];
        good &= decompress_quad<kAny>(h, live ? st.boff[t] : 0ull, pay + (live ? st.toff[t] : 0u),
                                      live, step, lane, st.indep != 0, o);
        // re-layout: lane L's block goes to row L of the buffer, 16-byte piece k at column
        // k ^ (L & 7) (conflict-free); then each piece P = 32 j + lane, read back in order,
        // is stored to the output, the warp writing 512 consecutive bytes per store
        const uint32_t row = obuf + uint32_t(lane) * 128u;
        const uint32_t sw = uint32_t(lane & 7) << 4;
#pragma unroll
        for (int k = 0; k < 8; ++k)
          sts128(row + ((uint32_t(k << 4)) ^ sw), make_float4(o[4 * k], o[4 * k + 1], o[4 * k + 2], o[4 * k + 3]));
        const uint32_t tmask = __ballot_sync(FULL, write_tile && (lane & 7) == 0);
        __syncwarp();
        const uint32_t e0 = uint32_t(kQuadTiles * qd) * kTile;  // the quad's first element
        if (tmask == 0x01010101u && e0 + kQuadTiles * kTile <= cnt) {
          // every tile of the quad is written in full: no per-store guards
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const uint32_t P = uint32_t(32 * j + lane);   // piece: row P >> 3, column P & 7
            const uint32_t rw = P >> 3;
            const float4 val = lds128(obuf + rw * 128u + (((P & 7u) ^ (rw & 7u)) << 4));
            *reinterpret_cast<float4*>(dout + e0 + 4 * P) = val;
          }
        } else {
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const uint32_t P = uint32_t(32 * j + lane);
            const uint32_t rw = P >> 3;
            const float4 val = lds128(obuf + rw * 128u + (((P & 7u) ^ (rw & 7u)) << 4));
            const uint32_t e = e0 + 4 * P;
            if (!((tmask >> (8 * (rw >> 3))) & 1u)) continue;  // (a tile not written)
            if (e + 4 <= cnt) {
              *reinterpret_cast<float4*>(dout + e) = val;
            } else {
              const float vals[4] = {val.x, val.y, val.z, val.w};
#pragma unroll
              for (int i = 0; i < 4; ++i)
                if (e + i < cnt) dout[e + i] = vals[i];
            }
          }
        }
        __syncwarp();  // the buffer is read before the next quad overwrites it
      }
    }
    if (!good && lane == 0) set_error(a.ctrl, fi, FSZ_ERR_CORRUPT);
    good = true;
    __syncwarp();
    if (lane == 0) mbar_arrive(&S.done[r]);
  }
}

}  // namespace

LaunchCfg decompress_cfg() {
  static DeviceCfgCache cache;
  return cache.get([] {
    LaunchCfg c;
    c.smem = int(sizeof(DecompressSmem));
    cudaFuncSetAttribute(fsz_decompress_kernel<false, false>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, c.smem);
    cudaFuncSetAttribute(fsz_decompress_kernel<true, false>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, c.smem);
    cudaFuncSetAttribute(fsz_decompress_kernel<false, true>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, c.smem);
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fsz_decompress_kernel<false, false>,
                                                  kThreads, c.smem);
    c.sms = sms;
    c.per = per > 0 ? per : 1;
    c.grid = sms * c.per;
    return c;
  });
}

void launch_decompress(const KernelArgs& args, cudaStream_t st, DecompressKind kind) {
  const LaunchCfg c = decompress_cfg();
  const int g = sched_grid(c, kSchedDecompress);
  KernelArgs a = args;
  a.ticket_chunks = uint32_t(g_schedule.d_ticket_chunks);
  a.records = uint32_t(g_schedule.d_records);
  a.min_tickets = uint32_t(g_schedule.min_tickets);
  if (kind == kDecompressAny)
    fsz_decompress_kernel<true, false><<<g, kThreads, c.smem, st>>>(a);
  else if (kind == kDecompressPrezeroed)
    fsz_decompress_kernel<false, true><<<g, kThreads, c.smem, st>>>(a);
  else
    fsz_decompress_kernel<false, false><<<g, kThreads, c.smem, st>>>(a);
}

}  // namespace fsz
