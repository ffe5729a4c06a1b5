// FSZ decompression kernel (Sec. 3.1 "Decompression", steps d1-d5).
//
// Persistent, warp-specialised CTAs; the roles hand chunks to one another through
// mbarriers:
//   header warp   takes a ticket, d1 reads the chunk's rate header, d2 derives the tile
//                 sizes and scans them, publishes the chunk's aggregate flag at once and
//                 leaves the chunk's record (headers, offsets, field parameters) in a ring
//                 of kRecs records, running ahead of decoding;
//   loader warp   d3 looks back for the chunk's byte offset (decoupled lookback) as soon
//                 as the record is in, publishes the inclusive prefix, then waits for a
//                 free payload stage and loads the chunk's payload into it with a 1-D TMA
//                 bulk copy (the lookback thus overlaps the decoding of earlier chunks);
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
constexpr int kStages = 2;   // payload stages
constexpr int kRecs = 6;     // chunk records in flight (fetched .. decoded)
constexpr int kQuadTiles = 4;  // tiles per decode warp and iteration
constexpr int kPayloadBytes = kDChunkTiles * kMaxDecTileBytes + 32;
static_assert(kDChunkTiles <= 32, "one lane per tile in the chunk scan");
static_assert(kPayloadBytes % 16 == 0, "stage size");
constexpr uint32_t kNoneChunk = 0xffffffffu;
constexpr int kLookbackPerLane = 4;  // 128-flag lookback window

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
  uint32_t shift;        // payload start inside the stage
  uint32_t ntiles;
  uint32_t cnt;          // valid elements of the chunk
  uint32_t indep;        // the stream's blocks are independent (no carried state)
  float step;
};

struct __align__(16) DecompressSmem {
  uint8_t payload[kStages][kPayloadBytes];
  float out[kDecodeWarps][kQuadTiles * kTile];  // per-warp re-layout of a quad's floats
  ChunkRec rec[kRecs];
  uint64_t fetched[kRecs], recfree[kRecs], full[kStages], empty[kStages];
};

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
  if (apply) {
#pragma unroll
    for (int i = 1; i < 32; ++i) x[i] += x[i - 1];
  }
  const uint32_t tot = x[31];
  uint32_t inc = tot;
#pragma unroll
  for (int o = 1; o < 8; o <<= 1) inc = scan_step_up<8>(inc, o);
  uint32_t ex = inc - tot;
  if (kAny && indep) ex = 0;
  ex += add;
  if (apply) {
#pragma unroll
    for (int i = 0; i < 32; ++i) x[i] += ex;
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
  const int nw = Rg > 0 ? Rg + 1 : 0;  // block g's words: sign map + Rg planes
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
  // d4: the block's words, back through the plane network, into sign-magnitude words v
  uint32_t v[32];
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = 0u;
  const int Rmax = int(__reduce_max_sync(FULL, uint32_t(Rg)));
  if (Rmax > 0) {
    const int nch = (Rmax + 8) >> 3;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      if (c < nch) {
        uint32_t X[8];
#pragma unroll
        for (int b = 0; b < 8; ++b) X[b] = 8 * c + b < nw ? lds32(blk + 4u * uint32_t(8 * c + b)) : 0u;
        swap_planes(X);
        // byte m of X[k] is byte c of element 8 m + 7 - k
        const uint32_t keep = 0x3210u & ~(0xFu << (4 * c));
#pragma unroll
        for (int k = 0; k < 8; ++k)
#pragma unroll
          for (int m = 0; m < 4; ++m)
            v[8 * m + 7 - k] = __byte_perm(v[8 * m + 7 - k], X[k], keep | ((4u + m) << (4 * c)));
      }
    }
  }
  // sign-magnitude back to residuals (two's-complement wrap-around arithmetic)
  uint32_t x[32];
#pragma unroll
  for (int i = 0; i < 32; ++i) x[i] = uint32_t(mad_s32(int(v[i] >> 1), mad_s32(int(v[i] & 1u), -2, 1), 0));
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

  if (tid == 0) {
    for (int k = 0; k < kRecs; ++k) {
      mbar_init(&S.fetched[k], 1);
      mbar_init(&S.recfree[k], kDecodeWarps);
    }
    for (int k = 0; k < kStages; ++k) {
      mbar_init(&S.full[k], 1);
      mbar_init(&S.empty[k], kDecodeWarps);
    }
    fence_mbar_init();
  }
  __syncthreads();

  if (warp == kHeaderWarp) {
    // ---------------------------------------------------------------- header warp
    const bool single = a.ctrl->nfields == 1;
    for (uint32_t seq = 0;; ++seq) {
      const int r = int(seq % kRecs);
      if (seq >= uint32_t(kRecs) && !mbar_wait(&S.recfree[r], ((seq / kRecs) - 1) & 1u, wait_ns)) {
        if (lane == 0) set_error(a.ctrl, nullptr, FSZ_ERR_TIMEOUT);
        return;
      }
      ChunkRec& q = S.rec[r];
      uint32_t c = 0;
      if (lane == 0) c = atomicAdd(&a.ctrl->ticket, 1u);
      c = __shfl_sync(FULL, c, 0);
      if (c >= total) {
        if (lane == 0) {
          q.chunk = kNoneChunk;
          mbar_arrive(&S.fetched[r]);
        }
        return;
      }
      FieldInfo* fi = single ? a.fields : a.fields + a.chunk_field[c];
      const uint64_t first = fi->chunk_first;
      const uint64_t lc = c - first;
      const uint64_t T = fi->T;
      const uint64_t tile0 = lc * kDChunkTiles;
      const int ntiles = int(min(uint64_t(kDChunkTiles), T - tile0));
      const uint8_t* sin = fi->sin;
      uint64_t hb = 0;
      if (lane < ntiles) hb = __ldg(reinterpret_cast<const unsigned long long*>(sin + 64) + tile0 + lane);
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
      if (lane == 0) {
        if (uint64_t(c) != a.skip_chunk) st_flag(a.flags + uint64_t(c) * kFlagStride, (lc == 0 ? kFlagIncl : kFlagAgg) | tot);
        q.chunk = c;
        q.lc = uint32_t(lc);
        q.last = (lc + 1 == fi->nchunks) ? 1u : 0u;
        q.tot = tot;
        q.bad = bad_hdr ? 1u : 0u;
        q.fi = fi;
        q.sin = sin;
        q.in_bytes = fi->in_bytes;
        q.data_bytes = fi->data_bytes;
        q.data_base = 64 + 8 * T;
        q.dout = fi->dout + tile0 * kTile;
        q.ntiles = uint32_t(ntiles);
        q.cnt = uint32_t(min(fi->n - tile0 * kTile, uint64_t(kDChunkElems)));
        q.step = fi->s;
        q.indep = (foff & kOffCross) ? 1u : 0u;
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&S.fetched[r]);
    }
  }

  if (warp == kLoaderWarp) {
    // ---------------------------------------------------------------- loader warp
    for (uint32_t seq = 0;; ++seq) {
      const int r = int(seq % kRecs), p = int(seq % kStages);
      if (!mbar_wait(&S.fetched[r], (seq / kRecs) & 1u, wait_ns)) {
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
        excl = lookback<kLookbackPerLane>(a.flags, int64_t(c), int64_t(c) - int64_t(q.lc),
                                          globaltimer_ns() + a.timeout_ns, &to);
        if (lane == 0) {
          if (to) set_error(a.ctrl, fi, FSZ_ERR_TIMEOUT);
          if (!skip) st_flag(a.flags + uint64_t(c) * kFlagStride, kFlagIncl | (excl + tot));
        }
      }
      // The payload stage frees once the decode warps are through chunk seq - kStages.
      if (seq >= uint32_t(kStages) && !mbar_wait(&S.empty[p], ((seq / kStages) - 1) & 1u, wait_ns)) {
        if (lane == 0) set_error(a.ctrl, nullptr, FSZ_ERR_TIMEOUT);
        return;
      }
      if (none) {
        if (lane == 0) mbar_arrive(&S.full[p]);
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
      if (lane == 0) {
        if (!valid && !skip) set_error(a.ctrl, fi, FSZ_ERR_CORRUPT);
        q.shift = uint32_t(src - a0);
        q.valid = valid ? 1u : 0u;
        if (bulk) {
          fence_proxy_async();
          mbar_expect_tx(&S.full[p], bulk);
          tma_load_1d(S.payload[p], reinterpret_cast<const void*>(a0), bulk, &S.full[p]);
        }
      }
      if (valid) {
        // Payload bytes past the last 16-byte boundary of the bulk copy: plain loads.
        const uint32_t lo = uint32_t(max(a1, src) - a0), hi = uint32_t(src + tot - a0);
        const uint8_t* gb = reinterpret_cast<const uint8_t*>(a0);
        for (uint32_t k = lo + 4 * uint32_t(lane); k < hi; k += 128)
          *reinterpret_cast<uint32_t*>(S.payload[p] + k) = *reinterpret_cast<const uint32_t*>(gb + k);
      }
      __threadfence_block();  // every lane's tail bytes before lane 0's arrival
      __syncwarp();
      if (lane == 0) mbar_arrive(&S.full[p]);
    }
  }

  // ------------------------------------------------------------------ decode warps
  const uint32_t obuf = smem_u32(S.out[warp]);
  bool good = true;
  for (uint32_t seq = 0;; ++seq) {
    const int r = int(seq % kRecs), p = int(seq % kStages);
    if (!mbar_wait(&S.full[p], (seq / kStages) & 1u, wait_ns)) {
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
      const uint32_t pay = smem_u32(S.payload[p]) + st.shift;
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
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const uint32_t P = uint32_t(32 * j + lane);   // piece: row P >> 3, column P & 7
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
        __syncwarp();  // the buffer is read before the next quad overwrites it
      }
    }
    if (!good && lane == 0) set_error(a.ctrl, fi, FSZ_ERR_CORRUPT);
    good = true;
    __syncwarp();
    if (lane == 0) {
      mbar_arrive(&S.empty[p]);
      mbar_arrive(&S.recfree[r]);
    }
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

void launch_decompress(const KernelArgs& a, cudaStream_t st, DecompressKind kind) {
  const LaunchCfg c = decompress_cfg();
  const int g = sched_grid(c, kSchedDecompress);
  if (kind == kDecompressAny)
    fsz_decompress_kernel<true, false><<<g, kThreads, c.smem, st>>>(a);
  else if (kind == kDecompressPrezeroed)
    fsz_decompress_kernel<false, true><<<g, kThreads, c.smem, st>>>(a);
  else
    fsz_decompress_kernel<false, false><<<g, kThreads, c.smem, st>>>(a);
}

}  // namespace fsz
