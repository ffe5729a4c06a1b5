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
//   decode warps  (8) d4 bit-unshuffle one tile at a time (lane j owns elements 8j..8j+7),
//                 d5 invert the prediction as warp-wide prefix sums (once for LZ1, twice
//                 for LZ2), add mu, d' = fl(float(q) s), and store the tile with a 1-D TMA
//                 bulk store from a per-warp double buffer.
#include "fsz_internal.cuh"

namespace fsz {

namespace {

constexpr int kDecodeWarps = 8;
constexpr int kHeaderWarp = kDecodeWarps;
constexpr int kLoaderWarp = kDecodeWarps + 1;
constexpr int kThreads = (kDecodeWarps + 2) * 32;
constexpr int kStages = 2;   // payload stages
constexpr int kRecs = 6;     // chunk records in flight (fetched .. decoded)
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
  uint8_t list[kDChunkTiles];   // pre-zeroed output: the tiles to decode (not all-zero ones)
  uint32_t ndec;                // how many
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
  float out[kDecodeWarps][2][kTile];  // per-warp double buffer for the TMA stores
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

// Decodes one tile with one warp; returns false if the tile's mean slot is malformed.
// kAny: the instance that also decodes streams without the cross-block state; for those
// (`indep`) the inverse prediction's prefix sums restart at every block (4 lanes, zero
// predecessors): the warp-wide prefix less the prefix at the block's start. The other
// instance carries none of that code (it costs the full method's decode 3 %).
template <bool kAny>
__device__ __forceinline__ bool decompress_tile(const uint64_t h, const uint64_t boff,
                                                const uint8_t* __restrict__ tp,
                                                float* __restrict__ out, const float s,
                                                const int lane, const bool indep) {
  constexpr uint32_t FULL = 0xffffffffu;
  const int g = lane >> 2, t = lane & 3;
  const bool second = (h & 0x80u) != 0, centred = (h & 0x40u) != 0;
  const int Rg = int((h >> (8 * g)) & 31u);
  // d2: words per block (rate + 1, or 0) and block offsets by a byte-wise prefix sum.
  const int offw = int((boff >> (8 * g)) & 0xFFu);
  const uint8_t* blk = tp + (centred ? 4 : 0) + 4 * offw;

  bool good = true;
  int mu = 0;
  if (centred) {
    const float muf = *reinterpret_cast<const float*>(tp);
    if (!(fabsf(muf) <= 16777216.0f)) {
      good = false;
    } else {
      mu = __float2int_rn(muf);
      if (__int2float_rn(mu) != muf) good = false;
    }
  }

  // d4: decode and bit-unshuffle: words -> per-lane plane bytes -> 8x8 transpose.
  uint32_t vv[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  const int Rmax = int(__reduce_max_sync(FULL, uint32_t(Rg)));
  const int nwords = Rg > 0 ? Rg + 1 : 0;  // block g's words: sign map + Rg planes
  if (Rmax > 0) {
    const int nch = (Rmax + 8) >> 3;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      if (c < nch) {
        const int w0 = 8 * c + t, w1 = w0 + 4;
        uint32_t lo = w0 < nwords ? reinterpret_cast<const uint32_t*>(blk)[w0] : 0u;
        uint32_t hi = w1 < nwords ? reinterpret_cast<const uint32_t*>(blk)[w1] : 0u;
        lo = transpose4x4_bytes(lo, t);
        hi = transpose4x4_bytes(hi, t);
        transpose8x8(lo, hi);
        // lo bytes 0..3 are byte c of v_7..v_4, hi bytes 0..3 byte c of v_3..v_0.
        const uint32_t keep = 0x3210u & ~(0xFu << (4 * c));
        vv[7] = __byte_perm(vv[7], lo, keep | (4u << (4 * c)));
        vv[6] = __byte_perm(vv[6], lo, keep | (5u << (4 * c)));
        vv[5] = __byte_perm(vv[5], lo, keep | (6u << (4 * c)));
        vv[4] = __byte_perm(vv[4], lo, keep | (7u << (4 * c)));
        vv[3] = __byte_perm(vv[3], hi, keep | (4u << (4 * c)));
        vv[2] = __byte_perm(vv[2], hi, keep | (5u << (4 * c)));
        vv[1] = __byte_perm(vv[1], hi, keep | (6u << (4 * c)));
        vv[0] = __byte_perm(vv[0], hi, keep | (7u << (4 * c)));
      }
    }
  }
  // Sign-magnitude back to residuals (two's-complement wrap-around arithmetic).
  uint32_t x[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    x[i] = uint32_t(mad_s32(int(vv[i] >> 1), mad_s32(int(vv[i] & 1u), -2, 1), 0));
  }
  // d5: inverse prediction. With zero predecessors, LZ1's q_i = l_i + q_{i-1} is an
  // inclusive prefix sum over the tile; LZ2's q_i = l_i + 2 q_{i-1} - q_{i-2} is the prefix
  // sum of the prefix sum (the first sum rebuilds the LZ1 residuals).
  auto prefix = [&](uint32_t (&v)[8]) {
#pragma unroll
    for (int i = 1; i < 8; ++i) v[i] += v[i - 1];
    const uint32_t tot = v[7];
    uint32_t inc = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) inc = scan_step_up(inc, o);
    uint32_t ex = inc - tot;
    if (kAny && indep) {  // less the inclusive prefix of the lane before the block's first
      const uint32_t b = __shfl_sync(FULL, inc, (lane & ~3) - 1);
      if (lane >= 4) ex -= b;
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] += ex;
  };
  if (second) prefix(x);
  prefix(x);
  float o[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) o[i] = __fmul_rn(__int2float_rn(int(x[i] + uint32_t(mu))), s);
  reinterpret_cast<float4*>(out)[2 * lane] = make_float4(o[0], o[1], o[2], o[3]);
  reinterpret_cast<float4*>(out)[2 * lane + 1] = make_float4(o[4], o[5], o[6], o[7]);
  return __all_sync(FULL, good);
}

// kAny: also decodes streams without the cross-block state. kPrezero: the output already
// holds zeros; tiles whose 8 blocks all have rate 0 and no mean (all +0.0) are neither
// decoded nor written (the adaptive pre-zero of Sec. 3.1 for high compression ratios).
template <bool kAny, bool kPrezero>
__global__ void __launch_bounds__(kThreads, 4) fsz_decompress_kernel(KernelArgs a) {
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
      uint32_t dmask = 0;
      if constexpr (kPrezero) {
        const bool dec = lane < ntiles && (hb & 0x1F1F1F1F1F1F1F5FULL) != 0;
        dmask = __ballot_sync(FULL, dec);
        if (dec) q.list[__popc(dmask & ((1u << lane) - 1u))] = uint8_t(lane);
      }
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
        q.ndec = uint32_t(__popc(dmask));
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
  uint32_t nstore = 0;
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
      const uint8_t* pay = S.payload[p] + st.shift;
      const int nloop = kPrezero ? int(st.ndec) : ntiles;
      for (int i = warp; i < nloop; i += kDecodeWarps) {
        const int tl = kPrezero ? int(st.list[i]) : i;
        float* buf = S.out[warp][nstore & 1u];
        if (lane == 0) asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
        __syncwarp();
        good &= decompress_tile<kAny>(st.hdr[tl], st.boff[tl], pay + st.toff[tl], buf, step, lane,
                                      st.indep != 0);
        fence_proxy_async();
        __syncwarp();
        const uint32_t k0 = uint32_t(tl) * kTile;
        const uint32_t valid_elems = min(uint32_t(kTile), cnt - k0);
        const uint32_t bulk = (valid_elems * 4) & ~15u;
        if (lane == 0 && bulk) {
          tma_store_1d(dout + k0, buf, bulk);
          tma_store_commit();
        }
        for (uint32_t k = bulk / 4 + lane; k < valid_elems; k += 32) dout[k0 + k] = buf[k];
        ++nstore;
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
  if (lane == 0) tma_store_wait_all();
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
