// FSZ decompression kernel (Sec. 3.1 "Decompression", steps d1-d5).
//
// One persistent CTA of 8 warps, software-pipelined over chunks of 32 tiles:
//   prepare(next)  [warp 0]  d1 read the chunk's rate header, d2 tile sizes, d3 scan:
//                            warp scan over tiles, then decoupled lookback over chunks;
//                            then a 1-D TMA bulk load of the chunk's payload into the
//                            other shared-memory stage;
//   decode(cur)    [warps]   d4 bit-unshuffle each tile with one warp (lane j owns
//                            elements 8j..8j+7), d5 inverse prediction as warp-wide
//                            prefix sums (once for LZ1, twice for LZ2), + mu, then
//                            d' = fl(float(q) s) into shared memory;
//   store(cur)               1-D TMA bulk store of the decoded floats.
// Warp 0 joins the tile queue once its prepare step is done.
#include "fsz_internal.cuh"

namespace fsz {

namespace {

constexpr int kWarps = 8;
constexpr int kThreads = kWarps * 32;
constexpr int kPayloadBytes = kChunkTiles * kMaxDecTileBytes + 32;
static_assert(kChunkTiles == 32, "one lane per tile in the chunk scan");
static_assert(kPayloadBytes % 16 == 0, "stage size");

struct __align__(16) DecompressSmem {
  uint8_t payload[2][kPayloadBytes];
  float out[kChunkElems];
  uint64_t hdr[2][kChunkTiles];
  uint32_t toff[2][kChunkTiles];
  uint64_t bar[2];
  uint64_t gbase[2];      // 16-byte aligned global address the stage starts at
  uint32_t chunk[2];      // ticket held by the stage
  uint32_t shift[2];      // payload start inside the stage
  uint32_t tail_lo[2];    // [tail_lo, tail_hi): bytes after the bulk part, plain loads
  uint32_t tail_hi[2];
  uint32_t valid[2];
  uint32_t next_tile;
  uint32_t abort;
};

// Bytes of a tile from its 8 header bytes: sum of S_b (Eq. 3) + 4 for a centred tile.
__device__ __forceinline__ uint32_t tile_bytes_from_header(uint64_t h) {
  const uint64_t R = h & 0x1F1F1F1F1F1F1F1FULL;
  const uint64_t W = R + (((R + 0x7F7F7F7F7F7F7F7FULL) & 0x8080808080808080ULL) >> 7);
  const uint32_t lo = uint32_t(W), hi = uint32_t(W >> 32);
  const uint32_t words = ((lo * 0x01010101u) >> 24) + ((hi * 0x01010101u) >> 24);
  return 4u * words + ((h & 0x40u) ? 4u : 0u);
}

__device__ __forceinline__ bool header_reserved_bits_set(uint64_t h) {
  return (h & 0x20u) || (h & 0xE0E0E0E0E0E0E000ULL);
}

// Decodes one tile with one warp; returns false if the tile's mean slot is malformed.
__device__ __forceinline__ bool decompress_tile(const uint64_t h, const uint8_t* __restrict__ tp,
                                                float* __restrict__ out, const float s,
                                                const int lane) {
  constexpr uint32_t FULL = 0xffffffffu;
  const int g = lane >> 2, t = lane & 3;
  const bool second = (h & 0x80u) != 0, centred = (h & 0x40u) != 0;
  const int Rg = int((h >> (8 * g)) & 31u);
  // d2: words per block (rate + 1, or 0) and block offsets by a byte-wise prefix sum.
  const uint64_t R = h & 0x1F1F1F1F1F1F1F1FULL;
  const uint64_t W = R + (((R + 0x7F7F7F7F7F7F7F7FULL) & 0x8080808080808080ULL) >> 7);
  const uint64_t P = W * 0x0101010101010101ULL;
  const int offw = g ? int((P >> (8 * (g - 1))) & 0xFFu) : 0;
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
  if (Rmax > 0) {
    const int nch = (Rmax + 8) >> 3;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      if (c < nch) {
        const int w0 = 8 * c + t, w1 = w0 + 4;
        uint32_t lo = (Rg > 0 && w0 <= Rg) ? reinterpret_cast<const uint32_t*>(blk)[w0] : 0u;
        uint32_t hi = (Rg > 0 && w1 <= Rg) ? reinterpret_cast<const uint32_t*>(blk)[w1] : 0u;
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
    const uint32_t m = vv[i] >> 1;
    x[i] = (vv[i] & 1u) ? 0u - m : m;
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
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(FULL, inc, o);
      if (lane >= o) inc += y;
    }
    const uint32_t ex = inc - tot;
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

__global__ void __launch_bounds__(kThreads, 2) fsz_decompress_kernel(KernelArgs a) {
  extern __shared__ __align__(128) uint8_t smem_raw[];
  DecompressSmem& S = *reinterpret_cast<DecompressSmem*>(smem_raw);
  constexpr uint32_t FULL = 0xffffffffu;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint64_t total = a.ctrl->total_chunks;

  if (tid == 0) {
    mbar_init(&S.bar[0], 1);
    mbar_init(&S.bar[1], 1);
    fence_mbar_init();
    S.abort = 0;
    S.next_tile = 0;
  }
  __syncthreads();

  // d1-d3 for the next ticket, and the payload load into stage s (one whole warp).
  auto prepare = [&](int s) {
    uint32_t c = 0;
    if (lane == 0) c = atomicAdd(&a.ctrl->ticket, 1u);
    c = __shfl_sync(FULL, c, 0);
    if (lane == 0) S.chunk[s] = c;
    if (c >= total) return;
    FieldInfo* fi = a.fields + a.chunk_field[c];
    const uint64_t lc = c - fi->chunk_first;
    const uint64_t T = fi->T;
    const uint64_t tile0 = lc * kChunkTiles;
    const int ntiles = int(min(uint64_t(kChunkTiles), T - tile0));
    uint64_t h = 0;
    if (lane < ntiles) h = __ldg(reinterpret_cast<const unsigned long long*>(fi->sin + 64) + tile0 + lane);
    S.hdr[s][lane] = h;
    const bool bad_hdr = __any_sync(FULL, lane < ntiles && header_reserved_bits_set(h));
    const uint32_t mine = lane < ntiles ? tile_bytes_from_header(h) : 0u;
    uint32_t inc = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(FULL, inc, o);
      if (lane >= o) inc += y;
    }
    S.toff[s][lane] = inc - mine;
    const uint32_t tot = __shfl_sync(FULL, inc, 31);
    const bool skip = (uint64_t(c) == a.skip_chunk);
    const bool first = (lc == 0);
    if (lane == 0 && !skip) st_release_u64(a.flags + c, (first ? kFlagIncl : kFlagAgg) | tot);
    uint64_t excl = 0;
    if (!first) {
      bool to = false;
      excl = lookback(a.flags, int64_t(c), int64_t(fi->chunk_first), globaltimer_ns() + a.timeout_ns,
                      &to);
      if (lane == 0) {
        if (to) set_error(a.ctrl, fi, FSZ_ERR_TIMEOUT);
        if (!skip) st_release_u64(a.flags + c, kFlagIncl | (excl + tot));
      }
    }
    if (lane == 0) {
      const uint64_t data_base = 64 + 8 * T;
      bool valid = !bad_hdr && !skip;
      if (data_base + excl + tot > fi->in_bytes) valid = false;
      if (lc + 1 == fi->nchunks && excl + tot != fi->data_bytes) valid = false;
      if (!valid && !skip) set_error(a.ctrl, fi, FSZ_ERR_CORRUPT);
      const uint64_t src = reinterpret_cast<uint64_t>(fi->sin) + data_base + excl;
      const uint64_t a0 = src & ~uint64_t(15);
      const uint64_t a1 = (src + tot) & ~uint64_t(15);
      const uint32_t bulk = (valid && a1 > a0) ? uint32_t(a1 - a0) : 0u;
      S.gbase[s] = a0;
      S.shift[s] = uint32_t(src - a0);
      S.tail_lo[s] = uint32_t(max(a1, src) - a0);
      S.tail_hi[s] = uint32_t(src + tot - a0);
      S.valid[s] = valid ? 1u : 0u;
      fence_proxy_async();
      mbar_arrive_expect_tx(&S.bar[s], bulk);
      if (bulk) tma_load_1d(S.payload[s], reinterpret_cast<const void*>(a0), bulk, &S.bar[s]);
    }
    __syncwarp();
  };

  if (warp == 0) prepare(0);
  __syncthreads();

  for (uint32_t it = 0;; ++it) {
    const int s = it & 1;
    const uint32_t c = S.chunk[s];
    if (c >= total) break;
    FieldInfo* fi = a.fields + a.chunk_field[c];
    const float step = fi->s;
    const uint64_t lc = c - fi->chunk_first;
    const uint64_t tile0 = lc * kChunkTiles;
    const int ntiles = int(min(uint64_t(kChunkTiles), fi->T - tile0));
    const uint64_t e0 = tile0 * kTile;
    const uint32_t cnt = uint32_t(min(fi->n - e0, uint64_t(kChunkElems)));

    if (tid == 0) {
      const uint32_t parity = (it >> 1) & 1u;
      uint64_t deadline = 0;
      uint32_t spins = 0;
      while (!mbar_try_wait(&S.bar[s], parity)) {
        if ((++spins & 255u) == 0) {
          const uint64_t now = globaltimer_ns();
          if (deadline == 0) {
            deadline = now + a.timeout_ns;
          } else if (now > deadline) {
            set_error(a.ctrl, fi, FSZ_ERR_TIMEOUT);
            S.abort = 1;
            break;
          }
        }
      }
      tma_store_wait_read_all();  // the previous chunk's store has read S.out
      S.next_tile = 0;
    }
    __syncthreads();
    if (S.abort) break;
    const bool valid = S.valid[s] != 0;
    if (valid) {
      // Payload bytes past the last 16-byte boundary of the bulk copy.
      const uint8_t* gb = reinterpret_cast<const uint8_t*>(S.gbase[s]);
      for (uint32_t k = S.tail_lo[s] + 4 * tid; k < S.tail_hi[s]; k += 4 * kThreads)
        *reinterpret_cast<uint32_t*>(S.payload[s] + k) = *reinterpret_cast<const uint32_t*>(gb + k);
    }
    __syncthreads();

    if (warp == 0) prepare(s ^ 1);
    if (valid) {
      bool good = true;
      for (;;) {
        uint32_t tl = 0;
        if (lane == 0) tl = atomicAdd(&S.next_tile, 1u);
        tl = __shfl_sync(FULL, tl, 0);
        if (tl >= uint32_t(ntiles)) break;
        good &= decompress_tile(S.hdr[s][tl], S.payload[s] + S.shift[s] + S.toff[s][tl],
                                S.out + tl * kTile, step, lane);
      }
      if (!good && lane == 0) set_error(a.ctrl, fi, FSZ_ERR_CORRUPT);
      fence_proxy_async();
    }
    __syncthreads();
    if (valid) {
      const uint32_t bulk = (cnt * 4) & ~15u;
      if (tid == 0 && bulk) {
        tma_store_1d(fi->dout + e0, S.out, bulk);
        tma_store_commit();
      }
      for (uint32_t k = bulk / 4 + tid; k < cnt; k += kThreads) fi->dout[e0 + k] = S.out[k];
    }
  }
  if (tid == 0) tma_store_wait_all();
}

}  // namespace

LaunchCfg decompress_cfg() {
  static LaunchCfg cfg = [] {
    LaunchCfg c;
    c.smem = int(sizeof(DecompressSmem));
    cudaFuncSetAttribute(fsz_decompress_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, c.smem);
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fsz_decompress_kernel, kThreads, c.smem);
    c.grid = sms * (per > 0 ? per : 1);
    return c;
  }();
  return cfg;
}

void launch_decompress(const KernelArgs& a, cudaStream_t st) {
  const LaunchCfg c = decompress_cfg();
  fsz_decompress_kernel<<<c.grid, kThreads, c.smem, st>>>(a);
}

}  // namespace fsz
