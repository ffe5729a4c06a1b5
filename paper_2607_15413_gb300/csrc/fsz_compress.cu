// FSZ single-pass compression kernel (Sec. 3.1 steps 1-5, Sec. 4).
//
// One persistent CTA of 8 warps loops over chunks of 32 tiles taken from a device
// ticket. Per chunk:
//   1. the chunk's 32 KiB were staged in shared memory by a 1-D TMA bulk copy issued
//      one chunk ahead (double buffer, mbarrier completion);
//   2. each warp quantizes, predicts, evaluates the four variants, selects and encodes
//      one tile at a time, entirely from registers, into a per-tile slot in shared
//      memory (steps 1-3 and 5 of Sec. 3.1: the tile is read once, from shared memory);
//   3. warp 0 scans the 32 tile sizes, publishes the chunk's aggregate, looks back over
//      the predecessors' flags for the chunk's exclusive byte offset (step 4, Sec. 4.4)
//      and publishes the inclusive prefix; the other warps write the rate header;
//   4. all warps copy the encoded tiles to their final place in the stream.
#include "fsz_internal.cuh"

namespace fsz {

namespace {

constexpr int kWarps = 8;
constexpr int kThreads = kWarps * 32;
constexpr int kSlot = kMaxTileBytes;
static_assert(kChunkTiles == 32, "one lane per tile in the chunk scan");
static_assert(kSlot % 4 == 0, "slots hold 32-bit words");

struct __align__(16) CompressSmem {
  float in[2][kChunkElems];
  uint8_t slot[kChunkTiles][kSlot];
  uint8_t hdr[kChunkTiles * 8];
  uint32_t tbytes[kChunkTiles];
  uint32_t toff[kChunkTiles];
  uint64_t bar[2];
  uint64_t excl;
  uint32_t chunk[2];
  uint32_t total;
  uint32_t abort;
};

__device__ __forceinline__ uint32_t block_cost(int R) { return R ? 4u + 4u * uint32_t(R) : 0u; }

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
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    int l = second ? l2[i] : l1[i];
    if (centred && lane == 0) {
      if (i == 0) l = q0 - mu;
      if (i == 1 && second) l = l2[1] + mu;
    }
    vv[i] = (uabs32(l) << 1) | (uint32_t(l) >> 31);
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

__global__ void __launch_bounds__(kThreads, 2) fsz_compress_kernel(KernelArgs a) {
  extern __shared__ __align__(128) uint8_t smem_raw[];
  CompressSmem& S = *reinterpret_cast<CompressSmem*>(smem_raw);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint64_t total = a.ctrl->total_chunks;

  if (tid == 0) {
    mbar_init(&S.bar[0], 1);
    mbar_init(&S.bar[1], 1);
    fence_mbar_init();
    S.abort = 0;
  }
  __syncthreads();

  // Takes the next ticket into stage s and starts its TMA load (thread 0).
  auto issue = [&](int s) {
    const uint32_t c = atomicAdd(&a.ctrl->ticket, 1u);
    S.chunk[s] = c;
    if (c < total) {
      const FieldInfo* fi = a.fields + a.chunk_field[c];
      const uint64_t e0 = (c - fi->chunk_first) * uint64_t(kChunkElems);
      const uint64_t cnt = min(fi->n - e0, uint64_t(kChunkElems));
      uint32_t bulk = uint32_t(cnt * 4) & ~15u;
      if (!(fi->s > 0.0f)) bulk = 0;  // field without a step: nothing to load
      fence_proxy_async();
      mbar_arrive_expect_tx(&S.bar[s], bulk);
      if (bulk) tma_load_1d(S.in[s], fi->in + e0, bulk, &S.bar[s]);
    }
  };

  if (tid == 0) {
    issue(0);
    issue(1);
  }
  __syncthreads();

  for (uint32_t it = 0;; ++it) {
    const int s = it & 1;
    const uint32_t c = S.chunk[s];
    if (c >= total) break;
    FieldInfo* fi = a.fields + a.chunk_field[c];
    const float r = fi->r;
    const bool ok = fi->s > 0.0f;
    const uint64_t lc = c - fi->chunk_first;
    const uint64_t T = fi->T;
    const uint64_t tile0 = lc * kChunkTiles;
    const int ntiles = int(min(uint64_t(kChunkTiles), T - tile0));
    const uint64_t e0 = tile0 * kTile;
    const uint32_t cnt = uint32_t(min(fi->n - e0, uint64_t(kChunkElems)));

    // Wait for the stage (bounded); one thread waits, the barrier publishes the data.
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
    }
    __syncthreads();
    if (S.abort) return;

    // Ragged end of a field: the bytes past the last 16-byte boundary by plain loads, and
    // zero padding up to the tile boundary (padding elements quantize to 0).
    if (ok && cnt < uint32_t(ntiles) * kTile) {
      const uint32_t bulk_elems = (cnt * 4 & ~15u) / 4;
      float* buf = S.in[s];
      for (uint32_t k = bulk_elems + tid; k < uint32_t(ntiles) * kTile; k += kThreads)
        buf[k] = k < cnt ? fi->in[e0 + k] : 0.0f;
      __syncthreads();
    }

    if (ok) {
      for (int tl = warp; tl < ntiles; tl += kWarps) {
        const uint32_t b = compress_tile(S.in[s] + tl * kTile, S.slot[tl], S.hdr + tl * 8, r, lane);
        if (lane == 0) S.tbytes[tl] = b;
      }
    }
    __syncthreads();
    if (tid == 32) issue(s);  // the stage is consumed: refill it (warp 0 scans meanwhile)

    if (warp == 0) {
      // Step 4 (Sec. 4.4): thread/warp level over the chunk's tiles, then device level.
      const uint32_t mine = (ok && lane < ntiles) ? S.tbytes[lane] : 0u;
      uint32_t inc = mine;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t x = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += x;
      }
      if (lane < ntiles) S.toff[lane] = inc - mine;
      const uint32_t tot = __shfl_sync(0xffffffffu, inc, 31);
      const bool skip = (uint64_t(c) == a.skip_chunk);
      const bool first = (lc == 0);
      if (lane == 0 && !skip) st_release_u64(a.flags + c, (first ? kFlagIncl : kFlagAgg) | tot);
      uint64_t excl = 0;
      if (!first) {
        bool to = false;
        excl = lookback(a.flags, int64_t(c), int64_t(fi->chunk_first),
                        globaltimer_ns() + a.timeout_ns, &to);
        if (lane == 0) {
          if (to) set_error(a.ctrl, fi, FSZ_ERR_TIMEOUT);
          if (!skip) st_release_u64(a.flags + c, kFlagIncl | (excl + tot));
        }
      }
      if (lane == 0) {
        S.excl = excl;
        S.total = tot;
      }
    } else if (ok) {
      // Rate header of the chunk's tiles: 8 bytes per tile at 64 + 8 * tile.
      const uint32_t* h32 = reinterpret_cast<const uint32_t*>(S.hdr);
      uint32_t* dst = reinterpret_cast<uint32_t*>(fi->out + 64 + 8 * tile0);
      for (int k = tid - 32; k < 2 * ntiles; k += kThreads - 32) dst[k] = h32[k];
    }
    __syncthreads();

    if (ok && uint64_t(c) != a.skip_chunk) {
      const uint64_t excl = S.excl;
      const uint32_t tot = S.total;
      const uint64_t data_base = 64 + 8 * T;
      if (data_base + excl + tot > fi->cap) {
        if (tid == 0) set_error(a.ctrl, fi, FSZ_ERR_CAPACITY);
      } else {
        uint8_t* base = fi->out + data_base + excl;
        for (int tl = warp; tl < ntiles; tl += kWarps) {
          const uint32_t nw = S.tbytes[tl] >> 2;
          const uint32_t* src = reinterpret_cast<const uint32_t*>(S.slot[tl]);
          uint32_t* dst = reinterpret_cast<uint32_t*>(base + S.toff[tl]);
          for (uint32_t k = lane; k < nw; k += 32) dst[k] = src[k];
        }
      }
      if (tid == 0 && lc + 1 == fi->nchunks) write_preamble(fi, excl + tot);
    }
    __syncthreads();
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
    c.grid = sms * (per > 0 ? per : 1);
    return c;
  }();
  return cfg;
}

void launch_compress(const KernelArgs& a, cudaStream_t st) {
  const LaunchCfg c = compress_cfg();
  fsz_compress_kernel<<<c.grid, kThreads, c.smem, st>>>(a);
}

}  // namespace fsz
