// FSZ single-pass compression kernel (Sec. 3.1 steps 1-5, Sec. 4).
//
// Persistent, warp-specialised CTAs (two per SM); the roles hand work to one another
// through mbarriers and shared counters (no CTA-wide barrier in the main loop):
//   compute warps  (kWarps) each stream their own quad (4 tiles) of every chunk into a
//                  private staging buffer with cp.async (16-byte pieces, zero-filled past
//                  the end of the field), one chunk ahead of the one they encode. Lane L of
//                  a warp holds block L & 7 of tile L >> 3 of its quad: 32 consecutive
//                  elements, read from the buffer with conflict-free 128-bit loads (the
//                  pieces sit in a 128-byte swizzled layout). They quantize, predict,
//                  evaluate the four variants, select and size the quad's tiles (steps 1-3;
//                  the input is read from HBM once), write the rate headers, and encode the
//                  quad as one contiguous run into the warp's ring in shared memory
//                  (step 5). The last warp to size a chunk scans the quads' sizes and
//                  publishes the chunk's aggregate flag before any warp has encoded it;
//   resolver warp  looks back for each chunk's exclusive byte offset (step 4, Sec. 4.4),
//                  publishes the inclusive prefix, and copies the runs of the first
//                  kResolverRuns compute warps to the stream before handing the chunk to
//                  the host warp;
//   host warp      takes a ticket per chunk just ahead of its use and leaves the chunk's
//                  parameters in one of kSets chunk slots; and places each chunk, once it
//                  is resolved and encoded, by copying the other compute warps' runs from
//                  their rings to the stream and giving the ring space back.
// The rings decouple encoding from the device-wide scan: chunks finish out of ticket order
// across the grid, and a chunk's offset is known only when every earlier chunk has
// published its size. Keeping the placement out of the compute warps keeps them within 96
// registers, so that 16 of them fit on an SM.
#include "fsz_internal.cuh"

namespace fsz {

namespace {

constexpr uint32_t FULL = 0xffffffffu;
constexpr int kQuadTiles = 4;                      // tiles per compute warp and chunk
constexpr int kWarps = kCChunkTiles / kQuadTiles;  // compute warps per CTA
constexpr int kHostWarp = kWarps;                  // tickets and placement
constexpr int kResolverWarp = kWarps + 1;
constexpr int kThreads = (kWarps + 2) * 32;
#ifndef FSZ_RESOLVER_RUNS
#define FSZ_RESOLVER_RUNS 4
#endif
// Placement split: the resolver copies the runs of compute warps 0 .. kResolverRuns - 1 of
// each chunk it resolves, before handing the chunk to the host, which copies the others.
constexpr int kResolverRuns = FSZ_RESOLVER_RUNS;
#ifndef FSZ_COMPRESS_SETS
#define FSZ_COMPRESS_SETS 12
#endif
#ifndef FSZ_RING_BYTES
#define FSZ_RING_BYTES 6144
#endif
constexpr int kSets = FSZ_COMPRESS_SETS;           // chunk slots per CTA
// The schedule's work assignment (kernel arguments): a ticket hands a CTA ticket_chunks
// consecutive chunks, and a chunk that follows the CTA's previous chunk in the same field
// takes its byte offset from it (the previous offset plus its size) instead of looking
// back; the ticket of chunk seq is taken when the compute warps begin chunk
// seq - ticket_lead.
static_assert(kMaxTicketChunks + kMaxCompressLead <= FSZ_COMPRESS_SETS, "schedule limits");
#ifndef FSZ_COMPRESS_CTAS
#define FSZ_COMPRESS_CTAS 2
#endif
constexpr int kCtasPerSm = FSZ_COMPRESS_CTAS;
constexpr int kQuadElems = kQuadTiles * kTile;     // 1024
constexpr int kQuadBytes = 4 * kQuadElems;         // 4096: a warp's staging buffer
constexpr int kMaxQuadOut = kQuadTiles * kMaxTileBytes;
// Ring bytes per compute warp. A run is contiguous: one that would run past the end
// starts at the ring's start instead, and the bytes it skips count as its own until it
// is placed.
constexpr int kRingAlloc = FSZ_RING_BYTES + kMaxQuadOut;
#ifndef FSZ_LOOKBACK_K
#define FSZ_LOOKBACK_K 2
#endif
constexpr int kLookbackPerLane = FSZ_LOOKBACK_K;   // lookback window: 32 K flags
constexpr uint32_t kNone = 0xffffffffu;
// Polling intervals of waits that sleep between tests (ns): the host warp, the resolver
// waiting for a chunk to be sized, the compute warps waiting for a ticket or ring space.
#ifndef FSZ_HOST_SLEEP_NS
#define FSZ_HOST_SLEEP_NS 100
#endif
#ifndef FSZ_RESOLVER_SLEEP_NS
#define FSZ_RESOLVER_SLEEP_NS 200
#endif
#ifndef FSZ_COMPUTE_SLEEP_NS
#define FSZ_COMPUTE_SLEEP_NS 100
#endif
constexpr uint32_t kHostSleepNs = FSZ_HOST_SLEEP_NS;
constexpr uint32_t kResolverSleepNs = FSZ_RESOLVER_SLEEP_NS;
constexpr uint32_t kComputeSleepNs = FSZ_COMPUTE_SLEEP_NS;
static_assert(kCChunkTiles == kWarps * kQuadTiles, "a chunk is one quad per compute warp");
static_assert(kRingAlloc >= 2 * kMaxQuadOut, "worst-case quads fit the ring");
static_assert(kRingAlloc % 16 == 0 && kQuadBytes % 1024 == 0, "alignment of the buffers");
static_assert(kWarps <= 32, "one lane per quad in the chunk scan");

// A chunk's parameters, read once from the field record by the host warp and kept in the
// chunk's slot until the chunk is placed.
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

struct __align__(1024) CompressSmem {
  float stage[kWarps][kQuadElems];                // per-warp staging (swizzled pieces)
  uint8_t ring[kWarps][kRingAlloc];               // encoded quads awaiting their offset
  ChunkInfo meta[kSets];
  uint64_t set_excl[kSets];                       // a resolved chunk's exclusive offset
  uint32_t qlen[kSets][kWarps];                   // each warp's quad run: bytes,
  uint32_t qoff[kSets][kWarps];                   // ... offset inside the chunk,
  uint32_t qpos[kSets][kWarps];                   // ... position in the warp's ring,
  uint32_t qalloc[kSets][kWarps];                 // ... ring bytes it holds (run + skipped end)
  uint32_t set_tot[kSets];
  uint32_t done_cnt[kSets];
  uint32_t ring_tail[kWarps];                     // ring bytes given back, per compute warp
  uint64_t info[kSets], computed[kSets], encoded[kSets], resolved[kSets], started[kSets];
};

static_assert(sizeof(CompressSmem) <= 227 * 1024, "shared memory of one CTA");

// Eq. 3: S_b = 0 for r_b = 0, else 4 + 4 r_b.
__device__ __forceinline__ uint32_t block_cost(int R) {
  return (uint32_t(R) + (R != 0 ? 1u : 0u)) << 2;
}

// Bit length of x (Sec. 4.1.2: r_b = ceil(log2(max |l| + 1))).
__device__ __forceinline__ int bitlen(uint32_t x) { return 32 - __clz(int(x)); }

// The sign-magnitude word v = 2|l| + sign by multiply-adds, l (2 - 4s) + s with s the sign
// bit: bit 0 is the sign-map bit, bit k + 1 magnitude bit-plane k (Sec. 4.3).
__device__ __forceinline__ uint32_t sign_mag_fma(int l) {
  const int sg = int(uint32_t(l) >> 31);
  return uint32_t(mad_s32(l, mad_s32(sg, -4, 2), sg));
}
__device__ __forceinline__ uint32_t sign_mag(int l) {
  return (uabs32(l) << 1) | (uint32_t(l) >> 31);
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
// Copies the first `bytes` (0..16) of the piece and zero-fills the rest of it.
__device__ __forceinline__ void cp_async16_fill(uint32_t dst, const void* src, uint32_t bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

__device__ __forceinline__ void sts32(uint32_t addr, uint32_t v) {
  asm volatile("st.shared.b32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}
__device__ __forceinline__ uint32_t lds32(uint32_t addr) {
  uint32_t v;
  asm volatile("ld.shared.b32 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
  return v;
}

__device__ __forceinline__ void st_release_cta(uint32_t* p, uint32_t v) {
  asm volatile("st.release.cta.shared::cta.u32 [%0], %1;" ::"r"(smem_u32(p)), "r"(v) : "memory");
}
__device__ __forceinline__ uint32_t ld_acquire_cta(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.cta.shared::cta.u32 %0, [%1];" : "=r"(v) : "r"(smem_u32(p)) : "memory");
  return v;
}

__device__ __forceinline__ float4 lds128(uint32_t addr) {
  float4 v;
  asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "r"(addr));
  return v;
}

// Staging layout of a quad (4 KiB): the 16-byte piece at quad offset o sits at
// o ^ (((o >> 7) & 7) << 4), so piece k of block g (128 bytes) lands in column k ^ g of the
// block's row and the 8 lanes reading piece k of blocks 0..7 hit 8 different bank groups.
//
// Issues the cp.async pieces of this warp's quad of a chunk: lane L copies pieces
// 32 j + L, j = 0..7 (each instruction of the warp reads 512 consecutive bytes). `qv` is
// the quad's count of valid elements (1..1024); pieces past it are zero-filled and read
// nothing beyond the field (their source operand is `safe`, the chunk's first element).
__device__ __forceinline__ void issue_quad(uint32_t buf, const float* src, uint32_t qv, int lane,
                                           const float* safe) {
  // piece 32 j + L is at byte 512 j + 16 L; its block is (4 j + (L >> 3)) & 7
  const uint32_t pe = uint32_t(16 * lane) ^ (uint32_t(lane >> 3) << 4);
  const uint32_t po = pe ^ 64u;
  const char* s = reinterpret_cast<const char*>(src) + 16 * lane;
  if (qv == uint32_t(kQuadElems)) {
#pragma unroll
    for (int j = 0; j < 8; ++j) cp_async16(buf + 512 * j + ((j & 1) ? po : pe), s + 512 * j);
  } else {
    const uint32_t vb = 4 * qv;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const uint32_t o = uint32_t(512 * j + 16 * lane);
      const uint32_t nb = o >= vb ? 0u : min(16u, vb - o);
      cp_async16_fill(buf + 512 * j + ((j & 1) ? po : pe),
                      nb ? static_cast<const void*>(s + 512 * j) : static_cast<const void*>(safe), nb);
    }
  }
  cp_async_commit();
}

// One byte-slice (bit-planes 8c .. 8c + 7) of a block's sign-magnitude words v[0..31] as the
// 8 stream words of those planes (Sec. 4.3: element j at bit 31 - j, most significant byte
// first, so stored little-endian element j sits at bit 8 (j >> 3) + 7 - (j & 7)).
// X[k] gathers byte c of elements 7 - k, 15 - k, 23 - k, 31 - k: bit 8 m + i of X[k] is bit
// i of element 8 m + 7 - k. Three delta swaps between register pairs (k, k ^ 2^t) exchange
// bit t of the register index with bit t of the bit index i, after which register b holds
// bit b of element 8 m + 7 - k at bit 8 m + k: the stream word of plane 8c + b.
template <int c>
__device__ __forceinline__ void planes8(const uint32_t (&v)[32], uint32_t (&X)[8]) {
  constexpr uint32_t sel = uint32_t(c) | (uint32_t(4 + c) << 4);
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const uint32_t a = __byte_perm(v[7 - k], v[15 - k], sel);
    const uint32_t b = __byte_perm(v[23 - k], v[31 - k], sel);
    X[k] = __byte_perm(a, b, 0x5410);
  }
  swap_planes(X);
}

// Compresses one quad (4 tiles) with one warp. Lane L = 8 tq + g holds block g of tile tq
// (elements 32 g .. 32 g + 31 of the tile) in d. `live`: the lane's tile exists. Writes the
// tile's rate-header byte of block g to hdr (the quad's 32 header bytes are consecutive),
// and returns this lane's block as (byte offset of its data inside the quad's run, word
// count), with the quad's run length in *qlen; the words go to ring + offset by encode().
// Switched-off features arrive as `restart` (this lane starts from zero predecessors: the
// tile's first block, and every block without the cross-block state) and as penalties
// pen2, pen3 (2^16 for the second-order and the centred variants when off). With kGiven
// the four tile costs come from `given` (this lane's tile, stride gT between variants): the
// multipass evaluation's encoding pass; they are equal, so the stream is the same.
struct QuadPlan {
  uint32_t v[32];   // sign-magnitude words of the selected variant
  uint32_t off;     // byte offset of this lane's block data in the quad's run
  int nw;           // the block's words (sign map + planes), 0 for rate 0 or a dead tile
  uint32_t mu_off;  // byte offset of the tile's mean slot (lane g = 0 of a centred tile)
  bool mu_slot;
  int mu;
  uint32_t qlen;    // the quad's run length (uniform)
  int Rmax;         // largest live rate of the quad (uniform)
};

template <bool kGiven>
__device__ __forceinline__ void plan_quad(const float (&d)[32], const float r, const int lane,
                                          const bool live, const bool restart, const int pen2,
                                          const int pen3, const uint32_t* __restrict__ given,
                                          const uint64_t gT, uint8_t* __restrict__ hdr,
                                          QuadPlan& P) {
  const int g = lane & 7;
  // Tile sum for centring (Sec. 4.2.2, variant 3) in the fixed order: the sums of elements
  // 8j..8j+7 left to right (four runs per lane: runs 4g .. 4g + 3), then a butterfly over
  // the run index by 16, 8, 4 (lanes xor 4, 2, 1 within the tile's 8 lanes), 2 and 1
  // (in-lane). Float addition is commutative, so both partners of a step get equal sums.
  float R[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    float acc = d[8 * m];
#pragma unroll
    for (int i = 1; i < 8; ++i) acc = __fadd_rn(acc, d[8 * m + i]);
    R[m] = acc;
  }
#pragma unroll
  for (int o = 4; o >= 1; o >>= 1)
#pragma unroll
    for (int m = 0; m < 4; ++m) R[m] = __fadd_rn(R[m], __shfl_xor_sync(FULL, R[m], o));
  const float S = __fadd_rn(__fadd_rn(R[0], R[2]), __fadd_rn(R[1], R[3]));

  // Step 1, quantize (Sec. 4.2.2): t = fl(d r) then the nearest integer, ties to even. Y
  // holds q + bits(M); differences of Y are differences of q.
  int Y[32];
#pragma unroll
  for (int i = 0; i < 32; ++i) Y[i] = __float_as_int(__fadd_rn(__fmul_rn(d[i], r), kMagic));
  const int mu =
      __float_as_int(__fadd_rn(__fmul_rn(__fmul_rn(S, 0.00390625f), r), kMagic)) - kMagicBits;

  // Residuals with the state carried across block boundaries (Eq. 2); the tile's first
  // predecessors are zero. LZ2 as the difference of LZ1 residuals:
  // l2_i = (q_i - q_{i-1}) - (q_{i-1} - q_{i-2}).
  int prevY = __shfl_up_sync(FULL, Y[31], 1, 8);
  int prevL = __shfl_up_sync(FULL, Y[31] - Y[30], 1, 8);
  if (restart) {
    prevY = kMagicBits;
    prevL = 0;
  }
  const int l1_0 = Y[0] - prevY;
  const int l2_0 = l1_0 - prevL;
  const int l1_1 = Y[1] - Y[0];
  const int l2_1 = l1_1 - l1_0;
  // Block maxima as ORs (same bit length). rest* leave out the tile's first residual(s),
  // the only ones centring changes (Eq. 4).
  // (four partial ORs each, so that the chains are short)
  uint32_t o1[4] = {uabs32(l1_1), 0u, 0u, 0u}, o2[4] = {0u, 0u, 0u, 0u};
  int lp = l1_1;
#pragma unroll
  for (int i = 2; i < 32; ++i) {
    const int l1 = Y[i] - Y[i - 1];
    o1[i & 3] |= uabs32(l1);
    o2[i & 3] |= uabs32(l1 - lp);
    lp = l1;
  }
  const uint32_t rest1 = (o1[0] | o1[1]) | (o1[2] | o1[3]);
  const uint32_t rest2 = (o2[0] | o2[1]) | (o2[2] | o2[3]);
  const int R1 = bitlen(rest1 | uabs32(l1_0));
  const int R2 = bitlen(rest2 | uabs32(l2_0) | uabs32(l2_1));
  // Centred block-0 rates (lane g = 0): l1c_0 = q_0 - mu, l2c_0 = q_0 - mu,
  // l2c_1 = q_1 - 2 q_0 + mu = l2_1 + mu; the rest of block 0 is unchanged (Eq. 4).
  const int q0 = Y[0] - kMagicBits;
  const uint32_t c10 = uabs32(q0 - mu);
  const uint32_t c21 = uabs32(l2_1 + mu);
  const int R1c = bitlen(rest1 | c10);
  const int R2c = bitlen(rest2 | c10 | c21);

  // Tile costs (Eq. 3; variants 3 and 4 pay 4 bytes for mu): sums over the tile's 8 lanes
  // of the block costs as 16-bit halves; centring changes block 0 only.
  const uint32_t S1 = block_cost(R1), S2 = block_cost(R2);
  uint32_t A = S1 | (S2 << 16);
  uint32_t B = g == 0 ? (block_cost(R1c) | (block_cost(R2c) << 16)) : A;
#pragma unroll
  for (int o = 1; o <= 4; o <<= 1) {
    A += __shfl_xor_sync(FULL, A, o);
    B += __shfl_xor_sync(FULL, B, o);
  }
  int C1 = int(A & 0xffffu), C2 = int(A >> 16);
  int C3 = 4 + int(B & 0xffffu) + pen3;
  int C4 = 4 + int(B >> 16) + pen2 + pen3;
  if constexpr (kGiven) {
    C1 = int(given[0]);
    C2 = int(given[gT]);
    C3 = int(given[2 * gT]);
    C4 = int(given[3 * gT]);
  }
  // Step 3: first strict minimum in the order LZ1, LZ2, LZ1c, LZ2c.
  int v = 0, best = C1;
  if (C2 + pen2 < best) { v = 1; best = C2; }
  if (C3 < best) { v = 2; best = C3; }
  if (C4 < best) { v = 3; best = C4; }
  const bool second = (v & 1) != 0, centred = v >= 2;

  int Rg = second ? R2 : R1;
  if (g == 0 && centred) Rg = second ? R2c : R1c;
  // Rate header (Sec. 3.1): block 0 carries bit 7 = order 2, bit 6 = centred.
  if (live) {
    uint32_t hb = uint32_t(Rg);
    if (g == 0) hb |= (second ? 0x80u : 0u) | (centred ? 0x40u : 0u);
    hdr[lane] = uint8_t(hb);
  }

  // Offsets: one scan over the quad's 32 blocks in stream order of the lane's bytes (its
  // block's data, preceded in block 0 of a centred tile by the 4-byte mean).
  const bool slot = live && centred && g == 0;
  const uint32_t mine = live ? block_cost(Rg) + (slot ? 4u : 0u) : 0u;
  uint32_t inc = mine;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) inc = scan_step_up<32>(inc, o);
  const uint32_t excl = inc - mine;
  P.qlen = __shfl_sync(FULL, inc, 31);
  P.mu_slot = slot;
  P.mu_off = excl;
  P.mu = mu;
  P.off = excl + (slot ? 4u : 0u);
  P.nw = live && Rg > 0 ? Rg + 1 : 0;
  P.Rmax = int(__reduce_max_sync(FULL, live ? uint32_t(Rg) : 0u));

  // Step 5: residuals of the selected variant as sign-magnitude words, in place over Y from
  // the top (v_i needs Y_i, Y_{i-1}, Y_{i-2}). The selected residual is l1_i + m l1_{i-1}
  // with m = 0 (LZ1) or -1 (LZ2).
  const int m = second ? -1 : 0;
  int up = Y[31] - Y[30];
#pragma unroll
  for (int i = 31; i >= 2; --i) {
    const int dn = Y[i - 1] - Y[i - 2];
    P.v[i] = sign_mag_fma(mad_s32(dn, m, up));
    up = dn;
  }
  P.v[1] = sign_mag_fma(mad_s32(l1_0, m, l1_1));
  P.v[0] = sign_mag_fma(mad_s32(prevL, m, l1_0));
  if (g == 0 && centred) {
    P.v[0] = sign_mag(q0 - mu);
    if (second) P.v[1] = sign_mag(l2_1 + mu);
  }
}

// Writes this lane's block words (sign map, then bit-planes from the least significant) at
// the shared-memory address blk, for the quad's byte-slices that any lane needs.
__device__ __forceinline__ void encode_block(const QuadPlan& P, uint32_t blk) {
  uint32_t X[8];
  if (P.Rmax > 0) {
    planes8<0>(P.v, X);
#pragma unroll
    for (int b = 0; b < 8; ++b)
      if (b < P.nw) sts32(blk + 4 * b, X[b]);
  }
  if (P.Rmax >= 8) {
    planes8<1>(P.v, X);
#pragma unroll
    for (int b = 0; b < 8; ++b)
      if (8 + b < P.nw) sts32(blk + 32 + 4 * b, X[b]);
  }
  if (P.Rmax >= 16) {
    planes8<2>(P.v, X);
#pragma unroll
    for (int b = 0; b < 8; ++b)
      if (16 + b < P.nw) sts32(blk + 64 + 4 * b, X[b]);
  }
}

// kGiven: the multipass evaluation's encoding pass (selection from a.given_costs).
// kFeat: fields' switched-off features honoured; without it the full method is compiled
// with none of that handling.
template <bool kGiven, bool kFeat>
__global__ void __launch_bounds__(kThreads, kCtasPerSm) fsz_compress_kernel(KernelArgs a) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  CompressSmem& S = *reinterpret_cast<CompressSmem*>(smem_raw);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint64_t total = a.ctrl->total_chunks;
  // mbarrier waits outlast the longest lookback wait, so a lookback that runs out is
  // reported as such rather than as a stalled pipeline.
  const uint64_t wait_ns = 4 * a.timeout_ns;

  if (tid == 0) {
    for (int k = 0; k < kSets; ++k) {
      mbar_init(&S.info[k], 1);
      mbar_init(&S.computed[k], 1);
      mbar_init(&S.encoded[k], kWarps);
      mbar_init(&S.resolved[k], 1);
      mbar_init(&S.started[k], 1);
      S.done_cnt[k] = 0;
    }
    for (int w = 0; w < kWarps; ++w) S.ring_tail[w] = 0;
    fence_mbar_init();
  }
  __syncthreads();

  if (warp == kHostWarp) {
    // ---------------------------------------------------------------- host
    // Tickets and placement, polled in turn:
    //  * the ticket of chunk seq is taken once the compute warps have begun chunk
    //    seq - lead (so the chunk order across the grid stays close to the ticket
    //    order) and its slot is free (chunk seq - kSets placed); lane 0 reads the field
    //    record and leaves the chunk's parameters in the slot;
    //  * chunk p is placed, in this CTA's order, once its offset is resolved and every
    //    compute warp has encoded its quad: each warp's run is copied from its ring to the
    //    stream and the ring space is given back.
    const bool single = a.ctrl->nfields == 1;
    const uint32_t group = launch_ticket_chunks(a.ticket_chunks, a.min_tickets, total, gridDim.x);
    const uint32_t lead = a.ticket_lead;
    uint32_t seq_t = 0, p = 0, end_seq = kNone;
    uint64_t deadline = globaltimer_ns() + wait_ns;
    for (;;) {
      bool progress = false;
      if (end_seq == kNone && seq_t + group - p <= uint32_t(kSets) &&
          (seq_t < lead || mbar_test(&S.started[(seq_t - lead) % kSets], ((seq_t - lead) / kSets) & 1u))) {
        uint32_t t = 0;
        if (lane == 0) t = atomicAdd(&a.ctrl->ticket, 1u);
        t = __shfl_sync(FULL, t, 0);
        for (uint32_t g = 0; g < group && end_seq == kNone; ++g) {
          const int b = int((seq_t + g) % kSets);
          const uint32_t c = t * group + g;
          if (lane == 0) {
            ChunkInfo& ci = S.meta[b];
            if (c >= total) {
              ci.chunk = kNone;
            } else {
              FieldInfo* fi = single ? a.fields : a.fields + a.chunk_field[c];
              const uint64_t first = fi->chunk_first;
              const uint64_t lc = c - first;
              const uint64_t tile0 = lc * kCChunkTiles;
              const uint64_t e0 = tile0 * kTile;
              const uint64_t T = fi->T;
              ci.chunk = c;
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
            }
            mbar_arrive(&S.info[b]);
          }
          if (c >= total) end_seq = seq_t + g;
        }
        seq_t = end_seq != kNone ? end_seq + 1 : seq_t + group;
        progress = true;
      }
      if (p < seq_t && p != end_seq) {
        const int b = int(p % kSets);
        const uint32_t par = (p / kSets) & 1u;
        if (mbar_test(&S.resolved[b], par) && mbar_test(&S.encoded[b], par)) {
          const ChunkInfo& ci = S.meta[b];
          if ((ci.flags & (kInfoOk | kInfoSkip)) == kInfoOk) {
            const uint64_t excl = S.set_excl[b];
            const uint32_t tot = S.set_tot[b];
            if (ci.data_base + excl + tot > ci.cap) {
              if (lane == 0) set_error(a.ctrl, ci.fi, FSZ_ERR_CAPACITY);
            } else {
              uint8_t* const base = ci.out + ci.data_base + excl;
              for (int w = kResolverRuns; w < kWarps; ++w) {
                const uint32_t nw = S.qlen[b][w] >> 2;
                const uint32_t src = smem_u32(S.ring[w]) + S.qpos[b][w];
                uint32_t* dst = reinterpret_cast<uint32_t*>(base + S.qoff[b][w]);
                for (uint32_t q0 = 0; q0 < nw; q0 += 128) {  // 4 words per lane in flight
                  uint32_t v[4];
#pragma unroll
                  for (int k = 0; k < 4; ++k) {
                    const uint32_t q = q0 + 32 * k + lane;
                    if (q < nw) v[k] = lds32(src + 4 * q);
                  }
#pragma unroll
                  for (int k = 0; k < 4; ++k) {
                    const uint32_t q = q0 + 32 * k + lane;
                    if (q < nw) dst[q] = v[k];
                  }
                }
              }
              if (lane == 0 && (ci.flags & kInfoLast)) write_preamble(ci.fi, excl + tot);
            }
          }
          // the runs are read: their ring space goes back to the compute warps
          __syncwarp();
          if (lane >= kResolverRuns && lane < kWarps) {
            __threadfence_block();
            st_release_cta(&S.ring_tail[lane], S.ring_tail[lane] + S.qalloc[b][lane]);
          }
          __syncwarp();
          ++p;
          progress = true;
        }
      }
      if (end_seq != kNone && p == end_seq) break;
      if (progress) {
        deadline = globaltimer_ns() + wait_ns;
      } else {
        __nanosleep(kHostSleepNs);
        if (globaltimer_ns() > deadline) {
          if (lane == 0) set_error(a.ctrl, nullptr, FSZ_ERR_TIMEOUT);
          break;
        }
      }
    }
    return;
  }

  if (warp == kResolverWarp) {
    // ---------------------------------------------------------------- resolver
    // Step 4 at device level, one chunk after another in this CTA's ticket order, as soon
    // as the chunk's aggregate is out: the compute warps keep encoding meanwhile.
    uint32_t prev_c = kNone, prev_tot = 0;
    const FieldInfo* prev_fi = nullptr;
    uint64_t prev_excl = 0;
    bool prev_held = true;  // the previous chunk's flags are held back (test hook)
    for (uint32_t seq = 0;; ++seq) {
      const int b = int(seq % kSets);
      if (!mbar_wait_idle(&S.computed[b], (seq / kSets) & 1u, wait_ns, kResolverSleepNs)) {
        if (lane == 0) set_error(a.ctrl, nullptr, FSZ_ERR_TIMEOUT);
        return;
      }
      const ChunkInfo& ci = S.meta[b];
      const uint32_t c = ci.chunk;
      if (c == kNone) return;
      const uint32_t flags = ci.flags;
      uint64_t excl = 0;
      if (!(flags & kInfoFirst)) {
        bool to = false;
        if (c == prev_c + 1 && ci.fi == prev_fi && !prev_held)
          excl = prev_excl + prev_tot;  // the CTA's previous chunk is the one before
        else
          excl = lookback<kLookbackPerLane>(a.flags, int64_t(c), int64_t(ci.chunk_first),
                                            globaltimer_ns() + a.timeout_ns, &to);
        if (lane == 0) {
          if (to) set_error(a.ctrl, ci.fi, FSZ_ERR_TIMEOUT);
          if (!(flags & kInfoSkip))
            st_flag(a.flags + uint64_t(c) * kFlagStride, kFlagIncl | (excl + S.set_tot[b]));
        }
      }
      prev_c = c;
      prev_fi = ci.fi;
      prev_excl = excl;
      prev_tot = S.set_tot[b];
      prev_held = (flags & kInfoSkip) != 0;
      if constexpr (kResolverRuns > 0) {
        // copy this warp's share of the runs once they are all encoded (the host copies
        // the rest after the chunk is handed over)
        if (!mbar_wait_idle(&S.encoded[b], (seq / kSets) & 1u, wait_ns, kResolverSleepNs)) {
          if (lane == 0) set_error(a.ctrl, nullptr, FSZ_ERR_TIMEOUT);
          return;
        }
        const uint32_t tot = S.set_tot[b];
        if ((flags & (kInfoOk | kInfoSkip)) == kInfoOk && ci.data_base + excl + tot <= ci.cap) {
          uint8_t* const base = ci.out + ci.data_base + excl;
          for (int w = 0; w < kResolverRuns; ++w) {
            const uint32_t nw = S.qlen[b][w] >> 2;
            const uint32_t src = smem_u32(S.ring[w]) + S.qpos[b][w];
            uint32_t* dst = reinterpret_cast<uint32_t*>(base + S.qoff[b][w]);
            for (uint32_t q0 = 0; q0 < nw; q0 += 128) {
              uint32_t v[4];
#pragma unroll
              for (int k = 0; k < 4; ++k) {
                const uint32_t q = q0 + 32 * k + lane;
                if (q < nw) v[k] = lds32(src + 4 * q);
              }
#pragma unroll
              for (int k = 0; k < 4; ++k) {
                const uint32_t q = q0 + 32 * k + lane;
                if (q < nw) dst[q] = v[k];
              }
            }
          }
        }
        __syncwarp();
        if (lane < kResolverRuns) {
          __threadfence_block();
          st_release_cta(&S.ring_tail[lane], S.ring_tail[lane] + S.qalloc[b][lane]);
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
  const uint32_t buf = smem_u32(S.stage[warp]);
  const uint32_t ring_u32 = smem_u32(S.ring[warp]);
  uint32_t head = 0;  // bytes this warp has written to its ring (warp-uniform, wrapping)
  uint32_t pos = 0;   // ... the position in the ring where the next run goes

  // The quad of a chunk that this warp loads: valid elements (0: nothing to load).
  auto quad_valid = [&](const ChunkInfo& ci) -> uint32_t {
    if (ci.chunk == kNone || !(ci.flags & kInfoOk)) return 0u;
    const int e0 = kQuadElems * warp;
    return ci.cnt > uint32_t(e0) ? min(ci.cnt - uint32_t(e0), uint32_t(kQuadElems)) : 0u;
  };

  bool ok_run = mbar_wait_idle(&S.info[0], 0u, wait_ns, kComputeSleepNs);
  if (!ok_run) {
    if (lane == 0) set_error(a.ctrl, nullptr, FSZ_ERR_TIMEOUT);
  } else {
    const uint32_t qv0 = quad_valid(S.meta[0]);
    if (qv0) issue_quad(buf, S.meta[0].in + kQuadElems * warp, qv0, lane, S.meta[0].in);
  }
  for (uint32_t u = 0; ok_run; ++u) {
    const int b = int(u % kSets);
    if (warp == 0 && lane == 0) mbar_arrive(&S.started[b]);  // step u begins
    const ChunkInfo& ci = S.meta[b];
    const uint32_t c = ci.chunk;
    const bool end = (c == kNone);
    const uint32_t qv = quad_valid(ci);
    const uint32_t flags = end ? 0u : ci.flags;
    float d[32];
    if (qv) {
      cp_async_wait_all();
      __syncwarp();
      // lane L reads block g = L & 7 of tile L >> 3: piece k at column k ^ g of its row
      const uint32_t row = buf + uint32_t(lane) * 128u;
      const uint32_t base = row | (uint32_t(lane & 7) << 4);
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const float4 x = lds128(base ^ uint32_t(k << 4));
        d[4 * k] = x.x; d[4 * k + 1] = x.y; d[4 * k + 2] = x.z; d[4 * k + 3] = x.w;
      }
    } else {
#pragma unroll
      for (int i = 0; i < 32; ++i) d[i] = 0.0f;
    }
    uint32_t qlen = 0;
    QuadPlan P;
    const int qt0 = kQuadTiles * warp;            // the quad's first tile in the chunk
    const bool any = !end && (flags & kInfoOk) && qt0 < int(ci.ntiles);
    if (any) {
      const int t = qt0 + (lane >> 3);
      const bool live = t < int(ci.ntiles);
      const uint32_t foff = kFeat ? ci.off : 0u;
      const bool restart = (lane & 7) == 0 || (foff & kOffCross);
      const int pen2 = (foff & kOffLz2) ? 0x10000 : 0;
      const int pen3 = (foff & kOffCenter) ? 0x10000 : 0;
      uint8_t* hdr = ci.out + 64 + 8 * (ci.tile0 + uint64_t(qt0));
      // (a lane of a missing tile reads the quad's first tile's given costs)
      plan_quad<kGiven>(d, ci.r, lane, live, restart, pen2, pen3,
                        a.given_costs + ci.tile0 + uint64_t(live ? t : qt0), a.given_T, hdr, P);
      qlen = P.qlen;
    }
    // sized: the last warp through the chunk scans the quads' sizes and publishes its
    // aggregate (step 4, warp level), before the quads are encoded; the end marker tells
    // the resolver that the CTA's chunks have run out
    if (lane == 0) S.qlen[b][warp] = qlen;
    uint32_t last = 0;
    if (lane == 0) {
      __threadfence_block();
      last = atomicAdd(&S.done_cnt[b], 1u) == uint32_t(kWarps - 1) ? 1u : 0u;
      __threadfence_block();
    }
    last = __shfl_sync(FULL, last, 0);
    if (last) {
      if (!end) {
        const uint32_t ql = lane < kWarps ? S.qlen[b][lane] : 0u;
        uint32_t inc = ql;
#pragma unroll
        for (int o = 1; o < kWarps; o <<= 1) inc = scan_step_up<32>(inc, o);
        if (lane < kWarps) S.qoff[b][lane] = inc - ql;
        const uint32_t tot = __shfl_sync(FULL, inc, kWarps - 1);
        if (lane == 0) {
          S.set_tot[b] = tot;
          if (!(flags & kInfoSkip))
            st_flag(a.flags + uint64_t(c) * kFlagStride,
                    ((flags & kInfoFirst) ? kFlagIncl : kFlagAgg) | tot);
        }
      }
      __syncwarp();
      if (lane == 0) {
        S.done_cnt[b] = 0;
        mbar_arrive(&S.computed[b]);
      }
    }
    if (end) break;
    // The next chunk's pieces go into the same buffer once every lane has its values.
    {
      const int b1 = int((u + 1) % kSets);
      if (!mbar_wait_idle(&S.info[b1], ((u + 1) / kSets) & 1u, wait_ns, kComputeSleepNs)) {
        if (lane == 0) set_error(a.ctrl, nullptr, FSZ_ERR_TIMEOUT);
        ok_run = false;
      } else {
        __syncwarp();  // every lane's loads of this buffer are done
        const ChunkInfo& cn = S.meta[b1];
        const uint32_t qv1 = quad_valid(cn);
        if (qv1) issue_quad(buf, cn.in + kQuadElems * warp, qv1, lane, cn.in);
      }
    }
    // room for the run in the ring (logical bytes), given back by the host as it places
    // the run's place: contiguous, from the ring's start if it would run past the end
    uint32_t skip = 0;
    if (pos + qlen > uint32_t(kRingAlloc)) {
      skip = uint32_t(kRingAlloc) - pos;
      pos = 0;
    }
    const uint32_t alloc = skip + qlen;  // (pos stays head mod kRingAlloc)
    if (any && uint32_t(kRingAlloc) - (head - ld_acquire_cta(&S.ring_tail[warp])) < alloc) {
      const uint64_t deadline = globaltimer_ns() + wait_ns;
      while (uint32_t(kRingAlloc) - (head - ld_acquire_cta(&S.ring_tail[warp])) < alloc) {
        __nanosleep(kComputeSleepNs);
        if (globaltimer_ns() > deadline) {
          if (lane == 0) set_error(a.ctrl, nullptr, FSZ_ERR_TIMEOUT);
          ok_run = false;
          break;
        }
      }
    }
    if (any && ok_run) {
      const uint32_t run = ring_u32 + pos;
      if (P.mu_slot) sts32(run + P.mu_off, __float_as_uint(__int2float_rn(P.mu)));
      encode_block(P, run + P.off);
    }
    if (lane == 0) {
      S.qpos[b][warp] = pos;
      S.qalloc[b][warp] = alloc;
    }
    head += alloc;
    pos += qlen;
    __syncwarp();
    if (lane == 0) mbar_arrive(&S.encoded[b]);  // this warp's run of the chunk is in its ring
  }
  cp_async_wait_all();
}

}  // namespace

LaunchCfg compress_cfg() {
  static DeviceCfgCache cache;
  return cache.get([] {
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
  });
}

void launch_compress(const KernelArgs& args, cudaStream_t st, CompressKind kind) {
  const LaunchCfg c = compress_cfg();
  const int g = sched_grid(c, kSchedCompress);
  KernelArgs a = args;
  a.ticket_chunks = uint32_t(g_schedule.c_ticket_chunks);
  a.ticket_lead = uint32_t(g_schedule.c_ticket_lead);
  a.min_tickets = uint32_t(g_schedule.min_tickets);
  if (kind == kCompressFeatures)
    fsz_compress_kernel<false, true><<<g, kThreads, c.smem, st>>>(a);
  else if (kind == kCompressGiven)
    fsz_compress_kernel<true, false><<<g, kThreads, c.smem, st>>>(a);
  else
    fsz_compress_kernel<false, false><<<g, kThreads, c.smem, st>>>(a);
}

}  // namespace fsz
