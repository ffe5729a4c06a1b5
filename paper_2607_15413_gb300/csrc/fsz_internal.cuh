// Internal definitions shared by the FSZ CUDA kernels (sm_103a).
//
// Work decomposition (GB300 design, not the paper's): a persistent CTA takes chunks of
// tiles by an atomic ticket, stages them in shared memory with 1-D TMA bulk copies
// (mbarrier-tracked) and gives each warp one 256-element tile at a time. Lane j of the
// warp owns the 8 consecutive elements 8j..8j+7, so the 4 lanes 4g..4g+3 hold block g
// (Sec. 3.1: a tile is 8 blocks of 32 elements). Residual chains stay in registers; a
// shuffle carries the state across lane and block boundaries.
#pragma once

#include <cstdint>
#include <mutex>
#include <cuda_runtime.h>

#include "../../include/fsz.h"

namespace fsz {

constexpr int kTile = 256;
constexpr int kMaxTileBytes = 772;    // 8 * (4 + 4 * 23) + 4, Eq. 3 with rate <= 23
constexpr int kMaxDecTileBytes = 1028;  // any header-valid tile: 8 * (4 + 4 * 31) + 4
// The quantization margin eps = (3Q + 4) 2^-23 is capped at 2^-4 (first tier); fields that
// need more take the second tier, capped at 2^-1. Q bounds |q|; Q < 2^21 keeps every
// residual below 2^23 (rate <= 23) and every quantized value exact in the float32 rounding.
constexpr uint32_t kQmax1 = 174761;   // largest Q with (3Q + 4) 2^-23 <= 2^-4
constexpr uint32_t kQmax2 = 1398100;  // largest Q with (3Q + 4) 2^-23 <= 2^-1
constexpr int kMinChunkTiles = 16;    // smallest chunk any kernel uses (workspace sizing)
// Tiles per work item (one ticket, one lookback flag). Compression (and its value-range
// pass, which shares the chunk -> field table) uses chunks of one 4-tile quad per compute
// warp of a CTA: 8 warps, 32 tiles. Decompression stages a chunk's whole payload at once:
// 32 tiles too, one quad per decode warp.
#ifndef FSZ_CCHUNK_TILES
#define FSZ_CCHUNK_TILES 32
#endif
constexpr int kCChunkTiles = FSZ_CCHUNK_TILES;
constexpr int kCChunkElems = kCChunkTiles * kTile;
constexpr int kDChunkTiles = 32;
constexpr int kDChunkElems = kDChunkTiles * kTile;
static_assert(kCChunkTiles >= kMinChunkTiles && kDChunkTiles >= kMinChunkTiles, "workspace sizing");
constexpr uint64_t kMaxElems = uint64_t(1) << 40;
constexpr uint64_t kDefaultTimeoutNs = 2000000000ull;

// Adding 1.5 * 2^23 to a float t with |t| < 2^22 rounds it to the nearest integer, ties to
// even, and leaves that integer in the low mantissa bits: bits(t + M) - bits(M) = rint(t).
constexpr float kMagic = 12582912.0f;
constexpr int kMagicBits = 0x4B400000;

// Decoupled-lookback flag word (Sec. 4.4): 2-bit state and a 62-bit byte count.
constexpr uint64_t kFlagAgg = uint64_t(1) << 62;   // local sum available
constexpr uint64_t kFlagIncl = uint64_t(2) << 62;  // inclusive prefix available
constexpr uint64_t kFlagValue = (uint64_t(1) << 62) - 1;
// Words between consecutive chunks' flags in the workspace (1: packed).
#ifndef FSZ_FLAG_STRIDE
#define FSZ_FLAG_STRIDE 1
#endif
constexpr int kFlagStride = FSZ_FLAG_STRIDE;

// Per-field state in the workspace: descriptor, value-range accumulators, derived step.
struct alignas(16) FieldInfo {
  // compression descriptor
  const float* in;
  uint8_t* out;
  uint64_t cap;
  uint64_t* out_bytes;
  // decompression descriptor
  const uint8_t* sin;
  uint64_t in_bytes;
  float* dout;
  uint64_t data_bytes;
  // shape
  uint64_t n;
  uint64_t T;
  uint64_t dims[3];
  uint32_t ndim;
  uint32_t mode;
  double eb_req;
  // chunk range of this field in the global ticket order
  uint64_t chunk_first;
  uint64_t nchunks;
  // value range (ordered-integer keys; the minimum is kept as the max of ~key)
  uint32_t min_inv_key;
  uint32_t max_key;
  uint32_t max_abs_bits;  // max of (bits & 0x7fffffff): >= 0x7f800000 means non-finite
  uint32_t done_chunks;
  // quantization step (valid once status == 0 after the value-range pass)
  double eb;
  float e, s, r;
  uint32_t Q;
  uint32_t status;
  uint32_t features_off;  // method features switched off (kOff* bits; 0: the full method)
};

// Features a compression may switch off, for the ablation of Sec. 6.4: the state carried
// across block boundaries (off: every block restarts from zero predecessors), the centred
// variants, the second-order variants. Centring is defined on the carried state (Eq. 4),
// so switching the state off requires switching centring off. The preamble records the
// bits (u32 at byte 52).
constexpr uint32_t kOffCross = 1u, kOffCenter = 2u, kOffLz2 = 4u;
__host__ __device__ __forceinline__ bool features_valid(uint32_t off) {
  return (off & ~(kOffCross | kOffCenter | kOffLz2)) == 0 &&
         (!(off & kOffCross) || (off & kOffCenter));
}

struct alignas(64) Ctrl {
  uint32_t status;       // first device-detected error of the call
  uint32_t ticket;       // chunk ticket (compress / decompress)
  uint32_t nfields;
  uint32_t pad0;
  uint64_t total_chunks;
  uint64_t chunk_cap;    // chunk slots available in the workspace
  uint32_t plan_done;
  uint32_t pad1[7];
};

// Workspace layout: [Ctrl][FieldInfo x nfields][u32 chunk->field x cap][u64 flags x cap].
struct WsLayout {
  uint64_t fields_off, map_off, flags_off, bytes;
  uint64_t chunk_cap;
};

inline WsLayout ws_layout(uint64_t tiles_upper, uint32_t nfields) {
  WsLayout L;
  L.chunk_cap = (tiles_upper + kMinChunkTiles - 1) / kMinChunkTiles + nfields + 1;
  L.fields_off = 256;
  L.map_off = L.fields_off + uint64_t(nfields) * sizeof(FieldInfo);
  L.flags_off = (L.map_off + 4 * L.chunk_cap + 127) & ~uint64_t(127);
  L.bytes = L.flags_off + 8 * kFlagStride * L.chunk_cap;
  return L;
}

struct KernelArgs {
  Ctrl* ctrl;
  FieldInfo* fields;
  const uint32_t* chunk_field;
  uint64_t* flags;
  uint64_t skip_chunk;  // test hook: this chunk publishes no flag
  uint64_t timeout_ns;  // bound on every spin-wait
  // multipass compression only: the four variants' tile costs, variant-major (given_T
  // per variant), from which the encoding pass selects
  const uint32_t* given_costs = nullptr;
  uint64_t given_T = 0;
  // work assignment (from the schedule, set by the launch functions)
  uint32_t ticket_chunks = 1;  // consecutive chunks per ticket
  uint32_t ticket_lead = 1;    // compression: tickets taken ahead of the compute warps
  uint32_t records = 0;        // decompression: chunks in flight per CTA
  uint32_t min_tickets = 0;    // tickets per CTA below which a launch takes smaller ones
};

// Chunks per ticket for one launch: the schedule's, or fewer (down to 1) while the launch
// would hand out fewer than min_tickets tickets per CTA, so that a launch of few chunks
// still spreads them over the grid and balances its end (min_tickets 0: always the
// schedule's). Every CTA of the launch computes the same value.
__device__ __forceinline__ uint32_t launch_ticket_chunks(uint32_t want, uint32_t min_tickets,
                                                         uint64_t total_chunks, uint32_t ctas) {
  uint32_t g = want;
  while (g > 1 && total_chunks < uint64_t(ctas) * g * min_tickets) --g;
  return g;
}

// ------------------------------------------------------------------ device helpers

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Lookback flags carry their whole message (state and byte count) in one 64-bit word and
// guard no other data, so relaxed device-scope accesses are enough.
__device__ __forceinline__ uint64_t ld_flag(const uint64_t* p) {
  uint64_t v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_flag(uint64_t* p, uint64_t v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Adds to the transaction count of the current phase without arriving.
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// try_wait that may suspend the thread for up to ~1 ms while the phase is incomplete
// (instead of spinning): it returns as soon as the phase completes.
__device__ __forceinline__ bool mbar_try_wait_sleep(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity), "r"(1000000u)
      : "memory");
  return ok != 0;
}

// Non-blocking test of the phase with the given parity.
__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// try_wait that may suspend the thread for up to `hint_ns` while the phase is incomplete.
__device__ __forceinline__ bool mbar_try_wait_for(uint64_t* bar, uint32_t parity, uint32_t hint_ns) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity), "r"(hint_ns)
      : "memory");
  return ok != 0;
}

// Waits for the phase of `bar` with the given parity; false if `timeout_ns` ran out first.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint64_t timeout_ns) {
  if (mbar_try_wait_sleep(bar, parity)) return true;
  const uint64_t deadline = globaltimer_ns() + timeout_ns;
  for (;;) {
    if (mbar_try_wait_sleep(bar, parity)) return true;
    if (globaltimer_ns() > deadline) return false;
  }
}

// Waits for the phase of `bar` with the given parity, sleeping about sleep_ns between
// tests: for warps with nothing else to do, so that their polling takes few issue slots
// from the working warps of the SM. False if timeout_ns ran out first.
__device__ __forceinline__ bool mbar_wait_idle(uint64_t* bar, uint32_t parity, uint64_t timeout_ns,
                                               uint32_t sleep_ns) {
  if (mbar_test(bar, parity)) return true;
  const uint64_t deadline = globaltimer_ns() + timeout_ns;
  for (;;) {
    __nanosleep(sleep_ns);
    if (mbar_test(bar, parity)) return true;
    if (globaltimer_ns() > deadline) return false;
  }
}

// 1-D TMA bulk copy global -> shared (16-byte aligned ends, size a multiple of 16).
__device__ __forceinline__ void tma_load_1d(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// 1-D TMA bulk copy shared -> global, tracked by bulk groups.
__device__ __forceinline__ void tma_store_1d(void* dst, const void* src, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst),
               "r"(smem_u32(src)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void tma_store_commit() {
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
__device__ __forceinline__ void tma_store_wait_read_all() {
  asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}
__device__ __forceinline__ void tma_store_wait_all() {
  asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

__device__ __forceinline__ void set_error(Ctrl* ctrl, FieldInfo* fi, uint32_t code) {
  if (fi) atomicCAS(&fi->status, 0u, code);
  atomicCAS(&ctrl->status, 0u, code);
}

__device__ __forceinline__ uint32_t uabs32(int32_t v) {
  return v < 0 ? 0u - static_cast<uint32_t>(v) : static_cast<uint32_t>(v);
}

// a * b + c as an integer multiply-add. The kernels' integer-logic pipe is their busiest
// and the multiply-add pipe has room, so shifts and selections by a 0/-1 factor that sit
// on the hot path are written this way.
__device__ __forceinline__ int mad_s32(int a, int b, int c) {
  int d;
  asm("mad.lo.s32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
}

// x << k as a multiply.
__device__ __forceinline__ uint32_t shl_fma(uint32_t x, int k) {
  return uint32_t(mad_s32(int(x), 1 << k, 0));
}

// The bit-plane network of both kernels. X[k] (k = 0..7) holds 4 bytes, byte m of X[k]
// standing for bits 0..7 of some element e(m, k); three delta swaps between register
// pairs (k, k ^ 2^t), t = 0, 1, 2, exchange bit t of the register index k with bit t of
// the bit index inside each byte, after which X[b] bit 8m + k is bit b of e(m, k): eight
// bit-plane words. Each swap is its own inverse and the three act on disjoint index
// bits, so the same network takes the plane words back to the bytes. (Delta swaps as in
// H. S. Warren, Hacker's Delight, "Transposing a bit matrix", here across registers.)
__device__ __forceinline__ void swap_planes(uint32_t (&X)[8]) {
#pragma unroll
  for (int t = 0; t < 3; ++t) {
    const int s = 1 << t;
    const uint32_t M = t == 0 ? 0x55555555u : (t == 1 ? 0x33333333u : 0x0F0F0F0Fu);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      if (k & s) continue;
      const uint32_t a = X[k], b = X[k | s];
      // b keeps its bits whose index has bit t set and takes a's bits with it set, moved
      // down; a keeps its bits with it clear and takes b's bits with it clear, moved up.
      X[k | s] = (b & ~M) | ((a >> s) & M);
      X[k] = (a & M) | (shl_fma(b, s) & ~M);
    }
  }
}

// One step of an inclusive scan: v += v of lane - o, where that lane exists within the
// segment of `width` lanes. The shuffle's own in-range predicate guards the add, so no
// lane-index compare is needed.
template <int kWidth = 32>
__device__ __forceinline__ uint32_t scan_step_up(uint32_t v, int o) {
  asm("{\n\t.reg .pred p;\n\t.reg .b32 y;\n\t"
      "shfl.sync.up.b32 y|p, %0, %1, %2, 0xffffffff;\n\t"
      "@p add.u32 %0, %0, y;\n\t}"
      : "+r"(v)
      : "r"(o), "n"((32 - kWidth) << 8));
  return v;
}

__device__ __forceinline__ uint64_t warp_sum_u64(uint64_t v) {
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Exclusive prefix of the chunks before `gchunk` within its field (Sec. 4.4, device
// level: decoupled lookback over the 3-state flags). Called by one whole warp. A window
// holds the 32 * K nearest predecessors not yet summed, interleaved so that each load
// instruction of the warp reads 32 consecutive flags (lane L, slot k holds distance
// 32 k + L, nearest first). The warp waits only for flags that are still unpublished AND
// nearer than the nearest inclusive prefix; then it sums every flag up to that prefix, or
// the whole window and moves on.
//
// A lookback costs about one L2 round trip per window, and the nearest inclusive prefix
// trails a chunk by the chunks that finish during about one lookback, so the window must
// cover what the grid finishes in one round trip. Upgrading other chunks' aggregate flags
// to inclusive ones during a lookback was measured several times slower (store contention
// on the flag lines) and is not done.
//
// Every spin is bounded by `deadline`; a wait that runs out reads as a zero inclusive
// prefix and sets *timed_out (the caller records FSZ_ERR_TIMEOUT and still publishes, so
// no successor waits forever).
#ifndef FSZ_LOOKBACK_SLEEP_NS
#define FSZ_LOOKBACK_SLEEP_NS 64
#endif
constexpr uint32_t kLookbackSleepNs = FSZ_LOOKBACK_SLEEP_NS;  // between polls of a window

template <int K>
__device__ __forceinline__ uint64_t lookback(const uint64_t* flags, int64_t gchunk, int64_t first,
                                             uint64_t deadline, bool* timed_out) {
  constexpr uint32_t FULL = 0xffffffffu;
  constexpr uint32_t kNoIncl = 1u << 20, kNoWait = 1u << 21;  // beyond any window distance
  static_assert(K >= 1 && K <= 32, "per-lane state masks are 32 bits");
  const int lane = threadIdx.x & 31;
  uint64_t excl = 0;
  bool to = false;
  int64_t pos = gchunk - 1;
  while (pos >= first) {
    // Aggregates are a chunk's byte count (< 2^16), so a slot keeps its value's low 32 bits
    // and the lane keeps, as bit masks, which slots are unpublished or inclusive; the full
    // value of the lane's nearest inclusive prefix is kept aside.
    uint32_t lo[K];
    uint32_t wait_mask = 0, incl_mask = 0;
    uint64_t incl_val = 0;
    auto take = [&](int k, uint64_t f) {
      const uint32_t st = uint32_t(f >> 62);
      lo[k] = uint32_t(f);
      const uint32_t bit = 1u << k;
      wait_mask = (st == 0) ? (wait_mask | bit) : (wait_mask & ~bit);
      if (st >= 2) {
        if ((incl_mask & ((bit << 1) - 1u)) == 0) incl_val = f & kFlagValue;  // nearest so far
        incl_mask |= bit;
      }
    };
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int64_t idx = pos - (32 * k + lane);
      take(k, idx >= first ? ld_flag(flags + idx * kFlagStride) : kFlagIncl);  // before the field: 0
    }
    uint32_t d_incl;
    for (uint32_t spins = 0;; ++spins) {
      const uint32_t my_incl = incl_mask ? uint32_t(32 * (__ffs(incl_mask) - 1) + lane) : kNoIncl;
      const uint32_t my_wait = wait_mask ? uint32_t(32 * (__ffs(wait_mask) - 1) + lane) : kNoWait;
      d_incl = __reduce_min_sync(FULL, my_incl);
      const uint32_t d_wait = __reduce_min_sync(FULL, my_wait);
      if (d_wait > d_incl) break;  // everything up to the nearest inclusive prefix is in
      if ((spins & 15u) == 15u && globaltimer_ns() > deadline) {
        to = true;  // give up: unpublished flags read as a zero inclusive prefix
#pragma unroll
        for (int k = 0; k < K; ++k)
          if (wait_mask & (1u << k)) take(k, kFlagIncl);
        continue;
      }
      __nanosleep(kLookbackSleepNs);
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const uint32_t d = uint32_t(32 * k + lane);
        if ((wait_mask & (1u << k)) && d < d_incl)
          take(k, ld_flag(flags + (pos - int64_t(d)) * kFlagStride));
      }
    }
    // Sum the aggregates nearer than the nearest inclusive prefix, then that prefix.
    uint32_t agg = 0;
#pragma unroll
    for (int k = 0; k < K; ++k)
      if (uint32_t(32 * k + lane) < d_incl) agg += lo[k];
    uint64_t mine = agg;
    if (d_incl != kNoIncl && uint32_t(lane) == (d_incl & 31u)) mine += incl_val;
    excl += warp_sum_u64(mine);
    if (d_incl != kNoIncl) break;
    pos -= 32 * K;
  }
  *timed_out = __any_sync(FULL, to);
  return excl;
}

// ------------------------------------------------------------------ float keys

__device__ __forceinline__ uint32_t float_key(float x) {
  uint32_t u = __float_as_uint(x);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float key_float(uint32_t k) {
  uint32_t u = (k & 0x80000000u) ? (k & 0x7fffffffu) : ~k;
  return __uint_as_float(u);
}

// 64-byte preamble of this library's stream (little-endian; written once per field by the
// CTA that finishes the field's last chunk), and the field's total size.
__device__ __forceinline__ void write_preamble(FieldInfo* fi, uint64_t data_bytes) {
  uint32_t w[16];
  w[0] = 0x315A5346u;  // "FSZ1"
  w[1] = 1u | (fi->ndim << 16) | (fi->mode << 24);
  w[2] = uint32_t(fi->n);
  w[3] = uint32_t(fi->n >> 32);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const uint64_t dk = uint32_t(k) < fi->ndim ? fi->dims[k] : 0;
    w[4 + 2 * k] = uint32_t(dk);
    w[5 + 2 * k] = uint32_t(dk >> 32);
  }
  const uint64_t eb = static_cast<uint64_t>(__double_as_longlong(fi->eb_req));
  w[10] = uint32_t(eb);
  w[11] = uint32_t(eb >> 32);
  w[12] = __float_as_uint(fi->s);
  w[13] = fi->features_off;
  w[14] = uint32_t(data_bytes);
  w[15] = uint32_t(data_bytes >> 32);
  uint4* dst = reinterpret_cast<uint4*>(fi->out);
#pragma unroll
  for (int k = 0; k < 4; ++k) dst[k] = make_uint4(w[4 * k], w[4 * k + 1], w[4 * k + 2], w[4 * k + 3]);
  const uint64_t total = 64 + 8 * fi->T + data_bytes;
  fi->data_bytes = data_bytes;
  if (fi->out_bytes) *fi->out_bytes = total;
}

// ------------------------------------------------------------------ launch helpers (host)

struct LaunchCfg {
  int grid;  // SMs x CTAs that fit per SM
  int smem;
  int sms;
  int per;   // CTAs per SM that fit
};

// A kernel's launch configuration for each device the library is used on: `init` (which
// sets the kernel's attributes and reads its occupancy on the current device) runs once per
// device, on first use there; later calls on that device reuse the result.
constexpr int kMaxDevices = 64;
struct DeviceCfgCache {
  std::mutex mu;
  LaunchCfg cfg[kMaxDevices];
  bool ready[kMaxDevices] = {};
  template <typename F>
  LaunchCfg get(F init) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) dev = 0;
    std::lock_guard<std::mutex> lock(mu);
    if (!ready[dev]) {
      cfg[dev] = init();
      ready[dev] = true;
    }
    return cfg[dev];
  }
};

// Persistent CTAs per SM chosen by fsz_set_schedule (0 = as many as fit), per kernel.
enum { kSchedStats = 0, kSchedCompress = 1, kSchedDecompress = 2 };
// Work assignment of the persistent kernels (set through fsz_set_schedule*; none of it
// changes a stream): CTAs per SM (0 = as many as fit) and, for compression and
// decompression, how many consecutive 32-tile chunks one ticket hands a CTA. Compression
// also sets how many tickets ahead of its compute warps a CTA takes, decompression how
// many chunks a CTA holds between ticket and decode.
constexpr int kMaxTicketChunks = 4;
constexpr int kMaxCompressLead = 3;
constexpr int kMaxDecRecords = 16;
struct Schedule {
  int ctas[3];
  int c_ticket_chunks, c_ticket_lead;
  int d_ticket_chunks, d_records;
  int min_tickets;
};
extern Schedule g_schedule;
inline int sched_grid(const LaunchCfg& c, int which) {
  const int want = g_schedule.ctas[which];
  const int per = (want > 0 && want < c.per) ? want : c.per;
  return c.sms * (per > 0 ? per : 1);
}

LaunchCfg stats_cfg();
LaunchCfg compress_cfg();
LaunchCfg decompress_cfg();

void launch_stats(const KernelArgs& a, cudaStream_t st);
// Compression kernel instances (feature-toggle builds of one kernel): the full method;
// with switched-off features honoured per field (fsz_compress_features, batches); the
// multipass evaluation's encoding pass (selection from a.given_costs).
enum CompressKind { kCompressFull = 0, kCompressFeatures = 1, kCompressGiven = 2 };
void launch_compress(const KernelArgs& a, cudaStream_t st, CompressKind kind = kCompressFull);
// The multipass evaluation: one pass per variant writing its tile costs, then the
// compression kernel selecting from them (a.given_costs).
void launch_cost_pass(const KernelArgs& a, int variant, uint32_t* costs, cudaStream_t st);

// Decoder instances: the full method's; one that also decodes streams without the
// cross-block state; one for a pre-zeroed output that skips all-zero tiles.
enum DecompressKind { kDecompressFull = 0, kDecompressAny = 1, kDecompressPrezeroed = 2 };
void launch_decompress(const KernelArgs& a, cudaStream_t st,
                       DecompressKind kind = kDecompressFull);
// Single-field set-up (clears the control words, the field record and chunk_cap lookback
// flags of the workspace, then fills in the field): no memset of the workspace needed.
void launch_setup_compress(const KernelArgs& a, const FieldInfo& fi, uint64_t chunk_cap, cudaStream_t st);
void launch_setup_decompress(const KernelArgs& a, const uint8_t* in, uint64_t in_bytes, float* out,
                             uint64_t cap_elems, uint64_t chunk_cap, cudaStream_t st);
void launch_plan_compress(const KernelArgs& a, const fsz_cfield* d_fields, uint32_t nfields,
                          uint64_t chunk_cap, cudaStream_t st);
void launch_plan_decompress(const KernelArgs& a, const fsz_dfield* d_fields, uint32_t nfields,
                            uint64_t chunk_cap, cudaStream_t st);

}  // namespace fsz
