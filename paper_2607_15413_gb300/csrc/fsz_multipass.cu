// The multipass evaluation that Sec. 6.3 ("Single-pass evaluation benefit") compares the
// single-pass design against: each of the four variants is evaluated in its own pass over
// the field, writing every tile's cost (Eq. 3, plus the 4-byte mean for the centred
// variants). A fifth pass, the compression kernel, selects from the four cost arrays and
// encodes. Same streams as the single-pass path; four more reads of the input.
//
// One warp per tile, lane j holding elements 8j..8j+7 (zero past n). Plain coalesced
// 128-bit loads from global memory; the pass is a stream over the input.
#include "fsz_internal.cuh"

namespace fsz {

namespace {

constexpr int kCostThreads = 256;

template <int kVariant>
__global__ void __launch_bounds__(kCostThreads) fsz_cost_pass_kernel(KernelArgs a, uint32_t* costs) {
  constexpr uint32_t FULL = 0xffffffffu;
  constexpr bool kCentred = kVariant >= 2;
  constexpr bool kSecond = (kVariant & 1) != 0;
  const FieldInfo* fi = a.fields;
  if (fi->status != 0) return;  // the value-range pass refused the field
  const float r = fi->r;
  const uint64_t n = fi->n, T = fi->T;
  const float* in = fi->in;
  const int lane = threadIdx.x & 31;
  const uint64_t nwarps = (uint64_t(gridDim.x) * kCostThreads) >> 5;
  for (uint64_t t = (uint64_t(blockIdx.x) * kCostThreads + threadIdx.x) >> 5; t < T; t += nwarps) {
    const uint64_t e0 = t * kTile + 8 * uint64_t(lane);
    float d[8];
    if (e0 + 8 <= n) {
      const float4 u = *reinterpret_cast<const float4*>(in + e0);
      const float4 v = *reinterpret_cast<const float4*>(in + e0 + 4);
      d[0] = u.x; d[1] = u.y; d[2] = u.z; d[3] = u.w; d[4] = v.x; d[5] = v.y; d[6] = v.z; d[7] = v.w;
    } else {
#pragma unroll
      for (int i = 0; i < 8; ++i) d[i] = e0 + i < n ? in[e0 + i] : 0.0f;
    }
    // quantize (Sec. 4.2.2): the nearest integer of fl(d r), ties to even
    uint32_t qh[8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
      qh[i] = uint32_t(__float_as_int(__fadd_rn(__fmul_rn(d[i], r), kMagic)) - kMagicBits);
    if constexpr (kCentred) {
      // the tile mean in the fixed order: lane j's 8-element run, then pairs 16, 8, 4, 2, 1
      float P = d[0];
#pragma unroll
      for (int i = 1; i < 8; ++i) P = __fadd_rn(P, d[i]);
#pragma unroll
      for (int o = 16; o >= 1; o >>= 1) P = __fadd_rn(P, __shfl_xor_sync(FULL, P, o));
      const uint32_t mu = uint32_t(
          __float_as_int(__fadd_rn(__fmul_rn(__fmul_rn(P, 0.00390625f), r), kMagic)) - kMagicBits);
#pragma unroll
      for (int i = 0; i < 8; ++i) qh[i] -= mu;
    }
    // residuals with the state carried across blocks (Eq. 2), zero before the tile
    uint32_t p1 = __shfl_up_sync(FULL, qh[7], 1), p2 = __shfl_up_sync(FULL, qh[6], 1);
    if (lane == 0) p1 = p2 = 0;
    uint32_t m = 0;  // OR of |l| (same bit length as the maximum)
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const uint32_t l = kSecond ? qh[i] - 2u * p1 + p2 : qh[i] - p1;
      m |= uabs32(int32_t(l));
      p2 = p1;
      p1 = qh[i];
    }
    // block = 4 lanes: its rate (Sec. 4.1.2) and cost S_b (Eq. 3), summed over the tile
    m |= __shfl_xor_sync(FULL, m, 1);
    m |= __shfl_xor_sync(FULL, m, 2);
    const uint32_t rate = 32u - uint32_t(__clz(int(m)));
    const uint32_t cb = (lane & 3) == 0 && rate > 0 ? 4u + 4u * rate : 0u;
    const uint32_t C = __reduce_add_sync(FULL, cb) + (kCentred ? 4u : 0u);
    if (lane == 0) costs[uint64_t(kVariant) * T + t] = C;
  }
}

int cost_grid() {
  static DeviceCfgCache cache;  // per device
  return cache.get([] {
    LaunchCfg c;
    c.grid = [&] {
      int dev = 0, sms = 0, per = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fsz_cost_pass_kernel<0>, kCostThreads, 0);
      return sms * (per > 0 ? per : 1);
    }();
    return c;
  }).grid;
}

}  // namespace

void launch_cost_pass(const KernelArgs& a, int variant, uint32_t* costs, cudaStream_t st) {
  const int g = cost_grid();
  switch (variant) {
    case 0: fsz_cost_pass_kernel<0><<<g, kCostThreads, 0, st>>>(a, costs); break;
    case 1: fsz_cost_pass_kernel<1><<<g, kCostThreads, 0, st>>>(a, costs); break;
    case 2: fsz_cost_pass_kernel<2><<<g, kCostThreads, 0, st>>>(a, costs); break;
    default: fsz_cost_pass_kernel<3><<<g, kCostThreads, 0, st>>>(a, costs); break;
  }
}

}  // namespace fsz
