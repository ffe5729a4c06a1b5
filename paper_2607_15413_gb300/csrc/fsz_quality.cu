// Reconstruction quality of a decompressed field against its original, for the
// rate-distortion evaluation of Sec. 6.2 (Fig. 8: PSNR against bit rate): max |d - d'|,
// the sum of squared errors, the count of errors above the bound, the original's value
// range, and from them PSNR, NRMSE and the bit rate.
//
// A stream over both arrays (8 bytes per element, HBM-bound): per element one float32
// difference, its magnitude and square; squares are summed in float32 over a thread's 8
// elements of an iteration and then added in float64 (GB300's float64 rate is a fraction
// of its float32 rate). CTA partials go to the workspace; the last CTA through (a
// counter) reduces them in CTA order, so the result does not depend on timing.
#include <algorithm>

#include "fsz_internal.cuh"

static_assert(sizeof(fsz_quality) == 72, "ABI struct size");

namespace fsz {

namespace {

constexpr int kQThreads = 256;
constexpr int kQMaxCtas = 4096;

struct QPartial {
  double sum_sq;
  unsigned long long over;
  float max_err, vmin, vmax, pad;
};

struct QWork {
  unsigned int done;
  unsigned int pad[3];
  QPartial part[kQMaxCtas];
};

__device__ __forceinline__ void q_accumulate(float d, float y, float ebf, float& mx, float& mn,
                                             float& vmx, unsigned long long& over, float& sq) {
  const float e = __fsub_rn(d, y);
  const float a = fabsf(e);
  mx = fmaxf(mx, a);
  over += a > ebf ? 1ull : 0ull;
  sq = __fmaf_rn(e, e, sq);
  mn = fminf(mn, d);
  vmx = fmaxf(vmx, d);
}

__global__ void __launch_bounds__(kQThreads) fsz_quality_kernel(const float* __restrict__ d,
                                                                const float* __restrict__ y,
                                                                uint64_t n, double eb,
                                                                uint64_t stream_bytes,
                                                                fsz_quality* out, QWork* w) {
  constexpr uint32_t FULL = 0xffffffffu;
  // |e| > eb for a float |e| exactly when |e| exceeds eb rounded down to float32
  const float ebf = __double2float_rd(eb);
  float mx = 0.0f, mn = INFINITY, vmx = -INFINITY;
  unsigned long long over = 0;
  double sum = 0.0;
  const uint64_t tid = uint64_t(blockIdx.x) * kQThreads + threadIdx.x;
  const uint64_t nth = uint64_t(gridDim.x) * kQThreads;
  const uint64_t n8 = n / 8;
  for (uint64_t k = tid; k < n8; k += nth) {
    const float4 d0 = reinterpret_cast<const float4*>(d)[2 * k];
    const float4 d1 = reinterpret_cast<const float4*>(d)[2 * k + 1];
    const float4 y0 = reinterpret_cast<const float4*>(y)[2 * k];
    const float4 y1 = reinterpret_cast<const float4*>(y)[2 * k + 1];
    float sq = 0.0f;
    q_accumulate(d0.x, y0.x, ebf, mx, mn, vmx, over, sq);
    q_accumulate(d0.y, y0.y, ebf, mx, mn, vmx, over, sq);
    q_accumulate(d0.z, y0.z, ebf, mx, mn, vmx, over, sq);
    q_accumulate(d0.w, y0.w, ebf, mx, mn, vmx, over, sq);
    q_accumulate(d1.x, y1.x, ebf, mx, mn, vmx, over, sq);
    q_accumulate(d1.y, y1.y, ebf, mx, mn, vmx, over, sq);
    q_accumulate(d1.z, y1.z, ebf, mx, mn, vmx, over, sq);
    q_accumulate(d1.w, y1.w, ebf, mx, mn, vmx, over, sq);
    sum += double(sq);
  }
  for (uint64_t i = 8 * n8 + tid; i < n; i += nth) {  // the last n mod 8 elements
    float sq = 0.0f;
    q_accumulate(d[i], y[i], ebf, mx, mn, vmx, over, sq);
    sum += double(sq);
  }
  // CTA reduction (warp shuffles, then the warps in order)
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) {
    mx = fmaxf(mx, __shfl_xor_sync(FULL, mx, o));
    mn = fminf(mn, __shfl_xor_sync(FULL, mn, o));
    vmx = fmaxf(vmx, __shfl_xor_sync(FULL, vmx, o));
    over += __shfl_xor_sync(FULL, over, o);
    sum += __shfl_xor_sync(FULL, sum, o);
  }
  __shared__ QPartial s_w[kQThreads / 32];
  __shared__ bool s_last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) s_w[warp] = QPartial{sum, over, mx, mn, vmx, 0.0f};
  __syncthreads();
  if (threadIdx.x == 0) {
    QPartial p = s_w[0];
    for (int k = 1; k < kQThreads / 32; ++k) {
      p.sum_sq += s_w[k].sum_sq;
      p.over += s_w[k].over;
      p.max_err = fmaxf(p.max_err, s_w[k].max_err);
      p.vmin = fminf(p.vmin, s_w[k].vmin);
      p.vmax = fmaxf(p.vmax, s_w[k].vmax);
    }
    w->part[blockIdx.x] = p;
    __threadfence();
    s_last = atomicAdd(&w->done, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!s_last || threadIdx.x != 0) return;
  __threadfence();
  QPartial t = w->part[0];
  for (unsigned int b = 1; b < gridDim.x; ++b) {
    const QPartial p = w->part[b];
    t.sum_sq += p.sum_sq;
    t.over += p.over;
    t.max_err = fmaxf(t.max_err, p.max_err);
    t.vmin = fminf(t.vmin, p.vmin);
    t.vmax = fmaxf(t.vmax, p.vmax);
  }
  const double range = double(t.vmax) - double(t.vmin);
  const double mse = t.sum_sq / double(n);
  fsz_quality r;
  r.n = n;
  r.over_bound = t.over;
  r.max_abs_err = double(t.max_err);
  r.sum_sq_err = t.sum_sq;
  r.min = double(t.vmin);
  r.max = double(t.vmax);
  r.psnr_db = mse > 0.0 ? 20.0 * log10(range) - 10.0 * log10(mse) : INFINITY;
  r.nrmse = range > 0.0 ? sqrt(mse) / range : 0.0;
  r.bit_rate = 8.0 * double(stream_bytes) / double(n);
  *out = r;
  w->done = 0;  // the workspace is ready for the next call
}

int quality_grid() {
  static DeviceCfgCache cache;  // per device
  return cache.get([] {
    LaunchCfg c;
    c.grid = [&] {
      int dev = 0, sms = 0, per = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fsz_quality_kernel, kQThreads, 0);
      return std::min(kQMaxCtas, sms * (per > 0 ? per : 1));
    }();
    return c;
  }).grid;
}

}  // namespace

}  // namespace fsz

extern "C" {

uint64_t fsz_quality_workspace_bytes(void) { return sizeof(fsz::QWork); }

fsz_status fsz_quality_stats(const float* d_orig, const float* d_recon, uint64_t n, double eb,
                             uint64_t stream_bytes, fsz_quality* d_out, void* d_ws,
                             uint64_t ws_bytes, fsz_stream stream) {
  if (d_orig == nullptr || d_recon == nullptr || d_out == nullptr || d_ws == nullptr || n == 0)
    return FSZ_ERR_INVALID_ARG;
  if (!(eb >= 0.0)) return FSZ_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(d_orig) | reinterpret_cast<uintptr_t>(d_recon) |
       reinterpret_cast<uintptr_t>(d_ws) | reinterpret_cast<uintptr_t>(d_out)) & 15)
    return FSZ_ERR_ALIGN;
  if (ws_bytes < sizeof(fsz::QWork)) return FSZ_ERR_WORKSPACE;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  // only the counter needs clearing: every CTA writes its partial before the last reads
  if (cudaMemsetAsync(d_ws, 0, 16, s) != cudaSuccess) return FSZ_ERR_CUDA;
  fsz::fsz_quality_kernel<<<fsz::quality_grid(), fsz::kQThreads, 0, s>>>(
      d_orig, d_recon, n, eb, stream_bytes, d_out, static_cast<fsz::QWork*>(d_ws));
  return cudaGetLastError() == cudaSuccess ? FSZ_OK : FSZ_ERR_CUDA;
}

}  // extern "C"
