// fsz_compress_noalloc: single-field compression with a built-in workspace.
//
// For callers that must not allocate device memory: plugins whose host framework owns
// every byte of device memory through its own pool (an allocation of their own would be
// refused or unaccounted for), and latency-critical paths that cannot afford the
// device-wide synchronisation an allocation can cause. Such a caller passes only its
// input and output buffers; the scratch the kernels need (control words, per-field
// state and lookback flags) lives in the file-scope array below, which every GPU that
// loads this library keeps for the life of the process.
#include <cmath>
#include <cstring>
#include <mutex>

#include "fsz_internal.cuh"

namespace {

using namespace fsz;

constexpr uint64_t kNoAllocMaxElems = uint64_t(FSZ_NOALLOC_MAX_ELEMS);
constexpr uint64_t kNoAllocMaxTiles = (kNoAllocMaxElems + kTile - 1) / kTile;

// Largest workspace a field of up to FSZ_NOALLOC_MAX_ELEMS elements needs.
constexpr uint64_t noalloc_scratch_bytes() {
  const uint64_t cap = (kNoAllocMaxTiles + kMinChunkTiles - 1) / kMinChunkTiles + 1 + 1;
  const uint64_t map_off = 256 + sizeof(FieldInfo);
  const uint64_t flags_off = (map_off + 4 * cap + 127) & ~uint64_t(127);
  return flags_off + 8 * kFlagStride * cap;
}
constexpr uint64_t kScratchBytes = (noalloc_scratch_bytes() + 255) & ~uint64_t(255);

static __device__ __align__(256) uint8_t g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once per device.
// The host symbol g_noalloc_scratch is only a handle; kernels must get this address.
fsz_status scratch_on_current_device(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return FSZ_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_mu);
  if (g_scratch_ptr[dev] == nullptr) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) {
      return FSZ_ERR_CUDA;
    }
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return FSZ_OK;
}

}  // namespace

extern "C" fsz_status fsz_compress_noalloc(const float* d_in, fsz_dims dims, fsz_eb_mode mode,
                                           double eb, void* d_out, uint64_t out_capacity,
                                           uint64_t* d_out_bytes, uint32_t* d_status,
                                           fsz_stream stream) {
  if (dims.ndim < 1 || dims.ndim > 3 || dims.reserved != 0) return FSZ_ERR_INVALID_ARG;
  uint64_t n = 1;
  for (uint32_t k = 0; k < dims.ndim; ++k) {
    const uint64_t dk = dims.dims[k];
    if (dk != 0 && n > kMaxElems / dk) return FSZ_ERR_INVALID_ARG;
    n *= dk;
  }
  if (n > kNoAllocMaxElems) return FSZ_ERR_WORKSPACE;  // beyond the built-in scratch
  if (mode != FSZ_EB_ABS && mode != FSZ_EB_REL) return FSZ_ERR_INVALID_ARG;
  if (!(eb > 0.0) || !std::isfinite(eb)) return FSZ_ERR_INVALID_ARG;
  if (d_out == nullptr || (n > 0 && d_in == nullptr)) return FSZ_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(d_in) & 15) || (reinterpret_cast<uintptr_t>(d_out) & 15))
    return FSZ_ERR_ALIGN;
  const uint64_t T = (n + kTile - 1) / kTile;
  if (out_capacity < 64 + 8 * T) return FSZ_ERR_CAPACITY;
  const WsLayout L = ws_layout(T, 1);
  if (L.bytes > kScratchBytes) return FSZ_ERR_WORKSPACE;

  void* ws = nullptr;
  fsz_status st = scratch_on_current_device(&ws);
  if (st != FSZ_OK) return st;

  FieldInfo desc;
  std::memset(&desc, 0, sizeof(desc));
  desc.in = d_in;
  desc.out = static_cast<uint8_t*>(d_out);
  desc.cap = out_capacity;
  desc.out_bytes = d_out_bytes;
  desc.n = n;
  desc.T = T;
  for (uint32_t k = 0; k < dims.ndim; ++k) desc.dims[k] = dims.dims[k];
  desc.ndim = dims.ndim;
  desc.mode = uint32_t(mode);
  desc.eb_req = eb;
  desc.nchunks = (T + kCChunkTiles - 1) / kCChunkTiles;

  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  // The array keeps the previous call's contents: clear the part this call uses.
  if (cudaMemsetAsync(ws, 0, L.bytes, s) != cudaSuccess) return FSZ_ERR_CUDA;
  uint8_t* base = static_cast<uint8_t*>(ws);
  KernelArgs a;
  a.ctrl = reinterpret_cast<Ctrl*>(base);
  a.fields = reinterpret_cast<FieldInfo*>(base + L.fields_off);
  a.chunk_field = reinterpret_cast<const uint32_t*>(base + L.map_off);
  a.flags = reinterpret_cast<uint64_t*>(base + L.flags_off);
  a.skip_chunk = ~uint64_t(0);
  a.timeout_ns = kDefaultTimeoutNs;
  launch_setup_compress(a, desc, L.chunk_cap, s);
  if (desc.nchunks > 0) {
    launch_stats(a, s);
    launch_compress(a, s);
  }
  if (d_status != nullptr &&
      cudaMemcpyAsync(d_status, &a.ctrl->status, sizeof(uint32_t), cudaMemcpyDeviceToDevice, s) !=
          cudaSuccess)
    return FSZ_ERR_CUDA;
  return cudaGetLastError() == cudaSuccess ? FSZ_OK : FSZ_ERR_CUDA;
}
