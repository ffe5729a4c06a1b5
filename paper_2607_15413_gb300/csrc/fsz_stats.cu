// Value-range pass, set-up and planning kernels.
//
// fsz_stats_kernel: min, max and finiteness of every field (Sec. 5.1: eb = REL x (max -
// min)), then the float32-safe quantization step of each field, derived on the device
// by whichever CTA finishes the field's last chunk, so the host never waits.
// Set-up kernels (one field) and planning kernels (a batch) fill the per-field state and
// the chunk -> field table that every later kernel of the call reads.
#include "fsz_internal.cuh"

namespace fsz {

namespace {

constexpr int kStatsThreads = 256;

// Derives eb, e, s = 2e and r = fl(1/s) from the field's range (reading of Sec. 5.1 and
// of the error-bound argument of Sec. 4.2.2): ABS takes eb as given, REL takes
// REL x (max - min) in float64 (REL x |max|, or REL, for a constant field). The half step
// e = eb (1 - eps) rounded toward zero, eps = (3Q + 4) 2^-23, Q = ceil(A / (2 eb (1 -
// c))) + 1, A = max |d|, with the cap c = 2^-4 where that gives eps <= 2^-4 and c = 2^-1
// (eps <= 2^-1) otherwise: the two float32 roundings of quantization and reconstruction
// then stay inside eb for every |q| <= Q.
__device__ uint32_t derive_params(FieldInfo* fi) {
  if (fi->max_abs_bits >= 0x7f800000u) return FSZ_ERR_NONFINITE;
  float vmin = 0.0f, vmax = 0.0f;
  if (fi->n > 0) {
    vmin = key_float(~fi->min_inv_key);
    vmax = key_float(fi->max_key);
  }
  double eb = fi->eb_req;
  if (fi->mode == FSZ_EB_REL) {
    double range = __dadd_rn(double(vmax), -double(vmin));
    if (range > 0.0) {
      eb = __dmul_rn(fi->eb_req, range);
    } else {
      double mag = fabs(double(vmax));
      eb = mag > 0.0 ? __dmul_rn(fi->eb_req, mag) : fi->eb_req;
    }
  }
  if (!(eb > 0.0) || isinf(eb)) return FSZ_ERR_EB_TOO_SMALL;
  const double two100 = 1267650600228229401496703205376.0;  // 2^100
  double eb_eff = eb < two100 ? eb : two100;
  double A = fmax(fabs(double(vmin)), fabs(double(vmax)));
  // first tier: K = A / (2 eb (1 - 2^-4)), eps <= 2^-4
  double K = __ddiv_rn(A, __dmul_rn(__dmul_rn(2.0, eb_eff), 0.9375));
  uint32_t Q = 0;
  if (K <= double(kQmax1) && uint32_t(ceil(K)) + 1u <= kQmax1) {
    Q = uint32_t(ceil(K)) + 1u;
  } else {
    // second tier, for fields the first refuses: K = A / (2 eb (1 - 2^-1)), eps <= 2^-1
    K = __ddiv_rn(A, __dmul_rn(__dmul_rn(2.0, eb_eff), 0.5));
    if (!(K <= double(kQmax2))) return FSZ_ERR_EB_TOO_SMALL;
    Q = uint32_t(ceil(K)) + 1u;
    if (Q > kQmax2) return FSZ_ERR_EB_TOO_SMALL;
  }
  double eps = __dmul_rn(double(3u * Q + 4u), 1.1920928955078125e-07);  // x 2^-23, exact
  double x = __dmul_rn(eb_eff, __dadd_rn(1.0, -eps));
  float e = __double2float_rz(x);
  if (!(e >= 7.888609052210118e-31f)) return FSZ_ERR_EB_TOO_SMALL;  // 2^-100
  float s = __fmul_rn(2.0f, e);
  fi->eb = eb;
  fi->e = e;
  fi->s = s;
  fi->r = __fdiv_rn(1.0f, s);
  fi->Q = Q;
  return FSZ_OK;
}

__device__ __forceinline__ void finish_field(Ctrl* ctrl, FieldInfo* fi) {
  if (fi->status != 0) return;
  uint32_t st = derive_params(fi);
  if (st != FSZ_OK) set_error(ctrl, fi, st);
}

__global__ void __launch_bounds__(kStatsThreads) fsz_stats_kernel(KernelArgs a) {
  __shared__ float s_lo[kStatsThreads / 32], s_hi[kStatsThreads / 32];
  __shared__ uint32_t s_abs[kStatsThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint64_t total = a.ctrl->total_chunks;

  float lo = __int_as_float(0x7f800000), hi = __int_as_float(0xff800000);
  uint32_t mabs = 0, my_items = 0;

  // Publishes this CTA's partial range of field f and counts the chunks it covered; the
  // CTA that completes the field's count derives the field's step.
  auto flush = [&](uint32_t f) {
    float l = lo, h = hi;
    uint32_t m = mabs;
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
      l = fminf(l, __shfl_xor_sync(0xffffffffu, l, o));
      h = fmaxf(h, __shfl_xor_sync(0xffffffffu, h, o));
      m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    }
    if (lane == 0) { s_lo[warp] = l; s_hi[warp] = h; s_abs[warp] = m; }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int w = 1; w < kStatsThreads / 32; ++w) {
        l = fminf(l, s_lo[w]);
        h = fmaxf(h, s_hi[w]);
        m = max(m, s_abs[w]);
      }
      FieldInfo* fi = a.fields + f;
      if (l <= h) {
        atomicMax(&fi->min_inv_key, ~float_key(l));
        atomicMax(&fi->max_key, float_key(h));
      }
      atomicMax(&fi->max_abs_bits, m);
      __threadfence();
      uint32_t prev = atomicAdd(&fi->done_chunks, my_items);
      if (uint64_t(prev) + my_items == fi->nchunks) {
        __threadfence();
        finish_field(a.ctrl, fi);
      }
    }
    __syncthreads();
    lo = __int_as_float(0x7f800000);
    hi = __int_as_float(0xff800000);
    mabs = 0;
    my_items = 0;
  };

  const bool single = a.ctrl->nfields == 1;  // (a single field's workspace has no chunk map)
  uint32_t cur_f = 0xffffffffu;
  for (uint64_t g = blockIdx.x; g < total; g += gridDim.x) {
    const uint32_t f = single ? 0u : a.chunk_field[g];
    if (f != cur_f) {
      if (cur_f != 0xffffffffu) flush(cur_f);
      cur_f = f;
    }
    const FieldInfo* fi = a.fields + f;
    const uint64_t e0 = (g - fi->chunk_first) * uint64_t(kCChunkElems);
    const uint64_t cnt = min(fi->n - e0, uint64_t(kCChunkElems));
    const float* p = fi->in + e0;
    const float4* p4 = reinterpret_cast<const float4*>(p);
    auto take4 = [&](float4 v) {
      lo = fminf(lo, fminf(fminf(v.x, v.y), fminf(v.z, v.w)));
      hi = fmaxf(hi, fmaxf(fmaxf(v.x, v.y), fmaxf(v.z, v.w)));
      uint32_t m0 = max(__float_as_uint(v.x) & 0x7fffffffu, __float_as_uint(v.y) & 0x7fffffffu);
      uint32_t m1 = max(__float_as_uint(v.z) & 0x7fffffffu, __float_as_uint(v.w) & 0x7fffffffu);
      mabs = max(mabs, max(m0, m1));
    };
    if (cnt == uint64_t(kCChunkElems)) {
      constexpr int kPer = kCChunkElems / 4 / kStatsThreads;
      float4 v[kPer];
#pragma unroll
      for (int u = 0; u < kPer; ++u) v[u] = __ldcs(p4 + threadIdx.x + u * kStatsThreads);
#pragma unroll
      for (int u = 0; u < kPer; ++u) take4(v[u]);
    } else {
      const uint64_t nv4 = cnt / 4;
      for (uint64_t k = threadIdx.x; k < nv4; k += kStatsThreads) take4(__ldcs(p4 + k));
      for (uint64_t k = nv4 * 4 + threadIdx.x; k < cnt; k += kStatsThreads) {
        float v = p[k];
        lo = fminf(lo, v);
        hi = fmaxf(hi, v);
        mabs = max(mabs, __float_as_uint(v) & 0x7fffffffu);
      }
    }
    if (threadIdx.x == 0) ++my_items;
  }
  if (cur_f != 0xffffffffu) flush(cur_f);
}

// Validates one compression descriptor and fills the field's shape (host-visible errors
// of the one-field entry point are checked again here for batches).
__device__ uint32_t plan_cfield(FieldInfo* fi, const fsz_cfield& d) {
  fi->in = d.in;
  fi->out = static_cast<uint8_t*>(d.out);
  fi->cap = d.out_capacity;
  fi->out_bytes = d.out_bytes;
  fi->mode = d.mode;
  fi->eb_req = d.eb;
  fi->ndim = d.dims.ndim;
  fi->nchunks = 0;
  fi->features_off = d.features_off;
  if (d.dims.ndim < 1 || d.dims.ndim > 3 || d.dims.reserved != 0 || !features_valid(d.features_off) ||
      d.mode > 1 || !(d.eb > 0.0) || isinf(d.eb) || d.out == nullptr)
    return FSZ_ERR_INVALID_ARG;
  uint64_t n = 1;
  for (uint32_t k = 0; k < d.dims.ndim; ++k) {
    const uint64_t dk = d.dims.dims[k];
    if (dk != 0 && n > kMaxElems / dk) return FSZ_ERR_INVALID_ARG;
    n *= dk;
    fi->dims[k] = dk;
  }
  if (n > kMaxElems) return FSZ_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(d.in) & 15) || (reinterpret_cast<uintptr_t>(d.out) & 15))
    return FSZ_ERR_ALIGN;
  if (n > 0 && d.in == nullptr) return FSZ_ERR_INVALID_ARG;
  const uint64_t T = (n + kTile - 1) / kTile;
  fi->n = n;
  fi->T = T;
  if (d.out_capacity < 64 + 8 * T) return FSZ_ERR_CAPACITY;
  fi->nchunks = (T + kCChunkTiles - 1) / kCChunkTiles;
  return FSZ_OK;
}

// Parses and checks a stream's preamble (the same rules as the format's definition:
// magic, version, ndim, mode, dims product, positive finite eb and step, sizes).
__device__ uint32_t plan_dfield(FieldInfo* fi, const uint8_t* in, uint64_t in_bytes, float* out,
                                uint64_t cap_elems) {
  fi->sin = in;
  fi->in_bytes = in_bytes;
  fi->dout = out;
  fi->nchunks = 0;
  if (in == nullptr || out == nullptr) return FSZ_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(in) & 15) || (reinterpret_cast<uintptr_t>(out) & 15))
    return FSZ_ERR_ALIGN;
  if (in_bytes < 64) return FSZ_ERR_CORRUPT;
  uint32_t w[16];
  const uint4* p = reinterpret_cast<const uint4*>(in);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const uint4 v = p[k];
    w[4 * k] = v.x; w[4 * k + 1] = v.y; w[4 * k + 2] = v.z; w[4 * k + 3] = v.w;
  }
  if (w[0] != 0x315A5346u || (w[1] & 0xFFFFu) != 1u) return FSZ_ERR_CORRUPT;
  const uint32_t ndim = (w[1] >> 16) & 0xFFu, mode = w[1] >> 24;
  if (ndim < 1 || ndim > 3 || mode > 1) return FSZ_ERR_CORRUPT;
  const uint64_t n = uint64_t(w[2]) | (uint64_t(w[3]) << 32);
  uint64_t prod = 1;
  for (uint32_t k = 0; k < 3; ++k) {
    const uint64_t dk = uint64_t(w[4 + 2 * k]) | (uint64_t(w[5 + 2 * k]) << 32);
    if (k >= ndim) {
      if (dk != 0) return FSZ_ERR_CORRUPT;
      continue;
    }
    if (dk != 0 && prod > kMaxElems / dk) return FSZ_ERR_CORRUPT;
    prod *= dk;
    fi->dims[k] = dk;
  }
  if (prod != n || n > kMaxElems) return FSZ_ERR_CORRUPT;
  const double eb = __longlong_as_double(static_cast<long long>(uint64_t(w[10]) | (uint64_t(w[11]) << 32)));
  const float sv = __uint_as_float(w[12]);
  if (!(eb > 0.0) || isinf(eb)) return FSZ_ERR_CORRUPT;
  if (!(sv >= 1.5777218104420236e-30f) || isinf(sv)) return FSZ_ERR_CORRUPT;  // 2^-99
  if (w[13] & 0xFF00u) return FSZ_ERR_INVALID_ARG;  // a tile configuration: fsz_decompress_tiled
  if (!features_valid(w[13])) return FSZ_ERR_CORRUPT;
  fi->features_off = w[13];
  const uint64_t db = uint64_t(w[14]) | (uint64_t(w[15]) << 32);
  const uint64_t T = (n + kTile - 1) / kTile;
  if (in_bytes - 64 < 8 * T) return FSZ_ERR_CORRUPT;
  if (db > in_bytes - 64 - 8 * T) return FSZ_ERR_CORRUPT;
  fi->n = n;
  fi->T = T;
  fi->ndim = ndim;
  fi->mode = mode;
  fi->eb_req = eb;
  fi->s = sv;
  fi->data_bytes = db;
  if (n > cap_elems) return FSZ_ERR_CAPACITY;
  fi->nchunks = (T + kDChunkTiles - 1) / kDChunkTiles;
  return FSZ_OK;
}

// A valid field of zero elements: its step, its 64-byte stream and its size.
__device__ void finish_empty_field(Ctrl* ctrl, FieldInfo* fi) {
  finish_field(ctrl, fi);
  if (fi->status == 0) write_preamble(fi, 0);
}

// One-field set-up for compression: the descriptor is validated on the host, so this
// copies it into the workspace.
// Set-up of a single-field call: thread 0 of CTA 0 clears the control words and the field
// record and fills them in; every other thread clears the lookback flags (nflags words),
// so that the call needs no separate memset.
constexpr int kSetupThreads = 256;
static_assert(sizeof(Ctrl) <= 256 && sizeof(Ctrl) % 8 == 0 && sizeof(FieldInfo) % 8 == 0,
              "control words and field record clear as 8-byte words");

__device__ __forceinline__ bool setup_clear(const KernelArgs& a, uint64_t nflags) {
  const uint64_t t = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t == 0) {
    uint64_t* c = reinterpret_cast<uint64_t*>(a.ctrl);
    for (uint32_t k = 0; k < sizeof(Ctrl) / 8; ++k) c[k] = 0;
    uint64_t* f = reinterpret_cast<uint64_t*>(a.fields);
    for (uint32_t k = 0; k < sizeof(FieldInfo) / 8; ++k) f[k] = 0;
    return true;
  }
  const uint64_t nthreads = uint64_t(gridDim.x) * blockDim.x - 1;
  for (uint64_t k = t - 1; k < nflags; k += nthreads) a.flags[k] = 0;
  return false;
}

__global__ void __launch_bounds__(kSetupThreads) fsz_setup_compress_kernel(KernelArgs a, FieldInfo desc,
                                                                           uint64_t nflags) {
  if (!setup_clear(a, nflags)) return;
  FieldInfo* fi = a.fields;
  fi->in = desc.in; fi->out = desc.out; fi->cap = desc.cap; fi->out_bytes = desc.out_bytes;
  fi->n = desc.n; fi->T = desc.T;
  fi->dims[0] = desc.dims[0]; fi->dims[1] = desc.dims[1]; fi->dims[2] = desc.dims[2];
  fi->ndim = desc.ndim; fi->mode = desc.mode; fi->eb_req = desc.eb_req;
  fi->features_off = desc.features_off;
  fi->chunk_first = 0;
  fi->nchunks = desc.nchunks;
  a.ctrl->nfields = 1;
  a.ctrl->total_chunks = desc.nchunks;
  if (desc.n == 0) finish_empty_field(a.ctrl, fi);
}

__global__ void __launch_bounds__(kSetupThreads) fsz_setup_decompress_kernel(
    KernelArgs a, const uint8_t* in, uint64_t in_bytes, float* out, uint64_t cap_elems,
    uint64_t chunk_cap, uint64_t nflags) {
  if (!setup_clear(a, nflags)) return;
  FieldInfo* fi = a.fields;
  uint32_t st = plan_dfield(fi, in, in_bytes, out, cap_elems);
  if (st == FSZ_OK && fi->nchunks > chunk_cap) st = FSZ_ERR_WORKSPACE;
  if (st != FSZ_OK) {
    set_error(a.ctrl, fi, st);
    fi->nchunks = 0;
  }
  fi->chunk_first = 0;
  a.ctrl->nfields = 1;
  a.ctrl->total_chunks = fi->nchunks;
}

// CTAs of a set-up launch: one plus one per 2048 flag words, at most 152.
inline int setup_grid(uint64_t nflags) {
  const uint64_t g = 1 + nflags / (8 * kSetupThreads);
  return int(g < 152 ? g : 152);
}

constexpr int kPlanThreads = 1024;

// Batch planning (one CTA): per-field checks, an exclusive scan of the fields' chunk
// counts (their ranges in the field-major ticket order) and the chunk -> field table.
template <bool kCompress>
__global__ void __launch_bounds__(kPlanThreads) fsz_plan_kernel(KernelArgs a, const void* d_fields,
                                                                uint32_t nfields, uint64_t chunk_cap) {
  __shared__ uint64_t s_warp[kPlanThreads / 32];
  __shared__ uint64_t s_carry;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) s_carry = 0;
  __syncthreads();
  for (uint32_t base = 0; base < nfields; base += kPlanThreads) {
    const uint32_t f = base + tid;
    uint64_t nch = 0;
    if (f < nfields) {
      FieldInfo* fi = a.fields + f;
      uint32_t st;
      if constexpr (kCompress) {
        st = plan_cfield(fi, static_cast<const fsz_cfield*>(d_fields)[f]);
      } else {
        const fsz_dfield d = static_cast<const fsz_dfield*>(d_fields)[f];
        st = plan_dfield(fi, static_cast<const uint8_t*>(d.in), d.in_bytes, d.out, d.out_capacity_elems);
      }
      if (st != FSZ_OK) {
        set_error(a.ctrl, fi, st);
        fi->nchunks = 0;
      }
      nch = fi->nchunks;
    }
    // block-wide exclusive scan of nch
    uint64_t inc = nch;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint64_t y = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += y;
    }
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    if (warp == 0) {
      uint64_t v = s_warp[lane];
      uint64_t vi = v;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint64_t y = __shfl_up_sync(0xffffffffu, vi, o);
        if (lane >= o) vi += y;
      }
      s_warp[lane] = vi - v;
    }
    __syncthreads();
    const uint64_t first = s_carry + s_warp[warp] + inc - nch;
    if (f < nfields) a.fields[f].chunk_first = first;
    __syncthreads();
    if (tid == kPlanThreads - 1) s_carry = first + nch;
    __syncthreads();
  }
  const uint64_t total = s_carry;
  if (tid == 0) {
    a.ctrl->nfields = nfields;
    if (total > chunk_cap) {
      set_error(a.ctrl, nullptr, FSZ_ERR_WORKSPACE);
      a.ctrl->total_chunks = 0;
    } else {
      a.ctrl->total_chunks = total;
    }
  }
  if (total > chunk_cap) return;
  // The chunk -> field table, one warp per field (the fields' ranges are disjoint), so
  // that the fields' record loads overlap rather than follow one another.
  uint32_t* map = const_cast<uint32_t*>(a.chunk_field);
  for (uint32_t f = uint32_t(warp); f < nfields; f += uint32_t(kPlanThreads / 32)) {
    const FieldInfo* fi = a.fields + f;
    const uint64_t c0 = fi->chunk_first, nc = fi->nchunks;
    for (uint64_t k = uint64_t(lane); k < nc; k += 32) map[c0 + k] = f;
  }
  if constexpr (kCompress) {
    for (uint32_t f = tid; f < nfields; f += kPlanThreads) {
      FieldInfo* fi = a.fields + f;
      if (fi->status == 0 && fi->n == 0) finish_empty_field(a.ctrl, fi);
    }
  }
}

}  // namespace

LaunchCfg stats_cfg() {
  static DeviceCfgCache cache;
  return cache.get([] {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fsz_stats_kernel, kStatsThreads, 0);
    LaunchCfg c;
    c.sms = sms;
    c.per = per > 0 ? per : 1;
    c.grid = sms * c.per;
    c.smem = 0;
    return c;
  });
}

void launch_stats(const KernelArgs& a, cudaStream_t st) {
  fsz_stats_kernel<<<sched_grid(stats_cfg(), kSchedStats), kStatsThreads, 0, st>>>(a);
}

void launch_setup_compress(const KernelArgs& a, const FieldInfo& fi, uint64_t chunk_cap, cudaStream_t st) {
  const uint64_t nflags = kFlagStride * chunk_cap;
  fsz_setup_compress_kernel<<<setup_grid(nflags), kSetupThreads, 0, st>>>(a, fi, nflags);
}

void launch_setup_decompress(const KernelArgs& a, const uint8_t* in, uint64_t in_bytes, float* out,
                             uint64_t cap_elems, uint64_t chunk_cap, cudaStream_t st) {
  const uint64_t nflags = kFlagStride * chunk_cap;
  fsz_setup_decompress_kernel<<<setup_grid(nflags), kSetupThreads, 0, st>>>(a, in, in_bytes, out,
                                                                            cap_elems, chunk_cap, nflags);
}

void launch_plan_compress(const KernelArgs& a, const fsz_cfield* d_fields, uint32_t nfields,
                          uint64_t chunk_cap, cudaStream_t st) {
  fsz_plan_kernel<true><<<1, kPlanThreads, 0, st>>>(a, d_fields, nfields, chunk_cap);
}

void launch_plan_decompress(const KernelArgs& a, const fsz_dfield* d_fields, uint32_t nfields,
                            uint64_t chunk_cap, cudaStream_t st) {
  fsz_plan_kernel<false><<<1, kPlanThreads, 0, st>>>(a, d_fields, nfields, chunk_cap);
}

}  // namespace fsz
