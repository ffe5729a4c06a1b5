// C ABI of the FSZ library (declared in include/fsz.h): argument checks on the host,
// workspace layout, and the launch sequence of each call. No call allocates memory or
// synchronises the host except fsz_check / fsz_check_batched.
#include <cmath>
#include <cstring>
#include <vector>

#include "fsz_internal.cuh"

static_assert(sizeof(fsz_dims) == 32 && sizeof(fsz_cfield) == 80 && sizeof(fsz_dfield) == 32,
              "C ABI struct layouts");

namespace fsz {
// The default schedule: CTAs per SM (0 = as many as fit), compression's chunks per ticket
// and ticket lead, decompression's chunks per ticket and chunks in flight, and the tickets
// per CTA below which a launch takes smaller tickets.
#ifndef FSZ_DEF_C_CHUNKS
#define FSZ_DEF_C_CHUNKS 2
#endif
#ifndef FSZ_DEF_C_LEAD
#define FSZ_DEF_C_LEAD 2
#endif
#ifndef FSZ_DEF_D_CHUNKS
#define FSZ_DEF_D_CHUNKS 4
#endif
#ifndef FSZ_DEF_D_RECORDS
#define FSZ_DEF_D_RECORDS 16
#endif
#ifndef FSZ_DEF_MIN_TICKETS
#define FSZ_DEF_MIN_TICKETS 4
#endif
constexpr Schedule kDefaultSchedule = {{0, 0, 0}, FSZ_DEF_C_CHUNKS, FSZ_DEF_C_LEAD, FSZ_DEF_D_CHUNKS,
                                       FSZ_DEF_D_RECORDS, FSZ_DEF_MIN_TICKETS};
Schedule g_schedule = kDefaultSchedule;
}

// A captured batched call (fsz_graph in the C ABI).
struct fsz_graph_s {
  cudaGraphExec_t exec;
};

namespace {

using namespace fsz;

uint64_t g_skip_chunk = ~uint64_t(0);
uint64_t g_timeout_ns = kDefaultTimeoutNs;

bool misaligned(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) != 0; }

fsz_status dims_count(const fsz_dims& dims, uint64_t* n) {
  if (dims.ndim < 1 || dims.ndim > 3 || dims.reserved != 0) return FSZ_ERR_INVALID_ARG;
  uint64_t p = 1;
  for (uint32_t k = 0; k < dims.ndim; ++k) {
    const uint64_t dk = dims.dims[k];
    if (dk != 0 && p > kMaxElems / dk) return FSZ_ERR_INVALID_ARG;
    p *= dk;
  }
  if (p > kMaxElems) return FSZ_ERR_INVALID_ARG;
  *n = p;
  return FSZ_OK;
}

KernelArgs make_args(void* d_ws, const WsLayout& L) {
  uint8_t* ws = static_cast<uint8_t*>(d_ws);
  KernelArgs a;
  a.ctrl = reinterpret_cast<Ctrl*>(ws);
  a.fields = reinterpret_cast<FieldInfo*>(ws + L.fields_off);
  a.chunk_field = reinterpret_cast<const uint32_t*>(ws + L.map_off);
  a.flags = reinterpret_cast<uint64_t*>(ws + L.flags_off);
  a.skip_chunk = g_skip_chunk;
  a.timeout_ns = g_timeout_ns;
  return a;
}

fsz_status launched() {
  return cudaGetLastError() == cudaSuccess ? FSZ_OK : FSZ_ERR_CUDA;
}

struct CompressCall {
  WsLayout L;
  FieldInfo desc;
};

fsz_status check_compress(const float* d_in, fsz_dims dims, fsz_eb_mode mode, double eb, void* d_out,
                          uint64_t out_capacity, void* d_ws, uint64_t ws_bytes, CompressCall* call,
                          uint32_t features_off = 0) {
  uint64_t n = 0;
  fsz_status st = dims_count(dims, &n);
  if (st != FSZ_OK) return st;
  if (mode != FSZ_EB_ABS && mode != FSZ_EB_REL) return FSZ_ERR_INVALID_ARG;
  if (!features_valid(features_off)) return FSZ_ERR_INVALID_ARG;
  if (!(eb > 0.0) || !std::isfinite(eb)) return FSZ_ERR_INVALID_ARG;
  if (d_out == nullptr || d_ws == nullptr || (n > 0 && d_in == nullptr)) return FSZ_ERR_INVALID_ARG;
  if (misaligned(d_in) || misaligned(d_out) || misaligned(d_ws)) return FSZ_ERR_ALIGN;
  const uint64_t T = (n + kTile - 1) / kTile;
  if (out_capacity < 64 + 8 * T) return FSZ_ERR_CAPACITY;
  call->L = ws_layout(T, 1);
  if (ws_bytes < call->L.bytes) return FSZ_ERR_WORKSPACE;
  FieldInfo& d = call->desc;
  std::memset(&d, 0, sizeof(d));
  d.in = d_in;
  d.out = static_cast<uint8_t*>(d_out);
  d.cap = out_capacity;
  d.n = n;
  d.T = T;
  for (uint32_t k = 0; k < dims.ndim; ++k) d.dims[k] = dims.dims[k];
  d.ndim = dims.ndim;
  d.mode = uint32_t(mode);
  d.eb_req = eb;
  d.features_off = features_off;
  d.nchunks = (T + kCChunkTiles - 1) / kCChunkTiles;
  return FSZ_OK;
}

// Value-range pass and step for one field, with its switched-off features recorded in
// the workspace's field record (read by the compression kernel and the preamble).
fsz_status prepare_one(const float* d_in, fsz_dims dims, fsz_eb_mode mode, double eb,
                       uint32_t features_off, void* d_out, uint64_t out_capacity,
                       uint64_t* d_out_bytes, void* d_ws, uint64_t ws_bytes, fsz_stream stream) {
  CompressCall call;
  fsz_status st = check_compress(d_in, dims, mode, eb, d_out, out_capacity, d_ws, ws_bytes, &call,
                                 features_off);
  if (st != FSZ_OK) return st;
  call.desc.out_bytes = d_out_bytes;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const KernelArgs a = make_args(d_ws, call.L);
  launch_setup_compress(a, call.desc, call.L.chunk_cap, s);  // (clears the workspace it uses)
  if (call.desc.nchunks > 0) launch_stats(a, s);
  return launched();
}

// One stream's decompression with the given decoder instance.
fsz_status decompress_one(const void* d_in, uint64_t in_bytes, float* d_out,
                          uint64_t out_capacity_elems, void* d_ws, uint64_t ws_bytes,
                          fsz_stream stream, DecompressKind kind) {
  if (d_in == nullptr || d_out == nullptr || d_ws == nullptr) return FSZ_ERR_INVALID_ARG;
  if (misaligned(d_in) || misaligned(d_out) || misaligned(d_ws)) return FSZ_ERR_ALIGN;
  if (out_capacity_elems > kMaxElems) out_capacity_elems = kMaxElems;
  const WsLayout L = ws_layout((out_capacity_elems + kTile - 1) / kTile, 1);
  if (ws_bytes < L.bytes) return FSZ_ERR_WORKSPACE;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const KernelArgs a = make_args(d_ws, L);
  launch_setup_decompress(a, static_cast<const uint8_t*>(d_in), in_bytes, d_out, out_capacity_elems,
                          L.chunk_cap, s);
  launch_decompress(a, s, kind);
  return launched();
}

template <typename F>
fsz_status capture_graph(F&& record, fsz_graph* out) {
  if (out == nullptr) return FSZ_ERR_INVALID_ARG;
  *out = nullptr;
  // Kernel attributes are set before the capture begins.
  (void)stats_cfg();
  (void)compress_cfg();
  (void)decompress_cfg();
  cudaStream_t s;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return FSZ_ERR_CUDA;
  fsz_status st = FSZ_OK;
  cudaGraph_t graph = nullptr;
  if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    st = FSZ_ERR_CUDA;
  } else {
    st = record(reinterpret_cast<fsz_stream>(s));
    if (cudaStreamEndCapture(s, &graph) != cudaSuccess && st == FSZ_OK) st = FSZ_ERR_CUDA;
  }
  cudaGraphExec_t exec = nullptr;
  if (st == FSZ_OK && cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) st = FSZ_ERR_CUDA;
  if (graph) cudaGraphDestroy(graph);
  cudaStreamDestroy(s);
  if (st != FSZ_OK) return st;
  *out = new fsz_graph_s{exec};
  return FSZ_OK;
}
}  // namespace

extern "C" {

uint64_t fsz_compress_bound(uint64_t n) {
  const uint64_t T = (n + kTile - 1) / kTile;
  return 64 + 8 * T + uint64_t(kMaxTileBytes) * T;
}

uint64_t fsz_workspace_bytes(uint64_t n) { return ws_layout((n + kTile - 1) / kTile, 1).bytes; }

uint64_t fsz_batch_workspace_bytes(uint64_t n_total, uint32_t nfields) {
  return ws_layout(n_total / kTile + nfields, nfields).bytes;
}

fsz_status fsz_compress_prepare(const float* d_in, fsz_dims dims, fsz_eb_mode mode, double eb,
                                void* d_out, uint64_t out_capacity, uint64_t* d_out_bytes,
                                void* d_ws, uint64_t ws_bytes, fsz_stream stream) {
  return prepare_one(d_in, dims, mode, eb, 0, d_out, out_capacity, d_out_bytes, d_ws, ws_bytes,
                     stream);
}

fsz_status fsz_compress_encode(const float* d_in, fsz_dims dims, fsz_eb_mode mode, double eb,
                               void* d_out, uint64_t out_capacity, uint64_t* d_out_bytes,
                               void* d_ws, uint64_t ws_bytes, fsz_stream stream) {
  (void)d_out_bytes;
  CompressCall call;
  fsz_status st = check_compress(d_in, dims, mode, eb, d_out, out_capacity, d_ws, ws_bytes, &call);
  if (st != FSZ_OK) return st;
  if (call.desc.nchunks == 0) return FSZ_OK;
  launch_compress(make_args(d_ws, call.L), reinterpret_cast<cudaStream_t>(stream), kCompressFull);
  return launched();
}

fsz_status fsz_compress(const float* d_in, fsz_dims dims, fsz_eb_mode mode, double eb, void* d_out,
                        uint64_t out_capacity, uint64_t* d_out_bytes, void* d_ws, uint64_t ws_bytes,
                        fsz_stream stream) {
  fsz_status st = fsz_compress_prepare(d_in, dims, mode, eb, d_out, out_capacity, d_out_bytes, d_ws,
                                       ws_bytes, stream);
  if (st != FSZ_OK) return st;
  return fsz_compress_encode(d_in, dims, mode, eb, d_out, out_capacity, d_out_bytes, d_ws, ws_bytes,
                             stream);
}

fsz_status fsz_compress_features(const float* d_in, fsz_dims dims, fsz_eb_mode mode, double eb,
                                 uint32_t features_off, void* d_out, uint64_t out_capacity,
                                 uint64_t* d_out_bytes, void* d_ws, uint64_t ws_bytes,
                                 fsz_stream stream) {
  fsz_status st = prepare_one(d_in, dims, mode, eb, features_off, d_out, out_capacity, d_out_bytes,
                              d_ws, ws_bytes, stream);
  if (st != FSZ_OK || features_off == 0)
    return st != FSZ_OK ? st
                        : fsz_compress_encode(d_in, dims, mode, eb, d_out, out_capacity, d_out_bytes,
                                              d_ws, ws_bytes, stream);
  CompressCall call;
  st = check_compress(d_in, dims, mode, eb, d_out, out_capacity, d_ws, ws_bytes, &call, features_off);
  if (st != FSZ_OK || call.desc.nchunks == 0) return st;
  launch_compress(make_args(d_ws, call.L), reinterpret_cast<cudaStream_t>(stream), kCompressFeatures);
  return launched();
}

fsz_status fsz_compress_multipass(const float* d_in, fsz_dims dims, fsz_eb_mode mode, double eb,
                                  void* d_out, uint64_t out_capacity, uint64_t* d_out_bytes,
                                  uint32_t* d_costs, void* d_ws, uint64_t ws_bytes,
                                  fsz_stream stream) {
  if (d_costs == nullptr) return FSZ_ERR_INVALID_ARG;
  if (misaligned(d_costs)) return FSZ_ERR_ALIGN;
  CompressCall call;
  fsz_status st = check_compress(d_in, dims, mode, eb, d_out, out_capacity, d_ws, ws_bytes, &call);
  if (st != FSZ_OK) return st;
  st = prepare_one(d_in, dims, mode, eb, 0, d_out, out_capacity, d_out_bytes, d_ws, ws_bytes, stream);
  if (st != FSZ_OK || call.desc.nchunks == 0) return st;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  KernelArgs a = make_args(d_ws, call.L);
  for (int v = 0; v < 4; ++v) launch_cost_pass(a, v, d_costs, s);
  a.given_costs = d_costs;
  a.given_T = call.desc.T;
  launch_compress(a, s, kCompressGiven);
  return launched();
}

fsz_status fsz_decompress(const void* d_in, uint64_t in_bytes, float* d_out, uint64_t out_capacity_elems,
                          void* d_ws, uint64_t ws_bytes, fsz_stream stream) {
  return decompress_one(d_in, in_bytes, d_out, out_capacity_elems, d_ws, ws_bytes, stream,
                        kDecompressFull);
}

fsz_status fsz_decompress_prezeroed(const void* d_in, uint64_t in_bytes, float* d_out,
                                    uint64_t out_capacity_elems, void* d_ws, uint64_t ws_bytes,
                                    fsz_stream stream) {
  return decompress_one(d_in, in_bytes, d_out, out_capacity_elems, d_ws, ws_bytes, stream,
                        kDecompressPrezeroed);
}

fsz_status fsz_decompress_any(const void* d_in, uint64_t in_bytes, float* d_out,
                              uint64_t out_capacity_elems, void* d_ws, uint64_t ws_bytes,
                              fsz_stream stream) {
  return decompress_one(d_in, in_bytes, d_out, out_capacity_elems, d_ws, ws_bytes, stream,
                        kDecompressAny);
}

fsz_status fsz_compress_batched(const fsz_cfield* d_fields, uint32_t nfields, uint64_t n_total,
                                void* d_ws, uint64_t ws_bytes, fsz_stream stream) {
  if (d_fields == nullptr || d_ws == nullptr || nfields == 0) return FSZ_ERR_INVALID_ARG;
  if (misaligned(d_ws)) return FSZ_ERR_ALIGN;
  const WsLayout L = ws_layout(n_total / kTile + nfields, nfields);
  if (ws_bytes < L.bytes) return FSZ_ERR_WORKSPACE;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (cudaMemsetAsync(d_ws, 0, L.bytes, s) != cudaSuccess) return FSZ_ERR_CUDA;
  const KernelArgs a = make_args(d_ws, L);
  launch_plan_compress(a, d_fields, nfields, L.chunk_cap, s);
  launch_stats(a, s);
  launch_compress(a, s, kCompressFeatures);  // fields may switch features off
  return launched();
}

fsz_status fsz_decompress_batched(const fsz_dfield* d_fields, uint32_t nfields,
                                  uint64_t n_total_capacity, void* d_ws, uint64_t ws_bytes,
                                  fsz_stream stream) {
  if (d_fields == nullptr || d_ws == nullptr || nfields == 0) return FSZ_ERR_INVALID_ARG;
  if (misaligned(d_ws)) return FSZ_ERR_ALIGN;
  const WsLayout L = ws_layout(n_total_capacity / kTile + nfields, nfields);
  if (ws_bytes < L.bytes) return FSZ_ERR_WORKSPACE;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (cudaMemsetAsync(d_ws, 0, L.bytes, s) != cudaSuccess) return FSZ_ERR_CUDA;
  const KernelArgs a = make_args(d_ws, L);
  launch_plan_decompress(a, d_fields, nfields, L.chunk_cap, s);
  launch_decompress(a, s);
  return launched();
}

// The status words are read on the caller's stream (an asynchronous copy, then a wait on
// that stream only), so a check never waits for work queued on other streams.
fsz_status fsz_check(const void* d_ws, fsz_stream stream) {
  if (d_ws == nullptr) return FSZ_ERR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  uint32_t status = 0;
  if (cudaMemcpyAsync(&status, d_ws, sizeof(status), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return FSZ_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return FSZ_ERR_CUDA;
  return static_cast<fsz_status>(status);
}

fsz_status fsz_check_batched(const void* d_ws, uint32_t nfields, uint32_t* h_status, fsz_stream stream) {
  if (d_ws == nullptr || (nfields > 0 && h_status == nullptr)) return FSZ_ERR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  std::vector<FieldInfo> fields(nfields);
  const uint8_t* ws = static_cast<const uint8_t*>(d_ws);
  uint32_t status = 0;
  if (nfields > 0 && cudaMemcpyAsync(fields.data(), ws + 256, sizeof(FieldInfo) * nfields,
                                     cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return FSZ_ERR_CUDA;
  if (cudaMemcpyAsync(&status, d_ws, sizeof(status), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return FSZ_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return FSZ_ERR_CUDA;
  for (uint32_t f = 0; f < nfields; ++f) h_status[f] = fields[f].status;
  return static_cast<fsz_status>(status);
}

fsz_status fsz_read_header(const void* h_first64, uint64_t* n, fsz_dims* dims, double* eb, float* step,
                           uint64_t* total_bytes) {
  if (h_first64 == nullptr) return FSZ_ERR_INVALID_ARG;
  const uint8_t* p = static_cast<const uint8_t*>(h_first64);
  auto u16 = [&](int o) { return uint32_t(p[o]) | (uint32_t(p[o + 1]) << 8); };
  auto u32 = [&](int o) { uint32_t v; std::memcpy(&v, p + o, 4); return v; };
  auto u64 = [&](int o) { uint64_t v; std::memcpy(&v, p + o, 8); return v; };
  if (std::memcmp(p, "FSZ1", 4) != 0 || u16(4) != 1) return FSZ_ERR_CORRUPT;
  const uint32_t nd = p[6];
  if (nd < 1 || nd > 3 || p[7] > 1) return FSZ_ERR_CORRUPT;
  const uint64_t nn = u64(8);
  fsz_dims d;
  std::memset(&d, 0, sizeof(d));
  d.ndim = nd;
  for (uint32_t k = 0; k < nd; ++k) d.dims[k] = u64(16 + 8 * k);
  uint64_t prod = 0;
  if (dims_count(d, &prod) != FSZ_OK || prod != nn) return FSZ_ERR_CORRUPT;
  if (!features_valid(u32(52))) return FSZ_ERR_CORRUPT;
  double e;
  std::memcpy(&e, p + 40, 8);
  float sv;
  uint32_t sb = u32(48);
  std::memcpy(&sv, &sb, 4);
  if (n) *n = nn;
  if (dims) *dims = d;
  if (eb) *eb = e;
  if (step) *step = sv;
  if (total_bytes) *total_bytes = 64 + 8 * ((nn + kTile - 1) / kTile) + u64(56);
  return FSZ_OK;
}

fsz_status fsz_set_schedule(uint32_t stats_ctas_per_sm, uint32_t compress_ctas_per_sm,
                            uint32_t decompress_ctas_per_sm) {
  if (stats_ctas_per_sm > 64 || compress_ctas_per_sm > 64 || decompress_ctas_per_sm > 64)
    return FSZ_ERR_INVALID_ARG;
  g_schedule.ctas[kSchedStats] = int(stats_ctas_per_sm);
  g_schedule.ctas[kSchedCompress] = int(compress_ctas_per_sm);
  g_schedule.ctas[kSchedDecompress] = int(decompress_ctas_per_sm);
  return FSZ_OK;
}

fsz_status fsz_set_schedule_ex(const fsz_schedule* sc) {
  if (sc == nullptr) {  // the defaults
    g_schedule = kDefaultSchedule;
    return FSZ_OK;
  }
  if (sc->stats_ctas_per_sm > 64 || sc->compress_ctas_per_sm > 64 || sc->decompress_ctas_per_sm > 64 ||
      sc->compress_ticket_chunks < 1 || sc->compress_ticket_chunks > uint32_t(kMaxTicketChunks) ||
      sc->compress_ticket_lead < 1 || sc->compress_ticket_lead > uint32_t(kMaxCompressLead) ||
      sc->decompress_ticket_chunks < 1 || sc->decompress_ticket_chunks > uint32_t(kMaxTicketChunks) ||
      sc->decompress_records < 2 * sc->decompress_ticket_chunks ||
      sc->decompress_records > uint32_t(kMaxDecRecords) || sc->min_tickets_per_cta > 64)
    return FSZ_ERR_INVALID_ARG;
  g_schedule.ctas[kSchedStats] = int(sc->stats_ctas_per_sm);
  g_schedule.ctas[kSchedCompress] = int(sc->compress_ctas_per_sm);
  g_schedule.ctas[kSchedDecompress] = int(sc->decompress_ctas_per_sm);
  g_schedule.c_ticket_chunks = int(sc->compress_ticket_chunks);
  g_schedule.c_ticket_lead = int(sc->compress_ticket_lead);
  g_schedule.d_ticket_chunks = int(sc->decompress_ticket_chunks);
  g_schedule.d_records = int(sc->decompress_records);
  g_schedule.min_tickets = int(sc->min_tickets_per_cta);
  return FSZ_OK;
}

fsz_status fsz_get_schedule(fsz_schedule* out) {
  if (out == nullptr) return FSZ_ERR_INVALID_ARG;
  out->stats_ctas_per_sm = uint32_t(g_schedule.ctas[kSchedStats]);
  out->compress_ctas_per_sm = uint32_t(g_schedule.ctas[kSchedCompress]);
  out->decompress_ctas_per_sm = uint32_t(g_schedule.ctas[kSchedDecompress]);
  out->compress_ticket_chunks = uint32_t(g_schedule.c_ticket_chunks);
  out->compress_ticket_lead = uint32_t(g_schedule.c_ticket_lead);
  out->decompress_ticket_chunks = uint32_t(g_schedule.d_ticket_chunks);
  out->decompress_records = uint32_t(g_schedule.d_records);
  out->min_tickets_per_cta = uint32_t(g_schedule.min_tickets);
  return FSZ_OK;
}

fsz_status fsz_get_schedule_limits(uint32_t* stats_max, uint32_t* compress_max, uint32_t* decompress_max,
                                   uint32_t* sms) {
  const LaunchCfg a = stats_cfg(), b = compress_cfg(), c = decompress_cfg();
  if (cudaGetLastError() != cudaSuccess) return FSZ_ERR_CUDA;
  if (stats_max) *stats_max = uint32_t(a.per);
  if (compress_max) *compress_max = uint32_t(b.per);
  if (decompress_max) *decompress_max = uint32_t(c.per);
  if (sms) *sms = uint32_t(b.sms);
  return FSZ_OK;
}

fsz_status fsz_graph_compress_batched(const fsz_cfield* d_fields, uint32_t nfields, uint64_t n_total,
                                      void* d_ws, uint64_t ws_bytes, fsz_graph* out) {
  return capture_graph([&](fsz_stream s) {
    return fsz_compress_batched(d_fields, nfields, n_total, d_ws, ws_bytes, s);
  }, out);
}

fsz_status fsz_graph_decompress_batched(const fsz_dfield* d_fields, uint32_t nfields,
                                        uint64_t n_total_capacity, void* d_ws, uint64_t ws_bytes,
                                        fsz_graph* out) {
  return capture_graph([&](fsz_stream s) {
    return fsz_decompress_batched(d_fields, nfields, n_total_capacity, d_ws, ws_bytes, s);
  }, out);
}

fsz_status fsz_graph_launch(fsz_graph g, fsz_stream stream) {
  if (g == nullptr) return FSZ_ERR_INVALID_ARG;
  return cudaGraphLaunch(g->exec, reinterpret_cast<cudaStream_t>(stream)) == cudaSuccess ? FSZ_OK
                                                                                     : FSZ_ERR_CUDA;
}

void fsz_graph_destroy(fsz_graph g) {
  if (g == nullptr) return;
  cudaGraphExecDestroy(g->exec);
  delete g;
}

void fsz_set_test_hooks(uint64_t skip_chunk, uint64_t timeout_ns) {
  g_skip_chunk = skip_chunk;
  g_timeout_ns = timeout_ns ? timeout_ns : kDefaultTimeoutNs;
}

const char* fsz_version(void) { return "fsz 1.0 sm_103a"; }

}  // extern "C"
