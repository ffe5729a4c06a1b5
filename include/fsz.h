/*
 * fsz.h - C ABI of the GB300 (sm_103a) FSZ compressor library.
 *
 * FSZ is the error-bounded lossy compressor for float32 arrays of "FSZ:
 * Breaking the Prediction-Throughput Trade-off in GPU Lossy Compression"
 * (arXiv 2607.15413). Compression quantizes each value with step 2*eb
 * (Sec. 4.2.2), runs first- or second-order Lorenzo prediction with the state
 * carried across the 8 blocks of every 256-element tile (Sec. 4.1), optionally
 * centred on the tile mean (Sec. 4.2.2), picks the cheapest of the four
 * variants per tile from one pass (Sec. 4.2.3), bit-plane encodes every
 * 32-element block (Sec. 4.3) and places the blocks with a device-wide
 * decoupled-lookback scan (Sec. 4.4). Decompression inverts every step
 * (Sec. 3.1, "Decompression"). Every reconstructed value d' satisfies
 * |d - d'| <= eb (Sec. 4.2.2, "Error-bound preservation"; Sec. 5.1).
 *
 * Stream layout (Sec. 3.1 "Compressed format", plus a 64-byte preamble of
 * this library): [preamble 64 B][rate header: 8 B per tile][tile data].
 * Preamble, little-endian: 0 magic "FSZ1"; 4 version u16 = 1; 6 ndim u8;
 * 7 eb mode u8; 8 n u64; 16/24/32 dims u64 (unused dims 0); 40 requested eb
 * f64; 48 step s f32; 52 features switched off u32 (fsz_feature_off bits; 0 for
 * the full method); 56 data bytes u64.
 *
 * Conventions for every call below:
 *  - Pointers named d_* are device pointers; h_* are host pointers. The caller
 *    owns every buffer; the library allocates no device memory on these paths.
 *  - Calls are asynchronous on `stream` and do not synchronise the host, so
 *    they can be captured into a CUDA graph. The return value reports only
 *    errors the host can see (arguments, alignment, sizes, launch failures).
 *    Errors found on the device (non-finite input, an error bound too small
 *    for the data, a corrupt stream, a lookback wait that ran out) are written
 *    to a status word inside the workspace and read back by fsz_check().
 *  - d_in, d_out and d_ws must be 16-byte aligned (FSZ_ERR_ALIGN otherwise).
 *  - The workspace must not be shared by calls that overlap on the GPU.
 */
#ifndef FSZ_H
#define FSZ_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Identical to cudaStream_t; declared here so that this header needs no CUDA header. */
typedef struct CUstream_st* fsz_stream;

typedef enum {
  FSZ_OK = 0,
  FSZ_ERR_INVALID_ARG = 1,  /* bad dims, eb <= 0 or not finite, unknown mode, null pointer */
  FSZ_ERR_ALIGN = 2,        /* a pointer is not 16-byte aligned */
  FSZ_ERR_NONFINITE = 3,    /* the field holds a NaN or an infinity (device-detected) */
  FSZ_ERR_EB_TOO_SMALL = 4, /* max|d| / (2 eb) beyond the quantizer's range (device-detected) */
  FSZ_ERR_CAPACITY = 5,     /* an output buffer is too small */
  FSZ_ERR_CORRUPT = 6,      /* the compressed stream is malformed (device-detected) */
  FSZ_ERR_TIMEOUT = 7,      /* a lookback wait ran past its time limit (device-detected) */
  FSZ_ERR_CUDA = 8,         /* a CUDA runtime call or a kernel launch failed */
  FSZ_ERR_WORKSPACE = 9,    /* the workspace is smaller than fsz_*_workspace_bytes() */
  FSZ_ERR_REJECTED = 10     /* a served request that can never fit the server's limits */
} fsz_status;

typedef enum { FSZ_EB_ABS = 0, FSZ_EB_REL = 1 } fsz_eb_mode;

/* Features of the method a compression may switch off, for the ablation of Sec. 6.4
 * (Table 7); 0 is the full method. FSZ_OFF_CROSS_BLOCK: every 32-element block restarts
 * from zero predecessors (independent blocks, as Sec. 2 C1 describes block-parallel
 * compressors) instead of carrying the state across blocks (Eq. 2). FSZ_OFF_CENTERING:
 * no centred variants (Sec. 4.2.2, variants 3-4). FSZ_OFF_LZ2: no second-order variants.
 * Centring is defined on the carried state (Eq. 4), so FSZ_OFF_CROSS_BLOCK requires
 * FSZ_OFF_CENTERING (FSZ_ERR_INVALID_ARG otherwise). The stream records the bits; a tile
 * that uses a switched-off feature is corrupt. fsz_decompress decodes streams with
 * centring or LZ2 switched off; a stream without the cross-block state needs
 * fsz_decompress_any (fsz_decompress and fsz_decompress_batched record
 * FSZ_ERR_INVALID_ARG for it). The compression and decompression kernels are built in
 * instances with and without the switched-off features' handling, so the full method
 * pays nothing for them. */
typedef enum { FSZ_OFF_CROSS_BLOCK = 1, FSZ_OFF_CENTERING = 2, FSZ_OFF_LZ2 = 4 } fsz_feature_off;

/* Shape metadata: n = dims[0] * ... * dims[ndim-1], row-major, dims[ndim-1] fastest.
 * The method itself is one-dimensional over the flattened array (Sec. 3.1). */
typedef struct {
  uint32_t ndim;     /* 1, 2 or 3 */
  uint32_t reserved; /* must be 0 */
  uint64_t dims[3];  /* entries beyond ndim are ignored */
} fsz_dims;

/* One field of a batched compression (lives in DEVICE memory, an array of nfields). */
typedef struct {
  const float* in;       /* device, 16-byte aligned, dims product elements */
  fsz_dims dims;
  uint32_t mode;         /* fsz_eb_mode */
  uint32_t features_off; /* fsz_feature_off bits; 0 for the full method */
  double eb;             /* absolute bound (ABS) or fraction of max - min (REL) */
  void* out;             /* device, 16-byte aligned */
  uint64_t out_capacity; /* bytes; fsz_compress_bound(n) always suffices */
  uint64_t* out_bytes;   /* device u64 receiving this field's stream size, or NULL */
} fsz_cfield;

/* One field of a batched decompression (lives in DEVICE memory, an array of nfields). */
typedef struct {
  const void* in;              /* device, 16-byte aligned stream */
  uint64_t in_bytes;           /* bytes readable at in (at least the stream size) */
  float* out;                  /* device, 16-byte aligned */
  uint64_t out_capacity_elems; /* elements writable at out */
} fsz_dfield;

/* ------------------------------------------------------------------ sizes */

/* Largest stream for n elements: 64 + 8 T + 772 T bytes, T = ceil(n / 256). A tile
 * costs at most 8 * (4 + 4 * 23) + 4 bytes because |q| stays below 2^21, so every residual
 * stays below 2^23 (Sec. 4.2.2, Eq. 3). */
uint64_t fsz_compress_bound(uint64_t n);

/* Workspace for fsz_compress / fsz_decompress of up to n elements. */
uint64_t fsz_workspace_bytes(uint64_t n);

/* Workspace for a batch of nfields fields holding n_total elements in all. */
uint64_t fsz_batch_workspace_bytes(uint64_t n_total, uint32_t nfields);

/* ------------------------------------------------------------------ single field */

/* Compress one field (Sec. 3.1 steps 1-5; eb per Sec. 5.1). Runs the value-range pass
 * (min, max, finiteness, and the step derived from them), then the single-pass
 * compression kernel. Writes the stream to d_out and its size to *d_out_bytes
 * (device u64, may be NULL). out_capacity must be at least 64 + 8T; a stream that
 * would exceed it sets FSZ_ERR_CAPACITY in the workspace status. */
fsz_status fsz_compress(const float* d_in, fsz_dims dims, fsz_eb_mode mode, double eb,
                        void* d_out, uint64_t out_capacity, uint64_t* d_out_bytes,
                        void* d_ws, uint64_t ws_bytes, fsz_stream stream);

/* fsz_compress with features of the method switched off (fsz_feature_off bits), for
 * ablation studies; features_off = 0 is fsz_compress. */
fsz_status fsz_compress_features(const float* d_in, fsz_dims dims, fsz_eb_mode mode, double eb,
                                 uint32_t features_off, void* d_out, uint64_t out_capacity,
                                 uint64_t* d_out_bytes, void* d_ws, uint64_t ws_bytes,
                                 fsz_stream stream);

/* The multipass evaluation that Sec. 6.3 ("Single-pass evaluation benefit") compares the
 * single-pass design against, for measuring that benefit: each of the four variants
 * (LZ1, LZ2, LZ1c, LZ2c) is costed in a pass of its own over the field, writing every
 * tile's cost (Eq. 3, plus 4 bytes for the mean of a centred variant) to
 * d_costs[v * T + t] (device, 4 T uint32, 16-byte aligned, T = ceil(n / 256)); a fifth
 * pass, the compression kernel, selects from those costs and encodes. The stream is the
 * same as fsz_compress's; the input is read five times instead of once. */
fsz_status fsz_compress_multipass(const float* d_in, fsz_dims dims, fsz_eb_mode mode, double eb,
                                  void* d_out, uint64_t out_capacity, uint64_t* d_out_bytes,
                                  uint32_t* d_costs, void* d_ws, uint64_t ws_bytes,
                                  fsz_stream stream);

/* The two halves of fsz_compress, for callers that time or schedule them apart.
 * fsz_compress_prepare: value-range pass (Sec. 5.1: eb = REL x (max - min)) and the
 * quantization step, written into the workspace. fsz_compress_encode: the single-pass
 * compression kernel (Sec. 3.1 steps 1-5) using the step in the workspace; it must
 * follow fsz_compress_prepare on the same workspace with the same arguments. */
fsz_status fsz_compress_prepare(const float* d_in, fsz_dims dims, fsz_eb_mode mode, double eb,
                                void* d_out, uint64_t out_capacity, uint64_t* d_out_bytes,
                                void* d_ws, uint64_t ws_bytes, fsz_stream stream);
fsz_status fsz_compress_encode(const float* d_in, fsz_dims dims, fsz_eb_mode mode, double eb,
                               void* d_out, uint64_t out_capacity, uint64_t* d_out_bytes,
                               void* d_ws, uint64_t ws_bytes, fsz_stream stream);

/* Decompress one stream (Sec. 3.1 "Decompression", steps d1-d5) into d_out.
 * out_capacity_elems also bounds the workspace needed (fsz_workspace_bytes of it). */
fsz_status fsz_decompress(const void* d_in, uint64_t in_bytes, float* d_out,
                          uint64_t out_capacity_elems, void* d_ws, uint64_t ws_bytes,
                          fsz_stream stream);

/* fsz_decompress into an output that already holds zeros: tiles whose 8 blocks all have
 * rate 0 and no mean decode to +0.0 and are neither decoded nor written (the pre-zero of
 * Sec. 3.1, which the paper enables above a compression ratio of 100). It pays off when
 * the zeros are already there (e.g. a buffer reused for sparse fields): on GB300 the full
 * decoder writes such a field at near the HBM write rate, so zero-filling first costs
 * more than it saves. Streams without the cross-block state are refused as by
 * fsz_decompress. */
fsz_status fsz_decompress_prezeroed(const void* d_in, uint64_t in_bytes, float* d_out,
                                    uint64_t out_capacity_elems, void* d_ws, uint64_t ws_bytes,
                                    fsz_stream stream);

/* fsz_decompress for any stream, including those compressed with FSZ_OFF_CROSS_BLOCK
 * (its inverse prediction restarts at every block). About 3 % slower than fsz_decompress
 * on the full method's streams, for which fsz_decompress is the call. */
fsz_status fsz_decompress_any(const void* d_in, uint64_t in_bytes, float* d_out,
                              uint64_t out_capacity_elems, void* d_ws, uint64_t ws_bytes,
                              fsz_stream stream);

/* ------------------------------------------------------------------ tile configurations */

/* The tile-configuration sweep of Sec. 6.5 (Table 8): `block` elements per block (32 or
 * 64) and `tile_blocks` blocks per tile (4, 8 or 16). A configured stream has tile_blocks
 * header bytes per tile and block-bit sign and plane words (block / 8 bytes, element j at
 * bit block - 1 - j, most significant byte first); the method word (preamble byte 52)
 * holds the configuration in bits 8-15 (0 for 32 x 8, the default). A generic two-read
 * path (a cost pass, a scan of tile sizes, an encoding pass; one warp per tile) for every
 * configuration; the default configuration's specialised single-pass kernels are
 * fsz_compress / fsz_decompress, and fsz_decompress refuses configured streams. */
uint64_t fsz_compress_bound_tiled(uint64_t n, uint32_t block, uint32_t tile_blocks);
/* Workspace for fsz_compress_tiled / fsz_decompress_tiled of up to n elements. */
uint64_t fsz_tiled_workspace_bytes(uint64_t n);
fsz_status fsz_compress_tiled(const float* d_in, fsz_dims dims, fsz_eb_mode mode, double eb,
                              uint32_t block, uint32_t tile_blocks, uint32_t features_off,
                              void* d_out, uint64_t out_capacity, uint64_t* d_out_bytes, void* d_ws,
                              uint64_t ws_bytes, fsz_stream stream);
/* Decodes a stream of any tile configuration (including the default). */
fsz_status fsz_decompress_tiled(const void* d_in, uint64_t in_bytes, float* d_out,
                                uint64_t out_capacity_elems, void* d_ws, uint64_t ws_bytes,
                                fsz_stream stream);

/* ------------------------------------------------------------------ quality */

/* Reconstruction quality for the rate-distortion evaluation of Sec. 6.2 (Fig. 8: PSNR
 * against bit rate). Written to DEVICE memory by fsz_quality_stats. */
typedef struct {
  uint64_t n;           /* elements compared */
  uint64_t over_bound;  /* elements with |d - d'| > eb (0 for a stream of this library) */
  double max_abs_err;   /* max |d - d'| */
  double sum_sq_err;    /* sum of (d - d')^2 */
  double min, max;      /* value range of the original d */
  double psnr_db;       /* 20 log10(max - min) - 10 log10(sum_sq_err / n); +inf if exact */
  double nrmse;         /* sqrt(sum_sq_err / n) / (max - min) (0 for a constant field) */
  double bit_rate;      /* bits per value: 8 stream_bytes / n */
} fsz_quality;

/* Workspace for fsz_quality_stats (a few hundred KB; independent of n). */
uint64_t fsz_quality_workspace_bytes(void);

/* Compares the original d_orig with its reconstruction d_recon (n float32 each, device,
 * 16-byte aligned) and writes the statistics to *d_out (device, 16-byte aligned).
 * Differences are float32 (exact for the close values a bounded reconstruction holds),
 * their squares summed in float32 over 8 elements and then in float64 in a fixed order:
 * the sum is deterministic and within a relative 1e-6 of the exact one. */
fsz_status fsz_quality_stats(const float* d_orig, const float* d_recon, uint64_t n, double eb,
                             uint64_t stream_bytes, fsz_quality* d_out, void* d_ws,
                             uint64_t ws_bytes, fsz_stream stream);

/* ------------------------------------------------------------------ batches */

/* Compress nfields fields in one persistent launch (plus a planning kernel and the
 * value-range pass): work items (field, chunk) are taken from one device ticket in
 * field-major order, each field keeps its own lookback flags and its own stream.
 * Each field's stream is byte-identical to fsz_compress of that field.
 * d_fields: DEVICE array of nfields fsz_cfield. */
fsz_status fsz_compress_batched(const fsz_cfield* d_fields, uint32_t nfields, uint64_t n_total,
                                void* d_ws, uint64_t ws_bytes, fsz_stream stream);

/* Decompress nfields streams in one persistent launch (plus a planning kernel).
 * d_fields: DEVICE array of nfields fsz_dfield. n_total_capacity = sum of the fields'
 * out_capacity_elems (sizes the workspace). */
fsz_status fsz_decompress_batched(const fsz_dfield* d_fields, uint32_t nfields,
                                  uint64_t n_total_capacity, void* d_ws, uint64_t ws_bytes,
                                  fsz_stream stream);

/* ------------------------------------------------------------------ graphs and schedules */

/* A CUDA graph holding one batched call (no counterpart in the paper: it removes the
 * host launch cost of the call's memset and kernels). The graph records the pointers and
 * sizes given here; the field tables and buffers they point to are read when the graph
 * runs, so their contents may change between launches, but not their addresses or the
 * number of fields. The graph itself holds host-side and driver resources only. */
typedef struct fsz_graph_s* fsz_graph;
fsz_status fsz_graph_compress_batched(const fsz_cfield* d_fields, uint32_t nfields, uint64_t n_total,
                                      void* d_ws, uint64_t ws_bytes, fsz_graph* out);
fsz_status fsz_graph_decompress_batched(const fsz_dfield* d_fields, uint32_t nfields,
                                        uint64_t n_total_capacity, void* d_ws, uint64_t ws_bytes,
                                        fsz_graph* out);
/* Runs the graph on `stream` (asynchronous); device status as for the captured call. */
fsz_status fsz_graph_launch(fsz_graph g, fsz_stream stream);
void fsz_graph_destroy(fsz_graph g);

/* Launch schedule for later calls in this process: persistent CTAs per SM for the
 * value-range, compression and decompression kernels; 0 = as many as fit (the default).
 * Values above what fits are clamped. Used by the autotuner; not thread-safe. */
fsz_status fsz_set_schedule(uint32_t stats_ctas_per_sm, uint32_t compress_ctas_per_sm,
                            uint32_t decompress_ctas_per_sm);
/* How many CTAs of each kernel fit per SM, and the SM count, on the current device. */
fsz_status fsz_get_schedule_limits(uint32_t* stats_max, uint32_t* compress_max,
                                   uint32_t* decompress_max, uint32_t* sms);

/* The full launch schedule (no counterpart in the paper, which fixes one tile-to-block
 * mapping; none of it changes a stream). The persistent kernels hand out work by atomic
 * tickets; a ticket covers `*_ticket_chunks` consecutive chunks of 32 tiles (1-4), the
 * unit of work a CTA takes, and in each of its chunks after the first the chunk's byte
 * offset follows from the previous one without a lookback (Sec. 4.4). Compression takes
 * tickets up to `compress_ticket_lead` chunks (1-3) ahead of its compute warps;
 * decompression keeps up to `decompress_records` chunks (2 x ticket chunks .. 16) between
 * ticket and decode per CTA. A launch whose chunks would give fewer than
 * `min_tickets_per_cta` tickets per CTA (0-64) at the requested ticket size takes tickets
 * of fewer chunks (down to 1), so that small fields and small batches still spread over
 * every CTA; 0 keeps the requested size at every launch size. Defaults: CTAs 0 (as many
 * as fit), compression 2 chunks per ticket with lead 2, decompression 4 chunks per ticket
 * and 16 records, 4 tickets per CTA. Read by every later call of this process at launch
 * (a CUDA graph keeps the schedule it was captured with). Used by the autotuner; not
 * thread-safe. */
typedef struct fsz_schedule {
  uint32_t stats_ctas_per_sm;
  uint32_t compress_ctas_per_sm;
  uint32_t decompress_ctas_per_sm;
  uint32_t compress_ticket_chunks;
  uint32_t compress_ticket_lead;
  uint32_t decompress_ticket_chunks;
  uint32_t decompress_records;
  uint32_t min_tickets_per_cta;
} fsz_schedule;
/* Installs `s` (NULL: the defaults). FSZ_ERR_INVALID_ARG if a field is out of range; the
 * schedule in force is then unchanged. */
fsz_status fsz_set_schedule_ex(const fsz_schedule* s);
/* The schedule in force (host pointer). */
fsz_status fsz_get_schedule(fsz_schedule* out);

/* ------------------------------------------------------------------ status and metadata */

/* Waits for `stream`, then returns the first device-detected error recorded in the
 * workspace by the last call that used it (FSZ_OK if none). For batches, the first
 * error of any field. */
fsz_status fsz_check(const void* d_ws, fsz_stream stream);

/* Per-field status of the last batched call (host array of nfields); waits for stream. */
fsz_status fsz_check_batched(const void* d_ws, uint32_t nfields, uint32_t* h_status,
                             fsz_stream stream);

/* Parses a stream's 64-byte preamble from HOST memory. Any output may be NULL. */
fsz_status fsz_read_header(const void* h_first64, uint64_t* n, fsz_dims* dims, double* eb,
                           float* step, uint64_t* total_bytes);

/* ------------------------------------------------------------------ no-allocation variant */

/* Largest field fsz_compress_noalloc accepts (2^28 elements, 1 GiB of float32). */
#define FSZ_NOALLOC_MAX_ELEMS (1ull << 28)

/* fsz_compress for callers that cannot allocate device memory (no counterpart in the
 * paper; an addition of this library). Examples: plugins whose host framework owns all
 * device memory through its own pool (an allocation of their own would be refused or
 * unaccounted for); latency-critical paths that cannot take the synchronisation an
 * allocation may cause.
 * The caller passes only the input and output buffers; the scratch the kernels need
 * lives in a fixed device array of about 0.8 MiB inside the library, which every GPU that
 * loads the library holds until the process exits. The function allocates nothing.
 *  - n above FSZ_NOALLOC_MAX_ELEMS returns FSZ_ERR_WORKSPACE; other argument errors as
 *    fsz_compress.
 *  - The first call on each device does that device's one-time set-up: it looks up the
 *    array's device address and sets the compression kernels' attributes (their dynamic
 *    shared-memory size) and reads their occupancy there, all non-stream runtime calls;
 *    make that first call before any stream capture begins.
 *  - All calls share the one array and each clears the part it uses on `stream`. Calls
 *    whose work overlaps on the GPU (different streams or threads without ordering)
 *    race on it and produce wrong streams: order them on one stream or serialise them.
 *  - d_status (device u32, may be NULL) receives the device-detected status of this
 *    call (0 = FSZ_OK); the stream and d_out_bytes are as for fsz_compress. */
fsz_status fsz_compress_noalloc(const float* d_in, fsz_dims dims, fsz_eb_mode mode, double eb,
                                void* d_out, uint64_t out_capacity, uint64_t* d_out_bytes,
                                uint32_t* d_status, fsz_stream stream);

/* ------------------------------------------------------------------ serving */

/* A continuous-batching request server (no counterpart in the paper: the serving pattern
 * this library adds around the batched path). Clients submit compress and decompress
 * requests whose inputs are on the device; one native scheduler thread owns every GPU call:
 *  - Arrival: a request enters the queue at its arrival_ns (at once if that has passed or
 *    is 0), in submission order: submitting requests ahead of their arrival times replays
 *    a trace without a client thread on the clock.
 *  - Admission: requests are admitted in arrival order while the device-memory budget
 *    allows. The budget counts the output memory the server allocates for a request (see
 *    fsz_server_request_cost) from its admission until the client releases its output,
 *    so the output memory the server holds never exceeds the budget: a client that keeps
 *    outputs, or polls completions slowly, holds back admission. A
 *    request that can never fit (cost above the whole budget, or more elements than a
 *    batch may hold) completes at once with FSZ_ERR_REJECTED. A request that does not fit
 *    yet waits at the head of the queue; later requests do not overtake it.
 *  - Batching: the head's kind (compress or decompress) picks the batch. It takes up to
 *    max_batch waiting requests of that kind in arrival order, reaching past requests of
 *    the other kind within a window of `scan` requests while holding their memory in
 *    reserve, so a skipped request still fits when its own batch goes next. A batch runs as
 *    one fsz_compress_batched / fsz_decompress_batched call on the first free slot (a
 *    stream of its own, with its own workspace). Requests that arrive while batches run
 *    are admitted and launched as slots and budget free up. With linger_us > 0, while
 *    other batches are running, a batch short of max_batch is launched only once its
 *    first request has waited linger_us, so that small requests arriving close together
 *    share a batch; an idle server launches at once.
 *  - Completion: a CUDA event per batch; each request's completion carries its status
 *    (that field's device status), its output and its latency (arrival to completion on
 *    the host's monotonic clock).
 * Outputs live in one device allocation per batch, from a memory pool of the server's own.
 * An output stays valid until fsz_server_release, which returns its cost to the budget;
 * the batch's allocation is freed when all its outputs are released. Every completion other
 * than FSZ_ERR_REJECTED must be released. Stopping (fsz_server_stop, fsz_server_destroy)
 * refuses, with FSZ_ERR_REJECTED, requests still waiting for memory that only a release
 * would return.
 * With sim_service_ns > 0 the server makes no CUDA call: a batch completes that long after
 * its launch, outputs are NULL (for testing the scheduling rules without a GPU). */
typedef struct fsz_server_s* fsz_server;
typedef enum { FSZ_REQ_COMPRESS = 0, FSZ_REQ_DECOMPRESS = 1 } fsz_request_kind;

typedef struct {
  uint64_t budget_bytes;     /* output memory the server may hold */
  uint32_t slots;            /* concurrent batches, 1..16 */
  uint32_t max_batch;        /* requests per batch, 1..4096 */
  uint32_t scan;             /* waiting requests looked at per batch (0: 4 * max_batch) */
  uint32_t linger_us;        /* while batches run, a batch short of max_batch waits up to this
                                long after its first request's arrival for more (0: none) */
  uint64_t max_batch_elems;  /* most elements one batch may hold; sizes the workspaces */
  uint64_t sim_service_ns;   /* 0 for the GPU; > 0 for the no-GPU test mode */
} fsz_server_config;

typedef struct {
  uint64_t id;          /* the caller's tag, returned with the completion */
  uint32_t kind;        /* fsz_request_kind */
  uint32_t mode;        /* compress: fsz_eb_mode */
  fsz_dims dims;        /* compress: the field's shape; decompress: unused (zeros) */
  double eb;            /* compress: the error bound */
  const void* d_in;     /* device: the float32 field, or the stream (16-byte aligned) */
  uint64_t in_bytes;    /* decompress: the stream's size */
  uint64_t n;           /* decompress: the element count */
  uint64_t arrival_ns;  /* monotonic clock (CLOCK_MONOTONIC) of arrival; 0 = at submission */
} fsz_request;

typedef struct {
  uint64_t id;
  int32_t status;       /* fsz_status of this request */
  uint32_t batch_size;  /* requests in its batch */
  uint64_t batch;       /* its batch's launch index (0, 1, ...); UINT64_MAX if rejected */
  void* d_out;          /* device: the stream (compress) or the float32 values (decompress) */
  uint64_t out_bytes;   /* the stream's size, or 4n */
  uint64_t latency_ns;  /* arrival to completion */
} fsz_completion;

typedef struct {
  uint64_t submitted, completed, rejected, batches, max_inflight, max_batch_seen;
  uint64_t admitted_while_busy, budget_free, bytes_in;
} fsz_server_stats;

/* Output bytes the server charges to its budget for a request (its allocation, rounded). */
uint64_t fsz_server_request_cost(const fsz_request* req);
fsz_status fsz_server_create(const fsz_server_config* cfg, fsz_server* out);
/* Queues a request (thread-safe, non-blocking). Argument errors are returned here. */
fsz_status fsz_server_submit(fsz_server s, const fsz_request* req);
/* Queues `count` requests from the host array h_reqs in order, under one lock; all or none
 * (the first argument error is returned and nothing is queued). */
fsz_status fsz_server_submit_many(fsz_server s, const fsz_request* h_reqs, uint64_t count);
/* Copies up to `max` completions to h_out, waiting up to wait_ns for the first; returns
 * how many (thread-safe). */
uint32_t fsz_server_poll(fsz_server s, fsz_completion* h_out, uint32_t max, uint64_t wait_ns);
/* Gives back request id's output; the memory is freed in order on `stream` once every
 * output of its batch has been released (thread-safe). */
fsz_status fsz_server_release(fsz_server s, uint64_t id, fsz_stream stream);
/* fsz_server_release for each of the `count` ids in h_ids; returns FSZ_ERR_INVALID_ARG if
 * any id was not held (the others are released all the same). */
fsz_status fsz_server_release_many(fsz_server s, const uint64_t* h_ids, uint64_t count,
                                   fsz_stream stream);
fsz_status fsz_server_get_stats(fsz_server s, fsz_server_stats* h_stats);
/* Stops the server: no further submissions are accepted; queued and running work is
 * finished, except requests that wait for memory only a release would return, which
 * complete with FSZ_ERR_REJECTED. Completions stay available to fsz_server_poll until
 * fsz_server_destroy (a polling thread can drain them first). Thread-safe; returns at once. */
fsz_status fsz_server_stop(fsz_server s);
/* fsz_server_stop, then waits for the scheduler to finish and frees the server. Outputs
 * not yet released are freed with it. */
fsz_status fsz_server_destroy(fsz_server s);
/* Device-to-device copy on `stream` (for clients without a CUDA binding of their own). */
fsz_status fsz_copy_device(void* d_dst, const void* d_src, uint64_t bytes, fsz_stream stream);

/* Test hooks for failure detection (not for production use): the chunk whose global
 * index equals skip_chunk publishes no lookback flag, so its successor's bounded wait
 * runs out after timeout_ns and records FSZ_ERR_TIMEOUT; the kernels still finish.
 * skip_chunk = UINT64_MAX disables the hook; timeout_ns = 0 restores the default (2 s). */
void fsz_set_test_hooks(uint64_t skip_chunk, uint64_t timeout_ns);

/* Library version and build target, e.g. "fsz 1.0 sm_103a". */
const char* fsz_version(void);

#ifdef __cplusplus
}
#endif

#endif /* FSZ_H */
