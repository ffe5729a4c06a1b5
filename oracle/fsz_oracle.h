/*
 * FSZ CPU oracle: TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded restatement of the FSZ compressed stream
 * ("FSZ: Breaking the Prediction-Throughput Trade-off in GPU Lossy
 * Compression", arXiv 2607.15413). Only the test suite, the smoke check and
 * the benchmark's CPU-baseline leg may load it. It shares no code, header,
 * table or constant with the CUDA library; the two agree because both follow
 * the paper and the readings of it fixed for this project.
 *
 * Conventions: element arrays are row-major float32, n = product of dims,
 * tiles of 256 elements = 8 blocks of 32 (Sec. 3.1 "Data organization").
 * Functions return one of the FSZO_* status codes.
 */
#ifndef FSZ_ORACLE_H
#define FSZ_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  FSZO_OK = 0,
  FSZO_ERR_INVALID_ARG = 1,
  FSZO_ERR_NONFINITE = 3,
  FSZO_ERR_EB_TOO_SMALL = 4,
  FSZO_ERR_CAPACITY = 5,
  FSZO_ERR_CORRUPT = 6
};

enum { FSZO_EB_ABS = 0, FSZO_EB_REL = 1 };

/* Variants in the paper's listed order (Sec. 4.2.2, "Four-Way Cost Analysis"). */
enum { FSZO_LZ1 = 0, FSZO_LZ2 = 1, FSZO_LZ1C = 2, FSZO_LZ2C = 3 };
/* Features of the method that can be switched off, for the ablation of Sec. 6.4 (0: the
 * full method). OFF_CROSS: every block restarts from zero predecessors (independent
 * blocks); OFF_CENTER: no centred variants; OFF_LZ2: no second-order variants. Centring is
 * defined on the carried state, so OFF_CROSS requires OFF_CENTER. The stream's preamble
 * records the bits (u32 at byte 52). */
enum { FSZO_OFF_CROSS = 1, FSZO_OFF_CENTER = 2, FSZO_OFF_LZ2 = 4 };

typedef struct {
  double eb;      /* absolute bound promised to the caller (ABS as given, REL x range) */
  double eb_eff;  /* eb clamped to at most 2^100 */
  double K;       /* A / (2 eb_eff (1 - 2^-4)) */
  uint32_t Q;     /* bound on |q|: ceil(K) + 1 */
  float e;        /* half step: eb_eff (1 - eps) rounded toward zero to float32 */
  float s;        /* quantization step 2e */
  float r;        /* 1/s in float32 */
} fszo_params_t;

/* Value range and finiteness of the field (Sec. 5.1, REL definition). */
int fszo_stats(const float* d, uint64_t n, float* vmin, float* vmax, int* all_finite);

/* Absolute bound and FP32-safe step (REL definition of Sec. 5.1; error-bound
 * argument of Sec. 4.2.2 made to hold in float32 arithmetic). */
int fszo_params(int mode, double eb_req, float vmin, float vmax, int all_finite,
                uint64_t n, fszo_params_t* p);

/* q = round(d / (2 eb)) as t = fl32(d * r), q = nearest integer, ties to even (Sec. 4.2.2). */
int32_t fszo_quantize(float d, float r);
/* d' = fl32(float(q) * s). */
float fszo_dequantize(int32_t q, float s);

/* Tile mean in the quantized domain, mu = round(mean / (2 eb)) (Sec. 4.2.2, variant 3). */
int32_t fszo_tile_mu(const float d[256], float r);

/* Residuals of one variant over a whole tile with zero-initialised predecessors and
 * the state carried across the 8 block boundaries (Eqs. 1-2 and Sec. 4.2.2). */
void fszo_tile_residuals(const int32_t q[256], int32_t mu, int variant, int32_t l[256]);

/* Block rate r_b = ceil(log2(max|l| + 1)) (Sec. 4.1.2) and block cost S_b (Eq. 3). */
uint32_t fszo_rate(uint32_t maxabs);
uint32_t fszo_block_cost(uint32_t rate);

/* Four-way costs from one pass over the tile (Sec. 4.2.3): LZ1 and LZ2 in one loop,
 * centred costs by adjusting block 0 only (Eq. 4). rates[v*8+b]. */
void fszo_tile_costs_single_pass(const int32_t q[256], int32_t mu, uint32_t C[4], uint8_t rates[32]);
/* The same four costs from four separate full passes (the naive evaluation). */
void fszo_tile_costs_four_pass(const int32_t q[256], int32_t mu, uint32_t C[4], uint8_t rates[32]);
/* First strict minimum in listed order (Sec. 4.2.2: "selects the variant with the minimum C"). */
int fszo_select(const uint32_t C[4]);

/* Worst-case stream size for n elements: 64 + 8T + 772T bytes (rates stay <= 23). */
uint64_t fszo_compress_bound(uint64_t n);

/* Whole-field compression. force_variant = -1 selects per tile (the method);
 * 0..3 forces one variant for every tile (test hook for the decoder). */
int fszo_compress(const float* d, uint32_t ndim, const uint64_t* dims, int mode, double eb_req,
                  uint8_t* out, uint64_t out_capacity, uint64_t* out_bytes, int force_variant);

/* Tiles [t0, t1) of a field, encoded with the given r = 1/s: their 8-byte rate headers
 * (8 (t1 - t0) bytes) and their data, as they appear in the whole field's stream. */
int fszo_compress_tiles(const float* d, uint64_t n, float r, uint64_t t0, uint64_t t1,
                        uint8_t* header_out, uint8_t* data_out, uint64_t data_cap,
                        uint64_t* data_bytes);

/* Parses the 64-byte preamble. */
int fszo_read_preamble(const uint8_t* in, uint64_t in_bytes, uint64_t* n, uint32_t* ndim,
                       uint64_t dims[3], double* eb_req, float* s, uint64_t* data_bytes);

/* The functions above with features switched off (FSZO_OFF_* bits; 0 = the full method).
 * Single-pass costs without the carried state cover LZ1 and LZ2 only (C = UINT32_MAX for
 * the centred ones); the four-pass costs evaluate all four residual sets as defined. */
int fszo_features_valid(uint32_t off);
void fszo_tile_residuals_f(const int32_t q[256], int32_t mu, int variant, uint32_t off,
                           int32_t l[256]);
void fszo_tile_costs_single_pass_f(const int32_t q[256], int32_t mu, uint32_t off, uint32_t C[4],
                                   uint8_t rates[32]);
void fszo_tile_costs_four_pass_f(const int32_t q[256], int32_t mu, uint32_t off, uint32_t C[4],
                                 uint8_t rates[32]);
int fszo_select_f(const uint32_t C[4], uint32_t off);
int fszo_compress_f(const float* d, uint32_t ndim, const uint64_t* dims, int mode, double eb_req,
                    uint32_t off, uint8_t* out, uint64_t out_capacity, uint64_t* out_bytes,
                    int force_variant);
int fszo_compress_tiles_f(const float* d, uint64_t n, float r, uint64_t t0, uint64_t t1,
                          uint32_t off, uint8_t* header_out, uint8_t* data_out,
                          uint64_t data_cap, uint64_t* data_bytes);
int fszo_read_preamble_f(const uint8_t* in, uint64_t in_bytes, uint64_t* n, uint32_t* ndim,
                         uint64_t dims[3], double* eb_req, float* s, uint64_t* data_bytes,
                         uint32_t* features_off);
/* Tile configurations (Sec. 6.5, Table 8): B elements per block (32 or 64), T blocks per
 * tile (4, 8 or 16). A configured stream has T header bytes per tile and B-bit sign and
 * plane words (B / 8 bytes, element j at bit B - 1 - j, most significant byte first); the
 * method word at byte 52 carries the configuration in bits 8-15 (fszo_tile_word; 0 for
 * B = 32, T = 8) besides the switched-off features. fszo_compress_cfg evaluates the four
 * variants by definition (one residual pass each); fszo_decompress decodes every
 * configuration. */
uint32_t fszo_tile_word(int B, int T);
uint64_t fszo_compress_bound_cfg(uint64_t n, int B, int T);
int fszo_compress_cfg(const float* d, uint32_t ndim, const uint64_t* dims, int mode, double eb_req,
                      uint32_t off, int B, int T, uint8_t* out, uint64_t out_capacity,
                      uint64_t* out_bytes);
/* Reconstruction quality for the rate-distortion evaluation of Sec. 6.2 (Fig. 8: PSNR
 * against bit rate). Differences in float64: max |d - d'|, the sum of (d - d')^2 (in
 * element order), elements with |d - d'| > eb, the original's min and max; then
 * PSNR = 20 log10(max - min) - 10 log10(sum / n) (+inf for an exact reconstruction),
 * NRMSE = sqrt(sum / n) / (max - min), bit rate = 8 stream_bytes / n. */
typedef struct {
  uint64_t n, over_bound;
  double max_abs_err, sum_sq_err, vmin, vmax, psnr_db, nrmse, bit_rate;
} fszo_quality_t;
int fszo_quality(const float* d, const float* y, uint64_t n, double eb, uint64_t stream_bytes,
                 fszo_quality_t* q);
/* Whole-stream decompression (Sec. 3.1 "Decompression", steps d1-d5). */
/* The 64-byte preamble of a stream (this project's addition). */
void fszo_write_preamble(uint8_t* out, uint32_t ndim, const uint64_t* dims, uint64_t n, int mode,
                         double eb_req, float s, uint32_t method_word, uint64_t data_bytes);
/* Tiles [t0, t1) of a default-configuration stream whose first tile starts data_off bytes
 * into the data region: elements [256 t0, min(n, 256 t1)) into out (from element 256 t0). */
int fszo_decompress_tiles(const uint8_t* in, uint64_t in_bytes, uint64_t t0, uint64_t t1,
                          uint64_t data_off, float* out);
int fszo_decompress(const uint8_t* in, uint64_t in_bytes, float* out, uint64_t out_capacity_elems,
                    uint64_t* n_out);
/* Same, but returns the reconstructed integers q instead of floats. */
int fszo_decompress_q(const uint8_t* in, uint64_t in_bytes, int32_t* q_out,
                      uint64_t out_capacity_elems, uint64_t* n_out);

#ifdef __cplusplus
}
#endif

#endif
