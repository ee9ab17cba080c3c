/*
 * jxl_recon.h - C ABI of the GB300 VarDCT pixel-reconstruction library.
 *
 * The library turns already entropy-decoded VarDCT data of the JPEG XL
 * committee draft (ISO/IEC 18181 CD, 2019) into pixels on one GPU:
 *
 *   F.2  DC dequantisation            dc = m_DC[c] * q
 *   F.3  AC dequantisation            bias, * AcMul, * dequant matrix (C.6.1)
 *   G    chroma from luma             X += kX * Y, B += kB * Y
 *   I.2.7 LLF from DC, I.2.4 inverse transforms of all 15 varblock shapes
 *   J.2  edge-preserving filter       (optional, C.10 `epf`)
 *   J.4  Gaborish                     (optional, C.10 `gab`)
 *   L.2  XYB -> linear RGB            then f32 / f16 linear or 8-bit sRGB
 *
 * Entropy decoding and codestream parsing are the caller's: the inputs are
 * the decoded fields of C.5.3-C.5.6 and C.8 as plain arrays.
 *
 * Conventions for every call:
 *  - Pointers are plain host or device addresses; sizes are element counts
 *    unless named *_bytes.  No call takes or returns framework objects.
 *  - The caller owns every buffer it passes.  Inputs and outputs, host or
 *    device, must stay valid and unmodified until jxl_recon_poll() for that
 *    ticket returns something other than JXLR_EAGAIN / JXLR_ETIMEDOUT (host
 *    buffers are copied asynchronously on the request's stream).
 *  - A negative jxlr_status is an error; jxl_recon_last_error() then holds
 *    a message for the calling thread.
 *  - Thread safety: one context may be driven by one submitting thread and
 *    one polling thread at the same time.
 */
#ifndef JXL_RECON_H_
#define JXL_RECON_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct jxl_recon_ctx jxl_recon_ctx;

typedef enum {
  JXLR_OK = 0,
  JXLR_EAGAIN = 1,         /* poll: the request has not finished yet          */
  JXLR_EINVAL = -1,        /* ill-formed input: varblock map not a tiling
                              (C.5.4), non-positive/infinite matrix (C.6.1),
                              bad sizes, strides or flags                     */
  JXLR_ENOMEM = -2,        /* the request alone exceeds the HBM cap, or a
                              device allocation failed                         */
  JXLR_EBUSY = -3,         /* admission refused for now (no free slot or not
                              enough free HBM under the cap): retry later     */
  JXLR_ECUDA = -4,         /* a CUDA runtime call failed                      */
  JXLR_ETIMEDOUT = -5,     /* poll: the timeout expired (request still runs)  */
  JXLR_ECANCELLED = -6     /* request dropped by jxl_recon_destroy()          */
} jxlr_status;

/* Output sample encodings.  All are interleaved [ysize][xsize][3] with the
 * caller's row stride.  Linear outputs are L.2's RGB divided by 255 (so the
 * nominal range is [0, 1]; samples outside it are kept).  U8_SRGB applies
 * the IEC 61966-2-1 transfer curve to clamp(linear, 0, 1) and rounds half
 * up.  F32_XYB returns the X, Y, B samples unchanged (L.2, colour_space ==
 * kXYB), after the enabled loop filters. */
typedef enum {
  JXLR_OUT_F32_LINEAR = 0,
  JXLR_OUT_F16_LINEAR = 1,
  JXLR_OUT_U8_SRGB = 2,
  JXLR_OUT_F32_XYB = 3
} jxlr_out_dtype;

typedef enum {
  JXLR_PREC_FP32 = 0,      /* every stage on FP32 CUDA cores                    */
  JXLR_PREC_TC_F16X3 = 1   /* the separable passes of varblocks larger than 8x8
                              (I.2.4.1) run on the tensor cores as FP16 hi/lo
                              split products (hi*hi + hi*lo + lo*hi) with FP32
                              accumulation, each operand row scaled by a power
                              of two; everything else as in FP32 mode         */
} jxlr_precision;

typedef struct {
  int device;              /* CUDA device ordinal                             */
  size_t hbm_cap_bytes;    /* device bytes the context may hold for request
                              scratch and staged inputs; 0 = no cap           */
  int max_slots;           /* requests in flight at once (>= 1); each slot
                              owns one CUDA stream and its scratch arena      */
  int precision;           /* a jxlr_precision                                */
  int timing;              /* 1: record CUDA events around every kernel so
                              jxl_recon_stage_ms() can report them            */
  void* cuda_stream;       /* NULL: one library stream per slot; else a
                              cudaStream_t of the caller that every slot
                              enqueues on (requests then run in order)        */
} jxl_recon_config;

/* Quantised coefficients (C.8), one int16 plane per channel X, Y, B, in the
 * varblock footprint layout: the coefficient (u, v) of the varblock whose
 * top-left sample is (x0, y0) is stored at column x0 + u, row y0 + v, u
 * horizontal frequency.  The LLF slots (u < W/8, v < H/8) of a W x H
 * varblock hold the quantised DC samples of its 8x8 blocks (x0/8 + u,
 * y0/8 + v) (F.2, I.2.7).  Planes cover the image padded to multiples of 8:
 * ceil8(ysize) rows of row_stride_elems >= ceil8(xsize) elements.
 * on_device: 1 = every input array of this submit (coefficients, maps,
 * quant field, CfL map, sharpness) is a device pointer; 0 = host pointers. */
typedef struct {
  uint32_t xsize, ysize;
  const int16_t* plane[3];
  size_t row_stride_elems;
  int on_device;
} jxl_recon_coeffs;

/* Chroma from luma (G, C.4.3, C.5.3): k = (kX, kB) pairs per 64x64 tile,
 * [ceil(Hp/64)][ceil(Wp/64)][2] float, and the DC factors.  The draft's u8
 * factors map to these by kX = (x - 128) / 256, kB = 0.935669 + (b - 128)/128. */
typedef struct {
  const float* k;
  float kx_dc, kb_dc;
} jxl_recon_cfl;

/* Loop filter (C.10), DC (C.4.1) and colour (L.2, A.4.5) parameters.
 * jxl_recon_filter_defaults() fills the draft's defaults with both filters
 * off.  sharpness: uint8 per 8x8 block [Hp/8][Wp/8] (C.5.6), same memory
 * space as the other inputs, needed only when epf != 0.  dequant: NULL for
 * the default matrices of C.6.1.1, or a host array of 10560 floats holding,
 * for code 0..14 and then channel 0..2, the H x W matrix row-major. */
typedef struct {
  int gab;
  float gab_w1[3], gab_w2[3];
  int epf;
  float epf_weight_min;
  float epf_scale[3];
  float epf_sharp_lut[8];
  float epf_range_max, epf_range_mul, epf_quant_mul;
  uint32_t epf_sigma_max;
  const uint8_t* sharpness;
  float m_dc[3];
  float inv_opsin[9];
  float opsin_bias[3];
  uint32_t target_nits_div50;
  const float* dequant;
  /* F.2 adaptive DC smoothing: 1 applies it, 0 skips it (the effect of
   * kSkipAdaptiveDCSmoothing).  The window half-width is m_dc / 2 (DC
   * quantisation without extra levels, C.5.2). */
  int dc_smooth;
  /* Annex H AC prediction from the DC2x2 image of each 256 x 256 group:
   * 1 applies it, 0 skips it (the effect of kSkipPredictLf). */
  int lf_predict;
  /* J.3 quantization constraint after the EPF (only with epf != 0): 1
   * applies it, clamping each coefficient of the filter residual to
   * +-qco_interval_mul times its interval (C.10: default 0.5). */
  int qco;
  float qco_interval_mul;
  /* K.5 noise synthesis after Gaborish (kNoise): 1 adds the noise of each
   * 256 x 256 group with the strength LUT of C.4.8 (16 entries, the decoded
   * u(10) / 1024 values). */
  int noise;
  float noise_lut[16];
} jxl_recon_filter_params;

/* Caller-owned output buffer of ysize rows, row_stride_bytes apart. */
typedef struct {
  void* data;
  size_t row_stride_bytes;
  int dtype;               /* a jxlr_out_dtype                                */
  int on_device;           /* 1: device buffer; 0: host buffer, written by a
                              copy that completes before poll returns OK      */
} jxl_recon_output;

/* Fills *p with the defaults of C.10, C.4.1 (m_DC of the synthetic
 * workloads: (0.02, 0.2, 0.2) / (64 sqrt 2)) and L.2; both filters, DC
 * smoothing, AC prediction, the quantization constraint and noise off. */
void jxl_recon_filter_defaults(jxl_recon_filter_params* p);

/* Creates a context on config->device: builds the constant tables (C.6.1
 * matrices, I.2.7 LLF maps, J.2.4 mul_table), one stream per slot.
 * Returns JXLR_OK and *out, or JXLR_EINVAL / JXLR_ECUDA. */
jxlr_status jxl_recon_create(const jxl_recon_config* config, jxl_recon_ctx** out);

/* Enqueues the reconstruction of one image and returns at once with a
 * ticket; the work runs on the slot's stream.  varblock_map: uint8 per 8x8
 * block [Hp/8][Wp/8], row-major, holding the DctSelect code (C.5.4, 0..14)
 * at a varblock's top-left block and 0xFF on the other blocks it covers.
 * quant_field: AcMul (C.5.5) as float per 8x8 block [Hp/8][Wp/8]; the
 * value at a varblock's top-left block applies to the whole varblock.
 * Host inputs are validated here (JXLR_EINVAL); device inputs are
 * validated on the device and reported by jxl_recon_poll().
 * Returns JXLR_OK, JXLR_EBUSY (no slot or no HBM now), JXLR_ENOMEM,
 * JXLR_EINVAL or JXLR_ECUDA. */
jxlr_status jxl_recon_submit(jxl_recon_ctx* ctx, const jxl_recon_coeffs* coeffs,
                             const uint8_t* varblock_map, const float* quant_field,
                             const jxl_recon_cfl* cfl_map,
                             const jxl_recon_filter_params* filter_params,
                             const jxl_recon_output* out, uint64_t* ticket);

/* Runs only the loop filters and the colour transform (J.2, J.4, L.2) on
 * XYB samples the caller already has: xyb is a device array of 3 planes
 * [3][ysize][row_stride_elems] float.  varblock_map and quant_field as in
 * jxl_recon_submit (device pointers; they define the EPF ranges and
 * sigma of J.2.4).  Same ticket semantics. */
jxlr_status jxl_recon_submit_xyb(jxl_recon_ctx* ctx, const float* xyb,
                                 uint32_t xsize, uint32_t ysize,
                                 size_t row_stride_elems,
                                 const uint8_t* varblock_map, const float* quant_field,
                                 const jxl_recon_filter_params* filter_params,
                                 const jxl_recon_output* out, uint64_t* ticket);

/* ---- JPEG1 direct rasterisation (M.6) ------------------------------------
 * One component of a JPEG1 coefficient stream.  coeffs: int16
 * [height_in_blocks][width_in_blocks][64] in the natural order of M.6.1
 * (index 8u + v, u the vertical and v the horizontal frequency), in the
 * memory space the stream's on_device names; quant: the component's 64
 * quantisation factors in the same order, always host memory.  h_samp,
 * v_samp: sampling factors (1 or 2); a component whose factor is below the
 * largest one is upsampled 2x along that axis (M.6.4).  gab: 1 when the
 * block-conditional Gaborish side channel of M.6.3 is present, with its
 * decoded weights (u(8) / 1024), threshold (u(8) / 16) and limit; cond: 1
 * when the coefficients are to be conditioned (M.6.1.1). */
typedef struct {
  uint32_t width_in_blocks, height_in_blocks;
  uint32_t h_samp, v_samp;
  const int16_t* coeffs;
  const uint16_t* quant;
  int gab;
  float gab_w1, gab_w2, gab_threshold;
  int gab_limit;
  /* 1: the DC / AC conditioning of M.6.1.1 with its max_gap and min_step
   * (u(8) / 64 from the side channel, or 0.5 / 0.5 by the decoder's choice). */
  int cond;
  float cond_max_gap, cond_min_step;
} jxl_jpeg_component;

/* num_components: 1 (grey) or 3 (Y, Cb, Cr).  The block grids must cover
 * the image: 8 x width_in_blocks x (largest h_samp / h_samp) >= xsize, and
 * likewise vertically.  on_device: 1 = coeffs are device pointers that stay
 * valid until poll returns something other than JXLR_EAGAIN; 0 = host. */
typedef struct {
  uint32_t xsize, ysize;
  uint32_t num_components;
  jxl_jpeg_component comp[3];
  int on_device;
} jxl_jpeg_stream;

/* Enqueues M.6.1 (dequantisation, with the M.6.1.1 conditioning of the
 * components that ask for it), M.6.2 (IDCT_2D), M.6.3, M.6.4, M.6.5 (YCbCr
 * -> RGB) and M.6.6 (cropping) for one stream.  The HDR transform of
 * M.6.5.1 is not performed.  Output: JXLR_OUT_U8_SRGB gives the rasterised samples
 * clamped to [0, 255] and rounded half up (no transfer function is applied:
 * the samples are already in the JPEG's colour encoding); F32_LINEAR and
 * F16_LINEAR give sample / 255 unclamped; F32_XYB is rejected.  Same ticket
 * semantics as jxl_recon_submit.  Returns JXLR_OK, JXLR_EINVAL, JXLR_EBUSY,
 * JXLR_ENOMEM or JXLR_ECUDA. */
jxlr_status jxl_recon_submit_jpeg(jxl_recon_ctx* ctx, const jxl_jpeg_stream* stream,
                                  const jxl_recon_output* out, uint64_t* ticket);

/* Waits up to timeout_us (0 = just test, < 0 = forever) for a ticket.
 * JXLR_OK when done (the ticket is then released; *latency_ms, if not
 * NULL, receives submit-to-completion time), JXLR_EAGAIN / JXLR_ETIMEDOUT
 * while running, JXLR_EINVAL for a device-side validation failure or an
 * unknown ticket, JXLR_ECUDA on a CUDA error. */
jxlr_status jxl_recon_poll(jxl_recon_ctx* ctx, uint64_t ticket, int64_t timeout_us,
                           double* latency_ms);

/* Device time of each stage of a finished request, in ms, when the
 * context was created with timing = 1: ms[0] validation, ms[1]
 * dequantisation + transforms, ms[2] filters + colour, ms[3] host<->device
 * copies.  Call after jxl_recon_poll() returned JXLR_OK for the ticket;
 * the values stay until the next completed request of that slot. */
jxlr_status jxl_recon_stage_ms(jxl_recon_ctx* ctx, uint64_t ticket, float ms[4]);

/* The edge-preserving filter of a finished request (J.2; context created
 * with timing = 1): *epf_ms is the device time of its kernel alone (part of
 * ms[2] of jxl_recon_stage_ms()), *epf_blocks the number of 8x8 blocks it
 * filtered, i.e. those with sigma >= 16 (J.2.4); the samples of the other
 * blocks pass through unchanged.  Both 0 when the request had no EPF or was
 * a batch / JPEG1 request.  Call after jxl_recon_poll() returned JXLR_OK. */
jxlr_status jxl_recon_epf_stats(jxl_recon_ctx* ctx, uint64_t ticket, float* epf_ms,
                                uint32_t* epf_blocks);

/* One request of a serving schedule: the arguments of jxl_recon_submit(). */
typedef struct {
  const jxl_recon_coeffs* coeffs;
  const uint8_t* varblock_map;
  const float* quant_field;
  const jxl_recon_cfl* cfl_map;
  const jxl_recon_filter_params* filter_params;
  const jxl_recon_output* out;
} jxl_recon_request;

typedef struct {
  double makespan_s;       /* first arrival to last completion                  */
  uint64_t busy_refusals;  /* admissions refused (no slot / HBM) and retried     */
  uint64_t completed;      /* requests finished                                  */
  uint32_t max_in_flight;  /* most requests running at once                      */
  uint64_t bypassed;       /* requests admitted ahead of an older refused one    */
} jxl_recon_serve_stats;

/* Request server (the draft's data-parallel decoding of independent images,
 * 6.2 / 6.4, as a service; no counterpart in the draft's text).  A
 * long-lived thread admits enqueued requests into the context as slots and
 * HBM under its cap free up (continuous batching): it scans the queue in
 * arrival order and submits each request the context accepts; a request
 * refused for want of HBM is passed by smaller ones behind it until it has
 * waited longer than age_bound_ms, after which nothing behind it is
 * admitted first.  Admitted requests run concurrently on their slots'
 * streams; the context runs each on a stream whose priority rises with the
 * image size (one level per factor of 4 in pixels from 256 Kpx), so large
 * requests, which set the tail latency, take the SMs they need and small
 * ones fill the rest.
 * jxl_recon_server_enqueue() is safe from any thread and returns at once; the
 * request's buffers (and, for host inputs, its host arrays) must stay valid
 * until jxl_recon_server_wait() returned for it.  wait: timeout_us < 0
 * blocks, 0 polls (JXLR_EAGAIN), > 0 waits at most that long
 * (JXLR_ETIMEDOUT); latency_ms = completion - enqueue.  A request that
 * submit rejects (JXLR_EINVAL, JXLR_ENOMEM, JXLR_ECUDA) reports that status
 * from wait.  stop drains the queue, joins the thread, fills stats (may be
 * NULL) and frees the server. */
typedef struct jxl_recon_server jxl_recon_server;
typedef struct {
  double age_bound_ms;     /* longest wait a refused request lets others pass   */
  int bypass;              /* 0: strict arrival order                           */
  double exclusive_mpx;    /* requests of at least this many Mpx run alone: one
                              is admitted only onto an idle device (the queue
                              behind it waits too) and nothing joins it; 0: off */
} jxl_recon_server_config;
jxlr_status jxl_recon_server_start(jxl_recon_ctx* ctx, const jxl_recon_server_config* cfg,
                                   jxl_recon_server** out);
jxlr_status jxl_recon_server_enqueue(jxl_recon_server* server, const jxl_recon_request* req,
                                     uint64_t* id);
jxlr_status jxl_recon_server_wait(jxl_recon_server* server, uint64_t id, int64_t timeout_us,
                                  double* latency_ms);
jxlr_status jxl_recon_server_stop(jxl_recon_server* server, jxl_recon_serve_stats* stats);

/* Replay of an arrival schedule through a request server (age bound 5 ms,
 * images of 8 Mpx and more alone):
 * the calling thread enqueues reqs[0..n) at arrival_s[i] seconds after the
 * call (non-decreasing) and waits for all.  latency_ms[i] receives
 * completion - arrival of request i (queueing included).  With max_slots = 1
 * the context runs one image at a time: the plain path.  Returns JXLR_OK, or
 * the first error a request produced (the others still complete). */
jxlr_status jxl_recon_serve(jxl_recon_ctx* ctx, const jxl_recon_request* reqs, size_t n,
                            const double* arrival_s, double* latency_ms,
                            jxl_recon_serve_stats* stats);

/* Multi-image batches (the draft's independent groups, 6.2, taken across
 * images): many uneven images reconstructed by one launch per kernel kind,
 * captured once in a CUDA graph and replayed by jxl_recon_batch_launch().
 * Every request must be device-resident (inputs and output) with the
 * default dequantisation matrices, and the context must have been created
 * with JXLR_PREC_FP32 (JXLR_EINVAL otherwise); the batch owns the scratch of all its
 * images (XYB, sigma, and with the EPF its output and block list;
 * allocated at creation).  Maps are validated at creation (JXLR_EINVAL).
 * With JXLR_BATCH_AUTOTUNE the grids of the three kernel kinds (transform,
 * J.2, Gaborish / colour) and the form of the last (TMA tiles or ordinary
 * loads) are chosen by timing candidates on this batch, all of which give
 * the same bits; the choice is remembered per batch class (images,
 * transform cells, images with the EPF, filter tiles, output-type mix) in
 * the process and in $JXLR_AUTOTUNE_CACHE if set.  Otherwise a remembered
 * choice is used, else one CTA per transform cell and filter tile (the J.2
 * kernel and the TMA form on their resident grids).  The inputs and outputs
 * of the requests must stay valid for the batch's lifetime. */
typedef struct jxl_recon_batch jxl_recon_batch;
#define JXLR_BATCH_AUTOTUNE 1
/* The Gaborish / colour kernel of the batch loads its tiles with ordinary
 * loads instead of TMA (the same results; without it the TMA form is used
 * whenever every filtered image's scratch allows it). */
#define JXLR_BATCH_PLAIN_LOADS 2

typedef struct {
  uint32_t images;
  uint64_t pixels;
  uint32_t recon_items, epf_items, filter_items;   /* cells / images with the EPF / tiles */
  int recon_grid, epf_grid, filter_grid;           /* CTAs per launch */
  int kernels_per_launch;
  int autotuned;                                   /* 0 no, 1 tuned now, 2 cached */
  int filter_tma;                                  /* 1: the Gaborish / colour kernel loads
                                                      its tiles by TMA */
  float kind_ms[3];                                /* tuned time of each kernel kind (0 if
                                                      not timed), ms */
  uint32_t mix;                                    /* output types: counts of u8, f16, f32
                                                      images in bits 0-7, 8-15, 16-23 */
} jxl_recon_batch_info;

jxlr_status jxl_recon_batch_create(jxl_recon_ctx* ctx, const jxl_recon_request* reqs, size_t n,
                                   int flags, jxl_recon_batch** out);
/* Enqueues the whole batch on cuda_stream (a cudaStream_t; NULL = legacy
 * default stream) and returns; completion is the stream's. */
jxlr_status jxl_recon_batch_launch(jxl_recon_batch* batch, void* cuda_stream);
jxlr_status jxl_recon_batch_query(const jxl_recon_batch* batch, jxl_recon_batch_info* info);
/* Error flags of the batch's launches so far (call once the launch's stream
 * has completed; a blocking device read): bit 8 = a bounded tile-load wait
 * of the Gaborish / colour kernel expired (its output is then not valid);
 * 0 = none.  JXLR_EINVAL on a null argument, JXLR_ECUDA if the read fails. */
jxlr_status jxl_recon_batch_status(const jxl_recon_batch* batch, uint32_t* flags);
jxlr_status jxl_recon_batch_destroy(jxl_recon_batch* batch);

/* Number of kernels the context has launched so far. */
uint64_t jxl_recon_launch_count(const jxl_recon_ctx* ctx);

/* Device bytes currently held by the context's slots. */
size_t jxl_recon_device_bytes(const jxl_recon_ctx* ctx);

/* Waits for all requests, frees everything.  Tickets not yet polled are
 * dropped (a later poll on them cannot happen: the context is gone). */
jxlr_status jxl_recon_destroy(jxl_recon_ctx* ctx);

/* Message of the last error on the calling thread ("" if none). */
const char* jxl_recon_last_error(const jxl_recon_ctx* ctx);

/* Size of the fixed device scratch of jxl_recon_run_noalloc(). */
#define JXL_RECON_NOALLOC_SCRATCH_BYTES ((size_t)64 << 20)

/* Reconstruction for callers that cannot allocate device memory.  (The
 * draft has no counterpart: this is a deployment variant of the submit
 * path.)  Some callers may not call cudaMalloc: a framework or service that
 * must account for every device byte through its own allocator, or code
 * for which an allocation's implicit device synchronisation is not
 * allowed.  This call creates no context and allocates no device memory
 * (host memory only for the tables it builds on its first call per device
 * and for error messages): the scratch of the transform kernel (planar XYB and
 * per-block EPF sigma, 12 B per padded pixel + 2 B per 8x8 block) is a
 * fixed array of JXL_RECON_NOALLOC_SCRATCH_BYTES inside the library, held
 * by every GPU that loads it until the process exits; a padded image that
 * needs more (about 5.5 Mpx with a loop filter on; no limit with both off)
 * is rejected with JXLR_EINVAL.
 * Inputs as for jxl_recon_submit() and all on the device (coeffs->on_device
 * = 1, out->on_device = 1); filter_params->dequant must be NULL (default
 * matrices).  The map is not validated: an ill-formed map gives unspecified
 * pixels but no out-of-bounds access (a varblock whose code is above 14 or
 * whose footprint is misaligned, leaves its 32x32 cell or the padded image
 * is skipped; a block no varblock covers is left unfiltered).  With the
 * EPF off and Gaborish on, the tiles are read with ordinary loads, so no
 * device wait can expire unreported.  The kernels are enqueued on
 * cuda_stream (a cudaStream_t; NULL = the legacy default stream) of the
 * current device and the call returns without waiting.
 * The first call on a device copies the constant tables to it and looks up
 * the scratch address; make that first call before any stream capture.
 * All calls share the scratch: calls whose work overlaps on the GPU race and
 * give wrong pixels, so order them on one stream.  Nothing needs clearing
 * between calls (every scratch element read is written first).
 * Returns JXLR_OK, JXLR_EINVAL (message in jxl_recon_last_error(NULL)) or
 * JXLR_ECUDA. */
jxlr_status jxl_recon_run_noalloc(const jxl_recon_coeffs* coeffs, const uint8_t* varblock_map,
                                  const float* quant_field, const jxl_recon_cfl* cfl_map,
                                  const jxl_recon_filter_params* filter_params,
                                  const jxl_recon_output* out, void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* JXL_RECON_H_ */
