/*
 * szgb.h -- C ABI of the GB300 (sm_103a) error-bounded lossy compressor for
 * FP32 1D/2D/3D/4D arrays: multilayer prediction from preceding decompressed
 * values (arXiv:1706.03791 Sec. III, Eq. predmodel), error-controlled
 * linear-scaling quantization into 2^m - 1 intervals with a truncated binary
 * representation for unpredictable values (Sec. IV-A, Sec. IV-B, Algorithm
 * 1), canonical Huffman coding of the quantization codes (Sec. IV-A), and the
 * matching decompression.
 *
 * Conventions
 *  - Every pointer is a plain host or device address; a flag argument says
 *    which.  The caller owns every buffer: the library never frees caller
 *    memory and keeps no caller pointer after a call returns.
 *  - Device buffers must be 4-byte aligned (16-byte alignment is faster).
 *  - shape[] lists extents slowest -> fastest (C order); only the first ndim
 *    entries are read.  Points are at most 2^32 - 1 per field.
 *  - Work is issued on the context's stream (szgb_set_stream); every entry
 *    point returns after the stream has finished the call's work.
 *  - Return value 0 on success, a negative SZGB_E* code otherwise
 *    (szgb_strerror gives the text).  On error, output buffers hold
 *    unspecified bytes.
 *  - A context is not thread-safe; use one per host thread.
 *
 * Stream format: a 128-byte little-endian header, a codebook of
 * (u16 symbol, u8 length) for the used quantization codes, one byte length
 * per chunk as u16 or u32, then the byte-padded chunks, each holding, for
 * every point, its canonical Huffman code (MSB first) and, after a code 0, the
 * unpredictable value's sign, exponent and top t mantissa bits.  A chunk is a
 * whole row (fastest-axis line), or C consecutive points of one (header byte
 * 116 holds C, 0 for whole rows); chunks follow row by row.  The same bytes are produced by the CPU oracle of the test-suite.
 * The format also carries 4D fields (the predictor of Sec. III in four
 * dimensions; ndim 4 at header byte 8, the slowest extent at byte 120, the
 * other three at bytes 16-40).  Every call but the autotuner takes them.
 */
#ifndef SZGB_H
#define SZGB_H
#include <stddef.h>
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

/* error codes */
#define SZGB_OK 0
#define SZGB_EINVAL (-1)      /* bad argument (shape, bound, n, m, alignment) */
#define SZGB_ENONFINITE (-2)  /* input holds NaN or Inf */
#define SZGB_ETRUNC (-3)      /* output buffer too small; needed size reported */
#define SZGB_ECORRUPT (-4)    /* stream fails a consistency check */
#define SZGB_ENOMEM (-5)      /* device allocation failed */
#define SZGB_EBUDGET (-6)     /* call needs more device memory than the budget */
#define SZGB_ETIMEOUT (-7)    /* a bounded device-side wait ran out */
#define SZGB_ECUDA (-8)       /* a CUDA runtime call failed */
#define SZGB_EUNSUPPORTED (-9)/* valid request this build does not run on GPU */
#define SZGB_ESCRATCH (-10)   /* request needs more than the fixed scratch of
                                 szgb_decompress_noalloc */

/* error-bound modes (Sec. II, metric 1): absolute, value-range relative,
 * or both (the smaller bound applies) */
#define SZGB_ABS 0
#define SZGB_REL 1
#define SZGB_ABS_AND_REL 2

typedef struct szgb_ctx szgb_ctx;

typedef struct {
    int ndim;           /* 1, 2, 3 or 4 */
    uint64_t shape[4];  /* extents, slowest -> fastest; entries past ndim
                           are ignored.  4D: shape[0] x shape[1] and the
                           point count below 2^32, the exact variant only */
    int mode;           /* SZGB_ABS / SZGB_REL / SZGB_ABS_AND_REL */
    double eb_abs;      /* absolute bound (>= 0), modes ABS, ABS_AND_REL */
    double eb_rel;      /* relative bound (>= 0) times (max - min) */
    int layers;         /* n of the n-layer predictor (Sec. III-B; the
                           paper's default is 1): 1..4 in every dimension
                           (the autotuner tunes the wavefront: 1D-3D with
                           n <= 2 in 3D) */
    int m;              /* 2..16: 2^m - 1 intervals; 0 = adaptive (Sec. IV-B) */
    double theta;       /* adaptive-m hit-rate threshold, e.g. 0.99 */
    int variant;        /* SZGB_VARIANT_EXACT (0): the paper's method;
                           SZGB_VARIANT_LATTICE (1): the separately labelled
                           lattice variant (below) */
    uint32_t chunk_points; /* Huffman chunk length along a row: a power of
                           two >= 32 cuts every row's payload into chunks of
                           that many points (decoded in parallel);
                           SZGB_CHUNK_ROWS: one chunk per row; 0: the size the
                           autotuner chose for the field's shape class, else
                           one chunk per row.  A length at least the row's
                           gives one chunk per row.  The lattice variant
                           always codes whole rows. */
} szgb_params;

#define SZGB_CHUNK_ROWS 0xFFFFFFFFu

/* The lattice variant is NOT the paper's method: values are first snapped to
 * the lattice of spacing 2 eb_f (p = rint(x * (1/(2 eb_f))) in binary32,
 * |p| < 2^30, eb_f > 0), the integer field is predicted by the same n-layer
 * coefficients from the neighbours' lattice values (not from decompressed
 * values), and the residual is coded like a quantization code; outliers
 * (residual beyond the radius, or a lattice value that misses the bound)
 * store the residual in 64 bits and, when needed, x exactly.  Every point
 * is still within the bound.  Compression and decompression are fully
 * parallel (no wavefront).  Its streams carry tag 1 in header byte 113 and
 * are never produced unless requested.  1D-3D with n <= 2; batches run such
 * fields one by one on their own kernels; the no-allocation path returns
 * SZGB_EUNSUPPORTED for its streams. */
#define SZGB_VARIANT_EXACT 0
#define SZGB_VARIANT_LATTICE 1

typedef struct {
    uint64_t n_points;      /* points in the field */
    uint64_t n_unpred;      /* unpredictable points (code 0) */
    uint64_t stream_bytes;  /* size of the compressed stream */
    int m;                  /* interval bits used (chosen when adaptive) */
    int maxlen;             /* longest Huffman code */
    uint32_t nsym;          /* quantization codes in use */
    float eb_f;             /* effective bound: largest float <= eb */
    float xmin, xmax;       /* value range of the input */
    int status;             /* 0, or this field's SZGB_E* code (batches) */
} szgb_stats;

/* Creates a context on CUDA device `device` that keeps at most
 * `device_mem_budget` bytes of device scratch (0 = no limit).  *out is set
 * on success.  Scratch is allocated on first use and kept for reuse. */
int szgb_create(szgb_ctx **out, int device, size_t device_mem_budget);
/* Frees the context and its scratch.  NULL is ignored. */
void szgb_destroy(szgb_ctx *ctx);
/* Issue work on `cuda_stream` (a cudaStream_t; NULL = the context's own
 * stream). */
int szgb_set_stream(szgb_ctx *ctx, void *cuda_stream);

/* Upper bound of the stream size for these parameters (bytes). */
size_t szgb_compress_bound(const szgb_params *p);

/* Compresses the FP32 array `data` (host or device) into `out` (host or
 * device, out_cap bytes).  *out_len receives the stream size, also when
 * SZGB_ETRUNC reports that out_cap is too small.  opt_stats may be NULL.
 * Fails with SZGB_ENONFINITE on NaN/Inf input, SZGB_EINVAL on bad
 * parameters.  Layers 1..4 in every dimension: 3D fields with n = 3, 4 and
 * 4D fields run on the tiled hyperplane kernels (one launch per diagonal of
 * tiles), 1D-3D fields otherwise on the wavefront.  A 4D field's stream says
 * ndim = 4 and keeps shape[0] at header byte 120; its rows of shape[3]
 * points are coded as those of the (shape[0] shape[1]) x shape[2] x shape[3]
 * view, whose szgb_compress_bound it never exceeds. */
int szgb_compress(szgb_ctx *ctx, const float *data, int data_on_device,
                  const szgb_params *p, uint8_t *out, size_t out_cap,
                  int out_on_device, size_t *out_len, szgb_stats *opt_stats);

/* As szgb_compress with device buffers only, and additionally writes (when
 * the pointers are not NULL, device memory, one entry per point in raster
 * order) the values the compressor recorded for later predictions -- the
 * exact decompressed values -- and the quantization codes.  For testing. */
int szgb_compress_trace(szgb_ctx *ctx, const float *data_dev, const szgb_params *p,
                        uint8_t *out_dev, size_t out_cap, size_t *out_len,
                        szgb_stats *opt_stats, float *recorded_dev,
                        uint16_t *codes_dev);

/* 4D fields (Sec. III: the n-layer predictor of Eq. predmodel with d = 4;
 * quantization and coding as for 1D-3D) with trace outputs: as
 * szgb_compress_trace of the device array data_dev with p->ndim = 4 and
 * p->shape = shape[0..3] (p->ndim and p->shape are ignored; the exact
 * variant only).  recorded_dev and codes_dev are NULL or device arrays of
 * one entry per point.  Errors as szgb_compress. */
int szgb_compress_4d(szgb_ctx *ctx, const float *data_dev, const uint64_t *shape,
                     const szgb_params *p, uint8_t *out_dev, size_t out_cap, size_t *out_len,
                     szgb_stats *opt_stats, float *recorded_dev, uint16_t *codes_dev);

/* Decompresses `in` (host or device, in_len bytes) into `out` (host or
 * device; out_cap_elems floats, at least the number of points).
 * SZGB_ECORRUPT when the stream is inconsistent. */
int szgb_decompress(szgb_ctx *ctx, const uint8_t *in, size_t in_len,
                    int in_on_device, float *out, size_t out_cap_elems,
                    int out_on_device);

/* Decompression that allocates no memory, for callers that cannot call
 * cudaMalloc: a service that keeps a fixed device-memory plan for its whole
 * life (an allocation that could fail, or fragment a planned pool, at an
 * arbitrary moment is not allowed there), or code running inside an
 * allocator or framework callback, where allocating would re-enter the
 * allocator.  The paper has no counterpart: this is an operational variant
 * of szgb_decompress with identical output.
 *  - in_dev (in_len bytes, 4-byte aligned) and out_dev (out_cap_elems floats,
 *    16-byte aligned) are device buffers owned by the caller, on the current
 *    device; work is issued on `cuda_stream` (a cudaStream_t of the current
 *    device, NULL = legacy default stream).  The call copies the 128-byte
 *    header to the host and waits for the stream twice (before the kernels,
 *    to read the header, and at the end); it returns after the stream has
 *    finished its work.
 *  - Scratch is a fixed 128 MiB static device array held by every GPU that
 *    loads the library until the process exits; a stream whose decompression
 *    needs more returns SZGB_ESCRATCH before any work is issued.
 *  - The first call on a device looks up that array's device address
 *    (cudaGetSymbolAddress, once per device).
 *  - Every call on a device shares the array; calls whose work overlaps on
 *    the GPU race.  It never calls cudaMalloc/cudaFree or an allocating
 *    library routine.
 *  - Errors: SZGB_EINVAL (null or misaligned buffer, out too small),
 *    SZGB_ECORRUPT (inconsistent stream), SZGB_EUNSUPPORTED (streams of
 *    the lattice variant), SZGB_ESCRATCH,
 *    SZGB_ETIMEOUT, SZGB_ECUDA, as szgb_decompress. */
int szgb_decompress_noalloc(const uint8_t *in_dev, size_t in_len, float *out_dev,
                            size_t out_cap_elems, void *cuda_stream);

/* Batched compression of `count` independent fields, all in device memory:
 * field i is data_dev[i] with params[i], its stream goes to out_dev[i]
 * (out_cap[i] bytes, 4-byte aligned; data 16-byte aligned).  The result of
 * every field is the same as szgb_compress of that field alone.  The
 * wavefronts of all fields run in one persistent launch (one per layer
 * count present); the per-field range, histogram, codebook and encoding
 * kernels overlap on auxiliary streams; the whole sequence is captured in a
 * CUDA graph on the first call and replayed while the arguments (pointers,
 * capacities, parameters) repeat (szgb_set_graphs(ctx, 0) launches directly
 * instead).  out_len[i] receives each stream size, also on SZGB_ETRUNC;
 * opt_stats is NULL or holds count entries.  Returns 0 or the error of the
 * first field (in batch order) that failed.  Fields the wavefront does not
 * carry (3D n = 3, 4; 4D; the lattice variant) run after the batch's
 * wavefront fields, one at a time on their own kernels, outside the graph.
 * A bad parameter of any field fails the call before any work. */
int szgb_compress_batch(szgb_ctx *ctx, int count, const float *const *data_dev,
                        const szgb_params *params, uint8_t *const *out_dev,
                        const size_t *out_cap, size_t *out_len, szgb_stats *opt_stats);

/* Batched decompression: stream i (in_dev[i], in_len[i] bytes, 4-byte
 * aligned) into out_dev[i] (out_cap_elems[i] floats, 16-byte aligned), all
 * device memory; one persistent wavefront launch as above (streams of
 * fields the wavefront does not carry run one at a time after it).
 * opt_status is NULL or receives count per-field codes. */
int szgb_decompress_batch(szgb_ctx *ctx, int count, const uint8_t *const *in_dev,
                          const size_t *in_len, float *const *out_dev,
                          const size_t *out_cap_elems, int *opt_status);

/* Autotuner.  Times compression + decompression of the device field
 * `data_dev` (params p) for every candidate wavefront shape (compute warps
 * per CTA: 2,4,6,8 in 3D, 1,2,4,8 in 1D/2D), then, with the fastest shape,
 * for every candidate Huffman chunk length (whole rows, 128, 256, 512, 1024
 * points, those shorter than a row), best of `reps` runs each, and keeps the
 * fastest pair for the field's shape class (dimension, layers, bit lengths
 * of planes/rows/columns); later calls on fields of that class with
 * chunk_points = 0 use it.  The shape changes the schedule only; the chunk
 * length changes the stream's chunking (and size) but not the decompressed
 * values.  *W_out and *ms_out (may be NULL) receive the shape and its time;
 * *pub_out receives the chosen chunk length (SZGB_CHUNK_ROWS for whole
 * rows).  SZGB_EUNSUPPORTED for 3D fields with n > 2 and 4D fields, which
 * do not run on the wavefront. */
int szgb_autotune(szgb_ctx *ctx, const float *data_dev, const szgb_params *p, int reps,
                  int *W_out, int *pub_out, double *ms_out);
/* As szgb_autotune for a batch: times szgb_compress_batch +
 * szgb_decompress_batch of the given device fields for every candidate
 * shape (compute warps per CTA 1,2,4,6,8), then for the chunk lengths whole
 * rows, 128 and 512 points, and keeps the fastest pair for every shape class
 * in the batch: the shape that is best for one field alone is often not the
 * one that fills the GPU best when many fields share it. */
int szgb_autotune_batch(szgb_ctx *ctx, int count, const float *const *data_dev,
                        const szgb_params *params, int reps, int *W_out, int *pub_out,
                        double *ms_out);
/* Save / load the autotuned table (a small text file). */
int szgb_tune_save(szgb_ctx *ctx, const char *path);
int szgb_tune_load(szgb_ctx *ctx, const char *path);

/* Capture batches in CUDA graphs (1, the default) or launch them directly (0). */
int szgb_set_graphs(szgb_ctx *ctx, int on);

/* Caps the grid of this context's persistent wavefront launches at
 * max_ctas CTAs (one CTA per SM; 0 = one per SM of the device, the
 * default).  A persistent launch holds its SMs until its last work item is
 * done, so kernels issued meanwhile on other streams (even higher-priority
 * ones) wait for SMs; a cap leaves the other SMs free for them (the serving
 * loop caps its large requests this way).  Changes the schedule only, never
 * the results.  SZGB_EINVAL for a negative cap. */
int szgb_set_wave_ctas(szgb_ctx *ctx, int max_ctas);

/* ---- test hooks for the bounded device-side waits -------------------------
 * Not part of the method (the paper has no counterpart): they let a test make
 * the wavefront's bounded waits run out without faulting or hanging the GPU.
 * szgb_debug_set_wait_limit sets the limit of every device-side wait of later
 * calls on this context (`ns` nanoseconds; 0 restores the default of 4 s).
 * szgb_debug_skip_item makes the wavefront CTA that takes work item `item`
 * (0-based, in every field of a call) return without running it or
 * publishing its state (-1 turns the hook off).  Its consumers then poll
 * halo words that are never written until the limit, set the device error
 * flag, publish an aborted state (which stops their own consumers) and
 * return; the call returns SZGB_ETIMEOUT and the context stays usable.
 * While an item is skipped, calls launch directly (no CUDA graphs).
 * SZGB_EINVAL for a null context or item < -1. */
int szgb_debug_set_wait_limit(szgb_ctx *ctx, uint64_t ns);
int szgb_debug_skip_item(szgb_ctx *ctx, int item);

/* ---- reconstruction quality (Sec. II, Metrics 1-3) ----------------------
 * One pass over a field x and its reconstruction y (both n float32 values in
 * device memory, any alignment), on the context's stream, in float64:
 *   max_abs_err = max |x_i - y_i|              (Metric 1, absolute error)
 *   max_rel_err = max_abs_err / R_X,  R_X = x_max - x_min (value range of x)
 *   rmse = sqrt(sum (x_i - y_i)^2 / n), nrmse = rmse / R_X,
 *   psnr = 20 log10(R_X / rmse)                 (Metric 2)
 *   pearson = cov(x, y) / (sigma_x sigma_y)     (Metric 3; population moments)
 * Undefined cases: R_X = 0 gives NaN for nrmse / max_rel_err and for psnr
 * unless rmse = 0 (psnr = +inf when the reconstruction is exact); a zero
 * standard deviation gives NaN for pearson.  Inputs are expected finite.
 * The result is deterministic (a fixed reduction order).  Blocks until done.
 * Returns SZGB_OK, SZGB_EINVAL (null pointer, n = 0), SZGB_ENOMEM, SZGB_ECUDA. */
typedef struct szgb_quality {
    double max_abs_err, max_rel_err;
    double rmse, nrmse, psnr;
    double pearson;
    double x_min, x_max;
    uint64_t n;
} szgb_quality;
int szgb_quality_dev(szgb_ctx *ctx, const float *x_dev, const float *y_dev, size_t n,
                     szgb_quality *out);

/* ---- prediction hitting rate (Sec. III, Table 2) -------------------------
 * Counts the points i of the field x whose n-layer prediction f_i (Sec. III,
 * the unified predictor), formed from the values v at i's preceding
 * neighbours, lies within eb of x_i: |x_i - f_i| <= eb (inclusive).  f_i is
 * the float32 value the compressor forms (terms in descending lexicographic
 * order, products and sums rounded one at a time, values outside the field
 * 0); the difference and the comparison are float64.  v = x gives the count
 * behind R_PH^orig; v = the values the compressor recorded (the recorded_dev
 * output of szgb_compress_trace or szgb_compress_4d, equal to the
 * decompressed field) gives the
 * count behind R_PH^decomp; divide by the number of points for the rate.
 *  - x_dev, v_dev: device, float32, raster order (last axis fastest), shape
 *    shape[0..ndim-1] (slowest first), ndim 1..4, extents 1..2^32-1 and fewer
 *    than 2^40 points; layers 1..4 in every dimension; eb >= 0.
 *  - runs on the context's stream and blocks until done; *n_hit is set on
 *    success.  Returns SZGB_OK, SZGB_EINVAL (null pointer, bad shape, layers
 *    or eb), SZGB_ENOMEM, SZGB_EBUDGET, SZGB_ECUDA. */
int szgb_hit_count_dev(szgb_ctx *ctx, const float *x_dev, const float *v_dev, int ndim,
                       const uint64_t *shape, int layers, double eb, uint64_t *n_hit);

/* ---- serving loop ------------------------------------------------------
 * Requests are taken as they arrive and run by worker threads, each with its
 * own context and stream, so that batches overlap on the device.  A worker
 * admits the oldest pending requests whose device footprint (input + output
 * + a scratch estimate) fits in the memory budget beside the requests in
 * flight, at most max_batch at a time, and runs them as one batched
 * compression and one batched decompression (continuous batching: requests
 * arriving meanwhile join the next batch).  Buffers and codebook tables stay
 * resident between batches.  The result of every request equals the result
 * of the single-field call. */
#define SZGB_OP_COMPRESS 0
#define SZGB_OP_DECOMPRESS 1

typedef struct szgb_server szgb_server;

typedef struct {
    int op;              /* SZGB_OP_COMPRESS or SZGB_OP_DECOMPRESS */
    const void *in;      /* host: the FP32 array (compress) or the stream (decompress) */
    size_t in_bytes;     /* bytes of `in` (compress: 4 x points of params.shape) */
    szgb_params params;  /* compress: shape, bound, n, m (ignored for decompress) */
    void *out;           /* host: room for the stream (compress) or the FP32 array */
    size_t out_cap;      /* bytes of `out` */
} szgb_request;

/* Creates a server on CUDA device `device` with `workers` worker threads
 * (1..16), admitting at most `device_mem_budget` bytes of request footprint
 * at a time and at most `max_batch` requests per batch. */
int szgb_server_create(szgb_server **out, int device, size_t device_mem_budget,
                       int workers, int max_batch);
/* Queues a request; the caller keeps `in` and `out` valid and untouched
 * until the request is done.  *ticket identifies it.  SZGB_EBUDGET when the
 * request alone exceeds the budget.  Requests the batched wavefront does not
 * carry (3D n = 3, 4; 4D; the lattice variant) run alone, on their own
 * kernels. */
int szgb_submit(szgb_server *srv, const szgb_request *req, uint64_t *ticket);
/* Non-blocking: *done = 1 once the request finished; then *status (its
 * SZGB_E* code) and *out_len (stream bytes, or 4 x points) are set and the
 * ticket is released. */
int szgb_poll(szgb_server *srv, uint64_t ticket, int *done, int *status, size_t *out_len);
/* Blocks until the request finished; then as szgb_poll with *done = 1.
 * When another thread takes the result of the same ticket first (by poll
 * or wait), returns SZGB_EINVAL. */
int szgb_wait(szgb_server *srv, uint64_t ticket, int *status, size_t *out_len);
/* Batches run, requests completed, and the peak admitted footprint. */
int szgb_server_stats(szgb_server *srv, uint64_t *batches, uint64_t *completed,
                      size_t *peak_reserved);
/* Finishes the pending requests, stops the workers and frees the server. */
void szgb_server_destroy(szgb_server *srv);

/* Algorithm 1, last step (Sec. IV-B): after a compression, the share of
 * points that fell into one of the 2^m - 1 quantization intervals,
 * R = (n_points - n_unpred) / n_points, is compared with the threshold
 * theta; below it a larger m is suggested.  Returns m + 1 (at most 16) when
 * R < theta, else m, and stores R in *hit_rate_out when it is not NULL.
 * Host only, no device work.  SZGB_EINVAL for a null st, n_points = 0,
 * n_unpred > n_points, m outside 2..16 or a NaN theta. */
int szgb_suggest_m(const szgb_stats *st, double theta, double *hit_rate_out);

/* Reads the header of a stream held in host memory: parameters (with the
 * m actually used, chunk_points = the stream's chunk length or
 * SZGB_CHUNK_ROWS, ndim 1..4 with the field's own extents) and the number
 * of unpredictable points.  SZGB_ECORRUPT for an inconsistent header. */
int szgb_stream_info(const uint8_t *in_host, size_t in_len, szgb_params *out,
                     uint64_t *n_unpred);

/* Per-phase device time of the calls made since the last reset, measured
 * with CUDA events on the context's stream when profiling is on.  Phase
 * names: szgb_phase_name(i) for i < szgb_num_phases().  ms[i] is the summed
 * time, calls[i] the number of timed launches. */
int szgb_set_profiling(szgb_ctx *ctx, int on);
int szgb_num_phases(void);
const char *szgb_phase_name(int i);
int szgb_phase_times(szgb_ctx *ctx, double *ms, uint64_t *calls, int n, int reset);

const char *szgb_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif
