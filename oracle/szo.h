/*
 * szo.h -- sequential CPU oracle of the error-bounded lossy compressor of
 * arXiv:1706.03791 (multilayer prediction, Sec. III; error-controlled
 * quantization and Huffman coding, Sec. IV; Algorithm 1).
 *
 * TEST INFRASTRUCTURE ONLY.  This library defines what the GPU path must
 * produce; it is linked only by the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark.  It shares no code, header or constant
 * table with the GPU library.
 *
 * Array convention: shape[] is slowest -> fastest (C order).  The paper's
 * method takes 1D..4D fields, handled as four extents with leading 1s (its
 * predictor is defined for any dimension); the lattice variant takes 1D..3D.
 * Error codes: 0 ok, -1 invalid argument, -2 non-finite input, -3 output
 * buffer too small (needed size in *out_len), -4 corrupt stream, -5 no memory.
 */
#ifndef SZO_H
#define SZO_H
#include <stddef.h>
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

/* Number of prediction terms, (n+1)^d - 1 (Algorithm 1, coefficient step),
 * d = 1..4. */
int szo_num_terms(int ndim, int layers);
/* Offsets k (3 ints each, leading zeros for d < 3; d <= 3) and integer
 * coefficients -prod_j (-1)^k_j C(n,k_j) of the n-layer predictor
 * (Eq. predmodel), in the summation order the oracle uses (descending
 * lexicographic k). */
int szo_terms(int ndim, int layers, int32_t *k_out, int64_t *coef_out);
/* The same with 4 ints per offset (leading zeros for d < 4), d = 1..4. */
int szo_terms4(int ndim, int layers, int32_t *k_out, int64_t *coef_out);
/* Prediction of every point from the values in V (Eq. predmodel), with
 * neighbours outside the domain taken as 0. */
int szo_predict_field(const float *V, int ndim, const uint64_t *shape,
                      int layers, float *pred_out);
/* Effective bound: eb (double) and eb_f (largest float <= eb). */
double szo_effective_eb(int mode, double eb_abs, double eb_rel, float xmin,
                        float xmax, float *eb_f_out);
/* Error-controlled quantization of one value (Sec. IV-A).  Returns the code
 * (0 = unpredictable) and the value recorded for later predictions. */
int szo_quantize(float x, float pred, float eb_f, int m, float *recorded);
/* Truncated binary representation of an unpredictable value: returns the
 * number of kept mantissa bits t and the truncated value. */
int szo_truncate(float x, float eb_f, float *truncated);
/* Huffman code lengths over nsym symbols (freq 0 = unused -> length 0). */
int szo_huffman_lengths(const uint64_t *freq, int nsym, uint8_t *len_out);
/* Canonical codes from code lengths. */
int szo_canonical_codes(const uint8_t *len, int nsym, uint64_t *code_out);
/* Adaptive choice of m from a sampled prediction hit rate (Sec. IV-B). */
int szo_choose_m(const float *x, int ndim, const uint64_t *shape, int layers,
                 float eb_f, double theta);
/* Worst-case stream size. */
size_t szo_stream_bound(int ndim, const uint64_t *shape);
/* Compress (1D..4D).  order 0 = raster order, 1 = hyperplane order (by
 * the sum of the coordinates).  A 4D stream keeps its slowest extent at
 * header byte 120.  Optional
 * outputs: recorded values (the decompressed values the compressor predicts
 * from) and the quantization codes, both in raster order. */
int szo_compress(const float *x, int ndim, const uint64_t *shape, int mode,
                 double eb_abs, double eb_rel, int layers, int m, double theta,
                 int order, uint8_t *out, size_t out_cap, size_t *out_len,
                 float *recorded_out, uint16_t *codes_out);
/* As szo_compress, with the Huffman payload cut into chunks of chunk_points
 * points along each row (a power of two >= 32; 0, or a value >= the row
 * length: one chunk per row).  Chunk s of row r holds the points
 * [s C, min(N, (s + 1) C)) of that row; chunks follow row by row, each in its
 * own byte-padded bit string with its byte length in the chunk table, and C
 * is stored at header byte 116 (0 for whole rows).  SZO_EINVAL for any other
 * chunk_points. */
int szo_compress_chunked(const float *x, int ndim, const uint64_t *shape, int mode,
                         double eb_abs, double eb_rel, int layers, int m, double theta,
                         int order, uint32_t chunk_points, uint8_t *out, size_t out_cap, size_t *out_len,
                         float *recorded_out, uint16_t *codes_out);
/* The lattice variant (not the paper's method; a separately labelled fully
 * parallel form, header byte 113 = 1): values snapped to the 2 eb_f lattice,
 * integer n-layer prediction from lattice values, residuals coded like the
 * quantization codes, outliers stored exactly (see szo.c).  eb must be > 0. */
int64_t szo_lattice_point(float x, float eb_f, int *ok);
float szo_lattice_value(int64_t p, float eb_f);
int szo_choose_m_lattice(const float *x, int ndim, const uint64_t *shape, int layers, float eb_f,
                         double theta);
int szo_compress_lattice(const float *x, int ndim, const uint64_t *shape, int mode, double eb_abs,
                         double eb_rel, int layers, int m, double theta, uint8_t *out, size_t out_cap,
                         size_t *out_len, float *recorded_out, uint16_t *codes_out);
/* Decompress (either variant); out_cap_elems must be >= number of points. */
int szo_decompress(const uint8_t *in, size_t in_len, float *out,
                   size_t out_cap_elems);

#ifdef __cplusplus
}
#endif
#endif
