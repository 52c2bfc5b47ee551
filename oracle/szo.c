/*
 * szo.c -- sequential CPU oracle of the error-bounded lossy compressor of
 * arXiv:1706.03791.
 *
 * TEST INFRASTRUCTURE ONLY: linked by the tests, the smoke check and the CPU
 * baseline of the benchmark; never by the product path.  It shares no code
 * with the GPU library.  Build with -O2 -ffp-contract=off (no FMA
 * contraction, no fast-math): every float operation below is one IEEE
 * binary32 operation rounded to nearest-even, in the order written.
 *
 * The method, in the paper's order (Algorithm 1):
 *   coefficients of the n-layer predictor, computed once (Eq. predmodel);
 *   for every point in raster order: predict from the preceding
 *   *decompressed* values, quantize the difference into 2^m - 1 intervals of
 *   width 2*eb (Sec. IV-A), fall back to a truncated binary representation
 *   when no interval holds the value, and record the decompressed value for
 *   later predictions;
 *   Huffman-code the quantization codes (Sec. IV-A, variable-length coding).
 *
 * Readings where the paper is silent (each is listed in the design notes):
 *   R1 neighbours outside the domain are 0;
 *   R2 prediction sum order: k in descending lexicographic order, the first
 *      product initialises the sum, each product and sum rounded;
 *   R3 eb_f = largest float <= eb, eb computed in double from the range;
 *   R4 q = rint((x - pred) * (1 / (2 eb_f))) (half-even); accepted when
 *      |q| <= 2^(m-1)-1 and |x - d'| < eb_f (or x == d'), code = q + 2^(m-1);
 *   R5 unpredictable values keep sign, exponent and the top t mantissa bits,
 *      t = clamp(max(e,1) - e_eb, 0, 23) (23 when eb_f is 0 or subnormal);
 *   R6 Huffman: two-queue merge over leaves sorted by (freq, symbol), leaf
 *      queue first on ties, one used symbol -> length 1, canonical codes;
 *   R7 adaptive m: sample points whose coordinates are all multiples of 8,
 *      predict from original values, smallest m in [2,16] whose hit count
 *      reaches ceil(theta * samples), else 16;
 *   R8 stream layout: little-endian header, codebook, per-row byte lengths,
 *      payload rows of MSB-first bits with inline unpredictable records.
 *
 * The lattice variant (szo_compress_lattice) is NOT the paper's method but a
 * separately labelled, fully parallel form of it: every value is snapped to
 * the lattice of spacing 2 eb_f first, p = rint(x * inv) in binary32 with
 * inv = 1 / (2 eb_f) rounded once, |p| < 2^30; the
 * integer field p is predicted by the same n-layer coefficients in exact
 * integer arithmetic from the *lattice* values of the neighbours (zero
 * outside the domain), and the residual r = p - pred takes the place of the
 * quantization code (code r + 2^(m-1) when |r| <= 2^(m-1)-1).  A point is an
 * outlier (code 0) when |r| is larger or its lattice value (float)p * 2 eb_f
 * (binary32) misses the bound (|x - v| < eb_f or x == v, as the quantizer's
 * check); its record is a flag bit (1: the lattice value is within
 * the bound), r as 64-bit two's complement and, when the flag is 0, the 32
 * bits of x.  Since the prediction never uses reconstructed values, every
 * residual is independent of the others, and the inverse of the predictor
 * (n prefix sums per axis) recovers p.
 */
#include "szo.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define SZO_OK 0
#define SZO_EINVAL (-1)
#define SZO_ENONFINITE (-2)
#define SZO_ETRUNC (-3)
#define SZO_ECORRUPT (-4)
#define SZO_ENOMEM (-5)

#define HDR_BYTES 128

/* ------------------------------------------------------------------ */
/* small helpers                                                        */

static uint32_t f2u(float f) { uint32_t u; memcpy(&u, &f, 4); return u; }
static float u2f(uint32_t u) { float f; memcpy(&f, &u, 4); return f; }

static int64_t binom(int n, int k) {
    if (k < 0 || k > n) return 0;
    int64_t r = 1;
    for (int i = 1; i <= k; i++) r = r * (n - k + i) / i;
    return r;
}

/* 1D..3D shape as three extents, slowest first, leading 1s (the lattice
 * variant) */
static int norm_shape(int ndim, const uint64_t *shape, uint64_t d[3]) {
    if (ndim < 1 || ndim > 3 || !shape) return SZO_EINVAL;
    d[0] = d[1] = 1;
    for (int a = 0; a < ndim; a++) d[3 - ndim + a] = shape[a];
    for (int a = 0; a < 3; a++) if (d[a] == 0) return SZO_EINVAL;
    return SZO_OK;
}

/* 1D..4D shape as four extents, slowest first, leading 1s (the paper's
 * method: its predictor is defined for any number of dimensions) */
static int norm_shape4(int ndim, const uint64_t *shape, uint64_t d[4]) {
    if (ndim < 1 || ndim > 4 || !shape) return SZO_EINVAL;
    d[0] = d[1] = d[2] = 1;
    for (int a = 0; a < ndim; a++) d[4 - ndim + a] = shape[a];
    for (int a = 0; a < 4; a++) if (d[a] == 0) return SZO_EINVAL;
    return SZO_OK;
}

/* ------------------------------------------------------------------ */
/* n-layer predictor (Sec. III, Eq. predmodel)                          */

int szo_num_terms(int ndim, int layers) {
    if (ndim < 1 || ndim > 4 || layers < 1) return SZO_EINVAL;
    int t = 1;
    for (int a = 0; a < ndim; a++) t *= (layers + 1);
    return t - 1;
}

/* Enumerates k in [0,n]^d \ {0} in descending lexicographic order (slowest
 * axis most significant) with coefficient -prod_j (-1)^k_j C(n, k_j); k is
 * written as 4 ints per term, leading zeros for d < 4. */
static int enum_terms(int ndim, int layers, int32_t *k4, int64_t *coef_out) {
    int T = szo_num_terms(ndim, layers);
    if (T < 0) return T;
    int n = layers, idx = 0;
    int total = T + 1;
    for (int code = total - 1; code >= 1; code--) {
        int k[4] = {0, 0, 0, 0}, c = code;
        for (int a = ndim - 1; a >= 0; a--) { k[4 - ndim + a] = c % (n + 1); c /= (n + 1); }
        int64_t prod = 1;
        for (int a = 0; a < 4; a++) {
            int64_t s = (k[a] & 1) ? -1 : 1;
            prod *= s * binom(n, k[a]);
        }
        if (k4) for (int a = 0; a < 4; a++) k4[4 * idx + a] = k[a];
        if (coef_out) coef_out[idx] = -prod;
        idx++;
    }
    return T;
}

int szo_terms(int ndim, int layers, int32_t *k_out, int64_t *coef_out) {
    if (ndim > 3) return SZO_EINVAL;
    int T = szo_num_terms(ndim, layers);
    if (T < 0) return T;
    int32_t *k4 = (int32_t *)malloc(sizeof(int32_t) * 4 * (size_t)T);
    if (!k4) return SZO_ENOMEM;
    enum_terms(ndim, layers, k4, coef_out);
    if (k_out)
        for (int i = 0; i < T; i++)
            for (int a = 0; a < 3; a++) k_out[3 * i + a] = k4[4 * i + 1 + a];
    free(k4);
    return T;
}

int szo_terms4(int ndim, int layers, int32_t *k_out, int64_t *coef_out) {
    return enum_terms(ndim, layers, k_out, coef_out);
}

typedef struct { int32_t k[4]; float c; } term_t;

static term_t *make_terms(int ndim, int layers, int *T_out) {
    int T = szo_num_terms(ndim, layers);
    if (T <= 0) return NULL;
    int32_t *k = (int32_t *)malloc(sizeof(int32_t) * 4 * T);
    int64_t *c = (int64_t *)malloc(sizeof(int64_t) * T);
    term_t *t = (term_t *)malloc(sizeof(term_t) * T);
    if (!k || !c || !t) { free(k); free(c); free(t); return NULL; }
    enum_terms(ndim, layers, k, c);
    for (int i = 0; i < T; i++) {
        for (int a = 0; a < 4; a++) t[i].k[a] = k[4 * i + a];
        t[i].c = (float)c[i];
    }
    free(k); free(c);
    *T_out = T;
    return t;
}

/* raster index of the point with coordinates x[0..3] */
static uint64_t lin4(const uint64_t d[4], const int64_t x[4]) {
    return (((uint64_t)x[0] * d[1] + (uint64_t)x[1]) * d[2] + (uint64_t)x[2]) * d[3] + (uint64_t)x[3];
}

/* f(x) = sum_k c_k V(x - k); V outside the domain = 0 (R1); summed in the
 * term order, first product initialising the sum (R2). */
static float predict_at(const float *V, const uint64_t d[4], const int64_t x[4], const term_t *t, int T) {
    float pred = 0.0f;
    for (int s = 0; s < T; s++) {
        int64_t y[4];
        int inside = 1;
        for (int a = 0; a < 4; a++) {
            y[a] = x[a] - t[s].k[a];
            if (y[a] < 0) inside = 0;
        }
        float v = inside ? V[lin4(d, y)] : 0.0f;
        float prod = t[s].c * v;
        pred = (s == 0) ? prod : pred + prod;
    }
    return pred;
}

int szo_predict_field(const float *V, int ndim, const uint64_t *shape, int layers,
                      float *pred_out) {
    uint64_t d[4];
    if (norm_shape4(ndim, shape, d) || !V || !pred_out) return SZO_EINVAL;
    int T;
    term_t *t = make_terms(ndim, layers, &T);
    if (!t) return SZO_EINVAL;
    int64_t x[4];
    for (x[0] = 0; x[0] < (int64_t)d[0]; x[0]++)
        for (x[1] = 0; x[1] < (int64_t)d[1]; x[1]++)
            for (x[2] = 0; x[2] < (int64_t)d[2]; x[2]++)
                for (x[3] = 0; x[3] < (int64_t)d[3]; x[3]++)
                    pred_out[lin4(d, x)] = predict_at(V, d, x, t, T);
    free(t);
    return SZO_OK;
}

/* ------------------------------------------------------------------ */
/* error bound (Sec. II metric 1) and quantization (Sec. IV-A)           */

double szo_effective_eb(int mode, double eb_abs, double eb_rel, float xmin,
                        float xmax, float *eb_f_out) {
    double range = (double)xmax - (double)xmin; /* exact in double */
    double eb;
    if (mode == 0) eb = eb_abs;
    else if (mode == 1) eb = eb_rel * range;
    else eb = fmin(eb_abs, eb_rel * range);
    float f = (float)eb;
    if ((double)f > eb) f = nextafterf(f, 0.0f); /* largest float <= eb (R3) */
    if (eb_f_out) *eb_f_out = f;
    return eb;
}

int szo_truncate(float x, float eb_f, float *truncated) {
    uint32_t u = f2u(x), ue = f2u(eb_f);
    int e = (int)((u >> 23) & 0xff);
    int eeb = (int)((ue >> 23) & 0xff);
    int t;
    if (eeb == 0) t = 23; /* eb_f is 0 or subnormal: keep every bit */
    else {
        int ee = e < 1 ? 1 : e;
        t = ee - eeb;
        if (t < 0) t = 0;
        if (t > 23) t = 23;
    }
    uint32_t keep = (t == 0) ? 0u : (((1u << t) - 1u) << (23 - t));
    uint32_t r = (u & 0xff800000u) | (u & keep);
    if (truncated) *truncated = u2f(r);
    return t;
}

/* Linear-scaling quantization: intervals of width 2 eb centred on
 * pred + q*2eb, q in [-(2^(m-1)-1), 2^(m-1)-1], coded q + 2^(m-1); code 0
 * marks an unpredictable value (R4, R5). */
int szo_quantize(float x, float pred, float eb_f, int m, float *recorded) {
    float twoeb = 2.0f * eb_f;
    float inv = (eb_f > 0.0f) ? 1.0f / twoeb : 0.0f;
    float radius = (float)((1 << (m - 1)) - 1);
    float diff = x - pred;
    float prodq = diff * inv;
    float q = rintf(prodq);
    if (fabsf(q) <= radius) {
        /* the interval's value is defined from the integer index, exactly as
         * the decompressor rebuilds it (so rint's -0.0 cannot matter) */
        int qi = (int)q;
        float step = (float)qi * twoeb;
        float dq = pred + step;
        float err = x - dq;
        if (fabsf(err) < eb_f || x == dq) {
            if (recorded) *recorded = dq;
            return qi + (1 << (m - 1));
        }
    }
    float tr;
    szo_truncate(x, eb_f, &tr);
    if (recorded) *recorded = tr;
    return 0;
}

/* ------------------------------------------------------------------ */
/* adaptive number of intervals (Sec. IV-B)                             */

int szo_choose_m(const float *x, int ndim, const uint64_t *shape, int layers,
                 float eb_f, double theta) {
    uint64_t d[4];
    if (norm_shape4(ndim, shape, d) || !x) return SZO_EINVAL;
    int T;
    term_t *t = make_terms(ndim, layers, &T);
    if (!t) return SZO_EINVAL;
    uint64_t need[17] = {0};
    uint64_t S = 0;
    float twoeb = 2.0f * eb_f;
    float inv = (eb_f > 0.0f) ? 1.0f / twoeb : 0.0f;
    int64_t c[4];
    for (c[0] = 0; c[0] < (int64_t)d[0]; c[0] += 8)
        for (c[1] = 0; c[1] < (int64_t)d[1]; c[1] += 8)
            for (c[2] = 0; c[2] < (int64_t)d[2]; c[2] += 8)
                for (c[3] = 0; c[3] < (int64_t)d[3]; c[3] += 8) {
                    S++;
                    float xv = x[lin4(d, c)];
                    float pred = predict_at(x, d, c, t, T); /* original values */
                    float diff = xv - pred;
                    float q = rintf(diff * inv);
                    if (!(fabsf(q) <= 32767.0f)) continue;
                    float dq = pred + (float)(int)q * twoeb;
                    if (!(fabsf(xv - dq) < eb_f || xv == dq)) continue;
                    float aq = fabsf(q);
                    int mm = 2;
                    while (aq > (float)((1 << (mm - 1)) - 1)) mm++;
                    need[mm]++;
                }
    free(t);
    double req = ceil(theta * (double)S);
    uint64_t cum = 0;
    for (int mm = 2; mm <= 16; mm++) {
        cum += need[mm];
        if ((double)cum >= req) return mm;
    }
    return 16;
}

/* ------------------------------------------------------------------ */
/* Huffman coding (Sec. IV-A: any number of symbols)                    */

typedef struct { uint64_t f; int32_t s; } leaf_t;

static int leaf_cmp(const void *a, const void *b) {
    const leaf_t *x = (const leaf_t *)a, *y = (const leaf_t *)b;
    if (x->f != y->f) return x->f < y->f ? -1 : 1;
    return x->s < y->s ? -1 : (x->s > y->s);
}

int szo_huffman_lengths(const uint64_t *freq, int nsym, uint8_t *len_out) {
    if (!freq || !len_out || nsym < 1) return SZO_EINVAL;
    memset(len_out, 0, (size_t)nsym);
    int n = 0;
    for (int s = 0; s < nsym; s++) if (freq[s]) n++;
    if (n == 0) return 0;
    leaf_t *lv = (leaf_t *)malloc(sizeof(leaf_t) * n);
    if (!lv) return SZO_ENOMEM;
    n = 0;
    for (int s = 0; s < nsym; s++) if (freq[s]) { lv[n].f = freq[s]; lv[n].s = s; n++; }
    if (n == 1) { len_out[lv[0].s] = 1; free(lv); return 1; }
    qsort(lv, (size_t)n, sizeof(leaf_t), leaf_cmp);
    int total = 2 * n - 1;
    uint64_t *w = (uint64_t *)malloc(sizeof(uint64_t) * total);
    int32_t *par = (int32_t *)malloc(sizeof(int32_t) * total);
    int32_t *dep = (int32_t *)malloc(sizeof(int32_t) * total);
    if (!w || !par || !dep) { free(lv); free(w); free(par); free(dep); return SZO_ENOMEM; }
    for (int i = 0; i < n; i++) w[i] = lv[i].f;
    /* two queues: leaves [q1, n) sorted; internal nodes [q2, next) in
     * creation order (their weights never decrease) */
    int q1 = 0, q2 = n, next = n;
    for (int step = 0; step < n - 1; step++) {
        int pick[2];
        for (int p = 0; p < 2; p++) {
            if (q1 < n && (q2 >= next || w[q1] <= w[q2])) pick[p] = q1++;
            else pick[p] = q2++;
        }
        w[next] = w[pick[0]] + w[pick[1]];
        par[pick[0]] = next;
        par[pick[1]] = next;
        next++;
    }
    dep[total - 1] = 0;
    for (int v = total - 2; v >= 0; v--) dep[v] = dep[par[v]] + 1;
    int maxlen = 0;
    for (int i = 0; i < n; i++) {
        len_out[lv[i].s] = (uint8_t)dep[i];
        if (dep[i] > maxlen) maxlen = dep[i];
    }
    free(lv); free(w); free(par); free(dep);
    return maxlen;
}

/* Canonical assignment: symbols ordered by (length, symbol); the first gets
 * code 0 and each next code is (previous + 1) shifted left by the length
 * increase. */
int szo_canonical_codes(const uint8_t *len, int nsym, uint64_t *code_out) {
    if (!len || !code_out || nsym < 1) return SZO_EINVAL;
    memset(code_out, 0, sizeof(uint64_t) * (size_t)nsym);
    uint64_t code = 0;
    int prev = 0, first = 1;
    for (int L = 1; L <= 64; L++)
        for (int s = 0; s < nsym; s++) {
            if (len[s] != L) continue;
            if (first) { code = 0; first = 0; }
            else code = (code + 1) << (L - prev);
            prev = L;
            code_out[s] = code;
        }
    return SZO_OK;
}

/* ------------------------------------------------------------------ */
/* bit I/O (MSB-first)                                                   */

typedef struct { uint8_t *p; uint64_t bit; } bw_t;

static void put_bits(bw_t *w, uint64_t v, int n) {
    for (int b = n - 1; b >= 0; b--) {
        if ((v >> b) & 1u) w->p[w->bit >> 3] |= (uint8_t)(0x80u >> (w->bit & 7));
        w->bit++;
    }
}

typedef struct { const uint8_t *p; uint64_t bit, end; } br_t;

static int get_bit(br_t *r) {
    if (r->bit >= r->end) return -1;
    int v = (r->p[r->bit >> 3] >> (7 - (r->bit & 7))) & 1;
    r->bit++;
    return v;
}

static int64_t get_bits(br_t *r, int n) {
    uint64_t v = 0;
    for (int i = 0; i < n; i++) {
        int b = get_bit(r);
        if (b < 0) return -1;
        v = (v << 1) | (uint64_t)b;
    }
    return (int64_t)v;
}

static void wr16(uint8_t *p, uint16_t v) { p[0] = (uint8_t)v; p[1] = (uint8_t)(v >> 8); }
static void wr32(uint8_t *p, uint32_t v) { for (int i = 0; i < 4; i++) p[i] = (uint8_t)(v >> (8 * i)); }
static void wr64(uint8_t *p, uint64_t v) { for (int i = 0; i < 8; i++) p[i] = (uint8_t)(v >> (8 * i)); }
static uint16_t rd16(const uint8_t *p) { return (uint16_t)(p[0] | (p[1] << 8)); }
static uint32_t rd32(const uint8_t *p) { uint32_t v = 0; for (int i = 3; i >= 0; i--) v = (v << 8) | p[i]; return v; }
static uint64_t rd64(const uint8_t *p) { uint64_t v = 0; for (int i = 7; i >= 0; i--) v = (v << 8) | p[i]; return v; }
static void wrf64(uint8_t *p, double d) { uint64_t u; memcpy(&u, &d, 8); wr64(p, u); }
static uint64_t pad4(uint64_t v) { return (v + 3) & ~(uint64_t)3; }

size_t szo_stream_bound(int ndim, const uint64_t *shape) {
    uint64_t d[4];
    if (norm_shape4(ndim, shape, d)) return 0;
    uint64_t N = d[0] * d[1] * d[2] * d[3], rows = d[0] * d[1] * d[2];
    uint64_t nch = rows * ((d[3] + 31) / 32); /* the most chunks: 32 points each */
    return (size_t)(HDR_BYTES + pad4(3 * 65536) + pad4(4 * nch) + nch + (N * 78 + 7) / 8 + 16);
}

/* ------------------------------------------------------------------ */
/* compression (Algorithm 1)                                           */

int szo_compress(const float *x, int ndim, const uint64_t *shape, int mode,
                 double eb_abs, double eb_rel, int layers, int m, double theta,
                 int order, uint8_t *out, size_t out_cap, size_t *out_len,
                 float *recorded_out, uint16_t *codes_out) {
    return szo_compress_chunked(x, ndim, shape, mode, eb_abs, eb_rel, layers, m, theta, order, 0, out, out_cap,
                                out_len, recorded_out, codes_out);
}

/* chunk length along a row: chunk_points when it splits the row, else the
 * whole row (0: whole rows) */
static uint64_t chunk_len(uint32_t chunk_points, uint64_t row_len) {
    return (chunk_points == 0 || chunk_points >= row_len) ? row_len : chunk_points;
}

static int chunk_points_valid(uint32_t c) { return c == 0 || (c >= 32 && (c & (c - 1)) == 0); }

int szo_compress_chunked(const float *x, int ndim, const uint64_t *shape, int mode,
                         double eb_abs, double eb_rel, int layers, int m, double theta,
                         int order, uint32_t chunk_points, uint8_t *out, size_t out_cap, size_t *out_len,
                         float *recorded_out, uint16_t *codes_out) {
    uint64_t d[4];
    if (!chunk_points_valid(chunk_points)) return SZO_EINVAL;
    if (norm_shape4(ndim, shape, d) || !x || !out_len) return SZO_EINVAL;
    if (mode < 0 || mode > 2 || layers < 1 || layers > 4) return SZO_EINVAL;
    if (m != 0 && (m < 2 || m > 16)) return SZO_EINVAL;
    if (mode != 1 && !(eb_abs >= 0.0)) return SZO_EINVAL;
    if (mode != 0 && !(eb_rel >= 0.0)) return SZO_EINVAL;
    uint64_t N = 1;
    for (int a = 0; a < 4; a++) {
        if (d[a] >= ((uint64_t)1 << 32)) return SZO_EINVAL;
        N *= d[a]; /* each factor < 2^32 and the product so far < 2^32 */
        if (N >= ((uint64_t)1 << 32)) return SZO_EINVAL;
    }

    /* range and finite check */
    float xmin = x[0], xmax = x[0];
    for (uint64_t p = 0; p < N; p++) {
        if (!isfinite(x[p])) return SZO_ENONFINITE;
        if (x[p] < xmin) xmin = x[p];
        if (x[p] > xmax) xmax = x[p];
    }
    /* the stored range is the value range: a signed zero is stored as +0 */
    xmin = xmin + 0.0f;
    xmax = xmax + 0.0f;
    float eb_f;
    szo_effective_eb(mode, eb_abs, eb_rel, xmin, xmax, &eb_f);
    int adaptive = (m == 0);
    if (adaptive) m = szo_choose_m(x, ndim, shape, layers, eb_f, theta);

    int T;
    term_t *t = make_terms(ndim, layers, &T);
    float *V = (float *)malloc(sizeof(float) * N);
    uint16_t *code = (uint16_t *)malloc(sizeof(uint16_t) * N);
    if (!t || !V || !code) { free(t); free(V); free(code); return SZO_ENOMEM; }

    /* the hot loop: predict, quantize, fall back, record */
    uint64_t K = 0;
    int64_t c[4];
    if (order == 0) {
        for (c[0] = 0; c[0] < (int64_t)d[0]; c[0]++)
            for (c[1] = 0; c[1] < (int64_t)d[1]; c[1]++)
                for (c[2] = 0; c[2] < (int64_t)d[2]; c[2]++)
                    for (c[3] = 0; c[3] < (int64_t)d[3]; c[3]++) {
                        uint64_t p = lin4(d, c);
                        float pred = predict_at(V, d, c, t, T);
                        code[p] = (uint16_t)szo_quantize(x[p], pred, eb_f, m, &V[p]);
                    }
    } else {
        /* hyperplane order: every point whose coordinates sum to h before
         * any point of h+1 */
        int64_t H = (int64_t)((d[0] - 1) + (d[1] - 1) + (d[2] - 1) + (d[3] - 1));
        for (int64_t h = 0; h <= H; h++)
            for (c[0] = 0; c[0] < (int64_t)d[0] && c[0] <= h; c[0]++)
                for (c[1] = 0; c[1] < (int64_t)d[1] && c[0] + c[1] <= h; c[1]++)
                    for (c[2] = 0; c[2] < (int64_t)d[2] && c[0] + c[1] + c[2] <= h; c[2]++) {
                        c[3] = h - c[0] - c[1] - c[2];
                        if (c[3] >= (int64_t)d[3]) continue;
                        uint64_t p = lin4(d, c);
                        float pred = predict_at(V, d, c, t, T);
                        code[p] = (uint16_t)szo_quantize(x[p], pred, eb_f, m, &V[p]);
                    }
    }
    for (uint64_t p = 0; p < N; p++) K += (code[p] == 0);

    /* Huffman coding of the codes */
    int nsymtot = 1 << m;
    uint64_t *freq = (uint64_t *)calloc((size_t)nsymtot, sizeof(uint64_t));
    uint8_t *len = (uint8_t *)malloc((size_t)nsymtot);
    uint64_t *cw = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)nsymtot);
    if (!freq || !len || !cw) { free(t); free(V); free(code); free(freq); free(len); free(cw); return SZO_ENOMEM; }
    for (uint64_t p = 0; p < N; p++) freq[code[p]]++;
    int maxlen = szo_huffman_lengths(freq, nsymtot, len);
    szo_canonical_codes(len, nsymtot, cw);
    uint32_t nsym = 0;
    for (int s = 0; s < nsymtot; s++) nsym += (len[s] != 0);

    /* chunks: each row is cut into pieces of Ce points (the last one
     * shorter), taken row by row; per-chunk bit counts are the code bits plus
     * 9 + t record bits after every code 0, rounded up to whole bytes */
    uint64_t rows = d[0] * d[1] * d[2], Nr = d[3];
    uint64_t Ce = chunk_len(chunk_points, Nr), nseg = (Nr + Ce - 1) / Ce, nch = rows * nseg;
    uint64_t *rowbytes = (uint64_t *)malloc(sizeof(uint64_t) * nch);
    if (!rowbytes) { free(t); free(V); free(code); free(freq); free(len); free(cw); return SZO_ENOMEM; }
    uint64_t payload = 0, maxrow = 0;
    for (uint64_t ch = 0; ch < nch; ch++) {
        uint64_t r = ch / nseg, l0 = (ch % nseg) * Ce, l1 = l0 + Ce < Nr ? l0 + Ce : Nr;
        uint64_t bits = 0;
        for (uint64_t l = l0; l < l1; l++) {
            uint64_t p = r * Nr + l;
            bits += len[code[p]];
            if (code[p] == 0) bits += 9 + (uint64_t)szo_truncate(x[p], eb_f, NULL);
        }
        rowbytes[ch] = (bits + 7) / 8;
        payload += rowbytes[ch];
        if (rowbytes[ch] > maxrow) maxrow = rowbytes[ch];
    }
    int tw = maxrow <= 0xffff ? 2 : 4;
    uint64_t cb_bytes = pad4(3 * (uint64_t)nsym);
    uint64_t tab_bytes = pad4((uint64_t)tw * nch);
    uint64_t total = HDR_BYTES + cb_bytes + tab_bytes + payload;
    *out_len = (size_t)total;
    int rc = SZO_OK;
    if (!out || out_cap < total) { rc = SZO_ETRUNC; goto done; }
    memset(out, 0, (size_t)total);

    /* header */
    out[0] = 'S'; out[1] = 'Z'; out[2] = 'G'; out[3] = 'B';
    wr16(out + 4, 1);
    wr16(out + 6, HDR_BYTES);
    out[8] = (uint8_t)ndim; out[9] = (uint8_t)layers; out[10] = (uint8_t)m; out[11] = (uint8_t)mode;
    out[12] = (uint8_t)maxlen; out[13] = (uint8_t)tw;
    /* the three fastest extents; a 4D field's slowest extent at byte 120 */
    wr64(out + 16, d[1]); wr64(out + 24, d[2]); wr64(out + 32, d[3]);
    if (ndim == 4) wr64(out + 120, d[0]);
    wrf64(out + 40, eb_abs); wrf64(out + 48, eb_rel);
    wr32(out + 56, f2u(eb_f)); wr32(out + 60, f2u(xmin)); wr32(out + 64, f2u(xmax));
    wr32(out + 68, nsym); wr64(out + 72, nch); wr64(out + 80, K);
    wr64(out + 88, payload); wr64(out + 96, total);
    wrf64(out + 104, theta); out[112] = (uint8_t)adaptive;
    wr32(out + 116, Ce < Nr ? (uint32_t)Ce : 0u); /* chunk length; 0: whole rows */

    /* codebook: (symbol, length) for the used symbols, ascending symbol */
    {
        uint8_t *cb = out + HDR_BYTES;
        uint32_t e = 0;
        for (int s = 0; s < nsymtot; s++)
            if (len[s]) { wr16(cb + 3 * e, (uint16_t)s); cb[3 * e + 2] = len[s]; e++; }
    }
    /* chunk table */
    {
        uint8_t *tb = out + HDR_BYTES + cb_bytes;
        for (uint64_t ch = 0; ch < nch; ch++) {
            if (tw == 2) wr16(tb + 2 * ch, (uint16_t)rowbytes[ch]);
            else wr32(tb + 4 * ch, (uint32_t)rowbytes[ch]);
        }
    }
    /* payload: every chunk starts on a byte */
    {
        uint8_t *pl = out + HDR_BYTES + cb_bytes + tab_bytes;
        uint64_t off = 0;
        for (uint64_t ch = 0; ch < nch; ch++) {
            uint64_t r = ch / nseg, l0 = (ch % nseg) * Ce, l1 = l0 + Ce < Nr ? l0 + Ce : Nr;
            bw_t w = {pl + off, 0};
            for (uint64_t l = l0; l < l1; l++) {
                uint64_t p = r * Nr + l;
                put_bits(&w, cw[code[p]], len[code[p]]);
                if (code[p] == 0) {
                    uint32_t u = f2u(x[p]);
                    int tt = szo_truncate(x[p], eb_f, NULL);
                    put_bits(&w, u >> 31, 1);
                    put_bits(&w, (u >> 23) & 0xff, 8);
                    if (tt) put_bits(&w, (u >> (23 - tt)) & ((1u << tt) - 1u), tt);
                }
            }
            off += rowbytes[ch];
        }
    }
    if (recorded_out) memcpy(recorded_out, V, sizeof(float) * N);
    if (codes_out) memcpy(codes_out, code, sizeof(uint16_t) * N);
done:
    free(rowbytes); free(t); free(V); free(code); free(freq); free(len); free(cw);
    return rc;
}

/* ------------------------------------------------------------------ */
/* the lattice variant                                                  */

typedef struct { int32_t k[3]; int64_t c; } iterm_t;

static iterm_t *make_iterms(int ndim, int layers, int *T_out) {
    int T = szo_num_terms(ndim, layers);
    if (T <= 0) return NULL;
    int32_t *k = (int32_t *)malloc(sizeof(int32_t) * 3 * T);
    int64_t *c = (int64_t *)malloc(sizeof(int64_t) * T);
    iterm_t *t = (iterm_t *)malloc(sizeof(iterm_t) * T);
    if (!k || !c || !t) { free(k); free(c); free(t); return NULL; }
    szo_terms(ndim, layers, k, c);
    for (int i = 0; i < T; i++) {
        t[i].k[0] = k[3 * i]; t[i].k[1] = k[3 * i + 1]; t[i].k[2] = k[3 * i + 2];
        t[i].c = c[i];
    }
    free(k); free(c);
    *T_out = T;
    return t;
}

/* integer prediction from lattice values, neighbours outside = 0.  Summed
 * modulo 2^64: exact for every stream the compressor writes (|p| < 2^30,
 * small coefficients), and free of signed overflow on corrupt input. */
static int64_t ipredict_at(const int64_t *P, const uint64_t d[3], int64_t i, int64_t j, int64_t l,
                           const iterm_t *t, int T) {
    uint64_t s = 0;
    for (int q = 0; q < T; q++) {
        int64_t ii = i - t[q].k[0], jj = j - t[q].k[1], ll = l - t[q].k[2];
        if (ii >= 0 && jj >= 0 && ll >= 0)
            s += (uint64_t)t[q].c * (uint64_t)P[((uint64_t)ii * d[1] + (uint64_t)jj) * d[2] + (uint64_t)ll];
    }
    return (int64_t)s;
}

/* the lattice integer of x and whether its lattice value is within the
 * bound; binary32 throughout, each operation rounded to nearest-even */
int64_t szo_lattice_point(float x, float eb_f, int *ok) {
    float twoeb = 2.0f * eb_f;
    float inv = 1.0f / twoeb;
    float y = rintf(x * inv);
    int64_t p = (int64_t)y;
    float v = (float)p * twoeb;
    if (ok) { float e = x - v; *ok = fabsf(e) < eb_f || x == v; }
    return p;
}

float szo_lattice_value(int64_t p, float eb_f) { return (float)p * (2.0f * eb_f); }

int szo_choose_m_lattice(const float *x, int ndim, const uint64_t *shape, int layers, float eb_f,
                         double theta) {
    uint64_t d[3];
    if (norm_shape(ndim, shape, d)) return 16;
    int T;
    iterm_t *t = make_iterms(ndim, layers, &T);
    if (!t) return 16;
    uint64_t S0 = (d[0] + 7) / 8, S1 = (d[1] + 7) / 8, S2 = (d[2] + 7) / 8, S = S0 * S1 * S2;
    uint64_t cnt[18] = {0};
    for (uint64_t a = 0; a < S0; a++)
        for (uint64_t b = 0; b < S1; b++)
            for (uint64_t c = 0; c < S2; c++) {
                int64_t i = (int64_t)(8 * a), j = (int64_t)(8 * b), l = (int64_t)(8 * c);
                int64_t pred = 0;
                for (int q = 0; q < T; q++) {
                    int64_t ii = i - t[q].k[0], jj = j - t[q].k[1], ll = l - t[q].k[2];
                    if (ii >= 0 && jj >= 0 && ll >= 0)
                        pred += t[q].c * szo_lattice_point(x[((uint64_t)ii * d[1] + (uint64_t)jj) * d[2] + (uint64_t)ll], eb_f, NULL);
                }
                int ok;
                int64_t p = szo_lattice_point(x[((uint64_t)i * d[1] + (uint64_t)j) * d[2] + (uint64_t)l], eb_f, &ok);
                int64_t r = p - pred, ar = r < 0 ? -r : r;
                if (!ok || ar > 32767) continue;
                int mm = 2;
                while (ar > ((int64_t)1 << (mm - 1)) - 1) mm++;
                cnt[mm]++;
            }
    free(t);
    double req = ceil(theta * (double)S);
    uint64_t cum = 0;
    for (int mm = 2; mm <= 16; mm++) {
        cum += cnt[mm];
        if ((double)cum >= req) return mm;
    }
    return 16;
}

int szo_compress_lattice(const float *x, int ndim, const uint64_t *shape, int mode, double eb_abs,
                         double eb_rel, int layers, int m, double theta, uint8_t *out, size_t out_cap,
                         size_t *out_len, float *recorded_out, uint16_t *codes_out) {
    uint64_t d[3];
    if (norm_shape(ndim, shape, d) || !x || !out_len) return SZO_EINVAL;
    if (mode < 0 || mode > 2 || layers < 1 || layers > 4) return SZO_EINVAL;
    if (m != 0 && (m < 2 || m > 16)) return SZO_EINVAL;
    if (mode != 1 && !(eb_abs >= 0.0)) return SZO_EINVAL;
    if (mode != 0 && !(eb_rel >= 0.0)) return SZO_EINVAL;
    uint64_t N = d[0] * d[1] * d[2];
    if (N >= ((uint64_t)1 << 32)) return SZO_EINVAL;
    float xmin = x[0], xmax = x[0];
    for (uint64_t p = 0; p < N; p++) {
        if (!isfinite(x[p])) return SZO_ENONFINITE;
        if (x[p] < xmin) xmin = x[p];
        if (x[p] > xmax) xmax = x[p];
    }
    xmin = xmin + 0.0f;
    xmax = xmax + 0.0f;
    float eb_f;
    szo_effective_eb(mode, eb_abs, eb_rel, xmin, xmax, &eb_f);
    /* the lattice needs a positive spacing and lattice integers below 2^30 */
    float amax = fmaxf(fabsf(xmin), fabsf(xmax));
    if (!(eb_f > 0.0f) || !(amax * (1.0f / (2.0f * eb_f)) < 1073741824.0f)) return SZO_EINVAL;
    int adaptive = (m == 0);
    if (adaptive) m = szo_choose_m_lattice(x, ndim, shape, layers, eb_f, theta);
    int T;
    iterm_t *t = make_iterms(ndim, layers, &T);
    int64_t *P = (int64_t *)malloc(sizeof(int64_t) * N);
    int64_t *R = (int64_t *)malloc(sizeof(int64_t) * N);
    uint8_t *okv = (uint8_t *)malloc(N);
    uint16_t *code = (uint16_t *)malloc(sizeof(uint16_t) * N);
    if (!t || !P || !R || !okv || !code) { free(t); free(P); free(R); free(okv); free(code); return SZO_ENOMEM; }
    for (uint64_t q = 0; q < N; q++) {
        int ok;
        P[q] = szo_lattice_point(x[q], eb_f, &ok);
        okv[q] = (uint8_t)ok;
    }
    const int64_t center = (int64_t)1 << (m - 1), radius = center - 1;
    uint64_t K = 0;
    for (uint64_t i = 0; i < d[0]; i++)
        for (uint64_t j = 0; j < d[1]; j++)
            for (uint64_t l = 0; l < d[2]; l++) {
                uint64_t q = (i * d[1] + j) * d[2] + l;
                R[q] = P[q] - ipredict_at(P, d, (int64_t)i, (int64_t)j, (int64_t)l, t, T);
                int64_t ar = R[q] < 0 ? -R[q] : R[q];
                code[q] = (okv[q] && ar <= radius) ? (uint16_t)(R[q] + center) : 0;
                K += code[q] == 0;
                if (recorded_out) recorded_out[q] = okv[q] ? szo_lattice_value(P[q], eb_f) : x[q];
            }
    /* Huffman coding of the codes, as in the exact path */
    int nsymtot = 1 << m;
    uint64_t *freq = (uint64_t *)calloc((size_t)nsymtot, sizeof(uint64_t));
    uint8_t *len = (uint8_t *)malloc((size_t)nsymtot);
    uint64_t *cw = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)nsymtot);
    uint64_t rows = d[0] * d[1], Nr = d[2];
    uint64_t *rowbytes = (uint64_t *)malloc(sizeof(uint64_t) * rows);
    int rc = SZO_OK;
    if (!freq || !len || !cw || !rowbytes) { rc = SZO_ENOMEM; goto done; }
    for (uint64_t q = 0; q < N; q++) freq[code[q]]++;
    int maxlen = szo_huffman_lengths(freq, nsymtot, len);
    szo_canonical_codes(len, nsymtot, cw);
    uint32_t nsym = 0;
    for (int s = 0; s < nsymtot; s++) nsym += (len[s] != 0);
    uint64_t payload = 0, maxrow = 0;
    for (uint64_t r = 0; r < rows; r++) {
        uint64_t bits = 0;
        for (uint64_t l = 0; l < Nr; l++) {
            uint64_t q = r * Nr + l;
            bits += len[code[q]];
            if (code[q] == 0) bits += 1 + 64 + (okv[q] ? 0 : 32);
        }
        rowbytes[r] = (bits + 7) / 8;
        payload += rowbytes[r];
        if (rowbytes[r] > maxrow) maxrow = rowbytes[r];
    }
    int tw = maxrow <= 0xffff ? 2 : 4;
    uint64_t cb_bytes = pad4(3 * (uint64_t)nsym), tab_bytes = pad4((uint64_t)tw * rows);
    uint64_t total = HDR_BYTES + cb_bytes + tab_bytes + payload;
    *out_len = (size_t)total;
    if (!out || out_cap < total) { rc = SZO_ETRUNC; goto done; }
    memset(out, 0, (size_t)total);
    out[0] = 'S'; out[1] = 'Z'; out[2] = 'G'; out[3] = 'B';
    wr16(out + 4, 1);
    wr16(out + 6, HDR_BYTES);
    out[8] = (uint8_t)ndim; out[9] = (uint8_t)layers; out[10] = (uint8_t)m; out[11] = (uint8_t)mode;
    out[12] = (uint8_t)maxlen; out[13] = (uint8_t)tw;
    wr64(out + 16, d[0]); wr64(out + 24, d[1]); wr64(out + 32, d[2]);
    wrf64(out + 40, eb_abs); wrf64(out + 48, eb_rel);
    wr32(out + 56, f2u(eb_f)); wr32(out + 60, f2u(xmin)); wr32(out + 64, f2u(xmax));
    wr32(out + 68, nsym); wr64(out + 72, rows); wr64(out + 80, K);
    wr64(out + 88, payload); wr64(out + 96, total);
    wrf64(out + 104, theta); out[112] = (uint8_t)adaptive;
    out[113] = 1; /* the lattice variant */
    {
        uint8_t *cb = out + HDR_BYTES;
        uint32_t e = 0;
        for (int s = 0; s < nsymtot; s++)
            if (len[s]) { wr16(cb + 3 * e, (uint16_t)s); cb[3 * e + 2] = len[s]; e++; }
        uint8_t *tb = out + HDR_BYTES + cb_bytes;
        for (uint64_t r = 0; r < rows; r++) {
            if (tw == 2) wr16(tb + 2 * r, (uint16_t)rowbytes[r]);
            else wr32(tb + 4 * r, (uint32_t)rowbytes[r]);
        }
        uint8_t *pl = tb + tab_bytes;
        uint64_t off = 0;
        for (uint64_t r = 0; r < rows; r++) {
            bw_t w = {pl + off, 0};
            for (uint64_t l = 0; l < Nr; l++) {
                uint64_t q = r * Nr + l;
                put_bits(&w, cw[code[q]], len[code[q]]);
                if (code[q] == 0) {
                    put_bits(&w, okv[q], 1);
                    put_bits(&w, (uint64_t)R[q] >> 32, 32);
                    put_bits(&w, (uint64_t)R[q] & 0xffffffffu, 32);
                    if (!okv[q]) put_bits(&w, f2u(x[q]), 32);
                }
            }
            off += rowbytes[r];
        }
    }
    if (codes_out) memcpy(codes_out, code, sizeof(uint16_t) * N);
done:
    free(t); free(P); free(R); free(okv); free(code); free(freq); free(len); free(cw); free(rowbytes);
    return rc;
}

/* ------------------------------------------------------------------ */
/* decompression (inverse path, same prediction in the same order)      */

int szo_decompress(const uint8_t *in, size_t in_len, float *out, size_t out_cap_elems) {
    if (!in || !out || in_len < HDR_BYTES) return SZO_EINVAL;
    if (!(in[0] == 'S' && in[1] == 'Z' && in[2] == 'G' && in[3] == 'B')) return SZO_ECORRUPT;
    if (rd16(in + 4) != 1 || rd16(in + 6) != HDR_BYTES) return SZO_ECORRUPT;
    int ndim = in[8], layers = in[9], m = in[10], tw = in[13];
    if (ndim < 1 || ndim > 4 || layers < 1 || layers > 4 || m < 2 || m > 16) return SZO_ECORRUPT;
    if (tw != 2 && tw != 4) return SZO_ECORRUPT;
    /* extents slowest first; a 4D field's slowest extent is at byte 120 */
    uint64_t d[4] = {ndim == 4 ? rd64(in + 120) : 1, rd64(in + 16), rd64(in + 24), rd64(in + 32)};
    uint64_t N = 1;
    for (int a = 0; a < 4; a++) {
        if (d[a] == 0 || d[a] >= ((uint64_t)1 << 32)) return SZO_ECORRUPT;
        N *= d[a];
        if (N >= ((uint64_t)1 << 32)) return SZO_ECORRUPT;
    }
    if (out_cap_elems < N) return SZO_EINVAL;
    float eb_f = u2f(rd32(in + 56));
    uint32_t nsym = rd32(in + 68);
    uint64_t nch = rd64(in + 72), K = rd64(in + 80), payload = rd64(in + 88), total = rd64(in + 96);
    uint64_t rows = d[0] * d[1] * d[2], Nr = d[3];
    uint32_t cpts = rd32(in + 116); /* chunk length; 0: whole rows */
    if (cpts && (!chunk_points_valid(cpts) || cpts >= Nr)) return SZO_ECORRUPT;
    uint64_t Ce = chunk_len(cpts, Nr), nseg = (Nr + Ce - 1) / Ce;
    if (nch != rows * nseg || nsym < 1 || nsym > (1u << m)) return SZO_ECORRUPT;
    uint64_t cb_bytes = pad4(3 * (uint64_t)nsym), tab_bytes = pad4((uint64_t)tw * nch);
    if (total != HDR_BYTES + cb_bytes + tab_bytes + payload || total > in_len) return SZO_ECORRUPT;

    int nsymtot = 1 << m;
    uint8_t *len = (uint8_t *)calloc((size_t)nsymtot, 1);
    uint64_t *cw = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)nsymtot);
    if (!len || !cw) { free(len); free(cw); return SZO_ENOMEM; }
    const uint8_t *cb = in + HDR_BYTES;
    int prev = -1;
    for (uint32_t e = 0; e < nsym; e++) {
        int s = rd16(cb + 3 * e), L = cb[3 * e + 2];
        if (s >= nsymtot || s <= prev || L < 1 || L > 64) { free(len); free(cw); return SZO_ECORRUPT; }
        len[s] = (uint8_t)L;
        prev = s;
    }
    szo_canonical_codes(len, nsymtot, cw);
    /* canonical decoding tables: the codes of length L are the consecutive
     * values first[L] .. first[L]+count[L]-1, taken by the symbols of that
     * length in ascending order (listed from sorted_sym + start[L]) */
    uint64_t first[65] = {0};
    uint32_t count[65] = {0}, start[65] = {0};
    int32_t *sorted_sym = (int32_t *)malloc(sizeof(int32_t) * nsym);
    if (!sorted_sym) { free(len); free(cw); return SZO_ENOMEM; }
    {
        uint32_t e = 0;
        for (int L = 1; L <= 64; L++) {
            start[L] = e;
            for (int s = 0; s < nsymtot; s++)
                if (len[s] == L) {
                    if (count[L] == 0) first[L] = cw[s];
                    count[L]++;
                    sorted_sym[e++] = s;
                }
        }
    }

    const int lattice = in[113] == 1;
    if (in[113] > 1 || (lattice && (ndim > 3 || cpts))) { free(len); free(cw); free(sorted_sym); return SZO_ECORRUPT; }
    const uint64_t d3[3] = {d[1], d[2], d[3]}; /* the lattice variant's 3-axis view (d[0] = 1) */
    int T;
    term_t *t = make_terms(ndim, layers, &T);
    iterm_t *it = lattice ? make_iterms(ndim, layers, &T) : NULL;
    int64_t *P = lattice ? (int64_t *)malloc(sizeof(int64_t) * N) : NULL;
    if (!t || (lattice && (!it || !P))) { free(t); free(it); free(P); free(len); free(cw); free(sorted_sym); return SZO_ENOMEM; }
    const uint8_t *tb = in + HDR_BYTES + cb_bytes;
    const uint8_t *pl = tb + tab_bytes;
    float twoeb = 2.0f * eb_f;
    int rc = SZO_OK;
    uint64_t off = 0, Kseen = 0;
    for (uint64_t ch = 0; ch < nch && rc == SZO_OK; ch++) {
        uint64_t nb = (tw == 2) ? rd16(tb + 2 * ch) : rd32(tb + 4 * ch);
        if (off + nb > payload) { rc = SZO_ECORRUPT; break; }
        br_t br = {pl + off, 0, nb * 8};
        /* chunk ch holds points l0 .. l1-1 of row r = ch / nseg, and row r the
         * points (r / (d1 d2), (r / d2) mod d1, r mod d2, 0..d3-1) */
        uint64_t r = ch / nseg, l0 = (ch % nseg) * Ce, l1 = l0 + Ce < Nr ? l0 + Ce : Nr;
        int64_t pt[4] = {(int64_t)(r / (d[1] * d[2])), (int64_t)((r / d[2]) % d[1]), (int64_t)(r % d[2]), 0};
        for (uint64_t l = l0; l < l1; l++) {
            pt[3] = (int64_t)l;
            /* bit-by-bit canonical decode */
            uint64_t c = 0;
            int L = 0, sym = -1;
            while (sym < 0) {
                int b = get_bit(&br);
                if (b < 0 || L >= 64) { rc = SZO_ECORRUPT; break; }
                c = (c << 1) | (uint64_t)b;
                L++;
                if (count[L] && c >= first[L] && c - first[L] < count[L])
                    sym = sorted_sym[start[L] + (uint32_t)(c - first[L])];
            }
            if (rc) break;
            uint64_t p = r * Nr + l;
            if (lattice) {
                /* p = r + integer prediction from the earlier lattice values */
                int64_t ipred = ipredict_at(P, d3, pt[1], pt[2], pt[3], it, T);
                if (sym != 0) {
                    P[p] = (int64_t)((uint64_t)ipred + (uint64_t)(int64_t)(sym - (1 << (m - 1))));
                    out[p] = szo_lattice_value(P[p], eb_f);
                } else {
                    int64_t ok = get_bits(&br, 1), hi = get_bits(&br, 32), lo = get_bits(&br, 32);
                    if (ok < 0 || hi < 0 || lo < 0) { rc = SZO_ECORRUPT; break; }
                    int64_t res = (int64_t)(((uint64_t)hi << 32) | (uint64_t)lo);
                    P[p] = (int64_t)((uint64_t)ipred + (uint64_t)res); /* modulo 2^64, as above */
                    if (ok) out[p] = szo_lattice_value(P[p], eb_f);
                    else {
                        int64_t u = get_bits(&br, 32);
                        if (u < 0) { rc = SZO_ECORRUPT; break; }
                        out[p] = u2f((uint32_t)u);
                    }
                    Kseen++;
                }
                continue;
            }
            float pred = predict_at(out, d, pt, t, T);
            if (sym != 0) {
                float step = (float)(sym - (1 << (m - 1))) * twoeb;
                out[p] = pred + step;
            } else {
                int64_t sg = get_bits(&br, 1), ex = get_bits(&br, 8);
                if (sg < 0 || ex < 0) { rc = SZO_ECORRUPT; break; }
                int tt;
                uint32_t ue = f2u(eb_f);
                int eeb = (int)((ue >> 23) & 0xff);
                if (eeb == 0) tt = 23;
                else { int ee = ex < 1 ? 1 : (int)ex; tt = ee - eeb; if (tt < 0) tt = 0; if (tt > 23) tt = 23; }
                int64_t mb = tt ? get_bits(&br, tt) : 0;
                if (mb < 0) { rc = SZO_ECORRUPT; break; }
                uint32_t u = ((uint32_t)sg << 31) | ((uint32_t)ex << 23) | ((uint32_t)mb << (23 - tt));
                out[p] = u2f(u);
                Kseen++;
            }
        }
        off += nb;
    }
    if (rc == SZO_OK && Kseen != K) rc = SZO_ECORRUPT;
    free(t); free(it); free(P); free(len); free(cw); free(sorted_sym);
    return rc;
}
