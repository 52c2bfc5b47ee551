/*
 * oracle_fuzz.c -- robustness of the oracle's stream reader: streams of the
 * exact method and of the lattice variant (1D..4D fields, several n, m and
 * bound modes) are corrupted at random (byte overwrites in the header and
 * the body, truncations, bit flips) and decoded.  Built with AddressSanitizer
 * and UndefinedBehaviorSanitizer by the test that runs it: every call must
 * return an error code or decode within the declared shape, with no invalid
 * memory access and no undefined behaviour.  The unmodified streams must
 * decode to exactly the values the compressor recorded.
 *
 * Usage: oracle_fuzz <seed> <mutations per stream>
 */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "../../oracle/szo.h"

static uint64_t rs;
static uint64_t rnd(void) { /* xorshift64* */
    rs ^= rs >> 12; rs ^= rs << 25; rs ^= rs >> 27;
    return rs * 2685821657736338717ull;
}
static double urand(void) { return (double)(rnd() >> 11) / 9007199254740992.0; }

#define CAP (1 << 16)

static int check_stream(const uint8_t *s, size_t len, const float *rec, uint64_t N, int muts,
                        uint64_t counts[3]) {
    float *out = (float *)malloc(sizeof(float) * CAP);
    uint8_t *m = (uint8_t *)malloc(len + 64);
    if (!out || !m) return 1;
    int rc = szo_decompress(s, len, out, CAP);
    if (rc != 0 || memcmp(out, rec, sizeof(float) * N) != 0) {
        fprintf(stderr, "clean stream failed to round-trip (rc %d)\n", rc);
        free(out); free(m);
        return 1;
    }
    for (int t = 0; t < muts; t++) {
        size_t ml = len;
        memcpy(m, s, len);
        int kind = (int)(rnd() % 4);
        int reps = 1 + (int)(rnd() % 4);
        for (int r = 0; r < reps; r++) {
            if (kind == 0) {         /* a header byte */
                m[rnd() % 128] = (uint8_t)rnd();
            } else if (kind == 1) {  /* a body byte */
                if (len > 128) m[128 + rnd() % (len - 128)] = (uint8_t)rnd();
            } else if (kind == 2) {  /* a bit anywhere */
                size_t b = rnd() % (len * 8);
                m[b / 8] ^= (uint8_t)(1u << (b % 8));
            } else {                 /* truncation */
                ml = (size_t)(rnd() % (len + 1));
            }
        }
        rc = szo_decompress(m, ml, out, CAP);
        counts[rc == 0 ? 0 : (rc == -4 ? 1 : 2)]++;
    }
    free(out); free(m);
    return 0;
}

int main(int argc, char **argv) {
    rs = argc > 1 ? strtoull(argv[1], NULL, 10) * 0x9e3779b97f4a7c15ull + 1 : 1;
    int muts = argc > 2 ? atoi(argv[2]) : 200;
    static const uint64_t shapes[][4] = {
        {1, 1, 1, 257}, {1, 1, 13, 17}, {1, 5, 6, 7}, {3, 4, 5, 6}, {1, 1, 1, 1}, {1, 1, 2, 1}};
    static const int ndims[] = {1, 2, 3, 4, 1, 2};
    uint64_t counts[3] = {0, 0, 0};
    size_t cap = 1 << 22;
    uint8_t *s = (uint8_t *)malloc(cap);
    float *x = (float *)malloc(sizeof(float) * CAP);
    float *rec = (float *)malloc(sizeof(float) * CAP);
    if (!s || !x || !rec) return 1;
    for (int f = 0; f < 6; f++) {
        int nd = ndims[f];
        const uint64_t *d4 = shapes[f];
        uint64_t N = d4[0] * d4[1] * d4[2] * d4[3];
        const uint64_t *shape = d4 + (4 - nd);
        for (int variant = 0; variant < 2; variant++) {
            if (variant == 1 && nd > 3) continue;
            for (int n = 1; n <= (variant ? 2 : 4); n++) {
                for (int mi = 0; mi < 3; mi++) {
                    int m = mi == 0 ? 0 : (mi == 1 ? 3 : 9);
                    /* the lattice form needs eb > 0: an absolute bound (a one-point
                     * field has range 0) */
                    int mode = variant ? 0 : (int)(rnd() % 3);
                    /* a smooth ramp with noise and an occasional outlier */
                    for (uint64_t p = 0; p < N; p++)
                        x[p] = (float)(0.01 * (double)p + 0.3 * sin(0.1 * (double)p) + 0.01 * urand() +
                                       (urand() < 0.01 ? 100.0 : 0.0));
                    size_t len = 0;
                    int rc = variant ? szo_compress_lattice(x, nd, shape, mode, 1e-3, 1e-3, n, m, 0.99, s, cap,
                                                            &len, rec, NULL)
                                     : szo_compress(x, nd, shape, mode, 1e-3, 1e-3, n, m, 0.99, 0, s, cap, &len,
                                                    rec, NULL);
                    if (rc != 0) {
                        fprintf(stderr, "compress failed: nd %d n %d m %d variant %d rc %d\n", nd, n, m, variant, rc);
                        free(s); free(x); free(rec);
                        return 1;
                    }
                    if (check_stream(s, len, rec, N, muts, counts)) {
                        free(s); free(x); free(rec);
                        return 1;
                    }
                }
            }
        }
    }
    printf("decoded %llu corrupt %llu other %llu\n", (unsigned long long)counts[0],
           (unsigned long long)counts[1], (unsigned long long)counts[2]);
    free(s); free(x); free(rec);
    return 0;
}
