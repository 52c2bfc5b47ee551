// hyper_kernels.cuh -- device code shared by the hyperplane kernels of 3D
// fields with n = 3, 4 layers and 4D fields (Sec. III, Eq. predmodel): the
// 4D term coefficients and prediction, the 4D adaptive-m sample and the 4D
// prediction hit (the tiled schedule itself is in hyper_tile.cuh).
//
// Included by k_hyper.cu after szgb_internal.cuh (which supplies DevState,
// QParams, load_qparams, quantize_tr, dequantize, trunc_value, sgn_binom and
// term_coef) and hyper_box.h; the host-side emulation test includes it the
// same way with host definitions of those, and runs these very kernels on the
// CPU against the oracle.
#ifndef SZGB_HYPER_KERNELS_CUH
#define SZGB_HYPER_KERNELS_CUH

namespace szgb {

// ---------------------------------------------------------------------------
// 4D fields D x P x M x N (the predictor of Eq. predmodel with d = 4): the same
// scheme over hyperplanes i0 + i + j + l = h.  Rows are the (i0, i, j) lines
// of length N, so the codes and every later stage see a field of D P M rows.

__host__ __device__ __forceinline__ constexpr int term_coef4(int n, int k0, int k1, int k2, int k3) {
    return -sgn_binom(n, k0) * sgn_binom(n, k1) * sgn_binom(n, k2) * sgn_binom(n, k3);
}

struct Dims4 {
    uint64_t D, P, M, N;
};

// n-layer prediction of point (a, i, j, l) from V, terms in descending
// lexicographic order of k, values outside the field 0.  RO: V is read-only
// for the kernel's lifetime (original values), else it was written by
// earlier launches and is read through L2.
template <int NL, bool RO>
__device__ __forceinline__ float predict4(const float* V, const Dims4& d, int64_t a, int64_t i, int64_t j,
                                          int64_t l) {
    float pred = 0.0f;
    bool first = true;
#pragma unroll
    for (int k0 = NL; k0 >= 0; k0--) {
#pragma unroll
        for (int k1 = NL; k1 >= 0; k1--) {
#pragma unroll
            for (int k2 = NL; k2 >= 0; k2--) {
#pragma unroll
                for (int k3 = NL; k3 >= 0; k3--) {
                    if (k0 == 0 && k1 == 0 && k2 == 0 && k3 == 0) continue;
                    const int64_t aa = a - k0, ii = i - k1, jj = j - k2, ll = l - k3;
                    float v = 0.0f;
                    if (aa >= 0 && ii >= 0 && jj >= 0 && ll >= 0) {
                        const float* q = V + (((uint64_t)aa * d.P + (uint64_t)ii) * d.M + (uint64_t)jj) * d.N + (uint64_t)ll;
                        v = RO ? __ldg(q) : __ldcg(q);
                    }
                    const float prod = __fmul_rn((float)term_coef4(NL, k0, k1, k2, k3), v);
                    pred = first ? prod : __fadd_rn(pred, prod);
                    first = false;
                }
            }
        }
    }
    return pred;
}

// One adaptive-m sample of a 4D field (sample index s over the points whose
// coordinates are all multiples of 8): the smallest m whose radius holds its
// q, predicted from the original values, or 0 when no interval holds it.
template <int NL>
__device__ __forceinline__ int adapt4_bucket(const float* __restrict__ x, const Dims4& d, uint64_t s, float ebf,
                                             float twoeb, float inv) {
    const uint64_t S1 = (d.P + 7) / 8, S2 = (d.M + 7) / 8, S3 = (d.N + 7) / 8;
    const uint64_t c3 = s % S3, r2 = s / S3, c2 = r2 % S2, r1 = r2 / S2, c1 = r1 % S1, c0 = r1 / S1;
    const int64_t a = (int64_t)(c0 * 8), i = (int64_t)(c1 * 8), j = (int64_t)(c2 * 8), l = (int64_t)(c3 * 8);
    const float xv = __ldg(x + (((uint64_t)a * d.P + (uint64_t)i) * d.M + (uint64_t)j) * d.N + (uint64_t)l);
    const float pred = predict4<NL, true>(x, d, a, i, j, l);
    const float diff = __fsub_rn(xv, pred);
    const float q = rintf(__fmul_rn(diff, inv));
    if (!(fabsf(q) <= 32767.0f)) return 0;
    const float qn = __fadd_rn(q, 0.0f);
    const float dq = __fadd_rn(pred, __fmul_rn(qn, twoeb));
    if (!(fabsf(__fsub_rn(xv, dq)) < ebf || xv == dq)) return 0;
    const int aq = (int)fabsf(q);
    int mm = 2;
    while (aq > (1 << (mm - 1)) - 1) mm++;
    return mm;
}

// Prediction hit of point s (raster index) of a 4D field (Sec. III): the
// n-layer prediction from the values V at its preceding neighbours lies
// within eb of x, compared in float64 (V = x: original values).
template <int NL>
__device__ __forceinline__ bool hit4_point(const float* __restrict__ x, const float* __restrict__ V, const Dims4& d,
                                           uint64_t s, double eb) {
    const uint64_t l = s % d.N, r1 = s / d.N, j = r1 % d.M, r2 = r1 / d.M, i = r2 % d.P, a = r2 / d.P;
    const float pred = predict4<NL, true>(V, d, (int64_t)a, (int64_t)i, (int64_t)j, (int64_t)l);
    return fabs((double)__ldg(x + s) - (double)pred) <= eb;
}

}  // namespace szgb

#endif
