// k_hyper.cu -- 3D fields with n = 3 or 4 layers (Sec. III, Eq. predmodel):
// the prediction, quantization, fallback and record of Algorithm 1, and the
// matching reconstruction, one hyperplane i + j + l = h per launch.
//
// A 3D wavefront lane would keep (n+1)^3 - 1 neighbour values in registers
// (63 at n = 3, 124 at n = 4), which does not fit beside the wavefront's
// helper warps.  Here every neighbour comes from the recorded values in
// global memory (L2-resident for the planes in flight) instead.  A point's
// neighbours all lie on earlier hyperplanes, so one launch per hyperplane on
// one stream is the whole schedule: a launch boundary orders the hyperplanes,
// and there is no device-side wait of any kind.  The arithmetic is the
// wavefront's: the same term order, products and sums rounded one at a time,
// the same quantizer and truncation.
#include "hyper_box.h"
#include "szgb_internal.cuh"

namespace szgb {

constexpr int kHyperThreads = 256;

// n-layer prediction of point (i, j, l) from V, terms in descending
// lexicographic order of k, values outside the field 0.  V is written by
// earlier launches, so it is read through L2 (no read-only cache).
template <int NL>
__device__ __forceinline__ float predict_hyper(const float* V, uint64_t M, uint64_t N, int64_t i, int64_t j,
                                               int64_t l) {
    float pred = 0.0f;
    bool first = true;
#pragma unroll
    for (int k0 = NL; k0 >= 0; k0--) {
#pragma unroll
        for (int k1 = NL; k1 >= 0; k1--) {
#pragma unroll
            for (int k2 = NL; k2 >= 0; k2--) {
                if (k0 == 0 && k1 == 0 && k2 == 0) continue;
                const int64_t ii = i - k0, jj = j - k1, ll = l - k2;
                float v = 0.0f;
                if (ii >= 0 && jj >= 0 && ll >= 0) v = __ldcg(V + ((uint64_t)ii * M + (uint64_t)jj) * N + (uint64_t)ll);
                const float prod = __fmul_rn((float)term_coef(NL, k0, k1, k2), v);
                pred = first ? prod : __fadd_rn(pred, prod);
                first = false;
            }
        }
    }
    return pred;
}

// One hyperplane.  DEC = false: x -> codes and recorded values V.
// DEC = true: codes (and, at code 0, the unpredictable value already in V,
// as the row decoder leaves it) -> reconstructed V.
template <int NL, bool DEC>
__global__ void __launch_bounds__(kHyperThreads) k_hyper(const float* __restrict__ x, float* V, uint16_t* codes,
                                                         uint64_t cpitch, uint64_t M, uint64_t N, int64_t h,
                                                         HyperBox b, const DevState* st) {
    if (st->err) return;
    const uint64_t t = blockIdx.x * (uint64_t)kHyperThreads + threadIdx.x;
    if (t >= b.ni * b.nj) return;
    const int64_t i = b.ilo + (int64_t)(t / b.nj), j = b.jlo + (int64_t)(t % b.nj), l = h - i - j;
    if (l < 0 || (uint64_t)l >= N) return;
    const QParams qp = load_qparams(st);
    const uint64_t row = (uint64_t)i * M + (uint64_t)j;
    const uint64_t p = row * N + (uint64_t)l;
    const float pred = predict_hyper<NL>(V, M, N, i, j, l);
    if (DEC) {
        const int code = codes[row * cpitch + (uint64_t)l];
        if (code) V[p] = dequantize(code, pred, qp);
    } else {
        const float xv = x[p];
        float rec;
        const int code = quantize_tr(xv, pred, trunc_value(xv, qp.e_eb), qp, rec);  // as the wavefront
        V[p] = rec;
        codes[row * cpitch + (uint64_t)l] = (uint16_t)code;
    }
}

template <int NL, bool DEC>
static int run_hyper(const float* x, float* V, uint16_t* codes, uint64_t cpitch, uint64_t P, uint64_t M, uint64_t N,
                     const DevState* st, cudaStream_t s) {
    const int64_t H = (int64_t)(P - 1) + (int64_t)(M - 1) + (int64_t)(N - 1);
    for (int64_t h = 0; h <= H; h++) {
        const HyperBox b = hyper_box(h, (int64_t)P, (int64_t)M, (int64_t)N);
        const uint64_t n = b.ni * b.nj;
        if (n == 0) continue;
        const unsigned blocks = (unsigned)((n + kHyperThreads - 1) / kHyperThreads);
        k_hyper<NL, DEC><<<blocks, kHyperThreads, 0, s>>>(x, V, codes, cpitch, M, N, h, b, st);
        if (cudaGetLastError() != cudaSuccess) return SZGB_ECUDA;
    }
    return SZGB_OK;
}

// Compression of a P x M x N field with n = 3 or 4 layers: codes (row pitch
// cpitch) and the recorded values V (N points, raster order).  The state
// holds the bound and m (range and adaptive-m kernels run before).
int launch_hyper_compress(int layers, const float* x, float* V, uint16_t* codes, uint64_t cpitch, uint64_t P,
                          uint64_t M, uint64_t N, const DevState* st, cudaStream_t s) {
    if (layers == 3) return run_hyper<3, false>(x, V, codes, cpitch, P, M, N, st, s);
    if (layers == 4) return run_hyper<4, false>(x, V, codes, cpitch, P, M, N, st, s);
    return SZGB_EUNSUPPORTED;
}

// Reconstruction: codes from the row decoder, unpredictable values already in
// out at their points; out is completed in place.
int launch_hyper_decompress(int layers, uint16_t* codes, uint64_t cpitch, float* out, uint64_t P, uint64_t M,
                            uint64_t N, const DevState* st, cudaStream_t s) {
    if (layers == 3) return run_hyper<3, true>(nullptr, out, codes, cpitch, P, M, N, st, s);
    if (layers == 4) return run_hyper<4, true>(nullptr, out, codes, cpitch, P, M, N, st, s);
    return SZGB_EUNSUPPORTED;
}

}  // namespace szgb
