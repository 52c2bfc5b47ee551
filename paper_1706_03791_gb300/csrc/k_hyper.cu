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

template <int NL, bool DEC>
__global__ void __launch_bounds__(kHyperThreads) k_hyper4(const float* __restrict__ x, float* V, uint16_t* codes,
                                                          uint64_t cpitch, Dims4 d, int64_t h, HyperBox4 b,
                                                          const DevState* st) {
    if (st->err) return;
    const uint64_t t = blockIdx.x * (uint64_t)kHyperThreads + threadIdx.x;
    const uint64_t plane = b.ni * b.nj;
    if (t >= b.na * plane) return;
    const int64_t a = b.alo + (int64_t)(t / plane), i = b.ilo + (int64_t)((t / b.nj) % b.ni),
                  j = b.jlo + (int64_t)(t % b.nj), l = h - a - i - j;
    if (l < 0 || (uint64_t)l >= d.N) return;
    const QParams qp = load_qparams(st);
    const uint64_t row = ((uint64_t)a * d.P + (uint64_t)i) * d.M + (uint64_t)j;
    const uint64_t p = row * d.N + (uint64_t)l;
    const float pred = predict4<NL, false>(V, d, a, i, j, l);
    if (DEC) {
        const int code = codes[row * cpitch + (uint64_t)l];
        if (code) V[p] = dequantize(code, pred, qp);
    } else {
        const float xv = x[p];
        float rec;
        const int code = quantize_tr(xv, pred, trunc_value(xv, qp.e_eb), qp, rec);
        V[p] = rec;
        codes[row * cpitch + (uint64_t)l] = (uint16_t)code;
    }
}

template <int NL, bool DEC>
static int run_hyper4(const float* x, float* V, uint16_t* codes, uint64_t cpitch, const Dims4& d,
                      const DevState* st, cudaStream_t s) {
    const int64_t H = (int64_t)(d.D - 1) + (int64_t)(d.P - 1) + (int64_t)(d.M - 1) + (int64_t)(d.N - 1);
    for (int64_t h = 0; h <= H; h++) {
        const HyperBox4 b = hyper_box4(h, (int64_t)d.D, (int64_t)d.P, (int64_t)d.M, (int64_t)d.N);
        const uint64_t n = b.na * b.ni * b.nj;
        if (n == 0) continue;
        const unsigned blocks = (unsigned)((n + kHyperThreads - 1) / kHyperThreads);
        k_hyper4<NL, DEC><<<blocks, kHyperThreads, 0, s>>>(x, V, codes, cpitch, d, h, b, st);
        if (cudaGetLastError() != cudaSuccess) return SZGB_ECUDA;
    }
    return SZGB_OK;
}

int launch_hyper4(bool dec, int layers, const float* x, float* V, uint16_t* codes, uint64_t cpitch, uint64_t D,
                  uint64_t P, uint64_t M, uint64_t N, const DevState* st, cudaStream_t s) {
    const Dims4 d = {D, P, M, N};
    switch (layers * 2 + (dec ? 1 : 0)) {
        case 2: return run_hyper4<1, false>(x, V, codes, cpitch, d, st, s);
        case 3: return run_hyper4<1, true>(x, V, codes, cpitch, d, st, s);
        case 4: return run_hyper4<2, false>(x, V, codes, cpitch, d, st, s);
        case 5: return run_hyper4<2, true>(x, V, codes, cpitch, d, st, s);
        case 6: return run_hyper4<3, false>(x, V, codes, cpitch, d, st, s);
        case 7: return run_hyper4<3, true>(x, V, codes, cpitch, d, st, s);
        case 8: return run_hyper4<4, false>(x, V, codes, cpitch, d, st, s);
        case 9: return run_hyper4<4, true>(x, V, codes, cpitch, d, st, s);
        default: return SZGB_EUNSUPPORTED;
    }
}

// Adaptive m of a 4D field: the samples are the points whose four coordinates
// are all multiples of 8, predicted from the original values, each counted
// under the smallest m whose radius holds its q; then the smallest m whose
// cumulative count reaches ceil(theta S), else 16 (as the 1D-3D kernel).
template <int NL>
__global__ void __launch_bounds__(256) k_adapt4(const float* __restrict__ x, Dims4 d, double theta, DevState* st) {
    __shared__ unsigned long long cnt[18];
    __shared__ bool last;
    if (st->err) return;
    if (threadIdx.x < 18) cnt[threadIdx.x] = 0;
    __syncthreads();
    const uint64_t S0 = (d.D + 7) / 8, S1 = (d.P + 7) / 8, S2 = (d.M + 7) / 8, S3 = (d.N + 7) / 8;
    const uint64_t S = S0 * S1 * S2 * S3;
    const float ebf = st->eb_f, twoeb = st->twoeb, inv = st->inv2eb;
    for (uint64_t s = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; s < S;
         s += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t c3 = s % S3, r2 = s / S3, c2 = r2 % S2, r1 = r2 / S2, c1 = r1 % S1, c0 = r1 / S1;
        const int64_t a = (int64_t)(c0 * 8), i = (int64_t)(c1 * 8), j = (int64_t)(c2 * 8), l = (int64_t)(c3 * 8);
        const float xv = __ldg(x + (((uint64_t)a * d.P + (uint64_t)i) * d.M + (uint64_t)j) * d.N + (uint64_t)l);
        const float pred = predict4<NL, true>(x, d, a, i, j, l);
        const float diff = __fsub_rn(xv, pred);
        const float q = rintf(__fmul_rn(diff, inv));
        if (!(fabsf(q) <= 32767.0f)) continue;
        const float qn = __fadd_rn(q, 0.0f);
        const float dq = __fadd_rn(pred, __fmul_rn(qn, twoeb));
        if (!(fabsf(__fsub_rn(xv, dq)) < ebf || xv == dq)) continue;
        const int aq = (int)fabsf(q);
        int mm = 2;
        while (aq > (1 << (mm - 1)) - 1) mm++;
        atomicAdd(&cnt[mm], 1ull);
    }
    __syncthreads();
    if (threadIdx.x < 18 && cnt[threadIdx.x]) atomicAdd(&st->need[threadIdx.x], cnt[threadIdx.x]);
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned t = atomicAdd(&st->adapt_blocks_done, 1u);
        last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!last || threadIdx.x != 0) return;
    __threadfence();
    const volatile unsigned long long* need = st->need;
    const double req = ceil(theta * (double)S);
    unsigned long long cum = 0;
    int m = 16;
    for (int mm = 2; mm <= 16; mm++) {
        cum += need[mm];
        if ((double)cum >= req) {
            m = mm;
            break;
        }
    }
    st->nsamples = S;
    st->m = m;
    st->center = 1 << (m - 1);
    st->radius = (float)((1 << (m - 1)) - 1);
}

int launch_adapt4(const float* x, uint64_t D, uint64_t P, uint64_t M, uint64_t N, int layers, double theta,
                  DevState* st, cudaStream_t s) {
    const Dims4 d = {D, P, M, N};
    const uint64_t S = ((D + 7) / 8) * ((P + 7) / 8) * ((M + 7) / 8) * ((N + 7) / 8);
    int blocks = (int)((S + 255) / 256);
    blocks = blocks > 1024 ? 1024 : (blocks < 1 ? 1 : blocks);
    switch (layers) {
        case 1: k_adapt4<1><<<blocks, 256, 0, s>>>(x, d, theta, st); break;
        case 2: k_adapt4<2><<<blocks, 256, 0, s>>>(x, d, theta, st); break;
        case 3: k_adapt4<3><<<blocks, 256, 0, s>>>(x, d, theta, st); break;
        case 4: k_adapt4<4><<<blocks, 256, 0, s>>>(x, d, theta, st); break;
        default: return SZGB_EUNSUPPORTED;
    }
    return cudaGetLastError() == cudaSuccess ? SZGB_OK : SZGB_ECUDA;
}

// The header of a 4D stream: written for the field's (D P) x M x N view, then
// ndim = 4, the extents P, M, N at bytes 16..40 and D at byte 120.
__global__ void k_patch_header4(uint8_t* h, uint64_t D, uint64_t P, const DevState* st) {
    if (!st->fits || st->err || threadIdx.x != 0 || blockIdx.x != 0) return;  // as the header writer
    h[8] = 4;
    for (int k = 0; k < 8; k++) {
        h[16 + k] = (uint8_t)(P >> (8 * k));
        h[120 + k] = (uint8_t)(D >> (8 * k));
    }
}

int launch_patch_header4(uint8_t* header, uint64_t D, uint64_t P, const DevState* st, cudaStream_t s) {
    k_patch_header4<<<1, 32, 0, s>>>(header, D, P, st);
    return cudaGetLastError() == cudaSuccess ? SZGB_OK : SZGB_ECUDA;
}

}  // namespace szgb
