// k_range.cu -- value range, finite check, effective error bound, and the
// adaptive choice of the interval count m.
//
// Range: R_X = x_max - x_min (Sec. II); the value-range-relative bound is
// eb = eb_rel * R_X, the effective bound eb_f the largest float <= eb.
// Adaptive m (Sec. IV-B): the smallest m whose 2^m - 1 intervals hold a
// fraction theta of a sample of points, predicted from original values.
#include <float.h>

#include "szgb_internal.cuh"

namespace szgb {

// ---------------------------------------------------------------------------
// K1: min / max / non-finite over the field; the last block to finish derives
// the bound and quantizer parameters.

__device__ __forceinline__ void minmax_acc(float v, float& mn, float& mx, unsigned& bad) {
    bad |= !isfinite(v);
    mn = fminf(mn, v);
    mx = fmaxf(mx, v);
}

__global__ void __launch_bounds__(256) k_range(const float* __restrict__ x, uint64_t n,
                                               float* partials, DevState* st, CallParams cp) {
    float mn = FLT_MAX, mx = -FLT_MAX;
    unsigned bad = 0;
    const uint64_t tid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    const uint64_t nthr = (uint64_t)gridDim.x * blockDim.x;
    if ((reinterpret_cast<uintptr_t>(x) & 15) == 0) {
        const float4* x4 = reinterpret_cast<const float4*>(x);
        uint64_t n4 = n / 4;
        // four independent 16-byte loads in flight per thread
        uint64_t i = tid;
        for (; i + 3 * nthr < n4; i += 4 * nthr) {
            float4 v[4];
#pragma unroll
            for (int k = 0; k < 4; k++) v[k] = __ldcs(x4 + i + k * nthr);
#pragma unroll
            for (int k = 0; k < 4; k++) {
                minmax_acc(v[k].x, mn, mx, bad);
                minmax_acc(v[k].y, mn, mx, bad);
                minmax_acc(v[k].z, mn, mx, bad);
                minmax_acc(v[k].w, mn, mx, bad);
            }
        }
        for (; i < n4; i += nthr) {
            float4 v = __ldcs(x4 + i);
            minmax_acc(v.x, mn, mx, bad);
            minmax_acc(v.y, mn, mx, bad);
            minmax_acc(v.z, mn, mx, bad);
            minmax_acc(v.w, mn, mx, bad);
        }
        for (uint64_t i = n4 * 4 + tid; i < n; i += nthr) minmax_acc(x[i], mn, mx, bad);
    } else {
        for (uint64_t i = tid; i < n; i += nthr) minmax_acc(x[i], mn, mx, bad);
    }
    for (int o = 16; o > 0; o >>= 1) {
        mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
        mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        bad |= __shfl_xor_sync(0xffffffffu, bad, o);
    }
    __shared__ float smn[8], smx[8];
    __shared__ unsigned sbad[8];
    __shared__ bool last;
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) { smn[w] = mn; smx[w] = mx; sbad[w] = bad; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = 1; i < (int)(blockDim.x >> 5); i++) {
            mn = fminf(mn, smn[i]);
            mx = fmaxf(mx, smx[i]);
            bad |= sbad[i];
        }
        partials[2 * blockIdx.x] = mn;
        partials[2 * blockIdx.x + 1] = mx;
        if (bad) atomicOr(&st->nonfinite, 1u);
        __threadfence();
        unsigned t = atomicAdd(&st->range_blocks_done, 1u);
        last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    // the last block: every thread folds a strided share of the partials,
    // then the block reduces them (min and max are exact in any order)
    __threadfence();
    const volatile float* vp = partials;
    mn = FLT_MAX;
    mx = -FLT_MAX;
    for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x) {
        mn = fminf(mn, vp[2 * b]);
        mx = fmaxf(mx, vp[2 * b + 1]);
    }
    for (int o = 16; o > 0; o >>= 1) {
        mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
        mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    __syncthreads();  // smn / smx are reused
    if (l == 0) { smn[w] = mn; smx[w] = mx; }
    __syncthreads();
    if (threadIdx.x != 0) return;
    for (int i = 1; i < (int)(blockDim.x >> 5); i++) {
        mn = fminf(mn, smn[i]);
        mx = fmaxf(mx, smx[i]);
    }
    // the stored range is the value range: a signed zero is stored as +0
    mn = __fadd_rn(mn, 0.0f);
    mx = __fadd_rn(mx, 0.0f);
    st->xmin = mn;
    st->xmax = mx;
    if (st->nonfinite) st->err |= kErrNonFinite;
    double range = (double)mx - (double)mn;
    double eb;
    if (cp.mode == SZGB_ABS) eb = cp.eb_abs;
    else if (cp.mode == SZGB_REL) eb = cp.eb_rel * range;
    else eb = fmin(cp.eb_abs, cp.eb_rel * range);
    float ebf = __double2float_rz(eb);  // largest float <= eb (eb >= 0)
    st->eb_f = ebf;
    float twoeb = __fmul_rn(2.0f, ebf);
    st->twoeb = twoeb;
    st->inv2eb = ebf > 0.0f ? __fdiv_rn(1.0f, twoeb) : 0.0f;
    st->e_eb = (int)((__float_as_uint(ebf) >> 23) & 0xffu);
    if (cp.variant == 1) {  // the lattice needs a positive spacing and integers below 2^30
        const float amax = fmaxf(fabsf(mn), fabsf(mx));
        if (!(ebf > 0.0f) || !(__fmul_rn(amax, __fdiv_rn(1.0f, __fmul_rn(2.0f, ebf))) < 1073741824.0f))
            st->err |= kErrRange;
    }
    st->adaptive = cp.m_user == 0;
    if (cp.m_user) {
        st->m = cp.m_user;
        st->center = 1 << (cp.m_user - 1);
        st->radius = (float)((1 << (cp.m_user - 1)) - 1);
    }
}

int launch_range(const float* x, uint64_t n, DevState* st, const CallParams& cp, float* partials,
                 int nblocks, cudaStream_t s) {
    k_range<<<nblocks, 256, 0, s>>>(x, n, partials, st, cp);
    return cudaGetLastError() == cudaSuccess ? 0 : SZGB_ECUDA;
}

// ---------------------------------------------------------------------------
// The field's rows at a 16-byte row pitch, for the wavefront's TMA tiles when
// the row length N is not a multiple of 4 (a TMA tile needs 16-byte row
// strides): row r of x goes to xp + r P, P = N rounded up to 4.  A warp
// copies one row at a time (coalesced loads and stores), grid-stride over
// the rows.

__global__ void __launch_bounds__(256) k_pitch_rows(const float* __restrict__ x, uint64_t rows, uint64_t N,
                                                    float* __restrict__ xp, uint64_t P) {
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const int lane = threadIdx.x & 31;
    for (uint64_t r = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < rows; r += nw) {
        const float* src = x + r * N;
        float* dst = xp + r * P;
#pragma unroll 4
        for (uint64_t c = (uint64_t)lane; c < N; c += 32) dst[c] = __ldg(src + c);
    }
}

int launch_pitch_rows(const float* x, uint64_t rows, uint64_t N, float* xp, uint64_t P, int sm_count, cudaStream_t s) {
    uint64_t blocks = (rows + 7) / 8;  // 8 warps a block
    const uint64_t cap = 8ull * (uint64_t)(sm_count > 0 ? sm_count : 1);
    blocks = blocks < 1 ? 1 : (blocks > cap ? cap : blocks);
    k_pitch_rows<<<(unsigned)blocks, 256, 0, s>>>(x, rows, N, xp, P);
    return cudaGetLastError() == cudaSuccess ? 0 : SZGB_ECUDA;
}

// ---------------------------------------------------------------------------
// K8: adaptive m.  Samples are the points whose coordinates are all multiples
// of 8; each is predicted from the ORIGINAL neighbour values with the n-layer
// stencil (terms in descending lexicographic order, products and sums rounded
// one by one) and counted under the smallest m whose radius holds its q.

template <int NL>
__device__ float predict_original(const float* __restrict__ x, uint64_t M, uint64_t N, int64_t i,
                                  int64_t j, int64_t l, int ndim) {
    float pred = 0.0f;
    bool first = true;
    const int K0 = (ndim == 3) ? NL : 0;
    const int K1 = (ndim >= 2) ? NL : 0;
#pragma unroll
    for (int k0 = NL; k0 >= 0; k0--) {
        if (k0 > K0) continue;
#pragma unroll
        for (int k1 = NL; k1 >= 0; k1--) {
            if (k1 > K1) continue;
#pragma unroll
            for (int k2 = NL; k2 >= 0; k2--) {
                if (k0 == 0 && k1 == 0 && k2 == 0) continue;
                int64_t ii = i - k0, jj = j - k1, ll = l - k2;
                float v = 0.0f;
                if (ii >= 0 && jj >= 0 && ll >= 0) v = __ldg(x + ((uint64_t)ii * M + (uint64_t)jj) * N + (uint64_t)ll);
                float prod = __fmul_rn((float)term_coef(NL, k0, k1, k2), v);
                pred = first ? prod : __fadd_rn(pred, prod);
                first = false;
            }
        }
    }
    return pred;
}

template <int NL>
__global__ void __launch_bounds__(256) k_adapt(const float* __restrict__ x, CallParams cp, DevState* st) {
    __shared__ unsigned long long cnt[18];
    __shared__ bool last;
    if (st->err) return;
    if (threadIdx.x < 18) cnt[threadIdx.x] = 0;
    __syncthreads();
    const uint64_t S0 = (cp.d0 + 7) / 8, S1 = (cp.d1 + 7) / 8, S2 = (cp.d2 + 7) / 8;
    const uint64_t S = S0 * S1 * S2;
    const float ebf = st->eb_f, twoeb = st->twoeb, inv = st->inv2eb;
    for (uint64_t s = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; s < S;
         s += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t a = s / (S1 * S2), r = s % (S1 * S2);
        int64_t i = (int64_t)(a * 8), j = (int64_t)((r / S2) * 8), l = (int64_t)((r % S2) * 8);
        float xv = __ldg(x + ((uint64_t)i * cp.d1 + (uint64_t)j) * cp.d2 + (uint64_t)l);
        float pred = predict_original<NL>(x, cp.d1, cp.d2, i, j, l, cp.ndim);
        float diff = __fsub_rn(xv, pred);
        float q = rintf(__fmul_rn(diff, inv));
        if (!(fabsf(q) <= 32767.0f)) continue;
        float qn = __fadd_rn(q, 0.0f);
        float dq = __fadd_rn(pred, __fmul_rn(qn, twoeb));
        if (!(fabsf(__fsub_rn(xv, dq)) < ebf || xv == dq)) continue;
        int aq = (int)fabsf(q);
        int mm = 2;
        while (aq > (1 << (mm - 1)) - 1) mm++;
        atomicAdd(&cnt[mm], 1ull);
    }
    __syncthreads();
    if (threadIdx.x < 18 && cnt[threadIdx.x]) atomicAdd(&st->need[threadIdx.x], cnt[threadIdx.x]);
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        unsigned t = atomicAdd(&st->adapt_blocks_done, 1u);
        last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!last || threadIdx.x != 0) return;
    __threadfence();
    const volatile unsigned long long* need = st->need;
    double req = ceil(cp.theta * (double)S);
    unsigned long long cum = 0;
    int m = 16;
    for (int mm = 2; mm <= 16; mm++) {
        cum += need[mm];
        if ((double)cum >= req) { m = mm; break; }
    }
    st->nsamples = S;
    st->m = m;
    st->center = 1 << (m - 1);
    st->radius = (float)((1 << (m - 1)) - 1);
}

int launch_adapt(const float* x, const CallParams& cp, DevState* st, cudaStream_t s) {
    uint64_t S = ((cp.d0 + 7) / 8) * ((cp.d1 + 7) / 8) * ((cp.d2 + 7) / 8);
    int blocks = (int)((S + 255) / 256);
    if (blocks > 1024) blocks = 1024;
    if (blocks < 1) blocks = 1;
    switch (cp.layers) {
        case 1: k_adapt<1><<<blocks, 256, 0, s>>>(x, cp, st); break;
        case 2: k_adapt<2><<<blocks, 256, 0, s>>>(x, cp, st); break;
        case 3: k_adapt<3><<<blocks, 256, 0, s>>>(x, cp, st); break;
        default: k_adapt<4><<<blocks, 256, 0, s>>>(x, cp, st); break;
    }
    return cudaGetLastError() == cudaSuccess ? 0 : SZGB_ECUDA;
}

// ---------------------------------------------------------------------------
// Prediction hitting rate (Sec. III): count the points whose n-layer
// prediction from the values V at the preceding neighbours lies within eb of
// x, |x - f(V)| <= eb (inclusive), the prediction formed in float32 exactly as
// above and the difference compared in float64.  V = x gives the rate on
// original values, V = the recorded (decompressed) values the rate the
// compressor sees.  Grid-stride over all points; per-warp sums, one atomic
// add per warp (an integer sum: the count does not depend on the schedule).

template <int NL>
__global__ void __launch_bounds__(256) k_hits(const float* __restrict__ x, const float* __restrict__ V,
                                              uint64_t d0, uint64_t d1, uint64_t d2, int ndim, double eb,
                                              unsigned long long* count) {
    const uint64_t plane = d1 * d2, N = d0 * plane;
    unsigned long long c = 0;
    for (uint64_t s = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; s < N;
         s += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t i = s / plane, r = s - i * plane, j = r / d2, l = r - j * d2;
        const float pred = predict_original<NL>(V, d1, d2, (int64_t)i, (int64_t)j, (int64_t)l, ndim);
        c += fabs((double)__ldg(x + s) - (double)pred) <= eb ? 1ull : 0ull;
    }
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, c);
}

// d0..d2: extents, slowest first, 1 for absent axes (a 2D field is 1 x d1 x d2)
int launch_hits(const float* x, const float* V, uint64_t d0, uint64_t d1, uint64_t d2, int ndim, int layers,
                double eb, unsigned long long* count, int sm_count, cudaStream_t s) {
    const uint64_t N = d0 * d1 * d2;
    uint64_t b = (N + 255) / 256;
    const uint64_t cap = 8ull * (uint64_t)(sm_count > 0 ? sm_count : 1);
    b = b < 1 ? 1 : (b > cap ? cap : b);
    const int blocks = (int)b;
    switch (layers) {
        case 1: k_hits<1><<<blocks, 256, 0, s>>>(x, V, d0, d1, d2, ndim, eb, count); break;
        case 2: k_hits<2><<<blocks, 256, 0, s>>>(x, V, d0, d1, d2, ndim, eb, count); break;
        case 3: k_hits<3><<<blocks, 256, 0, s>>>(x, V, d0, d1, d2, ndim, eb, count); break;
        default: k_hits<4><<<blocks, 256, 0, s>>>(x, V, d0, d1, d2, ndim, eb, count); break;
    }
    return cudaGetLastError() == cudaSuccess ? 0 : SZGB_ECUDA;
}

}  // namespace szgb
