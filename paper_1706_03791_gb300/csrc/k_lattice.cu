// k_lattice.cu -- the lattice variant: a separately labelled, fully parallel
// form of the compressor (it is not the paper's method and never replaces
// it; its streams carry their own tag).
//
// Every value is snapped to the lattice of spacing 2 eb_f: p = rint(x * inv)
// with inv = 1 / (2 eb_f) rounded once, in binary32, |p| < 2^30.  The integer
// field p is predicted by the n-layer coefficients (Eq. predmodel) from the
// lattice values of the neighbours -- never from reconstructed values -- so
// every residual r = p - pred is independent and computed in parallel.  The
// residual takes the place of the quantization code (r + 2^(m-1) when
// |r| <= 2^(m-1)-1); a point is an outlier (code 0) when |r| is larger or its
// lattice value (float)p * 2 eb_f misses the bound, and its record stores a
// flag (lattice value within the bound), r in 64 bits and, if the flag is 0,
// the 32 bits of x.  Decompression inverts the predictor with n inclusive
// prefix sums along every axis (the residual is the n-th mixed difference of
// p), in wrap-around int32: the sums are exact modulo 2^32 and p fits.
#include <algorithm>

#include "szgb_internal.cuh"

namespace szgb {

// ---------------------------------------------------------------------------
// compression

// lattice integers and the within-bound flag of every point
__global__ void __launch_bounds__(256) k_lattice_p(const float* __restrict__ x, uint64_t n, int32_t* P, uint8_t* OK,
                                                   const DevState* st) {
    if (st->err) return;
    const float eb = st->eb_f, twoeb = __fmul_rn(2.0f, eb), inv = __fdiv_rn(1.0f, twoeb);
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        bool ok;
        P[i] = lattice_point(x[i], inv, twoeb, eb, ok);
        OK[i] = ok ? 1 : 0;
    }
}

// residual code of every point; optional reconstructed values (tests)
template <int ND, int NL>
__global__ void __launch_bounds__(256) k_lattice_codes(const int32_t* __restrict__ P, const uint8_t* __restrict__ OK,
                                                       const float* __restrict__ x, uint64_t d0, uint64_t d1,
                                                       uint64_t d2, uint16_t* codes, uint64_t cpitch,
                                                       float* recorded, const DevState* st) {
    if (st->err) return;
    const int center = st->center;
    const int64_t radius = center - 1;
    const float twoeb = __fmul_rn(2.0f, st->eb_f);
    const uint64_t rows = d0 * d1;
    // a block walks rows; its threads cover the row's columns (coalesced)
    for (uint64_t row = blockIdx.x; row < rows; row += gridDim.x) {
        const uint64_t i = row / d1, j = row - i * d1;
        for (uint64_t l = threadIdx.x; l < d2; l += blockDim.x) {
            const uint64_t q = row * d2 + l;
            const int64_t r = lattice_resid<ND, NL>(P, d1, d2, (int64_t)i, (int64_t)j, (int64_t)l);
            const bool ok = OK[q] != 0;
            const int64_t ar = r < 0 ? -r : r;
            codes[row * cpitch + l] = (ok && ar <= radius) ? (uint16_t)(r + center) : (uint16_t)0;
            if (recorded) recorded[q] = ok ? lattice_value(P[q], twoeb) : x[q];
        }
    }
}

// adaptive m on lattice residuals of the sample points (coordinates all
// multiples of 8), the last block choosing the smallest m whose radius holds
// ceil(theta * samples) of them
template <int ND, int NL>
__global__ void __launch_bounds__(256) k_adapt_lattice(const float* __restrict__ x, CallParams cp, DevState* st) {
    __shared__ unsigned long long cnt[18];
    __shared__ bool last;
    if (st->err) return;
    if (threadIdx.x < 18) cnt[threadIdx.x] = 0;
    __syncthreads();
    const float eb = st->eb_f, twoeb = __fmul_rn(2.0f, eb), inv = __fdiv_rn(1.0f, twoeb);
    const uint64_t S0 = (cp.d0 + 7) / 8, S1 = (cp.d1 + 7) / 8, S2 = (cp.d2 + 7) / 8, S = S0 * S1 * S2;
    for (uint64_t s = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; s < S; s += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t a = s / (S1 * S2), b = s % (S1 * S2);
        const int64_t i = (int64_t)(a * 8), j = (int64_t)((b / S2) * 8), l = (int64_t)((b % S2) * 8);
        int64_t pred = 0;
#pragma unroll
        for (int k0 = NL; k0 >= 0; k0--) {
            if (ND < 3 && k0 > 0) continue;
#pragma unroll
            for (int k1 = NL; k1 >= 0; k1--) {
                if (ND < 2 && k1 > 0) continue;
#pragma unroll
                for (int k2 = NL; k2 >= 0; k2--) {
                    if (k0 == 0 && k1 == 0 && k2 == 0) continue;
                    const int64_t ii = i - k0, jj = j - k1, ll = l - k2;
                    if (ii < 0 || jj < 0 || ll < 0) continue;
                    bool okn;
                    const int64_t pn = lattice_point(x[((uint64_t)ii * cp.d1 + (uint64_t)jj) * cp.d2 + (uint64_t)ll],
                                                     inv, twoeb, eb, okn);
                    pred += (int64_t)term_coef(NL, k0, k1, k2) * pn;
                }
            }
        }
        bool ok;
        const int64_t p = lattice_point(x[((uint64_t)i * cp.d1 + (uint64_t)j) * cp.d2 + (uint64_t)l], inv, twoeb, eb, ok);
        const int64_t r = p - pred, ar = r < 0 ? -r : r;
        if (!ok || ar > 32767) continue;
        int mm = 2;
        while (ar > ((int64_t)1 << (mm - 1)) - 1) mm++;
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
    const double req = ceil(cp.theta * (double)S);
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

static int grid_for(uint64_t n, int block) {
    uint64_t g = (n + block - 1) / block;
    if (g > 152ull * 16) g = 152ull * 16;
    return (int)(g < 1 ? 1 : g);
}

int launch_lattice_compress(const float* x, const CallParams& cp, int32_t* P, uint8_t* OK, uint16_t* codes,
                            uint64_t cpitch, float* recorded, DevState* st, cudaStream_t s) {
    const uint64_t n = cp.d0 * cp.d1 * cp.d2;
    if (cp.m_user == 0) {
        const uint64_t S = ((cp.d0 + 7) / 8) * ((cp.d1 + 7) / 8) * ((cp.d2 + 7) / 8);
        int blocks = (int)std::min<uint64_t>(std::max<uint64_t>((S + 255) / 256, 1), 1024);
        if (cp.ndim == 3) {
            if (cp.layers == 1) k_adapt_lattice<3, 1><<<blocks, 256, 0, s>>>(x, cp, st);
            else k_adapt_lattice<3, 2><<<blocks, 256, 0, s>>>(x, cp, st);
        } else if (cp.ndim == 2) {
            if (cp.layers == 1) k_adapt_lattice<2, 1><<<blocks, 256, 0, s>>>(x, cp, st);
            else k_adapt_lattice<2, 2><<<blocks, 256, 0, s>>>(x, cp, st);
        } else {
            if (cp.layers == 1) k_adapt_lattice<1, 1><<<blocks, 256, 0, s>>>(x, cp, st);
            else k_adapt_lattice<1, 2><<<blocks, 256, 0, s>>>(x, cp, st);
        }
    }
    k_lattice_p<<<grid_for(n, 256), 256, 0, s>>>(x, n, P, OK, st);
    const uint64_t rows = cp.d0 * cp.d1;
    const int g = (int)std::min<uint64_t>(rows, 152ull * 32);
#define SZGB_LC(ND, NL) k_lattice_codes<ND, NL><<<g, 256, 0, s>>>(P, OK, x, cp.d0, cp.d1, cp.d2, codes, cpitch, recorded, st)
    if (cp.ndim == 3) {
        if (cp.layers == 1) SZGB_LC(3, 1);
        else SZGB_LC(3, 2);
    } else if (cp.ndim == 2) {
        if (cp.layers == 1) SZGB_LC(2, 1);
        else SZGB_LC(2, 2);
    } else {
        if (cp.layers == 1) SZGB_LC(1, 1);
        else SZGB_LC(1, 2);
    }
#undef SZGB_LC
    return cudaGetLastError() == cudaSuccess ? 0 : SZGB_ECUDA;
}

// ---------------------------------------------------------------------------
// decompression

// row decode: one lane per row; residuals (wrap-around int32) to R, and for
// outliers whose lattice value misses the bound, the stored x to `out` with
// EX = 1
constexpr int kLatDecWarps = 8;

__global__ void __launch_bounds__(kLatDecWarps * 32) k_lattice_decode_rows(
    const uint8_t* __restrict__ payload, const uint64_t* __restrict__ rowoff, const uint32_t* __restrict__ rowbytes,
    const uint8_t* stream_end, const uint32_t* __restrict__ lut, const uint32_t* __restrict__ dectab, int32_t* R,
    uint8_t* EX, float* out, uint64_t rows, uint64_t N, DevState* st) {
    __shared__ uint32_t s_lut[1 << kLutBits];
    __shared__ uint32_t s_tab[260];
    __shared__ int32_t s_tile[kLatDecWarps][32][33];  // odd word stride: conflict-free
    __shared__ int s_err;
    if (threadIdx.x == 0) s_err = *(volatile const unsigned*)&st->err != 0;
    __syncthreads();
    if (s_err) return;
    const int T = (int)st->lut_bits, maxlen = (int)st->maxlen, center = st->center;
    for (int i = threadIdx.x; i < (1 << T); i += blockDim.x) s_lut[i] = lut[i];
    for (int i = threadIdx.x; i < 260; i += blockDim.x) s_tab[i] = dectab[i];
    __syncthreads();
    const uint16_t* g_sorted = reinterpret_cast<const uint16_t*>(dectab + 260);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint64_t row0 = ((uint64_t)blockIdx.x * kLatDecWarps + warp) * 32, row = row0 + lane;
    const bool valid = row < rows;
    BitReader br;
    bool bad = false;
    if (valid) br.init(payload, rowoff[row], (uint64_t)(stream_end - payload));
    int32_t(*tile)[33] = s_tile[warp];
    for (uint64_t l0 = 0; l0 < N; l0 += 32) {
        const int ncol = (int)min((uint64_t)32, N - l0);
        for (int j = 0; j < ncol; j++) {
            int32_t rv = 0;
            if (valid) {
                const int code = decode_symbol(br, s_lut, T, s_tab, g_sorted, maxlen, bad);
                if (code) {
                    rv = code - center;
                } else {
                    const uint32_t ok = br.take(1);
                    br.take(32);  // the high word: r is needed modulo 2^32 only
                    rv = (int32_t)br.take(32);
                    if (!ok) {
                        out[row * N + l0 + j] = __uint_as_float(br.take(32));
                        EX[row * N + l0 + j] = 1;
                    }
                }
            }
            tile[lane][j] = rv;
        }
        __syncwarp();
        for (int t = 0; t < 32; t++) {
            const uint64_t r = row0 + t;
            if (r < rows && lane < ncol) R[r * N + l0 + lane] = tile[t][lane];
        }
        __syncwarp();
    }
    if (valid && (bad || br.consumed() > (uint64_t)rowbytes[row] * 8)) atomicOr(&st->err, kErrCorrupt);
}

// inclusive prefix sums (wrap-around int32) along one axis of [d0][d1][d2]
__global__ void __launch_bounds__(256) k_scan_axis2(int32_t* R, uint64_t rows, uint64_t N) {
    // one warp per row, 32 columns at a time
    const int lane = threadIdx.x & 31;
    const uint64_t w = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t r = w; r < rows; r += nw) {
        int32_t* p = R + r * N;
        uint32_t carry = 0;
        for (uint64_t l0 = 0; l0 < N; l0 += 32) {
            const uint64_t l = l0 + lane;
            uint32_t v = l < N ? (uint32_t)p[l] : 0u;
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, v, o);
                if (lane >= o) v += y;
            }
            v += carry;
            if (l < N) p[l] = (int32_t)v;
            carry = __shfl_sync(0xffffffffu, v, 31);
        }
    }
}

// along the middle (stride N, length d1) or first (stride d1*N, length d0)
// axis: one thread per line, eight loads in flight
__global__ void __launch_bounds__(256) k_scan_strided(int32_t* R, uint64_t nlines, uint64_t inner, uint64_t len,
                                                      uint64_t stride, uint64_t outer_stride) {
    const uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (t >= nlines) return;
    // line t: base = (t / inner) * outer_stride + (t % inner)
    int32_t* p = R + (t / inner) * outer_stride + (t % inner);
    uint32_t acc = 0;
    uint64_t k = 0;
    for (; k + 8 <= len; k += 8) {
        uint32_t v[8];
#pragma unroll
        for (int u = 0; u < 8; u++) v[u] = (uint32_t)p[(k + u) * stride];
#pragma unroll
        for (int u = 0; u < 8; u++) {
            acc += v[u];
            p[(k + u) * stride] = (int32_t)acc;
        }
    }
    for (; k < len; k++) {
        acc += (uint32_t)p[k * stride];
        p[k * stride] = (int32_t)acc;
    }
}

__global__ void __launch_bounds__(256) k_lattice_finish(const int32_t* __restrict__ R, const uint8_t* __restrict__ EX,
                                                        float* out, uint64_t n, const DevState* st) {
    if (st->err) return;
    const float twoeb = __fmul_rn(2.0f, st->eb_f);
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        if (!EX[i]) out[i] = lattice_value(R[i], twoeb);
}

int launch_lattice_decompress(const uint8_t* payload, const uint64_t* rowoff, const uint32_t* rowbytes,
                              const uint8_t* stream_end, const uint32_t* lut, const uint32_t* dec_tab, int ndim,
                              int layers, uint64_t d0, uint64_t d1, uint64_t d2, int32_t* R, uint8_t* EX, float* out,
                              DevState* st, cudaStream_t s) {
    const uint64_t rows = d0 * d1, n = rows * d2;
    if (cudaMemsetAsync(EX, 0, n, s) != cudaSuccess) return SZGB_ECUDA;
    const uint64_t per = 32ull * kLatDecWarps;
    k_lattice_decode_rows<<<(unsigned)((rows + per - 1) / per), kLatDecWarps * 32, 0, s>>>(
        payload, rowoff, rowbytes, stream_end, lut, dec_tab, R, EX, out, rows, d2, st);
    for (int rep = 0; rep < layers; rep++) {
        k_scan_axis2<<<grid_for(rows * 32, 256), 256, 0, s>>>(R, rows, d2);
        if (ndim >= 2 && d1 > 1) {
            const uint64_t nl = d0 * d2;  // lines along axis 1: one per (plane, column)
            k_scan_strided<<<(unsigned)((nl + 255) / 256), 256, 0, s>>>(R, nl, d2, d1, d2, d1 * d2);
        }
        if (ndim == 3 && d0 > 1) {
            const uint64_t nl = d1 * d2;  // lines along axis 0: one per (row, column)
            k_scan_strided<<<(unsigned)((nl + 255) / 256), 256, 0, s>>>(R, nl, nl, d0, d1 * d2, 0);
        }
    }
    k_lattice_finish<<<grid_for(n, 256), 256, 0, s>>>(R, EX, out, n, st);
    return cudaGetLastError() == cudaSuccess ? 0 : SZGB_ECUDA;
}

}  // namespace szgb
