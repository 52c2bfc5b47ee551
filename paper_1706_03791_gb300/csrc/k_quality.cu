// k_quality.cu -- reconstruction quality of a field (Sec. II, Metrics 1-3):
// the sums behind the maximum error, RMSE, NRMSE, PSNR and Pearson's
// coefficient, in float64, one pass over the original and its
// reconstruction.
//
// The value x_0 is subtracted from both inputs before the moments are summed,
// so that the covariance and the variances (differences of large sums for a
// field far from zero) keep their digits.  Per-thread partial sums, a warp and
// block reduction, per-block partials in a fixed order, and the last block to
// finish adds them in block order: the result does not depend on scheduling.
#include "szgb_internal.cuh"

namespace szgb {

constexpr int kQualThreads = 256;

struct QualSums {
    double se, sx, sy, sxx, syy, sxy, maxe, xmin, xmax;
};

__device__ __forceinline__ void qual_add(QualSums& a, float xf, float yf, double s) {
    const double x = (double)xf, y = (double)yf;
    const double e = x - y;
    a.se += e * e;
    a.maxe = fmax(a.maxe, fabs(e));
    const double xs = x - s, ys = y - s;
    a.sx += xs;
    a.sy += ys;
    a.sxx += xs * xs;
    a.syy += ys * ys;
    a.sxy += xs * ys;
    a.xmin = fmin(a.xmin, x);
    a.xmax = fmax(a.xmax, x);
}

__device__ __forceinline__ void qual_merge(QualSums& a, const QualSums& b) {
    a.se += b.se;
    a.sx += b.sx;
    a.sy += b.sy;
    a.sxx += b.sxx;
    a.syy += b.syy;
    a.sxy += b.sxy;
    a.maxe = fmax(a.maxe, b.maxe);
    a.xmin = fmin(a.xmin, b.xmin);
    a.xmax = fmax(a.xmax, b.xmax);
}

__device__ __forceinline__ QualSums qual_shfl(const QualSums& a, int o) {
    QualSums b;
    b.se = __shfl_xor_sync(0xffffffffu, a.se, o);
    b.sx = __shfl_xor_sync(0xffffffffu, a.sx, o);
    b.sy = __shfl_xor_sync(0xffffffffu, a.sy, o);
    b.sxx = __shfl_xor_sync(0xffffffffu, a.sxx, o);
    b.syy = __shfl_xor_sync(0xffffffffu, a.syy, o);
    b.sxy = __shfl_xor_sync(0xffffffffu, a.sxy, o);
    b.maxe = __shfl_xor_sync(0xffffffffu, a.maxe, o);
    b.xmin = __shfl_xor_sync(0xffffffffu, a.xmin, o);
    b.xmax = __shfl_xor_sync(0xffffffffu, a.xmax, o);
    return b;
}

// partials: gridDim.x records; done: a counter that starts at 0 (the last
// block resets it); out: the summed record
__global__ void __launch_bounds__(kQualThreads) k_quality(const float* __restrict__ x, const float* __restrict__ y,
                                                          uint64_t n, QualSums* partials, unsigned* done,
                                                          QualSums* out) {
    const double s = (double)x[0];
    QualSums a = {0, 0, 0, 0, 0, 0, 0, INFINITY, -INFINITY};
    const uint64_t tid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    const uint64_t nthr = (uint64_t)gridDim.x * blockDim.x;
    const bool vec = ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(y)) & 15) == 0;
    uint64_t done_n = 0;
    if (vec) {
        const float4* x4 = reinterpret_cast<const float4*>(x);
        const float4* y4 = reinterpret_cast<const float4*>(y);
        const uint64_t n4 = n / 4;
        for (uint64_t i = tid; i < n4; i += nthr) {
            const float4 u = __ldcs(x4 + i), v = __ldcs(y4 + i);
            qual_add(a, u.x, v.x, s);
            qual_add(a, u.y, v.y, s);
            qual_add(a, u.z, v.z, s);
            qual_add(a, u.w, v.w, s);
        }
        done_n = n4 * 4;
    }
    for (uint64_t i = done_n + tid; i < n; i += nthr) qual_add(a, x[i], y[i], s);
    for (int o = 16; o > 0; o >>= 1) qual_merge(a, qual_shfl(a, o));
    __shared__ QualSums sw[kQualThreads / 32];
    __shared__ bool last;
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sw[w] = a;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = 1; i < kQualThreads / 32; i++) qual_merge(a, sw[i]);
        partials[blockIdx.x] = a;
        __threadfence();
        last = atomicAdd(done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last || threadIdx.x != 0) return;
    __threadfence();
    const volatile QualSums* vp = partials;
    QualSums r = {0, 0, 0, 0, 0, 0, 0, INFINITY, -INFINITY};
    for (unsigned b = 0; b < gridDim.x; b++) {
        QualSums p;
        p.se = vp[b].se;
        p.sx = vp[b].sx;
        p.sy = vp[b].sy;
        p.sxx = vp[b].sxx;
        p.syy = vp[b].syy;
        p.sxy = vp[b].sxy;
        p.maxe = vp[b].maxe;
        p.xmin = vp[b].xmin;
        p.xmax = vp[b].xmax;
        qual_merge(r, p);
    }
    *out = r;
    *done = 0;
}

size_t quality_scratch_bytes(int blocks) { return ((size_t)blocks + 1) * sizeof(QualSums) + 64; }

int quality_blocks(uint64_t n, int sm_count) {
    uint64_t b = (n + 4ull * kQualThreads * 8 - 1) / (4ull * kQualThreads * 8);
    b = b < 1 ? 1 : b;
    return (int)(b > 4ull * (uint64_t)sm_count ? 4ull * (uint64_t)sm_count : b);
}

// scratch: quality_scratch_bytes(blocks), 16-byte aligned; the counter word
// at its end must be 0 (it is left at 0); host_out: 9 doubles (pinned):
// se, sx, sy, sxx, syy, sxy, max error, x_min, x_max
int launch_quality(const float* x, const float* y, uint64_t n, int blocks, void* scratch, double* host_out,
                   cudaStream_t s) {
    QualSums* partials = static_cast<QualSums*>(scratch);
    QualSums* out = partials + blocks;
    unsigned* done = reinterpret_cast<unsigned*>(out + 1);
    k_quality<<<blocks, kQualThreads, 0, s>>>(x, y, n, partials, done, out);
    if (cudaGetLastError() != cudaSuccess) return SZGB_ECUDA;
    if (cudaMemcpyAsync(host_out, out, sizeof(QualSums), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return SZGB_ECUDA;
    return SZGB_OK;
}

}  // namespace szgb
