// k_hyper.cu -- 3D fields with n = 3 or 4 layers, and 4D fields (Sec. III,
// Eq. predmodel): the prediction, quantization, fallback and record of
// Algorithm 1, and the matching reconstruction, on the tiled hyperplane
// schedule of hyper_tile.cuh (one launch per diagonal of tiles).
//
// A 3D wavefront lane would keep (n+1)^3 - 1 neighbour values in registers
// (63 at n = 3, 124 at n = 4), which does not fit beside the wavefront's
// helper warps.  Here a tile's CTA stages the tile with its halo of recorded
// values in shared memory and walks the tile's own hyperplanes there; a
// launch boundary orders the diagonals of tiles, and there is no device-side
// wait of any kind.  The arithmetic is the wavefront's: the same term order,
// products and sums rounded one at a time, the same quantizer and
// truncation.
#include "szgb_internal.cuh"
#include "hyper_box.h"
#include "hyper_kernels.cuh"
#include "hyper_tile.cuh"

namespace szgb {

template <int DIM, int NL, bool DEC>
__global__ void __launch_bounds__(TileGeom<DIM, NL>::THREADS)
    k_hyper_tile(const float* __restrict__ x, float* V, uint16_t* codes, uint64_t cpitch, Dims4 d, int64_t H,
                 HyperBox4 b, int64_t nL, const DevState* st) {
    using G = TileGeom<DIM, NL>;
    if (st->err) return;
    extern __shared__ __align__(16) unsigned char tile_smem[];
    float* Vs = reinterpret_cast<float*>(tile_smem);
    float* Xs = Vs + G::VPAD;
    uint16_t* Cs = reinterpret_cast<uint16_t*>(DEC ? Xs : Xs + G::XBOX);
    TileCtx t = {x, V, codes, cpitch, d, 0, 0, 0, 0};
    if (!tile_at<DIM, NL>(b, H, nL, blockIdx.x, &t)) return;  // the whole block
    const int tid = threadIdx.x;
    tile_load<DIM, NL, DEC>(t, Vs, Xs, Cs, tid);
    const QParams qp = load_qparams(st);
    __syncthreads();
    for (int s = 0; s < G::STEPS; s++) {
        tile_step<DIM, NL, DEC>(t, Vs, Xs, Cs, tid, s, qp);
        __syncthreads();
    }
    tile_store<DIM, NL, DEC>(t, Vs, Cs, tid);
}

// every diagonal of tiles of a D x P x M x N field (3D: D = 1), in order
template <int DIM, int NL, bool DEC>
static int run_tiles(const float* x, float* V, uint16_t* codes, uint64_t cpitch, const Dims4& d, const DevState* st,
                     cudaStream_t s) {
    using G = TileGeom<DIM, NL>;
    const size_t smem = G::smem_bytes(DEC);
    if (cudaFuncSetAttribute(k_hyper_tile<DIM, NL, DEC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return SZGB_ECUDA;
    const int64_t nA = (int64_t)((d.D + G::TA - 1) / G::TA), nI = (int64_t)((d.P + G::TI - 1) / G::TI),
                  nJ = (int64_t)((d.M + G::TJ - 1) / G::TJ), nL = (int64_t)((d.N + G::TL - 1) / G::TL);
    for (int64_t H = 0; H <= (nA - 1) + (nI - 1) + (nJ - 1) + (nL - 1); H++) {
        const HyperBox4 b = hyper_box4(H, nA, nI, nJ, nL);
        const uint64_t n = b.na * b.ni * b.nj;
        if (n == 0) continue;
        k_hyper_tile<DIM, NL, DEC><<<(unsigned)n, G::THREADS, smem, s>>>(x, V, codes, cpitch, d, H, b, nL, st);
        if (cudaGetLastError() != cudaSuccess) return SZGB_ECUDA;
    }
    return SZGB_OK;
}

// Compression of a P x M x N field with n = 3 or 4 layers: codes (row pitch
// cpitch) and the recorded values V (N points, raster order).  The state
// holds the bound and m (range and adaptive-m kernels run before).
int launch_hyper_compress(int layers, const float* x, float* V, uint16_t* codes, uint64_t cpitch, uint64_t P,
                          uint64_t M, uint64_t N, const DevState* st, cudaStream_t s) {
    const Dims4 d = {1, P, M, N};
    if (layers == 3) return run_tiles<3, 3, false>(x, V, codes, cpitch, d, st, s);
    if (layers == 4) return run_tiles<3, 4, false>(x, V, codes, cpitch, d, st, s);
    return SZGB_EUNSUPPORTED;
}

// Reconstruction: codes from the row decoder, unpredictable values already in
// out at their points; out is completed in place.
int launch_hyper_decompress(int layers, uint16_t* codes, uint64_t cpitch, float* out, uint64_t P, uint64_t M,
                            uint64_t N, const DevState* st, cudaStream_t s) {
    const Dims4 d = {1, P, M, N};
    if (layers == 3) return run_tiles<3, 3, true>(nullptr, out, codes, cpitch, d, st, s);
    if (layers == 4) return run_tiles<3, 4, true>(nullptr, out, codes, cpitch, d, st, s);
    return SZGB_EUNSUPPORTED;
}

int launch_hyper4(bool dec, int layers, const float* x, float* V, uint16_t* codes, uint64_t cpitch, uint64_t D,
                  uint64_t P, uint64_t M, uint64_t N, const DevState* st, cudaStream_t s) {
    const Dims4 d = {D, P, M, N};
    switch (layers * 2 + (dec ? 1 : 0)) {
        case 2: return run_tiles<4, 1, false>(x, V, codes, cpitch, d, st, s);
        case 3: return run_tiles<4, 1, true>(x, V, codes, cpitch, d, st, s);
        case 4: return run_tiles<4, 2, false>(x, V, codes, cpitch, d, st, s);
        case 5: return run_tiles<4, 2, true>(x, V, codes, cpitch, d, st, s);
        case 6: return run_tiles<4, 3, false>(x, V, codes, cpitch, d, st, s);
        case 7: return run_tiles<4, 3, true>(x, V, codes, cpitch, d, st, s);
        case 8: return run_tiles<4, 4, false>(x, V, codes, cpitch, d, st, s);
        case 9: return run_tiles<4, 4, true>(x, V, codes, cpitch, d, st, s);
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
    const uint64_t S = ((d.D + 7) / 8) * ((d.P + 7) / 8) * ((d.M + 7) / 8) * ((d.N + 7) / 8);
    const float ebf = st->eb_f, twoeb = st->twoeb, inv = st->inv2eb;
    for (uint64_t s = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; s < S;
         s += (uint64_t)gridDim.x * blockDim.x) {
        const int mm = adapt4_bucket<NL>(x, d, s, ebf, twoeb, inv);
        if (mm) atomicAdd(&cnt[mm], 1ull);
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

// Prediction hits of a 4D field, |x - f(V)| <= eb, added to *count: a
// grid-stride loop, per-warp sums, one atomic add per warp (an integer sum).
template <int NL>
__global__ void __launch_bounds__(256) k_hits4(const float* __restrict__ x, const float* __restrict__ V, Dims4 d,
                                               double eb, unsigned long long* count) {
    const uint64_t n = d.D * d.P * d.M * d.N;
    unsigned long long c = 0;
    for (uint64_t s = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; s < n; s += (uint64_t)gridDim.x * blockDim.x)
        c += hit4_point<NL>(x, V, d, s, eb) ? 1ull : 0ull;
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, c);
}

int launch_hits4(const float* x, const float* V, uint64_t D, uint64_t P, uint64_t M, uint64_t N, int layers,
                 double eb, unsigned long long* count, int sm_count, cudaStream_t s) {
    const Dims4 d = {D, P, M, N};
    const uint64_t n = D * P * M * N;
    uint64_t b = (n + 255) / 256;
    const uint64_t cap = 8ull * (uint64_t)(sm_count > 0 ? sm_count : 1);
    b = b < 1 ? 1 : (b > cap ? cap : b);
    switch (layers) {
        case 1: k_hits4<1><<<(unsigned)b, 256, 0, s>>>(x, V, d, eb, count); break;
        case 2: k_hits4<2><<<(unsigned)b, 256, 0, s>>>(x, V, d, eb, count); break;
        case 3: k_hits4<3><<<(unsigned)b, 256, 0, s>>>(x, V, d, eb, count); break;
        case 4: k_hits4<4><<<(unsigned)b, 256, 0, s>>>(x, V, d, eb, count); break;
        default: return SZGB_EINVAL;
    }
    return cudaGetLastError() == cudaSuccess ? SZGB_OK : SZGB_ECUDA;
}

}  // namespace szgb
