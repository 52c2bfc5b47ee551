// k_decode.cu -- the Huffman decode of every chunk of a stream (Sec. IV-A
// coding, undone), before the reconstruction wavefront: the codes go to a
// row-pitched array the wavefront reads, the values of unpredictable points
// straight to the output.
#include <cstring>
#include <mutex>

#include "szgb_internal.cuh"

namespace szgb {

// ---------------------------------------------------------------------------
// Huffman decode of every chunk (`chunk` points of a row, or the whole row),
// before the reconstruction wavefront: one lane per chunk, the 32 lanes of a
// warp on the same chunk of 32 consecutive rows.  A step looks up the next
// kMultiBits bits in the multi-symbol table and takes up to three codes at
// once (one code, by the single-symbol table or the canonical search, when
// the first code is longer, or near the end of the ring or of the chunk).
// Lanes advance at their own pace through a two-tile ring of 64 columns of
// their row; a 32-column tile is stored (coalesced, two codes a lane) once
// every lane of the warp has passed it.  The value of an unpredictable point
// (code 0: sign, exponent and top t mantissa bits) goes straight to its place
// in the output array.

struct DecodeArgs {
    const uint8_t* payload;
    const uint64_t* rowoff;
    const uint32_t* rowbytes;
    const uint8_t* stream_end;
    const uint32_t* lut;
    const uint32_t* dectab;
    uint16_t* codes;
    uint64_t cpitch;
    float* out;
    uint64_t rows, N;
    uint32_t chunk;  // chunk length along a row (a power of two >= 32), 0: whole rows
    uint32_t nseg;   // chunks per row
    DevState* st;
};

constexpr int kDecWarps = 8;
constexpr int kDecRing = 64;                  // ring columns per lane
constexpr int kDecRingStride = kDecRing + 2;  // u16 per ring row: an odd word stride
constexpr size_t kDecSmem = (size_t)(1u << kMultiBits) * 4 + (size_t)(1u << kLutBits) * 4 + 260 * 4 +
                            (size_t)kDecWarps * 32 * kDecRingStride * 2;

// chunk (blk % nseg) of rows [(blk / nseg) * 32 kDecWarps, ...) of one
// field; every thread of the block calls it
__device__ __forceinline__ void decode_rows_block(const DecodeArgs& D, uint64_t blk, uint32_t* dsm) {
    uint32_t* s_multi = dsm;
    uint32_t* s_lut = s_multi + (1u << kMultiBits);
    uint32_t* s_tab = s_lut + (1u << kLutBits);
    uint16_t* s_ring = reinterpret_cast<uint16_t*>(s_tab + 260);
    __shared__ int s_err;
    if (threadIdx.x == 0) s_err = *(volatile const unsigned*)&D.st->err != 0;
    __syncthreads();
    if (s_err) return;
    const int maxlen = (int)D.st->maxlen, e_eb = D.st->e_eb;
    const int lut_bits = (int)D.st->lut_bits;  // index bits of the single-code table (<= kLutBits)
    for (int i = threadIdx.x; i < (1 << kMultiBits); i += blockDim.x) s_multi[i] = D.dectab[kMultiOff + i];
    for (int i = threadIdx.x; i < (1 << lut_bits); i += blockDim.x) s_lut[i] = D.lut[i];
    for (int i = threadIdx.x; i < 260; i += blockDim.x) s_tab[i] = D.dectab[i];
    __syncthreads();
    const uint16_t* g_sorted = reinterpret_cast<const uint16_t*>(D.dectab + 260);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint64_t seg = blk % D.nseg;
    const uint64_t row0 = ((blk / D.nseg) * kDecWarps + warp) * 32;
    const uint64_t row = row0 + lane;
    const bool valid = row < D.rows;
    // this chunk's columns [cbeg, cend) (cbeg a multiple of 32)
    const uint64_t cbeg = D.chunk ? seg * D.chunk : 0;
    const uint64_t cend = D.chunk ? min(D.N, cbeg + D.chunk) : D.N;
    BitReader br;
    bool bad = false;
    uint64_t avail = 0;
    if (valid) {
        const uint64_t ch = row * D.nseg + seg;
        br.init(D.payload, D.rowoff[ch], (uint64_t)(D.stream_end - D.payload));
        avail = (uint64_t)D.rowbytes[ch] * 8;
    }
    uint16_t* const ring = s_ring + (size_t)warp * 32 * kDecRingStride;
    uint16_t* const myring = ring + lane * kDecRingStride;
    float* const orow = D.out + row * D.N;
    const uint64_t N = cend;  // the chunk ends the lane's work
    uint64_t col = valid ? cbeg : N;  // next column of this lane's chunk
    for (uint64_t tb = cbeg; tb < N; tb += 32) {
        const uint64_t tend = min(N, tb + 32), lim = min(N, tb + kDecRing);
        while (__any_sync(0xffffffffu, col < tend)) {
            if (col < lim) {
                bool esc = false;
                br.refill();
                const uint32_t e = s_multi[(uint32_t)(br.win >> (64 - kMultiBits))];
                const uint32_t n = e & 3u;
                if (n != 0 && col + n > lim && lim < N) {
                    // ahead of the warp by almost two tiles: wait for the next store
                } else if (n != 0 && col + n <= lim) {
                    const uint32_t used = (e >> 2) & 15u;
                    br.win <<= used;
                    br.nb -= (int)used;
                    uint32_t last;
                    if (n == 1) {
                        last = e >> 8;
                        myring[col & (kDecRing - 1)] = (uint16_t)last;
                    } else {
                        myring[col & (kDecRing - 1)] = (uint16_t)((e >> 8) & 0xffu);
                        myring[(col + 1) & (kDecRing - 1)] = (uint16_t)((e >> 16) & 0xffu);
                        last = (e >> 16) & 0xffu;
                        if (n == 3) {
                            last = e >> 24;
                            myring[(col + 2) & (kDecRing - 1)] = (uint16_t)last;
                        }
                    }
                    col += n;
                    esc = last == 0;
                } else {
                    // one code: the first code is longer than the multi-code
                    // table's window, or a multi-code step would pass the
                    // chunk end (the single-code table, else the canonical
                    // search)
                    const int code = decode_symbol(br, s_lut, lut_bits, s_tab, g_sorted, maxlen, bad);
                    myring[col & (kDecRing - 1)] = (uint16_t)code;
                    col += 1;
                    esc = code == 0;
                }
                if (esc) {
                    // the value of an unpredictable point: sign, exponent, top t bits
                    const uint32_t se = br.take(9);
                    const int t = trunc_bits(se << 23, e_eb);
                    const uint32_t mb = br.take(t);
                    orow[col - 1] = __uint_as_float((se << 23) | (t ? (mb << (23 - t)) : 0u));
                }
            }
        }
        __syncwarp();
        {
            // tile [tb, tend): two codes a lane, two rows per warp instruction;
            // a pair that ends past the row's last column lands in the row
            // pitch's padding
            const int q = lane & 15;
            const int c0 = (int)(tb & (kDecRing - 1)) + 2 * q;
            if (tb + 2 * q < tend) {
#pragma unroll 4
                for (int t = lane >> 4; t < 32; t += 2) {
                    const uint64_t r = row0 + t;
                    if (r < D.rows) {
                        const uint32_t v = *reinterpret_cast<const uint32_t*>(ring + t * kDecRingStride + c0);
                        *reinterpret_cast<uint32_t*>(D.codes + r * D.cpitch + tb + 2 * q) = v;
                    }
                }
            }
        }
        __syncwarp();
    }
    if (valid && (bad || br.consumed() > avail)) atomicOr(&D.st->err, kErrCorrupt);
}

__global__ void __launch_bounds__(kDecWarps * 32, 4) k_decode_rows(const __grid_constant__ DecodeArgs D) {
    extern __shared__ __align__(16) uint32_t dsm[];
    decode_rows_block(D, blockIdx.x, dsm);
}

// every field of a batch in one launch: field f owns blocks [blk[f], blk[f+1])
__global__ void __launch_bounds__(kDecWarps * 32, 4)
    k_decode_rows_batch(const DecodeArgs* __restrict__ F, const uint32_t* __restrict__ blk, int count) {
    extern __shared__ __align__(16) uint32_t dsm[];
    int lo = 0, hi = count - 1;  // the last field whose first block is <= blockIdx.x
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (blk[mid] <= blockIdx.x) lo = mid;
        else hi = mid - 1;
    }
    const DecodeArgs D = F[lo];
    decode_rows_block(D, blockIdx.x - blk[lo], dsm);
}

size_t decode_args_bytes() { return sizeof(DecodeArgs); }

uint32_t decode_rows_blocks(uint64_t rows, uint32_t chunk, uint64_t N) {
    return (uint32_t)((rows + 32ull * kDecWarps - 1) / (32ull * kDecWarps) * chunks_per_row(chunk, N));
}

void decode_args_fill(void* dst, const uint8_t* payload, const uint64_t* rowoff, const uint32_t* rowbytes,
                      const uint8_t* stream_end, const uint32_t* lut, const uint32_t* dec_tab, uint16_t* codes,
                      uint64_t cpitch, float* out, uint64_t rows, uint64_t N, uint32_t chunk, DevState* st) {
    DecodeArgs d;
    d.payload = payload;
    d.rowoff = rowoff;
    d.rowbytes = rowbytes;
    d.stream_end = stream_end;
    d.lut = lut;
    d.dectab = dec_tab;
    d.codes = codes;
    d.cpitch = cpitch;
    d.out = out;
    d.rows = rows;
    d.N = N;
    d.chunk = chunk;
    d.nseg = (uint32_t)chunks_per_row(chunk, N);
    d.st = st;
    memcpy(dst, &d, sizeof(d));
}

int launch_decode_rows_batch(const void* args_dev, const uint32_t* blk_dev, int count, uint32_t total_blocks,
                             cudaStream_t s) {
    if (count < 1 || total_blocks == 0) return SZGB_OK;
    static std::once_flag once;
    static bool ok = true;
    std::call_once(once, [] {
        ok = cudaFuncSetAttribute(k_decode_rows_batch, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)kDecSmem) == cudaSuccess;
        if (!ok) cudaGetLastError();
    });
    if (!ok) return SZGB_ECUDA;
    k_decode_rows_batch<<<total_blocks, kDecWarps * 32, kDecSmem, s>>>(static_cast<const DecodeArgs*>(args_dev),
                                                                       blk_dev, count);
    return cudaGetLastError() == cudaSuccess ? 0 : SZGB_ECUDA;
}

int launch_decode_rows(const uint8_t* payload, const uint64_t* rowoff, const uint32_t* rowbytes,
                       const uint8_t* stream_end, const uint32_t* lut, const uint32_t* dec_tab, uint16_t* codes,
                       uint64_t cpitch, float* out, uint64_t rows, uint64_t N, uint32_t chunk, DevState* st,
                       cudaStream_t s) {
    DecodeArgs d;
    d.payload = payload;
    d.rowoff = rowoff;
    d.rowbytes = rowbytes;
    d.stream_end = stream_end;
    d.lut = lut;
    d.dectab = dec_tab;
    d.codes = codes;
    d.cpitch = cpitch;
    d.out = out;
    d.rows = rows;
    d.N = N;
    d.chunk = chunk;
    d.nseg = (uint32_t)chunks_per_row(chunk, N);
    d.st = st;
    const uint64_t per = 32ull * kDecWarps;
    const uint64_t blocks = (rows + per - 1) / per * d.nseg;
    if (blocks == 0 || blocks > 0x7fffffffull) return SZGB_EINVAL;
    static std::once_flag once;
    static bool ok = true;
    std::call_once(once, [] {
        ok = cudaFuncSetAttribute(k_decode_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDecSmem) ==
             cudaSuccess;
        if (!ok) cudaGetLastError();
    });
    if (!ok) return SZGB_ECUDA;
    k_decode_rows<<<(unsigned)blocks, kDecWarps * 32, kDecSmem, s>>>(d);
    return cudaGetLastError() == cudaSuccess ? 0 : SZGB_ECUDA;
}

}  // namespace szgb
