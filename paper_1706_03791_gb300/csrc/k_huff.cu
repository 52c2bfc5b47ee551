// k_huff.cu -- variable-length (Huffman) coding of the quantization codes
// (Sec. IV-A: any number of symbols, 2^m for m up to 16) and the stream
// layout: histogram, codebook build, per-row bit lengths, row offsets, the
// payload writer, and the decoder tables.
//
// Codebook: the used symbols sorted by (frequency, symbol) are merged with
// two FIFO queues (leaves, internal nodes; a leaf is taken first on equal
// weights); a symbol's code length is its leaf depth (one used symbol gets
// length 1).  Codes are canonical: ordered by (length, symbol), consecutive
// within a length.
#include <cstring>
#include <mutex>

#include "szgb_internal.cuh"

namespace szgb {

// ---------------------------------------------------------------------------
// histogram of the codes over 2^m bins
//
// The codes are read as 16-byte vectors (8 codes; rows have a pitch of a
// multiple of 8 entries and the padding is skipped).  The distribution is
// concentrated around the centre code, so the kHistWin bins around it are
// counted in per-lane private counters laid out bin-major with the lane
// innermost (one bank per lane: no atomics, no conflicts); the other bins take
// shared-memory atomics on a block histogram (2^m <= 8192) or global ones.

constexpr int kHistThreads = 512;
constexpr int kHistWin = 32;
constexpr int kHistBlockBins = 8192;
constexpr size_t kHistSmem = (size_t)(kHistBlockBins + (kHistThreads / 32) * kHistWin * 32) * 4;

__global__ void __launch_bounds__(kHistThreads) k_hist(const uint16_t* __restrict__ codes, uint64_t rows,
                                                       uint64_t rowlen, uint64_t pitch, uint32_t* hist,
                                                       const DevState* st) {
    extern __shared__ uint32_t sh[];
    if (st->err) return;
    const int m = st->m;
    const int nb = 1 << m;
    const bool use_smem = nb <= kHistBlockBins;
    uint32_t* priv = sh + kHistBlockBins;
    if (use_smem)
        for (int i = threadIdx.x; i < nb; i += kHistThreads) sh[i] = 0;
    for (int i = threadIdx.x; i < (kHistThreads / 32) * kHistWin * 32; i += kHistThreads) priv[i] = 0;
    __syncthreads();
    uint32_t* H = use_smem ? sh : hist;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    uint32_t* P = priv + wib * kHistWin * 32 + lane;
    int lo = st->center - kHistWin / 2;
    lo = lo < 0 ? 0 : lo;
    const uint64_t vpr = pitch >> 3;  // vectors per row
    const uint64_t nvec = rows * vpr;
    const uint64_t stride = (uint64_t)gridDim.x * kHistThreads;
    // the (row, vector) of the thread's vector, advanced by the grid stride
    // with a carry instead of a division per vector
    const uint64_t v_first = blockIdx.x * (uint64_t)kHistThreads + threadIdx.x;
    const uint64_t sr = stride / vpr, sc = stride - sr * vpr;
    uint64_t vr = v_first / vpr, vc = v_first - vr * vpr;
    auto advance = [&](uint64_t& r, uint64_t& c) {
        r += sr;
        c += sc;
        if (c >= vpr) {
            c -= vpr;
            r++;
        }
    };
    // two vectors in flight per thread
    for (uint64_t v0 = v_first; v0 < nvec; v0 += 2 * stride) {
        uint4 q[2];
        int nv[2];
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const uint64_t v = v0 + h * stride;
            nv[h] = 0;
            q[h] = make_uint4(0u, 0u, 0u, 0u);
            if (v < nvec) {
                const uint64_t c0 = vc << 3;
                q[h] = __ldcs(reinterpret_cast<const uint4*>(codes + vr * pitch + c0));
                const uint64_t rem = rowlen - c0;
                nv[h] = rem < 8 ? (int)rem : 8;
            }
            advance(vr, vc);
        }
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const uint32_t w[4] = {q[h].x, q[h].y, q[h].z, q[h].w};
#pragma unroll
            for (int k = 0; k < 8; k++) {
                if (k < nv[h]) {
                    uint32_t c = (w[k >> 1] >> (16 * (k & 1))) & 0xffffu;
                    if (c >= (uint32_t)nb) c = 0;  // codes are < 2^m; never index past the bins
                    const uint32_t d = c - (uint32_t)lo;
                    if (d < (uint32_t)kHistWin) {
                        P[d * 32] += 1u;
                    } else {
                        atomicAdd(&H[c], 1u);
                    }
                }
            }
        }
    }
    __syncthreads();
    // window totals: warp wib sums bins wib, wib + 16, ... over all warps' lanes
    for (int b = wib; b < kHistWin; b += kHistThreads / 32) {
        uint32_t t = 0;
        for (int w2 = 0; w2 < kHistThreads / 32; w2++) t += priv[(w2 * kHistWin + b) * 32 + lane];
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0 && t && lo + b < nb) atomicAdd(&H[lo + b], t);
    }
    if (use_smem) {
        __syncthreads();
        for (int i = threadIdx.x; i < nb; i += kHistThreads)
            if (sh[i]) atomicAdd(&hist[i], sh[i]);
    }
}

int launch_histogram(const uint16_t* codes, uint64_t rows, uint64_t rowlen, uint64_t pitch, uint32_t* hist,
                     DevState* st, cudaStream_t s) {
    static std::once_flag once;
    static bool ok = true;
    std::call_once(once, [] {
        ok = cudaFuncSetAttribute(k_hist, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kHistSmem) ==
             cudaSuccess;
        if (!ok) cudaGetLastError();
    });
    if (!ok) return SZGB_ECUDA;
    const uint64_t nvec = rows * (pitch >> 3);
    uint64_t blocks = (nvec + kHistThreads * 4 - 1) / (kHistThreads * 4);
    if (blocks > 2 * 152) blocks = 2 * 152;
    if (blocks < 1) blocks = 1;
    k_hist<<<(int)blocks, kHistThreads, kHistSmem, s>>>(codes, rows, rowlen, pitch, hist, st);
    return cudaGetLastError() == cudaSuccess ? 0 : SZGB_ECUDA;
}

// ---------------------------------------------------------------------------
// codebook build: one CTA of 1024 threads.
//   sortbuf: >= 2^16 u64 keys (freq << 16 | symbol)
//   nodebuf: >= 4 * 2^16 u32 (parent links, depths)

constexpr int kCbThreads = 1024;
constexpr int kSmemSortCap = 8192;

__device__ void bitonic_sort(uint64_t* a, int n_pow2) {
    for (int k = 2; k <= n_pow2; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < n_pow2; i += blockDim.x) {
                int ixj = i ^ j;
                if (ixj > i) {
                    uint64_t x = a[i], y = a[ixj];
                    bool up = (i & k) == 0;
                    if ((x > y) == up) { a[i] = y; a[ixj] = x; }
                }
            }
            __syncthreads();
        }
    }
}

// canonical code assignment over symbols listed in ascending order: the code
// of a symbol of length L is first[L] + (number of earlier symbols of length
// L).  Done by warp 0, 32 symbols at a time.  cw_out[s] holds the encoder's
// table entry: the length in the top byte, the code below it (lengths are at
// most 46, so a code fits in 56 bits).
__device__ void canonical_assign(const uint32_t* syms, int n, const uint8_t* len, uint64_t* first_io,
                                 uint64_t* cw_out, uint32_t* rank_out) {
    if (threadIdx.x >= 32) return;
    const int lane = threadIdx.x;
    for (int base = 0; base < n; base += 32) {
        int i = base + lane;
        bool v = i < n;
        unsigned act = __ballot_sync(0xffffffffu, v);
        if (v) {
            uint32_t s = syms[i];
            int L = len[s];
            unsigned peers = __match_any_sync(act, L);
            int rank = __popc(peers & ((1u << lane) - 1u));
            uint64_t f = first_io[L];
            if (cw_out) cw_out[s] = ((uint64_t)L << 56) | (f + (uint64_t)rank);
            if (rank_out) rank_out[i] = (uint32_t)(f + rank);
            __syncwarp(act);
            if (rank == 0) first_io[L] = f + (uint64_t)__popc(peers);
        }
        __syncwarp();
    }
}

// block-wide exclusive scan of one value per thread (kCbThreads = 1024)
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t* s_tmp, uint32_t* total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_tmp[wid] = x;
    __syncthreads();
    if (wid == 0) {
        uint32_t t = s_tmp[lane];
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        s_tmp[lane] = t;
    }
    __syncthreads();
    const uint32_t ex = (wid ? s_tmp[wid - 1] : 0u) + x - v;
    *total = s_tmp[31];
    __syncthreads();
    return ex;
}

constexpr int kCbRing = 32768;                   // internal-node weight ring (>= n/2)
constexpr size_t kCbSmem = 65536 + 4 * kCbRing;  // region A (64 KB) + ring (128 KB)

// Codebook (R6).  Leaves sorted by (frequency, symbol): bitonic sort in shared
// memory up to 8192 used symbols, else a stable LSD radix sort by frequency of
// the symbol-ordered list.  The two-queue merge (one thread, the internal
// nodes in a shared-memory ring: the queue never holds more than n/2 nodes)
// gives every node its parent; depths follow top-down; canonical codes by
// (length, symbol).
// the codebook of one field; every thread of the CTA calls it
__device__ __forceinline__ void codebook_block(const uint32_t* __restrict__ hist, DevState* st, uint8_t* len,
                                               uint64_t* cw, uint64_t* sortbuf, uint32_t* nodebuf) {
    extern __shared__ __align__(16) unsigned char cb_smem[];
    uint64_t* s_keys = reinterpret_cast<uint64_t*>(cb_smem);          // region A: 8192 keys
    uint32_t* s_a32 = reinterpret_cast<uint32_t*>(cb_smem);           // region A: 16384 words
    uint32_t* s_ring = reinterpret_cast<uint32_t*>(cb_smem + 65536);  // internal weights
    uint8_t* s_dint = cb_smem + 65536;                                 // internal depths (after the merge)
    __shared__ uint32_t s_wsum[kCbThreads / 32];
    __shared__ uint32_t s_tmp[32];
    __shared__ uint32_t s_rowbase[16];
    __shared__ uint32_t s_n, s_maxf, s_maxlen;
    __shared__ uint32_t s_cnt[66];
    __shared__ uint64_t s_first[66];
    if (st->err) return;
    const int tid = threadIdx.x;
    const int m = st->m;
    const int ntot = 1 << m;
    uint32_t* usedlist = nodebuf;                 // [2^16] used symbols, ascending
    uint32_t* par = nodebuf + 65536;              // [2^17] parent of node
    uint32_t* leafw_g = nodebuf + 3 * 65536;      // [2^16] sorted leaf weights (large alphabets)
    uint32_t* sortedsym = nodebuf + 4 * 65536;    // [2^16] symbols in leaf order
    // 1. compact the used symbols (ascending) with their keys
    if (tid == 0) {
        s_n = 0;
        s_maxf = 0;
        s_maxlen = 0;
    }
    __syncthreads();
    for (int base = 0; base < ntot; base += kCbThreads) {
        int s = base + tid;
        uint32_t f = s < ntot ? hist[s] : 0u;
        bool u = f > 0;
        unsigned b = __ballot_sync(0xffffffffu, u);
        int wid = tid >> 5, ln = tid & 31;
        if (ln == 0) s_wsum[wid] = __popc(b);
        __syncthreads();
        if (tid == 0) {
            uint32_t acc = s_n;
            for (int w = 0; w < kCbThreads / 32; w++) { uint32_t t = s_wsum[w]; s_wsum[w] = acc; acc += t; }
            s_n = acc;
        }
        __syncthreads();
        if (u) {
            uint32_t pos = s_wsum[wid] + __popc(b & ((1u << ln) - 1u));
            usedlist[pos] = (uint32_t)s;
            sortbuf[pos] = ((uint64_t)f << 16) | (uint64_t)s;
            atomicMax(&s_maxf, f);
        }
        __syncthreads();
    }
    const int n = (int)s_n;
    for (int s = tid; s < ntot; s += kCbThreads) len[s] = 0;
    __syncthreads();
    if (n == 0) return;
    if (n == 1) {
        if (tid == 0) {
            uint32_t s = usedlist[0];
            len[s] = 1;
            cw[s] = 1ull << 56;  // length 1, code 0
            st->nsym = 1;
            st->maxlen = 1;
        }
        return;
    }
    // 2. leaves in (frequency, symbol) order: weights to region A (or global), symbols to sortedsym
    const bool leaves_smem = n <= 16384;
    if (n <= kSmemSortCap) {
        int np2 = 1;
        while (np2 < n) np2 <<= 1;
        for (int i = tid; i < np2; i += kCbThreads) s_keys[i] = i < n ? sortbuf[i] : ~0ull;
        __syncthreads();
        bitonic_sort(s_keys, np2);
        uint64_t tmp[kSmemSortCap / kCbThreads];
#pragma unroll
        for (int k = 0; k < kSmemSortCap / kCbThreads; k++) {
            const int i = tid + k * kCbThreads;
            tmp[k] = i < n ? s_keys[i] : 0ull;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kSmemSortCap / kCbThreads; k++) {
            const int i = tid + k * kCbThreads;
            if (i < n) {
                s_a32[i] = (uint32_t)(tmp[k] >> 16);
                sortedsym[i] = (uint32_t)(tmp[k] & 0xffffu);
            }
        }
    } else {
        // stable LSD radix sort by frequency, 4-bit digits, counters [digit][thread] in region A
        uint64_t* src = sortbuf;
        uint64_t* dst = sortbuf + 65536;
        const int chunk = (n + kCbThreads - 1) / kCbThreads;
        const int lo = min(n, tid * chunk), hi = min(n, lo + chunk);
        const int bits = 32 - __clz((int)s_maxf);
        for (int sh = 16; sh < 16 + bits; sh += 4) {
            for (int d = 0; d < 16; d++) s_a32[d * kCbThreads + tid] = 0;
            for (int i = lo; i < hi; i++) s_a32[(int)((src[i] >> sh) & 15u) * kCbThreads + tid]++;
            __syncthreads();
            for (int d = 0; d < 16; d++) {
                uint32_t tot;
                const uint32_t ex = block_excl_scan(s_a32[d * kCbThreads + tid], s_tmp, &tot);
                s_a32[d * kCbThreads + tid] = ex;
                if (tid == 0) s_rowbase[d] = tot;
            }
            __syncthreads();
            if (tid == 0) {
                uint32_t acc = 0;
                for (int d = 0; d < 16; d++) { uint32_t t = s_rowbase[d]; s_rowbase[d] = acc; acc += t; }
            }
            __syncthreads();
            for (int d = 0; d < 16; d++) s_a32[d * kCbThreads + tid] += s_rowbase[d];
            __syncthreads();
            for (int i = lo; i < hi; i++) {
                const uint64_t key = src[i];
                const int d = (int)((key >> sh) & 15u);
                dst[s_a32[d * kCbThreads + tid]++] = key;
            }
            __syncthreads();
            uint64_t* t = src;
            src = dst;
            dst = t;
        }
        for (int i = tid; i < n; i += kCbThreads) {
            const uint64_t key = src[i];
            sortedsym[i] = (uint32_t)(key & 0xffffu);
            if (leaves_smem) s_a32[i] = (uint32_t)(key >> 16);
            else leafw_g[i] = (uint32_t)(key >> 16);
        }
    }
    __syncthreads();
    // 3. two-queue merge (thread 0): leaves 0..n-1, internal nodes n..2n-2;
    //    a leaf is taken first on equal weight.  The fronts of both queues and
    //    the element behind each are kept in registers, so that a pick never
    //    waits for a shared-memory load: the load for the element behind is
    //    issued when the front moves up.
    if (tid == 0) {
        const uint32_t* LW = leaves_smem ? s_a32 : leafw_g;
        int q1 = 0, q2 = n, nxt = n;
        uint32_t wl = LW[0], wl1 = n > 1 ? LW[1] : 0u;  // leaf queue: front, behind it
        uint32_t wq = 0, wq1 = 0;                       // internal queue: front, behind it (if present)
        for (int step = 0; step < n - 1; step++) {
            int pk[2];
            uint32_t w[2];
#pragma unroll
            for (int k = 0; k < 2; k++) {
                const bool leaf = q1 < n && (q2 >= nxt || wl <= wq);
                if (leaf) {
                    pk[k] = q1;
                    w[k] = wl;
                    q1++;
                    wl = wl1;
                    wl1 = q1 + 1 < n ? LW[q1 + 1] : 0u;
                } else {
                    pk[k] = q2;
                    w[k] = wq;
                    q2++;
                    wq = wq1;
                    wq1 = q2 + 1 < nxt ? s_ring[(q2 + 1) & (kCbRing - 1)] : 0u;
                }
            }
            const uint32_t sum = w[0] + w[1];
            s_ring[nxt & (kCbRing - 1)] = sum;
            if (q2 == nxt) wq = sum;            // the queue was empty: the new node is its front
            else if (q2 + 1 == nxt) wq1 = sum;  // ... or the element behind the front
            par[pk[0]] = (uint32_t)nxt;
            par[pk[1]] = (uint32_t)nxt;
            nxt++;
        }
    }
    __syncthreads();
    // 4. depths of the internal nodes (node n + i is internal node i; the root
    //    is nint - 1; every parent has a larger index).  Up to 16384 internal
    //    nodes: pointer jumping -- every node holds an ancestor and its
    //    distance to it, and each round replaces the ancestor by the
    //    ancestor's ancestor (adding the distances) until every node reaches
    //    the root; two buffers, one barrier a round.  Beyond that: one pass
    //    top-down on one thread.
    const int nint = n - 1;
    if (nint <= 16384) {
        uint16_t* ancA = reinterpret_cast<uint16_t*>(cb_smem + 65536);  // ring region: 4 x 32 KB
        uint16_t* ancB = ancA + 16384;
        uint8_t* dA = cb_smem + 65536 + 65536;
        uint8_t* dB = dA + 16384;
        for (int i = tid; i < nint; i += kCbThreads) {
            const bool root = i == nint - 1;
            ancA[i] = (uint16_t)(root ? i : (int)(par[n + i] - (uint32_t)n));
            dA[i] = root ? 0 : 1;
        }
        __syncthreads();
        for (;;) {
            int moved = 0;
            for (int i = tid; i < nint; i += kCbThreads) {
                const int a = ancA[i];
                const int aa = ancA[a];
                ancB[i] = (uint16_t)aa;
                dB[i] = (uint8_t)(dA[i] + (a == aa ? 0 : dA[a]));
                moved |= a != aa;
            }
            const int any = __syncthreads_or(moved);
            uint16_t* ta = ancA;
            ancA = ancB;
            ancB = ta;
            uint8_t* td = dA;
            dA = dB;
            dB = td;
            if (!any) break;
        }
        // dA holds every internal node's depth (distance to the root)
        for (int i = tid; i < nint; i += kCbThreads) s_dint[i] = dA[i];  // s_dint lies before dA (ring region)
        __syncthreads();
    } else {
        if (tid == 0) {
            s_dint[nint - 1] = 0;  // the root, node 2n-2
            for (int v = nint - 2; v >= 0; v--) s_dint[v] = (uint8_t)(s_dint[par[n + v] - (uint32_t)n] + 1);
        }
        __syncthreads();
    }
    for (int i = tid; i < n; i += kCbThreads) {
        const uint32_t d = (uint32_t)s_dint[par[i] - (uint32_t)n] + 1u;
        len[sortedsym[i]] = (uint8_t)d;
        atomicMax(&s_maxlen, d);
    }
    __syncthreads();
    if (tid == 0) {
        st->nsym = (uint32_t)n;
        st->maxlen = s_maxlen;
    }
    // 5. canonical codes: first code of each length
    if (tid < 66) s_cnt[tid] = 0;
    __syncthreads();
    for (int i = tid; i < n; i += kCbThreads) atomicAdd(&s_cnt[len[usedlist[i]]], 1u);
    __syncthreads();
    if (tid == 0) {
        uint64_t code = 0;
        int prevL = 0;
        bool firstSeen = false;
        for (int L = 1; L <= 64; L++) {
            if (!s_cnt[L]) continue;
            if (!firstSeen) { code = 0; firstSeen = true; }
            else code = code << (L - prevL);
            s_first[L] = code;
            code += s_cnt[L];
            prevL = L;
        }
    }
    __syncthreads();
    canonical_assign(usedlist, n, len, s_first, cw, nullptr);
}

__global__ void __launch_bounds__(kCbThreads) k_codebook(const uint32_t* __restrict__ hist, DevState* st,
                                                          uint8_t* len, uint64_t* cw, uint64_t* sortbuf,
                                                          uint32_t* nodebuf) {
    codebook_block(hist, st, len, cw, sortbuf, nodebuf);
}

struct CodebookArgs {
    const uint32_t* hist;
    DevState* st;
    uint8_t* len;
    uint64_t* cw;
    uint64_t* sortbuf;
    uint32_t* nodebuf;
};

// every field of a batch in one launch, one CTA per field
__global__ void __launch_bounds__(kCbThreads) k_codebook_batch(const CodebookArgs* __restrict__ A) {
    const CodebookArgs a = A[blockIdx.x];
    codebook_block(a.hist, a.st, a.len, a.cw, a.sortbuf, a.nodebuf);
}

size_t codebook_args_bytes() { return sizeof(CodebookArgs); }

void codebook_args_fill(void* dst, const uint32_t* hist, DevState* st, uint8_t* len, uint64_t* cw, uint64_t* sortbuf,
                        uint32_t* nodebuf) {
    const CodebookArgs a = {hist, st, len, cw, sortbuf, nodebuf};
    memcpy(dst, &a, sizeof(a));
}

int launch_codebook_batch(const void* args_dev, int count, cudaStream_t s) {
    if (count < 1) return SZGB_OK;
    static std::once_flag once;
    static bool ok = false;
    std::call_once(once, [] {
        ok = cudaFuncSetAttribute(k_codebook_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kCbSmem) ==
             cudaSuccess;
        if (!ok) cudaGetLastError();
    });
    if (!ok) return SZGB_ECUDA;
    k_codebook_batch<<<count, kCbThreads, kCbSmem, s>>>(static_cast<const CodebookArgs*>(args_dev));
    return cudaGetLastError() == cudaSuccess ? 0 : SZGB_ECUDA;
}

int launch_codebook(const uint32_t* hist, DevState* st, uint8_t* len, uint64_t* cw, uint64_t* sortbuf,
                    uint32_t* nodebuf, cudaStream_t s) {
    static std::once_flag once;
    static bool ok = false;
    std::call_once(once, [] {
        ok = cudaFuncSetAttribute(k_codebook, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kCbSmem) ==
             cudaSuccess;
        if (!ok) cudaGetLastError();
    });
    if (!ok) return SZGB_ECUDA;
    k_codebook<<<1, kCbThreads, kCbSmem, s>>>(hist, st, len, cw, sortbuf, nodebuf);
    return cudaGetLastError() == cudaSuccess ? 0 : SZGB_ECUDA;
}

// ---------------------------------------------------------------------------
// per-chunk byte counts: Huffman code bits plus 9 + t record bits after code
// 0, rounded up to whole bytes (a chunk is `chunk` points of a row, or the
// whole row when chunk = 0)

// lattice variant when OK != nullptr: an outlier record is 1 + 64 bits, +32
// when its lattice value misses the bound.  One warp per row; a lane takes 8
// consecutive codes as one 16-byte vector, 256 codes a warp step (two steps
// in flight).  A chunk of at least 256 points (chunk sizes are powers of two)
// spans whole steps and its sum is carried from step to step; a shorter
// chunk is chunk / 8 aligned lanes of one step, summed by a shuffle
// reduction inside that lane group.
__global__ void __launch_bounds__(256) k_rowbits(const uint16_t* __restrict__ codes, uint64_t pitch,
                                                 const float* __restrict__ x, uint64_t rows,
                                                 uint64_t rowlen, uint32_t chunk, const uint8_t* __restrict__ len,
                                                 uint32_t* rowbytes, DevState* st, const uint8_t* __restrict__ OK) {
    const int lane = threadIdx.x & 31;
    const uint64_t wglob = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    if (st->err) return;
    const int e_eb = st->e_eb;
    const uint64_t nseg = chunks_per_row(chunk, rowlen);
    const int G = (chunk == 0 || chunk >= 256) ? 32 : (int)(chunk / 8);  // lanes per chunk in a step
    const int cshift = chunk ? __ffs((int)chunk) - 1 : 0;                // chunk is a power of two
    const uint64_t cmask = chunk ? (uint64_t)chunk - 1 : 0;
    unsigned long long kcount = 0;
    uint32_t maxb = 0;
    for (uint64_t r = wglob; r < rows; r += nw) {
        const uint64_t base = r * rowlen;
        const uint16_t* crow = codes + r * pitch;
        uint64_t carry = 0;  // bits of the current chunk in earlier steps (G = 32)
        for (uint64_t l0 = 0; l0 < rowlen; l0 += 512) {
            uint4 q[2];
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const uint64_t l = l0 + 256 * h + (uint64_t)lane * 8;
                q[h] = l < rowlen ? __ldcs(reinterpret_cast<const uint4*>(crow + l)) : make_uint4(0u, 0u, 0u, 0u);
            }
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const uint64_t lb = l0 + 256 * h;  // first point of the step (warp-uniform)
                if (lb >= rowlen) continue;
                const uint64_t l = lb + (uint64_t)lane * 8;
                const uint32_t w[4] = {q[h].x, q[h].y, q[h].z, q[h].w};
                const int nv = l < rowlen ? (rowlen - l < 8 ? (int)(rowlen - l) : 8) : 0;
                uint32_t bits = 0;  // at most 8 x (64 + 97) per lane, 32 lanes: fits 32 bits
#pragma unroll
                for (int k = 0; k < 8; k++) {
                    if (k < nv) {
                        const uint32_t c = (w[k >> 1] >> (16 * (k & 1))) & 0xffffu;
                        bits += __ldg(len + c);
                        if (c == 0) {
                            bits += OK ? (OK[base + l + k] ? 65u : 97u)
                                       : (uint32_t)(9 + trunc_bits(__float_as_uint(x[base + l + k]), e_eb));
                            kcount++;
                        }
                    }
                }
                for (int o = G >> 1; o > 0; o >>= 1) bits += __shfl_xor_sync(0xffffffffu, bits, o);
                if (G == 32) {
                    carry += bits;
                    const uint64_t send = lb + 256;
                    if (send >= rowlen || (chunk && (send & cmask) == 0)) {  // the chunk ends with this step
                        if (lane == 0) {
                            const uint32_t b = (uint32_t)((carry + 7) / 8);
                            rowbytes[r * nseg + (chunk ? lb >> cshift : 0)] = b;
                            maxb = b > maxb ? b : maxb;
                        }
                        carry = 0;
                    }
                } else if ((lane & (G - 1)) == 0 && l < rowlen) {
                    const uint32_t b = (uint32_t)((bits + 7) / 8);
                    rowbytes[r * nseg + (l >> cshift)] = b;
                    maxb = b > maxb ? b : maxb;
                }
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) maxb = max(maxb, __shfl_xor_sync(0xffffffffu, maxb, o));
    if (lane == 0 && maxb) atomicMax(&st->maxrow, maxb);
    for (int o = 16; o > 0; o >>= 1) kcount += __shfl_xor_sync(0xffffffffu, kcount, o);
    if (lane == 0 && kcount) atomicAdd(&st->K, kcount);
}

// Blocks of `fn` that are resident at once on the current device (its SMs times
// the blocks an SM holds at this block size and shared memory): a grid-stride
// kernel launched with exactly that many runs in one wave, with no partial
// second wave at the end.
static uint64_t resident_blocks(const void* fn, int block, size_t smem) {
    int dev = 0, sms = 0, per = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, block, smem) != cudaSuccess || per < 1 || sms < 1) {
        cudaGetLastError();
        return 152;
    }
    return (uint64_t)sms * (uint64_t)per;
}

int launch_rowbits(const uint16_t* codes, uint64_t pitch, const float* x, uint64_t rows, uint64_t rowlen,
                   uint32_t chunk, const uint8_t* len, uint32_t* rowbytes, DevState* st, cudaStream_t s,
                   const uint8_t* OK) {
    static const uint64_t resident = resident_blocks(reinterpret_cast<const void*>(k_rowbits), 256, 0);
    uint64_t warps = rows;
    uint64_t blocks = (warps * 32 + 255) / 256;
    if (blocks > resident) blocks = resident;
    if (blocks < 1) blocks = 1;
    k_rowbits<<<(int)blocks, 256, 0, s>>>(codes, pitch, x, rows, rowlen, chunk, len, rowbytes, st, OK);
    return cudaGetLastError() == cudaSuccess ? 0 : SZGB_ECUDA;
}

// ---------------------------------------------------------------------------
// exclusive scan of chunk byte counts -> chunk offsets.  One tile of 2048
// entries: one kernel.  Up to kScanAddMax tiles: the tile scans, then one
// kernel in which every tile adds the sum of the tiles before it (read from
// the tile sums, which it reduces itself).  More tiles: the tile sums are
// scanned by one warp in between (three kernels).  No kernel waits for another
// block.

constexpr int kScanTile = 2048;
constexpr int kScanAddMax = 1024;

// the payload's byte total is known: sizes of the stream's sections
// (compression) or the payload length to check (decompression)
__device__ __forceinline__ void scan_finalize(DevState* st, uint64_t rows, uint64_t acc, int finalize) {
    st->payload = acc;
    if (finalize) {
        const unsigned tw = st->maxrow <= 0xffffu ? 2u : 4u;
        st->table_width = tw;
        st->cb_bytes = (3ull * st->nsym + 3) & ~3ull;
        st->tab_bytes = ((uint64_t)tw * rows + 3) & ~3ull;
        st->total = (uint64_t)kHeaderBytes + st->cb_bytes + st->tab_bytes + acc;
        st->fits = st->total <= st->cap;
        if (!st->fits) st->err |= kErrOverflow;
    }
}

// in: the counts (tab == nullptr), or the stream's chunk table of `width`-byte
// little-endian entries (4-byte aligned), whose values are also written to
// counts_out.  A thread takes two consecutive entries; a warp-shuffle scan of
// the thread sums, then of the warp sums, gives every entry its exclusive
// prefix within the tile (two barriers).  A grid of one tile finalizes the
// state itself (st != nullptr).
__global__ void __launch_bounds__(1024) k_scan_local(const uint32_t* __restrict__ in, uint64_t n,
                                                     uint64_t* out, uint64_t* blocksums,
                                                     const uint8_t* __restrict__ tab, int width,
                                                     uint32_t* __restrict__ counts_out, DevState* st,
                                                     int finalize) {
    __shared__ uint64_t s_w[32];
    const uint64_t base = (uint64_t)blockIdx.x * kScanTile;
    const uint64_t i0 = base + 2 * (uint64_t)threadIdx.x;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t v0 = 0, v1 = 0;
    if (tab) {
        if (width == 2) {
            if (i0 + 1 < n) {
                const uint32_t u = *reinterpret_cast<const uint32_t*>(tab + 2 * i0);  // two entries
                v0 = u & 0xffffu;
                v1 = u >> 16;
            } else if (i0 < n) {
                v0 = *reinterpret_cast<const uint16_t*>(tab + 2 * i0);
            }
        } else {
            if (i0 < n) v0 = reinterpret_cast<const uint32_t*>(tab)[i0];
            if (i0 + 1 < n) v1 = reinterpret_cast<const uint32_t*>(tab)[i0 + 1];
        }
        if (i0 < n) counts_out[i0] = v0;
        if (i0 + 1 < n) counts_out[i0 + 1] = v1;
    } else {
        if (i0 < n) v0 = in[i0];
        if (i0 + 1 < n) v1 = in[i0 + 1];
    }
    const uint64_t t = (uint64_t)v0 + v1;
    uint64_t incl = t;  // inclusive scan of the thread sums within the warp
    for (int o = 1; o < 32; o <<= 1) {
        const uint64_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) s_w[wid] = incl;
    __syncthreads();
    if (wid == 0) {  // exclusive scan of the warp sums
        const uint64_t w = s_w[lane];
        uint64_t wi = w;
        for (int o = 1; o < 32; o <<= 1) {
            const uint64_t y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        s_w[lane] = wi - w;
        if (lane == 31) {
            if (st) scan_finalize(st, n, wi, finalize);
            else blocksums[blockIdx.x] = wi;
        }
    }
    __syncthreads();
    const uint64_t excl = s_w[wid] + incl - t;
    if (i0 < n) out[i0] = excl;
    if (i0 + 1 < n) out[i0 + 1] = excl + v0;
}

// one warp: exclusive scan of the block sums, 32 at a time (more than
// kScanAddMax tiles)
__global__ void __launch_bounds__(32) k_scan_blocks(uint64_t* blocksums, int nblocks, DevState* st,
                                                    uint64_t rows, int finalize) {
    const int lane = threadIdx.x;
    uint64_t acc = 0;
    for (int b0 = 0; b0 < nblocks; b0 += 32) {
        const int b = b0 + lane;
        const uint64_t t = b < nblocks ? blocksums[b] : 0;
        uint64_t incl = t;
        for (int o = 1; o < 32; o <<= 1) {
            const uint64_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (b < nblocks) blocksums[b] = acc + incl - t;
        acc += __shfl_sync(0xffffffffu, incl, 31);
    }
    if (lane == 0) scan_finalize(st, rows, acc, finalize);
}

// tile b's entries += the sum of tiles < b: blocksums already scanned
// (st == nullptr), or the tile sums, reduced here over [0, b); the last tile
// then finalizes the state
__global__ void __launch_bounds__(1024) k_scan_add(uint64_t* out, uint64_t n, const uint64_t* blocksums,
                                                   DevState* st, int finalize) {
    __shared__ uint64_t s_w[32];
    __shared__ uint64_t s_add;
    const int b = (int)blockIdx.x;
    if (!st) {
        if (threadIdx.x == 0) s_add = blocksums[b];
    } else {
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        uint64_t v = 0;
        for (int i = threadIdx.x; i < b; i += blockDim.x) v += blocksums[i];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) s_w[wid] = v;
        __syncthreads();
        if (wid == 0) {
            v = s_w[lane];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) {
                s_add = v;
                if (b == (int)gridDim.x - 1) scan_finalize(st, n, v + blocksums[b], finalize);
            }
        }
    }
    __syncthreads();
    const uint64_t base = (uint64_t)b * kScanTile;
    const uint64_t add = s_add;
    for (int i = threadIdx.x; i < kScanTile; i += blockDim.x)
        if (base + i < n) out[base + i] += add;
}

int launch_scan_rows(const uint32_t* rowbytes, uint64_t rows, uint64_t* rowoff, uint64_t* blocksums,
                     DevState* st, int finalize_compress, cudaStream_t s, const uint8_t* table, int width) {
    const uint64_t nb = (rows + kScanTile - 1) / kScanTile;
    const uint32_t* in = table ? nullptr : rowbytes;
    uint32_t* counts_out = const_cast<uint32_t*>(rowbytes);
    if (nb <= 1) {
        k_scan_local<<<1, 1024, 0, s>>>(in, rows, rowoff, blocksums, table, width, counts_out, st,
                                        finalize_compress);
    } else if (nb <= (uint64_t)kScanAddMax) {
        k_scan_local<<<(unsigned)nb, 1024, 0, s>>>(in, rows, rowoff, blocksums, table, width, counts_out, nullptr, 0);
        k_scan_add<<<(unsigned)nb, 1024, 0, s>>>(rowoff, rows, blocksums, st, finalize_compress);
    } else {
        k_scan_local<<<(unsigned)nb, 1024, 0, s>>>(in, rows, rowoff, blocksums, table, width, counts_out, nullptr, 0);
        k_scan_blocks<<<1, 32, 0, s>>>(blocksums, (int)nb, st, rows, finalize_compress);
        k_scan_add<<<(unsigned)nb, 1024, 0, s>>>(rowoff, rows, blocksums, nullptr, 0);
    }
    return cudaGetLastError() == cudaSuccess ? 0 : SZGB_ECUDA;
}

// ---------------------------------------------------------------------------
// stream writer

__device__ __forceinline__ void wr_u16(uint8_t* p, uint32_t v) { p[0] = (uint8_t)v; p[1] = (uint8_t)(v >> 8); }
__device__ __forceinline__ void wr_u32(uint8_t* p, uint32_t v) {
    for (int i = 0; i < 4; i++) p[i] = (uint8_t)(v >> (8 * i));
}
__device__ __forceinline__ void wr_u64(uint8_t* p, uint64_t v) {
    for (int i = 0; i < 8; i++) p[i] = (uint8_t)(v >> (8 * i));
}

// header, codebook section and chunk table
__global__ void __launch_bounds__(256) k_write_meta(const CallParams cp, uint64_t rows /* chunks */,
                                                    const uint8_t* __restrict__ len,
                                                    const uint32_t* __restrict__ usedlist,
                                                    const uint32_t* __restrict__ rowbytes,
                                                    const uint64_t* __restrict__ rowoff, uint8_t* out,
                                                    DevState* st) {
    if (!st->fits || st->err) return;
    const uint64_t cb = st->cb_bytes, tb = st->tab_bytes;
    const unsigned tw = st->table_width;
    const uint32_t nsym = st->nsym;
    uint8_t* cbp = out + kHeaderBytes;
    uint8_t* tab = cbp + cb;
    const uint64_t tid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    const uint64_t nthr = (uint64_t)gridDim.x * blockDim.x;
    if (tid == 0) {
        uint8_t* h = out;
        for (int i = 0; i < kHeaderBytes; i++) h[i] = 0;
        h[0] = 'S'; h[1] = 'Z'; h[2] = 'G'; h[3] = 'B';
        wr_u16(h + 4, 1);
        wr_u16(h + 6, kHeaderBytes);
        h[8] = (uint8_t)cp.ndim;
        h[9] = (uint8_t)cp.layers;
        h[10] = (uint8_t)st->m;
        h[11] = (uint8_t)cp.mode;
        h[12] = (uint8_t)st->maxlen;
        h[13] = (uint8_t)tw;
        wr_u64(h + 16, cp.d0);
        wr_u64(h + 24, cp.d1);
        wr_u64(h + 32, cp.d2);
        wr_u64(h + 40, (uint64_t)__double_as_longlong(cp.eb_abs));
        wr_u64(h + 48, (uint64_t)__double_as_longlong(cp.eb_rel));
        wr_u32(h + 56, __float_as_uint(st->eb_f));
        wr_u32(h + 60, __float_as_uint(st->xmin));
        wr_u32(h + 64, __float_as_uint(st->xmax));
        wr_u32(h + 68, nsym);
        wr_u64(h + 72, rows);
        wr_u64(h + 80, st->K);
        wr_u64(h + 88, st->payload);
        wr_u64(h + 96, st->total);
        wr_u64(h + 104, (uint64_t)__double_as_longlong(cp.theta));
        h[112] = (uint8_t)(cp.m_user == 0);
        h[113] = (uint8_t)cp.variant;
        wr_u32(h + 116, cp.chunk);  // chunk length along a row; 0: whole rows
    }
    for (uint64_t i = tid; i < cb; i += nthr) {
        uint64_t e = i / 3;
        int k = (int)(i % 3);
        uint8_t v = 0;
        if (e < nsym) {
            uint32_t s = usedlist[e];
            v = (k == 0) ? (uint8_t)s : (k == 1) ? (uint8_t)(s >> 8) : len[s];
        }
        cbp[i] = v;
    }
    for (uint64_t i = tid; i < tb; i += nthr) {
        uint64_t r = i / tw;
        int k = (int)(i % tw);
        tab[i] = (r < rows) ? (uint8_t)(rowbytes[r] >> (8 * k)) : 0;
    }
}

constexpr int kEncWarps = 8;
constexpr int kEncPts = 8;                   // consecutive points per lane (one 16-byte code vector)
constexpr int kEncChunk = 32 * kEncPts;      // points per warp step
// a step's bits: 256 points of at most 64 code bits and a 97-bit record, plus
// the carried partial word and the byte padding of up to 8 chunks ending in it
constexpr int kEncBufWords = (kEncChunk * (64 + 97) + 31) / 32 + 4;

// payload: one warp per row, 256 points per step.  Each lane sums the bit
// lengths of its 8 points; its bit position is its chunk's byte offset, plus
// the bits of that chunk in earlier steps (chunks of at least 256 points),
// plus a scan over the lanes of the chunk (a segmented warp scan when chunks
// are shorter than a step); the lane writes its bits MSB-first into a
// shared-memory word buffer (words it fills alone are stored, the two it may
// share with its neighbours are OR-ed).  A row's chunks are consecutive in
// the payload and each starts on a byte, so the padding between them is
// zero bits the buffer already holds.  Completed words go to the payload; the
// buffer is zero outside the carried word between steps.  Every payload byte
// belongs to exactly one row, so a word a row shares with a neighbour is
// written byte by byte for the row's own bytes only: no atomics, no zeroing
// pass.
__device__ __forceinline__ void store_word_bytes(uint8_t* plb, uint64_t gw, uint32_t val, uint32_t lo,
                                                 uint32_t hi) {
    // val: big-endian word value; write bytes covering bits [lo, hi) of it
    if (lo == 0 && hi == 32) {
        reinterpret_cast<uint32_t*>(plb)[gw] = bswap32(val);
    } else {
        for (uint32_t k = lo >> 3; k < ((hi + 7) >> 3); k++) plb[4 * gw + k] = (uint8_t)(val >> (24 - 8 * k));
    }
}

struct LatticeRec {
    const int32_t* P;   // lattice integers (nullptr: the paper's method)
    const uint8_t* OK;  // lattice value within the bound
    int ndim, layers;
    uint64_t d1;        // rows per plane (the row index of a point is plane * d1 + row)
};

// MSB-first bit writer of one lane into the warp's word buffer
struct LaneBits {
    uint32_t* buf;
    uint32_t wi, wfirst, nacc;
    uint64_t acc;
    __device__ __forceinline__ LaneBits(uint32_t* b, uint32_t off)
        : buf(b), wi(off >> 5), wfirst(off >> 5), nacc(off & 31), acc(0) {}
    // append the n low bits of v, n in [0, 32]
    __device__ __forceinline__ void put(uint32_t v, uint32_t n) {
        acc = (acc << n) | v;
        nacc += n;
        if (nacc >= 32) {
            nacc -= 32;
            const uint32_t w = (uint32_t)(acc >> nacc);
            if (wi == wfirst) atomicOr(buf + wi, w);
            else buf[wi] = w;
            wi++;
            acc &= (1ull << nacc) - 1ull;
        }
    }
    __device__ __forceinline__ void put64(uint64_t v, uint32_t n) {
        if (n > 32) {
            put((uint32_t)(v >> 32), n - 32);
            put((uint32_t)v, 32);
        } else {
            put((uint32_t)v, n);
        }
    }
    __device__ __forceinline__ void finish() {
        if (nacc) atomicOr(buf + wi, (uint32_t)(acc << (32 - nacc)));
    }
};

__global__ void __launch_bounds__(kEncWarps * 32) k_encode(const uint16_t* __restrict__ codes, uint64_t pitch,
                                                          const float* __restrict__ x, uint64_t rows,
                                                          uint64_t rowlen, uint32_t chunk,
                                                          const uint8_t* __restrict__ len,
                                                          const uint64_t* __restrict__ cw,
                                                          const uint64_t* __restrict__ rowoff,
                                                          uint8_t* out, DevState* st, const LatticeRec LR) {
    extern __shared__ uint32_t sbuf[];
    if (!st->fits || st->err) return;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    uint32_t* buf = sbuf + wib * kEncBufWords;
    uint8_t* plb = out + kHeaderBytes + st->cb_bytes + st->tab_bytes;
    const int e_eb = st->e_eb;
    const uint64_t wglob = blockIdx.x * (uint64_t)kEncWarps + wib;
    const uint64_t nw = (uint64_t)gridDim.x * kEncWarps;
    const uint64_t nseg = chunks_per_row(chunk, rowlen);
    const int G = (chunk == 0 || chunk >= kEncChunk) ? 32 : (int)(chunk / kEncPts);  // lanes per chunk in a step
    const int cshift = chunk ? __ffs((int)chunk) - 1 : 0;  // chunk is a power of two (0: whole rows)
    const uint64_t cmask = chunk ? (uint64_t)chunk - 1 : 0;
    for (int i = lane; i < kEncBufWords; i += 32) buf[i] = 0;
    __syncwarp();
    for (uint64_t r = wglob; r < rows; r += nw) {
        const uint64_t* const coff = rowoff + r * nseg;  // byte offsets of the row's chunks
        const uint64_t g0 = coff[0] * 8;          // first bit of the row in the payload
        const uint64_t w0 = g0 >> 5;              // its word
        const uint32_t lo0 = (uint32_t)(g0 & 31); // bits of w0 owned by earlier rows
        uint64_t curw = w0;                        // global word held in buf[0]
        uint32_t bitpos = lo0;                     // bits already used in buf[0]
        uint64_t carry = 0;                        // bits of the current chunk in earlier steps (G = 32)
        const uint64_t base = r * rowlen;
        const uint16_t* crow = codes + r * pitch;
        for (uint64_t l0 = 0; l0 < rowlen; l0 += kEncChunk) {
            const uint64_t l = l0 + (uint64_t)lane * kEncPts;
            const int nv = l < rowlen ? (rowlen - l < kEncPts ? (int)(rowlen - l) : kEncPts) : 0;
            uint32_t w[4] = {0u, 0u, 0u, 0u};
            if (nv) {
                const uint4 q = __ldcs(reinterpret_cast<const uint4*>(crow + l));
                w[0] = q.x;
                w[1] = q.y;
                w[2] = q.z;
                w[3] = q.w;
            }
            uint32_t nbits = 0;
            bool any0 = false;
            uint32_t L[kEncPts];
            uint64_t cwk[kEncPts];
#pragma unroll
            for (int k = 0; k < kEncPts; k++) {
                L[k] = 0;
                cwk[k] = 0;
                if (k < nv) {
                    const uint32_t c = (w[k >> 1] >> (16 * (k & 1))) & 0xffffu;
                    const uint64_t e = __ldg(cw + c);  // length << 56 | code
                    L[k] = (uint32_t)(e >> 56);
                    cwk[k] = e & ((1ull << 56) - 1ull);
                    nbits += L[k];
                    if (c == 0) {
                        any0 = true;
                        const uint32_t u = __float_as_uint(x[base + l + k]);
                        nbits += LR.P ? (LR.OK[base + l + k] ? 65u : 97u) : (uint32_t)(9 + trunc_bits(u, e_eb));
                    }
                }
            }
            uint32_t incl = nbits;  // inclusive scan over the lanes of this lane's chunk
            for (int o = 1; o < G; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
                if ((lane & (G - 1)) >= o) incl += y;
            }
            if (G == 32 && chunk && (l0 & cmask) == 0) carry = 0;  // a chunk starts with this step
            // this lane's chunk (lanes past the row end take the step's first)
            const uint64_t lc = (l < rowlen ? l : l0);
            const uint64_t cstart = coff[chunk ? lc >> cshift : 0] * 8 + (G == 32 ? carry : 0);
            const uint32_t off = (uint32_t)(cstart - curw * 32) + incl - nbits;
            // the step ends where its last lane with points ends
            const int last = (int)min((uint64_t)31, (rowlen - 1 - l0) / kEncPts);
            const uint32_t stepend = __shfl_sync(0xffffffffu, off + nbits, last);
            if (G == 32) carry += __shfl_sync(0xffffffffu, incl, 31);
            if (!any0 && nbits <= 64) {
                // common case: the lane's codes fit one 64-bit register; they
                // span at most three buffer words (OR-ed: neighbours may share them)
                uint64_t bits = 0;
#pragma unroll
                for (int k = 0; k < kEncPts; k++) bits = (bits << L[k]) | cwk[k];  // L <= 46
                if (nbits) {
                    const uint64_t a = bits << (64 - nbits);  // MSB-aligned
                    const uint32_t wi = off >> 5, sh = off & 31;
                    atomicOr(buf + wi, (uint32_t)(a >> (32 + sh)));
                    if (sh + nbits > 32) atomicOr(buf + wi + 1, (uint32_t)(a >> sh));
                    if (sh + nbits > 64) atomicOr(buf + wi + 2, (uint32_t)(a << (32 - sh)));
                }
            } else {
                LaneBits wr(buf, off);
#pragma unroll
                for (int k = 0; k < kEncPts; k++) {
                    if (k < nv) {
                        const uint32_t c = (w[k >> 1] >> (16 * (k & 1))) & 0xffffu;
                        wr.put64(cwk[k], L[k]);
                        if (any0 && c == 0) {
                            const uint32_t u = __float_as_uint(x[base + l + k]);
                            if (LR.P) {  // lattice record: flag, r (64 bits), x when the flag is 0
                                const bool lok = LR.OK[base + l + k] != 0;
                                const uint64_t lres = (uint64_t)lattice_resid_rt(
                                    LR.P, LR.ndim, LR.layers, LR.d1, rowlen, (int64_t)(r / LR.d1),
                                    (int64_t)(r % LR.d1), (int64_t)(l + k));
                                wr.put(lok ? 1u : 0u, 1);
                                wr.put64(lres, 64);
                                if (!lok) wr.put(u, 32);
                            } else {
                                const int t = trunc_bits(u, e_eb);
                                wr.put(u >> 23, 9);
                                if (t) wr.put((u >> (23 - t)) & ((1u << t) - 1u), (uint32_t)t);
                            }
                        }
                    }
                }
                wr.finish();
            }
            __syncwarp();
            const uint32_t end = stepend;
            const uint32_t full = end >> 5;
            for (uint32_t i = lane; i < full; i += 32) {
                const uint64_t gw = curw + i;
                store_word_bytes(plb, gw, buf[i], gw == w0 ? lo0 : 0u, 32u);
                buf[i] = 0;
            }
            __syncwarp();
            const uint32_t cword = buf[full];  // the partial word, carried to buf[0]
            __syncwarp();
            if (lane == 0 && full) {
                buf[0] = cword;
                buf[full] = 0;
            }
            __syncwarp();
            curw += full;
            bitpos = end & 31;
        }
        if (bitpos && lane == 0) store_word_bytes(plb, curw, buf[0], curw == w0 ? lo0 : 0u, bitpos);
        __syncwarp();
        if (lane == 0) buf[0] = 0;
        __syncwarp();
    }
}

int launch_write_meta(const CallParams& cp, uint64_t rows /* chunks */, const uint8_t* len, const uint32_t* usedlist,
                      const uint32_t* rowbytes, const uint64_t* rowoff, uint8_t* out, DevState* st,
                      cudaStream_t s) {
    uint64_t blocks = (rows + 255) / 256;
    if (blocks < 8) blocks = 8;
    if (blocks > 1024) blocks = 1024;
    k_write_meta<<<(int)blocks, 256, 0, s>>>(cp, rows, len, usedlist, rowbytes, rowoff, out, st);
    return cudaGetLastError() == cudaSuccess ? 0 : SZGB_ECUDA;
}

int launch_encode(const uint16_t* codes, uint64_t pitch, const float* x, uint64_t rows, uint64_t rowlen,
                  uint32_t chunk, const uint8_t* len,
                  const uint64_t* cw, const uint64_t* rowoff, uint8_t* out, DevState* st, cudaStream_t s,
                  const int32_t* P, const uint8_t* OK, int ndim, int layers, uint64_t d1) {
    LatticeRec LR;
    LR.P = P;
    LR.OK = OK;
    LR.ndim = ndim;
    LR.layers = layers;
    LR.d1 = d1;
    constexpr size_t smem = (size_t)kEncWarps * kEncBufWords * 4;
    static std::once_flag once;
    static bool ok = true;
    std::call_once(once, [] {
        ok = cudaFuncSetAttribute(k_encode, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) == cudaSuccess;
        if (!ok) cudaGetLastError();
    });
    if (!ok) return SZGB_ECUDA;
    static const uint64_t resident = resident_blocks(reinterpret_cast<const void*>(k_encode), kEncWarps * 32, smem);
    uint64_t blocks = (rows + kEncWarps - 1) / kEncWarps;
    if (blocks > resident) blocks = resident;
    if (blocks < 1) blocks = 1;
    k_encode<<<(int)blocks, kEncWarps * 32, smem, s>>>(codes, pitch, x, rows, rowlen, chunk, len, cw, rowoff, out, st,
                                                       LR);
    return cudaGetLastError() == cudaSuccess ? 0 : SZGB_ECUDA;
}

// ---------------------------------------------------------------------------
// decoder tables from the codebook section (one CTA).
//   lut[2^T]: (symbol << 8) | length for codes of length <= T (0 = longer)
//   dectab[0..64] first code low word per length, [65..129] high word,
//   [130..194] count, [195..259] start index into the sorted list,
//   then the symbols sorted by (length, symbol) as u16 (65536 entries),
//   then the multi-symbol table (kMultiBits index bits, see kMultiOff).

// the decoder tables of one field; every thread of the CTA calls it
__device__ __forceinline__ void decode_tables_block(const uint8_t* __restrict__ cb, uint32_t nsym, int m,
                                                    uint32_t* lut, uint32_t* dectab, uint8_t* lenbuf,
                                                    uint32_t* symbuf, DevState* st) {
    __shared__ uint32_t s_cnt[66];
    __shared__ uint64_t s_first[66];
    __shared__ uint64_t s_next[66];
    __shared__ uint32_t s_start[66];
    __shared__ int s_bad;
    __shared__ int s_maxlen;
    const int ntot = 1 << m;
    if (threadIdx.x < 66) { s_cnt[threadIdx.x] = 0; s_first[threadIdx.x] = 0; }
    if (threadIdx.x == 0) { s_bad = 0; s_maxlen = 0; }
    for (int s = threadIdx.x; s < ntot; s += blockDim.x) lenbuf[s] = 0;
    __syncthreads();
    for (uint32_t e = threadIdx.x; e < nsym; e += blockDim.x) {
        uint32_t s = cb[3 * e] | ((uint32_t)cb[3 * e + 1] << 8);
        uint32_t L = cb[3 * e + 2];
        uint32_t prev = e ? (cb[3 * (e - 1)] | ((uint32_t)cb[3 * (e - 1) + 1] << 8)) : 0;
        if (s >= (uint32_t)ntot || L < 1 || L > 64 || (e && s <= prev)) { s_bad = 1; continue; }
        lenbuf[s] = (uint8_t)L;
        symbuf[e] = s;
        atomicAdd(&s_cnt[L], 1u);
        atomicMax(&s_maxlen, (int)L);
    }
    __syncthreads();
    if (threadIdx.x == 0 && !s_bad) {
        // canonical first codes, start indices, and a Kraft check
        uint64_t code = 0;
        int prevL = 0;
        bool seen = false;
        uint32_t start = 0;
        for (int L = 1; L <= 64; L++) {
            s_start[L] = start;
            if (!s_cnt[L]) continue;
            if (!seen) { code = 0; seen = true; }
            else code = code << (L - prevL);
            s_first[L] = code;
            if (L < 64 && (code + s_cnt[L]) > (1ull << L)) s_bad = 1;
            code += s_cnt[L];
            prevL = L;
            start += s_cnt[L];
        }
        if (nsym == 1 && s_maxlen != 1) s_bad = 1;
    }
    __syncthreads();
    if (s_bad) {
        if (threadIdx.x == 0) st->err |= kErrCorrupt;
        return;
    }
    const int maxlen = s_maxlen;
    const int T = maxlen < kLutBits ? maxlen : kLutBits;
    for (int i = threadIdx.x; i < (1 << T); i += blockDim.x) lut[i] = 0;
    if (threadIdx.x < 65) {
        dectab[threadIdx.x] = (uint32_t)s_first[threadIdx.x];
        dectab[65 + threadIdx.x] = (uint32_t)(s_first[threadIdx.x] >> 32);
        dectab[130 + threadIdx.x] = s_cnt[threadIdx.x];
        dectab[195 + threadIdx.x] = s_start[threadIdx.x];
        s_next[threadIdx.x] = s_first[threadIdx.x];
    }
    __syncthreads();
    // ranks within each length (warp 0, ascending symbols) -> codes
    // sorted[start[L] + rank] = symbol; code = first[L] + rank
    uint16_t* sorted = reinterpret_cast<uint16_t*>(dectab + 260);
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        for (uint32_t base = 0; base < nsym; base += 32) {
            uint32_t i = base + lane;
            bool v = i < nsym;
            unsigned act = __ballot_sync(0xffffffffu, v);
            if (v) {
                uint32_t s = symbuf[i];
                int L = lenbuf[s];
                unsigned peers = __match_any_sync(act, L);
                int rank = __popc(peers & ((1u << lane) - 1u));
                uint64_t f = s_next[L];
                uint64_t code = f + (uint64_t)rank;
                uint32_t idx = s_start[L] + (uint32_t)(code - s_first[L]);
                sorted[idx] = (uint16_t)s;
                if (L <= T) {
                    uint32_t lo = (uint32_t)code << (T - L), n = 1u << (T - L);
                    for (uint32_t k = 0; k < n; k++) lut[lo + k] = (s << 8) | (uint32_t)L;
                }
                __syncwarp(act);
                if (rank == 0) s_next[L] = f + (uint64_t)__popc(peers);
            }
            __syncwarp();
        }
    }
    __syncthreads();
    // multi-symbol table: the codes that the next kMultiBits bits hold, taken
    // greedily -- up to 3 symbols < 256 (one of any size), stopping after an
    // escape (code 0: raw bits follow it); 0 when the first code is longer
    {
        constexpr int TB = kMultiBits;
        uint32_t* multi = dectab + kMultiOff;
        // first the single code at the top of every TB-bit window:
        // (symbol << 8) | length, 0 when it is longer than TB
        __shared__ uint32_t s_one[1u << kMultiBits];
        for (uint32_t i = threadIdx.x; i < (1u << TB); i += blockDim.x) {
            uint32_t e = 0;
            for (int l = 1; l <= TB && l <= maxlen; l++) {
                const uint64_t c = i >> (TB - l);
                if (s_cnt[l] && c >= s_first[l] && c - s_first[l] < s_cnt[l]) {
                    e = ((uint32_t)sorted[s_start[l] + (uint32_t)(c - s_first[l])] << 8) | (uint32_t)l;
                    break;
                }
            }
            s_one[i] = e;
        }
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < (1u << TB); i += blockDim.x) {
            const uint32_t e1 = s_one[i];
            const uint32_t s1 = e1 >> 8;
            uint32_t e = 0;
            if (e1) {
                uint32_t n = 1, used = e1 & 0xffu;
                uint32_t sy[3] = {s1, 0, 0};
                while (n < 3 && sy[n - 1] != 0 && sy[n - 1] < 256) {
                    const uint32_t ek = s_one[(i << used) & ((1u << TB) - 1u)];
                    const uint32_t Lk = ek & 0xffu, sk = ek >> 8;
                    if (!Lk || used + Lk > (uint32_t)TB || sk >= 256) break;
                    sy[n++] = sk;
                    used += Lk;
                }
                if (n == 1) e = 1u | (used << 2) | (s1 << 8);
                else e = n | (used << 2) | (sy[0] << 8) | (sy[1] << 16) | (sy[2] << 24);
            }
            multi[i] = e;
        }
    }
    if (threadIdx.x == 0) {
        st->maxlen = (uint32_t)maxlen;
        st->lut_bits = (uint32_t)T;
        st->nsym = nsym;
    }
}

__global__ void __launch_bounds__(1024) k_decode_tables(const uint8_t* __restrict__ cb, uint32_t nsym, int m,
                                                        uint32_t* lut, uint32_t* dectab, uint8_t* lenbuf,
                                                        uint32_t* symbuf, DevState* st) {
    decode_tables_block(cb, nsym, m, lut, dectab, lenbuf, symbuf, st);
}

struct TablesArgs {
    const uint8_t* cb;
    uint32_t* lut;
    uint32_t* dectab;
    uint8_t* lenbuf;
    uint32_t* symbuf;
    DevState* st;
    uint32_t nsym;
    int m;
};

// every field of a batch in one launch, one CTA per field
__global__ void __launch_bounds__(1024) k_decode_tables_batch(const TablesArgs* __restrict__ A) {
    const TablesArgs a = A[blockIdx.x];
    decode_tables_block(a.cb, a.nsym, a.m, a.lut, a.dectab, a.lenbuf, a.symbuf, a.st);
}

size_t tables_args_bytes() { return sizeof(TablesArgs); }

void tables_args_fill(void* dst, const uint8_t* codebook, uint32_t nsym, int m, uint32_t* lut, uint32_t* dec_tab,
                      uint8_t* lenbuf, uint32_t* symbuf, DevState* st) {
    const TablesArgs a = {codebook, lut, dec_tab, lenbuf, symbuf, st, nsym, m};
    memcpy(dst, &a, sizeof(a));
}

int launch_decode_tables_batch(const void* args_dev, int count, cudaStream_t s) {
    if (count < 1) return SZGB_OK;
    k_decode_tables_batch<<<count, 1024, 0, s>>>(static_cast<const TablesArgs*>(args_dev));
    return cudaGetLastError() == cudaSuccess ? 0 : SZGB_ECUDA;
}

int launch_decode_tables(const uint8_t* codebook, uint32_t nsym, int m, uint32_t* lut, uint32_t* dec_tab,
                         uint8_t* lenbuf, uint32_t* symbuf, DevState* st, cudaStream_t s) {
    k_decode_tables<<<1, 1024, 0, s>>>(codebook, nsym, m, lut, dec_tab, lenbuf, symbuf, st);
    return cudaGetLastError() == cudaSuccess ? 0 : SZGB_ECUDA;
}


}  // namespace szgb
