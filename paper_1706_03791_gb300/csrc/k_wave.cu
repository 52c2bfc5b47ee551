// k_wave.cu -- the wavefront kernels of the hot path.
//
// Compression (Algorithm 1, the per-point loop): every point is predicted by
// the n-layer predictor (Eq. predmodel) from the *recorded* (decompressed)
// values of its (n+1)^d - 1 preceding neighbours, quantized into 2^m - 1
// intervals of width 2 eb (Sec. IV-A) or stored as a truncated binary
// representation, and its recorded value is kept for later predictions.
// Decompression runs the same prediction in the same dependency order, with
// the Huffman decode of each row fused in (a row is one stream chunk).
//
// Parallel schedule.  A point depends only on neighbours with smaller
// (plane, row, column) offsets, so any order that respects that DAG gives
// identical bits.  The field is cut into lines along the fastest axis
// ("rows"); a lane owns one row and walks it in tiles of kTile = 4 columns,
// one tile per "sweep".  Lanes are skewed by one sweep per row (2D) or per
// row and per plane (3D), so every value a lane needs from another row or
// plane was produced in an EARLIER sweep and sits in a shared-memory ring;
// only the lane's own left neighbour chain is on the critical path.
//
//   2D: CTA = W warps = 32W consecutive rows, row rho processes tile
//       c = r - rho in sweep r.
//   3D: CTA = W warps (planes) x 32 lanes (rows), lane (w,t) processes tile
//       c = r - w - t in sweep r.
//
// A CTA boundary is crossed through global "halo" buffers: an extra warp per
// CTA copies the CTA's boundary rows/planes out of the ring after each sweep,
// publishes a progress counter (release), and prefetches the neighbouring
// CTAs' halos into the ring (acquire, cp.async), with bounded waits.  CTAs
// take work items from a ticket counter in dependency order, so a CTA only
// ever waits for CTAs that are already resident: forward progress holds for
// any grid size.
#include "szgb_internal.cuh"

namespace szgb {

constexpr int kPFX = 12;  // x prefetch depth (sweeps)
constexpr int kPFH = 3;   // halo prefetch depth (sweeps)

struct WaveArgs {
    WaveGeom g;
    // compress
    const float* x;
    uint16_t* codes;
    float* recorded;
    // decompress
    const uint8_t* payload;
    const uint64_t* rowoff;
    const uint32_t* rowbytes;
    const uint8_t* stream_end;
    const uint32_t* lut;
    const uint32_t* dectab;
    float* out;
    // common
    float* halo_row;
    float* halo_plane;
    unsigned int* prog;
    DevState* st;
    uint64_t timeout_ns;
};

__device__ __forceinline__ int posmod(int a, int m) {
    int r = a % m;
    return r < 0 ? r + m : r;
}

// Bounded wait until *p >= need; `seen` caches the last value observed so
// that a satisfied requirement costs no memory access.  Returns false on
// timeout.
__device__ __forceinline__ bool wait_progress(const unsigned int* p, unsigned int need, unsigned int& seen,
                                              uint64_t timeout_ns) {
    if (seen >= need) return true;
    seen = ld_acquire_u32(p);
    if (seen >= need) return true;
    uint64_t t0 = globaltimer();
    for (unsigned it = 0; it < (1u << 28); it++) {
        __nanosleep(64);
        seen = ld_acquire_u32(p);
        if (seen >= need) return true;
        if ((it & 63) == 63 && globaltimer() - t0 > timeout_ns) return false;
    }
    return false;
}

__device__ __forceinline__ void fence_acq_rel_gpu() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

// ---------------------------------------------------------------------------
// Prediction of the 4 points of a tile from the series of neighbour values.
// S[a][b][j]: values of the line at plane offset a, row offset b, for
// columns (tile start - NL + j), j in [0, NL + 4); S[0][0] is the own line.
// Terms are summed in descending lexicographic (a, b, e) order, the first
// product initialising the sum (as the oracle does).

template <int NL, int ND>
__device__ __forceinline__ float predict_partial(const float (&S)[NL + 1][NL + 1][NL + kTile], int k) {
    // all terms with (a, b) != (0, 0): in descending lexicographic order they
    // come before the own-line terms (0, 0, e)
    constexpr int A = (ND == 3) ? NL : 0;
    constexpr int B = (ND >= 2) ? NL : 0;  // a 1D field has only own-line terms
    float pred = 0.0f;
    bool first = true;
#pragma unroll
    for (int a = A; a >= 0; a--) {
#pragma unroll
        for (int b = B; b >= 0; b--) {
            if (a == 0 && b == 0) continue;
#pragma unroll
            for (int e = NL; e >= 0; e--) {
                const float v = S[a][b][NL + k - e];
                const int c = term_coef(NL, a, b, e);
                if (NL == 1) {
                    if (first) pred = (c > 0) ? v : -v;
                    else pred = (c > 0) ? __fadd_rn(pred, v) : __fsub_rn(pred, v);
                } else {
                    float prod = __fmul_rn((float)c, v);
                    pred = first ? prod : __fadd_rn(pred, prod);
                }
                first = false;
            }
        }
    }
    return pred;
}

// the own-line terms (0, 0, NL) ... (0, 0, 1) added last, in order; in 1D
// they are the only terms and the first one initialises the sum
template <int NL, int ND>
__device__ __forceinline__ float predict_own(float part, const float (&S)[NL + 1][NL + 1][NL + kTile], int k) {
    float pred = part;
#pragma unroll
    for (int e = NL; e >= 1; e--) {
        const float v = S[0][0][NL + k - e];
        const int c = term_coef(NL, 0, 0, e);
        const bool first = (ND == 1 && e == NL);
        if (NL == 1) {
            if (first) pred = (c > 0) ? v : -v;
            else pred = (c > 0) ? __fadd_rn(pred, v) : __fsub_rn(pred, v);
        } else {
            const float prod = __fmul_rn((float)c, v);
            pred = first ? prod : __fadd_rn(pred, prod);
        }
    }
    return pred;
}

// ---------------------------------------------------------------------------
// Per-lane bit reader over one row chunk (MSB-first), for decompression.

struct BitReader {
    const uint8_t* base;
    uint64_t wpos;       // byte offset of the next word to load (multiple of 4)
    uint64_t endoff;     // bytes available from base
    uint64_t win;        // valid bits, MSB aligned
    int nb;              // valid bits in win
    uint32_t pf0, pf1;   // the next two words (already requested)
    uint64_t consumed;   // bits consumed

    __device__ __forceinline__ uint32_t load_word(uint64_t off) const {
        if (off + 4 <= endoff) return bswap32(__ldg(reinterpret_cast<const uint32_t*>(base + off)));
        uint32_t v = 0;
        for (int i = 0; i < 4; i++) v = (v << 8) | (off + i < endoff ? (uint32_t)base[off + i] : 0u);
        return v;
    }
    __device__ __forceinline__ void init(const uint8_t* b, uint64_t start, uint64_t end) {
        base = b;
        endoff = end;
        uint64_t a = start & ~(uint64_t)3;
        int skip = (int)(start - a) * 8;
        uint32_t w0 = load_word(a);
        pf0 = load_word(a + 4);
        pf1 = load_word(a + 8);
        wpos = a + 12;
        win = ((uint64_t)w0 << 32) << skip;
        nb = 32 - skip;
        consumed = 0;
    }
    __device__ __forceinline__ void refill() {
        if (nb <= 32) {
            win |= (uint64_t)pf0 << (32 - nb);
            nb += 32;
            pf0 = pf1;
            pf1 = load_word(wpos);
            wpos += 4;
        }
    }
    // bit p (0 = next bit) looking past the window into the prefetched words
    __device__ __forceinline__ uint32_t bit_at(int p) const {
        if (p < nb) return (uint32_t)(win >> (63 - p)) & 1u;
        p -= nb;
        if (p < 32) return (pf0 >> (31 - p)) & 1u;
        p -= 32;
        return (pf1 >> (31 - p)) & 1u;
    }
    __device__ __forceinline__ void skip(int n) {
        consumed += (uint64_t)n;
        while (n > 0) {
            refill();
            int s = n < nb ? n : nb;
            win = (s == 64) ? 0 : (win << s);
            nb -= s;
            n -= s;
        }
    }
    __device__ __forceinline__ uint32_t take(int n) {  // n <= 32
        if (n == 0) return 0;
        refill();
        uint32_t v = (uint32_t)(win >> (64 - n));
        win <<= n;
        nb -= n;
        consumed += (uint64_t)n;
        return v;
    }
};

// decode one quantization code; long codes (> lut bits) by canonical search
__device__ __forceinline__ int decode_symbol(BitReader& br, const uint32_t* s_lut, int T,
                                             const uint32_t* s_tab, const uint16_t* g_sorted,
                                             int maxlen, bool& bad) {
    br.refill();
    uint32_t e = s_lut[(uint32_t)(br.win >> (64 - T))];
    int len = (int)(e & 0xffu);
    if (len != 0) {
        br.win <<= len;
        br.nb -= len;
        br.consumed += (uint64_t)len;
        return (int)(e >> 8);
    }
    // canonical search: the codes of length L are first[L] .. first[L]+count[L]-1
    uint64_t c = 0;
    for (int L = 1; L <= maxlen; L++) {
        c = (c << 1) | br.bit_at(L - 1);
        if (L <= T) continue;
        uint64_t first = ((uint64_t)s_tab[65 + L] << 32) | s_tab[L];
        uint32_t cnt = s_tab[130 + L];
        if (cnt && c >= first && c - first < cnt) {
            br.skip(L);
            return (int)g_sorted[s_tab[195 + L] + (uint32_t)(c - first)];
        }
    }
    bad = true;
    br.skip(1);
    return 0;
}

// ---------------------------------------------------------------------------
// The kernel.  ND = 2 (1D/2D fields) or 3; NL = layers; DEC = decompress.
//
// Ring: RD sweeps deep, each sweep slot holds one float4 (a tile of 4
// recorded values) per (plane slot, row slot); plane/row slots 0..NL-1 are
// the "virtual" lines that belong to neighbouring CTAs and are filled by the
// halo warp with cp.async, kPFH sweeps ahead, straight into their slot.
//
// Global halos written by the compute lanes as soon as a tile is done:
//   3D row halo   [P][nb1][NL][tpr]        the last NL rows of each row block
//   3D plane halo [nb0][nb1][NL][32][tpr]  the last NL planes of each plane block
//   2D row halo   [nb1][NL][tpr]
// The corner lines a CTA needs (previous planes x previous rows) come from
// the diagonal CTA's row halo.  Progress counters (sweeps completed) are
// published every g.pub sweeps after a fence.

template <int ND, int NL>
struct Cfg {
    static constexpr int RD = kPFH + (ND == 3 ? 2 * NL : NL) + 1;  // ring depth
    static constexpr int MAXE = (ND == 3) ? (NL * (32 + NL) + NL * kMaxWaveWarps + 31) / 32 : 1;  // entries per halo lane
};

template <int ND, int NL, bool DEC>
__global__ void __launch_bounds__((kMaxWaveWarps + 1) * 32) k_wave(WaveArgs A) {
    extern __shared__ __align__(16) unsigned char smem[];
    using C = Cfg<ND, NL>;
    constexpr int RD = C::RD;
    const WaveGeom& g = A.g;
    const int W = g.W;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const bool is_halo = (warp == W);
    __shared__ unsigned int s_ticket;
    __shared__ int s_abort;

    if (threadIdx.x == 0) {
        s_ticket = atomicAdd(&A.st->ticket, 1u);
        s_abort = 0;
    }
    __syncthreads();
    const int item = (int)s_ticket;
    const int ib = (ND == 3) ? item / g.nb1 : 0;
    const int jb = item % g.nb1;  // row block
    if (A.st->err) {  // an earlier stage failed: publish an aborted state and leave
        if (threadIdx.x == 0) st_release_u32(A.prog + item, kProgAbort);
        return;
    }

    const int NP = (ND == 3) ? (W + NL) : 1;
    const int NR = (ND == 3) ? (32 + NL) : (32 * W + NL);
    const int slotsz = NP * NR;  // float4 entries per ring slot
    float4* ring = reinterpret_cast<float4*>(smem);
    float4* xstage = ring + RD * slotsz;                     // [W][kPFX][32] (compress)
    uint32_t* s_lut = reinterpret_cast<uint32_t*>(xstage);   // (decompress)
    uint32_t* s_tab = s_lut + (1 << kLutBits);

    const int tpr = g.ntiles * kTile;  // halo row length (floats)
    const int r_last = g.nsweeps - 1;  // last compute sweep
    const unsigned final_prog = (unsigned)(r_last + 1);
    unsigned int* my_prog = A.prog + item;
    QParams qp = load_qparams(A.st);

    if (is_halo) {
        // ================= halo warp =================
        const int NE = (ND == 3) ? (NL * (32 + NL) + NL * W) : NL;
        const int row_lag = (ND == 3) ? 33 : (32 * W + 1);
        const int plane_lag = W + 1;
        const int diag_lag = W + 33;
        const unsigned* prog_row = nullptr;
        const unsigned* prog_plane = nullptr;
        const unsigned* prog_diag = nullptr;
        if (ND == 3) {
            if (jb > 0) prog_row = A.prog + ib * g.nb1 + jb - 1;
            if (ib > 0) prog_plane = A.prog + (ib - 1) * g.nb1 + jb;
            if (ib > 0 && jb > 0) prog_diag = A.prog + (ib - 1) * g.nb1 + jb - 1;
        } else if (jb > 0) {
            prog_row = A.prog + jb - 1;
        }
        // per-lane entries: ring offset within a slot, skew, source of tile 0
        int e_off[C::MAXE], e_skew[C::MAXE];
        const float* e_src[C::MAXE];
#pragma unroll
        for (int j = 0; j < C::MAXE; j++) {
            const int e = lane + 32 * j;
            e_off[j] = -1;
            e_skew[j] = 0;
            e_src[j] = nullptr;
            if (e >= NE) continue;
            int wp, rs;
            const float* src = nullptr;
            if (ND == 3) {
                if (e < NL * (32 + NL)) {
                    const int p = e / (32 + NL);
                    wp = p;
                    rs = e % (32 + NL);
                    if (ib > 0) {
                        if (rs >= NL) {
                            size_t off = ((((size_t)(ib - 1) * g.nb1 + jb) * NL + p) * 32 + (rs - NL)) * tpr;
                            src = A.halo_plane + off;
                        } else if (jb > 0) {
                            uint64_t plane = (uint64_t)(ib - 1) * W + W - NL + p;
                            size_t off = (((size_t)plane * g.nb1 + (jb - 1)) * NL + rs) * tpr;
                            src = A.halo_row + off;
                        }
                    }
                } else {
                    const int e2 = e - NL * (32 + NL);
                    const int w = e2 / NL, q = e2 % NL;
                    wp = NL + w;
                    rs = q;
                    const uint64_t plane = (uint64_t)ib * W + w;
                    if (jb > 0 && plane < g.P) {
                        size_t off = (((size_t)plane * g.nb1 + (jb - 1)) * NL + q) * tpr;
                        src = A.halo_row + off;
                    }
                }
            } else {
                wp = 0;
                rs = e;
                if (jb > 0) src = A.halo_row + ((size_t)(jb - 1) * NL + e) * tpr;
            }
            e_off[j] = wp * NR + rs;
            e_skew[j] = (ND == 3) ? (wp - NL) + (rs - NL) : (rs - NL);
            e_src[j] = src;
        }
        bool timed_out = false;
        unsigned seen_row = 0, seen_plane = 0, seen_diag = 0;
        const float* dummy = A.halo_row;  // a valid address for zero-fill copies

        // issue the cp.async loads of the virtual entries of sweep rp into
        // their ring slot, after the producers have published enough progress
        auto issue = [&](int rp) {
            if (lane == 0 && !timed_out) {
                if (prog_row) {
                    unsigned need = min((unsigned)max(rp + row_lag, 0), final_prog);
                    if (!wait_progress(prog_row, need, seen_row, A.timeout_ns)) timed_out = true;
                }
                if (prog_plane && !timed_out) {
                    unsigned need = min((unsigned)max(rp + plane_lag, 0), final_prog);
                    if (!wait_progress(prog_plane, need, seen_plane, A.timeout_ns)) timed_out = true;
                }
                if (prog_diag && !timed_out) {
                    unsigned need = min((unsigned)max(rp + diag_lag, 0), final_prog);
                    if (!wait_progress(prog_diag, need, seen_diag, A.timeout_ns)) timed_out = true;
                }
            }
            timed_out = __shfl_sync(0xffffffffu, timed_out ? 1 : 0, 0) != 0;
            float4* slot = ring + posmod(rp, RD) * slotsz;
#pragma unroll
            for (int j = 0; j < C::MAXE; j++) {
                if (e_off[j] < 0) continue;
                const int c = rp - e_skew[j];
                const bool ok = e_src[j] && !timed_out && c >= 0 && c < g.ntiles;
                cp_async16(slot + e_off[j], ok ? (const void*)(e_src[j] + (size_t)c * kTile) : (const void*)dummy,
                           ok ? 16 : 0);
            }
            cp_async_commit();
        };
        const int min_sweep = (ND == 3) ? -2 * NL : -NL;
        for (int rv = min_sweep; rv < kPFH; rv++) issue(rv);
        cp_async_wait<0>();
        __syncthreads();  // prologue: virtual entries of sweeps < kPFH in place

        for (int r = 0; r <= r_last; r++) {
            if (r > 0 && r % g.pub == 0) {  // sweeps < r are complete: publish
                fence_acq_rel_gpu();
                __syncwarp();
                if (lane == 0) st_release_u32(my_prog, (unsigned)r);
            }
            issue(r + kPFH);
            cp_async_wait<kPFH>();
            if (lane == 0 && timed_out) s_abort = 1;
            __syncthreads();
            if (s_abort) break;
        }
        cp_async_wait<0>();
        fence_acq_rel_gpu();
        __syncwarp();
        if (lane == 0) {
            if (s_abort) {
                atomicOr(&A.st->err, kErrTimeout);
                st_release_u32(my_prog, kProgAbort);
            } else {
                st_release_u32(my_prog, final_prog);
            }
        }
        return;
    }

    // ================= compute warps =================
    uint64_t plane, row;
    int skew, wp_own, rs_own;
    if (ND == 3) {
        plane = (uint64_t)ib * W + warp;
        row = (uint64_t)jb * 32 + lane;
        skew = warp + lane;
        wp_own = warp + NL;
        rs_own = lane + NL;
    } else {
        plane = 0;
        row = (uint64_t)jb * 32 * W + warp * 32 + lane;
        skew = warp * 32 + lane;
        wp_own = 0;
        rs_own = warp * 32 + lane + NL;
    }
    const bool valid = (plane < g.P) && (row < g.M);
    const uint64_t rowid = plane * g.M + row;
    const uint64_t rowbase = rowid * g.N;
    const int own_off = wp_own * NR + rs_own;
    // halo outputs written by this lane (null when the line has no consumer)
    float* hout_row = nullptr;
    float* hout_plane = nullptr;
    if (valid) {
        if (ND == 3) {
            if (lane >= 32 - NL && jb + 1 < g.nb1)
                hout_row = A.halo_row + (((size_t)plane * g.nb1 + jb) * NL + (lane - (32 - NL))) * tpr;
            if (warp >= W - NL && ib + 1 < g.nb0)
                hout_plane = A.halo_plane +
                             ((((size_t)ib * g.nb1 + jb) * NL + (warp - (W - NL))) * 32 + lane) * tpr;
        } else {
            if (warp == W - 1 && lane >= 32 - NL && jb + 1 < g.nb1)
                hout_row = A.halo_row + ((size_t)jb * NL + (lane - (32 - NL))) * tpr;
        }
    }

    // tails: the last NL values of the previous tile of every series
    float tail[NL + 1][NL + 1][NL];
#pragma unroll
    for (int a = 0; a <= NL; a++)
#pragma unroll
        for (int b = 0; b <= NL; b++)
#pragma unroll
            for (int j = 0; j < NL; j++) tail[a][b][j] = 0.0f;

    BitReader br;
    int T = 1, maxlen = 1;
    bool bad = false;
    uint64_t rowbits_avail = 0;
    if constexpr (DEC) {
        T = (int)A.st->lut_bits;
        maxlen = (int)A.st->maxlen;
        const int nthr = W * 32;
        for (int i = threadIdx.x; i < (1 << T); i += nthr) s_lut[i] = A.lut[i];
        for (int i = threadIdx.x; i < 260; i += nthr) s_tab[i] = A.dectab[i];
        asm volatile("bar.sync 1, %0;" ::"r"(nthr));
        if (valid) {
            uint64_t off = A.rowoff[rowid];
            rowbits_avail = (uint64_t)A.rowbytes[rowid] * 8;
            br.init(A.payload, off, (uint64_t)(A.stream_end - A.payload));
        }
    }
    const uint16_t* g_sorted = reinterpret_cast<const uint16_t*>(A.dectab + 260);

    float4* xs = xstage + warp * kPFX * 32 + lane;
    const float* xrow = A.x + rowbase;
    auto x_prefetch = [&](int rp) {
        if constexpr (!DEC) {
            const int c = rp - skew;
            float4* dst = xs + (rp % kPFX) * 32;
            const bool ok = valid && c >= 0 && c < g.ntiles;
            if (g.aligned) {
                const uint64_t col = (uint64_t)c * kTile;
                cp_async16(dst, ok ? (const void*)(xrow + col) : (const void*)A.x, ok ? 16 : 0);
            } else {
                float* d = reinterpret_cast<float*>(dst);
#pragma unroll
                for (int k = 0; k < kTile; k++) {
                    const uint64_t col = (uint64_t)c * kTile + k;
                    const bool in = ok && col < g.N;
                    cp_async4(d + k, in ? (const void*)(xrow + col) : (const void*)A.x, in ? 4 : 0);
                }
            }
            cp_async_commit();
        }
    };
    if constexpr (!DEC) {
        for (int rp = 0; rp < kPFX - 1; rp++) x_prefetch(rp);
    }
    __syncthreads();  // matches the halo warp's prologue barrier

    for (int r = 0; r <= r_last; r++) {
        if constexpr (!DEC) {
            x_prefetch(r + kPFX - 1);
            cp_async_wait<kPFX - 1>();
        }
        const int c = r - skew;
        if (c >= 0 && c < g.ntiles) {
            // neighbour series of this tile: tails + the ring entries written
            // a + b sweeps ago by the lane at (plane - a, row - b)
            float S[NL + 1][NL + 1][NL + kTile];
#pragma unroll
            for (int a = 0; a <= NL; a++)
#pragma unroll
                for (int b = 0; b <= NL; b++) {
#pragma unroll
                    for (int j = 0; j < NL; j++) S[a][b][j] = tail[a][b][j];
                    if ((ND != 3 && a > 0) || (a == 0 && b == 0)) {
#pragma unroll
                        for (int k = 0; k < kTile; k++) S[a][b][NL + k] = 0.0f;
                        continue;
                    }
                    const float4 v = ring[posmod(r - a - b, RD) * slotsz + own_off - a * NR - b];
                    S[a][b][NL + 0] = v.x;
                    S[a][b][NL + 1] = v.y;
                    S[a][b][NL + 2] = v.z;
                    S[a][b][NL + 3] = v.w;
                }
            // partial predictions: every term except the own-line ones,
            // summed in the method's order (they precede the own-line terms)
            float part[kTile];
#pragma unroll
            for (int k = 0; k < kTile; k++) part[k] = predict_partial<NL, ND>(S, k);
            int code[kTile];
            if constexpr (!DEC) {
                const float4 xv4 = xs[(r % kPFX) * 32];
                const float xv[kTile] = {xv4.x, xv4.y, xv4.z, xv4.w};
                float tr[kTile];
#pragma unroll
                for (int k = 0; k < kTile; k++) tr[k] = trunc_value(xv[k], qp.e_eb);
#pragma unroll
                for (int k = 0; k < kTile; k++) {
                    const float pred = predict_own<NL, ND>(part[k], S, k);
                    float V;
                    code[k] = quantize_tr(xv[k], pred, tr[k], qp, V);
                    S[0][0][NL + k] = V;
                }
            } else {
                float uv[kTile];
                const uint64_t col0 = (uint64_t)c * kTile;
#pragma unroll
                for (int k = 0; k < kTile; k++) {
                    code[k] = 0;
                    uv[k] = 0.0f;
                    if (valid && col0 + k < g.N) {
                        int sym = decode_symbol(br, s_lut, T, s_tab, g_sorted, maxlen, bad);
                        code[k] = sym;
                        if (sym == 0) {
                            uint32_t se = br.take(9);
                            int t = trunc_bits(se << 23, qp.e_eb);
                            uint32_t mb = br.take(t);
                            uv[k] = __uint_as_float((se << 23) | (t ? (mb << (23 - t)) : 0u));
                        }
                    }
                }
#pragma unroll
                for (int k = 0; k < kTile; k++) {
                    const float pred = predict_own<NL, ND>(part[k], S, k);
                    S[0][0][NL + k] = code[k] ? dequantize(code[k], pred, qp) : uv[k];
                }
            }
            const float4 vout = make_float4(S[0][0][NL], S[0][0][NL + 1], S[0][0][NL + 2], S[0][0][NL + 3]);
            ring[(r % RD) * slotsz + own_off] = vout;
            if (hout_row) *reinterpret_cast<float4*>(hout_row + (size_t)c * kTile) = vout;
            if (ND == 3 && hout_plane) *reinterpret_cast<float4*>(hout_plane + (size_t)c * kTile) = vout;
#pragma unroll
            for (int a = 0; a <= NL; a++)
#pragma unroll
                for (int b = 0; b <= NL; b++)
#pragma unroll
                    for (int j = 0; j < NL; j++) tail[a][b][j] = S[a][b][kTile + j];
            if (valid) {
                const uint64_t col = (uint64_t)c * kTile;
                const bool full = g.aligned && (col + kTile <= g.N);
                if constexpr (!DEC) {
                    if (full) {
                        uint2 pk;
                        pk.x = (uint32_t)code[0] | ((uint32_t)code[1] << 16);
                        pk.y = (uint32_t)code[2] | ((uint32_t)code[3] << 16);
                        *reinterpret_cast<uint2*>(A.codes + rowbase + col) = pk;
                        if (A.recorded) *reinterpret_cast<float4*>(A.recorded + rowbase + col) = vout;
                    } else {
                        const float vv[kTile] = {vout.x, vout.y, vout.z, vout.w};
#pragma unroll
                        for (int k = 0; k < kTile; k++)
                            if (col + k < g.N) {
                                A.codes[rowbase + col + k] = (uint16_t)code[k];
                                if (A.recorded) A.recorded[rowbase + col + k] = vv[k];
                            }
                    }
                } else {
                    if (full) {
                        *reinterpret_cast<float4*>(A.out + rowbase + col) = vout;
                    } else {
                        const float vv[kTile] = {vout.x, vout.y, vout.z, vout.w};
#pragma unroll
                        for (int k = 0; k < kTile; k++)
                            if (col + k < g.N) A.out[rowbase + col + k] = vv[k];
                    }
                }
            }
        }
        __syncthreads();
        if (s_abort) break;
    }
    if constexpr (!DEC) cp_async_wait<0>();
    if constexpr (DEC) {
        if (valid && (bad || br.consumed > rowbits_avail)) atomicOr(&A.st->err, kErrCorrupt);
    }
}

// ---------------------------------------------------------------------------
// host side

size_t wave_smem_bytes(const WaveGeom& g, int layers, bool decompress) {
    const int NL = layers, W = g.W;
    int RD, NP, NR;
    if (g.ndim == 3) {
        RD = kPFH + 2 * NL + 1; NP = W + NL; NR = 32 + NL;
    } else {
        RD = kPFH + NL + 1; NP = 1; NR = 32 * W + NL;
    }
    size_t b = (size_t)RD * NP * NR * 16;
    if (decompress) b += (size_t)(1 << kLutBits) * 4 + 260 * 4;
    else b += (size_t)W * kPFX * 32 * 16;
    return b;
}

template <int ND, int NL, bool DEC>
static int launch_t(const WaveArgs& a, cudaStream_t s) {
    size_t smem = wave_smem_bytes(a.g, NL, DEC);
    auto fn = k_wave<ND, NL, DEC>;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return SZGB_ECUDA;
    fn<<<a.g.num_ctas, (a.g.W + 1) * 32, smem, s>>>(a);
    return cudaGetLastError() == cudaSuccess ? 0 : SZGB_ECUDA;
}

template <bool DEC>
static int launch_any(const WaveArgs& a, int layers, cudaStream_t s) {
    if (a.g.ndim == 3) return layers == 1 ? launch_t<3, 1, DEC>(a, s) : launch_t<3, 2, DEC>(a, s);
    if (a.g.ndim == 2) return layers == 1 ? launch_t<2, 1, DEC>(a, s) : launch_t<2, 2, DEC>(a, s);
    return layers == 1 ? launch_t<1, 1, DEC>(a, s) : launch_t<1, 2, DEC>(a, s);
}

int launch_wave_compress(const WaveGeom& g, int layers, const float* x, uint16_t* codes,
                         float* recorded, float* halo_row, float* halo_plane, unsigned int* prog,
                         DevState* st, uint64_t timeout_ns, cudaStream_t s) {
    WaveArgs a = {};
    a.g = g;
    a.x = x;
    a.codes = codes;
    a.recorded = recorded;
    a.halo_row = halo_row;
    a.halo_plane = halo_plane;
    a.prog = prog;
    a.st = st;
    a.timeout_ns = timeout_ns;
    return launch_any<false>(a, layers, s);
}

int launch_wave_decompress(const WaveGeom& g, int layers, const uint8_t* payload,
                           const uint64_t* rowoff, const uint32_t* rowbytes,
                           const uint8_t* stream_end, const uint32_t* lut,
                           const uint32_t* dec_tab, float* out, float* halo_row,
                           float* halo_plane, unsigned int* prog, DevState* st,
                           uint64_t timeout_ns, cudaStream_t s) {
    WaveArgs a = {};
    a.g = g;
    a.payload = payload;
    a.rowoff = rowoff;
    a.rowbytes = rowbytes;
    a.stream_end = stream_end;
    a.lut = lut;
    a.dectab = dec_tab;
    a.out = out;
    a.halo_row = halo_row;
    a.halo_plane = halo_plane;
    a.prog = prog;
    a.st = st;
    a.timeout_ns = timeout_ns;
    return launch_any<true>(a, layers, s);
}

}  // namespace szgb
