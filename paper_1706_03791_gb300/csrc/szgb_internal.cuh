// szgb_internal.cuh -- shared definitions of the GB300 compressor library.
//
// Device-side state of one compress/decompress call, the per-point
// arithmetic of the method (prediction terms, error-controlled quantization,
// truncated representation of unpredictable values) and small PTX helpers.
// All float arithmetic on the data path uses explicit round-to-nearest
// intrinsics (__fadd_rn, __fmul_rn, ...) so that no FMA contraction can
// change a bit.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/szgb.h"

namespace szgb {

constexpr int kHeaderBytes = 128;
constexpr int kTile = 4;           // columns per sweep and lane (one float4)
constexpr int kMaxLayers = 4;      // n supported by the GPU kernels in 1D, 2D and 3D
constexpr int kMaxLayers3D = 2;    // n the 3D wavefront carries (a lane keeps (n+1)^3 - 1 values)
// layer counts the wavefront kernels (single, batched, no-allocation) carry
__host__ __device__ inline bool layers_supported(int ndim, int layers) {
    return layers >= 1 && layers <= (ndim == 3 ? kMaxLayers3D : kMaxLayers);
}
constexpr int kLutBits = 11;       // decoder lookup-table index bits
constexpr int kMaxWaveWarps = 8;   // compute warps per wavefront CTA (plus one halo warp)
constexpr uint32_t kProgAbort = 0x7fffffffu;

// Error flags raised on the device (DevState::err bitmask).
constexpr uint32_t kErrTimeout = 1u;
constexpr uint32_t kErrCorrupt = 2u;
constexpr uint32_t kErrNonFinite = 4u;
constexpr uint32_t kErrOverflow = 8u;   // stream does not fit in the output
constexpr uint32_t kErrRange = 16u;     // lattice variant: eb_f = 0 or lattice integers >= 2^30

// State of one call, in device memory (zeroed before the call).
struct DevState {
    // range (K1)
    unsigned int nonfinite;
    unsigned int range_blocks_done;
    float xmin, xmax;
    // bound and quantizer parameters
    float eb_f, twoeb, inv2eb, radius;
    int m, center, e_eb, adaptive;
    // adaptive m (K8)
    unsigned long long need[18];
    unsigned long long nsamples;
    unsigned int adapt_blocks_done;
    // wavefront scheduling
    unsigned int ticket;
    unsigned int err;
    // Huffman
    unsigned int nsym, maxlen;
    unsigned long long K;
    unsigned int maxrow;
    unsigned int table_width;
    unsigned long long cb_bytes, tab_bytes, payload, total, cap;
    unsigned int fits;
    unsigned int scan_blocks;
    // decoder
    unsigned int lut_bits;
};

// Parameters of a call that the host knows before launching.
struct CallParams {
    int ndim;
    uint64_t d0, d1, d2;     // extents, slowest -> fastest (leading 1s)
    int mode;
    double eb_abs, eb_rel;
    int layers;
    int m_user;              // 0 = adaptive
    double theta;
    int variant;             // 0 = the paper's method, 1 = the lattice variant
    uint32_t chunk;          // Huffman chunk length along a row: 0 = the whole
                             // row, else a power of two >= 32 below the row length
    uint64_t D4;             // 4D field D4 x P x M x N: D4, with d0 = D4 P
                             // (the (D4 P) x M x N view); 0 for 1D-3D
};

// chunks per row of a field whose rows hold `row_len` points
__host__ __device__ inline uint64_t chunks_per_row(uint32_t chunk, uint64_t row_len) {
    return chunk ? (row_len + chunk - 1) / chunk : 1;
}

// --------------------------------------------------------------------------
// prediction terms: k in [0,n]^3 \ {0} in descending lexicographic order with
// coefficient -prod_j (-1)^k_j C(n,k_j)  (Eq. predmodel; summation order R2)

// Iterative (not recursive) so that, with constant arguments after loop
// unrolling, the compiler folds it to a literal instead of emitting a call.
__host__ __device__ __forceinline__ constexpr int binom_c(int n, int k) {
    if (k < 0 || k > n) return 0;
    int r = 1;
    for (int i = 1; i <= k; i++) r = r * (n - i + 1) / i;
    return r;
}
__host__ __device__ __forceinline__ constexpr int sgn_binom(int n, int k) { return ((k & 1) ? -1 : 1) * binom_c(n, k); }
__host__ __device__ __forceinline__ constexpr int term_coef(int n, int k0, int k1, int k2) {
    return -sgn_binom(n, k0) * sgn_binom(n, k1) * sgn_binom(n, k2);
}

// --------------------------------------------------------------------------
// quantizer parameters in registers
struct QParams {
    float eb, twoeb, inv, radius;
    int center, e_eb;
};

__device__ __forceinline__ QParams load_qparams(const DevState* st) {
    QParams q;
    q.eb = st->eb_f;
    q.twoeb = st->twoeb;
    q.inv = st->inv2eb;
    q.radius = st->radius;
    q.center = st->center;
    q.e_eb = st->e_eb;
    return q;
}

// number of mantissa bits kept for an unpredictable value (R5)
__host__ __device__ __forceinline__ int trunc_bits(uint32_t u, int e_eb) {
    if (e_eb == 0) return 23;
    int e = (int)((u >> 23) & 0xffu);
    e = e < 1 ? 1 : e;
    int t = e - e_eb;
    t = t < 0 ? 0 : t;
    return t > 23 ? 23 : t;
}

__device__ __forceinline__ float trunc_value(float x, int e_eb) {
    uint32_t u = __float_as_uint(x);
    int t = trunc_bits(u, e_eb);
    return __uint_as_float(u & ~((1u << (23 - t)) - 1u));
}

// Error-controlled quantization of one value (Sec. IV-A).  Returns the code
// (0 = unpredictable) and sets V to the value recorded for later predictions.
// q + 0.0f equals (float)(int)q for the integral |q| <= radius and maps -0.0
// to +0.0, matching a reconstruction from the integer code.
__device__ __forceinline__ int quantize(float x, float pred, const QParams& qp, float& V) {
    float diff = __fsub_rn(x, pred);
    float q = rintf(__fmul_rn(diff, qp.inv));
    bool ok = fabsf(q) <= qp.radius;
    float qn = __fadd_rn(q, 0.0f);
    float dq = __fadd_rn(pred, __fmul_rn(qn, qp.twoeb));
    float err = __fsub_rn(x, dq);
    ok = ok && ((fabsf(err) < qp.eb) || (x == dq));
    V = ok ? dq : trunc_value(x, qp.e_eb);
    return ok ? ((int)qn + qp.center) : 0;
}

// As quantize, with the truncated representation of x computed beforehand
// (it does not depend on the prediction, so it stays off the dependency chain).
__device__ __forceinline__ int quantize_tr(float x, float pred, float tr, const QParams& qp, float& V) {
    const float diff = __fsub_rn(x, pred);
    const float q = rintf(__fmul_rn(diff, qp.inv));
    const float qn = __fadd_rn(q, 0.0f);
    const float dq = __fadd_rn(pred, __fmul_rn(qn, qp.twoeb));
    const float err = __fsub_rn(x, dq);
    const bool ok = (fabsf(q) <= qp.radius) & ((fabsf(err) < qp.eb) | (x == dq));
    V = ok ? dq : tr;
    return ok ? ((int)qn + qp.center) : 0;
}

// Reconstruction of a predictable value from its code.
__device__ __forceinline__ float dequantize(int code, float pred, const QParams& qp) {
    float qf = (float)(code - qp.center);
    return __fadd_rn(pred, __fmul_rn(qf, qp.twoeb));
}

// --------------------------------------------------------------------------
// PTX helpers

__device__ __forceinline__ unsigned int ld_acquire_u32(const unsigned int* p) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_u32(unsigned int* p, unsigned int v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint64_t globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
// 16-byte asynchronous global->shared copy, zero-filling when src_bytes < 16
__device__ __forceinline__ void cp_async16(void* dst, const void* src, int src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_addr(dst)), "l"(src),
                 "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async4(void* dst, const void* src, int src_bytes) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(smem_addr(dst)), "l"(src),
                 "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// mbarrier (shared memory, CTA scope)
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_inval(uint64_t* bar) {
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait for the phase with the given parity; false on timeout.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity, uint64_t timeout_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer();
    for (unsigned it = 0; it < (1u << 26); it++) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 15) == 15 && globaltimer() - t0 > timeout_ns) return false;
    }
    return false;
}
// TMA: 3D tiled tensor load (global -> shared, completes on an mbarrier) and
// store (shared -> global, bulk async-group); coordinates are element
// indices, fastest first.
__device__ __forceinline__ void tma_load_3d(void* dst, const void* tmap, int c0, int c1, int c2, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(smem_addr(dst)), "l"(tmap), "r"(c0), "r"(c1), "r"(c2), "r"(smem_addr(bar))
        : "memory");
}
__device__ __forceinline__ void tma_store_3d(const void* tmap, int c0, int c1, int c2, const void* src) {
    asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.tile.bulk_group [%0, {%1, %2, %3}], [%4];"
                 ::"l"(tmap), "r"(c0), "r"(c1), "r"(c2), "r"(smem_addr(src))
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void bulk_wait_read() {
    asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory");
}
template <int N>
__device__ __forceinline__ void bulk_wait() {
    asm volatile("cp.async.bulk.wait_group %0;" ::"n"(N) : "memory");
}
// orders this thread's generic-proxy shared-memory writes before later
// async-proxy (TMA) reads of them
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void prefetch_tmap(const void* tmap) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(tmap) : "memory");
}

// named CTA barriers (producer/consumer: one side arrives, the other syncs)
__device__ __forceinline__ void named_bar_sync(int id, int nthreads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}
__device__ __forceinline__ void named_bar_arrive(int id, int nthreads) {
    asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// predicated 32-bit shared-memory store (shared-window address)
__device__ __forceinline__ void st_shared_f32_if(bool p, uint32_t addr, float v) {
    asm volatile("{\n .reg .pred q;\n setp.ne.u32 q, %0, 0;\n @q st.shared.f32 [%1], %2;\n}" ::"r"((unsigned)p),
                 "r"(addr), "f"(v));
}

__device__ __forceinline__ uint32_t bswap32(uint32_t v) { return __byte_perm(v, 0, 0x0123); }

// ---------------------------------------------------------------------------
// Per-lane bit reader over one row chunk (MSB-first), for decompression.
// (used by the row decoders of both variants)

struct BitReader {
    const uint8_t* base;
    uint64_t wpos;       // byte offset of the next word to load (multiple of 4)
    uint64_t endoff;     // bytes available from base
    uint64_t win;        // valid bits, MSB aligned
    int nb;              // valid bits in win
    uint32_t pf0, pf1;   // the next two words, raw (as loaded, little-endian), at wpos - 8 and wpos - 4
    uint64_t start;      // byte offset of the first bit

    // A prefetch is a plain predicated load into its register: the byte order
    // is fixed only when the word enters the window, so the load is waited
    // for two refills after it was issued, not at once.
    __device__ __forceinline__ uint32_t load_raw(uint64_t off) const {
        uint32_t v = 0;
        if (off + 4 <= endoff) v = __ldg(reinterpret_cast<const uint32_t*>(base + off));
        return v;
    }
    // big-endian value of the word at off from its raw load (the last,
    // partial word of the stream is read byte by byte)
    __device__ __forceinline__ uint32_t word(uint64_t off, uint32_t raw) const {
        if (off + 4 <= endoff) return bswap32(raw);
        uint32_t v = 0;
        for (int i = 0; i < 4; i++) v = (v << 8) | (off + i < endoff ? (uint32_t)base[off + i] : 0u);
        return v;
    }
    __device__ __forceinline__ uint32_t load_word(uint64_t off) const { return word(off, load_raw(off)); }
    __device__ __forceinline__ void init(const uint8_t* b, uint64_t start, uint64_t end) {
        base = b;
        endoff = end;
        uint64_t a = start & ~(uint64_t)3;
        int skip = (int)(start - a) * 8;
        uint32_t w0 = load_word(a);
        pf0 = load_raw(a + 4);
        pf1 = load_raw(a + 8);
        wpos = a + 12;
        win = ((uint64_t)w0 << 32) << skip;
        nb = 32 - skip;
        this->start = start;
    }
    // bits consumed since init: those that entered the window, less the
    // ones still in it
    __device__ __forceinline__ uint64_t consumed() const { return 8 * (wpos - 8 - start) - (uint64_t)nb; }
    // top the window up to more than 32 valid bits
    __device__ __forceinline__ void refill() {
        if (nb <= 32) {
            win |= (uint64_t)word(wpos - 8, pf0) << (32 - nb);
            nb += 32;
            pf0 = pf1;
            pf1 = load_raw(wpos);
            wpos += 4;
        }
    }
    // bit p (0 = next bit) looking past the window into the prefetched words
    __device__ __forceinline__ uint32_t bit_at(int p) const {
        if (p < nb) return (uint32_t)(win >> (63 - p)) & 1u;
        p -= nb;
        if (p < 32) return (word(wpos - 8, pf0) >> (31 - p)) & 1u;
        p -= 32;
        return (word(wpos - 4, pf1) >> (31 - p)) & 1u;
    }
    __device__ __forceinline__ void skip(int n) {
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
        return v;
    }
};

// decode one quantization code; long codes (> lut bits) by canonical search
// (T = 0: no lookup table, canonical search only)
__device__ __forceinline__ int decode_symbol(BitReader& br, const uint32_t* s_lut, int T,
                                             const uint32_t* s_tab, const uint16_t* g_sorted,
                                             int maxlen, bool& bad) {
    br.refill();
    if (T > 0) {
        uint32_t e = s_lut[(uint32_t)(br.win >> (64 - T))];
        int len = (int)(e & 0xffu);
        if (len != 0) {
            br.win <<= len;
            br.nb -= len;
            return (int)(e >> 8);
        }
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

// --------------------------------------------------------------------------
// the lattice variant (a separately labelled, fully parallel form; see
// k_lattice.cu): lattice integer of x, p = rint(x * inv) in binary32 with
// inv = 1 / (2 eb_f), and whether v = (float)p * 2 eb_f is within the bound
// (|x - v| < eb_f or x == v)
__device__ __forceinline__ int32_t lattice_point(float x, float inv, float twoeb, float eb, bool& ok) {
    const int32_t p = (int32_t)rintf(__fmul_rn(x, inv));
    const float v = __fmul_rn(__int2float_rn(p), twoeb);
    ok = (fabsf(__fsub_rn(x, v)) < eb) | (x == v);
    return p;
}
__device__ __forceinline__ float lattice_value(int32_t p, float twoeb) { return __fmul_rn(__int2float_rn(p), twoeb); }

// integer residual p - sum_k c_k p(x - k) of the n-layer predictor over the
// lattice integers P ([d0][d1][d2]), neighbours outside the domain = 0
template <int ND, int NL>
__device__ __forceinline__ int64_t lattice_resid(const int32_t* __restrict__ P, uint64_t d1, uint64_t d2, int64_t i,
                                                 int64_t j, int64_t l) {
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
                pred += (int64_t)term_coef(NL, k0, k1, k2) * (int64_t)P[((uint64_t)ii * d1 + (uint64_t)jj) * d2 + (uint64_t)ll];
            }
        }
    }
    return (int64_t)P[((uint64_t)i * d1 + (uint64_t)j) * d2 + (uint64_t)l] - pred;
}

__device__ __forceinline__ int64_t lattice_resid_rt(const int32_t* P, int ndim, int layers, uint64_t d1, uint64_t d2,
                                                    int64_t i, int64_t j, int64_t l) {
    if (ndim == 3) return layers == 1 ? lattice_resid<3, 1>(P, d1, d2, i, j, l) : lattice_resid<3, 2>(P, d1, d2, i, j, l);
    if (ndim == 2) return layers == 1 ? lattice_resid<2, 1>(P, d1, d2, i, j, l) : lattice_resid<2, 2>(P, d1, d2, i, j, l);
    return layers == 1 ? lattice_resid<1, 1>(P, d1, d2, i, j, l) : lattice_resid<1, 2>(P, d1, d2, i, j, l);
}

// --------------------------------------------------------------------------
// geometry of the wavefront launch (host-computed, passed by value)
struct WaveGeom {
    int ndim;             // 1 and 2 use the row topology, 3 the plane x row one
    uint64_t P, M, N;     // extents (planes, rows, columns)
    int ntiles;           // ceil(N / kTile)
    int W;                // compute warps per CTA
    int nb0, nb1;         // CTA grid: 3D (plane blocks, row blocks); 2D (1, row blocks)
    int nsweeps;          // sweeps per CTA including the final flush sweep
    int aligned;          // rows start on 16-byte boundaries (N % 4 == 0)
    int num_ctas;
    int debug_skip;       // test hook: 1 + the work item that is never run
                          // (its consumers' bounded waits run out); 0 = none
};

// Wavefront geometry of a field for a given number of compute warps per CTA
// in 1D/2D (W2) and 3D (W3); any valid geometry gives the same values.
WaveGeom make_geom_w(const CallParams& cp, int layers, int W2, int W3);
// Halo line sizes of a wavefront launch in 32-bit units (every value travels
// as one 64-bit tagged word; the plane halo follows the row halo).
void halo_sizes(const WaveGeom& g, int layers, size_t* row_words, size_t* plane_words);

// Stream header fields (little-endian, 128 bytes; the layout is listed with
// the stream format in the library's header file).
struct Header {
    int ndim, layers, m, mode, maxlen, tw;
    uint64_t d0, d1, d2;
    double eb_abs, eb_rel, theta;
    float eb_f, xmin, xmax;
    uint32_t nsym;
    uint64_t nchunks, K, payload, total;
    int adaptive;
    int variant;
    uint32_t chunk;  // chunk length along a row (byte 116); 0 = whole rows
    uint64_t D4;     // 4D stream (ndim 4 at byte 8): the slowest extent (byte
                     // 120), with ndim = 3 and d0 = D4 P describing the
                     // (D4 P) x M x N view its rows are coded in; else 0
};
// Parses and checks a header held in host memory (a 4D one as its 3D view,
// with D4 set); SZGB_ECORRUPT for an inconsistent one.
int parse_header(const uint8_t* h, size_t in_len, Header* o);
// Fields the wavefront kernels carry (the persistent kernel of the single,
// batched and no-allocation calls): the paper's method, 1D-3D, the
// wavefront's layer counts.  The rest (3D n = 3, 4; 4D; the lattice
// variant) run on their own kernels through the single-field path.
inline bool wave_carries(const CallParams& cp) {
    return cp.variant == 0 && cp.D4 == 0 && layers_supported(cp.ndim, cp.layers);
}
inline bool wave_carries(const Header& h) {
    return h.variant == 0 && h.D4 == 0 && layers_supported(h.ndim, h.layers);
}
// The SZGB_E* code of the error flags a call left in its device state.
int dev_errors(const DevState& s);

// host launchers (each in its own translation unit)
int launch_range(const float* x, uint64_t n, DevState* st, const CallParams& cp, float* partials,
                 int nblocks, cudaStream_t s);
int launch_adapt(const float* x, const CallParams& cp, DevState* st, cudaStream_t s);
// 3D fields with n = 3, 4 layers, one launch per hyperplane (k_hyper.cu)
int launch_hyper_compress(int layers, const float* x, float* V, uint16_t* codes, uint64_t cpitch, uint64_t P,
                          uint64_t M, uint64_t N, const DevState* st, cudaStream_t s);
int launch_hyper_decompress(int layers, uint16_t* codes, uint64_t cpitch, float* out, uint64_t P, uint64_t M,
                            uint64_t N, const DevState* st, cudaStream_t s);
// 4D fields D x P x M x N (k_hyper.cu): hyperplane compression (dec = false)
// or reconstruction (dec = true), adaptive m, and the header's 4D fields
int launch_hyper4(bool dec, int layers, const float* x, float* V, uint16_t* codes, uint64_t cpitch, uint64_t D,
                  uint64_t P, uint64_t M, uint64_t N, const DevState* st, cudaStream_t s);
int launch_adapt4(const float* x, uint64_t D, uint64_t P, uint64_t M, uint64_t N, int layers, double theta,
                  DevState* st, cudaStream_t s);
int launch_patch_header4(uint8_t* header, uint64_t D, uint64_t P, const DevState* st, cudaStream_t s);
int launch_hits4(const float* x, const float* V, uint64_t D, uint64_t P, uint64_t M, uint64_t N, int layers,
                 double eb, unsigned long long* count, int sm_count, cudaStream_t s);
// prediction hits |x - f(V)| <= eb over a d0 x d1 x d2 field, added to *count
int launch_hits(const float* x, const float* V, uint64_t d0, uint64_t d1, uint64_t d2, int ndim, int layers,
                double eb, unsigned long long* count, int sm_count, cudaStream_t s);
// rows of x (N floats each) copied to xp at row pitch P (k_range.cu)
int launch_pitch_rows(const float* x, uint64_t rows, uint64_t N, float* xp, uint64_t P, int sm_count, cudaStream_t s);
// x: the input with row pitch x_pitch (N, or N rounded up to 4 when the rows
// were staged by launch_pitch_rows)
int launch_wave_compress(const WaveGeom& g, int layers, const float* x, uint64_t x_pitch, uint16_t* codes,
                         uint64_t codes_pitch, float* recorded, float* halo_row, float* halo_plane, unsigned int* prog,
                         DevState* st, uint64_t timeout_ns, cudaStream_t s);
// decompression: rows decoded first (codes into a row-pitched array, the
// values of unpredictable points into `out`), then the reconstruction wavefront
// the lattice variant (k_lattice.cu)
int launch_lattice_compress(const float* x, const CallParams& cp, int32_t* P, uint8_t* OK, uint16_t* codes,
                            uint64_t cpitch, float* recorded, DevState* st, cudaStream_t s);
int launch_lattice_decompress(const uint8_t* payload, const uint64_t* rowoff, const uint32_t* rowbytes,
                              const uint8_t* stream_end, const uint32_t* lut, const uint32_t* dec_tab, int ndim,
                              int layers, uint64_t d0, uint64_t d1, uint64_t d2, int32_t* R, uint8_t* EX, float* out,
                              DevState* st, cudaStream_t s);
// reconstruction quality: per-block partial sums and their total (k_quality.cu)
size_t quality_scratch_bytes(int blocks);
int quality_blocks(uint64_t n, int sm_count);
int launch_quality(const float* x, const float* y, uint64_t n, int blocks, void* scratch, double* host_out,
                   cudaStream_t s);
// batched codebook build and decoder tables: one CTA per field, arguments
// in a device table of *_args_bytes() records filled by *_args_fill
size_t codebook_args_bytes();
void codebook_args_fill(void* dst, const uint32_t* hist, DevState* st, uint8_t* len, uint64_t* cw, uint64_t* sortbuf,
                        uint32_t* nodebuf);
int launch_codebook_batch(const void* args_dev, int count, cudaStream_t s);
size_t tables_args_bytes();
void tables_args_fill(void* dst, const uint8_t* codebook, uint32_t nsym, int m, uint32_t* lut, uint32_t* dec_tab,
                      uint8_t* lenbuf, uint32_t* symbuf, DevState* st);
int launch_decode_tables_batch(const void* args_dev, int count, cudaStream_t s);
// batched row decode: a table of per-field arguments (decode_args_fill, one
// decode_args_bytes() record per field) and the prefix of per-field block
// counts (decode_rows_blocks), count + 1 entries, in device memory
size_t decode_args_bytes();
// (chunk = 0: one chunk per row; rowoff / rowbytes indexed row by row, then
// chunk by chunk)
uint32_t decode_rows_blocks(uint64_t rows, uint32_t chunk, uint64_t N);
void decode_args_fill(void* dst, const uint8_t* payload, const uint64_t* rowoff, const uint32_t* rowbytes,
                      const uint8_t* stream_end, const uint32_t* lut, const uint32_t* dec_tab, uint16_t* codes,
                      uint64_t cpitch, float* out, uint64_t rows, uint64_t N, uint32_t chunk, DevState* st);
int launch_decode_rows_batch(const void* args_dev, const uint32_t* blk_dev, int count, uint32_t total_blocks,
                             cudaStream_t s);
int launch_decode_rows(const uint8_t* payload, const uint64_t* rowoff, const uint32_t* rowbytes,
                       const uint8_t* stream_end, const uint32_t* lut, const uint32_t* dec_tab, uint16_t* codes,
                       uint64_t cpitch, float* out, uint64_t rows, uint64_t N, uint32_t chunk, DevState* st,
                       cudaStream_t s);
int launch_wave_decompress(const WaveGeom& g, int layers, const uint16_t* codes, uint64_t codes_pitch, float* out,
                           float* halo_row, float* halo_plane, unsigned int* prog, DevState* st,
                           uint64_t timeout_ns, cudaStream_t s);
size_t wave_smem_bytes(const WaveGeom& g, int layers, bool decompress);
// batched wavefront: a device table of per-field arguments (filled on the
// host, wave_args_bytes() each, 64-byte aligned) and a (field, item) order
size_t wave_args_bytes();
void wave_args_compress(void* dst, const WaveGeom& g, const float* x, uint64_t x_pitch, uint16_t* codes,
                        uint64_t codes_pitch, float* halo_row, float* halo_plane, unsigned int* prog, DevState* st,
                        uint64_t timeout_ns);
int wave_args_decompress(void* dst, const WaveGeom& g, const uint16_t* codes, uint64_t codes_pitch, float* out,
                         float* halo_row, float* halo_plane, unsigned int* prog, DevState* st, uint64_t timeout_ns);
int launch_wave_batch(const void* args_dev, const void* order_dev, unsigned total, unsigned* ticket_dev, int layers,
                      bool decompress, size_t smem, int grid, cudaStream_t s);

// Huffman / stream kernels (k_huff.cu)
int launch_histogram(const uint16_t* codes, uint64_t rows, uint64_t rowlen, uint64_t pitch, uint32_t* hist,
                     DevState* st, cudaStream_t s);
int launch_codebook(const uint32_t* hist, DevState* st, uint8_t* len, uint64_t* cw, uint64_t* sortbuf,
                    uint32_t* nodebuf, cudaStream_t s);
// per-chunk byte lengths (chunk = 0: one chunk per row), row by row
int launch_rowbits(const uint16_t* codes, uint64_t pitch, const float* x, uint64_t rows, uint64_t rowlen,
                   uint32_t chunk, const uint8_t* len, uint32_t* rowbytes, DevState* st, cudaStream_t s,
                   const uint8_t* OK = nullptr);
// exclusive scan of the chunk byte counts into offsets; with `table` (the
// stream's chunk table, entries of `width` bytes) the counts are read from it
// and stored in rowbytes (which is then written, not read)
int launch_scan_rows(const uint32_t* rowbytes, uint64_t rows, uint64_t* rowoff, uint64_t* blocksums,
                     DevState* st, int finalize_compress, cudaStream_t s, const uint8_t* table = nullptr,
                     int width = 0);
// header (chunk length cp.chunk at byte 116), codebook and a table of nchunks entries
int launch_write_meta(const CallParams& cp, uint64_t nchunks, const uint8_t* len, const uint32_t* usedlist,
                      const uint32_t* rowbytes, const uint64_t* rowoff, uint8_t* out, DevState* st,
                      cudaStream_t s);
// payload; rowoff holds every chunk's byte offset (chunk = 0: one per row)
int launch_encode(const uint16_t* codes, uint64_t pitch, const float* x, uint64_t rows, uint64_t rowlen,
                  uint32_t chunk, const uint8_t* len,
                  const uint64_t* cw, const uint64_t* rowoff, uint8_t* out, DevState* st, cudaStream_t s,
                  const int32_t* P = nullptr, const uint8_t* OK = nullptr, int ndim = 0, int layers = 0,
                  uint64_t d1 = 1);
int launch_decode_tables(const uint8_t* codebook, uint32_t nsym, int m, uint32_t* lut, uint32_t* dec_tab,
                         uint8_t* lenbuf, uint32_t* symbuf, DevState* st, cudaStream_t s);

// scratch sizes of the codebook build (elements)
constexpr size_t kSortBufU64 = 3 * 65536;
constexpr size_t kNodeBufU32 = 5 * 65536;
// decoder table words: lengths and first codes (260), the sorted symbols
// (65536 x u16), then the multi-symbol table (2^kMultiBits words)
constexpr int kMultiBits = 12;
constexpr size_t kMultiOff = 260 + 32768;
constexpr size_t kDecTabU32 = kMultiOff + (1u << kMultiBits);

}  // namespace szgb
