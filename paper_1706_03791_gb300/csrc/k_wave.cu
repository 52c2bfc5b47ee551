// k_wave.cu -- the wavefront kernels of the hot path.
//
// Compression (Algorithm 1, the per-point loop): every point is predicted by
// the n-layer predictor (Eq. predmodel) from the *recorded* (decompressed)
// values of its (n+1)^d - 1 preceding neighbours, quantized into 2^m - 1
// intervals of width 2 eb (Sec. IV-A) or stored as a truncated binary
// representation, and its recorded value is kept for later predictions.
// Decompression runs the same prediction in the same dependency order over
// the codes that k_decode_rows (k_decode.cu) decoded from the stream's chunks.
//
// Parallel schedule.  A point depends only on neighbours with smaller
// (plane, row, column) coordinates, so any order that respects that DAG gives
// identical bits.  The field is cut into lines along the fastest axis
// ("rows"); a lane owns one row and computes one column per step.
//   * Within a warp the 32 lanes hold 32 consecutive rows, lane t one column
//     behind lane t-1: the value of the row above at the same column was made
//     by lane t-1 in the previous step and arrives with one shfl.up.
//   * Warps are skewed by whole sweeps of 4 steps: in 3D warp w holds plane
//     i0+w (skew 4w), in 2D it holds the next 32 rows (skew 36w).  Their
//     values pass through shared-memory rings, with one CTA barrier per
//     sweep.  The plane ring is stored diagonally (row t at column l + t), so
//     every lane reads and writes one aligned float4 per sweep.
// Only the lane's own left neighbour and the shuffled upper neighbour are on
// the critical path; the descending summation order puts them last.
//
// Inputs and outputs are staged through shared memory: a warp's 32 rows are
// cut into 32 x 32 tiles; x tiles arrive by TMA, issued by a "staging"
// helper warp, and finished output tiles (codes, or decompressed values)
// leave with coalesced 16-byte stores by a "copy-out" helper warp; a lane
// reads its x and writes its result at the same tile position,
// bank-conflict-free.
//
// CTA boundaries go through global "halo" buffers.  The copy-out warp copies
// the boundary lines out of shared memory as 64-bit words that carry the
// value and a tag (single-copy-atomic stores, no fence), and two "halo-in"
// helper warps load the neighbouring CTAs' lines into the rings by polling
// those words until every tag is set (bounded waits): a block is usable the
// moment it is written, with no progress counter to publish.  The halo
// buffers are zeroed before every launch.  CTAs take work items from a
// ticket counter in dependency order, so a CTA only waits for CTAs that are
// already resident.
#include <cuda.h>

#include <cstring>
#include <mutex>

#include "szgb_internal.cuh"

namespace szgb {

constexpr int kPFX = 4;   // x tiles are loaded this many sweeps ahead
constexpr int kBarEnd = 5;    // named barrier of the four helper warps at the end of an item
// Per-sweep named barriers, two of each so that consecutive sweeps use
// different ones: "ready u" (barrier 6 + u % 2: sweep u's inputs are ready)
// and "done u" (barrier 8 + u % 2: the compute warps have finished sweep u).
// Every warp of the item takes part in both.
constexpr int kBarReady0 = 6;
constexpr int kBarDone0 = 8;
__device__ __forceinline__ void bar_ready_arrive(int u, int n) { named_bar_arrive(kBarReady0 + (u & 1), n); }
__device__ __forceinline__ void bar_ready_sync(int u, int n) { named_bar_sync(kBarReady0 + (u & 1), n); }
__device__ __forceinline__ void bar_done_arrive(int u, int n) { named_bar_arrive(kBarDone0 + (u & 1), n); }
__device__ __forceinline__ void bar_done_sync(int u, int n) { named_bar_sync(kBarDone0 + (u & 1), n); }
constexpr int kNoStop = 0x7fffffff;  // WaveCtl::stop_at when the item runs to the end
constexpr int kTW = 32;   // staging tile: 32 rows x kTW columns
constexpr int kTE = 32 * kTW;  // elements per staging tile
constexpr int kTS = 3;    // staging ring slots per warp
constexpr int kMbarBytes = 256;  // room for kMaxWaveWarps * kTS mbarriers, 128-byte multiple
constexpr int kRP = 32;   // plane ring: floats per row (8 blocks of 4 columns)
constexpr int kRPS = 36;  // plane ring row stride (9 float4: conflict-free)
constexpr int kRV = 64;   // virtual-row ring: floats per line

struct WaveArgs {
    // TMA descriptor of the 32 x 32 input staging tiles: x (compress) or the
    // decoded codes (decompress)
    CUtensorMap tm_x;
    int tma_x;
    int vec_out;      // output rows are 16-byte aligned: tiles leave as 16-byte stores
    uint64_t opitch;  // output row pitch (elements)
    uint64_t xpitch;  // input row pitch (elements; compress)
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
    // common: halo lines as 64-bit words (value bits | kHaloTag << 32), zeroed
    // before the launch; prog: per-item final / aborted state
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

// A halo word: the value's bits in the low half, kHaloTag in the high half.
// An aligned 64-bit access is single-copy atomic, so a reader that sees the
// tag sees the value written with it.
constexpr uint32_t kHaloTag = 0x5a5a0001u;
__device__ __forceinline__ uint64_t halo_word(float v) {
    return ((uint64_t)kHaloTag << 32) | __float_as_uint(v);
}
// one halo block: 4 words, 32-byte aligned (each 64-bit element of the vector
// access is single-copy atomic)
__device__ __forceinline__ void st_relaxed_block(uint64_t* p, uint64_t a, uint64_t b, uint64_t c, uint64_t d) {
    asm volatile("st.relaxed.gpu.global.v4.u64 [%0], {%1, %2, %3, %4};" ::"l"(p), "l"(a), "l"(b), "l"(c), "l"(d)
                 : "memory");
}
__device__ __forceinline__ void ld_relaxed_block(const uint64_t* p, uint64_t (&w)[4]) {
    asm volatile("ld.relaxed.gpu.global.v4.u64 {%0, %1, %2, %3}, [%4];"
                 : "=l"(w[0]), "=l"(w[1]), "=l"(w[2]), "=l"(w[3])
                 : "l"(p)
                 : "memory");
}
__device__ __forceinline__ bool halo_tagged(const uint64_t (&w)[4]) {
    return ((uint32_t)(w[0] >> 32) == kHaloTag) & ((uint32_t)(w[1] >> 32) == kHaloTag) &
           ((uint32_t)(w[2] >> 32) == kHaloTag) & ((uint32_t)(w[3] >> 32) == kHaloTag);
}

__device__ __forceinline__ void fence_acq_rel_gpu() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }
// The tensor map of an item lives in the argument table in global memory,
// which the host rewrites between launches (another field, or the other
// direction's map at the same address): order this thread's tensor-map
// accesses after those writes before its first tiled copy.
__device__ __forceinline__ void fence_tensormap_acquire(const void* tmap) {
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(tmap) : "memory");
}

// ---------------------------------------------------------------------------
// The kernel.  ND = 1, 2 (row topology) or 3 (plane x row); NL = layers;
// DEC = decompress.
//
// Shared memory:
//   PR  [NL+W][32][kRPS] plane ring (3D): plane slot w+NL holds warp w's
//       values, row t at diagonal column l+t; slots < NL are the previous
//       plane block's last planes (virtual planes, loaded by the halo warp)
//   VR  [NL+W][NL][kRV] virtual rows (3D): the NL rows above the CTA for
//       every plane slot (from the row halo of the CTA above, or for the
//       virtual planes from the diagonal CTA)
//   VR  [W][NL][kRV] (1D/2D): the NL rows above warp w (warp w-1's last
//       lanes; for warp 0 the CTA above, loaded by the halo warp)
//   XR  [W][kTS][32][kTW] f32 staging ring of x (compress)
//   OR  [W][kTS][32][kTW] staging ring of the outputs: u16 codes (compress)
//       or f32 values (decompress)
//   MB  [W][kTS] mbarriers of the TMA loads into XR
//   decoder tables (decompress)
// Global halos (64-bit tagged words, copied out of shared memory by the
// halo warp; a block is 4 consecutive columns):
//   3D row halo   [P][nb1][NL][npad]                  unshifted columns
//   3D plane halo [nb0][nb1][NL][(npad+32)/4][32][4]  diagonal columns l+t,
//                 block-major so that the 32 rows of a block are contiguous
//   2D row halo   [nb1][NL][npad]

template <int ND, int NL>
struct Cfg {
    static constexpr int MAXE = (ND == 3) ? (NL * 32 + NL * kMaxWaveWarps + NL * NL + 31) / 32 : 1;
};

// staging elements: compression reads x (f32) and writes codes (u16);
// decompression reads the decoded codes (u16) and writes values (f32)
template <bool DEC>
struct Elems {
    using In = float;
    using Out = uint16_t;
};
template <>
struct Elems<true> {
    using In = uint16_t;
    using Out = float;
};

// TR: also write the recorded (decompressed) values to A.recorded (tests)
// Per-CTA control words of one work item.
struct WaveCtl {
    unsigned int ticket;
    int stop_at;   // first sweep not to run (kNoStop: none); written by the
                   // deciding halo warp before it arrives on that sweep's ready barrier
    int timeout;   // a compute warp's bounded wait ran out
    int err;       // an earlier stage failed (read once, by thread 0)
    int mbar_live; // the mbarriers hold a previous item's state
};

// One work item (a block of planes x rows, or of rows) of one field.  Every
// thread of the CTA calls it; threads beyond the item's W + 4 warps return at
// once.  The caller separates items with __syncthreads().
template <int ND, int NL, bool DEC, bool TR>
__device__ __forceinline__ void wave_item(const WaveArgs& A, const int item, unsigned char* smem_raw, WaveCtl& S) {
    using C = Cfg<ND, NL>;
    using IT = typename Elems<DEC>::In;
    using OT = typename Elems<DEC>::Out;
    // value copies: in the batched kernel the arguments live in global
    // memory, and every named barrier (a memory clobber) would force the
    // per-sweep code to load them again
    const WaveGeom g = A.g;
    const uint64_t a_opitch = A.opitch;
    const uint64_t a_timeout = A.timeout_ns;
    const float* const a_x = A.x;
    float* const a_out = A.out;
    uint16_t* const a_codes = A.codes;
    // test hook: this item is never run and never publishes its state, so
    // its consumers' bounded waits run out (uniform over the CTA)
    if (g.debug_skip == item + 1) return;
    const int W = g.W;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const bool is_helper = (warp >= W);  // warps W and W + 3: halo lines in; W + 1: staging tiles; W + 2: halo lines out

    // shared-memory carve-up from a 128-byte boundary (TMA destinations);
    // the mbarriers sit first, at a place that does not depend on W
    unsigned char* smem = smem_raw + ((128u - (smem_addr(smem_raw) & 127u)) & 127u);
    uint64_t* MB = reinterpret_cast<uint64_t*>(smem);  // kMaxWaveWarps*kTS
    const int npl = (ND == 3) ? (NL + W) : 0;         // plane ring slots
    const int nvl = (ND == 3) ? (NL + W) : W + 1;     // virtual-row line groups
    const int nhr = (ND == 3) ? W : 0;                 // bottom-row line groups (3D)
    float* PR = reinterpret_cast<float*>(smem + kMbarBytes);             // npl*32*kRPS
    float* VR = PR + (size_t)npl * 32 * kRPS;                            // nvl*NL*kRV
    float* HR = VR + (size_t)nvl * NL * kRV;                             // nhr*NL*kRV
    IT* XR = reinterpret_cast<IT*>(HR + (size_t)nhr * NL * kRV);         // W*kTS*kTE inputs
    OT* OR = reinterpret_cast<OT*>(XR + (size_t)W * kTS * kTE);          // W*kTS*kTE outputs
    const bool tma_x = A.tma_x != 0;
    const bool vec_o = A.vec_out != 0;

    if (threadIdx.x == 0) {
        S.stop_at = kNoStop;
        S.timeout = 0;
        S.err = *(volatile const unsigned*)&A.st->err != 0;
        if (tma_x) {
            if (S.mbar_live)
                for (int i = 0; i < kMaxWaveWarps * kTS; i++) mbar_inval(MB + i);
            for (int i = 0; i < kMaxWaveWarps * kTS; i++) mbar_init(MB + i, 1);
            fence_mbar_init();
            S.mbar_live = 1;
        }
    }
    __syncthreads();
    const int ib = (ND == 3) ? item / g.nb1 : 0;
    const int jb = item % g.nb1;  // row block
    if (S.err) {  // an earlier stage failed: publish an aborted state and leave
        if (threadIdx.x == 0) st_release_u32(A.prog + item, kProgAbort);
        return;
    }
    if (warp > W + 3) return;  // a narrower item than the launch

    const int npad = g.ntiles * kTile;     // row halo line length
    const int nshift = npad + 32;          // plane halo line length (diagonal)
    const int nsweeps = g.nsweeps;
    const unsigned final_prog = (unsigned)nsweeps;
    unsigned int* my_prog = A.prog + item;
    const QParams qp = load_qparams(A.st);
    const int N = (int)g.N;
    const int nthr_all = (W + 4) * 32;  // threads of the per-sweep barriers

    if (is_helper) {
        // ================= helper warps: halo lines in (W, W + 3), staging tiles (W + 1), halo lines out (W + 2)
        // Iteration r of the helper warps (pipelined barriers): arrive on
        // "ready r" first (sweep r's inputs were prepared in iteration r - 1),
        // then wait on "done r - 1" (the compute warps have finished the
        // sweeps < r), then work while sweep r runs:
        //   halo-in warps (W, W + 3): land the halo blocks of sweep r + 1
        //     (requested in iteration r - 2) and request those of r + 3; W
        //     decides whether the CTA stops and writes the decision
        //     (S.stop_at = r) before its arrival on "ready r".
        //   staging warp (W + 1): waits until the x tiles of sweep r are in
        //     (when they are not loaded by TMA) before arriving, then loads x
        //     tiles ahead and stores the first half of the output tile
        //     finished in sweep r - 1.
        //   copy-out warp (W + 2): copies out the halo blocks completed in
        //     sweep r - 1, stores the second half of that output tile and, at
        //     the end, publishes the item's state.
        // The helper warps other than W read the decision after "done r - 1"
        // (the decider wrote it before taking part in that barrier; a later
        // decision names a later sweep, so reading it early changes nothing),
        // and sweep 0's after "ready 0".  Since helpers arrive on "ready r"
        // before the compute warps finish sweep r - 1, the compute warps pass
        // from one sweep to the next with a single barrier completion.
        // staging tiles of compute warp w: first row, valid rows, skew in
        // sweeps, and TMA coordinates (row, plane)
        auto tile_row0 = [&](int w) -> uint64_t {
            return (ND == 3) ? ((uint64_t)ib * W + w) * g.M + (uint64_t)jb * 32
                             : (uint64_t)jb * 32 * W + (uint64_t)w * 32;
        };
        auto tile_rows = [&](int w) -> int {
            if (ND == 3) {
                if ((uint64_t)ib * W + w >= g.P) return 0;
                return (int)min((uint64_t)32, g.M - (uint64_t)jb * 32);
            }
            const uint64_t r0 = (uint64_t)jb * 32 * W + (uint64_t)w * 32;
            return r0 >= g.M ? 0 : (int)min((uint64_t)32, g.M - r0);
        };
        unsigned wv_mask = 0;  // warps with valid rows
        for (int w = 0; w < W; w++)
            if (tile_rows(w) > 0) wv_mask |= 1u << w;
        auto tile_s4 = [&](int w) { return (ND == 3) ? w : 9 * w; };
        auto tma_row = [&](int w) { return (ND == 3) ? jb * 32 : (jb * W + w) * 32; };
        auto tma_plane = [&](int w) { return (ND == 3) ? ib * W + w : 0; };
        // Tile kt of warp w is read from sweep 8 kt + s4(w) on and, when
        // full, complete after sweep 8 kt + 15 + s4(w).  s4(w) = w (mod 8)
        // in both topologies, so for a given sweep only warp (sweep mod 8)
        // can start or finish a tile.
        // x tile first read in sweep u: issued kPFX + 1 sweeps ahead
        auto issue_x = [&](int u) {
            {
                if (u < 0) return;
                const int w = u & 7;
                if (!((wv_mask >> w) & 1u)) return;
                const int d = u - tile_s4(w);
                if (d < 0) return;
                const int kt = d >> 3, c0 = kt * kTW;
                if (c0 >= N) return;
                IT* slot = XR + ((size_t)w * kTS + kt % kTS) * kTE;
                if (tma_x) {
                    if (lane == 0) {
                        uint64_t* bar = MB + w * kTS + kt % kTS;
                        mbar_arrive_expect_tx(bar, kTE * (unsigned)sizeof(IT));
                        tma_load_3d(slot, &A.tm_x, c0, tma_row(w), tma_plane(w), bar);
                    }
                } else if constexpr (!DEC) {  // decompression always has TMA (its code array is ours)
                    const int nv = tile_rows(w);
                    const float* xr = a_x + tile_row0(w) * A.xpitch;
                    const int col = c0 + lane;
                    for (int t = 0; t < 32; t++) {
                        const bool ok = t < nv && col < N;
                        cp_async4(slot + t * kTW + lane,
                                  ok ? (const void*)(xr + (uint64_t)t * A.xpitch + col) : (const void*)a_x, ok ? 4 : 0);
                    }
                }
            }
        };
        // store rows [t_lo, t_hi) of output tile kt of warp w: read from
        // shared memory, written with coalesced stores (16 bytes a lane when
        // rows are 16-byte aligned: 4 lanes a u16 row, 8 an f32 row).  A
        // chunk that starts inside the row ends inside its pitch (codes: a
        // pitch of whole 8-code chunks; values: 4 | N when aligned).
        auto store_tile = [&](int w, int kt, int t_lo, int t_hi) {
            const int c0 = kt * kTW;
            const OT* slot = OR + ((size_t)w * kTS + kt % kTS) * kTE;
            const int nv = tile_rows(w);
            const uint64_t base = tile_row0(w) * a_opitch + (uint64_t)c0;
            OT* const og = DEC ? reinterpret_cast<OT*>(a_out) : reinterpret_cast<OT*>(a_codes);
            if (vec_o) {
                constexpr int EPC = 16 / (int)sizeof(OT);  // elements per 16-byte chunk
                constexpr int CPR = kTW / EPC;             // chunks per tile row
                constexpr int RPI = 32 / CPR;              // tile rows per warp instruction
                const int cr = lane % CPR, rr = lane / CPR;
                const bool in = c0 + cr * EPC < N;
#pragma unroll 4
                for (int t0 = t_lo; t0 < t_hi; t0 += RPI) {
                    const int t = t0 + rr;
                    if (!in || t >= nv) continue;
                    const uint4 v = *reinterpret_cast<const uint4*>(slot + t * kTW + cr * EPC);
                    *reinterpret_cast<uint4*>(og + base + (uint64_t)t * a_opitch + cr * EPC) = v;
                }
            } else {
                const bool in = c0 + lane < N;
                for (int t0 = t_lo; t0 < min(nv, t_hi); t0 += 8) {
                    OT v[8];
#pragma unroll
                    for (int i = 0; i < 8; i++) v[i] = slot[((t0 + i) & 31) * kTW + lane];
#pragma unroll
                    for (int i = 0; i < 8; i++) {
                        if (!in || t0 + i >= nv) continue;
                        og[base + (uint64_t)(t0 + i) * a_opitch + lane] = v[i];
                    }
                }
            }
        };
        const int nfull = N / kTW;  // full tiles per row
        // in iteration r (sweeps < r complete): rows [t_lo, t_hi) of the full
        // tile completed in sweep r - 1 (the staging and copy-out warps take
        // half a tile each)
        auto flush = [&](int r, int t_lo, int t_hi) {
            const int v = r - 16;
            if (v >= 0) {
                const int w = v & 7;
                if ((wv_mask >> w) & 1u) {
                    const int d = v - tile_s4(w);
                    if (d >= 0 && (d >> 3) < nfull) store_tile(w, d >> 3, t_lo, t_hi);
                }
            }
        };
        // full tiles of warp w stored inside the sweep loop
        auto flushed_in_loop = [&](int w) {
            const int lim = nsweeps - 17 - tile_s4(w);
            return lim < 0 ? 0 : min(nfull, lim / 8 + 1);
        };

        if (warp == W || warp == W + 3) {
            // two halo-in warps: W takes the even entry slots j (in 3D the
            // plane lines of the first plane) and decides whether the CTA
            // stops; W + 3 takes the odd slots (the row lines)
            const bool decider = warp == W;
            // entry kinds: 0 virtual plane line (PR slot p < NL, row t)
            //              1 virtual row of a real plane (VR slot w+NL, row q)
            //              2 virtual row of a virtual plane (VR slot p, row q)
            //              3 (1D/2D) virtual row of warp 0 (VR group 0, row q)
            const uint64_t* const hrow_g = reinterpret_cast<const uint64_t*>(A.halo_row);
            const uint64_t* const hplane_g = reinterpret_cast<const uint64_t*>(A.halo_plane);
            int e_kind[C::MAXE], e_uoff[C::MAXE], e_nblk[C::MAXE];
            float* e_dst[C::MAXE];  // shared address of block 0 of the line
            int e_dmask[C::MAXE];   // ring blocks - 1
            const uint64_t* e_src[C::MAXE];
            int e_bstr[C::MAXE];              // words between consecutive blocks of the line
            const unsigned* e_prog[C::MAXE];  // the producer's state word (aborts)
            const int NE = (ND == 3) ? (NL * 32 + NL * W + NL * NL) : NL;
#pragma unroll
            for (int j = 0; j < C::MAXE; j++) {
                const int e = lane + 32 * j;
                e_kind[j] = -1;
                e_uoff[j] = 0;
                e_nblk[j] = 0;
                e_dst[j] = nullptr;
                e_dmask[j] = 0;
                e_src[j] = nullptr;
                e_bstr[j] = 4;
                e_prog[j] = nullptr;
                if (e >= NE || (((j & 1) == 0) != decider)) continue;
                if (ND == 3) {
                    if (e < NL * 32) {
                        const int p = e / 32, t = e % 32;
                        e_kind[j] = 0;
                        e_uoff[j] = 0;
                        e_nblk[j] = nshift / 4;
                        e_dst[j] = PR + ((size_t)p * 32 + t) * kRPS;
                        e_dmask[j] = kRP / 4 - 1;
                        // rows past the field's end have no producer (their lanes are idle)
                        if (ib > 0 && (uint64_t)jb * 32 + t < g.M) {
                            e_src[j] = hplane_g + (((size_t)(ib - 1) * g.nb1 + jb) * NL + p) * 32 * nshift + t * 4;
                            e_bstr[j] = 32 * 4;
                            e_prog[j] = A.prog + (ib - 1) * g.nb1 + jb;
                        }
                    } else if (e < NL * 32 + NL * W) {
                        const int e2 = e - NL * 32, w = e2 / NL, q = e2 % NL;
                        e_kind[j] = 1;
                        e_uoff[j] = w;
                        e_nblk[j] = npad / 4;
                        e_dst[j] = VR + ((size_t)(w + NL) * NL + q) * kRV;
                        e_dmask[j] = kRV / 4 - 1;
                        const uint64_t plane = (uint64_t)ib * W + w;
                        if (jb > 0 && plane < g.P) {
                            e_src[j] = hrow_g + (((size_t)plane * g.nb1 + (jb - 1)) * NL + q) * npad;
                            e_prog[j] = A.prog + ib * g.nb1 + jb - 1;
                        }
                    } else {
                        const int e3 = e - NL * 32 - NL * W, p = e3 / NL, q = e3 % NL;
                        e_kind[j] = 2;
                        e_uoff[j] = p - NL;
                        e_nblk[j] = npad / 4;
                        e_dst[j] = VR + ((size_t)p * NL + q) * kRV;
                        e_dmask[j] = kRV / 4 - 1;
                        if (ib > 0 && jb > 0) {
                            const uint64_t plane = (uint64_t)(ib - 1) * W + W - NL + p;
                            e_src[j] = hrow_g + (((size_t)plane * g.nb1 + (jb - 1)) * NL + q) * npad;
                            e_prog[j] = A.prog + (ib - 1) * g.nb1 + jb - 1;
                        }
                    }
                } else {
                    e_kind[j] = 3;
                    e_uoff[j] = 0;
                    e_nblk[j] = npad / 4;
                    e_dst[j] = VR + (size_t)e * kRV;
                    e_dmask[j] = kRV / 4 - 1;
                    if (jb > 0) {
                        e_src[j] = hrow_g + ((size_t)(jb - 1) * NL + e) * npad;
                        e_prog[j] = A.prog + jb - 1;
                    }
                }
            }
            bool timed_out = false;

            // Halo blocks first needed in sweep u (u may be negative): issue()
            // requests them (the words land in registers), land() waits until
            // every requested word carries the tag -- polling again while the
            // producer has not written it, bounded, and giving up when the
            // producer reports an abort -- and stores the values into the rings.
            // Blocks outside a line, or of a CTA boundary without a producer,
            // are zeros.  Two sets of pending requests alternate between odd and
            // even sweeps, so requests are in flight for two sweeps before they
            // are needed and no register copy waits for a load.
            using PendV = uint64_t[C::MAXE][4];
            using PendB = int[C::MAXE];
            uint64_t pvA[C::MAXE][4], pvB[C::MAXE][4];
            int pbA[C::MAXE], pbB[C::MAXE];
#pragma unroll
            for (int j = 0; j < C::MAXE; j++) pbA[j] = pbB[j] = -1;
            auto issue = [&](int u, PendV& pv, PendB& pb) {
#pragma unroll
                for (int j = 0; j < C::MAXE; j++) {
                    pb[j] = -1;
                    if (e_kind[j] < 0) continue;
                    const int b = u - e_uoff[j];
                    if (b < 0) continue;  // columns before the line start are never read
                    pb[j] = b;
                    if (e_src[j] && b < e_nblk[j]) ld_relaxed_block(e_src[j] + (size_t)b * e_bstr[j], pv[j]);
                }
            };
            auto land = [&](PendV& pv, PendB& pb) {
#pragma unroll
                for (int j = 0; j < C::MAXE; j++) {
                    if (pb[j] < 0) continue;
                    const int b = pb[j];
                    float4 v = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                    if (e_src[j] && b < e_nblk[j]) {
                        if (!timed_out && !halo_tagged(pv[j])) {
                            const uint64_t t0 = globaltimer();
                            for (unsigned it = 1;; it++) {
                                __nanosleep(32);
                                ld_relaxed_block(e_src[j] + (size_t)b * e_bstr[j], pv[j]);
                                if (halo_tagged(pv[j])) break;
                                if ((it & 63) == 0 &&
                                    (ld_acquire_u32(e_prog[j]) == kProgAbort || globaltimer() - t0 > a_timeout ||
                                     it >= (1u << 28))) {
                                    timed_out = true;
                                    break;
                                }
                            }
                        }
                        if (!timed_out)
                            v = make_float4(__uint_as_float((uint32_t)pv[j][0]), __uint_as_float((uint32_t)pv[j][1]),
                                            __uint_as_float((uint32_t)pv[j][2]), __uint_as_float((uint32_t)pv[j][3]));
                    }
                    *reinterpret_cast<float4*>(e_dst[j] + (size_t)((b & e_dmask[j]) * 4)) = v;
                    pb[j] = -1;
                }
                timed_out = __any_sync(0xffffffffu, timed_out);
            };
            // prologue: every halo block needed up to sweep 1; requests for 2, 3
            for (int u = -2 * NL - 1; u < 2; u++) {
                issue(u, pvA, pbA);
                land(pvA, pbA);
            }
            issue(2, pvA, pbA);
            issue(3, pvB, pbB);
            // sweep 0: the decider arrives with its decision, the other halo-in
            // warp waits to read it and reports its own timeouts through
            // S.timeout (read by the decider after a later done barrier)
            if (decider) {
                if (lane == 0 && timed_out) S.stop_at = 0;
                __syncwarp();
                bar_ready_arrive(0, nthr_all);
            } else {
                if (lane == 0 && timed_out) S.timeout = 1;
                __syncwarp();
                bar_ready_sync(0, nthr_all);
            }
            bool stop = decider ? timed_out : (*(volatile int*)&S.stop_at <= 0);
            for (int r = 1; r <= nsweeps && !stop; r++) {
                if (decider) {
                    if (r < nsweeps) {
                        stop = __any_sync(0xffffffffu, timed_out || *(volatile int*)&S.timeout != 0);
                        if (lane == 0 && stop) S.stop_at = r;
                        __syncwarp();
                        bar_ready_arrive(r, nthr_all);  // sweep r
                    }
                    bar_done_sync(r - 1, nthr_all);  // sweeps < r are complete
                } else {
                    if (lane == 0 && timed_out) S.timeout = 1;
                    __syncwarp();
                    if (r < nsweeps) bar_ready_arrive(r, nthr_all);  // sweep r
                    bar_done_sync(r - 1, nthr_all);                  // sweeps < r are complete
                    stop = *(volatile int*)&S.stop_at <= r;
                }
                if (stop) break;
                if (r & 1) {
                    land(pvA, pbA);  // sweep r + 1
                    issue(r + 3, pvA, pbA);
                } else {
                    land(pvB, pbB);
                    issue(r + 3, pvB, pbB);
                }
            }
            // a timeout in the last landing marks the item aborted
            if (lane == 0 && timed_out) atomicMin(&S.stop_at, nsweeps);
            __syncwarp();
            named_bar_sync(kBarEnd, 4 * 32);  // the helper warps see the final S.stop_at
            return;
        }
        if (warp == W + 2) {
            // copy-out entries: the halo lines this CTA produces, moved from shared
            // memory to the global halo buffers one 4-column block per sweep
            //   3D row halo: warp w's bottom line q (HR), block b after sweep b+w+8
            //   3D plane halo: the last NL warps' plane-ring rows (diagonal), block
            //                  blk after sweep blk+w
            //   2D row halo: the last warp's bottom lines (VR group W), block b
            //                after sweep b+9W-1
            constexpr int MAXC = (ND == 3) ? (NL * kMaxWaveWarps + NL * 32 + 31) / 32 : 1;
            uint64_t* const hrow_o = reinterpret_cast<uint64_t*>(A.halo_row);
            uint64_t* const hplane_o = reinterpret_cast<uint64_t*>(A.halo_plane);
            const float* c_src[MAXC];
            uint64_t* c_dst[MAXC];
            int c_off[MAXC], c_nblk[MAXC], c_smask[MAXC], c_sstride[MAXC], c_bstr[MAXC];
#pragma unroll
            for (int j = 0; j < MAXC; j++) {
                const int e = lane + 32 * j;
                c_src[j] = nullptr;
                c_dst[j] = nullptr;
                c_off[j] = 0;
                c_nblk[j] = 0;
                c_smask[j] = 0;
                c_sstride[j] = 0;
                c_bstr[j] = 4;
                if (ND == 3) {
                    if (e < NL * W) {
                        const int w = e / NL, q = e % NL;
                        const uint64_t plane = (uint64_t)ib * W + w;
                        if (plane < g.P && jb + 1 < g.nb1) {
                            c_src[j] = HR + ((size_t)w * NL + q) * kRV;
                            c_dst[j] = hrow_o + (((size_t)plane * g.nb1 + jb) * NL + q) * npad;
                            c_off[j] = w + 9;
                            c_nblk[j] = npad / 4;
                            c_smask[j] = kRV / 4 - 1;
                        }
                    } else if (e < NL * W + NL * 32) {
                        const int e2 = e - NL * W, p2 = e2 / 32, t = e2 % 32, w = W - NL + p2;
                        const uint64_t plane = (uint64_t)ib * W + w, row = (uint64_t)jb * 32 + t;
                        if (ib + 1 < g.nb0 && plane < g.P && row < g.M) {
                            c_src[j] = PR + ((size_t)(w + NL) * 32 + t) * kRPS;
                            c_dst[j] = hplane_o + (((size_t)ib * g.nb1 + jb) * NL + p2) * 32 * nshift + t * 4;
                            c_bstr[j] = 32 * 4;
                            c_off[j] = w + 1;
                            c_nblk[j] = nshift / 4;
                            c_smask[j] = kRP / 4 - 1;
                        }
                    }
                } else if (e < NL && jb + 1 < g.nb1) {
                    c_src[j] = VR + ((size_t)W * NL + e) * kRV;
                    c_dst[j] = hrow_o + ((size_t)jb * NL + e) * npad;
                    c_off[j] = 9 * W;
                    c_nblk[j] = npad / 4;
                    c_smask[j] = kRV / 4 - 1;
                }
            }
            // in iteration r (sweeps < r complete): the blocks completed in sweep r - 1
            auto copy_out = [&](int r) {
#pragma unroll
                for (int j = 0; j < MAXC; j++) {
                    if (!c_src[j]) continue;
                    const int b = r - c_off[j];
                    if (b < 0 || b >= c_nblk[j]) continue;
                    const float4 v = *reinterpret_cast<const float4*>(c_src[j] + (b & c_smask[j]) * 4);
                    st_relaxed_block(c_dst[j] + (size_t)b * c_bstr[j], halo_word(v.x), halo_word(v.y), halo_word(v.z),
                                     halo_word(v.w));
                }
            };
            bar_ready_sync(0, nthr_all);
            bool stop = *(volatile int*)&S.stop_at <= 0;
            for (int r = 1; r <= nsweeps && !stop; r++) {
                if (r < nsweeps) bar_ready_arrive(r, nthr_all);  // sweep r
                bar_done_sync(r - 1, nthr_all);                  // sweeps < r are complete
                stop = *(volatile int*)&S.stop_at <= r;
                if (stop) break;
                copy_out(r);
                flush(r, 16, 32);
            }
            __syncwarp();
            named_bar_sync(kBarEnd, 4 * 32);
            const bool aborted = S.stop_at != kNoStop;
            if (!aborted) {
                // the halo blocks completed in the last sweeps
                for (int r = nsweeps; r <= nsweeps + 9 * W + 9; r++) copy_out(r);
                // the tiles not stored yet (every sweep is complete)
                const int ntl = (N + kTW - 1) / kTW;
                for (int w = 0; w < W; w++) {
                    if (!((wv_mask >> w) & 1u)) continue;
                    for (int kt = flushed_in_loop(w); kt < ntl; kt++) store_tile(w, kt, 0, 32);
                }
            }
            fence_acq_rel_gpu();
            __syncwarp();
            if (lane == 0) {
                if (aborted) {
                    atomicOr(&A.st->err, kErrTimeout);
                    st_release_u32(my_prog, kProgAbort);
                } else {
                    st_release_u32(my_prog, final_prog);
                }
            }
            return;
        }
        // staging warp; prologue: x tiles up to sweep kPFX
        int u_issued = kPFX;  // latest sweep whose x tiles were issued
        if (tma_x && lane == 0) fence_tensormap_acquire(&A.tm_x);
        for (int u = 0; u <= kPFX; u++) issue_x(u);
        cp_async_commit();
        cp_async_wait<0>();
        __syncwarp();
        bar_ready_sync(0, nthr_all);
        bool stop = *(volatile int*)&S.stop_at <= 0;
        for (int r = 1; r <= nsweeps && !stop; r++) {
            cp_async_wait<kPFX - 1>();  // x tiles of sweep r (when not loaded by TMA)
            __syncwarp();
            if (r < nsweeps) bar_ready_arrive(r, nthr_all);  // sweep r
            bar_done_sync(r - 1, nthr_all);                  // sweeps < r are complete
            stop = *(volatile int*)&S.stop_at <= r;
            if (stop) break;
            issue_x(r + kPFX);
            u_issued = r + kPFX;
            cp_async_commit();
            flush(r, 0, 16);
        }
        cp_async_wait<0>();
        __syncwarp();
        named_bar_sync(kBarEnd, 4 * 32);
        if (tma_x && S.stop_at != kNoStop && lane == 0) {
            // loads still in flight land in this CTA's shared memory: wait
            // for the latest load of every slot (the last 8 kTS sweeps issued
            // hold it) before leaving
            for (int u = max(0, u_issued - 8 * kTS + 1); u <= u_issued; u++) {
                const int w = u & 7;
                if (!((wv_mask >> w) & 1u)) continue;
                const int d = u - tile_s4(w);
                if (d < 0 || (d >> 3) * kTW >= N) continue;
                const int kt = d >> 3;
                mbar_wait_bounded(MB + w * kTS + kt % kTS, (unsigned)(kt / kTS) & 1u, a_timeout);
            }
        }
        __syncwarp();
        return;
    }

    // ================= compute warps =================
    uint64_t plane, row;
    int sig;  // warp skew in steps
    bool wvalid;  // the warp has valid rows
    if (ND == 3) {
        plane = (uint64_t)ib * W + warp;
        row = (uint64_t)jb * 32 + lane;
        sig = 4 * warp;
        wvalid = plane < g.P;
    } else {
        plane = 0;
        row = (uint64_t)jb * 32 * W + warp * 32 + lane;
        sig = 36 * warp;
        wvalid = (uint64_t)jb * 32 * W + warp * 32 < g.M;
    }
    const int s4 = sig / 4;
    const bool valid = (plane < g.P) && (row < g.M);
    const uint64_t rowid = plane * g.M + row;
    const uint64_t rowbase = rowid * g.N;
    float* const rec_row = TR ? A.recorded + rowbase : nullptr;
    const IT* const xw = XR + (size_t)warp * kTS * kTE + lane * kTW;  // this lane's tile rows
    const float* const out_row = DEC ? a_out + rowbase : nullptr;       // unpredictable values (decompress)
    OT* const ow = OR + (size_t)warp * kTS * kTE + lane * kTW;
    const int col0 = -lane - sig;  // column at step 0

    // lanes of the last NL rows keep their values in a shared line: in 3D
    // for the row halo (copied out by the halo warp), in 1D/2D as the next
    // warp's virtual rows (the last warp's group W is copied out as the row
    // halo).  The plane halo is copied out of the plane ring.
    const bool has_hr = lane >= 32 - NL;
    const int hr_q = has_hr ? lane - (32 - NL) : 0;
    const uint32_t hr_addr = smem_addr((ND == 3) ? HR + ((size_t)warp * NL + hr_q) * kRV
                                                 : VR + ((size_t)(warp + 1) * NL + hr_q) * kRV);
    // this lane's virtual-row lines (lanes t < NL): own plane and planes - a
    const float* vr_own = (ND == 3) ? VR + (size_t)(warp + NL) * NL * kRV : VR + (size_t)warp * NL * kRV;

    // neighbour histories: index [e] = column l - e
    float oV[NL + 1];                       // own line
    float Rr[NL + 1][NL + 1];               // rows above, own plane
    float Pp[NL + 1][NL + 1];               // planes below, own row (3D)
    float Qq[NL + 1][NL + 1][NL + 1];       // planes below, rows above (3D)
#pragma unroll
    for (int e = 0; e <= NL; e++) {
        oV[e] = 0.0f;
#pragma unroll
        for (int b = 0; b <= NL; b++) {
            Rr[b][e] = 0.0f;
            Pp[b][e] = 0.0f;
#pragma unroll
            for (int c = 0; c <= NL; c++) Qq[b][c][e] = 0.0f;
        }
    }


    for (int q = 0; q < nsweeps; q++) {
        bar_ready_sync(q, nthr_all);  // this sweep's inputs are ready
        if (*(volatile int*)&S.stop_at <= q) break;
        // this warp's next x tile is first read in this sweep: wait for its load
        if (tma_x && wvalid) {
            const int d = q - s4;
            if (d >= 0 && (d & 7) == 0 && (d >> 3) * kTW < N) {
                const int kt = d >> 3;
                if (!mbar_wait_bounded(MB + warp * kTS + kt % kTS, (unsigned)(kt / kTS) & 1u, a_timeout)) {
                    if (lane == 0) {
                        atomicOr(&A.st->err, kErrTimeout);
                        S.timeout = 1;  // the halo warp stops the CTA after this sweep
                    }
                }
            }
        }
        const int lq = 4 * q + col0;  // this lane's column at step 0 of the sweep
        const int wl0 = 4 * q - sig;  // lane 0's column at step 0 (warp-uniform)
        // a warp is idle in sweeps where none of its lanes has a column
        if (wl0 + 3 >= 0 && wl0 - 31 < N) {
            // 3D, one layer, a sweep whose 4 columns lie inside the row for
            // every lane: the same terms, order and arithmetic as the general
            // step below, without its boundary cases (the rows above lane 0
            // come as one float4 per sweep)
            bool interior = false;
            if constexpr (ND == 3 && NL == 1) {
                if (wl0 >= 31 && wl0 + 3 < N) {
                    interior = true;
                    const int blk = (q - warp) & (kRP / 4 - 1);
                    const float4 p4 = *reinterpret_cast<const float4*>(PR + ((size_t)warp * 32 + lane) * kRPS + blk * 4);
                    const int cl0 = wl0 & (kRV - 1);
                    const float4 r4 = *reinterpret_cast<const float4*>(vr_own + cl0);
                    const float4 q4 = *reinterpret_cast<const float4*>(VR + (size_t)warp * kRV + cl0);
                    const int c0 = lq & (kTW - 1);
                    const int sl0 = (int)(((unsigned)lq >> 5) % kTS) * kTE;
                    const int sl1 = (sl0 == (kTS - 1) * kTE) ? 0 : sl0 + kTE;
                    int tix[kTile];
#pragma unroll
                    for (int k = 0; k < kTile; k++) tix[k] = (c0 + k >= kTW) ? sl1 + c0 + k - kTW : sl0 + c0 + k;
                    int dc[kTile];
                    float du[kTile];
                    if constexpr (DEC) {
#pragma unroll
                        for (int k = 0; k < kTile; k++) {
                            dc[k] = (int)xw[tix[k]];
                            du[k] = 0.0f;
                            if (dc[k] == 0 && valid) du[k] = out_row[lq + k];
                        }
                    }
                    float vo[kTile];
#pragma unroll
                    for (int k = 0; k < kTile; k++) {
                        const float pk = (k == 0) ? p4.x : (k == 1) ? p4.y : (k == 2) ? p4.z : p4.w;
                        const float rk = (k == 0) ? r4.x : (k == 1) ? r4.y : (k == 2) ? r4.z : r4.w;
                        const float qk = (k == 0) ? q4.x : (k == 1) ? q4.y : (k == 2) ? q4.z : q4.w;
                        float nr = __shfl_up_sync(0xffffffffu, oV[1], 1);
                        float nq = __shfl_up_sync(0xffffffffu, Pp[1][0], 1);
                        nr = (lane == 0) ? rk : nr;
                        nq = (lane == 0) ? qk : nq;
                        Rr[1][1] = Rr[1][0];
                        Rr[1][0] = nr;
                        Pp[1][1] = Pp[1][0];
                        Pp[1][0] = pk;
                        Qq[1][1][1] = Qq[1][1][0];
                        Qq[1][1][0] = nq;
                        // descending (a, b, e): +(1,1,1) -(1,1,0) -(1,0,1) +(1,0,0) -(0,1,1) +(0,1,0) +(0,0,1)
                        float pred = Qq[1][1][1];
                        pred = __fsub_rn(pred, Qq[1][1][0]);
                        pred = __fsub_rn(pred, Pp[1][1]);
                        pred = __fadd_rn(pred, Pp[1][0]);
                        pred = __fsub_rn(pred, Rr[1][1]);
                        pred = __fadd_rn(pred, Rr[1][0]);
                        pred = __fadd_rn(pred, oV[1]);
                        float V;
                        if constexpr (!DEC) {
                            const float xv = xw[tix[k]];
                            const float tr = trunc_value(xv, qp.e_eb);
                            const int code = quantize_tr(xv, pred, tr, qp, V);
                            ow[tix[k]] = (uint16_t)code;
                        } else {
                            V = dc[k] ? dequantize(dc[k], pred, qp) : du[k];
                            ow[tix[k]] = V;
                        }
                        oV[1] = V;
                        vo[k] = V;
                        st_shared_f32_if(has_hr, hr_addr + 4u * (uint32_t)((lq + k) & (kRV - 1)), V);
                        if constexpr (TR) {
                            if (valid) rec_row[lq + k] = V;
                        }
                    }
                    *reinterpret_cast<float4*>(PR + ((size_t)(warp + NL) * 32 + lane) * kRPS + blk * 4) =
                        make_float4(vo[0], vo[1], vo[2], vo[3]);
                }
            }
            // 2D, one layer, the same for rows: in descending (b, e) order
            // -(1,1) +(1,0) +(0,1)
            if constexpr (ND == 2 && NL == 1) {
                if (wl0 >= 31 && wl0 + 3 < N) {
                    interior = true;
                    const int cl0 = wl0 & (kRV - 1);
                    const float4 r4 = *reinterpret_cast<const float4*>(vr_own + cl0);
                    const int c0 = lq & (kTW - 1);
                    const int sl0 = (int)(((unsigned)lq >> 5) % kTS) * kTE;
                    const int sl1 = (sl0 == (kTS - 1) * kTE) ? 0 : sl0 + kTE;
                    int tix[kTile];
#pragma unroll
                    for (int k = 0; k < kTile; k++) tix[k] = (c0 + k >= kTW) ? sl1 + c0 + k - kTW : sl0 + c0 + k;
                    int dc[kTile];
                    float du[kTile];
                    if constexpr (DEC) {
#pragma unroll
                        for (int k = 0; k < kTile; k++) {
                            dc[k] = (int)xw[tix[k]];
                            du[k] = 0.0f;
                            if (dc[k] == 0 && valid) du[k] = out_row[lq + k];
                        }
                    }
#pragma unroll
                    for (int k = 0; k < kTile; k++) {
                        const float rk = (k == 0) ? r4.x : (k == 1) ? r4.y : (k == 2) ? r4.z : r4.w;
                        float nr = __shfl_up_sync(0xffffffffu, oV[1], 1);
                        nr = (lane == 0) ? rk : nr;
                        Rr[1][1] = Rr[1][0];
                        Rr[1][0] = nr;
                        float pred = -Rr[1][1];
                        pred = __fadd_rn(pred, Rr[1][0]);
                        pred = __fadd_rn(pred, oV[1]);
                        float V;
                        if constexpr (!DEC) {
                            const float xv = xw[tix[k]];
                            const float tr = trunc_value(xv, qp.e_eb);
                            const int code = quantize_tr(xv, pred, tr, qp, V);
                            ow[tix[k]] = (uint16_t)code;
                        } else {
                            V = dc[k] ? dequantize(dc[k], pred, qp) : du[k];
                            ow[tix[k]] = V;
                        }
                        oV[1] = V;
                        st_shared_f32_if(has_hr, hr_addr + 4u * (uint32_t)((lq + k) & (kRV - 1)), V);
                        if constexpr (TR) {
                            if (valid) rec_row[lq + k] = V;
                        }
                    }
                }
            }
            if (!interior) {
                float4 pr[NL + 1];
                if (ND == 3) {
                    const int blk = (q - warp) & (kRP / 4 - 1);
#pragma unroll
                    for (int a = 1; a <= NL; a++)
                        pr[a] = *reinterpret_cast<const float4*>(PR + ((size_t)(warp + NL - a) * 32 + lane) * kRPS + blk * 4);
                }
                float vout[kTile];
                // staging slots of this sweep's columns (a sweep spans at most two tiles)
                const unsigned kt0 = lq > 0 ? (unsigned)lq >> 5 : 0u;
                const int sl0 = (int)(kt0 % kTS) * kTE;
                const int sl1 = (sl0 == (kTS - 1) * kTE) ? 0 : sl0 + kTE;
                // decompression: this sweep's codes and, for code 0, the stored
                // values, read before the dependent steps so that the loads'
                // latency overlaps them
                int dcode[kTile];
                float duv[kTile];
                if constexpr (DEC) {
#pragma unroll
                    for (int k = 0; k < kTile; k++) {
                        const int l = lq + k;
                        const bool act = (l >= 0) && (l < N);
                        const bool cross = lq >= 0 && (lq & (kTW - 1)) + k >= kTW;
                        const int ti = (cross ? sl1 : sl0) + (l & (kTW - 1));
                        dcode[k] = act ? (int)xw[ti] : 0;
                        duv[k] = 0.0f;
                        if (dcode[k] == 0 && valid && act) duv[k] = out_row[l];
                    }
                }
#pragma unroll
                for (int k = 0; k < kTile; k++) {
                    const int l = lq + k;
                    const bool act = (l >= 0) && (l < N);
                    // position of column l in this lane's staging rows
                    const bool cross = lq >= 0 && (lq & (kTW - 1)) + k >= kTW;
                    const int ti = (cross ? sl1 : sl0) + (l & (kTW - 1));
                    // ---- new neighbour values at column l (shuffles first: they
                    // read the values of the previous step)
                    float nR[NL + 1], nP[NL + 1], nQ[NL + 1][NL + 1];
                    // row t - b at column l is row (t - 1) - (b - 1) of the lane above,
                    // which held column l in the previous step
                    nR[1] = __shfl_up_sync(0xffffffffu, oV[1], 1);
#pragma unroll
                    for (int b = 2; b <= NL; b++) nR[b] = __shfl_up_sync(0xffffffffu, Rr[b - 1][0], 1);
                    if (ND == 3) {
#pragma unroll
                        for (int a = 1; a <= NL; a++) {
                            nP[a] = (k == 0) ? pr[a].x : (k == 1) ? pr[a].y : (k == 2) ? pr[a].z : pr[a].w;
                            nQ[a][1] = __shfl_up_sync(0xffffffffu, Pp[a][0], 1);
#pragma unroll
                            for (int b = 2; b <= NL; b++) nQ[a][b] = __shfl_up_sync(0xffffffffu, Qq[a][b - 1][0], 1);
                        }
                    }
                    // lanes next to the top of the block read the rows above
                    // (every lane loads, from a clamped line; lanes >= b discard)
                    if (ND >= 2) {
                        const int cl = l & (kRV - 1);
#pragma unroll
                        for (int b = 1; b <= NL; b++) {
                            const int vr = min(NL + lane - b, NL - 1);
                            const bool top = lane < b;
                            const float r_v = vr_own[vr * kRV + cl];
                            nR[b] = top ? r_v : nR[b];
                            if (ND == 3) {
#pragma unroll
                                for (int a = 1; a <= NL; a++) {
                                    const float q_v = VR[((size_t)(warp + NL - a) * NL + vr) * kRV + cl];
                                    nQ[a][b] = top ? q_v : nQ[a][b];
                                }
                            }
                        }
                    }
                    // shift histories, insert (zeros outside the row)
#pragma unroll
                    for (int b = 1; b <= NL; b++) {
#pragma unroll
                        for (int e = NL; e >= 1; e--) Rr[b][e] = Rr[b][e - 1];
                        Rr[b][0] = act ? nR[b] : 0.0f;
                    }
                    if (ND == 3) {
#pragma unroll
                        for (int a = 1; a <= NL; a++) {
#pragma unroll
                            for (int e = NL; e >= 1; e--) Pp[a][e] = Pp[a][e - 1];
                            Pp[a][0] = act ? nP[a] : 0.0f;
#pragma unroll
                            for (int b = 1; b <= NL; b++) {
#pragma unroll
                                for (int e = NL; e >= 1; e--) Qq[a][b][e] = Qq[a][b][e - 1];
                                Qq[a][b][0] = act ? nQ[a][b] : 0.0f;
                            }
                        }
                    }
                    // ---- prediction: terms in descending lexicographic (a, b, e)
                    float pred = 0.0f;
                    bool first = true;
                    constexpr int AA = (ND == 3) ? NL : 0;
                    constexpr int BB = (ND >= 2) ? NL : 0;
#pragma unroll
                    for (int a = AA; a >= 0; a--) {
#pragma unroll
                        for (int b = BB; b >= 0; b--) {
#pragma unroll
                            for (int e = NL; e >= 0; e--) {
                                if (a == 0 && b == 0 && e == 0) continue;
                                const float v = (a > 0 && b > 0) ? Qq[a][b][e]
                                              : (a > 0)          ? Pp[a][e]
                                              : (b > 0)          ? Rr[b][e]
                                                                 : oV[e];
                                const int c = term_coef(NL, a, b, e);
                                if (NL == 1) {
                                    if (first) pred = (c > 0) ? v : -v;
                                    else pred = (c > 0) ? __fadd_rn(pred, v) : __fsub_rn(pred, v);
                                } else {
                                    const float prod = __fmul_rn((float)c, v);
                                    pred = first ? prod : __fadd_rn(pred, prod);
                                }
                                first = false;
                            }
                        }
                    }
                    // ---- quantize (compress) / decode + dequantize (decompress)
                    float V;
                    int code = 0;
                    if constexpr (!DEC) {
                        const float xv = act ? xw[ti] : 0.0f;
                        const float tr = trunc_value(xv, qp.e_eb);
                        code = quantize_tr(xv, pred, tr, qp, V);
                    } else {
                        // the decode pass left the code in the tile and, for code
                        // 0, the unpredictable value in the output array
                        code = dcode[k];
                        V = code ? dequantize(code, pred, qp) : duv[k];
                    }
                    V = act ? V : 0.0f;
#pragma unroll
                    for (int e = NL; e >= 2; e--) oV[e] = oV[e - 1];
                    oV[1] = V;
                    vout[k] = V;
                    if (act) {
                        if constexpr (DEC) ow[ti] = V;
                        else ow[ti] = (uint16_t)code;
                    }
                    st_shared_f32_if(has_hr && act, hr_addr + 4u * (uint32_t)(l & (kRV - 1)), V);
                    if constexpr (TR) {
                        if (valid && act) rec_row[l] = V;
                    }
                }
                // this sweep's 4 values, diagonal block q - warp: plane ring and plane halo
                if (ND == 3) {
                    const int blk = q - warp;
                    const float4 v4 = make_float4(vout[0], vout[1], vout[2], vout[3]);
                    *reinterpret_cast<float4*>(PR + ((size_t)(warp + NL) * 32 + lane) * kRPS + (blk & (kRP / 4 - 1)) * 4) = v4;
                }
            }
        }
        bar_done_arrive(q, nthr_all);  // this warp has finished the sweep
    }
}

// one field, one work item per CTA (items from the field's ticket counter)
template <int ND, int NL, bool DEC, bool TR>
__global__ void __launch_bounds__((kMaxWaveWarps + 4) * 32, 1) k_wave(const __grid_constant__ WaveArgs A) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ WaveCtl S;
    if (threadIdx.x == 0) {
        S.ticket = atomicAdd(&A.st->ticket, 1u);
        S.mbar_live = 0;
    }
    __syncthreads();
    wave_item<ND, NL, DEC, TR>(A, (int)S.ticket, smem_raw, S);
}

// Many fields in one persistent launch: every CTA takes (field, item) pairs
// from a global ticket over `order`, which lists each field's items in
// dependency order (interleaved across fields), so a CTA only waits for
// items that resident CTAs took earlier.
template <int NL, bool DEC>
__global__ void __launch_bounds__((kMaxWaveWarps + 4) * 32, 1)
    k_wave_batch(const WaveArgs* __restrict__ F, const uint2* __restrict__ order, unsigned total, unsigned* ticket) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ WaveCtl S;
    if (threadIdx.x == 0) S.mbar_live = 0;
    for (;;) {
        if (threadIdx.x == 0) S.ticket = atomicAdd(ticket, 1u);
        __syncthreads();
        const unsigned t = S.ticket;
        if (t >= total) break;
        const uint2 o = order[t];
        const WaveArgs& A = F[o.x];
        const int nd = A.g.ndim;
        if (nd == 3) {
            if constexpr (NL <= kMaxLayers3D) wave_item<3, NL, DEC, false>(A, (int)o.y, smem_raw, S);
        } else if (nd == 2) {
            wave_item<2, NL, DEC, false>(A, (int)o.y, smem_raw, S);
        } else {
            wave_item<1, NL, DEC, false>(A, (int)o.y, smem_raw, S);
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// host side

size_t wave_smem_bytes(const WaveGeom& g, int layers, bool decompress) {
    const int NL = layers, W = g.W;
    const int npl = (g.ndim == 3) ? (NL + W) : 0;
    const int nvl = (g.ndim == 3) ? (NL + W) : W + 1;
    const int nhr = (g.ndim == 3) ? W : 0;
    size_t b = 128 + kMbarBytes;  // alignment slack, mbarriers
    b += (size_t)npl * 32 * kRPS * 4 + (size_t)(nvl + nhr) * NL * kRV * 4;
    b += (size_t)W * kTS * kTE * (4 + 2);  // input and output rings (f32 + u16 either way)
    (void)decompress;
    return b;
}

// cuTensorMapEncodeTiled, looked up once through the runtime (no link
// dependency on the driver library)
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
        else
            cudaGetLastError();
    });
    return fn;
}

// TMA descriptor of 32 x 32 tiles of a [P][M][N] array (row pitch `pitch`
// elements, f32 or u16); false when the array does not meet TMA's rules
// (16-byte aligned base and row pitch, int32 coordinates), in which case the
// kernel uses plain loads and stores
static bool encode_tiles(CUtensorMap* m, bool f32, const void* base, uint64_t N, uint64_t M, uint64_t P,
                         uint64_t pitch) {
    const uint64_t es = f32 ? 4 : 2;
    if (!base || (reinterpret_cast<uintptr_t>(base) & 15) || (pitch * es) % 16) return false;
    if (N >= (1ull << 31) || M * P >= (1ull << 31)) return false;
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[3] = {N, M, P};
    cuuint64_t strides[2] = {pitch * es, pitch * es * M};
    cuuint32_t box[3] = {(cuuint32_t)kTW, 32, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    return fn(m, f32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_UINT16, 3, const_cast<void*>(base),
              dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
              CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// The dynamic shared-memory limit of a kernel is raised once, to the device
// maximum, and never lowered: a per-launch value would race between host
// threads launching the same kernel with different sizes.
// (one flag per kernel: the template is instantiated per function)
template <auto Fn>
static int smem_limit_once(size_t need) {
    static std::once_flag once;
    static int limit = 0;
    std::call_once(once, [] {
        int dev = 0, mx = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&mx, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        cudaFuncAttributes fa;
        if (cudaFuncGetAttributes(&fa, Fn) != cudaSuccess) {  // the limit covers static + dynamic
            cudaGetLastError();
            return;
        }
        const int dyn = mx - (int)fa.sharedSizeBytes;
        if (cudaFuncSetAttribute(Fn, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn) == cudaSuccess) limit = dyn;
        else cudaGetLastError();
    });
    return (size_t)limit >= need ? 0 : SZGB_ECUDA;
}

template <int ND, int NL, bool DEC, bool TR>
static int launch_t(const WaveArgs& a, cudaStream_t s) {
    size_t smem = wave_smem_bytes(a.g, NL, DEC);
    auto fn = k_wave<ND, NL, DEC, TR>;
    if (smem_limit_once<k_wave<ND, NL, DEC, TR>>(smem)) return SZGB_ECUDA;
    fn<<<a.g.num_ctas, (a.g.W + 4) * 32, smem, s>>>(a);
    return cudaGetLastError() == cudaSuccess ? 0 : SZGB_ECUDA;
}

template <bool DEC, bool TR>
static int launch_nd(const WaveArgs& a, int layers, cudaStream_t s) {
    if (a.g.ndim == 3) return layers == 1 ? launch_t<3, 1, DEC, TR>(a, s) : launch_t<3, 2, DEC, TR>(a, s);
    if (a.g.ndim == 2) {
        switch (layers) {
            case 1: return launch_t<2, 1, DEC, TR>(a, s);
            case 2: return launch_t<2, 2, DEC, TR>(a, s);
            case 3: return launch_t<2, 3, DEC, TR>(a, s);
            default: return launch_t<2, 4, DEC, TR>(a, s);
        }
    }
    switch (layers) {
        case 1: return launch_t<1, 1, DEC, TR>(a, s);
        case 2: return launch_t<1, 2, DEC, TR>(a, s);
        case 3: return launch_t<1, 3, DEC, TR>(a, s);
        default: return launch_t<1, 4, DEC, TR>(a, s);
    }
}
template <bool DEC>
static int launch_any(const WaveArgs& a, int layers, cudaStream_t s) {
    if (!DEC && a.recorded) return launch_nd<false, true>(a, layers, s);
    return launch_nd<DEC, false>(a, layers, s);
}

static void fill_compress(WaveArgs& a, const WaveGeom& g, const float* x, uint64_t x_pitch, uint16_t* codes,
                          uint64_t codes_pitch, float* recorded, float* halo_row, float* halo_plane,
                          unsigned int* prog, DevState* st, uint64_t timeout_ns) {
    memset(&a, 0, sizeof(a));
    a.g = g;
    a.x = x;
    a.xpitch = x_pitch;
    a.codes = codes;
    a.opitch = codes_pitch;
    a.recorded = recorded;
    a.halo_row = halo_row;
    a.halo_plane = halo_plane;
    a.prog = prog;
    a.st = st;
    a.timeout_ns = timeout_ns;
    a.tma_x = encode_tiles(&a.tm_x, true, x, g.N, g.M, g.P, x_pitch) ? 1 : 0;
    a.vec_out = ((reinterpret_cast<uintptr_t>(codes) & 15) == 0 && (codes_pitch * 2) % 16 == 0) ? 1 : 0;
}

static void fill_decompress(WaveArgs& a, const WaveGeom& g, const uint16_t* codes, uint64_t codes_pitch, float* out,
                            float* halo_row, float* halo_plane, unsigned int* prog, DevState* st,
                            uint64_t timeout_ns) {
    memset(&a, 0, sizeof(a));
    a.g = g;
    a.codes = const_cast<uint16_t*>(codes);
    a.out = out;
    a.opitch = g.N;
    a.halo_row = halo_row;
    a.halo_plane = halo_plane;
    a.prog = prog;
    a.st = st;
    a.timeout_ns = timeout_ns;
    a.tma_x = encode_tiles(&a.tm_x, false, codes, g.N, g.M, g.P, codes_pitch) ? 1 : 0;
    a.vec_out = ((reinterpret_cast<uintptr_t>(out) & 15) == 0 && (g.N * 4) % 16 == 0) ? 1 : 0;
}

int launch_wave_compress(const WaveGeom& g, int layers, const float* x, uint64_t x_pitch, uint16_t* codes,
                         uint64_t codes_pitch, float* recorded, float* halo_row, float* halo_plane,
                         unsigned int* prog, DevState* st, uint64_t timeout_ns, cudaStream_t s) {
    WaveArgs a;
    fill_compress(a, g, x, x_pitch, codes, codes_pitch, recorded, halo_row, halo_plane, prog, st, timeout_ns);
    return launch_any<false>(a, layers, s);
}

int launch_wave_decompress(const WaveGeom& g, int layers, const uint16_t* codes, uint64_t codes_pitch, float* out,
                           float* halo_row, float* halo_plane, unsigned int* prog, DevState* st,
                           uint64_t timeout_ns, cudaStream_t s) {
    WaveArgs a;
    fill_decompress(a, g, codes, codes_pitch, out, halo_row, halo_plane, prog, st, timeout_ns);
    if (!a.tma_x) return SZGB_ECUDA;  // the code array is row-pitched and aligned: never expected
    return launch_any<true>(a, layers, s);
}

// ---------------------------------------------------------------------------
// batched launch

size_t wave_args_bytes() { return sizeof(WaveArgs); }

void wave_args_compress(void* dst, const WaveGeom& g, const float* x, uint64_t x_pitch, uint16_t* codes,
                        uint64_t codes_pitch, float* halo_row, float* halo_plane, unsigned int* prog, DevState* st,
                        uint64_t timeout_ns) {
    fill_compress(*static_cast<WaveArgs*>(dst), g, x, x_pitch, codes, codes_pitch, nullptr, halo_row, halo_plane,
                  prog, st, timeout_ns);
}

int wave_args_decompress(void* dst, const WaveGeom& g, const uint16_t* codes, uint64_t codes_pitch, float* out,
                         float* halo_row, float* halo_plane, unsigned int* prog, DevState* st, uint64_t timeout_ns) {
    WaveArgs& a = *static_cast<WaveArgs*>(dst);
    fill_decompress(a, g, codes, codes_pitch, out, halo_row, halo_plane, prog, st, timeout_ns);
    return a.tma_x ? 0 : SZGB_ECUDA;
}

template <int NL, bool DEC>
static int launch_batch_t(const WaveArgs* F, const uint2* order, unsigned total, unsigned* ticket_dev, size_t smem,
                          int grid, int block, cudaStream_t s) {
    if (smem_limit_once<k_wave_batch<NL, DEC>>(smem)) return SZGB_ECUDA;
    k_wave_batch<NL, DEC><<<grid, block, smem, s>>>(F, order, total, ticket_dev);
    return cudaGetLastError() == cudaSuccess ? 0 : SZGB_ECUDA;
}

int launch_wave_batch(const void* args_dev, const void* order_dev, unsigned total, unsigned* ticket_dev, int layers,
                      bool decompress, size_t smem, int grid, cudaStream_t s) {
    const WaveArgs* F = static_cast<const WaveArgs*>(args_dev);
    const uint2* order = static_cast<const uint2*>(order_dev);
    const int block = (kMaxWaveWarps + 4) * 32;
    if (grid < 1) grid = 1;
    switch ((decompress ? 4 : 0) + layers - 1) {
        case 0: return launch_batch_t<1, false>(F, order, total, ticket_dev, smem, grid, block, s);
        case 1: return launch_batch_t<2, false>(F, order, total, ticket_dev, smem, grid, block, s);
        case 2: return launch_batch_t<3, false>(F, order, total, ticket_dev, smem, grid, block, s);
        case 3: return launch_batch_t<4, false>(F, order, total, ticket_dev, smem, grid, block, s);
        case 4: return launch_batch_t<1, true>(F, order, total, ticket_dev, smem, grid, block, s);
        case 5: return launch_batch_t<2, true>(F, order, total, ticket_dev, smem, grid, block, s);
        case 6: return launch_batch_t<3, true>(F, order, total, ticket_dev, smem, grid, block, s);
        case 7: return launch_batch_t<4, true>(F, order, total, ticket_dev, smem, grid, block, s);
        default: return SZGB_EUNSUPPORTED;
    }
}

}  // namespace szgb
