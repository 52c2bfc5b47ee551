// hyper_tile.cuh -- the hyperplane schedule for the predictors the wavefront
// does not carry (3D fields with n = 3, 4 layers; 4D fields with n = 1..4;
// Sec. III, Eq. predmodel), done tile by tile in shared memory.
//
// Every prediction term reaches back by a k != 0 with k >= 0 componentwise,
// so a point depends only on points whose coordinate sum is smaller.  The
// field is cut into tiles of TA x TI x TJ x TL points (3D: TI x TJ x TL);
// tile (A, I, J, L) depends only on tiles whose index sum is smaller, so all
// tiles with A + I + J + L = H run in one launch, in increasing H.  A tile's
// CTA
//   1. loads the box [lo - n, lo + T) of recorded values (zero outside the
//      field; the part below lo was written by earlier launches) and its own
//      input (compression: x; reconstruction: the codes and, at code 0, the
//      unpredictable values the row decoder left in the output),
//   2. walks its own hyperplanes a + i + j + l = s (tile-local coordinates),
//      one thread per tile row (a, i, j), one __syncthreads per step: the
//      prediction reads only shared memory,
//   3. stores its points' recorded values (and codes) with coalesced rows.
// The arithmetic is the wavefront's and the oracle's: the same term order
// (descending lexicographic k), every product and sum rounded once, the
// same quantizer and truncation; values outside the field are 0.
//
// The three phases are separate functions so that the host-side emulation
// test can run them thread by thread (within a step no thread reads a point
// another thread writes in that step: such points have equal coordinate
// sums, never a neighbour's).
#ifndef SZGB_HYPER_TILE_CUH
#define SZGB_HYPER_TILE_CUH

namespace szgb {

template <int DIM, int NL>
struct TileGeom {
    // tile extents: 3D 8 x 32 x 32; 4D 4 x 4 x 8 x 32 (2 x 4 x 8 x 32 for n >= 3,
    // whose halo is wider)
    static constexpr int TA = DIM == 4 ? (NL <= 2 ? 4 : 2) : 1;
    static constexpr int TI = DIM == 4 ? 4 : 8;
    static constexpr int TJ = DIM == 4 ? 8 : 32;
    static constexpr int TL = 32;
    static constexpr int HA = DIM == 4 ? NL : 0;  // halo planes along the 4th axis (3D: none)
    static constexpr int BA = TA + HA, BI = TI + NL, BJ = TJ + NL;
    // even row length: lanes on consecutive rows, whose columns differ by
    // one, land BL - 1 words apart, an odd stride (distinct banks)
    static constexpr int BL = (TL + NL + 1) & ~1;
    static constexpr int VBOX = BA * BI * BJ * BL;  // recorded values (floats)
    static constexpr int VPAD = (VBOX + 3) & ~3;    // floats before x / codes (16-byte offset)
    static constexpr int XBOX = TA * TI * TJ * TL;  // own points: x (floats) and codes (u16)
    static constexpr int THREADS = TA * TI * TJ;    // one thread per tile row
    static constexpr int STEPS = TA + TI + TJ + TL - 3;
    static constexpr size_t smem_bytes(bool dec) {
        return (size_t)VPAD * 4 + (dec ? 0 : (size_t)XBOX * 4) + (size_t)XBOX * 2;
    }
};

// one tile of one launch: its extents, arrays and first point
struct TileCtx {
    const float* x;
    float* V;
    uint16_t* codes;
    uint64_t cpitch;
    Dims4 d;                 // field extents D x P x M x N (3D: D = 1)
    int64_t a0, i0, j0, l0;  // the tile's first point
};

// Tile of block `blk` on tile diagonal H: box b over the tile grid (its
// (A, I, J) triples), nL tiles along the rows.  False when the block's L is
// outside the grid (the box is a superset).
template <int DIM, int NL>
__host__ __device__ __forceinline__ bool tile_at(const HyperBox4& b, int64_t H, int64_t nL, uint64_t blk,
                                                 TileCtx* t) {
    using G = TileGeom<DIM, NL>;
    const uint64_t plane = b.ni * b.nj;
    const int64_t A = b.alo + (int64_t)(blk / plane), I = b.ilo + (int64_t)((blk / b.nj) % b.ni),
                  J = b.jlo + (int64_t)(blk % b.nj), L = H - A - I - J;
    if (L < 0 || L >= nL) return false;
    t->a0 = A * G::TA;
    t->i0 = I * G::TI;
    t->j0 = J * G::TJ;
    t->l0 = L * G::TL;
    return true;
}

__host__ __device__ __forceinline__ uint64_t field_index(const Dims4& d, int64_t a, int64_t i, int64_t j, int64_t l) {
    return (((uint64_t)a * d.P + (uint64_t)i) * d.M + (uint64_t)j) * d.N + (uint64_t)l;
}

__host__ __device__ __forceinline__ uint64_t code_index(const Dims4& d, uint64_t cpitch, int64_t a, int64_t i,
                                                        int64_t j, int64_t l) {
    return (((uint64_t)a * d.P + (uint64_t)i) * d.M + (uint64_t)j) * cpitch + (uint64_t)l;
}

// Phase 1 for thread tid: the box of recorded values (compression skips the
// tile's own points, which it computes; reconstruction keeps them, since the
// unpredictable values are already there), and the tile's x or codes, as
// asynchronous copies that zero-fill what lies outside the field; the thread
// waits for its own copies (the caller's barrier then publishes them).
// Codes move 8 at a time: a tile row starts on a multiple of 8 codes and a
// code row's pitch is a multiple of 8, so a group that starts inside the row
// ends inside its pitch.
template <int DIM, int NL, bool DEC>
__device__ __forceinline__ void tile_load(const TileCtx& t, float* Vs, float* Xs, uint16_t* Cs, int tid) {
    using G = TileGeom<DIM, NL>;
    for (int e = tid; e < G::VBOX; e += G::THREADS) {
        int r = e;
        const int bl = r % G::BL;
        r /= G::BL;
        const int bj = r % G::BJ;
        r /= G::BJ;
        const int bi = r % G::BI;
        const int ba = r / G::BI;
        const int64_t a = t.a0 + ba - G::HA, i = t.i0 + bi - NL, j = t.j0 + bj - NL, l = t.l0 + bl - NL;
        const bool inside = bl < G::TL + NL && a >= 0 && i >= 0 && j >= 0 && l >= 0 && (uint64_t)a < t.d.D &&
                            (uint64_t)i < t.d.P && (uint64_t)j < t.d.M && (uint64_t)l < t.d.N;
        const bool own = a >= t.a0 && i >= t.i0 && j >= t.j0 && l >= t.l0;
        const bool take = inside && (DEC || !own);
        cp_async4(Vs + e, take ? t.V + field_index(t.d, a, i, j, l) : t.V, take ? 4 : 0);
    }
    if (DEC) {
        for (int e = tid; e < G::XBOX / 8; e += G::THREADS) {
            int r = e;
            const int tl = (r % (G::TL / 8)) * 8;
            r /= G::TL / 8;
            const int tj = r % G::TJ;
            r /= G::TJ;
            const int ti = r % G::TI;
            const int ta = r / G::TI;
            const int64_t a = t.a0 + ta, i = t.i0 + ti, j = t.j0 + tj, l = t.l0 + tl;
            const bool inside =
                (uint64_t)a < t.d.D && (uint64_t)i < t.d.P && (uint64_t)j < t.d.M && (uint64_t)l < t.d.N;
            cp_async16(Cs + 8 * e, inside ? t.codes + code_index(t.d, t.cpitch, a, i, j, l) : t.codes, inside ? 16 : 0);
        }
    } else {
        for (int e = tid; e < G::XBOX; e += G::THREADS) {
            int r = e;
            const int tl = r % G::TL;
            r /= G::TL;
            const int tj = r % G::TJ;
            r /= G::TJ;
            const int ti = r % G::TI;
            const int ta = r / G::TI;
            const int64_t a = t.a0 + ta, i = t.i0 + ti, j = t.j0 + tj, l = t.l0 + tl;
            const bool inside =
                (uint64_t)a < t.d.D && (uint64_t)i < t.d.P && (uint64_t)j < t.d.M && (uint64_t)l < t.d.N;
            cp_async4(Xs + e, inside ? t.x + field_index(t.d, a, i, j, l) : t.x, inside ? 4 : 0);
        }
    }
    cp_async_commit();
    cp_async_wait<0>();
}

// Term t of the n-layer predictor (t = 0, 1, ... in descending
// lexicographic order of k, the all-zero k excluded): digit `axis` of k.
// Term t is the number (n+1)^DIM - 1 - t written in base n + 1.
template <int DIM, int NL>
__host__ __device__ __forceinline__ constexpr int term_digit(int t, int axis) {
    int u = 1;
    for (int a = 0; a < DIM; a++) u *= NL + 1;
    u = u - 1 - t;
    for (int a = DIM - 1; a > axis; a--) u /= NL + 1;
    return u % (NL + 1);
}

// n-layer prediction of the point at box index ve from the box of recorded
// values: terms in descending lexicographic order of k, each product and sum
// rounded once.  The values of 32 terms at a time are read first (so that
// their shared-memory loads overlap), then summed in that order.
template <int DIM, int NL>
__device__ __forceinline__ float predict_tile(const float* Vs, int ve) {
    using G = TileGeom<DIM, NL>;
    constexpr int T = DIM == 3 ? (NL + 1) * (NL + 1) * (NL + 1) - 1 : (NL + 1) * (NL + 1) * (NL + 1) * (NL + 1) - 1;
    constexpr int GRP = 32;
    float pred = 0.0f;
#pragma unroll
    for (int g0 = 0; g0 < T; g0 += GRP) {
        float v[GRP];
#pragma unroll
        for (int q = 0; q < GRP; q++) {
            const int t = g0 + q;
            if (t < T) {
                const int off = DIM == 3 ? (term_digit<DIM, NL>(t, 0) * G::BJ + term_digit<DIM, NL>(t, 1)) * G::BL +
                                               term_digit<DIM, NL>(t, 2)
                                         : ((term_digit<DIM, NL>(t, 0) * G::BI + term_digit<DIM, NL>(t, 1)) * G::BJ +
                                            term_digit<DIM, NL>(t, 2)) * G::BL + term_digit<DIM, NL>(t, 3);
                v[q] = Vs[ve - off];
            }
        }
#pragma unroll
        for (int q = 0; q < GRP; q++) {
            const int t = g0 + q;
            if (t < T) {
                const int c = DIM == 3 ? term_coef(NL, term_digit<DIM, NL>(t, 0), term_digit<DIM, NL>(t, 1),
                                                   term_digit<DIM, NL>(t, 2))
                                       : term_coef4(NL, term_digit<DIM, NL>(t, 0), term_digit<DIM, NL>(t, 1),
                                                    term_digit<DIM, NL>(t, 2), term_digit<DIM, NL>(t, 3));
                const float prod = __fmul_rn((float)c, v[q]);
                pred = t == 0 ? prod : __fadd_rn(pred, prod);
            }
        }
    }
    return pred;
}

// Phase 2, step s, thread tid: the point of its row on tile hyperplane s.
template <int DIM, int NL, bool DEC>
__device__ __forceinline__ void tile_step(const TileCtx& t, float* Vs, const float* Xs, uint16_t* Cs, int tid, int s,
                                          const QParams& qp) {
    using G = TileGeom<DIM, NL>;
    const int tj = tid % G::TJ, ti = (tid / G::TJ) % G::TI, ta = tid / (G::TJ * G::TI);
    const int tl = s - ta - ti - tj;
    if (tid >= G::THREADS || tl < 0 || tl >= G::TL) return;
    if ((uint64_t)(t.a0 + ta) >= t.d.D || (uint64_t)(t.i0 + ti) >= t.d.P || (uint64_t)(t.j0 + tj) >= t.d.M ||
        (uint64_t)(t.l0 + tl) >= t.d.N)
        return;
    const int ve = (((ta + G::HA) * G::BI + ti + NL) * G::BJ + tj + NL) * G::BL + tl + NL;
    const int xe = ((ta * G::TI + ti) * G::TJ + tj) * G::TL + tl;
    const float pred = predict_tile<DIM, NL>(Vs, ve);
    if (DEC) {
        const int code = Cs[xe];
        if (code) Vs[ve] = dequantize(code, pred, qp);
    } else {
        const float xv = Xs[xe];
        float rec;
        const int code = quantize_tr(xv, pred, trunc_value(xv, qp.e_eb), qp, rec);
        Vs[ve] = rec;
        Cs[xe] = (uint16_t)code;
    }
}

// Phase 3 for thread tid: the tile's recorded values (and codes) to global
// memory, rows of TL points.
template <int DIM, int NL, bool DEC>
__device__ __forceinline__ void tile_store(const TileCtx& t, const float* Vs, const uint16_t* Cs, int tid) {
    using G = TileGeom<DIM, NL>;
    for (int e = tid; e < G::XBOX; e += G::THREADS) {
        int r = e;
        const int tl = r % G::TL;
        r /= G::TL;
        const int tj = r % G::TJ;
        r /= G::TJ;
        const int ti = r % G::TI;
        const int ta = r / G::TI;
        const int64_t a = t.a0 + ta, i = t.i0 + ti, j = t.j0 + tj, l = t.l0 + tl;
        if ((uint64_t)a >= t.d.D || (uint64_t)i >= t.d.P || (uint64_t)j >= t.d.M || (uint64_t)l >= t.d.N) continue;
        const int ve = (((ta + G::HA) * G::BI + ti + NL) * G::BJ + tj + NL) * G::BL + tl + NL;
        t.V[field_index(t.d, a, i, j, l)] = Vs[ve];
        if (!DEC) t.codes[code_index(t.d, t.cpitch, a, i, j, l)] = Cs[e];
    }
}

}  // namespace szgb

#endif
