// hyper_emulate.cpp -- the hyperplane kernels' own device code
// (paper_1706_03791_gb300/csrc/hyper_tile.cuh and hyper_kernels.cuh), run on
// the host tile by tile, step by step, thread by thread, against the oracle: codes and recorded
// values of 3D fields with n = 3, 4 and of 4D fields with n = 1..4, their
// reconstruction from the codes and the unpredictable values, the 4D
// adaptive-m choice and the 4D prediction hit counts.  The CUDA intrinsics the kernels use are given their
// IEEE meaning (every product and sum rounded once, no contraction: build
// with -ffp-contract=off); the quantizer helpers are host transcriptions of
// the library's device helpers.
//
// Usage: hyper_emulate  -> "cases N failures F", exit status 0 iff F == 0.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <vector>

#define __global__
#define __device__
#define __host__
#define __forceinline__ inline
#define __launch_bounds__(x)

struct EmuIndex {
    unsigned x;
};
static EmuIndex blockIdx, threadIdx;

static inline float __fmul_rn(float a, float b) { return a * b; }
static inline float __fadd_rn(float a, float b) { return a + b; }
static inline float __fsub_rn(float a, float b) { return a - b; }
static inline float __ldg(const float* p) { return *p; }
static inline float __ldcg(const float* p) { return *p; }
static inline uint32_t __float_as_uint(float f) {
    uint32_t u;
    std::memcpy(&u, &f, 4);
    return u;
}
static inline float __uint_as_float(uint32_t u) {
    float f;
    std::memcpy(&f, &u, 4);
    return f;
}

namespace szgb {

struct DevState {
    unsigned err;
    float eb_f, twoeb, inv2eb, radius;
    int center, e_eb;
};
struct QParams {
    float eb, twoeb, inv, radius;
    int center, e_eb;
};
inline QParams load_qparams(const DevState* st) {
    return QParams{st->eb_f, st->twoeb, st->inv2eb, st->radius, st->center, st->e_eb};
}
constexpr int binom_c(int n, int k) {
    if (k < 0 || k > n) return 0;
    int r = 1;
    for (int i = 1; i <= k; i++) r = r * (n - i + 1) / i;
    return r;
}
constexpr int sgn_binom(int n, int k) { return ((k & 1) ? -1 : 1) * binom_c(n, k); }
constexpr int term_coef(int n, int k0, int k1, int k2) { return -sgn_binom(n, k0) * sgn_binom(n, k1) * sgn_binom(n, k2); }
inline int trunc_bits(uint32_t u, int e_eb) {
    if (e_eb == 0) return 23;
    int e = (int)((u >> 23) & 0xffu);
    e = e < 1 ? 1 : e;
    int t = e - e_eb;
    t = t < 0 ? 0 : t;
    return t > 23 ? 23 : t;
}
inline float trunc_value(float x, int e_eb) {
    const uint32_t u = __float_as_uint(x);
    const int t = trunc_bits(u, e_eb);
    return __uint_as_float(u & ~((1u << (23 - t)) - 1u));
}
inline int quantize_tr(float x, float pred, float tr, const QParams& qp, float& V) {
    const float diff = __fsub_rn(x, pred);
    const float q = std::rintf(__fmul_rn(diff, qp.inv));
    const float qn = __fadd_rn(q, 0.0f);
    const float dq = __fadd_rn(pred, __fmul_rn(qn, qp.twoeb));
    const float err = __fsub_rn(x, dq);
    const bool ok = (std::fabs(q) <= qp.radius) & ((std::fabs(err) < qp.eb) | (x == dq));
    V = ok ? dq : tr;
    return ok ? ((int)qn + qp.center) : 0;
}
// asynchronous global->shared copies: on the host, an immediate copy of
// src_bytes and zeros for the rest
inline void cp_async4(void* dst, const void* src, int src_bytes) {
    std::memset(dst, 0, 4);
    if (src_bytes) std::memcpy(dst, src, (size_t)src_bytes);
}
inline void cp_async16(void* dst, const void* src, int src_bytes) {
    std::memset(dst, 0, 16);
    if (src_bytes) std::memcpy(dst, src, (size_t)src_bytes);
}
inline void cp_async_commit() {}
template <int N>
inline void cp_async_wait() {}
inline float dequantize(int code, float pred, const QParams& qp) {
    const float qf = (float)(code - qp.center);
    return __fadd_rn(pred, __fmul_rn(qf, qp.twoeb));
}

}  // namespace szgb

#include "../../paper_1706_03791_gb300/csrc/hyper_box.h"
#include "../../paper_1706_03791_gb300/csrc/hyper_kernels.cuh"
#include "../../paper_1706_03791_gb300/csrc/hyper_tile.cuh"

extern "C" {
#include "../../oracle/szo.h"
}

using namespace szgb;

namespace {

uint64_t rs = 88172645463325252ull;
double urand() {
    rs ^= rs << 13;
    rs ^= rs >> 7;
    rs ^= rs << 17;
    return (double)(rs >> 11) / 9007199254740992.0;
}

// a smooth field with noise and a few outliers
std::vector<float> make_field(const std::vector<uint64_t>& shape) {
    uint64_t n = 1;
    for (uint64_t e : shape) n *= e;
    std::vector<float> x(n);
    for (uint64_t p = 0; p < n; p++) {
        uint64_t r = p;
        double v = 0.0;
        for (size_t a = shape.size(); a-- > 0;) {
            const double c = (double)(r % shape[a]) / (double)shape[a];
            r /= shape[a];
            v += std::sin(2.0 * c + (double)a) * (0.5 + 0.1 * (double)a);
        }
        v += 1e-3 * urand() + (urand() < 0.01 ? 5.0 : 0.0);
        x[p] = (float)v;
    }
    return x;
}

DevState state_for(const std::vector<float>& x, int mode, double eb_abs, double eb_rel, int m) {
    float mn = x[0], mx = x[0];
    for (float v : x) {
        mn = v < mn ? v : mn;
        mx = v > mx ? v : mx;
    }
    float ebf = 0.0f;
    szo_effective_eb(mode, eb_abs, eb_rel, mn + 0.0f, mx + 0.0f, &ebf);
    DevState st = {};
    st.eb_f = ebf;
    st.twoeb = 2.0f * ebf;
    st.inv2eb = ebf > 0.0f ? 1.0f / st.twoeb : 0.0f;
    st.e_eb = (int)((__float_as_uint(ebf) >> 23) & 0xffu);
    st.center = 1 << (m - 1);
    st.radius = (float)((1 << (m - 1)) - 1);
    return st;
}

// the tiled schedule, tile by tile and thread by thread: every thread's load,
// then every step of every thread, then every thread's store (no thread reads
// a point another thread writes in the same step)
template <int DIM, int NL, bool DEC>
void emulate_tiles(const float* x, float* V, uint16_t* codes, uint64_t cpitch, const Dims4& d, const DevState* st) {
    using G = TileGeom<DIM, NL>;
    const int64_t nA = (int64_t)((d.D + G::TA - 1) / G::TA), nI = (int64_t)((d.P + G::TI - 1) / G::TI),
                  nJ = (int64_t)((d.M + G::TJ - 1) / G::TJ), nL = (int64_t)((d.N + G::TL - 1) / G::TL);
    std::vector<float> Vs(G::VBOX), Xs(G::XBOX);
    std::vector<uint16_t> Cs(G::XBOX);
    const QParams qp = load_qparams(st);
    for (int64_t H = 0; H <= (nA - 1) + (nI - 1) + (nJ - 1) + (nL - 1); H++) {
        const HyperBox4 b = hyper_box4(H, nA, nI, nJ, nL);
        for (uint64_t blk = 0; blk < b.na * b.ni * b.nj; blk++) {
            TileCtx t = {x, V, codes, cpitch, d, 0, 0, 0, 0};
            if (!tile_at<DIM, NL>(b, H, nL, blk, &t)) continue;
            std::fill(Vs.begin(), Vs.end(), std::nanf(""));
            for (int tid = 0; tid < G::THREADS; tid++) tile_load<DIM, NL, DEC>(t, Vs.data(), Xs.data(), Cs.data(), tid);
            for (int s = 0; s < G::STEPS; s++)
                for (int tid = 0; tid < G::THREADS; tid++)
                    tile_step<DIM, NL, DEC>(t, Vs.data(), Xs.data(), Cs.data(), tid, s, qp);
            for (int tid = 0; tid < G::THREADS; tid++) tile_store<DIM, NL, DEC>(t, Vs.data(), Cs.data(), tid);
        }
    }
}

template <int NL>
int adapt4_m(const float* x, const Dims4& d, const DevState& st, double theta) {
    const uint64_t S = ((d.D + 7) / 8) * ((d.P + 7) / 8) * ((d.M + 7) / 8) * ((d.N + 7) / 8);
    uint64_t need[18] = {};
    for (uint64_t s = 0; s < S; s++) {
        const int mm = adapt4_bucket<NL>(x, d, s, st.eb_f, st.twoeb, st.inv2eb);
        if (mm) need[mm]++;
    }
    const double req = std::ceil(theta * (double)S);
    uint64_t cum = 0;
    for (int mm = 2; mm <= 16; mm++) {
        cum += need[mm];
        if ((double)cum >= req) return mm;
    }
    return 16;
}

// one field: emulated codes / recorded values / reconstruction against the oracle
template <int NL>
int run_case(const std::vector<uint64_t>& shape, int mode, double eb_abs, double eb_rel, int m_user) {
    const int nd = (int)shape.size();
    std::vector<float> x = make_field(shape);
    const uint64_t n = x.size();
    // the oracle with the same m (its choice when adaptive)
    int m = m_user;
    float ebf = 0.0f;
    {
        float mn = x[0], mx = x[0];
        for (float v : x) {
            mn = v < mn ? v : mn;
            mx = v > mx ? v : mx;
        }
        szo_effective_eb(mode, eb_abs, eb_rel, mn + 0.0f, mx + 0.0f, &ebf);
    }
    if (m == 0) m = szo_choose_m(x.data(), nd, shape.data(), NL, ebf, 0.99);
    std::vector<uint8_t> out(szo_stream_bound(nd, shape.data()));
    std::vector<float> rec(n);
    std::vector<uint16_t> code_ref(n);
    size_t olen = 0;
    if (szo_compress(x.data(), nd, shape.data(), mode, eb_abs, eb_rel, NL, m, 0.99, 0, out.data(), out.size(), &olen,
                     rec.data(), code_ref.data()) != 0)
        return 10;
    const DevState st = state_for(x, mode, eb_abs, eb_rel, m);
    if (st.eb_f != ebf) return 11;
    const uint64_t N = shape[nd - 1], rows = n / N, cpitch = (N + 7) & ~(uint64_t)7;
    std::vector<float> V(n, std::nanf(""));
    std::vector<uint16_t> codes(rows * cpitch, 0xffffu);
    Dims4 d = {1, 1, 1, 1};
    if (nd == 4) d = {shape[0], shape[1], shape[2], shape[3]};
    if (nd == 4) {
        if (m_user == 0 && adapt4_m<NL>(x.data(), d, st, 0.99) != m) return 12;
        emulate_tiles<4, NL, false>(x.data(), V.data(), codes.data(), cpitch, d, &st);
    } else {
        emulate_tiles<3, NL, false>(x.data(), V.data(), codes.data(), cpitch, {1, shape[0], shape[1], shape[2]}, &st);
    }
    for (uint64_t p = 0; p < n; p++) {
        if (codes[(p / N) * cpitch + p % N] != code_ref[p]) return 13;
        if (__float_as_uint(V[p]) != __float_as_uint(rec[p])) return 14;
    }
    // reconstruction: the row decoder leaves the unpredictable values in place
    std::vector<float> Y(n, std::nanf(""));
    for (uint64_t p = 0; p < n; p++)
        if (code_ref[p] == 0) Y[p] = rec[p];
    if (nd == 4) emulate_tiles<4, NL, true>(nullptr, Y.data(), codes.data(), cpitch, d, &st);
    else emulate_tiles<3, NL, true>(nullptr, Y.data(), codes.data(), cpitch, {1, shape[0], shape[1], shape[2]}, &st);
    for (uint64_t p = 0; p < n; p++)
        if (__float_as_uint(Y[p]) != __float_as_uint(rec[p])) return 15;
    if (nd == 4) {
        // prediction hits (Sec. III) from original and from recorded values
        std::vector<float> pred(n);
        for (int which = 0; which < 2; which++) {
            const float* V0 = which ? rec.data() : x.data();
            if (szo_predict_field(V0, 4, shape.data(), NL, pred.data()) != 0) return 16;
            uint64_t ref = 0, got = 0;
            for (uint64_t p = 0; p < n; p++) {
                ref += std::fabs((double)x[p] - (double)pred[p]) <= (double)ebf;
                got += hit4_point<NL>(x.data(), V0, d, p, (double)ebf);
            }
            if (got != ref) return 17;
        }
    }
    return 0;
}

}  // namespace

int main() {
    int cases = 0, bad = 0;
    auto check = [&](int r, const char* what) {
        cases++;
        if (r) {
            std::printf("%s: failure %d\n", what, r);
            bad++;
        }
    };
    // 3D, n = 3 and 4
    check(run_case<3>({7, 9, 11}, 1, 0.0, 1e-3, 0), "3d n3 rel adaptive");
    check(run_case<3>({5, 13, 6}, 0, 1e-3, 0.0, 8), "3d n3 abs m8");
    check(run_case<4>({6, 8, 10}, 1, 0.0, 1e-4, 0), "3d n4 rel adaptive");
    check(run_case<4>({1, 1, 40}, 1, 0.0, 1e-3, 10), "3d n4 unit extents");
    check(run_case<3>({9, 2, 17}, 2, 1e-3, 1e-4, 0), "3d n3 both");
    check(run_case<3>({20, 30, 7}, 1, 0.0, 1e-4, 0), "3d n3 boxes of several blocks");
    check(run_case<4>({18, 17, 5}, 1, 0.0, 1e-6, 16), "3d n4 m16 several blocks");
    // 4D, n = 1..4, adaptive m checked against the oracle's choice
    check(run_case<1>({5, 6, 7, 9}, 1, 0.0, 1e-3, 0), "4d n1");
    check(run_case<2>({4, 7, 6, 11}, 1, 0.0, 1e-4, 0), "4d n2");
    check(run_case<3>({6, 5, 5, 8}, 1, 0.0, 1e-3, 8), "4d n3 m8");
    check(run_case<4>({5, 5, 6, 6}, 0, 1e-3, 0.0, 0), "4d n4 abs");
    check(run_case<2>({1, 1, 3, 40}, 1, 0.0, 1e-4, 0), "4d unit");
    check(run_case<1>({9, 10, 9, 17}, 1, 0.0, 1e-4, 0), "4d samples");
    check(run_case<3>({8, 9, 8, 9}, 2, 1e-3, 1e-5, 0), "4d n3 both, several blocks");
    // several tiles along every axis, each with a ragged last tile
    check(run_case<3>({19, 37, 70}, 1, 0.0, 1e-4, 0), "3d n3 3x3x3 tiles");
    check(run_case<4>({17, 33, 65}, 1, 0.0, 1e-5, 0), "3d n4 3x3x3 tiles");
    check(run_case<1>({9, 10, 17, 40}, 1, 0.0, 1e-4, 0), "4d n1 3x3x3x2 tiles");
    check(run_case<2>({9, 6, 9, 33}, 0, 1e-3, 0.0, 0), "4d n2 3x2x2x2 tiles");
    check(run_case<4>({5, 9, 17, 33}, 1, 0.0, 1e-4, 0), "4d n4 3x3x3x2 tiles");
    std::printf("cases %d failures %d\n", cases, bad);
    return bad ? 1 : 0;
}
