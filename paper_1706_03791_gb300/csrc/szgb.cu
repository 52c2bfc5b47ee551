// szgb.cu -- the C ABI: context, device scratch, and the compress /
// decompress pipelines.
//
// compress:   range + bound (K1) -> adaptive m (K8, when m = 0) -> wavefront
//             predict + quantize (K2) -> histogram (K3) -> codebook (K4) ->
//             row bit lengths -> row offsets -> header/codebook/table ->
//             payload (K5).
// decompress: header (host) -> decoder tables -> row offsets -> wavefront
//             decode + reconstruct (K6 fused into K7).
// Every launch goes to the context's stream; a call returns after one
// stream synchronisation at its end.
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <vector>

#include "szgb_internal.cuh"

using namespace szgb;

namespace {

enum Phase {
    PH_H2D = 0, PH_RANGE, PH_ADAPT, PH_WAVE_C, PH_HIST, PH_CODEBOOK, PH_ROWBITS, PH_SCAN, PH_WRITE,
    PH_D2H, PH_DEC_TABLES, PH_DEC_SCAN, PH_WAVE_D, PH_DEC_ROWS, PH_N
};
const char* kPhaseNames[PH_N] = {"h2d", "range", "adapt", "wave_compress", "histogram", "codebook",
                                  "rowbits", "scan", "write", "d2h", "decode_tables", "decode_scan",
                                  "wave_decompress", "decode_rows"};

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

struct Arena {
    // offsets into the scratch allocation
    std::vector<std::pair<void**, size_t>> items;
    size_t total = 0;
    template <typename T>
    void add(T** p, size_t count) {
        items.push_back({reinterpret_cast<void**>(p), total});
        total = align_up(total + std::max<size_t>(count * sizeof(T), 1), 256);
    }
    void bind(void* base) {
        for (auto& it : items) *it.first = static_cast<char*>(base) + it.second;
    }
};

}  // namespace

constexpr int kAux = 8;  // auxiliary streams of the batched paths

// A captured batch: the arguments it was captured with and its executable graph.
struct BatchGraph {
    std::vector<uint64_t> key;
    cudaGraphExec_t exec = nullptr;
};

struct szgb_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t own_stream = nullptr;
    size_t budget = 0;
    void* scratch = nullptr;
    size_t scratch_cap = 0;
    DevState* h_state = nullptr;  // pinned: [0] state read back, [1] initial state, then the header bytes
    DevState* h_init = nullptr;
    uint8_t* h_hdr = nullptr;
    bool profiling = false;
    double ph_ms[PH_N] = {};
    uint64_t ph_calls[PH_N] = {};
    cudaEvent_t ev0[PH_N] = {}, ev1[PH_N] = {};
    int sm_count = 152;
    int W2 = 8, W3 = 8;
    uint64_t timeout_ns = 4000000000ull;
    // batched paths
    cudaStream_t aux[kAux] = {};
    cudaEvent_t ev_fork = nullptr, ev_join[kAux] = {};
    void* h_batch = nullptr;  // pinned host tables of a batch
    size_t h_batch_cap = 0;
    bool use_graphs = true;
    BatchGraph g_comp, g_dec;
    // autotuned wavefront shapes per shape class (see shape_class)
    struct Tune {
        int W;
        uint32_t chunk;  // requested chunk length (SZGB_CHUNK_ROWS: whole rows)
        double ms;
    };
    std::map<uint64_t, Tune> tune;
    int force_W = 0;            // set while the autotuner times a candidate
    uint32_t force_chunk = 0;   // likewise (a requested chunk length; 0: none)
    int debug_skip = 0;  // test hook: 1 + the wavefront work item never run; 0 = none
    int wave_ctas = 0;   // most CTAs of a persistent wavefront launch (0: one per SM)
};

namespace {

struct PhaseTimer {
    szgb_ctx* c;
    int ph;
    PhaseTimer(szgb_ctx* c_, int ph_) : c(c_), ph(ph_) {
        if (c->profiling) cudaEventRecord(c->ev0[ph], c->stream);
    }
    ~PhaseTimer() {
        if (!c->profiling) return;
        cudaEventRecord(c->ev1[ph], c->stream);
        cudaEventSynchronize(c->ev1[ph]);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, c->ev0[ph], c->ev1[ph]);
        c->ph_ms[ph] += ms;
        c->ph_calls[ph]++;
    }
};

int ensure_scratch(szgb_ctx* c, size_t need) {
    if (need <= c->scratch_cap) return SZGB_OK;
    if (c->budget && need > c->budget) return SZGB_EBUDGET;
    const size_t old_cap = c->scratch_cap;
    if (c->scratch) {
        cudaStreamSynchronize(c->stream);
        cudaFree(c->scratch);
        c->scratch = nullptr;
        c->scratch_cap = 0;
    }
    // grow at least twofold: a regrowth frees the old block, and cudaFree
    // waits for all work on the device
    size_t cap = align_up(std::max(need + need / 8, 2 * old_cap), 1 << 20);
    if (c->budget && cap > c->budget) cap = c->budget;  // need <= budget
    if (cudaMalloc(&c->scratch, cap) != cudaSuccess) {
        cudaGetLastError();
        return SZGB_ENOMEM;
    }
    c->scratch_cap = cap;
    return SZGB_OK;
}

// The chunk length a request gives a row of row_len points: 0 (whole rows)
// unless it is a power of two shorter than the row; the lattice variant codes
// whole rows.
uint32_t effective_chunk(uint32_t req, uint64_t row_len, int variant) {
    if (variant != SZGB_VARIANT_EXACT || req == 0 || req == SZGB_CHUNK_ROWS || req >= row_len) return 0;
    return req;
}

// A 4D field D x P x M x N becomes its (D P) x M x N view with cp->D4 = D:
// its rows of N points are coded as the view's (Sec. III with d = 4).
int check_params(const szgb_params* p, CallParams* cp) {
    if (!p || p->ndim < 1 || p->ndim > 4) return SZGB_EINVAL;
    for (int a = 0; a < p->ndim; a++)
        if (p->shape[a] == 0 || p->shape[a] > 0xffffffffull) return SZGB_EINVAL;
    uint64_t d[3] = {1, 1, 1};
    cp->D4 = 0;
    if (p->ndim == 4) {
        if (p->shape[0] * p->shape[1] > 0xffffffffull) return SZGB_EINVAL;
        d[0] = p->shape[0] * p->shape[1];
        d[1] = p->shape[2];
        d[2] = p->shape[3];
        cp->D4 = p->shape[0];
    } else {
        for (int a = 0; a < p->ndim; a++) d[3 - p->ndim + a] = p->shape[a];
    }
    unsigned __int128 n = (unsigned __int128)d[0] * d[1] * d[2];
    if (n >= ((unsigned __int128)1 << 32)) return SZGB_EINVAL;
    if (p->mode < 0 || p->mode > 2) return SZGB_EINVAL;
    if (p->mode != SZGB_REL && !(p->eb_abs >= 0.0)) return SZGB_EINVAL;
    if (p->mode != SZGB_ABS && !(p->eb_rel >= 0.0)) return SZGB_EINVAL;
    if (p->m != 0 && (p->m < 2 || p->m > 16)) return SZGB_EINVAL;
    if (p->layers < 1 || p->layers > 4) return SZGB_EINVAL;
    if (p->m == 0 && !(p->theta == p->theta)) return SZGB_EINVAL;
    cp->ndim = p->ndim == 4 ? 3 : p->ndim;
    cp->d0 = d[0];
    cp->d1 = d[1];
    cp->d2 = d[2];
    cp->mode = p->mode;
    cp->eb_abs = p->eb_abs;
    cp->eb_rel = p->eb_rel;
    cp->layers = p->layers;
    cp->m_user = p->m;
    cp->theta = p->theta;
    if (p->variant != SZGB_VARIANT_EXACT && p->variant != SZGB_VARIANT_LATTICE) return SZGB_EINVAL;
    cp->variant = p->variant;
    const uint32_t c = p->chunk_points;
    if (!(c == 0 || c == SZGB_CHUNK_ROWS || (c >= 32 && (c & (c - 1)) == 0))) return SZGB_EINVAL;
    cp->chunk = effective_chunk(c, cp->d2, cp->variant);
    // the lattice variant is built for 1D-3D with n <= 2; the autotuner
    // checks the wavefront's set (wave_carries) too
    if (p->variant == SZGB_VARIANT_LATTICE && (p->layers > 2 || p->ndim == 4)) return SZGB_EUNSUPPORTED;
    return SZGB_OK;
}

// Shape class of a field for the autotuner: dimension, layers and the bit
// lengths of the extents that set the wavefront's shape (3D: planes, rows,
// columns; 1D/2D: rows, columns).
uint64_t shape_class(const CallParams& cp, int layers) {
    auto bl = [](uint64_t v) { uint64_t b = 0; while (v) { b++; v >>= 1; } return b; };
    const uint64_t rows = cp.ndim == 3 ? cp.d1 : cp.d0 * cp.d1;
    const uint64_t planes = cp.ndim == 3 ? cp.d0 : 1;
    return ((uint64_t)cp.ndim << 56) | ((uint64_t)layers << 48) | (bl(planes) << 32) | (bl(rows) << 16) | bl(cp.d2);
}

// chunk_points = 0 takes the autotuned chunk length of the field's shape
// class (whole rows when there is none); a candidate being timed wins
void resolve_chunk(const szgb_ctx* c, const szgb_params* p, CallParams* cp) {
    uint32_t req = p->chunk_points;
    if (req == 0) {
        auto it = c->tune.find(shape_class(*cp, cp->layers));
        if (it != c->tune.end()) req = it->second.chunk;
    }
    if (c->force_chunk) req = c->force_chunk;
    cp->chunk = effective_chunk(req, cp->d2, cp->variant);
}

WaveGeom make_geom(const szgb_ctx* c, const CallParams& cp, int layers) {
    int W2 = c->W2, W3 = c->W3;
    auto it = c->tune.find(shape_class(cp, layers));
    if (it != c->tune.end()) {
        W2 = W3 = it->second.W;
    }
    if (c->force_W) W2 = W3 = c->force_W;
    WaveGeom g = make_geom_w(cp, layers, W2, W3);
    g.debug_skip = c->debug_skip;
    return g;
}

}  // namespace

WaveGeom szgb::make_geom_w(const CallParams& cp, int layers, int W2, int W3) {
    WaveGeom g = {};
    g.N = cp.d2;
    g.ntiles = (int)((cp.d2 + kTile - 1) / kTile);
    g.aligned = (cp.d2 % 4) == 0;
    if (cp.ndim == 3) {
        g.ndim = 3;
        g.P = cp.d0;
        g.M = cp.d1;
        int W = W3;
        if ((uint64_t)W > cp.d0) W = (int)cp.d0;
        if (W < 2 * layers) W = 2 * layers;  // the plane halo's rows all have sweeps >= 0
        g.W = W;
        g.nb0 = (int)((cp.d0 + W - 1) / W);
        g.nb1 = (int)((cp.d1 + 31) / 32);
        g.nsweeps = (int)((cp.d2 - 1 + 31 + 4 * (W - 1)) / 4) + 1;  // last step: column N-1 of warp W-1, lane 31
    } else {
        g.ndim = cp.ndim;
        g.P = 1;
        g.M = cp.d0 * cp.d1;  // 1D: a single row
        int W = W2;
        int need = (int)((g.M + 31) / 32);
        if (W > need) W = need;
        if (W < 1) W = 1;
        g.W = W;
        g.nb0 = 1;
        g.nb1 = (int)((g.M + 32ull * W - 1) / (32ull * W));
        g.nsweeps = (int)((cp.d2 - 1 + 31 + 36 * (W - 1)) / 4) + 1;  // last step: column N-1 of warp W-1, lane 31
    }
    g.num_ctas = g.nb0 * g.nb1;
    return g;
}

namespace {

// Halo line sizes in 32-bit units: every value travels as one 64-bit tagged
// word.  The plane halo follows the row halo in one allocation (one memset
// per launch); both counts are multiples of 64 (256-byte offsets).
}  // namespace

void szgb::halo_sizes(const WaveGeom& g, int layers, size_t* row_words, size_t* plane_words) {
    size_t tpr = (size_t)g.ntiles * kTile;
    size_t r, p;
    if (g.ndim == 3) {
        r = (size_t)g.P * g.nb1 * layers * tpr;
        p = (size_t)g.nb0 * g.nb1 * layers * 32 * (tpr + 32);
    } else {
        r = (size_t)g.nb1 * layers * tpr;
        p = 4;
    }
    *row_words = align_up(2 * r, 64);
    *plane_words = align_up(2 * p, 64);
}

namespace {

}  // namespace

int szgb::dev_errors(const DevState& s) {
    if (s.err & kErrNonFinite) return SZGB_ENONFINITE;
    if (s.err & kErrRange) return SZGB_EINVAL;
    if (s.err & kErrTimeout) return SZGB_ETIMEOUT;
    if (s.err & kErrCorrupt) return SZGB_ECORRUPT;
    if (s.err & kErrOverflow) return SZGB_ETRUNC;
    return SZGB_OK;
}

namespace {

// ---------------------------------------------------------------------------
// compress

int ensure_pinned(szgb_ctx* c, size_t need);

// a 64-byte aligned host buffer for one field's wavefront arguments (they
// hold TMA descriptors, which need that alignment)
struct ArgsBuf {
    std::vector<unsigned char> buf;
    void* p;
    explicit ArgsBuf(size_t n) : buf(n + 64) {
        p = reinterpret_cast<void*>((reinterpret_cast<uintptr_t>(buf.data()) + 63) & ~(uintptr_t)63);
    }
};

int launch_wave_one(szgb_ctx* c, const WaveGeom& g, int layers, bool dec, const void* host_args, char* stage,
                    char* dev_args, uint32_t* dev_order, unsigned* dev_ticket, cudaStream_t s);
int compress_batch_impl(szgb_ctx* c, int count, const float* const* data, const szgb_params* params,
                        uint8_t* const* out, const size_t* out_cap, size_t* out_len, szgb_stats* stats);
int decompress_batch_impl(szgb_ctx* c, int count, const uint8_t* const* in, const size_t* in_len,
                          float* const* out, const size_t* out_cap, int* status, const uint8_t* host_hdr = nullptr);

// grid of a persistent wavefront launch over n work items: one CTA per SM,
// at most the context's cap
int wave_grid(const szgb_ctx* c, size_t n) {
    size_t cap = (size_t)c->sm_count;
    if (c->wave_ctas > 0 && (size_t)c->wave_ctas < cap) cap = (size_t)c->wave_ctas;
    return (int)std::min(n, cap);
}

// A single device-resident field of the paper's method takes the batched
// path (one field): its whole pass is captured once in a CUDA graph and
// replayed, which removes most of the per-call launch gaps.  Profiled runs
// (per-kernel phase events), test hooks and autotuning candidates keep the
// direct path.
bool one_field_batched(const szgb_ctx* c) {
    return c->use_graphs && !c->profiling && !c->force_W && !c->debug_skip;
}

// a 4D field runs on its (D4 P) x M x N view (cp.D4 = D4)
int compress_impl(szgb_ctx* c, const float* data, int data_on_device, const szgb_params* p, uint8_t* out,
                  size_t out_cap, int out_on_device, size_t* out_len, szgb_stats* stats, float* rec_dev,
                  uint16_t* codes_dev) {
    if (!c || !data || !out_len) return SZGB_EINVAL;
    if (((uintptr_t)rec_dev % 16) != 0 || ((uintptr_t)codes_dev % 8) != 0) return SZGB_EINVAL;
    CallParams cp;
    int rc = check_params(p, &cp);
    if (rc) return rc;
    resolve_chunk(c, p, &cp);
    // 3D fields with n = 3, 4, and 4D fields: the hyperplane kernels instead of the wavefront
    const uint64_t D4 = cp.D4;
    const bool hyper = cp.variant == SZGB_VARIANT_EXACT && !wave_carries(cp);
    if (one_field_batched(c) && !hyper && !rec_dev && !codes_dev && cp.variant == SZGB_VARIANT_EXACT &&
        data_on_device && out_on_device && ((uintptr_t)data % 16) == 0 && ((uintptr_t)out % 4) == 0) {
        const float* d1[1] = {data};
        uint8_t* o1[1] = {out};
        const size_t cap1[1] = {out_cap};
        return compress_batch_impl(c, 1, d1, p, o1, cap1, out_len, stats);
    }
    if (cudaSetDevice(c->device) != cudaSuccess) return SZGB_ECUDA;
    const uint64_t N = cp.d0 * cp.d1 * cp.d2;
    const uint64_t rows = cp.d0 * cp.d1;
    const uint64_t rowlen = cp.d2;
    const uint64_t nch = rows * chunks_per_row(cp.chunk, rowlen);  // Huffman chunks
    const uint64_t cpitch = (rowlen + 7) & ~(uint64_t)7;  // codes row pitch: 16-byte rows
    const int layers = cp.layers;
    WaveGeom g = make_geom(c, cp, layers);
    size_t hrow, hplane;
    halo_sizes(g, layers, &hrow, &hplane);
    if (hyper) hrow = hplane = 0;  // no halo exchange: neighbours come from the recorded values
    const size_t bound = szgb_compress_bound(p);
    const bool direct_out = out_on_device && ((uintptr_t)out % 4 == 0) && out_cap >= bound;
    const bool direct_in = data_on_device && ((uintptr_t)data % 16 == 0);
    const int range_blocks = (int)std::min<uint64_t>(std::max<uint64_t>((N + 8191) / 8192, 1), 4ull * c->sm_count);

    DevState* st;
    float *xs, *partials, *halo_row, *halo_plane;
    uint16_t* codes;
    unsigned int* prog;
    uint32_t *hist, *rowbytes, *nodebuf;
    uint8_t *len, *ostage;
    uint64_t *cw, *sortbuf, *rowoff, *blocksums;
    Arena A;
    A.add(&st, 1);
    A.add(&partials, 2 * (size_t)range_blocks);
    A.add(&codes, rows * cpitch + 8);
    A.add(&halo_row, hrow + hplane);
    A.add(&prog, g.num_ctas);
    A.add(&hist, 65536);
    A.add(&len, 65536);
    A.add(&cw, 65536);
    A.add(&sortbuf, kSortBufU64);
    A.add(&nodebuf, kNodeBufU32);
    A.add(&rowbytes, nch);
    A.add(&rowoff, nch);
    A.add(&blocksums, (nch + 2047) / 2048 + 1);
    char* wargs;
    uint32_t* worder;
    unsigned* wticket;
    A.add(&wargs, wave_args_bytes());
    A.add(&worder, 2 * (size_t)g.num_ctas);
    A.add(&wticket, 1);
    int32_t* latP = nullptr;
    uint8_t* latOK = nullptr;
    if (cp.variant == SZGB_VARIANT_LATTICE) {
        A.add(&latP, N);
        A.add(&latOK, N);
    }
    if (!direct_in) A.add(&xs, N);
    else xs = nullptr;
    if (!direct_out) A.add(&ostage, bound);
    else ostage = nullptr;
    float* hvals = rec_dev;  // the hyperplane path's recorded values
    if (hyper && !rec_dev) A.add(&hvals, N);
    // the wavefront reads x through TMA tiles, which need 16-byte row
    // strides: rows of a length that is not a multiple of 4 are staged at
    // a pitch rounded up to 4
    const bool wave = cp.variant == SZGB_VARIANT_EXACT && !hyper;
    const uint64_t xpitch = (wave && rowlen % 4) ? (rowlen + 3) & ~(uint64_t)3 : rowlen;
    float* xpad = nullptr;
    if (xpitch != rowlen) A.add(&xpad, rows * xpitch);
    rc = ensure_scratch(c, A.total);
    if (rc) return rc;
    A.bind(c->scratch);
    halo_plane = halo_row + hrow;
    const float* x = direct_in ? data : xs;
    uint8_t* dst = direct_out ? out : ostage;
    cudaStream_t s = c->stream;

    DevState init = {};
    init.cap = direct_out ? out_cap : bound;
    if (!direct_in) {
        PhaseTimer t(c, PH_H2D);
        if (cudaMemcpyAsync(xs, data, N * 4, data_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s) != cudaSuccess)
            return SZGB_ECUDA;
    }
    *c->h_init = init;  // pinned: the copy is asynchronous
    if (cudaMemcpyAsync(st, c->h_init, sizeof(DevState), cudaMemcpyHostToDevice, s) != cudaSuccess) return SZGB_ECUDA;
    cudaMemsetAsync(prog, 0, sizeof(unsigned) * g.num_ctas, s);
    cudaMemsetAsync(halo_row, 0, (hrow + hplane) * 4, s);
    cudaMemsetAsync(hist, 0, 65536 * 4, s);
    {
        PhaseTimer t(c, PH_RANGE);
        if ((rc = launch_range(x, N, st, cp, partials, range_blocks, s))) return rc;
    }
    if (cp.variant == SZGB_VARIANT_LATTICE) {
        // the lattice variant: adaptive m, lattice integers and residual codes, all parallel
        PhaseTimer t(c, PH_WAVE_C);
        if ((rc = launch_lattice_compress(x, cp, latP, latOK, codes, cpitch, rec_dev, st, s))) return rc;
    } else if (cp.m_user == 0) {
        PhaseTimer t(c, PH_ADAPT);
        if (D4) {
            if ((rc = launch_adapt4(x, D4, cp.d0 / D4, cp.d1, cp.d2, layers, cp.theta, st, s))) return rc;
        } else if ((rc = launch_adapt(x, cp, st, s))) {
            return rc;
        }
    }
    if (cp.variant == SZGB_VARIANT_EXACT) {
        PhaseTimer t(c, PH_WAVE_C);
        if (D4) {
            if ((rc = launch_hyper4(false, layers, x, hvals, codes, cpitch, D4, cp.d0 / D4, cp.d1, cp.d2, st, s)))
                return rc;
        } else if (hyper) {
            if ((rc = launch_hyper_compress(layers, x, hvals, codes, cpitch, cp.d0, cp.d1, cp.d2, st, s))) return rc;
        } else {
            if (xpad && (rc = launch_pitch_rows(x, rows, rowlen, xpad, xpitch, c->sm_count, s))) return rc;
            const float* xw = xpad ? xpad : x;
            if (!rec_dev) {
                // the persistent kernel, items in ready-time order
                ArgsBuf ha(wave_args_bytes());
                wave_args_compress(ha.p, g, xw, xpitch, codes, cpitch, halo_row, halo_plane, prog, st,
                                   c->timeout_ns);
                if ((rc = ensure_pinned(c, align_up(wave_args_bytes(), 256) + 8 * (size_t)g.num_ctas))) return rc;
                if ((rc = launch_wave_one(c, g, layers, false, ha.p, static_cast<char*>(c->h_batch), wargs, worder,
                                          wticket, s)))
                    return rc;
            } else if ((rc = launch_wave_compress(g, layers, xw, xpitch, codes, cpitch, rec_dev, halo_row, halo_plane,
                                                  prog, st, c->timeout_ns, s))) {
                return rc;
            }
        }
    }
    {
        PhaseTimer t(c, PH_HIST);
        if ((rc = launch_histogram(codes, rows, rowlen, cpitch, hist, st, s))) return rc;
    }
    {
        PhaseTimer t(c, PH_CODEBOOK);
        if ((rc = launch_codebook(hist, st, len, cw, sortbuf, nodebuf, s))) return rc;
    }
    {
        PhaseTimer t(c, PH_ROWBITS);
        if ((rc = launch_rowbits(codes, cpitch, x, rows, rowlen, cp.chunk, len, rowbytes, st, s, latOK))) return rc;
    }
    {
        PhaseTimer t(c, PH_SCAN);
        if ((rc = launch_scan_rows(rowbytes, nch, rowoff, blocksums, st, 1, s))) return rc;
    }
    {
        PhaseTimer t(c, PH_WRITE);
        if ((rc = launch_write_meta(cp, nch, len, nodebuf, rowbytes, rowoff, dst, st, s))) return rc;
        if ((rc = launch_encode(codes, cpitch, x, rows, rowlen, cp.chunk, len, cw, rowoff, dst, st, s, latP, latOK,
                                cp.ndim, layers, cp.d1)))
            return rc;
        if (D4 && (rc = launch_patch_header4(dst, D4, cp.d0 / D4, st, s))) return rc;
    }
    if (codes_dev && cudaMemcpy2DAsync(codes_dev, rowlen * 2, codes, cpitch * 2, rowlen * 2, rows,
                                       cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return SZGB_ECUDA;
    if (cudaMemcpyAsync(c->h_state, st, sizeof(DevState), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return SZGB_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return SZGB_ECUDA;
    const DevState hs = *c->h_state;
    *out_len = (size_t)hs.total;
    rc = dev_errors(hs);
    if (rc == SZGB_OK && hs.total > out_cap) rc = SZGB_ETRUNC;
    if (rc) return rc;
    if (!direct_out) {
        PhaseTimer t(c, PH_D2H);
        if (cudaMemcpyAsync(out, ostage, hs.total, out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s) != cudaSuccess)
            return SZGB_ECUDA;
        if (cudaStreamSynchronize(s) != cudaSuccess) return SZGB_ECUDA;
    }
    if (stats) {
        stats->n_points = N;
        stats->n_unpred = hs.K;
        stats->stream_bytes = hs.total;
        stats->m = hs.m;
        stats->maxlen = (int)hs.maxlen;
        stats->nsym = hs.nsym;
        stats->eb_f = hs.eb_f;
        stats->xmin = hs.xmin;
        stats->xmax = hs.xmax;
        stats->status = SZGB_OK;
    }
    return SZGB_OK;
}

// ---------------------------------------------------------------------------
// stream header (host side)


uint64_t rd_le(const uint8_t* p, int n) {
    uint64_t v = 0;
    for (int i = n - 1; i >= 0; i--) v = (v << 8) | p[i];
    return v;
}

}  // namespace

int szgb::parse_header(const uint8_t* h, size_t in_len, Header* o) {
    if (in_len < (size_t)kHeaderBytes) return SZGB_ECORRUPT;
    if (!(h[0] == 'S' && h[1] == 'Z' && h[2] == 'G' && h[3] == 'B')) return SZGB_ECORRUPT;
    if (rd_le(h + 4, 2) != 1 || rd_le(h + 6, 2) != (uint64_t)kHeaderBytes) return SZGB_ECORRUPT;
    o->ndim = h[8];
    o->layers = h[9];
    o->m = h[10];
    o->mode = h[11];
    o->maxlen = h[12];
    o->tw = h[13];
    o->d0 = rd_le(h + 16, 8);
    o->d1 = rd_le(h + 24, 8);
    o->d2 = rd_le(h + 32, 8);
    uint64_t u;
    u = rd_le(h + 40, 8); memcpy(&o->eb_abs, &u, 8);
    u = rd_le(h + 48, 8); memcpy(&o->eb_rel, &u, 8);
    uint32_t v;
    v = (uint32_t)rd_le(h + 56, 4); memcpy(&o->eb_f, &v, 4);
    v = (uint32_t)rd_le(h + 60, 4); memcpy(&o->xmin, &v, 4);
    v = (uint32_t)rd_le(h + 64, 4); memcpy(&o->xmax, &v, 4);
    o->nsym = (uint32_t)rd_le(h + 68, 4);
    o->nchunks = rd_le(h + 72, 8);
    o->K = rd_le(h + 80, 8);
    o->payload = rd_le(h + 88, 8);
    o->total = rd_le(h + 96, 8);
    u = rd_le(h + 104, 8); memcpy(&o->theta, &u, 8);
    o->adaptive = h[112];
    o->variant = h[113];
    o->chunk = (uint32_t)rd_le(h + 116, 4);
    if (o->variant > 1) return SZGB_ECORRUPT;
    // a 4D field D x P x M x N (the predictor of Sec. III in four dimensions;
    // D at byte 120, P at byte 16) is checked as its (D P) x M x N view
    o->D4 = 0;
    if (o->ndim == 4 && o->variant == 0) {
        const uint64_t D = rd_le(h + 120, 8), P = o->d0;
        if (D == 0 || P == 0 || D > 0xffffffffull || P > 0xffffffffull || D * P > 0xffffffffull)
            return SZGB_ECORRUPT;
        o->ndim = 3;
        o->d0 = D * P;
        o->D4 = D;
    }
    if (o->ndim < 1 || o->ndim > 3 || o->layers < 1 || o->layers > 4 || o->m < 2 || o->m > 16) return SZGB_ECORRUPT;
    if (o->tw != 2 && o->tw != 4 || o->mode > 2) return SZGB_ECORRUPT;
    if (o->d0 == 0 || o->d1 == 0 || o->d2 == 0 || o->d0 > 0xffffffffull || o->d1 > 0xffffffffull ||
        o->d2 > 0xffffffffull)
        return SZGB_ECORRUPT;
    unsigned __int128 n = (unsigned __int128)o->d0 * o->d1 * o->d2;
    if (n >= ((unsigned __int128)1 << 32)) return SZGB_ECORRUPT;
    if (o->ndim < 3 && o->d0 != 1) return SZGB_ECORRUPT;
    if (o->ndim < 2 && o->d1 != 1) return SZGB_ECORRUPT;
    // chunks: whole rows (0), or a power of two >= 32 shorter than a row
    // (the lattice variant codes whole rows)
    if (o->chunk && (o->chunk < 32 || (o->chunk & (o->chunk - 1)) || o->chunk >= o->d2 || o->variant))
        return SZGB_ECORRUPT;
    if (o->nchunks != o->d0 * o->d1 * chunks_per_row(o->chunk, o->d2)) return SZGB_ECORRUPT;
    if (o->nsym < 1 || o->nsym > (1u << o->m) || o->maxlen < 1 || o->maxlen > 64) return SZGB_ECORRUPT;
    uint64_t cb = (3ull * o->nsym + 3) & ~3ull;
    uint64_t tb = ((uint64_t)o->tw * o->nchunks + 3) & ~3ull;
    if (o->total != (uint64_t)kHeaderBytes + cb + tb + o->payload || o->total > in_len) return SZGB_ECORRUPT;
    return SZGB_OK;
}

namespace {

int decompress_impl(szgb_ctx* c, const uint8_t* in, size_t in_len, int in_on_device, float* out,
                    size_t out_cap_elems, int out_on_device) {
    if (!c || !in || !out) return SZGB_EINVAL;
    if (cudaSetDevice(c->device) != cudaSuccess) return SZGB_ECUDA;
    cudaStream_t s = c->stream;
    uint8_t* hbuf = c->h_hdr;  // pinned
    if (in_len < (size_t)kHeaderBytes) return SZGB_ECORRUPT;
    if (in_on_device) {
        if (cudaMemcpyAsync(hbuf, in, kHeaderBytes, cudaMemcpyDeviceToHost, s) != cudaSuccess) return SZGB_ECUDA;
        if (cudaStreamSynchronize(s) != cudaSuccess) return SZGB_ECUDA;
    } else {
        memcpy(hbuf, in, kHeaderBytes);
    }
    // a 4D stream (D x P x M x N) is decoded as its (D P) x M x N view, then
    // reconstructed over the 4D hyperplanes
    Header H;
    int rc = parse_header(hbuf, in_len, &H);
    if (rc) return rc;
    if (H.variant == SZGB_VARIANT_LATTICE && H.layers > 2) return SZGB_EUNSUPPORTED;
    const uint64_t D4 = H.D4;
    // 3D fields with n = 3, 4, and 4D fields: the hyperplane kernels instead of the wavefront
    const bool hyper = H.variant == SZGB_VARIANT_EXACT && !wave_carries(H);
    const uint64_t N = H.d0 * H.d1 * H.d2;
    if (out_cap_elems < N) return SZGB_EINVAL;
    if (one_field_batched(c) && !hyper && H.variant == SZGB_VARIANT_EXACT && in_on_device && out_on_device &&
        ((uintptr_t)in % 4) == 0 && ((uintptr_t)out % 16) == 0)
        return decompress_batch_impl(c, 1, &in, &in_len, &out, &out_cap_elems, nullptr, hbuf);
    const uint64_t rows = H.d0 * H.d1, nch = H.nchunks;
    CallParams cp = {};
    cp.ndim = H.ndim;
    cp.d0 = H.d0;
    cp.d1 = H.d1;
    cp.d2 = H.d2;
    cp.layers = H.layers;
    WaveGeom g = make_geom(c, cp, H.layers);
    size_t hrow, hplane;
    halo_sizes(g, H.layers, &hrow, &hplane);
    if (hyper) hrow = hplane = 0;  // no halo exchange: neighbours come from the output
    const bool direct_in = in_on_device && ((uintptr_t)in % 4 == 0);
    const bool direct_out = out_on_device && ((uintptr_t)out % 16 == 0);
    DevState* st;
    float *halo_row, *halo_plane, *ostage;
    unsigned int* prog;
    uint32_t *rowbytes, *lut, *dectab, *symbuf;
    uint64_t *rowoff, *blocksums;
    uint8_t *lenbuf, *istage;
    uint16_t* codes;
    const uint64_t cpitch = (H.d2 + 7) & ~(uint64_t)7;
    const bool lattice = H.variant == SZGB_VARIANT_LATTICE;
    int32_t* latR = nullptr;
    uint8_t* latEX = nullptr;
    Arena A;
    A.add(&st, 1);
    if (lattice) {
        A.add(&latR, N);
        A.add(&latEX, N);
        codes = nullptr;
    } else {
        A.add(&codes, rows * cpitch + 8);
    }
    A.add(&halo_row, lattice ? 1 : hrow + hplane);
    A.add(&prog, g.num_ctas);
    A.add(&rowbytes, nch);
    A.add(&rowoff, nch);
    A.add(&blocksums, (nch + 2047) / 2048 + 1);
    A.add(&lut, (size_t)1 << kLutBits);
    A.add(&dectab, kDecTabU32);
    A.add(&lenbuf, 65536);
    A.add(&symbuf, 65536);
    char* wargs;
    uint32_t* worder;
    unsigned* wticket;
    A.add(&wargs, wave_args_bytes());
    A.add(&worder, 2 * (size_t)g.num_ctas);
    A.add(&wticket, 1);
    if (!direct_in) A.add(&istage, H.total + 16);
    else istage = nullptr;
    if (!direct_out) A.add(&ostage, N);
    else ostage = nullptr;
    rc = ensure_scratch(c, A.total);
    if (rc) return rc;
    A.bind(c->scratch);
    halo_plane = halo_row + hrow;
    const uint8_t* sb = direct_in ? in : istage;
    float* dst = direct_out ? out : ostage;
    if (!direct_in) {
        PhaseTimer t(c, PH_H2D);
        if (cudaMemcpyAsync(istage, in, H.total, in_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s) != cudaSuccess)
            return SZGB_ECUDA;
    }
    DevState init = {};
    init.eb_f = H.eb_f;
    init.twoeb = 2.0f * H.eb_f;
    init.m = H.m;
    init.center = 1 << (H.m - 1);
    init.radius = (float)((1 << (H.m - 1)) - 1);
    uint32_t ub;
    memcpy(&ub, &H.eb_f, 4);
    init.e_eb = (int)((ub >> 23) & 0xffu);
    *c->h_init = init;  // pinned: the copy is asynchronous
    if (cudaMemcpyAsync(st, c->h_init, sizeof(DevState), cudaMemcpyHostToDevice, s) != cudaSuccess) return SZGB_ECUDA;
    cudaMemsetAsync(prog, 0, sizeof(unsigned) * g.num_ctas, s);
    if (!lattice) cudaMemsetAsync(halo_row, 0, (hrow + hplane) * 4, s);
    const uint64_t cb = (3ull * H.nsym + 3) & ~3ull;
    const uint64_t tb = ((uint64_t)H.tw * nch + 3) & ~3ull;
    const uint8_t* codebook = sb + kHeaderBytes;
    const uint8_t* table = codebook + cb;
    const uint8_t* payload = table + tb;
    {
        PhaseTimer t(c, PH_DEC_TABLES);
        if ((rc = launch_decode_tables(codebook, H.nsym, H.m, lut, dectab, lenbuf, symbuf, st, s))) return rc;
    }
    {
        PhaseTimer t(c, PH_DEC_SCAN);
        if ((rc = launch_scan_rows(rowbytes, nch, rowoff, blocksums, st, 0, s, table, H.tw))) return rc;
    }
    if (lattice) {
        PhaseTimer t(c, PH_WAVE_D);
        if ((rc = launch_lattice_decompress(payload, rowoff, rowbytes, payload + H.payload, lut, dectab, H.ndim,
                                            H.layers, H.d0, H.d1, H.d2, latR, latEX, dst, st, s)))
            return rc;
    } else {
        {
            PhaseTimer t(c, PH_DEC_ROWS);
            if ((rc = launch_decode_rows(payload, rowoff, rowbytes, payload + H.payload, lut, dectab, codes, cpitch,
                                         dst, rows, H.d2, H.chunk, st, s)))
                return rc;
        }
        PhaseTimer t(c, PH_WAVE_D);
        if (D4) {
            if ((rc = launch_hyper4(true, H.layers, nullptr, dst, codes, cpitch, D4, H.d0 / D4, H.d1, H.d2, st, s)))
                return rc;
        } else if (hyper) {
            if ((rc = launch_hyper_decompress(H.layers, codes, cpitch, dst, H.d0, H.d1, H.d2, st, s))) return rc;
        } else {
            ArgsBuf ha(wave_args_bytes());
            if ((rc = wave_args_decompress(ha.p, g, codes, cpitch, dst, halo_row, halo_plane, prog, st,
                                           c->timeout_ns)))
                return rc;
            if ((rc = ensure_pinned(c, align_up(wave_args_bytes(), 256) + 8 * (size_t)g.num_ctas))) return rc;
            if ((rc = launch_wave_one(c, g, H.layers, true, ha.p, static_cast<char*>(c->h_batch), wargs, worder,
                                      wticket, s)))
                return rc;
        }
    }
    if (cudaMemcpyAsync(c->h_state, st, sizeof(DevState), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return SZGB_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return SZGB_ECUDA;
    const DevState hs = *c->h_state;
    rc = dev_errors(hs);
    if (rc == SZGB_OK && hs.payload != H.payload) rc = SZGB_ECORRUPT;
    if (rc) return rc;
    if (!direct_out) {
        PhaseTimer t(c, PH_D2H);
        if (cudaMemcpyAsync(out, ostage, N * 4, out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s) != cudaSuccess)
            return SZGB_ECUDA;
        if (cudaStreamSynchronize(s) != cudaSuccess) return SZGB_ECUDA;
    }
    return SZGB_OK;
}


uint64_t header_hash(const Header& h) {
    uint64_t v = 1469598103934665603ull;
    auto mix = [&](uint64_t x) { v = (v ^ x) * 1099511628211ull; };
    mix(h.ndim); mix(h.layers); mix(h.m); mix(h.tw); mix(h.d0); mix(h.d1); mix(h.d2); mix(h.nsym);
    mix(h.payload); mix(h.total); mix(h.chunk); mix(h.D4);
    uint32_t e;
    memcpy(&e, &h.eb_f, 4);
    mix(e);
    return v;
}

// ---------------------------------------------------------------------------
// batches of independent fields (device buffers): every field's wavefront in
// one persistent launch, the per-field kernels spread over auxiliary streams,
// the whole sequence captured once in a CUDA graph and replayed while the
// arguments repeat

int ensure_aux(szgb_ctx* c) {
    if (c->ev_fork) return SZGB_OK;
    for (int k = 0; k < kAux; k++) {
        if (cudaStreamCreateWithFlags(&c->aux[k], cudaStreamNonBlocking) != cudaSuccess) return SZGB_ECUDA;
        if (cudaEventCreateWithFlags(&c->ev_join[k], cudaEventDisableTiming) != cudaSuccess) return SZGB_ECUDA;
    }
    if (cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess) return SZGB_ECUDA;
    return SZGB_OK;
}

int ensure_pinned(szgb_ctx* c, size_t need) {
    if (need <= c->h_batch_cap) return SZGB_OK;
    const size_t old_cap = c->h_batch_cap;
    if (c->h_batch) {
        cudaStreamSynchronize(c->stream);
        cudaFreeHost(c->h_batch);
        c->h_batch = nullptr;
        c->h_batch_cap = 0;
    }
    // grow at least twofold from 1 MiB: cudaFreeHost waits for the device
    size_t cap = align_up(std::max(std::max(need + need / 4, (size_t)1 << 20), 2 * old_cap), 1 << 16);
    if (cudaMallocHost(&c->h_batch, cap) != cudaSuccess) {
        cudaGetLastError();
        return SZGB_ENOMEM;
    }
    c->h_batch_cap = cap;
    return SZGB_OK;
}

// fork: every auxiliary stream waits for the main stream; join: the reverse
void fork_aux(szgb_ctx* c) {
    cudaEventRecord(c->ev_fork, c->stream);
    for (int k = 0; k < kAux; k++) cudaStreamWaitEvent(c->aux[k], c->ev_fork, 0);
}
void join_aux(szgb_ctx* c) {
    for (int k = 0; k < kAux; k++) {
        cudaEventRecord(c->ev_join[k], c->aux[k]);
        cudaStreamWaitEvent(c->stream, c->ev_join[k], 0);
    }
}

void drop_graph(BatchGraph& G) {
    if (G.exec) cudaGraphExecDestroy(G.exec);
    G.exec = nullptr;
    G.key.clear();
}

// Runs `enqueue` on the main stream: directly, or from the cached graph when
// `key` matches, else captured into a new graph first.
template <typename F>
int run_batch(szgb_ctx* c, BatchGraph& G, const std::vector<uint64_t>& key, F enqueue) {
    cudaStream_t s = c->stream;
    if (!c->use_graphs || c->debug_skip) return enqueue();
    if (!(G.exec && G.key == key)) {
        drop_graph(G);
        if (cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed) != cudaSuccess) return SZGB_ECUDA;
        int rc = enqueue();
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamEndCapture(s, &graph);
        if (rc || e != cudaSuccess || !graph) {
            if (graph) cudaGraphDestroy(graph);
            cudaGetLastError();
            return rc ? rc : SZGB_ECUDA;
        }
        e = cudaGraphInstantiate(&G.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            G.exec = nullptr;
            cudaGetLastError();
            return SZGB_ECUDA;
        }
        G.key = key;
    }
    return cudaGraphLaunch(G.exec, s) == cudaSuccess ? SZGB_OK : SZGB_ECUDA;
}

struct CompPlan {
    CallParams cp;
    WaveGeom g;
    uint64_t n, rows, rowlen, cpitch, nch;
    size_t hrow, hplane;
    int range_blocks;
    // device scratch
    float *partials, *halo_row, *halo_plane;
    uint16_t* codes;
    uint32_t *rowbytes, *nodebuf;
    uint8_t* len;
    uint64_t *cw, *sortbuf, *rowoff, *blocksums;
    unsigned* prog;
    uint32_t* hist;
    float* xpad;      // rows staged at a 16-byte pitch for the wavefront (or null)
    uint64_t xpitch;  // row pitch of the wavefront's input
};

// The (field, item) order of a wavefront launch.  Items are taken in the
// order of the sweep at which their producers let them start: about W + 5
// sweeps per plane block and 14 per row block in 3D (the skew of the block
// plus prefetch and publication lag), 9W + 5 per row block in 1D/2D.  Every
// producer has a smaller key than its consumers, so the order respects the
// dependencies, and SMs go first to the items that can run first.
size_t build_order(const std::vector<int>& fields, const std::vector<WaveGeom>& geo, uint32_t* dst) {
    struct K {
        uint64_t key;
        uint32_t f, i;
    };
    std::vector<K> v;
    for (int f : fields) {
        const WaveGeom& g = geo[f];
        for (int i = 0; i < g.num_ctas; i++) {
            uint64_t key;
            if (g.ndim == 3) key = (uint64_t)(i / g.nb1) * (uint64_t)(g.W + 5) + (uint64_t)(i % g.nb1) * 14u;
            else key = (uint64_t)i * (uint64_t)(9 * g.W + 5);
            v.push_back({key, (uint32_t)f, (uint32_t)i});
        }
    }
    std::stable_sort(v.begin(), v.end(), [](const K& a, const K& b) {
        return a.key != b.key ? a.key < b.key : (a.f != b.f ? a.f < b.f : a.i < b.i);
    });
    for (size_t t = 0; t < v.size(); t++) {
        dst[2 * t] = v[t].f;
        dst[2 * t + 1] = v[t].i;
    }
    return v.size();
}

// One field's wavefront on the persistent (batch) kernel: its arguments and
// item order go to the device through the pinned staging area at `stage`.
int launch_wave_one(szgb_ctx* c, const WaveGeom& g, int layers, bool dec, const void* host_args, char* stage,
                    char* dev_args, uint32_t* dev_order, unsigned* dev_ticket, cudaStream_t s) {
    const size_t wsz = wave_args_bytes();
    memcpy(stage, host_args, wsz);
    uint32_t* ho = reinterpret_cast<uint32_t*>(stage + align_up(wsz, 256));
    std::vector<int> one{0};
    std::vector<WaveGeom> geo{g};
    const size_t n = build_order(one, geo, ho);
    if (cudaMemcpyAsync(dev_args, stage, wsz, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(dev_order, ho, 8 * n, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemsetAsync(dev_ticket, 0, sizeof(unsigned), s) != cudaSuccess)
        return SZGB_ECUDA;
    const int grid = wave_grid(c, n);
    return launch_wave_batch(dev_args, dev_order, (unsigned)n, dev_ticket, layers, dec,
                             wave_smem_bytes(g, layers, dec), grid, s);
}

int compress_batch_impl(szgb_ctx* c, int count, const float* const* data, const szgb_params* params,
                        uint8_t* const* out, const size_t* out_cap, size_t* out_len, szgb_stats* stats) {
    if (!c || count < 1 || !data || !params || !out || !out_cap || !out_len) return SZGB_EINVAL;
    if (cudaSetDevice(c->device) != cudaSuccess) return SZGB_ECUDA;
    int rc = ensure_aux(c);
    if (rc) return rc;
    std::vector<CompPlan> P(count);
    std::vector<int> nitems(count), by_layers[kMaxLayers];
    size_t smem[kMaxLayers] = {};
    for (int f = 0; f < count; f++) {
        CompPlan& q = P[f];
        if (!data[f] || !out[f] || ((uintptr_t)data[f] % 16) || ((uintptr_t)out[f] % 4)) return SZGB_EINVAL;
        if ((rc = check_params(&params[f], &q.cp))) return rc;
        resolve_chunk(c, &params[f], &q.cp);
        if (!wave_carries(q.cp)) return SZGB_EUNSUPPORTED;  // the public call routes these to compress_impl
        q.n = q.cp.d0 * q.cp.d1 * q.cp.d2;
        q.rows = q.cp.d0 * q.cp.d1;
        q.rowlen = q.cp.d2;
        q.nch = q.rows * chunks_per_row(q.cp.chunk, q.rowlen);
        q.cpitch = (q.rowlen + 7) & ~(uint64_t)7;
        q.g = make_geom(c, q.cp, q.cp.layers);
        halo_sizes(q.g, q.cp.layers, &q.hrow, &q.hplane);
        q.range_blocks = (int)std::min<uint64_t>(std::max<uint64_t>((q.n + 8191) / 8192, 1), 4ull * c->sm_count);
        nitems[f] = q.g.num_ctas;
        const int li = q.cp.layers - 1;
        by_layers[li].push_back(f);
        smem[li] = std::max(smem[li], wave_smem_bytes(q.g, q.cp.layers, false));
    }
    const size_t wsz = wave_args_bytes();
    size_t nprog = 0, total_items = 0;
    for (int f = 0; f < count; f++) nprog += (size_t)nitems[f], total_items += (size_t)nitems[f];

    // pinned host tables: initial states, wavefront arguments, order,
    // codebook arguments; the final states come back after them.  The device
    // copy of the tables has the same layout, so that one copy moves them.
    const size_t cbsz = codebook_args_bytes();
    const size_t o_st = 0, o_w = align_up((size_t)count * sizeof(DevState), 256);
    const size_t o_ord = align_up(o_w + (size_t)count * wsz, 256);
    const size_t o_cb = align_up(o_ord + 8 * total_items, 256);
    const size_t o_out = align_up(o_cb + (size_t)count * cbsz, 256);
    // what every pass starts from zero, in one region cleared by one memset:
    // tickets, item progress words, histograms, halo buffers
    size_t nhalo = 0;
    for (int f = 0; f < count; f++) nhalo += P[f].hrow + P[f].hplane;
    const size_t z_pr = align_up(4 * (size_t)kMaxLayers, 256);
    const size_t z_hi = align_up(z_pr + 4 * nprog, 256);
    const size_t z_ha = align_up(z_hi + 4 * (size_t)count * 65536, 256);
    const size_t z_end = align_up(z_ha + 4 * nhalo, 256);
    // device scratch
    char *dtab, *zero;
    Arena A;
    A.add(&dtab, o_out);
    A.add(&zero, z_end);
    for (int f = 0; f < count; f++) {
        CompPlan& q = P[f];
        A.add(&q.partials, 2 * (size_t)q.range_blocks);
        A.add(&q.codes, q.rows * q.cpitch + 8);
        A.add(&q.len, 65536);
        A.add(&q.cw, 65536);
        A.add(&q.sortbuf, kSortBufU64);
        A.add(&q.nodebuf, kNodeBufU32);
        A.add(&q.rowbytes, q.nch);
        A.add(&q.rowoff, q.nch);
        A.add(&q.blocksums, (q.nch + 2047) / 2048 + 1);
        q.xpitch = (q.rowlen + 3) & ~(uint64_t)3;  // TMA tiles need 16-byte row strides
        q.xpad = nullptr;
        if (q.xpitch != q.rowlen) A.add(&q.xpad, q.rows * q.xpitch);
        else q.xpitch = q.rowlen;
    }
    if ((rc = ensure_scratch(c, A.total))) return rc;
    A.bind(c->scratch);
    DevState* const st = reinterpret_cast<DevState*>(dtab + o_st);
    char* const wargs = dtab + o_w;
    uint32_t* const order = reinterpret_cast<uint32_t*>(dtab + o_ord);
    char* const cbargs = dtab + o_cb;
    unsigned* const tickets = reinterpret_cast<unsigned*>(zero);
    unsigned* const prog_all = reinterpret_cast<unsigned*>(zero + z_pr);
    uint32_t* const hist_all = reinterpret_cast<uint32_t*>(zero + z_hi);
    float* const halo_all = reinterpret_cast<float*>(zero + z_ha);
    {
        size_t po = 0, ho = 0;
        for (int f = 0; f < count; f++) {
            P[f].prog = prog_all + po;
            P[f].hist = hist_all + (size_t)f * 65536;
            P[f].halo_row = halo_all + ho;
            P[f].halo_plane = halo_all + ho + P[f].hrow;
            po += (size_t)nitems[f];
            ho += P[f].hrow + P[f].hplane;
        }
    }
    if ((rc = ensure_pinned(c, o_out + (size_t)count * sizeof(DevState)))) return rc;
    char* H = static_cast<char*>(c->h_batch);
    DevState* h_init = reinterpret_cast<DevState*>(H + o_st);
    DevState* h_fin = reinterpret_cast<DevState*>(H + o_out);
    for (int f = 0; f < count; f++) {
        h_init[f] = DevState{};
        h_init[f].cap = out_cap[f];
        wave_args_compress(H + o_w + (size_t)f * wsz, P[f].g, P[f].xpad ? P[f].xpad : data[f], P[f].xpitch,
                           P[f].codes, P[f].cpitch, P[f].halo_row, P[f].halo_plane, P[f].prog, st + f,
                           c->timeout_ns);
        codebook_args_fill(H + o_cb + (size_t)f * cbsz, P[f].hist, st + f, P[f].len, P[f].cw, P[f].sortbuf,
                           P[f].nodebuf);
    }
    uint32_t* h_order = reinterpret_cast<uint32_t*>(H + o_ord);
    size_t ord_at[kMaxLayers], ord_n[kMaxLayers];
    std::vector<WaveGeom> geo(count);
    for (int f = 0; f < count; f++) geo[f] = P[f].g;
    for (int li = 0, at = 0; li < kMaxLayers; li++) {  // one launch per layer count present
        ord_at[li] = at;
        ord_n[li] = build_order(by_layers[li], geo, h_order + 2 * at);
        at += (int)ord_n[li];
    }

    std::vector<uint64_t> key;
    key.push_back((uint64_t)count);
    key.push_back((uint64_t)(uintptr_t)c->scratch);
    key.push_back((uint64_t)(uintptr_t)c->h_batch);
    key.push_back((uint64_t)c->W2 | ((uint64_t)c->W3 << 16) | ((uint64_t)(uint32_t)c->wave_ctas << 32));
    for (int f = 0; f < count; f++) {
        key.push_back((uint64_t)(uintptr_t)data[f]);
        key.push_back((uint64_t)(uintptr_t)out[f]);
        key.push_back((uint64_t)out_cap[f]);
        const uint64_t* pw = reinterpret_cast<const uint64_t*>(&params[f]);
        for (size_t i = 0; i < sizeof(szgb_params) / 8; i++) key.push_back(pw[i]);
        key.push_back((uint64_t)P[f].g.W | ((uint64_t)P[f].cp.chunk << 8));  // the resolved shape and chunking
    }
    cudaStream_t s = c->stream;
    auto enqueue = [&]() -> int {
        int r;
        if (cudaMemcpyAsync(dtab, H, o_out, cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaMemsetAsync(zero, 0, z_end, s) != cudaSuccess)
            return SZGB_ECUDA;
        fork_aux(c);
        for (int f = 0; f < count; f++) {
            CompPlan& q = P[f];
            cudaStream_t a = c->aux[f % kAux];
            if ((r = launch_range(data[f], q.n, st + f, q.cp, q.partials, q.range_blocks, a))) return r;
            if (q.cp.m_user == 0 && (r = launch_adapt(data[f], q.cp, st + f, a))) return r;
            if (q.xpad && (r = launch_pitch_rows(data[f], q.rows, q.rowlen, q.xpad, q.xpitch, c->sm_count, a)))
                return r;
        }
        join_aux(c);
        for (int li = 0; li < kMaxLayers; li++) {
            if (!ord_n[li]) continue;
            const int grid = wave_grid(c, ord_n[li]);
            if ((r = launch_wave_batch(wargs, order + 2 * ord_at[li], (unsigned)ord_n[li], tickets + li, li + 1, false,
                                       smem[li], grid, s)))
                return r;
        }
        fork_aux(c);
        for (int f = 0; f < count; f++) {
            CompPlan& q = P[f];
            if ((r = launch_histogram(q.codes, q.rows, q.rowlen, q.cpitch, q.hist, st + f, c->aux[f % kAux]))) return r;
        }
        join_aux(c);
        // every field's codebook in one launch (one CTA each)
        if ((r = launch_codebook_batch(cbargs, count, s))) return r;
        fork_aux(c);
        for (int f = 0; f < count; f++) {
            CompPlan& q = P[f];
            cudaStream_t a = c->aux[f % kAux];
            if ((r = launch_rowbits(q.codes, q.cpitch, data[f], q.rows, q.rowlen, q.cp.chunk, q.len, q.rowbytes, st + f,
                                    a)))
                return r;
            if ((r = launch_scan_rows(q.rowbytes, q.nch, q.rowoff, q.blocksums, st + f, 1, a))) return r;
            if ((r = launch_write_meta(q.cp, q.nch, q.len, q.nodebuf, q.rowbytes, q.rowoff, out[f], st + f, a))) return r;
            if ((r = launch_encode(q.codes, q.cpitch, data[f], q.rows, q.rowlen, q.cp.chunk, q.len, q.cw, q.rowoff, out[f],
                                   st + f, a)))
                return r;
        }
        join_aux(c);
        if (cudaMemcpyAsync(h_fin, st, (size_t)count * sizeof(DevState), cudaMemcpyDeviceToHost, s) != cudaSuccess)
            return SZGB_ECUDA;
        return SZGB_OK;
    };
    if ((rc = run_batch(c, c->g_comp, key, enqueue))) return rc;
    if (cudaStreamSynchronize(s) != cudaSuccess) return SZGB_ECUDA;
    int first = SZGB_OK;
    for (int f = 0; f < count; f++) {
        const DevState& hs = h_fin[f];
        out_len[f] = (size_t)hs.total;
        int r = dev_errors(hs);
        if (r == SZGB_OK && hs.total > out_cap[f]) r = SZGB_ETRUNC;
        if (r && !first) first = r;
        if (stats) {
            stats[f].n_points = P[f].n;
            stats[f].n_unpred = hs.K;
            stats[f].stream_bytes = hs.total;
            stats[f].m = hs.m;
            stats[f].maxlen = (int)hs.maxlen;
            stats[f].nsym = hs.nsym;
            stats[f].eb_f = hs.eb_f;
            stats[f].xmin = hs.xmin;
            stats[f].xmax = hs.xmax;
            stats[f].status = r;
        }
    }
    return first;
}

struct DecPlan {
    Header H;
    CallParams cp;
    WaveGeom g;
    uint64_t n, rows, cpitch, nch;
    uint16_t* codes;
    size_t hrow, hplane;
    const uint8_t *codebook, *table, *payload;
    float *halo_row, *halo_plane;
    unsigned* prog;
    uint32_t *rowbytes, *lut, *dectab, *symbuf;
    uint64_t *rowoff, *blocksums;
    uint8_t* lenbuf;
};

// host_hdr: NULL, or the count headers (kHeaderBytes each) already on the host
int decompress_batch_impl(szgb_ctx* c, int count, const uint8_t* const* in, const size_t* in_len,
                          float* const* out, const size_t* out_cap, int* status, const uint8_t* host_hdr) {
    if (!c || count < 1 || !in || !in_len || !out || !out_cap) return SZGB_EINVAL;
    if (cudaSetDevice(c->device) != cudaSuccess) return SZGB_ECUDA;
    int rc = ensure_aux(c);
    if (rc) return rc;
    cudaStream_t s = c->stream;
    // headers to the host (one small copy per field, one synchronisation),
    // unless the caller read the header of its one field already
    const size_t hdr_bytes = (size_t)count * kHeaderBytes;
    if ((rc = ensure_pinned(c, hdr_bytes))) return rc;
    for (int f = 0; f < count; f++) {
        if (!in[f] || !out[f] || ((uintptr_t)in[f] % 4) || ((uintptr_t)out[f] % 16) || in_len[f] < (size_t)kHeaderBytes)
            return SZGB_EINVAL;
        if (host_hdr) {
            memcpy(static_cast<char*>(c->h_batch) + (size_t)f * kHeaderBytes, host_hdr + (size_t)f * kHeaderBytes,
                   kHeaderBytes);
        } else if (cudaMemcpyAsync(static_cast<char*>(c->h_batch) + (size_t)f * kHeaderBytes, in[f], kHeaderBytes,
                                   cudaMemcpyDeviceToHost, s) != cudaSuccess) {
            return SZGB_ECUDA;
        }
    }
    if (!host_hdr && cudaStreamSynchronize(s) != cudaSuccess) return SZGB_ECUDA;
    std::vector<DecPlan> P(count);
    std::vector<int> nitems(count), by_layers[kMaxLayers];
    size_t smem[kMaxLayers] = {};
    for (int f = 0; f < count; f++) {
        DecPlan& q = P[f];
        if ((rc = parse_header(static_cast<uint8_t*>(c->h_batch) + (size_t)f * kHeaderBytes, in_len[f], &q.H))) return rc;
        if (!wave_carries(q.H)) return SZGB_EUNSUPPORTED;  // the public call routes these to decompress_impl
        q.n = q.H.d0 * q.H.d1 * q.H.d2;
        if (out_cap[f] < q.n) return SZGB_EINVAL;
        q.rows = q.H.d0 * q.H.d1;
        q.nch = q.H.nchunks;
        q.cpitch = (q.H.d2 + 7) & ~(uint64_t)7;
        q.cp = CallParams{};
        q.cp.ndim = q.H.ndim;
        q.cp.d0 = q.H.d0;
        q.cp.d1 = q.H.d1;
        q.cp.d2 = q.H.d2;
        q.cp.layers = q.H.layers;
        q.g = make_geom(c, q.cp, q.H.layers);
        halo_sizes(q.g, q.H.layers, &q.hrow, &q.hplane);
        const uint64_t cb = (3ull * q.H.nsym + 3) & ~3ull, tb = ((uint64_t)q.H.tw * q.nch + 3) & ~3ull;
        q.codebook = in[f] + kHeaderBytes;
        q.table = q.codebook + cb;
        q.payload = q.table + tb;
        nitems[f] = q.g.num_ctas;
        const int li = q.H.layers - 1;
        by_layers[li].push_back(f);
        smem[li] = std::max(smem[li], wave_smem_bytes(q.g, q.H.layers, true));
    }
    const size_t wsz = wave_args_bytes();
    size_t nprog = 0, total_items = 0;
    for (int f = 0; f < count; f++) nprog += (size_t)nitems[f], total_items += (size_t)nitems[f];
    // pinned host tables: initial states, wavefront arguments, order, decode
    // and table arguments, decode block offsets; the final states come back
    // after them.  The device copy has the same layout (one copy).
    const size_t dsz = decode_args_bytes(), tsz = tables_args_bytes();
    const size_t o_st = 0, o_w = align_up((size_t)count * sizeof(DevState), 256);
    const size_t o_ord = align_up(o_w + (size_t)count * wsz, 256);
    const size_t o_dec = align_up(o_ord + 8 * total_items, 256);
    const size_t o_tab = align_up(o_dec + (size_t)count * dsz, 256);
    const size_t o_blk = align_up(o_tab + (size_t)count * tsz, 256);
    const size_t o_out = align_up(o_blk + 4 * ((size_t)count + 1), 256);
    // tickets, item progress words and halo buffers: one region, one memset
    size_t nhalo = 0;
    for (int f = 0; f < count; f++) nhalo += P[f].hrow + P[f].hplane;
    const size_t z_pr = align_up(4 * (size_t)kMaxLayers, 256);
    const size_t z_ha = align_up(z_pr + 4 * nprog, 256);
    const size_t z_end = align_up(z_ha + 4 * nhalo, 256);
    char *dtab, *zero;
    Arena A;
    A.add(&dtab, o_out);
    A.add(&zero, z_end);
    for (int f = 0; f < count; f++) {
        DecPlan& q = P[f];
        A.add(&q.codes, q.rows * q.cpitch + 8);
        A.add(&q.rowbytes, q.nch);
        A.add(&q.rowoff, q.nch);
        A.add(&q.blocksums, (q.nch + 2047) / 2048 + 1);
        A.add(&q.lut, (size_t)1 << kLutBits);
        A.add(&q.dectab, kDecTabU32);
        A.add(&q.lenbuf, 65536);
        A.add(&q.symbuf, 65536);
    }
    if ((rc = ensure_scratch(c, A.total))) return rc;
    A.bind(c->scratch);
    DevState* const st = reinterpret_cast<DevState*>(dtab + o_st);
    char* const wargs = dtab + o_w;
    uint32_t* const order = reinterpret_cast<uint32_t*>(dtab + o_ord);
    char* const dargs = dtab + o_dec;
    char* const targs = dtab + o_tab;
    uint32_t* const dblk = reinterpret_cast<uint32_t*>(dtab + o_blk);
    unsigned* const tickets = reinterpret_cast<unsigned*>(zero);
    unsigned* const prog_all = reinterpret_cast<unsigned*>(zero + z_pr);
    float* const halo_all = reinterpret_cast<float*>(zero + z_ha);
    {
        size_t po = 0, ho = 0;
        for (int f = 0; f < count; f++) {
            P[f].prog = prog_all + po;
            P[f].halo_row = halo_all + ho;
            P[f].halo_plane = halo_all + ho + P[f].hrow;
            ho += P[f].hrow + P[f].hplane;
            po += (size_t)nitems[f];
        }
    }
    if ((rc = ensure_pinned(c, o_out + (size_t)count * sizeof(DevState)))) return rc;
    char* Hb = static_cast<char*>(c->h_batch);
    DevState* h_init = reinterpret_cast<DevState*>(Hb + o_st);
    DevState* h_fin = reinterpret_cast<DevState*>(Hb + o_out);
    for (int f = 0; f < count; f++) {
        DecPlan& q = P[f];
        DevState& d = h_init[f];
        d = DevState{};
        d.eb_f = q.H.eb_f;
        d.twoeb = 2.0f * q.H.eb_f;
        d.m = q.H.m;
        d.center = 1 << (q.H.m - 1);
        d.radius = (float)((1 << (q.H.m - 1)) - 1);
        uint32_t ub;
        memcpy(&ub, &q.H.eb_f, 4);
        d.e_eb = (int)((ub >> 23) & 0xffu);
        if ((rc = wave_args_decompress(Hb + o_w + (size_t)f * wsz, q.g, q.codes, q.cpitch, out[f], q.halo_row,
                                       q.halo_plane, q.prog, st + f, c->timeout_ns)))
            return rc;
        decode_args_fill(Hb + o_dec + (size_t)f * dsz, q.payload, q.rowoff, q.rowbytes, q.payload + q.H.payload, q.lut,
                         q.dectab, q.codes, q.cpitch, out[f], q.rows, q.H.d2, q.H.chunk, st + f);
        tables_args_fill(Hb + o_tab + (size_t)f * tsz, q.codebook, q.H.nsym, q.H.m, q.lut, q.dectab, q.lenbuf, q.symbuf,
                         st + f);
    }
    // the row decode of every field in one launch
    uint32_t* h_blk = reinterpret_cast<uint32_t*>(Hb + o_blk);
    h_blk[0] = 0;
    for (int f = 0; f < count; f++) h_blk[f + 1] = h_blk[f] + decode_rows_blocks(P[f].rows, P[f].H.chunk, P[f].H.d2);
    const uint32_t dec_blocks = h_blk[count];
    uint32_t* h_order = reinterpret_cast<uint32_t*>(Hb + o_ord);
    size_t ord_at[kMaxLayers], ord_n[kMaxLayers];
    std::vector<WaveGeom> geo(count);
    for (int f = 0; f < count; f++) geo[f] = P[f].g;
    for (int li = 0, at = 0; li < kMaxLayers; li++) {  // one launch per layer count present
        ord_at[li] = at;
        ord_n[li] = build_order(by_layers[li], geo, h_order + 2 * at);
        at += (int)ord_n[li];
    }
    std::vector<uint64_t> key;
    key.push_back((uint64_t)count);
    key.push_back((uint64_t)(uintptr_t)c->scratch);
    key.push_back((uint64_t)(uintptr_t)c->h_batch);
    key.push_back((uint64_t)c->W2 | ((uint64_t)c->W3 << 16) | ((uint64_t)(uint32_t)c->wave_ctas << 32));
    for (int f = 0; f < count; f++) {
        key.push_back((uint64_t)(uintptr_t)in[f]);
        key.push_back((uint64_t)in_len[f]);
        key.push_back((uint64_t)(uintptr_t)out[f]);
        // the header fixes everything else the plan depends on
        key.push_back(header_hash(P[f].H));
    }
    auto enqueue = [&]() -> int {
        int r;
        if (cudaMemcpyAsync(dtab, Hb, o_out, cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaMemsetAsync(zero, 0, z_end, s) != cudaSuccess)
            return SZGB_ECUDA;
        // every field's chunk offsets (auxiliary streams) while the decoder
        // tables of every field are built in one launch (one CTA each)
        fork_aux(c);
        for (int f = 0; f < count; f++) {
            DecPlan& q = P[f];
            cudaStream_t a = c->aux[f % kAux];
            if ((r = launch_scan_rows(q.rowbytes, q.nch, q.rowoff, q.blocksums, st + f, 0, a, q.table, q.H.tw)))
                return r;
        }
        if ((r = launch_decode_tables_batch(targs, count, s))) return r;
        join_aux(c);
        if ((r = launch_decode_rows_batch(dargs, dblk, count, dec_blocks, s))) return r;
        for (int li = 0; li < kMaxLayers; li++) {
            if (!ord_n[li]) continue;
            const int grid = wave_grid(c, ord_n[li]);
            if ((r = launch_wave_batch(wargs, order + 2 * ord_at[li], (unsigned)ord_n[li], tickets + li, li + 1, true,
                                       smem[li], grid, s)))
                return r;
        }
        if (cudaMemcpyAsync(h_fin, st, (size_t)count * sizeof(DevState), cudaMemcpyDeviceToHost, s) != cudaSuccess)
            return SZGB_ECUDA;
        return SZGB_OK;
    };
    if ((rc = run_batch(c, c->g_dec, key, enqueue))) return rc;
    if (cudaStreamSynchronize(s) != cudaSuccess) return SZGB_ECUDA;
    int first = SZGB_OK;
    for (int f = 0; f < count; f++) {
        const DevState& hs = h_fin[f];
        int r = dev_errors(hs);
        if (r == SZGB_OK && hs.payload != P[f].H.payload) r = SZGB_ECORRUPT;
        if (r && !first) first = r;
        if (status) status[f] = r;
    }
    return first;
}
}  // namespace

// ---------------------------------------------------------------------------
// C ABI

extern "C" {

int szgb_create(szgb_ctx** out, int device, size_t device_mem_budget) {
    if (!out) return SZGB_EINVAL;
    *out = nullptr;
    if (cudaSetDevice(device) != cudaSuccess) return SZGB_ECUDA;
    szgb_ctx* c = new (std::nothrow) szgb_ctx();
    if (!c) return SZGB_ENOMEM;
    c->device = device;
    c->budget = device_mem_budget;
    if (cudaStreamCreateWithFlags(&c->own_stream, cudaStreamNonBlocking) != cudaSuccess) {
        delete c;
        return SZGB_ECUDA;
    }
    c->stream = c->own_stream;
    if (cudaMallocHost(&c->h_state, 2 * sizeof(DevState) + kHeaderBytes) != cudaSuccess) {
        cudaStreamDestroy(c->own_stream);
        delete c;
        return SZGB_ENOMEM;
    }
    for (int i = 0; i < PH_N; i++) {
        cudaEventCreate(&c->ev0[i]);
        cudaEventCreate(&c->ev1[i]);
    }
    c->h_init = c->h_state + 1;
    c->h_hdr = reinterpret_cast<uint8_t*>(c->h_state + 2);
    cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device);
    const char* e;
    if ((e = getenv("SZGB_W2"))) c->W2 = std::max(1, std::min(kMaxWaveWarps, atoi(e)));
    if ((e = getenv("SZGB_W3"))) c->W3 = std::max(1, std::min(kMaxWaveWarps, atoi(e)));
    *out = c;
    return SZGB_OK;
}

void szgb_destroy(szgb_ctx* c) {
    if (!c) return;
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    if (c->scratch) cudaFree(c->scratch);
    if (c->h_state) cudaFreeHost(c->h_state);
    for (int i = 0; i < PH_N; i++) {
        if (c->ev0[i]) cudaEventDestroy(c->ev0[i]);
        if (c->ev1[i]) cudaEventDestroy(c->ev1[i]);
    }
    drop_graph(c->g_comp);
    drop_graph(c->g_dec);
    for (int k = 0; k < kAux; k++) {
        if (c->aux[k]) cudaStreamDestroy(c->aux[k]);
        if (c->ev_join[k]) cudaEventDestroy(c->ev_join[k]);
    }
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->h_batch) cudaFreeHost(c->h_batch);
    if (c->own_stream) cudaStreamDestroy(c->own_stream);
    delete c;
}

// Batches: the fields the wavefront carries run as one batch (one persistent
// launch per pass); the others (3D n = 3, 4; 4D; the lattice variant) follow
// one by one on their own kernels through the single-field path.  Every
// field's result is that of the single-field call; the return value is the
// error of the first field (in batch order) that failed.
int szgb_compress_batch(szgb_ctx* c, int count, const float* const* data_dev, const szgb_params* params,
                        uint8_t* const* out_dev, const size_t* out_cap, size_t* out_len, szgb_stats* opt_stats) {
    if (!c || count < 1 || !data_dev || !params || !out_dev || !out_cap || !out_len) return SZGB_EINVAL;
    std::vector<int> wave, side;
    for (int f = 0; f < count; f++) {
        CallParams cp;
        int rc = check_params(&params[f], &cp);
        if (rc) return rc;
        if (!data_dev[f] || !out_dev[f] || ((uintptr_t)data_dev[f] % 16) || ((uintptr_t)out_dev[f] % 4))
            return SZGB_EINVAL;
        (wave_carries(cp) ? wave : side).push_back(f);
    }
    if (side.empty()) return compress_batch_impl(c, count, data_dev, params, out_dev, out_cap, out_len, opt_stats);
    std::vector<szgb_stats> st(count);
    std::vector<int> status(count, SZGB_OK);
    if (!wave.empty()) {
        const size_t k = wave.size();
        std::vector<const float*> d(k);
        std::vector<szgb_params> p(k);
        std::vector<uint8_t*> o(k);
        std::vector<size_t> cap(k), len(k);
        std::vector<szgb_stats> ws(k);
        for (size_t i = 0; i < k; i++) {
            d[i] = data_dev[wave[i]];
            p[i] = params[wave[i]];
            o[i] = out_dev[wave[i]];
            cap[i] = out_cap[wave[i]];
        }
        const int rc = compress_batch_impl(c, (int)k, d.data(), p.data(), o.data(), cap.data(), len.data(), ws.data());
        if (rc != SZGB_OK) {
            bool per_field = false;  // a field's own error, or one of the whole call
            for (size_t i = 0; i < k; i++) per_field |= ws[i].status == rc;
            if (!per_field) return rc;
        }
        for (size_t i = 0; i < k; i++) {
            out_len[wave[i]] = len[i];
            st[wave[i]] = ws[i];
            status[wave[i]] = ws[i].status;
        }
    }
    for (int f : side) {
        szgb_stats one = {};
        status[f] = compress_impl(c, data_dev[f], 1, &params[f], out_dev[f], out_cap[f], 1, &out_len[f], &one,
                                  nullptr, nullptr);
        if (status[f] == SZGB_ECUDA) return status[f];
        one.status = status[f];
        st[f] = one;
    }
    int first = SZGB_OK;
    for (int f = 0; f < count && !first; f++) first = status[f];
    if (opt_stats)
        for (int f = 0; f < count; f++) opt_stats[f] = st[f];
    return first;
}

int szgb_decompress_batch(szgb_ctx* c, int count, const uint8_t* const* in_dev, const size_t* in_len,
                          float* const* out_dev, const size_t* out_cap_elems, int* opt_status) {
    if (!c || count < 1 || !in_dev || !in_len || !out_dev || !out_cap_elems) return SZGB_EINVAL;
    if (cudaSetDevice(c->device) != cudaSuccess) return SZGB_ECUDA;
    // every header to the host (one small copy per field, one synchronisation)
    int rc = ensure_pinned(c, (size_t)count * kHeaderBytes);
    if (rc) return rc;
    for (int f = 0; f < count; f++) {
        if (!in_dev[f] || !out_dev[f] || ((uintptr_t)in_dev[f] % 4) || ((uintptr_t)out_dev[f] % 16) ||
            in_len[f] < (size_t)kHeaderBytes)
            return SZGB_EINVAL;
        if (cudaMemcpyAsync(static_cast<char*>(c->h_batch) + (size_t)f * kHeaderBytes, in_dev[f], kHeaderBytes,
                            cudaMemcpyDeviceToHost, c->stream) != cudaSuccess)
            return SZGB_ECUDA;
    }
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return SZGB_ECUDA;
    std::vector<uint8_t> hdr(static_cast<uint8_t*>(c->h_batch), static_cast<uint8_t*>(c->h_batch) + (size_t)count * kHeaderBytes);
    std::vector<int> wave, side;
    for (int f = 0; f < count; f++) {
        Header H;
        if ((rc = parse_header(hdr.data() + (size_t)f * kHeaderBytes, in_len[f], &H))) return rc;
        (wave_carries(H) ? wave : side).push_back(f);
    }
    if (side.empty())
        return decompress_batch_impl(c, count, in_dev, in_len, out_dev, out_cap_elems, opt_status, hdr.data());
    std::vector<int> status(count, SZGB_OK);
    if (!wave.empty()) {
        const size_t k = wave.size();
        std::vector<const uint8_t*> in(k);
        std::vector<size_t> len(k), cap(k);
        std::vector<float*> o(k);
        std::vector<uint8_t> h(k * kHeaderBytes);
        std::vector<int> ws(k, SZGB_OK);
        for (size_t i = 0; i < k; i++) {
            in[i] = in_dev[wave[i]];
            len[i] = in_len[wave[i]];
            o[i] = out_dev[wave[i]];
            cap[i] = out_cap_elems[wave[i]];
            memcpy(h.data() + i * kHeaderBytes, hdr.data() + (size_t)wave[i] * kHeaderBytes, kHeaderBytes);
        }
        rc = decompress_batch_impl(c, (int)k, in.data(), len.data(), o.data(), cap.data(), ws.data(), h.data());
        if (rc != SZGB_OK) {
            bool per_field = false;  // a field's own error, or one of the whole call
            for (size_t i = 0; i < k; i++) per_field |= ws[i] == rc;
            if (!per_field) return rc;
        }
        for (size_t i = 0; i < k; i++) status[wave[i]] = ws[i];
    }
    for (int f : side) {
        status[f] = decompress_impl(c, in_dev[f], in_len[f], 1, out_dev[f], out_cap_elems[f], 1);
        if (status[f] == SZGB_ECUDA) return status[f];
    }
    int first = SZGB_OK;
    for (int f = 0; f < count && !first; f++) first = status[f];
    if (opt_status)
        for (int f = 0; f < count; f++) opt_status[f] = status[f];
    return first;
}

int szgb_autotune(szgb_ctx* c, const float* data_dev, const szgb_params* p, int reps, int* W_out, int* pub_out,
                  double* ms_out) {
    CallParams cp;
    if (!c || !data_dev || !p) return SZGB_EINVAL;
    int rc = check_params(p, &cp);
    if (rc) return rc;
    if (cp.D4 || !layers_supported(cp.ndim, cp.layers)) return SZGB_EUNSUPPORTED;  // it tunes the wavefront
    if (cudaSetDevice(c->device) != cudaSuccess) return SZGB_ECUDA;
    if (reps < 1) reps = 1;
    const uint64_t N = cp.d0 * cp.d1 * cp.d2;
    const size_t bound = szgb_compress_bound(p);
    uint8_t* sbuf = nullptr;
    float* ybuf = nullptr;
    cudaEvent_t e0, e1;
    if (cudaMalloc(&sbuf, bound) != cudaSuccess || cudaMalloc(&ybuf, N * 4) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(sbuf);
        return SZGB_ENOMEM;
    }
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int Ws3[] = {2, 4, 6, 8}, Ws2[] = {1, 2, 4, 8};
    const int* Ws = cp.ndim == 3 ? Ws3 : Ws2;
    double best = 1e30;
    int bW = c->W3;
    uint32_t bC = SZGB_CHUNK_ROWS;
    const bool prof = c->profiling;
    c->profiling = false;
    // best of reps timed runs of one (shape, chunk) candidate (the first run warms up)
    auto time_candidate = [&](int W, uint32_t C) -> double {
        c->force_W = W;
        c->force_chunk = C;
        double tmin = 1e30;
        for (int r = 0; r <= reps && !rc; r++) {
            size_t olen = 0;
            cudaEventRecord(e0, c->stream);
            rc = compress_impl(c, data_dev, 1, p, sbuf, bound, 1, &olen, nullptr, nullptr, nullptr);
            if (!rc) rc = decompress_impl(c, sbuf, olen, 1, ybuf, N, 1);
            cudaEventRecord(e1, c->stream);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (r > 0) tmin = std::min(tmin, (double)ms);
        }
        return tmin;
    };
    // the wavefront shape with whole-row chunks, then the chunk length with that shape
    for (int wi = 0; wi < 4 && !rc; wi++) {
        if (cp.ndim == 3 && Ws[wi] < 2 * cp.layers) continue;
        const double t = time_candidate(Ws[wi], SZGB_CHUNK_ROWS);
        if (!rc && t < best) {
            best = t;
            bW = Ws[wi];
        }
    }
    const uint32_t Cs[] = {128, 256, 512, 1024};
    for (int ci = 0; ci < 4 && !rc; ci++) {
        if (Cs[ci] >= cp.d2) continue;
        const double t = time_candidate(bW, Cs[ci]);
        if (!rc && t < best) {
            best = t;
            bC = Cs[ci];
        }
    }
    c->force_W = 0;
    c->force_chunk = 0;
    c->profiling = prof;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sbuf);
    cudaFree(ybuf);
    if (rc) return rc;
    c->tune[shape_class(cp, cp.layers)] = szgb_ctx::Tune{bW, bC, best};
    drop_graph(c->g_comp);  // captured batches used the previous shapes
    drop_graph(c->g_dec);
    if (W_out) *W_out = bW;
    if (pub_out) *pub_out = (int)bC;
    if (ms_out) *ms_out = best;
    return SZGB_OK;
}

int szgb_autotune_batch(szgb_ctx* c, int count, const float* const* data_dev, const szgb_params* params, int reps,
                        int* W_out, int* pub_out, double* ms_out) {
    if (!c || count < 1 || !data_dev || !params) return SZGB_EINVAL;
    if (cudaSetDevice(c->device) != cudaSuccess) return SZGB_ECUDA;
    if (reps < 1) reps = 1;
    std::vector<CallParams> cps(count);
    std::vector<uint8_t*> sb(count, nullptr);
    std::vector<float*> yb(count, nullptr);
    std::vector<size_t> cap(count), len(count), ycap(count);
    int rc = SZGB_OK;
    bool any3 = false;
    int maxl = 1;
    for (int f = 0; f < count && !rc; f++) {
        rc = check_params(&params[f], &cps[f]);
        if (rc == SZGB_OK && (cps[f].D4 || !layers_supported(cps[f].ndim, cps[f].layers))) rc = SZGB_EUNSUPPORTED;
        if (rc) break;
        any3 |= cps[f].ndim == 3;
        maxl = std::max(maxl, cps[f].layers);
        cap[f] = szgb_compress_bound(&params[f]);
        ycap[f] = cps[f].d0 * cps[f].d1 * cps[f].d2;
        if (cudaMalloc(&sb[f], cap[f]) != cudaSuccess || cudaMalloc(&yb[f], ycap[f] * 4) != cudaSuccess) {
            cudaGetLastError();
            rc = SZGB_ENOMEM;
        }
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const bool graphs = c->use_graphs;
    c->use_graphs = false;
    const int Ws[] = {1, 2, 4, 6, 8};
    double best = 1e30;
    int bW = c->W3;
    uint32_t bC = SZGB_CHUNK_ROWS;
    uint64_t minrow = ~0ull;
    for (int f = 0; f < count && !rc; f++) minrow = std::min(minrow, cps[f].d2);
    auto time_candidate = [&](int W, uint32_t C) -> double {
        c->force_W = W;
        c->force_chunk = C;
        double tmin = 1e30;
        for (int r = 0; r <= reps && !rc; r++) {
            cudaEventRecord(e0, c->stream);
            rc = compress_batch_impl(c, count, data_dev, params, sb.data(), cap.data(), len.data(), nullptr);
            if (!rc) rc = decompress_batch_impl(c, count, sb.data(), len.data(), yb.data(), ycap.data(), nullptr);
            cudaEventRecord(e1, c->stream);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (r > 0) tmin = std::min(tmin, (double)ms);
        }
        return tmin;
    };
    for (int wi = 0; wi < 5 && !rc; wi++) {
        if (any3 && Ws[wi] < 2 * maxl) continue;
        const double t = time_candidate(Ws[wi], SZGB_CHUNK_ROWS);
        if (!rc && t < best) {
            best = t;
            bW = Ws[wi];
        }
    }
    const uint32_t Cs[] = {128, 512};
    for (int ci = 0; ci < 2 && !rc; ci++) {
        if (Cs[ci] >= minrow) continue;  // some field would keep whole rows: no clear measurement
        const double t = time_candidate(bW, Cs[ci]);
        if (!rc && t < best) {
            best = t;
            bC = Cs[ci];
        }
    }
    c->force_W = 0;
    c->force_chunk = 0;
    c->use_graphs = graphs;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    for (int f = 0; f < count; f++) {
        cudaFree(sb[f]);
        cudaFree(yb[f]);
    }
    if (rc) return rc;
    for (int f = 0; f < count; f++) c->tune[shape_class(cps[f], cps[f].layers)] = szgb_ctx::Tune{bW, bC, best};
    drop_graph(c->g_comp);
    drop_graph(c->g_dec);
    if (W_out) *W_out = bW;
    if (pub_out) *pub_out = (int)bC;
    if (ms_out) *ms_out = best;
    return SZGB_OK;
}

int szgb_tune_save(szgb_ctx* c, const char* path) {
    if (!c || !path) return SZGB_EINVAL;
    FILE* f = fopen(path, "w");
    if (!f) return SZGB_EINVAL;
    fprintf(f, "# szgb autotune v2: shape_class W chunk ms (chunk 4294967295: whole rows)\n");
    for (auto& kv : c->tune)
        fprintf(f, "%016llx %d %u %.6f\n", (unsigned long long)kv.first, kv.second.W, kv.second.chunk, kv.second.ms);
    fclose(f);
    return SZGB_OK;
}

int szgb_tune_load(szgb_ctx* c, const char* path) {
    if (!c || !path) return SZGB_EINVAL;
    FILE* f = fopen(path, "r");
    if (!f) return SZGB_EINVAL;
    char line[256];
    int rc = SZGB_OK;
    while (fgets(line, sizeof line, f)) {
        if (line[0] == '#' || line[0] == '\n') continue;
        unsigned long long k;
        int W;
        unsigned long C;  // a version-1 table held 0 here (whole rows)
        double ms;
        if (sscanf(line, "%llx %d %lu %lf", &k, &W, &C, &ms) != 4 || W < 1 || W > kMaxWaveWarps ||
            !(C == 0 || C == SZGB_CHUNK_ROWS || (C >= 32 && C <= 0x80000000ul && (C & (C - 1)) == 0))) {
            rc = SZGB_ECORRUPT;
            break;
        }
        c->tune[(uint64_t)k] = szgb_ctx::Tune{W, C ? (uint32_t)C : SZGB_CHUNK_ROWS, ms};
    }
    fclose(f);
    drop_graph(c->g_comp);
    drop_graph(c->g_dec);
    return rc;
}

int szgb_set_graphs(szgb_ctx* c, int on) {
    if (!c) return SZGB_EINVAL;
    c->use_graphs = on != 0;
    if (!c->use_graphs) {
        drop_graph(c->g_comp);
        drop_graph(c->g_dec);
    }
    return SZGB_OK;
}

int szgb_set_wave_ctas(szgb_ctx* c, int max_ctas) {
    if (!c || max_ctas < 0) return SZGB_EINVAL;
    c->wave_ctas = max_ctas;
    return SZGB_OK;
}

int szgb_debug_set_wait_limit(szgb_ctx* c, uint64_t ns) {
    if (!c) return SZGB_EINVAL;
    c->timeout_ns = ns ? ns : 4000000000ull;
    return SZGB_OK;
}

int szgb_debug_skip_item(szgb_ctx* c, int item) {
    if (!c || item < -1) return SZGB_EINVAL;
    c->debug_skip = item + 1;
    return SZGB_OK;
}

int szgb_quality_dev(szgb_ctx* c, const float* x_dev, const float* y_dev, size_t n, szgb_quality* out) {
    if (!c || !x_dev || !y_dev || !out || n == 0) return SZGB_EINVAL;
    if (cudaSetDevice(c->device) != cudaSuccess) return SZGB_ECUDA;
    const int blocks = quality_blocks(n, c->sm_count);
    const size_t need = quality_scratch_bytes(blocks);
    int rc;
    if ((rc = ensure_scratch(c, need))) return rc;
    if ((rc = ensure_pinned(c, 16 * sizeof(double)))) return rc;
    cudaStream_t s = c->stream;
    // the counter word at the end of the scratch starts at 0 (the kernel leaves it at 0)
    char* scratch = static_cast<char*>(c->scratch);
    const size_t counter_off = (size_t)(blocks + 1) * 9 * sizeof(double);
    if (cudaMemsetAsync(scratch + counter_off, 0, sizeof(unsigned), s) != cudaSuccess) return SZGB_ECUDA;
    double* h = static_cast<double*>(c->h_batch);
    if ((rc = launch_quality(x_dev, y_dev, n, blocks, scratch, h, s))) return rc;
    if (cudaStreamSynchronize(s) != cudaSuccess) return SZGB_ECUDA;
    const double se = h[0], sx = h[1], sy = h[2], sxx = h[3], syy = h[4], sxy = h[5];
    const double nn = (double)n;
    out->n = n;
    out->x_min = h[7];
    out->x_max = h[8];
    out->max_abs_err = h[6];
    const double rx = h[8] - h[7];
    out->rmse = std::sqrt(se / nn);
    out->max_rel_err = rx > 0 ? out->max_abs_err / rx : std::nan("");
    out->nrmse = rx > 0 ? out->rmse / rx : std::nan("");
    out->psnr = out->rmse == 0.0 ? INFINITY : (rx > 0 ? 20.0 * std::log10(rx / out->rmse) : std::nan(""));
    // moments of x - x_0 and y - x_0 (the shift cancels)
    const double mx = sx / nn, my = sy / nn;
    const double vx = sxx / nn - mx * mx, vy = syy / nn - my * my, cv = sxy / nn - mx * my;
    out->pearson = (vx > 0 && vy > 0) ? cv / std::sqrt(vx * vy) : std::nan("");
    return SZGB_OK;
}

int szgb_hit_count_dev(szgb_ctx* c, const float* x_dev, const float* v_dev, int ndim, const uint64_t* shape,
                       int layers, double eb, uint64_t* n_hit) {
    if (!c || !x_dev || !v_dev || !shape || !n_hit || ndim < 1 || ndim > 4 || layers < 1 || layers > kMaxLayers ||
        !(eb >= 0.0))
        return SZGB_EINVAL;
    uint64_t d[4] = {1, 1, 1, 1};  // slowest first; 1D-3D fields use d[1..3]
    for (int a = 0; a < ndim; a++) {
        if (shape[a] == 0 || shape[a] > 0xffffffffull) return SZGB_EINVAL;
        d[4 - ndim + a] = shape[a];
    }
    if ((unsigned __int128)d[0] * d[1] * d[2] * d[3] >= ((unsigned __int128)1 << 40)) return SZGB_EINVAL;
    if (cudaSetDevice(c->device) != cudaSuccess) return SZGB_ECUDA;
    int rc;
    if ((rc = ensure_scratch(c, 64))) return rc;
    if ((rc = ensure_pinned(c, 16 * sizeof(double)))) return rc;
    cudaStream_t s = c->stream;
    unsigned long long* count = static_cast<unsigned long long*>(c->scratch);
    if (cudaMemsetAsync(count, 0, sizeof(unsigned long long), s) != cudaSuccess) return SZGB_ECUDA;
    if (ndim == 4) rc = launch_hits4(x_dev, v_dev, d[0], d[1], d[2], d[3], layers, eb, count, c->sm_count, s);
    else rc = launch_hits(x_dev, v_dev, d[1], d[2], d[3], ndim, layers, eb, count, c->sm_count, s);
    if (rc) return rc;
    unsigned long long* h = static_cast<unsigned long long*>(c->h_batch);
    if (cudaMemcpyAsync(h, count, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return SZGB_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return SZGB_ECUDA;
    *n_hit = h[0];
    return SZGB_OK;
}

int szgb_set_stream(szgb_ctx* c, void* stream) {
    if (!c) return SZGB_EINVAL;
    cudaStream_t ns = stream ? static_cast<cudaStream_t>(stream) : c->own_stream;
    if (ns != c->stream) {  // captured graphs were recorded on the old stream
        drop_graph(c->g_comp);
        drop_graph(c->g_dec);
    }
    c->stream = ns;
    return SZGB_OK;
}

size_t szgb_compress_bound(const szgb_params* p) {
    CallParams cp;
    if (!p) return 0;
    int rc = check_params(p, &cp);
    if (rc != SZGB_OK && rc != SZGB_EUNSUPPORTED) return 0;
    uint64_t N = cp.d0 * cp.d1 * cp.d2, rows = cp.d0 * cp.d1;
    const uint64_t nch = rows * ((cp.d2 + 31) / 32);  // the most chunks (32 points each)
    // header + codebook + table + per point at most a 64-bit code and its
    // record (9 + 23 bits; lattice variant: 1 + 64 + 32 bits) + chunk padding
    const uint64_t per = cp.variant == SZGB_VARIANT_LATTICE ? 21 : 12;
    return (size_t)(kHeaderBytes + 3 * 65536 + 4 + 4 * nch + 4 + nch + N * per + 16);
}

int szgb_compress(szgb_ctx* c, const float* data, int data_on_device, const szgb_params* p, uint8_t* out,
                  size_t out_cap, int out_on_device, size_t* out_len, szgb_stats* opt_stats) {
    if (!out) return SZGB_EINVAL;
    return compress_impl(c, data, data_on_device, p, out, out_cap, out_on_device, out_len, opt_stats, nullptr,
                         nullptr);
}

int szgb_compress_trace(szgb_ctx* c, const float* data_dev, const szgb_params* p, uint8_t* out_dev,
                        size_t out_cap, size_t* out_len, szgb_stats* opt_stats, float* recorded_dev,
                        uint16_t* codes_dev) {
    if (!out_dev) return SZGB_EINVAL;
    return compress_impl(c, data_dev, 1, p, out_dev, out_cap, 1, out_len, opt_stats, recorded_dev, codes_dev);
}

int szgb_compress_4d(szgb_ctx* c, const float* data_dev, const uint64_t* shape, const szgb_params* p,
                     uint8_t* out_dev, size_t out_cap, size_t* out_len, szgb_stats* opt_stats, float* recorded_dev,
                     uint16_t* codes_dev) {
    if (!c || !data_dev || !shape || !p || !out_dev || !out_len) return SZGB_EINVAL;
    if (p->variant != SZGB_VARIANT_EXACT) return SZGB_EUNSUPPORTED;
    szgb_params q = *p;
    q.ndim = 4;
    for (int a = 0; a < 4; a++) q.shape[a] = shape[a];
    return compress_impl(c, data_dev, 1, &q, out_dev, out_cap, 1, out_len, opt_stats, recorded_dev, codes_dev);
}

int szgb_decompress(szgb_ctx* c, const uint8_t* in, size_t in_len, int in_on_device, float* out,
                    size_t out_cap_elems, int out_on_device) {
    return decompress_impl(c, in, in_len, in_on_device, out, out_cap_elems, out_on_device);
}

int szgb_suggest_m(const szgb_stats* st, double theta, double* hit_rate_out) {
    if (!st || st->n_points == 0 || st->n_unpred > st->n_points || st->m < 2 || st->m > 16 || !(theta == theta))
        return SZGB_EINVAL;
    // predictable points: those that fell into one of the 2^m - 1 intervals
    const double rate = (double)(st->n_points - st->n_unpred) / (double)st->n_points;
    if (hit_rate_out) *hit_rate_out = rate;
    return (rate < theta && st->m < 16) ? st->m + 1 : st->m;
}

int szgb_stream_info(const uint8_t* in_host, size_t in_len, szgb_params* out, uint64_t* n_unpred) {
    if (!in_host || !out) return SZGB_EINVAL;
    Header H;
    int rc = parse_header(in_host, in_len, &H);
    if (rc) return rc;
    memset(out, 0, sizeof(*out));
    if (H.D4) {
        out->ndim = 4;
        out->shape[0] = H.D4;
        out->shape[1] = H.d0 / H.D4;
        out->shape[2] = H.d1;
        out->shape[3] = H.d2;
    } else {
        out->ndim = H.ndim;
        uint64_t d[3] = {H.d0, H.d1, H.d2};
        for (int a = 0; a < H.ndim; a++) out->shape[a] = d[3 - H.ndim + a];
    }
    out->mode = H.mode;
    out->eb_abs = H.eb_abs;
    out->eb_rel = H.eb_rel;
    out->layers = H.layers;
    out->m = H.m;
    out->theta = H.theta;
    out->variant = H.variant;
    out->chunk_points = H.chunk ? H.chunk : SZGB_CHUNK_ROWS;
    if (n_unpred) *n_unpred = H.K;
    return SZGB_OK;
}

int szgb_set_profiling(szgb_ctx* c, int on) {
    if (!c) return SZGB_EINVAL;
    c->profiling = on != 0;
    return SZGB_OK;
}
int szgb_num_phases(void) { return PH_N; }
const char* szgb_phase_name(int i) { return (i >= 0 && i < PH_N) ? kPhaseNames[i] : ""; }
int szgb_phase_times(szgb_ctx* c, double* ms, uint64_t* calls, int n, int reset) {
    if (!c) return SZGB_EINVAL;
    for (int i = 0; i < n && i < PH_N; i++) {
        if (ms) ms[i] = c->ph_ms[i];
        if (calls) calls[i] = c->ph_calls[i];
    }
    if (reset) {
        for (int i = 0; i < PH_N; i++) { c->ph_ms[i] = 0; c->ph_calls[i] = 0; }
    }
    return SZGB_OK;
}

const char* szgb_strerror(int code) {
    switch (code) {
        case SZGB_OK: return "ok";
        case SZGB_EINVAL: return "invalid argument";
        case SZGB_ENONFINITE: return "input holds NaN or Inf";
        case SZGB_ETRUNC: return "output buffer too small";
        case SZGB_ECORRUPT: return "corrupt stream";
        case SZGB_ENOMEM: return "device allocation failed";
        case SZGB_EBUDGET: return "device memory budget exceeded";
        case SZGB_ETIMEOUT: return "device-side wait timed out";
        case SZGB_ECUDA: return "CUDA runtime error";
        case SZGB_EUNSUPPORTED: return "not supported on the GPU path";
        case SZGB_ESCRATCH: return "needs more than the fixed scratch of szgb_decompress_noalloc";
        default: return "unknown error";
    }
}

}  // extern "C"
