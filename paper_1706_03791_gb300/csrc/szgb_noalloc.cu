// szgb_noalloc.cu -- decompression that allocates no memory.
//
// Some callers cannot call cudaMalloc: a service that must keep a fixed
// device-memory plan for its whole life (an allocation that fails at an
// arbitrary moment, or that fragments a pre-planned pool, is not allowed
// there), or code that runs inside an allocator or framework callback, where
// allocating would re-enter the allocator.  szgb_decompress_noalloc serves
// them.  It runs the same kernels as szgb_decompress, but every scratch
// buffer those kernels use (halo rows/planes, progress counters, per-row byte
// lengths and offsets, decoder tables, call state) is carved out of the fixed
// array below, which every GPU that loads this library holds until the
// process exits.  Inputs and outputs are the caller's device buffers.
//
// The array is shared by every call on a device and keeps the last call's
// contents; what must start at zero is cleared on the stream at the start of
// each call.  Calls whose work overlaps on the GPU (two host threads, or two
// streams) race on the array.
#include <string.h>

#include <mutex>

#include "szgb_internal.cuh"

using namespace szgb;

namespace {

constexpr size_t kNoAllocScratchBytes = 128ull << 20;  // 128 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_setup_mu;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of the array on the current device, looked up once per
// device.  The host-side symbol is not a device address; only this address
// may be handed to kernels.
int scratch_address(void** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return SZGB_ECUDA;
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return SZGB_ECUDA;
        }
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return SZGB_OK;
}

size_t up256(size_t v) { return (v + 255) & ~(size_t)255; }

}  // namespace

extern "C" int szgb_decompress_noalloc(const uint8_t* in_dev, size_t in_len, float* out_dev,
                                       size_t out_cap_elems, void* cuda_stream) {
    if (!in_dev || !out_dev || in_len < (size_t)kHeaderBytes) return SZGB_EINVAL;
    if ((uintptr_t)in_dev % 4 || (uintptr_t)out_dev % 16) return SZGB_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    void* base = nullptr;
    int rc = scratch_address(&base);
    if (rc) return rc;

    // header (128 bytes) to the host stack
    uint8_t h[kHeaderBytes];
    if (cudaMemcpyAsync(h, in_dev, kHeaderBytes, cudaMemcpyDeviceToHost, s) != cudaSuccess) return SZGB_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return SZGB_ECUDA;
    Header H;
    if ((rc = parse_header(h, in_len, &H))) return rc;
    if (H.variant != SZGB_VARIANT_EXACT) return SZGB_EUNSUPPORTED;
    // 3D fields with n = 3, 4 and 4D fields: the hyperplane kernels (no halo
    // lines, no item states) after the same row decode
    const bool hyper = !wave_carries(H);
    const int ndim = H.ndim, layers = H.layers, m = H.m, tw = H.tw;
    const uint64_t d2 = H.d2;
    const uint32_t nsym = H.nsym;
    const uint64_t rows = H.d0 * H.d1, nch = H.nchunks, payload_bytes = H.payload;
    const uint64_t cb = (3ull * nsym + 3) & ~3ull, tb = ((uint64_t)tw * nch + 3) & ~3ull;

    // wavefront geometry: the same schedule as szgb_decompress with its
    // default shape (any valid schedule gives the same values)
    CallParams cp = {};
    cp.ndim = ndim;
    cp.d0 = H.d0;
    cp.d1 = H.d1;
    cp.d2 = H.d2;
    cp.layers = layers;
    const WaveGeom g = make_geom_w(cp, layers, kMaxWaveWarps, kMaxWaveWarps);
    size_t hrow = 0, hplane = 0;  // halo lines in 32-bit units
    if (!hyper) halo_sizes(g, layers, &hrow, &hplane);

    // carve the scratch
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = up256(off + (bytes ? bytes : 1)); return o; };
    const size_t o_st = take(sizeof(DevState));
    const size_t o_hrow = take((hrow + hplane) * 4), o_hplane = o_hrow + hrow * 4;
    const size_t o_prog = take((size_t)g.num_ctas * 4);
    const size_t o_rb = take(nch * 4), o_ro = take(nch * 8), o_bs = take(((nch + 2047) / 2048 + 1) * 8);
    const size_t o_lut = take(((size_t)1 << kLutBits) * 4), o_tab = take(kDecTabU32 * 4);
    const size_t o_len = take(65536), o_sym = take(65536 * 4);
    const uint64_t cpitch = (d2 + 7) & ~7ull;
    const size_t o_codes = take((rows * cpitch + 8) * 2);
    if (off > kNoAllocScratchBytes) return SZGB_ESCRATCH;
    if (out_cap_elems < H.d0 * H.d1 * H.d2) return SZGB_EINVAL;
    char* b = static_cast<char*>(base);
    DevState* st = reinterpret_cast<DevState*>(b + o_st);
    unsigned int* prog = reinterpret_cast<unsigned int*>(b + o_prog);
    uint32_t* rowbytes = reinterpret_cast<uint32_t*>(b + o_rb);
    uint64_t* rowoff = reinterpret_cast<uint64_t*>(b + o_ro);

    // clear what starts at zero: the call state, the item states and the halo lines
    uint32_t ebu;
    memcpy(&ebu, &H.eb_f, 4);
    DevState init = {};
    init.eb_f = H.eb_f;
    init.twoeb = 2.0f * H.eb_f;
    init.m = m;
    init.center = 1 << (m - 1);
    init.radius = (float)((1 << (m - 1)) - 1);
    init.e_eb = (int)((ebu >> 23) & 0xffu);
    if (cudaMemcpyAsync(st, &init, sizeof(DevState), cudaMemcpyHostToDevice, s) != cudaSuccess) return SZGB_ECUDA;
    if (cudaMemsetAsync(prog, 0, (size_t)g.num_ctas * 4, s) != cudaSuccess) return SZGB_ECUDA;
    if (cudaMemsetAsync(b + o_hrow, 0, (hrow + hplane) * 4, s) != cudaSuccess) return SZGB_ECUDA;

    const uint8_t* codebook = in_dev + kHeaderBytes;
    const uint8_t* table = codebook + cb;
    const uint8_t* payload = table + tb;
    uint32_t* lut = reinterpret_cast<uint32_t*>(b + o_lut);
    uint32_t* dectab = reinterpret_cast<uint32_t*>(b + o_tab);
    if ((rc = launch_decode_tables(codebook, nsym, m, lut, dectab, reinterpret_cast<uint8_t*>(b + o_len),
                                   reinterpret_cast<uint32_t*>(b + o_sym), st, s)))
        return rc;
    if ((rc = launch_scan_rows(rowbytes, nch, rowoff, reinterpret_cast<uint64_t*>(b + o_bs), st, 0, s, table, tw)))
        return rc;
    uint16_t* codes = reinterpret_cast<uint16_t*>(b + o_codes);
    if ((rc = launch_decode_rows(payload, rowoff, rowbytes, payload + payload_bytes, lut, dectab, codes, cpitch,
                                 out_dev, rows, d2, H.chunk, st, s)))
        return rc;
    if (H.D4) {
        rc = launch_hyper4(true, layers, nullptr, out_dev, codes, cpitch, H.D4, H.d0 / H.D4, H.d1, H.d2, st, s);
    } else if (hyper) {
        rc = launch_hyper_decompress(layers, codes, cpitch, out_dev, H.d0, H.d1, H.d2, st, s);
    } else {
        rc = launch_wave_decompress(g, layers, codes, cpitch, out_dev, reinterpret_cast<float*>(b + o_hrow),
                                    reinterpret_cast<float*>(b + o_hplane), prog, st, 4000000000ull, s);
    }
    if (rc) return rc;
    DevState hs;
    if (cudaMemcpyAsync(&hs, st, sizeof(DevState), cudaMemcpyDeviceToHost, s) != cudaSuccess) return SZGB_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return SZGB_ECUDA;
    if ((rc = dev_errors(hs))) return rc;
    if (hs.payload != payload_bytes) return SZGB_ECORRUPT;
    return SZGB_OK;
}
