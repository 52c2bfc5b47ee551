// szgb_server.cu -- serving loop: compress / decompress requests taken as they
// arrive, admitted by a device-memory budget, run as batches on several
// worker contexts whose work overlaps on the GPU (continuous batching).
//
// Every worker thread owns a library context (its own stream, device scratch
// and codebook tables, all kept resident between batches) and a resident
// device I/O arena.  A worker takes pending requests in arrival order that
// fit in the budget (at most max_batch), copies their host inputs to the
// device, runs one batched compression and one batched decompression, copies
// the results back and completes the requests.  Requests that arrive while a
// batch is on the GPU wait for the next free worker; with several workers,
// the copies and kernels of different batches overlap.
//
// Batches are formed by size, so that small requests do not wait behind
// large ones: a large request (I/O of kLargeBytes or more, or a field the
// wavefront does not carry: 3D n = 3, 4, 4D, the lattice variant) runs alone, a
// batch of small requests gathers at most kBatchBytes of I/O, and with two
// or more workers worker 0 takes small requests only, so that one worker is
// always free of large ones; the other workers take the oldest pending
// request's kind first.  A persistent wavefront launch holds its SMs until
// it ends, so a large request's wavefront runs on half of the SMs
// (szgb_set_wave_ctas) and small batches keep the rest.  A request's result
// is exactly the result of the single-field calls: batches change the
// schedule, never the bits.
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/szgb.h"

namespace {

size_t up256(size_t v) { return (v + 255) & ~(size_t)255; }
constexpr int kNoStatus = -1000;  // a batch call returned before reaching the field
constexpr size_t kLargeBytes = 128ull << 20;  // a request of this much I/O or more runs alone
constexpr size_t kBatchBytes = 64ull << 20;   // I/O bytes a batch of small requests gathers at most
constexpr size_t kCopyPiece = 16ull << 20;    // host<->device copies go in pieces of this size

// A host<->device copy in pieces, so that the copies of other workers'
// streams can be scheduled between them.
cudaError_t copy_pieces(void* dst, const void* src, size_t n, cudaMemcpyKind kind, cudaStream_t st) {
    for (size_t o = 0; o < n; o += kCopyPiece) {
        const size_t len = std::min(kCopyPiece, n - o);
        const cudaError_t e =
            cudaMemcpyAsync(static_cast<char*>(dst) + o, static_cast<const char*>(src) + o, len, kind, st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

struct Req {
    szgb_request r;
    uint64_t ticket = 0;
    uint64_t n_points = 0;
    size_t dev_in = 0, dev_out = 0;  // device bytes of input and output
    size_t need = 0;                  // admitted bytes (I/O + scratch estimate)
    bool wave = true;                 // runs on the batched wavefront
    int status = SZGB_OK;
    size_t out_len = 0;
    bool done = false;
};

}  // namespace

struct szgb_server {
    int device = 0;
    size_t budget = 0;
    int max_batch = 64;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Req*> pending;
    std::unordered_map<uint64_t, Req*> reqs;
    uint64_t next_ticket = 1;
    size_t reserved = 0, peak_reserved = 0;
    uint64_t batches = 0, completed = 0;
    bool stop = false;
    std::vector<std::thread> workers;
};

namespace {

// fields the batched wavefront carries: the paper's method, 1D-3D, up to
// n = 2 layers in 3D and n = 4 in 1D and 2D.  The others (3D n = 3, 4; 4D;
// the lattice variant) run on their own kernels, one field at a time.
bool on_wavefront(const szgb_params& p) {
    return p.variant == SZGB_VARIANT_EXACT && p.ndim >= 1 && p.ndim <= 3 && p.layers >= 1 &&
           p.layers <= (p.ndim == 3 ? 2 : 4);
}

// device scratch the library needs for one field, beyond its I/O buffers
// (wavefront: codes 2 B/pt, halos, per-row tables; hyperplane and lattice
// kernels: also 4-5 B/pt of recorded or lattice values; Huffman tables
// 3.6 MB per field)
size_t scratch_estimate(int op, uint64_t n_points, bool wave) {
    const double n = (double)n_points;
    if (op == SZGB_OP_COMPRESS) return (size_t)((wave ? 2.3 : 7.5) * n) + (4u << 20);
    return (size_t)((wave ? 0.3 : 5.3) * n) + (1u << 20);
}

// Debug trace: with SZGB_SERVER_TRACE=<file>, one line per batch (worker,
// requests, I/O bytes, and the seconds at which the batch was taken, its
// inputs were queued, its kernels returned and its outputs arrived).
double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}
struct Trace {
    FILE* f = nullptr;
    std::mutex mu;
    Trace() {
        const char* p = getenv("SZGB_SERVER_TRACE");
        if (p && *p) f = fopen(p, "a");
    }
    ~Trace() {
        if (f) fclose(f);
    }
};
Trace& trace() {
    static Trace t;
    return t;
}

void run_batch(szgb_server* S, szgb_ctx* ctx, cudaStream_t st, void*& dbuf, size_t& dcap,
               std::vector<Req*>& batch, double* t_in, double* t_run) {
    // device I/O layout of the batch
    std::vector<size_t> off_in(batch.size()), off_out(batch.size());
    size_t total = 0;
    for (size_t i = 0; i < batch.size(); i++) {
        off_in[i] = total;
        total += up256(batch[i]->dev_in);
        off_out[i] = total;
        total += up256(batch[i]->dev_out);
    }
    if (total > dcap) {
        if (dbuf) cudaFree(dbuf);
        dbuf = nullptr;
        dcap = 0;
        // grow at least twofold: every regrowth frees the old arena, and
        // cudaFree waits for the whole device (every worker's work)
        size_t cap = up256(std::max(total + total / 4, 2 * dcap));
        if (cudaMalloc(&dbuf, cap) != cudaSuccess) {
            cudaGetLastError();
            for (Req* q : batch) q->status = SZGB_ENOMEM;
            return;
        }
        dcap = cap;
    }
    char* D = static_cast<char*>(dbuf);
    for (size_t i = 0; i < batch.size(); i++) {
        if (copy_pieces(D + off_in[i], batch[i]->r.in, batch[i]->r.in_bytes, cudaMemcpyHostToDevice, st) !=
            cudaSuccess) {
            for (Req* q : batch) q->status = SZGB_ECUDA;
            return;
        }
    }
    *t_in = now_s();
    // one batched call per operation
    std::vector<size_t> ci, di;
    for (size_t i = 0; i < batch.size(); i++) (batch[i]->r.op == SZGB_OP_COMPRESS ? ci : di).push_back(i);
    if (!ci.empty()) {
        const int n = (int)ci.size();
        std::vector<const float*> in(n);
        std::vector<szgb_params> prm(n);
        std::vector<uint8_t*> out(n);
        std::vector<size_t> cap(n), len(n);
        std::vector<szgb_stats> sts(n);
        for (auto& x : sts) x.status = kNoStatus;
        for (int k = 0; k < n; k++) {
            const size_t i = ci[k];
            in[k] = reinterpret_cast<const float*>(D + off_in[i]);
            prm[k] = batch[i]->r.params;
            out[k] = reinterpret_cast<uint8_t*>(D + off_out[i]);
            cap[k] = batch[i]->dev_out;
        }
        int rc = szgb_compress_batch(ctx, n, in.data(), prm.data(), out.data(), cap.data(), len.data(), sts.data());
        for (int k = 0; k < n; k++) {
            Req* q = batch[ci[k]];
            // a per-field code when the batch reached its fields, else the call's
            q->status = sts[k].status != kNoStatus ? sts[k].status : (rc ? rc : SZGB_ECUDA);
            q->out_len = len[k];
            if (q->status == SZGB_OK && len[k] > q->r.out_cap) q->status = SZGB_ETRUNC;
            if (q->status == SZGB_OK &&
                copy_pieces(q->r.out, D + off_out[ci[k]], len[k], cudaMemcpyDeviceToHost, st) != cudaSuccess)
                q->status = SZGB_ECUDA;
        }
    }
    *t_run = now_s();
    if (!di.empty()) {
        const int n = (int)di.size();
        std::vector<const uint8_t*> in(n);
        std::vector<size_t> inl(n), cap(n);
        std::vector<float*> out(n);
        std::vector<int> sts(n, kNoStatus);
        for (int k = 0; k < n; k++) {
            const size_t i = di[k];
            in[k] = reinterpret_cast<const uint8_t*>(D + off_in[i]);
            inl[k] = batch[i]->r.in_bytes;
            out[k] = reinterpret_cast<float*>(D + off_out[i]);
            cap[k] = batch[i]->n_points;
        }
        int rc = szgb_decompress_batch(ctx, n, in.data(), inl.data(), out.data(), cap.data(), sts.data());
        for (int k = 0; k < n; k++) {
            Req* q = batch[di[k]];
            q->status = sts[k] != kNoStatus ? sts[k] : (rc ? rc : SZGB_ECUDA);
            q->out_len = q->n_points * 4;
            if (q->status == SZGB_OK &&
                copy_pieces(q->r.out, D + off_out[di[k]], q->out_len, cudaMemcpyDeviceToHost, st) != cudaSuccess)
                q->status = SZGB_ECUDA;
        }
    }
    if (cudaStreamSynchronize(st) != cudaSuccess)
        for (Req* q : batch) q->status = SZGB_ECUDA;
}

// a large request, or one that runs on the hyperplane or lattice kernels
// (one field at a time, after the batch's wavefront fields), runs alone
bool is_large(const Req* q) { return !q->wave || q->dev_in + q->dev_out >= kLargeBytes; }

// The next batch of worker `wid` from the pending queue (caller holds the
// lock): see the file comment.  Requests are taken in arrival order within
// their kind; a request that does not fit the budget stops the scan (no
// overtaking past the budget).
void take_batch(szgb_server* S, int wid, std::vector<Req*>& batch) {
    const bool small_only = wid == 0 && S->workers.size() >= 2;
    auto take = [&](std::deque<Req*>::iterator it) {
        Req* q = *it;
        S->reserved += q->need;
        S->peak_reserved = std::max(S->peak_reserved, S->reserved);
        batch.push_back(q);
        return S->pending.erase(it);
    };
    if (!small_only && !S->pending.empty() && is_large(S->pending.front())) {  // alone
        if (S->reserved + S->pending.front()->need <= S->budget) take(S->pending.begin());
        return;
    }
    size_t bytes = 0;
    for (auto it = S->pending.begin(); it != S->pending.end() && (int)batch.size() < S->max_batch;) {
        Req* q = *it;
        if (is_large(q)) {
            ++it;
            continue;
        }
        if (S->reserved + q->need > S->budget) break;
        if (!batch.empty() && bytes + q->dev_in + q->dev_out > kBatchBytes) break;
        bytes += q->dev_in + q->dev_out;
        it = take(it);
    }
}

void worker_main(szgb_server* S, int wid) {
    cudaSetDevice(S->device);
    szgb_ctx* ctx = nullptr;
    // batches of small requests run on a high-priority stream, a large
    // request on a low-priority one: when both have work ready, the small
    // batch's thread blocks are scheduled first
    cudaStream_t st_small = nullptr, st_large = nullptr;
    int init_rc = szgb_create(&ctx, S->device, 0);
    int prio_low = 0, prio_high = 0;
    if (init_rc == SZGB_OK && cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high) != cudaSuccess)
        init_rc = SZGB_ECUDA;
    if (init_rc == SZGB_OK &&
        (cudaStreamCreateWithPriority(&st_small, cudaStreamNonBlocking, prio_high) != cudaSuccess ||
         cudaStreamCreateWithPriority(&st_large, cudaStreamNonBlocking, prio_low) != cudaSuccess))
        init_rc = SZGB_ECUDA;
    if (init_rc == SZGB_OK) szgb_set_graphs(ctx, 0);  // every batch differs: launch directly
    int sms = 0;
    if (init_rc == SZGB_OK && cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, S->device) != cudaSuccess)
        init_rc = SZGB_ECUDA;
    void* dbuf = nullptr;
    size_t dcap = 0;
    for (;;) {
        std::vector<Req*> batch;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            for (;;) {
                if (S->stop && S->pending.empty()) break;
                take_batch(S, wid, batch);
                if (!batch.empty()) break;
                // stopping with only requests this worker does not take: leave
                // them to the workers that do
                if (S->stop && wid == 0 && S->workers.size() >= 2) break;
                S->cv_work.wait(lk);
            }
            if (batch.empty()) break;  // stopping, nothing pending
        }
        const double t_take = now_s();
        double t_in = t_take, t_run = t_take;
        if (init_rc != SZGB_OK) {
            for (Req* q : batch) q->status = init_rc;
        } else {
            const bool large = batch.size() == 1 && is_large(batch[0]);
            cudaStream_t st = large ? st_large : st_small;
            szgb_set_stream(ctx, st);
            // a large request's persistent wavefront takes half of the SMs:
            // two large requests run side by side, and the small batches'
            // kernels find SMs between their launches instead of waiting for
            // whole persistent launches
            szgb_set_wave_ctas(ctx, large ? sms / 2 : 0);
            run_batch(S, ctx, st, dbuf, dcap, batch, &t_in, &t_run);
        }
        if (trace().f) {
            size_t io = 0;
            for (Req* q : batch) io += q->dev_in + q->dev_out;
            std::lock_guard<std::mutex> tl(trace().mu);
            fprintf(trace().f, "%d %zu %zu %.6f %.6f %.6f %.6f\n", wid, batch.size(), io, t_take, t_in, t_run,
                    now_s());
        }
        {
            std::lock_guard<std::mutex> lk(S->mu);
            for (Req* q : batch) {
                q->done = true;
                S->reserved -= q->need;
            }
            S->batches++;
            S->completed += batch.size();
        }
        S->cv_done.notify_all();
        S->cv_work.notify_all();  // memory came free
    }
    if (dbuf) cudaFree(dbuf);
    if (ctx) szgb_destroy(ctx);
    if (st_small) cudaStreamDestroy(st_small);
    if (st_large) cudaStreamDestroy(st_large);
}

}  // namespace

extern "C" {

int szgb_server_create(szgb_server** out, int device, size_t device_mem_budget, int workers, int max_batch) {
    if (!out || workers < 1 || workers > 16 || max_batch < 1 || device_mem_budget == 0) return SZGB_EINVAL;
    *out = nullptr;
    szgb_server* S = new (std::nothrow) szgb_server();
    if (!S) return SZGB_ENOMEM;
    S->device = device;
    S->budget = device_mem_budget;
    S->max_batch = max_batch;
    {
        // the workers read S->workers.size() under the lock
        std::lock_guard<std::mutex> lk(S->mu);
        for (int i = 0; i < workers; i++) S->workers.emplace_back(worker_main, S, i);
    }
    *out = S;
    return SZGB_OK;
}

int szgb_submit(szgb_server* S, const szgb_request* r, uint64_t* ticket) {
    if (!S || !r || !ticket || !r->in || !r->out) return SZGB_EINVAL;
    Req* q = new (std::nothrow) Req();
    if (!q) return SZGB_ENOMEM;
    q->r = *r;
    if (r->op == SZGB_OP_COMPRESS) {
        const szgb_params& p = r->params;
        if (p.ndim < 1 || p.ndim > 4) {
            delete q;
            return SZGB_EINVAL;
        }
        q->wave = on_wavefront(p);
        uint64_t n = 1;
        for (int a = 0; a < p.ndim; a++) n *= p.shape[a];
        const size_t bound = szgb_compress_bound(&p);
        if (bound == 0 || r->in_bytes != n * 4) {
            delete q;
            return SZGB_EINVAL;
        }
        q->n_points = n;
        q->dev_in = r->in_bytes;
        // the stream is written on the device first; it may not exceed the
        // caller's capacity (SZGB_ETRUNC reports the size needed)
        q->dev_out = std::min(bound, std::max(r->out_cap, (size_t)4096));
    } else if (r->op == SZGB_OP_DECOMPRESS) {
        szgb_params p;
        uint64_t k = 0;
        int rc = szgb_stream_info(static_cast<const uint8_t*>(r->in), r->in_bytes, &p, &k);
        if (rc) {
            delete q;
            return rc;
        }
        uint64_t n = 1;
        for (int a = 0; a < p.ndim; a++) n *= p.shape[a];
        if (r->out_cap < n * 4) {
            delete q;
            return SZGB_EINVAL;
        }
        q->n_points = n;
        q->dev_in = r->in_bytes;
        q->dev_out = n * 4;
        q->wave = on_wavefront(p);
    } else {
        delete q;
        return SZGB_EINVAL;
    }
    q->need = up256(q->dev_in) + up256(q->dev_out) + scratch_estimate(r->op, q->n_points, q->wave);
    if (q->need > S->budget) {
        delete q;
        return SZGB_EBUDGET;
    }
    {
        std::lock_guard<std::mutex> lk(S->mu);
        q->ticket = S->next_ticket++;
        S->reqs[q->ticket] = q;
        S->pending.push_back(q);
        *ticket = q->ticket;
    }
    S->cv_work.notify_all();  // the worker that takes it may not be the first to wake
    return SZGB_OK;
}

int szgb_poll(szgb_server* S, uint64_t ticket, int* done, int* status, size_t* out_len) {
    if (!S || !done) return SZGB_EINVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return SZGB_EINVAL;
    Req* q = it->second;
    *done = q->done ? 1 : 0;
    if (q->done) {
        if (status) *status = q->status;
        if (out_len) *out_len = q->out_len;
        S->reqs.erase(it);
        delete q;
    }
    return SZGB_OK;
}

int szgb_wait(szgb_server* S, uint64_t ticket, int* status, size_t* out_len) {
    if (!S) return SZGB_EINVAL;
    std::unique_lock<std::mutex> lk(S->mu);
    if (S->reqs.find(ticket) == S->reqs.end()) return SZGB_EINVAL;
    // look the ticket up again on every wake-up: another caller may have
    // taken the result (and freed the request) meanwhile
    S->cv_done.wait(lk, [&] {
        auto jt = S->reqs.find(ticket);
        return jt == S->reqs.end() || jt->second->done;
    });
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return SZGB_EINVAL;
    Req* q = it->second;
    if (status) *status = q->status;
    if (out_len) *out_len = q->out_len;
    S->reqs.erase(it);
    delete q;
    return SZGB_OK;
}

int szgb_server_stats(szgb_server* S, uint64_t* batches, uint64_t* completed, size_t* peak_reserved) {
    if (!S) return SZGB_EINVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    if (batches) *batches = S->batches;
    if (completed) *completed = S->completed;
    if (peak_reserved) *peak_reserved = S->peak_reserved;
    return SZGB_OK;
}

void szgb_server_destroy(szgb_server* S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    for (auto& t : S->workers) t.join();
    for (auto& kv : S->reqs) delete kv.second;
    delete S;
}

}  // extern "C"
