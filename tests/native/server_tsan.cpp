// server_tsan.cpp -- the serving loop's host concurrency under
// ThreadSanitizer: several threads submit compress and decompress requests,
// take results by wait and by poll (two takers race for some tickets), and
// one thread reads the statistics throughout; then the server is destroyed
// with requests still queued.  A second server mixes large requests (run
// alone, never by worker 0) with small ones and is destroyed with a large
// request queued.  Built by the test that runs it, with the
// server source instrumented.  On a machine without a GPU every admitted
// request completes with SZGB_ECUDA, which exercises the same queue,
// admission and completion paths.
//
// Exit status 0 when every request completed exactly once with an expected
// status; ThreadSanitizer reports make the run fail on their own.
#include <atomic>
#include <cstdio>
#include <cstring>
#include <thread>
#include <vector>

#include "../../include/szgb.h"

namespace {

constexpr int kThreads = 4, kPerThread = 24, kRows = 24, kCols = 40;

szgb_params field_params() {
    szgb_params p;
    std::memset(&p, 0, sizeof(p));
    p.ndim = 2;
    p.shape[0] = kRows;
    p.shape[1] = kCols;
    p.mode = SZGB_REL;
    p.eb_rel = 1e-3;
    p.layers = 1;
    p.m = 8;
    p.theta = 0.99;
    return p;
}

bool expected(int status) { return status == SZGB_OK || status == SZGB_ECUDA; }

}  // namespace

int main() {
    szgb_server* S = nullptr;
    if (szgb_server_create(&S, 0, 64u << 20, 3, 4) != SZGB_OK) {
        std::fprintf(stderr, "server_create failed\n");
        return 1;
    }
    const int total = kThreads * kPerThread;
    std::vector<std::vector<float>> xs(total, std::vector<float>(kRows * kCols));
    std::vector<std::vector<unsigned char>> outs(total, std::vector<unsigned char>(1 << 16));
    for (int f = 0; f < total; f++)
        for (int i = 0; i < kRows * kCols; i++) xs[f][i] = 0.001f * (float)(i % 97) + 0.01f * (float)f;

    std::atomic<int> failures{0}, taken{0}, lost_races{0};
    std::atomic<bool> stats_run{true};
    std::thread stats([&] {
        while (stats_run.load()) {
            uint64_t b = 0, c = 0;
            size_t peak = 0;
            if (szgb_server_stats(S, &b, &c, &peak) != SZGB_OK || peak > (64u << 20)) failures++;
            std::this_thread::yield();
        }
    });
    std::vector<std::thread> th;
    for (int t = 0; t < kThreads; t++) {
        th.emplace_back([&, t] {
            std::vector<uint64_t> tickets;
            for (int i = 0; i < kPerThread; i++) {
                const int f = t * kPerThread + i;
                szgb_request r;
                std::memset(&r, 0, sizeof(r));
                r.op = SZGB_OP_COMPRESS;
                r.in = xs[f].data();
                r.in_bytes = xs[f].size() * sizeof(float);
                r.params = field_params();
                r.out = outs[f].data();
                r.out_cap = outs[f].size();
                uint64_t tk = 0;
                if (szgb_submit(S, &r, &tk) != SZGB_OK) failures++;
                tickets.push_back(tk);
                // a request that is refused before it is queued
                r.op = SZGB_OP_DECOMPRESS;
                r.in_bytes = 16;
                if (szgb_submit(S, &r, &tk) == SZGB_OK) failures++;
            }
            for (size_t i = 0; i < tickets.size(); i++) {
                int st = 0, done = 0;
                size_t len = 0;
                if (i % 3 == 0) {
                    if (szgb_wait(S, tickets[i], &st, &len) != SZGB_OK || !expected(st)) failures++;
                    taken++;
                } else if (i % 3 == 1) {
                    do {
                        if (szgb_poll(S, tickets[i], &done, &st, &len) != SZGB_OK) { failures++; break; }
                        if (!done) std::this_thread::yield();
                    } while (!done);
                    if (done) {
                        if (!expected(st)) failures++;
                        taken++;
                    }
                } else {
                    // two takers race for one result: exactly one gets it
                    std::atomic<int> got{0};
                    const uint64_t tk = tickets[i];
                    std::thread other([&] {
                        int s2 = 0;
                        size_t l2 = 0;
                        if (szgb_wait(S, tk, &s2, &l2) == SZGB_OK) {
                            if (!expected(s2)) failures++;
                            got++;
                        }
                    });
                    if (szgb_wait(S, tk, &st, &len) == SZGB_OK) {
                        if (!expected(st)) failures++;
                        got++;
                    }
                    other.join();
                    if (got.load() != 1) failures++;
                    taken++;
                    lost_races++;
                }
            }
        });
    }
    for (auto& x : th) x.join();
    stats_run = false;
    stats.join();
    uint64_t b = 0, c = 0;
    size_t peak = 0;
    szgb_server_stats(S, &b, &c, &peak);
    if ((int)c != total || taken.load() != total) failures++;
    // requests still queued when the server goes away are finished first
    for (int f = 0; f < 8; f++) {
        szgb_request r;
        std::memset(&r, 0, sizeof(r));
        r.op = SZGB_OP_COMPRESS;
        r.in = xs[f].data();
        r.in_bytes = xs[f].size() * sizeof(float);
        r.params = field_params();
        r.out = outs[f].data();
        r.out_cap = outs[f].size();
        uint64_t tk = 0;
        if (szgb_submit(S, &r, &tk) != SZGB_OK) failures++;
    }
    szgb_server_destroy(S);

    // size classes: requests of 128 MiB of I/O or more run alone, never on
    // worker 0; they must complete beside small ones, and a large request
    // still queued at destruction is finished too
    szgb_server* L = nullptr;
    if (szgb_server_create(&L, 0, 2ull << 30, 3, 8) != SZGB_OK) {
        std::fprintf(stderr, "server_create (large) failed\n");
        return 1;
    }
    const size_t big_rows = 4096, big_cols = 4200;  // 68.8 MB in, 64 MiB out: large
    std::vector<float> big(big_rows * big_cols, 0.5f);
    std::vector<unsigned char> big_out(64u << 20);
    szgb_params bp = field_params();
    bp.shape[0] = big_rows;
    bp.shape[1] = big_cols;
    std::vector<uint64_t> lt;
    for (int k = 0; k < 6; k++) {
        szgb_request r;
        std::memset(&r, 0, sizeof(r));
        r.op = SZGB_OP_COMPRESS;
        if (k % 3 == 1) {  // a large request between small ones
            r.in = big.data();
            r.in_bytes = big.size() * sizeof(float);
            r.params = bp;
            r.out = big_out.data();
            r.out_cap = big_out.size();
        } else {
            r.in = xs[k].data();
            r.in_bytes = xs[k].size() * sizeof(float);
            r.params = field_params();
            r.out = outs[k].data();
            r.out_cap = outs[k].size();
        }
        uint64_t tk = 0;
        if (szgb_submit(L, &r, &tk) != SZGB_OK) failures++;
        lt.push_back(tk);
    }
    for (uint64_t tk : lt) {
        int st = 0;
        size_t len = 0;
        if (szgb_wait(L, tk, &st, &len) != SZGB_OK || !expected(st)) failures++;
    }
    uint64_t lb = 0, lc = 0;
    szgb_server_stats(L, &lb, &lc, nullptr);
    if (lc != lt.size()) failures++;
    {
        szgb_request r;
        std::memset(&r, 0, sizeof(r));
        r.op = SZGB_OP_COMPRESS;
        r.in = big.data();
        r.in_bytes = big.size() * sizeof(float);
        r.params = bp;
        r.out = big_out.data();
        r.out_cap = big_out.size();
        uint64_t tk = 0;
        if (szgb_submit(L, &r, &tk) != SZGB_OK) failures++;
    }
    szgb_server_destroy(L);  // returns only after the queued large request ran

    std::printf("requests %d completed %llu batches %llu races %d large-phase %llu failures %d\n", total,
                (unsigned long long)c, (unsigned long long)b, lost_races.load(), (unsigned long long)lc,
                failures.load());
    return failures.load() == 0 ? 0 : 1;
}
