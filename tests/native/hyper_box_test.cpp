// hyper_box_test.cpp -- the hyperplane enumerations used by the 3D kernels
// for n >= 3 layers and by the 4D kernels: over every h, the valid entries of
// every box visit each point of the field exactly once, on the hyperplane of
// its coordinate sum; boxes stay inside the field and no hyperplane in range
// is empty.  Plain C++, no GPU.
#include <cstdio>
#include <vector>

#include "../../paper_1706_03791_gb300/csrc/hyper_box.h"

static int check(int64_t P, int64_t M, int64_t N) {
    std::vector<int> seen((size_t)(P * M * N), 0);
    const int64_t H = (P - 1) + (M - 1) + (N - 1);
    for (int64_t h = 0; h <= H; h++) {
        const HyperBox b = hyper_box(h, P, M, N);
        if (b.ni == 0 || b.nj == 0 || b.ni * b.nj > (uint64_t)(P * M)) return 1;
        uint64_t found = 0;
        for (uint64_t t = 0; t < b.ni * b.nj; t++) {
            const int64_t i = b.ilo + (int64_t)(t / b.nj), j = b.jlo + (int64_t)(t % b.nj), l = h - i - j;
            if (i < 0 || i >= P || j < 0 || j >= M) return 2;  // the box stays inside the field
            if (l < 0 || l >= N) continue;
            seen[(size_t)((i * M + j) * N + l)]++;
            found++;
        }
        if (found == 0) return 3;  // no hyperplane in range is empty
    }
    for (int v : seen)
        if (v != 1) return 4;
    return 0;
}

static int check4(int64_t D, int64_t P, int64_t M, int64_t N) {
    std::vector<int> seen((size_t)(D * P * M * N), 0);
    const int64_t H = (D - 1) + (P - 1) + (M - 1) + (N - 1);
    for (int64_t h = 0; h <= H; h++) {
        const HyperBox4 b = hyper_box4(h, D, P, M, N);
        const uint64_t n = b.na * b.ni * b.nj;
        if (n == 0 || n > (uint64_t)(D * P * M)) return 1;
        uint64_t found = 0;
        for (uint64_t t = 0; t < n; t++) {
            const int64_t a = b.alo + (int64_t)(t / (b.ni * b.nj)), i = b.ilo + (int64_t)((t / b.nj) % b.ni),
                          j = b.jlo + (int64_t)(t % b.nj), l = h - a - i - j;
            if (a < 0 || a >= D || i < 0 || i >= P || j < 0 || j >= M) return 2;
            if (l < 0 || l >= N) continue;
            seen[(size_t)(((a * P + i) * M + j) * N + l)]++;
            found++;
        }
        if (found == 0) return 3;
    }
    for (int v : seen)
        if (v != 1) return 4;
    return 0;
}

int main() {
    int bad = 0, cases = 0;
    const int64_t ext[] = {1, 2, 3, 4, 5, 7, 13, 32, 33};
    for (int64_t P : ext)
        for (int64_t M : ext)
            for (int64_t N : ext) {
                const int r = check(P, M, N);
                cases++;
                if (r) {
                    std::printf("shape %lld x %lld x %lld: failure %d\n", (long long)P, (long long)M, (long long)N, r);
                    bad++;
                }
            }
    const int64_t ext4[] = {1, 2, 3, 5, 8, 9};
    for (int64_t D : ext4)
        for (int64_t P : ext4)
            for (int64_t M : ext4)
                for (int64_t N : ext4) {
                    const int r = check4(D, P, M, N);
                    cases++;
                    if (r) {
                        std::printf("shape %lld x %lld x %lld x %lld: failure %d\n", (long long)D, (long long)P,
                                    (long long)M, (long long)N, r);
                        bad++;
                    }
                }
    std::printf("shapes %d failures %d\n", cases, bad);
    return bad ? 1 : 0;
}
