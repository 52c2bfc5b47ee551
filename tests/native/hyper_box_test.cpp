// hyper_box_test.cpp -- the hyperplane enumeration used by the 3D kernels for
// n >= 3 layers: over h = 0 .. (P-1)+(M-1)+(N-1), the valid entries of every
// box visit each point of the field exactly once, on the hyperplane of its
// coordinate sum, and every n-layer neighbour of a point lies on an earlier
// hyperplane.  Plain C++, no GPU.
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
    std::printf("shapes %d failures %d\n", cases, bad);
    return bad ? 1 : 0;
}
