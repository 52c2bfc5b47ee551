// hyper_box.h -- the points of one hyperplane i + j + l = h of a P x M x N
// field, as a box of (i, j) pairs with l = h - i - j.  Shared by the
// hyperplane kernels and their host-side enumeration test (plain C++).
//
// Every prediction term reaches back by k != 0 with k >= 0 componentwise, so
// all neighbours of a point lie on smaller hyperplanes: processing the
// hyperplanes in increasing h, each as one parallel step, gives the values of
// the raster-order loop exactly (Sec. III: only preceding values are used).
#ifndef SZGB_HYPER_BOX_H
#define SZGB_HYPER_BOX_H
#include <stdint.h>

#if defined(__CUDACC__)
#define SZGB_HD __host__ __device__ __forceinline__
#else
#define SZGB_HD inline
#endif

struct HyperBox {
    int64_t ilo, jlo;   // first i and j of the box
    uint64_t ni, nj;    // box extents; (i, j) = (ilo + t / nj, jlo + t % nj)
};

// The box of hyperplane h, 0 <= h <= (P - 1) + (M - 1) + (N - 1); P, M, N >= 1.
// Every point of the hyperplane is in the box exactly once; a box entry is a
// point iff 0 <= h - i - j < N.
SZGB_HD HyperBox hyper_box(int64_t h, int64_t P, int64_t M, int64_t N) {
    HyperBox b;
    const int64_t ilo = h - (M - 1) - (N - 1) > 0 ? h - (M - 1) - (N - 1) : 0;
    const int64_t ihi = h < P - 1 ? h : P - 1;
    const int64_t jlo = h - ihi - (N - 1) > 0 ? h - ihi - (N - 1) : 0;
    const int64_t jhi = h - ilo < M - 1 ? h - ilo : M - 1;
    b.ilo = ilo;
    b.jlo = jlo;
    b.ni = ihi >= ilo ? (uint64_t)(ihi - ilo + 1) : 0;
    b.nj = jhi >= jlo ? (uint64_t)(jhi - jlo + 1) : 0;
    return b;
}

// The box of hyperplane h = i0 + i + j + l of a D x P x M x N field, as
// (i0, i, j) triples with l = h - i0 - i - j; an entry is a point iff
// 0 <= l < N.  0 <= h <= (D-1) + (P-1) + (M-1) + (N-1); all extents >= 1.
struct HyperBox4 {
    int64_t alo, ilo, jlo;  // first i0, i, j of the box
    uint64_t na, ni, nj;    // extents; t -> (alo + t / (ni nj), ilo + (t / nj) % ni, jlo + t % nj)
};

SZGB_HD HyperBox4 hyper_box4(int64_t h, int64_t D, int64_t P, int64_t M, int64_t N) {
    HyperBox4 b;
    const int64_t rest3 = (P - 1) + (M - 1) + (N - 1), rest2 = (M - 1) + (N - 1);
    const int64_t alo = h - rest3 > 0 ? h - rest3 : 0;
    const int64_t ahi = h < D - 1 ? h : D - 1;
    const int64_t ilo = h - ahi - rest2 > 0 ? h - ahi - rest2 : 0;
    const int64_t ihi = h - alo < P - 1 ? h - alo : P - 1;
    const int64_t jlo = h - ahi - ihi - (N - 1) > 0 ? h - ahi - ihi - (N - 1) : 0;
    const int64_t jhi = h - alo - ilo < M - 1 ? h - alo - ilo : M - 1;
    b.alo = alo;
    b.ilo = ilo;
    b.jlo = jlo;
    b.na = ahi >= alo ? (uint64_t)(ahi - alo + 1) : 0;
    b.ni = ihi >= ilo ? (uint64_t)(ihi - ilo + 1) : 0;
    b.nj = jhi >= jlo ? (uint64_t)(jhi - jlo + 1) : 0;
    return b;
}

#endif
