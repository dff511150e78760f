// layout.cuh — where the 2D pipeline keeps its half spectra and filter.
//
// The row pass transforms two image rows as one complex row.  It pairs each
// row x with its mirror N - x (pair p: rows (p, N - p) for 0 < p < N/2, and
// (0, N/2) for p = 0), because the symmetrised filter of frequency row u,
// Hs[u][k] = (H[u][k] + H[-u][-k]) / 2, needs exactly filter rows u and -u:
// the block that owns the pair reads both once, contiguously.
//
// Intermediate layout ("slot order", private to the library): for each
// half-spectrum column k the N row values are contiguous (column-major), so
// the column pass reads and writes whole columns.  Within a column, rows are
// stored in the order the row pass produces them: groups of G pairs (G = the
// row pass's pairs per block, capped at N/2), each group holding its G
// "first" rows, then its G "mirror" rows:
//   slot(x) = (p / G) * 2G + side * G + (p mod G),
// with (p, side) the pair and side of row x.  A row-pass block therefore
// writes 2G consecutive slots of every column (64 bytes of complex64 for
// G = 4) and the inverse row pass reads them back the same way.
#pragma once

#include "gbfft.h"

namespace gbfft {

// Images of a launch given by the caller's device table of per-image
// pointers (a batched call): image z of the launch is ptrs[idx[z]], idx being
// the plan's list of the images of one shape.  ptrs == nullptr: the images
// are contiguous (base + z x image size), as in a one-shape plan.
struct ImgIndirect {
    const gbfft_image_ptrs *ptrs;
    const int *idx;
};

// Row-slab share of an image decomposed over ranks (Sec. 2's division of the
// work among processes, here by rows): a rank owns the pairs p0 .. p0 + P - 1
// (p0 and P multiples of the row pass's pairs per block), i.e. 2P slots of
// every half-spectrum column, which it keeps as [M/2][ld] with ld = 2P
// (column stride ld instead of N).  Global slot s of column k then lives on
// rank s / ld at local slot s mod ld.  The default {0, 0} is the whole image.
struct Slab {
    int p0, ld;
};

// Column-block share of the same decomposition: a rank transforms the Mloc
// half-spectrum columns kbase .. kbase + Mloc - 1, received from the ranks as
// [ranks][Mloc][ld] (chunk q = rank q's slots of these columns).  Local column
// kl, global slot s then sits at ((s / ld) Mloc + kl) ld + s mod ld, ld = 2^ls.
// ls = 0 means one contiguous column per k ([M/2][N], the whole image).
struct ColSlab {
    int ls, mloc, kbase;
};

// pair index and side (0: first row, 1: mirror row) of row x of an N-row image
__host__ __device__ __forceinline__ void pair_of(int x, int N, int &p, int &side) {
    const int h = N >> 1;
    if (x < h) {
        p = x;
        side = 0;
    } else if (x == h) {
        p = 0;
        side = 1;
    } else {
        p = N - x;
        side = 1;
    }
}

// rows of pair p
__host__ __device__ __forceinline__ void rows_of_pair(int p, int N, int &a, int &b) {
    a = p;
    b = p == 0 ? (N >> 1) : N - p;
}

// G is a power of two: log2g = log2(G)
__host__ __device__ __forceinline__ int slot_of(int x, int N, int log2g) {
    int p, side;
    pair_of(x, N, p, side);
    return ((p >> log2g) << (log2g + 1)) + (side << log2g) + (p & ((1 << log2g) - 1));
}

__host__ __device__ __forceinline__ int row_of_slot(int s, int N, int log2g) {
    const int grp = s >> (log2g + 1);
    const int side = (s >> log2g) & 1;
    const int p = (grp << log2g) + (s & ((1 << log2g) - 1));
    int a, b;
    rows_of_pair(p, N, a, b);
    return side ? b : a;
}

}  // namespace gbfft
