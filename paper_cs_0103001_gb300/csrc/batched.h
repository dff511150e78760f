// batched.h — tables shared by the batched (uneven sizes) pipeline kernels
// and the plan code.  Not installed.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include "gbfft.h"

namespace gbfft {

constexpr int kBatchRowThreads = 512;  // block of every row body for sides 16..4096
constexpr int kBatchColThreads = 256;  // block of every column body for sides 16..4096
constexpr int kBatchPrepThreads = 256; // block of the filter-preparation tiles
// stages: 0 = forward row pass, 1 = column pass, 2 = inverse row pass,
// 3 = filter preparation; they run in the order of kBatchOrder
constexpr int kBatchStages = 4;
constexpr int kBatchOrder[kBatchStages] = {3, 0, 1, 2};
constexpr int kBatchMinLog2 = 4, kBatchMaxLog2 = 12;

// One image of a batched plan; offsets are bytes into the workspace.
struct BatchImage {
    int rows, cols;     // N, M
    int log2r, log2c;
    int log2g;          // log2 of the row-pass pairs per block for this shape
    float scale;        // 1 / (N M)
    long long spec_off; // half spectra [M/2][N] complex64, slot order
    long long hs_off;   // prepared filter [M/2][N] float32
    long long beta_off; // packed-column coefficients [N] float32
    long long twc_off;  // twiddles of length M (row transforms)
    long long twr_off;  // twiddles of length N (column transforms)
};

// One block's worth of work: block bx of image img's regular launch (for the
// filter preparation: tile bx, row tiles first).
struct BatchItem {
    int img;
    int bx;
};

int batch_row_pairs(int cols);
size_t batch_row_smem(int cols, bool fwd);
int batch_col_width(int rows);
size_t batch_col_smem(int rows);
// filter-preparation tiles of an image: count, and shared memory of one
int batch_prep_tiles(int rows, int cols);
size_t batch_prep_smem(int rows, int cols);
cudaError_t batch_max_blocks_per_sm(int stage, size_t smem, int *blocks);
cudaError_t launch_batched_stage(int stage, int grid, size_t smem, const BatchImage *imgs, const BatchItem *items,
                                 int nitems, const gbfft_image_ptrs *ptrs, char *ws, cudaStream_t s);

}  // namespace gbfft
