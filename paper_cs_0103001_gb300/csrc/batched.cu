// batched.cu — the Sec. 5 pipeline over many images of uneven power-of-two
// sizes, each with its own filter, in four persistent kernel launches.
//
// A batched plan fixes the image shapes.  At bind time it uploads an image
// table (shape, workspace offsets) and one work list per stage: the thread
// blocks the regular kernels would launch for every image, (image, block)
// pairs, sorted by decreasing cost.  Each stage is one persistent launch of a
// few blocks per SM; block i takes items i, i + grid, i + 2 grid, ... (a
// fixed assignment: no counters to reset, the same work split every call),
// dispatching on the item's size to the same block bodies as the regular
// kernels (rows_impl.cuh, cols_impl.cuh).  The four launches can be captured
// once in a CUDA graph and replayed.  Blocks per SM are a tunable of the plan.
#include "batched.h"
#include "cols_impl.cuh"
#include "internal.h"
#include "rows_impl.cuh"

namespace gbfft {

// The per-size bodies are kept out of line: each gets its own register
// allocation instead of the union of all sizes inlined into one loop.
template <int L>
__device__ __noinline__ void fwd_case(const BatchImage &im, const gbfft_image_ptrs &pp, char *ws, int bx,
                                         unsigned char *sm) {
    rows_fwd_body<(1 << L)>(pp.img, reinterpret_cast<float2 *>(ws + im.spec_off), im.rows, im.log2g,
                            reinterpret_cast<const float2 *>(ws + im.twc_off), bx, sm);
}

template <int L>
__device__ __noinline__ void inv_case(const BatchImage &im, const gbfft_image_ptrs &pp, char *ws, int bx,
                                         unsigned char *sm) {
    rows_inv_body<(1 << L)>(reinterpret_cast<const float2 *>(ws + im.spec_off), pp.out, im.rows, im.log2g,
                            reinterpret_cast<const float2 *>(ws + im.twc_off), bx, sm);
}

template <int L>
__device__ __noinline__ void cols_case(const BatchImage &im, char *ws, int bx, unsigned char *sm) {
    cols_body<(1 << L)>(reinterpret_cast<float2 *>(ws + im.spec_off),
                        PreparedFilter{reinterpret_cast<const float *>(ws + im.hs_off),
                                       reinterpret_cast<const float *>(ws + im.beta_off), im.rows},
                        im.cols, im.log2g, reinterpret_cast<const float2 *>(ws + im.twr_off), bx, sm);
}

#define GBFFT_BATCH_SIZES(X) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11) X(12)

// columns per block of the column body for `rows`-row columns (ColCfg<N>::W)
__device__ __forceinline__ int batch_col_w(int rows) { return rows >= 4096 ? 1 : 4096 / rows; }

__global__ void __launch_bounds__(kBatchRowThreads, 2)
    k_batched_rows_fwd(const BatchImage *__restrict__ imgs, const BatchItem *__restrict__ items, int nitems,
                       const gbfft_image_ptrs *__restrict__ ptrs, char *ws) {
    extern __shared__ __align__(16) unsigned char smraw[];
    for (int i = blockIdx.x; i < nitems; i += gridDim.x) {
        const BatchItem it = items[i];
        const BatchImage im = imgs[it.img];
        const gbfft_image_ptrs pp = ptrs[it.img];
        __syncthreads();  // shared memory of the previous item is free
        if (!chk(it.bx >= 0 && it.bx < ((im.rows >> 1) >> im.log2g), CK_BATCH_ITEM)) continue;  // uniform
        switch (im.log2c) {
#define GBFFT_C(L) \
    case L: fwd_case<L>(im, pp, ws, it.bx, smraw); break;
            GBFFT_BATCH_SIZES(GBFFT_C)
#undef GBFFT_C
            default: break;
        }
    }
}

// Filter preparation tiles (rows_impl.cuh): kPrepRows x min(kPrepCols, cols/2)
// (16-row tiles for 16-row images); tile bx = column tile * row tiles + row tile.
__global__ void __launch_bounds__(kBatchPrepThreads)
    k_batched_prep(const BatchImage *__restrict__ imgs, const BatchItem *__restrict__ items, int nitems,
                   const gbfft_image_ptrs *__restrict__ ptrs, char *ws) {
    extern __shared__ __align__(16) unsigned char smraw[];
    float *tile = reinterpret_cast<float *>(smraw);
    for (int i = blockIdx.x; i < nitems; i += gridDim.x) {
        const BatchItem it = items[i];
        const BatchImage im = imgs[it.img];
        const gbfft_image_ptrs pp = ptrs[it.img];
        __syncthreads();  // the previous tile's shared memory is free
        const int kk = im.cols / 2 < kPrepCols ? im.cols / 2 : kPrepCols;
        const int log2k = __ffs(kk) - 1;
        float *hs = reinterpret_cast<float *>(ws + im.hs_off);
        float *beta = reinterpret_cast<float *>(ws + im.beta_off);
        if (im.rows >= kPrepRows) {
            const int nr = im.rows / kPrepRows;
            filter_prep_tile<kPrepRows, true>(pp.H, hs, beta, im.rows, im.cols, log2k, im.scale,
                                              (it.bx % nr) * kPrepRows, (it.bx / nr) * kk, tile);
        } else {  // 16-row images (the smallest batched side)
            filter_prep_tile<16, true>(pp.H, hs, beta, im.rows, im.cols, log2k, im.scale, 0, it.bx * kk, tile);
        }
    }
}

__global__ void __launch_bounds__(kBatchColThreads, 2)
    k_batched_cols(const BatchImage *__restrict__ imgs, const BatchItem *__restrict__ items, int nitems, char *ws) {
    extern __shared__ __align__(16) unsigned char smraw[];
    for (int i = blockIdx.x; i < nitems; i += gridDim.x) {
        const BatchItem it = items[i];
        const BatchImage im = imgs[it.img];
        __syncthreads();
        if (!chk(it.bx >= 0 && it.bx * batch_col_w(im.rows) < (im.cols >> 1), CK_BATCH_ITEM)) continue;  // uniform
        switch (im.log2r) {
#define GBFFT_C(L) \
    case L: cols_case<L>(im, ws, it.bx, smraw); break;
            GBFFT_BATCH_SIZES(GBFFT_C)
#undef GBFFT_C
            default: break;
        }
    }
}

__global__ void __launch_bounds__(kBatchRowThreads, 2)
    k_batched_rows_inv(const BatchImage *__restrict__ imgs, const BatchItem *__restrict__ items, int nitems,
                       const gbfft_image_ptrs *__restrict__ ptrs, char *ws) {
    extern __shared__ __align__(16) unsigned char smraw[];
    for (int i = blockIdx.x; i < nitems; i += gridDim.x) {
        const BatchItem it = items[i];
        const BatchImage im = imgs[it.img];
        const gbfft_image_ptrs pp = ptrs[it.img];
        __syncthreads();
        if (!chk(it.bx >= 0 && it.bx < ((im.rows >> 1) >> im.log2g), CK_BATCH_ITEM)) continue;  // uniform
        switch (im.log2c) {
#define GBFFT_C(L) \
    case L: inv_case<L>(im, pp, ws, it.bx, smraw); break;
            GBFFT_BATCH_SIZES(GBFFT_C)
#undef GBFFT_C
            default: break;
        }
    }
}

// ---- host side: shapes of the block bodies -------------------------------

cudaError_t check_take_batched(unsigned out[2]) { return check_word_take(out); }

int batch_row_pairs(int cols) {
    switch (ilog2(cols)) {
#define GBFFT_C(L) \
    case L: return RowCfg<(1 << L)>::PPC;
        GBFFT_BATCH_SIZES(GBFFT_C)
#undef GBFFT_C
        default: return 0;
    }
}

size_t batch_row_smem(int cols, bool fwd) {
    switch (ilog2(cols)) {
#define GBFFT_C(L) \
    case L: return fwd ? RowCfg<(1 << L)>::SMEM_FWD : RowCfg<(1 << L)>::SMEM;
        GBFFT_BATCH_SIZES(GBFFT_C)
#undef GBFFT_C
        default: return 0;
    }
}

int batch_col_width(int rows) {
    switch (ilog2(rows)) {
#define GBFFT_C(L) \
    case L: return ColCfg<(1 << L)>::W;
        GBFFT_BATCH_SIZES(GBFFT_C)
#undef GBFFT_C
        default: return 0;
    }
}

size_t batch_col_smem(int rows) {
    switch (ilog2(rows)) {
#define GBFFT_C(L) \
    case L: return ColCfg<(1 << L)>::SMEM;
        GBFFT_BATCH_SIZES(GBFFT_C)
#undef GBFFT_C
        default: return 0;
    }
}

int batch_prep_tiles(int rows, int cols) {
    const int kk = cols / 2 < kPrepCols ? cols / 2 : kPrepCols;
    const int rr = rows < kPrepRows ? rows : kPrepRows;
    return (rows / rr) * ((cols / 2) / kk);
}

size_t batch_prep_smem(int rows, int cols) {
    const int kk = cols / 2 < kPrepCols ? cols / 2 : kPrepCols;
    const int rr = rows < kPrepRows ? rows : kPrepRows;
    return (size_t)kk * (rr + 1) * sizeof(float);
}

static_assert(kPrepRows == 32 && (1 << kBatchMinLog2) == 16, "prep tiles: 32 rows, or 16 for 16-row images");
static_assert(RowCfg<16>::THREADS == kBatchRowThreads && RowCfg<4096>::THREADS == kBatchRowThreads,
              "row bodies of every batched size use the same block");
static_assert(ColCfg<16>::THREADS == kBatchColThreads && ColCfg<4096>::THREADS == kBatchColThreads,
              "column bodies of every batched size use the same block");

cudaError_t batch_max_blocks_per_sm(int stage, size_t smem, int *blocks) {
    const void *k = stage == 0   ? (const void *)k_batched_rows_fwd
                    : stage == 1 ? (const void *)k_batched_cols
                    : stage == 2 ? (const void *)k_batched_rows_inv
                                 : (const void *)k_batched_prep;
    const int threads = stage == 1 ? kBatchColThreads : stage == 3 ? kBatchPrepThreads : kBatchRowThreads;
    cudaError_t e = set_smem_attrs(k, smem, 2);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, k, threads, smem);
}

cudaError_t launch_batched_stage(int stage, int grid, size_t smem, const BatchImage *imgs, const BatchItem *items,
                                 int nitems, const gbfft_image_ptrs *ptrs, char *ws, cudaStream_t s) {
    if (nitems <= 0) return cudaSuccess;
    if (grid > nitems) grid = nitems;
    switch (stage) {
        case 0: k_batched_rows_fwd<<<grid, kBatchRowThreads, smem, s>>>(imgs, items, nitems, ptrs, ws); break;
        case 1: k_batched_cols<<<grid, kBatchColThreads, smem, s>>>(imgs, items, nitems, ws); break;
        case 3: k_batched_prep<<<grid, kBatchPrepThreads, smem, s>>>(imgs, items, nitems, ptrs, ws); break;
        case 2: k_batched_rows_inv<<<grid, kBatchRowThreads, smem, s>>>(imgs, items, nitems, ptrs, ws); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace gbfft
