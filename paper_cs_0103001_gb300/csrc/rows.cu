// rows.cu — launchers of the row passes of the Sec. 5 pipeline; the kernel
// bodies and the description of the method live in rows_impl.cuh.
#include "internal.h"
#include "rows_impl.cuh"

namespace gbfft {

int rows_pairs_per_block(int cols) {
    switch (ilog2(cols)) {
#define GBFFT_CASE(L) \
    case L: return RowCfg<(1 << L)>::PPC;
        GBFFT_CASE(1) GBFFT_CASE(2) GBFFT_CASE(3) GBFFT_CASE(4) GBFFT_CASE(5) GBFFT_CASE(6) GBFFT_CASE(7)
        GBFFT_CASE(8) GBFFT_CASE(9) GBFFT_CASE(10) GBFFT_CASE(11) GBFFT_CASE(12) GBFFT_CASE(13)
#undef GBFFT_CASE
        default: return 0;
    }
}

// Forward row pass over a chunk of images (blockIdx.y = image).
// filter_mode 1: image 0's blocks also prepare the shared filter from H;
// filter_mode 2: every image prepares its own from H + y * h_stride.
template <int M>
__global__ void __launch_bounds__(RowCfg<M>::THREADS)
    k_rows_fwd(const float *__restrict__ img, float2 *__restrict__ spec, const float *__restrict__ H,
               float *__restrict__ hs, float *__restrict__ beta, int N, int log2g, long long h_stride,
               int filter_mode, float scale, const float2 *__restrict__ tw) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const size_t y = blockIdx.y;
    const bool own = filter_mode == 2;
    rows_fwd_body<M>(img + y * N * M, spec + y * (M / 2) * N, H + (own ? y * h_stride : 0),
                     hs + (own ? y * (M / 2) * N : 0), beta + (own ? y * N : 0), N, log2g,
                     own || (filter_mode == 1 && y == 0), scale, tw, blockIdx.x, smraw);
}

template <int M>
__global__ void __launch_bounds__(RowCfg<M>::THREADS)
    k_rows_inv(const float2 *__restrict__ spec, float *__restrict__ out, int N, int log2g,
               const float2 *__restrict__ tw) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const size_t y = blockIdx.y;
    rows_inv_body<M>(spec + y * (M / 2) * N, out + y * N * M, N, log2g, tw, blockIdx.x, smraw);
}

template <int M> static cudaError_t set_smem(const void *kern) {
    if (RowCfg<M>::SMEM > 48 * 1024)
        return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)RowCfg<M>::SMEM);
    return cudaSuccess;
}

static int log2_pairs_per_block(int rows, int cols) {
    int g = rows_pairs_per_block(cols);
    if (g > rows / 2) g = rows / 2;
    return ilog2(g);
}

template <int M>
static cudaError_t run_rows_fwd(const RowsFwdArgs &a, cudaStream_t s) {
    typedef RowCfg<M> K;
    cudaError_t e = set_smem<M>((const void *)k_rows_fwd<M>);
    if (e != cudaSuccess) return e;
    const int lg = log2_pairs_per_block(a.rows, M);
    dim3 grid((a.rows / 2) >> lg, a.nimg);
    k_rows_fwd<M><<<grid, K::THREADS, K::SMEM, s>>>(a.img, static_cast<float2 *>(a.spec), a.H, a.hs, a.beta, a.rows,
                                                    lg, a.h_stride, a.filter_mode, a.scale,
                                                    static_cast<const float2 *>(a.tw));
    return cudaGetLastError();
}

template <int M>
static cudaError_t run_rows_inv(const void *spec, float *out, int rows, int nimg, const void *tw, cudaStream_t s) {
    typedef RowCfg<M> K;
    cudaError_t e = set_smem<M>((const void *)k_rows_inv<M>);
    if (e != cudaSuccess) return e;
    const int lg = log2_pairs_per_block(rows, M);
    dim3 grid((rows / 2) >> lg, nimg);
    k_rows_inv<M><<<grid, K::THREADS, K::SMEM, s>>>(static_cast<const float2 *>(spec), out, rows, lg,
                                                    static_cast<const float2 *>(tw));
    return cudaGetLastError();
}

cudaError_t launch_rows_fwd(const RowsFwdArgs &a, cudaStream_t s) {
    switch (ilog2(a.cols)) {
#define GBFFT_CASE(L) \
    case L: return run_rows_fwd<(1 << L)>(a, s);
        GBFFT_CASE(1) GBFFT_CASE(2) GBFFT_CASE(3) GBFFT_CASE(4) GBFFT_CASE(5) GBFFT_CASE(6) GBFFT_CASE(7)
        GBFFT_CASE(8) GBFFT_CASE(9) GBFFT_CASE(10) GBFFT_CASE(11) GBFFT_CASE(12) GBFFT_CASE(13)
#undef GBFFT_CASE
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_rows_inv(const void *spec, float *out, int rows, int cols, int nimg, const void *tw_cols,
                            cudaStream_t s) {
    switch (ilog2(cols)) {
#define GBFFT_CASE(L) \
    case L: return run_rows_inv<(1 << L)>(spec, out, rows, nimg, tw_cols, s);
        GBFFT_CASE(1) GBFFT_CASE(2) GBFFT_CASE(3) GBFFT_CASE(4) GBFFT_CASE(5) GBFFT_CASE(6) GBFFT_CASE(7)
        GBFFT_CASE(8) GBFFT_CASE(9) GBFFT_CASE(10) GBFFT_CASE(11) GBFFT_CASE(12) GBFFT_CASE(13)
#undef GBFFT_CASE
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace gbfft
