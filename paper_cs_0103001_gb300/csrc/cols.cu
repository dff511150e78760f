// cols.cu — launcher of the fused column pass of the Sec. 5 pipeline; the
// kernel body and the description of the method live in cols_impl.cuh.
#include "cols_impl.cuh"
#include "internal.h"

namespace gbfft {

template <int N>
__global__ void __launch_bounds__(ColCfg<N>::THREADS, 2)
    k_cols_filter(float2 *spec, const float *__restrict__ hs, const float *__restrict__ beta, long long hs_img,
                  long long beta_img, int M, int log2g, const float2 *__restrict__ tw) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const size_t y = blockIdx.y;
    cols_body<N>(spec + y * (M / 2) * N, hs + y * hs_img, beta + y * beta_img, M, log2g, tw, blockIdx.x, smraw);
}

template <int N>
static cudaError_t run_cols(void *spec, const float *hs, const float *beta, long long hs_img, long long beta_img,
                            int cols, int nimg, int log2g, const void *tw, cudaStream_t s) {
    typedef ColCfg<N> K;
    auto kern = k_cols_filter<N>;
    cudaError_t e = set_smem_attrs((const void *)kern, K::SMEM, 2);
    if (e != cudaSuccess) return e;
    const int half = cols / 2;
    dim3 grid((half + K::W - 1) / K::W, nimg);
    kern<<<grid, K::THREADS, K::SMEM, s>>>(static_cast<float2 *>(spec), hs, beta, hs_img, beta_img, cols, log2g,
                                           static_cast<const float2 *>(tw));
    return cudaGetLastError();
}

cudaError_t launch_cols_filter(void *spec, const float *hs, const float *beta, long long hs_img, long long beta_img,
                               int rows, int cols, int nimg, const void *tw_rows, cudaStream_t s) {
    int g = rows_pairs_per_block(cols);
    if (g > rows / 2) g = rows / 2;
    const int log2g = ilog2(g);
    switch (ilog2(rows)) {
#define GBFFT_CASE(L) \
    case L: return run_cols<(1 << L)>(spec, hs, beta, hs_img, beta_img, cols, nimg, log2g, tw_rows, s);
        GBFFT_CASE(1) GBFFT_CASE(2) GBFFT_CASE(3) GBFFT_CASE(4) GBFFT_CASE(5) GBFFT_CASE(6) GBFFT_CASE(7)
        GBFFT_CASE(8) GBFFT_CASE(9) GBFFT_CASE(10) GBFFT_CASE(11) GBFFT_CASE(12) GBFFT_CASE(13)
#undef GBFFT_CASE
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace gbfft
