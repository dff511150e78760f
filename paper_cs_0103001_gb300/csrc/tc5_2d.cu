// tc5_2d.cu — the Sec. 5 pipeline with its radix-16 passes on the
// fifth-generation tensor cores (tcgen05.mma, accumulators in tensor memory).
//
// Same three stages, block bodies and data layout as rows.cu / cols.cu, with
// the transform policy Tc5Fft<FMT> (fft_tc5.cuh).  Each kernel sets the
// policy up at its start (the DFT matrices in shared memory, an mbarrier, 32
// tensor-memory columns per 128 threads) and releases the tensor memory at
// its end; its shared memory follows the body's own.  Sides
// 512..4096, as the warp-level tensor-core variant (tc2d.cu).
#include "cols_impl.cuh"
#include "fft_tc5.cuh"
#include "internal.h"
#include "rows_impl.cuh"

namespace gbfft {

cudaError_t check_take_tc5(unsigned out[2]) { return check_word_take(out); }

template <int THREADS, int FMT> struct Tc5Smem {
    static constexpr size_t align128(size_t x) { return (x + 127) / 128 * 128; }
    // the body's shared memory, then the policy's own
    static constexpr size_t area(size_t body) { return align128(body); }
    static constexpr size_t total(size_t body) { return area(body) + Tc5Layout<FMT>::bytes(THREADS); }
};

template <int M, int FMT>
__global__ void __launch_bounds__(RowCfg<M>::THREADS, 1)
    k_rows_fwd_tc5(const float *__restrict__ img, float2 *__restrict__ spec, int N, int log2g,
                   const float2 *__restrict__ tw, int *status) {
    extern __shared__ __align__(128) unsigned char smraw[];
    typedef Tc5Smem<RowCfg<M>::THREADS, FMT> S;
    const size_t y = blockIdx.y;
    Tc5Fft<FMT> f;
    tc5_setup<FMT>(f.st, smraw + S::area(RowCfg<M>::SMEM), status);
    rows_fwd_body<M, Tc5Fft<FMT>>(img + y * N * M, spec + y * (M / 2) * N, N, log2g, tw, blockIdx.x, smraw, f);
    tc5_teardown(f.st);
}

template <int M, int FMT>
__global__ void __launch_bounds__(RowCfg<M>::THREADS, 1)
    k_rows_inv_tc5(const float2 *__restrict__ spec, float *__restrict__ out, int N, int log2g,
                   const float2 *__restrict__ tw, int *status) {
    extern __shared__ __align__(128) unsigned char smraw[];
    typedef Tc5Smem<RowCfg<M>::THREADS, FMT> S;
    const size_t y = blockIdx.y;
    Tc5Fft<FMT> f;
    tc5_setup<FMT>(f.st, smraw + S::area(RowCfg<M>::SMEM), status);
    rows_inv_body<M, Tc5Fft<FMT>>(spec + y * (M / 2) * N, out + y * N * M, N, log2g, tw, blockIdx.x, smraw, f);
    tc5_teardown(f.st);
}

template <int N, int FMT>
__global__ void __launch_bounds__(ColCfg<N>::THREADS, 2)
    k_cols_tc5(float2 *spec, const float *__restrict__ hs, const float *__restrict__ beta, long long hs_img,
               long long beta_img, int M, int log2g, const float2 *__restrict__ tw, int *status) {
    extern __shared__ __align__(128) unsigned char smraw[];
    typedef Tc5Smem<ColCfg<N>::THREADS, FMT> S;
    const size_t y = blockIdx.y;
    Tc5Fft<FMT> f;
    tc5_setup<FMT>(f.st, smraw + S::area(ColCfg<N>::SMEM), status);
    cols_body<N, Tc5Fft<FMT>>(spec + y * (M / 2) * N, PreparedFilter{hs + y * hs_img, beta + y * beta_img, N}, M,
                              log2g, tw, blockIdx.x, smraw, f);
    tc5_teardown(f.st);
}

template <int M, int FMT>
static cudaError_t rows_tc5(bool fwd, const void *src, void *dst, int rows, int nimg, const void *tw, int *status,
                            cudaStream_t s) {
    typedef RowCfg<M> K;
    static_assert(K::THREADS % 128 == 0, "whole groups of 128 butterflies");
    const size_t smem = Tc5Smem<K::THREADS, FMT>::total(K::SMEM);
    int g = K::PPC > rows / 2 ? rows / 2 : K::PPC;
    const int lg = ilog2(g);
    dim3 grid((rows / 2) >> lg, nimg);
    cudaError_t e;
    if (fwd) {
        e = set_smem_attrs((const void *)k_rows_fwd_tc5<M, FMT>, smem, 1);
        if (e != cudaSuccess) return e;
        k_rows_fwd_tc5<M, FMT><<<grid, K::THREADS, smem, s>>>(static_cast<const float *>(src),
                                                               static_cast<float2 *>(dst), rows, lg,
                                                               static_cast<const float2 *>(tw), status);
    } else {
        e = set_smem_attrs((const void *)k_rows_inv_tc5<M, FMT>, smem, 1);
        if (e != cudaSuccess) return e;
        k_rows_inv_tc5<M, FMT><<<grid, K::THREADS, smem, s>>>(static_cast<const float2 *>(src),
                                                               static_cast<float *>(dst), rows, lg,
                                                               static_cast<const float2 *>(tw), status);
    }
    return cudaGetLastError();
}

template <int N, int FMT>
static cudaError_t cols_tc5(void *spec, const float *hs, const float *beta, long long hs_img, long long beta_img,
                            int cols, int nimg, const void *tw, int *status, cudaStream_t s) {
    typedef ColCfg<N> K;
    static_assert(K::THREADS % 128 == 0, "whole groups of 128 butterflies");
    const size_t smem = Tc5Smem<K::THREADS, FMT>::total(K::SMEM);
    cudaError_t e = set_smem_attrs((const void *)k_cols_tc5<N, FMT>, smem, 2);
    if (e != cudaSuccess) return e;
    int g = rows_pairs_per_block(cols);
    if (g > N / 2) g = N / 2;
    dim3 grid((cols / 2 + K::W - 1) / K::W, nimg);
    k_cols_tc5<N, FMT><<<grid, K::THREADS, smem, s>>>(static_cast<float2 *>(spec), hs, beta, hs_img, beta_img, cols,
                                                      ilog2(g), static_cast<const float2 *>(tw), status);
    return cudaGetLastError();
}

#define GBFFT_TC5_SIZES(X) X(9) X(10) X(11) X(12)

cudaError_t launch_rows_tc5(bool fwd, const void *src, void *dst, int rows, int cols, int nimg, const void *tw,
                            int fmt, int *status, cudaStream_t s) {
    switch (ilog2(cols) * 4 + fmt) {
#define GBFFT_C(L)                                                                                              \
    case L * 4 + FMT_BF16X2: return rows_tc5<(1 << L), FMT_BF16X2>(fwd, src, dst, rows, nimg, tw, status, s); \
    case L * 4 + FMT_BF16X3: return rows_tc5<(1 << L), FMT_BF16X3>(fwd, src, dst, rows, nimg, tw, status, s); \
    case L * 4 + FMT_TF32X2: return rows_tc5<(1 << L), FMT_TF32X2>(fwd, src, dst, rows, nimg, tw, status, s);
        GBFFT_TC5_SIZES(GBFFT_C)
#undef GBFFT_C
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_cols_tc5(void *spec, const float *hs, const float *beta, long long hs_img, long long beta_img,
                            int rows, int cols, int nimg, const void *tw_rows, int fmt, int *status, cudaStream_t s) {
    switch (ilog2(rows) * 4 + fmt) {
#define GBFFT_C(L)                                                                                             \
    case L * 4 + FMT_BF16X2:                                                                                   \
        return cols_tc5<(1 << L), FMT_BF16X2>(spec, hs, beta, hs_img, beta_img, cols, nimg, tw_rows, status, s); \
    case L * 4 + FMT_BF16X3:                                                                                   \
        return cols_tc5<(1 << L), FMT_BF16X3>(spec, hs, beta, hs_img, beta_img, cols, nimg, tw_rows, status, s); \
    case L * 4 + FMT_TF32X2:                                                                                   \
        return cols_tc5<(1 << L), FMT_TF32X2>(spec, hs, beta, hs_img, beta_img, cols, nimg, tw_rows, status, s);
        GBFFT_TC5_SIZES(GBFFT_C)
#undef GBFFT_C
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace gbfft
