// tc2d.cu — the Sec. 5 pipeline with its radix-16 passes on the tensor cores.
//
// Same three stages and data layout as rows.cu / cols.cu (the same block
// bodies), with the transform policy TcFft<TERMS> (fft_tc.cuh): every radix-16
// Stockham pass becomes BF16-split DFT-matrix products on mma.sync, FP32
// accumulation.  TERMS = 2 keeps three products per term pair (about 16
// significant bits per pass), TERMS = 3 six (about 24).  Sides 512..4096: the
// tensor-core pass needs whole warps of butterflies (N/16 >= 32).
#include "cols_impl.cuh"
#include "fft_tc.cuh"
#include "internal.h"
#include "rows_impl.cuh"

namespace gbfft {

cudaError_t check_take_tc2d(unsigned out[2]) { return check_word_take(out); }

template <int THREADS, int TERMS>
__device__ __forceinline__ TcFft<TERMS> make_tc(unsigned char *smraw, size_t body_smem) {
    TcFft<TERMS> f;
    uint32_t *stage = reinterpret_cast<uint32_t *>(smraw + body_smem) +
                      (threadIdx.x >> 5) * TcState<TERMS>::WORDS_PER_WARP;
    tc_init<TERMS>(f.st, stage, threadIdx.x & 31);
    return f;
}

template <int THREADS, int TERMS> constexpr size_t tc_stage_bytes() {
    return (size_t)(THREADS / 32) * TcState<TERMS>::WORDS_PER_WARP * 4;
}

template <int M, int TERMS>
__global__ void __launch_bounds__(RowCfg<M>::THREADS, 1)
    k_rows_fwd_tc(const float *__restrict__ img, float2 *__restrict__ spec, int N, int log2g,
                  const float2 *__restrict__ tw) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const size_t y = blockIdx.y;
    TcFft<TERMS> f = make_tc<RowCfg<M>::THREADS, TERMS>(smraw, RowCfg<M>::SMEM);
    rows_fwd_body<M, TcFft<TERMS>>(img + y * N * M, spec + y * (M / 2) * N, N, log2g, tw, blockIdx.x, smraw, f);
}

template <int M, int TERMS>
__global__ void __launch_bounds__(RowCfg<M>::THREADS, 1)
    k_rows_inv_tc(const float2 *__restrict__ spec, float *__restrict__ out, int N, int log2g,
                  const float2 *__restrict__ tw) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const size_t y = blockIdx.y;
    TcFft<TERMS> f = make_tc<RowCfg<M>::THREADS, TERMS>(smraw, RowCfg<M>::SMEM);
    rows_inv_body<M, TcFft<TERMS>>(spec + y * (M / 2) * N, out + y * N * M, N, log2g, tw, blockIdx.x, smraw, f);
}

template <int N, int TERMS>
__global__ void __launch_bounds__(ColCfg<N>::THREADS, 2)
    k_cols_tc(float2 *spec, const float *__restrict__ hs, const float *__restrict__ beta, long long hs_img,
              long long beta_img, int M, int log2g, const float2 *__restrict__ tw) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const size_t y = blockIdx.y;
    TcFft<TERMS> f = make_tc<ColCfg<N>::THREADS, TERMS>(smraw, ColCfg<N>::SMEM);
    cols_body<N, TcFft<TERMS>>(spec + y * (M / 2) * N, PreparedFilter{hs + y * hs_img, beta + y * beta_img, N}, M,
                               log2g, tw, blockIdx.x, smraw, f);
}

bool tc_supported(int rows, int cols) {
    return rows >= 512 && rows <= 4096 && cols >= 512 && cols <= 4096;
}

template <int M, int TERMS>
static cudaError_t rows_tc(bool fwd, const void *src, void *dst, int rows, int nimg, const void *tw,
                           cudaStream_t s) {
    typedef RowCfg<M> K;
    const size_t smem = K::SMEM + tc_stage_bytes<K::THREADS, TERMS>();
    int g = K::PPC > rows / 2 ? rows / 2 : K::PPC;
    const int lg = ilog2(g);
    dim3 grid((rows / 2) >> lg, nimg);
    cudaError_t e;
    if (fwd) {
        e = set_smem_attrs((const void *)k_rows_fwd_tc<M, TERMS>, smem, 1);
        if (e != cudaSuccess) return e;
        k_rows_fwd_tc<M, TERMS><<<grid, K::THREADS, smem, s>>>(static_cast<const float *>(src),
                                                                static_cast<float2 *>(dst), rows, lg,
                                                                static_cast<const float2 *>(tw));
    } else {
        e = set_smem_attrs((const void *)k_rows_inv_tc<M, TERMS>, smem, 1);
        if (e != cudaSuccess) return e;
        k_rows_inv_tc<M, TERMS><<<grid, K::THREADS, smem, s>>>(static_cast<const float2 *>(src),
                                                                static_cast<float *>(dst), rows, lg,
                                                                static_cast<const float2 *>(tw));
    }
    return cudaGetLastError();
}

template <int N, int TERMS>
static cudaError_t cols_tc(void *spec, const float *hs, const float *beta, long long hs_img, long long beta_img,
                           int cols, int nimg, const void *tw, cudaStream_t s) {
    typedef ColCfg<N> K;
    const size_t smem = K::SMEM + tc_stage_bytes<K::THREADS, TERMS>();
    cudaError_t e = set_smem_attrs((const void *)k_cols_tc<N, TERMS>, smem, 2);
    if (e != cudaSuccess) return e;
    int g = rows_pairs_per_block(cols);
    if (g > N / 2) g = N / 2;
    dim3 grid((cols / 2 + K::W - 1) / K::W, nimg);
    k_cols_tc<N, TERMS><<<grid, K::THREADS, smem, s>>>(static_cast<float2 *>(spec), hs, beta, hs_img, beta_img, cols,
                                                       ilog2(g), static_cast<const float2 *>(tw));
    return cudaGetLastError();
}

#define GBFFT_TC_SIZES(X) X(9) X(10) X(11) X(12)

cudaError_t launch_rows_tc(bool fwd, const void *src, void *dst, int rows, int cols, int nimg, const void *tw,
                           int terms, cudaStream_t s) {
    switch (ilog2(cols) * 4 + terms) {
#define GBFFT_C(L)                                                                    \
    case L * 4 + 2: return rows_tc<(1 << L), 2>(fwd, src, dst, rows, nimg, tw, s); \
    case L * 4 + 3: return rows_tc<(1 << L), 3>(fwd, src, dst, rows, nimg, tw, s);
        GBFFT_TC_SIZES(GBFFT_C)
#undef GBFFT_C
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_cols_tc(void *spec, const float *hs, const float *beta, long long hs_img, long long beta_img,
                           int rows, int cols, int nimg, const void *tw_rows, int terms, cudaStream_t s) {
    switch (ilog2(rows) * 4 + terms) {
#define GBFFT_C(L)                                                                                           \
    case L * 4 + 2: return cols_tc<(1 << L), 2>(spec, hs, beta, hs_img, beta_img, cols, nimg, tw_rows, s); \
    case L * 4 + 3: return cols_tc<(1 << L), 3>(spec, hs, beta, hs_img, beta_img, cols, nimg, tw_rows, s);
        GBFFT_TC_SIZES(GBFFT_C)
#undef GBFFT_C
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace gbfft
