// cols.cu — launcher of the fused column pass of the Sec. 5 pipeline; the
// kernel body and the description of the method live in cols_impl.cuh.
#include <cmath>

#include "cols_impl.cuh"
#include "internal.h"

namespace gbfft {

template <int N>
__global__ void __launch_bounds__(ColCfg<N>::THREADS, 2)
    k_cols_filter(float2 *spec, const float *__restrict__ hs, const float *__restrict__ beta, long long hs_img,
                  long long beta_img, int M, int log2g, const float2 *__restrict__ tw) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const size_t y = blockIdx.y;
    cols_body<N>(spec + y * (M / 2) * N, PreparedFilter{hs + y * hs_img, beta + y * beta_img, N}, M, log2g, tw,
                 blockIdx.x, smraw);
}

// The column pass with an analytic filter (cols_impl.cuh) computed in place.
template <int N>
__global__ void __launch_bounds__(ColCfg<N>::THREADS, 2)
    k_cols_analytic(float2 *spec, AnalyticFilter filt, int M, int log2g, const float2 *__restrict__ tw) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const size_t y = blockIdx.y;
    cols_body<N>(spec + y * (M / 2) * N, filt, M, log2g, tw, blockIdx.x, smraw);
}

// Spectrum display (Sec. 5): the column FFTs of the row half spectra, and
// scale * sqrt(Re^2 + Im^2) of every bin in slot order.  The packed column 0
// (DC in re, Nyquist in im) splits into its two real-column spectra
// P = (Q + conj Q[-u]) / 2 (the DC column) and R = (Q - conj Q[-u]) / (2i)
// (the Nyquist column, written to nyq).
template <int N>
__global__ void __launch_bounds__(ColCfg<N>::THREADS)
    k_cols_spectrum(const float2 *__restrict__ spec, float *__restrict__ mag_T, float *__restrict__ nyq, float scale,
                    int M, int log2g, const float2 *__restrict__ tw) {
    typedef ColCfg<N> K;
    constexpr int E = K::E, T = K::T, W = K::W;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int w = threadIdx.x / T;
    const int t = threadIdx.x - w * T;
    float2 *ex = reinterpret_cast<float2 *>(smraw) + w * padded_len(N);
    const int k0 = blockIdx.x * W + w;
    const bool active = k0 < (M >> 1);
    const int k = active ? k0 : 0;
    const float2 *col = spec + (size_t)k * N;
    float2 v[E];
#pragma unroll
    for (int e = 0; e < E; ++e) v[e] = active ? col[slot_e<N, E, T>(t, e, log2g)] : make_float2(0.f, 0.f);
    fft_regs<N, E, -1>(v, ex, tw, t);
    if (blockIdx.x == 0) {  // the group of column 0 needs Q[-u] (uniform per block)
        __syncthreads();
#pragma unroll
        for (int e = 0; e < E; ++e) ex[pad16(t + T * e)] = v[e];
        __syncthreads();
    }
    if (!active) return;  // no barrier follows
    float *mcol = mag_T + (size_t)k * N;
    if (k != 0) {
#pragma unroll
        for (int e = 0; e < E; ++e)
            mcol[slot_e<N, E, T>(t, e, log2g)] = scale * sqrtf(v[e].x * v[e].x + v[e].y * v[e].y);
    } else {
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const float2 q = v[e], qm = ex[pad16((N - (t + T * e)) & (N - 1))];
            const float px = 0.5f * (q.x + qm.x), py = 0.5f * (q.y - qm.y);
            const float rx = 0.5f * (q.y + qm.y), ry = 0.5f * (qm.x - q.x);
            const int sl = slot_e<N, E, T>(t, e, log2g);
            mcol[sl] = scale * sqrtf(px * px + py * py);
            nyq[sl] = scale * sqrtf(rx * rx + ry * ry);
        }
    }
}

template <int N>
static cudaError_t run_spectrum(const void *spec, float *mag_T, float *nyq, float scale, int cols, int log2g,
                                const void *tw, cudaStream_t s) {
    typedef ColCfg<N> K;
    cudaError_t e = set_smem_attrs((const void *)k_cols_spectrum<N>, K::SMEM);
    if (e != cudaSuccess) return e;
    dim3 grid((cols / 2 + K::W - 1) / K::W);
    k_cols_spectrum<N><<<grid, K::THREADS, K::SMEM, s>>>(static_cast<const float2 *>(spec), mag_T, nyq, scale, cols,
                                                         log2g, static_cast<const float2 *>(tw));
    return cudaGetLastError();
}

cudaError_t launch_cols_spectrum(const void *spec, float *mag_T, float *nyq, float scale, int rows, int cols,
                                 const void *tw_rows, cudaStream_t s) {
    int g = rows_pairs_per_block(cols);
    if (g > rows / 2) g = rows / 2;
    const int log2g = ilog2(g);
    switch (ilog2(rows)) {
#define GBFFT_CASE(L) \
    case L: return run_spectrum<(1 << L)>(spec, mag_T, nyq, scale, cols, log2g, tw_rows, s);
        GBFFT_CASE(1) GBFFT_CASE(2) GBFFT_CASE(3) GBFFT_CASE(4) GBFFT_CASE(5) GBFFT_CASE(6) GBFFT_CASE(7)
        GBFFT_CASE(8) GBFFT_CASE(9) GBFFT_CASE(10) GBFFT_CASE(11) GBFFT_CASE(12) GBFFT_CASE(13)
#undef GBFFT_CASE
        default: return cudaErrorInvalidValue;
    }
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

template <int N>
static cudaError_t run_cols_analytic(void *spec, const AnalyticFilter &f, int cols, int nimg, int log2g, const void *tw,
                                     cudaStream_t s) {
    typedef ColCfg<N> K;
    cudaError_t e = set_smem_attrs((const void *)k_cols_analytic<N>, K::SMEM, 2);
    if (e != cudaSuccess) return e;
    dim3 grid((cols / 2 + K::W - 1) / K::W, nimg);
    k_cols_analytic<N><<<grid, K::THREADS, K::SMEM, s>>>(static_cast<float2 *>(spec), f, cols, log2g,
                                                         static_cast<const float2 *>(tw));
    return cudaGetLastError();
}

cudaError_t launch_cols_analytic(void *spec, int kind, double p0, double p1, int rows, int cols, int nimg,
                                 const void *tw_rows, cudaStream_t s) {
    AnalyticFilter f;
    f.kind = kind;
    f.N = rows;
    f.M = cols;
    f.s = (float)(1.0 / ((double)rows * cols));
    f.order = 0;
    f.p = 0.f;
    f.q = 0;
    if (kind == 1) {
        f.p = (float)(1.0 / (2.0 * p0 * p0));
    } else if (kind == 2) {
        f.order = (int)p0;
        f.p = (float)(1.0 / (p1 * p1));
    } else if (kind == 3) {
        const double b2 = std::floor(p0 * p0);
        f.q = b2 > 2147483647.0 ? 2147483647 : (int)b2;
    } else {
        return cudaErrorInvalidValue;
    }
    int g = rows_pairs_per_block(cols);
    if (g > rows / 2) g = rows / 2;
    const int log2g = ilog2(g);
    switch (ilog2(rows)) {
#define GBFFT_CASE(L) \
    case L: return run_cols_analytic<(1 << L)>(spec, f, cols, nimg, log2g, tw_rows, s);
        GBFFT_CASE(1) GBFFT_CASE(2) GBFFT_CASE(3) GBFFT_CASE(4) GBFFT_CASE(5) GBFFT_CASE(6) GBFFT_CASE(7)
        GBFFT_CASE(8) GBFFT_CASE(9) GBFFT_CASE(10) GBFFT_CASE(11) GBFFT_CASE(12) GBFFT_CASE(13)
#undef GBFFT_CASE
        default: return cudaErrorInvalidValue;
    }
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
