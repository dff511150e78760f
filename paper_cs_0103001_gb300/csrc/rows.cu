// rows.cu — the row passes of the Sec. 5 pipeline (fft2 -> filter -> ifft2).
//
// Sec. 4 computes a 2D transform as "FFT on rows, then FFT on columns".  The
// image is real, so two image rows a, b are transformed together as one
// complex row z = a + i b (length M); their spectra separate as
//   A[k] = (Z[k] + conj Z[M-k]) / 2,   B[k] = (Z[k] - conj Z[M-k]) / (2i).
// A real row has a Hermitian spectrum, so only bins 0..M/2 are kept; A[0] and
// A[M/2] are real and share one complex slot (re = DC, im = Nyquist).  A row's
// half spectrum is therefore M/2 complex64 values: the workspace holds
// [image][row][M/2] complex64 — half the bytes of a complex-to-complex pass.
//
// The inverse row pass rebuilds Z[k] = A[k] + i B[k] for all k from the two
// half spectra (A[M-k] = conj A[k]), runs one unscaled inverse FFT (Eq. E3)
// and writes Re z to row a and Im z to row b.
#include "fft_core.cuh"
#include "internal.h"

namespace gbfft {

template <int M> struct RowCfg {
    static constexpr int E = M < 16 ? M : (M >= 8192 ? 32 : 16);
    static constexpr int T = M / E;
    static constexpr int PPC = M < 16 ? 64 : (T >= 256 ? 1 : 256 / T);  // row pairs per block
    static constexpr int THREADS = T * PPC;
    static constexpr int SMS = padded_len(M);
    static constexpr size_t SMEM = (size_t)PPC * SMS * sizeof(float2);
};

// img [nimg][rows][M] float32 -> spec [nimg][rows][M/2] complex64, unscaled.
template <int M>
__global__ void __launch_bounds__(RowCfg<M>::THREADS)
    k_rows_fwd(const float *__restrict__ img, float2 *__restrict__ spec, int rows, const float2 *__restrict__ tw) {
    typedef RowCfg<M> K;
    constexpr int E = K::E, T = K::T, H2 = M / 2;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int g = threadIdx.x / T;
    const int t = threadIdx.x - g * T;
    float2 *sm = reinterpret_cast<float2 *>(smraw) + g * K::SMS;
    const int pair = blockIdx.x * K::PPC + g;
    const bool active = pair < (rows >> 1);
    const size_t img_off = (size_t)blockIdx.y * rows * M;
    float2 v[E];
    if (active) {
        const float *ra = img + img_off + (size_t)(2 * pair) * M;
        const float *rb = ra + M;
#pragma unroll
        for (int e = 0; e < E; ++e) v[e] = make_float2(ra[t + T * e], rb[t + T * e]);
    } else {
#pragma unroll
        for (int e = 0; e < E; ++e) v[e] = make_float2(0.f, 0.f);
    }
    fft_regs<M, E, -1>(v, sm, tw, t);
    __syncthreads();
#pragma unroll
    for (int e = 0; e < E; ++e) sm[pad16(t + T * e)] = v[e];
    __syncthreads();
    if (!active) return;
    float2 *sa = spec + (size_t)blockIdx.y * rows * H2 + (size_t)(2 * pair) * H2;
    float2 *sb = sa + H2;
#pragma unroll
    for (int e = 0; e < E / 2; ++e) {
        const int k = t + T * e;
        const float2 zk = v[e];
        float2 A, B;
        if (e == 0 && t == 0) {
            const float2 zn = v[E / 2];  // Z[M/2]
            A = make_float2(zk.x, zn.x);
            B = make_float2(zk.y, zn.y);
        } else {
            const float2 zm = sm[pad16(M - k)];
            A = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
            B = make_float2(0.5f * (zk.y + zm.y), 0.5f * (zm.x - zk.x));
        }
        sa[k] = A;
        sb[k] = B;
    }
}

// spec [nimg][rows][M/2] complex64 -> out [nimg][rows][M] float32, unscaled.
template <int M>
__global__ void __launch_bounds__(RowCfg<M>::THREADS)
    k_rows_inv(const float2 *__restrict__ spec, float *__restrict__ out, int rows, const float2 *__restrict__ tw) {
    typedef RowCfg<M> K;
    constexpr int E = K::E, T = K::T, H2 = M / 2;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int g = threadIdx.x / T;
    const int t = threadIdx.x - g * T;
    float2 *sm = reinterpret_cast<float2 *>(smraw) + g * K::SMS;
    const int pair = blockIdx.x * K::PPC + g;
    const bool active = pair < (rows >> 1);
    const float2 *sa = spec + (size_t)blockIdx.y * rows * H2 + (size_t)(2 * pair) * H2;
    const float2 *sb = sa + H2;
    float2 v[E];
    if (active) {
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int k = t + T * e;
            float2 a, b;
            if (e < E / 2) {  // 0 <= k < M/2
                a = sa[k];
                b = sb[k];
                if (e == 0 && t == 0) {
                    a.y = 0.f;
                    b.y = 0.f;
                }
            } else if (e == E / 2 && t == 0) {  // k = M/2: the packed Nyquist bins
                a = make_float2(sa[0].y, 0.f);
                b = make_float2(sb[0].y, 0.f);
            } else {  // M/2 < k < M: A[k] = conj A[M-k]
                const float2 am = sa[M - k], bm = sb[M - k];
                a = make_float2(am.x, -am.y);
                b = make_float2(bm.x, -bm.y);
            }
            v[e] = make_float2(a.x - b.y, a.y + b.x);  // A + i B
        }
    } else {
#pragma unroll
        for (int e = 0; e < E; ++e) v[e] = make_float2(0.f, 0.f);
    }
    fft_regs<M, E, 1>(v, sm, tw, t);
    if (!active) return;
    float *ra = out + (size_t)blockIdx.y * rows * M + (size_t)(2 * pair) * M;
    float *rb = ra + M;
#pragma unroll
    for (int e = 0; e < E; ++e) {
        ra[t + T * e] = v[e].x;
        rb[t + T * e] = v[e].y;
    }
}

template <int M>
static cudaError_t run_rows(bool fwd, const void *src, void *dst, int rows, int nimg, const void *tw,
                            cudaStream_t s) {
    typedef RowCfg<M> K;
    const int pairs = rows / 2;
    dim3 grid((pairs + K::PPC - 1) / K::PPC, nimg);
    if (fwd) {
        auto kern = k_rows_fwd<M>;
        if (K::SMEM > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)K::SMEM);
            if (e != cudaSuccess) return e;
        }
        kern<<<grid, K::THREADS, K::SMEM, s>>>(static_cast<const float *>(src), static_cast<float2 *>(dst), rows,
                                               static_cast<const float2 *>(tw));
    } else {
        auto kern = k_rows_inv<M>;
        if (K::SMEM > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)K::SMEM);
            if (e != cudaSuccess) return e;
        }
        kern<<<grid, K::THREADS, K::SMEM, s>>>(static_cast<const float2 *>(src), static_cast<float *>(dst), rows,
                                               static_cast<const float2 *>(tw));
    }
    return cudaGetLastError();
}

static cudaError_t dispatch_rows(bool fwd, const void *src, void *dst, int rows, int cols, int nimg, const void *tw,
                                 cudaStream_t s) {
    switch (ilog2(cols)) {
#define GBFFT_CASE(L) \
    case L: return run_rows<(1 << L)>(fwd, src, dst, rows, nimg, tw, s);
        GBFFT_CASE(1) GBFFT_CASE(2) GBFFT_CASE(3) GBFFT_CASE(4) GBFFT_CASE(5) GBFFT_CASE(6) GBFFT_CASE(7)
        GBFFT_CASE(8) GBFFT_CASE(9) GBFFT_CASE(10) GBFFT_CASE(11) GBFFT_CASE(12) GBFFT_CASE(13)
#undef GBFFT_CASE
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_rows_fwd(const float *img, void *spec, int rows, int cols, int nimg, const void *tw_cols,
                            cudaStream_t s) {
    return dispatch_rows(true, img, spec, rows, cols, nimg, tw_cols, s);
}

cudaError_t launch_rows_inv(const void *spec, float *out, int rows, int cols, int nimg, const void *tw_cols,
                            cudaStream_t s) {
    return dispatch_rows(false, spec, out, rows, cols, nimg, tw_cols, s);
}

}  // namespace gbfft
