// cols.cu — the fused column pass of the Sec. 5 pipeline.
//
// After the row pass the workspace holds, per image, the row half spectra
// [rows][M/2] complex64.  One thread block owns W adjacent columns k of it and
// runs, without leaving the chip:
//   column FFT (length N = rows, Eq. E2 direction, unscaled)
//   x s * Hs[u, k]        (the filter of Sec. 5 and the 2D scale s)
//   column inverse FFT    (Eq. E3, unscaled)
// and writes the columns back in place: one HBM read and one write of the
// spectrum, no transpose.  W columns of a row are W*8 contiguous bytes, so
// every warp access covers whole 32-byte sectors.
//
// Real part.  The pipeline's output Re(ifft2(H . F)) equals ifft2(Hs . F) with
// Hs[k] = (H[k] + H[-k]) / 2, because F (the spectrum of a real image) is
// Hermitian: the real part keeps only the even part of the filter.  Working on
// half spectra, the kernel therefore applies Hs, which reads H at (u, k) and
// at the mirrored bin (-u mod N, -k mod M).
//
// Column 0 packs two real-row spectra (DC in re, Nyquist in im, see rows.cu):
// q[x] = a[x] + i c[x].  Its column FFT Q splits as P = (Q + conj Q[-u]) / 2 and
// R = (Q - conj Q[-u]) / (2i); filtering P by Hs[u,0] and R by Hs[u,M/2] and
// recombining gives
//   Q'[u] = Q[u] (h0 + h1)/2 + conj(Q[-u]) (h0 - h1)/2,  h0 = Hs[u,0], h1 = Hs[u,M/2].
//
// Scale: per-axis convention, 1/M on rows and 1/N on columns, s = 1/(N M);
// both inverse transforms are unscaled (Eq. E3), so out = Re(ifft2(H fft2(img))).
#include "fft_core.cuh"
#include "internal.h"

namespace gbfft {

template <int N> struct ColCfg {
    static constexpr int E = N < 16 ? N : 16;
    static constexpr int T = N / E;
    // widest tile within 512 threads and ~140 KiB of shared memory
    static constexpr int WMAX_SMEM = 16384 / N;
    static constexpr int WMAX_THR = 512 / T;
    static constexpr int WMAX0 = WMAX_SMEM < WMAX_THR ? WMAX_SMEM : WMAX_THR;
    static constexpr int WMAX = WMAX0 > 64 ? 64 : (WMAX0 < 1 ? 1 : WMAX0);
};

template <int N>
__global__ void __launch_bounds__(512)
    k_cols_filter(float2 *spec, const float *__restrict__ H, long long h_stride, int M, float scale,
                  const float2 *__restrict__ tw) {
    typedef ColCfg<N> K;
    constexpr int E = K::E, T = K::T, W = K::WMAX;
    extern __shared__ __align__(16) unsigned char smraw[];
    float2 *sm = reinterpret_cast<float2 *>(smraw);
    const int w = threadIdx.x % W;
    const int t = threadIdx.x / W;
    const int half = M >> 1;
    const int k0 = blockIdx.x * W + w;
    const bool active = k0 < half;  // narrow spectra: surplus column slots idle
    const int k = active ? k0 : 0;
    float2 *col = spec + (size_t)blockIdx.y * N * half + k;
    const float *hb = H + (size_t)blockIdx.y * h_stride;

    float2 v[E];
#pragma unroll
    for (int e = 0; e < E; ++e) v[e] = active ? col[(size_t)(t + T * e) * half] : make_float2(0.f, 0.f);

    fft_regs<N, E, -1>(v, sm + w, tw, t, W);

    // x s * Hs[u, k]; the filter is read after the forward transform so it
    // does not hold registers during it
    if (blockIdx.x == 0) {  // tile of the packed column 0 needs Q[-u] (uniform per block)
        __syncthreads();
#pragma unroll
        for (int e = 0; e < E; ++e) sm[pad16(t + T * e) * W + w] = v[e];
        __syncthreads();
    }
    const int km = (M - k) & (M - 1);
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int u = t + T * e;
        const int um = (N - u) & (N - 1);
        if (k != 0) {
            v[e] = cscale(v[e], 0.5f * scale * (hb[u * M + k] + hb[um * M + km]));
        } else {
            const float h0 = 0.5f * (hb[u * M] + hb[um * M]);
            const float h1 = 0.5f * (hb[u * M + half] + hb[um * M + half]);
            const float alpha = 0.5f * scale * (h0 + h1), beta = 0.5f * scale * (h0 - h1);
            const float2 qm = sm[pad16(um) * W];
            v[e] = make_float2(alpha * v[e].x + beta * qm.x, alpha * v[e].y - beta * qm.y);
        }
    }

    fft_regs<N, E, 1>(v, sm + w, tw, t, W);

    if (!active) return;
#pragma unroll
    for (int e = 0; e < E; ++e) col[(size_t)(t + T * e) * half] = v[e];
}

template <int N>
static cudaError_t run_cols(void *spec, const float *H, long long h_stride, int cols, int nimg, float scale,
                            const void *tw, cudaStream_t s) {
    typedef ColCfg<N> K;
    const int half = cols / 2;
    constexpr int W = K::WMAX;
    const int threads = W * K::T;
    const size_t smem = (size_t)padded_len(N) * W * sizeof(float2);
    auto kern = k_cols_filter<N>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    dim3 grid((half + W - 1) / W, nimg);
    kern<<<grid, threads, smem, s>>>(static_cast<float2 *>(spec), H, h_stride, cols, scale,
                                     static_cast<const float2 *>(tw));
    return cudaGetLastError();
}

cudaError_t launch_cols_filter(void *spec, const float *H, long long h_stride, int rows, int cols, int nimg,
                               float scale, const void *tw_rows, cudaStream_t s) {
    switch (ilog2(rows)) {
#define GBFFT_CASE(L) \
    case L: return run_cols<(1 << L)>(spec, H, h_stride, cols, nimg, scale, tw_rows, s);
        GBFFT_CASE(1) GBFFT_CASE(2) GBFFT_CASE(3) GBFFT_CASE(4) GBFFT_CASE(5) GBFFT_CASE(6) GBFFT_CASE(7)
        GBFFT_CASE(8) GBFFT_CASE(9) GBFFT_CASE(10) GBFFT_CASE(11) GBFFT_CASE(12) GBFFT_CASE(13)
#undef GBFFT_CASE
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace gbfft
