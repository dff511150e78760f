// cols.cu — the fused column pass of the Sec. 5 pipeline.
//
// After the row pass the workspace holds, per image, the row half spectra
// [rows][M/2] complex64.  One thread block owns W adjacent columns k of it and
// runs, without leaving the chip:
//   column FFT (length N = rows, Eq. E2 direction, unscaled)
//   x s * Hs[u, k]        (the filter of Sec. 5 and the 2D scale s)
//   column inverse FFT    (Eq. E3, unscaled)
// and writes the columns back in place: one HBM read and one write of the
// spectrum, no transpose.
//
// Real part.  The pipeline's output Re(ifft2(H . F)) equals ifft2(Hs . F) with
// Hs[k] = (H[k] + H[-k]) / 2, because F (the spectrum of a real image) is
// Hermitian: the real part keeps only the even part of the filter.  Working on
// half spectra, the kernel therefore applies Hs, which reads H at (u, k) and
// at the mirrored bin (-u mod N, -k mod M).  Both filter columns of the tile
// are copied to shared memory with cp.async at the start, so the filter reads
// overlap the forward transform and hold no registers during it.
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

constexpr size_t kColsSmemLimit = 227 * 1024;

template <int N, int W> struct ColCfg {
    static constexpr int E = N < 16 ? N : 16;
    static constexpr int T = N / E;
    static constexpr int THREADS = W * T;
    static constexpr size_t SMEM = (size_t)padded_len(N) * W * 8 + 2 * (size_t)N * W * 4;
    static constexpr bool VALID = THREADS <= 1024 && SMEM <= kColsSmemLimit;
    // blocks per SM to aim for: up to 1024 resident threads, as many as the
    // shared memory allows (this caps the registers the compiler may use)
    static constexpr int BY_THR = 1024 / THREADS > 0 ? 1024 / THREADS : 1;
    static constexpr int BY_SMEM = (int)(kColsSmemLimit / (SMEM + 1024)) > 0 ? (int)(kColsSmemLimit / (SMEM + 1024)) : 1;
    static constexpr int MINB = BY_THR < BY_SMEM ? BY_THR : BY_SMEM;
};

template <int N, int W>
__global__ void __launch_bounds__(ColCfg<N, W>::THREADS, ColCfg<N, W>::MINB)
    k_cols_filter(float2 *spec, const float *__restrict__ H, long long h_stride, int M, float scale,
                  const float2 *__restrict__ tw) {
    typedef ColCfg<N, W> K;
    constexpr int E = K::E, T = K::T, NT = K::THREADS;
    extern __shared__ __align__(16) unsigned char smraw[];
    float2 *sm = reinterpret_cast<float2 *>(smraw);
    float *hd = reinterpret_cast<float *>(sm + padded_len(N) * W);  // H[u][k]     at u*W + w
    float *hm = hd + N * W;                                           // H[-u][-k]   at u*W + w
    const int tid = threadIdx.x;
    const int w = tid % W;
    const int t = tid / W;
    const int half = M >> 1;
    const int k0 = blockIdx.x * W;
    const bool active = k0 + w < half;  // narrow spectra: surplus column slots idle
    const int k = active ? k0 + w : 0;
    float2 *col = spec + (size_t)blockIdx.y * N * half + k;
    const float *hb = H + (size_t)blockIdx.y * h_stride;

    // stage the tile's filter columns (asynchronous; waited for after the FFT)
#pragma unroll
    for (int j = 0; j < E; ++j) {
        const int idx = tid + j * NT;
        const int u = idx / W, ww = idx % W;
        const int kc = (k0 + ww < half) ? k0 + ww : 0;
        const int um = (N - u) & (N - 1), kmc = (M - kc) & (M - 1);
        cp_async<4>(hd + idx, hb + (size_t)u * M + kc);
        cp_async<4>(hm + idx, hb + (size_t)um * M + kmc);
    }
    cp_async_commit();

    float2 v[E];
#pragma unroll
    for (int e = 0; e < E; ++e) v[e] = active ? col[(size_t)(t + T * e) * half] : make_float2(0.f, 0.f);

    fft_regs<N, E, -1>(v, sm + w, tw, t, W);

    cp_async_wait_all();
    __syncthreads();  // filter tile visible; exchange buffer free
    if (blockIdx.x == 0) {  // the packed column 0 needs Q[-u] (uniform per block)
#pragma unroll
        for (int e = 0; e < E; ++e) sm[pad16(t + T * e) * W + w] = v[e];
        __syncthreads();
    }
    if (k != 0) {
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int u = t + T * e;
            v[e] = cscale(v[e], 0.5f * scale * (hd[u * W + w] + hm[u * W + w]));
        }
    } else {
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int u = t + T * e;
            const int um = (N - u) & (N - 1);
            const float2 qm = sm[pad16(um) * W];
            const float h0 = 0.5f * (hd[u * W] + hm[u * W]);
            const float h1 = 0.5f * (hb[(size_t)u * M + half] + hb[(size_t)um * M + half]);
            const float alpha = 0.5f * scale * (h0 + h1), beta = 0.5f * scale * (h0 - h1);
            v[e] = make_float2(alpha * v[e].x + beta * qm.x, alpha * v[e].y - beta * qm.y);
        }
    }

    fft_regs<N, E, 1>(v, sm + w, tw, t, W);

    if (!active) return;
#pragma unroll
    for (int e = 0; e < E; ++e) col[(size_t)(t + T * e) * half] = v[e];
}

template <int N, int W>
static cudaError_t run_cols_w(void *spec, const float *H, long long h_stride, int cols, int nimg, float scale,
                              const void *tw, cudaStream_t s) {
    typedef ColCfg<N, W> K;
    if constexpr (!K::VALID) {
        return cudaErrorInvalidConfiguration;
    } else {
        const int half = cols / 2;
        auto kern = k_cols_filter<N, W>;
        if (K::SMEM > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)K::SMEM);
            if (e != cudaSuccess) return e;
        }
        dim3 grid((half + W - 1) / W, nimg);
        kern<<<grid, K::THREADS, K::SMEM, s>>>(static_cast<float2 *>(spec), H, h_stride, cols, scale,
                                               static_cast<const float2 *>(tw));
        return cudaGetLastError();
    }
}

// Default tile width per column length (widest whose block fits).
template <int N> constexpr int default_cols_w() {
    return N >= 8192 ? 1 : N >= 4096 ? 2 : N >= 2048 ? 4 : N >= 1024 ? 8 : 16;
}

// `variant` 0 = default width; 1..4 request W = 1, 2, 4, 8 (tuning); the width
// is capped by the number of half-spectrum columns.
template <int N>
static cudaError_t run_cols(void *spec, const float *H, long long h_stride, int cols, int nimg, float scale,
                            const void *tw, int variant, cudaStream_t s) {
    int W = variant == 0 ? default_cols_w<N>() : (1 << (variant - 1));
    if (W > cols / 2) W = cols / 2;
    switch (W) {
        case 1: return run_cols_w<N, 1>(spec, H, h_stride, cols, nimg, scale, tw, s);
        case 2: return run_cols_w<N, 2>(spec, H, h_stride, cols, nimg, scale, tw, s);
        case 4: return run_cols_w<N, 4>(spec, H, h_stride, cols, nimg, scale, tw, s);
        case 8: return run_cols_w<N, 8>(spec, H, h_stride, cols, nimg, scale, tw, s);
        case 16: return run_cols_w<N, 16>(spec, H, h_stride, cols, nimg, scale, tw, s);
        default: return cudaErrorInvalidValue;
    }
}

int cols_variants() { return 5; }

bool cols_variant_valid(int rows, int cols, int variant) {
    if (variant < 0 || variant > 5) return false;
    if (variant == 0) return true;
    int W = 1 << (variant - 1);
    if (W > cols / 2) W = cols / 2;
    const int E = rows < 16 ? rows : 16;
    const size_t smem = (size_t)padded_len(rows) * W * 8 + 2 * (size_t)rows * W * 4;
    return W * (rows / E) <= 1024 && smem <= kColsSmemLimit;
}

cudaError_t launch_cols_filter(void *spec, const float *H, long long h_stride, int rows, int cols, int nimg,
                               float scale, const void *tw_rows, cudaStream_t s, int variant) {
    switch (ilog2(rows)) {
#define GBFFT_CASE(L) \
    case L: return run_cols<(1 << L)>(spec, H, h_stride, cols, nimg, scale, tw_rows, variant, s);
        GBFFT_CASE(1) GBFFT_CASE(2) GBFFT_CASE(3) GBFFT_CASE(4) GBFFT_CASE(5) GBFFT_CASE(6) GBFFT_CASE(7)
        GBFFT_CASE(8) GBFFT_CASE(9) GBFFT_CASE(10) GBFFT_CASE(11) GBFFT_CASE(12) GBFFT_CASE(13)
#undef GBFFT_CASE
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace gbfft
