// cols_grad.cu — the fused column pass of the pipeline's adjoint.
//
// Forward: y_b = Re(ifft2(H . fft2(x_b))) = Re(A x_b) with A = s W^H diag(H) W,
// W the unscaled 2D DFT and s = 1/(N M) (per-axis scale; Sec. 4, Sec. 5).
// For a real filter A is Hermitian, so for an upstream gradient G_b = dL/dy_b
//   dL/dx_b = Re(A G_b)                                (the pipeline run on G_b)
//   dL/dH[k] = s sum_b Re(conj((W G_b)[k]) (W x_b)[k]).
// Both x and G are real, so (W G)(W x)* is Hermitian-symmetric and dL/dH is
// even: the half spectrum k = 0..M/2 gives every bin, the mirror bin
// (-u, -k) receiving the same value.
//
// One group of T threads owns one half-spectrum column k (slot order, see
// layout.cuh) and loops over the images of the chunk: column FFT of x's and
// of G's row spectra, accumulate Re(conj(WG) WX) in registers (no atomics;
// the order of the sum is fixed), then filter G's column with the prepared
// s * Hs and inverse-transform it in place for the inverse row pass, exactly
// as the forward column pass does.  The packed column 0 (DC in re, Nyquist in
// im) is split into its two real-column spectra P = (Q + conj Q[-u]) / 2 and
// R = (Q - conj Q[-u]) / (2i) first.  Sums go to a slot-order buffer
// [M/2 + 1][N] (column M/2 holds the Nyquist column) that k_grad_scatter
// finally writes out row-major, mirror bins included.
#include "fft_core.cuh"
#include "internal.h"
#include "layout.cuh"

namespace gbfft {

template <int N> struct GradCfg {
    static constexpr int E = N < 16 ? N : 16;
    static constexpr int T = N / E;
    static constexpr int W = T >= 256 ? 1 : 256 / T;
    static constexpr int THREADS = W * T;
    static constexpr size_t SMEM = 2 * (size_t)W * padded_len(N) * sizeof(float2);
};

template <int N, int E, int T>
__device__ __forceinline__ int grad_slot(int t, int e, int log2g) {
    int p, side;
    if (e < E / 2) {
        p = t + T * e;
        side = 0;
    } else {
        p = (e == E / 2 && t == 0) ? 0 : N - (t + T * e);
        side = 1;
    }
    return ((p >> log2g) << (log2g + 1)) + (side << log2g) + (p & ((1 << log2g) - 1));
}

template <int N>
__global__ void __launch_bounds__(GradCfg<N>::THREADS)
    k_cols_grad(const float2 *spec_x, float2 *spec_g, const float *__restrict__ hs, const float *__restrict__ beta,
                float *grad_T, int M, int nimg, int log2g, float scale, int accumulate,
                const float2 *__restrict__ tw) {
    typedef GradCfg<N> K;
    constexpr int E = K::E, T = K::T, W = K::W;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int w = threadIdx.x / T;
    const int t = threadIdx.x - w * T;
    float2 *exx = reinterpret_cast<float2 *>(smraw) + w * padded_len(N);
    float2 *exg = reinterpret_cast<float2 *>(smraw) + (W + w) * padded_len(N);
    const int half = M >> 1;
    const int k0 = blockIdx.x * W + w;
    const bool active = k0 < half;
    const int k = active ? k0 : 0;

    int sl[E];
    float h[E], acc[E], acc2[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        sl[e] = grad_slot<N, E, T>(t, e, log2g);
        h[e] = hs[(size_t)k * N + t + T * e];  // the prepared filter is in row order
        acc[e] = 0.f;
        acc2[e] = 0.f;
    }

    for (int b = 0; b < nimg; ++b) {
        const float2 *cx = spec_x + (size_t)b * half * N + (size_t)k * N;
        float2 *cg = spec_g + (size_t)b * half * N + (size_t)k * N;
        float2 vx[E], vg[E];
#pragma unroll
        for (int e = 0; e < E; ++e) vx[e] = active ? cx[sl[e]] : make_float2(0.f, 0.f);
        fft_regs<N, E, -1>(vx, exx, tw, t);
#pragma unroll
        for (int e = 0; e < E; ++e) vg[e] = active ? cg[sl[e]] : make_float2(0.f, 0.f);
        fft_regs<N, E, -1>(vg, exg, tw, t);
        if (blockIdx.x == 0) {  // column 0 needs bin -u of both spectra (uniform per block)
            __syncthreads();
#pragma unroll
            for (int e = 0; e < E; ++e) {
                exx[pad16(t + T * e)] = vx[e];
                exg[pad16(t + T * e)] = vg[e];
            }
            __syncthreads();
        }
        if (k != 0) {
#pragma unroll
            for (int e = 0; e < E; ++e) {
                acc[e] += vg[e].x * vx[e].x + vg[e].y * vx[e].y;
                vg[e] = cscale(vg[e], h[e]);
            }
        } else {
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int um = (N - (t + T * e)) & (N - 1);
                const float2 qx = exx[pad16(um)], qg = exg[pad16(um)];
                // P = (Q + conj Qm)/2, R = (Q - conj Qm)/(2i)
                const float2 px = make_float2(0.5f * (vx[e].x + qx.x), 0.5f * (vx[e].y - qx.y));
                const float2 rx = make_float2(0.5f * (vx[e].y + qx.y), 0.5f * (qx.x - vx[e].x));
                const float2 pg = make_float2(0.5f * (vg[e].x + qg.x), 0.5f * (vg[e].y - qg.y));
                const float2 rg = make_float2(0.5f * (vg[e].y + qg.y), 0.5f * (qg.x - vg[e].x));
                acc[e] += pg.x * px.x + pg.y * px.y;
                acc2[e] += rg.x * rx.x + rg.y * rx.y;
                const float bt = beta[t + T * e];
                vg[e] = make_float2(h[e] * vg[e].x + bt * qg.x, h[e] * vg[e].y - bt * qg.y);
            }
        }
        fft_regs<N, E, 1>(vg, exg, tw, t);
        if (active) {
#pragma unroll
            for (int e = 0; e < E; ++e) cg[sl[e]] = vg[e];
        }
    }
    if (!active) return;
    float *gcol = grad_T + (size_t)k * N;
#pragma unroll
    for (int e = 0; e < E; ++e) {
        float g = scale * acc[e];
        if (accumulate) g += gcol[sl[e]];
        gcol[sl[e]] = g;
    }
    if (k == 0) {
        float *ncol = grad_T + (size_t)half * N;
#pragma unroll
        for (int e = 0; e < E; ++e) {
            float g = scale * acc2[e];
            if (accumulate) g += ncol[sl[e]];
            ncol[sl[e]] = g;
        }
    }
}

// grad_T [M/2 + 1][N] (slot order) -> grad_H [N][M] row-major, mirror bins filled.
__global__ void __launch_bounds__(256)
    k_grad_scatter(const float *__restrict__ grad_T, const float *__restrict__ nyq, float *__restrict__ grad_H, int N,
                   int M, int log2g) {
    __shared__ float tile[32][33];
    const int half = M >> 1;
    const int kb = blockIdx.x * 32, sb = blockIdx.y * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;
    for (int i = ty; i < 32; i += 8) {
        const int k = kb + i, s = sb + tx;
        tile[i][tx] = (k < half && s < N) ? grad_T[(size_t)k * N + s] : (k == half && s < N) ? nyq[s] : 0.f;
    }
    __syncthreads();
    for (int i = ty; i < 32; i += 8) {
        const int s = sb + i, k = kb + tx;
        if (s >= N || k > half) continue;
        const int u = row_of_slot(s, N, log2g);
        const float g = tile[tx][i];
        if (k == 0 || k == half) {
            grad_H[(size_t)u * M + k] = g;
        } else {
            grad_H[(size_t)u * M + k] = g;
            grad_H[(size_t)((N - u) & (N - 1)) * M + (M - k)] = g;
        }
    }
}

template <int N>
static cudaError_t run_grad(const void *spec_x, void *spec_g, const float *hs, const float *beta, float *grad_T,
                            int cols, int nimg, int log2g, float scale, int accumulate, const void *tw,
                            cudaStream_t s) {
    typedef GradCfg<N> K;
    auto kern = k_cols_grad<N>;
    cudaError_t e = set_smem_attrs((const void *)kern, K::SMEM);
    if (e != cudaSuccess) return e;
    const int half = cols / 2;
    dim3 grid((half + K::W - 1) / K::W);
    kern<<<grid, K::THREADS, K::SMEM, s>>>(static_cast<const float2 *>(spec_x), static_cast<float2 *>(spec_g), hs,
                                           beta, grad_T, cols, nimg, log2g, scale, accumulate,
                                           static_cast<const float2 *>(tw));
    return cudaGetLastError();
}

cudaError_t launch_cols_grad(const void *spec_x, void *spec_g, const float *hs, const float *beta, float *grad_T,
                             int rows, int cols, int nimg, float scale, int accumulate, const void *tw_rows,
                             cudaStream_t s) {
    int g = rows_pairs_per_block(cols);
    if (g > rows / 2) g = rows / 2;
    const int log2g = ilog2(g);
    switch (ilog2(rows)) {
#define GBFFT_CASE(L)                                                                                      \
    case L:                                                                                                \
        return run_grad<(1 << L)>(spec_x, spec_g, hs, beta, grad_T, cols, nimg, log2g, scale, accumulate, \
                                  tw_rows, s);
        GBFFT_CASE(1) GBFFT_CASE(2) GBFFT_CASE(3) GBFFT_CASE(4) GBFFT_CASE(5) GBFFT_CASE(6) GBFFT_CASE(7)
        GBFFT_CASE(8) GBFFT_CASE(9) GBFFT_CASE(10) GBFFT_CASE(11) GBFFT_CASE(12) GBFFT_CASE(13)
#undef GBFFT_CASE
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_grad_scatter(const float *grad_T, const float *nyq, float *grad_H, int rows, int cols,
                                cudaStream_t s) {
    int g = rows_pairs_per_block(cols);
    if (g > rows / 2) g = rows / 2;
    dim3 grid((cols / 2 + 1 + 31) / 32, (rows + 31) / 32);
    k_grad_scatter<<<grid, dim3(32, 8), 0, s>>>(grad_T, nyq, grad_H, rows, cols, ilog2(g));
    return cudaGetLastError();
}

}  // namespace gbfft
