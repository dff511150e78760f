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
// One thread block owns W adjacent half-spectrum columns and loops over the
// images of the chunk: column FFT of x's and of G's row spectra, accumulate
// Re(conj(WG) WX) in registers (no atomics; the order of the sum is fixed),
// then filter G's column by s Hs and inverse-transform it in place for the
// inverse row pass, exactly as the forward column pass does.  The packed
// column 0 (DC in re, Nyquist in im) is split into its two real-column
// spectra P = (Q + conj Q[-u]) / 2 and R = (Q - conj Q[-u]) / (2i) first.
#include "fft_core.cuh"
#include "internal.h"

namespace gbfft {

template <int N> struct GradCfg {
    static constexpr int E = N < 16 ? N : 16;
    static constexpr int T = N / E;
    // shared memory per block: exchange buffers for x and G (2 x 8.5 B), the
    // running sums (4 B) and the filter tile H[u][k], H[-u][-k] (2 x 4 B) per
    // element and column, plus one N-float sum for the packed column
    static constexpr int WMAX_SMEM = 4096 / N;
    static constexpr int WMAX_THR = 512 / T;
    static constexpr int WMAX0 = WMAX_SMEM < WMAX_THR ? WMAX_SMEM : WMAX_THR;
    static constexpr int WMAX = WMAX0 > 64 ? 64 : (WMAX0 < 1 ? 1 : WMAX0);
    static constexpr size_t SMEM = 2 * (size_t)padded_len(N) * WMAX * 8 + (size_t)N * WMAX * (4 + 8) + (size_t)N * 4;
    static constexpr bool VALID = SMEM <= 227 * 1024;
    static constexpr int THREADS = WMAX * T;
};

template <int N>
__global__ void __launch_bounds__(GradCfg<N>::THREADS)
    k_cols_grad(const float2 *spec_x, float2 *spec_g, const float *__restrict__ H, float *grad_H, int M, int nimg,
                float scale, int accumulate, const float2 *__restrict__ tw) {
    typedef GradCfg<N> K;
    constexpr int E = K::E, T = K::T, W = K::WMAX;
    extern __shared__ __align__(16) unsigned char smraw[];
    float2 *smx = reinterpret_cast<float2 *>(smraw);
    float2 *smg = smx + padded_len(N) * W;
    // running sums of Re(conj(WG) WX) per thread and element: bin (u, k)
    // [packed column: (u, 0)] and, for the packed column only, (u, M/2)
    float *acc = reinterpret_cast<float *>(smg + padded_len(N) * W);
    float *hd = acc + N * W;  // H[u][k] at u*W + w (shared by every image)
    float *hm = hd + N * W;   // H[-u][-k]
    float *acc2 = hm + N * W; // packed column only, at u
    const int w = threadIdx.x % W;
    const int t = threadIdx.x / W;
    const int half = M >> 1;
    const int k0 = blockIdx.x * W + w;
    const bool active = k0 < half;
    const int k = active ? k0 : 0;
    const int km = (M - k) & (M - 1);
    const bool packed = active && k0 == 0;  // the packed DC/Nyquist column (block 0, w = 0)

    const int tid = threadIdx.x;
    constexpr int NT = W * T;
    const int k0b = blockIdx.x * W;
#pragma unroll
    for (int j = 0; j < E; ++j) {
        const int idx = tid + j * NT;
        const int u = idx / W, ww = idx % W;
        const int kc = (k0b + ww < half) ? k0b + ww : 0;
        const int um = (N - u) & (N - 1), kmc = (M - kc) & (M - 1);
        cp_async<4>(hd + idx, H + (size_t)u * M + kc);
        cp_async<4>(hm + idx, H + (size_t)um * M + kmc);
        acc[idx] = 0.f;
    }
    cp_async_commit();
    if (packed) {
#pragma unroll
        for (int e = 0; e < E; ++e) acc2[t + T * e] = 0.f;
    }
    cp_async_wait_all();

    for (int b = 0; b < nimg; ++b) {
        const float2 *cx = spec_x + (size_t)b * N * half + k;
        float2 *cg = spec_g + (size_t)b * N * half + k;
        float2 v[E];
        // x's column spectrum, parked in natural order in its exchange buffer
#pragma unroll
        for (int e = 0; e < E; ++e) v[e] = active ? cx[(t + T * e) * half] : make_float2(0.f, 0.f);
        fft_regs<N, E, -1>(v, smx + w, tw, t, W);
        __syncthreads();
#pragma unroll
        for (int e = 0; e < E; ++e) smx[pad16(t + T * e) * W + w] = v[e];
        // G's column spectrum in registers
#pragma unroll
        for (int e = 0; e < E; ++e) v[e] = active ? cg[(t + T * e) * half] : make_float2(0.f, 0.f);
        fft_regs<N, E, -1>(v, smg + w, tw, t, W);
        if (blockIdx.x == 0) {  // the packed column needs bin -u of G's spectrum too
            __syncthreads();
#pragma unroll
            for (int e = 0; e < E; ++e) smg[pad16(t + T * e) * W + w] = v[e];
        }
        __syncthreads();
        if (!packed) {
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int u = t + T * e;
                const float2 vx = smx[pad16(u) * W + w];
                acc[u * W + w] += v[e].x * vx.x + v[e].y * vx.y;
                v[e] = cscale(v[e], 0.5f * scale * (hd[u * W + w] + hm[u * W + w]));
            }
        } else {
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int u = t + T * e;
                const int um = (N - u) & (N - 1);
                const float2 vx = smx[pad16(u) * W];
                const float2 qx = smx[pad16(um) * W], qg = smg[pad16(um) * W];
                // P = (Q + conj Qm)/2, R = (Q - conj Qm)/(2i)
                const float2 px = make_float2(0.5f * (vx.x + qx.x), 0.5f * (vx.y - qx.y));
                const float2 rx = make_float2(0.5f * (vx.y + qx.y), 0.5f * (qx.x - vx.x));
                const float2 pg = make_float2(0.5f * (v[e].x + qg.x), 0.5f * (v[e].y - qg.y));
                const float2 rg = make_float2(0.5f * (v[e].y + qg.y), 0.5f * (qg.x - v[e].x));
                acc[u * W] += pg.x * px.x + pg.y * px.y;
                acc2[u] += rg.x * rx.x + rg.y * rx.y;
                const float h0 = 0.5f * (hd[u * W] + hm[u * W]);
                const float h1 = 0.5f * (H[u * M + half] + H[um * M + half]);
                const float alpha = 0.5f * scale * (h0 + h1), beta = 0.5f * scale * (h0 - h1);
                v[e] = make_float2(alpha * v[e].x + beta * qg.x, alpha * v[e].y - beta * qg.y);
            }
        }
        fft_regs<N, E, 1>(v, smg + w, tw, t, W);
        if (active) {
#pragma unroll
            for (int e = 0; e < E; ++e) cg[(t + T * e) * half] = v[e];
        }
        __syncthreads();  // smx is rewritten by the next image
    }
    if (!active) return;
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int u = t + T * e;
        const int um = (N - u) & (N - 1);
        if (!packed) {
            float g = scale * acc[u * W + w];
            if (accumulate) g += grad_H[u * M + k];
            grad_H[u * M + k] = g;
            grad_H[um * M + km] = g;  // even: same value at the mirror bin
        } else {
            float g0 = scale * acc[u * W], g1 = scale * acc2[u];
            if (accumulate) {
                g0 += grad_H[u * M];
                g1 += grad_H[u * M + half];
            }
            grad_H[u * M] = g0;
            grad_H[u * M + half] = g1;
        }
    }
}

template <int N>
static cudaError_t run_grad(const void *spec_x, void *spec_g, const float *H, float *grad_H, int cols, int nimg,
                            float scale, int accumulate, const void *tw, cudaStream_t s) {
    typedef GradCfg<N> K;
    constexpr int W = K::WMAX;
    const int half = cols / 2;
    const size_t smem = K::SMEM;
    if (!K::VALID) return cudaErrorInvalidConfiguration;
    auto kern = k_cols_grad<N>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    dim3 grid((half + W - 1) / W);
    kern<<<grid, W * K::T, smem, s>>>(static_cast<const float2 *>(spec_x), static_cast<float2 *>(spec_g), H, grad_H,
                                      cols, nimg, scale, accumulate, static_cast<const float2 *>(tw));
    return cudaGetLastError();
}

cudaError_t launch_cols_grad(const void *spec_x, void *spec_g, const float *H, float *grad_H, int rows, int cols,
                             int nimg, float scale, int accumulate, const void *tw_rows, cudaStream_t s) {
    switch (ilog2(rows)) {
#define GBFFT_CASE(L) \
    case L: return run_grad<(1 << L)>(spec_x, spec_g, H, grad_H, cols, nimg, scale, accumulate, tw_rows, s);
        GBFFT_CASE(1) GBFFT_CASE(2) GBFFT_CASE(3) GBFFT_CASE(4) GBFFT_CASE(5) GBFFT_CASE(6) GBFFT_CASE(7)
        GBFFT_CASE(8) GBFFT_CASE(9) GBFFT_CASE(10) GBFFT_CASE(11) GBFFT_CASE(12) GBFFT_CASE(13)
#undef GBFFT_CASE
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace gbfft
