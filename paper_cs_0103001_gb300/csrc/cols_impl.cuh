// cols_impl.cuh — the fused column pass of the Sec. 5 pipeline.
//
// The row pass leaves, per image, the row half spectra column-major in slot
// order (layout.cuh); the prepared filter s * Hs[u][k] is column-major in
// row order (column k: u = 0 .. N-1), so every warp reads it contiguously.
// One group of T threads owns one half-spectrum column k and runs, without
// leaving the chip:
//   column FFT (length N = rows, Eq. E2 direction, unscaled)
//   x s * Hs[u, k]        (the filter of Sec. 5 with the 2D scale s = 1/(N M))
//   column inverse FFT    (Eq. E3, unscaled)
// and writes the column back in place.  Column and filter are contiguous in
// memory, so every warp access is a full line; one HBM (or L2) read and one
// write of the spectrum, no transpose kernel.
//
// Real part.  The pipeline's output Re(ifft2(H . F)) equals ifft2(Hs . F) with
// Hs[k] = (H[k] + H[-k]) / 2, because F (the spectrum of a real image) is
// Hermitian: the real part keeps only the even part of the filter.
//
// Column 0 packs two real-row spectra (DC in re, Nyquist in im, see rows.cu):
// q[x] = a[x] + i c[x].  Its column FFT Q splits as P = (Q + conj Q[-u]) / 2 and
// R = (Q - conj Q[-u]) / (2i); filtering P by Hs[u,0] and R by Hs[u,M/2] and
// recombining gives
//   Q'[u] = alpha Q[u] + beta conj(Q[-u]),  alpha = s (h0 + h1)/2, beta = s (h0 - h1)/2,
// h0 = Hs[u,0], h1 = Hs[u,M/2]; the row pass stores alpha in the filter column
// 0 and beta in a separate vector.
#pragma once

#include "check.cuh"
#include "fft_core.cuh"
#include "fft_tc.cuh"
#include "layout.cuh"

namespace gbfft {

template <int N> struct ColCfg {
    static constexpr int E = N < 16 ? N : 16;
    static constexpr int T = N / E;
    static constexpr int W = T >= 256 ? 1 : 256 / T;  // columns per block
    static constexpr int THREADS = W * T;
    static constexpr size_t SMEM = (size_t)W * padded_len(N) * sizeof(float2);
};

// slot of row u = t + T e (compile-time e, so the branch folds away)
template <int N, int E, int T>
__device__ __forceinline__ int slot_e(int t, int e, int log2g) {
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

// One block's share of the column pass: half-spectrum columns bx*W .. bx*W + W - 1
// of one image.  spec: that image's half spectra [M/2][N] (slot order), filt:
// its filter (prepared arrays, or analytic).
// Filter policies of the column pass: h(u, k) = s Hs[u][k] of column k (k = 0:
// alpha) and b(u) = beta of the packed column, for the rows u = t + T e.
// The prepared filter of rows_impl.cuh, read from global memory:
struct PreparedFilter {
    static constexpr bool EARLY = false;  // read after the forward transform (no registers held during it)
    const float *hs, *beta;
    int N;
    __device__ __forceinline__ float h(int u, int k) const { return hs[(size_t)k * N + u]; }
    __device__ __forceinline__ float b(int u) const { return beta[u]; }
};

// Analytic filters computed in the column pass (no filter array is read).
// All three are even, H[-u][-k] = H[u][k], so Hs = H:
//   kind 1, Gaussian:    exp(-|f|^2 / (2 sigma^2)), p = 1 / (2 sigma^2)
//   kind 2, Butterworth: 1 / (1 + (|f|^2 / D0^2)^n), p = 1 / D0^2, order n
//   kind 3, disc (Eq. filtro): 0 where (u - N/2)^2 + (k - M/2)^2 <= b^2, else 1; q = floor(b^2)
// with |f|^2 = u~^2 + k~^2 over the wrapped bins (u~ = u for u < N/2, u - N above).
struct AnalyticFilter {
    static constexpr bool EARLY = true;  // computed while the column's loads are in flight
    int kind, order, N, M;
    float p, s;
    int q;  // disc: floor(b^2) (the squared distances are integers)
    __device__ __forceinline__ float H(int u, int k) const {
        if (kind == 3) {
            const int du = u - (N >> 1), dk = k - (M >> 1);
            return du * du + dk * dk <= q ? 0.f : 1.f;
        }
        const int wu = u < (N >> 1) ? u : u - N, wk = k < (M >> 1) ? k : k - M;
        const float r2 = (float)(wu * wu + wk * wk);  // exact below 2^24, one rounding above
        if (kind == 1) return expf(-r2 * p);
        // x^order by squaring (order 1..16), then the correctly rounded reciprocal
        const float x1 = r2 * p, x2 = x1 * x1, x4 = x2 * x2, x8 = x4 * x4;
        float y = (order & 1) ? x1 : 1.f;
        if (order & 2) y *= x2;
        if (order & 4) y *= x4;
        if (order & 8) y *= x8;
        if (order & 16) y *= x8 * x8;
        return __frcp_rn(1.f + y);
    }
    __device__ __forceinline__ float h(int u, int k) const {
        if (k != 0) return s * H(u, k);
        return 0.5f * s * (H(u, 0) + H(u, M >> 1));
    }
    __device__ __forceinline__ float b(int u) const { return 0.5f * s * (H(u, 0) - H(u, M >> 1)); }
};

// With cs.ls > 0 the block works on the column block of a decomposed image
// (layout.cuh, ColSlab): local columns 0 .. cs.mloc - 1 (global kbase + kl),
// slot s of column kl at spec + ((s >> ls) mloc + kl) 2^ls + (s mod 2^ls); the
// prepared filter holds those columns only (filt.h(u, kl)).
template <int N, typename FFT = Fp32Fft, typename FILT = PreparedFilter>
__device__ __forceinline__ void cols_body(float2 *spec, FILT filt, int M, int log2g, const float2 *__restrict__ tw,
                                          int bx, unsigned char *smraw, FFT fft = FFT(),
                                          ColSlab cs = ColSlab{0, 0, 0}) {
    typedef ColCfg<N> K;
    constexpr int E = K::E, T = K::T, W = K::W;
    const int w = threadIdx.x / T;
    const int t = threadIdx.x - w * T;
    float2 *ex = reinterpret_cast<float2 *>(smraw) + w * padded_len(N);
    const int half = cs.ls ? cs.mloc : M >> 1;  // columns of this launch
    const int k0 = bx * W + w;
    const bool active = k0 < half;  // narrow spectra: surplus column groups idle
    const int k = active ? k0 : 0;
    const bool has0 = cs.kbase == 0 && bx == 0;  // the block holds global column 0
    const bool kz = cs.kbase + k == 0;            // this group's column is global column 0
    float2 *col = spec + (size_t)k * N;
    auto at = [&](int s) -> float2 * {
        if (cs.ls == 0) return col + s;
        const int msk = (1 << cs.ls) - 1;
        return spec + ((size_t)((s >> cs.ls) * cs.mloc + k) << cs.ls) + (s & msk);
    };
    // checked build: every slot below N, the local column inside the block
    // of a decomposed image (the access is skipped where a check fails)
    auto ok = [&](int s) { return chk(s >= 0 && s < N, CK_COL_SLOT) && chk(cs.ls == 0 || k < cs.mloc, CK_COL_CHUNK); };

    float2 v[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int s = slot_e<N, E, T>(t, e, log2g);
        v[e] = active && ok(s) ? *at(s) : make_float2(0.f, 0.f);
    }

    float h[E];
    if constexpr (FILT::EARLY) {
#pragma unroll
        for (int e = 0; e < E; ++e) h[e] = filt.h(t + T * e, k);
    }

    fft.template run<N, E, -1>(v, ex, tw, t);

    if constexpr (!FILT::EARLY) {
#pragma unroll
        for (int e = 0; e < E; ++e) h[e] = filt.h(t + T * e, k);
    }

    if (has0) {  // the group of column 0 needs Q[-u] (uniform per block)
        __syncthreads();
#pragma unroll
        for (int e = 0; e < E; ++e) ex[pad16(t + T * e)] = v[e];
        __syncthreads();
    }
    if (!kz) {
#pragma unroll
        for (int e = 0; e < E; ++e) v[e] = cscale(v[e], h[e]);
    } else {
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int u = t + T * e;
            const float2 qm = ex[pad16((N - u) & (N - 1))];
            const float bt = filt.b(u);
            v[e] = make_float2(h[e] * v[e].x + bt * qm.x, h[e] * v[e].y - bt * qm.y);
        }
    }

    fft.template run<N, E, 1>(v, ex, tw, t);

    if (active) {
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int s = slot_e<N, E, T>(t, e, log2g);
            if (ok(s)) *at(s) = v[e];
        }
    }
}


}  // namespace gbfft
