// onchip.cu — the whole Sec. 5 pipeline (FFT -> filter -> IFFT) of a small
// image in one launch, without a trip of the spectrum through global memory.
//
// An R x M image (R, M powers of two, 16..256) is handled by one thread-block
// cluster of C CTAs.  The row pairs of the two-for-one row transform
// (layout.cuh: pair p = rows (p, R - p), pair 0 = rows (0, R/2)) are split
// evenly over the CTAs; each CTA keeps its rows' half spectra and prepared
// filter in its own shared memory, column-major ("slot" = side * PP + local
// pair).  The three steps of the pipeline then run back to back:
//   1. forward row FFTs of the CTA's pairs, separated into two half spectra,
//      and the filter of those frequency rows: s * Hs (s = 1/(R M), Hs the
//      even part of H), alpha/beta for the packed DC/Nyquist column;
//   2. (cluster barrier) the half-spectrum columns are split evenly over the
//      CTAs; each gathers its columns from every CTA's shared memory
//      (distributed shared memory), runs column FFT, filter, inverse column
//      FFT, and scatters them back;
//   3. (cluster barrier) inverse row FFTs of the CTA's pairs from its own
//      shared memory, real parts to the output rows.
// Global memory sees the compulsory traffic only: the image and the filter
// read once, the output written once.  The arithmetic is that of rows.cu /
// cols.cu (same FFT core, same separation and packed-column formulas).
#include <cooperative_groups.h>

#include "fft_core.cuh"
#include "internal.h"
#include "layout.cuh"

namespace cg = cooperative_groups;

namespace gbfft {

// WIDE: 8 row pairs per CTA and up to 16 CTAs per cluster (a size beyond the
// portable 8, allowed per kernel), for one or a few images: half the work of
// each SM, on twice the SMs.
template <int R, int M, bool WIDE = false> struct OnChipCfg {
    static constexpr int E = 16;
    static constexpr int RPC = WIDE ? 16 : 32, CMAX = WIDE ? 16 : 8;  // rows per CTA, largest cluster
    static constexpr int C = R / RPC < 1 ? 1 : (R / RPC > CMAX ? CMAX : R / RPC);  // CTAs per cluster
    static constexpr int PP = R / (2 * C);                                 // row pairs per CTA
    static constexpr int KC = (M / 2) / C;                                 // half-spectrum columns per CTA
    static constexpr int TR = M / E, TC = R / E;                           // threads per row / column FFT
    static constexpr int T0 = PP * TR > KC * TC ? PP * TR : KC * TC;
    static constexpr int THREADS = T0 < 32 ? 32 : (T0 > 512 ? 512 : T0);
    static constexpr int RG = PP < THREADS / TR ? PP : THREADS / TR;  // pairs per row iteration
    static constexpr int CG = KC < THREADS / TC ? KC : THREADS / TC;  // columns per column iteration
    static constexpr int SRS = 2 * PP + 1;  // column stride in slots (odd: conflict-free row-wise writes)
    static constexpr int SPEC = (M / 2) * SRS;  // complex slots of half spectra
    static constexpr int EXR = (THREADS / TR) * padded_len(M), EXC = (THREADS / TC) * padded_len(R);
    static constexpr int EXCH = EXR > EXC ? EXR : EXC;
    static constexpr int FLT = ((SPEC + 2 * PP + 3) / 4) * 4;  // floats: filter + beta, rounded to 16 bytes
    static constexpr size_t SMEM = (size_t)SPEC * 8 + (size_t)FLT * 4 + (size_t)EXCH * 8;
    static_assert(R >= 16 && M >= 16 && R <= 256 && M <= 256, "on-chip sizes");
    static_assert(KC >= 1 && PP % RG == 0 && KC % CG == 0, "work split");
};

// slot of row u within the cluster: owner CTA, index in its column
template <int R, int PP> __device__ __forceinline__ void owner_of(int u, int &cta, int &slot) {
    int p, side;
    pair_of(u, R, p, side);
    cta = p / PP;
    slot = side * PP + (p % PP);
}

// the wide form's split exists (every CTA gets at least one half-spectrum column)
template <int R, int M> constexpr bool onchip_wide_ok() { return R >= 128 && M / 2 >= (R / 16 > 16 ? 16 : R / 16); }

template <int R, int M, bool WIDE>
__global__ void __launch_bounds__(OnChipCfg<R, M, WIDE>::THREADS)
    k_onchip(const float *__restrict__ img, const float *__restrict__ H, float *__restrict__ out, long long h_stride,
             float scale, const float2 *__restrict__ twm, const float2 *__restrict__ twr, ImgIndirect ind) {
    typedef OnChipCfg<R, M, WIDE> K;
    constexpr int E = K::E, PP = K::PP, SRS = K::SRS, H2 = M / 2;
    extern __shared__ __align__(16) unsigned char smraw[];
    float2 *spec = reinterpret_cast<float2 *>(smraw);
    float *hsf = reinterpret_cast<float *>(spec + K::SPEC);
    float *bet = hsf + K::SPEC;
    float2 *exch = reinterpret_cast<float2 *>(hsf + K::FLT);

    cg::cluster_group cl = cg::this_cluster();
    const int c = (int)cl.block_rank();
    const size_t z = blockIdx.y;
    if (ind.ptrs) {
        const gbfft_image_ptrs pp = ind.ptrs[ind.idx[z]];
        img = pp.img;
        H = pp.H;
        out = pp.out;
    } else {
        img += z * R * M;
        out += z * R * M;
        H += z * h_stride;
    }

    // ---- 1. forward rows and the filter of their frequency rows
    {
        constexpr int TR = K::TR;
        const int g = threadIdx.x / TR, t = threadIdx.x - g * TR;
        float2 *ex = exch + g * padded_len(M);
        for (int i = 0; i < PP; i += K::RG) {
            const bool active = g < K::RG;
            const int lp = i + g;
            int a, b;
            rows_of_pair(active ? c * PP + lp : 0, R, a, b);
            float2 v[E];
#pragma unroll
            for (int e = 0; e < E; ++e)
                v[e] = active ? make_float2(img[(size_t)a * M + t + TR * e], img[(size_t)b * M + t + TR * e])
                              : make_float2(0.f, 0.f);
            // filter of frequency rows a and b, Hs[u][k] = (H[u][k] + H[-u][-k]) / 2 for
            // k = t + TR e < M/2 (k = 0: alpha and beta of the packed column), read
            // before the transform so that its latency overlaps the image's
            float ha[E / 2], hb[E / 2], b0a = 0.f, b0b = 0.f;
            {
                const int ma = (R - a) & (R - 1), mb = (R - b) & (R - 1);
                const float *Ha = H + (size_t)a * M, *Hma = H + (size_t)ma * M;
                const float *Hb = H + (size_t)b * M, *Hmb = H + (size_t)mb * M;
#pragma unroll
                for (int e = 0; e < E / 2; ++e) {
                    const int k = t + TR * e;
                    if (!active) {
                        ha[e] = hb[e] = 0.f;
                    } else if (e == 0 && t == 0) {
                        const float h0a = 0.5f * (Ha[0] + Hma[0]), h1a = 0.5f * (Ha[H2] + Hma[H2]);
                        const float h0b = 0.5f * (Hb[0] + Hmb[0]), h1b = 0.5f * (Hb[H2] + Hmb[H2]);
                        ha[e] = 0.5f * scale * (h0a + h1a);
                        hb[e] = 0.5f * scale * (h0b + h1b);
                        b0a = 0.5f * scale * (h0a - h1a);
                        b0b = 0.5f * scale * (h0b - h1b);
                    } else {
                        ha[e] = 0.5f * scale * (Ha[k] + Hma[M - k]);
                        hb[e] = 0.5f * scale * (Hb[k] + Hmb[M - k]);
                    }
                }
            }
            fft_regs<M, E, -1>(v, ex, twm, t);
            __syncthreads();
#pragma unroll
            for (int e = 0; e < E; ++e) ex[pad16(t + TR * e)] = v[e];
            __syncthreads();
            if (active) {
                // A[k] (row a) and B[k] (row b) for k = t + TR e < M/2; k = 0 packs (DC, Nyquist)
#pragma unroll
                for (int e = 0; e < E / 2; ++e) {
                    const int k = t + TR * e;
                    const float2 zk = v[e];
                    float2 A, B;
                    if (e == 0 && t == 0) {
                        const float2 zn = v[E / 2];
                        A = make_float2(zk.x, zn.x);
                        B = make_float2(zk.y, zn.y);
                        bet[lp] = b0a;
                        bet[PP + lp] = b0b;
                    } else {
                        const float2 zm = ex[pad16(M - k)];
                        A = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
                        B = make_float2(0.5f * (zk.y + zm.y), 0.5f * (zm.x - zk.x));
                    }
                    spec[k * SRS + lp] = A;
                    spec[k * SRS + PP + lp] = B;
                    hsf[k * SRS + lp] = ha[e];
                    hsf[k * SRS + PP + lp] = hb[e];
                }
            }
            __syncthreads();  // the exchange buffer is reused
        }
    }
    cl.sync();  // every CTA's half spectra and filter are complete

    // ---- 2. columns: gather, FFT, filter, inverse FFT, scatter
    {
        constexpr int TC = K::TC;
        const int w = threadIdx.x / TC, t = threadIdx.x - w * TC;
        float2 *ex = exch + w * padded_len(R);
        for (int j = 0; j < K::KC; j += K::CG) {
            const bool active = w < K::CG;
            const int k = c * K::KC + j + (active ? w : 0);
            // the column, its filter and (column 0) beta, gathered from their owners
            float2 v[E];
            float h[E], bt[E];
#pragma unroll
            for (int e = 0; e < E; ++e) {
                int cta, slot;
                owner_of<R, PP>(t + TC * e, cta, slot);
                const float2 *rs = cl.map_shared_rank(spec, cta);
                const float *rh = cl.map_shared_rank(hsf, cta);
                v[e] = active ? rs[k * SRS + slot] : make_float2(0.f, 0.f);
                h[e] = rh[k * SRS + slot];
                bt[e] = k == 0 ? rh[K::SPEC + slot] : 0.f;  // beta follows the filter
            }
            fft_regs<R, E, -1>(v, ex, twr, t);
            if (c == 0 && j == 0) {  // column 0 is in this group: it needs Q[-u] (uniform per block)
                __syncthreads();
#pragma unroll
                for (int e = 0; e < E; ++e) ex[pad16(t + TC * e)] = v[e];
                __syncthreads();
            }
            if (k != 0) {
#pragma unroll
                for (int e = 0; e < E; ++e) v[e] = cscale(v[e], h[e]);
            } else {
                // packed DC/Nyquist column: Q'[u] = alpha Q[u] + beta conj(Q[-u])
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const float2 qm = ex[pad16((R - (t + TC * e)) & (R - 1))];
                    v[e] = make_float2(h[e] * v[e].x + bt[e] * qm.x, h[e] * v[e].y - bt[e] * qm.y);
                }
            }
            fft_regs<R, E, 1>(v, ex, twr, t);
            if (active) {
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    int cta, slot;
                    owner_of<R, PP>(t + TC * e, cta, slot);
                    cl.map_shared_rank(spec, cta)[k * SRS + slot] = v[e];
                }
            }
            __syncthreads();  // the exchange buffer is reused
        }
    }
    cl.sync();  // every column is back in its owner's shared memory

    // ---- 3. inverse rows from this CTA's own shared memory
    {
        constexpr int TR = K::TR;
        const int g = threadIdx.x / TR, t = threadIdx.x - g * TR;
        float2 *ex = exch + g * padded_len(M);
        for (int i = 0; i < PP; i += K::RG) {
            const bool active = g < K::RG;
            const int lp = active ? i + g : 0;
            int a, b;
            rows_of_pair(c * PP + lp, R, a, b);
            float2 v[E];
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int k = t + TR * e;
                float2 A, B;
                if (e < E / 2) {
                    A = spec[k * SRS + lp];
                    B = spec[k * SRS + PP + lp];
                    if (e == 0 && t == 0) {
                        A.y = 0.f;
                        B.y = 0.f;
                    }
                } else if (e == E / 2 && t == 0) {  // k = M/2: the packed Nyquist bins
                    A = make_float2(spec[lp].y, 0.f);
                    B = make_float2(spec[PP + lp].y, 0.f);
                } else {  // A[k] = conj A[M-k]
                    const float2 am = spec[(M - k) * SRS + lp], bm = spec[(M - k) * SRS + PP + lp];
                    A = make_float2(am.x, -am.y);
                    B = make_float2(bm.x, -bm.y);
                }
                v[e] = make_float2(A.x - B.y, A.y + B.x);  // A + i B
            }
            fft_regs<M, E, 1>(v, ex, twm, t);
            if (active) {
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    out[(size_t)a * M + t + TR * e] = v[e].x;
                    out[(size_t)b * M + t + TR * e] = v[e].y;
                }
            }
            __syncthreads();  // the exchange buffer is reused
        }
    }
}

template <int R, int M, bool WIDE>
static cudaError_t onchip_launch(const float *img, const float *H, float *out, long long h_stride, int nimg,
                                 const void *twm, const void *twr, cudaStream_t s, ImgIndirect ind) {
    typedef OnChipCfg<R, M, WIDE> K;
    const void *kern = (const void *)k_onchip<R, M, WIDE>;
    cudaError_t e = set_smem_attrs(kern, K::SMEM);
    if (e == cudaSuccess && K::C > 8) e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
    const float scale = (float)(1.0 / ((double)R * M));
    for (int z0 = 0; z0 < nimg; z0 += 65535) {
        const int nz = nimg - z0 < 65535 ? nimg - z0 : 65535;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(K::C, nz, 1);
        cfg.blockDim = dim3(K::THREADS, 1, 1);
        cfg.dynamicSmemBytes = K::SMEM;
        cfg.stream = s;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = K::C;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        const ImgIndirect iz{ind.ptrs, ind.ptrs ? ind.idx + z0 : nullptr};
        e = cudaLaunchKernelEx(&cfg, k_onchip<R, M, WIDE>, ind.ptrs ? img : img + (size_t)z0 * R * M,
                               ind.ptrs ? H : H + (size_t)z0 * h_stride, ind.ptrs ? out : out + (size_t)z0 * R * M,
                               h_stride, scale, static_cast<const float2 *>(twm), static_cast<const float2 *>(twr), iz);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// The wide form where it exists, when nimg images of it fit the GPU's SMs at
// once and a cluster of its size can be resident (checked once per shape).
template <int R, int M>
static cudaError_t onchip_dispatch(const float *img, const float *H, float *out, long long h_stride, int nimg,
                                   const void *twm, const void *twr, cudaStream_t s, ImgIndirect ind) {
    if constexpr (onchip_wide_ok<R, M>()) {
        typedef OnChipCfg<R, M, true> K;
        static int wide = -1;  // per process (one device type): 1 if the wide cluster can be resident
        static int sms = 0;
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        if (wide < 0 && (cudaStreamIsCapturing(s, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone)) {
            (void)cudaGetLastError();
            // the first call of this shape is being captured: the portable form,
            // with no device queries inside the capture
            return onchip_launch<R, M, false>(img, H, out, h_stride, nimg, twm, twr, s, ind);
        }
        if (wide < 0) {
            const void *kern = (const void *)k_onchip<R, M, true>;
            int dev = 0, n = 0;
            cudaError_t e = set_smem_attrs(kern, K::SMEM);
            if (e == cudaSuccess && K::C > 8)
                e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
            if (e == cudaSuccess) e = cudaGetDevice(&dev);
            if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            if (e == cudaSuccess) {
                cudaLaunchConfig_t cfg = {};
                cfg.gridDim = dim3(K::C, 1, 1);
                cfg.blockDim = dim3(K::THREADS, 1, 1);
                cfg.dynamicSmemBytes = K::SMEM;
                cudaLaunchAttribute at[1];
                at[0].id = cudaLaunchAttributeClusterDimension;
                at[0].val.clusterDim.x = K::C;
                at[0].val.clusterDim.y = 1;
                at[0].val.clusterDim.z = 1;
                cfg.attrs = at;
                cfg.numAttrs = 1;
                e = cudaOccupancyMaxActiveClusters(&n, k_onchip<R, M, true>, &cfg);
            }
            if (e != cudaSuccess) {
                (void)cudaGetLastError();  // a refused query only means: not the wide form
                n = 0;
            }
            wide = n > 0 ? 1 : 0;
        }
        if (wide == 1 && (long long)nimg * K::C <= sms)
            return onchip_launch<R, M, true>(img, H, out, h_stride, nimg, twm, twr, s, ind);
    }
    return onchip_launch<R, M, false>(img, H, out, h_stride, nimg, twm, twr, s, ind);
}

bool onchip_supported(int rows, int cols) { return rows >= 16 && rows <= 256 && cols >= 16 && cols <= 256; }

#define GBFFT_OC_COLS(L, X) X(L, 4) X(L, 5) X(L, 6) X(L, 7) X(L, 8)
#define GBFFT_OC_ALL(X) GBFFT_OC_COLS(4, X) GBFFT_OC_COLS(5, X) GBFFT_OC_COLS(6, X) GBFFT_OC_COLS(7, X) GBFFT_OC_COLS(8, X)

cudaError_t launch_onchip(const float *img, const float *H, float *out, long long h_stride, int rows, int cols,
                          int nimg, const void *tw_cols, const void *tw_rows, cudaStream_t s, ImgIndirect ind) {
    if (nimg <= 0) return cudaSuccess;
    switch (ilog2(rows) * 16 + ilog2(cols)) {
#define GBFFT_C(LR, LC) \
    case LR * 16 + LC:                                                                                         \
        return onchip_dispatch<(1 << LR), (1 << LC)>(img, H, out, h_stride, nimg, tw_cols, tw_rows, s, ind);
        GBFFT_OC_ALL(GBFFT_C)
#undef GBFFT_C
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace gbfft
