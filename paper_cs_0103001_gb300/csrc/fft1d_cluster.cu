// fft1d_cluster.cu — batched 1D transforms of 2^15 .. 2^17 complex64 points,
// one thread-block cluster per transform, one read and one write of HBM.
//
// The four-step split of fourstep.cu (N = N1 N2, j = j1 N2 + j2,
// k = k1 + N1 k2) with its intermediate in distributed shared memory instead
// of a global buffer: the transform does not fit one CTA's shared memory, but
// it fits that of the C CTAs of one cluster.
//   A. CTA c owns columns j2 in [c N2/C, (c+1) N2/C): it reads them from HBM
//      (lanes along j2, so every warp access is a contiguous run), runs the
//      length-N1 column transforms, multiplies by W_N^(j2 k1) (a full table
//      [k1][j2] of the plan, each factor rounded once, read along j2 like the
//      data) and keeps the result in its shared memory, [j2 local][k1].
//   (cluster barrier)
//   B. CTA c owns rows k1 in [c N1/C, (c+1) N1/C): it gathers each row's N2
//      values from the C CTAs' shared memory, runs the length-N2 row
//      transforms and writes bin k1 + N1 k2 to HBM (lanes along k1:
//      contiguous runs again), scaled by 1/N for the forward transform
//      (Eq. E2); the inverse (Eq. E3) uses conjugate twiddles and no scale.
//   (cluster barrier: no CTA leaves while another still reads its memory)
#include <cooperative_groups.h>

#include "fft_core.cuh"
#include "internal.h"

namespace cg = cooperative_groups;

#ifndef GBFFT_CL_PTS
#define GBFFT_CL_PTS 8192  // points per CTA
#endif
#ifndef GBFFT_CL_CMAX
#define GBFFT_CL_CMAX 8  // largest cluster (8 is the portable limit)
#endif
#ifndef GBFFT_CL_MINB4K
#define GBFFT_CL_MINB4K 3  // CTAs per SM the registers are sized for at 4096 points per CTA
#endif

namespace gbfft {

template <int L> struct ClCfg {
    static constexpr int N = 1 << L;
    static constexpr int N1 = 1 << (L / 2), N2 = 1 << (L - L / 2);
    // CTAs per cluster: GBFFT_CL_PTS points each, up to the cluster size limit;
    // 256 threads, so that several CTAs fit an SM and one's memory phases
    // overlap another's transforms
    static constexpr int CMAX = GBFFT_CL_CMAX;
    static constexpr int C = N / GBFFT_CL_PTS < CMAX ? N / GBFFT_CL_PTS : CMAX;
    static constexpr int THREADS = 256, E = 16;      // 4096 points per round
    static constexpr int MINB = N / C <= 4096 ? GBFFT_CL_MINB4K : (N / C <= 8192 ? 2 : 1);
    static constexpr int T1 = N1 / E, WA = THREADS / T1;  // step A: columns per round
    static constexpr int T2 = N2 / E, WB = THREADS / T2;  // step B: rows per round
    static constexpr int CJ = N2 / C, CK = N1 / C;   // columns (A) and rows (B) per CTA
    static constexpr int TS = N1 + 1;                // tile row stride (odd: conflict-free)
    static constexpr int TILE = CJ * TS;
    // exchange layouts of the WA / WB interleaved transforms (fft_core.cuh)
    static constexpr int PSA = exch_pad_shift<float2>(N1, WA), PSB = exch_pad_shift<float2>(N2, WB);
    static constexpr int EXA = padded_len_ps<PSA>(N1) * WA, EXB = padded_len_ps<PSB>(N2) * WB;
    static constexpr int EXCH = EXA > EXB ? EXA : EXB;
    static constexpr size_t SMEM = (size_t)(TILE + EXCH) * sizeof(float2);
    static_assert(C >= 2 && C <= 16, "cluster size");
    static_assert(CJ % WA == 0 && CK % WB == 0, "whole rounds");
    static_assert(SMEM <= 227 * 1024, "shared memory");
};

template <int L, int DIR>
__global__ void __launch_bounds__(ClCfg<L>::THREADS, ClCfg<L>::MINB)
    k_fft1d_cluster(const float2 *in, float2 *out, const float2 *__restrict__ tw1, const float2 *__restrict__ tw2,
                    const float2 *__restrict__ tfull, float scale) {
    typedef ClCfg<L> K;
    constexpr int E = K::E, N1 = K::N1, N2 = K::N2, TS = K::TS;
    extern __shared__ __align__(16) unsigned char smraw[];
    float2 *tile = reinterpret_cast<float2 *>(smraw);
    float2 *exch = tile + K::TILE;
    cg::cluster_group cl = cg::this_cluster();
    const int c = (int)cl.block_rank();
    const size_t base = (size_t)blockIdx.y * K::N;
    const float2 *x = in + base;
    float2 *y = out + base;

    // ---- A. column transforms of this CTA's columns
    {
        // the whole input share in flight at once: column jl, row j1 -> tile[jl][j1]
        // (lanes along jl: contiguous in global memory)
        for (int i = threadIdx.x; i < K::CJ * N1; i += K::THREADS) {
            const int jl = i % K::CJ, j1 = i / K::CJ;
            cp_async<8>(tile + jl * TS + j1, x + (size_t)j1 * N2 + c * K::CJ + jl);
        }
        cp_async_commit();
        cp_async_wait_all();
        __syncthreads();
        const int w = threadIdx.x % K::WA, t = threadIdx.x / K::WA;
        for (int r = 0; r < K::CJ; r += K::WA) {
            const int jl = r + w, j2 = c * K::CJ + jl;
            float2 v[E];
#pragma unroll
            for (int e = 0; e < E; ++e) v[e] = tile[jl * TS + t + K::T1 * e];
            // fft_regs starts its first exchange with a block barrier, so every
            // read of this round's columns is done before they are overwritten
            static_assert(RadixPlan<N1>::P >= 2, "at least one exchange");
            fft_regs<N1, E, DIR, K::PSA>(v, exch + w, tw1, t, K::WA);
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int k1 = t + K::T1 * e;
                const float2 f = __ldg(tfull + k1 * N2 + j2);  // W_N^(k1 j2)
                tile[jl * TS + k1] = DIR < 0 ? cmul(v[e], f) : cmulc(v[e], f);
            }
            __syncthreads();  // the exchange buffer is reused
        }
    }
    cl.sync();

    // ---- B. row transforms of this CTA's rows, gathered from every CTA
    {
        const int w = threadIdx.x % K::WB, t = threadIdx.x / K::WB;
        for (int r = 0; r < K::CK; r += K::WB) {
            const int k1 = c * K::CK + r + w;
            float2 v[E];
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int j2 = t + K::T2 * e;
                const float2 *src = cl.map_shared_rank(tile, j2 / K::CJ);
                v[e] = src[(j2 % K::CJ) * TS + k1];
            }
            fft_regs<N2, E, DIR, K::PSB>(v, exch + w, tw2, t, K::WB);
#pragma unroll
            for (int e = 0; e < E; ++e) y[(size_t)(t + K::T2 * e) * N1 + k1] = cscale(v[e], scale);
            __syncthreads();  // the exchange buffer is reused
        }
    }
    cl.sync();  // every remote read of this CTA's tile is complete
}

template <int L>
static cudaError_t run_cluster(const void *in, void *out, long long batch, int dir, const void *tw1, const void *tw2,
                               const void *tfull, double scale, cudaStream_t s) {
    typedef ClCfg<L> K;
    auto kern = dir < 0 ? k_fft1d_cluster<L, -1> : k_fft1d_cluster<L, 1>;
    cudaError_t e = set_smem_attrs((const void *)kern, K::SMEM, K::MINB);
    if (e == cudaSuccess && K::C > 8)
        e = cudaFuncSetAttribute((const void *)kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
    for (long long b0 = 0; b0 < batch; b0 += 65535) {
        const unsigned nb = (unsigned)(batch - b0 < 65535 ? batch - b0 : 65535);
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(K::C, nb, 1);
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
        e = cudaLaunchKernelEx(&cfg, kern, static_cast<const float2 *>(in) + (size_t)b0 * K::N,
                               static_cast<float2 *>(out) + (size_t)b0 * K::N, static_cast<const float2 *>(tw1),
                               static_cast<const float2 *>(tw2), static_cast<const float2 *>(tfull), (float)scale);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

bool fft1d_cluster_supported(int log2n, bool dbl) { return !dbl && log2n >= 15 && log2n <= 17; }

cudaError_t launch_fft1d_cluster(const void *in, void *out, int log2n, long long batch, int dir, const void *tw_n1,
                                 const void *tw_n2, const void *tw_full, double scale, cudaStream_t s) {
    switch (log2n) {
        case 15: return run_cluster<15>(in, out, batch, dir, tw_n1, tw_n2, tw_full, scale, s);
        case 16: return run_cluster<16>(in, out, batch, dir, tw_n1, tw_n2, tw_full, scale, s);
        case 17: return run_cluster<17>(in, out, batch, dir, tw_n1, tw_n2, tw_full, scale, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace gbfft
