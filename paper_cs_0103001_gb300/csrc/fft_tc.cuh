// fft_tc.cuh — radix-16 Stockham passes on the tensor cores, split BF16.
//
// A radix-16 pass applies the 16-point DFT matrix F[k][n] = exp(DIR 2 pi i k n / 16)
// to many butterflies at once, which is a dense product Y = F X with X one
// column per butterfly.  Here it runs as mma.sync.m16n8k16 (BF16 operands,
// FP32 accumulation) on 8 butterflies per instruction.  BF16 keeps 8
// significant bits, so every operand is split into TERMS BF16 parts,
// x = x0 + x1 (+ x2), F = F0 + F1 (+ F2), and the product keeps the terms of
// combined order < TERMS: three products (x0F0, x0F1, x1F0) for TERMS = 2,
// six for TERMS = 3 (Henry, Tang and Heinecke, "Leveraging the bfloat16
// artificial intelligence datatype for higher-precision computations", 2019).
// In real arithmetic Yr = Fr Xr - Fi Xi and Yi = Fi Xr + Fr Xi.
//
// Data path of a pass, per warp (32 butterflies, one per thread): twiddle in
// FP32 as in fft_core.cuh; every thread splits its butterfly's inputs and
// writes them to the warp-private staging area (four groups of 8 butterflies);
// then, for each group, the warp runs the MMAs and the accumulators (output
// k = g, g + 8 of butterflies 2 tq, 2 tq + 1, with g = lane / 4, tq = lane mod
// 4) go straight to their Stockham destinations in the exchange buffer.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

#include "fft_core.cuh"

namespace gbfft {

// cos(2 pi m / 16) and sin(2 pi m / 16) from the three constants of the
// 16-point transform
__device__ __forceinline__ float cos16(int m) {
    const float c1 = 0.92387953251128675613f, s1 = 0.38268343236508977173f, h = 0.70710678118654752440f;
    const float q[4] = {1.f, c1, h, s1};  // cos of 0, pi/8, pi/4, 3pi/8
    m &= 15;
    const int r = m & 3, quad = m >> 2;  // angle = quad * pi/2 + r * pi/8
    float cr = q[r], sr = r == 0 ? 0.f : q[4 - r];
    switch (quad) {
        case 0: return cr;
        case 1: return -sr;
        case 2: return -cr;
        default: return sr;
    }
}
__device__ __forceinline__ float sin16(int m) { return cos16(m - 4); }

template <int TERMS>
__device__ __forceinline__ void bf16_split(float x, __nv_bfloat16 (&p)[TERMS]) {
    float r = x;
#pragma unroll
    for (int i = 0; i < TERMS; ++i) {
        p[i] = __float2bfloat16_rn(r);
        r -= __bfloat162float(p[i]);
    }
}

__device__ __forceinline__ uint32_t pack_bf16(__nv_bfloat16 lo, __nv_bfloat16 hi) {
    return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

__device__ __forceinline__ void mma_bf16_16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Per-thread operand state: A fragments of Fr = cos and Fs = sin (each split
// term; the pass applies the sign of its direction) and the warp's staging
// area: for each of the 4 groups of 8 butterflies, TERMS x {re, im} planes of
// 8 rows x 12 words.
template <int TERMS> struct TcState {
    uint32_t fr[TERMS][4], fi[TERMS][4];
    uint32_t *stg;
    static constexpr int PLANE = 8 * 12;                 // words per plane
    static constexpr int GROUP = 2 * TERMS * PLANE;      // words per group of 8 butterflies
    static constexpr int WORDS_PER_WARP = 4 * GROUP;
};

// A[k][n] = F[k][n] for the thread's fragment slots: reg0 (g, 2tq..2tq+1),
// reg1 (g+8, ..), reg2 (g, 2tq+8..), reg3 (g+8, 2tq+8..)
template <int TERMS>
__device__ __forceinline__ void tc_init(TcState<TERMS> &st, uint32_t *warp_stage, int lane) {
    const int g = lane >> 2, tq = lane & 3;
#pragma unroll
    for (int reg = 0; reg < 4; ++reg) {
        const int k = g + ((reg & 1) ? 8 : 0);
        const int n0 = 2 * tq + ((reg & 2) ? 8 : 0);
        __nv_bfloat16 r0[TERMS], r1[TERMS], i0[TERMS], i1[TERMS];
        bf16_split<TERMS>(cos16(k * n0), r0);
        bf16_split<TERMS>(cos16(k * (n0 + 1)), r1);
        bf16_split<TERMS>(sin16(k * n0), i0);
        bf16_split<TERMS>(sin16(k * (n0 + 1)), i1);
#pragma unroll
        for (int i = 0; i < TERMS; ++i) {
            st.fr[i][reg] = pack_bf16(r0[i], r1[i]);
            st.fi[i][reg] = pack_bf16(i0[i], i1[i]);
        }
    }
    st.stg = warp_stage;
}

// One radix-16 Stockham pass (stride NS) on the tensor cores.  E = 16: thread
// t owns butterfly j = t, inputs v[r] = element j + r N/16.  On exit v[e] is
// element t + T e of the pass output (exchange included, also after the last
// pass).  T = N/16 must be a multiple of 32 and every thread of the block
// must call it.
template <int N, int NS, int DIR, int TERMS>
__device__ __forceinline__ void tc_pass16(float2 (&v)[16], float2 *sm, const float2 *__restrict__ tw, int t, int S,
                                          TcState<TERMS> &st) {
    constexpr int T = N / 16;
    static_assert(T % 32 == 0, "tensor-core passes need whole warps of butterflies");
    if constexpr (NS > 1) {
        const float2 *twp = tw + (NS - 1) + (t & (NS - 1));
#pragma unroll
        for (int r = 1; r < 16; ++r) {
            const float2 w = __ldg(twp + (r - 1) * NS);
            v[r] = DIR < 0 ? cmul(v[r], w) : cmulc(v[r], w);
        }
    }
    const int lane = t & 31, g = lane >> 2, tq = lane & 3;
    const int warp_base = t - lane;
    constexpr int PLANE = TcState<TERMS>::PLANE, GROUP = TcState<TERMS>::GROUP;
    // every lane splits its own butterfly's 16 inputs and stages them as row
    // (lane mod 8) of group (lane / 8): plane 2i = re part i, 2i+1 = im part i
    {
        uint32_t *row = st.stg + (lane >> 3) * GROUP + (lane & 7) * 12;
#pragma unroll
        for (int i = 0; i < TERMS; ++i) {
            uint32_t wr[8], wi[8];
#pragma unroll
            for (int w = 0; w < 8; ++w) {
                __nv_bfloat16 a[TERMS], b[TERMS], c[TERMS], d[TERMS];
                bf16_split<TERMS>(v[2 * w].x, a);
                bf16_split<TERMS>(v[2 * w + 1].x, b);
                bf16_split<TERMS>(v[2 * w].y, c);
                bf16_split<TERMS>(v[2 * w + 1].y, d);
                wr[w] = pack_bf16(a[i], b[i]);
                wi[w] = pack_bf16(c[i], d[i]);
            }
            uint4 *pr = reinterpret_cast<uint4 *>(row + (2 * i) * PLANE);
            uint4 *pi = reinterpret_cast<uint4 *>(row + (2 * i + 1) * PLANE);
            pr[0] = make_uint4(wr[0], wr[1], wr[2], wr[3]);
            pr[1] = make_uint4(wr[4], wr[5], wr[6], wr[7]);
            pi[0] = make_uint4(wi[0], wi[1], wi[2], wi[3]);
            pi[1] = make_uint4(wi[4], wi[5], wi[6], wi[7]);
        }
    }
    __syncwarp();
    __syncthreads();  // the previous exchange's reads are complete
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const uint32_t *gs = st.stg + q * GROUP;
        uint32_t xr[TERMS][2], xi[TERMS][2];
#pragma unroll
        for (int i = 0; i < TERMS; ++i) {
            xr[i][0] = gs[(2 * i) * PLANE + g * 12 + tq];
            xr[i][1] = gs[(2 * i) * PLANE + g * 12 + tq + 4];
            xi[i][0] = gs[(2 * i + 1) * PLANE + g * 12 + tq];
            xi[i][1] = gs[(2 * i + 1) * PLANE + g * 12 + tq + 4];
        }
        // F = cos + DIR i sin:  Yr = cos Xr - DIR sin Xi,  Yi = DIR sin Xr + cos Xi
        float yr[4] = {0.f, 0.f, 0.f, 0.f}, yi[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int i = 0; i < TERMS; ++i) {
            uint32_t nfi[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) nfi[r] = st.fi[i][r] ^ 0x80008000u;  // -sin
#pragma unroll
            for (int j = 0; j + i < TERMS; ++j) {
                mma_bf16_16816(yr, st.fr[i], xr[j][0], xr[j][1]);
                mma_bf16_16816(yr, DIR < 0 ? st.fi[i] : nfi, xi[j][0], xi[j][1]);
                mma_bf16_16816(yi, DIR < 0 ? nfi : st.fi[i], xr[j][0], xr[j][1]);
                mma_bf16_16816(yi, st.fr[i], xi[j][0], xi[j][1]);
            }
        }
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const int j = warp_base + 8 * q + 2 * tq + c;
            const int base = (j / NS) * NS * 16 + (j & (NS - 1));
            sm[pad16(base + g * NS) * S] = make_float2(yr[c], yi[c]);
            sm[pad16(base + (g + 8) * NS) * S] = make_float2(yr[2 + c], yi[2 + c]);
        }
    }
    __syncwarp();  // the staging area is rewritten by the next pass
    __syncthreads();
#pragma unroll
    for (int e = 0; e < 16; ++e) v[e] = sm[pad16(t + T * e) * S];
}

template <int N, int DIR, int TERMS, int P> struct PassesTC {
    __device__ __forceinline__ static void run(float2 (&v)[16], float2 *sm, const float2 *__restrict__ tw, int t,
                                               int S, TcState<TERMS> &st) {
        constexpr int NP = RadixPlan<N>::P;
        constexpr int R = RadixPlan<N>::radix(P);
        constexpr int NS = RadixPlan<N>::stride(P);
        if constexpr (R == 16) {
            tc_pass16<N, NS, DIR, TERMS>(v, sm, tw, t, S, st);
        } else {
            stockham_pass<N, 16, R, NS, DIR, P == NP - 1, 4>(v, sm, tw, t, S);
        }
        if constexpr (P + 1 < NP) PassesTC<N, DIR, TERMS, P + 1>::run(v, sm, tw, t, S, st);
    }
};

// Same contract as fft_regs<N, 16, DIR> (v[e] = element / bin t + T e on entry
// and exit), with the radix-16 passes on the tensor cores.
template <int N, int DIR, int TERMS>
__device__ __forceinline__ void fft_regs_tc(float2 (&v)[16], float2 *sm, const float2 *__restrict__ tw, int t,
                                            int S, TcState<TERMS> &st) {
    PassesTC<N, DIR, TERMS, 0>::run(v, sm, tw, t, S, st);
}

// Transform policies for the block bodies: plain FP32 butterflies, or
// tensor-core radix-16 passes with a TERMS-way BF16 split.
struct Fp32Fft {
    template <int N, int E, int DIR>
    __device__ __forceinline__ void run(float2 (&v)[E], float2 *sm, const float2 *__restrict__ tw, int t,
                                        int S = 1) {
        fft_regs<N, E, DIR>(v, sm, tw, t, S);
    }
};

template <int TERMS> struct TcFft {
    TcState<TERMS> st;
    template <int N, int E, int DIR>
    __device__ __forceinline__ void run(float2 (&v)[E], float2 *sm, const float2 *__restrict__ tw, int t,
                                        int S = 1) {
        static_assert(E == 16, "tensor-core transforms hold 16 elements per thread");
        fft_regs_tc<N, DIR, TERMS>(v, sm, tw, t, S, st);
    }
};

}  // namespace gbfft
