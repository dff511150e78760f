// fft_tc5.cuh — radix-16 Stockham passes on the fifth-generation tensor cores
// (tcgen05.mma, accumulators in tensor memory), split precision.
//
// A radix-16 pass applies the 16-point DFT matrix F[k][n] = exp(DIR 2 pi i k n/16)
// to every butterfly of the block at once.  In real arithmetic, with one row
// per butterfly x = [Re x_0..15 | Im x_0..15] (32 values),
//   y = x B^T,  B = [[C, -S], [S, C]]  (C = cos(2 pi k n/16), S = DIR sin(2 pi k n/16)),
// and y = [Re y_0..15 | Im y_0..15]: a 128 x 32 x 32 product per 128 butterflies
// (tcgen05.mma with M = 128, N = 32; A = the butterflies' rows in shared
// memory, B = the DFT matrix in shared memory, D in 32 columns of tensor
// memory).  Operands are split into parts of a narrower type, x = x0 + x1
// (+ x2), B = B0 + B1 (+ B2), and the products of combined order < TERMS are
// accumulated in FP32 (Henry, Tang and Heinecke 2019 for BF16):
//   FMT_BF16X2: BF16 parts, TERMS = 2, 3 products (about 16 significant bits)
//   FMT_BF16X3: BF16 parts, TERMS = 3, 6 products (about 24 bits)
//   FMT_TF32X2: TF32 parts, TERMS = 2, 3 products (about 22 bits; the second
//               part is the exact FP32 residual, which the tensor core reads
//               to TF32 precision)
//
// A pass, for the butterfly j = t of every thread (E = 16 registers, as in
// fft_core.cuh): FP32 twiddles; every thread splits its row and stores it
// into its group's A tiles (128 butterflies per group, no-swizzle K-major
// layout: 8-row x 16-byte core matrices, K groups LBO = 128 bytes apart, row
// groups SBO apart); the group (four warps) meets at its own named barrier,
// its first thread issues the group's MMAs and commits them to the group's
// mbarrier; the group's threads wait (bounded), load their rows of D from
// tensor memory (each warp its lane quarter), and the outputs go to their
// Stockham destinations through the FP32 exchange buffer.  Groups run
// independently up to the exchange, so one group's MMAs overlap another's
// staging.  The A tiles have shared memory of their own: a group rewrites its
// tiles only after its previous MMAs completed.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

#include "check.cuh"
#include "fft_core.cuh"
#include "tma.cuh"

namespace gbfft {

enum { FMT_BF16X2 = 0, FMT_BF16X3 = 1, FMT_TF32X2 = 2 };

template <int FMT> struct Tc5Fmt {
    static constexpr bool TF32 = FMT == FMT_TF32X2;
    static constexpr int TERMS = FMT == FMT_BF16X3 ? 3 : 2;
    static constexpr int EB = TF32 ? 4 : 2;           // bytes per operand element
    static constexpr int ROWB = 32 * EB;              // bytes of one butterfly row (32 values)
    static constexpr int KG = ROWB / 16;              // K groups of 16 bytes per row
    static constexpr int SBO = KG * 128;              // bytes between 8-row groups
    static constexpr int TILE = 128 * ROWB;           // one part of one group: 128 rows
    static constexpr int KSTEPS = TF32 ? 4 : 2;       // MMAs per product (K = 8 or 16 each)
    static constexpr int BTILE = 32 * ROWB;           // one part of the DFT matrix: 32 rows
    static constexpr int NPROD = TERMS == 3 ? 6 : 3;  // products of combined order < TERMS
    // instruction descriptor: D FP32, A and B BF16 (kind::f16) or TF32 (kind::tf32),
    // both K-major, N = 32, M = 128
    static constexpr uint32_t IDESC = (1u << 4) | ((TF32 ? 2u : 1u) << 7) | ((TF32 ? 2u : 1u) << 10) |
                                      ((uint32_t)(32 >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
};

// shared-memory matrix descriptor: no swizzle, K-major, LBO between K groups,
// SBO between 8-row groups
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

// byte offset of element k of row m in a K-major no-swizzle tile
template <int FMT> __host__ __device__ __forceinline__ int tc5_off(int m, int k) {
    typedef Tc5Fmt<FMT> F;
    constexpr int PER = 16 / F::EB;  // elements per 16-byte core-matrix row
    return (m >> 3) * F::SBO + (k / PER) * 128 + (m & 7) * 16 + (k % PER) * F::EB;
}

// The block's tensor-core state (every thread holds the same values).
struct Tc5State {
    uint32_t tmem;   // tensor-memory base; group g's accumulator at column 32 g
    uint32_t a_sh;   // shared address of the A tiles [part][group]
    uint32_t b_sh;   // shared address of the DFT matrices [direction][part]
    uint32_t bar;    // shared address of this thread's group's MMA-completion mbarrier
    uint64_t *barp;  // the same mbarrier
    uint32_t phase;  // MMA batches of this group completed so far
    int ngroups;     // butterflies per pass / 128
    int *status;     // device status word for a wait that gave up (may be null)
};

// Waits for one batch of MMAs (each try suspends for a hardware time limit of
// microseconds at most); far more than a batch takes.
constexpr uint32_t kTc5Tries = 1u << 16;

// Bounded wait for phase `parity` of an mbarrier: mbarrier.try_wait suspends
// the thread in hardware until the phase completes or a time limit passes;
// at most `tries` such waits.
__device__ __forceinline__ bool mbar_try_wait_bounded(uint64_t *bar, uint32_t parity, uint32_t tries) {
    const uint32_t a = smem_u32(bar);
    for (uint32_t i = 0; i < tries; ++i) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

template <int FMT> struct Tc5Layout {
    typedef Tc5Fmt<FMT> F;
    // shared memory the policy needs beside the body's own: the A tiles, then
    // the DFT matrices, one mbarrier per group and the TMEM slot
    static constexpr size_t a_bytes(int threads) { return (size_t)F::TERMS * (threads / 128) * F::TILE; }
    static constexpr size_t b_bytes() { return (size_t)2 * F::TERMS * F::BTILE; }
    static constexpr size_t bytes(int threads) { return a_bytes(threads) + b_bytes() + 8 * 8 + 16; }
};

// TMEM columns for `groups` accumulators of 32 columns (a power of two >= 32)
__host__ __device__ constexpr int tc5_cols(int groups) {
    return groups <= 1 ? 32 : groups <= 2 ? 64 : groups <= 4 ? 128 : 256;
}

// Set up at kernel start (every thread of the block): DFT matrices into
// shared memory, the mbarriers, tensor memory.  `a` = Tc5Layout::bytes(blockDim.x)
// of shared memory (128-byte aligned) of the policy's own.
template <int FMT>
__device__ __forceinline__ void tc5_setup(Tc5State &st, unsigned char *a, int *status) {
    typedef Tc5Fmt<FMT> F;
    const int groups = blockDim.x / 128;
    unsigned char *b = a + Tc5Layout<FMT>::a_bytes(blockDim.x);
    uint64_t *bars = reinterpret_cast<uint64_t *>(b + Tc5Layout<FMT>::b_bytes());
    uint32_t *slot = reinterpret_cast<uint32_t *>(bars + 8);
    // B[n][k] for direction d (0: forward, DIR = -1; 1: inverse, DIR = +1):
    // n < 16: Re y_n = sum_k C x_re - S x_im;  n >= 16: Im y_(n-16) = S x_re + C x_im
    // cos and sin of 2 pi m / 16 from the exact constants of the 16-point
    // transform (cos of 0, pi/8, pi/4, 3 pi/8), in double
    auto cos16d = [](int m) {
        const double q[4] = {1.0, 0.92387953251128675612818318939678829, 0.70710678118654752440084436210484904,
                             0.38268343236508977172845998403039887};
        m &= 15;
        const int r = m & 3, quad = m >> 2;
        const double cr = q[r], sr = r == 0 ? 0.0 : q[4 - r];
        return quad == 0 ? cr : quad == 1 ? -sr : quad == 2 ? -cr : sr;
    };
    for (int idx = threadIdx.x; idx < 2 * 32 * 32; idx += blockDim.x) {
        const int d = idx >> 10, n = (idx >> 5) & 31, k = idx & 31;
        const int m = ((n & 15) * (k & 15)) & 15;
        const double c = cos16d(m), s = (d == 0 ? -1.0 : 1.0) * cos16d(m - 4);
        double v = n < 16 ? (k < 16 ? c : -s) : (k < 16 ? s : c);
        for (int i = 0; i < F::TERMS; ++i) {
            unsigned char *dst = b + (d * F::TERMS + i) * F::BTILE + tc5_off<FMT>(n, k);
            if constexpr (F::TF32) {
                // TF32 part: round to 10 explicit mantissa bits (the last part keeps the residual)
                float p = (float)v;
                if (i + 1 < F::TERMS) {
                    uint32_t u;
                    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(p));
                    p = __uint_as_float(u);
                }
                *reinterpret_cast<float *>(dst) = p;
                v -= (double)p;
            } else {
                const __nv_bfloat16 p = __float2bfloat16_rn((float)v);
                *reinterpret_cast<__nv_bfloat16 *>(dst) = p;
                v -= (double)__bfloat162float(p);
            }
        }
    }
    if (threadIdx.x < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(slot)),
                     "r"(tc5_cols(groups))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    if (threadIdx.x < groups) mbar_init(&bars[threadIdx.x], 1);
    fence_async_smem();
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    st.tmem = *slot;
    st.a_sh = smem_u32(a);
    st.b_sh = smem_u32(b);
    st.bar = smem_u32(&bars[threadIdx.x >> 7]);
    st.barp = &bars[threadIdx.x >> 7];
    st.phase = 0;
    st.ngroups = groups;
    st.status = status;
}

// At kernel end (every thread): give the tensor memory back.
__device__ __forceinline__ void tc5_teardown(const Tc5State &st) {
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (threadIdx.x < 32)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(st.tmem), "r"(tc5_cols(st.ngroups))
                     : "memory");
}

// two floats -> packed BF16 (a in the low half)
__device__ __forceinline__ uint32_t bf16x2_rn(float a, float b) {
    uint32_t r;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(b), "f"(a));
    return r;
}
__device__ __forceinline__ float bf16lo(uint32_t p) { return __uint_as_float(p << 16); }
__device__ __forceinline__ float bf16hi(uint32_t p) { return __uint_as_float(p & 0xFFFF0000u); }

// Store this thread's row (its butterfly's 16 inputs) as the TERMS parts of
// row m of group g's A tiles.
template <int FMT>
__device__ __forceinline__ void tc5_store_row(const Tc5State &st, const float2 (&v)[16], int g, int m) {
    typedef Tc5Fmt<FMT> F;
    // values in row order: x[k] = Re v[k] (k < 16), Im v[k - 16] (k >= 16)
    auto val = [&](int k) { return k < 16 ? v[k].x : v[k - 16].y; };
    if constexpr (F::TF32) {
#pragma unroll
        for (int q = 0; q < 8; ++q) {  // 16-byte chunk q of the row: values 4q .. 4q + 3
            uint32_t h[4], l[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const float x = val(4 * q + e);
                asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h[e]) : "f"(x));
                l[e] = __float_as_uint(x - __uint_as_float(h[e]));
            }
            const uint32_t off = (uint32_t)tc5_off<FMT>(m, 4 * q);
            const uint32_t a0 = st.a_sh + (uint32_t)(0 * st.ngroups + g) * F::TILE + off;
            const uint32_t a1 = st.a_sh + (uint32_t)(1 * st.ngroups + g) * F::TILE + off;
            asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};\n" ::"r"(a0), "r"(h[0]), "r"(h[1]), "r"(h[2]),
                         "r"(h[3])
                         : "memory");
            asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};\n" ::"r"(a1), "r"(l[0]), "r"(l[1]), "r"(l[2]),
                         "r"(l[3])
                         : "memory");
        }
    } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) {  // 16-byte chunk q: values 8q .. 8q + 7
            uint32_t p[F::TERMS][4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                float x0 = val(8 * q + 2 * e), x1 = val(8 * q + 2 * e + 1);
#pragma unroll
                for (int i = 0; i < F::TERMS; ++i) {
                    const uint32_t h = bf16x2_rn(x0, x1);
                    p[i][e] = h;
                    x0 -= bf16lo(h);
                    x1 -= bf16hi(h);
                }
            }
            const uint32_t off = (uint32_t)tc5_off<FMT>(m, 8 * q);
#pragma unroll
            for (int i = 0; i < F::TERMS; ++i) {
                const uint32_t ai = st.a_sh + (uint32_t)(i * st.ngroups + g) * F::TILE + off;
                asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};\n" ::"r"(ai), "r"(p[i][0]), "r"(p[i][1]),
                             "r"(p[i][2]), "r"(p[i][3])
                             : "memory");
            }
        }
    }
}

// One thread of group g: the group's MMAs, committed to the group's mbarrier.
template <int FMT, int DIR>
__device__ __forceinline__ void tc5_issue(const Tc5State &st, int g) {
    typedef Tc5Fmt<FMT> F;
    const int d = DIR < 0 ? 0 : 1;
    {
        const uint32_t dt = st.tmem + 32u * g;
        int first = 1;
#pragma unroll
        for (int i = 0; i < F::TERMS; ++i) {
#pragma unroll
            for (int j = 0; i + j < F::TERMS; ++j) {
                const uint32_t a = st.a_sh + (uint32_t)(i * st.ngroups + g) * F::TILE;
                const uint32_t b = st.b_sh + (uint32_t)(d * F::TERMS + j) * F::BTILE;
#pragma unroll
                for (int ks = 0; ks < F::KSTEPS; ++ks) {
                    const uint64_t ad = umma_desc(a + 256u * ks, 128u, (uint32_t)F::SBO);
                    const uint64_t bd = umma_desc(b + 256u * ks, 128u, (uint32_t)F::SBO);
                    const uint32_t acc = first ? 0u : 1u;
                    if constexpr (F::TF32)
                        asm volatile(
                            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                            " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(dt),
                            "l"(ad), "l"(bd), "r"(F::IDESC), "r"(acc)
                            : "memory");
                    else
                        asm volatile(
                            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dt),
                            "l"(ad), "l"(bd), "r"(F::IDESC), "r"(acc)
                            : "memory");
                    first = 0;
                }
            }
        }
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(st.bar)
                 : "memory");
}

// One radix-16 Stockham pass (stride NS) with the DFT on the tensor cores:
// same contract as stockham_pass<N, 16, 16, NS, DIR, LAST> (E = 16, thread t
// owns butterfly j = t; v[e] = element t + T e on exit).  Every thread of the
// block calls it; blockDim.x is a multiple of 128.
template <int N, int NS, int DIR, bool LAST, int FMT>
__device__ __forceinline__ void tc5_pass16(float2 (&v)[16], float2 *sm, const float2 *__restrict__ tw, int t, int S,
                                           Tc5State &st) {
    constexpr int T = N / 16;
    if constexpr (NS > 1) {  // twiddles in FP32 (six loads, as in fft_core.cuh)
        const float2 *twp = tw + (NS - 1) + (t & (NS - 1));
        float2 w1[4], w4[4];
#pragma unroll
        for (int q = 1; q < 4; ++q) {
            w1[q] = ldg_c(twp + (q - 1) * NS);
            w4[q] = ldg_c(twp + (4 * q - 1) * NS);
        }
#pragma unroll
        for (int r = 1; r < 16; ++r) {
            const int qa = r & 3, qb = r >> 2;
            const float2 w = qb == 0 ? w1[qa] : (qa == 0 ? w4[qb] : cmul(w1[qa], w4[qb]));
            v[r] = DIR < 0 ? cmul(v[r], w) : cmulc(v[r], w);
        }
    }
    const int row = threadIdx.x, g = row >> 7, m = row & 127;
    tc5_store_row<FMT>(st, v, g, m);  // the group's previous MMAs completed: its tiles are free
    fence_async_smem();
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    asm volatile("bar.sync %0, 128;\n" ::"r"(1 + g) : "memory");  // the group's rows are stored
    if (m == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        tc5_issue<FMT, DIR>(st, g);
    }
    const bool ok = mbar_try_wait_bounded(st.barp, st.phase & 1, kTc5Tries);
    ++st.phase;
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (!ok) {
        if (threadIdx.x == 0 && st.status) atomicExch(st.status, 1);
    } else if (chk(32 * g + 32 <= tc5_cols(st.ngroups), CK_TC5_TMEM)) {
        uint32_t r[32];
        const uint32_t ta = st.tmem + ((uint32_t)(32 * ((threadIdx.x >> 5) & 3)) << 16) + 32u * g;
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,"
            "%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
              "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]),
              "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]),
              "=r"(r[30]), "=r"(r[31])
            : "r"(ta));
        asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
        for (int k = 0; k < 16; ++k) v[k] = make_float2(__uint_as_float(r[k]), __uint_as_float(r[16 + k]));
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    if constexpr (!LAST) {
        __syncthreads();  // the MMAs' reads of A are complete (every thread waited), the exchange may overwrite it
        const int base = (t / NS) * NS * 16 + (t & (NS - 1));
#pragma unroll
        for (int r = 0; r < 16; ++r) sm[pad16(base + r * NS) * S] = v[r];
        __syncthreads();
#pragma unroll
        for (int e = 0; e < 16; ++e) v[e] = sm[pad16(t + T * e) * S];
    }
}

template <int N, int DIR, int FMT, int P> struct PassesTC5 {
    __device__ __forceinline__ static void run(float2 (&v)[16], float2 *sm, const float2 *__restrict__ tw, int t,
                                               int S, Tc5State &st) {
        constexpr int NP = RadixPlan<N>::P;
        constexpr int R = RadixPlan<N>::radix(P);
        constexpr int NS = RadixPlan<N>::stride(P);
        if constexpr (R == 16) {
            tc5_pass16<N, NS, DIR, P == NP - 1, FMT>(v, sm, tw, t, S, st);
        } else {
            stockham_pass<N, 16, R, NS, DIR, P == NP - 1, 4>(v, sm, tw, t, S);
        }
        if constexpr (P + 1 < NP) PassesTC5<N, DIR, FMT, P + 1>::run(v, sm, tw, t, S, st);
    }
};

// Transform policy for the block bodies (as Fp32Fft / TcFft in fft_tc.cuh).
template <int FMT> struct Tc5Fft {
    Tc5State st;
    template <int N, int E, int DIR>
    __device__ __forceinline__ void run(float2 (&v)[E], float2 *sm, const float2 *__restrict__ tw, int t,
                                        int S = 1) {
        static_assert(E == 16, "tensor-core transforms hold 16 elements per thread");
        PassesTC5<N, DIR, FMT, 0>::run(v, sm, tw, t, S, st);
    }
};

}  // namespace gbfft
