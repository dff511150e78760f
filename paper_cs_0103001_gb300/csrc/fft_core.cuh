// fft_core.cuh — register/shared-memory FFT building blocks for sm_103a.
//
// The transform is the DFT of Eq. E2 / Eq. E3 (arXiv cs/0103001).  The paper
// evaluates it with a radix-2 decimation-in-time tree (Sec. 2); here the same
// result is computed with a Stockham autosort schedule of radix-16 passes
// (plus one radix-2/4/8 pass when log2 N is not a multiple of 4), which is the
// tree with four levels merged into each pass and the bit reversal absorbed
// into the pass addressing.
//
// Data model.  One length-N transform is held by T = N/E threads, E complex
// values each.  Between passes, thread t holds the elements with index
// t + T*e in register e.  A pass of radix R with stride Ns (product of the
// radices already applied) makes every thread run E/R butterflies
// j = t + q*T: it takes inputs j + r*N/R (which are registers q + r*E/R),
// multiplies input r by W_{Ns R}^{r (j mod Ns)}, runs an R-point DFT and sends
// output r to index (j div Ns)*Ns*R + (j mod Ns) + r*Ns.  Outputs are
// exchanged through shared memory except after the last pass, whose outputs
// land exactly on index t + T*e of the same register: the result comes out
// in natural order, in the same register pattern as the input.
//
// Twiddles.  Pass p >= 1 (Ns = product of earlier radices) needs
// W_{Ns R}^{r m} for r = 1..R-1, m = 0..Ns-1.  They are stored in one table
// per length, pass p at offset Ns - 1, entry (r-1)*Ns + m, so consecutive
// threads read consecutive entries; the sizes telescope to N - 1 entries in
// all.  Entries hold the forward (negative-exponent) factor; inverse passes
// use the conjugate.  The table is built once per plan in FP64 and rounded
// once to the working precision.  A complex64 radix-16 pass reads only the
// factors r = 1, 2, 3, 4, 8, 12 and forms the others as products
// W^(a + 4b) = W^a W^(4b): six loads instead of fifteen, one more rounding
// for nine of the factors.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace gbfft {

// ---------------------------------------------------------------- types --
template <typename R> struct cvec;
template <> struct cvec<float> { typedef float2 type; };
template <> struct cvec<double> { typedef double2 type; };

__host__ __device__ constexpr int ilog2(long long n) { return n <= 1 ? 0 : 1 + ilog2(n >> 1); }

// Shared-memory index of element x: one pad slot per 16 elements keeps the
// strided Stockham writes free of bank conflicts.
__device__ __forceinline__ int pad16(int x) { return x + (x >> 4); }
__host__ __device__ constexpr int padded_len(int n) { return n + (n >> 4); }

// The same with one pad slot per 2^PS elements (pad_ps<4> = pad16).
template <int PS> __device__ __forceinline__ int pad_ps(int x) { return x + (x >> PS); }
template <int PS> __host__ __device__ constexpr int padded_len_ps(int n) { return n + (n >> PS); }

// Pad period for S transforms interleaved element by element (element x of
// transform w at pad(x) * S + w, thread (t, w) = (tid / S, tid % S)).  A
// shared-memory model of every exchange write and read (32 banks of 4 bytes;
// 8-byte accesses served per half warp, 16-byte ones per quarter warp, one
// wavefront per distinct word of the busiest bank; it reproduces the bank
// conflicts measured on these kernels) gives the minimum with one pad per 16
// elements for all lengths and interleaves used here except these, where the
// threads t of a half warp would write the first pass's outputs (radix 2 or
// 4, or the strided radix-16 writes at length 2048) to the same banks:
//   complex64  length 512, S = 8: one pad per 2;  1024, S = 8: per 4;
//              2048, S = 4: per 8;   complex128 length 2048, S = 4: per 8.
template <typename C> __host__ __device__ constexpr int exch_pad_shift(int n, int s) {
    return sizeof(C) == 8 ? (n == 512 && s == 8 ? 1 : n == 1024 && s == 8 ? 2 : n == 2048 && s == 4 ? 3 : 4)
                          : (n == 2048 && s == 4 ? 3 : 4);
}

// ---------------------------------------------------------- radix plan --
// Length N = 2^L.  N < 16: one pass of radix N.  Otherwise the first pass has
// radix 2^(L mod 4) (16 when L mod 4 = 0) and every later pass radix 16.
template <int N> struct RadixPlan {
    static constexpr int L = ilog2(N);
    static constexpr int P = N < 16 ? 1 : (L + 3) / 4;
    static constexpr int FIRST = N < 16 ? N : ((L & 3) == 0 ? 16 : (1 << (L & 3)));
    static constexpr int MAXR = N < 16 ? N : 16;
    __host__ __device__ static constexpr int radix(int p) { return p == 0 ? FIRST : 16; }
    __host__ __device__ static constexpr int stride(int p) { return p == 0 ? 1 : FIRST * (1 << (4 * (p - 1))); }
};

// Host-side mirror of RadixPlan for runtime N (twiddle-table generation).
__host__ __device__ inline int plan_passes(int n) {
    int L = ilog2(n);
    return n < 16 ? 1 : (L + 3) / 4;
}
__host__ __device__ inline int plan_radix(int n, int p) {
    int L = ilog2(n);
    int first = n < 16 ? n : ((L & 3) == 0 ? 16 : (1 << (L & 3)));
    return p == 0 ? first : 16;
}
__host__ __device__ inline int plan_stride(int n, int p) {
    if (p == 0) return 1;
    return plan_radix(n, 0) * (1 << (4 * (p - 1)));
}

// -------------------------------------------------------- complex math --
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return C{a.x + b.x, a.y + b.y}; }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return C{a.x - b.x, a.y - b.y}; }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
    return C{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
// a * conj(b)
template <typename C> __device__ __forceinline__ C cmulc(C a, C b) {
    return C{a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y};
}
template <typename C, typename S> __device__ __forceinline__ C cscale(C a, S s) { return C{a.x * s, a.y * s}; }
// a * (DIR * i): DIR = -1 multiplies by -i (forward), +1 by +i (inverse)
template <int DIR, typename C> __device__ __forceinline__ C mul_diri(C a) {
    return DIR < 0 ? C{a.y, -a.x} : C{-a.y, a.x};
}
// a * exp(DIR * i * pi/4) = a * (1 + DIR i)/sqrt(2)
template <int DIR, typename C> __device__ __forceinline__ C mul_w8(C a) {
    typedef decltype(a.x) R;
    const R h = R(0.70710678118654752440084436210484904);
    return DIR < 0 ? C{(a.x + a.y) * h, (a.y - a.x) * h} : C{(a.x - a.y) * h, (a.y + a.x) * h};
}
// a * exp(DIR * i * 3pi/4) = a * (-1 + DIR i)/sqrt(2)
template <int DIR, typename C> __device__ __forceinline__ C mul_w8_3(C a) {
    typedef decltype(a.x) R;
    const R h = R(0.70710678118654752440084436210484904);
    return DIR < 0 ? C{(a.y - a.x) * h, -(a.x + a.y) * h} : C{-(a.x + a.y) * h, (a.x - a.y) * h};
}
// a * (c + DIR i s)
template <int DIR, typename C, typename R> __device__ __forceinline__ C mul_cs(C a, R c, R s) {
    return DIR < 0 ? C{a.x * c + a.y * s, a.y * c - a.x * s} : C{a.x * c - a.y * s, a.y * c + a.x * s};
}

// ------------------------------------------------------- small DFTs ------
// In-place R-point DFT with exponent sign DIR, natural order in and out,
// unscaled: X_k = sum_n x_n exp(DIR 2 pi i n k / R).
template <int DIR, typename C> __device__ __forceinline__ void dft2(C &a, C &b) {
    C t = a;
    a = cadd(t, b);
    b = csub(t, b);
}

template <int DIR, typename C> __device__ __forceinline__ void dft4(C &x0, C &x1, C &x2, C &x3) {
    C t0 = cadd(x0, x2), t1 = csub(x0, x2);
    C t2 = cadd(x1, x3), t3 = mul_diri<DIR>(csub(x1, x3));
    x0 = cadd(t0, t2);
    x2 = csub(t0, t2);
    x1 = cadd(t1, t3);
    x3 = csub(t1, t3);
}

template <int DIR, typename C> __device__ __forceinline__ void dft8(C *x) {
    // even / odd halves, then combine with W8^k
    C e0 = x[0], e1 = x[2], e2 = x[4], e3 = x[6];
    C o0 = x[1], o1 = x[3], o2 = x[5], o3 = x[7];
    dft4<DIR>(e0, e1, e2, e3);
    dft4<DIR>(o0, o1, o2, o3);
    o1 = mul_w8<DIR>(o1);
    o2 = mul_diri<DIR>(o2);
    o3 = mul_w8_3<DIR>(o3);
    x[0] = cadd(e0, o0);
    x[4] = csub(e0, o0);
    x[1] = cadd(e1, o1);
    x[5] = csub(e1, o1);
    x[2] = cadd(e2, o2);
    x[6] = csub(e2, o2);
    x[3] = cadd(e3, o3);
    x[7] = csub(e3, o3);
}

template <int DIR, typename C> __device__ __forceinline__ void dft16(C *x) {
    typedef decltype(x[0].x) R;
    const R c1 = R(0.92387953251128675612818318939678829);  // cos(pi/8)
    const R s1 = R(0.38268343236508977172845998403039887);  // sin(pi/8)
    // n = 4 n1 + n2, k = k1 + 4 k2: four 4-point DFTs over n1 ...
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) dft4<DIR>(x[n2], x[4 + n2], x[8 + n2], x[12 + n2]);
    // ... now x[4 k1 + n2] = Y[n2][k1]; multiply by W16^(n2 k1)
    x[5] = mul_cs<DIR>(x[5], c1, s1);     // n2=1,k1=1: W^1
    x[6] = mul_w8<DIR>(x[6]);             // n2=2,k1=1: W^2
    x[7] = mul_cs<DIR>(x[7], s1, c1);     // n2=3,k1=1: W^3
    x[9] = mul_w8<DIR>(x[9]);             // n2=1,k1=2: W^2
    x[10] = mul_diri<DIR>(x[10]);         // n2=2,k1=2: W^4
    x[11] = mul_w8_3<DIR>(x[11]);         // n2=3,k1=2: W^6
    x[13] = mul_cs<DIR>(x[13], s1, c1);   // n2=1,k1=3: W^3
    x[14] = mul_w8_3<DIR>(x[14]);         // n2=2,k1=3: W^6
    x[15] = mul_cs<DIR>(x[15], -c1, -s1); // n2=3,k1=3: W^9
    // ... then four 4-point DFTs over n2 for each k1
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) dft4<DIR>(x[4 * k1], x[4 * k1 + 1], x[4 * k1 + 2], x[4 * k1 + 3]);
    // x[4 k1 + k2] = X[k1 + 4 k2]: transpose the 4x4 index grid to natural order
    C t;
    t = x[1]; x[1] = x[4]; x[4] = t;
    t = x[2]; x[2] = x[8]; x[8] = t;
    t = x[3]; x[3] = x[12]; x[12] = t;
    t = x[6]; x[6] = x[9]; x[9] = t;
    t = x[7]; x[7] = x[13]; x[13] = t;
    t = x[11]; x[11] = x[14]; x[14] = t;
}

template <int R, int DIR, typename C> __device__ __forceinline__ void dft(C *a) {
    if constexpr (R == 1) {
    } else if constexpr (R == 2) {
        dft2<DIR>(a[0], a[1]);
    } else if constexpr (R == 4) {
        dft4<DIR>(a[0], a[1], a[2], a[3]);
    } else if constexpr (R == 8) {
        dft8<DIR>(a);
    } else {
        static_assert(R == 16, "radix");
        dft16<DIR>(a);
    }
}

template <typename C> __device__ __forceinline__ C ldg_c(const C *p) { return __ldg(p); }

// ------------------------------------------------------ host helpers ------
// Allow `smem` bytes of dynamic shared memory per block and, when `blocks` >
// 0, ask for a shared memory carve-out just large enough for that many blocks
// per SM; the rest of the SM's 256 KB stays L1 cache (twiddle tables are read
// through L1).  blocks = 0 leaves the carve-out to the driver.
inline cudaError_t set_smem_attrs(const void *kern, size_t smem, int blocks = 0) {
    cudaError_t e = cudaSuccess;
    if (smem > 48 * 1024) e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (blocks <= 0 || e != cudaSuccess) return e;
    const size_t need = (smem + 1024) * (size_t)blocks;  // 1 KB per block is reserved by the system
    const size_t max_sm = 228 * 1024;
    int pct = (int)((need * 100 + max_sm - 1) / max_sm);
    if (pct > 100) pct = 100;
    if (e == cudaSuccess) e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, pct);
    return e;
}

// ----------------------------------------------- asynchronous copies ------
// cp.async (global -> shared without a register round trip); `bytes` is 4, 8
// or 16 and both addresses must be aligned to it.
template <int BYTES>
__device__ __forceinline__ void cp_async(void *smem_dst, const void *gmem_src) {
    static_assert(BYTES == 4 || BYTES == 8 || BYTES == 16, "cp.async size");
    const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(smem_dst));
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(d), "l"(gmem_src), "n"(BYTES) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// ------------------------------------------------------- one pass ---------
// sm: this transform's exchange buffer, element x at sm[pad16(x) * S]
// (S > 1 interleaves S transforms element by element).
template <int N, int E, int R, int NS, int DIR, bool LAST, int PS, typename C>
__device__ __forceinline__ void stockham_pass(C (&v)[E], C *sm, const C *__restrict__ tw, int t, int S) {
    constexpr int T = N / E;
    constexpr int Q = E / R;
    static_assert(E % R == 0, "elements per thread must be a multiple of the radix");
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int j = t + q * T;
        C a[R];
#pragma unroll
        for (int r = 0; r < R; ++r) a[r] = v[q + r * Q];
        if constexpr (NS > 1) {
            const C *twp = tw + (NS - 1) + (j & (NS - 1));
            if constexpr (R == 16 && sizeof(C) == 8) {
                C w1[4], w4[4];  // W^q and W^(4q), q = 1..3
#pragma unroll
                for (int q = 1; q < 4; ++q) {
                    w1[q] = ldg_c(twp + (q - 1) * NS);
                    w4[q] = ldg_c(twp + (4 * q - 1) * NS);
                }
#pragma unroll
                for (int r = 1; r < R; ++r) {
                    const int qa = r & 3, qb = r >> 2;
                    const C w = qb == 0 ? w1[qa] : (qa == 0 ? w4[qb] : cmul(w1[qa], w4[qb]));
                    a[r] = DIR < 0 ? cmul(a[r], w) : cmulc(a[r], w);
                }
            } else {
#pragma unroll
                for (int r = 1; r < R; ++r) {
                    const C w = ldg_c(twp + (r - 1) * NS);
                    a[r] = DIR < 0 ? cmul(a[r], w) : cmulc(a[r], w);
                }
            }
        }
        dft<R, DIR>(a);
#pragma unroll
        for (int r = 0; r < R; ++r) v[q + r * Q] = a[r];
    }
    if constexpr (!LAST) {
        __syncthreads();  // the previous exchange's reads are complete
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const int j = t + q * T;
            const int base = (j / NS) * NS * R + (j & (NS - 1));
#pragma unroll
            for (int r = 0; r < R; ++r) sm[pad_ps<PS>(base + r * NS) * S] = v[q + r * Q];
        }
        __syncthreads();
#pragma unroll
        for (int e = 0; e < E; ++e) v[e] = sm[pad_ps<PS>(t + T * e) * S];
    }
}

template <int N, int E, int DIR, int P, int PS, typename C> struct Passes {
    __device__ __forceinline__ static void run(C (&v)[E], C *sm, const C *__restrict__ tw, int t, int S) {
        constexpr int NP = RadixPlan<N>::P;
        constexpr int R = RadixPlan<N>::radix(P);
        constexpr int NS = RadixPlan<N>::stride(P);
        stockham_pass<N, E, R, NS, DIR, P == NP - 1, PS>(v, sm, tw, t, S);
        if constexpr (P + 1 < NP) Passes<N, E, DIR, P + 1, PS, C>::run(v, sm, tw, t, S);
    }
};

// Full unscaled length-N DFT with exponent sign DIR on the registers of the
// T = N/E threads of one transform.  On entry and on exit v[e] is element /
// bin t + T*e.  All threads of the block must call it (it contains
// __syncthreads when N needs more than one pass).  Element x of the exchange
// buffer is sm[pad_ps<PS>(x) * S]; S > 1 interleaves S transforms.
template <int N, int E, int DIR, int PS = 4, typename C>
__device__ __forceinline__ void fft_regs(C (&v)[E], C *sm, const C *__restrict__ tw, int t, int S = 1) {
    static_assert(N % E == 0 && E >= RadixPlan<N>::MAXR, "bad elements per thread");
    Passes<N, E, DIR, 0, PS, C>::run(v, sm, tw, t, S);
}

}  // namespace gbfft
