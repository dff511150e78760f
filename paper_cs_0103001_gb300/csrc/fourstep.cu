// fourstep.cu — batched 1D transforms longer than one thread block can hold.
//
// The paper splits the radix-2 tree of a length-N transform between 2^l
// processes (Sec. 2): each owns a subtree up to level m1 = m - l, and the
// upper levels combine the partial transforms.  On one GPU the same split is
// made along index bits, N = N1 * N2 (the "four-step" factorisation):
//   j = j1 N2 + j2,  k = k1 + N1 k2,
//   X[k1 + N1 k2] = sum_j2 W_N2^(j2 k2) [ W_N^(j2 k1) sum_j1 x[j1 N2 + j2] W_N1^(j1 k1) ].
// Pass A runs the inner length-N1 transforms down the columns j2 of the
// N1 x N2 row-major view and multiplies by W_N^(j2 k1).  A thread holds rows
// k1 = t + T e (T = N1/16, e < 16) of one column j2, so the factor splits as
// W_N^(t j2) (once per thread, from the two-level table) times
// W_N^(T e j2) = W_(16 N2)^(e j2) (a 16 x N2 table read along j2: adjacent
// threads read adjacent entries);
// pass B runs the outer length-N2 transforms along the rows k1 and stores
// bin k2 of row k1 at k1 + N1 k2, the natural order of X.  Both passes move a
// tile of W adjacent columns (pass A) or rows (pass B) per thread block so
// every global access is a run of W or 32/W contiguous elements.  The
// intermediate goes to a workspace chunk sized to stay in L2 when it can.
#include <cuda.h>

#include "fft_core.cuh"
#include "check.cuh"
#include "internal.h"
#include "tma.cuh"

#ifndef GBFFT_FS_BIGN
#define GBFFT_FS_BIGN 4096  // fp32 factor lengths from which a block has 1024 threads
#endif

namespace gbfft {

template <int N, typename R> struct FsCfg {
    // blocks per SM the register budget is sized for: 64 registers per thread
    // hold an fp32 transform's 16 elements; fp64 needs twice as many
    // threads per block at most: 1024 for long fp32 factors, so that a tile
    // spans at least four columns (32-byte runs); 512 otherwise (two blocks per SM)
    static constexpr int MAXT = sizeof(R) == 4 && N >= GBFFT_FS_BIGN ? 1024 : 512;
    static constexpr int MINB = sizeof(R) == 4 && MAXT <= 512 ? 2 : 1;
    static constexpr int E = N < 16 ? N : 16;
    static constexpr int T = N / E;
    static constexpr int SMEM_ELEMS = (sizeof(R) == 4 ? 16384 : 8192);
    static constexpr int W0 = SMEM_ELEMS / N < MAXT / T ? SMEM_ELEMS / N : MAXT / T;
    static constexpr int WMAX = W0 > 64 ? 64 : (W0 < 1 ? 1 : W0);
    // exchange layout of the WMAX interleaved transforms (fft_core.cuh)
    static constexpr int PS = exch_pad_shift<typename cvec<R>::type>(N, WMAX);
    static constexpr int PL = padded_len_ps<PS>(N);
};

// Shared memory of k_fourstep_b_tma: the input tile (W rows of pitch N + 2),
// the exchange buffer and the output box share one region.
template <int N> struct FsTmaB {
    typedef FsCfg<N, float> K;
    static constexpr size_t TILE = (size_t)K::WMAX * (N + 2), EXCH = (size_t)K::PL * K::WMAX;
    static constexpr size_t REGION_BYTES = (TILE > EXCH ? TILE : EXCH) * sizeof(float2);
    static constexpr size_t SMEM = REGION_BYTES + 16 + 128;  // + mbarrier and flag, + alignment slack
};

int fourstep_split(int log2n, bool dbl, int *log2n1, int *log2n2) {
    (void)dbl;
    *log2n1 = log2n / 2;
    *log2n2 = log2n - log2n / 2;
    return 0;
}

// W_N^idx (forward sign) from the two-level table: fine W_N^b, b < F; coarse W_N^(aF).
template <typename C>
__device__ __forceinline__ C tw_two_level(const C *__restrict__ t4, int idx, int log2f) {
    const int f = 1 << log2f;
    const C lo = __ldg(t4 + (idx & (f - 1)));
    const C hi = __ldg(t4 + f + (idx >> log2f));
    return cmul(hi, lo);
}

// Row k1 of pass B's input: row k1 itself (log2p = 0), or, for the last
// pass of a three-pass split, row (k1 mod P) (n1 / P) + k1 / P (P = 2^log2p):
// the middle pass leaves its rows in the order [k1'][k2'] with k1' < P, and
// the output index wants k1 = k1' + P k2'.
__device__ __forceinline__ size_t perm_row(int k1, int log2n1, int log2p) {
    if (log2p == 0) return (size_t)k1;
    return ((size_t)(k1 & ((1 << log2p) - 1)) << (log2n1 - log2p)) + (size_t)(k1 >> log2p);
}

// Pass A: column transforms of length N1 (= N) over the N1 x n2 view.
template <int N, int DIR, typename R>
__global__ void __launch_bounds__(FsCfg<N, R>::MAXT, FsCfg<N, R>::MINB)
    k_fourstep_a(const typename cvec<R>::type *in, typename cvec<R>::type *tmp, int log2n2,
                 const typename cvec<R>::type *__restrict__ tw, const typename cvec<R>::type *__restrict__ t4,
                 int log2f, const typename cvec<R>::type *__restrict__ t5) {
    typedef typename cvec<R>::type C;
    typedef FsCfg<N, R> K;
    constexpr int E = K::E, T = K::T, W = K::WMAX;
    extern __shared__ __align__(16) unsigned char smraw[];
    C *sm = reinterpret_cast<C *>(smraw);
    const int w = threadIdx.x % W;
    const int t = threadIdx.x / W;
    const int j2 = blockIdx.x * W + w;
    const size_t base = (size_t)blockIdx.y * ((size_t)N << log2n2) + j2;
    C v[E];
#pragma unroll
    for (int e = 0; e < E; ++e) v[e] = in[base + ((size_t)(t + T * e) << log2n2)];
    fft_regs<N, E, DIR, K::PS>(v, sm + w, tw, t, W);
    static_assert(E == 16, "rows t + T e with T = N1 / 16");
    const C a = tw_two_level(t4, t * j2, log2f);  // W_N^(t j2), t j2 < N / 16
    const C *t5j = t5 + j2;
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int k1 = t + T * e;
        const C f = cmul(a, __ldg(t5j + ((size_t)e << log2n2)));  // W_N^(k1 j2)
        v[e] = DIR < 0 ? cmul(v[e], f) : cmulc(v[e], f);
        tmp[base + ((size_t)k1 << log2n2)] = v[e];
    }
}

// Pass A for complex64 with its tile moved by the TMA: one thread loads the
// block's N1 x W tile (W adjacent columns, row pitch n2) as boxes of up to
// 256 rows into shared memory; the block waits on an mbarrier (bounded: a
// wait that gives up sets *status and the block leaves), reads its elements
// from the dense tile, and the transform reuses the same memory as its
// exchange buffer.  Twiddle as k_fourstep_a; with TSTORE the results go back
// into the dense tile and leave by tensor stores through tmap (the same
// geometry over the intermediate), else by plain stores.
template <int N, int DIR, bool TSTORE>
__global__ void __launch_bounds__(FsCfg<N, float>::MAXT, FsCfg<N, float>::MINB)
    k_fourstep_a_tma(const __grid_constant__ CUtensorMap map, const __grid_constant__ CUtensorMap tmap, float2 *tmp,
                     int log2n2, const float2 *__restrict__ tw, const float2 *__restrict__ t4, int log2f,
                     const float2 *__restrict__ t5, int *status) {
    typedef FsCfg<N, float> K;
    constexpr int E = K::E, T = K::T, W = K::WMAX, BR = N < 256 ? N : 256;
    constexpr size_t EXCH_BYTES = (size_t)K::PL * W * sizeof(float2);
    extern __shared__ __align__(128) unsigned char smraw[];
    unsigned char *base = smraw + ((128u - (smem_u32(smraw) & 127u)) & 127u);  // TMA wants 128-byte alignment
    float2 *sm = reinterpret_cast<float2 *>(base);
    uint64_t *bar = reinterpret_cast<uint64_t *>(base + EXCH_BYTES);
    int *ok = reinterpret_cast<int *>(base + EXCH_BYTES + 8);
    const int w = threadIdx.x % W;
    const int t = threadIdx.x / W;
    const int j2 = blockIdx.x * W + w;
    // checked build: the block's W columns inside n2 (uniform per block)
    if (!chk((blockIdx.x + 1) * W <= (1 << log2n2), CK_FS_A_TILE)) return;
    if (threadIdx.x == 0) mbar_init(bar, 1);
    __syncthreads();
    if (threadIdx.x == 0) {
        mbar_expect_tx(bar, (uint32_t)(N * W * sizeof(float2)));
        for (int r = 0; r < N; r += BR) tma_load_3d(sm + r * W, &map, 2 * blockIdx.x * W, r, blockIdx.y, bar);
        int done = mbar_wait_bounded(bar, 0, kTmaPolls) ? 1 : 0;
        if (!done) {
            atomicExch(status, 1);
            mbar_wait_bounded(bar, 0, kTmaPolls);  // one more bounded wait for the copies in flight
        }
        *ok = done;
    }
    __syncthreads();
    if (!*ok) return;  // uniform per block
    const size_t base_g = (size_t)blockIdx.y * ((size_t)N << log2n2) + j2;
    float2 v[E];
#pragma unroll
    for (int e = 0; e < E; ++e) v[e] = sm[(t + T * e) * W + w];
    // fft_regs starts its first exchange with a block barrier, after every
    // thread read its elements from the tile
    static_assert(RadixPlan<N>::P >= 2, "at least one exchange");
    fft_regs<N, E, DIR, K::PS>(v, sm + w, tw, t, W);
    static_assert(E == 16, "rows t + T e with T = N1 / 16");
    const float2 a = tw_two_level(t4, t * j2, log2f);
    const float2 *t5j = t5 + j2;
    if constexpr (TSTORE) __syncthreads();  // the last exchange's reads are complete
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int k1 = t + T * e;
        const float2 f = cmul(a, __ldg(t5j + ((size_t)e << log2n2)));
        v[e] = DIR < 0 ? cmul(v[e], f) : cmulc(v[e], f);
        if constexpr (TSTORE)
            sm[k1 * W + w] = v[e];
        else
            tmp[base_g + ((size_t)k1 << log2n2)] = v[e];
    }
    if constexpr (TSTORE) {
        fence_async_smem();
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int r = 0; r < N; r += BR) tma_store_3d(&tmap, 2 * blockIdx.x * W, r, blockIdx.y, sm + r * W);
            bulk_commit();
            bulk_wait_read();
        }
    }
}

// Pass B: row transforms of length N2 (= N) over the n1 x N2 view, stored at k1 + n1 k2.
template <int N, int DIR, typename R>
__global__ void __launch_bounds__(FsCfg<N, R>::MAXT, FsCfg<N, R>::MINB)
    k_fourstep_b(const typename cvec<R>::type *tmp, typename cvec<R>::type *out, int log2n1,
                 const typename cvec<R>::type *__restrict__ tw, R scale, int log2p) {
    typedef typename cvec<R>::type C;
    typedef FsCfg<N, R> K;
    constexpr int E = K::E, T = K::T, W = K::WMAX;
    extern __shared__ __align__(16) unsigned char smraw[];
    C *sm = reinterpret_cast<C *>(smraw);
    const int w = threadIdx.x % W;
    const int t = threadIdx.x / W;
    const int k1 = blockIdx.x * W + w;
    const size_t img = (size_t)blockIdx.y * ((size_t)N << log2n1);
    const C *row = tmp + img + (size_t)perm_row(k1, log2n1, log2p) * N;
    C v[E];
#pragma unroll
    for (int e = 0; e < E; ++e) v[e] = row[t + T * e];
    fft_regs<N, E, DIR, K::PS>(v, sm + w, tw, t, W);
    C *dst = out + img + k1;
#pragma unroll
    for (int e = 0; e < E; ++e) dst[(size_t)(t + T * e) << log2n1] = cscale(v[e], scale);
}

// Pass B for complex64 through the TMA: the block's W rows k1 (contiguous in
// the intermediate) arrive by bulk copies into rows of pitch N + 2 (so the
// W threads that read one column of the tile hit different banks), with a
// bounded mbarrier wait as in k_fourstep_a_tma; the transform reuses the
// memory as its exchange buffer; the scaled outputs go back into it as the
// dense box [k2][W] (W adjacent k1 of every row k2 of the n1-wide output
// view) and leave by tensor stores.
template <int N, int DIR>
__global__ void __launch_bounds__(FsCfg<N, float>::MAXT, FsCfg<N, float>::MINB)
    k_fourstep_b_tma(const float2 *tmp, const __grid_constant__ CUtensorMap omap, int log2n1,
                     const float2 *__restrict__ tw, float scale, int *status, int log2p) {
    typedef FsCfg<N, float> K;
    constexpr int E = K::E, T = K::T, W = K::WMAX, BR = N < 256 ? N : 256, RP = N + 2;
    extern __shared__ __align__(128) unsigned char smraw[];
    unsigned char *base = smraw + ((128u - (smem_u32(smraw) & 127u)) & 127u);
    float2 *sm = reinterpret_cast<float2 *>(base);
    uint64_t *bar = reinterpret_cast<uint64_t *>(base + FsTmaB<N>::REGION_BYTES);
    int *ok = reinterpret_cast<int *>(base + FsTmaB<N>::REGION_BYTES + 8);
    const int w = threadIdx.x % W;
    const int t = threadIdx.x / W;
    const int k10 = blockIdx.x * W;
    // checked build: the block's W rows inside n1 (uniform per block)
    if (!chk(k10 + W <= (1 << log2n1), CK_FS_B_ROWS)) return;
    if (threadIdx.x == 0) mbar_init(bar, 1);
    __syncthreads();
    if (threadIdx.x == 0) {
        mbar_expect_tx(bar, (uint32_t)(N * W * sizeof(float2)));
        const float2 *src = tmp + (size_t)blockIdx.y * ((size_t)N << log2n1);
        for (int r = 0; r < W; ++r)
            bulk_load(sm + r * RP, src + (size_t)perm_row(k10 + r, log2n1, log2p) * N, N * sizeof(float2), bar);
        int done = mbar_wait_bounded(bar, 0, kTmaPolls) ? 1 : 0;
        if (!done) {
            atomicExch(status, 1);
            mbar_wait_bounded(bar, 0, kTmaPolls);  // one more bounded wait for the copies in flight
        }
        *ok = done;
    }
    __syncthreads();
    if (!*ok) return;  // uniform per block
    float2 v[E];
#pragma unroll
    for (int e = 0; e < E; ++e) v[e] = sm[w * RP + t + T * e];
    static_assert(RadixPlan<N>::P >= 2, "at least one exchange");
    fft_regs<N, E, DIR, K::PS>(v, sm + w, tw, t, W);
    __syncthreads();  // the last exchange's reads are complete
#pragma unroll
    for (int e = 0; e < E; ++e) sm[(t + T * e) * W + w] = cscale(v[e], scale);
    fence_async_smem();
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int r = 0; r < N; r += BR) tma_store_3d(&omap, 2 * k10, r, blockIdx.y, sm + r * W);
        bulk_commit();
        bulk_wait_read();
    }
}

cudaError_t check_take_fourstep(unsigned out[2]) { return check_word_take(out); }

template <int N, typename R>
static cudaError_t run_a_tma(const void *in, void *tmp, int log2n2, long long nb, int dir, const void *tw,
                             const void *t4, int log2f, const void *t5, int *status, cudaStream_t s, bool *used) {
    *used = false;
    if constexpr (sizeof(R) != 4) {
        return cudaSuccess;
    } else {
        typedef FsCfg<N, float> K;
        constexpr int W = K::WMAX, BR = N < 256 ? N : 256;
        const EncodeTiledFn enc = encode_tiled();
        if (!enc || !status) return cudaSuccess;
        // the chunk as a 3D float tensor: {2 n2 (re, im of each column), N1 rows, nb transforms}
        const cuuint64_t n2 = 1ull << log2n2;
        cuuint64_t dims[3] = {2 * n2, (cuuint64_t)N, (cuuint64_t)nb};
        cuuint64_t strides[2] = {2 * n2 * sizeof(float), (cuuint64_t)N * 2 * n2 * sizeof(float)};
        cuuint32_t box[3] = {2 * W, BR, 1};
        cuuint32_t estr[3] = {1, 1, 1};
        CUtensorMap map, tmap;
        if (enc(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void *>(in), dims, strides, box, estr,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS ||
            enc(&tmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, tmp, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaSuccess;  // not encodable here: the caller runs the plain kernel
        const size_t smem = (size_t)K::PL * W * sizeof(float2) + 16 + 128;
        // tensor stores when two blocks share an SM: the block holds its shared
        // memory until the stores have read it, and the other block covers that
        auto kern = K::MINB >= 2 ? (dir < 0 ? k_fourstep_a_tma<N, -1, true> : k_fourstep_a_tma<N, 1, true>)
                                 : (dir < 0 ? k_fourstep_a_tma<N, -1, false> : k_fourstep_a_tma<N, 1, false>);
        cudaError_t e = set_smem_attrs((const void *)kern, smem, K::MINB);
        if (e != cudaSuccess) return e;
        dim3 grid((1 << log2n2) / W, (unsigned)nb);
        kern<<<grid, W * K::T, smem, s>>>(map, tmap, static_cast<float2 *>(tmp), log2n2, static_cast<const float2 *>(tw),
                                          static_cast<const float2 *>(t4), log2f, static_cast<const float2 *>(t5),
                                          status);
        *used = true;
        return cudaGetLastError();
    }
}

template <int N, typename R>
static cudaError_t run_a(const void *in, void *tmp, int log2n2, long long nb, int dir, const void *tw,
                         const void *t4, int log2f, const void *t5, int *status, cudaStream_t s) {
    if (nb > 65535) return cudaErrorInvalidConfiguration;
    bool used = false;
    cudaError_t te = run_a_tma<N, R>(in, tmp, log2n2, nb, dir, tw, t4, log2f, t5, status, s, &used);
    if (te != cudaSuccess || used) return te;
    typedef typename cvec<R>::type C;
    typedef FsCfg<N, R> K;
    constexpr int W = K::WMAX;  // <= 64 <= the other factor (>= 2^7)
    const size_t smem = (size_t)K::PL * W * sizeof(C);
    auto kern = dir < 0 ? k_fourstep_a<N, -1, R> : k_fourstep_a<N, 1, R>;
    cudaError_t e = set_smem_attrs((const void *)kern, smem, K::MINB);
    if (e != cudaSuccess) return e;
    if (nb > 65535) return cudaErrorInvalidConfiguration;
    dim3 grid((1 << log2n2) / W, (unsigned)nb);
    kern<<<grid, W * K::T, smem, s>>>(static_cast<const C *>(in), static_cast<C *>(tmp), log2n2,
                                      static_cast<const C *>(tw), static_cast<const C *>(t4), log2f,
                                      static_cast<const C *>(t5));
    return cudaGetLastError();
}

template <int N, typename R>
static cudaError_t run_b_tma(const void *tmp, void *out, int log2n1, long long nb, int dir, const void *tw,
                             double scale, int *status, cudaStream_t s, bool *used, int log2p) {
    *used = false;
    if constexpr (sizeof(R) != 4 || FsCfg<N, float>::MINB < 2) {
        // one block per SM: it would idle while its tensor stores drain
        return cudaSuccess;
    } else {
        typedef FsCfg<N, float> K;
        constexpr int W = K::WMAX, BR = N < 256 ? N : 256;
        const EncodeTiledFn enc = encode_tiled();
        if (!enc || !status) return cudaSuccess;
        // the output as a 3D float tensor: {2 n1 (re, im of each k1), N rows k2, nb transforms}
        const cuuint64_t n1 = 1ull << log2n1;
        cuuint64_t dims[3] = {2 * n1, (cuuint64_t)N, (cuuint64_t)nb};
        cuuint64_t strides[2] = {2 * n1 * sizeof(float), (cuuint64_t)N * 2 * n1 * sizeof(float)};
        cuuint32_t box[3] = {2 * W, BR, 1};
        cuuint32_t estr[3] = {1, 1, 1};
        CUtensorMap map;
        if (enc(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, out, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaSuccess;  // not encodable here: the caller runs the plain kernel
        const size_t smem = FsTmaB<N>::SMEM;
        auto kern = dir < 0 ? k_fourstep_b_tma<N, -1> : k_fourstep_b_tma<N, 1>;
        cudaError_t e = set_smem_attrs((const void *)kern, smem, K::MINB);
        if (e != cudaSuccess) return e;
        dim3 grid((unsigned)(n1 / W), (unsigned)nb);
        kern<<<grid, W * K::T, smem, s>>>(static_cast<const float2 *>(tmp), map, log2n1,
                                          static_cast<const float2 *>(tw), (float)scale, status, log2p);
        *used = true;
        return cudaGetLastError();
    }
}

template <int N, typename R>
static cudaError_t run_b(const void *tmp, void *out, int log2n1, long long nb, int dir, const void *tw, double scale,
                         int *status, cudaStream_t s, int log2p) {
    if (nb > 65535) return cudaErrorInvalidConfiguration;
    bool used = false;
    cudaError_t te = run_b_tma<N, R>(tmp, out, log2n1, nb, dir, tw, scale, status, s, &used, log2p);
    if (te != cudaSuccess || used) return te;
    typedef typename cvec<R>::type C;
    typedef FsCfg<N, R> K;
    constexpr int W = K::WMAX;  // <= 64 <= the other factor (>= 2^7)
    const size_t smem = (size_t)K::PL * W * sizeof(C);
    auto kern = dir < 0 ? k_fourstep_b<N, -1, R> : k_fourstep_b<N, 1, R>;
    cudaError_t e = set_smem_attrs((const void *)kern, smem, K::MINB);
    if (e != cudaSuccess) return e;
    if (nb > 65535) return cudaErrorInvalidConfiguration;
    dim3 grid((1 << log2n1) / W, (unsigned)nb);
    kern<<<grid, W * K::T, smem, s>>>(static_cast<const C *>(tmp), static_cast<C *>(out), log2n1,
                                      static_cast<const C *>(tw), (R)scale, log2p);
    return cudaGetLastError();
}

// Factor lengths that occur for 2^14 <= N <= 2^24: 2^7 .. 2^12.
#define GBFFT_FS_CASES(X) X(7) X(8) X(9) X(10) X(11) X(12)

template <typename R>
static cudaError_t dispatch_a(const void *in, void *tmp, int l1, int l2, long long nb, int dir, const void *tw,
                              const void *t4, int log2f, const void *t5, int *status, cudaStream_t s) {
    switch (l1) {
#define GBFFT_A(L) \
    case L: return run_a<(1 << L), R>(in, tmp, l2, nb, dir, tw, t4, log2f, t5, status, s);
        GBFFT_FS_CASES(GBFFT_A)
#undef GBFFT_A
        default: return cudaErrorInvalidValue;
    }
}

template <typename R>
static cudaError_t dispatch_b(const void *tmp, void *out, int l1, int l2, long long nb, int dir, const void *tw,
                              double scale, int *status, cudaStream_t s, int log2p) {
    switch (l2) {
#define GBFFT_B(L) \
    case L: return run_b<(1 << L), R>(tmp, out, l1, nb, dir, tw, scale, status, s, log2p);
        GBFFT_FS_CASES(GBFFT_B)
#undef GBFFT_B
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_fourstep_a(const void *in, void *tmp, int log2n, long long batch, bool dbl, int dir,
                              const void *tw_n1, const void *tw_4s, const void *tw_coarse, int *status,
                              cudaStream_t s) {
    int l1, l2;
    fourstep_split(log2n, dbl, &l1, &l2);
    const int log2f = (log2n + 1) / 2;
    return dbl ? dispatch_a<double>(in, tmp, l1, l2, batch, dir, tw_n1, tw_4s, log2f, tw_coarse, status, s)
               : dispatch_a<float>(in, tmp, l1, l2, batch, dir, tw_n1, tw_4s, log2f, tw_coarse, status, s);
}

cudaError_t launch_fourstep_b(const void *tmp, void *out, int log2n, long long batch, bool dbl, int dir,
                              const void *tw_n2, double scale, int *status, cudaStream_t s) {
    int l1, l2;
    fourstep_split(log2n, dbl, &l1, &l2);
    return dbl ? dispatch_b<double>(tmp, out, l1, l2, batch, dir, tw_n2, scale, status, s, 0)
               : dispatch_b<float>(tmp, out, l1, l2, batch, dir, tw_n2, scale, status, s, 0);
}

cudaError_t launch_fourstep_a_split(const void *in, void *tmp, int log2n1, int log2n2, long long batch, int dir,
                                    const void *tw_n1, const void *tw_4s, const void *tw_coarse, int *status,
                                    cudaStream_t s) {
    const int log2f = (log2n1 + log2n2 + 1) / 2;
    return dispatch_a<float>(in, tmp, log2n1, log2n2, batch, dir, tw_n1, tw_4s, log2f, tw_coarse, status, s);
}

cudaError_t launch_fourstep_b_split(const void *tmp, void *out, int log2n1, int log2n2, int log2p, long long batch,
                                    int dir, const void *tw_n2, double scale, int *status, cudaStream_t s) {
    return dispatch_b<float>(tmp, out, log2n1, log2n2, batch, dir, tw_n2, scale, status, s, log2p);
}

}  // namespace gbfft
