// cols.cu — launcher of the fused column pass of the Sec. 5 pipeline; the
// kernel body and the description of the method live in cols_impl.cuh.
#include <cmath>

#include "cols_impl.cuh"
#include "internal.h"
#include "tma.cuh"

namespace gbfft {

template <int N>
__global__ void __launch_bounds__(ColCfg<N>::THREADS, 2)
    k_cols_filter(float2 *spec, const float *__restrict__ hs, const float *__restrict__ beta, long long hs_img,
                  long long beta_img, int M, int log2g, const float2 *__restrict__ tw, ColSlab cs) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const size_t y = blockIdx.y;
    cols_body<N>(spec + y * (M / 2) * N, PreparedFilter{hs + y * hs_img, beta + y * beta_img, N}, M, log2g, tw,
                 blockIdx.x, smraw, Fp32Fft(), cs);
}

// The column pass with an analytic filter (cols_impl.cuh) computed in place.
template <int N>
__global__ void __launch_bounds__(ColCfg<N>::THREADS, 2)
    k_cols_analytic(float2 *spec, AnalyticFilter filt, int M, int log2g, const float2 *__restrict__ tw) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const size_t y = blockIdx.y;
    cols_body<N>(spec + y * (M / 2) * N, filt, M, log2g, tw, blockIdx.x, smraw);
}

// Spectrum display (Sec. 5): the column FFTs of the row half spectra, and
// scale * sqrt(Re^2 + Im^2) of every bin in slot order.  The packed column 0
// (DC in re, Nyquist in im) splits into its two real-column spectra
// P = (Q + conj Q[-u]) / 2 (the DC column) and R = (Q - conj Q[-u]) / (2i)
// (the Nyquist column, written to nyq).
template <int N>
__global__ void __launch_bounds__(ColCfg<N>::THREADS)
    k_cols_spectrum(const float2 *__restrict__ spec, float *__restrict__ mag_T, float *__restrict__ nyq, float scale,
                    int M, int log2g, const float2 *__restrict__ tw) {
    typedef ColCfg<N> K;
    constexpr int E = K::E, T = K::T, W = K::W;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int w = threadIdx.x / T;
    const int t = threadIdx.x - w * T;
    float2 *ex = reinterpret_cast<float2 *>(smraw) + w * padded_len(N);
    const int k0 = blockIdx.x * W + w;
    const bool active = k0 < (M >> 1);
    const int k = active ? k0 : 0;
    const float2 *col = spec + (size_t)k * N;
    float2 v[E];
#pragma unroll
    for (int e = 0; e < E; ++e) v[e] = active ? col[slot_e<N, E, T>(t, e, log2g)] : make_float2(0.f, 0.f);
    fft_regs<N, E, -1>(v, ex, tw, t);
    if (blockIdx.x == 0) {  // the group of column 0 needs Q[-u] (uniform per block)
        __syncthreads();
#pragma unroll
        for (int e = 0; e < E; ++e) ex[pad16(t + T * e)] = v[e];
        __syncthreads();
    }
    if (!active) return;  // no barrier follows
    float *mcol = mag_T + (size_t)k * N;
    if (k != 0) {
#pragma unroll
        for (int e = 0; e < E; ++e)
            mcol[slot_e<N, E, T>(t, e, log2g)] = scale * sqrtf(v[e].x * v[e].x + v[e].y * v[e].y);
    } else {
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const float2 q = v[e], qm = ex[pad16((N - (t + T * e)) & (N - 1))];
            const float px = 0.5f * (q.x + qm.x), py = 0.5f * (q.y - qm.y);
            const float rx = 0.5f * (q.y + qm.y), ry = 0.5f * (qm.x - q.x);
            const int sl = slot_e<N, E, T>(t, e, log2g);
            mcol[sl] = scale * sqrtf(px * px + py * py);
            nyq[sl] = scale * sqrtf(rx * rx + ry * ry);
        }
    }
}

template <int N>
static cudaError_t run_spectrum(const void *spec, float *mag_T, float *nyq, float scale, int cols, int log2g,
                                const void *tw, cudaStream_t s) {
    typedef ColCfg<N> K;
    cudaError_t e = set_smem_attrs((const void *)k_cols_spectrum<N>, K::SMEM);
    if (e != cudaSuccess) return e;
    dim3 grid((cols / 2 + K::W - 1) / K::W);
    k_cols_spectrum<N><<<grid, K::THREADS, K::SMEM, s>>>(static_cast<const float2 *>(spec), mag_T, nyq, scale, cols,
                                                         log2g, static_cast<const float2 *>(tw));
    return cudaGetLastError();
}

cudaError_t launch_cols_spectrum(const void *spec, float *mag_T, float *nyq, float scale, int rows, int cols,
                                 const void *tw_rows, cudaStream_t s) {
    int g = rows_pairs_per_block(cols);
    if (g > rows / 2) g = rows / 2;
    const int log2g = ilog2(g);
    switch (ilog2(rows)) {
#define GBFFT_CASE(L) \
    case L: return run_spectrum<(1 << L)>(spec, mag_T, nyq, scale, cols, log2g, tw_rows, s);
        GBFFT_CASE(1) GBFFT_CASE(2) GBFFT_CASE(3) GBFFT_CASE(4) GBFFT_CASE(5) GBFFT_CASE(6) GBFFT_CASE(7)
        GBFFT_CASE(8) GBFFT_CASE(9) GBFFT_CASE(10) GBFFT_CASE(11) GBFFT_CASE(12) GBFFT_CASE(13)
#undef GBFFT_CASE
        default: return cudaErrorInvalidValue;
    }
}

// ---- The column pass through the TMA (columns of 4096 rows: 256 threads per
// column, one column per block at a time; taller columns use the
// one-column-per-block kernel).  A column's N slots (contiguous, slot order) are viewed
// as N/16 rows of 128 bytes and move as 2D tensor boxes with the 128-byte
// swizzle (the 16-byte chunk c of row r sits at chunk c ^ (r mod 8)), which
// keeps the threads' slot-order reads and writes free of bank conflicts; the
// prepared filter column arrives by a bulk copy.  Each block is persistent:
// while it transforms one column in one buffer, the next column and its
// filter are already loading into the other (one mbarrier per buffer,
// bounded waits as in fourstep.cu).  Results go back into the buffer in the
// swizzled slot layout and leave by tensor stores; before a buffer is
// reloaded, its stores must have read it.  The arithmetic is cols_body's.
// A column of a decomposed image (layout.cuh, ColSlab) arrives in `nchunk`
// runs of `crows` rows, run q at row q * cstride + c * crows (one image); the
// runs land back to back in the buffer, so the slot order in shared memory is
// the same.  One image: nchunk = 1, crows = N/16.
// Two forms: the filter column bulk-copied beside its column (GF = false),
// or read from global memory (L2) after the forward transform (GF = true),
// which leaves more of the SM's memory to the L1 cache.  Two blocks per SM
// (BL): a third needs 80 registers per thread and spills (73 against 45 us at
// 4096^2, measured), so it is not offered.
template <int N, bool GF = false, int BL = 2> struct ColTmaCfg {
    typedef ColCfg<N> C;
    static constexpr int E = C::E, T = C::T, THREADS = C::THREADS;
    static_assert(C::W == 1 && T >= 64, "one column per block, slot rows aligned to the swizzle");
    static constexpr int ROWS = N / 16;
    static constexpr int BLOCKS = BL;  // per SM
    static constexpr size_t BUF = ((size_t)padded_len(N) * sizeof(float2) + 1023) / 1024 * 1024;
    static constexpr size_t FB = GF ? 0 : (size_t)N * sizeof(float);
    static constexpr size_t SMEM = 1024 + 2 * BUF + 2 * FB + 32;  // alignment slack, buffers, 2 mbarriers
};

// float2 index of slot s in a column tile stored with the 128-byte swizzle
__device__ __forceinline__ int swz128(int s) {
    const int row = s >> 4;
    return (row << 4) + ((((s >> 1) & 7) ^ (row & 7)) << 1) + (s & 1);
}

// One column of k_cols_filter_tma in buffer b (its copies complete), from the
// slot reads to the issue of its tensor stores.  Out of line: compiled on its
// own, so nothing of one column (twiddles, addresses) is kept in registers
// across the loop over columns.
template <int N, bool GF, int BL>
__device__ __noinline__ void cols_tma_column(const CUtensorMap *map, float2 *bf, const float *h,
                                             const float *bt, long long c, bool col0, bool prefetch, int b,
                                             const float2 *__restrict__ tw, int log2g, unsigned char *base,
                                             const float *hs, long long hs_img, int log2half, int crows,
                                             int boxr, long long cstride, int nchunk, long long nrows) {
    typedef ColTmaCfg<N, GF, BL> K;
    constexpr int E = K::E, T = K::T;
    const int t = threadIdx.x;
    const int G = 1 << log2g;
    // slots of rows t + T e (layout.cuh), affine in e because G divides T:
    // side 0 (e < E/2): b0 + 2 T e; side 1: b1 + 2 T (E - 1 - e), except row
    // N/2 (t = 0, e = E/2) in slot G.  2 T is a whole number of 8-row swizzle
    // blocks, so the swizzled index is affine in e as well.
    const int b0 = ((t >> log2g) << (log2g + 1)) + (t & (G - 1));
    const int b1 = (((-t) >> log2g) << (log2g + 1)) + G + ((-t) & (G - 1)) + 2 * T;
    const int i0 = swz128(b0), i1 = swz128(b1), ig = swz128(G);
    auto sidx = [&](int e) { return e < E / 2 ? i0 + 2 * T * e : (e == E / 2 && t == 0 ? ig : i1 + 2 * T * (E - 1 - e)); };
    float2 v[E];
#pragma unroll
    for (int e = 0; e < E; ++e) v[e] = bf[sidx(e)];
    if (prefetch && t == 0) {  // the next column and its filter into the other buffer
        const long long cn = c + gridDim.x;
        float2 *nb = reinterpret_cast<float2 *>(base + (b ^ 1) * K::BUF);
        float *nf = reinterpret_cast<float *>(base + 2 * K::BUF + (b ^ 1) * K::FB);
        uint64_t *bar = reinterpret_cast<uint64_t *>(base + 2 * K::BUF + 2 * K::FB) + (b ^ 1);
        bulk_wait_read();  // the other buffer's stores have read it
        mbar_expect_tx(bar, (uint32_t)(N * sizeof(float2) + K::FB));
        for (int q = 0; q < nchunk; ++q)
            for (int r = 0; r < crows; r += boxr)
                if (chk(q * cstride + cn * crows + r + boxr <= nrows, CK_COL_BOX))
                    tma_load_2d(nb + (q * crows + r) * 16, map, 0, (int)(q * cstride + cn * crows + r), bar);
        if constexpr (!GF)
            bulk_load(nf, hs + (cn >> log2half) * hs_img + (cn & ((1LL << log2half) - 1)) * N, N * sizeof(float),
                      bar);
    }
    // the first exchange starts with a block barrier: every thread has read
    // its slots before the buffer becomes the exchange buffer
    fft_regs<N, E, -1>(v, bf, tw, t);
    if (col0) {  // column 0 needs Q[-u] (uniform per block)
        __syncthreads();
#pragma unroll
        for (int e = 0; e < E; ++e) bf[pad16(t + T * e)] = v[e];
        __syncthreads();
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int u = t + T * e;
            const float2 qm = bf[pad16((N - u) & (N - 1))];
            const float hu = GF ? __ldg(h + u) : h[u], bu = bt[u];
            v[e] = make_float2(hu * v[e].x + bu * qm.x, hu * v[e].y - bu * qm.y);
        }
    } else {
#pragma unroll
        for (int e = 0; e < E; ++e) v[e] = cscale(v[e], GF ? __ldg(h + t + T * e) : h[t + T * e]);
    }
    fft_regs<N, E, 1>(v, bf, tw, t);
    __syncthreads();  // the last exchange's reads are complete
#pragma unroll
    for (int e = 0; e < E; ++e) bf[sidx(e)] = v[e];
    fence_async_smem();
    __syncthreads();
    if (t == 0) {
        for (int q = 0; q < nchunk; ++q)
            for (int r = 0; r < crows; r += boxr)
                if (chk(q * cstride + c * crows + r + boxr <= nrows, CK_COL_BOX))
                    tma_store_2d(map, 0, (int)(q * cstride + c * crows + r), bf + (q * crows + r) * 16);
        bulk_commit();
    }
}

template <int N, bool GF, int BL>
__global__ void __launch_bounds__(ColCfg<N>::THREADS, BL)
    k_cols_filter_tma(const __grid_constant__ CUtensorMap map, const float *__restrict__ hs,
                      const float *__restrict__ beta, long long hs_img, long long beta_img, int log2half,
                      long long ncols, int log2g, const float2 *__restrict__ tw, int *status, int crows, int boxr,
                      long long cstride, int nchunk, int kbase) {
    typedef ColTmaCfg<N, GF, BL> K;
    extern __shared__ __align__(1024) unsigned char smraw[];
    unsigned char *base = smraw + ((1024u - (smem_u32(smraw) & 1023u)) & 1023u);  // the swizzle repeats every 1 KB
    uint64_t *bar = reinterpret_cast<uint64_t *>(base + 2 * K::BUF + 2 * K::FB);
    const long long hmask = (1LL << log2half) - 1;
    const int t = threadIdx.x;
    pdl_release();  // the inverse row pass may launch and wait for this one
    if (t == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
    }
    pdl_wait();  // the forward row pass's spectra are complete
    __syncthreads();
    long long c = blockIdx.x;
    if (t == 0 && c < ncols) {  // the first column and its filter into buffer 0
        mbar_expect_tx(&bar[0], (uint32_t)(N * sizeof(float2) + K::FB));
        float2 *b0 = reinterpret_cast<float2 *>(base);
        for (int q = 0; q < nchunk; ++q)
            for (int r = 0; r < crows; r += boxr)
                if (chk(q * cstride + c * crows + r + boxr <= ncols * ColTmaCfg<N, GF, BL>::ROWS, CK_COL_BOX))
                    tma_load_2d(b0 + (q * crows + r) * 16, &map, 0, (int)(q * cstride + c * crows + r), &bar[0]);
        if constexpr (!GF)
            bulk_load(base + 2 * K::BUF, hs + (c >> log2half) * hs_img + (c & hmask) * N, N * sizeof(float),
                      &bar[0]);
    }
    for (int it = 0; c < ncols; c += gridDim.x, ++it) {
        const int b = it & 1;
        const bool ok = mbar_wait_bounded(&bar[b], (it >> 1) & 1, kTmaPolls);
        if (__syncthreads_or(!ok)) {  // uniform: give up on the rest of this block's columns
            if (t == 0) {
                atomicExch(status, 1);
                mbar_wait_bounded(&bar[b], (it >> 1) & 1, kTmaPolls);  // the copies in flight, bounded
            }
            break;
        }
        const float *h = GF ? hs + (c >> log2half) * hs_img + (c & hmask) * N  // this column's filter
                            : reinterpret_cast<const float *>(base + 2 * K::BUF + b * K::FB);
        cols_tma_column<N, GF, BL>(&map, reinterpret_cast<float2 *>(base + b * K::BUF), h,
                           beta + (c >> log2half) * beta_img, c, kbase == 0 && (c & hmask) == 0,
                           c + gridDim.x < ncols, b, tw, log2g, base, hs, hs_img, log2half, crows, boxr, cstride,
                           nchunk, ncols * K::ROWS);
    }
    if (t == 0) bulk_wait_read();  // every store has read its buffer before the block's memory goes
}

template <int N, bool GF, int BL>
static cudaError_t run_cols_tma(void *spec, const float *hs, const float *beta, long long hs_img, long long beta_img,
                                int cols, int nimg, int log2g, const void *tw, int *status, cudaStream_t s,
                                bool *used, ColSlab cs) {
    typedef ColTmaCfg<N, GF, BL> K;
    *used = false;
    const EncodeTiledFn enc = encode_tiled();
    if (!enc || !status || hs_img % 4 != 0) return cudaSuccess;
    const long long ncols = cs.ls ? cs.mloc : (long long)(cols / 2) * nimg;
    // runs of a column: one of N/16 rows, or one per rank of 2^ls / 16 rows
    // each (whole 1 KB swizzle periods, so every run lands 1024-byte aligned)
    const int crows = cs.ls ? (1 << cs.ls) / 16 : K::ROWS;
    const int nchunk = cs.ls ? N >> cs.ls : 1;
    if (crows < 8 || crows % 8 != 0) return cudaSuccess;
    const int boxr = crows < 256 ? crows : 256;
    const long long cstride = cs.ls ? (long long)cs.mloc * crows : 0;
    if (ncols * K::ROWS > 0x7fffffffLL) return cudaSuccess;
    // the spectra as rows of 16 slots (128 bytes): {32 floats, ncols * N / 16 rows}
    cuuint64_t dims[2] = {32, (cuuint64_t)(ncols * K::ROWS)};
    cuuint64_t strides[1] = {128};
    cuuint32_t box[2] = {32, (cuuint32_t)boxr};
    cuuint32_t estr[2] = {1, 1};
    CUtensorMap map;
    if (enc(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, spec, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaSuccess;
    auto kern = k_cols_filter_tma<N, GF, BL>;
    static int slots = 0;  // resident blocks (per process; one device type)
    if (slots == 0) {
        cudaError_t e = set_smem_attrs((const void *)kern, K::SMEM, K::BLOCKS);
        int dev = 0, sms = 0, per_sm = 0;
        if (e == cudaSuccess) e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, K::THREADS, K::SMEM);
        if (e != cudaSuccess) return e;
        if (per_sm < 1) return cudaSuccess;
        slots = sms * per_sm;
    }
    const long long rounds = (ncols + slots - 1) / slots;
    const long long grid = (ncols + rounds - 1) / rounds;  // the fewest blocks for the same number of rounds
    const int log2half = cs.ls ? ilog2(cs.mloc) : ilog2(cols / 2);
    cudaError_t e = launch_pdl(kern, dim3((unsigned)grid), dim3(K::THREADS), K::SMEM, s, map, hs, beta, hs_img,
                               beta_img, log2half, ncols, log2g, static_cast<const float2 *>(tw), status, crows,
                               boxr, cstride, nchunk, cs.kbase);
    *used = e == cudaSuccess;
    return e;
}

// form: 0 = the default (the TMA-fed persistent kernel with its filter in
// shared memory where it applies), 1 = that kernel, 2 = the TMA-fed kernel
// with the filter read from global memory, 3 = the one-column-per-block kernel.
template <int N>
static cudaError_t run_cols(void *spec, const float *hs, const float *beta, long long hs_img, long long beta_img,
                            int cols, int nimg, int log2g, const void *tw, int *status, cudaStream_t s, ColSlab cs,
                            int form) {
    typedef ColCfg<N> K;
    if constexpr (N >= 4096 && K::W == 1 && K::THREADS == 256) {
        if ((1 << log2g) <= K::T && cols >= 4 && form != 3) {
            bool used = false;
            cudaError_t e =
                form == 2 ? run_cols_tma<N, true, 2>(spec, hs, beta, hs_img, beta_img, cols, nimg, log2g, tw, status, s,
                                                     &used, cs)
                          : run_cols_tma<N, false, 2>(spec, hs, beta, hs_img, beta_img, cols, nimg, log2g, tw, status,
                                                      s, &used, cs);
            if (e != cudaSuccess || used) return e;
        }
    }
    auto kern = k_cols_filter<N>;
    cudaError_t e = set_smem_attrs((const void *)kern, K::SMEM, 2);
    if (e != cudaSuccess) return e;
    const int half = cs.ls ? cs.mloc : cols / 2;
    dim3 grid((half + K::W - 1) / K::W, nimg);
    kern<<<grid, K::THREADS, K::SMEM, s>>>(static_cast<float2 *>(spec), hs, beta, hs_img, beta_img, cols, log2g,
                                           static_cast<const float2 *>(tw), cs);
    return cudaGetLastError();
}

template <int N>
static cudaError_t run_cols_analytic(void *spec, const AnalyticFilter &f, int cols, int nimg, int log2g, const void *tw,
                                     cudaStream_t s) {
    typedef ColCfg<N> K;
    cudaError_t e = set_smem_attrs((const void *)k_cols_analytic<N>, K::SMEM, 2);
    if (e != cudaSuccess) return e;
    dim3 grid((cols / 2 + K::W - 1) / K::W, nimg);
    k_cols_analytic<N><<<grid, K::THREADS, K::SMEM, s>>>(static_cast<float2 *>(spec), f, cols, log2g,
                                                         static_cast<const float2 *>(tw));
    return cudaGetLastError();
}

cudaError_t launch_cols_analytic(void *spec, int kind, double p0, double p1, int rows, int cols, int nimg,
                                 const void *tw_rows, cudaStream_t s) {
    AnalyticFilter f;
    f.kind = kind;
    f.N = rows;
    f.M = cols;
    f.s = (float)(1.0 / ((double)rows * cols));
    f.order = 0;
    f.p = 0.f;
    f.q = 0;
    if (kind == 1) {
        f.p = (float)(1.0 / (2.0 * p0 * p0));
    } else if (kind == 2) {
        f.order = (int)p0;
        f.p = (float)(1.0 / (p1 * p1));
    } else if (kind == 3) {
        const double b2 = std::floor(p0 * p0);
        f.q = b2 > 2147483647.0 ? 2147483647 : (int)b2;
    } else {
        return cudaErrorInvalidValue;
    }
    int g = rows_pairs_per_block(cols);
    if (g > rows / 2) g = rows / 2;
    const int log2g = ilog2(g);
    switch (ilog2(rows)) {
#define GBFFT_CASE(L) \
    case L: return run_cols_analytic<(1 << L)>(spec, f, cols, nimg, log2g, tw_rows, s);
        GBFFT_CASE(1) GBFFT_CASE(2) GBFFT_CASE(3) GBFFT_CASE(4) GBFFT_CASE(5) GBFFT_CASE(6) GBFFT_CASE(7)
        GBFFT_CASE(8) GBFFT_CASE(9) GBFFT_CASE(10) GBFFT_CASE(11) GBFFT_CASE(12) GBFFT_CASE(13)
#undef GBFFT_CASE
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t check_take_cols(unsigned out[2]) { return check_word_take(out); }

cudaError_t launch_cols_filter(void *spec, const float *hs, const float *beta, long long hs_img, long long beta_img,
                               int rows, int cols, int nimg, const void *tw_rows, int *status, cudaStream_t s,
                               ColSlab cs, int form) {
    int g = rows_pairs_per_block(cols);
    if (g > rows / 2) g = rows / 2;
    const int log2g = ilog2(g);
    switch (ilog2(rows)) {
#define GBFFT_CASE(L)                                                                                        \
    case L:                                                                                                  \
        return run_cols<(1 << L)>(spec, hs, beta, hs_img, beta_img, cols, nimg, log2g, tw_rows, status, s, cs, \
                                  form);
        GBFFT_CASE(1) GBFFT_CASE(2) GBFFT_CASE(3) GBFFT_CASE(4) GBFFT_CASE(5) GBFFT_CASE(6) GBFFT_CASE(7)
        GBFFT_CASE(8) GBFFT_CASE(9) GBFFT_CASE(10) GBFFT_CASE(11) GBFFT_CASE(12) GBFFT_CASE(13)
#undef GBFFT_CASE
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace gbfft
