// rows_impl.cuh — the row passes of the Sec. 5 pipeline (fft2 -> filter -> ifft2).
//
// Sec. 4 computes a 2D transform as "FFT on rows, then FFT on columns".  The
// image is real, so two image rows a, b are transformed together as one
// complex row z = a + i b (length M); their spectra separate as
//   A[k] = (Z[k] + conj Z[M-k]) / 2,   B[k] = (Z[k] - conj Z[M-k]) / (2i).
// A real row has a Hermitian spectrum, so only bins 0..M/2 are kept; A[0] and
// A[M/2] are real and share one complex slot (re = DC, im = Nyquist).  The
// half spectra go to the workspace column-major in slot order (layout.cuh):
// each block keeps its rows' transforms in shared memory and writes 2G
// consecutive slots of every column, separating the spectra as it stores.
//
// The inverse pass reads its rows' slots back, rebuilds Z[k] = A[k] + i B[k]
// for all k (A[M-k] = conj A[k]), runs one unscaled inverse FFT (Eq. E3) and
// writes Re z to row a and Im z to row b.
#pragma once

#include "check.cuh"
#include "fft_core.cuh"
#include "fft_tc.cuh"
#include "layout.cuh"
#include "tma.cuh"

namespace gbfft {

// Sub-image of a zero-padded transform (Sec. 5 application path): the image
// has `rows` x `cols` pixels (row pitch `cols`) in the top-left corner of the
// N x M grid; the rest of the grid is zero on input and not written on output.
struct Crop {
    int rows, cols;
};

template <int M> struct RowCfg {
    static constexpr int E = M < 16 ? M : 16;
    static constexpr int T = M / E;
    // row pairs per block: 512 threads (two blocks per SM), at least 2 pairs
    // (32-byte runs of complex64 per column)
    static constexpr int PPC = (512 / T) > 2 ? 512 / T : 2;
    static constexpr int THREADS = PPC * T;  // 512, or 1024 for M = 8192
    static constexpr int EXCH = PPC * padded_len(M);  // one exchange buffer per pair
    static constexpr int STAGE = (M / 2) * 2 * PPC;   // the inverse pass's staging of its slots
    static constexpr size_t SMEM_FWD = (size_t)EXCH * sizeof(float2);
    static constexpr size_t SMEM = (size_t)(EXCH > STAGE ? EXCH : STAGE) * sizeof(float2);
};

// A[k] (side false) or B[k] (side true) of a row pair from its transform Z
// in exchange buffer exg (element x at exg[pad16(x)]):
//   A = (Z[k] + conj Z[M-k]) / 2,  B = (Z[k] - conj Z[M-k]) / (2i);
// k = 0 packs the real DC and Nyquist bins as (re, im).
template <int M>
__device__ __forceinline__ float2 split_ab(const float2 *exg, int k, bool side) {
    const float2 zk = exg[pad16(k)];
    if (k == 0) {
        const float2 zn = exg[pad16(M / 2)];
        return side ? make_float2(zk.y, zn.y) : make_float2(zk.x, zn.x);
    }
    const float2 zm = exg[pad16(M - k)];
    return side ? make_float2(0.5f * (zk.y + zm.y), 0.5f * (zm.x - zk.x))
                : make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
}

// A[k] and B[k] of a row pair at once (two reads of the exchange buffer).
template <int M>
__device__ __forceinline__ void split_both(const float2 *exg, int k, float2 &A, float2 &B) {
    const float2 zk = exg[pad16(k)];
    const float2 zm = exg[pad16(k == 0 ? M / 2 : M - k)];
    if (k == 0) {
        A = make_float2(zk.x, zm.x);
        B = make_float2(zk.y, zm.y);
    } else {
        A = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
        B = make_float2(0.5f * (zk.y + zm.y), 0.5f * (zm.x - zk.x));
    }
}

// One block's share of the forward row pass: row pairs bx*G .. bx*G + G - 1 of
// one image.  img: the image [N][M]; spec: its half spectra [M/2][N] (slot
// order).  Every thread of the block must call it; it ends after a
// block-wide barrier-free epilogue, so a caller that reuses shared memory
// must synchronise first.
// With PAD, img is the crop.rows x crop.cols sub-image (pitch crop.cols) and
// the rest of the grid reads as zero.  With TSTORE (G = PPC >= 2) the block's
// run of 2G slots of every column is gathered in shared memory as the box
// [k][2G] and leaves by tensor stores through omap (a 3D view {2N floats,
// M/2 columns, images} of the half spectra, with the 32-byte swizzle when
// PPC = 2) at image z; smraw is then 1024-byte aligned.
template <int M, typename FFT = Fp32Fft, bool PAD = false, bool TSTORE = false>
__device__ __forceinline__ void rows_fwd_body(const float *__restrict__ img, float2 *__restrict__ spec, int N,
                                              int log2g, const float2 *__restrict__ tw, int bx,
                                              unsigned char *smraw, FFT fft = FFT(), Crop crop = Crop{0, 0},
                                              const CUtensorMap *omap = nullptr, int z = 0, Slab slab = Slab{0, 0}) {
    typedef RowCfg<M> K;
    constexpr int E = K::E, T = K::T, H2 = M / 2;
    float2 *sm = reinterpret_cast<float2 *>(smraw);
    const int G = 1 << log2g;
    const int g = threadIdx.x / T;
    const int t = threadIdx.x - g * T;
    const int p = slab.p0 + bx * G + g;
    const size_t ld = slab.ld ? (size_t)slab.ld : (size_t)N;  // column stride of the half spectra
    // the grid covers exactly N/2 pairs in groups of G; a checked build also
    // verifies the pair and the block's run of 2G slots per column (uniform
    // per block: a block whose run fails stores nothing)
    const bool run_ok = chk((size_t)(bx + 1) * 2 * G <= ld, CK_ROW_RUN);
    const bool active = g < G && run_ok && chk(p < (N >> 1), CK_ROW_PAIR);
    int a, b;
    rows_of_pair(active ? p : 0, N, a, b);

    float2 v[E];
    if (PAD && active) {
        const float *ra = img + (size_t)a * crop.cols;
        const float *rb = img + (size_t)b * crop.cols;
        const bool va = a < crop.rows, vb = b < crop.rows;
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int x = t + T * e;
            v[e] = make_float2(va && x < crop.cols ? __ldcs(ra + x) : 0.f, vb && x < crop.cols ? __ldcs(rb + x) : 0.f);
        }
    } else if (active) {
        const float *ra = img + (size_t)a * M;
        const float *rb = img + (size_t)b * M;
#pragma unroll
        for (int e = 0; e < E; ++e) v[e] = make_float2(__ldcs(ra + t + T * e), __ldcs(rb + t + T * e));
    } else {
#pragma unroll
        for (int e = 0; e < E; ++e) v[e] = make_float2(0.f, 0.f);
    }
    float2 *ex = sm + g * padded_len(M);
    fft.template run<M, E, -1>(v, ex, tw, t);
    __syncthreads();
#pragma unroll
    for (int e = 0; e < E; ++e) ex[pad16(t + T * e)] = v[e];
    __syncthreads();
    // split the two rows' spectra while storing: a unit is column k and two
    // consecutive slots s, s + 1 of the block's run of 2G (s < G: A of pairs
    // s, s + 1; s >= G: B of pairs s - G, s - G + 1), 16 bytes per store
    float2 *sb = spec + (size_t)bx * 2 * G;
    if (!run_ok) return;  // uniform per block
    if constexpr (TSTORE && K::PPC == 2) {
        // two pairs: each thread takes whole columns k (4 of them), reads
        // Z0[k], Z0[M-k], Z1[k], Z1[M-k] once for the four outputs A0 A1 B0 B1,
        // and writes them as the two 16-byte chunks of box row k.  The box is
        // stored with the 32-byte swizzle (chunk c of row k at c ^ ((k / 4) mod
        // 2)), so the eight rows a quarter warp writes cover all 32 banks.
        constexpr int CPT = H2 / K::THREADS;
        static_assert(CPT * K::THREADS == H2, "whole columns per thread");
        float4 out[2 * CPT];
#pragma unroll
        for (int i = 0; i < CPT; ++i) {
            const int k = threadIdx.x + i * K::THREADS;
            float2 a0, b0, a1, b1;
            split_both<M>(sm, k, a0, b0);
            split_both<M>(sm + padded_len(M), k, a1, b1);
            out[2 * i] = make_float4(a0.x, a0.y, a1.x, a1.y);
            out[2 * i + 1] = make_float4(b0.x, b0.y, b1.x, b1.y);
        }
        __syncthreads();  // every read of the exchange buffers is complete
        float4 *box = reinterpret_cast<float4 *>(sm);
#pragma unroll
        for (int i = 0; i < CPT; ++i) {
            const int k = threadIdx.x + i * K::THREADS, f = (k >> 2) & 1;
            box[2 * k + f] = out[2 * i];
            box[2 * k + (f ^ 1)] = out[2 * i + 1];
        }
        fence_async_smem();
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int k0 = 0; k0 < H2; k0 += 256) tma_store_3d(omap, bx * 8, k0, z, sm + (size_t)k0 * 4);
            bulk_commit();
            bulk_wait_read();
        }
    } else if constexpr (TSTORE) {
        // every unit (k, s) of the block, K::UNITS per thread, into registers;
        // then into the box [k][2G] over the exchange buffers (16-byte stores,
        // consecutive units adjacent) and out by the TMA
        // G = PPC here (the launcher checks): H2 G units over G T threads, 8 each
        constexpr int U = (H2 * K::PPC) / K::THREADS;
        static_assert(U == 8 && 4 * K::PPC <= 256, "8 units per thread; box of at most 256 floats wide");
        float4 out[U];
#pragma unroll
        for (int i = 0; i < U; ++i) {
            const int idx = threadIdx.x + i * K::THREADS;
            const int k = idx >> log2g, s = (idx & (G - 1)) * 2;
            const bool side = s >= G;
            const int g0 = side ? s - G : s;
            const float2 x0 = split_ab<M>(sm + g0 * padded_len(M), k, side);
            const float2 x1 = split_ab<M>(sm + (g0 + 1) * padded_len(M), k, side);
            out[i] = make_float4(x0.x, x0.y, x1.x, x1.y);
        }
        __syncthreads();  // every read of the exchange buffers is complete
        float4 *box = reinterpret_cast<float4 *>(sm);
#pragma unroll
        for (int i = 0; i < U; ++i) box[threadIdx.x + i * K::THREADS] = out[i];
        fence_async_smem();
        __syncthreads();
        if (threadIdx.x == 0) {
            constexpr int BK = H2 < 256 ? H2 : 256;  // columns per box
            for (int k0 = 0; k0 < H2; k0 += BK)
                tma_store_3d(omap, bx * 4 * G, k0, z, sm + (size_t)k0 * 2 * G);
            bulk_commit();
            bulk_wait_read();
        }
    } else if (G >= 2) {
        const int n = H2 << log2g;
        for (int idx = threadIdx.x; idx < n; idx += K::THREADS) {
            const int k = idx >> log2g, s = (idx & (G - 1)) * 2;
            const bool side = s >= G;
            const int g0 = side ? s - G : s;
            const float2 x0 = split_ab<M>(sm + g0 * padded_len(M), k, side);
            const float2 x1 = split_ab<M>(sm + (g0 + 1) * padded_len(M), k, side);
            *reinterpret_cast<float4 *>(sb + k * ld + s) = make_float4(x0.x, x0.y, x1.x, x1.y);
        }
    } else {  // one pair per block (N = 2): its A and B side by side
        for (int k = threadIdx.x; k < H2; k += K::THREADS) {
            const float2 a = split_ab<M>(sm, k, false), b = split_ab<M>(sm, k, true);
            *reinterpret_cast<float4 *>(sb + k * ld) = make_float4(a.x, a.y, b.x, b.y);
        }
    }
}

// One block's share of the inverse row pass: spec [M/2][N] (slot order) of one
// image -> rows of pairs bx*G .. bx*G + G - 1 of out [N][M], unscaled.
// With PAD, only the crop.rows x crop.cols sub-image is written (pitch crop.cols).
// Staging of the inverse row pass: column k's 2G slots in row k (no padding);
// slot s of row k sits at s ^ h(k), an XOR of the low bits that spreads the
// reads of one slot for 16 consecutive k (a half warp) over all 16 bank
// pairs: h(k) = (k >> max(0, 3 - log2 G)) mod min(2G, 16).
__device__ __forceinline__ int stage_pos(int k, int s, int log2g) {
    const int sh = log2g < 3 ? 3 - log2g : 0;
    const int m = (log2g < 3 ? (2 << log2g) : 16) - 1;
    return (k << (log2g + 1)) + (s ^ ((k >> sh) & m));
}

// With TLOAD (PPC = G = 2) the block's run of 2G slots of every column
// arrives by tensor loads through imap (the forward pass's 3D view of the half
// spectra, 32-byte swizzle) into the box [k][4] at image z, on the mbarrier
// bar (bounded wait; a wait that gives up sets *status and the block leaves);
// smraw is then 1024-byte aligned.
template <int M, typename FFT = Fp32Fft, bool PAD = false, bool TLOAD = false>
__device__ __forceinline__ void rows_inv_body(const float2 *__restrict__ spec, float *__restrict__ out, int N,
                                              int log2g, const float2 *__restrict__ tw, int bx,
                                              unsigned char *smraw, FFT fft = FFT(), Crop crop = Crop{0, 0},
                                              const CUtensorMap *imap = nullptr, int z = 0, uint64_t *bar = nullptr,
                                              int *status = nullptr, Slab slab = Slab{0, 0}) {
    typedef RowCfg<M> K;
    constexpr int E = K::E, T = K::T, H2 = M / 2;
    float2 *sm = reinterpret_cast<float2 *>(smraw);
    const int G = 1 << log2g;
    const int g = threadIdx.x / T;
    const int t = threadIdx.x - g * T;
    const int p = slab.p0 + bx * G + g;
    const size_t ld = slab.ld ? (size_t)slab.ld : (size_t)N;  // column stride of the half spectra
    const bool run_ok = chk((size_t)(bx + 1) * 2 * G <= ld, CK_ROW_RUN);  // uniform per block
    const bool active = g < G && run_ok && chk(p < (N >> 1), CK_ROW_PAIR);
    int a, b;
    rows_of_pair(active ? p : 0, N, a, b);

    float2 *stg = sm;
    // slot s of column k in the staging: the XOR layout below, or (TLOAD) the
    // swizzled box: chunk s / 2 of row k at (s / 2) ^ ((k / 4) mod 2)
    auto spos = [&](int k, int s) {
        if constexpr (TLOAD)
            return 4 * k + 2 * ((s >> 1) ^ ((k >> 2) & 1)) + (s & 1);
        else
            return stage_pos(k, s, log2g);
    };
    if constexpr (TLOAD) {
        static_assert(K::PPC == 2, "two pairs per block");
        if (threadIdx.x == 0 && run_ok) {
            mbar_init(bar, 1);
            mbar_expect_tx(bar, (uint32_t)(H2 * 4 * sizeof(float2)));
            for (int k0 = 0; k0 < H2; k0 += 256) tma_load_3d(sm + (size_t)k0 * 4, imap, bx * 8, k0, z, bar);
        }
        __syncthreads();  // the barrier is initialised before anyone tests it
        const bool ok = !run_ok || mbar_wait_bounded(bar, 0, kTmaPolls);
        if (__syncthreads_or(!ok)) {
            if (threadIdx.x == 0) {
                atomicExch(status, 1);
                mbar_wait_bounded(bar, 0, kTmaPolls);  // the copies in flight, bounded
            }
            return;  // uniform
        }
    } else {
        const float2 *sb = spec + (size_t)bx * 2 * G;
        const int n = run_ok ? H2 << log2g : 0;
        for (int idx = threadIdx.x; idx < n; idx += K::THREADS) {
            const int k = idx >> log2g, s = (idx & (G - 1)) * 2;
            const float4 x = *reinterpret_cast<const float4 *>(sb + k * ld + s);
            stg[stage_pos(k, s, log2g)] = make_float2(x.x, x.y);
            stg[stage_pos(k, s + 1, log2g)] = make_float2(x.z, x.w);
        }
        __syncthreads();
    }
    float2 v[E];
    if (active) {
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int k = t + T * e;
            float2 A, B;
            if (e < E / 2) {  // 0 <= k < M/2
                A = stg[spos(k, g)];
                B = stg[spos(k, G + g)];
                if (e == 0 && t == 0) {
                    A.y = 0.f;
                    B.y = 0.f;
                }
            } else if (e == E / 2 && t == 0) {  // k = M/2: the packed Nyquist bins
                A = make_float2(stg[spos(0, g)].y, 0.f);
                B = make_float2(stg[spos(0, G + g)].y, 0.f);
            } else {  // M/2 < k < M: A[k] = conj A[M-k]
                const int km = M - k;
                const float2 am = stg[spos(km, g)], bm = stg[spos(km, G + g)];
                A = make_float2(am.x, -am.y);
                B = make_float2(bm.x, -bm.y);
            }
            v[e] = make_float2(A.x - B.y, A.y + B.x);  // A + i B
        }
    } else {
#pragma unroll
        for (int e = 0; e < E; ++e) v[e] = make_float2(0.f, 0.f);
    }
    // the exchange buffers overlap the staging area: the first exchange of
    // fft_regs starts with a block barrier, after every thread read its values
    fft.template run<M, E, 1>(v, sm + g * padded_len(M), tw, t);
    if (PAD && active) {
        float *ra = out + (size_t)a * crop.cols;
        float *rb = out + (size_t)b * crop.cols;
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int x = t + T * e;
            if (x < crop.cols) {
                if (a < crop.rows) __stcs(ra + x, v[e].x);
                if (b < crop.rows) __stcs(rb + x, v[e].y);
            }
        }
    } else if (active) {
        float *ra = out + (size_t)a * M;
        float *rb = out + (size_t)b * M;
#pragma unroll
        for (int e = 0; e < E; ++e) {
            __stcs(ra + t + T * e, v[e].x);
            __stcs(rb + t + T * e, v[e].y);
        }
    }
}

// ---- filter preparation ------------------------------------------------
// The column pass multiplies half-spectrum column k by s * Hs[u][k] (s =
// 1/(N M), Hs[u][k] = (H[u][k] + H[-u][-k]) / 2, the even part of the filter:
// the real part of the pipeline's output only sees it) and, in the packed
// column 0, uses alpha = s (h0 + h1) / 2 and beta = s (h0 - h1) / 2 with
// h0 = Hs[u][0], h1 = Hs[u][M/2].  They are prepared column-major in row
// order: hs[k][u] (alpha in k = 0), beta[u].
constexpr int kPrepRows = 32, kPrepCols = 64;  // tile of the preparation

// One tile of the filter preparation (block-wide; blockDim.x threads): rows
// u0 .. u0 + R - 1, half-spectrum columns k0 .. k0 + K - 1 (K = 2^log2k) of
// one filter H into hs (row order; column k at hs column k - kbeg) and beta;
// `tile` is K (R + 1) floats of shared memory.  Ends with the tile's global
// writes (no trailing barrier).
template <int R, bool QUADS>
__device__ __forceinline__ void filter_prep_tile(const float *__restrict__ hb, float *__restrict__ hsz,
                                                 float *__restrict__ betaz, int N, int M, int log2k, float scale,
                                                 int u0, int k0, float *tile, int kbeg = 0) {
    constexpr int SR = R + 1;  // tile row stride (odd: conflict-free column writes)
    const int K = 1 << log2k, H2 = M >> 1;
    const float hsc = 0.5f * scale;
    if (!chk(u0 + R <= N && k0 >= kbeg && k0 + K <= H2, CK_PREP_TILE)) return;  // uniform per block

    if (QUADS) {
        // unit = (row r, four consecutive columns); the mirror run [M-k-3, M-k]
        // comes from two aligned quads (for k = 0 the element M - k is column 0)
        const int nq = K >> 2, units = R << (log2k - 2);
        struct Unit {
            float4 f, m1;  // H[u][k .. k+3] and H[-u][M-k-4 .. M-k-1]
            float m0;      // H[-u][M-k] (H[-u][0] for k = 0)
        };
        auto load = [&](int q) {
            const int r = q >> (log2k - 2), kq = (q & (nq - 1)) << 2;
            const int u = u0 + r, mu = (N - u) & (N - 1);
            const int k = k0 + kq;
            const float *Hu = hb + (size_t)u * M, *Hm = hb + (size_t)mu * M;
            Unit x;
            x.f = __ldcs(reinterpret_cast<const float4 *>(Hu + k));
            x.m1 = __ldcs(reinterpret_cast<const float4 *>(Hm + (M - k - 4)));
            x.m0 = k == 0 ? Hm[0] : __ldcs(Hm + (M - k));
            return x;
        };
        auto stage = [&](int q, const Unit &x) {
            const int r = q >> (log2k - 2), kq = (q & (nq - 1)) << 2;
            const int u = u0 + r, mu = (N - u) & (N - 1);
            float v0;
            if (k0 + kq == 0) {
                const float h0 = 0.5f * (x.f.x + x.m0);
                const float h1 = 0.5f * (hb[(size_t)u * M + H2] + hb[(size_t)mu * M + H2]);
                v0 = hsc * (h0 + h1);
                betaz[u] = hsc * (h0 - h1);
            } else {
                v0 = hsc * (x.f.x + x.m0);
            }
            float *tc = tile + kq * SR + r;
            tc[0] = v0;
            tc[SR] = hsc * (x.f.y + x.m1.w);
            tc[2 * SR] = hsc * (x.f.z + x.m1.z);
            tc[3 * SR] = hsc * (x.f.w + x.m1.y);
        };
        // the usual tile (64 columns, 256 threads): U units per thread, every
        // load of the thread issued before the first is used (measured 4096^2
        // pipeline 133.0 -> 132.4 us: the preparation shares the SMs with the
        // forward row pass, so its blocks should not wait on one load at a time)
        constexpr int U = R / 16;
        if (U >= 1 && units == U * (int)blockDim.x) {
            Unit x[U >= 1 ? U : 1];
#pragma unroll
            for (int i = 0; i < U; ++i) x[i] = load(threadIdx.x + i * blockDim.x);
#pragma unroll
            for (int i = 0; i < U; ++i) stage(threadIdx.x + i * blockDim.x, x[i]);
        } else {
#pragma unroll 2
            for (int q = threadIdx.x; q < units; q += blockDim.x) stage(q, load(q));
        }
    } else {
        const int n = R << log2k;
        for (int idx = threadIdx.x; idx < n; idx += blockDim.x) {
            const int r = idx >> log2k, i = idx & (K - 1);
            const int u = u0 + r, mu = (N - u) & (N - 1);
            const int k = k0 + i;
            const float *Hu = hb + (size_t)u * M, *Hm = hb + (size_t)mu * M;
            float v;
            if (k == 0) {
                const float h0 = 0.5f * (Hu[0] + Hm[0]), h1 = 0.5f * (Hu[H2] + Hm[H2]);
                v = hsc * (h0 + h1);
                betaz[u] = hsc * (h0 - h1);
            } else {
                v = hsc * (__ldcs(Hu + k) + __ldcs(Hm + (M - k)));
            }
            tile[i * SR + r] = v;
        }
    }
    __syncthreads();
    float *hsb = hsz + u0;
    if (QUADS) {  // four rows per store: R >= 4 and u0 a multiple of R
        const int m = K * (R / 4);
        for (int idx = threadIdx.x; idx < m; idx += blockDim.x) {
            const int i = idx / (R / 4), r = (idx % (R / 4)) * 4;
            const float *tr = tile + i * SR + r;
            *reinterpret_cast<float4 *>(hsb + (size_t)(k0 - kbeg + i) * N + r) = make_float4(tr[0], tr[1], tr[2], tr[3]);
        }
    } else {
        const int m = K * R;
        for (int idx = threadIdx.x; idx < m; idx += blockDim.x) {
            const int i = idx / R, r = idx % R;
            hsb[(size_t)(k0 - kbeg + i) * N + r] = tile[i * SR + r];
        }
    }
}


}  // namespace gbfft
