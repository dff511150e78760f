// rows.cu — launchers of the row passes of the Sec. 5 pipeline; the kernel
// bodies and the description of the method live in rows_impl.cuh.
#include "internal.h"
#include "rows_impl.cuh"

#ifndef GBFFT_PREP_K
#define GBFFT_PREP_K 64  // half-spectrum columns per filter-preparation tile
#endif

namespace gbfft {

int rows_pairs_per_block(int cols) {
    switch (ilog2(cols)) {
#define GBFFT_CASE(L) \
    case L: return RowCfg<(1 << L)>::PPC;
        GBFFT_CASE(1) GBFFT_CASE(2) GBFFT_CASE(3) GBFFT_CASE(4) GBFFT_CASE(5) GBFFT_CASE(6) GBFFT_CASE(7)
        GBFFT_CASE(8) GBFFT_CASE(9) GBFFT_CASE(10) GBFFT_CASE(11) GBFFT_CASE(12) GBFFT_CASE(13)
#undef GBFFT_CASE
        default: return 0;
    }
}

// Forward row pass over a chunk of images (blockIdx.y = image).
// filter_mode 1: image 0's blocks also prepare the shared filter from H;
// filter_mode 2: every image prepares its own from H + y * h_stride.
template <int M>
__global__ void __launch_bounds__(RowCfg<M>::THREADS, RowCfg<M>::THREADS <= 512 ? 2 : 1)
    k_rows_fwd(const float *__restrict__ img, float2 *__restrict__ spec, const float *__restrict__ H,
               float *__restrict__ hs, float *__restrict__ beta, int N, int log2g, long long h_stride,
               int filter_mode, float scale, const float2 *__restrict__ tw) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const size_t y = blockIdx.y;
    const bool own = filter_mode == 2;
    rows_fwd_body<M>(img + y * N * M, spec + y * (M / 2) * N, H + (own ? y * h_stride : 0),
                     hs + (own ? y * (M / 2) * N : 0), beta + (own ? y * N : 0), N, log2g,
                     own || (filter_mode == 1 && y == 0), scale, tw, blockIdx.x, smraw);
}

template <int M>
__global__ void __launch_bounds__(RowCfg<M>::THREADS, RowCfg<M>::THREADS <= 512 ? 2 : 1)
    k_rows_inv(const float2 *__restrict__ spec, float *__restrict__ out, int N, int log2g,
               const float2 *__restrict__ tw) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const size_t y = blockIdx.y;
    rows_inv_body<M>(spec + y * (M / 2) * N, out + y * N * M, N, log2g, tw, blockIdx.x, smraw);
}

// Row passes of a zero-padded image (Sec. 5 application path): image y of the
// chunk is the crop.rows x crop.cols sub-image at img + y * img_stride; the
// forward pass reads zeros outside it, the inverse pass writes only inside it.
template <int M>
__global__ void __launch_bounds__(RowCfg<M>::THREADS, RowCfg<M>::THREADS <= 512 ? 2 : 1)
    k_rows_fwd_pad(const float *__restrict__ img, float2 *__restrict__ spec, int N, int log2g, Crop crop,
                   long long img_stride, const float2 *__restrict__ tw) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const size_t y = blockIdx.y;
    rows_fwd_body<M, Fp32Fft, true>(img + y * img_stride, spec + y * (M / 2) * N, nullptr, nullptr, nullptr, N,
                                    log2g, false, 0.f, tw, blockIdx.x, smraw, Fp32Fft(), crop);
}

template <int M>
__global__ void __launch_bounds__(RowCfg<M>::THREADS, RowCfg<M>::THREADS <= 512 ? 2 : 1)
    k_rows_inv_pad(const float2 *__restrict__ spec, float *__restrict__ out, int N, int log2g, Crop crop,
                   long long out_stride, const float2 *__restrict__ tw) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const size_t y = blockIdx.y;
    rows_inv_body<M, Fp32Fft, true>(spec + y * (M / 2) * N, out + y * out_stride, N, log2g, tw, blockIdx.x, smraw,
                                    Fp32Fft(), crop);
}

// Filter preparation on its own (the same values rows_fwd_body writes with
// `prep`), as a tiled transpose: block (bx, by) of image z covers P mirror-row
// pairs (a whole number of slot groups of G pairs) and K half-spectrum
// columns.  It reads filter rows u and -u in runs of K floats (the mirror run
// reversed), forms s * Hs[u][k] (column 0: alpha, plus beta), and writes each
// column's 2P slots as one contiguous run.  It touches no spectrum, so it runs
// concurrently with the forward row pass.
__global__ void __launch_bounds__(256)
    k_filter_prep(const float *__restrict__ H, float *__restrict__ hs, float *__restrict__ beta, int N, int M,
                  int log2g, int log2p, int log2k, float scale, long long h_stride, long long hs_img,
                  long long beta_img) {
    extern __shared__ __align__(16) unsigned char smraw[];
    float *tile = reinterpret_cast<float *>(smraw);
    const int G = 1 << log2g, P = 1 << log2p, K = 1 << log2k, H2 = M >> 1, SR = 2 * P + 1;
    const int p0 = blockIdx.x * P, k0 = blockIdx.y * K;
    const size_t z = blockIdx.z;
    const float *hb = H + z * h_stride;
    const float hsc = 0.5f * scale;
    // unit = (tile row r, four consecutive columns): row r = side * P + g is
    // pair p0 + g's first or mirror row u; filter row u gives Hs[u][k] with the
    // reversed run of row -u.
    const int nq = K >> 2, units = (2 * P) << (log2k - 2);
#pragma unroll 2
    for (int q = threadIdx.x; q < units; q += blockDim.x) {
        const int r = q >> (log2k - 2), kq = (q & (nq - 1)) << 2;
        const int side = r >> log2p, g = r & (P - 1);
        int a, b;
        rows_of_pair(p0 + g, N, a, b);
        const int u = side ? b : a, mu = (N - u) & (N - 1);
        const int ls = ((g >> log2g) << (log2g + 1)) + (side << log2g) + (g & (G - 1));
        const int k = k0 + kq;
        const float *Hu = hb + (size_t)u * M, *Hm = hb + (size_t)mu * M;
        const float4 f = __ldcs(reinterpret_cast<const float4 *>(Hu + k));
        // Hm[M - k - i], i = 0..3: the run [M-k-3, M-k] from two aligned quads
        // (for k = 0 the element M - k is column 0 of the mirror row, read below)
        const float4 m1 = __ldcs(reinterpret_cast<const float4 *>(Hm + (M - k - 4)));
        const float m0 = k == 0 ? Hm[0] : __ldcs(Hm + (M - k));
        float v0;
        if (k == 0) {
            const float h0 = 0.5f * (f.x + m0), h1 = 0.5f * (Hu[H2] + Hm[H2]);
            v0 = hsc * (h0 + h1);
            beta[z * beta_img + 2 * (size_t)p0 + ls] = hsc * (h0 - h1);
        } else {
            v0 = hsc * (f.x + m0);
        }
        float *tc = tile + kq * SR + ls;
        tc[0] = v0;
        tc[SR] = hsc * (f.y + m1.w);
        tc[2 * SR] = hsc * (f.z + m1.z);
        tc[3 * SR] = hsc * (f.w + m1.y);
    }
    __syncthreads();
    // each column's 2P slots, four per store (2P >= 4 and every run starts 16-byte aligned)
    float *hsb = hs + z * hs_img + 2 * (size_t)p0;
    const int m = K << (log2p - 1);
    for (int idx = threadIdx.x; idx < m; idx += blockDim.x) {
        const int i = idx >> (log2p - 1), s = (idx & ((P >> 1) - 1)) << 2;
        const float *tr = tile + i * SR + s;
        *reinterpret_cast<float4 *>(hsb + (size_t)(k0 + i) * N + s) = make_float4(tr[0], tr[1], tr[2], tr[3]);
    }
}

// Scalar form of the same tile for spectra narrower than four columns (cols < 8)
// or images of fewer than four rows.
__global__ void __launch_bounds__(256)
    k_filter_prep_small(const float *__restrict__ H, float *__restrict__ hs, float *__restrict__ beta, int N, int M,
                  int log2g, int log2p, int log2k, float scale, long long h_stride, long long hs_img,
                  long long beta_img) {
    extern __shared__ __align__(16) unsigned char smraw[];
    float *tile = reinterpret_cast<float *>(smraw);
    const int G = 1 << log2g, P = 1 << log2p, K = 1 << log2k, H2 = M >> 1, SR = 2 * P + 1;
    const int p0 = blockIdx.x * P, k0 = blockIdx.y * K;
    const size_t z = blockIdx.z;
    const float *hb = H + z * h_stride;
    // rows of the tile: r = side * P + g, pair p0 + g; local slot of that row
    const int n = (2 * P) << log2k;
    for (int idx = threadIdx.x; idx < n; idx += blockDim.x) {
        const int r = idx >> log2k, i = idx & (K - 1);
        const int side = r >> log2p, g = r & (P - 1);
        int a, b;
        rows_of_pair(p0 + g, N, a, b);
        const int u = side ? b : a, mu = (N - u) & (N - 1);
        const int ls = ((g >> log2g) << (log2g + 1)) + (side << log2g) + (g & (G - 1));
        const int k = k0 + i;
        const float *Hu = hb + (size_t)u * M, *Hm = hb + (size_t)mu * M;
        float v;
        if (k == 0) {
            const float h0 = 0.5f * (Hu[0] + Hm[0]), h1 = 0.5f * (Hu[H2] + Hm[H2]);
            v = 0.5f * scale * (h0 + h1);
            beta[z * beta_img + 2 * (size_t)p0 + ls] = 0.5f * scale * (h0 - h1);
        } else {
            v = 0.5f * scale * (__ldcs(Hu + k) + __ldcs(Hm + (M - k)));
        }
        tile[i * SR + ls] = v;
    }
    __syncthreads();
    float *hsb = hs + z * hs_img + 2 * (size_t)p0;
    const int m = K << (log2p + 1);
    for (int idx = threadIdx.x; idx < m; idx += blockDim.x) {
        const int i = idx >> (log2p + 1), s = idx & (2 * P - 1);
        hsb[(size_t)(k0 + i) * N + s] = tile[i * SR + s];
    }
}

cudaError_t launch_filter_prep(const float *H, float *hs, float *beta, int rows, int cols, int nimg, float scale,
                               long long h_stride, long long hs_img, long long beta_img, cudaStream_t s) {
    int g = rows_pairs_per_block(cols);
    if (g > rows / 2) g = rows / 2;
    int pp = g > 16 ? g : 16;  // pairs per tile: whole slot groups, runs of >= 32 slots
    if (pp > rows / 2) pp = rows / 2;
    int kk = cols / 2 < GBFFT_PREP_K ? cols / 2 : GBFFT_PREP_K;
    const size_t smem = (size_t)kk * (2 * pp + 1) * sizeof(float);
    const bool quads = kk >= 4 && pp >= 2;  // four columns per load, four slots per store
    const void *kern = quads ? (const void *)k_filter_prep : (const void *)k_filter_prep_small;
    cudaError_t e = set_smem_attrs(kern, smem);
    if (e != cudaSuccess) return e;
    dim3 grid((rows / 2) / pp, (cols / 2) / kk, nimg);
    if (quads)
        k_filter_prep<<<grid, 256, smem, s>>>(H, hs, beta, rows, cols, ilog2(g), ilog2(pp), ilog2(kk), scale, h_stride,
                                              hs_img, beta_img);
    else
        k_filter_prep_small<<<grid, 256, smem, s>>>(H, hs, beta, rows, cols, ilog2(g), ilog2(pp), ilog2(kk), scale,
                                                    h_stride, hs_img, beta_img);
    return cudaGetLastError();
}

template <int M> static cudaError_t set_smem(const void *kern) {
    return set_smem_attrs(kern, RowCfg<M>::SMEM, RowCfg<M>::THREADS <= 512 ? 2 : 1);
}

static int log2_pairs_per_block(int rows, int cols) {
    int g = rows_pairs_per_block(cols);
    if (g > rows / 2) g = rows / 2;
    return ilog2(g);
}

template <int M>
static cudaError_t run_rows_fwd(const RowsFwdArgs &a, cudaStream_t s) {
    typedef RowCfg<M> K;
    cudaError_t e = set_smem<M>((const void *)k_rows_fwd<M>);
    if (e != cudaSuccess) return e;
    const int lg = log2_pairs_per_block(a.rows, M);
    dim3 grid((a.rows / 2) >> lg, a.nimg);
    k_rows_fwd<M><<<grid, K::THREADS, K::SMEM, s>>>(a.img, static_cast<float2 *>(a.spec), a.H, a.hs, a.beta, a.rows,
                                                    lg, a.h_stride, a.filter_mode, a.scale,
                                                    static_cast<const float2 *>(a.tw));
    return cudaGetLastError();
}

template <int M>
static cudaError_t run_rows_inv(const void *spec, float *out, int rows, int nimg, const void *tw, cudaStream_t s) {
    typedef RowCfg<M> K;
    cudaError_t e = set_smem<M>((const void *)k_rows_inv<M>);
    if (e != cudaSuccess) return e;
    const int lg = log2_pairs_per_block(rows, M);
    dim3 grid((rows / 2) >> lg, nimg);
    k_rows_inv<M><<<grid, K::THREADS, K::SMEM, s>>>(static_cast<const float2 *>(spec), out, rows, lg,
                                                    static_cast<const float2 *>(tw));
    return cudaGetLastError();
}

template <int M>
static cudaError_t run_rows_pad(bool fwd, const void *src, void *dst, int rows, int nimg, int in_rows, int in_cols,
                                const void *tw, cudaStream_t s) {
    typedef RowCfg<M> K;
    const void *kern = fwd ? (const void *)k_rows_fwd_pad<M> : (const void *)k_rows_inv_pad<M>;
    cudaError_t e = set_smem<M>(kern);
    if (e != cudaSuccess) return e;
    const int lg = log2_pairs_per_block(rows, M);
    dim3 grid((rows / 2) >> lg, nimg);
    const Crop crop{in_rows, in_cols};
    const long long stride = (long long)in_rows * in_cols;
    if (fwd)
        k_rows_fwd_pad<M><<<grid, K::THREADS, K::SMEM, s>>>(static_cast<const float *>(src), static_cast<float2 *>(dst),
                                                             rows, lg, crop, stride, static_cast<const float2 *>(tw));
    else
        k_rows_inv_pad<M><<<grid, K::THREADS, K::SMEM, s>>>(static_cast<const float2 *>(src), static_cast<float *>(dst),
                                                             rows, lg, crop, stride, static_cast<const float2 *>(tw));
    return cudaGetLastError();
}

cudaError_t launch_rows_pad(bool fwd, const void *src, void *dst, int rows, int cols, int nimg, int in_rows,
                            int in_cols, const void *tw_cols, cudaStream_t s) {
    switch (ilog2(cols)) {
#define GBFFT_CASE(L) \
    case L: return run_rows_pad<(1 << L)>(fwd, src, dst, rows, nimg, in_rows, in_cols, tw_cols, s);
        GBFFT_CASE(1) GBFFT_CASE(2) GBFFT_CASE(3) GBFFT_CASE(4) GBFFT_CASE(5) GBFFT_CASE(6) GBFFT_CASE(7)
        GBFFT_CASE(8) GBFFT_CASE(9) GBFFT_CASE(10) GBFFT_CASE(11) GBFFT_CASE(12) GBFFT_CASE(13)
#undef GBFFT_CASE
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_rows_fwd(const RowsFwdArgs &a, cudaStream_t s) {
    switch (ilog2(a.cols)) {
#define GBFFT_CASE(L) \
    case L: return run_rows_fwd<(1 << L)>(a, s);
        GBFFT_CASE(1) GBFFT_CASE(2) GBFFT_CASE(3) GBFFT_CASE(4) GBFFT_CASE(5) GBFFT_CASE(6) GBFFT_CASE(7)
        GBFFT_CASE(8) GBFFT_CASE(9) GBFFT_CASE(10) GBFFT_CASE(11) GBFFT_CASE(12) GBFFT_CASE(13)
#undef GBFFT_CASE
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_rows_inv(const void *spec, float *out, int rows, int cols, int nimg, const void *tw_cols,
                            cudaStream_t s) {
    switch (ilog2(cols)) {
#define GBFFT_CASE(L) \
    case L: return run_rows_inv<(1 << L)>(spec, out, rows, nimg, tw_cols, s);
        GBFFT_CASE(1) GBFFT_CASE(2) GBFFT_CASE(3) GBFFT_CASE(4) GBFFT_CASE(5) GBFFT_CASE(6) GBFFT_CASE(7)
        GBFFT_CASE(8) GBFFT_CASE(9) GBFFT_CASE(10) GBFFT_CASE(11) GBFFT_CASE(12) GBFFT_CASE(13)
#undef GBFFT_CASE
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace gbfft
