// rows.cu — launchers of the row passes of the Sec. 5 pipeline; the kernel
// bodies and the description of the method live in rows_impl.cuh.
#include "internal.h"
#include "rows_impl.cuh"


namespace gbfft {

cudaError_t check_take_rows(unsigned out[2]) { return check_word_take(out); }

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
template <int M>
__global__ void __launch_bounds__(RowCfg<M>::THREADS, RowCfg<M>::THREADS <= 512 ? 2 : 1)
    k_rows_fwd(const float *__restrict__ img, float2 *__restrict__ spec, int N, int log2g,
               const float2 *__restrict__ tw, Slab slab, ImgIndirect ind) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const size_t y = blockIdx.y;
    const float *im = ind.ptrs ? ind.ptrs[ind.idx[y]].img : img + y * N * M;
    rows_fwd_body<M>(im, spec + y * (M / 2) * N, N, log2g, tw, blockIdx.x, smraw, Fp32Fft(), Crop{0, 0}, nullptr, 0,
                     slab);
}

template <int M>
__global__ void __launch_bounds__(RowCfg<M>::THREADS, RowCfg<M>::THREADS <= 512 ? 2 : 1)
    k_rows_inv(const float2 *__restrict__ spec, float *__restrict__ out, int N, int log2g,
               const float2 *__restrict__ tw, Slab slab, ImgIndirect ind) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const size_t y = blockIdx.y;
    float *o = ind.ptrs ? ind.ptrs[ind.idx[y]].out : out + y * N * M;
    rows_inv_body<M>(spec + y * (M / 2) * N, o, N, log2g, tw, blockIdx.x, smraw, Fp32Fft(), Crop{0, 0}, nullptr, 0,
                     nullptr, nullptr, slab);
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
    rows_fwd_body<M, Fp32Fft, true>(img + y * img_stride, spec + y * (M / 2) * N, N, log2g, tw, blockIdx.x, smraw,
                                    Fp32Fft(), crop);
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
// `prep`), as a tiled transpose: block (bx, by) of image z covers R filter
// rows u = bx R .. bx R + R - 1 and K half-spectrum columns.  For each row it
// reads a run of row u and the reversed run of row -u, forms s * Hs[u][k]
// (column 0: alpha, plus beta), and writes each column's R rows as one
// contiguous run (row order).  It touches no spectrum, so it runs
// concurrently with the forward row pass.
template <int R, bool QUADS>
__global__ void __launch_bounds__(256)
    k_filter_prep(const float *__restrict__ H, float *__restrict__ hs, float *__restrict__ beta, int N, int M,
                  int log2k, float scale, long long h_stride, long long hs_img, long long beta_img, int kbeg,
                  ImgIndirect ind) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const size_t z = blockIdx.z;
    const float *hz = ind.ptrs ? ind.ptrs[ind.idx[z]].H : H + z * h_stride;
    filter_prep_tile<R, QUADS>(hz, hs + z * hs_img, beta + z * beta_img, N, M, log2k, scale,
                               blockIdx.x * R, kbeg + (blockIdx.y << log2k), reinterpret_cast<float *>(smraw), kbeg);
}

cudaError_t launch_filter_prep(const float *H, float *hs, float *beta, int rows, int cols, int nimg, float scale,
                               long long h_stride, long long hs_img, long long beta_img, cudaStream_t s, int kbeg,
                               int kcnt, ImgIndirect ind) {
    const int ncol = kcnt > 0 ? kcnt : cols / 2;  // half-spectrum columns to prepare
    const int kk = ncol < kPrepCols ? ncol : kPrepCols;
    const int rr = rows < kPrepRows ? rows : kPrepRows;  // rows per tile
    const bool quads = kk >= 4 && rr >= 4;  // four columns per load, four rows per store
    const size_t smem = (size_t)kk * (rr + 1) * sizeof(float);
    dim3 grid(rows / rr, ncol / kk, nimg);
    cudaError_t e = cudaErrorInvalidValue;
    switch (rr * 2 + (quads ? 1 : 0)) {
#define GBFFT_R(RR, Q)                                                                                         \
    case RR * 2 + Q:                                                                                           \
        e = set_smem_attrs((const void *)k_filter_prep<RR, Q>, smem);                                          \
        if (e != cudaSuccess) return e;                                                                        \
        k_filter_prep<RR, Q><<<grid, 256, smem, s>>>(H, hs, beta, rows, cols, ilog2(kk), scale, h_stride, hs_img, \
                                                     beta_img, kbeg, ind);                                     \
        return cudaGetLastError();
        GBFFT_R(2, false) GBFFT_R(4, false) GBFFT_R(8, false) GBFFT_R(16, false) GBFFT_R(32, false)
        GBFFT_R(4, true) GBFFT_R(8, true) GBFFT_R(16, true) GBFFT_R(32, true)
#undef GBFFT_R
        default: return e;
    }
}

template <int M> static cudaError_t set_smem(const void *kern, size_t smem) {
    return set_smem_attrs(kern, smem, RowCfg<M>::THREADS <= 512 ? 2 : 1);
}

static int log2_pairs_per_block(int rows, int cols) {
    int g = rows_pairs_per_block(cols);
    if (g > rows / 2) g = rows / 2;
    return ilog2(g);
}

// The forward row pass with its half-spectrum runs leaving by tensor stores
// (rows_fwd_body with TSTORE): every block holds G = PPC pairs.
template <int M>
__global__ void __launch_bounds__(RowCfg<M>::THREADS, RowCfg<M>::THREADS <= 512 ? 2 : 1)
    k_rows_fwd_tma(const float *__restrict__ img, float2 *__restrict__ spec, int N, int log2g,
                   const float2 *__restrict__ tw, const __grid_constant__ CUtensorMap omap, Slab slab,
                   ImgIndirect ind) {
    extern __shared__ __align__(1024) unsigned char smraw[];
    unsigned char *base = smraw + ((1024u - (smem_u32(smraw) & 1023u)) & 1023u);  // the box's swizzle period
    pdl_release();  // the column pass may launch and wait for this one
    const size_t y = blockIdx.y;
    const float *im = ind.ptrs ? ind.ptrs[ind.idx[y]].img : img + y * N * M;
    rows_fwd_body<M, Fp32Fft, false, true>(im, spec + y * (M / 2) * N, N, log2g, tw, blockIdx.x, base, Fp32Fft(),
                                           Crop{0, 0}, &omap, (int)y, slab);
}

// Tensor map of the half spectra of nimg images ({2 rows floats, cols/2
// columns, images}, box {4 G floats, up to 256 columns, 1}) for
// k_rows_fwd_tma; false if the driver offers no encoder or refuses.
static bool spec_map(CUtensorMap *map, void *spec, int rows, int cols, int nimg, int g) {
    const EncodeTiledFn enc = encode_tiled();
    if (!enc) return false;
    const cuuint64_t h2 = (cuuint64_t)cols / 2;
    cuuint64_t dims[3] = {2 * (cuuint64_t)rows, h2, (cuuint64_t)nimg};
    cuuint64_t strides[2] = {(cuuint64_t)rows * 8, h2 * rows * 8};
    cuuint32_t box[3] = {(cuuint32_t)(4 * g), (cuuint32_t)(h2 < 256 ? h2 : 256), 1};
    cuuint32_t estr[3] = {1, 1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, spec, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               g == 2 ? CU_TENSOR_MAP_SWIZZLE_32B : CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// slab.ld > 0: one image, pairs slab.p0 .. slab.p0 + slab.ld / 2 - 1 into
// [M/2][slab.ld] (the launcher's caller checks that they fill whole blocks)
template <int M>
static cudaError_t run_rows_fwd(const float *img, void *spec, int rows, int nimg, const void *tw, cudaStream_t s,
                                Slab slab, ImgIndirect ind) {
    typedef RowCfg<M> K;
    const int ld = slab.ld ? slab.ld : rows;  // column stride of the half spectra written
    if constexpr (M >= 256 && 4 * K::PPC <= 256 && K::THREADS <= 512) {
        const int lg = log2_pairs_per_block(rows, M);
        CUtensorMap map;
        if ((1 << lg) == K::PPC && spec_map(&map, spec, ld, M, nimg, K::PPC)) {
            const size_t smem = K::SMEM_FWD + 1024;
            cudaError_t e = set_smem<M>((const void *)k_rows_fwd_tma<M>, smem);
            if (e != cudaSuccess) return e;
            dim3 grid((ld / 2) >> lg, nimg);
            k_rows_fwd_tma<M><<<grid, K::THREADS, smem, s>>>(img, static_cast<float2 *>(spec), rows, lg,
                                                             static_cast<const float2 *>(tw), map, slab, ind);
            return cudaGetLastError();
        }
    }
    cudaError_t e = set_smem<M>((const void *)k_rows_fwd<M>, K::SMEM_FWD);
    if (e != cudaSuccess) return e;
    const int lg = log2_pairs_per_block(rows, M);
    dim3 grid((ld / 2) >> lg, nimg);
    k_rows_fwd<M><<<grid, K::THREADS, K::SMEM_FWD, s>>>(img, static_cast<float2 *>(spec), rows, lg,
                                                    static_cast<const float2 *>(tw), slab, ind);
    return cudaGetLastError();
}

// The inverse row pass with its slot runs arriving by tensor loads
// (rows_inv_body with TLOAD): two pairs per block.
template <int M>
__global__ void __launch_bounds__(RowCfg<M>::THREADS, 2)
    k_rows_inv_tma(float *__restrict__ out, int N, int log2g, const float2 *__restrict__ tw,
                   const __grid_constant__ CUtensorMap imap, int *status, Slab slab, ImgIndirect ind) {
    extern __shared__ __align__(1024) unsigned char smraw[];
    unsigned char *base = smraw + ((1024u - (smem_u32(smraw) & 1023u)) & 1023u);  // the box's swizzle period
    uint64_t *bar = reinterpret_cast<uint64_t *>(base + RowCfg<M>::SMEM);
    pdl_wait();  // the column pass's spectra are complete
    const size_t y = blockIdx.y;
    float *o = ind.ptrs ? ind.ptrs[ind.idx[y]].out : out + y * N * M;
    rows_inv_body<M, Fp32Fft, false, true>(nullptr, o, N, log2g, tw, blockIdx.x, base, Fp32Fft(), Crop{0, 0}, &imap,
                                           (int)y, bar, status, slab);
}

// slab.ld > 0: one image, pairs slab.p0 .. from [M/2][slab.ld]
template <int M>
static cudaError_t run_rows_inv(const void *spec, float *out, int rows, int nimg, const void *tw, int *status,
                                cudaStream_t s, Slab slab, ImgIndirect ind) {
    typedef RowCfg<M> K;
    const int ld = slab.ld ? slab.ld : rows;  // column stride of the half spectra read
    if constexpr (K::PPC == 2 && K::THREADS <= 512) {
        const int lg = log2_pairs_per_block(rows, M);
        CUtensorMap map;
        if (status && (1 << lg) == 2 && spec_map(&map, const_cast<void *>(spec), ld, M, nimg, 2)) {
            const size_t smem = K::SMEM + 1024 + 16;
            cudaError_t e = set_smem<M>((const void *)k_rows_inv_tma<M>, smem);
            if (e != cudaSuccess) return e;
            dim3 grid((ld / 2) >> lg, nimg);
            return launch_pdl(k_rows_inv_tma<M>, grid, dim3(K::THREADS), smem, s, out, rows, lg,
                              static_cast<const float2 *>(tw), map, status, slab, ind);
        }
    }
    cudaError_t e = set_smem<M>((const void *)k_rows_inv<M>, K::SMEM);
    if (e != cudaSuccess) return e;
    const int lg = log2_pairs_per_block(rows, M);
    dim3 grid((ld / 2) >> lg, nimg);
    k_rows_inv<M><<<grid, K::THREADS, K::SMEM, s>>>(static_cast<const float2 *>(spec), out, rows, lg,
                                                    static_cast<const float2 *>(tw), slab, ind);
    return cudaGetLastError();
}

template <int M>
static cudaError_t run_rows_pad(bool fwd, const void *src, void *dst, int rows, int nimg, int in_rows, int in_cols,
                                const void *tw, cudaStream_t s) {
    typedef RowCfg<M> K;
    const void *kern = fwd ? (const void *)k_rows_fwd_pad<M> : (const void *)k_rows_inv_pad<M>;
    const size_t smem = fwd ? K::SMEM_FWD : K::SMEM;
    cudaError_t e = set_smem<M>(kern, smem);
    if (e != cudaSuccess) return e;
    const int lg = log2_pairs_per_block(rows, M);
    dim3 grid((rows / 2) >> lg, nimg);
    const Crop crop{in_rows, in_cols};
    const long long stride = (long long)in_rows * in_cols;
    if (fwd)
        k_rows_fwd_pad<M><<<grid, K::THREADS, smem, s>>>(static_cast<const float *>(src), static_cast<float2 *>(dst),
                                                             rows, lg, crop, stride, static_cast<const float2 *>(tw));
    else
        k_rows_inv_pad<M><<<grid, K::THREADS, smem, s>>>(static_cast<const float2 *>(src), static_cast<float *>(dst),
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

cudaError_t launch_rows_fwd(const float *img, void *spec, int rows, int cols, int nimg, const void *tw_cols,
                            cudaStream_t s, Slab slab, ImgIndirect ind) {
    switch (ilog2(cols)) {
#define GBFFT_CASE(L) \
    case L: return run_rows_fwd<(1 << L)>(img, spec, rows, nimg, tw_cols, s, slab, ind);
        GBFFT_CASE(1) GBFFT_CASE(2) GBFFT_CASE(3) GBFFT_CASE(4) GBFFT_CASE(5) GBFFT_CASE(6) GBFFT_CASE(7)
        GBFFT_CASE(8) GBFFT_CASE(9) GBFFT_CASE(10) GBFFT_CASE(11) GBFFT_CASE(12) GBFFT_CASE(13)
#undef GBFFT_CASE
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_rows_inv(const void *spec, float *out, int rows, int cols, int nimg, const void *tw_cols,
                            int *status, cudaStream_t s, Slab slab, ImgIndirect ind) {
    switch (ilog2(cols)) {
#define GBFFT_CASE(L) \
    case L: return run_rows_inv<(1 << L)>(spec, out, rows, nimg, tw_cols, status, s, slab, ind);
        GBFFT_CASE(1) GBFFT_CASE(2) GBFFT_CASE(3) GBFFT_CASE(4) GBFFT_CASE(5) GBFFT_CASE(6) GBFFT_CASE(7)
        GBFFT_CASE(8) GBFFT_CASE(9) GBFFT_CASE(10) GBFFT_CASE(11) GBFFT_CASE(12) GBFFT_CASE(13)
#undef GBFFT_CASE
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace gbfft
