// internal.h — launchers shared between the kernel files and the C ABI layer.
// Not installed; the public interface is include/gbfft.h.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "layout.cuh"

namespace gbfft {

// Largest length the one-pass batched kernel handles (whole transform in one
// thread block); longer transforms use the two-pass four-step schedule.
constexpr int kMaxSinglePassLog2F32 = 14;  // 16384 complex64 = 128 KiB + pad
constexpr int kMaxSinglePassLog2F64 = 13;  // 8192 complex128 = 128 KiB + pad
constexpr long long kFourStepChunkBytes = 512ll << 20;  // 1D four-step intermediate per chunk
constexpr long long kPipelineChunkBytes = 1ll << 30;     // 2D half spectra per chunk
constexpr int kMaxLog2 = 24;
constexpr int kMax2DLog2 = 13;

// Twiddle table of a length-n transform (n - 1 entries, see fft_core.cuh),
// computed in FP64 and rounded once to float (dbl = false) or kept in double.
cudaError_t launch_twiddles(void *tw, int n, bool dbl, cudaStream_t s);

// Four-step inter-pass factors W_N^(k1 * j2) for N = n1 * n2: a two-level
// table (coarse: W_N^(a * 64) for a < N/64, fine: W_N^b for b < 64).
cudaError_t launch_fourstep_twiddles(void *tw, int n, bool dbl, cudaStream_t s);

// One-pass batched C2C transform, in-place allowed.  dir = -1 forward (Eq. E2
// with `scale` = 1/n applied in the store), +1 inverse (scale 1).
// One thread-block cluster per transform for complex64 lengths 2^15 .. 2^17:
// the four-step split with its intermediate in distributed shared memory
// (the four-step plan's tables of lengths n1 and n2, and the full inter-pass
// table of launch_fourstep_full_twiddles).
bool fft1d_cluster_supported(int log2n, bool dbl);
cudaError_t launch_fft1d_cluster(const void *in, void *out, int log2n, long long batch, int dir, const void *tw_n1,
                                 const void *tw_n2, const void *tw_full, double scale, cudaStream_t s);
// complex64 table [n1][n2] of W_n^(k1 j2), each rounded once from FP64
cudaError_t launch_fourstep_full_twiddles(void *tw, int n, int log2n2, cudaStream_t s);
// One block whose bounded mbarrier wait cannot succeed: sets *status after
// `polls` tests (selftest.cu).
cudaError_t launch_wait_timeout(int *status, unsigned polls, cudaStream_t s);
// A launch the runtime refuses before it reaches the GPU (a block of 2048
// threads; the refusal does not poison the context).
cudaError_t launch_bad_config(cudaStream_t s);
// Index-bound check words of the GBFFT_CHECKED build (check.cuh), one per
// translation unit that checks: read and clear (synchronous).
cudaError_t check_take_rows(unsigned out[2]);
cudaError_t check_take_cols(unsigned out[2]);
cudaError_t check_take_batched(unsigned out[2]);
cudaError_t check_take_fourstep(unsigned out[2]);
cudaError_t check_take_tc2d(unsigned out[2]);
cudaError_t check_take_tc5(unsigned out[2]);
// Guard bands of a workspace (selftest.cu): write the fixed word into the n
// guards whose byte offsets are in the device table offs; count the 4-byte
// words that differ (or whose offset is invalid) into *bad.
cudaError_t launch_guard_fill(char *ws, const long long *offs, int n, long long ws_bytes, cudaStream_t s);
cudaError_t launch_guard_check(const char *ws, const long long *offs, int n, long long ws_bytes, unsigned *bad,
                               cudaStream_t s);
// Coarse inter-pass table of the split n = n1 n2 (n1 >= 16): entry e * n2 + j2
// holds W_(16 n2)^(e j2) = W_n^((n1/16) e j2), e < 16, j2 < n2.
cudaError_t launch_fourstep_coarse_twiddles(void *tw, int n2, bool dbl, cudaStream_t s);
cudaError_t launch_fft1d(const void *in, void *out, int log2n, long long batch, bool dbl, int dir,
                         const void *tw, double scale, cudaStream_t s);

// Four-step transform for n = n1 * n2 > one-pass maximum.
//   pass A: for each j2 < n2, length-n1 DFT over j1 of x[j1*n2 + j2] (stride n2),
//           times W_n^(k1*j2), written to tmp[k1*n2 + j2];
//   pass B: for each k1, length-n2 DFT over j2 of tmp[k1*n2 + j2], written to
//           out[k1 + n1*k2] (scaled by `scale`).
int fourstep_split(int log2n, bool dbl, int *log2n1, int *log2n2);
// tw_coarse: launch_fourstep_coarse_twiddles's table for n2.
cudaError_t launch_fourstep_a(const void *in, void *tmp, int log2n, long long batch, bool dbl, int dir,
                              const void *tw_n1, const void *tw_4s, const void *tw_coarse, int *status,
                              cudaStream_t s);
cudaError_t launch_fourstep_b(const void *tmp, void *out, int log2n, long long batch, bool dbl, int dir,
                              const void *tw_n2, double scale, int *status, cudaStream_t s);
// The same passes of complex64 with an explicit split n1 x n2 (the three-pass
// schedule below): pass A with the two-level table of n1 n2 and the coarse
// table of n2; pass B reading its row k1 from row (k1 mod 2^log2p) (n1 /
// 2^log2p) + k1 / 2^log2p of tmp when log2p > 0.
// Three passes for N = 2^24 = 256^3 (j = j1 2^16 + j2 256 + j3, k = k1 +
// 256 k2 + 2^16 k3): pass A over the 256 x 2^16 view (W_N twiddles) into
// tmp; pass A over each of its 256 rows as 256 x 256 (W_(2^16) twiddles) in
// place; pass B over rows k1 + 256 k2 (stored at k1 256 + k2, log2p = 8) into
// the output.  Every pass moves tiles of 32 transforms: 256-byte runs.
cudaError_t launch_fourstep_a_split(const void *in, void *tmp, int log2n1, int log2n2, long long batch, int dir,
                                    const void *tw_n1, const void *tw_4s, const void *tw_coarse, int *status,
                                    cudaStream_t s);
cudaError_t launch_fourstep_b_split(const void *tmp, void *out, int log2n1, int log2n2, int log2p, long long batch,
                                    int dir, const void *tw_n2, double scale, int *status, cudaStream_t s);

// 2D pipeline stages (float32 images).  Intermediate, per image: half spectra
// [cols/2][rows] complex64, column-major in slot order (layout.cuh; column 0
// packs (DC, Nyquist) of each real row); prepared filter s * Hs [cols/2][rows]
// float32 in the same order (column 0: alpha) and beta [rows].
int rows_pairs_per_block(int cols);
// Row passes of zero-padded images: fwd reads nimg in_rows x in_cols images
// (contiguous, pitch in_cols) as the top-left corner of rows x cols grids into
// spec; !fwd writes that corner of the inverse back (Sec. 5 application path).
cudaError_t launch_rows_pad(bool fwd, const void *src, void *dst, int rows, int cols, int nimg, int in_rows,
                            int in_cols, const void *tw_cols, cudaStream_t s);
// Spectrum display of one image from its row half spectra (slot order): the
// column FFTs of spec (not modified), |F| * scale into mag_T [cols/2][rows] and
// the Nyquist column into nyq [rows], both in slot order.
cudaError_t launch_cols_spectrum(const void *spec, float *mag_T, float *nyq, float scale, int rows, int cols,
                                 const void *tw_rows, cudaStream_t s);
// Forward row pass: nimg real images [rows][cols] -> half spectra
// [nimg][cols/2][rows] complex64, slot order (layout.cuh).
// With a slab (one image): only pairs slab.p0 .., into [cols/2][slab.ld].
// ind.ptrs != nullptr: image z of the launch at ind.ptrs[ind.idx[z]].img (img unused).
cudaError_t launch_rows_fwd(const float *img, void *spec, int rows, int cols, int nimg, const void *tw_cols,
                            cudaStream_t s, Slab slab = Slab{0, 0}, ImgIndirect ind = ImgIndirect{nullptr, nullptr});
// Prepared filter (rows_impl.cuh) for nimg filters H + i * h_stride into
// hs + i * hs_img, beta + i * beta_img.  kcnt > 0: only the half-spectrum
// columns kbeg .. kbeg + kcnt - 1, written as hs columns 0 .. kcnt - 1 (beta
// only when the range holds column 0).
cudaError_t launch_filter_prep(const float *H, float *hs, float *beta, int rows, int cols, int nimg, float scale,
                               long long h_stride, long long hs_img, long long beta_img, cudaStream_t s,
                               int kbeg = 0, int kcnt = 0, ImgIndirect ind = ImgIndirect{nullptr, nullptr});
// Column pass with an analytic filter computed in the kernel (no filter
// array): kind 1 Gaussian (p0 = sigma in bins), 2 Butterworth (p0 = order,
// p1 = cutoff D0 in bins), 3 disc of Eq. filtro (p0 = radius b); cols_impl.cuh.
cudaError_t launch_cols_analytic(void *spec, int kind, double p0, double p1, int rows, int cols, int nimg,
                                 const void *tw_rows, cudaStream_t s);
// hs_img / beta_img: elements between images' prepared filters (0 = shared)
// With cs.ls > 0 (one image): the column block of a decomposed image, spec in
// the received layout [ranks][cs.mloc][2^cs.ls] (layout.cuh, ColSlab), hs the
// prepared filter of those columns only.  form (columns of 4096 rows): 0 =
// default, 1 = TMA-fed with the filter in shared memory, 2 = TMA-fed with the
// filter read from global memory, 3 = one column per block.
cudaError_t launch_cols_filter(void *spec, const float *hs, const float *beta, long long hs_img, long long beta_img,
                               int rows, int cols, int nimg, const void *tw_rows, int *status, cudaStream_t s,
                               ColSlab cs = ColSlab{0, 0, 0}, int form = 0);
cudaError_t launch_rows_inv(const void *spec, float *out, int rows, int cols, int nimg, const void *tw_cols,
                            int *status, cudaStream_t s, Slab slab = Slab{0, 0},
                            ImgIndirect ind = ImgIndirect{nullptr, nullptr});
// Tensor-core variants (tc2d.cu): radix-16 passes as split-BF16 DFT-matrix
// products with `terms` = 2 or 3 BF16 parts per operand; sides 512..4096.
bool tc_supported(int rows, int cols);
bool onchip_supported(int rows, int cols);
cudaError_t launch_onchip(const float *img, const float *H, float *out, long long h_stride, int rows, int cols,
                          int nimg, const void *tw_cols, const void *tw_rows, cudaStream_t s,
                          ImgIndirect ind = ImgIndirect{nullptr, nullptr});
cudaError_t launch_rows_tc(bool fwd, const void *src, void *dst, int rows, int cols, int nimg, const void *tw,
                           int terms, cudaStream_t s);
cudaError_t launch_cols_tc(void *spec, const float *hs, const float *beta, long long hs_img, long long beta_img,
                           int rows, int cols, int nimg, const void *tw_rows, int terms, cudaStream_t s);
// Fifth-generation tensor-core variants (tc5_2d.cu, tcgen05.mma): fmt 0 =
// BF16 x 2 parts (3 products), 1 = BF16 x 3 (6 products), 2 = TF32 x 2 (3
// products); sides 512..4096; a bounded MMA wait that gives up sets *status.
cudaError_t launch_rows_tc5(bool fwd, const void *src, void *dst, int rows, int cols, int nimg, const void *tw,
                            int fmt, int *status, cudaStream_t s);
cudaError_t launch_cols_tc5(void *spec, const float *hs, const float *beta, long long hs_img, long long beta_img,
                            int rows, int cols, int nimg, const void *tw_rows, int fmt, int *status, cudaStream_t s);
// Adjoint column pass (cols_grad.cu): per column, loop over nimg images of
// spec_x / spec_g, accumulate scale * sum Re(conj(W G) W x) into grad_T
// [cols/2 + 1][rows] (slot order; added to its contents when `accumulate`),
// and filter + inverse-transform spec_g in place.  Shared filter only.
cudaError_t launch_cols_grad(const void *spec_x, void *spec_g, const float *hs, const float *beta, float *grad_T,
                             int rows, int cols, int nimg, float scale, int accumulate, const void *tw_rows,
                             cudaStream_t s);
// grad_T [cols/2][rows] and the Nyquist column nyq [rows] (slot order) ->
// grad_H [rows][cols] row-major (both bins of every mirror pair).
cudaError_t launch_grad_scatter(const float *grad_T, const float *nyq, float *grad_H, int rows, int cols,
                                cudaStream_t s);

}  // namespace gbfft
