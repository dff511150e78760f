// internal.h — launchers shared between the kernel files and the C ABI layer.
// Not installed; the public interface is include/gbfft.h.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace gbfft {

// Largest length the one-pass batched kernel handles (whole transform in one
// thread block); longer transforms use the two-pass four-step schedule.
constexpr int kMaxSinglePassLog2F32 = 14;  // 16384 complex64 = 128 KiB + pad
constexpr int kMaxSinglePassLog2F64 = 13;  // 8192 complex128 = 128 KiB + pad
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
cudaError_t launch_fft1d(const void *in, void *out, int log2n, long long batch, bool dbl, int dir,
                         const void *tw, double scale, cudaStream_t s);

// Four-step transform for n = n1 * n2 > one-pass maximum.
//   pass A: for each j2 < n2, length-n1 DFT over j1 of x[j1*n2 + j2] (stride n2),
//           times W_n^(k1*j2), written to tmp[k1*n2 + j2];
//   pass B: for each k1, length-n2 DFT over j2 of tmp[k1*n2 + j2], written to
//           out[k1 + n1*k2] (scaled by `scale`).
int fourstep_split(int log2n, bool dbl, int *log2n1, int *log2n2);
cudaError_t launch_fourstep_a(const void *in, void *tmp, int log2n, long long batch, bool dbl, int dir,
                              const void *tw_n1, const void *tw_4s, cudaStream_t s);
cudaError_t launch_fourstep_b(const void *tmp, void *out, int log2n, long long batch, bool dbl, int dir,
                              const void *tw_n2, double scale, cudaStream_t s);

// 2D pipeline stages (float32 images, complex64 half spectra [img][rows][cols/2],
// column 0 of a half spectrum row packs (DC, Nyquist) as (re, im)).
cudaError_t launch_rows_fwd(const float *img, void *spec, int rows, int cols, int nimg, const void *tw_cols,
                            cudaStream_t s);
// `variant` selects the column-tile width (0 = default; see cols.cu).
cudaError_t launch_cols_filter(void *spec, const float *H, long long h_stride, int rows, int cols, int nimg,
                               float scale, const void *tw_rows, cudaStream_t s, int variant = 0);
int cols_variants();
bool cols_variant_valid(int rows, int cols, int variant);
// Adjoint column pass (cols_grad.cu): per column tile, loop over nimg images of
// spec_x / spec_g, accumulate grad_H = scale * sum Re(conj(W G) W x) (added to
// grad_H's contents when `accumulate`), and filter + inverse-transform spec_g.
cudaError_t launch_cols_grad(const void *spec_x, void *spec_g, const float *H, float *grad_H, int rows, int cols,
                             int nimg, float scale, int accumulate, const void *tw_rows, cudaStream_t s);
cudaError_t launch_rows_inv(const void *spec, float *out, int rows, int cols, int nimg, const void *tw_cols,
                            cudaStream_t s);

}  // namespace gbfft
