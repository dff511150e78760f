/*
 * gbfft.h — C ABI of the GB300 FFT -> filter -> IFFT library (libgbfft.so).
 *
 * The library computes the transforms of Higuera, Sarria, Fonseca and
 * Idarraga, "Construction of an algorithm in parallel for the Fast Fourier
 * Transform" (arXiv cs/0103001) with hand-written CUDA kernels for sm_103a:
 *
 *   forward (Eq. E2 / Eq. coefFourier):  c_k = (1/N) sum_j f_j exp(-2 pi i k j / N)
 *   inverse (Eq. E3 at x_j = 2 pi j/N):  f_j = sum_k c_k exp(+2 pi i k j / N)   (no scale)
 *   2D (Sec. 4): rows, then columns; the per-axis convention (1/M on rows,
 *      1/N on columns) by default, Eq. 5 on request
 *   application (Sec. 5): out = Re(ifft2(H . fft2(img))) for a real image and
 *      a real filter H given in natural (unshifted) frequency order
 *
 * Conventions for every entry point:
 *   - Each call returns an int status (gbfft_status); nothing throws or exits.
 *   - Every data pointer is a DEVICE pointer owned by the caller, aligned to
 *     16 bytes (else GBFFT_ERR_MISALIGNED).  The library allocates no device
 *     memory: the caller provides a workspace sized by
 *     fft_plan_workspace_bytes() and binds it with fft_plan_bind_workspace().
 *   - Work is enqueued on the given stream and is asynchronous to the host.
 *     A plan holds host state only; one plan must not be used from two
 *     streams or threads at the same time.
 *   - Complex data are interleaved (re, im): complex64 = 2 x float32,
 *     complex128 = 2 x float64 (the paper ships each complex as a pair of
 *     real columns, Sec. 2).
 *   - Lengths are powers of two, N = 2^m with m >= 1 (Sec. 3); other lengths
 *     return GBFFT_ERR_INVALID_SIZE.
 *   - Launch failures are reported as GBFFT_ERR_CUDA; gbfft_last_cuda_error()
 *     gives the CUDA error code.
 */
#ifndef GBFFT_H
#define GBFFT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* A CUDA stream (layout-compatible with cudaStream_t); NULL = legacy stream. */
typedef struct CUstream_st *gbfft_stream_t;

typedef struct gbfft_plan *gbfft_plan_t;

/* Device-resident pointers of one image of a batched call (see
 * fft2_filter_ifft2_batched): its float32 image, filter and output, each
 * rows x cols row-major, 16-byte aligned. */
typedef struct {
    const float *img;
    const float *H;
    float *out;
} gbfft_image_ptrs;

typedef enum {
    GBFFT_C64 = 1,  /* complex64: float32 pairs; 2D images are float32 */
    GBFFT_C128 = 2, /* complex128: float64 pairs; 2D images are float64 */
} gbfft_dtype;

typedef enum {
    GBFFT_OK = 0,
    GBFFT_ERR_NULL = -1,         /* a required pointer is NULL */
    GBFFT_ERR_INVALID_SIZE = -2, /* length not 2^m, m out of range, batch < 1 */
    GBFFT_ERR_DTYPE = -3,        /* unknown or unsupported dtype for this call */
    GBFFT_ERR_MISALIGNED = -4,   /* a data pointer is not 16-byte aligned */
    GBFFT_ERR_WORKSPACE = -5,    /* no workspace bound, or the one given is too small */
    GBFFT_ERR_UNSUPPORTED = -6,  /* valid request the library does not implement */
    GBFFT_ERR_CUDA = -7,         /* a CUDA call or kernel launch failed */
    GBFFT_ERR_TIMEOUT = -8,      /* a bounded device-side wait gave up */
    GBFFT_ERR_INVALID_VALUE = -9 /* bad option key/value or wrong plan kind */
} gbfft_status;

/* Plan options (fft_plan_set_option). */
typedef enum {
    /* 2D scale convention: 0 = per-axis (default; forward 1/(N M), inverse 1),
     * 1 = Eq. 5 (forward 1/N with N = rows, inverse 1/M).  The filtered image
     * of fft2_filter_ifft2 is the same under both. */
    GBFFT_OPT_SCALE_CONVENTION = 1,
    /* Element stride between the filters of consecutive images in a batch:
     * 0 (default) shares one H; rows*cols gives each image its own.  Changes
     * fft_plan_workspace_bytes (one prepared filter per image in a chunk). */
    GBFFT_OPT_H_BATCH_STRIDE = 2,
    /* Arithmetic of the 2D pipeline's radix-16 passes: 0 = FP32 butterflies
     * (default); tensor cores with each operand split into narrower parts
     * and FP32 accumulation, on the warp-level MMA (mma.sync): 1 = 2 BF16
     * parts, 3 products (about 16 significant bits per pass), 2 = 3 BF16
     * parts, 6 products (about 24 bits); on the fifth-generation tensor
     * cores (tcgen05.mma, accumulators in tensor memory): 3 = 2 BF16 parts
     * (3 products), 4 = 3 BF16 parts (6 products), 5 = 2 TF32 parts (3
     * products, about 22 bits).  Nonzero values need a 2D plan with sides
     * 512..4096 (else GBFFT_ERR_UNSUPPORTED); the filter gradient of the
     * adjoint is always computed with FP32 butterflies. */
    GBFFT_OPT_PRECISION = 3,
    /* 2D: number of images whose spectra share the workspace at a time
     * (0 = as many as 1 GiB of half spectra holds, at most the batch).
     * Changes fft_plan_workspace_bytes. */
    GBFFT_OPT_IMAGES_PER_CHUNK = 4,
    /* 1 = record a CUDA event pair around every kernel launch of this plan
     * (read with gbfft_plan_profile_read) and run every kernel on the
     * caller's stream, one after the other, so each pair times one kernel;
     * 0 (default) = off. */
    GBFFT_OPT_PROFILE = 5,
    /* 2D: 1 = reserve the second spectrum buffer that the filter gradient of
     * fft2_filter_ifft2_backward needs (doubles the spectrum part of the
     * workspace); 0 (default) = forward and grad_img only. */
    GBFFT_OPT_ENABLE_BACKWARD = 6,
    /* Batched plans: thread blocks per SM of each persistent stage launch
     * (0 = as many as fit, the default; fft_plan_autotune sets it per stage).
     * fft_plan_get_option returns the four stages packed 8 bits each, from
     * the low byte: forward rows, columns, inverse rows, filter preparation. */
    GBFFT_OPT_BLOCKS_PER_SM = 7,
    /* Batched plans: 1 (default) = capture the three stage launches in a CUDA
     * graph on the first call and replay it while the image-pointer array and
     * the launch shapes stay the same; 0 = plain launches. */
    GBFFT_OPT_USE_GRAPH = 8,
    /* One-launch cluster paths.  2D plans with both sides 16..256: 1 (default)
     * or 2 = the whole pipeline of fft2_filter_ifft2 in one launch, one
     * thread-block cluster per image holding its half spectra in shared
     * memory (ignored with GBFFT_OPT_PRECISION != 0); 0 = the three-pass
     * path.  1D complex64 plans of length 2^15..2^17: 2 = one cluster per
     * transform, the four-step intermediate in distributed shared memory (one
     * HBM read and one write instead of two each); 0 or 1 (default) = the
     * four-step passes, which are faster at these lengths.  Same results up
     * to rounding order. */
    GBFFT_OPT_ONCHIP = 9,
    /* 2D plans, the fused column pass over columns of 4096 rows: 0 (default)
     * = the plan's choice (fft_plan_autotune's, else 1); 1 = persistent and
     * TMA-fed, the filter column bulk-copied beside its column; 2 = the same
     * with the filter read from global memory; 3 = one column per block.
     * Same results; other heights have one form. */
    GBFFT_OPT_COLUMN_FORM = 10,
    /* Batched plans: 0 (default) = the one-shape kernels once per shape class
     * over that class's images (reached through the image-pointer array),
     * the filter preparations and the small classes' on-chip pipelines on a
     * side stream; 1 = four persistent launches over largest-first work
     * lists of every image (GBFFT_OPT_BLOCKS_PER_SM applies).  Same results. */
    GBFFT_OPT_BATCH_FORM = 11,
    /* 1D complex64 plans of length 2^24: 3 (default, 0) = three passes of
     * length-256 transforms (N = 256^3: two column passes, the second in
     * place, and one row pass with transposed stores), each moving tiles of
     * 32 transforms (256-byte runs in HBM); 2 = the two passes of 4096 of
     * every other length, whose tiles hold 4 transforms (32-byte runs).  The
     * workspace changes: query fft_plan_workspace_bytes and bind again.
     * Same results up to rounding order. */
    GBFFT_OPT_FOURSTEP_PASSES = 12
} gbfft_option;

/* Stages reported by gbfft_plan_profile_read.  With the environment
 * variable GBFFT_NVTX=1 every stage launch is also wrapped in an NVTX range
 * named "gbfft <stage>" (fft1d, fourstep_a, ..., as below) for a profiler's
 * timeline. */
typedef enum {
    GBFFT_STAGE_FFT1D = 0,     /* one-pass batched 1D transform */
    GBFFT_STAGE_FOURSTEP_A = 1,/* four-step pass A (column FFTs + twiddle) */
    GBFFT_STAGE_FOURSTEP_B = 2,/* four-step pass B (row FFTs, transposed store) */
    GBFFT_STAGE_ROWS_FWD = 3,  /* 2D row pass, forward (real rows -> half spectra) */
    GBFFT_STAGE_COLS = 4,      /* 2D fused column pass: FFT -> x s H -> IFFT */
    GBFFT_STAGE_ROWS_INV = 5,  /* 2D row pass, inverse (half spectra -> real rows) */
    GBFFT_STAGE_COLS_GRAD = 6, /* 2D fused column pass of the adjoint (grad_H) */
    GBFFT_STAGE_TWIDDLES = 7,  /* twiddle-table generation (bind time) */
    GBFFT_STAGE_GRAPH = 8,     /* one replay of a batched plan's captured graph */
    GBFFT_STAGE_FILTER_PREP = 9, /* 2D: even part of the filter, slot order (side stream) */
    GBFFT_STAGE_ONCHIP = 10,   /* 2D small images: the whole pipeline in one cluster launch */
    GBFFT_STAGE_SPECTRUM = 11, /* 2D spectrum display: column FFTs, magnitudes, row-major write */
    GBFFT_STAGE_FFT1D_CLUSTER = 12, /* 1D 2^15..2^17: one thread-block cluster per transform */
    GBFFT_STAGE_COUNT = 13
} gbfft_stage;

/* ---- plans --------------------------------------------------------------- */

/* 1D batched complex-to-complex plan: `batch` contiguous transforms of length
 * n = 2^m, 1 <= m <= 24 (Eq. E2 forward, Eq. E3 inverse).  dtype C64 or C128.
 * On success *out receives a new plan (free with fft_plan_destroy). */
int fft_plan_create(int64_t n, int64_t batch, int dtype, gbfft_plan_t *out);

/* 2D plan for the Sec. 5 pipeline on `batch` real images of rows x cols
 * (row-major, rows = N = 2^a, cols = M = 2^b, 2 <= N, M <= 8192).
 * dtype C64 (float32 images). */
int fft2_plan_create(int64_t rows, int64_t cols, int64_t batch, int dtype, gbfft_plan_t *out);

/* Set a gbfft_option.  Returns GBFFT_ERR_INVALID_VALUE for an unknown key or
 * an out-of-range value.  Options that change the workspace size must be set
 * before fft_plan_bind_workspace. */
int fft_plan_set_option(gbfft_plan_t plan, int key, int64_t value);

/* Bytes of device workspace the plan needs (twiddle tables + spectra). */
int fft_plan_workspace_bytes(gbfft_plan_t plan, size_t *bytes);

/* Bind caller-owned device memory (>= fft_plan_workspace_bytes, 256-byte
 * aligned) as the plan's workspace and enqueue the generation of its twiddle
 * tables on `stream` (FP64 arithmetic, each factor rounded once).  The memory
 * must stay valid until the plan is destroyed or re-bound. */
int fft_plan_bind_workspace(gbfft_plan_t plan, void *workspace, size_t bytes, gbfft_stream_t stream);

/* 1D forward transform of a 1D plan: out = (1/N) DFT(in) per transform
 * (Eq. E2).  in and out hold batch x n complex values of the plan's dtype;
 * in == out (in place) is allowed, partial overlap is not. */
int fft_forward(gbfft_plan_t plan, const void *in, void *out, gbfft_stream_t stream);

/* 1D inverse transform: out_j = sum_k in_k exp(+2 pi i j k / N), unscaled
 * (Eq. E3).  Same layout and aliasing rules as fft_forward. */
int fft_inverse(gbfft_plan_t plan, const void *in, void *out, gbfft_stream_t stream);

/* Sec. 5 pipeline on a 2D plan: for each image b,
 *   out_b = Re(ifft2(H_b . fft2(img_b)))
 * img, out: batch x rows x cols float32 (row-major).  H: rows x cols float32
 * real filter in natural (unshifted) DFT order; image b uses
 * H + b * h_batch_stride (option GBFFT_OPT_H_BATCH_STRIDE, default 0).
 * The filter multiplies the real and the imaginary part of every spectral
 * value.  img == out is allowed.  The filter preparation runs on a side
 * stream of the plan, forked from and joined back to `stream` with events,
 * so the call stays ordered on `stream` (and can be captured in a graph). */
int fft2_filter_ifft2(gbfft_plan_t plan, const float *img, const float *H, float *out, gbfft_stream_t stream);

/* The same pipeline with one filter for many calls (Sec. 5's filter, fixed
 * while the images change, e.g. one PSF or low-pass over a stack of frames):
 * fft2_filter_prepare computes the filter's prepared form (the even part
 * s * Hs of the rows x cols real H, column-major, with the packed column's
 * alpha and beta) into the plan's workspace on `stream`;
 * fft2_filter_ifft2_prepared then runs the pipeline on `batch` images with
 * it, without reading H and without the preparation: results equal
 * fft2_filter_ifft2 with that H.  Needs a shared filter
 * (GBFFT_OPT_H_BATCH_STRIDE 0, else GBFFT_ERR_UNSUPPORTED).  The prepared
 * filter lives in the workspace region that fft2_filter_ifft2, _padded,
 * _backward, fft2_spectrum and fft_plan_autotune also use: any of those
 * calls, a new bind or an option that changes the workspace discards it, and
 * fft2_filter_ifft2_prepared then returns GBFFT_ERR_INVALID_VALUE until the
 * next fft2_filter_prepare.  Small sides (the on-chip path) run the
 * three-pass kernels here. */
int fft2_filter_prepare(gbfft_plan_t plan, const float *H, gbfft_stream_t stream);
int fft2_filter_ifft2_prepared(gbfft_plan_t plan, const float *img, float *out, gbfft_stream_t stream);

/* Sec. 5's application path for images whose sides are not powers of two:
 * each of the plan's `batch` images is in_rows x in_cols float32 (row-major,
 * contiguous, image b at img + b * in_rows * in_cols), 1 <= in_rows <= rows,
 * 1 <= in_cols <= cols of the plan.  The image is zero-padded to the plan's
 * rows x cols grid (zeros after its last row and last column), filtered as in
 * fft2_filter_ifft2 with H (rows x cols, on the padded grid, 16-byte aligned;
 * h_batch_stride applies), and the in_rows x in_cols top-left corner of the
 * result is written to out (same layout as img).  img and out need only
 * 4-byte alignment; img == out is allowed.  GBFFT_ERR_INVALID_SIZE for sizes
 * out of range; GBFFT_ERR_UNSUPPORTED with GBFFT_OPT_PRECISION != 0. */
int fft2_filter_ifft2_padded(gbfft_plan_t plan, const float *img, int64_t in_rows, int64_t in_cols, const float *H,
                             float *out, gbfft_stream_t stream);

/* Analytic filters of fft2_filter_ifft2_analytic. */
typedef enum {
    GBFFT_FILTER_GAUSSIAN = 1,    /* exp(-|f|^2 / (2 p0^2)); p0 = sigma in bins */
    GBFFT_FILTER_BUTTERWORTH = 2, /* 1 / (1 + (|f| / p1)^(2 p0)); p0 = order 1..16, p1 = cutoff in bins */
    GBFFT_FILTER_DISC = 3         /* Eq. filtro: 0 where (u - rows/2)^2 + (v - cols/2)^2 <= p0^2, else 1 */
} gbfft_filter_kind;

/* fft2_filter_ifft2 with a filter given by formula instead of an array: the
 * column pass computes H[u][v] for each bin (|f|^2 = u~^2 + v~^2 over the
 * wrapped bins, u~ = u for u < rows/2, u - rows above), so no filter is read
 * and none is prepared.  The three filters are even (H[-u][-v] = H[u][v]).
 * Same layouts, batching and aliasing as fft2_filter_ifft2 (FP32 path; with
 * GBFFT_OPT_PRECISION != 0, GBFFT_ERR_UNSUPPORTED).  GBFFT_ERR_INVALID_VALUE
 * for an unknown kind or parameters out of range. */
int fft2_filter_ifft2_analytic(gbfft_plan_t plan, const float *img, int kind, double p0, double p1, float *out,
                               gbfft_stream_t stream);

/* Spectrum display of Sec. 5: mag = sqrt(Re^2 + Im^2) of the 2D transform of
 * each image, zero-padded to the plan's grid as in fft2_filter_ifft2_padded
 * (in_rows = rows, in_cols = cols for no padding).  mag: batch x rows x cols
 * float32, natural (unshifted) frequency order, scaled per the plan's
 * GBFFT_OPT_SCALE_CONVENTION (per-axis: the DFT divided by rows * cols;
 * Eq. 5: by rows only).  Uses the plan's prepared-filter workspace as scratch:
 * a following fft2_filter_ifft2 prepares its filter again as usual. */
int fft2_spectrum(gbfft_plan_t plan, const float *img, int64_t in_rows, int64_t in_cols, float *mag,
                  gbfft_stream_t stream);

/* Adjoint of fft2_filter_ifft2 for an upstream gradient grad_out = dL/dout
 * (derived from Sec. 4's 2D-DFT and Sec. 5's filter; the paper has no
 * gradient):
 *   grad_img_b = Re(ifft2(H . fft2(grad_out_b)))          (same shape as img)
 *   grad_H[k]  = N M sum_b Re(conj(fft2(grad_out_b)[k]) fft2(img_b)[k])
 * with per-axis spectra.  grad_H (rows x cols float32) is overwritten with
 * the sum over the batch; it needs a shared H (h_batch_stride 0,
 * else GBFFT_ERR_UNSUPPORTED) and GBFFT_OPT_ENABLE_BACKWARD set before the
 * workspace is bound (else GBFFT_ERR_WORKSPACE).  grad_img or grad_H may be
 * NULL to skip that output; img may be NULL when grad_H is. */
int fft2_filter_ifft2_backward(gbfft_plan_t plan, const float *img, const float *H, const float *grad_out,
                               float *grad_img, float *grad_H, gbfft_stream_t stream);

/* Allocation-free form of fft2_filter_ifft2 (the paper has no counterpart;
 * it exists for callers that cannot allocate device memory while running:
 * loops that must not call cudaMalloc because it can block or synchronise
 * the device, and plugins whose host application owns every device
 * allocation and passes them only their inputs and outputs).
 * Same result as fft2_filter_ifft2 for `batch` float32 images of
 * rows x cols (row-major); image b uses filter H + b * h_batch_stride
 * (0 = one shared filter).  No plan and no workspace: the scratch memory is a
 * fixed device array inside the library (about 24.2 MiB, held on every GPU
 * that loads the library until the process exits).
 *   - rows, cols powers of two >= 2 with rows * cols <= 2048 * 2048; larger
 *     images return GBFFT_ERR_INVALID_SIZE.
 *   - The first call on a device sets that device up (with that device
 *     current): it looks the array up with cudaGetSymbolAddress, writes the
 *     twiddle tables of every length into it on `stream` and waits for
 *     them (cudaStreamSynchronize).  Make that first call before any stream
 *     capture.  Later calls never rewrite the tables.
 *   - All calls share the array and it keeps the last call's contents:
 *     calls that overlap on the GPU (other streams, unordered threads) race.
 *     Nothing in it needs to start at zero.
 *   - Allocates nothing: no cudaMalloc, cudaFree or allocating library call. */
int fft2_filter_ifft2_noalloc(int64_t rows, int64_t cols, int64_t batch, const float *img, const float *H,
                              int64_t h_batch_stride, float *out, gbfft_stream_t stream);

/* ---- one image decomposed over ranks (row slabs) ---------------------------
 *
 * The paper spreads its transform over 2^l processes, each computing its share
 * before the processes exchange results (Sec. 2, cost model Eq. multi /
 * Table 1).  These calls split one image of fft2_filter_ifft2 over `nranks`
 * ranks (one GPU each, or emulated on one GPU) by rows instead, with two
 * exchanges and no other communication:
 *   1. fft2_slab_rows_forward: rank r transforms its rows into `send`;
 *   2. exchange 1: chunk q of every rank's `send` goes to rank q, where the
 *      chunks arrive in rank order as `recv` (an all-to-all of equal chunks);
 *   3. fft2_slab_columns: rank r filters its block of spectrum columns in
 *      `recv` in place (column FFT, x s.Hs, column IFFT);
 *   4. exchange 2: chunk q of every rank's `recv` goes back to rank q, arriving
 *      in rank order as `back` (the same all-to-all);
 *   5. fft2_slab_rows_inverse: rank r writes its rows of `out`.
 * The exchanges are the caller's (e.g. NCCL all-to-all); every buffer holds
 * fft2_slab_exchange_elems() complex64 values, split into nranks equal
 * contiguous chunks.  The result equals fft2_filter_ifft2 on the whole image.
 *
 * Rank r owns the row pairs (p, rows - p) for p in [r P, (r + 1) P), P =
 * rows / (2 nranks) (pair 0 is rows 0 and rows/2): its rows are two runs,
 * [rP, (r+1)P) and the mirrors.  Its columns are the half-spectrum columns
 * [r C, (r + 1) C), C = cols / (2 nranks).  `img` and `out` are whole
 * rows x cols float32 images in the rank's memory; only the rank's own rows
 * are read and written.  rows, cols powers of two, cols >= 4, nranks a power
 * of two with P a positive multiple of the row pass's pairs per block (2 for
 * cols >= 256) and C >= 1, else GBFFT_ERR_INVALID_SIZE; rank outside
 * [0, nranks): GBFFT_ERR_INVALID_VALUE.  The plan's workspace (twiddles and
 * the rank's share of the prepared filter) is bound as usual. */
int fft2_slab_plan_create(int64_t rows, int64_t cols, int nranks, int rank, gbfft_plan_t *out);
/* Complex64 elements in each exchange buffer: (cols/2) x (rows/nranks). */
int fft2_slab_exchange_elems(gbfft_plan_t plan, int64_t *count);
/* Step 1: rows of this rank -> send, laid out [cols/2][rows/nranks]. */
int fft2_slab_rows_forward(gbfft_plan_t plan, const float *img, void *send, gbfft_stream_t stream);
/* Step 3: recv ([nranks][C][rows/nranks], chunk q from rank q) filtered in
 * place with H (rows x cols float32, the whole filter, on every rank). */
int fft2_slab_columns(gbfft_plan_t plan, void *recv, const float *H, gbfft_stream_t stream);
/* Step 5: back ([cols/2][rows/nranks], as step 1 wrote it) -> this rank's rows of out. */
int fft2_slab_rows_inverse(gbfft_plan_t plan, const void *back, float *out, gbfft_stream_t stream);

/* Batched plan for the Sec. 5 pipeline over `count` images of uneven sizes,
 * image i being rows[i] x cols[i] (powers of two, 16 <= rows, cols <= 4096),
 * each with its own filter of the same shape.  All images' spectra live in
 * the workspace at once (fft_plan_workspace_bytes); binding it uploads the
 * image table and the per-stage work lists and builds the twiddle tables. */
int fft2_batched_plan_create(int count, const int64_t *rows, const int64_t *cols, gbfft_plan_t *out);

/* Run a batched plan: out_i = Re(ifft2(H_i . fft2(img_i))) for every image.
 * `images` is a DEVICE array of `count` gbfft_image_ptrs (caller-owned; the
 * kernels read it when they run).  GBFFT_OPT_BATCH_FORM 0 (default): the
 * one-shape kernels once per shape class over that class's images (filter
 * preparations and the on-chip pipelines of sides <= 256 on a side stream);
 * 1: four persistent launches (filter preparation, forward rows, fused
 * columns, inverse rows), each over a largest-first work list of all
 * images.  With GBFFT_OPT_USE_GRAPH (default on) the launches are captured
 * once in a CUDA graph (on a private stream) and replayed on `stream`; the
 * graph is captured again when `images` points elsewhere. */
int fft2_filter_ifft2_batched(gbfft_plan_t plan, const gbfft_image_ptrs *images, gbfft_stream_t stream);

/* Device buffers the autotuner runs a 1D or 2D plan on (host struct):
 * 1D: in, out as for fft_forward (H unused); 2D: in = img, H, out as for
 * fft2_filter_ifft2.  `out` is written. */
typedef struct {
    const void *in;
    const float *H;
    void *out;
} gbfft_tune_args;

/* Tune a plan by timing its candidate configurations on `stream` (blocking;
 * each candidate's median of 7 runs; a later candidate replaces an earlier
 * one only if more than 1 % faster, so ties keep the default) and keep the
 * fastest in the plan's options:
 *   2D plans: GBFFT_OPT_COLUMN_FORM for columns of 4096 rows, and
 *     GBFFT_OPT_ONCHIP (on-chip or three-pass) for sides <= 256;
 *     args = a gbfft_tune_args.
 *   1D plans: the one-cluster path against the four-step passes for complex64
 *     lengths 2^15..2^17 (GBFFT_OPT_ONCHIP); args = a gbfft_tune_args.
 *   Batched plans: blocks per SM of each persistent stage
 *     (GBFFT_OPT_BLOCKS_PER_SM), then the form (GBFFT_OPT_BATCH_FORM);
 *     args = the device image array of fft2_filter_ifft2_batched.
 *   Slab plans: nothing to tune (GBFFT_OK).
 * Results are cached in a JSON file keyed by the GPU's name and SM count and
 * the plan's shape: a later call for the same key applies the stored choice
 * without timing.  The file is $GBFFT_TUNE_CACHE (empty: no cache), else
 * $XDG_CACHE_HOME/gbfft/tune.json or $HOME/.cache/gbfft/tune.json; a file
 * that cannot be read or written only means tuning again.  Every candidate
 * computes the same result (up to rounding order). */
int fft_plan_autotune(gbfft_plan_t plan, const void *args, gbfft_stream_t stream);

/* Read back an option (GBFFT_OPT_IMAGES_PER_CHUNK gives the chunk in use). */
int fft_plan_get_option(gbfft_plan_t plan, int key, int64_t *value);

/* Destroy a plan (host state only; the workspace belongs to the caller). */
int fft_plan_destroy(gbfft_plan_t plan);

/* ---- diagnostics ---------------------------------------------------------- */

/* Static string for a status code. */
const char *gbfft_status_string(int status);

/* The cudaError_t code behind the last GBFFT_ERR_CUDA on this host thread. */
int gbfft_last_cuda_error(void);

/* With GBFFT_OPT_PROFILE on: wait for the recorded events, add the elapsed
 * milliseconds and launch counts per gbfft_stage into ms[0..nstages) and
 * launches[0..nstages) (either may be NULL), then forget the records. */
int gbfft_plan_profile_read(gbfft_plan_t plan, double *ms, int64_t *launches, int nstages);

/* Read and clear the plan's device status word (synchronous: waits for the
 * plan's work on the device).  Kernels that wait on asynchronous copies (the
 * TMA-fed four-step passes of 1D complex64 plans and column pass of 2D plans)
 * wait a bounded time; one that gives up leaves its outputs unwritten and
 * records it here: GBFFT_ERR_TIMEOUT.  GBFFT_OK otherwise. */
int gbfft_device_status(gbfft_plan_t plan);

/* Guard bands (a stand-in for a memory checker, in every build): the plan's
 * workspace holds 256 bytes of a fixed pattern before, between and after its
 * regions (twiddle tables, prepared filters, spectra, work lists, ...),
 * written when the workspace is bound.  This call waits for the device
 * (cudaDeviceSynchronize), checks every band and writes the number of 4-byte
 * words found changed to *bad_words (0: no kernel wrote outside its region
 * into a band).  GBFFT_ERR_WORKSPACE if no workspace is bound. */
int gbfft_plan_check_guards(gbfft_plan_t plan, int64_t *bad_words);

/* Index-bound checks (a stand-in for a memory checker): in the library built
 * with GBFFT_CHECKED (libgbfft_checked.so), the kernels check the index
 * arithmetic of their pair and slot runs, tensor-map boxes, work-list items
 * and tensor-memory columns; a failing check records its site code (see
 * check.cuh) and the access is skipped (no trap).  This call waits for the
 * device, then writes the first failing site (0 = none) and the number of
 * failures since the last call, and clears them.  GBFFT_ERR_UNSUPPORTED in
 * the normal build. */
int gbfft_checked_take(int64_t *first_site, int64_t *failures);

/* Diagnostic of that path: launches on `stream` one block that waits on an
 * mbarrier no copy will ever complete, testing it at most `polls` times
 * (1 .. 2^22, each test followed by a 64 ns sleep); the wait gives up, records
 * a timeout in the plan's device status word, and the block returns.  The
 * next gbfft_device_status returns GBFFT_ERR_TIMEOUT.  Needs a bound
 * workspace; GBFFT_ERR_INVALID_VALUE for polls out of range. */
int gbfft_selftest_wait_timeout(gbfft_plan_t plan, int64_t polls, gbfft_stream_t stream);

/* Fault injection on the host, for tests of the failure paths (no GPU
 * fault is ever made):
 * gbfft_selftest_corrupt_work_item overwrites work item `index` of stage
 * `stage` (0 forward rows, 1 columns, 2 inverse rows, 3 filter preparation)
 * of a batched plan's host tables with (img, bx) and marks the plan unbound;
 * fft_plan_bind_workspace checks every item against its image's launch shape
 * before anything reaches the GPU and returns GBFFT_ERR_INVALID_VALUE for an
 * item out of range (GBFFT_ERR_INVALID_VALUE here for a plan that is not
 * batched or an index out of range).
 * gbfft_selftest_launch_config makes a launch the CUDA runtime refuses
 * (a block of 2048 threads) on `stream` and returns its status:
 * GBFFT_ERR_CUDA, with gbfft_last_cuda_error() the runtime's refusal code
 * (cudaErrorInvalidValue under CUDA 13); the refusal leaves the context
 * usable. */
int gbfft_selftest_corrupt_work_item(gbfft_plan_t plan, int stage, int64_t index, int img, int bx);
int gbfft_selftest_launch_config(gbfft_stream_t stream);

/* Diagnostic (the paper has no counterpart): measures the GPU's FMA
 * throughput, fp64 = 1 in double precision (the ALU roofline of the
 * complex128 transforms), 0 in single precision.  Runs a few short launches
 * of independent FMA chains on `stream` (all SMs) and waits for them; writes
 * the best rate in FLOP/s (2 per FMA) to *flops_per_s.  Allocates nothing.
 * GBFFT_ERR_NULL for a NULL output, GBFFT_ERR_INVALID_VALUE for fp64 not 0/1. */
int gbfft_measure_fma_peak(int fp64, double *flops_per_s, gbfft_stream_t stream);

/* Library version as 10000*major + 100*minor + patch. */
int gbfft_version(void);

#ifdef __cplusplus
}
#endif

#endif /* GBFFT_H */
