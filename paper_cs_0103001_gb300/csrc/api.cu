// api.cu — the C ABI of include/gbfft.h: plans, validation, workspace layout
// and the launch sequences.  Host code only; kernels live in the other files.
#include <cuda_runtime.h>
#include <stdint.h>

#include <new>
#include <vector>

#include "gbfft.h"
#include "internal.h"

using namespace gbfft;

namespace {

thread_local int g_last_cuda_error = 0;

struct ProfRec {
    int stage;
    cudaEvent_t a, b;
};

enum PlanKind { KIND_1D = 1, KIND_2D = 2 };

constexpr size_t kAlign = 256;
size_t align_up(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }

int ilog2_exact(int64_t n) {
    if (n < 1 || (n & (n - 1))) return -1;
    int l = 0;
    while ((int64_t(1) << l) < n) ++l;
    return l;
}

}  // namespace

struct gbfft_plan {
    int kind = 0;
    int dtype = 0;
    int64_t batch = 0;
    int log2n = 0;               // 1D length
    int log2r = 0, log2c = 0;    // 2D rows (N) and cols (M)
    int64_t opt_scale_conv = 0, opt_h_stride = 0, opt_precision = 0, opt_chunk = 0, opt_profile = 0;
    int64_t opt_backward = 0, opt_cols_variant = 0;
    // workspace
    char *ws = nullptr;
    size_t ws_bytes = 0;
    bool bound = false;
    // layout (byte offsets into ws)
    size_t off_tw0 = 0, off_tw1 = 0, off_tw2 = 0, off_buf = 0, off_buf2 = 0, need = 0;
    int64_t chunk = 0;           // transforms (1D four-step) or images (2D) per workspace chunk
    int fs_l1 = 0, fs_l2 = 0;    // four-step split
    std::vector<ProfRec> prof;
};

namespace {

bool is_dbl(const gbfft_plan *p) { return p->dtype == GBFFT_C128; }
size_t csize(const gbfft_plan *p) { return is_dbl(p) ? 16 : 8; }

int max_single_log2(const gbfft_plan *p) { return is_dbl(p) ? kMaxSinglePassLog2F64 : kMaxSinglePassLog2F32; }

int64_t l2_budget_bytes() {
    int dev = 0, l2 = 0;
    if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev) == cudaSuccess &&
        l2 > 0)
        return (int64_t)l2 * 3 / 8;
    cudaGetLastError();
    return 48ll << 20;
}

// Compute the workspace layout for the current options.
void layout(gbfft_plan *p) {
    size_t off = 0;
    if (p->kind == KIND_1D) {
        const int64_t n = int64_t(1) << p->log2n;
        if (p->log2n <= max_single_log2(p)) {
            p->off_tw0 = off;
            off = align_up(off + (size_t)n * csize(p));
            p->off_tw1 = p->off_tw2 = p->off_buf = off;
            p->chunk = p->batch;
        } else {
            fourstep_split(p->log2n, is_dbl(p), &p->fs_l1, &p->fs_l2);
            const int64_t n1 = int64_t(1) << p->fs_l1, n2 = int64_t(1) << p->fs_l2;
            const int lf = (p->log2n + 1) / 2;
            const int64_t n4s = (int64_t(1) << lf) + (n >> lf);
            p->off_tw0 = off;
            off = align_up(off + (size_t)n1 * csize(p));
            p->off_tw1 = off;
            off = align_up(off + (size_t)n2 * csize(p));
            p->off_tw2 = off;
            off = align_up(off + (size_t)n4s * csize(p));
            p->off_buf = off;
            int64_t chunk = p->opt_chunk;
            if (chunk <= 0) {
                chunk = l2_budget_bytes() / (n * (int64_t)csize(p));
                if (chunk < 1) chunk = 1;
            }
            if (chunk > p->batch) chunk = p->batch;
            p->chunk = chunk;
            off = align_up(off + (size_t)chunk * n * csize(p));
        }
    } else {
        const int64_t rows = int64_t(1) << p->log2r, cols = int64_t(1) << p->log2c;
        p->off_tw0 = off;  // row transforms (length cols)
        off = align_up(off + (size_t)cols * 8);
        p->off_tw1 = off;  // column transforms (length rows)
        off = align_up(off + (size_t)rows * 8);
        p->off_tw2 = off;
        p->off_buf = off;
        const int64_t img_bytes = rows * (cols / 2) * 8;
        int64_t chunk = p->opt_chunk;
        if (chunk <= 0) {
            chunk = l2_budget_bytes() / img_bytes;
            if (chunk < 1) chunk = 1;
        }
        if (chunk > p->batch) chunk = p->batch;
        if (chunk > 65535) chunk = 65535;
        p->chunk = chunk;
        off = align_up(off + (size_t)chunk * img_bytes);
        p->off_buf2 = off;  // second spectrum buffer for the adjoint (G's spectra)
        if (p->opt_backward) off = align_up(off + (size_t)chunk * img_bytes);
    }
    p->need = off;
}

int cuda_fail(cudaError_t e) {
    g_last_cuda_error = (int)e;
    return GBFFT_ERR_CUDA;
}

bool misaligned(const void *ptr) { return (reinterpret_cast<uintptr_t>(ptr) & 15u) != 0; }

// Launch wrapper that records a profiling event pair when enabled.
template <typename F>
int launch(gbfft_plan *p, int stage, cudaStream_t s, F &&f) {
    cudaEvent_t a = nullptr, b = nullptr;
    if (p->opt_profile) {
        if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
            if (a) cudaEventDestroy(a);
            return cuda_fail(cudaGetLastError());
        }
        cudaEventRecord(a, s);
    }
    cudaError_t e = f();
    if (p->opt_profile) {
        cudaEventRecord(b, s);
        p->prof.push_back(ProfRec{stage, a, b});
    }
    if (e != cudaSuccess) return cuda_fail(e);
    return GBFFT_OK;
}

int check_plan_ready(gbfft_plan *p) {
    if (!p) return GBFFT_ERR_NULL;
    if (!p->bound || p->ws_bytes < p->need) return GBFFT_ERR_WORKSPACE;
    return GBFFT_OK;
}

int run_1d(gbfft_plan *p, const void *in, void *out, int dir, cudaStream_t s) {
    int rc = check_plan_ready(p);
    if (rc) return rc;
    if (p->kind != KIND_1D) return GBFFT_ERR_INVALID_VALUE;
    if (!in || !out) return GBFFT_ERR_NULL;
    if (misaligned(in) || misaligned(out)) return GBFFT_ERR_MISALIGNED;
    const int64_t n = int64_t(1) << p->log2n;
    const double scale = dir < 0 ? 1.0 / (double)n : 1.0;
    const bool dbl = is_dbl(p);
    if (p->log2n <= max_single_log2(p)) {
        return launch(p, GBFFT_STAGE_FFT1D, s, [&] {
            return launch_fft1d(in, out, p->log2n, p->batch, dbl, dir, p->ws + p->off_tw0, scale, s);
        });
    }
    const size_t cs = csize(p);
    for (int64_t b0 = 0; b0 < p->batch; b0 += p->chunk) {
        const int64_t nb = (p->batch - b0 < p->chunk) ? p->batch - b0 : p->chunk;
        const char *src = static_cast<const char *>(in) + (size_t)b0 * n * cs;
        char *dst = static_cast<char *>(out) + (size_t)b0 * n * cs;
        rc = launch(p, GBFFT_STAGE_FOURSTEP_A, s, [&] {
            return launch_fourstep_a(src, p->ws + p->off_buf, p->log2n, nb, dbl, dir, p->ws + p->off_tw0,
                                     p->ws + p->off_tw2, s);
        });
        if (rc) return rc;
        rc = launch(p, GBFFT_STAGE_FOURSTEP_B, s, [&] {
            return launch_fourstep_b(p->ws + p->off_buf, dst, p->log2n, nb, dbl, dir, p->ws + p->off_tw1, scale, s);
        });
        if (rc) return rc;
    }
    return GBFFT_OK;
}

}  // namespace

extern "C" {

int gbfft_version(void) { return 100; }

const char *gbfft_status_string(int status) {
    switch (status) {
        case GBFFT_OK: return "ok";
        case GBFFT_ERR_NULL: return "null pointer";
        case GBFFT_ERR_INVALID_SIZE: return "invalid size (lengths must be 2^m within range, batch >= 1)";
        case GBFFT_ERR_DTYPE: return "unsupported dtype";
        case GBFFT_ERR_MISALIGNED: return "data pointer not 16-byte aligned";
        case GBFFT_ERR_WORKSPACE: return "workspace missing or too small";
        case GBFFT_ERR_UNSUPPORTED: return "unsupported request";
        case GBFFT_ERR_CUDA: return "CUDA error";
        case GBFFT_ERR_TIMEOUT: return "device-side wait timed out";
        case GBFFT_ERR_INVALID_VALUE: return "invalid value";
        default: return "unknown status";
    }
}

int gbfft_last_cuda_error(void) { return g_last_cuda_error; }

int fft_plan_create(int64_t n, int64_t batch, int dtype, gbfft_plan_t *out) {
    if (!out) return GBFFT_ERR_NULL;
    *out = nullptr;
    if (dtype != GBFFT_C64 && dtype != GBFFT_C128) return GBFFT_ERR_DTYPE;
    const int l = ilog2_exact(n);
    if (l < 1 || l > kMaxLog2 || batch < 1) return GBFFT_ERR_INVALID_SIZE;
    if ((int64_t(1) << l) * batch > (int64_t(1) << 40)) return GBFFT_ERR_INVALID_SIZE;
    gbfft_plan *p = new (std::nothrow) gbfft_plan();
    if (!p) return GBFFT_ERR_UNSUPPORTED;
    p->kind = KIND_1D;
    p->dtype = dtype;
    p->batch = batch;
    p->log2n = l;
    layout(p);
    *out = p;
    return GBFFT_OK;
}

int fft2_plan_create(int64_t rows, int64_t cols, int64_t batch, int dtype, gbfft_plan_t *out) {
    if (!out) return GBFFT_ERR_NULL;
    *out = nullptr;
    if (dtype != GBFFT_C64) return GBFFT_ERR_DTYPE;
    const int lr = ilog2_exact(rows), lc = ilog2_exact(cols);
    if (lr < 1 || lc < 1 || lr > kMax2DLog2 || lc > kMax2DLog2 || batch < 1) return GBFFT_ERR_INVALID_SIZE;
    gbfft_plan *p = new (std::nothrow) gbfft_plan();
    if (!p) return GBFFT_ERR_UNSUPPORTED;
    p->kind = KIND_2D;
    p->dtype = dtype;
    p->batch = batch;
    p->log2r = lr;
    p->log2c = lc;
    layout(p);
    *out = p;
    return GBFFT_OK;
}

int fft_plan_set_option(gbfft_plan_t p, int key, int64_t value) {
    if (!p) return GBFFT_ERR_NULL;
    switch (key) {
        case GBFFT_OPT_SCALE_CONVENTION:
            if (value != 0 && value != 1) return GBFFT_ERR_INVALID_VALUE;
            p->opt_scale_conv = value;
            return GBFFT_OK;
        case GBFFT_OPT_H_BATCH_STRIDE:
            if (p->kind != KIND_2D || value < 0) return GBFFT_ERR_INVALID_VALUE;
            p->opt_h_stride = value;
            return GBFFT_OK;
        case GBFFT_OPT_PRECISION:
            if (value != 0) return value == 1 ? GBFFT_ERR_UNSUPPORTED : GBFFT_ERR_INVALID_VALUE;
            p->opt_precision = value;
            return GBFFT_OK;
        case GBFFT_OPT_IMAGES_PER_CHUNK:
            if (value < 0) return GBFFT_ERR_INVALID_VALUE;
            p->opt_chunk = value;
            layout(p);
            return GBFFT_OK;
        case GBFFT_OPT_PROFILE:
            if (value != 0 && value != 1) return GBFFT_ERR_INVALID_VALUE;
            p->opt_profile = value;
            return GBFFT_OK;
        case GBFFT_OPT_COLS_TILE:
            if (p->kind != KIND_2D || !cols_variant_valid(1 << p->log2r, 1 << p->log2c, (int)value))
                return GBFFT_ERR_INVALID_VALUE;
            p->opt_cols_variant = value;
            return GBFFT_OK;
        case GBFFT_OPT_ENABLE_BACKWARD:
            if (p->kind != KIND_2D || (value != 0 && value != 1)) return GBFFT_ERR_INVALID_VALUE;
            p->opt_backward = value;
            layout(p);
            return GBFFT_OK;
        default: return GBFFT_ERR_INVALID_VALUE;
    }
}

int fft_plan_workspace_bytes(gbfft_plan_t p, size_t *bytes) {
    if (!p || !bytes) return GBFFT_ERR_NULL;
    *bytes = p->need;
    return GBFFT_OK;
}

int fft_plan_bind_workspace(gbfft_plan_t p, void *workspace, size_t bytes, gbfft_stream_t stream) {
    if (!p || !workspace) return GBFFT_ERR_NULL;
    if ((reinterpret_cast<uintptr_t>(workspace) & (kAlign - 1)) != 0) return GBFFT_ERR_MISALIGNED;
    if (bytes < p->need) return GBFFT_ERR_WORKSPACE;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    p->ws = static_cast<char *>(workspace);
    p->ws_bytes = bytes;
    p->bound = false;
    const bool dbl = is_dbl(p);
    int rc;
    if (p->kind == KIND_1D) {
        if (p->log2n <= max_single_log2(p)) {
            rc = launch(p, GBFFT_STAGE_TWIDDLES, s, [&] { return launch_twiddles(p->ws + p->off_tw0, 1 << p->log2n, dbl, s); });
        } else {
            rc = launch(p, GBFFT_STAGE_TWIDDLES, s, [&] {
                cudaError_t e = launch_twiddles(p->ws + p->off_tw0, 1 << p->fs_l1, dbl, s);
                if (e == cudaSuccess) e = launch_twiddles(p->ws + p->off_tw1, 1 << p->fs_l2, dbl, s);
                if (e == cudaSuccess) e = launch_fourstep_twiddles(p->ws + p->off_tw2, 1 << p->log2n, dbl, s);
                return e;
            });
        }
    } else {
        rc = launch(p, GBFFT_STAGE_TWIDDLES, s, [&] {
            cudaError_t e = launch_twiddles(p->ws + p->off_tw0, 1 << p->log2c, false, s);
            if (e == cudaSuccess) e = launch_twiddles(p->ws + p->off_tw1, 1 << p->log2r, false, s);
            return e;
        });
    }
    if (rc) return rc;
    p->bound = true;
    return GBFFT_OK;
}

int fft_forward(gbfft_plan_t p, const void *in, void *out, gbfft_stream_t stream) {
    return run_1d(p, in, out, -1, reinterpret_cast<cudaStream_t>(stream));
}

int fft_inverse(gbfft_plan_t p, const void *in, void *out, gbfft_stream_t stream) {
    return run_1d(p, in, out, +1, reinterpret_cast<cudaStream_t>(stream));
}

int fft2_filter_ifft2(gbfft_plan_t p, const float *img, const float *H, float *out, gbfft_stream_t stream) {
    int rc = check_plan_ready(p);
    if (rc) return rc;
    if (p->kind != KIND_2D) return GBFFT_ERR_INVALID_VALUE;
    if (!img || !H || !out) return GBFFT_ERR_NULL;
    if (misaligned(img) || misaligned(H) || misaligned(out)) return GBFFT_ERR_MISALIGNED;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int rows = 1 << p->log2r, cols = 1 << p->log2c;
    const int64_t np = (int64_t)rows * cols;
    const float scale = (float)(1.0 / (double)np);
    void *spec = p->ws + p->off_buf;
    const void *twc = p->ws + p->off_tw0, *twr = p->ws + p->off_tw1;
    for (int64_t b0 = 0; b0 < p->batch; b0 += p->chunk) {
        const int nb = (int)((p->batch - b0 < p->chunk) ? p->batch - b0 : p->chunk);
        const float *ib = img + b0 * np;
        float *ob = out + b0 * np;
        const float *hb = H + b0 * p->opt_h_stride;
        rc = launch(p, GBFFT_STAGE_ROWS_FWD, s, [&] { return launch_rows_fwd(ib, spec, rows, cols, nb, twc, s); });
        if (rc) return rc;
        rc = launch(p, GBFFT_STAGE_COLS, s, [&] {
            return launch_cols_filter(spec, hb, p->opt_h_stride, rows, cols, nb, scale, twr, s,
                                      (int)p->opt_cols_variant);
        });
        if (rc) return rc;
        rc = launch(p, GBFFT_STAGE_ROWS_INV, s, [&] { return launch_rows_inv(spec, ob, rows, cols, nb, twc, s); });
        if (rc) return rc;
    }
    return GBFFT_OK;
}

int fft2_filter_ifft2_backward(gbfft_plan_t p, const float *img, const float *H, const float *grad_out,
                               float *grad_img, float *grad_H, gbfft_stream_t stream) {
    int rc = check_plan_ready(p);
    if (rc) return rc;
    if (p->kind != KIND_2D) return GBFFT_ERR_INVALID_VALUE;
    if (!H || !grad_out || (grad_H && !img)) return GBFFT_ERR_NULL;
    if (misaligned(img) || misaligned(H) || misaligned(grad_out) || misaligned(grad_img) || misaligned(grad_H))
        return GBFFT_ERR_MISALIGNED;
    if (!grad_img && !grad_H) return GBFFT_OK;
    if (grad_H && p->opt_h_stride != 0) return GBFFT_ERR_UNSUPPORTED;  // grad of a shared filter only
    if (grad_H && !p->opt_backward) return GBFFT_ERR_WORKSPACE;        // needs the second spectrum buffer
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int rows = 1 << p->log2r, cols = 1 << p->log2c;
    const int64_t np = (int64_t)rows * cols;
    const float scale = (float)(1.0 / (double)np);
    void *spec_x = p->ws + p->off_buf, *spec_g = p->ws + p->off_buf2;
    const void *twc = p->ws + p->off_tw0, *twr = p->ws + p->off_tw1;
    for (int64_t b0 = 0; b0 < p->batch; b0 += p->chunk) {
        const int nb = (int)((p->batch - b0 < p->chunk) ? p->batch - b0 : p->chunk);
        const float *gb = grad_out + b0 * np;
        if (!grad_H) {  // grad_img only: the pipeline itself, applied to grad_out
            const float *hb = H + b0 * p->opt_h_stride;
            rc = launch(p, GBFFT_STAGE_ROWS_FWD, s, [&] { return launch_rows_fwd(gb, spec_x, rows, cols, nb, twc, s); });
            if (rc) return rc;
            rc = launch(p, GBFFT_STAGE_COLS, s, [&] {
                return launch_cols_filter(spec_x, hb, p->opt_h_stride, rows, cols, nb, scale, twr, s,
                                          (int)p->opt_cols_variant);
            });
            if (rc) return rc;
            rc = launch(p, GBFFT_STAGE_ROWS_INV, s,
                        [&] { return launch_rows_inv(spec_x, grad_img + b0 * np, rows, cols, nb, twc, s); });
            if (rc) return rc;
            continue;
        }
        rc = launch(p, GBFFT_STAGE_ROWS_FWD, s,
                    [&] { return launch_rows_fwd(img + b0 * np, spec_x, rows, cols, nb, twc, s); });
        if (rc) return rc;
        rc = launch(p, GBFFT_STAGE_ROWS_FWD, s, [&] { return launch_rows_fwd(gb, spec_g, rows, cols, nb, twc, s); });
        if (rc) return rc;
        rc = launch(p, GBFFT_STAGE_COLS_GRAD, s, [&] {
            return launch_cols_grad(spec_x, spec_g, H, grad_H, rows, cols, nb, scale, b0 > 0 ? 1 : 0, twr, s);
        });
        if (rc) return rc;
        if (grad_img) {
            rc = launch(p, GBFFT_STAGE_ROWS_INV, s,
                        [&] { return launch_rows_inv(spec_g, grad_img + b0 * np, rows, cols, nb, twc, s); });
            if (rc) return rc;
        }
    }
    return GBFFT_OK;
}

int fft_plan_destroy(gbfft_plan_t p) {
    if (!p) return GBFFT_ERR_NULL;
    for (auto &r : p->prof) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    delete p;
    return GBFFT_OK;
}

int gbfft_plan_profile_read(gbfft_plan_t p, double *ms, int64_t *launches, int nstages) {
    if (!p) return GBFFT_ERR_NULL;
    if (nstages < 0) return GBFFT_ERR_INVALID_VALUE;
    int rc = GBFFT_OK;
    for (auto &r : p->prof) {
        float t = 0.f;
        cudaError_t e = cudaEventSynchronize(r.b);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, r.a, r.b);
        if (e != cudaSuccess) rc = cuda_fail(e);
        if (r.stage < nstages) {
            if (ms) ms[r.stage] += t;
            if (launches) launches[r.stage] += 1;
        }
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    p->prof.clear();
    return rc;
}

}  // extern "C"
