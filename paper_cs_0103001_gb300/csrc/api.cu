// api.cu — the C ABI of include/gbfft.h: plans, validation, workspace layout
// and the launch sequences.  Host code only; kernels live in the other files.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <map>
#include <new>
#include <vector>

#include <cstdio>
#include <cstdlib>
#include <string>

#include <nvtx3/nvToolsExt.h>

#include "batched.h"
#include "check.cuh"
#include "gbfft.h"
#include "internal.h"
#include "tma.cuh"
#include "tune.h"

using namespace gbfft;

namespace {

thread_local int g_last_cuda_error = 0;

struct ProfRec {
    int stage;
    cudaEvent_t a, b;
};

enum PlanKind { KIND_1D = 1, KIND_2D = 2, KIND_BATCH = 3, KIND_SLAB = 4 };

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
    int64_t opt_backward = 0;
    // workspace
    char *ws = nullptr;
    size_t ws_bytes = 0;
    bool bound = false;
    // layout (byte offsets into ws)
    size_t off_tw0 = 0, off_tw1 = 0, off_tw2 = 0, off_tw3 = 0, off_tw5 = 0, off_buf = 0, off_buf2 = 0, need = 0;
    size_t off_status = 0;  // device status word (bounded waits that gave up)
    size_t off_hs = 0, off_beta = 0, off_grad = 0;  // 2D: prepared filter, beta, adjoint sums
    int64_t chunk = 0;           // transforms (1D four-step) or images (2D) per workspace chunk
    int nranks = 1, rank = 0;    // slab plans: the decomposition and this rank
    int fs_l1 = 0, fs_l2 = 0;    // four-step split
    bool fs3 = false;            // three passes of 256 (complex64, N = 2^24)
    bool prepared = false;       // 2D: the workspace holds a filter of fft2_filter_prepare
    size_t off_tw6 = 0, off_tw7 = 0;  // three passes: the middle pass's two-level and coarse tables
    std::vector<ProfRec> prof;
    // guard bands: kAlign bytes of a fixed pattern after every workspace
    // region (offsets here, and as a table in the workspace for the kernels
    // that fill and check them)
    std::vector<long long> guards;
    size_t off_guards = 0;
    // batched plans (KIND_BATCH)
    std::vector<BatchImage> bimgs;
    std::vector<BatchItem> bitems[kBatchStages];
    std::map<int, size_t> tw_off;  // twiddle table per distinct length
    size_t off_bimgs = 0, off_bitems[kBatchStages] = {0, 0, 0, 0};
    size_t bsmem[kBatchStages] = {0, 0, 0, 0};
    int64_t opt_bps[kBatchStages] = {0, 0, 0, 0};  // blocks per SM per stage (0 = as many as fit)
    int64_t opt_graph = 1;
    int64_t opt_onchip = 1;
    int64_t opt_colform = 0;  // column-pass form (GBFFT_OPT_COLUMN_FORM)
    int64_t opt_passes = 0;   // 1D complex64 2^24: two or three passes (GBFFT_OPT_FOURSTEP_PASSES)
    cudaStream_t cap_stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    const void *graph_ptrs = nullptr;
    int graph_grid[kBatchStages] = {0, 0, 0, 0};
    // 2D: side stream for the filter preparation, forked from / joined to the
    // caller's stream with events
    cudaStream_t aux = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_join2 = nullptr;
    // batched plans: the images grouped by shape (each class's spectra,
    // prepared filters and betas contiguous), and the form of the launches
    struct BatchClass {
        int rows, cols;
        std::vector<int> imgs;  // image indices, in input order
        size_t off_spec, off_hs, off_beta, off_idx;
    };
    std::vector<BatchClass> bclasses;
    int64_t opt_batch_form = 0;
};

namespace {

bool is_dbl(const gbfft_plan *p) { return p->dtype == GBFFT_C128; }
size_t csize(const gbfft_plan *p) { return is_dbl(p) ? 16 : 8; }

int max_single_log2(const gbfft_plan *p) { return is_dbl(p) ? kMaxSinglePassLog2F64 : kMaxSinglePassLog2F32; }

// End of a workspace region at `end`: the guard band after it, and where the
// next region starts.
size_t region_end(gbfft_plan *p, size_t end) {
    const size_t g = align_up(end);
    p->guards.push_back((long long)g);
    return g + kAlign;
}

// The guard table (one offset per guard, the table's own guard included)
// and the status words close the layout.
void layout_close(gbfft_plan *p, size_t off) {
    p->off_guards = off;
    const size_t n = p->guards.size() + 1;  // and the guard after the table itself
    off = align_up(off + n * sizeof(long long));
    p->guards.push_back((long long)off);
    off += kAlign;
    p->off_status = off;
    p->need = off + kAlign;
}

void layout_batched(gbfft_plan *p) {
    size_t off = kAlign;  // a guard band before the first region
    p->guards.assign(1, 0);
    p->off_bimgs = off;
    off = region_end(p, off + p->bimgs.size() * sizeof(BatchImage));
    for (int st = 0; st < kBatchStages; ++st) {
        p->off_bitems[st] = off;
        off = region_end(p, off + p->bitems[st].size() * sizeof(BatchItem));
    }
    p->tw_off.clear();
    for (const BatchImage &im : p->bimgs) {
        for (int len : {im.cols, im.rows}) {
            if (p->tw_off.count(len)) continue;
            p->tw_off[len] = off;
            off = region_end(p, off + (size_t)len * 8);
        }
    }
    // per shape class: spectra [n][M/2][N], prepared filters [n][M/2][N],
    // betas [n][N], image indices [n]; an image's regions are its slice
    for (auto &c : p->bclasses) {
        const size_t n = c.imgs.size(), half_px = (size_t)c.rows * (c.cols / 2);
        c.off_spec = off;
        off = region_end(p, off + n * half_px * 8);
        c.off_hs = off;
        off = region_end(p, off + n * half_px * 4);
        c.off_beta = off;
        off = region_end(p, off + n * (size_t)c.rows * 4);
        c.off_idx = off;
        off = region_end(p, off + n * sizeof(int));
        for (size_t j = 0; j < n; ++j) {
            BatchImage &im = p->bimgs[c.imgs[j]];
            im.twc_off = (long long)p->tw_off[im.cols];
            im.twr_off = (long long)p->tw_off[im.rows];
            im.spec_off = (long long)(c.off_spec + j * half_px * 8);
            im.hs_off = (long long)(c.off_hs + j * half_px * 4);
            im.beta_off = (long long)(c.off_beta + j * (size_t)c.rows * 4);
        }
    }
    layout_close(p, off);
}

// Compute the workspace layout for the current options.
// Three passes of 256 (complex64, N = 2^24, GBFFT_OPT_FOURSTEP_PASSES 3 or
// default): see launch_fourstep_a_split in internal.h.
bool fourstep3_applies(const gbfft_plan *p) {
    return p->kind == KIND_1D && !is_dbl(p) && p->log2n == 24 && p->opt_passes != 2;
}

void layout(gbfft_plan *p) {
    size_t off = kAlign;  // a guard band before the first region
    p->prepared = false;
    p->guards.assign(1, 0);
    if (p->kind == KIND_BATCH) {
        layout_batched(p);
        return;
    }
    if (p->kind == KIND_SLAB) {
        const int64_t rows = int64_t(1) << p->log2r, cols = int64_t(1) << p->log2c;
        const int64_t mloc = cols / 2 / p->nranks;  // this rank's half-spectrum columns
        p->off_tw0 = off;  // row transforms (length cols)
        off = region_end(p, off + (size_t)cols * 8);
        p->off_tw1 = off;  // column transforms (length rows)
        off = region_end(p, off + (size_t)rows * 8);
        p->off_hs = off;  // prepared filter of this rank's columns, [mloc][rows]
        off = region_end(p, off + (size_t)mloc * rows * 4);
        p->off_beta = off;
        off = region_end(p, off + (size_t)rows * 4);
        layout_close(p, off);
        return;
    }
    if (p->kind == KIND_1D) {
        const int64_t n = int64_t(1) << p->log2n;
        p->fs3 = false;
        if (p->log2n <= max_single_log2(p)) {
            p->off_tw0 = off;
            off = region_end(p, off + (size_t)n * csize(p));
            p->off_tw1 = p->off_tw2 = p->off_buf = off;
            p->chunk = p->batch;
        } else if (fourstep3_applies(p)) {
            // three passes of 256: one Stockham table (length 256), the first
            // pass's two-level (N) and coarse (16 x 2^16) tables, the middle
            // pass's two-level (2^16) and coarse (16 x 256) tables
            p->fs3 = true;
            p->fs_l1 = 8;
            p->fs_l2 = 16;
            const int lf = (p->log2n + 1) / 2;
            p->off_tw0 = p->off_tw1 = off;
            off = region_end(p, off + (size_t)256 * 8);
            p->off_tw2 = off;
            off = region_end(p, off + (size_t)((int64_t(1) << lf) + (n >> lf)) * 8);
            p->off_tw5 = off;
            off = region_end(p, off + (size_t)16 * 65536 * 8);
            p->off_tw6 = off;
            off = region_end(p, off + (size_t)(256 + 256) * 8);
            p->off_tw7 = off;
            off = region_end(p, off + (size_t)16 * 256 * 8);
            p->off_tw3 = off;
            p->off_buf = off;
            int64_t chunk = p->opt_chunk;
            if (chunk <= 0) chunk = kFourStepChunkBytes / (n * 8);
            if (chunk < 1) chunk = 1;
            if (chunk > p->batch) chunk = p->batch;
            p->chunk = chunk;
            off = region_end(p, off + (size_t)chunk * n * 8);
        } else {
            fourstep_split(p->log2n, is_dbl(p), &p->fs_l1, &p->fs_l2);
            const int64_t n1 = int64_t(1) << p->fs_l1, n2 = int64_t(1) << p->fs_l2;
            const int lf = (p->log2n + 1) / 2;
            const int64_t n4s = (int64_t(1) << lf) + (n >> lf);
            p->off_tw0 = off;
            off = region_end(p, off + (size_t)n1 * csize(p));
            p->off_tw1 = off;
            off = region_end(p, off + (size_t)n2 * csize(p));
            p->off_tw2 = off;
            off = region_end(p, off + (size_t)n4s * csize(p));
            p->off_tw5 = off;  // coarse inter-pass table of pass A
            off = region_end(p, off + (size_t)16 * n2 * csize(p));
            p->off_tw3 = off;  // full inter-pass table of the cluster path
            if (fft1d_cluster_supported(p->log2n, is_dbl(p))) off = region_end(p, off + (size_t)n * csize(p));
            p->off_buf = off;
            int64_t chunk = p->opt_chunk;
            if (chunk <= 0) {
                // a large chunk: one launch of many blocks per pass costs less than
                // keeping the intermediate in L2 gains (the passes are not HBM-bound)
                chunk = kFourStepChunkBytes / (n * (int64_t)csize(p));
                if (chunk < 1) chunk = 1;
            }
            if (chunk > p->batch) chunk = p->batch;
            p->chunk = chunk;
            off = region_end(p, off + (size_t)chunk * n * csize(p));
        }
    } else {
        const int64_t rows = int64_t(1) << p->log2r, cols = int64_t(1) << p->log2c;
        p->off_tw0 = off;  // row transforms (length cols)
        off = region_end(p, off + (size_t)cols * 8);
        p->off_tw1 = off;  // column transforms (length rows)
        off = region_end(p, off + (size_t)rows * 8);
        p->off_tw2 = off;
        const int64_t half_px = rows * (cols / 2);
        const int64_t img_bytes = half_px * 8;
        int64_t chunk = p->opt_chunk;
        if (chunk <= 0) {
            // many images per launch: the kernels are bound by the SM, not by HBM,
            // so fewer, larger launches beat an L2-sized spectrum buffer
            chunk = kPipelineChunkBytes / img_bytes;
            if (chunk < 1) chunk = 1;
        }
        if (chunk > p->batch) chunk = p->batch;
        if (chunk > 65535) chunk = 65535;
        p->chunk = chunk;
        const int64_t nfilt = p->opt_h_stride != 0 ? chunk : 1;  // prepared filters held at once
        p->off_hs = off;
        off = region_end(p, off + (size_t)nfilt * half_px * 4);
        p->off_beta = off;
        off = region_end(p, off + (size_t)nfilt * rows * 4);
        p->off_buf = off;
        off = region_end(p, off + (size_t)chunk * img_bytes);
        p->off_buf2 = off;  // G's spectra and the filter-gradient sums (adjoint only)
        p->off_grad = off;
        if (p->opt_backward) {
            off = region_end(p, off + (size_t)chunk * img_bytes);
            p->off_grad = off;
            off = region_end(p, off + (size_t)(cols / 2 + 1) * rows * 4);
        }
    }
    layout_close(p, off);
}

int cuda_fail(cudaError_t e) {
    g_last_cuda_error = (int)e;
    return GBFFT_ERR_CUDA;
}

bool misaligned(const void *ptr) { return (reinterpret_cast<uintptr_t>(ptr) & 15u) != 0; }

// Launch wrapper that records a profiling event pair when enabled.
template <typename F>
int launch(gbfft_plan *p, int stage, cudaStream_t s, F &&f) {
    // NVTX range per stage launch (GBFFT_NVTX=1; a profiler such as Nsight
    // Systems shows them on the host thread beside the kernels they issue)
    static const bool nvtx = [] {
        const char *v = getenv("GBFFT_NVTX");
        return v && v[0] && v[0] != '0';
    }();
    static const char *const names[GBFFT_STAGE_COUNT] = {
        "gbfft fft1d",  "gbfft fourstep_a", "gbfft fourstep_b",  "gbfft rows_fwd", "gbfft cols_filter",
        "gbfft rows_inv", "gbfft cols_grad", "gbfft twiddles",   "gbfft graph",    "gbfft filter_prep",
        "gbfft onchip", "gbfft spectrum",   "gbfft fft1d_cluster"};
    if (nvtx) nvtxRangePushA(stage >= 0 && stage < GBFFT_STAGE_COUNT ? names[stage] : "gbfft");
    struct Pop {
        bool on;
        ~Pop() {
            if (on) nvtxRangePop();
        }
    } pop{nvtx};
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
    if (p->opt_onchip == 2 && fft1d_cluster_supported(p->log2n, dbl)) {
        return launch(p, GBFFT_STAGE_FFT1D_CLUSTER, s, [&] {
            return launch_fft1d_cluster(in, out, p->log2n, p->batch, dir, p->ws + p->off_tw0, p->ws + p->off_tw1,
                                        p->ws + p->off_tw3, scale, s);
        });
    }
    const size_t cs = csize(p);
    if (p->fs3) {
        int *status = reinterpret_cast<int *>(p->ws + p->off_status);
        void *tmp = p->ws + p->off_buf;
        for (int64_t b0 = 0; b0 < p->batch; b0 += p->chunk) {
            const int64_t nb = (p->batch - b0 < p->chunk) ? p->batch - b0 : p->chunk;
            const char *src = static_cast<const char *>(in) + (size_t)b0 * n * cs;
            char *dst = static_cast<char *>(out) + (size_t)b0 * n * cs;
            rc = launch(p, GBFFT_STAGE_FOURSTEP_A, s, [&] {
                return launch_fourstep_a_split(src, tmp, 8, 16, nb, dir, p->ws + p->off_tw0, p->ws + p->off_tw2,
                                               p->ws + p->off_tw5, status, s);
            });
            if (rc) return rc;
            rc = launch(p, GBFFT_STAGE_FOURSTEP_A, s, [&] {
                return launch_fourstep_a_split(tmp, tmp, 8, 8, nb * 256, dir, p->ws + p->off_tw0, p->ws + p->off_tw6,
                                               p->ws + p->off_tw7, status, s);
            });
            if (rc) return rc;
            rc = launch(p, GBFFT_STAGE_FOURSTEP_B, s, [&] {
                return launch_fourstep_b_split(tmp, dst, 16, 8, 8, nb, dir, p->ws + p->off_tw0, scale, status, s);
            });
            if (rc) return rc;
        }
        return GBFFT_OK;
    }
    for (int64_t b0 = 0; b0 < p->batch; b0 += p->chunk) {
        const int64_t nb = (p->batch - b0 < p->chunk) ? p->batch - b0 : p->chunk;
        const char *src = static_cast<const char *>(in) + (size_t)b0 * n * cs;
        char *dst = static_cast<char *>(out) + (size_t)b0 * n * cs;
        rc = launch(p, GBFFT_STAGE_FOURSTEP_A, s, [&] {
            return launch_fourstep_a(src, p->ws + p->off_buf, p->log2n, nb, dbl, dir, p->ws + p->off_tw0,
                                     p->ws + p->off_tw2, p->ws + p->off_tw5,
                                     reinterpret_cast<int *>(p->ws + p->off_status), s);
        });
        if (rc) return rc;
        rc = launch(p, GBFFT_STAGE_FOURSTEP_B, s, [&] {
            return launch_fourstep_b(p->ws + p->off_buf, dst, p->log2n, nb, dbl, dir, p->ws + p->off_tw1, scale,
                                     reinterpret_cast<int *>(p->ws + p->off_status), s);
        });
        if (rc) return rc;
    }
    return GBFFT_OK;
}

int sm_count() {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return 0;
    return n;
}

// Grid of a batched stage: blocks per SM (option, else as many as fit) x SMs.
int batched_grid(gbfft_plan *p, int st, cudaError_t *err) {
    int fit = 0;
    *err = batch_max_blocks_per_sm(st, p->bsmem[st], &fit);
    if (*err != cudaSuccess) return 0;
    if (fit < 1) fit = 1;
    int bps = p->opt_bps[st] > 0 ? (int)p->opt_bps[st] : fit;
    if (bps > fit) bps = fit;
    return bps * sm_count();
}

cudaError_t ensure_aux(gbfft_plan *p) {
    cudaError_t e = cudaSuccess;
    if (!p->aux) e = cudaStreamCreateWithFlags(&p->aux, cudaStreamNonBlocking);
    if (e == cudaSuccess && !p->ev_fork) e = cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess && !p->ev_join) e = cudaEventCreateWithFlags(&p->ev_join, cudaEventDisableTiming);
    if (e == cudaSuccess && !p->ev_join2) e = cudaEventCreateWithFlags(&p->ev_join2, cudaEventDisableTiming);
    return e;
}

// Batched plan, class form: the one-shape kernels once per shape class over
// that class's images, the images reached through the caller's pointer table
// (ImgIndirect).  Side stream: the classes' filter preparations, then the
// small classes' one-launch on-chip pipelines; caller's stream: forward rows,
// (join the preparations) columns and inverse rows of the other classes.
cudaError_t batched_launch_classes(gbfft_plan *p, const gbfft_image_ptrs *ptrs, cudaStream_t s) {
    int *status = reinterpret_cast<int *>(p->ws + p->off_status);
    cudaError_t e = ensure_aux(p);
    if (e == cudaSuccess) e = cudaEventRecord(p->ev_fork, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(p->aux, p->ev_fork, 0);
    auto ind = [&](const gbfft_plan::BatchClass &c) {
        return ImgIndirect{ptrs, reinterpret_cast<const int *>(p->ws + c.off_idx)};
    };
    auto onchip = [&](const gbfft_plan::BatchClass &c) { return onchip_supported(c.rows, c.cols); };
    for (const auto &c : p->bclasses) {
        if (e != cudaSuccess || onchip(c)) continue;
        const long long half_px = (long long)c.rows * (c.cols / 2);
        e = launch_filter_prep(nullptr, reinterpret_cast<float *>(p->ws + c.off_hs),
                               reinterpret_cast<float *>(p->ws + c.off_beta), c.rows, c.cols, (int)c.imgs.size(),
                               (float)(1.0 / ((double)c.rows * c.cols)), 0, half_px, c.rows, p->aux, 0, 0, ind(c));
    }
    if (e == cudaSuccess) e = cudaEventRecord(p->ev_join, p->aux);
    for (const auto &c : p->bclasses) {
        if (e != cudaSuccess || !onchip(c)) continue;
        e = launch_onchip(nullptr, nullptr, nullptr, 0, c.rows, c.cols, (int)c.imgs.size(), p->ws + p->tw_off[c.cols],
                          p->ws + p->tw_off[c.rows], p->aux, ind(c));
    }
    if (e == cudaSuccess) e = cudaEventRecord(p->ev_join2, p->aux);
    for (const auto &c : p->bclasses) {
        if (e != cudaSuccess || onchip(c)) continue;
        e = launch_rows_fwd(nullptr, p->ws + c.off_spec, c.rows, c.cols, (int)c.imgs.size(), p->ws + p->tw_off[c.cols],
                            s, Slab{0, 0}, ind(c));
    }
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, p->ev_join, 0);
    for (const auto &c : p->bclasses) {
        if (e != cudaSuccess || onchip(c)) continue;
        const long long half_px = (long long)c.rows * (c.cols / 2);
        e = launch_cols_filter(p->ws + c.off_spec, reinterpret_cast<const float *>(p->ws + c.off_hs),
                               reinterpret_cast<const float *>(p->ws + c.off_beta), half_px, c.rows, c.rows, c.cols,
                               (int)c.imgs.size(), p->ws + p->tw_off[c.rows], status, s);
    }
    for (const auto &c : p->bclasses) {
        if (e != cudaSuccess || onchip(c)) continue;
        e = launch_rows_inv(p->ws + c.off_spec, nullptr, c.rows, c.cols, (int)c.imgs.size(), p->ws + p->tw_off[c.cols],
                            status, s, Slab{0, 0}, ind(c));
    }
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, p->ev_join2, 0);
    return e;
}

// The four stages of a batched plan: the filter preparation on the plan's side
// stream beside the forward row pass (it touches no spectrum), joined before
// the column pass; under stream capture the side stream joins the capture.
cudaError_t batched_launch_persistent(gbfft_plan *p, const gbfft_image_ptrs *ptrs, cudaStream_t s, const int *grid) {
    const BatchImage *imgs = reinterpret_cast<const BatchImage *>(p->ws + p->off_bimgs);
    auto stage = [&](int st, cudaStream_t on) {
        const BatchItem *items = reinterpret_cast<const BatchItem *>(p->ws + p->off_bitems[st]);
        return launch_batched_stage(st, grid[st], p->bsmem[st], imgs, items, (int)p->bitems[st].size(), ptrs, p->ws,
                                    on);
    };
    cudaError_t e = ensure_aux(p);
    if (e == cudaSuccess) e = cudaEventRecord(p->ev_fork, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(p->aux, p->ev_fork, 0);
    if (e == cudaSuccess) e = stage(3, p->aux);  // filter preparation
    if (e == cudaSuccess) e = cudaEventRecord(p->ev_join, p->aux);
    if (e == cudaSuccess) e = stage(0, s);  // forward rows
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, p->ev_join, 0);
    if (e == cudaSuccess) e = stage(1, s);  // columns
    if (e == cudaSuccess) e = stage(2, s);  // inverse rows
    return e;
}

cudaError_t batched_launch_all(gbfft_plan *p, const gbfft_image_ptrs *ptrs, cudaStream_t s, const int *grid) {
    return p->opt_batch_form == 1 ? batched_launch_persistent(p, ptrs, s, grid) : batched_launch_classes(p, ptrs, s);
}

void drop_graph(gbfft_plan *p) {
    if (p->graph_exec) cudaGraphExecDestroy(p->graph_exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    p->graph_exec = nullptr;
    p->graph = nullptr;
    p->graph_ptrs = nullptr;
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
            layout(p);
            return GBFFT_OK;
        case GBFFT_OPT_PRECISION:
            if (value < 0 || value > 5) return GBFFT_ERR_INVALID_VALUE;
            if (value != 0 && !(p->kind == KIND_2D && tc_supported(1 << p->log2r, 1 << p->log2c)))
                return GBFFT_ERR_UNSUPPORTED;
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
        case GBFFT_OPT_BLOCKS_PER_SM:
            if (p->kind != KIND_BATCH || value < 0 || value > 64) return GBFFT_ERR_INVALID_VALUE;
            for (int st = 0; st < kBatchStages; ++st) p->opt_bps[st] = value;
            drop_graph(p);
            return GBFFT_OK;
        case GBFFT_OPT_USE_GRAPH:
            if (p->kind != KIND_BATCH || (value != 0 && value != 1)) return GBFFT_ERR_INVALID_VALUE;
            p->opt_graph = value;
            drop_graph(p);
            return GBFFT_OK;
        case GBFFT_OPT_ONCHIP:
            if (p->kind == KIND_BATCH || value < 0 || value > 2) return GBFFT_ERR_INVALID_VALUE;
            p->opt_onchip = value;
            return GBFFT_OK;
        case GBFFT_OPT_ENABLE_BACKWARD:
            if (p->kind != KIND_2D || (value != 0 && value != 1)) return GBFFT_ERR_INVALID_VALUE;
            p->opt_backward = value;
            layout(p);
            return GBFFT_OK;
        case GBFFT_OPT_BATCH_FORM:
            if (p->kind != KIND_BATCH || (value != 0 && value != 1)) return GBFFT_ERR_INVALID_VALUE;
            p->opt_batch_form = value;
            drop_graph(p);
            return GBFFT_OK;
        case GBFFT_OPT_COLUMN_FORM:
            if ((p->kind != KIND_2D && p->kind != KIND_SLAB) || value < 0 || value > 3) return GBFFT_ERR_INVALID_VALUE;
            p->opt_colform = value;
            return GBFFT_OK;
        case GBFFT_OPT_FOURSTEP_PASSES:
            if (p->kind != KIND_1D || (value != 0 && value != 2 && value != 3)) return GBFFT_ERR_INVALID_VALUE;
            p->opt_passes = value;
            layout(p);
            p->bound = false;  // the workspace's regions moved: bind again
            return GBFFT_OK;
        default: return GBFFT_ERR_INVALID_VALUE;
    }
}

int fft_plan_workspace_bytes(gbfft_plan_t p, size_t *bytes) {
    if (!p || !bytes) return GBFFT_ERR_NULL;
    *bytes = p->need;
    return GBFFT_OK;
}

// The batched kernels index images and blocks through the plan's tables
// without checks: every work item must lie inside its image's launch shape
// and every class member must be an image of that shape.  Host only.
int check_batch_tables(const gbfft_plan *p) {
    const int n = (int)p->bimgs.size();
    for (int st = 0; st < kBatchStages; ++st)
        for (const BatchItem &it : p->bitems[st]) {
            if (it.img < 0 || it.img >= n || it.bx < 0) return GBFFT_ERR_INVALID_VALUE;
            const BatchImage &im = p->bimgs[it.img];
            int blocks;
            if (st == 0 || st == 2) {
                blocks = (im.rows / 2) >> im.log2g;
            } else if (st == 1) {
                const int w = batch_col_width(im.rows);
                blocks = (im.cols / 2 + w - 1) / w;
            } else {
                blocks = batch_prep_tiles(im.rows, im.cols);
            }
            if (it.bx >= blocks) return GBFFT_ERR_INVALID_VALUE;
        }
    for (const auto &c : p->bclasses)
        for (int i : c.imgs)
            if (i < 0 || i >= n || p->bimgs[i].rows != c.rows || p->bimgs[i].cols != c.cols)
                return GBFFT_ERR_INVALID_VALUE;
    return GBFFT_OK;
}

int fft_plan_bind_workspace(gbfft_plan_t p, void *workspace, size_t bytes, gbfft_stream_t stream) {
    if (!p || !workspace) return GBFFT_ERR_NULL;
    if ((reinterpret_cast<uintptr_t>(workspace) & (kAlign - 1)) != 0) return GBFFT_ERR_MISALIGNED;
    if (bytes < p->need) return GBFFT_ERR_WORKSPACE;
    if (p->kind == KIND_BATCH) {  // before anything reaches the GPU
        const int rc = check_batch_tables(p);
        if (rc) return rc;
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    p->ws = static_cast<char *>(workspace);
    p->ws_bytes = bytes;
    p->bound = false;
    p->prepared = false;
    const bool dbl = is_dbl(p);
    int rc;
    {
        // status words, then the guard table (from the plan's host copy, which
        // outlives the copy) and the guard bands
        cudaError_t e = cudaMemsetAsync(p->ws + p->off_status, 0, 2 * sizeof(int), s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(p->ws + p->off_guards, p->guards.data(), p->guards.size() * sizeof(long long),
                                cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess)
            e = launch_guard_fill(p->ws, reinterpret_cast<const long long *>(p->ws + p->off_guards),
                                  (int)p->guards.size(), (long long)p->ws_bytes, s);
        if (e != cudaSuccess) return cuda_fail(e);
    }
    if (p->kind == KIND_1D) {
        if (p->log2n <= max_single_log2(p)) {
            rc = launch(p, GBFFT_STAGE_TWIDDLES, s, [&] { return launch_twiddles(p->ws + p->off_tw0, 1 << p->log2n, dbl, s); });
        } else if (p->fs3) {
            rc = launch(p, GBFFT_STAGE_TWIDDLES, s, [&] {
                cudaError_t e = launch_twiddles(p->ws + p->off_tw0, 256, false, s);
                if (e == cudaSuccess) e = launch_fourstep_twiddles(p->ws + p->off_tw2, 1 << p->log2n, false, s);
                if (e == cudaSuccess) e = launch_fourstep_coarse_twiddles(p->ws + p->off_tw5, 65536, false, s);
                if (e == cudaSuccess) e = launch_fourstep_twiddles(p->ws + p->off_tw6, 65536, false, s);
                if (e == cudaSuccess) e = launch_fourstep_coarse_twiddles(p->ws + p->off_tw7, 256, false, s);
                return e;
            });
        } else {
            rc = launch(p, GBFFT_STAGE_TWIDDLES, s, [&] {
                cudaError_t e = launch_twiddles(p->ws + p->off_tw0, 1 << p->fs_l1, dbl, s);
                if (e == cudaSuccess) e = launch_twiddles(p->ws + p->off_tw1, 1 << p->fs_l2, dbl, s);
                if (e == cudaSuccess) e = launch_fourstep_twiddles(p->ws + p->off_tw2, 1 << p->log2n, dbl, s);
                if (e == cudaSuccess) e = launch_fourstep_coarse_twiddles(p->ws + p->off_tw5, 1 << p->fs_l2, dbl, s);
                if (e == cudaSuccess && fft1d_cluster_supported(p->log2n, dbl))
                    e = launch_fourstep_full_twiddles(p->ws + p->off_tw3, 1 << p->log2n, p->fs_l2, s);
                return e;
            });
        }
    } else if (p->kind == KIND_2D || p->kind == KIND_SLAB) {
        rc = launch(p, GBFFT_STAGE_TWIDDLES, s, [&] {
            cudaError_t e = launch_twiddles(p->ws + p->off_tw0, 1 << p->log2c, false, s);
            if (e == cudaSuccess) e = launch_twiddles(p->ws + p->off_tw1, 1 << p->log2r, false, s);
            return e;
        });
    } else {
        drop_graph(p);
        rc = launch(p, GBFFT_STAGE_TWIDDLES, s, [&] {
            // tables live in plan-owned host vectors, so the copies may complete later
            cudaError_t e = cudaMemcpyAsync(p->ws + p->off_bimgs, p->bimgs.data(),
                                            p->bimgs.size() * sizeof(BatchImage), cudaMemcpyHostToDevice, s);
            for (int st = 0; st < kBatchStages && e == cudaSuccess; ++st)
                e = cudaMemcpyAsync(p->ws + p->off_bitems[st], p->bitems[st].data(),
                                    p->bitems[st].size() * sizeof(BatchItem), cudaMemcpyHostToDevice, s);
            for (const auto &kv : p->tw_off)
                if (e == cudaSuccess) e = launch_twiddles(p->ws + kv.second, kv.first, false, s);
            for (const auto &c : p->bclasses)
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(p->ws + c.off_idx, c.imgs.data(), c.imgs.size() * sizeof(int),
                                        cudaMemcpyHostToDevice, s);
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


// One chunk of the Sec. 5 pipeline: filter preparation on the side stream
// while the forward row pass runs, then the fused column pass and the inverse
// row pass.
// crop_r, crop_c > 0: img and out are crop_r x crop_c images in the top-left
// corner of the plan's zero-padded grid (Sec. 5 application path).
// use_prepared: the filter of fft2_filter_prepare, already in the workspace
// (H unused; no preparation, and no on-chip path, which reads H itself).
static int pipeline_chunk(gbfft_plan *p, const float *img, const float *H, float *out, int nb, bool first,
                          cudaStream_t s, int crop_r = 0, int crop_c = 0, bool use_prepared = false) {
    const int rows = 1 << p->log2r, cols = 1 << p->log2c;
    const bool cropped = crop_r > 0;
    const int64_t half_px = (int64_t)rows * (cols / 2);
    const bool per_image = p->opt_h_stride != 0;
    void *spec = p->ws + p->off_buf;
    float *hs = reinterpret_cast<float *>(p->ws + p->off_hs);
    float *beta = reinterpret_cast<float *>(p->ws + p->off_beta);
    const float scale = (float)(1.0 / ((double)rows * cols));
    const void *tw = p->ws + p->off_tw0;
    // tensor-core radix-16 passes: warp-level split BF16 with `terms` parts
    // (precision 1, 2), or tcgen05 with format tc5 (precision 3, 4, 5)
    const int terms = (p->opt_precision == 1 || p->opt_precision == 2) ? (int)p->opt_precision + 1 : 0;
    const int tc5 = p->opt_precision >= 3 ? (int)p->opt_precision - 3 : -1;
    int *status = reinterpret_cast<int *>(p->ws + p->off_status);
    if (!use_prepared) p->prepared = false;  // every call with a filter of its own discards a prepared one
    if (!use_prepared && !terms && tc5 < 0 && !cropped && p->opt_onchip && onchip_supported(rows, cols)) {
        return launch(p, GBFFT_STAGE_ONCHIP, s, [&] {
            return launch_onchip(img, H, out, p->opt_h_stride, rows, cols, nb, p->ws + p->off_tw0,
                                 p->ws + p->off_tw1, s);
        });
    }
    const bool prep = !use_prepared && (per_image || first);  // a shared filter is prepared once per call
    // with profiling on, the preparation runs on the caller's stream so that
    // every kernel's events time that kernel alone
    const bool side = prep && !p->opt_profile;
    int rc;
    if (prep && !side) {
        rc = launch(p, GBFFT_STAGE_FILTER_PREP, s, [&] {
            return launch_filter_prep(H, hs, beta, rows, cols, per_image ? nb : 1, scale, p->opt_h_stride,
                                      per_image ? half_px : 0, per_image ? rows : 0, s);
        });
        if (rc) return rc;
    }
    if (side) {
        cudaError_t e = ensure_aux(p);
        if (e == cudaSuccess) e = cudaEventRecord(p->ev_fork, s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(p->aux, p->ev_fork, 0);
        if (e != cudaSuccess) return cuda_fail(e);
        rc = launch(p, GBFFT_STAGE_FILTER_PREP, p->aux, [&] {
            return launch_filter_prep(H, hs, beta, rows, cols, per_image ? nb : 1, scale, p->opt_h_stride,
                                      per_image ? half_px : 0, per_image ? rows : 0, p->aux);
        });
        if (rc) return rc;
        if ((e = cudaEventRecord(p->ev_join, p->aux)) != cudaSuccess) return cuda_fail(e);
    }
    rc = launch(p, GBFFT_STAGE_ROWS_FWD, s, [&] {
        if (cropped) return launch_rows_pad(true, img, spec, rows, cols, nb, crop_r, crop_c, tw, s);
        if (tc5 >= 0) return launch_rows_tc5(true, img, spec, rows, cols, nb, tw, tc5, status, s);
        return terms ? launch_rows_tc(true, img, spec, rows, cols, nb, tw, terms, s)
                     : launch_rows_fwd(img, spec, rows, cols, nb, tw, s);
    });
    if (rc) return rc;
    if (side) {
        cudaError_t e = cudaStreamWaitEvent(s, p->ev_join, 0);
        if (e != cudaSuccess) return cuda_fail(e);
    }
    const long long hs_img = per_image ? half_px : 0, beta_img = per_image ? rows : 0;
    rc = launch(p, GBFFT_STAGE_COLS, s, [&] {
        if (tc5 >= 0)
            return launch_cols_tc5(spec, hs, beta, hs_img, beta_img, rows, cols, nb, p->ws + p->off_tw1, tc5, status,
                                   s);
        return terms ? launch_cols_tc(spec, hs, beta, hs_img, beta_img, rows, cols, nb, p->ws + p->off_tw1, terms, s)
                     : launch_cols_filter(spec, hs, beta, hs_img, beta_img, rows, cols, nb, p->ws + p->off_tw1,
                                          reinterpret_cast<int *>(p->ws + p->off_status), s, ColSlab{0, 0, 0},
                                          (int)p->opt_colform);
    });
    if (rc) return rc;
    return launch(p, GBFFT_STAGE_ROWS_INV, s, [&] {
        if (cropped) return launch_rows_pad(false, spec, out, rows, cols, nb, crop_r, crop_c, tw, s);
        if (tc5 >= 0) return launch_rows_tc5(false, spec, out, rows, cols, nb, tw, tc5, status, s);
        return terms ? launch_rows_tc(false, spec, out, rows, cols, nb, tw, terms, s)
                     : launch_rows_inv(spec, out, rows, cols, nb, tw, reinterpret_cast<int *>(p->ws + p->off_status), s);
    });
}

int fft2_filter_ifft2(gbfft_plan_t p, const float *img, const float *H, float *out, gbfft_stream_t stream) {
    int rc = check_plan_ready(p);
    if (rc) return rc;
    if (p->kind != KIND_2D) return GBFFT_ERR_INVALID_VALUE;
    if (!img || !H || !out) return GBFFT_ERR_NULL;
    if (misaligned(img) || misaligned(H) || misaligned(out)) return GBFFT_ERR_MISALIGNED;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int64_t np = (int64_t)(1 << p->log2r) << p->log2c;
    for (int64_t b0 = 0; b0 < p->batch; b0 += p->chunk) {
        const int nb = (int)((p->batch - b0 < p->chunk) ? p->batch - b0 : p->chunk);
        rc = pipeline_chunk(p, img + b0 * np, H + b0 * p->opt_h_stride, out + b0 * np, nb, b0 == 0, s);
        if (rc) return rc;
    }
    return GBFFT_OK;
}

int fft2_filter_prepare(gbfft_plan_t p, const float *H, gbfft_stream_t stream) {
    int rc = check_plan_ready(p);
    if (rc) return rc;
    if (p->kind != KIND_2D) return GBFFT_ERR_INVALID_VALUE;
    if (!H) return GBFFT_ERR_NULL;
    if (misaligned(H)) return GBFFT_ERR_MISALIGNED;
    if (p->opt_h_stride != 0) return GBFFT_ERR_UNSUPPORTED;  // one filter for every image
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int rows = 1 << p->log2r, cols = 1 << p->log2c;
    const float scale = (float)(1.0 / ((double)rows * cols));
    p->prepared = false;
    rc = launch(p, GBFFT_STAGE_FILTER_PREP, s, [&] {
        return launch_filter_prep(H, reinterpret_cast<float *>(p->ws + p->off_hs),
                                  reinterpret_cast<float *>(p->ws + p->off_beta), rows, cols, 1, scale, 0, 0, 0, s);
    });
    if (rc) return rc;
    p->prepared = true;
    return GBFFT_OK;
}

int fft2_filter_ifft2_prepared(gbfft_plan_t p, const float *img, float *out, gbfft_stream_t stream) {
    int rc = check_plan_ready(p);
    if (rc) return rc;
    if (p->kind != KIND_2D) return GBFFT_ERR_INVALID_VALUE;
    if (!img || !out) return GBFFT_ERR_NULL;
    if (misaligned(img) || misaligned(out)) return GBFFT_ERR_MISALIGNED;
    if (!p->prepared) return GBFFT_ERR_INVALID_VALUE;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int64_t np = (int64_t)(1 << p->log2r) << p->log2c;
    for (int64_t b0 = 0; b0 < p->batch; b0 += p->chunk) {
        const int nb = (int)((p->batch - b0 < p->chunk) ? p->batch - b0 : p->chunk);
        rc = pipeline_chunk(p, img + b0 * np, nullptr, out + b0 * np, nb, b0 == 0, s, 0, 0, true);
        if (rc) return rc;
    }
    return GBFFT_OK;
}

static bool misaligned4(const void *q) { return (reinterpret_cast<uintptr_t>(q) & 3) != 0; }

int fft2_filter_ifft2_padded(gbfft_plan_t p, const float *img, int64_t in_rows, int64_t in_cols, const float *H,
                             float *out, gbfft_stream_t stream) {
    int rc = check_plan_ready(p);
    if (rc) return rc;
    if (p->kind != KIND_2D) return GBFFT_ERR_INVALID_VALUE;
    if (!img || !H || !out) return GBFFT_ERR_NULL;
    if (in_rows < 1 || in_cols < 1 || in_rows > (1 << p->log2r) || in_cols > (1 << p->log2c))
        return GBFFT_ERR_INVALID_SIZE;
    if (misaligned4(img) || misaligned4(out) || misaligned(H)) return GBFFT_ERR_MISALIGNED;
    if (p->opt_precision != 0) return GBFFT_ERR_UNSUPPORTED;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int64_t np = in_rows * in_cols;
    for (int64_t b0 = 0; b0 < p->batch; b0 += p->chunk) {
        const int nb = (int)((p->batch - b0 < p->chunk) ? p->batch - b0 : p->chunk);
        rc = pipeline_chunk(p, img + b0 * np, H + b0 * p->opt_h_stride, out + b0 * np, nb, b0 == 0, s, (int)in_rows,
                            (int)in_cols);
        if (rc) return rc;
    }
    return GBFFT_OK;
}

int fft2_filter_ifft2_analytic(gbfft_plan_t p, const float *img, int kind, double p0, double p1, float *out,
                               gbfft_stream_t stream) {
    int rc = check_plan_ready(p);
    if (rc) return rc;
    if (p->kind != KIND_2D) return GBFFT_ERR_INVALID_VALUE;
    if (!img || !out) return GBFFT_ERR_NULL;
    if (misaligned(img) || misaligned(out)) return GBFFT_ERR_MISALIGNED;
    const bool ok = (kind == GBFFT_FILTER_GAUSSIAN && p0 > 0.0) ||
                    (kind == GBFFT_FILTER_BUTTERWORTH && p0 >= 1.0 && p0 <= 16.0 && p0 == (double)(int)p0 && p1 > 0.0) ||
                    (kind == GBFFT_FILTER_DISC && p0 >= 0.0);
    if (!ok) return GBFFT_ERR_INVALID_VALUE;
    if (p->opt_precision != 0) return GBFFT_ERR_UNSUPPORTED;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int rows = 1 << p->log2r, cols = 1 << p->log2c;
    const int64_t np = (int64_t)rows * cols;
    void *spec = p->ws + p->off_buf;
    for (int64_t b0 = 0; b0 < p->batch; b0 += p->chunk) {
        const int nb = (int)((p->batch - b0 < p->chunk) ? p->batch - b0 : p->chunk);
        rc = launch(p, GBFFT_STAGE_ROWS_FWD, s, [&] {
            return launch_rows_fwd(img + b0 * np, spec, rows, cols, nb, p->ws + p->off_tw0, s);
        });
        if (rc) return rc;
        rc = launch(p, GBFFT_STAGE_COLS, s, [&] {
            return launch_cols_analytic(spec, kind, p0, p1, rows, cols, nb, p->ws + p->off_tw1, s);
        });
        if (rc) return rc;
        rc = launch(p, GBFFT_STAGE_ROWS_INV, s, [&] {
            return launch_rows_inv(spec, out + b0 * np, rows, cols, nb, p->ws + p->off_tw0,
                                   reinterpret_cast<int *>(p->ws + p->off_status), s);
        });
        if (rc) return rc;
    }
    return GBFFT_OK;
}

int fft2_spectrum(gbfft_plan_t p, const float *img, int64_t in_rows, int64_t in_cols, float *mag,
                  gbfft_stream_t stream) {
    int rc = check_plan_ready(p);
    if (rc) return rc;
    if (p->kind != KIND_2D) return GBFFT_ERR_INVALID_VALUE;
    if (!img || !mag) return GBFFT_ERR_NULL;
    const int rows = 1 << p->log2r, cols = 1 << p->log2c;
    if (in_rows < 1 || in_cols < 1 || in_rows > rows || in_cols > cols) return GBFFT_ERR_INVALID_SIZE;
    if (misaligned4(img) || misaligned4(mag)) return GBFFT_ERR_MISALIGNED;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    // per-axis: F = DFT2 / (rows cols); Eq. 5: cols times that
    const float scale = (float)(p->opt_scale_conv ? 1.0 / rows : 1.0 / ((double)rows * cols));
    float *mag_T = reinterpret_cast<float *>(p->ws + p->off_hs);  // the prepared-filter area is scratch here
    p->prepared = false;
    float *nyq = reinterpret_cast<float *>(p->ws + p->off_beta);
    const int64_t np = in_rows * in_cols;
    for (int64_t b0 = 0; b0 < p->batch; b0 += p->chunk) {
        const int nb = (int)((p->batch - b0 < p->chunk) ? p->batch - b0 : p->chunk);
        rc = launch(p, GBFFT_STAGE_ROWS_FWD, s, [&] {
            return launch_rows_pad(true, img + b0 * np, p->ws + p->off_buf, rows, cols, nb, (int)in_rows,
                                   (int)in_cols, p->ws + p->off_tw0, s);
        });
        if (rc) return rc;
        for (int i = 0; i < nb; ++i) {
            const char *spec = p->ws + p->off_buf + (size_t)i * (size_t)rows * (cols / 2) * 8;
            rc = launch(p, GBFFT_STAGE_SPECTRUM, s, [&] {
                cudaError_t e = launch_cols_spectrum(spec, mag_T, nyq, scale, rows, cols, p->ws + p->off_tw1, s);
                if (e == cudaSuccess)
                    e = launch_grad_scatter(mag_T, nyq, mag + (b0 + i) * (int64_t)rows * cols, rows, cols, s);
                return e;
            });
            if (rc) return rc;
        }
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
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int rows = 1 << p->log2r, cols = 1 << p->log2c;
    const int64_t np = (int64_t)rows * cols;
    if (!grad_H) {  // grad_img only: the pipeline itself, applied to grad_out
        for (int64_t b0 = 0; b0 < p->batch; b0 += p->chunk) {
            const int nb = (int)((p->batch - b0 < p->chunk) ? p->batch - b0 : p->chunk);
            rc = pipeline_chunk(p, grad_out + b0 * np, H + b0 * p->opt_h_stride, grad_img + b0 * np, nb, b0 == 0, s);
            if (rc) return rc;
        }
        return GBFFT_OK;
    }
    if (p->opt_h_stride != 0) return GBFFT_ERR_UNSUPPORTED;  // grad of a shared filter only
    if (!p->opt_backward) return GBFFT_ERR_WORKSPACE;         // needs the second spectrum buffer
    void *spec_x = p->ws + p->off_buf, *spec_g = p->ws + p->off_buf2;
    float *hs = reinterpret_cast<float *>(p->ws + p->off_hs);
    p->prepared = false;  // its own preparation overwrites the prepared filter
    float *beta = reinterpret_cast<float *>(p->ws + p->off_beta);
    float *grad_T = reinterpret_cast<float *>(p->ws + p->off_grad);
    const float scale = (float)(1.0 / (double)np);
    for (int64_t b0 = 0; b0 < p->batch; b0 += p->chunk) {
        const int nb = (int)((p->batch - b0 < p->chunk) ? p->batch - b0 : p->chunk);
        if (b0 == 0) {  // the shared filter, prepared once
            rc = launch(p, GBFFT_STAGE_FILTER_PREP, s, [&] {
                return launch_filter_prep(H, hs, beta, rows, cols, 1, scale, 0, 0, 0, s);
            });
            if (rc) return rc;
        }
        rc = launch(p, GBFFT_STAGE_ROWS_FWD, s, [&] {
            return launch_rows_fwd(img + b0 * np, spec_x, rows, cols, nb, p->ws + p->off_tw0, s);
        });
        if (rc) return rc;
        rc = launch(p, GBFFT_STAGE_ROWS_FWD, s, [&] {
            return launch_rows_fwd(grad_out + b0 * np, spec_g, rows, cols, nb, p->ws + p->off_tw0, s);
        });
        if (rc) return rc;
        rc = launch(p, GBFFT_STAGE_COLS_GRAD, s, [&] {
            return launch_cols_grad(spec_x, spec_g, hs, beta, grad_T, rows, cols, nb, scale, b0 > 0 ? 1 : 0,
                                    p->ws + p->off_tw1, s);
        });
        if (rc) return rc;
        if (grad_img) {
            rc = launch(p, GBFFT_STAGE_ROWS_INV, s, [&] {
                return launch_rows_inv(spec_g, grad_img + b0 * np, rows, cols, nb, p->ws + p->off_tw0,
                                       reinterpret_cast<int *>(p->ws + p->off_status), s);
            });
            if (rc) return rc;
        }
    }
    return launch(p, GBFFT_STAGE_COLS_GRAD, s, [&] {
        return launch_grad_scatter(grad_T, grad_T + (size_t)(cols / 2) * rows, grad_H, rows, cols, s);
    });
}

int fft2_slab_plan_create(int64_t rows, int64_t cols, int nranks, int rank, gbfft_plan_t *out) {
    if (!out) return GBFFT_ERR_NULL;
    *out = nullptr;
    const int lr = ilog2_exact(rows), lc = ilog2_exact(cols), ln = ilog2_exact(nranks);
    if (lr < 1 || lc < 2 || lr > kMax2DLog2 || lc > kMax2DLog2 || ln < 0) return GBFFT_ERR_INVALID_SIZE;
    if (rank < 0 || rank >= nranks) return GBFFT_ERR_INVALID_VALUE;
    // every rank: whole row-pass blocks of pairs and at least one column
    int g = rows_pairs_per_block((int)cols);
    if (g > rows / 2) g = (int)(rows / 2);
    const int64_t pairs = rows / 2 / nranks;
    if (pairs < g || pairs % g != 0 || cols / 2 / nranks < 1) return GBFFT_ERR_INVALID_SIZE;
    gbfft_plan *p = new (std::nothrow) gbfft_plan();
    if (!p) return GBFFT_ERR_UNSUPPORTED;
    p->kind = KIND_SLAB;
    p->dtype = GBFFT_C64;
    p->batch = 1;
    p->log2r = lr;
    p->log2c = lc;
    p->nranks = nranks;
    p->rank = rank;
    layout(p);
    *out = p;
    return GBFFT_OK;
}

int fft2_slab_exchange_elems(gbfft_plan_t p, int64_t *count) {
    if (!p || !count) return GBFFT_ERR_NULL;
    if (p->kind != KIND_SLAB) return GBFFT_ERR_INVALID_VALUE;
    *count = ((int64_t(1) << p->log2c) / 2) * ((int64_t(1) << p->log2r) / p->nranks);
    return GBFFT_OK;
}

static int slab_ready(gbfft_plan *p) {
    int rc = check_plan_ready(p);
    if (rc) return rc;
    return p->kind == KIND_SLAB ? GBFFT_OK : GBFFT_ERR_INVALID_VALUE;
}

int fft2_slab_rows_forward(gbfft_plan_t p, const float *img, void *send, gbfft_stream_t stream) {
    int rc = slab_ready(p);
    if (rc) return rc;
    if (!img || !send) return GBFFT_ERR_NULL;
    if (misaligned(img) || misaligned(send)) return GBFFT_ERR_MISALIGNED;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int rows = 1 << p->log2r, cols = 1 << p->log2c;
    const int ld = rows / p->nranks;  // this rank's slots per column
    return launch(p, GBFFT_STAGE_ROWS_FWD, s, [&] {
        return launch_rows_fwd(img, send, rows, cols, 1, p->ws + p->off_tw0, s, Slab{p->rank * ld / 2, ld});
    });
}

int fft2_slab_columns(gbfft_plan_t p, void *recv, const float *H, gbfft_stream_t stream) {
    int rc = slab_ready(p);
    if (rc) return rc;
    if (!recv || !H) return GBFFT_ERR_NULL;
    if (misaligned(recv) || misaligned(H)) return GBFFT_ERR_MISALIGNED;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int rows = 1 << p->log2r, cols = 1 << p->log2c;
    const int mloc = cols / 2 / p->nranks, kbase = p->rank * mloc;
    const int ld = rows / p->nranks;
    float *hs = reinterpret_cast<float *>(p->ws + p->off_hs);
    float *beta = reinterpret_cast<float *>(p->ws + p->off_beta);
    const float scale = (float)(1.0 / ((double)rows * cols));
    rc = launch(p, GBFFT_STAGE_FILTER_PREP, s, [&] {
        return launch_filter_prep(H, hs, beta, rows, cols, 1, scale, 0, 0, 0, s, kbase, mloc);
    });
    if (rc) return rc;
    return launch(p, GBFFT_STAGE_COLS, s, [&] {
        return launch_cols_filter(recv, hs, beta, 0, 0, rows, cols, 1, p->ws + p->off_tw1,
                                  reinterpret_cast<int *>(p->ws + p->off_status), s,
                                  ColSlab{ilog2_exact(ld), mloc, kbase}, (int)p->opt_colform);
    });
}

int fft2_slab_rows_inverse(gbfft_plan_t p, const void *back, float *out, gbfft_stream_t stream) {
    int rc = slab_ready(p);
    if (rc) return rc;
    if (!back || !out) return GBFFT_ERR_NULL;
    if (misaligned(back) || misaligned(out)) return GBFFT_ERR_MISALIGNED;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int rows = 1 << p->log2r, cols = 1 << p->log2c;
    const int ld = rows / p->nranks;
    return launch(p, GBFFT_STAGE_ROWS_INV, s, [&] {
        return launch_rows_inv(back, out, rows, cols, 1, p->ws + p->off_tw0,
                               reinterpret_cast<int *>(p->ws + p->off_status), s, Slab{p->rank * ld / 2, ld});
    });
}

int fft2_batched_plan_create(int count, const int64_t *rows, const int64_t *cols, gbfft_plan_t *out) {
    if (!out) return GBFFT_ERR_NULL;
    *out = nullptr;
    if (!rows || !cols) return GBFFT_ERR_NULL;
    if (count < 1) return GBFFT_ERR_INVALID_SIZE;
    gbfft_plan *p = new (std::nothrow) gbfft_plan();
    if (!p) return GBFFT_ERR_UNSUPPORTED;
    p->kind = KIND_BATCH;
    p->dtype = GBFFT_C64;
    p->batch = count;
    struct Costed {
        double cost;
        BatchItem it;
    };
    std::vector<Costed> work[kBatchStages];
    for (int i = 0; i < count; ++i) {
        const int lr = ilog2_exact(rows[i]), lc = ilog2_exact(cols[i]);
        if (lr < kBatchMinLog2 || lr > kBatchMaxLog2 || lc < kBatchMinLog2 || lc > kBatchMaxLog2) {
            delete p;
            return GBFFT_ERR_INVALID_SIZE;
        }
        BatchImage im = {};
        im.rows = (int)rows[i];
        im.cols = (int)cols[i];
        im.log2r = lr;
        im.log2c = lc;
        int g = batch_row_pairs(im.cols);
        if (g > im.rows / 2) g = im.rows / 2;
        im.log2g = ilog2_exact(g);
        im.scale = (float)(1.0 / ((double)im.rows * im.cols));
        p->bimgs.push_back(im);
        const int nrow = (im.rows / 2) / g;
        const double crow = 2.0 * g * im.cols * lc;
        for (int bx = 0; bx < nrow; ++bx) {
            work[0].push_back({crow, {i, bx}});
            work[2].push_back({crow, {i, bx}});
        }
        const int w = batch_col_width(im.rows);
        const int ncol = (im.cols / 2 + w - 1) / w;
        const double ccol = 2.0 * w * im.rows * lr;
        for (int bx = 0; bx < ncol; ++bx) work[1].push_back({ccol, {i, bx}});
        const int nprep = batch_prep_tiles(im.rows, im.cols);
        const double cprep = (double)im.rows * im.cols / 2 / nprep;
        for (int bx = 0; bx < nprep; ++bx) work[3].push_back({cprep, {i, bx}});
        p->bsmem[0] = std::max(p->bsmem[0], batch_row_smem(im.cols, true));
        p->bsmem[2] = std::max(p->bsmem[2], batch_row_smem(im.cols, false));
        p->bsmem[1] = std::max(p->bsmem[1], batch_col_smem(im.rows));
        p->bsmem[3] = std::max(p->bsmem[3], batch_prep_smem(im.rows, im.cols));
    }
    for (int st = 0; st < kBatchStages; ++st) {
        // largest first; equal costs keep image order
        std::stable_sort(work[st].begin(), work[st].end(),
                         [](const Costed &a, const Costed &b) { return a.cost > b.cost; });
        for (const Costed &c : work[st]) p->bitems[st].push_back(c.it);
    }
    // shape classes, the largest images first (their launches fill the GPU
    // while the small classes run beside them)
    std::map<std::pair<int, int>, int> cls;
    for (int i = 0; i < count; ++i) {
        const auto key = std::make_pair((int)rows[i], (int)cols[i]);
        auto it = cls.find(key);
        if (it == cls.end()) {
            it = cls.emplace(key, (int)p->bclasses.size()).first;
            p->bclasses.push_back(gbfft_plan::BatchClass{(int)rows[i], (int)cols[i], {}, 0, 0, 0, 0});
        }
        p->bclasses[it->second].imgs.push_back(i);
    }
    std::stable_sort(p->bclasses.begin(), p->bclasses.end(), [](const auto &a, const auto &b) {
        return (long long)a.rows * a.cols > (long long)b.rows * b.cols;
    });
    layout(p);
    *out = p;
    return GBFFT_OK;
}

int fft2_filter_ifft2_batched(gbfft_plan_t p, const gbfft_image_ptrs *images, gbfft_stream_t stream) {
    int rc = check_plan_ready(p);
    if (rc) return rc;
    if (p->kind != KIND_BATCH) return GBFFT_ERR_INVALID_VALUE;
    if (!images) return GBFFT_ERR_NULL;
    if (misaligned(images)) return GBFFT_ERR_MISALIGNED;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int grid[kBatchStages];
    cudaError_t e = cudaSuccess;
    for (int st = 0; st < kBatchStages; ++st) {
        grid[st] = batched_grid(p, st, &e);
        if (e != cudaSuccess) return cuda_fail(e);
    }
    if (!p->opt_graph && !p->opt_profile) {
        e = batched_launch_all(p, images, s, grid);
        return e == cudaSuccess ? GBFFT_OK : cuda_fail(e);
    }
    if (!p->opt_graph && p->opt_batch_form != 1) {  // profiling the class form: one event pair around it
        return launch(p, GBFFT_STAGE_GRAPH, s, [&] { return batched_launch_classes(p, images, s); });
    }
    if (!p->opt_graph) {  // profiling: every stage alone on the caller's stream
        for (int st : kBatchOrder) {
            const int stage = st == 0   ? GBFFT_STAGE_ROWS_FWD
                              : st == 1 ? GBFFT_STAGE_COLS
                              : st == 2 ? GBFFT_STAGE_ROWS_INV
                                        : GBFFT_STAGE_FILTER_PREP;
            rc = launch(p, stage, s, [&] {
                return launch_batched_stage(st, grid[st], p->bsmem[st],
                                            reinterpret_cast<const BatchImage *>(p->ws + p->off_bimgs),
                                            reinterpret_cast<const BatchItem *>(p->ws + p->off_bitems[st]),
                                            (int)p->bitems[st].size(), images, p->ws, s);
            });
            if (rc) return rc;
        }
        return GBFFT_OK;
    }
    bool same_grid = true;
    for (int st = 0; st < kBatchStages; ++st) same_grid = same_grid && p->graph_grid[st] == grid[st];
    if (!p->graph_exec || p->graph_ptrs != images || !same_grid) {
        drop_graph(p);
        if (!p->cap_stream && (e = cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking)) != cudaSuccess)
            return cuda_fail(e);
        e = cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return cuda_fail(e);
        cudaError_t le = batched_launch_all(p, images, p->cap_stream, grid);
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(p->cap_stream, &g);
        if (le != cudaSuccess || e != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return cuda_fail(le != cudaSuccess ? le : e);
        }
        p->graph = g;
        e = cudaGraphInstantiate(&p->graph_exec, p->graph, 0);
        if (e != cudaSuccess) {
            drop_graph(p);
            return cuda_fail(e);
        }
        p->graph_ptrs = images;
        for (int st = 0; st < kBatchStages; ++st) p->graph_grid[st] = grid[st];
    }
    return launch(p, GBFFT_STAGE_GRAPH, s, [&] { return cudaGraphLaunch(p->graph_exec, s); });
}

}  // extern "C"

// ---- autotuner ---------------------------------------------------------

namespace {

// Median of `reps` timed runs of f on s (one untimed run first), in ms.
template <typename F>
cudaError_t time_median(cudaStream_t s, int reps, F &&f, float *ms_out) {
    cudaEvent_t a = nullptr, b = nullptr;
    cudaError_t e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    std::vector<float> t;
    if (e == cudaSuccess && f() != GBFFT_OK) e = cudaErrorUnknown;
    for (int r = 0; r < reps && e == cudaSuccess; ++r) {
        e = cudaEventRecord(a, s);
        if (e == cudaSuccess && f() != GBFFT_OK) e = cudaErrorUnknown;
        if (e == cudaSuccess) e = cudaEventRecord(b, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(b);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
        t.push_back(ms);
    }
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    if (e == cudaSuccess) {
        std::sort(t.begin(), t.end());
        *ms_out = t[t.size() / 2];
    }
    return e;
}

std::string plan_signature(const gbfft_plan *p) {
    char buf[160];
    if (p->kind == KIND_1D) {
        snprintf(buf, sizeof buf, "1d:n=%d:b=%lld:t=%d", p->log2n, (long long)p->batch, p->dtype);
    } else if (p->kind == KIND_2D) {
        snprintf(buf, sizeof buf, "2d:r=%d:c=%d:b=%lld:h=%d:p=%lld:bw=%lld", p->log2r, p->log2c, (long long)p->batch,
                 p->opt_h_stride ? 1 : 0, (long long)p->opt_precision, (long long)p->opt_backward);
    } else if (p->kind == KIND_BATCH) {
        uint64_t h = 1469598103934665603ull;  // FNV-1a over the shapes
        for (const BatchImage &im : p->bimgs) {
            h = (h ^ (uint64_t)im.log2r) * 1099511628211ull;
            h = (h ^ (uint64_t)im.log2c) * 1099511628211ull;
        }
        snprintf(buf, sizeof buf, "batch:n=%zu:h=%016llx", p->bimgs.size(), (unsigned long long)h);
    } else {
        snprintf(buf, sizeof buf, "slab:r=%d:c=%d:n=%d", p->log2r, p->log2c, p->nranks);
    }
    return std::string(buf);
}

// Apply a cached entry; false if it lacks what this plan kind tunes.
bool apply_tuned(gbfft_plan *p, const TuneEntry &e) {
    auto get = [&](const char *k, int64_t *v) {
        auto it = e.find(k);
        if (it == e.end()) return false;
        *v = (int64_t)it->second;
        return true;
    };
    if (p->kind == KIND_BATCH) {
        int64_t v[kBatchStages];
        for (int st = 0; st < kBatchStages; ++st) {
            char k[8];
            snprintf(k, sizeof k, "bps%d", st);
            if (!get(k, &v[st]) || v[st] < 1 || v[st] > 64) return false;
        }
        int64_t form = 0;
        if (!get("form", &form) || form < 0 || form > 1) return false;
        for (int st = 0; st < kBatchStages; ++st) p->opt_bps[st] = v[st];
        p->opt_batch_form = form;
        drop_graph(p);
        return true;
    }
    int64_t form = 0, onchip = 0;
    if (!get("column_form", &form) || !get("onchip", &onchip)) return false;
    if (form < 0 || form > 3 || onchip < 0 || onchip > 2) return false;
    p->opt_colform = form;
    p->opt_onchip = onchip;
    return true;
}

// 2D plans: the column-pass form (columns of 4096 rows) and the one-launch
// on-chip path against the three-pass path (sides <= 256), timed on the
// caller's image, filter and output.
int tune_2d(gbfft_plan *p, const gbfft_tune_args *a, cudaStream_t s, TuneEntry &out) {
    const int rows = 1 << p->log2r, cols = 1 << p->log2c;
    std::vector<int> forms = {p->opt_colform ? (int)p->opt_colform : 1};
    if (rows == 4096 && p->opt_precision == 0) forms = {1, 2, 3};
    std::vector<int> onchips = {(int)p->opt_onchip};
    if (p->opt_precision == 0 && onchip_supported(rows, cols)) onchips = {1, 0};
    const float *img = static_cast<const float *>(a->in), *H = static_cast<const float *>(a->H);
    float *o = static_cast<float *>(a->out);
    float best = 0.f, first = 0.f;
    int bf = forms[0], bo = onchips[0];
    bool have = false;
    for (int oc : onchips) {
        for (int f : forms) {
            if (oc && onchip_supported(rows, cols) && f != forms[0]) continue;  // the on-chip path has no column pass
            p->opt_colform = f;
            p->opt_onchip = oc;
            float ms = 0.f;
            cudaError_t e = time_median(
                s, 7, [&] { return fft2_filter_ifft2(p, img, H, o, reinterpret_cast<gbfft_stream_t>(s)); }, &ms);
            if (e != cudaSuccess) return cuda_fail(e);
            if (!have) first = ms;
            if (!have || ms < 0.99f * best) {  // a later candidate must win by more than 1 %
                best = ms;
                bf = f;
                bo = oc;
                have = true;
            }
        }
    }
    p->opt_colform = bf;
    p->opt_onchip = bo;
    out["column_form"] = bf;
    out["onchip"] = bo;
    out["us"] = 1e3 * best;
    out["us_first_candidate"] = 1e3 * first;
    return GBFFT_OK;
}

// 1D plans: the one-cluster path against the four-step passes (complex64
// lengths 2^15 .. 2^17), timed on the caller's input and output.
int tune_1d(gbfft_plan *p, const gbfft_tune_args *a, cudaStream_t s, TuneEntry &out) {
    std::vector<int> onchips = {(int)p->opt_onchip};
    if (p->log2n > max_single_log2(p) && fft1d_cluster_supported(p->log2n, is_dbl(p))) onchips = {1, 2};
    float best = 0.f, first = 0.f;
    int bo = onchips[0];
    bool have = false;
    for (int oc : onchips) {
        p->opt_onchip = oc;
        float ms = 0.f;
        cudaError_t e = time_median(s, 7, [&] { return run_1d(p, a->in, a->out, -1, s); }, &ms);
        if (e != cudaSuccess) return cuda_fail(e);
        if (!have) first = ms;
        if (!have || ms < 0.99f * best) {
            best = ms;
            bo = oc;
            have = true;
        }
    }
    p->opt_onchip = bo;
    out["column_form"] = (double)p->opt_colform;
    out["onchip"] = bo;
    out["us"] = 1e3 * best;
    out["us_first_candidate"] = 1e3 * first;
    return GBFFT_OK;
}

// Batched plans: blocks per SM of each stage, each stage timed alone while
// the others keep their current shape.
int tune_batched(gbfft_plan *p, const gbfft_image_ptrs *images, cudaStream_t s, TuneEntry &out) {
    cudaEvent_t a = nullptr, b = nullptr;
    cudaError_t e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    if (e != cudaSuccess) return cuda_fail(e);
    const int nsm = sm_count();
    int grid[kBatchStages], fits[kBatchStages] = {1, 1, 1, 1};
    // occupancy of every stage first: this also sets each kernel's shared
    // memory attributes, which every launch below needs
    for (int st = 0; st < kBatchStages && e == cudaSuccess; ++st) {
        e = batch_max_blocks_per_sm(st, p->bsmem[st], &fits[st]);
        if (fits[st] < 1) fits[st] = 1;
    }
    for (int st = 0; st < kBatchStages && e == cudaSuccess; ++st) {
        const int fit = fits[st];
        for (int q = 0; q < kBatchStages; ++q) grid[q] = (p->opt_bps[q] > 0 ? (int)p->opt_bps[q] : fits[q]) * nsm;
        float best = 1e30f;
        int best_bps = fit;
        for (int bps = 1; bps <= fit && e == cudaSuccess; ++bps) {
            grid[st] = bps * nsm;
            float total = 0.f;
            for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
                for (int q : kBatchOrder) {
                    if (e != cudaSuccess) break;
                    if (q == st) e = cudaEventRecord(a, s);
                    if (e == cudaSuccess)
                        e = launch_batched_stage(q, grid[q], p->bsmem[q],
                                                 reinterpret_cast<const BatchImage *>(p->ws + p->off_bimgs),
                                                 reinterpret_cast<const BatchItem *>(p->ws + p->off_bitems[q]),
                                                 (int)p->bitems[q].size(), images, p->ws, s);
                    if (q == st && e == cudaSuccess) e = cudaEventRecord(b, s);
                }
                float ms = 0.f;
                if (e == cudaSuccess) e = cudaEventSynchronize(b);
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
                if (rep > 0) total += ms;  // first repetition warms up
            }
            if (e == cudaSuccess && total < best) {
                best = total;
                best_bps = bps;
            }
        }
        p->opt_bps[st] = best_bps;
        char k[8];
        snprintf(k, sizeof k, "bps%d", st);
        out[k] = best_bps;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    drop_graph(p);
    if (e != cudaSuccess) return cuda_fail(e);
    // then the form: per shape class (default) against the persistent launches
    for (int q = 0; q < kBatchStages; ++q) grid[q] = (int)p->opt_bps[q] * nsm;
    float best = 0.f, first = 0.f;
    int best_form = 0;
    for (int form : {0, 1}) {
        p->opt_batch_form = form;
        float ms = 0.f;
        e = time_median(s, 5, [&] { return batched_launch_all(p, images, s, grid) == cudaSuccess ? GBFFT_OK : GBFFT_ERR_CUDA; },
                        &ms);
        if (e != cudaSuccess) return cuda_fail(e);
        if (form == 0) first = ms;
        if (form == 0 || ms < 0.99f * best) {
            best = ms;
            best_form = form;
        }
    }
    p->opt_batch_form = best_form;
    drop_graph(p);
    out["form"] = best_form;
    out["us"] = 1e3 * best;
    out["us_first_candidate"] = 1e3 * first;
    return GBFFT_OK;
}

}  // namespace

extern "C" {

int fft_plan_autotune(gbfft_plan_t p, const void *args, gbfft_stream_t stream) {
    if (!p) return GBFFT_ERR_NULL;
    int rc = check_plan_ready(p);
    if (rc) return rc;
    if (p->kind == KIND_SLAB) return GBFFT_OK;  // its column pass is tuned through a one-image 2D plan
    if (!args) return GBFFT_ERR_NULL;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (p->kind != KIND_BATCH) {
        const gbfft_tune_args *a = static_cast<const gbfft_tune_args *>(args);
        if (!a->in || !a->out || (p->kind == KIND_2D && !a->H)) return GBFFT_ERR_NULL;
        if (misaligned(a->in) || misaligned(a->out) || (p->kind == KIND_2D && misaligned(a->H)))
            return GBFFT_ERR_MISALIGNED;
    }
    const std::string path = tune_cache_path();
    const std::string key = tune_device_key() + "|" + plan_signature(p);
    TuneCache cache;
    tune_cache_load(path, cache);
    auto hit = cache.find(key);
    if (hit != cache.end() && apply_tuned(p, hit->second)) return GBFFT_OK;
    TuneEntry e;
    if (p->kind == KIND_BATCH)
        rc = tune_batched(p, static_cast<const gbfft_image_ptrs *>(args), s, e);
    else if (p->kind == KIND_2D)
        rc = tune_2d(p, static_cast<const gbfft_tune_args *>(args), s, e);
    else
        rc = tune_1d(p, static_cast<const gbfft_tune_args *>(args), s, e);
    if (rc) return rc;
    if (!path.empty()) {
        tune_cache_load(path, cache);  // entries other processes stored meanwhile
        cache[key] = e;
        tune_cache_store(path, cache);  // a cache that cannot be written costs a re-tune, nothing else
    }
    return GBFFT_OK;
}

int fft_plan_get_option(gbfft_plan_t p, int key, int64_t *value) {
    if (!p || !value) return GBFFT_ERR_NULL;
    switch (key) {
        case GBFFT_OPT_SCALE_CONVENTION: *value = p->opt_scale_conv; return GBFFT_OK;
        case GBFFT_OPT_H_BATCH_STRIDE: *value = p->opt_h_stride; return GBFFT_OK;
        case GBFFT_OPT_PRECISION: *value = p->opt_precision; return GBFFT_OK;
        case GBFFT_OPT_IMAGES_PER_CHUNK: *value = p->chunk; return GBFFT_OK;
        case GBFFT_OPT_PROFILE: *value = p->opt_profile; return GBFFT_OK;
        case GBFFT_OPT_ENABLE_BACKWARD: *value = p->opt_backward; return GBFFT_OK;
        case GBFFT_OPT_BLOCKS_PER_SM:
            // three stages packed 8 bits each: forward rows | columns << 8 | inverse rows << 16
            *value = p->opt_bps[0] | (p->opt_bps[1] << 8) | (p->opt_bps[2] << 16) | (p->opt_bps[3] << 24);
            return GBFFT_OK;
        case GBFFT_OPT_USE_GRAPH: *value = p->opt_graph; return GBFFT_OK;
        case GBFFT_OPT_ONCHIP: *value = p->opt_onchip; return GBFFT_OK;
        case GBFFT_OPT_COLUMN_FORM: *value = p->opt_colform; return GBFFT_OK;
        case GBFFT_OPT_BATCH_FORM: *value = p->opt_batch_form; return GBFFT_OK;
        case GBFFT_OPT_FOURSTEP_PASSES: *value = p->fs3 ? 3 : 2; return GBFFT_OK;
        default: return GBFFT_ERR_INVALID_VALUE;
    }
}

int gbfft_device_status(gbfft_plan_t p) {
    int rc = check_plan_ready(p);
    if (rc) return rc;
    int word = 0;
    cudaError_t e = cudaMemcpy(&word, p->ws + p->off_status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && word != 0) e = cudaMemset(p->ws + p->off_status, 0, sizeof(int));
    if (e != cudaSuccess) return cuda_fail(e);
    return word ? GBFFT_ERR_TIMEOUT : GBFFT_OK;
}

int gbfft_plan_check_guards(gbfft_plan_t p, int64_t *bad_words) {
    int rc = check_plan_ready(p);
    if (rc) return rc;
    if (!bad_words) return GBFFT_ERR_NULL;
    // wait for the plan's work on every stream, then check on the legacy stream
    cudaError_t e = cudaDeviceSynchronize();
    unsigned *bad = reinterpret_cast<unsigned *>(p->ws + p->off_status + sizeof(int));
    if (e == cudaSuccess) e = cudaMemsetAsync(bad, 0, sizeof(unsigned), 0);
    if (e == cudaSuccess)
        e = launch_guard_check(p->ws, reinterpret_cast<const long long *>(p->ws + p->off_guards),
                               (int)p->guards.size(), (long long)p->ws_bytes, bad, 0);
    unsigned n = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&n, bad, sizeof n, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e);
    *bad_words = (int64_t)n;
    return GBFFT_OK;
}

int gbfft_checked_take(int64_t *first_site, int64_t *failures) {
    if (!first_site || !failures) return GBFFT_ERR_NULL;
    *first_site = 0;
    *failures = 0;
    if (!kChecked) return GBFFT_ERR_UNSUPPORTED;
    cudaError_t e = cudaDeviceSynchronize();
    cudaError_t (*takes[])(unsigned *) = {check_take_rows, check_take_cols, check_take_batched, check_take_fourstep,
                                          check_take_tc2d, check_take_tc5};
    for (auto take : takes) {
        unsigned w[2] = {0u, 0u};
        if (e == cudaSuccess) e = take(w);
        if (!*first_site && w[0]) *first_site = w[0];
        *failures += w[1];
    }
    return e == cudaSuccess ? GBFFT_OK : cuda_fail(e);
}

int gbfft_selftest_wait_timeout(gbfft_plan_t p, int64_t polls, gbfft_stream_t stream) {
    int rc = check_plan_ready(p);
    if (rc) return rc;
    if (polls < 1 || polls > (int64_t)kTmaPolls) return GBFFT_ERR_INVALID_VALUE;
    cudaError_t e = launch_wait_timeout(reinterpret_cast<int *>(p->ws + p->off_status), (unsigned)polls,
                                        static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? GBFFT_OK : cuda_fail(e);
}

int gbfft_selftest_corrupt_work_item(gbfft_plan_t p, int stage, int64_t index, int img, int bx) {
    if (!p) return GBFFT_ERR_NULL;
    if (p->kind != KIND_BATCH || stage < 0 || stage >= kBatchStages || index < 0 ||
        index >= (int64_t)p->bitems[stage].size())
        return GBFFT_ERR_INVALID_VALUE;
    p->bitems[stage][index] = BatchItem{img, bx};
    p->bound = false;  // the device copy no longer matches: the plan must be bound again
    return GBFFT_OK;
}

int gbfft_selftest_launch_config(gbfft_stream_t stream) {
    const cudaError_t e = launch_bad_config(static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? GBFFT_OK : cuda_fail(e);
}

int fft_plan_destroy(gbfft_plan_t p) {
    if (!p) return GBFFT_ERR_NULL;
    drop_graph(p);
    if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
    if (p->aux) cudaStreamDestroy(p->aux);
    if (p->ev_fork) cudaEventDestroy(p->ev_fork);
    if (p->ev_join) cudaEventDestroy(p->ev_join);
    if (p->ev_join2) cudaEventDestroy(p->ev_join2);
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
