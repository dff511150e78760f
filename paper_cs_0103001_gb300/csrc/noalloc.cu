// noalloc.cu — an allocation-free variant of the filter pipeline entry point.
//
// fft2_filter_ifft2 needs a workspace (twiddle tables and the half spectra
// between its three kernels) that the caller allocates and binds.  Some
// callers cannot do that: code that must not call cudaMalloc once it is
// running (real-time or embedded loops, where an allocation can block or
// synchronise the device), and plugins whose host application owns all device
// memory and hands them only their input and output buffers.
// fft2_filter_ifft2_noalloc gives them the same result with no workspace
// argument: its scratch is a fixed, file-scope __device__ array that lives in
// the library image, so the call allocates nothing.
//
// Costs and rules (also stated in gbfft.h):
//  - every GPU that loads the library holds kScratchBytes (about 24.2 MiB)
//    of device memory for this array until the process exits, used or not;
//  - rows * cols is limited to kMaxPixels; larger images are rejected;
//  - the first call on a device sets that device up: it looks the array up
//    and writes the twiddle tables of every supported length into it (on the
//    caller's stream, then waits for them); later calls only read the tables;
//  - all calls share the one array: calls whose work overlaps on the GPU
//    (different streams, or different host threads without ordering) race;
//  - the array keeps the previous call's contents; nothing here needs to
//    start at zero (spectra and prepared filter are fully rewritten by every
//    call, and the tables never change after set-up).
#include <cuda_runtime.h>

#include <mutex>

#include "gbfft.h"
#include "internal.h"

namespace {

constexpr long long kMaxPixels = 2048ll * 2048ll;               // rows * cols
// twiddle tables of every length n = 2 .. 8192 (n - 1 complex64 entries each),
// the table of length n at entry n: [n, 2n) for powers of two never overlap
constexpr size_t kTwiddleBytes = 2 * 8192 * 8;
constexpr size_t kFilterBytes = (size_t)kMaxPixels / 2 * 4;      // prepared filter, float32
constexpr size_t kBetaBytes = 8192 * 4;                          // packed-column coefficients
constexpr size_t kSpectrumBytes = (size_t)kMaxPixels / 2 * 8;    // half spectra, complex64
constexpr size_t kScratchBytes = kTwiddleBytes + kFilterBytes + kBetaBytes + kSpectrumBytes;  // ~24.2 MiB

static_assert(kTwiddleBytes >= 2 * (size_t(1) << gbfft::kMax2DLog2) * 8, "one table per length up to the 2D maximum");

__device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
struct DeviceState {
    unsigned char *base = nullptr;  // device address of g_scratch on this device, once set up
};
DeviceState g_dev[kMaxDevices];
std::mutex g_mu;

int is_pow2_in(long long n, int lo_log2, int hi_log2) {
    if (n < (1ll << lo_log2) || n > (1ll << hi_log2) || (n & (n - 1))) return 0;
    return 1;
}

}  // namespace

extern "C" int fft2_filter_ifft2_noalloc(int64_t rows, int64_t cols, int64_t batch, const float *img,
                                         const float *H, int64_t h_batch_stride, float *out,
                                         gbfft_stream_t stream) {
    using namespace gbfft;
    if (!img || !H || !out) return GBFFT_ERR_NULL;
    if (!is_pow2_in(rows, 1, kMax2DLog2) || !is_pow2_in(cols, 1, kMax2DLog2) || batch < 1 || h_batch_stride < 0)
        return GBFFT_ERR_INVALID_SIZE;
    if (rows * cols > kMaxPixels) return GBFFT_ERR_INVALID_SIZE;  // beyond the static scratch
    if ((reinterpret_cast<uintptr_t>(img) | reinterpret_cast<uintptr_t>(H) | reinterpret_cast<uintptr_t>(out)) & 15u)
        return GBFFT_ERR_MISALIGNED;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) return GBFFT_ERR_CUDA;

    std::lock_guard<std::mutex> lock(g_mu);
    DeviceState &st = g_dev[dev];
    if (!st.base) {
        // first call on this device (the current one): look up where the
        // array lives (the host-side symbol itself is not a device address),
        // then write every length's twiddle table and wait for them, so that
        // calls on any stream can read them afterwards
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p) return GBFFT_ERR_CUDA;
        unsigned char *base = static_cast<unsigned char *>(p);
        for (int n = 2; n <= (1 << kMax2DLog2) && e == cudaSuccess; n *= 2)
            e = launch_twiddles(base + (size_t)n * 8, n, false, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return GBFFT_ERR_CUDA;
        st.base = base;
    }
    const unsigned char *tw_c = st.base + (size_t)cols * 8;  // row transforms: length cols
    const unsigned char *tw_r = st.base + (size_t)rows * 8;  // column transforms: length rows
    float *hs = reinterpret_cast<float *>(st.base + kTwiddleBytes);
    float *beta = reinterpret_cast<float *>(st.base + kTwiddleBytes + kFilterBytes);
    unsigned char *spec = st.base + kTwiddleBytes + kFilterBytes + kBetaBytes;
    const long long np = rows * cols;
    for (long long b = 0; b < batch; ++b) {
        if (b == 0 || h_batch_stride != 0)  // prepare each filter once
            e = launch_filter_prep(H + b * h_batch_stride, hs, beta, (int)rows, (int)cols, 1,
                                   (float)(1.0 / (double)np), 0, 0, 0, s);
        if (e == cudaSuccess) e = launch_rows_fwd(img + b * np, spec, (int)rows, (int)cols, 1, tw_c, s);
        if (e == cudaSuccess) e = launch_cols_filter(spec, hs, beta, 0, 0, (int)rows, (int)cols, 1, tw_r, nullptr, s);
        if (e == cudaSuccess) e = launch_rows_inv(spec, out + b * np, (int)rows, (int)cols, 1, tw_c, nullptr, s);
        if (e != cudaSuccess) return GBFFT_ERR_CUDA;
    }
    return GBFFT_OK;
}
