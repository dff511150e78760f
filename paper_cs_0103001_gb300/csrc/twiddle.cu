// twiddle.cu — per-plan twiddle tables, computed on the GPU in FP64.
//
// Table 2 of arXiv cs/0103001 keeps the vector Z_j = exp(-2 pi i j / N) of
// all twiddle factors.  Each factor here is likewise computed from its exact
// integer phase with the FP64 sincospi routine and rounded once to the
// working precision; only the layout differs (per Stockham pass, see
// fft_core.cuh, and a two-level table for the four-step inter-pass factors).
#include "fft_core.cuh"
#include "internal.h"

namespace gbfft {

template <typename C>
__global__ void k_stockham_twiddles(C *tw, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int np = plan_passes(n);
    if (np < 2 || i >= n - 1) return;
    // pass p >= 1 owns entries [Ns_p - 1, Ns_{p+1} - 1), Ns_np = n
    int p = 1;
    while (p + 1 < np && i >= plan_stride(n, p + 1) - 1) ++p;
    const int ns = plan_stride(n, p);
    const int local = i - (ns - 1);
    const int r = local / ns + 1;
    const int m = local % ns;
    const long long ph = (long long)r * m;          // exact phase numerator
    const long long den = (long long)ns * plan_radix(n, p);
    double s, c;
    sincospi(-2.0 * (double)ph / (double)den, &s, &c);
    tw[i] = C{(decltype(tw[0].x))c, (decltype(tw[0].x))s};
}

// Two-level table for W_n^idx, idx < n: entries [0, F) hold W_n^b (b < F),
// entries [F, F + n/F) hold W_n^(a F) (a < n/F), with F = 2^ceil(log2(n)/2).
template <typename C>
__global__ void k_fourstep_twiddles(C *tw, int n, int log2f) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int f = 1 << log2f;
    const int total = f + (n >> log2f);
    if (i >= total) return;
    const long long ph = i < f ? (long long)i : (long long)(i - f) << log2f;
    double s, c;
    sincospi(-2.0 * (double)ph / (double)n, &s, &c);
    tw[i] = C{(decltype(tw[0].x))c, (decltype(tw[0].x))s};
}

// Full inter-pass table of the split n = n1 n2: entry k1 * n2 + j2 holds
// W_n^(k1 j2) (k1 j2 < n, so the phase needs no reduction).
__global__ void k_fourstep_full_twiddles(float2 *tw, int n, int log2n2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const long long ph = (long long)(i >> log2n2) * (i & ((1 << log2n2) - 1));
    double s, c;
    sincospi(-2.0 * (double)ph / (double)n, &s, &c);
    tw[i] = make_float2((float)c, (float)s);
}

// Coarse inter-pass table: entry e * n2 + j2 holds W_(16 n2)^(e j2) (e j2 < 16 n2).
template <typename C>
__global__ void k_fourstep_coarse_twiddles(C *tw, int n2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 16 * n2) return;
    const long long ph = (long long)(i / n2) * (i % n2);
    double s, c;
    sincospi(-2.0 * (double)ph / (16.0 * n2), &s, &c);
    tw[i] = C{(decltype(tw[0].x))c, (decltype(tw[0].x))s};
}

cudaError_t launch_fourstep_coarse_twiddles(void *tw, int n2, bool dbl, cudaStream_t s) {
    const int threads = 256;
    const int blocks = (16 * n2 + threads - 1) / threads;
    if (dbl)
        k_fourstep_coarse_twiddles<double2><<<blocks, threads, 0, s>>>(static_cast<double2 *>(tw), n2);
    else
        k_fourstep_coarse_twiddles<float2><<<blocks, threads, 0, s>>>(static_cast<float2 *>(tw), n2);
    return cudaGetLastError();
}

cudaError_t launch_fourstep_full_twiddles(void *tw, int n, int log2n2, cudaStream_t s) {
    const int threads = 256;
    k_fourstep_full_twiddles<<<(n + threads - 1) / threads, threads, 0, s>>>(static_cast<float2 *>(tw), n, log2n2);
    return cudaGetLastError();
}

cudaError_t launch_twiddles(void *tw, int n, bool dbl, cudaStream_t s) {
    if (n < 2) return cudaSuccess;
    const int threads = 256;
    const int blocks = (n + threads - 1) / threads;
    if (dbl)
        k_stockham_twiddles<double2><<<blocks, threads, 0, s>>>(static_cast<double2 *>(tw), n);
    else
        k_stockham_twiddles<float2><<<blocks, threads, 0, s>>>(static_cast<float2 *>(tw), n);
    return cudaGetLastError();
}

cudaError_t launch_fourstep_twiddles(void *tw, int n, bool dbl, cudaStream_t s) {
    const int L = ilog2(n);
    const int log2f = (L + 1) / 2;
    const int total = (1 << log2f) + (n >> log2f);
    const int threads = 256;
    const int blocks = (total + threads - 1) / threads;
    if (dbl)
        k_fourstep_twiddles<double2><<<blocks, threads, 0, s>>>(static_cast<double2 *>(tw), n, log2f);
    else
        k_fourstep_twiddles<float2><<<blocks, threads, 0, s>>>(static_cast<float2 *>(tw), n, log2f);
    return cudaGetLastError();
}

}  // namespace gbfft
