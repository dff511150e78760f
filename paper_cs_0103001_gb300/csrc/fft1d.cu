// fft1d.cu — batched 1D complex transforms (Eq. E2 forward, Eq. E3 inverse).
//
// One-pass kernel: a thread block owns BPC whole transforms of length N; the
// T = N/E threads of a transform load it straight from HBM in the register
// pattern of fft_core.cuh (consecutive threads read consecutive elements, so
// every warp access is a full 128/256-byte line), run all radix passes with
// shared-memory exchanges, and store it back coalesced with the 1/N of
// Eq. E2 folded into the store.
#include "fft_core.cuh"
#include "internal.h"

namespace gbfft {

template <int N, typename R> struct K1Cfg {
    static constexpr int E = N < 16 ? N : ((sizeof(R) == 4 && N >= 8192) ? 32 : 16);
    static constexpr int T = N / E;
    static constexpr int BPC = N < 16 ? 64 : (T >= 256 ? 1 : 256 / T);
    static constexpr int THREADS = T * BPC;
    static constexpr int SMS = N < 16 ? 0 : padded_len(N);  // complex slots per transform
    static constexpr size_t SMEM = (size_t)BPC * SMS * sizeof(typename cvec<R>::type);
};

template <int N, int DIR, typename R>
__global__ void __launch_bounds__(K1Cfg<N, R>::THREADS)
    k_fft1d(const typename cvec<R>::type *in, typename cvec<R>::type *out, long long batch,
            const typename cvec<R>::type *__restrict__ tw, R scale) {
    typedef typename cvec<R>::type C;
    typedef K1Cfg<N, R> K;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int g = threadIdx.x / K::T;
    const int t = threadIdx.x - g * K::T;
    C *sm = reinterpret_cast<C *>(smraw) + g * K::SMS;
    const long long b = (long long)blockIdx.x * K::BPC + g;
    const bool active = b < batch;
    C v[K::E];
    if (active) {
        const C *src = in + b * N;
#pragma unroll
        for (int e = 0; e < K::E; ++e) v[e] = src[t + K::T * e];
    } else {
#pragma unroll
        for (int e = 0; e < K::E; ++e) v[e] = C{0, 0};
    }
    fft_regs<N, K::E, DIR>(v, sm, tw, t);
    if (active) {
        C *dst = out + b * N;
#pragma unroll
        for (int e = 0; e < K::E; ++e) dst[t + K::T * e] = cscale(v[e], scale);
    }
}

template <int N, typename R>
static cudaError_t run_fft1d(const void *in, void *out, long long batch, int dir, const void *tw, double scale,
                             cudaStream_t s) {
    typedef typename cvec<R>::type C;
    typedef K1Cfg<N, R> K;
    const long long grid = (batch + K::BPC - 1) / K::BPC;
    if (grid > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    auto kern = dir < 0 ? k_fft1d<N, -1, R> : k_fft1d<N, 1, R>;
    cudaError_t e = set_smem_attrs((const void *)kern, K::SMEM);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)grid, K::THREADS, K::SMEM, s>>>(static_cast<const C *>(in), static_cast<C *>(out), batch,
                                                      static_cast<const C *>(tw), (R)scale);
    return cudaGetLastError();
}

template <typename R>
static cudaError_t dispatch_fft1d(const void *in, void *out, int log2n, long long batch, int dir, const void *tw,
                                  double scale, cudaStream_t s) {
    switch (log2n) {
#define GBFFT_CASE(L) \
    case L: return run_fft1d<(1 << L), R>(in, out, batch, dir, tw, scale, s);
        GBFFT_CASE(1) GBFFT_CASE(2) GBFFT_CASE(3) GBFFT_CASE(4) GBFFT_CASE(5) GBFFT_CASE(6) GBFFT_CASE(7)
        GBFFT_CASE(8) GBFFT_CASE(9) GBFFT_CASE(10) GBFFT_CASE(11) GBFFT_CASE(12) GBFFT_CASE(13)
#undef GBFFT_CASE
        case 14:
            if constexpr (sizeof(R) == 4) return run_fft1d<(1 << 14), R>(in, out, batch, dir, tw, scale, s);
            return cudaErrorInvalidValue;
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_fft1d(const void *in, void *out, int log2n, long long batch, bool dbl, int dir, const void *tw,
                         double scale, cudaStream_t s) {
    return dbl ? dispatch_fft1d<double>(in, out, log2n, batch, dir, tw, scale, s)
               : dispatch_fft1d<float>(in, out, log2n, batch, dir, tw, scale, s);
}

}  // namespace gbfft
