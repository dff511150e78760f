// check.cuh — index-bound checks of the GBFFT_CHECKED build (a stand-in for a
// memory checker): at the sites where the kernels derive an address from
// index arithmetic (pair and slot runs, tensor-map boxes, work-list items,
// tensor-memory columns), chk(ok, site) records the first failing site and
// counts failures in a device word, and the caller skips the access.  No
// trap, no assert.  In the normal build chk() is `true` and compiles away.
//
// Without relocatable device code every translation unit has its own word;
// each one that checks exports a reader (check_take_* in internal.h) that
// the C ABI's gbfft_checked_take collects.
#pragma once

#include <cuda_runtime.h>

namespace gbfft {

#ifdef GBFFT_CHECKED
constexpr bool kChecked = true;
#else
constexpr bool kChecked = false;
#endif

// [0] first failing site (0 = none), [1] number of failures
static __device__ unsigned int g_check_word[2];

__device__ __forceinline__ bool chk(bool ok, unsigned site) {
    if constexpr (kChecked) {
        if (!ok) {
            atomicCAS(&g_check_word[0], 0u, site);
            atomicAdd(&g_check_word[1], 1u);
        }
        return ok;
    } else {
        return true;
    }
}

// Host: this translation unit's word (synchronous), cleared after reading.
static inline cudaError_t check_word_take(unsigned out[2]) {
    cudaError_t e = cudaMemcpyFromSymbol(out, g_check_word, 2 * sizeof(unsigned));
    if (e == cudaSuccess && (out[0] | out[1])) {
        const unsigned z[2] = {0u, 0u};
        e = cudaMemcpyToSymbol(g_check_word, z, sizeof z);
    }
    return e;
}

// Check sites (the code names the file and place of the index arithmetic).
enum CheckSite : unsigned {
    CK_ROW_PAIR = 101,      // row pass: pair index below N/2
    CK_ROW_RUN = 102,       // row pass: the block's run of 2G slots inside its column (stride ld)
    CK_PREP_TILE = 103,     // filter preparation: tile inside the filter and the prepared columns
    CK_COL_SLOT = 201,      // column pass: slot index below N
    CK_COL_CHUNK = 202,     // column pass of a decomposed image: local column below mloc
    CK_COL_BOX = 203,       // TMA column pass: a box inside the tensor map's rows
    CK_BATCH_ITEM = 301,    // batched kernels: the item's block inside its image
    CK_FS_A_TILE = 401,     // four-step pass A: the block's columns inside n2
    CK_FS_B_ROWS = 402,     // four-step pass B: the block's rows inside n1
    CK_TC5_TMEM = 501,      // tcgen05 passes: accumulator columns inside the allocation
};

}  // namespace gbfft
