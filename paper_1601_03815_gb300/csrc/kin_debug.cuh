// Index checks of the KIN_DEBUG build (compute-sanitizer's substitute).
//
// With KIN_DEBUG defined, the stencil kernels check the global offsets and
// shared-memory slot and row indices they are about to use.  A failed check
// skips that access (no trap, no fault: the kernel runs on and the context
// stays usable) and records the first failure of the translation unit in a
// device word: bits 40..47 the check site, bits 0..39 the offending value.
// The host reads the word through debug_word_<unit>() and kin_debug_status.
// Without KIN_DEBUG every check is the constant true and compiles away.
#pragma once

#include <cuda_runtime.h>

namespace kin {

// Check sites.
enum : unsigned {
    DBG_DUGKS_LOAD = 1,   // global f-tilde read of the DUGKS tile (copy or load)
    DBG_DUGKS_STORE = 2,  // global store of the new f-tilde / velocity
    DBG_DUGKS_SLOT = 3,   // ring / staging slot index
    DBG_DUGKS_ROW = 4,    // row index of a y neighbour
    DBG_LBE_LOAD = 5,     // global pull of the LBE node
    DBG_LBE_STORE = 6,    // global store of the LBE node
};

#ifdef KIN_DEBUG
static __device__ unsigned long long g_kin_dbg = 0;

__device__ __forceinline__ bool kin_ok(bool ok, unsigned site, long long value) {
    if (!ok)
        atomicCAS(&g_kin_dbg, 0ull,
                  ((unsigned long long)site << 40) | ((unsigned long long)value & ((1ull << 40) - 1)));
    return ok;
}
#define KIN_CHECK(ok, site, value) ::kin::kin_ok((ok), (site), (long long)(value))
// Host accessor of this translation unit's word (reset: clear it after reading).
#define KIN_DEBUG_ACCESSOR(NAME)                                                      \
    cudaError_t NAME(unsigned long long* word, bool reset) {                          \
        cudaError_t e = cudaMemcpyFromSymbol(word, g_kin_dbg, sizeof(*word));           \
        if (e == cudaSuccess && reset) {                                                \
            const unsigned long long z = 0;                                             \
            e = cudaMemcpyToSymbol(g_kin_dbg, &z, sizeof(z));                           \
        }                                                                               \
        return e;                                                                       \
    }
#else
#define KIN_CHECK(ok, site, value) true
#define KIN_DEBUG_ACCESSOR(NAME)                                  \
    cudaError_t NAME(unsigned long long* word, bool) {            \
        *word = 0;                                                \
        return cudaSuccess;                                       \
    }
#endif

}  // namespace kin
