// Standalone launch of the fused DUGKS step (tile code in dugks_tile.cuh).
#include <atomic>

#include "dugks_tile.cuh"
#include "kin_internal.h"

namespace kin {

// VEL: also write the velocity of the new state to uvel (FP32-computed storage).
// EVEN = false: odd N with 2-byte storage, whose tile reads f-tilde from global
// memory directly instead of staging it.
template <typename S, int TY, bool VEL, bool EVEN>
__global__ void __launch_bounds__(32 * (TY + 2), 1)
    dugks_fused_kernel(const S* __restrict__ src, S* __restrict__ dst, int N, int zchunk,
                       DugksCoef<typename Traits<S>::C> kc, float* __restrict__ uvel) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    dugks_tile<S, TY, VEL, EVEN>(src, dst, N, blockIdx.x, blockIdx.y, blockIdx.z, zchunk, kc, smem_raw, uvel);
}

template <typename S, int TY, bool VEL, bool EVEN>
static cudaError_t launch_fused_e(const void* src, void* dst, int N, int zchunk,
                                  const DugksCoef<typename Traits<S>::C>& k, float* uvel, cudaStream_t stream) {
    const size_t smem = fused_smem_bytes<S, TY>();
    // the shared-memory limit is a per-device attribute of the kernel: set it
    // once for every device this process launches on
    static std::atomic<unsigned long long> configured{0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = dev < 64 ? 1ull << dev : 0ull;
    if (!bit || !(configured.load() & bit)) {
        e = cudaFuncSetAttribute(dugks_fused_kernel<S, TY, VEL, EVEN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
        if (e != cudaSuccess) return e;
        configured.fetch_or(bit);
    }
    if (zchunk <= 0) zchunk = 32;
    if (zchunk > N) zchunk = N;
    dim3 block(32, TY + 2);
    dim3 grid((N + 29) / 30, (N + TY - 1) / TY, (N + zchunk - 1) / zchunk);
    dugks_fused_kernel<S, TY, VEL, EVEN><<<grid, block, smem, stream>>>((const S*)src, (S*)dst, N, zchunk, k, uvel);
    return cudaGetLastError();
}

template <typename S, int TY, bool VEL>
static cudaError_t launch_fused_t(const void* src, void* dst, int N, int zchunk,
                                  const DugksCoef<typename Traits<S>::C>& k, float* uvel, cudaStream_t stream) {
    if constexpr (sizeof(S) == 2) {
        if (N % 2) return launch_fused_e<S, TY, VEL, false>(src, dst, N, zchunk, k, uvel, stream);
    }
    return launch_fused_e<S, TY, VEL, true>(src, dst, N, zchunk, k, uvel, stream);
}

template <typename S>
static cudaError_t launch_fused(const void* src, void* dst, int N, double nu, double dt, int ty,
                                int zchunk, float* uvel, cudaStream_t stream) {
    using C = typename Traits<S>::C;
    const DugksCoef<C> k = dugks_coef<C>(nu, dt);
    if constexpr (sizeof(C) == 8) {
        if (uvel) return cudaErrorInvalidValue;  // FP64 storage keeps the FP64 statistics path
        return launch_fused_t<S, 4, false>(src, dst, N, zchunk, k, nullptr, stream);
    } else {
        if (uvel) {
            if (ty == 4) return launch_fused_t<S, 4, true>(src, dst, N, zchunk, k, uvel, stream);
            return launch_fused_t<S, 8, true>(src, dst, N, zchunk, k, uvel, stream);
        }
        if (ty == 4) return launch_fused_t<S, 4, false>(src, dst, N, zchunk, k, nullptr, stream);
        return launch_fused_t<S, 8, false>(src, dst, N, zchunk, k, nullptr, stream);
    }
}

KIN_DEBUG_ACCESSOR(debug_word_dugks)

cudaError_t dugks_step_fused(int storage, const void* src, void* dst, int N, double nu, double dt,
                             int ty, int zchunk, cudaStream_t stream, float* uvel) {
    switch (storage) {
        case ST_F32: return launch_fused<float>(src, dst, N, nu, dt, ty, zchunk, uvel, stream);
        case ST_F16: return launch_fused<__half>(src, dst, N, nu, dt, ty, zchunk, uvel, stream);
        case ST_BF16: return launch_fused<__nv_bfloat16>(src, dst, N, nu, dt, ty, zchunk, uvel, stream);
        case ST_F64: return launch_fused<double>(src, dst, N, nu, dt, ty, zchunk, uvel, stream);
    }
    return cudaErrorInvalidValue;
}

}  // namespace kin
