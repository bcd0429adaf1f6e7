// Standalone launch of the fused DUGKS step (tile code in dugks_tile.cuh).
#include <atomic>

#include "dugks_tile.cuh"
#include "kin_internal.h"

namespace kin {

// VEL: also write the velocity of the new state to uvel (FP32-computed storage).
template <typename S, int TY, bool VEL>
__global__ void __launch_bounds__(32 * (TY + 2), 1)
    dugks_fused_kernel(const S* __restrict__ src, S* __restrict__ dst, int N, int zchunk,
                       DugksCoef<typename Traits<S>::C> kc, float* __restrict__ uvel) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    dugks_tile<S, TY, false, VEL>(src, dst, N, blockIdx.x, blockIdx.y, blockIdx.z, zchunk, kc, smem_raw,
                                  nullptr, nullptr, uvel);
}

template <typename S, int TY, bool VEL>
static cudaError_t launch_fused_t(const void* src, void* dst, int N, int zchunk,
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
        e = cudaFuncSetAttribute(dugks_fused_kernel<S, TY, VEL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
        if (e != cudaSuccess) return e;
        configured.fetch_or(bit);
    }
    if (zchunk <= 0) zchunk = 32;
    if (zchunk > N) zchunk = N;
    dim3 block(32, TY + 2);
    dim3 grid((N + 29) / 30, (N + TY - 1) / TY, (N + zchunk - 1) / zchunk);
    dugks_fused_kernel<S, TY, VEL><<<grid, block, smem, stream>>>((const S*)src, (S*)dst, N, zchunk, k, uvel);
    return cudaGetLastError();
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

// TMA-staged FP32 form (N a multiple of 4).
template <int TY>
__global__ void __launch_bounds__(32 * (TY + 2), 1)
    dugks_fused_tma_kernel(const __grid_constant__ CUtensorMap tmap, const float* __restrict__ src,
                           float* __restrict__ dst, int N, int zchunk, DugksCoef<float> kc, int* err) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    dugks_tile<float, TY, true>(src, dst, N, blockIdx.x, blockIdx.y, blockIdx.z, zchunk, kc, smem_raw, &tmap,
                                err);
}

template <int TY>
static cudaError_t launch_tma_t(const CUtensorMap& tmap, const float* src, float* dst, int N, int zchunk,
                                const DugksCoef<float>& k, int* err, cudaStream_t stream) {
    const size_t smem = fused_smem_bytes_v<float, TY, true>();
    static std::atomic<unsigned long long> configured{0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = dev < 64 ? 1ull << dev : 0ull;
    if (!bit || !(configured.load() & bit)) {
        e = cudaFuncSetAttribute(dugks_fused_tma_kernel<TY>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured.fetch_or(bit);
    }
    if (zchunk <= 0) zchunk = 32;
    if (zchunk > N) zchunk = N;
    dim3 block(32, TY + 2);
    dim3 grid((N + 29) / 30, (N + TY - 1) / TY, (N + zchunk - 1) / zchunk);
    dugks_fused_tma_kernel<TY><<<grid, block, smem, stream>>>(tmap, src, dst, N, zchunk, k, err);
    return cudaGetLastError();
}

cudaError_t dugks_step_fused_tma(const void* tmap, const void* src, void* dst, int N, double nu, double dt,
                                 int ty, int zchunk, int* err, cudaStream_t stream) {
    const DugksCoef<float> k = dugks_coef<float>(nu, dt);
    const CUtensorMap& m = *reinterpret_cast<const CUtensorMap*>(tmap);
    if (ty == 4) return launch_tma_t<4>(m, (const float*)src, (float*)dst, N, zchunk, k, err, stream);
    return launch_tma_t<8>(m, (const float*)src, (float*)dst, N, zchunk, k, err, stream);
}

// Tensor map of an FP32 state f[19][N][N][N] for the TMA staging of a tile of
// TY rows: dimensions (x, y, z, population), box TMA_W x (TY + 2) x 1 x 19.
cudaError_t dugks_make_tmap(void* tmap, const void* base, int N, int ty) {
    using Encode = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    static Encode encode = nullptr;
    if (!encode) {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
        encode = (Encode)fn;
    }
    if (N % 4 != 0) return cudaErrorInvalidValue;
    const cuuint64_t n = (cuuint64_t)N;
    const cuuint64_t dims[4] = {n, n, n, (cuuint64_t)Q};
    const cuuint64_t strides[3] = {n * 4, n * n * 4, n * n * n * 4};  // bytes, dimensions 1..3
    const cuuint32_t box[4] = {(cuuint32_t)TMA_W, (cuuint32_t)(ty + 2), 1, (cuuint32_t)Q};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    const CUresult r = encode((CUtensorMap*)tmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<void*>(base), dims,
                              strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

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
