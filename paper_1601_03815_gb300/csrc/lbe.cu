// Standalone launch of the MRT-LBE step (node update in lbe_node.cuh).
// HBM traffic per node: 19 loads + 19 stores of the storage type.
#include "kin_internal.h"
#include "lbe_node.cuh"

namespace kin {

template <typename S>
__global__ void __launch_bounds__(256) lbe_step_kernel(const S* __restrict__ src,
                                                       S* __restrict__ dst, int N, size_t plane,
                                                       MrtRates<typename Traits<S>::C> rates) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= N) return;
    lbe_node<S, false>(src, dst, N, plane, x, blockIdx.y, blockIdx.z, rates);
}

template <typename S>
static cudaError_t launch_lbe(const void* src, void* dst, int N, double nu, int bx,
                              cudaStream_t stream) {
    using C = typename Traits<S>::C;
    const MrtRates<C> r = lbe_rates<C>(nu);
    if (bx <= 0) bx = 128;
    if (bx > N) bx = ((N + 31) / 32) * 32;
    dim3 block(bx), grid((N + bx - 1) / bx, N, N);
    lbe_step_kernel<S><<<grid, block, 0, stream>>>((const S*)src, (S*)dst, N,
                                                    (size_t)N * N * N, r);
    return cudaGetLastError();
}

cudaError_t lbe_step(int storage, const void* src, void* dst, int N, double nu, int block_x,
                     cudaStream_t stream) {
    switch (storage) {
        case ST_F32: return launch_lbe<float>(src, dst, N, nu, block_x, stream);
        case ST_F16: return launch_lbe<__half>(src, dst, N, nu, block_x, stream);
        case ST_BF16: return launch_lbe<__nv_bfloat16>(src, dst, N, nu, block_x, stream);
        case ST_F64: return launch_lbe<double>(src, dst, N, nu, block_x, stream);
    }
    return cudaErrorInvalidValue;
}

}  // namespace kin
