// Standalone launch of the MRT-LBE step (node update in lbe_node.cuh).
// HBM traffic per node: 19 loads + 19 stores of the storage type.
#include "kin_internal.h"
#include "lbe_node.cuh"

#include <algorithm>
#include <cstring>

namespace kin {

template <typename S>
__global__ void __launch_bounds__(256) lbe_step_kernel(const S* __restrict__ src,
                                                       S* __restrict__ dst, int N, size_t plane,
                                                       MrtRates<typename Traits<S>::C> rates) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= N) return;
    lbe_node<S, false>(src, dst, N, plane, x, blockIdx.y, blockIdx.z, rates);
}

template <typename S, int V>
__global__ void __launch_bounds__(256) lbe_stepv_kernel(const S* __restrict__ src, S* __restrict__ dst,
                                                        int N, size_t plane, MrtRates<float> rates) {
    const int x = V * (blockIdx.x * blockDim.x + threadIdx.x);
    if (x >= N) return;
    lbe_vnode<S, V>(src, dst, N, plane, x, blockIdx.y, blockIdx.z, rates);
}

// Four cells a thread with the populations held packed (lbe_vnode4p), held to
// 96 registers instead of the 128 that four cells' 76 floats take, so that
// more warps are resident: 0.222 -> 0.214 ms (FP16) at 256^3, bitwise the
// same results.
template <typename S>
__global__ void __maxnreg__(96) lbe_stepv4_kernel(const S* __restrict__ src, S* __restrict__ dst, int N,
                                                  size_t plane, MrtRates<float> rates) {
    const int x = 4 * (blockIdx.x * blockDim.x + threadIdx.x);
    if (x >= N) return;
    lbe_vnode4p<S>(src, dst, N, plane, x, blockIdx.y, blockIdx.z, rates);
}

template <typename S, int V>
static cudaError_t launch_lbe_v(const S* src, S* dst, int N, const MrtRates<float>& r, int bx,
                                cudaStream_t stream) {
    const int nv = N / V;
    int b = bx > 0 ? std::min(bx, 256) : 128;
    if (b > nv) b = ((nv + 31) / 32) * 32;
    dim3 block(b), grid((nv + b - 1) / b, N, N);
    if constexpr (V == 4) lbe_stepv4_kernel<S><<<grid, block, 0, stream>>>(src, dst, N, (size_t)N * N * N, r);
    else lbe_stepv_kernel<S, V><<<grid, block, 0, stream>>>(src, dst, N, (size_t)N * N * N, r);
    return cudaGetLastError();
}

template <typename S>
static cudaError_t launch_lbe(const void* src, void* dst, int N, double nu, int bx,
                              cudaStream_t stream) {
    using C = typename Traits<S>::C;
    const MrtRates<C> r = lbe_rates<C>(nu);
    if constexpr (sizeof(S) == 2) {
        if (N % 4 == 0) return launch_lbe_v<S, 4>((const S*)src, (S*)dst, N, r, bx, stream);
        if (N % 2 == 0) return launch_lbe_v<S, 2>((const S*)src, (S*)dst, N, r, bx, stream);
    }
    if (bx <= 0) bx = 128;
    if (bx > 256) bx = 256;  // the kernel's launch bounds
    if (bx > N) bx = ((N + 31) / 32) * 32;
    dim3 block(bx), grid((N + bx - 1) / bx, N, N);
    lbe_step_kernel<S><<<grid, block, 0, stream>>>((const S*)src, (S*)dst, N,
                                                    (size_t)N * N * N, r);
    return cudaGetLastError();
}

// One iteration of the consistent initialisation (Sec. IV.A, after Mei et
// al.): the node update of lbe_node with the momentum held at rho0 u0 (FP64,
// [3][N^3]); see mrt_collide_t.
template <typename S>
__global__ void __launch_bounds__(256) lbe_consistent_kernel(const S* __restrict__ src, S* __restrict__ dst,
                                                             int N, size_t plane,
                                                             MrtRates<typename Traits<S>::C> rates,
                                                             const double* __restrict__ u0) {
    using C = typename Traits<S>::C;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= N) return;
    const int y = blockIdx.y, z = blockIdx.z;
    C f[Q];
    lbe_gather<S, false>(src, N, plane, x, y, z, f);
    const size_t c = (size_t)x + (size_t)N * (y + (size_t)N * z);
    C drho, jx, jy, jz;
    mrt_collide_t<true>(f, rates, drho, jx, jy, jz, (C)u0[c], (C)u0[plane + c], (C)u0[2 * plane + c]);
    lbe_scatter<S>(dst, N, plane, x, y, z, f);
}

template <typename S>
static cudaError_t launch_consistent(const void* src, void* dst, int N, double nu, const double* u0,
                                     cudaStream_t stream) {
    using C = typename Traits<S>::C;
    const int bx = N >= 128 ? 128 : ((N + 31) / 32) * 32;
    dim3 block(bx), grid((N + bx - 1) / bx, N, N);
    lbe_consistent_kernel<S><<<grid, block, 0, stream>>>((const S*)src, (S*)dst, N, (size_t)N * N * N,
                                                         lbe_rates<C>(nu), u0);
    return cudaGetLastError();
}

cudaError_t lbe_consistent_step(int storage, const void* src, void* dst, int N, double nu, const double* u0,
                                cudaStream_t stream) {
    switch (storage) {
        case ST_F32: return launch_consistent<float>(src, dst, N, nu, u0, stream);
        case ST_F16: return launch_consistent<__half>(src, dst, N, nu, u0, stream);
        case ST_BF16: return launch_consistent<__nv_bfloat16>(src, dst, N, nu, u0, stream);
        case ST_F64: return launch_consistent<double>(src, dst, N, nu, u0, stream);
    }
    return cudaErrorInvalidValue;
}

KIN_DEBUG_ACCESSOR(debug_word_lbe)

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
