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

// 2-byte storage moves a cell's 19 values as 38 bytes, so one element per
// thread and access leaves too few bytes in flight to fill HBM.  With N even,
// a thread takes the cells x = 2t and 2t + 1 and every load and store is an
// aligned 4-byte pair: populations with xi_x = 0 read their own pair; a
// population pulled from x - 1 (xi_x = +1) takes (x - 1, x) from the pair to
// the left and its own, one pulled from x + 1 its own and the pair to the
// right.  Each cell's arithmetic is that of lbe_node, so the results are
// bitwise those of lbe_step_kernel.
template <typename S>
struct Pair2;
template <>
struct Pair2<__half> {
    static __device__ __forceinline__ float2 load(const __half* p) {
        return __half22float2(__ldg(reinterpret_cast<const __half2*>(p)));
    }
    static __device__ __forceinline__ void store(__half* p, float a, float b) {
        *reinterpret_cast<__half2*>(p) = __floats2half2_rn(a, b);
    }
};
template <>
struct Pair2<__nv_bfloat16> {
    static __device__ __forceinline__ float2 load(const __nv_bfloat16* p) {
        return __bfloat1622float2(__ldg(reinterpret_cast<const __nv_bfloat162*>(p)));
    }
    static __device__ __forceinline__ void store(__nv_bfloat16* p, float a, float b) {
        *reinterpret_cast<__nv_bfloat162*>(p) = __floats2bfloat162_rn(a, b);
    }
};

template <typename S>
__global__ void __launch_bounds__(256) lbe_step2_kernel(const S* __restrict__ src, S* __restrict__ dst,
                                                        int N, size_t plane, MrtRates<float> rates) {
    const int x = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    if (x >= N) return;
    const int y = blockIdx.y, z = blockIdx.z;
    const int xl = x == 0 ? N - 2 : x - 2;  // the pair to the left, periodic
    const int xr = x + 2 == N ? 0 : x + 2;  // the pair to the right
    const int yo[3] = {wrap_dec(y, N) * N, y * N, wrap_inc(y, N) * N};
    const int zo[3] = {wrap_dec(z, N) * N * N, z * N * N, wrap_inc(z, N) * N * N};
    float fa[Q], fb[Q];
    static_for<0, Q>([&](auto ic) {
        constexpr int I = decltype(ic)::value;
        // row of the source cells x - xi_i (N <= 1024: row offsets fit in 32 bits)
        const S* row = src + (size_t)I * plane + (yo[1 - cy(I)] + zo[1 - cz(I)]);
        const float2 own = Pair2<S>::load(row + x);
        if constexpr (cx(I) == 0) {
            fa[I] = own.x;
            fb[I] = own.y;
        } else if constexpr (cx(I) > 0) {
            fa[I] = Pair2<S>::load(row + xl).y;
            fb[I] = own.x;
        } else {
            fa[I] = own.y;
            fb[I] = Pair2<S>::load(row + xr).x;
        }
    });
    float drho, jx, jy, jz;
    mrt_collide(fa, rates, drho, jx, jy, jz);
    mrt_collide(fb, rates, drho, jx, jy, jz);
    const int c = x + N * (y + N * z);
#pragma unroll
    for (int i = 0; i < Q; ++i) Pair2<S>::store(dst + (size_t)i * plane + c, fa[i], fb[i]);
}

template <typename S>
static cudaError_t launch_lbe(const void* src, void* dst, int N, double nu, int bx,
                              cudaStream_t stream) {
    using C = typename Traits<S>::C;
    const MrtRates<C> r = lbe_rates<C>(nu);
    if constexpr (sizeof(S) == 2) {
        if (N % 2 == 0) {
            const int half = N / 2;
            int b2 = bx > 0 ? bx : 128;
            if (b2 > half) b2 = ((half + 31) / 32) * 32;
            dim3 block(b2), grid((half + b2 - 1) / b2, N, N);
            lbe_step2_kernel<S><<<grid, block, 0, stream>>>((const S*)src, (S*)dst, N, (size_t)N * N * N, r);
            return cudaGetLastError();
        }
    }
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
