// Standalone launch of the MRT-LBE step (node update in lbe_node.cuh).
// HBM traffic per node: 19 loads + 19 stores of the storage type.
#include "kin_internal.h"
#include "lbe_node.cuh"

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

// 2-byte storage moves a cell's 19 values as 38 bytes, so one element per
// thread and access leaves too few bytes in flight to fill HBM.  A thread
// takes V = 4 consecutive cells (N % 4 == 0; V = 2 for other even N) and
// every load and store of its own cells is one aligned V-element vector: a
// population with xi_x = 0 reads its own vector, one pulled from x - 1
// (xi_x = +1) the element left of the vector and the vector's first V - 1,
// one pulled from x + 1 the vector's last V - 1 and the element to its right.
// Each cell's arithmetic is that of lbe_node, so the results are bitwise those
// of lbe_step_kernel.
template <typename S>
struct Pair2;
template <>
struct Pair2<__half> {
    static __device__ __forceinline__ float2 unpack(unsigned u) {
        __half2 h;
        memcpy(&h, &u, sizeof(u));
        return __half22float2(h);
    }
    static __device__ __forceinline__ unsigned pack(float a, float b) {
        const __half2 h = __floats2half2_rn(a, b);
        unsigned u;
        memcpy(&u, &h, sizeof(u));
        return u;
    }
};
template <>
struct Pair2<__nv_bfloat16> {
    static __device__ __forceinline__ float2 unpack(unsigned u) {
        __nv_bfloat162 h;
        memcpy(&h, &u, sizeof(u));
        return __bfloat1622float2(h);
    }
    static __device__ __forceinline__ unsigned pack(float a, float b) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        unsigned u;
        memcpy(&u, &h, sizeof(u));
        return u;
    }
};

// Aligned vectors of V = 2 (4 bytes) or 4 (8 bytes) 2-byte elements.
template <typename S, int V>
__device__ __forceinline__ void vload(const S* p, float (&o)[V]) {
    if constexpr (V == 2) {
        const float2 a = Pair2<S>::unpack(__ldg(reinterpret_cast<const unsigned*>(p)));
        o[0] = a.x;
        o[1] = a.y;
    } else {
        const uint2 w = __ldg(reinterpret_cast<const uint2*>(p));
        const float2 a = Pair2<S>::unpack(w.x), b = Pair2<S>::unpack(w.y);
        o[0] = a.x;
        o[1] = a.y;
        o[2] = b.x;
        o[3] = b.y;
    }
}
template <typename S, int V>
__device__ __forceinline__ void vstore(S* p, const float (&v)[V]) {
    if constexpr (V == 2) {
        *reinterpret_cast<unsigned*>(p) = Pair2<S>::pack(v[0], v[1]);
    } else {
        *reinterpret_cast<uint2*>(p) = make_uint2(Pair2<S>::pack(v[0], v[1]), Pair2<S>::pack(v[2], v[3]));
    }
}

template <typename S, int V>
__global__ void __launch_bounds__(256) lbe_stepv_kernel(const S* __restrict__ src, S* __restrict__ dst,
                                                        int N, size_t plane, MrtRates<float> rates) {
    const int x = V * (blockIdx.x * blockDim.x + threadIdx.x);
    if (x >= N) return;
    const int y = blockIdx.y, z = blockIdx.z;
    const int xm = x == 0 ? N - 1 : x - 1;  // the cell left of the vector, periodic
    const int xp = x + V == N ? 0 : x + V;  // the cell right of it
    const int yo[3] = {wrap_dec(y, N) * N, y * N, wrap_inc(y, N) * N};
    const int zo[3] = {wrap_dec(z, N) * N * N, z * N * N, wrap_inc(z, N) * N * N};
    float f[V][Q];
    static_for<0, Q>([&](auto ic) {
        constexpr int I = decltype(ic)::value;
        // row of the source cells x - xi_i (N <= 1024: row offsets fit in 32 bits)
        const S* row = src + (size_t)I * plane + (yo[1 - cy(I)] + zo[1 - cz(I)]);
        float own[V] = {};
        if (KIN_CHECK((size_t)(yo[1 - cy(I)] + zo[1 - cz(I)]) + x + V <= plane && xm < N && xp < N, DBG_LBE_LOAD,
                      yo[1 - cy(I)] + zo[1 - cz(I)] + x))
            vload<S, V>(row + x, own);
        if constexpr (cx(I) == 0) {
#pragma unroll
            for (int k = 0; k < V; ++k) f[k][I] = own[k];
        } else if constexpr (cx(I) > 0) {
            f[0][I] = Traits<S>::load(row + xm);
#pragma unroll
            for (int k = 1; k < V; ++k) f[k][I] = own[k - 1];
        } else {
#pragma unroll
            for (int k = 0; k < V - 1; ++k) f[k][I] = own[k + 1];
            f[V - 1][I] = Traits<S>::load(row + xp);
        }
    });
#pragma unroll
    for (int k = 0; k < V; ++k) {
        float drho, jx, jy, jz;
        mrt_collide(f[k], rates, drho, jx, jy, jz);
    }
    const int c = x + N * (y + N * z);
    if (!KIN_CHECK((size_t)c + V <= plane, DBG_LBE_STORE, c)) return;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        float v[V];
#pragma unroll
        for (int k = 0; k < V; ++k) v[k] = f[k][i];
        vstore<S, V>(dst + (size_t)i * plane + c, v);
    }
}

template <typename S, int V>
static cudaError_t launch_lbe_v(const S* src, S* dst, int N, const MrtRates<float>& r, int bx,
                                cudaStream_t stream) {
    const int nv = N / V;
    int b = bx > 0 ? bx : 128;
    if (b > nv) b = ((nv + 31) / 32) * 32;
    dim3 block(b), grid((nv + b - 1) / b, N, N);
    lbe_stepv_kernel<S, V><<<grid, block, 0, stream>>>(src, dst, N, (size_t)N * N * N, r);
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
