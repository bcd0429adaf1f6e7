// MRT-LBE time step for D3Q19 (Sec. II.B, Eq. 21), pull arrangement.
//
// The buffer holds buf_i(y) = f_i(y + xi_i, t): each thread gathers the 19
// pre-collision populations of its node x from buf_i(x - xi_i), relaxes them in
// moment space and writes f*_i(x) back at x, so every store is coalesced and
// only the loads of populations with xi_x != 0 are shifted by one element.
// HBM traffic per node: 19 loads + 19 stores of the storage type.
#include "kin_common.cuh"
#include "kin_internal.h"

namespace kin {

template <typename S>
__global__ void __launch_bounds__(256) lbe_step_kernel(const S* __restrict__ src,
                                                       S* __restrict__ dst, int N, size_t plane,
                                                       MrtRates<typename Traits<S>::C> rates) {
    using C = typename Traits<S>::C;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= N) return;
    const int y = blockIdx.y, z = blockIdx.z;
    const int xo[3] = {wrap_dec(x, N), x, wrap_inc(x, N)};
    const int yo[3] = {wrap_dec(y, N) * N, y * N, wrap_inc(y, N) * N};
    const int zo[3] = {wrap_dec(z, N) * N * N, z * N * N, wrap_inc(z, N) * N * N};

    C f[Q];
    // source of population i is x - xi_i: offset index 1 - xi
    static_for<0, Q>([&](auto ic) {
        constexpr int I = decltype(ic)::value;
        const int idx = xo[1 - cx(I)] + yo[1 - cy(I)] + zo[1 - cz(I)];
        f[I] = Traits<S>::load(src + (size_t)I * plane + idx);
    });
    C drho, jx, jy, jz;
    mrt_collide(f, rates, drho, jx, jy, jz);
    const int c = x + yo[1] + zo[1];
#pragma unroll
    for (int i = 0; i < Q; ++i) Traits<S>::store(dst + (size_t)i * plane + c, f[i]);
}

template <typename S>
static cudaError_t launch_lbe(const void* src, void* dst, int N, double nu, int bx,
                              cudaStream_t stream) {
    using C = typename Traits<S>::C;
    MrtRates<C> r;
    // Sec. IV.A with dt = dx = 1
    r.s1 = C(1.19);
    r.s2 = C(1.4);
    r.s4 = C(1.2);
    r.s9 = C(1.0 / (3.0 * nu + 0.5));
    r.s10 = C(1.4);
    r.s13 = r.s9;
    r.s16 = C(1.98);
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
