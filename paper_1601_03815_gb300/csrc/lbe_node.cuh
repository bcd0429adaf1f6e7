// MRT-LBE node update (Sec. II.B, Eq. 21) in the pull arrangement, shared by
// the standalone kernel (lbe.cu) and the persistent ensemble kernel.
//
// The buffer holds buf_i(y) = f_i(y + xi_i, t): the node x gathers its 19
// pre-collision populations from buf_i(x - xi_i), relaxes them in moment space
// and writes f*_i(x) back at x, so every store is coalesced and only the loads
// of populations with xi_x != 0 are shifted by one element.
#pragma once

#include "kin_common.cuh"
#include "kin_debug.cuh"

namespace kin {

// Sec. IV.A rates with dt = dx = 1.
template <typename C>
inline MrtRates<C> lbe_rates(double nu) {
    MrtRates<C> r;
    r.s1 = C(1.19);
    r.s2 = C(1.4);
    r.s4 = C(1.2);
    r.s9 = C(1.0 / (3.0 * nu + 0.5));
    r.s10 = C(1.4);
    r.s13 = r.s9;
    r.s16 = C(1.98);
    return r;
}

// COHERENT selects plain loads (data written earlier in the same launch by
// other thread blocks, read after an acquire) instead of the read-only path.
template <typename S, bool COHERENT>
__device__ __forceinline__ void lbe_gather(const S* __restrict__ src, int N, size_t plane, int x, int y,
                                           int z, typename Traits<S>::C (&f)[Q]) {
    using C = typename Traits<S>::C;
    const int xo[3] = {wrap_dec(x, N), x, wrap_inc(x, N)};
    const int yo[3] = {wrap_dec(y, N) * N, y * N, wrap_inc(y, N) * N};
    const int zo[3] = {wrap_dec(z, N) * N * N, z * N * N, wrap_inc(z, N) * N * N};
    // source of population i is x - xi_i: offset index 1 - xi
    static_for<0, Q>([&](auto ic) {
        constexpr int I = decltype(ic)::value;
        const int idx = xo[1 - cx(I)] + yo[1 - cy(I)] + zo[1 - cz(I)];
        if (!KIN_CHECK(idx >= 0 && (size_t)idx < plane, DBG_LBE_LOAD, idx)) f[I] = C(0);
        else if constexpr (COHERENT) f[I] = (C)src[(size_t)I * plane + idx];
        else f[I] = Traits<S>::load(src + (size_t)I * plane + idx);
    });
}

template <typename S>
__device__ __forceinline__ void lbe_scatter(S* __restrict__ dst, int N, size_t plane, int x, int y, int z,
                                            const typename Traits<S>::C (&f)[Q]) {
    const int c = x + N * (y + N * z);  // N <= 1024
    if (!KIN_CHECK(c >= 0 && (size_t)c < plane, DBG_LBE_STORE, c)) return;
#pragma unroll
    for (int i = 0; i < Q; ++i) Traits<S>::store(dst + (size_t)i * plane + c, f[i]);
}

template <typename S, bool COHERENT>
__device__ __forceinline__ void lbe_node(const S* __restrict__ src, S* __restrict__ dst, int N,
                                         size_t plane, int x, int y, int z,
                                         const MrtRates<typename Traits<S>::C>& rates) {
    using C = typename Traits<S>::C;
    C f[Q];
    lbe_gather<S, COHERENT>(src, N, plane, x, y, z, f);
    C drho, jx, jy, jz;
    mrt_collide(f, rates, drho, jx, jy, jz);
    lbe_scatter<S>(dst, N, plane, x, y, z, f);
}

// K nodes (cells c[0..K-1], linear index x + N (y + N z)) with every gather
// issued before the first collision, so that a thread keeps K times the loads
// in flight (used where few warps share an SM).
template <int K, typename S, bool COHERENT>
__device__ __forceinline__ void lbe_nodes(const S* __restrict__ src, S* __restrict__ dst, int N,
                                          size_t plane, const int (&c)[K],
                                          const MrtRates<typename Traits<S>::C>& rates) {
    using C = typename Traits<S>::C;
    C f[K][Q];
    int xyz[K][3];
    const int nn = N * N;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        xyz[k][2] = c[k] / nn;
        xyz[k][1] = (c[k] - xyz[k][2] * nn) / N;
        xyz[k][0] = c[k] - xyz[k][2] * nn - xyz[k][1] * N;
        lbe_gather<S, COHERENT>(src, N, plane, xyz[k][0], xyz[k][1], xyz[k][2], f[k]);
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
        C drho, jx, jy, jz;
        mrt_collide(f[k], rates, drho, jx, jy, jz);
    }
#pragma unroll
    for (int k = 0; k < K; ++k) lbe_scatter<S>(dst, N, plane, xyz[k][0], xyz[k][1], xyz[k][2], f[k]);
}

}  // namespace kin
