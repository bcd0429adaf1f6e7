// MRT-LBE node update (Sec. II.B, Eq. 21) in the pull arrangement, shared by
// the standalone kernels (lbe.cu) and the batched ensemble kernel.
//
// The buffer holds buf_i(y) = f_i(y + xi_i, t): the node x gathers its 19
// pre-collision populations from buf_i(x - xi_i), relaxes them in moment space
// and writes f*_i(x) back at x, so every store is coalesced and only the loads
// of populations with xi_x != 0 are shifted by one element.
#pragma once

#include "kin_common.cuh"
#include "kin_debug.cuh"

#include <cstring>

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

// 2-byte storage moves a cell's 19 values as 38 bytes, so one element per
// thread and access leaves too few bytes in flight to fill HBM.  A thread
// takes V = 4 consecutive cells (N % 4 == 0; V = 2 for other even N) and
// every load and store of its own cells is one aligned V-element vector: a
// population with xi_x = 0 reads its own vector, one pulled from x - 1
// (xi_x = +1) the element left of the vector and the vector's first V - 1,
// one pulled from x + 1 the vector's last V - 1 and the element to its right.
// Each cell's arithmetic is that of lbe_node, so the results are bitwise those
// of the one-cell form.
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

// One 2-byte value inside a packed word (hi: the upper half).
template <typename S>
struct Half1;
template <>
struct Half1<__half> {
    static __device__ __forceinline__ float get(unsigned w, bool hi) {
        return __half2float(__ushort_as_half((unsigned short)(hi ? w >> 16 : w & 0xffffu)));
    }
    static __device__ __forceinline__ unsigned put(unsigned w, bool hi, float v) {
        const unsigned b = __half_as_ushort(__float2half_rn(v));
        return hi ? (w & 0xffffu) | (b << 16) : (w & 0xffff0000u) | b;
    }
};
template <>
struct Half1<__nv_bfloat16> {
    static __device__ __forceinline__ float get(unsigned w, bool hi) {
        return __bfloat162float(__ushort_as_bfloat16((unsigned short)(hi ? w >> 16 : w & 0xffffu)));
    }
    static __device__ __forceinline__ unsigned put(unsigned w, bool hi, float v) {
        const unsigned b = __bfloat16_as_ushort(__float2bfloat16_rn(v));
        return hi ? (w & 0xffffu) | (b << 16) : (w & 0xffff0000u) | b;
    }
};

// Four consecutive cells with their populations held packed (two cells a
// word) between the loads and the stores; each cell is unpacked, relaxed and
// packed back in turn, so the thread holds 38 words and one cell's 19 floats
// instead of four cells' 76.  Same arithmetic per cell as lbe_node.
template <typename S>
__device__ __forceinline__ void lbe_vnode4p(const S* __restrict__ src, S* __restrict__ dst, int N, size_t plane,
                                            int x, int y, int z, const MrtRates<float>& rates) {
    const int xm = x == 0 ? N - 1 : x - 1;
    const int xp = x + 4 == N ? 0 : x + 4;
    const int yo[3] = {wrap_dec(y, N) * N, y * N, wrap_inc(y, N) * N};
    const int zo[3] = {wrap_dec(z, N) * N * N, z * N * N, wrap_inc(z, N) * N * N};
    unsigned w[Q][2];
    static_for<0, Q>([&](auto ic) {
        constexpr int I = decltype(ic)::value;
        const S* row = src + (size_t)I * plane + (yo[1 - cy(I)] + zo[1 - cz(I)]);
        uint2 own = make_uint2(0u, 0u);
        if (KIN_CHECK((size_t)(yo[1 - cy(I)] + zo[1 - cz(I)]) + x + 4 <= plane && xm < N && xp < N, DBG_LBE_LOAD,
                      yo[1 - cy(I)] + zo[1 - cz(I)] + x))
            own = __ldg(reinterpret_cast<const uint2*>(row + x));
        if constexpr (cx(I) == 0) {
            w[I][0] = own.x;
            w[I][1] = own.y;
        } else if constexpr (cx(I) > 0) {  // cells x - 1 .. x + 2
            const unsigned l = __ldg(reinterpret_cast<const unsigned short*>(row + xm));
            w[I][0] = __byte_perm(l, own.x, 0x5410);
            w[I][1] = __byte_perm(own.x, own.y, 0x5432);
        } else {  // cells x + 1 .. x + 4
            const unsigned r = __ldg(reinterpret_cast<const unsigned short*>(row + xp));
            w[I][0] = __byte_perm(own.x, own.y, 0x5432);
            w[I][1] = __byte_perm(own.y, r, 0x5432);
        }
    });
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        float f[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) f[i] = Half1<S>::get(w[i][k >> 1], k & 1);
        float drho, jx, jy, jz;
        mrt_collide(f, rates, drho, jx, jy, jz);
#pragma unroll
        for (int i = 0; i < Q; ++i) w[i][k >> 1] = Half1<S>::put(w[i][k >> 1], k & 1, f[i]);
    }
    const int c = x + N * (y + N * z);
    if (!KIN_CHECK((size_t)c + 4 <= plane, DBG_LBE_STORE, c)) return;
#pragma unroll
    for (int i = 0; i < Q; ++i) *reinterpret_cast<uint2*>(dst + (size_t)i * plane + c) = make_uint2(w[i][0], w[i][1]);
}

// One thread's V consecutive cells x .. x + V - 1 of row (y, z), x % V == 0.
template <typename S, int V>
__device__ __forceinline__ void lbe_vnode(const S* __restrict__ src, S* __restrict__ dst, int N, size_t plane,
                                          int x, int y, int z, const MrtRates<float>& rates) {
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


}  // namespace kin
