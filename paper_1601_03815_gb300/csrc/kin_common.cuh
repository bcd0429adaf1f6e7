// Device-side lattice definitions shared by the libkin kernels.
//
// D3Q19 (Sec. II.A, Eq. 5): population 0 is at rest, 1..6 move along the axes,
// 7..18 along the face diagonals; opposite velocities occupy slots (2p+1, 2p+2)
// for p = 0..8.  This order is part of the library's public layout (kin.h).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>
#include <utility>

namespace kin {

constexpr int Q = 19;
constexpr int NPAIR = 9;

// Velocity of the "positive" member of pair p (population 2p+1); the partner
// 2p+2 moves the opposite way.
__host__ __device__ constexpr int pair_x(int p) {
    return p == 0 ? 1 : p == 1 ? 0 : p == 2 ? 0 : p == 3 ? 1 : p == 4 ? 1 : p == 5 ? 1 : p == 6 ? 1 : 0;
}
__host__ __device__ constexpr int pair_y(int p) {
    return p == 0 ? 0 : p == 1 ? 1 : p == 2 ? 0 : p == 3 ? 1 : p == 4 ? -1 : p == 5 ? 0 : p == 6 ? 0 : 1;
}
__host__ __device__ constexpr int pair_z(int p) {
    return p == 0 ? 0 : p == 1 ? 0 : p == 2 ? 1 : p == 3 ? 0 : p == 4 ? 0 : p == 5 ? 1 : p == 6 ? -1
         : p == 7 ? 1 : -1;
}

// Velocity component a (0 = x, 1 = y, 2 = z) of population i.
__host__ __device__ constexpr int cx(int i) { return i == 0 ? 0 : ((i & 1) ? pair_x((i - 1) / 2) : -pair_x((i - 1) / 2)); }
__host__ __device__ constexpr int cy(int i) { return i == 0 ? 0 : ((i & 1) ? pair_y((i - 1) / 2) : -pair_y((i - 1) / 2)); }
__host__ __device__ constexpr int cz(int i) { return i == 0 ? 0 : ((i & 1) ? pair_z((i - 1) / 2) : -pair_z((i - 1) / 2)); }
__host__ __device__ constexpr int cc(int i, int a) { return a == 0 ? cx(i) : a == 1 ? cy(i) : cz(i); }

// Weights W_i (Sec. II.A) as exact rationals 12/36, 2/36, 1/36.
__host__ __device__ constexpr int w36(int i) { return i == 0 ? 12 : (i <= 6 ? 2 : 1); }

// ---------------------------------------------------------------------------
// Compile-time loop: calls f(std::integral_constant<int, I>) for I in [B, E).
template <int B, int E, typename F>
__device__ __forceinline__ void static_for(F&& f) {
    if constexpr (B < E) {
        f(std::integral_constant<int, B>{});
        static_for<B + 1, E>(static_cast<F&&>(f));
    }
}

// ---------------------------------------------------------------------------
// Storage types.  Arithmetic runs in Traits<S>::C.
template <typename S>
struct Traits;
template <>
struct Traits<float> {
    using C = float;
    static __device__ __forceinline__ C load(const float* p) { return __ldg(p); }
    static __device__ __forceinline__ void store(float* p, C v) { *p = v; }
    // the value a store followed by a load returns
    static __device__ __forceinline__ C rt(C v) { return v; }
    // stores the two members of a pair to p0, p1; returns what loads would return
    template <typename P>
    static __device__ __forceinline__ P store2(float* p0, float* p1, P v) {
        *p0 = v.x;
        *p1 = v.y;
        return v;
    }
};
template <>
struct Traits<double> {
    using C = double;
    static __device__ __forceinline__ C load(const double* p) { return __ldg(p); }
    static __device__ __forceinline__ void store(double* p, C v) { *p = v; }
    static __device__ __forceinline__ C rt(C v) { return v; }
    template <typename P>
    static __device__ __forceinline__ P store2(double* p0, double* p1, P v) {
        *p0 = v.x;
        *p1 = v.y;
        return v;
    }
};
template <>
struct Traits<__half> {
    using C = float;
    static __device__ __forceinline__ C load(const __half* p) { return __half2float(__ldg(p)); }
    static __device__ __forceinline__ void store(__half* p, C v) { *p = __float2half_rn(v); }
    static __device__ __forceinline__ C rt(C v) { return __half2float(__float2half_rn(v)); }
    // one paired round-to-nearest conversion, the same rounding as two single ones
    template <typename P>
    static __device__ __forceinline__ P store2(__half* p0, __half* p1, P v) {
        const __half2 h = __floats2half2_rn(v.x, v.y);
        *p0 = __low2half(h);
        *p1 = __high2half(h);
        return P{__low2float(h), __high2float(h)};
    }
};
template <>
struct Traits<__nv_bfloat16> {
    using C = float;
    static __device__ __forceinline__ C load(const __nv_bfloat16* p) {
        return __bfloat162float(__ldg(p));
    }
    static __device__ __forceinline__ void store(__nv_bfloat16* p, C v) { *p = __float2bfloat16_rn(v); }
    static __device__ __forceinline__ C rt(C v) { return __bfloat162float(__float2bfloat16_rn(v)); }
    template <typename P>
    static __device__ __forceinline__ P store2(__nv_bfloat16* p0, __nv_bfloat16* p1, P v) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(v.x, v.y);
        *p0 = __low2bfloat16(h);
        *p1 = __high2bfloat16(h);
        return P{__low2float(h), __high2float(h)};
    }
};

// ---------------------------------------------------------------------------
// Coefficient 3 W_i of the linear term of Eq. 7 for |xi_i|^2 = r2 (1 or 2).
// Exactly, 2 (3 W_1) + 8 (3 W_7) = 1 makes sum_i xi_i f_eq_i = rho0 u.  In FP32
// the rounded values fl(1/6), fl(1/12) sum to 1 + 3e-8, which a DUGKS step
// multiplies into the momentum every step (f-bar-plus = f + b (f_eq - f));
// so FP32 uses fl(1/12) and the FP32 value 5592405 * 2^-25 for which the sum
// is exactly 1.  FP64 keeps 1/6 and 1/12.
template <typename C>
__host__ __device__ constexpr C lin3w(int r2) {
    if constexpr (sizeof(C) == 4) return r2 == 1 ? C(5592405.0 / 33554432.0) : C(11184811.0 / 134217728.0);
    else return r2 == 1 ? C(1.0 / 6.0) : C(1.0 / 12.0);
}

// Discrete equilibrium of Eq. 7 with rho0 = 1, RT = 1/3:
//   f_eq_i = W_i [drho + 9/2 (xi.u)^2 - 3/2 |u|^2] + 3 W_i xi.u.
template <int I, typename C>
__device__ __forceinline__ C feq_i(C drho, C ux, C uy, C uz, C usq15) {
    constexpr int X = cx(I), Y = cy(I), Z = cz(I);
    C xu = C(0);
    if constexpr (X != 0) xu += C(X) * ux;
    if constexpr (Y != 0) xu += C(Y) * uy;
    if constexpr (Z != 0) xu += C(Z) * uz;
    const C w = C(w36(I)) / C(36);
    if constexpr (I == 0) return w * (drho - usq15);
    else return w * (drho + C(4.5) * xu * xu - usq15) + lin3w<C>(X * X + Y * Y + Z * Z) * xu;
}

// delta-rho = sum f, rho0 u = sum xi f (Eq. 8), rho0 = 1.
template <typename C>
__device__ __forceinline__ void moments(const C (&f)[Q], C& drho, C& jx, C& jy, C& jz) {
    C a[NPAIR], b[NPAIR];
#pragma unroll
    for (int p = 0; p < NPAIR; ++p) {
        a[p] = f[2 * p + 1] + f[2 * p + 2];
        b[p] = f[2 * p + 1] - f[2 * p + 2];
    }
    drho = f[0] + ((a[0] + a[1]) + a[2]) + (((a[3] + a[4]) + (a[5] + a[6])) + (a[7] + a[8]));
    jx = (b[0] + b[3]) + (b[4] + (b[5] + b[6]));
    jy = (b[1] + b[3]) - (b[4] - (b[7] + b[8]));
    jz = (b[2] + b[5]) - (b[6] - (b[7] - b[8]));
}

// ---------------------------------------------------------------------------
// MRT moment rows of Sec. II.B as integer polynomials of the velocity.
__host__ __device__ constexpr int mrow(int k, int x, int y, int z) {
    const int r2 = x * x + y * y + z * z;
    switch (k) {
        case 0: return 1;
        case 1: return 19 * r2 - 30;
        case 2: return (21 * r2 * r2 - 53 * r2 + 24) / 2;
        case 3: return x;
        case 4: return (5 * r2 - 9) * x;
        case 5: return y;
        case 6: return (5 * r2 - 9) * y;
        case 7: return z;
        case 8: return (5 * r2 - 9) * z;
        case 9: return 3 * x * x - r2;
        case 10: return (3 * r2 - 5) * (3 * x * x - r2);
        case 11: return y * y - z * z;
        case 12: return (3 * r2 - 5) * (y * y - z * z);
        case 13: return x * y;
        case 14: return y * z;
        case 15: return x * z;
        case 16: return (y * y - z * z) * x;
        case 17: return (z * z - x * x) * y;
        default: return (x * x - y * y) * z;
    }
}
// Squared norm of row k over the 19 velocities.
__host__ __device__ constexpr int mnorm(int k) {
    int s = 0;
    for (int i = 0; i < Q; ++i) {
        int v = mrow(k, cx(i), cy(i), cz(i));
        s += v * v;
    }
    return s;
}
// Non-conserved rows whose polynomial is even / odd in xi.
__host__ __device__ constexpr int even_row(int j) {
    return j == 0 ? 1 : j == 1 ? 2 : j == 2 ? 9 : j == 3 ? 10 : j == 4 ? 11 : j == 5 ? 12 : j == 6 ? 13
         : j == 7 ? 14 : 15;
}
__host__ __device__ constexpr int odd_row(int j) {
    return j == 0 ? 4 : j == 1 ? 6 : j == 2 ? 8 : j == 3 ? 16 : j == 4 ? 17 : 18;
}
constexpr int NEVEN = 9;
constexpr int NODD = 6;

// Relaxation rates (Sec. II.B, values of Sec. IV.A).
template <typename C>
struct MrtRates {
    C s1, s2, s4, s9, s10, s13, s16;
};
template <int K, typename C>
__device__ __forceinline__ C rate(const MrtRates<C>& r) {
    if constexpr (K == 1) return r.s1;
    else if constexpr (K == 2) return r.s2;
    else if constexpr (K == 4 || K == 6 || K == 8) return r.s4;
    else if constexpr (K == 9 || K == 11) return r.s9;
    else if constexpr (K == 10 || K == 12) return r.s10;
    else if constexpr (K == 13 || K == 14 || K == 15) return r.s13;
    else return r.s16;
}

// Equilibrium moments (Sec. II.B with omega_eps = omega_xx = 0,
// omega_epsj = -475/63, rho0 = 1).  Slot 9 holds 3 p_xx.
template <int K, typename C>
__device__ __forceinline__ C meq(C drho, C jx, C jy, C jz, C jj) {
    if constexpr (K == 1) return C(-11) * drho + C(19) * jj;
    else if constexpr (K == 2) return C(-475.0 / 63.0) * jj;
    else if constexpr (K == 4) return C(-2.0 / 3.0) * jx;
    else if constexpr (K == 6) return C(-2.0 / 3.0) * jy;
    else if constexpr (K == 8) return C(-2.0 / 3.0) * jz;
    else if constexpr (K == 9) return C(2) * jx * jx - (jy * jy + jz * jz);
    else if constexpr (K == 11) return jy * jy - jz * jz;
    else if constexpr (K == 13) return jx * jy;
    else if constexpr (K == 14) return jy * jz;
    else if constexpr (K == 15) return jx * jz;
    else return C(0);  // rows 10, 12 (omega_xx = 0) and 16-18
}

// One MRT collision in place (RHS of Eq. 21): f <- f - M^-1 S (M f - m_eq).
// M is orthogonal, so M^-1 = M^T diag(1/|M_k|^2); rows are even or odd in xi,
// so the work splits into the pair sums a_p = f_{2p+1} + f_{2p+2} (even rows)
// and differences b_p = f_{2p+1} - f_{2p+2} (odd rows).
// FIXJ: the equilibrium takes the prescribed momentum (jfx, jfy, jfz) and the
// momentum rows relax fully to it (the consistent initialisation, Sec. IV.A);
// otherwise the cell's own momentum, conserved.
template <bool FIXJ, typename C>
__device__ __forceinline__ void mrt_collide_t(C (&f)[Q], const MrtRates<C>& r, C& drho_out, C& jx_out,
                                              C& jy_out, C& jz_out, C jfx, C jfy, C jfz) {
    C a[NPAIR], b[NPAIR];
#pragma unroll
    for (int p = 0; p < NPAIR; ++p) {
        a[p] = f[2 * p + 1] + f[2 * p + 2];
        b[p] = f[2 * p + 1] - f[2 * p + 2];
    }
    const C f0 = f[0];
    const C drho = f0 + ((a[0] + a[1]) + a[2]) + (((a[3] + a[4]) + (a[5] + a[6])) + (a[7] + a[8]));
    const C jx = (b[0] + b[3]) + (b[4] + (b[5] + b[6]));
    const C jy = (b[1] + b[3]) - (b[4] - (b[7] + b[8]));
    const C jz = (b[2] + b[5]) - (b[6] - (b[7] - b[8]));
    drho_out = drho;
    jx_out = jx;
    jy_out = jy;
    jz_out = jz;
    const C jxe = FIXJ ? jfx : jx, jye = FIXJ ? jfy : jy, jze = FIXJ ? jfz : jz;
    const C jj = jxe * jxe + jye * jye + jze * jze;
    // FIXJ: (m - m_eq) / |M_k|^2 of the momentum rows at rate 1 (|M_3|^2 = 10)
    [[maybe_unused]] const C gjx = (jx - jfx) * C(0.1), gjy = (jy - jfy) * C(0.1), gjz = (jz - jfz) * C(0.1);

    C ge[NEVEN], go[NODD];
    static_for<0, NEVEN>([&](auto jc) {
        constexpr int J = decltype(jc)::value;
        constexpr int K = even_row(J);
        C m = C(mrow(K, 0, 0, 0)) * f0;
        static_for<0, NPAIR>([&](auto pc) {
            constexpr int P = decltype(pc)::value;
            constexpr int c = mrow(K, pair_x(P), pair_y(P), pair_z(P));
            if constexpr (c == 1) m += a[P];
            else if constexpr (c == -1) m -= a[P];
            else if constexpr (c != 0) m += C(c) * a[P];
        });
        ge[J] = rate<K>(r) * (m - meq<K>(drho, jxe, jye, jze, jj)) * (C(1) / C(mnorm(K)));
    });
    static_for<0, NODD>([&](auto jc) {
        constexpr int J = decltype(jc)::value;
        constexpr int K = odd_row(J);
        C m = C(0);
        static_for<0, NPAIR>([&](auto pc) {
            constexpr int P = decltype(pc)::value;
            constexpr int c = mrow(K, pair_x(P), pair_y(P), pair_z(P));
            if constexpr (c == 1) m += b[P];
            else if constexpr (c == -1) m -= b[P];
            else if constexpr (c != 0) m += C(c) * b[P];
        });
        go[J] = rate<K>(r) * (m - meq<K>(drho, jxe, jye, jze, jj)) * (C(1) / C(mnorm(K)));
    });
    // back transform: df_i = sum_k M_k,i g_k
    {
        C d0 = C(0);
        static_for<0, NEVEN>([&](auto jc) {
            constexpr int J = decltype(jc)::value;
            constexpr int c = mrow(even_row(J), 0, 0, 0);
            if constexpr (c != 0) d0 += C(c) * ge[J];
        });
        f[0] = f0 - d0;
    }
    static_for<0, NPAIR>([&](auto pc) {
        constexpr int P = decltype(pc)::value;
        C e = C(0), o = C(0);
        static_for<0, NEVEN>([&](auto jc) {
            constexpr int J = decltype(jc)::value;
            constexpr int c = mrow(even_row(J), pair_x(P), pair_y(P), pair_z(P));
            if constexpr (c == 1) e += ge[J];
            else if constexpr (c == -1) e -= ge[J];
            else if constexpr (c != 0) e += C(c) * ge[J];
        });
        static_for<0, NODD>([&](auto jc) {
            constexpr int J = decltype(jc)::value;
            constexpr int c = mrow(odd_row(J), pair_x(P), pair_y(P), pair_z(P));
            if constexpr (c == 1) o += go[J];
            else if constexpr (c == -1) o -= go[J];
            else if constexpr (c != 0) o += C(c) * go[J];
        });
        if constexpr (FIXJ) {
            // the momentum rows (M_3,5,7 = xi_x, xi_y, xi_z) relaxed with rate 1
            if constexpr (pair_x(P) != 0) o += C(pair_x(P)) * gjx;
            if constexpr (pair_y(P) != 0) o += C(pair_y(P)) * gjy;
            if constexpr (pair_z(P) != 0) o += C(pair_z(P)) * gjz;
        }
        f[2 * P + 1] -= e + o;
        f[2 * P + 2] -= e - o;
    });
}

template <typename C>
__device__ __forceinline__ void mrt_collide(C (&f)[Q], const MrtRates<C>& r, C& drho_out, C& jx_out,
                                            C& jy_out, C& jz_out) {
    mrt_collide_t<false>(f, r, drho_out, jx_out, jy_out, jz_out, C(0), C(0), C(0));
}

// Periodic neighbour of coordinate v in [0, n).
__device__ __forceinline__ int wrap_inc(int v, int n) { return v + 1 == n ? 0 : v + 1; }
__device__ __forceinline__ int wrap_dec(int v, int n) { return v == 0 ? n - 1 : v - 1; }

}  // namespace kin
