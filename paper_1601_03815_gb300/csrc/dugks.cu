// DUGKS time step for D3Q19 (Sec. II.A, Eqs. 9-20).
//
// Two launches per step:
//   dugks_prestep_kernel: f-tilde -> f-bar-plus (Eq. 19) into a scratch buffer
//   dugks_flux_kernel:    per cell, the six interface fluxes (Eqs. 13-18, 10)
//                         and the update f-tilde^{n+1} = f-tilde-plus - dt sum F
//                         (Eqs. 9, 20)
#include "dugks_face.cuh"
#include "kin_internal.h"

namespace kin {

template <typename C>
static DugksCoef<C> make_coef(double nu, double dt) {
    const double tau = 3.0 * nu;  // nu = tau RT, RT = 1/3
    const double h = 0.5 * dt;
    DugksCoef<C> k{};
    k.a = C((2.0 * tau - h) / (2.0 * tau + dt));
    k.b = C(3.0 * h / (2.0 * tau + dt));
    k.h = C(h);
    k.c1 = C(2.0 * tau / (2.0 * tau + h));
    k.c2 = C(h / (2.0 * tau + h));
    k.dt = C(dt);
    return k;
}

template <typename S>
__global__ void __launch_bounds__(256)
    dugks_prestep_kernel(const S* __restrict__ src, typename Traits<S>::C* __restrict__ fbp, int N,
                         size_t plane, DugksCoef<typename Traits<S>::C> k) {
    using C = typename Traits<S>::C;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= N) return;
    const size_t c = (size_t)x + (size_t)N * (blockIdx.y + (size_t)N * blockIdx.z);
    C f[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) f[i] = Traits<S>::load(src + i * plane + c);
    C drho, jx, jy, jz;
    moments(f, drho, jx, jy, jz);
    const C usq15 = C(1.5) * (jx * jx + jy * jy + jz * jz);
    static_for<0, Q>([&](auto ic) {
        constexpr int I = decltype(ic)::value;
        // Eq. 19 with a + b = 1 written so a fixed point stays exact in any precision
        fbp[I * plane + c] = f[I] + k.b * (feq_i<I>(drho, jx, jy, jz, usq15) - f[I]);
    });
}

template <typename S>
__global__ void __launch_bounds__(128)
    dugks_flux_kernel(const S* __restrict__ src, const typename Traits<S>::C* __restrict__ fbp,
                      S* __restrict__ dst, int N, size_t plane,
                      DugksCoef<typename Traits<S>::C> k) {
    using C = typename Traits<S>::C;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= N) return;
    const int y = blockIdx.y, z = blockIdx.z;
    const int c = x + N * (y + N * z);

    C G[Q];  // net outward flux sum per population
#pragma unroll
    for (int i = 0; i < Q; ++i) G[i] = C(0);

    // f-bar-plus at (x0 + dx, y0 + dy, z0 + dz), periodic, with |d| <= 2
    auto at = [&](int i, int px, int py, int pz) -> C {
        px = px < 0 ? px + N : (px >= N ? px - N : px);
        py = py < 0 ? py + N : (py >= N ? py - N : py);
        pz = pz < 0 ? pz + N : (pz >= N ? pz - N : pz);
        return __ldg(fbp + (size_t)i * plane + (px + N * (py + N * pz)));
    };
    static_for<0, 3>([&](auto ac) {
        constexpr int A = decltype(ac)::value;
        constexpr int AX = A == 0, AY = A == 1, AZ = A == 2;
        C Fp[Q], Fm[Q];
        // face at x + e_A/2 (L = this cell) and at x - e_A/2 (L = x - e_A)
        face_flux<A>([&](int i, int dx, int dy, int dz) { return at(i, x + dx, y + dy, z + dz); }, k,
                     Fp);
        face_flux<A>(
            [&](int i, int dx, int dy, int dz) {
                return at(i, x - AX + dx, y - AY + dy, z - AZ + dz);
            },
            k, Fm);
        static_for<0, Q>([&](auto ic) {
            constexpr int I = decltype(ic)::value;
            if constexpr (cc(I, A) != 0) G[I] += Fp[I] - Fm[I];
        });
    });
    // Eq. 20: f-tilde-plus = 4/3 fbp - 1/3 f-tilde; Eq. 9 with |V| = 1
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const C ft = Traits<S>::load(src + (size_t)i * plane + c);
        const C fb = fbp[(size_t)i * plane + c];
        const C ftp = fb + (fb - ft) * C(1.0 / 3.0);  // Eq. 20: 4/3 fbp - 1/3 ft
        Traits<S>::store(dst + (size_t)i * plane + c, ftp - k.dt * G[i]);
    }
}

template <typename S>
static cudaError_t launch_dugks(const void* src, void* dst, void* fbp, int N, double nu, double dt,
                                int bx, cudaStream_t stream) {
    using C = typename Traits<S>::C;
    const DugksCoef<C> k = make_coef<C>(nu, dt);
    const size_t plane = (size_t)N * N * N;
    int b1 = 128;
    if (b1 > N) b1 = ((N + 31) / 32) * 32;
    dim3 g1((N + b1 - 1) / b1, N, N);
    dugks_prestep_kernel<S><<<g1, b1, 0, stream>>>((const S*)src, (C*)fbp, N, plane, k);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (bx <= 0) bx = 128;
    if (bx > N) bx = ((N + 31) / 32) * 32;
    if (bx > 128) bx = 128;
    dim3 g2((N + bx - 1) / bx, N, N);
    dugks_flux_kernel<S><<<g2, bx, 0, stream>>>((const S*)src, (const C*)fbp, (S*)dst, N, plane, k);
    return cudaGetLastError();
}

size_t dugks_scratch_bytes(int storage) { return storage == ST_F64 ? 8 : 4; }

cudaError_t dugks_step(int storage, const void* src, void* dst, void* fbp, int N, double nu,
                       double dt, int block_x, cudaStream_t stream) {
    switch (storage) {
        case ST_F32: return launch_dugks<float>(src, dst, fbp, N, nu, dt, block_x, stream);
        case ST_F16: return launch_dugks<__half>(src, dst, fbp, N, nu, dt, block_x, stream);
        case ST_BF16: return launch_dugks<__nv_bfloat16>(src, dst, fbp, N, nu, dt, block_x, stream);
        case ST_F64: return launch_dugks<double>(src, dst, fbp, N, nu, dt, block_x, stream);
    }
    return cudaErrorInvalidValue;
}

// The momentum reset of one iteration of the consistent initialisation for
// DUGKS (Sec. IV.A, after Mei et al.): after a plain DUGKS step the momentum of
// f-tilde returns to rho0 u0 along the linear term of the equilibrium (Eq. 7),
// f_i += 3 W_i xi_i . rho0 (u0 - u), in place; the mass and the second
// moment are unchanged.
template <typename S>
__global__ void __launch_bounds__(256)
    dugks_reset_momentum_kernel(S* __restrict__ f, int N, size_t plane, const double* __restrict__ u0) {
    using C = typename Traits<S>::C;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= N) return;
    const size_t c = (size_t)x + (size_t)N * (blockIdx.y + (size_t)N * blockIdx.z);
    C v[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) v[i] = Traits<S>::load(f + i * plane + c);
    C drho, jx, jy, jz;
    moments(v, drho, jx, jy, jz);
    // rho0 = 1
    const C dx = C(u0[c]) - jx, dy = C(u0[plane + c]) - jy, dz = C(u0[2 * plane + c]) - jz;
    static_for<1, Q>([&](auto ic) {
        constexpr int I = decltype(ic)::value;
        constexpr int X = cx(I), Y = cy(I), Z = cz(I);
        C xd = C(0);
        if constexpr (X != 0) xd += C(X) * dx;
        if constexpr (Y != 0) xd += C(Y) * dy;
        if constexpr (Z != 0) xd += C(Z) * dz;
        Traits<S>::store(f + I * plane + c, v[I] + lin3w<C>(X * X + Y * Y + Z * Z) * xd);
    });
}

template <typename S>
static cudaError_t launch_reset(void* f, int N, const double* u0, cudaStream_t stream) {
    const int bx = N >= 128 ? 128 : ((N + 31) / 32) * 32;
    dim3 block(bx), grid((N + bx - 1) / bx, N, N);
    dugks_reset_momentum_kernel<S><<<grid, block, 0, stream>>>((S*)f, N, (size_t)N * N * N, u0);
    return cudaGetLastError();
}

cudaError_t dugks_reset_momentum(int storage, void* f, int N, const double* u0, cudaStream_t stream) {
    switch (storage) {
        case ST_F32: return launch_reset<float>(f, N, u0, stream);
        case ST_F16: return launch_reset<__half>(f, N, u0, stream);
        case ST_BF16: return launch_reset<__nv_bfloat16>(f, N, u0, stream);
        case ST_F64: return launch_reset<double>(f, N, u0, stream);
    }
    return cudaErrorInvalidValue;
}

}  // namespace kin
