// DUGKS interface flux for one cell face (Sec. II.A, Eqs. 13-18, 10).
#pragma once

#include "kin_common.cuh"
#include "pair_math.cuh"

namespace kin {

// Coefficients of one DUGKS step for relaxation time tau and step dt (h = dt/2):
//   Eq. 19: fbp = a ft + b feq,  a = (2tau - h)/(2tau + dt), b = 3h/(2tau + dt)
//   Eq. 18: f_face = c1 fbar + c2 feq_face, c1 = 2tau/(2tau + h), c2 = h/(2tau + h)
template <typename C>
struct DugksCoef {
    C a, b, h, c1, c2, dt;
    // Derived constants of the fused step (dugks_coef fills them):
    C hq;            // h / 4, weight of a tangential central difference at a face
    C qk[2];         // 4.5 c2 W for axis (0) and diagonal (1) velocities
    C qw[2];         // c2 W
    C ql[2];         // c2 times the linear-term coefficient 3 W
    Pr<C> cpp, cpm;  // (1/2 + h, 1/2 - h) and (1/2 - h, 1/2 + h)
    Pr<C> hqp, hqm;  // (-h/4, h/4) and (h/4, -h/4)
    Pr<C> b2;        // (b, b)
    Pr<C> c1p;       // (1 - c2, 1 - c2)
    Pr<C> third;     // (1/3, 1/3)
    Pr<C> dts;       // (-dt, dt)
};

// Interface flux through the face normal to axis A between L (the stencil
// origin) and R = L + e_A.  get(i, dx, dy, dz) returns f-bar-plus_i at
// L + (dx, dy, dz).  On return F[i] = xi_iA * f_i(x_b, t + h) for every i with
// xi_iA != 0 (other entries are left untouched).
//
// Reconstruction (Eqs. 13, 15, 16): the face value is the mean of the two
// cell values, the normal gradient their difference, and each tangential
// gradient component the mean of the two cells' central differences.
template <int A, typename C, typename Get>
__device__ __forceinline__ void face_flux(const Get& get, const DugksCoef<C>& k, C (&F)[Q]) {
    constexpr int AX = A == 0, AY = A == 1, AZ = A == 2;
    C fbar[Q];
    static_for<0, Q>([&](auto ic) {
        constexpr int I = decltype(ic)::value;
        const C L = get(I, 0, 0, 0);
        const C R = get(I, AX, AY, AZ);
        C s = C(0);
        if constexpr (cc(I, A) != 0) s = C(cc(I, A)) * (R - L);
        static_for<0, 3>([&](auto tc) {
            constexpr int T = decltype(tc)::value;
            if constexpr (T != A && cc(I, T) != 0) {
                constexpr int TX = T == 0, TY = T == 1, TZ = T == 2;
                const C dL = get(I, TX, TY, TZ) - get(I, -TX, -TY, -TZ);
                const C dR = get(I, AX + TX, AY + TY, AZ + TZ) - get(I, AX - TX, AY - TY, AZ - TZ);
                s += C(cc(I, T)) * (C(0.25) * (dL + dR));
            }
        });
        fbar[I] = C(0.5) * (L + R) - k.h * s;
    });
    C drho, jx, jy, jz;
    moments(fbar, drho, jx, jy, jz);
    const C usq15 = C(1.5) * (jx * jx + jy * jy + jz * jz);
    static_for<0, Q>([&](auto ic) {
        constexpr int I = decltype(ic)::value;
        if constexpr (cc(I, A) != 0) {
            const C fe = feq_i<I>(drho, jx, jy, jz, usq15);
            const C ff = fbar[I] + k.c2 * (fe - fbar[I]);  // Eq. 18, c1 + c2 = 1
            F[I] = cc(I, A) > 0 ? ff : -ff;
        }
    });
}

}  // namespace kin
