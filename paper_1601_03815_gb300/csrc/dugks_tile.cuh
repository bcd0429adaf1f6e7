// Fused DUGKS step (Sec. II.A, Eqs. 9-20): one launch, one read and one write
// of f-tilde per cell.
//
// Each CTA owns a 30 x TY column of cells and marches along z through a chunk
// of planes.  Its 32 x (TY + 2) threads cover the columns plus a one-cell halo;
// every thread runs the cell pre-step (Eq. 19) of its own column for the next
// plane into a three-plane ring of f-bar-plus in shared memory.
//
// Interface reconstruction splits exactly between the two cells of a face.
// With G_i^t(X) = fbp_i(X + e_t) - fbp_i(X - e_t) the Eq. 13/15/16 value at the
// face between L and R = L + e_a is
//   fbar_i = P_i^a(L) + M_i^a(R),
//   P_i^a = (1/2 + h xi_ia) X_i - (h/4) sum_{t != a} xi_it G_i^t,
//   M_i^a = (1/2 - h xi_ia) X_i - (h/4) sum_{t != a} xi_it G_i^t,
// where X = fbp at the cell, and the face moments (Eq. 17) split the same way
// through the moments of X and their tangential differences.  A cell therefore
// builds a "side record" per axis and sign (the 10 populations with
// xi_ia != 0 plus density and momentum), and a face flux (Eqs. 18, 10) needs
// one record from each neighbour: x neighbours exchange records by warp
// shuffles, y neighbours through shared memory, z neighbours are the same
// thread one plane apart.
#pragma once

#include "kin_common.cuh"
#include "dugks_face.cuh"

namespace kin {

// k-th population (k = 0..9) with xi_iA != 0, in increasing index order.
__host__ __device__ constexpr int flux_pop(int A, int k) {
    int n = 0;
    for (int i = 0; i < Q; ++i)
        if (cc(i, A) != 0) {
            if (n == k) return i;
            ++n;
        }
    return -1;
}
// Position of population i in the list of axis T, or -1.
__host__ __device__ constexpr int flux_index(int T, int i) {
    int n = 0;
    for (int j = 0; j < Q; ++j)
        if (cc(j, T) != 0) {
            if (j == i) return n;
            ++n;
        }
    return -1;
}
constexpr int NF = 10;   // populations crossing a face
constexpr int NREC = 14; // side record: 10 populations + density + 3 momentum

template <typename C, int TY>
struct FusedSmem {
    C ring[3][Q][TY + 2][32];
    C my[NREC][TY + 2][32];
    C fy[NF][TY + 1][32];
};

// Raw f-tilde staging for 4-byte storage, filled by cp.async: planes z - 1 and
// z (awaiting their update), z + 1 (next pre-step) and z + 2 (in flight while
// plane z is computed).  Other storage types read global memory directly.
template <typename S, int TY>
struct RawStage {
    S raw[4][Q][TY + 2][32];
};

template <typename S>
constexpr bool kAsyncStage = sizeof(S) == 4;

template <typename S>
__device__ __forceinline__ void cp_async_elem(S* smem_dst, const S* gsrc) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    if constexpr (sizeof(S) == 4) {
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(gsrc) : "memory");
    } else {
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(gsrc) : "memory");
    }
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

template <typename S, int TY>
constexpr size_t fused_smem_bytes() {
    using C = typename Traits<S>::C;
    return sizeof(FusedSmem<C, TY>) + (kAsyncStage<S> ? sizeof(RawStage<S, TY>) : 0);
}

template <typename C>
struct CellView {
    // tangential differences G[t][k] for population flux_pop(t, k)
    C G[3][NF];
    C X[Q];
    C drho, j[3], pi[3][3];
    C DJ[3];     // DJ_t = sum_i xi_it G_i^t
    C DP[3][3];  // DP[c][t] = sum_i xi_ic xi_it G_i^t
};

// Moments of X (delta-rho, j, Pi) via pair sums.
template <typename C>
__device__ __forceinline__ void cell_moments(CellView<C>& v) {
    C a[NPAIR], b[NPAIR];
#pragma unroll
    for (int p = 0; p < NPAIR; ++p) {
        a[p] = v.X[2 * p + 1] + v.X[2 * p + 2];
        b[p] = v.X[2 * p + 1] - v.X[2 * p + 2];
    }
    v.drho = v.X[0] + ((a[0] + a[1]) + a[2]) + (((a[3] + a[4]) + (a[5] + a[6])) + (a[7] + a[8]));
    v.j[0] = (b[0] + b[3]) + (b[4] + (b[5] + b[6]));
    v.j[1] = (b[1] + b[3]) - (b[4] - (b[7] + b[8]));
    v.j[2] = (b[2] + b[5]) - (b[6] - (b[7] - b[8]));
    // Pi_ab = sum xi_a xi_b X: diagonal from pairs with that component, off-diagonal from
    // the diagonal-velocity pairs (p = 3,4: xy; 5,6: xz; 7,8: yz)
    v.pi[0][0] = a[0] + ((a[3] + a[4]) + (a[5] + a[6]));
    v.pi[1][1] = a[1] + ((a[3] + a[4]) + (a[7] + a[8]));
    v.pi[2][2] = a[2] + ((a[5] + a[6]) + (a[7] + a[8]));
    v.pi[0][1] = v.pi[1][0] = a[3] - a[4];
    v.pi[0][2] = v.pi[2][0] = a[5] - a[6];
    v.pi[1][2] = v.pi[2][1] = a[7] - a[8];
}

// DJ and DP for the tangential directions T in the mask (bit t set).
template <int MASK, typename C>
__device__ __forceinline__ void cell_diffs(CellView<C>& v) {
    static_for<0, 3>([&](auto tc) {
        constexpr int T = decltype(tc)::value;
        if constexpr ((MASK >> T) & 1) {
            C dj = C(0), d[3] = {C(0), C(0), C(0)};
            static_for<0, NF>([&](auto kc) {
                constexpr int K = decltype(kc)::value;
                constexpr int I = flux_pop(T, K);
                const C g = v.G[T][K];
                if constexpr (cc(I, T) > 0) {
                    dj += g;
                } else {
                    dj -= g;
                }
                d[T] += g;  // xi_it^2 = 1
                static_for<0, 3>([&](auto ccn) {
                    constexpr int CC = decltype(ccn)::value;
                    if constexpr (CC != T && cc(I, CC) != 0) {
                        if constexpr (cc(I, CC) * cc(I, T) > 0) d[CC] += g;
                        else d[CC] -= g;
                    }
                });
            });
            v.DJ[T] = dj;
            v.DP[0][T] = d[0];
            v.DP[1][T] = d[1];
            v.DP[2][T] = d[2];
        }
    });
}

// Side record of a cell for axis A; SIGN = +1 gives P (cell is the left/lower
// neighbour), -1 gives M (cell is the right/upper neighbour).
template <int A, int SIGN, typename C>
__device__ __forceinline__ void side_record(const CellView<C>& v, C h, C hq, C (&rec)[NREC]) {
    constexpr int T1 = (A + 1) % 3, T2 = (A + 2) % 3;
    static_for<0, NF>([&](auto kc) {
        constexpr int K = decltype(kc)::value;
        constexpr int I = flux_pop(A, K);
        C t = C(0);
        if constexpr (cc(I, T1) != 0) {
            constexpr int k1 = flux_index(T1, I);
            t = cc(I, T1) > 0 ? v.G[T1][k1] : -v.G[T1][k1];
        }
        if constexpr (cc(I, T2) != 0) {
            constexpr int k2 = flux_index(T2, I);
            t += cc(I, T2) > 0 ? v.G[T2][k2] : -v.G[T2][k2];
        }
        constexpr int s = SIGN * cc(I, A);  // +1 or -1
        const C coef = s > 0 ? (C(0.5) + h) : (C(0.5) - h);
        rec[K] = coef * v.X[I] - hq * t;
    });
    const C sh = SIGN > 0 ? h : -h;
    rec[10] = C(0.5) * v.drho + sh * v.j[A] - hq * (v.DJ[T1] + v.DJ[T2]);
    static_for<0, 3>([&](auto ccn) {
        constexpr int CC = decltype(ccn)::value;
        rec[11 + CC] = C(0.5) * v.j[CC] + sh * v.pi[A][CC] - hq * (v.DP[CC][T1] + v.DP[CC][T2]);
    });
}

// Face flux F_k = xi_{iA} f_i(x_b, t + h) (Eqs. 17, 7, 18, 10) from the two side records.
template <int A, typename C>
__device__ __forceinline__ void face_from_records(const C (&P)[NREC], const C (&M)[NREC],
                                                  const DugksCoef<C>& k, C (&F)[NF]) {
    const C drho = P[10] + M[10];
    const C ux = P[11] + M[11], uy = P[12] + M[12], uz = P[13] + M[13];
    const C a0 = drho - C(1.5) * (ux * ux + uy * uy + uz * uz);
    static_for<0, NF>([&](auto kc) {
        constexpr int K = decltype(kc)::value;
        constexpr int I = flux_pop(A, K);
        C s = C(0);
        if constexpr (cx(I) != 0) s += C(cx(I)) * ux;
        if constexpr (cy(I) != 0) s += C(cy(I)) * uy;
        if constexpr (cz(I) != 0) s += C(cz(I)) * uz;
        const C w = C(w36(I)) / C(36);
        const C fe = w * (a0 + C(4.5) * s * s) + lin3w<C>(cx(I) * cx(I) + cy(I) * cy(I) + cz(I) * cz(I)) * s;
        const C fb = P[K] + M[K];
        const C ff = fb + k.c2 * (fe - fb);  // Eq. 18, c1 + c2 = 1
        F[K] = cc(I, A) > 0 ? ff : -ff;
    });
}

__device__ __forceinline__ int wrapc(int v, int n) {
    v %= n;
    return v < 0 ? v + n : v;
}

// One tile (tile coordinates bx, by, bz) of the fused step, run by a
// 32 x (TY + 2) thread block with fused_smem_bytes<S, TY>() of dynamic shared
// memory at smem_raw.  Also called by the persistent ensemble kernel.
template <typename S, int TY>
__device__ __forceinline__ void dugks_tile(const S* __restrict__ src, S* __restrict__ dst, int N,
                                           int bx, int by, int bz, int zchunk,
                                           const DugksCoef<typename Traits<S>::C>& kc,
                                           unsigned char* smem_raw) {
    using C = typename Traits<S>::C;
    FusedSmem<C, TY>& sm = *reinterpret_cast<FusedSmem<C, TY>*>(smem_raw);
    RawStage<S, TY>* stage = reinterpret_cast<RawStage<S, TY>*>(smem_raw + sizeof(FusedSmem<C, TY>));

    const int lane = threadIdx.x, row = threadIdx.y;
    const int x0 = bx * 30, y0 = by * TY, z0 = bz * zchunk;
    const int zend = min(z0 + zchunk, N);
    const int gxr = x0 - 1 + lane, gyr = y0 - 1 + row;
    const int gx = wrapc(gxr, N), gy = wrapc(gyr, N);
    const bool xin = lane >= 1 && lane <= 30;
    const bool yin = row >= 1 && row <= TY;
    const bool interior = xin && yin;
    const bool valid = interior && gxr < N && gyr < N;
    const size_t plane = (size_t)N * N * N;
    const size_t colidx = (size_t)gx + (size_t)N * gy;
    const size_t nn = (size_t)N * N;
    const C h = kc.h, hq = C(0.25) * kc.h;
    // x neighbours, clamped so the two halo lanes can run the interior code
    // path (their x differences are never used)
    const int lp = min(lane + 1, 31), lm = max(lane - 1, 0);

    // ring slots hold fbp of planes z-1, z, z+1; raw slots hold f-tilde of
    // planes z-1 (update), z (next update), z+1 (next pre-step), z+2 (in flight)
    auto slot_of = [&](int z) { return (z - z0 + 3) % 3; };
    auto rslot_of = [&](int z) { return (z - z0 + 4) & 3; };

    auto issue_plane = [&](int z) {
        if constexpr (kAsyncStage<S>) {
            const S* p = src + (size_t)wrapc(z, N) * nn + colidx;
            const int s = rslot_of(z);
#pragma unroll
            for (int i = 0; i < Q; ++i) cp_async_elem(&stage->raw[s][i][row][lane], p + i * plane);
            cp_async_commit();
        }
    };
    auto raw_value = [&](int z, int i) -> C {
        if constexpr (kAsyncStage<S>) {
            return (C)stage->raw[rslot_of(z)][i][row][lane];
        } else {
            return Traits<S>::load(src + (size_t)wrapc(z, N) * nn + colidx + i * plane);
        }
    };
    // Eq. 19 for this thread's column at plane z into the ring.
    auto prestep = [&](int z) {
        C f[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) f[i] = raw_value(z, i);
        C drho, jx, jy, jz;
        moments(f, drho, jx, jy, jz);
        const C usq15 = C(1.5) * (jx * jx + jy * jy + jz * jz);
        const int s = slot_of(z);
        static_for<0, Q>([&](auto ic) {
            constexpr int I = decltype(ic)::value;
            // Eq. 19 with a + b = 1 written so a fixed point stays exact in any precision
            sm.ring[s][I][row][lane] = f[I] + kc.b * (feq_i<I>(drho, jx, jy, jz, usq15) - f[I]);
        });
    };
    // Cell view at ring slot s with the tangential differences in MASK.
    auto gather = [&](int s, int sm1, int sp1, auto maskc, CellView<C>& v) {
        constexpr int MASK = decltype(maskc)::value;
#pragma unroll
        for (int i = 0; i < Q; ++i) v.X[i] = sm.ring[s][i][row][lane];
        static_for<0, 3>([&](auto tc) {
            constexpr int T = decltype(tc)::value;
            if constexpr ((MASK >> T) & 1) {
                static_for<0, NF>([&](auto kc2) {
                    constexpr int K = decltype(kc2)::value;
                    constexpr int I = flux_pop(T, K);
                    C g;
                    if constexpr (T == 0) g = sm.ring[s][I][row][lp] - sm.ring[s][I][row][lm];
                    else if constexpr (T == 1) g = sm.ring[s][I][row + 1][lane] - sm.ring[s][I][row - 1][lane];
                    else g = sm.ring[sp1][I][row][lane] - sm.ring[sm1][I][row][lane];
                    v.G[T][K] = g;
                });
            }
        });
        cell_moments(v);
        cell_diffs<MASK>(v);
    };

    issue_plane(z0 - 1);
    issue_plane(z0);
    cp_async_wait_all();
    prestep(z0 - 1);
    prestep(z0);
    issue_plane(z0 + 1);
    __syncthreads();
    C Pz[NREC];   // P^z record of the plane below the current one
    C Dprev[Q];   // face-flux sum of plane z-1, still missing its +z face
    if (interior) {
        CellView<C> v;
        gather(slot_of(z0 - 1), 0, 0, std::integral_constant<int, 3>{}, v);
        side_record<2, +1>(v, h, hq, Pz);
    }
#pragma unroll
    for (int i = 0; i < Q; ++i) Dprev[i] = C(0);

    for (int z = z0; z <= zend; ++z) {
        const bool last = z == zend;
        if (!last) {
            if constexpr (kAsyncStage<S>) cp_async_wait_all();
            prestep(z + 1);
            if (z + 2 <= zend) issue_plane(z + 2);
        }
        __syncthreads();  // ring slot of z + 1 complete; fy of plane z - 1 complete
        C Dcur[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) Dcur[i] = C(0);
        C Py[NREC];
        if (!last) {
            const int s0 = slot_of(z), sm1 = slot_of(z - 1), sp1 = slot_of(z + 1);
            CellView<C> v;
            // warp-uniform: rows 1..TY take every difference, the halo rows
            // only those their y records need
            if (yin) {
                gather(s0, sm1, sp1, std::integral_constant<int, 7>{}, v);
            } else {
                gather(s0, sm1, sp1, std::integral_constant<int, 5>{}, v);  // G^x, G^z
            }
            C Px[NREC], Mx[NREC];
            if (yin) {
                side_record<0, +1>(v, h, hq, Px);
                side_record<0, -1>(v, h, hq, Mx);
            }
            if (xin) {
                C My[NREC];
                side_record<1, +1>(v, h, hq, Py);
                side_record<1, -1>(v, h, hq, My);
#pragma unroll
                for (int r = 0; r < NREC; ++r) sm.my[r][row][lane] = My[r];
            }
            // x faces: this lane's face to the right uses the next lane's M record
            C Mn[NREC];
#pragma unroll
            for (int r = 0; r < NREC; ++r) Mn[r] = __shfl_down_sync(0xffffffffu, Mx[r], 1);
            C Fx[NF];
            if (yin && lane <= 30) face_from_records<0>(Px, Mn, kc, Fx);
            C Fl[NF];
#pragma unroll
            for (int r = 0; r < NF; ++r) Fl[r] = __shfl_up_sync(0xffffffffu, Fx[r], 1);
            if (interior) {
                static_for<0, NF>([&](auto kc2) {
                    constexpr int K = decltype(kc2)::value;
                    Dcur[flux_pop(0, K)] += Fx[K] - Fl[K];
                });
                // z face (z-1, z): P^z(z-1) carried, M^z(z) from this view
                C Mz[NREC], Fz[NF];
                side_record<2, -1>(v, h, hq, Mz);
                face_from_records<2>(Pz, Mz, kc, Fz);
                static_for<0, NF>([&](auto kc2) {
                    constexpr int K = decltype(kc2)::value;
                    Dprev[flux_pop(2, K)] += Fz[K];
                    Dcur[flux_pop(2, K)] -= Fz[K];
                });
                side_record<2, +1>(v, h, hq, Pz);
            }
        } else if (interior) {
            CellView<C> v;
            C Mz[NREC], Fz[NF];
            gather(slot_of(z), 0, 0, std::integral_constant<int, 3>{}, v);
            side_record<2, -1>(v, h, hq, Mz);
            face_from_records<2>(Pz, Mz, kc, Fz);
            static_for<0, NF>([&](auto kc2) {
                constexpr int K = decltype(kc2)::value;
                Dprev[flux_pop(2, K)] += Fz[K];
            });
        }
        // update plane z - 1 (Eqs. 20, 9): its y faces were computed one iteration ago
        if (z > z0 && interior) {
            static_for<0, NF>([&](auto kc2) {
                constexpr int K = decltype(kc2)::value;
                Dprev[flux_pop(1, K)] += sm.fy[K][row][lane] - sm.fy[K][row - 1][lane];
            });
            if (valid) {
                const size_t c = (size_t)(z - 1) * nn + colidx;
                const int sp = slot_of(z - 1);
#pragma unroll
                for (int i = 0; i < Q; ++i) {
                    const C ft = raw_value(z - 1, i);
                    const C fb = sm.ring[sp][i][row][lane];
                    Traits<S>::store(dst + i * plane + c,
                                     fb + (fb - ft) * C(1.0 / 3.0) - kc.dt * Dprev[i]);
                }
            }
        }
        __syncthreads();  // my of plane z complete; fy of plane z - 1 consumed
        if (!last && xin && row <= TY) {
            // y faces of plane z: face r between rows r and r + 1, r = 0..TY
            C Mu[NREC], Fy[NF];
#pragma unroll
            for (int r = 0; r < NREC; ++r) Mu[r] = sm.my[r][row + 1][lane];
            face_from_records<1>(Py, Mu, kc, Fy);
#pragma unroll
            for (int r = 0; r < NF; ++r) sm.fy[r][row][lane] = Fy[r];
        }
#pragma unroll
        for (int i = 0; i < Q; ++i) Dprev[i] = Dcur[i];
    }
}

// Coefficients of Eqs. 18-19 for viscosity nu (tau = nu / RT) and step dt.
template <typename C>
inline DugksCoef<C> dugks_coef(double nu, double dt) {
    const double tau = 3.0 * nu, h = 0.5 * dt;
    DugksCoef<C> k;
    k.a = C((2.0 * tau - h) / (2.0 * tau + dt));
    k.b = C(3.0 * h / (2.0 * tau + dt));
    k.h = C(h);
    k.c1 = C(2.0 * tau / (2.0 * tau + h));
    k.c2 = C(h / (2.0 * tau + h));
    k.dt = C(dt);
    return k;
}

}  // namespace kin
