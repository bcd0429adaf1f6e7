// Fused DUGKS step (Sec. II.A, Eqs. 9-20): one launch, one read and one write
// of f-tilde per cell.
//
// Each CTA owns a 30 x TY column of cells and marches along z through a chunk
// of planes.  Its 32 x (TY + 2) threads cover the columns plus a one-cell halo;
// every thread runs the cell pre-step (Eq. 19) of its own column for the next
// plane into a three-plane ring of f-bar-plus in shared memory, fed by
// cp.async copies of f-tilde issued two planes ahead (by four of the warps
// for every row; an issuer waits for its copies at the end of a plane and
// the next barrier publishes them).  Two block barriers per plane: one before
// the plane's work, whose first part is the pre-step of the next plane (only
// this thread reads the slot it fills until the next barrier, so its
// arithmetic interleaves with the faces of this plane), and one before the
// y faces.
//
// Interface reconstruction splits exactly between the two cells of a face.
// With G_i^t(X) = fbp_i(X + e_t) - fbp_i(X - e_t) the Eq. 13/15/16 value at the
// face between L and R = L + e_a is
//   fbar_i = P_i^a(L) + M_i^a(R),
//   P_i^a = (1/2 + h xi_ia) X_i - (h/4) sum_{t != a} xi_it G_i^t,
//   M_i^a = (1/2 - h xi_ia) X_i - (h/4) sum_{t != a} xi_it G_i^t,
// where X = fbp at the cell; summed over i, the face moments (Eq. 17) split the
// same way through the moments of X and their tangential differences.  A cell
// builds a "side record" per axis and sign (the 5 velocity pairs crossing the
// face plus density and momentum); a face (Eqs. 17, 7, 18, 10) needs one
// record from each neighbour: x neighbours exchange records by warp shuffles,
// y neighbours through shared memory, z neighbours are the same thread one
// plane apart.
//
// Updates lag one plane so the z face uses one cell view per plane.
//
// Opposite populations (2p+1, 2p+2) travel as one pair (pair_math.cuh): both
// always undergo the same operation with a fixed coefficient pattern, so one
// packed FP32x2 instruction serves both.  Flux sums are kept sign-folded,
// Dhat_p = (D_{2p+1}, -D_{2p+2}), so a face adds the same signed value to
// both members.
#pragma once

#include <type_traits>

#include "dugks_face.cuh"
#include "kin_common.cuh"
#include "kin_debug.cuh"
#include "pair_math.cuh"

namespace kin {

// ------------------------------------------------------------------ pair tables
constexpr int NC = 5;  // velocity pairs crossing a face

// Component a of the velocity of pair p (that of population 2p+1).
__host__ __device__ constexpr int pe(int p, int a) {
    return a == 0 ? pair_x(p) : a == 1 ? pair_y(p) : pair_z(p);
}
// k-th pair (k = 0..4) whose velocity has a nonzero A component.
__host__ __device__ constexpr int cross_pair(int A, int k) {
    int n = 0;
    for (int p = 0; p < NPAIR; ++p)
        if (pe(p, A) != 0) {
            if (n == k) return p;
            ++n;
        }
    return -1;
}
// Position of pair p in the list of axis A, or -1.
__host__ __device__ constexpr int cross_index(int A, int p) {
    int n = 0;
    for (int q = 0; q < NPAIR; ++q)
        if (pe(q, A) != 0) {
            if (q == p) return n;
            ++n;
        }
    return -1;
}
// The other nonzero axis of diagonal pair p crossing A (-1 for an axis pair).
__host__ __device__ constexpr int tang_axis(int p, int A) {
    for (int t = 0; t < 3; ++t)
        if (t != A && pe(p, t) != 0) return t;
    return -1;
}

// e_p . (x, y, z); the first nonzero component of every e_p is +1.
template <int P, typename C>
__device__ __forceinline__ C pdot(C x, C y, C z) {
    constexpr int X = pair_x(P), Y = pair_y(P), Z = pair_z(P);
    if constexpr (X != 0) {
        static_assert(X == 1, "pair velocity convention");
        if constexpr (Y != 0) return Y > 0 ? x + y : x - y;
        else if constexpr (Z != 0) return Z > 0 ? x + z : x - z;
        else return x;
    } else if constexpr (Y != 0) {
        static_assert(Y == 1, "pair velocity convention");
        if constexpr (Z != 0) return Z > 0 ? y + z : y - z;
        else return y;
    } else {
        static_assert(Z == 1, "pair velocity convention");
        return z;
    }
}

// ------------------------------------------------------------------ shared memory
template <typename C, int TY>
struct FusedSmem {
    Pr<C> ring[3][NPAIR][TY + 2][32];  // f-bar-plus pairs of planes z - 1, z, z + 1
    Pr<C> my[NC][TY + 2][32];          // y-face M records (pairs)
    Pr<C> fy[NC][TY + 1][32];          // y-face values
    C ring0[3][TY + 2][32];            // rest population of the ring
    C mym[4][TY + 2][32];              // y-face M records (density, momentum)
};

// Raw f-tilde staging for FP32 storage, filled by 4-byte cp.async copies:
// planes z - 1 and z (awaiting their update), z + 1 (next pre-step) and z + 2
// (in flight while plane z is computed).  One population per 128-byte row, so
// a warp's copy instruction fills one row without bank conflicts and touches
// one population plane; the pre-step and update read the two members of a
// pair with two 4-byte loads.  FP64 storage reads global memory directly.
template <int TY>
struct RawStage {
    float raw[4][Q][TY + 2][32];
};

template <typename S>
constexpr bool kAsyncStage = std::is_same<S, float>::value;

// Raw staging of 2-byte storage (FP16, BF16) for even N: lanes 0..16 of a
// row's warp copy the row of each population as 17 aligned 4-byte words, the
// 34 elements from x0 - 2; thread `lane` reads element lane + 1.  Odd N (a
// word would straddle the periodic wrap) reads global memory directly, in a
// separate instantiation (template flag EVEN = false) so that the even-N code
// carries neither the branch nor the registers of that path.
template <typename S, int TY>
struct RawStage16 {
    S raw[4][Q][TY + 2][34];
};
template <typename S>
constexpr bool kStage16 = sizeof(S) == 2;

template <typename S>
__device__ __forceinline__ float to_float(S v) {
    if constexpr (std::is_same<S, __half>::value) return __half2float(v);
    else return __bfloat162float(v);
}

__device__ __forceinline__ void cp_async4(void* smem_dst, const void* gsrc) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

template <typename S, int TY>
constexpr size_t fused_smem_bytes() {
    using C = typename Traits<S>::C;
    return sizeof(FusedSmem<C, TY>) +
           (kAsyncStage<S> ? sizeof(RawStage<TY>) : kStage16<S> ? sizeof(RawStage16<S, TY>) : 0);
}

// ------------------------------------------------------------------ cell view
template <typename C>
struct CellView {
    Pr<C> X[NPAIR];   // f-bar-plus pairs at the cell
    C X0;             // rest population
    Pr<C> G[3][NC];   // G[t][k] = X(+e_t) - X(-e_t) for pair cross_pair(t, k)
    C drho, j[3], pi[3][3];
    C hrho, hj[3];    // drho / 2, j / 2
    C DJ[3];          // DJ_t = sum_i xi_it G_i^t
    C DP[3][3];       // DP[c][t] = sum_i xi_ic xi_it G_i^t
};

// Moments of X (delta-rho, j, Pi = sum xi xi X) via pair sums and differences.
template <typename C>
__device__ __forceinline__ void view_moments(CellView<C>& v) {
    C a[NPAIR], b[NPAIR];
#pragma unroll
    for (int p = 0; p < NPAIR; ++p) {
        a[p] = v.X[p].x + v.X[p].y;
        b[p] = v.X[p].x - v.X[p].y;
    }
    const C s34 = a[3] + a[4], s56 = a[5] + a[6], s78 = a[7] + a[8];
    v.drho = v.X0 + (((a[0] + a[1]) + a[2]) + ((s34 + s56) + s78));
    v.j[0] = (b[0] + b[3]) + (b[4] + (b[5] + b[6]));
    v.j[1] = (b[1] + b[3]) - (b[4] - (b[7] + b[8]));
    v.j[2] = (b[2] + b[5]) - (b[6] - (b[7] - b[8]));
    v.pi[0][0] = a[0] + (s34 + s56);
    v.pi[1][1] = a[1] + (s34 + s78);
    v.pi[2][2] = a[2] + (s56 + s78);
    v.pi[0][1] = v.pi[1][0] = a[3] - a[4];
    v.pi[0][2] = v.pi[2][0] = a[5] - a[6];
    v.pi[1][2] = v.pi[2][1] = a[7] - a[8];
    v.hrho = C(0.5) * v.drho;
    v.hj[0] = C(0.5) * v.j[0];
    v.hj[1] = C(0.5) * v.j[1];
    v.hj[2] = C(0.5) * v.j[2];
}

// Coefficient of term k in a difference sum of axis T: W = 3 gives DJ_T
// (weight e_pT on G.x - G.y), W = c gives DP[c][T] (weight e_pc e_pT on
// G.x + G.y).
template <int T, int W>
__host__ __device__ constexpr int dcoef(int k) {
    return W == 3 ? pe(cross_pair(T, k), T) : pe(cross_pair(T, k), W) * pe(cross_pair(T, k), T);
}
// Signed sum of vals[k] over the nonzero coefficients, starting from the first
// term (no addition of zero).
template <int T, int W, int K, bool STARTED, typename C>
__device__ __forceinline__ C dsum(const C (&vals)[NC], C acc) {
    if constexpr (K == NC) {
        return acc;
    } else {
        constexpr int cf = dcoef<T, W>(K);
        if constexpr (cf == 0) {
            return dsum<T, W, K + 1, STARTED>(vals, acc);
        } else if constexpr (!STARTED) {
            return dsum<T, W, K + 1, true>(vals, cf > 0 ? vals[K] : -vals[K]);
        } else {
            return dsum<T, W, K + 1, true>(vals, cf > 0 ? acc + vals[K] : acc - vals[K]);
        }
    }
}

// DJ and DP for the tangential directions T in MASK (bit t set).
template <int MASK, typename C>
__device__ __forceinline__ void view_diffs(CellView<C>& v) {
    static_for<0, 3>([&](auto tc) {
        constexpr int T = decltype(tc)::value;
        if constexpr ((MASK >> T) & 1) {
            C sg[NC], dg[NC];
#pragma unroll
            for (int k = 0; k < NC; ++k) {
                sg[k] = v.G[T][k].x + v.G[T][k].y;
                dg[k] = v.G[T][k].x - v.G[T][k].y;
            }
            v.DJ[T] = dsum<T, 3, 0, false>(dg, C(0));
            v.DP[0][T] = dsum<T, 0, 0, false>(sg, C(0));
            v.DP[1][T] = dsum<T, 1, 0, false>(sg, C(0));
            v.DP[2][T] = dsum<T, 2, 0, false>(sg, C(0));
        }
    });
}

// ------------------------------------------------------------------ side records
template <typename C>
struct Rec {
    Pr<C> r[NC];  // pairs crossing the face, in cross_pair order
    C m[4];       // density, momentum
};

// P (cell on the lower side of the face along A) and M (upper side) records.
template <int A, bool WANT_P, bool WANT_M, typename C>
__device__ __forceinline__ void side_records(const CellView<C>& v, const DugksCoef<C>& k, Rec<C>& P,
                                             Rec<C>& M) {
    constexpr int T1 = (A + 1) % 3, T2 = (A + 2) % 3;
    static_for<0, NC>([&](auto kc) {
        constexpr int K = decltype(kc)::value;
        constexpr int p = cross_pair(A, K);
        constexpr int sg = pe(p, A);
        // (1/2 + h xi_iA) for the two members: P uses cpp when e_pA = +1
        [[maybe_unused]] const Pr<C> cP = sg > 0 ? k.cpp : k.cpm;
        [[maybe_unused]] const Pr<C> cM = sg > 0 ? k.cpm : k.cpp;
        if constexpr (p < 3) {
            if constexpr (WANT_P) P.r[K] = pmul(cP, v.X[p]);
            if constexpr (WANT_M) M.r[K] = pmul(cM, v.X[p]);
        } else {
            constexpr int T = tang_axis(p, A);
            constexpr int tau = pe(p, T);
            // -(h/4) xi_iT G_i^T for both members
            const Pr<C> ht = pmul(tau > 0 ? k.hqp : k.hqm, v.G[T][cross_index(T, p)]);
            if constexpr (WANT_P) P.r[K] = pfma(cP, v.X[p], ht);
            if constexpr (WANT_M) M.r[K] = pfma(cM, v.X[p], ht);
        }
    });
    const C br = fma(-k.hq, v.DJ[T1] + v.DJ[T2], v.hrho);
    if constexpr (WANT_P) P.m[0] = fma(k.h, v.j[A], br);
    if constexpr (WANT_M) M.m[0] = fma(-k.h, v.j[A], br);
    static_for<0, 3>([&](auto ccn) {
        constexpr int CC = decltype(ccn)::value;
        const C bc = fma(-k.hq, v.DP[CC][T1] + v.DP[CC][T2], v.hj[CC]);
        if constexpr (WANT_P) P.m[1 + CC] = fma(k.h, v.pi[A][CC], bc);
        if constexpr (WANT_M) M.m[1 + CC] = fma(-k.h, v.pi[A][CC], bc);
    });
}

// Face values f_i(x_b, t + h) = c1 fbar_i + c2 f_eq_i (Eqs. 17, 7, 18) of the
// pairs crossing the face along A, from the two side records.
template <int A, typename C>
__device__ __forceinline__ void face_values(const Rec<C>& P, const Rec<C>& M, const DugksCoef<C>& k,
                                            Pr<C> (&ff)[NC]) {
    const C rho = P.m[0] + M.m[0];
    const C ux = P.m[1] + M.m[1], uy = P.m[2] + M.m[2], uz = P.m[3] + M.m[3];
    const C a0 = fma(C(-1.5), fma(uz, uz, fma(uy, uy, ux * ux)), rho);
    const C wa_ax = k.qw[0] * a0, wa_dg = k.qw[1] * a0;
    static_for<0, NC>([&](auto kc) {
        constexpr int K = decltype(kc)::value;
        constexpr int p = cross_pair(A, K);
        constexpr int cls = p < 3 ? 0 : 1;
        const C s = pdot<p>(ux, uy, uz);
        const C q = fma(k.qk[cls] * s, s, cls == 0 ? wa_ax : wa_dg);  // c2 W (a0 + 9/2 s^2)
        const C l = k.ql[cls] * s;                                   // c2 3W s
        ff[K] = pfma(k.c1p, padd(P.r[K], M.r[K]), pmk(q + l, q - l));
    });
}

template <typename C>
__device__ __forceinline__ Pr<C> pshfl_down1(Pr<C> v) {
    return pmk(__shfl_down_sync(0xffffffffu, v.x, 1), __shfl_down_sync(0xffffffffu, v.y, 1));
}
template <typename C>
__device__ __forceinline__ Pr<C> pshfl_up1(Pr<C> v) {
    return pmk(__shfl_up_sync(0xffffffffu, v.x, 1), __shfl_up_sync(0xffffffffu, v.y, 1));
}

__device__ __forceinline__ int wrapc(int v, int n) {
    v %= n;
    return v < 0 ? v + n : v;
}

// ------------------------------------------------------------------ the tile
// One tile (tile coordinates bx, by, bz) of the fused step, run by a
// 32 x (TY + 2) thread block with fused_smem_bytes<S, TY>() of dynamic shared
// memory at smem_raw (16-byte aligned).  Also called by the persistent
// ensemble kernel.  With VEL (FP32-computed storage) the tile also writes
// rho0 u = sum xi f of the stored new state (Eq. 8) to uvel[3][N^3], summed in
// population order.
template <typename S, int TY, bool VEL = false, bool EVEN = true>
__device__ __forceinline__ void dugks_tile(const S* __restrict__ src, S* __restrict__ dst, int N,
                                           int bx, int by, int bz, int zchunk,
                                           const DugksCoef<typename Traits<S>::C>& kc,
                                           unsigned char* smem_raw, float* __restrict__ uvel = nullptr) {
    using C = typename Traits<S>::C;
    using P2 = Pr<C>;
    static_assert(!VEL || std::is_same<C, float>::value, "the fused velocity serves FP32-computed storage");
    FusedSmem<C, TY>& sm = *reinterpret_cast<FusedSmem<C, TY>*>(smem_raw);
    RawStage<TY>* stage = reinterpret_cast<RawStage<TY>*>(smem_raw + sizeof(FusedSmem<C, TY>));
    RawStage16<S, TY>* stage16 = reinterpret_cast<RawStage16<S, TY>*>(smem_raw + sizeof(FusedSmem<C, TY>));

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
    // x neighbours, clamped so the two halo lanes can run the interior code
    // path (their x differences are never used)
    const int lp = min(lane + 1, 31), lm = max(lane - 1, 0);

    auto zwrap = [&](int z) { return z < 0 ? z + N : (z >= N ? z - N : z); };
    auto rslot_of = [&](int z) { return (z - z0 + 4) & 3; };

    // 2-byte staging (EVEN: the caller guarantees an even N): this lane's word
    // starts at element x0 - 2 + 2 lane (even, so it never straddles the wrap)
    constexpr bool use16 = kStage16<S> && EVEN;
    const size_t rowidx = (size_t)N * gy + (size_t)wrapc(x0 - 2 + 2 * lane, N);

    // The staging copies of all rows are issued by the warps of rows r with
    // r % 4 >= 2 (rows 2, 3, 6, 7 of a 10-row block; warps are dealt to the
    // SM's four schedulers in turn, so these sit on the two that hold two
    // warps instead of three).  Row r2's copies go to issuer r2 % NI; an
    // issuer takes at most KR rows.  Measured against every thread copying
    // its own column: FP32 unchanged (0.961 vs 0.964 ms at 256^3), FP16 and
    // BF16 3 % faster (a 2-byte row is copied by 17 of the 32 lanes).
    constexpr int NW = TY + 2;
    constexpr int NI = (NW / 4) * 2 + (NW % 4 > 2 ? NW % 4 - 2 : 0);
    constexpr int KR = (NW + NI - 1) / NI;
    const bool issuer = (row & 3) >= 2;
    const int iidx = (row >> 2) * 2 + (row & 3) - 2;  // rank among the issuers (issuers only)
    unsigned icol[KR];  // y + N x part of each assigned row's column (x from this lane)
#pragma unroll
    for (int k = 0; k < KR; ++k) {
        const int r2 = iidx + k * NI;
        const int gy2 = wrapc(y0 - 1 + (r2 < NW ? r2 : 0), N);
        if constexpr (use16) icol[k] = (unsigned)N * gy2 + (unsigned)wrapc(x0 - 2 + 2 * lane, N);
        else icol[k] = (unsigned)gx + (unsigned)N * gy2;
    }

    // issuers only: the copies of plane z for their assigned rows
    auto issue_plane = [&](int z) {
        const int s = rslot_of(z);
#pragma unroll
        for (int k = 0; k < KR; ++k) {
            const int r2 = iidx + k * NI;
            if (r2 >= NW) continue;
            const size_t o = (size_t)zwrap(z) * nn + icol[k];
            if constexpr (use16) {
                if (lane <= 16) {
#pragma unroll
                    for (int i = 0; i < Q; ++i)
                        if (KIN_CHECK(o + i * plane + 1 < Q * plane, DBG_DUGKS_LOAD, o + i * plane + 1) &&
                            KIN_CHECK(s >= 0 && s < 4, DBG_DUGKS_SLOT, s))
                            cp_async4(&stage16->raw[s][i][r2][2 * lane], src + o + i * plane);
                }
            }
            if constexpr (kAsyncStage<S>) {
#pragma unroll
                for (int i = 0; i < Q; ++i)
                    if (KIN_CHECK(o + i * plane < Q * plane, DBG_DUGKS_LOAD, o + i * plane) &&
                        KIN_CHECK(s >= 0 && s < 4, DBG_DUGKS_SLOT, s))
                        cp_async4(&stage->raw[s][i][r2][lane], src + o + i * plane);
            }
        }
        cp_async_commit();
    };
    auto raw_pair = [&](int z, int q) -> P2 {
        if constexpr (kAsyncStage<S>) {
            const int s = rslot_of(z);
            return pmk(stage->raw[s][2 * q + 1][row][lane], stage->raw[s][2 * q + 2][row][lane]);
        } else if constexpr (use16) {
            const int s = rslot_of(z);
            return pmk(to_float(stage16->raw[s][2 * q + 1][row][lane + 1]),
                       to_float(stage16->raw[s][2 * q + 2][row][lane + 1]));
        } else {
            const size_t o = (size_t)zwrap(z) * nn + colidx;
            if (!KIN_CHECK(o + (2 * q + 2) * plane < Q * plane, DBG_DUGKS_LOAD, o + (2 * q + 2) * plane))
                return pmk(C(0), C(0));
            return pmk(Traits<S>::load(src + o + (2 * q + 1) * plane), Traits<S>::load(src + o + (2 * q + 2) * plane));
        }
    };
    auto raw_rest = [&](int z) -> C {
        if constexpr (kAsyncStage<S>) {
            return stage->raw[rslot_of(z)][0][row][lane];
        } else if constexpr (use16) {
            return to_float(stage16->raw[rslot_of(z)][0][row][lane + 1]);
        } else {
            const size_t o = (size_t)zwrap(z) * nn + colidx;
            if (!KIN_CHECK(o < plane, DBG_DUGKS_LOAD, o)) return C(0);
            return Traits<S>::load(src + o);
        }
    };

    // Eq. 19 for this thread's column at plane z into ring slot s:
    // fbp = f + b (f_eq - f), f_eq of a pair = q +/- l (Eq. 7).
    auto prestep = [&](int z, int s) {
        P2 f[NPAIR];
#pragma unroll
        for (int q = 0; q < NPAIR; ++q) f[q] = raw_pair(z, q);
        const C f0 = raw_rest(z);
        C a[NPAIR], b[NPAIR];
#pragma unroll
        for (int q = 0; q < NPAIR; ++q) {
            a[q] = f[q].x + f[q].y;
            b[q] = f[q].x - f[q].y;
        }
        const C drho = f0 + (((a[0] + a[1]) + a[2]) + (((a[3] + a[4]) + (a[5] + a[6])) + (a[7] + a[8])));
        const C jx = (b[0] + b[3]) + (b[4] + (b[5] + b[6]));
        const C jy = (b[1] + b[3]) - (b[4] - (b[7] + b[8]));
        const C jz = (b[2] + b[5]) - (b[6] - (b[7] - b[8]));
        const C a0 = fma(C(-1.5), fma(jz, jz, fma(jy, jy, jx * jx)), drho);
        const C wa_ax = (C(2) / C(36)) * a0, wa_dg = (C(1) / C(36)) * a0;
        static_for<0, NPAIR>([&](auto pc) {
            constexpr int PP = decltype(pc)::value;
            constexpr bool AX = PP < 3;
            const C sd = pdot<PP>(jx, jy, jz);
            // W (a0 + 9/2 s^2) with 9/2 W = 1/4 (axis) or 1/8 (diagonal)
            const C q = fma(C(AX ? 0.25 : 0.125) * sd, sd, AX ? wa_ax : wa_dg);
            const C l = lin3w<C>(AX ? 1 : 2) * sd;
            sm.ring[s][PP][row][lane] = pfma(kc.b2, psub(pmk(q + l, q - l), f[PP]), f[PP]);
        });
        sm.ring0[s][row][lane] = fma(kc.b, (C(12) / C(36)) * a0 - f0, f0);
    };

    // Cell view at ring slot s0 with the tangential differences in MASK.
    auto gather = [&](int s0, int sm1, int sp1, auto maskc, CellView<C>& v) {
        constexpr int MASK = decltype(maskc)::value;
#pragma unroll
        for (int q = 0; q < NPAIR; ++q) v.X[q] = sm.ring[s0][q][row][lane];
        v.X0 = sm.ring0[s0][row][lane];
        static_for<0, 3>([&](auto tc) {
            constexpr int T = decltype(tc)::value;
            if constexpr ((MASK >> T) & 1) {
                static_for<0, NC>([&](auto kc2) {
                    constexpr int K = decltype(kc2)::value;
                    constexpr int p = cross_pair(T, K);
                    if constexpr (T == 0) {
                        v.G[0][K] = psub(sm.ring[s0][p][row][lp], sm.ring[s0][p][row][lm]);
                    } else if constexpr (T == 1) {
                        if (KIN_CHECK(row >= 1 && row <= TY, DBG_DUGKS_ROW, row))
                            v.G[1][K] = psub(sm.ring[s0][p][row + 1][lane], sm.ring[s0][p][row - 1][lane]);
                    } else {
                        v.G[2][K] = psub(sm.ring[sp1][p][row][lane], sm.ring[sm1][p][row][lane]);
                    }
                });
            }
        });
        view_moments(v);
        view_diffs<MASK>(v);
    };

    // ring slots of planes z - 1, z, z + 1 (rotated every plane)
    int s_m1 = 2, s_0 = 0, s_p1 = 1;

    // Copies become visible to every thread by the issuer's wait followed by a
    // block barrier: the copies of plane z + 2, issued right after the first
    // barrier of plane z, are waited for at the end of plane z.
    constexpr bool staged = kAsyncStage<S> || use16;
    if constexpr (staged) {
        if (issuer) {
            issue_plane(z0 - 1);
            issue_plane(z0);
            if (z0 + 1 <= zend) issue_plane(z0 + 1);
            cp_async_wait_all();
        }
        __syncthreads();
    }
    prestep(z0 - 1, s_m1);
    prestep(z0, s_0);
    __syncthreads();

    Rec<C> Pz;        // P^z record of the plane below the current one
    P2 Dprev[NPAIR];  // sign-folded flux sums of plane z - 1, still missing its +z face
    P2 Dcur[NPAIR];
#pragma unroll
    for (int q = 0; q < NPAIR; ++q) {
        Dprev[q] = pmk(C(0), C(0));
        Dcur[q] = pmk(C(0), C(0));
    }
    if (interior) {
        CellView<C> v;
        Rec<C> unused;
        gather(s_m1, s_m1, s_m1, std::integral_constant<int, 3>{}, v);
        side_records<2, true, false>(v, kc, Pz, unused);
    }

    for (int z = z0; z <= zend; ++z) {
        const bool last = z == zend;
        if (!KIN_CHECK(s_m1 >= 0 && s_m1 < 3 && s_0 >= 0 && s_0 < 3 && s_p1 >= 0 && s_p1 < 3, DBG_DUGKS_SLOT,
                       s_m1 * 100 + s_0 * 10 + s_p1))
            break;
        __syncthreads();  // fy of plane z - 1 complete; my of plane z - 1 consumed
        Rec<C> Py;
        if (!last) {
            prestep(z + 1, s_p1);
            if constexpr (staged) {
                if (issuer && z + 2 <= zend) issue_plane(z + 2);
            }
            CellView<C> v;
            // warp-uniform: rows 1..TY take every difference, the halo rows
            // only those their y records need
            if (yin) {
                gather(s_0, s_m1, s_p1, std::integral_constant<int, 7>{}, v);
            } else {
                gather(s_0, s_m1, s_p1, std::integral_constant<int, 5>{}, v);  // G^x, G^z
            }
            if (yin) {
                // x faces: this lane's face to the right uses the next lane's M record
                Rec<C> Px, Mx, Mn;
                side_records<0, true, true>(v, kc, Px, Mx);
#pragma unroll
                for (int k = 0; k < NC; ++k) Mn.r[k] = pshfl_down1<C>(Mx.r[k]);
#pragma unroll
                for (int m = 0; m < 4; ++m) Mn.m[m] = __shfl_down_sync(0xffffffffu, Mx.m[m], 1);
                P2 ffx[NC];
                face_values<0>(Px, Mn, kc, ffx);
                static_for<0, NC>([&](auto kc2) {
                    constexpr int K = decltype(kc2)::value;
                    constexpr int p = cross_pair(0, K);
                    const P2 fl = pshfl_up1<C>(ffx[K]);
                    // Dhat = e_px (F(x + 1/2) - F(x - 1/2)), the first contribution
                    Dcur[p] = pe(p, 0) > 0 ? psub(ffx[K], fl) : psub(fl, ffx[K]);
                });
            }
            if (xin) {
                Rec<C> My;
                side_records<1, true, true>(v, kc, Py, My);
#pragma unroll
                for (int k = 0; k < NC; ++k) sm.my[k][row][lane] = My.r[k];
#pragma unroll
                for (int m = 0; m < 4; ++m) sm.mym[m][row][lane] = My.m[m];
            }
            if (interior) {
                // z face (z - 1, z): P^z(z - 1) carried, M^z(z) from this view
                Rec<C> Pn, Mz;
                side_records<2, true, true>(v, kc, Pn, Mz);
                P2 ffz[NC];
                face_values<2>(Pz, Mz, kc, ffz);
                static_for<0, NC>([&](auto kc2) {
                    constexpr int K = decltype(kc2)::value;
                    constexpr int p = cross_pair(2, K);
                    constexpr int sg = pe(p, 2);
                    Dprev[p] = padd_sg<sg>(Dprev[p], ffz[K]);
                    if constexpr (pe(p, 0) != 0) {
                        Dcur[p] = padd_sg<-sg>(Dcur[p], ffz[K]);
                    } else {
                        Dcur[p] = sg > 0 ? pneg(ffz[K]) : ffz[K];
                    }
                });
                Pz = Pn;
            }
        } else if (interior) {
            CellView<C> v;
            Rec<C> unused, Mz;
            gather(s_0, s_0, s_0, std::integral_constant<int, 3>{}, v);
            side_records<2, false, true>(v, kc, unused, Mz);
            P2 ffz[NC];
            face_values<2>(Pz, Mz, kc, ffz);
            static_for<0, NC>([&](auto kc2) {
                constexpr int K = decltype(kc2)::value;
                constexpr int p = cross_pair(2, K);
                Dprev[p] = padd_sg<pe(p, 2)>(Dprev[p], ffz[K]);
            });
        }
        // update plane z - 1 (Eqs. 20, 9): its y faces were computed one iteration ago
        if (z > z0 && interior) {
            static_for<0, NC>([&](auto kc2) {
                constexpr int K = decltype(kc2)::value;
                constexpr int p = cross_pair(1, K);
                constexpr int sg = pe(p, 1);
                const P2 dy = psub(sm.fy[K][row][lane], sm.fy[K][row - 1][lane]);
                if constexpr (pe(p, 0) != 0 || pe(p, 2) != 0) {
                    Dprev[p] = padd_sg<sg>(Dprev[p], dy);
                } else {
                    Dprev[p] = sg > 0 ? dy : pneg(dy);
                }
            });
            if (valid && KIN_CHECK((size_t)(z - 1) * nn + colidx < plane, DBG_DUGKS_STORE,
                                   (size_t)(z - 1) * nn + colidx)) {
                const size_t c = (size_t)(z - 1) * nn + colidx;
                [[maybe_unused]] C uv[3] = {C(0), C(0), C(0)};
                // velocity sums in population order: the same additions as the
                // separate velocity pass over the stored state
                [[maybe_unused]] auto vel_add = [&](auto ic, C v) {
                    constexpr int I = decltype(ic)::value;
                    if constexpr (cx(I) > 0) uv[0] += v;
                    if constexpr (cx(I) < 0) uv[0] -= v;
                    if constexpr (cy(I) > 0) uv[1] += v;
                    if constexpr (cy(I) < 0) uv[1] -= v;
                    if constexpr (cz(I) > 0) uv[2] += v;
                    if constexpr (cz(I) < 0) uv[2] -= v;
                };
                static_for<0, NPAIR>([&](auto pc) {
                    constexpr int PP = decltype(pc)::value;
                    const P2 xb = sm.ring[s_m1][PP][row][lane];
                    // f-tilde-plus = 4/3 fbp - 1/3 f-tilde (Eq. 20), minus dt times the flux sum (Eq. 9)
                    const P2 t = pfma(kc.third, psub(xb, raw_pair(z - 1, PP)), xb);
                    const P2 o = pfma(kc.dts, Dprev[PP], t);
                    // both members rounded by one paired conversion for 2-byte storage
                    [[maybe_unused]] const P2 r =
                        Traits<S>::store2(dst + (2 * PP + 1) * plane + c, dst + (2 * PP + 2) * plane + c, o);
                    if constexpr (VEL) {
                        vel_add(std::integral_constant<int, 2 * PP + 1>{}, r.x);
                        vel_add(std::integral_constant<int, 2 * PP + 2>{}, r.y);
                    }
                });
                const C xb0 = sm.ring0[s_m1][row][lane];
                Traits<S>::store(dst + c, fma(C(1.0 / 3.0), xb0 - raw_rest(z - 1), xb0));
                if constexpr (VEL) {
                    uvel[c] = uv[0];
                    uvel[plane + c] = uv[1];
                    uvel[2 * plane + c] = uv[2];
                }
            }
        }
        __syncthreads();  // my of plane z complete; fy of plane z - 1 consumed
        if (!last && xin && row <= TY) {
            // y faces of plane z: face r between rows r and r + 1, r = 0..TY
            Rec<C> Mu;
#pragma unroll
            for (int k = 0; k < NC; ++k) Mu.r[k] = sm.my[k][row + 1][lane];
#pragma unroll
            for (int m = 0; m < 4; ++m) Mu.m[m] = sm.mym[m][row + 1][lane];
            P2 ffy[NC];
            face_values<1>(Py, Mu, kc, ffy);
#pragma unroll
            for (int k = 0; k < NC; ++k) sm.fy[k][row][lane] = ffy[k];
        }
        if constexpr (staged) {
            if (issuer) cp_async_wait_all();  // plane z + 2, published by the next barrier
        }
#pragma unroll
        for (int q = 0; q < NPAIR; ++q) Dprev[q] = Dcur[q];
        const int st = s_m1;
        s_m1 = s_0;
        s_0 = s_p1;
        s_p1 = st;
    }
}

// Coefficients of Eqs. 18-19 for viscosity nu (tau = nu / RT) and step dt,
// with the derived constants of the fused tile.
template <typename C>
inline DugksCoef<C> dugks_coef(double nu, double dt) {
    const double tau = 3.0 * nu, h = 0.5 * dt;
    DugksCoef<C> k{};
    k.a = C((2.0 * tau - h) / (2.0 * tau + dt));
    k.b = C(3.0 * h / (2.0 * tau + dt));
    k.h = C(h);
    k.c1 = C(2.0 * tau / (2.0 * tau + h));
    k.c2 = C(h / (2.0 * tau + h));
    k.dt = C(dt);
    k.hq = C(0.25 * h);
    const C c2 = k.c2;
    k.qk[0] = c2 * C(0.25);
    k.qk[1] = c2 * C(0.125);
    k.qw[0] = c2 * (C(2) / C(36));
    k.qw[1] = c2 * (C(1) / C(36));
    k.ql[0] = c2 * lin3w<C>(1);
    k.ql[1] = c2 * lin3w<C>(2);
    k.cpp = pmk(C(0.5 + h), C(0.5 - h));
    k.cpm = pmk(C(0.5 - h), C(0.5 + h));
    k.hqp = pmk(-k.hq, k.hq);
    k.hqm = pmk(k.hq, -k.hq);
    k.b2 = pmk(k.b, k.b);
    const C c1 = C(1) - c2;
    k.c1p = pmk(c1, c1);
    k.third = pmk(C(1.0 / 3.0), C(1.0 / 3.0));
    k.dts = pmk(-k.dt, k.dt);
    return k;
}

}  // namespace kin
