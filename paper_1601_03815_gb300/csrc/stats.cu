// Statistics and state conversion kernels.
//
//   velocity_kernel        u = sum xi_i f_i (Eq. 8 / Eq. 12), FP64 out
//   velocity32_kernel      the same in FP32, for storage types computed in FP32
//   ed_partial_kernel      per-block FP64 sums of |u|^2 and s_ab s_ab
//   ed32_partial_kernel    the same from FP32 u: per-cell terms in FP32,
//                          per-thread and block sums in FP64
//   ed_final_kernel        fixed-order sum of the block partials -> {E, eps}
//   shell_partial_kernel   per-block shell sums of |u_hat|^2 / 2 (Eq. 27)
//   shell_final_kernel     fixed-order sum over blocks
// Every reduction runs in a fixed order for a given N, so results are
// bitwise reproducible.
#include "kin.h"
#include "kin_common.cuh"
#include "kin_internal.h"
#include "kin_sim.h"

#include <cufft.h>

#include <mutex>

namespace kin {

size_t storage_bytes(int storage) {
    switch (storage) {
        case ST_F32: return 4;
        case ST_F16: return 2;
        case ST_BF16: return 2;
        case ST_F64: return 8;
    }
    return 0;
}

// Canonical cell index of the stored element of population I for node x: the
// LBE pull layout stores f_i(x) at x - xi_i.
template <int I>
__device__ __forceinline__ int stored_index(int x, int y, int z, int N, bool shifted) {
    if (!shifted) return x + N * (y + N * z);
    int xs = x - cx(I), ys = y - cy(I), zs = z - cz(I);
    xs = xs < 0 ? xs + N : (xs >= N ? xs - N : xs);
    ys = ys < 0 ? ys + N : (ys >= N ? ys - N : ys);
    zs = zs < 0 ? zs + N : (zs >= N ? zs - N : zs);
    return xs + N * (ys + N * zs);
}

__device__ __forceinline__ int stored_index_rt(int i, int x, int y, int z, int N, bool shifted) {
    if (!shifted) return x + N * (y + N * z);
    int xs = x - cx(i), ys = y - cy(i), zs = z - cz(i);
    xs = xs < 0 ? xs + N : (xs >= N ? xs - N : xs);
    ys = ys < 0 ? ys + N : (ys >= N ? ys - N : ys);
    zs = zs < 0 ? zs + N : (zs >= N ? zs - N : zs);
    return xs + N * (ys + N * zs);
}

template <typename S>
__global__ void velocity_kernel(const S* __restrict__ st, bool shifted, int N, size_t plane,
                                double* __restrict__ u) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= N) return;
    const int y = blockIdx.y, z = blockIdx.z;
    double jx = 0.0, jy = 0.0, jz = 0.0;
    static_for<0, Q>([&](auto ic) {
        constexpr int I = decltype(ic)::value;
        const double v = (double)Traits<S>::load(st + I * plane + stored_index<I>(x, y, z, N, shifted));
        if constexpr (cx(I) != 0) jx += cx(I) * v;
        if constexpr (cy(I) != 0) jy += cy(I) * v;
        if constexpr (cz(I) != 0) jz += cz(I) * v;
    });
    const size_t c = (size_t)x + (size_t)N * (y + (size_t)N * z);
    u[c] = jx;
    u[plane + c] = jy;
    u[2 * plane + c] = jz;
}

// FP32 storage, FP32 arithmetic: u in FP32 (the per-cell sums of 19 terms
// carry the storage's own rounding; the FP64 path above serves FP64 storage).
template <typename S>
__global__ void velocity32_kernel(const S* __restrict__ st, bool shifted, int N, size_t plane,
                                  float* __restrict__ u) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= N) return;
    const int y = blockIdx.y, z = blockIdx.z;
    float j[3] = {0.0f, 0.0f, 0.0f};
    static_for<0, Q>([&](auto ic) {
        constexpr int I = decltype(ic)::value;
        const float v = (float)Traits<S>::load(st + I * plane + stored_index<I>(x, y, z, N, shifted));
        if constexpr (cx(I) > 0) j[0] += v;
        if constexpr (cx(I) < 0) j[0] -= v;
        if constexpr (cy(I) > 0) j[1] += v;
        if constexpr (cy(I) < 0) j[1] -= v;
        if constexpr (cz(I) > 0) j[2] += v;
        if constexpr (cz(I) < 0) j[2] -= v;
    });
    const size_t c = (size_t)x + (size_t)N * (y + (size_t)N * z);
    u[c] = j[0];
    u[plane + c] = j[1];
    u[2 * plane + c] = j[2];
}

constexpr int RED_THREADS = 256;

int stats_blocks(int N) {
    long long n = (long long)N * N * N;
    long long b = (n + RED_THREADS * 8 - 1) / (RED_THREADS * 8);
    if (b > kStatsMaxBlocks) b = kStatsMaxBlocks;
    if (b < 1) b = 1;
    return (int)b;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Block-then-warp reduction of |u|^2 and s_ab s_ab; each thread walks a fixed
// grid-stride sequence of cells.
__global__ void __launch_bounds__(RED_THREADS)
    ed_partial_kernel(const double* __restrict__ u, int N, double* __restrict__ partial) {
    const size_t n = (size_t)N * N * N;
    double se = 0.0, ss = 0.0;
    for (size_t c = (size_t)blockIdx.x * RED_THREADS + threadIdx.x; c < n;
         c += (size_t)gridDim.x * RED_THREADS) {
        const int x = (int)(c % N), y = (int)((c / N) % N), z = (int)(c / ((size_t)N * N));
        const size_t nb[3][2] = {
            {(size_t)wrap_inc(x, N) + (size_t)N * (y + (size_t)N * z),
             (size_t)wrap_dec(x, N) + (size_t)N * (y + (size_t)N * z)},
            {(size_t)x + (size_t)N * (wrap_inc(y, N) + (size_t)N * z),
             (size_t)x + (size_t)N * (wrap_dec(y, N) + (size_t)N * z)},
            {(size_t)x + (size_t)N * (y + (size_t)N * wrap_inc(z, N)),
             (size_t)x + (size_t)N * (y + (size_t)N * wrap_dec(z, N))}};
        double g[3][3];
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) g[a][b] = 0.5 * (u[b * n + nb[a][0]] - u[b * n + nb[a][1]]);
        double s2 = 0.0;
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                const double sab = 0.5 * (g[a][b] + g[b][a]);
                s2 += sab * sab;
            }
        ss += s2;
        se += u[c] * u[c] + u[n + c] * u[n + c] + u[2 * n + c] * u[2 * n + c];
    }
    __shared__ double sh[2][RED_THREADS / 32];
    se = warp_sum(se);
    ss = warp_sum(ss);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        sh[0][wid] = se;
        sh[1][wid] = ss;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < RED_THREADS / 32; ++w) {
            a += sh[0][w];
            b += sh[1][w];
        }
        partial[2 * blockIdx.x] = a;
        partial[2 * blockIdx.x + 1] = b;
    }
}

// FP32 counterpart of ed_partial_kernel: block b takes the rows (y, z) =
// b, b + gridDim.x, ... and its threads the cells of a row; the per-cell
// |u|^2 and s_ab s_ab are formed in FP32, summed in FP32 over at most 8 rows
// and then in FP64, in a fixed order.
__global__ void __launch_bounds__(RED_THREADS)
    ed32_partial_kernel(const float* __restrict__ u, int N, double* __restrict__ partial) {
    const size_t n = (size_t)N * N * N;
    // component bases; offsets inside a component fit in 32 bits (N <= 1024)
    const float* __restrict__ U[3] = {u, u + n, u + 2 * n};
    double se = 0.0, ss = 0.0;
    float fe = 0.0f, fs = 0.0f;
    int rows_in_chunk = 0;
    for (int r = blockIdx.x; r < N * N; r += gridDim.x) {
        if (rows_in_chunk == 8) {
            se += (double)fe;
            ss += (double)fs;
            fe = fs = 0.0f;
            rows_in_chunk = 0;
        }
        ++rows_in_chunk;
        const int y = r % N, z = r / N;
        const int row = N * r;
        const int rows[3][2] = {{row, row},
                                {N * (wrap_inc(y, N) + N * z), N * (wrap_dec(y, N) + N * z)},
                                {N * (y + N * wrap_inc(z, N)), N * (y + N * wrap_dec(z, N))}};
        for (int x = threadIdx.x; x < N; x += RED_THREADS) {
            const int xs[3][2] = {{wrap_inc(x, N), wrap_dec(x, N)}, {x, x}, {x, x}};
            float g[3][3];  // g[a][b] = d u_b / d x_a, central differences
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int b = 0; b < 3; ++b)
                    g[a][b] = 0.5f * (__ldg(U[b] + rows[a][0] + xs[a][0]) - __ldg(U[b] + rows[a][1] + xs[a][1]));
            float s2 = 0.0f;
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int b = 0; b < 3; ++b) {
                    const float sab = 0.5f * (g[a][b] + g[b][a]);
                    s2 += sab * sab;
                }
            const float u0 = __ldg(U[0] + row + x), u1 = __ldg(U[1] + row + x), u2 = __ldg(U[2] + row + x);
            fe += u0 * u0 + u1 * u1 + u2 * u2;
            fs += s2;
        }
    }
    se += (double)fe;
    ss += (double)fs;
    __shared__ double sh[2][RED_THREADS / 32];
    se = warp_sum(se);
    ss = warp_sum(ss);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        sh[0][wid] = se;
        sh[1][wid] = ss;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < RED_THREADS / 32; ++w) {
            a += sh[0][w];
            b += sh[1][w];
        }
        partial[2 * blockIdx.x] = a;
        partial[2 * blockIdx.x + 1] = b;
    }
}

// The same for N a multiple of 4, four cells per thread: a thread reads its
// four cells and their y and z neighbours as float4 and the two outer x
// neighbours as scalars, which cuts the load instructions fourfold.  Block b
// takes groups of rpi = RED_THREADS / (N/4) rows, b, b + gridDim.x, ...; the
// terms of a thread's cells are summed in cell order, in FP32 over at most 8
// row groups and then in FP64.
__global__ void __launch_bounds__(RED_THREADS)
    ed32v4_partial_kernel(const float* __restrict__ u, int N, double* __restrict__ partial) {
    const size_t n = (size_t)N * N * N;
    const float* __restrict__ U[3] = {u, u + n, u + 2 * n};
    const int gpr = N / 4, rpi = RED_THREADS / gpr;
    const int rsub = threadIdx.x / gpr, x = 4 * (threadIdx.x % gpr);
    const bool active = rsub < rpi;
    const int xm = (x == 0 ? N : x) - 1, xp = x + 4 == N ? 0 : x + 4;
    double se = 0.0, ss = 0.0;
    float fe = 0.0f, fs = 0.0f;
    int groups_in_chunk = 0;
    const int nrows = N * N;
    for (int rg = blockIdx.x; rg * rpi < nrows; rg += gridDim.x) {
        if (groups_in_chunk == 8) {
            se += (double)fe;
            ss += (double)fs;
            fe = fs = 0.0f;
            groups_in_chunk = 0;
        }
        ++groups_in_chunk;
        const int r = rg * rpi + rsub;
        if (!active || r >= nrows) continue;
        const int y = r % N, z = r / N;
        const int row = N * r;
        const int ryp = N * (wrap_inc(y, N) + N * z), rym = N * (wrap_dec(y, N) + N * z);
        const int rzp = N * (y + N * wrap_inc(z, N)), rzm = N * (y + N * wrap_dec(z, N));
        float g[4][3][3];  // g[cell][a][b] = d u_b / d x_a
        float c[4][3];
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const float4 cc = __ldg(reinterpret_cast<const float4*>(U[b] + row + x));
            const float4 yp = __ldg(reinterpret_cast<const float4*>(U[b] + ryp + x));
            const float4 ym = __ldg(reinterpret_cast<const float4*>(U[b] + rym + x));
            const float4 zp = __ldg(reinterpret_cast<const float4*>(U[b] + rzp + x));
            const float4 zm = __ldg(reinterpret_cast<const float4*>(U[b] + rzm + x));
            const float l = __ldg(U[b] + row + xm), rr = __ldg(U[b] + row + xp);
            g[0][0][b] = 0.5f * (cc.y - l);
            g[1][0][b] = 0.5f * (cc.z - cc.x);
            g[2][0][b] = 0.5f * (cc.w - cc.y);
            g[3][0][b] = 0.5f * (rr - cc.z);
            g[0][1][b] = 0.5f * (yp.x - ym.x);
            g[1][1][b] = 0.5f * (yp.y - ym.y);
            g[2][1][b] = 0.5f * (yp.z - ym.z);
            g[3][1][b] = 0.5f * (yp.w - ym.w);
            g[0][2][b] = 0.5f * (zp.x - zm.x);
            g[1][2][b] = 0.5f * (zp.y - zm.y);
            g[2][2][b] = 0.5f * (zp.z - zm.z);
            g[3][2][b] = 0.5f * (zp.w - zm.w);
            c[0][b] = cc.x;
            c[1][b] = cc.y;
            c[2][b] = cc.z;
            c[3][b] = cc.w;
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            float s2 = 0.0f;
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int b = 0; b < 3; ++b) {
                    const float sab = 0.5f * (g[j][a][b] + g[j][b][a]);
                    s2 += sab * sab;
                }
            fe += c[j][0] * c[j][0] + c[j][1] * c[j][1] + c[j][2] * c[j][2];
            fs += s2;
        }
    }
    se += (double)fe;
    ss += (double)fs;
    __shared__ double sh[2][RED_THREADS / 32];
    se = warp_sum(se);
    ss = warp_sum(ss);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        sh[0][wid] = se;
        sh[1][wid] = ss;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < RED_THREADS / 32; ++w) {
            a += sh[0][w];
            b += sh[1][w];
        }
        partial[2 * blockIdx.x] = a;
        partial[2 * blockIdx.x + 1] = b;
    }
}

// One block of FIN_THREADS: thread t sums partials t, t + FIN_THREADS, ... in
// order, then the warps and the block reduce in a fixed order.
constexpr int FIN_THREADS = 256;
__global__ void __launch_bounds__(FIN_THREADS)
    ed_final_kernel(const double* __restrict__ partial, int nblocks, size_t n, double nu,
                    double* __restrict__ out) {
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < nblocks; i += FIN_THREADS) {
        a += partial[2 * i];
        b += partial[2 * i + 1];
    }
    a = warp_sum(a);
    b = warp_sum(b);
    __shared__ double sh[2][FIN_THREADS / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        sh[0][wid] = a;
        sh[1][wid] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double ta = 0.0, tb = 0.0;
        for (int w = 0; w < FIN_THREADS / 32; ++w) {
            ta += sh[0][w];
            tb += sh[1][w];
        }
        out[0] = 0.5 * ta / (double)n;
        out[1] = 2.0 * nu * tb / (double)n;
    }
}

cudaError_t energy_dissipation(const double* u, int N, double nu, double* partials, double* out,
                               cudaStream_t stream) {
    const int nb = stats_blocks(N);
    ed_partial_kernel<<<nb, RED_THREADS, 0, stream>>>(u, N, partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    ed_final_kernel<<<1, FIN_THREADS, 0, stream>>>(partials, nb, (size_t)N * N * N, nu, out);
    return cudaGetLastError();
}

cudaError_t energy_dissipation32(const float* u, int N, double nu, double* partials, double* out,
                                 cudaStream_t stream) {
    const int nb = stats_blocks(N);
    if (N % 4 == 0 && N / 4 <= RED_THREADS)
        ed32v4_partial_kernel<<<nb, RED_THREADS, 0, stream>>>(u, N, partials);
    else
        ed32_partial_kernel<<<nb, RED_THREADS, 0, stream>>>(u, N, partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    ed_final_kernel<<<1, FIN_THREADS, 0, stream>>>(partials, nb, (size_t)N * N * N, nu, out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Spectrum shells.  Modes of the half-complex layout [kz][ky][kx],
// kx = 0..N/2; a mode with 0 < kx < N/2 also stands for its conjugate.
// Lanes of a warp that fall in the same shell are summed in lane order by the
// lowest lane, which adds the result to a warp-private shell array; the block
// then adds its warps' arrays in warp order.
constexpr int SPEC_THREADS = 256;

int spectrum_blocks(int N) {
    long long n = (long long)N * N * (N / 2 + 1);
    long long b = (n + SPEC_THREADS * 16 - 1) / (SPEC_THREADS * 16);
    if (b > 304) b = 304;
    if (b < 1) b = 1;
    return (int)b;
}

// CT: double2 (FP64 transform) or float2 (FP32 transform, |u_hat|^2 formed
// in FP32 and summed in FP64).
template <typename CT>
__global__ void __launch_bounds__(SPEC_THREADS)
    shell_partial_kernel(const CT* __restrict__ u0, const CT* __restrict__ u1,
                         const CT* __restrict__ u2, int N, int nshell, double inv,
                         int weight_n2, double* __restrict__ partial) {
    extern __shared__ double bins[];  // [SPEC_THREADS/32][nshell]
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    double* mybins = bins + wid * nshell;
    for (int s = lane; s < nshell; s += 32) mybins[s] = 0.0;
    __syncwarp();
    __shared__ double xch[SPEC_THREADS];  // lane values for the shell sums
    const int nh = N / 2 + 1;
    const int nmode = N * N * nh;  // < 2^31 for N <= 1024
    // each warp handles consecutive chunks of 32 modes
    const int nwarps = gridDim.x * (SPEC_THREADS / 32);
    const int gw = blockIdx.x * (SPEC_THREADS / 32) + wid;
    for (int base = gw * 32; base < nmode; base += nwarps * 32) {
        const int m = base + lane;
        int shell = -1;
        double e = 0.0;
        if (m < nmode) {
            const int kx = m % nh, t = m / nh;
            const int ky = t % N, kz = t / N;
            const int sy = ky > N / 2 ? ky - N : ky;
            const int sz = kz > N / 2 ? kz - N : kz;
            const int n2 = kx * kx + sy * sy + sz * sz;  // < 2^24: exact in FP32
            // nearest integer to |n|; |n| is never within FP32 rounding of a half-integer
            shell = (int)floorf(sqrtf((float)n2) + 0.5f);
            const CT a = u0[m], b = u1[m], c = u2[m];
            const double amp = (double)((a.x * a.x + a.y * a.y) + (b.x * b.x + b.y * b.y) + (c.x * c.x + c.y * c.y));
            const double w = (kx > 0 && 2 * kx < N) ? 2.0 : 1.0;
            e = 0.5 * amp * inv * inv * w;
            if (weight_n2) e *= (double)n2;
        }
        const unsigned same = __match_any_sync(0xffffffffu, shell);
        const int leader = __ffs(same) - 1;
        xch[threadIdx.x] = e;
        __syncwarp();
        if (lane == leader && shell >= 0 && shell < nshell) {
            // the lanes of this shell in lane order
            double acc = 0.0;
            for (unsigned msk = same; msk; msk &= msk - 1) acc += xch[wid * 32 + __ffs(msk) - 1];
            mybins[shell] += acc;
        }
        __syncwarp();
    }
    __syncthreads();
    for (int s = threadIdx.x; s < nshell; s += SPEC_THREADS) {
        double a = 0.0;
        for (int w = 0; w < SPEC_THREADS / 32; ++w) a += bins[w * nshell + s];
        partial[(size_t)blockIdx.x * nshell + s] = a;
    }
}

__global__ void shell_final_kernel(const double* __restrict__ partial, int nblocks, int nshell,
                                   double* __restrict__ out) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nshell) return;
    double a = 0.0;
    for (int b = 0; b < nblocks; ++b) a += partial[(size_t)b * nshell + s];
    out[s] = a;
}

// ---------------------------------------------------------------------------
// Spectral derivative d_a u_a of one component: u_hat (half-complex, unscaled
// D2Z output) times i k_a / N^3, the Nyquist wavenumber of axis a set to zero;
// the Z2D of the result is the derivative field.
__global__ void deriv_mult_kernel(double2* __restrict__ uh, int N, int axis) {
    const int nh = N / 2 + 1;
    const int kx = blockIdx.x * blockDim.x + threadIdx.x;
    if (kx >= nh) return;
    const int ky = blockIdx.y, kz = blockIdx.z;
    const size_t m = (size_t)kx + (size_t)nh * (ky + (size_t)N * kz);
    int n = axis == 0 ? kx : axis == 1 ? ky : kz;
    if (axis != 0 && n > N / 2) n -= N;
    const bool nyquist = (N % 2 == 0) && (n == N / 2 || n == -N / 2);
    const double inv = 1.0 / ((double)N * N * N);
    const double k = nyquist ? 0.0 : 2.0 * 3.14159265358979323846 * n / N * inv;
    const double2 v = uh[m];
    uh[m] = make_double2(-k * v.y, k * v.x);
}

constexpr int MOM_THREADS = 256;

// Block partials of sum d^2, d^3, d^4 for the three derivative fields d_a
// (fixed grid-stride order, then warp and block order): partial[9 b + 3 a + p].
__global__ void __launch_bounds__(MOM_THREADS)
    deriv_moments_kernel(const double* __restrict__ d, int N, double* __restrict__ partial) {
    const size_t n = (size_t)N * N * N;
    double acc[9];
#pragma unroll
    for (int j = 0; j < 9; ++j) acc[j] = 0.0;
    for (size_t c = (size_t)blockIdx.x * MOM_THREADS + threadIdx.x; c < n; c += (size_t)gridDim.x * MOM_THREADS) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const double v = d[a * n + c], v2 = v * v;
            acc[3 * a] += v2;
            acc[3 * a + 1] += v2 * v;
            acc[3 * a + 2] += v2 * v2;
        }
    }
    __shared__ double sh[9][MOM_THREADS / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < 9; ++j) {
        const double w = warp_sum(acc[j]);
        if (lane == 0) sh[j][wid] = w;
    }
    __syncthreads();
    if (threadIdx.x < 9) {
        double t = 0.0;
        for (int w = 0; w < MOM_THREADS / 32; ++w) t += sh[threadIdx.x][w];
        partial[9 * (size_t)blockIdx.x + threadIdx.x] = t;
    }
}

__global__ void deriv_moments_final_kernel(const double* __restrict__ partial, int nblocks, size_t n,
                                           double* __restrict__ out) {
    const int j = threadIdx.x;
    if (j >= 9) return;
    double t = 0.0;
    for (int b = 0; b < nblocks; ++b) t += partial[9 * (size_t)b + j];
    out[j] = t / (double)n;
}

int deriv_moment_blocks(int N) {
    long long n = (long long)N * N * N;
    long long b = (n + MOM_THREADS * 16 - 1) / (MOM_THREADS * 16);
    if (b > 608) b = 608;
    if (b < 1) b = 1;
    return (int)b;
}

cudaError_t derivative_multiply(double2* uh, int N, int axis, cudaStream_t stream) {
    const int nh = N / 2 + 1;
    const int bx = nh < 128 ? ((nh + 31) / 32) * 32 : 128;
    dim3 g((nh + bx - 1) / bx, N, N);
    deriv_mult_kernel<<<g, bx, 0, stream>>>(uh, N, axis);
    return cudaGetLastError();
}

cudaError_t derivative_moments(const double* d, int N, double* partial, double* out, cudaStream_t stream) {
    const int nb = deriv_moment_blocks(N);
    deriv_moments_kernel<<<nb, MOM_THREADS, 0, stream>>>(d, N, partial);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    deriv_moments_final_kernel<<<1, 32, 0, stream>>>(partial, nb, (size_t)N * N * N, out);
    return cudaGetLastError();
}

template <typename CT>
static cudaError_t spectrum_shells_t(const void* uh0, const void* uh1, const void* uh2, int N, int nshell,
                                     double inv, int weight_n2, double* partial, double* out,
                                     cudaStream_t stream) {
    const int nb = spectrum_blocks(N);
    const size_t smem = sizeof(double) * nshell * (SPEC_THREADS / 32);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(shell_partial_kernel<CT>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    shell_partial_kernel<CT><<<nb, SPEC_THREADS, smem, stream>>>(
        (const CT*)uh0, (const CT*)uh1, (const CT*)uh2, N, nshell, inv, weight_n2, partial);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    shell_final_kernel<<<(nshell + 127) / 128, 128, 0, stream>>>(partial, nb, nshell, out);
    return cudaGetLastError();
}

cudaError_t spectrum_shells(const void* uh0, const void* uh1, const void* uh2, int N, int nshell,
                            double inv, int weight_n2, double* partial, double* out,
                            cudaStream_t stream) {
    return spectrum_shells_t<double2>(uh0, uh1, uh2, N, nshell, inv, weight_n2, partial, out, stream);
}

cudaError_t spectrum_shells32(const void* uh0, const void* uh1, const void* uh2, int N, int nshell,
                              double inv, double* partial, double* out, cudaStream_t stream) {
    return spectrum_shells_t<float2>(uh0, uh1, uh2, N, nshell, inv, 0, partial, out, stream);
}

// ---------------------------------------------------------------------------
// f = f_eq(0, u) in the storage's compute type: FP64 for FP64 storage, FP32
// otherwise (FP64 arithmetic on this GPU runs at a small fraction of the FP32
// rate, and an FP32-stored state needs no more than FP32 arithmetic).
template <typename S>
__global__ void feq_kernel(const double* __restrict__ u, bool shifted, int N, size_t plane,
                           S* __restrict__ st) {
    using C = typename Traits<S>::C;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= N) return;
    const int y = blockIdx.y, z = blockIdx.z;
    const size_t c = (size_t)x + (size_t)N * (y + (size_t)N * z);
    const C ux = (C)u[c], uy = (C)u[plane + c], uz = (C)u[2 * plane + c];
    const C usq15 = C(1.5) * (ux * ux + uy * uy + uz * uz);
    static_for<0, Q>([&](auto ic) {
        constexpr int I = decltype(ic)::value;
        Traits<S>::store(st + I * plane + stored_index<I>(x, y, z, N, shifted), feq_i<I>(C(0), ux, uy, uz, usq15));
    });
}

template <typename S>
__global__ void set_pop_kernel(int i, const double* __restrict__ pl, bool shifted, int N,
                               size_t plane, S* __restrict__ st) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= N) return;
    const int y = blockIdx.y, z = blockIdx.z;
    const size_t c = (size_t)x + (size_t)N * (y + (size_t)N * z);
    Traits<S>::store(st + i * plane + stored_index_rt(i, x, y, z, N, shifted),
                     (typename Traits<S>::C)pl[c]);
}

template <typename S>
__global__ void get_pop_kernel(int i, const S* __restrict__ st, bool shifted, int N, size_t plane,
                               double* __restrict__ pl) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= N) return;
    const int y = blockIdx.y, z = blockIdx.z;
    const size_t c = (size_t)x + (size_t)N * (y + (size_t)N * z);
    pl[c] = (double)Traits<S>::load(st + i * plane + stored_index_rt(i, x, y, z, N, shifted));
}

template <typename S>
__global__ void sample_kernel(const S* __restrict__ st, bool shifted, int N, size_t plane,
                              const int64_t* __restrict__ cells, int64_t n, double* __restrict__ out) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * Q) return;
    const int64_t k = t / Q;
    const int i = (int)(t % Q);
    const int64_t c = cells[k];
    const int x = (int)(c % N), y = (int)((c / N) % N), z = (int)(c / ((int64_t)N * N));
    out[t] = (double)Traits<S>::load(st + i * plane + stored_index_rt(i, x, y, z, N, shifted));
}

// delta-rho of every cell (Eq. 8) into prev (mode 0), or (mode 1) the largest
// |delta-rho - prev| over the box into *maxbits as the bits of a
// non-negative float (ordered like the values, so atomicMax applies).
template <typename S>
__global__ void drho_change_kernel(const S* __restrict__ st, bool shifted, int N, size_t plane,
                                   double* __restrict__ prev, unsigned* maxbits, int mode) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z;
    float d = 0.0f;
    if (x < N) {
        double rho = 0.0;
        static_for<0, Q>([&](auto ic) {
            constexpr int I = decltype(ic)::value;
            rho += (double)Traits<S>::load(st + I * plane + stored_index<I>(x, y, z, N, shifted));
        });
        const size_t c = (size_t)x + (size_t)N * (y + (size_t)N * z);
        if (mode == 0) prev[c] = rho;
        else d = (float)fabs(rho - prev[c]);
    }
    if (mode == 1) {
        for (int o = 16; o > 0; o >>= 1) d = fmaxf(d, __shfl_down_sync(0xffffffffu, d, o));
        if ((threadIdx.x & 31) == 0) atomicMax(maxbits, __float_as_uint(d));
    }
}

__global__ void nonfinite_kernel(const double* __restrict__ v, size_t n, int* flag) {
    bool bad = false;
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (size_t)gridDim.x * blockDim.x)
        bad |= !isfinite(v[k]);
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flag, 1);
}

static dim3 row_grid(int N, int& bx) {
    bx = N >= 128 ? 128 : ((N + 31) / 32) * 32;
    return dim3((N + bx - 1) / bx, N, N);
}

#define KIN_DISPATCH(storage, CALL)                       \
    switch (storage) {                                    \
        case ST_F32: { using S = float; CALL; } break;    \
        case ST_F16: { using S = __half; CALL; } break;   \
        case ST_BF16: { using S = __nv_bfloat16; CALL; } break; \
        case ST_F64: { using S = double; CALL; } break;   \
        default: return cudaErrorInvalidValue;            \
    }

cudaError_t velocity_field(int storage, const void* state, bool shifted, int N, double* u,
                           cudaStream_t stream) {
    int bx;
    dim3 g = row_grid(N, bx);
    const size_t plane = (size_t)N * N * N;
    KIN_DISPATCH(storage, (velocity_kernel<S><<<g, bx, 0, stream>>>((const S*)state, shifted, N, plane, u)));
    return cudaGetLastError();
}

cudaError_t velocity_field32(int storage, const void* state, bool shifted, int N, float* u,
                             cudaStream_t stream) {
    int bx;
    dim3 g = row_grid(N, bx);
    const size_t plane = (size_t)N * N * N;
    switch (storage) {
        case ST_F32: velocity32_kernel<float><<<g, bx, 0, stream>>>((const float*)state, shifted, N, plane, u); break;
        case ST_F16: velocity32_kernel<__half><<<g, bx, 0, stream>>>((const __half*)state, shifted, N, plane, u); break;
        case ST_BF16:
            velocity32_kernel<__nv_bfloat16><<<g, bx, 0, stream>>>((const __nv_bfloat16*)state, shifted, N, plane, u);
            break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t equilibrium_from_velocity(int storage, const double* u, bool shifted, int N,
                                      void* state, cudaStream_t stream) {
    int bx;
    dim3 g = row_grid(N, bx);
    const size_t plane = (size_t)N * N * N;
    KIN_DISPATCH(storage, (feq_kernel<S><<<g, bx, 0, stream>>>(u, shifted, N, plane, (S*)state)));
    return cudaGetLastError();
}

cudaError_t set_population(int storage, int i, const double* pl, bool shifted, int N, void* state,
                           cudaStream_t stream) {
    int bx;
    dim3 g = row_grid(N, bx);
    const size_t plane = (size_t)N * N * N;
    KIN_DISPATCH(storage, (set_pop_kernel<S><<<g, bx, 0, stream>>>(i, pl, shifted, N, plane, (S*)state)));
    return cudaGetLastError();
}

cudaError_t get_population(int storage, int i, const void* state, bool shifted, int N, double* pl,
                           cudaStream_t stream) {
    int bx;
    dim3 g = row_grid(N, bx);
    const size_t plane = (size_t)N * N * N;
    KIN_DISPATCH(storage, (get_pop_kernel<S><<<g, bx, 0, stream>>>(i, (const S*)state, shifted, N, plane, pl)));
    return cudaGetLastError();
}

cudaError_t sample_cells(int storage, const void* state, bool shifted, int N, const int64_t* cells,
                         int64_t n, double* out, cudaStream_t stream) {
    if (n <= 0) return cudaSuccess;
    const size_t plane = (size_t)N * N * N;
    const int64_t tot = n * Q;
    const int threads = 256;
    const unsigned blocks = (unsigned)((tot + threads - 1) / threads);
    KIN_DISPATCH(storage, (sample_kernel<S><<<blocks, threads, 0, stream>>>((const S*)state, shifted, N, plane, cells, n, out)));
    return cudaGetLastError();
}

cudaError_t scan_nonfinite(const double* v, size_t n, int* flag, cudaStream_t stream) {
    nonfinite_kernel<<<304, 256, 0, stream>>>(v, n, flag);
    return cudaGetLastError();
}

cudaError_t drho_change(int storage, const void* state, bool shifted, int N, double* prev, unsigned* maxbits,
                        int mode, cudaStream_t stream) {
    int bx;
    dim3 g = row_grid(N, bx);
    const size_t plane = (size_t)N * N * N;
    KIN_DISPATCH(storage, (drho_change_kernel<S><<<g, bx, 0, stream>>>((const S*)state, shifted, N, plane, prev,
                                                                      maxbits, mode)));
    return cudaGetLastError();
}

}  // namespace kin

// ---------------------------------------------------------------------------
// E / eps reduction that allocates nothing.
//
// Some callers cannot let the library allocate device memory: a real-time
// loop must not call cudaMalloc or cudaFree (either can synchronise the whole
// device), and an application may have reserved all device memory for its own
// allocator (a framework's caching allocator, a fixed arena).  For them the
// per-block partial sums of the reduction live in this fixed array compiled
// into the library instead of in memory allocated per simulation.  It holds
// 2 x kStatsMaxBlocks doubles (19,456 bytes) and exists on every device that loads the
// library until the process exits.  Every call shares it and overwrites the
// partials it uses before reading them (nothing has to start at zero); calls
// whose kernels overlap on the GPU race on it.
namespace {

constexpr int kNoallocMaxBlocks = kin::kStatsMaxBlocks;
constexpr int kNoallocMaxN = 1024;
static_assert(kNoallocMaxBlocks >= kin::kStatsMaxBlocks, "partials must cover stats_blocks() for every N");

static __device__ __align__(256) double g_noalloc_partials[2 * kNoallocMaxBlocks];

// Device address of the array in the current device's context.  Looked up on
// every call, not cached: after a context reset the module is loaded again and
// the array may sit elsewhere.
double* noalloc_scratch(cudaError_t* err) {
    void* p = nullptr;
    *err = cudaGetSymbolAddress(&p, g_noalloc_partials);
    return *err == cudaSuccess ? (double*)p : nullptr;
}

}  // namespace

extern "C" int kin_energy_dissipation_noalloc(const double* u, int N, double nu, double* out,
                                              void* stream) {
    using namespace kin;
    if (!u || !out) return set_error(KIN_EINVAL, "NULL device pointer");
    if (N < 2 || N > kNoallocMaxN)
        return set_error(KIN_EINVAL,
                         "N = %d outside [2, %d], the sizes the fixed scratch of this entry point covers",
                         N, kNoallocMaxN);
    if (!(nu >= 0.0)) return set_error(KIN_EINVAL, "nu must be >= 0");
    const int nb = stats_blocks(N);
    if (nb > kNoallocMaxBlocks)
        return set_error(KIN_EINVAL, "reduction needs %d blocks, fixed scratch holds %d", nb,
                         kNoallocMaxBlocks);
    cudaError_t e;
    double* partials = noalloc_scratch(&e);
    if (!partials) return set_error(KIN_ECUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
    e = energy_dissipation(u, N, nu, partials, out, (cudaStream_t)stream);
    if (e != cudaSuccess) return set_error(KIN_ECUDA, "reduction launch: %s", cudaGetErrorString(e));
    return KIN_OK;
}

