// Seeded initial field of Sec. III (Eq. 25), generated on the device.
//
// The generator the paper leaves unstated is fixed as follows (the library's
// own implementation of a definition that the test inputs also follow):
//   * modes n with shell s(n) = floor(|n| + 1/2) in [1, N/2 - 1] are excited;
//   * canonical half space H: nz > 0, or nz = 0 and ny > 0, or nz = ny = 0 and
//     nx > 0; u_hat(-n) = conj(u_hat(n));
//   * for n in H, component c: counter m = ((kz N + ky) N + kx) 3 + c with
//     (kx, ky, kz) = n mod N; key = splitmix64 output 0 of the stream seeded
//     with `seed`; U1 = unit(output 2m), U2 = unit(output 2m + 1) of the
//     stream seeded with key; g = sqrt(-2 ln U1) exp(2 pi i U2)  (Box-Muller);
//   * projection u_hat -= n (n . u_hat) / |n|^2 (solenoidal field);
//   * shell and global rescaling are applied by the host code in kin_api.cu.
// splitmix64 (Steele, Lea & Flood, OOPSLA 2014): output m of the stream seeded
// with s is mix64(s + (m + 1) * 0x9E3779B97F4A7C15).
#include "kin_common.cuh"
#include "kin_init.h"

namespace kin {

__host__ __device__ inline uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__host__ __device__ inline uint64_t splitmix_out(uint64_t seed, uint64_t m) {
    return mix64(seed + (m + 1ull) * 0x9E3779B97F4A7C15ull);
}

uint64_t field_key(uint64_t seed) { return splitmix_out(seed, 0); }

__device__ inline double unit53(uint64_t v) { return ((double)(v >> 11) + 0.5) * 0x1.0p-53; }

__device__ inline int signed_k(int k, int N) { return k > N / 2 ? k - N : k; }

__global__ void gen_modes_kernel(int N, uint64_t key, double2* __restrict__ u0,
                                 double2* __restrict__ u1, double2* __restrict__ u2) {
    const int nh = N / 2 + 1;
    const size_t nmode = (size_t)N * N * nh;
    const size_t m = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= nmode) return;
    const int kx = (int)(m % nh);
    const int ky = (int)((m / nh) % N);
    const int kz = (int)(m / ((size_t)nh * N));
    const int sx = kx, sy = signed_k(ky, N), sz = signed_k(kz, N);
    const long long n2 = (long long)sx * sx + (long long)sy * sy + (long long)sz * sz;
    const int shell = (int)floor(sqrt((double)n2) + 0.5);
    double2 g[3] = {{0.0, 0.0}, {0.0, 0.0}, {0.0, 0.0}};
    if (shell >= 1 && shell <= N / 2 - 1) {
        const bool in_h = sz > 0 || (sz == 0 && sy > 0) || (sz == 0 && sy == 0 && sx > 0);
        const int ccx = ((in_h ? sx : -sx) % N + N) % N;
        const int ccy = ((in_h ? sy : -sy) % N + N) % N;
        const int ccz = ((in_h ? sz : -sz) % N + N) % N;
        const uint64_t base = (((uint64_t)ccz * N + (uint64_t)ccy) * N + (uint64_t)ccx) * 3ull;
        for (int c = 0; c < 3; ++c) {
            const uint64_t mc = base + (uint64_t)c;
            const double U1 = unit53(splitmix_out(key, 2ull * mc));
            const double U2 = unit53(splitmix_out(key, 2ull * mc + 1ull));
            const double r = sqrt(-2.0 * log(U1));
            const double ph = 2.0 * 3.141592653589793 * U2;
            g[c].x = r * cos(ph);
            g[c].y = in_h ? r * sin(ph) : -(r * sin(ph));
        }
        const double n2d = (double)n2;
        const double2 nd = {(sx * g[0].x + sy * g[1].x) + sz * g[2].x,
                            (sx * g[0].y + sy * g[1].y) + sz * g[2].y};
        g[0].x -= sx * nd.x / n2d;
        g[0].y -= sx * nd.y / n2d;
        g[1].x -= sy * nd.x / n2d;
        g[1].y -= sy * nd.y / n2d;
        g[2].x -= sz * nd.x / n2d;
        g[2].y -= sz * nd.y / n2d;
    }
    u0[m] = g[0];
    u1[m] = g[1];
    u2[m] = g[2];
}

__global__ void scale_modes_kernel(int N, const double* __restrict__ shell_scale, double glob,
                                   double2* __restrict__ u0, double2* __restrict__ u1,
                                   double2* __restrict__ u2) {
    const int nh = N / 2 + 1;
    const size_t nmode = (size_t)N * N * nh;
    const size_t m = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= nmode) return;
    const int kx = (int)(m % nh);
    const int ky = (int)((m / nh) % N);
    const int kz = (int)(m / ((size_t)nh * N));
    const int sy = signed_k(ky, N), sz = signed_k(kz, N);
    const long long n2 = (long long)kx * kx + (long long)sy * sy + (long long)sz * sz;
    const int shell = (int)floor(sqrt((double)n2) + 0.5);
    const double s = (shell >= 1 && shell <= N / 2 - 1) ? shell_scale[shell] : 0.0;
    double2* arr[3] = {u0, u1, u2};
    for (int c = 0; c < 3; ++c) {
        double2 v = arr[c][m];
        v.x = (v.x * s) * glob;
        v.y = (v.y * s) * glob;
        arr[c][m] = v;
    }
}

cudaError_t generate_modes(int N, uint64_t seed, double2* u0, double2* u1, double2* u2,
                           cudaStream_t stream) {
    const size_t nmode = (size_t)N * N * (N / 2 + 1);
    const unsigned blocks = (unsigned)((nmode + 255) / 256);
    gen_modes_kernel<<<blocks, 256, 0, stream>>>(N, field_key(seed), u0, u1, u2);
    return cudaGetLastError();
}

cudaError_t scale_modes(int N, const double* shell_scale, double glob, double2* u0, double2* u1,
                        double2* u2, cudaStream_t stream) {
    const size_t nmode = (size_t)N * N * (N / 2 + 1);
    const unsigned blocks = (unsigned)((nmode + 255) / 256);
    scale_modes_kernel<<<blocks, 256, 0, stream>>>(N, shell_scale, glob, u0, u1, u2);
    return cudaGetLastError();
}

}  // namespace kin
