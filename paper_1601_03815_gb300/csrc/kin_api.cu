// C ABI of libkin (declared in include/kin.h).
#include "kin.h"
#include "kin_common.cuh"
#include "kin_init.h"
#include "kin_internal.h"
#include "kin_sim.h"

#include <cufft.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <functional>
#include <queue>
#include <vector>

using namespace kin;



namespace {
thread_local char g_err[512] = "";
}  // namespace

int kin::set_error(int code, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

namespace {

int fail(int code, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

#define CK(call)                                                                             \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess)                                                               \
            return fail(e_ == cudaErrorMemoryAllocation ? KIN_ENOMEM : KIN_ECUDA, "%s: %s (%s:%d)", \
                        #call, cudaGetErrorString(e_), __FILE__, __LINE__);                  \
    } while (0)

#define CKFFT(call)                                                                         \
    do {                                                                                    \
        cufftResult r_ = (call);                                                            \
        if (r_ != CUFFT_SUCCESS)                                                            \
            return fail(KIN_ECUDA, "%s: cufft error %d (%s:%d)", #call, (int)r_, __FILE__, __LINE__); \
    } while (0)

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
        else prev = -1;
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

// Guard regions before and after each state buffer, filled with kGuardByte
// at creation: a kernel that writes outside the state shows up in
// kin_check_guards.
constexpr size_t kGuardBytes = 64 * 1024;
constexpr unsigned char kGuardByte = 0xA5;

// NVTX range over one API call (visible in Nsight timelines; a no-op without a
// tool attached).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};

size_t ncell(const kin_sim* s) { return (size_t)s->N * s->N * s->N; }
bool shifted(const kin_sim* s) { return s->scheme == KIN_LBE_MRT; }
size_t state_bytes(const kin_sim* s) { return Q * ncell(s) * storage_bytes(s->storage); }

int ensure_u(kin_sim* s) {
    if (!s->u) CK(cudaMalloc(&s->u, sizeof(double) * 3 * ncell(s)));
    const size_t need = std::max(2 * (size_t)std::max(stats_blocks(s->N), spectrum_blocks(s->N)) *
                                     (size_t)std::max(kin_num_shells(s->N), 2),
                                 9 * (size_t)deriv_moment_blocks(s->N));
    if (s->red_cap < need) {
        if (s->red) cudaFree(s->red);
        s->red = nullptr;
        CK(cudaMalloc(&s->red, sizeof(double) * need));
        s->red_cap = need;
    }
    if (!s->red_out) CK(cudaMalloc(&s->red_out, sizeof(double) * (16 + kin_num_shells(s->N))));
    return KIN_OK;
}

int ensure_uh(kin_sim* s) {
    if (!s->uh) CK(cudaMalloc(&s->uh, sizeof(double2) * 3 * (size_t)s->N * s->N * (s->N / 2 + 1)));
    return KIN_OK;
}

size_t nmode(const kin_sim* s) { return (size_t)s->N * s->N * (s->N / 2 + 1); }

int valid(const kin_sim* s) {
    if (!s) return fail(KIN_EINVAL, "NULL simulation handle");
    return KIN_OK;
}

// valid() and a defined state (not left part-way by a timed-out ensemble launch)
int usable(const kin_sim* s) {
    if (int r = valid(s)) return r;
    if (s->invalid)
        return fail(KIN_ESTATE, "the state is undefined after an ensemble launch gave up a wait; set it again "
                                "with kin_set_f, kin_set_velocity or kin_init_field");
    return KIN_OK;
}

// Planes per fused-DUGKS thread block when the caller has not chosen: as long
// as possible (fewer halo planes re-read) while the grid still has about two
// blocks per SM.
// Makespan, in plane-times, of the fused DUGKS launch with z chunks of zc
// planes: cols blocks per chunk, issued chunk by chunk (the grid's z index
// varies slowest), each occupying one of nsm SMs for its planes plus the
// ~1.5 plane-times of its prologue (two pre-steps and one cell view before
// the first face); every block goes to the SM that frees first.
double dugks_makespan(int N, long long cols, int zc, int nsm) {
    constexpr double kPrologue = 1.5;
    std::priority_queue<double, std::vector<double>, std::greater<double>> sm;
    for (int k = 0; k < nsm; ++k) sm.push(0.0);
    double end = 0.0;
    for (int z0 = 0; z0 < N; z0 += zc) {
        const double c = std::min(zc, N - z0) + kPrologue;
        for (long long b = 0; b < cols; ++b) {
            const double t = sm.top() + c;
            sm.pop();
            sm.push(t);
            end = std::max(end, t);
        }
    }
    return end;
}

// Planes per block of the fused DUGKS step.  With one block per SM the step
// lasts as long as its busiest SM, so a chunk length that leaves the last
// wave nearly empty costs up to a third of the step (128^3: 32 planes give
// 320 blocks, 2.1 waves).  When the columns alone fill fewer than 1.5 waves,
// every candidate is scored by the schedule above and the shortest taken (the
// longest chunk among those within 0.5 %: fewer halo planes re-read, longer
// runs of neighbouring columns in L2); measured at 32^3-192^3 this is within
// 1 % of the best chunk of a sweep.  Larger grids keep chunks that make about
// two waves of blocks, rounded down to 8 planes: at 256^3 that is 240 + 16
// planes, the measured optimum, which the schedule model (blind to cache
// effects) misranks by ~1 %.
// Rows per fused-DUGKS tile actually launched for this simulation's tuning.
int fused_tile_y(const kin_sim* s) {
    if (s->storage == ST_F64) return 4;
    return s->tile_y == 4 ? 4 : 8;
}

int auto_zchunk(kin_sim* s) {
    const int ty = fused_tile_y(s);
    if (s->zc_auto > 0 && s->zc_auto_ty == ty) return s->zc_auto;
    const int N = s->N;
    const long long cols = (long long)((N + 29) / 30) * ((N + ty - 1) / ty);
    s->zc_auto_ty = ty;
    if (2 * cols >= 3LL * s->num_sms) {
        long long zc = (long long)N * cols / (2LL * s->num_sms);
        zc = std::max(8LL, std::min<long long>(zc / 8 * 8, N));
        s->zc_auto = (int)zc;
        return s->zc_auto;
    }
    constexpr long long kMaxBlocks = 20000;
    int best_zc = N;
    double best = -1.0;
    for (int zc = N; zc >= 4; --zc) {
        const int nz = (N + zc - 1) / zc;
        if (nz > 64 || cols * nz > kMaxBlocks) continue;
        const double m = dugks_makespan(N, cols, zc, s->num_sms);
        if (best < 0.0 || m < best * (1.0 - 0.005)) {
            best = m;
            best_zc = zc;
        }
    }
    s->zc_auto = best_zc;
    return best_zc;
}

// KIN_ETIMEOUT (and clear the flag) if a kernel of this simulation gave up a
// bounded wait; call after the stream is synchronised.
int check_device_error(kin_sim* s) {
    int flag = 0;
    CK(cudaMemcpy(&flag, s->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag) {
        CK(cudaMemset(s->d_err, 0, sizeof(int)));
        return fail(KIN_ETIMEOUT, "a kernel of this simulation reported an error; the state is not valid");
    }
    return KIN_OK;
}

// The step goes to the fused cp.async DUGKS kernel, which can also write the
// new state's velocity (FP32-computed storage).
bool fused_velocity_ok(const kin_sim* s) {
    return s->scheme == KIN_DUGKS && s->storage != ST_F64 && s->variant != 1;
}

// One step; with uvel (only where fused_velocity_ok) the step also leaves the
// new state's velocity in s->u32.
int launch_step(kin_sim* s, float* uvel = nullptr) {
    const void* src = s->buf[s->cur];
    void* dst = s->buf[s->cur ^ 1];
    cudaError_t e;
    if (s->scheme == KIN_LBE_MRT)
        e = lbe_step(s->storage, src, dst, s->N, s->nu, s->block_lbe, s->stream);
    else if (s->variant == 1)
        e = dugks_step(s->storage, src, dst, s->fbp, s->N, s->nu, s->dt, s->block_dugks, s->stream);
    else
        e = dugks_step_fused(s->storage, src, dst, s->N, s->nu, s->dt, fused_tile_y(s),
                             s->zchunk > 0 ? s->zchunk : auto_zchunk(s), s->stream, uvel);
    if (e != cudaSuccess) return fail(KIN_ECUDA, "step launch: %s", cudaGetErrorString(e));
    s->launches += kin_step_launches(s);
    s->cur ^= 1;
    s->step += 1;
    s->epoch += 1;
    if (uvel) s->u32_epoch = s->epoch;
    return KIN_OK;
}

// Enqueue E and eps of the current state into red_out[0..1] (device).
int enqueue_energy_dissipation(kin_sim* s) {
    if (int r = ensure_u(s)) return r;
    if (s->storage == ST_F64) {
        CK(velocity_field(s->storage, s->buf[s->cur], shifted(s), s->N, s->u, s->stream));
        CK(energy_dissipation(s->u, s->N, s->nu, s->red, s->red_out, s->stream));
        s->launches += 3;
    } else {
        // FP32 arithmetic per cell (FP64 on this GPU runs at a small fraction
        // of the FP32 rate), FP64 sums; the velocity pass is skipped when u32
        // already holds this state's velocity (left by the step that made it,
        // or by an earlier call)
        if (!s->u32) CK(cudaMalloc(&s->u32, sizeof(float) * 3 * ncell(s)));
        if (s->u32_epoch != s->epoch) {
            CK(velocity_field32(s->storage, s->buf[s->cur], shifted(s), s->N, s->u32, s->stream));
            s->launches += 1;
            s->u32_epoch = s->epoch;
        }
        CK(energy_dissipation32(s->u32, s->N, s->nu, s->red, s->red_out, s->stream));
        s->launches += 2;
    }
    return KIN_OK;
}

}  // namespace

extern "C" {

int kin_lattice(int* xi, double* w) {
    if (!xi || !w) return fail(KIN_EINVAL, "NULL output");
    for (int i = 0; i < Q; ++i) {
        xi[3 * i + 0] = cx(i);
        xi[3 * i + 1] = cy(i);
        xi[3 * i + 2] = cz(i);
        w[i] = (double)w36(i) / 36.0;
    }
    return KIN_OK;
}

size_t kin_footprint_bytes(int N, int scheme, int storage) {
    if (N < 2 || storage < 0 || storage > 3) return 0;
    const size_t n = (size_t)N * N * N;
    (void)scheme;
    return 2 * Q * n * storage_bytes(storage);
}

int kin_num_shells(int N) {
    if (N < 1) return 0;
    const long long h = N / 2;
    const long long m = 3 * h * h;
    return 1 + (int)std::floor(std::sqrt((double)m) + 0.5);
}

int kin_create(int N, int scheme, double nu, double Ma, double dt, int storage, void* stream,
               kin_sim** out) {
    if (!out) return fail(KIN_EINVAL, "NULL output handle");
    *out = nullptr;
    if (N < 2 || N > 1024) return fail(KIN_EINVAL, "N = %d outside [2, 1024]", N);
    if (scheme != KIN_LBE_MRT && scheme != KIN_DUGKS) return fail(KIN_EINVAL, "unknown scheme %d", scheme);
    if (storage < KIN_F32 || storage > KIN_F64) return fail(KIN_EINVAL, "unknown storage %d", storage);
    if (!(nu > 0.0) || !std::isfinite(nu)) return fail(KIN_EINVAL, "nu must be positive, got %g", nu);
    if (!(Ma > 0.0) || !std::isfinite(Ma)) return fail(KIN_EINVAL, "Ma must be positive, got %g", Ma);
    if (scheme == KIN_LBE_MRT && std::fabs(dt - 1.0) > 1e-12)
        return fail(KIN_EINVAL, "LBE requires dt = 1 (dt = dx), got %g", dt);
    if (scheme == KIN_DUGKS && (!(dt > 0.0) || dt > 1.0 / std::sqrt(2.0) + 1e-12))
        return fail(KIN_EINVAL, "DUGKS requires 0 < dt <= 1/sqrt(2), got %g", dt);

    kin_sim* s = new kin_sim();
    s->N = N;
    s->scheme = scheme;
    s->storage = storage;
    s->nu = nu;
    s->Ma = Ma;
    s->dt = scheme == KIN_LBE_MRT ? 1.0 : dt;
    cudaGetDevice(&s->device);
    if (cudaDeviceGetAttribute(&s->num_sms, cudaDevAttrMultiProcessorCount, s->device) != cudaSuccess ||
        s->num_sms <= 0)
        s->num_sms = 152;
    auto bail = [&](int code) {
        kin_destroy(s);
        return code;
    };
    if (stream) {
        s->stream = (cudaStream_t)stream;
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return bail(fail(KIN_ECUDA, "stream: %s", cudaGetErrorString(e)));
        s->own_stream = true;
    }
    const size_t sb = state_bytes(s);
    for (int k = 0; k < 2; ++k) {
        cudaError_t e = cudaMalloc(&s->base[k], sb + 2 * kGuardBytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return bail(fail(KIN_ENOMEM, "state buffer of %zu bytes: %s", sb, cudaGetErrorString(e)));
        }
        s->buf[k] = static_cast<unsigned char*>(s->base[k]) + kGuardBytes;
        e = cudaMemsetAsync(s->base[k], kGuardByte, kGuardBytes, s->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(s->buf[k], 0, sb, s->stream);
        if (e == cudaSuccess)
            e = cudaMemsetAsync(static_cast<unsigned char*>(s->buf[k]) + sb, kGuardByte, kGuardBytes, s->stream);
        if (e != cudaSuccess) return bail(fail(KIN_ECUDA, "memset: %s", cudaGetErrorString(e)));
    }
    {
        cudaError_t e = cudaMalloc(&s->d_err, sizeof(int));
        if (e != cudaSuccess) return bail(fail(KIN_ENOMEM, "error flag: %s", cudaGetErrorString(e)));
        e = cudaMemsetAsync(s->d_err, 0, sizeof(int), s->stream);
        if (e != cudaSuccess) return bail(fail(KIN_ECUDA, "memset: %s", cudaGetErrorString(e)));
        e = cudaMallocHost(&s->h_pin, 4 * sizeof(double));
        if (e != cudaSuccess) return bail(fail(KIN_ENOMEM, "pinned words: %s", cudaGetErrorString(e)));
    }
    cudaError_t e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return bail(fail(KIN_ECUDA, "sync: %s", cudaGetErrorString(e)));
    *out = s;
    return KIN_OK;
}

void kin_destroy(kin_sim* s) {
    if (!s) return;
    DeviceGuard g(s->device);
    if (s->stream) cudaStreamSynchronize(s->stream);
    for (int k = 0; k < 2; ++k)
        if (s->base[k]) cudaFree(s->base[k]);
    if (s->fbp) cudaFree(s->fbp);
    if (s->u) cudaFree(s->u);
    if (s->u32) cudaFree(s->u32);
    if (s->d_err) cudaFree(s->d_err);
    if (s->h_pin) cudaFreeHost(s->h_pin);
    if (s->uh) cudaFree(s->uh);
    if (s->red) cudaFree(s->red);
    if (s->red_out) cudaFree(s->red_out);
    if (s->have_d2z) cufftDestroy(s->d2z);
    if (s->have_z2d) cufftDestroy(s->z2d);
    if (s->have_r2c) cufftDestroy(s->r2c);
    if (s->own_stream && s->stream) cudaStreamDestroy(s->stream);
    delete s;
}

int kin_set_velocity(kin_sim* s, const double* u) {
    if (int r = valid(s)) return r;
    if (!u) return fail(KIN_EINVAL, "NULL velocity");
    DeviceGuard g(s->device);
    if (int r = ensure_u(s)) return r;
    CK(cudaMemcpyAsync(s->u, u, sizeof(double) * 3 * ncell(s), cudaMemcpyHostToDevice, s->stream));
    CK(equilibrium_from_velocity(s->storage, s->u, shifted(s), s->N, s->buf[s->cur], s->stream));
    CK(cudaStreamSynchronize(s->stream));
    s->step = 0;
    s->epoch += 1;
    s->invalid = false;
    return KIN_OK;
}

int kin_init_field(kin_sim* s, uint64_t seed, double k0, double re_lambda) {
    NvtxRange nvtx_("kin_init_field");
    if (int r = valid(s)) return r;
    if (s->N < 4 || (s->N & 1)) return fail(KIN_EINVAL, "kin_init_field needs even N >= 4, got %d", s->N);
    if (!(k0 > 0.0) || !std::isfinite(k0)) return fail(KIN_EINVAL, "k0 must be positive");
    DeviceGuard g(s->device);
    if (int r = ensure_u(s)) return r;
    if (int r = ensure_uh(s)) return r;
    const int N = s->N;
    const size_t nm = nmode(s);
    double2* u0 = s->uh;
    double2* u1 = s->uh + nm;
    double2* u2 = s->uh + 2 * nm;
    CK(generate_modes(N, seed, u0, u1, u2, s->stream));
    const int nsh = kin_num_shells(N);
    CK(spectrum_shells(u0, u1, u2, N, nsh, 1.0, 0, s->red, s->red_out, s->stream));
    std::vector<double> e(nsh);
    CK(cudaMemcpyAsync(e.data(), s->red_out, sizeof(double) * nsh, cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    // shell targets E_t(s) = s^4 exp(-2 s^2 / k0^2), s = 1..N/2-1; global
    // factor so that <u.u> = 2 sum E = Ma^2 (u' = Ma c_s, c_s^2 = 1/3)
    const int smax = N / 2 - 1;
    std::vector<double> scale(nsh, 0.0);
    double total = 0.0;
    for (int sh = 1; sh <= smax; ++sh) {
        const double sd = (double)sh;
        const double et = sd * sd * sd * sd * std::exp(-2.0 * sd * sd / (k0 * k0));
        total += et;
        scale[sh] = e[sh] > 0.0 ? std::sqrt(et / e[sh]) : 0.0;
    }
    const double glob = std::sqrt(s->Ma * s->Ma / (2.0 * total));
    CK(cudaMemcpyAsync(s->red_out, scale.data(), sizeof(double) * nsh, cudaMemcpyHostToDevice, s->stream));
    CK(scale_modes(N, s->red_out, glob, u0, u1, u2, s->stream));
    // Omega = (2 pi / N)^2 sum |n|^2 |u_hat|^2 / 2 and <u.u> = 2 sum |u_hat|^2 / 2
    CK(spectrum_shells(u0, u1, u2, N, nsh, 1.0, 1, s->red, s->red_out, s->stream));
    CK(cudaMemcpyAsync(e.data(), s->red_out, sizeof(double) * nsh, cudaMemcpyDeviceToHost, s->stream));
    std::vector<double> e2(nsh);
    CK(spectrum_shells(u0, u1, u2, N, nsh, 1.0, 0, s->red, s->red_out, s->stream));
    CK(cudaMemcpyAsync(e2.data(), s->red_out, sizeof(double) * nsh, cudaMemcpyDeviceToHost, s->stream));
    // u(x) = sum_n u_hat(n) exp(i 2 pi n.x / N): unnormalised inverse transform
    if (!s->have_z2d) {
        CKFFT(cufftPlan3d(&s->z2d, N, N, N, CUFFT_Z2D));
        s->have_z2d = true;
    }
    CKFFT(cufftSetStream(s->z2d, s->stream));
    for (int c = 0; c < 3; ++c)
        CKFFT(cufftExecZ2D(s->z2d, (cufftDoubleComplex*)(s->uh + c * nm), s->u + c * ncell(s)));
    CK(equilibrium_from_velocity(s->storage, s->u, shifted(s), N, s->buf[s->cur], s->stream));
    CK(cudaStreamSynchronize(s->stream));
    double omega = 0.0, uu = 0.0;
    for (int sh = 0; sh < nsh; ++sh) {
        omega += e[sh];
        uu += e2[sh];
    }
    omega *= (2.0 * M_PI / N) * (2.0 * M_PI / N);
    uu *= 2.0;
    if (re_lambda > 0.0) {
        const double up2 = uu / 3.0;
        s->nu = up2 * std::sqrt(15.0 / (2.0 * omega)) / re_lambda;
    }
    s->step = 0;
    s->epoch += 1;
    s->invalid = false;
    return KIN_OK;
}

int kin_set_f(kin_sim* s, const double* f) {
    if (int r = valid(s)) return r;
    if (!f) return fail(KIN_EINVAL, "NULL f");
    DeviceGuard g(s->device);
    if (int r = ensure_u(s)) return r;
    const size_t n = ncell(s);
    for (int i = 0; i < Q; ++i) {
        CK(cudaMemcpyAsync(s->u, f + (size_t)i * n, sizeof(double) * n, cudaMemcpyHostToDevice, s->stream));
        CK(set_population(s->storage, i, s->u, shifted(s), s->N, s->buf[s->cur], s->stream));
    }
    CK(cudaStreamSynchronize(s->stream));
    s->step = 0;
    s->epoch += 1;
    s->invalid = false;
    return KIN_OK;
}

int kin_get_f(kin_sim* s, double* f) {
    if (int r = valid(s)) return r;
    if (!f) return fail(KIN_EINVAL, "NULL f");
    DeviceGuard g(s->device);
    if (int r = ensure_u(s)) return r;
    const size_t n = ncell(s);
    for (int i = 0; i < Q; ++i) {
        CK(get_population(s->storage, i, s->buf[s->cur], shifted(s), s->N, s->u, s->stream));
        CK(cudaMemcpyAsync(f + (size_t)i * n, s->u, sizeof(double) * n, cudaMemcpyDeviceToHost, s->stream));
        CK(cudaStreamSynchronize(s->stream));
    }
    return KIN_OK;
}

int kin_sample_f(kin_sim* s, const int64_t* cells, int64_t n, double* out) {
    if (int r = valid(s)) return r;
    if (n < 0 || (n > 0 && (!cells || !out))) return fail(KIN_EINVAL, "bad sample arguments");
    if (n == 0) return KIN_OK;
    const int64_t nc = (int64_t)ncell(s);
    for (int64_t k = 0; k < n; ++k)
        if (cells[k] < 0 || cells[k] >= nc) return fail(KIN_EINVAL, "cell index %lld out of range", (long long)cells[k]);
    DeviceGuard g(s->device);
    int64_t* dc = nullptr;
    double* dout = nullptr;
    CK(cudaMalloc(&dc, sizeof(int64_t) * n));
    cudaError_t e = cudaMalloc(&dout, sizeof(double) * n * Q);
    if (e != cudaSuccess) {
        cudaFree(dc);
        return fail(KIN_ENOMEM, "sample buffer: %s", cudaGetErrorString(e));
    }
    int rc = KIN_OK;
    do {
        if ((e = cudaMemcpyAsync(dc, cells, sizeof(int64_t) * n, cudaMemcpyHostToDevice, s->stream)) != cudaSuccess) break;
        if ((e = sample_cells(s->storage, s->buf[s->cur], shifted(s), s->N, dc, n, dout, s->stream)) != cudaSuccess) break;
        if ((e = cudaMemcpyAsync(out, dout, sizeof(double) * n * Q, cudaMemcpyDeviceToHost, s->stream)) != cudaSuccess) break;
        e = cudaStreamSynchronize(s->stream);
    } while (0);
    if (e != cudaSuccess) rc = fail(KIN_ECUDA, "sample: %s", cudaGetErrorString(e));
    cudaFree(dc);
    cudaFree(dout);
    return rc;
}

int kin_get_velocity(kin_sim* s, double* u) {
    if (int r = valid(s)) return r;
    if (!u) return fail(KIN_EINVAL, "NULL u");
    DeviceGuard g(s->device);
    if (int r = ensure_u(s)) return r;
    CK(velocity_field(s->storage, s->buf[s->cur], shifted(s), s->N, s->u, s->stream));
    CK(cudaMemcpyAsync(u, s->u, sizeof(double) * 3 * ncell(s), cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    return KIN_OK;
}

int kin_step(kin_sim* s, int n) {
    NvtxRange nvtx_("kin_step");
    if (int r = usable(s)) return r;
    if (n < 0) return fail(KIN_EINVAL, "negative step count");
    DeviceGuard g(s->device);
    for (int k = 0; k < n; ++k)
        if (int r = launch_step(s)) return r;
    return KIN_OK;
}

int kin_step_stats(kin_sim* s, int n, double* E, double* eps, double* Ek) {
    NvtxRange nvtx_("kin_step_stats");
    if (int r = usable(s)) return r;
    if (n < 0) return fail(KIN_EINVAL, "negative step count");
    DeviceGuard g(s->device);
    const bool fuse = n > 0 && fused_velocity_ok(s);
    if (fuse && !s->u32) CK(cudaMalloc(&s->u32, sizeof(float) * 3 * ncell(s)));
    for (int k = 0; k < n; ++k)
        if (int r = launch_step(s, fuse && k == n - 1 ? s->u32 : nullptr)) return r;
    return kin_stats(s, E, eps, Ek);
}

int kin_stats_async(kin_sim* s, double* out) {
    NvtxRange nvtx_("kin_stats_async");
    if (int r = usable(s)) return r;
    if (!out) return fail(KIN_EINVAL, "NULL output");
    DeviceGuard g(s->device);
    if (int r = enqueue_energy_dissipation(s)) return r;
    CK(cudaMemcpyAsync(out, s->red_out, 2 * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    return KIN_OK;
}

int kin_step_stats_async(kin_sim* s, int n, double* out) {
    NvtxRange nvtx_("kin_step_stats_async");
    if (int r = usable(s)) return r;
    if (n < 0) return fail(KIN_EINVAL, "negative step count");
    if (!out) return fail(KIN_EINVAL, "NULL output");
    DeviceGuard g(s->device);
    const bool fuse = n > 0 && fused_velocity_ok(s);
    if (fuse && !s->u32) CK(cudaMalloc(&s->u32, sizeof(float) * 3 * ncell(s)));
    for (int k = 0; k < n; ++k)
        if (int r = launch_step(s, fuse && k == n - 1 ? s->u32 : nullptr)) return r;
    return kin_stats_async(s, out);
}

int kin_init_consistent(kin_sim* s, int max_iter, double tol, int* iters, double* residual) {
    NvtxRange nvtx_("kin_init_consistent");
    if (int r = usable(s)) return r;
    if (max_iter < 1) return fail(KIN_EINVAL, "max_iter must be >= 1, got %d", max_iter);
    DeviceGuard g(s->device);
    if (int r = ensure_u(s)) return r;
    if (int r = ensure_uh(s)) return r;
    // u0: the velocity of the current state, held through the iteration
    CK(velocity_field(s->storage, s->buf[s->cur], shifted(s), s->N, s->u, s->stream));
    constexpr int kCheckEvery = 10;
    // scratch: the previous delta-rho (N^3 doubles) in the spectrum buffer,
    // the largest change in one word of the reduction buffer
    double* prev = reinterpret_cast<double*>(s->uh);
    unsigned* maxbits = reinterpret_cast<unsigned*>(s->red);
    double res = -1.0;
    int it = 0;
    while (it < max_iter) {
        ++it;
        const bool check = it % kCheckEvery == 0 || it == max_iter;
        if (check) CK(drho_change(s->storage, s->buf[s->cur], shifted(s), s->N, prev, maxbits, 0, s->stream));
        if (s->scheme == KIN_LBE_MRT) {
            CK(lbe_consistent_step(s->storage, s->buf[s->cur], s->buf[s->cur ^ 1], s->N, s->nu, s->u, s->stream));
            s->cur ^= 1;
            s->launches += 1;
        } else {
            // a plain DUGKS step, then the momentum back to rho0 u0
            if (int r = launch_step(s)) return r;
            CK(dugks_reset_momentum(s->storage, s->buf[s->cur], s->N, s->u, s->stream));
            s->launches += 1;
        }
        if (check) {
            CK(cudaMemsetAsync(maxbits, 0, sizeof(unsigned), s->stream));
            CK(drho_change(s->storage, s->buf[s->cur], shifted(s), s->N, prev, maxbits, 1, s->stream));
            unsigned bits = 0;
            CK(cudaMemcpyAsync(s->h_pin, maxbits, sizeof(unsigned), cudaMemcpyDeviceToHost, s->stream));
            CK(cudaStreamSynchronize(s->stream));
            std::memcpy(&bits, s->h_pin, sizeof(unsigned));
            float r;
            std::memcpy(&r, &bits, sizeof(float));
            res = r;
            s->launches += 2;
            if (!std::isfinite(res)) return fail(KIN_ENONFINITE, "consistent initialisation diverged");
            if (res <= tol) break;
        }
    }
    s->step = 0;
    s->epoch += 1;
    if (iters) *iters = it;
    if (residual) *residual = res;
    return KIN_OK;
}

int kin_stats(kin_sim* s, double* E, double* eps, double* Ek) {
    NvtxRange nvtx_("kin_stats");
    if (int r = usable(s)) return r;
    DeviceGuard g(s->device);
    if (int r = enqueue_energy_dissipation(s)) return r;
    // E, eps and the step kernels' error flag in one synchronisation
    CK(cudaMemcpyAsync(s->h_pin, s->red_out, 2 * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    CK(cudaMemcpyAsync(s->h_pin + 2, s->d_err, sizeof(int), cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    const double ed[2] = {s->h_pin[0], s->h_pin[1]};
    int flag = 0;
    std::memcpy(&flag, s->h_pin + 2, sizeof(int));
    if (flag) return check_device_error(s);
    if (E) *E = ed[0];
    if (eps) *eps = ed[1];
    if (!std::isfinite(ed[0]) || !std::isfinite(ed[1]))
        return fail(KIN_ENONFINITE, "non-finite statistics at step %lld", (long long)s->step);
    if (Ek) {
        if (int r = ensure_uh(s)) return r;
        const int N = s->N;
        const size_t nm = nmode(s);
        const int nsh = kin_num_shells(N);
        const double inv = 1.0 / ((double)N * N * N);
        if (s->storage == ST_F64) {
            if (!s->have_d2z) {
                CKFFT(cufftPlan3d(&s->d2z, N, N, N, CUFFT_D2Z));
                s->have_d2z = true;
            }
            CKFFT(cufftSetStream(s->d2z, s->stream));
            for (int c = 0; c < 3; ++c)
                CKFFT(cufftExecD2Z(s->d2z, s->u + c * ncell(s), (cufftDoubleComplex*)(s->uh + c * nm)));
            CK(spectrum_shells(s->uh, s->uh + nm, s->uh + 2 * nm, N, nsh, inv, 0, s->red, s->red_out,
                               s->stream));
        } else {
            // FP32 transforms of the FP32 velocity already formed above: their
            // rounding error spreads over every mode, far below the storage's
            // own rounding in any shell; |u_hat|^2 is summed in FP64.  The
            // complex output reuses the FP64 spectrum buffer.
            if (!s->have_r2c) {
                CKFFT(cufftPlan3d(&s->r2c, N, N, N, CUFFT_R2C));
                s->have_r2c = true;
            }
            CKFFT(cufftSetStream(s->r2c, s->stream));
            cufftComplex* uh32 = (cufftComplex*)s->uh;
            for (int c = 0; c < 3; ++c)
                CKFFT(cufftExecR2C(s->r2c, s->u32 + c * ncell(s), uh32 + c * nm));
            s->u32_epoch = ~0ull;  // the transforms may use their input as work space
            CK(spectrum_shells32(uh32, uh32 + nm, uh32 + 2 * nm, N, nsh, inv, s->red, s->red_out, s->stream));
        }
        s->launches += 2;
        CK(cudaMemcpyAsync(Ek, s->red_out, sizeof(double) * nsh, cudaMemcpyDeviceToHost, s->stream));
        CK(cudaStreamSynchronize(s->stream));
    }
    return KIN_OK;
}

int kin_derived_stats(kin_sim* s, double* out, double* D) {
    NvtxRange nvtx_("kin_derived_stats");
    if (int r = usable(s)) return r;
    if (!out) return fail(KIN_EINVAL, "NULL output");
    DeviceGuard g(s->device);
    if (int r = ensure_u(s)) return r;
    if (int r = ensure_uh(s)) return r;
    const int N = s->N;
    const size_t n = ncell(s), nm = nmode(s);
    CK(velocity_field(s->storage, s->buf[s->cur], shifted(s), N, s->u, s->stream));
    CK(energy_dissipation(s->u, N, s->nu, s->red, s->red_out, s->stream));
    double ed[2];
    CK(cudaMemcpyAsync(ed, s->red_out, sizeof(ed), cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    if (!std::isfinite(ed[0]))
        return fail(KIN_ENONFINITE, "non-finite statistics at step %lld", (long long)s->step);
    if (!s->have_d2z) {
        CKFFT(cufftPlan3d(&s->d2z, N, N, N, CUFFT_D2Z));
        s->have_d2z = true;
    }
    if (!s->have_z2d) {
        CKFFT(cufftPlan3d(&s->z2d, N, N, N, CUFFT_Z2D));
        s->have_z2d = true;
    }
    CKFFT(cufftSetStream(s->d2z, s->stream));
    CKFFT(cufftSetStream(s->z2d, s->stream));
    for (int c = 0; c < 3; ++c)
        CKFFT(cufftExecD2Z(s->d2z, s->u + c * n, (cufftDoubleComplex*)(s->uh + c * nm)));
    // shells of |n|^2 |u_hat|^2 / 2 (per mode), scaled below to D(s)
    const int nsh = kin_num_shells(N);
    const double inv = 1.0 / ((double)N * N * N);
    CK(spectrum_shells(s->uh, s->uh + nm, s->uh + 2 * nm, N, nsh, inv, 1, s->red, s->red_out, s->stream));
    std::vector<double> w(nsh);
    CK(cudaMemcpyAsync(w.data(), s->red_out, sizeof(double) * nsh, cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    // d_a u_a into the velocity scratch, component by component
    for (int a = 0; a < 3; ++a) {
        CK(derivative_multiply(s->uh + a * nm, N, a, s->stream));
        CKFFT(cufftExecZ2D(s->z2d, (cufftDoubleComplex*)(s->uh + a * nm), s->u + a * n));
    }
    CK(derivative_moments(s->u, N, s->red, s->red_out, s->stream));
    double m[9];
    CK(cudaMemcpyAsync(m, s->red_out, sizeof(m), cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    s->launches += 10;  // velocity, 2 + 2 reductions, 3 multiplies, 2 moment passes
    const double kf = 2.0 * 3.14159265358979323846 / N, nu = s->nu;
    double eps = 0.0;
    for (int k = 0; k < nsh; ++k) {
        const double d = 2.0 * nu * kf * kf * w[k];
        if (D) D[k] = d;
        eps += d;
    }
    const double E = ed[0], up = std::sqrt(2.0 * E / 3.0);
    const double lam = std::sqrt(15.0 * nu / eps) * up;
    out[0] = E;
    out[1] = up;
    out[2] = eps;
    out[3] = lam;
    out[4] = up * lam / nu;
    out[5] = std::pow(nu * nu * nu / eps, 0.25);
    out[6] = (m[1] + m[4] + m[7]) / (std::pow(m[0], 1.5) + std::pow(m[3], 1.5) + std::pow(m[6], 1.5));
    out[7] = (m[2] + m[5] + m[8]) / (m[0] * m[0] + m[3] * m[3] + m[6] * m[6]);
    return KIN_OK;
}

int kin_step_launches(const kin_sim* s) {
    if (!s) return 0;
    if (s->scheme == KIN_LBE_MRT) return 1;
    return s->variant == 1 ? 2 : 1;
}

int kin_set_tuning(kin_sim* s, int block_x, int tile_y, int zchunk, int variant) {
    if (int r = valid(s)) return r;
    if (block_x > 0 && (block_x % 32 || block_x > 1024)) return fail(KIN_EINVAL, "block_x %d", block_x);
    if (tile_y > 0 && tile_y != 4 && tile_y != 8) return fail(KIN_EINVAL, "tile_y must be 4 or 8");
    if (variant > 1) return fail(KIN_EINVAL, "variant %d", variant);
    if (variant == 1 && s->scheme == KIN_DUGKS && !s->fbp) {
        const size_t fb = Q * ncell(s) * dugks_scratch_bytes(s->storage);
        DeviceGuard g(s->device);
        CK(cudaMalloc(&s->fbp, fb));
    }
    if (block_x > 0) s->block_lbe = s->block_dugks = block_x;
    if (tile_y > 0) s->tile_y = tile_y;
    if (zchunk > 0) s->zchunk = zchunk;
    if (variant >= 0) s->variant = variant;
    return KIN_OK;
}

int64_t kin_kernel_launches(const kin_sim* s) { return s ? s->launches : 0; }

int kin_sync(kin_sim* s) {
    if (int r = valid(s)) return r;
    DeviceGuard g(s->device);
    CK(cudaStreamSynchronize(s->stream));
    return check_device_error(s);
}

double kin_get_nu(const kin_sim* s) { return s ? s->nu : 0.0; }
double kin_get_dt(const kin_sim* s) { return s ? s->dt : 0.0; }
double kin_get_time(const kin_sim* s) { return s ? (double)s->step * s->dt : 0.0; }
int64_t kin_get_step(const kin_sim* s) { return s ? s->step : 0; }
int kin_get_N(const kin_sim* s) { return s ? s->N : 0; }
int kin_get_scheme(const kin_sim* s) { return s ? s->scheme : -1; }
int kin_get_storage(const kin_sim* s) { return s ? s->storage : -1; }

const char* kin_strerror(int code) {
    switch (code) {
        case KIN_OK: return "ok";
        case KIN_EINVAL: return "invalid argument";
        case KIN_ENOMEM: return "out of device memory";
        case KIN_ECUDA: return "CUDA error";
        case KIN_ENONFINITE: return "non-finite state";
        case KIN_ETIMEOUT: return "device wait timed out";
        case KIN_ESTATE: return "invalid state";
        case KIN_EGUARD: return "a guard region of a state buffer was overwritten";
        case KIN_EDEBUG: return "an index check of the debug build failed";
    }
    return "unknown status";
}

const char* kin_last_error(void) { return g_err; }

int kin_check_guards(kin_sim* s) {
    if (int r = valid(s)) return r;
    DeviceGuard g(s->device);
    CK(cudaStreamSynchronize(s->stream));
    std::vector<unsigned char> h(kGuardBytes);
    const size_t sb = state_bytes(s);
    for (int k = 0; k < 2; ++k)
        for (int side = 0; side < 2; ++side) {
            const unsigned char* p =
                side == 0 ? static_cast<const unsigned char*>(s->base[k]) : static_cast<const unsigned char*>(s->buf[k]) + sb;
            CK(cudaMemcpy(h.data(), p, kGuardBytes, cudaMemcpyDeviceToHost));
            for (size_t b = 0; b < kGuardBytes; ++b)
                if (h[b] != kGuardByte)
                    return fail(KIN_EGUARD, "state buffer %d: guard %s the data overwritten at byte %zu", k,
                                side == 0 ? "before" : "after", b);
        }
    return KIN_OK;
}

int kin_test_corrupt_guard(kin_sim* s, int buffer, int side) {
    if (int r = valid(s)) return r;
    if (buffer < 0 || buffer > 1 || side < 0 || side > 1) return fail(KIN_EINVAL, "buffer and side are 0 or 1");
    DeviceGuard g(s->device);
    CK(cudaStreamSynchronize(s->stream));
    unsigned char* p = side == 0 ? static_cast<unsigned char*>(s->base[buffer]) + kGuardBytes / 2
                                 : static_cast<unsigned char*>(s->buf[buffer]) + state_bytes(s) + 7;
    CK(cudaMemset(p, kGuardByte ^ 0xFF, 1));
    return KIN_OK;
}

int kin_debug_status(int* is_debug, unsigned long long* word, int reset) {
#ifdef KIN_DEBUG
    if (is_debug) *is_debug = 1;
#else
    if (is_debug) *is_debug = 0;
#endif
    unsigned long long w[3] = {0, 0, 0};
    CK(debug_word_dugks(&w[0], reset != 0));
    CK(debug_word_lbe(&w[1], reset != 0));
    CK(debug_word_ensemble(&w[2], reset != 0));
    const unsigned long long first = w[0] ? w[0] : (w[1] ? w[1] : w[2]);
    if (word) *word = first;
    if (first)
        return fail(KIN_EDEBUG, "index check failed at site %llu with value %llu", first >> 40,
                    first & ((1ull << 40) - 1));
    return KIN_OK;
}

}  // extern "C"
