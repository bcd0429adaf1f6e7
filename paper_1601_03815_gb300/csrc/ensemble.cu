// Ensemble of independent simulations advanced by one persistent, cooperative
// kernel launch (captured in a CUDA graph).
//
// The work of one time step is a list of items (member, tile): a DUGKS tile
// of the fused step (dugks_tile.cuh) or a run of consecutive LBE nodes
// (lbe_node.cuh).  Thread blocks take (step, item) pairs one at a time from a
// global counter, all items of step s before any of step s + 1.  A member's
// step s may start only when all its tiles of step s - 1 are done: each
// finished tile adds one to the member's counter with a GPU-scope release, and
// a block waits for count >= s * tiles with acquire loads before touching the
// member.  All blocks are co-resident (cooperative launch) and every item a
// wait depends on was handed out earlier to a running block, so every wait is
// eventually satisfied; it is nevertheless bounded in time and sets a status
// word (and releases every other waiter) if it runs out.  Which block runs an
// item does not change what the item computes.
//
// Double buffering: step s reads buf[(cur + s) & 1] and writes the other
// buffer; the member barrier makes every read of step s - 1 precede every
// write of step s + 1 to the same buffer.
#include "dugks_tile.cuh"
#include "kin.h"
#include "kin_internal.h"
#include "kin_sim.h"
#include "lbe_node.cuh"

#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cstddef>
#include <map>
#include <vector>

namespace kin {

struct EnsMember {
    float* buf[2];
    int N, scheme, cur, ntiles;
    int tiles_x, tiles_y, zchunk;
    int lbe_nodes;  // nodes per LBE item
    MrtRates<float> rates;
    DugksCoef<float> coef;
};

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void red_release_add(unsigned* p, unsigned v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_relaxed(const int* p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

template <int TY>
__global__ void __launch_bounds__(32 * (TY + 2), 1)
    ensemble_kernel(const EnsMember* __restrict__ mem, const int2* __restrict__ items, int nitems,
                    int nsteps, unsigned* done, unsigned* next_item, int* status, long long wait_cycles,
                    int stall_test) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_abort;
    __shared__ unsigned s_idx;
    const int tid = threadIdx.y * 32 + threadIdx.x;
    constexpr int NT = 32 * (TY + 2);
    // Blocks take (step, item) pairs in order from a global counter: every
    // item of step s is handed out before any of step s + 1, so an item only
    // waits on items already running in resident blocks.
    const unsigned total = (unsigned)nsteps * (unsigned)nitems;
    for (;;) {
        if (tid == 0) s_idx = atomicAdd(next_item, 1u);
        __syncthreads();
        const unsigned idx = s_idx;
        if (idx >= total) return;
        {
            const int s = (int)(idx / (unsigned)nitems), it = (int)(idx % (unsigned)nitems);
            const int2 item = items[it];
            const EnsMember& M = mem[item.x];
            if (tid == 0) {
                int abort = ld_relaxed(status) != 0;
                // stall_test raises the target of step 1 beyond reach, to
                // exercise the bounded wait
                const unsigned target = (unsigned)s * (unsigned)M.ntiles + (stall_test && s == 1 ? 1u : 0u);
                if (!abort && s > 0) {
                    const long long t0 = clock64();
                    while (ld_acquire(&done[item.x]) < target) {
                        if (ld_relaxed(status) != 0) {
                            abort = 1;
                            break;
                        }
                        if (clock64() - t0 > wait_cycles) {
                            atomicCAS(status, 0, 1);
                            abort = 1;
                            break;
                        }
                        __nanosleep(100);
                    }
                }
                s_abort = abort;
            }
            __syncthreads();
            if (s_abort) return;
            const int par = (M.cur + s) & 1;
            const float* src = M.buf[par];
            float* dst = M.buf[par ^ 1];
            const int N = M.N;
            if (M.scheme == KIN_LBE_MRT) {
                const size_t plane = (size_t)N * N * N;
                // N <= 1024, so node indices fit in 32 bits
                const int c0 = item.y * M.lbe_nodes;
                const int c1 = (int)min((long long)c0 + M.lbe_nodes, (long long)plane);
                constexpr int K = 3;  // nodes per thread in flight
                const MrtRates<float> rates = M.rates;
                int c = c0 + tid;
                for (; c + (K - 1) * NT < c1; c += K * NT) {
                    int cs[K];
#pragma unroll
                    for (int k = 0; k < K; ++k) cs[k] = c + k * NT;
                    lbe_nodes<K, float, true>(src, dst, N, plane, cs, rates);
                }
                for (; c < c1; c += NT) {
                    const int cs[1] = {c};
                    lbe_nodes<1, float, true>(src, dst, N, plane, cs, rates);
                }
            } else {
                const int per = M.tiles_x * M.tiles_y;
                const int bz = item.y / per, r = item.y % per;
                // a local copy of the member's coefficients: passed as a
                // reference into the member table in global memory, the items
                // ran 13 % slower
                const DugksCoef<float> kc = M.coef;
                dugks_tile<float, TY>(src, dst, N, r % M.tiles_x, r / M.tiles_x, bz, M.zchunk, kc, smem_raw);
            }
            __syncthreads();
            if (tid == 0) red_release_add(&done[item.x], 1u);
        }
    }
}

KIN_DEBUG_ACCESSOR(debug_word_ensemble)

}  // namespace kin

using namespace kin;

struct kin_ensemble {
    std::vector<kin_sim*> members;
    int device = 0;
    cudaStream_t stream = nullptr;
    int tile_y = 8, zchunk = 16, lbe_nodes = 4096;
    EnsMember* d_mem = nullptr;
    int2* d_items = nullptr;
    unsigned* d_done = nullptr;
    int* d_status = nullptr;
    int nitems = 0;
    int grid = 0;
    double wait_seconds = 10.0;
    // graph cache keyed by step count
    std::map<int, cudaGraphExec_t> graphs;
    int64_t launches = 0;
    std::vector<EnsMember> h_table;  // host copy of the last table sent
};

namespace {

int ens_fail(int code, const char* what, cudaError_t e) {
    return set_error(code, "%s: %s", what, cudaGetErrorString(e));
}

#define ECK(call)                                                                      \
    do {                                                                               \
        cudaError_t e_ = (call);                                                       \
        if (e_ != cudaSuccess) return ens_fail(KIN_ECUDA, #call, e_);                  \
    } while (0)

void drop_graphs(kin_ensemble* e) {
    for (auto& kv : e->graphs) cudaGraphExecDestroy(kv.second);
    e->graphs.clear();
}

template <int TY>
int configure(kin_ensemble* e) {
    const size_t smem = fused_smem_bytes<float, TY>();
    ECK(cudaFuncSetAttribute(ensemble_kernel<TY>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0, nsm = 0;
    ECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ensemble_kernel<TY>, 32 * (TY + 2), smem));
    ECK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, e->device));
    if (per_sm < 1) return set_error(KIN_ECUDA, "ensemble kernel does not fit on an SM");
    e->grid = std::min(per_sm * nsm, std::max(e->nitems, 1));
    return KIN_OK;
}

// Member table from the members' current state (buffers, parity, nu, dt).
std::vector<EnsMember> member_table(const kin_ensemble* e) {
    std::vector<EnsMember> tab(e->members.size());
    for (size_t m = 0; m < e->members.size(); ++m) {
        const kin_sim* s = e->members[m];
        EnsMember& M = tab[m];
        M.buf[0] = (float*)s->buf[0];
        M.buf[1] = (float*)s->buf[1];
        M.N = s->N;
        M.scheme = s->scheme;
        M.cur = s->cur;
        M.rates = lbe_rates<float>(s->nu);
        M.coef = dugks_coef<float>(s->nu, s->dt);
        if (s->scheme == KIN_LBE_MRT) {
            const long long n = (long long)s->N * s->N * s->N;
            M.lbe_nodes = e->lbe_nodes;
            M.ntiles = (int)((n + e->lbe_nodes - 1) / e->lbe_nodes);
            M.tiles_x = M.tiles_y = M.zchunk = 0;
        } else {
            const int zc = std::min(e->zchunk, s->N);
            M.tiles_x = (s->N + 29) / 30;
            M.tiles_y = (s->N + e->tile_y - 1) / e->tile_y;
            M.zchunk = zc;
            M.ntiles = M.tiles_x * M.tiles_y * ((s->N + zc - 1) / zc);
            M.lbe_nodes = 0;
        }
    }
    return tab;
}

// Work list for the current tuning; items of big members first so their long
// critical paths start early.
int build_tables(kin_ensemble* e) {
    const std::vector<EnsMember> tab = member_table(e);
    std::vector<int> order(e->members.size());
    for (size_t m = 0; m < order.size(); ++m) order[m] = (int)m;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        return e->members[a]->N > e->members[b]->N;
    });
    std::vector<int2> items;
    for (int m : order)
        for (int t = 0; t < tab[m].ntiles; ++t) items.push_back(make_int2(m, t));
    if (e->d_items) cudaFree(e->d_items);
    e->d_items = nullptr;
    e->nitems = (int)items.size();
    ECK(cudaMalloc(&e->d_items, sizeof(int2) * std::max<size_t>(items.size(), 1)));
    ECK(cudaMemcpy(e->d_items, items.data(), sizeof(int2) * items.size(), cudaMemcpyHostToDevice));
    drop_graphs(e);
    return e->tile_y == 4 ? configure<4>(e) : configure<8>(e);
}

long long wait_cycles(const kin_ensemble* e) {
    int khz = 0;
    cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, e->device);
    if (khz <= 0) khz = 2000000;
    return (long long)(e->wait_seconds * 1e3 * khz);
}

int launch(kin_ensemble* e, int nsteps, int stall_test) {
    const size_t smem = e->tile_y == 4 ? fused_smem_bytes<float, 4>() : fused_smem_bytes<float, 8>();
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(e->grid);
    cfg.blockDim = dim3(32, e->tile_y + 2);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = e->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const long long wc = wait_cycles(e);
    cudaError_t err;
    if (e->tile_y == 4)
        err = cudaLaunchKernelEx(&cfg, ensemble_kernel<4>, (const EnsMember*)e->d_mem, (const int2*)e->d_items,
                                 e->nitems, nsteps, e->d_done, e->d_done + e->members.size(), e->d_status,
                                 wc, stall_test);
    else
        err = cudaLaunchKernelEx(&cfg, ensemble_kernel<8>, (const EnsMember*)e->d_mem, (const int2*)e->d_items,
                                 e->nitems, nsteps, e->d_done, e->d_done + e->members.size(), e->d_status,
                                 wc, stall_test);
    if (err != cudaSuccess) return ens_fail(KIN_ECUDA, "ensemble launch", err);
    return KIN_OK;
}

int sync_members(kin_ensemble* e) {
    for (kin_sim* s : e->members) ECK(cudaStreamSynchronize(s->stream));
    return KIN_OK;
}

int refresh_table(kin_ensemble* e) {
    e->h_table = member_table(e);
    ECK(cudaMemcpyAsync(e->d_mem, e->h_table.data(), sizeof(EnsMember) * e->h_table.size(),
                        cudaMemcpyHostToDevice, e->stream));
    return KIN_OK;
}

int run(kin_ensemble* e, int nsteps, int stall_test) {
    if (int r = sync_members(e)) return r;
    if (int r = refresh_table(e)) return r;
    if (stall_test) {
        ECK(cudaMemsetAsync(e->d_done, 0, sizeof(unsigned) * (e->members.size() + 1), e->stream));
        ECK(cudaMemsetAsync(e->d_status, 0, sizeof(int), e->stream));
        if (int r = launch(e, nsteps, 1)) return r;
    } else {
        auto it = e->graphs.find(nsteps);
        if (it == e->graphs.end()) {
            cudaGraph_t g = nullptr;
            ECK(cudaStreamBeginCapture(e->stream, cudaStreamCaptureModeThreadLocal));
            cudaMemsetAsync(e->d_done, 0, sizeof(unsigned) * (e->members.size() + 1), e->stream);
            cudaMemsetAsync(e->d_status, 0, sizeof(int), e->stream);
            const int rl = launch(e, nsteps, 0);
            cudaError_t ce = cudaStreamEndCapture(e->stream, &g);
            if (rl != KIN_OK) {
                if (g) cudaGraphDestroy(g);
                return rl;
            }
            if (ce != cudaSuccess) return ens_fail(KIN_ECUDA, "graph capture", ce);
            cudaGraphExec_t ex = nullptr;
            ce = cudaGraphInstantiate(&ex, g, 0);
            cudaGraphDestroy(g);
            if (ce != cudaSuccess) return ens_fail(KIN_ECUDA, "graph instantiate", ce);
            it = e->graphs.emplace(nsteps, ex).first;
        }
        ECK(cudaGraphLaunch(it->second, e->stream));
    }
    int status = 0;
    ECK(cudaMemcpyAsync(&status, e->d_status, sizeof(int), cudaMemcpyDeviceToHost, e->stream));
    ECK(cudaStreamSynchronize(e->stream));
    e->launches += 1;
    if (status != 0) {
        // items of several steps may have run: no member's state is known to
        // be a whole step, so every member refuses work until it is set again
        for (kin_sim* s : e->members) s->invalid = true;
        return set_error(KIN_ETIMEOUT, "ensemble member barrier timed out; the members' states are undefined");
    }
    for (kin_sim* s : e->members) {
        s->cur ^= (nsteps & 1);
        s->step += nsteps;
        s->epoch += 1;
    }
    return KIN_OK;
}

}  // namespace

extern "C" {

int kin_ensemble_create(kin_sim* const* members, int n, kin_ensemble** out) {
    if (!out || n <= 0 || !members) return set_error(KIN_EINVAL, "bad ensemble arguments");
    *out = nullptr;
    int dev = -1;
    for (int m = 0; m < n; ++m) {
        const kin_sim* s = members[m];
        if (!s) return set_error(KIN_EINVAL, "NULL member %d", m);
        if (s->storage != KIN_F32) return set_error(KIN_EINVAL, "ensemble members must use KIN_F32 storage");
        if (dev >= 0 && s->device != dev) return set_error(KIN_EINVAL, "members on different devices");
        dev = s->device;
        for (int k = 0; k < m; ++k)
            if (members[k] == s) return set_error(KIN_EINVAL, "member %d listed twice", m);
    }
    kin_ensemble* e = new kin_ensemble();
    e->members.assign(members, members + n);
    e->device = dev;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(dev);
    auto bail = [&](int code) {
        kin_ensemble_destroy(e);
        cudaSetDevice(prev);
        return code;
    };
    cudaError_t c;
    if ((c = cudaStreamCreateWithFlags(&e->stream, cudaStreamNonBlocking)) != cudaSuccess)
        return bail(ens_fail(KIN_ECUDA, "stream", c));
    if ((c = cudaMalloc(&e->d_mem, sizeof(EnsMember) * n)) != cudaSuccess) return bail(ens_fail(KIN_ENOMEM, "table", c));
    // one completion counter per member, then the work counter
    if ((c = cudaMalloc(&e->d_done, sizeof(unsigned) * (n + 1))) != cudaSuccess)
        return bail(ens_fail(KIN_ENOMEM, "counters", c));
    if ((c = cudaMalloc(&e->d_status, sizeof(int))) != cudaSuccess) return bail(ens_fail(KIN_ENOMEM, "status", c));
    if (int r = build_tables(e)) return bail(r);
    cudaSetDevice(prev);
    *out = e;
    return KIN_OK;
}

int kin_ensemble_set_tuning(kin_ensemble* e, int tile_y, int zchunk, int lbe_nodes) {
    if (!e) return set_error(KIN_EINVAL, "NULL ensemble");
    if (tile_y > 0 && tile_y != 4 && tile_y != 8) return set_error(KIN_EINVAL, "tile_y must be 4 or 8");
    if (lbe_nodes > 0 && lbe_nodes % 32) return set_error(KIN_EINVAL, "lbe_nodes must be a multiple of 32");
    if (tile_y > 0) e->tile_y = tile_y;
    if (zchunk > 0) e->zchunk = zchunk;
    if (lbe_nodes > 0) e->lbe_nodes = lbe_nodes;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(e->device);
    const int r = build_tables(e);
    cudaSetDevice(prev);
    return r;
}

int kin_ensemble_step(kin_ensemble* e, int nsteps) {
    if (!e) return set_error(KIN_EINVAL, "NULL ensemble");
    if (nsteps < 0) return set_error(KIN_EINVAL, "negative step count");
    if (nsteps == 0) return KIN_OK;
    for (const kin_sim* s : e->members)
        if (s->invalid) return set_error(KIN_ESTATE, "a member's state is undefined (set it again first)");
    nvtxRangePushA("kin_ensemble_step");
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(e->device);
    // the kernel numbers (step, item) pairs and member progress in 32 bits:
    // split the steps into launches of at most max_steps
    const unsigned long long max_steps =
        std::max<unsigned long long>(1, (0xffffffffull - (unsigned long long)e->grid) / std::max(e->nitems, 1));
    int r = KIN_OK;
    for (long long left = nsteps; left > 0 && r == KIN_OK;) {
        const int n = (int)std::min<unsigned long long>((unsigned long long)left, max_steps);
        r = run(e, n, 0);
        left -= n;
    }
    cudaSetDevice(prev);
    nvtxRangePop();
    return r;
}

int kin_ensemble_test_timeout(kin_ensemble* e, double seconds) {
    if (!e || !(seconds > 0.0)) return set_error(KIN_EINVAL, "bad arguments");
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(e->device);
    const double keep = e->wait_seconds;
    e->wait_seconds = seconds;
    const int r = run(e, 2, 1);
    e->wait_seconds = keep;
    cudaSetDevice(prev);
    return r;
}

int kin_ensemble_info(const kin_ensemble* e, int* nitems, int* grid, int64_t* launches) {
    if (!e) return set_error(KIN_EINVAL, "NULL ensemble");
    if (nitems) *nitems = e->nitems;
    if (grid) *grid = e->grid;
    if (launches) *launches = e->launches;
    return KIN_OK;
}

void kin_ensemble_destroy(kin_ensemble* e) {
    if (!e) return;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(e->device);
    if (e->stream) cudaStreamSynchronize(e->stream);
    drop_graphs(e);
    if (e->d_items) cudaFree(e->d_items);
    if (e->d_mem) cudaFree(e->d_mem);
    if (e->d_done) cudaFree(e->d_done);
    if (e->d_status) cudaFree(e->d_status);
    if (e->stream) cudaStreamDestroy(e->stream);
    cudaSetDevice(prev);
    delete e;
}

}  // extern "C"
