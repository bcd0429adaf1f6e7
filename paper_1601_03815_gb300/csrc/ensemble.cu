// Ensemble of independent simulations advanced together by one CUDA graph
// launch per kin_ensemble_step call.
//
// DUGKS members: one persistent, cooperative kernel runs all their steps.  The
// work of one time step is a list of items (member, tile) of the fused step
// (dugks_tile.cuh).  Thread blocks take (step, item) pairs one at a time from
// a global counter, all items of step s before any of step s + 1.  A member's
// step s may start only when all its tiles of step s - 1 are done: each
// finished tile adds one to the member's counter with a GPU-scope release, and
// a block waits for count >= s * tiles with acquire loads before touching the
// member.  Every item a wait depends on was handed out earlier to a running
// block, so every wait is eventually satisfied whether or not all blocks are
// resident; it is nevertheless bounded in time and sets a status word (and
// releases every other waiter) if it runs out.
//
// LBE members: one batched launch per step covers every LBE member of a
// storage type (a block takes consecutive nodes of one member), on a second
// stream of the same graph.  With both schemes present the persistent kernel
// runs 6-row tiles (8 warps, 160 KB of shared memory, at most 160 registers
// a thread), which leave room for three 4-warp FP32 LBE blocks (56 registers
// a thread, no shared memory) on each SM: the memory-bound LBE nodes use the
// bandwidth and issue slots that the issue-bound DUGKS tiles leave.  The two
// kernels never wait on each other; consecutive LBE steps are ordered by
// their stream.
//
// Which block runs an item does not change what it computes: a member's
// results are bitwise those of stepping it alone.
//
// Double buffering: step s reads buf[(cur + s) & 1] and writes the other
// buffer; the member barrier (DUGKS) or the stream order (LBE) makes every
// read of step s - 1 precede every write of step s + 1 to the same buffer.
#include "dugks_tile.cuh"
#include "kin.h"
#include "kin_internal.h"
#include "kin_sim.h"
#include "lbe_node.cuh"

#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <climits>
#include <cstddef>
#include <map>
#include <vector>

namespace kin {

// DUGKS member of the persistent kernel
struct EnsMember {
    void* buf[2];
    int N, storage, cur, ntiles;
    int tiles_x, tiles_y, zchunk;
    DugksCoef<float> coef;
};

// LBE member of the batched launch of its storage type
struct LbeMember {
    void* buf[2];
    int N, cur, V;    // V consecutive cells a thread (as the standalone LBE step)
    unsigned block0;  // its first block in the batched grid
    MrtRates<float> rates;
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

// One fused-DUGKS tile t of member M at buffer parity par.
template <typename S, int TY>
__device__ __forceinline__ void ensemble_tile(const EnsMember& M, int par, int t, unsigned char* smem_raw) {
    const int per = M.tiles_x * M.tiles_y;
    const int bz = t / per, r = t % per;
    // a local copy of the member's coefficients: passed as a reference into
    // the member table in global memory, the items ran 13 % slower
    const DugksCoef<float> kc = M.coef;
    dugks_tile<S, TY>(static_cast<const S*>(M.buf[par]), static_cast<S*>(M.buf[par ^ 1]), M.N, r % M.tiles_x,
                      r / M.tiles_x, bz, M.zchunk, kc, smem_raw);
}

// WIDE: some member has 2-byte storage (even N); without it the kernel holds
// only the FP32 tile and its registers.
template <int TY, bool WIDE>
__device__ __forceinline__ void ensemble_body(const EnsMember* __restrict__ mem, const int2* __restrict__ items,
                                              int nitems, int nsteps, unsigned* done, unsigned* next_item,
                                              int* status, long long wait_cycles, int stall_test) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_abort;
    __shared__ unsigned s_idx;
    const int tid = threadIdx.y * 32 + threadIdx.x;
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
            if constexpr (WIDE) {
                if (M.storage == ST_F16) ensemble_tile<__half, TY>(M, par, item.y, smem_raw);
                else if (M.storage == ST_BF16) ensemble_tile<__nv_bfloat16, TY>(M, par, item.y, smem_raw);
                else ensemble_tile<float, TY>(M, par, item.y, smem_raw);
            } else {
                ensemble_tile<float, TY>(M, par, item.y, smem_raw);
            }
            __syncthreads();
            if (tid == 0) red_release_add(&done[item.x], 1u);
        }
    }
}

#define KIN_ENSEMBLE_PARAMS                                                                            \
    const EnsMember *__restrict__ mem, const int2 *__restrict__ items, int nitems, int nsteps, unsigned *done, \
        unsigned *next_item, int *status, long long wait_cycles, int stall_test

template <int TY, bool WIDE>
__global__ void __launch_bounds__(32 * (TY + 2), 1) ensemble_kernel(KIN_ENSEMBLE_PARAMS) {
    ensemble_body<TY, WIDE>(mem, items, nitems, nsteps, done, next_item, status, wait_cycles, stall_test);
}

// 6-row tiles, the form beside which LBE blocks run: held to 160 registers a
// thread (152 used; at the compiler's free choice it takes 214), so that the
// 8-warp block leaves most of the SM's registers to the LBE blocks.
template <bool WIDE>
__global__ void __maxnreg__(160) ensemble_kernel6(KIN_ENSEMBLE_PARAMS) {
    ensemble_body<6, WIDE>(mem, items, nitems, nsteps, done, next_item, status, wait_cycles, stall_test);
}

template <int TY, bool WIDE>
constexpr auto ensemble_kernel_for() {
    if constexpr (TY == 6) return ensemble_kernel6<WIDE>;
    else return ensemble_kernel<TY, WIDE>;
}

// One LBE step of every member in tab[0 .. nmem) (one storage type): block b
// belongs to the member with the largest block0 <= b and takes blockDim.x * V
// consecutive cells of it (linear index x + N (y + N z)); each thread updates V
// cells of one row exactly as the standalone LBE step does.  FP32 blocks are
// held to 56 registers a thread, so that two 128-thread blocks fit beside a
// DUGKS block (the 2-byte vector forms would spill there).
template <typename S>
__global__ void __launch_bounds__(128, sizeof(S) == 4 ? 9 : 1) lbe_batch_kernel(const LbeMember* __restrict__ tab, int nmem, int step) {
    const unsigned b = blockIdx.x;
    int lo = 0, hi = nmem - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (tab[mid].block0 <= b) lo = mid;
        else hi = mid - 1;
    }
    const LbeMember& M = tab[lo];
    const int N = M.N, V = M.V;
    // N <= 1024: cell indices fit in 32 bits
    const unsigned n3 = (unsigned)N * N * N, nn = (unsigned)N * N;
    const unsigned c = ((b - M.block0) * blockDim.x + threadIdx.x) * V;
    if (c >= n3) return;
    const size_t plane = n3;
    const int z = (int)(c / nn), r = (int)(c - z * nn), y = r / N, x = r - y * N;
    const int par = (M.cur + step) & 1;
    const S* src = static_cast<const S*>(M.buf[par]);
    S* dst = static_cast<S*>(M.buf[par ^ 1]);
    const MrtRates<float> rates = M.rates;
    if constexpr (sizeof(S) == 2) {
        if (V == 4) return lbe_vnode4p<S>(src, dst, N, plane, x, y, z, rates);
        if (V == 2) return lbe_vnode<S, 2>(src, dst, N, plane, x, y, z, rates);
    }
    lbe_node<S, false>(src, dst, N, plane, x, y, z, rates);
}

KIN_DEBUG_ACCESSOR(debug_word_ensemble)

}  // namespace kin

using namespace kin;

struct kin_ensemble {
    std::vector<kin_sim*> members;
    std::vector<int> dugks_ids, lbe_ids;  // members of each scheme, in member order
    bool wide = false;                    // a DUGKS member has 2-byte storage
    int device = 0;
    cudaStream_t stream = nullptr;  // persistent DUGKS launch (and the graph's origin)
    cudaStream_t side = nullptr;    // batched LBE launches inside the graph
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // tile_y 6 (8 warps a DUGKS block) when both schemes are present, else 8;
    // see kin_ensemble_create
    int tile_y = 8, zchunk = 16, lbe_block = 128;
    EnsMember* d_mem = nullptr;
    LbeMember* d_lbe = nullptr;
    int2* d_items = nullptr;
    unsigned* d_done = nullptr;
    int* d_status = nullptr;
    int nitems = 0;  // DUGKS items per step
    int grid = 0;    // blocks of the persistent launch
    // batched LBE launches, one per storage type (FP32, FP16, BF16): their
    // members' range in the LBE table and their blocks per step
    int lbe_off[3] = {0, 0, 0}, lbe_count[3] = {0, 0, 0};
    unsigned lbe_blocks[3] = {0, 0, 0};
    double wait_seconds = 10.0;
    // graph cache keyed by step count
    std::map<int, cudaGraphExec_t> graphs;
    int64_t launches = 0;
};

namespace {

// Steps per graph when there are LBE members (one kernel node each).
constexpr int kMaxGraphSteps = 256;

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

template <int TY, bool WIDE>
size_t persistent_smem() {
    return WIDE ? std::max(fused_smem_bytes<float, TY>(),
                           std::max(fused_smem_bytes<__half, TY>(), fused_smem_bytes<__nv_bfloat16, TY>()))
                : fused_smem_bytes<float, TY>();
}

template <int TY, bool WIDE>
int configure(kin_ensemble* e) {
    const size_t smem = persistent_smem<TY, WIDE>();
    ECK(cudaFuncSetAttribute(ensemble_kernel_for<TY, WIDE>(), cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem));
    int per_sm = 0, nsm = 0;
    ECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ensemble_kernel_for<TY, WIDE>(), 32 * (TY + 2),
                                                      smem));
    ECK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, e->device));
    if (per_sm < 1) return set_error(KIN_ECUDA, "ensemble kernel does not fit on an SM");
    e->grid = std::min(per_sm * nsm, std::max(e->nitems, 1));
    return KIN_OK;
}

int storage_group(int storage) { return storage == ST_F16 ? 1 : storage == ST_BF16 ? 2 : 0; }

// Cells a thread of the batched LBE launch updates: as the standalone step.
int lbe_vector(const kin_sim* s) {
    if (s->storage == ST_F32) return 1;
    return s->N % 4 == 0 ? 4 : s->N % 2 == 0 ? 2 : 1;
}

// DUGKS table from the members' current state (buffers, parity, nu, dt).
std::vector<EnsMember> dugks_table(const kin_ensemble* e) {
    std::vector<EnsMember> tab(e->dugks_ids.size());
    for (size_t d = 0; d < tab.size(); ++d) {
        const kin_sim* s = e->members[e->dugks_ids[d]];
        EnsMember& M = tab[d];
        M.buf[0] = s->buf[0];
        M.buf[1] = s->buf[1];
        M.N = s->N;
        M.storage = s->storage;
        M.cur = s->cur;
        M.coef = dugks_coef<float>(s->nu, s->dt);
        const int zc = std::min(e->zchunk, s->N);
        M.tiles_x = (s->N + 29) / 30;
        M.tiles_y = (s->N + e->tile_y - 1) / e->tile_y;
        M.zchunk = zc;
        M.ntiles = M.tiles_x * M.tiles_y * ((s->N + zc - 1) / zc);
    }
    return tab;
}

// LBE table, grouped by storage type (FP32, FP16, BF16), each group's blocks
// numbered from 0; fills the group ranges of e.
std::vector<LbeMember> lbe_table(kin_ensemble* e) {
    std::vector<LbeMember> tab;
    for (int g = 0; g < 3; ++g) {
        e->lbe_off[g] = (int)tab.size();
        unsigned long long blocks = 0;
        for (int m : e->lbe_ids) {
            const kin_sim* s = e->members[m];
            if (storage_group(s->storage) != g) continue;
            LbeMember L;
            L.buf[0] = s->buf[0];
            L.buf[1] = s->buf[1];
            L.N = s->N;
            L.cur = s->cur;
            L.V = lbe_vector(s);
            L.block0 = (unsigned)blocks;
            L.rates = lbe_rates<float>(s->nu);
            const unsigned long long threads = (unsigned long long)s->N * s->N * s->N / L.V;
            blocks += (threads + e->lbe_block - 1) / e->lbe_block;
            tab.push_back(L);
        }
        e->lbe_count[g] = (int)tab.size() - e->lbe_off[g];
        e->lbe_blocks[g] = (unsigned)std::min<unsigned long long>(blocks, 0xffffffffull);
    }
    return tab;
}

int launch_persistent_config(kin_ensemble* e) {
    if (e->nitems == 0) {
        e->grid = 0;
        return KIN_OK;
    }
    if (e->tile_y == 4) return e->wide ? configure<4, true>(e) : configure<4, false>(e);
    if (e->tile_y == 6) return e->wide ? configure<6, true>(e) : configure<6, false>(e);
    return e->wide ? configure<8, true>(e) : configure<8, false>(e);
}

// Work list for the current tuning; items of big members first so their long
// critical paths start early.
int build_tables(kin_ensemble* e) {
    const std::vector<EnsMember> tab = dugks_table(e);
    std::vector<int> order(tab.size());
    for (size_t d = 0; d < order.size(); ++d) order[d] = (int)d;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return tab[a].N > tab[b].N; });
    std::vector<int2> items;
    for (int d : order)
        for (int t = 0; t < tab[d].ntiles; ++t) items.push_back(make_int2(d, t));
    if (e->d_items) cudaFree(e->d_items);
    e->d_items = nullptr;
    e->nitems = (int)items.size();
    ECK(cudaMalloc(&e->d_items, sizeof(int2) * std::max<size_t>(items.size(), 1)));
    if (!items.empty())
        ECK(cudaMemcpy(e->d_items, items.data(), sizeof(int2) * items.size(), cudaMemcpyHostToDevice));
    lbe_table(e);
    for (int g = 0; g < 3; ++g)
        if (e->lbe_blocks[g] > (unsigned)INT_MAX)
            return set_error(KIN_EINVAL, "the LBE members need more than 2^31 - 1 thread blocks a step");
    drop_graphs(e);
    return launch_persistent_config(e);
}

long long wait_cycles(const kin_ensemble* e) {
    int khz = 0;
    cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, e->device);
    if (khz <= 0) khz = 2000000;
    return (long long)(e->wait_seconds * 1e3 * khz);
}

template <int TY, bool WIDE>
cudaError_t launch_persistent_t(kin_ensemble* e, int nsteps, int stall_test) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(e->grid);
    cfg.blockDim = dim3(32, TY + 2);
    cfg.dynamicSmemBytes = persistent_smem<TY, WIDE>();
    cfg.stream = e->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const int nd = (int)e->dugks_ids.size();
    return cudaLaunchKernelEx(&cfg, ensemble_kernel_for<TY, WIDE>(), (const EnsMember*)e->d_mem,
                              (const int2*)e->d_items, e->nitems, nsteps, e->d_done, e->d_done + nd, e->d_status,
                              wait_cycles(e), stall_test);
}

int launch_persistent(kin_ensemble* e, int nsteps, int stall_test) {
    cudaError_t err;
    if (e->tile_y == 4)
        err = e->wide ? launch_persistent_t<4, true>(e, nsteps, stall_test)
                      : launch_persistent_t<4, false>(e, nsteps, stall_test);
    else if (e->tile_y == 6)
        err = e->wide ? launch_persistent_t<6, true>(e, nsteps, stall_test)
                      : launch_persistent_t<6, false>(e, nsteps, stall_test);
    else
        err = e->wide ? launch_persistent_t<8, true>(e, nsteps, stall_test)
                      : launch_persistent_t<8, false>(e, nsteps, stall_test);
    if (err != cudaSuccess) return ens_fail(KIN_ECUDA, "ensemble launch", err);
    return KIN_OK;
}

// Step `step` (counted from the start of the launch) of every LBE member.
int launch_lbe(kin_ensemble* e, int step, cudaStream_t stream) {
    for (int g = 0; g < 3; ++g) {
        if (e->lbe_count[g] == 0) continue;
        const LbeMember* tab = e->d_lbe + e->lbe_off[g];
        const dim3 grid(e->lbe_blocks[g]), block(e->lbe_block);
        if (g == 0) lbe_batch_kernel<float><<<grid, block, 0, stream>>>(tab, e->lbe_count[g], step);
        else if (g == 1) lbe_batch_kernel<__half><<<grid, block, 0, stream>>>(tab, e->lbe_count[g], step);
        else lbe_batch_kernel<__nv_bfloat16><<<grid, block, 0, stream>>>(tab, e->lbe_count[g], step);
        const cudaError_t err = cudaGetLastError();
        if (err != cudaSuccess) return ens_fail(KIN_ECUDA, "batched LBE launch", err);
    }
    return KIN_OK;
}

int sync_members(kin_ensemble* e) {
    for (kin_sim* s : e->members) ECK(cudaStreamSynchronize(s->stream));
    return KIN_OK;
}

int refresh_tables(kin_ensemble* e) {
    static_assert(sizeof(EnsMember) % 8 == 0 && sizeof(LbeMember) % 8 == 0, "table entries hold pointers");
    const std::vector<EnsMember> d = dugks_table(e);
    const std::vector<LbeMember> l = lbe_table(e);
    if (!d.empty())
        ECK(cudaMemcpyAsync(e->d_mem, d.data(), sizeof(EnsMember) * d.size(), cudaMemcpyHostToDevice, e->stream));
    if (!l.empty())
        ECK(cudaMemcpyAsync(e->d_lbe, l.data(), sizeof(LbeMember) * l.size(), cudaMemcpyHostToDevice, e->stream));
    // the copies read the host vectors: finish them before they go out of scope
    ECK(cudaStreamSynchronize(e->stream));
    return KIN_OK;
}

// Graph of nsteps steps: the persistent DUGKS launch on e->stream and, forked
// onto e->side, one batched LBE launch per step.
int capture(kin_ensemble* e, int nsteps, cudaGraphExec_t* out) {
    const int nd = (int)e->dugks_ids.size();
    const bool dugks = e->nitems > 0, lbe = !e->lbe_ids.empty();
    const bool fork = dugks && lbe;
    cudaGraph_t g = nullptr;
    ECK(cudaStreamBeginCapture(e->stream, cudaStreamCaptureModeThreadLocal));
    int rl = KIN_OK;
    cudaError_t ce = cudaSuccess;
    if (dugks) {
        ce = cudaMemsetAsync(e->d_done, 0, sizeof(unsigned) * (nd + 1), e->stream);
        if (ce == cudaSuccess) ce = cudaMemsetAsync(e->d_status, 0, sizeof(int), e->stream);
    }
    cudaStream_t lbe_stream = e->stream;
    if (fork && ce == cudaSuccess) {
        ce = cudaEventRecord(e->ev_fork, e->stream);
        if (ce == cudaSuccess) ce = cudaStreamWaitEvent(e->side, e->ev_fork, 0);
        lbe_stream = e->side;
    }
    if (ce != cudaSuccess) rl = ens_fail(KIN_ECUDA, "graph capture", ce);
    if (rl == KIN_OK && dugks) rl = launch_persistent(e, nsteps, 0);
    for (int s = 0; s < nsteps && rl == KIN_OK && lbe; ++s) rl = launch_lbe(e, s, lbe_stream);
    if (fork) {
        // join the side stream even after an error, so the capture can end
        cudaEventRecord(e->ev_join, e->side);
        cudaStreamWaitEvent(e->stream, e->ev_join, 0);
    }
    ce = cudaStreamEndCapture(e->stream, &g);
    if (rl != KIN_OK) {
        if (g) cudaGraphDestroy(g);
        return rl;
    }
    if (ce != cudaSuccess) return ens_fail(KIN_ECUDA, "graph capture", ce);
    ce = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (ce != cudaSuccess) return ens_fail(KIN_ECUDA, "graph instantiate", ce);
    return KIN_OK;
}

int run(kin_ensemble* e, int nsteps, int stall_test) {
    if (int r = sync_members(e)) return r;
    if (int r = refresh_tables(e)) return r;
    if (stall_test) {
        // the persistent launch alone, with a member barrier it cannot pass
        const int nd = (int)e->dugks_ids.size();
        ECK(cudaMemsetAsync(e->d_done, 0, sizeof(unsigned) * (nd + 1), e->stream));
        ECK(cudaMemsetAsync(e->d_status, 0, sizeof(int), e->stream));
        if (int r = launch_persistent(e, nsteps, 1)) return r;
    } else {
        auto it = e->graphs.find(nsteps);
        if (it == e->graphs.end()) {
            cudaGraphExec_t ex = nullptr;
            if (int r = capture(e, nsteps, &ex)) return r;
            it = e->graphs.emplace(nsteps, ex).first;
        }
        ECK(cudaGraphLaunch(it->second, e->stream));
    }
    int status = 0;
    if (e->nitems > 0) ECK(cudaMemcpyAsync(&status, e->d_status, sizeof(int), cudaMemcpyDeviceToHost, e->stream));
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
        if (s->storage == ST_F64)
            return set_error(KIN_EINVAL, "ensemble members use KIN_F32, KIN_F16 or KIN_BF16 storage");
        if (s->scheme == KIN_DUGKS && s->storage != ST_F32 && s->N % 2)
            return set_error(KIN_EINVAL, "member %d: a DUGKS member with 2-byte storage needs an even N", m);
        if (dev >= 0 && s->device != dev) return set_error(KIN_EINVAL, "members on different devices");
        dev = s->device;
        for (int k = 0; k < m; ++k)
            if (members[k] == s) return set_error(KIN_EINVAL, "member %d listed twice", m);
    }
    kin_ensemble* e = new kin_ensemble();
    e->members.assign(members, members + n);
    for (int m = 0; m < n; ++m) {
        if (members[m]->scheme == KIN_DUGKS) {
            e->dugks_ids.push_back(m);
            if (members[m]->storage != ST_F32) e->wide = true;
        } else {
            e->lbe_ids.push_back(m);
        }
    }
    // Measured: LBE blocks of any size ran beside 6- and 8-warp DUGKS blocks
    // (4- and 6-row tiles) and never beside the 10-warp blocks of 8-row tiles,
    // even with those held to 152 registers a thread; so when both schemes
    // are present the DUGKS tiles have 6 rows.
    if (!e->dugks_ids.empty() && !e->lbe_ids.empty()) e->tile_y = 6;
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
    if ((c = cudaStreamCreateWithFlags(&e->side, cudaStreamNonBlocking)) != cudaSuccess)
        return bail(ens_fail(KIN_ECUDA, "stream", c));
    if ((c = cudaEventCreateWithFlags(&e->ev_fork, cudaEventDisableTiming)) != cudaSuccess ||
        (c = cudaEventCreateWithFlags(&e->ev_join, cudaEventDisableTiming)) != cudaSuccess)
        return bail(ens_fail(KIN_ECUDA, "event", c));
    if ((c = cudaMalloc(&e->d_mem, sizeof(EnsMember) * n)) != cudaSuccess) return bail(ens_fail(KIN_ENOMEM, "table", c));
    if ((c = cudaMalloc(&e->d_lbe, sizeof(LbeMember) * n)) != cudaSuccess) return bail(ens_fail(KIN_ENOMEM, "table", c));
    // one completion counter per DUGKS member, then the work counter
    if ((c = cudaMalloc(&e->d_done, sizeof(unsigned) * (n + 1))) != cudaSuccess)
        return bail(ens_fail(KIN_ENOMEM, "counters", c));
    if ((c = cudaMalloc(&e->d_status, sizeof(int))) != cudaSuccess) return bail(ens_fail(KIN_ENOMEM, "status", c));
    if (int r = build_tables(e)) return bail(r);
    cudaSetDevice(prev);
    *out = e;
    return KIN_OK;
}

int kin_ensemble_set_tuning(kin_ensemble* e, int tile_y, int zchunk, int lbe_block) {
    if (!e) return set_error(KIN_EINVAL, "NULL ensemble");
    if (tile_y > 0 && tile_y != 4 && tile_y != 6 && tile_y != 8)
        return set_error(KIN_EINVAL, "tile_y must be 4, 6 or 8");
    if (lbe_block > 0 && (lbe_block % 32 || lbe_block > 128))
        return set_error(KIN_EINVAL, "lbe_block must be a multiple of 32, at most 128");
    if (tile_y > 0) e->tile_y = tile_y;
    if (zchunk > 0) e->zchunk = zchunk;
    if (lbe_block > 0) e->lbe_block = lbe_block;
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
    // the persistent kernel numbers (step, item) pairs and member progress in
    // 32 bits, and a graph holds one LBE launch per step: split the steps
    // into launches of at most max_steps
    unsigned long long max_steps =
        std::max<unsigned long long>(1, (0xffffffffull - (unsigned long long)e->grid) / std::max(e->nitems, 1));
    if (!e->lbe_ids.empty()) max_steps = std::min<unsigned long long>(max_steps, kMaxGraphSteps);
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
    if (e->nitems == 0) return set_error(KIN_EINVAL, "no DUGKS member: the ensemble has no member barrier");
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
    if (nitems) *nitems = e->nitems + (int)(e->lbe_blocks[0] + e->lbe_blocks[1] + e->lbe_blocks[2]);
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
    if (e->side) cudaStreamSynchronize(e->side);
    drop_graphs(e);
    if (e->d_items) cudaFree(e->d_items);
    if (e->d_mem) cudaFree(e->d_mem);
    if (e->d_lbe) cudaFree(e->d_lbe);
    if (e->d_done) cudaFree(e->d_done);
    if (e->d_status) cudaFree(e->d_status);
    if (e->ev_fork) cudaEventDestroy(e->ev_fork);
    if (e->ev_join) cudaEventDestroy(e->ev_join);
    if (e->side) cudaStreamDestroy(e->side);
    if (e->stream) cudaStreamDestroy(e->stream);
    cudaSetDevice(prev);
    delete e;
}

}  // extern "C"
