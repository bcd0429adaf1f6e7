// Internal: the simulation handle behind the opaque kin_sim of kin.h.
#pragma once

#include <cufft.h>
#include <cuda_runtime.h>
#include <stdint.h>

struct kin_sim {
    int N = 0, scheme = 0, storage = 0;
    double nu = 0, Ma = 0, dt = 0;
    int device = 0;
    int num_sms = 152;  // multiprocessors of `device`, read at creation
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    void* buf[2] = {nullptr, nullptr};
    void* base[2] = {nullptr, nullptr};  // allocations: guard region, buf[k], guard region
    int cur = 0;
    void* fbp = nullptr;  // DUGKS f-bar-plus scratch
    int64_t step = 0;
    // set when an ensemble launch gave up a bounded wait part-way: the state
    // is undefined until kin_set_f, kin_set_velocity or kin_init_field
    bool invalid = false;
    // statistics scratch (lazy)
    double* u = nullptr;      // 3 N^3
    float* u32 = nullptr;     // 3 N^3, the E / eps path of FP32-computed storage
    double2* uh = nullptr;    // 3 N^2 (N/2+1)
    double* red = nullptr;    // block partials
    double* red_out = nullptr;
    size_t red_cap = 0;
    cufftHandle d2z = 0, z2d = 0, r2c = 0;
    bool have_d2z = false, have_z2d = false, have_r2c = false;
    int block_lbe = 0, block_dugks = 0;
    int tile_y = 8, zchunk = 0, variant = 0;  // zchunk 0: chosen per launch
    int zc_auto = 0, zc_auto_ty = 0;  // the chosen z chunk and the tile height it was chosen for
    int* d_err = nullptr;  // set by a kernel whose bounded wait gave up
    double* h_pin = nullptr;  // pinned host words: E, eps, and the error flag
    int64_t launches = 0;  // own kernel launches
    // state version: bumped by every step and every write of the state; u32
    // holds the velocity of the state of version u32_epoch
    uint64_t epoch = 0, u32_epoch = ~0ull;
};


namespace kin {
// Record a failure for kin_last_error(); returns code.
int set_error(int code, const char* fmt, ...);
}  // namespace kin
