// Internal interface between the libkin translation units (not installed).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace kin {

// Storage codes match enum kin_storage in kin.h.
enum { ST_F32 = 0, ST_F16 = 1, ST_BF16 = 2, ST_F64 = 3 };
enum { SC_LBE = 0, SC_DUGKS = 1 };

size_t storage_bytes(int storage);

// MRT-LBE step (Eq. 21) in the pull arrangement: the buffer holds
// buf_i(y) = f_i(y + xi_i, t) (pre-collision populations displaced by -xi_i);
// one launch reads buf_i(x - xi_i) = f_i(x, t), collides and writes the
// post-collision f*_i(x) to dst, which then holds buf for t + 1.
cudaError_t lbe_step(int storage, const void* src, void* dst, int N, double nu, int block_x,
                     cudaStream_t stream);

// DUGKS step (Eqs. 9-20).  fbp is scratch of 19 N^3 compute-type values.
cudaError_t dugks_step(int storage, const void* src, void* dst, void* fbp, int N, double nu,
                       double dt, int block_x, cudaStream_t stream);

// Fused single-launch DUGKS step; tile_y in {4, 8} (FP64 always uses 4),
// zchunk planes per CTA.
// uvel: NULL, or (FP32-computed storage) uvel[3][N^3] receives the velocity
// of the new state, bitwise equal to velocity_field32 of it.
cudaError_t dugks_step_fused(int storage, const void* src, void* dst, int N, double nu, double dt,
                             int tile_y, int zchunk, cudaStream_t stream, float* uvel = nullptr);

// The momentum reset of a DUGKS consistent-initialisation iteration: f-tilde
// (in place) gets momentum rho0 u0 (FP64 [3][N^3], device) back along the
// linear term of the equilibrium.
cudaError_t dugks_reset_momentum(int storage, void* f, int N, const double* u0, cudaStream_t stream);

// One iteration of the consistent initialisation of an LBE state (pull
// layout): the step with the momentum held at u0 (FP64 [3][N^3], device).
cudaError_t lbe_consistent_step(int storage, const void* src, void* dst, int N, double nu, const double* u0,
                                cudaStream_t stream);
// delta-rho of a state into prev (mode 0), or max |delta-rho - prev| into
// *maxbits as float bits (mode 1; *maxbits must start at 0).
cudaError_t drho_change(int storage, const void* state, bool shifted, int N, double* prev, unsigned* maxbits,
                        int mode, cudaStream_t stream);

// Compute-type size of the DUGKS scratch element (4 or 8 bytes).
size_t dugks_scratch_bytes(int storage);

// u[3][N^3] (double) of the state; `shifted` selects the LBE pull layout.
cudaError_t velocity_field(int storage, const void* state, bool shifted, int N, double* u,
                           cudaStream_t stream);

// E and eps sums: partials[2 * nblocks] then out[2] = {E, eps} (FP64, fixed
// order).  nblocks = stats_blocks(N) <= kStatsMaxBlocks (8 per SM on 152 SMs).
constexpr int kStatsMaxBlocks = 1216;
int stats_blocks(int N);
// FP32 statistics path for storage types computed in FP32 (F32, F16, BF16).
cudaError_t velocity_field32(int storage, const void* state, bool shifted, int N, float* u,
                             cudaStream_t stream);
cudaError_t energy_dissipation32(const float* u, int N, double nu, double* partials, double* out,
                                 cudaStream_t stream);
// Derived statistics: spectral derivative of one component in place, and the
// moments <d^p> (p = 2, 3, 4) of three derivative fields d[3][N^3] -> out[9].
cudaError_t derivative_multiply(double2* uh, int N, int axis, cudaStream_t stream);
cudaError_t derivative_moments(const double* d, int N, double* partial, double* out, cudaStream_t stream);
int deriv_moment_blocks(int N);
cudaError_t energy_dissipation(const double* u, int N, double nu, double* partials, double* out,
                               cudaStream_t stream);

// Shell sums of |inv * X|^2 / 2 over the half-complex arrays X of the three
// components (inv = N^-3 for raw D2Z output); with weight_n2 each mode is
// weighted by |n|^2.  partial[nblocks][nshell], out[nshell].
int spectrum_blocks(int N);
// E(k) shells from FP32 transforms (float2 half-complex, unscaled R2C output).
cudaError_t spectrum_shells32(const void* uh0, const void* uh1, const void* uh2, int N, int nshell,
                              double inv, double* partial, double* out, cudaStream_t stream);
cudaError_t spectrum_shells(const void* uh0, const void* uh1, const void* uh2, int N, int nshell,
                            double inv, int weight_n2, double* partial, double* out,
                            cudaStream_t stream);

// state = f_eq(0, u) (Eq. 7), written in the scheme's layout.
cudaError_t equilibrium_from_velocity(int storage, const double* u, bool shifted, int N,
                                      void* state, cudaStream_t stream);

// Population plane i: state <- plane (canonical FP64), or plane <- state.
cudaError_t set_population(int storage, int i, const double* plane, bool shifted, int N,
                           void* state, cudaStream_t stream);
cudaError_t get_population(int storage, int i, const void* state, bool shifted, int N,
                           double* plane, cudaStream_t stream);

// out[n][19] canonical f at cells[n].
cudaError_t sample_cells(int storage, const void* state, bool shifted, int N,
                         const int64_t* cells, int64_t n, double* out, cudaStream_t stream);

// First failed index check of a KIN_DEBUG build in the translation units of
// the fused DUGKS step, the LBE step and the ensemble kernel (0: none, or not
// a debug build); reset clears it.
cudaError_t debug_word_dugks(unsigned long long* word, bool reset);
cudaError_t debug_word_lbe(unsigned long long* word, bool reset);
cudaError_t debug_word_ensemble(unsigned long long* word, bool reset);

// Non-finite check of a double array: flag[0] |= 1 if any element is NaN/Inf.
cudaError_t scan_nonfinite(const double* v, size_t n, int* flag, cudaStream_t stream);

}  // namespace kin
