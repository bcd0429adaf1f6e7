/*
 * libkin: GB300 (sm_103a) CUDA library for the per-time-step update of the
 * D3Q19 distributions of decaying homogeneous isotropic turbulence on a
 * periodic N^3 box, with the two schemes compared by Wang, Wang & Guo,
 * "Comparison of the LBE and DUGKS methods for DNS of decaying homogeneous
 * isotropic turbulence" (arXiv:1601.03815):
 *   KIN_LBE_MRT  MRT lattice Boltzmann collide-and-stream, Sec. II.B, Eq. 21
 *   KIN_DUGKS    discrete unified gas-kinetic scheme, Sec. II.A, Eqs. 9-20
 *
 * Units: lattice units, dx = 1, c = 1, RT = c_s^2 = 1/3, rho0 = 1.
 *
 * Host array layouts (all FP64, owned by the caller, never retained):
 *   distributions  f[i][z][y][x], x fastest, 19 * N^3 doubles; population i
 *                  has velocity kin_lattice()[i]; f_i is the deviation from
 *                  W_i rho0 (Eq. 7 carries no rest part).  For KIN_LBE_MRT
 *                  this is the pre-collision f at t_n (left side of Eq. 21 at
 *                  t_n); for KIN_DUGKS it is the cell-averaged f-tilde at t_n
 *                  (Eq. 9).
 *   velocity       u[c][z][y][x], c = x, y, z, 3 * N^3 doubles.
 *
 * Every int-returning call returns KIN_OK (0) or a negative KIN_E* code;
 * kin_strerror() names the code and kin_last_error() describes the last
 * failure on the calling thread.  No call retains a host pointer beyond the
 * stream work it enqueues.  All device work is ordered on the simulation's
 * stream; calls that return host data synchronise that stream first, except
 * kin_stats_async / kin_step_stats_async, which enqueue their copy.
 */
#ifndef KIN_H
#define KIN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct kin_sim kin_sim;

enum kin_scheme { KIN_LBE_MRT = 0, KIN_DUGKS = 1 };

/* Storage precision of f in device memory.  KIN_F32/F16/BF16 compute in FP32;
 * KIN_F64 stores and computes in FP64.  Reductions (E, eps, spectrum) always
 * accumulate in FP64. */
enum kin_storage { KIN_F32 = 0, KIN_F16 = 1, KIN_BF16 = 2, KIN_F64 = 3 };

enum kin_status {
    KIN_OK = 0,
    KIN_EINVAL = -1,     /* bad argument (size, scheme, dt, NULL pointer) */
    KIN_ENOMEM = -2,     /* device allocation failed */
    KIN_ECUDA = -3,      /* a CUDA / cuFFT call failed */
    KIN_ENONFINITE = -4, /* the state holds NaN/Inf (the run blew up) */
    KIN_ETIMEOUT = -5,   /* a bounded device-side wait gave up */
    KIN_ESTATE = -6,     /* call not valid in the current state */
    KIN_EGUARD = -7,     /* a guard region around a state buffer was overwritten */
    KIN_EDEBUG = -8      /* an index check of the debug build failed */
};

/* D3Q19 velocity set (Sec. II.A, Eq. 5) in the population order used by every
 * array of this library: xi[3*i + a], i = 0..18, and weights w[19]. */
int kin_lattice(int* xi, double* w);

/* Bytes of device memory a simulation of this size holds after kin_create
 * (state buffers only; statistics add 3*N^3 doubles on first use, the
 * spectrum a further 3*N^2*(N/2+1) complex doubles). */
size_t kin_footprint_bytes(int N, int scheme, int storage);

/* Create a simulation on the current CUDA device.
 *   N        box edge, 2 <= N <= 1024
 *   scheme   KIN_LBE_MRT or KIN_DUGKS
 *   nu       kinematic viscosity (> 0).  LBE: s9 = s13 = 1/(3 nu + 1/2)
 *            (Sec. IV.A, Eq. 23).  DUGKS: tau = nu / RT.
 *   Ma       target Mach number u'/c_s used by kin_init_field (> 0)
 *   dt       time step.  LBE: must be 1 (dt = dx).  DUGKS: 0 < dt <= 1/sqrt(2)
 *            (CFL number gamma = sqrt(2) dt <= 1, Sec. IV.A).
 *   storage  enum kin_storage
 *   stream   cudaStream_t to run on, or NULL for a stream the library owns
 *   out      receives the handle; the state starts at rest (f = 0)
 * Errors: KIN_EINVAL, KIN_ENOMEM, KIN_ECUDA. */
int kin_create(int N, int scheme, double nu, double Ma, double dt, int storage, void* stream,
               kin_sim** out);

/* Seeded initial field of Sec. III, Eq. 25 (solenoidal Gaussian field with
 * E(k) = k^4 exp(-2 k^2 / k0^2) on integer shells 1..N/2-1, rescaled so that
 * u' = Ma c_s, Eq. 29), then f = f_eq(0, u0) (Eq. 7).  Random numbers come from
 * the splitmix64 stream described in kin_inputs.  If re_lambda > 0 the
 * viscosity is reset so that the field has Taylor-microscale Reynolds number
 * re_lambda (Eqs. 26, 28, 30: nu = u'^2 sqrt(15 / (2 Omega)) / Re_lambda,
 * Omega = sum |k|^2 E(k)); otherwise nu is kept.  Resets time to 0.
 * Requires even N >= 4.  Synchronous. */
int kin_init_field(kin_sim* sim, uint64_t seed, double k0, double re_lambda);

/* f = f_eq(0, u) everywhere (Eq. 7) from a host velocity field [3][N^3].
 * Resets time to 0.  Synchronous. */
int kin_set_velocity(kin_sim* sim, const double* u);

/* Load / read the state in the canonical host layout (see top of file).
 * Synchronous. kin_set_f resets time to 0. */
int kin_set_f(kin_sim* sim, const double* f);
int kin_get_f(kin_sim* sim, double* f);

/* Canonical f at n cells (linear indices x + N (y + N z)) into out[n][19].
 * Synchronous. */
int kin_sample_f(kin_sim* sim, const int64_t* cells, int64_t n, double* out);

/* Velocity field u[3][N^3] (host) of the current state (Eq. 8 / Eq. 12).
 * Synchronous. */
int kin_get_velocity(kin_sim* sim, double* u);

/* Consistent initial distributions (Sec. IV.A: the paper's LBE and DUGKS
 * runs start from distributions that carry the initial pressure and the
 * non-equilibrium part, obtained by the iteration of Mei et al.).  The
 * velocity u0 of the current state (as set by kin_init_field or
 * kin_set_velocity) is held fixed while steps repeat, so only the density
 * evolves, towards c_s^2 lap(delta-rho) = -d_a d_b (u0_a u0_b):
 *   MRT-LBE: the equilibrium takes the momentum rho0 u0 and the momentum
 *            rows relax fully to it, the other rows with the Sec. IV.A rates;
 *   DUGKS:   a plain step (Eqs. 9-20), after which the momentum of f-tilde
 *            returns to rho0 u0 along the linear term of the equilibrium,
 *            f_i += 3 W_i xi_i . rho0 (u0 - u) (the mass and the second
 *            moment unchanged).
 * Every 10 iterations (and at the last) the change of delta-rho over one
 * iteration, max over the box, is measured; the iteration stops when it is
 * <= tol or after max_iter >= 1 iterations.  *iters (may be NULL) receives the
 * iterations done, *residual (may be NULL) the last measured change.  The
 * state then holds the result as the state at step 0.  Synchronous.
 * KIN_EINVAL for max_iter < 1; KIN_ENONFINITE if it diverges. */
int kin_init_consistent(kin_sim* sim, int max_iter, double tol, int* iters, double* residual);

/* Enqueue n >= 0 time steps on the simulation's stream and return. */
int kin_step(kin_sim* sim, int n);

/* Statistics of the current state (synchronises the stream):
 *   E    = <u.u>/2, the kinetic energy per unit mass (Eq. 26 via Parseval)
 *   eps  = 2 nu <s_ab s_ab>, s_ab from periodic second-order central
 *          differences of u (grid form of Eq. 26)
 *   Ek   NULL, or kin_num_shells(N) doubles: E(s) = sum over modes with
 *          floor(|n| + 1/2) = s of |u_hat|^2 / 2, u_hat = N^-3 FFT(u) (Eq. 27)
 * Any output pointer may be NULL.  Reductions run in a fixed order: the
 * result is bitwise reproducible for a given state.  FP64 storage is reduced
 * in FP64 throughout; for FP32, FP16 and BF16 storage the velocity, E, eps
 * and the transforms of Ek are formed in FP32 and every sum is taken in FP64
 * (relative error ~1e-6 and below).
 * Returns KIN_ENONFINITE if E is not finite. */
int kin_stats(kin_sim* sim, double* E, double* eps, double* Ek);

/* kin_step(sim, n) followed by kin_stats(sim, E, eps, Ek), with the same
 * results bit for bit.  For DUGKS with FP32, FP16 or BF16 storage on the
 * fused step (variant 0) the last step also writes the velocity of the state
 * it produces (Eq. 8, summed in the order the separate velocity pass uses),
 * so the statistics skip that pass over the 19 populations.  Synchronises the
 * stream; errors as kin_step and kin_stats. */
int kin_step_stats(kin_sim* sim, int n, double* E, double* eps, double* Ek);

/* Asynchronous E and eps: enqueue, on the simulation's stream, the E and eps
 * of the state at that point of the stream (the kin_stats arithmetic, bitwise
 * the same values) and a copy of them into out[0] (E) and out[1] (eps), and
 * return without waiting.  out: 2 doubles of host memory that the caller
 * keeps valid until the copy has completed (kin_sync, or an event recorded on
 * the stream after this call); page-locked memory keeps the call asynchronous
 * (a copy into pageable memory waits for the stream).  No check of the values
 * is made: the caller tests them for finiteness once they have arrived, and
 * errors reported by the simulation's kernels surface at the next kin_sync.
 * KIN_EINVAL for out == NULL. */
int kin_stats_async(kin_sim* sim, double* out);

/* kin_step(sim, n) followed by kin_stats_async(sim, out), with the fused
 * velocity of kin_step_stats on the last step. */
int kin_step_stats_async(kin_sim* sim, int n, double* out);

/* Derived statistics of the current state (Sec. III; synchronises the stream):
 *   out[0] E          <u.u>/2
 *   out[1] u'         sqrt(<u.u>/3)
 *   out[2] eps        spectral dissipation 2 nu sum_k |k|^2 E_k (Eq. 26),
 *                     k = 2 pi n / N
 *   out[3] lambda     transverse Taylor microscale sqrt(15 nu / eps) u'
 *   out[4] Re_lambda  u' lambda / nu
 *   out[5] eta        Kolmogorov length (nu^3 / eps)^(1/4)
 *   out[6] S          velocity-derivative skewness
 *   out[7] F          velocity-derivative flatness
 *   D   NULL, or kin_num_shells(N) doubles: the dissipation spectrum
 *       D(s) = 2 nu sum over the modes of shell s of |k|^2 |u_hat|^2 / 2,
 *       so sum_s D(s) = eps
 * S = sum_a <(d_a u_a)^3> / sum_a <(d_a u_a)^2>^(3/2) and
 * F = sum_a <(d_a u_a)^4> / sum_a <(d_a u_a)^2>^2 over a = x, y, z, with
 * spectral derivatives (i k_a u_hat, the Nyquist wavenumber dropped).  The
 * printed formulas of S and F carry an extra factor 3 in the denominator,
 * read as a misprint (it would give a Gaussian field the flatness 1, not 3).
 * Everything in FP64; uses the statistics scratch and overwrites nothing of
 * the state.  Returns KIN_ENONFINITE if E is not finite. */
int kin_derived_stats(kin_sim* sim, double* out, double* D);

/* E and eps (as in kin_stats) of a velocity field u[3][N^3] (FP64, x fastest)
 * that is already in device memory, written to out[0] = E and out[1] = eps
 * (device memory), enqueued on `stream` (NULL = default stream); returns after
 * the launch.  The paper has no counterpart: this entry point exists for
 * callers that cannot let the library allocate device memory, such as
 * real-time loops that must not call cudaMalloc/cudaFree (both can
 * synchronise the device) or applications whose device memory is reserved by
 * their own allocator.  It allocates nothing: its scratch, the partial sums of
 * the reduction, is a fixed 19,456-byte array inside the library that every
 * device loading the library keeps until the process exits.  Every call looks
 * up that array's address in the current device's context
 * (cudaGetSymbolAddress); the first call on a device also loads the library's
 * device code there, so make it before any stream capture.  All calls
 * share the array: calls whose work overlaps on the GPU race and must be
 * ordered by the caller (one stream, or events).  N must be in [2, 1024];
 * larger N returns KIN_EINVAL.  nu >= 0.  u and out are the caller's. */
int kin_energy_dissipation_noalloc(const double* u, int N, double nu, double* out, void* stream);

/* Checks that stand in for a memory checker (no counterpart in the paper).
 * kin_check_guards: each state buffer sits between two 64 KiB guard regions
 * filled with the byte 0xA5 at kin_create; after the stream is synchronised
 * the four regions are read back and compared.  KIN_OK, or KIN_EGUARD naming
 * the buffer, side and first changed byte (a kernel wrote outside the state).
 * Synchronous.
 * kin_debug_status: *is_debug (may be NULL) = 1 when this library was built
 * with KIN_DEBUG, whose stencil kernels check every global offset and the
 * shared-memory slot and row indices before use, skip an access that fails
 * and record the first failure (bits 40..47: check site, bits 0..39: the
 * offending value) instead of trapping.  *word (may be NULL) receives that
 * record, 0 if every check passed (always 0 in the release build); reset != 0
 * clears it.  Returns KIN_EDEBUG if a check failed, else KIN_OK.  Acts on the
 * current device. */
int kin_check_guards(kin_sim* sim);
int kin_debug_status(int* is_debug, unsigned long long* word, int reset);

/* Test hook for kin_check_guards: the host changes one byte of a guard region
 * (buffer 0 or 1, side 0 = before the data, 1 = after) with cudaMemset.
 * Synchronous.  KIN_EINVAL for other buffer or side values. */
int kin_test_corrupt_guard(kin_sim* sim, int buffer, int side);

/* Number of spectrum shells for edge N: 1 + floor(sqrt(3) (N/2) + 1/2). */
int kin_num_shells(int N);

/* Launch-shape tuning (all values <= 0 keep the current setting):
 *   block_x  threads per block along x (multiple of 32, <= 1024) of the
 *            LBE step (used up to 256) and of the two-launch DUGKS form
 *            (up to 128); with FP16/BF16 storage and even N an LBE thread
 *            takes 4 cells, or 2 when N % 4 != 0
 *   tile_y   DUGKS fused kernel: rows per tile, 4 or 8
 *   zchunk   DUGKS fused kernel: planes each thread block marches through
 *            (default: when a plane's tile columns fill fewer than 1.5
 *            waves of blocks, the length with the shortest list schedule of
 *            the grid; otherwise about two waves of blocks)
 *   variant  DUGKS: 0 = fused single launch, f-tilde staged in shared
 *            memory by cp.async copies two planes ahead (default); 1 = two
 *            launches (pre-step into scratch, then flux + update)
 * The fused step's results do not depend on tile_y or zchunk (bitwise); the
 * two-launch form sums the same terms in another order (rounding only).
 * Other variant values return KIN_EINVAL. */
int kin_set_tuning(kin_sim* sim, int block_x, int tile_y, int zchunk, int variant);

/* Number of kernel launches one kin_step(sim, 1) enqueues. */
int kin_step_launches(const kin_sim* sim);

/* Total launches of this library's own kernels for sim since kin_create
 * (cuFFT's kernels are not counted). */
int64_t kin_kernel_launches(const kin_sim* sim);

/* Block until the simulation's stream is idle. */
int kin_sync(kin_sim* sim);

double kin_get_nu(const kin_sim* sim);
double kin_get_dt(const kin_sim* sim);
double kin_get_time(const kin_sim* sim);  /* steps taken * dt */
int64_t kin_get_step(const kin_sim* sim); /* steps taken since the last reset */
int kin_get_N(const kin_sim* sim);
int kin_get_scheme(const kin_sim* sim);
int kin_get_storage(const kin_sim* sim);

/* Human-readable name of a status code; never NULL. */
const char* kin_strerror(int code);

/* Description of the last failure on the calling thread ("" if none). */
const char* kin_last_error(void);

/* Release all device memory of sim; NULL-safe. */
void kin_destroy(kin_sim* sim);

/* ------------------------------------------------------------------------
 * Ensembles: many independent simulations (any mix of N and scheme; KIN_F32,
 * KIN_F16 or KIN_BF16 storage, 2-byte DUGKS members with even N; one device)
 * advanced together by ONE CUDA graph launch per kin_ensemble_step call (per
 * 256 steps when there are LBE members): a persistent, cooperative kernel
 * runs every step of the DUGKS members, and, on a parallel stream of the same
 * graph, one batched launch per step and storage type updates all LBE
 * members, its blocks sharing the SMs with the DUGKS blocks.  Each member's
 * results are bitwise identical to stepping it alone with kin_step (a cell's
 * arithmetic does not depend on the tile shape or the launch).  There is no
 * counterpart of this batching in the paper, which runs one simulation.
 */
typedef struct kin_ensemble kin_ensemble;

/* members: n distinct handles; the ensemble keeps the pointers (the caller
 * keeps ownership and must destroy the ensemble before any member). */
int kin_ensemble_create(kin_sim* const* members, int n, kin_ensemble** out);

/* Work decomposition: tile_y (4, 6 or 8; default 6 when the ensemble holds
 * both schemes, so that LBE blocks fit beside each DUGKS block, else 8) and
 * zchunk of the DUGKS tiles, lbe_block (a multiple of 32, at most 128) threads
 * per block of the batched LBE launches; values <= 0 keep the setting. */
int kin_ensemble_set_tuning(kin_ensemble* ens, int tile_y, int zchunk, int lbe_block);

/* Advance every member by nsteps (synchronous): one graph launch, or one per
 * 256 steps when there are LBE members (a graph holds one LBE launch per
 * step).  Members must be idle; their streams are synchronised first.
 * Returns KIN_ETIMEOUT if a member barrier inside the persistent kernel waited
 * longer than its bound; every member's state is then undefined and the
 * member returns KIN_ESTATE from any call that reads or steps it until its
 * state is set again (kin_set_f, kin_set_velocity, kin_init_field). */
int kin_ensemble_step(kin_ensemble* ens, int nsteps);

/* Run the persistent kernel alone with a member barrier that cannot be
 * satisfied and a wait bound of `seconds`: must return KIN_ETIMEOUT promptly,
 * with every member then refusing work (KIN_ESTATE) until set again.  For
 * testing the bounded wait; KIN_EINVAL without DUGKS members. */
int kin_ensemble_test_timeout(kin_ensemble* ens, double seconds);

/* Work per step (DUGKS tiles + batched LBE thread blocks), thread blocks of
 * the persistent launch (0 without DUGKS members), graph launches so far. */
int kin_ensemble_info(const kin_ensemble* ens, int* nitems, int* grid, int64_t* launches);

void kin_ensemble_destroy(kin_ensemble* ens);

#ifdef __cplusplus
}
#endif
#endif /* KIN_H */
