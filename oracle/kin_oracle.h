/*
 * FP64 CPU oracle for the two kinetic schemes compared in Wang, Wang & Guo,
 * "Comparison of the LBE and DUGKS methods for DNS of decaying homogeneous
 * isotropic turbulence" (arXiv:1601.03815).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link or
 * call this code: only tests/, the smoke check and the benchmark's CPU
 * baseline leg use it.  It shares no code, header or table with the CUDA
 * library; the two meet only through the public data layout described below.
 *
 * Layout of every distribution array: f[i][z][y][x], x fastest, 19 planes of
 * nx*ny*nz doubles, population order given by orc_lattice().  The stored
 * variable is the paper's f_i, i.e. the deviation from W_i*rho0 (Eq. 7 has no
 * rest part), with rho0 = 1, RT = c_s^2 = 1/3, c = 1, dx = 1.
 *
 * Parity status of each function (pins live in tests/test_oracle_*.py):
 *   orc_lattice, orc_feq            pinned (quadrature and moment identities)
 *   orc_mrt_matrix                  pinned (orthogonality, row norms)
 *   orc_mrt_meq                     pinned for rows 0,1,3-9,11,13-18 (equal to
 *                                   M.f_eq); rows 2, 10, 12 (epsilon, 3pi_xx,
 *                                   pi_ww) are free parameters of the model
 *                                   (omega_eps = omega_xx = 0,
 *                                   omega_epsj = -475/63): parity unpinned
 *                                   beyond their use in the conservation and
 *                                   viscous-decay pins
 *   orc_mrt_collide, orc_lbe_step   pinned (BGK special case, conservation,
 *                                   Taylor-Green / shear-wave decay)
 *   orc_dugks_*                     pinned (Eq. 19/20 against Eqs. 11/14,
 *                                   conservation, uniform flow, decay)
 *   orc_macro, orc_energy_dissipation pinned (closed forms on single modes)
 */
#ifndef KIN_ORACLE_H
#define KIN_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

/* D3Q19 velocity set and weights (Sec. II.A, Eq. 5 and the weights after it). */
void orc_lattice(int xi[19 * 3], double w[19]);

/* Discrete equilibrium, Eq. 7, rho0 = 1, RT = 1/3. */
void orc_feq(double drho, double ux, double uy, double uz, double feq[19]);

/* delta-rho = sum f, rho0 u = sum xi f  (Eqs. 8, 12, 17, 22). */
void orc_moments(const double f[19], double* drho, double j[3]);

/* MRT transformation matrix M, row-major [k][alpha], rows as in Sec. II.B. */
void orc_mrt_matrix(double M[19 * 19]);

/* Equilibrium moments m_eq(delta-rho, j), Sec. II.B, with the parameters of
 * Sec. IV.A: omega_eps = omega_xx = 0, omega_epsj = -475/63, rho0 = 1. */
void orc_mrt_meq(double drho, double jx, double jy, double jz, double meq[19]);

/* Relaxation rates S = diag(...) of Sec. II.B with the values of Sec. IV.A:
 * s1 = 1.19, s2 = s10 = 1.4, s4 = 1.2, s9 = s13 = dt/(3 nu + dt/2), s16 = 1.98. */
void orc_mrt_rates(double nu, double s[19]);

/* One MRT collision: fpost = f - M^-1 S (M f - meq)  (RHS of Eq. 21), with a
 * dense FP64 inverse of M.  meq is passed in so special cases can be tested. */
void orc_mrt_collide(const double s[19], const double f[19], const double meq[19],
                     double fpost[19]);

/* One LBE time step, Eq. 21: collide at every node with rates s, then push
 * f*_i(x) to x + xi_i with periodic wrap.  fin and fout must not alias.
 * Returns 0, or -1 on bad sizes. */
int orc_lbe_step(int nx, int ny, int nz, const double s[19], const double* fin, double* fout);

/* DUGKS relaxation time from the viscosity: tau = nu / RT (BGK relation). */
double orc_dugks_tau(double nu);

/* DUGKS cell pre-step, Eqs. 19 and 20, for one cell:
 * fbp = (2tau-h)/(2tau+dt) ft + 3h/(2tau+dt) feq(ft),  ftp = 4/3 fbp - 1/3 ft. */
void orc_dugks_prestep_cell(double tau, double dt, const double ft[19], double fbp[19],
                            double ftp[19]);

/* One DUGKS time step (Eqs. 9-20): pre-step, interface reconstruction with the
 * central (linear-interpolation) gradient, interface equilibrium, interface
 * distribution, flux divergence.  fin and fout must not alias.
 * Returns 0, -1 on bad sizes, -2 on allocation failure. */
int orc_dugks_step(int nx, int ny, int nz, double nu, double dt, const double* fin,
                   double* fout);

/* f = f_eq(drho, u) at every cell (Eq. 7); drho may be NULL (zero).
 * u is [3][n] with n = nx*ny*nz, f is [19][n]. */
void orc_equilibrium_field(int nx, int ny, int nz, const double* drho, const double* u,
                           double* f);

/* Per-cell delta-rho [n] and velocity u[3][n] from f (Eq. 8 / Eq. 12). */
void orc_macro(int nx, int ny, int nz, const double* f, double* drho, double* u);

/* Volume-averaged kinetic energy E = <u.u>/2 and finite-difference dissipation
 * eps = 2 nu <s_ab s_ab>, s_ab from second-order central differences of u on
 * the periodic grid (the discrete form of Eq. 26 used for per-step logging). */
void orc_energy_dissipation(int nx, int ny, int nz, double nu, const double* u, double* E,
                            double* eps);

/* Number of OpenMP threads the oracle runs with (1 without OpenMP). */
int orc_num_threads(void);
void orc_set_num_threads(int n);

#ifdef __cplusplus
}
#endif
#endif
