/*
 * FP64 CPU oracle for the LBE (MRT, D3Q19) and DUGKS schemes of Wang, Wang &
 * Guo, arXiv:1601.03815.  TEST INFRASTRUCTURE ONLY (see kin_oracle.h): plain,
 * slow and literal, so it can be checked against the paper by eye.  Equation
 * numbers follow the paper's numbered equations in order of appearance.
 */
#include "kin_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define Q 19

/* Sec. II.A, Eq. 5: the rest velocity (printed "(0,0)"), the six axis
 * velocities (i = 1..6) and the twelve face-diagonal velocities (i = 7..18),
 * in units of c = sqrt(3RT) = 1.  Opposite velocities are adjacent (i, i+1)
 * for odd i. */
static const int XI[Q][3] = {
    {0, 0, 0},
    {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},  {0, -1, 0}, {0, 0, 1},  {0, 0, -1},
    {1, 1, 0},  {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0},
    {1, 0, 1},  {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
    {0, 1, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};

/* Weights W_0 = 1/3, W_1..6 = 1/18, W_7..18 = 1/36 (Sec. II.A). */
static double weight(int i) {
    if (i == 0) return 1.0 / 3.0;
    if (i <= 6) return 1.0 / 18.0;
    return 1.0 / 36.0;
}

static const double RHO0 = 1.0;
static const double RT = 1.0 / 3.0;

void orc_lattice(int xi[Q * 3], double w[Q]) {
    for (int i = 0; i < Q; ++i) {
        for (int a = 0; a < 3; ++a) xi[3 * i + a] = XI[i][a];
        w[i] = weight(i);
    }
}

/* Eq. 7: f_eq_i = W_i [drho + rho0 (xi.u/RT + (xi.u)^2/(2 RT^2) - |u|^2/(2RT))]. */
void orc_feq(double drho, double ux, double uy, double uz, double feq[Q]) {
    double uu = ux * ux + uy * uy + uz * uz;
    for (int i = 0; i < Q; ++i) {
        double xu = XI[i][0] * ux + XI[i][1] * uy + XI[i][2] * uz;
        feq[i] = weight(i) *
                 (drho + RHO0 * (xu / RT + xu * xu / (2.0 * RT * RT) - uu / (2.0 * RT)));
    }
}

/* Eq. 8: delta-rho = sum_i f_i, rho0 u = sum_i xi_i f_i. */
void orc_moments(const double f[Q], double* drho, double j[3]) {
    double r = 0.0, jx = 0.0, jy = 0.0, jz = 0.0;
    for (int i = 0; i < Q; ++i) {
        r += f[i];
        jx += XI[i][0] * f[i];
        jy += XI[i][1] * f[i];
        jz += XI[i][2] * f[i];
    }
    *drho = r;
    j[0] = jx;
    j[1] = jy;
    j[2] = jz;
}

/* Sec. II.B: the rows M_k,alpha as polynomials of xi_alpha (||xi||^0 = 1 for
 * the rest velocity). */
void orc_mrt_matrix(double M[Q * Q]) {
    for (int a = 0; a < Q; ++a) {
        double x = XI[a][0], y = XI[a][1], z = XI[a][2];
        double r2 = x * x + y * y + z * z;
        double r4 = r2 * r2;
        M[0 * Q + a] = 1.0;
        M[1 * Q + a] = 19.0 * r2 - 30.0;
        M[2 * Q + a] = (21.0 * r4 - 53.0 * r2 + 24.0) / 2.0;
        M[3 * Q + a] = x;
        M[4 * Q + a] = (5.0 * r2 - 9.0) * x;
        M[5 * Q + a] = y;
        M[6 * Q + a] = (5.0 * r2 - 9.0) * y;
        M[7 * Q + a] = z;
        M[8 * Q + a] = (5.0 * r2 - 9.0) * z;
        M[9 * Q + a] = 3.0 * x * x - r2;
        M[10 * Q + a] = (3.0 * r2 - 5.0) * (3.0 * x * x - r2);
        M[11 * Q + a] = y * y - z * z;
        M[12 * Q + a] = (3.0 * r2 - 5.0) * (y * y - z * z);
        M[13 * Q + a] = x * y;
        M[14 * Q + a] = y * z;
        M[15 * Q + a] = x * z;
        M[16 * Q + a] = (y * y - z * z) * x;
        M[17 * Q + a] = (z * z - x * x) * y;
        M[18 * Q + a] = (x * x - y * y) * z;
    }
}

/* Sec. II.B equilibrium moments with the model's free parameters: eps_eq =
 * omega_eps drho + omega_epsj j^2 / rho0, pi_eq = omega_xx p_eq.  The moment
 * vector holds 3p_xx and 3pi_xx in slots 9 and 10, so slot 9 is 3 * p_xx_eq
 * and slot 10 is omega_xx * 3 * p_xx_eq. */
void orc_mrt_meq_w(double drho, double jx, double jy, double jz, double omega_eps, double omega_epsj,
                   double omega_xx, double meq[Q]) {
    double jj = jx * jx + jy * jy + jz * jz;
    double pxx = (2.0 * jx * jx - (jy * jy + jz * jz)) / (3.0 * RHO0);
    double pww = (jy * jy - jz * jz) / RHO0;
    meq[0] = drho;
    meq[1] = -11.0 * drho + 19.0 / RHO0 * jj;
    meq[2] = omega_eps * drho + omega_epsj / RHO0 * jj;
    meq[3] = jx;
    meq[4] = -2.0 / 3.0 * jx;
    meq[5] = jy;
    meq[6] = -2.0 / 3.0 * jy;
    meq[7] = jz;
    meq[8] = -2.0 / 3.0 * jz;
    meq[9] = 3.0 * pxx;
    meq[10] = 3.0 * omega_xx * pxx;
    meq[11] = pww;
    meq[12] = omega_xx * pww;
    meq[13] = jx * jy / RHO0;
    meq[14] = jy * jz / RHO0;
    meq[15] = jx * jz / RHO0;
    meq[16] = 0.0;
    meq[17] = 0.0;
    meq[18] = 0.0;
}

/* The paper's values (Sec. IV.A): omega_eps = omega_xx = 0, omega_epsj = -475/63. */
void orc_mrt_meq(double drho, double jx, double jy, double jz, double meq[Q]) {
    orc_mrt_meq_w(drho, jx, jy, jz, 0.0, -475.0 / 63.0, 0.0, meq);
}

/* S = diag(0, s1, s2, 0, s4, 0, s4, 0, s4, s9, s10, s9, s10, s13, s13, s13,
 * s16, s16, s16) (Sec. II.B) with the Sec. IV.A values, dt = dx = 1. */
void orc_mrt_rates(double nu, double s[Q]) {
    const double dt = 1.0;
    double s1 = 1.19, s2 = 1.4, s4 = 1.2, s10 = 1.4, s16 = 1.98;
    double s9 = dt / (3.0 * nu + 0.5 * dt);
    double s13 = s9;
    double S[Q] = {0.0, s1,  s2,  0.0, s4,  0.0, s4,  0.0, s4, s9,
                   s10, s9,  s10, s13, s13, s13, s16, s16, s16};
    memcpy(s, S, sizeof(S));
}

/* Dense Gauss-Jordan inverse with partial pivoting. */
static void invert(const double* A, double* Ainv, int n) {
    double* a = (double*)malloc(sizeof(double) * n * 2 * n);
    for (int r = 0; r < n; ++r)
        for (int c = 0; c < 2 * n; ++c)
            a[r * 2 * n + c] = c < n ? A[r * n + c] : (c - n == r ? 1.0 : 0.0);
    for (int col = 0; col < n; ++col) {
        int piv = col;
        for (int r = col + 1; r < n; ++r)
            if (fabs(a[r * 2 * n + col]) > fabs(a[piv * 2 * n + col])) piv = r;
        if (piv != col)
            for (int c = 0; c < 2 * n; ++c) {
                double t = a[col * 2 * n + c];
                a[col * 2 * n + c] = a[piv * 2 * n + c];
                a[piv * 2 * n + c] = t;
            }
        double p = a[col * 2 * n + col];
        for (int c = 0; c < 2 * n; ++c) a[col * 2 * n + c] /= p;
        for (int r = 0; r < n; ++r) {
            if (r == col) continue;
            double fct = a[r * 2 * n + col];
            if (fct == 0.0) continue;
            for (int c = 0; c < 2 * n; ++c) a[r * 2 * n + c] -= fct * a[col * 2 * n + c];
        }
    }
    for (int r = 0; r < n; ++r)
        for (int c = 0; c < n; ++c) Ainv[r * n + c] = a[r * 2 * n + n + c];
    free(a);
}

static void collide_with(const double* M, const double* Minv, const double s[Q],
                         const double f[Q], const double meq[Q], double fpost[Q]) {
    double dm[Q];
    for (int k = 0; k < Q; ++k) {
        double m = 0.0;
        for (int a = 0; a < Q; ++a) m += M[k * Q + a] * f[a];
        dm[k] = s[k] * (m - meq[k]);
    }
    for (int a = 0; a < Q; ++a) {
        double df = 0.0;
        for (int k = 0; k < Q; ++k) df += Minv[a * Q + k] * dm[k];
        fpost[a] = f[a] - df;
    }
}

void orc_mrt_collide(const double s[Q], const double f[Q], const double meq[Q],
                     double fpost[Q]) {
    double M[Q * Q], Minv[Q * Q];
    orc_mrt_matrix(M);
    invert(M, Minv, Q);
    collide_with(M, Minv, s, f, meq, fpost);
}

static inline int wrap(int a, int n) {
    a %= n;
    return a < 0 ? a + n : a;
}

/* Eq. 21: f(x + xi_i dt, t + dt) = f(x, t) - M^-1 S [m(x,t) - m_eq(x,t)]. */
int orc_lbe_step(int nx, int ny, int nz, const double s[Q], const double* fin, double* fout) {
    if (nx <= 0 || ny <= 0 || nz <= 0) return -1;
    const long n = (long)nx * ny * nz;
    double M[Q * Q], Minv[Q * Q];
    orc_mrt_matrix(M);
    invert(M, Minv, Q);
#pragma omp parallel for schedule(static)
    for (long c = 0; c < n; ++c) {
        int x = (int)(c % nx), y = (int)((c / nx) % ny), z = (int)(c / ((long)nx * ny));
        double f[Q], fpost[Q], meq[Q], drho, j[3];
        for (int i = 0; i < Q; ++i) f[i] = fin[i * n + c];
        orc_moments(f, &drho, j);
        orc_mrt_meq(drho, j[0], j[1], j[2], meq);
        collide_with(M, Minv, s, f, meq, fpost);
        for (int i = 0; i < Q; ++i) {
            long d = wrap(x + XI[i][0], nx) + (long)nx * (wrap(y + XI[i][1], ny) +
                                                          (long)ny * wrap(z + XI[i][2], nz));
            fout[i * n + d] = fpost[i];
        }
    }
    return 0;
}

/* One iteration of the consistent initialisation the paper cites for its
 * initial distributions (Sec. IV.A; Mei et al. 2006): the LBE step of Eq. 21
 * with the velocity held at the prescribed u0 ([3][n], rho0 = 1).  The
 * equilibrium moments take the momentum rho0 u0, and the momentum rows, whose
 * rate is immaterial in the plain step (they are conserved), relax fully to
 * it (rate 1); every other row keeps its rate s.  Only the density evolves,
 * by streaming, until it stops changing. */
int orc_lbe_consistent_step(int nx, int ny, int nz, const double s[Q], const double* u0, const double* fin,
                            double* fout) {
    if (nx <= 0 || ny <= 0 || nz <= 0) return -1;
    const long n = (long)nx * ny * nz;
    double M[Q * Q], Minv[Q * Q], sc[Q];
    orc_mrt_matrix(M);
    invert(M, Minv, Q);
    for (int k = 0; k < Q; ++k) sc[k] = s[k];
    sc[3] = sc[5] = sc[7] = 1.0; /* momentum rows: j_x, j_y, j_z */
#pragma omp parallel for schedule(static)
    for (long c = 0; c < n; ++c) {
        int x = (int)(c % nx), y = (int)((c / nx) % ny), z = (int)(c / ((long)nx * ny));
        double f[Q], fpost[Q], meq[Q], drho, j[3];
        for (int i = 0; i < Q; ++i) f[i] = fin[i * n + c];
        orc_moments(f, &drho, j);
        orc_mrt_meq(drho, RHO0 * u0[c], RHO0 * u0[n + c], RHO0 * u0[2 * n + c], meq);
        collide_with(M, Minv, sc, f, meq, fpost);
        for (int i = 0; i < Q; ++i) {
            long d = wrap(x + XI[i][0], nx) + (long)nx * (wrap(y + XI[i][1], ny) +
                                                          (long)ny * wrap(z + XI[i][2], nz));
            fout[i * n + d] = fpost[i];
        }
    }
    return 0;
}

/* The paper does not state tau(nu) for DUGKS; the BGK model of Eq. 6 gives
 * nu = tau RT, so tau = nu / RT = 3 nu. */
double orc_dugks_tau(double nu) { return nu / RT; }

/* Eqs. 19 and 20 with h = dt/2 and f_eq from the cell's own moments. */
void orc_dugks_prestep_cell(double tau, double dt, const double ft[Q], double fbp[Q],
                            double ftp[Q]) {
    double h = 0.5 * dt, drho, j[3], feq[Q];
    orc_moments(ft, &drho, j);
    orc_feq(drho, j[0] / RHO0, j[1] / RHO0, j[2] / RHO0, feq);
    for (int i = 0; i < Q; ++i) {
        fbp[i] = (2.0 * tau - h) / (2.0 * tau + dt) * ft[i] + 3.0 * h / (2.0 * tau + dt) * feq[i];
        ftp[i] = 4.0 / 3.0 * fbp[i] - 1.0 / 3.0 * ft[i];
    }
}

int orc_dugks_step(int nx, int ny, int nz, double nu, double dt, const double* fin,
                   double* fout) {
    if (nx <= 0 || ny <= 0 || nz <= 0) return -1;
    const long n = (long)nx * ny * nz;
    const int dims[3] = {nx, ny, nz};
    const double tau = orc_dugks_tau(nu), h = 0.5 * dt;
    double* fbp = (double*)malloc(sizeof(double) * Q * n);
    double* ftp = (double*)malloc(sizeof(double) * Q * n);
    double* flux = (double*)malloc(sizeof(double) * 3 * Q * n); /* [a][i][cell] */
    if (!fbp || !ftp || !flux) {
        free(fbp);
        free(ftp);
        free(flux);
        return -2;
    }

    /* 1. Cell pre-step: f-bar-plus and f-tilde-plus from f-tilde (Eqs. 19, 20). */
#pragma omp parallel for schedule(static)
    for (long c = 0; c < n; ++c) {
        double ft[Q], b[Q], p[Q];
        for (int i = 0; i < Q; ++i) ft[i] = fin[i * n + c];
        orc_dugks_prestep_cell(tau, dt, ft, b, p);
        for (int i = 0; i < Q; ++i) {
            fbp[i * n + c] = b[i];
            ftp[i * n + c] = p[i];
        }
    }

    /* 2. Interface distribution and flux at x_b = x_c + e_a/2 for a = x, y, z.
     * Eqs. 15/16: the interface value and its normal gradient come from linear
     * interpolation between the two cell centres; the tangential gradient
     * components are the mean of the two cells' central differences.  Eq. 13:
     * f-bar(x_b, t+h) = f-bar-plus(x_b) - h xi.sigma_b.  Eq. 17: interface
     * moments; Eq. 7: interface equilibrium; Eq. 18: interface f; Eq. 10: the
     * flux (xi.n) f through a unit face. */
#pragma omp parallel for schedule(static)
    for (long c = 0; c < n; ++c) {
        int pos[3] = {(int)(c % nx), (int)((c / nx) % ny), (int)(c / ((long)nx * ny))};
        for (int a = 0; a < 3; ++a) {
            double fbar[Q], feqb[Q], drho, j[3];
            for (int i = 0; i < Q; ++i) {
                /* cell value at L = c (+ offset) and R = c + e_a (+ offset) */
#define CELL(dxv, dyv, dzv)                                                              \
    (wrap(pos[0] + (dxv), nx) + (long)nx * (wrap(pos[1] + (dyv), ny) +                     \
                                            (long)ny * wrap(pos[2] + (dzv), nz)))
                int ea[3] = {a == 0, a == 1, a == 2};
                double L = fbp[i * n + c];
                double R = fbp[i * n + CELL(ea[0], ea[1], ea[2])];
                double sigma[3];
                sigma[a] = R - L;
                for (int t = 0; t < 3; ++t) {
                    if (t == a) continue;
                    int et[3] = {t == 0, t == 1, t == 2};
                    double Lp = fbp[i * n + CELL(et[0], et[1], et[2])];
                    double Lm = fbp[i * n + CELL(-et[0], -et[1], -et[2])];
                    double Rp = fbp[i * n + CELL(ea[0] + et[0], ea[1] + et[1], ea[2] + et[2])];
                    double Rm = fbp[i * n + CELL(ea[0] - et[0], ea[1] - et[1], ea[2] - et[2])];
                    sigma[t] = 0.5 * ((Lp - Lm) / 2.0 + (Rp - Rm) / 2.0);
                }
#undef CELL
                double fb_plus = 0.5 * (L + R);
                double xs = XI[i][0] * sigma[0] + XI[i][1] * sigma[1] + XI[i][2] * sigma[2];
                fbar[i] = fb_plus - h * xs;
            }
            orc_moments(fbar, &drho, j);
            orc_feq(drho, j[0] / RHO0, j[1] / RHO0, j[2] / RHO0, feqb);
            for (int i = 0; i < Q; ++i) {
                double fface = 2.0 * tau / (2.0 * tau + h) * fbar[i] + h / (2.0 * tau + h) * feqb[i];
                flux[((long)a * Q + i) * n + c] = XI[i][a] * fface;
            }
        }
    }

    /* 3. Eq. 9 with |V_j| = 1 and unit faces: the outward normal is +e_a on
     * the face at x_c + e_a/2 and -e_a on the face at x_c - e_a/2. */
#pragma omp parallel for schedule(static)
    for (long c = 0; c < n; ++c) {
        int pos[3] = {(int)(c % nx), (int)((c / nx) % ny), (int)(c / ((long)nx * ny))};
        long lower[3];
        lower[0] = wrap(pos[0] - 1, nx) + (long)nx * (pos[1] + (long)ny * pos[2]);
        lower[1] = pos[0] + (long)nx * (wrap(pos[1] - 1, ny) + (long)ny * pos[2]);
        lower[2] = pos[0] + (long)nx * (pos[1] + (long)ny * wrap(pos[2] - 1, nz));
        for (int i = 0; i < Q; ++i) {
            double F = 0.0;
            for (int a = 0; a < 3; ++a)
                F += flux[((long)a * Q + i) * n + c] - flux[((long)a * Q + i) * n + lower[a]];
            fout[i * n + c] = ftp[i * n + c] - dt * F;
        }
    }
    (void)dims;
    free(fbp);
    free(ftp);
    free(flux);
    return 0;
}

void orc_equilibrium_field(int nx, int ny, int nz, const double* drho, const double* u,
                           double* f) {
    const long n = (long)nx * ny * nz;
#pragma omp parallel for schedule(static)
    for (long c = 0; c < n; ++c) {
        double feq[Q];
        orc_feq(drho ? drho[c] : 0.0, u[c], u[n + c], u[2 * n + c], feq);
        for (int i = 0; i < Q; ++i) f[i * n + c] = feq[i];
    }
}

void orc_macro(int nx, int ny, int nz, const double* f, double* drho, double* u) {
    const long n = (long)nx * ny * nz;
#pragma omp parallel for schedule(static)
    for (long c = 0; c < n; ++c) {
        double fl[Q], r, j[3];
        for (int i = 0; i < Q; ++i) fl[i] = f[i * n + c];
        orc_moments(fl, &r, j);
        if (drho) drho[c] = r;
        for (int a = 0; a < 3; ++a) u[a * n + c] = j[a] / RHO0;
    }
}

/* E = <u.u>/2 (Eq. 26 via Parseval); eps = 2 nu <s_ab s_ab> with
 * s_ab = (d_a u_b + d_b u_a)/2 and d_a the periodic central difference. */
void orc_energy_dissipation(int nx, int ny, int nz, double nu, const double* u, double* E,
                            double* eps) {
    const long n = (long)nx * ny * nz;
    double se = 0.0, ss = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : se, ss)
    for (long c = 0; c < n; ++c) {
        int x = (int)(c % nx), y = (int)((c / nx) % ny), z = (int)(c / ((long)nx * ny));
        long nb[3][2] = {
            {wrap(x + 1, nx) + (long)nx * (y + (long)ny * z), wrap(x - 1, nx) + (long)nx * (y + (long)ny * z)},
            {x + (long)nx * (wrap(y + 1, ny) + (long)ny * z), x + (long)nx * (wrap(y - 1, ny) + (long)ny * z)},
            {x + (long)nx * (y + (long)ny * wrap(z + 1, nz)), x + (long)nx * (y + (long)ny * wrap(z - 1, nz))}};
        double g[3][3]; /* g[a][b] = d_a u_b */
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) g[a][b] = (u[b * n + nb[a][0]] - u[b * n + nb[a][1]]) / 2.0;
        double s2 = 0.0;
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                double sab = 0.5 * (g[a][b] + g[b][a]);
                s2 += sab * sab;
            }
        ss += s2;
        se += u[c] * u[c] + u[n + c] * u[n + c] + u[2 * n + c] * u[2 * n + c];
    }
    *E = 0.5 * se / (double)n;
    *eps = 2.0 * nu * ss / (double)n;
}

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_num_threads(int nthreads) {
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}
