/*
 * sgpe_oracle.c -- plain, slow FP64 CPU oracle of the split-step Crank-Nicolson
 * time step for the spin-1 spin-orbit (SO) and Rabi coupled Gross-Pitaevskii
 * equation of arXiv:2009.13507 ("Spin-1 spin-orbit- and Rabi-coupled
 * Bose-Einstein condensate solver").
 *
 * TEST INFRASTRUCTURE. Only the tests, the smoke check and the CPU-baseline
 * leg of the benchmark load this file's library. The CUDA product path shares
 * no code, header, table or constant with it and never calls it.
 *
 * Everything is double precision with C99 `double complex`; every substep is
 * written out in the paper's notation, one grid point (or one line) at a time,
 * with no fusion, blocking or reordering.
 *
 * State layout: psi[(j*ny + iy)*nx + ix], j = 0, 1, 2 for the spin components
 * +1, 0, -1 (the paper's CP(L, I, J), L = 1, 2, 3, Sec. 3). ny = 1 in 1D.
 * Grid: x_i = (i - nx/2) dx, y_k = (k - ny/2) dy (the paper's NX2 = N/2 origin,
 * Sec. 3); homogeneous Dirichlet ghosts (psi = 0) outside the grid.
 *
 * Time: z = dt in imaginary time, z = i dt in real time; every substep applies
 * (an approximation of) exp(-z H_k), which is the real-time update of Sec. 2
 * and Appendix A with dt -> -i dt in imaginary time.
 *
 * Threads: the loops over independent grid points and independent lines may
 * run on several OpenMP threads (orc_set_threads; one thread by default). Each
 * point or line is computed by the same code whichever thread runs it, and
 * every sum over the grid (norms, observables) stays one sequential loop, so
 * the results are bitwise the same for any thread count.
 *
 * Parity: the substeps are pinned by the CPU tests (dense solves, scipy expm,
 * finite-difference derivatives against Eqs. (1)-(2), Hermiticity and norm
 * identities, closed-form ground-state energies, the paper's Table 4 energies).
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static int g_threads = 1;

/* Number of threads for the point and line loops (n <= 0: all available). */
void orc_set_threads(int n) {
#ifdef _OPENMP
    g_threads = n > 0 ? n : omp_get_num_procs();
#else
    (void)n;
    g_threads = 1;
#endif
}
int orc_get_threads(void) { return g_threads; }

typedef double complex cplx;

typedef struct {
    int dim, nx, ny;     /* ny = 1 in 1D */
    double dx, dy;
    double c0, c2;       /* density-density and spin-exchange nonlinearities, Eqs. (1)-(2) */
    int so_type;         /* 1D: 0 none, 1 gamma p_x Sigma_x, 2 gamma p_x Sigma_y, 3 gamma p_x Sigma_z;
                            2D: 0 none, 1 Rashba (eta=1), 2 Dresselhaus (eta=-1), 3 equal mix (eta=0)
                            (OPT_SO, Sec. 3) */
    double gamma, omega; /* SO strength gamma, Rabi strength Omega */
    double wx, wy;       /* trap V = (wx^2 x^2 + wy^2 y^2)/2; the paper uses wx = wy = 1 (Sec. 2) */
    double dt;           /* time step Delta */
    int renorm;          /* 0 none, 1 Eq. (DJ2), 2 Eq. (DJ) with magnetisation mag */
    double mag;
    int split;           /* 0: Lie splitting, one full dt per substep (the paper's successive
                            treatment); 1: Strang splitting (half steps around the kinetic step) */
    int so_mode;         /* 0: SO by explicit Euler, Eqs. (p1)-(p2); 1: SO by Crank-Nicolson */
} orc_params;

#define IDX(p, j, iy, ix) ((((size_t)(j)) * (p)->ny + (size_t)(iy)) * (p)->nx + (size_t)(ix))

static double xcoord(const orc_params* p, int ix) { return (ix - p->nx / 2) * p->dx; }
static double ycoord(const orc_params* p, int iy) { return p->dim == 2 ? (iy - p->ny / 2) * p->dy : 0.0; }

/* Trap V(r) = (wx^2 x^2 + wy^2 y^2)/2 (Sec. 2, with kappa = wy/wx). */
static double trap(const orc_params* p, int ix, int iy) {
    double x = xcoord(p, ix), y = ycoord(p, iy);
    return 0.5 * (p->wx * p->wx * x * x + p->wy * p->wy * y * y);
}

/* Central first difference of component j along x (or y), zero ghosts. */
static cplx dfx(const orc_params* p, const cplx* f, int j, int iy, int ix) {
    cplx fp = (ix + 1 < p->nx) ? f[IDX(p, j, iy, ix + 1)] : 0.0;
    cplx fm = (ix - 1 >= 0) ? f[IDX(p, j, iy, ix - 1)] : 0.0;
    return (fp - fm) / (2.0 * p->dx);
}
static cplx dfy(const orc_params* p, const cplx* f, int j, int iy, int ix) {
    if (p->dim != 2) return 0.0;
    cplx fp = (iy + 1 < p->ny) ? f[IDX(p, j, iy + 1, ix)] : 0.0;
    cplx fm = (iy - 1 >= 0) ? f[IDX(p, j, iy - 1, ix)] : 0.0;
    return (fp - fm) / (2.0 * p->dy);
}

/*
 * H_SO psi at one point: the SO terms gamma f_{+1}, gamma g, gamma f_{-1} of
 * Eqs. (1)-(2) as given in Sec. 2.
 *  1D Sigma_x: f_{+-} = -i gt d_x psi_0, g = -i gt (d_x psi_+ + d_x psi_-), gt = gamma/sqrt2.
 *  1D Sigma_y: the operator gamma p_x Sigma_y with Sigma_y of Eq. (smat):
 *              f_+ = -gt d_x psi_0, f_- = +gt d_x psi_0, g = gt (d_x psi_+ - d_x psi_-).
 *              (The printed 1D Sigma_y terms carry an extra factor i that makes
 *              them non-Hermitian; this is the form derived from the operator,
 *              which also equals the 2D formula at eta = 0 up to the sign of gamma.)
 *  1D Sigma_z: f_{+-} = -+ i gamma d_x psi_{+-}, g = 0.
 *  2D gamma(eta p_y Sigma_x - p_x Sigma_y):
 *              f_{+-} = -i gt (eta d_y psi_0 +- i d_x psi_0),
 *              g = -i gt (-i d_x psi_+ + i d_x psi_- + eta d_y psi_+ + eta d_y psi_-).
 */
static void hso_point(const orc_params* p, const cplx* f, int iy, int ix, cplx h[3]) {
    h[0] = h[1] = h[2] = 0.0;
    if (p->so_type == 0 || p->gamma == 0.0) return;
    const double gt = p->gamma / sqrt(2.0);
    if (p->dim == 1) {
        cplx dp = dfx(p, f, 0, iy, ix), d0 = dfx(p, f, 1, iy, ix), dm = dfx(p, f, 2, iy, ix);
        if (p->so_type == 1) {
            h[0] = -I * gt * d0;
            h[1] = -I * gt * (dp + dm);
            h[2] = -I * gt * d0;
        } else if (p->so_type == 2) {
            h[0] = -gt * d0;
            h[1] = gt * (dp - dm);
            h[2] = gt * d0;
        } else if (p->so_type == 3) {
            h[0] = -I * p->gamma * dp;
            h[1] = 0.0;
            h[2] = I * p->gamma * dm;
        }
    } else {
        double eta = p->so_type == 1 ? 1.0 : (p->so_type == 2 ? -1.0 : 0.0);
        cplx dxp = dfx(p, f, 0, iy, ix), dx0 = dfx(p, f, 1, iy, ix), dxm = dfx(p, f, 2, iy, ix);
        cplx dyp = dfy(p, f, 0, iy, ix), dy0 = dfy(p, f, 1, iy, ix), dym = dfy(p, f, 2, iy, ix);
        h[0] = -I * gt * (eta * dy0 + I * dx0);
        h[2] = -I * gt * (eta * dy0 - I * dx0);
        h[1] = -I * gt * (-I * dxp + I * dxm + eta * dyp + eta * dym);
    }
}

/*
 * SO substep, Appendix A Eqs. (p1)-(p2): explicit Euler with the SO terms
 * evaluated on the state at time t (all points from the same input):
 * psi_j <- psi_j - z (H_SO psi)_j.  In real time z = i dt this is the paper's
 * psi_{+-} <- psi_{+-} - dt gt d_x psi_0 for Sigma_x.
 */
void orc_so(const orc_params* p, cplx* psi, cplx z) {
    size_t n = (size_t)3 * p->nx * p->ny;
    cplx* old = malloc(n * sizeof(cplx));
    memcpy(old, psi, n * sizeof(cplx));
#pragma omp parallel for num_threads(g_threads) schedule(static)
    for (int iy = 0; iy < p->ny; iy++)
        for (int ix = 0; ix < p->nx; ix++) {
            cplx h[3];
            hso_point(p, old, iy, ix, h);
            for (int j = 0; j < 3; j++) psi[IDX(p, j, iy, ix)] = old[IDX(p, j, iy, ix)] - z * h[j];
        }
    free(old);
}

/* 3x3 complex matrices (row major) for the block elimination below. */
static void m3_mul(const cplx* a, const cplx* b, cplx* c) {
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            cplx t = 0.0;
            for (int k = 0; k < 3; k++) t += a[3 * i + k] * b[3 * k + j];
            c[3 * i + j] = t;
        }
}
static void m3_vec(const cplx* a, const cplx* x, cplx* y) {
    for (int i = 0; i < 3; i++) y[i] = a[3 * i] * x[0] + a[3 * i + 1] * x[1] + a[3 * i + 2] * x[2];
}
/* inverse by the adjugate (the matrices here are I + small terms) */
static void m3_inv(const cplx* a, cplx* r) {
    cplx c00 = a[4] * a[8] - a[5] * a[7], c01 = a[5] * a[6] - a[3] * a[8], c02 = a[3] * a[7] - a[4] * a[6];
    cplx c10 = a[2] * a[7] - a[1] * a[8], c11 = a[0] * a[8] - a[2] * a[6], c12 = a[1] * a[6] - a[0] * a[7];
    cplx c20 = a[1] * a[5] - a[2] * a[4], c21 = a[2] * a[3] - a[0] * a[5], c22 = a[0] * a[4] - a[1] * a[3];
    cplx det = a[0] * c00 + a[1] * c01 + a[2] * c02;
    r[0] = c00 / det; r[1] = c10 / det; r[2] = c20 / det;
    r[3] = c01 / det; r[4] = c11 / det; r[5] = c21 / det;
    r[6] = c02 / det; r[7] = c12 / det; r[8] = c22 / det;
}

/*
 * Crank-Nicolson for the SO operator of one line: H = g S p with p = -i d/ds
 * (the central difference of the SO substep, zero ghosts), S a 3x3 spin
 * matrix of Eq. (smat) and g a real strength:
 *   (I + z/2 H) psi' = (I - z/2 H) psi,
 * a block-tridiagonal system in the three components: with B = -i z g S / (4 h),
 *   row i:  -B psi'_{i-1} + psi'_i + B psi'_{i+1} = psi_i - B (psi_{i+1} - psi_{i-1}),
 * solved by block Gaussian elimination (3x3 blocks, no pivoting).
 * f: the line's components at f[j*cstride + i*stride], n points.
 */
static void so_cn_line(cplx* f, size_t cstride, size_t stride, int n, const cplx S[9], double g, double h, cplx z) {
    cplx B[9];
    for (int k = 0; k < 9; k++) B[k] = -I * z * g * S[k] / (4.0 * h);
    cplx* r = malloc((size_t)n * 3 * sizeof(cplx));
    cplx* Ch = malloc((size_t)n * 9 * sizeof(cplx));
    for (int i = 0; i < n; i++) {
        cplx d[3];
        for (int j = 0; j < 3; j++) {
            cplx up = i + 1 < n ? f[j * cstride + (i + 1) * stride] : 0.0;
            cplx dn = i > 0 ? f[j * cstride + (i - 1) * stride] : 0.0;
            d[j] = up - dn;
        }
        cplx Bd[3];
        m3_vec(B, d, Bd);
        for (int j = 0; j < 3; j++) r[3 * i + j] = f[j * cstride + i * stride] - Bd[j];
    }
    /* forward elimination: M_i = I + B Ch_{i-1}, Ch_i = M_i^{-1} B, r_i <- M_i^{-1} (r_i + B r_{i-1}) */
    for (int i = 0; i < n; i++) {
        cplx M[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1}, Mi[9], t[3];
        if (i > 0) {
            cplx BC[9];
            m3_mul(B, &Ch[9 * (i - 1)], BC);
            for (int k = 0; k < 9; k++) M[k] += BC[k];
            m3_vec(B, &r[3 * (i - 1)], t);
            for (int j = 0; j < 3; j++) r[3 * i + j] += t[j];
        }
        m3_inv(M, Mi);
        m3_mul(Mi, B, &Ch[9 * i]);
        m3_vec(Mi, &r[3 * i], t);
        for (int j = 0; j < 3; j++) r[3 * i + j] = t[j];
    }
    /* back substitution: x_i = r_i - Ch_i x_{i+1} */
    for (int i = n - 2; i >= 0; i--) {
        cplx t[3];
        m3_vec(&Ch[9 * i], &r[3 * (i + 1)], t);
        for (int j = 0; j < 3; j++) r[3 * i + j] -= t[j];
    }
    for (int i = 0; i < n; i++)
        for (int j = 0; j < 3; j++) f[j * cstride + i * stride] = r[3 * i + j];
    free(r);
    free(Ch);
}

/*
 * SO substep by Crank-Nicolson instead of explicit Euler: the SO operator of
 * Sec. 2 treated like the kinetic term. 1D: H_SO = gamma S p_x with S = Sigma_x,
 * Sigma_y or Sigma_z (OPT_SO 1..3), one block line per grid. 2D: H_SO =
 * gamma (eta p_y Sigma_x - p_x Sigma_y) = H_x + H_y, H_x = -gamma Sigma_y p_x
 * along x lines and H_y = gamma eta Sigma_x p_y along y lines, each by
 * Crank-Nicolson in turn (x then y; y then x when reverse), as the kinetic term
 * is treated along x and then y. Each factor is a Cayley transform of a
 * Hermitian operator, so in real time the substep conserves the norm.
 */
void orc_so_cn(const orc_params* p, cplx* psi, cplx z, int reverse) {
    if (p->so_type == 0 || p->gamma == 0.0) return;
    const double r2 = 1.0 / sqrt(2.0);
    const cplx SX[9] = {0, r2, 0, r2, 0, r2, 0, r2, 0};
    const cplx SY[9] = {0, -I * r2, 0, I * r2, 0, -I * r2, 0, I * r2, 0};
    const cplx SZ[9] = {1, 0, 0, 0, 0, 0, 0, 0, -1};
    const size_t plane = (size_t)p->nx * p->ny;
    if (p->dim == 1) {
        const cplx* S = p->so_type == 1 ? SX : (p->so_type == 2 ? SY : SZ);
        so_cn_line(psi, plane, 1, p->nx, S, p->gamma, p->dx, z);
        return;
    }
    const double eta = p->so_type == 1 ? 1.0 : (p->so_type == 2 ? -1.0 : 0.0);
    for (int pass = 0; pass < 2; pass++) {
        const int along_x = (pass == 0) != (reverse != 0);
        if (along_x) {
#pragma omp parallel for num_threads(g_threads) schedule(static)
            for (int iy = 0; iy < p->ny; iy++) so_cn_line(&psi[IDX(p, 0, iy, 0)], plane, 1, p->nx, SY, -p->gamma, p->dx, z);
        } else if (eta != 0.0) {
#pragma omp parallel for num_threads(g_threads) schedule(static)
            for (int ix = 0; ix < p->nx; ix++)
                so_cn_line(&psi[IDX(p, 0, 0, ix)], plane, (size_t)p->nx, p->ny, SX, eta * p->gamma, p->dy, z);
        }
    }
}

/*
 * CALCNU substep (Sec. 3): the trap and the square-bracket (diagonal) terms of
 * Eqs. (1)-(2) with the densities of the substep's input held fixed:
 *   mu_{+-} = V + c0 rho + c2 (rho_{+-} - rho_{-+} + rho_0),
 *   mu_0    = V + c0 rho + c2 (rho_+ + rho_-),
 *   psi_j <- exp(-z mu_j) psi_j.
 */
void orc_calcnu(const orc_params* p, cplx* psi, cplx z) {
#pragma omp parallel for num_threads(g_threads) schedule(static)
    for (int iy = 0; iy < p->ny; iy++)
        for (int ix = 0; ix < p->nx; ix++) {
            cplx* pp = &psi[IDX(p, 0, iy, ix)];
            cplx* p0 = &psi[IDX(p, 1, iy, ix)];
            cplx* pm = &psi[IDX(p, 2, iy, ix)];
            double rp = creal(*pp * conj(*pp)), r0 = creal(*p0 * conj(*p0)), rm = creal(*pm * conj(*pm));
            double rho = rp + r0 + rm;
            double V = trap(p, ix, iy);
            double mup = V + p->c0 * rho + p->c2 * (rp - rm + r0);
            double mu0 = V + p->c0 * rho + p->c2 * (rp + rm);
            double mum = V + p->c0 * rho + p->c2 * (rm - rp + r0);
            *pp *= cexp(-z * mup);
            *p0 *= cexp(-z * mu0);
            *pm *= cexp(-z * mum);
        }
}

/*
 * HERM substep, Appendix A Eqs. (nu) and (11): with
 *   a = c2 psi_-^* psi_0 + Ot,  b = c2 psi_0^* psi_+ + Ot,  Ot = Omega/sqrt2,
 * taken from the substep's input, the matrix A = [[0,a,0],[a*,0,b],[0,b*,0]]
 * has eigenvalues C, 0, -C (C = sqrt(|a|^2+|b|^2)) and eigenvector matrix V;
 * psi <- V diag(exp(-z lambda_k)) V^{-1} psi.  At C = 0 the matrix A vanishes
 * and the update is the identity (V^{-1} is undefined there).
 */
void orc_herm(const orc_params* p, cplx* psi, cplx z, double omega) {
    const double Ot = omega / sqrt(2.0);
#pragma omp parallel for num_threads(g_threads) schedule(static)
    for (int iy = 0; iy < p->ny; iy++)
        for (int ix = 0; ix < p->nx; ix++) {
            cplx* pp = &psi[IDX(p, 0, iy, ix)];
            cplx* p0 = &psi[IDX(p, 1, iy, ix)];
            cplx* pm = &psi[IDX(p, 2, iy, ix)];
            cplx a = p->c2 * conj(*pm) * *p0 + Ot;
            cplx b = p->c2 * conj(*p0) * *pp + Ot;
            double C = sqrt(creal(a * conj(a)) + creal(b * conj(b)));
            if (C == 0.0) continue;
            cplx V[3][3] = {{a, b, a}, {C, 0.0, -C}, {conj(b), -conj(a), conj(b)}};
            cplx W[3][3] = {{conj(a), C, b}, {2.0 * conj(b), 0.0, -2.0 * a}, {conj(a), -C, b}};
            double s = 1.0 / (2.0 * C * C);
            cplx e[3] = {cexp(-z * C), 1.0, cexp(z * C)};
            cplx in[3] = {*pp, *p0, *pm}, u[3], out[3];
            for (int k = 0; k < 3; k++) {
                u[k] = 0.0;
                for (int l = 0; l < 3; l++) u[k] += s * W[k][l] * in[l];
                u[k] *= e[k];
            }
            for (int k = 0; k < 3; k++) {
                out[k] = 0.0;
                for (int l = 0; l < 3; l++) out[k] += V[k][l] * u[l];
            }
            *pp = out[0];
            *p0 = out[1];
            *pm = out[2];
        }
}

/*
 * Crank-Nicolson for the kinetic term -1/2 d^2/ds^2 along one line (COEF + LU /
 * LUX / LUY, Sec. 3): with the 3-point second difference and bt = z/(4 h^2),
 *   (1 + 2 bt) y_i - bt (y_{i-1} + y_{i+1}) = (1 - 2 bt) x_i + bt (x_{i-1} + x_{i+1}),
 * zero ghosts; solved by Gaussian elimination of the tridiagonal system
 * without pivoting (Thomas algorithm; the matrix is diagonally dominant).
 */
static void cn_line(cplx* f, size_t stride, int n, cplx bt) {
    cplx* r = malloc(n * sizeof(cplx));
    cplx* cp = malloc(n * sizeof(cplx));
    for (int i = 0; i < n; i++) {
        cplx xm = i > 0 ? f[(i - 1) * stride] : 0.0;
        cplx xp = i + 1 < n ? f[(i + 1) * stride] : 0.0;
        r[i] = (1.0 - 2.0 * bt) * f[i * stride] + bt * (xm + xp);
    }
    cplx diag = 1.0 + 2.0 * bt, off = -bt;
    /* forward elimination */
    cp[0] = off / diag;
    r[0] = r[0] / diag;
    for (int i = 1; i < n; i++) {
        cplx den = diag - off * cp[i - 1];
        cp[i] = off / den;
        r[i] = (r[i] - off * r[i - 1]) / den;
    }
    /* back substitution */
    for (int i = n - 2; i >= 0; i--) r[i] -= cp[i] * r[i + 1];
    for (int i = 0; i < n; i++) f[i * stride] = r[i];
    free(r);
    free(cp);
}

void orc_cn_x(const orc_params* p, cplx* psi, cplx z) {
    cplx bt = z / (4.0 * p->dx * p->dx);
#pragma omp parallel for collapse(2) num_threads(g_threads) schedule(static)
    for (int j = 0; j < 3; j++)
        for (int iy = 0; iy < p->ny; iy++) cn_line(&psi[IDX(p, j, iy, 0)], 1, p->nx, bt);
}

void orc_cn_y(const orc_params* p, cplx* psi, cplx z) {
    if (p->dim != 2) return;
    cplx bt = z / (4.0 * p->dy * p->dy);
#pragma omp parallel for collapse(2) num_threads(g_threads) schedule(static)
    for (int j = 0; j < 3; j++)
        for (int ix = 0; ix < p->nx; ix++) cn_line(&psi[IDX(p, j, 0, ix)], (size_t)p->nx, p->ny, bt);
}

static double cell(const orc_params* p) { return p->dim == 2 ? p->dx * p->dy : p->dx; }

/* N_j = integral of rho_j, by the grid sum (Riemann rule) over all points. */
void orc_norms(const orc_params* p, const cplx* psi, double N[3]) {
    for (int j = 0; j < 3; j++) {
        double s = 0.0;
        for (int iy = 0; iy < p->ny; iy++)
            for (int ix = 0; ix < p->nx; ix++) {
                cplx v = psi[IDX(p, j, iy, ix)];
                s += creal(v * conj(v));
            }
        N[j] = s * cell(p);
    }
}

/*
 * RENORM (Appendix A): psi_j <- d_j psi_j with Eq. (DJ2),
 * d_j = 1/sqrt(N_0 + N_+ + N_-), or with Eq. (DJ) for fixed magnetisation m:
 *   d_0 = sqrt(1-m^2) / sqrt(N_0 + sqrt(4(1-m^2) N_+ N_- + m^2 N_0^2)),
 *   d_{+-} = sqrt(1 +- m - d_0^2 N_0) / sqrt(2 N_{+-}).
 * A component with N_j = 0 is left as it is (d_j has no value there), and so
 * is a state whose norm is zero.
 */
void orc_renorm(const orc_params* p, cplx* psi) {
    double N[3], d[3];
    orc_norms(p, psi, N);
    if (!(N[0] + N[1] + N[2] > 0.0)) return;
    if (p->renorm == 1) {
        d[0] = d[1] = d[2] = 1.0 / sqrt(N[0] + N[1] + N[2]);
    } else if (p->renorm == 2) {
        double m = p->mag;
        double den = N[1] + sqrt(4.0 * (1.0 - m * m) * N[0] * N[2] + m * m * N[1] * N[1]);
        if (!(den > 0.0)) return;
        d[1] = sqrt(1.0 - m * m) / sqrt(den);
        d[0] = N[0] > 0.0 ? sqrt(1.0 + m - d[1] * d[1] * N[1]) / sqrt(2.0 * N[0]) : 1.0;
        d[2] = N[2] > 0.0 ? sqrt(1.0 - m - d[1] * d[1] * N[1]) / sqrt(2.0 * N[2]) : 1.0;
        if (!(N[1] > 0.0)) d[1] = 1.0;
    } else {
        return;
    }
#pragma omp parallel for collapse(2) num_threads(g_threads) schedule(static)
    for (int j = 0; j < 3; j++)
        for (int iy = 0; iy < p->ny; iy++)
            for (int ix = 0; ix < p->nx; ix++) psi[IDX(p, j, iy, ix)] *= d[j];
}

/*
 * One or more full split steps (Sec. 3, "treated successively"): in the order
 * SO -> CALCNU -> HERM -> CN along x -> CN along y (2D) -> RENORM (imaginary
 * time only, when renorm != 0).  omega_t (nullable) gives Omega for step n.
 */
void orc_step(const orc_params* p, cplx* psi, int nsteps, int imag, const double* omega_t) {
    cplx z = imag ? (cplx)p->dt : I * p->dt;
    for (int n = 0; n < nsteps; n++) {
        double om = omega_t ? omega_t[n] : p->omega;
        if (!p->split) {
            if (p->so_mode) orc_so_cn(p, psi, z, 0);
            else orc_so(p, psi, z);
            orc_calcnu(p, psi, z);
            orc_herm(p, psi, z, om);
            orc_cn_x(p, psi, z);
            orc_cn_y(p, psi, z);
        } else {
            /* Strang: the same substeps with z/2 around the kinetic step (CN along
               x and y, which commute), then again in the reverse order */
            cplx h = 0.5 * z;
            if (p->so_mode) orc_so_cn(p, psi, h, 0);
            else orc_so(p, psi, h);
            orc_calcnu(p, psi, h);
            orc_herm(p, psi, h, om);
            orc_cn_x(p, psi, z);
            orc_cn_y(p, psi, z);
            orc_herm(p, psi, h, om);
            orc_calcnu(p, psi, h);
            if (p->so_mode) orc_so_cn(p, psi, h, 1);
            else orc_so(p, psi, h);
        }
        if (imag && p->renorm) orc_renorm(p, psi);
    }
}

/* One named substep, for per-substep tests: 0 SO, 1 CALCNU, 2 HERM, 3 CN-x, 4 CN-y, 5 RENORM,
   6 SO by Crank-Nicolson (x lines, then y lines), 7 the same in the reverse order. */
int orc_substep(const orc_params* p, cplx* psi, int which, int imag, double omega) {
    cplx z = imag ? (cplx)p->dt : I * p->dt;
    switch (which) {
        case 0: orc_so(p, psi, z); return 0;
        case 1: orc_calcnu(p, psi, z); return 0;
        case 2: orc_herm(p, psi, z, omega); return 0;
        case 3: orc_cn_x(p, psi, z); return 0;
        case 4: orc_cn_y(p, psi, z); return 0;
        case 5: orc_renorm(p, psi); return 0;
        case 6: orc_so_cn(p, psi, z, 0); return 0;
        case 7: orc_so_cn(p, psi, z, 1); return 0;
        default: return -1;
    }
}

/* Apply H_SO to the whole state (used for the energy and by the tests). */
void orc_apply_hso(const orc_params* p, const cplx* psi, cplx* out) {
    for (int iy = 0; iy < p->ny; iy++)
        for (int ix = 0; ix < p->nx; ix++) {
            cplx h[3];
            hso_point(p, psi, iy, ix, h);
            for (int j = 0; j < 3; j++) out[IDX(p, j, iy, ix)] = h[j];
        }
}

/*
 * Observables (ENERGY, LENGTH / RADIUS, Sec. 3), written to out[16]:
 *  0-2 N_+, N_0, N_-;  3 N = sum N_j;  4 m = N_+ - N_- (Eq. (noma));
 *  5 E, the energy functional Eq. (energy) on the grid;  6 mu;
 *  7-9 rms_j = sqrt(sum r^2 rho_j / sum rho_j);  10 rms of the total density;
 *  11-15 the parts of E: kinetic, trap, interaction (c0, c2), Rabi, SO.
 * Kinetic part: 1/2 sum_j sum over all grid links, ghost links included, of
 * |forward difference|^2 (this equals <psi, -1/2 D2 psi> with zero ghosts).
 * Interaction: 1/2 [c0 rho^2 + c2 (rho_+^2 + rho_-^2 + 2 rho_+ rho_0 + 2 rho_- rho_0
 *               - 2 rho_+ rho_- + 2 psi_-^* psi_0^2 psi_+^* + 2 c.c.)].
 * Rabi: (Omega/sqrt2) [(psi_+^* + psi_-^*) psi_0 + c.c.].  SO: Re sum_j psi_j^* (H_SO psi)_j.
 * mu = (E_kin + E_trap + E_SO + E_Rabi + 2 E_int) / N.
 * All integrals are grid sums times dx (dx dy in 2D).
 */
void orc_observables(const orc_params* p, const cplx* psi, double omega, double* out) {
    double w = cell(p);
    double N[3] = {0, 0, 0}, r2[3] = {0, 0, 0};
    double ekin = 0, etrap = 0, eint = 0, erabi = 0, eso = 0;
    const double Ot = omega / sqrt(2.0);
    size_t n = (size_t)3 * p->nx * p->ny;
    cplx* h = malloc(n * sizeof(cplx));
    orc_apply_hso(p, psi, h);
    for (int j = 0; j < 3; j++) {
        /* x links: (ix-1, ix) for ix = 0..nx, ghosts at -1 and nx */
        for (int iy = 0; iy < p->ny; iy++)
            for (int ix = 0; ix <= p->nx; ix++) {
                cplx a = ix < p->nx ? psi[IDX(p, j, iy, ix)] : 0.0;
                cplx b = ix > 0 ? psi[IDX(p, j, iy, ix - 1)] : 0.0;
                cplx d = (a - b) / p->dx;
                ekin += 0.5 * creal(d * conj(d));
            }
        if (p->dim == 2)
            for (int ix = 0; ix < p->nx; ix++)
                for (int iy = 0; iy <= p->ny; iy++) {
                    cplx a = iy < p->ny ? psi[IDX(p, j, iy, ix)] : 0.0;
                    cplx b = iy > 0 ? psi[IDX(p, j, iy - 1, ix)] : 0.0;
                    cplx d = (a - b) / p->dy;
                    ekin += 0.5 * creal(d * conj(d));
                }
    }
    for (int iy = 0; iy < p->ny; iy++)
        for (int ix = 0; ix < p->nx; ix++) {
            cplx pp = psi[IDX(p, 0, iy, ix)], p0 = psi[IDX(p, 1, iy, ix)], pm = psi[IDX(p, 2, iy, ix)];
            double rp = creal(pp * conj(pp)), r0 = creal(p0 * conj(p0)), rm = creal(pm * conj(pm));
            double rho = rp + r0 + rm;
            double x = xcoord(p, ix), y = ycoord(p, iy), rr = x * x + y * y;
            N[0] += rp;
            N[1] += r0;
            N[2] += rm;
            r2[0] += rr * rp;
            r2[1] += rr * r0;
            r2[2] += rr * rm;
            etrap += trap(p, ix, iy) * rho;
            cplx X = conj(pm) * p0 * p0 * conj(pp);
            eint += 0.5 * (p->c0 * rho * rho +
                           p->c2 * (rp * rp + rm * rm + 2.0 * rp * r0 + 2.0 * rm * r0 - 2.0 * rp * rm +
                                    2.0 * creal(X + conj(X))));
            cplx R = (conj(pp) + conj(pm)) * p0;
            erabi += Ot * creal(R + conj(R));
            for (int j = 0; j < 3; j++) eso += creal(conj(psi[IDX(p, j, iy, ix)]) * h[IDX(p, j, iy, ix)]);
        }
    free(h);
    double Nt = (N[0] + N[1] + N[2]) * w;
    out[0] = N[0] * w;
    out[1] = N[1] * w;
    out[2] = N[2] * w;
    out[3] = Nt;
    out[4] = (N[0] - N[2]) * w;
    ekin *= w;
    etrap *= w;
    eint *= w;
    erabi *= w;
    eso *= w;
    out[5] = ekin + etrap + eint + erabi + eso;
    out[6] = Nt > 0 ? (ekin + etrap + eso + erabi + 2.0 * eint) / Nt : 0.0;
    for (int j = 0; j < 3; j++) out[7 + j] = N[j] > 0 ? sqrt(r2[j] / N[j]) : 0.0;
    double Ns = N[0] + N[1] + N[2];
    out[10] = Ns > 0 ? sqrt((r2[0] + r2[1] + r2[2]) / Ns) : 0.0;
    out[11] = ekin;
    out[12] = etrap;
    out[13] = eint;
    out[14] = erabi;
    out[15] = eso;
}
