/*
 * physics.c -- plain FP64 CPU step functions of the two PDE workloads.
 *
 * TEST INFRASTRUCTURE (see oracle.c). These are the definitions the executor's PDE
 * loop chains are checked against; they use plain periodic (modular) indexing on
 * dense arrays without halos, no tiling and no ghost layers.
 *
 * Compressible Euler, 2-D (the stand-in for the CloverLeaf 2-D hydrodynamics of
 * arXiv 1709.02125 Sec. 5.1): conserved U = (rho, mx, my, E) on an nx x ny periodic
 * grid, ideal gas p = (gamma - 1)(E - (mx u + my v)/2), u = mx/rho, v = my/rho,
 * fluxes F = (mx, mx u + p, mx v, (E + p) u), G = (my, my u, my v + p, (E + p) v).
 * One MacCormack step with lx = dt/dx, ly = dt/dy:
 *   predictor  Us = U - lx (F[i+1] - F[i]) - ly (G[j+1] - G[j])
 *   corrector  Un = 0.5 (U + Us - lx (Fs[i] - Fs[i-1]) - ly (Gs[j] - Gs[j-1]))
 *                   - eps4 (d4x U + d4y U),
 *   d4x U = U[i-2] - 4 U[i-1] + 6 U[i] - 4 U[i+1] + U[i+2] (likewise in y),
 * where Fs, Gs are the fluxes of Us. The time step is
 *   dt = CFL * min over cells of min(dx / (|u| + c), dy / (|v| + c)), c = sqrt(gamma p / rho).
 *
 * Compressible Navier-Stokes, 3-D (stand-in for the OpenSBLI Taylor-Green vortex,
 * Sec. 5.1): conserved U = (rho, rho u, rho v, rho w, rho E), nondimensional with
 * p = (gamma - 1)(rho E - rho |u|^2 / 2), T = gamma Ma^2 p / rho, constant viscosity mu,
 * conductivity k = mu / ((gamma - 1) Ma^2 Pr). Fluxes in direction j:
 *   rho u_j,  rho u_i u_j + p delta_ij - tau_ij,  (rho E + p) u_j - u_i tau_ij - k dT/dx_j,
 * tau_ij = mu (du_i/dx_j + du_j/dx_i - 2/3 delta_ij div u). Spatial derivatives are the
 * fourth-order central difference D f = (f[-2] - 8 f[-1] + 8 f[+1] - f[+2]) / (12 h);
 * the residual is R = - sum_j D_j(flux_j) (divergence form; velocity and temperature
 * gradients are taken first, so second derivatives are first derivatives of first
 * derivatives). Time stepping: Williamson's low-storage RK3,
 *   dU = A_s dU + dt R(U); U = U + B_s dU, A = (0, -5/9, -153/128), B = (1/3, 15/16, 8/15).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

static inline int wrap(int i, int n) { return ((i % n) + n) % n; }

/* ---------------------------------------------------------------- Euler ---- */
#define IX2(i, j) ((size_t)wrap(j, ny) * (size_t)nx + (size_t)wrap(i, nx))

static void euler_flux(int nx, int ny, const double* U, double gamma, double* F, double* G)
{
    const size_t N = (size_t)nx * ny;
    const double* r = U;
    const double* mx = U + N;
    const double* my = U + 2 * N;
    const double* E = U + 3 * N;
    size_t q;
#pragma omp parallel for schedule(static)
    for (q = 0; q < N; ++q) {
        double u = mx[q] / r[q];
        double v = my[q] / r[q];
        double p = (gamma - 1.0) * (E[q] - 0.5 * (mx[q] * u + my[q] * v));
        F[q] = mx[q];
        F[N + q] = mx[q] * u + p;
        F[2 * N + q] = mx[q] * v;
        F[3 * N + q] = (E[q] + p) * u;
        G[q] = my[q];
        G[N + q] = my[q] * u;
        G[2 * N + q] = my[q] * v + p;
        G[3 * N + q] = (E[q] + p) * v;
    }
}

/* One MacCormack step of the periodic Euler system; U is (4, ny, nx), updated in place. */
void or_euler_step(int nx, int ny, double* U, double dt, double dx, double dy, double gamma,
                   double eps4)
{
    const size_t N = (size_t)nx * ny;
    double* F = (double*)malloc(sizeof(double) * 4 * N);
    double* G = (double*)malloc(sizeof(double) * 4 * N);
    double* Us = (double*)malloc(sizeof(double) * 4 * N);
    double* Un = (double*)malloc(sizeof(double) * 4 * N);
    const double lx = dt / dx, ly = dt / dy;
    euler_flux(nx, ny, U, gamma, F, G);
    int j;
#pragma omp parallel for schedule(static)
    for (j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i)
            for (int k = 0; k < 4; ++k) {
                const double* Fk = F + k * N;
                const double* Gk = G + k * N;
                Us[k * N + IX2(i, j)] = U[k * N + IX2(i, j)] - lx * (Fk[IX2(i + 1, j)] - Fk[IX2(i, j)])
                                        - ly * (Gk[IX2(i, j + 1)] - Gk[IX2(i, j)]);
            }
    euler_flux(nx, ny, Us, gamma, F, G);
#pragma omp parallel for schedule(static)
    for (j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i)
            for (int k = 0; k < 4; ++k) {
                const double* Uk = U + k * N;
                const double* Fk = F + k * N;
                const double* Gk = G + k * N;
                double d4x = Uk[IX2(i - 2, j)] - 4.0 * Uk[IX2(i - 1, j)] + 6.0 * Uk[IX2(i, j)]
                             - 4.0 * Uk[IX2(i + 1, j)] + Uk[IX2(i + 2, j)];
                double d4y = Uk[IX2(i, j - 2)] - 4.0 * Uk[IX2(i, j - 1)] + 6.0 * Uk[IX2(i, j)]
                             - 4.0 * Uk[IX2(i, j + 1)] + Uk[IX2(i, j + 2)];
                Un[k * N + IX2(i, j)] = 0.5 * (Uk[IX2(i, j)] + Us[k * N + IX2(i, j)]
                                               - lx * (Fk[IX2(i, j)] - Fk[IX2(i - 1, j)])
                                               - ly * (Gk[IX2(i, j)] - Gk[IX2(i, j - 1)]))
                                        - eps4 * (d4x + d4y);
            }
    memcpy(U, Un, sizeof(double) * 4 * N);
    free(F); free(G); free(Us); free(Un);
}

/* min over cells of min(dx / (|u| + c), dy / (|v| + c)) (the CFL number is applied by
 * the caller). */
double or_euler_dt(int nx, int ny, const double* U, double dx, double dy, double gamma)
{
    const size_t N = (size_t)nx * ny;
    double m = INFINITY;
    for (size_t q = 0; q < N; ++q) {
        double r = U[q], u = U[N + q] / r, v = U[2 * N + q] / r;
        double p = (gamma - 1.0) * (U[3 * N + q] - 0.5 * (U[N + q] * u + U[2 * N + q] * v));
        double c = sqrt(gamma * p / r);
        double a = dx / (fabs(u) + c), b = dy / (fabs(v) + c);
        double t = a < b ? a : b;
        if (t < m) m = t;
    }
    return m;
}

/* ------------------------------------------------------------ Navier-Stokes ---- */
#define IX3(i, j, k) (((size_t)wrap(k, nz) * (size_t)ny + (size_t)wrap(j, ny)) * (size_t)nx + (size_t)wrap(i, nx))

/* fourth-order central first derivative along axis a of f at (i, j, k) */
static inline double d1(const double* f, int nx, int ny, int nz, int i, int j, int k, int a, double h)
{
    int di = a == 0, dj = a == 1, dk = a == 2;
    double fm2 = f[IX3(i - 2 * di, j - 2 * dj, k - 2 * dk)];
    double fm1 = f[IX3(i - di, j - dj, k - dk)];
    double fp1 = f[IX3(i + di, j + dj, k + dk)];
    double fp2 = f[IX3(i + 2 * di, j + 2 * dj, k + 2 * dk)];
    return ((fm2 - 8.0 * fm1) + (8.0 * fp1 - fp2)) / (12.0 * h);
}

/* Flux of conserved component m (0 rho, 1-3 momentum, 4 energy) in direction a at
 * point c, from the state U, the primitives W = (u, v, w, p, T) and the gradients D
 * (D[3f + b] = d(u, v, w, T)_f / dx_b). */
static double ns_flux(const double* U, const double* W, const double* D, size_t N, double mu,
                      double kc, int m, int a, size_t c)
{
    const double vel[3] = {W[c], W[N + c], W[2 * N + c]};
    const double p = W[3 * N + c];
    const double div = D[0 * N + c] + D[4 * N + c] + D[8 * N + c];
    double tau[3];  /* tau[b] = tau_{b a} */
    for (int b = 0; b < 3; ++b)
        tau[b] = mu * (D[(3 * b + a) * N + c] + D[(3 * a + b) * N + c] - (b == a ? (2.0 / 3.0) * div : 0.0));
    if (m == 0) return U[(size_t)(a + 1) * N + c];
    if (m <= 3) return U[(size_t)m * N + c] * vel[a] + (m - 1 == a ? p : 0.0) - tau[m - 1];
    return (U[4 * N + c] + p) * vel[a] - (vel[0] * tau[0] + vel[1] * tau[1] + vel[2] * tau[2])
           - kc * D[(9 + a) * N + c];
}

/* Residual R(U) of the periodic NS system. U and R are (5, nz, ny, nx).
 * prm = [gamma, Ma, Re, Pr, hx, hy, hz] (mu = 1/Re; Re <= 0 means inviscid). */
void or_ns_residual(int nx, int ny, int nz, const double* U, const double* prm, double* R)
{
    const size_t N = (size_t)nx * ny * nz;
    const double gamma = prm[0], Ma = prm[1], Re = prm[2], Pr = prm[3];
    const double h[3] = {prm[4], prm[5], prm[6]};
    const double mu = Re > 0 ? 1.0 / Re : 0.0;
    const double kc = mu / ((gamma - 1.0) * Ma * Ma * Pr);
    double* W = (double*)malloc(sizeof(double) * 5 * N);   /* u, v, w, p, T */
    double* D = (double*)malloc(sizeof(double) * 12 * N);  /* d{u,v,w,T}/d{x,y,z} */
    size_t q;
#pragma omp parallel for schedule(static)
    for (q = 0; q < N; ++q) {
        double r = U[q];
        double u = U[N + q] / r, v = U[2 * N + q] / r, w = U[3 * N + q] / r;
        double p = (gamma - 1.0) * (U[4 * N + q] - 0.5 * (U[N + q] * u + U[2 * N + q] * v + U[3 * N + q] * w));
        W[q] = u; W[N + q] = v; W[2 * N + q] = w; W[3 * N + q] = p;
        W[4 * N + q] = gamma * Ma * Ma * p / r;
    }
    int k;
#pragma omp parallel for schedule(static)
    for (k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                size_t c = IX3(i, j, k);
                for (int f = 0; f < 4; ++f) {
                    const double* src = W + (f == 3 ? 4 : f) * N;  /* u, v, w, T */
                    for (int a = 0; a < 3; ++a) D[(3 * f + a) * N + c] = d1(src, nx, ny, nz, i, j, k, a, h[a]);
                }
            }
#pragma omp parallel for schedule(static)
    for (k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                size_t c = IX3(i, j, k);
                for (int m = 0; m < 5; ++m) {
                    double r = 0.0;
                    for (int a = 0; a < 3; ++a) {
                        int di = a == 0, dj = a == 1, dk = a == 2;
                        size_t cm2 = IX3(i - 2 * di, j - 2 * dj, k - 2 * dk), cm1 = IX3(i - di, j - dj, k - dk);
                        size_t cp1 = IX3(i + di, j + dj, k + dk), cp2 = IX3(i + 2 * di, j + 2 * dj, k + 2 * dk);
                        double fm2 = ns_flux(U, W, D, N, mu, kc, m, a, cm2);
                        double fm1 = ns_flux(U, W, D, N, mu, kc, m, a, cm1);
                        double fp1 = ns_flux(U, W, D, N, mu, kc, m, a, cp1);
                        double fp2 = ns_flux(U, W, D, N, mu, kc, m, a, cp2);
                        r = r - ((fm2 - 8.0 * fm1) + (8.0 * fp1 - fp2)) / (12.0 * h[a]);
                    }
                    R[m * N + c] = r;
                }
            }
    free(W);
    free(D);
}

/* One step of Williamson's low-storage RK3 (three stages). U is (5, nz, ny, nx). */
void or_ns_step(int nx, int ny, int nz, double* U, double dt, const double* prm)
{
    static const double A[3] = {0.0, -5.0 / 9.0, -153.0 / 128.0};
    static const double B[3] = {1.0 / 3.0, 15.0 / 16.0, 8.0 / 15.0};
    const size_t N = (size_t)nx * ny * nz;
    double* dU = (double*)calloc(5 * N, sizeof(double));
    double* R = (double*)malloc(sizeof(double) * 5 * N);
    for (int s = 0; s < 3; ++s) {
        or_ns_residual(nx, ny, nz, U, prm, R);
        size_t q;
#pragma omp parallel for schedule(static)
        for (q = 0; q < 5 * N; ++q) {
            dU[q] = A[s] * dU[q] + dt * R[q];
            U[q] = U[q] + B[s] * dU[q];
        }
    }
    free(dU);
    free(R);
}
