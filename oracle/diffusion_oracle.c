/*
 * Oracle for the substrate diffusion step: plain, slow, FP64, CPU only.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file; only the tests and the CPU-baseline leg of the benchmark
 * do.  It shares no code, header or constant with the CUDA library.
 *
 * The paper names the microenvironment solver and the gradient computation
 * as load-imbalanced regions of the simulation, each a loop over a domain of
 * 75 x 75 x 75 voxels (Sec. 5.1, Sec. 5.2), but states no numerical method.
 * The statement implemented here (ours):
 *
 *   S substrate densities rho_s on nx x ny x nz cubic voxels of side dx
 *   (voxel v = x + nx (y + ny z), array [s][v]), each with a diffusion
 *   coefficient D_s and a decay rate lambda_s, no-flux faces.  One step of
 *   length dt splits d rho/dt = D lap(rho) - lambda rho into three
 *   one-dimensional backward-Euler solves, along x, then y, then z, the decay
 *   shared equally among them.  Along a line of n voxels, with
 *   k = D dt / dx^2 and e = lambda dt / 3, the new values solve
 *       (1 + k + e) r_0     - k r_1                     = old_0
 *      -k r_{i-1} + (1 + 2k + e) r_i - k r_{i+1}        = old_i   (0 < i < n-1)
 *      -k r_{n-2} + (1 + k + e) r_{n-1}                  = old_{n-1}
 *   (for n = 1: (1 + e) r_0 = old_0), the face rows being the interior rows
 *   with a mirrored neighbour (no flux through the face).
 *
 *   The solve is the textbook Thomas algorithm (forward elimination, then
 *   back substitution), dividing by each pivot, in FP64 with no contraction:
 *      m_0 = T_00;  c_i = -k / m_i;  m_i = T_ii + k c_{i-1}   (i >= 1)
 *      forward  r_0 = old_0 / m_0;  r_i = (old_i + k r_{i-1}) / m_i
 *      backward r_i = r_i - c_i r_{i+1}   (i = n-2 .. 0)
 *   (Any other arrangement of the same elimination, e.g. multiplying by
 *   reciprocal pivots, agrees with this one to rounding only.)
 *
 *   Gradient of rho_s along each axis: central differences
 *   (rho[i+1] - rho[i-1]) / (2 dx) inside, one-sided differences at the two
 *   faces, zero on an axis of one voxel; array [s][axis][v].
 *
 * Build: compiled with the mechanics oracle into liboracle.so (gcc -O2
 * -ffp-contract=off, no fast-math).
 */
#include <stdint.h>
#include <stdlib.h>

/* Thomas coefficients of one axis: pivots m[0..n), c[0..n-1). */
static void coefficients(int64_t n, double k, double e, double* m, double* c) {
    for (int64_t i = 0; i < n; ++i) {
        double diag;
        if (n == 1) diag = 1.0 + e;
        else if (i == 0 || i == n - 1) diag = 1.0 + k + e;
        else diag = 1.0 + 2.0 * k + e;
        m[i] = i == 0 ? diag : diag + k * c[i - 1];
        if (i < n - 1) c[i] = -k / m[i];
    }
}

/* One line of n values at p[0], p[stride], ... solved in place. */
static void solve_line(double* p, int64_t stride, int64_t n, double k, const double* m, const double* c) {
    p[0] = p[0] / m[0];
    for (int64_t i = 1; i < n; ++i) p[i * stride] = (p[i * stride] + k * p[(i - 1) * stride]) / m[i];
    for (int64_t i = n - 2; i >= 0; --i) p[i * stride] = p[i * stride] - c[i] * p[(i + 1) * stride];
}

int oracle_diffusion_step(int64_t nx, int64_t ny, int64_t nz, int32_t S, double* rho, const double* D,
                          const double* lambda, double dx, double dt, int64_t steps) {
    const int64_t nmax = nx > ny ? (nx > nz ? nx : nz) : (ny > nz ? ny : nz);
    double* m = malloc(sizeof(double) * (size_t)nmax);
    double* c = malloc(sizeof(double) * (size_t)nmax);
    if (!m || !c) {
        free(m);
        free(c);
        return -1;
    }
    const int64_t nv = nx * ny * nz;
    for (int64_t step = 0; step < steps; ++step) {
        for (int32_t s = 0; s < S; ++s) {
            double* r = rho + (int64_t)s * nv;
            const double k = D[s] * dt / (dx * dx);
            const double e = lambda[s] * dt / 3.0;
            /* x lines */
            coefficients(nx, k, e, m, c);
            for (int64_t z = 0; z < nz; ++z)
                for (int64_t y = 0; y < ny; ++y) solve_line(r + nx * (y + ny * z), 1, nx, k, m, c);
            /* y lines */
            coefficients(ny, k, e, m, c);
            for (int64_t z = 0; z < nz; ++z)
                for (int64_t x = 0; x < nx; ++x) solve_line(r + x + nx * ny * z, nx, ny, k, m, c);
            /* z lines */
            coefficients(nz, k, e, m, c);
            for (int64_t y = 0; y < ny; ++y)
                for (int64_t x = 0; x < nx; ++x) solve_line(r + x + nx * y, nx * ny, nz, k, m, c);
        }
    }
    free(m);
    free(c);
    return 0;
}

void oracle_diffusion_gradient(int64_t nx, int64_t ny, int64_t nz, int32_t S, const double* rho, double dx,
                               double* grad) {
    const int64_t nv = nx * ny * nz;
    const int64_t n[3] = {nx, ny, nz};
    const int64_t stride[3] = {1, nx, nx * ny};
    for (int32_t s = 0; s < S; ++s)
        for (int a = 0; a < 3; ++a)
            for (int64_t z = 0; z < nz; ++z)
                for (int64_t y = 0; y < ny; ++y)
                    for (int64_t x = 0; x < nx; ++x) {
                        const int64_t v = x + nx * (y + ny * z);
                        const int64_t i = a == 0 ? x : (a == 1 ? y : z);
                        const double* r = rho + (int64_t)s * nv;
                        double g;
                        if (n[a] == 1) g = 0.0;
                        else if (i == 0) g = (r[v + stride[a]] - r[v]) / dx;
                        else if (i == n[a] - 1) g = (r[v] - r[v - stride[a]]) / dx;
                        else g = (r[v + stride[a]] - r[v - stride[a]]) / (2.0 * dx);
                        grad[((int64_t)s * 3 + a) * nv + v] = g;
                    }
}
