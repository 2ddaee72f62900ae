/*
 * FP64 CPU oracle for the pressure-projection step of the hybrid CNN + Jacobi
 * incompressible solver (arXiv 2109.09363).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call, link or
 * load this file; only the test-suite, the smoke check and the CPU-baseline leg
 * of the benchmark do.  It shares no code with the CUDA library.
 *
 * Everything here is written to be read against the paper, not to be fast:
 *   - MAC staggered grid, finite differences, boolean obstacle field  (Sec. 2.2)
 *   - corrected velocity u = u* - (dt/rho0) grad p                    (Eq. 2)
 *   - Poisson equation (dt/rho0) lap p = div u*                        (Eq. 3)
 *   - Jacobi iteration X_{t+1} = D^{-1}(b - (L+U) X_t)                 (Sec. 2.2)
 *   - E_1 = mean |div u|, E_inf = max |div u|                          (Sec. 4.1)
 *   - hybrid rule: iterate until E <= E_t                              (Sec. 3.3, Fig. 5)
 *
 * Conventions (the paper leaves them open; the readings are listed in the
 * design notes):
 *   cell (i, j): i = column (x), j = row; row 0 is the top of the image.
 *   u[b][j][i], i = 0..nx : face between cells (i-1, j) and (i, j).
 *   v[b][j][i], j = 0..ny : face between cells (i, j-1) and (i, j).
 *   flags[b][j][i] != 0   : solid cell.
 *   A face is open when it is not on the domain boundary and both cells next
 *   to it are fluid; every other face is closed and carries zero velocity.
 *   phi = (dt/rho0) p, so that the discrete Laplacian is the unit stencil.
 *   E_1 divides by all nx*ny cells (solid cells count as zero divergence).
 *
 * Sums that reach a reported number are taken in a fixed order (row by row,
 * then rows in order) so that results do not depend on the thread count.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---------------------------------------------------------------- geometry */

static int is_fluid(const uint8_t *fl, int ny, int nx, int j, int i)
{
    (void)ny;
    return fl[(size_t)j * nx + i] == 0;
}

/* u face (j, i) is open: interior column and both neighbours fluid */
static int open_u(const uint8_t *fl, int ny, int nx, int j, int i)
{
    if (i <= 0 || i >= nx) return 0;
    return is_fluid(fl, ny, nx, j, i - 1) && is_fluid(fl, ny, nx, j, i);
}

/* v face (j, i) is open: interior row and both neighbours fluid */
static int open_v(const uint8_t *fl, int ny, int nx, int j, int i)
{
    if (j <= 0 || j >= ny) return 0;
    return is_fluid(fl, ny, nx, j - 1, i) && is_fluid(fl, ny, nx, j, i);
}

/* Open-face bits of a cell: 1 = west (u face i), 2 = east (u face i+1),
 * 4 = north (v face j, towards row j-1), 8 = south (v face j+1).  Solid cells
 * have no open face. */
void or_face_mask(const uint8_t *flags, int B, int ny, int nx, uint8_t *mask)
{
    for (int b = 0; b < B; ++b) {
        const uint8_t *fl = flags + (size_t)b * ny * nx;
        uint8_t *m = mask + (size_t)b * ny * nx;
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                int bits = 0;
                if (is_fluid(fl, ny, nx, j, i)) {
                    if (open_u(fl, ny, nx, j, i)) bits |= 1;
                    if (open_u(fl, ny, nx, j, i + 1)) bits |= 2;
                    if (open_v(fl, ny, nx, j, i)) bits |= 4;
                    if (open_v(fl, ny, nx, j + 1, i)) bits |= 8;
                }
                m[(size_t)j * nx + i] = (uint8_t)bits;
            }
    }
}

/* ------------------------------------------------------- divergence (Eq. 3) */

/* Set the velocity of every closed face to zero (static walls and obstacles). */
void or_zero_closed_faces(double *u, double *v, const uint8_t *flags, int B, int ny, int nx)
{
    for (int b = 0; b < B; ++b) {
        const uint8_t *fl = flags + (size_t)b * ny * nx;
        double *ub = u + (size_t)b * ny * (nx + 1);
        double *vb = v + (size_t)b * (ny + 1) * nx;
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i <= nx; ++i)
                if (!open_u(fl, ny, nx, j, i)) ub[(size_t)j * (nx + 1) + i] = 0.0;
        for (int j = 0; j <= ny; ++j)
            for (int i = 0; i < nx; ++i)
                if (!open_v(fl, ny, nx, j, i)) vb[(size_t)j * nx + i] = 0.0;
    }
}

/* First-order forward difference of the face velocities, dx = 1; only open
 * faces carry flux.  Solid cells get zero. */
static void divergence_one(const double *u, const double *v, const uint8_t *fl,
                           int ny, int nx, double *div)
{
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            double d = 0.0;
            if (is_fluid(fl, ny, nx, j, i)) {
                double ue = open_u(fl, ny, nx, j, i + 1) ? u[(size_t)j * (nx + 1) + i + 1] : 0.0;
                double uw = open_u(fl, ny, nx, j, i) ? u[(size_t)j * (nx + 1) + i] : 0.0;
                double vs = open_v(fl, ny, nx, j + 1, i) ? v[(size_t)(j + 1) * nx + i] : 0.0;
                double vn = open_v(fl, ny, nx, j, i) ? v[(size_t)j * nx + i] : 0.0;
                d = (ue - uw) + (vs - vn);
            }
            div[(size_t)j * nx + i] = d;
        }
}

void or_divergence(const double *u, const double *v, const uint8_t *flags, int B, int ny,
                   int nx, double *div)
{
    for (int b = 0; b < B; ++b)
        divergence_one(u + (size_t)b * ny * (nx + 1), v + (size_t)b * (ny + 1) * nx,
                       flags + (size_t)b * ny * nx, ny, nx, div + (size_t)b * ny * nx);
}

/* ----------------------------------------------- Laplacian, Jacobi, residual */

/* Discrete Laplacian with zero-flux (Neumann) closed faces:
 * (L phi)_c = sum over open faces of (phi_nb - phi_c). */
static double laplacian_at(const double *phi, const uint8_t *fl, int ny, int nx, int j, int i)
{
    double c = phi[(size_t)j * nx + i], s = 0.0;
    if (open_u(fl, ny, nx, j, i)) s += phi[(size_t)j * nx + i - 1] - c;
    if (open_u(fl, ny, nx, j, i + 1)) s += phi[(size_t)j * nx + i + 1] - c;
    if (open_v(fl, ny, nx, j, i)) s += phi[(size_t)(j - 1) * nx + i] - c;
    if (open_v(fl, ny, nx, j + 1, i)) s += phi[(size_t)(j + 1) * nx + i] - c;
    return s;
}

static int open_count(const uint8_t *fl, int ny, int nx, int j, int i)
{
    return open_u(fl, ny, nx, j, i) + open_u(fl, ny, nx, j, i + 1) + open_v(fl, ny, nx, j, i) +
           open_v(fl, ny, nx, j + 1, i);
}

/* residual r_c = div_c - (L phi)_c on fluid cells, 0 on solid cells */
static double residual_at(const double *phi, const double *div, const uint8_t *fl, int ny,
                          int nx, int j, int i)
{
    if (!is_fluid(fl, ny, nx, j, i)) return 0.0;
    return div[(size_t)j * nx + i] - laplacian_at(phi, fl, ny, nx, j, i);
}

/* One Jacobi sweep, X_{t+1} = D^{-1}(b - (L+U) X_t), written per cell:
 * phi'_c = (sum over open faces of phi_nb - div_c) / n_c.  Cells with no open
 * face (solid or isolated) are set to zero. */
static void sweep_one(const double *phi, const double *div, const uint8_t *fl, int ny, int nx,
                      double *out)
{
#pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            double val = 0.0;
            int n = is_fluid(fl, ny, nx, j, i) ? open_count(fl, ny, nx, j, i) : 0;
            if (n > 0) {
                double s = 0.0;
                if (open_u(fl, ny, nx, j, i)) s += phi[(size_t)j * nx + i - 1];
                if (open_u(fl, ny, nx, j, i + 1)) s += phi[(size_t)j * nx + i + 1];
                if (open_v(fl, ny, nx, j, i)) s += phi[(size_t)(j - 1) * nx + i];
                if (open_v(fl, ny, nx, j + 1, i)) s += phi[(size_t)(j + 1) * nx + i];
                val = (s - div[(size_t)j * nx + i]) / (double)n;
            }
            out[(size_t)j * nx + i] = val;
        }
}

void or_jacobi_sweep(const double *phi, const double *div, const uint8_t *flags, int B, int ny,
                     int nx, double *out)
{
    for (int b = 0; b < B; ++b)
        sweep_one(phi + (size_t)b * ny * nx, div + (size_t)b * ny * nx,
                  flags + (size_t)b * ny * nx, ny, nx, out + (size_t)b * ny * nx);
}

/* E(phi) = sum_c |r_c(phi)| / (nx * ny), summed row by row in order. */
static double mean_abs_residual(const double *phi, const double *div, const uint8_t *fl, int ny,
                                int nx, double *rowbuf)
{
#pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; ++j) {
        double s = 0.0;
        for (int i = 0; i < nx; ++i) s += fabs(residual_at(phi, div, fl, ny, nx, j, i));
        rowbuf[j] = s;
    }
    double tot = 0.0;
    for (int j = 0; j < ny; ++j) tot += rowbuf[j];
    return tot / ((double)nx * (double)ny);
}

void or_residual(const double *phi, const double *div, const uint8_t *flags, int B, int ny,
                 int nx, double *r)
{
    for (int b = 0; b < B; ++b)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i)
                r[(size_t)b * ny * nx + (size_t)j * nx + i] =
                    residual_at(phi + (size_t)b * ny * nx, div + (size_t)b * ny * nx,
                                flags + (size_t)b * ny * nx, ny, nx, j, i);
}

void or_mean_abs_residual(const double *phi, const double *div, const uint8_t *flags, int B,
                          int ny, int nx, double *e_out)
{
    double *rowbuf = (double *)malloc(sizeof(double) * (size_t)ny);
    for (int b = 0; b < B; ++b)
        e_out[b] = mean_abs_residual(phi + (size_t)b * ny * nx, div + (size_t)b * ny * nx,
                                     flags + (size_t)b * ny * nx, ny, nx, rowbuf);
    free(rowbuf);
}

/* ------------------------------------------------------ correction (Eq. 2) */

/* u = u* - grad phi on open faces, 0 on closed faces; p = phi * rho0 / dt. */
static void correct_one(double *u, double *v, const double *phi, const uint8_t *fl, int ny,
                        int nx)
{
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i <= nx; ++i) {
            double *f = &u[(size_t)j * (nx + 1) + i];
            if (open_u(fl, ny, nx, j, i))
                *f = *f - (phi[(size_t)j * nx + i] - phi[(size_t)j * nx + i - 1]);
            else
                *f = 0.0;
        }
    for (int j = 0; j <= ny; ++j)
        for (int i = 0; i < nx; ++i) {
            double *f = &v[(size_t)j * nx + i];
            if (open_v(fl, ny, nx, j, i))
                *f = *f - (phi[(size_t)j * nx + i] - phi[(size_t)(j - 1) * nx + i]);
            else
                *f = 0.0;
        }
}

void or_correct(double *u, double *v, const double *phi, const uint8_t *flags, int B, int ny,
                int nx)
{
    for (int b = 0; b < B; ++b)
        correct_one(u + (size_t)b * ny * (nx + 1), v + (size_t)b * (ny + 1) * nx,
                    phi + (size_t)b * ny * nx, flags + (size_t)b * ny * nx, ny, nx);
}

/* E_1 = mean |div u| over all cells and E_inf = max |div u|. */
void or_div_norms(const double *u, const double *v, const uint8_t *flags, int B, int ny, int nx,
                  double *e1, double *einf)
{
    double *div = (double *)malloc(sizeof(double) * (size_t)ny * nx);
    for (int b = 0; b < B; ++b) {
        divergence_one(u + (size_t)b * ny * (nx + 1), v + (size_t)b * (ny + 1) * nx,
                       flags + (size_t)b * ny * nx, ny, nx, div);
        double tot = 0.0, mx = 0.0;
        for (int j = 0; j < ny; ++j) {
            double s = 0.0;
            for (int i = 0; i < nx; ++i) {
                double a = fabs(div[(size_t)j * nx + i]);
                s += a;
                if (a > mx) mx = a;
            }
            tot += s;
        }
        e1[b] = tot / ((double)nx * (double)ny);
        einf[b] = mx;
    }
    free(div);
}

/* ------------------------------------------------ projection (Sec. 2.2, 3.3) */

/*
 * Pressure projection of B independent grids, in place on (u, v).
 *   1. zero the closed faces of u*;  2. div = div u*  (Eq. 3, right-hand side);
 *   3. phi_0 = given initial guess (the CNN output of the hybrid method) or 0;
 *   4. for k = 0, 1, ...: E_k = mean |r(phi_k)|; stop if E_k <= E_t (converged)
 *      or if k == max_iters (not converged); else phi_{k+1} = Jacobi(phi_k);
 *      with fixed_iters > 0 the test is skipped and exactly fixed_iters sweeps run;
 *   5. correct u (Eq. 2); p = phi rho0 / dt;
 *   6. E_1 and E_inf of the corrected velocity.
 * e_hist (optional, [B][hist_len]) receives E_k for k < hist_len (NAN beyond
 * the stopping point) so that tests can read the margin at the crossing.
 */
void or_project(double *u, double *v, const uint8_t *flags, int B, int ny, int nx,
                double threshold, int max_iters, int fixed_iters, double dt, double rho0,
                const double *phi0, double *p_out, double *phi_out, int32_t *iters_out,
                double *e1_out, double *einf_out, uint8_t *converged_out, double *e_hist,
                int hist_len)
{
    size_t cells = (size_t)ny * nx;
    double *div = (double *)malloc(sizeof(double) * cells);
    double *a = (double *)malloc(sizeof(double) * cells);
    double *c = (double *)malloc(sizeof(double) * cells);
    double *rowbuf = (double *)malloc(sizeof(double) * (size_t)ny);
    for (int b = 0; b < B; ++b) {
        double *ub = u + (size_t)b * ny * (nx + 1);
        double *vb = v + (size_t)b * (ny + 1) * nx;
        const uint8_t *fl = flags + (size_t)b * cells;
        or_zero_closed_faces(ub, vb, fl, 1, ny, nx);
        divergence_one(ub, vb, fl, ny, nx, div);
        /* a cell without an open face (solid or walled in) carries no pressure
         * unknown: its phi_0 is set to zero */
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                size_t q = (size_t)j * nx + i;
                int dof = is_fluid(fl, ny, nx, j, i) && open_count(fl, ny, nx, j, i) > 0;
                a[q] = (phi0 && dof) ? phi0[(size_t)b * cells + q] : 0.0;
            }
        double *hist = e_hist ? e_hist + (size_t)b * hist_len : NULL;
        if (hist)
            for (int q = 0; q < hist_len; ++q) hist[q] = NAN;
        int k = 0, conv = 0;
        if (fixed_iters > 0) {
            for (k = 0; k < fixed_iters; ++k) {
                sweep_one(a, div, fl, ny, nx, c);
                double *t = a; a = c; c = t;
            }
            conv = 1;
        } else {
            for (k = 0;; ++k) {
                double e = mean_abs_residual(a, div, fl, ny, nx, rowbuf);
                if (hist && k < hist_len) hist[k] = e;
                if (e <= threshold) { conv = 1; break; }
                if (k == max_iters) { conv = 0; break; }
                sweep_one(a, div, fl, ny, nx, c);
                double *t = a; a = c; c = t;
            }
        }
        correct_one(ub, vb, a, fl, ny, nx);
        for (size_t q = 0; q < cells; ++q) {
            if (p_out) p_out[(size_t)b * cells + q] = a[q] * rho0 / dt;
            if (phi_out) phi_out[(size_t)b * cells + q] = a[q];
        }
        iters_out[b] = k;
        converged_out[b] = (uint8_t)conv;
        or_div_norms(ub, vb, fl, 1, ny, nx, &e1_out[b], &einf_out[b]);
    }
    free(div); free(a); free(c); free(rowbuf);
}

/* ------------------------------------------------ adjoint of the projection */

/*
 * Adjoint (transpose) of the affine map phi_0 -> phi_k of k Jacobi sweeps
 * with right-hand side div.  The paper states only that the gradient of the
 * correction is known (Sec. 3.2); the transposes are written out here from the
 * forward definitions:
 *   forward  phi_{t+1} = D^{-1} (W phi_t - div)      (W: open-face adjacency)
 *   backward lam_t = W D^{-1} lam_{t+1},  g_div -= D^{-1} lam_{t+1}
 * with D^{-1} = 0 on cells without an open face.  Returns g_phi0 = lam_0 and
 * accumulates into g_div.
 */
void or_jacobi_adjoint(const double *g_phik, const uint8_t *flags, int B, int ny, int nx, int k,
                       double *g_phi0, double *g_div)
{
    size_t cells = (size_t)ny * nx;
    double *lam = (double *)malloc(sizeof(double) * cells);
    double *nxt = (double *)malloc(sizeof(double) * cells);
    for (int b = 0; b < B; ++b) {
        const uint8_t *fl = flags + (size_t)b * cells;
        memcpy(lam, g_phik + (size_t)b * cells, sizeof(double) * cells);
        double *gd = g_div + (size_t)b * cells;
        for (int t = 0; t < k; ++t) {
            /* mu = D^{-1} lam */
            for (int j = 0; j < ny; ++j)
                for (int i = 0; i < nx; ++i) {
                    int n = is_fluid(fl, ny, nx, j, i) ? open_count(fl, ny, nx, j, i) : 0;
                    double mu = n > 0 ? lam[(size_t)j * nx + i] / (double)n : 0.0;
                    nxt[(size_t)j * nx + i] = mu;
                    gd[(size_t)j * nx + i] -= mu;
                }
            /* lam_t = W mu : each cell gathers mu of its open-face neighbours */
            for (int j = 0; j < ny; ++j)
                for (int i = 0; i < nx; ++i) {
                    double s = 0.0;
                    if (is_fluid(fl, ny, nx, j, i)) {
                        if (open_u(fl, ny, nx, j, i)) s += nxt[(size_t)j * nx + i - 1];
                        if (open_u(fl, ny, nx, j, i + 1)) s += nxt[(size_t)j * nx + i + 1];
                        if (open_v(fl, ny, nx, j, i)) s += nxt[(size_t)(j - 1) * nx + i];
                        if (open_v(fl, ny, nx, j + 1, i)) s += nxt[(size_t)(j + 1) * nx + i];
                    }
                    lam[(size_t)j * nx + i] = s;
                }
        }
        memcpy(g_phi0 + (size_t)b * cells, lam, sizeof(double) * cells);
    }
    free(lam); free(nxt);
}

/* --------------------------------------------------------- thread control */

int or_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}
