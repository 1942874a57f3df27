/*
 * FP64 CPU oracle of the constant-density acoustic wave stepper
 * (arXiv 2204.03775, Section II, Eq. 1-2 and Algorithm 1).
 *
 * TEST INFRASTRUCTURE ONLY. This file is the slow, plain reference that the
 * CUDA path is checked against. Only the tests, the smoke check and the
 * benchmark's CPU-baseline / reference leg may load it. It shares no code,
 * header, table or constant with the CUDA library, and the CUDA library never
 * calls it.
 *
 * Everything is double precision. Loops are the textbook triple loops; the
 * only parallelism is an OpenMP "parallel for" over the outer z loop, which
 * does not change any result (every point is computed independently).
 *
 * Grid convention: interior points (i, j, k), 0 <= i < nx, 0 <= j < ny,
 * 0 <= k < nz, x fastest, k = 0 is the top plane. Internal wavefield arrays
 * carry a 4-cell halo on every face (the paper extends each column by four
 * cells on each side, Section III-B), stored as [nz+8][ny+8][nx+8].
 * User-facing arrays are unpadded [nz][ny][nx].
 *
 * Readings of the paper that this file takes (the paper leaves them open):
 *  - coefficients c_0..c_4 are the 8th-order central Taylor weights of the
 *    second derivative, supplied by the caller (the Python shim solves for
 *    them in exact rational arithmetic); the centre weight is applied once
 *    per axis (Section III-C-2 folds c_x0 + c_y0 + c_z0 into a single
 *    multiply of the centre cell);
 *  - the velocity enters per point through (v dt)^2, as in Eq. 2;
 *  - the source of Eq. 2's right-hand side is a Ricker wavelet added, after
 *    damping, to u^{n+1} at one cell, scaled by (v_s dt)^2, with t_n = n dt;
 *  - boundaries: zero-Dirichlet halo (or periodic, for tests only);
 *  - absorbing layer: Cerjan taper g = gx(i) gy(j) gz(k), applied as
 *    u^{n+1} = g (2 u^n - g u^{n-1} + (v dt)^2 Lap u^n), i.e. both time
 *    levels are multiplied by g after each plain step;
 *  - receivers record u^{n+1} at their cell after step n.
 */
#include <math.h>
#include <stddef.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define HALO 4

/* Offset of interior point (i, j, k) (each may lie in [-4, n+4)) in a padded
 * [nz+8][ny+8][nx+8] array. */
static size_t pidx(int i, int j, int k, int nx, int ny)
{
    return ((size_t)(k + HALO) * (size_t)(ny + 2 * HALO) + (size_t)(j + HALO))
               * (size_t)(nx + 2 * HALO)
           + (size_t)(i + HALO);
}

static size_t uidx(int i, int j, int k, int nx, int ny)
{
    return ((size_t)k * (size_t)ny + (size_t)j) * (size_t)nx + (size_t)i;
}

static size_t padded_size(int nx, int ny, int nz)
{
    return (size_t)(nx + 2 * HALO) * (size_t)(ny + 2 * HALO) * (size_t)(nz + 2 * HALO);
}

static int wrap(int i, int n)
{
    int r = i % n;
    return r < 0 ? r + n : r;
}

int or_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Fill the 4-cell halo of a padded array: zeros (Dirichlet) or periodic
 * images of the interior (used only by the convergence and dispersion tests). */
void or_fill_halo(double *u, int nx, int ny, int nz, int periodic)
{
    for (int k = -HALO; k < nz + HALO; ++k)
        for (int j = -HALO; j < ny + HALO; ++j)
            for (int i = -HALO; i < nx + HALO; ++i) {
                int inside = i >= 0 && i < nx && j >= 0 && j < ny && k >= 0 && k < nz;
                if (inside)
                    continue;
                u[pidx(i, j, k, nx, ny)] =
                    periodic ? u[pidx(wrap(i, nx), wrap(j, ny), wrap(k, nz), nx, ny)] : 0.0;
            }
}

/* 25-point star Laplacian at one interior point (Section II, the 25-point
 * formula; neighbour sets of Section III-C): for each axis, the 8th-order
 * second difference c_0 u + sum_{m=1..4} c_m (u(+m) + u(-m)), summed over the
 * three axes and divided by h^2. */
static double lap_at(const double *u, int i, int j, int k, int nx, int ny,
                     double h, const double *c)
{
    double lx = c[0] * u[pidx(i, j, k, nx, ny)];
    double ly = c[0] * u[pidx(i, j, k, nx, ny)];
    double lz = c[0] * u[pidx(i, j, k, nx, ny)];
    for (int m = 1; m <= 4; ++m) {
        lx += c[m] * (u[pidx(i + m, j, k, nx, ny)] + u[pidx(i - m, j, k, nx, ny)]);
        ly += c[m] * (u[pidx(i, j + m, k, nx, ny)] + u[pidx(i, j - m, k, nx, ny)]);
        lz += c[m] * (u[pidx(i, j, k + m, nx, ny)] + u[pidx(i, j, k - m, nx, ny)]);
    }
    return (lx + ly + lz) / (h * h);
}

/* Laplacian of a padded field whose halo the caller has filled; the result
 * is written unpadded. Used directly by the polynomial-exactness and
 * convergence tests. */
void or_laplacian(const double *u_padded, double *lap, int nx, int ny, int nz,
                  double h, const double *c)
{
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i)
                lap[uidx(i, j, k, nx, ny)] = lap_at(u_padded, i, j, k, nx, ny, h, c);
}

/* Cerjan taper for the cell at index idx of an axis of n cells: with d its
 * distance (in cells) to the nearer outer face, g = exp(-(a (nb - d))^2) for
 * d < nb and 1 elsewhere. The paper evaluates no boundary condition (Section
 * II); this absorbing layer is the build's addition. */
double or_cerjan(int idx, int n, int nb, double a)
{
    int d = idx < n - 1 - idx ? idx : n - 1 - idx;
    if (nb <= 0 || d >= nb)
        return 1.0;
    double x = a * (double)(nb - d);
    return exp(-x * x);
}

/* Ricker wavelet amp (1 - 2 pi^2 f0^2 tau^2) exp(-pi^2 f0^2 tau^2), tau = t - t0:
 * the source time function f^n of Eq. 2 as used here (the paper names none). */
double or_ricker(double t, double f0, double t0, double amp)
{
    const double pi = 3.14159265358979323846;
    double tau = t - t0;
    double x = pi * pi * f0 * f0 * tau * tau;
    return amp * (1.0 - 2.0 * x) * exp(-x);
}

/*
 * Time loop of Algorithm 1 with the update of Eq. 2.
 *
 * The computed box is the interior [0,nx) x [0,ny) x [0,nz). When win is not
 * NULL it is {ox, oy, oz, NX, NY, NZ}: the box is the window starting at
 * global cell (ox, oy, oz) of an NX x NY x NZ grid; damping factors use the
 * global coordinates, source and receiver cells are given in global
 * coordinates, and the window's outside is zero. That equals the full-grid
 * result inside the window whenever the wavefield cannot reach the window's
 * faces that are not faces of the global grid (4 cells per step at most).
 *
 *   vel        [nz][ny][nx] velocity (m/s) of the box
 *   c          5 coefficients c_0..c_4 (unscaled; divided by h^2 here)
 *   nb, a      Cerjan width (cells) and strength; nb = 0 disables damping
 *   src_ijk    [nsrc][3] global source cells; src_par [nsrc][3] = f0, t0, amp
 *   src_series NULL, or [nsrc][nt]: the source function f^{n0+n} of each
 *              source, used instead of the Ricker wavelet
 *   rec_ijk    [nrec][3] global receiver cells
 *   nt         number of steps; n0 = global index of the first step
 *   u_init, uprev_init   initial u^{n0}, u^{n0-1} of the box (NULL = zero)
 *   periodic   1 = periodic halo (tests only), 0 = zero-Dirichlet
 *   traces     [nrec][nt]: traces[r][n] = u^{n0+n+1} at receiver r (may be NULL)
 *   u_out, uprev_out     final u^{n0+nt}, u^{n0+nt-1} of the box (may be NULL)
 * Returns 0, or -1 on a bad argument or a failed allocation.
 */
int or_run(int nx, int ny, int nz, double h, double dt, const double *c,
           const double *vel, int nb, double a,
           int nsrc, const int *src_ijk, const double *src_par,
           int nrec, const int *rec_ijk, int nt, long long n0,
           const double *u_init, const double *uprev_init, int periodic,
           const int *win, const double *src_series,
           double *traces, double *u_out, double *uprev_out)
{
    if (nx < 1 || ny < 1 || nz < 1 || nt < 0 || h <= 0.0 || dt <= 0.0)
        return -1;
    int ox = 0, oy = 0, oz = 0, NX = nx, NY = ny, NZ = nz;
    if (win) {
        ox = win[0]; oy = win[1]; oz = win[2];
        NX = win[3]; NY = win[4]; NZ = win[5];
        if (ox < 0 || oy < 0 || oz < 0 || ox + nx > NX || oy + ny > NY || oz + nz > NZ)
            return -1;
    }
    for (int s = 0; s < nsrc; ++s) {
        int i = src_ijk[3 * s] - ox, j = src_ijk[3 * s + 1] - oy, k = src_ijk[3 * s + 2] - oz;
        if (i < 0 || i >= nx || j < 0 || j >= ny || k < 0 || k >= nz)
            return -1;
    }
    for (int r = 0; r < nrec; ++r) {
        int i = rec_ijk[3 * r] - ox, j = rec_ijk[3 * r + 1] - oy, k = rec_ijk[3 * r + 2] - oz;
        if (i < 0 || i >= nx || j < 0 || j >= ny || k < 0 || k >= nz)
            return -1;
    }

    size_t np = padded_size(nx, ny, nz);
    double *u_prev = calloc(np, sizeof(double));
    double *u_cur = calloc(np, sizeof(double));
    double *u_next = calloc(np, sizeof(double));
    double *gx = malloc(sizeof(double) * (size_t)nx);
    double *gy = malloc(sizeof(double) * (size_t)ny);
    double *gz = malloc(sizeof(double) * (size_t)nz);
    if (!u_prev || !u_cur || !u_next || !gx || !gy || !gz) {
        free(u_prev); free(u_cur); free(u_next); free(gx); free(gy); free(gz);
        return -1;
    }
    for (int i = 0; i < nx; ++i) gx[i] = or_cerjan(ox + i, NX, nb, a);
    for (int j = 0; j < ny; ++j) gy[j] = or_cerjan(oy + j, NY, nb, a);
    for (int k = 0; k < nz; ++k) gz[k] = or_cerjan(oz + k, NZ, nb, a);

    /* u^0 := 0 (Algorithm 1), or the caller's state. */
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                size_t p = pidx(i, j, k, nx, ny), q = uidx(i, j, k, nx, ny);
                u_cur[p] = u_init ? u_init[q] : 0.0;
                u_prev[p] = uprev_init ? uprev_init[q] : 0.0;
            }

    for (int n = 0; n < nt; ++n) {
        or_fill_halo(u_cur, nx, ny, nz, periodic);

        /* Eq. 2: u^{n+1} = Q u^n - u^{n-1}, Q = 2 + dt^2 V^2 Lap, then the
         * absorbing taper on both time levels. */
#pragma omp parallel for schedule(static)
        for (int k = 0; k < nz; ++k)
            for (int j = 0; j < ny; ++j)
                for (int i = 0; i < nx; ++i) {
                    size_t p = pidx(i, j, k, nx, ny);
                    double v = vel[uidx(i, j, k, nx, ny)];
                    double vdt2 = (v * dt) * (v * dt);
                    double g = gx[i] * gy[j] * gz[k];
                    double L = lap_at(u_cur, i, j, k, nx, ny, h, c);
                    u_next[p] = g * (2.0 * u_cur[p] - g * u_prev[p] + vdt2 * L);
                }

        /* Right-hand side of Eq. 2: dt^2 V^2 f^n at the source cell. */
        double t = (double)(n0 + n) * dt;
        for (int s = 0; s < nsrc; ++s) {
            int i = src_ijk[3 * s] - ox, j = src_ijk[3 * s + 1] - oy, k = src_ijk[3 * s + 2] - oz;
            double v = vel[uidx(i, j, k, nx, ny)];
            double f = src_series ? src_series[(size_t)s * (size_t)nt + (size_t)n]
                                  : or_ricker(t, src_par[3 * s], src_par[3 * s + 1], src_par[3 * s + 2]);
            u_next[pidx(i, j, k, nx, ny)] += (v * dt) * (v * dt) * f;
        }

        if (traces)
            for (int r = 0; r < nrec; ++r) {
                int i = rec_ijk[3 * r] - ox, j = rec_ijk[3 * r + 1] - oy, k = rec_ijk[3 * r + 2] - oz;
                traces[(size_t)r * (size_t)nt + (size_t)n] = u_next[pidx(i, j, k, nx, ny)];
            }

        double *tmp = u_prev;
        u_prev = u_cur;
        u_cur = u_next;
        u_next = tmp;
    }

    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                size_t p = pidx(i, j, k, nx, ny), q = uidx(i, j, k, nx, ny);
                if (u_out) u_out[q] = u_cur[p];
                if (uprev_out) uprev_out[q] = u_prev[p];
            }

    free(u_prev); free(u_cur); free(u_next); free(gx); free(gy); free(gz);
    return 0;
}

/*
 * Misfit J = 1/2 sum_r sum_n (u^{n+1}[rec_r] - d_obs[r][n])^2 of a run from
 * rest (nt steps, Eq. 2 with the taper and sources as in or_run, zero
 * Dirichlet halo) and its exact discrete gradient with respect to the
 * squared slowness m = 1/V^2 of every cell, by the adjoint (Lagrange
 * multiplier) recurrence of the step equations. The paper has no adjoint;
 * this is the build's extension, written in the plain multiplier form.
 *
 * With W = (V dt)^2, G the taper, A = G (2 + W L), B = G^2 and the step
 * u^{n+1} = A u^n - B u^{n-1} + f^n (f^n = W_s s_n at the source cell), the
 * multipliers obey, for k = nt .. 1 with lambda^{nt+1} = lambda^{nt+2} = 0,
 *     lambda^k = A^T lambda^{k+1} - B^T lambda^{k+2} + r^k,
 *     A^T lambda = 2 G lambda + L (W G lambda),   B^T lambda = G^2 lambda,
 * r^k = dJ/du^k = sum_r (u^k[rec_r] - d_obs[r][k-1]) e_{rec_r}; and
 *     dJ/dW_i = sum_n lambda^{n+1}_i (G_i (L u^n)_i + [i = s] s_n),
 *     dJ/dm_i = dJ/dW_i * dW_i/dm_i = -W_i V_i^2 dJ/dW_i.
 * Every forward state is kept (small grids only).
 *
 * Outputs: *misfit; grad_m [nz][ny][nx]; traces [nrec][nt] (may be NULL);
 * dj_dsrc [nsrc][nt] = dJ/ds_n = lambda^{n+1}_s W_s (may be NULL), the
 * adjoint of the map from source functions to traces.
 * Returns 0, or -1 on a bad argument or a failed allocation.
 */
int or_adjoint_gradient(int nx, int ny, int nz, double h, double dt, const double *c,
                        const double *vel, int nb, double a,
                        int nsrc, const int *src_ijk, const double *src_par,
                        const double *src_series,
                        int nrec, const int *rec_ijk, int nt, const double *d_obs,
                        double *misfit, double *grad_m, double *traces, double *dj_dsrc)
{
    if (nx < 1 || ny < 1 || nz < 1 || nt < 1 || nrec < 1 || h <= 0.0 || dt <= 0.0)
        return -1;
    size_t np = padded_size(nx, ny, nz), nc = (size_t)nx * ny * nz;
    double *states = calloc(np * (size_t)(nt + 2), sizeof(double));  /* u^{-1}, u^0 .. u^nt */
    double *lam = calloc(np * 3, sizeof(double));                  /* lambda^{k}, ^{k+1}, ^{k+2} */
    double *q = calloc(np, sizeof(double));
    double *w = malloc(sizeof(double) * nc), *g = malloc(sizeof(double) * nc);
    double *gw = calloc(nc, sizeof(double));
    double *tr = malloc(sizeof(double) * (size_t)nrec * nt);
    if (!states || !lam || !q || !w || !g || !gw || !tr) {
        free(states); free(lam); free(q); free(w); free(g); free(gw); free(tr);
        return -1;
    }
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                size_t o = uidx(i, j, k, nx, ny);
                w[o] = (vel[o] * dt) * (vel[o] * dt);
                g[o] = or_cerjan(i, nx, nb, a) * or_cerjan(j, ny, nb, a) * or_cerjan(k, nz, nb, a);
            }
#define STATE(n) (states + np * (size_t)((n) + 1))   /* u^n, n = -1 .. nt */

    /* forward, keeping every state */
    for (int n = 0; n < nt; ++n) {
        double *um = STATE(n - 1), *u = STATE(n), *un = STATE(n + 1);
#pragma omp parallel for schedule(static)
        for (int k = 0; k < nz; ++k)
            for (int j = 0; j < ny; ++j)
                for (int i = 0; i < nx; ++i) {
                    size_t p = pidx(i, j, k, nx, ny), o = uidx(i, j, k, nx, ny);
                    double L = lap_at(u, i, j, k, nx, ny, h, c);
                    un[p] = g[o] * (2.0 * u[p] - g[o] * um[p] + w[o] * L);
                }
        for (int s = 0; s < nsrc; ++s) {
            int i = src_ijk[3 * s], j = src_ijk[3 * s + 1], k = src_ijk[3 * s + 2];
            double f = src_series ? src_series[(size_t)s * nt + n]
                                  : or_ricker(n * dt, src_par[3 * s], src_par[3 * s + 1],
                                              src_par[3 * s + 2]);
            un[pidx(i, j, k, nx, ny)] += w[uidx(i, j, k, nx, ny)] * f;
        }
        for (int r = 0; r < nrec; ++r)
            tr[(size_t)r * nt + n] = un[pidx(rec_ijk[3 * r], rec_ijk[3 * r + 1], rec_ijk[3 * r + 2], nx, ny)];
    }
    double J = 0.0;
    for (size_t t = 0; t < (size_t)nrec * nt; ++t) {
        double d = tr[t] - d_obs[t];
        J += 0.5 * d * d;
    }

    /* backward: lambda^k for k = nt .. 1 (rotating three buffers) */
    double *lk2 = lam, *lk1 = lam + np, *lk = lam + 2 * np;   /* ^{k+2}, ^{k+1}, ^k */
    for (int kk = nt; kk >= 1; --kk) {
        /* q = W G lambda^{k+1} on the padded grid, zero halo */
        for (int k = 0; k < nz; ++k)
            for (int j = 0; j < ny; ++j)
                for (int i = 0; i < nx; ++i) {
                    size_t p = pidx(i, j, k, nx, ny), o = uidx(i, j, k, nx, ny);
                    q[p] = w[o] * g[o] * lk1[p];
                }
#pragma omp parallel for schedule(static)
        for (int k = 0; k < nz; ++k)
            for (int j = 0; j < ny; ++j)
                for (int i = 0; i < nx; ++i) {
                    size_t p = pidx(i, j, k, nx, ny), o = uidx(i, j, k, nx, ny);
                    lk[p] = 2.0 * g[o] * lk1[p] + lap_at(q, i, j, k, nx, ny, h, c)
                            - g[o] * g[o] * lk2[p];
                }
        for (int r = 0; r < nrec; ++r) {
            size_t p = pidx(rec_ijk[3 * r], rec_ijk[3 * r + 1], rec_ijk[3 * r + 2], nx, ny);
            lk[p] += tr[(size_t)r * nt + (kk - 1)] - d_obs[(size_t)r * nt + (kk - 1)];
        }
        /* lambda^k = lambda^{n+1} with n = kk - 1: gradient terms of step n */
        {
            const int n = kk - 1;
            double *u = STATE(n);
#pragma omp parallel for schedule(static)
            for (int k = 0; k < nz; ++k)
                for (int j = 0; j < ny; ++j)
                    for (int i = 0; i < nx; ++i) {
                        size_t p = pidx(i, j, k, nx, ny), o = uidx(i, j, k, nx, ny);
                        gw[o] += lk[p] * g[o] * lap_at(u, i, j, k, nx, ny, h, c);
                    }
            for (int s = 0; s < nsrc; ++s) {
                int i = src_ijk[3 * s], j = src_ijk[3 * s + 1], k = src_ijk[3 * s + 2];
                size_t p = pidx(i, j, k, nx, ny), o = uidx(i, j, k, nx, ny);
                double f = src_series ? src_series[(size_t)s * nt + n]
                                      : or_ricker(n * dt, src_par[3 * s], src_par[3 * s + 1],
                                                  src_par[3 * s + 2]);
                gw[o] += lk[p] * f;
                if (dj_dsrc) dj_dsrc[(size_t)s * nt + n] = lk[p] * w[o];
            }
        }
        double *tmp = lk2;
        lk2 = lk1;
        lk1 = lk;
        lk = tmp;
    }
#undef STATE
    for (size_t o = 0; o < nc; ++o) grad_m[o] = -w[o] * vel[o] * vel[o] * gw[o];
    *misfit = J;
    if (traces) memcpy(traces, tr, sizeof(double) * (size_t)nrec * nt);
    free(states); free(lam); free(q); free(w); free(g); free(gw); free(tr);
    return 0;
}
