/*
 * FP64 reference implementation ("oracle") of the formal solution used by the test suite.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline
 * leg may load this library.  It shares no code, header, table or constant with the CUDA path.
 * Every routine is a plain transcription of the discrete method, written for reading, not speed.
 *
 * Conventions
 *   fields   [nlam][npt] row-major, npt = nx*ny*nz with x fastest (regular) or the site index
 *   dirs     [ndir][3] unit vectors (mu_x, mu_y, mu_z), mu_z != 0; wdir[ndir] with sum 1
 *   bc       0 = thermal bottom (I = S) and zero top, 1 = zero on both walls,
 *            2 = inflow array I_bc[ndir][nlam][nb] on the wall each ray enters through
 *            (nb = nx*ny for the regular grid, nsites for the Voronoi grid)
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* ---------------------------------------------------------------------------------------
 * Linear-S integration over one optical-depth interval (Sect. 2.5: S linearly interpolated
 * across the interval; Eq. 2).  With d = delta tau, the source integral over the interval is
 *   int_0^d S(t) exp(-(d - t)) dt = w0 * S_up + w1 * S_here,
 *   e0 = 1 - exp(-d),  e1 = d - e0,  w1 = e1 / d,  w0 = e0 - w1 = e0 / d - exp(-d).
 * Below d = 1e-6 the cancellation in e1 is avoided with the Taylor series of w0 and w1; w0 is
 * evaluated as e0 / d - exp(-d), which keeps its relative precision for very thick intervals
 * (there w0 -> 1/d while w1 -> 1, and e0 - w1 would cancel).
 * ------------------------------------------------------------------------------------- */
void orc_linear_weights(double d, double *ex, double *w0, double *w1)
{
    if (d < 1e-6) {
        *ex = exp(-d);
        *w1 = d * (0.5 - d * (1.0 / 6.0 - d / 24.0));
        *w0 = d * (0.5 - d * (1.0 / 3.0 - d / 8.0));
        return;
    }
    double e0 = -expm1(-d);
    *ex = exp(-d);
    *w1 = (d - e0) / d;
    *w0 = e0 / d - *ex;
}

/* derivatives of (exp(-d), w0, w1) with respect to d, for the adjoint */
void orc_linear_weights_deriv(double d, double *dex, double *dw0, double *dw1)
{
    if (d < 1e-6) {
        *dex = -exp(-d);
        *dw1 = 0.5 - d * (1.0 / 3.0 - d / 8.0);
        *dw0 = 0.5 - d * (2.0 / 3.0 - d * 3.0 / 8.0);
        return;
    }
    double ex = exp(-d);
    double e0 = -expm1(-d);
    *dex = -ex;
    *dw1 = (e0 - d * ex) / (d * d);
    *dw0 = ex - *dw1;
}

/* ---------------------------------------------------------------------------------------
 * Regular grid: plane-to-plane short characteristics (Sect. 2.6, after Kunasz & Auer).
 * For a point of plane k the upwind point is where the ray through it crosses the previous
 * plane of the sweep (k-1 for mu_z > 0, k+1 for mu_z < 0).  I, S and alpha are bilinearly
 * interpolated there; periodic in x and y, or (periodic = 0) with zero inflow intensity and
 * edge-clamped S, alpha outside the box.  delta tau = (alpha_up + alpha) / 2 * ds.
 * ------------------------------------------------------------------------------------- */
typedef struct {
    int nx, ny, nz;
    double dx, dy;
    const double *z;
    int periodic;
} orc_reg;

static inline int wrap(int i, int n) { i %= n; return i < 0 ? i + n : i; }

/* bilinear stencil of the upwind point: 4 plane indices (or -1 = outside), 4 weights */
static void upwind_stencil(const orc_reg *g, int i, int j, double ox, double oy, int idx[4],
                           double wt[4])
{
    double fx = (double)i - ox / g->dx;
    double fy = (double)j - oy / g->dy;
    double fx0 = floor(fx), fy0 = floor(fy);
    double tx = fx - fx0, ty = fy - fy0;
    int i0 = (int)fx0, j0 = (int)fy0;
    int ii[2] = {i0, i0 + 1}, jj[2] = {j0, j0 + 1};
    double wx[2] = {1.0 - tx, tx}, wy[2] = {1.0 - ty, ty};
    for (int b = 0; b < 2; ++b)
        for (int a = 0; a < 2; ++a) {
            int c = 2 * b + a;
            int xi = ii[a], yj = jj[b];
            wt[c] = wx[a] * wy[b];
            if (g->periodic) {
                idx[c] = wrap(yj, g->ny) * g->nx + wrap(xi, g->nx);
            } else if (xi < 0 || xi >= g->nx || yj < 0 || yj >= g->ny) {
                idx[c] = -1 - ((xi < 0 ? 0 : (xi >= g->nx ? g->nx - 1 : xi)) +
                               g->nx * (yj < 0 ? 0 : (yj >= g->ny ? g->ny - 1 : yj)));
            } else {
                idx[c] = yj * g->nx + xi;
            }
        }
}

/* one direction, one wavelength: intensity I[npt] of the whole grid */
static void sc_one(const orc_reg *g, const double *mu, const double *al, const double *S,
                   int bc, const double *ibc, double *I)
{
    const int nx = g->nx, ny = g->ny, nz = g->nz, np = nx * ny;
    const int up = mu[2] > 0.0;
    const int k0 = up ? 0 : nz - 1;
    for (int p = 0; p < np; ++p) {
        double v;
        if (bc == 2) v = ibc[p];
        else if (bc == 0 && up) v = S[k0 * np + p];
        else v = 0.0;
        I[k0 * np + p] = v;
    }
    for (int s = 1; s < nz; ++s) {
        int k = up ? s : nz - 1 - s;
        int ku = up ? k - 1 : k + 1;
        double dz = fabs(g->z[k] - g->z[ku]);
        double ds = dz / fabs(mu[2]);
        double ox = ds * mu[0], oy = ds * mu[1];
        const double *Iu = I + (size_t)ku * np, *Su = S + (size_t)ku * np, *Au = al + (size_t)ku * np;
#pragma omp parallel for schedule(static)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                int idx[4];
                double wt[4];
                upwind_stencil(g, i, j, ox, oy, idx, wt);
                double iu = 0.0, su = 0.0, au = 0.0;
                for (int c = 0; c < 4; ++c) {
                    if (idx[c] >= 0) {
                        iu += wt[c] * Iu[idx[c]];
                        su += wt[c] * Su[idx[c]];
                        au += wt[c] * Au[idx[c]];
                    } else {
                        int q = -1 - idx[c];        /* outside: no inflow, clamped S, alpha */
                        su += wt[c] * Su[q];
                        au += wt[c] * Au[q];
                    }
                }
                int p = k * np + j * nx + i;
                double d = 0.5 * (au + al[p]) * ds, ex, w0, w1;
                orc_linear_weights(d, &ex, &w0, &w1);
                I[p] = iu * ex + w0 * su + w1 * S[p];
            }
    }
}

/* J[nlam][npt] = sum_d w_d I_d; optional I_out[ndir][nlam][npt] */
int orc_sc_regular(int nx, int ny, int nz, double dx, double dy, const double *z, int periodic,
                   int ndir, const double *dirs, const double *wdir, int nlam,
                   const double *alpha, const double *S, int bc, const double *ibc, double *J,
                   double *I_out)
{
    orc_reg g = {nx, ny, nz, dx, dy, z, periodic};
    size_t npt = (size_t)nx * ny * nz, nb = (size_t)nx * ny;
    double *I = (double *)malloc(npt * sizeof(double));
    if (!I) return -1;
    memset(J, 0, sizeof(double) * npt * nlam);
    for (int d = 0; d < ndir; ++d)
        for (int l = 0; l < nlam; ++l) {
            sc_one(&g, dirs + 3 * d, alpha + l * npt, S + l * npt, bc,
                   ibc ? ibc + ((size_t)d * nlam + l) * nb : NULL, I);
            for (size_t p = 0; p < npt; ++p) J[l * npt + p] += wdir[d] * I[p];
            if (I_out) memcpy(I_out + ((size_t)d * nlam + l) * npt, I, npt * sizeof(double));
        }
    free(I);
    return 0;
}

/* ---------------------------------------------------------------------------------------
 * Adjoint of the regular sweep for one direction: given gI[nlam][npt] (the gradient of a
 * scalar loss with respect to the intensity of this direction at every point), accumulate
 * g_alpha, g_S [nlam][npt].  Hand-derived reverse of sc_one: planes in reverse sweep order,
 * each interpolation transposed into a scatter onto the four upwind corners.
 * ------------------------------------------------------------------------------------- */
int orc_sc_regular_adjoint(int nx, int ny, int nz, double dx, double dy, const double *z,
                           int periodic, const double *mu, int nlam, const double *alpha,
                           const double *S, int bc, const double *gI, double *g_alpha,
                           double *g_S)
{
    orc_reg g = {nx, ny, nz, dx, dy, z, periodic};
    size_t npt = (size_t)nx * ny * nz, np = (size_t)nx * ny;
    double *I = (double *)malloc(npt * sizeof(double));
    double *gi = (double *)malloc(npt * sizeof(double));
    if (!I || !gi) { free(I); free(gi); return -1; }
    const int up = mu[2] > 0.0;
    for (int l = 0; l < nlam; ++l) {
        const double *al = alpha + l * npt, *Sl = S + l * npt;
        double *ga = g_alpha + l * npt, *gs = g_S + l * npt;
        sc_one(&g, mu, al, Sl, bc, NULL, I);
        memcpy(gi, gI + l * npt, npt * sizeof(double));
        for (int s = nz - 1; s >= 1; --s) {
            int k = up ? s : nz - 1 - s;
            int ku = up ? k - 1 : k + 1;
            double dz = fabs(g.z[k] - g.z[ku]);
            double ds = dz / fabs(mu[2]);
            double ox = ds * mu[0], oy = ds * mu[1];
            for (int j = 0; j < ny; ++j)
                for (int i = 0; i < nx; ++i) {
                    int idx[4];
                    double wt[4];
                    upwind_stencil(&g, i, j, ox, oy, idx, wt);
                    double iu = 0.0, su = 0.0, au = 0.0;
                    for (int c = 0; c < 4; ++c) {
                        int q = idx[c] >= 0 ? idx[c] : -1 - idx[c];
                        if (idx[c] >= 0) iu += wt[c] * I[ku * np + q];
                        su += wt[c] * Sl[ku * np + q];
                        au += wt[c] * al[ku * np + q];
                    }
                    size_t p = k * np + j * nx + i;
                    double d = 0.5 * (au + al[p]) * ds, ex, w0, w1, dex, dw0, dw1;
                    orc_linear_weights(d, &ex, &w0, &w1);
                    orc_linear_weights_deriv(d, &dex, &dw0, &dw1);
                    double gb = gi[p];
                    double gd = gb * (iu * dex + su * dw0 + Sl[p] * dw1);
                    gs[p] += w1 * gb;
                    ga[p] += 0.5 * ds * gd;
                    for (int c = 0; c < 4; ++c) {
                        int q = idx[c] >= 0 ? idx[c] : -1 - idx[c];
                        if (idx[c] >= 0) gi[ku * np + q] += wt[c] * ex * gb;
                        gs[ku * np + q] += wt[c] * w0 * gb;
                        ga[ku * np + q] += wt[c] * 0.5 * ds * gd;
                    }
                }
        }
        /* boundary plane: thermal bottom inflow I = S */
        if (bc == 0 && up)
            for (size_t p = 0; p < np; ++p) gs[p] += gi[p];
    }
    free(I);
    free(gi);
    return 0;
}

/* ---------------------------------------------------------------------------------------
 * Regular grid: face-hitting short characteristics (Kunasz & Auer 1988, the scheme Sect. 2.6
 * names for the regular-grid solver).  The ray through a point of plane k is followed upwind
 * to the first face of the grid cell it enters:
 *   - the plane face (the previous plane of the sweep) when dz/|mu_z| <= dx/|mu_x| and
 *     dz/|mu_z| <= dy/|mu_y|: the upwind point lies within one cell of the point's column and
 *     I, S, alpha are bilinearly interpolated there in that plane;
 *   - otherwise the vertical face x = x_i - sx dx (when dx/|mu_x| < dy/|mu_y|), else
 *     y = y_j - sy dy (on a tie the ray meets the edge the two faces share, and both give the
 *     same upwind point): I, S, alpha are bilinearly interpolated on that face between its two grid
 *     lines (j and j - sy, or i and i - sx) and the two planes k and k -/+ 1.
 * Segment length t = the distance to that face; delta tau = (alpha_up + alpha) / 2 * t; S
 * linear across the interval (Eq. 2).  Periodic in x and y.
 *
 * On a vertical face two of the four corners lie in plane k itself, so the intensities of the
 * plane depend on one another along the face-normal axis a, around the periodic box.  In sweep
 * order a_0, a_1, ..., a_{n-1} (the line before a_0 is a_{n-1}) each line x_m of intensities
 * over the other axis b obeys x_m = C_m x_{m-1} + r_m, with C_m the weights of the two corners
 * in plane k times e^-dtau and r_m all the rest.  Composing the n steps gives
 * x_{n-1} = P x_{n-1} + q; (1 - P) x_{n-1} = q is solved by Gaussian elimination with partial
 * pivoting, and one more pass along a yields every line.
 * ------------------------------------------------------------------------------------- */

/* A x = b for a dense n x n row-major A (overwritten); b becomes x.  -1 if singular. */
static int gauss_solve(int n, double *A, double *b)
{
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (fabs(A[(size_t)r * n + c]) > fabs(A[(size_t)piv * n + c])) piv = r;
        if (A[(size_t)piv * n + c] == 0.0) return -1;
        if (piv != c) {
            for (int k = 0; k < n; ++k) {
                double t = A[(size_t)c * n + k];
                A[(size_t)c * n + k] = A[(size_t)piv * n + k];
                A[(size_t)piv * n + k] = t;
            }
            double t = b[c];
            b[c] = b[piv];
            b[piv] = t;
        }
        for (int r = c + 1; r < n; ++r) {
            double f = A[(size_t)r * n + c] / A[(size_t)c * n + c];
            for (int k = c; k < n; ++k) A[(size_t)r * n + k] -= f * A[(size_t)c * n + k];
            b[r] -= f * b[c];
        }
    }
    for (int c = n - 1; c >= 0; --c) {
        double s = b[c];
        for (int k = c + 1; k < n; ++k) s -= A[(size_t)c * n + k] * b[k];
        b[c] = s / A[(size_t)c * n + c];
    }
    return 0;
}

/* index in a plane of the point at position a on the face-normal axis and b on the other */
typedef struct {
    int a_is_x, nx;
} orc_axes;

static inline int plane_index(const orc_axes *ax, int a, int b)
{
    return ax->a_is_x ? b * ax->nx + a : a * ax->nx + b;
}

typedef struct {
    double *c0, *c1, *r;       /* [np] per point, indexed like the plane */
    double *X, *X2, *A;        /* [nb][nb] */
    double *v, *v2, *x;        /* [nb] */
} orc_face_work;

static void face_work_free(orc_face_work *w)
{
    free(w->c0); free(w->c1); free(w->r);
    free(w->X); free(w->X2); free(w->A);
    free(w->v); free(w->v2); free(w->x);
}

static int face_work_alloc(orc_face_work *w, int np, int nbmax)
{
    size_t n2 = (size_t)nbmax * nbmax;
    w->c0 = malloc(np * sizeof(double));
    w->c1 = malloc(np * sizeof(double));
    w->r = malloc(np * sizeof(double));
    w->X = malloc(n2 * sizeof(double));
    w->X2 = malloc(n2 * sizeof(double));
    w->A = malloc(n2 * sizeof(double));
    w->v = malloc(nbmax * sizeof(double));
    w->v2 = malloc(nbmax * sizeof(double));
    w->x = malloc(nbmax * sizeof(double));
    if (!w->c0 || !w->c1 || !w->r || !w->X || !w->X2 || !w->A || !w->v || !w->v2 || !w->x) {
        face_work_free(w);
        return -1;
    }
    return 0;
}

/* one direction, one wavelength: intensity I[npt] of the whole grid; -1 if a plane's system
 * is singular */
static int sc_face_one(const orc_reg *g, const double *mu, const double *al, const double *S,
                       int bc, const double *ibc, double *I, orc_face_work *w)
{
    const int nx = g->nx, ny = g->ny, nz = g->nz, np = nx * ny;
    const int up = mu[2] > 0.0;
    const int k0 = up ? 0 : nz - 1;
    for (int p = 0; p < np; ++p) {
        double v;
        if (bc == 2) v = ibc[p];
        else if (bc == 0 && up) v = S[k0 * np + p];
        else v = 0.0;
        I[k0 * np + p] = v;
    }
    const double tx = mu[0] != 0.0 ? g->dx / fabs(mu[0]) : INFINITY;
    const double ty = mu[1] != 0.0 ? g->dy / fabs(mu[1]) : INFINITY;
    const int sx = mu[0] >= 0.0 ? 1 : -1, sy = mu[1] >= 0.0 ? 1 : -1;
    for (int s = 1; s < nz; ++s) {
        const int k = up ? s : nz - 1 - s;
        const int ku = up ? k - 1 : k + 1;
        const double dz = fabs(g->z[k] - g->z[ku]);
        const double tz = dz / fabs(mu[2]);
        double *Ik = I + (size_t)k * np;
        const double *Iu = I + (size_t)ku * np;
        const double *Sk = S + (size_t)k * np, *Su = S + (size_t)ku * np;
        const double *Ak = al + (size_t)k * np, *Au = al + (size_t)ku * np;
        if (tz <= tx && tz <= ty) {
            /* plane face: the four corners around the upwind point in plane ku */
            const double t = tz;
            const double fx = t * fabs(mu[0]) / g->dx, fy = t * fabs(mu[1]) / g->dy;
            for (int j = 0; j < ny; ++j)
                for (int i = 0; i < nx; ++i) {
                    const int i1 = wrap(i - sx, nx), j1 = wrap(j - sy, ny);
                    const int c[4] = {j * nx + i, j * nx + i1, j1 * nx + i, j1 * nx + i1};
                    const double wt[4] = {(1.0 - fx) * (1.0 - fy), fx * (1.0 - fy),
                                          (1.0 - fx) * fy, fx * fy};
                    double iu = 0.0, su = 0.0, au = 0.0;
                    for (int q = 0; q < 4; ++q) {
                        iu += wt[q] * Iu[c[q]];
                        su += wt[q] * Su[c[q]];
                        au += wt[q] * Au[c[q]];
                    }
                    const int p = j * nx + i;
                    double ex, w0, w1;
                    orc_linear_weights(0.5 * (au + Ak[p]) * t, &ex, &w0, &w1);
                    Ik[p] = iu * ex + w0 * su + w1 * Sk[p];
                }
            continue;
        }
        /* vertical face, normal to axis a */
        const orc_axes ax = {tx < ty, nx};
        const int na = ax.a_is_x ? nx : ny, nb = ax.a_is_x ? ny : nx;
        const int sa = ax.a_is_x ? sx : sy, sb = ax.a_is_x ? sy : sx;
        const double t = ax.a_is_x ? tx : ty;
        const double fb = t * (ax.a_is_x ? fabs(mu[1]) / g->dy : fabs(mu[0]) / g->dx);
        const double fz = t * fabs(mu[2]) / dz;
        const double wk0 = (1.0 - fz) * (1.0 - fb), wk1 = (1.0 - fz) * fb;   /* plane k */
        const double wu0 = fz * (1.0 - fb), wu1 = fz * fb;                   /* plane ku */
        for (int a = 0; a < na; ++a)
            for (int b = 0; b < nb; ++b) {
                const int a1 = wrap(a - sa, na), b1 = wrap(b - sb, nb);
                const int p = plane_index(&ax, a, b);
                const int q0 = plane_index(&ax, a1, b), q1 = plane_index(&ax, a1, b1);
                const double su = wk0 * Sk[q0] + wk1 * Sk[q1] + wu0 * Su[q0] + wu1 * Su[q1];
                const double au = wk0 * Ak[q0] + wk1 * Ak[q1] + wu0 * Au[q0] + wu1 * Au[q1];
                double ex, w0, w1;
                orc_linear_weights(0.5 * (au + Ak[p]) * t, &ex, &w0, &w1);
                w->c0[p] = ex * wk0;
                w->c1[p] = ex * wk1;
                w->r[p] = ex * (wu0 * Iu[q0] + wu1 * Iu[q1]) + w0 * su + w1 * Sk[p];
            }
        /* x_m = X_m y + v_m with y the unknown last line; X_{-1} = 1, v_{-1} = 0 */
        for (int r = 0; r < nb; ++r) {
            for (int c = 0; c < nb; ++c) w->X[(size_t)r * nb + c] = r == c ? 1.0 : 0.0;
            w->v[r] = 0.0;
        }
        for (int m = 0; m < na; ++m) {
            const int a = sa > 0 ? m : na - 1 - m;
            for (int b = 0; b < nb; ++b) {
                const int b1 = wrap(b - sb, nb), p = plane_index(&ax, a, b);
                for (int c = 0; c < nb; ++c)
                    w->X2[(size_t)b * nb + c] = w->c0[p] * w->X[(size_t)b * nb + c] +
                                                w->c1[p] * w->X[(size_t)b1 * nb + c];
                w->v2[b] = w->c0[p] * w->v[b] + w->c1[p] * w->v[b1] + w->r[p];
            }
            double *t1 = w->X; w->X = w->X2; w->X2 = t1;
            double *t2 = w->v; w->v = w->v2; w->v2 = t2;
        }
        for (int r = 0; r < nb; ++r) {
            for (int c = 0; c < nb; ++c)
                w->A[(size_t)r * nb + c] = (r == c ? 1.0 : 0.0) - w->X[(size_t)r * nb + c];
            w->x[r] = w->v[r];
        }
        if (gauss_solve(nb, w->A, w->x)) return -1;
        /* the pass along a from the closed cycle: w->x holds the line before a_0 */
        for (int m = 0; m < na; ++m) {
            const int a = sa > 0 ? m : na - 1 - m;
            for (int b = 0; b < nb; ++b) {
                const int b1 = wrap(b - sb, nb), p = plane_index(&ax, a, b);
                w->v2[b] = w->c0[p] * w->x[b] + w->c1[p] * w->x[b1] + w->r[p];
                Ik[p] = w->v2[b];
            }
            double *t2 = w->x; w->x = w->v2; w->v2 = t2;
        }
    }
    return 0;
}

/* J[nlam][npt] = sum_d w_d I_d; optional I_out[ndir][nlam][npt].  Periodic in x and y.
 * Returns -1 on an allocation failure or a singular plane system. */
int orc_sc_regular_face(int nx, int ny, int nz, double dx, double dy, const double *z, int ndir,
                        const double *dirs, const double *wdir, int nlam, const double *alpha,
                        const double *S, int bc, const double *ibc, double *J, double *I_out)
{
    orc_reg g = {nx, ny, nz, dx, dy, z, 1};
    const size_t npt = (size_t)nx * ny * nz, nb = (size_t)nx * ny;
    const int nbmax = nx > ny ? nx : ny;
    int failed = 0;
    memset(J, 0, sizeof(double) * npt * nlam);
    for (int d = 0; d < ndir; ++d) {
#pragma omp parallel for schedule(dynamic) reduction(| : failed)
        for (int l = 0; l < nlam; ++l) {
            orc_face_work w;
            double *I = (double *)malloc(npt * sizeof(double));
            if (!I || face_work_alloc(&w, nx * ny, nbmax)) {
                free(I);
                failed = 1;
                continue;
            }
            if (sc_face_one(&g, dirs + 3 * d, alpha + l * npt, S + l * npt, bc,
                            ibc ? ibc + ((size_t)d * nlam + l) * nb : NULL, I, &w))
                failed = 1;
            for (size_t p = 0; p < npt; ++p) J[l * npt + p] += wdir[d] * I[p];
            if (I_out) memcpy(I_out + ((size_t)d * nlam + l) * npt, I, npt * sizeof(double));
            face_work_free(&w);
            free(I);
        }
    }
    return failed ? -1 : 0;
}

/* ---------------------------------------------------------------------------------------
 * Voronoi grid (Sect. 2.5, Eq. 5 and the weight formula after it).
 * Upwind candidates of site i for direction u: Delaunay neighbours k whose line toward i makes
 * v = u . e(k->i) > 0 and that lie on the upwind side in height, (z_i - z_k) sign(mu_z) > 0.
 * The two with the largest v are kept (ties to the smaller neighbour code, then image shift);
 * w_k = v_k^r / (v_1^r + v_2^r).  A mirror ghost beyond a wall stands for the wall: the
 * virtual upwind node sits where the line crosses the wall, carries the site's own alpha and S
 * and the wall's inflow intensity.  A site with no candidate takes the neighbour on the upwind
 * side in height that is most nearly vertical (weight 1).
 * Output tables per (dir, site): k[2] (site index, -1 bottom wall, -2 top wall), w[2], len[2].
 * ------------------------------------------------------------------------------------- */
static void nbr_pos(const double *xyz, int64_t code, int8_t shift, const double box[6],
                    double out[3], int *wall, int64_t *site)
{
    int sx = shift / 3 - 1, sy = shift % 3 - 1;
    double Lx = box[1] - box[0], Ly = box[3] - box[2];
    int64_t k;
    if (code >= 0) { k = code; *wall = 0; }
    else if (((-code - 1) & 1) == 0) { k = (-code - 1) / 2; *wall = 1; }
    else { k = (-code - 2) / 2; *wall = 2; }
    *site = k;
    out[0] = xyz[3 * k] + sx * Lx;
    out[1] = xyz[3 * k + 1] + sy * Ly;
    out[2] = xyz[3 * k + 2];
    if (*wall == 1) out[2] = 2.0 * box[4] - out[2];
    if (*wall == 2) out[2] = 2.0 * box[5] - out[2];
}

int orc_voronoi_tables(int64_t n, const double *xyz, const int64_t *off, const int32_t *code,
                       const int8_t *shift, const double *box, int ndir, const double *dirs,
                       double r_exp, int32_t *k_out, double *w_out, double *len_out,
                       int32_t *level_out, int64_t *n_fallback)
{
    int64_t nfb = 0;
    for (int d = 0; d < ndir; ++d) {
        const double *u = dirs + 3 * d;
        double sgn = u[2] > 0 ? 1.0 : -1.0;
#pragma omp parallel for schedule(static) reduction(+ : nfb)
        for (int64_t i = 0; i < n; ++i) {
            const double *xi = xyz + 3 * i;
            int nc = 0;
            double bv[2] = {-1.0, -1.0}, bl[2] = {0, 0};
            int64_t bk[2] = {0, 0}, bc_[2] = {0, 0};
            int bs[2] = {0, 0};
            double fb_score = -1.0, fb_len = 0.0;
            int64_t fb_k = 0;
            for (int64_t e = off[i]; e < off[i + 1]; ++e) {
                double p[3];
                int wall;
                int64_t site;
                nbr_pos(xyz, code[e], shift[e], box, p, &wall, &site);
                double dv[3] = {xi[0] - p[0], xi[1] - p[1], xi[2] - p[2]};
                double len = sqrt(dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2]);
                if ((xi[2] - p[2]) * sgn <= 0.0) continue;      /* not upwind in height */
                double v = (u[0] * dv[0] + u[1] * dv[1] + u[2] * dv[2]) / len;
                /* geometric length to the wall crossing for a ghost */
                double seg = len;
                int64_t kk = site;
                if (wall == 1) { seg = len * (xi[2] - box[4]) / (xi[2] - p[2]); kk = -1; }
                if (wall == 2) { seg = len * (xi[2] - box[5]) / (xi[2] - p[2]); kk = -2; }
                double vs = (xi[2] - p[2]) * sgn / len;
                if (vs > fb_score) { fb_score = vs; fb_k = kk; fb_len = seg; }
                if (v <= 0.0) continue;
                /* rank by v desc, then code asc, then shift asc */
                int better0 = v > bv[0] || (v == bv[0] && (code[e] < bc_[0] ||
                              (code[e] == bc_[0] && shift[e] < bs[0])));
                int better1 = v > bv[1] || (v == bv[1] && (code[e] < bc_[1] ||
                              (code[e] == bc_[1] && shift[e] < bs[1])));
                if (nc == 0 || better0) {
                    bv[1] = bv[0]; bk[1] = bk[0]; bl[1] = bl[0]; bc_[1] = bc_[0]; bs[1] = bs[0];
                    bv[0] = v; bk[0] = kk; bl[0] = seg; bc_[0] = code[e]; bs[0] = shift[e];
                } else if (nc == 1 || better1) {
                    bv[1] = v; bk[1] = kk; bl[1] = seg; bc_[1] = code[e]; bs[1] = shift[e];
                }
                nc++;
            }
            size_t o = (size_t)d * n + i;
            if (nc >= 2) {
                double a = pow(bv[0], r_exp), b = pow(bv[1], r_exp);
                k_out[2 * o] = (int32_t)bk[0]; k_out[2 * o + 1] = (int32_t)bk[1];
                w_out[2 * o] = a / (a + b); w_out[2 * o + 1] = b / (a + b);
                len_out[2 * o] = bl[0]; len_out[2 * o + 1] = bl[1];
            } else if (nc == 1) {
                k_out[2 * o] = k_out[2 * o + 1] = (int32_t)bk[0];
                w_out[2 * o] = 1.0; w_out[2 * o + 1] = 0.0;
                len_out[2 * o] = len_out[2 * o + 1] = bl[0];
            } else {
                nfb++;
                if (fb_score < 0.0) {          /* nothing upwind in height: the wall itself */
                    fb_k = sgn > 0 ? -1 : -2;
                    fb_len = (sgn > 0 ? xi[2] - box[4] : box[5] - xi[2]) / fabs(u[2]);
                }
                k_out[2 * o] = k_out[2 * o + 1] = (int32_t)fb_k;
                w_out[2 * o] = 1.0; w_out[2 * o + 1] = 0.0;
                len_out[2 * o] = len_out[2 * o + 1] = fb_len;
            }
        }
        /* dependency levels: visit sites in upwind height order (a topological order because
           every upwind link goes strictly upwind in height) */
        int64_t *ord = (int64_t *)malloc(n * sizeof(int64_t));
        double *key = (double *)malloc(n * sizeof(double));
        if (!ord || !key) { free(ord); free(key); return -1; }
        for (int64_t i = 0; i < n; ++i) { ord[i] = i; key[i] = xyz[3 * i + 2] * sgn; }
        /* simple heap sort by key (keeps the oracle free of external helpers) */
        for (int64_t s = n / 2 - 1; s >= 0; --s) {
            int64_t r = s;
            for (;;) {
                int64_t c = 2 * r + 1;
                if (c >= n) break;
                if (c + 1 < n && key[ord[c + 1]] > key[ord[c]]) c++;
                if (key[ord[c]] <= key[ord[r]]) break;
                int64_t t = ord[c]; ord[c] = ord[r]; ord[r] = t; r = c;
            }
        }
        for (int64_t e = n - 1; e > 0; --e) {
            int64_t t = ord[0]; ord[0] = ord[e]; ord[e] = t;
            int64_t r = 0;
            for (;;) {
                int64_t c = 2 * r + 1;
                if (c >= e) break;
                if (c + 1 < e && key[ord[c + 1]] > key[ord[c]]) c++;
                if (key[ord[c]] <= key[ord[r]]) break;
                int64_t t2 = ord[c]; ord[c] = ord[r]; ord[r] = t2; r = c;
            }
        }
        int32_t *lv = level_out + (size_t)d * n;
        for (int64_t q = 0; q < n; ++q) {
            int64_t i = ord[q];
            size_t o = (size_t)d * n + i;
            int L = 0;
            for (int c = 0; c < 2; ++c) {
                int32_t k = k_out[2 * o + c];
                if (k >= 0 && lv[k] + 1 > L) L = lv[k] + 1;
            }
            lv[i] = L;
        }
        free(ord);
        free(key);
    }
    if (n_fallback) *n_fallback = nfb;
    return 0;
}

/* I for one direction, all wavelengths, sites visited level by level (order = level CSR) */
static void vor_one(int64_t n, int nlam, const int32_t *k, const double *w, const double *len,
                    const int64_t *order, const double *alpha, const double *S, int bc, int up,
                    const double *ibc, double *I)
{
    for (int64_t q = 0; q < n; ++q) {
        int64_t i = order[q];
        for (int l = 0; l < nlam; ++l) {
            const double *al = alpha + (size_t)l * n, *Sl = S + (size_t)l * n;
            double acc = 0.0;
            for (int c = 0; c < 2; ++c) {
                double wk = w[2 * i + c];
                if (wk == 0.0) continue;
                int32_t kk = k[2 * i + c];
                double Ik, Sk, ak;
                if (kk >= 0) {
                    Ik = I[(size_t)l * n + kk]; Sk = Sl[kk]; ak = al[kk];
                } else {
                    Sk = Sl[i]; ak = al[i];
                    if (bc == 2) Ik = ibc[(size_t)l * n + i];
                    else if (bc == 0 && up && kk == -1) Ik = Sl[i];
                    else Ik = 0.0;
                }
                double d = 0.5 * (ak + al[i]) * len[2 * i + c], ex, w0, w1;
                orc_linear_weights(d, &ex, &w0, &w1);
                acc += wk * (Ik * ex + w0 * Sk + w1 * Sl[i]);
            }
            I[(size_t)l * n + i] = acc;
        }
    }
}

/* order[ndir][n]: sites of each direction in a valid upwind order (e.g. by level) */
int orc_voronoi_fs(int64_t n, int ndir, const double *dirs, const double *wdir, const int32_t *k,
                   const double *w, const double *len, const int64_t *order, int nlam,
                   const double *alpha, const double *S, int bc, const double *ibc, double *J,
                   double *I_out)
{
    size_t nn = (size_t)n * nlam;
    double *I = (double *)malloc(nn * sizeof(double));
    if (!I) return -1;
    memset(J, 0, nn * sizeof(double));
    for (int d = 0; d < ndir; ++d) {
        size_t o = (size_t)d * n;
        vor_one(n, nlam, k + 2 * o, w + 2 * o, len + 2 * o, order + o, alpha, S, bc,
                dirs[3 * d + 2] > 0.0, ibc ? ibc + (size_t)d * nn : NULL, I);
        for (size_t p = 0; p < nn; ++p) J[p] += wdir[d] * I[p];
        if (I_out) memcpy(I_out + (size_t)d * nn, I, nn * sizeof(double));
    }
    free(I);
    return 0;
}

/* Adjoint of vor_one for one direction: sites visited in reverse upwind order. */
int orc_voronoi_adjoint(int64_t n, const int32_t *k, const double *w, const double *len,
                        const int64_t *order, int up, int nlam, const double *alpha,
                        const double *S, int bc, const double *gI, double *g_alpha, double *g_S)
{
    size_t nn = (size_t)n * nlam;
    double *I = (double *)malloc(nn * sizeof(double));
    double *gi = (double *)malloc(nn * sizeof(double));
    if (!I || !gi) { free(I); free(gi); return -1; }
    vor_one(n, nlam, k, w, len, order, alpha, S, bc, up, NULL, I);
    memcpy(gi, gI, nn * sizeof(double));
    for (int64_t q = n - 1; q >= 0; --q) {
        int64_t i = order[q];
        for (int l = 0; l < nlam; ++l) {
            const double *al = alpha + (size_t)l * n, *Sl = S + (size_t)l * n;
            double *ga = g_alpha + (size_t)l * n, *gs = g_S + (size_t)l * n;
            double gb = gi[(size_t)l * n + i];
            for (int c = 0; c < 2; ++c) {
                double wk = w[2 * i + c];
                if (wk == 0.0) continue;
                int32_t kk = k[2 * i + c];
                double Ik, Sk, ak;
                if (kk >= 0) {
                    Ik = I[(size_t)l * n + kk]; Sk = Sl[kk]; ak = al[kk];
                } else {
                    Sk = Sl[i]; ak = al[i];
                    Ik = (bc == 0 && up && kk == -1) ? Sl[i] : 0.0;
                }
                double ds = len[2 * i + c];
                double d = 0.5 * (ak + al[i]) * ds, ex, w0, w1, dex, dw0, dw1;
                orc_linear_weights(d, &ex, &w0, &w1);
                orc_linear_weights_deriv(d, &dex, &dw0, &dw1);
                double g = wk * gb;
                double gd = g * (Ik * dex + Sk * dw0 + Sl[i] * dw1);
                gs[i] += w1 * g;
                ga[i] += 0.5 * ds * gd;
                if (kk >= 0) {
                    gi[(size_t)l * n + kk] += ex * g;
                    gs[kk] += w0 * g;
                    ga[kk] += 0.5 * ds * gd;
                } else {
                    gs[i] += w0 * g;
                    ga[i] += 0.5 * ds * gd;
                    if (bc == 0 && up && kk == -1) gs[i] += ex * g;
                }
            }
        }
    }
    free(I);
    free(gi);
    return 0;
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
