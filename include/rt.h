/*
 * rt.h -- C ABI of the GB300 formal-solution library (librt.so).
 *
 * The library solves the 3D radiative-transfer formal solution of Udnaes & Pereira (2023,
 * arXiv:2306.01041) on two kinds of grid:
 *   - a regular Cartesian grid, by plane-to-plane short characteristics (Sect. 2.6, after
 *     Kunasz & Auer 1988), swept plane by plane;
 *   - an irregular (Voronoi) grid, by transport along Delaunay lines from the two upwind
 *     neighbours that best match each ray (Sect. 2.5, Eq. 5 and the weight formula after it),
 *     swept in per-direction dependency levels;
 * integrating the source function linearly across each optical-depth interval (Sect. 2.5,
 * Eq. 2), accumulating J over angles (Sect. 2.1, Eq. 4), and closing each Lambda iteration with
 * statistical equilibrium of a 2 + 1 level hydrogen-like atom (Sect. 2.2, Table 1).
 *
 * Conventions for every call
 *   - Field arrays are device pointers owned by the caller, FP32, layout [nlam][npt], with
 *     npt = nx*ny*nz (x fastest, then y, then z) on a regular grid or the site index on a
 *     Voronoi grid.  They must be 16-byte aligned, else RT_EINVAL.
 *   - The library owns the grid tables and the scratch it allocates for a grid.
 *   - Calls are asynchronous on the given CUDA stream (NULL = legacy default stream), except
 *     rt_grid_create, rt_lambda_iterate and rt_lambda_iterate_ali, which synchronise on their
 *     stream.
 *   - No call aborts.  Errors come back as rt_status; rt_last_error() returns a message for the
 *     calling host thread.  Device-side failures (a non-finite value, an exhausted wait) are
 *     recorded in a device error word and surfaced by the next synchronising call.
 *   - Directions: ndir unit vectors (mu_x, mu_y, mu_z), none with mu_z = 0, with weights wdir
 *     summing to 1; J = sum_d wdir[d] I_d (Sect. 2.5, fixed-angle quadrature).
 *   - Boundary conditions (the paper leaves them open; see rt_bc):
 *       RT_BC_THERMAL: rays entering through the bottom wall carry I = S there; through the top
 *                      wall, I = 0.
 *       RT_BC_ZERO:    I = 0 on both walls.
 *       RT_BC_ARRAY:   the caller supplies the entering intensity I_bc[ndir][nlam][nb] on the
 *                      wall each direction enters through (nb = nx*ny on a regular grid, in
 *                      x-fastest order; nb = nsites on a Voronoi grid, the value taken by a site
 *                      whose upwind line starts at the wall).
 */
#ifndef RT_H
#define RT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rt_grid *rt_grid_t;

typedef enum {
    RT_OK = 0,
    RT_EINVAL = 1,     /* bad argument, size or alignment */
    RT_ENOMEM = 2,     /* device or host allocation failed */
    RT_ECUDA = 3,      /* a CUDA call failed */
    RT_ECYCLE = 4,     /* Voronoi upwind links do not form a DAG */
    RT_ETIMEOUT = 5,   /* a bounded device wait gave up */
    RT_ENAN = 6,       /* a non-finite value was produced */
    RT_ECAPACITY = 7,  /* a persistent launch cannot be co-resident */
    RT_ENOCONV = 8     /* max_iter reached before the tolerance */
} rt_status;

enum rt_grid_kind { RT_GRID_REGULAR = 0, RT_GRID_VORONOI = 1 };
enum rt_bc { RT_BC_THERMAL = 0, RT_BC_ZERO = 1, RT_BC_ARRAY = 2 };

/* Grid description; every pointer is host memory, copied by rt_grid_create. */
typedef struct {
    int kind;                 /* RT_GRID_REGULAR or RT_GRID_VORONOI */
    /* regular grid: uniform dx, dy; z[nz] strictly ascending (may be non-uniform) */
    int nx, ny, nz;
    double dx, dy;
    const double *z;
    /* Voronoi grid: sites and their Delaunay neighbours in CSR form.  nbr_idx[e] >= 0 is a
     * site; -1-2k is the mirror image of site k in the bottom wall (z = box[4]) and -2-2k its
     * mirror in the top wall (z = box[5]).  nbr_shift[e] = (sx+1)*3 + (sy+1) selects the
     * periodic image (sx, sy in {-1,0,1}) of that neighbour; NULL means (0, 0) for all. */
    int64_t nsites;
    const double *xyz;        /* [nsites][3] */
    const int64_t *nbr_off;   /* [nsites+1] */
    const int32_t *nbr_idx;   /* [nbr_off[nsites]] */
    const int8_t *nbr_shift;  /* [nbr_off[nsites]] or NULL */
    double box[6];            /* x0, x1, y0, y1, z0, z1 */
    int periodic_xy;          /* 1: periodic in x and y; 0: closed sides with zero inflow */
    int ndir;                 /* number of quadrature directions, 1..64 */
    const double *dirs;       /* [ndir][3] unit vectors */
    const double *wdir;       /* [ndir] weights */
    double r_exponent;        /* exponent r of the two-line weights (Sect. 2.5; paper: 7) */
} rt_grid_desc;

/* Builds a grid: validates the description, precomputes the regular-grid upwind stencils or the
 * Voronoi upwind tables (two best-aligned upwind neighbours per site and direction, weights
 * v^r / sum v^r, Delaunay segment lengths) and per-direction dependency levels, and uploads
 * them.  Returns RT_ECYCLE if the Voronoi upwind links are not acyclic.  Synchronous. */
rt_status rt_grid_create(const rt_grid_desc *desc, void *stream, rt_grid_t *out);
void rt_grid_destroy(rt_grid_t grid);

/* Host-side facts about a built grid.  Any output pointer may be NULL.
 * npt: points/sites; ntop: points on the emergent layer (nx*ny, or the Voronoi sites whose
 * neighbour list holds a top-wall mirror); max_levels: the largest number of dependency levels
 * over the directions (nz on a regular grid); n_fallback: Voronoi (site, direction) pairs that
 * had no upwind neighbour with v > 0 and took the most nearly vertical upwind neighbour. */
rt_status rt_grid_info(rt_grid_t grid, int64_t *npt, int64_t *ntop, int *max_levels,
                       int64_t *n_fallback);

/* Copies the (site, direction) upwind tables to host arrays for inspection:
 * k[ndir][nsites][2] (site, -1 bottom wall, -2 top wall), w[ndir][nsites][2],
 * len[ndir][nsites][2] (metres), level[ndir][nsites].  Voronoi grids only.  Synchronous. */
rt_status rt_grid_tables(rt_grid_t grid, int32_t *k, float *w, float *len, int32_t *level);

/* Rebuilds a Voronoi grid's upwind tables and dependency levels on the GPU: the definition of
 * rt_grid_create's host build (two best-aligned upwind neighbours, weights v^r / sum v^r,
 * segment lengths, levels), every geometric step one IEEE double operation in the same order, so
 * the choices are the host build's; the levels come from relaxation passes over the links.  The
 * new tables replace the grid's in place (same device arrays, so batches made from the grid stay
 * valid); rt_grid_tables and rt_grid_info then report them.  Synchronous; allocates and frees a
 * device buffer the size of the neighbour lists and the tables.  RT_EINVAL for a regular grid. */
rt_status rt_grid_build_tables_device(rt_grid_t grid, void *stream);

/* Emergent-layer point indices (host array of ntop entries). */
rt_status rt_grid_top_points(rt_grid_t grid, int64_t *idx);

/* Short-characteristics scheme of a regular grid (Sect. 2.6 cites Kunasz & Auer 1988 for it):
 *   RT_SC_PLANE (default): plane to plane -- the upwind point of a point of plane k is where the
 *     ray crosses the previous plane of the sweep, however far from the point's column;
 *   RT_SC_FACE: face hitting -- the upwind point is on the first face of the cell the ray enters:
 *     the previous plane when dz/|mu_z| <= dx/|mu_x| and dy/|mu_y|, else the vertical face x_i -
 *     sx dx (when dx/|mu_x| < dy/|mu_y|) or y_j - sy dy, where I, S, alpha are bilinear between the
 *     face's two grid lines and the planes k and k -/+ 1.  The intensities of a plane then depend on
 *     one another around the periodic box; that cycle is closed to a relative 1e-9 of the plane's
 *     intensities.
 * The scheme applies to rt_formal_solution and so to the Lambda iterations; rt_lambda_star,
 * rt_emergent_intensity and the adjoint stay plane to plane.  RT_SC_FACE needs periodic sides and
 * nx, ny <= 256; its tables (per direction and plane) are built on first selection (synchronous).
 * Its formal solution keeps every plane of every (wavelength, direction) in the grid's scratch
 * (nlam * ndir * npt floats) and forms J from them afterwards when that fits a quarter of the
 * device's memory (the environment variable RT_FACE_VOLUME_MB sets another limit), else it sums J
 * after every plane step; both give J to FP32 rounding of the same sum.
 * RT_EINVAL for a Voronoi grid, closed sides, larger planes, or planes so far apart that the
 * cycle would need more than 16 laps of the box to close. */
enum rt_sc_scheme { RT_SC_PLANE = 0, RT_SC_FACE = 1 };
rt_status rt_grid_set_scheme(rt_grid_t grid, int scheme);

/* Formal solution (Eq. 2 along every ray of the quadrature) and J = sum_d w_d I_d (Eq. 4).
 * alpha, S: [nlam][npt] device; J: [nlam][npt] device, overwritten.
 * I_bc: device [ndir][nlam][nb] when bc == RT_BC_ARRAY, else ignored.
 * I_dir: optional device [ndir][nlam][npt] receiving every directional intensity, or NULL. */
rt_status rt_formal_solution(rt_grid_t grid, int nlam, const float *alpha, const float *S,
                             int bc, const float *I_bc, float *J, float *I_dir, void *stream);

/* ---- atom, source terms and the Lambda iteration (Sect. 2.1-2.2) --------------------------- */
/* Model atom: levels 1, 2 and the continuum p (Table 1), line 1-2 with oscillator strength f,
 * bound-free from 1 and from 2 (Kramers cross sections), a Voigt line profile with damping a
 * and the Doppler width of the hydrogen mass, collisions C21 = q n_e T^-1/2 and
 * C_ip = q n_e T^-1/2 exp(-E_ip/kT) (their inverses by detailed balance), and a grey background
 * alpha_bg = kappa0 rho (T/5000)^9 with source function B.  Wavelength nodes lam[nlam] (m) with
 * quadrature weights wlam[nlam] (m); kind[j] = 0 for a line node, 1 for the bound-free node of
 * level 1, 2 for that of level 2 (each node feeds the rate integral of its kind).
 * The atom's derived constants are held in constant memory, one copy per device, and uploaded
 * (synchronously) by a call whose atom differs from the previous call's on that device: calls
 * with different atoms must not overlap on the GPU. */
typedef struct {
    double E_cm[3];           /* level energies, cm^-1 (the third is the continuum edge) */
    double g[3];              /* statistical weights */
    double f_line;
    double voigt_a;
    double q_coll;            /* m^3 s^-1 K^1/2 */
    double kappa0;            /* m^2 kg^-1 */
    int nlam;
    const double *lam;        /* host [nlam] */
    const double *wlam;       /* host [nlam] */
    const int32_t *kind;      /* host [nlam] */
} rt_atom;

/* Atmosphere on the grid's points: device FP32 arrays [npt]. */
typedef struct {
    const float *T, *rho, *ne, *nH;
} rt_atmos;

/* LTE continuum of the synthetic atmospheres: alpha = kappa0 rho (T/5000)^9, S = B_lam(T) in
 * W m^-2 m^-1 sr^-1, at one wavelength lam (m).  alpha, S: device [npt]. */
rt_status rt_source_terms_lte(int64_t npt, const float *T, const float *rho, double kappa0,
                              double lam, float *alpha, float *S, void *stream);

/* alpha, S [nlam][npt] of the atom from the populations pops [3][npt] (n1, n2, n_p). */
rt_status rt_source_terms(rt_grid_t grid, const rt_atom *atom, const rt_atmos *atm,
                          const float *pops, float *alpha, float *S, void *stream);

/* Saha-Boltzmann (LTE) populations pops [3][npt], the starting point of the iteration. */
rt_status rt_lte_populations(rt_grid_t grid, const rt_atom *atom, const rt_atmos *atm,
                             float *pops, void *stream);

/* Radiative + collisional rates from J [nlam][npt] and the statistical-equilibrium solution:
 * pops [3][npt] is read (old) and overwritten (new); *dmax_dev (device float, may be NULL)
 * receives max over points and levels of |n_new - n_old| / n_new. */
rt_status rt_statistical_equilibrium(rt_grid_t grid, const rt_atom *atom, const rt_atmos *atm,
                                     const float *J, float *pops, float *dmax_dev, void *stream);

/* Lambda iteration (Sect. 2.1, Eq. 3-4): pops [3][npt] device, in = start (e.g. LTE),
 * out = last iterate.  Iterates source terms -> formal solution (RT_BC_THERMAL) -> rates ->
 * statistical equilibrium until max |dn/n| < tol or max_iter iterations (RT_ENOCONV then).
 * iters_out (host, may be NULL); history (host [max_iter], may be NULL) gets max |dn/n| per
 * iteration.  use_graph != 0 captures one iteration in a CUDA graph and replays it.
 * Synchronises once per iteration to read the convergence scalar. */
rt_status rt_lambda_iterate(rt_grid_t grid, const rt_atom *atom, const rt_atmos *atm,
                            float *pops, int max_iter, double tol, int *iters_out,
                            float *history, int use_graph, void *stream);

/* ---- accelerated Lambda iteration ------------------------------------------------------------
 * The paper iterates plain Lambda (Sect. 2.1) and notes that accelerated schemes need far fewer
 * iterations.  Here each point's own contribution to its J is treated implicitly: with
 * Lambda*_p = dJ_p/dS_p (opacities fixed), the new populations solve
 *     n = SE( J + Lambda* (S(n) - S_old) )
 * at every point.  At a converged state S(n) = S_old, so the fixed point is the Lambda
 * iteration's; only the number of iterations changes. */

/* Lambda* [nlam][npt] (device, overwritten) of the opacities alpha [nlam][npt]: the sum over
 * directions of w_d times the weight with which S at a point enters its own intensity (w1 of
 * the interval ending there, Eq. 2; 1 where a ray starts at the point under RT_BC_THERMAL; on a
 * Voronoi grid, w0 + w1 (+ e^-d under thermal inflow) for a wall neighbour, which stands in with
 * the site's own S).  bc: RT_BC_THERMAL, RT_BC_ZERO, or RT_BC_ARRAY (inflow independent of S,
 * as ZERO).  The first call on a Voronoi grid uploads site-ordered tables (allocates). */
rt_status rt_lambda_star(rt_grid_t grid, int nlam, const float *alpha, int bc, float *Lstar,
                         void *stream);

/* One accelerated statistical-equilibrium update: J, Lstar and S_old [nlam][npt] (S_old the
 * source function of the current populations, from which J was computed); pops [3][npt] read
 * (current) and overwritten (new); *dmax_dev (device, may be NULL) as for
 * rt_statistical_equilibrium.  The local equation is solved by `newton` (0..16) Newton steps on
 * the logarithms of the two smaller populations (forward-difference Jacobian); 0 gives the plain
 * update. */
rt_status rt_statistical_equilibrium_ali(rt_grid_t grid, const rt_atom *atom,
                                         const rt_atmos *atm, const float *J, const float *Lstar,
                                         const float *S_old, float *pops, float *dmax_dev,
                                         int newton, void *stream);

/* Accelerated Lambda iteration: as rt_lambda_iterate, with the update of
 * rt_statistical_equilibrium_ali (newton steps, 0..16; 1 suffices after the first iterations).
 * fixed_lstar != 0: Lambda* from the opacities of the starting populations, held fixed (the
 * fixed point does not depend on Lambda*, only the rate of convergence does); 0: recomputed from
 * every iteration's opacities.  Takes at most 64 wavelengths. */
rt_status rt_lambda_iterate_ali(rt_grid_t grid, const rt_atom *atom, const rt_atmos *atm,
                                float *pops, int max_iter, double tol, int *iters_out,
                                float *history, int use_graph, int newton, int fixed_lstar,
                                void *stream);

/* ---- Ng acceleration (not in the paper) -------------------------------------------------------
 * A least-squares extrapolation of a fixed-point iteration from its last four iterates x0 (newest)
 * .. x3: with d0 = x0 - x1, d1 = x1 - x2, d2 = x2 - x3, (a, b) minimise the norm of
 * d0 - a (d0 - d1) - b (d0 - d2) weighted by 1/x0^2, and x = (1 - a - b) x0 + a x1 + b x2; exact
 * when the error spans two eigenvectors of the iteration. */

/* x0..x3, out: device float [n]; scratch: 64 bytes of device memory; *ok (host) = 1 if out was
 * written with every entry positive (else out is unspecified: keep x0).  Synchronises on
 * stream. */
rt_status rt_ng_extrapolate(int64_t n, const float *x0, const float *x1, const float *x2,
                            const float *x3, float *out, void *scratch, int *ok, void *stream);

/* The Lambda iteration with every option: newton = -1 plain, 0..16 accelerated (as
 * rt_lambda_iterate_ali, with fixed_lstar); ng_period > 0 applies the Ng extrapolation to the
 * populations after every ng_period-th iteration from the fourth on (kept only if every
 * population stays positive); 0 never.  Other arguments as rt_lambda_iterate. */
rt_status rt_lambda_iterate_ex(rt_grid_t grid, const rt_atom *atom, const rt_atmos *atm,
                               float *pops, int max_iter, double tol, int *iters_out,
                               float *history, int use_graph, int newton, int fixed_lstar,
                               int ng_period, void *stream);

/* ---- final synthesis on a Voronoi grid (Sect. 2.5, last paragraphs) ---------------------------
 * The paper takes the emergent intensity not from the irregular grid, whose upper layers hold few
 * sites, but from the original mesh: the converged populations are interpolated to the mesh by
 * inverse-distance weighting over the two nearest sites (weights 1/d normalised; (1, 0) on a
 * site), and a formal solution along vertical long characteristics follows (rt_emergent_intensity
 * with dir = (0, 0, 1) on the regular grid, whose rays then run along the mesh columns). */
typedef struct rt_idw *rt_idw_t;

/* Two-nearest table of every point of `mesh` (a regular grid; point (i, j, k) at (i dx, j dy,
 * z_k) in the sites' frame) among the sites of `voronoi`: exact, minimum-image distances in the
 * periodic x and y, ties to the smaller site index.  Built on the host (OpenMP) and uploaded;
 * synchronous.  *out is owned by the caller (rt_idw_destroy). */
rt_status rt_idw_create(rt_grid_t voronoi, rt_grid_t mesh, rt_idw_t *out);
void rt_idw_destroy(rt_idw_t table);

/* The table on the host: k [npt][2] site indices, w [npt][2] weights (caller-owned arrays). */
rt_status rt_idw_table(rt_idw_t table, int32_t *k, float *w);

/* dst [nf][npt_mesh] = w1 src[nf][k1] + w2 src[nf][k2] (device arrays; src [nf][nsites]). */
rt_status rt_idw_interpolate(rt_idw_t table, int nf, const float *src, float *dst, void *stream);

/* ---- emergent intensity and its adjoint (Sect. 2.5-2.6; Eq. 2 differentiated) -------------- */
/* Intensity along one direction dir[3] (mu_z > 0) at the emergent layer:
 * I_top [nlam][ntop] (device).  Regular grid: the top plane.  Voronoi grid: the sites listed by
 * rt_grid_top_points.  bc as for rt_formal_solution (RT_BC_ARRAY not accepted here). */
rt_status rt_emergent_intensity(rt_grid_t grid, const double dir[3], int nlam,
                                const float *alpha, const float *S, int bc, float *I_top,
                                void *stream);

/* Emergent map (Sect. 2.5, last paragraph): the intensity along dir at the emergent layer, on an
 * npx x npy pixel grid, map [nlam][npy][npx] (device, x fastest).  Regular grid: the top plane
 * itself (npx = nx and npy = ny required; pixel (i, j) is grid point (i, j)).  Voronoi grid: the
 * intensities at the sites of rt_grid_top_points, resampled to pixel (i, j) at
 * (x0 + i Lx / npx, y0 + j Ly / npy) by inverse-distance weighting over the two nearest of those
 * sites in (x, y) -- minimum image in the periodic x and y, ties to the smaller site index,
 * weights 1/d normalised, (1, 0) on a site.  The pixel table is built on the host on the first
 * call for an (npx, npy) and kept with the grid (allocates then).  bc as for
 * rt_emergent_intensity. */
rt_status rt_emergent_map(rt_grid_t grid, const double dir[3], int nlam, const float *alpha,
                          const float *S, int bc, int npx, int npy, float *map, void *stream);

/* Gradient of L = sum(gI_top * I_top) with respect to alpha and S at every point, for the
 * emergent intensity above: g_alpha, g_S [nlam][npt] device, overwritten.  The forward
 * intensities are kept only every ckpt_stride planes/levels (>= 1) and recomputed in between;
 * ws is a device workspace of rt_adjoint_workspace_size bytes (16-byte aligned). */
size_t rt_adjoint_workspace_size(rt_grid_t grid, int nlam, int ckpt_stride);
rt_status rt_formal_solution_adjoint(rt_grid_t grid, const double dir[3], int nlam,
                                     const float *alpha, const float *S, int bc,
                                     const float *gI_top, float *g_alpha, float *g_S,
                                     int ckpt_stride, void *ws, size_t ws_bytes, void *stream);

/* Chain rule to temperature: g_T [npt] = sum_lam (g_alpha dalpha/dT + g_S dS/dT) with the
 * populations held fixed (the atom's source terms, derivatives by forward-mode dual numbers). */
rt_status rt_source_terms_adjoint(rt_grid_t grid, const rt_atom *atom, const rt_atmos *atm,
                                  const float *pops, const float *g_alpha, const float *g_S,
                                  float *g_T, void *stream);

/* LTE continuum counterpart: g_T = g_alpha dalpha/dT + g_S dB/dT at one wavelength. */
rt_status rt_source_terms_lte_adjoint(int64_t npt, const float *T, const float *rho,
                                      double kappa0, double lam, const float *g_alpha,
                                      const float *g_S, float *g_T, void *stream);

/* ---- batched persistent sweep over several Voronoi grids ------------------------------------ */
typedef struct rt_batch *rt_batch_t;

/* A batch of Voronoi grids (same ndir) solved by one persistent level-scheduled launch.
 * lam_chunk[b] (host, may be NULL for the built-in chunk of 8) is the wavelength chunk each work
 * item of grid b carries, rounded up to a multiple of 8 (a site's wavelengths are held in a row
 * padded to whole chunks, a chunk filling whole 32-byte sectors) and to at most the block size; threads is the block size (0 = built-in; a multiple of 32 up to 512).  At most 128
 * wavelengths.  Allocates the batch's fields: per grid 2 + ndir floats per (site, wavelength) of
 * the padded rows. */
rt_status rt_batch_create(const rt_grid_t *grids, int ngrids, int nlam, const int *lam_chunk,
                          int threads, rt_batch_t *out);
void rt_batch_destroy(rt_batch_t batch);

/* Formal solution of every grid of the batch: alpha[b], S[b], J[b] are device [nlam][npt_b]. */
rt_status rt_batch_formal_solution(rt_batch_t batch, const float *const *alpha,
                                   const float *const *S, int bc, float *const *J,
                                   void *stream);

/* Lambda iteration (Sect. 2.1, Eq. 3-4) of every atmosphere of the batch together: per iteration
 * the source terms of each atmosphere, one batched formal solution of all of them (RT_BC_THERMAL),
 * and the rates and statistical equilibrium of each, until the largest relative population change
 * over every atmosphere is below tol or max_iter iterations have run (RT_ENOCONV then).  One model
 * atom serves the whole batch (atom->nlam must equal the batch's nlam); atms[b] (host array of
 * ngrids descriptions of device fields) and pops[b] (host array of ngrids device pointers, each
 * [3][npt_b], in = start, out = last iterate) per atmosphere.  iters_out, history as for
 * rt_lambda_iterate.  use_graph != 0 captures one iteration of the whole batch in a CUDA graph and
 * replays it.  Uses each grid's iteration scratch (allocated on first use); synchronises once per
 * iteration to read the convergence scalar. */
rt_status rt_batch_lambda_iterate(rt_batch_t batch, const rt_atom *atom, const rt_atmos *atms,
                                  float *const *pops, int max_iter, double tol, int *iters_out,
                                  float *history, int use_graph, void *stream);

/* ---- site sampling (Sect. 2.4) -------------------------------------------------------------
 * Rejection sampling of Voronoi sites: proposals uniform in the box are kept where the target f is
 * at least a uniform rejection level times max f, until nsites are kept.  Proposal p = 0, 1, 2, ...
 * is the Philox4x64-10 block (Salmon et al. 2011) of counter (p, 0, 0, 0) under key (seed, 0); its
 * words w0..w3 give u_i = (w_i >> 11) 2^-53, the position (x0 + u0 (x1 - x0), y0 + u1 (y1 - y0),
 * z0 + u2 (z1 - z0)) and the level u3.  f is trilinear between the mesh points
 * (x0 + i (x1 - x0)/nx, y0 + j (y1 - y0)/ny, z[k]), periodic in x and y, clamped to
 * [z[0], z[nz-1]] in z, each step lerp(a, b, t) = a + t (b - a) in IEEE double; the proposal is kept
 * iff f(r) >= u3 max f.  The sites are the first nsites kept proposals in proposal order: the same
 * for a seed on any device.  The Delaunay neighbours of the sites (rt_grid_desc) are built
 * elsewhere.
 * f: device float [nz][ny][nx], finite, >= 0, not all zero; z: host [nz] strictly ascending,
 * nz >= 2; box: host [6] (x0, x1, y0, y1, z0, z1); xyz: device double [nsites][3], 8-byte aligned
 * (output); *nproposals (host, may be NULL): the proposals drawn up to the last kept one.
 * Allocates and frees a small device buffer; synchronises on stream once per 2^22 proposals.
 * RT_EINVAL for a bad argument or target; RT_ENOCONV when 1000 nsites + 2^20 proposals have not
 * given nsites sites. */
rt_status rt_sample_sites(int nx, int ny, int nz, const double *z, const double *box,
                          const float *f, int64_t nsites, uint64_t seed, double *xyz,
                          int64_t *nproposals, void *stream);

/* ---- allocation-free variant -------------------------------------------------------------- */
/* No counterpart in the paper.  For callers that cannot allocate device memory (host callbacks
 * and stream-ordered code that must not synchronise the device, plugins whose host application
 * owns every allocation, processes under a fixed device-memory budget): the regular-grid formal
 * solution and J of rt_formal_solution (same per-plane sweep), with the grid described directly
 * by host arrays (as in rt_grid_desc: z[nz], dirs[ndir][3], wdir[ndir]) instead of a grid object,
 * and its upwind-plane scratch taken from a fixed file-scope device array of 4 Mi floats (16 MiB),
 * which every GPU that loads the library holds until the process exits.  It calls no cudaMalloc,
 * cudaFree or allocating library routine.  alpha, S: device [nlam][nx*ny*nz]; J: device output,
 * overwritten; I_bc: device [ndir][nlam][nx*ny] for RT_BC_ARRAY, else NULL.
 * Limits: 2 * nlam * (directions per hemisphere) * nx * ny <= 4194304 floats, at most 32
 * directions per hemisphere; larger problems return RT_EINVAL with a message, before any device
 * work.  Every call looks up the array's device address in the CUDA context current on the
 * calling thread (cudaGetSymbolAddress, which allocates nothing), so it works in the runtime's
 * primary context, in a context the host application created, and after cudaDeviceReset.  The
 * first call in a context may load the library's device code and reserve the 16 MiB array there
 * (with lazy module loading this happens at that call, not when the library is loaded), and can
 * fail with RT_ECUDA under a device-memory budget that has no room left; make that first call
 * before any stream capture.  All calls share the one array, which keeps the last call's contents
 * (nothing in it needs to start at zero): calls that overlap on the GPU -- on different streams,
 * or from different host threads -- race on it and must be serialised by the caller.
 * Asynchronous on `stream`. */
rt_status rt_formal_solution_regular_noalloc(int nx, int ny, int nz, double dx, double dy,
                                             const double *z, int periodic_xy, int ndir,
                                             const double *dirs, const double *wdir, int nlam,
                                             const float *alpha, const float *S, int bc,
                                             const float *I_bc, float *J, void *stream);

const char *rt_last_error(void);

/* Number of kernel launches the library has issued in this process (all devices, all threads),
 * counting launches recorded into a CUDA graph under stream capture once, at capture.  Host-only,
 * never fails.  The paper has no counterpart: this is instrumentation for benchmarks. */
unsigned long long rt_kernel_launches(void);

/* Host-only diagnostic: G(v) = 2 v F(v) - 1 (F = Dawson's integral) from the double-precision
 * series that seeds the device Voigt tables; lets CPU tests check the tables' source. */
double rt_debug_G_host(double v);

#ifdef __cplusplus
}
#endif

#endif /* RT_H */
