// Diagonal of the Lambda operator (Lambda*), for the accelerated Lambda iteration.
//
// Lambda*_p = dJ_p / dS_p at fixed opacities.  With S linear across every interval (Sect. 2.5,
// Eq. 2) the source function of point p reaches the intensity at p only through the weight w1
// of the interval that ends at p, or, where the ray starts at p, through the inflow rule
// (thermal inflow I = S on the bottom wall for upward rays).  On a Voronoi grid a wall neighbour
// stands in with the site's own S and alpha, so it adds w0 (and e^-d under thermal inflow) to
// the site's weight.  One thread per (point, wavelength) sums w_d times that weight over the
// directions in index order; the points are independent (no sweep order).
#include <algorithm>
#include <vector>

#include "device_common.cuh"
#include "rt_impl.h"

namespace rt {

struct LstRegArgs {
    const float *alpha;        // [nlam][npt]
    float *L;                  // [nlam][npt]
    const Stencil *st;         // [nz][ndir]
    int nx, ny, nz, np, ndir, periodic, thermal;
    float w[MAX_DIR];
    int up[MAX_DIR];
};

__global__ void __launch_bounds__(256) lambda_star_regular_kernel(const LstRegArgs a)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    const int k = blockIdx.y, l = blockIdx.z;
    if (q >= a.np) return;
    const int i = q % a.nx, j = q / a.nx;
    const size_t npt = (size_t)a.np * a.nz;
    const float *al = a.alpha + (size_t)l * npt;
    const float ak = __ldg(al + (size_t)k * a.np + q);
    float acc = 0.f;
    for (int d = 0; d < a.ndir; ++d) {
        const bool up = a.up[d];
        if (k == (up ? 0 : a.nz - 1)) {            // the ray starts here
            if (up && a.thermal) acc += a.w[d];
            continue;
        }
        const int ku = up ? k - 1 : k + 1;
        const Stencil s = a.st[(size_t)k * a.ndir + d];
        const float *Au = al + (size_t)ku * a.np;
        const float ws[4] = {s.w0, s.w1, s.w2, s.w3};
        float au = 0.f;
        int xs[2], ys[2];
        if (a.periodic) {   // axm, aym: the offsets reduced to [0, nx), [0, ny)
            xs[0] = i + s.axm;
            xs[0] -= xs[0] >= a.nx ? a.nx : 0;
            xs[1] = xs[0] + 1 == a.nx ? 0 : xs[0] + 1;
            ys[0] = j + s.aym;
            ys[0] -= ys[0] >= a.ny ? a.ny : 0;
            ys[1] = ys[0] + 1 == a.ny ? 0 : ys[0] + 1;
        } else {
            xs[0] = min(max(i + s.ax, 0), a.nx - 1);
            xs[1] = min(max(i + s.ax + 1, 0), a.nx - 1);
            ys[0] = min(max(j + s.ay, 0), a.ny - 1);
            ys[1] = min(max(j + s.ay + 1, 0), a.ny - 1);
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) au += ws[c] * __ldg(Au + ys[c >> 1] * a.nx + xs[c & 1]);
        float ex, w0, w1;
        lin_weights((au + ak) * s.hds, ex, w0, w1);
        acc += a.w[d] * w1;
    }
    a.L[(size_t)l * npt + (size_t)k * a.np + q] = acc;
}

struct LstVorArgs {
    const float *alpha;        // [nlam][n]
    float *L;                  // [nlam][n]
    const Upwind *up;          // [ndir][n] site order
    int n, nlam, ndir, thermal;
    float w[MAX_DIR];
    int updir[MAX_DIR];
};

__global__ void __launch_bounds__(256) lambda_star_voronoi_kernel(const LstVorArgs a)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)a.n * a.nlam) return;
    const int l = (int)(t / a.n);
    const int i = (int)(t % a.n);
    const float *al = a.alpha + (size_t)l * a.n;
    const float ai = __ldg(al + i);
    float acc = 0.f;
    for (int d = 0; d < a.ndir; ++d) {
        const Upwind u = a.up[(size_t)d * a.n + i];
        float own = 0.f;
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const int k = c ? u.k2 : u.k1;
            const float wk = c ? 1.f - u.w1 : u.w1;
            if (wk == 0.f) continue;
            const float len = c ? u.l2 : u.l1;
            const float ak = k >= 0 ? __ldg(al + k) : ai;
            float ex, w0, w1;
            lin_weights(0.5f * (ak + ai) * len, ex, w0, w1);
            float o = w1;
            if (k < 0) o += w0 + ((a.thermal && a.updir[d] && k == -1) ? ex : 0.f);
            own += wk * o;
        }
        acc += a.w[d] * own;
    }
    a.L[t] = acc;
}

// site-ordered upwind records of the quadrature directions on the device (built once)
static rt_status voronoi_site_records(rt_grid *g, const Upwind **out)
{
    if (!g->d_up_site) {
        const size_t bytes = g->vt.h_up.size() * sizeof(Upwind);
        RT_CUDA(cudaMalloc(&g->d_up_site, bytes));
        RT_CUDA(cudaMemcpy(g->d_up_site, g->vt.h_up.data(), bytes, cudaMemcpyHostToDevice));
    }
    *out = g->d_up_site;
    return RT_OK;
}

rt_status lambda_star_prepare(rt_grid *g)
{
    if (g->kind != RT_GRID_VORONOI) return RT_OK;
    const Upwind *u;
    return voronoi_site_records(g, &u);
}

rt_status lambda_star(rt_grid *g, int nlam, const float *alpha, int bc, float *L, cudaStream_t st)
{
    if (g->ndir > MAX_DIR) return fail(RT_EINVAL, "too many directions");
    const int thermal = bc == RT_BC_THERMAL;
    if (g->kind == RT_GRID_REGULAR) {
        LstRegArgs a;
        a.alpha = alpha;
        a.L = L;
        a.st = g->d_stencil;
        a.nx = g->nx;
        a.ny = g->ny;
        a.nz = g->nz;
        a.np = g->nx * g->ny;
        a.ndir = g->ndir;
        a.periodic = g->periodic;
        a.thermal = thermal;
        for (int d = 0; d < g->ndir; ++d) {
            a.w[d] = (float)g->wdir[d];
            a.up[d] = g->dirs[3 * d + 2] > 0;
        }
        dim3 grid((unsigned)((a.np + 255) / 256), (unsigned)g->nz, (unsigned)nlam);
        note_launch();
        lambda_star_regular_kernel<<<grid, 256, 0, st>>>(a);
    } else {
        LstVorArgs a;
        RT_TRY(voronoi_site_records(g, &a.up));
        a.alpha = alpha;
        a.L = L;
        a.n = (int)g->nsites;
        a.nlam = nlam;
        a.ndir = g->ndir;
        a.thermal = thermal;
        for (int d = 0; d < g->ndir; ++d) {
            a.w[d] = (float)g->wdir[d];
            a.updir[d] = g->dirs[3 * d + 2] > 0;
        }
        const int64_t work = (int64_t)a.n * nlam;
        note_launch();
        lambda_star_voronoi_kernel<<<(unsigned)((work + 255) / 256), 256, 0, st>>>(a);
    }
    RT_CUDA(cudaGetLastError());
    return RT_OK;
}

}  // namespace rt

using namespace rt;

extern "C" rt_status rt_lambda_star(rt_grid_t g, int nlam, const float *alpha, int bc, float *L,
                                    void *stream)
{
    return guarded([&]() -> rt_status {
        if (!g || !alpha || !L) return fail(RT_EINVAL, "null argument");
        if (nlam < 1) return fail(RT_EINVAL, "nlam must be >= 1");
        if (bc != RT_BC_THERMAL && bc != RT_BC_ZERO && bc != RT_BC_ARRAY)
            return fail(RT_EINVAL, "bc must be THERMAL, ZERO or ARRAY");
        return lambda_star(g, nlam, alpha, bc, L, (cudaStream_t)stream);
    });
}
