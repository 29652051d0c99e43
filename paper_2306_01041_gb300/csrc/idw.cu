// Final synthesis on a Voronoi grid (Sect. 2.5, last paragraphs): the converged site populations
// are interpolated back to the original mesh by inverse-distance weighting over the two nearest
// sites, and the emergent intensity is then a formal solution on that mesh along vertical long
// characteristics (rt_emergent_intensity with mu = 1 on the regular grid).
//
// The two-nearest table is geometry, built once per (Voronoi grid, mesh) pair on the host, exact:
// sites binned in a uniform cell grid (about two per cell on average), each mesh point searched
// in Chebyshev shells of cells around its own until the second-nearest distance is within the
// radius no unvisited cell can beat; minimum-image distances in the periodic x and y, ties to
// the smaller site index.  Weights 1/d, normalised; (1, 0) on a site.  Mesh point (i, j, k) is
// at (i dx, j dy, z_k) in the sites' frame.  The interpolation is a gather kernel.
#include <algorithm>
#include <cmath>
#include <vector>

#include "device_common.cuh"
#include "rt_impl.h"

struct rt_idw {
    int64_t npt = 0, nsites = 0;
    int2 *d_k = nullptr;
    float2 *d_w = nullptr;
    std::vector<int2> h_k;
    std::vector<float2> h_w;
    ~rt_idw()
    {
        cudaFree(d_k);
        cudaFree(d_w);
    }
};

namespace rt {

__global__ void idw_gather_kernel(const int2 *__restrict__ k, const float2 *__restrict__ w,
                                  const float *__restrict__ src, float *__restrict__ dst,
                                  int64_t npt, int64_t ns, int nf)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= npt * nf) return;
    const int f = (int)(t / npt);
    const int64_t p = t % npt;
    const int2 kk = k[p];
    const float2 ww = w[p];
    const float *s = src + (size_t)f * ns;
    dst[t] = ww.x * __ldg(s + kk.x) + ww.y * __ldg(s + kk.y);
}

namespace {

struct Bins {
    int nc[3];
    double lo[3], len[3], h[3];
    std::vector<int64_t> start;   // [ncells + 1]
    std::vector<int32_t> site;    // sites, by cell
    int cell(int axis, double v) const
    {
        int c = (int)std::floor((v - lo[axis]) / len[axis] * nc[axis]);
        if (axis < 2) {
            c %= nc[axis];
            return c < 0 ? c + nc[axis] : c;
        }
        return std::min(std::max(c, 0), nc[axis] - 1);
    }
};

Bins make_bins(const rt_grid *v)
{
    Bins b;
    const int64_t n = v->nsites;
    for (int a = 0; a < 3; ++a) {
        b.lo[a] = v->box[2 * a];
        b.len[a] = v->box[2 * a + 1] - v->box[2 * a];
    }
    const double vol = b.len[0] * b.len[1] * b.len[2];
    const double h = std::cbrt(vol / std::max<double>(1.0, 0.5 * (double)n));
    for (int a = 0; a < 3; ++a) {
        b.nc[a] = std::max(1, std::min(1024, (int)(b.len[a] / h)));
        b.h[a] = b.len[a] / b.nc[a];
    }
    const int64_t ncell = (int64_t)b.nc[0] * b.nc[1] * b.nc[2];
    std::vector<int64_t> cnt(ncell + 1, 0);
    std::vector<int64_t> cid(n);
    for (int64_t s = 0; s < n; ++s) {
        const double *p = &v->xyz[3 * s];
        cid[s] = ((int64_t)b.cell(2, p[2]) * b.nc[1] + b.cell(1, p[1])) * b.nc[0] + b.cell(0, p[0]);
        ++cnt[cid[s] + 1];
    }
    for (int64_t c = 0; c < ncell; ++c) cnt[c + 1] += cnt[c];
    b.start = cnt;
    b.site.resize(n);
    for (int64_t s = 0; s < n; ++s) b.site[cnt[cid[s]]++] = (int32_t)s;   // stable by index
    return b;
}

struct Near {
    double d2;
    int32_t k;
};

inline bool closer(const Near &a, const Near &b) { return a.d2 < b.d2 || (a.d2 == b.d2 && a.k < b.k); }

void two_nearest(const rt_grid *v, const Bins &b, const double q[3], Near &n1, Near &n2)
{
    n1 = {INFINITY, -1};
    n2 = {INFINITY, -1};
    const double Lx = b.len[0], Ly = b.len[1];
    const int c0[3] = {b.cell(0, q[0]), b.cell(1, q[1]), b.cell(2, q[2])};
    const double hmin = std::min(b.h[0], std::min(b.h[1], b.h[2]));
    const int rmax = std::max(b.nc[0], std::max(b.nc[1], b.nc[2]));
    for (int r = 0; r <= rmax; ++r) {
        for (int dz = -r; dz <= r; ++dz) {
            const int cz = c0[2] + dz;
            if (cz < 0 || cz >= b.nc[2]) continue;
            for (int dy = -r; dy <= r; ++dy)
                for (int dx = -r; dx <= r; ++dx) {
                    if (std::max(std::abs(dx), std::max(std::abs(dy), std::abs(dz))) != r) continue;
                    const int cx = ((c0[0] + dx) % b.nc[0] + b.nc[0]) % b.nc[0];
                    const int cy = ((c0[1] + dy) % b.nc[1] + b.nc[1]) % b.nc[1];
                    const int64_t c = ((int64_t)cz * b.nc[1] + cy) * b.nc[0] + cx;
                    for (int64_t e = b.start[c]; e < b.start[c + 1]; ++e) {
                        const int32_t s = b.site[e];
                        if (s == n1.k || s == n2.k) continue;   // a wrapped shell revisits cells
                        const double *p = &v->xyz[3 * (size_t)s];
                        double ex = p[0] - q[0], ey = p[1] - q[1], ez = p[2] - q[2];
                        ex -= Lx * std::nearbyint(ex / Lx);
                        ey -= Ly * std::nearbyint(ey / Ly);
                        const Near cand{ex * ex + ey * ey + ez * ez, s};
                        if (closer(cand, n1)) {
                            n2 = n1;
                            n1 = cand;
                        } else if (closer(cand, n2)) {
                            n2 = cand;
                        }
                    }
                }
        }
        // every unvisited site lies at least r cells away from the query's cell
        const double reach = r * hmin;
        if (n2.k >= 0 && n2.d2 <= reach * reach) break;
    }
}

}  // namespace

// Pixel table of the emergent map on a Voronoi grid: the two nearest emergent-layer sites of every
// pixel in (x, y), with their weights, and a buffer for the intensities at those sites.
struct MapTable {
    int npx = 0, npy = 0;
    int64_t ntop = 0;
    int2 *d_k = nullptr;      // [npy * npx] positions in the grid's top list
    float2 *d_w = nullptr;
    float *d_itop = nullptr;  // [nlam][ntop]
    int itop_nlam = 0;
};

void map_release(MapTable *t)
{
    if (!t) return;
    cudaFree(t->d_k);
    cudaFree(t->d_w);
    cudaFree(t->d_itop);
    delete t;
}

// Builds (or reuses) the pixel table of an npx x npy map: pixel (i, j) at (x0 + i Lx / npx,
// y0 + j Ly / npy); two nearest top sites by distance in (x, y) with the minimum image in the
// periodic x and y, ties to the earlier site of the top list (the smaller site index); weights
// 1/d normalised, (1, 0) on a site.
static rt_status map_table(rt_grid *g, int npx, int npy, int nlam, MapTable **out)
{
    MapTable *t = g->map;
    if (!t || t->npx != npx || t->npy != npy) {
        map_release(t);
        g->map = nullptr;
        t = new MapTable();
        t->npx = npx;
        t->npy = npy;
        t->ntop = (int64_t)g->top.size();
        const double Lx = g->box[1] - g->box[0], Ly = g->box[3] - g->box[2];
        const int64_t np = (int64_t)npx * npy;
        std::vector<int2> hk(np);
        std::vector<float2> hw(np);
    #pragma omp parallel for schedule(static)
        for (int64_t p = 0; p < np; ++p) {
            const double qx = g->box[0] + (double)(p % npx) * Lx / npx;
            const double qy = g->box[2] + (double)(p / npx) * Ly / npy;
            double d1 = INFINITY, d2 = INFINITY;
            int k1 = -1, k2 = -1;
            for (int64_t q = 0; q < t->ntop; ++q) {
                const double *s = &g->xyz[3 * (size_t)g->top[q]];
                double ex = s[0] - qx, ey = s[1] - qy;
                ex -= Lx * std::nearbyint(ex / Lx);
                ey -= Ly * std::nearbyint(ey / Ly);
                const double d = ex * ex + ey * ey;
                if (d < d1) {
                    d2 = d1;
                    k2 = k1;
                    d1 = d;
                    k1 = (int)q;
                } else if (d < d2) {
                    d2 = d;
                    k2 = (int)q;
                }
            }
            float w1 = 1.f, w2 = 0.f;
            if (d1 > 0.0) {
                const double a = 1.0 / std::sqrt(d1), c = 1.0 / std::sqrt(d2);
                w1 = (float)(a / (a + c));
                w2 = (float)(c / (a + c));
            }
            hk[p] = make_int2(k1, k2);
            hw[p] = make_float2(w1, w2);
        }
        cudaError_t e = cudaMalloc(&t->d_k, np * sizeof(int2));
        if (e == cudaSuccess) e = cudaMalloc(&t->d_w, np * sizeof(float2));
        if (e == cudaSuccess) e = cudaMemcpy(t->d_k, hk.data(), np * sizeof(int2), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(t->d_w, hw.data(), np * sizeof(float2), cudaMemcpyHostToDevice);
        g->map = t;
        if (e != cudaSuccess) return cuda_fail(e, "emergent map table upload");
    }
    if (t->itop_nlam < nlam) {
        cudaFree(t->d_itop);
        t->d_itop = nullptr;
        t->itop_nlam = 0;
        RT_CUDA(cudaMalloc(&t->d_itop, (size_t)nlam * std::max<int64_t>(1, t->ntop) * sizeof(float)));
        t->itop_nlam = nlam;
    }
    *out = t;
    return RT_OK;
}

}  // namespace rt

using namespace rt;

extern "C" {

rt_status rt_idw_create(rt_grid_t voronoi, rt_grid_t mesh, rt_idw_t *out)
{
    return guarded([&]() -> rt_status {
        if (!voronoi || !mesh || !out) return fail(RT_EINVAL, "null argument");
        *out = nullptr;
        if (voronoi->kind != RT_GRID_VORONOI || mesh->kind != RT_GRID_REGULAR)
            return fail(RT_EINVAL, "rt_idw_create takes a Voronoi grid and a regular grid");
        if (voronoi->nsites < 2) return fail(RT_EINVAL, "need at least two sites");
        rt_idw *t = new (std::nothrow) rt_idw();
        if (!t) return fail(RT_ENOMEM, "host allocation failed");
        t->npt = mesh->npt;
        t->nsites = voronoi->nsites;
        const Bins b = make_bins(voronoi);
        t->h_k.resize(t->npt);
        t->h_w.resize(t->npt);
        const int nx = mesh->nx, ny = mesh->ny;
    #pragma omp parallel for schedule(dynamic, 256)
        for (int64_t p = 0; p < t->npt; ++p) {
            const int i = (int)(p % nx), j = (int)((p / nx) % ny), k = (int)(p / ((int64_t)nx * ny));
            const double q[3] = {i * mesh->dx, j * mesh->dy, mesh->z[k]};
            Near n1, n2;
            two_nearest(voronoi, b, q, n1, n2);
            const double d1 = std::sqrt(n1.d2), d2 = std::sqrt(n2.d2);
            float w1 = 1.f, w2 = 0.f;
            if (d1 > 0.0) {
                const double a = 1.0 / d1, c = 1.0 / d2;
                w1 = (float)(a / (a + c));
                w2 = (float)(c / (a + c));
            }
            t->h_k[p] = make_int2(n1.k, n2.k);
            t->h_w[p] = make_float2(w1, w2);
        }
        cudaError_t e = cudaMalloc(&t->d_k, t->npt * sizeof(int2));
        if (e == cudaSuccess) e = cudaMalloc(&t->d_w, t->npt * sizeof(float2));
        if (e == cudaSuccess)
            e = cudaMemcpy(t->d_k, t->h_k.data(), t->npt * sizeof(int2), cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(t->d_w, t->h_w.data(), t->npt * sizeof(float2), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            delete t;
            return cuda_fail(e, "idw table upload");
        }
        *out = t;
        return RT_OK;
    });
}

void rt_idw_destroy(rt_idw_t t) { delete t; }

rt_status rt_idw_table(rt_idw_t t, int32_t *k, float *w)
{
    return guarded([&]() -> rt_status {
        if (!t || !k || !w) return fail(RT_EINVAL, "null argument");
        for (int64_t p = 0; p < t->npt; ++p) {
            k[2 * p] = t->h_k[p].x;
            k[2 * p + 1] = t->h_k[p].y;
            w[2 * p] = t->h_w[p].x;
            w[2 * p + 1] = t->h_w[p].y;
        }
        return RT_OK;
    });
}

rt_status rt_idw_interpolate(rt_idw_t t, int nf, const float *src, float *dst, void *stream)
{
    return guarded([&]() -> rt_status {
        if (!t || !src || !dst) return fail(RT_EINVAL, "null argument");
        if (nf < 1) return fail(RT_EINVAL, "nf must be >= 1");
        const int64_t work = t->npt * nf;
        note_launch();
        idw_gather_kernel<<<(unsigned)((work + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
            t->d_k, t->d_w, src, dst, t->npt, t->nsites, nf);
        RT_CUDA(cudaGetLastError());
        return RT_OK;
    });
}

rt_status rt_emergent_map(rt_grid_t g, const double dir[3], int nlam, const float *alpha,
                          const float *S, int bc, int npx, int npy, float *map, void *stream)
{
    return guarded([&]() -> rt_status {
        if (!g || !dir || !alpha || !S || !map) return fail(RT_EINVAL, "null argument");
        if (nlam < 1 || npx < 1 || npy < 1) return fail(RT_EINVAL, "nlam, npx and npy must be >= 1");
        if (g->kind == RT_GRID_REGULAR) {
            if (npx != g->nx || npy != g->ny)
                return fail(RT_EINVAL, "on a regular grid the map is the top plane: npx = nx, npy = ny");
            return rt_emergent_intensity(g, dir, nlam, alpha, S, bc, map, stream);
        }
        if (g->top.size() < 2) return fail(RT_EINVAL, "need at least two emergent-layer sites");
        MapTable *t = nullptr;
        RT_TRY(map_table(g, npx, npy, nlam, &t));
        RT_TRY(rt_emergent_intensity(g, dir, nlam, alpha, S, bc, t->d_itop, stream));
        const int64_t np = (int64_t)npx * npy, work = np * nlam;
        note_launch();
        idw_gather_kernel<<<(unsigned)((work + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
            t->d_k, t->d_w, t->d_itop, map, np, t->ntop, nlam);
        RT_CUDA(cudaGetLastError());
        return RT_OK;
    });
}

}  // extern "C"
