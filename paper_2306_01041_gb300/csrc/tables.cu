// Voronoi upwind tables and dependency levels built on the GPU (Sect. 2.5, Eq. 5 and the weight
// formula after it): the same definition as the host build of rt_grid_create.
//
// For site i and direction u, every Delaunay neighbour k strictly upwind in height competes with
// v = u . e(k -> i) > 0; the two largest v win (ties: smaller neighbour code, then smaller image
// shift), with weights v^r / (v1^r + v2^r) and the Delaunay segment lengths (a wall mirror stands
// for the wall: its segment runs from the wall crossing to the site).  With no competitor, the most
// nearly vertical upwind neighbour, else the wall itself.  Every geometric quantity is computed
// with one IEEE double operation per step in the order of that definition (explicit
// round-to-nearest intrinsics, nothing fused), so the choices are those of the host build.
//
// Levels: 0 for a site fed only by walls, else one more than its deepest upwind site.  Every link
// goes strictly upwind in height, so the links form a DAG and the levels are the fixed point of
// level(i) = max(level(i), 1 + level(k)) over the links, reached by repeated passes (each pass at
// least one level deeper; levels only grow, so reading a neighbour's level while it is updated
// is harmless).  The slot order by level is built on the host from the levels.
#include <algorithm>
#include <cmath>
#include <vector>

#include "device_common.cuh"
#include "rt_impl.h"

namespace rt {

struct TabArgs {
    const double *xyz;       // [n][3]
    const int64_t *off;      // [n + 1]
    const int32_t *code;     // [ne]
    const int8_t *shift;     // [ne] or null (image (0, 0))
    const double *dirs;      // [ndir][3]
    double box[6];
    double r_exp;
    int64_t n;
    Upwind *up;              // [ndir][n], site order
    unsigned long long *nfb;
    unsigned *err;
};

struct Cand {
    double v, len;
    int32_t code;
    int shift, k;
};

__device__ __forceinline__ bool beats(const Cand &a, const Cand &b)
{
    if (a.v != b.v) return a.v > b.v;
    if (a.code != b.code) return a.code < b.code;
    return a.shift < b.shift;
}

__global__ void __launch_bounds__(256) voronoi_tables_kernel(TabArgs a)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int d = blockIdx.y;
    if (i >= a.n) return;
    const double u0 = a.dirs[3 * d], u1 = a.dirs[3 * d + 1], u2 = a.dirs[3 * d + 2];
    const double sgn = u2 > 0.0 ? 1.0 : -1.0;
    const double xi0 = a.xyz[3 * i], xi1 = a.xyz[3 * i + 1], xi2 = a.xyz[3 * i + 2];
    const double Lx = __dsub_rn(a.box[1], a.box[0]), Ly = __dsub_rn(a.box[3], a.box[2]);
    Cand best[2];
    int nc = 0;
    double vert_best = -1.0, vert_len = 0.0;
    int vert_k = 0;
    for (int64_t e = a.off[i]; e < a.off[i + 1]; ++e) {
        const int32_t code = a.code[e];
        const int sh = a.shift ? (int)a.shift[e] : 4;
        int64_t k;
        int wall;
        if (code >= 0) {
            k = code;
            wall = 0;
        } else {
            const int64_t c = -(int64_t)code - 1;   // 2k (bottom mirror) or 2k + 1 (top mirror)
            k = c >> 1;
            wall = (c & 1) ? 2 : 1;
        }
        if (k < 0 || k >= a.n || sh < 0 || sh > 8) {   // validated on the host; never taken
            flag_error(a.err, ERR_INDEX);
            continue;
        }
        const int sx = sh / 3 - 1, sy = sh % 3 - 1;
        const double p0 = __dadd_rn(a.xyz[3 * k], __dmul_rn((double)sx, Lx));
        const double p1 = __dadd_rn(a.xyz[3 * k + 1], __dmul_rn((double)sy, Ly));
        double p2 = a.xyz[3 * k + 2];
        if (wall == 1) p2 = __dsub_rn(__dmul_rn(2.0, a.box[4]), p2);
        if (wall == 2) p2 = __dsub_rn(__dmul_rn(2.0, a.box[5]), p2);
        const double dzv = __dsub_rn(xi2, p2);
        if (__dmul_rn(dzv, sgn) <= 0.0) continue;              // not upwind in height
        const double dv0 = __dsub_rn(xi0, p0), dv1 = __dsub_rn(xi1, p1);
        const double len = __dsqrt_rn(
            __dadd_rn(__dadd_rn(__dmul_rn(dv0, dv0), __dmul_rn(dv1, dv1)), __dmul_rn(dzv, dzv)));
        double seg = len;
        int kk = (int)k;
        if (wall) {
            const double zw = wall == 1 ? a.box[4] : a.box[5];
            seg = __ddiv_rn(__dmul_rn(len, __dsub_rn(xi2, zw)), dzv);
            kk = -wall;
        }
        const double vs = __ddiv_rn(__dmul_rn(dzv, sgn), len);
        if (vs > vert_best) {
            vert_best = vs;
            vert_k = kk;
            vert_len = seg;
        }
        const double v = __ddiv_rn(
            __dadd_rn(__dadd_rn(__dmul_rn(u0, dv0), __dmul_rn(u1, dv1)), __dmul_rn(u2, dzv)), len);
        if (!(v > 0.0)) continue;
        const Cand c{v, seg, code, sh, kk};
        if (nc == 0 || beats(c, best[0])) {
            best[1] = best[0];
            best[0] = c;
        } else if (nc == 1 || beats(c, best[1])) {
            best[1] = c;
        }
        ++nc;
    }
    Upwind w;
    if (nc >= 2) {
        const double p = pow(best[0].v, a.r_exp), q = pow(best[1].v, a.r_exp);
        w = Upwind{best[0].k, best[1].k, (float)(p / (p + q)), (float)best[0].len,
                   (float)best[1].len};
    } else if (nc == 1) {
        w = Upwind{best[0].k, best[0].k, 1.0f, (float)best[0].len, (float)best[0].len};
    } else {
        atomicAdd(a.nfb, 1ull);
        if (vert_best < 0.0) {                // nothing upwind in height: the wall itself
            vert_k = u2 > 0.0 ? -1 : -2;
            vert_len = __ddiv_rn(u2 > 0.0 ? __dsub_rn(xi2, a.box[4]) : __dsub_rn(a.box[5], xi2),
                                 fabs(u2));
        }
        w = Upwind{vert_k, vert_k, 1.0f, (float)vert_len, (float)vert_len};
    }
    a.up[(size_t)d * a.n + i] = w;
}

// one relaxation pass of the levels of every (site, direction); *changed = 1 if any grew
__global__ void __launch_bounds__(256) voronoi_levels_kernel(const Upwind *up, int64_t n,
                                                             int *level, unsigned *changed,
                                                             unsigned *err)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int d = blockIdx.y;
    if (i >= n) return;
    const Upwind r = up[(size_t)d * n + i];
    volatile int *lv = level + (size_t)d * n;
    int L = 0;
    const int ks[2] = {r.k1, r.k2};
    for (int c = 0; c < 2; ++c) {
        const int k = ks[c];
        if (k < 0) continue;
        if (k >= n) {
            flag_error(err, ERR_INDEX);
            continue;
        }
        L = max(L, lv[k] + 1);
    }
    if (L > lv[i]) {
        atomicMax(level + (size_t)d * n + i, L);
        *(volatile unsigned *)changed = 1u;
    }
}

}  // namespace rt

using namespace rt;

namespace rt {

// The upwind tables and levels of the grid's quadrature directions, built on the device and
// written into g->vt (host copies, slot order, device arrays; the arrays are reused when they
// exist, so batches made from the grid keep valid pointers).
rt_status voronoi_build_tables_device(rt_grid *g, cudaStream_t st)
{
    {
        const int64_t n = g->nsites;
        const int nd = g->ndir;
        VorTables &vt0 = g->vt;
        if (vt0.ndir != nd || vt0.h_up.size() != (size_t)nd * n) {
            vt0.ndir = nd;
            vt0.dirs.assign(g->dirs.begin(), g->dirs.end());
            vt0.h_up.assign((size_t)nd * n, Upwind{});
            vt0.h_level.assign((size_t)nd * n, 0);
            vt0.h_upd.clear();
        }
    }
    {
        const int64_t n = g->nsites;
        const int nd = g->ndir;
        const int64_t ne = g->nbr_off[n];
        const bool has_shift = !g->nbr_shift.empty();
        struct Buf {
            void *p = nullptr;
            ~Buf() { if (p) cudaFree(p); }
        } buf;
        auto up8 = [](size_t b) { return (b + 255) & ~(size_t)255; };
        const size_t b_xyz = up8(3 * n * sizeof(double)), b_off = up8((n + 1) * sizeof(int64_t));
        const size_t b_code = up8(ne * sizeof(int32_t)), b_shift = up8(has_shift ? ne : 1);
        const size_t b_dirs = up8(3 * nd * sizeof(double));
        const size_t b_up = up8((size_t)nd * n * sizeof(Upwind));
        const size_t b_lv = up8((size_t)nd * n * sizeof(int));
        const size_t total = b_xyz + b_off + b_code + b_shift + b_dirs + b_up + b_lv + 256;
        RT_CUDA(cudaMalloc(&buf.p, total));
        char *c = (char *)buf.p;
        double *d_xyz = (double *)c;
        c += b_xyz;
        int64_t *d_off = (int64_t *)c;
        c += b_off;
        int32_t *d_code = (int32_t *)c;
        c += b_code;
        int8_t *d_shift = (int8_t *)c;
        c += b_shift;
        double *d_dirs = (double *)c;
        c += b_dirs;
        Upwind *d_up = (Upwind *)c;
        c += b_up;
        int *d_level = (int *)c;
        c += b_lv;
        unsigned long long *d_nfb = (unsigned long long *)c;
        unsigned *d_changed = (unsigned *)(d_nfb + 1);
        RT_CUDA(cudaMemcpyAsync(d_xyz, g->xyz.data(), 3 * n * sizeof(double),
                                cudaMemcpyHostToDevice, st));
        RT_CUDA(cudaMemcpyAsync(d_off, g->nbr_off.data(), (n + 1) * sizeof(int64_t),
                                cudaMemcpyHostToDevice, st));
        RT_CUDA(cudaMemcpyAsync(d_code, g->nbr_idx.data(), ne * sizeof(int32_t),
                                cudaMemcpyHostToDevice, st));
        if (has_shift)
            RT_CUDA(cudaMemcpyAsync(d_shift, g->nbr_shift.data(), ne, cudaMemcpyHostToDevice, st));
        RT_CUDA(cudaMemcpyAsync(d_dirs, g->dirs.data(), 3 * nd * sizeof(double),
                                cudaMemcpyHostToDevice, st));
        RT_CUDA(cudaMemsetAsync(d_level, 0, (size_t)nd * n * sizeof(int), st));
        RT_CUDA(cudaMemsetAsync(d_nfb, 0, sizeof(unsigned long long), st));
        TabArgs a;
        a.xyz = d_xyz;
        a.off = d_off;
        a.code = d_code;
        a.shift = has_shift ? d_shift : nullptr;
        a.dirs = d_dirs;
        for (int q = 0; q < 6; ++q) a.box[q] = g->box[q];
        a.r_exp = g->r_exp;
        a.n = n;
        a.up = d_up;
        a.nfb = d_nfb;
        a.err = g->d_err;
        const dim3 grid((unsigned)((n + 255) / 256), (unsigned)nd);
        note_launch();
        voronoi_tables_kernel<<<grid, 256, 0, st>>>(a);
        RT_CUDA(cudaGetLastError());
        // levels: passes until none grows (at most n + 1 passes in a DAG), four per check
        unsigned h_changed = 1;
        int64_t passes = 0;
        while (h_changed) {
            if (passes > n + 4) return fail(RT_ECYCLE, "upwind links are not acyclic");
            RT_CUDA(cudaMemsetAsync(d_changed, 0, sizeof(unsigned), st));
            note_launch(4);
            for (int r = 0; r < 4; ++r)
                voronoi_levels_kernel<<<grid, 256, 0, st>>>(d_up, n, d_level, d_changed, g->d_err);
            RT_CUDA(cudaMemcpyAsync(&h_changed, d_changed, sizeof(unsigned),
                                    cudaMemcpyDeviceToHost, st));
            RT_CUDA(cudaStreamSynchronize(st));
            passes += 4;
        }
        RT_TRY(check_dev_error(g, st));
        VorTables &vt = g->vt;
        unsigned long long nfb = 0;
        RT_CUDA(cudaMemcpyAsync(vt.h_up.data(), d_up, (size_t)nd * n * sizeof(Upwind),
                                cudaMemcpyDeviceToHost, st));
        RT_CUDA(cudaMemcpyAsync(vt.h_level.data(), d_level, (size_t)nd * n * sizeof(int),
                                cudaMemcpyDeviceToHost, st));
        RT_CUDA(cudaMemcpyAsync(&nfb, d_nfb, sizeof(nfb), cudaMemcpyDeviceToHost, st));
        RT_CUDA(cudaStreamSynchronize(st));
        vt.n_fallback = (int64_t)nfb;
        // slot order and upload into the grid's existing device arrays (batches made from this
        // grid keep valid pointers)
        RT_TRY(voronoi_upload_slots(vt, n, st));
        g->max_levels = vt.max_levels;
        g->n_fallback = vt.n_fallback;
        return RT_OK;
    }
}

}  // namespace rt

extern "C" rt_status rt_grid_build_tables_device(rt_grid_t g, void *stream)
{
    return guarded([&]() -> rt_status {
        if (!g) return fail(RT_EINVAL, "null grid");
        if (g->kind != RT_GRID_VORONOI) return fail(RT_EINVAL, "Voronoi grids only");
        RT_TRY(voronoi_build_tables_device(g, (cudaStream_t)stream));
        // caches derived from the tables
        if (g->self_batch) rt_batch_destroy(g->self_batch);
        g->self_batch = nullptr;
        g->self_batch_nlam = 0;
        if (g->d_up_site)
            RT_CUDA(cudaMemcpy(g->d_up_site, g->vt.h_up.data(), g->vt.h_up.size() * sizeof(Upwind),
                               cudaMemcpyHostToDevice));
        return RT_OK;
    });
}
