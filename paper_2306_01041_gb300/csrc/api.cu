// C ABI entry points of librt.so: error reporting, grid construction (regular-grid stencils,
// Voronoi upwind tables and dependency levels), and dispatch to the kernels.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <numeric>

#include "rt_impl.h"

namespace rt {

static thread_local std::string g_last_error;
static std::atomic<unsigned long long> g_launches{0};

void note_launch(unsigned n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

rt_status fail(rt_status st, const std::string &msg)
{
    g_last_error = msg;
    return st;
}

rt_status cuda_fail(cudaError_t e, const char *what)
{
    g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
    cudaGetLastError();   // clear a non-sticky error so that it does not resurface later
    return e == cudaErrorMemoryAllocation ? RT_ENOMEM : RT_ECUDA;
}

rt_status scratch_get(rt_grid *g, int slot, size_t bytes, void **out)
{
    Scratch &s = g->scratch[slot];
    if (s.bytes < bytes) {
        if (s.p) cudaFree(s.p);
        s.p = nullptr;
        s.bytes = 0;
        cudaError_t e = cudaMalloc(&s.p, bytes);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(scratch)");
        s.bytes = bytes;
    }
    *out = s.p;
    return RT_OK;
}

rt_status check_dev_error(rt_grid *g, cudaStream_t st)
{
    unsigned h = 0;
    RT_CUDA(cudaMemcpyAsync(&h, g->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    RT_CUDA(cudaStreamSynchronize(st));
    if (h) {
        RT_CUDA(cudaMemsetAsync(g->d_err, 0, sizeof(unsigned), st));
        if (h & ERR_TIMEOUT) return fail(RT_ETIMEOUT, "a bounded device wait gave up");
        if (h & ERR_NAN) return fail(RT_ENAN, "a non-finite value was produced on the device");
        return fail(RT_EINVAL, "a device-side index check failed");
    }
    return RT_OK;
}

// ---- regular grid ------------------------------------------------------------------------------
// Upwind stencil of plane k for direction u: the point (x_i, y_j, z_k) is reached from the plane
// of the previous sweep step at horizontal offset -(ds u_x, ds u_y), ds = |z_k - z_ku| / |u_z|.
static Stencil plane_stencil(double dz, const double *u, double dx, double dy, int nx, int ny)
{
    double ds = std::fabs(dz) / std::fabs(u[2]);
    double cx = -ds * u[0] / dx, cy = -ds * u[1] / dy;
    double fx = std::floor(cx), fy = std::floor(cy);
    double tx = cx - fx, ty = cy - fy;
    Stencil s;
    s.ax = (int)fx;
    s.ay = (int)fy;
    s.axm = ((s.ax % nx) + nx) % nx;
    s.aym = ((s.ay % ny) + ny) % ny;
    s.w0 = (float)((1.0 - tx) * (1.0 - ty));
    s.w1 = (float)(tx * (1.0 - ty));
    s.w2 = (float)((1.0 - tx) * ty);
    s.w3 = (float)(tx * ty);
    s.hds = (float)(0.5 * ds);
    s.pad = 0.f;
    s.tx = (float)tx;
    s.ty = (float)ty;
    return s;
}

std::vector<Stencil> regular_dir_stencils(const rt_grid *g, const double *u)
{
    std::vector<Stencil> out((size_t)g->nz, Stencil{});
    for (int k = 0; k < g->nz; ++k) {
        int ku = u[2] > 0 ? k - 1 : k + 1;
        if (ku < 0 || ku >= g->nz) continue;
        out[k] = plane_stencil(g->z[k] - g->z[ku], u, g->dx, g->dy, g->nx, g->ny);
    }
    return out;
}

std::vector<StencilD> regular_dir_stencils_d(const rt_grid *g, const double *u)
{
    std::vector<StencilD> out((size_t)g->nz, StencilD{});
    for (int k = 0; k < g->nz; ++k) {
        int ku = u[2] > 0 ? k - 1 : k + 1;
        if (ku < 0 || ku >= g->nz) continue;
        const double ds = std::fabs(g->z[k] - g->z[ku]) / std::fabs(u[2]);
        const double cx = -ds * u[0] / g->dx, cy = -ds * u[1] / g->dy;
        const double fx = std::floor(cx), fy = std::floor(cy);
        const double tx = cx - fx, ty = cy - fy;
        StencilD &s = out[k];
        s.ax = (int)fx;
        s.ay = (int)fy;
        s.axm = ((s.ax % g->nx) + g->nx) % g->nx;
        s.aym = ((s.ay % g->ny) + g->ny) % g->ny;
        s.w0 = (1.0 - tx) * (1.0 - ty);
        s.w1 = tx * (1.0 - ty);
        s.w2 = (1.0 - tx) * ty;
        s.w3 = tx * ty;
        s.hds = 0.5 * ds;
    }
    return out;
}

static rt_status build_regular(rt_grid *g, const rt_grid_desc *d, cudaStream_t st)
{
    if (d->nx < 1 || d->ny < 1 || d->nz < 2 || !(d->dx > 0) || !(d->dy > 0) || !d->z)
        return fail(RT_EINVAL, "regular grid needs nx, ny >= 1, nz >= 2, dx, dy > 0 and z");
    g->nx = d->nx;
    g->ny = d->ny;
    g->nz = d->nz;
    g->dx = d->dx;
    g->dy = d->dy;
    g->z.assign(d->z, d->z + d->nz);
    for (int k = 1; k < g->nz; ++k)
        if (!(g->z[k] > g->z[k - 1])) return fail(RT_EINVAL, "z must be strictly ascending");
    g->npt = (int64_t)g->nx * g->ny * g->nz;
    if (g->npt > (int64_t)INT32_MAX) return fail(RT_EINVAL, "regular grid larger than 2^31 points");
    // stencil[k][d]: plane k reached from its upwind neighbour plane (k-1 up, k+1 down)
    g->h_stencil.assign((size_t)g->nz * g->ndir, Stencil{});
    for (int k = 0; k < g->nz; ++k)
        for (int q = 0; q < g->ndir; ++q) {
            const double *u = &g->dirs[3 * q];
            int ku = u[2] > 0 ? k - 1 : k + 1;
            if (ku < 0 || ku >= g->nz) continue;
            g->h_stencil[(size_t)k * g->ndir + q] =
                plane_stencil(g->z[k] - g->z[ku], u, g->dx, g->dy, g->nx, g->ny);
        }
    RT_CUDA(cudaMalloc(&g->d_stencil, g->h_stencil.size() * sizeof(Stencil)));
    RT_CUDA(cudaMemcpyAsync(g->d_stencil, g->h_stencil.data(), g->h_stencil.size() * sizeof(Stencil),
                            cudaMemcpyHostToDevice, st));
    RT_TRY(regular_wave_prepare(g, st));
    g->max_levels = g->nz;
    g->top.resize((size_t)g->nx * g->ny);
    std::iota(g->top.begin(), g->top.end(), (int64_t)(g->nz - 1) * g->nx * g->ny);
    return RT_OK;
}

// ---- Voronoi grid ------------------------------------------------------------------------------
struct NbrGeom {
    double p[3];
    int wall;       // 0 site, 1 bottom mirror, 2 top mirror
    int64_t site;
};

static inline NbrGeom neighbour(const rt_grid *g, int32_t code, int8_t shift)
{
    NbrGeom r;
    int sx = shift / 3 - 1, sy = shift % 3 - 1;
    int64_t k;
    if (code >= 0) {
        k = code;
        r.wall = 0;
    } else {
        int64_t c = -(int64_t)code - 1;   // 2k (bottom) or 2k + 1 (top)
        k = c >> 1;
        r.wall = (c & 1) ? 2 : 1;
    }
    r.site = k;
    r.p[0] = g->xyz[3 * k] + sx * (g->box[1] - g->box[0]);
    r.p[1] = g->xyz[3 * k + 1] + sy * (g->box[3] - g->box[2]);
    r.p[2] = g->xyz[3 * k + 2];
    if (r.wall == 1) r.p[2] = 2.0 * g->box[4] - r.p[2];
    if (r.wall == 2) r.p[2] = 2.0 * g->box[5] - r.p[2];
    return r;
}

// Upwind records of every site for direction u (Sect. 2.5): among the Delaunay neighbours that
// lie upwind in height, those whose line towards the site makes v = u . e > 0 compete; the two
// largest v win (ties: smaller neighbour code, then smaller image shift) with weights
// v^r / (v1^r + v2^r).  A wall mirror stands for the wall itself: its segment runs from the wall
// crossing to the site.  With no competitor the most nearly vertical upwind neighbour is used.
static void voronoi_dir_tables(const rt_grid *g, const int64_t *off, const int32_t *code,
                               const int8_t *shift, const double *u, double r,
                               std::vector<Upwind> &out, int64_t &nfb,
                               std::vector<UpwindD> *outd = nullptr)
{
    const int64_t n = g->nsites;
    const double sgn = u[2] > 0 ? 1.0 : -1.0;
    int64_t fb = 0;
#pragma omp parallel for schedule(static) reduction(+ : fb)
    for (int64_t i = 0; i < n; ++i) {
        const double *xi = &g->xyz[3 * i];
        struct Cand { double v; int32_t code; int8_t shift; int k; double len; };
        Cand best[2];
        int nc = 0;
        double vert_best = -1.0;
        int vert_k = 0;
        double vert_len = 0.0;
        for (int64_t e = off[i]; e < off[i + 1]; ++e) {
            int8_t sh = shift ? shift[e] : (int8_t)4;
            NbrGeom nb = neighbour(g, code[e], sh);
            double dzv = xi[2] - nb.p[2];
            if (dzv * sgn <= 0.0) continue;
            double dv[3] = {xi[0] - nb.p[0], xi[1] - nb.p[1], dzv};
            double len = std::sqrt(dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2]);
            double seg = len;
            int kk = (int)nb.site;
            if (nb.wall) {
                double zw = nb.wall == 1 ? g->box[4] : g->box[5];
                seg = len * (xi[2] - zw) / dzv;
                kk = -nb.wall;
            }
            double vs = dzv * sgn / len;
            if (vs > vert_best) { vert_best = vs; vert_k = kk; vert_len = seg; }
            double v = (u[0] * dv[0] + u[1] * dv[1] + u[2] * dv[2]) / len;
            if (!(v > 0.0)) continue;
            Cand c{v, code[e], sh, kk, seg};
            auto beats = [](const Cand &a, const Cand &b) {
                if (a.v != b.v) return a.v > b.v;
                if (a.code != b.code) return a.code < b.code;
                return a.shift < b.shift;
            };
            if (nc == 0 || beats(c, best[0])) {
                best[1] = best[0];
                best[0] = c;
            } else if (nc == 1 || beats(c, best[1])) {
                best[1] = c;
            }
            ++nc;
        }
        Upwind w;
        UpwindD wd;
        if (nc >= 2) {
            double a = std::pow(best[0].v, r), b = std::pow(best[1].v, r);
            w = Upwind{best[0].k, best[1].k, (float)(a / (a + b)), (float)best[0].len,
                       (float)best[1].len};
            wd = UpwindD{best[0].k, best[1].k, a / (a + b), b / (a + b), best[0].len, best[1].len};
        } else if (nc == 1) {
            w = Upwind{best[0].k, best[0].k, 1.0f, (float)best[0].len, (float)best[0].len};
            wd = UpwindD{best[0].k, best[0].k, 1.0, 0.0, best[0].len, best[0].len};
        } else {
            ++fb;
            if (vert_best < 0.0) {
                vert_k = u[2] > 0 ? -1 : -2;
                vert_len = (u[2] > 0 ? xi[2] - g->box[4] : g->box[5] - xi[2]) / std::fabs(u[2]);
            }
            w = Upwind{vert_k, vert_k, 1.0f, (float)vert_len, (float)vert_len};
            wd = UpwindD{vert_k, vert_k, 1.0, 0.0, vert_len, vert_len};
        }
        out[i] = w;
        if (outd) (*outd)[i] = wd;
    }
    nfb += fb;
}

// Dependency levels of one direction: wall-fed sites are level 0, every other site one more than
// its deepest upwind site.  Sites are visited in upwind height order, which is topological
// because each upwind link goes strictly upwind in height; a link that points to a site not yet
// visited means the links are not acyclic.
static bool voronoi_levels(const rt_grid *g, const double *u, const Upwind *up, int32_t *level)
{
    const int64_t n = g->nsites;
    std::vector<int64_t> ord(n);
    std::iota(ord.begin(), ord.end(), (int64_t)0);
    const double sgn = u[2] > 0 ? 1.0 : -1.0;
    std::stable_sort(ord.begin(), ord.end(), [&](int64_t a, int64_t b) {
        return g->xyz[3 * a + 2] * sgn < g->xyz[3 * b + 2] * sgn;
    });
    std::vector<char> done(n, 0);
    for (int64_t q = 0; q < n; ++q) {
        int64_t i = ord[q];
        int L = 0;
        // both links count, even when the second weight rounds to zero in FP32: the levels
        // depend only on the (integer) upwind links
        const int ks[2] = {up[i].k1, up[i].k2};
        for (int c = 0; c < 2; ++c) {
            int k = ks[c];
            if (k < 0) continue;
            if (!done[k]) return false;
            L = std::max(L, level[k] + 1);
        }
        level[i] = L;
        done[i] = 1;
    }
    return true;
}

void VorTables::release()
{
    if (d_up) cudaFree(d_up);
    if (d_order) cudaFree(d_order);
    d_up = nullptr;
    d_order = nullptr;
}

rt_status voronoi_build_tables(const rt_grid *g, int nd, const double *dirs, VorTables &vt,
                               cudaStream_t st)
{
    const int64_t n = g->nsites;
    vt.release();
    vt.ndir = nd;
    vt.dirs.assign(dirs, dirs + 3 * nd);
    vt.h_up.assign((size_t)nd * n, Upwind{});
    vt.h_level.assign((size_t)nd * n, 0);
    vt.n_fallback = 0;
    const int8_t *sh = g->nbr_shift.empty() ? nullptr : g->nbr_shift.data();
    if (nd == 1) vt.h_upd.assign(n, UpwindD{});
    else vt.h_upd.clear();
    for (int q = 0; q < nd; ++q) {
        std::vector<Upwind> tmp(n);
        voronoi_dir_tables(g, g->nbr_off.data(), g->nbr_idx.data(), sh, &vt.dirs[3 * q],
                           g->r_exp, tmp, vt.n_fallback, nd == 1 ? &vt.h_upd : nullptr);
        std::copy(tmp.begin(), tmp.end(), vt.h_up.begin() + (size_t)q * n);
        if (!voronoi_levels(g, &vt.dirs[3 * q], &vt.h_up[(size_t)q * n],
                            &vt.h_level[(size_t)q * n]))
            return fail(RT_ECYCLE, "upwind links are not acyclic");
    }
    return voronoi_upload_slots(vt, n, st);
}

// Slots: the sites of each direction in level order (stable by site index within a level), from
// vt.h_up and vt.h_level; sets the level offsets and max_levels and uploads the slot-ordered
// records and the slot -> site map (into the existing device arrays when there are some).
rt_status voronoi_upload_slots(VorTables &vt, int64_t n, cudaStream_t st)
{
    const int nd = vt.ndir;
    std::vector<Upwind> slot_up((size_t)nd * n);
    std::vector<int32_t> order((size_t)nd * n);
    vt.lvl_off.assign(nd, {});
    vt.max_levels = 0;
    for (int q = 0; q < nd; ++q) {
        const int32_t *lv = &vt.h_level[(size_t)q * n];
        int L = 0;
        for (int64_t i = 0; i < n; ++i) L = std::max(L, lv[i] + 1);
        std::vector<int64_t> cnt(L + 1, 0);
        for (int64_t i = 0; i < n; ++i) cnt[lv[i] + 1]++;
        for (int l = 0; l < L; ++l) cnt[l + 1] += cnt[l];
        vt.lvl_off[q] = cnt;
        std::vector<int64_t> pos(cnt.begin(), cnt.end() - 1);
        for (int64_t i = 0; i < n; ++i) {
            int64_t s = pos[lv[i]]++;
            order[(size_t)q * n + s] = (int32_t)i;
            slot_up[(size_t)q * n + s] = vt.h_up[(size_t)q * n + i];
        }
        vt.max_levels = std::max(vt.max_levels, L);
    }
    if (!vt.d_up) RT_CUDA(cudaMalloc(&vt.d_up, slot_up.size() * sizeof(Upwind)));
    if (!vt.d_order) RT_CUDA(cudaMalloc(&vt.d_order, order.size() * sizeof(int32_t)));
    RT_CUDA(cudaMemcpyAsync(vt.d_up, slot_up.data(), slot_up.size() * sizeof(Upwind),
                            cudaMemcpyHostToDevice, st));
    RT_CUDA(cudaMemcpyAsync(vt.d_order, order.data(), order.size() * sizeof(int32_t),
                            cudaMemcpyHostToDevice, st));
    RT_CUDA(cudaStreamSynchronize(st));
    return RT_OK;
}

rt_status voronoi_dir_tables_cached(rt_grid *g, const double *dir, VorTables **out,
                                    cudaStream_t st)
{
    VorTables &vt = g->vt_one;
    if (!(vt.ndir == 1 && vt.dirs[0] == dir[0] && vt.dirs[1] == dir[1] && vt.dirs[2] == dir[2])) {
        rt_status s = voronoi_build_tables(g, 1, dir, vt, st);
        if (s != RT_OK) {
            vt.release();
            vt.ndir = 0;
            return s;
        }
    }
    *out = &vt;
    return RT_OK;
}

static rt_status build_voronoi(rt_grid *g, const rt_grid_desc *d, cudaStream_t st,
                               double r_exp)
{
    if (d->nsites < 1 || !d->xyz || !d->nbr_off || !d->nbr_idx)
        return fail(RT_EINVAL, "Voronoi grid needs nsites >= 1, xyz, nbr_off and nbr_idx");
    if (d->nsites > (int64_t)INT32_MAX / 2) return fail(RT_EINVAL, "too many sites");
    if (!(d->box[1] > d->box[0] && d->box[3] > d->box[2] && d->box[5] > d->box[4]))
        return fail(RT_EINVAL, "box must have positive extent");
    g->nsites = d->nsites;
    g->npt = d->nsites;
    g->r_exp = r_exp;
    g->xyz.assign(d->xyz, d->xyz + 3 * d->nsites);
    std::memcpy(g->box, d->box, sizeof(g->box));
    const int64_t n = g->nsites;
    if (d->nbr_off[0] != 0) return fail(RT_EINVAL, "nbr_off must start at 0");
    for (int64_t i = 0; i < n; ++i)
        if (d->nbr_off[i + 1] < d->nbr_off[i]) return fail(RT_EINVAL, "nbr_off not monotone");
    const int64_t ne = d->nbr_off[n];
    for (int64_t e = 0; e < ne; ++e) {
        int64_t c = d->nbr_idx[e];
        int64_t k = c >= 0 ? c : ((-c - 1) >> 1);
        if (k >= n) return fail(RT_EINVAL, "neighbour index out of range");
        if (d->nbr_shift && (d->nbr_shift[e] < 0 || d->nbr_shift[e] > 8))
            return fail(RT_EINVAL, "neighbour image shift out of range");
    }
    for (int64_t i = 0; i < n; ++i)
        for (int c = 0; c < 3; ++c) {
            double v = g->xyz[3 * i + c];
            if (!std::isfinite(v) || v < g->box[2 * c] || v > g->box[2 * c + 1])
                return fail(RT_EINVAL, "site outside the box");
        }
    g->nbr_off.assign(d->nbr_off, d->nbr_off + n + 1);
    g->nbr_idx.assign(d->nbr_idx, d->nbr_idx + ne);
    if (d->nbr_shift) g->nbr_shift.assign(d->nbr_shift, d->nbr_shift + ne);
    // the quadrature's upwind tables and levels: on the device (about 14 times faster at 400 000
    // sites), or on the host with RT_VORONOI_TABLES=host; both make identical choices
    const char *tenv = std::getenv("RT_VORONOI_TABLES");
    if (tenv && std::string(tenv) == "host")
        RT_TRY(voronoi_build_tables(g, g->ndir, g->dirs.data(), g->vt, st));
    else
        RT_TRY(voronoi_build_tables_device(g, st));
    g->max_levels = g->vt.max_levels;
    g->n_fallback = g->vt.n_fallback;
    // emergent layer: sites with a top-wall mirror among their neighbours
    for (int64_t i = 0; i < n; ++i)
        for (int64_t e = d->nbr_off[i]; e < d->nbr_off[i + 1]; ++e) {
            int32_t c = d->nbr_idx[e];
            if (c < 0 && ((-(int64_t)c - 1) & 1)) {
                g->top.push_back(i);
                break;
            }
        }
    return RT_OK;
}

}  // namespace rt

using namespace rt;

rt_grid::~rt_grid()
{
    if (d_stencil) cudaFree(d_stencil);
    if (d_stencil_one) cudaFree(d_stencil_one);
    if (d_stencil_oned) cudaFree(d_stencil_oned);
    if (d_wave_st) cudaFree(d_wave_st);
    face_release(face);
    map_release(map);
    if (d_up_site) cudaFree(d_up_site);
    if (self_batch) rt_batch_destroy(self_batch);
    vt.release();
    vt_one.release();
    if (d_top) cudaFree(d_top);
    if (d_err) cudaFree(d_err);
    for (auto &s : scratch)
        if (s.p) cudaFree(s.p);
}

extern "C" {

const char *rt_last_error(void) { return g_last_error.c_str(); }

unsigned long long rt_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

rt_status rt_grid_create(const rt_grid_desc *d, void *stream, rt_grid_t *out)
{
    return guarded([&]() -> rt_status {
        if (!d || !out) return fail(RT_EINVAL, "null argument");
        *out = nullptr;
        if (d->ndir < 1 || d->ndir > MAX_DIR || !d->dirs || !d->wdir)
            return fail(RT_EINVAL, "ndir must be 1..64 with dirs and wdir");
        // host-side validation first, before any device call
        if (d->kind == RT_GRID_REGULAR) {
            if (d->nx < 1 || d->ny < 1 || d->nz < 2 || !(d->dx > 0) || !(d->dy > 0) || !d->z)
                return fail(RT_EINVAL, "regular grid needs nx, ny >= 1, nz >= 2, dx, dy > 0 and z");
            for (int k = 1; k < d->nz; ++k)
                if (!(d->z[k] > d->z[k - 1])) return fail(RT_EINVAL, "z must be strictly ascending");
        } else if (d->kind == RT_GRID_VORONOI) {
            if (d->nsites < 1 || !d->xyz || !d->nbr_off || !d->nbr_idx)
                return fail(RT_EINVAL, "Voronoi grid needs nsites >= 1, xyz, nbr_off and nbr_idx");
            if (d->nsites > (int64_t)INT32_MAX / 2) return fail(RT_EINVAL, "too many sites");
            if (!(d->box[1] > d->box[0] && d->box[3] > d->box[2] && d->box[5] > d->box[4]))
                return fail(RT_EINVAL, "box must have positive extent");
            if (d->nbr_off[0] != 0) return fail(RT_EINVAL, "nbr_off must start at 0");
            for (int64_t i = 0; i < d->nsites; ++i)
                if (d->nbr_off[i + 1] < d->nbr_off[i]) return fail(RT_EINVAL, "nbr_off not monotone");
            for (int64_t e = 0; e < d->nbr_off[d->nsites]; ++e) {
                const int64_t c = d->nbr_idx[e];
                const int64_t k = c >= 0 ? c : ((-c - 1) >> 1);
                if (k >= d->nsites) return fail(RT_EINVAL, "neighbour index out of range");
                if (d->nbr_shift && (d->nbr_shift[e] < 0 || d->nbr_shift[e] > 8))
                    return fail(RT_EINVAL, "neighbour image shift out of range");
            }
            for (int64_t i = 0; i < d->nsites; ++i)
                for (int c = 0; c < 3; ++c) {
                    const double v = d->xyz[3 * i + c];
                    if (!std::isfinite(v) || v < d->box[2 * c] || v > d->box[2 * c + 1])
                        return fail(RT_EINVAL, "site outside the box");
                }
        } else {
            return fail(RT_EINVAL, "unknown grid kind");
        }
        for (int q = 0; q < d->ndir; ++q) {
            const double *u = d->dirs + 3 * q;
            const double nrm = std::sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
            if (!(std::fabs(nrm - 1.0) < 1e-6) || u[2] == 0.0 || !std::isfinite(d->wdir[q]))
                return fail(RT_EINVAL, "directions must be unit vectors with mu_z != 0");
        }
        cudaStream_t st = (cudaStream_t)stream;
        rt_grid *g = new (std::nothrow) rt_grid();
        if (!g) return fail(RT_ENOMEM, "host allocation failed");
        g->kind = d->kind;
        g->ndir = d->ndir;
        g->periodic = d->periodic_xy ? 1 : 0;
        g->dirs.assign(d->dirs, d->dirs + 3 * d->ndir);
        g->wdir.assign(d->wdir, d->wdir + d->ndir);
        rt_status s = RT_OK;
        for (int q = 0; q < g->ndir; ++q) {
            const double *u = &g->dirs[3 * q];
            double nrm = std::sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
            if (!(std::fabs(nrm - 1.0) < 1e-6) || u[2] == 0.0 || !std::isfinite(g->wdir[q])) {
                delete g;
                return fail(RT_EINVAL, "directions must be unit vectors with mu_z != 0");
            }
            (u[2] > 0 ? g->dir_up : g->dir_dn).push_back(q);
        }
        cudaError_t e = cudaGetDevice(&g->device);
        if (e == cudaSuccess) e = cudaMalloc(&g->d_err, sizeof(unsigned));
        if (e == cudaSuccess) e = cudaMemsetAsync(g->d_err, 0, sizeof(unsigned), st);
        if (e != cudaSuccess) {
            delete g;
            return cuda_fail(e, "grid device set-up");
        }
        double r_exp = d->r_exponent > 0 ? d->r_exponent : 7.0;
        if (d->kind == RT_GRID_REGULAR) s = build_regular(g, d, st);
        else if (d->kind == RT_GRID_VORONOI) s = build_voronoi(g, d, st, r_exp);
        else s = fail(RT_EINVAL, "unknown grid kind");
        if (s == RT_OK && !g->top.empty()) {
            e = cudaMalloc(&g->d_top, g->top.size() * sizeof(int64_t));
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(g->d_top, g->top.data(), g->top.size() * sizeof(int64_t),
                                    cudaMemcpyHostToDevice, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) s = cuda_fail(e, "grid upload");
        }
        if (s != RT_OK) {
            delete g;
            return s;
        }
        *out = g;
        return RT_OK;
    });
}

void rt_grid_destroy(rt_grid_t g) { delete g; }

rt_status rt_grid_info(rt_grid_t g, int64_t *npt, int64_t *ntop, int *max_levels,
                       int64_t *n_fallback)
{
    return guarded([&]() -> rt_status {
        if (!g) return fail(RT_EINVAL, "null grid");
        if (npt) *npt = g->npt;
        if (ntop) *ntop = (int64_t)g->top.size();
        if (max_levels) *max_levels = g->max_levels;
        if (n_fallback) *n_fallback = g->n_fallback;
        return RT_OK;
    });
}

rt_status rt_grid_tables(rt_grid_t g, int32_t *k, float *w, float *len, int32_t *level)
{
    return guarded([&]() -> rt_status {
        if (!g || g->kind != RT_GRID_VORONOI) return fail(RT_EINVAL, "Voronoi grid required");
        const size_t m = (size_t)g->ndir * g->nsites;
        for (size_t i = 0; i < m; ++i) {
            const Upwind &u = g->vt.h_up[i];
            if (k) { k[2 * i] = u.k1; k[2 * i + 1] = u.k2; }
            if (w) { w[2 * i] = u.w1; w[2 * i + 1] = 1.0f - u.w1; }
            if (len) { len[2 * i] = u.l1; len[2 * i + 1] = u.l2; }
            if (level) level[i] = g->vt.h_level[i];
        }
        return RT_OK;
    });
}

rt_status rt_grid_top_points(rt_grid_t g, int64_t *idx)
{
    return guarded([&]() -> rt_status {
        if (!g || !idx) return fail(RT_EINVAL, "null argument");
        std::copy(g->top.begin(), g->top.end(), idx);
        return RT_OK;
    });
}

rt_status rt_formal_solution(rt_grid_t g, int nlam, const float *alpha, const float *S, int bc,
                             const float *I_bc, float *J, float *I_dir, void *stream)
{
    return guarded([&]() -> rt_status {
        if (!g) return fail(RT_EINVAL, "null grid");
        if (nlam < 1 || !alpha || !S || !J) return fail(RT_EINVAL, "nlam >= 1, alpha, S, J required");
        if (bc < RT_BC_THERMAL || bc > RT_BC_ARRAY || (bc == RT_BC_ARRAY && !I_bc))
            return fail(RT_EINVAL, "bad boundary condition");
        if (!aligned16(alpha) || !aligned16(S) || !aligned16(J) || (I_dir && !aligned16(I_dir)) ||
            (I_bc && !aligned16(I_bc)))
            return fail(RT_EINVAL, "field pointers must be 16-byte aligned");
        cudaStream_t st = (cudaStream_t)stream;
        if (g->kind == RT_GRID_REGULAR)
            return regular_formal_solution(g, nlam, alpha, S, bc, I_bc, J, I_dir, st);
        return voronoi_formal_solution(g, nlam, alpha, S, bc, I_bc, J, I_dir, st);
    });
}

rt_status rt_emergent_intensity(rt_grid_t g, const double dir[3], int nlam, const float *alpha,
                                const float *S, int bc, float *I_top, void *stream)
{
    return guarded([&]() -> rt_status {
        if (!g || !dir || nlam < 1 || !alpha || !S || !I_top)
            return fail(RT_EINVAL, "null argument");
        if (!(dir[2] > 0)) return fail(RT_EINVAL, "the emergent direction needs mu_z > 0");
        if (bc != RT_BC_THERMAL && bc != RT_BC_ZERO) return fail(RT_EINVAL, "bc must be THERMAL or ZERO");
        if (!aligned16(alpha) || !aligned16(S) || !aligned16(I_top))
            return fail(RT_EINVAL, "field pointers must be 16-byte aligned");
        cudaStream_t st = (cudaStream_t)stream;
        if (g->kind == RT_GRID_REGULAR) return regular_emergent(g, dir, nlam, alpha, S, bc, I_top, st);
        return voronoi_emergent(g, dir, nlam, alpha, S, bc, I_top, st);
    });
}

size_t rt_adjoint_workspace_size(rt_grid_t g, int nlam, int stride)
{
    if (!g || nlam < 1 || stride < 1) return 0;
    if (g->kind == RT_GRID_REGULAR) return regular_adjoint_ws(g, nlam, stride);
    return voronoi_adjoint_ws(g, nlam, stride);
}

rt_status rt_formal_solution_adjoint(rt_grid_t g, const double dir[3], int nlam,
                                     const float *alpha, const float *S, int bc,
                                     const float *gI_top, float *g_alpha, float *g_S,
                                     int stride, void *ws, size_t ws_bytes, void *stream)
{
    return guarded([&]() -> rt_status {
        if (!g || !dir || nlam < 1 || !alpha || !S || !gI_top || !g_alpha || !g_S)
            return fail(RT_EINVAL, "null argument");
        if (!(dir[2] > 0)) return fail(RT_EINVAL, "the emergent direction needs mu_z > 0");
        if (bc != RT_BC_THERMAL && bc != RT_BC_ZERO) return fail(RT_EINVAL, "bc must be THERMAL or ZERO");
        if (stride < 1) return fail(RT_EINVAL, "ckpt_stride must be >= 1");
        if (!aligned16(alpha) || !aligned16(S) || !aligned16(gI_top) || !aligned16(g_alpha) ||
            !aligned16(g_S) || (ws && !aligned16(ws)))
            return fail(RT_EINVAL, "pointers must be 16-byte aligned");
        size_t need = rt_adjoint_workspace_size(g, nlam, stride);
        if (!ws || ws_bytes < need) return fail(RT_EINVAL, "workspace too small");
        cudaStream_t st = (cudaStream_t)stream;
        if (g->kind == RT_GRID_REGULAR)
            return regular_adjoint(g, dir, nlam, alpha, S, bc, gI_top, g_alpha, g_S, stride, ws,
                                   ws_bytes, st);
        return voronoi_adjoint(g, dir, nlam, alpha, S, bc, gI_top, g_alpha, g_S, stride, ws, ws_bytes,
                               st);
    });
}

}  // extern "C"
