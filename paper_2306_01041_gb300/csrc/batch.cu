// Batched persistent sweep over several Voronoi grids of uneven size.
//
// Work item = (grid, direction, wavelength chunk).  A block takes an item from a device queue and
// sweeps the levels of that direction for its wavelengths, with one __syncthreads between levels;
// each direction writes its own intensity array, so the 24 directions of a grid run concurrently
// and the dependent chain of an item is one direction's levels, not all 24 of them.  J is then
// formed by a reduction over the directions in index order (the same order and arithmetic as the
// per-direction launches, so the results are identical).  No block ever waits for another: no
// co-residency requirement and no device-side spin.  The grid is sized to the number of blocks
// that fit at once (persistent) and items are queued largest first.
//
// Layout: site-major rows of P = nc cs wavelengths (the atom's, padded to whole chunks), cut into
// chunks of cs (a multiple of 8) at offsets c cs: a chunk of a site fills whole 32-byte sectors,
// so an upwind gather reads only the sectors it uses, and the items of the other chunks of the
// same direction, which sweep the same sites at about the same time, read the same lines.
// A thread keeps one wavelength lane (tid % cs) for a whole item and steps through the level's
// sites, three at a time so that three independent gather chains are in flight.
#include <algorithm>
#include <cstdlib>
#include <cmath>
#include <numeric>

#include "device_common.cuh"
#include "rt_impl.h"

namespace rt {

// Sites are renumbered inside the batch along a space-filling (Morton) curve, so that sites close
// in space are close in memory, and each level's slots hold its sites in that order: the sites a
// warp updates together, and their upwind neighbours, close to them in space, lie in nearby lines
// (measured on the 8-atmosphere batch: 107 G updates/s against 98 in the grids' own numbering,
// whose sites come in sampling order).  perm maps a grid's site index to the batch's.
struct BatchGridDev {
    const Upwind *up;          // [ndir][n] slot order, neighbours in the batch's numbering
    const int32_t *order;      // [ndir][n]: the batch's index of the site each slot holds
    const int32_t *perm;       // [n]: grid site index -> batch index
    const int64_t *lvl;        // level offsets, all directions concatenated
    const int32_t *lvl_base;   // [ndir + 1] start of each direction's offsets in lvl
    const float2 *SA;          // (S, alpha) of (chunk c, site p, lane j) at c cstr + p ss + j
    float *I;                  // [ndir] blocks of n P floats, the same layout per direction
    int n, cs, nc, P;          // P = nc cs
    int ss, cstr;              // site and chunk strides: rows of P per site (ss = P, cstr = cs)
};

// Floats of one grid's field block (the pairs, one I per direction), rounded up to 64 floats so
// that every grid's block starts on a 256-byte boundary.
static inline size_t batch_grid_floats(int64_t nsites, int P, int ndir)
{
    const size_t m = (size_t)nsites * P;
    return ((2 + (size_t)ndir) * m + 63) & ~(size_t)63;
}

// Interleaves the low 21 bits of v with two zero bits between each (Morton code of one axis).
static inline uint64_t morton_spread(uint64_t v)
{
    v &= 0x1fffff;
    v = (v | v << 32) & 0x1f00000000ffffull;
    v = (v | v << 16) & 0x1f0000ff0000ffull;
    v = (v | v << 8) & 0x100f00f00f00f00full;
    v = (v | v << 4) & 0x10c30c30c30c30c3ull;
    v = (v | v << 2) & 0x1249249249249249ull;
    return v;
}

// The batch's tables of one grid: perm (Morton order of the sites in the box), and per direction
// the slots of each level sorted by the batch index, with the upwind neighbours renumbered.  The
// level offsets are the grid's (a level keeps its sites).
static void batch_locality_tables(const rt_grid *g, std::vector<int32_t> &perm,
                                  std::vector<Upwind> &up, std::vector<int32_t> &order)
{
    const int64_t n = g->nsites;
    const int nd = g->ndir;
    std::vector<uint64_t> key((size_t)n);
    for (int64_t i = 0; i < n; ++i) {
        uint64_t c[3];
        for (int a = 0; a < 3; ++a) {
            const double lo = g->box[2 * a], hi = g->box[2 * a + 1];
            double t = (g->xyz[3 * i + a] - lo) / (hi - lo);
            t = std::min(1.0, std::max(0.0, t));
            c[a] = (uint64_t)(t * 2097151.0);
        }
        key[i] = morton_spread(c[0]) | morton_spread(c[1]) << 1 | morton_spread(c[2]) << 2;
    }
    std::vector<int32_t> idx((size_t)n);
    std::iota(idx.begin(), idx.end(), 0);
    std::stable_sort(idx.begin(), idx.end(), [&](int32_t x, int32_t y) { return key[x] < key[y]; });
    perm.assign((size_t)n, 0);
    for (int64_t r = 0; r < n; ++r) perm[idx[r]] = (int32_t)r;
    up.assign((size_t)nd * n, Upwind{});
    order.assign((size_t)nd * n, 0);
#pragma omp parallel for schedule(dynamic, 1)
    for (int d = 0; d < nd; ++d) {
        const int32_t *lev = g->vt.h_level.data() + (size_t)d * n;
        const Upwind *hu = g->vt.h_up.data() + (size_t)d * n;
        std::vector<uint64_t> k((size_t)n);
        for (int64_t i = 0; i < n; ++i) k[i] = (uint64_t)(uint32_t)lev[i] << 32 | (uint32_t)perm[i];
        std::sort(k.begin(), k.end());
        for (int64_t s = 0; s < n; ++s) {
            const int32_t p = (int32_t)(k[s] & 0xffffffffu);
            const int32_t i = idx[p];
            Upwind u = hu[i];
            if (u.k1 >= 0) u.k1 = perm[u.k1];
            if (u.k2 >= 0) u.k2 = perm[u.k2];
            up[(size_t)d * n + s] = u;
            order[(size_t)d * n + s] = p;
        }
    }
}

struct BatchItem {
    int grid, dir, chunk, lcv;   // lcv: valid wavelengths of the chunk (the last may be short)
};

struct BatchArgs {
    const BatchGridDev *grids;
    const BatchItem *items;
    int *queue;
    const float *wdir;         // [ndir]
    const float *up_flag;      // [ndir] 1 for mu_z > 0
    unsigned *err;
    int nitems, ndir, nlam, bc;
};

// The loads of one (site, wavelength) update: the site's own (S, alpha) and, per upwind line, the
// upwind intensity and (S, alpha).  SA and I point at the item's chunk (a site's lanes ss apart
// from the next site's), j is the thread's wavelength lane.
struct VorGather {
    float Si, Ai, I1, S1, A1, I2, S2, A2;
};

__device__ __forceinline__ VorGather vor_gather(const float2 *SA, const float *I, const Upwind &u,
                                                int i, int j, int ss, float inflow_scale)
{
    VorGather r;
    const float2 own = __ldg(SA + (size_t)i * ss + j);
    r.Si = own.x;
    r.Ai = own.y;
    // a wall neighbour (k < 0) takes the site's own S and alpha; -1 (inflow wall of the sweep)
    // brings the boundary intensity S * inflow_scale (1 thermal, 0 otherwise), -2 zero
    if (u.k1 >= 0) {
        const size_t kl = (size_t)u.k1 * ss + j;
        r.I1 = I[kl];
        const float2 sa = __ldg(SA + kl);
        r.S1 = sa.x;
        r.A1 = sa.y;
    } else {
        r.S1 = r.Si;
        r.A1 = r.Ai;
        r.I1 = u.k1 == -1 ? r.Si * inflow_scale : 0.f;
    }
    if (u.k2 >= 0 && u.w1 != 1.f) {
        const size_t kl = (size_t)u.k2 * ss + j;
        r.I2 = I[kl];
        const float2 sa = __ldg(SA + kl);
        r.S2 = sa.x;
        r.A2 = sa.y;
    } else {
        r.S2 = r.Si;
        r.A2 = r.Ai;
        r.I2 = u.k2 == -1 ? r.Si * inflow_scale : 0.f;
    }
    return r;
}

__device__ __forceinline__ float vor_update(const Upwind &u, const VorGather &r)
{
    float acc = 0.f;
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        const float wk = c ? 1.f - u.w1 : u.w1;
        if (wk == 0.f) continue;
        const float len = c ? u.l2 : u.l1;
        const float Ik = c ? r.I2 : r.I1, Sk = c ? r.S2 : r.S1, Ak = c ? r.A2 : r.A1;
        float ex, w0, w1;
        lin_weights(0.5f * (Ak + r.Ai) * len, ex, w0, w1);
        acc += wk * (Ik * ex + w0 * Sk + w1 * r.Si);
    }
    return acc;
}

// U: updates a thread keeps in flight (sites of the level U steps apart, independent gathers);
// measured on the 8-atmosphere batch: 2 -> 93.6, 3 -> 98.1, 4 -> 62.0 G updates/s (4 spills
// registers at two blocks of 512 threads per SM); loading the next iteration's upwind records
// ahead (which leaves room for only 2 in flight) measured 96.1 against 107.3 for 3 without.
constexpr int BATCH_INFLIGHT = 3;
template <int U>
__global__ void __launch_bounds__(512, 2) batch_sweep_kernel(const BatchArgs a)
{
    __shared__ int item_s;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) item_s = atomicAdd(a.queue, 1);
        __syncthreads();
        const int it = item_s;
        if (it >= a.nitems) return;
        const BatchItem item = a.items[it];
        const BatchGridDev g = a.grids[item.grid];
        const int d = item.dir, cs = g.cs;
        const Upwind *up = g.up + (size_t)d * g.n;
        const int32_t *order = g.order + (size_t)d * g.n;
        // this item's chunk of (S, alpha) and of the direction's intensity
        const float2 *SA = g.SA + (size_t)item.chunk * g.cstr;
        float *I = g.I + (size_t)d * g.n * g.P + (size_t)item.chunk * g.cstr;
        const int ss = g.ss;
        const int b0 = g.lvl_base[d], b1 = g.lvl_base[d + 1];
        const float inflow = (a.bc == RT_BC_THERMAL && a.up_flag[d] > 0.f) ? 1.f : 0.f;
        // this thread's wavelength lane and first slot offset, fixed for the item; the threads
        // beyond the last whole group of cs lanes, and the lanes past the chunk's end, sit out
        const int step = blockDim.x / cs;
        const int j = threadIdx.x % cs, soff = threadIdx.x / cs;
        const bool active = soff < step && j < item.lcv;
        for (int L = b0; L + 1 < b1; ++L) {
            const int64_t s1 = g.lvl[L + 1];
            if (active) {
                for (int64_t s = g.lvl[L] + soff; s < s1; s += U * step) {
                    Upwind u[U];
                    int i[U];
                    bool v[U];
#pragma unroll
                    for (int q = 0; q < U; ++q) {
                        const int64_t sq = s + (int64_t)q * step;
                        v[q] = sq < s1;
                        u[q] = up[v[q] ? sq : s];
                        i[q] = order[v[q] ? sq : s];
                    }
                    VorGather gq[U];
#pragma unroll
                    for (int q = 0; q < U; ++q) gq[q] = vor_gather(SA, I, u[q], i[q], j, ss, inflow);
#pragma unroll
                    for (int q = 0; q < U; ++q)
                        if (v[q]) I[(size_t)i[q] * ss + j] = vor_update(u[q], gq[q]);
                }
            }
            __syncthreads();
        }
    }
}

// J[l][i] = sum_d w_d I_d, directions in index order, for 32 sites (in the grid's numbering) per
// block: the sums are formed along each site's rows (32-byte pieces per chunk) and written
// wavelength-major through a shared tile.
__global__ void batch_reduce_kernel(const float *__restrict__ I, float *__restrict__ J,
                                    const float *__restrict__ wdir, const int32_t *__restrict__ perm,
                                    int ndir, int n, int cs, int nc, int ss, int cstr, int nlam,
                                    unsigned *err)
{
    __shared__ float tile[128][33];
    const int i0 = blockIdx.x * 32, P = nc * cs;
    const size_t dstride = (size_t)n * P;
    for (int e = threadIdx.x; e < 32 * P; e += blockDim.x) {
        const int il = e / P, l = e % P, i = i0 + il;
        if (i >= n || l >= nlam) continue;
        const size_t q = (size_t)(l / cs) * cstr + (size_t)perm[i] * ss + l % cs;
        float acc = wdir[0] * I[q];
        for (int d = 1; d < ndir; ++d) acc = acc + wdir[d] * I[(size_t)d * dstride + q];
        if (!isfinite(acc)) flag_error(err, ERR_NAN);
        tile[l][il] = acc;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < 32 * nlam; e += blockDim.x) {
        const int l = e / 32, il = e % 32, i = i0 + il;
        if (i < n) J[(size_t)l * n + i] = tile[l][il];
    }
}

// S, alpha [nlam][n] -> the (S, alpha) rows [nc][n][cs] in the batch's numbering, 32 sites per
// block; the padding lanes are zero (never read).
__global__ void batch_pack_kernel(const float *__restrict__ S, const float *__restrict__ A,
                                  float2 *__restrict__ SA, const int32_t *__restrict__ perm, int n,
                                  int cs, int nc, int ss, int cstr, int nlam)
{
    __shared__ float ts[128][33], ta[128][33];
    const int i0 = blockIdx.x * 32, P = nc * cs;
    for (int e = threadIdx.x; e < 32 * nlam; e += blockDim.x) {
        const int l = e / 32, il = e % 32, i = i0 + il;
        if (i < n) {
            const size_t q = (size_t)l * n + i;
            ts[l][il] = S[q];
            ta[l][il] = A[q];
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < 32 * P; e += blockDim.x) {
        const int il = e / P, l = e % P, i = i0 + il;
        if (i >= n) continue;
        SA[(size_t)(l / cs) * cstr + (size_t)perm[i] * ss + l % cs] =
            l < nlam ? make_float2(ts[l][il], ta[l][il]) : make_float2(0.f, 0.f);
    }
}

}  // namespace rt

using namespace rt;

struct rt_batch {
    std::vector<rt_grid *> grids;
    int nlam = 0, ndir = 0, threads = 512, blocks = 0;
    std::vector<BatchItem> h_items;
    BatchItem *d_items = nullptr;
    BatchGridDev *d_grids = nullptr;
    std::vector<BatchGridDev> h_grids;
    int64_t *d_lvl = nullptr;
    int32_t *d_lvl_base = nullptr;
    float *d_wdir = nullptr, *d_upf = nullptr;
    float *d_fields = nullptr;   // per grid (S, alpha) [nc][n][cs] and I [ndir][nc][n][cs]
    std::vector<void *> d_tables;   // per grid: the batch's upwind records, slot order, perm
    int *d_queue = nullptr;
    unsigned *d_err = nullptr;
    unsigned *err = nullptr;     // where kernels flag errors: d_err, or the grid's for a batch of one
    ~rt_batch()
    {
        cudaFree(d_items);
        cudaFree(d_grids);
        cudaFree(d_lvl);
        cudaFree(d_lvl_base);
        cudaFree(d_wdir);
        cudaFree(d_upf);
        cudaFree(d_fields);
        cudaFree(d_queue);
        cudaFree(d_err);
        for (void *p : d_tables) cudaFree(p);
    }
};

namespace rt {

int batch_ngrids(const rt_batch *b) { return (int)b->grids.size(); }
rt_grid *batch_grid(const rt_batch *b, int i) { return b->grids[i]; }
int batch_nlam(const rt_batch *b) { return b->nlam; }

rt_status batch_check_error(rt_batch *b, cudaStream_t st)
{
    unsigned h = 0;
    RT_CUDA(cudaMemcpyAsync(&h, b->err, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    RT_CUDA(cudaStreamSynchronize(st));
    if (h) {
        RT_CUDA(cudaMemsetAsync(b->err, 0, sizeof(unsigned), st));
        if (h & ERR_NAN) return fail(RT_ENAN, "a non-finite value was produced on the device");
        return fail(RT_EINVAL, "a device-side check failed in the batched sweep");
    }
    return RT_OK;
}

}  // namespace rt

extern "C" {

rt_status rt_batch_create(const rt_grid_t *grids, int ngrids, int nlam, const int *lam_chunk,
                          int threads, rt_batch_t *out)
{
    return guarded([&]() -> rt_status {
        if (!grids || ngrids < 1 || nlam < 1 || !out) return fail(RT_EINVAL, "bad argument");
        *out = nullptr;
        rt_batch *b = new (std::nothrow) rt_batch();
        if (!b) return fail(RT_ENOMEM, "host allocation failed");
        b->nlam = nlam;
        b->ndir = grids[0]->ndir;
        b->threads = threads > 0 ? threads : 512;
        if (b->threads > 512 || b->threads % 32) {
            delete b;
            return fail(RT_EINVAL, "threads must be a multiple of 32 up to 512");
        }

        for (int i = 0; i < ngrids; ++i) {
            rt_grid *g = grids[i];
            if (!g || g->kind != RT_GRID_VORONOI || g->ndir != b->ndir) {
                delete b;
                return fail(RT_EINVAL, "batch grids must be Voronoi grids with the same directions");
            }
            for (int d = 0; d < g->ndir; ++d)
                if (g->wdir[d] != grids[0]->wdir[d] || g->dirs[3 * d + 2] != grids[0]->dirs[3 * d + 2]) {
                    delete b;
                    return fail(RT_EINVAL, "batch grids must share the quadrature");
                }
            b->grids.push_back(g);
        }
        int dev = 0, nsm = 0, per_sm = 0;
        RT_CUDA(cudaGetDevice(&dev));
        RT_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
        RT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_sweep_kernel<BATCH_INFLIGHT>,
                                                              b->threads, 0));
        if (per_sm < 1) {
            delete b;
            return fail(RT_ECAPACITY, "the batched sweep kernel cannot be resident");
        }
        b->blocks = nsm * per_sm;
        if (nlam > 128) {
            delete b;
            return fail(RT_EINVAL, "the batched sweep takes at most 128 wavelengths");
        }
        // chunks: the requested wavelength count per item, rounded up to a multiple of 8 floats
        // (the chunk stride cs): a chunk of a site fills whole 32-byte sectors.  Default 8: the
        // smallest sector-exact chunk gives the most items (the parallelism of the launch) and
        // measured fastest both for one grid and for the 8-atmosphere batch.
        const int nlam8 = (nlam + 7) & ~7;
        std::vector<int> cs(ngrids), nc(ngrids);
        for (int i = 0; i < ngrids; ++i) {
            int lc = lam_chunk ? lam_chunk[i] : 8;
            lc = std::max(1, std::min(nlam, lc));
            cs[i] = std::min(std::min(nlam8, (lc + 7) & ~7), b->threads & ~7);
            nc[i] = (nlam + cs[i] - 1) / cs[i];
            for (int d = 0; d < b->ndir; ++d)
                for (int c = 0; c < nc[i]; ++c)
                    b->h_items.push_back(BatchItem{i, d, c, std::min(cs[i], nlam - c * cs[i])});
        }
        std::stable_sort(b->h_items.begin(), b->h_items.end(), [&](const BatchItem &x, const BatchItem &y) {
            return (double)grids[x.grid]->nsites * x.lcv > (double)grids[y.grid]->nsites * y.lcv;
        });
        // device tables
        std::vector<int64_t> lvl;
        std::vector<int32_t> base;
        std::vector<size_t> base_at(ngrids);
        for (int i = 0; i < ngrids; ++i) {
            base_at[i] = base.size();
            for (int d = 0; d < b->ndir; ++d) {
                base.push_back((int32_t)lvl.size());
                const auto &o = grids[i]->vt.lvl_off[d];
                lvl.insert(lvl.end(), o.begin(), o.end());
            }
            base.push_back((int32_t)lvl.size());
        }
        size_t fsz = 0;
        std::vector<int> P(ngrids);
        for (int i = 0; i < ngrids; ++i) {
            P[i] = nc[i] * cs[i];
            fsz += batch_grid_floats(grids[i]->nsites, P[i], b->ndir);
        }
        std::vector<float> wd(b->ndir), uf(b->ndir);
        for (int d = 0; d < b->ndir; ++d) {
            wd[d] = (float)grids[0]->wdir[d];
            uf[d] = grids[0]->dirs[3 * d + 2] > 0 ? 1.f : 0.f;
        }
        cudaError_t e = cudaSuccess;
    #define BT(x)                                                   \
        do {                                                        \
            if (e == cudaSuccess) e = (x);                          \
        } while (0)
        BT(cudaMalloc(&b->d_items, b->h_items.size() * sizeof(BatchItem)));
        BT(cudaMalloc(&b->d_grids, ngrids * sizeof(BatchGridDev)));
        BT(cudaMalloc(&b->d_lvl, lvl.size() * sizeof(int64_t)));
        BT(cudaMalloc(&b->d_lvl_base, base.size() * sizeof(int32_t)));
        BT(cudaMalloc(&b->d_wdir, b->ndir * sizeof(float)));
        BT(cudaMalloc(&b->d_upf, b->ndir * sizeof(float)));
        BT(cudaMalloc(&b->d_fields, fsz * sizeof(float)));
        BT(cudaMalloc(&b->d_queue, sizeof(int)));
        BT(cudaMalloc(&b->d_err, sizeof(unsigned)));
        if (e != cudaSuccess) {
            delete b;
            return cuda_fail(e, "batch allocation");
        }
        float *f = b->d_fields;
        for (int i = 0; i < ngrids; ++i) {
            rt_grid *g = grids[i];
            const size_t m = (size_t)g->nsites * P[i];
            std::vector<int32_t> perm, order;
            std::vector<Upwind> up;
            if (g->vt.h_up.size() != (size_t)b->ndir * g->nsites ||
                g->vt.h_level.size() != (size_t)b->ndir * g->nsites) {
                delete b;
                return fail(RT_EINVAL, "a batch grid has no host copy of its upwind tables");
            }
            batch_locality_tables(g, perm, up, order);
            void *tu = nullptr, *to = nullptr, *tp = nullptr;
            BT(cudaMalloc(&tu, up.size() * sizeof(Upwind)));
            if (tu) b->d_tables.push_back(tu);
            BT(cudaMalloc(&to, order.size() * sizeof(int32_t)));
            if (to) b->d_tables.push_back(to);
            BT(cudaMalloc(&tp, perm.size() * sizeof(int32_t)));
            if (tp) b->d_tables.push_back(tp);
            BT(cudaMemcpy(tu, up.data(), up.size() * sizeof(Upwind), cudaMemcpyHostToDevice));
            BT(cudaMemcpy(to, order.data(), order.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
            BT(cudaMemcpy(tp, perm.data(), perm.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
            if (e != cudaSuccess) {
                delete b;
                return cuda_fail(e, "batch tables");
            }
            BatchGridDev gd;
            gd.up = static_cast<const Upwind *>(tu);
            gd.order = static_cast<const int32_t *>(to);
            gd.perm = static_cast<const int32_t *>(tp);
            gd.lvl = b->d_lvl;
            gd.lvl_base = b->d_lvl_base + base_at[i];
            gd.SA = reinterpret_cast<const float2 *>(f);
            gd.I = f + 2 * m;
            gd.n = (int)g->nsites;
            gd.cs = cs[i];
            gd.nc = nc[i];
            gd.P = P[i];
            // site-major rows: the concurrent chunk items of a direction share each site's
            // lines (measured on the 8-atmosphere batch: 107 G updates/s against 90 with the
            // chunks in separate slabs)
            gd.ss = P[i];
            gd.cstr = cs[i];
            f += batch_grid_floats(g->nsites, P[i], b->ndir);
            b->h_grids.push_back(gd);
        }
        BT(cudaMemcpy(b->d_items, b->h_items.data(), b->h_items.size() * sizeof(BatchItem),
                      cudaMemcpyHostToDevice));
        BT(cudaMemcpy(b->d_grids, b->h_grids.data(), ngrids * sizeof(BatchGridDev),
                      cudaMemcpyHostToDevice));
        BT(cudaMemcpy(b->d_lvl, lvl.data(), lvl.size() * sizeof(int64_t), cudaMemcpyHostToDevice));
        BT(cudaMemcpy(b->d_lvl_base, base.data(), base.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
        BT(cudaMemcpy(b->d_wdir, wd.data(), b->ndir * sizeof(float), cudaMemcpyHostToDevice));
        BT(cudaMemcpy(b->d_upf, uf.data(), b->ndir * sizeof(float), cudaMemcpyHostToDevice));
        BT(cudaMemset(b->d_err, 0, sizeof(unsigned)));
        b->err = ngrids == 1 ? grids[0]->d_err : b->d_err;
    #undef BT
        if (e != cudaSuccess) {
            delete b;
            return cuda_fail(e, "batch upload");
        }
        *out = b;
        return RT_OK;
    });
}

void rt_batch_destroy(rt_batch_t b) { delete b; }

rt_status rt_batch_formal_solution(rt_batch_t b, const float *const *alpha, const float *const *S,
                                   int bc, float *const *J, void *stream)
{
    return guarded([&]() -> rt_status {
        if (!b || !alpha || !S || !J) return fail(RT_EINVAL, "null argument");
        if (bc != RT_BC_THERMAL && bc != RT_BC_ZERO) return fail(RT_EINVAL, "bc must be THERMAL or ZERO");
        cudaStream_t st = (cudaStream_t)stream;
        const int ng = (int)b->grids.size();
        for (int i = 0; i < ng; ++i) {
            if (!alpha[i] || !S[i] || !J[i]) return fail(RT_EINVAL, "null field");
            const BatchGridDev &g = b->h_grids[i];
            note_launch();
            batch_pack_kernel<<<(unsigned)((g.n + 31) / 32), 256, 0, st>>>(
                S[i], alpha[i], const_cast<float2 *>(g.SA), g.perm, g.n, g.cs, g.nc, g.ss, g.cstr,
                b->nlam);
        }
        RT_CUDA(cudaMemsetAsync(b->d_queue, 0, sizeof(int), st));
        BatchArgs a;
        a.grids = b->d_grids;
        a.items = b->d_items;
        a.queue = b->d_queue;
        a.wdir = b->d_wdir;
        a.up_flag = b->d_upf;
        a.err = b->err;
        a.nitems = (int)b->h_items.size();
        a.ndir = b->ndir;
        a.nlam = b->nlam;
        a.bc = bc;
        const int blocks = std::min<int>(b->blocks, a.nitems);
        note_launch();
        batch_sweep_kernel<BATCH_INFLIGHT><<<blocks, b->threads, 0, st>>>(a);
        for (int i = 0; i < ng; ++i) {
            const BatchGridDev &g = b->h_grids[i];
            note_launch();
            batch_reduce_kernel<<<(unsigned)((g.n + 31) / 32), 256, 0, st>>>(
                g.I, J[i], b->d_wdir, g.perm, b->ndir, g.n, g.cs, g.nc, g.ss, g.cstr, b->nlam,
                b->err);
        }
        RT_CUDA(cudaGetLastError());
        return RT_OK;
    });
}

}  // extern "C"
