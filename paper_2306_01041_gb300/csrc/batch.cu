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
#include <cmath>
#include <numeric>

#include "device_common.cuh"
#include "rt_impl.h"

namespace rt {

struct BatchGridDev {
    const Upwind *up;          // [ndir][n] slot order
    const int32_t *order;      // [ndir][n]
    const int64_t *lvl;        // level offsets, all directions concatenated
    const int32_t *lvl_base;   // [ndir + 1] start of each direction's offsets in lvl
    const float2 *SA;          // [n][P] (S, alpha): the two are always gathered together
    float *I;                  // [ndir][n][P] one intensity array per direction
    int n, cs, nc, P;          // P = nc cs
};

// Floats of one grid's field block (the pairs, one I per direction), rounded up to 64 floats so
// that every grid's block starts on a 256-byte boundary.
static inline size_t batch_grid_floats(int64_t nsites, int P, int ndir)
{
    const size_t m = (size_t)nsites * P;
    return ((2 + (size_t)ndir) * m + 63) & ~(size_t)63;
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
// upwind intensity and (S, alpha).  c0 is the chunk's offset in a row (c cs) plus the lane.
struct VorGather {
    float Si, Ai, I1, S1, A1, I2, S2, A2;
};

__device__ __forceinline__ VorGather vor_gather(const BatchGridDev &g, const float *I, const Upwind &u,
                                                int i, size_t c0, int P, float inflow_scale)
{
    VorGather r;
    const float2 own = __ldg(g.SA + c0 + (size_t)i * P);
    r.Si = own.x;
    r.Ai = own.y;
    // a wall neighbour (k < 0) takes the site's own S and alpha; -1 (inflow wall of the sweep)
    // brings the boundary intensity S * inflow_scale (1 thermal, 0 otherwise), -2 zero
    if (u.k1 >= 0) {
        const size_t kl = c0 + (size_t)u.k1 * P;
        r.I1 = I[kl];
        const float2 sa = __ldg(g.SA + kl);
        r.S1 = sa.x;
        r.A1 = sa.y;
    } else {
        r.S1 = r.Si;
        r.A1 = r.Ai;
        r.I1 = u.k1 == -1 ? r.Si * inflow_scale : 0.f;
    }
    if (u.k2 >= 0 && u.w1 != 1.f) {
        const size_t kl = c0 + (size_t)u.k2 * P;
        r.I2 = I[kl];
        const float2 sa = __ldg(g.SA + kl);
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
// registers at two blocks of 512 threads per SM).
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
        float *I = g.I + (size_t)d * g.n * g.P;
        const int b0 = g.lvl_base[d], b1 = g.lvl_base[d + 1];
        const float inflow = (a.bc == RT_BC_THERMAL && a.up_flag[d] > 0.f) ? 1.f : 0.f;
        // this thread's wavelength lane and first slot offset, fixed for the item; the threads
        // beyond the last whole group of cs lanes, and the lanes past the chunk's end, sit out
        const int step = blockDim.x / cs;
        const int j = threadIdx.x % cs, soff = threadIdx.x / cs;
        const bool active = soff < step && j < item.lcv;
        const size_t c0 = (size_t)item.chunk * cs + j;
        const int P = g.P;
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
                    for (int q = 0; q < U; ++q) gq[q] = vor_gather(g, I, u[q], i[q], c0, P, inflow);
#pragma unroll
                    for (int q = 0; q < U; ++q)
                        if (v[q]) I[c0 + (size_t)i[q] * P] = vor_update(u[q], gq[q]);
                }
            }
            __syncthreads();
        }
    }
}

// J[l][i] = sum_d w_d I_d, directions in index order, for 32 sites per block: the sums are formed
// along the sites' rows (coalesced reads) and written wavelength-major through a shared tile.
__global__ void batch_reduce_kernel(const float *__restrict__ I, float *__restrict__ J,
                                    const float *__restrict__ wdir, int ndir, int n, int P,
                                    int nlam, unsigned *err)
{
    __shared__ float tile[128][33];
    const int i0 = blockIdx.x * 32;
    const size_t dstride = (size_t)n * P;
    for (int e = threadIdx.x; e < 32 * P; e += blockDim.x) {
        const int il = e / P, l = e % P, i = i0 + il;
        if (i >= n || l >= nlam) continue;
        const size_t q = (size_t)i * P + l;
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

// S, alpha [nlam][n] -> the (S, alpha) rows [n][P], 32 sites per block; the padding lanes are zero
// (never read).
__global__ void batch_pack_kernel(const float *__restrict__ S, const float *__restrict__ A,
                                  float2 *__restrict__ SA, int n, int P, int nlam)
{
    __shared__ float ts[128][33], ta[128][33];
    const int i0 = blockIdx.x * 32;
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
        SA[(size_t)i * P + l] = l < nlam ? make_float2(ts[l][il], ta[l][il]) : make_float2(0.f, 0.f);
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
    float *d_fields = nullptr;   // per grid (S, alpha) [n][P] and I [ndir][n][P]
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
            BatchGridDev gd;
            gd.up = g->vt.d_up;
            gd.order = g->vt.d_order;
            gd.lvl = b->d_lvl;
            gd.lvl_base = b->d_lvl_base + base_at[i];
            gd.SA = reinterpret_cast<const float2 *>(f);
            gd.I = f + 2 * m;
            gd.n = (int)g->nsites;
            gd.cs = cs[i];
            gd.nc = nc[i];
            gd.P = P[i];
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
                S[i], alpha[i], const_cast<float2 *>(g.SA), g.n, g.P, b->nlam);
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
                g.I, J[i], b->d_wdir, b->ndir, g.n, g.P, b->nlam, b->err);
        }
        RT_CUDA(cudaGetLastError());
        return RT_OK;
    });
}

}  // extern "C"
