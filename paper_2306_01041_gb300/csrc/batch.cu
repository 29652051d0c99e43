// Batched persistent sweep over several Voronoi grids of uneven size.
//
// Work item = (grid, direction, wavelength chunk).  A block takes an item from a device queue and
// sweeps the levels of that direction for its wavelengths, with one __syncthreads between levels;
// each direction writes its own intensity array, so the 24 directions of a grid run concurrently
// and the dependent chain of an item is one direction's levels, not all 24 of them.  J is then
// formed by a reduction over the directions in index order (the same order and arithmetic as the
// per-direction launches, so the results are identical).  No block ever waits for another: no
// co-residency requirement and no device-side spin.  The grid is sized to the number of blocks
// that fit at once (persistent) and items are queued largest first; chunk sizes per grid balance
// the items' work (sites x chunk).
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
    const float2 *SA;          // [n][nlam] (S, alpha): the two are always gathered together
    float *I;                  // [ndir][n][nlam] one intensity array per direction
    float *J;                  // [n][nlam]
    int n;
};

// Floats of one grid's field block: (S, alpha) pairs, J, one I per direction; rounded up to an
// even count so that the next grid's pairs stay 8-byte aligned.
static inline size_t batch_grid_floats(int64_t nsites, int nlam, int ndir)
{
    const size_t m = (size_t)nsites * nlam;
    return ((3 + (size_t)ndir) * m + 1) & ~(size_t)1;
}

struct BatchItem {
    int grid, dir, c0, lc;
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

// One (site, wavelength) update of a level, split into its loads (gather) and its arithmetic, so
// that a thread can have the loads of one update in flight with the table loads of the next.
struct VorGather {
    float Si, Ai, I1, S1, A1, I2, S2, A2;
};

__device__ __forceinline__ VorGather vor_gather(const BatchGridDev &g, const float *I, const Upwind &u,
                                                int i, int l, int nlam, float inflow_scale)
{
    VorGather r;
    const size_t il = (size_t)i * nlam + l;
    const float2 own = __ldg(g.SA + il);
    r.Si = own.x;
    r.Ai = own.y;
    // a wall neighbour (k < 0) takes the site's own S and alpha; -1 (inflow wall of the sweep)
    // brings the boundary intensity S * inflow_scale (1 thermal, 0 otherwise), -2 zero
    if (u.k1 >= 0) {
        const size_t kl = (size_t)u.k1 * nlam + l;
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
        const size_t kl = (size_t)u.k2 * nlam + l;
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
        const int d = item.dir;
        const Upwind *up = g.up + (size_t)d * g.n;
        const int32_t *order = g.order + (size_t)d * g.n;
        float *I = g.I + (size_t)d * g.n * a.nlam;
        const int b0 = g.lvl_base[d], b1 = g.lvl_base[d + 1];
        const float inflow = (a.bc == RT_BC_THERMAL && a.up_flag[d] > 0.f) ? 1.f : 0.f;
        const int lc = item.lc;
        const int64_t B = blockDim.x;
        for (int L = b0; L + 1 < b1; ++L) {
            const int64_t s0 = g.lvl[L], s1 = g.lvl[L + 1];
            const int64_t work = (s1 - s0) * lc;
            // the tables (upwind record, site) of a thread's next update are loaded before the
            // gathers of the current one: two independent load streams in flight per thread
            auto table = [&](int64_t t, Upwind &uu, int &ii, int &ll) {
                const int64_t slot = s0 + t / lc;
                ll = item.c0 + (int)(t % lc);
                uu = up[slot];
                ii = order[slot];
            };
            int64_t t = threadIdx.x;
            Upwind u;
            int i = 0, l = 0;
            if (t < work) table(t, u, i, l);
            while (t < work) {
                const int64_t tn = t + B;
                Upwind un;
                int in = 0, ln = 0;
                if (tn < work) table(tn, un, in, ln);
                const VorGather gr = vor_gather(g, I, u, i, l, a.nlam, inflow);
                I[(size_t)i * a.nlam + l] = vor_update(u, gr);
                t = tn;
                u = un;
                i = in;
                l = ln;
            }
            __syncthreads();
        }
    }
}

// J[i][l] = sum_d w_d I_d[i][l], directions in index order
__global__ void batch_reduce_kernel(const float *I, float *J, const float *wdir, int ndir,
                                    size_t m, unsigned *err)
{
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= m) return;
    float acc = wdir[0] * I[t];
    for (int d = 1; d < ndir; ++d) acc = acc + wdir[d] * I[(size_t)d * m + t];
    if (!isfinite(acc)) flag_error(err, ERR_NAN);
    J[t] = acc;
}

__global__ void transpose_kernel_b(const float *__restrict__ in, float *__restrict__ out, int rows,
                                   int cols)
{
    __shared__ float tile[32][33];
    int c = blockIdx.x * 32 + threadIdx.x;
    int r0 = blockIdx.y * 32;
    for (int dr = threadIdx.y; dr < 32; dr += blockDim.y) {
        int r = r0 + dr;
        if (r < rows && c < cols) tile[dr][threadIdx.x] = in[(size_t)r * cols + c];
    }
    __syncthreads();
    int r = r0 + threadIdx.x;
    for (int dc = threadIdx.y; dc < 32; dc += blockDim.y) {
        int cc = blockIdx.x * 32 + dc;
        if (r < rows && cc < cols) out[(size_t)cc * rows + r] = tile[threadIdx.x][dc];
    }
}

static void transpose_b(const float *in, float *out, int rows, int cols, cudaStream_t st)
{
    dim3 grid((cols + 31) / 32, (rows + 31) / 32);
    note_launch();
    transpose_kernel_b<<<grid, dim3(32, 8), 0, st>>>(in, out, rows, cols);
}

// S, alpha [rows][cols] -> (S, alpha) pairs [cols][rows]
__global__ void transpose_pair_kernel(const float *__restrict__ S, const float *__restrict__ A,
                                      float2 *__restrict__ out, int rows, int cols)
{
    __shared__ float ts[32][33], ta[32][33];
    int c = blockIdx.x * 32 + threadIdx.x;
    int r0 = blockIdx.y * 32;
    for (int dr = threadIdx.y; dr < 32; dr += blockDim.y) {
        int r = r0 + dr;
        if (r < rows && c < cols) {
            ts[dr][threadIdx.x] = S[(size_t)r * cols + c];
            ta[dr][threadIdx.x] = A[(size_t)r * cols + c];
        }
    }
    __syncthreads();
    int r = r0 + threadIdx.x;
    for (int dc = threadIdx.y; dc < 32; dc += blockDim.y) {
        int cc = blockIdx.x * 32 + dc;
        if (r < rows && cc < cols)
            out[(size_t)cc * rows + r] = make_float2(ts[threadIdx.x][dc], ta[threadIdx.x][dc]);
    }
}

static void transpose_pair(const float *S, const float *A, float2 *out, int rows, int cols,
                           cudaStream_t st)
{
    dim3 grid((cols + 31) / 32, (rows + 31) / 32);
    note_launch();
    transpose_pair_kernel<<<grid, dim3(32, 8), 0, st>>>(S, A, out, rows, cols);
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
    float *d_fields = nullptr;   // per grid A, S, J [n][nlam] and I [ndir][n][nlam]
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
        int64_t ntot = 0, nmin = INT64_MAX;
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
            ntot += g->nsites;
            nmin = std::min<int64_t>(nmin, g->nsites);
        }
        int dev = 0, nsm = 0, per_sm = 0;
        RT_CUDA(cudaGetDevice(&dev));
        RT_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
        RT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_sweep_kernel, b->threads, 0));
        if (per_sm < 1) {
            delete b;
            return fail(RT_ECAPACITY, "the batched sweep kernel cannot be resident");
        }
        b->blocks = nsm * per_sm;
        // items: default chunk sizes make every item carry about the same number of (site, lambda,
        // direction) updates, about total / (2 * resident blocks)
        for (int i = 0; i < ngrids; ++i) {
            int lc;
            if (lam_chunk) {
                lc = lam_chunk[i];
            } else {
                const double target = (double)ntot * nlam * b->ndir / (2.0 * b->blocks);
                lc = (int)std::lround(target / (double)grids[i]->nsites);
            }
            lc = std::max(1, std::min(nlam, lc));
            for (int d = 0; d < b->ndir; ++d)
                for (int c0 = 0; c0 < nlam; c0 += lc)
                    b->h_items.push_back(BatchItem{i, d, c0, std::min(lc, nlam - c0)});
        }
        std::stable_sort(b->h_items.begin(), b->h_items.end(), [&](const BatchItem &x, const BatchItem &y) {
            return (double)grids[x.grid]->nsites * x.lc > (double)grids[y.grid]->nsites * y.lc;
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
        for (int i = 0; i < ngrids; ++i) fsz += batch_grid_floats(grids[i]->nsites, nlam, b->ndir);
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
            const size_t m = (size_t)g->nsites * nlam;
            BatchGridDev gd;
            gd.up = g->vt.d_up;
            gd.order = g->vt.d_order;
            gd.lvl = b->d_lvl;
            gd.lvl_base = b->d_lvl_base + base_at[i];
            gd.SA = reinterpret_cast<const float2 *>(f);
            gd.J = f + 2 * m;
            gd.I = f + 3 * m;
            gd.n = (int)g->nsites;
            f += batch_grid_floats(g->nsites, nlam, b->ndir);
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
            transpose_pair(S[i], alpha[i], const_cast<float2 *>(g.SA), b->nlam, g.n, st);
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
        batch_sweep_kernel<<<blocks, b->threads, 0, st>>>(a);
        for (int i = 0; i < ng; ++i) {
            const BatchGridDev &g = b->h_grids[i];
            const size_t m = (size_t)g.n * b->nlam;
            note_launch();
            batch_reduce_kernel<<<(unsigned)((m + 255) / 256), 256, 0, st>>>(g.I, g.J, b->d_wdir,
                                                                             b->ndir, m, b->err);
            transpose_b(g.J, J[i], g.n, b->nlam, st);
        }
        RT_CUDA(cudaGetLastError());
        return RT_OK;
    });
}

}  // extern "C"
