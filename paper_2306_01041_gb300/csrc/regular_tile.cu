// Regular grid, per-plane sweep with shared-memory tiles (same arithmetic as sc_plane_kernel).
//
// One launch per plane step, as in sc_plane_kernel, with the upwind planes of all directions in
// the L2-resident ping-pong buffer.  A block takes (tile, wavelength) items: it copies the tile of
// the upwind plane of every direction of the hemisphere, with a halo wide enough for the largest
// stencil offset, and the interleaved (S, alpha) of the upwind plane into shared memory with
// coalesced loads (rows wrap periodically), then computes every point of the tile for every
// direction from shared memory.  Within a plane the stencil of a direction is a constant offset,
// so each corner read is a fixed displacement from the point's own slot: no wrap arithmetic per
// update.  A thread owns two points of the tile (independent dependency chains) and loops over
// the directions, accumulating J in registers in a fixed order.
#include <algorithm>
#include <cstdlib>
#include <string>

#include "device_common.cuh"
#include "rt_impl.h"

namespace rt {

constexpr int TL_W = 32;          // tile width (x)
constexpr int TL_H = 16;          // tile height (y)
constexpr int TL_THREADS = 256;   // two points per thread (rows y and y + 8)
constexpr int TL_MAX_DH = 16;

struct TileArgs {
    const float *alpha, *S;   // [nlam][npt]
    const float *Iprev;       // [nlam][ndh][np]
    float *Inext;
    float *J;
    unsigned *err;
    int nx, ny, nz, np, nlam, ndh, up, first, step, k, ku;
    int hx, hy;               // halo widths
    int tiles_x, ntiles;
    int dg[TL_MAX_DH];
    float w[TL_MAX_DH];
    int off[TL_MAX_DH];       // corner (0,0) displacement in the shared tile: ay * pitch + ax
    float cw[TL_MAX_DH][4];   // bilinear weights
    float hds[TL_MAX_DH];
};

__device__ __forceinline__ int wrapi(int v, int n)
{
    v %= n;
    return v < 0 ? v + n : v;
}

__global__ void __launch_bounds__(TL_THREADS) sc_tile_kernel(const TileArgs a)
{
    extern __shared__ __align__(16) float smt[];
    const int pw = TL_W + 2 * a.hx, ph = TL_H + 2 * a.hy;   // pitch and rows of a staged tile
    const int tsz = pw * ph;
    float *It = smt;                                         // [ndh][ph][pw]
    // (S, alpha) pairs after the intensity tiles, on an 8-byte boundary
    float2 *SA = reinterpret_cast<float2 *>(smt + (((size_t)a.ndh * tsz + 1) & ~(size_t)1));
    const int tid = threadIdx.x;
    const int lx = tid % TL_W, ly = tid / TL_W;              // ly in 0..7
    const size_t npt = (size_t)a.np * a.nz;
    const int nitems = a.ntiles * a.nlam;
    for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
        const int l = item / a.ntiles, tile = item % a.ntiles;
        const int x0 = (tile % a.tiles_x) * TL_W, y0 = (tile / a.tiles_x) * TL_H;
        const float *al = a.alpha + (size_t)l * npt, *Sl = a.S + (size_t)l * npt;
        __syncthreads();   // the previous item's reads of the tile are done
        // stage the upwind plane: every direction's intensity and (S, alpha), with halo
        for (int e = tid; e < tsz; e += TL_THREADS) {
            const int r = e / pw, c = e % pw;
            const int gy = wrapi(y0 - a.hy + r, a.ny), gx = wrapi(x0 - a.hx + c, a.nx);
            const size_t g = (size_t)gy * a.nx + gx;
            SA[e] = make_float2(__ldg(Sl + (size_t)a.ku * a.np + g), __ldg(al + (size_t)a.ku * a.np + g));
            for (int d = 0; d < a.ndh; ++d)
                It[d * tsz + e] = __ldg(a.Iprev + ((size_t)l * a.ndh + d) * a.np + g);
        }
        __syncthreads();
        // two points per thread: (lx, ly) and (lx, ly + 8)
        int gxy[2];
        float Sk[2], ak[2], jacc[2] = {0.f, 0.f};
        int slot[2];
        bool ok[2];
#pragma unroll
        for (int m = 0; m < 2; ++m) {
            const int x = x0 + lx, y = y0 + ly + 8 * m;
            ok[m] = x < a.nx && y < a.ny;
            gxy[m] = ok[m] ? y * a.nx + x : 0;
            slot[m] = (ly + 8 * m + a.hy) * pw + lx + a.hx;
            Sk[m] = ok[m] ? __ldg(Sl + (size_t)a.k * a.np + gxy[m]) : 0.f;
            ak[m] = ok[m] ? __ldg(al + (size_t)a.k * a.np + gxy[m]) : 0.f;
        }
        for (int d = 0; d < a.ndh; ++d) {
            const float c0 = a.cw[d][0], c1 = a.cw[d][1], c2 = a.cw[d][2], c3 = a.cw[d][3];
            const float hds = a.hds[d];
            const float *Id = It + d * tsz;
#pragma unroll
            for (int m = 0; m < 2; ++m) {
                const int o = slot[m] + a.off[d];
                const float iu = c0 * Id[o] + c1 * Id[o + 1] + c2 * Id[o + pw] + c3 * Id[o + pw + 1];
                const float2 s00 = SA[o], s10 = SA[o + 1], s01 = SA[o + pw], s11 = SA[o + pw + 1];
                const float su = c0 * s00.x + c1 * s10.x + c2 * s01.x + c3 * s11.x;
                const float au = c0 * s00.y + c1 * s10.y + c2 * s01.y + c3 * s11.y;
                const float dt = (au + ak[m]) * hds;
                float ex, w0, w1;
                lin_weights(dt, ex, w0, w1);
                const float v = iu * ex + w0 * su + w1 * Sk[m];
                if (ok[m]) a.Inext[((size_t)l * a.ndh + d) * a.np + gxy[m]] = v;
                jacc[m] += a.w[d] * v;
            }
        }
#pragma unroll
        for (int m = 0; m < 2; ++m) {
            if (!ok[m]) continue;
            float *Jp = a.J + (size_t)l * npt + (size_t)a.k * a.np + gxy[m];
            const float v = a.first ? jacc[m] : *Jp + jacc[m];
            if (!isfinite(v)) flag_error(a.err, ERR_NAN);
            *Jp = v;
        }
    }
}

// boundary plane of a hemisphere: the rule for every direction, and J
__global__ void sc_tile_boundary_kernel(const TileArgs a, int bc)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    const int l = blockIdx.y;
    if (q >= a.np) return;
    const size_t npt = (size_t)a.np * a.nz;
    const float Sk = __ldg(a.S + (size_t)l * npt + (size_t)a.k * a.np + q);
    const float v = (bc == RT_BC_THERMAL && a.up) ? Sk : 0.f;
    float jacc = 0.f;
    for (int d = 0; d < a.ndh; ++d) {
        a.Inext[((size_t)l * a.ndh + d) * a.np + q] = v;
        jacc += a.w[d] * v;
    }
    float *Jp = a.J + (size_t)l * npt + (size_t)a.k * a.np + q;
    *Jp = a.first ? jacc : *Jp + jacc;
}

static bool tile_plan(const rt_grid *g, int &hx, int &hy)
{
    const char *env = std::getenv("RT_REGULAR_SWEEP");
    if (env && (std::string(env) == "plane" || std::string(env) == "cluster")) return false;
    if (!g->periodic || g->dir_up.size() > TL_MAX_DH || g->dir_dn.size() > TL_MAX_DH) return false;
    // corners reach x + ax .. x + ax + 1 and y + ay .. y + ay + 1
    int lx = 0, rx = 0, ly = 0, ry = 0;
    for (const Stencil &s : g->h_stencil) {
        lx = std::max(lx, -s.ax);
        rx = std::max(rx, s.ax + 1);
        ly = std::max(ly, -s.ay);
        ry = std::max(ry, s.ay + 1);
    }
    hx = std::max(lx, rx);
    hy = std::max(ly, ry);
    return hx <= 8 && hy <= 8;
}

rt_status regular_tile_sweep(rt_grid *g, int nlam, const float *alpha, const float *S, int bc,
                             float *J, float *buf0, float *buf1, cudaStream_t st, bool *done)
{
    *done = false;
    int hx, hy;
    if (bc == RT_BC_ARRAY || !tile_plan(g, hx, hy)) return RT_OK;
    TileArgs a;
    a.alpha = alpha;
    a.S = S;
    a.J = J;
    a.err = g->d_err;
    a.nx = g->nx;
    a.ny = g->ny;
    a.nz = g->nz;
    a.np = g->nx * g->ny;
    a.nlam = nlam;
    a.hx = hx;
    a.hy = hy;
    a.tiles_x = (g->nx + TL_W - 1) / TL_W;
    a.ntiles = a.tiles_x * ((g->ny + TL_H - 1) / TL_H);
    const int pw = TL_W + 2 * hx, ph = TL_H + 2 * hy, tsz = pw * ph;
    int dev = 0, nsm = 0;
    RT_CUDA(cudaGetDevice(&dev));
    RT_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    float *bufs[2] = {buf0, buf1};
    int first = 1;
    for (int hemi = 0; hemi < 2; ++hemi) {
        const std::vector<int> &dirs = hemi == 0 ? g->dir_up : g->dir_dn;
        if (dirs.empty()) continue;
        a.up = hemi == 0;
        a.first = first;
        a.ndh = (int)dirs.size();
        for (int d = 0; d < a.ndh; ++d) {
            a.dg[d] = dirs[d];
            a.w[d] = (float)g->wdir[dirs[d]];
        }
        const size_t smem = ((size_t)a.ndh * tsz + 1) * sizeof(float) + (size_t)tsz * sizeof(float2);
        RT_CUDA(cudaFuncSetAttribute(sc_tile_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem));
        int per_sm = 0;
        RT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sc_tile_kernel, TL_THREADS,
                                                              smem));
        const int nitems = a.ntiles * nlam;
        const int blocks = std::max(1, std::min(nitems, std::max(per_sm, 1) * nsm));
        for (int s = 0; s < g->nz; ++s) {
            a.step = s;
            a.k = a.up ? s : g->nz - 1 - s;
            a.ku = a.up ? a.k - 1 : a.k + 1;
            a.Iprev = bufs[(s + 1) & 1];
            a.Inext = bufs[s & 1];
            if (s == 0) {
                sc_tile_boundary_kernel<<<dim3((a.np + 255) / 256, nlam), 256, 0, st>>>(a, bc);
                continue;
            }
            for (int d = 0; d < a.ndh; ++d) {
                const Stencil &sc = g->h_stencil[(size_t)a.k * g->ndir + dirs[d]];
                a.off[d] = sc.ay * pw + sc.ax;
                a.cw[d][0] = sc.w0;
                a.cw[d][1] = sc.w1;
                a.cw[d][2] = sc.w2;
                a.cw[d][3] = sc.w3;
                a.hds[d] = sc.hds;
            }
            sc_tile_kernel<<<blocks, TL_THREADS, smem, st>>>(a);
        }
        first = 0;
    }
    RT_CUDA(cudaGetLastError());
    *done = true;
    return RT_OK;
}

}  // namespace rt
