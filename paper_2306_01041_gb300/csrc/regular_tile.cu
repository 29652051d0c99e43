// Regular grid, per-plane sweep with shared-memory tiles (same arithmetic as sc_plane_kernel).
//
// One launch per plane step, as in sc_plane_kernel, with the upwind planes of all directions in
// the L2-resident ping-pong buffer.  A block takes (tile, wavelength) items: it copies the tile of
// the upwind plane of every direction of the hemisphere, with a halo wide enough for the largest
// stencil offset, and the interleaved (S, alpha) of the upwind plane into shared memory (16-byte
// loads; rows wrap periodically), then computes every point of the tile for every direction from
// shared memory.  Within a plane the stencil of a direction is a constant offset, so each corner
// read is a fixed displacement from the point's own slot: no wrap arithmetic per update.  A thread
// owns four points of the tile (independent dependency chains) and loops over the directions,
// accumulating J in registers in a fixed order.  With the direction count known at compile time
// (12 per hemisphere for the S4 set) the direction loop is unrolled and every per-direction
// constant (offset, bilinear weights, half path length, quadrature weight) is an operand from the
// kernel's constant bank.
#include <algorithm>
#include <cstdlib>
#include <string>

#include "device_common.cuh"
#include "rt_impl.h"

namespace rt {

constexpr int TL_W = 32;          // tile width (x)
constexpr int TL_THREADS = 512;
constexpr int TL_ROWS = TL_THREADS / TL_W;   // rows covered by one pass of the block (16)
constexpr int TL_PPT = 2;         // points per thread (rows y and y + 16)
constexpr int TL_H = TL_ROWS * TL_PPT;       // tile height (y)
constexpr int TL_HXP = 4;         // x halo, padded to 4 floats for 16-byte staging
constexpr int TL_PW = TL_W + 2 * TL_HXP;
constexpr int TL_MAX_DH = 16;

struct TileArgs {
    const float *alpha, *S;   // [nlam][npt]
    const float *Iprev;       // [nlam][ndh][np]
    float *Inext;
    float *J;
    unsigned *err;
    int nx, ny, nz, np, nlam, ndh, up, first, step, k, ku;
    int hy;                   // y halo
    int wrap1;                // 1: the staged tile wraps at most once (single-step wrap)
    int tiles_x, ntiles;
    int dg[TL_MAX_DH];
    float w[TL_MAX_DH];
    int off[TL_MAX_DH];       // corner (0,0) displacement in the shared tile: ay * pitch + ax
    float cw[TL_MAX_DH][4];   // bilinear weights
    float hds[TL_MAX_DH];
};

__device__ __forceinline__ int wrapi(int v, int n, bool once)
{
    if (once) {
        v += v < 0 ? n : 0;
        return v >= n ? v - n : v;
    }
    v %= n;
    return v < 0 ? v + n : v;
}

template <int NDH>
__global__ void __launch_bounds__(TL_THREADS, 2) sc_tile_kernel(const TileArgs a)
{
    extern __shared__ __align__(16) float smt[];
    const int ndh = NDH > 0 ? NDH : a.ndh;
    const int ph = TL_H + 2 * a.hy;
    const int tsz = TL_PW * ph;                              // floats per staged tile
    float *It = smt;                                         // [ndh][ph][TL_PW]
    float2 *SA = reinterpret_cast<float2 *>(smt + (size_t)ndh * tsz);   // [ph][TL_PW]
    const int tid = threadIdx.x;
    const int lx = tid % TL_W, ly = tid / TL_W;              // ly in 0..TL_ROWS-1
    const size_t npt = (size_t)a.np * a.nz;
    const int nitems = a.ntiles * a.nlam;
    const int q4 = TL_PW / 4;                                // float4 per staged row
    for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
        const int l = item / a.ntiles, tile = item % a.ntiles;
        const int x0 = (tile % a.tiles_x) * TL_W, y0 = (tile / a.tiles_x) * TL_H;
        const float *al = a.alpha + (size_t)l * npt, *Sl = a.S + (size_t)l * npt;
        const float *Su = Sl + (size_t)a.ku * a.np, *Au = al + (size_t)a.ku * a.np;
        __syncthreads();   // the previous item's reads of the tile are done
        // stage the upwind plane (every direction's intensity, and S with alpha), with halo;
        // a float4 never straddles the periodic seam because nx and x0 - TL_HXP are multiples of 4
        for (int e = tid; e < ph * q4; e += TL_THREADS) {
            const int r = e / q4, c4 = e % q4;
            const int gy = wrapi(y0 - a.hy + r, a.ny, a.wrap1);
            const int gx = wrapi(x0 - TL_HXP + 4 * c4, a.nx, a.wrap1);
            const size_t g = (size_t)gy * a.nx + gx;
            const float4 sv = __ldg(reinterpret_cast<const float4 *>(Su + g));
            const float4 av = __ldg(reinterpret_cast<const float4 *>(Au + g));
            float4 *sa = reinterpret_cast<float4 *>(SA + r * TL_PW + 4 * c4);
            sa[0] = make_float4(sv.x, av.x, sv.y, av.y);
            sa[1] = make_float4(sv.z, av.z, sv.w, av.w);
#pragma unroll
            for (int d = 0; d < (NDH > 0 ? NDH : TL_MAX_DH); ++d) {
                if (NDH == 0 && d >= ndh) break;
                const float4 iv = __ldg(reinterpret_cast<const float4 *>(
                    a.Iprev + ((size_t)l * ndh + d) * a.np + g));
                reinterpret_cast<float4 *>(It + d * tsz + r * TL_PW)[c4] = iv;
            }
        }
        __syncthreads();
        int gxy[TL_PPT], slot[TL_PPT];
        float Sk[TL_PPT], ak[TL_PPT], jacc[TL_PPT];
        bool ok[TL_PPT];
#pragma unroll
        for (int m = 0; m < TL_PPT; ++m) {
            const int x = x0 + lx, y = y0 + ly + TL_ROWS * m;
            ok[m] = x < a.nx && y < a.ny;
            gxy[m] = ok[m] ? y * a.nx + x : 0;
            slot[m] = (ly + TL_ROWS * m + a.hy) * TL_PW + lx + TL_HXP;
            Sk[m] = ok[m] ? __ldg(Sl + (size_t)a.k * a.np + gxy[m]) : 0.f;
            ak[m] = ok[m] ? __ldg(al + (size_t)a.k * a.np + gxy[m]) : 0.f;
            jacc[m] = 0.f;
        }
        float *In = a.Inext + (size_t)l * ndh * a.np;
#pragma unroll
        for (int d = 0; d < (NDH > 0 ? NDH : TL_MAX_DH); ++d) {
            if (NDH == 0 && d >= ndh) break;
            const float c0 = a.cw[d][0], c1 = a.cw[d][1], c2 = a.cw[d][2], c3 = a.cw[d][3];
            const float hds = a.hds[d], wd = a.w[d];
            const float *Id = It + d * tsz;
#pragma unroll
            for (int m = 0; m < TL_PPT; ++m) {
                const int o = slot[m] + a.off[d];
                const float iu = c0 * Id[o] + c1 * Id[o + 1] + c2 * Id[o + TL_PW] + c3 * Id[o + TL_PW + 1];
                const float2 s00 = SA[o], s10 = SA[o + 1], s01 = SA[o + TL_PW], s11 = SA[o + TL_PW + 1];
                const float su = c0 * s00.x + c1 * s10.x + c2 * s01.x + c3 * s11.x;
                const float au = c0 * s00.y + c1 * s10.y + c2 * s01.y + c3 * s11.y;
                const float dt = (au + ak[m]) * hds;
                float ex, w0, w1;
                lin_weights(dt, ex, w0, w1);
                const float v = iu * ex + w0 * su + w1 * Sk[m];
                if (ok[m]) In[(size_t)d * a.np + gxy[m]] = v;
                jacc[m] += wd * v;
            }
        }
#pragma unroll
        for (int m = 0; m < TL_PPT; ++m) {
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

static bool tile_plan(const rt_grid *g, int &hy)
{
    const char *env = std::getenv("RT_REGULAR_SWEEP");
    if (env && (std::string(env) == "plane" || std::string(env) == "cluster")) return false;
    if (!g->periodic || g->nx % 4 || g->dir_up.size() > TL_MAX_DH || g->dir_dn.size() > TL_MAX_DH)
        return false;
    // corners reach x + ax .. x + ax + 1 and y + ay .. y + ay + 1
    int lx = 0, rx = 0, ly = 0, ry = 0;
    for (const Stencil &s : g->h_stencil) {
        lx = std::max(lx, -s.ax);
        rx = std::max(rx, s.ax + 1);
        ly = std::max(ly, -s.ay);
        ry = std::max(ry, s.ay + 1);
    }
    hy = std::max(ly, ry);
    return std::max(lx, rx) <= TL_HXP && hy <= 8;
}

template <int NDH>
static rt_status launch_planes(rt_grid *g, TileArgs &a, const std::vector<int> &dirs, int bc,
                               int nlam, float **bufs, cudaStream_t st)
{
    const int ph = TL_H + 2 * a.hy, tsz = TL_PW * ph;
    const size_t smem = ((size_t)a.ndh * tsz) * sizeof(float) + (size_t)tsz * sizeof(float2);
    RT_CUDA(cudaFuncSetAttribute(sc_tile_kernel<NDH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem));
    int per_sm = 0, dev = 0, nsm = 0;
    RT_CUDA(cudaGetDevice(&dev));
    RT_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    RT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sc_tile_kernel<NDH>, TL_THREADS,
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
            a.off[d] = sc.ay * TL_PW + sc.ax;
            a.cw[d][0] = sc.w0;
            a.cw[d][1] = sc.w1;
            a.cw[d][2] = sc.w2;
            a.cw[d][3] = sc.w3;
            a.hds[d] = sc.hds;
        }
        sc_tile_kernel<NDH><<<blocks, TL_THREADS, smem, st>>>(a);
    }
    RT_CUDA(cudaGetLastError());
    return RT_OK;
}

rt_status regular_tile_sweep(rt_grid *g, int nlam, const float *alpha, const float *S, int bc,
                             float *J, float *buf0, float *buf1, cudaStream_t st, bool *done)
{
    *done = false;
    int hy;
    if (bc == RT_BC_ARRAY || !tile_plan(g, hy)) return RT_OK;
    if (!aligned16(alpha) || !aligned16(S)) return RT_OK;
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
    a.hy = hy;
    a.tiles_x = (g->nx + TL_W - 1) / TL_W;
    a.ntiles = a.tiles_x * ((g->ny + TL_H - 1) / TL_H);
    a.wrap1 = (g->nx >= TL_PW && g->ny >= TL_H + 2 * hy) ? 1 : 0;
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
        if (a.ndh == 12) RT_TRY(launch_planes<12>(g, a, dirs, bc, nlam, bufs, st));
        else RT_TRY(launch_planes<0>(g, a, dirs, bc, nlam, bufs, st));
        first = 0;
    }
    *done = true;
    return RT_OK;
}

}  // namespace rt
