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

// What one (plane, wavelength, tile) item needs beyond the launch-wide arguments.
struct PlaneCtx {
    int k, ku, up, first;
    const float *Iprev;
    float *Inext;
};

// One (tile, wavelength) item of one plane step.  COHERENT selects L2-coherent loads of the
// upwind intensities (the persistent kernel reads planes written by other blocks of the same
// launch, which the non-coherent read-only path could serve stale).
template <int NDH, bool COHERENT>
__device__ __forceinline__ void tile_item(const TileArgs &a, const PlaneCtx &c, int l, int tile,
                                          float *smt)
{
    const int ndh = NDH > 0 ? NDH : a.ndh;
    const int ph = TL_H + 2 * a.hy;
    const int tsz = TL_PW * ph;                              // floats per staged tile
    float *It = smt;                                         // [ndh][ph][TL_PW]
    float2 *SA = reinterpret_cast<float2 *>(smt + (size_t)ndh * tsz);   // [ph][TL_PW]
    const int tid = threadIdx.x;
    const int lx = tid % TL_W, ly = tid / TL_W;              // ly in 0..TL_ROWS-1
    const size_t npt = (size_t)a.np * a.nz;
    const int q4 = TL_PW / 4;                                // float4 per staged row
    const int x0 = (tile % a.tiles_x) * TL_W, y0 = (tile / a.tiles_x) * TL_H;
    const float *al = a.alpha + (size_t)l * npt, *Sl = a.S + (size_t)l * npt;
    const float *Su = Sl + (size_t)c.ku * a.np, *Au = al + (size_t)c.ku * a.np;
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
            const float4 *src = reinterpret_cast<const float4 *>(
                c.Iprev + ((size_t)l * ndh + d) * a.np + g);
            const float4 iv = COHERENT ? __ldcg(src) : __ldg(src);
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
        Sk[m] = ok[m] ? __ldg(Sl + (size_t)c.k * a.np + gxy[m]) : 0.f;
        ak[m] = ok[m] ? __ldg(al + (size_t)c.k * a.np + gxy[m]) : 0.f;
        jacc[m] = 0.f;
    }
    float *In = c.Inext + (size_t)l * ndh * a.np;
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
            if (ok[m]) {
                if (COHERENT) __stcg(In + (size_t)d * a.np + gxy[m], v);
                else In[(size_t)d * a.np + gxy[m]] = v;
            }
            jacc[m] += wd * v;
        }
    }
#pragma unroll
    for (int m = 0; m < TL_PPT; ++m) {
        if (!ok[m]) continue;
        float *Jp = a.J + (size_t)l * npt + (size_t)c.k * a.np + gxy[m];
        const float v = c.first ? jacc[m] : (COHERENT ? __ldcg(Jp) : *Jp) + jacc[m];
        if (!isfinite(v)) flag_error(a.err, ERR_NAN);
        if (COHERENT) __stcg(Jp, v);
        else *Jp = v;
    }
}

template <int NDH>
__global__ void __launch_bounds__(TL_THREADS, 2) sc_tile_kernel(const TileArgs a)
{
    extern __shared__ __align__(16) float smt[];
    const PlaneCtx c{a.k, a.ku, a.up, a.first, a.Iprev, a.Inext};
    const int nitems = a.ntiles * a.nlam;
    for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
        __syncthreads();   // the previous item's reads of the tile are done
        tile_item<NDH, false>(a, c, item / a.ntiles, item % a.ntiles, smt);
    }
}

// Boundary plane of one tile and wavelength: the rule for every direction, and J.
template <int NDH>
__device__ __forceinline__ void boundary_item(const TileArgs &a, const PlaneCtx &c, int l, int tile,
                                              int bc)
{
    const int ndh = NDH > 0 ? NDH : a.ndh;
    const int x0 = (tile % a.tiles_x) * TL_W, y0 = (tile / a.tiles_x) * TL_H;
    const size_t npt = (size_t)a.np * a.nz;
    for (int e = threadIdx.x; e < TL_W * TL_H; e += TL_THREADS) {
        const int x = x0 + e % TL_W, y = y0 + e / TL_W;
        if (x >= a.nx || y >= a.ny) continue;
        const int q = y * a.nx + x;
        const float Sk = __ldg(a.S + (size_t)l * npt + (size_t)c.k * a.np + q);
        const float v = (bc == RT_BC_THERMAL && c.up) ? Sk : 0.f;
        float jacc = 0.f;
        for (int d = 0; d < ndh; ++d) {
            __stcg(c.Inext + ((size_t)l * ndh + d) * a.np + q, v);
            jacc += a.w[d] * v;
        }
        float *Jp = a.J + (size_t)l * npt + (size_t)c.k * a.np + q;
        __stcg(Jp, c.first ? jacc : __ldcg(Jp) + jacc);
    }
}

// Persistent wavefront sweep of both hemispheres in one launch.  Items (hemisphere, plane step,
// wavelength, tile) are taken from a device counter in that order.  An item waits for the items
// of the previous step on the 3 x 3 neighbouring tiles (its upwind data, and the last readers of
// the ring slot it overwrites) and, in the downward hemisphere, for the upward item of the same
// plane and tile (J accumulates upward first).  A block claims its next item when it starts the
// current one (hiding the counter's latency); every awaited item still precedes the awaiting one
// in counter order, so by induction on the smallest unfinished item the waits cannot deadlock,
// whatever the residency.  Lanes 0..9 of warp 0 poll the flags in parallel; the completion flag
// is a release store by thread 0 after the block barrier, the wait an acquire load before it.
// Each wait is bounded: past the limit the block records ERR_TIMEOUT and goes on.
struct WaveArgs {
    TileArgs t[2];             // per hemisphere: stencils (identical for every plane), weights
    float *ring[2][2];         // [hemisphere][step parity] upwind planes [nlam][ndh][np]
    int *queue;
    int *done;                 // [2][nz][nlam][ntiles] completion flags
    int nd[2];
    int bc, first_hemi;
};

// Bounded wait for a completion flag.  Once any wait of the launch has timed out (ERR_TIMEOUT in
// *err) every later wait gives up at once, so a failed launch ends after one time-out, not one per
// item.
__device__ __forceinline__ bool wait_flag(const int *f, const unsigned *err)
{
    int v;
    for (int it = 0; it < (1 << 20); ++it) {
        asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(f) : "memory");
        if (v) return true;
        if ((it & 255) == 255 && (*(volatile const unsigned *)err & ERR_TIMEOUT)) return false;
        __nanosleep(32);
    }
    return false;
}

template <int NDH>
__global__ void __launch_bounds__(TL_THREADS, 2) sc_wave_kernel(WaveArgs w)
{
    extern __shared__ __align__(16) float smt[];
    __shared__ int item_s;
    const TileArgs &a = w.t[0];
    const int nt = a.ntiles, nl = a.nlam, nz = a.nz;
    const int per_hemi = nz * nl * nt;
    const int total = 2 * per_hemi;
    const int tx = a.tiles_x, ty = nt / a.tiles_x;
    if (threadIdx.x == 0) item_s = atomicAdd(w.queue, 1);
    for (;;) {
        __syncthreads();   // item_s is published; the previous item is finished by every thread
        const int item = item_s;
        if (item >= total) return;
        int next = 0;
        if (threadIdx.x == 0) next = atomicAdd(w.queue, 1);
        const int h = item / per_hemi;
        int rem = item % per_hemi;
        const int s = rem / (nl * nt);
        rem %= nl * nt;
        const int l = rem / nt, tile = rem % nt;
        const bool up = h == 0;
        const int k = up ? s : nz - 1 - s;
        PlaneCtx c;
        c.k = k;
        c.ku = up ? k - 1 : k + 1;
        c.up = up;
        c.first = (h == w.first_hemi);
        c.Iprev = w.ring[h][(s + 1) & 1];
        c.Inext = w.ring[h][s & 1];
        if (threadIdx.x < 32) {
            const int lane = threadIdx.x;
            const int *f = nullptr;
            if (lane < 9 && s > 0) {
                const int tx0 = tile % tx, ty0 = tile / tx;
                const int nx_ = (tx0 + lane % 3 - 1 + tx) % tx, ny_ = (ty0 + lane / 3 - 1 + ty) % ty;
                f = w.done + ((size_t)(h * nz + s - 1) * nl + l) * nt + ny_ * tx + nx_;
            } else if (lane == 9 && h == 1 && !c.first) {   // the upward J of this plane and tile
                f = w.done + ((size_t)(0 * nz + k) * nl + l) * nt + tile;
            }
            const bool ok = __all_sync(0xffffffffu, f ? wait_flag(f, a.err) : true);
            if (lane == 0 && !ok) flag_error(a.err, ERR_TIMEOUT);
        }
        __syncthreads();
        // one inlined copy per hemisphere keeps every per-direction constant a static operand
        if (h == 0) {
            if (s == 0) boundary_item<NDH>(w.t[0], c, l, tile, w.bc);
            else tile_item<NDH, true>(w.t[0], c, l, tile, smt);
        } else {
            if (s == 0) boundary_item<NDH>(w.t[1], c, l, tile, w.bc);
            else tile_item<NDH, true>(w.t[1], c, l, tile, smt);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int *f = w.done + ((size_t)(h * nz + s) * nl + l) * nt + tile;
            asm volatile("st.release.gpu.global.b32 [%0], %1;" :: "l"(f), "r"(1) : "memory");
            item_s = next;
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
            note_launch();
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
        note_launch();
        sc_tile_kernel<NDH><<<blocks, TL_THREADS, smem, st>>>(a);
    }
    RT_CUDA(cudaGetLastError());
    return RT_OK;
}

// The persistent wavefront sweep applies when every plane has the same stencil per direction
// (uniform z spacing), both hemispheres have 12 directions, and the stencil reach stays within
// one tile.
static bool uniform_stencils(const rt_grid *g)
{
    for (int q = 0; q < g->ndir; ++q) {
        const bool up = g->dirs[3 * q + 2] > 0;
        const int k0 = up ? 1 : 0, k1 = up ? g->nz - 1 : g->nz - 2, kref = up ? 1 : g->nz - 2;
        const Stencil &r = g->h_stencil[(size_t)kref * g->ndir + q];
        for (int k = k0; k <= k1; ++k) {
            const Stencil &a = g->h_stencil[(size_t)k * g->ndir + q];
            if (a.ax != r.ax || a.ay != r.ay || a.w0 != r.w0 || a.w1 != r.w1 || a.w2 != r.w2 ||
                a.w3 != r.w3 || a.hds != r.hds)
                return false;
        }
    }
    return true;
}

size_t regular_wave_scratch(const rt_grid *g, int nlam)
{
    const size_t plane = (size_t)nlam * 12 * g->nx * g->ny;
    const size_t ntiles = (size_t)((g->nx + TL_W - 1) / TL_W) * ((g->ny + TL_H - 1) / TL_H);
    const size_t nflags = 2 * (size_t)g->nz * nlam * ntiles;
    return 4 * plane * sizeof(float) + (nflags + 64) * sizeof(int);
}

static rt_status wave_sweep(rt_grid *g, TileArgs &base, int nlam, int bc, cudaStream_t st,
                            bool *done)
{
    const char *env = std::getenv("RT_REGULAR_SWEEP");
    if (env && std::string(env) == "tile") return RT_OK;   // per-plane launches requested
    if (g->dir_up.size() != 12 || g->dir_dn.size() != 12 || g->nz < 3 || !uniform_stencils(g))
        return RT_OK;
    WaveArgs w;
    const std::vector<int> *hs[2] = {&g->dir_up, &g->dir_dn};
    for (int h = 0; h < 2; ++h) {
        TileArgs &a = w.t[h];
        a = base;
        a.ndh = 12;
        a.up = h == 0;
        const int kref = h == 0 ? 1 : g->nz - 2;   // every plane shares this stencil
        for (int d = 0; d < 12; ++d) {
            const int q = (*hs[h])[d];
            const Stencil &sc = g->h_stencil[(size_t)kref * g->ndir + q];
            a.dg[d] = q;
            a.w[d] = (float)g->wdir[q];
            a.off[d] = sc.ay * TL_PW + sc.ax;
            a.cw[d][0] = sc.w0;
            a.cw[d][1] = sc.w1;
            a.cw[d][2] = sc.w2;
            a.cw[d][3] = sc.w3;
            a.hds[d] = sc.hds;
        }
        w.nd[h] = 12;
    }
    const size_t plane = (size_t)nlam * 12 * g->nx * g->ny;
    const size_t nflags = 2 * (size_t)g->nz * nlam * base.ntiles;
    void *p;
    RT_TRY(scratch_get(g, 3, regular_wave_scratch(g, nlam), &p));
    float *f = (float *)p;
    w.ring[0][0] = f;
    w.ring[0][1] = f + plane;
    w.ring[1][0] = f + 2 * plane;
    w.ring[1][1] = f + 3 * plane;
    w.queue = (int *)(f + 4 * plane);
    w.done = w.queue + 32;
    w.bc = bc;
    w.first_hemi = 0;
    RT_CUDA(cudaMemsetAsync(w.queue, 0, (nflags + 32) * sizeof(int), st));
    const int ph = TL_H + 2 * base.hy, tsz = TL_PW * ph;
    const size_t smem = (12 * (size_t)tsz) * sizeof(float) + (size_t)tsz * sizeof(float2);
    RT_CUDA(cudaFuncSetAttribute(sc_wave_kernel<12>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem));
    int per_sm = 0, dev = 0, nsm = 0;
    RT_CUDA(cudaGetDevice(&dev));
    RT_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    RT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sc_wave_kernel<12>, TL_THREADS,
                                                          smem));
    if (per_sm < 1) return RT_OK;
    note_launch();
    sc_wave_kernel<12><<<per_sm * nsm, TL_THREADS, smem, st>>>(w);
    RT_CUDA(cudaGetLastError());
    *done = true;
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
    RT_TRY(wave_sweep(g, a, nlam, bc, st, done));
    if (*done) return RT_OK;
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
