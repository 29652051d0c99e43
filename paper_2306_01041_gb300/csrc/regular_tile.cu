// Regular grid sweeps with shared-memory tiles (same arithmetic as sc_plane_kernel).
//
// The unit of work is a (plane step, wavelength, 32 x 32 tile) item.  A block copies the tile of
// the upwind plane of every direction of the hemisphere, with a halo wide enough for the largest
// stencil offset, and (S, alpha) of the upwind plane as pairs for x and x + 1, into shared memory
// (16-byte loads; rows wrap periodically), then computes every point of the tile for every
// direction from shared memory.  Within a plane the stencil of a direction is a constant offset,
// so each corner read is a fixed displacement from the point's own slot: no wrap arithmetic per
// update.  A thread owns two vertically adjacent points (their corner rows overlap) and loops
// over the directions, accumulating J in registers in a fixed order.  With the direction count
// known at compile time (12 per hemisphere for the S4 set) the direction loop is unrolled and
// every per-direction constant (offset, bilinear weights, half path length, quadrature weight) is
// an operand from the kernel's constant bank.
//
// Three schedules of the same items: sc_wave_kernel (default) runs the whole formal solution as
// one persistent launch ordered by a device counter and per-item completion flags;
// sc_pipe_kernel (opt-in) is that schedule with the next item's staging in flight during the
// current one; sc_tile_kernel launches once per plane step.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <type_traits>
#include <string>

#include "device_common.cuh"
#include "rt_impl.h"

namespace rt {

constexpr int TL_W = 32;          // tile width (x)
constexpr int TL_THREADS = 512;
constexpr int TL_ROWS = TL_THREADS / TL_W;   // rows covered by one pass of the block (16)
constexpr int TL_PPT = 2;         // points per thread (tile rows 2 ly and 2 ly + 1)
static_assert(TL_PPT == 2, "tile_updates shares corner rows between exactly two points");
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
    float hds_min;            // min over the directions of hds
    int lchunk;               // persistent sweeps: wavelengths swept together through all planes
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

// One direction's stencil on one plane for the persistent sweep on non-uniform z (the uniform case
// keeps these in the kernel's constant bank instead): bilinear weights, half path length,
// quadrature weight, corner displacement in the staged tile; hds_min is the plane's minimum hds.
struct WaveSt {
    float c0, c1, c2, c3;
    float hds, wd;
    int off;
    float hds_min;
};
static_assert(sizeof(WaveSt) == 32, "WaveSt is two float4");

// Interval weights for d >= 0.1 only: the same arithmetic as the d >= 0.1 branch of lin_weights.
__device__ __forceinline__ void lin_weights_thick(float d, float &ex, float &w0, float &w1)
{
    ex = exp_neg(d);
    const float e0 = 1.0f - ex;
    const float r = rcp_fast(d);
    w1 = fmaf(-e0, r, 1.0f);
    w0 = fmaf(e0, r, -ex);
}

// Per-point updates of one staged item for every direction.  THICK: every interval of the item
// has d >= 0.1, so only the exact interval weights are evaluated.
template <int NDH, bool WAVE, bool THICK, bool PP>
__device__ __forceinline__ void tile_updates(const TileArgs &a, const WaveSt *sts, const float *It,
                                             const float4 *SA, int tsz, const int (&slot)[TL_PPT],
                                             const float (&Sk)[TL_PPT], const float (&ak)[TL_PPT],
                                             const bool (&ok)[TL_PPT], float *In, size_t dstride,
                                             size_t mstride, float (&jacc)[TL_PPT])
{
    const int ndh = NDH > 0 ? NDH : a.ndh;
#pragma unroll
    for (int d = 0; d < (NDH > 0 ? NDH : TL_MAX_DH); ++d) {
        if (NDH == 0 && d >= ndh) break;
        float c0, c1, c2, c3, hds, wd;
        int off;
        if (PP) {   // per-plane stencil from shared memory (two broadcast loads)
            const float4 q0 = reinterpret_cast<const float4 *>(sts)[2 * d];
            const float4 q1 = reinterpret_cast<const float4 *>(sts)[2 * d + 1];
            c0 = q0.x, c1 = q0.y, c2 = q0.z, c3 = q0.w;
            hds = q1.x, wd = q1.y, off = __float_as_int(q1.z);
        } else {    // the same stencil on every plane: constant-bank operands
            c0 = a.cw[d][0], c1 = a.cw[d][1], c2 = a.cw[d][2], c3 = a.cw[d][3];
            hds = a.hds[d], wd = a.w[d], off = a.off[d];
        }
        const float *Id = It + d * tsz;
        // the thread's two points are vertically adjacent: their corner rows overlap, so three
        // rows of intensity corners and (S, alpha) pairs serve both
        const int o = slot[0] + off;
        const float ic[3][2] = {{Id[o], Id[o + 1]},
                                {Id[o + TL_PW], Id[o + TL_PW + 1]},
                                {Id[o + 2 * TL_PW], Id[o + 2 * TL_PW + 1]}};
        const float4 pc[3] = {SA[o], SA[o + TL_PW], SA[o + 2 * TL_PW]};   // (S, alpha) at x, x + 1
#pragma unroll
        for (int m = 0; m < TL_PPT; ++m) {
            const float iu = c0 * ic[m][0] + c1 * ic[m][1] + c2 * ic[m + 1][0] + c3 * ic[m + 1][1];
            const float4 p0 = pc[m], p1 = pc[m + 1];
            const float su = c0 * p0.x + c1 * p0.z + c2 * p1.x + c3 * p1.z;
            const float au = c0 * p0.y + c1 * p0.w + c2 * p1.y + c3 * p1.w;
            const float dt = (au + ak[m]) * hds;
            float ex, w0, w1;
            if (THICK) lin_weights_thick(dt, ex, w0, w1);
            else lin_weights(dt, ex, w0, w1);
            const float v = iu * ex + w0 * su + w1 * Sk[m];
            if (ok[m]) {
                float *dst = In + d * dstride + m * mstride;
                if (WAVE) __stcg(dst, v);
                else *dst = v;
            }
            jacc[m] += wd * v;
        }
    }
}

// S and alpha of an item's upwind plane into the shared (S, alpha) pairs (slot x holds x and
// x + 1), with halo; returns the smallest alpha this thread staged.  No dependency on other
// items: the persistent kernel issues these loads while it waits for the upwind intensities.
template <int HY>
__device__ __forceinline__ float tile_stage_sa(const TileArgs &a, const PlaneCtx &c, int l, int x0,
                                               int y0, float *smt, int ndh)
{
    const int hy = HY > 0 ? HY : a.hy;
    const int ph = TL_H + 2 * hy, tsz = TL_PW * ph, q4 = TL_PW / 4;
    float4 *SA = reinterpret_cast<float4 *>(smt + (size_t)ndh * tsz);
    const size_t npt = (size_t)a.np * a.nz;
    const float *Su = a.S + (size_t)l * npt + (size_t)c.ku * a.np;
    const float *Au = a.alpha + (size_t)l * npt + (size_t)c.ku * a.np;
    float amin = __int_as_float(0x7f800000);
    for (int e = threadIdx.x; e < ph * q4; e += TL_THREADS) {
        const int r = e / q4, c4 = e % q4;
        const int gy = wrapi(y0 - hy + r, a.ny, a.wrap1);
        const int gx = wrapi(x0 - TL_HXP + 4 * c4, a.nx, a.wrap1);
        const int gx4 = wrapi(gx + 4, a.nx, true);
        const size_t g = (size_t)gy * a.nx + gx, g4 = (size_t)gy * a.nx + gx4;
        const float4 sv = __ldg(reinterpret_cast<const float4 *>(Su + g));
        const float4 av = __ldg(reinterpret_cast<const float4 *>(Au + g));
        const float s4 = __ldg(Su + g4), a4 = __ldg(Au + g4);
        float4 *sa = SA + r * TL_PW + 4 * c4;
        sa[0] = make_float4(sv.x, av.x, sv.y, av.y);
        sa[1] = make_float4(sv.y, av.y, sv.z, av.z);
        sa[2] = make_float4(sv.z, av.z, sv.w, av.w);
        sa[3] = make_float4(sv.w, av.w, s4, a4);
        amin = fminf(amin, fminf(fminf(av.x, av.y), fminf(av.z, av.w)));
    }
    return amin;
}

// One (tile, wavelength) item of one plane step.  WAVE selects the persistent kernel's variant:
// L2-coherent loads of the upwind intensities (planes written by other blocks of the same launch,
// which the non-coherent read-only path could serve stale) and its tile-major intensity ring
// [nlam][ntiles][ndh][TL_H][TL_W]; otherwise the ring is [nlam][ndh][nx * ny].  PP: the plane's
// stencils come from the table gst (copied to the shared sts), else from the arguments.
// SA_DONE: the (S, alpha) pairs were staged before (tile_stage_sa), amin_in their minimum alpha.
template <int NDH, bool WAVE, bool PP, int HY = 0, bool SA_DONE = false>
__device__ __forceinline__ void tile_item(const TileArgs &a, const PlaneCtx &c, int l, int tile,
                                          int x0, int y0, float *smt, const WaveSt *gst,
                                          WaveSt *sts, float amin_in = 0.f)
{
    const int ndh = NDH > 0 ? NDH : a.ndh;
    const int hy = HY > 0 ? HY : a.hy;                       // compile-time where HY > 0
    const int ph = TL_H + 2 * hy;
    const int tsz = TL_PW * ph;                              // slots per staged tile
    float *It = smt;                                         // [ndh][ph][TL_PW]
    float4 *SA = reinterpret_cast<float4 *>(smt + (size_t)ndh * tsz);   // [ph][TL_PW]
    const int tid = threadIdx.x;
    const int lx = tid % TL_W, ly = tid / TL_W;              // ly in 0..TL_ROWS-1
    const size_t npt = (size_t)a.np * a.nz;
    const int q4 = TL_PW / 4;                                // float4 per staged row
    const float *al = a.alpha + (size_t)l * npt, *Sl = a.S + (size_t)l * npt;
    const float *Su = Sl + (size_t)c.ku * a.np, *Au = al + (size_t)c.ku * a.np;
    // stage the upwind plane (every direction's intensity, and S with alpha), with halo; slot x
    // of SA holds (S, alpha) at x and x + 1.  A float4 never straddles the periodic seam because
    // nx and x0 - TL_HXP are multiples of 4.  amin: smallest upwind alpha this thread staged.
    // the item's own points: S and alpha on plane k, loaded before the staging (latency overlap)
    int gxy[TL_PPT], slot[TL_PPT];
    float Sk[TL_PPT], ak[TL_PPT], jacc[TL_PPT];
    bool ok[TL_PPT];
#pragma unroll
    for (int m = 0; m < TL_PPT; ++m) {   // rows 2 ly and 2 ly + 1 of the tile
        const int x = x0 + lx, y = y0 + TL_PPT * ly + m;
        ok[m] = x < a.nx && y < a.ny;
        gxy[m] = ok[m] ? y * a.nx + x : 0;
        slot[m] = (TL_PPT * ly + m + hy) * TL_PW + lx + TL_HXP;
        Sk[m] = ok[m] ? __ldg(Sl + (size_t)c.k * a.np + gxy[m]) : 0.f;
        ak[m] = ok[m] ? __ldg(al + (size_t)c.k * a.np + gxy[m]) : 0.f;
        jacc[m] = 0.f;
    }
    if (PP && tid < NDH * 8)
        reinterpret_cast<int *>(sts)[tid] = __ldg(reinterpret_cast<const int *>(gst) + tid);
    const float hds_min = PP ? __ldg(&gst->hds_min) : a.hds_min;
    float amin = SA_DONE ? amin_in : __int_as_float(0x7f800000);
    for (int e = tid; e < ph * q4; e += TL_THREADS) {
        const int r = e / q4, c4 = e % q4;
        const int gy = wrapi(y0 - hy + r, a.ny, a.wrap1);
        const int gx = wrapi(x0 - TL_HXP + 4 * c4, a.nx, a.wrap1);
        const size_t g = (size_t)gy * a.nx + gx;
        if (!SA_DONE) {
            const int gx4 = wrapi(gx + 4, a.nx, true);
            const size_t g4 = (size_t)gy * a.nx + gx4;
            const float4 sv = __ldg(reinterpret_cast<const float4 *>(Su + g));
            const float4 av = __ldg(reinterpret_cast<const float4 *>(Au + g));
            const float s4 = __ldg(Su + g4), a4 = __ldg(Au + g4);
            float4 *sa = SA + r * TL_PW + 4 * c4;
            sa[0] = make_float4(sv.x, av.x, sv.y, av.y);
            sa[1] = make_float4(sv.y, av.y, sv.z, av.z);
            sa[2] = make_float4(sv.z, av.z, sv.w, av.w);
            sa[3] = make_float4(sv.w, av.w, s4, a4);
            amin = fminf(amin, fminf(fminf(av.x, av.y), fminf(av.z, av.w)));
        }
        const float *src0;
        size_t dstep;
        if (WAVE) {
            const int tt = (gy / TL_H) * a.tiles_x + gx / TL_W;
            src0 = c.Iprev + (((size_t)l * a.ntiles + tt) * ndh) * (TL_W * TL_H) +
                   (gy % TL_H) * TL_W + gx % TL_W;
            dstep = TL_W * TL_H;
        } else {
            src0 = c.Iprev + (size_t)l * ndh * a.np + g;
            dstep = a.np;
        }
#pragma unroll
        for (int d = 0; d < (NDH > 0 ? NDH : TL_MAX_DH); ++d) {
            if (NDH == 0 && d >= ndh) break;
            const float4 *src = reinterpret_cast<const float4 *>(src0 + d * dstep);
            const float4 iv = WAVE ? __ldcg(src) : __ldg(src);
            reinterpret_cast<float4 *>(It + d * tsz + r * TL_PW)[c4] = iv;
        }
    }
    // d = (alpha_up + alpha_k) * hds >= amin * hds_min: the whole item is thick when every
    // thread's staged alpha clears the bound (the barrier that publishes the tile decides it);
    // the 1e-4 margin covers the rounding of the interpolated alpha, so that an interval the
    // general path would send to the series never takes the exact formula
    const bool thick = __syncthreads_and(amin * hds_min >= 0.1f * 1.0001f);
    float *In;
    size_t dstride, mstride;
    if (WAVE) {
        In = c.Inext + ((size_t)l * a.ntiles + tile) * ndh * (TL_W * TL_H) + TL_PPT * ly * TL_W + lx;
        dstride = TL_W * TL_H;
        mstride = TL_W;
    } else {
        In = c.Inext + (size_t)l * ndh * a.np + gxy[0];
        dstride = a.np;
        mstride = (size_t)a.nx;
    }
    if (thick)
        tile_updates<NDH, WAVE, true, PP>(a, sts, It, SA, tsz, slot, Sk, ak, ok, In, dstride,
                                          mstride, jacc);
    else
        tile_updates<NDH, WAVE, false, PP>(a, sts, It, SA, tsz, slot, Sk, ak, ok, In, dstride,
                                           mstride, jacc);
#pragma unroll
    for (int m = 0; m < TL_PPT; ++m) {
        if (!ok[m]) continue;
        float *Jp = a.J + (size_t)l * npt + (size_t)c.k * a.np + gxy[m];
        const float v = c.first ? jacc[m] : (WAVE ? __ldcg(Jp) : *Jp) + jacc[m];
        if (!isfinite(v)) flag_error(a.err, ERR_NAN);
        if (WAVE) __stcg(Jp, v);
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
        const int l = item / a.ntiles, tile = item % a.ntiles;
        tile_item<NDH, false, false>(a, c, l, tile, (tile % a.tiles_x) * TL_W,
                                     (tile / a.tiles_x) * TL_H, smt, nullptr, nullptr);
    }
}

// Boundary plane of one tile and wavelength (persistent kernel): the rule for every direction
// into the tile-major ring, and J.
template <int NDH>
__device__ __forceinline__ void boundary_item(const TileArgs &a, const PlaneCtx &c, int l, int tile,
                                              int x0, int y0, int bc)
{
    const int ndh = NDH > 0 ? NDH : a.ndh;
    const size_t npt = (size_t)a.np * a.nz;
    float *In = c.Inext + ((size_t)l * a.ntiles + tile) * ndh * (TL_W * TL_H);
    for (int e = threadIdx.x; e < TL_W * TL_H; e += TL_THREADS) {
        const int x = x0 + e % TL_W, y = y0 + e / TL_W;
        if (x >= a.nx || y >= a.ny) continue;
        const int q = y * a.nx + x;
        const float Sk = __ldg(a.S + (size_t)l * npt + (size_t)c.k * a.np + q);
        const float v = (bc == RT_BC_THERMAL && c.up) ? Sk : 0.f;
        float jacc = 0.f;
        for (int d = 0; d < ndh; ++d) {
            __stcg(In + (size_t)d * (TL_W * TL_H) + e, v);
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
    const WaveSt *st;          // [nz][2][12] per-plane stencils (non-uniform z), else null
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

struct WaveItem {
    int item, h, s, l, tile, x0, y0, pad;
};

// Item order of the persistent sweeps: hemisphere, then chunks of `lchunk` wavelengths (the last
// may be shorter), then plane step, wavelength within the chunk, tile.  A chunk goes through all
// planes before the next starts, which bounds the intensity ring that must stay in L2 between a
// step and the next to lchunk x tiles items.  Every item's dependencies (previous step of the
// same wavelength; the upward item of the same plane) come earlier in this order.
__device__ __forceinline__ WaveItem wave_decode(const TileArgs &a, int item)
{
    const int nt = a.ntiles, nl = a.nlam, nz = a.nz, lc = a.lchunk;
    const int per_hemi = nz * nl * nt;
    WaveItem it;
    it.item = item;
    it.h = item / per_hemi;
    int rem = item - it.h * per_hemi;
    const int per_chunk = nz * lc * nt, full = nl / lc;
    int c = rem / per_chunk;
    if (c > full) c = full;
    const int l0 = c * lc, lcc = c < full ? lc : nl - l0;
    rem -= c * per_chunk;
    it.s = rem / (lcc * nt);
    rem -= it.s * (lcc * nt);
    it.l = l0 + rem / nt;
    it.tile = rem % nt;
    it.x0 = (it.tile % a.tiles_x) * TL_W;
    it.y0 = (it.tile / a.tiles_x) * TL_H;
    it.pad = 0;
    return it;
}

// PP: per-plane stencils from the table (non-uniform z); else the constant-bank stencils.
// HY > 0: the stencil reach in rows, fixed at compile time (shared-memory offsets become
// immediates); 0: from the arguments.
template <int NDH, bool PP, int HY>
__global__ void __launch_bounds__(TL_THREADS, 2) sc_wave_kernel(WaveArgs w)
{
    extern __shared__ __align__(16) float smt[];
    __shared__ WaveItem cur;
    __shared__ __align__(16) WaveSt sts[PP ? NDH : 1];
    const TileArgs &a = w.t[0];
    const int nt = a.ntiles, nl = a.nlam, nz = a.nz;
    const int total = 2 * nz * nl * nt;
    const int tx = a.tiles_x, ty = nt / a.tiles_x;
    if (threadIdx.x == 0) cur = wave_decode(a, atomicAdd(w.queue, 1));
    __syncthreads();
    for (;;) {
        const WaveItem it = cur;   // published by the barrier that ended the previous item
        if (it.item >= total) return;
        int next = 0;
        if (threadIdx.x == 0) next = atomicAdd(w.queue, 1);
        const int h = it.h, s = it.s, l = it.l, tile = it.tile;
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
        // S and alpha of the upwind plane depend on no other item: staged while warp 0 waits
        const float amin = s > 0 ? tile_stage_sa<HY>(w.t[0], c, l, it.x0, it.y0, smt, NDH) : 0.f;
        __syncthreads();
        if (PP) {
            // one code copy for both hemispheres: the stencils and weights come from the table
            if (s == 0) boundary_item<NDH>(w.t[h], c, l, tile, it.x0, it.y0, w.bc);
            else tile_item<NDH, true, true, HY, true>(w.t[0], c, l, tile, it.x0, it.y0, smt,
                                                      w.st + ((size_t)k * 2 + h) * NDH, sts, amin);
        } else if (h == 0) {
            // one inlined copy per hemisphere keeps every per-direction constant a static operand
            if (s == 0) boundary_item<NDH>(w.t[0], c, l, tile, it.x0, it.y0, w.bc);
            else tile_item<NDH, true, false, HY, true>(w.t[0], c, l, tile, it.x0, it.y0, smt,
                                                       nullptr, nullptr, amin);
        } else {
            if (s == 0) boundary_item<NDH>(w.t[1], c, l, tile, it.x0, it.y0, w.bc);
            else tile_item<NDH, true, false, HY, true>(w.t[1], c, l, tile, it.x0, it.y0, smt,
                                                       nullptr, nullptr, amin);
        }
        // every thread read `cur` before the dependency barrier above, so the next item can be
        // published now, by the barrier that also ends this one
        if (threadIdx.x == 0) cur = wave_decode(a, next);
        __syncthreads();
        if (threadIdx.x == 0) {
            int *f = w.done + ((size_t)(h * nz + s) * nl + l) * nt + tile;
            asm volatile("st.release.gpu.global.b32 [%0], %1;" :: "l"(f), "r"(1) : "memory");
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

// The staged tile covers every stencil: periodic x and y, nx a multiple of 4 (16-byte rows),
// corner reach within the x halo and at most 8 rows in y.
static bool tile_geometry(const rt_grid *g, int &hy)
{
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

static bool tile_plan(const rt_grid *g, int &hy)
{
    const char *env = std::getenv("RT_REGULAR_SWEEP");
    if (env && (std::string(env) == "plane" || std::string(env) == "cluster")) return false;
    return tile_geometry(g, hy);
}

template <int NDH>
static rt_status launch_planes(rt_grid *g, TileArgs &a, const std::vector<int> &dirs, int bc,
                               int nlam, float **bufs, cudaStream_t st)
{
    const int ph = TL_H + 2 * a.hy, tsz = TL_PW * ph;
    const size_t smem = ((size_t)a.ndh * tsz) * sizeof(float) + (size_t)tsz * sizeof(float4);
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
            a.hds_min = d == 0 ? sc.hds : std::min(a.hds_min, sc.hds);
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

static rt_status pipe_sweep(rt_grid *g, const WaveArgs &wv, int nlam, cudaStream_t st, bool *done);
static bool pipe_geometry(const rt_grid *g, int hy);
static size_t pipe_scratch(const rt_grid *g, int nlam, int hy);

size_t regular_wave_scratch(const rt_grid *g, int nlam)
{
    const size_t ntiles = (size_t)((g->nx + TL_W - 1) / TL_W) * ((g->ny + TL_H - 1) / TL_H);
    const size_t plane = (size_t)nlam * ntiles * 12 * TL_W * TL_H;   // tile-major ring slot
    const size_t nflags = 2 * (size_t)g->nz * nlam * ntiles;
    size_t bytes = 4 * plane * sizeof(float) + (nflags + 64) * sizeof(int);
    int hy;
    if (tile_geometry(g, hy) && pipe_geometry(g, hy)) bytes = std::max(bytes, pipe_scratch(g, nlam, hy));
    return bytes;
}

rt_status regular_wave_prepare(rt_grid *g, cudaStream_t st)
{
    int hy;
    if (!tile_geometry(g, hy) || g->dir_up.size() != 12 || g->dir_dn.size() != 12 || g->nz < 3)
        return RT_OK;
    std::vector<WaveSt> t((size_t)g->nz * 2 * 12, WaveSt{0, 0, 0, 0, 0, 0, 0, 0});
    const std::vector<int> *hs[2] = {&g->dir_up, &g->dir_dn};
    for (int k = 0; k < g->nz; ++k)
        for (int h = 0; h < 2; ++h) {
            if ((h == 0 && k == 0) || (h == 1 && k == g->nz - 1)) continue;   // boundary planes
            WaveSt *e = &t[((size_t)k * 2 + h) * 12];
            float hmin = 0.f;
            for (int d = 0; d < 12; ++d) {
                const int q = (*hs[h])[d];
                const Stencil &sc = g->h_stencil[(size_t)k * g->ndir + q];
                e[d].c0 = sc.w0;
                e[d].c1 = sc.w1;
                e[d].c2 = sc.w2;
                e[d].c3 = sc.w3;
                e[d].hds = sc.hds;
                e[d].wd = (float)g->wdir[q];
                e[d].off = sc.ay * TL_PW + sc.ax;
                hmin = d == 0 ? sc.hds : std::min(hmin, sc.hds);
            }
            for (int d = 0; d < 12; ++d) e[d].hds_min = hmin;
        }
    g->h_wave_st.resize(t.size() * sizeof(WaveSt));
    std::memcpy(g->h_wave_st.data(), t.data(), g->h_wave_st.size());
    RT_CUDA(cudaMalloc(&g->d_wave_st, g->h_wave_st.size()));
    RT_CUDA(cudaMemcpyAsync(g->d_wave_st, g->h_wave_st.data(), g->h_wave_st.size(),
                            cudaMemcpyHostToDevice, st));
    return RT_OK;
}

static rt_status wave_sweep(rt_grid *g, TileArgs &base, int nlam, int bc, cudaStream_t st,
                            bool *done)
{
    const char *env = std::getenv("RT_REGULAR_SWEEP");
    if (env && std::string(env) == "tile") return RT_OK;   // per-plane launches requested
    if (g->dir_up.size() != 12 || g->dir_dn.size() != 12 || g->nz < 3) return RT_OK;
    const bool pp = !uniform_stencils(g);
    if (pp && !g->d_wave_st) return RT_OK;
    WaveArgs w;
    w.st = pp ? static_cast<const WaveSt *>(g->d_wave_st) : nullptr;
    const std::vector<int> *hs[2] = {&g->dir_up, &g->dir_dn};
    for (int h = 0; h < 2; ++h) {
        TileArgs &a = w.t[h];
        a = base;
        a.ndh = 12;
        a.up = h == 0;
        // uniform z: every plane shares this stencil (otherwise the table holds them)
        const int kref = h == 0 ? 1 : g->nz - 2;
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
            a.hds_min = d == 0 ? sc.hds : std::min(a.hds_min, sc.hds);
        }
        w.nd[h] = 12;
    }
    w.bc = bc;
    w.first_hemi = 0;
    {
        // wavelengths per chunk: enough items per plane step (about 1.5 per resident block at
        // two blocks per SM) that an item's neighbours of the previous step are normally done
        // when it is claimed, and no more, so that the intensity ring of the chunk stays in L2;
        // chunks of equal size (a short last chunk starves the blocks).  At 128 x 128 and 52
        // wavelengths: two chunks of 26.  RT_WAVE_LCHUNK overrides (tuning).
        int dev = 0, nsm = 0;
        RT_CUDA(cudaGetDevice(&dev));
        RT_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
        const int target = std::max(1, (3 * nsm + base.ntiles - 1) / base.ntiles);
        const int nch = std::max(1, (nlam + target / 2) / target);
        int lc = (nlam + nch - 1) / nch;
        if (const char *e = std::getenv("RT_WAVE_LCHUNK")) lc = std::atoi(e);
        lc = std::max(1, std::min(nlam, lc));
        w.t[0].lchunk = w.t[1].lchunk = lc;
    }
    RT_TRY(pipe_sweep(g, w, nlam, st, done));
    if (*done) return RT_OK;
    const size_t plane = (size_t)nlam * base.ntiles * 12 * TL_W * TL_H;
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
    const int ph = TL_H + 2 * base.hy, tsz = TL_PW * ph;
    const size_t smem = (12 * (size_t)tsz) * sizeof(float) + (size_t)tsz * sizeof(float4);
    void (*kern)(WaveArgs);
    switch (base.hy * 2 + (pp ? 1 : 0)) {
    case 2: kern = sc_wave_kernel<12, false, 1>; break;
    case 3: kern = sc_wave_kernel<12, true, 1>; break;
    case 4: kern = sc_wave_kernel<12, false, 2>; break;
    case 5: kern = sc_wave_kernel<12, true, 2>; break;
    case 6: kern = sc_wave_kernel<12, false, 3>; break;
    case 7: kern = sc_wave_kernel<12, true, 3>; break;
    case 8: kern = sc_wave_kernel<12, false, 4>; break;
    case 9: kern = sc_wave_kernel<12, true, 4>; break;
    default: kern = pp ? sc_wave_kernel<12, true, 0> : sc_wave_kernel<12, false, 0>; break;
    }
    RT_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0, dev = 0, nsm = 0;
    RT_CUDA(cudaGetDevice(&dev));
    RT_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    RT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, TL_THREADS, smem));
    if (per_sm < 1) return RT_OK;
    RT_CUDA(cudaMemsetAsync(w.queue, 0, (nflags + 32) * sizeof(int), st));
    note_launch();
    kern<<<per_sm * nsm, TL_THREADS, smem, st>>>(w);
    RT_CUDA(cudaGetLastError());
    *done = true;
    return RT_OK;
}

// ---- Pipelined persistent sweep ------------------------------------------------------------------
//
// The wavefront schedule of sc_wave_kernel with the staging of the next item overlapped with the
// computation of the current one.  One block of 512 threads per SM holds two staging buffers.
// The intensity ring is tile major with each tile's halo stored beside it,
// [nlam][tile][12][PH][TL_PW], so the 12 upwind planes an item needs are one contiguous block:
// a single cp.async.bulk (the TMA engine, completion counted on an mbarrier) brings it into
// shared memory.  S and alpha of the upwind plane (caller's arrays, periodic wrap) arrive by
// 16-byte cp.async and are interleaved into (S, alpha) pairs for x and x + 1 after landing.
// Writers store each point into its own tile's region and, near a tile edge, into the halo of
// the neighbouring tile(s).  Applies to planes whose sides are multiples of 32 (at least 64) and
// stencils within HY <= 4 rows.
//
// Ordering: an item's intensities are requested only once its 3 x 3 neighbours of the previous
// step are complete.  The request for the next item is attempted (without waiting) while the
// current one is computed; if the neighbours are not complete yet, it is made after the current
// item is published.  A block only ever waits for items that precede, in counter order, every
// item it holds, so by induction on the smallest unfinished item the waits cannot deadlock.
// All waits are bounded (ERR_TIMEOUT).
constexpr int PL_THREADS = 512;

struct PipeArgs {
    TileArgs t[2];             // per hemisphere (uniform z: the stencils as in sc_wave_kernel)
    const WaveSt *st;          // [nz][2][12] per-plane stencils (non-uniform z), else null
    float *ring[2][2];         // [hemisphere][step parity] padded tile-major planes
    int *queue;
    int *done;                 // [2][nz][nlam][ntiles] completion flags
    int bc, first_hemi;
};

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *m, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(m)), "r"(parity)
        : "memory");
    return ok != 0;
}

// bounded wait for phase `parity` of an mbarrier to complete
__device__ __forceinline__ bool mbar_wait(uint64_t *m, uint32_t parity)
{
    for (int it = 0; it < (1 << 20); ++it)
        if (mbar_try_wait(m, parity)) return true;
    return false;
}

// one thread: announce `bytes` on the mbarrier and start the bulk copy global -> shared
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *m)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                 :: "r"(smem_addr(m)), "r"(bytes) : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        :: "r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(m)) : "memory");
}

__device__ __forceinline__ void cp_async16(void *dst, const void *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" :: "r"(smem_addr(dst)), "l"(src)
                 : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" :: "n"(N) : "memory"); }

// flag index of item (h, s, l, tile)
__device__ __forceinline__ size_t flag_at(const TileArgs &a, int h, int s, int l, int tile)
{
    return ((size_t)(h * a.nz + s) * a.nlam + l) * a.ntiles + tile;
}

// lanes 0..8 of one warp: the 3 x 3 neighbour flags of item `it` at its previous step.
// blocking = false: one look; true: bounded wait.  Returns the warp-wide "all complete".
__device__ __forceinline__ bool deps_ready(const PipeArgs &w, const WaveItem &it, bool blocking)
{
    const TileArgs &a = w.t[0];
    const int lane = threadIdx.x & 31;
    bool ok = true;
    if (lane < 9) {
        const int tx = a.tiles_x, ty = a.ntiles / a.tiles_x;
        const int tx0 = it.tile % tx, ty0 = it.tile / tx;
        const int nx_ = (tx0 + lane % 3 - 1 + tx) % tx, ny_ = (ty0 + lane / 3 - 1 + ty) % ty;
        const int *f = w.done + flag_at(a, it.h, it.s - 1, it.l, ny_ * tx + nx_);
        if (blocking) {
            ok = wait_flag(f, a.err);
        } else {
            int v;
            asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(f) : "memory");
            ok = v != 0;
        }
    }
    return __all_sync(0xffffffffu, ok);
}

// S and alpha of item `it`'s upwind plane into raw[0] (S) and raw[TSZ] (alpha), and of its own
// points into own[0] and own[TL_W * TL_H]: 16-byte copies
template <int HY>
__device__ __forceinline__ void stage_sa_async(const TileArgs &a, const WaveItem &it, float *raw,
                                               float *own)
{
    constexpr int PH = TL_H + 2 * HY, TSZ = PH * TL_PW, Q4 = TL_PW / 4;
    const bool up = it.h == 0;
    const int k = up ? it.s : a.nz - 1 - it.s;
    const int ku = up ? k - 1 : k + 1;
    const size_t npt = (size_t)a.np * a.nz;
    const float *Sl = a.S + (size_t)it.l * npt, *Al = a.alpha + (size_t)it.l * npt;
    const float *Su = Sl + (size_t)ku * a.np, *Au = Al + (size_t)ku * a.np;
    for (int e = threadIdx.x; e < PH * Q4; e += PL_THREADS) {
        const int r = e / Q4, c4 = e % Q4;
        const int gy = wrapi(it.y0 - HY + r, a.ny, true);
        const int gx = wrapi(it.x0 - TL_HXP + 4 * c4, a.nx, true);
        const size_t g = (size_t)gy * a.nx + gx;
        cp_async16(raw + r * TL_PW + 4 * c4, Su + g);
        cp_async16(raw + TSZ + r * TL_PW + 4 * c4, Au + g);
    }
    if (threadIdx.x < TL_H * TL_W / 4) {
        const int r = threadIdx.x / (TL_W / 4), c4 = threadIdx.x % (TL_W / 4);
        const size_t g = (size_t)k * a.np + (size_t)(it.y0 + r) * a.nx + it.x0 + 4 * c4;
        cp_async16(own + r * TL_W + 4 * c4, Sl + g);
        cp_async16(own + TL_W * TL_H + r * TL_W + 4 * c4, Al + g);
    }
}

// where a thread's point (row yl of the tile, column lx) is stored in the padded ring, as offsets
// from the ring slot's wavelength base: its own tile's region and, near a tile edge, the halo of
// the neighbouring tile(s); -1 where there is no such copy
template <int HY>
struct RingDst {
    int own, xc, yc, cc;
};

template <int HY>
__device__ __forceinline__ RingDst<HY> ring_dst(const TileArgs &a, int tile, int lx, int yl)
{
    constexpr int PH = TL_H + 2 * HY, TSZ = PH * TL_PW, REG = 12 * TSZ;
    const int tx = a.tiles_x, ty = a.ntiles / a.tiles_x;
    const int tx0 = tile % tx, ty0 = tile / tx;
    RingDst<HY> r;
    r.own = tile * REG + (yl + HY) * TL_PW + lx + TL_HXP;
    int ntx = -1, col = 0, nty = -1, row = 0;
    if (lx < TL_HXP) ntx = (tx0 + tx - 1) % tx, col = lx + TL_W + TL_HXP;
    else if (lx >= TL_W - TL_HXP) ntx = (tx0 + 1) % tx, col = lx - (TL_W - TL_HXP);
    if (yl < HY) nty = (ty0 + ty - 1) % ty, row = yl + TL_H + HY;
    else if (yl >= TL_H - HY) nty = (ty0 + 1) % ty, row = yl - (TL_H - HY);
    r.xc = ntx >= 0 ? (ty0 * tx + ntx) * REG + (yl + HY) * TL_PW + col : -1;
    r.yc = nty >= 0 ? (nty * tx + tx0) * REG + row * TL_PW + lx + TL_HXP : -1;
    r.cc = (ntx >= 0 && nty >= 0) ? (nty * tx + ntx) * REG + row * TL_PW + col : -1;
    return r;
}

template <int HY>
__device__ __forceinline__ void ring_store(float *base, const RingDst<HY> &r, int d, float v)
{
    constexpr int TSZ = (TL_H + 2 * HY) * TL_PW;
    __stcg(base + r.own + d * TSZ, v);
    if (r.xc >= 0) __stcg(base + r.xc + d * TSZ, v);
    if (r.yc >= 0) {
        __stcg(base + r.yc + d * TSZ, v);
        if (r.cc >= 0) __stcg(base + r.cc + d * TSZ, v);
    }
}

template <int HY, bool PP>
__global__ void __launch_bounds__(PL_THREADS, 1) sc_pipe_kernel(PipeArgs w)
{
    constexpr int PH = TL_H + 2 * HY, TSZ = PH * TL_PW, REG = 12 * TSZ, NP = TL_W * TL_H;
    extern __shared__ __align__(128) float smp[];
    float *It = smp;                                             // [2][12][TSZ]
    float *raw = smp + 2 * REG;                                  // [2][2][TSZ] upwind (S, alpha)
    float *own = raw + 4 * TSZ;                                  // [2][2][NP] own plane (S, alpha)
    float4 *SA = reinterpret_cast<float4 *>(own + 4 * NP);       // [TSZ]
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ WaveItem cur_s, nxt_s;
    __shared__ int pf_s[2];   // [b]: the next item's intensities were requested during item b
    __shared__ __align__(16) WaveSt sts[PP ? 12 : 1];
    const TileArgs &a0 = w.t[0];
    const int nt = a0.ntiles, nl = a0.nlam, nz = a0.nz;
    const int total = 2 * nz * nl * nt;
    const int tid = threadIdx.x, lx = tid % TL_W, ly = tid / TL_W;
    const size_t npt = (size_t)a0.np * nz;

    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_addr(&mbar[0])) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_addr(&mbar[1])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        cur_s = wave_decode(a0, atomicAdd(w.queue, 1));
        nxt_s = wave_decode(a0, atomicAdd(w.queue, 1));
        pf_s[0] = pf_s[1] = 0;
    }
    __syncthreads();
    uint32_t phase0 = 0, phase1 = 0;
    int b = 0;
    {
        // the first item: wait for its neighbours (nothing else is held), then request it
        const WaveItem c0 = cur_s;
        if (c0.item >= total) return;
        if (c0.s > 0) {
            if (tid < 32) {
                const bool ok = deps_ready(w, c0, true);
                if (tid == 0) {
                    if (!ok) flag_error(a0.err, ERR_TIMEOUT);
                    asm volatile("fence.proxy.async.global;" ::: "memory");
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    bulk_load(It, w.ring[c0.h][(c0.s + 1) & 1] + ((size_t)c0.l * nt + c0.tile) * REG,
                              REG * sizeof(float), &mbar[0]);
                }
            }
            stage_sa_async<HY>(a0, c0, raw, own);
        }
        cp_async_commit();
    }
    for (;;) {
        // cur_s and nxt_s were written before the barrier that ended the previous item
        const WaveItem cur = cur_s, nxt = nxt_s;
        if (cur.item >= total) break;
        int claim = 0;
        if (tid == 0) {
            claim = atomicAdd(w.queue, 1);
            pf_s[b] = 0;
        }
        const bool nxt_valid = nxt.item < total;
        float *It_c = It + b * REG, *raw_c = raw + b * 2 * TSZ, *own_c = own + b * 2 * NP;
        float *It_n = It + (b ^ 1) * REG;
        // 1. S and alpha of the next item (inputs: no dependency)
        if (nxt_valid && nxt.s > 0) stage_sa_async<HY>(a0, nxt, raw + (b ^ 1) * 2 * TSZ,
                                                       own + (b ^ 1) * 2 * NP);
        cp_async_commit();
        // 2. the current item's staged data
        bool lost = false;
        if (cur.s > 0) {
            lost = !mbar_wait(&mbar[b], b ? phase1 : phase0);
            if (b) phase1 ^= 1u;
            else phase0 ^= 1u;
        }
        cp_async_wait<1>();
        if (__syncthreads_or(lost)) {
            // the bulk copy did not complete: record it, give any copy still in flight a bounded
            // time to land, and leave
            if (tid == 0) {
                flag_error(a0.err, ERR_TIMEOUT);
                if (pf_s[b ^ 1]) mbar_wait(&mbar[b ^ 1], b ? phase0 : phase1);
            }
            cp_async_wait<0>();
            return;
        }
        const bool up = cur.h == 0;
        const int k = up ? cur.s : nz - 1 - cur.s;
        const TileArgs &a = w.t[cur.h];
        // 3. the consumed ring region is dead: drop it from L2 without a write-back; (S, alpha)
        //    pairs; the thick-item vote; per-plane stencils; the J dependency; an attempt to
        //    request the next item's intensities
        float amin = __int_as_float(0x7f800000);
        if (cur.s > 0) {
            {   // REG floats = REG / 32 lines of 128 bytes (the region starts on a line)
                const float *src = w.ring[cur.h][(cur.s + 1) & 1] + ((size_t)cur.l * nt + cur.tile) * REG;
                for (int q = tid; q < REG / 32; q += PL_THREADS)
                    asm volatile("discard.global.L2 [%0], 128;" :: "l"(src + q * 32) : "memory");
            }
            for (int e = tid; e < TSZ; e += PL_THREADS) {
                const int c = e % TL_PW;
                const float s0 = raw_c[e], a0v = raw_c[TSZ + e];
                const float s1 = c + 1 < TL_PW ? raw_c[e + 1] : s0;
                const float a1 = c + 1 < TL_PW ? raw_c[TSZ + e + 1] : a0v;
                SA[e] = make_float4(s0, a0v, s1, a1);
                amin = fminf(amin, a0v);
            }
            if (PP && tid < 12 * 8)
                reinterpret_cast<int *>(sts)[tid] = __ldg(
                    reinterpret_cast<const int *>(w.st + ((size_t)k * 2 + cur.h) * 12) + tid);
        }
        const bool first = cur.h == w.first_hemi;
        if (tid < 32) {
            if (!first) {   // the upward J of this plane and tile is complete
                bool ok = true;
                if (tid == 0) ok = wait_flag(w.done + flag_at(a0, 0, k, cur.l, cur.tile), a0.err);
                ok = __shfl_sync(0xffffffffu, ok, 0);
                if (tid == 0 && !ok) flag_error(a0.err, ERR_TIMEOUT);
            }
            if (nxt_valid && nxt.s > 0 && deps_ready(w, nxt, false)) {
                if (tid == 0) {
                    asm volatile("fence.proxy.async.global;" ::: "memory");
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    bulk_load(It_n, w.ring[nxt.h][(nxt.s + 1) & 1] +
                                        ((size_t)nxt.l * nt + nxt.tile) * REG,
                              REG * sizeof(float), &mbar[b ^ 1]);
                    pf_s[b] = 1;
                }
            }
        }
        const float hds_min = PP ? (cur.s > 0 ? __ldg(&w.st[((size_t)k * 2 + cur.h) * 12].hds_min) : 0.f)
                                 : a.hds_min;
        const bool thick = __syncthreads_and(cur.s > 0 && amin * hds_min >= 0.1f * 1.0001f);
        // 4. the item
        float *ringn = w.ring[cur.h][cur.s & 1] + (size_t)cur.l * nt * REG;
        float jacc[TL_PPT], jold[TL_PPT];
        int gxy[TL_PPT];
        RingDst<HY> dst[TL_PPT];
#pragma unroll
        for (int m = 0; m < TL_PPT; ++m) {
            const int yl = ly + TL_ROWS * m;
            gxy[m] = (cur.y0 + yl) * a0.nx + cur.x0 + lx;
            dst[m] = ring_dst<HY>(a0, cur.tile, lx, yl);
            jacc[m] = 0.f;
            jold[m] = first ? 0.f : __ldcg(a0.J + (size_t)cur.l * npt + (size_t)k * a0.np + gxy[m]);
        }
        if (cur.s == 0) {
            const float *Sl = a0.S + (size_t)cur.l * npt + (size_t)k * a0.np;
#pragma unroll
            for (int m = 0; m < TL_PPT; ++m) {
                const float Sk = __ldg(Sl + gxy[m]);
                const float v = (w.bc == RT_BC_THERMAL && up) ? Sk : 0.f;
#pragma unroll
                for (int d = 0; d < 12; ++d) {
                    ring_store<HY>(ringn, dst[m], d, v);
                    jacc[m] += a.w[d] * v;
                }
            }
        } else {
            float Sk[TL_PPT], ak[TL_PPT];
            int slot[TL_PPT];
#pragma unroll
            for (int m = 0; m < TL_PPT; ++m) {
                const int q = (ly + TL_ROWS * m) * TL_W + lx;
                Sk[m] = own_c[q];
                ak[m] = own_c[NP + q];
                slot[m] = (ly + TL_ROWS * m + HY) * TL_PW + lx + TL_HXP;
            }
            auto body = [&](auto thick_tag) {
                constexpr bool THICK = decltype(thick_tag)::value;
#pragma unroll
                for (int d = 0; d < 12; ++d) {
                    float c0, c1, c2, c3, hds, wd;
                    int off;
                    if (PP) {
                        const float4 q0 = reinterpret_cast<const float4 *>(sts)[2 * d];
                        const float4 q1 = reinterpret_cast<const float4 *>(sts)[2 * d + 1];
                        c0 = q0.x, c1 = q0.y, c2 = q0.z, c3 = q0.w;
                        hds = q1.x, wd = q1.y, off = __float_as_int(q1.z);
                    } else {
                        c0 = a.cw[d][0], c1 = a.cw[d][1], c2 = a.cw[d][2], c3 = a.cw[d][3];
                        hds = a.hds[d], wd = a.w[d], off = a.off[d];
                    }
                    const float *Id = It_c + d * TSZ;
#pragma unroll
                    for (int m = 0; m < TL_PPT; ++m) {
                        const int o = slot[m] + off;
                        const float iu = c0 * Id[o] + c1 * Id[o + 1] + c2 * Id[o + TL_PW] +
                                         c3 * Id[o + TL_PW + 1];
                        const float4 p0 = SA[o], p1 = SA[o + TL_PW];
                        const float su = c0 * p0.x + c1 * p0.z + c2 * p1.x + c3 * p1.z;
                        const float au = c0 * p0.y + c1 * p0.w + c2 * p1.y + c3 * p1.w;
                        const float dt = (au + ak[m]) * hds;
                        float ex, w0, w1;
                        if (THICK) lin_weights_thick(dt, ex, w0, w1);
                        else lin_weights(dt, ex, w0, w1);
                        const float v = iu * ex + w0 * su + w1 * Sk[m];
                        ring_store<HY>(ringn, dst[m], d, v);
                        jacc[m] += wd * v;
                    }
                }
            };
            if (thick) body(std::true_type{});
            else body(std::false_type{});
        }
#pragma unroll
        for (int m = 0; m < TL_PPT; ++m) {
            float *Jp = a0.J + (size_t)cur.l * npt + (size_t)k * a0.np + gxy[m];
            const float v = first ? jacc[m] : jold[m] + jacc[m];
            if (!isfinite(v)) flag_error(a0.err, ERR_NAN);
            __stcg(Jp, v);
        }
        // the ring stores are read next by the bulk copies (async proxy) of other blocks
        asm volatile("fence.proxy.async.global;" ::: "memory");
        if (tid == 0) {   // every thread read cur_s and nxt_s before the first barrier of the item
            cur_s = nxt;
            nxt_s = wave_decode(a0, claim);
        }
        __syncthreads();
        // 5. publish the item; request the next one now if the attempt above found it not ready
        if (tid == 0) {
            int *f = w.done + flag_at(a0, cur.h, cur.s, cur.l, cur.tile);
            asm volatile("st.release.gpu.global.b32 [%0], %1;" :: "l"(f), "r"(1) : "memory");
        }
        if (tid < 32 && !pf_s[b] && nxt_valid && nxt.s > 0) {
            const bool ok = deps_ready(w, nxt, true);
            if (tid == 0) {
                if (!ok) flag_error(a0.err, ERR_TIMEOUT);
                asm volatile("fence.proxy.async.global;" ::: "memory");
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                bulk_load(It_n, w.ring[nxt.h][(nxt.s + 1) & 1] + ((size_t)nxt.l * nt + nxt.tile) * REG,
                          REG * sizeof(float), &mbar[b ^ 1]);
            }
        }
        b ^= 1;
    }
    cp_async_wait<0>();
}

// Scratch of the pipelined sweep: 4 padded ring slots, flags, counter.
static size_t pipe_scratch(const rt_grid *g, int nlam, int hy)
{
    const size_t ntiles = (size_t)(g->nx / TL_W) * (g->ny / TL_H);
    const size_t slot = (size_t)nlam * ntiles * 12 * (TL_H + 2 * hy) * TL_PW;
    const size_t nflags = 2 * (size_t)g->nz * nlam * ntiles;
    return 4 * slot * sizeof(float) + (nflags + 64) * sizeof(int);
}

static bool pipe_geometry(const rt_grid *g, int hy)
{
    return g->nx % TL_W == 0 && g->ny % TL_H == 0 && g->nx >= 2 * TL_W && g->ny >= 2 * TL_H &&
           hy >= 1 && hy <= 4;
}

static bool pipe_applies(const rt_grid *g, int hy)
{
    const char *env = std::getenv("RT_REGULAR_SWEEP");   // opt-in: RT_REGULAR_SWEEP=pipe
    return env && std::string(env) == "pipe" && pipe_geometry(g, hy);
}

template <int HY, bool PP>
static rt_status launch_pipe(PipeArgs &w, cudaStream_t st)
{
    constexpr int PH = TL_H + 2 * HY, TSZ = PH * TL_PW;
    const size_t smem = (size_t)(2 * 12 * TSZ + 4 * TSZ + 4 * TL_W * TL_H) * sizeof(float) +
                        (size_t)TSZ * sizeof(float4);
    RT_CUDA(cudaFuncSetAttribute(sc_pipe_kernel<HY, PP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem));
    int per_sm = 0, dev = 0, nsm = 0;
    RT_CUDA(cudaGetDevice(&dev));
    RT_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    RT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sc_pipe_kernel<HY, PP>, PL_THREADS,
                                                          smem));
    if (per_sm < 1) return fail(RT_ECAPACITY, "pipelined sweep cannot be resident");
    note_launch();
    sc_pipe_kernel<HY, PP><<<per_sm * nsm, PL_THREADS, smem, st>>>(w);
    RT_CUDA(cudaGetLastError());
    return RT_OK;
}

static rt_status pipe_sweep(rt_grid *g, const WaveArgs &wv, int nlam, cudaStream_t st, bool *done)
{
    const int hy = wv.t[0].hy;
    if (!pipe_applies(g, hy)) return RT_OK;
    const bool pp = wv.st != nullptr;
    PipeArgs w;
    w.t[0] = wv.t[0];
    w.t[1] = wv.t[1];
    w.st = wv.st;
    w.bc = wv.bc;
    w.first_hemi = wv.first_hemi;
    const size_t ntiles = (size_t)wv.t[0].ntiles;
    const size_t slot = (size_t)nlam * ntiles * 12 * (TL_H + 2 * hy) * TL_PW;
    const size_t nflags = 2 * (size_t)g->nz * nlam * ntiles;
    void *p;
    RT_TRY(scratch_get(g, 3, pipe_scratch(g, nlam, hy), &p));
    float *f = (float *)p;
    w.ring[0][0] = f;
    w.ring[0][1] = f + slot;
    w.ring[1][0] = f + 2 * slot;
    w.ring[1][1] = f + 3 * slot;
    w.queue = (int *)(f + 4 * slot);
    w.done = w.queue + 32;
    RT_CUDA(cudaMemsetAsync(w.queue, 0, (nflags + 32) * sizeof(int), st));
    rt_status r;
    switch (hy * 2 + (pp ? 1 : 0)) {
    case 2: r = launch_pipe<1, false>(w, st); break;
    case 3: r = launch_pipe<1, true>(w, st); break;
    case 4: r = launch_pipe<2, false>(w, st); break;
    case 5: r = launch_pipe<2, true>(w, st); break;
    case 6: r = launch_pipe<3, false>(w, st); break;
    case 7: r = launch_pipe<3, true>(w, st); break;
    case 8: r = launch_pipe<4, false>(w, st); break;
    default: r = launch_pipe<4, true>(w, st); break;
    }
    RT_TRY(r);
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
    a.lchunk = nlam;
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
