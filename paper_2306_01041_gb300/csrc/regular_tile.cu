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
// Two schedules of the same items: sc_wave_kernel (default) runs the whole formal solution as
// one persistent launch ordered by a device counter and per-item completion flags;
// sc_tile_kernel launches once per plane step.
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

// Per-point updates of one staged item for every direction.  THICK: every interval of the item
// has d >= 0.1, so only the exact interval weights are evaluated.  The thread's two points (tile
// rows R and R + 1) share every per-direction coefficient, so their arithmetic runs as packed
// FP32 pairs (component 0: row R, component 1: row R + 1), in the operation order of the scalar
// forms: iu = c0 I00 + c1 I01 + c2 I10 + c3 I11 (a product, then fused multiply-adds), the same
// for S and alpha, dtau = (alpha_up + alpha) hds, I = iu e^-d + w0 S_up + w1 S, J += w I.
// The staged (S, alpha) element at (row q, x) holds S and alpha at x and x + 1, so three 16-byte
// loads (rows q .. q + 2) give every S and alpha corner of both points.
template <int NDH, bool WAVE, bool THICK, bool PP>
__device__ __forceinline__ void tile_updates(const TileArgs &a, const WaveSt *sts, const float *It,
                                             const float4 *SA, int tsz, const int (&slot)[TL_PPT],
                                             const float (&Sk)[TL_PPT], const float (&ak)[TL_PPT],
                                             const bool (&ok)[TL_PPT], float *In, size_t dstride,
                                             size_t mstride, float (&jacc)[TL_PPT])
{
    const int ndh = NDH > 0 ? NDH : a.ndh;
    const float2 Sk2 = make_float2(Sk[0], Sk[1]), ak2 = make_float2(ak[0], ak[1]);
    float2 j2 = make_float2(jacc[0], jacc[1]);
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
        const int o = slot[0] + off;
        // three rows of intensity corners serve both points
        const float i00 = Id[o], i01 = Id[o + 1];
        const float i10 = Id[o + TL_PW], i11 = Id[o + TL_PW + 1];
        const float i20 = Id[o + 2 * TL_PW], i21 = Id[o + 2 * TL_PW + 1];
        float2 iu = mul2(f2(c0), make_float2(i00, i10));
        iu = fma2(f2(c1), make_float2(i01, i11), iu);
        iu = fma2(f2(c2), make_float2(i10, i20), iu);
        iu = fma2(f2(c3), make_float2(i11, i21), iu);
        // (S, alpha) at x and x + 1 of three rows: rows 0-1 serve the first point, 1-2 the second
        const float4 p0 = SA[o], p1 = SA[o + TL_PW], p2 = SA[o + 2 * TL_PW];
        float2 su = mul2(f2(c0), make_float2(p0.x, p1.x));
        su = fma2(f2(c1), make_float2(p0.z, p1.z), su);
        su = fma2(f2(c2), make_float2(p1.x, p2.x), su);
        su = fma2(f2(c3), make_float2(p1.z, p2.z), su);
        float2 au = mul2(f2(c0), make_float2(p0.y, p1.y));
        au = fma2(f2(c1), make_float2(p0.w, p1.w), au);
        au = fma2(f2(c2), make_float2(p1.y, p2.y), au);
        au = fma2(f2(c3), make_float2(p1.w, p2.w), au);
        const float2 dt = mul2(add2(au, ak2), f2(hds));
        float2 ex, w0, w1;
        if (THICK) {
            lin_weights_thick2(dt, ex, w0, w1);
        } else {
            lin_weights(dt.x, ex.x, w0.x, w1.x);
            lin_weights(dt.y, ex.y, w0.y, w1.y);
        }
        float2 v = mul2(iu, ex);
        v = fma2(w0, su, v);
        v = fma2(w1, Sk2, v);
        const float vv[2] = {v.x, v.y};
#pragma unroll
        for (int m = 0; m < TL_PPT; ++m) {
            if (ok[m]) {
                float *dst = In + d * dstride + m * mstride;
                if (WAVE) __stcg(dst, vv[m]);
                else *dst = vv[m];
            }
        }
        j2 = fma2(f2(wd), v, j2);
    }
    jacc[0] = j2.x;
    jacc[1] = j2.y;
}

// S and alpha of an item's upwind plane into the shared (S, alpha) pairs (slot x of row r holds
// (S, alpha) at x and x + 1), with halo; element e covers four slots of row e / (TL_PW / 4) from
// two 16-byte loads and two scalar ones.  A float4 never straddles the periodic seam because nx
// and x0 - TL_HXP are multiples of 4.  Returns the smallest alpha this thread staged.  No
// dependency on other items: the persistent kernel issues these loads while it waits for the
// upwind intensities.
__device__ __forceinline__ float stage_sa_row(const TileArgs &a, const float *Su, const float *Au,
                                              int x0, int y0, int hy, int e, float4 *SA)
{
    const int q4 = TL_PW / 4;
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
    return fminf(fminf(av.x, av.y), fminf(av.z, av.w));
}

template <int HY>
__device__ __forceinline__ float tile_stage_sa(const TileArgs &a, const PlaneCtx &c, int l, int x0,
                                               int y0, float *smt, int ndh)
{
    const int hy = HY > 0 ? HY : a.hy;
    const int ph = TL_H + 2 * hy, tsz = TL_PW * ph;
    float4 *SA = reinterpret_cast<float4 *>(smt + (size_t)ndh * tsz);
    const size_t npt = (size_t)a.np * a.nz;
    const float *Su = a.S + (size_t)l * npt + (size_t)c.ku * a.np;
    const float *Au = a.alpha + (size_t)l * npt + (size_t)c.ku * a.np;
    float amin = __int_as_float(0x7f800000);
    for (int e = threadIdx.x; e < ph * (TL_PW / 4); e += TL_THREADS)
        amin = fminf(amin, stage_sa_row(a, Su, Au, x0, y0, hy, e, SA));
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
    if (!SA_DONE)
        for (int e = tid; e < ph * q4; e += TL_THREADS)
            amin = fminf(amin, stage_sa_row(a, Su, Au, x0, y0, hy, e, SA));
    for (int e = tid; e < ph * q4; e += TL_THREADS) {
        const int r = e / q4, c4 = e % q4;
        const int gy = wrapi(y0 - hy + r, a.ny, a.wrap1);
        const int gx = wrapi(x0 - TL_HXP + 4 * c4, a.nx, a.wrap1);
        const size_t g = (size_t)gy * a.nx + gx;

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

size_t regular_wave_table_offset(const rt_grid *g)
{
    return (size_t)g->nz * 2 * 12 * sizeof(WaveSt);
}

size_t regular_wave_scratch(const rt_grid *g, int nlam)
{
    // the tile-major ring slots and flags of sc_wave_kernel, or the pipelined sweep's rings,
    // whichever is larger
    const size_t ntiles = (size_t)((g->nx + TL_W - 1) / TL_W) * ((g->ny + TL_H - 1) / TL_H);
    const size_t plane = (size_t)nlam * ntiles * 12 * TL_W * TL_H;
    const size_t nflags = 2 * (size_t)g->nz * nlam * ntiles;
    return std::max(4 * plane * sizeof(float) + (nflags + 64) * sizeof(int),
                    regular_pipe_scratch(g, nlam));
}

rt_status regular_wave_prepare(rt_grid *g, cudaStream_t st)
{
    int hy;
    if (!tile_geometry(g, hy) || g->dir_up.size() != 12 || g->dir_dn.size() != 12 || g->nz < 3)
        return RT_OK;
    std::vector<WaveSt> t((size_t)g->nz * 2 * 12, WaveSt{0, 0, 0, 0, 0, 0, 0, 0});
    std::vector<PlaneStencil> rt_((size_t)g->nz * 2 * 12, PlaneStencil{});
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
                PlaneStencil &r = rt_[((size_t)k * 2 + h) * 12 + d];
                r.tx = make_float2(sc.tx, sc.tx);
                r.ux = make_float2(1.0f - sc.tx, 1.0f - sc.tx);
                r.ty = make_float2(sc.ty, sc.ty);
                r.uy = make_float2(1.0f - sc.ty, 1.0f - sc.ty);
                r.hds = sc.hds;
                r.wd = (float)g->wdir[q];
                r.off = sc.ay * TL_PW + sc.ax;
            }
            for (int d = 0; d < 12; ++d) {
                e[d].hds_min = hmin;
                rt_[((size_t)k * 2 + h) * 12 + d].hds_min = hmin;
            }
        }
    // [WaveSt table][PlaneStencil table]
    g->h_wave_st.resize(t.size() * sizeof(WaveSt) + rt_.size() * sizeof(PlaneStencil));
    std::memcpy(g->h_wave_st.data(), t.data(), t.size() * sizeof(WaveSt));
    std::memcpy(g->h_wave_st.data() + t.size() * sizeof(WaveSt), rt_.data(),
                rt_.size() * sizeof(PlaneStencil));
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

rt_status regular_tile_sweep(rt_grid *g, int nlam, const float *alpha, const float *S, int bc,
                             float *J, float *buf0, float *buf1, cudaStream_t st, bool *done)
{
    *done = false;
    RT_TRY(regular_pipe_sweep(g, nlam, alpha, S, bc, J, st, done));
    if (*done) return RT_OK;
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
