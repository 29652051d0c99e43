// Persistent wavefront sweep of the regular grid (plane-to-plane short characteristics,
// Sect. 2.6; linear S over each interval, Eq. 2; J accumulated over the quadrature, Eq. 4) with
// warp specialisation: in every block one producer warp stages the next item with the tensor
// memory accelerator while eight consumer warps compute the current one and a ninth warp
// publishes finished items.
//
// Items are (hemisphere, plane step, wavelength, 32 x 16 tile), taken from a device counter in the
// order of the other wavefront sweeps (hemisphere, wavelength chunk, step, wavelength, tile); an
// item needs the 3 x 3 neighbouring tiles of the previous step (and, downward, the upward item of
// the same plane and tile, whose J it adds to).  The producer claims an item (the claim of the
// following one is issued at once), waits (bounded) for those, waits for a free stage of the
// two-stage shared-memory ring, and issues the tile copies:
//   * every direction's intensity on the upwind plane, with halo, from the intensity ring;
//   * S and alpha of the upwind plane, with halo, from the same ring (the items of the previous
//     step stored their own S and alpha there next to their intensities);
//   * S and alpha of the item's own plane and, downward, the J tile, from the caller's arrays;
//   * the plane's stencils (one bulk copy).
// The intensity ring is stored with a periodic halo (4 columns and hy rows on each side), which
// the writers fill with copies of the edge points, so that every staged tile is one tensor copy.
// Consumers read only shared memory: a thread owns two vertically consecutive points of one column
// and walks down them for each direction; bilinear interpolation is separable, so each upwind row
// is loaded and interpolated along x once and serves both points of the thread whose corners it
// holds.  The consumer warps signal the releasing warp through a block-scope barrier when their
// stores are done; that warp frees the stage and publishes the item with one release at GPU scope,
// so the consumers never wait for their stores to drain.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <string>

#include "device_common.cuh"
#include "rt_impl.h"

namespace rt {

namespace {

constexpr int PW = 32;               // tile width (x)
constexpr int PHX = 4;               // staged x halo: the stencil reach in columns
constexpr int PPW = PW + 2 * PHX;    // staged row (40 points)
constexpr int NCW = 8;               // consumer warps
constexpr int SEG = 2;               // points per consumer thread (one column)
constexpr int TH = NCW * SEG;        // tile height (16)
constexpr int NTHR = (NCW + 2) * 32; // consumer warps, the producer warp, the releasing warp
constexpr int NDH = 12;              // directions per hemisphere

using PipeSt = PlaneStencil;   // the per-plane stencil table built with the grid

struct PipeMaps {
    CUtensorMap ring_i;    // float  [4][nlam * 12][ny + 2 hy][nx + 8]
    CUtensorMap ring_sa;   // float2 [4][nlam][ny + 2 hy][nx + 8] (S, alpha)
    CUtensorMap S, alpha;  // float  [nlam * nz][ny][nx]: the caller's arrays
    CUtensorMap J;
};

struct PipeArgs {
    const PipeSt *st;      // [nz][2][12]
    float *ring_i;         // layouts of ring_i and ring_sa above; slot h * 2 + (step & 1)
    float2 *ring_sa;
    float *J;
    unsigned *err;
    int *queue;
    int *done;             // [2][nz][nlam][ntiles]: 1 once the item is published
    float wd[2][NDH];      // quadrature weights per hemisphere (boundary planes)
    int nx, ny, nz, np, nlam, hy, px, py, tiles_x, ntiles, lchunk, bc;
};

// What the producer hands the consumers with a stage.
struct PipeDesc {
    int item, h, s, l, tile, x0, y0, stop;
};

// Shared memory of one stage (HY: halo rows); offsets in bytes, every region 128-byte aligned.
template <int HY> struct StageLayout {
    static constexpr int PH = TH + 2 * HY;
    static constexpr int TSZ = PPW * PH;                      // points per staged plane
    static constexpr int I_OFF = 0;                            // float [12][PH][PPW]
    static constexpr int SA_OFF = I_OFF + NDH * TSZ * 4;       // float2 [PH][PPW]
    static constexpr int S_OFF = SA_OFF + TSZ * 8;             // float [TH][PW]
    static constexpr int A_OFF = S_OFF + TH * PW * 4;
    static constexpr int J_OFF = A_OFF + TH * PW * 4;
    static constexpr int ST_OFF = J_OFF + TH * PW * 4;         // PipeSt [12]
    static constexpr int BYTES = (ST_OFF + NDH * 48 + 127) / 128 * 128;
    static_assert(SA_OFF % 128 == 0 && S_OFF % 128 == 0 && ST_OFF % 128 == 0, "alignment");
};

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *b, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(b)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *b)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(smem_u32(b)) : "memory");
}

__device__ __forceinline__ void mbar_arrive_tx(uint64_t *b, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                 :: "r"(smem_u32(b)), "r"(bytes) : "memory");
}

// Test for the completion of the phase of the given parity, with a suspend-time hint of 10
// microseconds (the hardware may hold the thread while the phase is open, up to the hint).
__device__ __forceinline__ bool mbar_test(uint64_t *b, unsigned parity)
{
    uint32_t ok;
    asm volatile("{\n .reg .pred p;\n"
                 " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
                 " selp.u32 %0, 1, 0, p;\n}"
                 : "=r"(ok) : "r"(smem_u32(b)), "r"(parity), "r"(10000u) : "memory");
    return ok != 0;
}

// Bounded wait (at most about a second) for the completion of the barrier phase of the given
// parity, sleeping SLEEP nanoseconds between polls so that a waiting warp takes few issue slots
// from the working ones.  Once any wait of the launch has timed out every later wait gives up
// after a few polls.
template <int SLEEP>
__device__ __forceinline__ bool mbar_wait(uint64_t *b, unsigned parity, const unsigned *err)
{
    for (int it = 0; it < (1 << 17); ++it) {
        if (mbar_test(b, parity)) return true;
        if ((it & 15) == 15 && (*(volatile const unsigned *)err & ERR_TIMEOUT)) return false;
        if (SLEEP) __nanosleep(SLEEP);
    }
    return false;
}

// Bounded wait until a completion counter reaches `target`.
__device__ __forceinline__ bool wait_count(const int *f, int target, const unsigned *err)
{
    int v;
    for (int it = 0; it < (1 << 20); ++it) {
        asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(f) : "memory");
        if (v >= target) return true;
        if ((it & 255) == 255 && (*(volatile const unsigned *)err & ERR_TIMEOUT)) return false;
        __nanosleep(32);
    }
    return false;
}

__device__ __forceinline__ void tma_3d(void *dst, const CUtensorMap *m, int c0, int c1, int c2,
                                       uint64_t *bar)
{
    asm volatile("cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                 " [%0], [%1, {%2, %3, %4}], [%5];"
                 :: "r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(m)), "r"(c0), "r"(c1),
                    "r"(c2), "r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tma_4d(void *dst, const CUtensorMap *m, int c0, int c1, int c2,
                                       int c3, uint64_t *bar)
{
    asm volatile("cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                 " [%0], [%1, {%2, %3, %4, %5}], [%6];"
                 :: "r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(m)), "r"(c0), "r"(c1),
                    "r"(c2), "r"(c3), "r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void bulk_copy(void *dst, const void *src, unsigned bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes"
                 " [%0], [%1], %2, [%3];"
                 :: "r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes),
                    "r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ PipeDesc pipe_decode(const PipeArgs &a, int item)
{
    const int nt = a.ntiles, nl = a.nlam, nz = a.nz, lc = a.lchunk;
    const int per_hemi = nz * nl * nt;
    PipeDesc it;
    it.item = item;
    it.stop = 0;
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
    it.x0 = (it.tile % a.tiles_x) * PW;
    it.y0 = (it.tile / a.tiles_x) * TH;
    return it;
}

// Periodic copies of a ring value (the halo of the padded ring): cx columns and cyo rows
// (pre-multiplied by the row pitch) from its own slot; zero where there is none.
template <class T>
__device__ __forceinline__ void ring_copies(T *p, int cyo, int cx, T v)
{
    if (cx) __stcg(p + cx, v);
    if (cyo) {
        __stcg(p + cyo, v);
        if (cx) __stcg(p + cyo + cx, v);
    }
}

// One item on the consumer side.  Warp w owns rows SEG w .. SEG w + SEG - 1 of the tile: a thread
// walks down its column of SEG points for each direction (or applies the inflow rule on the first
// plane of a hemisphere) and stores the intensities into the ring, with their periodic copies in
// EDGE items (those with points within the halo's reach of a side), then J and the plane's
// (S, alpha).  THICK: every interval of the warp's updates has optical depth >= 0.1, so only the
// exact interval weights are evaluated (no branch per update).  FULL: every point of the tile is
// inside the grid (no check per store).
template <int HY, bool THICK, bool EDGE, bool FULL>
__device__ __forceinline__ void consume(const PipeArgs &a, const char *stg, const PipeDesc &it,
                                        int lane, int warp)
{
    constexpr bool edge = EDGE;
    using L = StageLayout<HY>;
    const float *It = reinterpret_cast<const float *>(stg + L::I_OFF);
    const float2 *SA = reinterpret_cast<const float2 *>(stg + L::SA_OFF);
    const float *So = reinterpret_cast<const float *>(stg + L::S_OFF);
    const float *Ao = reinterpret_cast<const float *>(stg + L::A_OFF);
    const float *Jo = reinterpret_cast<const float *>(stg + L::J_OFF);
    const PipeSt *sts = reinterpret_cast<const PipeSt *>(stg + L::ST_OFF);
    const int h = it.h, s = it.s, l = it.l;
    const bool up = h == 0;
    const int k = up ? s : a.nz - 1 - s;
    const int hp = h * 2 + (s & 1);
    const int r0 = warp * SEG;
    const int x = it.x0 + lane;
    const bool okx = x < a.nx;
    const int px = a.px;
    const int cx = edge ? (x < PHX ? a.nx : (x >= a.nx - PHX ? -a.nx : 0)) : 0;
    int roff[SEG], cyo[SEG];
    bool ok[SEG];
    float Sk[SEG], ak[SEG], jacc[SEG];
#pragma unroll
    for (int j = 0; j < SEG; ++j) {
        const int y = it.y0 + r0 + j;
        ok[j] = FULL || (okx && y < a.ny);
        roff[j] = (y + HY) * px + x + PHX;
        cyo[j] = edge ? (y < HY ? a.ny * px : (y >= a.ny - HY ? -a.ny * px : 0)) : 0;
        Sk[j] = So[(r0 + j) * PW + lane];
        ak[j] = Ao[(r0 + j) * PW + lane];
        jacc[j] = 0.f;
    }
    const size_t plane = (size_t)a.py * px;
    float *ci = a.ring_i + ((size_t)hp * a.nlam + l) * NDH * plane;
    if (s == 0) {
        // first plane of the hemisphere: the inflow rule for every direction
#pragma unroll 1
        for (int d = 0; d < NDH; ++d) {
            const float wd = a.wd[h][d];
#pragma unroll
            for (int j = 0; j < SEG; ++j) {
                const float vv = (a.bc == RT_BC_THERMAL && up) ? Sk[j] : 0.f;
                if (ok[j]) {
                    __stcg(ci + d * plane + roff[j], vv);
                    if (edge) ring_copies(ci + d * plane + roff[j], cyo[j], cx, vv);
                }
                jacc[j] = fmaf(wd, vv, jacc[j]);
            }
        }
    } else {
        constexpr int TSZ = L::TSZ;
        const int o0 = (r0 + HY) * PPW + lane + PHX;   // the thread's first point in the stage
#pragma unroll 2
        for (int d = 0; d < NDH; ++d) {
            const float4 *q = reinterpret_cast<const float4 *>(sts + d);
            const float4 q0 = q[0], q1 = q[1], q2 = q[2];
            const float2 tx = make_float2(q0.x, q0.y), ux = make_float2(q0.z, q0.w);
            const float2 ty = make_float2(q1.x, q1.y), uy = make_float2(q1.z, q1.w);
            const float hds = q2.x, wd = q2.y;
            const int o = o0 + __float_as_int(q2.z);
            const float *Id = It + d * TSZ + o;
            const float2 *P = SA + o;
            // row values (interpolated along x) of the first upwind row
            float rI = fmaf(tx.x, Id[1], ux.x * Id[0]);
            float2 rsa = fma2(tx, P[1], mul2(ux, P[0]));
#pragma unroll
            for (int j = 0; j < SEG; ++j) {
                const float i0 = Id[(j + 1) * PPW], i1 = Id[(j + 1) * PPW + 1];
                const float2 p0 = P[(j + 1) * PPW], p1 = P[(j + 1) * PPW + 1];
                const float nI = fmaf(tx.x, i1, ux.x * i0);
                const float2 nsa = fma2(tx, p1, mul2(ux, p0));
                const float iu = fmaf(ty.x, nI, uy.x * rI);      // I, S, alpha at the upwind
                const float2 sa = fma2(ty, nsa, mul2(uy, rsa));  // point (S in x, alpha in y)
                const float dt = (sa.y + ak[j]) * hds;           // trapezoidal optical depth
                float ex, w0, w1;
                if (THICK) lin_weights_thick(dt, ex, w0, w1);
                else lin_weights(dt, ex, w0, w1);
                float vv = iu * ex;
                vv = fmaf(w0, sa.x, vv);
                vv = fmaf(w1, Sk[j], vv);
                if (ok[j]) {
                    __stcg(ci + d * plane + roff[j], vv);
                    if (edge) ring_copies(ci + d * plane + roff[j], cyo[j], cx, vv);
                }
                jacc[j] = fmaf(wd, vv, jacc[j]);
                rI = nI;
                rsa = nsa;
            }
        }
    }
    {
        // this plane's S and alpha, the upwind values of the next step
        float2 *cs = a.ring_sa + ((size_t)hp * a.nlam + l) * plane;
        const size_t npt = (size_t)a.np * a.nz;
#pragma unroll
        for (int j = 0; j < SEG; ++j) {
            if (!ok[j]) continue;
            const float2 sv = make_float2(Sk[j], ak[j]);
            __stcg(cs + roff[j], sv);
            if (edge) ring_copies(cs + roff[j], cyo[j], cx, sv);
            const int y = it.y0 + r0 + j;
            float *Jp = a.J + (size_t)l * npt + (size_t)k * a.np + (size_t)y * a.nx + x;
            const float vj = up ? jacc[j] : Jo[(r0 + j) * PW + lane] + jacc[j];
            if (!isfinite(vj)) flag_error(a.err, ERR_NAN);
            __stcg(Jp, vj);
        }
    }
}

template <int HY>
__global__ void __launch_bounds__(NTHR, 2)
sc_pipe_kernel(const __grid_constant__ PipeMaps maps, const PipeArgs a)
{
    using L = StageLayout<HY>;
    extern __shared__ __align__(128) char smraw[];
    // the stages start on a 128-byte boundary (tensor copies)
    char *smp = smraw + ((128u - (smem_u32(smraw) & 127u)) & 127u);
    // full: staged (producer, with the copies' bytes); stored: the consumer warps' stores of the
    // item are done; empty: the stage may be refilled (the releasing warp, after reading it)
    __shared__ __align__(8) uint64_t full[2], stored[2], empty[2];
    __shared__ PipeDesc desc[2];
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    if (threadIdx.x == 0) {
        for (int i = 0; i < 2; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&stored[i], NCW);
            mbar_init(&empty[i], 1);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const int nt = a.ntiles, nl = a.nlam, nz = a.nz;
    const int total = 2 * nz * nl * nt;
    if (warp == NCW) {
        // producer: claim, wait for the upwind items, wait for a free stage, stage.  The claim of
        // the following item is issued as soon as this one is known, and the upwind items are
        // awaited before the stage is, so that both latencies overlap the consumers' work.
        const int txn = a.tiles_x, tyn = nt / a.tiles_x;
        int next = 0;
        if (lane == 0) next = atomicAdd(a.queue, 1);
        for (int n = 0;; ++n) {
            const int st = n & 1;
            const int item = __shfl_sync(0xffffffffu, next, 0);
            if (item < total && lane == 0) next = atomicAdd(a.queue, 1);
            if (item >= total) {
                if (n >= 2) {
                    const bool ok = mbar_wait<64>(&empty[st], ((n >> 1) - 1) & 1, a.err);
                    if (!ok && lane == 0) flag_error(a.err, ERR_TIMEOUT);
                }
                if (lane == 0) {
                    desc[st].stop = 1;
                    mbar_arrive(&full[st]);
                }
                break;
            }
            const PipeDesc it = pipe_decode(a, item);
            const int h = it.h, s = it.s, l = it.l, tile = it.tile;
            const int k = h == 0 ? s : nz - 1 - s;
            const int *f = nullptr;
            if (lane < 9 && s > 0) {
                const int tx0 = tile % txn, ty0 = tile / txn;
                const int nx_ = (tx0 + lane % 3 - 1 + txn) % txn;
                const int ny_ = (ty0 + lane / 3 - 1 + tyn) % tyn;
                f = a.done + ((size_t)(h * nz + s - 1) * nl + l) * nt + ny_ * txn + nx_;
            } else if (lane == 9 && h == 1) {   // J of this plane and tile from the upward sweep
                f = a.done + ((size_t)(0 * nz + k) * nl + l) * nt + tile;
            }
            const bool ok = __all_sync(0xffffffffu, f ? wait_count(f, 1, a.err) : true);
            if (n >= 2) {   // the consumers are done with what this stage held two items ago
                const bool okb = mbar_wait<64>(&empty[st], ((n >> 1) - 1) & 1, a.err);
                if (!okb && lane == 0) flag_error(a.err, ERR_TIMEOUT);
            }
            __syncwarp();   // every lane's acquire precedes lane 0's copies
            if (lane == 0) {
                if (!ok) flag_error(a.err, ERR_TIMEOUT);
                // what the awaited items stored through ordinary writes (acquired above), before
                // the tensor reads
                asm volatile("fence.proxy.async.global;" ::: "memory");
                char *stg = smp + st * L::BYTES;
                desc[st] = it;
                unsigned bytes = 2 * TH * PW * 4 + (h == 1 ? TH * PW * 4 : 0);
                if (s > 0) bytes += NDH * L::TSZ * 4 + L::TSZ * 8 + NDH * 48;
                mbar_arrive_tx(&full[st], bytes);
                const int zl = l * nz + k;
                tma_3d(stg + L::S_OFF, &maps.S, it.x0, it.y0, zl, &full[st]);
                tma_3d(stg + L::A_OFF, &maps.alpha, it.x0, it.y0, zl, &full[st]);
                if (h == 1) tma_3d(stg + L::J_OFF, &maps.J, it.x0, it.y0, zl, &full[st]);
                if (s > 0) {
                    const int hp = h * 2 + ((s - 1) & 1);
                    tma_4d(stg + L::I_OFF, &maps.ring_i, it.x0, it.y0, l * NDH, hp, &full[st]);
                    tma_4d(stg + L::SA_OFF, &maps.ring_sa, it.x0, it.y0, l, hp, &full[st]);
                    bulk_copy(stg + L::ST_OFF, a.st + ((size_t)k * 2 + h) * NDH, NDH * 48,
                              &full[st]);
                }
            }
            __syncwarp();
        }
    } else if (warp < NCW) {
        // consumers
        for (int m = 0;; ++m) {
            const int st = m & 1;
            const bool ok = mbar_wait<20>(&full[st], (m >> 1) & 1, a.err);
            if (!ok && lane == 0) flag_error(a.err, ERR_TIMEOUT);
            const PipeDesc it = desc[st];
            if (it.stop) break;
            const char *stg = smp + st * L::BYTES;
            // items whose points have periodic copies in the ring's halo
            const bool edge = it.x0 < PHX || it.x0 + PW > a.nx - PHX || it.y0 < HY ||
                              it.y0 + TH > a.ny - HY;
            // d = (alpha_up + alpha_k) hds >= amin hds_min, amin the smallest staged alpha in the
            // rows this warp reads; the 1e-4 margin covers the rounding of the interpolated alpha
            bool thick = false;
            if (it.s > 0) {
                const float2 *SA = reinterpret_cast<const float2 *>(stg + L::SA_OFF);
                const int rr = warp * SEG;
                float amin = __int_as_float(0x7f800000);
                for (int e = lane; e < (SEG + 2 * HY) * PPW; e += 32)
                    amin = fminf(amin, SA[rr * PPW + e].y);
#pragma unroll
                for (int sh = 16; sh > 0; sh >>= 1)
                    amin = fminf(amin, __shfl_xor_sync(0xffffffffu, amin, sh));
                const float hmin = reinterpret_cast<const PipeSt *>(stg + L::ST_OFF)[0].hds_min;
                thick = amin * hmin >= 0.1f * 1.0001f;
            }
            // whole tiles (every point inside the grid) store without a per-point check
            // (5.08 against 5.35 ms at 128^3; choosing the edge copies per warp as well, so that
            // warps without edge points skip them, measured 5.23 ms: more code variants)
            const bool full = it.x0 + PW <= a.nx && it.y0 + TH <= a.ny;
            if (edge) {
                if (full) {
                    if (thick) consume<HY, true, true, true>(a, stg, it, lane, warp);
                    else consume<HY, false, true, true>(a, stg, it, lane, warp);
                } else {
                    if (thick) consume<HY, true, true, false>(a, stg, it, lane, warp);
                    else consume<HY, false, true, false>(a, stg, it, lane, warp);
                }
            } else {
                if (thick) consume<HY, true, false, true>(a, stg, it, lane, warp);
                else consume<HY, false, false, true>(a, stg, it, lane, warp);
            }
            // the warp's ring and J stores (and its reads of the stage) are done
            __syncwarp();
            if (lane == 0) mbar_arrive(&stored[st]);
        }
    } else {
        // releasing warp: once the consumer warps have stored an item, frees its stage and
        // publishes the item (a release at GPU scope, which orders the consumers' stores that the
        // barrier made visible to this warp before the flag); the fence's wait for the stores is
        // spent here, not by the consumers
        for (int m = 0;; ++m) {
            const int st = m & 1;
            bool ok = mbar_wait<256>(&full[st], (m >> 1) & 1, a.err);
            const PipeDesc it = desc[st];
            if (it.stop) break;
            ok = mbar_wait<256>(&stored[st], (m >> 1) & 1, a.err) && ok;
            __syncwarp();
            if (lane == 0) {
                if (!ok) flag_error(a.err, ERR_TIMEOUT);
                mbar_arrive(&empty[st]);
                int *f = a.done + ((size_t)(it.h * nz + it.s) * nl + it.l) * nt + it.tile;
                asm volatile("red.release.gpu.global.add.s32 [%0], 1;" :: "l"(f) : "memory");
            }
            __syncwarp();
        }
    }
}

// ---- host --------------------------------------------------------------------------------------

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            p = nullptr;
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }();
    return fn;
}

bool encode(CUtensorMap *m, CUtensorMapDataType t, int rank, void *base, const cuuint64_t *dims,
            const cuuint64_t *strides, const cuuint32_t *box)
{
    auto fn = tensor_map_encoder();
    if (!fn) return false;
    const cuuint32_t es[4] = {1, 1, 1, 1};
    return fn(m, t, (cuuint32_t)rank, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Stencil reach (halo rows) of the grid's planes, or -1 where the staged tile cannot cover it.
int pipe_halo(const rt_grid *g)
{
    int lx = 0, rx = 0, ly = 0, ry = 0;
    for (const Stencil &s : g->h_stencil) {
        lx = std::max(lx, -s.ax);
        rx = std::max(rx, s.ax + 1);
        ly = std::max(ly, -s.ay);
        ry = std::max(ry, s.ay + 1);
    }
    const int hy = std::max(1, std::max(ly, ry));
    return std::max(lx, rx) <= PHX && hy <= 3 ? hy : -1;
}

}  // namespace

// Conditions of the pipelined sweep: periodic sides, 12 directions per hemisphere, nx a multiple
// of 4 and at least one tile wide and high, a stencil reach of at most 4 columns and 3 rows, and a
// last tile row at least hy high when there are more than 3 tile rows (the items that read a
// point's periodic copies are then the 3 x 3 neighbours of the item that writes it).
static bool pipe_applies(const rt_grid *g, int &hy)
{
    if (!g->periodic || g->nx % 4 || g->nx < PW || g->ny < TH || g->nz < 3 || !g->d_wave_st ||
        g->dir_up.size() != NDH || g->dir_dn.size() != NDH)
        return false;
    hy = pipe_halo(g);
    if (hy < 1 || hy > g->ny) return false;
    const int tyn = (g->ny + TH - 1) / TH;
    if (tyn > 3 && g->ny - (tyn - 1) * TH < hy) return false;
    return tensor_map_encoder() != nullptr;
}

size_t regular_pipe_scratch(const rt_grid *g, int nlam)
{
    int hy;
    if (!pipe_applies(g, hy)) return 0;
    const size_t plane = (size_t)(g->ny + 2 * hy) * (g->nx + 2 * PHX);
    const size_t ntiles = (size_t)((g->nx + PW - 1) / PW) * ((g->ny + TH - 1) / TH);
    return 4 * (size_t)nlam * NDH * plane * sizeof(float) + 4 * (size_t)nlam * plane * 8 +
           (2 * (size_t)g->nz * nlam * ntiles + 64) * sizeof(int);
}

template <int HY>
static rt_status pipe_launch(const PipeMaps &maps, const PipeArgs &a, int blocks, cudaStream_t st)
{
    const size_t smem = 2 * (size_t)StageLayout<HY>::BYTES + 128;
    RT_CUDA(cudaMemsetAsync(a.queue, 0, (2 * (size_t)a.nz * a.nlam * a.ntiles + 32) * sizeof(int),
                            st));
    note_launch();
    sc_pipe_kernel<HY><<<blocks, NTHR, smem, st>>>(maps, a);
    RT_CUDA(cudaGetLastError());
    return RT_OK;
}

template <int HY>
static rt_status pipe_occupancy(int *per_sm)
{
    const size_t smem = 2 * (size_t)StageLayout<HY>::BYTES + 128;
    RT_CUDA(cudaFuncSetAttribute(sc_pipe_kernel<HY>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem));
    RT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, sc_pipe_kernel<HY>, NTHR, smem));
    return RT_OK;
}

rt_status regular_pipe_sweep(rt_grid *g, int nlam, const float *alpha, const float *S, int bc,
                             float *J, cudaStream_t st, bool *done)
{
    *done = false;
    int hy;
    if (bc == RT_BC_ARRAY || !pipe_applies(g, hy)) return RT_OK;
    if (!aligned16(alpha) || !aligned16(S) || !aligned16(J)) return RT_OK;
    if (const char *e = std::getenv("RT_REGULAR_SWEEP"))
        if (std::string(e) != "pipe") return RT_OK;   // another sweep requested
    PipeArgs a;
    std::memset(&a, 0, sizeof(a));
    a.nx = g->nx;
    a.ny = g->ny;
    a.nz = g->nz;
    a.np = g->nx * g->ny;
    a.nlam = nlam;
    a.hy = hy;
    a.px = g->nx + 2 * PHX;
    a.py = g->ny + 2 * hy;
    a.tiles_x = (g->nx + PW - 1) / PW;
    a.ntiles = a.tiles_x * ((g->ny + TH - 1) / TH);
    a.bc = bc;
    a.J = J;
    a.err = g->d_err;
    a.st = reinterpret_cast<const PipeSt *>(static_cast<const char *>(g->d_wave_st) +
                                            regular_wave_table_offset(g));
    const std::vector<int> *hs[2] = {&g->dir_up, &g->dir_dn};
    for (int h = 0; h < 2; ++h)
        for (int d = 0; d < NDH; ++d) a.wd[h][d] = (float)g->wdir[(*hs[h])[d]];
    int per_sm = 0, dev = 0, nsm = 0;
    switch (hy) {
    case 1: RT_TRY(pipe_occupancy<1>(&per_sm)); break;
    case 2: RT_TRY(pipe_occupancy<2>(&per_sm)); break;
    default: RT_TRY(pipe_occupancy<3>(&per_sm)); break;
    }
    if (per_sm < 1) return RT_OK;
    RT_CUDA(cudaGetDevice(&dev));
    RT_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const int blocks = per_sm * nsm;
    {
        // wavelengths per chunk: a plane step of a chunk holds several times the items that the
        // blocks hold in flight (three each: two staged, one claimed), so that the upwind items
        // of a claimed item are normally done; chunks of equal size.  At 128 x 128 and 52
        // wavelengths this is one chunk: measured 5.35 ms against 5.67 ms with two chunks of 26
        // and 6.57 ms with three, although the rings of all wavelengths then exceed the L2 share
        // (L2 eviction hints that favour the ring made it slower).  RT_WAVE_LCHUNK overrides.
        const int target = std::max(1, (4 * blocks + a.ntiles - 1) / a.ntiles);
        const int nch = std::max(1, (nlam + target / 2) / target);
        int lc = (nlam + nch - 1) / nch;
        if (const char *e = std::getenv("RT_WAVE_LCHUNK")) lc = std::atoi(e);
        a.lchunk = std::max(1, std::min(nlam, lc));
    }
    const size_t plane = (size_t)a.py * a.px;
    void *p;
    RT_TRY(scratch_get(g, 3, regular_wave_scratch(g, nlam), &p));
    a.ring_i = static_cast<float *>(p);
    a.ring_sa = reinterpret_cast<float2 *>(a.ring_i + 4 * (size_t)nlam * NDH * plane);
    a.queue = reinterpret_cast<int *>(a.ring_sa + 4 * (size_t)nlam * plane);
    a.done = a.queue + 32;
    PipeMaps maps;
    std::memset(&maps, 0, sizeof(maps));
    const int PH = TH + 2 * hy;
    {
        const cuuint64_t dims[4] = {(cuuint64_t)a.px, (cuuint64_t)a.py, (cuuint64_t)nlam * NDH, 4};
        const cuuint64_t str[3] = {(cuuint64_t)a.px * 4, plane * 4, plane * nlam * NDH * 4};
        const cuuint32_t box[4] = {PPW, (cuuint32_t)PH, NDH, 1};
        if (!encode(&maps.ring_i, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, a.ring_i, dims, str, box))
            return RT_OK;
    }
    {
        const cuuint64_t dims[4] = {(cuuint64_t)a.px, (cuuint64_t)a.py, (cuuint64_t)nlam, 4};
        const cuuint64_t str[3] = {(cuuint64_t)a.px * 8, plane * 8, plane * nlam * 8};
        const cuuint32_t box[4] = {PPW, (cuuint32_t)PH, 1, 1};
        if (!encode(&maps.ring_sa, CU_TENSOR_MAP_DATA_TYPE_UINT64, 4, a.ring_sa, dims, str, box))
            return RT_OK;
    }
    {
        const cuuint64_t dims[3] = {(cuuint64_t)g->nx, (cuuint64_t)g->ny,
                                    (cuuint64_t)g->nz * nlam};
        const cuuint64_t str[2] = {(cuuint64_t)g->nx * 4, (cuuint64_t)g->nx * g->ny * 4};
        const cuuint32_t box[3] = {PW, TH, 1};
        if (!encode(&maps.S, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float *>(S), dims, str,
                    box) ||
            !encode(&maps.alpha, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float *>(alpha),
                    dims, str, box) ||
            !encode(&maps.J, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, J, dims, str, box))
            return RT_OK;
    }
    switch (hy) {
    case 1: RT_TRY(pipe_launch<1>(maps, a, blocks, st)); break;
    case 2: RT_TRY(pipe_launch<2>(maps, a, blocks, st)); break;
    default: RT_TRY(pipe_launch<3>(maps, a, blocks, st)); break;
    }
    *done = true;
    return RT_OK;
}

}  // namespace rt
