// Rejection sampling of Voronoi sites (Sect. 2.4): a proposal uniform in the box is kept when the
// target there is at least a uniform random rejection level, until the wanted number of sites.
//
// Random numbers: Philox4x64-10 (Salmon, Moraes, Dror & Shaw 2011, "Parallel random numbers: as
// easy as 1, 2, 3"), written from its published definition.  Proposal p draws the block of
// counter (p, 0, 0, 0) under key (seed, 0); u_i = (w_i >> 11) 2^-53 gives the position and the
// rejection level u_3.  The target is trilinear on a mesh, periodic in x and y, clamped in z; every
// floating-point step is one IEEE double operation in a fixed order (explicit round-to-nearest
// intrinsics, so nothing is contracted into a fused multiply-add), so a proposal's fate does not
// depend on the device or the launch shape.  The sites are the first nsites kept proposals in
// proposal order.
//
// Work decomposition.  Batches of 2^22 proposals: each 256-thread block takes 4096 consecutive
// proposals (16 per thread, consecutive), counts its kept ones (block scan); one block turns the
// 1024 counts into offsets; the blocks then recompute their proposals and write the kept ones at
// their global rank.  The host reads one count per batch.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>

#include "device_common.cuh"
#include "rt_impl.h"

namespace rt {

constexpr int SMP_THREADS = 256;
constexpr int SMP_PER_THREAD = 16;
constexpr int SMP_PER_BLOCK = SMP_THREADS * SMP_PER_THREAD;     // 4096
constexpr int SMP_BLOCKS = 1024;
constexpr uint64_t SMP_BATCH = (uint64_t)SMP_PER_BLOCK * SMP_BLOCKS;   // 2^22

struct SampleArgs {
    const float *f;        // [nz][ny][nx]
    const double *z;       // [nz]
    double box[6];
    double fmax;
    uint64_t seed;
    int nx, ny, nz;
};

__device__ __forceinline__ void philox4x64_10(uint64_t c[4], uint64_t k0, uint64_t k1)
{
    const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
    const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k0 += W0;
            k1 += W1;
        }
        const uint64_t hi0 = __umul64hi(M0, c[0]), lo0 = M0 * c[0];
        const uint64_t hi1 = __umul64hi(M1, c[2]), lo1 = M1 * c[2];
        const uint64_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
    }
}

__device__ __forceinline__ double uniform53(uint64_t w)
{
    return __dmul_rn(__ull2double_rn(w >> 11), 1.1102230246251565404e-16);   // 2^-53
}

__device__ __forceinline__ double lerp_rn(double a, double b, double t)
{
    return __dadd_rn(a, __dmul_rn(t, __dsub_rn(b, a)));
}

// proposal p: position into r[3]; returns whether it is kept
__device__ bool propose(const SampleArgs &a, uint64_t p, double r[3])
{
    uint64_t c[4] = {p, 0ull, 0ull, 0ull};
    philox4x64_10(c, a.seed, 0ull);
    const double u0 = uniform53(c[0]), u1 = uniform53(c[1]), u2 = uniform53(c[2]),
                 u3 = uniform53(c[3]);
    const double x0 = a.box[0], x1 = a.box[1], y0 = a.box[2], y1 = a.box[3];
    r[0] = __dadd_rn(x0, __dmul_rn(u0, __dsub_rn(x1, x0)));
    r[1] = __dadd_rn(y0, __dmul_rn(u1, __dsub_rn(y1, y0)));
    r[2] = __dadd_rn(a.box[4], __dmul_rn(u2, __dsub_rn(a.box[5], a.box[4])));
    // trilinear target at r
    const double dx = __ddiv_rn(__dsub_rn(x1, x0), (double)a.nx);
    const double dy = __ddiv_rn(__dsub_rn(y1, y0), (double)a.ny);
    const double fx = __ddiv_rn(__dsub_rn(r[0], x0), dx);
    const double fy = __ddiv_rn(__dsub_rn(r[1], y0), dy);
    const double fi = floor(fx), fj = floor(fy);
    const double tx = __dsub_rn(fx, fi), ty = __dsub_rn(fy, fj);
    const int i0 = (int)(((long long)fi % a.nx + a.nx) % a.nx), i1 = i0 + 1 == a.nx ? 0 : i0 + 1;
    const int j0 = (int)(((long long)fj % a.ny + a.ny) % a.ny), j1 = j0 + 1 == a.ny ? 0 : j0 + 1;
    // k0: the last plane at or below r_z, within [0, nz - 2]
    int lo = 0, hi = a.nz;                    // number of planes at or below r_z, by bisection
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (a.z[mid] <= r[2]) lo = mid + 1;
        else hi = mid;
    }
    int k0 = lo - 1;
    k0 = k0 < 0 ? 0 : (k0 > a.nz - 2 ? a.nz - 2 : k0);
    const int k1 = k0 + 1;
    double tz = __ddiv_rn(__dsub_rn(r[2], a.z[k0]), __dsub_rn(a.z[k1], a.z[k0]));
    if (r[2] <= a.z[0]) tz = 0.0;
    else if (r[2] >= a.z[a.nz - 1]) tz = 1.0;
    const size_t np = (size_t)a.nx * a.ny;
    auto F = [&](int k, int j, int i) -> double {
        return (double)__ldg(a.f + (size_t)k * np + (size_t)j * a.nx + i);
    };
    const double c00 = lerp_rn(F(k0, j0, i0), F(k0, j0, i1), tx);
    const double c10 = lerp_rn(F(k0, j1, i0), F(k0, j1, i1), tx);
    const double c01 = lerp_rn(F(k1, j0, i0), F(k1, j0, i1), tx);
    const double c11 = lerp_rn(F(k1, j1, i0), F(k1, j1, i1), tx);
    const double v = lerp_rn(lerp_rn(c00, c10, ty), lerp_rn(c01, c11, ty), tz);
    return v >= __dmul_rn(u3, a.fmax);
}

// exclusive scan of one int per thread over the block (blockDim a multiple of 32, <= 1024);
// *total gets the block's sum
__device__ int block_exclusive_scan(int v, int *total)
{
    __shared__ int wsum[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int s = lane < nw ? wsum[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < nw) wsum[lane] = s;       // inclusive sums of the warps
    }
    __syncthreads();
    const int before = warp ? wsum[warp - 1] : 0;
    *total = wsum[nw - 1];
    __syncthreads();                          // wsum is reused by the next call
    return before + x - v;
}

__global__ void __launch_bounds__(SMP_THREADS) sample_count_kernel(SampleArgs a, uint64_t base,
                                                                   int *counts)
{
    const uint64_t p0 = base + (uint64_t)blockIdx.x * SMP_PER_BLOCK +
                        (uint64_t)threadIdx.x * SMP_PER_THREAD;
    int n = 0;
    double r[3];
    for (int i = 0; i < SMP_PER_THREAD; ++i) n += propose(a, p0 + i, r) ? 1 : 0;
    int total;
    block_exclusive_scan(n, &total);
    if (threadIdx.x == 0) counts[blockIdx.x] = total;
}

// offsets[b] = sum of counts before b; *sum = all
__global__ void __launch_bounds__(SMP_BLOCKS) sample_offsets_kernel(const int *counts, int *offsets,
                                                                    int *sum)
{
    int total;
    const int e = block_exclusive_scan(counts[threadIdx.x], &total);
    offsets[threadIdx.x] = e;
    if (threadIdx.x == 0) *sum = total;
}

// writes the kept proposals of rank < need to xyz[(have + rank)][3]; *last = 1 + the proposal
// index of rank need - 1
__global__ void __launch_bounds__(SMP_THREADS) sample_write_kernel(SampleArgs a, uint64_t base,
                                                                   const int *offsets, int64_t have,
                                                                   int64_t need, double *xyz,
                                                                   unsigned long long *last)
{
    const uint64_t p0 = base + (uint64_t)blockIdx.x * SMP_PER_BLOCK +
                        (uint64_t)threadIdx.x * SMP_PER_THREAD;
    unsigned mask = 0;
    double r[3];
    for (int i = 0; i < SMP_PER_THREAD; ++i)
        if (propose(a, p0 + i, r)) mask |= 1u << i;
    int total;
    int64_t rank = (int64_t)offsets[blockIdx.x] + block_exclusive_scan(__popc(mask), &total);
    for (int i = 0; i < SMP_PER_THREAD && rank < need; ++i) {
        if (!((mask >> i) & 1u)) continue;
        propose(a, p0 + i, r);
        double *o = xyz + (size_t)(have + rank) * 3;
        o[0] = r[0];
        o[1] = r[1];
        o[2] = r[2];
        if (rank == need - 1) *last = (unsigned long long)(p0 + i + 1);
        ++rank;
    }
}

// max of f and a flag for any negative or non-finite value
__global__ void sample_check_kernel(const float *f, size_t n, unsigned *fmax_bits, unsigned *bad)
{
    unsigned m = 0;
    bool b = false;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        const float v = f[i];
        if (!(v >= 0.f) || !isfinite(v)) b = true;
        else m = max(m, __float_as_uint(v));   // non-negative floats order as their bits
    }
    for (int o = 16; o; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(fmax_bits, m);
    if (__any_sync(0xffffffffu, b) && (threadIdx.x & 31) == 0) atomicOr(bad, 1u);
}

}  // namespace rt

using namespace rt;

extern "C" rt_status rt_sample_sites(int nx, int ny, int nz, const double *z, const double *box,
                                     const float *f, int64_t nsites, uint64_t seed, double *xyz,
                                     int64_t *nproposals, void *stream)
{
    return guarded([&]() -> rt_status {
        if (nx < 1 || ny < 1 || nz < 2 || !z || !box || !f || nsites < 1 || !xyz)
            return fail(RT_EINVAL, "sample_sites: bad argument");
        if ((int64_t)nx * ny * nz > ((int64_t)1 << 40)) return fail(RT_EINVAL, "mesh too large");
        for (int k = 1; k < nz; ++k)
            if (!(z[k] > z[k - 1])) return fail(RT_EINVAL, "z must be strictly ascending");
        if (!(box[1] > box[0] && box[3] > box[2] && box[5] > box[4]))
            return fail(RT_EINVAL, "box must have positive extent");
        if ((uintptr_t)xyz % 8) return fail(RT_EINVAL, "xyz must be 8-byte aligned");
        cudaStream_t st = (cudaStream_t)stream;
        const size_t n = (size_t)nx * ny * nz;
        // device scratch: z, counts, offsets, sum, last, fmax bits, bad flag
        struct Buf {
            void *p = nullptr;
            ~Buf() { if (p) cudaFree(p); }
        } buf;
        const size_t zb = (size_t)nz * sizeof(double);
        const size_t bytes = zb + 2 * SMP_BLOCKS * sizeof(int) + 64;
        RT_CUDA(cudaMalloc(&buf.p, bytes));
        double *dz = (double *)buf.p;
        int *counts = (int *)((char *)buf.p + zb);
        int *offsets = counts + SMP_BLOCKS;
        int *sum = offsets + SMP_BLOCKS;
        unsigned long long *last = (unsigned long long *)(((uintptr_t)(sum + 1) + 7) & ~(uintptr_t)7);
        unsigned *fmax_bits = (unsigned *)(last + 1);
        unsigned *bad = fmax_bits + 1;
        RT_CUDA(cudaMemcpyAsync(dz, z, zb, cudaMemcpyHostToDevice, st));
        RT_CUDA(cudaMemsetAsync(fmax_bits, 0, 2 * sizeof(unsigned), st));
        note_launch();
        sample_check_kernel<<<1216, 256, 0, st>>>(f, n, fmax_bits, bad);
        unsigned h[2];
        RT_CUDA(cudaMemcpyAsync(h, fmax_bits, sizeof(h), cudaMemcpyDeviceToHost, st));
        RT_CUDA(cudaStreamSynchronize(st));
        float fmax;
        std::memcpy(&fmax, &h[0], sizeof(float));
        if (h[1]) return fail(RT_EINVAL, "sample_sites: target must be finite and non-negative");
        if (!(fmax > 0.f)) return fail(RT_EINVAL, "sample_sites: target is zero everywhere");
        SampleArgs a;
        a.f = f;
        a.z = dz;
        for (int c = 0; c < 6; ++c) a.box[c] = box[c];
        a.fmax = (double)fmax;
        a.seed = seed;
        a.nx = nx;
        a.ny = ny;
        a.nz = nz;
        const uint64_t max_prop = 1000ull * (uint64_t)nsites + (1ull << 20);
        int64_t have = 0;
        uint64_t base = 0;
        unsigned long long h_last = 0;
        while (have < nsites) {
            if (base >= max_prop)
                return fail(RT_ENOCONV, "sample_sites: too few proposals accepted");
            note_launch(2);
            sample_count_kernel<<<SMP_BLOCKS, SMP_THREADS, 0, st>>>(a, base, counts);
            sample_offsets_kernel<<<1, SMP_BLOCKS, 0, st>>>(counts, offsets, sum);
            int h_sum = 0;
            RT_CUDA(cudaMemcpyAsync(&h_sum, sum, sizeof(int), cudaMemcpyDeviceToHost, st));
            RT_CUDA(cudaStreamSynchronize(st));
            if (h_sum > 0) {
                const int64_t need = nsites - have;
                note_launch();
                sample_write_kernel<<<SMP_BLOCKS, SMP_THREADS, 0, st>>>(a, base, offsets, have, need,
                                                                      xyz, last);
                RT_CUDA(cudaGetLastError());
                if (h_sum >= need) {
                    RT_CUDA(cudaMemcpyAsync(&h_last, last, sizeof(h_last), cudaMemcpyDeviceToHost, st));
                    RT_CUDA(cudaStreamSynchronize(st));
                }
                have += std::min<int64_t>(h_sum, need);
            }
            base += SMP_BATCH;
        }
        if (nproposals) *nproposals = (int64_t)h_last;
        return RT_OK;
    });
}
