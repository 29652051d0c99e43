// Regular grid, fused sweep with thread-block clusters (same arithmetic as sc_plane_kernel).
//
// One cluster of C CTAs owns a whole x-y plane for one wavelength and sweeps both hemispheres
// through all planes in a single launch.  CTA r of the cluster owns rows [r R, r R + R) (R = ny/C)
// for every direction of the hemisphere and keeps them, with H halo rows above and below, in
// shared memory for the whole sweep: the upwind planes never leave the SM.  After computing a
// plane, a thread that produced a row within H of its band edge also stores the value into the
// halo rows of the neighbouring CTA through distributed shared memory; one hardware cluster
// barrier per plane then publishes the halos and retires the previous plane.  S and alpha of the
// next plane are fetched into registers while the current plane is computed.  There is no
// device-side spin anywhere: the only waits are the CTA and cluster barriers.
#include <cooperative_groups.h>

#include <algorithm>
#include <cstdlib>

#include "device_common.cuh"
#include "rt_impl.h"

namespace cg = cooperative_groups;

namespace rt {

constexpr int CL_THREADS = 512;
constexpr int CL_MAX_DH = 16;
constexpr int CL_MAX_F4 = 4;   // float4 prefetch slots per thread per field

struct ClusterArgs {
    const float *alpha, *S;    // [nlam][npt]
    float *J;                  // [nlam][npt]
    const Stencil *st;         // [nz][ndir]
    unsigned *err;
    int nx, ny, nz, nlam, ndir, R, H, C, bc;
    int nd[2];                 // directions of the up / down hemisphere
    int dg[2][CL_MAX_DH];
    float w[2][CL_MAX_DH];
};

__global__ void __launch_bounds__(CL_THREADS, 1) sc_cluster_kernel(const ClusterArgs a)
{
    cg::cluster_group cl = cg::this_cluster();
    const int C = a.C, R = a.R, H = a.H, nx = a.nx, ny = a.ny, nz = a.nz;
    const int RH = R + 2 * H, plane_f = RH * nx;
    const int r = (int)cl.block_rank();
    const int ndmax = max(a.nd[0], a.nd[1]);
    extern __shared__ __align__(16) float sm[];
    // buffer b of a pair is selected arithmetically (no runtime-indexed pointer arrays)
    float *const I0 = sm;
    const size_t ibuf = (size_t)ndmax * plane_f;
    float *const PS0 = sm + 2 * ibuf;               // PS[b] = PS0 + b * plane_f
    float *const PA0 = PS0 + 2 * (size_t)plane_f;   // PA[b] = PA0 + b * plane_f
    __shared__ Stencil sst[CL_MAX_DH];
    const int rlo = (r + C - 1) % C, rhi = (r + 1) % C;
    float *const Ilo0 = cl.map_shared_rank(I0, rlo);
    float *const Ihi0 = cl.map_shared_rank(I0, rhi);
    const int tid = threadIdx.x;
    const int cluster_id = blockIdx.x / C, nclusters = gridDim.x / C;
    const size_t np = (size_t)nx * ny, npt = np * nz;
    const int npts = R * nx;
    const int nf4 = plane_f / 4;   // float4 per field per plane (band + halo)

    // band + halo rows of plane k of field F into registers (rows wrap periodically)
    float4 rs[CL_MAX_F4], ra[CL_MAX_F4];
    auto fetch = [&](const float *Sl, const float *Al, int k) {
#pragma unroll
        for (int m = 0; m < CL_MAX_F4; ++m) {
            const int e = tid + m * CL_THREADS;
            if (e < nf4) {
                const int row = (e * 4) / nx, col = (e * 4) % nx;
                int gy = r * R - H + row;
                gy += (gy < 0) ? ny : 0;
                gy -= (gy >= ny) ? ny : 0;
                const size_t o = (size_t)k * np + (size_t)gy * nx + col;
                rs[m] = __ldg(reinterpret_cast<const float4 *>(Sl + o));
                ra[m] = __ldg(reinterpret_cast<const float4 *>(Al + o));
            }
        }
    };
    auto deposit = [&](int b) {
#pragma unroll
        for (int m = 0; m < CL_MAX_F4; ++m) {
            const int e = tid + m * CL_THREADS;
            if (e < nf4) {
                reinterpret_cast<float4 *>(PS0 + (size_t)b * plane_f)[e] = rs[m];
                reinterpret_cast<float4 *>(PA0 + (size_t)b * plane_f)[e] = ra[m];
            }
        }
    };

    for (int l = cluster_id; l < a.nlam; l += nclusters) {
        const float *Sl = a.S + (size_t)l * npt;
        const float *Al = a.alpha + (size_t)l * npt;
        float *Jl = a.J + (size_t)l * npt;
        for (int hemi = 0; hemi < 2; ++hemi) {
            const int nd = a.nd[hemi];
            if (nd == 0) continue;
            const bool up = hemi == 0;
            const bool first = (hemi == 0) || (a.nd[0] == 0);
            // step 0: the boundary plane, every local row (band and halo) set from the rule
            const int k0 = up ? 0 : nz - 1;
            fetch(Sl, Al, k0);
            deposit(0);
            __syncthreads();
            for (int e = tid; e < nd * plane_f; e += CL_THREADS) {
                const int rem = e % plane_f;
                I0[e] = (a.bc == RT_BC_THERMAL && up) ? PS0[rem] : 0.f;
            }
            __syncthreads();
            for (int p = tid; p < npts; p += CL_THREADS) {
                const int jl = H + p / nx, i = p % nx;
                float jacc = 0.f;
                for (int d = 0; d < nd; ++d) jacc += a.w[hemi][d] * I0[(size_t)d * plane_f + jl * nx + i];
                float *Jp = Jl + (size_t)k0 * np + (size_t)(r * R + p / nx) * nx + i;
                *Jp = first ? jacc : *Jp + jacc;
            }
            fetch(Sl, Al, up ? 1 : nz - 2);
            cl.sync();   // neighbours' step-0 buffers are complete before anyone writes halos
            for (int s = 1; s < nz; ++s) {
                const int cur = s & 1, prev = cur ^ 1;
                const int k = up ? s : nz - 1 - s;
                deposit(cur);
                if (tid < nd) sst[tid] = a.st[(size_t)k * a.ndir + a.dg[hemi][tid]];
                __syncthreads();
                if (s + 1 < nz) fetch(Sl, Al, up ? s + 1 : nz - 2 - s);
                const float *Sp = PS0 + (size_t)prev * plane_f, *Ap = PA0 + (size_t)prev * plane_f;
                const float *Sc = PS0 + (size_t)cur * plane_f, *Ac = PA0 + (size_t)cur * plane_f;
                const float *Ip = I0 + (size_t)prev * ibuf;
                float *Ic = I0 + (size_t)cur * ibuf;
                float *Il = Ilo0 + (size_t)cur * ibuf, *Ih = Ihi0 + (size_t)cur * ibuf;
                for (int p = tid; p < npts; p += CL_THREADS) {
                    const int jb = p / nx, jl = H + jb, i = p % nx;
                    const float Sk = Sc[jl * nx + i];
                    const float ak = Ac[jl * nx + i];
                    float jacc = 0.f;
                    for (int d = 0; d < nd; ++d) {
                        const Stencil sc = sst[d];
                        int x0 = i + sc.axm;
                        x0 -= (x0 >= nx) ? nx : 0;
                        const int x1 = x0 + 1 == nx ? 0 : x0 + 1;
                        const int r0 = jl + sc.ay, r1 = r0 + 1;
                        const int o00 = r0 * nx + x0, o10 = r0 * nx + x1;
                        const int o01 = r1 * nx + x0, o11 = r1 * nx + x1;
                        const float *Iu = Ip + (size_t)d * plane_f;
                        const float iu = sc.w0 * Iu[o00] + sc.w1 * Iu[o10] + sc.w2 * Iu[o01] +
                                         sc.w3 * Iu[o11];
                        const float su = sc.w0 * Sp[o00] + sc.w1 * Sp[o10] + sc.w2 * Sp[o01] +
                                         sc.w3 * Sp[o11];
                        const float au = sc.w0 * Ap[o00] + sc.w1 * Ap[o10] + sc.w2 * Ap[o01] +
                                         sc.w3 * Ap[o11];
                        const float dt = (au + ak) * sc.hds;
                        float ex, w0, w1;
                        lin_weights(dt, ex, w0, w1);
                        const float v = iu * ex + w0 * su + w1 * Sk;
                        const size_t o = (size_t)d * plane_f;
                        Ic[o + jl * nx + i] = v;
                        if (jb < H) Il[o + (H + R + jb) * nx + i] = v;
                        if (jb >= R - H) Ih[o + (jb - (R - H)) * nx + i] = v;
                        jacc += a.w[hemi][d] * v;
                    }
                    float *Jp = Jl + (size_t)k * np + (size_t)(r * R + jb) * nx + i;
                    const float v = first ? jacc : *Jp + jacc;
                    if (!isfinite(v)) flag_error(a.err, ERR_NAN);
                    *Jp = v;
                }
                cl.sync();
            }
        }
    }
}

// Chooses the cluster shape for this grid, or returns false when the fused kernel does not
// apply (then the per-plane kernel is used).
static bool cluster_plan(const rt_grid *g, int nlam, int &C, int &R, int &H, size_t &smem)
{
    // opt-in: on GB300 at most 7 clusters of 16 are co-resident (112 of 152 SMs), and the
    // tiled per-plane kernel measures faster at the benchmark size
    const char *env = std::getenv("RT_REGULAR_SWEEP");
    const bool forced = env && std::string(env) == "cluster";
    if (!forced) return false;
    if (!g->periodic || g->nx % 4 || g->dir_up.size() > CL_MAX_DH || g->dir_dn.size() > CL_MAX_DH)
        return false;
    // halo width from the stencils: rows j + ay .. j + ay + 1 must stay within [j - H, j + H]
    int lo = 0, hi = 0;
    for (const Stencil &s : g->h_stencil) {
        lo = std::max(lo, -s.ay);
        hi = std::max(hi, s.ay + 1);
    }
    H = std::max(lo, hi);
    const int ndmax = (int)std::max(g->dir_up.size(), g->dir_dn.size());
    int dev = 0, optin = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    for (int c : {1, 2, 4, 8, 16}) {
        if (g->ny % c) continue;
        const int r = g->ny / c;
        if (r < H) break;
        const size_t rh = (size_t)(r + 2 * H) * g->nx;
        const size_t bytes = (2 * (size_t)ndmax * rh + 4 * rh) * sizeof(float);
        if (bytes + 2048 > (size_t)optin) continue;
        if (rh / 4 > (size_t)CL_MAX_F4 * CL_THREADS) continue;
        if (!forced && (size_t)nlam * c < (size_t)nsm / 2) continue;   // too few CTAs to fill
        C = c;
        R = r;
        smem = bytes;
        return true;
    }
    return false;
}

rt_status regular_cluster_sweep(rt_grid *g, int nlam, const float *alpha, const float *S, int bc,
                                float *J, cudaStream_t st, bool *done)
{
    *done = false;
    int C, R, H;
    size_t smem;
    if (bc == RT_BC_ARRAY || !cluster_plan(g, nlam, C, R, H, smem)) return RT_OK;
    ClusterArgs a;
    a.alpha = alpha;
    a.S = S;
    a.J = J;
    a.st = g->d_stencil;
    a.err = g->d_err;
    a.nx = g->nx;
    a.ny = g->ny;
    a.nz = g->nz;
    a.nlam = nlam;
    a.ndir = g->ndir;
    a.R = R;
    a.H = H;
    a.C = C;
    a.bc = bc;
    const std::vector<int> *hs[2] = {&g->dir_up, &g->dir_dn};
    for (int h = 0; h < 2; ++h) {
        a.nd[h] = (int)hs[h]->size();
        for (int d = 0; d < a.nd[h]; ++d) {
            a.dg[h][d] = (*hs[h])[d];
            a.w[h][d] = (float)g->wdir[(*hs[h])[d]];
        }
    }
    RT_CUDA(cudaFuncSetAttribute(sc_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem));
    if (C > 8)
        RT_CUDA(cudaFuncSetAttribute(sc_cluster_kernel,
                                     cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.blockDim = dim3(CL_THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cfg.gridDim = dim3(C * 64);
    int maxc = 0;
    RT_CUDA(cudaOccupancyMaxActiveClusters(&maxc, sc_cluster_kernel, &cfg));
    if (maxc < 1) return RT_OK;   // cannot be resident: fall back
    const int ncl = std::min(maxc, nlam);
    cfg.gridDim = dim3(C * ncl);
    note_launch();
    RT_CUDA(cudaLaunchKernelEx(&cfg, sc_cluster_kernel, a));
    *done = true;
    return RT_OK;
}

}  // namespace rt
