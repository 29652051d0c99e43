// Regular-grid formal solution that allocates nothing.
//
// Some callers cannot call cudaMalloc: code running inside a host callback or a stream-ordered
// region that must not synchronise the device, plugins whose host application owns every
// allocation, and processes that run under a fixed device-memory budget.  For them this entry
// point computes the same per-plane short-characteristics sweep and J as rt_formal_solution on a
// regular grid, but takes its upwind-plane scratch from a file-scope device array of fixed size
// and its per-plane stencils as kernel arguments, so it needs no grid object and no device
// allocation at all.  The caller passes the inputs and the output.
#include <cmath>
#include <vector>

#include "device_common.cuh"
#include "rt_impl.h"

namespace rt {

// 4 Mi floats = 16 MiB, held by every GPU that loads the library until the process exits.
constexpr size_t NOALLOC_SCRATCH_FLOATS = (size_t)4 << 20;
constexpr int NOALLOC_MAX_DH = 32;

static __device__ __align__(256) float g_noalloc_scratch[NOALLOC_SCRATCH_FLOATS];

struct NoAllocPlane {
    const float *alpha, *S;   // [nlam][npt]
    const float *Iprev;       // [nlam][ndh][np] (static scratch)
    float *Inext;
    float *J;
    const float *I_bc;        // [ndir][nlam][np] or null
    int nx, ny, nz, np, nlam, ndh, up, periodic, bc, first, step;
    int dg[NOALLOC_MAX_DH];
    float w[NOALLOC_MAX_DH];
    Stencil st[NOALLOC_MAX_DH];   // this plane's stencil of every direction of the hemisphere
};

__global__ void __launch_bounds__(256) sc_plane_noalloc_kernel(const NoAllocPlane a)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    const int l = blockIdx.y;
    if (q >= a.np) return;
    const int i = q % a.nx, j = q / a.nx;
    const int k = a.up ? a.step : a.nz - 1 - a.step;
    const size_t npt = (size_t)a.np * a.nz;
    const float *al = a.alpha + (size_t)l * npt;
    const float *Sl = a.S + (size_t)l * npt;
    const float Sk = __ldg(Sl + (size_t)k * a.np + q);
    float jacc = 0.f;
    if (a.step == 0) {
        for (int d = 0; d < a.ndh; ++d) {
            float v;
            if (a.bc == RT_BC_ARRAY) v = __ldg(a.I_bc + ((size_t)a.dg[d] * a.nlam + l) * a.np + q);
            else v = (a.bc == RT_BC_THERMAL && a.up) ? Sk : 0.f;
            a.Inext[((size_t)l * a.ndh + d) * a.np + q] = v;
            jacc += a.w[d] * v;
        }
    } else {
        const int ku = a.up ? k - 1 : k + 1;
        const float ak = __ldg(al + (size_t)k * a.np + q);
        const float *Su = Sl + (size_t)ku * a.np;
        const float *Au = al + (size_t)ku * a.np;
        for (int d = 0; d < a.ndh; ++d) {
            const Stencil &s = a.st[d];
            const float *Iu = a.Iprev + ((size_t)l * a.ndh + d) * a.np;
            float iu = 0.f, su = 0.f, au = 0.f;
            const int xs[2] = {i + s.ax, i + s.ax + 1}, ys[2] = {j + s.ay, j + s.ay + 1};
            const float ws[4] = {s.w0, s.w1, s.w2, s.w3};
            for (int c = 0; c < 4; ++c) {
                int x = xs[c & 1], y = ys[c >> 1];
                bool in = true;
                if (a.periodic) {
                    x = ((x % a.nx) + a.nx) % a.nx;
                    y = ((y % a.ny) + a.ny) % a.ny;
                } else {
                    in = x >= 0 && x < a.nx && y >= 0 && y < a.ny;
                    x = min(max(x, 0), a.nx - 1);
                    y = min(max(y, 0), a.ny - 1);
                }
                const int o = y * a.nx + x;
                if (in) iu += ws[c] * Iu[o];
                su += ws[c] * __ldg(Su + o);
                au += ws[c] * __ldg(Au + o);
            }
            float ex, w0, w1;
            lin_weights((au + ak) * s.hds, ex, w0, w1);
            const float v = iu * ex + w0 * su + w1 * Sk;
            a.Inext[((size_t)l * a.ndh + d) * a.np + q] = v;
            jacc += a.w[d] * v;
        }
    }
    float *Jp = a.J + (size_t)l * npt + (size_t)k * a.np + q;
    *Jp = a.first ? jacc : *Jp + jacc;
}

// Device address of the static scratch in the context current on the calling thread.  The
// address belongs to a CUDA context, not to a device ordinal: a host application may run its own
// driver context, and cudaDeviceReset replaces the primary one.  So it is looked up on every call,
// which allocates nothing (the first lookup in a context may load the library's device code and
// reserve the array there).
static rt_status noalloc_scratch(float **out)
{
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(static scratch)");
    *out = (float *)p;
    return RT_OK;
}

}  // namespace rt

using namespace rt;

extern "C" rt_status rt_formal_solution_regular_noalloc(
    int nx, int ny, int nz, double dx, double dy, const double *z, int periodic_xy, int ndir,
    const double *dirs, const double *wdir, int nlam, const float *alpha, const float *S, int bc,
    const float *I_bc, float *J, void *stream)
{
    return guarded([&]() -> rt_status {
        if (nx < 1 || ny < 1 || nz < 2 || !(dx > 0) || !(dy > 0) || !z || ndir < 1 || !dirs ||
            !wdir || nlam < 1 || nlam > 65535 || !alpha || !S || !J)
            return fail(RT_EINVAL, "bad argument");
        if (bc < RT_BC_THERMAL || bc > RT_BC_ARRAY || (bc == RT_BC_ARRAY && !I_bc))
            return fail(RT_EINVAL, "bad boundary condition");
        for (int k = 1; k < nz; ++k)
            if (!(z[k] > z[k - 1])) return fail(RT_EINVAL, "z must be strictly ascending");
        std::vector<int> hemi[2];
        for (int q = 0; q < ndir; ++q) {
            const double *u = dirs + 3 * q;
            if (u[2] == 0.0) return fail(RT_EINVAL, "directions need mu_z != 0");
            hemi[u[2] > 0 ? 0 : 1].push_back(q);
        }
        const size_t np = (size_t)nx * ny;
        const size_t ndh = std::max(hemi[0].size(), hemi[1].size());
        if (ndh > (size_t)NOALLOC_MAX_DH) return fail(RT_EINVAL, "at most 32 directions per hemisphere");
        const size_t need = 2 * (size_t)nlam * ndh * np;
        if (need > NOALLOC_SCRATCH_FLOATS)
            return fail(RT_EINVAL, "problem exceeds the static scratch: 2 * nlam * (directions per "
                                   "hemisphere) * nx * ny must not exceed 4194304 floats");
        float *scratch;
        RT_TRY(noalloc_scratch(&scratch));
        float *bufs[2] = {scratch, scratch + (size_t)nlam * ndh * np};
        cudaStream_t st = (cudaStream_t)stream;
        NoAllocPlane a;
        a.alpha = alpha;
        a.S = S;
        a.J = J;
        a.I_bc = I_bc;
        a.nx = nx;
        a.ny = ny;
        a.nz = nz;
        a.np = (int)np;
        a.nlam = nlam;
        a.periodic = periodic_xy ? 1 : 0;
        a.bc = bc;
        dim3 grid((unsigned)((np + 255) / 256), nlam);
        int first = 1;
        for (int h = 0; h < 2; ++h) {
            if (hemi[h].empty()) continue;
            a.up = h == 0;
            a.first = first;
            a.ndh = (int)hemi[h].size();
            for (int d = 0; d < a.ndh; ++d) {
                a.dg[d] = hemi[h][d];
                a.w[d] = (float)wdir[hemi[h][d]];
            }
            for (int s = 0; s < nz; ++s) {
                const int k = a.up ? s : nz - 1 - s;
                if (s > 0) {
                    const int ku = a.up ? k - 1 : k + 1;
                    for (int d = 0; d < a.ndh; ++d) {
                        const double *u = dirs + 3 * hemi[h][d];
                        const double ds = std::fabs(z[k] - z[ku]) / std::fabs(u[2]);
                        const double cx = -ds * u[0] / dx, cy = -ds * u[1] / dy;
                        const double fx = std::floor(cx), fy = std::floor(cy);
                        const double tx = cx - fx, ty = cy - fy;
                        Stencil &sc = a.st[d];
                        sc.ax = (int)fx;
                        sc.ay = (int)fy;
                        sc.axm = ((sc.ax % nx) + nx) % nx;
                        sc.aym = ((sc.ay % ny) + ny) % ny;
                        sc.w0 = (float)((1.0 - tx) * (1.0 - ty));
                        sc.w1 = (float)(tx * (1.0 - ty));
                        sc.w2 = (float)((1.0 - tx) * ty);
                        sc.w3 = (float)(tx * ty);
                        sc.hds = (float)(0.5 * ds);
                        sc.pad = 0.f;
                    }
                }
                a.step = s;
                a.Iprev = bufs[(s + 1) & 1];
                a.Inext = bufs[s & 1];
                note_launch();
                sc_plane_noalloc_kernel<<<grid, 256, 0, st>>>(a);
            }
            first = 0;
        }
        RT_CUDA(cudaGetLastError());
        return RT_OK;
    });
}
