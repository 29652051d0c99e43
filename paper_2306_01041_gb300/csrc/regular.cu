// Regular grid: plane-to-plane short characteristics (Sect. 2.6, after Kunasz & Auer 1988) with
// linear S across each interval (Sect. 2.5, Eq. 2), J accumulated over the hemisphere's
// directions in registers (Eq. 4); the emergent intensity of one direction and its adjoint.
//
// Sweep organisation: one launch per plane step.  A thread owns one point of the plane and one
// wavelength and loops over the directions of the hemisphere, so J is summed in a fixed order
// without atomics; the upwind plane of every direction lives in a ping-pong buffer
// [nlam][ndir_h][nx*ny] that stays resident in L2 between the launches.
#include <algorithm>
#include <cmath>

#include "device_common.cuh"
#include "rt_impl.h"

namespace rt {

template <class T, class ST = Stencil> struct SweepArgsT {
    const float *alpha, *S;      // [nlam][npt]
    const T *Iprev;              // [nlam][ndh][np]
    T *Inext;                    // [nlam][ndh][np]
    float *J;                    // [nlam][npt] or null
    float *I_dir;                // [ndir][nlam][npt] or null
    const float *I_bc;           // [ndir][nlam][np] or null
    const ST *st;                // [nz][st_stride]
    unsigned *err;
    int nx, ny, nz, np, nlam, ndh, ndir, st_stride;
    int up, periodic, bc, first;
    int dg[MAX_DIR];             // global direction index of each hemisphere slot
    int dst[MAX_DIR];            // stencil column of each hemisphere slot
    float w[MAX_DIR];            // quadrature weight of each slot
};
using SweepArgs = SweepArgsT<float>;

template <class T, class ST>
__device__ __forceinline__ T bilerp(const T *__restrict__ P, int o00, int o10, int o01, int o11,
                                    const ST &s)
{
    return (T)s.w0 * __ldg(P + o00) + (T)s.w1 * __ldg(P + o10) + (T)s.w2 * __ldg(P + o01) +
           (T)s.w3 * __ldg(P + o11);
}

template <class T, class ST>
__device__ __forceinline__ T bilerp_f(const float *__restrict__ P, int o00, int o10, int o01,
                                      int o11, const ST &s)
{
    return (T)s.w0 * (T)__ldg(P + o00) + (T)s.w1 * (T)__ldg(P + o10) +
           (T)s.w2 * (T)__ldg(P + o01) + (T)s.w3 * (T)__ldg(P + o11);
}

// T = float for the formal solution; T = double for the adjoint's forward recomputation
template <class T, class ST = Stencil>
__global__ void __launch_bounds__(256) sc_plane_kernel(const SweepArgsT<T, ST> a, int step)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    const int l = blockIdx.y;
    if (q >= a.np) return;
    const int i = q % a.nx, j = q / a.nx;
    const int k = a.up ? step : a.nz - 1 - step;
    const size_t npt = (size_t)a.np * a.nz;
    const float *al = a.alpha + (size_t)l * npt;
    const float *Sl = a.S + (size_t)l * npt;
    const T Sk = (T)__ldg(Sl + (size_t)k * a.np + q);
    T jacc = 0;
    if (step == 0) {
        for (int d = 0; d < a.ndh; ++d) {
            T v;
            if (a.bc == RT_BC_ARRAY)
                v = (T)__ldg(a.I_bc + ((size_t)a.dg[d] * a.nlam + l) * a.np + q);
            else
                v = (a.bc == RT_BC_THERMAL && a.up) ? Sk : (T)0;
            a.Inext[((size_t)l * a.ndh + d) * a.np + q] = v;
            jacc += (T)a.w[d] * v;
            if (a.I_dir)
                a.I_dir[((size_t)a.dg[d] * a.nlam + l) * npt + (size_t)k * a.np + q] = (float)v;
        }
    } else {
        const int ku = a.up ? k - 1 : k + 1;
        const T ak = (T)__ldg(al + (size_t)k * a.np + q);
        const float *Su = Sl + (size_t)ku * a.np;
        const float *Au = al + (size_t)ku * a.np;
        for (int d = 0; d < a.ndh; ++d) {
            const ST s = a.st[(size_t)k * a.st_stride + a.dst[d]];
            const T *Iu = a.Iprev + ((size_t)l * a.ndh + d) * a.np;
            T iu, su, au;
            if (a.periodic) {
                int x0 = i + s.axm;
                x0 -= (x0 >= a.nx) ? a.nx : 0;
                int x1 = x0 + 1 == a.nx ? 0 : x0 + 1;
                int y0 = j + s.aym;
                y0 -= (y0 >= a.ny) ? a.ny : 0;
                int y1 = y0 + 1 == a.ny ? 0 : y0 + 1;
                const int o00 = y0 * a.nx + x0, o10 = y0 * a.nx + x1;
                const int o01 = y1 * a.nx + x0, o11 = y1 * a.nx + x1;
                iu = bilerp<T, ST>(Iu, o00, o10, o01, o11, s);
                su = bilerp_f<T, ST>(Su, o00, o10, o01, o11, s);
                au = bilerp_f<T, ST>(Au, o00, o10, o01, o11, s);
            } else {
                // closed sides: no intensity enters from outside; S, alpha clamped to the edge
                const int xs[2] = {i + s.ax, i + s.ax + 1}, ys[2] = {j + s.ay, j + s.ay + 1};
                const T ws[4] = {(T)s.w0, (T)s.w1, (T)s.w2, (T)s.w3};
                iu = su = au = 0;
                for (int c = 0; c < 4; ++c) {
                    const int x = xs[c & 1], y = ys[c >> 1];
                    const bool in = x >= 0 && x < a.nx && y >= 0 && y < a.ny;
                    const int xc = min(max(x, 0), a.nx - 1), yc = min(max(y, 0), a.ny - 1);
                    const int o = yc * a.nx + xc;
                    if (in) iu += ws[c] * __ldg(Iu + o);
                    su += ws[c] * (T)__ldg(Su + o);
                    au += ws[c] * (T)__ldg(Au + o);
                }
            }
            const T dt = (au + ak) * (T)s.hds;
            T ex, w0, w1;
            lin_weights(dt, ex, w0, w1);
            const T v = iu * ex + w0 * su + w1 * Sk;
            a.Inext[((size_t)l * a.ndh + d) * a.np + q] = v;
            jacc += (T)a.w[d] * v;
            if (a.I_dir)
                a.I_dir[((size_t)a.dg[d] * a.nlam + l) * npt + (size_t)k * a.np + q] = (float)v;
        }
    }
    if (a.J) {
        float *Jp = a.J + (size_t)l * npt + (size_t)k * a.np + q;
        const float v = a.first ? (float)jacc : *Jp + (float)jacc;
        if (!isfinite(v)) flag_error(a.err, ERR_NAN);
        *Jp = v;
    }
}

// one hemisphere (the directions in `dirs`) over all planes; returns the last Inext buffer
static rt_status sweep_hemisphere(rt_grid *g, const std::vector<int> &dirs,
                                  const std::vector<float> &w, const Stencil *st, int st_stride,
                                  const std::vector<int> &st_col, int up, int nlam,
                                  const float *alpha, const float *S, int bc, const float *I_bc,
                                  float *J, int first, float *I_dir, float *buf0, float *buf1,
                                  float **last, cudaStream_t stream)
{
    SweepArgs a;
    a.alpha = alpha;
    a.S = S;
    a.J = J;
    a.I_dir = I_dir;
    a.I_bc = I_bc;
    a.st = st;
    a.err = g->d_err;
    a.nx = g->nx;
    a.ny = g->ny;
    a.nz = g->nz;
    a.np = g->nx * g->ny;
    a.nlam = nlam;
    a.ndh = (int)dirs.size();
    a.ndir = g->ndir;
    a.st_stride = st_stride;
    a.up = up;
    a.periodic = g->periodic;
    a.bc = bc;
    a.first = first;
    for (int d = 0; d < a.ndh; ++d) {
        a.dg[d] = dirs[d];
        a.dst[d] = st_col[d];
        a.w[d] = w[d];
    }
    dim3 grid((a.np + 255) / 256, nlam);
    float *bufs[2] = {buf0, buf1};
    for (int s = 0; s < g->nz; ++s) {
        a.Iprev = bufs[(s + 1) & 1];
        a.Inext = bufs[s & 1];
        note_launch();
        sc_plane_kernel<float><<<grid, 256, 0, stream>>>(a, s);
    }
    RT_CUDA(cudaGetLastError());
    *last = bufs[(g->nz - 1) & 1];
    return RT_OK;
}

rt_status regular_formal_solution(rt_grid *g, int nlam, const float *alpha, const float *S,
                                  int bc, const float *I_bc, float *J, float *I_dir,
                                  cudaStream_t st)
{
    if (nlam > 65535) return fail(RT_EINVAL, "nlam too large");
    if (g->sc_face) return face_formal_solution(g, nlam, alpha, S, bc, I_bc, J, I_dir, st);
    const size_t np = (size_t)g->nx * g->ny;
    const size_t ndh = std::max(g->dir_up.size(), g->dir_dn.size());
    void *p;
    RT_TRY(scratch_get(g, 0, 2 * (size_t)nlam * ndh * np * sizeof(float), &p));
    float *b0 = (float *)p, *b1 = b0 + (size_t)nlam * ndh * np;
    if (!I_dir) {
        bool done = false;
        RT_TRY(regular_tile_sweep(g, nlam, alpha, S, bc, J, b0, b1, st, &done));
        if (done) return RT_OK;
    }
    int first = 1;
    for (int hemi = 0; hemi < 2; ++hemi) {
        const std::vector<int> &dirs = hemi == 0 ? g->dir_up : g->dir_dn;
        if (dirs.empty()) continue;
        std::vector<float> w;
        for (int d : dirs) w.push_back((float)g->wdir[d]);
        float *last;
        RT_TRY(sweep_hemisphere(g, dirs, w, g->d_stencil, g->ndir, dirs, hemi == 0, nlam, alpha,
                                S, bc, I_bc, J, first, I_dir, b0, b1, &last, st));
        first = 0;
    }
    return RT_OK;
}

static rt_status one_dir_stencil(rt_grid *g, const double *dir, cudaStream_t st)
{
    if (g->d_stencil_one && g->one_dir[0] == dir[0] && g->one_dir[1] == dir[1] &&
        g->one_dir[2] == dir[2])
        return RT_OK;
    g->h_stencil_one = regular_dir_stencils(g, dir);
    g->h_stencil_oned = regular_dir_stencils_d(g, dir);
    if (!g->d_stencil_one) RT_CUDA(cudaMalloc(&g->d_stencil_one, g->nz * sizeof(Stencil)));
    if (!g->d_stencil_oned) RT_CUDA(cudaMalloc(&g->d_stencil_oned, g->nz * sizeof(StencilD)));
    RT_CUDA(cudaMemcpyAsync(g->d_stencil_one, g->h_stencil_one.data(), g->nz * sizeof(Stencil),
                            cudaMemcpyHostToDevice, st));
    RT_CUDA(cudaMemcpyAsync(g->d_stencil_oned, g->h_stencil_oned.data(), g->nz * sizeof(StencilD),
                            cudaMemcpyHostToDevice, st));
    RT_CUDA(cudaStreamSynchronize(st));
    g->one_dir[0] = dir[0];
    g->one_dir[1] = dir[1];
    g->one_dir[2] = dir[2];
    return RT_OK;
}

rt_status regular_emergent(rt_grid *g, const double *dir, int nlam, const float *alpha,
                           const float *S, int bc, float *I_top, cudaStream_t st)
{
    RT_TRY(one_dir_stencil(g, dir, st));
    const size_t np = (size_t)g->nx * g->ny;
    void *p;
    RT_TRY(scratch_get(g, 1, (size_t)nlam * np * sizeof(float), &p));
    float *last;
    std::vector<int> d1{0}, c1{0};
    std::vector<float> w1{1.f};
    // the top plane is written by the last step directly into I_top
    float *b = (float *)p;
    float *bufs[2];
    bufs[(g->nz - 1) & 1] = I_top;
    bufs[g->nz & 1] = b;
    RT_TRY(sweep_hemisphere(g, d1, w1, g->d_stencil_one, 1, c1, 1, nlam, alpha, S, bc, nullptr,
                            nullptr, 1, nullptr, bufs[0], bufs[1], &last, st));
    return RT_OK;
}

// ---- adjoint ---------------------------------------------------------------------------------
// Reverse sweep of one direction.  For plane k reached from plane ku = k - 1:
//   I_k = I_up e + w0 S_up + w1 S_k,  I_up = sum_c b_c I_ku(c) (same for S_up, alpha_up),
//   dtau = (alpha_up + alpha_k) hds.
// Pass A (points p of plane k, with gb = dL/dI_k(p)):
//   g_S_k += w1 gb;  gd = gb (I_up de + S_up dw0 + S_k dw1);  g_alpha_k += hds gd;
//   and the per-point factors E = e gb, W = w0 gb, D = hds gd for the upwind plane.
// Pass B (points q of plane ku): the transposed interpolation is a gather at the negated offset:
//   dL/dI_ku(q) = sum_c b_c E(q - a - c),  g_S_ku += sum_c b_c W(.),  g_alpha_ku += sum_c b_c D(.).
struct AdjArgs {
    const float *alpha, *S;   // [nlam][npt]
    const double *Iku;        // forward I of plane ku [nlam][np]
    const double *gIk;        // dL/dI of plane k [nlam][np]
    double *gIku;             // dL/dI of plane ku (out) [nlam][np]
    double *EWD;              // [3][nlam][np]
    double *g_alpha, *g_S;    // [nlam][npt] accumulators
    StencilD s;
    int nx, ny, np, nlam, k, ku;
    size_t npt;
};

// The adjoint runs in FP64: dL/dalpha collects differences (S_k - I_up, S_up - S_k) that cancel
// in optically thick layers, and one direction at a few wavelengths is a small volume.
__global__ void adj_pass_a(const AdjArgs a)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    const int l = blockIdx.y;
    if (q >= a.np) return;
    const int i = q % a.nx, j = q / a.nx;
    const StencilD &s = a.s;
    int x0 = i + s.axm;
    x0 -= (x0 >= a.nx) ? a.nx : 0;
    int x1 = x0 + 1 == a.nx ? 0 : x0 + 1;
    int y0 = j + s.aym;
    y0 -= (y0 >= a.ny) ? a.ny : 0;
    int y1 = y0 + 1 == a.ny ? 0 : y0 + 1;
    const int o00 = y0 * a.nx + x0, o10 = y0 * a.nx + x1, o01 = y1 * a.nx + x0,
              o11 = y1 * a.nx + x1;
    const float *al = a.alpha + (size_t)l * a.npt, *Sl = a.S + (size_t)l * a.npt;
    const double iu = bilerp<double, StencilD>(a.Iku + (size_t)l * a.np, o00, o10, o01, o11, s);
    const double su = bilerp_f<double, StencilD>(Sl + (size_t)a.ku * a.np, o00, o10, o01, o11, s);
    const double au = bilerp_f<double, StencilD>(al + (size_t)a.ku * a.np, o00, o10, o01, o11, s);
    const size_t pk = (size_t)l * a.npt + (size_t)a.k * a.np + q;
    const double Sk = (double)__ldg(Sl + (size_t)a.k * a.np + q);
    const double hds = (double)s.hds;
    const double dt = (au + (double)__ldg(al + (size_t)a.k * a.np + q)) * hds;
    double ex, w0, w1, dex, dw0, dw1;
    lin_weights(dt, ex, w0, w1);
    lin_weights_deriv(dt, ex, dex, dw0, dw1);
    const double gb = a.gIk[(size_t)l * a.np + q];
    // dI/ddtau = -e I_up + w0' S_up + w1' S_k = e (S_k - I_up) + w0' (S_up - S_k)  (w0' + w1' = e)
    const double gd = gb * (ex * (Sk - iu) + dw0 * (su - Sk));
    a.g_S[pk] += w1 * gb;
    a.g_alpha[pk] += hds * gd;
    const size_t m = (size_t)a.nlam * a.np;
    a.EWD[(size_t)l * a.np + q] = ex * gb;
    a.EWD[m + (size_t)l * a.np + q] = w0 * gb;
    a.EWD[2 * m + (size_t)l * a.np + q] = hds * gd;
}

__global__ void adj_pass_b(const AdjArgs a)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    const int l = blockIdx.y;
    if (q >= a.np) return;
    const int i = q % a.nx, j = q / a.nx;
    const StencilD &s = a.s;
    // p = q - a - c for the corners c = (0,0), (1,0), (0,1), (1,1) with weights w0..w3
    int xa = i - s.axm;
    xa += (xa < 0) ? a.nx : 0;                 // q.x - a.x (mod nx)
    int xb = xa - 1 < 0 ? a.nx - 1 : xa - 1;   // q.x - a.x - 1
    int ya = j - s.aym;
    ya += (ya < 0) ? a.ny : 0;
    int yb = ya - 1 < 0 ? a.ny - 1 : ya - 1;
    const int p00 = ya * a.nx + xa, p10 = ya * a.nx + xb, p01 = yb * a.nx + xa,
              p11 = yb * a.nx + xb;
    const size_t m = (size_t)a.nlam * a.np;
    const double *E = a.EWD + (size_t)l * a.np, *W = E + m, *D = E + 2 * m;
    const double c0 = s.w0, c1 = s.w1, c2 = s.w2, c3 = s.w3;
    const double gi = c0 * E[p00] + c1 * E[p10] + c2 * E[p01] + c3 * E[p11];
    const double gw = c0 * W[p00] + c1 * W[p10] + c2 * W[p01] + c3 * W[p11];
    const double gdd = c0 * D[p00] + c1 * D[p10] + c2 * D[p01] + c3 * D[p11];
    const size_t pk = (size_t)l * a.npt + (size_t)a.ku * a.np + q;
    a.gIku[(size_t)l * a.np + q] = gi;
    a.g_S[pk] += gw;
    a.g_alpha[pk] += gdd;
}

__global__ void adj_boundary(double *g_S, const double *gI0, int np, int nlam, size_t npt)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    const int l = blockIdx.y;
    if (q >= np) return;
    g_S[(size_t)l * npt + q] += gI0[(size_t)l * np + q];
}

__global__ void to_float_kernel(const double *in, float *out, size_t n)
{
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) out[t] = (float)in[t];
}

__global__ void to_double_kernel(const float *in, double *out, size_t n)
{
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) out[t] = (double)in[t];
}

// Workspace (FP64): checkpoints [ncp][nlam][np] (forward plane c*stride), segment planes
// [stride][nlam][np], EWD [3][nlam][np] (also the rolling pair of the first forward pass),
// adjoint planes [2][nlam][np], and the two gradient accumulators [2][nlam][npt].
size_t regular_adjoint_ws(rt_grid *g, int nlam, int stride)
{
    const size_t plane = (size_t)nlam * g->nx * g->ny * sizeof(double);
    const size_t ncp = (size_t)(g->nz + stride - 1) / stride;
    return (ncp + (size_t)stride + 3 + 2 + 2 * (size_t)g->nz) * plane;
}

rt_status regular_adjoint(rt_grid *g, const double *dir, int nlam, const float *alpha,
                          const float *S, int bc, const float *gI_top, float *g_alpha, float *g_S,
                          int stride, void *ws, size_t ws_bytes, cudaStream_t st)
{
    (void)ws_bytes;
    if (!g->periodic) return fail(RT_EINVAL, "the regular-grid adjoint needs periodic sides");
    RT_TRY(one_dir_stencil(g, dir, st));
    const int nz = g->nz;
    const size_t np = (size_t)g->nx * g->ny, plane = (size_t)nlam * np;
    const size_t npt = np * nz;
    const int ncp = (nz + stride - 1) / stride;
    double *ckpt = (double *)ws;
    double *seg = ckpt + (size_t)ncp * plane;
    double *EWD = seg + (size_t)stride * plane;
    double *gA = EWD + 3 * plane, *gB = gA + plane;
    double *accA = gB + plane, *accS = accA + (size_t)nlam * npt;
    const size_t pbytes = plane * sizeof(double);
    RT_CUDA(cudaMemsetAsync(accA, 0, 2 * (size_t)nlam * npt * sizeof(double), st));
    SweepArgsT<double, StencilD> a;
    a.alpha = alpha;
    a.S = S;
    a.J = nullptr;
    a.I_dir = nullptr;
    a.I_bc = nullptr;
    a.st = g->d_stencil_oned;
    a.err = g->d_err;
    a.nx = g->nx;
    a.ny = g->ny;
    a.nz = nz;
    a.np = (int)np;
    a.nlam = nlam;
    a.ndh = 1;
    a.ndir = 1;
    a.st_stride = 1;
    a.up = 1;
    a.periodic = 1;
    a.bc = bc;
    a.first = 1;
    a.dg[0] = 0;
    a.dst[0] = 0;
    a.w[0] = 1.f;
    dim3 grid((unsigned)((np + 255) / 256), nlam);
    auto step = [&](int k, const double *prev, double *next) {
        a.Iprev = prev;
        a.Inext = next;
        note_launch();
        sc_plane_kernel<double, StencilD><<<grid, 256, 0, st>>>(a, k);
    };
    // forward sweep keeping plane c*stride of every segment
    double *roll[2] = {EWD, EWD + plane};
    for (int k = 0; k < nz; ++k) {
        step(k, roll[(k + 1) & 1], roll[k & 1]);
        if (k % stride == 0)
            RT_CUDA(cudaMemcpyAsync(ckpt + (size_t)(k / stride) * plane, roll[k & 1], pbytes,
                                    cudaMemcpyDeviceToDevice, st));
    }
    // reverse sweep: segment c recomputes planes k0 .. kmax-1 and back-propagates kmax .. k0+1
    const unsigned cb = (unsigned)((plane + 255) / 256);
    note_launch();
    to_double_kernel<<<cb, 256, 0, st>>>(gI_top, gA, plane);
    AdjArgs b;
    b.alpha = alpha;
    b.S = S;
    b.EWD = EWD;
    b.g_alpha = accA;
    b.g_S = accS;
    b.nx = g->nx;
    b.ny = g->ny;
    b.np = (int)np;
    b.nlam = nlam;
    b.npt = npt;
    double *gcur = gA, *gnext = gB;
    for (int c = ncp - 1; c >= 0; --c) {
        const int k0 = c * stride, kmax = std::min(k0 + stride, nz - 1);
        if (kmax < k0 + 1) continue;
        RT_CUDA(cudaMemcpyAsync(seg, ckpt + (size_t)c * plane, pbytes, cudaMemcpyDeviceToDevice,
                                st));
        for (int k = k0 + 1; k < kmax; ++k)
            step(k, seg + (size_t)(k - 1 - k0) * plane, seg + (size_t)(k - k0) * plane);
        for (int k = kmax; k >= k0 + 1; --k) {
            b.k = k;
            b.ku = k - 1;
            b.s = g->h_stencil_oned[k];
            b.Iku = seg + (size_t)(k - 1 - k0) * plane;
            b.gIk = gcur;
            b.gIku = gnext;
            note_launch();
            adj_pass_a<<<grid, 256, 0, st>>>(b);
            note_launch();
            adj_pass_b<<<grid, 256, 0, st>>>(b);
            std::swap(gcur, gnext);
        }
    }
    if (bc == RT_BC_THERMAL) {
        note_launch();
        adj_boundary<<<grid, 256, 0, st>>>(accS, gcur, (int)np, nlam, npt);
    }
    const size_t tot = (size_t)nlam * npt;
    note_launch();
    to_float_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(accA, g_alpha, tot);
    note_launch();
    to_float_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(accS, g_S, tot);
    RT_CUDA(cudaGetLastError());
    return RT_OK;
}

}  // namespace rt
