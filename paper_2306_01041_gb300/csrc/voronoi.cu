// Voronoi grid: transport along Delaunay lines from the two best-aligned upwind neighbours
// (Sect. 2.5, Eq. 5 and the weight formula after it) with linear S across each segment (Eq. 2),
// swept per direction in dependency levels; J = sum_d w_d I_d (Eq. 4) in a fixed direction order.
//
// Layout: the fields are transposed once per call to site-major [nsites][nlam] so that the
// gather of an upwind site reads one contiguous wavelength vector; a thread owns one
// (site, wavelength) of the current level.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <string>

#include "device_common.cuh"
#include "rt_impl.h"

namespace rt {

// [rows][cols] -> [cols][rows]
__global__ void transpose_kernel(const float *__restrict__ in, float *__restrict__ out, int rows,
                                 int cols)
{
    __shared__ float tile[32][33];
    int c = blockIdx.x * 32 + threadIdx.x;
    int r0 = blockIdx.y * 32;
    for (int dr = threadIdx.y; dr < 32; dr += blockDim.y) {
        int r = r0 + dr;
        if (r < rows && c < cols) tile[dr][threadIdx.x] = in[(size_t)r * cols + c];
    }
    __syncthreads();
    int r = r0 + threadIdx.x;
    for (int dc = threadIdx.y; dc < 32; dc += blockDim.y) {
        int cc = blockIdx.x * 32 + dc;
        if (r < rows && cc < cols) out[(size_t)cc * rows + r] = tile[threadIdx.x][dc];
    }
}

static void transpose(const float *in, float *out, int rows, int cols, cudaStream_t st)
{
    dim3 grid((cols + 31) / 32, (rows + 31) / 32);
    note_launch();
    transpose_kernel<<<grid, dim3(32, 8), 0, st>>>(in, out, rows, cols);
}

__device__ __forceinline__ float w2_of(const Upwind &u) { return 1.f - u.w1; }
__device__ __forceinline__ double w2_of(const UpwindD &u) { return u.w2; }

template <class T, class UP = Upwind> struct VorArgsT {
    const UP *up;            // records of this direction (slot order, or site order if by_site)
    const int32_t *order;    // slot -> site
    const float *A, *S;      // [n][nlam]
    T *I;                    // [n][nlam] this direction
    float *J;                // [n][nlam] or null
    const float *I_bc;       // [nlam][n] of this direction (RT_BC_ARRAY) or null
    unsigned *err;
    int64_t s0, s1;          // slot range of the level
    int nlam, n, up_dir, bc, first, by_site;
    float w;
};
using VorArgs = VorArgsT<float>;

// Intensity of one site for one wavelength (Eq. 5 with linear S on each segment); T = float for
// the formal solution, double for the adjoint's forward pass.
template <class T, class UP>
__device__ __forceinline__ T site_intensity(const UP &u, int i, int l, const VorArgsT<T, UP> &a)
{
    const size_t il = (size_t)i * a.nlam + l;
    const T Si = (T)__ldg(a.S + il), Ai = (T)__ldg(a.A + il);
    T acc = 0;
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        const int k = c ? u.k2 : u.k1;
        const T wk = (T)(c ? w2_of(u) : u.w1);
        const T len = (T)(c ? u.l2 : u.l1);
        if (wk == (T)0) continue;
        T Ik, Sk, Ak;
        if (k >= 0) {
            const size_t kl = (size_t)k * a.nlam + l;
            Ik = a.I[kl];
            Sk = (T)__ldg(a.S + kl);
            Ak = (T)__ldg(a.A + kl);
        } else {
            Sk = Si;
            Ak = Ai;
            if (a.bc == RT_BC_ARRAY) Ik = (T)__ldg(a.I_bc + (size_t)l * a.n + i);
            else Ik = (a.bc == RT_BC_THERMAL && a.up_dir && k == -1) ? Si : (T)0;
        }
        T ex, w0, w1;
        lin_weights((T)0.5 * (Ak + Ai) * len, ex, w0, w1);
        acc += wk * (Ik * ex + w0 * Sk + w1 * Si);
    }
    return acc;
}

template <class T, class UP>
__global__ void __launch_bounds__(256) vor_level_kernel(const VorArgsT<T, UP> a)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t slot = a.s0 + t / a.nlam;
    const int l = (int)(t % a.nlam);
    if (slot >= a.s1) return;
    const int i = a.order[slot];
    const UP u = a.by_site ? a.up[i] : a.up[slot];
    const T v = site_intensity<T, UP>(u, i, l, a);
    const size_t il = (size_t)i * a.nlam + l;
    a.I[il] = v;
    if (a.J) {
        const float jv = a.first ? a.w * (float)v : a.J[il] + a.w * (float)v;
        if (!isfinite(jv)) flag_error(a.err, ERR_NAN);
        a.J[il] = jv;
    }
}

template <class T, class UP>
static void sweep_direction(const rt_grid *g, const VorTables &vt, int d, VorArgsT<T, UP> &a,
                            cudaStream_t st, const UP *site_records = nullptr)
{
    const int64_t n = g->nsites;
    if (site_records) {
        a.up = site_records;
        a.by_site = 1;
    } else {
        a.up = reinterpret_cast<const UP *>(vt.d_up) + (size_t)d * n;
        a.by_site = 0;
    }
    a.order = vt.d_order + (size_t)d * n;
    a.up_dir = vt.dirs[3 * d + 2] > 0;
    const std::vector<int64_t> &off = vt.lvl_off[d];
    for (size_t L = 0; L + 1 < off.size(); ++L) {
        a.s0 = off[L];
        a.s1 = off[L + 1];
        const int64_t work = (a.s1 - a.s0) * a.nlam;
        if (work <= 0) continue;
        note_launch();
        vor_level_kernel<T, UP><<<(unsigned)((work + 255) / 256), 256, 0, st>>>(a);
    }
}

// The persistent all-direction sweep (the batched kernel on this grid alone) applies to the
// plain formal solution: J only, thermal or zero inflow.  RT_VORONOI_SWEEP=levels selects the
// per-direction, per-level launches instead.
static bool self_batch_applies(int bc, const float *I_dir)
{
    const char *env = std::getenv("RT_VORONOI_SWEEP");
    if (env && std::string(env) == "levels") return false;
    return bc != RT_BC_ARRAY && !I_dir;
}

// The batch keeps (S, alpha) and one intensity array per direction for all its wavelengths,
// (2 + ndir) n P floats with P the wavelengths rounded up to 8.  When that exceeds half the free
// device memory (RT_VORONOI_BATCH_MB sets another budget), the batch is built for the largest
// divisor of nlam that fits and the formal solution runs the wavelengths in that many equal
// chunks: every wavelength is computed the same way, so J is the same.
static int self_batch_chunk(const rt_grid *g, int nlam)
{
    size_t budget = 0, total = 0;
    if (cudaMemGetInfo(&budget, &total) != cudaSuccess) return nlam;
    budget /= 2;
    if (const char *e = std::getenv("RT_VORONOI_BATCH_MB")) budget = (size_t)std::atoll(e) << 20;
    for (int d = nlam; d > 1; --d) {
        if (nlam % d) continue;
        const size_t bytes = (size_t)(2 + g->ndir) * g->nsites * (size_t)((d + 7) & ~7) * 4;
        if (bytes <= budget) return d;
    }
    return 1;
}

rt_status voronoi_prepare(rt_grid *g, int nlam)
{
    if (!self_batch_applies(RT_BC_THERMAL, nullptr)) return RT_OK;
    if (g->self_batch && g->self_batch_nlam == nlam) return RT_OK;
    if (g->self_batch) rt_batch_destroy(g->self_batch);
    g->self_batch = nullptr;
    rt_grid_t gg = g;
    RT_TRY(rt_batch_create(&gg, 1, self_batch_chunk(g, nlam), nullptr, 0, &g->self_batch));
    g->self_batch_nlam = nlam;
    return RT_OK;
}

rt_status voronoi_formal_solution(rt_grid *g, int nlam, const float *alpha, const float *S,
                                  int bc, const float *I_bc, float *J, float *I_dir,
                                  cudaStream_t st)
{
    if (self_batch_applies(bc, I_dir)) {
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        RT_CUDA(cudaStreamIsCapturing(st, &cap));
        // building the batch allocates: not while a stream is being captured
        if (cap == cudaStreamCaptureStatusNone) RT_TRY(voronoi_prepare(g, nlam));
        if (g->self_batch && g->self_batch_nlam == nlam) {
            const int nlc = batch_nlam(g->self_batch);   // a divisor of nlam
            const size_t n = (size_t)g->nsites;
            for (int l0 = 0; l0 < nlam; l0 += nlc) {
                const float *al[1] = {alpha + l0 * n}, *Sl[1] = {S + l0 * n};
                float *Jl[1] = {J + l0 * n};
                RT_TRY(rt_batch_formal_solution(g->self_batch, al, Sl, bc, Jl, st));
            }
            return RT_OK;
        }
    }
    const int64_t n = g->nsites;
    const size_t f = (size_t)n * nlam;
    void *p;
    RT_TRY(scratch_get(g, 0, 4 * f * sizeof(float) + (bc == RT_BC_ARRAY ? 0 : 0), &p));
    float *At = (float *)p, *St = At + f, *It = St + f, *Jt = It + f;
    transpose(alpha, At, nlam, (int)n, st);
    transpose(S, St, nlam, (int)n, st);
    VorArgs a;
    a.A = At;
    a.S = St;
    a.I = It;
    a.J = Jt;
    a.err = g->d_err;
    a.nlam = nlam;
    a.n = (int)n;
    a.bc = bc;
    for (int d = 0; d < g->ndir; ++d) {
        a.first = d == 0;
        a.w = (float)g->wdir[d];
        a.I_bc = bc == RT_BC_ARRAY ? I_bc + (size_t)d * f : nullptr;
        sweep_direction<float>(g, g->vt, d, a, st);
        if (I_dir) transpose(It, I_dir + (size_t)d * f, (int)n, nlam, st);
    }
    transpose(Jt, J, (int)n, nlam, st);
    RT_CUDA(cudaGetLastError());
    return RT_OK;
}

__global__ void gather_top_kernel(const float *I, const int64_t *top, float *out, int64_t ntop,
                                  int nlam)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ntop * nlam) return;
    const int l = (int)(t / ntop);
    const int64_t s = t % ntop;
    out[t] = I[(size_t)top[s] * nlam + l];
}

// forward sweep of one direction into It [n][nlam] (At, St already transposed); with
// site_records (FP64, site order) the adjoint's forward pass uses the unrounded tables
template <class T, class UP = Upwind>
static rt_status one_dir_forward(rt_grid *g, const VorTables &vt, int nlam, const float *At,
                                 const float *St, T *It, int bc, cudaStream_t st,
                                 const UP *site_records = nullptr)
{
    VorArgsT<T, UP> a;
    a.A = At;
    a.S = St;
    a.I = It;
    a.J = nullptr;
    a.I_bc = nullptr;
    a.err = g->d_err;
    a.nlam = nlam;
    a.n = (int)g->nsites;
    a.bc = bc;
    a.first = 1;
    a.w = 1.f;
    sweep_direction<T, UP>(g, vt, 0, a, st, site_records);
    RT_CUDA(cudaGetLastError());
    return RT_OK;
}

rt_status voronoi_emergent(rt_grid *g, const double *dir, int nlam, const float *alpha,
                           const float *S, int bc, float *I_top, cudaStream_t st)
{
    VorTables *vt;
    RT_TRY(voronoi_dir_tables_cached(g, dir, &vt, st));
    const int64_t n = g->nsites;
    const size_t f = (size_t)n * nlam;
    void *p;
    RT_TRY(scratch_get(g, 1, 3 * f * sizeof(float), &p));
    float *At = (float *)p, *St = At + f, *It = St + f;
    transpose(alpha, At, nlam, (int)n, st);
    transpose(S, St, nlam, (int)n, st);
    RT_TRY(one_dir_forward<float>(g, *vt, nlam, At, St, It, bc, st));
    const int64_t ntop = (int64_t)g->top.size();
    if (ntop) {
        note_launch();
        gather_top_kernel<<<(unsigned)((ntop * nlam + 255) / 256), 256, 0, st>>>(It, g->d_top,
                                                                                 I_top, ntop, nlam);
    }
    RT_CUDA(cudaGetLastError());
    return RT_OK;
}

// ---- adjoint ---------------------------------------------------------------------------------
// Reverse level order with a downwind list per site (the transpose of the upwind links), so
// every adjoint value is a gather: for site k with downwind pairs (i, c) (k is the c-th upwind of
// i), dL/dI_k = gI_loss(k) + sum w_c(i) e_c(i) dL/dI_i and the S, alpha gradients collect the
// matching w0 and dtau terms; then k adds the terms of its own segments (w1 S_k and alpha_k).
struct AdjV {
    const UpwindD *up_site;  // [n] FP64 records in site order
    const int32_t *order;    // level-ordered sites
    const int64_t *doff;     // [n+1] downwind CSR
    const int32_t *dsite;    // downwind site
    const int8_t *dcomp;     // which upwind slot (0, 1) of that site
    const float *A, *S;      // [n][nlam]
    const double *I;         // [n][nlam] forward intensity (FP64)
    double *G;               // [n][nlam] dL/dI (seeded with the loss gradient)
    double *gA, *gS;         // [n][nlam]
    int64_t s0, s1;
    int nlam, up_dir, bc;
};

// FP64 throughout (see the regular adjoint for why).
__global__ void __launch_bounds__(256) vor_adj_level(const AdjV a)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t slot = a.s0 + t / a.nlam;
    const int l = (int)(t % a.nlam);
    if (slot >= a.s1) return;
    const int k = a.order[slot];
    const size_t kl = (size_t)k * a.nlam + l;
    const double Sk = __ldg(a.S + kl), Ak = __ldg(a.A + kl), Ik = a.I[kl];
    double g = a.G[kl], gs = 0.0, ga = 0.0;
    // contributions of the downwind sites (all at higher levels, already final)
    for (int64_t e = a.doff[k]; e < a.doff[k + 1]; ++e) {
        const int i = a.dsite[e];
        const int c = a.dcomp[e];
        const UpwindD u = a.up_site[i];
        const double wk = c ? u.w2 : u.w1;
        const double len = c ? u.l2 : u.l1;
        const size_t il = (size_t)i * a.nlam + l;
        const double Si = __ldg(a.S + il), Ai = __ldg(a.A + il), gi = a.G[il] * wk;
        const double dt = 0.5 * (Ak + Ai) * len;
        double ex, w0, w1, dex, dw0, dw1;
        lin_weights(dt, ex, w0, w1);
        lin_weights_deriv(dt, ex, dex, dw0, dw1);
        // dI/ddtau = e (S_i - I_k) + w0' (S_k - S_i), from w0' + w1' = e
        const double gd = gi * (ex * (Si - Ik) + dw0 * (Sk - Si));
        g += ex * gi;
        gs += w0 * gi;
        ga += 0.5 * len * gd;
    }
    a.G[kl] = g;
    // k's own segments
    const UpwindD u = a.up_site[k];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        const int m = c ? u.k2 : u.k1;
        const double wk = c ? u.w2 : u.w1;
        const double len = c ? u.l2 : u.l1;
        if (wk == 0.0) continue;
        double Im, Sm, Am;
        const bool wall = m < 0;
        const bool thermal = wall && a.bc == RT_BC_THERMAL && a.up_dir && m == -1;
        if (!wall) {
            const size_t ml = (size_t)m * a.nlam + l;
            Im = a.I[ml];
            Sm = __ldg(a.S + ml);
            Am = __ldg(a.A + ml);
        } else {
            Sm = Sk;
            Am = Ak;
            Im = thermal ? Sk : 0.0;
        }
        const double dt = 0.5 * (Am + Ak) * len;
        double ex, w0, w1, dex, dw0, dw1;
        lin_weights(dt, ex, w0, w1);
        lin_weights_deriv(dt, ex, dex, dw0, dw1);
        const double gk = wk * g;
        const double gd = gk * (ex * (Sk - Im) + dw0 * (Sm - Sk));
        gs += w1 * gk;
        ga += 0.5 * len * gd;
        if (wall) {   // the wall node carries the site's own S and alpha (and I = S if thermal)
            gs += w0 * gk + (thermal ? ex * gk : 0.0);
            ga += 0.5 * len * gd;
        }
    }
    a.gS[kl] = gs;
    a.gA[kl] = ga;
}

__global__ void scatter_top_kernel(const float *gI_top, const int64_t *top, double *G,
                                   int64_t ntop, int nlam)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ntop * nlam) return;
    const int l = (int)(t / ntop);
    const int64_t s = t % ntop;
    G[(size_t)top[s] * nlam + l] = gI_top[t];
}

// [n][nlam] double -> [nlam][n] float
__global__ void transpose_d2f_kernel(const double *in, float *out, int64_t n, int nlam)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * nlam) return;
    const int l = (int)(t / n);
    const int64_t i = t % n;
    out[t] = (float)in[(size_t)i * nlam + l];
}

// workspace: At, St float [n][nlam]; It, G, gAt, gSt double [n][nlam]; up_site [n];
// downwind CSR (n + 1 offsets, 2n sites, 2n slots)
size_t voronoi_adjoint_ws(rt_grid *g, int nlam, int stride)
{
    (void)stride;
    const size_t n = (size_t)g->nsites;
    return 2 * n * nlam * sizeof(float) + 4 * n * nlam * sizeof(double) + n * sizeof(UpwindD) +
           (n + 1) * sizeof(int64_t) + 2 * n * sizeof(int32_t) + 2 * n * sizeof(int8_t) + 64 * 8;
}

static inline char *align_up(char *p)
{
    return (char *)(((uintptr_t)p + 63) & ~(uintptr_t)63);
}

rt_status voronoi_adjoint(rt_grid *g, const double *dir, int nlam, const float *alpha,
                          const float *S, int bc, const float *gI_top, float *g_alpha, float *g_S,
                          int stride, void *ws, size_t ws_bytes, cudaStream_t st)
{
    (void)stride;
    (void)ws_bytes;
    VorTables *vt;
    RT_TRY(voronoi_dir_tables_cached(g, dir, &vt, st));
    const int64_t n = g->nsites;
    const size_t f = (size_t)n * nlam;
    // downwind CSR of this direction (host)
    std::vector<int64_t> doff(n + 1, 0);
    for (int64_t i = 0; i < n; ++i) {
        const UpwindD &u = vt->h_upd[i];
        if (u.k1 >= 0) doff[u.k1 + 1]++;
        if (u.w2 > 0.0 && u.k2 >= 0) doff[u.k2 + 1]++;
    }
    for (int64_t i = 0; i < n; ++i) doff[i + 1] += doff[i];
    std::vector<int32_t> dsite(std::max<int64_t>(doff[n], 1));
    std::vector<int8_t> dcomp(std::max<int64_t>(doff[n], 1));
    std::vector<int64_t> pos(doff.begin(), doff.end() - 1);
    for (int64_t i = 0; i < n; ++i) {
        const UpwindD &u = vt->h_upd[i];
        if (u.k1 >= 0) { dsite[pos[u.k1]] = (int32_t)i; dcomp[pos[u.k1]++] = 0; }
        if (u.w2 > 0.0 && u.k2 >= 0) { dsite[pos[u.k2]] = (int32_t)i; dcomp[pos[u.k2]++] = 1; }
    }
    char *c = align_up((char *)ws);
    float *At = (float *)c, *St = At + f;
    c = align_up((char *)(St + f));
    double *It = (double *)c, *G = It + f, *gAt = G + f, *gSt = gAt + f;
    c = align_up((char *)(gSt + f));
    UpwindD *d_up_site = (UpwindD *)c;
    c = align_up((char *)(d_up_site + n));
    int64_t *d_doff = (int64_t *)c;
    c = align_up((char *)(d_doff + n + 1));
    int32_t *d_dsite = (int32_t *)c;
    c = align_up((char *)(d_dsite + std::max<int64_t>(doff[n], 1)));
    int8_t *d_dcomp = (int8_t *)c;
    RT_CUDA(cudaMemcpyAsync(d_up_site, vt->h_upd.data(), n * sizeof(UpwindD),
                            cudaMemcpyHostToDevice, st));
    RT_CUDA(cudaMemcpyAsync(d_doff, doff.data(), (n + 1) * sizeof(int64_t), cudaMemcpyHostToDevice,
                            st));
    if (doff[n]) {
        RT_CUDA(cudaMemcpyAsync(d_dsite, dsite.data(), doff[n] * sizeof(int32_t),
                                cudaMemcpyHostToDevice, st));
        RT_CUDA(cudaMemcpyAsync(d_dcomp, dcomp.data(), doff[n] * sizeof(int8_t),
                                cudaMemcpyHostToDevice, st));
    }
    transpose(alpha, At, nlam, (int)n, st);
    transpose(S, St, nlam, (int)n, st);
    const rt_status fwd = one_dir_forward<double, UpwindD>(g, *vt, nlam, At, St, It, bc, st,
                                                           d_up_site);
    if (fwd != RT_OK) return fwd;
    RT_CUDA(cudaMemsetAsync(G, 0, f * sizeof(double), st));
    const int64_t ntop = (int64_t)g->top.size();
    if (ntop) {
        note_launch();
        scatter_top_kernel<<<(unsigned)((ntop * nlam + 255) / 256), 256, 0, st>>>(gI_top, g->d_top,
                                                                                  G, ntop, nlam);
    }
    AdjV a;
    a.up_site = d_up_site;
    a.order = vt->d_order;
    a.doff = d_doff;
    a.dsite = d_dsite;
    a.dcomp = d_dcomp;
    a.A = At;
    a.S = St;
    a.I = It;
    a.G = G;
    a.gA = gAt;
    a.gS = gSt;
    a.nlam = nlam;
    a.up_dir = 1;
    a.bc = bc;
    const std::vector<int64_t> &off = vt->lvl_off[0];
    for (int L = (int)off.size() - 2; L >= 0; --L) {
        a.s0 = off[L];
        a.s1 = off[L + 1];
        const int64_t work = (a.s1 - a.s0) * nlam;
        if (work <= 0) continue;
        note_launch();
        vor_adj_level<<<(unsigned)((work + 255) / 256), 256, 0, st>>>(a);
    }
    const unsigned tb = (unsigned)((f + 255) / 256);
    note_launch();
    transpose_d2f_kernel<<<tb, 256, 0, st>>>(gAt, g_alpha, n, nlam);
    note_launch();
    transpose_d2f_kernel<<<tb, 256, 0, st>>>(gSt, g_S, n, nlam);
    RT_CUDA(cudaGetLastError());
    // the host vectors above were copied with pageable cudaMemcpyAsync, which completes its
    // read of host memory before returning
    return RT_OK;
}

}  // namespace rt
