// The 2 + 1 level hydrogen-like atom (Sect. 2.2, Table 1): opacity and source function from the
// populations, Saha-Boltzmann start, radiative + collisional rates, statistical equilibrium, and
// the Lambda iteration that ties them to the formal solution (Sect. 2.1, Eq. 3-4).
//
// Every transition i -> j (i lower) uses the LTE ratio g_ij(lambda) = (n_i/n_j)* e^(-hc/lambda kT):
//   alpha_ij = sigma (n_i - n_j g_ij),  eta_ij = sigma n_j g_ij 2hc^2/lambda^5,
//   R_ij = 4pi/(hc) sum_w sigma lambda J,  R_ji = 4pi/(hc) sum_w sigma lambda g_ij (2hc^2/lambda^5 + J).
// The line profile is a Voigt function with a small damping a, evaluated by its expansion in a:
//   H(a, v) = e^-v^2 (1 + a^2 (1 - 2 v^2)) + (2a/sqrt(pi)) G(v) + O(a^3),  G(v) = 2 v F(v) - 1,
// F Dawson's integral.  G is held as piecewise polynomials (built on the host from Dawson's
// integral by Rybicki's sampling-theorem series) on [0, 8) and by its asymptotic series beyond.
// Statistical equilibrium of three levels is solved by the Markov-chain-tree formula, whose terms
// are all positive: every population keeps full FP32 relative precision however small it is.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "device_common.cuh"
#include "rt_impl.h"

namespace rt {

// ---- constants (CODATA 2018) -------------------------------------------------------------------
static const double kH = 6.62607015e-34, kC = 299792458.0, kK = 1.380649e-23;
static const double kME = 9.1093837015e-31, kQE = 1.602176634e-19, kEPS0 = 8.8541878128e-12;
static const double kMH = 1.6735575e-27;

constexpr int MAX_LAM = 128;
constexpr int G_PIECES = 32;          // G(v) on [0, 8) in pieces of width 0.25
constexpr int G_DEG = 8;              // coefficients per piece (degree 7)

struct AtomDev {
    int nlam, nline;
    float lam0, dld_coef;             // Doppler width = dld_coef * sqrt(T)
    float a;                          // Voigt damping
    float c_line;                     // sigma_line = c_line * phi
    float E21;                        // J
    float chi[2];                     // ionisation energies of levels 1, 2 (J)
    float g1_g2, saha_g[2];           // g1/g2 and g_i/(2 g_p)
    float saha_c;                     // (h^2 / (2 pi m_e k))^(3/2)
    float q, kappa0;
    float inv_k;                      // 1/k
    // per wavelength
    float lam[MAX_LAM];
    float dlam[MAX_LAM];              // lambda - lambda0 (taken in double: FP32 would cancel)
    int kind[MAX_LAM];
    float wline[MAX_LAM];             // line quadrature weight (profile normalisation)
    float sig_bf[2][MAX_LAM];         // bound-free cross sections (0 above the edge)
    float dE_line[MAX_LAM];           // hc/lambda0 - hc/lambda (J)
    float dchi[2][MAX_LAM];           // chi_i - hc/lambda (J)
    float b_l5[MAX_LAM];              // 2hc^2/lambda^5
    float hc_lk[MAX_LAM];             // hc/(lambda k)
    float rate_f[MAX_LAM];            // 4 pi w lambda / (hc)
};

__constant__ AtomDev c_atom;
__constant__ float c_gpoly[G_PIECES * G_DEG];

// ---- Dawson's integral and G(v) on the host ----------------------------------------------------
// Rybicki's series: F(x) = lim_{h->0} pi^-1/2 sum_{n odd} exp(-(x - n h)^2) / n.
static double dawson_host(double x)
{
    const double h = 0.2;
    double s = 0.0;
    const int nmax = (int)std::ceil((std::fabs(x) + 8.0) / h) | 1;
    for (int n = -nmax; n <= nmax; n += 2) {
        const double t = x - n * h;
        s += std::exp(-t * t) / n;
    }
    return s / std::sqrt(M_PI);
}

static double G_host(double v) { return 2.0 * v * dawson_host(v) - 1.0; }

// Chebyshev interpolation at the Chebyshev points of each piece, converted to monomials of
// t = (v - centre) / half-width.
static void build_gpoly(std::vector<float> &out)
{
    out.assign(G_PIECES * G_DEG, 0.f);
    const double width = 8.0 / G_PIECES, hw = 0.5 * width;
    for (int p = 0; p < G_PIECES; ++p) {
        const double c = (p + 0.5) * width;
        double f[G_DEG], cheb[G_DEG];
        for (int m = 0; m < G_DEG; ++m) {
            const double t = std::cos(M_PI * (m + 0.5) / G_DEG);
            f[m] = G_host(c + hw * t);
        }
        for (int j = 0; j < G_DEG; ++j) {
            double s = 0.0;
            for (int m = 0; m < G_DEG; ++m) s += f[m] * std::cos(M_PI * j * (m + 0.5) / G_DEG);
            cheb[j] = (j == 0 ? 1.0 : 2.0) * s / G_DEG;
        }
        // monomial coefficients: T_j(t) expanded by the recurrence T_{j+1} = 2t T_j - T_{j-1}
        double T[G_DEG][G_DEG] = {{0}};
        T[0][0] = 1.0;
        if (G_DEG > 1) T[1][1] = 1.0;
        for (int j = 2; j < G_DEG; ++j)
            for (int e = 0; e < G_DEG; ++e)
                T[j][e] = (e > 0 ? 2.0 * T[j - 1][e - 1] : 0.0) - T[j - 2][e];
        for (int e = 0; e < G_DEG; ++e) {
            double s = 0.0;
            for (int j = 0; j < G_DEG; ++j) s += cheb[j] * T[j][e];
            out[p * G_DEG + e] = (float)s;
        }
    }
}

// ---- a scalar type carrying a derivative (forward mode), for the temperature chain rule -------
struct Dual {
    float v, d;
    __host__ __device__ Dual(float v_ = 0.f, float d_ = 0.f) : v(v_), d(d_) {}
};
__host__ __device__ inline Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
__host__ __device__ inline Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
__host__ __device__ inline Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
__host__ __device__ inline Dual operator/(Dual a, Dual b)
{
    float r = a.v / b.v;
    return Dual(r, (a.d - r * b.d) / b.v);
}
__host__ __device__ inline Dual operator*(float s, Dual a) { return Dual(s * a.v, s * a.d); }
__device__ inline Dual dexp(Dual a) { float e = expf(a.v); return Dual(e, e * a.d); }
__device__ inline Dual dexpm1(Dual a) { return Dual(expm1f(a.v), expf(a.v) * a.d); }
__device__ inline Dual dsqrt(Dual a) { float s = sqrtf(a.v); return Dual(s, 0.5f * a.d / s); }
__device__ inline float dexp(float a) { return expf(a); }
__device__ inline float dexpm1(float a) { return expm1f(a); }
__device__ inline float dsqrt(float a) { return sqrtf(a); }
__device__ inline float val(float a) { return a; }
__device__ inline float val(Dual a) { return a.v; }
template <class R> __device__ inline R mk(float v) { return R(v); }

// G(v) for v >= 0: piecewise polynomial on [0, 8), asymptotic series beyond.  ``tab`` is the
// block's shared-memory copy of the coefficients: the piece differs from thread to thread, and
// divergent reads of __constant__ memory would serialise.
template <class R> __device__ inline R G_eval(R v, const float *tab)
{
    const float vv = val(v);
    if (vv < 8.0f) {
        int p = min((int)(vv * (G_PIECES / 8.0f)), G_PIECES - 1);
        const float c = (p + 0.5f) * (8.0f / G_PIECES);
        const R t = (v - R(c)) * R(2.0f * G_PIECES / 8.0f);
        const float *co = tab + p * G_DEG;
        R s = R(co[G_DEG - 1]);
        for (int e = G_DEG - 2; e >= 0; --e) s = s * t + R(co[e]);
        return s;
    }
    // sum_{k>=1} (2k-1)!! / (2 v^2)^k, six terms
    const R x = R(1.0f) / (R(2.0f) * v * v);
    R s = R(10395.0f);
    s = s * x + R(945.0f);
    s = s * x + R(105.0f);
    s = s * x + R(15.0f);
    s = s * x + R(3.0f);
    s = s * x + R(1.0f);
    return s * x;
}

// Voigt H(a, v) for small a (see the file header)
template <class R> __device__ inline R voigt_H(float a, R v, const float *tab)
{
    R av = v;
    if (val(v) < 0.f) av = R(0.f) - v;   // H is even in v
    const R v2 = av * av;
    const R e = dexp(R(0.f) - v2);
    return e * (R(1.f) + R(a * a) * (R(1.f) - R(2.f) * v2)) +
           R(2.f * a * 0.56418958354775628f) * G_eval(av, tab);
}

// the coefficient table into shared memory (every thread of the block calls this)
__device__ inline void load_gtab(float *tab)
{
    for (int i = threadIdx.x; i < G_PIECES * G_DEG; i += blockDim.x) tab[i] = c_gpoly[i];
    __syncthreads();
}

// Planck function B_lambda(T) with x = hc/(lambda k T)
template <class R> __device__ inline R planck_dev(int j, R T)
{
    const R x = R(c_atom.hc_lk[j]) / T;
    return R(c_atom.b_l5[j]) / dexpm1(x);
}

// alpha and eta at node j of one point
template <class R>
__device__ inline void source_node(int j, R T, R rho, float ne, const float *pops, R phi_j,
                                   R &alpha, R &S)
{
    const AtomDev &A = c_atom;
    const R t5 = T * R(1.0f / 5000.0f);
    R t9 = t5 * t5;
    t9 = t9 * t9;
    t9 = t9 * t9 * t5;
    const R abg = R(A.kappa0) * rho * t9;
    const R kT = T * R(1.380649e-23f);
    const R B = planck_dev<R>(j, T);
    R al = abg, eta = abg * B;
    if (A.kind[j] == 0) {
        const R sig = R(A.c_line) * phi_j;
        const R g = R(A.g1_g2) * dexp(R(A.dE_line[j]) / kT);
        al = al + sig * (R(pops[0]) - R(pops[1]) * g);
        eta = eta + sig * R(pops[1]) * g * R(A.b_l5[j]);
    }
    const R tm32 = R(1.f) / (T * dsqrt(T));
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const float sb = A.sig_bf[i][j];
        if (sb == 0.f) continue;
        const R g = R(ne * A.saha_g[i] * A.saha_c) * tm32 * dexp(R(A.dchi[i][j]) / kT);
        al = al + R(sb) * (R(pops[i]) - R(pops[2]) * g);
        eta = eta + R(sb) * R(pops[2]) * g * R(A.b_l5[j]);
    }
    alpha = al;
    S = eta / al;
}

// The line profile at every line node of one point, normalised so that sum_j w_j phi_j = 1;
// ph[j] is indexed by the node (entries of continuum nodes are left unset).
template <class R> __device__ inline void line_profiles(R dld, const float *tab, R *ph)
{
    R s = R(0.f);
    const R inv = R(1.f) / dld;
    for (int j = 0; j < c_atom.nlam; ++j) {
        if (c_atom.kind[j] != 0) continue;
        const R v = R(c_atom.dlam[j]) * inv;
        ph[j] = voigt_H<R>(c_atom.a, v, tab) * R(0.56418958354775628f) * inv;
        s = s + R(c_atom.wline[j]) * ph[j];
    }
    const R ninv = R(1.f) / s;
    for (int j = 0; j < c_atom.nlam; ++j)
        if (c_atom.kind[j] == 0) ph[j] = ph[j] * ninv;
}

__global__ void source_terms_kernel(int64_t npt, const float *T, const float *rho, const float *ne,
                                    const float *pops, float *alpha, float *S, unsigned *err)
{
    __shared__ float tab[G_PIECES * G_DEG];
    load_gtab(tab);
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npt) return;
    const float t = T[p], r = rho[p], e = ne[p];
    const float pp[3] = {pops[p], pops[npt + p], pops[2 * npt + p]};
    float ph[MAX_LAM];
    line_profiles<float>(c_atom.dld_coef * sqrtf(t), tab, ph);
    bool bad = false;
    for (int j = 0; j < c_atom.nlam; ++j) {
        float a, s;
        source_node<float>(j, t, r, e, pp, c_atom.kind[j] == 0 ? ph[j] : 0.f, a, s);
        alpha[(size_t)j * npt + p] = a;
        S[(size_t)j * npt + p] = s;
        bad |= !isfinite(a) || !isfinite(s);
    }
    if (bad) flag_error(err, ERR_NAN);
}

// g_T = sum_j (g_alpha_j dalpha_j/dT + g_S_j dS_j/dT), populations fixed
__global__ void source_terms_adjoint_kernel(int64_t npt, const float *T, const float *rho,
                                            const float *ne, const float *pops, const float *ga,
                                            const float *gs, float *gT)
{
    __shared__ float tab[G_PIECES * G_DEG];
    load_gtab(tab);
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npt) return;
    const Dual t(T[p], 1.f);
    const Dual r(rho[p], 0.f);
    const float e = ne[p];
    const float pp[3] = {pops[p], pops[npt + p], pops[2 * npt + p]};
    Dual ph[MAX_LAM];
    line_profiles<Dual>(Dual(c_atom.dld_coef) * dsqrt(t), tab, ph);
    float acc = 0.f;
    for (int j = 0; j < c_atom.nlam; ++j) {
        Dual a, s;
        source_node<Dual>(j, t, r, e, pp, c_atom.kind[j] == 0 ? ph[j] : Dual(0.f), a, s);
        acc += ga[(size_t)j * npt + p] * a.d + gs[(size_t)j * npt + p] * s.d;
    }
    gT[p] = acc;
}

__global__ void lte_pops_kernel(int64_t npt, const float *T, const float *ne, const float *nH,
                                float *pops)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npt) return;
    const AtomDev &A = c_atom;
    const float t = T[p], kT = t * 1.380649e-23f;
    const float r21 = (1.f / A.g1_g2) * expf(-A.E21 / kT);
    // n_p / n_1 = 1 / (n_e Phi_1),  Phi_1 = g1/(2 g_p) (h^2/(2 pi m_e k T))^1.5 e^(chi_1/kT)
    const float rp1 = t * sqrtf(t) * expf(-A.chi[0] / kT) / (ne[p] * A.saha_g[0] * A.saha_c);
    const float n1 = nH[p] / (1.f + r21 + rp1);
    pops[p] = n1;
    pops[npt + p] = n1 * r21;
    pops[2 * npt + p] = n1 * rp1;
}

__device__ inline void atomic_max_pos(float *addr, float v)
{
    // non-negative floats order like their bit patterns
    atomicMax(reinterpret_cast<unsigned *>(addr), __float_as_uint(v));
}

// Radiative rate coefficients of node j at one point: the node feeds transition lo -> hi with
// R_lo,hi += fs J and R_hi,lo += fs g (2hc^2/lambda^5 + J).
__device__ inline void node_rate(int j, float e, float kT, float tm32, const float *ph, float &fs,
                                 float &g, int &lo, int &hi)
{
    const AtomDev &A = c_atom;
    float sig;
    if (A.kind[j] == 0) {
        sig = A.c_line * ph[j];
        g = A.g1_g2 * expf(A.dE_line[j] / kT);
        lo = 0;
        hi = 1;
    } else {
        const int i = A.kind[j] - 1;
        sig = A.sig_bf[i][j];
        g = e * A.saha_g[i] * A.saha_c * tm32 * expf(A.dchi[i][j] / kT);
        lo = i;
        hi = 2;
    }
    fs = A.rate_f[j] * sig;
}

__device__ inline void add_collisions(float (&P)[3][3], float t, float e, float kT, float tm32)
{
    const AtomDev &A = c_atom;
    const float cb = A.q * e * rsqrtf(t);
    P[1][0] += cb;
    P[0][1] += cb * (1.f / A.g1_g2) * expf(-A.E21 / kT);
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const float cip = cb * expf(-A.chi[i] / kT);
        P[i][2] += cip;
        // C_pi = C_ip n_e Phi_i = cb n_e g_i/(2 g_p) saha_c T^-1.5 (exponentials cancel);
        // n_e saha_c is formed first: cb n_e alone can exceed the FP32 range
        P[2][i] += cb * ((e * A.saha_c) * tm32 * A.saha_g[i]);
    }
}

// Steady state of the three-level rate matrix P (rates i -> j), scaled to n1 + n2 + np = nH.
__device__ inline void mct_solve(float (&P)[3][3], float nH, float (&nn)[3])
{
    // scale to avoid FP32 range issues in the products
    float m = 0.f;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) m = fmaxf(m, P[a][b]);
    const float s = 1.f / m;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) P[a][b] *= s;
    // Markov-chain-tree steady state of three levels
    const float t1 = P[1][0] * P[2][0] + P[1][2] * P[2][0] + P[2][1] * P[1][0];
    const float t2 = P[0][1] * P[2][1] + P[0][2] * P[2][1] + P[2][0] * P[0][1];
    const float t3 = P[0][2] * P[1][2] + P[0][1] * P[1][2] + P[1][0] * P[0][2];
    const float f = nH / (t1 + t2 + t3);
    nn[0] = t1 * f;
    nn[1] = t2 * f;
    nn[2] = t3 * f;
}

// new populations of one point: max |dn/n| into a block maximum, then one atomic per block
__device__ inline void store_pops(int64_t npt, int64_t p, const float (&nn)[3], float *pops,
                                  float *dmax, unsigned *err, bool active)
{
    float change = 0.f;
    if (active) {
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const float old = pops[(size_t)i * npt + p];
            change = fmaxf(change, fabsf(nn[i] - old) / nn[i]);
            pops[(size_t)i * npt + p] = nn[i];
        }
        if (!isfinite(change)) {
            flag_error(err, ERR_NAN);
            change = 0.f;
        }
    }
    __shared__ float red[8];
    float v = change;
    for (int o = 16; o; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.f;
        for (int o = 4; o; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (threadIdx.x == 0 && dmax) atomic_max_pos(dmax, v);
    }
}

// rates -> statistical equilibrium -> new populations and max |dn/n|
__global__ void __launch_bounds__(256) se_kernel(int64_t npt, const float *T, const float *ne,
                                                 const float *nH, const float *J, float *pops,
                                                 float *dmax, unsigned *err)
{
    __shared__ float tab[G_PIECES * G_DEG];
    load_gtab(tab);
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float nn[3] = {0.f, 0.f, 0.f};
    if (p < npt) {
        const AtomDev &A = c_atom;
        const float t = T[p], e = ne[p], kT = t * 1.380649e-23f;
        float ph[MAX_LAM];
        line_profiles<float>(A.dld_coef * sqrtf(t), tab, ph);
        const float tm32 = 1.f / (t * sqrtf(t));
        float P[3][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
        for (int j = 0; j < A.nlam; ++j) {
            const float Jj = J[(size_t)j * npt + p];
            float fs, g;
            int lo, hi;
            node_rate(j, e, kT, tm32, ph, fs, g, lo, hi);
            P[lo][hi] += fs * Jj;
            P[hi][lo] += fs * g * (A.b_l5[j] + Jj);
        }
        add_collisions(P, t, e, kT, tm32);
        mct_solve(P, nH[p], nn);
    }
    store_pops(npt, p, nn, pops, dmax, err, p < npt);
}

// Accelerated update (the point's own contribution to J treated implicitly): the populations n
// with n = SE(J + Lambda* (S(n) - S_old)), by Newton's method on the logarithms of the two
// smaller populations from the current ones (the largest follows from n1 + n2 + np = nH), with
// a forward-difference Jacobian (step 1e-3 in log n).  A step that is not finite or leaves no
// room for the largest population is replaced by the plain update; newton = 0 is the plain
// update.  At a fixed point of the iteration the current populations solve the equation, so
// the step is zero there.
//
// One warp per point: lane q holds wavelength nodes q and q + 32 (nlam <= 64), with the node's
// opacity and emissivity as linear functions of (n1, n2, np) -- alpha = a0 + a1 n1 + a2 n2 +
// ap np, eta = e0 + e2 n2 + ep np (the same terms as source_node) -- so one evaluation of the
// rates costs a few multiply-adds per node and a warp reduction.  A block of 8 warps takes 32
// consecutive points and stages their J, Lambda*, S_old rows through shared memory (coalesced).
constexpr int ALI_PTS = 32, ALI_WARPS = 8;

__global__ void __launch_bounds__(ALI_WARPS * 32, 3) se_ali_kernel(
    int64_t npt, const float *T, const float *rho, const float *ne, const float *nH,
    const float *J, const float *L, const float *S_old, float *pops, float *dmax, unsigned *err,
    int newton)
{
    __shared__ float tab[G_PIECES * G_DEG];
    __shared__ float sJ[64][ALI_PTS], sL[64][ALI_PTS], sS[64][ALI_PTS];
    __shared__ float red[ALI_WARPS];
    // per-node atom constants: lanes read different nodes, which the constant cache serialises
    enum { N_DLAM, N_WLINE, N_SB0, N_SB1, N_DEL, N_DCHI0, N_DCHI1, N_BL5, N_HCLK, N_RATEF, N_KIND,
           N_COUNT };
    __shared__ float snode[N_COUNT][64];
    load_gtab(tab);
    const AtomDev &A = c_atom;
    const int nl = A.nlam;
    for (int j = threadIdx.x; j < nl; j += blockDim.x) {
        snode[N_DLAM][j] = A.dlam[j];
        snode[N_WLINE][j] = A.wline[j];
        snode[N_SB0][j] = A.sig_bf[0][j];
        snode[N_SB1][j] = A.sig_bf[1][j];
        snode[N_DEL][j] = A.dE_line[j];
        snode[N_DCHI0][j] = A.dchi[0][j];
        snode[N_DCHI1][j] = A.dchi[1][j];
        snode[N_BL5][j] = A.b_l5[j];
        snode[N_HCLK][j] = A.hc_lk[j];
        snode[N_RATEF][j] = A.rate_f[j];
        snode[N_KIND][j] = (float)A.kind[j];
    }
    const int64_t p0 = (int64_t)blockIdx.x * ALI_PTS;
    for (int e = threadIdx.x; e < nl * ALI_PTS; e += blockDim.x) {
        const int l = e / ALI_PTS, c = e % ALI_PTS;
        const int64_t p = p0 + c;
        const bool in = p < npt;
        sJ[l][c] = in ? J[(size_t)l * npt + p] : 0.f;
        sL[l][c] = in ? L[(size_t)l * npt + p] : 0.f;
        sS[l][c] = in ? S_old[(size_t)l * npt + p] : 0.f;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float wmax = 0.f;
    for (int c = warp; c < ALI_PTS; c += ALI_WARPS) {
        const int64_t p = p0 + c;
        if (p >= npt) break;
        const float t = T[p], r = rho[p], e = ne[p], nh = nH[p], kT = t * 1.380649e-23f;
        const float tm32 = 1.f / (t * sqrtf(t));
        const float t5 = t * (1.f / 5000.f);
        float t9 = t5 * t5;
        t9 = t9 * t9;
        t9 = t9 * t9 * t5;
        const float abg = A.kappa0 * r * t9;
        // line profile of this point, normalised over the line nodes
        const float dld = A.dld_coef * sqrtf(t), inv = 1.f / dld;
        float phr[2] = {0.f, 0.f}, psum = 0.f;
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int j = lane + 32 * q;
            if (j < nl && snode[N_KIND][j] == 0.f) {
                phr[q] = voigt_H<float>(A.a, snode[N_DLAM][j] * inv, tab) * 0.56418958354775628f * inv;
                psum += snode[N_WLINE][j] * phr[q];
            }
        }
        for (int o = 16; o; o >>= 1) psum += __shfl_xor_sync(0xffffffffu, psum, o);
        const float ninv = 1.f / psum;
        // per node: linear opacity and emissivity, rate coefficients, J_eff and Lambda*
        float ca0[2], ca1[2], ca2[2], cap[2], ce0[2], ce2[2], cep[2], jef[2], lst[2], fs[2],
            fsg[2], fsgb[2];
        int tr[2];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int j = lane + 32 * q;
            tr[q] = -1;
            if (j >= nl) continue;
            const int kd = (int)snode[N_KIND][j];
            const float bl5 = snode[N_BL5][j];
            const float B = bl5 / expm1f(snode[N_HCLK][j] / t);   // as planck_dev
            const float sigl = kd == 0 ? A.c_line * phr[q] * ninv : 0.f;
            const float gl = kd == 0 ? A.g1_g2 * expf(snode[N_DEL][j] / kT) : 0.f;
            float sb[2], gb[2];
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                sb[i] = snode[N_SB0 + i][j];
                gb[i] = sb[i] == 0.f ? 0.f
                                     : (e * A.saha_g[i] * A.saha_c) * tm32 *
                                           expf(snode[N_DCHI0 + i][j] / kT);
            }
            ca0[q] = abg;
            ca1[q] = sigl + sb[0];
            ca2[q] = sb[1] - sigl * gl;
            cap[q] = -(sb[0] * gb[0] + sb[1] * gb[1]);
            ce0[q] = abg * B;
            ce2[q] = bl5 * sigl * gl;
            cep[q] = bl5 * (sb[0] * gb[0] + sb[1] * gb[1]);
            lst[q] = sL[j][c];
            jef[q] = sJ[j][c] - lst[q] * sS[j][c];
            const float sig = kd == 0 ? sigl : (kd == 1 ? sb[0] : sb[1]);
            const float gg = kd == 0 ? gl : (kd == 1 ? gb[0] : gb[1]);
            fs[q] = snode[N_RATEF][j] * sig;
            fsg[q] = fs[q] * gg;
            fsgb[q] = fsg[q] * bl5;
            tr[q] = kd;
        }
        // collisional rates: independent of the populations
        float Pc[3][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
        add_collisions(Pc, t, e, kT, tm32);
        // the plain update with the radiation of the populations n (identical in every lane)
        auto G = [&](const float (&n)[3], float (&out)[3]) {
            float up[3] = {0.f, 0.f, 0.f}, dn[3] = {0.f, 0.f, 0.f};
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                if (tr[q] < 0) continue;
                const float al = ca0[q] + ca1[q] * n[0] + ca2[q] * n[1] + cap[q] * n[2];
                const float et = ce0[q] + ce2[q] * n[1] + cep[q] * n[2];
                const float Jj = jef[q] + lst[q] * (et / al);
#pragma unroll
                for (int k = 0; k < 3; ++k)
                    if (tr[q] == k) {
                        up[k] += fs[q] * Jj;
                        dn[k] += fsg[q] * Jj + fsgb[q];
                    }
            }
#pragma unroll
            for (int k = 0; k < 3; ++k)
                for (int o = 16; o; o >>= 1) {
                    up[k] += __shfl_xor_sync(0xffffffffu, up[k], o);
                    dn[k] += __shfl_xor_sync(0xffffffffu, dn[k], o);
                }
            float P[3][3] = {{0.f, up[0] + Pc[0][1], up[1] + Pc[0][2]},
                             {dn[0] + Pc[1][0], 0.f, up[2] + Pc[1][2]},
                             {dn[1] + Pc[2][0], dn[2] + Pc[2][1], 0.f}};
            mct_solve(P, nh, out);
        };
        const float cur[3] = {pops[p], pops[npt + p], pops[2 * npt + p]};
        float nn[3];
        if (newton == 0) {
            G(cur, nn);
        } else {
            const int big = (cur[0] >= cur[1] && cur[0] >= cur[2]) ? 0 : (cur[1] >= cur[2] ? 1 : 2);
            const int s0 = big == 0 ? 1 : 0, s1 = big == 2 ? 1 : 2;
            // runtime level indices through selects (an indexed array would live in local memory)
            auto pick = [](const float (&v)[3], int i) { return i == 0 ? v[0] : (i == 1 ? v[1] : v[2]); };
            float x[2] = {pick(cur, s0), pick(cur, s1)};
            auto full = [&](const float (&xx)[2], float (&n)[3]) {
                const float rest = nh - xx[0] - xx[1];
#pragma unroll
                for (int k = 0; k < 3; ++k) n[k] = k == big ? rest : (k == s0 ? xx[0] : xx[1]);
            };
            const float h = 1e-3f, eh = expf(h);
            for (int it = 0; it < newton; ++it) {
                float n[3], g0[3];
                full(x, n);
                G(n, g0);
                const float H0[2] = {logf(pick(g0, s0)) - logf(x[0]), logf(pick(g0, s1)) - logf(x[1])};
                float Jm[2][2];
#pragma unroll
                for (int cc = 0; cc < 2; ++cc) {
                    float xp[2] = {x[0], x[1]};
                    xp[cc] *= eh;
                    float np_[3], gp[3];
                    full(xp, np_);
                    G(np_, gp);
                    Jm[0][cc] = (logf(pick(gp, s0)) - logf(xp[0]) - H0[0]) / h;
                    Jm[1][cc] = (logf(pick(gp, s1)) - logf(xp[1]) - H0[1]) / h;
                }
                const float det = Jm[0][0] * Jm[1][1] - Jm[0][1] * Jm[1][0];
                const float st0 = (Jm[1][1] * H0[0] - Jm[0][1] * H0[1]) / det;
                const float st1 = (-Jm[1][0] * H0[0] + Jm[0][0] * H0[1]) / det;
                const float xn0 = x[0] * expf(-st0), xn1 = x[1] * expf(-st1);
                const bool bad = !isfinite(xn0) || !isfinite(xn1) || !(xn0 + xn1 < nh);
                x[0] = bad ? pick(g0, s0) : xn0;
                x[1] = bad ? pick(g0, s1) : xn1;
            }
            full(x, nn);
        }
        if (lane == 0) {
            float change = 0.f;
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                change = fmaxf(change, fabsf(nn[i] - cur[i]) / nn[i]);
                pops[(size_t)i * npt + p] = nn[i];
            }
            if (!isfinite(change)) {
                flag_error(err, ERR_NAN);
                change = 0.f;
            }
            wmax = fmaxf(wmax, change);
        }
    }
    if (lane == 0) red[warp] = wmax;
    __syncthreads();
    if (threadIdx.x == 0 && dmax) {
        float v = 0.f;
        for (int w = 0; w < ALI_WARPS; ++w) v = fmaxf(v, red[w]);
        atomic_max_pos(dmax, v);
    }
}

static inline unsigned ali_blocks(int64_t n) { return (unsigned)((n + ALI_PTS - 1) / ALI_PTS); }

__global__ void lte_source_kernel(int64_t npt, const float *T, const float *rho, float kappa0,
                                  float b_l5, float hc_lk, float *alpha, float *S)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npt) return;
    const float t = T[p];
    const float t5 = t * (1.f / 5000.f);
    float t9 = t5 * t5;
    t9 = t9 * t9;
    t9 = t9 * t9 * t5;
    alpha[p] = kappa0 * rho[p] * t9;
    S[p] = b_l5 / expm1f(hc_lk / t);
}

__global__ void lte_source_adjoint_kernel(int64_t npt, const float *T, const float *rho,
                                          float kappa0, float b_l5, float hc_lk, const float *ga,
                                          const float *gs, float *gT)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npt) return;
    const float t = T[p];
    const float t5 = t * (1.f / 5000.f);
    float t9 = t5 * t5;
    t9 = t9 * t9;
    t9 = t9 * t9 * t5;
    const float alpha = kappa0 * rho[p] * t9;
    const float x = hc_lk / t;
    const float em = expm1f(x);
    const float B = b_l5 / em;
    const float dB = B * x / t * (em + 1.f) / em;
    gT[p] = ga[p] * 9.f * alpha / t + gs[p] * dB;
}

// ---- host side ------------------------------------------------------------------------------------
// The atom's constants live in __constant__ memory, one copy per device: uploaded when the atom
// differs from the last one uploaded to the current device (per-device cache under a mutex, so
// host threads and devices do not mix).
constexpr int MAX_DEVICES = 64;

static rt_status load_atom(const rt_atom *at)
{
    static std::mutex mu;
    static std::vector<float> gpoly;
    static bool gp_done[MAX_DEVICES] = {};
    if (!at || !at->lam || !at->wlam || !at->kind) return fail(RT_EINVAL, "incomplete atom");
    if (at->nlam < 1 || at->nlam > MAX_LAM) return fail(RT_EINVAL, "atom nlam must be 1..128");
    int dev = 0;
    RT_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= MAX_DEVICES) return fail(RT_EINVAL, "device index beyond 63");
    std::lock_guard<std::mutex> lock(mu);
    if (!gp_done[dev]) {
        if (gpoly.empty()) build_gpoly(gpoly);
        RT_CUDA(cudaMemcpyToSymbol(c_gpoly, gpoly.data(), gpoly.size() * sizeof(float)));
        gp_done[dev] = true;
    }
    AtomDev A;
    std::memset(&A, 0, sizeof(A));
    const double hc = kH * kC;
    const double E[3] = {at->E_cm[0] * 100.0 * hc, at->E_cm[1] * 100.0 * hc, at->E_cm[2] * 100.0 * hc};
    const double lam0 = hc / (E[1] - E[0]);
    const double edge[2] = {hc / (E[2] - E[0]), hc / (E[2] - E[1])};
    const double kram = 64.0 * std::pow(M_PI, 4) * kME * std::pow(kQE, 10) /
                        (3.0 * std::sqrt(3.0) * kC * std::pow(kH, 6) * std::pow(4.0 * M_PI * kEPS0, 5));
    double sig_edge[2];
    for (int i = 0; i < 2; ++i) sig_edge[i] = kram / (std::pow(i + 1.0, 5) * std::pow(kC / edge[i], 3));
    A.nlam = at->nlam;
    A.lam0 = (float)lam0;
    A.dld_coef = (float)(lam0 / kC * std::sqrt(2.0 * kK / kMH));
    A.a = (float)at->voigt_a;
    A.c_line = (float)(M_PI * kQE * kQE / (4.0 * M_PI * kEPS0 * kME * kC) * at->f_line * lam0 * lam0 / kC);
    A.E21 = (float)(E[1] - E[0]);
    A.chi[0] = (float)(E[2] - E[0]);
    A.chi[1] = (float)(E[2] - E[1]);
    A.g1_g2 = (float)(at->g[0] / at->g[1]);
    A.saha_g[0] = (float)(at->g[0] / (2.0 * at->g[2]));
    A.saha_g[1] = (float)(at->g[1] / (2.0 * at->g[2]));
    A.saha_c = (float)std::pow(kH * kH / (2.0 * M_PI * kME * kK), 1.5);
    A.q = (float)at->q_coll;
    A.kappa0 = (float)at->kappa0;
    A.inv_k = (float)(1.0 / kK);
    int nline = 0;
    for (int j = 0; j < at->nlam; ++j) {
        const double l = at->lam[j];
        if (!(l > 0) || at->kind[j] < 0 || at->kind[j] > 2) return fail(RT_EINVAL, "bad wavelength node");
        A.lam[j] = (float)l;
        A.dlam[j] = (float)(l - lam0);
        A.kind[j] = at->kind[j];
        A.wline[j] = at->kind[j] == 0 ? (float)at->wlam[j] : 0.f;
        nline += at->kind[j] == 0;
        for (int i = 0; i < 2; ++i) {
            A.sig_bf[i][j] = l <= edge[i] ? (float)(sig_edge[i] * std::pow(l / edge[i], 3)) : 0.f;
            A.dchi[i][j] = (float)((E[2] - E[i]) - hc / l);
        }
        A.dE_line[j] = (float)(hc / lam0 - hc / l);
        A.b_l5[j] = (float)(2.0 * hc * kC / std::pow(l, 5));
        A.hc_lk[j] = (float)(hc / (l * kK));
        A.rate_f[j] = (float)(4.0 * M_PI * at->wlam[j] * l / hc);
    }
    if (nline == 0) return fail(RT_EINVAL, "atom has no line node");
    A.nline = nline;
    // upload only when the atom changed on this device (the copy goes through the legacy default
    // stream and is synchronous)
    static AtomDev last[MAX_DEVICES];
    static bool have_last[MAX_DEVICES] = {};
    if (!have_last[dev] || std::memcmp(&last[dev], &A, sizeof(A)) != 0) {
        RT_CUDA(cudaMemcpyToSymbol(c_atom, &A, sizeof(A)));
        last[dev] = A;
        have_last[dev] = true;
    }
    return RT_OK;
}

static rt_status check_atmos(rt_grid *g, const rt_atmos *atm, const float *pops)
{
    if (!g || !atm || !atm->T || !atm->rho || !atm->ne || !atm->nH || !pops)
        return fail(RT_EINVAL, "null argument");
    return RT_OK;
}

}  // namespace rt

using namespace rt;

extern "C" {

rt_status rt_source_terms_lte(int64_t npt, const float *T, const float *rho, double kappa0,
                              double lam, float *alpha, float *S, void *stream)
{
    return guarded([&]() -> rt_status {
        if (npt < 1 || !T || !rho || !alpha || !S || !(lam > 0)) return fail(RT_EINVAL, "bad argument");
        const double hc = kH * kC;
        note_launch();
        lte_source_kernel<<<(unsigned)((npt + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
            npt, T, rho, (float)kappa0, (float)(2.0 * hc * kC / std::pow(lam, 5)),
            (float)(hc / (lam * kK)), alpha, S);
        RT_CUDA(cudaGetLastError());
        return RT_OK;
    });
}

rt_status rt_source_terms_lte_adjoint(int64_t npt, const float *T, const float *rho,
                                      double kappa0, double lam, const float *g_alpha,
                                      const float *g_S, float *g_T, void *stream)
{
    return guarded([&]() -> rt_status {
        if (npt < 1 || !T || !rho || !g_alpha || !g_S || !g_T) return fail(RT_EINVAL, "bad argument");
        const double hc = kH * kC;
        note_launch();
        lte_source_adjoint_kernel<<<(unsigned)((npt + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
            npt, T, rho, (float)kappa0, (float)(2.0 * hc * kC / std::pow(lam, 5)),
            (float)(hc / (lam * kK)), g_alpha, g_S, g_T);
        RT_CUDA(cudaGetLastError());
        return RT_OK;
    });
}

rt_status rt_source_terms(rt_grid_t g, const rt_atom *atom, const rt_atmos *atm,
                          const float *pops, float *alpha, float *S, void *stream)
{
    return guarded([&]() -> rt_status {
        RT_TRY(check_atmos(g, atm, pops));
        if (!alpha || !S) return fail(RT_EINVAL, "null output");
        RT_TRY(load_atom(atom));
        const int64_t n = g->npt;
        note_launch();
        source_terms_kernel<<<(unsigned)((n + 127) / 128), 128, 0, (cudaStream_t)stream>>>(
            n, atm->T, atm->rho, atm->ne, pops, alpha, S, g->d_err);
        RT_CUDA(cudaGetLastError());
        return RT_OK;
    });
}

rt_status rt_source_terms_adjoint(rt_grid_t g, const rt_atom *atom, const rt_atmos *atm,
                                  const float *pops, const float *g_alpha, const float *g_S,
                                  float *g_T, void *stream)
{
    return guarded([&]() -> rt_status {
        RT_TRY(check_atmos(g, atm, pops));
        if (!g_alpha || !g_S || !g_T) return fail(RT_EINVAL, "null argument");
        RT_TRY(load_atom(atom));
        const int64_t n = g->npt;
        note_launch();
        source_terms_adjoint_kernel<<<(unsigned)((n + 127) / 128), 128, 0, (cudaStream_t)stream>>>(
            n, atm->T, atm->rho, atm->ne, pops, g_alpha, g_S, g_T);
        RT_CUDA(cudaGetLastError());
        return RT_OK;
    });
}

rt_status rt_lte_populations(rt_grid_t g, const rt_atom *atom, const rt_atmos *atm, float *pops,
                             void *stream)
{
    return guarded([&]() -> rt_status {
        RT_TRY(check_atmos(g, atm, pops));
        RT_TRY(load_atom(atom));
        const int64_t n = g->npt;
        note_launch();
        lte_pops_kernel<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
            n, atm->T, atm->ne, atm->nH, pops);
        RT_CUDA(cudaGetLastError());
        return RT_OK;
    });
}

rt_status rt_statistical_equilibrium(rt_grid_t g, const rt_atom *atom, const rt_atmos *atm,
                                     const float *J, float *pops, float *dmax_dev, void *stream)
{
    return guarded([&]() -> rt_status {
        RT_TRY(check_atmos(g, atm, pops));
        if (!J) return fail(RT_EINVAL, "null J");
        RT_TRY(load_atom(atom));
        const int64_t n = g->npt;
        note_launch();
        se_kernel<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
            n, atm->T, atm->ne, atm->nH, J, pops, dmax_dev, g->d_err);
        RT_CUDA(cudaGetLastError());
        return RT_OK;
    });
}

rt_status rt_statistical_equilibrium_ali(rt_grid_t g, const rt_atom *atom, const rt_atmos *atm,
                                         const float *J, const float *Lstar, const float *S_old,
                                         float *pops, float *dmax_dev, int newton, void *stream)
{
    return guarded([&]() -> rt_status {
        RT_TRY(check_atmos(g, atm, pops));
        if (!J || !Lstar || !S_old) return fail(RT_EINVAL, "null J, Lstar or S_old");
        if (newton < 0 || newton > 16) return fail(RT_EINVAL, "newton must be in 0..16");
        if (atom->nlam > 64) return fail(RT_EINVAL, "the accelerated update takes at most 64 wavelengths");
        RT_TRY(load_atom(atom));
        const int64_t n = g->npt;
        note_launch();
        se_ali_kernel<<<ali_blocks(n), ALI_WARPS * 32, 0, (cudaStream_t)stream>>>(
            n, atm->T, atm->rho, atm->ne, atm->nH, J, Lstar, S_old, pops, dmax_dev, g->d_err, newton);
        RT_CUDA(cudaGetLastError());
        return RT_OK;
    });
}

}  // extern "C"

// The Lambda iteration loop; newton < 0: plain, else accelerated with that many Newton steps
// and Lambda* either from the starting opacities, held fixed (fixed_lstar), or recomputed from
// every iteration's opacities.  ng_period > 0: Ng extrapolation from the last four iterates after
// every ng_period-th iteration (from the fourth on), kept only if every population stays positive.
static rt_status iterate(rt_grid_t g, const rt_atom *atom, const rt_atmos *atm, float *pops,
                         int max_iter, double tol, int *iters_out, float *history, int use_graph,
                         int newton, int fixed_lstar, int ng_period, void *stream)
{
    RT_TRY(check_atmos(g, atm, pops));
    if (max_iter < 1) return fail(RT_EINVAL, "max_iter must be >= 1");
    RT_TRY(load_atom(atom));
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t n = g->npt;
    const int nlam = atom->nlam;
    // scratch 2: alpha, S, J [nlam][n] (+ Lambda* when accelerated) + dmax
    const bool ali = newton >= 0;
    const size_t nf = (ali ? 4 : 3) * (size_t)nlam * n;
    const size_t nh = ng_period > 0 ? 5 * 3 * (size_t)n : 0;   // Ng: 4 iterates + the result
    void *p;
    RT_TRY(scratch_get(g, 2, (nf + nh) * sizeof(float) + 256, &p));
    float *alpha = (float *)p, *S = alpha + (size_t)nlam * n, *J = S + (size_t)nlam * n;
    float *L = ali ? J + (size_t)nlam * n : nullptr;
    float *hist = (float *)p + nf;                 // [5][3 n]
    float *dmax = (float *)p + nf + nh;
    void *ngs = (void *)((((uintptr_t)dmax + 16) + 63) & ~(uintptr_t)63);   // 64 B, in the pad
    if (ali) RT_TRY(lambda_star_prepare(g));
    dmax = (float *)(((uintptr_t)dmax + 15) & ~(uintptr_t)15);
    float *h_dmax = nullptr;
    RT_CUDA(cudaMallocHost(&h_dmax, sizeof(float)));
    struct Guard {
        float *h;
        cudaGraphExec_t ex = nullptr;
        cudaGraph_t gr = nullptr;
        ~Guard()
        {
            if (ex) cudaGraphExecDestroy(ex);
            if (gr) cudaGraphDestroy(gr);
            cudaFreeHost(h);
        }
    } guard{h_dmax};
    auto enqueue = [&]() -> rt_status {
        RT_CUDA(cudaMemsetAsync(dmax, 0, sizeof(float), st));
        note_launch();
        source_terms_kernel<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(
            n, atm->T, atm->rho, atm->ne, pops, alpha, S, g->d_err);
        RT_TRY(rt_formal_solution(g, nlam, alpha, S, RT_BC_THERMAL, nullptr, J, nullptr, st));
        note_launch();
        if (ali) {
            if (!fixed_lstar) RT_TRY(lambda_star(g, nlam, alpha, RT_BC_THERMAL, L, st));
            se_ali_kernel<<<ali_blocks(n), ALI_WARPS * 32, 0, st>>>(
                n, atm->T, atm->rho, atm->ne, atm->nH, J, L, S, pops, dmax, g->d_err, newton);
        } else {
            se_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, atm->T, atm->ne, atm->nH,
                                                                    J, pops, dmax, g->d_err);
        }
        RT_CUDA(cudaMemcpyAsync(h_dmax, dmax, sizeof(float), cudaMemcpyDeviceToHost, st));
        return RT_OK;
    };
    if (ali && fixed_lstar) {
        // Lambda* of the starting populations' opacities, held fixed: the fixed point of the
        // iteration does not depend on Lambda*, only its rate of convergence does
        note_launch();
        source_terms_kernel<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(
            n, atm->T, atm->rho, atm->ne, pops, alpha, S, g->d_err);
        RT_TRY(lambda_star(g, nlam, alpha, RT_BC_THERMAL, L, st));
    }
    cudaStream_t cs = nullptr;       // capture stream (the legacy default stream cannot be captured)
    cudaEvent_t ev = nullptr;
    struct StreamGuard {
        cudaStream_t *s;
        cudaEvent_t *e;
        ~StreamGuard()
        {
            if (*e) cudaEventDestroy(*e);
            if (*s) cudaStreamDestroy(*s);
        }
    } sguard{&cs, &ev};
    if (use_graph) {
        // the formal solution allocates its scratch on first use: do that before capturing
        void *q;
        const size_t ndh = std::max(g->dir_up.size(), g->dir_dn.size());
        if (g->kind == RT_GRID_REGULAR && g->sc_face) {
            RT_TRY(face_prepare(g, nlam));
        } else if (g->kind == RT_GRID_REGULAR) {
            RT_TRY(scratch_get(g, 0, 2 * (size_t)nlam * ndh * g->nx * g->ny * sizeof(float), &q));
            RT_TRY(scratch_get(g, 3, regular_wave_scratch(g, nlam), &q));
        }
        else {
            RT_TRY(scratch_get(g, 0, 4 * (size_t)n * nlam * sizeof(float), &q));
            RT_TRY(voronoi_prepare(g, nlam));
        }
        RT_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        RT_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        RT_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
        cudaStream_t user = st;
        st = cs;
        rt_status s = enqueue();
        st = user;
        cudaError_t e = cudaStreamEndCapture(cs, &guard.gr);
        if (s != RT_OK) {
            cudaGetLastError();
            return s;
        }
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
        RT_CUDA(cudaGraphInstantiate(&guard.ex, guard.gr, 0));
    }
    int it = 0;
    rt_status result = RT_ENOCONV;
    for (it = 1; it <= max_iter; ++it) {
        if (use_graph) RT_CUDA(cudaGraphLaunch(guard.ex, st));
        else RT_TRY(enqueue());
        RT_CUDA(cudaStreamSynchronize(st));
        RT_TRY(check_dev_error(g, st));
        const float d = *h_dmax;
        if (history) history[it - 1] = d;
        if (d < tol) {
            result = RT_OK;
            break;
        }
        if (ng_period > 0) {
            const size_t m = 3 * (size_t)n;
            float *H[4];
            for (int q = 0; q < 4; ++q) H[q] = hist + (size_t)((it - q) & 3) * m;
            RT_CUDA(cudaMemcpyAsync(H[0], pops, m * sizeof(float), cudaMemcpyDeviceToDevice, st));
            if (it >= 4 && it % ng_period == 0) {
                int ok = 0;
                float *out = hist + 4 * m;
                RT_TRY(ng_extrapolate(H[0], H[1], H[2], H[3], (int64_t)m, out, ngs, st, &ok));
                if (ok) {
                    RT_CUDA(cudaMemcpyAsync(pops, out, m * sizeof(float), cudaMemcpyDeviceToDevice,
                                            st));
                    RT_CUDA(cudaMemcpyAsync(H[0], out, m * sizeof(float),
                                            cudaMemcpyDeviceToDevice, st));
                }
            }
        }
    }
    if (iters_out) *iters_out = std::min(it, max_iter);
    if (result == RT_ENOCONV) fail(RT_ENOCONV, "max_iter reached before the tolerance");
    return result;
}

extern "C" {

rt_status rt_lambda_iterate(rt_grid_t g, const rt_atom *atom, const rt_atmos *atm, float *pops,
                            int max_iter, double tol, int *iters_out, float *history,
                            int use_graph, void *stream)
{
    return guarded([&]() -> rt_status {
        return iterate(g, atom, atm, pops, max_iter, tol, iters_out, history, use_graph, -1, 0, 0,
                       stream);
    });
}

rt_status rt_lambda_iterate_ali(rt_grid_t g, const rt_atom *atom, const rt_atmos *atm,
                                float *pops, int max_iter, double tol, int *iters_out,
                                float *history, int use_graph, int newton, int fixed_lstar,
                                void *stream)
{
    return guarded([&]() -> rt_status {
        if (newton < 0 || newton > 16) return fail(RT_EINVAL, "newton must be in 0..16");
        if (atom && atom->nlam > 64)
            return fail(RT_EINVAL, "the accelerated update takes at most 64 wavelengths");
        return iterate(g, atom, atm, pops, max_iter, tol, iters_out, history, use_graph, newton,
                       fixed_lstar, 0, stream);
    });
}

rt_status rt_lambda_iterate_ex(rt_grid_t g, const rt_atom *atom, const rt_atmos *atm,
                               float *pops, int max_iter, double tol, int *iters_out,
                               float *history, int use_graph, int newton, int fixed_lstar,
                               int ng_period, void *stream)
{
    return guarded([&]() -> rt_status {
        if (newton < -1 || newton > 16) return fail(RT_EINVAL, "newton must be in -1..16");
        if (ng_period < 0) return fail(RT_EINVAL, "ng_period must be >= 0");
        if (newton >= 0 && atom && atom->nlam > 64)
            return fail(RT_EINVAL, "the accelerated update takes at most 64 wavelengths");
        return iterate(g, atom, atm, pops, max_iter, tol, iters_out, history, use_graph, newton,
                       fixed_lstar, ng_period, stream);
    });
}

// The Lambda iteration of every atmosphere of a batch at once: per atmosphere the source terms,
// then one batched formal solution of all of them, then per atmosphere the statistical
// equilibrium, all writing one shared convergence scalar (the largest change over every
// atmosphere).  One model atom serves the whole batch (its constants live in constant memory).
rt_status rt_batch_lambda_iterate(rt_batch_t b, const rt_atom *atom, const rt_atmos *atms,
                                  float *const *pops, int max_iter, double tol, int *iters_out,
                                  float *history, int use_graph, void *stream)
{
    return guarded([&]() -> rt_status {
        if (!b || !atms || !pops) return fail(RT_EINVAL, "null argument");
        if (max_iter < 1) return fail(RT_EINVAL, "max_iter must be >= 1");
        const int ng = batch_ngrids(b);
        const int nlam = batch_nlam(b);
        if (!atom || atom->nlam != nlam)
            return fail(RT_EINVAL, "the atom's wavelength count must equal the batch's");
        for (int i = 0; i < ng; ++i) RT_TRY(check_atmos(batch_grid(b, i), &atms[i], pops[i]));
        RT_TRY(load_atom(atom));
        cudaStream_t st = (cudaStream_t)stream;
        // per atmosphere: alpha, S, J [nlam][n] in the grid's iteration scratch; the convergence
        // scalar in the first grid's
        std::vector<float *> A(ng), S(ng), J(ng);
        float *dmax = nullptr;
        for (int i = 0; i < ng; ++i) {
            rt_grid *g = batch_grid(b, i);
            const size_t m = (size_t)nlam * g->npt;
            void *p;
            RT_TRY(scratch_get(g, 2, 3 * m * sizeof(float) + 256, &p));
            A[i] = (float *)p;
            S[i] = A[i] + m;
            J[i] = S[i] + m;
            if (i == 0) dmax = (float *)((((uintptr_t)(J[i] + m)) + 15) & ~(uintptr_t)15);
        }
        float *h_dmax = nullptr;
        RT_CUDA(cudaMallocHost(&h_dmax, sizeof(float)));
        struct Guard {
            float *h;
            cudaGraphExec_t ex = nullptr;
            cudaGraph_t gr = nullptr;
            cudaStream_t cs = nullptr;
            ~Guard()
            {
                if (ex) cudaGraphExecDestroy(ex);
                if (gr) cudaGraphDestroy(gr);
                if (cs) cudaStreamDestroy(cs);
                cudaFreeHost(h);
            }
        } guard{h_dmax};
        auto enqueue = [&](cudaStream_t s) -> rt_status {
            RT_CUDA(cudaMemsetAsync(dmax, 0, sizeof(float), s));
            for (int i = 0; i < ng; ++i) {
                rt_grid *g = batch_grid(b, i);
                const int64_t n = g->npt;
                note_launch();
                source_terms_kernel<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(
                    n, atms[i].T, atms[i].rho, atms[i].ne, pops[i], A[i], S[i], g->d_err);
            }
            RT_TRY(rt_batch_formal_solution(b, A.data(), S.data(), RT_BC_THERMAL, J.data(), s));
            for (int i = 0; i < ng; ++i) {
                rt_grid *g = batch_grid(b, i);
                const int64_t n = g->npt;
                note_launch();
                se_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(
                    n, atms[i].T, atms[i].ne, atms[i].nH, J[i], pops[i], dmax, g->d_err);
            }
            RT_CUDA(cudaMemcpyAsync(h_dmax, dmax, sizeof(float), cudaMemcpyDeviceToHost, s));
            return RT_OK;
        };
        if (use_graph) {
            RT_CUDA(cudaStreamCreateWithFlags(&guard.cs, cudaStreamNonBlocking));
            RT_CUDA(cudaStreamBeginCapture(guard.cs, cudaStreamCaptureModeThreadLocal));
            rt_status s = enqueue(guard.cs);
            cudaError_t e = cudaStreamEndCapture(guard.cs, &guard.gr);
            if (s != RT_OK) {
                cudaGetLastError();
                return s;
            }
            if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
            RT_CUDA(cudaGraphInstantiate(&guard.ex, guard.gr, 0));
        }
        int it = 0;
        rt_status result = RT_ENOCONV;
        for (it = 1; it <= max_iter; ++it) {
            if (use_graph) RT_CUDA(cudaGraphLaunch(guard.ex, st));
            else RT_TRY(enqueue(st));
            RT_CUDA(cudaStreamSynchronize(st));
            for (int i = 0; i < ng; ++i) RT_TRY(check_dev_error(batch_grid(b, i), st));
            RT_TRY(batch_check_error(b, st));
            const float d = *h_dmax;
            if (history) history[it - 1] = d;
            if (d < tol) {
                result = RT_OK;
                break;
            }
        }
        if (iters_out) *iters_out = std::min(it, max_iter);
        if (result == RT_ENOCONV) fail(RT_ENOCONV, "max_iter reached before the tolerance");
        return result;
    });
}

// Host evaluation of the device Voigt function for testing: H(a, v) in FP32 arithmetic is not
// reproduced here; this returns G(v) = 2 v F(v) - 1 from the double-precision Dawson series that
// seeds the device tables.
double rt_debug_G_host(double v) { return G_host(v); }

}  // extern "C"
