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

// rates -> statistical equilibrium -> new populations and max |dn/n|
__global__ void __launch_bounds__(256) se_kernel(int64_t npt, const float *T, const float *ne,
                                                 const float *nH, const float *J, float *pops,
                                                 float *dmax, unsigned *err)
{
    __shared__ float tab[G_PIECES * G_DEG];
    load_gtab(tab);
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float change = 0.f;
    if (p < npt) {
        const AtomDev &A = c_atom;
        const float t = T[p], e = ne[p], kT = t * 1.380649e-23f;
        float ph[MAX_LAM];
        line_profiles<float>(A.dld_coef * sqrtf(t), tab, ph);
        const float tm32 = 1.f / (t * sqrtf(t));
        float P[3][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
        for (int j = 0; j < A.nlam; ++j) {
            const float Jj = J[(size_t)j * npt + p];
            float sig, g;
            int lo, hi;
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
            const float fs = A.rate_f[j] * sig;
            P[lo][hi] += fs * Jj;
            P[hi][lo] += fs * g * (A.b_l5[j] + Jj);
        }
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
        const float f = nH[p] / (t1 + t2 + t3);
        const float nn[3] = {t1 * f, t2 * f, t3 * f};
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
    // block max, then one atomic per block
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
static rt_status load_atom(const rt_atom *at)
{
    static std::vector<float> gpoly;
    static bool gp_done = false;
    if (!at || !at->lam || !at->wlam || !at->kind) return fail(RT_EINVAL, "incomplete atom");
    if (at->nlam < 1 || at->nlam > MAX_LAM) return fail(RT_EINVAL, "atom nlam must be 1..128");
    if (!gp_done) {
        build_gpoly(gpoly);
        gp_done = true;
        RT_CUDA(cudaMemcpyToSymbol(c_gpoly, gpoly.data(), gpoly.size() * sizeof(float)));
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
    // upload only when the atom changed (the copy goes through the legacy default stream)
    static AtomDev last;
    static bool have_last = false;
    if (!have_last || std::memcmp(&last, &A, sizeof(A)) != 0) {
        RT_CUDA(cudaMemcpyToSymbol(c_atom, &A, sizeof(A)));
        last = A;
        have_last = true;
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
    if (npt < 1 || !T || !rho || !alpha || !S || !(lam > 0)) return fail(RT_EINVAL, "bad argument");
    const double hc = kH * kC;
    note_launch();
    lte_source_kernel<<<(unsigned)((npt + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
        npt, T, rho, (float)kappa0, (float)(2.0 * hc * kC / std::pow(lam, 5)),
        (float)(hc / (lam * kK)), alpha, S);
    RT_CUDA(cudaGetLastError());
    return RT_OK;
}

rt_status rt_source_terms_lte_adjoint(int64_t npt, const float *T, const float *rho,
                                      double kappa0, double lam, const float *g_alpha,
                                      const float *g_S, float *g_T, void *stream)
{
    if (npt < 1 || !T || !rho || !g_alpha || !g_S || !g_T) return fail(RT_EINVAL, "bad argument");
    const double hc = kH * kC;
    note_launch();
    lte_source_adjoint_kernel<<<(unsigned)((npt + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
        npt, T, rho, (float)kappa0, (float)(2.0 * hc * kC / std::pow(lam, 5)),
        (float)(hc / (lam * kK)), g_alpha, g_S, g_T);
    RT_CUDA(cudaGetLastError());
    return RT_OK;
}

rt_status rt_source_terms(rt_grid_t g, const rt_atom *atom, const rt_atmos *atm,
                          const float *pops, float *alpha, float *S, void *stream)
{
    RT_TRY(check_atmos(g, atm, pops));
    if (!alpha || !S) return fail(RT_EINVAL, "null output");
    RT_TRY(load_atom(atom));
    const int64_t n = g->npt;
    note_launch();
    source_terms_kernel<<<(unsigned)((n + 127) / 128), 128, 0, (cudaStream_t)stream>>>(
        n, atm->T, atm->rho, atm->ne, pops, alpha, S, g->d_err);
    RT_CUDA(cudaGetLastError());
    return RT_OK;
}

rt_status rt_source_terms_adjoint(rt_grid_t g, const rt_atom *atom, const rt_atmos *atm,
                                  const float *pops, const float *g_alpha, const float *g_S,
                                  float *g_T, void *stream)
{
    RT_TRY(check_atmos(g, atm, pops));
    if (!g_alpha || !g_S || !g_T) return fail(RT_EINVAL, "null argument");
    RT_TRY(load_atom(atom));
    const int64_t n = g->npt;
    note_launch();
    source_terms_adjoint_kernel<<<(unsigned)((n + 127) / 128), 128, 0, (cudaStream_t)stream>>>(
        n, atm->T, atm->rho, atm->ne, pops, g_alpha, g_S, g_T);
    RT_CUDA(cudaGetLastError());
    return RT_OK;
}

rt_status rt_lte_populations(rt_grid_t g, const rt_atom *atom, const rt_atmos *atm, float *pops,
                             void *stream)
{
    RT_TRY(check_atmos(g, atm, pops));
    RT_TRY(load_atom(atom));
    const int64_t n = g->npt;
    note_launch();
    lte_pops_kernel<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
        n, atm->T, atm->ne, atm->nH, pops);
    RT_CUDA(cudaGetLastError());
    return RT_OK;
}

rt_status rt_statistical_equilibrium(rt_grid_t g, const rt_atom *atom, const rt_atmos *atm,
                                     const float *J, float *pops, float *dmax_dev, void *stream)
{
    RT_TRY(check_atmos(g, atm, pops));
    if (!J) return fail(RT_EINVAL, "null J");
    RT_TRY(load_atom(atom));
    const int64_t n = g->npt;
    note_launch();
    se_kernel<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
        n, atm->T, atm->ne, atm->nH, J, pops, dmax_dev, g->d_err);
    RT_CUDA(cudaGetLastError());
    return RT_OK;
}

rt_status rt_lambda_iterate(rt_grid_t g, const rt_atom *atom, const rt_atmos *atm, float *pops,
                            int max_iter, double tol, int *iters_out, float *history,
                            int use_graph, void *stream)
{
    RT_TRY(check_atmos(g, atm, pops));
    if (max_iter < 1) return fail(RT_EINVAL, "max_iter must be >= 1");
    RT_TRY(load_atom(atom));
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t n = g->npt;
    const int nlam = atom->nlam;
    // scratch 2: alpha, S, J [nlam][n] + dmax
    void *p;
    RT_TRY(scratch_get(g, 2, 3 * (size_t)nlam * n * sizeof(float) + 256, &p));
    float *alpha = (float *)p, *S = alpha + (size_t)nlam * n, *J = S + (size_t)nlam * n;
    float *dmax = J + (size_t)nlam * n;
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
        se_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, atm->T, atm->ne, atm->nH, J,
                                                                pops, dmax, g->d_err);
        RT_CUDA(cudaMemcpyAsync(h_dmax, dmax, sizeof(float), cudaMemcpyDeviceToHost, st));
        return RT_OK;
    };
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
        if (g->kind == RT_GRID_REGULAR) {
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
    }
    if (iters_out) *iters_out = std::min(it, max_iter);
    if (result == RT_ENOCONV) fail(RT_ENOCONV, "max_iter reached before the tolerance");
    return result;
}

// Host evaluation of the device Voigt function for testing: H(a, v) in FP32 arithmetic is not
// reproduced here; this returns G(v) = 2 v F(v) - 1 from the double-precision Dawson series that
// seeds the device tables.
double rt_debug_G_host(double v) { return G_host(v); }

}  // extern "C"
