// Face-hitting short characteristics on the regular grid (Kunasz & Auer 1988, the scheme Sect. 2.6
// names for the regular-grid solver), selected per grid by rt_grid_set_scheme(RT_SC_FACE).
//
// The ray through a point of plane k is followed upwind to the first face of the cell it enters.
// If that is the plane face (dz/|mu_z| <= dx/|mu_x|, dy/|mu_y|), the upwind point lies within one
// cell of the point's column in the previous plane of the sweep and I, S, alpha are bilinear there.
// Otherwise it is a vertical face normal to the axis a (x when dx/|mu_x| < dy/|mu_y|, else y), and
// I, S, alpha are bilinear on that face between the grid lines b and b - s_b and the planes k and
// k -/+ 1: two of the four corners lie in plane k itself, one line upwind along a.  Segment length
// t, delta tau = (alpha_up + alpha) t / 2, S linear across the interval (Eq. 2).  Periodic in x, y.
//
// Work decomposition.  One block per (wavelength, group of up to 12 directions of one hemisphere),
// one warp per direction.  A warp keeps one plane of intensities per (wavelength, direction) in
// global memory, stored line by line along a ([a][b], b contiguous), and sweeps each plane line by
// line in upwind order along a, the lanes across b: line a needs only line a - s_a of planes k and
// k -/+ 1 (and, on the plane face, line a of plane k -/+ 1), staged in a two-line ring in shared
// memory, while the next line's loads are in flight.  Directions whose lines run along x read S and
// alpha from copies transposed to [nlam][nz][x][y] once per call, so that every line load is
// contiguous.  Either every plane of the sweep is kept (J formed afterwards, below), or the plane
// buffer is updated in place: line a of the previous plane is no longer needed once line a of
// this plane is computed (the ring holds it for the next line).
//
// Vertical faces couple a plane's lines around the periodic box.  Each line's dependence on the
// line before it has total weight (1 - f_z) e^-dtau <= 1 - f_z, f_z = t |mu_z| / dz < 1, so the walk
// starts W lines before the first line it stores, from the previous plane's intensities, with
// (1 - f_z)^W <= 1e-9: the stored lines then carry the periodic solution to far below FP32
// rounding.  The plane face has no such coupling (W = 0).
//
// J = sum_d w_d I_d.  Where the device's memory allows, the sweep keeps every plane of every
// (wavelength, direction) and one kernel afterwards sums them per point in the tables' direction
// order (directions with a = x hold their planes transposed, so their tiles pass through shared
// memory); the sweep's warps then never wait for one another.  Otherwise, after each plane, the
// block sums w_d I_d over its directions into its J partial, and a second kernel adds the
// partials of the other groups to J in a fixed order.
#include <cmath>
#include <cstdlib>
#include <vector>

#include "device_common.cuh"
#include "rt_impl.h"

namespace rt {

constexpr int FACE_MAXW = 12;        // directions (warps) per block
constexpr int FACE_MAXNB = 256;      // largest nx, ny
constexpr double FACE_EPS = 1e-9;    // closure truncation of the periodic plane system

struct FaceDir {
    int dir;          // index in the grid's direction list
    int a_is_x;       // 1: lines run along x (face x = x_i - s_a dx), 0: along y
    int sa, sb;       // upwind steps +-1 along a and b
    int up;           // mu_z > 0
    float w;          // quadrature weight
};

// per (direction, plane step): X_up = (1 - fb) (wA X_u[a][b] + wU X_u[a-sa][b] + wK X_k[a-sa][b])
//                                    + fb (same at b - sb), X_u the upwind plane, X_k this plane
struct FaceStep {
    float t, wA, wU, wK, fb;
    int warm;         // lines walked before the first stored one (vertical face), else 0
};

struct FaceTables {
    FaceDir *d_dirs = nullptr;     // [ndir], grouped
    int nxd = 0;                   // directions whose lines run along x
    FaceStep *d_steps = nullptr;   // [ndir][nz] by grid direction index, step s = 1 .. nz-1
    int *d_first = nullptr;        // [ngroups + 1]
    int ngroups = 0, wpb = 0, nbpad = 0;
    int has_x = 0;                 // some direction's lines run along x
};

void face_release(FaceTables *t)
{
    if (!t) return;
    if (t->d_dirs) cudaFree(t->d_dirs);
    if (t->d_steps) cudaFree(t->d_steps);
    if (t->d_first) cudaFree(t->d_first);
    delete t;
}

struct FaceArgs {
    const float *alpha, *S, *I_bc;
    const float *AT, *ST;          // [nlam][nz][nx][ny] transposed copies (lines along x)
    float *I_dir, *J, *Jp, *buf;
    const FaceDir *dirs;
    const FaceStep *steps;
    const int *first;
    unsigned *err;
    int nx, ny, nz, nlam, ndir, bc, nbpad;
    int defer;                     // 1: buf holds every plane [nlam][ndir][nz][np]; J afterwards
};

enum { R_IK, R_SK, R_AK, R_IU, R_SU, R_AU };

template <int MAXM>
__global__ void __launch_bounds__(FACE_MAXW * 32, 1) face_sweep_kernel(FaceArgs a)
{
    extern __shared__ float sm[];
    __shared__ FaceDir sdir[FACE_MAXW];
    // J of a plane: per direction of the group its plane buffer, weight and slot among the
    // directions whose planes are held transposed (-1: held as [y][x])
    __shared__ const float *sbq[FACE_MAXW];
    __shared__ float swq[FACE_MAXW];
    __shared__ int sxq[FACE_MAXW], sxinv[FACE_MAXW];
    const int lam = blockIdx.x, grp = blockIdx.y;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    const int d0 = a.first[grp], nd = a.first[grp + 1] - d0;
    if (threadIdx.x < nd) sdir[threadIdx.x] = a.dirs[d0 + threadIdx.x];
    __syncthreads();
    if (threadIdx.x == 0) {
        int xi = 0;
        for (int q = 0; q < nd; ++q) {
            sbq[q] = a.buf + ((size_t)lam * a.ndir + sdir[q].dir) * (size_t)a.nx * a.ny;
            swq[q] = sdir[q].w;
            sxq[q] = -1;
            if (sdir[q].a_is_x) {
                sxinv[xi] = q;
                sxq[q] = xi++;
            }
        }
    }
    __syncthreads();
    const int nx = a.nx, ny = a.ny, nz = a.nz, np = nx * ny;
    const size_t npt = (size_t)np * nz;
    const bool active = warp < nd;
    const FaceDir D = sdir[active ? warp : 0];
    const int up = sdir[0].up;
    const int na = D.a_is_x ? nx : ny, nb = D.a_is_x ? ny : nx;
    // S and alpha with this direction's lines contiguous: [nz][na][nb]
    const float *Sl = (D.a_is_x ? a.ST : a.S) + (size_t)lam * npt;
    const float *Al = (D.a_is_x ? a.AT : a.alpha) + (size_t)lam * npt;
    // this direction's plane buffer (line-major): one plane updated in place, or, when J is
    // formed after the sweep, every plane (written at plane k, read at the upwind plane ku)
    float *const bufd = a.buf + ((size_t)lam * a.ndir + D.dir) * np * (a.defer ? (size_t)nz : 1);
    float *buf = bufd, *bufu = bufd;
    float *ring = sm + (size_t)warp * 12 * a.nbpad;
    float *tile = sm + (size_t)wpb * 12 * a.nbpad;
    float *Jout = (grp == 0 ? a.J : a.Jp + (size_t)(grp - 1) * a.nlam * npt) + (size_t)lam * npt;
    float *Idir = a.I_dir ? a.I_dir + ((size_t)D.dir * a.nlam + lam) * npt : nullptr;
    const int nbpad = a.nbpad;
#define RING(arr, slot, b) ring[((arr) * 2 + (slot)) * nbpad + (b)]

    // field index of position b on line al of plane k, and its index in the line-major copies
    auto fidx = [&](int k, int al, int b) -> size_t {
        return (size_t)k * np + (D.a_is_x ? (size_t)b * nx + al : (size_t)al * nx + b);
    };
    auto lidx = [&](int k, int al, int b) -> size_t {
        return (size_t)k * np + (size_t)al * nb + b;
    };

    // J partial of plane k: sum over the group's directions in group order
    // transposed directions of the group, and the 32 x 32 tiles the shared tile buffer (room for
    // wpb transposed tiles) holds at once: the tiles of one batch share each pair of barriers
    int nxd = 0;
    for (int q = 0; q < nd; ++q) nxd += sxq[q] >= 0;
    const int tpb = nxd ? max(1, wpb / nxd) : 4;
    const int tcx = (nx + 31) >> 5, ntile = tcx * ((ny + 31) >> 5);
    auto j_plane = [&](int k) {
        float *Jk = Jout + (size_t)k * np;
        for (int t0 = 0; t0 < ntile; t0 += tpb) {
            const int nt = min(tpb, ntile - t0);
            for (int e = threadIdx.x; e < nt * nxd * 1024; e += blockDim.x) {
                const int tb = e / (nxd * 1024), xi = (e / 1024) % nxd, r = (e >> 5) & 31, c = e & 31;
                const int t = t0 + tb, i = (t % tcx) * 32 + r, j = (t / tcx) * 32 + c;
                tile[((tb * nxd + xi) * 32 + r) * 33 + c] =
                    (i < nx && j < ny) ? sbq[sxinv[xi]][i * ny + j] : 0.f;
            }
            __syncthreads();
            for (int e = threadIdx.x; e < nt * 1024; e += blockDim.x) {
                const int tb = e >> 10, r = (e >> 5) & 31, c = e & 31, t = t0 + tb;
                const int i = (t % tcx) * 32 + c, j = (t / tcx) * 32 + r;
                if (i >= nx || j >= ny) continue;
                const int f = j * nx + i;
                float acc = 0.f;
                for (int q = 0; q < nd; ++q) {   // the group's order
                    const int xi = sxq[q];
                    const float v = xi >= 0 ? tile[((tb * nxd + xi) * 32 + c) * 33 + r] : sbq[q][f];
                    acc = fmaf(swq[q], v, acc);
                }
                if (!isfinite(acc)) flag_error(a.err, ERR_NAN);
                Jk[f] = acc;
            }
            __syncthreads();
        }
    };

    // the wall plane the rays enter through
    const int k0 = up ? 0 : nz - 1;
    if (active) {
        for (int m = lane; m < np; m += 32) {
            const int al = m / nb, b = m - al * nb;
            const size_t f = fidx(k0, al, b);
            float v = 0.f;
            if (a.bc == RT_BC_ARRAY)
                v = __ldg(a.I_bc + ((size_t)D.dir * a.nlam + lam) * np + (f - (size_t)k0 * np));
            else if (a.bc == RT_BC_THERMAL && up)
                v = __ldg(Sl + lidx(k0, al, b));
            buf[m + (a.defer ? (size_t)k0 * np : 0)] = v;
            if (Idir) Idir[f] = v;
        }
    }
    if (!a.defer) {
        __syncthreads();
        j_plane(k0);
    }

    const int M = (nb + 31) >> 5;
    for (int s = 1; s < nz; ++s) {
        const int k = up ? s : nz - 1 - s, ku = up ? k - 1 : k + 1;
        if (a.defer) {
            buf = bufd + (size_t)k * np;
            bufu = bufd + (size_t)ku * np;
        }
        if (active) {
            const FaceStep st = a.steps[(size_t)D.dir * nz + s];
            // line of the m-th step of the walk (m < 0: the lines before the first stored one)
            auto line_of = [&](int m) {
                int r = m % na;
                if (r < 0) r += na;
                return D.sa > 0 ? r : na - 1 - r;
            };
            // a ring of PD lines in flight: the loads of a line are issued PD line steps before
            // the line is computed (the loop is unrolled by PD so that every buffer is a fixed set
            // of registers)
            constexpr int PD = MAXM <= 4 ? 3 : 2;
            float pf[PD][5][MAXM];
            auto fetch = [&](float (&buf5)[5][MAXM], int al) {
#pragma unroll
                for (int q = 0; q < MAXM; ++q) {
                    const int b = lane + 32 * q;
                    if (q < M && b < nb) {
                        const size_t fk = lidx(k, al, b), fu = lidx(ku, al, b);
                        buf5[0][q] = __ldg(Sl + fk);
                        buf5[1][q] = __ldg(Al + fk);
                        buf5[2][q] = bufu[(size_t)al * nb + b];
                        buf5[3][q] = __ldg(Sl + fu);
                        buf5[4][q] = __ldg(Al + fu);
                    }
                }
            };
            auto stash = [&](const float (&buf5)[5][MAXM], int slot) {
#pragma unroll
                for (int q = 0; q < MAXM; ++q) {
                    const int b = lane + 32 * q;
                    if (q < M && b < nb) {
                        RING(R_SK, slot, b) = buf5[0][q];
                        RING(R_AK, slot, b) = buf5[1][q];
                        RING(R_IU, slot, b) = buf5[2][q];
                        RING(R_SU, slot, b) = buf5[3][q];
                        RING(R_AU, slot, b) = buf5[4][q];
                    }
                }
            };
            const float g1 = st.fb, g0 = 1.f - st.fb;
            int slot = 0;
            const int m0 = -st.warm;
            fetch(pf[0], line_of(m0 - 1));
            stash(pf[0], slot);
            // this plane's intensity on the line before the walk: the previous plane's as a start
            // (vertical face), unused on the plane face (wK = 0)
#pragma unroll
            for (int q = 0; q < MAXM; ++q) {
                const int b = lane + 32 * q;
                if (q < M && b < nb) RING(R_IK, slot, b) = st.wK != 0.f ? pf[0][2][q] : 0.f;
            }
#pragma unroll
            for (int p = 0; p < PD; ++p)
                if (m0 + p < na) fetch(pf[p], line_of(m0 + p));
            __syncwarp();
            // one line step: stash the line's prefetched inputs, refill the buffer PD lines ahead,
            // compute the line
            auto step = [&](float (&buf5)[5][MAXM], int m) {
                const int al = line_of(m);
                slot ^= 1;
                const int cur = slot, prv = slot ^ 1;
                stash(buf5, cur);
                if (m + PD < na) fetch(buf5, line_of(m + PD));
                __syncwarp();
                const bool store = m >= 0;
#pragma unroll
                for (int q = 0; q < MAXM; ++q) {
                    const int b = lane + 32 * q;
                    if (q < M && b < nb) {
                        const int b1 = D.sb > 0 ? (b == 0 ? nb - 1 : b - 1) : (b == nb - 1 ? 0 : b + 1);
                        const float iu =
                            g0 * (st.wA * RING(R_IU, cur, b) + st.wU * RING(R_IU, prv, b) +
                                  st.wK * RING(R_IK, prv, b)) +
                            g1 * (st.wA * RING(R_IU, cur, b1) + st.wU * RING(R_IU, prv, b1) +
                                  st.wK * RING(R_IK, prv, b1));
                        const float su =
                            g0 * (st.wA * RING(R_SU, cur, b) + st.wU * RING(R_SU, prv, b) +
                                  st.wK * RING(R_SK, prv, b)) +
                            g1 * (st.wA * RING(R_SU, cur, b1) + st.wU * RING(R_SU, prv, b1) +
                                  st.wK * RING(R_SK, prv, b1));
                        const float au =
                            g0 * (st.wA * RING(R_AU, cur, b) + st.wU * RING(R_AU, prv, b) +
                                  st.wK * RING(R_AK, prv, b)) +
                            g1 * (st.wA * RING(R_AU, cur, b1) + st.wU * RING(R_AU, prv, b1) +
                                  st.wK * RING(R_AK, prv, b1));
                        const float ak = RING(R_AK, cur, b), sk = RING(R_SK, cur, b);
                        float ex, w0, w1;
                        lin_weights(0.5f * (au + ak) * st.t, ex, w0, w1);
                        const float v = fmaf(iu, ex, fmaf(w0, su, w1 * sk));
                        RING(R_IK, cur, b) = v;
                        if (store) {
                            buf[(size_t)al * nb + b] = v;
                            if (Idir) Idir[fidx(k, al, b)] = v;
                        }
                    }
                }
                __syncwarp();
            };
            for (int m = m0; m < na; m += PD) {
#pragma unroll
                for (int p = 0; p < PD; ++p)
                    if (m + p < na) step(pf[p], m + p);
            }
        }
        if (!a.defer) {
            __syncthreads();
            j_plane(k);
        }
    }
#undef RING
}

// J of every point from the directions' planes kept by the sweep: J = sum over the directions in
// the tables' order of w_d I_d, the planes of directions whose lines run along x transposed
// through shared memory ([nxd][32][33] per 32 x 32 tile).  One block per (tile, plane, wavelength),
// FJ_PTS points a thread.  Every direction's source is addressed through one generic pointer (a
// global plane or a shared tile), so that the loop over directions has no branch and the loads
// of several directions are in flight at once.
constexpr int FJ_THREADS = 256, FJ_PTS = 1024 / FJ_THREADS;

__global__ void __launch_bounds__(FJ_THREADS) face_j_kernel(const float *__restrict__ vol,
                                                            float *__restrict__ J,
                                                            const FaceDir *__restrict__ dirs,
                                                            int ndir, int nx, int ny, int nz,
                                                            unsigned *err)
{
    extern __shared__ float tl[];
    __shared__ const float *src[MAX_DIR];   // the direction's plane, or its transposed tile
    __shared__ float wq[MAX_DIR];
    __shared__ const float *xpl[MAX_DIR];   // the planes held as [x][y], by tile slot
    __shared__ int isx[MAX_DIR];
    __shared__ int nxd;
    const int tcx = (nx + 31) >> 5;
    const int ti = (blockIdx.x % tcx) * 32, tj = (blockIdx.x / tcx) * 32;
    const int k = blockIdx.y, lam = blockIdx.z;
    const size_t np = (size_t)nx * ny;
    // the direction table, set up by the first warp (two directions a lane, MAX_DIR = 64): a
    // direction's tile slot is the number of directions along x before it in the table
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        unsigned bal[2];
        FaceDir D[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int q = lane + 32 * h;
            if (q < ndir) D[h] = dirs[q];
            bal[h] = __ballot_sync(0xffffffffu, q < ndir && D[h].a_is_x);
        }
        const unsigned lt = (1u << lane) - 1u;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int q = lane + 32 * h;
            if (q >= ndir) continue;
            const float *pl = vol + (((size_t)lam * ndir + D[h].dir) * nz + k) * np;
            wq[q] = D[h].w;
            isx[q] = D[h].a_is_x;
            if (D[h].a_is_x) {
                const int xi = (h ? __popc(bal[0]) : 0) + __popc(bal[h] & lt);
                xpl[xi] = pl;
                src[q] = tl + xi * 32 * 33;
            } else {
                src[q] = pl;
            }
        }
        if (lane == 0) nxd = __popc(bal[0]) + __popc(bal[1]);
    }
    __syncthreads();
    // stage the planes held as [x][y], transposed
#pragma unroll 2
    for (int xi = 0; xi < nxd; ++xi) {
        const float *pl = xpl[xi];
#pragma unroll
        for (int u = 0; u < FJ_PTS; ++u) {
            const int e = threadIdx.x + FJ_THREADS * u, r = e >> 5, c = e & 31;
            const int i = ti + r, j = tj + c;
            tl[(xi * 32 + r) * 33 + c] = (i < nx && j < ny) ? pl[(size_t)i * ny + j] : 0.f;
        }
    }
    __syncthreads();
    // per point: offset in a [y][x] plane (clamped into the plane) and in a transposed tile
    size_t goff[FJ_PTS];
    int toff[FJ_PTS];
    float acc[FJ_PTS];
#pragma unroll
    for (int u = 0; u < FJ_PTS; ++u) {
        const int e = threadIdx.x + FJ_THREADS * u, r = e >> 5, c = e & 31;
        const int i = min(ti + c, nx - 1), j = min(tj + r, ny - 1);
        goff[u] = (size_t)j * nx + i;
        toff[u] = c * 33 + r;
        acc[u] = 0.f;
    }
#pragma unroll 2
    for (int q = 0; q < ndir; ++q) {
        const float *b = src[q];
        const bool x = isx[q];
        const float w = wq[q];
#pragma unroll
        for (int u = 0; u < FJ_PTS; ++u) acc[u] = fmaf(w, b[x ? (size_t)toff[u] : goff[u]], acc[u]);
    }
#pragma unroll
    for (int u = 0; u < FJ_PTS; ++u) {
        const int e = threadIdx.x + FJ_THREADS * u, r = e >> 5, c = e & 31;
        const int i = ti + c, j = tj + r;
        if (i >= nx || j >= ny) continue;
        if (!isfinite(acc[u])) flag_error(err, ERR_NAN);
        J[((size_t)lam * nz + k) * np + (size_t)j * nx + i] = acc[u];
    }
}

// in [planes][ny][nx] -> out [planes][nx][ny]
__global__ void face_transpose_kernel(const float *__restrict__ in, float *__restrict__ out, int nx,
                                      int ny, int nplanes)
{
    __shared__ float t[32][33];
    const size_t np = (size_t)nx * ny;
    const int i0 = blockIdx.x * 32, j0 = blockIdx.y * 32;
    for (int p = blockIdx.z; p < nplanes; p += gridDim.z) {
        const float *src = in + (size_t)p * np;
        float *dst = out + (size_t)p * np;
        for (int r = threadIdx.y; r < 32; r += blockDim.y) {
            const int j = j0 + r, i = i0 + threadIdx.x;
            if (i < nx && j < ny) t[r][threadIdx.x] = src[(size_t)j * nx + i];
        }
        __syncthreads();
        for (int r = threadIdx.y; r < 32; r += blockDim.y) {
            const int i = i0 + r, j = j0 + threadIdx.x;
            if (i < nx && j < ny) dst[(size_t)i * ny + j] = t[threadIdx.x][r];
        }
        __syncthreads();
    }
}

// J += the other groups' partials, in group order
__global__ void face_sum_kernel(float *J, const float *Jp, int nparts, size_t n)
{
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        float v = J[i];
        for (int p = 0; p < nparts; ++p) v += Jp[(size_t)p * n + i];
        J[i] = v;
    }
}

static int face_maxm(const rt_grid *g) { return std::max(g->nx, g->ny) <= 128 ? 4 : 8; }

static size_t face_smem(const FaceTables *t)
{
    return ((size_t)t->wpb * 12 * t->nbpad + (size_t)t->wpb * 32 * 33) * sizeof(float);
}

static rt_status face_build(rt_grid *g)
{
    const double *z = g->z.data();
    std::vector<FaceDir> dirs;
    std::vector<int> first;
    std::vector<FaceStep> steps((size_t)g->ndir * g->nz, FaceStep{0, 0, 0, 0, 0, 0});
    int wpb = 0;
    for (int hemi = 0; hemi < 2; ++hemi) {
        const std::vector<int> &list = hemi == 0 ? g->dir_up : g->dir_dn;
        for (size_t c = 0; c < list.size(); c += FACE_MAXW) {
            first.push_back((int)dirs.size());
            const size_t e = std::min(list.size(), c + FACE_MAXW);
            wpb = std::max(wpb, (int)(e - c));
            for (size_t i = c; i < e; ++i) {
                const int q = list[i];
                const double *u = &g->dirs[3 * q];
                const double tx = u[0] != 0.0 ? g->dx / std::fabs(u[0]) : INFINITY;
                const double ty = u[1] != 0.0 ? g->dy / std::fabs(u[1]) : INFINITY;
                FaceDir d;
                d.dir = q;
                d.a_is_x = tx < ty;
                const double ua = d.a_is_x ? u[0] : u[1], ub = d.a_is_x ? u[1] : u[0];
                const double da = d.a_is_x ? g->dx : g->dy, db = d.a_is_x ? g->dy : g->dx;
                const int na = d.a_is_x ? g->nx : g->ny;
                d.sa = ua >= 0.0 ? 1 : -1;
                d.sb = ub >= 0.0 ? 1 : -1;
                d.up = u[2] > 0.0;
                d.w = (float)g->wdir[q];
                dirs.push_back(d);
                for (int s = 1; s < g->nz; ++s) {
                    const int k = d.up ? s : g->nz - 1 - s, ku = d.up ? k - 1 : k + 1;
                    const double dz = std::fabs(z[k] - z[ku]);
                    const double tz = dz / std::fabs(u[2]);
                    FaceStep &f = steps[(size_t)q * g->nz + s];
                    if (tz <= tx && tz <= ty) {
                        const double fa = tz * std::fabs(ua) / da;
                        f = FaceStep{(float)tz, (float)(1.0 - fa), (float)fa, 0.f,
                                     (float)(tz * std::fabs(ub) / db), 0};
                    } else {
                        const double t = d.a_is_x ? tx : ty;
                        const double fz = t * std::fabs(u[2]) / dz;
                        int warm = 0;
                        if (fz < 1.0) {
                            const double w = std::ceil(std::log(FACE_EPS) / std::log1p(-fz));
                            if (!(w <= 16.0 * na))
                                return fail(RT_EINVAL, "face scheme: plane spacing too coarse for "
                                                       "the periodic closure (over 16 laps)");
                            warm = (int)w;
                        }
                        f = FaceStep{(float)t, 0.f, (float)fz, (float)(1.0 - fz),
                                     (float)(t * std::fabs(ub) / db), warm};
                    }
                }
            }
        }
    }
    first.push_back((int)dirs.size());
    FaceTables *t = new FaceTables;
    for (const FaceDir &d : dirs) t->has_x |= d.a_is_x;
    t->ngroups = (int)first.size() - 1;
    t->wpb = wpb;
    for (const FaceDir &d : dirs) t->nxd += d.a_is_x;
    t->nbpad = (std::max(g->nx, g->ny) + 31) / 32 * 32;
    cudaError_t e = cudaMalloc(&t->d_dirs, dirs.size() * sizeof(FaceDir));
    if (e == cudaSuccess) e = cudaMalloc(&t->d_steps, steps.size() * sizeof(FaceStep));
    if (e == cudaSuccess) e = cudaMalloc(&t->d_first, first.size() * sizeof(int));
    if (e == cudaSuccess)
        e = cudaMemcpy(t->d_dirs, dirs.data(), dirs.size() * sizeof(FaceDir), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(t->d_steps, steps.data(), steps.size() * sizeof(FaceStep),
                       cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(t->d_first, first.data(), first.size() * sizeof(int), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        // the largest any grid can ask of each instance, so that no grid lowers another's limit
        const int s4 = (int)((FACE_MAXW * 12 * 128 + FACE_MAXW * 32 * 33) * sizeof(float));
        const int s8 = (int)((FACE_MAXW * 12 * 256 + FACE_MAXW * 32 * 33) * sizeof(float));
        e = face_maxm(g) == 4
                ? cudaFuncSetAttribute(face_sweep_kernel<4>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, s4)
                : cudaFuncSetAttribute(face_sweep_kernel<8>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, s8);
    }
    if (e != cudaSuccess) {
        face_release(t);
        return cuda_fail(e, "face scheme tables");
    }
    face_release(g->face);
    g->face = t;
    return RT_OK;
}

// J after the sweep: the directions' planes of every plane step are kept ([nlam][ndir][npt],
// 10.5 GB at 128^3 x 52 wavelengths x 24 directions) when that fits a quarter of the device's
// memory (RT_FACE_VOLUME_MB sets another budget) and the transposed tiles of the directions
// along x fit the J pass's shared memory; the warps then never wait for one another and one
// bandwidth-bound pass forms J.  Otherwise each block sums its directions' planes after every
// plane step.
static size_t face_j_smem(const FaceTables *t)
{
    return (size_t)std::max(t->nxd, 1) * 32 * 33 * sizeof(float);
}

static bool face_defer(const rt_grid *g, int nlam)
{
    if (face_j_smem(g->face) > 200 * 1024 || nlam > 65535 || g->nz > 65535) return false;
    size_t budget = 0, free_b = 0;
    if (cudaMemGetInfo(&free_b, &budget) != cudaSuccess) return false;
    budget /= 4;
    if (const char *e = std::getenv("RT_FACE_VOLUME_MB")) budget = (size_t)std::atoll(e) << 20;
    return (size_t)nlam * g->ndir * (size_t)g->npt * sizeof(float) <= budget;
}

// scratch: plane buffers [nlam][ndir][np] and J partials [ngroups-1][nlam][npt] (or, J after the
// sweep, every plane [nlam][ndir][npt]), and, when some direction's lines run along x, the
// transposed S and alpha [2][nlam][npt]
static size_t face_scratch_bytes(const rt_grid *g, int nlam, bool defer)
{
    const size_t np = (size_t)g->nx * g->ny;
    const size_t planes = defer ? (size_t)nlam * g->ndir * np * g->nz
                                : (size_t)nlam * g->ndir * np +
                                      (size_t)(g->face->ngroups - 1) * nlam * np * g->nz;
    return (planes + (size_t)2 * g->face->has_x * nlam * np * g->nz) * sizeof(float);
}

rt_status face_prepare(rt_grid *g, int nlam)
{
    void *p;
    return scratch_get(g, 4, face_scratch_bytes(g, nlam, face_defer(g, nlam)), &p);
}

rt_status face_formal_solution(rt_grid *g, int nlam, const float *alpha, const float *S, int bc,
                               const float *I_bc, float *J, float *I_dir, cudaStream_t st)
{
    const FaceTables *t = g->face;
    const bool defer = face_defer(g, nlam);
    void *p;
    RT_TRY(scratch_get(g, 4, face_scratch_bytes(g, nlam, defer), &p));
    FaceArgs a;
    a.alpha = alpha;
    a.S = S;
    a.I_bc = bc == RT_BC_ARRAY ? I_bc : nullptr;
    a.I_dir = I_dir;
    a.J = J;
    a.buf = (float *)p;
    a.defer = defer ? 1 : 0;
    a.Jp = defer ? nullptr : a.buf + (size_t)nlam * g->ndir * g->nx * g->ny;
    a.ST = a.AT = nullptr;
    if (t->has_x) {
        float *ST = defer ? a.buf + (size_t)nlam * g->ndir * g->npt
                          : a.Jp + (size_t)(t->ngroups - 1) * nlam * g->npt;
        float *AT = ST + (size_t)nlam * g->npt;
        const int nplanes = nlam * g->nz;
        const dim3 tg((g->nx + 31) / 32, (g->ny + 31) / 32, (unsigned)std::min(nplanes, 65535));
        note_launch(2);
        face_transpose_kernel<<<tg, dim3(32, 8), 0, st>>>(S, ST, g->nx, g->ny, nplanes);
        face_transpose_kernel<<<tg, dim3(32, 8), 0, st>>>(alpha, AT, g->nx, g->ny, nplanes);
        RT_CUDA(cudaGetLastError());
        a.ST = ST;
        a.AT = AT;
    }
    a.dirs = t->d_dirs;
    a.steps = t->d_steps;
    a.first = t->d_first;
    a.err = g->d_err;
    a.nx = g->nx;
    a.ny = g->ny;
    a.nz = g->nz;
    a.nlam = nlam;
    a.ndir = g->ndir;
    a.bc = bc;
    a.nbpad = t->nbpad;
    const dim3 grid((unsigned)nlam, (unsigned)t->ngroups);
    const size_t smem = face_smem(t);
    note_launch();
    if (face_maxm(g) == 4)
        face_sweep_kernel<4><<<grid, 32 * t->wpb, smem, st>>>(a);
    else
        face_sweep_kernel<8><<<grid, 32 * t->wpb, smem, st>>>(a);
    RT_CUDA(cudaGetLastError());
    if (defer) {
        const size_t jsm = face_j_smem(t);
        if (jsm > 48 * 1024)
            RT_CUDA(cudaFuncSetAttribute(face_j_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)jsm));
        const dim3 jg((unsigned)(((g->nx + 31) / 32) * ((g->ny + 31) / 32)), (unsigned)g->nz,
                      (unsigned)nlam);
        note_launch();
        face_j_kernel<<<jg, 256, jsm, st>>>(a.buf, J, t->d_dirs, g->ndir, g->nx, g->ny, g->nz,
                                            g->d_err);
        RT_CUDA(cudaGetLastError());
    } else if (t->ngroups > 1) {
        note_launch();
        face_sum_kernel<<<1216, 256, 0, st>>>(J, a.Jp, t->ngroups - 1, (size_t)nlam * g->npt);
        RT_CUDA(cudaGetLastError());
    }
    return RT_OK;
}

}  // namespace rt

using namespace rt;

extern "C" rt_status rt_grid_set_scheme(rt_grid_t g, int scheme)
{
    return guarded([&]() -> rt_status {
        if (!g) return fail(RT_EINVAL, "null grid");
        if (scheme != RT_SC_PLANE && scheme != RT_SC_FACE) return fail(RT_EINVAL, "unknown scheme");
        if (scheme == RT_SC_FACE) {
            if (g->kind != RT_GRID_REGULAR) return fail(RT_EINVAL, "the face scheme is for regular grids");
            if (!g->periodic) return fail(RT_EINVAL, "the face scheme needs periodic sides");
            if (std::max(g->nx, g->ny) > FACE_MAXNB) return fail(RT_EINVAL, "face scheme: nx, ny <= 256");
            if (!g->face) RT_TRY(face_build(g));
        }
        g->sc_face = scheme == RT_SC_FACE;
        return RT_OK;
    });
}
