// Internal declarations shared by the translation units of librt.so (host and device).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <exception>
#include <new>
#include <string>
#include <vector>

#include "../../include/rt.h"

namespace rt {

// ---- error reporting --------------------------------------------------------------------------
rt_status fail(rt_status st, const std::string &msg);
rt_status cuda_fail(cudaError_t e, const char *what);
#define RT_CUDA(call)                                                 \
    do {                                                              \
        cudaError_t e_ = (call);                                      \
        if (e_ != cudaSuccess) return ::rt::cuda_fail(e_, #call);     \
    } while (0)
#define RT_TRY(call)                                                  \
    do {                                                              \
        rt_status s_ = (call);                                        \
        if (s_ != RT_OK) return s_;                                   \
    } while (0)

// The body of a C ABI entry point: a failed host allocation or any other C++ exception becomes a
// status (and a message) instead of crossing the C boundary.
template <class F>
rt_status guarded(F &&body)
{
    try {
        return body();
    } catch (const std::bad_alloc &) {
        return fail(RT_ENOMEM, "host allocation failed");
    } catch (const std::exception &e) {
        return fail(RT_EINVAL, e.what());
    } catch (...) {
        return fail(RT_EINVAL, "unexpected host exception");
    }
}

// process-wide count of kernel launches issued by the library (also those recorded into a graph)
void note_launch(unsigned n = 1);

inline bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// device error word bits (rt::DevErr in the grid)
enum : unsigned { ERR_NAN = 1u, ERR_TIMEOUT = 2u, ERR_INDEX = 4u };

constexpr int MAX_DIR = 64;

// ---- regular grid: per (plane, direction) upwind stencil ----------------------------------------
// The upwind point of (i, j) in plane k lies at (i + ax + tx, j + ay + ty) of the upwind plane,
// tx, ty in [0, 1).  Bilinear weights w[0..3] for corners (ax,ay), (ax+1,ay), (ax,ay+1),
// (ax+1,ay+1); hds = half the path length between the planes (so dtau = (a_up + a) * hds).
// axm, aym: ax, ay reduced modulo nx, ny (periodic wrap without integer division on the device).
struct Stencil {
    int ax, ay, axm, aym;
    float w0, w1, w2, w3;
    float hds;
    float pad;
    float tx, ty;     // fractional offsets: w0 = (1 - tx)(1 - ty), w1 = tx (1 - ty), w2 = (1 - tx) ty
};

// One direction's stencil on one plane as the pipelined regular sweep reads it (three 16-byte
// loads): (v, v) pairs of the fractional offsets and of their complements, half path length,
// quadrature weight, corner displacement in the staged tile (ay * 40 + ax) and the plane's smallest
// half path length over the hemisphere.
struct PlaneStencil {
    float2 tx, ux, ty, uy;
    float hds, wd;
    int off;
    float hds_min;
};
static_assert(sizeof(PlaneStencil) == 48, "PlaneStencil is three float4");

// FP64 stencil of one direction, for the adjoint's forward recomputation.
struct StencilD {
    int ax, ay, axm, aym;
    double w0, w1, w2, w3;
    double hds;
};

// ---- Voronoi grid: per (direction, site) upwind record --------------------------------------------
// k1, k2: upwind site (>= 0) or wall (-1 bottom, -2 top); w1 (w2 = 1 - w1; w1 = 1 and w2 = 0
// with a single upwind line); l1, l2: segment lengths.
struct Upwind {
    int k1, k2;
    float w1, l1, l2;
};

// FP64 record (the adjoint of one direction): w2 held explicitly.
struct UpwindD {
    int k1, k2;
    double w1, w2, l1, l2;
};

// Upwind tables of a set of directions on one Voronoi grid.
struct VorTables {
    int ndir = 0;
    std::vector<double> dirs;                  // [ndir][3]
    std::vector<Upwind> h_up;                  // [ndir][nsites], site order
    std::vector<UpwindD> h_upd;                // FP64 copy (single-direction tables only)
    std::vector<int32_t> h_level;              // [ndir][nsites]
    std::vector<std::vector<int64_t>> lvl_off; // per direction: level offsets into the slots
    Upwind *d_up = nullptr;                    // [ndir][nsites], slot (level) order
    int32_t *d_order = nullptr;                // [ndir][nsites]: site held by each slot
    int max_levels = 0;
    int64_t n_fallback = 0;
    void release();
};

struct FaceTables;                             // face-hitting scheme tables (regular_face.cu)
void face_release(FaceTables *t);
struct MapTable;                               // emergent map's pixel table (idw.cu)
void map_release(MapTable *t);

struct Scratch {
    void *p = nullptr;
    size_t bytes = 0;
};

}  // namespace rt

struct rt_grid {
    int kind;
    int device;
    int ndir;
    std::vector<double> dirs, wdir;
    int periodic;
    int64_t npt;
    // regular
    int nx = 0, ny = 0, nz = 0;
    double dx = 0, dy = 0;
    std::vector<double> z;
    std::vector<int> dir_up, dir_dn;           // direction indices per hemisphere
    rt::Stencil *d_stencil = nullptr;          // [nz][ndir]; plane k's stencil to its upwind
    std::vector<rt::Stencil> h_stencil;
    rt::Stencil *d_stencil_one = nullptr;      // [nz]: one extra direction (emergent/adjoint)
    std::vector<rt::Stencil> h_stencil_one;
    rt::StencilD *d_stencil_oned = nullptr;    // FP64 copy for the adjoint
    std::vector<rt::StencilD> h_stencil_oned;
    double one_dir[3] = {0, 0, 0};
    void *d_wave_st = nullptr;                 // [nz][2][12] per-plane stencils of the wavefront sweep
    std::vector<char> h_wave_st;
    int sc_face = 0;                           // rt_grid_set_scheme(RT_SC_FACE) selected
    rt::FaceTables *face = nullptr;
    // voronoi
    std::vector<double> xyz;
    double box[6];
    int64_t nsites = 0;
    double r_exp = 7.0;
    std::vector<int64_t> nbr_off;
    std::vector<int32_t> nbr_idx;
    std::vector<int8_t> nbr_shift;
    rt::VorTables vt;                          // the quadrature directions
    rt::VorTables vt_one;                      // cache: one extra direction (emergent/adjoint)
    rt::Upwind *d_up_site = nullptr;           // [ndir][nsites] records in site order (Lambda*)
    rt_batch *self_batch = nullptr;            // persistent all-direction sweep of this grid alone
    int self_batch_nlam = 0;
    int64_t n_fallback = 0;
    int max_levels = 0;
    std::vector<int64_t> top;                  // emergent-layer points
    int64_t *d_top = nullptr;
    rt::MapTable *map = nullptr;               // cache: pixel table of rt_emergent_map
    // shared
    unsigned *d_err = nullptr;                 // device error word
    rt::Scratch scratch[5];
    ~rt_grid();
};

namespace rt {
rt_status scratch_get(rt_grid *g, int slot, size_t bytes, void **out);
rt_status check_dev_error(rt_grid *g, cudaStream_t st);

// launchers (defined in the .cu files)
rt_status regular_formal_solution(rt_grid *g, int nlam, const float *alpha, const float *S, int bc,
                                  const float *I_bc, float *J, float *I_dir, cudaStream_t st);
// face-hitting sweep of a grid whose scheme is RT_SC_FACE; face_prepare allocates its scratch
rt_status face_formal_solution(rt_grid *g, int nlam, const float *alpha, const float *S, int bc,
                               const float *I_bc, float *J, float *I_dir, cudaStream_t st);
rt_status face_prepare(rt_grid *g, int nlam);
// Voronoi tables: slot order, level offsets and upload from vt.h_up and vt.h_level
rt_status voronoi_upload_slots(VorTables &vt, int64_t n, cudaStream_t st);
// tiled per-plane sweep (default on periodic grids); *done = false when it does not apply
rt_status regular_tile_sweep(rt_grid *g, int nlam, const float *alpha, const float *S, int bc,
                             float *J, float *buf0, float *buf1, cudaStream_t st, bool *done);
size_t regular_wave_scratch(const rt_grid *g, int nlam);
// byte offset, in the wavefront sweep's device table, of the per-plane stencil table with
// fractional offsets (48-byte entries [nz][2][12])
size_t regular_wave_table_offset(const rt_grid *g);
// pipelined wavefront sweep (producer warp, tensor copies); *done = false when it does not apply
rt_status regular_pipe_sweep(rt_grid *g, int nlam, const float *alpha, const float *S, int bc,
                             float *J, cudaStream_t st, bool *done);
size_t regular_pipe_scratch(const rt_grid *g, int nlam);
// Voronoi: builds what the formal solution of nlam wavelengths allocates on first use (call
// outside stream capture)
rt_status voronoi_prepare(rt_grid *g, int nlam);
// Lambda* [nlam][npt] (diagonal of the Lambda operator) of the opacities alpha
rt_status lambda_star(rt_grid *g, int nlam, const float *alpha, int bc, float *L, cudaStream_t st);
// allocates what lambda_star needs on first use (call outside stream capture)
rt_status lambda_star_prepare(rt_grid *g);
// Ng extrapolation of four iterates into out (n floats); *ok = 1 if written with every entry
// positive.  scratch: 64 bytes of device memory.  Synchronises on st.
rt_status ng_extrapolate(const float *x0, const float *x1, const float *x2, const float *x3,
                         int64_t n, float *out, void *scratch, cudaStream_t st, int *ok);
// builds and uploads the wavefront sweep's per-plane stencil table (no-op where it cannot apply)
rt_status regular_wave_prepare(rt_grid *g, cudaStream_t st);
rt_status regular_emergent(rt_grid *g, const double *dir, int nlam, const float *alpha,
                           const float *S, int bc, float *I_top, cudaStream_t st);
size_t regular_adjoint_ws(rt_grid *g, int nlam, int stride);
rt_status regular_adjoint(rt_grid *g, const double *dir, int nlam, const float *alpha,
                          const float *S, int bc, const float *gI_top, float *g_alpha, float *g_S,
                          int stride, void *ws, size_t ws_bytes, cudaStream_t st);
rt_status voronoi_formal_solution(rt_grid *g, int nlam, const float *alpha, const float *S, int bc,
                                  const float *I_bc, float *J, float *I_dir, cudaStream_t st);
rt_status voronoi_emergent(rt_grid *g, const double *dir, int nlam, const float *alpha,
                           const float *S, int bc, float *I_top, cudaStream_t st);
size_t voronoi_adjoint_ws(rt_grid *g, int nlam, int stride);
rt_status voronoi_adjoint(rt_grid *g, const double *dir, int nlam, const float *alpha,
                          const float *S, int bc, const float *gI_top, float *g_alpha, float *g_S,
                          int stride, void *ws, size_t ws_bytes, cudaStream_t st);
// stencils of one direction for every plane (regular grid), host-built
std::vector<Stencil> regular_dir_stencils(const rt_grid *g, const double *u);
std::vector<StencilD> regular_dir_stencils_d(const rt_grid *g, const double *u);
// upwind tables of the given directions (Voronoi), built on the host and uploaded
rt_status voronoi_build_tables(const rt_grid *g, int ndir, const double *dirs, VorTables &vt,
                               cudaStream_t st);
// the upwind tables and levels of the grid's quadrature directions built on the device (the
// default of rt_grid_create; RT_VORONOI_TABLES=host selects voronoi_build_tables)
rt_status voronoi_build_tables_device(rt_grid *g, cudaStream_t st);
// tables of one extra direction, cached on the grid
rt_status voronoi_dir_tables_cached(rt_grid *g, const double *dir, VorTables **out,
                                    cudaStream_t st);
// a batch's grids and wavelength count (batch.cu), and its device error word: read, reset and
// turned into a status (synchronises on st)
int batch_ngrids(const rt_batch *b);
rt_grid *batch_grid(const rt_batch *b, int i);
int batch_nlam(const rt_batch *b);
rt_status batch_check_error(rt_batch *b, cudaStream_t st);
}  // namespace rt
