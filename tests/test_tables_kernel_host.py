"""The GPU table kernels' source (csrc/tables.cu: voronoi_tables_kernel, voronoi_levels_kernel),
compiled for the host and run thread by thread, against the FP64 oracle (CPU only).

The kernels compute every geometric step with explicit round-to-nearest double intrinsics; on
the host those are the plain IEEE double operations (compiled without contraction), so the run
performs the same arithmetic.  This checks the kernels' indexing, tie rules, wall handling and
level relaxation on every CPU test run; the run on the GPU is test_gpu_tables_device.py.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
from helpers import lattice_grid, tie_directions
from synth import delaunay_neighbours, s4_quadrature

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "paper_2306_01041_gb300", "csrc", "tables.cu")

# host definitions of what the kernels use from CUDA and from the library's headers
PRELUDE = r"""
#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstdint>
#include <cstdio>
#include <vector>
#define __global__
#define __device__
#define __forceinline__ inline
#define __launch_bounds__(x)
struct D3 { unsigned x, y, z; };
static D3 blockIdx, blockDim, threadIdx;
static inline double __dadd_rn(double a, double b) { return a + b; }
static inline double __dsub_rn(double a, double b) { return a - b; }
static inline double __dmul_rn(double a, double b) { return a * b; }
static inline double __ddiv_rn(double a, double b) { return a / b; }
static inline double __dsqrt_rn(double a) { return std::sqrt(a); }
static inline unsigned long long atomicAdd(unsigned long long *p, unsigned long long v)
{ unsigned long long o = *p; *p += v; return o; }
static inline int atomicMax(int *p, int v) { int o = *p; if (v > o) *p = v; return o; }
using std::fabs; using std::max; using std::pow;
namespace rt {
enum : unsigned { ERR_NAN = 1u, ERR_TIMEOUT = 2u, ERR_INDEX = 4u };
struct Upwind { int k1, k2; float w1, l1, l2; };
static inline void flag_error(unsigned *err, unsigned bit) { if (err) *err |= bit; }
}
"""

# reads one grid, runs every (block, thread) of the table kernel, then level passes until none
# grows, writes the records, the levels, the fallback count and the error word
DRIVER = r"""
using namespace rt;
template <class T> static void rd(FILE *f, T *p, size_t n) { if (fread(p, sizeof(T), n, f) != n) throw 1; }
int main(int argc, char **argv)
{
    FILE *f = fopen(argv[1], "rb");
    int64_t n, ne; int nd; double box[6], r;
    rd(f, &n, 1); rd(f, &ne, 1); rd(f, &nd, 1); rd(f, box, 6); rd(f, &r, 1);
    std::vector<double> xyz(3 * n), dirs(3 * nd);
    std::vector<int64_t> off(n + 1); std::vector<int32_t> code(ne); std::vector<int8_t> shift(ne);
    rd(f, xyz.data(), 3 * n); rd(f, off.data(), n + 1); rd(f, code.data(), ne);
    rd(f, shift.data(), ne); rd(f, dirs.data(), 3 * nd);
    fclose(f);
    std::vector<Upwind> up((size_t)nd * n);
    std::vector<int> level((size_t)nd * n, 0);
    unsigned long long nfb = 0;
    unsigned err = 0, changed = 1;
    TabArgs a;
    a.xyz = xyz.data(); a.off = off.data(); a.code = code.data(); a.shift = shift.data();
    a.dirs = dirs.data(); a.r_exp = r; a.n = n; a.up = up.data(); a.nfb = &nfb; a.err = &err;
    for (int q = 0; q < 6; ++q) a.box[q] = box[q];
    const unsigned nbx = (unsigned)((n + 255) / 256);
    blockDim.x = 256;
    for (unsigned by = 0; by < (unsigned)nd; ++by)
        for (unsigned bx = 0; bx < nbx; ++bx)
            for (unsigned t = 0; t < 256; ++t) {
                blockIdx.x = bx; blockIdx.y = by; threadIdx.x = t;
                voronoi_tables_kernel(a);
            }
    for (int pass = 0; changed && pass <= n + 1; ++pass) {
        changed = 0;
        for (unsigned by = 0; by < (unsigned)nd; ++by)
            for (unsigned bx = 0; bx < nbx; ++bx)
                for (unsigned t = 0; t < 256; ++t) {
                    blockIdx.x = bx; blockIdx.y = by; threadIdx.x = t;
                    voronoi_levels_kernel(up.data(), n, level.data(), &changed, &err);
                }
    }
    FILE *o = fopen(argv[2], "wb");
    fwrite(up.data(), sizeof(Upwind), up.size(), o);
    fwrite(level.data(), sizeof(int), level.size(), o);
    fwrite(&nfb, 8, 1, o);
    fwrite(&err, 4, 1, o);
    fwrite(&changed, 4, 1, o);
    fclose(o);
    return 0;
}
"""


@pytest.fixture(scope="module")
def host_tables(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    src = open(SRC).read()
    a = src.index("namespace rt {")
    b = src.index("}  // namespace rt") + len("}  // namespace rt")
    d = tmp_path_factory.mktemp("tables_host")
    cpp = d / "tables_host.cpp"
    cpp.write_text(PRELUDE + src[a:b] + DRIVER)
    exe = d / "tables_host"
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-o", str(exe),
                           str(cpp)])

    def run(g, dirs):
        n = len(g["xyz"])
        ne = int(g["nbr_off"][-1])
        inp, out = d / "in.bin", d / "out.bin"
        with open(inp, "wb") as f:
            np.array([n, ne], np.int64).tofile(f)
            np.array([len(dirs)], np.int32).tofile(f)
            np.array(g["box"], np.float64).tofile(f)
            np.array([7.0]).tofile(f)
            np.ascontiguousarray(g["xyz"], np.float64).tofile(f)
            np.asarray(g["nbr_off"], np.int64).tofile(f)
            np.asarray(g["nbr_idx"], np.int32).tofile(f)
            np.asarray(g["nbr_shift"], np.int8).tofile(f)
            np.ascontiguousarray(dirs, np.float64).tofile(f)
        subprocess.check_call([str(exe), str(inp), str(out)])
        nd = len(dirs)
        rec = np.dtype([("k1", "<i4"), ("k2", "<i4"), ("w1", "<f4"), ("l1", "<f4"), ("l2", "<f4")])
        raw = out.read_bytes()
        up = np.frombuffer(raw[:nd * n * 20], rec).reshape(nd, n)
        lev = np.frombuffer(raw[nd * n * 20:nd * n * 24], np.int32).reshape(nd, n)
        nfb, = np.frombuffer(raw[nd * n * 24:nd * n * 24 + 8], np.uint64)
        err, changed = np.frombuffer(raw[nd * n * 24 + 8:], np.uint32)
        return up, lev, int(nfb), int(err), int(changed)
    return run


def _random_grid(seed, n):
    rng = np.random.default_rng(seed)
    box = (0.0, 1.0, 0.0, 1.0, 0.0, 1.0)
    xyz = rng.random((n, 3)) ** np.array([1.0, 1.0, 2.0])     # denser near the bottom wall
    off, code, shift = delaunay_neighbours(xyz, box)
    return dict(xyz=xyz, nbr_off=off, nbr_idx=code, nbr_shift=shift, box=box)


@pytest.mark.parametrize("grid", ["random400", "random1500", "lattice", "column"])
def test_table_kernels_reproduce_the_oracle(host_tables, grid):
    """Random sites (Delaunay neighbours with periodic images and wall mirrors) with the S4
    directions, and a lattice with directions for which two neighbours tie exactly for second
    place (the tie rules decide)."""
    g = {"random400": lambda: _random_grid(1, 400), "random1500": lambda: _random_grid(3, 1500),
         "lattice": lambda: lattice_grid(4), "column": lambda: lattice_grid(1, 4)}[grid]()
    dirs = tie_directions()[0] if grid in ("lattice", "column") else s4_quadrature()[0]
    up, lev, nfb, err, changed = host_tables(g, dirs)
    ref = oracle.voronoi_tables(g["xyz"], g["nbr_off"], g["nbr_idx"], g["nbr_shift"], g["box"],
                                dirs, 7.0)
    assert err == 0 and changed == 0
    np.testing.assert_array_equal(np.stack([up["k1"], up["k2"]], -1), ref["k"])
    np.testing.assert_array_equal(lev, ref["level"])
    np.testing.assert_allclose(up["w1"], ref["w"][:, :, 0], rtol=1e-6, atol=1e-7)
    np.testing.assert_allclose(np.stack([up["l1"], up["l2"]], -1), ref["len"], rtol=1e-6)
    assert nfb == ref["n_fallback"]
