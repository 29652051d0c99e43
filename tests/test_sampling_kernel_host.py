"""The GPU sampler's proposal function (csrc/sampling.cu: Philox4x64-10, position, trilinear
target, keep decision), compiled for the host and run proposal by proposal, against the oracle
(CPU only): positions and decisions must be identical, bit for bit.

The device code uses explicit round-to-nearest double intrinsics; on the host they are the plain
IEEE double operations (no contraction), so the run performs the same arithmetic.  The GPU run is
test_gpu_sampling.py.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle.sampling import interpolate, proposals

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "paper_2306_01041_gb300", "csrc", "sampling.cu")

PRELUDE = r"""
#include <cmath>
#include <cstddef>
#include <cstdint>
#include <cstdio>
#include <vector>
#define __global__
#define __device__
#define __forceinline__ inline
#define __launch_bounds__(x)
static inline double __dadd_rn(double a, double b) { return a + b; }
static inline double __dsub_rn(double a, double b) { return a - b; }
static inline double __dmul_rn(double a, double b) { return a * b; }
static inline double __ddiv_rn(double a, double b) { return a / b; }
static inline double __ull2double_rn(unsigned long long v) { return (double)v; }
static inline uint64_t __umul64hi(uint64_t a, uint64_t b)
{ return (uint64_t)(((unsigned __int128)a * b) >> 64); }
template <class T> static inline T __ldg(const T *p) { return *p; }
using std::floor;
"""

DRIVER = r"""
using namespace rt;
template <class T> static void rd(FILE *f, T *p, size_t n) { if (fread(p, sizeof(T), n, f) != n) throw 1; }
int main(int argc, char **argv)
{
    FILE *f = fopen(argv[1], "rb");
    int nx, ny, nz; long long count; unsigned long long seed; double box[6], fmax;
    rd(f, &nx, 1); rd(f, &ny, 1); rd(f, &nz, 1); rd(f, &count, 1); rd(f, &seed, 1);
    rd(f, box, 6); rd(f, &fmax, 1);
    std::vector<double> z(nz); std::vector<float> tf((size_t)nx * ny * nz);
    rd(f, z.data(), nz); rd(f, tf.data(), tf.size());
    fclose(f);
    SampleArgs a;
    a.f = tf.data(); a.z = z.data(); a.fmax = fmax; a.seed = seed; a.nx = nx; a.ny = ny; a.nz = nz;
    for (int q = 0; q < 6; ++q) a.box[q] = box[q];
    FILE *o = fopen(argv[2], "wb");
    for (long long p = 0; p < count; ++p) {
        double r[3];
        const unsigned char keep = propose(a, (uint64_t)p, r) ? 1 : 0;
        fwrite(r, 8, 3, o);
        fwrite(&keep, 1, 1, o);
    }
    fclose(o);
    return 0;
}
"""


@pytest.fixture(scope="module")
def host_propose(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    src = open(SRC).read()
    a = src.index("namespace rt {")
    b = src.index("// exclusive scan of one int per thread")
    d = tmp_path_factory.mktemp("sampling_host")
    cpp = d / "propose_host.cpp"
    cpp.write_text(PRELUDE + src[a:b] + "}  // namespace rt\n" + DRIVER)
    exe = d / "propose_host"
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-o", str(exe),
                           str(cpp)])

    def run(f, z, box, count, seed):
        nz, ny, nx = f.shape
        inp, out = d / "in.bin", d / "out.bin"
        with open(inp, "wb") as fh:
            np.array([nx, ny, nz], np.int32).tofile(fh)
            np.array([count], np.int64).tofile(fh)
            np.array([seed], np.uint64).tofile(fh)
            np.array(box, np.float64).tofile(fh)
            np.array([float(f.astype(np.float64).max())]).tofile(fh)
            np.asarray(z, np.float64).tofile(fh)
            np.ascontiguousarray(f, np.float32).tofile(fh)
        subprocess.check_call([str(exe), str(inp), str(out)])
        rec = np.fromfile(out, np.dtype([("r", "<f8", 3), ("keep", "u1")]))
        return rec["r"], rec["keep"].astype(bool)
    return run


@pytest.mark.parametrize("seed", [7, 2 ** 64 - 3])
def test_proposals_and_decisions_equal_the_oracle(host_propose, seed):
    rng = np.random.default_rng(4)
    nx, ny, nz = 9, 7, 11
    z = np.sort(np.r_[-0.45, 2.4, rng.uniform(-0.45, 2.4, nz - 2)])   # proposals below and above
    f = (rng.uniform(0.0, 1.0, (nz, ny, nx)) ** 3).astype(np.float32)
    box = (0.0, 6.0, 0.0, 6.0, -0.5, 2.5)
    count = 20000
    pos, keep = host_propose(f, z, box, count, seed)
    ref_pos, prej = proposals(seed, 0, count, box)
    ref_keep = interpolate(f.astype(np.float64), z, box, ref_pos) >= prej * float(f.max())
    assert np.array_equal(pos, ref_pos)
    assert np.array_equal(keep, ref_keep)
    assert 0 < keep.sum() < count
