// Ng acceleration of the Lambda iteration: a least-squares extrapolation from the last four
// iterates (not in the paper, which iterates plain Lambda, Sect. 2.1).
//
// With x0 the newest iterate and d0 = x0 - x1, d1 = x1 - x2, d2 = x2 - x3, the coefficients (a, b)
// minimise the weighted norm of d0 - a (d0 - d1) - b (d0 - d2) (weights 1/x0^2: every population
// counts by its relative change), and x = (1 - a - b) x0 + a x1 + b x2.  The five inner products
// are accumulated in FP64 (block sums, one FP64 atomic per block and product); the 2 x 2 system
// is solved on the host; the combination is written only if every entry stays positive.
#include <cmath>

#include "device_common.cuh"
#include "rt_impl.h"

namespace rt {

__global__ void __launch_bounds__(256) ng_dots_kernel(const float *x0, const float *x1,
                                                      const float *x2, const float *x3, int64_t n,
                                                      double *out)
{
    double acc[5] = {0, 0, 0, 0, 0};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double a0 = x0[i], a1 = x1[i], a2 = x2[i], a3 = x3[i];
        const double w = 1.0 / (a0 * a0);
        const double d0 = a0 - a1, d1 = a1 - a2, d2 = a2 - a3;
        const double u = d0 - d1, v = d0 - d2;
        acc[0] += w * u * u;
        acc[1] += w * u * v;
        acc[2] += w * v * v;
        acc[3] += w * d0 * u;
        acc[4] += w * d0 * v;
    }
    __shared__ double red[8][5];
#pragma unroll
    for (int k = 0; k < 5; ++k)
        for (int o = 16; o; o >>= 1) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], o);
    if ((threadIdx.x & 31) == 0)
#pragma unroll
        for (int k = 0; k < 5; ++k) red[threadIdx.x >> 5][k] = acc[k];
    __syncthreads();
    if (threadIdx.x < 5) {
        double s = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w][threadIdx.x];
        atomicAdd(out + threadIdx.x, s);
    }
}

// out = (1 - a - b) x0 + a x1 + b x2; *bad counts entries that are not positive
__global__ void ng_combine_kernel(const float *x0, const float *x1, const float *x2, double a,
                                  double b, int64_t n, float *out, int *bad)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double v = (1.0 - a - b) * x0[i] + a * x1[i] + b * x2[i];
    if (!(v > 0.0)) atomicAdd(bad, 1);
    out[i] = (float)v;
}

// The extrapolation into out (device, n floats); *ok = 1 if it was written with every entry
// positive and the system was regular, else 0 (out then unspecified).  scratch: 64 bytes of
// device memory.  Synchronises on st.
rt_status ng_extrapolate(const float *x0, const float *x1, const float *x2, const float *x3,
                         int64_t n, float *out, void *scratch, cudaStream_t st, int *ok)
{
    double *dots = static_cast<double *>(scratch);
    int *bad = reinterpret_cast<int *>(dots + 5);
    *ok = 0;
    RT_CUDA(cudaMemsetAsync(scratch, 0, 5 * sizeof(double) + sizeof(int), st));
    note_launch();
    ng_dots_kernel<<<304, 256, 0, st>>>(x0, x1, x2, x3, n, dots);
    double h[5];
    RT_CUDA(cudaMemcpyAsync(h, dots, sizeof(h), cudaMemcpyDeviceToHost, st));
    RT_CUDA(cudaStreamSynchronize(st));
    const double det = h[0] * h[2] - h[1] * h[1];
    if (!(std::fabs(det) > 1e-300) || !std::isfinite(det)) return RT_OK;
    const double a = (h[3] * h[2] - h[1] * h[4]) / det;
    const double b = (h[0] * h[4] - h[1] * h[3]) / det;
    if (!std::isfinite(a) || !std::isfinite(b)) return RT_OK;
    note_launch();
    ng_combine_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(x0, x1, x2, a, b, n, out, bad);
    int hb = 0;
    RT_CUDA(cudaMemcpyAsync(&hb, bad, sizeof(int), cudaMemcpyDeviceToHost, st));
    RT_CUDA(cudaStreamSynchronize(st));
    *ok = hb == 0;
    return RT_OK;
}

}  // namespace rt

using namespace rt;

extern "C" rt_status rt_ng_extrapolate(int64_t n, const float *x0, const float *x1,
                                       const float *x2, const float *x3, float *out,
                                       void *scratch, int *ok, void *stream)
{
    return guarded([&]() -> rt_status {
        if (n < 1 || !x0 || !x1 || !x2 || !x3 || !out || !scratch || !ok)
            return fail(RT_EINVAL, "bad argument");
        return ng_extrapolate(x0, x1, x2, x3, n, out, scratch, (cudaStream_t)stream, ok);
    });
}
