// Device helpers shared by the kernels of librt.so.
#pragma once

#include <cuda_runtime.h>

namespace rt {

// e^-d from the hardware base-2 exponential, e^-d = 2^(-d log2 e); flushes results below the
// smallest normal float (d > 87) to zero.  Relative error about 2^-22 (PTX ex2.approx).
__device__ __forceinline__ float exp_neg(float d)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(d * -1.4426950408889634f));
    return y;
}

// 1/x from the hardware reciprocal (PTX rcp.approx, about 1 ulp; x must be a normal float).
__device__ __forceinline__ float rcp_fast(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Linear-S integration over one optical-depth interval d (Sect. 2.5: S linear across the
// interval; Eq. 2):  I = I_up e^-d + w0 S_up + w1 S with e0 = 1 - e^-d, w1 = 1 - e0 / d,
// w0 = e0 / d - e^-d (= e0 - w1).  Below d = 0.1 both weights come from their Taylor series
// (truncated after d^5, relative error < 3e-8): in optically thin layers I can be far below S, so
// the weights need relative, not just absolute, accuracy.  Above, q = e0 / d (fast reciprocal;
// e0 >= 0.095 there keeps full relative precision), w1 = 1 - q and w0 = q - e^-d.  w0 is not taken
// as e0 - w1: for d beyond ~1e7 w1 rounds to 1 in FP32 and the difference would lose w0 ~ 1/d
// entirely, while w0 S_up still matters where S_up exceeds S by a factor near d.  The packed pair
// form (lin_weights_thick2) performs the same operations in the same order.
__device__ __forceinline__ void lin_weights(float d, float &ex, float &w0, float &w1)
{
    ex = exp_neg(d);
    if (d < 0.1f) {   // neighbouring points have similar dtau: the branch is warp-uniform
        w1 = d * (0.5f + d * (-1.0f / 6.0f + d * (1.0f / 24.0f +
                                                d * (-1.0f / 120.0f + d * (1.0f / 720.0f)))));
        w0 = d * (0.5f + d * (-1.0f / 3.0f + d * (1.0f / 8.0f +
                                                d * (-1.0f / 30.0f + d * (1.0f / 144.0f)))));
    } else {
        const float e0 = 1.0f - ex;
        const float q = __fmul_rn(e0, rcp_fast(d));   // rounded once, not fused below
        w1 = 1.0f - q;
        w0 = q - ex;
    }
}

// Interval weights for d >= 0.1 only: the same arithmetic as the d >= 0.1 branch of lin_weights.
__device__ __forceinline__ void lin_weights_thick(float d, float &ex, float &w0, float &w1)
{
    ex = exp_neg(d);
    const float e0 = 1.0f - ex;
    const float q = __fmul_rn(e0, rcp_fast(d));
    w1 = 1.0f - q;
    w0 = q - ex;
}

// ---- two points at once: packed FP32 pairs (the f32x2 arithmetic of sm_100 and later) ---------
// The same operations as the scalar forms above, on the two components of a float2 (one rounding
// per component, as the scalar FMA): the stencil weights of a direction are shared by a thread's
// two points, so their interpolations and interval weights run as pairs.
__device__ __forceinline__ float2 f2(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }

// Interval weights of two thick intervals (d >= 0.1 in both components): the arithmetic of the
// d >= 0.1 branch of lin_weights, e0 / d formed once and w1 = 1 - e0 / d, w0 = e0 / d - e^-d.
__device__ __forceinline__ void lin_weights_thick2(float2 d, float2 &ex, float2 &w0, float2 &w1)
{
    const float2 m = mul2(d, f2(-1.4426950408889634f));
    float y0, y1, r0, r1;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y0) : "f"(m.x));
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y1) : "f"(m.y));
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r0) : "f"(d.x));
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r1) : "f"(d.y));
    ex = make_float2(y0, y1);
    const float2 e0 = fma2(ex, f2(-1.0f), f2(1.0f));
    const float2 q = mul2(e0, make_float2(r0, r1));
    w1 = fma2(q, f2(-1.0f), f2(1.0f));
    w0 = fma2(ex, f2(-1.0f), q);
}

// FP64 variant (used by the adjoint sweeps): series below d = 1e-3, truncation < 1e-19.
__device__ __forceinline__ void lin_weights(double d, double &ex, double &w0, double &w1)
{
    ex = exp(-d);
    if (d < 1e-3) {
        w1 = d * (0.5 + d * (-1.0 / 6.0 + d * (1.0 / 24.0 + d * (-1.0 / 120.0 + d * (1.0 / 720.0)))));
        w0 = d * (0.5 + d * (-1.0 / 3.0 + d * (1.0 / 8.0 + d * (-1.0 / 30.0 + d * (1.0 / 144.0)))));
    } else {
        const double e0 = -expm1(-d);
        w1 = (d - e0) / d;
        w0 = e0 / d - ex;
    }
}

__device__ __forceinline__ void lin_weights_deriv(double d, double ex, double &dex, double &dw0,
                                                  double &dw1)
{
    dex = -ex;
    if (d < 1e-3) {
        dw1 = 0.5 + d * (-1.0 / 3.0 + d * (1.0 / 8.0 + d * (-1.0 / 30.0 + d * (1.0 / 144.0))));
        dw0 = 0.5 + d * (-2.0 / 3.0 + d * (3.0 / 8.0 + d * (-2.0 / 15.0 + d * (5.0 / 144.0))));
    } else {
        const double e0 = -expm1(-d);
        dw1 = (e0 - d * ex) / (d * d);
        dw0 = ex - dw1;
    }
}

// d/dd of (e^-d, w0, w1), for the adjoint sweeps.
__device__ __forceinline__ void lin_weights_deriv(float d, float ex, float &dex, float &dw0,
                                                  float &dw1)
{
    dex = -ex;
    if (d < 0.1f) {
        // dw1/dd = 1/2 - d/3 + d^2/8 - d^3/30 + d^4/144
        dw1 = 0.5f + d * (-1.0f / 3.0f + d * (1.0f / 8.0f + d * (-1.0f / 30.0f + d * (1.0f / 144.0f))));
        // dw0/dd = e^-d - dw1/dd = 1/2 - 2d/3 + 3d^2/8 - 2d^3/15 + 5d^4/144
        dw0 = 0.5f + d * (-2.0f / 3.0f + d * (3.0f / 8.0f + d * (-2.0f / 15.0f +
                                                                d * (5.0f / 144.0f))));
    } else {
        float r = __frcp_rn(d);
        float e0 = 1.0f - ex;
        dw1 = (e0 - d * ex) * r * r;
        dw0 = ex - dw1;
    }
}

__device__ __forceinline__ void flag_error(unsigned *err, unsigned bit)
{
    if (err) atomicOr(err, bit);
}

}  // namespace rt
