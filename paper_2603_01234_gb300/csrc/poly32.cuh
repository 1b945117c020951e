// Generated by gen_poly32.py -- do not edit.
// FP32 cosine cutoff (Eq. 8): with y = r / r_c - 1/2 and z = y^2,
//   f_c / 2 = 1/4 - y P(z),   f_c' / 2 = -Q(z) / r_c.
// Least-squares fits at Chebyshev nodes, coefficients fixed one at a time in FP32.
// Emulated FP32 error: f_c/2 mean signed +1.0e-10, max 3.8e-08;
//   Q mean signed -9.6e-10, max 1.2e-07 (mean weighted by r^2).
// tanh(x) = x + x^3 R(x^2) on [-1, 1], fitted the same way; emulated FP32 error:
//   max 5.1e-08, largest mean signed over eighths of [0, 1] 1.6e-10.
#pragma once

namespace nep {

__device__ __forceinline__ float cut_p(float z)
{
    return fmaf(fmaf(fmaf(fmaf(0.019246120005846024f, z, -0.14947454631328583f), z, 0.6374998688697815f), z, -1.2919260263442993f), z, 0.7853981256484985f);
}

__device__ __forceinline__ float cut_q(float z)
{
    return fmaf(fmaf(fmaf(fmaf(0.17255288362503052f, z, -1.046057939529419f), z, 3.187469482421875f), z, -3.875777244567871f), z, 0.7853981256484985f);
}

__device__ __forceinline__ float tanh_r_poly(float z)
{
    return fmaf(fmaf(fmaf(fmaf(fmaf(fmaf(fmaf(0.00011460282257758081f, z, -0.0008126287721097469f), z, 0.0030302144587039948f), z, -0.008552024140954018f), z, 0.021763261407613754f), z, -0.05394722521305084f), z, 0.13333120942115784f), z, -0.33333325386047363f);
}

}  // namespace nep
