// Generated by gen_sh.py -- real orthonormal spherical harmonics, l = 1..4.
// Index k = l*l - 1 + (m + l); each Y_k is a homogeneous harmonic polynomial of
// degree l in the components of the unit vector (x, y, z).
#pragma once

template <typename real>
__device__ __forceinline__ void sh_eval(real x, real y, real z, real* Y)
{
    const real x2 = x * x, y2 = y * y, z2 = z * z, x3 = x2 * x, y3 = y2 * y, z3 = z2 * z;
    const real x4 = x2 * x2, y4 = y2 * y2, z4 = z2 * z2;
    (void)x3; (void)y3; (void)z3; (void)x4; (void)y4; (void)z4;
    Y[0] = real(0.48860251190291992)*y;
    Y[1] = real(0.48860251190291992)*z;
    Y[2] = real(0.48860251190291992)*x;
    Y[3] = real(1.0925484305920791)*x*y;
    Y[4] = real(1.0925484305920791)*y*z;
    Y[5] = -real(0.31539156525252001)*x2 - real(0.31539156525252001)*y2 + real(0.63078313050504001)*z2;
    Y[6] = real(1.0925484305920791)*x*z;
    Y[7] = real(0.54627421529603954)*x2 - real(0.54627421529603954)*y2;
    Y[8] = real(1.7701307697799305)*x2*y - real(0.59004358992664351)*y3;
    Y[9] = real(2.8906114426405541)*x*y*z;
    Y[10] = -real(0.45704579946446574)*x2*y - real(0.45704579946446574)*y3 + real(1.8281831978578629)*y*z2;
    Y[11] = -real(1.1195289977703462)*x2*z - real(1.1195289977703462)*y2*z + real(0.74635266518023078)*z3;
    Y[12] = -real(0.45704579946446574)*x3 - real(0.45704579946446574)*x*y2 + real(1.8281831978578629)*x*z2;
    Y[13] = real(1.445305721320277)*x2*z - real(1.445305721320277)*y2*z;
    Y[14] = real(0.59004358992664351)*x3 - real(1.7701307697799305)*x*y2;
    Y[15] = real(2.5033429417967045)*x3*y - real(2.5033429417967045)*x*y3;
    Y[16] = real(5.3103923093397916)*x2*y*z - real(1.7701307697799305)*y3*z;
    Y[17] = -real(0.94617469575756002)*x3*y - real(0.94617469575756002)*x*y3 + real(5.6770481745453601)*x*y*z2;
    Y[18] = -real(2.0071396306718675)*x2*y*z - real(2.0071396306718675)*y3*z + real(2.6761861742291567)*y*z3;
    Y[19] = real(0.31735664074561291)*x4 + real(0.63471328149122582)*x2*y2 - real(2.5388531259649033)*x2*z2 + real(0.31735664074561291)*y4 - real(2.5388531259649033)*y2*z2 + real(0.84628437532163443)*z4;
    Y[20] = -real(2.0071396306718675)*x3*z - real(2.0071396306718675)*x*y2*z + real(2.6761861742291567)*x*z3;
    Y[21] = -real(0.47308734787878001)*x4 + real(2.8385240872726801)*x2*z2 + real(0.47308734787878001)*y4 - real(2.8385240872726801)*y2*z2;
    Y[22] = real(1.7701307697799305)*x3*z - real(5.3103923093397916)*x*y2*z;
    Y[23] = real(0.62583573544917613)*x4 - real(3.7550144126950568)*x2*y2 + real(0.62583573544917613)*y4;
}

// Sphere-reduced form: with z^2 = 1 - x^2 - y^2 each Y_k equals A_k(x, y) + z B_k(x, y)
// on the unit sphere, deg A_k <= 4, deg B_k <= 3 (the two forms have equal values and
// equal surface gradients there).  A 25-entry coefficient vector holds block A
// (x^a y^b, a + b <= 4) at sh_red_a(a) + b and block B (z x^a y^b, a + b <= 3) at
// sh_red_b(a) + b.
constexpr int kShRed = 25;
__host__ __device__ constexpr int sh_red_a(int a) { return a * 5 - a * (a - 1) / 2; }
__host__ __device__ constexpr int sh_red_b(int a) { return 15 + a * 4 - a * (a - 1) / 2; }

// psi = sum_k phi[k] (reduced form of Y_k): the reduced coefficients of sum_k phi[k] Y_k
template <typename real>
__device__ __forceinline__ void sh_reduce(const real* phi, real* psi)
{
    psi[0] = real(0.63078313050504001) * phi[5] + real(0.84628437532163443) * phi[19];
    psi[1] = real(0.48860251190291992) * phi[0] + real(1.8281831978578629) * phi[10];
    psi[2] = real(-0.94617469575756002) * phi[5] + real(-0.54627421529603954) * phi[7] + real(-4.2314218766081722) * phi[19] + real(-2.8385240872726801) * phi[21];
    psi[3] = real(-0.59004358992664351) * phi[8] + real(-2.2852289973223287) * phi[10];
    psi[4] = real(3.7024941420321506) * phi[19] + real(3.3116114351514601) * phi[21] + real(0.62583573544917613) * phi[23];
    psi[5] = real(0.48860251190291992) * phi[2] + real(1.8281831978578629) * phi[12];
    psi[6] = real(1.0925484305920791) * phi[3] + real(5.6770481745453601) * phi[17];
    psi[7] = real(-2.2852289973223287) * phi[12] + real(-1.7701307697799305) * phi[14];
    psi[8] = real(-2.5033429417967045) * phi[15] + real(-6.6232228703029201) * phi[17];
    psi[9] = real(-0.94617469575756002) * phi[5] + real(0.54627421529603954) * phi[7] + real(-4.2314218766081722) * phi[19] + real(2.8385240872726801) * phi[21];
    psi[10] = real(1.7701307697799305) * phi[8] + real(-2.2852289973223287) * phi[10];
    psi[11] = real(7.4049882840643013) * phi[19] + real(-3.7550144126950568) * phi[23];
    psi[12] = real(-2.2852289973223287) * phi[12] + real(0.59004358992664351) * phi[14];
    psi[13] = real(2.5033429417967045) * phi[15] + real(-6.6232228703029201) * phi[17];
    psi[14] = real(3.7024941420321506) * phi[19] + real(-3.3116114351514601) * phi[21] + real(0.62583573544917613) * phi[23];
    psi[15] = real(0.48860251190291992) * phi[1] + real(0.74635266518023078) * phi[11];
    psi[16] = real(1.0925484305920791) * phi[4] + real(2.6761861742291567) * phi[18];
    psi[17] = real(-1.8658816629505770) * phi[11] + real(-1.4453057213202770) * phi[13];
    psi[18] = real(-1.7701307697799305) * phi[16] + real(-4.6833258049010242) * phi[18];
    psi[19] = real(1.0925484305920791) * phi[6] + real(2.6761861742291567) * phi[20];
    psi[20] = real(2.8906114426405541) * phi[9];
    psi[21] = real(-4.6833258049010242) * phi[20] + real(-5.3103923093397916) * phi[22];
    psi[22] = real(-1.8658816629505770) * phi[11] + real(1.4453057213202770) * phi[13];
    psi[23] = real(5.3103923093397916) * phi[16] + real(-4.6833258049010242) * phi[18];
    psi[24] = real(-4.6833258049010242) * phi[20] + real(1.7701307697799305) * phi[22];
}
