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

// ga += sum_k A[k] grad Y_k,  gb += sum_k B[k] grad Y_k  (gradient of the polynomial)
template <typename real>
__device__ __forceinline__ void sh_grad2(real x, real y, real z, const real* A, const real* B,
                                         real* ga, real* gb)
{
    const real x2 = x * x, y2 = y * y, z2 = z * z, x3 = x2 * x, y3 = y2 * y, z3 = z2 * z;
    const real x4 = x2 * x2, y4 = y2 * y2, z4 = z2 * z2;
    (void)x3; (void)y3; (void)z3; (void)x4; (void)y4; (void)z4;
    { const real t = real(0.48860251190291992); ga[1] += A[0] * t; gb[1] += B[0] * t; }
    { const real t = real(0.48860251190291992); ga[2] += A[1] * t; gb[2] += B[1] * t; }
    { const real t = real(0.48860251190291992); ga[0] += A[2] * t; gb[0] += B[2] * t; }
    { const real t = real(1.0925484305920791)*y; ga[0] += A[3] * t; gb[0] += B[3] * t; }
    { const real t = real(1.0925484305920791)*x; ga[1] += A[3] * t; gb[1] += B[3] * t; }
    { const real t = real(1.0925484305920791)*z; ga[1] += A[4] * t; gb[1] += B[4] * t; }
    { const real t = real(1.0925484305920791)*y; ga[2] += A[4] * t; gb[2] += B[4] * t; }
    { const real t = -real(0.63078313050504001)*x; ga[0] += A[5] * t; gb[0] += B[5] * t; }
    { const real t = -real(0.63078313050504001)*y; ga[1] += A[5] * t; gb[1] += B[5] * t; }
    { const real t = real(1.26156626101008)*z; ga[2] += A[5] * t; gb[2] += B[5] * t; }
    { const real t = real(1.0925484305920791)*z; ga[0] += A[6] * t; gb[0] += B[6] * t; }
    { const real t = real(1.0925484305920791)*x; ga[2] += A[6] * t; gb[2] += B[6] * t; }
    { const real t = real(1.0925484305920791)*x; ga[0] += A[7] * t; gb[0] += B[7] * t; }
    { const real t = -real(1.0925484305920791)*y; ga[1] += A[7] * t; gb[1] += B[7] * t; }
    { const real t = real(3.5402615395598611)*x*y; ga[0] += A[8] * t; gb[0] += B[8] * t; }
    { const real t = real(1.7701307697799305)*x2 - real(1.7701307697799305)*y2; ga[1] += A[8] * t; gb[1] += B[8] * t; }
    { const real t = real(2.8906114426405541)*y*z; ga[0] += A[9] * t; gb[0] += B[9] * t; }
    { const real t = real(2.8906114426405541)*x*z; ga[1] += A[9] * t; gb[1] += B[9] * t; }
    { const real t = real(2.8906114426405541)*x*y; ga[2] += A[9] * t; gb[2] += B[9] * t; }
    { const real t = -real(0.91409159892893147)*x*y; ga[0] += A[10] * t; gb[0] += B[10] * t; }
    { const real t = -real(0.45704579946446574)*x2 - real(1.3711373983933972)*y2 + real(1.8281831978578629)*z2; ga[1] += A[10] * t; gb[1] += B[10] * t; }
    { const real t = real(3.6563663957157259)*y*z; ga[2] += A[10] * t; gb[2] += B[10] * t; }
    { const real t = -real(2.2390579955406923)*x*z; ga[0] += A[11] * t; gb[0] += B[11] * t; }
    { const real t = -real(2.2390579955406923)*y*z; ga[1] += A[11] * t; gb[1] += B[11] * t; }
    { const real t = -real(1.1195289977703462)*x2 - real(1.1195289977703462)*y2 + real(2.2390579955406923)*z2; ga[2] += A[11] * t; gb[2] += B[11] * t; }
    { const real t = -real(1.3711373983933972)*x2 - real(0.45704579946446574)*y2 + real(1.8281831978578629)*z2; ga[0] += A[12] * t; gb[0] += B[12] * t; }
    { const real t = -real(0.91409159892893147)*x*y; ga[1] += A[12] * t; gb[1] += B[12] * t; }
    { const real t = real(3.6563663957157259)*x*z; ga[2] += A[12] * t; gb[2] += B[12] * t; }
    { const real t = real(2.8906114426405541)*x*z; ga[0] += A[13] * t; gb[0] += B[13] * t; }
    { const real t = -real(2.8906114426405541)*y*z; ga[1] += A[13] * t; gb[1] += B[13] * t; }
    { const real t = real(1.445305721320277)*x2 - real(1.445305721320277)*y2; ga[2] += A[13] * t; gb[2] += B[13] * t; }
    { const real t = real(1.7701307697799305)*x2 - real(1.7701307697799305)*y2; ga[0] += A[14] * t; gb[0] += B[14] * t; }
    { const real t = -real(3.5402615395598611)*x*y; ga[1] += A[14] * t; gb[1] += B[14] * t; }
    { const real t = real(7.5100288253901136)*x2*y - real(2.5033429417967045)*y3; ga[0] += A[15] * t; gb[0] += B[15] * t; }
    { const real t = real(2.5033429417967045)*x3 - real(7.5100288253901136)*x*y2; ga[1] += A[15] * t; gb[1] += B[15] * t; }
    { const real t = real(10.620784618679583)*x*y*z; ga[0] += A[16] * t; gb[0] += B[16] * t; }
    { const real t = real(5.3103923093397916)*x2*z - real(5.3103923093397916)*y2*z; ga[1] += A[16] * t; gb[1] += B[16] * t; }
    { const real t = real(5.3103923093397916)*x2*y - real(1.7701307697799305)*y3; ga[2] += A[16] * t; gb[2] += B[16] * t; }
    { const real t = -real(2.8385240872726801)*x2*y - real(0.94617469575756002)*y3 + real(5.6770481745453601)*y*z2; ga[0] += A[17] * t; gb[0] += B[17] * t; }
    { const real t = -real(0.94617469575756002)*x3 - real(2.8385240872726801)*x*y2 + real(5.6770481745453601)*x*z2; ga[1] += A[17] * t; gb[1] += B[17] * t; }
    { const real t = real(11.35409634909072)*x*y*z; ga[2] += A[17] * t; gb[2] += B[17] * t; }
    { const real t = -real(4.014279261343735)*x*y*z; ga[0] += A[18] * t; gb[0] += B[18] * t; }
    { const real t = -real(2.0071396306718675)*x2*z - real(6.0214188920156025)*y2*z + real(2.6761861742291567)*z3; ga[1] += A[18] * t; gb[1] += B[18] * t; }
    { const real t = -real(2.0071396306718675)*x2*y - real(2.0071396306718675)*y3 + real(8.02855852268747)*y*z2; ga[2] += A[18] * t; gb[2] += B[18] * t; }
    { const real t = real(1.2694265629824516)*x3 + real(1.2694265629824516)*x*y2 - real(5.0777062519298066)*x*z2; ga[0] += A[19] * t; gb[0] += B[19] * t; }
    { const real t = real(1.2694265629824516)*x2*y + real(1.2694265629824516)*y3 - real(5.0777062519298066)*y*z2; ga[1] += A[19] * t; gb[1] += B[19] * t; }
    { const real t = -real(5.0777062519298066)*x2*z - real(5.0777062519298066)*y2*z + real(3.3851375012865377)*z3; ga[2] += A[19] * t; gb[2] += B[19] * t; }
    { const real t = -real(6.0214188920156025)*x2*z - real(2.0071396306718675)*y2*z + real(2.6761861742291567)*z3; ga[0] += A[20] * t; gb[0] += B[20] * t; }
    { const real t = -real(4.014279261343735)*x*y*z; ga[1] += A[20] * t; gb[1] += B[20] * t; }
    { const real t = -real(2.0071396306718675)*x3 - real(2.0071396306718675)*x*y2 + real(8.02855852268747)*x*z2; ga[2] += A[20] * t; gb[2] += B[20] * t; }
    { const real t = -real(1.89234939151512)*x3 + real(5.6770481745453601)*x*z2; ga[0] += A[21] * t; gb[0] += B[21] * t; }
    { const real t = real(1.89234939151512)*y3 - real(5.6770481745453601)*y*z2; ga[1] += A[21] * t; gb[1] += B[21] * t; }
    { const real t = real(5.6770481745453601)*x2*z - real(5.6770481745453601)*y2*z; ga[2] += A[21] * t; gb[2] += B[21] * t; }
    { const real t = real(5.3103923093397916)*x2*z - real(5.3103923093397916)*y2*z; ga[0] += A[22] * t; gb[0] += B[22] * t; }
    { const real t = -real(10.620784618679583)*x*y*z; ga[1] += A[22] * t; gb[1] += B[22] * t; }
    { const real t = real(1.7701307697799305)*x3 - real(5.3103923093397916)*x*y2; ga[2] += A[22] * t; gb[2] += B[22] * t; }
    { const real t = real(2.5033429417967045)*x3 - real(7.5100288253901136)*x*y2; ga[0] += A[23] * t; gb[0] += B[23] * t; }
    { const real t = -real(7.5100288253901136)*x2*y + real(2.5033429417967045)*y3; ga[1] += A[23] * t; gb[1] += B[23] * t; }
}

template <typename real>
struct ShMono {
    real x, y, z, x2, y2, z2, x3, y3, z3, x4, y4, z4;
};

template <typename real>
__device__ __forceinline__ ShMono<real> sh_mono(real x, real y, real z)
{
    ShMono<real> m;
    m.x = x; m.y = y; m.z = z;
    m.x2 = x * x; m.y2 = y * y; m.z2 = z * z;
    m.x3 = m.x2 * x; m.y3 = m.y2 * y; m.z3 = m.z2 * z;
    m.x4 = m.x2 * m.x2; m.y4 = m.y2 * m.y2; m.z4 = m.z2 * m.z2;
    return m;
}

template <typename real>
__device__ __forceinline__ void sh_val_grad(int k, const ShMono<real>& m, real& v, real& gx, real& gy,
                                            real& gz)
{
    const real x = m.x, y = m.y, z = m.z, x2 = m.x2, y2 = m.y2, z2 = m.z2;
    const real x3 = m.x3, y3 = m.y3, z3 = m.z3, x4 = m.x4, y4 = m.y4, z4 = m.z4;
    (void)x3; (void)y3; (void)z3; (void)x4; (void)y4; (void)z4;
    switch (k) {
    case 0:
        v = real(0.48860251190291992)*y;
        gx = real(0);
        gy = real(0.48860251190291992);
        gz = real(0);
        break;
    case 1:
        v = real(0.48860251190291992)*z;
        gx = real(0);
        gy = real(0);
        gz = real(0.48860251190291992);
        break;
    case 2:
        v = real(0.48860251190291992)*x;
        gx = real(0.48860251190291992);
        gy = real(0);
        gz = real(0);
        break;
    case 3:
        v = real(1.0925484305920791)*x*y;
        gx = real(1.0925484305920791)*y;
        gy = real(1.0925484305920791)*x;
        gz = real(0);
        break;
    case 4:
        v = real(1.0925484305920791)*y*z;
        gx = real(0);
        gy = real(1.0925484305920791)*z;
        gz = real(1.0925484305920791)*y;
        break;
    case 5:
        v = -real(0.31539156525252001)*x2 - real(0.31539156525252001)*y2 + real(0.63078313050504001)*z2;
        gx = -real(0.63078313050504001)*x;
        gy = -real(0.63078313050504001)*y;
        gz = real(1.26156626101008)*z;
        break;
    case 6:
        v = real(1.0925484305920791)*x*z;
        gx = real(1.0925484305920791)*z;
        gy = real(0);
        gz = real(1.0925484305920791)*x;
        break;
    case 7:
        v = real(0.54627421529603954)*x2 - real(0.54627421529603954)*y2;
        gx = real(1.0925484305920791)*x;
        gy = -real(1.0925484305920791)*y;
        gz = real(0);
        break;
    case 8:
        v = real(1.7701307697799305)*x2*y - real(0.59004358992664351)*y3;
        gx = real(3.5402615395598611)*x*y;
        gy = real(1.7701307697799305)*x2 - real(1.7701307697799305)*y2;
        gz = real(0);
        break;
    case 9:
        v = real(2.8906114426405541)*x*y*z;
        gx = real(2.8906114426405541)*y*z;
        gy = real(2.8906114426405541)*x*z;
        gz = real(2.8906114426405541)*x*y;
        break;
    case 10:
        v = -real(0.45704579946446574)*x2*y - real(0.45704579946446574)*y3 + real(1.8281831978578629)*y*z2;
        gx = -real(0.91409159892893147)*x*y;
        gy = -real(0.45704579946446574)*x2 - real(1.3711373983933972)*y2 + real(1.8281831978578629)*z2;
        gz = real(3.6563663957157259)*y*z;
        break;
    case 11:
        v = -real(1.1195289977703462)*x2*z - real(1.1195289977703462)*y2*z + real(0.74635266518023078)*z3;
        gx = -real(2.2390579955406923)*x*z;
        gy = -real(2.2390579955406923)*y*z;
        gz = -real(1.1195289977703462)*x2 - real(1.1195289977703462)*y2 + real(2.2390579955406923)*z2;
        break;
    case 12:
        v = -real(0.45704579946446574)*x3 - real(0.45704579946446574)*x*y2 + real(1.8281831978578629)*x*z2;
        gx = -real(1.3711373983933972)*x2 - real(0.45704579946446574)*y2 + real(1.8281831978578629)*z2;
        gy = -real(0.91409159892893147)*x*y;
        gz = real(3.6563663957157259)*x*z;
        break;
    case 13:
        v = real(1.445305721320277)*x2*z - real(1.445305721320277)*y2*z;
        gx = real(2.8906114426405541)*x*z;
        gy = -real(2.8906114426405541)*y*z;
        gz = real(1.445305721320277)*x2 - real(1.445305721320277)*y2;
        break;
    case 14:
        v = real(0.59004358992664351)*x3 - real(1.7701307697799305)*x*y2;
        gx = real(1.7701307697799305)*x2 - real(1.7701307697799305)*y2;
        gy = -real(3.5402615395598611)*x*y;
        gz = real(0);
        break;
    case 15:
        v = real(2.5033429417967045)*x3*y - real(2.5033429417967045)*x*y3;
        gx = real(7.5100288253901136)*x2*y - real(2.5033429417967045)*y3;
        gy = real(2.5033429417967045)*x3 - real(7.5100288253901136)*x*y2;
        gz = real(0);
        break;
    case 16:
        v = real(5.3103923093397916)*x2*y*z - real(1.7701307697799305)*y3*z;
        gx = real(10.620784618679583)*x*y*z;
        gy = real(5.3103923093397916)*x2*z - real(5.3103923093397916)*y2*z;
        gz = real(5.3103923093397916)*x2*y - real(1.7701307697799305)*y3;
        break;
    case 17:
        v = -real(0.94617469575756002)*x3*y - real(0.94617469575756002)*x*y3 + real(5.6770481745453601)*x*y*z2;
        gx = -real(2.8385240872726801)*x2*y - real(0.94617469575756002)*y3 + real(5.6770481745453601)*y*z2;
        gy = -real(0.94617469575756002)*x3 - real(2.8385240872726801)*x*y2 + real(5.6770481745453601)*x*z2;
        gz = real(11.35409634909072)*x*y*z;
        break;
    case 18:
        v = -real(2.0071396306718675)*x2*y*z - real(2.0071396306718675)*y3*z + real(2.6761861742291567)*y*z3;
        gx = -real(4.014279261343735)*x*y*z;
        gy = -real(2.0071396306718675)*x2*z - real(6.0214188920156025)*y2*z + real(2.6761861742291567)*z3;
        gz = -real(2.0071396306718675)*x2*y - real(2.0071396306718675)*y3 + real(8.02855852268747)*y*z2;
        break;
    case 19:
        v = real(0.31735664074561291)*x4 + real(0.63471328149122582)*x2*y2 - real(2.5388531259649033)*x2*z2 + real(0.31735664074561291)*y4 - real(2.5388531259649033)*y2*z2 + real(0.84628437532163443)*z4;
        gx = real(1.2694265629824516)*x3 + real(1.2694265629824516)*x*y2 - real(5.0777062519298066)*x*z2;
        gy = real(1.2694265629824516)*x2*y + real(1.2694265629824516)*y3 - real(5.0777062519298066)*y*z2;
        gz = -real(5.0777062519298066)*x2*z - real(5.0777062519298066)*y2*z + real(3.3851375012865377)*z3;
        break;
    case 20:
        v = -real(2.0071396306718675)*x3*z - real(2.0071396306718675)*x*y2*z + real(2.6761861742291567)*x*z3;
        gx = -real(6.0214188920156025)*x2*z - real(2.0071396306718675)*y2*z + real(2.6761861742291567)*z3;
        gy = -real(4.014279261343735)*x*y*z;
        gz = -real(2.0071396306718675)*x3 - real(2.0071396306718675)*x*y2 + real(8.02855852268747)*x*z2;
        break;
    case 21:
        v = -real(0.47308734787878001)*x4 + real(2.8385240872726801)*x2*z2 + real(0.47308734787878001)*y4 - real(2.8385240872726801)*y2*z2;
        gx = -real(1.89234939151512)*x3 + real(5.6770481745453601)*x*z2;
        gy = real(1.89234939151512)*y3 - real(5.6770481745453601)*y*z2;
        gz = real(5.6770481745453601)*x2*z - real(5.6770481745453601)*y2*z;
        break;
    case 22:
        v = real(1.7701307697799305)*x3*z - real(5.3103923093397916)*x*y2*z;
        gx = real(5.3103923093397916)*x2*z - real(5.3103923093397916)*y2*z;
        gy = -real(10.620784618679583)*x*y*z;
        gz = real(1.7701307697799305)*x3 - real(5.3103923093397916)*x*y2;
        break;
    case 23:
        v = real(0.62583573544917613)*x4 - real(3.7550144126950568)*x2*y2 + real(0.62583573544917613)*y4;
        gx = real(2.5033429417967045)*x3 - real(7.5100288253901136)*x*y2;
        gy = -real(7.5100288253901136)*x2*y + real(2.5033429417967045)*y3;
        gz = real(0);
        break;
    default:
        v = gx = gy = gz = real(0);
    }
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
