// Descriptor + network kernel and force + virial kernel (Eq. 1-8, 15, 16).
//
// k_descriptor (one thread per sorted particle i):
//   radial   q_n   = sum_j g_n(r_ij)                              (Eq. 3, 6-8)
//   angular  A_nlm = sum_j g_n(r_ij) Y_lm(u_ij), q_nl = sum_m A^2  (Eq. 4-5)
//            with real orthonormal Y_lm (for real g_n, sum_m (-1)^m A_m A_-m of
//            the complex harmonics equals sum_m A_m^2 of the real ones)
//   network  U_i (Eq. 2) and dU_i/dq
//   stores   U_i;  e_i^t[k] = sum_n dU_i/dq_n c^{t_i t}_{nk} for every partner type t
//            (the radial gradient folded into the basis: dU_i/dr_ij|radial =
//            sum_k e_i^{t_j}[k] f_k'(r_ij) u_ij);  Phi_nlm = dU_i/dA_nlm = 2 dU_i/dq_nl A_nlm
//
// Forces and virials (one thread per sorted particle i), with
//   F_i = sum_j (f_ij - f_ji),   W_i = sum_j r_ij (x) f_ji   (Eq. 15),
// f_ij = dU_i/dr_ij, and E = sum U_i, W = sum W_i reduced in FP64 (Eq. 1, 16) by
// a deterministic last-block pass:
//   FP32  k_descriptor also evaluates the angular pairs, in scatter form, from
//         Phi_i while it is in registers (Phi never reaches memory): F_i keeps
//         f_ij, and -f_ij (and W_j's term) go to j through 64-bit fixed-point
//         atomic adds (order-independent sums); k_force_radial then takes the
//         radial pairs in gather form (f_ij and f_ji from i's and j's stored
//         gradient vectors), adds the accumulated angular part and writes the
//         outputs
//   FP64  k_descriptor stores the sphere-reduced form of Phi; k_force takes both
//         kinds of pair in gather form, no atomics
//
// Angular pair gradient.  For A = g(r) Y(u), u = r/|r|:
//   dA/dr = g' Y(u) u + (g / r) (grad Y(u) - (u . grad Y(u)) u),
// in which only the surface gradient of Y enters.  Both forms evaluate
// P_n = sum_lm Phi_nlm Y_lm through its sphere-reduced polynomial (sh_reduce,
// sh_red_eval), which has P_n's values and surface gradients on the unit sphere;
// the reverse pair is the same evaluation at -u with j's coefficients.
#include <cuda_bf16.h>

#include "nep_common.cuh"
#include "poly32.cuh"
#include "sh_poly.cuh"
static_assert(kShRed == nep::kPsiComp, "the FP64 form's coefficient buffer holds the sphere-reduced form");

namespace nep {

__host__ __device__ constexpr int l_of(int k) { return k < 3 ? 1 : (k < 8 ? 2 : (k < 15 ? 3 : 4)); }
constexpr int kNLM = 24;
// The FP32 kernels are compiled for 2 and for 3 resident blocks per SM (which caps
// registers per thread); the runtime picks one per handle (autotuned).

// The cutoff of Eq. 8 halved, f_c / 2, and its derivative halved, f_c' / 2, at
// x = r / r_c in [0, 1].  FP32 evaluates the polynomials of poly32.cuh
// (the hardware sine and cosine err by about 1e-7 with a consistent sign, which
// summed over pairs biases the energy); FP64 uses the accurate sincospi.
__device__ __forceinline__ float cut_half(float x)
{
    const float y = x - 0.5f;
    return fmaf(-y, cut_p(y * y), 0.25f);
}
__device__ __forceinline__ double cut_half(double x)
{
    return 0.25 + 0.25 * cospi(x);
}
__device__ __forceinline__ void cut_half_d(float x, float inv_rc, float* hf, float* hdf)
{
    const float y = x - 0.5f;
    const float z = y * y;
    *hf = fmaf(-y, cut_p(z), 0.25f);
    *hdf = -cut_q(z) * inv_rc;
}
__device__ __forceinline__ void cut_half_d(double x, double inv_rc, double* hf, double* hdf)
{
    double s, c;
    sincospi(x, &s, &c);
    *hf = 0.25 + 0.25 * c;
    *hdf = (-0.25 * 3.14159265358979323846) * inv_rc * s;
}

// Chebyshev basis f_k(r) of Eq. 7 with the cutoff of Eq. 8, k = 0..K-1, by the
// three-term recurrence T_{k+1} = 2 x T_k - T_{k-1}.
// x = r / r_c from the inverse cutoff and its FP32 rounding residual (FP64: exact enough)
__device__ __forceinline__ float scaled_r(float r, float inv_rc, float inv_lo) { return fmaf(r, inv_lo, r * inv_rc); }
__device__ __forceinline__ double scaled_r(double r, double inv_rc, double) { return r * inv_rc; }

template <typename real, int K>
__device__ __forceinline__ void basis(real r, real inv_rc, real inv_lo, real* f)
{
    const real xr = scaled_r(r, inv_rc, inv_lo);
    const real hf = cut_half(xr);  // f_c / 2
    const real s = xr - real(1);
    const real x = real(2) * s * s - real(1);
    const real x2 = x + x;
    real t0 = real(1), t1 = x;
    f[0] = hf + hf;
    if (K > 1) f[1] = hf * x + hf;
#pragma unroll
    for (int k = 2; k < K; ++k) {
        const real t2 = x2 * t1 - t0;
        f[k] = hf * t2 + hf;  // (T_k + 1) f_c / 2
        t0 = t1;
        t1 = t2;
    }
}

// Pair sums of the basis, split as f_k = (f_c/2) T_k + f_c/2: acc[k] += (f_c/2) T_k
// and hs += f_c/2, so that sum_j f_k = acc[k] + hs (one FMA per term instead of a
// product and an add).
template <typename real, int K>
__device__ __forceinline__ void basis_acc(real r, real inv_rc, real inv_lo, real (&acc)[K], real& hs)
{
    const real xr = scaled_r(r, inv_rc, inv_lo);
    const real hf = cut_half(xr);  // f_c / 2
    const real s = xr - real(1);
    const real x = real(2) * s * s - real(1);
    const real x2 = x + x;
    real t0 = real(1), t1 = x;
    hs += hf;
    acc[0] += hf;
    if (K > 1) acc[1] = fma(hf, x, acc[1]);
#pragma unroll
    for (int k = 2; k < K; ++k) {
        const real t2 = x2 * t1 - t0;
        acc[k] = fma(hf, t2, acc[k]);
        t0 = t1;
        t1 = t2;
    }
}

// f_k and df_k/dr:  df_k = 1/2 [T_k'(x) x'(r) f_c + (T_k + 1) f_c'],
// with T'_{k+1} = 2 T_k + 2 x T'_k - T'_{k-1}.
template <typename real, int K>
__device__ __forceinline__ void basis_d(real r, real inv_rc, real inv_lo, real* f, real* df)
{
    const real xr = scaled_r(r, inv_rc, inv_lo);
    real hf, hdf;  // f_c / 2, f_c' / 2
    cut_half_d(xr, inv_rc, &hf, &hdf);
    const real s = xr - real(1);
    const real x = real(2) * s * s - real(1);
    const real hdx = real(4) * s * inv_rc * hf;                             // x'(r) f_c / 2
    const real x2 = x + x;
    real t0 = real(1), t1 = x, d0 = real(0), d1 = real(1);
    f[0] = hf + hf;
    df[0] = hdf + hdf;
    if (K > 1) {
        f[1] = hf * x + hf;
        df[1] = hdx + (hdf * x + hdf);
    }
#pragma unroll
    for (int k = 2; k < K; ++k) {
        const real t2 = x2 * t1 - t0;
        const real d2 = real(2) * t1 + (x2 * d1 - d0);
        f[k] = hf * t2 + hf;
        df[k] = d2 * hdx + (hdf * t2 + hdf);
        t0 = t1;
        t1 = t2;
        d0 = d1;
        d1 = d2;
    }
}

// Pair vector r_ij from i's and j's records and the entry's cell offset.
template <typename real>
__device__ __forceinline__ void pair_vec(const real* len, const PosRec<real>& ri, const PosRec<real>& rj, uint32_t e,
                                         real& dx, real& dy, real& dz)
{
    const uint32_t code = e >> kJBits;
    dx = (rj.x - ri.x) + (real)((int)(code & 7u) - 2) * len[0];
    dy = (rj.y - ri.y) + (real)((int)((code >> 3) & 7u) - 2) * len[1];
    dz = (rj.z - ri.z) + (real)((int)((code >> 6) & 7u) - 2) * len[2];
}

// Software-pipelined walk over one particle's neighbour list: the entries are
// loaded two iterations ahead and the neighbour's record one iteration ahead, so
// the dependent load chain (entry -> record) overlaps the previous pair's math.
template <typename real>
struct NbrWalk {
    const uint32_t* nl;  // &list[0][i]
    size_t stride;
    int cnt;
    const PosRec<real>* rec;
    uint32_t e0, e1;
    PosRec<real> r0;
    __device__ __forceinline__ NbrWalk(const uint32_t* list, int n, int i, int c, const PosRec<real>* recs)
        : nl(list + i), stride((size_t)n), cnt(c), rec(recs)
    {
        e0 = c > 0 ? nl[0] : 0u;
        e1 = c > 1 ? nl[stride] : 0u;
        r0 = rec[e0 & kJMask];  // index 0 is valid even for an empty list
    }
    // current entry and record, then advance the pipeline (s = current index)
    __device__ __forceinline__ void next(int s, uint32_t& e, PosRec<real>& rj)
    {
        e = e0;
        rj = r0;
        e0 = e1;
        e1 = (s + 2 < cnt) ? nl[(size_t)(s + 2) * stride] : 0u;
        r0 = rec[e0 & kJMask];
    }
};

// Walk over a column-major neighbour list whose entries are loaded 4 to 8 pairs
// ahead of use (the list is streamed from L2; a short loop body cannot hide that
// latency with a shallower prefetch).  body(entry) is called for every entry in order.
template <typename Body>
__device__ __forceinline__ void walk4(const uint32_t* nl, size_t stride, int cnt, Body&& body)
{
    auto ld = [&](int s) { return s < cnt ? nl[(size_t)s * stride] : 0u; };
    uint32_t q0 = ld(0), q1 = ld(1), q2 = ld(2), q3 = ld(3);
    int s = 0;
    for (; s + 4 <= cnt; s += 4) {
        const uint32_t a0 = q0, a1 = q1, a2 = q2, a3 = q3;
        q0 = ld(s + 4);
        q1 = ld(s + 5);
        q2 = ld(s + 6);
        q3 = ld(s + 7);
        body(a0);
        body(a1);
        body(a2);
        body(a3);
    }
    if (s < cnt) body(q0);
    if (s + 1 < cnt) body(q1);
    if (s + 2 < cnt) body(q2);
}

// walk4 generalised to groups of CH entries (CH = 4 or 8): the next group's
// entries are loaded while the current group is evaluated, so up to 2 CH entries
// (and CH pairs' neighbour loads) are in flight per thread.
template <int CH, typename Body>
__device__ __forceinline__ void walk_chunk(const uint32_t* nl, size_t stride, int cnt, Body&& body)
{
    auto ld = [&](int s) { return s < cnt ? nl[(size_t)s * stride] : 0u; };
    uint32_t q[CH];
#pragma unroll
    for (int u = 0; u < CH; ++u) q[u] = ld(u);
    int s = 0;
    for (; s + CH <= cnt; s += CH) {
        uint32_t cur[CH];
#pragma unroll
        for (int u = 0; u < CH; ++u) {
            cur[u] = q[u];
            q[u] = ld(s + CH + u);
        }
#pragma unroll
        for (int u = 0; u < CH; ++u) body(cur[u]);
    }
#pragma unroll
    for (int u = 0; u < CH - 1; ++u)
        if (s + u < cnt) body(q[u]);
}

// walk4 with the entry's position in its group of four passed as the second
// argument (0..3, a constant after unrolling), so that a body can keep four
// partial sums: each then grows to a quarter of the total, which cuts the FP32
// rounding of a long accumulation about four-fold at no extra instructions.
template <typename Body>
__device__ __forceinline__ void walk4p(const uint32_t* nl, size_t stride, int cnt, Body&& body)
{
    auto ld = [&](int s) { return s < cnt ? nl[(size_t)s * stride] : 0u; };
    uint32_t q0 = ld(0), q1 = ld(1), q2 = ld(2), q3 = ld(3);
    int s = 0;
    for (; s + 4 <= cnt; s += 4) {
        const uint32_t a0 = q0, a1 = q1, a2 = q2, a3 = q3;
        q0 = ld(s + 4);
        q1 = ld(s + 5);
        q2 = ld(s + 6);
        q3 = ld(s + 7);
        body(a0, 0);
        body(a1, 1);
        body(a2, 2);
        body(a3, 3);
    }
    if (s < cnt) body(q0, 0);
    if (s + 1 < cnt) body(q1, 1);
    if (s + 2 < cnt) body(q2, 2);
}

// 4 consecutive reals (16-byte aligned) into registers
__device__ __forceinline__ void load4(const float* p, float* o)
{
    const float4 v = *reinterpret_cast<const float4*>(p);
    o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
}
__device__ __forceinline__ void load4(const double* p, double* o)
{
    const double2 v0 = reinterpret_cast<const double2*>(p)[0], v1 = reinterpret_cast<const double2*>(p)[1];
    o[0] = v0.x; o[1] = v0.y; o[2] = v1.x; o[3] = v1.y;
}

template <typename real, int N>
__device__ __forceinline__ void loadN(const real* p, real* o)
{
#pragma unroll
    for (int k = 0; k + 3 < N; k += 4) load4(p + k, o + k);
#pragma unroll
    for (int k = N & ~3; k < N; ++k) o[k] = p[k];
}

// 1/sqrt(x): the hardware estimate refined by one Newton-Raphson step on
// f(y) = y^-2 - x, y' = y + y (1 - x y^2) / 2.  The estimate's error has a small
// consistent sign, which through |u| = |r| / r and the homogeneous harmonics would
// bias the angular descriptors; after the step the quadratic term is ~1e-14 and
// what remains is the (unsigned) rounding of y^2.
// A type pair's n x K coefficient table into registers.  A one-type model's single
// table starts on a 16-byte boundary and is read with vector loads; several types'
// tables sit at odd strides (bank spread) and are read as scalars.
template <typename real, int N>
__device__ __forceinline__ void load_coef(const real* c, bool aligned, real (&o)[N])
{
    if (aligned) {
        loadN<real, N>(c, o);
    } else {
#pragma unroll
        for (int q = 0; q < N; ++q) o[q] = c[q];
    }
}

__device__ __forceinline__ float rsqrt_r(float x)
{
    const float y = rsqrtf(x);
    const float e = fmaf(-x, y * y, 1.0f);
    return fmaf(0.5f * y, e, y);
}
__device__ __forceinline__ double rsqrt_r(double x) { return rsqrt(x); }

// tanh in FP32.  Each hidden unit's pre-activation keeps one sign over most
// particles, so an activation whose rounding error leans one way on part of its
// range biases every particle's energy alike; CUDA's tanhf does (about -9e-9 on
// [1/4, 1/2]).  Here: on |x| < 1 the odd polynomial of poly32.cuh (mean error below
// 2e-10 on every eighth of the range); beyond, (1 - e) / (1 + e) with
// e = exp(-2|x|), where no cancellation remains, divided through a reciprocal
// refined by one Newton-Raphson step.
__device__ __forceinline__ float tanh_r(float x)
{
    const float a = fabsf(x);
    if (a < 1.0f) {
        const float z = x * x;
        return fmaf(x * z, tanh_r_poly(z), x);
    }
    const float e = expf(-2.0f * a);
    const float d = 1.0f + e;
    float r = __fdividef(1.0f, d);
    r = fmaf(r, fmaf(-d, r, 1.0f), r);
    return copysignf((1.0f - e) * r, x);
}
__device__ __forceinline__ double tanh_r(double x) { return tanh(x); }

template <typename real>
__device__ __forceinline__ void stage_params(const real* __restrict__ src, real* dst, int count)
{
    for (int k = threadIdx.x; k < count; k += blockDim.x) dst[k] = src[k];
    __syncthreads();
}

// ---- the hidden layer (Eq. 2) on tensor cores with BF16 weights -----------------
// A warp evaluates the network of its 32 particles (one per lane) as
//   X = Q W0^T       (32 x ND by ND x H: the hidden pre-activations)
//   dQ = D W0        (32 x H by H x ND: dU/dq, D = w1 (1 - h^2))
// with mma.sync m16n8k16 (BF16 operands, FP32 accumulation).  W0 is rounded to
// BF16 once, on the host; each activation (Q, D) is split into a BF16 head and a
// BF16 tail (x = hi + lo, exact to about 2^-16 relative) and multiplied as two
// products, so the result is the FP32 evaluation of the model with BF16 weights
// and the forces stay the gradient of its energy.  Q is transposed into fragment
// order through a warp-private shared tile; the FP32 accumulators of X are exactly
// the A fragments of the D product, so D never leaves registers; dQ comes back to
// the lanes through the same tile.  Particles of a type other than t are masked
// out of type t's products.
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);  // .x (low half) = lo
    return *reinterpret_cast<uint32_t*>(&v);
}

// (x0, x1) as packed BF16 heads and packed BF16 tails: x = head + tail
__device__ __forceinline__ void split_bf16(float x0, float x1, uint32_t& head, uint32_t& tail)
{
    const __nv_bfloat16 h0 = __float2bfloat16_rn(x0), h1 = __float2bfloat16_rn(x1);
    head = pack_bf16(__bfloat162float(h0), __bfloat162float(h1));
    tail = pack_bf16(x0 - __bfloat162float(h0), x1 - __bfloat162float(h1));
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

template <int ND>
__device__ __forceinline__ void net_bf16(const float* P, const ParamLayout& off, int T, int H, int ti,
                                         const float (&q)[ND], float& U, float (&dq)[ND], unsigned char* scratch)
{
    constexpr int KPF = net_kpf(ND), SF = net_sf(ND), NDP = net_ndp(ND), KS = KPF / 16, NB = NDP / 8;
    constexpr int QT = 32 * (SF / 2);  // words of one Q tile
    const int HP = net_hp(H), SB = HP + 8;
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, g = lane >> 2, c = lane & 3;
    uint32_t* Qw = reinterpret_cast<uint32_t*>(scratch);  // [2 (head, tail)][32][SF / 2] words
#pragma unroll
    for (int v = 0; v < KPF / 2; ++v) {
        uint32_t hd, tl;
        split_bf16(2 * v < ND ? q[2 * v] : 0.f, 2 * v + 1 < ND ? q[2 * v + 1] : 0.f, hd, tl);
        Qw[lane * (SF / 2) + v] = hd;
        Qw[QT + lane * (SF / 2) + v] = tl;
    }
    __syncwarp();
    uint32_t af[2][2][KS][4];  // [head/tail][m tile][k step]
#pragma unroll
    for (int pt = 0; pt < 2; ++pt)
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
#pragma unroll
            for (int kk = 0; kk < KS; ++kk) {
                const int r0 = 16 * mt + g;
                const uint32_t* Qp = Qw + pt * QT;
                af[pt][mt][kk][0] = Qp[r0 * (SF / 2) + 8 * kk + c];
                af[pt][mt][kk][1] = Qp[(r0 + 8) * (SF / 2) + 8 * kk + c];
                af[pt][mt][kk][2] = Qp[r0 * (SF / 2) + 8 * kk + 4 + c];
                af[pt][mt][kk][3] = Qp[(r0 + 8) * (SF / 2) + 8 * kk + 4 + c];
            }
    __syncwarp();  // the tile is reused for dQ below
    int rt[2][2];  // types of this lane's fragment rows 16 mt + g + 8 h
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int h = 0; h < 2; ++h) rt[mt][h] = __shfl_sync(FULL, ti, 16 * mt + g + 8 * h);
    const uint16_t* W0f = reinterpret_cast<const uint16_t*>(P + off.w0f);
    const uint16_t* W0b = reinterpret_cast<const uint16_t*>(P + off.w0b);
    const float* b0 = P + off.b0;
    const float* w1 = P + off.w1;
    const float* b0l = P + off.b0l;  // FP32 rounding residuals of b0, w1 (b1 below)
    const float* w1l = P + off.w1l;
    float up[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
    float dacc[2][NB][4];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nb = 0; nb < NB; ++nb)
#pragma unroll
            for (int e = 0; e < 4; ++e) dacc[mt][nb][e] = 0.f;
    for (int ch = 0; ch < HP / 16; ++ch) {  // 16 hidden units at a time
        float x[2][2][4];
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
#pragma unroll
            for (int nl = 0; nl < 2; ++nl)
#pragma unroll
                for (int e = 0; e < 4; ++e) x[mt][nl][e] = 0.f;
        for (int t = 0; t < T; ++t) {
            if (T > 1 && !__any_sync(FULL, ti == t)) continue;
            const uint32_t* Wf = reinterpret_cast<const uint32_t*>(W0f + (size_t)t * HP * SF);
#pragma unroll
            for (int nl = 0; nl < 2; ++nl) {
                const int nrow = 16 * ch + 8 * nl + g;  // hidden unit of this lane's B column
                uint32_t b[KS][2];
#pragma unroll
                for (int kk = 0; kk < KS; ++kk) {
                    b[kk][0] = Wf[nrow * (SF / 2) + 8 * kk + c];
                    b[kk][1] = Wf[nrow * (SF / 2) + 8 * kk + 4 + c];
                }
#pragma unroll
                for (int mt = 0; mt < 2; ++mt) {
                    float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
                    for (int kk = 0; kk < KS; ++kk) {
                        mma_bf16(acc, af[1][mt][kk], b[kk][0], b[kk][1]);  // tails first (smaller)
                        mma_bf16(acc, af[0][mt][kk], b[kk][0], b[kk][1]);
                    }
#pragma unroll
                    for (int e = 0; e < 4; ++e)
                        if (T == 1 || rt[mt][e >> 1] == t) x[mt][nl][e] = acc[e];
                }
            }
        }
        // h = tanh(x - b0), the energy terms, and D = w1 (1 - h^2) in A-fragment order
        uint32_t ca[2][2][4];  // [head/tail][m tile]
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
            float d[2][4];
#pragma unroll
            for (int nl = 0; nl < 2; ++nl)
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int col = 16 * ch + 8 * nl + 2 * c + (e & 1);
                    const int t = rt[mt][e >> 1];
                    float coef = 0.f;
                    if (col < H) {
                        const float h = tanh_r(x[mt][nl][e] - b0[t * H + col] - b0l[t * H + col]);
                        const float w = w1[t * H + col];
                        up[mt][e >> 1] += w * h + w1l[t * H + col] * h;
                        coef = w * (1.f - h * h);
                    }
                    d[nl][e] = coef;
                }
            split_bf16(d[0][0], d[0][1], ca[0][mt][0], ca[1][mt][0]);
            split_bf16(d[0][2], d[0][3], ca[0][mt][1], ca[1][mt][1]);
            split_bf16(d[1][0], d[1][1], ca[0][mt][2], ca[1][mt][2]);
            split_bf16(d[1][2], d[1][3], ca[0][mt][3], ca[1][mt][3]);
        }
        for (int t = 0; t < T; ++t) {
            if (T > 1 && !__any_sync(FULL, ti == t)) continue;
            const uint32_t* Wb = reinterpret_cast<const uint32_t*>(W0b + (size_t)t * NDP * SB);
            uint32_t cm[2][2][4];
#pragma unroll
            for (int pt = 0; pt < 2; ++pt)
#pragma unroll
                for (int mt = 0; mt < 2; ++mt) {
                    const bool k0 = T == 1 || rt[mt][0] == t, k1 = T == 1 || rt[mt][1] == t;
                    cm[pt][mt][0] = k0 ? ca[pt][mt][0] : 0u;
                    cm[pt][mt][1] = k1 ? ca[pt][mt][1] : 0u;
                    cm[pt][mt][2] = k0 ? ca[pt][mt][2] : 0u;
                    cm[pt][mt][3] = k1 ? ca[pt][mt][3] : 0u;
                }
#pragma unroll
            for (int nb = 0; nb < NB; ++nb) {
                const int vrow = 8 * nb + g;  // descriptor index of this lane's B column
                const uint32_t bb0 = Wb[vrow * (SB / 2) + 8 * ch + c], bb1 = Wb[vrow * (SB / 2) + 8 * ch + 4 + c];
#pragma unroll
                for (int mt = 0; mt < 2; ++mt) {
                    mma_bf16(dacc[mt][nb], cm[1][mt], bb0, bb1);
                    mma_bf16(dacc[mt][nb], cm[0][mt], bb0, bb1);
                }
            }
        }
    }
    // U: sum the quad's partial sums, then each lane takes its own row's
    float rs[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        float v = up[k >> 1][k & 1];
        v += __shfl_xor_sync(FULL, v, 1);
        v += __shfl_xor_sync(FULL, v, 2);
        rs[k] = v;  // row 16 (k >> 1) + 8 (k & 1) + g
    }
    float mine = 0.f;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float v = __shfl_sync(FULL, rs[k], 4 * (lane & 7));
        if ((lane >> 3) == k) mine = v;
    }
    U = mine - P[off.b1 + ti] - P[off.b1l + ti];
    // dQ back to one row per lane
    float* Dw = reinterpret_cast<float*>(scratch);  // [32][NDP + 1]
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nb = 0; nb < NB; ++nb)
#pragma unroll
            for (int e = 0; e < 4; ++e)
                Dw[(16 * mt + g + 8 * (e >> 1)) * (NDP + 1) + 8 * nb + 2 * c + (e & 1)] = dacc[mt][nb][e];
    __syncwarp();
#pragma unroll
    for (int v = 0; v < ND; ++v) dq[v] = Dw[lane * (NDP + 1) + v];
    __syncwarp();
}

// Four-body invariant of one radial channel's l = 2 moments and its gradient.
// a[0..4] are A_n2m in the real basis of sh_eval (xy, yz, 2z^2 - x^2 - y^2, xz,
// x^2 - y^2).  sum_m a_m Y_2m(u) = u^T M u for the traceless symmetric M built
// below, and M = 15 / (8 pi) Q with Q = sum_j g_j (u_j u_j^T - I/3) (addition
// theorem for l = 2).  The Wigner-coupled triple product
// sum (2 2 2; m1 m2 m3) A_2m1 A_2m2 A_2m3 is the cubic invariant kappa tr(Q^3),
// kappa = (2 2 2; 0 0 0) (5 / 4 pi)^(3/2) 9/2, so q4 = kQ4 tr(M^3) with
// kQ4 = kappa (8 pi / 15)^3 = -32 sqrt(14) pi^(3/2) / 525.  d tr(M^3) / dM = 3 M^2.
constexpr double kQ4 = -1.2699291782903164;
constexpr double kY2xy = 1.0925484305920792;  // sqrt(15 / 4 pi): Y_2 of xy, yz, xz
constexpr double kY2zz = 0.31539156525252005; // sqrt(5 / 16 pi): Y_2 of 2z^2 - x^2 - y^2
constexpr double kY2xx = 0.5462742152960396;  // sqrt(15 / 16 pi): Y_2 of x^2 - y^2

template <typename real>
__device__ __forceinline__ real four_body(const real* a, real* grad)
{
    const real c1 = real(kY2xy), c0 = real(kY2zz), c2 = real(kY2xx);
    const real hxy = real(0.5) * c1 * a[0], hyz = real(0.5) * c1 * a[1], hxz = real(0.5) * c1 * a[3];
    const real mxx = c2 * a[4] - c0 * a[2], myy = -c2 * a[4] - c0 * a[2], mzz = real(2) * c0 * a[2];
    // M^2 (symmetric)
    const real sxx = mxx * mxx + hxy * hxy + hxz * hxz;
    const real syy = hxy * hxy + myy * myy + hyz * hyz;
    const real szz = hxz * hxz + hyz * hyz + mzz * mzz;
    const real sxy = mxx * hxy + hxy * myy + hxz * hyz;
    const real sxz = mxx * hxz + hxy * hyz + hxz * mzz;
    const real syz = hxy * hxz + myy * hyz + hyz * mzz;
    const real tr3 = mxx * sxx + myy * syy + mzz * szz + real(2) * (hxy * sxy + hxz * sxz + hyz * syz);
    // dq4/da_m = kQ4 * 3 * sum_ab (M^2)_ab dM_ab/da_m
    const real k3 = real(3 * kQ4);
    grad[0] = k3 * c1 * sxy;
    grad[1] = k3 * c1 * syz;
    grad[2] = k3 * c0 * (real(2) * szz - sxx - syy);
    grad[3] = k3 * c1 * sxz;
    grad[4] = k3 * c2 * (sxx - syy);
    return real(kQ4) * tr3;
}

// Per-thread state of the force pass for one particle i.
template <typename real, int KRP>
struct ForceCtx {
    PosRec<real> ri;
    int i, ti, T;
    real len[3];
    real F[3];
    real W[9];
};

// 64-bit fixed-point accumulation (2^-32 units): integer sums do not depend on the
// order in which atomic adds arrive, so scattered forces stay bitwise reproducible.
constexpr float kFixScale = 4294967296.0f;  // 2^32 fixed-point units per eV/A (or eV)

__device__ __forceinline__ void fix_add(unsigned long long* p, float v)
{
    atomicAdd(p, (unsigned long long)__float2ll_rn(v * kFixScale));
}

// A fixed-point sum in FP32, the working precision of the forces (kept off the FP64
// pipe)
__device__ __forceinline__ float fix_value_f(unsigned long long v) { return (float)(long long)v * (1.0f / kFixScale); }

__device__ __forceinline__ float mul_rn(float x, float y) { return __fmul_rn(x, y); }
__device__ __forceinline__ double mul_rn(double x, double y) { return __dmul_rn(x, y); }

// One block of a sphere-reduced polynomial (layout of sh_reduce): the value and the x and
// y derivatives of sum_{a+b<=D} c[o(a) + b] x^a y^b, by Horner's scheme in y for each
// power of x (with the y-derivative) nested in Horner's scheme in x (with the
// x-derivative).
template <int D, bool BLOCK_B, typename real>
__device__ __forceinline__ void red_block(const real* c, real x, real y, real& v, real& vx, real& vy)
{
#pragma unroll
    for (int a = D; a >= 0; --a) {
        const int o = BLOCK_B ? sh_red_b(a) : sh_red_a(a);
        real al = c[o + D - a], dal = real(0);
#pragma unroll
        for (int b = D - a - 1; b >= 0; --b) {
            dal = b == D - a - 1 ? al : fma(dal, y, al);
            al = fma(al, y, c[o + b]);
        }
        if (a == D) {
            v = al;
            vx = vy = real(0);
        } else if (a == D - 1) {
            vx = v;
            v = fma(v, x, al);
            vy = dal;
        } else {
            vx = fma(vx, x, v);
            v = fma(v, x, al);
            vy = fma(vy, x, dal);
        }
    }
}

// Value and gradient at (x, y, z) of the sphere-reduced polynomial c (sh_reduce):
// P = A + z B, grad P = (A_x + z B_x, A_y + z B_y, B).  On the unit sphere P equals
// the harmonic sum it was reduced from, and grad P differs from that sum's gradient
// only along the normal.
template <typename real>
__device__ __forceinline__ void sh_red_eval(const real* c, real x, real y, real z, real& v, real& vx, real& vy,
                                            real& vz)
{
    real pa, pax, pay, pb, pbx, pby;
    red_block<4, false>(c, x, y, pa, pax, pay);
    red_block<3, true>(c, x, y, pb, pbx, pby);
    v = fma(z, pb, pa);
    vx = fma(z, pbx, pax);
    vy = fma(z, pby, pay);
    vz = pb;
}

template <typename real, int NA, int KA, typename Ctx>
__device__ __forceinline__ void force_angular_phi_reg(const EvalArgs<real>& a, const real* P, const ParamLayout& off,
                                                      const real (&Psi)[NA][kShRed], Ctx& c, bool per_bead);

template <typename real, int NR, int NA, int KR, int KA, int NET, int MBT, int FUSE>
__device__ __forceinline__ void descriptor_item(const EvalArgs<real>& a, const WorkItem it, unsigned char* smem_raw);

// One work item per block (launch grids cover the item capacity; blocks past the
// batch's item count exit): the block stages its model's tables, then one thread
// per particle runs descriptor_item.
template <typename real, int NR, int NA, int KR, int KA, int MB, int NET = 0, int MBT = 0, int FUSE = 0>
__global__ void __launch_bounds__(kBlock, sizeof(real) == 4 ? MB : 1) k_descriptor(EvalArgs<real> a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if ((int)blockIdx.x >= a.counts->n_items) return;
    const WorkItem it = a.items[blockIdx.x];
    const ModelDesc<real>& md = a.models[a.reqs[it.req].model];
    stage_params(md.params, reinterpret_cast<real*>(smem_raw), md.off.total);
    descriptor_item<real, NR, NA, KR, KA, NET, MBT, FUSE>(a, it, smem_raw);
}

template <typename real, int NR, int NA, int KR, int KA, int NET, int MBT, int FUSE>
__device__ __forceinline__ void descriptor_item(const EvalArgs<real>& a, const WorkItem it, unsigned char* smem_raw)
{
    // MBT = 1: the four-body q4_n (l = 2) and five-body q5_n = q_n1^2 follow the
    // three-body descriptors (both always; a model with one of them has zero weights
    // on the other)
    constexpr int ND = NR + NA * (4 + 2 * MBT);
    constexpr int KRP = (KR + 3) & ~3;
    real* P = reinterpret_cast<real*>(smem_raw);
    const ReqInfo& rq = a.reqs[it.req];
    const ModelDesc<real> md = a.models[rq.model];
    const ParamLayout off = md.off;
    // NET = 1 evaluates the network warp-wide: a lane past the item's end follows
    // the item's last particle and writes nothing
    const bool live = NET == 0 || it.begin + (int)threadIdx.x < it.end;
    const int i = live ? it.begin + threadIdx.x : it.end - 1;
    if (NET == 0 && i >= it.end) return;
    const int T = md.T, H = md.H;
    const real len[3] = {(real)rq.g.len[0], (real)rq.g.len[1], (real)rq.g.len[2]};
    const PosRec<real> ri = a.rec[i];
    const int ti = ri.t;
    real q[ND];
#pragma unroll
    for (int v = 0; v < ND; ++v) q[v] = real(0);

    // ---- radial descriptors (Eq. 3, 6-8) ----
    const int cR = min(a.cntR[i], a.mnR);
    if (T == 1) {
        // one pair type: q_n = sum_k c_nk (sum_j f_k(r_ij)), contracted once per bead;
        // the pair sums are kept as four partial sums (see walk4p)
        real fp[4][KR], hp[4];
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            hp[p] = real(0);
#pragma unroll
            for (int k = 0; k < KR; ++k) fp[p][k] = real(0);
        }
        const real inv_rc = P[off.rcRi], inv_lo = P[off.rcRl];
        walk4p(a.nlR + i, (size_t)a.n, cR, [&](uint32_t e, int p) {
            const PosRec<real> rj = a.rec[e & kJMask];
            real dx, dy, dz;
            pair_vec(len, ri, rj, e, dx, dy, dz);
            const real r2 = dx * dx + dy * dy + dz * dz;
            const real r = r2 * rsqrt_r(r2);
            basis_acc<real, KR>(r, inv_rc, inv_lo, fp[p], hp[p]);
        });
        const real hs = (hp[0] + hp[1]) + (hp[2] + hp[3]);
        real fs[KR];
#pragma unroll
        for (int k = 0; k < KR; ++k) fs[k] = ((fp[0][k] + fp[1][k]) + (fp[2][k] + fp[3][k])) + hs;
        const real* c = P + off.cR;
#pragma unroll
        for (int nn = 0; nn < NR; ++nn) {
            real g = real(0);
#pragma unroll
            for (int k = 0; k < KR; ++k) g += c[nn * KR + k] * fs[k];
            if constexpr (sizeof(real) == 4) {  // plus the coefficients' FP32 rounding residuals
                const real* cl = P + off.cRl;
                real gl = real(0);
#pragma unroll
                for (int k = 0; k < KR; ++k) gl += cl[nn * KR + k] * fs[k];
                g += gl;
            }
            q[nn] = g;
        }
    } else {
        real qp[4][NR];  // four partial sums (see walk4p)
#pragma unroll
        for (int p = 0; p < 4; ++p)
#pragma unroll
            for (int nn = 0; nn < NR; ++nn) qp[p][nn] = real(0);
        walk4p(a.nlR + i, (size_t)a.n, cR, [&](uint32_t e, int p) {
            const PosRec<real> rj = a.rec[e & kJMask];
            real dx, dy, dz;
            pair_vec(len, ri, rj, e, dx, dy, dz);
            const real r2 = dx * dx + dy * dy + dz * dz;
            const real r = r2 * rsqrt_r(r2);
            const int tp = ti * T + rj.t;
            real f[KR];
            basis<real, KR>(r, P[off.rcRi + tp], P[off.rcRl + tp], f);
            const real* c = P + off.cR + tp * coef_stride(NR, KR);
#pragma unroll
            for (int nn = 0; nn < NR; ++nn) {
                real g = real(0);
#pragma unroll
                for (int k = 0; k < KR; ++k) g += c[nn * KR + k] * f[k];
                qp[p][nn] += g;
            }
        });
#pragma unroll
        for (int nn = 0; nn < NR; ++nn) q[nn] = (qp[0][nn] + qp[1][nn]) + (qp[2][nn] + qp[3][nn]);
    }

    // ---- angular moments A_nlm (Eq. 5) ----
    real A[NA][kNLM];
#pragma unroll
    for (int nn = 0; nn < NA; ++nn)
#pragma unroll
        for (int k = 0; k < kNLM; ++k) A[nn][k] = real(0);
    const int cA = min(a.cntA[i], a.mnA);
    NbrWalk<real> wa(a.nlA, a.n, i, cA, a.rec);
    for (int s = 0; s < cA; ++s) {
        uint32_t e;
        PosRec<real> rj;
        wa.next(s, e, rj);
        real dx, dy, dz;
        pair_vec(len, ri, rj, e, dx, dy, dz);
        const real r2 = dx * dx + dy * dy + dz * dz;
        const real inv_r = rsqrt_r(r2);
        const real r = r2 * inv_r;
        const int tp = ti * T + rj.t;
        real f[KA];
        basis<real, KA>(r, P[off.rcAi + tp], P[off.rcAl + tp], f);
        real Y[kNLM];
        sh_eval(dx * inv_r, dy * inv_r, dz * inv_r, Y);
        const real* crow = P + off.cA + tp * coef_stride(NA, KA);
#pragma unroll
        for (int nn = 0; nn < NA; ++nn) {
            // one coefficient row at a time: the fence keeps the compiler from loading
            // every row up front, which would hold 32 more registers across the sums
            real cr[KA];
            load_coef(crow + nn * KA, T == 1 && KA % 4 == 0, cr);
            real g = real(0);
#pragma unroll
            for (int k = 0; k < KA; ++k) g += cr[k] * f[k];
#pragma unroll
            for (int k = 0; k < kNLM; ++k) A[nn][k] += g * Y[k];
            asm volatile("" ::: "memory");
        }
    }
    // q_nl (Eq. 4)
#pragma unroll
    for (int nn = 0; nn < NA; ++nn)
#pragma unroll
        for (int k = 0; k < kNLM; ++k) q[NR + (l_of(k) - 1) * NA + nn] += A[nn][k] * A[nn][k];
    // four- and five-body terms; g4 keeps dq4/dA_n2m for the adjoint below
    real g4[MBT ? NA : 1][5];
    if constexpr (MBT == 1) {
#pragma unroll
        for (int nn = 0; nn < NA; ++nn) {
            q[NR + 4 * NA + nn] = four_body(&A[nn][3], g4[nn]);
            q[NR + 5 * NA + nn] = q[NR + nn] * q[NR + nn];
        }
    }

    // ---- network (Eq. 2) and dU/dq ----
    real U;
    real dq[ND];
    if constexpr (NET == 1) {
        unsigned char* scratch = smem_raw + (((size_t)off.total * sizeof(real) + 15) & ~(size_t)15) +
                                 (size_t)(threadIdx.x >> 5) * net_scratch(ND);
        net_bf16<ND>(P, off, T, H, ti, q, U, dq, scratch);
        if (!live) return;
    } else {
        // The FP32 form adds the parameters' rounding residuals (tables ...l) in
        // separate accumulators, so the energy is that of the caller's FP64 weights;
        // the gradient (forces, whose tolerance is far looser) uses the FP32 weights.
        constexpr bool kRes = sizeof(real) == 4;
        const real* b0 = P + off.b0 + ti * H;
        const real* w1 = P + off.w1 + ti * H;
        const real* b0l = P + (kRes ? off.b0l : off.b0) + ti * H;
        const real* w1l = P + (kRes ? off.w1l : off.w1) + ti * H;
        U = -P[off.b1 + ti];
        real Ul = kRes ? -P[off.b1l + ti] : real(0);
#pragma unroll
        for (int v = 0; v < ND; ++v) dq[v] = real(0);
        if (T == 1) {
            // one type: W0 rows padded to a multiple of 4 and 16-byte aligned, read as
            // vectors once per hidden unit and kept for the gradient (every lane reads
            // the same row, a broadcast)
            constexpr int NDV = (ND + 3) & ~3;
            const real* w0 = P + off.w0;
            const real* w0l = P + (kRes ? off.w0l : off.w0);
            for (int mu = 0; mu < H; ++mu) {
                real w[NDV];
                loadN<real, NDV>(w0 + mu * NDV, w);
                real x = -b0[mu];
#pragma unroll
                for (int v = 0; v < ND; ++v) x += w[v] * q[v];
                if constexpr (kRes) {  // residual row four entries at a time (vector loads)
                    real xl = -b0l[mu];
#pragma unroll
                    for (int v4 = 0; v4 < NDV; v4 += 4) {
                        real wl[4];
                        load4(w0l + mu * NDV + v4, wl);
#pragma unroll
                        for (int u = 0; u < 4; ++u)
                            if (v4 + u < ND) xl += wl[u] * q[v4 + u];
                    }
                    x += xl;
                }
                const real h = tanh_r(x);
                U += w1[mu] * h;
                if constexpr (kRes) Ul += w1l[mu] * h;
                const real coef = w1[mu] * (real(1) - h * h);
#pragma unroll
                for (int v = 0; v < ND; ++v) dq[v] += coef * w[v];
            }
        } else {
            // several types: unpadded rows (padded ones put the rows that lanes of
            // different types read at once into the same shared-memory banks)
            const real* w0 = P + off.w0 + ti * H * ND;
            const real* w0l = P + (kRes ? off.w0l : off.w0) + ti * H * ND;
            for (int mu = 0; mu < H; ++mu) {
                real x = -b0[mu];
#pragma unroll
                for (int v = 0; v < ND; ++v) x += w0[mu * ND + v] * q[v];
                if constexpr (kRes) {
                    real xl = -b0l[mu];
#pragma unroll
                    for (int v = 0; v < ND; ++v) xl += w0l[mu * ND + v] * q[v];
                    x += xl;
                }
                const real h = tanh_r(x);
                U += w1[mu] * h;
                if constexpr (kRes) Ul += w1l[mu] * h;
                const real coef = w1[mu] * (real(1) - h * h);
#pragma unroll
                for (int v = 0; v < ND; ++v) dq[v] += coef * w0[mu * ND + v];
            }
        }
        if constexpr (kRes) U += Ul;
    }
    a.U[i] = U;
    // e_i^t[k] = sum_n dU/dq_n c^{t_i t}_{nk}
    real* ei = a.e + (size_t)i * a.e_stride;
    for (int t = 0; t < T; ++t) {
        const real* c = P + off.cR + (ti * T + t) * coef_stride(NR, KR);
#pragma unroll
        for (int k = 0; k < KRP; ++k) {
            real v = real(0);
            if (k < KR) {
#pragma unroll
                for (int nn = 0; nn < NR; ++nn) v += dq[nn] * c[nn * KR + k];
            }
            ei[t * KRP + k] = v;
        }
    }
    if constexpr (MBT == 1) {
        // dq5/dA_n1m = 2 q_n1 dq_n1/dA_n1m: fold into the l = 1 coefficient
#pragma unroll
        for (int nn = 0; nn < NA; ++nn) dq[NR + nn] += real(2) * q[NR + nn] * dq[NR + 5 * NA + nn];
    }
    if constexpr (FUSE == 1) {
        // Phi_nlm in place of A_nlm, in registers; then the angular pairs' forces
        // in scatter form (f_ij from Phi_i alone) while Phi_i is still here
#pragma unroll
        for (int k = 0; k < kNLM; ++k)
#pragma unroll
            for (int nn = 0; nn < NA; ++nn) {
                real v = real(2) * dq[NR + (l_of(k) - 1) * NA + nn] * A[nn][k];
                if constexpr (MBT == 1)
                    if (k >= 3 && k < 8) v += dq[NR + 4 * NA + nn] * g4[nn][k - 3];
                A[nn][k] = v;
            }
        // each P_n = sum_k Phi_nk Y_k in its sphere-reduced form (see sh_red_eval)
        real Psi[NA][kShRed];
#pragma unroll
        for (int nn = 0; nn < NA; ++nn) sh_reduce(A[nn], Psi[nn]);
        ForceCtx<real, KRP> c;
        c.i = i;
        c.T = T;
        c.ri = ri;
        c.ti = ti;
#pragma unroll
        for (int k = 0; k < 3; ++k) c.len[k] = len[k];
#pragma unroll
        for (int k = 0; k < 3; ++k) c.F[k] = real(0);
#pragma unroll
        for (int k = 0; k < 9; ++k) c.W[k] = real(0);
        const bool per_bead = a.virial != nullptr;
        force_angular_phi_reg<real, NA, KA>(a, P, off, Psi, c, per_bead);
        // F_i's angular part into i's line; the thread's angular virial sum (what
        // the totals use, with or without per-particle virials) as plain stores
        unsigned long long* acc_i = a.accF + (size_t)i * 4;
#pragma unroll
        for (int p = 0; p < 3; ++p) fix_add(acc_i + p, c.F[p]);
#pragma unroll
        for (int k = 0; k < 9; ++k) a.wsum[(size_t)k * a.n + i] = c.W[k];
    } else {
        // The sphere-reduced coefficients of each P_n = sum_k Phi_nk Y_k (sh_reduce),
        // stored component-major, [kShRed][n][NAP]: for one component the rows of
        // consecutive particles are adjacent, so a warp's row loads are contiguous
        constexpr int NAP = phi_pad(NA);
        real* ph = a.phi + (size_t)i * NAP;
        const size_t kstride = (size_t)a.n * NAP;
#pragma unroll
        for (int nn = 0; nn < NA; ++nn) {
            real phi[kNLM], psi[kShRed];
#pragma unroll
            for (int k = 0; k < kNLM; ++k) {
                phi[k] = real(2) * dq[NR + (l_of(k) - 1) * NA + nn] * A[nn][k];
                if constexpr (MBT == 1)
                    if (k >= 3 && k < 8) phi[k] += dq[NR + 4 * NA + nn] * g4[nn][k - 3];
            }
            sh_reduce(phi, psi);
#pragma unroll
            for (int m = 0; m < kShRed; ++m) ph[m * kstride + nn] = psi[m];
        }
#pragma unroll
        for (int nn = NA; nn < NAP; ++nn)
#pragma unroll
            for (int m = 0; m < kShRed; ++m) ph[m * kstride + nn] = real(0);
    }
}

template <typename real>
__device__ __forceinline__ real warp_sum(real v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// FP64 sums of (E, W[9]) over each request, in a fixed order whatever the timing:
//   1. each block sums its particles: the 10 values of its threads go to shared
//      memory, 80 threads sum 16 each (value k = t / 8, a stride-8 subset), then 10
//      threads sum the 8 parts, into partial[item];
//   2. the last block of each group of kGroup consecutive items of a request (counted
//      from the request's first item) sums the group's block partials and writes the
//      group sum over the group's first partial;
//   3. the last group of the request sums the group sums into totals[req].
// The summing threads take fixed subsets, so a request sums alike alone or in a
// batch.  Spreading the sums over the groups' last blocks keeps the serial tail of
// the kernel (FP64 arithmetic is scarce on this part) to two short passes.

// out[k] = sum over b < nb of src[b * 10 + k] (L2 reads: written by other blocks),
// with 120 threads in a fixed order; the result is valid in threads < 10
__device__ __forceinline__ double sum_partials(const double* src, int nb, int stride_items, double (&part)[10][12])
{
    const int t = threadIdx.x;
    if (t < 120) {
        const int k = t % 10, q = t / 10;
        double s = 0.0;
#pragma unroll 4
        for (int b = q; b < nb; b += 12) s += __ldcg(src + (size_t)b * stride_items * 10 + k);
        part[k][q] = s;
    }
    __syncthreads();
    double s = 0.0;
    if (t < 10) {
#pragma unroll
        for (int q = 0; q < 12; ++q) s += part[t][q];
    }
    return s;
}

template <int BS>
__device__ __forceinline__ void reduce_totals(double (&v)[10], int item, const WorkItem& it, const ReqInfo& rq,
                                              double* partial, unsigned int* gcounter, unsigned int* counter,
                                              double* totals)
{
    static_assert(BS % 8 == 0 && BS >= 120, "block size");
    __shared__ double red[10][BS + 8];  // row stride 2 words mod 32 apart: 2-way for 64-bit loads
    __shared__ double part[10][12];
    __shared__ bool last;
    const int t = threadIdx.x;
#pragma unroll
    for (int k = 0; k < 10; ++k) red[k][t] = v[k];
    __syncthreads();
    if (t < 80) {
        const int k = t >> 3, q = t & 7;
        double s = 0.0;
#pragma unroll
        for (int j = 0; j < BS / 8; ++j) s += red[k][8 * j + q];
        part[k][q] = s;
    }
    __syncthreads();
    if (t < 10) {
        double s = 0.0;
#pragma unroll
        for (int q = 0; q < 8; ++q) s += part[t][q];
        partial[(size_t)item * 10 + t] = s;
        __threadfence();  // the writers publish their partials before the count below
    }
    __syncthreads();
    const int rel = item - rq.item_begin;
    const int n_items = rq.item_end - rq.item_begin;
    const int g0 = rq.item_begin + rel / kGroup * kGroup;  // the group's first item
    const int gn = min(kGroup, rq.item_end - g0);
    if (t == 0) last = (atomicAdd(&gcounter[g0], 1u) == (unsigned int)gn - 1u);
    __syncthreads();
    if (!last) return;
    __threadfence();
    const double gs = sum_partials(partial + (size_t)g0 * 10, gn, 1, part);
    const int ng = (n_items + kGroup - 1) / kGroup;
    if (ng == 1) {  // one group: its sum is the total
        if (t < 10) totals[(size_t)it.req * 10 + t] = gs;
        if (t == 0) gcounter[g0] = 0u;
        return;
    }
    if (t < 10) {
        partial[(size_t)g0 * 10 + t] = gs;  // over the group's first partial
        if (t == 0) gcounter[g0] = 0u;
        __threadfence();
    }
    __syncthreads();
    if (t == 0) last = (atomicAdd(&counter[it.req], 1u) == (unsigned int)ng - 1u);
    __syncthreads();
    if (!last) return;
    __threadfence();
    const double ts = sum_partials(partial + (size_t)rq.item_begin * 10, ng, kGroup, part);
    if (t < 10) totals[(size_t)it.req * 10 + t] = ts;
    if (t == 0) counter[it.req] = 0u;
}

// Radial pairs of slots s0, s0 + ds, ... :
//   f_ij = (e_i^{t_j} . f') u,  f_ji = -(e_j^{t_i} . f') u,  F_i += f_ij - f_ji,
//   W_i += r_ij (x) f_ji.  The pair body has no branch, so the scheduler can
//   interleave the four bodies of each walk step.  f_ji is parallel to r_ij, so the
//   radial terms of W_i are symmetric: with SYM, c.W[0..5] holds xx, yy, zz, xy, xz,
//   yz of the radial part alone (6 products per pair instead of 9).
template <typename real, int NR, int KR, bool SYM = false, int CH = 4>
__device__ __forceinline__ void force_radial(const EvalArgs<real>& a, const real* P, const ParamLayout& off,
                                             ForceCtx<real, (KR + 3) & ~3>& c, int s0, int ds)
{
    constexpr int KRP = (KR + 3) & ~3;
    const real* e_i = a.e + (size_t)c.i * a.e_stride;
    const int cR = min(a.cntR[c.i], a.mnR);
    const int cnt = cR > s0 ? (cR - s0 + ds - 1) / ds : 0;
    const int T = c.T, ti = c.ti;
    auto radial_pair = [&](uint32_t e, const real* eij) {
        const int j = (int)(e & kJMask);
        const PosRec<real> rj = a.rec[j];
        real eji[KRP];
        loadN<real, KRP>(a.e + (size_t)j * a.e_stride + ti * KRP, eji);
        real dx, dy, dz;
        pair_vec(c.len, c.ri, rj, e, dx, dy, dz);
        const real r2 = dx * dx + dy * dy + dz * dz;
        const real inv_r = rsqrt_r(r2);
        const real r = r2 * inv_r;
        real f[KR], df[KR];
        basis_d<real, KR>(r, P[off.rcRi + ti * T + rj.t], P[off.rcRl + ti * T + rj.t], f, df);
        real ai = real(0), bj = real(0);
#pragma unroll
        for (int k = 0; k < KR; ++k) {
            ai += eij[k] * df[k];
            bj += eji[k] * df[k];
        }
        const real ux = dx * inv_r, uy = dy * inv_r, uz = dz * inv_r;
        const real fs = ai + bj;
        c.F[0] += fs * ux;
        c.F[1] += fs * uy;
        c.F[2] += fs * uz;
        if constexpr (SYM) {
            const real w = bj * inv_r;
            const real wx = w * dx, wy = w * dy, wz = w * dz;
            c.W[0] -= wx * dx;
            c.W[1] -= wy * dy;
            c.W[2] -= wz * dz;
            c.W[3] -= wx * dy;
            c.W[4] -= wx * dz;
            c.W[5] -= wy * dz;
        } else {
            const real d[3] = {dx, dy, dz}, u[3] = {ux, uy, uz};
#pragma unroll
            for (int p = 0; p < 3; ++p) {
                const real bd = bj * d[p];
#pragma unroll
                for (int q = 0; q < 3; ++q) c.W[3 * p + q] -= bd * u[q];
            }
        }
    };
    const uint32_t* nl = a.nlR + (size_t)s0 * a.n + c.i;
    const size_t stride = (size_t)ds * a.n;
    if (T == 1) {
        real ei1[KRP];  // the one partner type's vector
        loadN<real, KRP>(e_i, ei1);
        walk_chunk<CH>(nl, stride, cnt, [&](uint32_t e) { radial_pair(e, ei1); });
    } else {
        walk_chunk<CH>(nl, stride, cnt, [&](uint32_t e) {
            real eij[KRP];
            loadN<real, KRP>(e_i + a.rec[e & kJMask].t * KRP, eij);
            radial_pair(e, eij);
        });
    }
}

// Angular pairs in gather form: f_ij from i's reduced coefficients at u and f_ji from
// j's at -u (the reduced form holds the harmonic sum's values on the whole sphere,
// so no parity factor is needed):
//   f_ij = D_i u + (ga_i - (u . ga_i) u) / r,  D_i = sum_n g_n' P_in(u), ga_i = sum_n g_n grad P_in(u),
// and f_ji likewise at -u with j's coefficients and type-pair functions (see
// force_angular_phi_reg for the derivation).  F_i += f_ij - f_ji, W_i += r_ij (x) f_ji.
template <typename real, int NA, int KA, typename Ctx>
__device__ __forceinline__ void force_angular_red(const EvalArgs<real>& a, const real* P, const ParamLayout& off,
                                                  Ctx& c)
{
    const int T = c.T, ti = c.ti;
    constexpr int NAP = phi_pad(NA);
    const size_t kstride = (size_t)a.n * NAP;
    const real* psi_i = a.phi + (size_t)c.i * NAP;
    const int cA = min(a.cntA[c.i], a.mnA);
    NbrWalk<real> wa(a.nlA, a.n, c.i, cA, a.rec);
    for (int s = 0; s < cA; ++s) {
        uint32_t e;
        PosRec<real> rj;
        wa.next(s, e, rj);
        const int j = (int)(e & kJMask);
        real dx, dy, dz;
        pair_vec(c.len, c.ri, rj, e, dx, dy, dz);
        const real r2 = dx * dx + dy * dy + dz * dz;
        const real inv_r = rsqrt_r(r2);
        const real r = r2 * inv_r;
        const int tij = ti * T + rj.t, tji = rj.t * T + ti;
        real f[KA], df[KA];
        basis_d<real, KA>(r, P[off.rcAi + tij], P[off.rcAl + tij], f, df);
        real gi[NA], dgi[NA], gj[NA], dgj[NA];
        {
            const real* cc = P + off.cA + tij * coef_stride(NA, KA);
#pragma unroll
            for (int nn = 0; nn < NA; ++nn) {
                real s0 = real(0), s1 = real(0);
#pragma unroll
                for (int k = 0; k < KA; ++k) {
                    s0 += cc[nn * KA + k] * f[k];
                    s1 += cc[nn * KA + k] * df[k];
                }
                gi[nn] = s0;
                dgi[nn] = s1;
            }
        }
        if (tji == tij) {
#pragma unroll
            for (int nn = 0; nn < NA; ++nn) {
                gj[nn] = gi[nn];
                dgj[nn] = dgi[nn];
            }
        } else {
            const real* cc = P + off.cA + tji * coef_stride(NA, KA);
#pragma unroll
            for (int nn = 0; nn < NA; ++nn) {
                real s0 = real(0), s1 = real(0);
#pragma unroll
                for (int k = 0; k < KA; ++k) {
                    s0 += cc[nn * KA + k] * f[k];
                    s1 += cc[nn * KA + k] * df[k];
                }
                gj[nn] = s0;
                dgj[nn] = s1;
            }
        }
        const real ux = dx * inv_r, uy = dy * inv_r, uz = dz * inv_r;
        const real* psi_j = a.phi + (size_t)j * NAP;
        real Di = real(0), Dj = real(0);
        real ga[3] = {real(0), real(0), real(0)}, gb[3] = {real(0), real(0), real(0)};
#pragma unroll
        for (int nn = 0; nn < NA; ++nn) {
            real ci[kShRed], cj[kShRed];
#pragma unroll
            for (int m = 0; m < kShRed; ++m) {
                ci[m] = psi_i[m * kstride + nn];
                cj[m] = psi_j[m * kstride + nn];
            }
            real v, vx, vy, vz;
            sh_red_eval(ci, ux, uy, uz, v, vx, vy, vz);
            Di += dgi[nn] * v;
            ga[0] += gi[nn] * vx;
            ga[1] += gi[nn] * vy;
            ga[2] += gi[nn] * vz;
            sh_red_eval(cj, -ux, -uy, -uz, v, vx, vy, vz);
            Dj += dgj[nn] * v;
            gb[0] += gj[nn] * vx;
            gb[1] += gj[nn] * vy;
            gb[2] += gj[nn] * vz;
        }
        // f_ij, and f_ji with u' = -u: f_ji = -Dj u + (gb - (u . gb) u) / r
        const real pa = (ux * ga[0] + uy * ga[1] + uz * ga[2]) * inv_r;
        const real pb = (ux * gb[0] + uy * gb[1] + uz * gb[2]) * inv_r;
        const real u[3] = {ux, uy, uz}, d[3] = {dx, dy, dz};
        real fji[3];
#pragma unroll
        for (int p = 0; p < 3; ++p) {
            const real fij = (Di - pa) * u[p] + ga[p] * inv_r;
            fji[p] = (-Dj - pb) * u[p] + gb[p] * inv_r;
            c.F[p] += fij - fji[p];
        }
#pragma unroll
        for (int p = 0; p < 3; ++p)
#pragma unroll
            for (int q = 0; q < 3; ++q) c.W[3 * p + q] += d[p] * fji[q];
    }
}

// The MD step's closing half-kick of particle ui (caller index; lu within its
// request) from its final force, rounded as the separate kick kernel rounds it.
template <typename real>
__device__ __forceinline__ void closing_kick(const EvalArgs<real>& a, const ReqInfo& rq, int ui, int lu,
                                             const double (&F)[3])
{
    const int t = a.kick_types[ui];
    const double im = a.kick_im.v[t >= 0 && t < kMdMaxTypes ? t : 0];
    double* v = a.kick_vel + (size_t)3 * rq.begin + lu;
#pragma unroll
    for (int p = 0; p < 3; ++p) v[(size_t)p * rq.n] = half_kick(v[(size_t)p * rq.n], a.kick_half_dt, F[p], im);
}

template <typename real>
__device__ __forceinline__ void force_outputs(const EvalArgs<real>& a, const ReqInfo& rq, int i, const real* F,
                                              const real* W, double (&tot)[10])
{
    const int ui = a.perm[i];
    const int lu = ui - rq.begin;  // index within the request's output blocks
    const real Ui = a.U[i];
    if (lu >= 0 && lu < rq.n) {
        double* fo = a.force + (size_t)3 * rq.begin + lu;
#pragma unroll
        for (int p = 0; p < 3; ++p) fo[(size_t)p * rq.n] = (double)F[p];
        if (a.kick_vel) {
            double F64[3] = {(double)F[0], (double)F[1], (double)F[2]};
            closing_kick(a, rq, ui, lu, F64);
        }
        if (a.virial) {
            double* vo = a.virial + (size_t)9 * rq.begin + lu;
#pragma unroll
            for (int k = 0; k < 9; ++k) vo[(size_t)k * rq.n] = (double)W[k];
        }
        if (a.site) a.site[ui] = (double)Ui;
    } else if (a.err) {  // see kErrCellList
        atomicOr(a.err, kErrCellList);
    }
    tot[0] = (double)Ui;
#pragma unroll
    for (int k = 0; k < 9; ++k) tot[1 + k] = (double)W[k];
}

// One thread per particle.
template <typename real, int NR, int NA, int KR, int KA, int MB>
__global__ void __launch_bounds__(kBlock, sizeof(real) == 4 ? MB : 1) k_force(EvalArgs<real> a)
{
    constexpr int KRP = (KR + 3) & ~3;
    // i's reduced coefficients are read through L1 (a shared-memory copy would take L1
    // capacity that the neighbours' records and gradients need more)
    extern __shared__ __align__(16) unsigned char smem_raw[];
    real* P = reinterpret_cast<real*>(smem_raw);
    const int w = blockIdx.x;  // one work item per block (see k_descriptor)
    if (w >= a.counts->n_items) return;
    const WorkItem it = a.items[w];
    const ReqInfo& rq = a.reqs[it.req];
    const ModelDesc<real> md = a.models[rq.model];
    const ParamLayout off = md.off;
    stage_params(md.params, P, off.n_cut_coef);
    const int i = it.begin + threadIdx.x;
    double tot[10];
#pragma unroll
    for (int k = 0; k < 10; ++k) tot[k] = 0.0;
    if (i < it.end) {
        ForceCtx<real, KRP> c;
        c.i = i;
        c.T = md.T;
        c.ri = a.rec[i];
        c.ti = c.ri.t;
        for (int k = 0; k < 3; ++k) c.len[k] = (real)rq.g.len[k];
#pragma unroll
        for (int k = 0; k < 3; ++k) c.F[k] = real(0);
#pragma unroll
        for (int k = 0; k < 9; ++k) c.W[k] = real(0);
        force_radial<real, NR, KR>(a, P, off, c, 0, 1);
        force_angular_red<real, NA, KA>(a, P, off, c);
        force_outputs(a, rq, i, c.F, c.W, tot);
    }
    reduce_totals<kBlock>(tot, w, it, rq, a.partial, a.gcounter, a.counter, a.totals);
}

// ---- FP32 form: angular pairs in scatter form inside the descriptor kernel ------
// Each ordered angular pair is evaluated once, by the thread of its centre i, from
// Phi_i alone while it is still in registers: f_ij = dU_i/dr_ij.  F_i gains f_ij
// in registers; F_j loses it (and W_j gains r_ji (x) f_ij) through the fixed-point
// atomic adds.  For A = g(r) Y(u), u = r / |r|, the gradient with respect to r is
//   dA/dr = g' Y(u) u + (g / r) (grad Y(u) - (u . grad Y(u)) u),
// where grad Y may be the gradient of any function equal to Y on the unit sphere
// (only its surface part enters).  Summed over the components with
// P_n = sum_k Phi_nk Y_k:
//   f_ij = (sum_n g_n' P_n(u)) u + (ga - (u . ga) u) / r,   ga = sum_n g_n grad P_n(u),
// evaluated from each P_n's sphere-reduced form Psi_n (sh_red_eval).
template <typename real, int NA, int KA, typename Ctx>
__device__ __forceinline__ void force_angular_phi_reg(const EvalArgs<real>& a, const real* P, const ParamLayout& off,
                                                      const real (&Psi)[NA][kShRed], Ctx& c, bool per_bead)
{
    const int T = c.T, ti = c.ti;
    const int cA = min(a.cntA[c.i], a.mnA);
    NbrWalk<real> wa(a.nlA, a.n, c.i, cA, a.rec);
    for (int s = 0; s < cA; ++s) {
        uint32_t e;
        PosRec<real> rj;
        wa.next(s, e, rj);
        const int j = (int)(e & kJMask);
        real dx, dy, dz;
        pair_vec(c.len, c.ri, rj, e, dx, dy, dz);
        const real r2 = dx * dx + dy * dy + dz * dz;
        const real inv_r = rsqrt_r(r2);
        const real r = r2 * inv_r;
        const int tij = ti * T + rj.t;
        real f[KA], df[KA];
        basis_d<real, KA>(r, P[off.rcAi + tij], P[off.rcAl + tij], f, df);
        real g[NA], dg[NA];
        const real* crow = P + off.cA + tij * coef_stride(NA, KA);
#pragma unroll
        for (int nn = 0; nn < NA; ++nn) {
            real cr[KA];  // one row at a time (see the angular moments)
            load_coef(crow + nn * KA, T == 1 && KA % 4 == 0, cr);
            real s0 = real(0), s1 = real(0);
#pragma unroll
            for (int k = 0; k < KA; ++k) {
                s0 += cr[k] * f[k];
                s1 += cr[k] * df[k];
            }
            g[nn] = s0;
            dg[nn] = s1;
            asm volatile("" ::: "memory");
        }
        const real ux = dx * inv_r, uy = dy * inv_r, uz = dz * inv_r;
        real D = real(0);
        real ga[3] = {real(0), real(0), real(0)};
#pragma unroll
        for (int nn = 0; nn < NA; ++nn) {
            real v, vx, vy, vz;
            sh_red_eval(Psi[nn], ux, uy, uz, v, vx, vy, vz);
            D += dg[nn] * v;
            ga[0] += g[nn] * vx;
            ga[1] += g[nn] * vy;
            ga[2] += g[nn] * vz;
        }
        const real sr = D - (ux * ga[0] + uy * ga[1] + uz * ga[2]) * inv_r;
        const real fij[3] = {sr * ux + ga[0] * inv_r, sr * uy + ga[1] * inv_r, sr * uz + ga[2] * inv_r};
        unsigned long long* acc_j = a.accF + (size_t)j * 4;
#pragma unroll
        for (int p = 0; p < 3; ++p) {
            c.F[p] += fij[p];
            fix_add(acc_j + p, -fij[p]);
        }
        // W_j += r_ji (x) f_ij; each product is rounded on its own, so the thread's
        // sum (the totals) is the same whether or not it is also scattered
        const real d[3] = {dx, dy, dz};
        unsigned long long* accw_j = per_bead ? a.accW + (size_t)j * 12 : nullptr;
#pragma unroll
        for (int p = 0; p < 3; ++p)
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                const real w = mul_rn(-d[p], fij[q]);
                c.W[3 * p + q] += w;
                if (per_bead) fix_add(accw_j + 3 * p + q, w);
            }
    }
}

// Radial pairs in gather form, then i's outputs.  By the time this kernel runs the
// descriptor kernel has finished every scatter, so i's fixed-point line holds the
// angular part of F_i (its own and what its neighbours sent) and of W_i (per-particle
// virials), or the thread's angular virial sum (totals only).  The kernel adds the
// radial part, writes the caller-order FP64 outputs, clears the line for the next
// evaluation, and reduces E and W in FP64 (Eq. 1, 16).
// MB: resident blocks per SM (a register budget); CH: neighbour entries per walk
// group (4 or 8), both chosen per configuration by the autotuner.
template <typename real, int NR, int KR, int MB, int CH>
__global__ void __launch_bounds__(kBlock, MB) k_force_radial(EvalArgs<real> a)
{
    constexpr int KRP = (KR + 3) & ~3;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    real* P = reinterpret_cast<real*>(smem_raw);
    const int w = blockIdx.x;  // one work item per block (see k_descriptor)
    if (w >= a.counts->n_items) return;
    const WorkItem it = a.items[w];
    const ReqInfo& rq = a.reqs[it.req];
    const ModelDesc<real> md = a.models[rq.model];
    const ParamLayout off = md.off;
    const int i = it.begin + threadIdx.x;
    stage_params(md.params, P, off.n_cut_coef);
    double tot[10];
#pragma unroll
    for (int k = 0; k < 10; ++k) tot[k] = 0.0;
    if (i < it.end) {
        ForceCtx<real, KRP> c;
        c.i = i;
        c.T = md.T;
        c.ri = a.rec[i];
        c.ti = c.ri.t;
        for (int k = 0; k < 3; ++k) c.len[k] = (real)rq.g.len[k];
#pragma unroll
        for (int k = 0; k < 3; ++k) c.F[k] = real(0);
#pragma unroll
        for (int k = 0; k < 9; ++k) c.W[k] = real(0);
        force_radial<real, NR, KR, true, CH>(a, P, off, c, 0, 1);
        // the radial virial in full (row-major 3 x 3) from its symmetric part
        const real Wr[9] = {c.W[0], c.W[3], c.W[4], c.W[3], c.W[1], c.W[5], c.W[4], c.W[5], c.W[2]};
        ulonglong2* line = reinterpret_cast<ulonglong2*>(a.accF + (size_t)i * 4);
        const ulonglong2 f01 = line[0], f2x = line[1];
        line[0] = line[1] = make_ulonglong2(0ull, 0ull);
        const int ui = a.perm[i];
        const int lu = ui - rq.begin;
        const bool out_ok = lu >= 0 && lu < rq.n;  // see kErrCellList
        if (!out_ok && a.err) atomicOr(a.err, kErrCellList);
        double* fo = a.force + (size_t)3 * rq.begin + lu;
        // F_i: the angular part from the fixed-point line plus the radial part, added in
        // the working precision and widened once (FP64 arithmetic is scarce)
        double Fi[3] = {(double)(fix_value_f(f01.x) + c.F[0]), (double)(fix_value_f(f01.y) + c.F[1]),
                        (double)(fix_value_f(f2x.x) + c.F[2])};
        if (out_ok) {
            fo[0] = Fi[0];
            fo[rq.n] = Fi[1];
            fo[(size_t)2 * rq.n] = Fi[2];
            if (a.kick_vel) closing_kick(a, rq, ui, lu, Fi);
        }
        if (a.virial) {  // W_i: the angular terms its neighbours sent, plus its radial terms
            ulonglong2* wl = reinterpret_cast<ulonglong2*>(a.accW + (size_t)i * 12);
            double* vo = a.virial + (size_t)9 * rq.begin + lu;
#pragma unroll
            for (int q = 0; q < 5; ++q) {
                const ulonglong2 v = wl[q];
                wl[q] = make_ulonglong2(0ull, 0ull);
                if (out_ok) {
                    vo[(size_t)(2 * q) * rq.n] = (double)(fix_value_f(v.x) + Wr[2 * q]);
                    if (2 * q + 1 < 9) vo[(size_t)(2 * q + 1) * rq.n] = (double)(fix_value_f(v.y) + Wr[2 * q + 1]);
                }
            }
        }
        const real Ui = a.U[i];
        if (a.site && out_ok) a.site[ui] = (double)Ui;
        tot[0] = (double)Ui;
        // i's contribution to the virial total: its angular sum plus its radial terms,
        // added in the working precision and widened once (FP64 arithmetic is scarce)
#pragma unroll
        for (int k = 0; k < 9; ++k) tot[1 + k] = (double)(a.wsum[(size_t)k * a.n + i] + Wr[k]);
    }
    reduce_totals<kBlock>(tot, w, it, rq, a.partial, a.gcounter, a.counter, a.totals);
}

// ---- shape dispatch -----------------------------------------------------------
#define NEP_SHAPES(X) X(5, 4, 8, 8) X(5, 5, 9, 9)

template <typename real>
bool evaluate_shape_supported(int nR, int nA, int KR, int KA)
{
#define NEP_CASE(a_, b_, c_, d_) \
    if (nR == a_ && nA == b_ && KR == c_ && KA == d_) return true;
    NEP_SHAPES(NEP_CASE)
#undef NEP_CASE
    return false;
}

// FP32: the descriptor kernel with the angular forces fused (K1) and the radial /
// output kernel (K2); FP64: the descriptor kernel storing the reduced form of Phi and
// the gather-form force kernel.  Variants: resident blocks per SM (register caps), and for the
// descriptor the network form (NET) and the many-body terms (MBT).
template <typename real, int A_, int B_, int C_, int D_, int MB>
cudaError_t set_smem_desc(size_t smem)
{
    constexpr int FU = sizeof(real) == 4 ? 1 : 0;
    cudaError_t e = cudaFuncSetAttribute(k_descriptor<real, A_, B_, C_, D_, MB, 0, 0, FU>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_descriptor<real, A_, B_, C_, D_, MB, 0, 1, FU>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e != cudaSuccess) return e;
    if constexpr (sizeof(real) == 4) {
        e = cudaFuncSetAttribute(k_descriptor<real, A_, B_, C_, D_, MB, 1, 0, 1>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(k_descriptor<real, A_, B_, C_, D_, MB, 1, 1, 1>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    }
    return e;
}

template <typename real, int A_, int B_, int C_, int D_, int MB>
cudaError_t set_smem_force(size_t smem)
{
    if constexpr (sizeof(real) == 4) {
        cudaError_t e = cudaFuncSetAttribute(k_force_radial<real, A_, C_, MB, 4>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        return cudaFuncSetAttribute(k_force_radial<real, A_, C_, MB, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem);
    } else
        return cudaFuncSetAttribute(k_force<real, A_, B_, C_, D_, MB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem);
}

template <typename real>
cudaError_t evaluate_set_smem(int nR, int nA, int KR, int KA, size_t smem_desc, size_t smem_force)
{
#define NEP_CASE(a_, b_, c_, d_)                                                                 \
    if (nR == a_ && nA == b_ && KR == c_ && KA == d_) {                                          \
        cudaError_t e;                                                                           \
        if ((e = set_smem_desc<real, a_, b_, c_, d_, 2>(smem_desc)) != cudaSuccess) return e;    \
        if ((e = set_smem_desc<real, a_, b_, c_, d_, 3>(smem_desc)) != cudaSuccess) return e;    \
        if ((e = set_smem_force<real, a_, b_, c_, d_, 3>(smem_force)) != cudaSuccess) return e;  \
        if constexpr (sizeof(real) == 4) { /* K2 also at 4 and 5 blocks per SM */                \
            if ((e = set_smem_force<real, a_, b_, c_, d_, 4>(smem_force)) != cudaSuccess) return e; \
            if ((e = set_smem_force<real, a_, b_, c_, d_, 5>(smem_force)) != cudaSuccess) return e; \
        } else {                                                                                 \
            if ((e = set_smem_force<real, a_, b_, c_, d_, 2>(smem_force)) != cudaSuccess) return e; \
        }                                                                                        \
        return cudaSuccess;                                                                      \
    }
    NEP_SHAPES(NEP_CASE)
#undef NEP_CASE
    return cudaErrorInvalidValue;
}

template <typename real, int NR, int NA, int KR, int KA, int MBT>
cudaError_t launch_descriptor(const EvalArgs<real>& a, int nb, size_t smem, cudaStream_t st, int mb_desc)
{
    if constexpr (sizeof(real) == 4) {
        if (a.net_bf16) {
            if (mb_desc == 2) return launch_k(k_descriptor<real, NR, NA, KR, KA, 2, 1, MBT, 1>, nb, kBlock, smem, st, a);
            return launch_k(k_descriptor<real, NR, NA, KR, KA, 3, 1, MBT, 1>, nb, kBlock, smem, st, a);
        }
        if (mb_desc == 2) return launch_k(k_descriptor<real, NR, NA, KR, KA, 2, 0, MBT, 1>, nb, kBlock, smem, st, a);
        return launch_k(k_descriptor<real, NR, NA, KR, KA, 3, 0, MBT, 1>, nb, kBlock, smem, st, a);
    } else {
        if (mb_desc == 2) return launch_k(k_descriptor<real, NR, NA, KR, KA, 2, 0, MBT, 0>, nb, kBlock, smem, st, a);
        return launch_k(k_descriptor<real, NR, NA, KR, KA, 3, 0, MBT, 0>, nb, kBlock, smem, st, a);
    }
}

// The FP32 radial kernel in its (blocks per SM, walk chunk) variant.
template <typename real, int NR, int KR>
cudaError_t launch_force_radial(const EvalArgs<real>& a, int nb, size_t smem, cudaStream_t st, int mb, int ch)
{
    if (ch == 8) {
        if (mb == 5) return launch_k(k_force_radial<real, NR, KR, 5, 8>, nb, kBlock, smem, st, a);
        if (mb == 4) return launch_k(k_force_radial<real, NR, KR, 4, 8>, nb, kBlock, smem, st, a);
        return launch_k(k_force_radial<real, NR, KR, 3, 8>, nb, kBlock, smem, st, a);
    }
    if (mb == 5) return launch_k(k_force_radial<real, NR, KR, 5, 4>, nb, kBlock, smem, st, a);
    if (mb == 4) return launch_k(k_force_radial<real, NR, KR, 4, 4>, nb, kBlock, smem, st, a);
    return launch_k(k_force_radial<real, NR, KR, 3, 4>, nb, kBlock, smem, st, a);
}

template <typename real>
cudaError_t launch_evaluate(int nR, int nA, int KR, int KA, const EvalArgs<real>& a, int items_cap, size_t smem_desc,
                            size_t smem_force, cudaStream_t st, cudaEvent_t mid, int mb_desc, int mb_force,
                            int ch_force)
{
    const int nb = items_cap;
    if constexpr (sizeof(real) == 4) {
        if (!a.accF || !a.wsum) return cudaErrorInvalidValue;  // the FP32 form scatters into a.accF
    }
#define NEP_CASE(a_, b_, c_, d_)                                                                          \
    if (nR == a_ && nA == b_ && KR == c_ && KA == d_) {                                                   \
        cudaError_t e = a.many_body ? launch_descriptor<real, a_, b_, c_, d_, 1>(a, nb, smem_desc, st, mb_desc) \
                                    : launch_descriptor<real, a_, b_, c_, d_, 0>(a, nb, smem_desc, st, mb_desc); \
        if (e != cudaSuccess) return e;                                                                   \
        if (mid && (e = cudaEventRecord(mid, st)) != cudaSuccess) return e;                               \
        if constexpr (sizeof(real) == 4) {                                                                \
            return launch_force_radial<real, a_, c_>(a, nb, smem_force, st, mb_force, ch_force);          \
        } else {                                                                                          \
            if (mb_force == 3) return launch_k(k_force<real, a_, b_, c_, d_, 3>, nb, kBlock, smem_force, st, a); \
            return launch_k(k_force<real, a_, b_, c_, d_, 2>, nb, kBlock, smem_force, st, a);          \
        }                                                                                                 \
    }
    NEP_SHAPES(NEP_CASE)
#undef NEP_CASE
    return cudaErrorInvalidValue;
}

#define NEP_INSTANTIATE(real)                                                                             \
    template bool evaluate_shape_supported<real>(int, int, int, int);                                     \
    template cudaError_t evaluate_set_smem<real>(int, int, int, int, size_t, size_t);                     \
    template cudaError_t launch_evaluate<real>(int, int, int, int, const EvalArgs<real>&, int, size_t, size_t, \
                                               cudaStream_t, cudaEvent_t, int, int, int);
NEP_INSTANTIATE(float)
NEP_INSTANTIATE(double)
#undef NEP_INSTANTIATE

}  // namespace nep
