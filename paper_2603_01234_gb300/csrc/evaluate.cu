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
// k_force (one thread per sorted particle i, gather form, no atomics):
//   for every neighbour j the pair gradients f_ij = dU_i/dr_ij and
//   f_ji = dU_j/dr_ji are rebuilt from i's and j's stored gradients, and
//     F_i = sum_j (f_ij - f_ji),   W_i = sum_j r_ij (x) f_ji   (Eq. 15)
//   then E = sum U_i and W = sum W_i are reduced in FP64 (Eq. 1, 16) with a
//   deterministic last-block pass.
//
// Angular pair gradient.  For A = g(r) Y(u), u = r/|r|, with Y a homogeneous
// polynomial of degree l:  dA/dr = (g' - l g / r) Y u + (g / r) grad Y(u).
// For the reverse pair, u -> -u gives Y(-u) = (-1)^l Y(u) and
// grad Y(-u) = (-1)^(l-1) grad Y(u), so f_ji is the same contraction with
// Phi_j scaled by (-1)^l, negated.
#include <cuda_bf16.h>

#include "nep_common.cuh"
#include "sh_poly.cuh"

namespace nep {

__host__ __device__ constexpr int l_of(int k) { return k < 3 ? 1 : (k < 8 ? 2 : (k < 15 ? 3 : 4)); }
constexpr int kNLM = 24;
// The FP32 kernels are compiled for 2 and for 3 resident blocks per SM (which caps
// registers per thread); the runtime picks one per handle (autotuned).

// sin(pi x), cos(pi x) for x = r / r_c in [0, 1].  FP32 uses the hardware
// approximations (absolute error below 4e-7 on [0, pi]); FP64 the accurate routine.
__device__ __forceinline__ void sincospi_r(float x, float* s, float* c)
{
    const float t = 3.14159265358979f * x;
    *s = __sinf(t);
    *c = __cosf(t);
}
__device__ __forceinline__ void sincospi_r(double x, double* s, double* c) { sincospi(x, s, c); }

// Chebyshev basis f_k(r) of Eq. 7 with the cutoff of Eq. 8, k = 0..K-1, by the
// three-term recurrence T_{k+1} = 2 x T_k - T_{k-1}.
template <typename real, int K>
__device__ __forceinline__ void basis(real r, real inv_rc, real* f)
{
    real sn, cs;
    sincospi_r(r * inv_rc, &sn, &cs);
    const real hf = real(0.25) + real(0.25) * cs;  // f_c / 2
    const real s = r * inv_rc - real(1);
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

// f_k and df_k/dr:  df_k = 1/2 [T_k'(x) x'(r) f_c + (T_k + 1) f_c'],
// with T'_{k+1} = 2 T_k + 2 x T'_k - T'_{k-1}.
template <typename real, int K>
__device__ __forceinline__ void basis_d(real r, real inv_rc, real* f, real* df)
{
    real sn, cs;
    sincospi_r(r * inv_rc, &sn, &cs);
    const real hf = real(0.25) + real(0.25) * cs;                           // f_c / 2
    const real hdf = real(-0.25 * 3.14159265358979323846) * inv_rc * sn;    // f_c' / 2
    const real s = r * inv_rc - real(1);
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

__device__ __forceinline__ float rsqrt_r(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsqrt_r(double x) { return rsqrt(x); }

template <typename real>
__device__ __forceinline__ void stage_params(const real* __restrict__ src, real* dst, int count)
{
    for (int k = threadIdx.x; k < count; k += blockDim.x) dst[k] = src[k];
    __syncthreads();
}

// ---- the hidden layer (Eq. 2) on the tensor cores (tcgen05), BF16 weights ------
// A block's 128 particles are the 128 rows of two products per type t:
//   X_t = Q W0_t^T        (128 x ND by ND x H: the hidden pre-activations)
//   dQ_t = D W0_t          (128 x H by H x ND: dU/dq, D = w1 (1 - h^2))
// issued by one thread as tcgen05.mma (kind::f16, BF16 operands from shared memory,
// FP32 accumulators in tensor memory).  Each thread writes its own row of Q (then
// of D) into shared memory and reads its own row of X (then dQ) back from tensor
// memory lane threadIdx.x with tcgen05.ld; with several types a warp reads the
// region of each type its lanes hold and every lane keeps its own type's row.  W0 is rounded to BF16 once, on the host; each
// activation is split into a BF16 head and tail (x = hi + lo, exact to about 2^-16
// relative) multiplied as two products, so the result is the FP32 evaluation of
// the model with BF16 weights and the forces stay the gradient of its energy.
//
// Operands use the canonical K-major layout without swizzle: 8 x 8 BF16 core
// matrices of 128 contiguous bytes, 128 bytes apart along K (the descriptor's
// leading offset) and 16 K bytes apart along the rows (its stride offset).

// shared-memory matrix descriptor (K-major, no swizzle)
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, uint32_t sbo)
{
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)(128u >> 4) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// instruction descriptor: FP32 accumulator, BF16 A and B, both K-major, M = 128
__device__ __forceinline__ uint32_t tc_idesc(int n)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t dtmem, uint64_t da, uint64_t db, uint32_t idesc, bool acc)
{
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.u32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
        "l"(da), "l"(db), "r"(idesc), "r"((uint32_t)acc));
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Wait (bounded) for the given phase of an mbarrier; false if it did not complete.
__device__ __forceinline__ bool tc_wait(uint64_t* mbar, uint32_t phase)
{
    uint32_t done = 0;
    for (int it = 0; it < (1 << 24) && !done; ++it)
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(smem_addr(mbar)), "r"(phase));
    return done != 0;
}

// 16 consecutive FP32 columns of this thread's tensor-memory lane
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float (&v)[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int k = 0; k < 16; ++k) v[k] = __uint_as_float(r[k]);
}

// 16 columns at `taddr` + t * stride of the region of type t = ti.  The address of
// tcgen05.ld is warp-wide, so the warp reads the region of every type present
// among its lanes and each lane keeps its own type's.
__device__ __forceinline__ void tc_ld_type(uint32_t taddr, int stride, int T, int ti, float (&v)[16])
{
    if (T == 1) {
        tc_ld16(taddr, v);
        return;
    }
    for (int t = 0; t < T; ++t) {
        if (!__any_sync(0xffffffffu, ti == t)) continue;
        float w[16];
        tc_ld16(taddr + (uint32_t)(t * stride), w);
        if (t == ti)
#pragma unroll
            for (int k = 0; k < 16; ++k) v[k] = w[k];
    }
}

// 8 consecutive K values of one row as BF16 heads and tails (two 16-byte chunks)
__device__ __forceinline__ void tc_put8(unsigned char* hi_row, unsigned char* lo_row, const float* x)
{
    uint32_t h[4], l[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const __nv_bfloat16 h0 = __float2bfloat16_rn(x[2 * k]), h1 = __float2bfloat16_rn(x[2 * k + 1]);
        const __nv_bfloat16 l0 = __float2bfloat16_rn(x[2 * k] - __bfloat162float(h0));
        const __nv_bfloat16 l1 = __float2bfloat16_rn(x[2 * k + 1] - __bfloat162float(h1));
        h[k] = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
        l[k] = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
    }
    *reinterpret_cast<uint4*>(hi_row) = make_uint4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<uint4*>(lo_row) = make_uint4(l[0], l[1], l[2], l[3]);
}

// byte offset of row r, K chunk kc (8 values) in a canonical K-major tile with K columns
__device__ __forceinline__ uint32_t tc_off(int r, int kc, int K)
{
    return (uint32_t)((r >> 3) * (K * 16) + kc * 128 + (r & 7) * 16);
}

// The network of this thread's particle (all 128 threads of the block take part;
// `scratch` is the block's operand area of tc_scratch bytes, 16-byte aligned).
template <int ND>
__device__ __forceinline__ void net_tc(const float* P, const float* __restrict__ gparams, const ParamLayout& off,
                                       int T, int H, int ti, const float (&q)[ND], float& U, float (&dq)[ND],
                                       unsigned char* scratch, int* err)
{
    constexpr int KPF = net_kpf(ND), NDP = net_ndp(ND);
    const int HP = net_hp(H), tid = threadIdx.x, warp = tid >> 5;
    const int cols = tc_cols(T, H);
    // every operand the tensor cores read starts on a 128-byte boundary
    unsigned char* region = scratch + ((128u - (smem_addr(scratch) & 127u)) & 127u);
    unsigned char* A_hi = region;
    unsigned char* A_lo = region + tc_tile(H, ND);  // head and tail tiles
    unsigned char* Wf = region + 2 * tc_tile(H, ND);  // [T][HP x KPF] tiles
    unsigned char* Wb = Wf + (size_t)T * HP * KPF * 2;  // [T][32 x HP] tiles
    uint64_t* mbar = reinterpret_cast<uint64_t*>(region + 2 * tc_tile(H, ND) + tc_wtiles(T, H, ND));
    uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 1);
    {  // W0 tiles from the model's parameters (16-byte copies)
        const uint4* src = reinterpret_cast<const uint4*>(gparams + off.w0f);
        uint4* dst = reinterpret_cast<uint4*>(Wf);
        for (int k = tid; k < tc_wtiles(T, H, ND) / 16; k += blockDim.x) dst[k] = src[k];
    }
    if (tid == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(mbar)));
    // Q: this thread's row, K = KPF
    {
        float v[KPF];
#pragma unroll
        for (int k = 0; k < KPF; ++k) v[k] = k < ND ? q[k] : 0.f;
#pragma unroll
        for (int kc = 0; kc < KPF / 8; ++kc) tc_put8(A_hi + tc_off(tid, kc, KPF), A_lo + tc_off(tid, kc, KPF), v + 8 * kc);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // visible to the tensor cores
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tslot)),
                     "r"(cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;
    if (tid == 0) {  // X_t = Q W0_t^T into columns [t HP, (t + 1) HP)
        const uint32_t idesc = tc_idesc(HP);
        for (int t = 0; t < T; ++t)
            for (int ks = 0; ks < KPF / 16; ++ks)
                for (int part = 0; part < 2; ++part) {
                    const unsigned char* Ap = part ? A_lo : A_hi;
                    tc_mma(tmem + (uint32_t)(t * HP), tc_desc(smem_addr(Ap) + ks * 256, KPF * 16),
                           tc_desc(smem_addr(Wf + (size_t)t * HP * KPF * 2) + ks * 256, KPF * 16), idesc,
                           ks > 0 || part > 0);
                }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_addr(mbar)));
    }
    bool ok = tc_wait(mbar, 0);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // h = tanh(x - b0), the energy, and D = w1 (1 - h^2), 16 hidden units at a time
    const float* b0 = P + off.b0 + ti * H;
    const float* w1 = P + off.w1 + ti * H;
    const uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16);
    float u = 0.f;
    for (int c = 0; c < HP / 16; ++c) {
        float x[16], d[16];
        tc_ld_type(lane_addr + (uint32_t)(16 * c), HP, T, ti, x);
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const int col = 16 * c + k;
            d[k] = 0.f;
            if (col < H) {
                const float h = tanhf(x[k] - b0[col]);
                u += w1[col] * h;
                d[k] = w1[col] * (1.f - h * h);
            }
        }
        tc_put8(A_hi + tc_off(tid, 2 * c, HP), A_lo + tc_off(tid, 2 * c, HP), d);
        tc_put8(A_hi + tc_off(tid, 2 * c + 1, HP), A_lo + tc_off(tid, 2 * c + 1, HP), d + 8);
    }
    U = u - P[off.b1 + ti];
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();  // every X row is read before the columns are reused
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (tid == 0) {  // dQ_t = D W0_t into columns [32 t, 32 t + 32)
        const uint32_t idesc = tc_idesc(32);
        for (int t = 0; t < T; ++t)
            for (int ks = 0; ks < HP / 16; ++ks)
                for (int part = 0; part < 2; ++part) {
                    const unsigned char* Ap = part ? A_lo : A_hi;
                    tc_mma(tmem + (uint32_t)(32 * t), tc_desc(smem_addr(Ap) + ks * 256, HP * 16),
                           tc_desc(smem_addr(Wb + (size_t)t * 32 * HP * 2) + ks * 256, HP * 16), idesc,
                           ks > 0 || part > 0);
                }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_addr(mbar)));
    }
    ok = tc_wait(mbar, 1) && ok;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
    for (int c = 0; c < NDP / 16 + (NDP % 16 ? 1 : 0); ++c) {
        float v[16];
        tc_ld_type(lane_addr + (uint32_t)(16 * c), 32, T, ti, v);
#pragma unroll
        for (int k = 0; k < 16; ++k)
            if (16 * c + k < ND) dq[16 * c + k] = v[k];
    }
    if (!ok) {  // a wait ran out: report it and poison this particle's results
        if (err) atomicOr(err, 4);
        U = __int_as_float(0x7fc00000);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(cols));
}

template <typename real, int NR, int NA, int KR, int KA, int MB, int NET = 0>
__global__ void __launch_bounds__(kBlock, sizeof(real) == 4 ? MB : 1) k_descriptor(EvalArgs<real> a)
{
    constexpr int ND = NR + NA * 4;
    constexpr int KRP = (KR + 3) & ~3;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    real* P = reinterpret_cast<real*>(smem_raw);
    const WorkItem it = a.items[blockIdx.x];
    const ReqInfo& rq = a.reqs[it.req];
    const ModelDesc<real> md = a.models[rq.model];
    const ParamLayout off = md.off;
    // NET = 1 keeps the BF16 weight tiles out of the staged prefix (they are copied
    // to an aligned operand area instead)
    const int staged = NET == 1 ? off.w0f : off.total;
    stage_params(md.params, P, staged);
    // NET = 1 evaluates the network block-wide: a lane past the item's end follows
    // the item's last particle and writes nothing
    const bool live = NET == 0 || it.begin + (int)threadIdx.x < it.end;
    const int i = live ? it.begin + threadIdx.x : it.end - 1;
    if (NET == 0 && i >= it.end) return;
    if (live && a.acc) {  // the scatter accumulators of i start the force pass at zero
        ulonglong2* z = reinterpret_cast<ulonglong2*>(a.acc + (size_t)i * 16);
#pragma unroll
        for (int k = 0; k < 6; ++k) z[k] = make_ulonglong2(0ull, 0ull);
    }
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
        // one pair type: q_n = sum_k c_nk (sum_j f_k(r_ij)), contracted once per bead
        real fs[KR];
#pragma unroll
        for (int k = 0; k < KR; ++k) fs[k] = real(0);
        const real inv_rc = P[off.rcRi];
        walk4(a.nlR + i, (size_t)a.n, cR, [&](uint32_t e) {
            const PosRec<real> rj = a.rec[e & kJMask];
            real dx, dy, dz;
            pair_vec(len, ri, rj, e, dx, dy, dz);
            const real r2 = dx * dx + dy * dy + dz * dz;
            const real r = r2 * rsqrt_r(r2);
            real f[KR];
            basis<real, KR>(r, inv_rc, f);
#pragma unroll
            for (int k = 0; k < KR; ++k) fs[k] += f[k];
        });
        const real* c = P + off.cR;
#pragma unroll
        for (int nn = 0; nn < NR; ++nn) {
            real g = real(0);
#pragma unroll
            for (int k = 0; k < KR; ++k) g += c[nn * KR + k] * fs[k];
            q[nn] = g;
        }
    } else {
        walk4(a.nlR + i, (size_t)a.n, cR, [&](uint32_t e) {
            const PosRec<real> rj = a.rec[e & kJMask];
            real dx, dy, dz;
            pair_vec(len, ri, rj, e, dx, dy, dz);
            const real r2 = dx * dx + dy * dy + dz * dz;
            const real r = r2 * rsqrt_r(r2);
            const int tp = ti * T + rj.t;
            real f[KR];
            basis<real, KR>(r, P[off.rcRi + tp], f);
            const real* c = P + off.cR + tp * NR * KR;
#pragma unroll
            for (int nn = 0; nn < NR; ++nn) {
                real g = real(0);
#pragma unroll
                for (int k = 0; k < KR; ++k) g += c[nn * KR + k] * f[k];
                q[nn] += g;
            }
        });
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
        basis<real, KA>(r, P[off.rcAi + tp], f);
        const real* c = P + off.cA + tp * NA * KA;
        real Y[kNLM];
        sh_eval(dx * inv_r, dy * inv_r, dz * inv_r, Y);
#pragma unroll
        for (int nn = 0; nn < NA; ++nn) {
            real g = real(0);
#pragma unroll
            for (int k = 0; k < KA; ++k) g += c[nn * KA + k] * f[k];
#pragma unroll
            for (int k = 0; k < kNLM; ++k) A[nn][k] += g * Y[k];
        }
    }
    // q_nl (Eq. 4)
#pragma unroll
    for (int nn = 0; nn < NA; ++nn)
#pragma unroll
        for (int k = 0; k < kNLM; ++k) q[NR + (l_of(k) - 1) * NA + nn] += A[nn][k] * A[nn][k];

    // ---- network (Eq. 2) and dU/dq ----
    real U;
    real dq[ND];
    if constexpr (NET == 1) {
        unsigned char* scratch = smem_raw + (((size_t)staged * sizeof(real) + 15) & ~(size_t)15);
        net_tc<ND>(P, md.params, off, T, H, ti, q, U, dq, scratch, a.err);
        if (!live) return;
    } else {
        const real* w0 = P + off.w0 + ti * H * ND;
        const real* b0 = P + off.b0 + ti * H;
        const real* w1 = P + off.w1 + ti * H;
        U = -P[off.b1 + ti];
#pragma unroll
        for (int v = 0; v < ND; ++v) dq[v] = real(0);
        for (int mu = 0; mu < H; ++mu) {
            real x = -b0[mu];
#pragma unroll
            for (int v = 0; v < ND; ++v) x += w0[mu * ND + v] * q[v];
            const real h = tanh(x);
            U += w1[mu] * h;
            const real coef = w1[mu] * (real(1) - h * h);
#pragma unroll
            for (int v = 0; v < ND; ++v) dq[v] += coef * w0[mu * ND + v];
        }
    }
    a.U[i] = U;
    // e_i^t[k] = sum_n dU/dq_n c^{t_i t}_{nk}
    real* ei = a.e + (size_t)i * a.e_stride;
    for (int t = 0; t < T; ++t) {
        const real* c = P + off.cR + (ti * T + t) * NR * KR;
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
    // Phi is stored component-major, [24][n][NAP]: for one component the rows of
    // consecutive particles are adjacent, so a warp's row loads are contiguous
    constexpr int NAP = phi_pad(NA);
    real* ph = a.phi + (size_t)i * NAP;
    const size_t kstride = (size_t)a.n * NAP;
#pragma unroll
    for (int k = 0; k < kNLM; ++k)
#pragma unroll
        for (int nn = 0; nn < NAP; ++nn)
            ph[k * kstride + nn] = nn < NA ? real(2) * dq[NR + (l_of(k) - 1) * NA + nn] * A[nn][k] : real(0);
}

template <typename real>
__device__ __forceinline__ real warp_sum(real v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// FP64 block partials of (E, W[9]); the last block of a request sums its request's
// partials in item order (deterministic) into totals[req].
template <int BS>
__device__ __forceinline__ void reduce_totals(double (&v)[10], const WorkItem& it, const ReqInfo& rq,
                                              double* partial, unsigned int* counter, double* totals)
{
    __shared__ double red[BS / 32][10];
    __shared__ bool last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 10; ++k) {
        const double s = warp_sum(v[k]);
        if (lane == 0) red[warp][k] = s;
    }
    __syncthreads();
    if (threadIdx.x < 10) {
        double s = 0.0;
#pragma unroll
        for (int w = 0; w < BS / 32; ++w) s += red[w][threadIdx.x];
        partial[(size_t)blockIdx.x * 10 + threadIdx.x] = s;
    }
    __threadfence();
    __syncthreads();
    const unsigned int n_items = (unsigned int)(rq.item_end - rq.item_begin);
    if (threadIdx.x == 0) last = (atomicAdd(&counter[it.req], 1u) == n_items - 1);
    __syncthreads();
    if (!last) return;
    __threadfence();
    if (threadIdx.x < 10) {
        double s = 0.0;
        const volatile double* p = partial;
        for (int b = rq.item_begin; b < rq.item_end; ++b) s += p[(size_t)b * 10 + threadIdx.x];
        totals[(size_t)it.req * 10 + threadIdx.x] = s;
    }
    if (threadIdx.x == 0) counter[it.req] = 0u;
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

// Per-thread state of the force pass for one particle i.
template <typename real, int KRP>
struct ForceCtx {
    PosRec<real> ri;
    int i, ti, T;
    real len[3];
    real F[3];
    real W[9];
};

// Radial pairs of slots s0, s0 + ds, ... :
//   f_ij = (e_i^{t_j} . f') u,  f_ji = -(e_j^{t_i} . f') u,  F_i += f_ij - f_ji,
//   W_i += r_ij (x) f_ji.  The pair body has no branch, so the scheduler can
//   interleave the four bodies of each walk step.
template <typename real, int NR, int KR>
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
        basis_d<real, KR>(r, P[off.rcRi + ti * T + rj.t], f, df);
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
        const real d[3] = {dx, dy, dz}, u[3] = {ux, uy, uz};
#pragma unroll
        for (int p = 0; p < 3; ++p) {
            const real bd = bj * d[p];
#pragma unroll
            for (int q = 0; q < 3; ++q) c.W[3 * p + q] -= bd * u[q];
        }
    };
    const uint32_t* nl = a.nlR + (size_t)s0 * a.n + c.i;
    const size_t stride = (size_t)ds * a.n;
    if (T == 1) {
        real ei1[KRP];  // the one partner type's vector
        loadN<real, KRP>(e_i, ei1);
        walk4(nl, stride, cnt, [&](uint32_t e) { radial_pair(e, ei1); });
    } else {
        walk4(nl, stride, cnt, [&](uint32_t e) {
            real eij[KRP];
            loadN<real, KRP>(e_i + a.rec[e & kJMask].t * KRP, eij);
            radial_pair(e, eij);
        });
    }
}

// Angular pairs, harmonic components k in [K0, K1) of every pair.  For
// A = g(r) Y(u): dA/dr = (g' - l g / r) Y u + (g / r) grad Y; the reverse pair uses
// Y(-u) = (-1)^l Y(u), so f_ji is the same contraction with Phi_j (-1)^l, negated.
template <typename real, int NA, int KA, int K0, int K1, typename Ctx>
__device__ __forceinline__ void force_angular_k(const EvalArgs<real>& a, const real* P, const ParamLayout& off,
                                                Ctx& c)
{
    const int T = c.T, ti = c.ti;
    constexpr int NAP = phi_pad(NA);
    const size_t kstride = (size_t)a.n * NAP;
    const real* phi_i = a.phi + (size_t)c.i * NAP;
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
        basis_d<real, KA>(r, P[off.rcAi + tij], f, df);
        real gi[NA], dgi[NA], gj[NA], dgj[NA];
        {
            const real* cc = P + off.cA + tij * NA * KA;
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
            const real* cc = P + off.cA + tji * NA * KA;
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
        const ShMono<real> mono = sh_mono(ux, uy, uz);
        const real* phi_j = a.phi + (size_t)j * NAP;
        real si = real(0), sj = real(0);
        real ga[3] = {real(0), real(0), real(0)}, gb[3] = {real(0), real(0), real(0)};
#pragma unroll
        for (int k = K0; k < K1; ++k) {
            const real lr = real(l_of(k)) * inv_r;
            real pi_[NA], pj[NA];
            loadN<real, NA>(phi_i + k * kstride, pi_);
            loadN<real, NA>(phi_j + k * kstride, pj);
            real Gi_ = real(0), dGi = real(0), Gj_ = real(0), dGj = real(0);
#pragma unroll
            for (int nn = 0; nn < NA; ++nn) {
                Gi_ += pi_[nn] * gi[nn];
                dGi += pi_[nn] * dgi[nn];
                Gj_ += pj[nn] * gj[nn];
                dGj += pj[nn] * dgj[nn];
            }
            if (l_of(k) & 1) {
                Gj_ = -Gj_;
                dGj = -dGj;
            }
            real y, gx, gy, gz;
            sh_val_grad(k, mono, y, gx, gy, gz);
            si += (dGi - lr * Gi_) * y;
            sj += (dGj - lr * Gj_) * y;
            const real Gs = Gi_ + Gj_;
            ga[0] += Gs * gx;
            ga[1] += Gs * gy;
            ga[2] += Gs * gz;
            gb[0] += Gj_ * gx;
            gb[1] += Gj_ * gy;
            gb[2] += Gj_ * gz;
        }
        // F_i += f_ij - f_ji;  -f_ji = sj u + gb / r;  W_i += r_ij (x) f_ji
        const real u[3] = {ux, uy, uz}, d[3] = {dx, dy, dz};
        real vj[3];
#pragma unroll
        for (int p = 0; p < 3; ++p) {
            c.F[p] += (si + sj) * u[p] + ga[p] * inv_r;
            vj[p] = sj * u[p] + gb[p] * inv_r;
        }
#pragma unroll
        for (int p = 0; p < 3; ++p)
#pragma unroll
            for (int q = 0; q < 3; ++q) c.W[3 * p + q] -= d[p] * vj[q];
    }
}

template <typename real>
__device__ __forceinline__ void force_outputs(const EvalArgs<real>& a, const ReqInfo& rq, int i, const real* F,
                                              const real* W, double (&tot)[10])
{
    const int ui = a.perm[i];
    const int lu = ui - rq.begin;  // index within the request's output blocks
    const real Ui = a.U[i];
    double* fo = a.force + (size_t)3 * rq.begin + lu;
#pragma unroll
    for (int p = 0; p < 3; ++p) fo[(size_t)p * rq.n] = (double)F[p];
    if (a.virial) {
        double* vo = a.virial + (size_t)9 * rq.begin + lu;
#pragma unroll
        for (int k = 0; k < 9; ++k) vo[(size_t)k * rq.n] = (double)W[k];
    }
    if (a.site) a.site[ui] = (double)Ui;
    tot[0] = (double)Ui;
#pragma unroll
    for (int k = 0; k < 9; ++k) tot[1 + k] = (double)W[k];
}

// One thread per particle.
template <typename real, int NR, int NA, int KR, int KA, int MB>
__global__ void __launch_bounds__(kBlock, sizeof(real) == 4 ? MB : 1) k_force(EvalArgs<real> a)
{
    constexpr int KRP = (KR + 3) & ~3;
    // i's Phi is read through L1 (a shared-memory copy would take L1 capacity that
    // the neighbours' records and gradients need more)
    extern __shared__ __align__(16) unsigned char smem_raw[];
    real* P = reinterpret_cast<real*>(smem_raw);
    const WorkItem it = a.items[blockIdx.x];
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
        force_angular_k<real, NA, KA, 0, kNLM>(a, P, off, c);
        force_outputs(a, rq, i, c.F, c.W, tot);
    }
    reduce_totals<kBlock>(tot, it, rq, a.partial, a.counter, a.totals);
}

// ---- FP32 scatter form -----------------------------------------------------------
// Each ordered angular pair is evaluated once, by the thread of its centre i, which
// contracts only Phi_i: f_ij = dU_i/dr_ij.  F_i gains f_ij in registers; F_j loses
// it and W_j gains r_ji (x) f_ij through 64-bit fixed-point atomic adds.  Integer
// sums do not depend on the order in which the adds arrive, so the results stay
// bitwise reproducible.  The radial pairs stay in gather form (their reverse term
// needs only j's 8-entry gradient vector).
constexpr float kFixScale = 4294967296.0f;  // 2^32 fixed-point units per eV/A (or eV)
constexpr double kFixUnit = 1.0 / 4294967296.0;

__device__ __forceinline__ void fix_add(unsigned long long* p, float v)
{
    atomicAdd(p, (unsigned long long)__float2ll_rn(v * kFixScale));
}

__device__ __forceinline__ double fix_value(unsigned long long v) { return (double)(long long)v * kFixUnit; }

__device__ __forceinline__ float mul_rn(float x, float y) { return __fmul_rn(x, y); }
__device__ __forceinline__ double mul_rn(double x, double y) { return __dmul_rn(x, y); }

template <typename real, int NA, int KA, typename Ctx>
__device__ __forceinline__ void force_angular_scatter(const EvalArgs<real>& a, const real* P, const ParamLayout& off,
                                                      Ctx& c, bool per_bead)
{
    const int T = c.T, ti = c.ti;
    constexpr int NAP = phi_pad(NA);
    const size_t kstride = (size_t)a.n * NAP;
    const real* phi_i = a.phi + (size_t)c.i * NAP;
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
        basis_d<real, KA>(r, P[off.rcAi + tij], f, df);
        real g[NA], dg[NA];
        const real* cc = P + off.cA + tij * NA * KA;
#pragma unroll
        for (int nn = 0; nn < NA; ++nn) {
            real s0 = real(0), s1 = real(0);
#pragma unroll
            for (int k = 0; k < KA; ++k) {
                s0 += cc[nn * KA + k] * f[k];
                s1 += cc[nn * KA + k] * df[k];
            }
            g[nn] = s0;
            dg[nn] = s1;
        }
        const real ux = dx * inv_r, uy = dy * inv_r, uz = dz * inv_r;
        const ShMono<real> mono = sh_mono(ux, uy, uz);
        real sr = real(0);
        real ga[3] = {real(0), real(0), real(0)};
#pragma unroll
        for (int k = 0; k < kNLM; ++k) {
            real pi_[NA];
            loadN<real, NA>(phi_i + k * kstride, pi_);
            real G = real(0), dG = real(0);
#pragma unroll
            for (int nn = 0; nn < NA; ++nn) {
                G += pi_[nn] * g[nn];
                dG += pi_[nn] * dg[nn];
            }
            real y, gx, gy, gz;
            sh_val_grad(k, mono, y, gx, gy, gz);
            sr += (dG - real(l_of(k)) * inv_r * G) * y;
            ga[0] += G * gx;
            ga[1] += G * gy;
            ga[2] += G * gz;
        }
        const real fij[3] = {sr * ux + ga[0] * inv_r, sr * uy + ga[1] * inv_r, sr * uz + ga[2] * inv_r};
        unsigned long long* acc_j = a.acc + (size_t)j * 16;
#pragma unroll
        for (int p = 0; p < 3; ++p) {
            c.F[p] += fij[p];
            fix_add(acc_j + p, -fij[p]);
        }
        const real d[3] = {dx, dy, dz};
#pragma unroll
        for (int p = 0; p < 3; ++p)
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                // W_j += r_ji (x) f_ij; the product is rounded on its own so that the
                // totals do not depend on whether it is also scattered
                const real w = mul_rn(-d[p], fij[q]);
                c.W[3 * p + q] += w;  // c.W feeds only the totals here
                if (per_bead) fix_add(acc_j + 3 + 3 * p + q, w);
            }
    }
}

// One thread per particle: radial pairs in gather form, angular pairs scattered.
// Without per-particle virial output only the force is scattered; the virial
// contributions of a thread's pairs go straight into the FP64 totals.
template <typename real, int NR, int NA, int KR, int KA, int MB>
__global__ void __launch_bounds__(kBlock, MB) k_force_scatter(EvalArgs<real> a)
{
    constexpr int KRP = (KR + 3) & ~3;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    real* P = reinterpret_cast<real*>(smem_raw);
    const WorkItem it = a.items[blockIdx.x];
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
        unsigned long long* acc_i = a.acc + (size_t)i * 16;
        const bool per_bead = a.virial != nullptr;
        if (per_bead)  // W_i's radial part is complete here
#pragma unroll
            for (int k = 0; k < 9; ++k) fix_add(acc_i + 3 + k, c.W[k]);
        force_angular_scatter<real, NA, KA>(a, P, off, c, per_bead);
#pragma unroll
        for (int p = 0; p < 3; ++p) fix_add(acc_i + p, c.F[p]);
        const real Ui = a.U[i];
        if (a.site) a.site[a.perm[i]] = (double)Ui;
        tot[0] = (double)Ui;
#pragma unroll
        for (int k = 0; k < 9; ++k) tot[1 + k] = (double)c.W[k];
    }
    reduce_totals<kBlock>(tot, it, rq, a.partial, a.counter, a.totals);
}

// The accumulated F_i (and W_i) to the caller-order FP64 outputs.
template <typename real>
__global__ void __launch_bounds__(kBlock) k_scatter_outputs(EvalArgs<real> a)
{
    const WorkItem it = a.items[blockIdx.x];
    const ReqInfo& rq = a.reqs[it.req];
    const int i = it.begin + threadIdx.x;
    if (i >= it.end) return;
    const ulonglong2* acc = reinterpret_cast<const ulonglong2*>(a.acc + (size_t)i * 16);
    const int lu = a.perm[i] - rq.begin;
    const ulonglong2 w01 = acc[0], w23 = acc[1];
    double* fo = a.force + (size_t)3 * rq.begin + lu;
    fo[0] = fix_value(w01.x);
    fo[rq.n] = fix_value(w01.y);
    fo[(size_t)2 * rq.n] = fix_value(w23.x);
    if (a.virial) {
        double* vo = a.virial + (size_t)9 * rq.begin + lu;
        vo[0] = fix_value(w23.y);
#pragma unroll
        for (int q = 2; q < 6; ++q) {  // words 2q, 2q + 1 are W[2q - 3], W[2q - 2]
            const ulonglong2 w = acc[q];
            vo[(size_t)(2 * q - 3) * rq.n] = fix_value(w.x);
            vo[(size_t)(2 * q - 2) * rq.n] = fix_value(w.y);
        }
    }
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

template <typename real>
cudaError_t evaluate_set_smem(int nR, int nA, int KR, int KA, size_t smem_desc, size_t smem_force)
{
#define NEP_SET(a_, b_, c_, d_, mb_)                                                                          \
    {                                                                                                         \
        cudaError_t e = cudaFuncSetAttribute(k_descriptor<real, a_, b_, c_, d_, mb_>,                         \
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_desc);    \
        if (e != cudaSuccess) return e;                                                                       \
        if constexpr (sizeof(real) == 4) {                                                                    \
            e = cudaFuncSetAttribute(k_descriptor<real, a_, b_, c_, d_, mb_, 1>,                              \
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_desc);            \
            if (e != cudaSuccess) return e;                                                                   \
        }                                                                                                     \
        if constexpr (sizeof(real) == 4)                                                                      \
            e = cudaFuncSetAttribute(k_force_scatter<real, a_, b_, c_, d_, mb_>,                              \
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_force);           \
        else                                                                                                  \
            e = cudaFuncSetAttribute(k_force<real, a_, b_, c_, d_, mb_>,                                      \
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_force);           \
        if (e != cudaSuccess) return e;                                                                       \
    }
#define NEP_CASE(a_, b_, c_, d_)                                  \
    if (nR == a_ && nA == b_ && KR == c_ && KA == d_) {           \
        NEP_SET(a_, b_, c_, d_, 2)                                \
        NEP_SET(a_, b_, c_, d_, 3)                                \
        return cudaSuccess;                                       \
    }
    NEP_SHAPES(NEP_CASE)
#undef NEP_CASE
#undef NEP_SET
    return cudaErrorInvalidValue;
}

template <typename real>
cudaError_t launch_evaluate(int nR, int nA, int KR, int KA, const EvalArgs<real>& a, int n_items, size_t smem_desc,
                            size_t smem_force, cudaStream_t st, cudaEvent_t mid, int mb_desc, int mb_force)
{
    const int nb = n_items;
    if constexpr (sizeof(real) == 4) {
        if (!a.acc) return cudaErrorInvalidValue;  // the FP32 form scatters into a.acc
    }
#define NEP_CASE(a_, b_, c_, d_)                                                                            \
    if (nR == a_ && nA == b_ && KR == c_ && KA == d_) {                                                     \
        if (sizeof(real) == 4 && a.net_bf16) {                                                              \
            if constexpr (sizeof(real) == 4) {                                                              \
                if (mb_desc == 2) k_descriptor<real, a_, b_, c_, d_, 2, 1><<<nb, kBlock, smem_desc, st>>>(a); \
                else k_descriptor<real, a_, b_, c_, d_, 3, 1><<<nb, kBlock, smem_desc, st>>>(a);            \
            }                                                                                               \
        } else if (mb_desc == 2) {                                                                          \
            k_descriptor<real, a_, b_, c_, d_, 2><<<nb, kBlock, smem_desc, st>>>(a);                        \
        } else {                                                                                            \
            k_descriptor<real, a_, b_, c_, d_, 3><<<nb, kBlock, smem_desc, st>>>(a);                        \
        }                                                                                                   \
        if (mid) cudaEventRecord(mid, st);                                                                  \
        if constexpr (sizeof(real) == 4) {                                                                  \
            if (mb_force == 3) k_force_scatter<real, a_, b_, c_, d_, 3><<<nb, kBlock, smem_force, st>>>(a); \
            else k_force_scatter<real, a_, b_, c_, d_, 2><<<nb, kBlock, smem_force, st>>>(a);               \
            k_scatter_outputs<real><<<nb, kBlock, 0, st>>>(a);                                              \
        } else {                                                                                            \
            if (mb_force == 3) k_force<real, a_, b_, c_, d_, 3><<<nb, kBlock, smem_force, st>>>(a);         \
            else k_force<real, a_, b_, c_, d_, 2><<<nb, kBlock, smem_force, st>>>(a);                       \
        }                                                                                                   \
        return cudaGetLastError();                                                                          \
    }
    NEP_SHAPES(NEP_CASE)
#undef NEP_CASE
    return cudaErrorInvalidValue;
}

#define NEP_INSTANTIATE(real)                                                                             \
    template bool evaluate_shape_supported<real>(int, int, int, int);                                     \
    template cudaError_t evaluate_set_smem<real>(int, int, int, int, size_t, size_t);                     \
    template cudaError_t launch_evaluate<real>(int, int, int, int, const EvalArgs<real>&, int, size_t, size_t, \
                                               cudaStream_t, cudaEvent_t, int, int);
NEP_INSTANTIATE(float)
NEP_INSTANTIATE(double)
#undef NEP_INSTANTIATE

}  // namespace nep
