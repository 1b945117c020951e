// Internal definitions shared by the CUDA translation units of the NEP library.
//
// Every kernel works on a batch of requests (configurations).  The particles of
// all requests are concatenated; request r owns [begin, begin + n).  Each request
// has its own box, cell grid (its cells are numbered from cell_base in one global
// cell numbering) and model.  Work is cut into work items: up to kBlock particles
// of one request, one thread block per item, so a block stages one model's tables
// and contributes to one request's FP64 totals.  A single configuration is a
// batch of one request.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>

namespace nep {

// Launch helper: the kernels of the evaluation and MD pipeline are launched
// through cudaLaunchKernelEx, which returns launch errors directly.
template <typename... P, typename... A>
inline cudaError_t launch_k(void (*kernel)(P...), int grid, int block, size_t smem, cudaStream_t st,
                              A&&... args)
{
    cudaLaunchConfig_t c = {};
    c.gridDim = dim3((unsigned)grid);
    c.blockDim = dim3((unsigned)block);
    c.dynamicSmemBytes = smem;
    c.stream = st;
    c.numAttrs = 0;
    return cudaLaunchKernelEx(&c, kernel, std::forward<A>(args)...);
}

// A neighbour entry packs the sorted index j (low 23 bits) and the cell offset
// (dx, dy, dz) in [-2, 2]^3 of j's cell relative to i's cell (3 bits each).
constexpr int kJBits = 23;
constexpr uint32_t kJMask = (1u << kJBits) - 1u;
constexpr int kMaxN = (1 << kJBits) - 1;
constexpr int kMaxS = 2;
constexpr int kMaxTypes = 16;
constexpr int kBlock = 128;          // threads per block = particles per work item
constexpr int kScanItems = 4096;     // cells per block of the scan

// BF16 network tables (the hidden layer as two tensor-core products per warp of
// 32 particles): padded sizes in BF16 elements.
__host__ __device__ constexpr int net_kpf(int nd) { return (nd + 15) & ~15; }  // K of X = Q W0^T
__host__ __device__ constexpr int net_sf(int nd) { return net_kpf(nd) + 8; }    // row stride (bank spread)
__host__ __device__ constexpr int net_ndp(int nd) { return (nd + 7) & ~7; }     // N of dQ = D W0
__host__ __device__ constexpr int net_hp(int h) { return (h + 15) & ~15; }       // N of X, K of dQ
// per-warp shared scratch of the BF16 network, bytes
__host__ __device__ constexpr int net_scratch(int nd)
{
    // two BF16 tiles of Q (head, tail), later one FP32 tile of dQ
    return (2 * 32 * net_sf(nd) * 2 > 32 * (net_ndp(nd) + 1) * 4 ? 2 * 32 * net_sf(nd) * 2
                                                                   : 32 * (net_ndp(nd) + 1) * 4);
}

// Distance (elements) between the type pairs' coefficient tables of n x K entries:
// odd, so that lanes reading different pairs' tables hit different shared-memory
// banks.  A compile-time function of the shape, used alike by host and kernels.
__host__ __device__ constexpr int coef_stride(int n, int k) { return (n * k) | 1; }

// Row length of Phi_i per harmonic component: n_A padded to a multiple of 4 so that
// every row starts on a 16-byte boundary (vector loads).
__host__ __device__ constexpr int phi_pad(int nA) { return (nA + 3) & ~3; }
// Coefficients per n of the sphere-reduced form of sum_k dU/dA_nk Y_k, the FP64 form's
// per-particle angular adjoint (the kShRed of sh_poly.cuh)
constexpr int kPsiComp = 25;

__host__ __device__ inline uint32_t pack_entry(int j, int dx, int dy, int dz)
{
    return (uint32_t)j | ((uint32_t)((dx + 2) | ((dy + 2) << 3) | ((dz + 2) << 6)) << kJBits);
}

// Cell-relative position of a particle and its type.  The position is stored
// relative to the origin of the particle's cell, so that pair vectors built as
// (x_j - x_i) + offset * cell_len keep full precision in FP32 in any box size.
template <typename real>
struct alignas(4 * sizeof(real)) PosRec {
    real x, y, z;
    int t;
};

static_assert(sizeof(PosRec<float>) == 16 && sizeof(PosRec<double>) == 32, "record layout");

// A record through the read-only data path (the records do not change while a
// kernel reads them).
__device__ __forceinline__ PosRec<float> ldg_rec(const PosRec<float>* p)
{
    const float4 v = __ldg(reinterpret_cast<const float4*>(p));
    PosRec<float> r;
    r.x = v.x;
    r.y = v.y;
    r.z = v.z;
    r.t = __float_as_int(v.w);
    return r;
}
__device__ __forceinline__ PosRec<double> ldg_rec(const PosRec<double>* p)
{
    const double2* q = reinterpret_cast<const double2*>(p);
    const double2 a = __ldg(q), b = __ldg(q + 1);
    PosRec<double> r;
    r.x = a.x;
    r.y = a.y;
    r.z = b.x;
    r.t = (int)(unsigned int)(__double_as_longlong(b.y) & 0xffffffffll);  // t is the word's low half
    return r;
}

// Cell grid of one configuration.
struct CellGrid {
    int nc[3];      // cells per axis
    int S[3];       // search range in cells per axis
    int pbc[3];
    int ncell;
    double len[3];      // cell side
    double inv_len[3];  // 1 / len (cell index by multiplication)
    double box[3];
};

// Wrap onto a periodic axis of length L: positions already in [0, L) are kept;
// others become x - L floor(x / L), and a result that rounds to L (or below 0)
// becomes 0.  Moving particles leave the box rarely, so the FP64 division (slow
// on this GPU) runs only for the few outside.  On the device the range test
// compares bit patterns: for L > 0, 0 <= x < L exactly when x's bits, read as an
// unsigned integer, are below L's (negative x, -0 and NaN have larger patterns),
// which keeps the test off the FP64 pipe.
__host__ __device__ inline double wrap_periodic(double x, double L)
{
#ifdef __CUDA_ARCH__
    if ((unsigned long long)__double_as_longlong(x) < (unsigned long long)__double_as_longlong(L)) return x;
#else
    if (x >= 0.0 && x < L) return x;
#endif
    x = x - L * floor(x / L);
    return (x >= L || x < 0.0) ? 0.0 : x;
}

// x is neither infinite nor NaN (exponent bits not all set), by integer test
__device__ __forceinline__ bool finite_bits(double x)
{
    return ((unsigned long long)__double_as_longlong(x) & 0x7ff0000000000000ull) != 0x7ff0000000000000ull;
}

// Per-type values passed by value to the integration kernels (at most 16 types).
constexpr int kMdMaxTypes = 16;
struct TypeTable {
    double v[kMdMaxTypes];
};

// Velocity-Verlet half-kick and drift of one coordinate, as every integration
// kernel forms them (explicit FMAs, so fused and separate kernels round alike).
__device__ __forceinline__ double half_kick(double v, double half_dt, double f, double im)
{
    return fma(half_dt * f, im, v);
}
__device__ __forceinline__ double drift(double x, double dt, double v) { return fma(dt, v, x); }

// Offsets (in elements of `real`) of the model tables inside one device buffer.
struct ParamLayout {
    int rcR2, rcA2, rcRi, rcAi; // [T][T] each: squared and inverse cutoffs
    int rcRl, rcAl;             // [T][T] each: rounding residuals of the inverse cutoffs
                                // (1/r_c - rcRi in FP32; zero in FP64)
    int cR, cA;                 // [T][T] tables of [nR][KR] and [nA][KA], coef_stride apart
    int w0, b0, w1, b1;         // [T][H][ND], [T][H], [T][H], [T]
    int w0l, b0l, w1l, b1l;     // FP32 form: the rounding residuals x - (float)x of w0, b0, w1, b1
                                // (same layouts; -1 in the FP64 form)
    int cRl;                    // FP32 form: residuals of the cR tables (-1 in the FP64 form)
    int w0f, w0b;               // BF16-weight network form: W0 as BF16 MMA operands (-1 when absent),
                                // [T][net_hp(H)][net_sf(ND)] and [T][net_ndp(ND)][net_hp(H) + 8]
    int n_cut_coef;             // elements of the cutoff + coefficient prefix
    int total;                  // all elements
};

// One model of a batch (device table).
template <typename real>
struct ModelDesc {
    const real* params;
    ParamLayout off;
    int T, H;
};

// One request of a batch (device table).
struct ReqInfo {
    CellGrid g;
    int cell_base;              // first global cell of this request
    int begin, n;               // particle range in the concatenated arrays
    int model;                  // index into the model table
    int item_begin, item_end;   // work items of this request
};

// One block of work: particles [begin, end) of request `req` (end - begin <= kBlock).
struct WorkItem {
    int req, begin, end;
};

// Sizes of the batch in progress, in device memory ahead of its tables.  The
// kernels take their loop bounds from here and loop over work items with a grid
// stride, so launch shapes depend only on capacities: one captured CUDA graph then
// serves every batch that fits them.
struct PlanCounts {
    int n, n_items, ncell, n_req;
};

template <typename real>
struct NeighborArgs {
    int n, mnR, mnA;            // n: the list stride (particle capacity)
    const PlanCounts* counts;
    const WorkItem* items;
    const ReqInfo* reqs;
    const ModelDesc<real>* models;
    const int* cell_start;      // [ncell_total + 1]
    const int* cell_s;          // [n] global cell of sorted particle
    const PosRec<real>* rec;    // [n] sorted
    uint32_t* nlR;              // [mnR][n]
    uint32_t* nlA;              // [mnA][n]
    int* cntR;                  // [n]
    int* cntA;                  // [n]
    int* maxcnt;                // [2]
    unsigned long long* accF;   // FP32 form: [n][4] fixed-point force lines, zeroed here for the evaluation (or null)
    unsigned long long* accW;   // FP32 form with per-particle virials: [n][12] fixed-point virial lines (or null)
    PosRec<float>* rec32 = nullptr;  // FP64 form: FP32 copies of rec, written here to screen the
                                     // distance tests (null: every test in FP64)
};

// Shared memory of the neighbour kernels for T types: the squared cutoffs of both
// lists, and in FP64 their FP32 screening bounds (see neighbors_item).
template <typename real>
constexpr size_t neighbor_smem(int T)
{
    return (2 * sizeof(real) + (sizeof(real) == 8 ? 4 * sizeof(float) : 0)) * (size_t)T * (size_t)T;
}

// Work items per group of the totals' two-level reduction (see reduce_totals).
constexpr int kGroup = 32;

// Bits of the error word (flags[2]): 1 a non-finite position, 2 a type out of range
// (both input errors), kErrCellList an index derived from the cell list that falls
// outside its array.  The last cannot arise from any input; the kernels that check
// for it skip the access, so an internal inconsistency fails the call instead of
// touching memory out of bounds.
constexpr int kErrCellList = 4;

template <typename real>
struct EvalArgs {
    int n, mnR, mnA;            // n: the list / array stride (particle capacity)
    const PlanCounts* counts;
    const WorkItem* items;
    const ReqInfo* reqs;
    const ModelDesc<real>* models;
    const PosRec<real>* rec;    // [n] sorted
    const uint32_t* nlR;
    const uint32_t* nlA;
    const int* cntR;
    const int* cntA;
    real* U;                    // [n] sorted site energies
    real* e;                    // [n][e_stride] radial gradient folded into the basis
    int e_stride;               // Tmax * KRP
    real* phi;                  // FP64 form: [kPsiComp][n][phi_pad(NA)] the sphere-reduced coefficients of
                                // P_n = sum_lm (dU/dA_nlm) Y_lm, zero padded
    int net_bf16;               // 1: the hidden layer's products in BF16 on tensor cores
    int many_body;              // 1: the four- and five-body descriptors follow the three-body ones
    const int* perm;            // sorted slot -> caller index
    double* force;              // per request [3][n_r] blocks (required)
    double* virial;             // per request [9][n_r] blocks, or null
    double* site;               // [n] or null
    unsigned long long* accF;   // FP32 form: [n][4] fixed-point F[3] (2^-32 eV/A units); zero on entry,
                                // left zero by the radial/output kernel
    unsigned long long* accW;   // FP32 form with per-particle virials: [n][12] fixed-point W[9] (2^-32 eV),
                                // same rules; used only when virial is non-null
    float* wsum;                // FP32 form: [9][n] each thread's angular virial sum (for the totals)
    double* partial;            // [items][10] per work item (E, W[9])
    unsigned int* counter;      // [requests] last-group counters (self-resetting)
    unsigned int* gcounter;     // [items] last-block counters of the item groups, at each
                                // group's first item (self-resetting)
    double* totals;             // [requests][10]: E, W[9]
    int* err = nullptr;         // the error word (kErrCellList on an inconsistent cell list)
    // MD: the step's closing half-kick applied by the output pass as soon as F_i is
    // final, v_i <- half_kick(v_i, kick_half_dt, F_i, kick_im[t_i]), with the same
    // rounding as a separate kick kernel; kick_vel per request [3][n_r] blocks, or
    // null (no kick).  kick_types is indexed by caller index.
    double* kick_vel = nullptr;
    const int* kick_types = nullptr;
    double kick_half_dt = 0.0;
    TypeTable kick_im = {};
};

// ---- host-side launchers (defined in the .cu files) ----
// Grids are sized by the capacities (n_cap particles, items_cap work items,
// ncell_cap cells); the sizes in effect come from *counts.  The cell counters must
// be zero on entry (the scan clears them for the next build); zero_counts clears
// them first for callers whose buffers may hold anything.
template <typename real>
cudaError_t launch_cell_build(const PlanCounts* counts, int n_cap, int items_cap, int ncell_cap, bool zero_counts,
                              bool skip_bin,
                              const WorkItem* items, const ReqInfo* reqs, const ModelDesc<real>* models,
                              const double* pos, const int* types, int* cell_of, PosRec<real>* rec_user,
                              int* cell_count, int* cell_start_local, int* block_off, int* cell_fill, int* perm_tmp,
                              int* perm, int* cell_start, int* cell_s, PosRec<real>* rec_sorted, int* err,
                              cudaStream_t st);

// The MD step's opening: n_kicks (1 or 2) velocity half-kicks v += dt/2 F/m (two when
// the previous step's closing kick was deferred into this one), the drift
// r += dt v, the wrap, and the cell binning of the new positions (what k_bin does),
// in one pass; the cell build then runs with skip_bin.  A single request (the MD
// configuration), one work item per block.
template <typename real>
cudaError_t launch_kick_drift_bin(const PlanCounts* counts, int items_cap, const WorkItem* items,
                                  const ReqInfo* reqs, const ModelDesc<real>* models, const int* types,
                                  const TypeTable& inv_m_acc, int n_kicks, double half_dt, double dt, double* pos,
                                  double* vel, const double* force, int* cell_of, PosRec<real>* rec_user,
                                  int* cell_count, int* err, cudaStream_t st);

template <typename real>
cudaError_t launch_neighbors(const NeighborArgs<real>& a, int items_cap, size_t smem, cudaStream_t st);

// Shape-dispatched evaluation; returns cudaErrorInvalidValue for an uncompiled shape.
// mb_desc / mb_force: resident blocks per SM of the FP32 kernel variants (2 or 3; the
// force kernel also 4).  The FP64 form has one effective variant of each.
// The FP32 form needs a.acc (the scatter accumulators); the FP64 form ignores it.
template <typename real>
cudaError_t launch_evaluate(int nR, int nA, int KR, int KA, const EvalArgs<real>& a, int items_cap, size_t smem_desc,
                            size_t smem_force, cudaStream_t st, cudaEvent_t mid = nullptr, int mb_desc = 3,
                            int mb_force = 3, int ch_force = 4);

template <typename real>
bool evaluate_shape_supported(int nR, int nA, int KR, int KA);

template <typename real>
cudaError_t evaluate_set_smem(int nR, int nA, int KR, int KA, size_t smem_desc, size_t smem_force);

cudaError_t launch_kick(int n, const int* types, const double* inv_m_acc, int T, double half_dt, double* vel,
                        const double* force, cudaStream_t st);
cudaError_t launch_sample(int n, const int* types, const double* mass, int T, const double* vel,
                          const double* totals, double* partial, unsigned int* counter, double* thermo,
                          int* sample_index, int step_stride, cudaStream_t st);
cudaError_t launch_scale(int n, double* pos, double sx, double sy, double sz, cudaStream_t st);
// Bussi stochastic velocity rescaling after a step (noise[2*step]: R1, chi^2(N_f - 1)).
cudaError_t launch_bussi(int n, const int* types, const double* mass, int T, double* vel, double* partial,
                         unsigned int* counter, const double* noise, int* step, double c, double kbar, double n_f,
                         double* alpha, cudaStream_t st);

// HNEMD driving force F_i += F_e . W_i - F_e . W / N (virial [9][n], totals[1..9] = W).
cudaError_t launch_hnemd_force(int n, const double fe[3], const double* virial, const double* totals, double* force,
                               cudaStream_t st);
// Heat current (J_pot, J_kin) of the step added to acc[6]; at a sampling step the
// interval average goes to rows[*sample_index][6] and acc is cleared.
// partial: [blocks][6] doubles.
cudaError_t launch_heat(int n, const int* types, const double* mass, int T, const double* vel, const double* site,
                        const double* virial, double* partial, unsigned int* counter, double* acc, double* rows,
                        const int* sample_index, int sample, int step_stride, cudaStream_t st);

// Coarse-grained mapping: bead positions (Eq. 9), summed forces (Eq. 12) and virials (Eq. 14).
cudaError_t launch_cg_map(int n_cg, int n_aa, const int* start, const int* atoms, const double* mass,
                          const double* pos, const double* force, const double* virial, const CellGrid& g,
                          int accumulate, double* bpos, double* bforce, double* bvirial, cudaStream_t st);

}  // namespace nep
