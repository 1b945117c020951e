// Cell list and neighbour lists (the neighbour search that precedes Eq. 3-5).
//
// Per batch of configurations (requests), each with its own box and cell grid:
//   k_bin        wrap periodic axes, bin every particle into a cell, store its
//                cell-relative position (FP32 or FP64) and count cell members
//   k_scan       exclusive scan of the cell counts (two levels, one launch)
//   k_scatter    counting-sort scatter of particle indices into cell order
//   k_cell_rank  order each cell's members by caller index (deterministic order)
//                and gather the records into cell order
//   k_neighbors  one thread per particle scans the (2S+1)^3 surrounding cells and
//                writes the radial (r < r_c^R) and angular (r < r_c^A) lists
//                (k_neighbors_warp: one warp per particle, for small batches)
#include "nep_common.cuh"

namespace nep {

// Bin particle i (caller index, request q) at position x: wrap periodic axes, find
// its cell, store its cell-relative record and count it in its cell.
template <typename real>
__device__ __forceinline__ void bin_one(const ReqInfo& q, int i, double (&x)[3], int t, int n_types,
                                        int* __restrict__ cell_of, PosRec<real>* __restrict__ rec,
                                        int* __restrict__ cell_count, int* __restrict__ err)
{
    const CellGrid& g = q.g;
    int c3[3];
    real xr[3];
    // FP64 work is kept to what the result needs (the part's FP64 rate is low): the
    // floor and the clamp are one rounding conversion and integer compares, and the
    // cell-relative position one FMA
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (!finite_bits(x[a])) {
            atomicOr(err, 1);
            x[a] = 0.0;
        }
        if (g.pbc[a]) x[a] = wrap_periodic(x[a], g.box[a]);
        const int c = min(max(__double2int_rd(x[a] * g.inv_len[a]), 0), g.nc[a] - 1);  // saturating floor
        c3[a] = c;
        xr[a] = (real)fma(-(double)c, g.len[a], x[a]);
    }
    if (t < 0 || t >= n_types) {
        atomicOr(err, 2);
        t = 0;
    }
    const int cell = q.cell_base + (c3[2] * g.nc[1] + c3[1]) * g.nc[0] + c3[0];
    cell_of[i] = cell;
    PosRec<real> r;
    r.x = xr[0];
    r.y = xr[1];
    r.z = xr[2];
    r.t = t;
    rec[i] = r;
    atomicAdd(&cell_count[cell], 1);
}

template <typename real>
__global__ void __launch_bounds__(kBlock) k_bin(const PlanCounts* __restrict__ pc, const WorkItem* __restrict__ items,
                                                const ReqInfo* __restrict__ reqs,
                                                const ModelDesc<real>* __restrict__ models,
                                                const double* __restrict__ pos, const int* __restrict__ types,
                                                int* __restrict__ cell_of, PosRec<real>* __restrict__ rec,
                                                int* __restrict__ cell_count, int* __restrict__ err)
{
    const int n_items = pc->n_items;
    for (int w = blockIdx.x; w < n_items; w += gridDim.x) {
        const WorkItem it = items[w];
        const int i = it.begin + threadIdx.x;
        if (i >= it.end) continue;
        const ReqInfo& q = reqs[it.req];
        const int local = i - q.begin;
        double x[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) x[a] = pos[(size_t)3 * q.begin + (size_t)a * q.n + local];
        bin_one<real>(q, i, x, types[i], models[q.model].T, cell_of, rec, cell_count, err);
    }
}

// The MD step's opening kicks, drift and binning in one pass (one request).
template <typename real>
__global__ void __launch_bounds__(kBlock) k_kick_drift_bin(const PlanCounts* __restrict__ pc,
                                                           const WorkItem* __restrict__ items,
                                                           const ReqInfo* __restrict__ reqs,
                                                           const ModelDesc<real>* __restrict__ models,
                                                           const int* __restrict__ types, TypeTable inv_m_acc,
                                                           int n_kicks, double half_dt, double dt,
                                                           double* __restrict__ pos, double* __restrict__ vel,
                                                           const double* __restrict__ force, int* __restrict__ cell_of,
                                                           PosRec<real>* __restrict__ rec, int* __restrict__ cell_count,
                                                           int* __restrict__ err)
{
    if ((int)blockIdx.x >= pc->n_items) return;
    const WorkItem it = items[blockIdx.x];
    const int i = it.begin + threadIdx.x;
    if (i >= it.end) return;
    const ReqInfo& q = reqs[it.req];
    const int n = q.n, local = i - q.begin;
    const int t = types[i];
    const int T = models[q.model].T;
    const double im = inv_m_acc.v[t >= 0 && t < T ? t : 0];
    double x[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const size_t k = (size_t)3 * q.begin + (size_t)a * n + local;
        double v = vel[k];
        const double f = force[k];
        for (int s = 0; s < n_kicks; ++s) v = half_kick(v, half_dt, f, im);  // separately rounded, as two kernels
        vel[k] = v;
        double xa = drift(pos[k], dt, v);
        if (q.g.pbc[a]) xa = wrap_periodic(xa, q.g.box[a]);
        pos[k] = xa;
        x[a] = xa;
    }
    bin_one<real>(q, i, x, t, T, cell_of, rec, cell_count, err);
}

template <typename real>
cudaError_t launch_kick_drift_bin(const PlanCounts* counts, int items_cap, const WorkItem* items,
                                  const ReqInfo* reqs, const ModelDesc<real>* models, const int* types,
                                  const TypeTable& inv_m_acc, int n_kicks, double half_dt, double dt, double* pos,
                                  double* vel, const double* force, int* cell_of, PosRec<real>* rec_user,
                                  int* cell_count, int* err, cudaStream_t st)
{
    if (items_cap < 1 || n_kicks < 1 || n_kicks > 2) return cudaErrorInvalidValue;
    return launch_k(k_kick_drift_bin<real>, items_cap, kBlock, 0, st, counts, items, reqs, models, types, inv_m_acc,
                      n_kicks, half_dt, dt, pos, vel, force, cell_of, rec_user, cell_count, err);
}

// Exclusive scan of v[0..4) over a block of 1024 threads (4 values per thread);
// returns the thread's first exclusive prefix and the block total in *total.
__device__ __forceinline__ int block_scan4(const int (&v)[4], int* warp_tot, int* total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int s = v[0] + v[1] + v[2] + v[3];
    int incl = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int w = warp_tot[lane];
        int wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        warp_tot[lane] = wi - w;  // exclusive prefix of warp totals
        if (lane == 31) warp_tot[32] = wi;
    }
    __syncthreads();
    const int run = warp_tot[warp] + incl - s;
    *total = warp_tot[32];
    __syncthreads();  // warp_tot is reused by the caller's next scan
    return run;
}

// Two-level exclusive scan of the cell counts in one launch.  Each block scans
// kScanItems counts (4 per thread, 1024 threads) into local[] and its total into
// block_sum[blk]; the last block to finish (a counter at block_sum[kScanItems],
// self-resetting) scans the block totals in place (nb <= kScanItems).  The counters
// it reads (cell counts and the scatter's fill counters) are cleared here for the
// next build.
__global__ void __launch_bounds__(1024) k_scan(const PlanCounts* __restrict__ pc, int* __restrict__ count,
                                               int* __restrict__ local, int* __restrict__ block_sum,
                                               int* __restrict__ fill)
{
    __shared__ int warp_tot[33];
    __shared__ bool last;
    const int ncell = pc->ncell;
    const int nb = (ncell + kScanItems - 1) / kScanItems;
    for (int blk = blockIdx.x; blk < nb; blk += gridDim.x) {
        const int base = blk * kScanItems + threadIdx.x * 4;
        int v[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            v[k] = 0;
            if (base + k < ncell) {
                v[k] = count[base + k];
                count[base + k] = 0;
                fill[base + k] = 0;
            }
        }
        int total;
        int run = block_scan4(v, warp_tot, &total);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (base + k < ncell) local[base + k] = run;
            run += v[k];
        }
        if (threadIdx.x == 0) block_sum[blk] = total;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = (atomicAdd(&block_sum[kScanItems], 1) == (int)gridDim.x - 1);
    __syncthreads();
    if (!last) return;
    __threadfence();
    const int base = threadIdx.x * 4;
    int v[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] = (base + k < nb) ? __ldcg(block_sum + base + k) : 0;
    int total;
    int run = block_scan4(v, warp_tot, &total);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (base + k < nb) block_sum[base + k] = run;
        run += v[k];
    }
    if (threadIdx.x == 0) block_sum[kScanItems] = 0;
}

// Counting-sort scatter (thread per particle, arbitrary order within a cell) and the
// cell start offsets (thread per cell).  This kernel and k_cell_rank check the
// indices they derive from the cell arrays and, should one ever fall outside its
// array (an internal inconsistency, never an input error), set kErrCellList in the
// error word and skip the access instead of touching memory out of bounds; every
// cell start is kept within [0, n], and the neighbour kernels clamp each particle's
// cell into its grid, so their searches stay inside the arrays too.
__global__ void __launch_bounds__(kBlock) k_scatter(const PlanCounts* __restrict__ pc, const int* __restrict__ cell_of,
                                                    const int* __restrict__ local, const int* __restrict__ block_off,
                                                    int* __restrict__ fill, int* __restrict__ perm_tmp,
                                                    int* __restrict__ cell_start, int* __restrict__ err)
{
    const int n = pc->n, ncell = pc->ncell;
    const int total = n > ncell + 1 ? n : ncell + 1;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
        if (t < n) {
            const int c = cell_of[t];
            if (c < 0 || c >= ncell) {
                atomicOr(err, kErrCellList);
            } else {
                const int slot = local[c] + block_off[c / kScanItems] + atomicAdd(&fill[c], 1);
                if (slot < 0 || slot >= n)
                    atomicOr(err, kErrCellList);
                else
                    perm_tmp[slot] = t;
            }
        }
        if (t < ncell) {  // kept within [0, n], so that no cell's range leaves the particles
            const int v = local[t] + block_off[t / kScanItems];
            if (v < 0 || v > n) atomicOr(err, kErrCellList);
            cell_start[t] = min(max(v, 0), n);
        }
        if (t == ncell) cell_start[ncell] = n;
    }
}

// Deterministic order within each cell (by caller index): thread per slot, rank =
// number of the cell's members with a smaller caller index; gathers the records.
template <typename real>
__global__ void __launch_bounds__(kBlock) k_cell_rank(const PlanCounts* __restrict__ pc,
                                                      const int* __restrict__ cell_of,
                                                      const int* __restrict__ cell_start,
                                                      const int* __restrict__ perm_tmp, int* __restrict__ perm,
                                                      int* __restrict__ cell_s, const PosRec<real>* __restrict__ rec,
                                                      PosRec<real>* __restrict__ rec_s, int* __restrict__ err)
{
    const int n = pc->n, ncell = pc->ncell;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const int v = perm_tmp[k];
        const int c = (v >= 0 && v < n) ? cell_of[v] : -1;
        if (c < 0 || c >= ncell) {
            atomicOr(err, kErrCellList);
            continue;
        }
        const int b = cell_start[c], e = cell_start[c + 1];
        if (b < 0 || b > e || e > n) {
            atomicOr(err, kErrCellList);
            continue;
        }
        int rank = 0;
        for (int q = b; q < e; ++q) rank += perm_tmp[q] < v;
        const int dst = b + rank;
        if (dst >= e) {
            atomicOr(err, kErrCellList);
            continue;
        }
        perm[dst] = v;
        cell_s[dst] = c;
        rec_s[dst] = rec[v];
    }
}

template <typename real>
cudaError_t launch_cell_build(const PlanCounts* counts, int n_cap, int items_cap, int ncell_cap, bool zero_counts,
                              bool skip_bin, const WorkItem* items, const ReqInfo* reqs, const ModelDesc<real>* models,
                              const double* pos, const int* types, int* cell_of, PosRec<real>* rec_user,
                              int* cell_count, int* cell_start_local, int* block_off, int* cell_fill, int* perm_tmp,
                              int* perm, int* cell_start, int* cell_s, PosRec<real>* rec_sorted, int* err,
                              cudaStream_t st)
{
    const int nb_scan = (ncell_cap + kScanItems - 1) / kScanItems;
    if (nb_scan > kScanItems || n_cap < 1 || items_cap < 1) return cudaErrorInvalidValue;
    cudaError_t e;
    if (zero_counts) {
        if ((e = cudaMemsetAsync(cell_count, 0, sizeof(int) * ncell_cap, st)) != cudaSuccess) return e;
        if ((e = cudaMemsetAsync(cell_fill, 0, sizeof(int) * ncell_cap, st)) != cudaSuccess) return e;
        if ((e = cudaMemsetAsync(block_off + kScanItems, 0, sizeof(int), st)) != cudaSuccess) return e;
    }
    if (!skip_bin &&
        (e = launch_k(k_bin<real>, items_cap, kBlock, 0, st, counts, items, reqs, models, pos, types, cell_of,
                        rec_user, cell_count, err)) != cudaSuccess)
        return e;
    if ((e = launch_k(k_scan, nb_scan, 1024, 0, st, counts, cell_count, cell_start_local, block_off, cell_fill)) !=
        cudaSuccess)
        return e;
    const int nt = (n_cap > ncell_cap + 1 ? n_cap : ncell_cap + 1);
    if ((e = launch_k(k_scatter, (nt + kBlock - 1) / kBlock, kBlock, 0, st, counts, cell_of, cell_start_local,
                        block_off, cell_fill, perm_tmp, cell_start, err)) != cudaSuccess)
        return e;
    return launch_k(k_cell_rank<real>, (n_cap + kBlock - 1) / kBlock, kBlock, 0, st, counts, cell_of, cell_start,
                      perm_tmp, perm, cell_s, rec_user, rec_sorted, err);
}

// One thread per sorted particle i: scan the cells at offsets [-S, S]^3 from i's
// cell in its request's grid and keep every (j, offset) with r^2 < r_c^2(t_i, t_j).
// A warp's particles are consecutive in cell order (about two cells of a water
// box), so in SIMT the warp tests the union of their neighbourhoods whatever the
// per-thread scheme; the candidate body is therefore kept branch-free, with the
// tests predicating the stores (masks with store loops afterwards, and skipping
// cells out of reach, were measured slower: both make the lanes diverge).
template <typename real>
__device__ __forceinline__ void neighbors_item(const NeighborArgs<real>& a, const WorkItem it, real* cut);

template <typename real>
__global__ void __launch_bounds__(kBlock) k_neighbors(NeighborArgs<real> a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    real* cut = reinterpret_cast<real*>(smem_raw);  // rcR2[T*T], rcA2[T*T]
    // one work item per block: launch grids cover the item capacity, blocks past the
    // batch's item count exit
    if ((int)blockIdx.x >= a.counts->n_items) return;
    neighbors_item(a, a.items[blockIdx.x], cut);
}

template <typename real>
__device__ __forceinline__ void neighbors_item(const NeighborArgs<real>& a, const WorkItem it, real* cut)
{
    const ReqInfo& q = a.reqs[it.req];
    const ModelDesc<real> md = a.models[q.model];
    const int T = md.T, TT = T * T;
    for (int k = threadIdx.x; k < TT; k += blockDim.x) {
        cut[k] = md.params[md.off.rcR2 + k];
        cut[TT + k] = md.params[md.off.rcA2 + k];
    }
    // FP64 with a.rec32: each distance test is screened in FP32 first.  For
    // cell-relative coordinates of i and j within 2 len of their cell's origin on
    // every axis (all of them except particles outside the box on an open axis), the
    // FP32 pair vector is within d = sqrt(3) len 2^-19 of the exact one, so its r^2
    // is within eps = 2 r_c d + d^2 + 3 2^-24 r_c^2 of the exact r^2 wherever it
    // could decide.  Below r_c^2 - 4 eps the FP64 test would accept, above
    // r_c^2 + 4 eps it would reject; in between, and for any particle beyond the
    // 2 len range, the FP64 test decides, so the lists are exactly the FP64 ones.
    constexpr bool kScreen = sizeof(real) == 8;
    const bool screened = kScreen && a.rec32 != nullptr;
    float* screen = reinterpret_cast<float*>(cut + 2 * TT);  // [2 TT][lo, hi]
    if (screened) {
        const double lmax = fmax(q.g.len[0], fmax(q.g.len[1], q.g.len[2]));
        const double d = 1.7320508075688772 * lmax * 0x1p-19;
        for (int k = threadIdx.x; k < 2 * TT; k += blockDim.x) {
            const double c2 = k < TT ? (double)md.params[md.off.rcR2 + k] : (double)md.params[md.off.rcA2 + k - TT];
            const double eps = 4.0 * (2.0 * sqrt(c2) * d + d * d + 3.0 * 0x1p-24 * c2);
            screen[2 * k] = __double2float_rd(c2 - eps);
            screen[2 * k + 1] = __double2float_ru(c2 + eps);
        }
    }
    __syncthreads();
    const int i = it.begin + threadIdx.x;
    int nr = 0, na = 0;
    if (i < it.end) {
        const CellGrid& g = q.g;
        const PosRec<real> ri = a.rec[i];
        // clamped into the request's grid: an out-of-range cell (which k_cell_rank
        // reports) cannot take the search outside the cell arrays
        const int c = min(max(a.cell_s[i] - q.cell_base, 0), g.ncell - 1);
        const int cx = c % g.nc[0], cy = (c / g.nc[0]) % g.nc[1], cz = c / (g.nc[0] * g.nc[1]);
        const real* cutR = cut + ri.t * T;
        const real* cutA = cut + TT + ri.t * T;
        const real cR1 = cutR[0], cA1 = cutA[0];  // the one pair type of a one-type model
        const float* scrR = screen + 2 * (ri.t * T);  // FP64 screening bounds of i's row
        const float* scrA = screen + 2 * (TT + ri.t * T);
        PosRec<float> ri32 = {};
        if (screened) ri32 = a.rec32[i];
        const float lxf = (float)g.len[0], lyf = (float)g.len[1], lzf = (float)g.len[2];
        // the range the screening bound covers (2 len per axis, rounded down)
        const float mx = 1.99f * lxf, my = 1.99f * lyf, mz = 1.99f * lzf;
        const bool i_screened =
            screened && fabsf(ri32.x) <= mx && fabsf(ri32.y) <= my && fabsf(ri32.z) <= mz;
        const real lx = (real)g.len[0], ly = (real)g.len[1], lz = (real)g.len[2];
        const int ncx = g.nc[0], ncy = g.nc[1], ncz = g.nc[2];
        // slot s of particle i's list is entry s * n + i (slot-major); the launcher
        // guarantees capacity * n <= 2^32, so the index fits 32 bits
        const uint32_t stride = (uint32_t)a.n, col = (uint32_t)i;
        for (int dz = -g.S[2]; dz <= g.S[2]; ++dz) {
            int z = cz + dz;
            if (g.pbc[2]) {  // |dz| <= 2, so at most two corrections even for one cell per axis
                while (z < 0) z += ncz;
                while (z >= ncz) z -= ncz;
            } else if (z < 0 || z >= ncz) {
                continue;
            }
            for (int dy = -g.S[1]; dy <= g.S[1]; ++dy) {
                int y = cy + dy;
                if (g.pbc[1]) {
                    while (y < 0) y += ncy;
                    while (y >= ncy) y -= ncy;
                } else if (y < 0 || y >= ncy) {
                    continue;
                }
                for (int dx = -g.S[0]; dx <= g.S[0]; ++dx) {
                    int x = cx + dx;
                    if (g.pbc[0]) {
                        while (x < 0) x += ncx;
                        while (x >= ncx) x -= ncx;
                    } else if (x < 0 || x >= ncx) {
                        continue;
                    }
                    const int cell = q.cell_base + (z * ncy + y) * ncx + x;
                    // j's position relative to i is (r_j + offset) - r_i = r_j - b
                    const real bx = ri.x - (real)dx * lx, by = ri.y - (real)dy * ly, bz = ri.z - (real)dz * lz;
                    const uint32_t code = ((uint32_t)((dx + 2) | ((dy + 2) << 3) | ((dz + 2) << 6))) << kJBits;
                    const int kb = a.cell_start[cell], ke = a.cell_start[cell + 1];  // within [0, n] (k_scatter)
                    // branch-free body: the tests predicate the stores and the counts; i
                    // itself (zero offset) is the one candidate at r = 0 to leave out, tested
                    // for only in i's own cell (center: the same for every lane of the warp)
                    auto candidate = [&](int k, const PosRec<real>& rj, real cR2, real cA2, bool center) {
                        const real ddx = rj.x - bx, ddy = rj.y - by, ddz = rj.z - bz;
                        const real r2 = ddx * ddx + ddy * ddy + ddz * ddz;
                        const uint32_t ent = (uint32_t)k | code;
                        const bool other = !center || k != i;
                        const bool inR = (r2 < cR2) & other, inA = (r2 < cA2) & other;
                        if (inR & (nr < a.mnR)) a.nlR[(uint32_t)nr * stride + col] = ent;
                        if (inA & (na < a.mnA)) a.nlA[(uint32_t)na * stride + col] = ent;
                        nr += inR;
                        na += inA;
                    };
                    // FP64 screened: the FP32 record decides outside the band around
                    // each cutoff, the FP64 record inside it
                    const float bxf = ri32.x - (float)dx * lxf, byf = ri32.y - (float)dy * lyf,
                                bzf = ri32.z - (float)dz * lzf;
                    auto screened_candidate = [&](int k, bool center) {
                        const PosRec<float> rf = ldg_rec(a.rec32 + k);
                        const float fx = rf.x - bxf, fy = rf.y - byf, fz = rf.z - bzf;
                        const float r2f = fx * fx + fy * fy + fz * fz;
                        const int tp = 2 * rf.t;
                        bool inR = r2f < scrR[tp], inA = r2f < scrA[tp];
                        const bool j_far = !(fabsf(rf.x) <= mx && fabsf(rf.y) <= my && fabsf(rf.z) <= mz);
                        if (j_far || (r2f < scrR[tp + 1]) != inR || (r2f < scrA[tp + 1]) != inA) {
                            const PosRec<real> rj = ldg_rec(a.rec + k);
                            const real ddx = rj.x - bx, ddy = rj.y - by, ddz = rj.z - bz;
                            const real r2 = ddx * ddx + ddy * ddy + ddz * ddz;
                            inR = r2 < cutR[rf.t];
                            inA = r2 < cutA[rf.t];
                        }
                        const uint32_t ent = (uint32_t)k | code;
                        const bool other = !center || k != i;
                        inR &= other;
                        inA &= other;
                        if (inR & (nr < a.mnR)) a.nlR[(uint32_t)nr * stride + col] = ent;
                        if (inA & (na < a.mnA)) a.nlA[(uint32_t)na * stride + col] = ent;
                        nr += inR;
                        na += inA;
                    };
                    const bool center = dx == 0 && dy == 0 && dz == 0;
                    if (kScreen && i_screened) {
                        if (center) {
#pragma unroll 2
                            for (int k = kb; k < ke; ++k) screened_candidate(k, true);
                        } else {
#pragma unroll 2
                            for (int k = kb; k < ke; ++k) screened_candidate(k, false);
                        }
                    } else if (T == 1) {  // one pair type: deeper unrolling (measured faster)
                        if (center) {
#pragma unroll 4
                            for (int k = kb; k < ke; ++k) candidate(k, ldg_rec(a.rec + k), cR1, cA1, true);
                        } else {
#pragma unroll 4
                            for (int k = kb; k < ke; ++k) candidate(k, ldg_rec(a.rec + k), cR1, cA1, false);
                        }
                    } else {  // per-type cutoffs from shared memory (unroll 4 measured slower)
                        if (center) {
#pragma unroll 2
                            for (int k = kb; k < ke; ++k) {
                                const PosRec<real> rj = ldg_rec(a.rec + k);
                                candidate(k, rj, cutR[rj.t], cutA[rj.t], true);
                            }
                        } else {
#pragma unroll 2
                            for (int k = kb; k < ke; ++k) {
                                const PosRec<real> rj = ldg_rec(a.rec + k);
                                candidate(k, rj, cutR[rj.t], cutA[rj.t], false);
                            }
                        }
                    }
                }
            }
        }
        a.cntR[i] = nr;
        a.cntA[i] = na;
        if (a.accF) {  // i's fixed-point lines start the evaluation at zero
            ulonglong2* zl = reinterpret_cast<ulonglong2*>(a.accF + (size_t)i * 4);
            zl[0] = zl[1] = make_ulonglong2(0ull, 0ull);
        }
        if (a.accW) {
            ulonglong2* zl = reinterpret_cast<ulonglong2*>(a.accW + (size_t)i * 12);
#pragma unroll
            for (int k = 0; k < 6; ++k) zl[k] = make_ulonglong2(0ull, 0ull);
        }
    }
    // warp maxima, then one atomic per warp
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        nr = max(nr, __shfl_xor_sync(0xffffffffu, nr, o));
        na = max(na, __shfl_xor_sync(0xffffffffu, na, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(&a.maxcnt[0], nr);
        atomicMax(&a.maxcnt[1], na);
    }
}

// Small batches: one warp per particle.  With few work items the thread-per-particle
// kernel leaves most SMs idle and each thread's candidate loop (about 500 candidates
// for water) is the whole kernel's latency.  Here the warp's lanes test 32 of the
// particle's candidates at a time (consecutive records of one stencil cell, a
// coalesced load), and ballots compact the accepted ones in candidate order, so the
// lists are exactly those the thread-per-particle kernel writes.  A block of kBlock
// threads takes kBlock / 32 particles of one work item.
constexpr int kNbrWarpParticles = kBlock / 32;

template <typename real>
__global__ void __launch_bounds__(kBlock) k_neighbors_warp(NeighborArgs<real> a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    real* cut = reinterpret_cast<real*>(smem_raw);  // rcR2[T*T], rcA2[T*T]
    constexpr int kPerItem = kBlock / kNbrWarpParticles;  // blocks per work item
    const int item = (int)blockIdx.x / kPerItem;
    if (item >= a.counts->n_items) return;
    const WorkItem it = a.items[item];
    const ReqInfo& q = a.reqs[it.req];
    const ModelDesc<real> md = a.models[q.model];
    const int T = md.T, TT = T * T;
    for (int k = threadIdx.x; k < TT; k += blockDim.x) {
        cut[k] = md.params[md.off.rcR2 + k];
        cut[TT + k] = md.params[md.off.rcA2 + k];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const unsigned below = (1u << lane) - 1u;
    const int i = it.begin + ((int)blockIdx.x % kPerItem) * kNbrWarpParticles + ((int)threadIdx.x >> 5);
    if (i >= it.end) return;  // warp-uniform
    const CellGrid& g = q.g;
    const PosRec<real> ri = a.rec[i];
    const int c = min(max(a.cell_s[i] - q.cell_base, 0), g.ncell - 1);  // clamped as in k_neighbors
    const int cx = c % g.nc[0], cy = (c / g.nc[0]) % g.nc[1], cz = c / (g.nc[0] * g.nc[1]);
    const real* cutR = cut + ri.t * T;
    const real* cutA = cut + TT + ri.t * T;
    const real lx = (real)g.len[0], ly = (real)g.len[1], lz = (real)g.len[2];
    const int ncx = g.nc[0], ncy = g.nc[1], ncz = g.nc[2];
    const uint32_t stride = (uint32_t)a.n, col = (uint32_t)i;
    int nr = 0, na = 0;  // warp-uniform
    for (int dz = -g.S[2]; dz <= g.S[2]; ++dz) {
        int z = cz + dz;
        if (g.pbc[2]) {
            while (z < 0) z += ncz;
            while (z >= ncz) z -= ncz;
        } else if (z < 0 || z >= ncz) {
            continue;
        }
        for (int dy = -g.S[1]; dy <= g.S[1]; ++dy) {
            int y = cy + dy;
            if (g.pbc[1]) {
                while (y < 0) y += ncy;
                while (y >= ncy) y -= ncy;
            } else if (y < 0 || y >= ncy) {
                continue;
            }
            for (int dx = -g.S[0]; dx <= g.S[0]; ++dx) {
                int x = cx + dx;
                if (g.pbc[0]) {
                    while (x < 0) x += ncx;
                    while (x >= ncx) x -= ncx;
                } else if (x < 0 || x >= ncx) {
                    continue;
                }
                const int cell = q.cell_base + (z * ncy + y) * ncx + x;
                const real bx = ri.x - (real)dx * lx, by = ri.y - (real)dy * ly, bz = ri.z - (real)dz * lz;
                const uint32_t code = ((uint32_t)((dx + 2) | ((dy + 2) << 3) | ((dz + 2) << 6))) << kJBits;
                const int kb = a.cell_start[cell], ke = a.cell_start[cell + 1];  // within [0, n] (k_scatter)
                const int self = (dx == 0 && dy == 0 && dz == 0) ? i : -1;
                for (int k0 = kb; k0 < ke; k0 += 32) {
                    const int k = k0 + lane;
                    bool inR = false, inA = false;
                    if (k < ke) {
                        const PosRec<real> rj = ldg_rec(a.rec + k);
                        const real ddx = rj.x - bx, ddy = rj.y - by, ddz = rj.z - bz;
                        const real r2 = ddx * ddx + ddy * ddy + ddz * ddz;
                        const bool other = k != self;
                        inR = (r2 < cutR[rj.t]) & other;
                        inA = (r2 < cutA[rj.t]) & other;
                    }
                    const unsigned mR = __ballot_sync(0xffffffffu, inR), mA = __ballot_sync(0xffffffffu, inA);
                    const uint32_t ent = (uint32_t)k | code;
                    const int sR = nr + __popc(mR & below), sA = na + __popc(mA & below);
                    if (inR && sR < a.mnR) a.nlR[(uint32_t)sR * stride + col] = ent;
                    if (inA && sA < a.mnA) a.nlA[(uint32_t)sA * stride + col] = ent;
                    nr += __popc(mR);
                    na += __popc(mA);
                }
            }
        }
    }
    if (lane == 0) {
        a.cntR[i] = nr;
        a.cntA[i] = na;
        atomicMax(&a.maxcnt[0], nr);
        atomicMax(&a.maxcnt[1], na);
    }
    if (a.accF && lane < 2) {  // i's fixed-point lines start the evaluation at zero
        reinterpret_cast<ulonglong2*>(a.accF + (size_t)i * 4)[lane] = make_ulonglong2(0ull, 0ull);
    }
    if (a.accW && lane < 6) {
        reinterpret_cast<ulonglong2*>(a.accW + (size_t)i * 12)[lane] = make_ulonglong2(0ull, 0ull);
    }
}

// Work items up to which the warp-per-particle kernel runs.  Measured on water boxes
// (neighbour stage, ms): 16 items 0.027 (warp) against 0.084 (thread per particle),
// 40 items 0.033 / 0.071, 79 items 0.055 / 0.066, 118 items 0.076 / 0.070, 157 items
// 0.097 / 0.073.
constexpr int kNbrWarpMaxItems = 96;

// FP64 form: the FP32 copies of the sorted records that screen the distance tests
// of k_neighbors (one conversion per particle instead of per candidate)
__global__ void __launch_bounds__(kBlock) k_round_records(const PlanCounts* __restrict__ pc,
                                                          const PosRec<double>* __restrict__ rec,
                                                          PosRec<float>* __restrict__ rec32)
{
    const int n = pc->n;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const PosRec<double> r = rec[k];
        PosRec<float> f;
        f.x = (float)r.x;
        f.y = (float)r.y;
        f.z = (float)r.z;
        f.t = r.t;
        rec32[k] = f;
    }
}

template <typename real>
cudaError_t launch_neighbors(const NeighborArgs<real>& a, int items_cap, size_t smem, cudaStream_t st)
{
    // the kernels index the slot-major lists with 32-bit slot * n + i
    if ((unsigned long long)(a.mnR > a.mnA ? a.mnR : a.mnA) * (unsigned long long)a.n > (1ull << 32))
        return cudaErrorInvalidValue;
    if (items_cap <= kNbrWarpMaxItems)  // FP64 here tests every pair in FP64
        return launch_k(k_neighbors_warp<real>, items_cap * (kBlock / kNbrWarpParticles), kBlock, smem, st, a);
    if constexpr (sizeof(real) == 8) {
        if (a.rec32) {
            const cudaError_t e = launch_k(k_round_records, (a.n + kBlock - 1) / kBlock, kBlock, 0, st, a.counts, a.rec,
                                           a.rec32);
            if (e != cudaSuccess) return e;
        }
    }
    return launch_k(k_neighbors<real>, items_cap, kBlock, smem, st, a);
}

#define NEP_INSTANTIATE(real)                                                                                   \
    template cudaError_t launch_kick_drift_bin<real>(const PlanCounts*, int, const WorkItem*, const ReqInfo*, \
                                                     const ModelDesc<real>*, const int*, const TypeTable&, int,   \
                                                     double, double, double*, double*, const double*, int*,       \
                                                     PosRec<real>*, int*, int*, cudaStream_t);                    \
    template cudaError_t launch_cell_build<real>(const PlanCounts*, int, int, int, bool, bool, const WorkItem*, \
                                                 const ReqInfo*, const ModelDesc<real>*, const double*,           \
                                                 const int*, int*, PosRec<real>*, int*, int*, int*, int*, int*,   \
                                                 int*, int*, int*, PosRec<real>*, int*, cudaStream_t);            \
    template cudaError_t launch_neighbors<real>(const NeighborArgs<real>&, int, size_t, cudaStream_t);
NEP_INSTANTIATE(float)
NEP_INSTANTIATE(double)
#undef NEP_INSTANTIATE

}  // namespace nep
