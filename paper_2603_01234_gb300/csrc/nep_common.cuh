// Internal definitions shared by the CUDA translation units of the NEP library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace nep {

// A neighbour entry packs the sorted index j (low 23 bits) and the cell offset
// (dx, dy, dz) in [-2, 2]^3 of j's cell relative to i's cell (3 bits each).
constexpr int kJBits = 23;
constexpr uint32_t kJMask = (1u << kJBits) - 1u;
constexpr int kMaxN = (1 << kJBits) - 1;
constexpr int kMaxS = 2;
constexpr int kMaxTypes = 16;
constexpr int kBlock = 128;          // threads per block of the per-bead kernels
constexpr int kScanItems = 4096;     // cells per block of the scan

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

// Cell grid of one configuration.
struct CellGrid {
    int nc[3];      // cells per axis
    int S[3];       // search range in cells per axis
    int pbc[3];
    int ncell;
    double len[3];  // cell side
    double box[3];
};

// Offsets (in elements of `real`) of the model tables inside one device buffer.
struct ParamLayout {
    int rcR2, rcA2, rcRi, rcAi; // [T][T] each: squared and inverse cutoffs
    int cR, cA;                 // [T][T][nR][KR], [T][T][nA][KA]
    int w0, b0, w1, b1;         // [T][H][ND], [T][H], [T][H], [T]
    int n_cut_coef;             // elements of the cutoff + coefficient prefix
    int total;                  // all elements
};

template <typename real>
struct NeighborArgs {
    int n, T, mnR, mnA;
    CellGrid g;
    const int* cell_start;      // [ncell + 1]
    const int* cell_s;          // [n] cell of sorted particle
    const PosRec<real>* rec;    // [n] sorted
    const real* params;         // model tables (cutoff prefix used)
    ParamLayout off;
    uint32_t* nlR;              // [mnR][n]
    uint32_t* nlA;              // [mnA][n]
    int* cntR;                  // [n]
    int* cntA;                  // [n]
    int* maxcnt;                // [2]
};

template <typename real>
struct EvalArgs {
    int n, T, H, mnR, mnA;
    real len[3];                // cell side, for the packed offsets
    const PosRec<real>* rec;    // [n] sorted
    const uint32_t* nlR;
    const uint32_t* nlA;
    const int* cntR;
    const int* cntA;
    const real* params;
    ParamLayout off;
    real* U;                    // [n] sorted site energies
    real* e;                    // [n][T][KRP] radial gradient folded into the basis
    real* phi;                  // [n][24][NA] dU/dA_nlm
    int tile_offset;            // byte offset of the force kernel's Phi tile in dynamic smem
    const int* perm;            // sorted slot -> caller index
    double* force;              // [3][n] caller order (required)
    double* virial;             // [9][n] caller order or null
    double* site;               // [n] caller order or null
    double* partial;            // [gridDim][10] per-block (E, W[9])
    unsigned int* counter;      // last-block counter (self-resetting)
    double* totals;             // [10]: E, W[9]
};

// ---- host-side launchers (defined in the .cu files) ----
template <typename real>
cudaError_t launch_cell_build(int n, const double* pos, const int* types, int T, const CellGrid& g,
                              int* cell_of, PosRec<real>* rec_user, int* cell_count, int* cell_start_local,
                              int* block_off, int* cell_fill, int* perm, int* cell_start, int* cell_s,
                              PosRec<real>* rec_sorted, int* err, cudaStream_t st);

template <typename real>
cudaError_t launch_neighbors(const NeighborArgs<real>& a, cudaStream_t st);

// Shape-dispatched evaluation; returns cudaErrorInvalidValue for an uncompiled shape.
template <typename real>
cudaError_t launch_evaluate(int nR, int nA, int KR, int KA, const EvalArgs<real>& a, size_t smem_desc,
                            size_t smem_force, cudaStream_t st, cudaEvent_t mid = nullptr);

template <typename real>
bool evaluate_shape_supported(int nR, int nA, int KR, int KA);

template <typename real>
cudaError_t evaluate_set_smem(int nR, int nA, int KR, int KA, size_t smem_desc, size_t smem_force);

cudaError_t launch_kick_drift(int n, const int* types, const double* inv_m_acc, int T, double half_dt, double dt,
                              const CellGrid& g, double* pos, double* vel, const double* force, cudaStream_t st);
cudaError_t launch_kick(int n, const int* types, const double* inv_m_acc, int T, double half_dt, double* vel,
                        const double* force, cudaStream_t st);
cudaError_t launch_sample(int n, const int* types, const double* mass, int T, const double* vel,
                          const double* totals, double* partial, unsigned int* counter, double* thermo,
                          int* sample_index, int step_stride, cudaStream_t st);
cudaError_t launch_scale(int n, double* pos, double sx, double sy, double sz, cudaStream_t st);

}  // namespace nep
