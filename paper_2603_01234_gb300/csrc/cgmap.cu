// Coarse-grained mapping of an atomistic configuration onto beads (paper Sec. II.B-C):
//   Eq. 9   R_I = sum_{i in I} C_Ii r_i,  C_Ii = m_i / sum_{i' in I} m_i'
//   Eq. 12  F_I = sum_{i in I} f_i          (instantaneous; time averages accumulate)
//   Eq. 14  W_I = sum_{i in I} W_i
// One thread per bead walks its atoms in the order given, so sums are deterministic.
// On periodic axes each atom is taken at its image nearest to the group's first
// atom before weighting (a group must be smaller than half the box), and the
// bead position is wrapped back into [0, L).
#include "nep_common.cuh"

namespace nep {

__global__ void __launch_bounds__(kBlock) k_cg_map(int n_cg, int n_aa, const int* __restrict__ start,
                                                   const int* __restrict__ atoms, const double* __restrict__ mass,
                                                   const double* __restrict__ pos, const double* __restrict__ force,
                                                   const double* __restrict__ virial, CellGrid g, int accumulate,
                                                   double* __restrict__ bpos, double* __restrict__ bforce,
                                                   double* __restrict__ bvirial)
{
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= n_cg) return;
    const int b = start[I], e = start[I + 1];
    if (bpos && e > b) {
        const int a0 = atoms[b];
        double ref[3], acc[3] = {0.0, 0.0, 0.0}, msum = 0.0;
        for (int a = 0; a < 3; ++a) ref[a] = pos[(size_t)a * n_aa + a0];
        for (int k = b; k < e; ++k) {
            const int i = atoms[k];
            const double mi = mass[i];
            for (int a = 0; a < 3; ++a) {
                double d = pos[(size_t)a * n_aa + i] - ref[a];
                if (g.pbc[a]) d -= g.box[a] * rint(d / g.box[a]);
                acc[a] += mi * d;
            }
            msum += mi;
        }
        for (int a = 0; a < 3; ++a) {
            double x = ref[a] + acc[a] / msum;
            if (g.pbc[a]) x = wrap_periodic(x, g.box[a]);
            bpos[(size_t)a * n_cg + I] = x;
        }
    }
    if (bforce && force) {
        for (int a = 0; a < 3; ++a) {
            double s = 0.0;
            for (int k = b; k < e; ++k) s += force[(size_t)a * n_aa + atoms[k]];
            double* o = bforce + (size_t)a * n_cg + I;
            *o = accumulate ? *o + s : s;
        }
    }
    if (bvirial && virial) {
        for (int c = 0; c < 9; ++c) {
            double s = 0.0;
            for (int k = b; k < e; ++k) s += virial[(size_t)c * n_aa + atoms[k]];
            double* o = bvirial + (size_t)c * n_cg + I;
            *o = accumulate ? *o + s : s;
        }
    }
}

cudaError_t launch_cg_map(int n_cg, int n_aa, const int* start, const int* atoms, const double* mass,
                          const double* pos, const double* force, const double* virial, const CellGrid& g,
                          int accumulate, double* bpos, double* bforce, double* bvirial, cudaStream_t st)
{
    k_cg_map<<<(n_cg + kBlock - 1) / kBlock, kBlock, 0, st>>>(n_cg, n_aa, start, atoms, mass, pos, force, virial, g,
                                                              accumulate, bpos, bforce, bvirial);
    return cudaGetLastError();
}

}  // namespace nep
