// Velocity-Verlet NVE integration in FP64 (the MD loop in which the potential is
// evaluated) and the kinetic-energy sample.
//   (the opening kick, drift and wrap run fused with the cell binning: k_kick_drift_bin;
//   the closing kick normally runs in the radial-force/output kernel)
//   k_kick         v += dt/2 F/m, the closing kick when the HNEMD force must be added
//                  to the forces first
//   k_sample       E_kin = sum 1/2 m v^2 (FP64, deterministic last-block total) and
//                  one thermo row (step, E_pot, E_kin, W[9])
//   k_bussi_ke     E_kin and the stochastic-velocity-rescaling factor (Bussi,
//                  Donadio, Parrinello 2007) from the step's two random numbers
//   k_scale_vel    v *= alpha
//   k_hnemd_force  HNEMD driving force (Fan et al., Phys. Rev. B 99, 064308, 2019)
//                  F_i += F_e . W_i - F_e . W / N, with W_i the per-particle virial
//                  of Eq. 15 and W = sum_i W_i (Eq. 16)
//   k_heat         heat current J_pot = sum_i W_i v_i, J_kin = sum_i (1/2 m v^2 + U_i) v_i
//                  (Fan et al., Phys. Rev. B 92, 094301, 2015), summed over the steps
//                  of a sampling interval and written as the interval's average
#include "nep_common.cuh"

namespace nep {

// 1 eV / (Angstrom amu) in Angstrom / fs^2 (acceleration of a force in eV/A on a mass in amu)
constexpr double kAcc = 9.648533212e-3;

// Sum of partial[b * NC + c] over the nb blocks, by the whole (last) block: fixed
// strides per thread and a fixed tree, so the result does not depend on timing.
// Every thread receives the totals.
template <int NC>
__device__ __forceinline__ void last_block_sum(const double* partial, unsigned nb, double (&out)[NC])
{
    __shared__ double red[kBlock / 32][NC];
    double s[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) s[c] = 0.0;
    for (unsigned b = threadIdx.x; b < nb; b += blockDim.x)
#pragma unroll
        for (int c = 0; c < NC; ++c) s[c] += __ldcg(partial + (size_t)b * NC + c);  // L2: other blocks' words
#pragma unroll
    for (int c = 0; c < NC; ++c) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s[c] += __shfl_xor_sync(0xffffffffu, s[c], o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5][c] = s[c];
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        double t = 0.0;
        for (int w = 0; w < kBlock / 32; ++w) t += red[w][c];
        out[c] = t;
    }
}

__global__ void __launch_bounds__(kBlock) k_kick(int n, const int* __restrict__ types, TypeTable inv_m_acc,
                                                 double half_dt, double* __restrict__ vel,
                                                 const double* __restrict__ force)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double im = inv_m_acc.v[types[i]];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const size_t k = (size_t)a * n + i;
        vel[k] = half_kick(vel[k], half_dt, force[k], im);
    }
}

__global__ void __launch_bounds__(kBlock) k_sample(int n, const int* __restrict__ types, TypeTable mass,
                                                   const double* __restrict__ vel, const double* __restrict__ totals,
                                                   double* __restrict__ partial, unsigned int* __restrict__ counter,
                                                   double* __restrict__ thermo, int* __restrict__ sample_index,
                                                   int step_stride)
{
    __shared__ double red[kBlock / 32];
    __shared__ bool last;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double ke = 0.0;
    if (i < n) {
        const double m = mass.v[types[i]];
        for (int a = 0; a < 3; ++a) {
            const double v = vel[(size_t)a * n + i];
            ke += 0.5 * m * v * v;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ke += __shfl_xor_sync(0xffffffffu, ke, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = ke;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < kBlock / 32; ++w) s += red[w];
        partial[blockIdx.x] = s;
        __threadfence();
        last = (atomicAdd(counter, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double tot[1];
    last_block_sum<1>(partial, gridDim.x, tot);
    if (threadIdx.x != 0) return;
    const double s = tot[0];
    const int row = *sample_index;
    double* t = thermo + (size_t)row * 12;
    t[0] = (double)((row + 1) * step_stride);
    t[1] = totals[0];
    t[2] = s / kAcc;
    for (int k = 0; k < 9; ++k) t[3 + k] = totals[1 + k];
    *sample_index = row + 1;
    *counter = 0u;
}

// Stochastic velocity rescaling: with c = exp(-dt/tau), Kbar = N_f k_B T / 2 and the
// step's random numbers R1 ~ N(0,1), S ~ chi^2(N_f - 1),
//   K' = c K + (1 - c) Kbar / N_f (R1^2 + S) + 2 R1 sqrt(c (1 - c) K Kbar / N_f),
// and velocities are scaled by alpha = sqrt(K' / K).  The last block computes
// alpha (FP64) into *alpha and advances *step.
__global__ void __launch_bounds__(kBlock) k_bussi_ke(int n, const int* __restrict__ types, TypeTable mass,
                                                     const double* __restrict__ vel, double* __restrict__ partial,
                                                     unsigned int* __restrict__ counter, const double* __restrict__ noise,
                                                     int* __restrict__ step, double c, double kbar, double n_f,
                                                     double* __restrict__ alpha)
{
    __shared__ double red[kBlock / 32];
    __shared__ bool last;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double ke = 0.0;
    if (i < n) {
        const double m = mass.v[types[i]];
        for (int a = 0; a < 3; ++a) {
            const double v = vel[(size_t)a * n + i];
            ke += 0.5 * m * v * v;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ke += __shfl_xor_sync(0xffffffffu, ke, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = ke;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < kBlock / 32; ++w) s += red[w];
        partial[blockIdx.x] = s;
        __threadfence();
        last = (atomicAdd(counter, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double tot[1];
    last_block_sum<1>(partial, gridDim.x, tot);
    if (threadIdx.x != 0) return;
    const double K = tot[0] / kAcc;  // eV
    const int k = *step;
    const double r1 = noise[2 * k], chi = noise[2 * k + 1];
    double a2 = 1.0;
    if (K > 0.0) {
        const double Kn = c * K + (1.0 - c) * kbar / n_f * (r1 * r1 + chi) + 2.0 * r1 * sqrt(c * (1.0 - c) * K * kbar / n_f);
        a2 = Kn > 0.0 ? Kn / K : 0.0;
    }
    *alpha = sqrt(a2);
    *step = k + 1;
    *counter = 0u;
}

__global__ void __launch_bounds__(kBlock) k_scale_vel(int n, double* __restrict__ vel, const double* __restrict__ alpha)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double a = *alpha;
    vel[i] *= a;
    vel[(size_t)n + i] *= a;
    vel[(size_t)2 * n + i] *= a;
}

// (F_e . W)_b = sum_a Fe_a W[a][b]; W is row-major [9][n], totals[1 + 3a + b] its sum.
__global__ void __launch_bounds__(kBlock) k_hnemd_force(int n, double fe0, double fe1, double fe2,
                                                        const double* __restrict__ virial,
                                                        const double* __restrict__ totals, double* __restrict__ force)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double inv_n = 1.0 / n;
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        const double mean = (fe0 * totals[1 + b] + fe1 * totals[4 + b] + fe2 * totals[7 + b]) * inv_n;
        const double f = fe0 * virial[(size_t)b * n + i] + fe1 * virial[(size_t)(3 + b) * n + i] +
                         fe2 * virial[(size_t)(6 + b) * n + i];
        force[(size_t)b * n + i] += f - mean;
    }
}

// acc[6] accumulates (J_pot, J_kin) over the steps of a sampling interval; at a
// sampling step the last block writes acc / step_stride to row *sample_index of
// rows (read before k_sample advances it) and clears acc.
__global__ void __launch_bounds__(kBlock) k_heat(int n, const int* __restrict__ types, TypeTable mass,
                                                 const double* __restrict__ vel, const double* __restrict__ site,
                                                 const double* __restrict__ virial, double* __restrict__ partial,
                                                 unsigned int* __restrict__ counter, double* __restrict__ acc,
                                                 double* __restrict__ rows, const int* __restrict__ sample_index,
                                                 int sample, int step_stride)
{
    __shared__ double red[kBlock / 32][6];
    __shared__ bool last;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double j[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    if (i < n) {
        double v[3], v2 = 0.0;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            v[a] = vel[(size_t)a * n + i];
            v2 += v[a] * v[a];
        }
        const double Ei = 0.5 * mass.v[types[i]] * v2 / kAcc + site[i];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
#pragma unroll
            for (int b = 0; b < 3; ++b) j[a] += virial[(size_t)(3 * a + b) * n + i] * v[b];
            j[3 + a] = Ei * v[a];
        }
    }
#pragma unroll
    for (int k = 0; k < 6; ++k)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) j[k] += __shfl_xor_sync(0xffffffffu, j[k], o);
    if ((threadIdx.x & 31) == 0)
#pragma unroll
        for (int k = 0; k < 6; ++k) red[threadIdx.x >> 5][k] = j[k];
    __syncthreads();
    if (threadIdx.x < 6) {
        double s = 0.0;
        for (int w = 0; w < kBlock / 32; ++w) s += red[w][threadIdx.x];
        partial[(size_t)6 * blockIdx.x + threadIdx.x] = s;
        __threadfence();  // each writer publishes its partial before the block is counted
    }
    __syncthreads();
    if (threadIdx.x == 0) last = (atomicAdd(counter, 1u) == gridDim.x - 1);
    __syncthreads();
    if (!last) return;
    __threadfence();
    double tot[6];
    last_block_sum<6>(partial, gridDim.x, tot);
    if (threadIdx.x < 6) {
        double s = 0.0;
#pragma unroll
        for (int k = 0; k < 6; ++k)
            if (k == (int)threadIdx.x) s = tot[k];
        const double t = acc[threadIdx.x] + s;
        if (sample) {
            rows[(size_t)6 * (*sample_index) + threadIdx.x] = t / step_stride;
            acc[threadIdx.x] = 0.0;
        } else {
            acc[threadIdx.x] = t;
        }
    }
    if (threadIdx.x == 0) *counter = 0u;
}

__global__ void k_scale(int n, double* __restrict__ pos, double sx, double sy, double sz)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    pos[i] *= sx;
    pos[(size_t)n + i] *= sy;
    pos[(size_t)2 * n + i] *= sz;
}

static TypeTable make_table(const double* v, int T)
{
    TypeTable t;
    for (int k = 0; k < kMdMaxTypes; ++k) t.v[k] = k < T ? v[k] : 0.0;
    return t;
}

cudaError_t launch_kick(int n, const int* types, const double* inv_m_acc, int T, double half_dt, double* vel,
                        const double* force, cudaStream_t st)
{
    if (T > kMdMaxTypes) return cudaErrorInvalidValue;
    k_kick<<<(n + kBlock - 1) / kBlock, kBlock, 0, st>>>(n, types, make_table(inv_m_acc, T), half_dt, vel, force);
    return cudaGetLastError();
}

cudaError_t launch_sample(int n, const int* types, const double* mass, int T, const double* vel,
                          const double* totals, double* partial, unsigned int* counter, double* thermo,
                          int* sample_index, int step_stride, cudaStream_t st)
{
    if (T > kMdMaxTypes) return cudaErrorInvalidValue;
    k_sample<<<(n + kBlock - 1) / kBlock, kBlock, 0, st>>>(n, types, make_table(mass, T), vel, totals, partial,
                                                           counter, thermo, sample_index, step_stride);
    return cudaGetLastError();
}

cudaError_t launch_bussi(int n, const int* types, const double* mass, int T, double* vel, double* partial,
                         unsigned int* counter, const double* noise, int* step, double c, double kbar, double n_f,
                         double* alpha, cudaStream_t st)
{
    if (T > kMdMaxTypes) return cudaErrorInvalidValue;
    const int nb = (n + kBlock - 1) / kBlock;
    k_bussi_ke<<<nb, kBlock, 0, st>>>(n, types, make_table(mass, T), vel, partial, counter, noise, step, c, kbar, n_f,
                                      alpha);
    k_scale_vel<<<nb, kBlock, 0, st>>>(n, vel, alpha);
    return cudaGetLastError();
}

cudaError_t launch_hnemd_force(int n, const double fe[3], const double* virial, const double* totals, double* force,
                               cudaStream_t st)
{
    k_hnemd_force<<<(n + kBlock - 1) / kBlock, kBlock, 0, st>>>(n, fe[0], fe[1], fe[2], virial, totals, force);
    return cudaGetLastError();
}

cudaError_t launch_heat(int n, const int* types, const double* mass, int T, const double* vel, const double* site,
                        const double* virial, double* partial, unsigned int* counter, double* acc, double* rows,
                        const int* sample_index, int sample, int step_stride, cudaStream_t st)
{
    if (T > kMdMaxTypes) return cudaErrorInvalidValue;
    k_heat<<<(n + kBlock - 1) / kBlock, kBlock, 0, st>>>(n, types, make_table(mass, T), vel, site, virial, partial,
                                                         counter, acc, rows, sample_index, sample, step_stride);
    return cudaGetLastError();
}

cudaError_t launch_scale(int n, double* pos, double sx, double sy, double sz, cudaStream_t st)
{
    k_scale<<<(n + kBlock - 1) / kBlock, kBlock, 0, st>>>(n, pos, sx, sy, sz);
    return cudaGetLastError();
}

}  // namespace nep
