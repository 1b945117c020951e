/*
 * nep.h -- C ABI of the GB300 (sm_103a) NEP evaluator: energy, forces and per-bead
 * virial of a neuroevolution potential (NEP4 form) over a cell-list neighbour
 * list, and a velocity-Verlet MD step, as used by the NEP-CG and NEP-AACG models
 * of arXiv 2603.01234.
 *
 * What is computed (paper Sec. II.A, Sec. II.C):
 *   E   = sum_i U_i                                                   (Eq. 1)
 *   U_i = sum_mu w1_mu tanh(sum_nu w0_{mu nu} q_nu - b0_mu) - b1      (Eq. 2)
 *   q_n   = sum_{j != i} g_n(r_ij),            0 <= n < n_R           (Eq. 3)
 *   q_nl  = sum_m (-1)^m A_nlm A_nl(-m),        1 <= l <= l_max        (Eq. 4)
 *   A_nlm = sum_{j != i} g_n(r_ij) Y_lm(r_ij),  0 <= n < n_A           (Eq. 5)
 *   q4_n  = sum_{m1 m2 m3} (2 2 2; m1 m2 m3) A_n2m1 A_n2m2 A_n2m3     (four-body)
 *   q5_n  = (q_n1)^2                                                  (five-body)
 *   g_n(r) = sum_{k < K} c^{t_i t_j}_{nk} f_k(r)                        (Eq. 6)
 *   f_k(r) = 1/2 [T_k(2 (r/r_c - 1)^2 - 1) + 1] f_c(r)                  (Eq. 7)
 *   f_c(r) = 1/2 [1 + cos(pi r / r_c)] for r < r_c, else 0              (Eq. 8)
 *   F_i = -dE/dr_i
 *   W_i = sum_{j != i} r_ij (x) dU_j/dr_ji,  r_ij = r_j - r_i           (Eq. 15)
 *   W   = sum_i W_i                                                    (Eq. 16)
 * The radial descriptors use the radial cutoff and basis size, the angular ones
 * the angular cutoff and basis size (Sec. II.A).  Sec. II.A takes the four- and
 * five-body terms from the GPUMD paper (Fan et al., J. Chem. Phys. 157, 114801,
 * 2022); the forms above are the cubic invariant of the l = 2 moments (Wigner 3j
 * coupling, complex orthonormal Y_lm) and the quartic invariant of the l = 1
 * moments, each the only rotational invariant of its degree.  Type information enters only
 * through c^{t_i t_j}, the per-type network and the per-pair cutoffs.
 *
 * Conventions
 *   - Units: Angstrom, eV, amu, fs.  Outputs are always double precision.
 *   - Arrays of particles are structure-of-arrays: pos[3][n] means x[0..n), then
 *     y, then z.  Per-bead virials are [9][n] with component 3*alpha + beta.
 *   - Particle types are 0-based int32 < n_types.
 *   - Boxes are orthorhombic: box[3] side lengths, pbc[3] (1 = periodic).  On a
 *     periodic axis positions may lie anywhere (they are wrapped to [0, L)
 *     internally); an open axis uses [0, L) only to bin particles.
 *   - A pair is a neighbour when r < r_c(t_i, t_j).  Periodic images count,
 *     including images of the particle itself; r_c may exceed L/2 but not 2 L on a
 *     periodic axis (NEP_ERR_BOX_TOO_SMALL otherwise).
 *   - The caller owns every buffer it passes.  The library owns the model handle,
 *     the device copies of the parameters and a grow-only device workspace.
 *   - Calls on one handle must not overlap (the workspace is per handle); handles
 *     are independent.
 *   - Every call returns NEP_OK (0) or a negative NEP_ERR_* code and never
 *     throws; nep_last_error() returns a message for the last failure.
 */
#ifndef NEP_GB300_H
#define NEP_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define NEP_OK 0
#define NEP_ERR_ARG (-1)                /* invalid argument (message in nep_last_error) */
#define NEP_ERR_OOM (-2)                /* device allocation failed */
#define NEP_ERR_NEIGHBOR_OVERFLOW (-3)  /* a neighbour list outgrew its capacity during MD */
#define NEP_ERR_BOX_TOO_SMALL (-4)      /* r_c > 2 L on a periodic axis */
#define NEP_ERR_TIMEOUT (-5)            /* a bounded device wait ran out */
#define NEP_ERR_CUDA (-6)               /* a CUDA runtime error (message in nep_last_error) */
#define NEP_ERR_UNSUPPORTED (-7)        /* basis / descriptor sizes without a compiled kernel */

/* precision of the evaluation */
#define NEP_FP64 0  /* every step in double precision: the plain reference form */
#define NEP_FP32 1  /* FP32 descriptors, network and pair forces; FP64 reductions,
                       positions, velocities and integration */
#define NEP_FP32_BF16 2  /* NEP_FP32 with BF16 hidden-layer weights: W0 (Eq. 2) is rounded
                            to BF16 once, and both products of the hidden layer (the
                            pre-activations W0 q and dU/dq = W0^T (w1 (1 - h^2))) run on
                            tensor cores with each activation split into two BF16 terms
                            and FP32 accumulation.  The results are the FP32 form's for
                            the model with BF16-rounded W0, and forces stay the gradient
                            of its energy. */

/* memory kind of the caller's particle arrays */
#define NEP_HOST 0
#define NEP_DEVICE 1

typedef struct nep_model nep_model;

/* Library version, (major << 16) | minor. */
int nep_version(void);

/* Text of a status code; static storage. */
const char* nep_error_string(int code);

/* Message of the last failed call on this thread; static thread-local storage. */
const char* nep_last_error(void);

/*
 * Create a model on CUDA device `device` (Sec. II.A, Eq. 2-8).
 *   n_types            T >= 1
 *   rc_radial[T*T]     radial cutoff of the pair (t_i, t_j); must be symmetric
 *   rc_angular[T*T]    angular cutoff of the pair; must be symmetric
 *   n_basis_radial     K_R = N_bas^R + 1 Chebyshev basis functions (Eq. 6-7)
 *   n_basis_angular    K_A = N_bas^A + 1
 *   n_desc_radial      n_R = n_max^R + 1 radial descriptors (Eq. 3)
 *   n_desc_angular     n_A = n_max^A + 1 radial functions of the angular part
 *   l_max              l_max^3b (Eq. 4); currently 4
 *   l_max_4b           0 (no four-body term) or 2 (q4_n, n < n_A)
 *   l_max_5b           0 (no five-body term) or 1 (q5_n, n < n_A)
 *   hidden             N_neu, hidden-layer width (Eq. 2)
 *   c_radial[T][T][n_R][K_R], c_angular[T][T][n_A][K_A]   c^{t_i t_j}_{nk} (Eq. 6)
 *   w0[T][H][N_des], b0[T][H], w1[T][H], b1[T]            per-type network (Eq. 2)
 *     with N_des = n_R + n_A * (l_max + [l_max_4b = 2] + [l_max_5b = 1]),
 *     descriptor order q_0..q_{n_R-1}, then for l = 1..l_max, n = 0..n_A-1: q_nl,
 *     then q4_0..q4_{n_A-1} (if present), then q5_0..q5_{n_A-1} (if present).
 *     The four- and five-body terms share the angular g_n (c_angular).
 *   precision          NEP_FP64, NEP_FP32 or NEP_FP32_BF16
 * All arrays are host memory, row-major double, read during the call only.
 * Returns NEP_ERR_UNSUPPORTED for (n_R, n_A, K_R, K_A, l_max, l_max_4b, l_max_5b)
 * without a compiled kernel; the compiled set is listed by nep_supported_shape().
 * Models batched together (nep_compute_batch) must agree on whether any
 * many-body term is present.
 */
int nep_create(nep_model** out, int n_types, const double* rc_radial, const double* rc_angular,
               int n_basis_radial, int n_basis_angular, int n_desc_radial, int n_desc_angular,
               int l_max, int l_max_4b, int l_max_5b, int hidden, const double* c_radial,
               const double* c_angular,
               const double* w0, const double* b0, const double* w1, const double* b1,
               int precision, int device);

/* 1 if kernels for these sizes are compiled in, else 0. */
int nep_supported_shape(int n_desc_radial, int n_desc_angular, int n_basis_radial,
                        int n_basis_angular, int l_max, int l_max_4b, int l_max_5b);

/* Free the model and its device workspace.  NULL is accepted. */
int nep_destroy(nep_model* m);

/*
 * Energy, forces and virials of one configuration (Eq. 1-8, 15, 16).
 *   n                 number of particles, 1 <= n < 2^23
 *   types[n], pos[3][n]                    inputs
 *   box[3], pbc[3]    host arrays
 *   mem               NEP_HOST: every array pointer below is host memory;
 *                     NEP_DEVICE: every array pointer is device memory on the
 *                     model's device (box and pbc stay host arrays)
 *   stream            cudaStream_t to run on (NULL = the legacy default stream)
 *   energy_total[1], virial_total[9]       E and W (FP64 sums); may be NULL
 *   site_energy[n]    U_i; may be NULL
 *   force[3][n]       F_i; may be NULL
 *   virial[9][n]      W_i; may be NULL
 * The call returns when the results are written (it synchronises `stream`).
 * Neighbour-list capacity grows automatically.
 */
int nep_compute(nep_model* m, int n, const int32_t* types, const double* pos, const double box[3],
                const int32_t pbc[3], int mem, void* stream, double* energy_total, double* virial_total,
                double* site_energy, double* force, double* virial);

/*
 * Many configurations in one pass of the pipeline (the batched form): one cell
 * build, one neighbour pass, one descriptor pass and one force pass cover every
 * request, each request with its own box, cell grid and model.
 *   models[n_models]   handles created with the same device, precision and
 *                      descriptor / basis sizes (their types, cutoffs, widths and
 *                      parameters may differ); the batch uses models[0]'s workspace
 *   n_req              number of requests; request r has req_n[r] particles and
 *                      uses models[req_model[r]]
 *   req_box[n_req][3], req_pbc[n_req][3]      host arrays
 *   types, pos         the requests' particles concatenated: request r's types at
 *                      types + o_r and its positions as an SoA block [3][n_r] at
 *                      pos + 3 o_r, where o_r = sum_{q<r} n_q
 *   mem, stream        as in nep_compute (all arrays below in the same memory)
 *   energy[n_req], virial_total[n_req][9]     per-request totals (FP64 sums)
 *   site_energy        [sum n_r] concatenated like types, or NULL
 *   force              blocks [3][n_r] at force + 3 o_r (NULL allowed)
 *   virial             blocks [9][n_r] at virial + 9 o_r, or NULL
 * Results equal those of one nep_compute per request.  Synchronous like
 * nep_compute; at most 2^23 particles in total.
 * The call synchronises once: the whole pipeline, the output copies and the status
 * words are enqueued together, and a neighbour list that outgrew its capacity is
 * grown and the batch run again (the capacity then stays).  Capacities are
 * rounded up to size classes (at most 1/8 more than the batch) and the pipeline is
 * captured as a CUDA graph cached on models[0] by its launch shapes and pointers,
 * so later batches of a similar size (and the same buffers) replay it.
 */
int nep_compute_batch(nep_model* const* models, int n_models, int n_req, const int32_t* req_n,
                      const int32_t* req_model, const double* req_box, const int32_t* req_pbc,
                      const int32_t* types, const double* pos, int mem, void* stream, double* energy,
                      double* virial_total, double* site_energy, double* force, double* virial);

/*
 * n_steps velocity-Verlet NVE steps (the MD loop of Sec. III.D):
 *   v += dt/2 F/m;  r += dt v;  wrap periodic axes;  F = F(r);  v += dt/2 F/m.
 *   masses[T]         host, amu per type
 *   pos[3][n], vel[3][n] (Angstrom/fs), force[3][n]   state, updated in place
 *   forces_valid      1: `force` holds F(pos) on entry; 0: it is computed first
 *   dt_fs             time step in fs
 *   sample_every      > 0: after every sample_every-th step one thermo row is
 *                     written; 0: no rows
 *   thermo            host [n_steps / sample_every][12]: step, E_pot, E_kin,
 *                     W_tot[9] (eV); may be NULL when sample_every == 0
 *   mem, stream       as in nep_compute (box, pbc, masses, thermo: host)
 * The steps run in chunks (sample_every steps, else up to 50); one chunk is
 * captured as a CUDA graph, cached on the handle by its arguments, and replayed.
 * Synchrony: with mem = NEP_DEVICE and a non-NULL stream the call only enqueues
 * work on `stream` and returns; device-side status (neighbour overflow,
 * non-finite positions) is then reported by the next call on the handle or by
 * nep_sync(), and thermo rows are valid after nep_sync().  Otherwise the call
 * returns when the steps are done.
 * Neighbour-list capacity is probed synchronously once per configuration shape
 * (n and cell grid) and set to 1.5 times the largest count plus 8; it is raised
 * the same way when the counts, projected two chunks ahead at the last chunk's
 * growth, pass 80% of it.  That check runs between chunks and lags one chunk behind
 * the GPU, so a sudden jump in the counts (beyond the projection and the 1.5x
 * headroom within two chunks) can still overflow; short chunks (a small
 * sample_every) shrink that window.  NEP_ERR_NEIGHBOR_OVERFLOW means a list
 * outgrew its capacity: the state of that call is undefined and the capacity is
 * raised for the next, so the caller retries from its saved state.
 */
int nep_md_step(nep_model* m, int n, const int32_t* types, const double* masses, const double box[3],
                const int32_t pbc[3], double* pos, double* vel, double* force, int forces_valid,
                int n_steps, double dt_fs, int sample_every, double* thermo, int mem, void* stream);

/*
 * n_steps velocity-Verlet steps in the canonical ensemble (the NVT runs of the
 * paper's benchmark, Sec. III.D): nep_md_step followed, after every step, by
 * stochastic velocity rescaling (Bussi, Donadio, Parrinello, J. Chem. Phys. 126,
 * 014101, 2007).  With K the kinetic energy, N_f = 3 n - 3, Kbar = N_f k_B T / 2,
 * c = exp(-dt / tau) and the step's random numbers R1 ~ N(0, 1) and
 * S ~ chi^2(N_f - 1):
 *   K' = c K + (1 - c) (Kbar / N_f) (R1^2 + S) + 2 R1 sqrt(c (1 - c) K Kbar / N_f),
 * and every velocity is multiplied by sqrt(K' / K) (FP64).
 *   temperature_K, tau_fs   target temperature and coupling time
 *   noise                   host [n_steps][2]: (R1, S) of each step; the caller
 *                           draws them, so runs are reproducible
 * Every other argument and rule as in nep_md_step.
 */
int nep_md_step_nvt(nep_model* m, int n, const int32_t* types, const double* masses, const double box[3],
                    const int32_t pbc[3], double* pos, double* vel, double* force, int forces_valid, int n_steps,
                    double dt_fs, double temperature_K, double tau_fs, const double* noise, int sample_every,
                    double* thermo, int mem, void* stream);

/*
 * n_steps homogeneous non-equilibrium MD (HNEMD) steps for the thermal
 * conductivity (Sec. III.B; the method of Fan et al., Phys. Rev. B 99, 064308,
 * 2019).  Each step is the nep_md_step_nvt step (or the NVE step when noise is
 * NULL) with a driving force added to the force after every evaluation:
 *   F_i += F_e . W_i - (1/n) sum_j F_e . W_j,   (F_e . W_i)_b = sum_a Fe_a W_i[a][b],
 * W_i the per-particle virial of Eq. 15.  The forces then add power F_e . J_pot
 * and no net momentum.  After the step's thermostat the heat current
 *   J_pot = sum_i W_i v_i,   J_kin = sum_i (1/2 m_i v_i^2 + U_i) v_i
 * (Fan et al., Phys. Rev. B 92, 094301, 2015; eV Angstrom / fs) is taken, and its
 * average over each sampling interval is written.  The thermal conductivity
 * follows as kappa_ab = <J_a> / (T V Fe_b).
 *   fe             host [3], F_e in 1/Angstrom
 *   noise          host [n_steps][2] as in nep_md_step_nvt, or NULL for no
 *                  thermostat (temperature_K and tau_fs are then ignored)
 *   heat           host [n_steps / sample_every][6]: (J_pot, J_kin) averaged over
 *                  the sample_every steps of each interval; NULL for none
 *                  (requires sample_every > 0 otherwise)
 *   force          the total force, driving force included: on entry when
 *                  forces_valid is 1 (as left by a previous call), on return
 * Every other argument and rule as in nep_md_step.
 */
int nep_md_step_hnemd(nep_model* m, int n, const int32_t* types, const double* masses, const double box[3],
                      const int32_t pbc[3], double* pos, double* vel, double* force, int forces_valid, int n_steps,
                      double dt_fs, const double fe[3], double temperature_K, double tau_fs, const double* noise,
                      int sample_every, double* thermo, double* heat, int mem, void* stream);

/*
 * Coarse-grained mapping of an atomistic configuration onto beads (Sec. II.B-C):
 *   R_I = sum_{i in I} (m_i / M_I) r_i                 bead position (Eq. 9)
 *   F_I = sum_{i in I} f_i                             bead force    (Eq. 12)
 *   W_I = sum_{i in I} W_i                             bead virial   (Eq. 14)
 * Groups are CSR: bead I owns atoms group_atoms[group_start[I] .. group_start[I+1]).
 * On periodic axes every atom is taken at its image nearest to the group's first
 * atom (groups must be smaller than half the box) and R_I is wrapped to [0, L).
 *   atom_mass[n_aa], atom_pos[3][n_aa]; atom_force[3][n_aa], atom_virial[9][n_aa]
 *   may be NULL (then the matching bead output is left alone)
 *   accumulate   0: overwrite bead_force / bead_virial; 1: add to them (the
 *                constrained time averages of Eq. 12 and Eq. 14 are such sums
 *                divided by the number of frames)
 *   bead_pos[3][n_cg], bead_force[3][n_cg], bead_virial[9][n_cg]   outputs or NULL
 * mem / stream as in nep_compute; the handle supplies device and workspace.
 */
int nep_cg_map(nep_model* m, int n_cg, const int32_t* group_start, const int32_t* group_atoms, int n_aa,
               const double* atom_mass, const double* atom_pos, const double* atom_force,
               const double* atom_virial, const double box[3], const int32_t pbc[3], int accumulate, int mem,
               void* stream, double* bead_pos, double* bead_force, double* bead_virial);

/*
 * Virial correction of a coarse-grained training target (Eq. 17):
 *   W -> W + (N_AA - N_CG) k_B T I,   virial[9] row-major, eV.  Host function.
 */
int nep_virial_correction(double* virial, int n_atoms, int n_beads, double temperature_K);

/* Wait for the handle's asynchronous MD work and return its deferred status. */
int nep_sync(nep_model* m);

/* pos[3][n] *= scale[3] per axis (affine box strain); same memory rules as above. */
int nep_scale_positions(nep_model* m, int n, double* pos, const double scale[3], int mem, void* stream);

/*
 * Neighbour lists as built by the library (for inspection and tests).
 *   kind        0 = radial (r < r_c^R), 1 = angular (r < r_c^A)
 *   capacity    entries per particle in the output arrays
 *   count[n]    number of neighbours of each particle (may exceed capacity)
 *   j[n][capacity], shift[n][capacity][3]   neighbour index and periodic image
 *               shift in box lengths, relative to the wrapped positions
 * Host buffers; inputs as in nep_compute with mem = NEP_HOST.
 */
int nep_neighbors(nep_model* m, int n, const int32_t* types, const double* pos, const double box[3],
                  const int32_t pbc[3], int kind, int capacity, int32_t* count, int32_t* j, int32_t* shift);

/*
 * Per-stage device timing of MD steps (CUDA events on the launch stream).  While
 * enabled, nep_md_step runs its steps without graph capture and records events
 * around each stage of every step.  Enabling (or re-enabling) resets the sums.
 */
int nep_set_timing(nep_model* m, int enable);

/*
 * Summed device time in ms of each stage over the timed steps, waiting for the
 * pending events first:  stage_ms[6] = opening kick+drift+binning, rest of the
 * cell build, neighbour lists, descriptor+network+angular forces, radial
 * forces+outputs (with the closing kick unless the HNEMD force is on), and what
 * follows (separate kick, thermostat, heat current, thermo row);  steps = steps
 * timed.
 */
int nep_get_timing(nep_model* m, double* stage_ms, long long* steps);

/*
 * nep_compute_static -- nep_compute that allocates no device memory.
 * The paper has no counterpart: this exists for callers of this library that
 * cannot allocate.  cudaFree, and cudaMalloc when its pool must grow, synchronise
 * the whole device; an allocation can fail mid-simulation when other parts of the
 * program hold the memory; and hosts that budget every byte of device memory at
 * start-up (an MD engine, a serving process) forbid hidden allocations.
 *
 * The scratch is one fixed array in device global memory that is part of the
 * library image: 15,456,000 bytes (about 14.7 MiB), held on every GPU that loads the
 * library until the process exits.  Limits of one call: n <= 4096 particles, a
 * model of at most 4 types, a cell grid of at most 32768 cells, at most 256
 * radial and 128 angular neighbours per particle.  Larger inputs are rejected with
 * NEP_ERR_ARG (the message names the limit); more neighbours give
 * NEP_ERR_NEIGHBOR_OVERFLOW.
 *
 *   m             a handle from nep_create (its parameters are read, nothing grows)
 *   types, pos    device arrays as in nep_compute with mem = NEP_DEVICE
 *   box, pbc      host arrays
 *   stream        cudaStream_t, or NULL for the legacy default stream
 *   outputs       device arrays, each may be NULL, as in nep_compute
 * The results equal nep_compute's (same kernels, same order).  The call returns
 * when they are written; it calls no cudaMalloc, cudaFree or other allocating
 * routine.  Set-up: the first call on a device, with that device current, looks
 * up the array's device address (cudaGetSymbolAddress) once; make that first call
 * before any stream capture.  Every call on every handle shares the one array and
 * leaves its contents behind (the words that must start at zero are cleared by
 * each call), so calls whose GPU work overlaps -- from different handles, streams
 * or threads -- race and give wrong results: serialise them.
 */
int nep_compute_static(nep_model* m, int n, const int32_t* types, const double* pos, const double box[3],
                       const int32_t pbc[3], void* stream, double* energy_total, double* virial_total,
                       double* site_energy, double* force, double* virial);

/*
 * Autotuner.  The FP32 descriptor kernel is compiled in variants that keep 2 or 3
 * thread blocks resident per SM, and the radial-force kernel in variants that keep
 * 3, 4 or 5 resident (a register budget per thread) and walk the neighbour list in
 * groups of 4 or 8 entries (the next group's entries load while the current group
 * is evaluated).  nep_autotune evaluates the configuration several times with each
 * variant, times the two kernels separately with CUDA events, and keeps for each
 * kernel its default (3 blocks; groups of 4) unless another variant is at least 5%
 * faster; the first nep_md_step of a new configuration shape (n and cell grid) does
 * the same unless disabled.  All variants give identical results.  Inputs as in
 * nep_compute; the chosen variants are returned (any output may be NULL).
 */
int nep_autotune(nep_model* m, int n, const int32_t* types, const double* pos, const double box[3],
                 const int32_t pbc[3], int mem, void* stream, int* mb_desc, int* mb_force, int* chunk);

/* Set the variants (descriptor 2 or 3 blocks per SM; radial force 3, 4 or 5 blocks
 * per SM and chunk 4 or 8) and whether MD calls tune automatically (1/0); other
 * values give NEP_ERR_ARG. */
int nep_set_tuning(nep_model* m, int autotune, int mb_desc, int mb_force, int chunk);

/* The variants in use. */
int nep_get_tuning(nep_model* m, int* mb_desc, int* mb_force, int* chunk);

/* Current neighbour-list capacities (entries per particle). */
int nep_get_capacity(nep_model* m, int* radial, int* angular);

/* Set the neighbour-list capacities (entries per particle, >= 1).  A list holds
 * capacity x n entries, at most 2^32 (larger lists give NEP_ERR_ARG when built). */
int nep_set_capacity(nep_model* m, int radial, int angular);

/*
 * Device workspace bytes that one request adds to a batch of nep_compute_batch on
 * models[0]'s workspace (the same models[n_models] as the batch; the request uses
 * models[model], n particles, box and pbc as in the batch): particle arrays
 * (strided by the batch's largest type count), neighbour lists at models[0]'s
 * current capacities (or, before it has evaluated anything, the first-call
 * estimate from this request's density), cell arrays, work items and the request's
 * own entries, plus the staging of host-memory calls.  A batch allocates at most
 * 9/8 of the sum over its requests (size classes).  For admission of requests by
 * memory; computes on the host only.
 */
int nep_request_workspace(nep_model* const* models, int n_models, int model, int n, const double box[3],
                          const int32_t pbc[3], size_t* bytes);

/* Device bytes m's workspace holds now (every buffer the library allocated for
 * evaluations and MD on m; the model parameters are not counted). */
int nep_workspace_bytes(nep_model* m, size_t* bytes);

/* Page-locked host memory (cudaMallocHost) for request and result buffers: copies
 * between it and the device run at full link speed.  Free with nep_host_free. */
int nep_host_alloc(size_t bytes, void** out);
int nep_host_free(void* p);

#ifdef __cplusplus
}
#endif

#endif /* NEP_GB300_H */
