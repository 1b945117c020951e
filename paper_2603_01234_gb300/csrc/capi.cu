// C ABI (include/nep.h) and the runtime behind it: model parameters on the device,
// a grow-only workspace per handle, the per-configuration pipeline
//   cell build -> neighbour lists -> descriptor + network -> forces + virials + FP64 totals
// and the velocity-Verlet loop captured as a CUDA graph.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <functional>
#include <string>
#include <vector>

#include "nep.h"
#include "nep_common.cuh"

using namespace nep;

namespace {

thread_local std::string g_last_error;

int fail(int code, const std::string& msg)
{
    g_last_error = msg;
    return code;
}

#define NEP_CUDA(call)                                                                                 \
    do {                                                                                               \
        cudaError_t e_ = (call);                                                                       \
        if (e_ != cudaSuccess) {                                                                       \
            return fail(e_ == cudaErrorMemoryAllocation ? NEP_ERR_OOM : NEP_ERR_CUDA,                  \
                        std::string(#call) + ": " + cudaGetErrorString(e_));                           \
        }                                                                                              \
    } while (0)

#define NEP_TRY(call)              \
    do {                           \
        int r_ = (call);           \
        if (r_ != NEP_OK) return r_; \
    } while (0)

constexpr double kAcc = 9.648533212e-3;  // 1 eV/(A amu) in A/fs^2

template <typename T>
int grow(T*& p, size_t& cap, size_t want)
{
    if (want <= cap && p) return NEP_OK;
    size_t nc = std::max(want, cap + cap / 4);
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
    cudaError_t e = cudaMalloc((void**)&p, nc * sizeof(T) + 16);
    if (e != cudaSuccess) return fail(NEP_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    cap = nc;
    return NEP_OK;
}

struct Buf {
    void* p = nullptr;
    size_t cap = 0;  // bytes
    int ensure(size_t bytes)
    {
        if (bytes <= cap && p) return NEP_OK;
        size_t nc = std::max(bytes, cap + cap / 4);
        if (p) cudaFree(p);
        p = nullptr;
        cap = 0;
        cudaError_t e = cudaMalloc(&p, nc + 256);
        if (e != cudaSuccess) return fail(NEP_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
        cap = nc;
        return NEP_OK;
    }
    void release()
    {
        if (p) cudaFree(p);
        p = nullptr;
        cap = 0;
    }
    template <typename T>
    T* as() const { return reinterpret_cast<T*>(p); }
};

// Per-stage device timing of MD steps: a ring of event sets, one set per step.
// Stage k of a step lies between events k and k+1:
//   0 kick+drift, 1 cell build, 2 neighbour lists, 3 descriptor+network,
//   4 force+virial, 5 kick (+ sample)
struct StageTimer {
    static constexpr int kRing = 64, kEv = 7;
    bool on = false;
    bool created = false;
    cudaEvent_t ev[kRing][kEv];
    bool pending[kRing] = {};
    int head = 0;
    double acc[kEv - 1] = {};
    long long steps = 0;
    int create()
    {
        if (created) return 0;
        for (int r = 0; r < kRing; ++r)
            for (int k = 0; k < kEv; ++k)
                if (cudaEventCreate(&ev[r][k]) != cudaSuccess) return -1;
        created = true;
        return 0;
    }
    void collect(int r)
    {
        if (!pending[r]) return;
        cudaEventSynchronize(ev[r][kEv - 1]);
        for (int k = 0; k + 1 < kEv; ++k) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, ev[r][k], ev[r][k + 1]) == cudaSuccess) acc[k] += ms;
        }
        ++steps;
        pending[r] = false;
    }
    void drain()
    {
        for (int r = 0; r < kRing; ++r) collect((head + r) % kRing);
    }
    void reset()
    {
        drain();
        for (double& a : acc) a = 0.0;
        steps = 0;
    }
    void destroy()
    {
        if (!created) return;
        drain();
        for (int r = 0; r < kRing; ++r)
            for (int k = 0; k < kEv; ++k) cudaEventDestroy(ev[r][k]);
        created = false;
    }
};

struct GraphCache {
    cudaGraphExec_t exec = nullptr;
    std::vector<unsigned char> key;
    void reset()
    {
        if (exec) cudaGraphExecDestroy(exec);
        exec = nullptr;
        key.clear();
    }
};
constexpr size_t kEvalGraphs = 16;  // evaluation graphs kept per handle


// Host copy of one batch layout and its device tables (counts, requests, work
// items, models).  Launch shapes and workspace strides follow the capacities
// (n_cap, items_cap, ncell_cap >= the counts): equal to the counts for a single
// configuration, rounded up to a size class for batches, so that batches of
// similar size replay one captured graph.
struct Plan {
    std::vector<ReqInfo> reqs;
    std::vector<WorkItem> items;
    std::vector<unsigned char> models;  // ModelDesc<real> entries, raw bytes
    int n = 0, ncell = 0, n_models = 0;
    int n_cap = 0, items_cap = 0, ncell_cap = 0, req_cap = 0;
    int Tmax = 1;
    size_t smem_desc = 0, smem_force = 0, smem_nbr = 0;
    std::vector<unsigned char> key;     // identity of the uploaded tables
    Buf dev;                            // [counts | reqs | items | models] on the device
    size_t off_reqs = 0, off_items = 0, off_models = 0;
};

// Size class of a batch dimension: x rounded up to a multiple of 1/8 of the power
// of two below it (at least `quantum`), so a class wastes at most 1/8.
int size_class(int x, int quantum)
{
    if (x <= quantum) return quantum;
    int p2 = 1;
    while (p2 * 2 <= x) p2 *= 2;
    const int step = std::max(quantum, p2 / 8);
    return (int)(((long long)x + step - 1) / step * step);
}

// Capacities equal to the counts (single configurations, MD) or rounded to size
// classes (batches).
void set_caps(Plan& p, bool classes)
{
    const int n_items = (int)p.items.size();
    if (!classes) {
        p.n_cap = p.n;
        p.items_cap = n_items;
        p.ncell_cap = p.ncell;
        p.req_cap = (int)p.reqs.size();
        return;
    }
    p.n_cap = size_class(p.n, kBlock);
    p.items_cap = size_class(n_items, 8);
    p.ncell_cap = (p.ncell + kScanItems - 1) / kScanItems * kScanItems;  // whole scan tiles
    p.req_cap = (int)p.reqs.size();
}

}  // namespace

struct nep_model {
    int device = 0;
    int precision = NEP_FP32;
    int T = 1, nR = 0, nA = 0, KR = 0, KA = 0, L = 4, H = 0, ND = 0, KRP = 0;
    int L4 = 0, L5 = 0;  // l_max of the four-body (0 or 2) and five-body (0 or 1) terms
    int MBT = 0;         // 1: the kernels carry both many-body blocks (ND counts them)
    double rc_max = 0.0;
    std::vector<double> rcR, rcA;
    ParamLayout off{};
    Buf params;
    size_t real_size = 4;
    size_t smem_desc = 0, smem_force = 0;
    int mnR = 0, mnA = 0;  // neighbour capacities
    int mb_desc = 3, mb_force = 3;  // register-cap variants of the FP32 evaluation kernels
    int ch_force = 4;               // neighbour entries per walk group of the FP32 radial kernel
    bool autotune = true;           // tune the variants on the first MD call of a configuration shape
    cudaStream_t st = nullptr;   // internal stream, used when the caller passes NULL
    cudaStream_t cur = nullptr;  // stream of the call in progress
    cudaEvent_t ev_in = nullptr, ev_out = nullptr, ev_flags = nullptr, ev_plan = nullptr;
    int* h_async = nullptr;      // pinned copy of the status words after an asynchronous MD call
    bool async_pending = false;
    cudaStream_t async_stream = nullptr;
    bool plan_pending = false;   // a table upload from the pinned staging is in flight
    // MD sizing state: the last configuration the capacities were checked for
    int md_n = -1;
    CellGrid md_grid{};
    // workspace
    Buf cell_of, rec_user, perm_tmp, perm, rec_s, cell_s, cntR, cntA, nlR, nlA, U, e, phi;
    Buf rec32;  // FP64 form: FP32 copies of the sorted records (neighbour screening)
    Buf cell_count, cell_local, block_off, cell_fill, cell_start;
    Buf partial, partial2, counters, gcounters, totals, flags, thermo, sample_index;
    Buf acc;  // FP32 form: force and virial fixed-point lines, thread virial sums (acc_bytes)
    bool eval_per_bead = false;  // the evaluation in progress returns per-particle virials
    bool cells_dirty = true;     // the cell counters may be non-zero (new buffer, or a build that failed)
    Buf types_d, pos_d, vel_d, force_d, virial_d, site_d, force_tmp, totals_tmp;
    Buf noise_d, bussi;  // thermostat: random numbers of the call; [step, alpha] words
    Buf md_virial, md_site, heat, heat_rows;  // HNEMD: per-particle W_i and U_i; acc[6] + counter; rows
    int* h_flags = nullptr;        // pinned: maxcnt[2], err
    double* h_totals = nullptr;    // pinned [10 * requests]
    size_t h_totals_cap = 0;
    unsigned char* h_stage = nullptr;  // pinned staging of the plan tables
    size_t h_stage_cap = 0;
    size_t n_lists = 0;  // particles the lists were sized for
    Plan plan;
    GraphCache graph;                    // MD step chunk
    std::vector<GraphCache> eval_graphs;  // nep_compute / nep_compute_batch evaluations
    std::vector<size_t> eval_seen;        // hashes of evaluation shapes seen once (captured on the next)
    StageTimer timer;
};

namespace {

struct Guard {  // make the device current for the duration of a call
    int prev = -1;
    explicit Guard(int dev)
    {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~Guard()
    {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

int make_grid(const nep_model* m, double rc_max, const double box[3], const int32_t pbc[3], CellGrid& g)
{
    long long ncell = 1;
    for (int a = 0; a < 3; ++a) {
        if (!(box[a] > 0.0) || !isfinite(box[a])) return fail(NEP_ERR_ARG, "box lengths must be positive and finite");
        g.pbc[a] = pbc[a] ? 1 : 0;
        g.box[a] = box[a];
        int nc = (int)floor(box[a] / rc_max);
        if (nc < 1) nc = 1;
        if (nc > 1024) nc = 1024;
        g.nc[a] = nc;
        g.len[a] = box[a] / nc;
        g.inv_len[a] = 1.0 / g.len[a];
        if (g.pbc[a]) {
            int S = (int)ceil(rc_max / g.len[a] - 1e-12);
            if (S < 1) S = 1;
            if (S > kMaxS) return fail(NEP_ERR_BOX_TOO_SMALL, "cutoff exceeds twice the box length on a periodic axis");
            g.S[a] = S;
        } else {
            g.S[a] = 1;
        }
        ncell *= nc;
    }
    if (ncell > (long long)kScanItems * kScanItems) return fail(NEP_ERR_ARG, "cell grid too large");
    g.ncell = (int)ncell;
    (void)m;
    return NEP_OK;
}

int make_grid(const nep_model* m, const double box[3], const int32_t pbc[3], CellGrid& g)
{
    return make_grid(m, m->rc_max, box, pbc, g);
}

// ---- plans -------------------------------------------------------------------
template <typename real>
ModelDesc<real> model_desc(const nep_model* m)
{
    ModelDesc<real> d;
    d.params = m->params.as<real>();
    d.off = m->off;
    d.T = m->T;
    d.H = m->H;
    return d;
}

// Work items: the request's particles cut into blocks of kBlock.
void add_request(Plan& p, const CellGrid& g, int n, int model)
{
    ReqInfo r;
    r.g = g;
    r.cell_base = p.ncell;
    r.begin = p.n;
    r.n = n;
    r.model = model;
    r.item_begin = (int)p.items.size();
    for (int b = 0; b < n; b += kBlock) p.items.push_back(WorkItem{(int)p.reqs.size(), p.n + b, p.n + std::min(n, b + kBlock)});
    r.item_end = (int)p.items.size();
    p.reqs.push_back(r);
    p.n += n;
    p.ncell += g.ncell;
}

template <typename real>
void set_models(Plan& p, nep_model* const* models, int n_models)
{
    p.n_models = n_models;
    p.models.resize(sizeof(ModelDesc<real>) * n_models);
    p.Tmax = 1;
    p.smem_desc = p.smem_force = p.smem_nbr = 0;
    for (int k = 0; k < n_models; ++k) {
        ModelDesc<real> d = model_desc<real>(models[k]);
        memcpy(p.models.data() + k * sizeof d, &d, sizeof d);
        p.Tmax = std::max(p.Tmax, models[k]->T);
        p.smem_desc = std::max(p.smem_desc, models[k]->smem_desc);
        p.smem_force = std::max(p.smem_force, models[k]->smem_force);
        p.smem_nbr = std::max(p.smem_nbr, neighbor_smem<real>(models[k]->T));
    }
}

constexpr size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

// Upload the plan's tables (through pinned staging) unless they are unchanged.
int upload_plan(nep_model* m, Plan& p, bool force_upload = false)
{
    std::vector<unsigned char> key;
    auto put = [&](const void* q, size_t s) {
        const unsigned char* b = (const unsigned char*)q;
        key.insert(key.end(), b, b + s);
    };
    const PlanCounts counts{p.n, (int)p.items.size(), p.ncell, (int)p.reqs.size()};
    put(&counts, sizeof counts);
    put(p.reqs.data(), sizeof(ReqInfo) * p.reqs.size());
    put(p.items.data(), sizeof(WorkItem) * p.items.size());
    put(p.models.data(), p.models.size());
    if (!force_upload && key == p.key && p.dev.p) return NEP_OK;
    // [counts | models | items | requests]: the items region is laid out by
    // capacity, so the offsets (which the kernels' arguments carry, and a captured
    // graph keeps) depend only on the model count and the item capacity
    p.off_models = align16(sizeof(PlanCounts));
    p.off_items = p.off_models + align16(p.models.size());
    p.off_reqs = p.off_items + align16(sizeof(WorkItem) * std::max<size_t>(p.items_cap, p.items.size()));
    const size_t bytes = p.off_reqs + sizeof(ReqInfo) * p.reqs.size();
    NEP_TRY(p.dev.ensure(bytes));
    if (m->plan_pending) NEP_CUDA(cudaEventSynchronize(m->ev_plan));  // staging free again
    m->plan_pending = false;
    if (bytes > m->h_stage_cap) {
        if (m->h_stage) cudaFreeHost(m->h_stage);
        m->h_stage = nullptr;
        m->h_stage_cap = 0;
        NEP_CUDA(cudaMallocHost((void**)&m->h_stage, bytes + bytes / 2));
        m->h_stage_cap = bytes + bytes / 2;
    }
    memcpy(m->h_stage, &counts, sizeof counts);
    memcpy(m->h_stage + p.off_reqs, p.reqs.data(), sizeof(ReqInfo) * p.reqs.size());
    memcpy(m->h_stage + p.off_items, p.items.data(), sizeof(WorkItem) * p.items.size());
    memcpy(m->h_stage + p.off_models, p.models.data(), p.models.size());
    NEP_CUDA(cudaMemcpyAsync(p.dev.p, m->h_stage, bytes, cudaMemcpyHostToDevice, m->cur));
    NEP_CUDA(cudaEventRecord(m->ev_plan, m->cur));
    m->plan_pending = true;
    p.key = key;
    return NEP_OK;
}

const PlanCounts* d_counts(const Plan& p) { return p.dev.as<PlanCounts>(); }
const ReqInfo* d_reqs(const Plan& p) { return (const ReqInfo*)((const unsigned char*)p.dev.p + p.off_reqs); }
const WorkItem* d_items(const Plan& p) { return (const WorkItem*)((const unsigned char*)p.dev.p + p.off_items); }
template <typename real>
const ModelDesc<real>* d_models(const Plan& p)
{
    return (const ModelDesc<real>*)((const unsigned char*)p.dev.p + p.off_models);
}

template <typename real>
int single_plan(nep_model* m, int n, const CellGrid& g)
{
    Plan& p = m->plan;
    p.reqs.clear();
    p.items.clear();
    p.n = p.ncell = 0;
    add_request(p, g, n, 0);
    set_caps(p, false);
    nep_model* one[1] = {m};
    set_models<real>(p, one, 1);
    return upload_plan(m, p);
}

// ---- workspace ---------------------------------------------------------------
// The FP32 form's accumulators for n particles in one buffer: force lines, virial
// lines, thread virial sums.
size_t acc_bytes(size_t n) { return 32 * n + 96 * n + 36 * n; }
unsigned long long* acc_force(void* base) { return (unsigned long long*)base; }
unsigned long long* acc_virial(void* base, size_t n) { return (unsigned long long*)((char*)base + 32 * n); }
float* acc_wsum(void* base, size_t n) { return (float*)((char*)base + 128 * n); }

int ensure_particles(nep_model* m, int n, int n_items, int n_req, int Tmax)
{
    const size_t rs = m->real_size;
    const size_t rec_sz = 4 * rs;
    NEP_TRY(m->cell_of.ensure(sizeof(int) * n));
    NEP_TRY(m->rec_user.ensure(rec_sz * n));
    NEP_TRY(m->perm_tmp.ensure(sizeof(int) * n));
    NEP_TRY(m->perm.ensure(sizeof(int) * n));
    NEP_TRY(m->rec_s.ensure(rec_sz * n));
    NEP_TRY(m->cell_s.ensure(sizeof(int) * n));
    NEP_TRY(m->cntR.ensure(sizeof(int) * n));
    NEP_TRY(m->cntA.ensure(sizeof(int) * n));
    NEP_TRY(m->U.ensure(rs * n));
    NEP_TRY(m->e.ensure(rs * Tmax * m->KRP * (size_t)n));
    if (m->precision == NEP_FP64) NEP_TRY(m->phi.ensure(rs * kPsiComp * phi_pad(m->nA) * (size_t)n));  // FP32 keeps them in registers
    if (m->precision == NEP_FP64) NEP_TRY(m->rec32.ensure(16 * (size_t)n));
    NEP_TRY(m->partial.ensure(sizeof(double) * 10 * (size_t)n_items));
    // FP32 form: force lines [n][4] u64, virial lines [n][12] u64, thread virial sums [9][n] float
    if (m->precision != NEP_FP64) NEP_TRY(m->acc.ensure(acc_bytes(n)));
    NEP_TRY(m->partial2.ensure(sizeof(double) * 6 * ((n + kBlock - 1) / kBlock)));
    NEP_TRY(m->force_tmp.ensure(sizeof(double) * 3 * (size_t)n));
    const size_t old_req = m->counters.cap / sizeof(unsigned int);
    NEP_TRY(m->counters.ensure(sizeof(unsigned int) * (n_req + 2)));
    if (m->counters.cap / sizeof(unsigned int) != old_req)  // fresh buffer: counters start at zero
        NEP_CUDA(cudaMemsetAsync(m->counters.p, 0, m->counters.cap, m->cur));
    NEP_TRY(m->totals.ensure(sizeof(double) * 10 * (size_t)n_req));
    const size_t old_items = m->gcounters.cap;
    NEP_TRY(m->gcounters.ensure(sizeof(unsigned int) * (size_t)n_items));
    if (m->gcounters.cap != old_items) NEP_CUDA(cudaMemsetAsync(m->gcounters.p, 0, m->gcounters.cap, m->cur));
    return NEP_OK;
}

int ensure_lists(nep_model* m, int n)
{
    NEP_TRY(m->nlR.ensure(sizeof(uint32_t) * (size_t)m->mnR * n));
    NEP_TRY(m->nlA.ensure(sizeof(uint32_t) * (size_t)m->mnA * n));
    m->n_lists = n;
    return NEP_OK;
}

int ensure_cells(nep_model* m, int ncell)
{
    // the scan leaves the cell and fill counters zero for the next build; a new
    // buffer starts with anything in it, so the next build clears them first
    const void* c0 = m->cell_count.p;
    const void* f0 = m->cell_fill.p;
    const void* b0 = m->block_off.p;
    NEP_TRY(m->cell_count.ensure(sizeof(int) * ncell));
    NEP_TRY(m->cell_local.ensure(sizeof(int) * ncell));
    NEP_TRY(m->block_off.ensure(sizeof(int) * (kScanItems + 1)));
    NEP_TRY(m->cell_fill.ensure(sizeof(int) * ncell));
    NEP_TRY(m->cell_start.ensure(sizeof(int) * (ncell + 1)));
    if (m->cell_count.p != c0 || m->cell_fill.p != f0 || m->block_off.p != b0) m->cells_dirty = true;
    return NEP_OK;
}

int ensure_plan_workspace(nep_model* m, const Plan& p)
{
    NEP_TRY(ensure_particles(m, p.n_cap, p.items_cap, (int)p.reqs.size(), p.Tmax));
    NEP_TRY(ensure_cells(m, p.ncell_cap));
    if ((size_t)p.n_cap > m->n_lists || !m->nlR.p) NEP_TRY(ensure_lists(m, p.n_cap));
    return NEP_OK;
}

// Estimated neighbour counts from the density of the box (first sizing only).
void initial_capacity(nep_model* m, int n, const double box[3])
{
    if (m->mnR > 0 && m->mnA > 0) return;
    double V = box[0] * box[1] * box[2];
    double rho = n / V;
    double rR = 0, rA = 0;
    for (double v : m->rcR) rR = std::max(rR, v);
    for (double v : m->rcA) rA = std::max(rA, v);
    auto est = [&](double rc) {
        double c = 4.18879 * rc * rc * rc * rho * 1.3 + 16;
        int k = (int)std::min(c, 4096.0);
        return (k + 7) & ~7;
    };
    if (m->mnR <= 0) m->mnR = est(rR);
    if (m->mnA <= 0) m->mnA = est(rA);
}

// ---- pipeline stages ----------------------------------------------------------
template <typename real>
int run_cells(nep_model* m, const Plan& p, const int* types_d, const double* pos_d)
{
    cudaError_t e = launch_cell_build<real>(
        d_counts(p), p.n_cap, p.items_cap, p.ncell_cap, m->cells_dirty, false, d_items(p), d_reqs(p), d_models<real>(p),
        pos_d, types_d, m->cell_of.as<int>(), m->rec_user.as<PosRec<real>>(), m->cell_count.as<int>(),
        m->cell_local.as<int>(), m->block_off.as<int>(), m->cell_fill.as<int>(), m->perm_tmp.as<int>(),
        m->perm.as<int>(), m->cell_start.as<int>(), m->cell_s.as<int>(), m->rec_s.as<PosRec<real>>(),
        m->flags.as<int>() + 2, m->cur);
    if (e != cudaSuccess) {
        m->cells_dirty = true;
        return fail(NEP_ERR_CUDA, std::string("cell build: ") + cudaGetErrorString(e));
    }
    m->cells_dirty = false;
    return NEP_OK;
}

// The MD step's opening (kicks, drift, binning in one kernel) and the rest of the
// cell build.  Counters that may be dirty are cleared before the binning counts.
template <typename real>
int run_kick_drift_cells(nep_model* m, const Plan& p, const int* types_d, const double* inv_m_acc, int n_kicks,
                         double half_dt, double dt, double* pos, double* vel, const double* force,
                         cudaEvent_t* ev = nullptr)
{
    if (m->cells_dirty) {
        NEP_CUDA(cudaMemsetAsync(m->cell_count.p, 0, sizeof(int) * p.ncell_cap, m->cur));
        NEP_CUDA(cudaMemsetAsync(m->cell_fill.p, 0, sizeof(int) * p.ncell_cap, m->cur));
    }
    TypeTable tt;
    for (int k = 0; k < kMdMaxTypes; ++k) tt.v[k] = k < m->T ? inv_m_acc[k] : 0.0;
    cudaError_t e = launch_kick_drift_bin<real>(d_counts(p), p.items_cap, d_items(p), d_reqs(p), d_models<real>(p),
                                                types_d, tt, n_kicks, half_dt, dt, pos, vel, force,
                                                m->cell_of.as<int>(), m->rec_user.as<PosRec<real>>(),
                                                m->cell_count.as<int>(), m->flags.as<int>() + 2, m->cur);
    if (e == cudaSuccess && ev) e = cudaEventRecord(ev[1], m->cur);
    if (e == cudaSuccess)
        e = launch_cell_build<real>(d_counts(p), p.n_cap, p.items_cap, p.ncell_cap, false, true, d_items(p), d_reqs(p),
                                    d_models<real>(p), pos, types_d, m->cell_of.as<int>(),
                                    m->rec_user.as<PosRec<real>>(), m->cell_count.as<int>(), m->cell_local.as<int>(),
                                    m->block_off.as<int>(), m->cell_fill.as<int>(), m->perm_tmp.as<int>(),
                                    m->perm.as<int>(), m->cell_start.as<int>(), m->cell_s.as<int>(),
                                    m->rec_s.as<PosRec<real>>(), m->flags.as<int>() + 2, m->cur);
    if (e != cudaSuccess) {
        m->cells_dirty = true;
        return fail(NEP_ERR_CUDA, std::string("kick/drift + cell build: ") + cudaGetErrorString(e));
    }
    m->cells_dirty = false;
    return NEP_OK;
}

template <typename real>
int run_neighbors(nep_model* m, const Plan& p)
{
    NeighborArgs<real> a;
    a.n = p.n_cap;
    a.mnR = m->mnR;
    a.mnA = m->mnA;
    a.counts = d_counts(p);
    a.items = d_items(p);
    a.reqs = d_reqs(p);
    a.models = d_models<real>(p);
    a.cell_start = m->cell_start.as<int>();
    a.cell_s = m->cell_s.as<int>();
    a.rec = m->rec_s.as<PosRec<real>>();
    a.nlR = m->nlR.as<uint32_t>();
    a.nlA = m->nlA.as<uint32_t>();
    a.cntR = m->cntR.as<int>();
    a.cntA = m->cntA.as<int>();
    a.maxcnt = m->flags.as<int>();
    // the FP32 form's fixed-point lines are zeroed by the neighbour kernel (virial
    // lines only when this evaluation returns per-particle virials)
    a.accF = m->precision != NEP_FP64 ? acc_force(m->acc.p) : nullptr;
    a.accW = m->precision != NEP_FP64 && m->eval_per_bead ? acc_virial(m->acc.p, p.n_cap) : nullptr;
    a.rec32 = m->precision == NEP_FP64 ? m->rec32.as<PosRec<float>>() : nullptr;
    if ((uint64_t)std::max(a.mnR, a.mnA) * (uint64_t)a.n > (1ull << 32))
        return fail(NEP_ERR_ARG, "neighbour lists beyond 2^32 entries (capacity x particles)");
    cudaError_t e = launch_neighbors<real>(a, p.items_cap, p.smem_nbr, m->cur);
    if (e != cudaSuccess) return fail(NEP_ERR_CUDA, std::string("neighbours: ") + cudaGetErrorString(e));
    return NEP_OK;
}

// The MD step's closing half-kick, when the output pass applies it.
struct FusedKick {
    double* vel;
    const int* types;
    const double* inv_m_acc;  // host, [T]
    double half_dt;
};

template <typename real>
int run_evaluate(nep_model* m, const Plan& p, double* force, double* virial, double* site, double* totals,
                 cudaEvent_t mid = nullptr, const FusedKick* kick = nullptr)
{
    EvalArgs<real> a;
    a.n = p.n_cap;
    a.mnR = m->mnR;
    a.mnA = m->mnA;
    a.counts = d_counts(p);
    a.items = d_items(p);
    a.reqs = d_reqs(p);
    a.models = d_models<real>(p);
    a.rec = m->rec_s.as<PosRec<real>>();
    a.nlR = m->nlR.as<uint32_t>();
    a.nlA = m->nlA.as<uint32_t>();
    a.cntR = m->cntR.as<int>();
    a.cntA = m->cntA.as<int>();
    a.U = m->U.as<real>();
    a.e = m->e.as<real>();
    a.e_stride = p.Tmax * m->KRP;
    a.phi = m->phi.as<real>();
    a.net_bf16 = m->precision == NEP_FP32_BF16;
    a.many_body = m->MBT;
    a.perm = m->perm.as<int>();
    a.force = force;
    a.virial = virial;
    a.site = site;
    a.accF = acc_force(m->acc.p);
    a.accW = acc_virial(m->acc.p, p.n_cap);
    a.wsum = acc_wsum(m->acc.p, p.n_cap);
    a.partial = m->partial.as<double>();
    a.counter = m->counters.as<unsigned int>() + 2;
    a.gcounter = m->gcounters.as<unsigned int>();
    a.err = m->flags.as<int>() + 2;
    a.totals = totals;
    if (kick) {
        if (m->T > kMdMaxTypes) return fail(NEP_ERR_ARG, "too many types for MD");
        a.kick_vel = kick->vel;
        a.kick_types = kick->types;
        a.kick_half_dt = kick->half_dt;
        for (int t = 0; t < kMdMaxTypes; ++t) a.kick_im.v[t] = t < m->T ? kick->inv_m_acc[t] : 0.0;
    }
    cudaError_t e = launch_evaluate<real>(m->nR, m->nA, m->KR, m->KA, a, p.items_cap, p.smem_desc,
                                          p.smem_force, m->cur, mid, m->mb_desc, m->mb_force, m->ch_force);
    if (e != cudaSuccess) return fail(NEP_ERR_CUDA, std::string("evaluate: ") + cudaGetErrorString(e));
    return NEP_OK;
}

// The error word's bits (see kErrCellList) as a status.
int status_error(int word)
{
    if (word & 1) return fail(NEP_ERR_ARG, "non-finite position");
    if (word & 2) return fail(NEP_ERR_ARG, "particle type out of range");
    if (word & kErrCellList) return fail(NEP_ERR_CUDA, "internal error: inconsistent cell list (access skipped)");
    return NEP_OK;
}

template <typename real>
int check_lists(nep_model* m, const Plan& p)
{
    // read maxcnt and the error word; grow and rebuild on overflow
    for (int attempt = 0; attempt < 3; ++attempt) {
        NEP_CUDA(cudaMemcpyAsync(m->h_flags, m->flags.p, 3 * sizeof(int), cudaMemcpyDeviceToHost, m->cur));
        NEP_CUDA(cudaStreamSynchronize(m->cur));
        NEP_TRY(status_error(m->h_flags[2]));
        int needR = m->h_flags[0], needA = m->h_flags[1];
        if (needR <= m->mnR && needA <= m->mnA) return NEP_OK;
        if (needR > m->mnR) m->mnR = ((int)(needR * 1.25) + 8 + 7) & ~7;
        if (needA > m->mnA) m->mnA = ((int)(needA * 1.25) + 8 + 7) & ~7;
        NEP_TRY(ensure_lists(m, p.n_cap));
        NEP_CUDA(cudaMemsetAsync(m->flags.p, 0, 2 * sizeof(int), m->cur));
        NEP_TRY(run_neighbors<real>(m, p));
    }
    return fail(NEP_ERR_NEIGHBOR_OVERFLOW, "neighbour capacity did not converge");
}

// Full evaluation of the uploaded plan on device arrays, with a synchronous check of
// the list sizes before the evaluation (used where the call synchronises anyway).
// force must be non-null.
template <typename real>
int evaluate_plan(nep_model* m, const Plan& p, const int* types_d, const double* pos_d, double* force,
                  double* virial, double* site, double* totals)
{
    NEP_TRY(ensure_plan_workspace(m, p));
    m->eval_per_bead = virial != nullptr;
    NEP_CUDA(cudaMemsetAsync(m->flags.p, 0, 3 * sizeof(int), m->cur));
    NEP_TRY(run_cells<real>(m, p, types_d, pos_d));
    NEP_TRY(run_neighbors<real>(m, p));
    NEP_TRY(check_lists<real>(m, p));
    NEP_TRY(run_evaluate<real>(m, p, force, virial, site, totals));
    return NEP_OK;
}

// The evaluation pipeline of the uploaded plan with no host synchronisation: status
// words cleared, cell build, neighbour lists, descriptor + forces.  List overflow
// and bad inputs are read afterwards from the status words (eval_status).
template <typename real>
int eval_pipeline(nep_model* m, const Plan& p, const int* types_d, const double* pos_d, double* force,
                  double* virial, double* site, double* totals)
{
    NEP_CUDA(cudaMemsetAsync(m->flags.p, 0, 3 * sizeof(int), m->cur));
    NEP_TRY(run_cells<real>(m, p, types_d, pos_d));
    NEP_TRY(run_neighbors<real>(m, p));
    NEP_TRY(run_evaluate<real>(m, p, force, virial, site, totals));
    return NEP_OK;
}

// The device addresses of every workspace buffer a pipeline launch bakes in: part
// of every graph key, so a graph is never replayed after a buffer moved.
void put_workspace_ptrs(std::vector<unsigned char>& key, const nep_model* m)
{
    const Buf* bufs[] = {&m->cell_of, &m->rec_user, &m->perm_tmp, &m->perm, &m->rec_s, &m->cell_s, &m->cntR,
                         &m->cntA, &m->nlR, &m->nlA, &m->U, &m->e, &m->phi, &m->rec32, &m->cell_count, &m->cell_local,
                         &m->block_off, &m->cell_fill, &m->cell_start, &m->partial, &m->partial2, &m->counters,
                         &m->gcounters, &m->totals, &m->flags, &m->thermo, &m->sample_index, &m->acc, &m->bussi,
                         &m->md_virial, &m->md_site, &m->heat, &m->heat_rows};
    for (const Buf* b : bufs) {
        const unsigned char* q = (const unsigned char*)&b->p;
        key.insert(key.end(), q, q + sizeof(void*));
    }
}

// Everything a captured evaluation graph bakes in: launch shapes, shared-memory
// sizes, kernel variants, list capacities and every device pointer.
template <typename real>
std::vector<unsigned char> eval_graph_key(const nep_model* m, const Plan& p, const void* const* io, int n_io)
{
    std::vector<unsigned char> key;
    auto put = [&](const void* q, size_t sz) {
        const unsigned char* b = (const unsigned char*)q;
        key.insert(key.end(), b, b + sz);
    };
    const int ints[] = {p.n_cap, p.items_cap, p.ncell_cap, p.Tmax, m->mnR, m->mnA, m->mb_desc, m->mb_force, m->ch_force,
                        m->eval_per_bead ? 1 : 0, m->precision, m->MBT, (int)sizeof(real)};
    put(ints, sizeof ints);
    const size_t sm[] = {p.smem_desc, p.smem_force, p.smem_nbr, p.off_reqs, p.off_items, p.off_models};
    put(sm, sizeof sm);
    put_workspace_ptrs(key, m);
    put(&p.dev.p, sizeof(void*));
    put(io, sizeof(void*) * n_io);
    return key;
}

// The evaluation pipeline, replayed from a captured CUDA graph when one matches
// (cached on the handle, a few at a time).  Batches are planned with rounded
// capacities and the kernels read the actual sizes from the device, so batches of
// similar size share one graph.  A build whose cell counters may be dirty runs
// eagerly (it clears them first).
template <typename real>
int eval_launch(nep_model* m, const Plan& p, const int* types_d, const double* pos_d, double* force,
                double* virial, double* site, double* totals)
{
    NEP_TRY(ensure_plan_workspace(m, p));
    m->eval_per_bead = virial != nullptr;
    if (m->cells_dirty) return eval_pipeline<real>(m, p, types_d, pos_d, force, virial, site, totals);
    const void* io[] = {types_d, pos_d, force, virial, site, totals};
    std::vector<unsigned char> key = eval_graph_key<real>(m, p, io, 6);
    for (size_t k = 0; k < m->eval_graphs.size(); ++k)
        if (m->eval_graphs[k].key == key) {
            NEP_CUDA(cudaGraphLaunch(m->eval_graphs[k].exec, m->cur));
            return NEP_OK;
        }
    // a shape seen for the first time runs eagerly (capturing and instantiating a
    // graph costs more than launching its nodes once); the second time it is
    // captured, and replayed from then on
    const size_t h = std::hash<std::string>()(std::string(key.begin(), key.end()));
    if (std::find(m->eval_seen.begin(), m->eval_seen.end(), h) == m->eval_seen.end()) {
        m->eval_seen.push_back(h);
        if (m->eval_seen.size() > 4 * kEvalGraphs) m->eval_seen.erase(m->eval_seen.begin());
        return eval_pipeline<real>(m, p, types_d, pos_d, force, virial, site, totals);
    }
    NEP_CUDA(cudaStreamBeginCapture(m->cur, cudaStreamCaptureModeThreadLocal));
    const int rc = eval_pipeline<real>(m, p, types_d, pos_d, force, virial, site, totals);
    cudaGraph_t graph = nullptr;
    cudaError_t ec = cudaStreamEndCapture(m->cur, &graph);
    if (rc != NEP_OK) {
        if (graph) cudaGraphDestroy(graph);
        m->cells_dirty = true;
        return rc;
    }
    if (ec != cudaSuccess) return fail(NEP_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(ec));
    GraphCache gc;
    ec = cudaGraphInstantiate(&gc.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ec != cudaSuccess) return fail(NEP_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(ec));
    gc.key = key;
    if (m->eval_graphs.size() >= kEvalGraphs) {  // drop the oldest
        m->eval_graphs.front().reset();
        m->eval_graphs.erase(m->eval_graphs.begin());
    }
    m->eval_graphs.push_back(gc);
    NEP_CUDA(cudaGraphLaunch(m->eval_graphs.back().exec, m->cur));
    return NEP_OK;
}

// Deferred status of an evaluation, read from h_flags after the call synchronised:
// a bad input fails the call; lists that outgrew their capacity are grown and the
// caller runs the evaluation again (retry = true).
int eval_status(nep_model* m, bool& retry)
{
    retry = false;
    NEP_TRY(status_error(m->h_flags[2]));
    const int needR = m->h_flags[0], needA = m->h_flags[1];
    if (needR <= m->mnR && needA <= m->mnA) return NEP_OK;
    if (needR > m->mnR) m->mnR = ((int)(needR * 1.25) + 8 + 7) & ~7;
    if (needA > m->mnA) m->mnA = ((int)(needA * 1.25) + 8 + 7) & ~7;
    m->n_lists = 0;  // reallocate at the new capacity
    retry = true;
    return NEP_OK;
}

int validate_common(nep_model* m, int n, const void* types, const void* pos, const double* box, const int32_t* pbc,
                    int mem)
{
    if (!m) return fail(NEP_ERR_ARG, "null model");
    if (n < 1 || n > kMaxN) return fail(NEP_ERR_ARG, "n out of range [1, 2^23)");
    if (!types || !pos || !box || !pbc) return fail(NEP_ERR_ARG, "null input array");
    if (mem != NEP_HOST && mem != NEP_DEVICE) return fail(NEP_ERR_ARG, "mem must be NEP_HOST or NEP_DEVICE");
    return NEP_OK;
}

// Work runs on the caller's stream; a NULL stream (the legacy default stream, which
// cannot be captured into a graph) is replaced by the handle's internal stream,
// ordered after the legacy stream on entry and before it on exit.
int enter(nep_model* m, void* stream)
{
    if (stream) {
        m->cur = (cudaStream_t)stream;
        return NEP_OK;
    }
    m->cur = m->st;
    NEP_CUDA(cudaEventRecord(m->ev_in, (cudaStream_t)0));
    NEP_CUDA(cudaStreamWaitEvent(m->st, m->ev_in, 0));
    return NEP_OK;
}

int leave(nep_model* m, void* stream, bool sync = true)
{
    if (!stream) {
        NEP_CUDA(cudaEventRecord(m->ev_out, m->st));
        NEP_CUDA(cudaStreamWaitEvent((cudaStream_t)0, m->ev_out, 0));
    }
    if (sync) NEP_CUDA(cudaStreamSynchronize(m->cur));
    return NEP_OK;
}

int ensure_host_totals(nep_model* m, size_t count)
{
    if (count <= m->h_totals_cap) return NEP_OK;
    if (m->h_totals) cudaFreeHost(m->h_totals);
    m->h_totals = nullptr;
    m->h_totals_cap = 0;
    NEP_CUDA(cudaMallocHost((void**)&m->h_totals, sizeof(double) * count));
    m->h_totals_cap = count;
    return NEP_OK;
}

template <typename real>
int compute_impl(nep_model* m, int n, const int32_t* types, const double* pos, const double box[3],
                 const int32_t pbc[3], int mem, void* stream, double* energy_total, double* virial_total,
                 double* site_energy, double* force, double* virial)
{
    CellGrid g;
    NEP_TRY(make_grid(m, box, pbc, g));
    NEP_TRY(enter(m, stream));
    initial_capacity(m, n, box);
    NEP_TRY(single_plan<real>(m, n, g));
    NEP_TRY(ensure_plan_workspace(m, m->plan));
    const int* types_d = types;
    const double* pos_d = pos;
    double *force_d = force, *virial_d = virial, *site_d = site_energy;
    if (mem == NEP_HOST) {
        NEP_TRY(m->types_d.ensure(sizeof(int) * n));
        NEP_TRY(m->pos_d.ensure(sizeof(double) * 3 * (size_t)n));
        NEP_CUDA(cudaMemcpyAsync(m->types_d.p, types, sizeof(int) * n, cudaMemcpyHostToDevice, m->cur));
        NEP_CUDA(cudaMemcpyAsync(m->pos_d.p, pos, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, m->cur));
        types_d = m->types_d.as<int>();
        pos_d = m->pos_d.as<double>();
        NEP_TRY(m->force_d.ensure(sizeof(double) * 3 * (size_t)n));
        force_d = m->force_d.as<double>();
        virial_d = nullptr;
        site_d = nullptr;
        if (virial) {
            NEP_TRY(m->virial_d.ensure(sizeof(double) * 9 * (size_t)n));
            virial_d = m->virial_d.as<double>();
        }
        if (site_energy) {
            NEP_TRY(m->site_d.ensure(sizeof(double) * (size_t)n));
            site_d = m->site_d.as<double>();
        }
    } else if (!force_d) {
        force_d = m->force_tmp.as<double>();
    }
    double* totals = m->totals.as<double>();
    NEP_TRY(ensure_host_totals(m, 10));
    // one synchronisation per call: the evaluation, its outputs and its status words
    // are enqueued together; lists that overflowed are grown and the call runs again
    for (int attempt = 0;; ++attempt) {
        NEP_TRY(eval_launch<real>(m, m->plan, types_d, pos_d, force_d, virial_d, site_d, totals));
        if (mem == NEP_HOST) {
            if (force) NEP_CUDA(cudaMemcpyAsync(force, force_d, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, m->cur));
            if (virial)
                NEP_CUDA(cudaMemcpyAsync(virial, virial_d, sizeof(double) * 9 * n, cudaMemcpyDeviceToHost, m->cur));
            if (site_energy)
                NEP_CUDA(cudaMemcpyAsync(site_energy, site_d, sizeof(double) * n, cudaMemcpyDeviceToHost, m->cur));
            NEP_CUDA(cudaMemcpyAsync(m->h_totals, totals, sizeof(double) * 10, cudaMemcpyDeviceToHost, m->cur));
        } else {
            if (energy_total)
                NEP_CUDA(cudaMemcpyAsync(energy_total, totals, sizeof(double), cudaMemcpyDeviceToDevice, m->cur));
            if (virial_total)
                NEP_CUDA(cudaMemcpyAsync(virial_total, totals + 1, sizeof(double) * 9, cudaMemcpyDeviceToDevice,
                                         m->cur));
        }
        NEP_CUDA(cudaMemcpyAsync(m->h_flags, m->flags.p, 3 * sizeof(int), cudaMemcpyDeviceToHost, m->cur));
        NEP_TRY(leave(m, stream));
        bool retry = false;
        NEP_TRY(eval_status(m, retry));
        if (!retry) break;
        if (attempt == 2) return fail(NEP_ERR_NEIGHBOR_OVERFLOW, "neighbour capacity did not converge");
        NEP_TRY(enter(m, stream));
    }
    if (mem == NEP_HOST) {
        if (energy_total) *energy_total = m->h_totals[0];
        if (virial_total)
            for (int k = 0; k < 9; ++k) virial_total[k] = m->h_totals[1 + k];
    }
    return NEP_OK;
}

// Timing events of one autotuning pass, destroyed on every exit path.
struct TuneEvents {
    cudaEvent_t e[3] = {nullptr, nullptr, nullptr};
    ~TuneEvents()
    {
        for (cudaEvent_t x : e)
            if (x) cudaEventDestroy(x);
    }
};

// Autotuner: time the register-cap variants of the two evaluation kernels on the
// plan's configuration (lists already built) and keep the fastest of each.  An
// event between the two launches times each kernel on its own, so the descriptor
// and force variants are chosen independently; every variant runs in each of
// several interleaved rounds and keeps its minimum, which steadies choices between
// variants a few percent apart.  More resident blocks hide more latency but leave
// fewer registers per thread; which wins depends on the configuration (the
// 4-block force variant wins with few pairs per particle or several types).  The
// variants compute the same arithmetic, so the choice does not change results.
template <typename real>
int autotune_plan(nep_model* m, const Plan& p, double* force_d)
{
    if (m->precision == NEP_FP64) return NEP_OK;  // one FP64 variant only
    TuneEvents ev;
    for (cudaEvent_t& x : ev.e) NEP_CUDA(cudaEventCreate(&x));
    cudaEvent_t e0 = ev.e[0], em = ev.e[1], e1 = ev.e[2];
    // variants: the descriptor kernel at 2 or 3 blocks per SM; the radial kernel at
    // 3, 4 or 5 blocks per SM, each with walk groups of 4 or 8 neighbour entries.
    // Each trial runs one descriptor and one radial variant; every radial variant
    // appears once per round and each descriptor variant three times.
    struct Trial {
        int md, mf, ch;
    };
    const Trial trials[6] = {{2, 3, 4}, {3, 3, 8}, {2, 4, 4}, {3, 4, 8}, {2, 5, 4}, {3, 5, 8}};
    const Trial trials2[6] = {{3, 3, 4}, {2, 3, 8}, {3, 4, 4}, {2, 4, 8}, {3, 5, 4}, {2, 5, 8}};
    float best_d[4] = {1e30f, 1e30f, 1e30f, 1e30f};  // by blocks per SM
    float best_f[6][9];                              // [blocks per SM][chunk]
    for (auto& r : best_f)
        for (float& x : r) x = 1e30f;
    const int keep_d = m->mb_desc, keep_f = m->mb_force, keep_c = m->ch_force;
    auto trial = [&](const Trial& t, bool timed) -> int {
        m->mb_desc = t.md;
        m->mb_force = t.mf;
        m->ch_force = t.ch;
        NEP_CUDA(cudaEventRecord(e0, m->cur));
        NEP_TRY(run_evaluate<real>(m, p, force_d, nullptr, nullptr, m->totals.as<double>(), em));
        NEP_CUDA(cudaEventRecord(e1, m->cur));
        NEP_CUDA(cudaEventSynchronize(e1));
        if (!timed) return NEP_OK;
        float td = 0.f, tf = 0.f;
        NEP_CUDA(cudaEventElapsedTime(&td, e0, em));
        NEP_CUDA(cudaEventElapsedTime(&tf, em, e1));
        best_d[t.md] = std::min(best_d[t.md], td);
        best_f[t.mf][t.ch] = std::min(best_f[t.mf][t.ch], tf);
        return NEP_OK;
    };
    int rc = NEP_OK;
    for (int round = -1; round < 4 && rc == NEP_OK; ++round)  // round -1 warms up
        for (int c = 0; c < 6 && rc == NEP_OK; ++c) rc = trial((round & 1) ? trials2[c] : trials[c], round >= 0);
    m->mb_desc = keep_d;
    m->mb_force = keep_f;
    m->ch_force = keep_c;
    if (rc != NEP_OK) return rc;
    // leave the default (3 blocks, groups of 4) only for a clear win: timed back to
    // back in isolation the variants can rank a few percent differently than inside
    // an MD step (measured on 100k-bead water: 4 blocks won here by up to 3-4% and
    // lost 1-2% in the step; where 4 blocks win in the step they win by 7-12%)
    const float margin = 0.95f;
    m->mb_desc = best_d[2] < margin * best_d[3] ? 2 : 3;
    int bf = 3, bc = 4;
    for (int v = 3; v <= 5; ++v)
        for (int c = 4; c <= 8; c += 4)
            if (best_f[v][c] < margin * best_f[3][4] && best_f[v][c] < best_f[bf][bc]) {
                bf = v;
                bc = c;
            }
    m->mb_force = bf;
    m->ch_force = bc;
    return NEP_OK;
}

// Stochastic-velocity-rescaling thermostat of an MD call (inactive when noise is null).
struct Thermostat {
    const double* noise = nullptr;  // device [n_steps][2]
    double c = 1.0, kbar = 0.0, n_f = 1.0;
};

// HNEMD driving force and heat-current sampling of an MD call (inactive when on == 0).
struct Drive {
    int on = 0;
    double fe[3] = {0.0, 0.0, 0.0};
    double* virial = nullptr;  // device [9][n] per-particle virial of the step
    double* site = nullptr;    // device [n] site energies of the step
    double* acc = nullptr;     // device [6] interval sums; followed by the block counter
    double* rows = nullptr;    // device [samples][6] interval averages
};

// The force evaluation of an MD step, with the driving force added when it is on.
template <typename real>
int md_forces(nep_model* m, const Plan& p, int n, double* force, const Drive& dr, cudaEvent_t mid = nullptr,
              const FusedKick* kick = nullptr)
{
    if (kick && dr.on) return fail(NEP_ERR_ARG, "the driving force precedes the closing kick");
    NEP_TRY(run_evaluate<real>(m, p, force, dr.on ? dr.virial : nullptr, dr.on ? dr.site : nullptr,
                               m->totals.as<double>(), mid, kick));
    if (dr.on) {
        cudaError_t e = launch_hnemd_force(n, dr.fe, dr.virial, m->totals.as<double>(), force, m->cur);
        if (e != cudaSuccess) return fail(NEP_ERR_CUDA, std::string("driving force: ") + cudaGetErrorString(e));
    }
    return NEP_OK;
}

// One MD step's launches (used eagerly and under stream capture).
template <typename real>
// n_kicks: the opening half-kicks (2 when the previous step's closing kick was
// deferred into this step's opening); close: emit this step's closing kick (a step
// defers it only when nothing before the next step's opening reads the velocities:
// no thermo row, thermostat or heat current, and not the last step of the call).
// Kicks are separately rounded either way, so deferral changes no result.
int md_step_launches(nep_model* m, int n, const int* types_d, const double* inv_m_acc, const double* mass,
                     const CellGrid& g, double* pos, double* vel, double* force, double dt, bool sample,
                     int step_stride, const Thermostat& th, const Drive& dr, int n_kicks, bool close)
{
    const Plan& p = m->plan;
    cudaEvent_t* ev = nullptr;
    if (m->timer.on) {
        const int r = m->timer.head;
        m->timer.collect(r);  // reuse of a ring slot waits for its previous step
        ev = m->timer.ev[r];
        m->timer.pending[r] = true;
        m->timer.head = (r + 1) % StageTimer::kRing;
        NEP_CUDA(cudaEventRecord(ev[0], m->cur));
    }
    (void)g;  // the kernels take the grid from the plan's request table
    if (!close && (sample || th.noise || dr.on)) return fail(NEP_ERR_ARG, "closing kick cannot be deferred here");
    // stage 0: kicks + drift + binning; stage 1: the rest of the cell build
    NEP_TRY(run_kick_drift_cells<real>(m, p, types_d, inv_m_acc, n_kicks, 0.5 * dt, dt, pos, vel, force, ev));
    if (ev) NEP_CUDA(cudaEventRecord(ev[2], m->cur));
    NEP_TRY(run_neighbors<real>(m, p));
    if (ev) NEP_CUDA(cudaEventRecord(ev[3], m->cur));
    // the closing kick rides on the output pass unless the driving force still has
    // to be added to the forces
    const bool fuse_kick = close && !dr.on;
    const FusedKick kick = {vel, types_d, inv_m_acc, 0.5 * dt};
    NEP_TRY(md_forces<real>(m, p, n, force, dr, ev ? ev[4] : nullptr, fuse_kick ? &kick : nullptr));
    if (ev) NEP_CUDA(cudaEventRecord(ev[5], m->cur));
    cudaError_t e = cudaSuccess;
    if (close && !fuse_kick) {
        e = launch_kick(n, types_d, inv_m_acc, m->T, 0.5 * dt, vel, force, m->cur);
        if (e != cudaSuccess) return fail(NEP_ERR_CUDA, std::string("kick: ") + cudaGetErrorString(e));
    }
    if (th.noise) {
        e = launch_bussi(n, types_d, mass, m->T, vel, m->partial2.as<double>(), m->counters.as<unsigned int>(),
                         th.noise, m->bussi.as<int>(), th.c, th.kbar, th.n_f, m->bussi.as<double>() + 1, m->cur);
        if (e != cudaSuccess) return fail(NEP_ERR_CUDA, std::string("thermostat: ") + cudaGetErrorString(e));
    }
    if (dr.on) {
        e = launch_heat(n, types_d, mass, m->T, vel, dr.site, dr.virial, m->partial2.as<double>(),
                        reinterpret_cast<unsigned int*>(dr.acc + 6), dr.acc, dr.rows, m->sample_index.as<int>(),
                        sample ? 1 : 0, step_stride, m->cur);
        if (e != cudaSuccess) return fail(NEP_ERR_CUDA, std::string("heat current: ") + cudaGetErrorString(e));
    }
    if (sample) {
        e = launch_sample(n, types_d, mass, m->T, vel, m->totals.as<double>(), m->partial2.as<double>(),
                          m->counters.as<unsigned int>() + 1, m->thermo.as<double>(), m->sample_index.as<int>(),
                          step_stride, m->cur);
        if (e != cudaSuccess) return fail(NEP_ERR_CUDA, std::string("sample: ") + cudaGetErrorString(e));
    }
    if (ev) NEP_CUDA(cudaEventRecord(ev[6], m->cur));
    return NEP_OK;
}

// Deferred status of asynchronous MD calls: maxima of the neighbour counts and the
// error word accumulate on the device; after each asynchronous call they are copied
// to pinned memory and inspected at the next call (or by nep_sync).
int inspect_async(nep_model* m, bool wait)
{
    if (!m->async_pending) return NEP_OK;
    if (wait) {
        NEP_CUDA(cudaEventSynchronize(m->ev_flags));
    } else if (cudaEventQuery(m->ev_flags) != cudaSuccess) {
        (void)cudaGetLastError();  // cudaErrorNotReady is not an error
        return NEP_OK;
    }
    m->async_pending = false;
    const int needR = m->h_async[0], needA = m->h_async[1], err = m->h_async[2];
    bool grow_now = needR * 5 > m->mnR * 4 || needA * 5 > m->mnA * 4;
    if (err || grow_now) {
        // a later call on this stream runs after the current work; reset the words there
        NEP_CUDA(cudaMemsetAsync(m->flags.p, 0, 3 * sizeof(int), m->async_stream));
    }
    if (err & kErrCellList) return status_error(err);
    if (err) return fail(NEP_ERR_ARG, "non-finite position or bad type during MD");
    if (grow_now) {
        const bool overflow = needR > m->mnR || needA > m->mnA;
        m->mnR = std::max(m->mnR, ((int)(needR * 1.5) + 8 + 7) & ~7);
        m->mnA = std::max(m->mnA, ((int)(needA * 1.5) + 8 + 7) & ~7);
        m->n_lists = 0;
        m->graph.reset();
        if (overflow) return fail(NEP_ERR_NEIGHBOR_OVERFLOW, "a neighbour list outgrew its capacity during MD");
    }
    return NEP_OK;
}

template <typename real>
int md_impl(nep_model* m, int n, const int32_t* types, const double* masses, const double box[3],
            const int32_t pbc[3], double* pos, double* vel, double* force, int forces_valid, int n_steps,
            double dt, int sample_every, double* thermo, int mem, void* stream, double temp_K = 0.0,
            double tau_fs = 0.0, const double* noise = nullptr, const double* fe = nullptr, double* heat = nullptr)
{
    CellGrid g;
    NEP_TRY(make_grid(m, box, pbc, g));
    if (n_steps < 0) return fail(NEP_ERR_ARG, "n_steps < 0");
    if (sample_every < 0) return fail(NEP_ERR_ARG, "sample_every < 0");
    if (sample_every > 0 && !thermo) return fail(NEP_ERR_ARG, "thermo is NULL");
    if (!masses || !vel || !force) return fail(NEP_ERR_ARG, "null masses, velocity or force");
    std::vector<double> inv_m(m->T), mass(m->T);
    for (int t = 0; t < m->T; ++t) {
        if (!(masses[t] > 0.0)) return fail(NEP_ERR_ARG, "masses must be positive");
        inv_m[t] = kAcc / masses[t];
        mass[t] = masses[t];
    }
    NEP_TRY(inspect_async(m, false));
    NEP_TRY(enter(m, stream));
    const bool async = (mem == NEP_DEVICE && stream != nullptr);
    initial_capacity(m, n, box);
    NEP_TRY(single_plan<real>(m, n, g));
    const Plan& p = m->plan;
    const int* types_d = types;
    double *pos_d = pos, *vel_d = vel, *force_d = force;
    if (mem == NEP_HOST) {
        NEP_TRY(m->types_d.ensure(sizeof(int) * n));
        NEP_TRY(m->pos_d.ensure(sizeof(double) * 3 * (size_t)n));
        NEP_TRY(m->vel_d.ensure(sizeof(double) * 3 * (size_t)n));
        NEP_TRY(m->force_d.ensure(sizeof(double) * 3 * (size_t)n));
        NEP_CUDA(cudaMemcpyAsync(m->types_d.p, types, sizeof(int) * n, cudaMemcpyHostToDevice, m->cur));
        NEP_CUDA(cudaMemcpyAsync(m->pos_d.p, pos, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, m->cur));
        NEP_CUDA(cudaMemcpyAsync(m->vel_d.p, vel, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, m->cur));
        if (forces_valid)
            NEP_CUDA(cudaMemcpyAsync(m->force_d.p, force, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, m->cur));
        types_d = m->types_d.as<int>();
        pos_d = m->pos_d.as<double>();
        vel_d = m->vel_d.as<double>();
        force_d = m->force_d.as<double>();
    }
    NEP_TRY(ensure_plan_workspace(m, p));
    const int n_samples = sample_every > 0 ? n_steps / sample_every : 0;
    Drive dr;
    if (fe) {
        NEP_TRY(m->md_virial.ensure(sizeof(double) * 9 * (size_t)n));
        NEP_TRY(m->md_site.ensure(sizeof(double) * (size_t)n));
        NEP_TRY(m->heat.ensure(sizeof(double) * 8));
        NEP_TRY(m->heat_rows.ensure(sizeof(double) * 6 * std::max(1, n_samples)));
        NEP_CUDA(cudaMemsetAsync(m->heat.p, 0, sizeof(double) * 8, m->cur));  // sums and counter
        dr.on = 1;
        for (int a = 0; a < 3; ++a) dr.fe[a] = fe[a];
        dr.virial = m->md_virial.as<double>();
        dr.site = m->md_site.as<double>();
        dr.acc = m->heat.as<double>();
        dr.rows = m->heat_rows.as<double>();
    }
    m->eval_per_bead = dr.on != 0;

    // Size the neighbour lists (one synchronous probe, and the autotuner) only for a
    // new configuration shape: particle count, cells per axis, search ranges and
    // periodicity.  A box that changes within those (a strain schedule rescaling it
    // by 0.1%) keeps the lists' capacities and the tuned variants; the step graph,
    // whose key holds the whole grid, is captured again.  Continuation calls rely
    // on the deferred status.
    const bool new_shape = (n != m->md_n) || memcmp(g.nc, m->md_grid.nc, sizeof g.nc) != 0 ||
                           memcmp(g.S, m->md_grid.S, sizeof g.S) != 0 || memcmp(g.pbc, m->md_grid.pbc, sizeof g.pbc) != 0;
    if (new_shape || !forces_valid) {
        NEP_CUDA(cudaMemsetAsync(m->flags.p, 0, 3 * sizeof(int), m->cur));
        NEP_TRY(run_cells<real>(m, p, types_d, pos_d));
        NEP_TRY(run_neighbors<real>(m, p));
        if (new_shape) {
            NEP_TRY(check_lists<real>(m, p));
            const int wantR = ((int)(m->h_flags[0] * 1.5) + 8 + 7) & ~7;
            const int wantA = ((int)(m->h_flags[1] * 1.5) + 8 + 7) & ~7;
            if (wantR > m->mnR || wantA > m->mnA) {
                m->mnR = std::max(m->mnR, wantR);
                m->mnA = std::max(m->mnA, wantA);
                NEP_TRY(ensure_lists(m, n));
                NEP_TRY(run_neighbors<real>(m, p));
            }
            m->md_n = n;
            m->md_grid = g;
            if (m->autotune) NEP_TRY(autotune_plan<real>(m, p, m->force_tmp.as<double>()));
            NEP_CUDA(cudaMemsetAsync(m->flags.p, 0, 3 * sizeof(int), m->cur));
        }
        if (!forces_valid) NEP_TRY(md_forces<real>(m, p, n, force_d, dr));
    }
    m->eval_per_bead = dr.on != 0;
    Thermostat th;
    if (noise) {
        NEP_TRY(m->noise_d.ensure(sizeof(double) * 2 * std::max(1, n_steps)));
        NEP_TRY(m->bussi.ensure(sizeof(double) * 2));
        if (n_steps > 0)
            NEP_CUDA(cudaMemcpyAsync(m->noise_d.p, noise, sizeof(double) * 2 * n_steps, cudaMemcpyHostToDevice,
                                     m->cur));
        NEP_CUDA(cudaMemsetAsync(m->bussi.p, 0, sizeof(int), m->cur));  // step index of the call
        th.noise = m->noise_d.as<double>();
        th.c = exp(-dt / tau_fs);
        th.n_f = 3.0 * n - 3.0;
        th.kbar = 0.5 * th.n_f * 8.617333262e-5 * temp_K;
    }
    NEP_TRY(m->thermo.ensure(sizeof(double) * 12 * std::max(1, n_samples)));
    NEP_TRY(m->sample_index.ensure(sizeof(int)));
    if (n_samples > 0) NEP_CUDA(cudaMemsetAsync(m->sample_index.p, 0, sizeof(int), m->cur));

    // the steps run in chunks; one chunk is captured once as a CUDA graph (cached
    // by its arguments) and replayed.  After each chunk the status words are
    // copied to pinned memory and inspected one chunk later (so the GPU never
    // waits for the host); counts above 80% of capacity grow the lists and the
    // graph is captured again before the next chunk.
    const int chunk = sample_every > 0 ? sample_every : std::max(1, std::min(n_steps, 50));
    int done = 0;
    auto capture = [&]() -> int {
        std::vector<unsigned char> key;
        auto put = [&](const void* q, size_t sz) {
            const unsigned char* b = (const unsigned char*)q;
            key.insert(key.end(), b, b + sz);
        };
        const void* ptrs[] = {types_d, pos_d, vel_d, force_d, m->cur, p.dev.p};
        put(ptrs, sizeof ptrs);
        put_workspace_ptrs(key, m);
        put(&n, sizeof n);
        put(&g, sizeof g);
        put(&dt, sizeof dt);
        put(&chunk, sizeof chunk);
        put(&sample_every, sizeof sample_every);
        put(&m->mnR, sizeof m->mnR);
        put(&m->mnA, sizeof m->mnA);
        put(inv_m.data(), sizeof(double) * m->T);
        put(&th, sizeof th);
        put(&m->mb_desc, sizeof m->mb_desc);
        put(&m->mb_force, sizeof m->mb_force);
        put(&m->ch_force, sizeof m->ch_force);
        const size_t offs[] = {p.off_reqs, p.off_items, p.off_models};
        put(offs, sizeof offs);
        const void* tptr[] = {m->bussi.p, dr.virial, dr.site, dr.acc, dr.rows};
        put(tptr, sizeof tptr);
        put(&dr.on, sizeof dr.on);
        put(dr.fe, sizeof dr.fe);
        if (m->graph.exec && m->graph.key == key) return NEP_OK;
        m->graph.reset();
        NEP_CUDA(cudaStreamBeginCapture(m->cur, cudaStreamCaptureModeThreadLocal));
        int rc = NEP_OK;
        bool prev_close = true;
        for (int s = 0; s < chunk && rc == NEP_OK; ++s) {
            const bool smp = sample_every > 0 && s == chunk - 1;
            const bool close = s == chunk - 1 || smp || th.noise || dr.on;
            rc = md_step_launches<real>(m, n, types_d, inv_m.data(), mass.data(), g, pos_d, vel_d, force_d, dt, smp,
                                        sample_every, th, dr, prev_close ? 1 : 2, close);
            prev_close = close;
        }
        cudaGraph_t graph = nullptr;
        cudaError_t ec = cudaStreamEndCapture(m->cur, &graph);
        if (rc != NEP_OK) {
            if (graph) cudaGraphDestroy(graph);
            return rc;
        }
        if (ec != cudaSuccess) return fail(NEP_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(ec));
        ec = cudaGraphInstantiate(&m->graph.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ec != cudaSuccess) return fail(NEP_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(ec));
        m->graph.key = key;
        return NEP_OK;
    };
    if (n_steps >= chunk && !m->timer.on) {  // stage timing runs the steps eagerly
        NEP_TRY(capture());
        const bool check = n_steps >= 2 * chunk;
        bool pending = false;
        int prevR = -1, prevA = -1;  // the counts' running maxima one chunk earlier
        for (; done + chunk <= n_steps; done += chunk) {
            NEP_CUDA(cudaGraphLaunch(m->graph.exec, m->cur));
            if (!check) continue;
            if (pending) {  // the previous chunk's status
                NEP_CUDA(cudaEventSynchronize(m->ev_flags));
                const int needR = m->h_async[0], needA = m->h_async[1];
                if (m->h_async[2]) {
                    NEP_CUDA(cudaStreamSynchronize(m->cur));
                    if (m->h_async[2] & kErrCellList) return status_error(m->h_async[2]);
                    return fail(NEP_ERR_ARG, "non-finite position or bad type during MD");
                }
                if (needR > m->mnR || needA > m->mnA) {
                    NEP_CUDA(cudaStreamSynchronize(m->cur));
                    NEP_CUDA(cudaMemsetAsync(m->flags.p, 0, 3 * sizeof(int), m->cur));
                    m->mnR = std::max(m->mnR, ((int)(needR * 1.5) + 8 + 7) & ~7);
                    m->mnA = std::max(m->mnA, ((int)(needA * 1.5) + 8 + 7) & ~7);
                    m->n_lists = 0;
                    m->graph.reset();
                    return fail(NEP_ERR_NEIGHBOR_OVERFLOW, "a neighbour list outgrew its capacity during MD");
                }
                // the counts two chunks ahead (the chunk in flight and the next) at the
                // last chunk's growth, so that a structure whose neighbour counts grow
                // steadily gets room before it overflows
                const int projR = needR + (prevR >= 0 ? 2 * std::max(0, needR - prevR) : 0);
                const int projA = needA + (prevA >= 0 ? 2 * std::max(0, needA - prevA) : 0);
                prevR = needR;
                prevA = needA;
                if (projR * 5 > m->mnR * 4 || projA * 5 > m->mnA * 4) {
                    // grow before the lists overflow: finish the chunk in flight, then
                    // resize and capture again
                    NEP_CUDA(cudaStreamSynchronize(m->cur));
                    m->mnR = std::max(m->mnR, ((int)(projR * 1.5) + 8 + 7) & ~7);
                    m->mnA = std::max(m->mnA, ((int)(projA * 1.5) + 8 + 7) & ~7);
                    NEP_TRY(ensure_lists(m, n));
                    NEP_TRY(capture());
                }
            }
            NEP_CUDA(cudaMemcpyAsync(m->h_async, m->flags.p, 3 * sizeof(int), cudaMemcpyDeviceToHost, m->cur));
            NEP_CUDA(cudaEventRecord(m->ev_flags, m->cur));
            pending = true;
        }
    }
    for (bool prev_close = true; done < n_steps; ++done) {
        const bool smp = sample_every > 0 && (done + 1) % sample_every == 0;
        const bool close = done == n_steps - 1 || smp || th.noise || dr.on;
        NEP_TRY(md_step_launches<real>(m, n, types_d, inv_m.data(), mass.data(), g, pos_d, vel_d, force_d, dt, smp,
                                       sample_every, th, dr, prev_close ? 1 : 2, close));
        prev_close = close;
    }
    NEP_CUDA(cudaMemcpyAsync(m->h_async, m->flags.p, 3 * sizeof(int), cudaMemcpyDeviceToHost, m->cur));
    NEP_CUDA(cudaEventRecord(m->ev_flags, m->cur));
    m->async_pending = true;
    m->async_stream = m->cur;
    if (n_samples > 0)
        NEP_CUDA(cudaMemcpyAsync(thermo, m->thermo.p, sizeof(double) * 12 * n_samples, cudaMemcpyDeviceToHost, m->cur));
    if (heat && n_samples > 0)
        NEP_CUDA(cudaMemcpyAsync(heat, m->heat_rows.p, sizeof(double) * 6 * n_samples, cudaMemcpyDeviceToHost, m->cur));
    if (mem == NEP_HOST) {
        NEP_CUDA(cudaMemcpyAsync(pos, pos_d, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, m->cur));
        NEP_CUDA(cudaMemcpyAsync(vel, vel_d, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, m->cur));
        NEP_CUDA(cudaMemcpyAsync(force, force_d, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, m->cur));
    }
    NEP_TRY(leave(m, stream, !async));
    if (!async) NEP_TRY(inspect_async(m, true));
    return NEP_OK;
}

template <typename real>
int neighbors_impl(nep_model* m, int n, const int32_t* types, const double* pos, const double box[3],
                   const int32_t pbc[3], int kind, int capacity, int32_t* count, int32_t* jout, int32_t* shift)
{
    CellGrid g;
    NEP_TRY(make_grid(m, box, pbc, g));
    NEP_TRY(enter(m, nullptr));
    initial_capacity(m, n, box);
    NEP_TRY(single_plan<real>(m, n, g));
    const Plan& p = m->plan;
    NEP_TRY(ensure_plan_workspace(m, p));
    NEP_TRY(m->types_d.ensure(sizeof(int) * n));
    NEP_TRY(m->pos_d.ensure(sizeof(double) * 3 * (size_t)n));
    NEP_CUDA(cudaMemcpyAsync(m->types_d.p, types, sizeof(int) * n, cudaMemcpyHostToDevice, m->cur));
    NEP_CUDA(cudaMemcpyAsync(m->pos_d.p, pos, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, m->cur));
    NEP_CUDA(cudaMemsetAsync(m->flags.p, 0, 3 * sizeof(int), m->cur));
    m->eval_per_bead = false;
    NEP_TRY(run_cells<real>(m, p, m->types_d.as<int>(), m->pos_d.as<double>()));
    NEP_TRY(run_neighbors<real>(m, p));
    NEP_TRY(check_lists<real>(m, p));
    const int mn = kind == 0 ? m->mnR : m->mnA;
    std::vector<uint32_t> nl((size_t)mn * n);
    std::vector<int> cnt(n), perm(n), cell_s(n);
    NEP_CUDA(cudaMemcpyAsync(nl.data(), kind == 0 ? m->nlR.p : m->nlA.p, sizeof(uint32_t) * nl.size(),
                             cudaMemcpyDeviceToHost, m->cur));
    NEP_CUDA(cudaMemcpyAsync(cnt.data(), kind == 0 ? m->cntR.p : m->cntA.p, sizeof(int) * n, cudaMemcpyDeviceToHost,
                             m->cur));
    NEP_CUDA(cudaMemcpyAsync(perm.data(), m->perm.p, sizeof(int) * n, cudaMemcpyDeviceToHost, m->cur));
    NEP_CUDA(cudaMemcpyAsync(cell_s.data(), m->cell_s.p, sizeof(int) * n, cudaMemcpyDeviceToHost, m->cur));
    NEP_TRY(leave(m, nullptr));
    for (int i = 0; i < n; ++i) {
        const int ui = perm[i];
        const int c = cell_s[i];
        const int ci[3] = {c % g.nc[0], (c / g.nc[0]) % g.nc[1], c / (g.nc[0] * g.nc[1])};
        count[ui] = cnt[i];
        for (int s = 0; s < std::min(cnt[i], std::min(mn, capacity)); ++s) {
            const uint32_t e = nl[(size_t)s * n + i];
            const int k = (int)(e & kJMask);
            const uint32_t code = e >> kJBits;
            const int d[3] = {(int)(code & 7u) - 2, (int)((code >> 3) & 7u) - 2, (int)((code >> 6) & 7u) - 2};
            const int cj = cell_s[k];
            const int cjv[3] = {cj % g.nc[0], (cj / g.nc[0]) % g.nc[1], cj / (g.nc[0] * g.nc[1])};
            jout[(size_t)ui * capacity + s] = perm[k];
            for (int a = 0; a < 3; ++a) {
                int sh = 0;
                if (g.pbc[a]) {
                    const int v = ci[a] + d[a] - cjv[a];  // multiple of nc
                    sh = (v >= 0 ? v / g.nc[a] : -((-v) / g.nc[a]));
                }
                shift[((size_t)ui * capacity + s) * 3 + a] = sh;
            }
        }
    }
    return NEP_OK;
}

// Many configurations, possibly of several models, in one pass of the pipeline.
template <typename real>
int batch_impl(nep_model* const* models, int n_models, int n_req, const int32_t* req_n, const int32_t* req_model,
               const double* req_box, const int32_t* req_pbc, const int32_t* types, const double* pos, int mem,
               void* stream, double* energy, double* virial_total, double* site_energy, double* force,
               double* virial)
{
    nep_model* m = models[0];
    double rc_max = 0.0;
    for (int k = 0; k < n_models; ++k) rc_max = std::max(rc_max, models[k]->rc_max);
    Plan& p = m->plan;
    p.reqs.clear();
    p.items.clear();
    p.n = p.ncell = 0;
    long long total = 0;
    for (int r = 0; r < n_req; ++r) {
        if (req_n[r] < 1) return fail(NEP_ERR_ARG, "every request needs at least one particle");
        if (req_model[r] < 0 || req_model[r] >= n_models) return fail(NEP_ERR_ARG, "request model index out of range");
        total += req_n[r];
        if (total > kMaxN) return fail(NEP_ERR_ARG, "batch exceeds 2^23 particles");
        CellGrid g;
        NEP_TRY(make_grid(models[req_model[r]], models[req_model[r]]->rc_max, req_box + 3 * r, req_pbc + 3 * r, g));
        if ((long long)p.ncell + g.ncell > (long long)kScanItems * kScanItems)
            return fail(NEP_ERR_ARG, "batch cell grids too large");
        add_request(p, g, req_n[r], req_model[r]);
    }
    set_caps(p, true);  // size classes: batches of similar size replay one graph
    set_models<real>(p, models, n_models);
    (void)rc_max;
    NEP_TRY(enter(m, stream));
    {
        double box_avg[3] = {0, 0, 0};  // first sizing of the lists from the largest request
        int rmax = 0;
        for (int r = 1; r < n_req; ++r)
            if (req_n[r] > req_n[rmax]) rmax = r;
        for (int a = 0; a < 3; ++a) box_avg[a] = req_box[3 * rmax + a];
        initial_capacity(m, req_n[rmax], box_avg);
    }
    NEP_TRY(upload_plan(m, p));
    NEP_TRY(ensure_plan_workspace(m, p));
    const int n = p.n;
    const int* types_d = types;
    const double* pos_d = pos;
    double *force_d = force, *virial_d = virial, *site_d = site_energy;
    if (mem == NEP_HOST) {
        NEP_TRY(m->types_d.ensure(sizeof(int) * n));
        NEP_TRY(m->pos_d.ensure(sizeof(double) * 3 * (size_t)n));
        NEP_CUDA(cudaMemcpyAsync(m->types_d.p, types, sizeof(int) * n, cudaMemcpyHostToDevice, m->cur));
        NEP_CUDA(cudaMemcpyAsync(m->pos_d.p, pos, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, m->cur));
        types_d = m->types_d.as<int>();
        pos_d = m->pos_d.as<double>();
        NEP_TRY(m->force_d.ensure(sizeof(double) * 3 * (size_t)n));
        force_d = m->force_d.as<double>();
        virial_d = site_d = nullptr;
        if (virial) {
            NEP_TRY(m->virial_d.ensure(sizeof(double) * 9 * (size_t)n));
            virial_d = m->virial_d.as<double>();
        }
        if (site_energy) {
            NEP_TRY(m->site_d.ensure(sizeof(double) * (size_t)n));
            site_d = m->site_d.as<double>();
        }
    } else if (!force_d) {
        force_d = m->force_tmp.as<double>();
    }
    double* totals = m->totals.as<double>();
    NEP_TRY(ensure_host_totals(m, 10 * (size_t)n_req));
    // one synchronisation per batch (see compute_impl)
    for (int attempt = 0;; ++attempt) {
        NEP_TRY(eval_launch<real>(m, p, types_d, pos_d, force_d, virial_d, site_d, totals));
        if (mem == NEP_HOST) {
            if (force) NEP_CUDA(cudaMemcpyAsync(force, force_d, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, m->cur));
            if (virial)
                NEP_CUDA(cudaMemcpyAsync(virial, virial_d, sizeof(double) * 9 * n, cudaMemcpyDeviceToHost, m->cur));
            if (site_energy)
                NEP_CUDA(cudaMemcpyAsync(site_energy, site_d, sizeof(double) * n, cudaMemcpyDeviceToHost, m->cur));
            NEP_CUDA(cudaMemcpyAsync(m->h_totals, totals, sizeof(double) * 10 * n_req, cudaMemcpyDeviceToHost,
                                     m->cur));
        } else {
            // totals [req][10] -> energy[req], virial_total[req][9] on the device
            if (energy)
                NEP_CUDA(cudaMemcpy2DAsync(energy, sizeof(double), totals, 10 * sizeof(double), sizeof(double), n_req,
                                           cudaMemcpyDeviceToDevice, m->cur));
            if (virial_total)
                NEP_CUDA(cudaMemcpy2DAsync(virial_total, 9 * sizeof(double), totals + 1, 10 * sizeof(double),
                                           9 * sizeof(double), n_req, cudaMemcpyDeviceToDevice, m->cur));
        }
        NEP_CUDA(cudaMemcpyAsync(m->h_flags, m->flags.p, 3 * sizeof(int), cudaMemcpyDeviceToHost, m->cur));
        NEP_TRY(leave(m, stream));
        bool retry = false;
        NEP_TRY(eval_status(m, retry));
        if (!retry) break;
        if (attempt == 2) return fail(NEP_ERR_NEIGHBOR_OVERFLOW, "neighbour capacity did not converge");
        NEP_TRY(enter(m, stream));
    }
    if (mem == NEP_HOST)
        for (int r = 0; r < n_req; ++r) {
            if (energy) energy[r] = m->h_totals[10 * r];
            if (virial_total)
                for (int k = 0; k < 9; ++k) virial_total[9 * r + k] = m->h_totals[10 * r + 1 + k];
        }
    return NEP_OK;
}

}  // namespace

extern "C" {

int nep_version(void) { return (0 << 16) | 2; }

const char* nep_error_string(int code)
{
    switch (code) {
    case NEP_OK: return "ok";
    case NEP_ERR_ARG: return "invalid argument";
    case NEP_ERR_OOM: return "device out of memory";
    case NEP_ERR_NEIGHBOR_OVERFLOW: return "neighbour list overflow";
    case NEP_ERR_BOX_TOO_SMALL: return "box too small for the cutoff";
    case NEP_ERR_TIMEOUT: return "device wait timed out";
    case NEP_ERR_CUDA: return "CUDA error";
    case NEP_ERR_UNSUPPORTED: return "unsupported descriptor or basis sizes";
    default: return "unknown status";
    }
}

const char* nep_last_error(void) { return g_last_error.c_str(); }

int nep_supported_shape(int n_desc_radial, int n_desc_angular, int n_basis_radial, int n_basis_angular, int l_max,
                        int l_max_4b, int l_max_5b)
{
    return l_max == 4 && (l_max_4b == 0 || l_max_4b == 2) && (l_max_5b == 0 || l_max_5b == 1) &&
           evaluate_shape_supported<float>(n_desc_radial, n_desc_angular, n_basis_radial, n_basis_angular);
}

int nep_destroy(nep_model* m)
{
    if (!m) return NEP_OK;
    Guard guard(m->device);
    if (m->st) cudaStreamSynchronize(m->st);
    if (m->async_pending && m->ev_flags) cudaEventSynchronize(m->ev_flags);
    if (m->plan_pending && m->ev_plan) cudaEventSynchronize(m->ev_plan);
    m->graph.reset();
    for (GraphCache& g : m->eval_graphs) g.reset();
    m->eval_graphs.clear();
    m->timer.destroy();
    Buf* bufs[] = {&m->params, &m->cell_of, &m->rec_user, &m->perm_tmp, &m->perm, &m->rec_s, &m->cell_s, &m->cntR,
                   &m->cntA, &m->nlR, &m->nlA, &m->U, &m->e, &m->phi, &m->rec32, &m->cell_count, &m->cell_local, &m->block_off,
                   &m->cell_fill, &m->cell_start, &m->partial, &m->partial2, &m->counters, &m->gcounters,
                   &m->totals, &m->flags,
                   &m->thermo, &m->sample_index, &m->types_d, &m->pos_d, &m->vel_d, &m->force_d, &m->virial_d,
                   &m->site_d, &m->force_tmp, &m->totals_tmp, &m->plan.dev, &m->noise_d, &m->bussi,
                   &m->md_virial, &m->md_site, &m->heat, &m->heat_rows, &m->acc};
    for (Buf* b : bufs) b->release();
    if (m->h_flags) cudaFreeHost(m->h_flags);
    if (m->h_totals) cudaFreeHost(m->h_totals);
    if (m->h_async) cudaFreeHost(m->h_async);
    if (m->h_stage) cudaFreeHost(m->h_stage);
    if (m->ev_flags) cudaEventDestroy(m->ev_flags);
    if (m->ev_plan) cudaEventDestroy(m->ev_plan);
    if (m->ev_in) cudaEventDestroy(m->ev_in);
    if (m->ev_out) cudaEventDestroy(m->ev_out);
    if (m->st) cudaStreamDestroy(m->st);
    delete m;
    return NEP_OK;
}

int nep_create(nep_model** out, int n_types, const double* rc_radial, const double* rc_angular, int n_basis_radial,
               int n_basis_angular, int n_desc_radial, int n_desc_angular, int l_max, int l_max_4b, int l_max_5b,
               int hidden,
               const double* c_radial, const double* c_angular, const double* w0, const double* b0, const double* w1,
               const double* b1, int precision, int device)
{
    if (!out) return fail(NEP_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (n_types < 1 || n_types > kMaxTypes) return fail(NEP_ERR_ARG, "n_types out of range [1, 16]");
    if (hidden < 1 || hidden > 4096) return fail(NEP_ERR_ARG, "hidden out of range");
    if (precision != NEP_FP32 && precision != NEP_FP64 && precision != NEP_FP32_BF16)
        return fail(NEP_ERR_ARG, "unknown precision");
    if (!rc_radial || !rc_angular || !c_radial || !c_angular || !w0 || !b0 || !w1 || !b1)
        return fail(NEP_ERR_ARG, "null parameter array");
    if (!nep_supported_shape(n_desc_radial, n_desc_angular, n_basis_radial, n_basis_angular, l_max, l_max_4b,
                             l_max_5b))
        return fail(NEP_ERR_UNSUPPORTED, "no compiled kernel for these descriptor / basis sizes");
    const int T = n_types;
    for (int a = 0; a < T; ++a)
        for (int b = 0; b < T; ++b) {
            const double r1 = rc_radial[a * T + b], r2 = rc_angular[a * T + b];
            if (!(r1 > 0.0) || !(r2 > 0.0) || !isfinite(r1) || !isfinite(r2))
                return fail(NEP_ERR_ARG, "cutoffs must be positive and finite");
            if (r1 != rc_radial[b * T + a] || r2 != rc_angular[b * T + a])
                return fail(NEP_ERR_ARG, "cutoff tables must be symmetric");
        }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) return fail(NEP_ERR_CUDA, "no CUDA device");
    if (device < 0 || device >= ndev) return fail(NEP_ERR_ARG, "device out of range");
    Guard guard(device);

    nep_model* m = new nep_model();
    m->device = device;
    m->precision = precision;
    m->T = T;
    m->nR = n_desc_radial;
    m->nA = n_desc_angular;
    m->KR = n_basis_radial;
    m->KA = n_basis_angular;
    m->L = l_max;
    m->L4 = l_max_4b;
    m->L5 = l_max_5b;
    m->MBT = (l_max_4b > 0 || l_max_5b > 0) ? 1 : 0;
    m->H = hidden;
    // device layout: with MBT both many-body blocks are present (q4 then q5); a
    // model with only one of them gets zero weights on the other, which changes no
    // sum (0 * q adds an exact zero) and no gradient
    m->ND = m->nR + m->nA * (m->L + 2 * m->MBT);
    const int nd_user = m->nR + m->nA * (m->L + (l_max_4b > 0) + (l_max_5b > 0));
    m->KRP = (m->KR + 3) & ~3;
    m->rcR.assign(rc_radial, rc_radial + T * T);
    m->rcA.assign(rc_angular, rc_angular + T * T);
    for (int k = 0; k < T * T; ++k) m->rc_max = std::max(m->rc_max, std::max(m->rcR[k], m->rcA[k]));
    m->real_size = precision == NEP_FP64 ? 8 : 4;

    // parameter layout: cutoffs and coefficient tables first (the force kernel
    // stages only that prefix), then the network
    ParamLayout& o = m->off;
    int p = 0;
    const int TT = T * T;
    o.rcR2 = p; p += TT;
    o.rcA2 = p; p += TT;
    o.rcRi = p; p += TT;
    o.rcAi = p; p += TT;
    o.rcRl = p; p += TT;
    o.rcAl = p; p += TT;
    const int cRs = coef_stride(m->nR, m->KR), cAs = coef_stride(m->nA, m->KA);
    o.cR = p; p += TT * cRs;
    if (T == 1) p = (p + 3) & ~3;  // one type: its angular table is read with 16-byte vector loads
    o.cA = p; p += TT * cAs;
    o.n_cut_coef = p;
    // W0 rows: one type pads them to a multiple of 4 reals at a 16-byte aligned start
    // (the descriptor kernel reads them as vectors); several types keep ND per row
    const int w0s = T == 1 ? ((m->ND + 3) & ~3) : m->ND;
    if (T == 1) p = (p + 3) & ~3;
    o.w0 = p; p += T * hidden * w0s;
    o.b0 = p; p += T * hidden;
    o.w1 = p; p += T * hidden;
    o.b1 = p; p += T;
    // FP32 form: each network parameter and radial coefficient also as its rounding
    // residual, so that the kernels evaluate the caller's FP64 model to ~1e-14 rather
    // than a model rounded to FP32 (the rounding is the same for every particle and
    // would otherwise add a consistent offset to every site energy)
    o.w0l = o.b0l = o.w1l = o.b1l = o.cRl = -1;
    if (precision != NEP_FP64) {
        if (T == 1) p = (p + 3) & ~3;
        o.w0l = p; p += T * hidden * w0s;
        o.b0l = p; p += T * hidden;
        o.w1l = p; p += T * hidden;
        o.b1l = p; p += T;
        o.cRl = p; p += TT * cRs;
    }
    o.w0f = o.w0b = -1;
    const int nd = m->ND, hp = net_hp(hidden);
    if (precision == NEP_FP32_BF16) {  // BF16 copies of W0 laid out as MMA B operands
        p = (p + 3) & ~3;              // 16-byte aligned
        o.w0f = p; p += T * hp * net_sf(nd) / 2;
        o.w0b = p; p += T * net_ndp(nd) * (hp + 8) / 2;
    }
    o.total = p;
    std::vector<double> h(p);
    for (int k = 0; k < TT; ++k) {
        h[o.rcR2 + k] = m->rcR[k] * m->rcR[k];
        h[o.rcA2 + k] = m->rcA[k] * m->rcA[k];
        h[o.rcRi + k] = 1.0 / m->rcR[k];
        h[o.rcAi + k] = 1.0 / m->rcA[k];
        // the FP32 kernels form r / r_c as r (hi + lo): FP32 1/r_c alone is off by up
        // to 6e-8 relative, the same for every pair of a type pair, which would shift
        // every cutoff value one way
        h[o.rcRl + k] = precision == NEP_FP64 ? 0.0 : 1.0 / m->rcR[k] - (double)(float)(1.0 / m->rcR[k]);
        h[o.rcAl + k] = precision == NEP_FP64 ? 0.0 : 1.0 / m->rcA[k] - (double)(float)(1.0 / m->rcA[k]);
    }
    for (int k = 0; k < TT; ++k) {  // pair tables at odd strides
        std::copy(c_radial + (size_t)k * m->nR * m->KR, c_radial + (size_t)(k + 1) * m->nR * m->KR,
                  h.begin() + o.cR + k * cRs);
        std::copy(c_angular + (size_t)k * m->nA * m->KA, c_angular + (size_t)(k + 1) * m->nA * m->KA,
                  h.begin() + o.cA + k * cAs);
    }
    for (int t = 0; t < T; ++t)
        for (int mu = 0; mu < hidden; ++mu) {
            const double* src = w0 + ((size_t)t * hidden + mu) * nd_user;
            double* dst = h.data() + o.w0 + ((size_t)t * hidden + mu) * w0s;
            const int d3 = m->nR + m->nA * m->L;
            std::copy(src, src + d3, dst);
            int k = d3;
            if (l_max_4b > 0) {
                std::copy(src + k, src + k + m->nA, dst + d3);
                k += m->nA;
            }
            if (l_max_5b > 0) std::copy(src + k, src + k + m->nA, dst + d3 + m->nA);
        }
    std::copy(b0, b0 + T * hidden, h.begin() + o.b0);
    std::copy(w1, w1 + T * hidden, h.begin() + o.w1);
    std::copy(b1, b1 + T, h.begin() + o.b1);
    if (o.w0l >= 0) {  // rounding residuals of the FP32 tables
        auto residual = [&](int hi, int lo, int count) {
            for (int k = 0; k < count; ++k) h[lo + k] = h[hi + k] - (double)(float)h[hi + k];
        };
        residual(o.w0, o.w0l, T * hidden * w0s);
        residual(o.b0, o.b0l, T * hidden);
        residual(o.w1, o.w1l, T * hidden);
        residual(o.b1, o.b1l, T);
        residual(o.cR, o.cRl, TT * cRs);
    }

    auto cleanup = [&](int code) {
        nep_destroy(m);
        return code;
    };
    if (m->params.ensure(m->real_size * p) != NEP_OK) return cleanup(NEP_ERR_OOM);
    if (precision == NEP_FP64) {
        if (cudaMemcpy(m->params.p, h.data(), sizeof(double) * p, cudaMemcpyHostToDevice) != cudaSuccess)
            return cleanup(fail(NEP_ERR_CUDA, "parameter upload failed"));
    } else {
        std::vector<float> hf(h.begin(), h.end());
        if (precision == NEP_FP32_BF16) {
            // W0[t][mu][v] rounded to FP32 and then to BF16 (round to nearest even)
            auto bf16 = [](double x) -> uint16_t {
                const float f = (float)x;
                uint32_t u;
                memcpy(&u, &f, 4);
                if ((u & 0x7fffffffu) > 0x7f800000u) return 0x7fc0;  // NaN
                u += 0x7fffu + ((u >> 16) & 1u);
                return (uint16_t)(u >> 16);
            };
            const int sf = net_sf(nd), ndp = net_ndp(nd), sb = hp + 8;
            std::vector<uint16_t> wf((size_t)T * hp * sf, 0), wb((size_t)T * ndp * sb, 0);
            for (int t = 0; t < T; ++t)
                for (int mu = 0; mu < hidden; ++mu)
                    for (int v = 0; v < nd; ++v) {
                        const uint16_t b = bf16(h[o.w0 + ((size_t)t * hidden + mu) * w0s + v]);
                        wf[((size_t)t * hp + mu) * sf + v] = b;   // [t][mu][v]: X = Q W0^T
                        wb[((size_t)t * ndp + v) * sb + mu] = b;  // [t][v][mu]: dQ = D W0
                    }
            memcpy(hf.data() + o.w0f, wf.data(), wf.size() * 2);
            memcpy(hf.data() + o.w0b, wb.data(), wb.size() * 2);
        }
        if (cudaMemcpy(m->params.p, hf.data(), sizeof(float) * p, cudaMemcpyHostToDevice) != cudaSuccess)
            return cleanup(fail(NEP_ERR_CUDA, "parameter upload failed"));
    }
    m->smem_desc = m->real_size * o.total;
    if (precision == NEP_FP32_BF16)  // plus the per-warp scratch of the network products
        m->smem_desc = ((m->smem_desc + 15) & ~(size_t)15) + (size_t)(kBlock / 32) * net_scratch(nd);
    // the force kernel stages the cutoff + coefficient prefix only
    m->smem_force = m->real_size * o.n_cut_coef;
    if (m->smem_desc > 200 * 1024 || m->smem_force > 200 * 1024)
        return cleanup(fail(NEP_ERR_ARG, "model too large for shared-memory staging"));
    // the attribute is per kernel, shared by all handles: allow the largest staging size
    const size_t smem_cap = 200 * 1024;
    cudaError_t e = precision == NEP_FP64
                        ? evaluate_set_smem<double>(m->nR, m->nA, m->KR, m->KA, smem_cap, smem_cap)
                        : evaluate_set_smem<float>(m->nR, m->nA, m->KR, m->KA, smem_cap, smem_cap);
    if (e != cudaSuccess) return cleanup(fail(NEP_ERR_CUDA, std::string("smem attribute: ") + cudaGetErrorString(e)));
    if (cudaStreamCreateWithFlags(&m->st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&m->ev_in, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&m->ev_out, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&m->ev_flags, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&m->ev_plan, cudaEventDisableTiming) != cudaSuccess)
        return cleanup(fail(NEP_ERR_CUDA, "stream/event creation failed"));
    if (m->flags.ensure(sizeof(int) * 4) != NEP_OK) return cleanup(NEP_ERR_OOM);
    if (cudaMemset(m->flags.p, 0, sizeof(int) * 4) != cudaSuccess ||
        cudaMallocHost((void**)&m->h_flags, sizeof(int) * 4) != cudaSuccess ||
        cudaMallocHost((void**)&m->h_async, sizeof(int) * 4) != cudaSuccess ||
        cudaMallocHost((void**)&m->h_stage, 16384) != cudaSuccess ||
        cudaMallocHost((void**)&m->h_totals, sizeof(double) * 10) != cudaSuccess)
        return cleanup(fail(NEP_ERR_CUDA, "workspace initialisation failed"));
    m->h_stage_cap = 16384;
    m->h_totals_cap = 10;
    *out = m;
    return NEP_OK;
}

int nep_compute(nep_model* m, int n, const int32_t* types, const double* pos, const double box[3],
                const int32_t pbc[3], int mem, void* stream, double* energy_total, double* virial_total,
                double* site_energy, double* force, double* virial)
{
    NEP_TRY(validate_common(m, n, types, pos, box, pbc, mem));
    Guard guard(m->device);
    NEP_TRY(inspect_async(m, true));
    return m->precision == NEP_FP64
               ? compute_impl<double>(m, n, types, pos, box, pbc, mem, stream, energy_total, virial_total, site_energy,
                                      force, virial)
               : compute_impl<float>(m, n, types, pos, box, pbc, mem, stream, energy_total, virial_total, site_energy,
                                     force, virial);
}

int nep_compute_batch(nep_model* const* models, int n_models, int n_req, const int32_t* req_n,
                      const int32_t* req_model, const double* req_box, const int32_t* req_pbc, const int32_t* types,
                      const double* pos, int mem, void* stream, double* energy, double* virial_total,
                      double* site_energy, double* force, double* virial)
{
    if (!models || n_models < 1 || !models[0]) return fail(NEP_ERR_ARG, "no models");
    if (n_req < 1 || !req_n || !req_model || !req_box || !req_pbc || !types || !pos)
        return fail(NEP_ERR_ARG, "bad request arrays");
    if (mem != NEP_HOST && mem != NEP_DEVICE) return fail(NEP_ERR_ARG, "mem must be NEP_HOST or NEP_DEVICE");
    nep_model* m = models[0];
    for (int k = 0; k < n_models; ++k) {
        const nep_model* o = models[k];
        if (!o) return fail(NEP_ERR_ARG, "null model in batch");
        if (o->device != m->device || o->precision != m->precision || o->nR != m->nR || o->nA != m->nA ||
            o->KR != m->KR || o->KA != m->KA || o->L != m->L || o->MBT != m->MBT)
            return fail(NEP_ERR_ARG, "batched models must share device, precision and descriptor sizes");
    }
    Guard guard(m->device);
    NEP_TRY(inspect_async(m, true));
    return m->precision == NEP_FP64
               ? batch_impl<double>(models, n_models, n_req, req_n, req_model, req_box, req_pbc, types, pos, mem,
                                    stream, energy, virial_total, site_energy, force, virial)
               : batch_impl<float>(models, n_models, n_req, req_n, req_model, req_box, req_pbc, types, pos, mem,
                                   stream, energy, virial_total, site_energy, force, virial);
}

int nep_md_step(nep_model* m, int n, const int32_t* types, const double* masses, const double box[3],
                const int32_t pbc[3], double* pos, double* vel, double* force, int forces_valid, int n_steps,
                double dt_fs, int sample_every, double* thermo, int mem, void* stream)
{
    NEP_TRY(validate_common(m, n, types, pos, box, pbc, mem));
    if (!(dt_fs > 0.0) || !isfinite(dt_fs)) return fail(NEP_ERR_ARG, "dt must be positive");
    Guard guard(m->device);
    return m->precision == NEP_FP64
               ? md_impl<double>(m, n, types, masses, box, pbc, pos, vel, force, forces_valid, n_steps, dt_fs,
                                 sample_every, thermo, mem, stream)
               : md_impl<float>(m, n, types, masses, box, pbc, pos, vel, force, forces_valid, n_steps, dt_fs,
                                sample_every, thermo, mem, stream);
}

int nep_md_step_nvt(nep_model* m, int n, const int32_t* types, const double* masses, const double box[3],
                    const int32_t pbc[3], double* pos, double* vel, double* force, int forces_valid, int n_steps,
                    double dt_fs, double temperature_K, double tau_fs, const double* noise, int sample_every,
                    double* thermo, int mem, void* stream)
{
    NEP_TRY(validate_common(m, n, types, pos, box, pbc, mem));
    if (!(dt_fs > 0.0) || !isfinite(dt_fs)) return fail(NEP_ERR_ARG, "dt must be positive");
    if (!(temperature_K >= 0.0) || !(tau_fs > 0.0)) return fail(NEP_ERR_ARG, "need temperature >= 0 and tau > 0");
    if (!noise && n_steps > 0) return fail(NEP_ERR_ARG, "noise is NULL");
    if (n < 2) return fail(NEP_ERR_ARG, "the thermostat needs n >= 2");
    Guard guard(m->device);
    return m->precision == NEP_FP64
               ? md_impl<double>(m, n, types, masses, box, pbc, pos, vel, force, forces_valid, n_steps, dt_fs,
                                 sample_every, thermo, mem, stream, temperature_K, tau_fs, noise)
               : md_impl<float>(m, n, types, masses, box, pbc, pos, vel, force, forces_valid, n_steps, dt_fs,
                                sample_every, thermo, mem, stream, temperature_K, tau_fs, noise);
}

int nep_md_step_hnemd(nep_model* m, int n, const int32_t* types, const double* masses, const double box[3],
                      const int32_t pbc[3], double* pos, double* vel, double* force, int forces_valid, int n_steps,
                      double dt_fs, const double fe[3], double temperature_K, double tau_fs, const double* noise,
                      int sample_every, double* thermo, double* heat, int mem, void* stream)
{
    NEP_TRY(validate_common(m, n, types, pos, box, pbc, mem));
    if (!(dt_fs > 0.0) || !isfinite(dt_fs)) return fail(NEP_ERR_ARG, "dt must be positive");
    if (!fe || !isfinite(fe[0]) || !isfinite(fe[1]) || !isfinite(fe[2]))
        return fail(NEP_ERR_ARG, "the driving force parameter must be three finite numbers");
    if (noise && (!(temperature_K >= 0.0) || !(tau_fs > 0.0)))
        return fail(NEP_ERR_ARG, "need temperature >= 0 and tau > 0");
    if (noise && n < 2) return fail(NEP_ERR_ARG, "the thermostat needs n >= 2");
    if (heat && sample_every <= 0) return fail(NEP_ERR_ARG, "heat rows need sample_every > 0");
    Guard guard(m->device);
    return m->precision == NEP_FP64
               ? md_impl<double>(m, n, types, masses, box, pbc, pos, vel, force, forces_valid, n_steps, dt_fs,
                                 sample_every, thermo, mem, stream, temperature_K, tau_fs, noise, fe, heat)
               : md_impl<float>(m, n, types, masses, box, pbc, pos, vel, force, forces_valid, n_steps, dt_fs,
                                sample_every, thermo, mem, stream, temperature_K, tau_fs, noise, fe, heat);
}

int nep_cg_map(nep_model* m, int n_cg, const int32_t* group_start, const int32_t* group_atoms, int n_aa,
               const double* atom_mass, const double* atom_pos, const double* atom_force, const double* atom_virial,
               const double box[3], const int32_t pbc[3], int accumulate, int mem, void* stream, double* bead_pos,
               double* bead_force, double* bead_virial)
{
    if (!m) return fail(NEP_ERR_ARG, "null model");
    if (n_cg < 1 || n_aa < 1 || !group_start || !group_atoms || !atom_mass || !atom_pos || !box || !pbc)
        return fail(NEP_ERR_ARG, "bad mapping arguments");
    if (mem != NEP_HOST && mem != NEP_DEVICE) return fail(NEP_ERR_ARG, "mem must be NEP_HOST or NEP_DEVICE");
    CellGrid g{};
    for (int a = 0; a < 3; ++a) {
        if (!(box[a] > 0.0)) return fail(NEP_ERR_ARG, "box lengths must be positive");
        g.box[a] = box[a];
        g.pbc[a] = pbc[a] ? 1 : 0;
    }
    Guard guard(m->device);
    NEP_TRY(inspect_async(m, true));
    NEP_TRY(enter(m, stream));
    if (mem == NEP_DEVICE) {
        cudaError_t e = launch_cg_map(n_cg, n_aa, group_start, group_atoms, atom_mass, atom_pos, atom_force,
                                      atom_virial, g, accumulate, bead_pos, bead_force, bead_virial, m->cur);
        if (e != cudaSuccess) return fail(NEP_ERR_CUDA, std::string("cg map: ") + cudaGetErrorString(e));
        return leave(m, stream);
    }
    // host memory: stage through one device buffer
    const int n_members = group_start[n_cg];
    if (n_members < 0 || n_members > n_aa) return fail(NEP_ERR_ARG, "group_start[n_cg] out of range");
    const size_t b_int = sizeof(int) * ((size_t)n_cg + 1 + n_members);
    const size_t b_aa = sizeof(double) * (size_t)n_aa * (1 + 3 + (atom_force ? 3 : 0) + (atom_virial ? 9 : 0));
    const size_t b_cg = sizeof(double) * (size_t)n_cg * (3 + 3 + 9);
    NEP_TRY(m->force_tmp.ensure(b_int + b_aa + b_cg + 64));
    unsigned char* base = (unsigned char*)m->force_tmp.p;
    int* d_start = (int*)base;
    int* d_atoms = d_start + n_cg + 1;
    double* d = (double*)(base + ((b_int + 7) & ~(size_t)7));
    double* d_mass = d;
    double* d_pos = d_mass + n_aa;
    double* d_force = atom_force ? d_pos + 3 * (size_t)n_aa : nullptr;
    double* d_vir = atom_virial ? (d_force ? d_force : d_pos) + 3 * (size_t)n_aa : nullptr;
    double* d_out = (d_vir ? d_vir + 9 * (size_t)n_aa : (d_force ? d_force + 3 * (size_t)n_aa : d_pos + 3 * (size_t)n_aa));
    double* o_pos = d_out;
    double* o_force = o_pos + 3 * (size_t)n_cg;
    double* o_vir = o_force + 3 * (size_t)n_cg;
    NEP_CUDA(cudaMemcpyAsync(d_start, group_start, sizeof(int) * (n_cg + 1), cudaMemcpyHostToDevice, m->cur));
    NEP_CUDA(cudaMemcpyAsync(d_atoms, group_atoms, sizeof(int) * n_members, cudaMemcpyHostToDevice, m->cur));
    NEP_CUDA(cudaMemcpyAsync(d_mass, atom_mass, sizeof(double) * n_aa, cudaMemcpyHostToDevice, m->cur));
    NEP_CUDA(cudaMemcpyAsync(d_pos, atom_pos, sizeof(double) * 3 * n_aa, cudaMemcpyHostToDevice, m->cur));
    if (d_force) NEP_CUDA(cudaMemcpyAsync(d_force, atom_force, sizeof(double) * 3 * n_aa, cudaMemcpyHostToDevice, m->cur));
    if (d_vir) NEP_CUDA(cudaMemcpyAsync(d_vir, atom_virial, sizeof(double) * 9 * n_aa, cudaMemcpyHostToDevice, m->cur));
    if (accumulate) {
        if (bead_force) NEP_CUDA(cudaMemcpyAsync(o_force, bead_force, sizeof(double) * 3 * n_cg, cudaMemcpyHostToDevice, m->cur));
        if (bead_virial) NEP_CUDA(cudaMemcpyAsync(o_vir, bead_virial, sizeof(double) * 9 * n_cg, cudaMemcpyHostToDevice, m->cur));
    }
    cudaError_t e = launch_cg_map(n_cg, n_aa, d_start, d_atoms, d_mass, d_pos, d_force, d_vir, g, accumulate,
                                  bead_pos ? o_pos : nullptr, bead_force ? o_force : nullptr,
                                  bead_virial ? o_vir : nullptr, m->cur);
    if (e != cudaSuccess) return fail(NEP_ERR_CUDA, std::string("cg map: ") + cudaGetErrorString(e));
    if (bead_pos) NEP_CUDA(cudaMemcpyAsync(bead_pos, o_pos, sizeof(double) * 3 * n_cg, cudaMemcpyDeviceToHost, m->cur));
    if (bead_force && d_force)
        NEP_CUDA(cudaMemcpyAsync(bead_force, o_force, sizeof(double) * 3 * n_cg, cudaMemcpyDeviceToHost, m->cur));
    if (bead_virial && d_vir)
        NEP_CUDA(cudaMemcpyAsync(bead_virial, o_vir, sizeof(double) * 9 * n_cg, cudaMemcpyDeviceToHost, m->cur));
    return leave(m, stream);
}

int nep_virial_correction(double* virial, int n_atoms, int n_beads, double temperature_K)
{
    if (!virial || n_atoms < 0 || n_beads < 0 || !(temperature_K >= 0.0)) return fail(NEP_ERR_ARG, "bad argument");
    const double add = (double)(n_atoms - n_beads) * 8.617333262e-5 * temperature_K;
    virial[0] += add;
    virial[4] += add;
    virial[8] += add;
    return NEP_OK;
}

int nep_autotune(nep_model* m, int n, const int32_t* types, const double* pos, const double box[3],
                 const int32_t pbc[3], int mem, void* stream, int* mb_desc, int* mb_force, int* chunk)
{
    NEP_TRY(validate_common(m, n, types, pos, box, pbc, mem));
    Guard guard(m->device);
    NEP_TRY(inspect_async(m, true));
    CellGrid g;
    NEP_TRY(make_grid(m, box, pbc, g));
    NEP_TRY(enter(m, stream));
    initial_capacity(m, n, box);
    const int* types_d = types;
    const double* pos_d = pos;
    if (mem == NEP_HOST) {
        NEP_TRY(m->types_d.ensure(sizeof(int) * n));
        NEP_TRY(m->pos_d.ensure(sizeof(double) * 3 * (size_t)n));
        NEP_CUDA(cudaMemcpyAsync(m->types_d.p, types, sizeof(int) * n, cudaMemcpyHostToDevice, m->cur));
        NEP_CUDA(cudaMemcpyAsync(m->pos_d.p, pos, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, m->cur));
        types_d = m->types_d.as<int>();
        pos_d = m->pos_d.as<double>();
    }
    int rc;
    if (m->precision == NEP_FP64) {
        rc = single_plan<double>(m, n, g);
        if (rc == NEP_OK) rc = ensure_plan_workspace(m, m->plan);
        if (rc == NEP_OK) rc = evaluate_plan<double>(m, m->plan, types_d, pos_d, m->force_tmp.as<double>(), nullptr,
                                                     nullptr, m->totals.as<double>());
    } else {
        rc = single_plan<float>(m, n, g);
        if (rc == NEP_OK) rc = ensure_plan_workspace(m, m->plan);
        if (rc == NEP_OK) rc = evaluate_plan<float>(m, m->plan, types_d, pos_d, m->force_tmp.as<double>(), nullptr,
                                                    nullptr, m->totals.as<double>());
        if (rc == NEP_OK) rc = autotune_plan<float>(m, m->plan, m->force_tmp.as<double>());
    }
    NEP_TRY(rc);
    NEP_TRY(leave(m, stream));
    if (mb_desc) *mb_desc = m->mb_desc;
    if (mb_force) *mb_force = m->mb_force;
    if (chunk) *chunk = m->ch_force;
    return NEP_OK;
}

int nep_set_tuning(nep_model* m, int autotune, int mb_desc, int mb_force, int chunk)
{
    if (!m) return fail(NEP_ERR_ARG, "null model");
    if ((mb_desc != 2 && mb_desc != 3) || (mb_force < 3 || mb_force > 5) || (chunk != 4 && chunk != 8))
        return fail(NEP_ERR_ARG, "kernel variants: descriptor 2 or 3, force 3, 4 or 5, chunk 4 or 8");
    m->autotune = autotune != 0;
    m->mb_desc = mb_desc;
    m->mb_force = mb_force;
    m->ch_force = chunk;
    m->graph.reset();
    return NEP_OK;
}

int nep_get_tuning(nep_model* m, int* mb_desc, int* mb_force, int* chunk)
{
    if (!m) return fail(NEP_ERR_ARG, "null model");
    if (mb_desc) *mb_desc = m->mb_desc;
    if (mb_force) *mb_force = m->mb_force;
    if (chunk) *chunk = m->ch_force;
    return NEP_OK;
}

int nep_sync(nep_model* m)
{
    if (!m) return fail(NEP_ERR_ARG, "null model");
    Guard guard(m->device);
    return inspect_async(m, true);
}

int nep_scale_positions(nep_model* m, int n, double* pos, const double scale[3], int mem, void* stream)
{
    if (!m || !pos || !scale || n < 1) return fail(NEP_ERR_ARG, "bad argument");
    if (mem == NEP_HOST) {
        for (int a = 0; a < 3; ++a)
            for (int i = 0; i < n; ++i) pos[(size_t)a * n + i] *= scale[a];
        return NEP_OK;
    }
    Guard guard(m->device);
    cudaError_t e = launch_scale(n, pos, scale[0], scale[1], scale[2], (cudaStream_t)stream);
    if (e != cudaSuccess) return fail(NEP_ERR_CUDA, cudaGetErrorString(e));
    return NEP_OK;
}

int nep_neighbors(nep_model* m, int n, const int32_t* types, const double* pos, const double box[3],
                  const int32_t pbc[3], int kind, int capacity, int32_t* count, int32_t* j, int32_t* shift)
{
    NEP_TRY(validate_common(m, n, types, pos, box, pbc, NEP_HOST));
    if (kind != 0 && kind != 1) return fail(NEP_ERR_ARG, "kind must be 0 or 1");
    if (capacity < 1 || !count || !j || !shift) return fail(NEP_ERR_ARG, "bad output buffers");
    Guard guard(m->device);
    NEP_TRY(inspect_async(m, true));
    return m->precision == NEP_FP64 ? neighbors_impl<double>(m, n, types, pos, box, pbc, kind, capacity, count, j, shift)
                                    : neighbors_impl<float>(m, n, types, pos, box, pbc, kind, capacity, count, j, shift);
}

int nep_set_timing(nep_model* m, int enable)
{
    if (!m) return fail(NEP_ERR_ARG, "null model");
    Guard guard(m->device);
    if (enable && m->timer.create() != 0) return fail(NEP_ERR_CUDA, "event creation failed");
    m->timer.reset();
    m->timer.on = enable != 0;
    return NEP_OK;
}

int nep_get_timing(nep_model* m, double* stage_ms, long long* steps)
{
    if (!m) return fail(NEP_ERR_ARG, "null model");
    Guard guard(m->device);
    m->timer.drain();
    if (stage_ms)
        for (int k = 0; k < StageTimer::kEv - 1; ++k) stage_ms[k] = m->timer.acc[k];
    if (steps) *steps = m->timer.steps;
    return NEP_OK;
}

int nep_get_capacity(nep_model* m, int* radial, int* angular)
{
    if (!m) return fail(NEP_ERR_ARG, "null model");
    if (radial) *radial = m->mnR;
    if (angular) *angular = m->mnA;
    return NEP_OK;
}

// Device bytes one request adds to a batch on models[0]'s workspace: the sizes
// ensure_plan_workspace, ensure_lists and the host-call staging of batch_impl
// allocate, per particle, per cell, per work item and per request, with the
// batch's largest type count (the gradient array's stride) and models[0]'s list
// capacities.
int nep_request_workspace(nep_model* const* models, int n_models, int model, int n, const double box[3],
                          const int32_t pbc[3], size_t* bytes)
{
    if (!models || n_models < 1 || model < 0 || model >= n_models || n < 1 || !box || !pbc || !bytes)
        return fail(NEP_ERR_ARG, "bad argument");
    const nep_model* m = models[0];
    int Tmax = 1;
    for (int k = 0; k < n_models; ++k) {
        if (!models[k]) return fail(NEP_ERR_ARG, "null model");
        Tmax = std::max(Tmax, models[k]->T);
    }
    CellGrid g;
    NEP_TRY(make_grid(models[model], models[model]->rc_max, box, pbc, g));
    int mnR = m->mnR, mnA = m->mnA;
    if (mnR <= 0 || mnA <= 0) {  // not sized yet: the first-call estimate from the density
        const double rho = n / (box[0] * box[1] * box[2]);
        double rR = 0, rA = 0;
        for (double v : m->rcR) rR = std::max(rR, v);
        for (double v : m->rcA) rA = std::max(rA, v);
        auto est = [&](double rc) { return (std::min((int)(4.18879 * rc * rc * rc * rho * 1.3 + 16), 4096) + 7) & ~7; };
        if (mnR <= 0) mnR = est(rR);
        if (mnA <= 0) mnA = est(rA);
    }
    const size_t rs = m->real_size;
    // cell_of, rec_user, perm_tmp, perm, rec_s, cell_s, cntR, cntA, U, e, force_tmp, partial2
    size_t per_particle = 4 + 4 * rs + 4 + 4 + 4 * rs + 4 + 4 + 4 + rs + rs * Tmax * m->KRP + 24 + 1;
    if (m->precision == NEP_FP64) per_particle += rs * kPsiComp * phi_pad(m->nA) + 16;
    else per_particle += acc_bytes(1);            // fixed-point lines, thread virial sums
    per_particle += 4 * (size_t)(mnR + mnA);      // neighbour lists
    per_particle += 4 + 24 + 24 + 72 + 8;          // host-call staging: types, positions, F, W, U
    const size_t per_cell = 16;                    // count, local prefix, fill, start
    const size_t items = ((size_t)n + kBlock - 1) / kBlock;
    const size_t per_item = 10 * sizeof(double) + sizeof(WorkItem) + sizeof(unsigned int);  // + group counter
    const size_t per_req = sizeof(ReqInfo) + 10 * sizeof(double) + sizeof(unsigned int);
    *bytes = per_particle * n + per_cell * g.ncell + per_item * items + per_req;
    return NEP_OK;
}

int nep_workspace_bytes(nep_model* m, size_t* bytes)
{
    if (!m || !bytes) return fail(NEP_ERR_ARG, "bad argument");
    const Buf* bufs[] = {&m->cell_of, &m->rec_user, &m->perm_tmp, &m->perm, &m->rec_s, &m->cell_s, &m->cntR,
                         &m->cntA, &m->nlR, &m->nlA, &m->U, &m->e, &m->phi, &m->rec32, &m->cell_count, &m->cell_local,
                         &m->block_off, &m->cell_fill, &m->cell_start, &m->partial, &m->partial2, &m->counters,
                         &m->gcounters, &m->totals, &m->flags, &m->thermo, &m->sample_index, &m->types_d,
                         &m->pos_d, &m->vel_d, &m->force_d, &m->virial_d, &m->site_d, &m->force_tmp,
                         &m->totals_tmp, &m->plan.dev,
                         &m->noise_d, &m->bussi, &m->md_virial, &m->md_site, &m->heat, &m->heat_rows, &m->acc};
    size_t t = 0;
    for (const Buf* b : bufs) t += b->p ? b->cap : 0;
    *bytes = t;
    return NEP_OK;
}

int nep_host_alloc(size_t bytes, void** out)
{
    if (!out) return fail(NEP_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (bytes == 0) return fail(NEP_ERR_ARG, "zero bytes");
    cudaError_t e = cudaMallocHost(out, bytes);
    if (e != cudaSuccess) return fail(NEP_ERR_OOM, std::string("cudaMallocHost: ") + cudaGetErrorString(e));
    return NEP_OK;
}

int nep_host_free(void* p)
{
    if (!p) return NEP_OK;
    cudaError_t e = cudaFreeHost(p);
    if (e != cudaSuccess) return fail(NEP_ERR_CUDA, std::string("cudaFreeHost: ") + cudaGetErrorString(e));
    return NEP_OK;
}

int nep_set_capacity(nep_model* m, int radial, int angular)
{
    if (!m || radial < 1 || angular < 1) return fail(NEP_ERR_ARG, "bad capacity");
    m->mnR = (radial + 7) & ~7;
    m->mnA = (angular + 7) & ~7;
    m->n_lists = 0;
    m->graph.reset();
    return NEP_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// nep_compute_static: nep_compute without any device allocation.
//
// Some callers cannot let a library call cudaMalloc or cudaFree: cudaFree (and,
// when the pool has to grow, cudaMalloc) synchronises the whole device, an
// allocation can fail in the middle of a long simulation when another part of the
// program holds the memory, and hosts that account for every byte of device
// memory (an MD engine with a fixed budget, a serving process sized at start-up)
// forbid hidden allocations.  For them this entry point takes its scratch from
// one fixed array in device global memory that is part of the library image.
// The array costs kStaticScratchBytes on every GPU that loads the library, until
// the process exits.
// ---------------------------------------------------------------------------
#include <mutex>

namespace {

constexpr int kStaticMaxN = 4096;        // particles per call
constexpr int kStaticMaxCells = 32768;   // cells of the call's grid
constexpr int kStaticMNR = 256;          // radial neighbours per particle
constexpr int kStaticMNA = 128;          // angular neighbours per particle
constexpr int kStaticMaxNA = phi_pad(5);  // padded n_A of the compiled shapes
constexpr int kStaticMaxT = 4;           // particle types of the model
constexpr int kStaticMaxKRP = 12;        // padded K_R
constexpr int kStaticMaxItems = (kStaticMaxN + kBlock - 1) / kBlock;
static_assert(kStaticMaxItems <= kGroup, "the static path's totals use one item group");
constexpr size_t kStaticTableBytes = 2048;  // one request, its work items, one model
constexpr int kStaticMaxDevices = 64;
// the counts, the request, its work items and one model table must fit the table region
static_assert(align16(sizeof(PlanCounts)) + align16(sizeof(ReqInfo)) + align16(sizeof(WorkItem) * kStaticMaxItems) +
                      sizeof(ModelDesc<double>) <= kStaticTableBytes,
              "static table region too small for the counts, the request, its work items and the model table");

constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Byte layout of the scratch for n particles, ncell cells, real of rs bytes.
struct StaticLayout {
    size_t cell_of, rec_user, perm_tmp, perm, rec_s, cell_s, cntR, cntA, U, e, phi, force;
    size_t nlR, nlA, cell_count, cell_local, block_off, cell_fill, cell_start;
    size_t partial, counters, totals, flags, tables, acc, end;
};

constexpr StaticLayout static_layout(size_t n, size_t ncell, size_t rs, size_t nA, size_t ekrp)
{
    StaticLayout L{};
    size_t p = 0;
    L.cell_of = p; p = align256(p + 4 * n);
    L.rec_user = p; p = align256(p + 4 * rs * n);
    L.perm_tmp = p; p = align256(p + 4 * n);
    L.perm = p; p = align256(p + 4 * n);
    L.rec_s = p; p = align256(p + 4 * rs * n);
    L.cell_s = p; p = align256(p + 4 * n);
    L.cntR = p; p = align256(p + 4 * n);
    L.cntA = p; p = align256(p + 4 * n);
    L.U = p; p = align256(p + rs * n);
    L.e = p; p = align256(p + rs * ekrp * n);
    L.phi = p; p = align256(p + rs * kPsiComp * nA * n);
    L.force = p; p = align256(p + 8 * 3 * n);
    L.nlR = p; p = align256(p + 4 * (size_t)kStaticMNR * n);
    L.nlA = p; p = align256(p + 4 * (size_t)kStaticMNA * n);
    L.cell_count = p; p = align256(p + 4 * ncell);
    L.cell_local = p; p = align256(p + 4 * ncell);
    L.block_off = p; p = align256(p + 4 * (kScanItems + 1));
    L.cell_fill = p; p = align256(p + 4 * ncell);
    L.cell_start = p; p = align256(p + 4 * (ncell + 1));
    L.partial = p; p = align256(p + 8 * 10 * ((n + kBlock - 1) / kBlock));
    L.counters = p; p = align256(p + 16);
    L.totals = p; p = align256(p + 8 * 10);
    L.flags = p; p = align256(p + 16);
    L.tables = p; p = align256(p + kStaticTableBytes);
    L.acc = p; p = align256(p + (rs == 4 ? (32 + 96 + 36) * n : 0));  // FP32 force / virial lines, virial sums
    L.end = p;
    return L;
}

// worst case: FP64, the largest compiled n_A, every limit at its maximum
constexpr size_t kStaticScratchBytes =
    align256(static_layout(kStaticMaxN, kStaticMaxCells, 8, kStaticMaxNA, kStaticMaxT * kStaticMaxKRP).end);

// The scratch.  In host code this name is only a stand-in for the device symbol;
// its device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_static_mutex;
void* g_static_ptr[kStaticMaxDevices] = {};

// Device address of the scratch on `device` (current device); resolved once per device.
int static_scratch(int device, unsigned char** out)
{
    if (device < 0 || device >= kStaticMaxDevices) return fail(NEP_ERR_ARG, "device index too large");
    std::lock_guard<std::mutex> lock(g_static_mutex);
    if (!g_static_ptr[device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || !p)
            return fail(NEP_ERR_CUDA, std::string("cudaGetSymbolAddress(static scratch): ") + cudaGetErrorString(e));
        g_static_ptr[device] = p;
    }
    *out = (unsigned char*)g_static_ptr[device];
    return NEP_OK;
}

template <typename real>
int compute_static_impl(nep_model* m, int n, const int32_t* types, const double* pos, const CellGrid& g,
                        double* energy_total, double* virial_total, double* site_energy, double* force,
                        double* virial)
{
    unsigned char* base = nullptr;
    NEP_TRY(static_scratch(m->device, &base));
    const StaticLayout L = static_layout(n, g.ncell, sizeof(real), phi_pad(m->nA), (size_t)m->T * m->KRP);
    if (L.end > kStaticScratchBytes) return fail(NEP_ERR_ARG, "static scratch too small for this call");
    // the request, its work items and the model table, staged through the handle's
    // pinned buffer (allocated by nep_create) into the scratch
    ReqInfo rq;
    rq.g = g;
    rq.cell_base = 0;
    rq.begin = 0;
    rq.n = n;
    rq.model = 0;
    rq.item_begin = 0;
    WorkItem items[kStaticMaxItems];
    int n_items = 0;
    for (int b = 0; b < n; b += kBlock) items[n_items++] = WorkItem{0, b, std::min(n, b + kBlock)};
    rq.item_end = n_items;
    const ModelDesc<real> md = model_desc<real>(m);
    const PlanCounts counts{n, n_items, g.ncell, 1};
    const size_t off_rq = align16(sizeof(PlanCounts)), off_items = off_rq + align16(sizeof(ReqInfo)),
                 off_models = off_items + align16(sizeof(WorkItem) * n_items);
    if (m->plan_pending) NEP_CUDA(cudaEventSynchronize(m->ev_plan));
    memcpy(m->h_stage, &counts, sizeof counts);
    memcpy(m->h_stage + off_rq, &rq, sizeof rq);
    memcpy(m->h_stage + off_items, items, sizeof(WorkItem) * n_items);
    memcpy(m->h_stage + off_models, &md, sizeof md);
    unsigned char* tables = base + L.tables;
    NEP_CUDA(cudaMemcpyAsync(tables, m->h_stage, off_models + sizeof md, cudaMemcpyHostToDevice, m->cur));
    NEP_CUDA(cudaEventRecord(m->ev_plan, m->cur));
    m->plan_pending = true;
    const PlanCounts* d_cnt = (const PlanCounts*)tables;
    const ReqInfo* d_rq = (const ReqInfo*)(tables + off_rq);
    const WorkItem* d_it = (const WorkItem*)(tables + off_items);
    const ModelDesc<real>* d_md = (const ModelDesc<real>*)(tables + off_models);

    int* flags = (int*)(base + L.flags);
    unsigned int* counters = (unsigned int*)(base + L.counters);
    double* totals = (double*)(base + L.totals);
    // what must start at zero: the overflow/error words and the last-block counter
    // (the cell counters are cleared by the cell build itself)
    NEP_CUDA(cudaMemsetAsync(flags, 0, 16, m->cur));
    NEP_CUDA(cudaMemsetAsync(counters, 0, 16, m->cur));
    // the scratch's regions move with n, so the cell counters are cleared here
    cudaError_t e = launch_cell_build<real>(
        d_cnt, n, n_items, g.ncell, true, false, d_it, d_rq, d_md, pos, types, (int*)(base + L.cell_of),
        (PosRec<real>*)(base + L.rec_user), (int*)(base + L.cell_count), (int*)(base + L.cell_local),
        (int*)(base + L.block_off), (int*)(base + L.cell_fill), (int*)(base + L.perm_tmp), (int*)(base + L.perm),
        (int*)(base + L.cell_start), (int*)(base + L.cell_s), (PosRec<real>*)(base + L.rec_s), flags + 2, m->cur);
    if (e != cudaSuccess) return fail(NEP_ERR_CUDA, std::string("cell build: ") + cudaGetErrorString(e));
    NeighborArgs<real> na;
    na.n = n;
    na.mnR = kStaticMNR;
    na.mnA = kStaticMNA;
    na.counts = d_cnt;
    na.items = d_it;
    na.reqs = d_rq;
    na.models = d_md;
    na.cell_start = (int*)(base + L.cell_start);
    na.cell_s = (int*)(base + L.cell_s);
    na.rec = (PosRec<real>*)(base + L.rec_s);
    na.nlR = (uint32_t*)(base + L.nlR);
    na.nlA = (uint32_t*)(base + L.nlA);
    na.cntR = (int*)(base + L.cntR);
    na.cntA = (int*)(base + L.cntA);
    na.maxcnt = flags;
    na.accF = sizeof(real) == 4 ? acc_force(base + L.acc) : nullptr;
    na.accW = sizeof(real) == 4 && virial ? acc_virial(base + L.acc, n) : nullptr;
    e = launch_neighbors<real>(na, n_items, neighbor_smem<real>(m->T), m->cur);
    if (e != cudaSuccess) return fail(NEP_ERR_CUDA, std::string("neighbours: ") + cudaGetErrorString(e));
    EvalArgs<real> a;
    a.n = n;
    a.mnR = kStaticMNR;
    a.mnA = kStaticMNA;
    a.counts = d_cnt;
    a.items = d_it;
    a.reqs = d_rq;
    a.models = d_md;
    a.rec = na.rec;
    a.nlR = na.nlR;
    a.nlA = na.nlA;
    a.cntR = na.cntR;
    a.cntA = na.cntA;
    a.U = (real*)(base + L.U);
    a.e = (real*)(base + L.e);
    a.e_stride = m->T * m->KRP;
    a.phi = (real*)(base + L.phi);
    a.net_bf16 = m->precision == NEP_FP32_BF16;
    a.many_body = m->MBT;
    a.perm = (int*)(base + L.perm);
    a.force = force ? force : (double*)(base + L.force);
    a.virial = virial;
    a.site = site_energy;
    a.accF = sizeof(real) == 4 ? acc_force(base + L.acc) : nullptr;
    a.accW = sizeof(real) == 4 ? acc_virial(base + L.acc, n) : nullptr;
    a.wsum = sizeof(real) == 4 ? acc_wsum(base + L.acc, n) : nullptr;
    a.partial = (double*)(base + L.partial);
    a.counter = counters;
    a.gcounter = counters + 1;  // one group: at most kStaticMaxN / 128 <= 32 work items
    a.err = flags + 2;
    a.totals = totals;
    e = launch_evaluate<real>(m->nR, m->nA, m->KR, m->KA, a, n_items, m->smem_desc, m->smem_force, m->cur, nullptr,
                              m->mb_desc, m->mb_force, m->ch_force);
    if (e != cudaSuccess) return fail(NEP_ERR_CUDA, std::string("evaluate: ") + cudaGetErrorString(e));
    if (energy_total) NEP_CUDA(cudaMemcpyAsync(energy_total, totals, sizeof(double), cudaMemcpyDeviceToDevice, m->cur));
    if (virial_total)
        NEP_CUDA(cudaMemcpyAsync(virial_total, totals + 1, 9 * sizeof(double), cudaMemcpyDeviceToDevice, m->cur));
    // the handle's pinned status buffer (allocated by nep_create) receives the words
    NEP_CUDA(cudaMemcpyAsync(m->h_flags, flags, 3 * sizeof(int), cudaMemcpyDeviceToHost, m->cur));
    NEP_CUDA(cudaStreamSynchronize(m->cur));
    NEP_TRY(status_error(m->h_flags[2]));
    if (m->h_flags[0] > kStaticMNR || m->h_flags[1] > kStaticMNA)
        return fail(NEP_ERR_NEIGHBOR_OVERFLOW, "more neighbours than the static lists hold (256 radial, 128 angular)");
    return NEP_OK;
}

}  // namespace

extern "C" int nep_compute_static(nep_model* m, int n, const int32_t* types, const double* pos, const double box[3],
                                  const int32_t pbc[3], void* stream, double* energy_total, double* virial_total,
                                  double* site_energy, double* force, double* virial)
{
    if (!m) return fail(NEP_ERR_ARG, "null model");
    if (n < 1 || n > kStaticMaxN)
        return fail(NEP_ERR_ARG, "nep_compute_static: n must be in [1, 4096] (static scratch limit)");
    if (m->T > kStaticMaxT) return fail(NEP_ERR_ARG, "nep_compute_static: models of at most 4 types");
    if (!types || !pos || !box || !pbc) return fail(NEP_ERR_ARG, "null input array");
    CellGrid g;
    NEP_TRY(make_grid(m, box, pbc, g));
    if (g.ncell > kStaticMaxCells)
        return fail(NEP_ERR_ARG, "nep_compute_static: cell grid exceeds 32768 cells (static scratch limit)");
    Guard guard(m->device);
    m->cur = stream ? (cudaStream_t)stream : m->st;
    if (!stream) {
        NEP_CUDA(cudaEventRecord(m->ev_in, (cudaStream_t)0));
        NEP_CUDA(cudaStreamWaitEvent(m->st, m->ev_in, 0));
    }
    int rc = m->precision == NEP_FP64
                 ? compute_static_impl<double>(m, n, types, pos, g, energy_total, virial_total, site_energy, force,
                                               virial)
                 : compute_static_impl<float>(m, n, types, pos, g, energy_total, virial_total, site_energy, force,
                                              virial);
    if (!stream) {
        NEP_CUDA(cudaEventRecord(m->ev_out, m->st));
        NEP_CUDA(cudaStreamWaitEvent((cudaStream_t)0, m->ev_out, 0));
    }
    return rc;
}
