// crm_api.cu -- host side of the C ABI declared in include/crm.h.
//
// The handle keeps the inputs on the host until the first step, then
// "commits": sizes the grid, allocates the device arrays and uploads the
// particles.  Each step enqueues the kernels of Alg. 2 / Alg. 3 on the
// handle's stream: a rebuild every ps_freq steps (in active-domain runs the
// rebuild first refreshes the activity flags and regathers the working set),
// then the two RK2 stages.
//
// Without active boxes the working set is every particle and nothing is
// synchronised inside crm_step.  With active boxes the working-set size is
// decided on the device; when it outgrows a capacity the step is abandoned on
// the device (an abort word every later kernel checks), and the host, which
// runs the steps in chunks of at most S_I steps, grows the arrays by G and
// resumes from that step.  Every S_I steps it shrinks them to the current size
// when they are less than S full (ManageArrayMemory, Sec. 3.2).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "crm_adjoint.cuh"
#include "crm_internal.cuh"

using namespace crm;

namespace {
enum { G_STATIC, G_WORK, G_WIN, G_CAND, G_ADJ, G_TAPE, G_COUNT };
// device counters word layout
enum { C_NF, C_NM, C_N, C_NA, C_NE, C_NEED_F, C_NEED_M, C_NEED_CELLS, C_NEED_CAND, C_USE_CELLS,
       C_USE_CAND, C_WORDS = 16 };
}  // namespace

struct crm_terrain {
    crm_params P{};
    cudaStream_t st = nullptr;
    std::string msg;

    // inputs, insertion order
    std::vector<double> hx, hu, hs, hr;          // SPH
    std::vector<double> hmloc;                   // marker body-frame / world coordinates
    std::vector<int> hmbody;                     // body of each marker, -1 fixed
    std::vector<BodyDev> hbodies;
    std::vector<int> box_body_h;
    std::vector<double> box_half_h, box_off_h;
    double t_delay = 0.0;

    bool committed = false;
    bool lists_valid = false;
    bool frozen = false;          // a device wait gave up: no stepping until crm_load_state
    bool active = false;          // any active box
    bool have_working = false;    // working set holds state not yet written back
    bool boxes_in_force = false;  // the last active step was after t_delay
    int64_t step_index = 0;
    double time = 0.0;
    int64_t nFtot = 0, nMtot = 0;
    DevParams dp{};

    // capacities
    int64_t capF = 0, capM = 0, Mcap = 0, cand_cap = 0;

    // device state: working set
    int cur = 0;
    StageArrays A[2]{}, MID{};
    uint32_t *pid[2]{};
    SortScratch ss{};
    uint32_t *start = nullptr, *nbr = nullptr, *nnb = nullptr;
    float4 *mforce = nullptr;
    double *partial = nullptr;   // FP64 wrench partials [block][body][6]
    // CUDA graphs of whole steps (runs without active boxes, timing off)
    struct StepGraph {
        cudaGraphExec_t exec = nullptr;
        double dt = 0.0;
    };
    // a step with / without the Alg. 2 rebuild, one per current buffer (a graph
    // bakes in the buffer pointers; a search without a skin swaps the buffers)
    StepGraph g_search[2], g_plain[2];
    // the same steps with the co-simulation exchange (crm_cosim_step) inside the
    // graph: the bodies' new motion from pinned staging before, their state and
    // the error word back to it after
    StepGraph x_search[2], x_plain[2];
    unsigned long long *step_ctr = nullptr;   // active domains: device step index (abort tag)
    void drop_graphs()
    {
        for (int b = 0; b < 2; ++b) {
            for (StepGraph *G : {&g_search[b], &g_plain[b], &x_search[b], &x_plain[b]}) {
                if (G->exec) cudaGraphExecDestroy(G->exec);
                G->exec = nullptr;
            }
        }
    }
    cudaStream_t cap_st = nullptr;   // private stream the graphs are captured on
    bool graphs = true;
    // Verlet skin (non-active runs with skin > 0)
    bool skin_on = false;
    int tile_log2[3] = {0, 0, 0};   // cell tiles of the sort order (crm_set_cell_tile)
    int abs32 = 0;                  // test-only absolute FP32 positions (crm_debug_absolute_fp32)
    uint32_t *sk_nbr = nullptr, *sk_nnb = nullptr;
    float4 *xref = nullptr;
    int *gate = nullptr;
    int64_t searches_at_reset = 0, searched = 0;
    // static
    double *mloc = nullptr;
    BodyDev *bodies = nullptr;
    BodyFrame *mid_frames = nullptr;             // bodies at the step midpoint
    uint32_t *act = nullptr, *act_body = nullptr;   // markers with fluid in reach (all, on bodies)
    uint32_t *act_bcount = nullptr;
    int *n_act = nullptr;                          // [2]: sizes of act, act_body
    cudaStream_t side = nullptr;                   // the wrench pass beside pair stage 2
    // the checkpointed backward: the reverse sweep runs on its own stream while
    // the handle's stream re-runs the previous segment (events: re-run done and
    // sweep done, per tape set)
    cudaStream_t adj_st = nullptr;
    cudaEvent_t adj_ev[4] = {nullptr, nullptr, nullptr, nullptr};
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    int *err = nullptr, *counts = nullptr, *win = nullptr, *abort_flag = nullptr;
    int *h_counts = nullptr;      // pinned mirror: counters + abort word
    BodyDev *h_xbodies = nullptr; // pinned staging of the co-simulation exchange: the
                                  // bodies, then one int (the error word)
    // active domains: master store and candidates
    StageArrays Mst{};
    uint32_t *mpid = nullptr, *mslot_of_pid = nullptr;
    int *mcol = nullptr, *colF = nullptr, *colM = nullptr, *fixed_order = nullptr,
        *body_markers = nullptr, *drift = nullptr;
    int n_fixed = 0, n_bodym = 0;
    int *box_body = nullptr;
    double *box_half = nullptr, *box_off = nullptr;
    void *frames = nullptr;
    int *ranges = nullptr, *rinfo = nullptr;
    uint32_t *cinc = nullptr, *cslot = nullptr;
    uint8_t *ckind = nullptr;
    SortScratch cscan{};

    // reverse sweep (crm_eval_rates_vjp, crm_adjoint_*): workspace sized for the
    // working set, and the tape of one checkpoint segment
    struct AdjTape {
        StageArrays Y0, YM;          // slot arrays at y_n and y_mid (markers with their state)
        uint32_t *pid, *nbr, *nnb;   // slot order and lists of the step
        uint32_t *act, *act_body;    // the step's markers with fluid in reach (all, on bodies)
        int *n_act;                  // [2]: their counts
        BodyDev *bodies;             // bodies before the step
        BodyFrame *frames;           // bodies at the step midpoint
        BodyDev *after;              // bodies after the step (its wrench, the updated rates)
        float *sum0, *sumM;          // fluid pair sums of the two stages ([13][capF])
        cudaGraphExec_t rec[2];      // the recording step as a graph, per current buffer
        double rec_dt;
    };
    struct Adjoint {
        bool ready = false;
        float4 *coef = nullptr, *coefB = nullptr;
        float *l_mid = nullptr, *l_y0 = nullptr, *l_ins = nullptr, *l_rate = nullptr,
              *l_macc = nullptr, *sums = nullptr;
        double *gpar = nullptr, *gbody = nullptr, *lb[2]{}, *lwrench = nullptr;
        // trajectory: checkpoints every `every` steps (plus the final state),
        // the bodies after each step, the objective's adjoints
        int64_t n_steps = 0;
        int every = 0, n_ckpt = 0;
        int64_t alloc_steps = -1;     // shape the tape and checkpoints were allocated for
        int alloc_every = -1;
        double dt = 0.0;
        size_t ckpt_bytes = 0;
        char *ckpt = nullptr;
        BodyDev *hist = nullptr;
        double *lw_obj = nullptr, *lc_obj = nullptr;
        // checkpointed runs: two tape sets of one segment each (a re-run fills one
        // while the sweep reads the other); the step index and time of each
        // checkpoint, for the stream-ordered restore
        std::vector<AdjTape> tape;
        std::vector<std::pair<int64_t, double>> ckpt_at;
    } adj;

    std::vector<void *> allocs[G_COUNT];
    bool oom = false;

    // measurement: launch counters and optional per-launch CUDA events
    crm_profile prof{};
    bool timing = false;
    std::vector<cudaEvent_t> ev_pool;
    struct Timed { int k; cudaEvent_t a, b; };
    std::vector<Timed> pending;

    int fail(int code, const std::string &m)
    {
        msg = m;
        return code;
    }
    template <class T> T *dalloc(int group, size_t count)
    {
        void *p = nullptr;
        if (cudaMalloc(&p, std::max<size_t>(count, 1) * sizeof(T)) != cudaSuccess) {
            cudaGetLastError();
            oom = true;
            return nullptr;
        }
        allocs[group].push_back(p);
        return (T *)p;
    }
    void free_group(int group)
    {
        for (void *p : allocs[group])
            if (p) cudaFree(p);
        allocs[group].clear();
    }
};

namespace {

int cuda_fail(crm_terrain *t, cudaError_t e, const char *where)
{
    return t->fail(CRM_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CRM_CUDA(t, call)                                       \
    do {                                                        \
        cudaError_t e_ = (call);                                \
        if (e_ != cudaSuccess) return cuda_fail((t), e_, #call); \
    } while (0)

bool finite_all(const double *a, size_t n)
{
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(a[i])) return false;
    return true;
}

int validate(const crm_params *p, std::string &why)
{
    auto bad = [&](const char *m) { why = m; return CRM_EINVAL; };
    if (!(p->rho0 > 0)) return bad("rho0 must be > 0");
    if (!(p->E > 0)) return bad("E must be > 0");
    if (!(p->nu > -1.0 && p->nu < 0.5)) return bad("nu must lie in (-1, 0.5)");
    if (!(p->mu_s >= 0) || !(p->mu_2 >= 0)) return bad("mu_s, mu_2 must be >= 0");
    if (!(p->cohesion >= 0)) return bad("cohesion must be >= 0");
    if (!(p->I0 > 0) || !(p->grain_d > 0)) return bad("I0, grain_d must be > 0");
    if (!(p->d0 > 0) || !(p->h > 0)) return bad("d0, h must be > 0");
    if (p->kernel != CRM_KERNEL_CUBIC && p->kernel != CRM_KERNEL_WENDLAND)
        return bad("kernel must be CRM_KERNEL_CUBIC or CRM_KERNEL_WENDLAND");
    if (p->av_mode < 0 || p->av_mode > 2) return bad("av_mode must be 0, 1 or 2");
    if (!(p->av_gamma >= 0) || !(p->av_xi2_over_h2 > 0)) return bad("av_gamma >= 0, av_xi2_over_h2 > 0");
    if (!finite_all(p->gravity, 3)) return bad("gravity must be finite");
    if (p->ps_freq < 1) return bad("ps_freq must be >= 1");
    if (p->max_neighbors < 8 || p->max_neighbors > 1024) return bad("max_neighbors must lie in [8, 1024]");
    for (int k = 0; k < 3; ++k)
        if (!std::isfinite(p->domain_min[k]) || !std::isfinite(p->domain_max[k])
            || !(p->domain_max[k] > p->domain_min[k]))
            return bad("domain_max must exceed domain_min on every axis");
    if (!(p->growth >= 1.0) || !(p->shrink_ratio > 0 && p->shrink_ratio <= 1.0) || p->shrink_interval < 1)
        return bad("growth >= 1, shrink_ratio in (0, 1], shrink_interval >= 1");
    if (p->pair_lanes < 0 || p->pair_lanes > 4 || p->pair_lanes == 3)
        return bad("pair_lanes must be 0, 1, 2 or 4");
    if (!(p->skin >= 0.0 && p->skin < 1.0)) return bad("skin must lie in [0, 1)");
    return CRM_OK;
}

// Grid and device constants (cells of size 2h over the domain, Sec. 3.1).
int make_devparams(crm_terrain *t)
{
    const crm_params &P = t->P;
    DevParams &d = t->dp;
    const double skin = t->skin_on ? P.skin : 0.0;
    // cells of 2h (1 + skin), rounded up to an FP32 value: the kernels shift
    // offsets by whole cells in FP32, so that shift and the FP64 grid agree exactly
    const double cell_req = 2.0 * P.h * (1.0 + skin);
    float cell_f = (float)cell_req;
    if ((double)cell_f < cell_req) cell_f = std::nextafter(cell_f, INFINITY);
    const double cell = (double)cell_f;
    int64_t G[3];
    for (int k = 0; k < 3; ++k) {
        G[k] = (int64_t)std::ceil((P.domain_max[k] - P.domain_min[k]) / cell);
        if (G[k] < 1) G[k] = 1;
    }
    if ((double)G[0] * (double)G[1] * (double)G[2] >= 4294967295.0)
        return t->fail(CRM_EINVAL, "grid of 2h cells over the domain exceeds 2^32 cells");
    const double pi = 3.14159265358979323846;
    const double Gm = P.E / (2.0 * (1.0 + P.nu)), Km = P.E / (3.0 * (1.0 - 2.0 * P.nu));
    const double m = P.rho0 * P.d0 * P.d0 * P.d0;
    d.h = (float)P.h;
    d.inv_h = (float)(1.0 / P.h);
    d.four_h2 = (float)(4.0 * P.h * P.h);
    d.cell = (float)cell;
    d.kernel = P.kernel;
    if (P.kernel == CRM_KERNEL_WENDLAND) {
        const double a = 21.0 / (16.0 * pi * P.h * P.h * P.h);
        d.kw = (float)a;
        d.kdw = (float)(-5.0 * a / (P.h * P.h));   // (dW/dr) / r = kdw (1 - q/2)^3
    } else {
        d.kw = (float)(1.0 / (pi * P.h * P.h * P.h));
        d.kdw = (float)(1.0 / (pi * P.h * P.h * P.h * P.h));
    }
    d.m = (float)m;
    d.rho0 = (float)P.rho0;
    d.G = (float)Gm;
    d.K = (float)Km;
    d.av_c = (float)(P.av_gamma * P.h * std::sqrt(Km / P.rho0) * m);
    d.xi2 = (float)(P.av_xi2_over_h2 * P.h * P.h);
    d.av_mode = P.av_mode;
    d.gx = (float)P.gravity[0];
    d.gy = (float)P.gravity[1];
    d.gz = (float)P.gravity[2];
    for (int k = 0; k < 3; ++k) d.g64[k] = P.gravity[k];
    d.mu_s = (float)P.mu_s;
    d.mu_2 = (float)P.mu_2;
    d.I0 = (float)P.I0;
    d.grain_d = (float)P.grain_d;
    d.cohesion = (float)P.cohesion;
    d.GX = (int)G[0]; d.GY = (int)G[1]; d.GZ = (int)G[2];
    d.dmin_x = P.domain_min[0];
    d.dmin_y = P.domain_min[1];
    d.dmin_z = P.domain_min[2];
    d.cell_d = cell;
    d.pair_lanes = P.pair_lanes;
    {
        int dev = 0, nsm = 0;
        if (cudaGetDevice(&dev) != cudaSuccess
            || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess
            || nsm < 1) {
            cudaGetLastError();
            nsm = 148;
        }
        d.n_sm = nsm;
    }
    d.abs32 = t->abs32;
    d.act_skin = t->active && t->skin_on ? 1 : 0;
    // the gathered working set reaches a margin beyond the grown boxes; the skin
    // test also calls for a new gather once a point of a grown box may have moved
    // 0.95 of it (a margin of four times the particles' displacement bound: the
    // boxes of turning wheels reach far from their centres)
    d.act_margin = d.act_skin ? 4.0 * P.h * skin : 0.0;
    d.box_thr2 = (float)(0.95 * d.act_margin * 0.95 * d.act_margin);
    d.tbx = t->tile_log2[0];
    d.tby = t->tile_log2[1];
    d.tbz = t->tile_log2[2];
    d.maxnb = P.max_neighbors;
    d.sk_r2 = (float)(cell * cell);
    d.disp_thr2 = (float)(0.95 * skin * P.h * 0.95 * skin * P.h);
    const double grow3 = (1.0 + skin) * (1.0 + skin) * (1.0 + skin);
    d.skin_cap = (int)std::ceil(P.max_neighbors * grow3 * 1.05) + 8;
    d.gate = nullptr;
    return CRM_OK;
}

bool inside_domain(const crm_params &P, const double *x)
{
    for (int k = 0; k < 3; ++k)
        if (!(x[k] >= P.domain_min[k] && x[k] < P.domain_max[k])) return false;
    return true;
}

void cell_of(const DevParams &d, const double *x, int c[3], float o[3])
{
    const double dm[3] = {d.dmin_x, d.dmin_y, d.dmin_z};
    for (int k = 0; k < 3; ++k) {
        c[k] = (int)std::floor((x[k] - dm[k]) / d.cell_d);
        o[k] = (float)(x[k] - (dm[k] + c[k] * d.cell_d));
    }
}

float cell_bits(const DevParams &d, const int c[3])
{
    const uint32_t g = ((uint32_t)c[2] * (uint32_t)d.GY + (uint32_t)c[1]) * (uint32_t)d.GX
                       + (uint32_t)c[0];
    float f;
    std::memcpy(&f, &g, 4);
    return f;
}

int latched_error(crm_terrain *t)
{
    int e = 0;
    CRM_CUDA(t, cudaMemcpyAsync(&e, t->err, sizeof(int), cudaMemcpyDeviceToHost, t->st));
    CRM_CUDA(t, cudaStreamSynchronize(t->st));
    if (e == 0) return CRM_OK;
    CRM_CUDA(t, cudaMemsetAsync(t->err, 0, sizeof(int), t->st));
    if (e & ERR_TIMEOUT) t->frozen = true;   // its kernels return at once (abort word)
    if (e & ERR_NONFINITE) return t->fail(CRM_ENONFINITE, "the particle state became non-finite");
    if (e & ERR_ESCAPED) return t->fail(CRM_EESCAPED, "a particle or marker left the grid domain");
    if (e & ERR_CAPACITY)
        return t->fail(CRM_ECAPACITY, "a neighbour list exceeded max_neighbors");
    return t->fail(CRM_ETIMEOUT, "a bounded device-side wait gave up");
}

// Free the adjoint's tape (and the recording graphs that point into it).
void drop_tape(crm_terrain *t)
{
    for (crm_terrain::AdjTape &T : t->adj.tape)
        for (cudaGraphExec_t &g : T.rec)
            if (g) {
                cudaGraphExecDestroy(g);
                g = nullptr;
            }
    t->adj.tape.clear();
    t->free_group(G_TAPE);
}

// Working-set arrays for capF fluid + capM marker slots.
int alloc_working(crm_terrain *t)
{
    t->drop_graphs();   // graphs bake in the array pointers
    t->free_group(G_WORK);
    drop_tape(t);              // the sweep's workspace follows the working set
    t->free_group(G_ADJ);
    t->adj = crm_terrain::Adjoint{};
    DevParams &d = t->dp;
    const int64_t N = t->capF + t->capM;
    if (N >= (int64_t)kIndexMask)
        return t->fail(CRM_EINVAL, "working set beyond the 2^26 slots a neighbour entry addresses");
    d.capF = (int)t->capF;
    d.capM = (int)t->capM;
    d.capN = (int)N;
    d.ell = (uint32_t)std::max<int64_t>(N, 1);
    for (int b = 0; b < 2; ++b) {
        t->A[b].pos = t->dalloc<float4>(G_WORK, N);
        t->A[b].vel = t->dalloc<float4>(G_WORK, N);
        t->A[b].sA = t->dalloc<float4>(G_WORK, N);
        t->A[b].sB = t->dalloc<float2>(G_WORK, N);
        t->pid[b] = t->dalloc<uint32_t>(G_WORK, N);
    }
    t->MID.pos = t->dalloc<float4>(G_WORK, N);
    t->MID.vel = t->dalloc<float4>(G_WORK, N);
    t->MID.sA = t->dalloc<float4>(G_WORK, N);
    t->MID.sB = t->dalloc<float2>(G_WORK, N);
    t->ss.keys = t->dalloc<uint32_t>(G_WORK, N);
    t->ss.rank = t->dalloc<uint32_t>(G_WORK, N);
    t->ss.tmp = t->dalloc<uint32_t>(G_WORK, N);
    t->nbr = t->dalloc<uint32_t>(G_WORK, (size_t)d.maxnb * d.ell);
    t->nnb = t->dalloc<uint32_t>(G_WORK, N);
    t->mforce = t->dalloc<float4>(G_WORK, t->capM);
    t->partial = t->dalloc<double>(G_WORK, (size_t)wrench_blocks(t->n_bodym)
                                               * std::max<size_t>(t->hbodies.size(), 1) * 6);
    t->act = t->dalloc<uint32_t>(G_WORK, t->capM);
    t->act_body = t->dalloc<uint32_t>(G_WORK, std::max(t->n_bodym, 1));
    t->act_bcount = t->dalloc<uint32_t>(G_WORK, 2 * (size_t)compact_blocks(d));
    t->n_act = t->dalloc<int>(G_WORK, 2);
    if (t->skin_on) {
        t->sk_nbr = t->dalloc<uint32_t>(G_WORK, (size_t)d.skin_cap * d.ell);
        t->sk_nnb = t->dalloc<uint32_t>(G_WORK, N);
        t->xref = t->dalloc<float4>(G_WORK, N);
    }
    if (t->oom) return t->fail(CRM_ENOMEM, "device allocation of the working set failed");
    if (t->skin_on) {
        CRM_CUDA(t, cudaMemsetAsync(t->sk_nnb, 0, N * sizeof(uint32_t), t->st));
        // the first rebuild searches (the count of searches runs on: the launch
        // counters read differences of it)
        const int g0[GATE_SEARCHES] = {1, 0, 1, 0};
        CRM_CUDA(t, cudaMemcpyAsync(t->gate, g0, sizeof(g0), cudaMemcpyHostToDevice, t->st));
        CRM_CUDA(t, cudaStreamSynchronize(t->st));
    }
    CRM_CUDA(t, cudaMemsetAsync(t->nnb, 0, N * sizeof(uint32_t), t->st));
    CRM_CUDA(t, cudaMemsetAsync(t->mforce, 0, std::max<int64_t>(t->capM, 1) * sizeof(float4), t->st));
    CRM_CUDA(t, cudaMemsetAsync(t->n_act, 0, 2 * sizeof(int), t->st));
    t->cur = 0;
    t->lists_valid = false;
    return CRM_OK;
}

// Counting-sort key space: 2 Mcap + 1 cell counters and ranges.
int alloc_window(crm_terrain *t)
{
    t->drop_graphs();
    t->free_group(G_WIN);
    t->dp.M = (uint32_t)t->Mcap;
    const size_t nk = 2 * (size_t)t->Mcap + 1;
    t->ss.count = t->dalloc<uint32_t>(G_WIN, nk);
    t->ss.n_tiles = ((int64_t)nk + kScanTile - 1) / kScanTile;
    t->ss.tile_status = t->dalloc<unsigned long long>(G_WIN, t->ss.n_tiles);
    t->ss.ctr = t->dalloc<uint32_t>(G_WIN, 4);
    t->start = t->dalloc<uint32_t>(G_WIN, nk);
    if (t->oom) return t->fail(CRM_ENOMEM, "device allocation of the cell arrays failed");
    CRM_CUDA(t, cudaMemsetAsync(t->ss.count, 0, nk * sizeof(uint32_t), t->st));
    CRM_CUDA(t, cudaMemsetAsync(t->ss.tile_status, 0, t->ss.n_tiles * sizeof(unsigned long long), t->st));
    CRM_CUDA(t, cudaMemsetAsync(t->ss.ctr, 0, 4 * sizeof(uint32_t), t->st));
    return CRM_OK;
}

// Candidate arrays of the activity pass (active domains).
int alloc_cand(crm_terrain *t)
{
    t->drop_graphs();
    t->free_group(G_CAND);
    const size_t n = (size_t)t->cand_cap + 1;
    t->cinc = t->dalloc<uint32_t>(G_CAND, n);
    t->cslot = t->dalloc<uint32_t>(G_CAND, n);
    t->ckind = t->dalloc<uint8_t>(G_CAND, n);
    t->cscan.n_tiles = ((int64_t)n + kScanTile - 1) / kScanTile;
    t->cscan.tile_status = t->dalloc<unsigned long long>(G_CAND, t->cscan.n_tiles);
    t->cscan.ctr = t->dalloc<uint32_t>(G_CAND, 4);
    if (t->oom) return t->fail(CRM_ENOMEM, "device allocation of the activity arrays failed");
    CRM_CUDA(t, cudaMemsetAsync(t->cinc, 0, n * sizeof(uint32_t), t->st));
    CRM_CUDA(t, cudaMemsetAsync(t->cscan.tile_status, 0, t->cscan.n_tiles * sizeof(unsigned long long), t->st));
    CRM_CUDA(t, cudaMemsetAsync(t->cscan.ctr, 0, 4 * sizeof(uint32_t), t->st));
    return CRM_OK;
}

template <class T> int upload(crm_terrain *t, T *dev, const T *host, size_t n)
{
    if (n == 0) return CRM_OK;
    CRM_CUDA(t, cudaMemcpyAsync(dev, host, n * sizeof(T), cudaMemcpyHostToDevice, t->st));
    return CRM_OK;
}

// Host estimate of the window cells and candidate count of the boxes at the
// bodies' current poses (initial capacities of an active-domain run).
void estimate_active(crm_terrain *t, const std::vector<int> &colF_h, const std::vector<int> &colM_h,
                     int64_t &cells, int64_t &cand, int64_t &fluid)
{
    const DevParams &d = t->dp;
    const int G[3] = {d.GX, d.GY, d.GZ};
    const double dm[3] = {d.dmin_x, d.dmin_y, d.dmin_z};
    int lo[3] = {G[0], G[1], G[2]}, hi[3] = {-1, -1, -1};
    cand = 0;
    fluid = 0;
    for (size_t b = 0; b < t->box_body_h.size(); ++b) {
        const BodyDev &B = t->hbodies[t->box_body_h[b]];
        const double *q = B.pose + 3;
        const double w = q[0], x = q[1], y = q[2], z = q[3];
        const double R[9] = {1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y),
                             2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x),
                             2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)};
        double eg[3], c[3], vol = 1.0;
        for (int k = 0; k < 3; ++k) {
            eg[k] = t->box_half_h[3 * b + k] + 2.0 * t->P.h + d.act_margin;
            vol *= 2.0 * eg[k];
        }
        for (int k = 0; k < 3; ++k)
            c[k] = B.pose[k] + R[3 * k] * t->box_off_h[3 * b] + R[3 * k + 1] * t->box_off_h[3 * b + 1]
                   + R[3 * k + 2] * t->box_off_h[3 * b + 2];
        int xa = 0, xb = -1;
        for (int k = 0; k < 3; ++k) {
            const double ext = std::fabs(R[3 * k]) * eg[0] + std::fabs(R[3 * k + 1]) * eg[1]
                               + std::fabs(R[3 * k + 2]) * eg[2];
            int a = std::max((int)std::floor((c[k] - ext - dm[k]) / d.cell_d) - 1, 0);
            int e = std::min((int)std::floor((c[k] + ext - dm[k]) / d.cell_d) + 1, G[k] - 1);
            lo[k] = std::min(lo[k], a);
            hi[k] = std::max(hi[k], e);
            if (k == 0) { xa = a; xb = e; }
        }
        if (xb >= xa) cand += colF_h[xb + 1] - colF_h[xa] + colM_h[xb + 1] - colM_h[xa];
        fluid += (int64_t)(vol / (t->P.d0 * t->P.d0 * t->P.d0));
    }
    cells = key_cells(std::max(hi[0] - lo[0] + 1, 1), std::max(hi[1] - lo[1] + 1, 1),
                      std::max(hi[2] - lo[2] + 1, 1));
}

int commit(crm_terrain *t)
{
    if (t->committed) return CRM_OK;
    const int64_t nF = t->nFtot, nM = t->nMtot, N = nF + nM;
    if (N >= (int64_t)kPidIndexMask)
        return t->fail(CRM_EINVAL, "more than 2^29 - 1 particles and markers in one terrain");
    for (const BodyDev &b : t->hbodies)
        if ((b.dof & (7 << 3)) && !(b.inertia[0] > 0 && b.inertia[1] > 0 && b.inertia[2] > 0))
            return t->fail(CRM_EINVAL, "a body with free angular DOFs needs crm_set_body_inertia");
    t->active = !t->box_body_h.empty();
    t->skin_on = t->P.skin > 0.0;
    int rc = make_devparams(t);
    if (rc) return rc;
    DevParams &d = t->dp;
    d.n_bodies = (int)t->hbodies.size();
    // id range of each body's markers (one contiguous range per crm_add_rigid_body)
    {
        std::vector<int64_t> lo(d.n_bodies, -1), hi(d.n_bodies, -1);
        for (int64_t a = 0; a < nM; ++a) {
            const int b = t->hmbody[a];
            if (b < 0) continue;
            if (lo[b] < 0) lo[b] = a;
            else if (a != hi[b]) return t->fail(CRM_EINVAL, "body markers not contiguous");
            hi[b] = a + 1;
        }
        for (int b = 0; b < d.n_bodies; ++b) {
            d.body_lo[b] = (uint32_t)(lo[b] < 0 ? 0 : nF + lo[b]);
            d.body_hi[b] = (uint32_t)(lo[b] < 0 ? 0 : nF + hi[b]);
        }
    }
    // largest marker arm of each body, and the reference pose of the skin bound
    for (size_t b = 0; b < t->hbodies.size(); ++b) {
        BodyDev &B = t->hbodies[b];
        B.rmax = 0.0;
        for (int k = 0; k < 7; ++k) B.ref_pose[k] = B.pose[k];
    }
    for (int64_t a = 0; a < nM; ++a) {
        const int b = t->hmbody[a];
        if (b < 0) continue;
        const double *x = &t->hmloc[3 * a];
        t->hbodies[b].rmax = std::max(t->hbodies[b].rmax, std::sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]));
    }
    for (BodyDev &B : t->hbodies) B.box_reach = 0.0;
    if (d.act_skin) {
        // bound on the distance of a grown box's points from the body's centre
        for (size_t k = 0; k < t->box_body_h.size(); ++k) {
            const double *o = &t->box_off_h[3 * k], *e = &t->box_half_h[3 * k];
            double e2 = 0.0;
            for (int a = 0; a < 3; ++a) e2 += (e[a] + 2.0 * t->P.h) * (e[a] + 2.0 * t->P.h);
            const double reach = std::sqrt(o[0] * o[0] + o[1] * o[1] + o[2] * o[2]) + std::sqrt(e2);
            BodyDev &B = t->hbodies[t->box_body_h[k]];
            B.box_reach = std::max(B.box_reach, reach);
        }
    }
    const int64_t full_cells = key_cells(d.GX, d.GY, d.GZ);
    cudaStream_t st = t->st;
    t->n_bodym = (int)std::count_if(t->hmbody.begin(), t->hmbody.end(), [](int b) { return b >= 0; });

    // static device state
    t->mloc = t->dalloc<double>(G_STATIC, 3 * nM);
    // the error word right after the bodies: the co-simulation exchange reads both
    // back with one copy
    t->bodies = t->dalloc<BodyDev>(G_STATIC, t->hbodies.size() + 1);
    t->mid_frames = t->dalloc<BodyFrame>(G_STATIC, kMaxBodies);
    t->err = t->bodies ? reinterpret_cast<int *>(t->bodies + t->hbodies.size()) : nullptr;
    t->counts = t->dalloc<int>(G_STATIC, C_WORDS);
    t->win = t->dalloc<int>(G_STATIC, 8);
    t->abort_flag = t->dalloc<int>(G_STATIC, 1);
    t->gate = t->dalloc<int>(G_STATIC, GATE_WORDS);
    if (t->oom) return t->fail(CRM_ENOMEM, "device allocation failed");
    CRM_CUDA(t, cudaMemsetAsync(t->gate, 0, GATE_WORDS * sizeof(int), t->st));
    if (t->skin_on) d.gate = t->gate;
    if (!t->h_counts && cudaMallocHost(&t->h_counts, (C_WORDS + 2) * sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        t->h_counts = nullptr;
        return t->fail(CRM_ENOMEM, "pinned host allocation failed");
    }
    d.sizes = t->counts;
    d.win = t->win;
    d.abort = t->abort_flag;
    if (!t->side) {
        // side stream of the wrench pass; without it everything stays on the handle's stream
        if (cudaStreamCreateWithFlags(&t->side, cudaStreamNonBlocking) != cudaSuccess
            || cudaEventCreateWithFlags(&t->ev_fork, cudaEventDisableTiming) != cudaSuccess
            || cudaEventCreateWithFlags(&t->ev_join, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            if (t->side) cudaStreamDestroy(t->side);
            if (t->ev_fork) cudaEventDestroy(t->ev_fork);
            t->side = nullptr;
            t->ev_fork = t->ev_join = nullptr;
        }
    }
    CRM_CUDA(t, cudaMemsetAsync(t->err, 0, sizeof(int), st));
    CRM_CUDA(t, cudaMemsetAsync(t->abort_flag, 0, sizeof(int), st));
    CRM_CUDA(t, cudaMemsetAsync(t->counts, 0, C_WORDS * sizeof(int), st));
    if (nM) {
        rc = upload(t, t->mloc, t->hmloc.data(), 3 * nM);
        if (rc) return rc;
    }
    if (!t->hbodies.empty()) {
        rc = upload(t, t->bodies, t->hbodies.data(), t->hbodies.size());
        if (rc) return rc;
    }

    // test-only absolute FP32 layout: the inputs as FP32 coordinates
    if (t->abs32) {
        for (double &v : t->hx) v = (double)(float)v;
        for (int64_t a = 0; a < nM; ++a)
            if (t->hmbody[a] < 0)
                for (int k = 0; k < 3; ++k) t->hmloc[3 * a + k] = (double)(float)t->hmloc[3 * a + k];
    }
    // initial state, converted to cell-relative form on the host
    std::vector<float4> pos(nF), vel(nF), sA(nF);
    std::vector<float2> sB(nF);
    std::vector<int> cx(nF);
    for (int64_t i = 0; i < nF; ++i) {
        int c[3];
        float o[3];
        cell_of(d, &t->hx[3 * i], c, o);
        cx[i] = c[0];
        pos[i] = make_float4(o[0], o[1], o[2], cell_bits(d, c));
        vel[i] = make_float4((float)t->hu[3 * i], (float)t->hu[3 * i + 1], (float)t->hu[3 * i + 2],
                             (float)t->hr[i]);
        const double *s = &t->hs[6 * i];
        sA[i] = make_float4((float)s[0], (float)s[1], (float)s[2], (float)s[3]);
        sB[i] = make_float2((float)s[4], (float)s[5]);
    }

    if (!t->active) {
        // every particle is in the working set for good
        t->capF = nF;
        t->capM = nM;
        t->Mcap = full_cells;
        if (2.0 * (double)t->Mcap + 1.0 >= 2147483647.0)
            return t->fail(CRM_EINVAL, "grid too large for the cell sort (2M + 1 >= 2^31)");
        rc = alloc_working(t);
        if (!rc) rc = alloc_window(t);
        if (rc) return rc;
        std::vector<float4> p4(N), v4(N), a4(N);
        std::vector<float2> b2(N);
        std::vector<uint32_t> pid(N);
        for (int64_t i = 0; i < N; ++i) {
            if (i < nF) {
                p4[i] = pos[i]; v4[i] = vel[i]; a4[i] = sA[i]; b2[i] = sB[i];
            } else {
                p4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
                v4[i] = make_float4(0.f, 0.f, 0.f, (float)t->P.rho0);
                a4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
                b2[i] = make_float2(0.f, 0.f);
            }
            pid[i] = (uint32_t)i;
        }
        const int c = t->cur;
        rc = upload(t, t->A[c].pos, p4.data(), N);
        if (!rc) rc = upload(t, t->A[c].vel, v4.data(), N);
        if (!rc) rc = upload(t, t->A[c].sA, a4.data(), N);
        if (!rc) rc = upload(t, t->A[c].sB, b2.data(), N);
        if (!rc) rc = upload(t, t->pid[c], pid.data(), N);
        if (rc) return rc;
        const int sizes[5] = {(int)nF, (int)nM, (int)N, (int)nF, 0};
        const int win[6] = {0, 0, 0, d.GX, d.GY, d.GZ};
        rc = upload(t, t->counts, sizes, 5);
        if (!rc) rc = upload(t, t->win, win, 6);
        if (rc) return rc;
        CRM_CUDA(t, cudaStreamSynchronize(st));
        if (cudaStreamCreateWithFlags(&t->cap_st, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            t->cap_st = nullptr;   // direct launches only
        }
        t->committed = true;
        return CRM_OK;
    }

    // ---- active domains: master store sorted by cell, x slowest --------------
    std::vector<int64_t> key(nF);
    std::vector<int> order(nF);
    for (int64_t i = 0; i < nF; ++i) {
        int c[3];
        float o[3];
        cell_of(d, &t->hx[3 * i], c, o);
        key[i] = ((int64_t)c[0] * d.GY + c[1]) * d.GZ + c[2];
    }
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return key[a] < key[b]; });
    std::vector<float4> mp(nF), mv(nF), ma(nF);
    std::vector<float2> mb(nF);
    std::vector<uint32_t> mpid(nF), mslot(nF);
    std::vector<int> mcol(nF), colF(d.GX + 1, 0), colM(d.GX + 1, 0);
    for (int64_t m = 0; m < nF; ++m) {
        const int i = order[m];
        mp[m] = pos[i]; mv[m] = vel[i]; ma[m] = sA[i]; mb[m] = sB[i];
        mpid[m] = (uint32_t)i;
        mslot[i] = (uint32_t)m;
        mcol[m] = cx[i];
        colF[cx[i] + 1] += 1;
    }
    for (int x = 0; x < d.GX; ++x) colF[x + 1] += colF[x];
    std::vector<int> fixed, bodym;
    for (int64_t a = 0; a < nM; ++a) {
        if (t->hmbody[a] < 0) fixed.push_back((int)a);
        else bodym.push_back((int)(nF + a));
    }
    std::vector<int64_t> fkey(fixed.size());
    for (size_t k = 0; k < fixed.size(); ++k) {
        int c[3];
        float o[3];
        cell_of(d, &t->hmloc[3 * (size_t)fixed[k]], c, o);
        fkey[k] = ((int64_t)c[0] * d.GY + c[1]) * d.GZ + c[2];
    }
    std::vector<int> forder(fixed.size());
    std::iota(forder.begin(), forder.end(), 0);
    std::stable_sort(forder.begin(), forder.end(), [&](int a, int b) { return fkey[a] < fkey[b]; });
    std::vector<int> fixed_sorted(fixed.size());
    for (size_t k = 0; k < fixed.size(); ++k) {
        fixed_sorted[k] = fixed[forder[k]];
        const int x = (int)(fkey[forder[k]] / ((int64_t)d.GY * d.GZ));
        colM[x + 1] += 1;
    }
    for (int x = 0; x < d.GX; ++x) colM[x + 1] += colM[x];
    t->n_fixed = (int)fixed.size();
    t->n_bodym = (int)bodym.size();

    t->Mst.pos = t->dalloc<float4>(G_STATIC, nF);
    t->Mst.vel = t->dalloc<float4>(G_STATIC, nF);
    t->Mst.sA = t->dalloc<float4>(G_STATIC, nF);
    t->Mst.sB = t->dalloc<float2>(G_STATIC, nF);
    t->mpid = t->dalloc<uint32_t>(G_STATIC, nF);
    t->mslot_of_pid = t->dalloc<uint32_t>(G_STATIC, nF);
    t->mcol = t->dalloc<int>(G_STATIC, nF);
    t->colF = t->dalloc<int>(G_STATIC, d.GX + 1);
    t->colM = t->dalloc<int>(G_STATIC, d.GX + 1);
    t->fixed_order = t->dalloc<int>(G_STATIC, fixed.size());
    t->body_markers = t->dalloc<int>(G_STATIC, bodym.size());
    t->drift = t->dalloc<int>(G_STATIC, 1);
    t->step_ctr = t->dalloc<unsigned long long>(G_STATIC, 1);
    d.step_ctr = t->step_ctr;
    const size_t nbox = t->box_body_h.size();
    t->box_body = t->dalloc<int>(G_STATIC, nbox);
    t->box_half = t->dalloc<double>(G_STATIC, 3 * nbox);
    t->box_off = t->dalloc<double>(G_STATIC, 3 * nbox);
    t->frames = t->dalloc<char>(G_STATIC, box_frame_bytes() * kMaxBodies);
    t->ranges = t->dalloc<int>(G_STATIC, 4 * kMaxBodies + 4);
    t->rinfo = t->dalloc<int>(G_STATIC, 4 * kMaxBodies + 8);
    if (t->oom) return t->fail(CRM_ENOMEM, "device allocation of the master store failed");
    rc = upload(t, t->Mst.pos, mp.data(), nF);
    if (!rc) rc = upload(t, t->Mst.vel, mv.data(), nF);
    if (!rc) rc = upload(t, t->Mst.sA, ma.data(), nF);
    if (!rc) rc = upload(t, t->Mst.sB, mb.data(), nF);
    if (!rc) rc = upload(t, t->mpid, mpid.data(), nF);
    if (!rc) rc = upload(t, t->mslot_of_pid, mslot.data(), nF);
    if (!rc) rc = upload(t, t->mcol, mcol.data(), nF);
    if (!rc) rc = upload(t, t->colF, colF.data(), colF.size());
    if (!rc) rc = upload(t, t->colM, colM.data(), colM.size());
    if (!rc) rc = upload(t, t->fixed_order, fixed_sorted.data(), fixed_sorted.size());
    if (!rc) rc = upload(t, t->body_markers, bodym.data(), bodym.size());
    if (!rc) rc = upload(t, t->box_body, t->box_body_h.data(), nbox);
    if (!rc) rc = upload(t, t->box_half, t->box_half_h.data(), 3 * nbox);
    if (!rc) rc = upload(t, t->box_off, t->box_off_h.data(), 3 * nbox);
    if (rc) return rc;
    CRM_CUDA(t, cudaMemsetAsync(t->drift, 0, sizeof(int), st));

    // initial capacities: everything when the first step is before t_delay
    // (Alg. 3 processes all particles then), else the boxes' estimate
    if (!(0.0 > t->t_delay)) {
        t->capF = std::max<int64_t>(nF, 1);
        t->capM = std::max<int64_t>(nM, 1);
        t->Mcap = full_cells;
        t->cand_cap = std::max<int64_t>(nF + t->n_fixed, 1);
    } else {
        int64_t cells = 0, cand = 0, fl = 0;
        estimate_active(t, colF, colM, cells, cand, fl);
        t->capF = std::max<int64_t>(std::min<int64_t>(nF, (int64_t)(t->P.growth * fl) + 256), 1);
        t->capM = std::max<int64_t>(std::min<int64_t>(nM, t->n_bodym + t->capF), 1);
        t->Mcap = std::min<int64_t>(full_cells, (int64_t)(cells * 1.5) + 64);
        t->cand_cap = std::max<int64_t>((int64_t)(cand * t->P.growth) + 256, 1);
    }
    if (2.0 * (double)t->Mcap + 1.0 >= 2147483647.0)
        return t->fail(CRM_EINVAL, "grid too large for the cell sort (2M + 1 >= 2^31)");
    rc = alloc_working(t);
    if (!rc) rc = alloc_window(t);
    if (!rc) rc = alloc_cand(t);
    if (rc) return rc;
    CRM_CUDA(t, cudaStreamSynchronize(st));
    if (cudaStreamCreateWithFlags(&t->cap_st, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        t->cap_st = nullptr;   // direct launches only
    }
    t->committed = true;
    t->have_working = false;
    return CRM_OK;
}

enum KernelId { K_KEYS, K_SCAN, K_SCATTER, K_REORDER, K_NEIGHBORS, K_COMPACT, K_BCE, K_PAIR1,
                K_PAIR2, K_SKIN, K_EXPORT, K_ADJ };
const char *const kKernelNames[CRM_NUM_KERNELS] = {
    "keys", "scan", "scatter", "reorder", "neighbors", "compact", "bce", "pair_stage1",
    "pair_stage2", "skin", "export", "adjoint"};

// Enqueue one kernel through `launch`, counting it and, when timing is on,
// bracketing it with two events on the handle's stream.  The active-domain
// kernels are counted under "keys" (flags, compaction, gather), "scan" and
// "export" (write-back to the master store).
template <class F> void launch(crm_terrain *t, int k, F &&f, int kernels = 1)
{
    t->prof.launches[k] += kernels;
    if (!t->timing) {
        f();
        return;
    }
    cudaEvent_t ev[2];
    for (int q = 0; q < 2; ++q) {
        if (!t->ev_pool.empty()) {
            ev[q] = t->ev_pool.back();
            t->ev_pool.pop_back();
        } else if (cudaEventCreate(&ev[q]) != cudaSuccess) {
            cudaGetLastError();
            ev[q] = nullptr;
        }
    }
    if (ev[0] && ev[1]) cudaEventRecord(ev[0], t->st);
    f();
    if (ev[0] && ev[1]) {
        cudaEventRecord(ev[1], t->st);
        t->pending.push_back({k, ev[0], ev[1]});
    }
}

// The next rebuild gathers and searches (with the skin, whatever the
// displacement test says): the working set or the lists are gone.
int invalidate_lists(crm_terrain *t)
{
    t->lists_valid = false;
    if (t->committed && t->skin_on)
        CRM_CUDA(t, cudaMemsetAsync(t->gate + GATE_FORCE, 1, sizeof(int), t->st));   // nonzero
    return CRM_OK;
}

// Launch count of a kernel of the gated rebuild: with the skin (and no event
// timing) the searches the decision actually ran are counted at profile_read.
int gated_count(const crm_terrain *t, int gated) { return gated && t->skin_on && !t->timing ? 0 : 1; }

// Write the Active particles of the working set back to the master store.
// gated: as part of a step's rebuild (with the skin, run only when the search
// is due); else unconditionally (before reading the master store).
void scatter_back(crm_terrain *t, int gated = 0)
{
    if (!t->active || !t->have_working) return;
    const int c = t->cur;
    launch(t, K_EXPORT, [&] { launch_scatter_back(t->dp, t->A[c], t->pid[c], t->mslot_of_pid,
                                                  t->mcol, t->Mst, t->drift, gated, t->st); },
           gated_count(t, gated));
}

// Activity flags, counts and the gather of the working set (Alg. 3 items 1-3).
void activity_pass(crm_terrain *t)
{
    const DevParams &d = t->dp;
    const int all = !(t->time > t->t_delay);
    const int c = t->cur;
    scatter_back(t, t->skin_on ? 1 : 0);
    const int nbox = (int)t->box_body_h.size();
    const int n1 = gated_count(t, 1);
    launch(t, K_KEYS, [&] { launch_box_prep(d, nbox, t->box_body, t->box_half, t->box_off,
                                            t->bodies, t->colF, t->colM, t->drift, all,
                                            (int)t->nFtot, t->n_fixed, t->cand_cap, t->frames,
                                            t->win, t->ranges, t->rinfo, t->counts, t->abort_flag,
                                            t->step_index, t->st); }, n1);
    launch(t, K_KEYS, [&] { launch_activity(d, nbox, t->frames, t->ranges, t->rinfo, t->Mst.pos,
                                            t->mloc, t->fixed_order, all, t->cand_cap, t->cinc,
                                            t->ckind, t->counts, t->abort_flag, t->st); }, n1);
    launch(t, K_SCAN, [&] { launch_scan_reset(t->cinc, t->cslot, t->cand_cap + 1, t->cscan, t->err,
                                              t->st, t->skin_on ? t->gate : nullptr,
                                              t->abort_flag); }, n1);
    launch(t, K_KEYS, [&] { launch_active_sizes(d, t->rinfo, t->cslot, t->n_bodym, t->counts,
                                                t->abort_flag, t->step_index, t->st); }, n1);
    launch(t, K_KEYS, [&] { launch_gather(d, t->ranges, t->rinfo, t->ckind, t->cslot, t->Mst,
                                          t->mpid, t->fixed_order, t->body_markers, t->n_bodym,
                                          (int)t->nFtot, t->cand_cap, t->A[c], t->pid[c],
                                          t->counts, t->abort_flag, t->st); }, n1);
    t->have_working = true;
}

// Alg. 2 "PreprocessNeighborList" + Alg. 1.  Without a skin: keys, counting
// sort, reorder into the other buffer, 2h search.  With a skin: a device-side
// decision gates the sort and the skin-radius search (written back into the
// current buffer); the stage-1 kernels then filter the exact lists from the
// skin lists.
void enqueue_search(crm_terrain *t)
{
    const int c = t->cur, n = 1 - c;
    const DevParams &d = t->dp;
    launch(t, K_KEYS, [&] { launch_keys(d, t->A[c], t->pid[c], t->mloc, t->bodies,
                                        t->ss, t->err, (int)t->nFtot, t->st); });
    launch(t, K_SCAN, [&] { launch_scan_reset(t->ss.count, t->start, 2 * (int64_t)d.M + 1, t->ss,
                                              t->err, t->st, d.gate, t->abort_flag); });
    launch(t, K_SCATTER, [&] { launch_scatter(d, t->ss, t->start, t->st); });
    launch(t, K_REORDER, [&] { launch_reorder(d, t->ss, t->start, t->A[c], t->pid[c], t->A[n],
                                              t->pid[n], t->st); });
    if (t->skin_on) {
        launch(t, K_NEIGHBORS, [&] { launch_neighbors(d, t->A[n].pos, t->start, t->sk_nbr,
                                                      t->sk_nnb, d.skin_cap, d.sk_r2, t->err,
                                                      t->st, d.four_h2); });
        launch(t, K_SKIN, [&] { launch_copyback(d, t->A[n], t->pid[n], t->A[c], t->pid[c], t->xref,
                                                t->bodies, t->st); });
        if (d.capM > 0)
            launch(t, K_COMPACT, [&] { launch_compact_markers(d, t->sk_nnb, t->pid[c], t->nnb,
                                                              t->act_bcount, t->act, t->act_body,
                                                              t->n_act, t->st); }, 2);
    } else {
        launch(t, K_NEIGHBORS, [&] { launch_neighbors(d, t->A[n].pos, t->start, t->nbr, t->nnb,
                                                      d.maxnb, d.four_h2, t->err, t->st); });
        if (d.capM > 0)
            launch(t, K_COMPACT, [&] { launch_compact_markers(d, t->nnb, t->pid[n], nullptr,
                                                              t->act_bcount, t->act, t->act_body,
                                                              t->n_act, t->st); }, 2);
    }
}

void rebuild(crm_terrain *t)
{
    const DevParams &d = t->dp;
    // with the skin, the decision gates the gather of the working set too
    if (t->skin_on && (d.capN > 0 || t->active))
        launch(t, K_SKIN, [&] { launch_decide(d, t->gate, 0ull, 0, t->st,
                                              t->active ? t->counts : nullptr); });
    if (t->active) activity_pass(t);
    if (d.capN > 0) enqueue_search(t);
    if (!t->skin_on) t->cur = 1 - t->cur;
    t->lists_valid = true;
    t->prof.rebuilds += 1;
}

// BCE state at stage offset tau; accel 1 (stage 2) also reduces the wrench
// and advances the bodies by dt when `integrate`.
// `filter` (stage 1 right after a rebuild with the skin): the kernel walks the
// skin lists and writes the exact lists for the rest of the step.
void bce(crm_terrain *t, StageArrays S, double tau, int accel, double dt = 0.0, int integrate = 0,
         bool filter = false, cudaStream_t st = nullptr)
{
    const DevParams &d = t->dp;
    if (d.capM == 0) return;
    const int c = t->cur;
    int *gate = t->skin_on ? t->gate : nullptr;
    const uint32_t *skl = filter ? t->sk_nbr : nullptr, *skn = filter ? t->sk_nnb : nullptr;
    const uint32_t *act = accel == 2 ? nullptr : (accel == 1 ? t->act_body : t->act);
    const int *n_act = accel == 1 ? t->n_act + 1 : t->n_act;
    launch(t, K_BCE, [&] { launch_bce(d, S, t->A[c].pos, t->pid[c], t->mloc, t->bodies, t->nbr,
                                      t->nnb, tau, accel, (int)t->nFtot, t->mforce, t->partial,
                                      dt, integrate, gate, st ? st : t->st, skl, skn,
                                      t->err, t->mid_frames, act, n_act, t->n_bodym); },
           accel == 1 ? 2 : 1);
}

void pair(crm_terrain *t, int mode, StageArrays S, StageArrays Y, float dt, RateOut out,
          bool filter = false)
{
    const DevParams &d = t->dp;
    if (d.capF == 0) return;
    const int k = mode == kStage2 ? K_PAIR2 : K_PAIR1;
    const uint32_t *flags = t->active ? t->pid[t->cur] : nullptr;
    const float4 *xref = t->skin_on ? t->xref : nullptr;
    int *gate = t->skin_on ? t->gate : nullptr;
    const uint32_t *skl = filter ? t->sk_nbr : nullptr, *skn = filter ? t->sk_nnb : nullptr;
    launch(t, k, [&] { launch_pair(mode, d, S, Y, t->MID, t->nbr, t->nnb, flags, dt, out, t->err,
                                   xref, gate, t->st, skl, skn); });
}

// One RK2 step.  The body markers' accelerations, the FP64 wrench and the body
// update only feed the next step, so they run on a side stream beside pair
// stage 2 (a parallel branch of the step graph); the step ends after both.
void enqueue_stages(crm_terrain *t, double dt, bool filter)
{
    const int c = t->cur;
    RateOut none{};
    if (t->active && t->skin_on && t->dp.capF > 0) {
        // the step's Active / Extended counts start from zero (the skin decision
        // resets them in a step that runs it)
        if (!filter) cudaMemsetAsync(t->counts + C_NA, 0, 2 * sizeof(int), t->st);
        const int all = !(t->time > t->t_delay);
        launch(t, K_SKIN, [&] { launch_flags(t->dp, (int)t->box_body_h.size(), t->box_body,
                                             t->box_half, t->box_off, t->bodies, all, t->pid[c],
                                             t->A[c].pos, t->counts, t->st); });
    }
    bce(t, t->A[c], 0.0, 0, dt, 0, filter);   // also the bodies' midpoint frames
    pair(t, kStage1, t->A[c], t->A[c], (float)dt, none, filter);
    bce(t, t->MID, 0.5 * dt, 0);               // marker state at the midpoint
    const bool wrench = t->dp.capM > 0 && t->dp.n_bodies > 0;
    const bool fork = wrench && t->side != nullptr && !t->timing;
    if (fork) {
        cudaEventRecord(t->ev_fork, t->st);
        cudaStreamWaitEvent(t->side, t->ev_fork, 0);
    }
    if (wrench) bce(t, t->MID, 0.5 * dt, 1, dt, 1, false, fork ? t->side : nullptr);
    pair(t, kStage2, t->MID, t->A[c], (float)dt, none);
    if (fork) {
        cudaEventRecord(t->ev_join, t->side);
        cudaStreamWaitEvent(t->st, t->ev_join, 0);
    }
}

void one_step(crm_terrain *t, double dt)
{
    const int ps = t->P.ps_freq;
    const bool search = !t->lists_valid || t->step_index % ps == 0;
    if (search) rebuild(t);
    enqueue_stages(t, dt, search && t->skin_on);
    t->step_index += 1;
    t->time += dt;
    t->prof.steps += 1;
}

// The co-simulation exchange of crm_cosim_step as stream work: the bodies' new
// pose and twist from the pinned staging (before a step), or every body's state
// and the error word back to it (after).
void exchange_in(crm_terrain *t)
{
    for (size_t b = 0; b < t->hbodies.size(); ++b)
        cudaMemcpyAsync(&t->bodies[b], &t->h_xbodies[b], 13 * sizeof(double), cudaMemcpyHostToDevice,
                        t->st);
}

void exchange_out(crm_terrain *t)
{
    const size_t nb = t->hbodies.size();
    if (nb > 0)   // the bodies and the error word behind them (the staging's layout too)
        cudaMemcpyAsync(t->h_xbodies, t->bodies, nb * sizeof(BodyDev) + sizeof(int),
                        cudaMemcpyDeviceToHost, t->st);
    else
        cudaMemcpyAsync((int *)(t->h_xbodies + 1), t->err, sizeof(int), cudaMemcpyDeviceToHost, t->st);
}

// Capture one step into an executable graph: with the skin, the decision
// kernel switches a conditional node around the cell sort and search.  With
// `exchange` the graph also holds the co-simulation exchange around the step.
int capture_step(crm_terrain *t, double dt, bool search, crm_terrain::StepGraph &G,
                 bool exchange = false)
{
    if (G.exec) {
        cudaGraphExecDestroy(G.exec);
        G.exec = nullptr;
    }
    const cudaStreamCaptureMode mode = cudaStreamCaptureModeThreadLocal;
    cudaStream_t user = t->st;
    const bool timing = t->timing;
    const crm_profile saved = t->prof;
    const int cur = t->cur;
    t->st = t->cap_st;
    t->timing = false;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaGraphCreate(&g, 0);
    const DevParams &d = t->dp;
    if (e == cudaSuccess && search && t->skin_on) {
        cudaGraphConditionalHandle h;
        e = cudaGraphConditionalHandleCreate(&h, g, 0, cudaGraphCondAssignDefault);
        cudaGraphNode_t dec = nullptr, cn = nullptr;
        if (e == cudaSuccess) e = cudaStreamBeginCaptureToGraph(t->st, g, nullptr, nullptr, 0, mode);
        if (e == cudaSuccess) {
            if (exchange) exchange_in(t);
            launch_decide(d, t->gate, (unsigned long long)h, 1, t->st,
                          t->active ? t->counts : nullptr);
            cudaStreamCaptureStatus cs;
            const cudaGraphNode_t *deps = nullptr;
            size_t nd = 0;
            e = cudaStreamGetCaptureInfo(t->st, &cs, nullptr, nullptr, &deps, nullptr, &nd);
            if (e == cudaSuccess && nd == 1) dec = deps[0];   // the decision kernel
            const cudaError_t e2 = cudaStreamEndCapture(t->st, &g);
            if (e == cudaSuccess) e = e2;
            if (e == cudaSuccess && dec == nullptr) e = cudaErrorUnknown;
        }
        cudaGraphNodeParams cp = {};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = h;
        cp.conditional.type = cudaGraphCondTypeIf;
        cp.conditional.size = 1;
        if (e == cudaSuccess) e = cudaGraphAddNode(&cn, g, &dec, nullptr, 1, &cp);
        if (e == cudaSuccess) {
            cudaGraph_t body = cp.conditional.phGraph_out[0];
            e = cudaStreamBeginCaptureToGraph(t->st, body, nullptr, nullptr, 0, mode);
            if (e == cudaSuccess) {
                if (t->active) activity_pass(t);
                if (d.capN > 0) enqueue_search(t);
                e = cudaStreamEndCapture(t->st, &body);
            }
        }
        if (e == cudaSuccess) e = cudaStreamBeginCaptureToGraph(t->st, g, &cn, nullptr, 1, mode);
        if (e == cudaSuccess) {
            enqueue_stages(t, dt, true);
            if (exchange) exchange_out(t);
            e = cudaStreamEndCapture(t->st, &g);
        }
    } else if (e == cudaSuccess) {
        e = cudaStreamBeginCaptureToGraph(t->st, g, nullptr, nullptr, 0, mode);
        if (e == cudaSuccess) {
            if (exchange) exchange_in(t);
            if (search) {
                if (t->active) activity_pass(t);
                enqueue_search(t);
                t->cur = 1 - t->cur;
            }
            enqueue_stages(t, dt, false);
            if (exchange) exchange_out(t);
            e = cudaStreamEndCapture(t->st, &g);
        }
    }
    t->cur = cur;
    t->st = user;
    t->timing = timing;
    t->prof = saved;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&G.exec, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        cudaGetLastError();
        G.exec = nullptr;
        return t->fail(CRM_ECUDA, std::string("step graph capture failed: ") + cudaGetErrorString(e));
    }
    G.dt = dt;
    return CRM_OK;
}

// One step by graph replay (same kernels as one_step); with `exchange` the
// graph that holds the co-simulation exchange too (crm_cosim_step).
int graph_step(crm_terrain *t, double dt, bool exchange = false)
{
    const bool search = !t->lists_valid || t->step_index % t->P.ps_freq == 0;
    crm_terrain::StepGraph &G = exchange ? (search ? t->x_search[t->cur] : t->x_plain[t->cur])
                                         : (search ? t->g_search[t->cur] : t->g_plain[t->cur]);
    if (!G.exec || G.dt != dt) {
        if (capture_step(t, dt, search, G, exchange) != CRM_OK) {
            // no graph on this device / driver: direct launches from now on
            t->graphs = false;
            t->msg.clear();
            if (exchange) exchange_in(t);
            one_step(t, dt);
            if (exchange) exchange_out(t);
            CRM_CUDA(t, cudaGetLastError());
            return CRM_OK;
        }
    }
    CRM_CUDA(t, cudaGraphLaunch(G.exec, t->st));
    const DevParams &d = t->dp;
    // launch bookkeeping of the replayed kernels (the searches that the skin
    // decision actually ran are read back from the device at profile_read)
    if (search) {
        if (t->skin_on) {
            t->prof.launches[K_SKIN] += 1;
            if (t->active && d.capF > 0) t->prof.launches[K_SKIN] += 1;   // the step's flags
        } else {
            t->prof.launches[K_KEYS] += 1;
            t->prof.launches[K_SCAN] += 1;
            t->prof.launches[K_SCATTER] += 1;
            t->prof.launches[K_REORDER] += 1;
            t->prof.launches[K_NEIGHBORS] += 1;
            if (d.capM > 0) t->prof.launches[K_COMPACT] += 2;
            if (t->active) {   // scatter-back, box prep, activity, scan, sizes, gather
                t->prof.launches[K_EXPORT] += 1;
                t->prof.launches[K_KEYS] += 4;
                t->prof.launches[K_SCAN] += 1;
            }
            t->cur = 1 - t->cur;
        }
        t->prof.rebuilds += 1;
        t->lists_valid = true;
    }
    if (d.capM > 0) t->prof.launches[K_BCE] += d.n_bodies > 0 ? 4 : 2;
    if (d.capF > 0) {
        t->prof.launches[K_PAIR1] += 1;
        t->prof.launches[K_PAIR2] += 1;
    }
    t->step_index += 1;
    t->time += dt;
    t->prof.steps += 1;
    return CRM_OK;
}

int read_counts(crm_terrain *t)
{
    CRM_CUDA(t, cudaMemcpyAsync(t->h_counts, t->counts, C_WORDS * sizeof(int), cudaMemcpyDeviceToHost,
                                t->st));
    CRM_CUDA(t, cudaMemcpyAsync(t->h_counts + C_WORDS, t->abort_flag, sizeof(int),
                                cudaMemcpyDeviceToHost, t->st));
    CRM_CUDA(t, cudaStreamSynchronize(t->st));
    return CRM_OK;
}

int64_t grown(int64_t need, double G) { return (int64_t)std::ceil((double)need * G) + 64; }

// Active-domain stepping: chunks of at most S_I steps, then a sync to handle a
// capacity overflow (grow by G and resume at the abandoned step) and, at S_I
// boundaries, the shrink test of ManageArrayMemory (Sec. 3.2).
int step_active(crm_terrain *t, double dt, int n_steps)
{
    const int SI = t->P.shrink_interval;
    int remaining = n_steps;
    int guard = 0, rc0 = CRM_OK;
    while (remaining > 0) {
        const int64_t s0 = t->step_index;
        const double t0 = t->time;
        const int chunk = (int)std::min<int64_t>(remaining, SI - (s0 % SI));
        const unsigned long long s0d = (unsigned long long)s0;
        CRM_CUDA(t, cudaMemcpyAsync(t->step_ctr, &s0d, sizeof(s0d), cudaMemcpyHostToDevice, t->st));
        for (int s = 0; s < chunk; ++s) {
            // with the skin, the working set gathered while every particle was
            // processed is replaced by the boxes' one at the first step after t_delay
            const bool boxes = t->time > t->t_delay;
            if (t->skin_on && boxes && !t->boxes_in_force) {
                rc0 = invalidate_lists(t);
                if (rc0) return rc0;
            }
            t->boxes_in_force = boxes;
            // graph replay once the working set exists and the boxes are in force
            // (before t_delay every particle is processed, a different launch set)
            if (t->graphs && !t->timing && t->cap_st && t->have_working && t->lists_valid
                && t->time > t->t_delay) {
                int rg = graph_step(t, dt);
                if (rg) return rg;
            } else {
                one_step(t, dt);
            }
        }
        CRM_CUDA(t, cudaGetLastError());
        int rc = read_counts(t);
        if (rc) return rc;
        const int ab = t->h_counts[C_WORDS];
        if (ab == kAbortTimeout) return latched_error(t);   // frozen until crm_load_state
        if (ab != 0) {
            if (++guard > 64) return t->fail(CRM_ENOMEM, "active-set capacity kept overflowing");
            const int64_t failed = (int64_t)ab - 1;
            const int64_t done = failed - s0;
            t->step_index = failed;
            t->time = t0 + (double)done * dt;
            remaining -= (int)done;
            t->prof.steps -= (chunk - done);
            const int *h = t->h_counts;
            const double G = t->P.growth;
            bool work = false, win = false, cand = false;
            if (h[C_NEED_F] > t->capF) { t->capF = grown(h[C_NEED_F], G); work = true; }
            if (h[C_NEED_M] > t->capM) { t->capM = grown(h[C_NEED_M], G); work = true; }
            if (h[C_NEED_CELLS] > t->Mcap) { t->Mcap = grown(h[C_NEED_CELLS], G); win = true; }
            if (h[C_NEED_CAND] > t->cand_cap) { t->cand_cap = grown(h[C_NEED_CAND], G); cand = true; }
            if (2.0 * (double)t->Mcap + 1.0 >= 2147483647.0)
                return t->fail(CRM_EINVAL, "active window too large for the cell sort");
            // the abandoned rebuild already wrote the working set back to the master
            t->have_working = false;
            if (work) { rc = alloc_working(t); if (rc) return rc; }
            if (win) { rc = alloc_window(t); if (rc) return rc; }
            if (cand) { rc = alloc_cand(t); if (rc) return rc; }
            rc = invalidate_lists(t);
            if (rc) return rc;
            CRM_CUDA(t, cudaMemsetAsync(t->abort_flag, 0, sizeof(int), t->st));
            CRM_CUDA(t, cudaMemsetAsync(t->counts + C_NEED_F, 0, 4 * sizeof(int), t->st));
            continue;
        }
        remaining -= chunk;
        if (t->step_index % SI == 0) {
            // shrink the working arrays to the current size when under S full
            const int64_t nF = t->h_counts[C_NF], nM = t->h_counts[C_NM];
            const double S = t->P.shrink_ratio;
            const bool shrink = (t->capF > 0 && (double)nF / (double)t->capF < S)
                                || (t->capM > 0 && (double)nM / (double)t->capM < S);
            if (shrink) {
                scatter_back(t);
                t->have_working = false;
                t->capF = std::max<int64_t>(nF, 1);
                t->capM = std::max<int64_t>(nM, 1);
                rc = alloc_working(t);
                if (!rc) rc = invalidate_lists(t);
                if (rc) return rc;
            }
            // the cell window and the candidate ranges follow the same rule (the
            // first step before t_delay sizes them for the whole terrain)
            const int64_t cells = t->h_counts[C_USE_CELLS], cand = t->h_counts[C_USE_CAND];
            if (cells > 0 && (double)cells / (double)t->Mcap < S) {
                t->Mcap = cells;
                rc = alloc_window(t);
                if (!rc) rc = invalidate_lists(t);
                if (rc) return rc;
            }
            if (cand > 0 && (double)cand / (double)t->cand_cap < S) {
                t->cand_cap = cand;
                rc = alloc_cand(t);
                if (rc) return rc;
            }
        }
    }
    return CRM_OK;
}

template <class T> int download(crm_terrain *t, T *host, const T *dev, size_t n)
{
    if (n == 0 || host == nullptr) return CRM_OK;
    CRM_CUDA(t, cudaMemcpyAsync(host, dev, n * sizeof(T), cudaMemcpyDeviceToHost, t->st));
    return CRM_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
extern "C" {

int crm_version(void) { return 100; }

const char *crm_status_string(int s)
{
    switch (s) {
    case CRM_OK: return "CRM_OK";
    case CRM_EINVAL: return "CRM_EINVAL";
    case CRM_ENOMEM: return "CRM_ENOMEM";
    case CRM_ECAPACITY: return "CRM_ECAPACITY";
    case CRM_EESCAPED: return "CRM_EESCAPED";
    case CRM_ENONFINITE: return "CRM_ENONFINITE";
    case CRM_ETIMEOUT: return "CRM_ETIMEOUT";
    case CRM_ECUDA: return "CRM_ECUDA";
    case CRM_ESTATE: return "CRM_ESTATE";
    default: return "CRM_UNKNOWN";
    }
}

void crm_default_params(crm_params *p)
{
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->rho0 = 1700.0;
    p->E = 1.0e6;
    p->nu = 0.3;
    p->mu_s = p->mu_2 = std::tan(30.0 * 3.14159265358979323846 / 180.0);
    p->I0 = 0.08;
    p->grain_d = 0.002;
    p->cohesion = 0.0;
    p->d0 = 0.01;
    p->h = 0.012;
    p->kernel = CRM_KERNEL_CUBIC;
    p->av_mode = CRM_AV_UNILATERAL;
    p->av_gamma = 0.02;
    p->av_xi2_over_h2 = 0.01;
    p->gravity[2] = -9.81;
    p->ps_freq = 1;
    p->max_neighbors = 96;
    for (int k = 0; k < 3; ++k) {
        p->domain_min[k] = 0.0;
        p->domain_max[k] = 1.0;
    }
    p->growth = 1.2;
    p->shrink_ratio = 0.75;
    p->shrink_interval = 50;
    p->skin = 0.1;
}

int crm_capacity_policy(int64_t need, int64_t cap, int64_t step, double growth,
                        double shrink_ratio, int32_t shrink_interval, int64_t *new_cap)
{
    if (!new_cap || need < 0 || cap < 0 || !(growth >= 1.0) || !(shrink_ratio > 0)
        || shrink_interval < 1)
        return CRM_EINVAL;
    int64_t c = cap;
    if (need > cap) c = (int64_t)std::ceil((double)need * growth);
    else if (step % shrink_interval == 0 && cap > 0 && (double)need / (double)cap < shrink_ratio)
        c = need;
    *new_cap = c;
    return CRM_OK;
}

int crm_create(const crm_params *p, void *cuda_stream, crm_terrain **out)
{
    if (!out) return CRM_EINVAL;
    *out = nullptr;
    if (!p) return CRM_EINVAL;
    std::string why;
    if (validate(p, why) != CRM_OK) {
        std::fprintf(stderr, "crm_create: %s\n", why.c_str());
        return CRM_EINVAL;
    }
    crm_terrain *t = new (std::nothrow) crm_terrain();
    if (!t) return CRM_ENOMEM;
    t->P = *p;
    t->st = (cudaStream_t)cuda_stream;
    *out = t;
    return CRM_OK;
}

int crm_destroy(crm_terrain *t)
{
    if (!t) return CRM_OK;
    if (t->committed) cudaStreamSynchronize(t->st);
    for (auto &r : t->pending) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (cudaEvent_t e : t->ev_pool) cudaEventDestroy(e);
    t->drop_graphs();
    if (t->cap_st) cudaStreamDestroy(t->cap_st);
    if (t->side) {
        cudaStreamSynchronize(t->side);
        cudaStreamDestroy(t->side);
        cudaEventDestroy(t->ev_fork);
        cudaEventDestroy(t->ev_join);
    }
    if (t->adj_st) {
        cudaStreamSynchronize(t->adj_st);
        cudaStreamDestroy(t->adj_st);
        for (cudaEvent_t e : t->adj_ev) cudaEventDestroy(e);
    }
    drop_tape(t);
    for (int g = 0; g < G_COUNT; ++g) t->free_group(g);
    if (t->h_counts) cudaFreeHost(t->h_counts);
    if (t->h_xbodies) cudaFreeHost(t->h_xbodies);
    delete t;
    return CRM_OK;
}

const char *crm_last_error(const crm_terrain *t) { return t ? t->msg.c_str() : ""; }

int crm_add_sph(crm_terrain *t, int64_t n, const double *xyz, const double *vel,
                const double *stress6, const double *rho)
{
    if (!t) return CRM_EINVAL;
    if (t->committed) return t->fail(CRM_ESTATE, "crm_add_sph after the first step");
    if (n < 0 || (n > 0 && !xyz)) return t->fail(CRM_EINVAL, "crm_add_sph: bad n or null xyz");
    for (int64_t i = 0; i < n; ++i)
        if (!inside_domain(t->P, xyz + 3 * i))
            return t->fail(CRM_EINVAL, "crm_add_sph: particle outside [domain_min, domain_max)");
    if (!finite_all(xyz, 3 * n) || (vel && !finite_all(vel, 3 * n))
        || (stress6 && !finite_all(stress6, 6 * n)) || (rho && !finite_all(rho, n)))
        return t->fail(CRM_EINVAL, "crm_add_sph: non-finite input");
    if (rho)
        for (int64_t i = 0; i < n; ++i)
            if (!(rho[i] > 0)) return t->fail(CRM_EINVAL, "crm_add_sph: density must be > 0");
    t->hx.insert(t->hx.end(), xyz, xyz + 3 * n);
    for (int64_t i = 0; i < n; ++i) {
        for (int k = 0; k < 3; ++k) t->hu.push_back(vel ? vel[3 * i + k] : 0.0);
        for (int k = 0; k < 6; ++k) t->hs.push_back(stress6 ? stress6[6 * i + k] : 0.0);
        t->hr.push_back(rho ? rho[i] : t->P.rho0);
    }
    t->nFtot += n;
    return CRM_OK;
}

int crm_add_fixed_bce(crm_terrain *t, int64_t n, const double *xyz)
{
    if (!t) return CRM_EINVAL;
    if (t->committed) return t->fail(CRM_ESTATE, "crm_add_fixed_bce after the first step");
    if (n < 0 || (n > 0 && !xyz)) return t->fail(CRM_EINVAL, "crm_add_fixed_bce: bad n or null xyz");
    if (!finite_all(xyz, 3 * n)) return t->fail(CRM_EINVAL, "crm_add_fixed_bce: non-finite input");
    for (int64_t i = 0; i < n; ++i)
        if (!inside_domain(t->P, xyz + 3 * i))
            return t->fail(CRM_EINVAL, "crm_add_fixed_bce: marker outside the domain");
    t->hmloc.insert(t->hmloc.end(), xyz, xyz + 3 * n);
    t->hmbody.insert(t->hmbody.end(), (size_t)n, -1);
    t->nMtot += n;
    return CRM_OK;
}

int crm_add_rigid_body(crm_terrain *t, int64_t n, const double *xloc, const double pose[7],
                       const double twist[6], double mass, int32_t dof_mask, int32_t *body_id)
{
    if (!t) return CRM_EINVAL;
    if (t->committed) return t->fail(CRM_ESTATE, "crm_add_rigid_body after the first step");
    if (n < 0 || (n > 0 && !xloc) || !pose || !twist)
        return t->fail(CRM_EINVAL, "crm_add_rigid_body: bad n or null array");
    if (!(mass > 0) || (dof_mask & ~63)) return t->fail(CRM_EINVAL, "crm_add_rigid_body: mass > 0, dof_mask in 0..63");
    if ((int)t->hbodies.size() >= kMaxBodies) return t->fail(CRM_EINVAL, "at most 16 bodies");
    if (!finite_all(xloc, 3 * n) || !finite_all(pose, 7) || !finite_all(twist, 6))
        return t->fail(CRM_EINVAL, "crm_add_rigid_body: non-finite input");
    const double qn = std::sqrt(pose[3] * pose[3] + pose[4] * pose[4] + pose[5] * pose[5] + pose[6] * pose[6]);
    if (!(qn > 0.5 && qn < 2.0)) return t->fail(CRM_EINVAL, "crm_add_rigid_body: quaternion not normalised");
    BodyDev b{};
    for (int k = 0; k < 3; ++k) b.pose[k] = pose[k];
    for (int k = 3; k < 7; ++k) b.pose[k] = pose[k] / qn;
    for (int k = 0; k < 6; ++k) b.twist[k] = twist[k];
    b.mass = mass;
    b.inv_mass = 1.0 / mass;
    b.dof = dof_mask;
    const int id = (int)t->hbodies.size();
    t->hbodies.push_back(b);
    t->hmloc.insert(t->hmloc.end(), xloc, xloc + 3 * n);
    t->hmbody.insert(t->hmbody.end(), (size_t)n, id);
    t->nMtot += n;
    if (body_id) *body_id = id;
    return CRM_OK;
}

}  // extern "C"

namespace {
// The host copy of a body's motion, checked and with the quaternion normalised.
int set_motion_host(crm_terrain *t, int32_t body, const double pose[7], const double twist[6])
{
    if (body < 0 || body >= (int)t->hbodies.size() || !pose || !twist)
        return t->fail(CRM_EINVAL, "crm_set_body_motion: bad body or null array");
    if (!finite_all(pose, 7) || !finite_all(twist, 6)) return t->fail(CRM_EINVAL, "non-finite motion");
    const double qn = std::sqrt(pose[3] * pose[3] + pose[4] * pose[4] + pose[5] * pose[5] + pose[6] * pose[6]);
    if (!(qn > 0.5 && qn < 2.0)) return t->fail(CRM_EINVAL, "crm_set_body_motion: quaternion not normalised");
    BodyDev &b = t->hbodies[body];
    for (int k = 0; k < 3; ++k) b.pose[k] = pose[k];
    for (int k = 3; k < 7; ++k) b.pose[k] = pose[k] / qn;
    for (int k = 0; k < 6; ++k) b.twist[k] = twist[k];
    return CRM_OK;
}
}  // namespace

extern "C" {

int crm_set_body_motion(crm_terrain *t, int32_t body, const double pose[7], const double twist[6])
{
    if (!t) return CRM_EINVAL;
    const int rc = set_motion_host(t, body, pose, twist);
    if (rc) return rc;
    BodyDev &b = t->hbodies[body];
    if (t->committed)
        CRM_CUDA(t, cudaMemcpyAsync(&t->bodies[body], &b, 13 * sizeof(double),
                                    cudaMemcpyHostToDevice, t->st));
    return CRM_OK;
}

int crm_set_body_inertia(crm_terrain *t, int32_t body, const double inertia[3])
{
    if (!t) return CRM_EINVAL;
    if (body < 0 || body >= (int)t->hbodies.size() || !inertia)
        return t->fail(CRM_EINVAL, "crm_set_body_inertia: bad body or null array");
    if (!finite_all(inertia, 3) || !(inertia[0] > 0 && inertia[1] > 0 && inertia[2] > 0))
        return t->fail(CRM_EINVAL, "crm_set_body_inertia: moments must be finite and > 0");
    BodyDev &b = t->hbodies[body];
    for (int k = 0; k < 3; ++k) b.inertia[k] = inertia[k];
    if (t->committed)
        CRM_CUDA(t, cudaMemcpyAsync(t->bodies[body].inertia, b.inertia, sizeof(b.inertia),
                                    cudaMemcpyHostToDevice, t->st));
    return CRM_OK;
}

int crm_set_body_load(crm_terrain *t, int32_t body, const double force[3], const double torque[3])
{
    if (!t) return CRM_EINVAL;
    if (body < 0 || body >= (int)t->hbodies.size() || !force || !torque)
        return t->fail(CRM_EINVAL, "crm_set_body_load: bad body or null array");
    if (!finite_all(force, 3) || !finite_all(torque, 3))
        return t->fail(CRM_EINVAL, "crm_set_body_load: non-finite load");
    BodyDev &b = t->hbodies[body];
    for (int k = 0; k < 3; ++k) {
        b.load[k] = force[k];
        b.load[3 + k] = torque[k];
    }
    if (t->committed)
        CRM_CUDA(t, cudaMemcpyAsync(t->bodies[body].load, b.load, sizeof(b.load),
                                    cudaMemcpyHostToDevice, t->st));
    return CRM_OK;
}

int crm_get_body_state(crm_terrain *t, int32_t body, double pose[7], double twist[6])
{
    if (!t) return CRM_EINVAL;
    if (body < 0 || body >= (int)t->hbodies.size()) return t->fail(CRM_EINVAL, "bad body");
    BodyDev &b = t->hbodies[body];
    if (t->committed) {
        CRM_CUDA(t, cudaMemcpyAsync(&b, &t->bodies[body], sizeof(BodyDev), cudaMemcpyDeviceToHost, t->st));
        CRM_CUDA(t, cudaStreamSynchronize(t->st));
    }
    if (pose) std::memcpy(pose, b.pose, 7 * sizeof(double));
    if (twist) std::memcpy(twist, b.twist, 6 * sizeof(double));
    return CRM_OK;
}

int crm_add_active_box(crm_terrain *t, int32_t body, const double half[3], const double off[3],
                       double t_delay)
{
    if (!t) return CRM_EINVAL;
    if (t->committed) return t->fail(CRM_ESTATE, "crm_add_active_box after the first step");
    if (body < 0 || body >= (int)t->hbodies.size() || !half || !off)
        return t->fail(CRM_EINVAL, "crm_add_active_box: bad body or null array");
    if (!finite_all(half, 3) || !finite_all(off, 3) || !std::isfinite(t_delay))
        return t->fail(CRM_EINVAL, "crm_add_active_box: non-finite input");
    if (!(half[0] > 0 && half[1] > 0 && half[2] > 0))
        return t->fail(CRM_EINVAL, "crm_add_active_box: half extents must be > 0");
    if ((int)t->box_body_h.size() >= kMaxBodies) return t->fail(CRM_EINVAL, "at most 16 active boxes");
    t->box_body_h.push_back(body);
    t->box_half_h.insert(t->box_half_h.end(), half, half + 3);
    t->box_off_h.insert(t->box_off_h.end(), off, off + 3);
    t->t_delay = t->box_body_h.size() == 1 ? t_delay : std::max(t->t_delay, t_delay);
    return CRM_OK;
}

int crm_step(crm_terrain *t, double dt, int32_t n_steps)
{
    if (!t) return CRM_EINVAL;
    if (!(dt > 0) || !std::isfinite(dt) || n_steps < 0) return t->fail(CRM_EINVAL, "crm_step: dt > 0, n_steps >= 0");
    if (t->frozen)
        return t->fail(CRM_ESTATE, "terrain frozen after a device wait gave up; crm_load_state a checkpoint");
    int rc = commit(t);
    if (rc) return rc;
    if (t->active) return step_active(t, dt, n_steps);
    if (t->graphs && !t->timing && t->cap_st && t->dp.capN > 0) {
        for (int s = 0; s < n_steps; ++s) {
            rc = graph_step(t, dt);
            if (rc) return rc;
        }
        return CRM_OK;
    }
    for (int s = 0; s < n_steps; ++s) one_step(t, dt);
    CRM_CUDA(t, cudaGetLastError());
    return CRM_OK;
}

int crm_sync(crm_terrain *t)
{
    if (!t) return CRM_EINVAL;
    if (!t->committed) return CRM_OK;
    return latched_error(t);
}

int crm_get_particles(crm_terrain *t, int64_t cap, double *xyz, float *vel, float *stress6,
                      float *rho, int64_t *n_out)
{
    if (!t) return CRM_EINVAL;
    const int64_t n = t->nFtot;
    if (n_out) *n_out = n;
    if (cap < n) return t->fail(CRM_EINVAL, "crm_get_particles: cap smaller than the particle count");
    if (!t->committed) {
        for (int64_t i = 0; i < n; ++i) {
            if (xyz) for (int k = 0; k < 3; ++k) xyz[3 * i + k] = t->hx[3 * i + k];
            if (vel) for (int k = 0; k < 3; ++k) vel[3 * i + k] = (float)t->hu[3 * i + k];
            if (stress6) for (int k = 0; k < 6; ++k) stress6[6 * i + k] = (float)t->hs[6 * i + k];
            if (rho) rho[i] = (float)t->hr[i];
        }
        return CRM_OK;
    }
    const size_t bytes = n * (3 * sizeof(double) + 10 * sizeof(float));
    void *buf = nullptr;
    CRM_CUDA(t, cudaMallocAsync(&buf, std::max<size_t>(bytes, 16), t->st));
    double *dx = (double *)buf;
    float *dv = (float *)(dx + 3 * n), *ds = dv + 3 * n, *dr = ds + 6 * n;
    if (n > 0) {
        if (t->active) {
            scatter_back(t);
            launch(t, K_EXPORT, [&] { launch_export_master(t->dp, t->Mst, t->mpid, (int)n, dx, dv,
                                                           ds, dr, t->st); });
        } else {
            launch(t, K_EXPORT, [&] { launch_export(t->dp, t->A[t->cur], t->pid[t->cur], dx, dv, ds,
                                                    dr, t->st); });
        }
    }
    int rc = download(t, xyz, dx, 3 * n);
    if (!rc) rc = download(t, vel, dv, 3 * n);
    if (!rc) rc = download(t, stress6, ds, 6 * n);
    if (!rc) rc = download(t, rho, dr, n);
    cudaFreeAsync(buf, t->st);
    if (rc) return rc;
    return latched_error(t);
}

int crm_cosim_step(crm_terrain *t, const double *pose_in, const double *twist_in, double dt,
                   int32_t n_steps, double *wrench_out, double *pose_out, double *twist_out)
{
    if (!t) return CRM_EINVAL;
    if (t->frozen)
        return t->fail(CRM_ESTATE, "terrain frozen after a device wait gave up; crm_load_state a checkpoint");
    const int nb = (int)t->hbodies.size();
    if ((pose_in == nullptr) != (twist_in == nullptr))
        return t->fail(CRM_EINVAL, "crm_cosim_step: give both pose and twist, or neither");
    if (pose_in) {
        for (int b = 0; b < nb; ++b) {
            const int rc = set_motion_host(t, b, pose_in + 7 * b, twist_in + 6 * b);
            if (rc) return rc;
        }
    }
    int rc = commit(t);
    if (rc) return rc;
    if (!t->h_xbodies) {
        void *h = nullptr;
        if (cudaMallocHost(&h, std::max(nb, 1) * sizeof(BodyDev) + sizeof(int)) != cudaSuccess) {
            cudaGetLastError();
            return t->fail(CRM_ENOMEM, "crm_cosim_step: pinned staging allocation failed");
        }
        t->h_xbodies = (BodyDev *)h;
    }
    int *h_err = (int *)(t->h_xbodies + std::max(nb, 1));
    if (pose_in)   // the new motions through pinned memory: truly asynchronous uploads
        for (int b = 0; b < nb; ++b)
            std::memcpy(t->h_xbodies[b].pose, t->hbodies[b].pose, 13 * sizeof(double));
    if (n_steps == 1 && pose_in && !t->active && t->graphs && !t->timing && t->cap_st
        && t->dp.capN > 0) {
        // one exchange step: upload, step and read-back replayed as one graph
        if (!(dt > 0) || !std::isfinite(dt)) return t->fail(CRM_EINVAL, "crm_cosim_step: dt > 0");
        rc = graph_step(t, dt, true);
        if (rc) return rc;
    } else {
        if (pose_in) exchange_in(t);
        if (n_steps > 0) {
            rc = crm_step(t, dt, n_steps);
            if (rc) return rc;
        }
        exchange_out(t);
    }
    CRM_CUDA(t, cudaGetLastError());
    CRM_CUDA(t, cudaStreamSynchronize(t->st));
    if (*h_err != 0) return latched_error(t);
    for (int b = 0; b < nb; ++b) {
        t->hbodies[b] = t->h_xbodies[b];
        if (wrench_out) std::memcpy(wrench_out + 6 * b, t->h_xbodies[b].wrench, 6 * sizeof(double));
        if (pose_out) std::memcpy(pose_out + 7 * b, t->h_xbodies[b].pose, 7 * sizeof(double));
        if (twist_out) std::memcpy(twist_out + 6 * b, t->h_xbodies[b].twist, 6 * sizeof(double));
    }
    return CRM_OK;
}

int crm_get_diagnostics(crm_terrain *t, double *out)
{
    if (!t || !out) return CRM_EINVAL;
    const double m = t->P.rho0 * t->P.d0 * t->P.d0 * t->P.d0;
    const int64_t n = t->nFtot;
    if (!t->committed) {
        for (int k = 0; k < CRM_NUM_DIAG; ++k) out[k] = 0.0;
        for (int64_t i = 0; i < n; ++i) {
            const double *x = &t->hx[3 * i], *u = &t->hu[3 * i];
            out[CRM_DIAG_COUNT] += 1.0;
            out[CRM_DIAG_MASS] += m;
            out[CRM_DIAG_VOLUME] += m / t->hr[i];
            for (int k = 0; k < 3; ++k) out[CRM_DIAG_MOMENTUM + k] += m * u[k];
            out[CRM_DIAG_ANGULAR + 0] += m * (x[1] * u[2] - x[2] * u[1]);
            out[CRM_DIAG_ANGULAR + 1] += m * (x[2] * u[0] - x[0] * u[2]);
            out[CRM_DIAG_ANGULAR + 2] += m * (x[0] * u[1] - x[1] * u[0]);
            out[CRM_DIAG_KINETIC] += 0.5 * m * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
        }
        return CRM_OK;
    }
    const size_t nd = diag_scratch_doubles();
    double *buf = nullptr;
    CRM_CUDA(t, cudaMallocAsync((void **)&buf, nd * sizeof(double), t->st));
    if (t->active) {
        scatter_back(t);   // the master store holds every particle, Active or not
        launch(t, K_EXPORT, [&] { launch_diagnostics(t->dp, t->Mst, nullptr, (int)n, m, buf, t->st); });
    } else {
        launch(t, K_EXPORT, [&] { launch_diagnostics(t->dp, t->A[t->cur], t->dp.sizes, 0, m, buf,
                                                     t->st); });
    }
    int rc = download(t, out, buf + (nd - CRM_NUM_DIAG), CRM_NUM_DIAG);
    cudaFreeAsync(buf, t->st);
    if (rc) return rc;
    return latched_error(t);   // synchronises the stream
}

int crm_get_body_wrench(crm_terrain *t, int32_t body, double force[3], double torque[3])
{
    if (!t) return CRM_EINVAL;
    if (body < 0 || body >= (int)t->hbodies.size()) return t->fail(CRM_EINVAL, "bad body");
    BodyDev &b = t->hbodies[body];
    if (t->committed) {
        CRM_CUDA(t, cudaMemcpyAsync(&b, &t->bodies[body], sizeof(BodyDev), cudaMemcpyDeviceToHost, t->st));
        int rc = latched_error(t);
        if (rc) return rc;
    }
    if (force) std::memcpy(force, b.wrench, 3 * sizeof(double));
    if (torque) std::memcpy(torque, b.wrench + 3, 3 * sizeof(double));
    return CRM_OK;
}

int crm_get_counts(crm_terrain *t, int64_t *n_active, int64_t *n_extended, int64_t *n_bce)
{
    if (!t) return CRM_EINVAL;
    int64_t a = t->nFtot, e = 0, b = t->nMtot;
    if (t->committed && t->active) {
        int rc = read_counts(t);
        if (rc) return rc;
        a = t->h_counts[C_NA];
        e = t->h_counts[C_NE];
        b = t->h_counts[C_NM];
    }
    if (n_active) *n_active = a;
    if (n_extended) *n_extended = e;
    if (n_bce) *n_bce = b;
    return CRM_OK;
}

int crm_eval_rates(crm_terrain *t, int64_t cap_sph, float *drho, float *dvel, float *dstress,
                   int64_t cap_markers, float *marker_acc, float *marker_vel, float *marker_stress)
{
    if (!t) return CRM_EINVAL;
    if (t->frozen)
        return t->fail(CRM_ESTATE, "terrain frozen after a device wait gave up; crm_load_state a checkpoint");
    if (cap_sph < t->nFtot || cap_markers < t->nMtot)
        return t->fail(CRM_EINVAL, "crm_eval_rates: output capacity too small");
    int rc = commit(t);
    if (rc) return rc;
    rebuild(t);
    if (t->active) {
        rc = read_counts(t);
        if (rc) return rc;
        if (t->h_counts[C_WORDS] != 0) {
            CRM_CUDA(t, cudaMemsetAsync(t->abort_flag, 0, sizeof(int), t->st));
            t->have_working = false;   // the abandoned rebuild wrote it back
            rc = invalidate_lists(t);
            if (rc) return rc;
            return t->fail(CRM_ENOMEM, "crm_eval_rates: active set exceeds its capacity; step once first");
        }
    }
    const int c = t->cur;
    const DevParams &d = t->dp;
    const int64_t nF = t->nFtot, nM = t->nMtot;
    const int64_t wF = d.capF;
    const size_t rate_bytes = wF * (sizeof(float) + 2 * sizeof(float4) + sizeof(float2));
    const size_t out_bytes = (nF * 10 + nM * 12) * sizeof(float);
    void *buf = nullptr;
    CRM_CUDA(t, cudaMallocAsync(&buf, std::max<size_t>(rate_bytes + out_bytes + 64, 64), t->st));
    char *b = (char *)buf;
    RateOut r{};
    r.du = (float4 *)b;
    r.dsA = r.du + wF;
    r.dsB = (float2 *)(r.dsA + wF);
    r.drho = (float *)(r.dsB + wF);
    float *o = r.drho + wF;
    float *odrho = o, *odu = o + nF, *ods = odu + 3 * nF, *omacc = ods + 6 * nF,
          *omvel = omacc + 3 * nM, *omsig = omvel + 3 * nM;
    CRM_CUDA(t, cudaMemsetAsync(o, 0, out_bytes, t->st));
    if (t->active && t->skin_on && d.capF > 0) {
        const int all = !(t->time > t->t_delay);
        launch(t, K_SKIN, [&] { launch_flags(d, (int)t->box_body_h.size(), t->box_body,
                                             t->box_half, t->box_off, t->bodies, all, t->pid[c],
                                             t->A[c].pos, t->counts, t->st); });
    }
    if (t->skin_on) {
        // exact lists from the skin lists first (marker and fluid rows)
        bce(t, t->A[c], 0.0, 0, 0.0, 0, true);
        pair(t, kEval, t->A[c], t->A[c], 0.0f, r, true);
        bce(t, t->A[c], 0.0, 2);
    } else {
        bce(t, t->A[c], 0.0, 2);
        pair(t, kEval, t->A[c], t->A[c], 0.0f, r);
    }
    if (d.capN > 0)
        launch(t, K_EXPORT, [&] { launch_export_rates(d, t->pid[c], r, t->A[c], t->mforce,
                                                      (int)t->nFtot, odrho, odu, ods, omacc, omvel,
                                                      omsig, t->st); });
    rc = download(t, drho, odrho, nF);
    if (!rc) rc = download(t, dvel, odu, 3 * nF);
    if (!rc) rc = download(t, dstress, ods, 6 * nF);
    if (!rc) rc = download(t, marker_acc, omacc, 3 * nM);
    if (!rc) rc = download(t, marker_vel, omvel, 3 * nM);
    if (!rc) rc = download(t, marker_stress, omsig, 6 * nM);
    cudaFreeAsync(buf, t->st);
    if (rc) return rc;
    return latched_error(t);
}

int crm_get_neighbors(crm_terrain *t, int64_t cap, int64_t *offset, int32_t *list, int64_t *nnz)
{
    if (!t) return CRM_EINVAL;
    if (!t->committed || !t->lists_valid) return t->fail(CRM_ESTATE, "crm_get_neighbors: no lists built yet");
    const DevParams &d = t->dp;
    const int64_t W = d.capN, Ntot = t->nFtot + t->nMtot;
    int hs[3] = {0, 0, 0};
    std::vector<uint32_t> nnb(W), pid(W), tab((size_t)d.maxnb * d.ell);
    int rc = download(t, hs, (const int *)t->counts, 3);
    if (!rc) rc = download(t, nnb.data(), t->nnb, W);
    if (!rc) rc = download(t, pid.data(), t->pid[t->cur], W);
    if (!rc) rc = download(t, tab.data(), t->nbr, tab.size());
    if (rc) return rc;
    rc = latched_error(t);
    if (rc) return rc;
    const int64_t N = hs[2];
    std::vector<int64_t> cnt(Ntot + 1, 0);
    for (int64_t s = 0; s < N; ++s) cnt[pid_index(pid[s]) + 1] = nnb[s];
    for (int64_t i = 0; i < Ntot; ++i) cnt[i + 1] += cnt[i];
    if (nnz) *nnz = cnt[Ntot];
    if (offset) std::memcpy(offset, cnt.data(), (Ntot + 1) * sizeof(int64_t));
    if (!list) return CRM_OK;
    if (cap < cnt[Ntot]) return t->fail(CRM_EINVAL, "crm_get_neighbors: list capacity too small");
    for (int64_t s = 0; s < N; ++s) {
        const int64_t o = cnt[pid_index(pid[s])];
        for (uint32_t k = 0; k < nnb[s]; ++k)
            list[o + k] = (int32_t)pid_index(pid[tab[(size_t)k * d.ell + s] & kIndexMask]);
        std::sort(list + o, list + o + nnb[s]);
    }
    return CRM_OK;
}

// The next step re-sorts and searches whatever the skin test says (a change
// of the sort order makes the cell ranges of the last search stale).
static int force_search(crm_terrain *t)
{
    t->lists_valid = false;
    if (!t->committed || !t->skin_on) return CRM_OK;
    static const int one = 1;
    CRM_CUDA(t, cudaMemcpyAsync(t->gate + GATE_FORCE, &one, sizeof(int), cudaMemcpyHostToDevice,
                                t->st));
    CRM_CUDA(t, cudaStreamSynchronize(t->st));
    return CRM_OK;
}

int crm_debug_absolute_fp32(crm_terrain *t, int32_t on)
{
    if (!t || (on != 0 && on != 1)) return CRM_EINVAL;
    if (t->committed) return t->fail(CRM_ESTATE, "crm_debug_absolute_fp32: before the first step");
    t->abs32 = on;
    return CRM_OK;
}

int crm_debug_wait_fault(int32_t on)
{
    if (on != 0 && on != 1) return CRM_EINVAL;
    return set_wait_fault(on) == 0 ? CRM_OK : CRM_ECUDA;
}

int crm_set_cell_tile(crm_terrain *t, int32_t nx, int32_t ny, int32_t nz)
{
    if (!t) return CRM_EINVAL;
    auto lg = [](int v, int mx) { for (int k = 0; (1 << k) <= mx; ++k) if ((1 << k) == v) return k; return -1; };
    const int bx = lg(nx, kTileX), by = lg(ny, kTileY), bz = lg(nz, kTileZ);
    if (bx < 0 || by < 0 || bz < 0)
        return t->fail(CRM_EINVAL, "crm_set_cell_tile: powers of two up to 8 x 4 x 4");
    t->tile_log2[0] = bx;
    t->tile_log2[1] = by;
    t->tile_log2[2] = bz;
    t->dp.tbx = bx;
    t->dp.tby = by;
    t->dp.tbz = bz;
    t->drop_graphs();   // the captured launches hold the old shape
    return force_search(t);
}

int crm_set_pair_lanes(crm_terrain *t, int32_t lanes)
{
    if (!t) return CRM_EINVAL;
    if (lanes < 0 || lanes > 4 || lanes == 3)
        return t->fail(CRM_EINVAL, "crm_set_pair_lanes: 0, 1, 2 or 4");
    t->P.pair_lanes = lanes;
    t->dp.pair_lanes = lanes;
    t->drop_graphs();   // the captured launches hold the old choice
    return CRM_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batches: several terrains stepped together, each on its own stream, so that
// small terrains share the GPU instead of leaving it partly idle one after the
// other.  A step of the batch is one replayed step graph per member; the
// batch's stream forks to the members' streams and joins them again.
struct crm_batch {
    std::vector<crm_terrain *> m;
    cudaStream_t st = nullptr;
    cudaEvent_t fork = nullptr;
    std::vector<cudaEvent_t> join;
    std::string msg;
    // persistent form (crm_batch_set_persistent): one step graph for the whole
    // batch -- every member's search decision and gated search, then one
    // persistent launch per stage over all members
    bool persistent = false;
    cudaStream_t cap = nullptr, side = nullptr;   // capture streams
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<double> gdt;                      // the time steps of the graph
    MemberDev *dmem = nullptr;                    // device tables of the graph
    int *dtab = nullptr;
    unsigned *dqueue = nullptr;
    int launches_per_step = 0;
    void drop()
    {
        if (exec) cudaGraphExecDestroy(exec);
        exec = nullptr;
        if (dmem) cudaFree(dmem);
        if (dtab) cudaFree(dtab);
        if (dqueue) cudaFree(dqueue);
        dmem = nullptr;
        dtab = nullptr;
        dqueue = nullptr;
        gdt.clear();
    }
};

namespace {

// Capture terrain t's search decision and its gated cell search (the
// conditional branch of its step graph) into graph g as a root branch; *out
// receives the conditional node.
int append_member_search(crm_terrain *t, cudaGraph_t g, cudaGraphNode_t *out)
{
    const cudaStreamCaptureMode mode = cudaStreamCaptureModeThreadLocal;
    cudaStream_t user = t->st;
    const bool timing = t->timing;
    const crm_profile saved = t->prof;
    t->st = t->cap_st;
    t->timing = false;
    const DevParams &d = t->dp;
    cudaGraphConditionalHandle h;
    cudaError_t e = cudaGraphConditionalHandleCreate(&h, g, 0, cudaGraphCondAssignDefault);
    cudaGraphNode_t dec = nullptr;
    if (e == cudaSuccess) e = cudaStreamBeginCaptureToGraph(t->st, g, nullptr, nullptr, 0, mode);
    if (e == cudaSuccess) {
        launch_decide(d, t->gate, (unsigned long long)h, 1, t->st);
        cudaStreamCaptureStatus cs;
        const cudaGraphNode_t *deps = nullptr;
        size_t nd = 0;
        e = cudaStreamGetCaptureInfo(t->st, &cs, nullptr, nullptr, &deps, nullptr, &nd);
        if (e == cudaSuccess && nd == 1) dec = deps[0];
        cudaGraph_t g2 = g;
        const cudaError_t e2 = cudaStreamEndCapture(t->st, &g2);
        if (e == cudaSuccess) e = e2;
        if (e == cudaSuccess && dec == nullptr) e = cudaErrorUnknown;
    }
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeIf;
    cp.conditional.size = 1;
    cudaGraphNode_t cn = nullptr;
    if (e == cudaSuccess) e = cudaGraphAddNode(&cn, g, &dec, nullptr, 1, &cp);
    if (e == cudaSuccess) {
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        e = cudaStreamBeginCaptureToGraph(t->st, body, nullptr, nullptr, 0, mode);
        if (e == cudaSuccess) {
            enqueue_search(t);
            e = cudaStreamEndCapture(t->st, &body);
        }
    }
    t->st = user;
    t->timing = timing;
    t->prof = saved;
    if (e != cudaSuccess) {
        cudaGetLastError();
        return CRM_ECUDA;
    }
    *out = cn;
    return CRM_OK;
}

// Work table of one batched launch (members and their block counts) appended to
// the host table; returns {offset of the member list, offset of the prefix
// offsets, count, total blocks}.
struct Work { int mlist, off, n, total; };

Work add_work(std::vector<int> &tab, const std::vector<std::pair<int, int>> &mb)
{
    Work w{(int)tab.size(), 0, (int)mb.size(), 0};
    for (auto &x : mb) tab.push_back(x.first);
    w.off = (int)tab.size();
    int acc = 0;
    tab.push_back(0);
    for (auto &x : mb) {
        acc += x.second;
        tab.push_back(acc);
    }
    w.total = acc;
    return w;
}

// Build the persistent batch step graph for time steps dt (member i: dt[i]).
int batch_build(crm_batch *b, const double *dt)
{
    b->drop();
    const int n = (int)b->m.size();
    for (int i = 0; i < n; ++i) {
        crm_terrain *t = b->m[i];
        int rc = commit(t);
        if (rc) return rc;
        if (!t->skin_on || t->active || t->P.ps_freq != 1 || !t->graphs || !t->cap_st
            || t->dp.capN < 1 || t->frozen) {
            b->msg = "persistent batch: every member needs a Verlet skin, ps_freq 1, no active "
                     "boxes and step graphs";
            return CRM_EINVAL;
        }
    }
    // members' descriptors
    std::vector<MemberDev> hm(n);
    for (int i = 0; i < n; ++i) {
        crm_terrain *t = b->m[i];
        const int c = t->cur;
        MemberDev &M = hm[i];
        M.p = t->dp;
        M.S = t->A[c];
        M.MID = t->MID;
        M.pid = t->pid[c];
        M.mloc = t->mloc;
        M.bodies = t->bodies;
        M.frames = t->mid_frames;
        M.nbr = t->nbr;
        M.nnb = t->nnb;
        M.sk_nbr = t->sk_nbr;
        M.sk_nnb = t->sk_nnb;
        M.act = t->act;
        M.act_body = t->act_body;
        M.n_act = t->n_act;
        M.mforce = t->mforce;
        M.partial = t->partial;
        M.xref = t->xref;
        M.gate = t->gate;
        M.err = t->err;
        M.n_fluid_total = (int)t->nFtot;
        M.n_bodym = (int)t->n_bodym;
        M.dt = dt[i];
    }
    // work tables: BCE state launches, the wrench, stage 1 by kernel shape, stage 2
    // by (lanes, kernel shape), the (member, body) pairs of the body updates
    std::vector<int> tab;
    std::vector<std::pair<int, int>> bce, wr;
    std::vector<int> pairs;
    std::vector<std::pair<int, std::vector<std::pair<int, int>>>> p1, p2;   // key -> members
    auto group = [](std::vector<std::pair<int, std::vector<std::pair<int, int>>>> &gs, int key)
        -> std::vector<std::pair<int, int>> & {
        for (auto &g : gs)
            if (g.first == key) return g.second;
        gs.push_back({key, {}});
        return gs.back().second;
    };
    for (int i = 0; i < n; ++i) {
        const DevParams &d = hm[i].p;
        if (d.capM > 0) bce.push_back({i, (int)bce_blocks(d)});
        if (d.capM > 0 && d.n_bodies > 0) {
            wr.push_back({i, (int)wrench_blocks(b->m[i]->n_bodym)});
            for (int q = 0; q < d.n_bodies; ++q) {
                pairs.push_back(i);
                pairs.push_back(q);
            }
        }
        if (d.capF > 0) {
            const int kav = pair_kav(d), ln = pair_lanes_of(d), fl = pair_filter_lanes(ln);
            group(p1, 8 * kav + fl).push_back({i, (int)grid_for((int64_t)d.capF * fl, 128)});
            group(p2, 8 * kav + ln).push_back({i, (int)grid_for((int64_t)d.capF * ln, 128)});
        }
    }
    const Work w_bce = add_work(tab, bce), w_wr = add_work(tab, wr);
    std::vector<std::pair<int, Work>> w1, w2;
    for (auto &g : p1) w1.push_back({g.first, add_work(tab, g.second)});
    for (auto &g : p2) w2.push_back({g.first, add_work(tab, g.second)});
    const int pair_at = (int)tab.size();
    tab.insert(tab.end(), pairs.begin(), pairs.end());
    const int nq = 4 + (int)w1.size() + (int)w2.size();
    if (cudaMalloc(&b->dmem, sizeof(MemberDev) * n) != cudaSuccess
        || cudaMalloc(&b->dtab, sizeof(int) * std::max<size_t>(tab.size(), 1)) != cudaSuccess
        || cudaMalloc(&b->dqueue, sizeof(unsigned) * 2 * nq) != cudaSuccess) {
        cudaGetLastError();
        b->drop();
        return CRM_ENOMEM;
    }
    if (cudaMemcpy(b->dmem, hm.data(), sizeof(MemberDev) * n, cudaMemcpyHostToDevice) != cudaSuccess
        || cudaMemcpy(b->dtab, tab.data(), sizeof(int) * tab.size(), cudaMemcpyHostToDevice)
               != cudaSuccess
        || cudaMemset(b->dqueue, 0, sizeof(unsigned) * 2 * nq) != cudaSuccess) {
        cudaGetLastError();
        b->drop();
        return CRM_ECUDA;
    }
    // the graph: every member's search branch, then the batched stages
    cudaGraph_t g = nullptr;
    if (cudaGraphCreate(&g, 0) != cudaSuccess) return CRM_ECUDA;
    std::vector<cudaGraphNode_t> deps(n);
    for (int i = 0; i < n; ++i) {
        const int rc = append_member_search(b->m[i], g, &deps[i]);
        if (rc) {
            cudaGraphDestroy(g);
            b->drop();
            return rc;
        }
    }
    const cudaStreamCaptureMode mode = cudaStreamCaptureModeThreadLocal;
    cudaError_t e = cudaStreamBeginCaptureToGraph(b->cap, g, deps.data(), nullptr, deps.size(), mode);
    int launches = 0;
    if (e == cudaSuccess) {
        const int *T = b->dtab;
        unsigned *Q = b->dqueue;
        auto bce_go = [&](int kind, const Work &w, cudaStream_t s, unsigned *q) {
            if (w.total > 0) {
                launch_batch_bce(kind, b->dmem, T + w.mlist, T + w.off, w.n, w.total, q, s);
                ++launches;
            }
        };
        bce_go(0, w_bce, b->cap, Q);
        int qi = 4;
        for (auto &x : w1) {
            launch_batch_pair(kStage1, x.first % 8, x.first / 8, b->dmem, T + x.second.mlist,
                              T + x.second.off, x.second.n, x.second.total, Q + 2 * qi++, b->cap);
            ++launches;
        }
        bce_go(1, w_bce, b->cap, Q + 2);
        const bool fork = w_wr.total > 0;
        if (fork) {
            cudaEventRecord(b->ev_fork, b->cap);
            cudaStreamWaitEvent(b->side, b->ev_fork, 0);
            bce_go(2, w_wr, b->side, Q + 4);
            launch_batch_reduce(b->dmem, T + pair_at, (int)pairs.size() / 2, b->side);
            ++launches;
        }
        for (auto &x : w2) {
            launch_batch_pair(kStage2, x.first % 8, x.first / 8, b->dmem, T + x.second.mlist,
                              T + x.second.off, x.second.n, x.second.total, Q + 2 * qi++, b->cap);
            ++launches;
        }
        if (fork) {
            cudaEventRecord(b->ev_join, b->side);
            cudaStreamWaitEvent(b->cap, b->ev_join, 0);
        }
        e = cudaStreamEndCapture(b->cap, &g);
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        cudaGetLastError();
        b->drop();
        b->msg = std::string("persistent batch graph: ") + cudaGetErrorString(e);
        return CRM_ECUDA;
    }
    b->launches_per_step = launches;
    b->gdt.assign(dt, dt + n);
    return CRM_OK;
}

// One step of every member by the persistent batch graph, and the members'
// host bookkeeping of it (as graph_step keeps it).
int batch_graph_step(crm_batch *b, const double *dt)
{
    const int n = (int)b->m.size();
    bool same = b->exec && (int)b->gdt.size() == n;
    for (int i = 0; same && i < n; ++i) same = b->gdt[i] == dt[i];
    if (!same) {
        const int rc = batch_build(b, dt);
        if (rc) return rc;
    }
    if (cudaGraphLaunch(b->exec, b->st) != cudaSuccess) return CRM_ECUDA;
    for (int i = 0; i < n; ++i) {
        crm_terrain *t = b->m[i];
        t->prof.launches[K_SKIN] += 1;
        if (t->dp.capM > 0) t->prof.launches[K_BCE] += t->dp.n_bodies > 0 ? 4 : 2;
        if (t->dp.capF > 0) {
            t->prof.launches[K_PAIR1] += 1;
            t->prof.launches[K_PAIR2] += 1;
        }
        t->prof.rebuilds += 1;
        t->lists_valid = true;
        t->step_index += 1;
        t->time += dt[i];
        t->prof.steps += 1;
    }
    return CRM_OK;
}

}  // namespace

extern "C" {

int crm_batch_create(int32_t n, crm_terrain *const *members, void *stream, crm_batch **out)
{
    if (!out || n < 1 || !members) return CRM_EINVAL;
    *out = nullptr;
    for (int i = 0; i < n; ++i) {
        if (!members[i] || members[i]->st == nullptr) return CRM_EINVAL;   // not the legacy stream
        for (int k = 0; k < i; ++k)
            if (members[k] == members[i]) return CRM_EINVAL;
    }
    crm_batch *b = new crm_batch();
    b->m.assign(members, members + n);
    b->st = (cudaStream_t)stream;
    b->join.assign(n, nullptr);
    bool ok = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) == cudaSuccess
              && cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming) == cudaSuccess
              && cudaEventCreateWithFlags(&b->ev_join, cudaEventDisableTiming) == cudaSuccess
              && cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) == cudaSuccess
              && cudaStreamCreateWithFlags(&b->side, cudaStreamNonBlocking) == cudaSuccess;
    for (int i = 0; ok && i < n; ++i)
        ok = cudaEventCreateWithFlags(&b->join[i], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        crm_batch_destroy(b);
        return CRM_ECUDA;
    }
    *out = b;
    return CRM_OK;
}

int crm_batch_destroy(crm_batch *b)
{
    if (!b) return CRM_OK;
    b->drop();
    if (b->cap) cudaStreamDestroy(b->cap);
    if (b->side) cudaStreamDestroy(b->side);
    if (b->ev_fork) cudaEventDestroy(b->ev_fork);
    if (b->ev_join) cudaEventDestroy(b->ev_join);
    if (b->fork) cudaEventDestroy(b->fork);
    for (cudaEvent_t e : b->join)
        if (e) cudaEventDestroy(e);
    delete b;
    return CRM_OK;
}

int crm_batch_step(crm_batch *b, const double *dt, int32_t n_steps)
{
    if (!b || !dt || n_steps < 0) return CRM_EINVAL;
    const int n = (int)b->m.size();
    if (b->persistent) {
        // the batch's stream waits for the members' pending work, runs the steps,
        // and the members' streams wait for it
        for (int i = 0; i < n; ++i) {
            if (b->m[i]->frozen) return CRM_ESTATE;
            if (cudaEventRecord(b->join[i], b->m[i]->st) != cudaSuccess
                || cudaStreamWaitEvent(b->st, b->join[i], 0) != cudaSuccess)
                return CRM_ECUDA;
        }
        for (int s = 0; s < n_steps; ++s) {
            const int rc = batch_graph_step(b, dt);
            if (rc) return rc;
        }
        if (cudaEventRecord(b->fork, b->st) != cudaSuccess) return CRM_ECUDA;
        for (int i = 0; i < n; ++i)
            if (cudaStreamWaitEvent(b->m[i]->st, b->fork, 0) != cudaSuccess) return CRM_ECUDA;
        return CRM_OK;
    }
    if (cudaEventRecord(b->fork, b->st) != cudaSuccess) return CRM_ECUDA;
    for (int i = 0; i < n; ++i)
        if (cudaStreamWaitEvent(b->m[i]->st, b->fork, 0) != cudaSuccess) return CRM_ECUDA;
    // step-major order: every member's step k is enqueued before any step k + 1
    for (int s = 0; s < n_steps; ++s)
        for (int i = 0; i < n; ++i) {
            const int rc = crm_step(b->m[i], dt[i], 1);
            if (rc) return rc;
        }
    for (int i = 0; i < n; ++i) {
        if (cudaEventRecord(b->join[i], b->m[i]->st) != cudaSuccess) return CRM_ECUDA;
        if (cudaStreamWaitEvent(b->st, b->join[i], 0) != cudaSuccess) return CRM_ECUDA;
    }
    return CRM_OK;
}

int crm_batch_set_persistent(crm_batch *b, int32_t on)
{
    if (!b || (on != 0 && on != 1)) return CRM_EINVAL;
    b->persistent = on != 0;
    b->drop();
    return CRM_OK;
}

int crm_batch_autotune(crm_batch *b, const double *dt, int32_t trial_steps, int32_t *choice)
{
    if (!b || !dt || trial_steps < 1) return CRM_EINVAL;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        return CRM_ECUDA;
    }
    // candidates: lanes per particle of the exact-list pair kernels x cell tiles
    // of the sort order (row-major, and 4 x 2 x 2 cells)
    static const int tiles[2][3] = {{1, 1, 1}, {4, 2, 2}};
    int rc = CRM_OK;
    for (size_t i = 0; i < b->m.size() && rc == CRM_OK; ++i) {
        crm_terrain *t = b->m[i];
        float best = 0.f;
        int pick_l = 2, pick_t = 0;
        bool first = true;
        for (int tl = 0; tl < 2 && rc == CRM_OK; ++tl)
            for (int lanes = 1; lanes <= 4 && rc == CRM_OK; lanes *= 2) {
                crm_set_pair_lanes(t, lanes);
                rc = crm_set_cell_tile(t, tiles[tl][0], tiles[tl][1], tiles[tl][2]);
                if (rc) break;
                rc = crm_step(t, dt[i], 1);   // capture the graphs (and re-sort) outside the timing
                if (rc) break;
                cudaEventRecord(e0, t->st);
                rc = crm_step(t, dt[i], trial_steps);
                cudaEventRecord(e1, t->st);
                if (rc) break;
                float ms = 0.f;
                if (cudaEventSynchronize(e1) != cudaSuccess
                    || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
                    cudaGetLastError();
                    rc = CRM_ECUDA;
                    break;
                }
                if (first || ms < best) {
                    best = ms;
                    pick_l = lanes;
                    pick_t = tl;
                    first = false;
                }
            }
        if (rc == CRM_OK) {
            crm_set_pair_lanes(t, pick_l);
            rc = crm_set_cell_tile(t, tiles[pick_t][0], tiles[pick_t][1], tiles[pick_t][2]);
            if (choice)
                choice[i] = pick_l | tiles[pick_t][0] << 4 | tiles[pick_t][1] << 8
                            | tiles[pick_t][2] << 12;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->drop();   // the persistent graph holds the old choices
    return rc;
}

const char *crm_kernel_name(int32_t k)
{
    return (k >= 0 && k < CRM_NUM_KERNELS) ? kKernelNames[k] : "";
}

int crm_profile_reset(crm_terrain *t, int32_t timing)
{
    if (!t) return CRM_EINVAL;
    if (!t->pending.empty()) {
        CRM_CUDA(t, cudaStreamSynchronize(t->st));
        for (auto &r : t->pending) {
            t->ev_pool.push_back(r.a);
            t->ev_pool.push_back(r.b);
        }
        t->pending.clear();
    }
    std::memset(&t->prof, 0, sizeof(t->prof));
    t->timing = timing != 0;
    t->searched = 0;
    if (t->committed && t->skin_on) {
        int g[GATE_WORDS];
        CRM_CUDA(t, cudaMemcpy(g, t->gate, sizeof(g), cudaMemcpyDeviceToHost));
        t->searches_at_reset = g[GATE_SEARCHES];
    }
    return CRM_OK;
}

int crm_profile_read(crm_terrain *t, crm_profile *out)
{
    if (!t || !out) return CRM_EINVAL;
    if (t->committed) CRM_CUDA(t, cudaStreamSynchronize(t->st));
    if (t->committed && t->skin_on) {
        // cell searches the skin decision ran since the reset (each is keys,
        // scan, scatter, reorder, search and copy-back)
        int g[GATE_WORDS];
        CRM_CUDA(t, cudaMemcpy(g, t->gate, sizeof(g), cudaMemcpyDeviceToHost));
        const int64_t n = g[GATE_SEARCHES] - t->searches_at_reset;
        t->searches_at_reset = g[GATE_SEARCHES];
        if (!t->timing) {
            t->prof.launches[K_KEYS] = t->prof.launches[K_SCAN] = t->prof.launches[K_SCATTER] = 0;
            t->prof.launches[K_REORDER] = t->prof.launches[K_NEIGHBORS] = 0;
            t->prof.launches[K_COMPACT] = 0;
        }
        t->searched += n;
        if (!t->timing) {
            t->prof.launches[K_KEYS] += t->searched;
            t->prof.launches[K_SCAN] += t->searched;
            t->prof.launches[K_SCATTER] += t->searched;
            t->prof.launches[K_REORDER] += t->searched;
            t->prof.launches[K_NEIGHBORS] += t->searched;
            t->prof.launches[K_SKIN] += t->searched;
            if (t->dp.capM > 0) t->prof.launches[K_COMPACT] += 2 * t->searched;
            if (t->active) {   // the gated gather: write-back, box prep, activity, scan, sizes, gather
                t->prof.launches[K_EXPORT] += n;
                t->prof.launches[K_KEYS] += 4 * t->searched;
                t->prof.launches[K_SCAN] += t->searched;
            }
        }
    }
    for (auto &r : t->pending) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) t->prof.ms[r.k] += ms;
        else cudaGetLastError();
        t->ev_pool.push_back(r.a);
        t->ev_pool.push_back(r.b);
    }
    t->pending.clear();
    *out = t->prof;
    return CRM_OK;
}

// Checkpoint layout: 64-byte header (step, time, particle count, bodies,
// active flag, drift), then the state arrays (the working set without active
// boxes, the master store with them) and the bodies.
int crm_state_bytes(crm_terrain *t, size_t *bytes)
{
    if (!t || !bytes) return CRM_EINVAL;
    const int64_t n = t->box_body_h.empty() ? t->nFtot + t->nMtot : t->nFtot;
    *bytes = 64 + n * (3 * sizeof(float4) + sizeof(float2) + sizeof(uint32_t))
             + t->hbodies.size() * sizeof(BodyDev);
    return CRM_OK;
}

int crm_save_state(crm_terrain *t, void *dev_buf, size_t cap, size_t *used)
{
    if (!t || !dev_buf) return CRM_EINVAL;
    int rc = commit(t);
    if (rc) return rc;
    size_t need = 0;
    crm_state_bytes(t, &need);
    if (used) *used = need;
    if (cap < need) return t->fail(CRM_EINVAL, "crm_save_state: buffer too small");
    scatter_back(t);
    const bool act = t->active;
    const int64_t n = act ? t->nFtot : t->nFtot + t->nMtot;
    const int c = t->cur;
    const StageArrays S = act ? t->Mst : t->A[c];
    const uint32_t *P = act ? t->mpid : t->pid[c];
    char *b = (char *)dev_buf;
    int64_t hdr[6] = {t->step_index, 0, n, (int64_t)t->hbodies.size(), act ? 1 : 0, 0};
    std::memcpy(&hdr[1], &t->time, sizeof(double));
    CRM_CUDA(t, cudaMemcpyAsync(b, hdr, 48, cudaMemcpyHostToDevice, t->st));
    if (act) CRM_CUDA(t, cudaMemcpyAsync(b + 48, t->drift, sizeof(int), cudaMemcpyDeviceToDevice, t->st));
    size_t o = 64;
    auto put = [&](const void *src, size_t nb) {
        cudaError_t e = cudaMemcpyAsync(b + o, src, nb, cudaMemcpyDeviceToDevice, t->st);
        o += nb;
        return e;
    };
    CRM_CUDA(t, put(S.pos, n * sizeof(float4)));
    CRM_CUDA(t, put(S.vel, n * sizeof(float4)));
    CRM_CUDA(t, put(S.sA, n * sizeof(float4)));
    CRM_CUDA(t, put(S.sB, n * sizeof(float2)));
    CRM_CUDA(t, put(P, n * sizeof(uint32_t)));
    if (!t->hbodies.empty()) CRM_CUDA(t, put(t->bodies, t->hbodies.size() * sizeof(BodyDev)));
    CRM_CUDA(t, cudaStreamSynchronize(t->st));
    return CRM_OK;
}

int crm_load_state(crm_terrain *t, const void *dev_buf, size_t used)
{
    if (!t || !dev_buf) return CRM_EINVAL;
    int rc = commit(t);
    if (rc) return rc;
    size_t need = 0;
    crm_state_bytes(t, &need);
    if (used != need) return t->fail(CRM_EINVAL, "crm_load_state: size does not match this terrain");
    int64_t hdr[6];
    CRM_CUDA(t, cudaMemcpyAsync(hdr, dev_buf, 48, cudaMemcpyDeviceToHost, t->st));
    CRM_CUDA(t, cudaStreamSynchronize(t->st));
    const bool act = t->active;
    const int64_t n = act ? t->nFtot : t->nFtot + t->nMtot;
    if (hdr[2] != n || hdr[3] != (int64_t)t->hbodies.size() || hdr[4] != (act ? 1 : 0))
        return t->fail(CRM_EINVAL, "crm_load_state: checkpoint of a different terrain");
    const int c = t->cur;
    const StageArrays S = act ? t->Mst : t->A[c];
    uint32_t *P = act ? t->mpid : t->pid[c];
    const char *b = (const char *)dev_buf;
    if (act) CRM_CUDA(t, cudaMemcpyAsync(t->drift, b + 48, sizeof(int), cudaMemcpyDeviceToDevice, t->st));
    size_t o = 64;
    auto get = [&](void *dst, size_t nb) {
        cudaError_t e = cudaMemcpyAsync(dst, b + o, nb, cudaMemcpyDeviceToDevice, t->st);
        o += nb;
        return e;
    };
    CRM_CUDA(t, get(S.pos, n * sizeof(float4)));
    CRM_CUDA(t, get(S.vel, n * sizeof(float4)));
    CRM_CUDA(t, get(S.sA, n * sizeof(float4)));
    CRM_CUDA(t, get(S.sB, n * sizeof(float2)));
    CRM_CUDA(t, get(P, n * sizeof(uint32_t)));
    if (!t->hbodies.empty()) CRM_CUDA(t, get(t->bodies, t->hbodies.size() * sizeof(BodyDev)));
    t->step_index = hdr[0];
    std::memcpy(&t->time, &hdr[1], sizeof(double));
    t->lists_valid = false;
    t->have_working = false;
    // a terrain frozen by a device wait that gave up resumes from the checkpoint
    CRM_CUDA(t, cudaMemsetAsync(t->abort_flag, 0, sizeof(int), t->st));
    CRM_CUDA(t, cudaMemsetAsync(t->err, 0, sizeof(int), t->st));
    t->frozen = false;
    if (t->skin_on) {
        const int g0[GATE_SEARCHES] = {1, 0, 1, 0};
        CRM_CUDA(t, cudaMemcpyAsync(t->gate, g0, sizeof(g0), cudaMemcpyHostToDevice, t->st));
    }
    CRM_CUDA(t, cudaStreamSynchronize(t->st));
    return CRM_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Reverse sweep: the hand-derived adjoint of one rate evaluation and of a run
// of midpoint steps (kernels in crm_adjoint.cu).  A run is recorded as
// checkpoints every `every` steps; the backward pass restores each segment's
// checkpoint, re-runs its steps with direct launches while copying each step's
// stage arrays, lists and bodies to the tape, and then sweeps the segment's
// steps in reverse.  The adjoints of the fluid state live in insertion order
// between steps (the cell sort re-orders the slots every step).
namespace {

int adj_workspace(crm_terrain *t)
{
    crm_terrain::Adjoint &A = t->adj;
    if (A.ready) return CRM_OK;
    const DevParams &d = t->dp;
    const size_t nb = std::max<size_t>(t->hbodies.size(), 1);
    const size_t nF = (size_t)std::max<int64_t>(t->nFtot, 1), nM = (size_t)std::max<int64_t>(t->nMtot, 1);
    A.coef = t->dalloc<float4>(G_ADJ, 4 * (size_t)std::max(d.capN, 1));
    A.coefB = t->dalloc<float4>(G_ADJ, 4 * (size_t)std::max(d.capM, 1));
    A.l_mid = t->dalloc<float>(G_ADJ, (size_t)kNumAdj * std::max(d.capF, 1));
    A.l_y0 = t->dalloc<float>(G_ADJ, (size_t)kNumAdj * std::max(d.capF, 1));
    A.l_ins = t->dalloc<float>(G_ADJ, (size_t)kNumAdj * nF);
    A.l_rate = t->dalloc<float>(G_ADJ, 10 * nF);
    A.l_macc = t->dalloc<float>(G_ADJ, 3 * nM);
    A.sums = t->dalloc<float>(G_ADJ, 13 * (size_t)std::max(d.capF, 1));
    A.gpar = t->dalloc<double>(G_ADJ, kNumGradAcc);
    A.gbody = t->dalloc<double>(G_ADJ, 2 * kBodyAdj * nb);
    A.lb[0] = t->dalloc<double>(G_ADJ, kBodyAdj * nb);
    A.lb[1] = t->dalloc<double>(G_ADJ, kBodyAdj * nb);
    A.lwrench = t->dalloc<double>(G_ADJ, 6 * nb);
    if (t->oom) {
        t->oom = false;
        t->free_group(G_ADJ);
        A = crm_terrain::Adjoint{};
        return t->fail(CRM_ENOMEM, "device allocation of the adjoint workspace failed");
    }
    A.ready = true;
    return CRM_OK;
}

// What the sweep supports: no active boxes; for runs, a cell search every step
// without a skin (so that a re-run reproduces the recorded lists).
int adj_support(crm_terrain *t, bool run, const char *who)
{
    const std::string w(who);
    if (t->active) return t->fail(CRM_EINVAL, w + ": active domains are not differentiated");
    if (!run) return CRM_OK;
    if (t->skin_on || t->P.ps_freq != 1)
        return t->fail(CRM_EINVAL, w + ": needs skin = 0 and ps_freq = 1");
    return CRM_OK;
}

crm_terrain::AdjTape no_tape() { return crm_terrain::AdjTape{}; }

AdjIO adj_io(crm_terrain *t, float dt)
{
    const DevParams &d = t->dp;
    crm_terrain::Adjoint &A = t->adj;
    AdjIO io{};
    io.coef = A.coef;
    io.coefB = A.coefB;
    io.l_rate = A.l_rate;
    io.l_macc = nullptr;
    io.l_wrench = A.lwrench;
    io.l_next = A.l_ins;
    io.l_mid = A.l_mid;
    io.l_y0 = A.l_y0;
    io.l_out = A.l_y0;
    io.slot_stride = std::max(d.capF, 1);
    io.n_fluid = std::max<int64_t>(t->nFtot, 1);
    io.dt = dt;
    return io;
}

// Accumulated parameter adjoints (G, K, m, viscosity constant, direct rho0,
// mu_s, cohesion, mu_2, I0, grain diameter) -> the public parameters: G = E / (2 (1 + nu)),
// K = E / (3 (1 - 2 nu)), m = rho0 d0^3, c = gamma h sqrt(K / rho0) m.
void grads_from_acc(const crm_params &P, const double *a, double *g)
{
    const double Gm = P.E / (2.0 * (1.0 + P.nu)), Km = P.E / (3.0 * (1.0 - 2.0 * P.nu));
    const double m = P.rho0 * P.d0 * P.d0 * P.d0;
    const double c1 = P.h * std::sqrt(Km / P.rho0) * m;   // dc / dgamma
    const double c = P.av_gamma * c1;
    g[CRM_GRAD_E] = (a[kGradG] * Gm + a[kGradK] * Km + 0.5 * a[kGradAvc] * c) / P.E;
    g[CRM_GRAD_NU] = -a[kGradG] * Gm / (1.0 + P.nu) + (2.0 * a[kGradK] * Km + a[kGradAvc] * c) / (1.0 - 2.0 * P.nu);
    g[CRM_GRAD_RHO0] = a[kGradRho0] + a[kGradM] * m / P.rho0 + 0.5 * a[kGradAvc] * c / P.rho0;
    g[CRM_GRAD_MU_S] = a[kGradMu];
    g[CRM_GRAD_COHESION] = a[kGradCoh];
    g[CRM_GRAD_AV_GAMMA] = a[kGradAvc] * c1;
    g[CRM_GRAD_MU_2] = a[kGradMu2];
    g[CRM_GRAD_I0] = a[kGradI0];
    g[CRM_GRAD_GRAIN_D] = a[kGradGrain];
}

// Fluid adjoints (insertion order, FP32 on the device) -> caller's FP64
// arrays; body and parameter adjoints likewise.
int adj_export(crm_terrain *t, const double *lb_dev, double *g_xyz, double *g_vel,
               double *g_stress, double *g_rho, double *g_body, double *g_params)
{
    crm_terrain::Adjoint &A = t->adj;
    const int64_t nF = t->nFtot;
    const size_t nb = t->hbodies.size();
    std::vector<float> l((size_t)kNumAdj * std::max<int64_t>(nF, 1));
    std::vector<double> acc(kNumGradAcc), lb(kBodyAdj * std::max<size_t>(nb, 1));
    if (nF > 0 && (g_xyz || g_vel || g_stress || g_rho))
        CRM_CUDA(t, cudaMemcpyAsync(l.data(), A.l_ins, l.size() * sizeof(float), cudaMemcpyDeviceToHost, t->st));
    CRM_CUDA(t, cudaMemcpyAsync(acc.data(), A.gpar, kNumGradAcc * sizeof(double), cudaMemcpyDeviceToHost, t->st));
    if (nb > 0 && g_body && lb_dev)
        CRM_CUDA(t, cudaMemcpyAsync(lb.data(), lb_dev, kBodyAdj * nb * sizeof(double), cudaMemcpyDeviceToHost, t->st));
    CRM_CUDA(t, cudaStreamSynchronize(t->st));
    int rc = latched_error(t);
    if (rc) return rc;
    for (int64_t i = 0; i < nF; ++i) {
        for (int k = 0; k < 3; ++k) {
            if (g_xyz) g_xyz[3 * i + k] = l[(size_t)(kAdjX + k) * nF + i];
            if (g_vel) g_vel[3 * i + k] = l[(size_t)(kAdjU + k) * nF + i];
        }
        if (g_stress)
            for (int k = 0; k < 6; ++k) g_stress[6 * i + k] = l[(size_t)(kAdjS + k) * nF + i];
        if (g_rho) g_rho[i] = l[(size_t)kAdjR * nF + i];
    }
    if (g_body && lb_dev) std::memcpy(g_body, lb.data(), kBodyAdj * nb * sizeof(double));
    if (g_params) grads_from_acc(t->P, acc.data(), g_params);
    return CRM_OK;
}

// The device work of one recorded step: the step's kernels (those of the graph
// of a search step) with its stage arrays, lists and bodies copied to the tape.
// Flips t->cur as a rebuild does.
int enqueue_record(crm_terrain *t, double dt, crm_terrain::AdjTape &T)
{
    const DevParams &d = t->dp;
    const size_t N = (size_t)std::max(d.capN, 1), nb = t->hbodies.size();
    auto copy = [&](void *dst, const void *src, size_t bytes) {
        return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, t->st);
    };
    auto copy_stage = [&](StageArrays &dst, const StageArrays &src) {
        cudaError_t e = copy(dst.pos, src.pos, N * sizeof(float4));
        if (e == cudaSuccess) e = copy(dst.vel, src.vel, N * sizeof(float4));
        if (e == cudaSuccess) e = copy(dst.sA, src.sA, N * sizeof(float4));
        if (e == cudaSuccess) e = copy(dst.sB, src.sB, N * sizeof(float2));
        return e;
    };
    if (nb > 0) CRM_CUDA(t, copy(T.bodies, t->bodies, nb * sizeof(BodyDev)));
    // the step's cell search writes its lists and its compaction of the markers
    // with fluid in reach into the tape slot, and the stages read them there (no
    // copy of the list table)
    struct ListsIn {   // the terrain's own tables again on every way out
        crm_terrain *t;
        uint32_t *nbr, *nnb, *act, *act_body;
        int *n_act;
        ~ListsIn()
        {
            t->nbr = nbr; t->nnb = nnb;
            t->act = act; t->act_body = act_body; t->n_act = n_act;
        }
    } own{t, t->nbr, t->nnb, t->act, t->act_body, t->n_act};
    t->nbr = T.nbr;
    t->nnb = T.nnb;
    t->act = T.act;
    t->act_body = T.act_body;
    t->n_act = T.n_act;
    rebuild(t);
    const int c = t->cur;
    RateOut r1{}, r2{};
    r1.sums = T.sum0;
    r2.sums = T.sumM;
    bce(t, t->A[c], 0.0, 0, dt, 0, false);
    pair(t, kStage1, t->A[c], t->A[c], (float)dt, r1);
    CRM_CUDA(t, copy_stage(T.Y0, t->A[c]));
    CRM_CUDA(t, copy(T.pid, t->pid[c], N * sizeof(uint32_t)));
    if (nb > 0) CRM_CUDA(t, copy(T.frames, t->mid_frames, nb * sizeof(BodyFrame)));
    bce(t, t->MID, 0.5 * dt, 0);
    if (d.capM > 0 && d.n_bodies > 0) bce(t, t->MID, 0.5 * dt, 1, dt, 1);
    pair(t, kStage2, t->MID, t->A[c], (float)dt, r2);
    CRM_CUDA(t, copy_stage(T.YM, t->MID));
    if (nb > 0) CRM_CUDA(t, copy(T.after, t->bodies, nb * sizeof(BodyDev)));
    return CRM_OK;
}

// One step of the run recorded to tape slot T: a graph per slot and current
// buffer, captured at its first use and replayed for every later segment (the
// tape and working arrays it points into stay put), else direct launches.
int record_step(crm_terrain *t, double dt, crm_terrain::AdjTape &T, bool use_graph = true)
{
    const int par = t->cur;
    cudaGraphExec_t &G = T.rec[par];
    if (G && T.rec_dt != dt) {
        cudaGraphExecDestroy(G);
        G = nullptr;
    }
    if (!G && use_graph && t->graphs && t->cap_st && !t->timing) {
        cudaStream_t user = t->st;
        const crm_profile saved = t->prof;
        const bool lv = t->lists_valid;
        t->st = t->cap_st;
        cudaGraph_t g = nullptr;
        int rc = CRM_OK;
        cudaError_t e = cudaStreamBeginCapture(t->st, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            rc = enqueue_record(t, dt, T);
            e = cudaStreamEndCapture(t->st, &g);
        }
        t->cur = par;
        t->st = user;
        t->prof = saved;
        t->lists_valid = lv;
        if (e == cudaSuccess && rc == CRM_OK) e = cudaGraphInstantiate(&G, g, 0);
        if (g) cudaGraphDestroy(g);
        if (e != cudaSuccess || rc != CRM_OK) {
            cudaGetLastError();
            G = nullptr;
            t->msg.clear();
        }
        T.rec_dt = dt;
    }
    if (G) {
        CRM_CUDA(t, cudaGraphLaunch(G, t->st));
        t->cur = 1 - t->cur;        // the replayed rebuild's buffer swap
        t->lists_valid = true;
        t->prof.rebuilds += 1;
    } else {
        int rc = enqueue_record(t, dt, T);
        if (rc) return rc;
    }
    t->step_index += 1;
    t->time += dt;
    CRM_CUDA(t, cudaGetLastError());
    return CRM_OK;
}

// Reverse sweep of step s from its tape: the adjoint of y_{s+1} (insertion
// order, A.l_ins) and of the bodies after the step (A.lb[0]) become those of
// y_s and of the bodies before it.
int vjp_step(crm_terrain *t, const crm_terrain::AdjTape &T, int64_t s)
{
    const DevParams &d = t->dp;
    crm_terrain::Adjoint &A = t->adj;
    const int nb = (int)t->hbodies.size();
    const double dt = A.dt;
    const AdjStage Vm{T.YM, T.nbr, T.nnb, T.pid, t->mloc, T.bodies, T.frames, (int)t->nFtot,
                      T.sumM};
    const AdjStage V0{T.Y0, T.nbr, T.nnb, T.pid, t->mloc, T.bodies, nullptr, (int)t->nFtot,
                      T.sum0};
    const AdjIO io = adj_io(t, (float)dt);
    double *g0 = A.gbody, *gm = A.gbody + kBodyAdj * std::max(nb, 1);
    const double *lw = A.lw_obj ? A.lw_obj + (size_t)s * nb * 6 : nullptr;
    const double *lc = A.lc_obj ? A.lc_obj + (size_t)s * nb * 3 : nullptr;
    if (nb > 0) {
        launch(t, K_ADJ, [&] { launch_adj_body_pre(nb, T.bodies, T.after, dt, A.lb[0], lw, lc,
                                                   A.lwrench, A.lb[1], A.gbody, t->st); });
    }
    // stage 2 (at y_mid, with the wrench's marker accelerations)
    launch(t, K_ADJ, [&] { launch_adj_fluid_coef(kAdjStage2, d, Vm, T.Y0, io, A.gpar, t->st); });
    const bool acc = nb > 0 && d.capM > 0;
    launch(t, K_ADJ, [&] { launch_adj_marker(acc, d, Vm, io, A.gpar, gm, t->st, T.act, T.n_act); });
    launch(t, K_ADJ, [&] { launch_adj_fluid(acc, kAdjAccumulate, d, Vm, io, A.l_mid, nullptr,
                                            A.gpar, t->st); });
    // stage 1 (at y_n)
    launch(t, K_ADJ, [&] { launch_adj_fluid_coef(kAdjStage1, d, V0, T.Y0, io, A.gpar, t->st); });
    launch(t, K_ADJ, [&] { launch_adj_marker(false, d, V0, io, A.gpar, g0, t->st, T.act, T.n_act); });
    launch(t, K_ADJ, [&] { launch_adj_fluid(false, kAdjFinal, d, V0, io, A.l_y0, A.l_ins, A.gpar,
                                            t->st); });
    if (nb > 0) {
        launch(t, K_ADJ, [&] { launch_adj_body_post(nb, T.bodies, dt, g0, gm, A.lb[1], t->st); });
        std::swap(A.lb[0], A.lb[1]);
    }
    CRM_CUDA(t, cudaGetLastError());
    return CRM_OK;
}

// Restore checkpoint g of the recorded run into the working arrays, in stream
// order on the handle's stream: no host synchronisation, and no header read
// back (the checkpoint was written by crm_adjoint_forward on this terrain, in
// crm_save_state's layout, and the host kept its step index and time).
int restore_ckpt(crm_terrain *t, int64_t g)
{
    crm_terrain::Adjoint &A = t->adj;
    const int64_t n = t->nFtot + t->nMtot;
    const StageArrays S = t->A[t->cur];
    const char *b = A.ckpt + (size_t)g * A.ckpt_bytes;
    size_t o = 64;
    auto get = [&](void *dst, size_t nb) {
        cudaError_t e = cudaMemcpyAsync(dst, b + o, nb, cudaMemcpyDeviceToDevice, t->st);
        o += nb;
        return e;
    };
    CRM_CUDA(t, get(S.pos, n * sizeof(float4)));
    CRM_CUDA(t, get(S.vel, n * sizeof(float4)));
    CRM_CUDA(t, get(S.sA, n * sizeof(float4)));
    CRM_CUDA(t, get(S.sB, n * sizeof(float2)));
    CRM_CUDA(t, get(t->pid[t->cur], n * sizeof(uint32_t)));
    if (!t->hbodies.empty()) CRM_CUDA(t, get(t->bodies, t->hbodies.size() * sizeof(BodyDev)));
    t->step_index = A.ckpt_at[(size_t)g].first;
    t->time = A.ckpt_at[(size_t)g].second;
    t->lists_valid = false;
    t->have_working = false;
    CRM_CUDA(t, cudaMemsetAsync(t->abort_flag, 0, sizeof(int), t->st));
    CRM_CUDA(t, cudaMemsetAsync(t->err, 0, sizeof(int), t->st));
    t->frozen = false;
    return CRM_OK;
}

// Re-run segment g (from its checkpoint) into tape set `set` on the handle's stream.
int rerun_segment(crm_terrain *t, int64_t g, int set)
{
    crm_terrain::Adjoint &A = t->adj;
    const int64_t seg = A.every, s0 = g * A.every, s1 = std::min<int64_t>(A.n_steps, s0 + A.every);
    int rc = restore_ckpt(t, g);
    for (int64_t s = s0; s < s1 && rc == CRM_OK; ++s)
        rc = record_step(t, A.dt, A.tape[(size_t)(set * seg + (s - s0))]);
    return rc;
}

}  // namespace

extern "C" {

int crm_eval_rates_vjp(crm_terrain *t, int64_t cap_sph, const float *l_drho, const float *l_dvel,
                       const float *l_dstress, int64_t cap_markers, const float *l_macc,
                       double *g_xyz, double *g_vel, double *g_stress, double *g_rho,
                       double *g_body, double *g_params)
{
    if (!t) return CRM_EINVAL;
    if (t->frozen)
        return t->fail(CRM_ESTATE, "terrain frozen after a device wait gave up; crm_load_state a checkpoint");
    if (cap_sph < t->nFtot || (l_macc && cap_markers < t->nMtot))
        return t->fail(CRM_EINVAL, "crm_eval_rates_vjp: adjoint capacity too small");
    int rc = commit(t);
    if (rc) return rc;
    rc = adj_support(t, false, "crm_eval_rates_vjp");
    if (rc) return rc;
    rc = adj_workspace(t);
    if (rc) return rc;
    crm_terrain::Adjoint &A = t->adj;
    const int64_t nF = t->nFtot, nM = t->nMtot;
    // the rate adjoints, insertion order: drho [n], du [3n], dsigma [6n]
    std::vector<float> lr((size_t)10 * std::max<int64_t>(nF, 1), 0.0f);
    for (int64_t i = 0; i < nF; ++i) {
        if (l_drho) lr[i] = l_drho[i];
        for (int k = 0; k < 3; ++k) lr[nF + 3 * i + k] = l_dvel ? l_dvel[3 * i + k] : 0.0f;
        for (int k = 0; k < 6; ++k) lr[4 * nF + 6 * i + k] = l_dstress ? l_dstress[6 * i + k] : 0.0f;
    }
    CRM_CUDA(t, cudaMemcpyAsync(A.l_rate, lr.data(), lr.size() * sizeof(float), cudaMemcpyHostToDevice, t->st));
    if (l_macc && nM > 0)
        CRM_CUDA(t, cudaMemcpyAsync(A.l_macc, l_macc, 3 * nM * sizeof(float), cudaMemcpyHostToDevice, t->st));
    // the forward evaluation (lists, marker state) as crm_eval_rates runs it
    rebuild(t);
    const int c = t->cur;
    const DevParams &d = t->dp;
    const size_t wF = (size_t)std::max(d.capF, 1);
    void *buf = nullptr;
    CRM_CUDA(t, cudaMallocAsync(&buf, wF * (sizeof(float) + 2 * sizeof(float4) + sizeof(float2)) + 64, t->st));
    RateOut r{};
    r.du = (float4 *)buf;
    r.dsA = r.du + wF;
    r.dsB = (float2 *)(r.dsA + wF);
    r.drho = (float *)(r.dsB + wF);
    r.sums = A.sums;
    if (t->skin_on) {
        bce(t, t->A[c], 0.0, 0, 0.0, 0, true);
        pair(t, kEval, t->A[c], t->A[c], 0.0f, r, true);
        bce(t, t->A[c], 0.0, 2);
    } else {
        bce(t, t->A[c], 0.0, 2);
        pair(t, kEval, t->A[c], t->A[c], 0.0f, r);
    }
    cudaFreeAsync(buf, t->st);
    const size_t nb = t->hbodies.size();
    CRM_CUDA(t, cudaMemsetAsync(A.gpar, 0, kNumGradAcc * sizeof(double), t->st));
    CRM_CUDA(t, cudaMemsetAsync(A.gbody, 0, kBodyAdj * std::max<size_t>(nb, 1) * sizeof(double), t->st));
    const AdjStage V{t->A[c], t->nbr, t->nnb, t->pid[c], t->mloc, t->bodies, nullptr, (int)nF,
                     A.sums};
    AdjIO io = adj_io(t, 0.0f);
    io.l_macc = (l_macc && nM > 0) ? A.l_macc : nullptr;
    const bool acc = io.l_macc != nullptr;
    if (d.capF > 0) launch(t, K_ADJ, [&] { launch_adj_fluid_coef(kAdjEval, d, V, t->A[c], io, A.gpar, t->st); });
    if (d.capM > 0) {
        launch(t, K_ADJ, [&] { launch_adj_marker(acc, d, V, io, A.gpar, A.gbody, t->st); });
    }
    if (nF > 0)
        CRM_CUDA(t, cudaMemsetAsync(A.l_ins, 0, (size_t)kNumAdj * nF * sizeof(float), t->st));
    if (d.capF > 0)
        launch(t, K_ADJ, [&] { launch_adj_fluid(acc, kAdjFinal, d, V, io, A.l_y0, A.l_ins, A.gpar, t->st); });
    CRM_CUDA(t, cudaGetLastError());
    return adj_export(t, A.gbody, g_xyz, g_vel, g_stress, g_rho, g_body, g_params);
}

int crm_adjoint_forward(crm_terrain *t, double dt, int64_t n_steps, int32_t every,
                        double *wrench_hist, double *pose_hist)
{
    if (!t) return CRM_EINVAL;
    if (t->frozen)
        return t->fail(CRM_ESTATE, "terrain frozen after a device wait gave up; crm_load_state a checkpoint");
    if (!(dt > 0) || !std::isfinite(dt) || n_steps < 1 || every < 0)
        return t->fail(CRM_EINVAL, "crm_adjoint_forward: dt > 0, n_steps >= 1, every >= 0");
    int rc = commit(t);
    if (rc) return rc;
    rc = adj_support(t, true, "crm_adjoint_forward");
    if (rc) return rc;
    rc = adj_workspace(t);
    if (rc) return rc;
    crm_terrain::Adjoint &A = t->adj;
    A.n_steps = 0;
    const DevParams &d = t->dp;
    const size_t nb = t->hbodies.size();
    // every == 0: the whole run's tape stays resident (no checkpoints, no re-run)
    const bool resident = every == 0;
    // a run of the same shape reuses the tape and checkpoints allocated before
    const bool reuse = A.alloc_steps == n_steps && A.alloc_every == every && !A.tape.empty();
    if (!reuse) {
        drop_tape(t);
        A.alloc_steps = -1;
        A.alloc_every = -1;
    }
    size_t sb = 0;
    crm_state_bytes(t, &sb);
    A.ckpt_bytes = (sb + 255) / 256 * 256;
    A.n_ckpt = resident ? 0 : (int)((n_steps + every - 1) / every) + 1;
    if (!reuse) {
        A.ckpt = resident ? nullptr : t->dalloc<char>(G_TAPE, A.ckpt_bytes * A.n_ckpt);
        A.hist = t->dalloc<BodyDev>(G_TAPE, std::max<size_t>(nb, 1) * n_steps);
        A.lw_obj = t->dalloc<double>(G_TAPE, std::max<size_t>(nb, 1) * 6 * n_steps);
        A.lc_obj = t->dalloc<double>(G_TAPE, std::max<size_t>(nb, 1) * 3 * n_steps);
    }
    // the tape of the whole run when resident, else two tape sets of one segment
    // each (the backward re-runs one segment into a set while it sweeps the other)
    const int64_t seg = resident ? n_steps : std::min<int64_t>(every, n_steps);
    const int64_t slots = resident ? seg : 2 * seg;
    const size_t N = (size_t)std::max(d.capN, 1);
    for (int64_t k = reuse ? slots : 0; k < slots && !t->oom; ++k) {
        crm_terrain::AdjTape T = no_tape();
        for (StageArrays *S : {&T.Y0, &T.YM}) {
            S->pos = t->dalloc<float4>(G_TAPE, N);
            S->vel = t->dalloc<float4>(G_TAPE, N);
            S->sA = t->dalloc<float4>(G_TAPE, N);
            S->sB = t->dalloc<float2>(G_TAPE, N);
        }
        T.pid = t->dalloc<uint32_t>(G_TAPE, N);
        T.nbr = t->dalloc<uint32_t>(G_TAPE, (size_t)d.maxnb * d.ell);
        T.nnb = t->dalloc<uint32_t>(G_TAPE, N);
        T.act = t->dalloc<uint32_t>(G_TAPE, std::max<size_t>(d.capM, 1));
        T.act_body = t->dalloc<uint32_t>(G_TAPE, std::max(t->n_bodym, 1));
        T.n_act = t->dalloc<int>(G_TAPE, 2);
        T.bodies = t->dalloc<BodyDev>(G_TAPE, std::max<size_t>(nb, 1));
        T.frames = t->dalloc<BodyFrame>(G_TAPE, std::max<size_t>(nb, 1));
        T.after = t->dalloc<BodyDev>(G_TAPE, std::max<size_t>(nb, 1));
        T.sum0 = t->dalloc<float>(G_TAPE, 13 * (size_t)std::max(d.capF, 1));
        T.sumM = t->dalloc<float>(G_TAPE, 13 * (size_t)std::max(d.capF, 1));
        T.rec[0] = T.rec[1] = nullptr;
        T.rec_dt = 0.0;
        A.tape.push_back(T);
    }
    if (t->oom) {
        t->oom = false;
        drop_tape(t);
        return t->fail(CRM_ENOMEM, "crm_adjoint_forward: device allocation of the checkpoints and tape failed");
    }
    A.alloc_steps = n_steps;
    A.alloc_every = every;
    A.dt = dt;
    A.every = every;
    A.ckpt_at.assign(A.n_ckpt, {0, 0.0});
    size_t used = 0;
    for (int64_t s = 0; s < n_steps; ++s) {
        if (resident) {
            // each slot's recording graph is captured at its first use and replayed
            // by later runs of the same shape (the tape is reused)
            rc = record_step(t, dt, A.tape[(size_t)s]);
        } else {
            if (s % every == 0) {
                A.ckpt_at[(size_t)(s / every)] = {t->step_index, t->time};
                rc = crm_save_state(t, A.ckpt + (size_t)(s / every) * A.ckpt_bytes, A.ckpt_bytes, &used);
                if (rc) return rc;
            }
            rc = crm_step(t, dt, 1);
        }
        if (rc) return rc;
        if (nb > 0)
            CRM_CUDA(t, cudaMemcpyAsync(A.hist + (size_t)s * nb, t->bodies, nb * sizeof(BodyDev),
                                        cudaMemcpyDeviceToDevice, t->st));
    }
    // the recorded steps' lists are in the tape, not in the terrain's own table
    if (resident) t->lists_valid = false;
    if (!resident) {
        A.ckpt_at[(size_t)(A.n_ckpt - 1)] = {t->step_index, t->time};
        rc = crm_save_state(t, A.ckpt + (size_t)(A.n_ckpt - 1) * A.ckpt_bytes, A.ckpt_bytes, &used);
        if (rc) return rc;
    }
    rc = latched_error(t);
    if (rc) return rc;
    if (nb > 0 && (wrench_hist || pose_hist)) {
        std::vector<BodyDev> h(nb * n_steps);
        CRM_CUDA(t, cudaMemcpyAsync(h.data(), A.hist, h.size() * sizeof(BodyDev), cudaMemcpyDeviceToHost, t->st));
        CRM_CUDA(t, cudaStreamSynchronize(t->st));
        for (size_t q = 0; q < h.size(); ++q) {
            if (wrench_hist) std::memcpy(wrench_hist + 6 * q, h[q].wrench, 6 * sizeof(double));
            if (pose_hist) std::memcpy(pose_hist + 7 * q, h[q].pose, 7 * sizeof(double));
        }
    }
    A.n_steps = n_steps;
    return CRM_OK;
}

int crm_adjoint_backward(crm_terrain *t, const double *l_wrench, const double *l_center,
                         const double *l_xyz, const double *l_vel, const double *l_stress,
                         const double *l_rho, double *g_params, double *g_xyz, double *g_vel,
                         double *g_stress, double *g_rho, double *g_body)
{
    if (!t) return CRM_EINVAL;
    if (t->frozen)
        return t->fail(CRM_ESTATE, "terrain frozen after a device wait gave up; crm_load_state a checkpoint");
    crm_terrain::Adjoint &A = t->adj;
    if (!A.ready || A.n_steps < 1 || A.tape.empty())
        return t->fail(CRM_ESTATE, "crm_adjoint_backward: no run recorded by crm_adjoint_forward");
    const int64_t n = A.n_steps;
    const size_t nb = t->hbodies.size();
    if (nb > 0) {
        std::vector<double> w(nb * 6 * n, 0.0), c(nb * 3 * n, 0.0);
        if (l_wrench) std::memcpy(w.data(), l_wrench, w.size() * sizeof(double));
        if (l_center) std::memcpy(c.data(), l_center, c.size() * sizeof(double));
        CRM_CUDA(t, cudaMemcpyAsync(A.lw_obj, w.data(), w.size() * sizeof(double), cudaMemcpyHostToDevice, t->st));
        CRM_CUDA(t, cudaMemcpyAsync(A.lc_obj, c.data(), c.size() * sizeof(double), cudaMemcpyHostToDevice, t->st));
        CRM_CUDA(t, cudaMemsetAsync(A.lb[0], 0, kBodyAdj * nb * sizeof(double), t->st));
        // (the host copies above read pageable memory: finish them before the
        // vectors go out of scope)
        CRM_CUDA(t, cudaStreamSynchronize(t->st));
    }
    CRM_CUDA(t, cudaMemsetAsync(A.gpar, 0, kNumGradAcc * sizeof(double), t->st));
    const int64_t nF = t->nFtot;
    if (nF > 0) {
        // the objective's terms on the final SPH state (insertion order, component-major)
        std::vector<float> l((size_t)kNumAdj * nF, 0.0f);
        for (int64_t i = 0; i < nF; ++i) {
            for (int k = 0; k < 3; ++k) {
                if (l_xyz) l[(size_t)(kAdjX + k) * nF + i] = (float)l_xyz[3 * i + k];
                if (l_vel) l[(size_t)(kAdjU + k) * nF + i] = (float)l_vel[3 * i + k];
            }
            if (l_stress)
                for (int k = 0; k < 6; ++k) l[(size_t)(kAdjS + k) * nF + i] = (float)l_stress[6 * i + k];
            if (l_rho) l[(size_t)kAdjR * nF + i] = (float)l_rho[i];
        }
        CRM_CUDA(t, cudaMemcpyAsync(A.l_ins, l.data(), l.size() * sizeof(float), cudaMemcpyHostToDevice, t->st));
        CRM_CUDA(t, cudaStreamSynchronize(t->st));
    }
    if (A.every == 0) {
        // resident tape: the reverse sweep alone
        for (int64_t s = n - 1; s >= 0; --s) {
            int rc = vjp_step(t, A.tape[(size_t)s], s);
            if (rc) return rc;
        }
        return adj_export(t, A.lb[0], g_xyz, g_vel, g_stress, g_rho, g_body, g_params);
    }
    // Segments in reverse.  The handle's stream re-runs segment g - 1 into one
    // tape set while the sweep stream sweeps segment g from the other: the
    // sweep of g waits for its re-run, and the re-run of g - 1 waits for the
    // sweep of g + 1, which read the set it overwrites.
    if (!t->adj_st) {
        bool ok = cudaStreamCreateWithFlags(&t->adj_st, cudaStreamNonBlocking) == cudaSuccess;
        for (cudaEvent_t &e : t->adj_ev)
            ok = ok && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess;
        if (!ok) {
            cudaGetLastError();
            return t->fail(CRM_ECUDA, "crm_adjoint_backward: stream or event creation failed");
        }
    }
    cudaStream_t R = t->st, S = t->adj_st;
    cudaEvent_t *rerun_done = t->adj_ev, *swept = t->adj_ev + 2;
    const int64_t seg = A.every, n_seg = (n + A.every - 1) / A.every;
    // the sweep starts after the objective's adjoints and the accumulators are set
    CRM_CUDA(t, cudaEventRecord(swept[0], R));
    CRM_CUDA(t, cudaStreamWaitEvent(S, swept[0], 0));
    int rc = rerun_segment(t, n_seg - 1, (int)((n_seg - 1) % 2));
    if (rc) return rc;
    CRM_CUDA(t, cudaEventRecord(rerun_done[(n_seg - 1) % 2], R));
    for (int64_t g = n_seg - 1; g >= 0; --g) {
        const int set = (int)(g % 2);
        const int64_t s0 = g * A.every, s1 = std::min<int64_t>(n, s0 + A.every);
        CRM_CUDA(t, cudaStreamWaitEvent(S, rerun_done[set], 0));
        t->st = S;
        for (int64_t s = s1 - 1; s >= s0 && rc == CRM_OK; --s)
            rc = vjp_step(t, A.tape[(size_t)(set * seg + (s - s0))], s);
        t->st = R;
        if (rc) return rc;
        CRM_CUDA(t, cudaEventRecord(swept[set], S));
        if (g > 0) {
            CRM_CUDA(t, cudaStreamWaitEvent(R, swept[1 - set], 0));   // (the sweep of g + 1)
            rc = rerun_segment(t, g - 1, 1 - set);
            if (rc) return rc;
            CRM_CUDA(t, cudaEventRecord(rerun_done[1 - set], R));
        }
    }
    CRM_CUDA(t, cudaEventRecord(swept[0], S));
    CRM_CUDA(t, cudaStreamWaitEvent(R, swept[0], 0));
    // leave the terrain as the forward run left it
    size_t sb = 0;
    crm_state_bytes(t, &sb);
    rc = crm_load_state(t, A.ckpt + (size_t)(A.n_ckpt - 1) * A.ckpt_bytes, sb);
    if (rc) return rc;
    return adj_export(t, A.lb[0], g_xyz, g_vel, g_stress, g_rho, g_body, g_params);
}

}  // extern "C"
