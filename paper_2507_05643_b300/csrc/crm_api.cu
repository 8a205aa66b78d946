// crm_api.cu -- host side of the C ABI declared in include/crm.h.
//
// The handle keeps the inputs on the host until the first step, then
// "commits": sizes the grid, allocates every device array once and uploads
// the particles in insertion order; the first rebuild sorts them by cell.
// Each step enqueues the kernels of Alg. 2 (rebuild every ps_freq steps) and
// the two RK2 stages on the handle's stream.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "crm_internal.cuh"

using namespace crm;

struct crm_terrain {
    crm_params P{};
    cudaStream_t st = nullptr;
    std::string msg;

    // inputs, insertion order
    std::vector<double> hx, hu, hs, hr;          // SPH
    std::vector<double> hmloc;                   // marker body-frame / world coordinates
    std::vector<int> hmbody;                     // body of each marker, -1 fixed
    std::vector<BodyDev> hbodies;
    struct Box { int body; double half[3], off[3], t_delay; };
    std::vector<Box> boxes;

    bool committed = false;
    bool lists_valid = false;
    int64_t step_index = 0;
    double time = 0.0;
    int64_t nFtot = 0, nMtot = 0;
    DevParams dp{};

    // device state
    int cur = 0;
    StageArrays A[2]{}, MID{};
    uint32_t *pid[2]{};
    SortScratch ss{};
    uint32_t *start = nullptr, *nbr = nullptr, *nnb = nullptr;
    double *mloc = nullptr;
    int *mbody = nullptr;
    BodyDev *bodies = nullptr;
    float4 *mforce = nullptr, *mtorque = nullptr;
    double *partial = nullptr;
    int *err = nullptr;
    std::vector<void *> allocs;
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
    template <class T> T *dalloc(size_t count)
    {
        void *p = nullptr;
        if (cudaMalloc(&p, std::max<size_t>(count, 1) * sizeof(T)) != cudaSuccess) {
            cudaGetLastError();
            oom = true;
            return nullptr;
        }
        allocs.push_back(p);
        return (T *)p;
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
    if (p->kernel != CRM_KERNEL_CUBIC) return bad("kernel must be CRM_KERNEL_CUBIC");
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
    return CRM_OK;
}

// Grid and device constants (cells of size 2h over the domain, Sec. 3.1).
int make_devparams(crm_terrain *t)
{
    const crm_params &P = t->P;
    DevParams &d = t->dp;
    const double cell = 2.0 * P.h;
    int64_t G[3];
    for (int k = 0; k < 3; ++k) {
        G[k] = (int64_t)std::ceil((P.domain_max[k] - P.domain_min[k]) / cell);
        if (G[k] < 1) G[k] = 1;
    }
    if ((double)G[0] * (double)G[1] * (double)G[2] >= 4294967295.0)
        return t->fail(CRM_EINVAL, "grid of 2h cells over the domain exceeds 2^32 cells");
    const double Mw = (double)G[0] * G[1] * G[2];
    if (2.0 * Mw + 1.0 >= 2147483647.0)
        return t->fail(CRM_EINVAL, "grid too large for the cell sort (2M + 1 >= 2^31)");
    const double pi = 3.14159265358979323846;
    const double Gm = P.E / (2.0 * (1.0 + P.nu)), Km = P.E / (3.0 * (1.0 - 2.0 * P.nu));
    const double m = P.rho0 * P.d0 * P.d0 * P.d0;
    d.h = (float)P.h;
    d.inv_h = (float)(1.0 / P.h);
    d.four_h2 = (float)(4.0 * P.h * P.h);
    d.cell = (float)cell;
    d.kw = (float)(1.0 / (pi * P.h * P.h * P.h));
    d.kdw = (float)(1.0 / (pi * P.h * P.h * P.h * P.h));
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
    d.mu_s = (float)P.mu_s;
    d.mu_2 = (float)P.mu_2;
    d.I0 = (float)P.I0;
    d.grain_d = (float)P.grain_d;
    d.cohesion = (float)P.cohesion;
    d.GX = (int)G[0]; d.GY = (int)G[1]; d.GZ = (int)G[2];
    d.wx0 = d.wy0 = d.wz0 = 0;
    d.WX = d.GX; d.WY = d.GY; d.WZ = d.GZ;
    d.M = (uint32_t)(G[0] * G[1] * G[2]);
    d.dmin_x = P.domain_min[0];
    d.dmin_y = P.domain_min[1];
    d.dmin_z = P.domain_min[2];
    d.cell_d = cell;
    d.maxnb = P.max_neighbors;
    return CRM_OK;
}

bool inside_domain(const crm_params &P, const double *x)
{
    for (int k = 0; k < 3; ++k)
        if (!(x[k] >= P.domain_min[k] && x[k] < P.domain_max[k])) return false;
    return true;
}

int latched_error(crm_terrain *t)
{
    int e = 0;
    CRM_CUDA(t, cudaMemcpyAsync(&e, t->err, sizeof(int), cudaMemcpyDeviceToHost, t->st));
    CRM_CUDA(t, cudaStreamSynchronize(t->st));
    if (e == 0) return CRM_OK;
    CRM_CUDA(t, cudaMemsetAsync(t->err, 0, sizeof(int), t->st));
    if (e & ERR_NONFINITE) return t->fail(CRM_ENONFINITE, "the particle state became non-finite");
    if (e & ERR_ESCAPED) return t->fail(CRM_EESCAPED, "a particle or marker left the grid domain");
    if (e & ERR_CAPACITY)
        return t->fail(CRM_ECAPACITY, "a neighbour list exceeded max_neighbors");
    return t->fail(CRM_ETIMEOUT, "a bounded device-side wait gave up");
}

int commit(crm_terrain *t)
{
    if (t->committed) return CRM_OK;
    const int64_t nF = t->nFtot, nM = t->nMtot, N = nF + nM;
    if (N >= (int64_t)kIndexMask)
        return t->fail(CRM_EINVAL, "more than 2^26 particles and markers in one terrain");
    int rc = make_devparams(t);
    if (rc) return rc;
    DevParams &d = t->dp;
    d.nF = (int)nF;
    d.nM = (int)nM;
    d.N = (int)N;
    d.ell = (uint32_t)std::max<int64_t>(N, 1);
    d.n_bodies = (int)t->hbodies.size();
    const size_t nk = 2 * (size_t)d.M + 1;

    for (int b = 0; b < 2; ++b) {
        t->A[b].pos = t->dalloc<float4>(N);
        t->A[b].vel = t->dalloc<float4>(N);
        t->A[b].sA = t->dalloc<float4>(N);
        t->A[b].sB = t->dalloc<float2>(N);
        t->pid[b] = t->dalloc<uint32_t>(N);
    }
    t->MID.pos = t->dalloc<float4>(N);
    t->MID.vel = t->dalloc<float4>(N);
    t->MID.sA = t->dalloc<float4>(N);
    t->MID.sB = t->dalloc<float2>(N);
    t->ss.keys = t->dalloc<uint32_t>(N);
    t->ss.rank = t->dalloc<uint32_t>(N);
    t->ss.tmp = t->dalloc<uint32_t>(N);
    t->ss.count = t->dalloc<uint32_t>(nk);
    t->ss.n_tiles = ((int64_t)nk + kScanTile - 1) / kScanTile;
    t->ss.tile_status = t->dalloc<unsigned long long>(t->ss.n_tiles);
    t->ss.ctr = t->dalloc<uint32_t>(4);
    t->start = t->dalloc<uint32_t>(nk);
    t->nbr = t->dalloc<uint32_t>((size_t)d.maxnb * d.ell);
    t->nnb = t->dalloc<uint32_t>(N);
    t->mloc = t->dalloc<double>(3 * nM);
    t->mbody = t->dalloc<int>(nM);
    t->bodies = t->dalloc<BodyDev>(t->hbodies.size());
    t->mforce = t->dalloc<float4>(nM);
    t->mtorque = t->dalloc<float4>(nM);
    t->partial = t->dalloc<double>((size_t)grid_for(nM) * std::max<size_t>(t->hbodies.size(), 1) * 6);
    t->err = t->dalloc<int>(1);
    if (t->oom) return t->fail(CRM_ENOMEM, "device allocation failed");

    // initial state in insertion order: SPH first, then markers
    std::vector<float4> pos(N), vel(N), sA(N);
    std::vector<float2> sB(N);
    std::vector<uint32_t> pid(N);
    const double cell = d.cell_d;
    for (int64_t i = 0; i < nF; ++i) {
        const double *x = &t->hx[3 * i];
        int c[3];
        float o[3];
        const double dm[3] = {d.dmin_x, d.dmin_y, d.dmin_z};
        for (int k = 0; k < 3; ++k) {
            c[k] = (int)std::floor((x[k] - dm[k]) / cell);
            o[k] = (float)(x[k] - (dm[k] + c[k] * cell));
        }
        const uint32_t g = ((uint32_t)c[2] * (uint32_t)d.GY + (uint32_t)c[1]) * (uint32_t)d.GX
                           + (uint32_t)c[0];
        uint32_t gb;
        std::memcpy(&gb, &g, 4);
        float gf;
        std::memcpy(&gf, &gb, 4);
        pos[i] = make_float4(o[0], o[1], o[2], gf);
        vel[i] = make_float4((float)t->hu[3 * i], (float)t->hu[3 * i + 1], (float)t->hu[3 * i + 2],
                             (float)t->hr[i]);
        const double *s = &t->hs[6 * i];
        sA[i] = make_float4((float)s[0], (float)s[1], (float)s[2], (float)s[3]);
        sB[i] = make_float2((float)s[4], (float)s[5]);
        pid[i] = (uint32_t)i;
    }
    for (int64_t a = 0; a < nM; ++a) {
        pos[nF + a] = make_float4(0.f, 0.f, 0.f, 0.f);
        vel[nF + a] = make_float4(0.f, 0.f, 0.f, (float)t->P.rho0);
        sA[nF + a] = make_float4(0.f, 0.f, 0.f, 0.f);
        sB[nF + a] = make_float2(0.f, 0.f);
        pid[nF + a] = (uint32_t)(nF + a);
    }
    cudaStream_t st = t->st;
    const int c = t->cur;
    CRM_CUDA(t, cudaMemcpyAsync(t->A[c].pos, pos.data(), N * sizeof(float4), cudaMemcpyHostToDevice, st));
    CRM_CUDA(t, cudaMemcpyAsync(t->A[c].vel, vel.data(), N * sizeof(float4), cudaMemcpyHostToDevice, st));
    CRM_CUDA(t, cudaMemcpyAsync(t->A[c].sA, sA.data(), N * sizeof(float4), cudaMemcpyHostToDevice, st));
    CRM_CUDA(t, cudaMemcpyAsync(t->A[c].sB, sB.data(), N * sizeof(float2), cudaMemcpyHostToDevice, st));
    CRM_CUDA(t, cudaMemcpyAsync(t->pid[c], pid.data(), N * sizeof(uint32_t), cudaMemcpyHostToDevice, st));
    if (nM) {
        CRM_CUDA(t, cudaMemcpyAsync(t->mloc, t->hmloc.data(), 3 * nM * sizeof(double),
                                    cudaMemcpyHostToDevice, st));
        CRM_CUDA(t, cudaMemcpyAsync(t->mbody, t->hmbody.data(), nM * sizeof(int),
                                    cudaMemcpyHostToDevice, st));
    }
    if (!t->hbodies.empty())
        CRM_CUDA(t, cudaMemcpyAsync(t->bodies, t->hbodies.data(), t->hbodies.size() * sizeof(BodyDev),
                                    cudaMemcpyHostToDevice, st));
    CRM_CUDA(t, cudaMemsetAsync(t->ss.count, 0, nk * sizeof(uint32_t), st));
    CRM_CUDA(t, cudaMemsetAsync(t->ss.tile_status, 0, t->ss.n_tiles * sizeof(unsigned long long), st));
    CRM_CUDA(t, cudaMemsetAsync(t->ss.ctr, 0, 4 * sizeof(uint32_t), st));
    CRM_CUDA(t, cudaMemsetAsync(t->nnb, 0, N * sizeof(uint32_t), st));
    CRM_CUDA(t, cudaMemsetAsync(t->err, 0, sizeof(int), st));
    CRM_CUDA(t, cudaMemsetAsync(t->mforce, 0, std::max<int64_t>(nM, 1) * sizeof(float4), st));
    // the host staging vectors die at return: wait for the copies
    CRM_CUDA(t, cudaStreamSynchronize(st));
    t->committed = true;
    t->lists_valid = false;
    return CRM_OK;
}

enum KernelId { K_KEYS, K_SCAN, K_SCATTER, K_REORDER, K_NEIGHBORS, K_BCE, K_PAIR1, K_PAIR2,
                K_WRENCH, K_BODY, K_EXPORT };
const char *const kKernelNames[CRM_NUM_KERNELS] = {
    "keys", "scan", "scatter", "reorder", "neighbors", "bce", "pair_stage1", "pair_stage2",
    "wrench_partial", "body_update", "export"};

// Enqueue one kernel through `launch`, counting it and, when timing is on,
// bracketing it with two events on the handle's stream.
template <class F> void launch(crm_terrain *t, int k, F &&f)
{
    t->prof.launches[k] += 1;
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

void rebuild(crm_terrain *t)
{
    const int c = t->cur, n = 1 - c;
    const DevParams &d = t->dp;
    if (d.N > 0) {
        launch(t, K_KEYS, [&] { launch_keys(d, t->A[c], t->pid[c], t->mloc, t->mbody, t->bodies,
                                            t->ss, t->err, (int)t->nFtot, t->st); });
        launch(t, K_SCAN, [&] { launch_scan_reset(t->ss.count, t->start, 2 * (int64_t)d.M + 1,
                                                  t->ss, t->err, t->st); });
        launch(t, K_SCATTER, [&] { launch_scatter(d, t->ss, t->start, t->st); });
        launch(t, K_REORDER, [&] { launch_reorder(d, t->ss, t->start, t->A[c], t->pid[c], t->A[n],
                                                  t->pid[n], t->st); });
        launch(t, K_NEIGHBORS,
               [&] { launch_neighbors(d, t->A[n].pos, t->start, t->nbr, t->nnb, t->err, t->st); });
    }
    t->cur = n;
    t->lists_valid = true;
    t->prof.rebuilds += 1;
}

void bce(crm_terrain *t, StageArrays S, double tau, int accel)
{
    const DevParams &d = t->dp;
    if (d.nM == 0) return;
    const int c = t->cur;
    launch(t, K_BCE, [&] { launch_bce(d, S, t->A[c].pos, t->pid[c], t->mloc, t->mbody, t->bodies,
                                      t->nbr, t->nnb, tau, accel, (int)t->nFtot, t->mforce,
                                      t->mtorque, t->st); });
}

void pair(crm_terrain *t, int mode, StageArrays S, StageArrays Y, float dt, RateOut out)
{
    const DevParams &d = t->dp;
    if (d.nF == 0) return;
    const int k = mode == kStage2 ? K_PAIR2 : K_PAIR1;
    launch(t, k, [&] { launch_pair(mode, d, S, Y, t->MID, t->nbr, t->nnb, nullptr, dt, out, t->err,
                                   t->st); });
}

void wrench(crm_terrain *t, double dt, int integrate)
{
    const DevParams &d = t->dp;
    if (d.n_bodies == 0) return;
    if (d.nM > 0)
        launch(t, K_WRENCH, [&] { launch_wrench_partial(d, t->mforce, t->mtorque, t->partial, t->st); });
    launch(t, K_BODY, [&] { launch_body_update(d, t->partial, t->bodies, dt, integrate, t->st); });
}

void one_step(crm_terrain *t, double dt)
{
    const int ps = t->P.ps_freq;
    if (!t->lists_valid || t->step_index % ps == 0) rebuild(t);
    const int c = t->cur;
    RateOut none{};
    bce(t, t->A[c], 0.0, 0);
    pair(t, kStage1, t->A[c], t->A[c], (float)dt, none);
    bce(t, t->MID, 0.5 * dt, 1);
    pair(t, kStage2, t->MID, t->A[c], (float)dt, none);
    wrench(t, dt, 1);
    t->step_index += 1;
    t->time += dt;
    t->prof.steps += 1;
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
    for (void *p : t->allocs)
        if (p) cudaFree(p);
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
    if (!(mass > 0) || (dof_mask & ~7)) return t->fail(CRM_EINVAL, "crm_add_rigid_body: mass > 0, dof_mask in 0..7");
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
    b.dof = dof_mask;
    const int id = (int)t->hbodies.size();
    t->hbodies.push_back(b);
    t->hmloc.insert(t->hmloc.end(), xloc, xloc + 3 * n);
    t->hmbody.insert(t->hmbody.end(), (size_t)n, id);
    t->nMtot += n;
    if (body_id) *body_id = id;
    return CRM_OK;
}

int crm_set_body_motion(crm_terrain *t, int32_t body, const double pose[7], const double twist[6])
{
    if (!t) return CRM_EINVAL;
    if (body < 0 || body >= (int)t->hbodies.size() || !pose || !twist)
        return t->fail(CRM_EINVAL, "crm_set_body_motion: bad body or null array");
    if (!finite_all(pose, 7) || !finite_all(twist, 6)) return t->fail(CRM_EINVAL, "non-finite motion");
    BodyDev &b = t->hbodies[body];
    for (int k = 0; k < 7; ++k) b.pose[k] = pose[k];
    for (int k = 0; k < 6; ++k) b.twist[k] = twist[k];
    if (t->committed)
        CRM_CUDA(t, cudaMemcpyAsync(&t->bodies[body], &b, 13 * sizeof(double),
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
    return t->fail(CRM_EINVAL, "crm_add_active_box: active domains are not available in this build");
}

int crm_step(crm_terrain *t, double dt, int32_t n_steps)
{
    if (!t) return CRM_EINVAL;
    if (!(dt > 0) || !std::isfinite(dt) || n_steps < 0) return t->fail(CRM_EINVAL, "crm_step: dt > 0, n_steps >= 0");
    int rc = commit(t);
    if (rc) return rc;
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
    double *dx = nullptr;
    float *dv = nullptr, *ds = nullptr, *dr = nullptr;
    const size_t bytes = n * (3 * sizeof(double) + 10 * sizeof(float));
    void *buf = nullptr;
    CRM_CUDA(t, cudaMallocAsync(&buf, std::max<size_t>(bytes, 16), t->st));
    dx = (double *)buf;
    dv = (float *)(dx + 3 * n);
    ds = dv + 3 * n;
    dr = ds + 6 * n;
    if (n > 0)
        launch(t, K_EXPORT, [&] { launch_export(t->dp, t->A[t->cur], t->pid[t->cur], dx, dv, ds, dr,
                                                t->st); });
    int rc = download(t, xyz, dx, 3 * n);
    if (!rc) rc = download(t, vel, dv, 3 * n);
    if (!rc) rc = download(t, stress6, ds, 6 * n);
    if (!rc) rc = download(t, rho, dr, n);
    cudaFreeAsync(buf, t->st);
    if (rc) return rc;
    return latched_error(t);
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
    if (n_active) *n_active = t->nFtot;
    if (n_extended) *n_extended = 0;
    if (n_bce) *n_bce = t->nMtot;
    return CRM_OK;
}

int crm_eval_rates(crm_terrain *t, int64_t cap_sph, float *drho, float *dvel, float *dstress,
                   int64_t cap_markers, float *marker_acc, float *marker_vel, float *marker_stress)
{
    if (!t) return CRM_EINVAL;
    if (cap_sph < t->nFtot || cap_markers < t->nMtot)
        return t->fail(CRM_EINVAL, "crm_eval_rates: output capacity too small");
    int rc = commit(t);
    if (rc) return rc;
    rebuild(t);
    const int c = t->cur;
    const DevParams &d = t->dp;
    const int64_t nF = t->nFtot, nM = t->nMtot;
    // rates in slot order, then insertion-order outputs, in one device block
    const size_t rate_bytes = nF * (sizeof(float) + 2 * sizeof(float4) + sizeof(float2));
    const size_t out_bytes = (nF * 10 + nM * 12) * sizeof(float);
    void *buf = nullptr;
    CRM_CUDA(t, cudaMallocAsync(&buf, std::max<size_t>(rate_bytes + out_bytes + 64, 64), t->st));
    char *b = (char *)buf;
    RateOut r;
    r.du = (float4 *)b;
    r.dsA = r.du + nF;
    r.dsB = (float2 *)(r.dsA + nF);
    r.drho = (float *)(r.dsB + nF);
    float *o = r.drho + nF;
    float *odrho = o, *odu = o + nF, *ods = odu + 3 * nF, *omacc = ods + 6 * nF,
          *omvel = omacc + 3 * nM, *omsig = omvel + 3 * nM;
    bce(t, t->A[c], 0.0, 2);
    pair(t, kEval, t->A[c], t->A[c], 0.0f, r);
    if (d.N > 0)
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
    const int64_t N = d.N;
    std::vector<uint32_t> nnb(N), pid(N), tab((size_t)d.maxnb * d.ell);
    int rc = download(t, nnb.data(), t->nnb, N);
    if (!rc) rc = download(t, pid.data(), t->pid[t->cur], N);
    if (!rc) rc = download(t, tab.data(), t->nbr, tab.size());
    if (rc) return rc;
    rc = latched_error(t);
    if (rc) return rc;
    std::vector<int64_t> cnt(N + 1, 0);
    for (int64_t s = 0; s < N; ++s) cnt[pid[s] + 1] = nnb[s];
    for (int64_t i = 0; i < N; ++i) cnt[i + 1] += cnt[i];
    if (nnz) *nnz = cnt[N];
    if (offset) std::memcpy(offset, cnt.data(), (N + 1) * sizeof(int64_t));
    if (!list) return CRM_OK;
    if (cap < cnt[N]) return t->fail(CRM_EINVAL, "crm_get_neighbors: list capacity too small");
    for (int64_t s = 0; s < N; ++s) {
        const int64_t o = cnt[pid[s]];
        for (uint32_t k = 0; k < nnb[s]; ++k)
            list[o + k] = (int32_t)pid[tab[(size_t)k * d.ell + s] & kIndexMask];
        std::sort(list + o, list + o + nnb[s]);
    }
    return CRM_OK;
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
    return CRM_OK;
}

int crm_profile_read(crm_terrain *t, crm_profile *out)
{
    if (!t || !out) return CRM_EINVAL;
    if (t->committed) CRM_CUDA(t, cudaStreamSynchronize(t->st));
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

int crm_state_bytes(crm_terrain *t, size_t *bytes)
{
    if (!t || !bytes) return CRM_EINVAL;
    const int64_t N = t->nFtot + t->nMtot;
    *bytes = 64 + N * (3 * sizeof(float4) + sizeof(float2) + sizeof(uint32_t))
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
    const int64_t N = t->dp.N;
    const int c = t->cur;
    char *b = (char *)dev_buf;
    int64_t hdr[4] = {t->step_index, 0, N, (int64_t)t->hbodies.size()};
    std::memcpy(&hdr[1], &t->time, sizeof(double));
    CRM_CUDA(t, cudaMemcpyAsync(b, hdr, sizeof(hdr), cudaMemcpyHostToDevice, t->st));
    size_t o = 64;
    auto put = [&](const void *src, size_t n) {
        cudaError_t e = cudaMemcpyAsync(b + o, src, n, cudaMemcpyDeviceToDevice, t->st);
        o += n;
        return e;
    };
    CRM_CUDA(t, put(t->A[c].pos, N * sizeof(float4)));
    CRM_CUDA(t, put(t->A[c].vel, N * sizeof(float4)));
    CRM_CUDA(t, put(t->A[c].sA, N * sizeof(float4)));
    CRM_CUDA(t, put(t->A[c].sB, N * sizeof(float2)));
    CRM_CUDA(t, put(t->pid[c], N * sizeof(uint32_t)));
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
    int64_t hdr[4];
    CRM_CUDA(t, cudaMemcpyAsync(hdr, dev_buf, sizeof(hdr), cudaMemcpyDeviceToHost, t->st));
    CRM_CUDA(t, cudaStreamSynchronize(t->st));
    if (hdr[2] != t->dp.N || hdr[3] != (int64_t)t->hbodies.size())
        return t->fail(CRM_EINVAL, "crm_load_state: checkpoint of a different terrain");
    const int64_t N = t->dp.N;
    const int c = t->cur;
    const char *b = (const char *)dev_buf;
    size_t o = 64;
    auto get = [&](void *dst, size_t n) {
        cudaError_t e = cudaMemcpyAsync(dst, b + o, n, cudaMemcpyDeviceToDevice, t->st);
        o += n;
        return e;
    };
    CRM_CUDA(t, get(t->A[c].pos, N * sizeof(float4)));
    CRM_CUDA(t, get(t->A[c].vel, N * sizeof(float4)));
    CRM_CUDA(t, get(t->A[c].sA, N * sizeof(float4)));
    CRM_CUDA(t, get(t->A[c].sB, N * sizeof(float2)));
    CRM_CUDA(t, get(t->pid[c], N * sizeof(uint32_t)));
    if (!t->hbodies.empty()) CRM_CUDA(t, get(t->bodies, t->hbodies.size() * sizeof(BodyDev)));
    t->step_index = hdr[0];
    std::memcpy(&t->time, &hdr[1], sizeof(double));
    t->lists_valid = false;
    CRM_CUDA(t, cudaStreamSynchronize(t->st));
    return CRM_OK;
}

}  // extern "C"
