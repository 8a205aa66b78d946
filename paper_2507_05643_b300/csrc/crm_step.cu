// crm_step.cu -- per-stage kernels of the SPH continuum step (Sec. 2.1-2.4).
//
// One step (explicit midpoint, Sec. 2.2) runs (k_bce in crm_bce.cu)
//   k_bce(tau = 0)          marker velocity / stress from the fluid at y_n
//   k_pair<kStage1>         rates f(y_n) of every fluid particle, fused with
//                           y_mid = y_n + dt/2 f(y_n)
//   k_bce(tau = dt/2)       markers at the midpoint, their accelerations, the
//                           per-block FP64 force / torque partials
//   k_pair<kStage2>         rates f(y_mid), fused with y_{n+1} = y_n + dt f(y_mid)
//                           and the return map of Sec. 2.3
//                           (the last block sums the FP64 wrench and moves the bodies)
// Every particle owns its outputs (gather form): no float atomics, so a step
// is bitwise reproducible.
#include <algorithm>

#include "crm_internal.cuh"

namespace crm {


// Stress rate from the velocity gradient L (L_ab = du_a/dx_b), Eqs.
// stress_rate_hypoelastic / stress_rate_jaumann / stress_rate:
//   dsigma = Omega sigma - sigma Omega + 2G (eps - tr(eps)/3 I) + K tr(eps) I,
//   eps = (L + L^T)/2, Omega = (L - L^T)/2.
// s and out are (xx, yy, zz, xy, xz, yz).
__device__ __forceinline__ void stress_rate(const float L[9], const float s[6], float G, float K,
                                            float out[6])
{
    const float a = 0.5f * (L[1] - L[3]);   // Omega_xy
    const float b = 0.5f * (L[2] - L[6]);   // Omega_xz
    const float c = 0.5f * (L[5] - L[7]);   // Omega_yz
    const float exx = L[0], eyy = L[4], ezz = L[8];
    const float exy = 0.5f * (L[1] + L[3]), exz = 0.5f * (L[2] + L[6]), eyz = 0.5f * (L[5] + L[7]);
    const float tr = exx + eyy + ezz;
    const float iso = (K - 2.0f * G / 3.0f) * tr;
    const float G2 = 2.0f * G;
    out[0] = 2.0f * (a * s[3] + b * s[4]) + G2 * exx + iso;
    out[1] = 2.0f * (c * s[5] - a * s[3]) + G2 * eyy + iso;
    out[2] = -2.0f * (b * s[4] + c * s[5]) + G2 * ezz + iso;
    out[3] = a * (s[1] - s[0]) + b * s[5] + c * s[4] + G2 * exy;
    out[4] = b * (s[2] - s[0]) + a * s[5] - c * s[3] + G2 * exz;
    out[5] = c * (s[2] - s[1]) - a * s[4] - b * s[3] + G2 * eyz;
}

__device__ __forceinline__ float taubar(const float s[6])
{
    const float p = -(s[0] + s[1] + s[2]) * (1.0f / 3.0f);
    const float t0 = s[0] + p, t1 = s[1] + p, t2 = s[2] + p;
    return sqrtf(0.5f * (t0 * t0 + t1 * t1 + t2 * t2)
                 + (s[3] * s[3] + s[4] * s[4] + s[5] * s[5]));
}

// Return map of Sec. 2.3 on the trial stress s (in place); sn = stress at t_n
// (for the mu(I) shear rate).
__device__ __forceinline__ void return_map(float s[6], const float sn[6], const DevParams &p,
                                           float dt)
{
    const float ps = -(s[0] + s[1] + s[2]) * (1.0f / 3.0f);
    // Step 1: tension cut-off at p_cri = -c / mu_s
    if (p.mu_s > 0.0f && ps < -p.cohesion / p.mu_s) {
        for (int k = 0; k < 6; ++k) s[k] = 0.0f;
        return;
    }
    const float tb = taubar(s);
    // Step 2: mu(I); with mu_2 = mu_s the rate term vanishes
    float mu = p.mu_s;
    if (p.mu_2 != p.mu_s) {
        const float gdot = (tb - taubar(sn)) / (p.G * dt);
        if (gdot > 0.0f && ps > 0.0f) {
            const float I = gdot * p.grain_d * sqrtf(p.rho0 / ps);
            mu = p.mu_s + (p.mu_2 - p.mu_s) / (1.0f + p.I0 / I);
        }
    }
    // Step 3: admissible trial stress is kept
    const float tmax = mu * ps + p.cohesion;
    if (tb <= tmax) return;
    // Step 4: radial return in deviatoric space, pressure kept
    const float f = tmax / tb;
    s[0] = -ps + f * (s[0] + ps);
    s[1] = -ps + f * (s[1] + ps);
    s[2] = -ps + f * (s[2] + ps);
    s[3] *= f; s[4] *= f; s[5] *= f;
}

// Pair sums of fluid particle i (Eqs. continuity_dis, momentum_dis, the
// artificial viscosity of Sec. 2.2 and the F2 velocity gradient), then the
// stage epilogue.  Neighbours j are fluid particles and BCE markers, whose
// velocity/stress slots hold the extrapolated marker state and whose density
// slot holds rho0.  V_j = m / rho_j.

constexpr int kPairBlock = 128;   // pair kernels: blocks of 128 threads
constexpr int kPairLanes = 2;     // lanes per fluid particle in the pair kernels

// Running sums of one particle's pairs.  The momentum sum of Eq. momentum_dis,
// sum_j V_j (sigma_i + sigma_j) . grad_i W_ij, is kept as sum_j sigma_j . (V_j
// grad_i W_ij) (mx, my, mz) and G = sum_j V_j grad_i W_ij, so that sigma_i . G is
// added once per particle; the continuity sum sum_j V_j u_ji . grad_i W_ij is the
// trace of the velocity-gradient sum L.
struct PairAcc {
    float mx, my, mz, Gx, Gy, Gz, avx, avy, avz;
    float L[9];
};

// One pair (i, j) with r = x_i - x_j, 0 < |r| < 2h, added to the sums of i.
// V_j grad_i W_ij is formed once, so every sum is a chain of FMAs.  KAV =
// 3 kernel + viscosity mode (compile-time, so the pair carries no mode tests);
// the spline's two pieces and the unilateral switch are selects, not branches
// (the lanes of a warp do not diverge on them).
template <int KAV>
__device__ __forceinline__ void pair_terms(const DevParams &p, const float4 &vi, const float4 &ai,
                                           const float2 &bi, const float4 &vj, const float4 &aj,
                                           const float2 &bj, float rx, float ry, float rz,
                                           float r2, PairAcc &A)
{
    constexpr int KER = KAV / 3, AV = KAV % 3;
    // (a pair at r = 0 -- two particles at one point -- adds nothing: r = 0 makes
    // every term vanish once 1/r is kept finite)
    const float rinv = rsqrtf(fmaxf(r2, 1e-30f));
    const float q = r2 * rinv * p.inv_h;
    float f;
    if (KER == CRM_KERNEL_WENDLAND) {
        // dW/dr = -5 a q (1 - q/2)^3 / h, so (dW/dr) / r = -5 a (1 - q/2)^3 / h^2
        const float t = 1.0f - 0.5f * q;
        f = p.kdw * t * t * t;
    } else {
        const float t = 2.0f - q;
        const float inner = p.kdw * q * (2.25f * q - 3.0f);
        const float outer = -0.75f * p.kdw * t * t;
        f = (q < 1.0f ? inner : outer) * rinv;
    }
    const float Vj = __fdividef(p.m, vj.w);   // MUFU reciprocal: ~2 ulp
    const float fv = f * Vj;
    const float gx = fv * rx, gy = fv * ry, gz = fv * rz;       // V_j grad_i W_ij
    const float ux = vj.x - vi.x, uy = vj.y - vi.y, uz = vj.z - vi.z;   // u_ji
    // momentum (F3): sigma_j . grad W here, sigma_i . sum grad W in the epilogue
    A.Gx += gx; A.Gy += gy; A.Gz += gz;
    A.mx = fmaf(aj.x, gx, fmaf(aj.w, gy, fmaf(bj.x, gz, A.mx)));
    A.my = fmaf(aj.w, gx, fmaf(aj.y, gy, fmaf(bj.y, gz, A.my)));
    A.mz = fmaf(bj.x, gx, fmaf(bj.y, gy, fmaf(aj.z, gz, A.mz)));
    // velocity gradient (F2): L += u_ji (x) V_j grad W; continuity (F2) is its trace
    A.L[0] = fmaf(ux, gx, A.L[0]); A.L[1] = fmaf(ux, gy, A.L[1]); A.L[2] = fmaf(ux, gz, A.L[2]);
    A.L[3] = fmaf(uy, gx, A.L[3]); A.L[4] = fmaf(uy, gy, A.L[4]); A.L[5] = fmaf(uy, gz, A.L[5]);
    A.L[6] = fmaf(uz, gx, A.L[6]); A.L[7] = fmaf(uz, gy, A.L[7]); A.L[8] = fmaf(uz, gz, A.L[8]);
    // artificial viscosity: v_ij . r_ij = -(u_ji . r_ij), along grad W = f r
    if (AV != CRM_AV_NONE) {
        const float vr = -(ux * rx + uy * ry + uz * rz);
        float fa = f * __fdividef(2.0f * p.av_c * vr, (vi.w + vj.w) * (r2 + p.xi2));
        if (AV == CRM_AV_UNILATERAL) fa = vr < 0.0f ? fa : 0.0f;
        A.avx = fmaf(fa, rx, A.avx);
        A.avy = fmaf(fa, ry, A.avy);
        A.avz = fmaf(fa, rz, A.avz);
    }
}

// Stage epilogue of fluid particle i from its pair sums A: the rates (the
// F2 / F3 sums, gravity, the Jaumann stress rate), then per MODE the rates
// themselves (kEval), y_mid = y_n + dt/2 f(y_n) (kStage1), or
// y_{n+1} = y_n + dt f(y_mid) with the return map of Sec. 2.3 (kStage2; S holds
// y_mid and Y holds y_n of particle i).
template <int MODE>
__device__ __forceinline__ void stage_epilogue(const DevParams &p, int i, const float4 &pi,
                                               const float4 &vi, const float4 &ai,
                                               const float2 &bi, const PairAcc &A, StageArrays S,
                                               StageArrays Y, StageArrays MID, float dt,
                                               RateOut out, int *__restrict__ err,
                                               const float4 *__restrict__ xref,
                                               int *__restrict__ gate)
{
    const float si[6] = {ai.x, ai.y, ai.z, ai.w, bi.x, bi.y};
    const float cont = A.L[0] + A.L[4] + A.L[8];
    const float mx = fmaf(si[0], A.Gx, fmaf(si[3], A.Gy, fmaf(si[4], A.Gz, A.mx)));
    const float my = fmaf(si[3], A.Gx, fmaf(si[1], A.Gy, fmaf(si[5], A.Gz, A.my)));
    const float mz = fmaf(si[4], A.Gx, fmaf(si[5], A.Gy, fmaf(si[2], A.Gz, A.mz)));
    if (out.sums != nullptr) {
        const size_t cs = (size_t)p.capF;
        out.sums[i] = cont;
        out.sums[cs + i] = mx;
        out.sums[2 * cs + i] = my;
        out.sums[3 * cs + i] = mz;
#pragma unroll
        for (int k = 0; k < 9; ++k) out.sums[(4 + k) * cs + i] = A.L[k];
    }
    const float rinv_i = 1.0f / vi.w;
    const float drho = -vi.w * cont;
    const float dux = mx * rinv_i + p.gx + A.avx;
    const float duy = my * rinv_i + p.gy + A.avy;
    const float duz = mz * rinv_i + p.gz + A.avz;
    float ds[6];
    stress_rate(A.L, si, p.G, p.K, ds);
    if (MODE == kEval) {
        out.drho[i] = drho;
        out.du[i] = make_float4(dux, duy, duz, 0.f);
        out.dsA[i] = make_float4(ds[0], ds[1], ds[2], ds[3]);
        out.dsB[i] = make_float2(ds[4], ds[5]);
    } else if (MODE == kStage1) {
        const float h = 0.5f * dt;
        const float4 mp = make_float4(fmaf(h, vi.x, pi.x), fmaf(h, vi.y, pi.y), fmaf(h, vi.z, pi.z),
                                      pi.w);
        MID.pos[i] = p.abs32 ? round_absolute(p, mp) : mp;
        MID.vel[i] = make_float4(fmaf(h, dux, vi.x), fmaf(h, duy, vi.y), fmaf(h, duz, vi.z),
                                 fmaf(h, drho, vi.w));
        MID.sA[i] = make_float4(fmaf(h, ds[0], si[0]), fmaf(h, ds[1], si[1]), fmaf(h, ds[2], si[2]),
                                fmaf(h, ds[3], si[3]));
        MID.sB[i] = make_float2(fmaf(h, ds[4], si[4]), fmaf(h, ds[5], si[5]));
    } else {
        // y_{n+1} = y_n + dt f(y_mid); S holds y_mid, Y holds y_n of particle i
        const float4 p0 = Y.pos[i];
        const float4 v0 = Y.vel[i];
        const float4 a0 = Y.sA[i];
        const float2 b0 = Y.sB[i];
        const float sn[6] = {a0.x, a0.y, a0.z, a0.w, b0.x, b0.y};
        float s1[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) s1[k] = fmaf(dt, ds[k], sn[k]);
        return_map(s1, sn, p, dt);
        const float4 np = make_float4(fmaf(dt, vi.x, p0.x), fmaf(dt, vi.y, p0.y),
                                      fmaf(dt, vi.z, p0.z), p0.w);
        const float4 nv = make_float4(fmaf(dt, dux, v0.x), fmaf(dt, duy, v0.y),
                                      fmaf(dt, duz, v0.z), fmaf(dt, drho, v0.w));
        const float chk = np.x + np.y + np.z + nv.x + nv.y + nv.z + nv.w + s1[0] + s1[1] + s1[2]
                          + s1[3] + s1[4] + s1[5];
        if (!isfinite(chk)) atomicOr(err, ERR_NONFINITE);
        if (xref != nullptr) {
            // largest squared displacement since the last cell search (skin); a
            // max over the lanes that are here, then one atomic per group
            const float4 r0 = xref[i];
            const float ddx = np.x - r0.x, ddy = np.y - r0.y, ddz = np.z - r0.z;
            const int d2 = __float_as_int(ddx * ddx + ddy * ddy + ddz * ddz);
            const unsigned am = __activemask();
            const int mx = __reduce_max_sync(am, d2);
            if ((threadIdx.x & 31) == __ffs(am) - 1) atomicMax(gate + GATE_DISP, mx);
        }
        Y.pos[i] = p.abs32 ? round_absolute(p, np) : np;
        Y.vel[i] = nv;
        Y.sA[i] = make_float4(s1[0], s1[1], s1[2], s1[3]);
        Y.sB[i] = make_float2(s1[4], s1[5]);
    }
}

// LANES (1, 2 or 4) lanes share particle i: each walks every LANES-th entry of its list and
// the sums are combined by shuffles (more warps in flight for the gathers of a
// grid that would otherwise fill each SM only partly).  FILTER (stage 1 with a
// skin): the list walked is the skin list, and the pairs closer than 2h at y_n
// are written, in list order, as the exact list for the rest of the step.
// The pair sums and stage epilogue of fluid particle i (lane q of its LANES),
// for i < limit.
template <int MODE, bool FILTER, int LANES, int KAV>
__device__ __forceinline__ void pair_one(const DevParams &p, int i, int q, int limit,
                                         StageArrays S, StageArrays Y,
                                         StageArrays MID, const ListIO &io,
                                         const uint32_t *__restrict__ pid, float dt, RateOut out,
                                         int *__restrict__ err, const float4 *__restrict__ xref,
                                         int *__restrict__ gate)
{
    const bool valid = i < limit;
    // Extended-Active particles (active domains) are read-only neighbours
    const bool adv = valid && (pid == nullptr || !(pid[i] & kExtendedBit));
    if (valid && !adv && q == 0) {
        if (FILTER) io.out_n[i] = 0u;
        if (MODE == kStage1) {
            MID.pos[i] = S.pos[i];
            MID.vel[i] = S.vel[i];
            MID.sA[i] = S.sA[i];
            MID.sB[i] = S.sB[i];
        } else if (MODE == kEval) {
            out.drho[i] = 0.0f;
            out.du[i] = make_float4(0.f, 0.f, 0.f, 0.f);
            out.dsA[i] = make_float4(0.f, 0.f, 0.f, 0.f);
            out.dsB[i] = make_float2(0.f, 0.f);
        }
    }
    if (LANES == 1 && !adv) return;
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    const float4 pi = adv ? S.pos[i] : z4;
    const float4 vi = adv ? S.vel[i] : z4;
    const float4 ai = adv ? S.sA[i] : z4;
    const float2 bi = adv ? S.sB[i] : make_float2(0.f, 0.f);
    PairAcc A;
    A.mx = A.my = A.mz = A.Gx = A.Gy = A.Gz = A.avx = A.avy = A.avz = 0.f;
#pragma unroll
    for (int k = 0; k < 9; ++k) A.L[k] = 0.f;
    // a skin list (FILTER) holds the pairs within 2h at its search at the front
    // (count: the low half of its count word) and the rest of the skin radius at the
    // back of its skin_cap entries (the high half); an exact list is one front part
    const uint32_t nw = adv ? io.in_n[i] : 0u;
    const int nn = FILTER ? (int)(nw & 0xFFFFu) : (int)nw;
    const int ns = FILTER ? (int)(nw >> 16) : 0;
    const uint32_t *row = io.in + (adv ? i : 0);
    int cnt = 0;
    // the lane's next list entry is fetched one iteration ahead
    uint32_t e_nx = q < nn ? ld_list(row + (size_t)q * p.ell) : 0u;
    if (!FILTER || LANES == 1) {
        // on an exact list, and on a skin list's front, the neighbour's whole state
        // is gathered at once (one load round per iteration)
        const size_t step = (size_t)LANES * p.ell;
        const uint32_t *nxt = row + (size_t)(q + LANES) * p.ell;   // entry k + LANES
        uint32_t *out = FILTER ? io.out + i : nullptr;                // exact entry cnt
        for (int k = q; k < nn; k += LANES, nxt += step) {
            const uint32_t e = e_nx;
            if (k + LANES < nn) e_nx = ld_list(nxt);
            const uint32_t j = e & kIndexMask;
            const float3 sh = entry_shift(e, p.cell);
            const float4 pj = __ldg(&S.pos[j]);
            float4 vj, aj;
            float2 bj;
            vj = __ldg(&S.vel[j]);
            aj = __ldg(&S.sA[j]);
            bj = __ldg(&S.sB[j]);
            const float rx = pi.x - pj.x - sh.x, ry = pi.y - pj.y - sh.y, rz = pi.z - pj.z - sh.z;
            const float r2 = rx * rx + ry * ry + rz * rz;
            if (!(r2 < p.four_h2)) continue;
            if (FILTER) {
                if (cnt < p.maxnb) {
                    *out = e;
                    out += p.ell;
                }
                ++cnt;
            }
            pair_terms<KAV>(p, vi, ai, bi, vj, aj, bj, rx, ry, rz, r2, A);
        }
        if (FILTER && ns > 0) {
            // the skin list's back: few of its candidates have come within 2h, so
            // each is tested on its position alone, and the kept ones wait in a
            // short queue so that the lanes of a warp sum them together afterwards
            // (one pair evaluation per queued entry rather than one per candidate
            // some lane keeps); a full queue sums at once
            uint32_t q0 = 0u, q1 = 0u, q2 = 0u, q3 = 0u;
            int nq = 0;
            // a kept candidate: written to the exact list, queued (or summed at once
            // when the queue is full)
            auto keep = [&](uint32_t e, float rx, float ry, float rz, float r2) {
                if (cnt < p.maxnb) {
                    *out = e;
                    out += p.ell;
                }
                ++cnt;
                if (nq < 4) {
                    q0 = nq == 0 ? e : q0;
                    q1 = nq == 1 ? e : q1;
                    q2 = nq == 2 ? e : q2;
                    q3 = nq == 3 ? e : q3;
                    ++nq;
                } else {
                    const uint32_t j = e & kIndexMask;
                    pair_terms<KAV>(p, vi, ai, bi, __ldg(&S.vel[j]), __ldg(&S.sA[j]),
                                    __ldg(&S.sB[j]), rx, ry, rz, r2, A);
                }
            };
            // two candidates per iteration, their positions fetched together (the
            // next two list words one iteration ahead)
            const uint32_t *sp = row + (size_t)(p.skin_cap - 1) * p.ell;
            uint32_t na = ld_list(sp), nb = ns > 1 ? ld_list(sp - p.ell) : 0u;
            for (int m = 0; m < ns; m += 2, sp -= 2 * p.ell) {
                const uint32_t ea = na, eb = nb;
                const bool two = m + 1 < ns;
                if (m + 2 < ns) na = ld_list(sp - 2 * p.ell);
                if (m + 3 < ns) nb = ld_list(sp - 3 * p.ell);
                const float3 sha = entry_shift(ea, p.cell), shb = entry_shift(eb, p.cell);
                const float4 pa = __ldg(&S.pos[ea & kIndexMask]);
                const float4 pb = two ? __ldg(&S.pos[eb & kIndexMask]) : pa;
                const float ax = pi.x - pa.x - sha.x, ay = pi.y - pa.y - sha.y, az = pi.z - pa.z - sha.z;
                const float a2 = ax * ax + ay * ay + az * az;
                if (a2 < p.four_h2) keep(ea, ax, ay, az, a2);
                const float bx = pi.x - pb.x - shb.x, by = pi.y - pb.y - shb.y, bz = pi.z - pb.z - shb.z;
                const float b2 = bx * bx + by * by + bz * bz;
                if (two && b2 < p.four_h2) keep(eb, bx, by, bz, b2);
            }
            for (int m = 0; m < nq; ++m) {
                const uint32_t e = m == 0 ? q0 : (m == 1 ? q1 : (m == 2 ? q2 : q3));
                const uint32_t j = e & kIndexMask;
                const float3 sh = entry_shift(e, p.cell);
                const float4 pj = __ldg(&S.pos[j]);
                const float4 vj = __ldg(&S.vel[j]);
                const float4 aj = __ldg(&S.sA[j]);
                const float2 bj = __ldg(&S.sB[j]);
                const float rx = pi.x - pj.x - sh.x, ry = pi.y - pj.y - sh.y, rz = pi.z - pj.z - sh.z;
                pair_terms<KAV>(p, vi, ai, bi, vj, aj, bj, rx, ry, rz, rx * rx + ry * ry + rz * rz, A);
            }
        }
    } else {
        // filtering with a lane group: the skin list's front, then its back, in
        // warp-uniform rounds, in each of which the group's lanes test consecutive
        // candidates and place the kept ones by ballot
        const int lane = threadIdx.x & 31;
        for (int part = 0; part < 2; ++part) {
            const int len = part == 0 ? nn : ns;
            // the part's k-th entry sits at first + k * stride
            const ptrdiff_t stride = part == 0 ? (ptrdiff_t)p.ell : -(ptrdiff_t)p.ell;
            const uint32_t *first = part == 0 ? row : row + (size_t)(p.skin_cap - 1) * p.ell;
            if (part == 1) e_nx = q < len ? ld_list(first + q * stride) : 0u;
            const int rounds = __reduce_max_sync(0xffffffffu, (len + LANES - 1) / LANES);
            for (int r = 0; r < rounds; ++r) {
                const int k = r * LANES + q;
                const uint32_t e = e_nx;
                if (k + LANES < len) e_nx = ld_list(first + (k + LANES) * stride);
                bool keep = false;
                float rx = 0.f, ry = 0.f, rz = 0.f, r2 = 0.f;
                uint32_t j = 0;
                if (k < len) {
                    j = e & kIndexMask;
                    const float3 sh = entry_shift(e, p.cell);
                    const float4 pj = __ldg(&S.pos[j]);
                    rx = pi.x - pj.x - sh.x; ry = pi.y - pj.y - sh.y; rz = pi.z - pj.z - sh.z;
                    r2 = rx * rx + ry * ry + rz * rz;
                    keep = r2 < p.four_h2;
                }
                const unsigned b = __ballot_sync(0xffffffffu, keep);
                const unsigned g = (b >> (lane & ~(LANES - 1))) & ((1u << LANES) - 1u);
                const int at = cnt + __popc(g & ((1u << q) - 1u));
                if (keep && at < p.maxnb) io.out[(size_t)at * p.ell + i] = e;
                cnt += __popc(g);
                if (!keep) continue;
                const float4 vj = __ldg(&S.vel[j]);
                const float4 aj = __ldg(&S.sA[j]);
                const float2 bj = __ldg(&S.sB[j]);
                pair_terms<KAV>(p, vi, ai, bi, vj, aj, bj, rx, ry, rz, r2, A);
            }
        }
    }
    if (LANES > 1) {
#pragma unroll
        for (int o = 1; o < LANES; o <<= 1) {
            A.mx += __shfl_xor_sync(0xffffffffu, A.mx, o);
            A.Gx += __shfl_xor_sync(0xffffffffu, A.Gx, o);
            A.Gy += __shfl_xor_sync(0xffffffffu, A.Gy, o);
            A.Gz += __shfl_xor_sync(0xffffffffu, A.Gz, o);
            A.my += __shfl_xor_sync(0xffffffffu, A.my, o);
            A.mz += __shfl_xor_sync(0xffffffffu, A.mz, o);
            A.avx += __shfl_xor_sync(0xffffffffu, A.avx, o);
            A.avy += __shfl_xor_sync(0xffffffffu, A.avy, o);
            A.avz += __shfl_xor_sync(0xffffffffu, A.avz, o);
#pragma unroll
            for (int k = 0; k < 9; ++k) A.L[k] += __shfl_xor_sync(0xffffffffu, A.L[k], o);
        }
        if (!adv || q != 0) return;
    }
    if (FILTER) {
        if (cnt > p.maxnb) atomicOr(err, ERR_CAPACITY);
        io.out_n[i] = (uint32_t)min(cnt, p.maxnb);
    }
    stage_epilogue<MODE>(p, i, pi, vi, ai, bi, A, S, Y, MID, dt, out, err, xref, gate);
}

template <int MODE, bool FILTER, int LANES, int KAV>
__global__ void __launch_bounds__(kPairBlock, LANES == 2 ? 8 : 7)
k_pair(DevParams p, StageArrays S, StageArrays Y, StageArrays MID, ListIO io,
       const uint32_t *__restrict__ pid, float dt, RateOut out, int *__restrict__ err,
       const float4 *__restrict__ xref, int *__restrict__ gate)
{
    if (*p.abort) return;
    if (MODE == kStage2 && p.step_ctr != nullptr && blockIdx.x == 0 && threadIdx.x == 0)
        atomicAdd(p.step_ctr, 1ull);   // the step completes (no abort seen)
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    pair_one<MODE, FILTER, LANES, KAV>(p, t / LANES, t % LANES, __ldg(p.sizes), S, Y, MID,
                                       io, pid, dt, out, err, xref, gate);
}

// Batched form (crm_batch): persistent blocks take virtual blocks of the
// members' own pair launches off the work queue (an atomic ticket) and run them
// as those launches would: stage 1 filtering the skin lists, stage 2 on the
// exact lists, each with the member's lanes.
template <int MODE, int LANES, int KAV>
__global__ void __launch_bounds__(kPairBlock, LANES == 2 ? 8 : 7)
k_batch_pair(const MemberDev *__restrict__ mem, const int *__restrict__ mlist,
             const int *__restrict__ off, int n, unsigned *queue)
{
    __shared__ int s_item;
    __shared__ MemberDev M;
    const int total = __ldg(off + n);
    int cur = -1;   // the member whose descriptor is loaded
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_item = (int)atomicAdd(queue, 1u) * kBatchChunk;
        __syncthreads();
        const int it0 = s_item;
        if (it0 >= total) break;
        const int it1 = min(it0 + kBatchChunk, total);
        for (int it = it0; it < it1; ++it) {
            int lo = 0, hi = n - 1;   // off[lo] <= it < off[lo + 1]
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (__ldg(off + mid) <= it) lo = mid; else hi = mid - 1;
            }
            if (lo != cur) {   // block-uniform
                __syncthreads();
                load_member(mem + __ldg(mlist + lo), &M);
                __syncthreads();
                cur = lo;
            }
            if (*M.p.abort) continue;
            const int t = (it - __ldg(off + lo)) * kPairBlock + threadIdx.x;
            const RateOut none{};
            if (MODE == kStage1) {
                const ListIO io{M.sk_nbr, M.sk_nnb, M.nbr, M.nnb, M.err};
                pair_one<kStage1, true, LANES, KAV>(M.p, t / LANES, t % LANES, __ldg(M.p.sizes),
                                                    M.S, M.S, M.MID, io, nullptr,
                                                    (float)M.dt, none, M.err, nullptr, nullptr);
            } else {
                const ListIO io{M.nbr, M.nnb, nullptr, nullptr, M.err};
                pair_one<kStage2, false, LANES, KAV>(M.p, t / LANES, t % LANES, __ldg(M.p.sizes),
                                                     M.MID, M.S, M.MID, io, nullptr,
                                                     (float)M.dt, none, M.err, M.xref, M.gate);
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0 && atomicAdd(queue + 1, 1u) == gridDim.x - 1) {
        queue[0] = 0u;   // every block has stopped claiming: reset for the next launch
        queue[1] = 0u;
    }
}

// Sorted fluid slots -> insertion order (absolute FP64 positions).
__global__ void k_export(DevParams p, StageArrays S, const uint32_t *__restrict__ pid,
                         double *__restrict__ xyz, float *__restrict__ vel,
                         float *__restrict__ sig, float *__restrict__ rho)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= __ldg(p.sizes)) return;
    const uint32_t id = pid[s];
    const float4 ps = S.pos[s];
    int ix, iy, iz;
    decode_cell(__float_as_uint(ps.w), p, ix, iy, iz);
    xyz[3 * (size_t)id + 0] = p.dmin_x + ix * p.cell_d + (double)ps.x;
    xyz[3 * (size_t)id + 1] = p.dmin_y + iy * p.cell_d + (double)ps.y;
    xyz[3 * (size_t)id + 2] = p.dmin_z + iz * p.cell_d + (double)ps.z;
    const float4 v = S.vel[s];
    vel[3 * (size_t)id + 0] = v.x; vel[3 * (size_t)id + 1] = v.y; vel[3 * (size_t)id + 2] = v.z;
    rho[id] = v.w;
    const float4 a = S.sA[s];
    const float2 b = S.sB[s];
    float *o = sig + 6 * (size_t)id;
    o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w; o[4] = b.x; o[5] = b.y;
}

// Rates and marker state of an evaluation, sorted slots -> insertion order.
__global__ void k_export_rates(DevParams p, const uint32_t *__restrict__ pid, RateOut r,
                               StageArrays S, const float4 *__restrict__ mforce,
                               int n_fluid_total, float *__restrict__ drho,
                               float *__restrict__ du, float *__restrict__ ds,
                               float *__restrict__ macc, float *__restrict__ mvel,
                               float *__restrict__ msig)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const Sizes z = load_sizes(p);
    if (s >= z.N) return;
    const uint32_t id = pid_index(pid[s]);
    if (s < z.nF) {
        drho[id] = r.drho[s];
        const float4 a = r.du[s];
        du[3 * (size_t)id] = a.x; du[3 * (size_t)id + 1] = a.y; du[3 * (size_t)id + 2] = a.z;
        const float4 b = r.dsA[s];
        const float2 c = r.dsB[s];
        float *o = ds + 6 * (size_t)id;
        o[0] = b.x; o[1] = b.y; o[2] = b.z; o[3] = b.w; o[4] = c.x; o[5] = c.y;
    } else {
        const size_t m = (size_t)id - (size_t)n_fluid_total;
        const float4 f = mforce[s - z.nF];
        const float im = 1.0f / p.m;
        macc[3 * m] = f.x * im; macc[3 * m + 1] = f.y * im; macc[3 * m + 2] = f.z * im;
        const float4 v = S.vel[s];
        mvel[3 * m] = v.x; mvel[3 * m + 1] = v.y; mvel[3 * m + 2] = v.z;
        const float4 a = S.sA[s];
        const float2 b = S.sB[s];
        float *o = msig + 6 * m;
        o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w; o[4] = b.x; o[5] = b.y;
    }
}

// ---------------------------------------------------------------------------
// Host-side launchers used by the API translation unit.
template <int KAV>
void launch_pair_k(int mode, int LN, const DevParams &p, StageArrays S, StageArrays Y,
                   StageArrays MID, const uint32_t *nbr, const uint32_t *nnb,
                   const uint32_t *pid, float dt, RateOut out, int *err, const float4 *xref,
                   int *gate, cudaStream_t st, const uint32_t *sk_nbr, const uint32_t *sk_nnb)
{
    constexpr int B = kPairBlock;
    const unsigned g = grid_for((int64_t)p.capF * LN, B);
    const unsigned g1 = grid_for(p.capF, B);
    if (sk_nbr != nullptr) {   // stage 1 or an evaluation right after a skin search
        const ListIO L{sk_nbr, sk_nnb, const_cast<uint32_t *>(nbr), const_cast<uint32_t *>(nnb), err};
        if (pair_filter_lanes(LN) == 4) {
            if (mode == kStage1)
                k_pair<kStage1, true, 4, KAV><<<g, B, 0, st>>>(p, S, Y, MID, L, pid, dt, out, err,
                                                               nullptr, nullptr);
            else
                k_pair<kEval, true, 4, KAV><<<g, B, 0, st>>>(p, S, Y, MID, L, pid, dt, out, err,
                                                             nullptr, nullptr);
        } else if (mode == kStage1) {
            k_pair<kStage1, true, 1, KAV><<<g1, B, 0, st>>>(p, S, Y, MID, L, pid, dt, out, err,
                                                            nullptr, nullptr);
        } else {
            k_pair<kEval, true, 1, KAV><<<g1, B, 0, st>>>(p, S, Y, MID, L, pid, dt, out, err,
                                                          nullptr, nullptr);
        }
        return;
    }
    const ListIO L{nbr, nnb, nullptr, nullptr, err};
#define CRM_PAIR(LNS)                                                                           \
    do {                                                                                        \
        if (mode == kStage1)                                                                    \
            k_pair<kStage1, false, LNS, KAV><<<g, B, 0, st>>>(p, S, Y, MID, L, pid, dt, out, err, \
                                                              nullptr, nullptr);                \
        else if (mode == kStage2)                                                               \
            k_pair<kStage2, false, LNS, KAV><<<g, B, 0, st>>>(p, S, Y, MID, L, pid, dt, out, err, \
                                                              xref, gate);                      \
        else                                                                                    \
            k_pair<kEval, false, LNS, KAV><<<g, B, 0, st>>>(p, S, Y, MID, L, pid, dt, out, err,   \
                                                            nullptr, nullptr);                  \
    } while (0)
    if (LN == 1) CRM_PAIR(1);
    else if (LN == 4) CRM_PAIR(4);
    else CRM_PAIR(2);
#undef CRM_PAIR
}

void launch_pair(int mode, const DevParams &p, StageArrays S, StageArrays Y, StageArrays MID,
                 const uint32_t *nbr, const uint32_t *nnb, const uint32_t *integrate, float dt,
                 RateOut out, int *err, const float4 *xref, int *gate, cudaStream_t st,
                 const uint32_t *sk_nbr, const uint32_t *sk_nnb)
{
    // the kernels on exact lists take p.pair_lanes (1, 2 or 4), a per-terrain
    // tuning knob; by default four lanes while four threads per particle still
    // fit the GPU's resident threads (a small working set otherwise leaves most
    // warp slots empty), else kPairLanes.  The filtering kernels follow with four
    // lanes, else one (on a large working set the lane group's ballot per
    // candidate costs more than the extra warps gain).
    const int LN = p.pair_lanes != 0 ? p.pair_lanes
                                     : ((int64_t)p.capF * 4 <= (int64_t)p.n_sm * 2048 ? 4 : kPairLanes);
    const int kav = 3 * (p.kernel == CRM_KERNEL_WENDLAND ? 1 : 0)
                    + (p.av_mode == CRM_AV_BILATERAL ? 1 : p.av_mode == CRM_AV_UNILATERAL ? 2 : 0);
#define CRM_KAV(K)                                                                               \
    case K:                                                                                      \
        launch_pair_k<K>(mode, LN, p, S, Y, MID, nbr, nnb, integrate, dt, out, err, xref, gate,  \
                         st, sk_nbr, sk_nnb);                                                    \
        break
    switch (kav) {
        CRM_KAV(0); CRM_KAV(1); CRM_KAV(2); CRM_KAV(3); CRM_KAV(4); CRM_KAV(5);
    }
#undef CRM_KAV
}

int pair_kav(const DevParams &p)
{
    return 3 * (p.kernel == CRM_KERNEL_WENDLAND ? 1 : 0)
           + (p.av_mode == CRM_AV_BILATERAL ? 1 : p.av_mode == CRM_AV_UNILATERAL ? 2 : 0);
}

int pair_lanes_of(const DevParams &p)
{
    return p.pair_lanes != 0 ? p.pair_lanes
                             : ((int64_t)p.capF * 4 <= (int64_t)p.n_sm * 2048 ? 4 : kPairLanes);
}

template <int MODE, int LANES, int KAV>
void batch_pair_go(const MemberDev *mem, const int *mlist, const int *off, int n, int total,
                   unsigned *queue, cudaStream_t st)
{
    int dev = 0, nsm = 148, per_sm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_pair<MODE, LANES, KAV>,
                                                      kPairBlock, 0) != cudaSuccess
        || per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    const unsigned g = (unsigned)std::min<int64_t>((int64_t)nsm * per_sm,
                                                   (total + kBatchChunk - 1) / kBatchChunk);
    k_batch_pair<MODE, LANES, KAV><<<g, kPairBlock, 0, st>>>(mem, mlist, off, n, queue);
}

template <int KAV>
void batch_pair_k(int mode, int lanes, const MemberDev *mem, const int *mlist, const int *off,
                  int n, int total, unsigned *queue, cudaStream_t st)
{
    if (mode == kStage1) {
        if (lanes == 4) batch_pair_go<kStage1, 4, KAV>(mem, mlist, off, n, total, queue, st);
        else batch_pair_go<kStage1, 1, KAV>(mem, mlist, off, n, total, queue, st);
    } else if (lanes == 1) batch_pair_go<kStage2, 1, KAV>(mem, mlist, off, n, total, queue, st);
    else if (lanes == 4) batch_pair_go<kStage2, 4, KAV>(mem, mlist, off, n, total, queue, st);
    else batch_pair_go<kStage2, 2, KAV>(mem, mlist, off, n, total, queue, st);
}

void launch_batch_pair(int mode, int lanes, int kav, const MemberDev *mem, const int *mlist,
                       const int *off, int n, int total, unsigned *queue, cudaStream_t st)
{
    if (total < 1) return;
    switch (kav) {
    case 0: batch_pair_k<0>(mode, lanes, mem, mlist, off, n, total, queue, st); break;
    case 1: batch_pair_k<1>(mode, lanes, mem, mlist, off, n, total, queue, st); break;
    case 2: batch_pair_k<2>(mode, lanes, mem, mlist, off, n, total, queue, st); break;
    case 3: batch_pair_k<3>(mode, lanes, mem, mlist, off, n, total, queue, st); break;
    case 4: batch_pair_k<4>(mode, lanes, mem, mlist, off, n, total, queue, st); break;
    default: batch_pair_k<5>(mode, lanes, mem, mlist, off, n, total, queue, st); break;
    }
}

void launch_export(const DevParams &p, StageArrays S, const uint32_t *pid, double *xyz, float *vel,
                   float *sig, float *rho, cudaStream_t st)
{
    k_export<<<grid_for(p.capF), kBlock, 0, st>>>(p, S, pid, xyz, vel, sig, rho);
}

void launch_export_rates(const DevParams &p, const uint32_t *pid, RateOut r, StageArrays S,
                         const float4 *mforce, int n_fluid_total, float *drho, float *du,
                         float *ds, float *macc, float *mvel, float *msig, cudaStream_t st)
{
    k_export_rates<<<grid_for(p.capN), kBlock, 0, st>>>(p, pid, r, S, mforce, n_fluid_total, drho, du,
                                                     ds, macc, mvel, msig);
}

}  // namespace crm
