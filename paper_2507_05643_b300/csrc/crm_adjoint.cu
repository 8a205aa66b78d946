// crm_adjoint.cu -- reverse sweep (vector-Jacobian product) of the rate
// evaluation and of the midpoint step (Sec. 2.1-2.4), hand-derived.
//
// Forward, for a target i (a fluid particle, or a marker for its acceleration)
// and a list neighbour j: r = x_i - x_j, g = F(|r|) r with F = W'(r) / r,
// V_j = m / rho_j, u = u_j - u_i,
//   cont += V_j u.g,  M += V_j (sigma_i + sigma_j) g,  L += V_j u (x) g,
//   A += f g,  f = 2 c vr / ((rho_i + rho_j)(r^2 + xi^2)),  vr = -u.r  (when the
//   viscosity acts),  c = gamma h sqrt(K / rho0) m.
// Fluid rates: rho' = -rho_i cont, u' = M / rho_i + g + A, sigma' = Jaumann(L, sigma_i).
// Marker acceleration a = M / rho0 + A (rho_i = rho0), force m a.
// Marker state (BCE, Sec. 2.4) over the fluid f in reach, W = W(|x_a - x_f|):
//   w = sum W, su = sum u_f W, ss = sum sigma_f W, sr = sum rho_f (x_a - x_f) W,
//   u_a = 2 u_b - su / w,  sigma_a = (ss - ((g - a_b).sr) I) / w  (w > 0), else
//   u_a = u_b, sigma_a = 0.
//
// The sweep is in gather form -- every thread owns the adjoints it writes, no
// float atomics on particle data -- in three passes per stage:
//   fluid coefficients  adjoints of (cont, M, L, A) of every fluid target and the
//                       local terms (Jaumann, 1/rho_i, the return map, the
//                       integrator's identity parts), from the pair sums that the
//                       forward's pair kernel wrote to the tape;
//   marker gather       per marker: the adjoints of (M, A) of its acceleration
//                       (the rate evaluation's marker accelerations, or a step's
//                       body wrench), the adjoint of its BCE state (from the fluid
//                       pairs that read it and its own acceleration pairs), the
//                       BCE coefficients (w, su, ss, sr), the terms of its own
//                       position, summed per body (FP64);
//   fluid gather        per fluid particle: its own pairs (its coefficients), the
//                       pairs of the neighbours that read it (their
//                       coefficients), and its share of the markers' BCE sums.
// Neighbour lists are those of the forward (frozen) and every branch (the
// unilateral viscosity switch, the return map's cases, an empty BCE sum) is the
// one the forward took.  Rigid-body rotations are held fixed: the body adjoints
// are those of the centre, the linear velocity and the linear acceleration.
#include "crm_adjoint.cuh"

namespace crm {

constexpr int kAdjBlock = 128;

// dF/dr for F(r) = W'(r) / r: (W'' - F) / r.
__device__ __forceinline__ float kernel_dF_dr(float q, float rinv, const DevParams &p)
{
    if (p.kernel == CRM_KERNEL_WENDLAND) {
        const float t = 1.0f - 0.5f * q;
        return -1.5f * p.kdw * t * t * p.inv_h;   // F = kdw (1 - q/2)^3
    }
    const float F = kernel_dw_over_r(q, rinv, p);
    // cubic: W'' = kdw / h (4.5 q - 3) for q < 1, 1.5 kdw / h (2 - q) for 1 <= q < 2
    const float w2 = q < 1.0f ? p.kdw * p.inv_h * (4.5f * q - 3.0f)
                              : 1.5f * p.kdw * p.inv_h * (2.0f - q);
    return (w2 - F) * rinv;
}

// Adjoints of one target's pair sums.
struct Coef {
    float lc, lM[3], lL[9], lA[3];   // cont, M, L (row-major), A
};

// A slot's coefficients as four float4 (64 contiguous bytes):
// (cont, M), (L0..L3), (L4..L7), (L8, A).
__device__ __forceinline__ Coef load_coef(const float4 *c4, int s)
{
    const float4 a = c4[4 * (size_t)s], b = c4[4 * (size_t)s + 1], c = c4[4 * (size_t)s + 2],
                 d = c4[4 * (size_t)s + 3];
    Coef C;
    C.lc = a.x; C.lM[0] = a.y; C.lM[1] = a.z; C.lM[2] = a.w;
    C.lL[0] = b.x; C.lL[1] = b.y; C.lL[2] = b.z; C.lL[3] = b.w;
    C.lL[4] = c.x; C.lL[5] = c.y; C.lL[6] = c.z; C.lL[7] = c.w;
    C.lL[8] = d.x; C.lA[0] = d.y; C.lA[1] = d.z; C.lA[2] = d.w;
    return C;
}

__device__ __forceinline__ void store_coef(float4 *c4, int s, const Coef &C)
{
    c4[4 * (size_t)s] = make_float4(C.lc, C.lM[0], C.lM[1], C.lM[2]);
    c4[4 * (size_t)s + 1] = make_float4(C.lL[0], C.lL[1], C.lL[2], C.lL[3]);
    c4[4 * (size_t)s + 2] = make_float4(C.lL[4], C.lL[5], C.lL[6], C.lL[7]);
    c4[4 * (size_t)s + 3] = make_float4(C.lL[8], C.lA[0], C.lA[1], C.lA[2]);
}

// A marker's BCE coefficients, padded to four float4.
__device__ __forceinline__ void load_bce(const float4 *b4, int m, float cb[kNumBceCoef])
{
    const float4 a = b4[4 * (size_t)m], b = b4[4 * (size_t)m + 1], c = b4[4 * (size_t)m + 2],
                 d = b4[4 * (size_t)m + 3];
    cb[0] = a.x; cb[1] = a.y; cb[2] = a.z; cb[3] = a.w;
    cb[4] = b.x; cb[5] = b.y; cb[6] = b.z; cb[7] = b.w;
    cb[8] = c.x; cb[9] = c.y; cb[10] = c.z; cb[11] = c.w;
    cb[12] = d.x;
}

__device__ __forceinline__ void store_bce(float4 *b4, int m, const float cb[kNumBceCoef])
{
    b4[4 * (size_t)m] = make_float4(cb[0], cb[1], cb[2], cb[3]);
    b4[4 * (size_t)m + 1] = make_float4(cb[4], cb[5], cb[6], cb[7]);
    b4[4 * (size_t)m + 2] = make_float4(cb[8], cb[9], cb[10], cb[11]);
    b4[4 * (size_t)m + 3] = make_float4(cb[12], 0.f, 0.f, 0.f);
}

// Sum over the LANES lanes that share a particle (every lane of the warp calls it).
template <int LANES>
__device__ __forceinline__ float lane_sum(float v)
{
#pragma unroll
    for (int o = 1; o < LANES; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Adjoint of one particle's inputs: position, velocity, stress, density.
struct Adj {
    float x[3], u[3], s[6], rho;
};

__device__ __forceinline__ void adj_zero(Adj &a)
{
#pragma unroll
    for (int k = 0; k < 3; ++k) a.x[k] = a.u[k] = 0.f;
#pragma unroll
    for (int k = 0; k < 6; ++k) a.s[k] = 0.f;
    a.rho = 0.f;
}

__device__ __forceinline__ void adj_load(const float *a, int64_t st, int64_t s, Adj &o)
{
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        o.x[k] = a[(kAdjX + k) * st + s];
        o.u[k] = a[(kAdjU + k) * st + s];
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) o.s[k] = a[(kAdjS + k) * st + s];
    o.rho = a[kAdjR * st + s];
}

__device__ __forceinline__ void adj_store(float *a, int64_t st, int64_t s, const Adj &o)
{
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        a[(kAdjX + k) * st + s] = o.x[k];
        a[(kAdjU + k) * st + s] = o.u[k];
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) a[(kAdjS + k) * st + s] = o.s[k];
    a[kAdjR * st + s] = o.rho;
}

// Parameter adjoints of one thread (FP64).
struct ParAcc {
    double v[kNumGradAcc];
};

__device__ __forceinline__ void par_zero(ParAcc &a)
{
#pragma unroll
    for (int k = 0; k < kNumGradAcc; ++k) a.v[k] = 0.0;
}

// Block sum of the parameter adjoints, one FP64 atomic per block and entry.
__device__ __forceinline__ void par_flush(const ParAcc &a, double *g)
{
    __shared__ double red[kAdjBlock / 32][kNumGradAcc];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < kNumGradAcc; ++k) {
        double v = a.v[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) red[warp][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < kNumGradAcc) {
        double s = 0.0;
        for (int w = 0; w < kAdjBlock / 32; ++w) s += red[w][threadIdx.x];
        if (s != 0.0) atomicAdd(g + threadIdx.x, s);
    }
}

// Particle state as the pair kernels read it.
struct PState {
    float4 v;    // u, rho
    float4 a;    // sigma xx yy zz xy
    float2 b;    // sigma xz yz
};

__device__ __forceinline__ PState load_state(const StageArrays &S, int s)
{
    return PState{S.vel[s], S.sA[s], S.sB[s]};
}

// Both directed pairs of the unordered pair {i, j}, seen from i (r = x_i - x_j,
// 0 < |r| < 2h): OWN, the pair with target i (coefficients Ci, i's own sums);
// OTHER, the pair with target j that reads i as its neighbour (coefficients Cj;
// in it r' = -r, g' = -g, u' = -u, V' = m / rho_i, and the viscosity factor is
// the same).  Adds both pairs' adjoints of i's inputs to `a` and the OWN pair's
// parameter terms to `par`.  Densities are the states' (a marker's is rho0).
// The two share the kernel, its derivative, the stress sum and the viscosity
// factor, which is why they are evaluated together.
template <bool OWN, bool OTHER>
__device__ __forceinline__ void pair_vjp_both(const DevParams &p, const Coef &Ci, const Coef &Cj,
                                              float rx, float ry, float rz, float r2,
                                              const PState &I, const PState &J, Adj &a,
                                              ParAcc &par)
{
    const float rinv = rsqrtf(r2);
    const float q = r2 * rinv * p.inv_h;
    const float F = kernel_dw_over_r(q, rinv, p);
    const float dFr = kernel_dF_dr(q, rinv, p) * rinv;
    const float g[3] = {F * rx, F * ry, F * rz};
    const float r[3] = {rx, ry, rz};
    const float rho_i = I.v.w, rho_j = J.v.w;
    const float u[3] = {J.v.x - I.v.x, J.v.y - I.v.y, J.v.z - I.v.z};
    const float Sxx = I.a.x + J.a.x, Syy = I.a.y + J.a.y, Szz = I.a.z + J.a.z;
    const float Sxy = I.a.w + J.a.w, Sxz = I.b.x + J.b.x, Syz = I.b.y + J.b.y;
    const float Sg[3] = {Sxx * g[0] + Sxy * g[1] + Sxz * g[2], Sxy * g[0] + Syy * g[1] + Syz * g[2],
                         Sxz * g[0] + Syz * g[1] + Szz * g[2]};
    const float ug = u[0] * g[0] + u[1] * g[1] + u[2] * g[2];
    // viscosity: vr = -u.r for both directions, rho_i + rho_j, r^2 + xi^2
    bool av = false;
    float vr = 0.f, inv = 0.f, fac = 0.f;
    const float rs = rho_i + rho_j, d2 = r2 + p.xi2;
    if (p.av_mode != CRM_AV_NONE) {
        vr = -(u[0] * rx + u[1] * ry + u[2] * rz);
        av = p.av_mode == CRM_AV_BILATERAL || vr < 0.0f;
        if (av) {
            inv = 1.0f / (rs * d2);
            fac = 2.0f * p.av_c * vr * inv;
        }
    }
    if (OWN) {
        const Coef &C = Ci;
        const float V = p.m / rho_j;
        float Lg[3], LTu[3], SlM[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            Lg[k] = C.lL[3 * k] * g[0] + C.lL[3 * k + 1] * g[1] + C.lL[3 * k + 2] * g[2];
            LTu[k] = C.lL[k] * u[0] + C.lL[3 + k] * u[1] + C.lL[6 + k] * u[2];
        }
        SlM[0] = Sxx * C.lM[0] + Sxy * C.lM[1] + Sxz * C.lM[2];
        SlM[1] = Sxy * C.lM[0] + Syy * C.lM[1] + Syz * C.lM[2];
        SlM[2] = Sxz * C.lM[0] + Syz * C.lM[1] + Szz * C.lM[2];
        const float Vb = C.lc * ug + C.lM[0] * Sg[0] + C.lM[1] * Sg[1] + C.lM[2] * Sg[2]
                         + u[0] * Lg[0] + u[1] * Lg[1] + u[2] * Lg[2];
        float gb[3], ub[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            gb[k] = V * (C.lc * u[k] + SlM[k] + LTu[k]);
            ub[k] = V * (C.lc * g[k] + Lg[k]);
        }
        float rb[3] = {0.f, 0.f, 0.f};
        if (av) {
            const float fb = C.lA[0] * g[0] + C.lA[1] * g[1] + C.lA[2] * g[2];
            const float vrb = 2.0f * p.av_c * fb * inv;
            const float r2b = -fb * fac / d2;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                gb[k] += fac * C.lA[k];
                ub[k] -= vrb * r[k];
                rb[k] = 2.0f * r2b * r[k] - vrb * u[k];
            }
            a.rho += -fb * fac / rs;
            par.v[kGradAvc] += (double)(2.0f * vr * fb * inv);
        }
        const float rg = (rx * gb[0] + ry * gb[1] + rz * gb[2]) * dFr;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            a.x[k] += rb[k] + F * gb[k] + rg * r[k];
            a.u[k] -= ub[k];
        }
        a.s[0] += V * C.lM[0] * g[0];
        a.s[1] += V * C.lM[1] * g[1];
        a.s[2] += V * C.lM[2] * g[2];
        a.s[3] += V * (C.lM[0] * g[1] + C.lM[1] * g[0]);
        a.s[4] += V * (C.lM[0] * g[2] + C.lM[2] * g[0]);
        a.s[5] += V * (C.lM[1] * g[2] + C.lM[2] * g[1]);
        par.v[kGradM] += (double)(Vb / rho_j);
    }
    if (OTHER) {
        // target j, neighbour i: in j's frame r' = -r, g' = -g, u' = -u, V' = m / rho_i
        const Coef &C = Cj;
        const float V = p.m / rho_i;
        float Lg[3], LTu[3], SlM[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            Lg[k] = C.lL[3 * k] * g[0] + C.lL[3 * k + 1] * g[1] + C.lL[3 * k + 2] * g[2];
            LTu[k] = C.lL[k] * u[0] + C.lL[3 + k] * u[1] + C.lL[6 + k] * u[2];
        }
        SlM[0] = Sxx * C.lM[0] + Sxy * C.lM[1] + Sxz * C.lM[2];
        SlM[1] = Sxy * C.lM[0] + Syy * C.lM[1] + Syz * C.lM[2];
        SlM[2] = Sxz * C.lM[0] + Syz * C.lM[1] + Szz * C.lM[2];
        // u'.g' = u.g, S g' = -S g, u'.(lL g') = u.(lL g)
        const float Vb = C.lc * ug - (C.lM[0] * Sg[0] + C.lM[1] * Sg[1] + C.lM[2] * Sg[2])
                         + u[0] * Lg[0] + u[1] * Lg[1] + u[2] * Lg[2];
        // gb' = V (lc u' + S lM + lL^T u') + fac lA,  ub' = V (lc g' + lL g') - vrb' r'
        float gb[3], ub[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            gb[k] = V * (-C.lc * u[k] + SlM[k] - LTu[k]);
            ub[k] = -V * (C.lc * g[k] + Lg[k]);
        }
        // rb' (adjoint of r') = F gb' + (r'.gb') dF/|r| r' + 2 r2b' r' - vrb' u', and
        // x_i enters r' with a minus sign
        float rb[3] = {0.f, 0.f, 0.f};
        float rsum = 0.f;
        if (av) {
            const float fb = -(C.lA[0] * g[0] + C.lA[1] * g[1] + C.lA[2] * g[2]);   // lA . g'
            const float vrb = 2.0f * p.av_c * fb * inv;
            const float r2b = -fb * fac / d2;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                gb[k] += fac * C.lA[k];
                ub[k] += vrb * r[k];                   // -vrb' r' = +vrb' r
                rb[k] = -2.0f * r2b * r[k] + vrb * u[k];
            }
            rsum = -fb * fac / rs;
        }
        const float rg = (rx * gb[0] + ry * gb[1] + rz * gb[2]) * dFr;   // (r'.gb') r' = (r.gb') r
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            a.x[k] -= rb[k] + F * gb[k] + rg * r[k];
            a.u[k] += ub[k];
        }
        // sym(lM (x) g') = -sym(lM (x) g)
        a.s[0] -= V * C.lM[0] * g[0];
        a.s[1] -= V * C.lM[1] * g[1];
        a.s[2] -= V * C.lM[2] * g[2];
        a.s[3] -= V * (C.lM[0] * g[1] + C.lM[1] * g[0]);
        a.s[4] -= V * (C.lM[0] * g[2] + C.lM[2] * g[0]);
        a.s[5] -= V * (C.lM[1] * g[2] + C.lM[2] * g[1]);
        a.rho += rsum - V / rho_i * Vb;
    }
}

__device__ __forceinline__ float taubar6(const float s[6])
{
    const float p = -(s[0] + s[1] + s[2]) * (1.0f / 3.0f);
    const float t0 = s[0] + p, t1 = s[1] + p, t2 = s[2] + p;
    return sqrtf(0.5f * (t0 * t0 + t1 * t1 + t2 * t2) + (s[3] * s[3] + s[4] * s[4] + s[5] * s[5]));
}

// Adjoint of taubar (the norm of the deviator, shear entries counted twice):
// adds ltb d taubar / d s to ls (as a 6-vector).
__device__ __forceinline__ void taubar_vjp(const float s[6], float tb, float ltb, float ls[6])
{
    if (!(tb > 0.0f) || ltb == 0.0f) return;
    const float ps = -(s[0] + s[1] + s[2]) * (1.0f / 3.0f);
    const float D[3] = {s[0] + ps, s[1] + ps, s[2] + ps};
    const float itb = 1.0f / tb;
    // tb^2 = 0.5 (D0^2 + D1^2 + D2^2) + s3^2 + s4^2 + s5^2, D = s + ps, ps = -tr/3
    float lD[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) lD[k] = 0.5f * ltb * D[k] * itb;
    const float lps = lD[0] + lD[1] + lD[2];
#pragma unroll
    for (int k = 0; k < 3; ++k) ls[k] += lD[k] - lps * (1.0f / 3.0f);
#pragma unroll
    for (int k = 3; k < 6; ++k) ls[k] += ltb * s[k] * itb;
}

// Backward of the return map of Sec. 2.3: lo = adjoint of the mapped stress, s
// = trial stress, sn = stress at t_n (the mu(I) shear rate); writes the trial
// stress's adjoint to ls, adds the adjoint of sn to lsn and the parameters' to
// par.  With mu(I) off (mu_2 = mu_s) the friction coefficient's adjoint is
// mu_s's with mu_2 moving along.
__device__ __forceinline__ void return_map_vjp(const float s[6], const float sn[6], float dt,
                                               const float lo[6], const DevParams &p, float ls[6],
                                               float lsn[6], ParAcc &par)
{
    const float ps = -(s[0] + s[1] + s[2]) * (1.0f / 3.0f);
    if (p.mu_s > 0.0f && ps < -p.cohesion / p.mu_s) {   // tension cut-off: sigma = 0
#pragma unroll
        for (int k = 0; k < 6; ++k) ls[k] = 0.f;
        return;
    }
    const float tb = taubar6(s);
    // mu(I) as the forward takes it
    float mu = p.mu_s, I = 0.f, gdot = 0.f, tbn = 0.f;
    bool rate = false;
    if (p.mu_2 != p.mu_s) {
        tbn = taubar6(sn);
        gdot = (tb - tbn) / (p.G * dt);
        if (gdot > 0.0f && ps > 0.0f) {
            I = gdot * p.grain_d * sqrtf(p.rho0 / ps);
            mu = p.mu_s + (p.mu_2 - p.mu_s) / (1.0f + p.I0 / I);
            rate = true;
        }
    }
    const float tmax = mu * ps + p.cohesion;
    if (tb <= tmax) {                                   // admissible: identity
#pragma unroll
        for (int k = 0; k < 6; ++k) ls[k] = lo[k];
        return;
    }
    // out = -ps I + f D, D = deviator of s, f = tmax / tb
    const float f = tmax / tb;
    const float D[6] = {s[0] + ps, s[1] + ps, s[2] + ps, s[3], s[4], s[5]};
    float lf = 0.f;
#pragma unroll
    for (int k = 0; k < 6; ++k) lf += lo[k] * D[k];
    float lps = -(lo[0] + lo[1] + lo[2]);
    const float ltmax = lf / tb;
    float ltb = -lf * f / tb;
    par.v[kGradCoh] += (double)ltmax;
    lps += ltmax * mu;
    const float lmu = ltmax * ps;
    if (!rate) {
        par.v[kGradMu] += (double)lmu;
    } else {
        // mu = mu_s + (mu_2 - mu_s) / (1 + I0 / I), I = gdot d sqrt(rho0 / ps),
        // gdot = (tb - taubar(sn)) / (G dt)
        const float den = I + p.I0, dmu = p.mu_2 - p.mu_s;
        par.v[kGradMu] += (double)(lmu * p.I0 / den);
        par.v[kGradMu2] += (double)(lmu * I / den);
        par.v[kGradI0] += (double)(-lmu * dmu * I / (den * den));
        const float lI = lmu * dmu * p.I0 / (den * den);
        par.v[kGradGrain] += (double)(lI * I / p.grain_d);
        par.v[kGradRho0] += (double)(lI * I / (2.0f * p.rho0));
        lps -= lI * I / (2.0f * ps);
        const float lg = lI * p.grain_d * sqrtf(p.rho0 / ps);   // lI dI/dgdot
        ltb += lg / (p.G * dt);
        par.v[kGradG] += (double)(-lg * gdot / p.G);
        taubar_vjp(sn, tbn, -lg / (p.G * dt), lsn);
    }
    float lD[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) lD[k] = f * lo[k];
    // tb^2 = 0.5 (D0^2 + D1^2 + D2^2) + D3^2 + D4^2 + D5^2
    const float itb = 1.0f / tb;
#pragma unroll
    for (int k = 0; k < 3; ++k) lD[k] += 0.5f * ltb * D[k] * itb;
#pragma unroll
    for (int k = 3; k < 6; ++k) lD[k] += ltb * D[k] * itb;
    lps += lD[0] + lD[1] + lD[2];
#pragma unroll
    for (int k = 0; k < 3; ++k) ls[k] = lD[k] - lps * (1.0f / 3.0f);
#pragma unroll
    for (int k = 3; k < 6; ++k) ls[k] = lD[k];
}

// Jaumann rate, forward (the pair kernels' formula) -- for the trial stress.
__device__ __forceinline__ void jaumann(const float L[9], const float s[6], float G, float K,
                                        float out[6])
{
    const float a = 0.5f * (L[1] - L[3]), b = 0.5f * (L[2] - L[6]), c = 0.5f * (L[5] - L[7]);
    const float exx = L[0], eyy = L[4], ezz = L[8];
    const float exy = 0.5f * (L[1] + L[3]), exz = 0.5f * (L[2] + L[6]), eyz = 0.5f * (L[5] + L[7]);
    const float iso = (K - 2.0f * G / 3.0f) * (exx + eyy + ezz);
    const float G2 = 2.0f * G;
    out[0] = 2.0f * (a * s[3] + b * s[4]) + G2 * exx + iso;
    out[1] = 2.0f * (c * s[5] - a * s[3]) + G2 * eyy + iso;
    out[2] = -2.0f * (b * s[4] + c * s[5]) + G2 * ezz + iso;
    out[3] = a * (s[1] - s[0]) + b * s[5] + c * s[4] + G2 * exy;
    out[4] = b * (s[2] - s[0]) + a * s[5] - c * s[3] + G2 * exz;
    out[5] = c * (s[2] - s[1]) - a * s[4] - b * s[3] + G2 * eyz;
}

// Backward of the Jaumann rate: l6 = adjoint of the rate (6-vector), s6 the
// stress, L the velocity gradient.  Writes the adjoint of L to lL, adds the
// stress's to ls and the moduli's to par.
__device__ __forceinline__ void jaumann_vjp(const float L[9], const float s6[6], const float l6[6],
                                            const DevParams &p, float lL[9], float ls[6],
                                            ParAcc &par)
{
    // the 6-vector adjoint as a symmetric matrix (off-diagonals halved)
    const float Lm[9] = {l6[0], 0.5f * l6[3], 0.5f * l6[4], 0.5f * l6[3], l6[1], 0.5f * l6[5],
                         0.5f * l6[4], 0.5f * l6[5], l6[2]};
    const float s[9] = {s6[0], s6[3], s6[4], s6[3], s6[1], s6[5], s6[4], s6[5], s6[2]};
    float eps[9], om[9];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            eps[3 * a + b] = 0.5f * (L[3 * a + b] + L[3 * b + a]);
            om[3 * a + b] = 0.5f * (L[3 * a + b] - L[3 * b + a]);
        }
    const float tr_e = eps[0] + eps[4] + eps[8], tr_l = Lm[0] + Lm[4] + Lm[8];
    float omb[9], sbm[9];
    double gG = 0.0;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            float lsg = 0.f, sl = 0.f, ol = 0.f, lo = 0.f;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                lsg += Lm[3 * a + c] * s[3 * c + b];
                sl += s[3 * a + c] * Lm[3 * c + b];
                ol += om[3 * a + c] * Lm[3 * c + b];
                lo += Lm[3 * a + c] * om[3 * c + b];
            }
            omb[3 * a + b] = lsg - sl;   // adjoint of Omega: Lam s - s Lam
            sbm[3 * a + b] = lo - ol;    // adjoint of sigma: Lam Omega - Omega Lam
            gG += 2.0 * (double)Lm[3 * a + b] * (double)(eps[3 * a + b] - (a == b ? tr_e / 3.0f : 0.0f));
        }
    par.v[kGradG] += gG;
    par.v[kGradK] += (double)tr_l * (double)tr_e;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const float eb = 2.0f * p.G * (Lm[3 * a + b] - (a == b ? tr_l / 3.0f : 0.0f))
                             + (a == b ? p.K * tr_l : 0.0f);
            lL[3 * a + b] = eb + 0.5f * (omb[3 * a + b] - omb[3 * b + a]);
        }
    ls[0] += sbm[0]; ls[1] += sbm[4]; ls[2] += sbm[8];
    ls[3] += sbm[1] + sbm[3]; ls[4] += sbm[2] + sbm[6]; ls[5] += sbm[5] + sbm[7];
}

// ---------------------------------------------------------------------------
// Lanes per particle of the gather passes: each lane walks every LANES-th entry
// of the list and the sums are combined by shuffles (a 30k-particle bin would
// otherwise leave most of the GPU's warp slots empty).
constexpr int kAdjLanes = 4;

// Pass 1: fluid coefficients, from the pair sums the forward pair kernel wrote
// (one thread per particle, no list walk).  MODE kAdjEval: the rates' adjoints come from
// l_rate (insertion order) and the local terms are written to l_out (slot
// order).  MODE kAdjStage2: the state is y_mid (V.S), y_n is Y0 and the
// adjoint of y_{n+1} is read from l_next (insertion order); the local terms at
// y_mid go to l_mid and those at y_n (the integrator's identity parts through
// the return map) to l_y0.  MODE kAdjStage1: the state is y_n and the adjoint
// of y_mid is l_mid (complete); everything is added to l_y0.
template <int MODE>
__global__ void __launch_bounds__(kAdjBlock)
k_adj_fluid_coef(DevParams p, AdjStage V, StageArrays Y0, AdjIO io, double *gpar)
{
    const Sizes z = load_sizes(p);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = i < z.nF;
    ParAcc par;
    par_zero(par);
    const StageArrays &S = V.S;
    // the forward's pair sums of this stage (written by the pair kernel)
    float cont = 0.f, M[3] = {0.f, 0.f, 0.f}, L[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) L[k] = 0.f;
    PState I{};
    if (valid) {
        I = load_state(S, i);
        const size_t cs = (size_t)p.capF;
        cont = V.sums[i];
#pragma unroll
        for (int k = 0; k < 3; ++k) M[k] = V.sums[(1 + k) * cs + i];
#pragma unroll
        for (int k = 0; k < 9; ++k) L[k] = V.sums[(4 + k) * cs + i];
    }
    if (valid) {
        const float si[6] = {I.a.x, I.a.y, I.a.z, I.a.w, I.b.x, I.b.y};
        const uint32_t id = pid_index(V.pid[i]);
        const int64_t ns = io.n_fluid;          // stride of the insertion-order arrays
        float lr[10];                           // adjoints of the rates
        Adj y0;                                 // terms on y_n (the step's passes)
        adj_zero(y0);
        Adj loc;                                // local terms on this stage's state
        adj_zero(loc);
        if (MODE == kAdjEval) {
            lr[0] = io.l_rate[(size_t)id];
#pragma unroll
            for (int k = 0; k < 3; ++k) lr[1 + k] = io.l_rate[ns + 3 * (size_t)id + k];
#pragma unroll
            for (int k = 0; k < 6; ++k) lr[4 + k] = io.l_rate[4 * ns + 6 * (size_t)id + k];
        } else if (MODE == kAdjStage2) {
            // y_{n+1} = y_n + dt f(y_mid), x_{n+1} = x_n + dt u_mid, then the return map
            Adj ln;
            adj_load(io.l_next, ns, id, ln);
            const float dt = io.dt;
            float ds[6];
            jaumann(L, si, p.G, p.K, ds);
            const float4 a0 = Y0.sA[i];
            const float2 b0 = Y0.sB[i];
            const float sn[6] = {a0.x, a0.y, a0.z, a0.w, b0.x, b0.y};
            float trial[6], ltr[6], lsn[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int k = 0; k < 6; ++k) trial[k] = fmaf(dt, ds[k], sn[k]);
            return_map_vjp(trial, sn, dt, ln.s, p, ltr, lsn, par);
            lr[0] = dt * ln.rho;
#pragma unroll
            for (int k = 0; k < 3; ++k) lr[1 + k] = dt * ln.u[k];
#pragma unroll
            for (int k = 0; k < 6; ++k) lr[4 + k] = dt * ltr[k];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                y0.x[k] = ln.x[k];
                y0.u[k] = ln.u[k];
                loc.u[k] = dt * ln.x[k];
            }
#pragma unroll
            for (int k = 0; k < 6; ++k) y0.s[k] = ltr[k] + lsn[k];   // trial = sn + dt ds
            y0.rho = ln.rho;
        } else {
            // y_mid = y_n + dt/2 f(y_n), x_mid = x_n + dt/2 u_n
            Adj lm;
            adj_load(io.l_mid, io.slot_stride, i, lm);
            const float h = 0.5f * io.dt;
            lr[0] = h * lm.rho;
#pragma unroll
            for (int k = 0; k < 3; ++k) lr[1 + k] = h * lm.u[k];
#pragma unroll
            for (int k = 0; k < 6; ++k) lr[4 + k] = h * lm.s[k];
            adj_load(io.l_y0, io.slot_stride, i, y0);
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                y0.x[k] += lm.x[k];
                y0.u[k] += lm.u[k] + h * lm.x[k];
            }
#pragma unroll
            for (int k = 0; k < 6; ++k) y0.s[k] += lm.s[k];
            y0.rho += lm.rho;
        }
        // rates -> coefficients and local terms at this stage's state
        const float rho = I.v.w;
        Coef C;
        C.lc = -rho * lr[0];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            C.lM[k] = lr[1 + k] / rho;
            C.lA[k] = lr[1 + k];
        }
        loc.rho += -cont * lr[0] - (M[0] * lr[1] + M[1] * lr[2] + M[2] * lr[3]) / (rho * rho);
        jaumann_vjp(L, si, lr + 4, p, C.lL, loc.s, par);
        store_coef(io.coef, i, C);
        if (MODE == kAdjEval) {
            adj_store(io.l_out, io.slot_stride, i, loc);
        } else if (MODE == kAdjStage2) {
            adj_store(io.l_mid, io.slot_stride, i, loc);
            adj_store(io.l_y0, io.slot_stride, i, y0);
        } else {
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                y0.x[k] += loc.x[k];
                y0.u[k] += loc.u[k];
            }
#pragma unroll
            for (int k = 0; k < 6; ++k) y0.s[k] += loc.s[k];
            y0.rho += loc.rho;
            adj_store(io.l_y0, io.slot_stride, i, y0);
        }
    }
    par_flush(par, gpar);
}

// Rigid-body kinematics of a marker slot: world arm, body velocity and
// acceleration at the marker (FP32); returns the body index (-1: fixed marker).
__device__ __forceinline__ int marker_body_kin(const DevParams &p, const AdjStage &V, int s,
                                               float ub[3], float ab[3], float arm[3])
{
    const uint32_t id = V.pid[s];
    const int b = pid_body(p, id);
#pragma unroll
    for (int k = 0; k < 3; ++k) ub[k] = ab[k] = arm[k] = 0.f;
    if (b >= 0) {
        const int mi = (int)pid_index(id) - V.n_fluid_total;
        double x[3];
        if (V.frames == nullptr) marker_now(V.bodies[b], V.mloc + 3 * (int64_t)mi, x, ub, ab, arm);
        else marker_at(V.frames[b], V.mloc + 3 * (int64_t)mi, x, ub, ab, arm);
    }
    return b;
}

// Pass 2: marker gather.  ACC: the markers' own acceleration pairs carry
// adjoints (their coefficients are formed here and stored for pass 3).  Writes
// the BCE coefficients of every marker slot and adds the body adjoints (centre,
// velocity, acceleration) to gbody [body][9].
// act (nullable): the marker slots that have fluid in reach, n_act[0] of them;
// the others add nothing and their coefficients are never read (a fluid
// particle lists a marker exactly when the marker lists it), so a launch given
// act serves those markers only.
template <bool ACC, int LANES>
__global__ void __launch_bounds__(kAdjBlock)
k_adj_marker(DevParams p, AdjStage V, AdjIO io, double *gpar, double *gbody,
             const uint32_t *__restrict__ act, const int *__restrict__ n_act)
{
    const Sizes z = load_sizes(p);
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    int s;
    bool valid;
    if (act != nullptr) {
        const int na = __ldg(n_act);
        if ((int)(blockIdx.x * blockDim.x / LANES) >= na) return;   // block-uniform
        valid = t / LANES < na;
        s = valid ? (int)__ldg(act + t / LANES) : z.N;
    } else {
        s = z.nF + t / LANES;
        valid = s < z.N;
    }
    const int q = t % LANES;
    ParAcc par;
    par_zero(par);
    const int nn = valid ? (int)V.nnb[s] : 0;
    float ub[3] = {0.f, 0.f, 0.f}, ab[3] = {0.f, 0.f, 0.f}, arm[3] = {0.f, 0.f, 0.f};
    int body = -1;
    if (valid && nn > 0) body = marker_body_kin(p, V, s, ub, ab, arm);
    const StageArrays &S = V.S;
    const float4 pa = nn > 0 ? S.pos[s] : make_float4(0.f, 0.f, 0.f, 0.f);
    PState A0{};
    if (nn > 0) A0 = load_state(S, s);
    // ACC: the adjoint of the marker's acceleration a = M / rho0 + A -- from
    // l_macc (the rate evaluation) or from its body's wrench (a step: force m a,
    // torque arm x m a, so l_a = m (l_F + l_T x arm) plus the direct term of m) --
    // and its pair-sum coefficients, stored for the fluid gather
    Coef Ca{};
    float la3[3] = {0.f, 0.f, 0.f};
    bool direct_m = false;
    if (ACC && nn > 0) {
        if (io.l_macc != nullptr) {
            const size_t mi = (size_t)pid_index(V.pid[s]) - (size_t)V.n_fluid_total;
#pragma unroll
            for (int k = 0; k < 3; ++k) la3[k] = io.l_macc[3 * mi + k];
        } else if (body >= 0) {
            const double *wr = io.l_wrench + 6 * body;
            const float lF[3] = {(float)wr[0], (float)wr[1], (float)wr[2]};
            const float lT[3] = {(float)wr[3], (float)wr[4], (float)wr[5]};
            // (arm x f) . lT = f . (lT x arm)
            const float lf[3] = {lF[0] + lT[1] * arm[2] - lT[2] * arm[1],
                                 lF[1] + lT[2] * arm[0] - lT[0] * arm[2],
                                 lF[2] + lT[0] * arm[1] - lT[1] * arm[0]};
#pragma unroll
            for (int k = 0; k < 3; ++k) la3[k] = p.m * lf[k];
            direct_m = true;
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            Ca.lM[k] = la3[k] / p.rho0;
            Ca.lA[k] = la3[k];
        }
        if (q == 0) store_coef(io.coef, s, Ca);
    }
    Adj la;
    adj_zero(la);
    float w = 0.f, su[3] = {0.f, 0.f, 0.f}, ss[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    float sr[3] = {0.f, 0.f, 0.f};
    float Ms[3] = {0.f, 0.f, 0.f}, As[3] = {0.f, 0.f, 0.f};   // the acceleration's sums (ACC)
    for (int k = q; k < nn; k += LANES) {
        const uint32_t e = V.nbr[(size_t)k * p.ell + s];
        const uint32_t f = e & kIndexMask;
        const float3 sh = entry_shift(e, p.cell);
        // the fluid particle's position, state and pair coefficients in one load round
        const float4 pf = S.pos[f];
        const PState Fs = load_state(S, f);
        const Coef Cf = load_coef(io.coef, (int)f);
        const float rx = pa.x - pf.x - sh.x, ry = pa.y - pf.y - sh.y, rz = pa.z - pf.z - sh.z;
        const float r2 = rx * rx + ry * ry + rz * rz;
        if (!(r2 < p.four_h2)) continue;
        const float W = kernel_w(sqrtf(r2) * p.inv_h, p);
        w += W;
        su[0] += Fs.v.x * W; su[1] += Fs.v.y * W; su[2] += Fs.v.z * W;
        ss[0] += Fs.a.x * W; ss[1] += Fs.a.y * W; ss[2] += Fs.a.z * W;
        ss[3] += Fs.a.w * W; ss[4] += Fs.b.x * W; ss[5] += Fs.b.y * W;
        const float rw = Fs.v.w * W;
        sr[0] += rw * rx; sr[1] += rw * ry; sr[2] += rw * rz;
        if (r2 == 0.0f) continue;
        if (ACC) {
            // M and A of the forward, for the terms of 1 / rho0 and of m in m a
            const float rinv = rsqrtf(r2);
            const float F = kernel_dw_over_r(r2 * rinv * p.inv_h, rinv, p);
            const float g[3] = {F * rx, F * ry, F * rz};
            const float Vf = p.m / Fs.v.w;
            const float Sxx = A0.a.x + Fs.a.x, Syy = A0.a.y + Fs.a.y, Szz = A0.a.z + Fs.a.z;
            const float Sxy = A0.a.w + Fs.a.w, Sxz = A0.b.x + Fs.b.x, Syz = A0.b.y + Fs.b.y;
            Ms[0] += Vf * (Sxx * g[0] + Sxy * g[1] + Sxz * g[2]);
            Ms[1] += Vf * (Sxy * g[0] + Syy * g[1] + Syz * g[2]);
            Ms[2] += Vf * (Sxz * g[0] + Syz * g[1] + Szz * g[2]);
            if (p.av_mode != CRM_AV_NONE) {
                const float vr = (A0.v.x - Fs.v.x) * rx + (A0.v.y - Fs.v.y) * ry + (A0.v.z - Fs.v.z) * rz;
                if (p.av_mode == CRM_AV_BILATERAL || vr < 0.0f) {
                    const float fac = 2.0f * p.av_c * vr / ((p.rho0 + Fs.v.w) * (r2 + p.xi2));
#pragma unroll
                    for (int c = 0; c < 3; ++c) As[c] += fac * g[c];
                }
            }
        }
        // the marker's own acceleration pair (ACC) and the fluid particle's pair
        // that reads this marker
        pair_vjp_both<ACC, true>(p, Ca, Cf, rx, ry, rz, r2, A0, Fs, la, par);
    }
    if (ACC) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            Ms[k] = lane_sum<LANES>(Ms[k]);
            As[k] = lane_sum<LANES>(As[k]);
        }
        if (q == 0 && (la3[0] != 0.f || la3[1] != 0.f || la3[2] != 0.f)) {
            const double ir = 1.0 / (double)p.rho0;
            double drho0 = 0.0, dm = 0.0;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                drho0 -= (double)la3[k] * (double)Ms[k] * ir * ir;
                dm += (double)la3[k] * ((double)Ms[k] * ir + (double)As[k]);
            }
            par.v[kGradRho0] += drho0;
            if (direct_m) par.v[kGradM] += dm / (double)p.m;
        }
    }
    w = lane_sum<LANES>(w);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        su[k] = lane_sum<LANES>(su[k]);
        sr[k] = lane_sum<LANES>(sr[k]);
        la.x[k] = lane_sum<LANES>(la.x[k]);
        la.u[k] = lane_sum<LANES>(la.u[k]);
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        ss[k] = lane_sum<LANES>(ss[k]);
        la.s[k] = lane_sum<LANES>(la.s[k]);
    }
    la.rho = lane_sum<LANES>(la.rho);
    // BCE extrapolation backward (every lane of the marker, redundantly)
    float cb[kNumBceCoef];
#pragma unroll
    for (int k = 0; k < kNumBceCoef; ++k) cb[k] = 0.f;
    float lub[3] = {0.f, 0.f, 0.f}, lab[3] = {0.f, 0.f, 0.f}, px[3] = {0.f, 0.f, 0.f};
    if (w > 0.f) {
        const float iw = 1.0f / w;
        const float ua[3] = {2.f * ub[0] - su[0] * iw, 2.f * ub[1] - su[1] * iw,
                             2.f * ub[2] - su[2] * iw};
        const float gp = (p.gx - ab[0]) * sr[0] + (p.gy - ab[1]) * sr[1] + (p.gz - ab[2]) * sr[2];
        const float sa[6] = {(ss[0] - gp) * iw, (ss[1] - gp) * iw, (ss[2] - gp) * iw,
                             ss[3] * iw, ss[4] * iw, ss[5] * iw};
        float lw = 0.f;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            cb[kBceSu + k] = -la.u[k] * iw;
            lw += la.u[k] * (2.f * ub[k] - ua[k]) * iw;   // su / w^2 = (2 ub - ua) / w
            lub[k] = 2.f * la.u[k];
        }
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            cb[kBceSs + k] = la.s[k] * iw;
            lw -= la.s[k] * sa[k] * iw;
        }
        const float lgp = -(la.s[0] + la.s[1] + la.s[2]) * iw;
        cb[kBceSr + 0] = lgp * (p.gx - ab[0]);
        cb[kBceSr + 1] = lgp * (p.gy - ab[1]);
        cb[kBceSr + 2] = lgp * (p.gz - ab[2]);
#pragma unroll
        for (int k = 0; k < 3; ++k) lab[k] = -lgp * sr[k];
        cb[kBceW] = lw;
        // the marker position in its BCE sums
        for (int k = q; k < nn; k += LANES) {
            const uint32_t e = V.nbr[(size_t)k * p.ell + s];
            const uint32_t f = e & kIndexMask;
            const float3 sh = entry_shift(e, p.cell);
            const float4 pf = S.pos[f];
            const float rx = pa.x - pf.x - sh.x, ry = pa.y - pf.y - sh.y, rz = pa.z - pf.z - sh.z;
            const float r2 = rx * rx + ry * ry + rz * rz;
            if (!(r2 < p.four_h2) || r2 == 0.0f) continue;
            const PState Fs = load_state(S, f);
            const float rinv = rsqrtf(r2);
            const float qk = r2 * rinv * p.inv_h;
            const float W = kernel_w(sqrtf(r2) * p.inv_h, p);
            const float F = kernel_dw_over_r(qk, rinv, p);
            const float lW = cb[kBceW] + cb[kBceSu] * Fs.v.x + cb[kBceSu + 1] * Fs.v.y
                             + cb[kBceSu + 2] * Fs.v.z + cb[kBceSs] * Fs.a.x
                             + cb[kBceSs + 1] * Fs.a.y + cb[kBceSs + 2] * Fs.a.z
                             + cb[kBceSs + 3] * Fs.a.w + cb[kBceSs + 4] * Fs.b.x
                             + cb[kBceSs + 5] * Fs.b.y
                             + Fs.v.w * (cb[kBceSr] * rx + cb[kBceSr + 1] * ry + cb[kBceSr + 2] * rz);
            const float rw = Fs.v.w * W, fl = lW * F;
            px[0] += rw * cb[kBceSr] + fl * rx;
            px[1] += rw * cb[kBceSr + 1] + fl * ry;
            px[2] += rw * cb[kBceSr + 2] + fl * rz;
        }
    } else {
#pragma unroll
        for (int k = 0; k < 3; ++k) lub[k] = la.u[k];
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) la.x[k] += lane_sum<LANES>(px[k]);
    if (valid && q == 0) {
        store_bce(io.coefB, s - z.nF, cb);
        par.v[kGradRho0] += (double)la.rho;     // the marker density is rho0
    }
    if (q != 0) body = -1;
    // the body's rotation: the marker sits at r = R l from the centre (a world-frame
    // turn d theta moves it by d theta x r) and moves with u_b = v + w x r and
    // a_b = acc + alpha x r + w x (w x r); in a step's wrench the marker force
    // f = m a also acts at the arm r (torque r x f)
    float lth[3] = {0.f, 0.f, 0.f}, lom[3] = {0.f, 0.f, 0.f}, lal[3] = {0.f, 0.f, 0.f};
    if (body >= 0) {
        const double *tw = V.bodies[body].twist + 3;
        const float om[3] = {(float)tw[0], (float)tw[1], (float)tw[2]};
        float lr[3] = {la.x[0], la.x[1], la.x[2]};
        if (ACC && io.l_macc == nullptr) {
            const double *wr = io.l_wrench + 6 * body;
            const float lT[3] = {(float)wr[3], (float)wr[4], (float)wr[5]};
            float fm[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) fm[k] = p.m * (Ms[k] / p.rho0 + As[k]);
            // (r x f) . lT = r . (f x lT)
            lr[0] += fm[1] * lT[2] - fm[2] * lT[1];
            lr[1] += fm[2] * lT[0] - fm[0] * lT[2];
            lr[2] += fm[0] * lT[1] - fm[1] * lT[0];
        }
        // u_b = v + w x r: (w x r) . l = r . (l x w) = w . (r x l)
        lr[0] += lub[1] * om[2] - lub[2] * om[1];
        lr[1] += lub[2] * om[0] - lub[0] * om[2];
        lr[2] += lub[0] * om[1] - lub[1] * om[0];
        lom[0] += arm[1] * lub[2] - arm[2] * lub[1];
        lom[1] += arm[2] * lub[0] - arm[0] * lub[2];
        lom[2] += arm[0] * lub[1] - arm[1] * lub[0];
        // a_b = acc + alpha x r + w x q, q = w x r
        const double *al = V.bodies[body].alpha;
        const float alp[3] = {(float)al[0], (float)al[1], (float)al[2]};
        lal[0] = arm[1] * lab[2] - arm[2] * lab[1];
        lal[1] = arm[2] * lab[0] - arm[0] * lab[2];
        lal[2] = arm[0] * lab[1] - arm[1] * lab[0];
        lr[0] += lab[1] * alp[2] - lab[2] * alp[1];
        lr[1] += lab[2] * alp[0] - lab[0] * alp[2];
        lr[2] += lab[0] * alp[1] - lab[1] * alp[0];
        const float qv[3] = {om[1] * arm[2] - om[2] * arm[1], om[2] * arm[0] - om[0] * arm[2],
                             om[0] * arm[1] - om[1] * arm[0]};
        const float lq[3] = {lab[1] * om[2] - lab[2] * om[1], lab[2] * om[0] - lab[0] * om[2],
                             lab[0] * om[1] - lab[1] * om[0]};   // l_q = l_a x w
        lom[0] += qv[1] * lab[2] - qv[2] * lab[1];
        lom[1] += qv[2] * lab[0] - qv[0] * lab[2];
        lom[2] += qv[0] * lab[1] - qv[1] * lab[0];
        lr[0] += lq[1] * om[2] - lq[2] * om[1];
        lr[1] += lq[2] * om[0] - lq[0] * om[2];
        lr[2] += lq[0] * om[1] - lq[1] * om[0];
        lom[0] += arm[1] * lq[2] - arm[2] * lq[1];
        lom[1] += arm[2] * lq[0] - arm[0] * lq[2];
        lom[2] += arm[0] * lq[1] - arm[1] * lq[0];
        // d r = d theta x r: the turn's adjoint is r x l_r
        lth[0] = arm[1] * lr[2] - arm[2] * lr[1];
        lth[1] = arm[2] * lr[0] - arm[0] * lr[2];
        lth[2] = arm[0] * lr[1] - arm[1] * lr[0];
    }
    par_flush(par, gpar);
    // per-body sums: warp reduction, one FP64 atomic per warp and entry
    const int lane = threadIdx.x & 31;
    for (int b = 0; b < p.n_bodies; ++b) {
        const bool mine = body == b;
        if (!__any_sync(0xffffffffu, mine)) continue;
        double v[kBodyAdj];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            v[kBodyC + k] = mine ? la.x[k] : 0.0;
            v[kBodyV + k] = mine ? lub[k] : 0.0;
            v[kBodyA + k] = mine ? lab[k] : 0.0;
            v[kBodyTheta + k] = mine ? lth[k] : 0.0;
            v[kBodyW + k] = mine ? lom[k] : 0.0;
            v[kBodyAlpha + k] = mine ? lal[k] : 0.0;
        }
#pragma unroll
        for (int k = 0; k < kBodyAdj; ++k) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
            if (lane == 0 && v[k] != 0.0) atomicAdd(gbody + kBodyAdj * b + k, v[k]);
        }
    }
}

// Pass 3: fluid gather.  ACC: the markers in the list carry acceleration
// coefficients.  OUT kAdjAccumulate: the sums are added to l_acc (slot order);
// kAdjFinal: l_acc (slot order) plus the sums is written to l_final at the
// particle's insertion index.
template <bool ACC, int OUT, int LANES>
__global__ void __launch_bounds__(kAdjBlock)
k_adj_fluid(DevParams p, AdjStage V, AdjIO io, float *l_acc, float *l_final, double *gpar)
{
    __syncthreads();
    const Sizes z = load_sizes(p);
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = t / LANES, q = t % LANES;
    const bool valid = i < z.nF;
    ParAcc par;
    par_zero(par);
    Adj a;
    adj_zero(a);
    if (valid) {
        const StageArrays &S = V.S;
        const float4 pi = S.pos[i];
        const PState I = load_state(S, i);
        const Coef Ci = load_coef(io.coef, i);
        const int nn = (int)V.nnb[i];
        for (int k = q; k < nn; k += LANES) {
            const uint32_t e = V.nbr[(size_t)k * p.ell + i];
            const uint32_t j = e & kIndexMask;
            const float3 sh = entry_shift(e, p.cell);
            // the neighbour's position, state and pair coefficients in one load round
            // (the list holds the pairs within 2h at y_n: nearly all pass the test)
            const float4 pj = S.pos[j];
            const PState J = load_state(S, j);
            const bool marker = (int)j >= z.nF;
            Coef Cj;
            if (!marker || ACC) Cj = load_coef(io.coef, (int)j);
            const float rx = pi.x - pj.x - sh.x, ry = pi.y - pj.y - sh.y, rz = pi.z - pj.z - sh.z;
            const float r2 = rx * rx + ry * ry + rz * rz;
            if (!(r2 < p.four_h2)) continue;
            if (r2 != 0.0f) {
                // own pair (i target) and the neighbour's pair that reads i (j
                // target; a marker's only with acceleration adjoints)
                if (!marker || ACC) {
                    pair_vjp_both<true, true>(p, Ci, Cj, rx, ry, rz, r2, I, J, a, par);
                } else {
                    pair_vjp_both<true, false>(p, Ci, Ci, rx, ry, rz, r2, I, J, a, par);
                }
            }
            if (marker) {
                // i in marker j's BCE sums: r_a = x_j - x_i = -r
                float cb[kNumBceCoef];
                load_bce(io.coefB, (int)j - z.nF, cb);
                const float ax = -rx, ay = -ry, az = -rz;
                const float W = kernel_w(sqrtf(r2) * p.inv_h, p);
                const float lsr = cb[kBceSr] * ax + cb[kBceSr + 1] * ay + cb[kBceSr + 2] * az;
                const float lW = cb[kBceW] + cb[kBceSu] * I.v.x + cb[kBceSu + 1] * I.v.y
                                 + cb[kBceSu + 2] * I.v.z + cb[kBceSs] * I.a.x + cb[kBceSs + 1] * I.a.y
                                 + cb[kBceSs + 2] * I.a.z + cb[kBceSs + 3] * I.a.w
                                 + cb[kBceSs + 4] * I.b.x + cb[kBceSs + 5] * I.b.y + I.v.w * lsr;
#pragma unroll
                for (int c = 0; c < 3; ++c) a.u[c] += cb[kBceSu + c] * W;
#pragma unroll
                for (int c = 0; c < 6; ++c) a.s[c] += cb[kBceSs + c] * W;
                a.rho += lsr * W;
                if (r2 != 0.0f) {
                    const float rinv = rsqrtf(r2);
                    const float F = kernel_dw_over_r(r2 * rinv * p.inv_h, rinv, p);
                    const float rw = I.v.w * W, fl = lW * F;
                    a.x[0] -= rw * cb[kBceSr] + fl * ax;
                    a.x[1] -= rw * cb[kBceSr + 1] + fl * ay;
                    a.x[2] -= rw * cb[kBceSr + 2] + fl * az;
                }
            }
        }
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        a.x[k] = lane_sum<LANES>(a.x[k]);
        a.u[k] = lane_sum<LANES>(a.u[k]);
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) a.s[k] = lane_sum<LANES>(a.s[k]);
    a.rho = lane_sum<LANES>(a.rho);
    if (valid && q == 0) {
        Adj b;
        adj_load(l_acc, io.slot_stride, i, b);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            a.x[k] += b.x[k];
            a.u[k] += b.u[k];
        }
#pragma unroll
        for (int k = 0; k < 6; ++k) a.s[k] += b.s[k];
        a.rho += b.rho;
        if (OUT == kAdjAccumulate) adj_store(l_acc, io.slot_stride, i, a);
        else adj_store(l_final, io.n_fluid, pid_index(V.pid[i]), a);
    }
    par_flush(par, gpar);
}

// The turn of a step: dq = exp(phi / 2) with phi = w tau (qadvance), applied in
// the world frame, so an orientation perturbed by the world-frame rotation
// vector d theta stays perturbed by R(dq) d theta after the turn, and a change
// d w of the rate turns it by J(phi) tau d w, J the left Jacobian of SO(3):
// J(phi) = I + (1 - cos t) / t^2 [phi]x + (t - sin t) / t^3 [phi]x^2, t = |phi|.
// turn_adjoint(w, tau, l) returns R(dq)^T l in lt and adds tau J(phi)^T l to lw.
__device__ __forceinline__ void turn_adjoint(const double w[3], double tau, const double l[3],
                                             double lt[3], double lw[3])
{
    const double ph[3] = {w[0] * tau, w[1] * tau, w[2] * tau};
    const double t2 = ph[0] * ph[0] + ph[1] * ph[1] + ph[2] * ph[2];
    // R(dq)^T l: rotate l by the conjugate of dq = (cos(t/2), sin(t/2) phi / t)
    double dq[4];
    const double zero[4] = {1.0, 0.0, 0.0, 0.0};
    qadvance(zero, w, tau, dq);
    const double dqc[4] = {dq[0], -dq[1], -dq[2], -dq[3]};
    qrot(dqc, l, lt);
    // J^T l = l - a (phi x l) + b (phi x (phi x l)); Maclaurin series of a, b for small t
    double a, b;
    if (t2 <= 1e-2) {
        a = 0.5 - t2 * (1.0 / 24.0) * (1.0 - t2 * (1.0 / 30.0));
        b = 1.0 / 6.0 - t2 * (1.0 / 120.0) * (1.0 - t2 * (1.0 / 42.0));
    } else {
        const double t = sqrt(t2);
        a = (1.0 - cos(t)) / t2;
        b = (t - sin(t)) / (t2 * t);
    }
    const double c1[3] = {ph[1] * l[2] - ph[2] * l[1], ph[2] * l[0] - ph[0] * l[2],
                          ph[0] * l[1] - ph[1] * l[0]};
    const double c2[3] = {ph[1] * c1[2] - ph[2] * c1[1], ph[2] * c1[0] - ph[0] * c1[2],
                          ph[0] * c1[1] - ph[1] * c1[0]};
    for (int k = 0; k < 3; ++k) lw[k] += tau * (l[k] - a * c1[k] + b * c2[k]);
}

// I_w v = R diag(I) R^T v, and its inverse, with R the rotation of quaternion q.
__device__ __forceinline__ void inertia_world(const double q[4], const double I[3], const double v[3],
                                              bool inverse, double o[3])
{
    const double w = q[0], x = q[1], y = q[2], z = q[3];
    const double R[3][3] = {{1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)},
                            {2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)},
                            {2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)}};
    double t[3];
    for (int r = 0; r < 3; ++r) {
        const double d = R[0][r] * v[0] + R[1][r] * v[1] + R[2][r] * v[2];
        t[r] = inverse ? d / I[r] : d * I[r];
    }
    for (int r = 0; r < 3; ++r) o[r] = R[r][0] * t[0] + R[r][1] * t[1] + R[r][2] * t[2];
}

__device__ __forceinline__ void cross3(const double a[3], const double b[3], double o[3])
{
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

// Body adjoint of the update at the end of a step (Sec. 2.4, symplectic Euler
// on the free DOFs: v' = v + dt (F/m + g), w' = w + dt wd with
// wd = I_w^-1 (T - w x I_w w), I_w = R diag(I) R^T at t_n; then c' = c + dt v'
// and q' = exp(w' dt / 2) q; acc' and alpha' are the free components of the
// accelerations): from the adjoints of the body after the step (lb_next
// [body][kBodyAdj], plus the objective's terms on the wrench and the centre) to
// the adjoint of the soil wrench (l_wrench) and the partial adjoint of the body
// before the step (lb_cur).  bodies / after: the bodies before / after the step.
// It also clears the body's two stage accumulators (gbody [2][nb][kBodyAdj]) for
// the marker passes that follow.  One thread per body.
__global__ void k_adj_body_pre(int nb, const BodyDev *bodies, const BodyDev *after, double dt,
                               const double *lb_next, const double *lw_obj, const double *lc_obj,
                               double *l_wrench, double *lb_cur, double *gbody)
{
    const int b = threadIdx.x;
    if (b >= nb) return;
    for (int k = 0; k < kBodyAdj; ++k) {
        gbody[kBodyAdj * b + k] = 0.0;
        gbody[kBodyAdj * (nb + b) + k] = 0.0;
    }
    const BodyDev &B = bodies[b];
    const double *ln = lb_next + kBodyAdj * b;
    double *lc_ = lb_cur + kBodyAdj * b;
    double lc[3], lv[3];
    for (int k = 0; k < 3; ++k) {
        lc[k] = ln[kBodyC + k] + (lc_obj ? lc_obj[3 * b + k] : 0.0);
        lv[k] = ln[kBodyV + k] + dt * lc[k];           // c' = c + dt v'
    }
    for (int k = 0; k < 3; ++k) {
        double lF = 0.0;
        if (B.dof & (1 << k)) {
            const double la = ln[kBodyA + k] + dt * lv[k];   // v' = v + dt a, acc' = a
            lF = la / B.mass;
        }
        l_wrench[6 * b + k] = lF + (lw_obj ? lw_obj[6 * b + k] : 0.0);
        l_wrench[6 * b + 3 + k] = lw_obj ? lw_obj[6 * b + 3 + k] : 0.0;
        lc_[kBodyC + k] = lc[k];
        lc_[kBodyV + k] = lv[k];
        lc_[kBodyA + k] = 0.0;
        lc_[kBodyW + k] = 0.0;
        lc_[kBodyAlpha + k] = 0.0;
    }
    // q' = exp(w' dt / 2) q
    double lw1[3] = {ln[kBodyW], ln[kBodyW + 1], ln[kBodyW + 2]};
    turn_adjoint(after[b].twist + 3, dt, ln + kBodyTheta, lc_ + kBodyTheta, lw1);
    // w' = w + dt wd on the free components (w' = w on the others), alpha' = wd there
    double lwd[3] = {0.0, 0.0, 0.0};
    bool free_rot = false;
    for (int k = 0; k < 3; ++k) {
        lc_[kBodyW + k] = lw1[k];
        if (B.dof & (8 << k)) {
            lwd[k] = dt * lw1[k] + ln[kBodyAlpha + k];
            free_rot = true;
        }
    }
    if (free_rot) {
        // wd = I_w^-1 rhs, rhs = T - w x h, h = I_w w, I_w = R diag(I) R^T; a world
        // turn d theta changes I_w by [d theta]x I_w - I_w [d theta]x
        const double *q = B.pose + 3, *w = B.twist + 3;
        double h[3], rhs[3], wd[3], lrhs[3];
        inertia_world(q, B.inertia, w, false, h);
        double wxh[3];
        cross3(w, h, wxh);
        for (int k = 0; k < 3; ++k) rhs[k] = after[b].wrench[3 + k] + B.load[3 + k] - wxh[k];
        inertia_world(q, B.inertia, rhs, true, wd);
        inertia_world(q, B.inertia, lwd, true, lrhs);
        for (int k = 0; k < 3; ++k) l_wrench[6 * b + 3 + k] += lrhs[k];   // rhs = T - ...
        double t1[3], t2[3];
        cross3(wd, lwd, t1);
        cross3(rhs, lrhs, t2);
        for (int k = 0; k < 3; ++k) lc_[kBodyTheta + k] += t1[k] - t2[k];     // through I_w^-1
        // rhs = T - w x h: (w x h) . l = w . (h x l) = h . (l x w)
        double hxl[3], lh[3], Ilh[3], wxIlh[3], hxlh[3];
        cross3(h, lrhs, hxl);
        cross3(w, lrhs, lh);                    // l_h = -(l x w) = w x l
        inertia_world(q, B.inertia, lh, false, Ilh);
        cross3(w, Ilh, wxIlh);
        cross3(h, lh, hxlh);
        for (int k = 0; k < 3; ++k) {
            lc_[kBodyW + k] += -hxl[k] + Ilh[k];                   // h = I_w w
            lc_[kBodyTheta + k] += hxlh[k] - wxIlh[k];            // through I_w in h
        }
    }
}

// The stages' body adjoints into the body before the step: the midpoint
// markers sit at c + dt/2 v, turned by exp(w dt / 4), with velocity v, rate w
// and acceleration acc (of the previous update); the stage-1 markers at c.
__global__ void k_adj_body_post(int nb, const BodyDev *bodies, double dt, const double *g0,
                                const double *gm, double *lb)
{
    const int b = threadIdx.x;
    if (b >= nb) return;
    const double *a0 = g0 + kBodyAdj * b, *am = gm + kBodyAdj * b;
    double *l = lb + kBodyAdj * b;
    for (int k = 0; k < 3; ++k) {
        l[kBodyC + k] += a0[kBodyC + k] + am[kBodyC + k];
        l[kBodyV + k] += a0[kBodyV + k] + am[kBodyV + k] + 0.5 * dt * am[kBodyC + k];
        l[kBodyA + k] += a0[kBodyA + k] + am[kBodyA + k];
        l[kBodyTheta + k] += a0[kBodyTheta + k];
        l[kBodyW + k] += a0[kBodyW + k] + am[kBodyW + k];
        l[kBodyAlpha + k] += a0[kBodyAlpha + k] + am[kBodyAlpha + k];
    }
    double lt[3];
    turn_adjoint(bodies[b].twist + 3, 0.5 * dt, am + kBodyTheta, lt, l + kBodyW);
    for (int k = 0; k < 3; ++k) l[kBodyTheta + k] += lt[k];
}

// ---------------------------------------------------------------------------
void launch_adj_fluid_coef(int mode, const DevParams &p, const AdjStage &V, StageArrays Y0,
                           const AdjIO &io, double *gpar, cudaStream_t st)
{
    const unsigned g = grid_for(p.capF, kAdjBlock);
    if (mode == kAdjEval)
        k_adj_fluid_coef<kAdjEval><<<g, kAdjBlock, 0, st>>>(p, V, Y0, io, gpar);
    else if (mode == kAdjStage2)
        k_adj_fluid_coef<kAdjStage2><<<g, kAdjBlock, 0, st>>>(p, V, Y0, io, gpar);
    else
        k_adj_fluid_coef<kAdjStage1><<<g, kAdjBlock, 0, st>>>(p, V, Y0, io, gpar);
}

void launch_adj_marker(bool acc, const DevParams &p, const AdjStage &V, const AdjIO &io,
                       double *gpar, double *gbody, cudaStream_t st, const uint32_t *act,
                       const int *n_act)
{
    if (p.capM == 0) return;
    constexpr int LN = kAdjLanes;
    const unsigned g = grid_for((int64_t)p.capM * LN, kAdjBlock);
    if (acc) k_adj_marker<true, LN><<<g, kAdjBlock, 0, st>>>(p, V, io, gpar, gbody, act, n_act);
    else k_adj_marker<false, LN><<<g, kAdjBlock, 0, st>>>(p, V, io, gpar, gbody, act, n_act);
}

void launch_adj_fluid(bool acc, int out, const DevParams &p, const AdjStage &V, const AdjIO &io,
                      float *l_acc, float *l_final, double *gpar, cudaStream_t st)
{
    constexpr int LN = kAdjLanes;
    const unsigned g = grid_for((int64_t)p.capF * LN, kAdjBlock);
    if (acc) {
        if (out == kAdjAccumulate)
            k_adj_fluid<true, kAdjAccumulate, LN><<<g, kAdjBlock, 0, st>>>(p, V, io, l_acc, l_final, gpar);
        else
            k_adj_fluid<true, kAdjFinal, LN><<<g, kAdjBlock, 0, st>>>(p, V, io, l_acc, l_final, gpar);
    } else {
        if (out == kAdjAccumulate)
            k_adj_fluid<false, kAdjAccumulate, LN><<<g, kAdjBlock, 0, st>>>(p, V, io, l_acc, l_final, gpar);
        else
            k_adj_fluid<false, kAdjFinal, LN><<<g, kAdjBlock, 0, st>>>(p, V, io, l_acc, l_final, gpar);
    }
}

static_assert(kMaxBodies <= 32, "the body kernels run one warp, one thread per body");

void launch_adj_body_pre(int nb, const BodyDev *bodies, const BodyDev *after, double dt,
                         const double *lb_next, const double *lw_obj, const double *lc_obj,
                         double *l_wrench, double *lb_cur, double *gbody, cudaStream_t st)
{
    if (nb == 0) return;
    k_adj_body_pre<<<1, 32, 0, st>>>(nb, bodies, after, dt, lb_next, lw_obj, lc_obj, l_wrench,
                                     lb_cur, gbody);
}

void launch_adj_body_post(int nb, const BodyDev *bodies, double dt, const double *g0,
                          const double *gm, double *lb, cudaStream_t st)
{
    if (nb == 0) return;
    k_adj_body_post<<<1, 32, 0, st>>>(nb, bodies, dt, g0, gm, lb);
}

}  // namespace crm
