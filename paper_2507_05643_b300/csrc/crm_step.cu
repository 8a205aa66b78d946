// crm_step.cu -- per-stage kernels of the SPH continuum step (Sec. 2.1-2.4).
//
// One step (explicit midpoint, Sec. 2.2) runs
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
#include "crm_internal.cuh"

namespace crm {

// Cell offsets of the neighbour codes (dx, dy, dz in {-1, 0, 1}) times the cell
// size, built once per block in shared memory.
__device__ __forceinline__ void fill_shift_table(float4 *lut, float cell)
{
    const int t = threadIdx.x;
    if (t < 64) {
        const int dx = (t & 3) - 1, dy = ((t >> 2) & 3) - 1, dz = (t >> 4) - 1;
        lut[t] = make_float4((float)dx * cell, (float)dy * cell, (float)dz * cell, 0.0f);
    }
}

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
// Neighbour lists a kernel walks (and, when filtering, writes).
struct ListIO {
    const uint32_t *in;   // list walked (the skin list when filtering)
    const uint32_t *in_n;
    uint32_t *out;        // exact list written when filtering
    uint32_t *out_n;
    int *err;
};

constexpr int kPairBlock = 128;   // pair kernels: 7 blocks of 128 per SM (72 registers)

template <int MODE, bool FILTER>
__global__ void __launch_bounds__(kPairBlock, 7)
k_pair(DevParams p, StageArrays S, StageArrays Y, StageArrays MID, ListIO io,
       const uint32_t *__restrict__ pid, float dt, RateOut out, int *__restrict__ err,
       const float4 *__restrict__ xref, int *__restrict__ gate)
{
    if (*p.abort) return;
    __shared__ float4 lut[64];
    fill_shift_table(lut, p.cell);
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= __ldg(p.sizes)) return;
    // Extended-Active particles (active domains) are read-only neighbours
    const bool adv = pid == nullptr || !(pid[i] & kExtendedBit);
    if (!adv) {
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
        return;
    }
    const float4 pi = S.pos[i];
    const float4 vi = S.vel[i];
    const float4 ai = S.sA[i];
    const float2 bi = S.sB[i];
    float cont = 0.f, mx = 0.f, my = 0.f, mz = 0.f, avx = 0.f, avy = 0.f, avz = 0.f;
    float L[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) L[k] = 0.f;
    const int nn = (int)io.in_n[i];
    const uint32_t *row = io.in + i;
    int cnt = 0;
    // the next list entry is fetched one iteration ahead; on an exact list the
    // neighbour's whole state is gathered at once (one load round per
    // iteration), on a skin list only after the distance test
    uint32_t e_nx = nn > 0 ? __ldg(row) : 0u;
    for (int k = 0; k < nn; ++k) {
        const uint32_t e = e_nx;
        if (k + 1 < nn) e_nx = __ldg(row + (size_t)(k + 1) * p.ell);
        const uint32_t j = e & kIndexMask;
        const float4 sh = lut[e >> kIndexBits];
        const float4 pj = __ldg(&S.pos[j]);
        float4 vj, aj;
        float2 bj;
        if (!FILTER) {
            vj = __ldg(&S.vel[j]);
            aj = __ldg(&S.sA[j]);
            bj = __ldg(&S.sB[j]);
        }
        const float rx = pi.x - pj.x - sh.x, ry = pi.y - pj.y - sh.y, rz = pi.z - pj.z - sh.z;
        const float r2 = rx * rx + ry * ry + rz * rz;
        if (!(r2 < p.four_h2)) continue;
        if (FILTER) {
            // stage 1 with a skin: the pairs closer than 2h now are the exact list
            if (cnt < p.maxnb) io.out[(size_t)cnt * p.ell + i] = e;
            ++cnt;
            vj = __ldg(&S.vel[j]);
            aj = __ldg(&S.sA[j]);
            bj = __ldg(&S.sB[j]);
        }
        if (r2 == 0.0f) continue;
        const float rinv = rsqrtf(r2);
        const float q = r2 * rinv * p.inv_h;
        const float f = kernel_dw_over_r(q, rinv, p);
        const float gx = f * rx, gy = f * ry, gz = f * rz;          // grad_i W_ij
        const float Vj = __fdividef(p.m, vj.w);   // MUFU reciprocal: ~2 ulp
        const float ux = vj.x - vi.x, uy = vj.y - vi.y, uz = vj.z - vi.z;   // u_ji
        // continuity (F2)
        cont = fmaf(Vj, ux * gx + uy * gy + uz * gz, cont);
        // momentum (F3): (sigma_i + sigma_j) . grad W
        const float sxx = ai.x + aj.x, syy = ai.y + aj.y, szz = ai.z + aj.z;
        const float sxy = ai.w + aj.w, sxz = bi.x + bj.x, syz = bi.y + bj.y;
        mx = fmaf(Vj, sxx * gx + sxy * gy + sxz * gz, mx);
        my = fmaf(Vj, sxy * gx + syy * gy + syz * gz, my);
        mz = fmaf(Vj, sxz * gx + syz * gy + szz * gz, mz);
        // velocity gradient (F2): L += V_j u_ji (x) grad W
        const float vx = Vj * ux, vy = Vj * uy, vz = Vj * uz;
        L[0] = fmaf(vx, gx, L[0]); L[1] = fmaf(vx, gy, L[1]); L[2] = fmaf(vx, gz, L[2]);
        L[3] = fmaf(vy, gx, L[3]); L[4] = fmaf(vy, gy, L[4]); L[5] = fmaf(vy, gz, L[5]);
        L[6] = fmaf(vz, gx, L[6]); L[7] = fmaf(vz, gy, L[7]); L[8] = fmaf(vz, gz, L[8]);
        // artificial viscosity: v_ij . r_ij = -(u_ji . r_ij)
        if (p.av_mode != CRM_AV_NONE) {
            const float vr = -(ux * rx + uy * ry + uz * rz);
            if (p.av_mode == CRM_AV_BILATERAL || vr < 0.0f) {
                const float fac = __fdividef(2.0f * p.av_c * vr, (vi.w + vj.w) * (r2 + p.xi2));
                avx = fmaf(fac, gx, avx);
                avy = fmaf(fac, gy, avy);
                avz = fmaf(fac, gz, avz);
            }
        }
    }
    if (FILTER) {
        if (cnt > p.maxnb) atomicOr(err, ERR_CAPACITY);
        io.out_n[i] = (uint32_t)min(cnt, p.maxnb);
    }
    const float rinv_i = 1.0f / vi.w;
    const float drho = -vi.w * cont;
    const float dux = mx * rinv_i + p.gx + avx;
    const float duy = my * rinv_i + p.gy + avy;
    const float duz = mz * rinv_i + p.gz + avz;
    const float si[6] = {ai.x, ai.y, ai.z, ai.w, bi.x, bi.y};
    float ds[6];
    stress_rate(L, si, p.G, p.K, ds);
    if (MODE == kEval) {
        out.drho[i] = drho;
        out.du[i] = make_float4(dux, duy, duz, 0.f);
        out.dsA[i] = make_float4(ds[0], ds[1], ds[2], ds[3]);
        out.dsB[i] = make_float2(ds[4], ds[5]);
    } else if (MODE == kStage1) {
        const float h = 0.5f * dt;
        MID.pos[i] = make_float4(fmaf(h, vi.x, pi.x), fmaf(h, vi.y, pi.y), fmaf(h, vi.z, pi.z), pi.w);
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
        Y.pos[i] = np;
        Y.vel[i] = nv;
        Y.sA[i] = make_float4(s1[0], s1[1], s1[2], s1[3]);
        Y.sB[i] = make_float2(s1[4], s1[5]);
    }
}

// BCE marker state (Sec. 2.4) at stage offset tau, written into the marker
// slots of S.  The home cell of each slot is read from `home_pos` -- the main
// arrays, whose cell ids the last rebuild set -- so that the marker offset is
// relative to the cell its neighbour codes were built against.
//   Velocity (Adami): u_a = 2 u_body - sum_f u_f W / sum_f W.
//   Stress: sigma_a = [sum_f sigma_f W - ((g - a_body) . sum_f rho_f (x_a - x_f) W) I]
//   / sum_f W (the pressure extrapolation of the cited scheme in stress form);
//   without fluid in reach u_a = u_body and sigma_a = 0.
// ACCEL: 0 = state only; 1 = also the accelerations of body markers, reduced
// per block into FP64 force / torque partials, after which the last block to
// finish sums the partials in a fixed order and advances the bodies (the wrench
// and body update of Sec. 2.4); 2 = the accelerations of every marker, written
// to mforce (rate evaluation).  Acceleration: a_a = (1/rho0) sum_f V_f
// (sigma_a + sigma_f) . grad_a W_af + AV, no gravity.
// FILTER (stage 1 with a Verlet skin): the marker walks its skin list and keeps
// the fluid particles closer than 2h as its exact list for the rest of the step.
// Each marker is served by kBceLanes lanes that stride over its list; a marker
// without fluid neighbours is not read by anyone (the relation is symmetric),
// so its lanes only take part in the warp and block reductions.
struct BodyStep {
    double *partial;      // [block][body][6]
    unsigned *ticket;     // last-block counter (reset by the last block)
    BodyDev *bodies;      // advanced by the last block
    double dt;
    int integrate;
    int *gate;            // skin bookkeeping (nullable): marker displacement bound
};


constexpr int kBceLanes = 4;   // lanes sharing one marker's neighbour list

// Sum over the kBceLanes lanes of a marker's group (every lane of the warp calls it).
__device__ __forceinline__ float group_sum(float v)
{
#pragma unroll
    for (int o = 1; o < kBceLanes; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// ACCEL == 1 tail of k_bce: FP64 per-block partial wrench of every body, then
// the last block sums the partials in a fixed order and advances the bodies.
__device__ __forceinline__ void body_wrench_tail(const DevParams &p, const float f[3],
                                                 const float arm[3], int body, bool mine,
                                                 const BodyStep &bs, unsigned &s_bodies,
                                                 unsigned &s_last, double (*red)[6])
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (mine) atomicOr(&s_bodies, 1u << body);
    __syncthreads();
    const int nb = p.n_bodies;
    for (int b = 0; b < nb; ++b) {
        const bool present = (s_bodies >> b) & 1u;
        if (present) {
            double v[6] = {0, 0, 0, 0, 0, 0};
            if (mine && body == b) {
                v[0] = f[0]; v[1] = f[1]; v[2] = f[2];
                v[3] = (double)arm[1] * f[2] - (double)arm[2] * f[1];
                v[4] = (double)arm[2] * f[0] - (double)arm[0] * f[2];
                v[5] = (double)arm[0] * f[1] - (double)arm[1] * f[0];
            }
#pragma unroll
            for (int k = 0; k < 6; ++k)
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], off);
            if (lane == 0)
#pragma unroll
                for (int k = 0; k < 6; ++k) red[warp][k] = v[k];
        }
        __syncthreads();
        if (threadIdx.x < 6) {
            double a = 0.0;
            if (present)
                for (int w = 0; w < kBlock / 32; ++w) a += red[w][threadIdx.x];
            bs.partial[((size_t)blockIdx.x * nb + b) * 6 + threadIdx.x] = a;
        }
        __syncthreads();
    }
    __threadfence();
    if (threadIdx.x == 0) s_last = atomicAdd(bs.ticket, 1u) == gridDim.x - 1 ? 1u : 0u;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    for (int b = 0; b < nb; ++b) {
        double v[6] = {0, 0, 0, 0, 0, 0};
        for (unsigned q = threadIdx.x; q < gridDim.x; q += blockDim.x)
#pragma unroll
            for (int k = 0; k < 6; ++k)
                v[k] += ((volatile double *)bs.partial)[((size_t)q * nb + b) * 6 + k];
#pragma unroll
        for (int k = 0; k < 6; ++k)
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], off);
        if (lane == 0)
#pragma unroll
            for (int k = 0; k < 6; ++k) red[warp][k] = v[k];
        __syncthreads();
        if (threadIdx.x == 0) {
            double W[6] = {0, 0, 0, 0, 0, 0};
            for (int w = 0; w < kBlock / 32; ++w)
                for (int k = 0; k < 6; ++k) W[k] += red[w][k];
            BodyDev &B = bs.bodies[b];
            for (int k = 0; k < 6; ++k) B.wrench[k] = W[k];
            if (bs.integrate) {
                // symplectic Euler on the free linear DOFs: v += dt (F/m + g), x += dt v;
                // prescribed DOFs move with their velocity; the orientation turns by dt w
                for (int k = 0; k < 3; ++k) {
                    if (B.dof & (1 << k)) {
                        const double a = W[k] / B.mass + p.g64[k];
                        B.twist[k] += bs.dt * a;
                        B.acc[k] = a;
                    } else {
                        B.acc[k] = 0.0;
                    }
                    B.pose[k] += bs.dt * B.twist[k];
                }
                double q[4];
                qadvance(B.pose + 3, B.twist + 3, bs.dt, q);
                for (int k = 0; k < 4; ++k) B.pose[3 + k] = q[k];
                if (bs.gate != nullptr) {
                    // every marker of the body has moved at most |dc| + 2 sin(theta/2) rmax
                    // since the last cell search (theta: rotation since then)
                    double dc2 = 0.0, w = 0.0;
                    for (int k = 0; k < 3; ++k) {
                        const double d = B.pose[k] - B.ref_pose[k];
                        dc2 += d * d;
                    }
                    for (int k = 0; k < 4; ++k) w += B.pose[3 + k] * B.ref_pose[3 + k];
                    const double sh = sqrt(fmax(0.0, 1.0 - w * w));
                    const double d = sqrt(dc2) + 2.0 * sh * B.rmax;
                    atomicMax(bs.gate + GATE_DISP, __float_as_int((float)(d * d) * 1.0001f));
                }
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) *bs.ticket = 0u;
}

template <int ACCEL, bool FILTER>
__global__ void __launch_bounds__(kBlock)
k_bce(DevParams p, StageArrays S, const float4 *__restrict__ home_pos,
      const uint32_t *__restrict__ pid, const double *__restrict__ mloc,
      const BodyDev *bodies, BodyFrame *frames, ListIO L, const uint32_t *__restrict__ act,
      const int *__restrict__ n_act, double tau, int n_fluid_total, float4 *__restrict__ mforce,
      BodyStep bs)
{
    static_assert(!(FILTER && ACCEL != 0), "filtering runs in stage 1 only (no accelerations)");
    if (*p.abort) return;
    __shared__ float4 lut[64];
    __shared__ double red[kBlock / 32][6];
    __shared__ unsigned s_bodies, s_last;
    if (tau == 0.0 && frames != nullptr && bs.dt > 0.0 && blockIdx.x == 0
        && (int)threadIdx.x < p.n_bodies) {
        // the midpoint frames of the following stage-2 launch, once per step
        body_frame(bodies[threadIdx.x], 0.5 * bs.dt, frames[threadIdx.x]);
    }
    fill_shift_table(lut, p.cell);
    if (threadIdx.x == 0) s_bodies = 0u;
    __syncthreads();
    const Sizes z = load_sizes(p);
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int q = t & (kBceLanes - 1);           // lane within the marker's group
    int s;
    bool valid;
    if (act != nullptr) {                        // the markers with fluid in reach
        const int mk = t / kBceLanes;
        valid = mk < __ldg(n_act);
        s = valid ? (int)__ldg(&act[mk]) : z.N;
    } else {                                     // every marker slot
        s = z.nF + t / kBceLanes;
        valid = s < z.N;
    }
    const int nn = valid ? (int)L.in_n[s] : 0;
    const bool work = nn > 0 || (ACCEL == 2 && valid);
    int body = -1;
    float f[3] = {0.f, 0.f, 0.f}, arm[3] = {0.f, 0.f, 0.f};
    if (__any_sync(0xffffffffu, work)) {
        float o[3] = {0.f, 0.f, 0.f}, ub[3] = {0.f, 0.f, 0.f}, ab[3] = {0.f, 0.f, 0.f};
        float4 home = make_float4(0.f, 0.f, 0.f, 0.f);
        if (work) {
            const uint32_t id = pid[s];
            body = pid_body(id);
            home = home_pos[s];
            if (body >= 0) {
                const int mi = (int)pid_index(id) - n_fluid_total;
                double x[3];
                if (tau == 0.0) marker_now(bodies[body], mloc + 3 * (int64_t)mi, x, ub, ab, arm);
                else marker_at(frames[body], mloc + 3 * (int64_t)mi, x, ub, ab, arm);
                int ix, iy, iz;
                decode_cell(__float_as_uint(home.w), p, ix, iy, iz);
                o[0] = (float)(x[0] - (p.dmin_x + ix * p.cell_d));
                o[1] = (float)(x[1] - (p.dmin_y + iy * p.cell_d));
                o[2] = (float)(x[2] - (p.dmin_z + iz * p.cell_d));
            } else {
                o[0] = home.x; o[1] = home.y; o[2] = home.z;   // fixed: the searched offset
            }
        }
        // pass 1: extrapolation sums, the list strided over the group's lanes
        // (warp-uniform round count; the next entry is fetched one round ahead)
        const uint32_t *row = L.in + s;
        const int rounds = __reduce_max_sync(0xffffffffu, (nn + kBceLanes - 1) / kBceLanes);
        float w = 0.f, sux = 0.f, suy = 0.f, suz = 0.f, sr[3] = {0.f, 0.f, 0.f};
        float ss[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        int cnt = 0;
        uint32_t e_nx = q < nn ? __ldg(row + (size_t)q * p.ell) : 0u;
        for (int r = 0; r < rounds; ++r) {
            const int k = r * kBceLanes + q;
            const uint32_t e = e_nx;
            if (k + kBceLanes < nn) e_nx = __ldg(row + (size_t)(k + kBceLanes) * p.ell);
            bool keep = false;
            float W = 0.f;
            float4 vj = make_float4(0.f, 0.f, 0.f, 0.f), aj = vj;
            float2 bj = make_float2(0.f, 0.f);
            float rx = 0.f, ry = 0.f, rz = 0.f;
            if (k < nn) {
                const uint32_t j = e & kIndexMask;
                const float4 sh = lut[e >> kIndexBits];
                const float4 pj = __ldg(&S.pos[j]);
                vj = __ldg(&S.vel[j]);
                aj = __ldg(&S.sA[j]);
                bj = __ldg(&S.sB[j]);
                rx = o[0] - pj.x - sh.x; ry = o[1] - pj.y - sh.y; rz = o[2] - pj.z - sh.z;
                const float r2 = rx * rx + ry * ry + rz * rz;
                keep = r2 < p.four_h2;
                if (keep) W = kernel_w(sqrtf(r2) * p.inv_h, p);
            }
            if (FILTER) {
                // the kept entries, in list order, become the exact list
                const unsigned b = __ballot_sync(0xffffffffu, keep);
                const unsigned g = (b >> ((threadIdx.x & 31) & ~(kBceLanes - 1))) & ((1u << kBceLanes) - 1u);
                const int at = cnt + __popc(g & ((1u << q) - 1u));
                if (keep && at < p.maxnb) L.out[(size_t)at * p.ell + s] = e;
                cnt += __popc(g);
            }
            w += W;
            sux = fmaf(vj.x, W, sux); suy = fmaf(vj.y, W, suy); suz = fmaf(vj.z, W, suz);
            ss[0] = fmaf(aj.x, W, ss[0]); ss[1] = fmaf(aj.y, W, ss[1]); ss[2] = fmaf(aj.z, W, ss[2]);
            ss[3] = fmaf(aj.w, W, ss[3]); ss[4] = fmaf(bj.x, W, ss[4]); ss[5] = fmaf(bj.y, W, ss[5]);
            const float rw = vj.w * W;
            sr[0] = fmaf(rw, rx, sr[0]); sr[1] = fmaf(rw, ry, sr[1]); sr[2] = fmaf(rw, rz, sr[2]);
        }
        w = group_sum(w);
        sux = group_sum(sux); suy = group_sum(suy); suz = group_sum(suz);
#pragma unroll
        for (int k = 0; k < 6; ++k) ss[k] = group_sum(ss[k]);
#pragma unroll
        for (int k = 0; k < 3; ++k) sr[k] = group_sum(sr[k]);
        if (FILTER && q == 0 && valid) {
            if (cnt > p.maxnb) atomicOr(L.err, ERR_CAPACITY);
            L.out_n[s] = (uint32_t)min(cnt, p.maxnb);
        }
        float ua[3], sa[6];
        if (w > 0.f) {
            const float iw = 1.0f / w;
            ua[0] = 2.f * ub[0] - sux * iw;
            ua[1] = 2.f * ub[1] - suy * iw;
            ua[2] = 2.f * ub[2] - suz * iw;
            const float gp = (p.gx - ab[0]) * sr[0] + (p.gy - ab[1]) * sr[1] + (p.gz - ab[2]) * sr[2];
            sa[0] = (ss[0] - gp) * iw; sa[1] = (ss[1] - gp) * iw; sa[2] = (ss[2] - gp) * iw;
            sa[3] = ss[3] * iw; sa[4] = ss[4] * iw; sa[5] = ss[5] * iw;
        } else {
            ua[0] = ub[0]; ua[1] = ub[1]; ua[2] = ub[2];
#pragma unroll
            for (int k = 0; k < 6; ++k) sa[k] = 0.f;
        }
        if (work && q == 0) {
            S.pos[s] = make_float4(o[0], o[1], o[2], home.w);
            S.vel[s] = make_float4(ua[0], ua[1], ua[2], p.rho0);
            S.sA[s] = make_float4(sa[0], sa[1], sa[2], sa[3]);
            S.sB[s] = make_float2(sa[4], sa[5]);
        }
        if constexpr (ACCEL != 0) {
            // pass 2: marker accelerations (body markers for the wrench; every
            // marker for the rate evaluation)
            const int n2 = (ACCEL == 2 || body >= 0) ? nn : 0;
            const int rounds2 = __reduce_max_sync(0xffffffffu, (n2 + kBceLanes - 1) / kBceLanes);
            float mx = 0.f, my = 0.f, mz = 0.f, avx = 0.f, avy = 0.f, avz = 0.f;
            e_nx = q < n2 ? __ldg(row + (size_t)q * p.ell) : 0u;
            for (int r = 0; r < rounds2; ++r) {
                const int k = r * kBceLanes + q;
                const uint32_t e = e_nx;
                if (k + kBceLanes < n2) e_nx = __ldg(row + (size_t)(k + kBceLanes) * p.ell);
                if (k >= n2) continue;
                const uint32_t j = e & kIndexMask;
                const float4 sh = lut[e >> kIndexBits];
                const float4 pj = __ldg(&S.pos[j]);
                const float4 vj = __ldg(&S.vel[j]);
                const float4 aj = __ldg(&S.sA[j]);
                const float2 bj = __ldg(&S.sB[j]);
                const float rx = o[0] - pj.x - sh.x, ry = o[1] - pj.y - sh.y, rz = o[2] - pj.z - sh.z;
                const float r2 = rx * rx + ry * ry + rz * rz;
                if (!(r2 < p.four_h2) || r2 == 0.0f) continue;
                const float rinv = rsqrtf(r2);
                const float fk = kernel_dw_over_r(r2 * rinv * p.inv_h, rinv, p);
                const float gx = fk * rx, gy = fk * ry, gz = fk * rz;
                const float Vj = __fdividef(p.m, vj.w);   // MUFU reciprocal: ~2 ulp
                const float sxx = sa[0] + aj.x, syy = sa[1] + aj.y, szz = sa[2] + aj.z;
                const float sxy = sa[3] + aj.w, sxz = sa[4] + bj.x, syz = sa[5] + bj.y;
                mx = fmaf(Vj, sxx * gx + sxy * gy + sxz * gz, mx);
                my = fmaf(Vj, sxy * gx + syy * gy + syz * gz, my);
                mz = fmaf(Vj, sxz * gx + syz * gy + szz * gz, mz);
                if (p.av_mode != CRM_AV_NONE) {
                    const float vr = (ua[0] - vj.x) * rx + (ua[1] - vj.y) * ry + (ua[2] - vj.z) * rz;
                    if (p.av_mode == CRM_AV_BILATERAL || vr < 0.0f) {
                        const float fac = __fdividef(2.0f * p.av_c * vr, (p.rho0 + vj.w) * (r2 + p.xi2));
                        avx = fmaf(fac, gx, avx);
                        avy = fmaf(fac, gy, avy);
                        avz = fmaf(fac, gz, avz);
                    }
                }
            }
            if (rounds2 > 0) {
                mx = group_sum(mx); my = group_sum(my); mz = group_sum(mz);
                avx = group_sum(avx); avy = group_sum(avy); avz = group_sum(avz);
            }
            const float ir = 1.0f / p.rho0;
            f[0] = p.m * (mx * ir + avx);
            f[1] = p.m * (my * ir + avy);
            f[2] = p.m * (mz * ir + avz);
        }
    } else if (FILTER && valid && q == 0) {
        L.out_n[s] = 0u;
    }
    if constexpr (ACCEL == 2) {
        if (valid && q == 0) mforce[s - z.nF] = make_float4(f[0], f[1], f[2], __int_as_float(body));
    } else if constexpr (ACCEL == 1) {
        body_wrench_tail(p, f, arm, body, q == 0 && nn > 0 && body >= 0, bs, s_bodies, s_last, red);
    }
}

// Markers with a non-empty list, compacted in slot order at each list rebuild
// (most wall markers have no fluid in reach; the BCE kernels then run over the
// active ones only).  Two passes without inter-block waits: per-block counts,
// then each block sums the counts before it and places its markers by ballot.
constexpr int kCompactBlock = 256;

__global__ void __launch_bounds__(kCompactBlock)
k_marker_counts(DevParams p, const uint32_t *__restrict__ nnb, uint32_t *__restrict__ bcount)
{
    if (*p.abort || gated_off(p)) return;
    const Sizes z = load_sizes(p);
    const int s = z.nF + blockIdx.x * blockDim.x + threadIdx.x;
    const int c = __syncthreads_count(s < z.N && nnb[s] > 0u);
    if (threadIdx.x == 0) bcount[blockIdx.x] = (uint32_t)c;
}

__global__ void __launch_bounds__(kCompactBlock)
k_marker_compact(DevParams p, const uint32_t *__restrict__ nnb, const uint32_t *__restrict__ bcount,
                 uint32_t *__restrict__ act, int *__restrict__ n_act, uint32_t *__restrict__ nnb_exact)
{
    if (*p.abort || gated_off(p)) return;
    __shared__ uint32_t s_sum[kCompactBlock / 32], s_cnt[kCompactBlock / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t acc = 0;
    for (int b = threadIdx.x; b < (int)blockIdx.x; b += blockDim.x) acc += bcount[b];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    const Sizes z = load_sizes(p);
    const int s = z.nF + blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = s < z.N;
    const bool a = valid && nnb[s] > 0u;
    const unsigned bits = __ballot_sync(0xffffffffu, a);
    if (lane == 0) {
        s_sum[warp] = acc;
        s_cnt[warp] = (uint32_t)__popc(bits);
    }
    __syncthreads();
    uint32_t off = 0;
    for (int w = 0; w < kCompactBlock / 32; ++w) off += s_sum[w] + (w < warp ? s_cnt[w] : 0u);
    if (a) act[off + __popc(bits & ((1u << lane) - 1u))] = (uint32_t)s;
    else if (valid && nnb_exact != nullptr) nnb_exact[s] = 0u;   // no skin neighbours: none within 2h
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == kCompactBlock - 1)
        *n_act = (int)(off + __popc(bits & ((1u << lane) - 1u)) + (a ? 1u : 0u));
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
void launch_pair(int mode, const DevParams &p, StageArrays S, StageArrays Y, StageArrays MID,
                 const uint32_t *nbr, const uint32_t *nnb, const uint32_t *integrate, float dt,
                 RateOut out, int *err, const float4 *xref, int *gate, cudaStream_t st,
                 const uint32_t *sk_nbr, const uint32_t *sk_nnb)
{
    const unsigned g = grid_for(p.capF, kPairBlock);
    if (mode == kStage1 && sk_nbr != nullptr) {
        const ListIO L{sk_nbr, sk_nnb, const_cast<uint32_t *>(nbr), const_cast<uint32_t *>(nnb), err};
        k_pair<kStage1, true><<<g, kPairBlock, 0, st>>>(p, S, Y, MID, L, integrate, dt, out, err,
                                                     nullptr, nullptr);
        return;
    }
    if (mode == kEval && sk_nbr != nullptr) {
        const ListIO L{sk_nbr, sk_nnb, const_cast<uint32_t *>(nbr), const_cast<uint32_t *>(nnb), err};
        k_pair<kEval, true><<<g, kPairBlock, 0, st>>>(p, S, Y, MID, L, integrate, dt, out, err,
                                                   nullptr, nullptr);
        return;
    }
    const ListIO L{nbr, nnb, nullptr, nullptr, err};
    if (mode == kStage1)
        k_pair<kStage1, false><<<g, kPairBlock, 0, st>>>(p, S, Y, MID, L, integrate, dt, out, err,
                                                      nullptr, nullptr);
    else if (mode == kStage2)
        k_pair<kStage2, false><<<g, kPairBlock, 0, st>>>(p, S, Y, MID, L, integrate, dt, out, err,
                                                      xref, gate);
    else
        k_pair<kEval, false><<<g, kPairBlock, 0, st>>>(p, S, Y, MID, L, integrate, dt, out, err,
                                                    nullptr, nullptr);
}

void launch_bce(const DevParams &p, StageArrays S, const float4 *home_pos, const uint32_t *pid,
                const double *mloc, BodyDev *bodies, const uint32_t *nbr, const uint32_t *nnb,
                double tau, int accel, int n_fluid_total, float4 *mforce, double *partial,
                unsigned *ticket, double dt, int integrate, int *gate, cudaStream_t st,
                const uint32_t *sk_nbr, const uint32_t *sk_nnb, int *err, BodyFrame *frames,
                const uint32_t *act, const int *n_act)
{
    const unsigned g = bce_blocks(p);
    BodyStep bs{partial, ticket, bodies, dt, integrate, gate};
    if (sk_nbr != nullptr) {   // stage 1 with a skin (no accelerations)
        const ListIO L{sk_nbr, sk_nnb, const_cast<uint32_t *>(nbr), const_cast<uint32_t *>(nnb), err};
        k_bce<0, true><<<g, kBlock, 0, st>>>(p, S, home_pos, pid, mloc, bodies, frames, L, act, n_act, tau,
                                             n_fluid_total, mforce, bs);
        return;
    }
    const ListIO L{nbr, nnb, nullptr, nullptr, err};
    if (accel == 0)
        k_bce<0, false><<<g, kBlock, 0, st>>>(p, S, home_pos, pid, mloc, bodies, frames, L, act, n_act, tau,
                                              n_fluid_total, mforce, bs);
    else if (accel == 1)
        k_bce<1, false><<<g, kBlock, 0, st>>>(p, S, home_pos, pid, mloc, bodies, frames, L, act, n_act, tau,
                                              n_fluid_total, mforce, bs);
    else
        k_bce<2, false><<<g, kBlock, 0, st>>>(p, S, home_pos, pid, mloc, bodies, frames, L, act, n_act, tau,
                                              n_fluid_total, mforce, bs);
}

unsigned bce_blocks(const DevParams &p) { return grid_for((int64_t)p.capM * kBceLanes); }

unsigned compact_blocks(const DevParams &p) { return grid_for(p.capM, kCompactBlock); }

void launch_compact_markers(const DevParams &p, const uint32_t *nnb, uint32_t *nnb_exact,
                            uint32_t *bcount, uint32_t *act, int *n_act, cudaStream_t st)
{
    const unsigned g = compact_blocks(p);
    k_marker_counts<<<g, kCompactBlock, 0, st>>>(p, nnb, bcount);
    k_marker_compact<<<g, kCompactBlock, 0, st>>>(p, nnb, bcount, act, n_act, nnb_exact);
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
