// crm_bce.cu -- BCE boundary markers (Sec. 2.4): marker state extrapolated from
// the fluid, marker accelerations, the FP64 body wrench and the body update,
// and the compaction of the markers that have fluid in reach.
#include <algorithm>

#include "crm_internal.cuh"

namespace crm {

// BCE marker state (Sec. 2.4) at stage offset tau, written into the marker
// slots of S.  The home cell of each slot is read from `home_pos` -- the main
// arrays, whose cell ids the last rebuild set -- so that the marker offset is
// relative to the cell its neighbour codes were built against.
//   Velocity (Adami): u_a = 2 u_body - sum_f u_f W / sum_f W.
//   Stress: sigma_a = [sum_f sigma_f W - ((g - a_body) . sum_f rho_f (x_a - x_f) W) I]
//   / sum_f W (the pressure extrapolation of the cited scheme in stress form);
//   without fluid in reach u_a = u_body and sigma_a = 0.
// ACCEL: 0 = state only; 1 = the forces of the active body markers (their
// state already written by a state launch on the same arrays), summed per block
// and body into FP64 force / torque partials, which k_body_reduce sums in a
// fixed order before the body update (the wrench and body update of Sec. 2.4);
// 2 = state and accelerations of every marker, the forces written to mforce
// (rate evaluation).  Acceleration: a_a = (1/rho0) sum_f V_f
// (sigma_a + sigma_f) . grad_a W_af + AV, no gravity.
// FILTER (stage 1 with a Verlet skin): the marker walks its skin list and keeps
// the fluid particles closer than 2h as its exact list for the rest of the step.
// Each marker is served by kBceLanes lanes that stride over its list; a marker
// without fluid neighbours is not read by anyone (the relation is symmetric),
// so its lanes only take part in the warp and block reductions.
struct BodyStep {
    double *partial;      // [block][body][6]: FP64 wrench partials of the wrench pass
    BodyDev *bodies;      // advanced by k_body_reduce
    double dt;
    int integrate;
    int *gate;            // skin bookkeeping (nullable): marker displacement bound
};


constexpr int kBceLanes = 4;      // lanes sharing one marker's neighbour list
constexpr int kWrenchLanes = 16;  // the same for the wrench pass: its few body markers
                                  // would otherwise leave the GPU nearly idle

// Sum over the LANES lanes of a marker's group (every lane of the warp calls it).
template <int LANES>
__device__ __forceinline__ float group_sum(float v)
{
#pragma unroll
    for (int o = 1; o < LANES; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// The end-of-step update of body b from its summed soil wrench W (Sec. 2.4):
// symplectic Euler on the free DOFs with the soil wrench plus the external load,
// v += dt (F/m + g), w += dt I_w^-1 (T - w x I_w w) (I_w = R diag(I) R^T at t_n),
// then x += dt v and the orientation turns by dt w; prescribed DOFs keep their
// velocity.
__device__ __forceinline__ void body_update(const DevParams &p, const BodyStep &bs, int b,
                                            const double W[6])
{
    BodyDev &B = bs.bodies[b];
    for (int k = 0; k < 6; ++k) B.wrench[k] = W[k];
    if (!bs.integrate) return;
    double F[3], T[3], wdot[3] = {0.0, 0.0, 0.0};
    for (int k = 0; k < 3; ++k) {
        F[k] = W[k] + B.load[k];
        T[k] = W[3 + k] + B.load[3 + k];
    }
    if (B.dof & (7 << 3)) {
        const double qw = B.pose[3], qx = B.pose[4], qy = B.pose[5], qz = B.pose[6];
        const double R[3][3] = {
            {1 - 2 * (qy * qy + qz * qz), 2 * (qx * qy - qw * qz), 2 * (qx * qz + qw * qy)},
            {2 * (qx * qy + qw * qz), 1 - 2 * (qx * qx + qz * qz), 2 * (qy * qz - qw * qx)},
            {2 * (qx * qz - qw * qy), 2 * (qy * qz + qw * qx), 1 - 2 * (qx * qx + qy * qy)}};
        const double *w = B.twist + 3;
        double L[3], rb[3];
        for (int r = 0; r < 3; ++r)   // body-frame w, times I
            rb[r] = B.inertia[r] * (R[0][r] * w[0] + R[1][r] * w[1] + R[2][r] * w[2]);
        for (int r = 0; r < 3; ++r) L[r] = R[r][0] * rb[0] + R[r][1] * rb[1] + R[r][2] * rb[2];
        const double rhs[3] = {T[0] - (w[1] * L[2] - w[2] * L[1]), T[1] - (w[2] * L[0] - w[0] * L[2]),
                               T[2] - (w[0] * L[1] - w[1] * L[0])};
        for (int r = 0; r < 3; ++r)
            rb[r] = (R[0][r] * rhs[0] + R[1][r] * rhs[1] + R[2][r] * rhs[2]) / B.inertia[r];
        for (int r = 0; r < 3; ++r) wdot[r] = R[r][0] * rb[0] + R[r][1] * rb[1] + R[r][2] * rb[2];
    }
    for (int k = 0; k < 3; ++k) {
        if (B.dof & (1 << k)) {
            const double a = F[k] * B.inv_mass + p.g64[k];
            B.twist[k] += bs.dt * a;
            B.acc[k] = a;
        } else {
            B.acc[k] = 0.0;
        }
        if (B.dof & (8 << k)) {
            B.twist[3 + k] += bs.dt * wdot[k];
            B.alpha[k] = wdot[k];
        } else {
            B.alpha[k] = 0.0;
        }
        B.pose[k] += bs.dt * B.twist[k];
    }
    double q[4];
    qadvance(B.pose + 3, B.twist + 3, bs.dt, q);
    for (int k = 0; k < 4; ++k) B.pose[3 + k] = q[k];
    if (bs.gate != nullptr) {
        // every marker of the body has moved at most |dc| + 2 sin(theta/2) rmax
        // since the last cell search (theta: rotation since then)
        // (a bound compared with an FP32 threshold: its square roots in FP32,
        // the 1.0001 margin covering their rounding)
        double dc2 = 0.0, w = 0.0;
        for (int k = 0; k < 3; ++k) {
            const double d = B.pose[k] - B.ref_pose[k];
            dc2 += d * d;
        }
        for (int k = 0; k < 4; ++k) w += B.pose[3 + k] * B.ref_pose[3 + k];
        const float sh = sqrtf((float)fmax(0.0, 1.0 - w * w)), dc = sqrtf((float)dc2);
        const float d = dc + 2.0f * sh * (float)B.rmax;
        atomicMax(bs.gate + GATE_DISP, __float_as_int(d * d * 1.0001f));
        if (p.act_skin) {   // the same bound for the body's grown active boxes
            const float db = dc + 2.0f * sh * (float)B.box_reach;
            atomicMax(bs.gate + GATE_BOX, __float_as_int(db * db * 1.0001f));
        }
    }
}

// Wrench partials of one block of the wrench pass: for every body with a
// marker in the block, the FP64 sum of its markers' forces and torques about
// the centre (torque = arm x f, each product exact in FP64), a fixed shuffle
// tree per warp and the warps in order.  FP64 arithmetic is slow on this part,
// so it is spread over the blocks (one partial each) and kept off one SM.
__device__ __forceinline__ void block_wrench_partial(const DevParams &p, const float f[3],
                                                     const float arm[3], int body, bool mine,
                                                     const BodyStep &bs, unsigned &s_bodies,
                                                     double (*red)[6], int vb)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (mine) atomicOr(&s_bodies, 1u << body);
    __syncthreads();
    const int nb = p.n_bodies;
    const unsigned present_all = s_bodies;
    for (int b = 0; b < nb; ++b) {
        const bool present = (present_all >> b) & 1u;
        if (present) {
            double v[6] = {0, 0, 0, 0, 0, 0};
            if (mine && body == b) {
                v[0] = f[0]; v[1] = f[1]; v[2] = f[2];
                v[3] = (double)arm[1] * f[2] - (double)arm[2] * f[1];
                v[4] = (double)arm[2] * f[0] - (double)arm[0] * f[2];
                v[5] = (double)arm[0] * f[1] - (double)arm[1] * f[0];
            }
            if (__any_sync(0xffffffffu, mine && body == b)) {
#pragma unroll
                for (int k = 0; k < 6; ++k)
#pragma unroll
                    for (int off = 16; off > 0; off >>= 1)
                        v[k] += __shfl_down_sync(0xffffffffu, v[k], off);
            }
            if (lane == 0)
#pragma unroll
                for (int k = 0; k < 6; ++k) red[warp][k] = v[k];
        }
        __syncthreads();
        if (threadIdx.x < 6) {
            double a = 0.0;
            if (present)
                for (int w = 0; w < kBlock / 32; ++w) a += red[w][threadIdx.x];
            bs.partial[((size_t)vb * nb + b) * 6 + threadIdx.x] = a;
        }
        __syncthreads();
    }
}

// The work of block vb of a k_bce launch (a kBlock-thread block; every thread
// of the block calls it; red and s_bodies are the block's shared arrays).
template <int ACCEL, bool FILTER, int LANES, int BS = kBlock>
__device__ __forceinline__ void bce_block(const DevParams &p, StageArrays S,
                                          const float4 *__restrict__ home_pos,
                                          const uint32_t *__restrict__ pid,
                                          const double *__restrict__ mloc, const BodyDev *bodies,
                                          BodyFrame *frames, const ListIO &L,
                                          const uint32_t *__restrict__ act,
                                          const int *__restrict__ n_act, double tau,
                                          int n_fluid_total, float4 *__restrict__ mforce,
                                          const BodyStep &bs, int vb,
                                          double (*red)[6], unsigned &s_bodies)
{
    static_assert(!(FILTER && ACCEL != 0), "filtering runs in stage 1 only (no accelerations)");
    if (tau == 0.0 && frames != nullptr && bs.dt > 0.0 && vb == 0
        && (int)threadIdx.x < p.n_bodies) {
        // the midpoint frames of the following stage-2 launch, once per step
        body_frame(bodies[threadIdx.x], 0.5 * bs.dt, frames[threadIdx.x]);
    }
    if (threadIdx.x == 0) s_bodies = 0u;
    __syncthreads();
    const Sizes z = load_sizes(p);
    const int t = vb * BS + threadIdx.x;
    const int q = t & (LANES - 1);           // lane within the marker's group
    int s;
    bool valid;
    if (act != nullptr) {                        // the markers with fluid in reach
        const int mk = t / LANES;
        valid = mk < __ldg(n_act);
        s = valid ? (int)__ldg(&act[mk]) : z.N;
    } else {                                     // every marker slot
        s = z.nF + t / LANES;
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
            body = pid_body(p, id);
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
        const uint32_t *row = L.in + s;
        float ua[3], sa[6];
        uint32_t e_nx;
        if constexpr (ACCEL == 1) {
            // the wrench pass follows a state pass over the same arrays: the
            // marker's extrapolated velocity and stress are in its slot
            const float4 vs = S.vel[s], as = S.sA[s];
            const float2 bs2 = S.sB[s];
            ua[0] = vs.x; ua[1] = vs.y; ua[2] = vs.z;
            sa[0] = as.x; sa[1] = as.y; sa[2] = as.z; sa[3] = as.w; sa[4] = bs2.x; sa[5] = bs2.y;
        } else {
        // pass 1: extrapolation sums, the list strided over the group's lanes
        // (warp-uniform round count; the next entry is fetched one round ahead)
        const int rounds = __reduce_max_sync(0xffffffffu, (nn + LANES - 1) / LANES);
        float w = 0.f, sux = 0.f, suy = 0.f, suz = 0.f, sr[3] = {0.f, 0.f, 0.f};
        float ss[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        int cnt = 0;
        e_nx = q < nn ? ld_list(row + (size_t)q * p.ell) : 0u;
        for (int r = 0; r < rounds; ++r) {
            const int k = r * LANES + q;
            const uint32_t e = e_nx;
            if (k + LANES < nn) e_nx = ld_list(row + (size_t)(k + LANES) * p.ell);
            bool keep = false;
            float W = 0.f;
            float4 vj = make_float4(0.f, 0.f, 0.f, 0.f), aj = vj;
            float2 bj = make_float2(0.f, 0.f);
            float rx = 0.f, ry = 0.f, rz = 0.f;
            if (k < nn) {
                const uint32_t j = e & kIndexMask;
                const float3 sh = entry_shift(e, p.cell);
                const float4 pj = __ldg(&S.pos[j]);
                vj = __ldg(&S.vel[j]);
                aj = __ldg(&S.sA[j]);
                bj = __ldg(&S.sB[j]);
                rx = o[0] - pj.x - sh.x; ry = o[1] - pj.y - sh.y; rz = o[2] - pj.z - sh.z;
                const float r2 = rx * rx + ry * ry + rz * rz;
                keep = r2 < p.four_h2;
                // (active domains with a skin: fluid outside every grown box is in the
                // working set's margin only, and no marker reads it)
                if (FILTER && p.act_skin && keep && (__ldg(pid + j) & kOutsideBit)) keep = false;
                if (keep) W = kernel_w(sqrtf(r2) * p.inv_h, p);
            }
            if (FILTER) {
                // the kept entries, in list order, become the exact list
                const unsigned b = __ballot_sync(0xffffffffu, keep);
                const unsigned g = (b >> ((threadIdx.x & 31) & ~(LANES - 1))) & ((1u << LANES) - 1u);
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
        w = group_sum<LANES>(w);
        sux = group_sum<LANES>(sux); suy = group_sum<LANES>(suy); suz = group_sum<LANES>(suz);
#pragma unroll
        for (int k = 0; k < 6; ++k) ss[k] = group_sum<LANES>(ss[k]);
#pragma unroll
        for (int k = 0; k < 3; ++k) sr[k] = group_sum<LANES>(sr[k]);
        if (FILTER && q == 0 && valid) {
            if (cnt > p.maxnb) atomicOr(L.err, ERR_CAPACITY);
            L.out_n[s] = (uint32_t)min(cnt, p.maxnb);
        }
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
            const float4 mp = make_float4(o[0], o[1], o[2], home.w);
            S.pos[s] = p.abs32 ? round_absolute(p, mp) : mp;
            S.vel[s] = make_float4(ua[0], ua[1], ua[2], p.rho0);
            S.sA[s] = make_float4(sa[0], sa[1], sa[2], sa[3]);
            S.sB[s] = make_float2(sa[4], sa[5]);
        }
        }   // pass 1
        if constexpr (ACCEL != 0) {
            // pass 2: marker accelerations (body markers for the wrench; every
            // marker for the rate evaluation)
            const int n2 = (ACCEL == 2 || body >= 0) ? nn : 0;
            const int rounds2 = __reduce_max_sync(0xffffffffu, (n2 + LANES - 1) / LANES);
            float mx = 0.f, my = 0.f, mz = 0.f, avx = 0.f, avy = 0.f, avz = 0.f;
            e_nx = q < n2 ? ld_list(row + (size_t)q * p.ell) : 0u;
            for (int r = 0; r < rounds2; ++r) {
                const int k = r * LANES + q;
                const uint32_t e = e_nx;
                if (k + LANES < n2) e_nx = ld_list(row + (size_t)(k + LANES) * p.ell);
                if (k >= n2) continue;
                const uint32_t j = e & kIndexMask;
                const float3 sh = entry_shift(e, p.cell);
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
                mx = group_sum<LANES>(mx); my = group_sum<LANES>(my); mz = group_sum<LANES>(mz);
                avx = group_sum<LANES>(avx); avy = group_sum<LANES>(avy); avz = group_sum<LANES>(avz);
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
        block_wrench_partial(p, f, arm, body, valid && q == 0 && nn > 0 && body >= 0, bs, s_bodies,
                             red, vb);
    }
}

template <int ACCEL, bool FILTER, int LANES = kBceLanes, int BS = kBlock>
__global__ void __launch_bounds__(BS)
k_bce(DevParams p, StageArrays S, const float4 *__restrict__ home_pos,
      const uint32_t *__restrict__ pid, const double *__restrict__ mloc,
      const BodyDev *bodies, BodyFrame *frames, ListIO L, const uint32_t *__restrict__ act,
      const int *__restrict__ n_act, double tau, int n_fluid_total, float4 *__restrict__ mforce,
      BodyStep bs)
{
    if (*p.abort) return;
    __shared__ double red[kBlock / 32][6];
    __shared__ unsigned s_bodies;
    if constexpr (ACCEL == 1) {   // one partial per block: one block per virtual block
        bce_block<ACCEL, FILTER, LANES>(p, S, home_pos, pid, mloc, bodies, frames, L, act, n_act,
                                        tau, n_fluid_total, mforce, bs, blockIdx.x, red, s_bodies);
        return;
    }
    // the state passes: a grid of at most one wave takes the virtual blocks that
    // hold markers in turn (block 0 always runs: it writes the midpoint frames)
    const int live = act != nullptr ? __ldg(n_act) : __ldg(p.sizes + 2) - __ldg(p.sizes);
    const int nvb = max(1, (int)(((int64_t)live * LANES + BS - 1) / BS));
    for (int vb = blockIdx.x; vb < nvb; vb += gridDim.x)
        bce_block<ACCEL, FILTER, LANES, BS>(p, S, home_pos, pid, mloc, bodies, frames, L, act,
                                            n_act, tau, n_fluid_total, mforce, bs, vb, red, s_bodies);
}

// The state passes run in blocks of kBceStateBlock threads: smaller blocks even
// out the uneven marker work (list lengths, body kinematics) over the SMs.
constexpr int kBceStateBlock = 128;

// Grid of a state pass: the blocks the markers need, at most one wave of the
// kernel's resident blocks.
template <int ACCEL, bool FILTER>
unsigned bce_state_grid(const DevParams &p)
{
    static int per_sm = 0;
    if (per_sm == 0) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                &per_sm, k_bce<ACCEL, FILTER, kBceLanes, kBceStateBlock>, kBceStateBlock, 0)
                != cudaSuccess
            || per_sm < 1) {
            cudaGetLastError();
            per_sm = 1;
        }
    }
    return (unsigned)std::min<int64_t>(grid_for((int64_t)p.capM * kBceLanes, kBceStateBlock),
                                       (int64_t)std::max(p.n_sm, 1) * per_sm);
}

// The soil wrench of body b = blockIdx.x (Sec. 2.4): the sum of the wrench
// pass's block partials in a fixed order (lane l takes blocks l, l + 32, ...,
// then a fixed shuffle tree), then the body update -- one warp per body.
__device__ __forceinline__ void body_reduce_warp(const DevParams &p, const BodyStep &bs, int b,
                                                 const int *__restrict__ n_act_body)
{
    const int lane = threadIdx.x & 31, nb = p.n_bodies;
    // the blocks of the wrench pass that held active body markers
    const int n_blocks = (int)grid_for((int64_t)__ldg(n_act_body) * kWrenchLanes);
    double v[6] = {0, 0, 0, 0, 0, 0};
    for (int q = lane; q < n_blocks; q += 32)
#pragma unroll
        for (int k = 0; k < 6; ++k) v[k] += bs.partial[((size_t)q * nb + b) * 6 + k];
#pragma unroll
    for (int k = 0; k < 6; ++k)
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], off);
    if (lane == 0) body_update(p, bs, b, v);
}

__global__ void __launch_bounds__(32)
k_body_reduce(DevParams p, BodyStep bs, const int *__restrict__ n_act_body)
{
    if (*p.abort) return;
    body_reduce_warp(p, bs, blockIdx.x, n_act_body);
}

// ---------------------------------------------------------------------------
// Batched forms (crm_batch): persistent blocks take virtual blocks off the
// launch's work queue -- an atomic ticket, no waiting -- and run the member's
// block exactly as its own launch would (same lanes, same arithmetic, same
// partial slots), so a batched step equals the members' own steps bit for bit.
__device__ __forceinline__ int batch_member(const int *__restrict__ off, int n, int it)
{
    int lo = 0, hi = n - 1;   // off[lo] <= it < off[lo + 1]
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(off + mid) <= it) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ void batch_done(unsigned *queue)
{
    __syncthreads();
    if (threadIdx.x == 0 && atomicAdd(queue + 1, 1u) == gridDim.x - 1) {
        queue[0] = 0u;   // every block has stopped claiming: reset for the next launch
        queue[1] = 0u;
    }
}

template <int KIND>
__global__ void __launch_bounds__(kBlock)
k_batch_bce(const MemberDev *__restrict__ mem, const int *__restrict__ mlist,
            const int *__restrict__ off, int n, unsigned *queue)
{
    __shared__ double red[kBlock / 32][6];
    __shared__ unsigned s_bodies;
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
            const int k = batch_member(off, n, it);
            if (k != cur) {   // block-uniform
                __syncthreads();
                load_member(mem + __ldg(mlist + k), &M);
                cur = k;
            }
            if (*M.p.abort) continue;
            const int vb = it - __ldg(off + k);
            // the state passes: virtual blocks past the member's markers with fluid in
            // reach hold none (block 0 still runs: it writes the midpoint frames)
            if (KIND != 2 && vb > 0 && (int64_t)vb * kBlock >= (int64_t)*M.n_act * kBceLanes)
                continue;
            __syncthreads();   // the previous virtual block's readers of red are done
            if (KIND == 0) {
                const ListIO L{M.sk_nbr, M.sk_nnb, M.nbr, M.nnb, M.err};
                const BodyStep bs{M.partial, M.bodies, M.dt, 0, M.gate};
                bce_block<0, true, kBceLanes>(M.p, M.S, M.S.pos, M.pid, M.mloc, M.bodies, M.frames,
                                              L, M.act, M.n_act, 0.0, M.n_fluid_total, M.mforce, bs,
                                              vb, red, s_bodies);
            } else if (KIND == 1) {
                const ListIO L{M.nbr, M.nnb, nullptr, nullptr, M.err};
                const BodyStep bs{M.partial, M.bodies, 0.0, 0, M.gate};
                bce_block<0, false, kBceLanes>(M.p, M.MID, M.S.pos, M.pid, M.mloc, M.bodies,
                                               M.frames, L, M.act, M.n_act, 0.5 * M.dt,
                                               M.n_fluid_total, M.mforce, bs, vb, red,
                                               s_bodies);
            } else {
                const ListIO L{M.nbr, M.nnb, nullptr, nullptr, M.err};
                const BodyStep bs{M.partial, M.bodies, M.dt, 1, M.gate};
                bce_block<1, false, kWrenchLanes>(M.p, M.MID, M.S.pos, M.pid, M.mloc, M.bodies,
                                                  M.frames, L, M.act_body, M.n_act + 1, 0.5 * M.dt,
                                                  M.n_fluid_total, M.mforce, bs, vb, red,
                                                  s_bodies);
            }
        }
    }
    batch_done(queue);
}

// One warp per (member, body) pair: pairs[2 k], pairs[2 k + 1].
__global__ void __launch_bounds__(32)
k_batch_reduce(const MemberDev *__restrict__ mem, const int *__restrict__ pairs)
{
    const MemberDev &M = mem[__ldg(pairs + 2 * blockIdx.x)];
    if (*M.p.abort) return;
    const BodyStep bs{M.partial, M.bodies, M.dt, 1, M.gate};
    body_reduce_warp(M.p, bs, __ldg(pairs + 2 * blockIdx.x + 1), M.n_act + 1);
}

// Markers with a non-empty list, compacted in slot order at each list rebuild
// (most wall markers have no fluid in reach; the BCE kernels then run over the
// active ones only).  Two passes without inter-block waits: per-block counts,
// then each block sums the counts before it and places its markers by ballot.
constexpr int kCompactBlock = 256;

// list 0: every marker with a non-empty list; list 1: those of them on a body.
__device__ __forceinline__ void marker_activity(const DevParams &p, const Sizes &z,
                                                const uint32_t *nnb, const uint32_t *pid, int s,
                                                bool &valid, bool a[2])
{
    valid = s < z.N;
    a[0] = valid && nnb[s] > 0u;
    a[1] = a[0] && pid_body(p, pid[s]) >= 0;
}

__global__ void __launch_bounds__(kCompactBlock)
k_marker_counts(DevParams p, const uint32_t *__restrict__ nnb, const uint32_t *__restrict__ pid,
                uint32_t *__restrict__ bcount)
{
    if (*p.abort || gated_off(p)) return;
    const Sizes z = load_sizes(p);
    bool valid, a[2];
    marker_activity(p, z, nnb, pid, z.nF + blockIdx.x * blockDim.x + threadIdx.x, valid, a);
    const int c0 = __syncthreads_count(a[0]);
    const int c1 = __syncthreads_count(a[1]);
    if (threadIdx.x == 0) {
        bcount[2 * blockIdx.x] = (uint32_t)c0;
        bcount[2 * blockIdx.x + 1] = (uint32_t)c1;
    }
}

__global__ void __launch_bounds__(kCompactBlock)
k_marker_compact(DevParams p, const uint32_t *__restrict__ nnb, const uint32_t *__restrict__ pid,
                 const uint32_t *__restrict__ bcount, uint32_t *__restrict__ act,
                 uint32_t *__restrict__ act_body, int *__restrict__ n_act,
                 uint32_t *__restrict__ nnb_exact)
{
    if (*p.abort || gated_off(p)) return;
    __shared__ uint32_t s_sum[2][kCompactBlock / 32], s_cnt[2][kCompactBlock / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t acc[2] = {0u, 0u};
    for (int b = threadIdx.x; b < (int)blockIdx.x; b += blockDim.x) {
        acc[0] += bcount[2 * b];
        acc[1] += bcount[2 * b + 1];
    }
    const Sizes z = load_sizes(p);
    const int s = z.nF + blockIdx.x * blockDim.x + threadIdx.x;
    bool valid, a[2];
    marker_activity(p, z, nnb, pid, s, valid, a);
    unsigned bits[2];
#pragma unroll
    for (int l = 0; l < 2; ++l) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc[l] += __shfl_xor_sync(0xffffffffu, acc[l], o);
        bits[l] = __ballot_sync(0xffffffffu, a[l]);
        if (lane == 0) {
            s_sum[l][warp] = acc[l];
            s_cnt[l][warp] = (uint32_t)__popc(bits[l]);
        }
    }
    __syncthreads();
    const unsigned below = (1u << lane) - 1u;
    uint32_t *const out[2] = {act, act_body};
#pragma unroll
    for (int l = 0; l < 2; ++l) {
        uint32_t off = 0;
        for (int w = 0; w < kCompactBlock / 32; ++w) off += s_sum[l][w] + (w < warp ? s_cnt[l][w] : 0u);
        const uint32_t at = off + __popc(bits[l] & below);
        if (a[l]) out[l][at] = (uint32_t)s;
        if (blockIdx.x == gridDim.x - 1 && threadIdx.x == kCompactBlock - 1)
            n_act[l] = (int)(at + (a[l] ? 1u : 0u));
    }
    if (valid && !a[0] && nnb_exact != nullptr) nnb_exact[s] = 0u;   // no skin neighbours: none within 2h
}

// ---------------------------------------------------------------------------
// Host-side launchers used by the API translation unit.
void launch_bce(const DevParams &p, StageArrays S, const float4 *home_pos, const uint32_t *pid,
                const double *mloc, BodyDev *bodies, const uint32_t *nbr, const uint32_t *nnb,
                double tau, int accel, int n_fluid_total, float4 *mforce, double *partial,
                double dt, int integrate, int *gate, cudaStream_t st,
                const uint32_t *sk_nbr, const uint32_t *sk_nnb, int *err, BodyFrame *frames,
                const uint32_t *act, const int *n_act, int64_t body_markers)
{
    BodyStep bs{partial, bodies, dt, integrate, gate};
    if (sk_nbr != nullptr) {   // stage 1 with a skin (no accelerations)
        const ListIO L{sk_nbr, sk_nnb, const_cast<uint32_t *>(nbr), const_cast<uint32_t *>(nnb), err};
        k_bce<0, true, kBceLanes, kBceStateBlock><<<bce_state_grid<0, true>(p), kBceStateBlock, 0, st>>>(
            p, S, home_pos, pid, mloc, bodies, frames, L, act, n_act, tau, n_fluid_total, mforce, bs);
        return;
    }
    const ListIO L{nbr, nnb, nullptr, nullptr, err};
    if (accel == 0) {
        k_bce<0, false, kBceLanes, kBceStateBlock><<<bce_state_grid<0, false>(p), kBceStateBlock, 0,
                                                    st>>>(
            p, S, home_pos, pid, mloc, bodies, frames, L, act, n_act, tau, n_fluid_total, mforce, bs);
    } else if (accel == 1) {
        k_bce<1, false, kWrenchLanes><<<wrench_blocks(body_markers), kBlock, 0, st>>>(
            p, S, home_pos, pid, mloc, bodies, frames, L, act, n_act, tau, n_fluid_total, mforce, bs);
        k_body_reduce<<<(unsigned)std::max(p.n_bodies, 1), 32, 0, st>>>(p, bs, n_act);
    } else {
        k_bce<2, false, kBceLanes, kBceStateBlock><<<bce_state_grid<2, false>(p), kBceStateBlock, 0,
                                                    st>>>(
            p, S, home_pos, pid, mloc, bodies, frames, L, act, n_act, tau, n_fluid_total, mforce, bs);
    }
}

void launch_batch_bce(int kind, const MemberDev *mem, const int *mlist, const int *off, int n,
                      int total, unsigned *queue, cudaStream_t st)
{
    if (total < 1) return;
    int dev = 0, nsm = 148, per_sm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const void *f = kind == 0 ? (const void *)k_batch_bce<0>
                              : kind == 1 ? (const void *)k_batch_bce<1> : (const void *)k_batch_bce<2>;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, f, kBlock, 0) != cudaSuccess
        || per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    const unsigned g = (unsigned)std::min<int64_t>((int64_t)nsm * per_sm,
                                                   (total + kBatchChunk - 1) / kBatchChunk);
    if (kind == 0) k_batch_bce<0><<<g, kBlock, 0, st>>>(mem, mlist, off, n, queue);
    else if (kind == 1) k_batch_bce<1><<<g, kBlock, 0, st>>>(mem, mlist, off, n, queue);
    else k_batch_bce<2><<<g, kBlock, 0, st>>>(mem, mlist, off, n, queue);
}

void launch_batch_reduce(const MemberDev *mem, const int *pairs, int npairs, cudaStream_t st)
{
    if (npairs > 0) k_batch_reduce<<<(unsigned)npairs, 32, 0, st>>>(mem, pairs);
}

unsigned bce_blocks(const DevParams &p) { return grid_for((int64_t)p.capM * kBceLanes); }

unsigned wrench_blocks(int64_t body_markers) { return grid_for(body_markers * kWrenchLanes); }

unsigned compact_blocks(const DevParams &p) { return grid_for(p.capM, kCompactBlock); }

void launch_compact_markers(const DevParams &p, const uint32_t *nnb, const uint32_t *pid,
                            uint32_t *nnb_exact, uint32_t *bcount, uint32_t *act,
                            uint32_t *act_body, int *n_act, cudaStream_t st)
{
    const unsigned g = compact_blocks(p);
    k_marker_counts<<<g, kCompactBlock, 0, st>>>(p, nnb, pid, bcount);
    k_marker_compact<<<g, kCompactBlock, 0, st>>>(p, nnb, pid, bcount, act, act_body, n_act,
                                                  nnb_exact);
}

}  // namespace crm
