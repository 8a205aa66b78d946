// crm_active.cu -- active domains (Sec. 3.2, Alg. 3): activity flags against
// oriented boxes attached to bodies, counts of Active / Extended-Active
// particles, and the compaction of those particles into the working set that
// the rest of the step processes.
//
// Layout.  Every SPH particle lives in a master store sorted once, at commit,
// by global cell with x slowest; colStart[x] is the first master slot of
// x-column x.  Particles are never re-sorted in the master: an Active particle
// is gathered into the working set, advanced there, and written back to its
// master slot, so its cell can drift away from the column it is filed under.
// The largest such drift (in columns) is tracked with atomicMax at write-back,
// so a box covering columns [xa, xb] finds every particle it can contain in
// the master slots of columns [xa - drift, xb + drift] -- one contiguous
// range.  Fixed wall markers get the same column index (they never move).
// The scan over a step is therefore proportional to the boxes' slabs, not to
// the terrain.
#include <algorithm>

#include "crm_internal.cuh"

namespace crm {

// Oriented box of one step: centre, rotation (body frame -> world), half
// extents, and the same grown by 2h.
struct BoxFrame {
    double c[3];
    double R[9];
    double e[3];
    double eg[3];   // grown by 2h
    double em[3];   // grown by 2h and the working-set margin (act_margin)
};

// Frame of box b at the bodies' current poses (FP64).
__device__ __forceinline__ void box_frame(const DevParams &p, int b, const int *box_body,
                                          const double *box_half, const double *box_off,
                                          const BodyDev *bodies, BoxFrame &F)
{
    const double grow = 2.0 * (double)p.h;
    const BodyDev &B = bodies[box_body[b]];
    const double *q = B.pose + 3;
    const double w = q[0], x = q[1], y = q[2], z = q[3];
    const double R[9] = {1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y),
                         2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x),
                         2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)};
    for (int k = 0; k < 9; ++k) F.R[k] = R[k];
    for (int k = 0; k < 3; ++k) {
        F.c[k] = B.pose[k] + R[3 * k] * box_off[3 * b] + R[3 * k + 1] * box_off[3 * b + 1]
                 + R[3 * k + 2] * box_off[3 * b + 2];
        F.e[k] = box_half[3 * b + k];
        F.eg[k] = box_half[3 * b + k] + grow;
        F.em[k] = F.eg[k] + p.act_margin;
    }
}

// ---------------------------------------------------------------------------
// k_box_prep: one block.  Box frames at the start of the step, the working
// window (union of the grown boxes' cell ranges, plus one cell), and the
// candidate master ranges: for fluid and for fixed markers, the union of the
// column ranges [xa - drift, xb + drift] of every box.  `all_active` (t <=
// t_delay, Alg. 3) takes the whole master and the whole grid instead.
//   ranges[2 * r], ranges[2 * r + 1]: master slot range r (fluid ranges first)
//   rinfo[0] = number of fluid ranges, [1] = number of marker ranges,
//   rinfo[2] = fluid candidates, [3] = all candidates, rinfo[4 + r] = prefix
//   offset of range r in the flattened candidate index.
__global__ void k_box_prep(DevParams p, int nbox, const int *__restrict__ box_body,
                           const double *__restrict__ box_half, const double *__restrict__ box_off,
                           const BodyDev *__restrict__ bodies, const int *__restrict__ colF,
                           const int *__restrict__ colM, const int *__restrict__ drift,
                           int all_active, int n_fluid_master, int n_fixed_master,
                           int64_t cand_cap, BoxFrame *__restrict__ frames, int *__restrict__ win,
                           int *__restrict__ ranges, int *__restrict__ rinfo,
                           int *__restrict__ counts, int *__restrict__ abort_flag,
                           int64_t step_tag)
{
    if (*abort_flag || gated_off(p)) return;
    const int G[3] = {p.GX, p.GY, p.GZ};
    const double dmin[3] = {p.dmin_x, p.dmin_y, p.dmin_z};
    const double inv_cell = 1.0 / p.cell_d;
    // the boxes' frames and cell ranges, one thread per box (FP64 work is slow:
    // keep it parallel); the window below pads every range by one cell
    __shared__ int s_lo[kMaxBodies][3], s_hi[kMaxBodies][3];
    if ((int)threadIdx.x < nbox) {
        const int b = threadIdx.x;
        BoxFrame &F = frames[b];
        box_frame(p, b, box_body, box_half, box_off, bodies, F);
        const double *R = F.R;
        for (int k = 0; k < 3; ++k) {
            const double ext = fabs(R[3 * k]) * F.em[0] + fabs(R[3 * k + 1]) * F.em[1]
                               + fabs(R[3 * k + 2]) * F.em[2];
            s_lo[b][k] = max((int)floor((F.c[k] - ext - dmin[k]) * inv_cell) - 1, 0);
            s_hi[b][k] = min((int)floor((F.c[k] + ext - dmin[k]) * inv_cell) + 1, G[k] - 1);
        }
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    if (p.step_ctr != nullptr) step_tag = (int64_t)*p.step_ctr;
    if (!p.act_skin) {   // (with the skin the step's flag pass counts, after k_decide's reset)
        counts[3] = 0;
        counts[4] = 0;
    }
    int lo[3] = {G[0], G[1], G[2]}, hi[3] = {-1, -1, -1};
    int xa[kMaxBodies], xb[kMaxBodies];
    for (int b = 0; b < nbox; ++b) {
        for (int k = 0; k < 3; ++k) {
            lo[k] = min(lo[k], s_lo[b][k]);
            hi[k] = max(hi[k], s_hi[b][k]);
        }
        xa[b] = s_lo[b][0];
        xb[b] = s_hi[b][0];
    }
    if (all_active || nbox == 0) {
        for (int k = 0; k < 3; ++k) { lo[k] = 0; hi[k] = G[k] - 1; }
    }
    const int64_t cells = key_cells(max(hi[0] - lo[0] + 1, 1), max(hi[1] - lo[1] + 1, 1),
                                    max(hi[2] - lo[2] + 1, 1));
    if (hi[0] < lo[0] || hi[1] < lo[1] || hi[2] < lo[2]) {   // boxes outside the grid
        for (int k = 0; k < 3; ++k) { lo[k] = 0; hi[k] = 0; }
    }
    counts[9] = (int)min(cells, (int64_t)0x7fffffff);   // window in use (shrink policy)
    if (cells > (int64_t)p.M) {
        counts[7] = (int)min(cells, (int64_t)0x7fffffff);
        atomicCAS(abort_flag, 0, (int)(step_tag + 1));
        return;
    }
    for (int k = 0; k < 3; ++k) {
        win[k] = lo[k];
        win[3 + k] = max(hi[k] - lo[k] + 1, 1);
    }
    // candidate master ranges (merged; fluid first, then fixed markers)
    const int d = *drift;
    int nr = 0;
    int64_t total = 0;
    int nrange[2] = {0, 0};
    rinfo[2] = 0;
    for (int kind = 0; kind < 2; ++kind) {
        const int *col = kind == 0 ? colF : colM;
        const int nmaster = kind == 0 ? n_fluid_master : n_fixed_master;
        if (nmaster == 0) continue;
        int a0[kMaxBodies], b0[kMaxBodies], m = 0;
        if (all_active) {
            a0[0] = 0; b0[0] = G[0] - 1; m = 1;
        } else {
            for (int b = 0; b < nbox; ++b) {
                a0[m] = max(xa[b] - d, 0);
                b0[m] = min(xb[b] + d, G[0] - 1);
                ++m;
            }
        }
        // insertion sort by start, then merge overlapping / touching column ranges
        for (int i = 1; i < m; ++i)
            for (int j = i; j > 0 && a0[j] < a0[j - 1]; --j) {
                int t = a0[j]; a0[j] = a0[j - 1]; a0[j - 1] = t;
                t = b0[j]; b0[j] = b0[j - 1]; b0[j - 1] = t;
            }
        int i = 0;
        while (i < m) {
            int ca = a0[i], cb = b0[i];
            int j = i + 1;
            while (j < m && a0[j] <= cb + 1) { cb = max(cb, b0[j]); ++j; }
            const int s0 = col[ca], s1 = col[cb + 1];
            if (s1 > s0) {
                ranges[2 * nr] = s0;
                ranges[2 * nr + 1] = s1;
                rinfo[4 + nr] = (int)total;
                total += s1 - s0;
                ++nr;
                ++nrange[kind];
            }
            i = j;
        }
        if (kind == 0) rinfo[2] = (int)total;
    }
    rinfo[0] = nrange[0];
    rinfo[1] = nrange[1];
    rinfo[3] = (int)min(total, (int64_t)0x7fffffff);
    rinfo[4 + nr] = (int)total;
    counts[10] = (int)min(total, (int64_t)0x7fffffff);   // candidates in use (shrink policy)
    if (total > cand_cap) {
        counts[8] = (int)min(total, (int64_t)0x7fffffff);
        atomicCAS(abort_flag, 0, (int)(step_tag + 1));
    }
}

// Position of a master fluid particle in FP64 (cell corner + offset).
__device__ __forceinline__ void abs_pos(const DevParams &p, float4 ps, double x[3])
{
    int ix, iy, iz;
    decode_cell(__float_as_uint(ps.w), p, ix, iy, iz);
    x[0] = p.dmin_x + ix * p.cell_d + (double)ps.x;
    x[1] = p.dmin_y + iy * p.cell_d + (double)ps.y;
    x[2] = p.dmin_z + iz * p.cell_d + (double)ps.z;
}

// Activity of a point against the step's boxes: 2 inside a box (Active), 1
// inside a box grown by 2h (Extended-Active), else 0 -- the box-frame test of
// UpdateActivity, in FP64.
// With a working-set margin, 3: inside a box grown by 2h and the margin only.
__device__ __forceinline__ int activity(const double x[3], int nbox, const BoxFrame *F)
{
    int best = 0;
    for (int b = 0; b < nbox; ++b) {
        const double d[3] = {x[0] - F[b].c[0], x[1] - F[b].c[1], x[2] - F[b].c[2]};
        int in = 1, ext = 1, mar = 1;
        for (int k = 0; k < 3; ++k) {
            const double l = F[b].R[k] * d[0] + F[b].R[3 + k] * d[1] + F[b].R[6 + k] * d[2];
            if (fabs(l) > F[b].e[k]) in = 0;
            if (fabs(l) > F[b].eg[k]) ext = 0;
            if (fabs(l) > F[b].em[k]) mar = 0;
        }
        if (in) return 2;
        if (ext) best = 1;
        else if (mar && best == 0) best = 3;
    }
    return best;
}

__device__ __forceinline__ int range_of(const int *rinfo, int nr, int c)
{
    int lo = 0, hi = nr - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (rinfo[4 + mid] <= c) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// UpdateActivity (Alg. 3): flag every candidate; include[c] = 1 for Active and
// Extended-Active fluid and for fixed markers within a grown box.  Counts of
// Active and Extended fluid go to counts[3], counts[4] (integer atomics).
__global__ void k_activity(DevParams p, int nbox, const BoxFrame *__restrict__ frames,
                           const int *__restrict__ ranges, const int *__restrict__ rinfo,
                           const float4 *__restrict__ mpos, const double *__restrict__ mloc,
                           const int *__restrict__ fixed_order, int all_active, int64_t cand_cap,
                           uint32_t *__restrict__ include, uint8_t *__restrict__ kind,
                           int *__restrict__ counts, const int *__restrict__ abort_flag)
{
    if (*abort_flag || gated_off(p)) return;
    __shared__ BoxFrame F[kMaxBodies];
    for (int b = threadIdx.x; b < nbox; b += blockDim.x) F[b] = frames[b];
    __syncthreads();
    const int nr = rinfo[0] + rinfo[1];
    const int nfc = rinfo[2], total = rinfo[3];
    int na = 0, ne = 0;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < cand_cap;
         c += (int64_t)gridDim.x * blockDim.x) {
        uint32_t inc = 0;
        uint8_t k = 0;
        if (c < total) {
            const int r = range_of(rinfo, nr, (int)c);
            const int m = ranges[2 * r] + ((int)c - rinfo[4 + r]);
            double x[3];
            if (c < nfc) {
                abs_pos(p, mpos[m], x);
            } else {
                const int a = fixed_order[m];
                x[0] = mloc[3 * (int64_t)a]; x[1] = mloc[3 * (int64_t)a + 1]; x[2] = mloc[3 * (int64_t)a + 2];
            }
            const int f = all_active ? 2 : activity(x, nbox, F);
            inc = f > 0 ? 1u : 0u;
            k = (uint8_t)f;
            if (c < nfc && !p.act_skin) {
                na += f == 2;
                ne += f == 1;
            }
        }
        include[c] = inc;
        kind[c] = k;
    }
    for (int o = 16; o > 0; o >>= 1) {
        na += __shfl_down_sync(0xffffffffu, na, o);
        ne += __shfl_down_sync(0xffffffffu, ne, o);
    }
    if ((threadIdx.x & 31) == 0 && (na | ne)) {
        atomicAdd(&counts[3], na);
        atomicAdd(&counts[4], ne);
    }
}

// ComputeActiveCount / ManageArrayMemory, device half: sizes of the working
// set from the exclusive scan of the include flags; overflow of a capacity
// aborts the step (every later kernel of the step sees the flag and returns).
__global__ void k_active_sizes(DevParams p, const int *__restrict__ rinfo,
                               const uint32_t *__restrict__ slot, int n_body_markers,
                               int *__restrict__ counts, int *__restrict__ abort_flag,
                               int64_t step_tag)
{
    if (threadIdx.x != 0 || *abort_flag || gated_off(p)) return;
    if (p.step_ctr != nullptr) step_tag = (int64_t)*p.step_ctr;
    const int nfc = rinfo[2], total = rinfo[3];
    const int nF = (int)slot[nfc];
    const int nfix = (int)slot[total] - nF;
    const int nM = nfix + n_body_markers;
    counts[5] = nF;
    counts[6] = nM;
    if (nF > p.capF || nM > p.capM) {
        atomicCAS(abort_flag, 0, (int)(step_tag + 1));
        return;
    }
    counts[0] = nF;
    counts[1] = nM;
    counts[2] = nF + nM;
}

// Gather the included candidates (and every body marker) into the unsorted
// working arrays; Extended-Active fluid carries kExtendedBit in its pid.
__global__ void k_gather(DevParams p, const int *__restrict__ ranges, const int *__restrict__ rinfo,
                         const uint8_t *__restrict__ kind,
                         const uint32_t *__restrict__ slot, StageArrays M,
                         const uint32_t *__restrict__ mpid, const int *__restrict__ fixed_order,
                         const int *__restrict__ body_markers, int n_body_markers,
                         int n_fluid_total, int64_t cand_cap, StageArrays W,
                         uint32_t *__restrict__ wpid, const int *__restrict__ counts,
                         const int *__restrict__ abort_flag)
{
    if (*abort_flag || gated_off(p)) return;
    const int nr = rinfo[0] + rinfo[1];
    const int nfc = rinfo[2], total = rinfo[3];
    const int nF = counts[0];
    const int64_t span = (int64_t)max(total, 0) + n_body_markers;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < span;
         c += (int64_t)gridDim.x * blockDim.x) {
        if (c < total) {
            if (kind[c] == 0) continue;   // (the scan has consumed `include`)
            const int r = range_of(rinfo, nr, (int)c);
            const int m = ranges[2 * r] + ((int)c - rinfo[4 + r]);
            const uint32_t w = slot[c];
            if (c < nfc) {
                W.pos[w] = M.pos[m];
                W.vel[w] = M.vel[m];
                W.sA[w] = M.sA[m];
                W.sB[w] = M.sB[m];
                const uint8_t kd = kind[c];
                wpid[w] = mpid[m] | (kd == 2 ? 0u
                                             : kd == 1 ? kExtendedBit : kExtendedBit | kOutsideBit);
            } else {
                W.pos[w] = make_float4(0.f, 0.f, 0.f, 0.f);
                W.vel[w] = make_float4(0.f, 0.f, 0.f, p.rho0);
                W.sA[w] = make_float4(0.f, 0.f, 0.f, 0.f);
                W.sB[w] = make_float2(0.f, 0.f);
                wpid[w] = (uint32_t)(n_fluid_total + fixed_order[m]);
            }
        } else {
            const int k = (int)(c - total);
            const uint32_t w = (uint32_t)((int64_t)slot[total] + k);
            W.pos[w] = make_float4(0.f, 0.f, 0.f, 0.f);
            W.vel[w] = make_float4(0.f, 0.f, 0.f, p.rho0);
            W.sA[w] = make_float4(0.f, 0.f, 0.f, 0.f);
            W.sB[w] = make_float2(0.f, 0.f);
            wpid[w] = (uint32_t)body_markers[k];   // marker id
        }
    }
    (void)cand_cap;
    (void)nF;
}

// Write the Active particles of the (sorted) working set back to their master
// slots and track how far, in x-columns, any of them has drifted from the
// column its master slot is filed under.
// (With the skin the working set persists across steps: the particles written
// back are those integrated at some step since it was gathered.)  gated: part
// of a step's gated rebuild (skipped unless the cell search is due).
__global__ void k_scatter_back(DevParams p, StageArrays W, const uint32_t *__restrict__ wpid,
                               const uint32_t *__restrict__ mslot_of_pid,
                               const int *__restrict__ mcol, StageArrays M, int *__restrict__ drift,
                               int gated)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    int dmax = 0;
    if (*p.abort || (gated && gated_off(p))) return;
    if (s < __ldg(p.sizes)) {
        const uint32_t id = wpid[s];
        if (p.act_skin ? (id & kTouchedBit) != 0u : !(id & kExtendedBit)) {
            const uint32_t m = mslot_of_pid[pid_index(id)];
            const float4 ps = W.pos[s];
            M.pos[m] = ps;
            M.vel[m] = W.vel[s];
            M.sA[m] = W.sA[s];
            M.sB[m] = W.sB[s];
            int ix, iy, iz;
            decode_cell(__float_as_uint(ps.w), p, ix, iy, iz);
            // an offset may have left its home cell since the last re-homing
            ix += (int)floorf(ps.x / p.cell);
            dmax = abs(ix - mcol[m]);
        }
    }
    for (int o = 16; o > 0; o >>= 1) dmax = max(dmax, __shfl_down_sync(0xffffffffu, dmax, o));
    if ((threadIdx.x & 31) == 0 && dmax > 0) atomicMax(drift, dmax);
}

// Master store -> insertion order (absolute FP64 positions).
__global__ void k_export_master(DevParams p, StageArrays M, const uint32_t *__restrict__ mpid,
                                int n, double *__restrict__ xyz, float *__restrict__ vel,
                                float *__restrict__ sig, float *__restrict__ rho)
{
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= n) return;
    const uint32_t id = mpid[m];
    double x[3];
    abs_pos(p, M.pos[m], x);
    for (int k = 0; k < 3; ++k) xyz[3 * (size_t)id + k] = x[k];
    const float4 v = M.vel[m];
    vel[3 * (size_t)id] = v.x; vel[3 * (size_t)id + 1] = v.y; vel[3 * (size_t)id + 2] = v.z;
    rho[id] = v.w;
    const float4 a = M.sA[m];
    const float2 b = M.sB[m];
    float *o = sig + 6 * (size_t)id;
    o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w; o[4] = b.x; o[5] = b.y;
}

// ---------------------------------------------------------------------------
void launch_box_prep(const DevParams &p, int nbox, const int *box_body, const double *box_half,
                     const double *box_off, const BodyDev *bodies, const int *colF,
                     const int *colM, const int *drift, int all_active, int n_fluid_master,
                     int n_fixed_master, int64_t cand_cap, void *frames, int *win, int *ranges,
                     int *rinfo, int *counts, int *abort_flag, int64_t step_tag, cudaStream_t st)
{
    k_box_prep<<<1, 32, 0, st>>>(p, nbox, box_body, box_half, box_off, bodies, colF, colM, drift,
                                 all_active, n_fluid_master, n_fixed_master, cand_cap,
                                 (BoxFrame *)frames, win, ranges, rinfo, counts, abort_flag,
                                 step_tag);
}

void launch_activity(const DevParams &p, int nbox, const void *frames, const int *ranges,
                     const int *rinfo, const float4 *mpos, const double *mloc,
                     const int *fixed_order, int all_active, int64_t cand_cap, uint32_t *include,
                     uint8_t *kind, int *counts, const int *abort_flag, cudaStream_t st)
{
    const unsigned g = (unsigned)std::min<int64_t>(grid_for(cand_cap), (int64_t)p.n_sm * 16);
    k_activity<<<g, kBlock, 0, st>>>(p, nbox, (const BoxFrame *)frames, ranges, rinfo, mpos, mloc,
                                     fixed_order, all_active, cand_cap, include, kind, counts,
                                     abort_flag);
}

void launch_active_sizes(const DevParams &p, const int *rinfo, const uint32_t *slot,
                         int n_body_markers, int *counts, int *abort_flag, int64_t step_tag,
                         cudaStream_t st)
{
    k_active_sizes<<<1, 32, 0, st>>>(p, rinfo, slot, n_body_markers, counts, abort_flag, step_tag);
}

void launch_gather(const DevParams &p, const int *ranges, const int *rinfo,
                   const uint8_t *kind, const uint32_t *slot,
                   StageArrays M, const uint32_t *mpid, const int *fixed_order,
                   const int *body_markers, int n_body_markers, int n_fluid_total,
                   int64_t cand_cap, StageArrays W, uint32_t *wpid, const int *counts,
                   const int *abort_flag, cudaStream_t st)
{
    const unsigned g = (unsigned)std::min<int64_t>(grid_for(cand_cap + n_body_markers), (int64_t)p.n_sm * 16);
    k_gather<<<g, kBlock, 0, st>>>(p, ranges, rinfo, kind, slot, M, mpid, fixed_order,
                                   body_markers, n_body_markers, n_fluid_total, cand_cap, W, wpid,
                                   counts, abort_flag);
}

void launch_scatter_back(const DevParams &p, StageArrays W, const uint32_t *wpid,
                         const uint32_t *mslot_of_pid, const int *mcol, StageArrays M, int *drift,
                         int gated, cudaStream_t st)
{
    k_scatter_back<<<grid_for(p.capF), kBlock, 0, st>>>(p, W, wpid, mslot_of_pid, mcol, M, drift,
                                                        gated);
}

// The activity of every working-set fluid particle against this step's boxes
// (Alg. 3 UpdateActivity at every step, on the persisting working set): the
// pid bits and the Active / Extended counts.  Each block computes the frames
// of the step's boxes (FP64) for itself.
__global__ void __launch_bounds__(kBlock)
k_flags(DevParams p, int nbox, const int *__restrict__ box_body,
        const double *__restrict__ box_half, const double *__restrict__ box_off,
        const BodyDev *__restrict__ bodies, int all_active, uint32_t *__restrict__ pid,
        const float4 *__restrict__ pos, int *__restrict__ counts)
{
    __shared__ BoxFrame F[kMaxBodies];
    if (*p.abort) return;
    if ((int)threadIdx.x < nbox) box_frame(p, threadIdx.x, box_body, box_half, box_off, bodies,
                                           F[threadIdx.x]);
    __syncthreads();
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    int na = 0, ne = 0;
    if (s < __ldg(p.sizes)) {
        double x[3];
        abs_pos(p, pos[s], x);
        const int f = all_active ? 2 : activity(x, nbox, F);
        const uint32_t id = pid[s];
        uint32_t out = id & (kPidIndexMask | kTouchedBit);
        if (f == 2) out |= kTouchedBit;
        else if (f == 1) out |= kExtendedBit;
        else out |= kExtendedBit | kOutsideBit;
        if (out != id) pid[s] = out;
        na = f == 2;
        ne = f == 1;
    }
    for (int o = 16; o > 0; o >>= 1) {
        na += __shfl_down_sync(0xffffffffu, na, o);
        ne += __shfl_down_sync(0xffffffffu, ne, o);
    }
    if ((threadIdx.x & 31) == 0 && (na | ne)) {
        atomicAdd(&counts[3], na);
        atomicAdd(&counts[4], ne);
    }
}

void launch_flags(const DevParams &p, int nbox, const int *box_body, const double *box_half,
                  const double *box_off, const BodyDev *bodies, int all_active, uint32_t *pid,
                  const float4 *pos, int *counts, cudaStream_t st)
{
    k_flags<<<grid_for(p.capF), kBlock, 0, st>>>(p, nbox, box_body, box_half, box_off, bodies,
                                                 all_active, pid, pos, counts);
}

void launch_export_master(const DevParams &p, StageArrays M, const uint32_t *mpid, int n,
                          double *xyz, float *vel, float *sig, float *rho, cudaStream_t st)
{
    k_export_master<<<grid_for(n), kBlock, 0, st>>>(p, M, mpid, n, xyz, vel, sig, rho);
}

size_t box_frame_bytes() { return sizeof(BoxFrame); }

// ---------------------------------------------------------------------------
// FP64 diagnostics of the SPH particles: the state is FP32, its global sums are
// FP64 (count, mass, volume sum m / rho, linear momentum sum m u, angular
// momentum about the world origin sum m x (x) u with absolute FP64 positions,
// kinetic energy sum m |u|^2 / 2).  Deterministic: a fixed grid walking the
// slots with a fixed stride, a fixed tree inside each block, then one warp
// summing the block partials in block order.
constexpr int kDiagBlocks = 296;

__global__ void __launch_bounds__(kBlock)
k_diag_partial(DevParams p, StageArrays S, const int *__restrict__ n_dev, int n_host, double m,
               double *__restrict__ partial)
{
    const int n = n_dev != nullptr ? __ldg(n_dev) : n_host;
    double v[CRM_NUM_DIAG];
#pragma unroll
    for (int k = 0; k < CRM_NUM_DIAG; ++k) v[k] = 0.0;
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
        double x[3];
        abs_pos(p, S.pos[s], x);
        const float4 u4 = S.vel[s];
        const double ux = u4.x, uy = u4.y, uz = u4.z;
        v[0] += 1.0;
        v[1] += m;
        v[2] += m / (double)u4.w;
        v[3] += m * ux;
        v[4] += m * uy;
        v[5] += m * uz;
        v[6] += m * (x[1] * uz - x[2] * uy);
        v[7] += m * (x[2] * ux - x[0] * uz);
        v[8] += m * (x[0] * uy - x[1] * ux);
        v[9] += 0.5 * m * (ux * ux + uy * uy + uz * uz);
    }
    __shared__ double red[kBlock / 32][CRM_NUM_DIAG];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < CRM_NUM_DIAG; ++k) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
        if (lane == 0) red[warp][k] = v[k];
    }
    __syncthreads();
    if (threadIdx.x < CRM_NUM_DIAG) {
        double a = 0.0;
        for (int w = 0; w < kBlock / 32; ++w) a += red[w][threadIdx.x];
        partial[(size_t)blockIdx.x * CRM_NUM_DIAG + threadIdx.x] = a;
    }
}

__global__ void k_diag_final(const double *__restrict__ partial, double *__restrict__ out)
{
    if (threadIdx.x >= CRM_NUM_DIAG) return;
    double a = 0.0;
    for (int b = 0; b < kDiagBlocks; ++b) a += partial[(size_t)b * CRM_NUM_DIAG + threadIdx.x];
    out[threadIdx.x] = a;
}

size_t diag_scratch_doubles() { return (size_t)(kDiagBlocks + 1) * CRM_NUM_DIAG; }

void launch_diagnostics(const DevParams &p, StageArrays S, const int *n_dev, int n_host, double m,
                        double *scratch, cudaStream_t st)
{
    k_diag_partial<<<kDiagBlocks, kBlock, 0, st>>>(p, S, n_dev, n_host, m, scratch);
    k_diag_final<<<1, 32, 0, st>>>(scratch, scratch + (size_t)kDiagBlocks * CRM_NUM_DIAG);
}

}  // namespace crm
