// crm_bin.cu -- cell binning and neighbour lists (Sec. 3.1, Alg. 1).
//
// Binning is a counting sort over cells rather than a comparison or radix
// sort: the keys are cell ids, so one pass of per-key arrival ranks (atomic),
// one exclusive scan and one scatter sort the particles, and the scan of the
// per-cell counts IS the cellStart array (cellEnd[c] = cellStart[c + 1]).
// The atomic ranks make the arrival order within a cell nondeterministic; a
// fix-up pass re-ranks every element by its input index inside its cell, so
// the result equals a stable sort by (cell, input index) on every run.
#include <algorithm>
#include <cstdio>
#include <mutex>

#include "crm_internal.cuh"

namespace crm {

// ---------------------------------------------------------------------------
// Exclusive scan, single pass with decoupled look-back.  Tile status words:
// high half = (epoch << 2) | state, low half = value; state 1 = tile
// aggregate, 2 = inclusive prefix.  Tiles are numbered in launch order by a
// ticket, so every tile waits only on tiles that are already running; each
// wait is bounded and sets ERR_TIMEOUT instead of spinning forever.  The last
// tile to finish resets the ticket and advances the epoch, so the status
// words never need clearing (a zeroed word has state 0 and is never valid).
namespace {
constexpr uint32_t kAgg = 1u, kIncl = 2u;
constexpr int kSpinLimit = 1 << 22;
constexpr int kFaultSpinLimit = 1000;

// Test switch of the device-wait failure path (crm_debug_wait_fault): when
// set, the first tile of every look-back scan publishes nothing and every wait
// gives up after kFaultSpinLimit polls, so the waits of the later tiles run out
// (they return with ERR_TIMEOUT; nothing hangs and nothing faults).
__device__ int g_wait_fault = 0;

__device__ __forceinline__ int pad(int k) { return k + (k >> 5); }

__global__ void __launch_bounds__(kScanThreads)
k_scan(uint32_t *__restrict__ count, uint32_t *__restrict__ start, int64_t n,
       unsigned long long *status, uint32_t *ctr, int64_t n_tiles, int *err,
       const int *__restrict__ gate, int *abort_word)
{
    if (gate != nullptr && __ldg(gate) == 0) return;   // every block: uniform
    __shared__ uint32_t s_items[kScanTile + kScanTile / 32];
    __shared__ uint32_t s_warp[kScanThreads / 32];
    __shared__ uint32_t s_tile, s_epoch, s_prefix;
    __shared__ int s_fault;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    if (t == 0) {
        s_tile = atomicAdd(&ctr[0], 1u);
        s_epoch = (((volatile uint32_t *)ctr)[1] + 1u) & 0x3FFFFFFFu;
        s_fault = *(volatile int *)&g_wait_fault;
    }
    __syncthreads();
    const int64_t tile = s_tile;
    const uint32_t epoch = s_epoch;
    const int64_t base = tile * kScanTile;
    for (int k = t; k < kScanTile; k += kScanThreads) {
        const int64_t g = base + k;
        s_items[pad(k)] = g < n ? count[g] : 0u;
    }
    __syncthreads();
    uint32_t v[kScanItems];
    uint32_t sum = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        v[i] = s_items[pad(t * kScanItems + i)];
        sum += v[i];
    }
    uint32_t incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < kScanThreads / 32 ? s_warp[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < kScanThreads / 32) s_warp[lane] = w;
    }
    __syncthreads();
    const uint32_t excl = incl - sum + (warp > 0 ? s_warp[warp - 1] : 0u);
    const uint32_t agg = s_warp[kScanThreads / 32 - 1];
    if (t == 0) {
        uint32_t prefix = 0;
        if (tile > 0) {
            atomicExch(&status[tile],
                       ((unsigned long long)((epoch << 2) | kAgg) << 32) | agg);
            int64_t j = tile - 1;
            int spins = 0;
            while (true) {
                const unsigned long long w = ((volatile unsigned long long *)status)[j];
                const uint32_t hi = (uint32_t)(w >> 32);
                const uint32_t st = hi & 3u;
                if (st != 0u && (hi >> 2) == epoch) {
                    prefix += (uint32_t)w;
                    if (st == kIncl) break;
                    --j;
                    spins = 0;
                } else if (++spins > (s_fault ? kFaultSpinLimit : kSpinLimit)) {
                    atomicOr(err, ERR_TIMEOUT);
                    // every later kernel of the terrain's enqueued work returns at
                    // once: none of them indexes with these partial cell ranges
                    if (abort_word != nullptr) atomicExch(abort_word, kAbortTimeout);
                    break;
                } else {
                    __nanosleep(32);
                }
            }
        }
        if (!(s_fault && tile == 0))
            atomicExch(&status[tile],
                       ((unsigned long long)((epoch << 2) | kIncl) << 32) | (prefix + agg));
        s_prefix = prefix;
    }
    __syncthreads();
    uint32_t run = s_prefix + excl;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        s_items[pad(t * kScanItems + i)] = run;
        run += v[i];
    }
    __syncthreads();
    for (int k = t; k < kScanTile; k += kScanThreads) {
        const int64_t g = base + k;
        if (g < n) {
            start[g] = s_items[pad(k)];
            count[g] = 0u;
        }
    }
    if (t == 0) {
        __threadfence();
        if (atomicAdd(&ctr[2], 1u) == (uint32_t)(n_tiles - 1)) {
            ctr[0] = 0u;
            ctr[2] = 0u;
            __threadfence();
            atomicAdd(&ctr[1], 1u);
        }
    }
}
}  // namespace

void launch_scan_reset(uint32_t *count, uint32_t *start, int64_t n, const SortScratch &s,
                       int *err, cudaStream_t st, const int *gate, int *abort_word)
{
    const int64_t tiles = (n + kScanTile - 1) / kScanTile;
    k_scan<<<(unsigned)tiles, kScanThreads, 0, st>>>(count, start, n, s.tile_status, s.ctr,
                                                     tiles, err, gate, abort_word);
}

int set_wait_fault(int on)
{
    const int v = on ? 1 : 0;
    return cudaMemcpyToSymbol(g_wait_fault, &v, sizeof(int)) == cudaSuccess ? 0 : -1;
}

// ---------------------------------------------------------------------------
// Counting-sort passes shared by the terrain and the stateless entry point.
namespace {

// slot of element i in the cell-sorted order before the stable fix-up
__global__ void k_scatter(const uint32_t *__restrict__ keys, const uint32_t *__restrict__ rank,
                          const uint32_t *__restrict__ start, uint32_t *__restrict__ tmp,
                          int64_t n, const int *__restrict__ n_dev,
                          const int *__restrict__ abort_flag, const int *__restrict__ gate = nullptr)
{
    if ((abort_flag && *abort_flag) || (gate != nullptr && __ldg(gate) == 0)) return;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (n_dev ? (int64_t)__ldg(n_dev) : n)) return;
    tmp[start[keys[i]] + rank[i]] = (uint32_t)i;
}

// H3 of the stateless call: cell of each point (clamped into the grid), and the
// count of each cell.
__global__ void k_hash_points(const float *__restrict__ xyz, int64_t n, float inv_cell, int X,
                              int Y, int Z, uint32_t *__restrict__ cell,
                              uint32_t *__restrict__ count)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float x = xyz[3 * i], y = xyz[3 * i + 1], z = xyz[3 * i + 2];
    int ix = (int)floorf(x * inv_cell), iy = (int)floorf(y * inv_cell),
        iz = (int)floorf(z * inv_cell);
    ix = min(max(ix, 0), X - 1);
    iy = min(max(iy, 0), Y - 1);
    iz = min(max(iz, 0), Z - 1);
    const uint32_t c = ((uint32_t)iz * (uint32_t)Y + (uint32_t)iy) * (uint32_t)X + (uint32_t)ix;
    cell[i] = c;
    atomicAdd(&count[c], 1u);
}

// H4 of the stateless call: a stable least-significant-digit radix sort of
// (cell, input index) by cell, 8 bits per pass, O(n) work per pass whatever
// the distribution of points over cells (a cell holding all n points costs no
// more than n distinct cells).  A pass: each block counts the digits of its
// tile of kRadixTile elements (k_radix_hist, written digit-major: hist[d *
// tiles + b]); one exclusive scan of that array gives every (digit, tile) its
// output offset, so tiles keep their order within a digit; k_radix_scatter
// ranks each tile's elements by digit in input order (warp match, then the
// warps in order) and writes them there.  Every kernel does nothing once a
// wait of a scan has given up (*err & ERR_TIMEOUT).
constexpr int kRadixThreads = 256;
constexpr int kRadixItems = 8;
constexpr int kRadixTile = kRadixThreads * kRadixItems;
constexpr int kRadixWarps = kRadixThreads / 32;

__global__ void __launch_bounds__(kRadixThreads)
k_radix_hist(const uint32_t *__restrict__ keys, int64_t n, int shift, int64_t tiles,
             uint32_t *__restrict__ hist, const int *__restrict__ err)
{
    __shared__ uint32_t h[256];
    if (*(volatile const int *)err & ERR_TIMEOUT) return;   // uniform over the grid
    h[threadIdx.x] = 0u;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kRadixTile;
    for (int k = threadIdx.x; k < kRadixTile; k += kRadixThreads) {
        const int64_t i = base + k;
        if (i < n) atomicAdd(&h[(keys[i] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * tiles + blockIdx.x] = h[threadIdx.x];
}

// vals_in == nullptr: the values are the input indices.  keys_out == nullptr:
// the last pass (only the values are kept).
__global__ void __launch_bounds__(kRadixThreads)
k_radix_scatter(const uint32_t *__restrict__ keys_in, const uint32_t *__restrict__ vals_in,
                int64_t n, int shift, int64_t tiles, const uint32_t *__restrict__ offs,
                uint32_t *__restrict__ keys_out, uint32_t *__restrict__ vals_out,
                const int *__restrict__ err)
{
    __shared__ uint32_t run[256];                 // elements of each digit placed so far
    __shared__ uint32_t wcnt[kRadixWarps][256];   // this round: per warp, per digit
    if (*(volatile const int *)err & ERR_TIMEOUT) return;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    run[t] = offs[(int64_t)t * tiles + blockIdx.x];
    const int64_t base = (int64_t)blockIdx.x * kRadixTile;
    for (int r = 0; r < kRadixItems; ++r) {
        for (int w = 0; w < kRadixWarps; ++w) wcnt[w][t] = 0u;
        __syncthreads();
        const int64_t i = base + (int64_t)r * kRadixThreads + t;   // input order within the tile
        const bool ok = i < n;
        const uint32_t key = ok ? keys_in[i] : 0u;
        const uint32_t d = ok ? (key >> shift) & 255u : 256u + (uint32_t)lane;   // never matches
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const uint32_t below = (uint32_t)__popc(peers & ((1u << lane) - 1u));
        if (ok && below == 0u) wcnt[warp][d] = (uint32_t)__popc(peers);
        __syncthreads();
        // digit t: exclusive prefix over the warps, in warp order
        uint32_t acc = run[t];
        for (int w = 0; w < kRadixWarps; ++w) {
            const uint32_t c = wcnt[w][t];
            wcnt[w][t] = acc;
            acc += c;
        }
        __syncthreads();
        if (ok) {
            const uint32_t at = wcnt[warp][d] + below;
            vals_out[at] = vals_in ? vals_in[i] : (uint32_t)i;
            if (keys_out) keys_out[at] = key;
        }
        __syncthreads();
        run[t] = acc;
    }
}

// After the sort: when a wait gave up, cell_start[ncell] is set to a value no
// successful call leaves there (a successful call leaves n).
__global__ void k_bin_status(uint32_t *__restrict__ cell_start, int64_t ncell,
                             const int *__restrict__ err)
{
    if (*(volatile const int *)err & ERR_TIMEOUT) cell_start[ncell] = 0xFFFFFFFFu;
}
}  // namespace

// ---------------------------------------------------------------------------
// Terrain rebuild kernels.

// Key generation (Sec. 3.1 step 1, calcGridPos / calcGridID).  Fluid particles
// are re-homed into the cell their offset now lies in; markers get their
// kinematic position at the start of the step.  The key is the cell index
// inside the working window, offset by M for markers, so one counting sort
// yields fluid slots [0, nF) then marker slots [nF, N), each cell-sorted.
__global__ void k_keys(DevParams p, float4 *__restrict__ pos, const uint32_t *__restrict__ pid,
                       const double *__restrict__ mloc,
                       const BodyDev *__restrict__ bodies, uint32_t *__restrict__ keys,
                       uint32_t *__restrict__ rank, uint32_t *__restrict__ count,
                       int *__restrict__ err, int n_fluid_total)
{
    if (*p.abort || gated_off(p)) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const Sizes z = load_sizes(p);
    if (i >= z.N) return;
    const Window W = load_window(p);
    float4 ps = pos[i];
    int ix, iy, iz;
    uint32_t seg;
    bool bad = false;
    if (i < z.nF) {
        seg = 0;
        decode_cell(__float_as_uint(ps.w), p, ix, iy, iz);
        if (!(isfinite(ps.x) && isfinite(ps.y) && isfinite(ps.z))) {
            atomicOr(err, ERR_NONFINITE);
            ps.x = ps.y = ps.z = 0.0f;
        }
        const float inv = 1.0f / p.cell;
        const int fx = (int)floorf(ps.x * inv), fy = (int)floorf(ps.y * inv),
                  fz = (int)floorf(ps.z * inv);
        if (fx | fy | fz) {
            ix += fx; iy += fy; iz += fz;
            ps.x -= (float)fx * p.cell;
            ps.y -= (float)fy * p.cell;
            ps.z -= (float)fz * p.cell;
        }
    } else {
        seg = 1;
        const uint32_t id = pid[i];
        const int mi = (int)pid_index(id) - n_fluid_total;
        const int body = pid_body(p, id);
        const double *xl = mloc + 3 * (int64_t)mi;
        double x[3] = {xl[0], xl[1], xl[2]};   // fixed marker: its world position
        if (body >= 0) {
            float u[3], a[3], arm[3];
            marker_now(bodies[body], xl, x, u, a, arm);
        }
        const double fx = floor((x[0] - p.dmin_x) / p.cell_d);
        const double fy = floor((x[1] - p.dmin_y) / p.cell_d);
        const double fz = floor((x[2] - p.dmin_z) / p.cell_d);
        ix = (int)fmin(fmax(fx, -1.0), (double)p.GX);
        iy = (int)fmin(fmax(fy, -1.0), (double)p.GY);
        iz = (int)fmin(fmax(fz, -1.0), (double)p.GZ);
        ps.x = (float)(x[0] - (p.dmin_x + ix * p.cell_d));
        ps.y = (float)(x[1] - (p.dmin_y + iy * p.cell_d));
        ps.z = (float)(x[2] - (p.dmin_z + iz * p.cell_d));
    }
    int lx = ix - W.x0, ly = iy - W.y0, lz = iz - W.z0;
    if (lx < 0 || ly < 0 || lz < 0 || lx >= W.X || ly >= W.Y || lz >= W.Z) {
        bad = true;
        lx = min(max(lx, 0), W.X - 1);
        ly = min(max(ly, 0), W.Y - 1);
        lz = min(max(lz, 0), W.Z - 1);
        ix = lx + W.x0; iy = ly + W.y0; iz = lz + W.z0;
    }
    if (bad) atomicOr(err, ERR_ESCAPED);
    const uint32_t key = seg * p.M + cell_key(lx, ly, lz, W, p);
    keys[i] = key;
    rank[i] = atomicAdd(&count[key], 1u);
    ps.w = __uint_as_float(encode_cell(ix, iy, iz, p));
    pos[i] = ps;
}

// Final slot of the element k_scatter put at slot s, for the terrain: inside a
// cell the particles are ordered by their x offset (ties by input index), so
// the cells of an x-row are sorted by x and the neighbour search can stop a
// scan once the x-gap alone exceeds the cut-off.
__device__ __forceinline__ uint32_t xsorted_slot(const uint32_t *__restrict__ keys,
                                                 const uint32_t *__restrict__ start,
                                                 const uint32_t *__restrict__ tmp,
                                                 const float4 *__restrict__ pos, uint32_t i)
{
    const uint32_t key = keys[i];
    const uint32_t b = start[key], e = start[key + 1];
    const float xi = pos[i].x;
    uint32_t r = 0;
    for (uint32_t u = b; u < e; ++u) {
        const uint32_t k = tmp[u];
        const float xk = pos[k].x;
        r += (xk < xi || (xk == xi && k < i)) ? 1u : 0u;
    }
    return b + r;
}

// Stable fix-up + gather of every particle array into sorted order (H4).
__global__ void k_reorder(const int *__restrict__ n_dev, const uint32_t *__restrict__ keys,
                          const uint32_t *__restrict__ start, const uint32_t *__restrict__ tmp,
                          StageArrays src, const uint32_t *__restrict__ pid_src, StageArrays dst,
                          uint32_t *__restrict__ pid_dst, const int *__restrict__ abort_flag,
                          const int *__restrict__ gate)
{
    if (*abort_flag || (gate != nullptr && __ldg(gate) == 0)) return;
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= __ldg(n_dev)) return;
    const uint32_t i = tmp[s];
    const uint32_t d = xsorted_slot(keys, start, tmp, src.pos, i);
    dst.pos[d] = src.pos[i];
    dst.vel[d] = src.vel[i];
    dst.sA[d] = src.sA[i];
    dst.sB[d] = src.sB[i];
    pid_dst[d] = pid_src[i];
}

// Neighbour lists (Alg. 1): for particle s scan the 27 cells around its home
// cell and keep j when |x_s - x_j| < 2h (strict).  Fluid particles take fluid
// and marker neighbours, markers take fluid neighbours only.  The scan is cell
// by cell, so the cell offset (dx, dy, dz) of j is a loop constant; a row
// (dy, dz) whose nearest face is already 2h away is skipped, and because every
// cell is sorted by x only a top run of the left cell (found walking down from
// its right end) and a bottom run of the right cell (read until the x-gap alone
// reaches the remaining radius) can hold neighbours.  (Both cut-offs carry a
// 1e-5 relative margin, so they never drop a pair the full test would keep.)
// The list is an ELL table nbr[k * ell + s] (coalesced across a warp) in
// ascending slot order (fluid segment first, cells in key order, each cell
// upwards), so the k-th entries of neighbouring particles -- neighbouring lanes
// of the pair kernels -- are close in memory; each entry is j | code << 26 with
// code = (dx+1) | (dy+1) << 2 | (dz+1) << 4, which the pair kernels use to
// rebuild x_s - x_j from the cell-relative offsets.  (A skin search splits each
// fluid particle's list: the pairs within 2h in that order at the front, the rest
// of the skin radius in that order at the back, from the last entry down.)
//
// One row (dy, dz) of the 27-cell stencil in segment seg (0 fluid, 1 markers):
// the neighbours of particle s in cells dx = -1, 0, 1, counted and, with `nbr`,
// written in ascending slot order: those closer than sqrt(r2in) (the inner part)
// from list position at_in on, the others (the shell between sqrt(r2in) and the
// search radius) from position cap - 1 - at_sh downward.  Returns the two counts.
// The candidates are fetched BATCH at a time (their loads in flight together)
// and then taken in order, as a one-by-one walk would.
constexpr int kSearchBatch = 4;   // candidates in flight per row walk of a one-lane search

template <int BATCH>
__device__ __forceinline__ int2 row_neighbors(const DevParams &p, const float4 *__restrict__ pos,
                                             const uint32_t *__restrict__ start, const Window &W,
                                             int s, const float4 &ps, int lx, int ly, int lz,
                                             int seg, int dy, int dz, float r2cut, float lim2,
                                             float r2in, uint32_t *__restrict__ nbr, int at_in,
                                             int at_sh, int cap)
{
    const int lz2 = lz + dz, ly2 = ly + dy;
    if (lz2 < 0 || lz2 >= W.Z || ly2 < 0 || ly2 >= W.Y) return make_int2(0, 0);
    const float cell = p.cell;
    const float gz = dz < 0 ? fmaxf(ps.z, 0.f) : (dz > 0 ? fmaxf(cell - ps.z, 0.f) : 0.f);
    const float gy = dy < 0 ? fmaxf(ps.y, 0.f) : (dy > 0 ? fmaxf(cell - ps.y, 0.f) : 0.f);
    const float d2 = gy * gy + gz * gz;
    if (d2 >= lim2) return make_int2(0, 0);
    const float R = sqrtf(lim2 - d2);
    const float sy = ps.y - (float)dy * cell, sz = ps.z - (float)dz * cell;
    const uint32_t kb = seg * p.M;
    const uint32_t codeyz = (uint32_t)(dy + 1) << 2 | (uint32_t)(dz + 1) << 4;
    int cnt = 0, csh = 0;
#pragma unroll
    for (int dx = -1; dx <= 1; ++dx) {
        const int lx2 = lx + dx;
        if (lx2 < 0 || lx2 >= W.X) continue;
        const uint32_t key = kb + cell_key(lx2, ly2, lz2, W, p);
        const int jb = (int)start[key], je = (int)start[key + 1];
        const float sx = ps.x - (float)dx * cell;
        const uint32_t tag = ((uint32_t)(dx + 1) | codeyz) << kIndexBits;
        // cells are x-sorted: in the left cell only a top run is within R in
        // x (found walking down), in the right cell only a bottom run
        int j0 = jb;
        if (dx < 0) {
            j0 = je;
            bool more = true;
            while (more && j0 > jb) {
                float xs[BATCH];
#pragma unroll
                for (int u = 0; u < BATCH; ++u) xs[u] = j0 - 1 - u >= jb ? pos[j0 - 1 - u].x : 0.f;
#pragma unroll
                for (int u = 0; u < BATCH; ++u) {
                    if (more && j0 > jb && fabsf(sx - xs[u]) < R) --j0;
                    else more = false;
                }
            }
        }
        bool more = true;
        for (int j = j0; more && j < je; j += BATCH) {
            float4 pb[BATCH];
#pragma unroll
            for (int u = 0; u < BATCH; ++u)
                pb[u] = j + u < je ? pos[j + u] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int u = 0; u < BATCH; ++u) {
                if (!more || j + u >= je) break;
                const float rx = sx - pb[u].x;
                if (dx > 0 && fabsf(rx) >= R) {
                    more = false;
                    break;
                }
                const float ry = sy - pb[u].y, rz = sz - pb[u].z;
                const float r2 = rx * rx + ry * ry + rz * rz;
                if (r2 < r2cut && j + u != s) {
                    const uint32_t e = (uint32_t)(j + u) | tag;
                    if (r2 < r2in) {
                        if (nbr != nullptr && at_in + cnt < cap) nbr[(size_t)(at_in + cnt) * p.ell + s] = e;
                        ++cnt;
                    } else {
                        const int k = cap - 1 - (at_sh + csh);
                        if (nbr != nullptr && k >= 0) nbr[(size_t)k * p.ell + s] = e;
                        ++csh;
                    }
                }
            }
        }
    }
    return make_int2(cnt, csh);
}

// LANES lanes share a particle.  One lane walks the 18 rows (fluid then marker
// segment, each dz-major) in order, writing as it goes.  With more, the rows are
// dealt out round robin; the lanes count their rows, agree on the rows' offsets
// by shuffles, and write their rows' entries there: the same list at a fraction
// of the serial latency but twice the reads, which pays only while the grid is
// small against the GPU (launch_neighbors picks).
// r2in > 0 (the skin search): a fluid particle's list holds the pairs closer than
// sqrt(r2in) at the list's front and the rest of the search radius at the back of
// its cap entries, nnb = inner count | shell count << 16 (the filtering stage 1
// tests the shell's candidates apart); markers' lists are one front part.
template <int LANES>
__global__ void __launch_bounds__(kBlock)
k_neighbors(DevParams p, const float4 *__restrict__ pos, const uint32_t *__restrict__ start,
            uint32_t *__restrict__ nbr, uint32_t *__restrict__ nnb, int cap, float r2cut,
            float r2in, int *__restrict__ err)
{
    constexpr int kSearchLanes = LANES;
    if (*p.abort || gated_off(p)) return;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int s = t / kSearchLanes, q = t % kSearchLanes;
    const Sizes z = load_sizes(p);
    const bool valid = s < z.N;
    const Window W = load_window(p);
    float4 ps = make_float4(0.f, 0.f, 0.f, 0.f);
    int lx = 0, ly = 0, lz = 0;
    if (valid) {
        ps = pos[s];
        int ix, iy, iz;
        decode_cell(__float_as_uint(ps.w), p, ix, iy, iz);
        lx = ix - W.x0; ly = iy - W.y0; lz = iz - W.z0;
    }
    const int rows = valid ? (s < z.nF ? 18 : 9) : 0;
    const float lim2 = r2cut * (1.0f + 1e-5f);
    const float rin = (r2in > 0.0f && s < z.nF) ? r2in : 3.0e38f;   // the inner part's radius^2
    if constexpr (LANES == 1) {
        if (!valid) return;
        int cin = 0, csh = 0;
        for (int r = 0; r < rows; ++r) {
            const int2 c = row_neighbors<kSearchBatch>(p, pos, start, W, s, ps, lx, ly, lz, r / 9,
                                                       (r / 3) % 3 - 1, r % 3 - 1, r2cut, lim2, rin,
                                                       nbr, cin, csh, cap);
            cin += c.x;
            csh += c.y;
        }
        if (cin + csh > cap) atomicOr(err, ERR_CAPACITY);
        nnb[s] = (uint32_t)min(cin, cap) | (uint32_t)min(csh, cap) << 16;
        return;
    }
    constexpr int kPer = (18 + kSearchLanes - 1) / kSearchLanes;
    int2 c[kPer];
    int off[kPer], offs[kPer];
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
        const int r = k * kSearchLanes + q;
        c[k] = r < rows ? row_neighbors<1>(p, pos, start, W, s, ps, lx, ly, lz, r / 9,
                                           (r / 3) % 3 - 1, r % 3 - 1, r2cut, lim2, rin, nullptr,
                                           0, 0, cap)
                        : make_int2(0, 0);
        off[k] = offs[k] = 0;
    }
    // rows in order: row r is lane (r % kSearchLanes)'s entry r / kSearchLanes
    const int base = (threadIdx.x & 31) & ~(kSearchLanes - 1);
    int run = 0, runs = 0;
#pragma unroll
    for (int r = 0; r < 18; ++r) {
        const int n_r = __shfl_sync(0xffffffffu, c[r / kSearchLanes].x, base + r % kSearchLanes);
        const int s_r = __shfl_sync(0xffffffffu, c[r / kSearchLanes].y, base + r % kSearchLanes);
        if (r % kSearchLanes == q) {
            off[r / kSearchLanes] = run;
            offs[r / kSearchLanes] = runs;
        }
        run += n_r;
        runs += s_r;
    }
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
        const int r = k * kSearchLanes + q;
        if (r < rows && (c[k].x > 0 || c[k].y > 0))
            row_neighbors<1>(p, pos, start, W, s, ps, lx, ly, lz, r / 9, (r / 3) % 3 - 1, r % 3 - 1,
                             r2cut, lim2, rin, nbr, off[k], offs[k], cap);
    }
    if (valid && q == 0) {
        if (run + runs > cap) atomicOr(err, ERR_CAPACITY);
        nnb[s] = (uint32_t)min(run, cap) | (uint32_t)min(runs, cap) << 16;
    }
}

// Host launchers of the terrain rebuild, one kernel each.
void launch_keys(const DevParams &p, StageArrays cur, const uint32_t *pid_cur, const double *mloc,
                 const BodyDev *bodies, const SortScratch &s, int *err,
                 int n_fluid_total, cudaStream_t st)
{
    k_keys<<<grid_for(p.capN), kBlock, 0, st>>>(p, cur.pos, pid_cur, mloc, bodies, s.keys,
                                             s.rank, s.count, err, n_fluid_total);
}

void launch_scatter(const DevParams &p, const SortScratch &s, const uint32_t *start,
                    cudaStream_t st)
{
    k_scatter<<<grid_for(p.capN), kBlock, 0, st>>>(s.keys, s.rank, start, s.tmp, p.capN,
                                                   p.sizes + 2, p.abort, p.gate);
}

void launch_reorder(const DevParams &p, const SortScratch &s, const uint32_t *start,
                    StageArrays cur, const uint32_t *pid_cur, StageArrays nxt, uint32_t *pid_nxt,
                    cudaStream_t st)
{
    k_reorder<<<grid_for(p.capN), kBlock, 0, st>>>(p.sizes + 2, s.keys, start, s.tmp, cur, pid_cur,
                                                   nxt, pid_nxt, p.abort, p.gate);
}

void launch_neighbors(const DevParams &p, const float4 *pos, const uint32_t *start, uint32_t *nbr,
                      uint32_t *nnb, int cap, float r2cut, int *err, cudaStream_t st, float r2in)
{
    // lanes per particle: eight up to four waves of the GPU's threads (each lane
    // walks at most three rows of the stencil: on the 25,600-particle active set of
    // the rover strip 76 against 82 us with four lanes, 90 with sixteen), else one
    // (the 191,000 slots of the 120,000-particle wheel bin: 146 us with one lane
    // against 233 us with eight, whose 1.5 M threads made eight waves)
    if ((int64_t)p.capN * 8 <= (int64_t)p.n_sm * 2048 * 4)
        k_neighbors<8><<<grid_for((int64_t)p.capN * 8), kBlock, 0, st>>>(p, pos, start, nbr, nnb,
                                                                         cap, r2cut, r2in, err);
    else
        k_neighbors<1><<<grid_for(p.capN), kBlock, 0, st>>>(p, pos, start, nbr, nnb, cap, r2cut,
                                                            r2in, err);
}

// ---------------------------------------------------------------------------
// Verlet skin.  Alg. 2 asks for the exact 2h neighbour sets of the positions at
// each rebuild step.  With a skin s the cell search keeps every pair closer
// than R = 2h (1 + s); as long as no particle has moved more than s h since that
// search, every pair now closer than 2h is in those lists, so filtering them
// gives exactly the sets a fresh search would.  The search (and the cell sort
// before it) is redone only when the largest displacement reaches s h.

// k_decide: the cell search is due when forced or when the largest squared
// displacement since the last search reached disp_thr2.  With a graph
// conditional handle, it also switches the graph's rebuild branch.
__global__ void k_decide(DevParams p, int *__restrict__ gate,
                         cudaGraphConditionalHandle h, int use_handle, int *__restrict__ counts)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    if (counts != nullptr) {   // the step's Active / Extended counts start from zero
        counts[3] = 0;
        counts[4] = 0;
    }
    int due = 0;
    if (!*p.abort) {
        const float d2 = __int_as_float(gate[GATE_DISP]);
        due = (gate[GATE_FORCE] != 0 || !(d2 < p.disp_thr2)) ? 1 : 0;
        // with active boxes: also when a box may have left the working set's margin
        if (p.act_skin && !(__int_as_float(gate[GATE_BOX]) < p.box_thr2)) due = 1;
    }
    gate[GATE_REBUILD] = due;
    if (due) {
        gate[GATE_DISP] = 0;
        gate[GATE_BOX] = 0;
        gate[GATE_FORCE] = 0;
        gate[GATE_SEARCHES] += 1;
    }
    if (use_handle) cudaGraphSetConditional(h, (unsigned)due);
}

// After a search: the re-sorted arrays become the current ones, the searched
// positions become the displacement reference, and so do the body poses.
__global__ void k_copyback(DevParams p, StageArrays src, const uint32_t *__restrict__ pid_src,
                           StageArrays dst, uint32_t *__restrict__ pid_dst,
                           float4 *__restrict__ xref, BodyDev *__restrict__ bodies)
{
    if (*p.abort || gated_off(p)) return;
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s == 0)
        for (int b = 0; b < p.n_bodies; ++b)
            for (int k = 0; k < 7; ++k) bodies[b].ref_pose[k] = bodies[b].pose[k];
    if (s >= __ldg(p.sizes + 2)) return;
    const float4 ps = src.pos[s];
    dst.pos[s] = ps;
    dst.vel[s] = src.vel[s];
    dst.sA[s] = src.sA[s];
    dst.sB[s] = src.sB[s];
    pid_dst[s] = pid_src[s];
    xref[s] = ps;
}

void launch_decide(const DevParams &p, int *gate, unsigned long long cond_handle, int use_handle,
                   cudaStream_t st, int *counts)
{
    k_decide<<<1, 32, 0, st>>>(p, gate, (cudaGraphConditionalHandle)cond_handle, use_handle,
                               counts);
}

void launch_copyback(const DevParams &p, StageArrays src, const uint32_t *pid_src, StageArrays dst,
                     uint32_t *pid_dst, float4 *xref, BodyDev *bodies, cudaStream_t st)
{
    k_copyback<<<grid_for(p.capN), kBlock, 0, st>>>(p, src, pid_src, dst, pid_dst, xref, bodies);
}

}  // namespace crm

// ---------------------------------------------------------------------------
// Stateless binning entry points (include/crm.h).
namespace {
inline size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// Scratch of one stateless binning call: the radix sort's key/value buffers
// (two pairs, ping-ponged), the digit histograms and their offsets, the cell
// counts, the look-back words of the scans and the counters (ctr[3] collects
// device-side failures).
struct BinLayout {
    size_t kA, vA, kB, vB, hist, offs, count, status, ctr, total;
    int64_t radix_tiles, scan_tiles;
};

BinLayout bin_layout(int64_t n, int64_t ncell)
{
    BinLayout L;
    const int64_t nn = n > 0 ? n : 1;
    L.radix_tiles = (nn + crm::kRadixTile - 1) / crm::kRadixTile;
    const int64_t nh = 256 * L.radix_tiles;
    L.scan_tiles = (std::max<int64_t>(ncell + 1, nh) + crm::kScanTile - 1) / crm::kScanTile;
    size_t o = 0;
    L.kA = o;     o += align256(sizeof(uint32_t) * (size_t)nn);
    L.vA = o;     o += align256(sizeof(uint32_t) * (size_t)nn);
    L.kB = o;     o += align256(sizeof(uint32_t) * (size_t)nn);
    L.vB = o;     o += align256(sizeof(uint32_t) * (size_t)nn);
    L.hist = o;   o += align256(sizeof(uint32_t) * (size_t)nh);
    L.offs = o;   o += align256(sizeof(uint32_t) * (size_t)nh);
    L.count = o;  o += align256(sizeof(uint32_t) * (size_t)(ncell + 1));
    L.status = o; o += align256(sizeof(unsigned long long) * (size_t)L.scan_tiles);
    L.ctr = o;    o += align256(sizeof(uint32_t) * 4);
    L.total = o;
    return L;
}

bool bin_args_ok(const float *xyz, int64_t n, float cell_size, const int32_t dims[3],
                 const uint32_t *cell_out, const uint32_t *perm_out, const uint32_t *cell_start_out)
{
    if (!dims || !cell_start_out || n < 0 || n >= (int64_t(1) << 31)) return false;
    if (n > 0 && (!xyz || !cell_out || !perm_out)) return false;
    if (!(cell_size > 0.0f) || dims[0] < 1 || dims[1] < 1 || dims[2] < 1) return false;
    return (int64_t)dims[0] * dims[1] * dims[2] < (int64_t(1) << 31);
}

// The binning itself on a scratch area laid out by L.  The parts that must
// start at zero (cell counts, look-back words, counters) are cleared here; the
// rest is written before it is read.
int bin_points_on(const float *xyz, int64_t n, float cell_size, const int32_t dims[3],
                  uint32_t *cell_out, uint32_t *perm_out, uint32_t *cell_start_out, char *base,
                  const BinLayout &L, cudaStream_t st)
{
    const int64_t ncell = (int64_t)dims[0] * dims[1] * dims[2];
    if (cudaMemsetAsync(base + L.count, 0, sizeof(uint32_t) * (size_t)(ncell + 1), st) != cudaSuccess
        || cudaMemsetAsync(base + L.status, 0, L.total - L.status, st) != cudaSuccess)
        return CRM_ECUDA;
    crm::SortScratch s{};
    s.count = (uint32_t *)(base + L.count);
    s.tile_status = (unsigned long long *)(base + L.status);
    s.ctr = (uint32_t *)(base + L.ctr);
    int *err = (int *)(s.ctr + 3);
    if (n > 0)
        crm::k_hash_points<<<crm::grid_for(n), crm::kBlock, 0, st>>>(
            xyz, n, 1.0f / cell_size, dims[0], dims[1], dims[2], cell_out, s.count);
    crm::launch_scan_reset(s.count, cell_start_out, ncell + 1, s, err, st);
    if (n > 0) {
        int bits = 1;
        while (bits < 31 && ((ncell - 1) >> bits) != 0) ++bits;
        const int passes = (bits + 7) / 8;
        const int64_t tiles = L.radix_tiles;
        uint32_t *hist = (uint32_t *)(base + L.hist), *offs = (uint32_t *)(base + L.offs);
        uint32_t *kbuf[2] = {(uint32_t *)(base + L.kA), (uint32_t *)(base + L.kB)};
        uint32_t *vbuf[2] = {(uint32_t *)(base + L.vA), (uint32_t *)(base + L.vB)};
        const uint32_t *kin = cell_out, *vin = nullptr;
        for (int ps = 0; ps < passes; ++ps) {
            const bool last = ps == passes - 1;
            uint32_t *kout = last ? nullptr : kbuf[ps & 1];
            uint32_t *vout = last ? perm_out : vbuf[ps & 1];
            crm::k_radix_hist<<<(unsigned)tiles, crm::kRadixThreads, 0, st>>>(kin, n, 8 * ps, tiles,
                                                                           hist, err);
            crm::launch_scan_reset(hist, offs, 256 * tiles, s, err, st);
            crm::k_radix_scatter<<<(unsigned)tiles, crm::kRadixThreads, 0, st>>>(
                kin, vin, n, 8 * ps, tiles, offs, kout, vout, err);
            kin = kout;
            vin = vout;
        }
    }
    crm::k_bin_status<<<1, 1, 0, st>>>(cell_start_out, ncell, err);
    return cudaGetLastError() == cudaSuccess ? CRM_OK : CRM_ECUDA;
}
}  // namespace

extern "C" size_t crm_bin_scratch_bytes(int64_t n, int64_t ncell)
{
    if (n < 0 || ncell < 1) return 0;
    return bin_layout(n, ncell).total;
}

extern "C" int crm_bin_points(const float *xyz, int64_t n, float cell_size, const int32_t dims[3],
                              uint32_t *cell_out, uint32_t *perm_out, uint32_t *cell_start_out,
                              void *scratch, size_t scratch_bytes, void *cuda_stream)
{
    if (!bin_args_ok(xyz, n, cell_size, dims, cell_out, perm_out, cell_start_out) || !scratch)
        return CRM_EINVAL;
    if (((uintptr_t)scratch & 255u) != 0) return CRM_EINVAL;
    const BinLayout L = bin_layout(n, (int64_t)dims[0] * dims[1] * dims[2]);
    if (scratch_bytes < L.total) return CRM_EINVAL;
    return bin_points_on(xyz, n, cell_size, dims, cell_out, perm_out, cell_start_out,
                         (char *)scratch, L, (cudaStream_t)cuda_stream);
}

// ---------------------------------------------------------------------------
// Allocation-free variant of crm_bin_points (include/crm.h).
//
// For callers that cannot allocate device memory at the time they bin --
// for example code running inside a host callback or a real-time loop where
// cudaMalloc would stall or is forbidden, or a caller whose device memory is
// fully reserved by its own allocator -- the scratch of the sort lives in one
// file-scope device array instead of a caller buffer.  That array is part of
// the library image: every GPU that loads the library holds
// kNoAllocScratchBytes of it until the process exits.
namespace {
constexpr int64_t kNoAllocMaxPoints = int64_t(1) << 20;        // 1,048,576 points
constexpr int64_t kNoAllocMaxCells = (int64_t(1) << 20) - 1;   // 1,048,575 cells
// the layout at both limits bounds the layout of every admissible call
// (each part grows with n or ncell)
constexpr size_t kNoAllocScratchBytes = 22 * (size_t(1) << 20);   // 23,068,672 B

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of g_noalloc_scratch for the current device and context,
// looked up with cudaGetSymbolAddress (host code must not use the symbol
// itself: on the host it is only a stand-in).  The lookup is repeated whenever
// the current context differs from the one the cached address belongs to (a
// device reset gives the device a new primary context and the module a new
// address).
constexpr int kMaxDevices = 64;
struct NoAllocAddr {
    void *ptr = nullptr;
    unsigned long long ctx = 0;
};
NoAllocAddr g_noalloc_addr[kMaxDevices];
std::mutex g_noalloc_mutex;

using CtxGetId = int (*)(void *ctx, unsigned long long *id);
using CtxGetCurrent = int (*)(void **ctx);

// Id of the current context (0 when the driver entry points are unavailable;
// the address is then looked up on every call).
unsigned long long current_ctx_id()
{
    static CtxGetCurrent get_cur = nullptr;
    static CtxGetId get_id = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        cudaDriverEntryPointQueryResult q;
        void *f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess
            && q == cudaDriverEntryPointSuccess)
            get_cur = (CtxGetCurrent)f;
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess
            && q == cudaDriverEntryPointSuccess)
            get_id = (CtxGetId)f;
        cudaGetLastError();
    }
    void *ctx = nullptr;
    unsigned long long id = 0;
    if (!get_cur || !get_id || get_cur(&ctx) != 0 || !ctx || get_id(ctx, &id) != 0) return 0;
    return id;
}

int noalloc_scratch(void **out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return CRM_ECUDA;
    }
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    const unsigned long long ctx = current_ctx_id();
    NoAllocAddr &a = g_noalloc_addr[dev];
    if (!a.ptr || ctx == 0 || a.ctx != ctx) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            a = NoAllocAddr{};
            return CRM_ECUDA;
        }
        a.ptr = p;
        a.ctx = ctx;
    }
    *out = a.ptr;
    return CRM_OK;
}
}  // namespace

extern "C" int crm_bin_points_noalloc(const float *xyz, int64_t n, float cell_size,
                                      const int32_t dims[3], uint32_t *cell_out,
                                      uint32_t *perm_out, uint32_t *cell_start_out,
                                      void *cuda_stream)
{
    if (!bin_args_ok(xyz, n, cell_size, dims, cell_out, perm_out, cell_start_out))
        return CRM_EINVAL;
    const int64_t ncell = (int64_t)dims[0] * dims[1] * dims[2];
    if (n > kNoAllocMaxPoints || ncell > kNoAllocMaxCells) {
        std::fprintf(stderr,
                     "crm_bin_points_noalloc: %lld points / %lld cells exceed the built-in "
                     "scratch limits of %lld points and %lld cells; use crm_bin_points with a "
                     "caller scratch buffer\n",
                     (long long)n, (long long)ncell, (long long)kNoAllocMaxPoints,
                     (long long)kNoAllocMaxCells);
        return CRM_EINVAL;
    }
    const BinLayout L = bin_layout(n, ncell);
    if (L.total > kNoAllocScratchBytes) return CRM_EINVAL;   // cannot happen within the limits
    void *addr = nullptr;
    const int rc = noalloc_scratch(&addr);
    if (rc != CRM_OK) return rc;
    return bin_points_on(xyz, n, cell_size, dims, cell_out, perm_out, cell_start_out,
                         (char *)addr, L, (cudaStream_t)cuda_stream);
}
