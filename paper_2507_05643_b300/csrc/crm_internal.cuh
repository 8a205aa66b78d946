// crm_internal.cuh -- internal types and device helpers of the sm_103a SPH
// terrain library.  Everything here is private to the library; the public
// surface is include/crm.h.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/crm.h"

namespace crm {

// Device-side failure bits, latched with atomicOr into one word per handle.
enum : int {
    ERR_CAPACITY = 1,   // a neighbour list overflowed max_neighbors
    ERR_ESCAPED = 2,    // a particle left the grid window
    ERR_NONFINITE = 4,  // non-finite state after an update
    ERR_TIMEOUT = 8,    // a bounded spin-wait gave up
};

// Abort word value of a device wait that gave up (a terrain's abort word
// otherwise holds 0, or 1 + the step whose capacity overflowed).
constexpr int kAbortTimeout = (int)0x80000000;

constexpr int kMaxBodies = 16;
constexpr uint32_t kExtendedBit = 0x80000000u;   // pid flag: Extended-Active (read-only)
// particle id: insertion index in bits 0..28 (fluid particles, then markers);
// bit 31 = not integrated this step (Extended-Active, or outside); with active
// domains and a Verlet skin, bit 30 = outside every box grown by 2h (in the
// working set's margin: read by nobody) and bit 29 = integrated at some step
// since the working set was gathered (written back to the master store).  Each
// body's markers hold one contiguous id range.
constexpr uint32_t kOutsideBit = 0x40000000u;
constexpr uint32_t kTouchedBit = 0x20000000u;
constexpr uint32_t kPidIndexMask = 0x1FFFFFFFu;
__host__ __device__ __forceinline__ uint32_t pid_index(uint32_t id) { return id & kPidIndexMask; }
constexpr uint32_t kIndexBits = 26;                 // neighbour entry: j | code << 26
constexpr uint32_t kIndexMask = (1u << kIndexBits) - 1u;
constexpr int kBlock = 256;

// Constants of one terrain, passed by value to every kernel.  Single
// precision for the particle arithmetic, double for the grid origin and the
// rigid-body kinematics.
struct DevParams {
    // kernel and material (Sec. 2.1-2.3)
    float h, inv_h, four_h2, cell;        // cell = 2h (Sec. 3.1)
    int kernel;                           // CRM_KERNEL_CUBIC / CRM_KERNEL_WENDLAND
    float kw, kdw;                        // cubic: 1/(pi h^3), 1/(pi h^4); Wendland:
                                          // a = 21/(16 pi h^3), -5 a / h^2
    float m, rho0, G, K;                  // particle mass rho0 d0^3, moduli
    float av_c, xi2;                      // gamma_a h c_s m, xi^2
    int av_mode;
    float gx, gy, gz;
    double g64[3];                        // gravity in FP64 for the body update
    float mu_s, mu_2, I0, grain_d, cohesion;
    // global grid: cell coordinates (ix, iy, iz), c = (iz GY + iy) GX + ix
    int GX, GY, GZ;
    uint32_t M;                           // cells reserved for the working window
    double dmin_x, dmin_y, dmin_z, cell_d;
    // capacities of the working set (grid sizes; the sorted working arrays
    // hold fluid slots [0, nF) then markers [nF, N), nF <= capF, N <= capN)
    int capF, capM, capN;
    int maxnb;
    uint32_t ell;                         // stride of the neighbour table (>= capN)
    int n_bodies;
    uint32_t body_lo[kMaxBodies], body_hi[kMaxBodies];   // particle-id range of each body's markers
    int n_sm;                             // multiprocessors of the device (launch shapes)
    int act_skin;                         // active domains with a Verlet skin: the working
    double act_margin;                    // set is gathered act_margin beyond the boxes
                                          // grown by 2h and kept across steps, until a
    float box_thr2;                       // box may have moved sqrt(box_thr2) < act_margin
    int abs32;                            // test-only: every stored position rounded to an
                                          // absolute FP32 coordinate (crm_debug_absolute_fp32)
    int tbx, tby, tbz;                    // cell tiles of the sort order: log2 of their
                                          // size in cells along x, y, z (see cell_key)
    int pair_lanes;                       // lanes per fluid particle in the exact-list pair
                                          // kernels: 1, 2, or 0 for the default
    unsigned long long *step_ctr;         // active domains: index of the running step (the
                                          // abort tag), advanced by pair stage 2; else null
    // device-resident sizes of the current working set: nF, nM, N, and the
    // window of the cell sort: x0, y0, z0 (global cells) and X, Y, Z
    // (X Y Z <= M).  Kept on the device so that a step needs no host sync.
    const int *sizes;
    const int *win;
    // nonzero once a step of an active-domain run has overflowed a capacity:
    // every later kernel of the enqueued steps returns at once
    const int *abort;
    // Verlet skin: the cell search runs with radius^2 sk_r2 and writes lists of
    // up to skin_cap entries; it is due (gate[0]) once some particle has moved
    // disp_thr2 (squared) since the last search.  gate == nullptr: no skin,
    // every rebuild searches the cells for the exact 2h sets.
    float sk_r2, disp_thr2;
    int skin_cap;
    const int *gate;
};

// gate word layout: [0] rebuild due this step, [1] max squared displacement
// since the last search (float bits, compared as int), [2] forced rebuild
// [3] cell searches done (counter, for the launch bookkeeping)
enum { GATE_REBUILD = 0, GATE_DISP = 1, GATE_FORCE = 2, GATE_BOX = 3, GATE_SEARCHES = 4, GATE_WORDS = 5 };

__device__ __forceinline__ bool gated_off(const DevParams &p)
{
    return p.gate != nullptr && __ldg(p.gate + GATE_REBUILD) == 0;
}

struct Sizes { int nF, nM, N; };
struct Window { int x0, y0, z0, X, Y, Z; };

// Cell keys of the counting sort.  The cells of the window are grouped into
// tiles of 2^tbx x 2^tby x 2^tbz cells; tiles are numbered x fastest, then y,
// then z, and so are the cells inside a tile; key = tile * (tile size) +
// position in the tile.  Slots are sorted by key, so a run of consecutive
// slots -- the particles one thread block or one SM works on -- is a compact
// 3-D piece of the terrain, whose neighbourhood stays in L1, rather than a
// long thin run along x.  Tiles of 1 x 1 x 1 give the row-major order
// c = (z Y + y) X + x.  Tile sizes are at most kTileX x kTileY x kTileZ, so
// every key lies below key_cells(X, Y, Z).
constexpr int kTileX = 8, kTileY = 4, kTileZ = 4;
__host__ __device__ __forceinline__ int64_t key_cells(int64_t X, int64_t Y, int64_t Z)
{
    return ((X + kTileX - 1) / kTileX * kTileX) * ((Y + kTileY - 1) / kTileY * kTileY)
           * ((Z + kTileZ - 1) / kTileZ * kTileZ);
}

template <class P>
__device__ __forceinline__ uint32_t cell_key(int lx, int ly, int lz, const Window &W, const P &p)
{
    const uint32_t bx = (uint32_t)p.tbx, by = (uint32_t)p.tby, bz = (uint32_t)p.tbz;
    const uint32_t x = (uint32_t)lx, y = (uint32_t)ly, z = (uint32_t)lz;
    const uint32_t nbx = ((uint32_t)W.X + (1u << bx) - 1u) >> bx;
    const uint32_t nby = ((uint32_t)W.Y + (1u << by) - 1u) >> by;
    const uint32_t tile = ((z >> bz) * nby + (y >> by)) * nbx + (x >> bx);
    const uint32_t local = ((((z & ((1u << bz) - 1u)) << by) | (y & ((1u << by) - 1u))) << bx)
                           | (x & ((1u << bx) - 1u));
    return (tile << (bx + by + bz)) | local;
}

__device__ __forceinline__ Sizes load_sizes(const DevParams &p)
{
    return Sizes{__ldg(p.sizes), __ldg(p.sizes + 1), __ldg(p.sizes + 2)};
}

__device__ __forceinline__ Window load_window(const DevParams &p)
{
    return Window{__ldg(p.win), __ldg(p.win + 1), __ldg(p.win + 2),
                  __ldg(p.win + 3), __ldg(p.win + 4), __ldg(p.win + 5)};
}

// Rigid body state on the device (FP64, Sec. 2.4 FSI exchange).
struct BodyDev {
    double pose[7];     // x, y, z, qw, qx, qy, qz
    double twist[6];    // v (world), w (world)
    double acc[3];      // linear acceleration of the centre at the last update
    double wrench[6];   // force, torque about the centre (last step)
    double mass;
    int dof;
    int pad;
    double ref_pose[7]; // pose at the last cell search (skin bookkeeping)
    double rmax;        // largest marker distance from the centre
    double alpha[3];    // angular acceleration at the last update (free angular DOFs)
    double inertia[3];  // principal moments of inertia in the body frame
    double load[6];     // external force and torque about the centre, added to the soil's
    double inv_mass;    // 1 / mass (FP64 division is a long sequence on the device)
    double box_reach;   // largest distance from the centre of a point of the body's active
                        // boxes grown by 2h (active domains with a skin; else 0)
};

// Body of the particle with id `id`: -1 for fluid particles and fixed markers.
__device__ __forceinline__ int pid_body(const DevParams &p, uint32_t id)
{
    const uint32_t k = pid_index(id);
    int b = -1;
    for (int q = 0; q < p.n_bodies; ++q)
        if (k >= p.body_lo[q] && k < p.body_hi[q]) b = q;
    return b;
}

// Stage arrays: the state every pair kernel gathers neighbours from.
struct StageArrays {
    float4 *pos;   // offset from the home cell corner (x, y, z), home cell id bits
    float4 *vel;   // u (x, y, z), rho
    float4 *sA;    // sigma xx, yy, zz, xy
    float2 *sB;    // sigma xz, yz
};

// ---------------------------------------------------------------------------
// Cubic spline (Monaghan M4), 3-D normalisation 1/(pi h^3), support 2h.
__device__ __forceinline__ float kernel_w(float q, const DevParams &p)
{
    if (p.kernel == CRM_KERNEL_WENDLAND) {
        // quintic Wendland: a (1 - q/2)^4 (2q + 1)
        const float t = fmaxf(1.0f - 0.5f * q, 0.0f), t2 = t * t;
        return p.kw * t2 * t2 * fmaf(2.0f, q, 1.0f);
    }
    if (q < 1.0f) return p.kw * (1.0f + q * q * (0.75f * q - 1.5f));
    const float t = 2.0f - q;
    return q < 2.0f ? 0.25f * p.kw * t * t * t : 0.0f;
}

// (dW/dr) / r; q < 2 is the caller's guarantee.
__device__ __forceinline__ float kernel_dw_over_r(float q, float rinv, const DevParams &p)
{
    if (p.kernel == CRM_KERNEL_WENDLAND) {
        // dW/dr = -5 a q (1 - q/2)^3 / h, so (dW/dr) / r = -5 a (1 - q/2)^3 / h^2
        const float t = 1.0f - 0.5f * q;
        return p.kdw * t * t * t;
    }
    float d;
    if (q < 1.0f) {
        d = p.kdw * q * (2.25f * q - 3.0f);
    } else {
        const float t = 2.0f - q;
        d = -0.75f * p.kdw * t * t;
    }
    return d * rinv;
}

__device__ __forceinline__ void decode_cell(uint32_t c, const DevParams &p, int &ix, int &iy,
                                            int &iz)
{
    ix = (int)(c % (uint32_t)p.GX);
    const uint32_t t = c / (uint32_t)p.GX;
    iy = (int)(t % (uint32_t)p.GY);
    iz = (int)(t / (uint32_t)p.GY);
}

__device__ __forceinline__ uint32_t encode_cell(int ix, int iy, int iz, const DevParams &p)
{
    return ((uint32_t)iz * (uint32_t)p.GY + (uint32_t)iy) * (uint32_t)p.GX + (uint32_t)ix;
}

// ---------------------------------------------------------------------------
// FP64 rigid-body kinematics.  The pose at stage offset tau is the pose
// advanced by the current twist held constant.
__device__ __forceinline__ void qmul(const double a[4], const double b[4], double o[4])
{
    o[0] = a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
    o[1] = a[0] * b[1] + a[1] * b[0] + a[2] * b[3] - a[3] * b[2];
    o[2] = a[0] * b[2] - a[1] * b[3] + a[2] * b[0] + a[3] * b[1];
    o[3] = a[0] * b[3] + a[1] * b[2] - a[2] * b[1] + a[3] * b[0];
}

__device__ __forceinline__ void qrot(const double q[4], const double v[3], double o[3])
{
    // o = v + 2 qv x (qv x v + w v)
    const double w = q[0], x = q[1], y = q[2], z = q[3];
    const double tx = y * v[2] - z * v[1] + w * v[0];
    const double ty = z * v[0] - x * v[2] + w * v[1];
    const double tz = x * v[1] - y * v[0] + w * v[2];
    o[0] = v[0] + 2.0 * (y * tz - z * ty);
    o[1] = v[1] + 2.0 * (z * tx - x * tz);
    o[2] = v[2] + 2.0 * (x * ty - y * tx);
}

// q turned by the rotation vector w tau: dq = (cos phi, sin(phi) w / |w|),
// phi = |w| tau / 2.  A step turns a body by a tiny angle, where the Maclaurin
// series of cos and sin(phi)/phi, cut after the phi^8 terms, are exact in FP64
// (the first dropped term is below phi^10 / 10! < 3e-20 for phi <= 0.05) and
// far cheaper than FP64 trigonometry; larger angles take sincos.
__device__ __forceinline__ void qadvance(const double q[4], const double w[3], double tau,
                                         double o[4])
{
    const double w2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
    const double phi2 = 0.25 * w2 * tau * tau;
    double c, sw;   // cos(phi), sin(phi) / |w|
    if (phi2 <= 0.0025) {
        // products with the reciprocals (an FP64 division is a long software
        // sequence; these differ from it by at most an ulp)
        const double x = phi2;
        c = 1.0 - x * 0.5 * (1.0 - x * (1.0 / 12.0) * (1.0 - x * (1.0 / 30.0) * (1.0 - x * (1.0 / 56.0))));
        sw = 0.5 * tau * (1.0 - x * (1.0 / 6.0) * (1.0 - x * (1.0 / 20.0) * (1.0 - x * (1.0 / 42.0)
                                                                     * (1.0 - x * (1.0 / 72.0)))));
    } else {
        const double wn = sqrt(w2);
        double s;
        sincos(0.5 * wn * tau, &s, &c);
        sw = s / wn;
    }
    const double dq[4] = {c, sw * w[0], sw * w[1], sw * w[2]};
    qmul(dq, q, o);
    const double n = rsqrt(o[0] * o[0] + o[1] * o[1] + o[2] * o[2] + o[3] * o[3]);
    o[0] *= n; o[1] *= n; o[2] *= n; o[3] *= n;
}

// A body's frame at one stage offset: centre and rotation in FP64 (computed
// once per body and block, so the per-marker work is one FP64 matrix product),
// twist and linear acceleration in FP32.
struct BodyFrame {
    double c[3];
    double R[9];   // row-major rotation of the body-local marker positions
    float v[3], w[3], acc[3], alpha[3];
};

__device__ __forceinline__ void body_frame(const BodyDev &b, double tau, BodyFrame &F)
{
    double q[4];
    qadvance(b.pose + 3, b.twist + 3, tau, q);
    const double w = q[0], x = q[1], y = q[2], z = q[3];
    F.R[0] = 1.0 - 2.0 * (y * y + z * z); F.R[1] = 2.0 * (x * y - w * z); F.R[2] = 2.0 * (x * z + w * y);
    F.R[3] = 2.0 * (x * y + w * z); F.R[4] = 1.0 - 2.0 * (x * x + z * z); F.R[5] = 2.0 * (y * z - w * x);
    F.R[6] = 2.0 * (x * z - w * y); F.R[7] = 2.0 * (y * z + w * x); F.R[8] = 1.0 - 2.0 * (x * x + y * y);
    for (int k = 0; k < 3; ++k) {
        F.c[k] = b.pose[k] + tau * b.twist[k];
        F.v[k] = (float)b.twist[k];
        F.w[k] = (float)b.twist[3 + k];
        F.acc[k] = (float)b.acc[k];
        F.alpha[k] = (float)b.alpha[k];
    }
}

// Rigid velocity v + w x r and acceleration a_c + alpha x r + w x (w x r) of a
// body marker with arm r (FP32 is enough: they enter the FP32 rates), and the
// FP64 world position c + r.
__device__ __forceinline__ void marker_kin(const double c[3], const double r[3], const float v[3],
                                           const float w[3], const float acc[3],
                                           const float alpha[3], double x[3], float u[3],
                                           float a[3], float arm[3])
{
    const float rf[3] = {(float)r[0], (float)r[1], (float)r[2]};
    const float wr[3] = {w[1] * rf[2] - w[2] * rf[1], w[2] * rf[0] - w[0] * rf[2],
                         w[0] * rf[1] - w[1] * rf[0]};
    const float wwr[3] = {w[1] * wr[2] - w[2] * wr[1], w[2] * wr[0] - w[0] * wr[2],
                          w[0] * wr[1] - w[1] * wr[0]};
    const float ar[3] = {alpha[1] * rf[2] - alpha[2] * rf[1], alpha[2] * rf[0] - alpha[0] * rf[2],
                         alpha[0] * rf[1] - alpha[1] * rf[0]};
    for (int k = 0; k < 3; ++k) {
        x[k] = c[k] + r[k];
        u[k] = v[k] + wr[k];
        a[k] = acc[k] + ar[k] + wwr[k];
        arm[k] = rf[k];
    }
}

// A body marker at stage offset tau from a precomputed frame.
__device__ __forceinline__ void marker_at(const BodyFrame &F, const double *xloc, double x[3],
                                          float u[3], float a[3], float arm[3])
{
    const double l0 = xloc[0], l1 = xloc[1], l2 = xloc[2];
    const double r[3] = {fma(F.R[0], l0, fma(F.R[1], l1, F.R[2] * l2)),
                         fma(F.R[3], l0, fma(F.R[4], l1, F.R[5] * l2)),
                         fma(F.R[6], l0, fma(F.R[7], l1, F.R[8] * l2))};
    marker_kin(F.c, r, F.v, F.w, F.acc, F.alpha, x, u, a, arm);
}

// A body marker at the current pose (stage offset 0): one quaternion rotation,
// no trigonometry (the stored quaternion is kept normalised).
__device__ __forceinline__ void marker_now(const BodyDev &b, const double *xloc, double x[3],
                                           float u[3], float a[3], float arm[3])
{
    double r[3];
    qrot(b.pose + 3, xloc, r);
    const float v[3] = {(float)b.twist[0], (float)b.twist[1], (float)b.twist[2]};
    const float w[3] = {(float)b.twist[3], (float)b.twist[4], (float)b.twist[5]};
    const float acc[3] = {(float)b.acc[0], (float)b.acc[1], (float)b.acc[2]};
    const float al[3] = {(float)b.alpha[0], (float)b.alpha[1], (float)b.alpha[2]};
    marker_kin(b.pose, r, v, w, acc, al, x, u, a, arm);
}

// A neighbour-list word: read once per kernel, so it is fetched without
// allocating in L1 (which is left to the neighbours' state, re-read by ~56
// particles each).
__device__ __forceinline__ uint32_t ld_list(const uint32_t *p)
{
    uint32_t v;
    asm("ld.global.nc.L1::no_allocate.u32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}

// A cell-relative position rounded as an absolute FP32 coordinate would be
// (the test-only comparison layout of crm_debug_absolute_fp32): the offset
// becomes fp32(corner + offset) - corner.
__device__ __forceinline__ float4 round_absolute(const DevParams &p, float4 ps)
{
    int ix, iy, iz;
    decode_cell(__float_as_uint(ps.w), p, ix, iy, iz);
    const double cx = p.dmin_x + ix * p.cell_d, cy = p.dmin_y + iy * p.cell_d,
                 cz = p.dmin_z + iz * p.cell_d;
    ps.x = (float)((double)(float)(cx + (double)ps.x) - cx);
    ps.y = (float)((double)(float)(cy + (double)ps.y) - cy);
    ps.z = (float)((double)(float)(cz + (double)ps.z) - cz);
    return ps;
}

// Cell offset of a neighbour entry e = j | code << 26 (code = (dx+1) | (dy+1)
// << 2 | (dz+1) << 4, dx, dy, dz in {-1, 0, 1}) times the cell size, in
// registers: 2^23 + c has the bit pattern 0x4B000000 | c for small c, so
// (2^23 + c) - (2^23 + 1) = c - 1 exactly, with no integer-to-float
// conversion, and the products with the cell size are exact.
__device__ __forceinline__ float3 entry_shift(uint32_t e, float cell)
{
    const uint32_t c = e >> kIndexBits;
    const float fx = __uint_as_float(0x4B000000u | (c & 3u)) - 8388609.0f;
    const float fy = __uint_as_float(0x4B000000u | ((c >> 2) & 3u)) - 8388609.0f;
    const float fz = __uint_as_float(0x4B000000u | (c >> 4)) - 8388609.0f;
    return make_float3(fx * cell, fy * cell, fz * cell);
}

// Neighbour lists a kernel walks (and, when filtering, writes).
struct ListIO {
    const uint32_t *in;   // list walked (the skin list when filtering)
    const uint32_t *in_n;
    uint32_t *out;        // exact list written when filtering
    uint32_t *out_n;
    int *err;
};

// ---------------------------------------------------------------------------
// Launch helpers shared by the translation units.
__host__ __device__ inline unsigned grid_for(int64_t n, int block = kBlock)
{
    const int64_t g = (n + block - 1) / block;
    return (unsigned)(g > 0 ? g : 1);
}

// Scratch of one counting sort (Sec. 3.1 steps 2-3).
struct SortScratch {
    uint32_t *keys;         // n
    uint32_t *rank;         // n: arrival rank within the key (atomic)
    uint32_t *tmp;          // n: slot -> input index before the stable fix-up
    uint32_t *count;        // nkeys + 1, zero between uses
    unsigned long long *tile_status;  // scan look-back words
    uint32_t *ctr;          // [0] ticket, [1] epoch, [2] done
    int64_t n_tiles;
};

constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanTile = kScanThreads * kScanItems;

// Exclusive scan of count[0..n) into start[0..n), resetting count to zero.
// Single pass, decoupled look-back; every wait is bounded (ERR_TIMEOUT).
// On a timed-out wait the scan also sets *abort_word (when given) to
// kAbortTimeout.
void launch_scan_reset(uint32_t *count, uint32_t *start, int64_t n, const SortScratch &s,
                       int *err, cudaStream_t st, const int *gate = nullptr,
                       int *abort_word = nullptr);
// Device-wait fault switch of the current device (crm_debug_wait_fault): 0 on success.
int set_wait_fault(int on);

// Rebuild (Alg. 2 "PreprocessNeighborList" + Alg. 1), one kernel per launcher:
// keys + arrival ranks, exclusive scan of the counts (cell ranges, 2M + 1
// entries), scatter, stable reorder of every particle array from `cur` into
// `nxt`, and the neighbour table.
void launch_keys(const DevParams &p, StageArrays cur, const uint32_t *pid_cur, const double *mloc,
                 const BodyDev *bodies, const SortScratch &s, int *err,
                 int n_fluid_total, cudaStream_t st);
void launch_scatter(const DevParams &p, const SortScratch &s, const uint32_t *start,
                    cudaStream_t st);
void launch_reorder(const DevParams &p, const SortScratch &s, const uint32_t *start,
                    StageArrays cur, const uint32_t *pid_cur, StageArrays nxt, uint32_t *pid_nxt,
                    cudaStream_t st);
// r2in > 0: fluid lists split into the pairs closer than sqrt(r2in) (front) and
// the rest of the radius (back of the cap entries), nnb = inner | shell << 16.
void launch_neighbors(const DevParams &p, const float4 *pos, const uint32_t *start, uint32_t *nbr,
                      uint32_t *nnb, int cap, float r2cut, int *err, cudaStream_t st,
                      float r2in = 0.0f);
// Verlet skin (Alg. 2 with a skin): decide whether the cell search is due and
// copy the re-sorted arrays back (the stage-1 kernels filter the skin lists
// down to the exact 2h lists).
void launch_decide(const DevParams &p, int *gate, unsigned long long cond_handle, int use_handle,
                   cudaStream_t st, int *counts = nullptr);
// Active domains with a Verlet skin: the activity of every working-set fluid
// particle against this step's boxes (Active / Extended-Active / outside bits
// of its pid) and the Active and Extended counts (counts[3], counts[4]).
void launch_flags(const DevParams &p, int nbox, const int *box_body, const double *box_half,
                  const double *box_off, const BodyDev *bodies, int all_active, uint32_t *pid,
                  const float4 *pos, int *counts, cudaStream_t st);
void launch_copyback(const DevParams &p, StageArrays src, const uint32_t *pid_src, StageArrays dst,
                     uint32_t *pid_dst, float4 *xref, BodyDev *bodies, cudaStream_t st);


struct RateOut {
    float *drho;    // [slot]
    float4 *du;     // [slot] (x, y, z, 0)
    float4 *dsA;    // [slot] xx, yy, zz, xy
    float2 *dsB;    // [slot] xz, yz
    float *sums;    // nullable, any mode: each fluid particle's pair sums (continuity,
                    // M (3), L (9)), component-major [13][capF] (for the adjoint's tape)
};

enum { kStage1 = 0, kStage2 = 1, kEval = 2 };

// Pair sums of the fluid particles; with sk_nbr (stage 1 with a skin) the
// particles walk their skin lists and write their exact lists to nbr / nnb.
void launch_pair(int mode, const DevParams &p, StageArrays S, StageArrays Y, StageArrays MID,
                 const uint32_t *nbr, const uint32_t *nnb, const uint32_t *pid, float dt,
                 RateOut out, int *err, const float4 *xref, int *gate, cudaStream_t st,
                 const uint32_t *sk_nbr = nullptr, const uint32_t *sk_nnb = nullptr);
// BCE state of every marker slot of S at stage offset tau; accel 1 instead
// sums the active body markers' forces and torques per block into FP64
// partials (wrench_blocks(body_markers) blocks x bodies x 6), then a second
// kernel sums the partials per body in a fixed order and advances the bodies
// by dt (integrate != 0); accel 2 writes every marker's force to mforce.  With
// sk_nbr (stage 1 with a skin) the markers walk their skin lists and write
// their exact lists to nbr / nnb.  frames (kMaxBodies entries): a launch at
// tau = 0 with dt > 0 writes the bodies' frames at dt / 2 there, and a launch
// at tau != 0 takes its marker kinematics from them.  act / n_act: the marker
// slots to process (nullptr: every marker slot); accel 1 takes the active body
// markers (at most body_markers of them) and reads their state from S.
void launch_bce(const DevParams &p, StageArrays S, const float4 *home_pos, const uint32_t *pid,
                const double *mloc, BodyDev *bodies, const uint32_t *nbr, const uint32_t *nnb,
                double tau, int accel, int n_fluid_total, float4 *mforce, double *partial,
                double dt, int integrate, int *gate, cudaStream_t st,
                const uint32_t *sk_nbr, const uint32_t *sk_nnb, int *err, BodyFrame *frames,
                const uint32_t *act, const int *n_act, int64_t body_markers);
unsigned bce_blocks(const DevParams &p);
unsigned wrench_blocks(int64_t body_markers);
// Marker slots whose list (nnb: the skin lists with a skin) is non-empty, in
// slot order, into act[0 .. n_act[0]), and those of them on a body into
// act_body[0 .. n_act[1]); with nnb_exact the exact counts of the others are
// zeroed.  bcount: 2 compact_blocks(p) words.  Gated like the search.
unsigned compact_blocks(const DevParams &p);
void launch_compact_markers(const DevParams &p, const uint32_t *nnb, const uint32_t *pid,
                            uint32_t *nnb_exact, uint32_t *bcount, uint32_t *act,
                            uint32_t *act_body, int *n_act, cudaStream_t st);
void launch_export(const DevParams &p, StageArrays S, const uint32_t *pid, double *xyz, float *vel,
                   float *sig, float *rho, cudaStream_t st);
void launch_export_rates(const DevParams &p, const uint32_t *pid, RateOut r, StageArrays S,
                         const float4 *mforce, int n_fluid_total, float *drho, float *du,
                         float *ds, float *macc, float *mvel, float *msig, cudaStream_t st);

// ---------------------------------------------------------------------------
// Batches in one persistent launch per stage (crm_batch).  A member as the
// batched stage kernels see it: its constants and the arrays of its step (a
// member with a Verlet skin, without active boxes: its current buffer is fixed).
struct MemberDev {
    DevParams p;
    StageArrays S, MID;                  // current stage arrays, midpoint arrays
    const uint32_t *pid;
    const double *mloc;
    BodyDev *bodies;
    BodyFrame *frames;                   // midpoint body frames
    uint32_t *nbr, *nnb;                 // exact lists (written by stage 1)
    const uint32_t *sk_nbr, *sk_nnb;     // skin lists
    const uint32_t *act, *act_body;      // markers with fluid in reach, those on bodies
    const int *n_act;                    // their counts
    float4 *mforce;
    double *partial;                     // wrench partials
    const float4 *xref;                  // positions at the last search (skin)
    int *gate, *err;
    int n_fluid_total, n_bodym;
    double dt;
};

// Virtual blocks claimed per ticket of a batched launch: one, so that every
// virtual block starts after a block barrier (the lanes of a warp that share a
// particle then always combine their sums within one virtual block).
constexpr int kBatchChunk = 1;

// Copy of a member's descriptor into the block's shared memory (every thread
// of the block calls it; a barrier follows), so that its fields are reloaded
// from shared memory instead of held in registers.
__device__ __forceinline__ void load_member(const MemberDev *src, MemberDev *dst)
{
    static_assert(sizeof(MemberDev) % 4 == 0, "word copy");
    const int *a = reinterpret_cast<const int *>(src);
    int *b = reinterpret_cast<int *>(dst);
    for (int k = threadIdx.x; k < (int)(sizeof(MemberDev) / 4); k += blockDim.x) b[k] = __ldg(a + k);
    __syncthreads();
}

// A batched launch's work: members mlist[k], k < n, own the virtual blocks
// [off[k], off[k + 1]) (each virtual block = one block of that member's own
// launch); queue = {ticket, done}, zero between launches (the last block to
// finish resets it).  Kinds of the BCE launch: 0 stage-1 marker state with the
// skin-list filter, 1 midpoint marker state, 2 wrench forces and partials.
void launch_batch_bce(int kind, const MemberDev *mem, const int *mlist, const int *off, int n,
                      int total, unsigned *queue, cudaStream_t st);
void launch_batch_reduce(const MemberDev *mem, const int *pairs, int npairs, cudaStream_t st);
void launch_batch_pair(int mode, int lanes, int kav, const MemberDev *mem, const int *mlist,
                       const int *off, int n, int total, unsigned *queue, cudaStream_t st);
int pair_kav(const DevParams &p);
int pair_lanes_of(const DevParams &p);
// Lanes per particle of the filtering pair kernels, given the other kernels' lanes.
inline int pair_filter_lanes(int lanes) { return lanes == 4 ? 4 : 1; }

// Active domains (Sec. 3.2, Alg. 3), crm_active.cu.
size_t box_frame_bytes();
void launch_box_prep(const DevParams &p, int nbox, const int *box_body, const double *box_half,
                     const double *box_off, const BodyDev *bodies, const int *colF,
                     const int *colM, const int *drift, int all_active, int n_fluid_master,
                     int n_fixed_master, int64_t cand_cap, void *frames, int *win, int *ranges,
                     int *rinfo, int *counts, int *abort_flag, int64_t step_tag, cudaStream_t st);
void launch_activity(const DevParams &p, int nbox, const void *frames, const int *ranges,
                     const int *rinfo, const float4 *mpos, const double *mloc,
                     const int *fixed_order, int all_active, int64_t cand_cap, uint32_t *include,
                     uint8_t *kind, int *counts, const int *abort_flag, cudaStream_t st);
void launch_active_sizes(const DevParams &p, const int *rinfo, const uint32_t *slot,
                         int n_body_markers, int *counts, int *abort_flag, int64_t step_tag,
                         cudaStream_t st);
void launch_gather(const DevParams &p, const int *ranges, const int *rinfo,
                   const uint8_t *kind, const uint32_t *slot,
                   StageArrays M, const uint32_t *mpid, const int *fixed_order,
                   const int *body_markers, int n_body_markers, int n_fluid_total,
                   int64_t cand_cap, StageArrays W, uint32_t *wpid, const int *counts,
                   const int *abort_flag, cudaStream_t st);
void launch_scatter_back(const DevParams &p, StageArrays W, const uint32_t *wpid,
                         const uint32_t *mslot_of_pid, const int *mcol, StageArrays M, int *drift, int gated,
                         cudaStream_t st);
void launch_export_master(const DevParams &p, StageArrays M, const uint32_t *mpid, int n,
                          double *xyz, float *vel, float *sig, float *rho, cudaStream_t st);
// FP64 global sums of the first n SPH slots of S (n from n_dev when non-null):
// scratch holds diag_scratch_doubles() doubles, the CRM_NUM_DIAG results last.
size_t diag_scratch_doubles();
void launch_diagnostics(const DevParams &p, StageArrays S, const int *n_dev, int n_host, double m,
                        double *scratch, cudaStream_t st);

}  // namespace crm
