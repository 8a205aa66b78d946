// crm_adjoint.cuh -- types and launchers of the reverse sweep (crm_adjoint.cu).
#pragma once

#include "crm_internal.cuh"

namespace crm {

// Component-major adjoint arrays: component k of slot s at a[k * stride + s].
enum : int { kAdjX = 0, kAdjU = 3, kAdjS = 6, kAdjR = 12, kNumAdj = 13 };
// Pair-sum coefficients: cont, M (3), L (9, row-major), A (3).
enum : int { kNumCoef = 16 };
// BCE coefficients of a marker: w, su (3), ss (6), sr (3).
enum : int { kBceW = 0, kBceSu = 1, kBceSs = 4, kBceSr = 10, kNumBceCoef = 13 };
// Parameter adjoints accumulated on the device (FP64): shear and bulk modulus,
// particle mass, viscosity constant gamma h c_s m, rho0 where it enters
// directly (marker density, 1 / rho0 of the marker accelerations), friction
// coefficient, cohesion, and the mu(I) constants mu_2, I0, grain diameter.
enum : int { kGradG = 0, kGradK, kGradM, kGradAvc, kGradRho0, kGradMu, kGradCoh, kGradMu2,
             kGradI0, kGradGrain, kNumGradAcc };
// Body adjoints, per body: centre (3), linear velocity (3), linear acceleration
// (3), world-frame rotation vector of the orientation (3), angular velocity (3),
// angular acceleration (3).
enum : int { kBodyC = 0, kBodyV = 3, kBodyA = 6, kBodyTheta = 9, kBodyW = 12, kBodyAlpha = 15,
             kBodyAdj = 18 };
// Stage of a sweep pass.
enum : int { kAdjEval = 0, kAdjStage1 = 1, kAdjStage2 = 2 };
enum : int { kAdjAccumulate = 0, kAdjFinal = 1 };

// The forward state one stage's passes read: the slot arrays (fluid, then
// markers with their extrapolated state), the lists, and the bodies (frames ==
// nullptr: markers at the bodies' current pose, else at the given frames).
struct AdjStage {
    StageArrays S;
    const uint32_t *nbr, *nnb, *pid;
    const double *mloc;
    const BodyDev *bodies;
    const BodyFrame *frames;
    int n_fluid_total;
    const float *sums;   // the forward's fluid pair sums at this stage, [13][capF]
};

struct AdjIO {
    float4 *coef;                // 4 per slot (fluid and marker slots): kNumCoef values
    float4 *coefB;               // 4 per marker (slot - nF): kNumBceCoef values, padded
    const float *l_rate;         // evaluation: rate adjoints, insertion order
                                 // (drho [n], du [3n], dsigma [6n])
    const float *l_macc;         // evaluation: marker acceleration adjoints [3 n_markers]
    const double *l_wrench;      // step: adjoint of each body's soil wrench [6 nb]
    const float *l_next;         // step: adjoint of y_{n+1}, kNumAdj x n_fluid, insertion order
    float *l_mid;                // step: adjoint of y_mid, slot order
    float *l_y0;                 // step: adjoint of y_n, slot order
    float *l_out;                // evaluation: local terms, slot order
    int64_t slot_stride;         // stride of the slot-order adjoint arrays
    int64_t n_fluid;             // stride of the insertion-order arrays
    float dt;
};

void launch_adj_fluid_coef(int mode, const DevParams &p, const AdjStage &V, StageArrays Y0,
                           const AdjIO &io, double *gpar, cudaStream_t st);
// act / n_act (nullable): the markers with fluid in reach (every marker slot when null)
void launch_adj_marker(bool acc, const DevParams &p, const AdjStage &V, const AdjIO &io,
                       double *gpar, double *gbody, cudaStream_t st,
                       const uint32_t *act = nullptr, const int *n_act = nullptr);
void launch_adj_fluid(bool acc, int out, const DevParams &p, const AdjStage &V, const AdjIO &io,
                      float *l_acc, float *l_final, double *gpar, cudaStream_t st);
void launch_adj_body_pre(int nb, const BodyDev *bodies, const BodyDev *after, double dt,
                         const double *lb_next, const double *lw_obj, const double *lc_obj,
                         double *l_wrench, double *lb_cur, double *gbody, cudaStream_t st);
void launch_adj_body_post(int nb, const BodyDev *bodies, double dt, const double *g0,
                          const double *gm, double *lb, cudaStream_t st);

}  // namespace crm
