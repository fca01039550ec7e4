// Residual VJP kernels (lskum_adjoint.cu). Internal numbering, FP64.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "lskum_device.cuh"

namespace lskum {

// T: double (the FP64 product) or float (the FP32 product of a mixed
// context); the geometry cotangents (wbar, abar, dbar) are FP64 in both
template <class T>
struct AdjParamsT {
    DevGeom g;
    const T *q;            // [n][4] q-variables of the state
    const T *qg;           // [n][8] final q-derivative iterate (order 2)
    const T *Rbar;         // [n][4] residual cotangent
    T *qbar;               // [n][4] q cotangent (accumulated)
    T *gbar;               // [n][8] cotangent of the final q-derivative iterate
    T *ebar;               // [nnz][4] cotangent of the neighbour's reconstructed state, per edge
    double2 *wbar;         // [nnz] cotangents of the sub-stencil weights (w_s, w_n)
    double2 *abar;         // [nnz] cotangents of the full-stencil weights (a_x, a_y)
    double2 *dbar;         // [nnz] cotangent of the edge offset P_i - P_0
    const int32_t *toff;   // [n+1] transpose CSR: incoming edges of each point
    const int32_t *tedge;  // [nnz] edge ids, grouped by destination, in edge order
    const int32_t *tsrc;   // [nnz] owner point of each incoming edge
    const int32_t *perm;   // internal point -> input point
    double inv_gm1;
    int g14;               // gamma == 1.4: beta^(-1/(gamma-1)) = beta^-2.5 (as the forward kernels)
    int order;
};
using AdjParams = AdjParamsT<double>;

cudaError_t build_transpose_csr(int64_t n, int64_t nnz, const int32_t *off, const int32_t *idx, int32_t *toff,
                                int32_t *tedge, int32_t *tsrc, cudaStream_t s);
// flux adjoint: owner pass, then the neighbour-side gather (initialises qbar, gbar, ebar, wbar; adds into
// dbar, which the caller zeroes once per product)
template <class T>
cudaError_t launch_adj_flux(const AdjParamsT<T> &P, cudaStream_t s);
// one E15 pass in reverse: gbar_in is the cotangent of this pass's output,
// gbar_out receives that of its input iterate gprev (nullptr for the first-order pass)
template <class T>
cudaError_t launch_adj_grad(const AdjParamsT<T> &P, const T *gprev, const T *gbar_in, T *gbar_out, cudaStream_t s);
// the limiter (limiter_K > 0) in reverse, between the flux adjoint and the
// last pass's: gbar_in is the cotangent of the limited last iterate, graw the
// unlimited one; gbar_out receives the unlimited iterate's cotangent; adds
// into qbar (the point and, through lidx/lval ([n][4] scratch), its extreme
// neighbours) and into dbar (the largest-shift and nearest-neighbour edges)
cudaError_t launch_adj_limit(const AdjParams &P, const double *graw, const double *gbar_in, double *gbar_out,
                             int32_t *lidx, double *lval, double limK, cudaStream_t s);
// least-squares weight cotangents (abar, wbar) into the offset cotangents dbar
cudaError_t launch_adj_weights(const AdjParams &P, cudaStream_t s);
// offsets (dbar) plus per-point cotangents pxy (internal, or nullptr) to x_bar, y_bar in input
// order (either may be nullptr), written or added
cudaError_t launch_adj_points(const AdjParams &P, const double2 *pxy, double *x_bar, double *y_bar, bool accumulate,
                              cudaStream_t s);
// Ub_acc ([n][4], internal order) += (dq/dU)^T qbar at the internal state U
template <class T>
cudaError_t launch_adj_state(const AdjParamsT<T> &P, const double *U, double *Ub_acc, cudaStream_t s);

// b[i] = (float)a[i], i < m
cudaError_t launch_to_float(int64_t m, const double *a, float *b, cudaStream_t s);

// pseudo-time update: boundary treatment and time step of the points
struct StageParams {
    int64_t n;
    const uint8_t *flag;
    const double2 *nrm;
    const double *dt;
    const uint16_t *pcase;    // batch: case of each point, or nullptr
    const double *case_uinf;  // batch: free stream of each case, or nullptr
    double Uinf[4];
};
// U' = P(U^n - c dt R)
cudaError_t launch_stage_fwd(const StageParams &S, const double *Un, const double *R, double c, double *Uout,
                             cudaStream_t s);
// reverse of one stage (see lskum_adjoint.cu)
cudaError_t launch_stage_adj(const StageParams &S, const double *Ub_out, const double *R, double c, bool init,
                             double *Uacc, double *dtbar, double *Rbar, cudaStream_t s);
cudaError_t launch_stage_adj_rk4_final(const StageParams &S, const double *Ub_out, const double *const R[4],
                                       double *Uacc, double *dtbar, double *const Rb[4], cudaStream_t s);
// reverse of the local time step: Uacc += (ddt/dU)^T dtbar, dbar of the nearest-neighbour edge
cudaError_t launch_dt_adj(const StageParams &S, const DevGeom &g, double cfl, double inv_gm1, const double *U,
                          const double *dtbar, double *Uacc, double2 *dbar, cudaStream_t s);
// reverse of the force integrals of one wall contour for the force cotangent (fxb, fyb)
cudaError_t launch_forces_adj(int64_t nwall, double gamma, double qinf, const int32_t *wall, const double *ds,
                              const double2 *nrm, const double2 *xy, const double *U, double fxb, double fyb,
                              double *Uacc, double *dsbar, double2 *pxy, cudaStream_t s);

}  // namespace lskum
