// Residual VJP kernels (lskum_adjoint.cu). Internal numbering, FP64.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "lskum_device.cuh"

namespace lskum {

struct AdjParams {
    DevGeom g;
    const double *q;       // [n][4] q-variables of the state
    const double *qg;      // [n][8] final q-derivative iterate (order 2)
    const double *Rbar;    // [n][4] residual cotangent
    double *qbar;          // [n][4] q cotangent (accumulated)
    double *gbar;          // [n][8] cotangent of the final q-derivative iterate
    double *ebar;          // [nnz][4] cotangent of the neighbour's reconstructed state, per edge
    double2 *wbar;         // [nnz] cotangents of the sub-stencil weights (w_s, w_n)
    double2 *abar;         // [nnz] cotangents of the full-stencil weights (a_x, a_y)
    double2 *dbar;         // [nnz] cotangent of the edge offset P_i - P_0
    const int32_t *toff;   // [n+1] transpose CSR: incoming edges of each point
    const int32_t *tedge;  // [nnz] edge ids, grouped by destination, in edge order
    const int32_t *tsrc;   // [nnz] owner point of each incoming edge
    const int32_t *perm;   // internal point -> input point
    double inv_gm1;
    int order;
};

cudaError_t build_transpose_csr(int64_t n, int64_t nnz, const int32_t *off, const int32_t *idx, int32_t *toff,
                                int32_t *tedge, int32_t *tsrc, cudaStream_t s);
// flux adjoint: owner pass, then the neighbour-side gather (initialises qbar, gbar, ebar, wbar, dbar)
cudaError_t launch_adj_flux(const AdjParams &P, cudaStream_t s);
// one E15 pass in reverse: gbar_in is the cotangent of this pass's output,
// gbar_out receives that of its input iterate gprev (nullptr for the first-order pass)
cudaError_t launch_adj_grad(const AdjParams &P, const double *gprev, const double *gbar_in, double *gbar_out,
                            cudaStream_t s);
// weights to offsets to points; x_bar, y_bar in input order (either may be nullptr)
cudaError_t launch_adj_geometry(const AdjParams &P, double *x_bar, double *y_bar, cudaStream_t s);
// U_bar ([4][n], input order) from qbar at the internal state U ([n][4])
cudaError_t launch_adj_state(const AdjParams &P, const double *U, double *U_bar, cudaStream_t s);

}  // namespace lskum
