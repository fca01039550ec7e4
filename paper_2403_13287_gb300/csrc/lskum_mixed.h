// Mixed-precision kernels (lskum_mixed.cu): FP32 geometry view and launchers.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "lskum_device.cuh"

namespace lskum {

// flag bit: this point's least-squares closure runs in FP64
enum : uint8_t { FLAG_FP64_CLOSURE = 0x80 };

struct MixedGeom {
    int64_t n;
    const float2 *__restrict__ nrm;     // frame normal
    const uint8_t *__restrict__ flag;   // bits 0-1 point flag, bit 7 FP64 closure
    const float *__restrict__ dmin;     // nearest-neighbour distance
    const int32_t *__restrict__ off;
    const int32_t *__restrict__ idx;
    const uint8_t *__restrict__ mask;
    const float2 *__restrict__ dxy;     // per edge: P_i - P_0
    const float2 *__restrict__ lsw;     // per edge: full-stencil weights
    const float2 *__restrict__ fxw;     // per edge: sub-stencil weights
    const double2 *__restrict__ fxw64;  // per edge: FP64 sub-stencil weights
};

struct MixedFluxParams {
    MixedGeom g;
    const double2 *nrm64;  // FP64 normals (wall projection)
    const float *q;        // [n][4]
    const float *qg;       // [n][8] or nullptr
    const double *Un;      // [n][4]
    double *Uout;
    double *acc;
    float *qout;
    double *dt;
    double *R;
    double *norm_part;
    int *status;
    double Uinf[4];
    float gamma, inv_gm1, cfl;
    int g14;
    int order, mode, stage;
};

cudaError_t launch_mixed_prep(const DevGeom &g, const MixedGeom &m, uint8_t *flag, int *n_fp64,
                              cudaStream_t s);
cudaError_t launch_qgrad_mixed(const MixedGeom &g, const float *q, const float *qg_old, float *qg_new,
                               double limiter_K, cudaStream_t s);
cudaError_t launch_flux_mixed(const MixedFluxParams &P, cudaStream_t s);
cudaError_t launch_q_from_U_mixed(int64_t n, const Gas &gas, const double *U, float *q, int *status,
                                  cudaStream_t s);
cudaError_t launch_grad_out_f(int64_t n, const int32_t *perm, const float *qg, double *qx, double *qy,
                              cudaStream_t s);

}  // namespace lskum
