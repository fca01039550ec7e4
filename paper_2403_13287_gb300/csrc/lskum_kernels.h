// Host-side launchers of the hot-path kernels (lskum_kernels.cu).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "lskum_device.cuh"

namespace lskum {

struct FluxLaunch {
    const double *q;
    const double *qg;
    const double *Un;
    double *Uout;
    double *acc;
    double *qout;
    double *dt;
    double *R;
    double *norm_part;
    int *status;
    const uint16_t *pcase;
    const double *case_uinf;
    double cfl;
    int order;
    int mode;   // 0 residual only, 1 forward Euler, 2 RK4 stage
    int stage;
};

// One q-derivative pass. First pass (qg_old == nullptr): the first-order
// solve into qg_new, limited when limiter_K > 0, else with the limiter's
// extremum measure ([n][4]) stored to ext when ext != nullptr. Inner pass:
// needs g1, the first pass's result for the same q, and, when limiter_K > 0,
// the ext a first pass stored (cudaErrorInvalidValue without them).
cudaError_t launch_qgrad(const DevGeom &g, const double *q, const double *qg_old, const double *g1,
                         double *qg_new, double *ext, double limiter_K, cudaStream_t s);
cudaError_t launch_flux(const DevGeom &g, const Gas &gas, const FluxLaunch &L, cudaStream_t s);
// residue of every case into out_base[*counter * ncases + c] (when 0 <= *counter < cap), then ++*counter;
// part holds a pair of sums per warp of 32 points (residue_parts(n) values); chunk is scratch of
// ncases * maxchunks values, maxchunks = the largest residue_chunks() of a case
cudaError_t launch_residue_finish(const double *part, const int64_t *case_start, int ncases, int maxchunks,
                                  double *chunk, double *out_base, int *counter, int cap, cudaStream_t s);
int64_t residue_parts(int64_t n);
int residue_chunks(int64_t case_points);
cudaError_t launch_q_from_U(int64_t n, const Gas &gas, const double *U, double *q, int *status,
                            cudaStream_t s);
cudaError_t launch_timestep(int64_t n, const Gas &gas, double cfl, const double *dmin, const double *U,
                            double *dt, cudaStream_t s);
cudaError_t launch_forces(int64_t nwall, const Gas &gas, double qinf, const int32_t *wall,
                          const double *ds, const double2 *nrm, const double *U, double cosa,
                          double sina, double *cp, double *clcd, cudaStream_t s);

// error text for calls without a context (lskum_api.cu)
void set_global_error(const char *msg);

// create-time geometry (lskum_setup.cu). im: the mirror images of the
// kinetic boundary mode (im.off == nullptr: none); kinetic = the mode is on
// (wall and far-field points then need all four sub-stencils)
struct ImageEdges {
    const int32_t *off = nullptr, *idx = nullptr;
    const uint8_t *mask = nullptr;
    double2 *lsw = nullptr, *fxw = nullptr, *hd = nullptr;
    int kinetic = 0;
};
cudaError_t launch_geometry(int64_t n, const double2 *xy, const double2 *nrm, const uint8_t *flag,
                            const int32_t *off, const int32_t *idx, uint8_t *mask, double2 *lsw,
                            double2 *fxw, double *dmin, int *bad, const ImageEdges &im, cudaStream_t s);

cudaError_t morton_permutation(int64_t n, const double2 *xy, double xmin, double ymin, double scale,
                               int32_t *perm, cudaStream_t s);
cudaError_t launch_permute_points(int64_t n, const int32_t *perm, const double *x, const double *y,
                                  const double *nx, const double *ny, const int32_t *flags,
                                  double2 *xy, double2 *nrm, uint8_t *flag, int32_t *inv,
                                  cudaStream_t s);
cudaError_t permute_csr(int64_t n, const int32_t *perm, const int32_t *inv, const int32_t *off_in,
                        const int32_t *idx_in, int32_t *off_out, int32_t *idx_out, cudaStream_t s);
cudaError_t launch_state_in(int64_t n, const int32_t *perm, const double *Uin_cm, double *U_pm,
                            cudaStream_t s);
cudaError_t launch_state_out(int64_t n, const int32_t *perm, const double *U_pm, double *Uout_cm,
                             cudaStream_t s);
cudaError_t launch_grad_out(int64_t n, const int32_t *perm, const double *qg, double *qx_cm,
                            double *qy_cm, cudaStream_t s);
cudaError_t launch_scalar_out(int64_t n, const int32_t *perm, const double *v, double *out,
                              cudaStream_t s);
cudaError_t launch_mask_out(int64_t n, const int32_t *inv, const int32_t *off_in,
                            const int32_t *off_int, const uint8_t *mask_int, uint8_t *mask_in,
                            cudaStream_t s);
cudaError_t launch_fill_state(int64_t n, const double Uinf[4], double *U, cudaStream_t s);
// hd[e] = (P_i - P_0)/2 for every edge e = (P_0 -> P_i)
cudaError_t launch_half_offsets(int64_t n, const double2 *xy, const int32_t *off, const int32_t *idx, double2 *hd,
                                float2 *hd_f, cudaStream_t s);
cudaError_t launch_fill_state_cases(int64_t n, const uint16_t *pcase, const double *case_uinf, double *U,
                                    cudaStream_t s);
// stable sort of 64-bit keys into a permutation (perm[k] = input index of the k-th smallest key)
cudaError_t sort_permutation(int64_t n, const uint64_t *keys, int32_t *perm, cudaStream_t s);
// host Morton code of a point in [0, 2^bits)^2 cells of the box (xmin, ymin, scale = cells per unit)
uint64_t morton_code_host(double x, double y, double xmin, double ymin, double scale, int bits);

}  // namespace lskum
