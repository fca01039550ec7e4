// Mixed-precision kernels (lskum_mixed.cu): FP32 geometry view and launchers.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "lskum_device.cuh"

namespace lskum {

// flag bit: this point's least-squares closure runs in FP64
enum : uint8_t { FLAG_FP64_CLOSURE = 0x80 };

// Edge arrays are in the SELL-32 layout: slot s of point p at
// slice_off[p / 32] + 32 s + p % 32 (see lskum_mixed.cu).
struct MixedGeom {
    int64_t n;
    const float2 *__restrict__ nrm;       // frame normal
    const uint8_t *__restrict__ flag;     // bits 0-1 point flag, bit 7 FP64 closure
    const float *__restrict__ dmin;       // nearest-neighbour distance
    const int32_t *__restrict__ off;      // CSR offsets (degree = off[p+1] - off[p])
    const int32_t *__restrict__ slice_off;
    const int32_t *__restrict__ sidx;     // per slot: neighbour index | sub-stencil bits << 28
    const float2 *__restrict__ ga;        // per slot: (a_x, a_y) full-stencil weights
    const float4 *__restrict__ gm;        // per point: (Sxx, Sxy, Syy, 0), the full-stencil normal
                                          // matrix M; the slot's offset is d = M a
    const float4 *__restrict__ gf;        // per slot: (dx, dy, w_s, w_n) sub-stencil weights
    const double2 *__restrict__ fxw64;    // per slot: FP64 sub-stencil weights
    // kinetic boundary mode (all nullptr otherwise): mirror images of the
    // neighbours of wall and far-field points, CSR per point (see DevGeom)
    const int32_t *__restrict__ ioff;
    const int32_t *__restrict__ iidx;
    const uint8_t *__restrict__ imask;
    const float2 *__restrict__ ilsw;      // full-stencil weights (the offset is d = M a)
    const float4 *__restrict__ igf;       // (dx, dy, w_s, w_n) of the image
    const double2 *__restrict__ ifxw64;   // FP64 sub-stencil weights of the image
    const float *__restrict__ qinf;       // [cases][4] q of each case's free stream
    const uint16_t *__restrict__ pcase;   // per point: its case in a batch, or nullptr
    // staged flux variants: tiles of kTile points (tile t = points
    // [kTile t, kTile t + kTile)); the neighbours outside a tile, each once,
    // at tile_idx[tile_off[t] ..] (the first kHaloCap are staged); per slot
    // sloc = its row in the tile's staged block (own points 0..kTile-1, then
    // the staged outside neighbours) | sub-stencil bits << 12, the row being
    // kSlotGlobal where the neighbour was not staged
    const int32_t *__restrict__ tile_off;
    const int32_t *__restrict__ tile_idx;
    const uint16_t *__restrict__ sloc;
};

static constexpr int32_t kSlotIndexMask = 0x0fffffff;  // mixed layout: n < 2^28
static constexpr int kTile = 64;                        // points per staged tile (= its CTA)
static constexpr int kHaloCap = 160;                    // outside neighbours staged per tile
static constexpr uint16_t kSlotGlobal = 0x1ff;          // sloc row: not staged
static constexpr uint16_t kSlotRowMask = 0x1ff;

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
    double *norm_part;        // per warp: pair of R_rho^2 sums (see warp_residue_pair)
    int *status;
    const uint16_t *pcase;    // per point: its case in a batch, or nullptr (one case)
    const double *case_uinf;  // [cases][4] free stream per case, or nullptr (Uinf)
    double Uinf[4];
    float gamma, inv_gm1, cfl;
    int g14;
    int order, mode, stage;
};

// ilsw_f/igf receive the FP32 weights and offsets of the images (kinetic mode, else nullptr)
cudaError_t launch_mixed_prep(const DevGeom &g, uint8_t *flag, float2 *nrm_f, float *dmin_f, float4 *gm,
                              float2 *dxy_f, float2 *lsw_f, float2 *fxw_f, float2 *ilsw_f, float4 *igf,
                              int *n_fp64, cudaStream_t s);
cudaError_t launch_sell_fill(int64_t n, const int32_t *off, const int32_t *slice_off, const int32_t *idx,
                             const uint8_t *mask, const float2 *dxy, const float2 *lsw, const float2 *fxw,
                             const double2 *fxw64, const MixedGeom &m, cudaStream_t s);
// launch-shape variants (threads per block, minimum resident blocks per SM);
// kernel_class 0 = flux, 1 = q-derivatives; variant 0 is the default
int mixed_variants(int kernel_class);
void mixed_variant_shape(int kernel_class, int variant, int *threads, int *min_blocks);
// One q-derivative pass in FP32, with the same pass rules as launch_qgrad:
// an inner pass (qg_old != nullptr) needs g1, the first pass's result for the
// same q, and, when limited, the ext a first pass stored.
cudaError_t launch_qgrad_mixed(const MixedGeom &g, const float *q, const float *qg_old, const float *g1,
                               float *qg_new, float *ext, double limiter_K, cudaStream_t s, int variant);
cudaError_t launch_flux_mixed(const MixedFluxParams &P, cudaStream_t s, int variant);
cudaError_t launch_q_from_U_mixed(int64_t n, const Gas &gas, const double *U, float *q, int *status,
                                  cudaStream_t s);
cudaError_t launch_grad_out_f(int64_t n, const int32_t *perm, const float *qg, double *qx, double *qy,
                              cudaStream_t s);

}  // namespace lskum
