// Mixed-precision form of the hot path (not in the paper, which argues for
// FP64 throughout). q, grad q, the least-squares weights and the split-flux
// arithmetic are FP32; the state U, the RK accumulation, the residue and the
// forces stay FP64, and so does the least-squares closure (weights and
// accumulation) at points whose sub-stencil weights amplify rounding.
//
// Per-edge arrays: dxy (float2, the FP64 offset rounded once, so no FP32
// coordinate differences are formed), lsw/fxw (float2 copies of the FP64
// weights). Per point: nrm (float2), dmin (float), flag bit 7 = FP64 closure.
#include "lskum_device.cuh"
#include "lskum_kernels.h"
#include "lskum_mixed.h"

namespace lskum {

// --------------------------------------------------------------------------
// create time: FP32 geometry and the FP64-closure flag
// A point's closure runs in FP64 when, for one of its sub-stencils,
// sum_i |w_i| |P_i - P_0| > kAmpLimit: the weights then cancel strongly and
// FP32 weights/accumulation would lose more than a few bits.
// --------------------------------------------------------------------------
static constexpr double kAmpLimit = 16.0;

// kinetic boundary mode: the images (g.ioff != nullptr) enter the sums and
// the amplification test like neighbours, at their mirrored offsets
__global__ void __launch_bounds__(128) k_mixed_prep(DevGeom g, uint8_t *__restrict__ flag,
                                                    float2 *__restrict__ nrm_f, float *__restrict__ dmin_f,
                                                    float4 *__restrict__ gm, float2 *__restrict__ dxy_f,
                                                    float2 *__restrict__ lsw_f, float2 *__restrict__ fxw_f,
                                                    float2 *__restrict__ ilsw_f, float4 *__restrict__ igf,
                                                    int *n_fp64)
{
    const int64_t n = g.n;
    const double2 *__restrict__ xy = g.xy;
    const double2 *__restrict__ nrm = g.nrm;
    const double *__restrict__ dmin = g.dmin;
    const int32_t *__restrict__ off = g.off;
    const int32_t *__restrict__ idx = g.idx;
    const uint8_t *__restrict__ mask = g.mask;
    const double2 *__restrict__ lsw = g.lsw;
    const double2 *__restrict__ fxw = g.fxw;
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const double2 P0 = xy[p];
    double amp[4] = {0.0, 0.0, 0.0, 0.0};
    double Sxx = 0.0, Sxy = 0.0, Syy = 0.0;
    for (int e = off[p]; e < off[p + 1]; ++e) {
        const double2 Pi = xy[idx[e]];
        const double dx = Pi.x - P0.x, dy = Pi.y - P0.y;
        Sxx += dx * dx;
        Sxy += dx * dy;
        Syy += dy * dy;
        const double d = sqrt(dx * dx + dy * dy);
        dxy_f[e] = make_float2((float)dx, (float)dy);
        const double2 a = lsw[e], w = fxw[e];
        lsw_f[e] = make_float2((float)a.x, (float)a.y);
        fxw_f[e] = make_float2((float)w.x, (float)w.y);
        const uint8_t m = mask[e];
        if (m & M_XPOS) amp[0] += fabs(w.x) * d;
        if (m & M_XNEG) amp[1] += fabs(w.x) * d;
        if (m & M_YPOS) amp[2] += fabs(w.y) * d;
        if (m & M_YNEG) amp[3] += fabs(w.y) * d;
    }
    const double2 n0 = nrm[p];
    if (g.ioff) {
        for (int e = g.ioff[p]; e < g.ioff[p + 1]; ++e) {
            const double2 Pi = xy[g.iidx[e]];
            double dx = Pi.x - P0.x, dy = Pi.y - P0.y;
            const double dn = dx * n0.x + dy * n0.y;
            dx = dx - 2.0 * dn * n0.x;
            dy = dy - 2.0 * dn * n0.y;
            Sxx += dx * dx;
            Sxy += dx * dy;
            Syy += dy * dy;
            const double d = sqrt(dx * dx + dy * dy);
            const double2 a = g.ilsw[e], w = g.ifxw[e];
            ilsw_f[e] = make_float2((float)a.x, (float)a.y);
            igf[e] = make_float4((float)dx, (float)dy, (float)w.x, (float)w.y);
            const uint8_t m = g.imask[e];
            if (m & M_XPOS) amp[0] += fabs(w.x) * d;
            if (m & M_XNEG) amp[1] += fabs(w.x) * d;
            if (m & M_YPOS) amp[2] += fabs(w.y) * d;
            if (m & M_YNEG) amp[3] += fabs(w.y) * d;
        }
    }
    nrm_f[p] = make_float2((float)n0.x, (float)n0.y);
    gm[p] = make_float4((float)Sxx, (float)Sxy, (float)Syy, 0.0f);
    dmin_f[p] = (float)dmin[p];
    const double a = fmax(fmax(amp[0], amp[1]), fmax(amp[2], amp[3]));
    if (a > kAmpLimit) {
        flag[p] |= FLAG_FP64_CLOSURE;
        atomicAdd(n_fp64, 1);
    }
}

cudaError_t launch_mixed_prep(const DevGeom &g, uint8_t *flag, float2 *nrm_f, float *dmin_f, float4 *gm,
                              float2 *dxy_f, float2 *lsw_f, float2 *fxw_f, float2 *ilsw_f, float4 *igf,
                              int *n_fp64, cudaStream_t s)
{
    k_mixed_prep<<<(unsigned)((g.n + 127) / 128), 128, 0, s>>>(g, flag, nrm_f, dmin_f, gm, dxy_f, lsw_f, fxw_f,
                                                               ilsw_f, igf, n_fp64);
    return cudaGetLastError();
}

// --------------------------------------------------------------------------
// Edge layout of the mixed kernels: sliced ELL with slices of 32 points
// (SELL-32). One thread per point; a warp handles the 32 points of one slice,
// and slot s of all 32 points is stored contiguously at
// slice_off[slice] + 32 s + lane, so every per-edge load of a warp is one
// coalesced run. A slice is as deep as its largest degree; shorter rows stop
// early (on these clouds almost all points have 8 neighbours).
// --------------------------------------------------------------------------

// create time: scatter the CSR rows of the FP32 (and FP64-closure) edge arrays
// into the SELL-32 layout; padding slots keep weight 0 and index = the point
__global__ void __launch_bounds__(256) k_sell_fill(int64_t n, const int32_t *__restrict__ off,
                                                   const int32_t *__restrict__ slice_off,
                                                   const int32_t *__restrict__ idx,
                                                   const uint8_t *__restrict__ mask,
                                                   const float2 *__restrict__ dxy, const float2 *__restrict__ lsw,
                                                   const float2 *__restrict__ fxw, const double2 *__restrict__ fxw64,
                                                   int32_t *__restrict__ s_idx, float2 *__restrict__ s_ga,
                                                   float4 *__restrict__ s_gf, double2 *__restrict__ s_fxw64)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int64_t slice = p >> 5, lane = p & 31;
    const int depth = (slice_off[slice + 1] - slice_off[slice]) >> 5;
    const int e0 = off[p], deg = off[p + 1] - e0;
    for (int s = 0; s < depth; ++s) {
        const int64_t d = slice_off[slice] + 32 * s + lane;
        if (s < deg) {
            const int e = e0 + s;
            s_idx[d] = idx[e] | ((int32_t)mask[e] << 28);
            s_ga[d] = lsw[e];
            s_gf[d] = make_float4(dxy[e].x, dxy[e].y, fxw[e].x, fxw[e].y);
            s_fxw64[d] = fxw64[e];
        } else {
            s_idx[d] = (int32_t)p;
            s_ga[d] = make_float2(0.0f, 0.0f);
            s_gf[d] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            s_fxw64[d] = make_double2(0.0, 0.0);
        }
    }
}

cudaError_t launch_sell_fill(int64_t n, const int32_t *off, const int32_t *slice_off, const int32_t *idx,
                             const uint8_t *mask, const float2 *dxy, const float2 *lsw, const float2 *fxw,
                             const double2 *fxw64, const MixedGeom &m, cudaStream_t s)
{
    k_sell_fill<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(
        n, off, slice_off, idx, mask, dxy, lsw, fxw, fxw64, const_cast<int32_t *>(m.sidx),
        const_cast<float2 *>(m.ga), const_cast<float4 *>(m.gf), const_cast<double2 *>(m.fxw64));
    return cudaGetLastError();
}

// Kinetic boundary mode: the q carried by the image (entry e of the image
// CSR) of a neighbour P_i of P_0 (see image_q of the FP64 kernels), with
// d the image's offset: the reflection across the tangent line of P_i's own
// reconstruction q_i - d_i.grad q_i / 2 (d_i the reflection of d) when
// recon, else of q_i; the free stream qf for a far-field image.
__device__ __forceinline__ void image_q_f(const MixedGeom &g, int e, uint8_t m, float2 n0, const float *qf,
                                          const float *__restrict__ q, const float *__restrict__ qg, float2 d,
                                          bool recon, float qi[4])
{
    if (m & M_IMG_FAR) {
#pragma unroll
        for (int k = 0; k < 4; ++k) qi[k] = qf[k];
        return;
    }
    const int i = g.iidx[e];
    load4f(q, i, qi);
    if (recon) {
        reflect2(d.x, d.y, n0.x, n0.y);
        float gi[8];
        gather8f(qg, i, gi);
#pragma unroll
        for (int k = 0; k < 4; ++k) qi[k] = qi[k] - 0.5f * (d.x * gi[k] + d.y * gi[4 + k]);
    }
    reflect2(qi[1], qi[2], n0.x, n0.y);
}

// --------------------------------------------------------------------------
// q_derivatives() in FP32 (E15; the same passes as k_qgrad of the FP64 form)
// --------------------------------------------------------------------------
// KIN: the kinetic boundary mode (a separate instantiation keeps the plain
// kernels' registers as they are)
// PASS: bit 1 an inner iteration, G1 - sum_e a_e (d_e/2 . grad q_i) +
// grad q_0 / 2 with G1 = g1 the first pass's result (so no q_i is gathered);
// bit 0 the limiter at its end, phi = f(x_m, d_m) when x_m < 2 d_m, else 1
// (x_m = min(D+, -D-), d_m the largest |d_e/2 . grad q|: see k_qgrad); bit 2
// a first pass that stores x_m for a limited inner pass. One instantiation
// per kind of pass keeps each one's registers to what it uses.
template <int THREADS, int MINB, bool KIN, int PASS>
__global__ void __launch_bounds__(THREADS, MINB) k_qgrad_mixed(MixedGeom g, const float *__restrict__ q,
                                                               const float *__restrict__ qg_old,
                                                               const float *__restrict__ g1,
                                                               float *__restrict__ qg_new, float *__restrict__ ext,
                                                               float limK)
{
    constexpr bool INNER = (PASS & 2) != 0, LIMIT = (PASS & 1) != 0;
    constexpr bool EXTR = !INNER && (PASS & 5) != 0;   // extrema found in this pass
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= g.n) return;
    const int deg = g.off[p + 1] - g.off[p];
    const int64_t base = g.slice_off[p >> 5] + (p & 31);
    float sx[4], sy[4];
    // largest and smallest q_i - q_0 (P_0's own difference: 0)
    float dhi[4] = {0.0f, 0.0f, 0.0f, 0.0f}, dlo[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    // the slot's offset d = M a (a = M^-1 d): recovered from the weights, so
    // a slot carries 8 bytes of geometry instead of 16
    float4 M = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    if (INNER || LIMIT) M = g.gm[p];
    if constexpr (!INNER) {
        float q0[4];
        load4f(q, p, q0);
#pragma unroll
        for (int k = 0; k < 4; ++k) sx[k] = sy[k] = 0.0f;
        auto add = [&](const float qi[4], float2 a) {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float dq = qi[k] - q0[k];
                if constexpr (EXTR) {
                    dhi[k] = fmaxf(dhi[k], dq);
                    dlo[k] = fminf(dlo[k], dq);
                }
                sx[k] += a.x * dq;
                sy[k] += a.y * dq;
            }
        };
#pragma unroll 4
        for (int s = 0; s < deg; ++s) {
            const int64_t e = base + 32 * s;
            float qi[4];
            load4f(q, g.sidx[e] & kSlotIndexMask, qi);
            add(qi, g.ga[e]);
        }
        if constexpr (KIN) {
            // kinetic boundary mode: the mirror images of the neighbours
            const int f0 = g.ioff[p], f1 = g.ioff[p + 1];
            if (f0 < f1) {
                const float2 n0 = g.nrm[p];
                const float *qf = g.qinf + 4 * (g.pcase ? (int)g.pcase[p] : 0);
                for (int e = f0; e < f1; ++e) {
                    float qi[4];
                    image_q_f(g, e, g.imask[e], n0, qf, q, nullptr, make_float2(0.0f, 0.0f), false, qi);
                    add(qi, g.ilsw[e]);
                }
            }
        }
    } else {
        float t[8];
        load8f(g1, p, t);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            sx[k] = t[k];
            sy[k] = t[4 + k];
        }
        // neighbour indices are read two slots ahead, so that no gather of
        // the (2x unrolled) loop waits for the read of its own index (8 %
        // faster inner passes; the first pass, with its short gathers of q,
        // was 5 % slower that way and keeps the plain loop)
        int i0 = deg > 0 ? g.sidx[base] & kSlotIndexMask : 0;
        int i1 = deg > 1 ? g.sidx[base + 32] & kSlotIndexMask : 0;
#pragma unroll 2
        for (int s = 0; s < deg; ++s) {
            const int64_t e = base + 32 * s;
            const int i = i0;
            i0 = i1;
            if (s + 2 < deg) i1 = g.sidx[e + 64] & kSlotIndexMask;
            const float2 a = g.ga[e];
            const float2 d = make_float2(M.x * a.x + M.y * a.y, M.y * a.x + M.z * a.y);
            float gi[8];
            gather8f(qg_old, i, gi);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float c = 0.5f * (d.x * gi[k] + d.y * gi[4 + k]);
                sx[k] -= a.x * c;
                sy[k] -= a.y * c;
            }
        }
        if constexpr (KIN) {
            // a wall image's q~ is the reflection of q_i - d'.grad q_i / 2, d'
            // the reflection of the image's offset, so its correction is the
            // reflection of d'.grad q_i / 2; far-field images carry no gradient
            const int f0 = g.ioff[p], f1 = g.ioff[p + 1];
            if (f0 < f1) {
                const float2 n0 = g.nrm[p];
                for (int e = f0; e < f1; ++e) {
                    if (g.imask[e] & M_IMG_FAR) continue;
                    const float2 a = g.ilsw[e];
                    const float4 r = g.igf[e];
                    float2 d = make_float2(r.x, r.y);
                    reflect2(d.x, d.y, n0.x, n0.y);
                    float gi[8], c[4];
                    gather8f(qg_old, g.iidx[e], gi);
#pragma unroll
                    for (int k = 0; k < 4; ++k) c[k] = 0.5f * (d.x * gi[k] + d.y * gi[4 + k]);
                    reflect2(c[1], c[2], n0.x, n0.y);
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        sx[k] -= a.x * c[k];
                        sy[k] -= a.y * c[k];
                    }
                }
            }
        }
        // sum_e a_e (d_e . g_0) = g_0 (the weights satisfy sum_e a_e d_e^T = I,
        // to FP32 rounding), so the +1/2 d_e . g_0 of every corrected
        // difference (E14) adds up to g_0 / 2
        load8f(qg_old, p, t);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            sx[k] += 0.5f * t[k];
            sy[k] += 0.5f * t[4 + k];
        }
    }
    float xm[4];
    if constexpr (EXTR) {
#pragma unroll
        for (int k = 0; k < 4; ++k) xm[k] = fminf(dhi[k], -dlo[k]);
    }
    if constexpr (LIMIT) {
        if constexpr (INNER) load4f(ext, p, xm);
        float dmax[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        // the weights are read again (from L1); unrolled so that several
        // reads are in flight (a maximum does not depend on the order)
#pragma unroll 4
        for (int s = 0; s < deg; ++s) {
            const float2 a = g.ga[base + 32 * s];
            const float2 d = make_float2(M.x * a.x + M.y * a.y, M.y * a.x + M.z * a.y);
#pragma unroll
            for (int k = 0; k < 4; ++k) dmax[k] = fmaxf(dmax[k], fabsf(0.5f * (d.x * sx[k] + d.y * sy[k])));
        }
        if constexpr (KIN) {
            for (int e = g.ioff[p]; e < g.ioff[p + 1]; ++e) {
                const float4 r = g.igf[e];
#pragma unroll
                for (int k = 0; k < 4; ++k) dmax[k] = fmaxf(dmax[k], fabsf(0.5f * (r.x * sx[k] + r.y * sy[k])));
            }
        }
        const float h = g.dmin[p] * limK;
        const float eps2 = h * h * h;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            // f(x, d) = (x (x + 2d) + eps^2) / (x (x + d) + 2d^2 + eps^2)
            const float x = xm[k], d = dmax[k], d2 = 2.0f * d;
            const float num = fmaf(x, x + d2, eps2);
            const float den = fmaf(x, x + d, fmaf(d2, d, eps2));
            const float phi = x < d2 ? num / den : 1.0f;
            sx[k] *= phi;
            sy[k] *= phi;
        }
    } else if constexpr (EXTR) {
        store4f(ext, p, xm);
    }
    const float out[8] = {sx[0], sx[1], sx[2], sx[3], sy[0], sy[1], sy[2], sy[3]};
    store8f(qg_new, p, out);
}

// --------------------------------------------------------------------------
// flux_residual() + timestep() + state_update(), mixed. The neighbour loop
// runs in FP32; the state U stays FP64 and is updated by one FP64 add per
// component from an FP32 increment (U_k <- U_k - inc_k), the RK combination
// of the stage residuals being formed in FP32. FP64 <-> FP32 conversions go
// through the integer pipe.
// --------------------------------------------------------------------------
// the point's own q and grad q from its thread's slot of shared memory
// (three float4: q, grad q x, grad q y); volatile, so the compiler reads them
// where they are used instead of keeping them in registers across the loop,
// and ordered after the stores that filled the slot (memory clobber)
__device__ __forceinline__ void own_row(const float4 *slot, bool second, float q[4], float gq[8])
{
    const unsigned a = (unsigned)__cvta_generic_to_shared(slot);
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(q[0]), "=f"(q[1]), "=f"(q[2]), "=f"(q[3])
                 : "r"(a)
                 : "memory");
    if (second) {
        asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                     : "=f"(gq[0]), "=f"(gq[1]), "=f"(gq[2]), "=f"(gq[3])
                     : "r"(a + 16)
                     : "memory");
        asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                     : "=f"(gq[4]), "=f"(gq[5]), "=f"(gq[6]), "=f"(gq[7])
                     : "r"(a + 32)
                     : "memory");
    }
}

// a 16-byte copy from global to this thread's shared memory that bypasses
// the registers (cp.async; both addresses 16-byte aligned), grouped by
// commit and awaited by wait (this thread's own copies; the data is then
// visible to this thread)
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"((unsigned)__cvta_generic_to_shared(smem)),
                 "l"(gmem)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// PTX prefetch of the line holding a into L2 (a hint; a must be a valid
// global address)
__device__ __forceinline__ void prefetch_l2(const void *a)
{
    asm volatile("prefetch.global.L2 [%0];" ::"l"(a));
}

__device__ __forceinline__ void flag_nonphysical_m(int *status, int64_t p)
{
    atomicOr(status, STATUS_NONPHYSICAL);
    atomicMin(status + 1, (int)p);
}

// q~ of E14 at both ends of a slot as pairs (x: the neighbour, y: P_0):
// q - (d.grad q)/2 with d the slot's offset (order 2), else q; scalar
// arithmetic written straight into the pair registers
__device__ __forceinline__ void recon_pair(const float qi[4], const float gi[8], const float q0[4],
                                           const float g0[8], float2 d, bool second, float2 qt[4])
{
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (second) {
            qt[k].x = qi[k] - 0.5f * (d.x * gi[k] + d.y * gi[4 + k]);
            qt[k].y = q0[k] - 0.5f * (d.x * g0[k] + d.y * g0[4 + k]);
        } else {
            qt[k] = make_float2(qi[k], q0[k]);
        }
    }
}

// q and grad q of row r of a staged tile (shared memory)
__device__ __forceinline__ void row_f(const float4 *sq, const float4 *sg, int r, bool second, float q[4],
                                      float gq[8])
{
    const float4 a = sq[r];
    q[0] = a.x; q[1] = a.y; q[2] = a.z; q[3] = a.w;
    if (second) {
        const float4 b = sg[2 * r], c = sg[2 * r + 1];
        gq[0] = b.x; gq[1] = b.y; gq[2] = b.z; gq[3] = b.w;
        gq[4] = c.x; gq[5] = c.y; gq[6] = c.z; gq[7] = c.w;
    }
}

// One member's term of E11 in FP32 (the weights' FP64 copy w64[e] at points
// with an FP64 closure), frame (t, n) of P_0, R in the order [mass,
// s-momentum, n-momentum, energy]; see edge_residual of the FP64 kernels.
// Both ends are evaluated as one pair (packed FP32x2 arithmetic).
__device__ __forceinline__ void edge_residual_f(const float2 qt[4], uint32_t m, float2 w, bool fp64,
                                                const double2 *__restrict__ w64, int64_t e, float2 n0,
                                                float tx, float ty, float inv_gm1, int g14, float R[4],
                                                double R64[4], bool &ok)
{
    // equal reconstructed states have dG = 0 exactly; the two flux
    // evaluations may be compiled along different paths, so equality is
    // decided on q~, not on G
    if (qt[0].x == qt[0].y && qt[1].x == qt[1].y && qt[2].x == qt[2].y && qt[3].x == qt[3].y) return;
    PrimF2 s;
    ok &= prim_from_q_f2(qt, inv_gm1, g14, s);
    const float2 us = fma2(s.v, pr2(ty), mul2(s.u, pr2(tx)));
    const float2 un = fma2(s.v, pr2(n0.y), mul2(s.u, pr2(n0.x)));
    float dGs[4] = {0, 0, 0, 0}, dGn[4] = {0, 0, 0, 0};
    if (w.x != 0.0f) {
        const float sg = (m & M_XPOS) ? 1.0f : -1.0f;
        float2 G[4];
        split_flux_f2(sg, s, us, un, G);
#pragma unroll
        for (int k = 0; k < 4; ++k) dGs[k] = __fsub_rn(G[k].x, G[k].y);
    }
    if (w.y != 0.0f) {
        const float sg = (m & M_YPOS) ? 1.0f : -1.0f;
        float2 G[4];
        split_flux_f2(sg, s, un, us, G);
        // Gn components are [mass, n-momentum, s-momentum, energy]
        dGn[0] = __fsub_rn(G[0].x, G[0].y);
        dGn[1] = __fsub_rn(G[2].x, G[2].y);
        dGn[2] = __fsub_rn(G[1].x, G[1].y);
        dGn[3] = __fsub_rn(G[3].x, G[3].y);
    }
    if (fp64) {
        const double2 ww = w64[e];
#pragma unroll
        for (int k = 0; k < 4; ++k) R64[k] += ww.x * (double)dGs[k] + ww.y * (double)dGn[k];
    } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) R[k] += w.x * dGs[k] + w.y * dGn[k];
    }
}

// PF: software-pipelined neighbour loop (the next slot's record and
// neighbour values, and the index of the slot after it, are loaded while the
// current slot's fluxes are evaluated). In the plain boundary mode the
// neighbour values travel by cp.async into this thread's slot of shared
// memory and the point's own q and grad q wait there too, so that neither
// holds registers across the loop: 80 registers without spills, 24 resident
// warps per SM at 64 x 12 instead of 20 at 96 registers.
// STAGE: the CTA is one tile of kTile points. It first copies the q and
// grad q of its own points and of up to kHaloCap neighbours outside the tile
// (each once, the list made at create) into shared memory with independent
// loads, then runs the neighbour loop on those rows: no gathered value is
// read from global memory inside the loop, only the streamed slot records
// (a neighbour beyond the cap is read from global memory as before).
template <int THREADS, int MINB, bool PF, bool KIN, bool STAGE = false>
__global__ void __launch_bounds__(THREADS, MINB) k_flux_update_mixed(MixedFluxParams P)
{
    const MixedGeom &g = P.g;
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = p < g.n;
    const float4 *sq = nullptr, *sg = nullptr;
    if constexpr (STAGE) {
        static_assert(THREADS == kTile, "a staged CTA is one tile");
        __shared__ float4 s_q[kTile + kHaloCap];
        __shared__ float4 s_g[2 * (kTile + kHaloCap)];
        const int h0 = g.tile_off[blockIdx.x];
        const int nh = min(g.tile_off[blockIdx.x + 1] - h0, kHaloCap);
        const bool second = P.order == 2;
        for (int r = threadIdx.x; r < kTile + nh; r += kTile) {
            const int64_t i = r < kTile ? (int64_t)blockIdx.x * kTile + r : (int64_t)g.tile_idx[h0 + r - kTile];
            if (i < g.n) {
                s_q[r] = __ldg(reinterpret_cast<const float4 *>(P.q) + i);
                if (second) {
                    s_g[2 * r] = __ldg(reinterpret_cast<const float4 *>(P.qg) + 2 * i);
                    s_g[2 * r + 1] = __ldg(reinterpret_cast<const float4 *>(P.qg) + 2 * i + 1);
                }
            }
        }
        __syncthreads();
        sq = s_q;
        sg = s_g;
    }
    // pipelined plain-mode loop: the point's own row waits in shared memory
    // (this thread's slot) during the neighbour loop instead of in registers
    constexpr bool OWN_SMEM = PF && !STAGE && !KIN;
    __shared__ float4 s_own[OWN_SMEM ? 3 * THREADS : 1];
    // and the next slot's neighbour row is copied there too (cp.async, two
    // buffers: the one being read and the one being filled)
    __shared__ float4 s_nb[OWN_SMEM ? 2 * 3 * THREADS : 1];
    // the point's own loads are all issued before its flag is tested, so
    // that they are in flight together (far-field points read them in vain)
    uint8_t fl = FLAG_FARFIELD;
    int deg = 0;
    int64_t base = 0;
    float2 n0 = make_float2(0.0f, 0.0f);
    float q0[4] = {0.0f, 0.0f, 0.0f, 0.0f}, g0[8] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
    const bool second = P.order == 2;
    if (live) {
        fl = g.flag[p];
        deg = g.off[p + 1] - g.off[p];
        base = g.slice_off[p >> 5] + (p & 31);
        n0 = g.nrm[p];
        if constexpr (STAGE) {
            row_f(sq, sg, threadIdx.x, second, q0, g0);
        } else {
            load4f(P.q, p, q0);
            if (second) load8f(P.qg, p, g0);
        }
        if constexpr (OWN_SMEM) {
            s_own[3 * threadIdx.x] = make_float4(q0[0], q0[1], q0[2], q0[3]);
            s_own[3 * threadIdx.x + 1] = make_float4(g0[0], g0[1], g0[2], g0[3]);
            s_own[3 * threadIdx.x + 2] = make_float4(g0[4], g0[5], g0[6], g0[7]);
        }
        if (P.mode != 0) {
            // the state update's inputs are brought into L2 while the fluxes
            // are evaluated (a hint: no register waits for it)
            prefetch_l2(P.Un + 4 * p);
            if (P.mode == 2 && P.stage > 0) {
                prefetch_l2(P.dt + p);
                prefetch_l2(reinterpret_cast<const float *>(P.acc) + 4 * p);
            } else {
                prefetch_l2(g.dmin + p);
            }
        }
    }
    const uint8_t flag = fl & 3;
    const bool fp64 = (fl & FLAG_FP64_CLOSURE) != 0;
    float Rl[4] = {0.0f, 0.0f, 0.0f, 0.0f};  // residual, global frame
    double R64g[4] = {0.0, 0.0, 0.0, 0.0};   // FP64-closure points
    // far-field points are held at the free stream, except in the kinetic boundary mode
    if (live && (flag != FLAG_FARFIELD || KIN)) {
        const float tx = n0.y, ty = -n0.x;
        float R[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        double R64[4] = {0.0, 0.0, 0.0, 0.0};
        bool ok = true;
        float4 rec_n = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        int32_t im_n = 0, im_nn = 0;  // slot records one ahead, indices two ahead
        float q_n[4] = {0, 0, 0, 0}, g_n[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        if constexpr (STAGE) {
            // only the slot records are prefetched; the rows are in shared memory
            uint16_t sl_n = 0;
            if (deg > 0) {
                rec_n = g.gf[base];
                sl_n = g.sloc[base];
            }
            for (int s = 0; s < deg; ++s) {
                const int64_t e = base + 32 * s;
                const float4 rec = rec_n;
                const uint16_t sl = sl_n;
                if (s + 1 < deg) {
                    rec_n = g.gf[e + 32];
                    sl_n = g.sloc[e + 32];
                }
                const float2 w = make_float2(rec.z, rec.w);
                if (w.x == 0.0f && w.y == 0.0f) continue;
                const uint32_t m = (uint32_t)sl >> 12;
                const int row = sl & kSlotRowMask;
                float qi[4], gi[8];
                if (row != kSlotGlobal) {
                    row_f(sq, sg, row, second, qi, gi);
                } else {
                    const int i = g.sidx[e] & kSlotIndexMask;
                    load4f(P.q, i, qi);
                    if (second) gather8f(P.qg, i, gi);
                }
                float2 qt[4];
                recon_pair(qi, gi, q0, g0, make_float2(rec.x, rec.y), second, qt);
                edge_residual_f(qt, m, w, fp64, g.fxw64, e, n0, tx, ty, P.inv_gm1, P.g14, R, R64, ok);
            }
        } else if constexpr (OWN_SMEM) {
            if (deg > 0) {
                rec_n = g.gf[base];
                im_n = g.sidx[base];
                const int i = im_n & kSlotIndexMask;
                float4 *b = s_nb + 3 * threadIdx.x;
                cp_async16(b, reinterpret_cast<const float4 *>(P.q) + i);
                if (second) {
                    cp_async16(b + 1, reinterpret_cast<const float4 *>(P.qg) + 2 * i);
                    cp_async16(b + 2, reinterpret_cast<const float4 *>(P.qg) + 2 * i + 1);
                }
                cp_async_commit();
            }
            if (deg > 1) im_nn = g.sidx[base + 32];
        } else if constexpr (PF) {
            if (deg > 0) {
                rec_n = g.gf[base];
                im_n = g.sidx[base];
                const int i = im_n & kSlotIndexMask;
                load4f(P.q, i, q_n);
                if (second) gather8f(P.qg, i, g_n);
            }
            if (deg > 1) im_nn = g.sidx[base + 32];
        }
        if constexpr (!STAGE) for (int s = 0; s < deg; ++s) {
            const int64_t e = base + 32 * s;
            float2 qt[4];
            uint32_t m;
            float2 w, d;
            if constexpr (OWN_SMEM) {
                const float4 rec = rec_n;
                const int32_t im = im_n;
                // slot s's row has landed in buffer s & 1; slot s + 1's is
                // copied into the other buffer while slot s is evaluated
                cp_async_wait_all();
                float qi[4], gi[8];
                own_row(s_nb + 3 * (THREADS * (s & 1) + threadIdx.x), second, qi, gi);
                if (s + 1 < deg) {
                    rec_n = g.gf[e + 32];
                    im_n = im_nn;
                    const int in = im_n & kSlotIndexMask;
                    float4 *b = s_nb + 3 * (THREADS * ((s + 1) & 1) + threadIdx.x);
                    cp_async16(b, reinterpret_cast<const float4 *>(P.q) + in);
                    if (second) {
                        cp_async16(b + 1, reinterpret_cast<const float4 *>(P.qg) + 2 * in);
                        cp_async16(b + 2, reinterpret_cast<const float4 *>(P.qg) + 2 * in + 1);
                    }
                    cp_async_commit();
                    if (s + 2 < deg) im_nn = g.sidx[e + 64];
                }
                w = make_float2(rec.z, rec.w);
                if (w.x == 0.0f && w.y == 0.0f) continue;
                m = (uint32_t)im >> 28;
                d = make_float2(rec.x, rec.y);
                float q0s[4], g0s[8];
                own_row(s_own + 3 * threadIdx.x, second, q0s, g0s);
                recon_pair(qi, gi, q0s, g0s, d, second, qt);
            } else if constexpr (PF) {
                const float4 rec = rec_n;
                const int32_t im = im_n;
                float qi[4], gi[8];
#pragma unroll
                for (int k = 0; k < 4; ++k) qi[k] = q_n[k];
#pragma unroll
                for (int k = 0; k < 8; ++k) gi[k] = g_n[k];
                if (s + 1 < deg) {
                    // the gathers of slot s + 1 use an index read one
                    // iteration ago, so they issue without waiting for it
                    rec_n = g.gf[e + 32];
                    im_n = im_nn;
                    const int in = im_n & kSlotIndexMask;
                    load4f(P.q, in, q_n);
                    if (second) gather8f(P.qg, in, g_n);
                    if (s + 2 < deg) im_nn = g.sidx[e + 64];
                }
                w = make_float2(rec.z, rec.w);
                if (w.x == 0.0f && w.y == 0.0f) continue;
                m = (uint32_t)im >> 28;
                d = make_float2(rec.x, rec.y);
                recon_pair(qi, gi, q0, g0, d, second, qt);
            } else {
                const float4 rec = g.gf[e];
                w = make_float2(rec.z, rec.w);
                if (w.x == 0.0f && w.y == 0.0f) continue;
                const int32_t im = g.sidx[e];
                const int i = im & kSlotIndexMask;
                m = (uint32_t)im >> 28;
                float qi[4], gi[8];
                load4f(P.q, i, qi);
                if (second) gather8f(P.qg, i, gi);
                d = make_float2(rec.x, rec.y);
                recon_pair(qi, gi, q0, g0, d, second, qt);
            }
            edge_residual_f(qt, m, w, fp64, g.fxw64, e, n0, tx, ty, P.inv_gm1, P.g14, R, R64, ok);
        }
        if constexpr (KIN) {
            // kinetic boundary mode: the mirror images of the neighbours
            const int f0 = g.ioff[p], f1 = g.ioff[p + 1];
            const float *qf = g.qinf + 4 * (g.pcase ? (int)g.pcase[p] : 0);
            for (int e = f0; e < f1; ++e) {
                const float4 rec = g.igf[e];
                const float2 d = make_float2(rec.x, rec.y), w = make_float2(rec.z, rec.w);
                const uint8_t m = g.imask[e];
                float qti[4];
                image_q_f(g, e, m, n0, qf, P.q, P.qg, d, second, qti);
                float2 qt[4];
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    qt[k] = make_float2(qti[k], second ? q0[k] - 0.5f * (d.x * g0[k] + d.y * g0[4 + k]) : q0[k]);
                edge_residual_f(qt, m, w, fp64, g.ifxw64, e, n0, tx, ty, P.inv_gm1, P.g14, R, R64, ok);
            }
        }
        if (!ok) flag_nonphysical_m(P.status, p);
        if (fp64) {
            const double txd = (double)tx, tyd = (double)ty;
            R64g[0] = R64[0];
            R64g[1] = R64[1] * txd + R64[2] * (double)n0.x;
            R64g[2] = R64[1] * tyd + R64[2] * (double)n0.y;
            R64g[3] = R64[3];
#pragma unroll
            for (int k = 0; k < 4; ++k) Rl[k] = (float)R64g[k];
        } else {
            Rl[0] = R[0];
            Rl[1] = R[1] * tx + R[2] * n0.x;
            Rl[2] = R[1] * ty + R[2] * n0.y;
            Rl[3] = R[3];
        }
    }

    if (P.mode == 0) {
        if (live) {
            double Rd[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) Rd[k] = fp64 ? R64g[k] : f32_to_f64_ip(Rl[k]);
            store4(P.R, p, Rd);
        }
        return;
    }

    float r0sq = 0.0f;
    if (live) {
        double Un[4];
        float Unf[4];
        load4(P.Un, p, Un);
#pragma unroll
        for (int k = 0; k < 4; ++k) Unf[k] = f64_to_f32_ip(Un[k]);
        float dt;
        if (P.mode == 1 || P.stage == 0) {
            // timestep() in FP32: dt = CFL min|P_i - P_0| / (|u| + 3 sqrt(p/rho))
            const float ir = __fdividef(1.0f, Unf[0]);
            const float u = Unf[1] * ir, v = Unf[2] * ir;
            const float pr = (P.gamma - 1.0f) * (Unf[3] - 0.5f * (Unf[1] * u + Unf[2] * v));
            dt = P.cfl * g.dmin[p] / (sqrtf(u * u + v * v) + 3.0f * sqrtf(pr * ir));
            P.dt[p] = f32_to_f64_ip(dt);
        } else {
            dt = f64_to_f32_ip(P.dt[p]);
        }
        float *accf = reinterpret_cast<float *>(P.acc);
        float inc[4];  // U_new = U^n - inc
        if (P.mode == 1) {
#pragma unroll
            for (int k = 0; k < 4; ++k) inc[k] = dt * Rl[k];
        } else {
            float a[4] = {Rl[0], Rl[1], Rl[2], Rl[3]};
            if (P.stage > 0) {
                float o[4];
                load4f(accf, p, o);
                const float c = P.stage < 3 ? 2.0f : 1.0f;
#pragma unroll
                for (int k = 0; k < 4; ++k) a[k] = o[k] + c * Rl[k];
            }
            if (P.stage < 3) {
                store4f(accf, p, a);
                const float c = P.stage == 2 ? dt : 0.5f * dt;
#pragma unroll
                for (int k = 0; k < 4; ++k) inc[k] = c * Rl[k];
            } else {
                const float c = dt * (1.0f / 6.0f);
#pragma unroll
                for (int k = 0; k < 4; ++k) inc[k] = c * a[k];
            }
        }
        double Unew[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) Unew[k] = Un[k] - f32_to_f64_ip(inc[k]);
        if (flag == FLAG_WALL) {
            // remove the normal momentum (FP64, wall points only)
            const double2 n0 = P.nrm64[p];
            const double mn = Unew[1] * n0.x + Unew[2] * n0.y;
            Unew[1] = Unew[1] - mn * n0.x;
            Unew[2] = Unew[2] - mn * n0.y;
        } else if (flag == FLAG_FARFIELD && !KIN) {
            const double *Ui = P.case_uinf ? P.case_uinf + 4 * (int)P.pcase[p] : P.Uinf;
#pragma unroll
            for (int k = 0; k < 4; ++k) Unew[k] = Ui[k];
        }
        store4(P.Uout, p, Unew);
        float Uf[4], qn[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) Uf[k] = f64_to_f32_ip(Unew[k]);
        if (!q_from_Uf(Uf, P.gamma, P.inv_gm1, qn)) flag_nonphysical_m(P.status, p);
        store4f(P.qout, p, qn);
        r0sq = Rl[0] * Rl[0];
    }

    // residue partials, one pair per warp (FP32 within the warp): the points
    // of the warp's first case, and the rest (a second case that starts
    // inside the warp; every case has at least 32 points)
    if (P.mode == 1 || P.stage == 0) warp_residue_pair(P.pcase, p, live, r0sq, P.norm_part);
}

__global__ void __launch_bounds__(256) k_q_from_U_mixed(int64_t n, float gamma, float inv_gm1,
                                                        const double *__restrict__ U,
                                                        float *__restrict__ q, int *status)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    double u[4];
    float qq[4];
    load4(U, p, u);
    if (!q_from_U_f(u, gamma, inv_gm1, qq)) flag_nonphysical_m(status, p);
    store4f(q, p, qq);
}

__global__ void __launch_bounds__(256) k_grad_out_f(int64_t n, const int32_t *__restrict__ perm,
                                                    const float *__restrict__ qg, double *__restrict__ qx,
                                                    double *__restrict__ qy)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int64_t o = perm[p];
    float v[8];
    load8f(qg, p, v);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        qx[k * n + o] = (double)v[k];
        qy[k * n + o] = (double)v[4 + k];
    }
}

// launch-shape variants of the two hot kernels, chosen by the autotuner:
// (threads per block, minimum resident blocks per SM for the register cap)
template <int T, int M, bool KIN>
static cudaError_t qgrad_v(const MixedGeom &g, const float *q, const float *qg_old, const float *g1, float *qg_new,
                           float *ext, float limK, cudaStream_t s)
{
    const unsigned nb = (unsigned)((g.n + T - 1) / T);
    const bool inner = qg_old != nullptr, limit = limK > 0.0f;
    const int pass = inner ? (2 | (limit ? 1 : 0)) : limit ? 1 : ext ? 4 : 0;
    switch (pass) {
    case 0: k_qgrad_mixed<T, M, KIN, 0><<<nb, T, 0, s>>>(g, q, qg_old, g1, qg_new, ext, limK); break;
    case 1: k_qgrad_mixed<T, M, KIN, 1><<<nb, T, 0, s>>>(g, q, qg_old, g1, qg_new, ext, limK); break;
    case 2: k_qgrad_mixed<T, M, KIN, 2><<<nb, T, 0, s>>>(g, q, qg_old, g1, qg_new, ext, limK); break;
    case 4: k_qgrad_mixed<T, M, KIN, 4><<<nb, T, 0, s>>>(g, q, qg_old, g1, qg_new, ext, limK); break;
    default: k_qgrad_mixed<T, M, KIN, 3><<<nb, T, 0, s>>>(g, q, qg_old, g1, qg_new, ext, limK); break;
    }
    return cudaGetLastError();
}

template <int T, int M, bool PF, bool KIN, bool STAGE = false>
static cudaError_t flux_v(const MixedFluxParams &P, cudaStream_t s)
{
    if (STAGE && (!P.g.tile_off || !P.g.tile_idx || !P.g.sloc)) return cudaErrorInvalidValue;
    k_flux_update_mixed<T, M, PF, KIN, STAGE><<<(unsigned)((P.g.n + T - 1) / T), T, 0, s>>>(P);
    return cudaGetLastError();
}

using QgradFn = cudaError_t (*)(const MixedGeom &, const float *, const float *, const float *, float *, float *,
                                float, cudaStream_t);
using FluxFn = cudaError_t (*)(const MixedFluxParams &, cudaStream_t);

// [plain, kinetic boundary mode][variant]
template <bool K>
struct VariantTable {
    static constexpr QgradFn qgrad[] = {qgrad_v<128, 8, K>, qgrad_v<64, 16, K>, qgrad_v<256, 4, K>,
                                        qgrad_v<128, 6, K>, qgrad_v<256, 3, K>, qgrad_v<96, 10, K>};
    static constexpr FluxFn flux[] = {
        flux_v<128, 7, false, K>, flux_v<64, 14, false, K>, flux_v<256, 3, false, K>, flux_v<128, 6, false, K>,
        flux_v<128, 8, false, K>, flux_v<256, 4, false, K>, flux_v<128, 7, true, K>,  flux_v<64, 14, true, K>,
        flux_v<256, 3, true, K>,  flux_v<128, 6, true, K>,  flux_v<128, 8, true, K>,  flux_v<256, 4, true, K>,
        flux_v<128, 5, true, K>,  flux_v<128, 4, true, K>,  flux_v<64, 8, true, K>,   flux_v<96, 6, true, K>,
        flux_v<128, 3, true, K>,
        // staged tiles (one 64-point tile per CTA, rows in shared memory)
        flux_v<64, 14, true, K, true>, flux_v<64, 16, true, K, true>, flux_v<64, 12, true, K, true>,
        flux_v<64, 10, true, K, true>, flux_v<64, 8, true, K, true>,
        // the pipelined loop at 64 threads with the register budgets between
        // shapes 7 (spills) and 14
        flux_v<64, 12, true, K>, flux_v<64, 10, true, K>};
};
static const QgradFn *const kQgradVariants[2] = {VariantTable<false>::qgrad, VariantTable<true>::qgrad};
static const FluxFn *const kFluxVariants[2] = {VariantTable<false>::flux, VariantTable<true>::flux};
static constexpr int kNumQgradVariants = sizeof VariantTable<false>::qgrad / sizeof(QgradFn);
static constexpr int kNumFluxVariants = sizeof VariantTable<false>::flux / sizeof(FluxFn);
static const int kQgradShape[][2] = {{128, 8}, {64, 16}, {256, 4}, {128, 6}, {256, 3}, {96, 10}};
// flux shapes 6-11 repeat 0-5 with the software-pipelined neighbour loop,
// 12-16 and 22-23 give that loop more registers, 17-21 stage each tile's
// rows in shared memory
static const int kFluxShape[][2] = {{128, 7}, {64, 14}, {256, 3}, {128, 6}, {128, 8}, {256, 4},
                                    {128, 7}, {64, 14}, {256, 3}, {128, 6}, {128, 8}, {256, 4},
                                    {128, 5}, {128, 4}, {64, 8},  {96, 6},  {128, 3},
                                    {64, 14}, {64, 16}, {64, 12}, {64, 10}, {64, 8},
                                    {64, 12}, {64, 10}};
static_assert(sizeof kFluxShape / sizeof kFluxShape[0] == kNumFluxVariants, "one shape per flux variant");


int mixed_variants(int kernel_class)
{
    return kernel_class == 0 ? kNumFluxVariants : kNumQgradVariants;
}

void mixed_variant_shape(int kernel_class, int v, int *threads, int *min_blocks)
{
    const int(*t)[2] = kernel_class == 0 ? kFluxShape : kQgradShape;
    *threads = t[v][0];
    *min_blocks = t[v][1];
}

cudaError_t launch_qgrad_mixed(const MixedGeom &g, const float *q, const float *qg_old, const float *g1,
                               float *qg_new, float *ext, double limiter_K, cudaStream_t s, int variant)
{
    if (variant < 0 || variant >= kNumQgradVariants) return cudaErrorInvalidValue;
    if (qg_old && (!g1 || (limiter_K > 0.0 && !ext))) return cudaErrorInvalidValue;
    return kQgradVariants[g.ioff ? 1 : 0][variant](g, q, qg_old, g1, qg_new, ext, (float)limiter_K, s);
}

cudaError_t launch_flux_mixed(const MixedFluxParams &P, cudaStream_t s, int variant)
{
    if (variant < 0 || variant >= kNumFluxVariants) return cudaErrorInvalidValue;
    return kFluxVariants[P.g.ioff ? 1 : 0][variant](P, s);
}

cudaError_t launch_q_from_U_mixed(int64_t n, const Gas &gas, const double *U, float *q, int *status,
                                  cudaStream_t s)
{
    k_q_from_U_mixed<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, (float)gas.gamma, (float)gas.inv_gm1,
                                                                 U, q, status);
    return cudaGetLastError();
}

cudaError_t launch_grad_out_f(int64_t n, const int32_t *perm, const float *qg, double *qx, double *qy,
                              cudaStream_t s)
{
    k_grad_out_f<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, perm, qg, qx, qy);
    return cudaGetLastError();
}

}  // namespace lskum
