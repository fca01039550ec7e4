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

__global__ void __launch_bounds__(128) k_mixed_prep(int64_t n, const double2 *__restrict__ xy,
                                                    const double2 *__restrict__ nrm,
                                                    const double *__restrict__ dmin,
                                                    const int32_t *__restrict__ off,
                                                    const int32_t *__restrict__ idx,
                                                    const uint8_t *__restrict__ mask,
                                                    const double2 *__restrict__ lsw,
                                                    const double2 *__restrict__ fxw,
                                                    uint8_t *__restrict__ flag, float2 *__restrict__ nrm_f,
                                                    float *__restrict__ dmin_f, float2 *__restrict__ dxy_f,
                                                    float2 *__restrict__ lsw_f, float2 *__restrict__ fxw_f,
                                                    int *n_fp64)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const double2 P0 = xy[p];
    double amp[4] = {0.0, 0.0, 0.0, 0.0};
    for (int e = off[p]; e < off[p + 1]; ++e) {
        const double2 Pi = xy[idx[e]];
        const double dx = Pi.x - P0.x, dy = Pi.y - P0.y;
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
    nrm_f[p] = make_float2((float)n0.x, (float)n0.y);
    dmin_f[p] = (float)dmin[p];
    const double a = fmax(fmax(amp[0], amp[1]), fmax(amp[2], amp[3]));
    if (a > kAmpLimit) {
        flag[p] |= FLAG_FP64_CLOSURE;
        atomicAdd(n_fp64, 1);
    }
}

cudaError_t launch_mixed_prep(const DevGeom &g, const MixedGeom &m, uint8_t *flag, int *n_fp64,
                              cudaStream_t s)
{
    k_mixed_prep<<<(unsigned)((g.n + 127) / 128), 128, 0, s>>>(
        g.n, g.xy, g.nrm, g.dmin, g.off, g.idx, g.mask, g.lsw, g.fxw, flag,
        const_cast<float2 *>(m.nrm), const_cast<float *>(m.dmin), const_cast<float2 *>(m.dxy),
        const_cast<float2 *>(m.lsw), const_cast<float2 *>(m.fxw), n_fp64);
    return cudaGetLastError();
}

__device__ __forceinline__ float venkat_f(float D, float d, float eps2)
{
    return (D * D + eps2 + 2.0f * D * d) / (D * D + 2.0f * d * d + D * d + eps2);
}

// --------------------------------------------------------------------------
// q_derivatives() in FP32 (E15; same structure as k_qgrad)
// --------------------------------------------------------------------------
__global__ void __launch_bounds__(128) k_qgrad_mixed(MixedGeom g, const float *__restrict__ q,
                                                     const float *__restrict__ qg_old,
                                                     float *__restrict__ qg_new, float limK)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= g.n) return;
    float q0[4], g0[8], sx[4] = {0, 0, 0, 0}, sy[4] = {0, 0, 0, 0};
    load4f(q, p, q0);
    const bool inner = qg_old != nullptr;
    const bool limit = limK > 0.0f;
    if (inner) load8f(qg_old, p, g0);
    float qmax[4] = {q0[0], q0[1], q0[2], q0[3]}, qmin[4] = {q0[0], q0[1], q0[2], q0[3]};
    const int e0 = g.off[p], e1 = g.off[p + 1];
    for (int e = e0; e < e1; ++e) {
        const int i = g.idx[e];
        const float2 a = g.lsw[e];
        float qi[4];
        load4f(q, i, qi);
        float dq[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            dq[k] = qi[k] - q0[k];
            qmax[k] = fmaxf(qmax[k], qi[k]);
            qmin[k] = fminf(qmin[k], qi[k]);
        }
        if (inner) {
            float gi[8];
            load8f(qg_old, i, gi);
            const float2 d = g.dxy[e];
#pragma unroll
            for (int k = 0; k < 4; ++k)
                dq[k] = dq[k] - 0.5f * (d.x * (gi[k] - g0[k]) + d.y * (gi[4 + k] - g0[4 + k]));
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            sx[k] += a.x * dq[k];
            sy[k] += a.y * dq[k];
        }
    }
    if (limit) {
        float dmax[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        for (int e = e0; e < e1; ++e) {
            const float2 d = g.dxy[e];
#pragma unroll
            for (int k = 0; k < 4; ++k) dmax[k] = fmaxf(dmax[k], fabsf(0.5f * (d.x * sx[k] + d.y * sy[k])));
        }
        const float h = g.dmin[p] * limK;
        const float eps2 = h * h * h;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            float phi = 1.0f;
            if (dmax[k] > 0.0f) {
                phi = fminf(phi, venkat_f(qmax[k] - q0[k], dmax[k], eps2));
                phi = fminf(phi, venkat_f(qmin[k] - q0[k], -dmax[k], eps2));
            }
            sx[k] *= phi;
            sy[k] *= phi;
        }
    }
    float out[8] = {sx[0], sx[1], sx[2], sx[3], sy[0], sy[1], sy[2], sy[3]};
    store8f(qg_new, p, out);
}

// --------------------------------------------------------------------------
// flux_residual() + timestep() + state_update(), mixed: the neighbour loop in
// FP32, the update of U and the residue partials in FP64.
// --------------------------------------------------------------------------
__device__ __forceinline__ void flag_nonphysical_m(int *status, int64_t p)
{
    atomicOr(status, STATUS_NONPHYSICAL);
    atomicMin(status + 1, (int)p);
}

__global__ void __launch_bounds__(128) k_flux_update_mixed(MixedFluxParams P)
{
    const MixedGeom &g = P.g;
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double Rg[4] = {0.0, 0.0, 0.0, 0.0};
    const bool live = p < g.n;
    uint8_t fl = FLAG_FARFIELD;
    if (live) fl = g.flag[p];
    const uint8_t flag = fl & 3;
    if (live && flag != FLAG_FARFIELD) {
        const bool fp64 = (fl & FLAG_FP64_CLOSURE) != 0;
        const float2 n0 = g.nrm[p];
        const float tx = n0.y, ty = -n0.x;
        float q0[4], g0[8];
        load4f(P.q, p, q0);
        const bool second = P.order == 2;
        if (second) load8f(P.qg, p, g0);
        float R[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        double R64[4] = {0.0, 0.0, 0.0, 0.0};
        bool ok = true;
        const int e0 = g.off[p], e1 = g.off[p + 1];
        for (int e = e0; e < e1; ++e) {
            const float2 w = g.fxw[e];
            if (w.x == 0.0f && w.y == 0.0f) continue;
            const int i = g.idx[e];
            const uint8_t m = g.mask[e];
            float qti[4], qt0[4];
            load4f(P.q, i, qti);
#pragma unroll
            for (int k = 0; k < 4; ++k) qt0[k] = q0[k];
            if (second) {
                const float2 d = g.dxy[e];
                float gi[8];
                load8f(P.qg, i, gi);
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    qti[k] = qti[k] - 0.5f * (d.x * gi[k] + d.y * gi[4 + k]);
                    qt0[k] = qt0[k] - 0.5f * (d.x * g0[k] + d.y * g0[4 + k]);
                }
            }
            PrimF si, s0;
            ok &= prim_from_q_f(qti, P.inv_gm1, P.g14, si);
            ok &= prim_from_q_f(qt0, P.inv_gm1, P.g14, s0);
            const float us_i = si.u * tx + si.v * ty, un_i = si.u * n0.x + si.v * n0.y;
            const float us_0 = s0.u * tx + s0.v * ty, un_0 = s0.u * n0.x + s0.v * n0.y;
            const float rE_i = si.p * P.inv_gm1 + 0.5f * si.rho * (us_i * us_i + un_i * un_i);
            const float rE_0 = s0.p * P.inv_gm1 + 0.5f * s0.rho * (us_0 * us_0 + un_0 * un_0);
            float dGs[4] = {0, 0, 0, 0}, dGn[4] = {0, 0, 0, 0};
            if (w.x != 0.0f) {
                const float sg = (m & M_XPOS) ? 1.0f : -1.0f;
                float Gi[4], G0[4];
                split_flux_f(sg, si, us_i, un_i, rE_i, Gi);
                split_flux_f(sg, s0, us_0, un_0, rE_0, G0);
#pragma unroll
                for (int k = 0; k < 4; ++k) dGs[k] = __fsub_rn(Gi[k], G0[k]);
            }
            if (w.y != 0.0f) {
                const float sg = (m & M_YPOS) ? 1.0f : -1.0f;
                float Gi[4], G0[4];
                split_flux_f(sg, si, un_i, us_i, rE_i, Gi);
                split_flux_f(sg, s0, un_0, us_0, rE_0, G0);
                // Gn components are [mass, n-momentum, s-momentum, energy]
                dGn[0] = __fsub_rn(Gi[0], G0[0]);
                dGn[1] = __fsub_rn(Gi[2], G0[2]);
                dGn[2] = __fsub_rn(Gi[1], G0[1]);
                dGn[3] = __fsub_rn(Gi[3], G0[3]);
            }
            if (fp64) {
                const double2 w64 = g.fxw64[e];
#pragma unroll
                for (int k = 0; k < 4; ++k) R64[k] += w64.x * (double)dGs[k] + w64.y * (double)dGn[k];
            } else {
#pragma unroll
                for (int k = 0; k < 4; ++k) R[k] += w.x * dGs[k] + w.y * dGn[k];
            }
        }
        if (!ok) flag_nonphysical_m(P.status, p);
        if (!fp64) {
#pragma unroll
            for (int k = 0; k < 4; ++k) R64[k] = (double)R[k];
        }
        const double txd = (double)tx, tyd = (double)ty;
        Rg[0] = R64[0];
        Rg[1] = R64[1] * txd + R64[2] * (double)n0.x;
        Rg[2] = R64[1] * tyd + R64[2] * (double)n0.y;
        Rg[3] = R64[3];
    }

    if (P.mode == 0) {
        if (live) store4(P.R, p, Rg);
        return;
    }

    if (live) {
        double Un[4], Unew[4];
        load4(P.Un, p, Un);
        double dt;
        if (P.mode == 1 || P.stage == 0) {
            // timestep() in FP32: dt = CFL min|P_i - P_0| / (|u| + 3 sqrt(p/rho))
            const float rho = (float)Un[0], m1 = (float)Un[1], m2 = (float)Un[2], E = (float)Un[3];
            const float ir = __fdividef(1.0f, rho);
            const float u = m1 * ir, v = m2 * ir;
            const float pr = (P.gamma - 1.0f) * (E - 0.5f * (m1 * u + m2 * v));
            dt = (double)(P.cfl * g.dmin[p] / (sqrtf(u * u + v * v) + 3.0f * sqrtf(pr * ir)));
            P.dt[p] = dt;
        } else {
            dt = P.dt[p];
        }
        if (P.mode == 1) {
#pragma unroll
            for (int k = 0; k < 4; ++k) Unew[k] = Un[k] - dt * Rg[k];
        } else {
            double a[4];
            if (P.stage == 0) {
#pragma unroll
                for (int k = 0; k < 4; ++k) a[k] = Rg[k];
            } else {
                load4(P.acc, p, a);
                const double c = P.stage < 3 ? 2.0 : 1.0;
#pragma unroll
                for (int k = 0; k < 4; ++k) a[k] = a[k] + c * Rg[k];
            }
            if (P.stage < 3) {
                store4(P.acc, p, a);
                const double c = (P.stage == 2) ? dt : 0.5 * dt;
#pragma unroll
                for (int k = 0; k < 4; ++k) Unew[k] = Un[k] - c * Rg[k];
            } else {
                const double c = dt / 6.0;
#pragma unroll
                for (int k = 0; k < 4; ++k) Unew[k] = Un[k] - c * a[k];
            }
        }
        if (flag == FLAG_WALL) {
            const double2 n0 = P.nrm64[p];
            const double mn = Unew[1] * n0.x + Unew[2] * n0.y;
            Unew[1] = Unew[1] - mn * n0.x;
            Unew[2] = Unew[2] - mn * n0.y;
        } else if (flag == FLAG_FARFIELD) {
#pragma unroll
            for (int k = 0; k < 4; ++k) Unew[k] = P.Uinf[k];
        }
        store4(P.Uout, p, Unew);
        float qn[4];
        if (!q_from_U_f(Unew, P.gamma, P.inv_gm1, qn)) flag_nonphysical_m(P.status, p);
        store4f(P.qout, p, qn);
    }

    if (P.mode == 1 || P.stage == 0) {
        double s = Rg[0] * Rg[0];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        __shared__ double ws[4];
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        if (lane == 0) ws[wid] = s;
        __syncthreads();
        if (threadIdx.x == 0) P.norm_part[blockIdx.x] = (ws[0] + ws[1]) + (ws[2] + ws[3]);
    }
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

cudaError_t launch_qgrad_mixed(const MixedGeom &g, const float *q, const float *qg_old, float *qg_new,
                               double limiter_K, cudaStream_t s)
{
    k_qgrad_mixed<<<(unsigned)((g.n + 127) / 128), 128, 0, s>>>(g, q, qg_old, qg_new, (float)limiter_K);
    return cudaGetLastError();
}

cudaError_t launch_flux_mixed(const MixedFluxParams &P, cudaStream_t s)
{
    k_flux_update_mixed<<<(unsigned)((P.g.n + 127) / 128), 128, 0, s>>>(P);
    return cudaGetLastError();
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
