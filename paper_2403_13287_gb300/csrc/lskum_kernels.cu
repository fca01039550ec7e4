// Hot-path kernels of q-LSKUM (arXiv 2403.13287): q-derivatives (E14, E15),
// the fused flux residual + state update (E10-E12, E16 / RK4) and the
// reductions (residue, forces). One thread per point; the neighbour loop
// gathers q, q-derivatives and coordinates of the stencil.
#include "lskum_device.cuh"
#include "lskum_kernels.h"

namespace lskum {

// --------------------------------------------------------------------------
// q_derivatives(): one least-squares solve of E15 per point.
//   first order (qg_old == nullptr):  grad q_0 = sum_e a_e (q_i - q_0)
//   inner iteration (Jacobi):         dq~ = dq - 1/2 [dx (qx_i - qx_0) + dy (qy_i - qy_0)]
// with the previous iterate qg_old read at every point and the new one
// written to qg_new (no point reads what this pass writes).
// --------------------------------------------------------------------------
// 1/M for a positive normal M: the approximate reciprocal of PTX
// (rcp.approx.ftz.f64) refined by two steps of Newton's iteration for 1/M,
// r <- r + r (1 - M r), each of which squares the relative error; the
// limiter's phi needs no correctly rounded quotient, and the limited
// q-derivative parity tests hold it to far below 1e-12.
__device__ __forceinline__ double rcp_newton(double M)
{
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(M));
    double e = fma(-M, r, 1.0);
    r = fma(r, e, r);
    e = fma(-M, r, 1.0);
    return fma(r, e, r);
}

// Kinetic boundary mode: the q carried by the image (entry e of the image
// CSR) of a neighbour P_i of P_0, reconstructed (E14) with the image's half
// offset hs when recon: the reflection across the tangent line (normal n0)
// of P_i's own reconstruction q_i - h.grad q_i, h the reflection of hs
// (reflecting the gas reflects q1, q2 and every gradient, and the image of
// a field at the image of a point is the reflection of its value there);
// the free stream qf for a far-field image (zero gradient).
__device__ __forceinline__ void image_q(const DevGeom &g, int e, uint8_t m, double2 n0, const double *qf,
                                       const double *__restrict__ q, const double *__restrict__ qg, double2 hs,
                                       bool recon, double qi[4])
{
    if (m & M_IMG_FAR) {
#pragma unroll
        for (int k = 0; k < 4; ++k) qi[k] = qf[k];
        return;
    }
    const int i = g.iidx[e];
    load4(q, i, qi);
    if (recon) {
        double2 h = hs;
        reflect2(h.x, h.y, n0.x, n0.y);
        double gi[8];
        load8(qg, i, gi);
#pragma unroll
        for (int k = 0; k < 4; ++k) qi[k] = fma(-h.y, gi[4 + k], fma(-h.x, gi[k], qi[k]));
    }
    reflect2(qi[1], qi[2], n0.x, n0.y);
}

// Order-preserving integer image of a double (anything but NaN): its IEEE
// bits as a signed integer with the magnitude bits of negative values
// inverted, so that integer order is numeric order (-0 just below +0); the
// map is its own inverse. FP64 min/max issue at the FP64 rate on this part,
// 1/64 of the integer ALU rate, so the stencil extrema take this form.
__device__ __forceinline__ long long order_key(long long b) { return b ^ ((b >> 63) & 0x7fffffffffffffffLL); }

// Kinds of q-derivative pass (the template argument PASS): QG_INNER an inner
// iteration, QG_LIMIT the limiter applied at its end, QG_EXTREMA a first
// pass that also stores the limiter's extremum measure for a limited inner
// pass that follows.
enum { QG_LIMIT = 1, QG_INNER = 2, QG_EXTREMA = 4 };

// d_m = max_e |h_e . (sx, sy)| of each component, bit for bit the value of
// the plain FP64 loop over the edges, with FP64 products only on the edges
// that can hold the maximum. An FP32 pass bounds every edge's value: with
// a = hf_x sf and b = hf_y tf (h, sx, sy rounded to FP32), the FP32
// v = |a + b| lies within 4.01 u (|h_x sx| + |h_y sy|) of the FP64 |r_e|
// (u = 2^-24: the three roundings to FP32, the two products and the sum,
// each within u relative; r_e within 2^-52 of the exact value), and the
// margin c = 2^-20 (|a| + |b|) + 2^-120 exceeds that with room for the
// roundings of c, v - c and v + c (the absolute term covers FP32 underflow).
// So L = max_e fl(v - c) <= max_e |r_e|, and the edge holding the maximum
// has fl(v + c) >= L. A second FP32 pass marks the edges with
// !(fl(v + c) < L) (a NaN or an overflow marks the edge too); the marked
// edges (one bit each: at most LSKUM_MAX_DEGREE = 25) are then evaluated in
// FP64 exactly as the plain loop evaluates them.
__device__ __forceinline__ void largest_shift_screened(const DevGeom &g, int e0, int e1, const double sx[4],
                                                       const double sy[4], unsigned long long dm[4])
{
    constexpr float kMargin = 9.5367431640625e-07f;  // 2^-20 = 16 u
    constexpr float kTiny = 7.52316384526264e-37f;   // 2^-120
    float sf[4], tf[4], L[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        sf[k] = __double2float_rn(sx[k]);
        tf[k] = __double2float_rn(sy[k]);
        L[k] = 0.0f;
    }
    for (int e = e0; e < e1; ++e) {
        const float2 h = g.hd_f[e];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float a = h.x * sf[k], b = h.y * tf[k];
            const float c = fmaf(kMargin, fabsf(a) + fabsf(b), kTiny);
            L[k] = fmaxf(L[k], fabsf(a + b) - c);
        }
    }
    uint32_t cand[4] = {0u, 0u, 0u, 0u};
    for (int e = e0; e < e1; ++e) {
        const float2 h = g.hd_f[e];
        const uint32_t bit = 1u << (e - e0);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float a = h.x * sf[k], b = h.y * tf[k];
            const float c = fmaf(kMargin, fabsf(a) + fabsf(b), kTiny);
            if (!(fabsf(a + b) + c < L[k])) cand[k] |= bit;
        }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        uint32_t m = cand[k];
        while (m) {
            const int j = __ffs(m) - 1;
            m &= m - 1;
            const double2 h = g.hd[e0 + j];
            dm[k] = max(dm[k], abs_bits(fma(h.x, sx[k], h.y * sy[k])));
        }
    }
}

// One pass, by kind:
//   first:  G1 = sum_e a_e (q_i - q_0), the first-order solve;
//   inner:  G1 - sum_e a_e (h_e . grad q_i) + grad q_0 / 2, which is the sum
//           of a_e (q_i - q_0 - h_e . (grad q_i - grad q_0)) over the stencil
//           (h_e the half offset (P_i - P_0)/2): the weights a_e = M^-1 d_e,
//           M = sum_e d_e d_e^T, satisfy sum_e a_e d_e^T = I, so the terms in
//           grad q_0 add up to grad q_0 / 2, and the first-order part is the
//           stored G1 (g1) of the same state.
// The limiter scales each component of the result by Venkatakrishnan's
// phi = min over every reconstruction shift +-h_e.grad q of
// f(D, d) = (D^2 + eps^2 + 2Dd) / (D^2 + 2d^2 + Dd + eps^2), D the stencil
// maximum minus q_0 for a positive shift, the minimum minus q_0 for a
// negative one, eps^2 = (K min_e |P_i - P_0|)^3. With x = |D| and
// d = |shift|, f = N/M has N - M = d (x - 2d): f < 1 exactly when x < 2d;
// f increases in x up to x = 2d + sqrt(8d^2 + eps^2) > 2d and stays above 1
// beyond; and for fixed x < 2d it decreases in d. So phi is 1 unless
// x_m = min(D+, -D-) < 2 d_m, d_m the largest |h_e.grad q|, and then it is
// f(x_m, d_m): one quotient per component (a reciprocal and two Newton steps).
// KIN: the kinetic boundary mode (mirror images in g.ioff...; a separate
// instantiation keeps the plain kernel's registers as they are)
template <bool KIN, int PASS>
__global__ void __launch_bounds__(128) k_qgrad(DevGeom g, const double *__restrict__ q,
                                               const double *__restrict__ qg_old, const double *__restrict__ g1,
                                               double *__restrict__ qg_new, double *__restrict__ ext, double limK)
{
    constexpr bool INNER = (PASS & QG_INNER) != 0, LIMIT = (PASS & QG_LIMIT) != 0;
    constexpr bool EXTR = !INNER && (PASS & (QG_LIMIT | QG_EXTREMA)) != 0;   // extrema found here
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= g.n) return;
    double sx[4], sy[4];
    // order keys of the largest and smallest q_i - q_0 (P_0's own difference: +0)
    long long kmax[4] = {0, 0, 0, 0}, kmin[4] = {0, 0, 0, 0};
    const int e0 = g.off[p], e1 = g.off[p + 1];
    double2 xy0 = make_double2(0.0, 0.0);
    if ((INNER || LIMIT) && !g.hd) xy0 = g.xy[p];
    if constexpr (!INNER) {
        double q0[4];
        load4(q, p, q0);
#pragma unroll
        for (int k = 0; k < 4; ++k) sx[k] = sy[k] = 0.0;
        auto add = [&](const double qi[4], double2 a) {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const double dq = qi[k] - q0[k];
                if constexpr (EXTR) {
                    const long long key = order_key(__double_as_longlong(dq));
                    kmax[k] = max(kmax[k], key);
                    kmin[k] = min(kmin[k], key);
                }
                sx[k] = fma(a.x, dq, sx[k]);
                sy[k] = fma(a.y, dq, sy[k]);
            }
        };
        for (int e = e0; e < e1; ++e) {
            double qi[4];
            load4(q, g.idx[e], qi);
            add(qi, g.lsw[e]);
        }
        if constexpr (KIN) {
            // kinetic boundary mode: the mirror images of the neighbours
            const int f0 = g.ioff[p], f1 = g.ioff[p + 1];
            if (f0 < f1) {
                const double2 n0 = g.nrm[p];
                const double *qf = g.qinf + 4 * (g.pcase ? (int)g.pcase[p] : 0);
                for (int e = f0; e < f1; ++e) {
                    double qi[4];
                    image_q(g, e, g.imask[e], n0, qf, q, nullptr, make_double2(0.0, 0.0), false, qi);
                    add(qi, g.ilsw[e]);
                }
            }
        }
    } else {
        double t[8];
        load8(g1, p, t);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            sx[k] = t[k];
            sy[k] = t[4 + k];
        }
        for (int e = e0; e < e1; ++e) {
            const int i = g.idx[e];
            const double2 a = g.lsw[e];
            double2 h;
            if (g.hd) {
                h = g.hd[e];
            } else {
                const double2 xyi = g.xy[i];
                h = make_double2(0.5 * (xyi.x - xy0.x), 0.5 * (xyi.y - xy0.y));
            }
            double gi[8];
            load8(qg_old, i, gi);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const double c = fma(h.y, gi[4 + k], h.x * gi[k]);
                sx[k] = fma(-a.x, c, sx[k]);
                sy[k] = fma(-a.y, c, sy[k]);
            }
        }
        if constexpr (KIN) {
            // a wall image's q~ is the reflection of q_i - h.grad q_i, h the
            // reflection of the image's half offset, so its correction is the
            // reflection of h.grad q_i; far-field images carry no gradient
            const int f0 = g.ioff[p], f1 = g.ioff[p + 1];
            if (f0 < f1) {
                const double2 n0 = g.nrm[p];
                for (int e = f0; e < f1; ++e) {
                    if (g.imask[e] & M_IMG_FAR) continue;
                    const double2 a = g.ilsw[e];
                    double2 h = g.ihd[e];
                    reflect2(h.x, h.y, n0.x, n0.y);
                    double gi[8], c[4];
                    load8(qg_old, g.iidx[e], gi);
#pragma unroll
                    for (int k = 0; k < 4; ++k) c[k] = fma(-h.y, gi[4 + k], -h.x * gi[k]);
                    reflect2(c[1], c[2], n0.x, n0.y);
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        sx[k] = fma(a.x, c[k], sx[k]);
                        sy[k] = fma(a.y, c[k], sy[k]);
                    }
                }
            }
        }
        load8(qg_old, p, t);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            sx[k] = fma(0.5, t[k], sx[k]);
            sy[k] = fma(0.5, t[4 + k], sy[k]);
        }
    }
    // x_m = min(D+, -D-) per component
    double xm[4];
    if constexpr (EXTR) {
#pragma unroll
        for (int k = 0; k < 4; ++k)
            xm[k] = __longlong_as_double((long long)min((unsigned long long)kmax[k],
                                                        abs_bits(__longlong_as_double(order_key(kmin[k])))));
    }
    if constexpr (LIMIT) {
        if constexpr (INNER) load4(ext, p, xm);
        unsigned long long dm[4] = {0, 0, 0, 0};   // bits of d_m (non-negative doubles order as integers)
        if (g.hd_f && e1 - e0 <= 32) {
            largest_shift_screened(g, e0, e1, sx, sy, dm);
        } else {
            for (int e = e0; e < e1; ++e) {
                double2 h;
                if (g.hd) {
                    h = g.hd[e];
                } else {
                    const double2 xyi = g.xy[g.idx[e]];
                    h = make_double2(0.5 * (xyi.x - xy0.x), 0.5 * (xyi.y - xy0.y));
                }
#pragma unroll
                for (int k = 0; k < 4; ++k) dm[k] = max(dm[k], abs_bits(fma(h.x, sx[k], h.y * sy[k])));
            }
        }
        if constexpr (KIN) {
            for (int e = g.ioff[p]; e < g.ioff[p + 1]; ++e) {
                const double2 h = g.ihd[e];
#pragma unroll
                for (int k = 0; k < 4; ++k) dm[k] = max(dm[k], abs_bits(fma(h.x, sx[k], h.y * sy[k])));
            }
        }
        const double hK = g.dmin[p] * limK;
        const double eps2 = hK * hK * hK;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            // f(x, d) = N / M, N = x (x + 2d) + eps^2, M = x (x + d) + (2d^2 + eps^2),
            // evaluated for every component (warps diverge on x < 2d anyway)
            const double x = xm[k], d = __longlong_as_double((long long)dm[k]), d2 = 2.0 * d;
            const double N = fma(x, x + d2, eps2);
            const double M = fma(x, x + d, fma(d2, d, eps2));
            const double phi = x < d2 ? N * rcp_newton(M) : 1.0;
            sx[k] *= phi;
            sy[k] *= phi;
        }
    } else if constexpr (EXTR) {
        store4(ext, p, xm);
    }
    double out[8] = {sx[0], sx[1], sx[2], sx[3], sy[0], sy[1], sy[2], sy[3]};
    store8(qg_new, p, out);
}

// --------------------------------------------------------------------------
// flux_residual() + timestep() + state_update() (+ residue partials), fused.
// For each neighbour P_i of P_0 (frame t = (ny, -nx), n = (nx, ny)):
//   q~_i = q_i - 1/2 (dx qx_i + dy qy_i),  q~_0 = q_0 - 1/2 (dx qx_0 + dy qy_0)   (E14)
//   R += w_s [Gs(q~_i) - Gs(q~_0)] + w_n [Gn(q~_i) - Gn(q~_0)]                    (E11)
// where Gs is Gx+ or Gx- and Gn is Gy+ or Gy- by the edge's sub-stencil.
// --------------------------------------------------------------------------
struct FluxParams {
    DevGeom g;
    Gas gas;
    const double *q;    // [n][4] q of the state being evaluated
    const double *qg;   // [n][8] q-derivatives, or nullptr (first order)
    const double *Un;   // [n][4] U^n (update modes)
    double *Uout;       // [n][4] next stage state / U^{n+1}
    double *acc;        // [n][4] RK4 accumulator
    double *qout;       // [n][4] q of Uout
    double *dt;         // [n] local time step (computed at stage 0)
    double *R;          // [n][4] residual output (residual mode)
    double *norm_part;  // per warp: pair of R_rho^2 sums (stage 0), see warp_residue_pair
    int *status;        // [0] status bits, [1] smallest offending internal point
    const uint16_t *pcase;    // per point: its case in a batch, or nullptr (one case)
    const double *case_uinf;  // [cases][4] free stream per case, or nullptr (gas.Uinf)
    double cfl;
    int order;
    int mode;   // 0 residual only, 1 forward Euler, 2 RK4
    int stage;  // RK4 stage 0..3
};

__device__ __forceinline__ void flag_nonphysical(int *status, int64_t p)
{
    atomicOr(status, STATUS_NONPHYSICAL);
    atomicMin(status + 1, (int)p);
}

// One member's term of E11: w_s [Gs(q~_i) - Gs(q~_0)] + w_n [Gn(q~_i) - Gn(q~_0)],
// Gs = Gx+ or Gx- and Gn = Gy+ or Gy- by the member's sub-stencil bits m,
// in the frame (t, n) of P_0; R in the order [mass, s-momentum, n-momentum, energy].
__device__ __forceinline__ void edge_residual(const double qti[4], const double qt0[4], uint8_t m, double2 w,
                                              double2 n0, double tx, double ty, const Gas &gas, double R[4],
                                              bool &ok)
{
    // equal reconstructed states have dG = 0 exactly (compared as bit patterns,
    // on the integer pipe; +0 against -0 only costs a flux evaluation giving dG = 0)
    if (((__double_as_longlong(qti[0]) ^ __double_as_longlong(qt0[0])) |
         (__double_as_longlong(qti[1]) ^ __double_as_longlong(qt0[1])) |
         (__double_as_longlong(qti[2]) ^ __double_as_longlong(qt0[2])) |
         (__double_as_longlong(qti[3]) ^ __double_as_longlong(qt0[3]))) == 0)
        return;
    Prim si, s0;
    ok &= prim_from_q(qti, gas, tx, ty, n0, si);
    ok &= prim_from_q(qt0, gas, tx, ty, n0, s0);
    const double us_i = si.us, un_i = si.un, us_0 = s0.us, un_0 = s0.un;
    // w != 0 tested on the bits (integer pipe; +-0 are the zeros)
    if ((__double_as_longlong(w.x) & ~(long long)kSignBit) != 0) {
        const unsigned long long sg = (m & M_XPOS) ? 0ull : kSignBit;
        double Gi[4], G0[4];
        split_flux(sg, si, us_i, un_i, si.Ss, Gi);
        split_flux(sg, s0, us_0, un_0, s0.Ss, G0);
        // dG = G(q~_i) - G(q~_0) from the two rounded fluxes: an unfused
        // subtraction, so equal states give exactly zero (a contracted
        // fma(rho_i, m_i, -rho_0 m_0) would leave a product's rounding)
#pragma unroll
        for (int k = 0; k < 4; ++k) R[k] += w.x * __dsub_rn(Gi[k], G0[k]);
    }
    if ((__double_as_longlong(w.y) & ~(long long)kSignBit) != 0) {
        const unsigned long long sg = (m & M_YPOS) ? 0ull : kSignBit;
        double Gi[4], G0[4];
        split_flux(sg, si, un_i, us_i, si.Sn, Gi);
        split_flux(sg, s0, un_0, us_0, s0.Sn, G0);
        // Gn components are [mass, n-momentum, s-momentum, energy]
        R[0] += w.y * __dsub_rn(Gi[0], G0[0]);
        R[1] += w.y * __dsub_rn(Gi[2], G0[2]);
        R[2] += w.y * __dsub_rn(Gi[1], G0[1]);
        R[3] += w.y * __dsub_rn(Gi[3], G0[3]);
    }
}

template <bool KIN>
__global__ void __launch_bounds__(128) k_flux_update(FluxParams P)
{
    const DevGeom &g = P.g;
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double Rg[4] = {0.0, 0.0, 0.0, 0.0};
    const bool live = p < g.n;
    uint8_t flag = FLAG_FARFIELD;
    if (live) flag = g.flag[p] & 3;  // bit 7 marks FP64 closures in mixed contexts
    // far-field points are held at the free stream, except in the kinetic boundary mode
    if (live && (flag != FLAG_FARFIELD || KIN)) {
        const double2 xy0 = g.xy[p];
        const double2 n0 = g.nrm[p];
        const double tx = n0.y, ty = -n0.x;
        double q0[4], g0[8];
        load4(P.q, p, q0);
        const bool second = P.order == 2;
        if (second) load8(P.qg, p, g0);
        double R[4] = {0.0, 0.0, 0.0, 0.0};
        bool ok = true;
        const int e0 = g.off[p], e1 = g.off[p + 1];
        for (int e = e0; e < e1; ++e) {
            const double2 w = g.fxw[e];
            // weights outside every needed sub-stencil are +0 exactly: tested on the bits
            if ((__double_as_longlong(w.x) | __double_as_longlong(w.y)) == 0) continue;
            const int i = g.idx[e];
            const uint8_t m = g.mask[e];
            double qti[4], qt0[4];
            load4(P.q, i, qti);
#pragma unroll
            for (int k = 0; k < 4; ++k) qt0[k] = q0[k];
            if (second) {
                double2 h;
                if (g.hd) {
                    h = g.hd[e];
                } else {
                    const double2 xyi = g.xy[i];
                    h = make_double2(0.5 * (xyi.x - xy0.x), 0.5 * (xyi.y - xy0.y));
                }
                double gi[8];
                load8(P.qg, i, gi);
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    qti[k] = fma(-h.y, gi[4 + k], fma(-h.x, gi[k], qti[k]));
                    qt0[k] = fma(-h.y, g0[4 + k], fma(-h.x, g0[k], qt0[k]));
                }
            }
            edge_residual(qti, qt0, m, w, n0, tx, ty, P.gas, R, ok);
        }
        if constexpr (KIN) {
            // kinetic boundary mode: the mirror images of the neighbours
            const int f0 = g.ioff[p], f1 = g.ioff[p + 1];
            const double *qf = g.qinf + 4 * (g.pcase ? (int)g.pcase[p] : 0);
            for (int e = f0; e < f1; ++e) {
                const double2 w = g.ifxw[e];
                const uint8_t m = g.imask[e];
                const double2 hs = g.ihd[e];
                double qti[4], qt0[4];
                image_q(g, e, m, n0, qf, P.q, P.qg, hs, second, qti);
#pragma unroll
                for (int k = 0; k < 4; ++k) qt0[k] = second ? fma(-hs.y, g0[4 + k], fma(-hs.x, g0[k], q0[k])) : q0[k];
                edge_residual(qti, qt0, m, w, n0, tx, ty, P.gas, R, ok);
            }
        }
        if (!ok) flag_nonphysical(P.status, p);
        Rg[0] = R[0];
        Rg[1] = R[1] * tx + R[2] * n0.x;
        Rg[2] = R[1] * ty + R[2] * n0.y;
        Rg[3] = R[3];
    }

    if (P.mode == 0) {
        if (live) store4(P.R, p, Rg);
        return;
    }

    // ---- time step and state update ----
    if (live) {
        double Un[4], Unew[4];
        load4(P.Un, p, Un);
        double dt;
        if (P.mode == 1 || P.stage == 0) {
            // timestep(): dt = CFL min|P_i - P_0| / (|u| + 3 sqrt(p/rho))
            const double rho = Un[0], u = Un[1] / rho, v = Un[2] / rho;
            const double pr = (P.gas.gamma - 1.0) * (Un[3] - 0.5 * rho * (u * u + v * v));
            dt = P.cfl * g.dmin[p] / (sqrt(u * u + v * v) + 3.0 * sqrt(pr / rho));
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
                if (P.stage < 3) {
#pragma unroll
                    for (int k = 0; k < 4; ++k) a[k] = a[k] + 2.0 * Rg[k];
                } else {
#pragma unroll
                    for (int k = 0; k < 4; ++k) a[k] = a[k] + Rg[k];
                }
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
            const double2 n0 = g.nrm[p];
            const double mn = Unew[1] * n0.x + Unew[2] * n0.y;
            Unew[1] = Unew[1] - mn * n0.x;
            Unew[2] = Unew[2] - mn * n0.y;
        } else if (flag == FLAG_FARFIELD && !KIN) {
            const double *Ui = P.case_uinf ? P.case_uinf + 4 * (int)P.pcase[p] : P.gas.Uinf;
#pragma unroll
            for (int k = 0; k < 4; ++k) Unew[k] = Ui[k];
        }
        store4(P.Uout, p, Unew);
        double qn[4];
        if (!q_from_U(Unew, P.gas, qn)) flag_nonphysical(P.status, p);
        store4(P.qout, p, qn);
    }

    // ---- residue partials: a pair of R_rho^2 sums per warp, at stage 0 ----
    if (P.mode == 1 || P.stage == 0) warp_residue_pair(P.pcase, p, live, Rg[0] * Rg[0], P.norm_part);
}

// residue() of every case = sqrt(sum R_rho^2)/n_case from the per-warp
// pairs, in a fixed order. Case c owns points [start[c], start[c+1]); a warp
// whose first point lies in c contributes its first sum, a warp that starts
// in the case before contributes its second. Stage 1: block (j, c) sums
// chunk j (kResidueChunk warps) of case c; stage 2: one block sums each
// case's chunks and writes out[(*counter) * ncases + c], then advances the
// counter (so one captured iteration can be replayed), bounded by cap.
static constexpr int kResidueChunk = 2048;

__global__ void __launch_bounds__(256) k_residue_chunks(const double *__restrict__ part,
                                                        const int64_t *__restrict__ start, int maxchunks,
                                                        double *__restrict__ chunk)
{
    const int c = blockIdx.y, j = blockIdx.x;
    const int64_t p0 = start[c], p1 = start[c + 1];
    const int64_t w0 = p0 >> 5, w1 = (p1 - 1) >> 5;
    const int64_t a = w0 + (int64_t)j * kResidueChunk;
    const int64_t b = min(w1 + 1, a + kResidueChunk);
    double s = 0.0;
    for (int64_t w = a + threadIdx.x; w < b; w += blockDim.x) s += part[2 * w + ((w << 5) >= p0 ? 0 : 1)];
    __shared__ double sm[256];
    sm[threadIdx.x] = s;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if (threadIdx.x < h) sm[threadIdx.x] += sm[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) chunk[(int64_t)c * maxchunks + j] = sm[0];
}

__global__ void __launch_bounds__(256) k_residue_finish(const double *__restrict__ chunk,
                                                        const int64_t *__restrict__ start, int ncases, int maxchunks,
                                                        double *__restrict__ out_base, int *counter, int cap)
{
    __shared__ double sm[256];
    const int it = *counter;
    for (int c = 0; c < ncases; ++c) {
        const int64_t p0 = start[c], p1 = start[c + 1];
        const int64_t nw = ((p1 - 1) >> 5) - (p0 >> 5) + 1;
        const int nch = (int)((nw + kResidueChunk - 1) / kResidueChunk);
        double s = 0.0;
        for (int j = threadIdx.x; j < nch; j += blockDim.x) s += chunk[(int64_t)c * maxchunks + j];
        sm[threadIdx.x] = s;
        __syncthreads();
        for (int h = 128; h > 0; h >>= 1) {
            if (threadIdx.x < h) sm[threadIdx.x] += sm[threadIdx.x + h];
            __syncthreads();
        }
        if (threadIdx.x == 0 && it >= 0 && it < cap) out_base[(int64_t)it * ncases + c] = sqrt(sm[0]) / (double)(p1 - p0);
        __syncthreads();
    }
    if (threadIdx.x == 0) *counter = it + 1;
}

int residue_chunks(int64_t case_points) { return (int)((((case_points + 31) >> 5) + 1 + kResidueChunk - 1) / kResidueChunk); }

// q-variables of every point from U (used when a state is loaded)
__global__ void __launch_bounds__(256) k_q_from_U(int64_t n, Gas gas, const double *__restrict__ U,
                                                  double *__restrict__ q, int *status)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    double u[4], qq[4];
    load4(U, p, u);
    if (!q_from_U(u, gas, qq)) flag_nonphysical(status, p);
    store4(q, p, qq);
}

// timestep() alone: dt = CFL min|P_i - P_0| / (|u| + 3 sqrt(p/rho)) from U
__global__ void __launch_bounds__(256) k_timestep(int64_t n, Gas gas, double cfl,
                                                  const double *__restrict__ dmin,
                                                  const double *__restrict__ U, double *__restrict__ dt)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    double Un[4];
    load4(U, p, Un);
    const double rho = Un[0], u = Un[1] / rho, v = Un[2] / rho;
    const double pr = (gas.gamma - 1.0) * (Un[3] - 0.5 * rho * (u * u + v * v));
    dt[p] = cfl * dmin[p] / (sqrt(u * u + v * v) + 3.0 * sqrt(pr / rho));
}

// forces: per wall point (contour order) Cp and -Cp n ds; one block sums them
__global__ void __launch_bounds__(256) k_forces(int64_t nwall, Gas gas, double qinf,
                                                const int32_t *__restrict__ wall,
                                                const double *__restrict__ ds,
                                                const double2 *__restrict__ nrm,
                                                const double *__restrict__ U, double cosa, double sina,
                                                double *__restrict__ cp, double *__restrict__ clcd)
{
    __shared__ double sx[256], sy[256];
    double fx = 0.0, fy = 0.0;
    const double p_inf = 1.0 / gas.gamma;
    for (int64_t w = threadIdx.x; w < nwall; w += blockDim.x) {
        const int p = wall[w];
        double u[4];
        load4(U, p, u);
        const double rho = u[0], a = u[1] / rho, b = u[2] / rho;
        const double pr = (gas.gamma - 1.0) * (u[3] - 0.5 * rho * (a * a + b * b));
        const double c = (pr - p_inf) / qinf;
        cp[w] = c;
        const double2 n = nrm[p];
        fx -= c * n.x * ds[w];
        fy -= c * n.y * ds[w];
    }
    sx[threadIdx.x] = fx;
    sy[threadIdx.x] = fy;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            sx[threadIdx.x] += sx[threadIdx.x + w];
            sy[threadIdx.x] += sy[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        clcd[0] = sy[0] * cosa - sx[0] * sina;
        clcd[1] = sx[0] * cosa + sy[0] * sina;
    }
}

// ----------------------------------------------------------------------------
// launchers
// ----------------------------------------------------------------------------
static inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

template <bool KIN>
static void qgrad_pass(int pass, const DevGeom &g, const double *q, const double *qg_old, const double *g1,
                       double *qg_new, double *ext, double limK, cudaStream_t s)
{
    const unsigned nb = blocks_for(g.n, 128);
    switch (pass) {
    case 0: k_qgrad<KIN, 0><<<nb, 128, 0, s>>>(g, q, qg_old, g1, qg_new, ext, limK); break;
    case QG_EXTREMA: k_qgrad<KIN, QG_EXTREMA><<<nb, 128, 0, s>>>(g, q, qg_old, g1, qg_new, ext, limK); break;
    case QG_LIMIT: k_qgrad<KIN, QG_LIMIT><<<nb, 128, 0, s>>>(g, q, qg_old, g1, qg_new, ext, limK); break;
    case QG_INNER: k_qgrad<KIN, QG_INNER><<<nb, 128, 0, s>>>(g, q, qg_old, g1, qg_new, ext, limK); break;
    default: k_qgrad<KIN, QG_INNER | QG_LIMIT><<<nb, 128, 0, s>>>(g, q, qg_old, g1, qg_new, ext, limK); break;
    }
}

cudaError_t launch_qgrad(const DevGeom &g, const double *q, const double *qg_old, const double *g1,
                         double *qg_new, double *ext, double limiter_K, cudaStream_t s)
{
    const bool inner = qg_old != nullptr, limit = limiter_K > 0.0;
    if (inner && (!g1 || (limit && !ext))) return cudaErrorInvalidValue;
    const int pass = inner ? (QG_INNER | (limit ? QG_LIMIT : 0)) : limit ? QG_LIMIT : ext ? QG_EXTREMA : 0;
    if (g.ioff) qgrad_pass<true>(pass, g, q, qg_old, g1, qg_new, ext, limiter_K, s);
    else qgrad_pass<false>(pass, g, q, qg_old, g1, qg_new, ext, limiter_K, s);
    return cudaGetLastError();
}

int64_t residue_parts(int64_t n) { return 2 * ((n + 31) / 32); }

cudaError_t launch_flux(const DevGeom &g, const Gas &gas, const FluxLaunch &L, cudaStream_t s)
{
    FluxParams P;
    P.g = g;
    P.gas = gas;
    P.q = L.q; P.qg = L.qg; P.Un = L.Un; P.Uout = L.Uout; P.acc = L.acc; P.qout = L.qout;
    P.dt = L.dt; P.R = L.R; P.norm_part = L.norm_part; P.status = L.status;
    P.pcase = L.pcase; P.case_uinf = L.case_uinf;
    P.cfl = L.cfl; P.order = L.order; P.mode = L.mode; P.stage = L.stage;
    if (g.ioff) k_flux_update<true><<<blocks_for(g.n, 128), 128, 0, s>>>(P);
    else k_flux_update<false><<<blocks_for(g.n, 128), 128, 0, s>>>(P);
    return cudaGetLastError();
}

cudaError_t launch_residue_finish(const double *part, const int64_t *case_start, int ncases, int maxchunks,
                                  double *chunk, double *out_base, int *counter, int cap, cudaStream_t s)
{
    k_residue_chunks<<<dim3(maxchunks, ncases), 256, 0, s>>>(part, case_start, maxchunks, chunk);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    k_residue_finish<<<1, 256, 0, s>>>(chunk, case_start, ncases, maxchunks, out_base, counter, cap);
    return cudaGetLastError();
}

cudaError_t launch_q_from_U(int64_t n, const Gas &gas, const double *U, double *q, int *status,
                            cudaStream_t s)
{
    k_q_from_U<<<blocks_for(n, 256), 256, 0, s>>>(n, gas, U, q, status);
    return cudaGetLastError();
}

cudaError_t launch_timestep(int64_t n, const Gas &gas, double cfl, const double *dmin, const double *U,
                            double *dt, cudaStream_t s)
{
    k_timestep<<<blocks_for(n, 256), 256, 0, s>>>(n, gas, cfl, dmin, U, dt);
    return cudaGetLastError();
}

cudaError_t launch_forces(int64_t nwall, const Gas &gas, double qinf, const int32_t *wall,
                          const double *ds, const double2 *nrm, const double *U, double cosa,
                          double sina, double *cp, double *clcd, cudaStream_t s)
{
    k_forces<<<1, 256, 0, s>>>(nwall, gas, qinf, wall, ds, nrm, U, cosa, sina, cp, clcd);
    return cudaGetLastError();
}

}  // namespace lskum
