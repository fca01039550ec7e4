// Vector-Jacobian product of the q-LSKUM residual (E10 with E11, E13-E15):
// U_bar = (dR/dU)^T R_bar and (x_bar, y_bar) = (dR/dx, dR/dy)^T R_bar, in
// FP64, for the unlimited scheme of order 1 or 2.
//
// Reverse pass, every sum a gather (no atomics, bitwise reproducible):
//   flux      per point (owner of its edges): the transposed split-flux
//             Jacobians at both reconstructed states applied to the
//             cotangents (FP64: reverse mode through the regrouped split
//             fluxes; FP32: forward-mode duals, 4 tangents), giving
//             cotangents of the owner's q~_0, of each neighbour's q~_i (kept
//             per edge) and of the sub-stencil weights;
//   gather    per point over its incoming edges (transpose CSR): the
//             neighbour-side cotangents;
//   gradient  the K+1 least-squares passes of E15 in reverse (saved forward
//             iterates), each pass one kernel with an outgoing-edge loop
//             (owner terms, weight and offset cotangents) and an incoming-
//             edge loop (neighbour terms);
//   geometry  least-squares weight cotangents back to edge offsets
//             (a = M^-1 d with M = sum d d^T gives d_bar_k = b_k - B d_k,
//             b = M^-1 a_bar, B = sum (b a^T + a b^T)), then offsets to
//             points by one more gather;
//   state     q_bar to U_bar through the E13 Jacobian.
#include <cub/cub.cuh>
#include <type_traits>

#include "lskum_adjoint.h"

namespace lskum {

namespace {

// ---------------------------------------------------------------------------
// forward-mode dual number with four tangents, over T (double, or float for
// the FP32 product)
// ---------------------------------------------------------------------------
template <class T>
struct D4T {
    T v, d[4];
};
using D4 = D4T<double>;

// elementary functions: in FP64 the forward kernels' own forms (the
// table-driven exp, and erf(S) with exp(-S^2) from one Taylor-table row),
// in FP32 the library's
[[maybe_unused]] __device__ __forceinline__ double m_exp(double x) { return exp_tab(x); }
__device__ __forceinline__ float m_exp(float x) { return expf(x); }
__device__ __forceinline__ double m_log(double x) { return log(x); }
__device__ __forceinline__ float m_log(float x) { return logf(x); }
__device__ __forceinline__ double m_sqrt(double x) { return sqrt(x); }
[[maybe_unused]] __device__ __forceinline__ float m_sqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double m_rsqrt(double x) { return rsqrt(x); }
__device__ __forceinline__ float m_rsqrt(float x) { return rsqrtf(x); }
__device__ __forceinline__ void m_erf_gauss(double S, double &erfS, double &e) { erf_exp(S, erfS, e); }
__device__ __forceinline__ void m_erf_gauss(float S, float &erfS, float &e)
{
    erfS = erff(S);
    e = expf(-S * S);
}

template <class T>
__device__ __forceinline__ D4T<T> dconst(T v)
{
    D4T<T> r;
    r.v = v;
#pragma unroll
    for (int k = 0; k < 4; ++k) r.d[k] = T(0);
    return r;
}
template <class T>
__device__ __forceinline__ D4T<T> operator+(const D4T<T> &a, const D4T<T> &b)
{
    D4T<T> r;
    r.v = a.v + b.v;
#pragma unroll
    for (int k = 0; k < 4; ++k) r.d[k] = a.d[k] + b.d[k];
    return r;
}
template <class T>
__device__ __forceinline__ D4T<T> operator-(const D4T<T> &a, const D4T<T> &b)
{
    D4T<T> r;
    r.v = a.v - b.v;
#pragma unroll
    for (int k = 0; k < 4; ++k) r.d[k] = a.d[k] - b.d[k];
    return r;
}
template <class T>
__device__ __forceinline__ D4T<T> operator*(const D4T<T> &a, const D4T<T> &b)
{
    D4T<T> r;
    r.v = a.v * b.v;
#pragma unroll
    for (int k = 0; k < 4; ++k) r.d[k] = a.d[k] * b.v + a.v * b.d[k];
    return r;
}
template <class T>
__device__ __forceinline__ D4T<T> operator*(T s, const D4T<T> &a)
{
    D4T<T> r;
    r.v = s * a.v;
#pragma unroll
    for (int k = 0; k < 4; ++k) r.d[k] = s * a.d[k];
    return r;
}
template <class T>
__device__ __forceinline__ D4T<T> operator+(T s, const D4T<T> &a)
{
    D4T<T> r = a;
    r.v = s + a.v;
    return r;
}
// f(a) with f(a.v) = fv and f'(a.v) = df
template <class T>
__device__ __forceinline__ D4T<T> chain(const D4T<T> &a, T fv, T df)
{
    D4T<T> r;
    r.v = fv;
#pragma unroll
    for (int k = 0; k < 4; ++k) r.d[k] = df * a.d[k];
    return r;
}
template <class T>
__device__ __forceinline__ D4T<T> recip(const D4T<T> &a)
{
    const T r = T(1) / a.v;
    return chain(a, r, -r * r);
}
template <class T>
__device__ __forceinline__ D4T<T> dexp(const D4T<T> &a)
{
    const T e = m_exp(a.v);
    return chain(a, e, e);
}
template <class T>
__device__ __forceinline__ D4T<T> dlog(const D4T<T> &a)
{
    return chain(a, m_log(a.v), T(1) / a.v);
}
template <class T>
__device__ __forceinline__ D4T<T> dsqrt(const D4T<T> &a)
{
    const T s = m_sqrt(a.v);
    return chain(a, s, T(0.5) / s);
}

// The dual-number forms below serve the FP32 product; the FP64 product runs
// state_adjoint_rev (reverse mode through the forward kernels' regrouped
// split fluxes).
template <class T>
struct PrimDT {
    D4T<T> rho, u, v, p, sqb, rsb;
};

// inverse of E13 over duals: beta = -q4/2, u = -q2/q4, v = -q3/q4,
// rho = exp(q1 + beta |u|^2) beta^(-1/(gamma-1)), p = rho/(2 beta). From
// rsb = 1/sqrt(beta) and ib = 1/beta as the forward kernels form them:
// 1/q4 = -ib/2 (derivative -ib^2/4), sqrt(beta) = beta rsb (rsb/2),
// 1/sqrt(beta) (-rsb ib/2), and for gamma = 1.4 beta^-2.5 = rsb ib^2
// (-2.5 rsb ib^3) in place of exp(-2.5 ln beta)
template <class T>
__device__ __forceinline__ PrimDT<T> prim_d(const D4T<T> qt[4], T inv_gm1, bool g14)
{
    PrimDT<T> s;
    const D4T<T> beta = T(-0.5) * qt[3];
    const T rsb = m_rsqrt(beta.v), ib = rsb * rsb;
    const D4T<T> r = chain(qt[3], T(-0.5) * ib, T(-0.25) * ib * ib);
    s.u = T(-1) * (qt[1] * r);
    s.v = T(-1) * (qt[2] * r);
    s.sqb = chain(beta, beta.v * rsb, T(0.5) * rsb);
    s.rsb = chain(beta, rsb, T(-0.5) * rsb * ib);
    const D4T<T> ke = beta * (s.u * s.u + s.v * s.v);
    if (g14) {
        const T b25 = rsb * ib * ib;
        s.rho = dexp(qt[0] + ke) * chain(beta, b25, T(-2.5) * b25 * ib);
    } else {
        s.rho = dexp(qt[0] - inv_gm1 * dlog(beta) + ke);
    }
    s.p = T(-1) * (s.rho * r);
    return s;
}

// split flux along a direction over duals, in the paper's form
template <class T>
__device__ __forceinline__ void split_flux_d(T sgn, const PrimDT<T> &s, const D4T<T> &un, const D4T<T> &ut,
                                             T inv_gm1, D4T<T> G[4])
{
    const D4T<T> S = un * s.sqb;
    T erfv, e;
    m_erf_gauss(S.v, erfv, e);
    const D4T<T> erfS = chain(S, erfv, T(1.1283791670955126) * e);         // 2/sqrt(pi)
    const D4T<T> eS = chain(S, e, T(-2) * S.v * e);
    const D4T<T> A = T(0.5) * (T(1) + sgn * erfS);
    const D4T<T> B = T(0.28209479177387814) * (eS * s.rsb);                 // 1/(2 sqrt(pi))
    const D4T<T> rhoE = inv_gm1 * s.p + T(0.5) * (s.rho * (un * un + ut * ut));
    const D4T<T> m = un * A + sgn * B;
    G[0] = s.rho * m;
    G[1] = (s.p + s.rho * un * un) * A + sgn * (s.rho * un * B);
    G[2] = s.rho * ut * m;
    G[3] = (rhoE + s.p) * un * A + sgn * ((rhoE + T(0.5) * s.p) * B);
}

__device__ __forceinline__ void ld4(const double *a, int64_t p, double v[4])
{
    const double2 *a2 = reinterpret_cast<const double2 *>(a);
    const double2 lo = a2[2 * p], hi = a2[2 * p + 1];
    v[0] = lo.x; v[1] = lo.y; v[2] = hi.x; v[3] = hi.y;
}
__device__ __forceinline__ void st4(double *a, int64_t p, const double v[4])
{
    double2 *a2 = reinterpret_cast<double2 *>(a);
    a2[2 * p] = make_double2(v[0], v[1]);
    a2[2 * p + 1] = make_double2(v[2], v[3]);
}
__device__ __forceinline__ void ld8(const double *a, int64_t p, double v[8])
{
    ld4(a, 2 * p, v);
    ld4(a, 2 * p + 1, v + 4);
}
__device__ __forceinline__ void st8(double *a, int64_t p, const double v[8])
{
    st4(a, 2 * p, v);
    st4(a, 2 * p + 1, v + 4);
}
__device__ __forceinline__ void ld4(const float *a, int64_t p, float v[4])
{
    const float4 t = reinterpret_cast<const float4 *>(a)[p];
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
__device__ __forceinline__ void st4(float *a, int64_t p, const float v[4])
{
    reinterpret_cast<float4 *>(a)[p] = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void ld8(const float *a, int64_t p, float v[8])
{
    ld4(a, 2 * p, v);
    ld4(a, 2 * p + 1, v + 4);
}
__device__ __forceinline__ void st8(float *a, int64_t p, const float v[8])
{
    st4(a, 2 * p, v);
    st4(a, 2 * p + 1, v + 4);
}

// sub-stencil slots of an edge: x-sub (0 x+, 1 x-) and y-sub (2 y+, 3 y-), -1 if none
__device__ __forceinline__ int xsub(uint8_t m) { return (m & M_XPOS) ? 0 : ((m & M_XNEG) ? 1 : -1); }
__device__ __forceinline__ int ysub(uint8_t m) { return (m & M_YPOS) ? 2 : ((m & M_YNEG) ? 3 : -1); }
__device__ __forceinline__ bool sub_needed(uint8_t f, int k)
{
    return k >= 0 && (f == FLAG_INTERIOR || (f == FLAG_WALL && k != 2));
}

// cotangent of one reconstructed state: sum over the split fluxes it feeds,
// cs (frame order) against Gs and cn (frame order) against Gn, plus the
// flux values for the weight cotangents

template <class T>
__device__ __forceinline__ void state_adjoint(const T qt[4], T tx, T ty, T nx, T ny, bool use_s, T sg_s, bool use_n,
                                              T sg_n, const T cs[4], const T cn[4], T inv_gm1, bool g14, T qbar[4],
                                              T Gs[4], T Gn[4])
{
    D4T<T> q[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        q[k] = dconst(qt[k]);
        q[k].d[k] = T(1);
    }
    const PrimDT<T> s = prim_d(q, inv_gm1, g14);
    const D4T<T> us = tx * s.u + ty * s.v;
    const D4T<T> un = nx * s.u + ny * s.v;
#pragma unroll
    for (int k = 0; k < 4; ++k) qbar[k] = T(0);
    if (use_s) {
        D4T<T> G[4];
        split_flux_d(sg_s, s, us, un, inv_gm1, G);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            Gs[c] = G[c].v;
#pragma unroll
            for (int k = 0; k < 4; ++k) qbar[k] += cs[c] * G[c].d[k];
        }
    }
    if (use_n) {
        D4T<T> G[4];
        split_flux_d(sg_n, s, un, us, inv_gm1, G);
        // Gn components are [mass, n-momentum, s-momentum, energy]
        const int fr[4] = {0, 2, 1, 3};
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            Gn[fr[c]] = G[c].v;
#pragma unroll
            for (int k = 0; k < 4; ++k) qbar[k] += cn[fr[c]] * G[c].d[k];
        }
    }
}

// FP64 form of state_adjoint in reverse mode: the split fluxes in the forward
// kernels' regrouped form once, then their adjoint, so that
// q_bar = sum over the needed directions of (dG/dq~)^T c without forming the
// Jacobians. Primal, with (u_d, u_t) = (u.t, u.n) for the s direction and
// (u.n, u.t) for the n direction:
//   beta = -q4/2, r = beta^-1/2, hib = r^2/2 (= p/rho), u.t = (q2 tx + q3 ty) hib,
//   sqb = beta r, w2 = |u|^2, rho/2 = exp(q1 + beta w2)/2 beta^(-1/(gamma-1)),
//   h = (1/(gamma-1) + 1) hib + w2/2, qb = hib/2, rrc = (rho/2) r/sqrt(pi);
//   S = u_d sqb, fe = sgn erf S, Q = rho/2 (1 + fe), W = sgn rrc exp(-S^2),
//   G0 = u_d Q + W, G1 = u_d G0 + Q hib, G2 = u_t G0, G3 = h G0 - qb W.
__device__ __forceinline__ void state_adjoint_rev(const double qt[4], double tx, double ty, double nx, double ny,
                                                  bool use_s, double sg_s, bool use_n, double sg_n,
                                                  const double cs[4], const double cn[4], double inv_gm1, bool g14,
                                                  double qbar[4], double Gs[4], double Gn[4])
{
    const double beta = -0.5 * qt[3];
    const double rsb = m_rsqrt(beta), ib = rsb * rsb, hib = 0.5 * ib;
    const double qs = qt[1] * tx + qt[2] * ty, qn = qt[1] * nx + qt[2] * ny;
    const double us = qs * hib, un = qn * hib;
    const double sqb = beta * rsb;
    const double w2 = us * us + un * un;
    double hrho, fb = 1.0;   // fb = beta^-2.5 for gamma = 1.4
    if (g14) {
        fb = rsb * (ib * ib);
        hrho = exp_tab(qt[0] + beta * w2, -1) * fb;
    } else {
        hrho = exp_tab(qt[0] + beta * w2 - inv_gm1 * m_log(beta), -1);
    }
    const double h = (inv_gm1 + 1.0) * hib + 0.5 * w2;
    const double qb = 0.5 * hib;
    const double rrc = hrho * rsb * 0.5641895835477563;   // 1/sqrt(pi)
    double b_us = 0.0, b_un = 0.0, b_sqb = 0.0, b_hrho = 0.0, b_hib = 0.0, b_rrc = 0.0, b_h = 0.0, b_qb = 0.0;
    // one direction: primal G (in the direction's order) and its adjoint for cotangent c
    auto dir = [&](double ud, double ut, double sg, const double c[4], double G[4], double &b_ud, double &b_ut) {
        const double S = ud * sqb;
        double erfv, e;
        m_erf_gauss(S, erfv, e);
        const double fe = sg * erfv;
        const double Q = hrho + hrho * fe;
        const double W = sg * e * rrc;
        const double G0 = ud * Q + W;
        G[0] = G0;
        G[1] = ud * G0 + Q * hib;
        G[2] = ut * G0;
        G[3] = h * G0 - qb * W;
        const double bG0 = c[0] + c[1] * ud + c[2] * ut + c[3] * h;
        b_h += c[3] * G0;
        b_qb -= c[3] * W;
        b_ut += c[2] * G0;
        b_hib += c[1] * Q;
        const double bQ = c[1] * hib + bG0 * ud;
        const double bW = bG0 - c[3] * qb;
        b_ud += c[1] * G0 + bG0 * Q;
        b_rrc += bW * sg * e;
        b_hrho += bQ * (1.0 + fe);
        // fe = sgn erf S (erf' = 2/sqrt(pi) e), e = exp(-S^2) (e' = -2 S e)
        const double bS = (bQ * hrho * sg * 1.1283791670955126 - bW * sg * rrc * 2.0 * S) * e;
        b_ud += bS * sqb;
        b_sqb += bS * ud;
    };
    if (use_s) dir(us, un, sg_s, cs, Gs, b_us, b_un);
    if (use_n) {
        const double c[4] = {cn[0], cn[2], cn[1], cn[3]};   // Gn is [mass, n-momentum, s-momentum, energy]
        double G[4];
        dir(un, us, sg_n, c, G, b_un, b_us);
        Gn[0] = G[0];
        Gn[1] = G[2];
        Gn[2] = G[1];
        Gn[3] = G[3];
    }
    // per-state factors, in reverse
    b_hrho += b_rrc * rsb * 0.5641895835477563;
    double b_rsb = b_rrc * hrho * 0.5641895835477563;
    b_hib += 0.5 * b_qb + (inv_gm1 + 1.0) * b_h;
    double b_w2 = 0.5 * b_h;
    const double bx = b_hrho * hrho;   // d(rho/2)/dx = rho/2 for the exponent's argument x
    double b_beta = bx * w2;
    if (g14) b_beta += bx * (-2.5 * ib);   // beta^-2.5: relative derivative -2.5/beta
    else b_beta -= bx * inv_gm1 * ib;      // -ln(beta)/(gamma-1)
    b_w2 += bx * beta;
    b_us += 2.0 * us * b_w2;
    b_un += 2.0 * un * b_w2;
    b_beta += b_sqb * rsb;
    b_rsb += b_sqb * beta;
    const double b_qs = b_us * hib, b_qn = b_un * hib;
    b_hib += b_us * qs + b_un * qn;
    b_rsb += b_hib * rsb;                  // hib = rsb^2/2
    b_beta -= 0.5 * b_rsb * rsb * ib;      // rsb = beta^-1/2
    qbar[0] = bx;
    qbar[1] = b_qs * tx + b_qn * nx;
    qbar[2] = b_qs * ty + b_qn * ny;
    qbar[3] = -0.5 * b_beta;
}

// ---------------------------------------------------------------------------
// flux adjoint, owner side
// ---------------------------------------------------------------------------
template <class T>
__global__ void __launch_bounds__(128) k_adj_flux(AdjParamsT<T> P)
{
    const DevGeom &g = P.g;
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= g.n) return;
    const uint8_t f = g.flag[p] & 3;
    const bool second = P.order == 2;
    const T h = T(0.5);
    T qb0[4] = {0, 0, 0, 0}, gb0[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    const int e0 = g.off[p], e1 = g.off[p + 1];
    if (f == FLAG_FARFIELD) {
        // R = 0 there: no cotangent flows from this point
        for (int e = e0; e < e1; ++e) {
            st4(P.ebar, e, qb0);
            P.wbar[e] = make_double2(0.0, 0.0);
        }
        st4(P.qbar, p, qb0);
        if (second) st8(P.gbar, p, gb0);
        return;
    }
    const double2 xy0 = g.xy[p];
    const double2 n0d = g.nrm[p];
    const T nx = T(n0d.x), ny = T(n0d.y);
    const T tx = ny, ty = -nx;
    const T inv_gm1 = T(P.inv_gm1);
    T Rb[4], q0[4], g0[8];
    ld4(P.Rbar, p, Rb);
    // frame-order cotangent of R_local: R_global = (R0, R1 t + R2 n, R3)
    const T Rl[4] = {Rb[0], Rb[1] * tx + Rb[2] * ty, Rb[1] * nx + Rb[2] * ny, Rb[3]};
    ld4(P.q, p, q0);
    if (second) ld8(P.qg, p, g0);
    for (int e = e0; e < e1; ++e) {
        const int i = g.idx[e];
        const uint8_t m = g.mask[e];
        const int ks = xsub(m), kn = ysub(m);
        const bool us_ = sub_needed(f, ks), un_ = sub_needed(f, kn);
        const double2 wd = g.fxw[e];
        const T wx = T(wd.x), wy = T(wd.y);
        T qti[4], qt0[4];
        ld4(P.q, i, qti);
        T dx = T(0), dy = T(0), gi[8];
#pragma unroll
        for (int k = 0; k < 4; ++k) qt0[k] = q0[k];
        if (second) {
            const double2 xyi = g.xy[i];
            dx = T(xyi.x - xy0.x);
            dy = T(xyi.y - xy0.y);
            ld8(P.qg, i, gi);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                qti[k] = qti[k] - h * (dx * gi[k] + dy * gi[4 + k]);
                qt0[k] = qt0[k] - h * (dx * g0[k] + dy * g0[4 + k]);
            }
        }
        T cs[4], cn[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            cs[k] = us_ ? wx * Rl[k] : T(0);
            cn[k] = un_ ? wy * Rl[k] : T(0);
        }
        T qbi[4], qbo[4], Gsi[4] = {0, 0, 0, 0}, Gni[4] = {0, 0, 0, 0}, Gs0[4] = {0, 0, 0, 0},
                              Gn0[4] = {0, 0, 0, 0};
        const T sgs = (m & M_XPOS) ? T(1) : T(-1), sgn = (m & M_YPOS) ? T(1) : T(-1);
        if (us_ || un_) {
            if constexpr (std::is_same<T, double>::value) {
                state_adjoint_rev(qti, tx, ty, nx, ny, us_, sgs, un_, sgn, cs, cn, inv_gm1, P.g14 != 0, qbi, Gsi, Gni);
                state_adjoint_rev(qt0, tx, ty, nx, ny, us_, sgs, un_, sgn, cs, cn, inv_gm1, P.g14 != 0, qbo, Gs0, Gn0);
            } else {
                state_adjoint(qti, tx, ty, nx, ny, us_, sgs, un_, sgn, cs, cn, inv_gm1, P.g14 != 0, qbi, Gsi, Gni);
                state_adjoint(qt0, tx, ty, nx, ny, us_, sgs, un_, sgn, cs, cn, inv_gm1, P.g14 != 0, qbo, Gs0, Gn0);
            }
        } else {
#pragma unroll
            for (int k = 0; k < 4; ++k) qbi[k] = qbo[k] = T(0);
        }
        // R += w (G(q~_i) - G(q~_0)): + for the neighbour, - for the owner
        T wbx = T(0), wby = T(0);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            wbx += Rl[k] * (Gsi[k] - Gs0[k]);
            wby += Rl[k] * (Gni[k] - Gn0[k]);
            qbo[k] = -qbo[k];
        }
        P.wbar[e] = make_double2(us_ ? (double)wbx : 0.0, un_ ? (double)wby : 0.0);
        st4(P.ebar, e, qbi);
        T dxb = T(0), dyb = T(0);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            qb0[k] += qbo[k];
            if (second) {
                // q~_0 = q_0 - (dx qx_0 + dy qy_0)/2
                gb0[k] -= h * dx * qbo[k];
                gb0[4 + k] -= h * dy * qbo[k];
                dxb -= h * qbo[k] * g0[k];
                dyb -= h * qbo[k] * g0[4 + k];
            }
        }
        double2 db = P.dbar[e];
        db.x += (double)dxb;
        db.y += (double)dyb;
        P.dbar[e] = db;
    }
    st4(P.qbar, p, qb0);
    if (second) st8(P.gbar, p, gb0);
}

// ---------------------------------------------------------------------------
// flux adjoint, neighbour side: point p gathers the cotangents of q~_p over
// the edges that reach it
// ---------------------------------------------------------------------------
template <class T>
__global__ void __launch_bounds__(128) k_adj_flux_gather(AdjParamsT<T> P)
{
    const DevGeom &g = P.g;
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= g.n) return;
    const bool second = P.order == 2;
    const T h = T(0.5);
    T qb[4], gb[8], gp[8];
    ld4(P.qbar, p, qb);
    if (second) {
        ld8(P.gbar, p, gb);
        ld8(P.qg, p, gp);
    }
    const double2 xyp = g.xy[p];
    for (int t = P.toff[p]; t < P.toff[p + 1]; ++t) {
        const int e = P.tedge[t];
        T eb[4];
        ld4(P.ebar, e, eb);
#pragma unroll
        for (int k = 0; k < 4; ++k) qb[k] += eb[k];
        if (second) {
            const double2 xys = g.xy[P.tsrc[t]];
            const T dx = T(xyp.x - xys.x), dy = T(xyp.y - xys.y);
            T dxb = T(0), dyb = T(0);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                // q~_p = q_p - (dx qx_p + dy qy_p)/2 on this edge
                gb[k] -= h * dx * eb[k];
                gb[4 + k] -= h * dy * eb[k];
                dxb -= h * eb[k] * gp[k];
                dyb -= h * eb[k] * gp[4 + k];
            }
            double2 d = P.dbar[e];
            d.x += (double)dxb;
            d.y += (double)dyb;
            P.dbar[e] = d;
        }
    }
    st4(P.qbar, p, qb);
    if (second) st8(P.gbar, p, gb);
}

// ---------------------------------------------------------------------------
// one least-squares pass of E15 in reverse. Forward (per component c):
//   g_p = sum_e a_e s_e,  s_e = (q_i - q_p) - [dx (gx'_i - gx'_p) + dy (gy'_i - gy'_p)]/2
// with g' the previous iterate (absent in the first-order pass).
// ---------------------------------------------------------------------------
template <class T>
__global__ void __launch_bounds__(128) k_adj_grad(AdjParamsT<T> P, const T *__restrict__ gprev,
                                                  const T *__restrict__ gbar_in, T *__restrict__ gbar_out)
{
    const DevGeom &g = P.g;
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= g.n) return;
    const bool inner = gprev != nullptr;
    T qb[4], gb[8], qp[4], gbo[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    ld4(P.qbar, p, qb);
    ld8(gbar_in, p, gb);
    ld4(P.q, p, qp);
    const double2 xyp = g.xy[p];
    // an inner pass is sum_e a_e (q_i - q_0 - h_e.grad q_i) + grad q_0 / 2
    // (h_e the half offset; the terms in grad q_0 add up to grad q_0 / 2 since
    // sum_e a_e d_e^T = I, and the forward passes take them so), so grad q_0
    // gets gb / 2 and neither the weights nor the offsets see grad q_0
    if (inner) {
#pragma unroll
        for (int k = 0; k < 8; ++k) gbo[k] = T(0.5) * gb[k];
    }
    // outgoing edges: owner terms, and the cotangents of a_e and of the offsets
    for (int e = g.off[p]; e < g.off[p + 1]; ++e) {
        const int i = g.idx[e];
        const double2 ad = g.lsw[e];
        const T ax = T(ad.x), ay = T(ad.y);
        T qi[4], gi[8];
        ld4(P.q, i, qi);
        T hx = T(0), hy = T(0);
        if (inner) {
            ld8(gprev, i, gi);
            double2 hh;
            if (g.hd) {
                hh = g.hd[e];
            } else {
                const double2 xyi = g.xy[i];
                hh = make_double2(0.5 * (xyi.x - xyp.x), 0.5 * (xyi.y - xyp.y));
            }
            hx = T(hh.x);
            hy = T(hh.y);
        }
        T abx = T(0), aby = T(0), dbx = T(0), dby = T(0);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const T sb = ax * gb[k] + ay * gb[4 + k];
            T s = qi[k] - qp[k];
            if (inner) {
                s = s - (hx * gi[k] + hy * gi[4 + k]);
                // d_e = 2 h_e: d_bar = -(sb/2) grad q_i
                dbx -= T(0.5) * sb * gi[k];
                dby -= T(0.5) * sb * gi[4 + k];
            }
            qb[k] -= sb;
            abx += s * gb[k];
            aby += s * gb[4 + k];
        }
        double2 ab = P.abar[e];
        ab.x += (double)abx;
        ab.y += (double)aby;
        P.abar[e] = ab;
        if (inner) {
            double2 db = P.dbar[e];
            db.x += (double)dbx;
            db.y += (double)dby;
            P.dbar[e] = db;
        }
    }
    // incoming edges: the terms of this point as a neighbour
    for (int t = P.toff[p]; t < P.toff[p + 1]; ++t) {
        const int e = P.tedge[t], src = P.tsrc[t];
        const double2 ad = g.lsw[e];
        const T ax = T(ad.x), ay = T(ad.y);
        T gs[8];
        ld8(gbar_in, src, gs);
        T hx = T(0), hy = T(0);
        if (inner) {
            double2 hh;
            if (g.hd) {
                hh = g.hd[e];
            } else {
                const double2 xys = g.xy[src];
                hh = make_double2(0.5 * (xyp.x - xys.x), 0.5 * (xyp.y - xys.y));
            }
            hx = T(hh.x);
            hy = T(hh.y);
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const T sb = ax * gs[k] + ay * gs[4 + k];
            qb[k] += sb;
            if (inner) {
                gbo[k] -= hx * sb;
                gbo[4 + k] -= hy * sb;
            }
        }
    }
    st4(P.qbar, p, qb);
    if (inner) st8(gbar_out, p, gbo);
}

// ---------------------------------------------------------------------------
// Venkatakrishnan's limiter in reverse. Forward (k_qgrad's limited pass, per
// component): g = phi g_raw with phi = f(x_m, d_m) when x_m < 2 d_m, else 1;
//   f(x, d) = N/M, N = x (x + 2d) + eps^2, M = x (x + d) + 2 d^2 + eps^2,
//   x_m = min(D+, -D-), D+- the largest / smallest q_i - q_0 over the stencil
//   and P_0 itself (0), d_m = max_e |h_e . g_raw| (h_e the half offset),
//   eps^2 = (K dmin)^3, dmin the nearest neighbour's distance.
// With G = gbar . g_raw (the cotangent of phi):
//   g_raw_bar = phi gbar + G f_d s h*          (h* the edge of d_m, s the sign
//                                               of h*.g_raw)
//   x_m = q_i - q_0 (D+) or q_0 - q_j (-D-): q_0 and the extreme neighbour get
//         -+ G f_x; the neighbour's share is handed over through lidx/lval
//         and added by k_adj_limit_gather
//   the offsets: d* = 2 h* gets G f_d s g_raw / 2, the nearest neighbour's
//         offset gets 3 K^3 dmin^2 G f_eps d/|d| (through eps^2)
// The choices are the forward's: the first largest (smallest) q_i - q_0 in
// row order, P_0's own 0 winning ties; the first largest |h . g_raw|; the
// first nearest neighbour by squared distance. Where phi = 1 the limiter is
// inactive and gbar passes through.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128) k_adj_limit(AdjParams P, const double *__restrict__ graw,
                                                   const double *__restrict__ gbar_in, double *__restrict__ gbar_out,
                                                   int32_t *__restrict__ lidx, double *__restrict__ lval,
                                                   double limK)
{
    const DevGeom &g = P.g;
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= g.n) return;
    double q0[4], gr[8], gb[8], qb[4];
    ld4(P.q, p, q0);
    ld8(graw, p, gr);
    ld8(gbar_in, p, gb);
    ld4(P.qbar, p, qb);
    const double2 P0 = g.xy[p];
    double dmx[4] = {0.0, 0.0, 0.0, 0.0}, dmn[4] = {0.0, 0.0, 0.0, 0.0}, hm[4] = {-1.0, -1.0, -1.0, -1.0};
    int emx[4] = {-1, -1, -1, -1}, emn[4] = {-1, -1, -1, -1}, eh[4] = {-1, -1, -1, -1};
    double sh[4] = {0.0, 0.0, 0.0, 0.0};
    double2 hh[4];
    int enear = -1;
    double d2near = 0.0;
    for (int e = g.off[p]; e < g.off[p + 1]; ++e) {
        const int i = g.idx[e];
        double qi[4];
        ld4(P.q, i, qi);
        const double2 Pi = g.xy[i];
        const double dx = Pi.x - P0.x, dy = Pi.y - P0.y;
        const double2 h = g.hd ? g.hd[e] : make_double2(0.5 * dx, 0.5 * dy);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const double dq = qi[k] - q0[k];
            if (dq > dmx[k]) {
                dmx[k] = dq;
                emx[k] = e;
            }
            if (dq < dmn[k]) {
                dmn[k] = dq;
                emn[k] = e;
            }
            const double c = fma(h.x, gr[k], h.y * gr[4 + k]);
            if (fabs(c) > hm[k]) {
                hm[k] = fabs(c);
                eh[k] = e;
                sh[k] = c < 0.0 ? -1.0 : 1.0;
                hh[k] = h;
            }
        }
        const double d2 = dx * dx + dy * dy;
        if (enear < 0 || d2 < d2near) {
            enear = e;
            d2near = d2;
        }
    }
    const double dmin = g.dmin[p], hK = dmin * limK, eps2 = hK * hK * hK;
    double go[8];
    double dminb = 0.0;
    int32_t li[4] = {-1, -1, -1, -1};
    double lv[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        go[k] = gb[k];
        go[4 + k] = gb[4 + k];
        const bool plus = dmx[k] <= -dmn[k];
        const double x = plus ? dmx[k] : -dmn[k], d = hm[k];
        if (eh[k] < 0 || !(x < 2.0 * d)) continue;   // phi = 1
        const double N = fma(x, x + 2.0 * d, eps2), M = fma(x, x + d, fma(2.0 * d, d, eps2));
        const double phi = N / M, iM2 = 1.0 / (M * M);
        const double fx = ((2.0 * x + 2.0 * d) * M - N * (2.0 * x + d)) * iM2;
        const double fd = (2.0 * x * M - N * (x + 4.0 * d)) * iM2;
        const double fe = (M - N) * iM2;
        const double G = gb[k] * gr[k] + gb[4 + k] * gr[4 + k];
        const double gd = G * fd * sh[k];
        go[k] = phi * gb[k] + gd * hh[k].x;
        go[4 + k] = phi * gb[4 + k] + gd * hh[k].y;
        const double xb = G * fx;
        if (plus && emx[k] >= 0) {
            qb[k] -= xb;
            li[k] = emx[k];
            lv[k] = xb;
        } else if (!plus && emn[k] >= 0) {
            qb[k] += xb;
            li[k] = emn[k];
            lv[k] = -xb;
        }
        // d* = 2 h*: its offset cotangent is half that of h*
        double2 db = P.dbar[eh[k]];
        db.x += 0.5 * gd * gr[k];
        db.y += 0.5 * gd * gr[4 + k];
        P.dbar[eh[k]] = db;
        dminb += G * fe * 3.0 * limK * limK * limK * dmin * dmin;
    }
    if (dminb != 0.0 && enear >= 0 && dmin > 0.0) {
        const double2 Pi = g.xy[g.idx[enear]];
        double2 db = P.dbar[enear];
        db.x += dminb * (Pi.x - P0.x) / dmin;
        db.y += dminb * (Pi.y - P0.y) / dmin;
        P.dbar[enear] = db;
    }
    st4(P.qbar, p, qb);
    st8(gbar_out, p, go);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        lidx[4 * p + k] = li[k];
        lval[4 * p + k] = lv[k];
    }
}

// the extreme neighbours' share of the limiter's q cotangent (k_adj_limit),
// gathered over each point's incoming edges (no atomics)
__global__ void __launch_bounds__(128) k_adj_limit_gather(AdjParams P, const int32_t *__restrict__ lidx,
                                                          const double *__restrict__ lval)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P.g.n) return;
    const int t0 = P.toff[p], t1 = P.toff[p + 1];
    if (t0 == t1) return;
    double qb[4];
    ld4(P.qbar, p, qb);
    bool any = false;
    for (int t = t0; t < t1; ++t) {
        const int e = P.tedge[t];
        const int64_t src = P.tsrc[t];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (lidx[4 * src + k] == e) {
                qb[k] += lval[4 * src + k];
                any = true;
            }
        }
    }
    if (any) st4(P.qbar, p, qb);
}

// ---------------------------------------------------------------------------
// least-squares weights back to edge offsets (owner side)
// ---------------------------------------------------------------------------
struct Sym2 {
    double xx, xy, yy;
};

__global__ void __launch_bounds__(128) k_adj_weights(AdjParams P)
{
    const DevGeom &g = P.g;
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= g.n) return;
    const uint8_t f = g.flag[p] & 3;
    const bool full = P.order == 2;
    const double2 xy0 = g.xy[p];
    const double2 n0 = g.nrm[p];
    const double tx = n0.y, ty = -n0.x;
    const int e0 = g.off[p], e1 = g.off[p + 1];
    // normal-equation sums: full stencil (global frame) and the sub-stencils (s, n)
    Sym2 M = {0, 0, 0}, Ms[4] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    for (int e = e0; e < e1; ++e) {
        const double2 xyi = g.xy[g.idx[e]];
        const double dx = xyi.x - xy0.x, dy = xyi.y - xy0.y;
        const double ds = dx * tx + dy * ty, dn = dx * n0.x + dy * n0.y;
        M.xx += dx * dx; M.xy += dx * dy; M.yy += dy * dy;
        const uint8_t m = g.mask[e];
        const int ks = xsub(m), kn = ysub(m);
        if (ks >= 0) { Ms[ks].xx += ds * ds; Ms[ks].xy += ds * dn; Ms[ks].yy += dn * dn; }
        if (kn >= 0) { Ms[kn].xx += ds * ds; Ms[kn].xy += ds * dn; Ms[kn].yy += dn * dn; }
    }
    // inverses (M^-1 = [[yy, -xy], [-xy, xx]] / det)
    auto inv = [](const Sym2 &A) {
        const double det = A.xx * A.yy - A.xy * A.xy;
        Sym2 r = {A.yy / det, -A.xy / det, A.xx / det};
        return r;
    };
    const Sym2 Mi = inv(M);
    Sym2 Msi[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) Msi[k] = sub_needed(f, k) ? inv(Ms[k]) : Sym2{0, 0, 0};
    // B = sum (b a^T + a b^T) per system, with a = M^-1 d and b = M^-1 a_bar
    Sym2 B = {0, 0, 0}, Bs[4] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    for (int pass = 0; pass < 2; ++pass) {
        for (int e = e0; e < e1; ++e) {
            const double2 xyi = g.xy[g.idx[e]];
            const double dx = xyi.x - xy0.x, dy = xyi.y - xy0.y;
            const double ds = dx * tx + dy * ty, dn = dx * n0.x + dy * n0.y;
            const uint8_t m = g.mask[e];
            const int ks = xsub(m), kn = ysub(m);
            double gx = 0.0, gy = 0.0;   // offset cotangent, global frame
            double gs = 0.0, gn = 0.0;   // offset cotangent, (s, n) frame
            if (full) {
                const double2 ab = P.abar[e];
                const double ax = Mi.xx * dx + Mi.xy * dy, ay = Mi.xy * dx + Mi.yy * dy;
                const double bx = Mi.xx * ab.x + Mi.xy * ab.y, by = Mi.xy * ab.x + Mi.yy * ab.y;
                if (pass == 0) {
                    B.xx += 2.0 * bx * ax;
                    B.xy += bx * ay + ax * by;
                    B.yy += 2.0 * by * ay;
                } else {
                    gx += bx - (B.xx * dx + B.xy * dy);
                    gy += by - (B.xy * dx + B.yy * dy);
                }
            }
            const double2 wb = P.wbar[e];
            // x-sub weight = row 0 of M_s^-1 d, y-sub weight = row 1
            for (int h = 0; h < 2; ++h) {
                const int k = h == 0 ? ks : kn;
                if (!sub_needed(f, k)) continue;
                const Sym2 &Ai = Msi[k];
                const double as = Ai.xx * ds + Ai.xy * dn, an = Ai.xy * ds + Ai.yy * dn;
                const double abs_ = h == 0 ? wb.x : 0.0, abn = h == 0 ? 0.0 : wb.y;
                const double bs = Ai.xx * abs_ + Ai.xy * abn, bn = Ai.xy * abs_ + Ai.yy * abn;
                if (pass == 0) {
                    Bs[k].xx += 2.0 * bs * as;
                    Bs[k].xy += bs * an + as * bn;
                    Bs[k].yy += 2.0 * bn * an;
                } else {
                    gs += bs - (Bs[k].xx * ds + Bs[k].xy * dn);
                    gn += bn - (Bs[k].xy * ds + Bs[k].yy * dn);
                }
            }
            if (pass == 1) {
                // ds = dx tx + dy ty, dn = dx nx + dy ny
                double2 d = P.dbar[e];
                d.x += gx + gs * tx + gn * n0.x;
                d.y += gy + gs * ty + gn * n0.y;
                P.dbar[e] = d;
            }
        }
    }
}

// offsets d_e = P_dst - P_src back to points: x_bar_p = sum_in d_bar - sum_out d_bar,
// plus the per-point cotangents already gathered in pxy (internal order, or nullptr)
__global__ void __launch_bounds__(256) k_adj_points(AdjParams P, const double2 *__restrict__ pxy,
                                                    double *__restrict__ xb_out, double *__restrict__ yb_out,
                                                    int accumulate)
{
    const DevGeom &g = P.g;
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= g.n) return;
    double xb = 0.0, yb = 0.0;
    if (pxy) {
        xb = pxy[p].x;
        yb = pxy[p].y;
    }
    for (int t = P.toff[p]; t < P.toff[p + 1]; ++t) {
        const double2 d = P.dbar[P.tedge[t]];
        xb += d.x;
        yb += d.y;
    }
    for (int e = g.off[p]; e < g.off[p + 1]; ++e) {
        const double2 d = P.dbar[e];
        xb -= d.x;
        yb -= d.y;
    }
    const int32_t o = P.perm[p];
    if (xb_out) xb_out[o] = accumulate ? xb_out[o] + xb : xb;
    if (yb_out) yb_out[o] = accumulate ? yb_out[o] + yb : yb;
}

// q_bar to U_bar through E13 (duals over the four conserved variables);
// adds into Ub_acc ([n][4], internal order)
template <class T>
__global__ void __launch_bounds__(256) k_adj_state(AdjParamsT<T> P, const double *__restrict__ U,
                                                   double *__restrict__ Ub_acc)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t n = P.g.n;
    if (p >= n) return;
    double u[4], qb[4];
    ld4(U, p, u);
    T qt[4];
    ld4(P.qbar, p, qt);
#pragma unroll
    for (int k = 0; k < 4; ++k) qb[k] = (double)qt[k];
    D4 Ud[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        Ud[k] = dconst(u[k]);
        Ud[k].d[k] = 1.0;
    }
    const D4 rinv = recip(Ud[0]);
    const D4 u1 = Ud[1] * rinv, u2 = Ud[2] * rinv;
    const D4 pr = (1.0 / P.inv_gm1) * (Ud[3] - 0.5 * (Ud[0] * (u1 * u1 + u2 * u2)));
    const D4 beta = 0.5 * (Ud[0] * recip(pr));
    D4 q[4];
    q[0] = dlog(Ud[0]) + P.inv_gm1 * dlog(beta) - beta * (u1 * u1 + u2 * u2);
    q[1] = 2.0 * (beta * u1);
    q[2] = 2.0 * (beta * u2);
    q[3] = -2.0 * beta;
    double ub[4];
    ld4(Ub_acc, p, ub);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        double s = 0.0;
#pragma unroll
        for (int c = 0; c < 4; ++c) s += qb[c] * q[c].d[k];
        ub[k] += s;
    }
    st4(Ub_acc, p, ub);
}

// ---------------------------------------------------------------------------
// transpose CSR: incoming edges of every point, in edge order
// ---------------------------------------------------------------------------
__global__ void k_edge_src(int64_t n, const int32_t *__restrict__ off, int32_t *__restrict__ esrc)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    for (int e = off[p]; e < off[p + 1]; ++e) esrc[e] = (int32_t)p;
}

__global__ void k_iota(int64_t m, int32_t *__restrict__ v)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < m) v[t] = (int32_t)t;
}

// toff[p] = first position of key p in the sorted keys (lower bound)
__global__ void k_toff(int64_t n, int64_t nnz, const int32_t *__restrict__ keys, int32_t *__restrict__ toff)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p > n) return;
    int64_t lo = 0, hi = nnz;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (keys[mid] < p) lo = mid + 1;
        else hi = mid;
    }
    toff[p] = (int32_t)lo;
}

__global__ void k_tsrc(int64_t nnz, const int32_t *__restrict__ tedge, const int32_t *__restrict__ esrc,
                       int32_t *__restrict__ tsrc)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < nnz) tsrc[t] = esrc[tedge[t]];
}

unsigned blocks(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

cudaError_t build_transpose_csr(int64_t n, int64_t nnz, const int32_t *off, const int32_t *idx, int32_t *toff,
                                int32_t *tedge, int32_t *tsrc, cudaStream_t s)
{
    int32_t *esrc = nullptr, *iota = nullptr, *keys = nullptr;
    void *tmp = nullptr;
    size_t tmp_bytes = 0;
    cudaError_t err = cudaSuccess;
    const int64_t m = nnz > 0 ? nnz : 1;
    do {
        if ((err = cudaMallocAsync(&esrc, m * sizeof(int32_t), s)) != cudaSuccess) break;
        if ((err = cudaMallocAsync(&iota, m * sizeof(int32_t), s)) != cudaSuccess) break;
        if ((err = cudaMallocAsync(&keys, m * sizeof(int32_t), s)) != cudaSuccess) break;
        k_edge_src<<<blocks(n, 256), 256, 0, s>>>(n, off, esrc);
        k_iota<<<blocks(m, 256), 256, 0, s>>>(nnz, iota);
        if ((err = cudaGetLastError()) != cudaSuccess) break;
        if (nnz > 0) {
            // stable: equal destinations keep edge order
            err = cub::DeviceRadixSort::SortPairs(nullptr, tmp_bytes, idx, keys, iota, tedge, (int)nnz, 0, 32, s);
            if (err != cudaSuccess) break;
            if ((err = cudaMallocAsync(&tmp, tmp_bytes, s)) != cudaSuccess) break;
            err = cub::DeviceRadixSort::SortPairs(tmp, tmp_bytes, idx, keys, iota, tedge, (int)nnz, 0, 32, s);
            if (err != cudaSuccess) break;
        }
        k_toff<<<blocks(n + 1, 256), 256, 0, s>>>(n, nnz, keys, toff);
        if (nnz > 0) k_tsrc<<<blocks(nnz, 256), 256, 0, s>>>(nnz, tedge, esrc, tsrc);
        err = cudaGetLastError();
    } while (0);
    if (tmp) cudaFreeAsync(tmp, s);
    if (keys) cudaFreeAsync(keys, s);
    if (iota) cudaFreeAsync(iota, s);
    if (esrc) cudaFreeAsync(esrc, s);
    return err;
}

template <class T>
cudaError_t launch_adj_flux(const AdjParamsT<T> &P, cudaStream_t s)
{
    k_adj_flux<T><<<blocks(P.g.n, 128), 128, 0, s>>>(P);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    k_adj_flux_gather<T><<<blocks(P.g.n, 128), 128, 0, s>>>(P);
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_adj_grad(const AdjParamsT<T> &P, const T *gprev, const T *gbar_in, T *gbar_out, cudaStream_t s)
{
    k_adj_grad<T><<<blocks(P.g.n, 128), 128, 0, s>>>(P, gprev, gbar_in, gbar_out);
    return cudaGetLastError();
}

cudaError_t launch_adj_limit(const AdjParams &P, const double *graw, const double *gbar_in, double *gbar_out,
                             int32_t *lidx, double *lval, double limK, cudaStream_t s)
{
    k_adj_limit<<<blocks(P.g.n, 128), 128, 0, s>>>(P, graw, gbar_in, gbar_out, lidx, lval, limK);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    k_adj_limit_gather<<<blocks(P.g.n, 128), 128, 0, s>>>(P, lidx, lval);
    return cudaGetLastError();
}

cudaError_t launch_adj_weights(const AdjParams &P, cudaStream_t s)
{
    k_adj_weights<<<blocks(P.g.n, 128), 128, 0, s>>>(P);
    return cudaGetLastError();
}

cudaError_t launch_adj_points(const AdjParams &P, const double2 *pxy, double *x_bar, double *y_bar, bool accumulate,
                              cudaStream_t s)
{
    k_adj_points<<<blocks(P.g.n, 256), 256, 0, s>>>(P, pxy, x_bar, y_bar, accumulate ? 1 : 0);
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_adj_state(const AdjParamsT<T> &P, const double *U, double *Ub_acc, cudaStream_t s)
{
    k_adj_state<T><<<blocks(P.g.n, 256), 256, 0, s>>>(P, U, Ub_acc);
    return cudaGetLastError();
}

__global__ void k_to_float(int64_t m, const double *__restrict__ a, float *__restrict__ b)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < m) b[t] = (float)a[t];
}

cudaError_t launch_to_float(int64_t m, const double *a, float *b, cudaStream_t s)
{
    if (m <= 0) return cudaSuccess;
    k_to_float<<<blocks(m, 256), 256, 0, s>>>(m, a, b);
    return cudaGetLastError();
}

template cudaError_t launch_adj_flux<double>(const AdjParamsT<double> &, cudaStream_t);
template cudaError_t launch_adj_flux<float>(const AdjParamsT<float> &, cudaStream_t);
template cudaError_t launch_adj_grad<double>(const AdjParamsT<double> &, const double *, const double *, double *,
                                             cudaStream_t);
template cudaError_t launch_adj_grad<float>(const AdjParamsT<float> &, const float *, const float *, float *,
                                            cudaStream_t);
template cudaError_t launch_adj_state<double>(const AdjParamsT<double> &, const double *, double *, cudaStream_t);
template cudaError_t launch_adj_state<float>(const AdjParamsT<float> &, const double *, double *, cudaStream_t);

// ---------------------------------------------------------------------------
// pseudo-time update in forward (stage states for the reverse sweep) and in
// reverse. A stage maps U^n and a residual R to
//   U' = P(U^n - c dt R),
// P the boundary treatment: wall points lose the normal momentum (a symmetric
// projection), far-field points are reset to the free stream (no dependence).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_stage_fwd(StageParams S, const double *__restrict__ Un,
                                                   const double *__restrict__ R, double c,
                                                   double *__restrict__ Uout)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= S.n) return;
    const uint8_t f = S.flag[p] & 3;
    double u[4], r[4], o[4];
    ld4(Un, p, u);
    ld4(R, p, r);
    const double cdt = c * S.dt[p];
#pragma unroll
    for (int k = 0; k < 4; ++k) o[k] = u[k] - cdt * r[k];
    if (f == FLAG_WALL) {
        const double2 n0 = S.nrm[p];
        const double mn = o[1] * n0.x + o[2] * n0.y;
        o[1] = o[1] - mn * n0.x;
        o[2] = o[2] - mn * n0.y;
    } else if (f == FLAG_FARFIELD) {
        const double *Ui = S.case_uinf ? S.case_uinf + 4 * (int)S.pcase[p] : S.Uinf;
#pragma unroll
        for (int k = 0; k < 4; ++k) o[k] = Ui[k];
    }
    st4(Uout, p, o);
}

// reverse of one stage: v = P^T Ub_out; Uacc += v; dtbar (+)= -c sum_k R_k v_k;
// Rbar (+)= -c dt v (assigned when init, else added)
__global__ void __launch_bounds__(256) k_stage_adj(StageParams S, const double *__restrict__ Ub_out,
                                                   const double *__restrict__ R, double c, int init,
                                                   double *__restrict__ Uacc, double *__restrict__ dtbar,
                                                   double *__restrict__ Rbar)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= S.n) return;
    const uint8_t f = S.flag[p] & 3;
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    if (f != FLAG_FARFIELD) {
        ld4(Ub_out, p, v);
        if (f == FLAG_WALL) {
            const double2 n0 = S.nrm[p];
            const double mn = v[1] * n0.x + v[2] * n0.y;
            v[1] = v[1] - mn * n0.x;
            v[2] = v[2] - mn * n0.y;
        }
    }
    double a[4], r[4], rb[4] = {0.0, 0.0, 0.0, 0.0};
    ld4(Uacc, p, a);
    ld4(R, p, r);
    if (!init) ld4(Rbar, p, rb);
    const double dt = S.dt[p];
    double tb = 0.0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        a[k] += v[k];
        tb -= c * r[k] * v[k];
        rb[k] -= c * dt * v[k];
    }
    st4(Uacc, p, a);
    st4(Rbar, p, rb);
    dtbar[p] = init ? tb : dtbar[p] + tb;
}

// reverse of the last RK4 stage U^{n+1} = P(U^n - dt/6 (R0 + 2 R1 + 2 R2 + R3))
__global__ void __launch_bounds__(256) k_stage_adj_rk4_final(StageParams S, const double *__restrict__ Ub_out,
                                                             const double *__restrict__ R0,
                                                             const double *__restrict__ R1,
                                                             const double *__restrict__ R2,
                                                             const double *__restrict__ R3,
                                                             double *__restrict__ Uacc, double *__restrict__ dtbar,
                                                             double *__restrict__ Rb0, double *__restrict__ Rb1,
                                                             double *__restrict__ Rb2, double *__restrict__ Rb3)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= S.n) return;
    const uint8_t f = S.flag[p] & 3;
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    if (f != FLAG_FARFIELD) {
        ld4(Ub_out, p, v);
        if (f == FLAG_WALL) {
            const double2 n0 = S.nrm[p];
            const double mn = v[1] * n0.x + v[2] * n0.y;
            v[1] = v[1] - mn * n0.x;
            v[2] = v[2] - mn * n0.y;
        }
    }
    double a[4], r0[4], r1[4], r2[4], r3[4], b0[4], b1[4];
    ld4(Uacc, p, a);
    ld4(R0, p, r0);
    ld4(R1, p, r1);
    ld4(R2, p, r2);
    ld4(R3, p, r3);
    const double dt = S.dt[p];
    double tb = 0.0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        a[k] += v[k];
        tb -= (r0[k] + 2.0 * r1[k] + 2.0 * r2[k] + r3[k]) * v[k] / 6.0;
        b0[k] = -dt / 6.0 * v[k];
        b1[k] = -dt / 3.0 * v[k];
    }
    st4(Uacc, p, a);
    st4(Rb0, p, b0);
    st4(Rb1, p, b1);
    st4(Rb2, p, b1);
    st4(Rb3, p, b0);
    dtbar[p] = tb;
}

// reverse of timestep(): dt = CFL dmin / (|u| + 3 sqrt(p/rho)), dmin the
// distance to the nearest neighbour (the first of equals in row order)
__global__ void __launch_bounds__(256) k_dt_adj(StageParams S, DevGeom g, double cfl, double inv_gm1,
                                                const double *__restrict__ U, const double *__restrict__ dtbar,
                                                double *__restrict__ Uacc, double2 *__restrict__ dbar)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= S.n) return;
    const double tb = dtbar[p];
    double u[4];
    ld4(U, p, u);
    D4 Ud[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        Ud[k] = dconst(u[k]);
        Ud[k].d[k] = 1.0;
    }
    const D4 rinv = recip(Ud[0]);
    const D4 uu = Ud[1] * rinv, vv = Ud[2] * rinv;
    const D4 pr = (1.0 / inv_gm1) * (Ud[3] - 0.5 * (Ud[0] * (uu * uu + vv * vv)));
    const D4 speed = dsqrt(uu * uu + vv * vv) + 3.0 * dsqrt(pr * rinv);
    const D4 inv_speed = recip(speed);
    const double dmin = g.dmin[p];
    double a[4];
    ld4(Uacc, p, a);
#pragma unroll
    for (int k = 0; k < 4; ++k) a[k] += tb * cfl * dmin * inv_speed.d[k];
    st4(Uacc, p, a);
    // dmin = |P_i - P_0| of the nearest neighbour
    const double db = tb * cfl * inv_speed.v;
    const double2 P0 = g.xy[p];
    int best = -1;
    double d2best = 0.0;
    for (int e = g.off[p]; e < g.off[p + 1]; ++e) {
        const double2 Pi = g.xy[g.idx[e]];
        const double dx = Pi.x - P0.x, dy = Pi.y - P0.y;
        const double d2 = dx * dx + dy * dy;
        if (best < 0 || d2 < d2best) {
            best = e;
            d2best = d2;
        }
    }
    if (best >= 0 && dmin > 0.0) {
        const double2 Pi = g.xy[g.idx[best]];
        double2 d = dbar[best];
        d.x += db * (Pi.x - P0.x) / dmin;
        d.y += db * (Pi.y - P0.y) / dmin;
        dbar[best] = d;
    }
}

// forces: Cp_w = (p_w - p_inf)/q_inf, (fx, fy) = -sum Cp n ds, Cl = fy cos a - fx sin a,
// Cd = fx cos a + fy sin a. Per wall entry: U cotangent at the wall point and
// the cotangent of its arc-length weight ds_w
__global__ void __launch_bounds__(256) k_forces_adj(int64_t nwall, double gamma, double qinf,
                                                    const int32_t *__restrict__ wall,
                                                    const double *__restrict__ ds,
                                                    const double2 *__restrict__ nrm,
                                                    const double *__restrict__ U, double fxb, double fyb,
                                                    double *__restrict__ Uacc, double *__restrict__ dsbar)
{
    const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= nwall) return;
    const int p = wall[w];
    double u[4];
    ld4(U, p, u);
    const double rho = u[0], a = u[1] / rho, b = u[2] / rho;
    const double pr = (gamma - 1.0) * (u[3] - 0.5 * rho * (a * a + b * b));
    const double c = (pr - 1.0 / gamma) / qinf;
    const double2 n = nrm[p];
    const double fn = fxb * n.x + fyb * n.y;
    const double cb = -fn * ds[w];
    dsbar[w] = -c * fn;
    const double pb = cb / qinf, gm1 = gamma - 1.0;
    double ub[4];
    ld4(Uacc, p, ub);
    ub[0] += pb * gm1 * 0.5 * (a * a + b * b);
    ub[1] += -pb * gm1 * a;
    ub[2] += -pb * gm1 * b;
    ub[3] += pb * gm1;
    st4(Uacc, p, ub);
}

// ds_w = (|P_{w+1} - P_w| + |P_w - P_{w-1}|)/2 on the closed contour: point
// cotangents of the wall coordinates (added into pxy, internal order)
__global__ void __launch_bounds__(256) k_forces_xy_adj(int64_t nwall, const int32_t *__restrict__ wall,
                                                       const double2 *__restrict__ xy,
                                                       const double *__restrict__ dsbar,
                                                       double2 *__restrict__ pxy)
{
    const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= nwall) return;
    const int64_t wp = (w + nwall - 1) % nwall, wn = (w + 1) % nwall;
    const double2 P = xy[wall[w]], Pp = xy[wall[wp]], Pn = xy[wall[wn]];
    const double lp = sqrt((P.x - Pp.x) * (P.x - Pp.x) + (P.y - Pp.y) * (P.y - Pp.y));
    const double ln = sqrt((Pn.x - P.x) * (Pn.x - P.x) + (Pn.y - P.y) * (Pn.y - P.y));
    // segment (w-1, w) feeds ds_{w-1} and ds_w; segment (w, w+1) feeds ds_w and ds_{w+1}
    const double gp = 0.5 * (dsbar[wp] + dsbar[w]) / lp, gn = 0.5 * (dsbar[w] + dsbar[wn]) / ln;
    double2 o = pxy[wall[w]];
    o.x += gp * (P.x - Pp.x) - gn * (Pn.x - P.x);
    o.y += gp * (P.y - Pp.y) - gn * (Pn.y - P.y);
    pxy[wall[w]] = o;
}

cudaError_t launch_stage_fwd(const StageParams &S, const double *Un, const double *R, double c, double *Uout,
                             cudaStream_t s)
{
    k_stage_fwd<<<blocks(S.n, 256), 256, 0, s>>>(S, Un, R, c, Uout);
    return cudaGetLastError();
}

cudaError_t launch_stage_adj(const StageParams &S, const double *Ub_out, const double *R, double c, bool init,
                             double *Uacc, double *dtbar, double *Rbar, cudaStream_t s)
{
    k_stage_adj<<<blocks(S.n, 256), 256, 0, s>>>(S, Ub_out, R, c, init ? 1 : 0, Uacc, dtbar, Rbar);
    return cudaGetLastError();
}

cudaError_t launch_stage_adj_rk4_final(const StageParams &S, const double *Ub_out, const double *const R[4],
                                       double *Uacc, double *dtbar, double *const Rb[4], cudaStream_t s)
{
    k_stage_adj_rk4_final<<<blocks(S.n, 256), 256, 0, s>>>(S, Ub_out, R[0], R[1], R[2], R[3], Uacc, dtbar, Rb[0],
                                                          Rb[1], Rb[2], Rb[3]);
    return cudaGetLastError();
}

cudaError_t launch_dt_adj(const StageParams &S, const DevGeom &g, double cfl, double inv_gm1, const double *U,
                          const double *dtbar, double *Uacc, double2 *dbar, cudaStream_t s)
{
    k_dt_adj<<<blocks(S.n, 256), 256, 0, s>>>(S, g, cfl, inv_gm1, U, dtbar, Uacc, dbar);
    return cudaGetLastError();
}

cudaError_t launch_forces_adj(int64_t nwall, double gamma, double qinf, const int32_t *wall, const double *ds,
                              const double2 *nrm, const double2 *xy, const double *U, double fxb, double fyb,
                              double *Uacc, double *dsbar, double2 *pxy, cudaStream_t s)
{
    if (nwall <= 0) return cudaSuccess;
    k_forces_adj<<<blocks(nwall, 256), 256, 0, s>>>(nwall, gamma, qinf, wall, ds, nrm, U, fxb, fyb, Uacc, dsbar);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    k_forces_xy_adj<<<blocks(nwall, 256), 256, 0, s>>>(nwall, wall, xy, dsbar, pxy);
    return cudaGetLastError();
}

}  // namespace lskum
