// Device-side building blocks of the q-LSKUM hot path (arXiv 2403.13287, Sec. 2).
//
// Internal layout (points renumbered by the context's permutation):
//   xy[p], nrm[p]       double2   coordinates and unit normal (nx, ny)
//   flag[p]             uint8     0 interior, 1 wall, 2 far-field
//   off[p], idx[e]      int32     CSR connectivity N(P_0), rows in caller order
//   mask[e]             uint8     sub-stencil bits (x+ 1, x- 2, y+ 4, y- 8)
//   lsw[e]              double2   full-stencil least-squares weights (a_x, a_y):
//                                 grad f(P_0) = sum_e (a_x, a_y)_e (f_i - f_0)  (E9)
//   hd[e]               double2   (P_i - P_0)/2 (FP64 contexts): the half offset of
//                                 the E14 reconstruction and correction terms
//   fxw[e]              double2   sub-stencil weights (w_s, w_n): the edge's
//                                 coefficient in dG/ds of its x+- sub-stencil and
//                                 in dG/dn of its y+- sub-stencil (E11)
//   U, q                double[n][4]   conserved state and q-variables (E13)
//   qg                  double[n][8]   (qx0..3, qy0..3), global-frame q-derivatives
// The weights are the closed-form 2x2 least-squares solutions written as a
// linear combination of the perturbations; they depend on geometry only and
// are computed once, in FP64, when the context is created.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "fp64_tables.h"

namespace lskum {

enum : uint8_t { FLAG_INTERIOR = 0, FLAG_WALL = 1, FLAG_FARFIELD = 2 };
enum : uint8_t { M_XPOS = 1, M_XNEG = 2, M_YPOS = 4, M_YNEG = 8 };
// kinetic boundary mode: the member is the mirror image of a neighbour across
// the tangent line of P_0, carrying the reflected gas (wall) or the free
// stream with zero gradient (far field)
enum : uint8_t { M_IMG_WALL = 16, M_IMG_FAR = 32 };

enum : int { STATUS_NONPHYSICAL = 1, STATUS_DEGENERATE = 2 };

struct DevGeom {
    int64_t n;
    const double2 *__restrict__ xy;
    const double2 *__restrict__ nrm;
    const uint8_t *__restrict__ flag;
    const double *__restrict__ dmin;
    const int32_t *__restrict__ off;
    const int32_t *__restrict__ idx;
    const uint8_t *__restrict__ mask;
    const double2 *__restrict__ lsw;
    const double2 *__restrict__ fxw;
    const double2 *__restrict__ hd;  // FP64 contexts: per edge (P_i - P_0)/2, or nullptr
    const float2 *__restrict__ hd_f; // FP64 contexts: hd rounded to FP32 (the limiter's screening of d_m), or nullptr
    // kinetic boundary mode (all nullptr otherwise): the mirror images of the
    // neighbours of each wall and far-field point, per point in CSR form
    // (rows are empty at interior points); an image of P_i has local offsets
    // (ds_i, -dn_i) and the x+- membership of P_i with y+ and y- swapped
    const int32_t *__restrict__ ioff;    // [n+1]
    const int32_t *__restrict__ iidx;    // the neighbour whose image this is
    const uint8_t *__restrict__ imask;   // sub-stencil bits | M_IMG_WALL or M_IMG_FAR
    const double2 *__restrict__ ilsw;    // full-stencil weights of the images
    const double2 *__restrict__ ifxw;    // sub-stencil weights of the images
    const double2 *__restrict__ ihd;     // FP64 contexts: half offsets of the images
    const double *__restrict__ qinf;     // [cases][4] q of each case's free stream
    const uint16_t *__restrict__ pcase;  // per point: its case in a batch, or nullptr
};

// reflection of the vector (a, b) across the line with unit normal n
template <typename T>
__device__ __forceinline__ void reflect2(T &a, T &b, T nx, T ny)
{
    const T c = a * nx + b * ny;
    a = a - T(2) * c * nx;
    b = b - T(2) * c * ny;
}

// Free-stream and gas constants handed to every kernel.
struct Gas {
    double gamma;
    double inv_gm1;  // 1/(gamma - 1)
    double hc;       // gamma/(2 (gamma - 1)): enthalpy per unit mass h = hc/beta + |u|^2/2
    int g14;         // gamma == 1.4: beta^(-1/(gamma-1)) = beta^(-2.5) without log
    double Uinf[4];
};

// Primitive state of a (modified) q-vector, E13 inverted:
//   beta = -q4/2, u = q2/(2 beta), v = q3/(2 beta),
//   rho = exp(q1 + beta (u^2 + v^2)) beta^(-1/(gamma-1)), p = rho/(2 beta),
// with the velocity taken in the frame (t, n) of P_0.
struct Prim {
    double us, un;  // u.t, u.n
    double Ss, Sn;  // S = u.t sqrt(beta), u.n sqrt(beta): the split fluxes' arguments
    double hrho;    // rho/2
    double hp;      // p/2
    double h;       // (rho E + p)/rho
    double qb;      // 1/(4 beta) = h - (rho E + p/2)/rho
    double rrc;     // rho/(2 sqrt(pi beta)), so that rho B = rrc exp(-S^2)
};

// exp(x) 2^k, table-driven (P. T. P. Tang, ACM TOMS 15 (1989) 144-157):
// x = n ln2/4096 + r, |r| <= ln2/8192, n = 4096 m + j, exp(x) = 2^m 2^(j/4096) p(r)
// with p the degree-3 Taylor polynomial (gen_fp64_tables.py): 8 FP64
// instructions. The factor 2^(m+k) is an addition to the exponent field on
// the integer pipe: for |x| < 706 and |k| <= 2 the biased exponent of the
// result stays within [1, 2044] (2^(j/4096) p(r) lies in [1/2, 2] and
// |m| <= 1019). |x| >= 706 (or NaN), found from the high word of x on the
// integer pipe, goes to the library exp.
__device__ __forceinline__ double exp_tab(double x, int k = 0)
{
    int xhi;
    asm("{ .reg .b32 lo; mov.b64 {lo, %0}, %1; }" : "=r"(xhi) : "d"(x));
    if ((xhi & 0x7fffffff) >= 0x40861000) return ldexp(exp(x), k);  // 0x40861000: high word of 706.0
    const double magic = 0x1.8p52;
    const double t = fma(x, LSKUM_EXP_INV_L, magic);
    const int n = __double2loint(t);  // round-to-nearest integer held in the low word
    const double kd = t - magic;
    double r = fma(-kd, LSKUM_EXP_L_HI, x);
    r = fma(-kd, LSKUM_EXP_L_LO, r);
    double p = fma(r, 1.0 / 6.0, 0.5);
    p = fma(p, r, 1.0);
    p = fma(p, r, 1.0);
    const double tp = __ldg(&kExp2Table[n & (LSKUM_EXP_N - 1)]) * p;
    return __hiloint2double(__double2hiint(tp) + ((n >> LSKUM_EXP_LOG2N) + k) * (1 << 20), __double2loint(tp));
}

// a double strictly between 0 and +inf (not 0, negative, inf or NaN), tested
// on its bit pattern (integer pipe)
__device__ __forceinline__ bool finite_positive(double x)
{
    const long long b = __double_as_longlong(x);
    return b > 0 && b < 0x7ff0000000000000ll;
}

// the magnitude bits of x (sign bit cleared) by an integer AND that the
// compiler cannot turn into an FP64 absolute value, which would be issued on
// the FP64 pipe
__device__ __forceinline__ unsigned long long abs_bits(double x)
{
    unsigned long long b;
    asm("and.b64 %0, %1, 0x7fffffffffffffff;" : "=l"(b) : "l"(__double_as_longlong(x)));
    return b;
}

// x/2 for a positive normal x whose half is normal: the exponent field
// decremented on the integer pipe, bitwise the FP64 product 0.5 x there
__device__ __forceinline__ double half_of(double x)
{
    return __longlong_as_double(__double_as_longlong(x) - (1ll << 52));
}

// u.t = (q2 tx + q3 ty)/(2 beta) and u.n alike, straight from q (no u, v);
// exp_tab(., -1) gives rho/2 without a multiplication.
__device__ __forceinline__ bool prim_from_q(const double qt[4], const Gas &gas, double tx, double ty, double2 n0,
                                            Prim &s)
{
    // beta = -q4/2 as an exponent decrement of |q4|, bitwise the FP64 product:
    // q4 must be negative and normal with a normal half; anything else (zero,
    // positive, not finite, |q4| < 2^-1021, i.e. p/rho > 1e307) is non-physical
    const long long b3 = __double_as_longlong(qt[3]);
    const unsigned e3 = (unsigned)(b3 >> 52) & 0x7ffu;
    if (!(b3 < 0 && e3 >= 2u && e3 < 0x7ffu)) return false;
    const double beta = __longlong_as_double((long long)abs_bits(qt[3]) - (1ll << 52));
    const double rsb = rsqrt(beta);
    const double ib = rsb * rsb;           // 1/beta, so 1/q4 = -ib/2 without a division
    // ib/2 and ib/4 are exact exponent decrements while ib/4 is normal (biased
    // exponent of ib at least 3); beta above 1/16 of the largest double
    // (p/rho below 1e-307) is reported non-physical instead
    const bool ib_ok = (__double_as_longlong(ib) >> 52) > 2;
    const double hib = half_of(ib);
    // u.t = m_t/(2 beta) and S_t = u.t sqrt(beta) = m_t/(2 sqrt(beta)), with
    // m_t = q2 tx + q3 ty: 1/(2 sqrt(beta)) is rsb/2, an exponent decrement,
    // so no sqrt(beta) is formed (u.n and S_n alike)
    const double mt = fma(qt[1], tx, qt[2] * ty), mn = fma(qt[1], n0.x, qt[2] * n0.y);
    const double hrsb = half_of(rsb);
    s.us = mt * hib;
    s.un = mn * hib;
    s.Ss = mt * hrsb;
    s.Sn = mn * hrsb;
    const double w2 = fma(s.us, s.us, s.un * s.un);   // |u|^2
    double hrho;
    if (gas.g14) {
        // beta^-2.5 = beta^-1/2 (1/beta)^2
        hrho = exp_tab(fma(beta, w2, qt[0]), -1) * (rsb * (ib * ib));
    } else {
        hrho = exp_tab(fma(beta, w2, qt[0] - log(beta) * gas.inv_gm1), -1);
    }
    s.hrho = hrho;
    s.hp = hrho * hib;                     // p/2 = rho/(4 beta)
    // per unit mass: p/rho = 1/(2 beta), rho E = p/(gamma-1) + rho |u|^2/2
    s.h = fma(gas.hc, ib, 0.5 * w2);
    s.qb = half_of(hib);
    s.rrc = hrho * (rsb * 0.5641895835477563);  // 1/sqrt(pi)
    return finite_positive(hrho) && ib_ok;
}

// erf(S) and exp(-S^2) together, from one row of a Taylor table: on the grid
// s_k = k/1024 (0 <= s_k <= 6) the row holds the degree-4 Taylor coefficients
// of both functions in d = |S| - s_k (|d| <= 1/2048), so each is one Horner
// chain with an absolute error of about one unit in the last place of 1
// (gen_fp64_tables.py; the first omitted terms are below 1e-17). The nearest
// grid index comes from the top bits of |S| by integer operations, so the
// FP64 pipe sees one subtraction and 8 fused multiply-adds. |S| >= 6:
// erf = +-1 (erfc(6) = 2e-17) and exp(-S^2) directly.
__device__ __forceinline__ void erf_exp(double S, double &erfS, double &eS)
{
    // the words of |S| straight from S's bits: a materialised fabs would be
    // an FP64 instruction
    unsigned lo;
    int hi;
    asm("mov.b64 {%0, %1}, %2;" : "=r"(lo), "=r"(hi) : "d"(S));
    hi &= 0x7fffffff;
    if (hi >= 0x40180000) {  // |S| >= 6
        erfS = copysign(1.0, S);
        eS = exp(-S * S);
        return;
    }
    // an FP32 copy of a (truncated mantissa) built from the FP64 bits
    const float af = hi < ((1023 - 30) << 20)
                         ? 0.0f
                         : __int_as_float(((hi - ((1023 - 127) << 20)) << 3) | (int)(lo >> 29));
    const int k = __float2int_rn(af * (float)LSKUM_ERF_STEP);
    const double2 *r = reinterpret_cast<const double2 *>(kErfExpTable[k]);
    double v[LSKUM_ERF_ROW];
#pragma unroll
    for (int j = 0; j < LSKUM_ERF_ROW / 2; ++j) {
        const double2 t = __ldg(r + j);
        v[2 * j] = t.x;
        v[2 * j + 1] = t.y;
    }
    const double d = fabs(S) - v[0];   // |.| as an operand modifier of the subtraction
    double c = v[1 + LSKUM_ERF_DEG], e = v[2 + 2 * LSKUM_ERF_DEG];
#pragma unroll
    for (int n = LSKUM_ERF_DEG - 1; n >= 0; --n) {
        c = fma(c, d, v[1 + n]);
        e = fma(e, d, v[2 + LSKUM_ERF_DEG + n]);
    }
    erfS = copysign(c, S);
    eS = e;
}

// the sign of x flipped when sbit is the sign bit (x unchanged for sbit = 0):
// a multiplication by -1 or +1 done on the integer pipe
__device__ __forceinline__ double flip_sign(double x, unsigned long long sbit)
{
    return __longlong_as_double(__double_as_longlong(x) ^ (long long)sbit);
}

static constexpr unsigned long long kSignBit = 0x8000000000000000ull;


// Kinetic split flux along a direction: normal velocity un, transverse ut,
// sgn = +1 for G+, -1 for G- (half-range moments of the Maxwellian):
//   S = un sqrt(beta), A = (1 + sgn erf S)/2, B = exp(-S^2)/(2 sqrt(pi beta))
//   G = [rho(un A + sgn B), (p + rho un^2) A + sgn rho un B,
//        rho ut (un A + sgn B), (rhoE + p) un A + sgn (rhoE + p/2) B]
// evaluated as Q = rho A = rho/2 (1 + sgn erf S), W = sgn rho B:
// G0 = un Q + W, G1 = p A + un G0, G2 = ut G0, and with h = (rhoE + p)/rho,
// e2 = (rhoE + p/2)/rho = h - 1/(4 beta): G3 = h un Q + e2 W = h G0 - W/(4 beta).
// sbit = 0 for G+, kSignBit for G-: the products by sgn are sign flips. S
// (= un sqrt(beta)) comes from prim_from_q.
__device__ __forceinline__ void split_flux(unsigned long long sbit, const Prim &s, double un, double ut,
                                           double S, double G[4])
{
    double erfS, eS;
    erf_exp(S, erfS, eS);
    const double fe = flip_sign(erfS, sbit);
    const double Q = fma(s.hrho, fe, s.hrho);
    const double W = eS * flip_sign(s.rrc, sbit);
    G[0] = fma(un, Q, W);
    G[1] = fma(un, G[0], fma(s.hp, fe, s.hp));
    G[2] = ut * G[0];
    G[3] = fma(s.h, G[0], -s.qb * W);
}

// per-warp pair of residue partial sums (lo: lanes in the case of the warp's
// first point, hi: the others, i.e. a second case that starts inside the
// warp; every case has at least 32 points), summed in T within the warp and
// stored in FP64
template <typename T>
__device__ __forceinline__ void warp_residue_pair(const uint16_t *pcase, int64_t p, bool live, T r2, double *part)
{
    const int lane = threadIdx.x & 31;
    const int c = (pcase && live) ? (int)pcase[p] : 0;
    const int c0 = __shfl_sync(0xffffffffu, c, 0);
    T lo = (c == c0) ? r2 : T(0), hi = (c == c0) ? T(0) : r2;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lo += __shfl_down_sync(0xffffffffu, lo, o);
        hi += __shfl_down_sync(0xffffffffu, hi, o);
    }
    // warps wholly past the last point write nothing
    if (lane == 0 && live) {
        const int64_t w = p >> 5;
        part[2 * w] = (double)lo;
        part[2 * w + 1] = (double)hi;
    }
}

__device__ __forceinline__ void load4(const double *a, int64_t p, double v[4])
{
    const double2 *a2 = reinterpret_cast<const double2 *>(a);
    double2 lo = a2[2 * p], hi = a2[2 * p + 1];
    v[0] = lo.x; v[1] = lo.y; v[2] = hi.x; v[3] = hi.y;
}

__device__ __forceinline__ void store4(double *a, int64_t p, const double v[4])
{
    double2 *a2 = reinterpret_cast<double2 *>(a);
    a2[2 * p] = make_double2(v[0], v[1]);
    a2[2 * p + 1] = make_double2(v[2], v[3]);
}

__device__ __forceinline__ void load8(const double *a, int64_t p, double v[8])
{
    const double2 *a2 = reinterpret_cast<const double2 *>(a);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        double2 t = a2[4 * p + k];
        v[2 * k] = t.x; v[2 * k + 1] = t.y;
    }
}

__device__ __forceinline__ void store8(double *a, int64_t p, const double v[8])
{
    double2 *a2 = reinterpret_cast<double2 *>(a);
#pragma unroll
    for (int k = 0; k < 4; ++k) a2[4 * p + k] = make_double2(v[2 * k], v[2 * k + 1]);
}

// q-variables of a conserved state (E13), same operation order as the
// primitive form: rho, u = m/rho, p = (gamma-1)(E - rho|u|^2/2), beta = rho/(2p)
__device__ __forceinline__ bool q_from_U(const double U[4], const Gas &gas, double q[4])
{
    const double rho = U[0];
    const double irho = 1.0 / rho;
    const double u = U[1] * irho, v = U[2] * irho;
    const double p = (gas.gamma - 1.0) * (U[3] - 0.5 * rho * (u * u + v * v));
    const double beta = 0.5 * rho / p;
    // gamma = 1.4: ln rho + 2.5 ln beta as one logarithm of rho beta^2 sqrt(beta)
    const double lrb = gas.g14 ? log(rho * (beta * beta) * sqrt(beta)) : log(rho) + log(beta) * gas.inv_gm1;
    q[0] = lrb - beta * (u * u + v * v);
    q[1] = 2.0 * beta * u;
    q[2] = 2.0 * beta * v;
    q[3] = -2.0 * beta;
    return rho > 0.0 && p > 0.0 && isfinite(q[0]);
}

// ---------------------------------------------------------------------------
// FP32 forms for the mixed-precision flux kernel (same formulas as above), on
// a pair of states at once: the two ends of a stencil edge (x: q~_i,
// y: q~_0) take identical arithmetic, so each multiply, add and fused
// multiply-add of the pair is one packed FP32x2 instruction (FFMA2 / FMUL2 /
// FADD2 of sm_100 and later, round to nearest like the scalar ones); the
// special functions (reciprocal square root, exp, reciprocal) stay per
// component.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 pr2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

struct PrimF2 {
    float2 rho, u, v, p, sqb;
    float2 h, e2;  // (rho E + p)/rho, (rho E + p/2)/rho
    float2 rrc;    // rho rsb / (2 sqrt(pi)), so that rho B = rrc exp(-S^2)
};

__device__ __forceinline__ bool prim_from_q_f2(const float2 qt[4], float inv_gm1, bool g14, PrimF2 &s)
{
    const float2 beta = mul2(pr2(-0.5f), qt[3]);
    if (!(beta.x > 0.0f && beta.y > 0.0f)) return false;
    const float2 rsb = make_float2(rsqrtf(beta.x), rsqrtf(beta.y));
    const float2 ib = mul2(rsb, rsb);     // 1/beta
    const float2 hib = mul2(pr2(0.5f), ib);
    s.u = mul2(qt[1], hib);
    s.v = mul2(qt[2], hib);
    s.sqb = mul2(beta, rsb);
    const float2 u2 = fma2(s.u, s.u, mul2(s.v, s.v));
    const float2 ex = fma2(beta, u2, qt[0]);
    // __expf: relative error about |arg| * 6e-8 here (|arg| < ~20), within
    // the FP32 budget of the form
    if (g14) {
        const float2 e = make_float2(__expf(ex.x), __expf(ex.y));
        s.rho = mul2(mul2(e, rsb), mul2(ib, ib));
    } else {
        const float2 lb = make_float2(__logf(beta.x), __logf(beta.y));
        const float2 a = fma2(lb, pr2(-inv_gm1), ex);
        s.rho = make_float2(__expf(a.x), __expf(a.y));
    }
    s.p = mul2(s.rho, hib);
    const float2 hu2 = mul2(pr2(0.5f), u2);
    s.h = fma2(pr2(0.5f * (inv_gm1 + 1.0f)), ib, hu2);
    s.e2 = fma2(pr2(0.5f * (inv_gm1 + 0.5f)), ib, hu2);
    s.rrc = mul2(s.rho, mul2(rsb, pr2(0.28209479177387814f)));
    return isfinite(s.rho.x) && s.rho.x > 0.0f && isfinite(s.rho.y) && s.rho.y > 0.0f;
}

// A+- = (1 +- erf S)/2 with erfc from Abramowitz & Stegun 7.1.26 (Hastings):
// erfc(x) = (a1 t + a2 t^2 + a3 t^3 + a4 t^4 + a5 t^5) exp(-x^2), t = 1/(1 + p x),
// x >= 0, |error| <= 1.5e-7, about one FP32 ulp of 1. exp(-S^2) is shared with
// B, and the smaller of A+ and A- is formed directly (no 1 - erf cancellation).
__device__ __forceinline__ float2 half_range_A2(float sgn, float2 S, float2 e)
{
    const float2 x = make_float2(fabsf(S.x), fabsf(S.y));
    const float2 den = fma2(pr2(0.3275911f), x, pr2(1.0f));
    const float2 t = make_float2(__fdividef(1.0f, den.x), __fdividef(1.0f, den.y));
    float2 poly = fma2(t, pr2(1.061405429f), pr2(-1.453152027f));
    poly = fma2(t, poly, pr2(1.421413741f));
    poly = fma2(t, poly, pr2(-0.284496736f));
    poly = fma2(t, poly, pr2(0.254829592f));
    const float2 small = mul2(mul2(pr2(0.5f), mul2(t, poly)), e);  // (1 - erf|S|)/2
    const float2 large = fma2(small, pr2(-1.0f), pr2(1.0f));
    // A+ is the large one for S > 0, A- for S < 0
    return make_float2(sgn * S.x >= 0.0f ? large.x : small.x, sgn * S.y >= 0.0f ? large.y : small.y);
}

// the split flux of both states, regrouped as split_flux: Q = rho A, W = sgn rho B
__device__ __forceinline__ void split_flux_f2(float sgn, const PrimF2 &s, float2 un, float2 ut, float2 G[4])
{
    const float2 S = mul2(un, s.sqb);
    const float2 S2 = mul2(S, S);
    const float2 e = make_float2(__expf(-S2.x), __expf(-S2.y));
    const float2 A = half_range_A2(sgn, S, e);
    const float2 Q = mul2(s.rho, A);
    const float2 W = mul2(e, mul2(pr2(sgn), s.rrc));
    G[0] = fma2(un, Q, W);
    G[1] = fma2(un, G[0], mul2(s.p, A));
    G[2] = mul2(ut, G[0]);
    G[3] = fma2(mul2(s.h, un), Q, mul2(s.e2, W));
}

__device__ __forceinline__ void load4f(const float *a, int64_t p, float v[4])
{
    const float4 t = reinterpret_cast<const float4 *>(a)[p];
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}

__device__ __forceinline__ void store4f(float *a, int64_t p, const float v[4])
{
    reinterpret_cast<float4 *>(a)[p] = make_float4(v[0], v[1], v[2], v[3]);
}

// the 8 floats of row p of a read-only [n][8] array (32-byte aligned rows) as
// one 256-bit load through the non-coherent path: half the load instructions
// of two float4 loads for the neighbour gathers
__device__ __forceinline__ void gather8f(const float *a, int64_t p, float v[8])
{
    asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7])
        : "l"(a + 8 * p));
}

__device__ __forceinline__ void load8f(const float *a, int64_t p, float v[8])
{
    const float4 *a4 = reinterpret_cast<const float4 *>(a);
    const float4 lo = a4[2 * p], hi = a4[2 * p + 1];
    v[0] = lo.x; v[1] = lo.y; v[2] = lo.z; v[3] = lo.w;
    v[4] = hi.x; v[5] = hi.y; v[6] = hi.z; v[7] = hi.w;
}

__device__ __forceinline__ void store8f(float *a, int64_t p, const float v[8])
{
    float4 *a4 = reinterpret_cast<float4 *>(a);
    a4[2 * p] = make_float4(v[0], v[1], v[2], v[3]);
    a4[2 * p + 1] = make_float4(v[4], v[5], v[6], v[7]);
}

// FP64 <-> FP32 conversions on the integer pipe. On this GPU the FP64 pipe
// runs at 1/64 of the FP32 rate, and a conversion instruction occupies it like
// an FP64 add, so the mixed kernels move state values across with bit
// arithmetic, branch-free. double -> float rounds the 29 dropped mantissa
// bits half away from zero, flushes magnitudes below the FP32 normal range to
// zero and saturates above it to infinity (NaN stays NaN); float -> double is
// exact for normal numbers and flushes FP32 subnormals to zero.
__device__ __forceinline__ float f64_to_f32_ip(double x)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned int sign = (unsigned int)(b >> 32) & 0x80000000u;
    const unsigned long long mag = b & 0x7fffffffffffffffull;
    const unsigned int e = (unsigned int)(mag >> 52);
    const long long f = (long long)((mag + (1ull << 28)) >> 29) - ((long long)(1023 - 127) << 23);
    unsigned int out = (unsigned int)f;
    out = e < 1023u - 126u ? 0u : out;
    out = f >= 0x7f800000ll ? 0x7f800000u : out;
    out = e == 2047u ? ((mag & 0xfffffffffffffull) ? 0x7fc00000u : 0x7f800000u) : out;
    return __uint_as_float(sign | out);
}

__device__ __forceinline__ double f32_to_f64_ip(float f)
{
    const unsigned int b = __float_as_uint(f);
    const unsigned int mag = b & 0x7fffffffu;
    const unsigned long long sign = (unsigned long long)(b & 0x80000000u) << 32;
    unsigned long long out = ((unsigned long long)mag + ((unsigned long long)(1023 - 127) << 23)) << 29;
    out = mag < 0x00800000u ? 0ull : out;
    out = mag >= 0x7f800000u ? ((0x7ffull << 52) | ((unsigned long long)(mag & 0x7fffffu) << 29)) : out;
    return __longlong_as_double((long long)(sign | out));
}

// q-variables (E13) of an FP32 copy of the state
__device__ __forceinline__ bool q_from_Uf(const float U[4], float gamma, float inv_gm1, float q[4])
{
    const float rho = U[0], m1 = U[1], m2 = U[2], E = U[3];
    const float ir = __fdividef(1.0f, rho);
    const float u = m1 * ir, v = m2 * ir;
    const float p = (gamma - 1.0f) * (E - 0.5f * (m1 * u + m2 * v));
    const float beta = 0.5f * rho * __fdividef(1.0f, p);
    q[0] = logf(rho) + logf(beta) * inv_gm1 - beta * (u * u + v * v);
    q[1] = 2.0f * beta * u;
    q[2] = 2.0f * beta * v;
    q[3] = -2.0f * beta;
    return rho > 0.0f && p > 0.0f && isfinite(q[0]);
}

// q-variables (E13) of an FP64 state, evaluated in FP32
__device__ __forceinline__ bool q_from_U_f(const double Ud[4], float gamma, float inv_gm1, float q[4])
{
    const float rho = (float)Ud[0], m1 = (float)Ud[1], m2 = (float)Ud[2], E = (float)Ud[3];
    const float ir = __fdividef(1.0f, rho);
    const float u = m1 * ir, v = m2 * ir;
    const float p = (gamma - 1.0f) * (E - 0.5f * (m1 * u + m2 * v));
    const float beta = 0.5f * rho * __fdividef(1.0f, p);
    q[0] = logf(rho) + logf(beta) * inv_gm1 - beta * (u * u + v * v);
    q[1] = 2.0f * beta * u;
    q[2] = 2.0f * beta * v;
    q[3] = -2.0f * beta;
    return rho > 0.0f && p > 0.0f && isfinite(q[0]);
}

}  // namespace lskum
