/*
 * Plain FP64 CPU oracle of the q-LSKUM hot path (arXiv 2403.13287).
 *
 * TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the bench's
 * CPU-baseline leg load this file; the CUDA product path never does, and the
 * two share no code. It is written to be checked by eye against the paper:
 * serial loops over points in input order, neighbours in CSR order, FP64,
 * glibc erf/exp/log/sqrt, and it must be compiled with -ffp-contract=off.
 *
 * Routine names follow Algorithm 1 of the paper: q_variables, q_derivatives,
 * flux_residual, timestep, state_update, residue. Where the paper is silent
 * the reading used is stated at the routine (free stream, boundary
 * conditions, local time step, RK4, residue norm, forces). The kinetic
 * boundary mode (orc_residual_bc / orc_solve_bc with boundary = 1) is a
 * reading of the kinetic wall and far-field conditions the paper cites
 * without stating them; see "Stencil members".
 *
 * Arrays of 4 components are stored component-major: A[k*n + p].
 *
 * Points are independent within a pass (q_variables, each q_derivatives
 * solve, the limiter, flux_residual, timestep, each state update): every
 * point reads the previous pass's arrays and writes only its own entries.
 * Built with -fopenmp (the host-core timing build) those loops share the
 * points out among threads; each point's own sums still run serially in CSR
 * order, so both builds give the same bits. Without -fopenmp the pragmas are
 * ignored and every loop runs in input order.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_INTERIOR 0
#define ORC_WALL 1
#define ORC_FARFIELD 2

/* one byte per CSR entry: membership in the four sub-stencils (Sec. 2) */
#define ORC_XPOS 1u /* N_x+ : dx_i < 0 (upwind side of Gx+) */
#define ORC_XNEG 2u /* N_x- : dx_i > 0 */
#define ORC_YPOS 4u /* N_y+ : dy_i < 0 */
#define ORC_YNEG 8u /* N_y- : dy_i > 0 */

#define ORC_OK 0
#define ORC_ERR_DEGENERATE 3
#define ORC_ERR_NONPHYSICAL 6

/* relative threshold below which a 2x2 least-squares matrix counts as singular */
#define ORC_DET_EPS 1e-10

static const double ORC_PI = 3.14159265358979323846;

/* ------------------------------------------------------------------------ */
/* Local frame of a point: tangent t = (ny, -nx), normal n = (nx, ny).      */
/* The paper's (x, y) at a point are its (s, n) here (Sec. 2, E9-E12).      */
/* ------------------------------------------------------------------------ */

/*
 * Sub-stencil split, Sec. 2 after E12: N_x+- = {P_i in N(P_0) : dx_i <> 0},
 * likewise for y, with dx, dy measured in the point's local frame. An exact
 * zero joins neither sub-stencil (the inequalities are strict).
 */
int orc_split_stencils(int64_t n, const double *x, const double *y,
                       const double *nx, const double *ny,
                       const int32_t *off, const int32_t *idx, uint8_t *mask)
{
    for (int64_t p = 0; p < n; ++p) {
        for (int64_t e = off[p]; e < off[p + 1]; ++e) {
            int64_t i = idx[e];
            double dx = x[i] - x[p];
            double dy = y[i] - y[p];
            double ds = dx * ny[p] - dy * nx[p];
            double dn = dx * nx[p] + dy * ny[p];
            uint8_t m = 0;
            if (ds < 0.0) m |= ORC_XPOS;
            if (ds > 0.0) m |= ORC_XNEG;
            if (dn < 0.0) m |= ORC_YPOS;
            if (dn > 0.0) m |= ORC_YNEG;
            mask[e] = m;
        }
    }
    return ORC_OK;
}

/* threads of the OpenMP timing build (1 in the serial build) */
int orc_set_threads(int threads)
{
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
    return omp_get_max_threads();
#else
    (void)threads;
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* State conversions                                                        */
/* ------------------------------------------------------------------------ */

/* U = [rho, rho u1, rho u2, rho E] -> primitive (rho, u1, u2, p) */
static void prim_from_U(double gamma, const double U[4], double prim[4])
{
    double rho = U[0];
    double u1 = U[1] / rho;
    double u2 = U[2] / rho;
    double p = (gamma - 1.0) * (U[3] - 0.5 * rho * (u1 * u1 + u2 * u2));
    prim[0] = rho; prim[1] = u1; prim[2] = u2; prim[3] = p;
}

static void U_from_prim(double gamma, const double prim[4], double U[4])
{
    double rho = prim[0], u1 = prim[1], u2 = prim[2], p = prim[3];
    U[0] = rho;
    U[1] = rho * u1;
    U[2] = rho * u2;
    U[3] = p / (gamma - 1.0) + 0.5 * rho * (u1 * u1 + u2 * u2);
}

/* E13: q = [ln rho + ln(beta)/(gamma-1) - beta(u1^2+u2^2), 2 beta u1, 2 beta u2, -2 beta], beta = rho/(2p) */
static void q_from_prim(double gamma, const double prim[4], double q[4])
{
    double rho = prim[0], u1 = prim[1], u2 = prim[2], p = prim[3];
    double beta = 0.5 * rho / p;
    q[0] = log(rho) + log(beta) / (gamma - 1.0) - beta * (u1 * u1 + u2 * u2);
    q[1] = 2.0 * beta * u1;
    q[2] = 2.0 * beta * u2;
    q[3] = -2.0 * beta;
}

/* inverse of E13; returns 0 if q does not describe a physical state (beta <= 0) */
static int prim_from_q(double gamma, const double q[4], double prim[4])
{
    double beta = -0.5 * q[3];
    if (!(beta > 0.0)) return 0;
    double u1 = q[1] / (2.0 * beta);
    double u2 = q[2] / (2.0 * beta);
    double rho = exp(q[0] - log(beta) / (gamma - 1.0) + beta * (u1 * u1 + u2 * u2));
    double p = rho / (2.0 * beta);
    prim[0] = rho; prim[1] = u1; prim[2] = u2; prim[3] = p;
    return isfinite(rho) && rho > 0.0;
}

/* q_variables() of Algorithm 1 applied to a conserved state U[4][n] */
int orc_q_variables(int64_t n, double gamma, const double *U, double *q)
{
    int rc = ORC_OK;
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < n; ++p) {
        double u[4], pr[4], qq[4];
        for (int k = 0; k < 4; ++k) u[k] = U[k * n + p];
        prim_from_U(gamma, u, pr);
        if (!(pr[0] > 0.0) || !(pr[3] > 0.0)) {
#pragma omp atomic write
            rc = ORC_ERR_NONPHYSICAL;
            continue;
        }
        q_from_prim(gamma, pr, qq);
        for (int k = 0; k < 4; ++k) q[k * n + p] = qq[k];
    }
    return rc;
}

/* inverse map, q[4][n] -> U[4][n] (used by the round-trip checks) */
int orc_U_from_q(int64_t n, double gamma, const double *q, double *U)
{
    for (int64_t p = 0; p < n; ++p) {
        double qq[4], pr[4], u[4];
        for (int k = 0; k < 4; ++k) qq[k] = q[k * n + p];
        if (!prim_from_q(gamma, qq, pr)) return ORC_ERR_NONPHYSICAL;
        U_from_prim(gamma, pr, u);
        for (int k = 0; k < 4; ++k) U[k * n + p] = u[k];
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Kinetic split fluxes (the half-range moments of the Maxwellian behind    */
/* E2/E3; the paper cites them without printing them).                      */
/* Along a direction with normal velocity un and transverse velocity ut:    */
/*   beta = rho/(2p), S = un sqrt(beta), A+- = (1 +- erf S)/2,              */
/*   B = exp(-S^2)/(2 sqrt(pi beta)), rhoE = p/(gamma-1) + rho(un^2+ut^2)/2 */
/*   G+- = [ rho(un A +- B),                                                */
/*           (p + rho un^2) A +- rho un B,                                  */
/*           rho ut (un A +- B),                                            */
/*           (rhoE + p) un A +- (rhoE + p/2) B ]                            */
/* Components are ordered [mass, normal momentum, transverse momentum,      */
/* energy]. sign = +1 gives G+, sign = -1 gives G-.                         */
/* ------------------------------------------------------------------------ */
void orc_split_flux(double gamma, double rho, double un, double ut, double p,
                    int sign, double G[4])
{
    double beta = 0.5 * rho / p;
    double S = un * sqrt(beta);
    double s = (sign > 0) ? 1.0 : -1.0;
    double A = 0.5 * (1.0 + s * erf(S));
    double B = exp(-S * S) / (2.0 * sqrt(ORC_PI * beta));
    double rhoE = p / (gamma - 1.0) + 0.5 * rho * (un * un + ut * ut);
    G[0] = rho * (un * A + s * B);
    G[1] = (p + rho * un * un) * A + s * rho * un * B;
    G[2] = rho * ut * (un * A + s * B);
    G[3] = (rhoE + p) * un * A + s * (rhoE + 0.5 * p) * B;
}

/* Euler flux along a direction, same component order (split fluxes sum to it) */
void orc_euler_flux(double gamma, double rho, double un, double ut, double p, double G[4])
{
    double rhoE = p / (gamma - 1.0) + 0.5 * rho * (un * un + ut * ut);
    G[0] = rho * un;
    G[1] = p + rho * un * un;
    G[2] = rho * un * ut;
    G[3] = (rhoE + p) * un;
}

/* ------------------------------------------------------------------------ */
/* Stencil members. In the plain boundary reading the stencil of P_0 is its */
/* list of neighbours. The kinetic boundary mode (not in the paper, which   */
/* cites kinetic wall and far-field conditions without stating them;       */
/* reading) also gives a wall or far-field point the mirror image of every  */
/* neighbour across its tangent line: local offsets (ds, -dn), so the x+-   */
/* membership is kept and y+ and y- swap. A neighbour on the line (dn = 0)  */
/* is its own image and adds none. At a wall point the image carries the    */
/* specularly reflected gas: the velocity part (q1, q2) of q and every      */
/* gradient reflected across the line, so that the image of a field is     */
/* q*(P_0 + M d) = Mq(P_0 + d), M = I - 2 n n^T. At a far-field point the   */
/* image carries the free stream with zero gradient (the gas outside the    */
/* domain). The point is then treated by the interior formulas (all four    */
/* sub-stencils, the same least squares, limiter and reconstruction) on the */
/* augmented stencil.                                                       */
/* ------------------------------------------------------------------------ */
#define ORC_IMG_NONE 0
#define ORC_IMG_WALL 1
#define ORC_IMG_FAR 2

typedef struct {
    int64_t n;
    const double *x, *y;
    const double *nx, *ny;   /* NULL: no frame (gradients only, plain mode) */
    const int32_t *flags;    /* NULL: plain mode */
    const int32_t *off, *idx;
    const uint8_t *mask;     /* NULL: no sub-stencils (gradients only) */
    int kinetic;             /* 1: kinetic boundary mode */
    double qinf[4];          /* q of the free stream (kinetic mode) */
} orc_geom;

typedef struct {
    int64_t i;       /* the neighbour, or the neighbour whose image this is */
    int image;       /* ORC_IMG_* */
    double dx, dy;   /* offset from P_0, global frame */
    double ds, dn;   /* offset from P_0, frame of P_0 */
    uint8_t mask;    /* sub-stencils */
} orc_member;

static int64_t max_degree(const orc_geom *g)
{
    int64_t m = 0;
    for (int64_t p = 0; p < g->n; ++p)
        if (g->off[p + 1] - g->off[p] > m) m = g->off[p + 1] - g->off[p];
    return m;
}

static int is_kinetic_boundary(const orc_geom *g, int64_t p)
{
    return g->kinetic && (g->flags[p] == ORC_WALL || g->flags[p] == ORC_FARFIELD);
}

/* the members of the stencil of P_0 = p into mem[] (room for 2 x degree);
 * returns their number: the neighbours in CSR order, then the images */
static int64_t stencil_members(const orc_geom *g, int64_t p, orc_member *mem)
{
    double tx = 0.0, ty = 0.0, nnx = 0.0, nny = 0.0;
    if (g->nx) { tx = g->ny[p]; ty = -g->nx[p]; nnx = g->nx[p]; nny = g->ny[p]; }
    int64_t c = 0;
    for (int64_t e = g->off[p]; e < g->off[p + 1]; ++e) {
        orc_member *m = &mem[c++];
        m->i = g->idx[e];
        m->image = ORC_IMG_NONE;
        m->dx = g->x[m->i] - g->x[p];
        m->dy = g->y[m->i] - g->y[p];
        m->ds = m->dx * tx + m->dy * ty;
        m->dn = m->dx * nnx + m->dy * nny;
        m->mask = g->mask ? g->mask[e] : 0;
    }
    if (!is_kinetic_boundary(g, p)) return c;
    const int kind = g->flags[p] == ORC_WALL ? ORC_IMG_WALL : ORC_IMG_FAR;
    const int64_t nr = c;
    for (int64_t j = 0; j < nr; ++j) {
        const orc_member *r = &mem[j];
        if (r->dn == 0.0) continue;
        orc_member *m = &mem[c++];
        m->i = r->i;
        m->image = kind;
        m->dx = r->dx - 2.0 * r->dn * nnx;
        m->dy = r->dy - 2.0 * r->dn * nny;
        m->ds = r->ds;
        m->dn = -r->dn;
        m->mask = (uint8_t)((r->mask & (ORC_XPOS | ORC_XNEG)) | ((r->mask & ORC_YPOS) ? ORC_YNEG : 0u) |
                            ((r->mask & ORC_YNEG) ? ORC_YPOS : 0u));
    }
    return c;
}

/* reflect the vector (a, b) across the line with unit normal (nx, ny) */
static void reflect(double *a, double *b, double nx, double ny)
{
    double c = *a * nx + *b * ny;
    *a = *a - 2.0 * c * nx;
    *b = *b - 2.0 * c * ny;
}

/* q and its gradient (nullable inputs give zero) carried by a member of the
 * stencil of P_0 = p */
static void member_state(const orc_geom *g, int64_t p, const orc_member *m, const double *q,
                         const double *qx, const double *qy, double qi[4], double gx[4], double gy[4])
{
    const int64_t n = g->n;
    if (m->image == ORC_IMG_FAR) {
        for (int k = 0; k < 4; ++k) { qi[k] = g->qinf[k]; gx[k] = 0.0; gy[k] = 0.0; }
        return;
    }
    for (int k = 0; k < 4; ++k) {
        qi[k] = q[k * n + m->i];
        gx[k] = qx ? qx[k * n + m->i] : 0.0;
        gy[k] = qy ? qy[k * n + m->i] : 0.0;
    }
    if (m->image == ORC_IMG_WALL) {
        const double nx = g->nx[p], ny = g->ny[p];
        reflect(&qi[1], &qi[2], nx, ny);                              /* velocity part of q */
        for (int k = 0; k < 4; ++k) reflect(&gx[k], &gy[k], nx, ny);  /* d/dx of the image */
        reflect(&gx[1], &gx[2], nx, ny);                              /* and its velocity part */
        reflect(&gy[1], &gy[2], nx, ny);
    }
}

/* ------------------------------------------------------------------------ */
/* q_derivatives(): E15 with the modified variables of E14, solved by inner */
/* iterations. Iteration 0 is the first-order least-squares gradient (E9    */
/* with dq in place of dF~); each of the `inner` iterations that follow     */
/* evaluates the right side of E15 with the previous iterate at every point */
/* (Jacobi). orc_q_derivatives_pass is one such solve: with qx_old = NULL  */
/* it is the first-order one, else one inner iteration from qx_old, qy_old. */
/*   dq~_i = dq_i - 1/2 [dx_i (qx_i - qx_0) + dy_i (qy_i - qy_0)]            */
/* The full stencil N(P_0) does not depend on the frame and the 2x2 least-  */
/* squares gradient is rotation-equivariant, so this is done in the global  */
/* (x, y) frame and qx, qy are global-frame derivatives.                    */
/* ------------------------------------------------------------------------ */
static int q_derivatives_point(const orc_geom *g, int64_t p, const double *q, const double *qx_old,
                               const double *qy_old, double *qx, double *qy, orc_member *mem)
{
    const int64_t n = g->n;
    double sxx = 0.0, sxy = 0.0, syy = 0.0;
    double sxq[4] = {0, 0, 0, 0}, syq[4] = {0, 0, 0, 0};
    const int64_t cnt = stencil_members(g, p, mem);
    for (int64_t j = 0; j < cnt; ++j) {
        const orc_member *m = &mem[j];
        double dx = m->dx, dy = m->dy;
        double qi[4], gxi[4], gyi[4];
        member_state(g, p, m, q, qx_old, qy_old, qi, gxi, gyi);
        sxx += dx * dx;
        sxy += dx * dy;
        syy += dy * dy;
        for (int k = 0; k < 4; ++k) {
            double dq = qi[k] - q[k * n + p];
            if (qx_old) {
                dq = dq - 0.5 * (dx * (gxi[k] - qx_old[k * n + p])
                                 + dy * (gyi[k] - qy_old[k * n + p]));
            }
            sxq[k] += dx * dq;
            syq[k] += dy * dq;
        }
    }
    double det = sxx * syy - sxy * sxy;
    if (!(det > ORC_DET_EPS * sxx * syy)) return ORC_ERR_DEGENERATE;
    for (int k = 0; k < 4; ++k) {
        qx[k * n + p] = (syy * sxq[k] - sxy * syq[k]) / det;
        qy[k * n + p] = (sxx * syq[k] - sxy * sxq[k]) / det;
    }
    return ORC_OK;
}

/* room for the members of any stencil: the neighbours and their images */
static size_t member_room(const orc_geom *g)
{
    return (size_t)(2 * max_degree(g) + 1) * sizeof(orc_member);
}

/* keep the first error a thread met (any one of them, with threads) */
static void merge_status(int *rc, int mine)
{
    if (mine == ORC_OK) return;
#pragma omp critical(orc_status)
    {
        if (*rc == ORC_OK) *rc = mine;
    }
}

static int q_derivatives_pass(const orc_geom *g, const double *q, const double *qx_old,
                              const double *qy_old, double *qx, double *qy)
{
    const size_t room = member_room(g);
    int rc = ORC_OK;
#pragma omp parallel
    {
        orc_member *mem = (orc_member *)malloc(room);
        int mine = mem ? ORC_OK : -1;
#pragma omp for schedule(dynamic, 256)
        for (int64_t p = 0; p < g->n; ++p)
            if (mine == ORC_OK) mine = q_derivatives_point(g, p, q, qx_old, qy_old, qx, qy, mem);
        free(mem);
        merge_status(&rc, mine);
    }
    return rc;
}

static int q_derivatives(const orc_geom *g, const double *q, int inner, double *qx, double *qy)
{
    int rc = q_derivatives_pass(g, q, NULL, NULL, qx, qy);
    size_t bytes = (size_t)4 * (size_t)g->n * sizeof(double);
    double *ox = NULL, *oy = NULL;
    if (rc == ORC_OK && inner > 0) {
        ox = (double *)malloc(bytes);
        oy = (double *)malloc(bytes);
        if (!ox || !oy) rc = -1;
    }
    for (int it = 0; it < inner && rc == ORC_OK; ++it) {
        memcpy(ox, qx, bytes);
        memcpy(oy, qy, bytes);
        rc = q_derivatives_pass(g, q, ox, oy, qx, qy);
    }
    free(ox); free(oy);
    return rc;
}

static orc_geom plain_geom(int64_t n, const double *x, const double *y, const int32_t *off,
                           const int32_t *idx)
{
    orc_geom g;
    memset(&g, 0, sizeof g);
    g.n = n; g.x = x; g.y = y; g.off = off; g.idx = idx;
    return g;
}

int orc_q_derivatives_pass(int64_t n, const double *x, const double *y,
                           const int32_t *off, const int32_t *idx,
                           const double *q, const double *qx_old, const double *qy_old,
                           double *qx, double *qy)
{
    orc_geom g = plain_geom(n, x, y, off, idx);
    return q_derivatives_pass(&g, q, qx_old, qy_old, qx, qy);
}

int orc_q_derivatives(int64_t n, const double *x, const double *y,
                      const int32_t *off, const int32_t *idx,
                      const double *q, int inner, double *qx, double *qy)
{
    orc_geom g = plain_geom(n, x, y, off, idx);
    return q_derivatives(&g, q, inner, qx, qy);
}

/* ------------------------------------------------------------------------ */
/* Limiter (not in the paper; optional reading). The reconstruction of E14  */
/* moves q from P_0 by d = -1/2 dx_i.grad q_0 (as q~_0) and by +1/2 dx_i.   */
/* grad q_0 (when P_0 is the neighbour P_i of another point), for every     */
/* neighbour. Venkatakrishnan's limiter (J. Comput. Phys. 118, 1995)        */
/* scales each component's gradient at P_0 by                               */
/*   phi = min(1, min over all such d of f(d)),                             */
/*   f(d) = (D^2 + eps^2 + 2 D d) / (D^2 + 2 d^2 + D d + eps^2), d != 0,    */
/* with D = max(q over P_0 and N(P_0)) - q_0 for d > 0, min(...) - q_0 for  */
/* d < 0, and eps^2 = (K h)^3, h the distance to the nearest neighbour.     */
/* ------------------------------------------------------------------------ */
static double venkat(double D, double d, double eps2)
{
    return (D * D + eps2 + 2.0 * D * d) / (D * D + 2.0 * d * d + D * d + eps2);
}

static void limit_point(const orc_geom *g, int64_t p, const double *q, double K, double *qx,
                        double *qy, orc_member *mem)
{
    const int64_t n = g->n;
    const int64_t cnt = stencil_members(g, p, mem);
    double h = INFINITY;
    for (int64_t j = 0; j < cnt; ++j) {
        double d = sqrt(mem[j].dx * mem[j].dx + mem[j].dy * mem[j].dy);
        if (d < h) h = d;
    }
    double eps2 = (K * h) * (K * h) * (K * h);
    double qmax[4], qmin[4];
    for (int k = 0; k < 4; ++k) qmax[k] = qmin[k] = q[k * n + p];
    for (int64_t j = 0; j < cnt; ++j) {
        double qi[4], gxi[4], gyi[4];
        member_state(g, p, &mem[j], q, NULL, NULL, qi, gxi, gyi);
        for (int k = 0; k < 4; ++k) {
            if (qi[k] > qmax[k]) qmax[k] = qi[k];
            if (qi[k] < qmin[k]) qmin[k] = qi[k];
        }
    }
    for (int k = 0; k < 4; ++k) {
        double q0 = q[k * n + p];
        double phi = 1.0;
        for (int64_t j = 0; j < cnt; ++j) {
            double half = 0.5 * (mem[j].dx * qx[k * n + p] + mem[j].dy * qy[k * n + p]);
            for (int sgn = -1; sgn <= 1; sgn += 2) {
                double d = sgn * half;
                double f = 1.0;
                if (d > 0.0) f = venkat(qmax[k] - q0, d, eps2);
                else if (d < 0.0) f = venkat(qmin[k] - q0, d, eps2);
                if (f < phi) phi = f;
            }
        }
        qx[k * n + p] *= phi;
        qy[k * n + p] *= phi;
    }
}

/* each point scales only its own gradients and reads only q, so the points
 * are independent */
static int limit_gradients(const orc_geom *g, const double *q, double K, double *qx, double *qy)
{
    const size_t room = member_room(g);
    int rc = ORC_OK;
#pragma omp parallel
    {
        orc_member *mem = (orc_member *)malloc(room);
        int mine = mem ? ORC_OK : -1;
#pragma omp for schedule(dynamic, 256)
        for (int64_t p = 0; p < g->n; ++p)
            if (mine == ORC_OK) limit_point(g, p, q, K, qx, qy, mem);
        free(mem);
        merge_status(&rc, mine);
    }
    return rc;
}

int orc_limit_gradients(int64_t n, const double *x, const double *y, const int32_t *off,
                        const int32_t *idx, const double *q, double K, double *qx, double *qy)
{
    orc_geom g = plain_geom(n, x, y, off, idx);
    return limit_gradients(&g, q, K, qx, qy);
}

/* ------------------------------------------------------------------------ */
/* flux_residual(): E10 with E11/E12 and the q~ of E14.                     */
/* At point P_0 with frame (t, n), for each neighbour P_i:                  */
/*   q~_i = q_i - 1/2 (dx_i qx_i + dy_i qy_i),                              */
/*   q~_0 = q_0 - 1/2 (dx_i qx_0 + dy_i qy_0)   (order 2; order 1: q~ = q)  */
/* both converted to primitive variables, their velocities taken in the     */
/* frame of P_0 (u_s = u.t, u_n = u.n). On each sub-stencil the split-flux  */
/* perturbation dG_i = G(q~_i) - G(q~_0) enters E11:                        */
/*   dGs/ds = (S_nn S_s(dG) - S_sn S_n(dG)) / (S_ss S_nn - S_sn^2)          */
/*   dGn/dn = (S_ss S_n(dG) - S_sn S_s(dG)) / (S_ss S_nn - S_sn^2)          */
/* with S_ab the sums of products of the offsets ds_i, dn_i over that       */
/* sub-stencil. R = dGs+/ds + dGs-/ds + dGn+/dn + dGn-/dn, momentum rotated */
/* back to (x, y).                                                          */
/* Boundary reading (the paper states none): wall points (n into the fluid) */
/* drop dGn+/dn, which has no upwind points; far-field points get R = 0.    */
/* In the kinetic boundary mode both use all four terms on the stencil     */
/* augmented by their mirror images (stencil members above).               */
/* If `scale` is not NULL it receives, per point and component, the sum    */
/* over the terms of |LS weight_i| (|G(q~_i)| + |G(q~_0)|): the magnitude   */
/* of what is summed before cancellation (used to scale rounding tests).    */
/* ------------------------------------------------------------------------ */

/* split flux along direction d (0: s, 1: n) from a global-frame primitive
 * state, returned in the frame order [mass, s-momentum, n-momentum, energy] */
static void frame_split_flux(double gamma, const double prim[4], double tx, double ty,
                             double nx, double ny, int dir, int sign, double G[4])
{
    double us = prim[1] * tx + prim[2] * ty;
    double un = prim[1] * nx + prim[2] * ny;
    double g[4];
    if (dir == 0) {
        orc_split_flux(gamma, prim[0], us, un, prim[3], sign, g);
        G[0] = g[0]; G[1] = g[1]; G[2] = g[2]; G[3] = g[3];
    } else {
        orc_split_flux(gamma, prim[0], un, us, prim[3], sign, g);
        G[0] = g[0]; G[1] = g[2]; G[2] = g[1]; G[3] = g[3];
    }
}

/* q~ of E14 at a member (order 2; order 1: q~ = q) and at P_0 towards it */
static void reconstruct(const orc_geom *g, int64_t p, const orc_member *m, const double *q,
                        const double *qx, const double *qy, int order, double qt_i[4], double qt_0[4])
{
    const int64_t n = g->n;
    double qi[4], gxi[4], gyi[4];
    member_state(g, p, m, q, qx, qy, qi, gxi, gyi);
    for (int k = 0; k < 4; ++k) {
        if (order == 2) {
            qt_i[k] = qi[k] - 0.5 * (m->dx * gxi[k] + m->dy * gyi[k]);
            qt_0[k] = q[k * n + p] - 0.5 * (m->dx * qx[k * n + p] + m->dy * qy[k * n + p]);
        } else {
            qt_i[k] = qi[k];
            qt_0[k] = q[k * n + p];
        }
    }
}

static const uint8_t sub_bit[4] = {ORC_XPOS, ORC_XNEG, ORC_YPOS, ORC_YNEG};
static const int sub_dir[4] = {0, 0, 1, 1};
static const int sub_sign[4] = {+1, -1, +1, -1};

static int flux_residual_point(const orc_geom *g, int64_t p, double gamma, const double *q,
                               const double *qx, const double *qy, int order, double *R,
                               double *scale, orc_member *mem)
{
    const int64_t n = g->n;
    double Rl[4] = {0, 0, 0, 0}, Sc[4] = {0, 0, 0, 0};
    int flag = g->flags[p];
    int kinetic = is_kinetic_boundary(g, p);
    if (flag != ORC_FARFIELD || kinetic) {
        double tx = g->ny[p], ty = -g->nx[p], nnx = g->nx[p], nny = g->ny[p];
        const int64_t cnt = stencil_members(g, p, mem);
        for (int sub = 0; sub < 4; ++sub) {
            /* plain reading: no dGn+/dn at the wall */
            if (flag == ORC_WALL && !kinetic && sub == 2) continue;
            double sss = 0.0, ssn = 0.0, snn = 0.0;
            double ssG[4] = {0, 0, 0, 0}, snG[4] = {0, 0, 0, 0};
            for (int64_t j = 0; j < cnt; ++j) {
                const orc_member *m = &mem[j];
                if (!(m->mask & sub_bit[sub])) continue;
                double ds = m->ds, dn = m->dn;
                double qt_i[4], qt_0[4], pr_i[4], pr_0[4], Gi[4], G0[4];
                reconstruct(g, p, m, q, qx, qy, order, qt_i, qt_0);
                if (!prim_from_q(gamma, qt_i, pr_i) || !prim_from_q(gamma, qt_0, pr_0))
                    return ORC_ERR_NONPHYSICAL;
                frame_split_flux(gamma, pr_i, tx, ty, nnx, nny, sub_dir[sub], sub_sign[sub], Gi);
                frame_split_flux(gamma, pr_0, tx, ty, nnx, nny, sub_dir[sub], sub_sign[sub], G0);
                sss += ds * ds;
                ssn += ds * dn;
                snn += dn * dn;
                for (int k = 0; k < 4; ++k) {
                    double dG = Gi[k] - G0[k];
                    ssG[k] += ds * dG;
                    snG[k] += dn * dG;
                }
            }
            double det = sss * snn - ssn * ssn;
            if (!(det > ORC_DET_EPS * sss * snn)) return ORC_ERR_DEGENERATE;
            for (int k = 0; k < 4; ++k) {
                double d;
                if (sub_dir[sub] == 0) d = (snn * ssG[k] - ssn * snG[k]) / det;
                else d = (sss * snG[k] - ssn * ssG[k]) / det;
                Rl[k] += d;
            }
            if (scale) {
                for (int64_t j = 0; j < cnt; ++j) {
                    const orc_member *m = &mem[j];
                    if (!(m->mask & sub_bit[sub])) continue;
                    double ds = m->ds, dn = m->dn;
                    double w = (sub_dir[sub] == 0) ? (snn * ds - ssn * dn) / det
                                                   : (sss * dn - ssn * ds) / det;
                    double qt_i[4], qt_0[4], pr_i[4], pr_0[4], Gi[4], G0[4];
                    reconstruct(g, p, m, q, qx, qy, order, qt_i, qt_0);
                    prim_from_q(gamma, qt_i, pr_i);
                    prim_from_q(gamma, qt_0, pr_0);
                    frame_split_flux(gamma, pr_i, tx, ty, nnx, nny, sub_dir[sub], sub_sign[sub], Gi);
                    frame_split_flux(gamma, pr_0, tx, ty, nnx, nny, sub_dir[sub], sub_sign[sub], G0);
                    for (int k = 0; k < 4; ++k) Sc[k] += fabs(w) * (fabs(Gi[k]) + fabs(G0[k]));
                }
            }
        }
    }
    /* rotate the momentum components from (s, n) back to (x, y) */
    double tx = g->ny[p], ty = -g->nx[p];
    R[0 * n + p] = Rl[0];
    R[1 * n + p] = Rl[1] * tx + Rl[2] * g->nx[p];
    R[2 * n + p] = Rl[1] * ty + Rl[2] * g->ny[p];
    R[3 * n + p] = Rl[3];
    if (scale) {
        scale[0 * n + p] = Sc[0];
        scale[1 * n + p] = Sc[1] + Sc[2];
        scale[2 * n + p] = Sc[1] + Sc[2];
        scale[3 * n + p] = Sc[3];
    }
    return ORC_OK;
}

static int flux_residual(const orc_geom *g, double gamma, const double *q, const double *qx,
                         const double *qy, int order, double *R, double *scale)
{
    const size_t room = member_room(g);
    int rc = ORC_OK;
#pragma omp parallel
    {
        orc_member *mem = (orc_member *)malloc(room);
        int mine = mem ? ORC_OK : -1;
#pragma omp for schedule(dynamic, 256)
        for (int64_t p = 0; p < g->n; ++p)
            if (mine == ORC_OK) mine = flux_residual_point(g, p, gamma, q, qx, qy, order, R, scale, mem);
        free(mem);
        merge_status(&rc, mine);
    }
    return rc;
}

int orc_flux_residual(int64_t n, double gamma,
                      const double *x, const double *y, const double *nx, const double *ny,
                      const int32_t *flags, const int32_t *off, const int32_t *idx,
                      const uint8_t *mask, const double *q, const double *qx,
                      const double *qy, int order, double *R, double *scale)
{
    orc_geom g = plain_geom(n, x, y, off, idx);
    g.nx = nx; g.ny = ny; g.flags = flags; g.mask = mask;
    return flux_residual(&g, gamma, q, qx, qy, order, R, scale);
}

/* ------------------------------------------------------------------------ */
/* timestep(): local time step. The paper names the routine but not its    */
/* formula; reading: dt_0 = CFL min_i |P_i - P_0| / (|u_0| + 3 sqrt(p_0/rho_0)), */
/* the fastest molecular speed taken as three thermal speeds past the flow. */
/* ------------------------------------------------------------------------ */
int orc_timestep(int64_t n, double gamma, double cfl, const double *x, const double *y,
                 const int32_t *off, const int32_t *idx, const double *U, double *dt)
{
    int rc = ORC_OK;
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < n; ++p) {
        double u[4], pr[4];
        for (int k = 0; k < 4; ++k) u[k] = U[k * n + p];
        prim_from_U(gamma, u, pr);
        if (!(pr[0] > 0.0) || !(pr[3] > 0.0)) {
#pragma omp atomic write
            rc = ORC_ERR_NONPHYSICAL;
            continue;
        }
        double speed = sqrt(pr[1] * pr[1] + pr[2] * pr[2]) + 3.0 * sqrt(pr[3] / pr[0]);
        double dmin = INFINITY;
        for (int64_t e = off[p]; e < off[p + 1]; ++e) {
            int64_t i = idx[e];
            double dx = x[i] - x[p];
            double dy = y[i] - y[p];
            double d = sqrt(dx * dx + dy * dy);
            if (d < dmin) dmin = d;
        }
        dt[p] = cfl * dmin / speed;
    }
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Free stream (reading): rho = 1, p = 1/gamma (unit sound speed),         */
/* u = M (cos a, sin a).                                                    */
/* ------------------------------------------------------------------------ */
void orc_freestream(double gamma, double mach, double aoa_deg, double U[4])
{
    double a = aoa_deg * ORC_PI / 180.0;
    double prim[4] = {1.0, mach * cos(a), mach * sin(a), 1.0 / gamma};
    U_from_prim(gamma, prim, U);
}

/* boundary treatment after every update (reading): wall points lose their
 * normal momentum, far-field points are held at the free stream (plain
 * mode) or updated like the other points (kinetic boundary mode) */
static void apply_boundary(int64_t n, const int32_t *flags, const double *nx,
                           const double *ny, const double Uinf[4], int kinetic, double *U)
{
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < n; ++p) {
        if (flags[p] == ORC_WALL) {
            double mn = U[1 * n + p] * nx[p] + U[2 * n + p] * ny[p];
            U[1 * n + p] = U[1 * n + p] - mn * nx[p];
            U[2 * n + p] = U[2 * n + p] - mn * ny[p];
        } else if (flags[p] == ORC_FARFIELD && !kinetic) {
            for (int k = 0; k < 4; ++k) U[k * n + p] = Uinf[k];
        }
    }
}

/* residue(): L2 norm of the density residual over the points, divided by n
 * (reading; the paper gives the name only) */
double orc_residue(int64_t n, const double *R)
{
    double s = 0.0;
    for (int64_t p = 0; p < n; ++p) s += R[p] * R[p];
    return sqrt(s) / (double)n;
}

/* ------------------------------------------------------------------------ */
/* Time integration. A residual callback lets the same update rules be      */
/* checked on a residual with a known answer.                               */
/* ------------------------------------------------------------------------ */
typedef int (*orc_residual_fn)(const double *U, double *R, void *user);

/* E16, forward Euler with the local time step: U^{n+1} = U^n - dt R(U^n) */
static int euler_step(int64_t n, const int32_t *flags, const double *nx, const double *ny,
                      const double Uinf[4], int kinetic, const double *dt, double *U,
                      orc_residual_fn res, void *user, double *R0_out)
{
    double *R = (double *)malloc((size_t)4 * n * sizeof(double));
    if (!R) return -1;
    int rc = res(U, R, user);
    if (rc == ORC_OK) {
        for (int k = 0; k < 4; ++k)
#pragma omp parallel for schedule(static)
            for (int64_t p = 0; p < n; ++p)
                U[k * n + p] = U[k * n + p] - dt[p] * R[k * n + p];
        apply_boundary(n, flags, nx, ny, Uinf, kinetic, U);
        if (R0_out) memcpy(R0_out, R, (size_t)4 * n * sizeof(double));
    }
    free(R);
    return rc;
}

int orc_euler_step(int64_t n, const int32_t *flags, const double *nx, const double *ny,
                   const double Uinf[4], const double *dt, double *U,
                   orc_residual_fn res, void *user, double *R0_out)
{
    return euler_step(n, flags, nx, ny, Uinf, 0, dt, U, res, user, R0_out);
}

/* Classical four-stage Runge-Kutta with the local dt frozen at U^n (not in
 * the paper, which uses forward Euler; reading):
 *   U1 = U^n - dt/2 R(U^n), U2 = U^n - dt/2 R(U1), U3 = U^n - dt R(U2),
 *   U^{n+1} = U^n - dt/6 (R(U^n) + 2 R(U1) + 2 R(U2) + R(U3)),
 * the boundary treatment applied after every stage. */
static int rk4_step(int64_t n, const int32_t *flags, const double *nx, const double *ny,
                    const double Uinf[4], int kinetic, const double *dt, double *U,
                    orc_residual_fn res, void *user, double *R0_out)
{
    size_t bytes = (size_t)4 * n * sizeof(double);
    double *Un = (double *)malloc(bytes), *Us = (double *)malloc(bytes);
    double *R0 = (double *)malloc(bytes), *R1 = (double *)malloc(bytes);
    double *R2 = (double *)malloc(bytes), *R3 = (double *)malloc(bytes);
    int rc = -1;
    if (!Un || !Us || !R0 || !R1 || !R2 || !R3) goto done;
    memcpy(Un, U, bytes);
    rc = res(Un, R0, user);
    if (rc) goto done;
    for (int k = 0; k < 4; ++k)
#pragma omp parallel for schedule(static)
        for (int64_t p = 0; p < n; ++p) Us[k * n + p] = Un[k * n + p] - 0.5 * dt[p] * R0[k * n + p];
    apply_boundary(n, flags, nx, ny, Uinf, kinetic, Us);
    rc = res(Us, R1, user);
    if (rc) goto done;
    for (int k = 0; k < 4; ++k)
#pragma omp parallel for schedule(static)
        for (int64_t p = 0; p < n; ++p) Us[k * n + p] = Un[k * n + p] - 0.5 * dt[p] * R1[k * n + p];
    apply_boundary(n, flags, nx, ny, Uinf, kinetic, Us);
    rc = res(Us, R2, user);
    if (rc) goto done;
    for (int k = 0; k < 4; ++k)
#pragma omp parallel for schedule(static)
        for (int64_t p = 0; p < n; ++p) Us[k * n + p] = Un[k * n + p] - dt[p] * R2[k * n + p];
    apply_boundary(n, flags, nx, ny, Uinf, kinetic, Us);
    rc = res(Us, R3, user);
    if (rc) goto done;
    for (int k = 0; k < 4; ++k)
#pragma omp parallel for schedule(static)
        for (int64_t p = 0; p < n; ++p) {
            int64_t a = k * n + p;
            U[a] = Un[a] - dt[p] / 6.0 * (R0[a] + 2.0 * R1[a] + 2.0 * R2[a] + R3[a]);
        }
    apply_boundary(n, flags, nx, ny, Uinf, kinetic, U);
    if (R0_out) memcpy(R0_out, R0, bytes);
done:
    free(Un); free(Us); free(R0); free(R1); free(R2); free(R3);
    return rc;
}

int orc_rk4_step(int64_t n, const int32_t *flags, const double *nx, const double *ny,
                 const double Uinf[4], const double *dt, double *U,
                 orc_residual_fn res, void *user, double *R0_out)
{
    return rk4_step(n, flags, nx, ny, Uinf, 0, dt, U, res, user, R0_out);
}

/* ------------------------------------------------------------------------ */
/* The residual of the whole scheme: q_variables, q_derivatives,            */
/* flux_residual (Algorithm 1).                                             */
/* ------------------------------------------------------------------------ */
typedef struct {
    orc_geom g;
    double gamma;
    int order, inner;
    double limiter_K; /* > 0: Venkatakrishnan limiter with this K */
    double *q, *qx, *qy;
} orc_scheme;

static int scheme_residual(const double *U, double *R, void *user)
{
    orc_scheme *s = (orc_scheme *)user;
    int rc = orc_q_variables(s->g.n, s->gamma, U, s->q);
    if (rc) return rc;
    if (s->order == 2) {
        rc = q_derivatives(&s->g, s->q, s->inner, s->qx, s->qy);
        if (rc) return rc;
        if (s->limiter_K > 0.0) limit_gradients(&s->g, s->q, s->limiter_K, s->qx, s->qy);
    }
    return flux_residual(&s->g, s->gamma, s->q, s->qx, s->qy, s->order, R, NULL);
}

/* q of the free stream, by the same conversion as a point held at U_inf */
static void freestream_q(double gamma, double mach, double aoa_deg, double q[4])
{
    double U[4], pr[4];
    orc_freestream(gamma, mach, aoa_deg, U);
    prim_from_U(gamma, U, pr);
    q_from_prim(gamma, pr, q);
}

static orc_geom scheme_geom(int64_t n, const double *x, const double *y, const double *nx,
                            const double *ny, const int32_t *flags, const int32_t *off,
                            const int32_t *idx, const uint8_t *mask, int boundary, double gamma,
                            double mach, double aoa_deg)
{
    orc_geom g = plain_geom(n, x, y, off, idx);
    g.nx = nx; g.ny = ny; g.flags = flags; g.mask = mask;
    g.kinetic = boundary == 1;
    if (g.kinetic) freestream_q(gamma, mach, aoa_deg, g.qinf);
    return g;
}

/* one residual evaluation R(U); qx, qy (nullable) receive the derivatives.
 * boundary: 0 plain reading, 1 kinetic boundary mode (mach and aoa_deg give
 * the free stream of the far-field images) */
int orc_residual_bc(int64_t n, double gamma, const double *x, const double *y,
                    const double *nx, const double *ny, const int32_t *flags,
                    const int32_t *off, const int32_t *idx, const uint8_t *mask,
                    int order, int inner, double limiter_K, int boundary, double mach,
                    double aoa_deg, const double *U, double *R, double *scale,
                    double *qx_out, double *qy_out)
{
    orc_geom g = scheme_geom(n, x, y, nx, ny, flags, off, idx, mask, boundary, gamma, mach, aoa_deg);
    size_t bytes = (size_t)4 * n * sizeof(double);
    double *q = (double *)malloc(bytes), *qx = (double *)calloc(4 * (size_t)n, sizeof(double));
    double *qy = (double *)calloc(4 * (size_t)n, sizeof(double));
    int rc = -1;
    if (!q || !qx || !qy) goto done;
    rc = orc_q_variables(n, gamma, U, q);
    if (rc) goto done;
    if (order == 2) {
        rc = q_derivatives(&g, q, inner, qx, qy);
        if (rc) goto done;
        if (limiter_K > 0.0) limit_gradients(&g, q, limiter_K, qx, qy);
    }
    rc = flux_residual(&g, gamma, q, qx, qy, order, R, scale);
    if (qx_out) memcpy(qx_out, qx, bytes);
    if (qy_out) memcpy(qy_out, qy, bytes);
done:
    free(q); free(qx); free(qy);
    return rc;
}

int orc_residual(int64_t n, double gamma, const double *x, const double *y,
                 const double *nx, const double *ny, const int32_t *flags,
                 const int32_t *off, const int32_t *idx, const uint8_t *mask,
                 int order, int inner, double limiter_K, const double *U, double *R,
                 double *scale, double *qx_out, double *qy_out)
{
    return orc_residual_bc(n, gamma, x, y, nx, ny, flags, off, idx, mask, order, inner, limiter_K, 0,
                           0.0, 0.0, U, R, scale, qx_out, qy_out);
}

/* ------------------------------------------------------------------------ */
/* Forces (reading; the paper reduces lift and drag but gives no formula):  */
/* Cp_i = (p_i - p_inf)/(rho_inf V_inf^2 / 2) at the wall points in contour */
/* order, ds_i = (|P_{i+1} - P_i| + |P_i - P_{i-1}|)/2 on the closed        */
/* contour, c = -sum Cp_i n_i ds_i (n into the fluid, unit chord),          */
/* Cl = c_y cos a - c_x sin a, Cd = c_x cos a + c_y sin a.                  */
/* ------------------------------------------------------------------------ */
int orc_forces(int64_t n, double gamma, double mach, double aoa_deg, const double *U,
               const double *x, const double *y, const double *nx, const double *ny,
               int64_t nwall, const int32_t *wall_order, double *cl, double *cd, double *cp)
{
    double a = aoa_deg * ORC_PI / 180.0;
    double rho_inf = 1.0, p_inf = 1.0 / gamma, V = mach;
    double qinf = 0.5 * rho_inf * V * V;
    double cx = 0.0, cy = 0.0;
    for (int64_t w = 0; w < nwall; ++w) {
        int64_t p = wall_order[w];
        int64_t pn = wall_order[(w + 1) % nwall];
        int64_t pp = wall_order[(w + nwall - 1) % nwall];
        double u[4], pr[4];
        for (int k = 0; k < 4; ++k) u[k] = U[k * n + p];
        prim_from_U(gamma, u, pr);
        double c = (pr[3] - p_inf) / qinf;
        double dsn = sqrt((x[pn] - x[p]) * (x[pn] - x[p]) + (y[pn] - y[p]) * (y[pn] - y[p]));
        double dsp = sqrt((x[p] - x[pp]) * (x[p] - x[pp]) + (y[p] - y[pp]) * (y[p] - y[pp]));
        double ds = 0.5 * (dsn + dsp);
        cx -= c * nx[p] * ds;
        cy -= c * ny[p] * ds;
        if (cp) cp[w] = c;
    }
    *cl = cy * cos(a) - cx * sin(a);
    *cd = cx * cos(a) + cy * sin(a);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* The solver loop of Algorithm 1: per iteration q_variables,               */
/* q_derivatives, flux_residual, timestep, state_update, residue.           */
/* scheme 0: forward Euler (E16); scheme 1: RK4 (reading above).            */
/* boundary 0: plain reading; 1: kinetic boundary mode (stencil members).  */
/* U[4][n] holds the initial state on entry and the final one on exit;      */
/* res_history[it] (nullable) receives residue() of R(U^it).                */
/* ------------------------------------------------------------------------ */
int orc_solve_bc(int64_t n, double gamma, const double *x, const double *y,
                 const double *nx, const double *ny, const int32_t *flags,
                 const int32_t *off, const int32_t *idx, const uint8_t *mask,
                 int order, int inner, double limiter_K, int boundary, int scheme, double cfl,
                 double mach, double aoa_deg, int n_iters, double *U, double *res_history)
{
    size_t bytes = (size_t)4 * n * sizeof(double);
    orc_scheme s;
    s.g = scheme_geom(n, x, y, nx, ny, flags, off, idx, mask, boundary, gamma, mach, aoa_deg);
    s.gamma = gamma;
    s.order = order; s.inner = inner; s.limiter_K = limiter_K;
    s.q = (double *)malloc(bytes);
    s.qx = (double *)calloc(4 * (size_t)n, sizeof(double));
    s.qy = (double *)calloc(4 * (size_t)n, sizeof(double));
    double *dt = (double *)malloc((size_t)n * sizeof(double));
    double *R0 = (double *)malloc(bytes);
    double Uinf[4];
    int rc = -1;
    if (!s.q || !s.qx || !s.qy || !dt || !R0) goto done;
    orc_freestream(gamma, mach, aoa_deg, Uinf);
    rc = ORC_OK;
    for (int it = 0; it < n_iters && rc == ORC_OK; ++it) {
        rc = orc_timestep(n, gamma, cfl, x, y, off, idx, U, dt);
        if (rc) break;
        if (scheme == 1) rc = rk4_step(n, flags, nx, ny, Uinf, s.g.kinetic, dt, U, scheme_residual, &s, R0);
        else rc = euler_step(n, flags, nx, ny, Uinf, s.g.kinetic, dt, U, scheme_residual, &s, R0);
        if (rc) break;
        if (res_history) res_history[it] = orc_residue(n, R0);
    }
done:
    free(s.q); free(s.qx); free(s.qy); free(dt); free(R0);
    return rc;
}

int orc_solve(int64_t n, double gamma, const double *x, const double *y,
              const double *nx, const double *ny, const int32_t *flags,
              const int32_t *off, const int32_t *idx, const uint8_t *mask,
              int order, int inner, double limiter_K, int scheme, double cfl, double mach,
              double aoa_deg, int n_iters, double *U, double *res_history)
{
    return orc_solve_bc(n, gamma, x, y, nx, ny, flags, off, idx, mask, order, inner, limiter_K, 0, scheme,
                        cfl, mach, aoa_deg, n_iters, U, res_history);
}
