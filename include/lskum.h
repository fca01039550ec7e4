/*
 * lskum.h - C ABI of the GB300 (sm_103a) q-LSKUM hot path.
 *
 * q-LSKUM (arXiv 2403.13287, Sec. 2 and Algorithm 1): meshfree least-squares
 * kinetic upwind method for the 2D Euler equations on a point cloud. Per
 * pseudo-time iteration and per point: q-variables (E13), least-squares
 * q-derivatives with defect-correction inner iterations (E14, E15), the sum
 * of kinetic split-flux derivatives over the x+-/y+- sub-stencils (E10-E12),
 * a local time step and the state update (E16; or RK4).
 *
 * Conventions shared by every call
 * - Points are numbered 0..n-1 in the caller's ("input") order; every array
 *   the caller sees is in input order. The library may renumber points
 *   internally (lskum_config.reorder) and keeps the permutation to itself.
 * - Arrays of the four conserved variables U = [rho, rho u, rho v, rho E]
 *   (and of residuals, q-derivatives) are component-major: A[k*n + p].
 * - "device" pointers are CUDA device memory owned by the caller (e.g. a
 *   contiguous torch tensor's data_ptr()); they are used on the context's
 *   stream, asynchronously, unless a call says it synchronises. "host"
 *   pointers are ordinary CPU memory.
 * - Host input arrays passed to lskum_create are copied; the caller keeps
 *   ownership. The context owns all of its device workspace.
 * - Every call returns an lskum_status; the library never aborts or exits.
 *   After a failure lskum_last_error() describes it (per context).
 * - Calls on one context are not thread-safe; different contexts are
 *   independent.
 */
#ifndef LSKUM_H
#define LSKUM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LSKUM_OK = 0,
    LSKUM_ERR_ARG = 1,                /* bad argument (null pointer, size, config value) */
    LSKUM_ERR_CONNECTIVITY = 2,       /* CSR malformed: index out of range, self loop, duplicate, degree > 25 */
    LSKUM_ERR_DEGENERATE_STENCIL = 3, /* a needed (sub-)stencil has a singular 2x2 least-squares matrix */
    LSKUM_ERR_CUDA = 4,               /* a CUDA runtime call failed */
    LSKUM_ERR_OOM = 5,                /* device allocation failed */
    LSKUM_ERR_NONPHYSICAL = 6,        /* a state with rho <= 0, p <= 0 (FP64 form: p/rho outside
                                         [1e-307, 1e307]) or a non-finite value appeared */
    LSKUM_ERR_TIMEOUT = 7             /* a bounded device-side wait ran out */
} lskum_status;

/* point flags */
#define LSKUM_POINT_INTERIOR 0
#define LSKUM_POINT_WALL 1     /* on the body; normal points into the fluid */
#define LSKUM_POINT_FARFIELD 2 /* outer boundary; normal points out of the domain */

/* sub-stencil bits of lskum_get_stencil_masks (Sec. 2, after E12), measured in
 * the point's frame: tangent t = (ny, -nx), normal n = (nx, ny) */
#define LSKUM_MASK_XPOS 1u /* ds < 0 : upwind points of Gx+ */
#define LSKUM_MASK_XNEG 2u /* ds > 0 : upwind points of Gx- */
#define LSKUM_MASK_YPOS 4u /* dn < 0 : upwind points of Gy+ */
#define LSKUM_MASK_YNEG 8u /* dn > 0 : upwind points of Gy- */

#define LSKUM_MAX_DEGREE 25

typedef struct {
    int order;        /* 1: first-order LSKUM (dG uses q); 2: q-LSKUM (dG uses q~ of E14) */
    int inner_iters;  /* inner iterations of E15 after the first-order solve (paper: 3) */
    int time_scheme;  /* 0: forward Euler with local dt (E16); 1: classical RK4 with dt frozen per iteration */
    double cfl;       /* local time step dt = cfl * min|P_i - P_0| / (|u| + 3 sqrt(p/rho)) */
    double mach;      /* free stream: rho = 1, p = 1/gamma, |u| = mach */
    double aoa_deg;   /* angle of attack of the free stream, degrees */
    double gamma;     /* ratio of specific heats (paper: 1.4) */
    int precision;    /* 0: FP64 throughout. 1: mixed (not in the paper): q, grad q, the LS
                       * weights and the split-flux arithmetic in FP32; U, the RK update, the
                       * residue, the forces and the LS closure of points whose sub-stencil
                       * weights amplify rounding (sum |w_i||P_i - P_0| > 16) in FP64 */
    int reorder;      /* internal numbering for gather locality: 0 the input order; 1 Morton (Z-order) of
                       * the coordinates; 2 reverse Cuthill-McKee of the stencil graph (a batch keeps
                       * each case's points together in either) */
    double limiter_K; /* order 2 only. 0: no limiter (the paper's scheme). > 0: Venkatakrishnan's
                       * limiter (J. Comput. Phys. 118, 1995; not in the paper) scales each
                       * component of grad q at P_0 by phi = min(1, f(D+, d+), f(D-, -d+)),
                       * f(D, d) = (D^2 + e^2 + 2Dd)/(D^2 + 2d^2 + Dd + e^2), d+ the largest
                       * |(P_i - P_0).grad q|/2, D+- = max/min of q over P_0 and N(P_0) minus
                       * q_0, e^2 = (K h)^3, h the nearest-neighbour distance */
    int boundary;     /* LSKUM_BOUNDARY_PLAIN or LSKUM_BOUNDARY_KINETIC (below) */
} lskum_config;

/*
 * Boundary treatment (the paper cites kinetic wall and far-field conditions
 * after E10 without stating them).
 * LSKUM_BOUNDARY_PLAIN: a wall point drops dGy+/dy (no upwind points inside
 *   the body) and loses its normal momentum after every update; far-field
 *   points are held at the free stream.
 * LSKUM_BOUNDARY_KINETIC: a wall or far-field point P_0 also sees the mirror
 *   image of each neighbour P_i across its tangent line (local offsets
 *   (ds_i, -dn_i); a neighbour with dn_i = 0 is its own image and adds none).
 *   At a wall point the image carries the specularly reflected gas (the
 *   velocity part of q and every gradient reflected across the line); at a
 *   far-field point it carries the free stream with zero gradient. The point
 *   then takes the interior formulas on the augmented stencil: q-derivatives
 *   (E15), limiter, all four split-flux derivatives (E10-E12). Far-field
 *   points are updated like interior points; wall points still lose their
 *   normal momentum. The derivative calls (lskum_residual_vjp,
 *   lskum_step_vjp) need LSKUM_BOUNDARY_PLAIN.
 */
#define LSKUM_BOUNDARY_PLAIN 0
#define LSKUM_BOUNDARY_KINETIC 1

typedef struct lskum_ctx lskum_ctx;

/*
 * Build a solver context on the current CUDA device (Sec. 3: preprocessor()).
 *   n                      number of points (>= 1, < 2^31)
 *   x, y, nx, ny           host float64[n]: coordinates and unit normals
 *   flags                  host int32[n]: LSKUM_POINT_*
 *   nbr_offsets            host int32[n+1]: CSR row starts, nbr_offsets[0] = 0
 *   nbr_idx                host int32[nbr_offsets[n]]: neighbour lists N(P_0); the
 *                          order within a row is the summation order of every
 *                          least-squares sum at that point
 *   n_wall, wall_order     host int32[n_wall]: wall points in contour order
 *                          (closed contour; used by lskum_forces). n_wall may be 0.
 *   cfg                    host; copied
 *   cuda_stream            cudaStream_t to run on, or NULL for the legacy default stream
 *   out                    receives the context (NULL on failure)
 * Validates the CSR (LSKUM_ERR_CONNECTIVITY) and every needed stencil: the full
 * stencil at every point, N_x+, N_x-, N_y+, N_y- at interior points and N_x+,
 * N_x-, N_y- at wall points must have det > 1e-10 * Sxx * Syy
 * (LSKUM_ERR_DEGENERATE_STENCIL; the message names the first bad point). In
 * the kinetic boundary mode wall and far-field points need all five stencils,
 * each augmented by the mirror images.
 * Initialises the state to the free stream. Synchronises.
 */
lskum_status lskum_create(int64_t n, const double *x, const double *y, const double *nx,
                          const double *ny, const int32_t *flags, const int32_t *nbr_offsets,
                          const int32_t *nbr_idx, int64_t n_wall, const int32_t *wall_order,
                          const lskum_config *cfg, void *cuda_stream, lskum_ctx **out);

/*
 * One case of a batch: a cloud (as for lskum_create) and its free stream.
 * Cases may share their arrays (e.g. one cloud under several flow conditions).
 */
typedef struct {
    int64_t n;                      /* points of this case (>= 32) */
    const double *x, *y, *nx, *ny;  /* host float64[n] */
    const int32_t *flags;           /* host int32[n] */
    const int32_t *nbr_offsets;     /* host int32[n+1], this case's own numbering */
    const int32_t *nbr_idx;         /* host int32[nbr_offsets[n]] */
    int64_t n_wall;                 /* wall points (closed contour) or 0 */
    const int32_t *wall_order;      /* host int32[n_wall] */
    double mach, aoa_deg;           /* this case's free stream (cfg.mach/aoa_deg are not used) */
} lskum_case;

/*
 * Build one context that advances n_cases independent solves together (not in
 * the paper): every kernel runs once over the disjoint union of the cases'
 * clouds, so small and uneven cases share launches and graph replays. The
 * context's points are the cases' points concatenated in case order (case k
 * occupies [first_k, first_k + n_k) of every caller-visible array, see
 * lskum_case_range); the connectivity stays within each case. Each case has
 * its own free stream (far-field values, initial state, forces), residue and
 * wall contour; cfg supplies everything else. lskum_step's res_history then
 * holds n_iters * n_cases values, iteration-major (res[it * n_cases + k]);
 * lskum_residual, lskum_residual_vjp, lskum_get_state/set_state and the
 * timing calls act on all cases at once; forces come from lskum_case_forces.
 * Validation and errors as lskum_create, per case. Synchronises.
 *   n_cases   1 .. 65535
 */
lskum_status lskum_create_batch(int n_cases, const lskum_case *cases, const lskum_config *cfg, void *cuda_stream,
                                lskum_ctx **out);

/* Number of cases of a context (1 for lskum_create). */
int lskum_case_count(const lskum_ctx *ctx);

/* Input-order point range and wall-entry range of case k (any pointer may be NULL). */
lskum_status lskum_case_range(const lskum_ctx *ctx, int k, int64_t *first, int64_t *count, int64_t *wall_first,
                              int64_t *wall_count);

/* Free everything the context owns. NULL is allowed. */
void lskum_destroy(lskum_ctx *ctx);

/* Last error message of this context ("" if none); valid until the next call on it. */
const char *lskum_last_error(const lskum_ctx *ctx);

/*
 * Run n_iters pseudo-time iterations of Algorithm 1 on the context's state:
 * per iteration q_variables, q_derivatives (order 2), flux_residual, timestep
 * and state_update (forward Euler, E16, or RK4), then residue().
 *   res_history  host float64[n_iters] or NULL: residue of each iteration,
 *                sqrt(sum_p R_rho(U^n)_p^2) / n
 * Wall points lose their normal momentum after every update; far-field points
 * are held at the free stream (plain boundary mode) or updated (kinetic
 * mode). Synchronises once at the end. On
 * LSKUM_ERR_NONPHYSICAL the state is rolled back to its value at entry.
 */
lskum_status lskum_step(lskum_ctx *ctx, int n_iters, double *res_history);

/*
 * Residual R(U) = dGx+/dx + dGx-/dx + dGy+/dy + dGy-/dy of E10 (q~ of E14 for
 * order 2), momentum in global (x, y) components; far-field points get 0 in
 * the plain boundary mode.
 *   U  device float64[4*n] in input order, or NULL for the context's state
 *   R  device float64[4*n] in input order (written)
 * Does not change the context's state (its scratch buffers are reused).
 */
lskum_status lskum_residual(lskum_ctx *ctx, const double *U, double *R);

/*
 * Vector-Jacobian product of the residual above (the E10 residual with E11
 * closures, the E14 reconstruction and the E15 q-derivatives, differentiated
 * in reverse): for a cotangent R_bar,
 *   U_bar = (dR/dU)^T R_bar,  x_bar = (dR/dx)^T R_bar,  y_bar = (dR/dy)^T R_bar.
 * The derivative in x and y holds the frame normals, the connectivity and the
 * sub-stencil membership fixed (they are inputs, not functions of x and y).
 * Computed in FP64 whatever the context's precision, for the FP64 residual,
 * unless flags has LSKUM_VJP_FP32 (mixed contexts only).
 *   U      device float64[4*n] in input order, or NULL for the context's state
 *   R_bar  device float64[4*n] in input order
 *   U_bar  device float64[4*n] in input order (written), or NULL
 *   x_bar, y_bar  device float64[n] in input order (written, or added into with
 *                 LSKUM_VJP_ACCUMULATE_XY), or NULL
 *   flags  0, or LSKUM_VJP_ACCUMULATE_XY and/or LSKUM_VJP_FP32
 * With limiter_K > 0 the limiter is differentiated too (FP64 product only;
 * LSKUM_ERR_ARG with LSKUM_VJP_FP32): it is piecewise smooth, and the
 * product is that of the branch the forward takes, with the forward's
 * choices (the first stencil extremum, the first largest reconstruction
 * shift, the first nearest neighbour in row order). Its workspace (about
 * 0.53 KB per point plus 88 B per edge for K = 3: 0.8 GB at 640k points;
 * 0.16 KB per point more with the limiter) is allocated on the first call
 * and kept. The kinetic boundary mode is not differentiated (LSKUM_ERR_ARG).
 * Does not change the context's state.
 */
#define LSKUM_VJP_ACCUMULATE_XY 1 /* flags: add into x_bar, y_bar instead of overwriting them */
#define LSKUM_VJP_FP32 2          /* lskum_residual_vjp flags: the product in FP32 (mixed contexts): q, the
                                   * q-derivative iterates (the mixed form's FP32 passes) and the reverse pass
                                   * in FP32; geometry cotangents and the E13 Jacobian in FP64. U_bar agrees
                                   * with the FP64 product to ~1e-4 of its largest entry; x_bar, y_bar only to
                                   * ~1e-2 (the FP32 flux differences in the weight cotangents cancel), so
                                   * coordinate gradients should use the FP64 product */

lskum_status lskum_residual_vjp(lskum_ctx *ctx, const double *U, const double *R_bar, double *U_bar,
                                double *x_bar, double *y_bar, int flags);

/*
 * Vector-Jacobian product of one pseudo-time iteration, the map U^n -> U^{n+1}
 * that lskum_step(ctx, 1, .) applies: residual(s), local time step frozen at
 * U^n (its nearest-neighbour distance differentiated through the nearest
 * neighbour, the first of equals in row order), forward Euler (E16) or the
 * four RK4 stages, the wall projection after every stage and the far-field
 * reset. For the cotangent U_bar_next of U^{n+1}:
 *   U_bar = (dU^{n+1}/dU^n)^T U_bar_next,  x_bar, y_bar likewise.
 * Differentiates the FP64 scheme whatever the context's precision; the stage
 * states are recomputed in FP64. Frame normals, connectivity and sub-stencil
 * membership are held fixed, as in lskum_residual_vjp, and the limiter is
 * differentiated as there.
 *   U           device float64[4*n] in input order, or NULL for the context's state
 *   U_bar_next  device float64[4*n] in input order
 *   U_bar       device float64[4*n] in input order (written), or NULL
 *   x_bar, y_bar  device float64[n] in input order (written, or added into with
 *                 flags = LSKUM_VJP_ACCUMULATE_XY), or NULL
 * Workspace: about 0.45 KB per point more than lskum_residual_vjp, allocated on
 * the first call. Does not change the context's state.
 */
lskum_status lskum_step_vjp(lskum_ctx *ctx, const double *U, const double *U_bar_next, double *U_bar,
                            double *x_bar, double *y_bar, int flags);

/*
 * Vector-Jacobian product of the lift and drag of case k (lskum_case_forces;
 * k = 0 for a single context) at the context's state:
 *   U_bar = cl_bar dCl/dU + cd_bar dCd/dU,  x_bar, y_bar likewise
 * (only wall points have non-zero entries; the frame normals are held fixed
 * and the arc-length weights ds are differentiated).
 *   U_bar, x_bar, y_bar  device float64 in input order ([4*n], [n], [n]; written), or NULL
 *   flags  0 or LSKUM_VJP_ACCUMULATE_XY (add into x_bar, y_bar)
 */
lskum_status lskum_forces_vjp(lskum_ctx *ctx, int k, double cl_bar, double cd_bar, double *U_bar, double *x_bar,
                              double *y_bar, int flags);

/*
 * q-derivatives of E15 (global x, y frame) after the configured inner
 * iterations (order 2) or the first-order solve (order 1), for state U.
 *   U       device float64[4*n] or NULL (context state)
 *   qx, qy  device float64[4*n], written
 */
lskum_status lskum_q_derivatives(lskum_ctx *ctx, const double *U, double *qx, double *qy);

/* Local time step of every point for state U (device [4*n] or NULL) into dt (device float64[n]). */
lskum_status lskum_timestep(lskum_ctx *ctx, const double *U, double *dt);

/*
 * Lift and drag of the current state: Cp_i = (p_i - p_inf) / (rho_inf |u_inf|^2 / 2)
 * at the wall points in contour order, c = -sum_i Cp_i n_i ds_i with
 * ds_i = (|P_{i+1} - P_i| + |P_i - P_{i-1}|) / 2, Cl = c_y cos a - c_x sin a,
 * Cd = c_x cos a + c_y sin a.
 *   cl, cd  host double*, written
 *   cp      host float64[n_wall] or NULL, in wall_order order
 * Synchronises.
 */
lskum_status lskum_forces(lskum_ctx *ctx, double *cl, double *cd, double *cp);

/* Copy the state out of / into the context. U is float64[4*n] in input order,
 * host memory if on_host != 0 else device memory. set_state synchronises for
 * host input; q-variables are refreshed from the new state. */
lskum_status lskum_get_state(lskum_ctx *ctx, double *U, int on_host);
lskum_status lskum_set_state(lskum_ctx *ctx, const double *U, int on_host);

/* Sub-stencil masks computed at create, one byte per CSR entry of the input
 * connectivity (LSKUM_MASK_* bits), written to host uint8[nnz]. Synchronises. */
lskum_status lskum_get_stencil_masks(lskum_ctx *ctx, uint8_t *mask);

/* Internal numbering: perm[new] = input index of internal point `new`
 * (host int32[n]). Identity when reorder = 0. Synchronises. */
lskum_status lskum_get_permutation(lskum_ctx *ctx, int32_t *perm);

/* Number of kernel launches the library has issued on this context so far. */
int64_t lskum_launch_count(const lskum_ctx *ctx);

/*
 * q-derivatives without any device allocation, for callers that cannot
 * allocate device memory where they call from: a framework whose caching
 * allocator owns the GPU's memory, a step loop that must not pay the device
 * synchronisation that cudaMalloc/cudaFree imply, or a process that was
 * handed a fixed memory budget. It needs no context either. The paper has no
 * counterpart: this is a plumbing variant of lskum_q_derivatives.
 *
 * Computes the q-variables from U and their least-squares derivatives, with
 * the same arithmetic as lskum_q_derivatives of an unlimited context (the
 * first-order solve, then inner_iters Jacobi inner iterations), in the global
 * frame, with the 2x2 sums formed on the fly. All pointers are caller-owned
 * device memory, in the caller's numbering:
 *   n                     number of points, 1 <= n <= LSKUM_NOALLOC_MAX_POINTS
 *   x, y                  float64[n]
 *   nbr_offsets, nbr_idx  int32[n+1], int32[nbr_offsets[n]]: a CSR. nbr_idx must
 *                         hold nbr_offsets[n] entries (the caller's
 *                         responsibility: a plain pointer carries no size).
 *                         A row that runs backwards, leaves [0, nbr_offsets[n]]
 *                         or has more than LSKUM_MAX_DEGREE entries, and a
 *                         neighbour index outside [0, n), are skipped by the
 *                         kernels and reported as LSKUM_ERR_CONNECTIVITY
 *   U                     float64[4*n] conserved state (component-major)
 *   qx, qy                float64[4*n], written
 *   cuda_stream           cudaStream_t, or NULL for the legacy default stream
 * Scratch (q and two gradient buffers, 160 bytes per point) lives in one
 * statically sized __device__ array of LSKUM_NOALLOC_MAX_POINTS points
 * (21 MB), which every GPU that loads the library holds until the process
 * exits. The first call on a device looks up that array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture. The address is kept for the life of the
 * process: do not call this on a device after cudaDeviceReset there. All
 * calls share the one array: calls whose work overlaps on the GPU (other
 * threads, other streams) race and must be serialised by the caller. The
 * status words at the head of the array are cleared at the start of every
 * call; the rest is written before it is read. The call synchronises the
 * stream at its end to read its status word. A point whose stencil has a
 * singular 2x2 least-squares matrix gets non-finite derivatives.
 * Errors: LSKUM_ERR_ARG (n out of range, NULL pointer, inner_iters outside
 * [0, 1000]), LSKUM_ERR_CONNECTIVITY, LSKUM_ERR_NONPHYSICAL (a point with
 * rho <= 0 or p <= 0), LSKUM_ERR_CUDA; message via lskum_last_error(NULL).
 */
#define LSKUM_NOALLOC_MAX_POINTS 131072
lskum_status lskum_q_derivatives_noalloc(int64_t n, const double *x, const double *y,
                                         const int32_t *nbr_offsets, const int32_t *nbr_idx,
                                         const double *U, double gamma, int inner_iters,
                                         double *qx, double *qy, void *cuda_stream);

/* Kernel classes for lskum_kernel_time */
/*
 * Launch-shape autotuner (mixed-precision contexts; not in the paper). The
 * mixed flux kernel and the mixed q-derivative pass are each compiled in
 * several shapes (threads per block, minimum resident blocks per SM, which
 * caps registers). lskum_autotune times every shape on this context's own
 * cloud and state (reps launches each after one warm-up, CUDA events on the
 * context's stream; the flux in residual mode, the q-derivatives as one inner
 * pass), keeps the fastest of each and reports them. The state is not
 * changed. A shape changes only the register budget the compiler works
 * with, and through it which FP32 multiply-adds are contracted: results of
 * different shapes agree to FP32 rounding, not bitwise. Synchronises.
 * LSKUM_ERR_ARG on an FP64 context.
 */
typedef struct {
    /* flux variants 6 and up use a software-pipelined neighbour loop (the next
     * slot's data is loaded while the current slot is evaluated) */
    int flux_variant, flux_threads, flux_min_blocks;
    int qgrad_variant, qgrad_threads, qgrad_min_blocks;
    double flux_ms, qgrad_ms;                  /* per launch, chosen shape */
    double flux_ms_default, qgrad_ms_default;  /* per launch, shape 0 */
} lskum_tuning;

lskum_status lskum_autotune(lskum_ctx *ctx, int reps, lskum_tuning *out);

/* Select shapes directly (0 is the default of each kernel). */
lskum_status lskum_set_tuning(lskum_ctx *ctx, int flux_variant, int qgrad_variant);

/*
 * Mixed contexts: *count receives the number of points whose least-squares
 * closures run in FP64 because FP32 would lose bits there (a sub-stencil
 * with sum |w_i||P_i - P_0| > 16; not in the paper, a property of the mixed
 * form). 0 for an FP64 context. Does not synchronise. LSKUM_ERR_ARG on a null
 * argument.
 */
lskum_status lskum_mixed_fp64_points(lskum_ctx *ctx, int64_t *count);

/*
 * Lift and drag of case k (a batch) or of the only case: as lskum_forces,
 * with case k's free stream; cp receives its n_wall values in its contour order.
 */
lskum_status lskum_case_forces(lskum_ctx *ctx, int k, double *cl, double *cd, double *cp);

/*
 * Measured arithmetic peak of the current device, for throughput reports (the
 * paper has no counterpart: these are the denominators of the ALU rooflines of
 * the flux kernels). kind 0: FP64 fused multiply-add; 1: FP32 fused
 * multiply-add; 2: packed FP32x2 fused multiply-add (FFMA2). Runs `reps` timed
 * launches (after one warm-up) of independent multiply-add chains filling
 * every SM on cuda_stream (NULL: the legacy default stream) and writes the
 * best rate in GFLOP/s (2 flops per multiply-add) to *gflops. Allocates and
 * frees a 4 KB device buffer; synchronises. LSKUM_ERR_ARG for a kind outside
 * 0..2, reps outside 1..100 or a NULL gflops.
 */
lskum_status lskum_probe_peak(int kind, int reps, void *cuda_stream, double *gflops);

#define LSKUM_KERNEL_FLUX 0  /* fused flux residual + state update */
#define LSKUM_KERNEL_QGRAD 1 /* one least-squares q-derivative pass */
#define LSKUM_KERNEL_CLASSES 2

/*
 * Per-kernel timing for throughput reports: while enabled, every launch of a
 * timed kernel class is bracketed by CUDA events recorded on the context's
 * stream. lskum_profile(ctx, 1) enables and clears the record, (ctx, 0)
 * disables it. lskum_kernel_time synchronises and returns the summed event
 * time (milliseconds) and launch count of one class since it was enabled.
 */
lskum_status lskum_profile(lskum_ctx *ctx, int enable);
lskum_status lskum_kernel_time(lskum_ctx *ctx, int kernel_class, double *total_ms, int64_t *launches);

#ifdef __cplusplus
}
#endif

#endif /* LSKUM_H */
